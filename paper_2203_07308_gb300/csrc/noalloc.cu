// pnp_full_grad_noalloc: the full gradient A^T(Ax - b) for callers that cannot
// allocate device memory.  Some host programs may not call cudaMalloc once they
// are running: a scanner's real-time reconstruction service that fixes its
// memory at start-up so that no request can fail or stall on allocation, or a
// plug-in inside an application whose own allocator owns every byte of the
// GPU.  Such a caller can still pass its input and output buffers, but not a
// workspace.  This entry point therefore keeps its scratch (ray tables,
// coefficient image, residual sinogram) in a fixed array compiled into the
// library, so it allocates nothing at all.
//
// The array lives in every GPU that loads the library until the process exits
// (PNP_NOALLOC_SCRATCH_BYTES).  All calls share it and it keeps the last call's
// contents; every call rewrites all of the scratch it reads, so nothing has to
// start at zero.  Calls that overlap on the GPU (other streams, other host
// threads, concurrent graphs) race on the array and give wrong results: issue
// them one after another on one device.  It is the unweighted gradient (no
// pnp_set_weights weights: those belong to a workspace).  The device address of
// the array is looked up on a device's first call and kept for the life of the
// process; it does not survive cudaDeviceReset of that device.
#include <cuda_runtime.h>

#include <mutex>

#include "pnp_internal.cuh"

namespace pnp {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[PNP_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {};

inline size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// Device address of the scratch array on the current device.  The array's name
// in host code is only a stand-in symbol, never a device pointer, so the address
// is looked up once per device (with that device current) and cached.
int scratch_address(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(PNP_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(PNP_EUNSUPPORTED, "device ordinal %d >= %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return fail(PNP_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return PNP_OK;
}

}  // namespace
}  // namespace pnp

using namespace pnp;

// Scratch bytes the entry point needs for geometry g (g already validated).
static size_t noalloc_bytes(const pnp_geom* g)
{
    const size_t nr = (size_t)g->n_views * g->n_det;
    const size_t qw = (size_t)g->n + 2 * kPad - 1;
    size_t off = 0;
    off = up256(off + nr * sizeof(float4));                                 // rayf
    off = up256(off + nr * sizeof(float2));                                 // rayi
    off = up256(off + nr * sizeof(int2));                                   // rayk
    off = up256(off + (size_t)g->n_views * sizeof(float4));                 // view
    off = up256(off + (size_t)g->batch * qw * qw * sizeof(float4));         // quad
    off = up256(off + (size_t)g->batch * nr * sizeof(float));               // residual
    return off;
}

extern "C" int pnp_full_grad_noalloc(const pnp_geom* g, const float* d_x, const float* d_b, float* d_g,
                                     void* stream)
{
    clear_error();
    if (int e = validate_geom(g)) return e;
    if (!d_x || !d_b || !d_g) return fail(PNP_EINVAL, "x, b and g are required");
    if (d_x == d_g) return fail(PNP_EINVAL, "x and g must not alias");
    const size_t need = noalloc_bytes(g);
    if (need > (size_t)PNP_NOALLOC_SCRATCH_BYTES)
        return fail(PNP_EINVAL,
                    "pnp_full_grad_noalloc: this geometry needs %zu bytes of scratch, more than the "
                    "library's fixed %zu; use pnp_full_grad with a caller-allocated workspace",
                    need, (size_t)PNP_NOALLOC_SCRATCH_BYTES);
    void* base = nullptr;
    if (int e = scratch_address(&base)) return e;
    char* ws = (char*)base;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nr = (size_t)g->n_views * g->n_det;
    LevelLayout lv;
    lv.factor = 1;
    lv.ns = g->n;
    lv.qw = g->n + 2 * kPad - 1;
    size_t off = 0;
    lv.off_rayf = off; off = up256(off + nr * sizeof(float4));
    lv.off_rayi = off; off = up256(off + nr * sizeof(float2));
    lv.off_rayk = off; off = up256(off + nr * sizeof(int2));
    lv.off_view = off; off = up256(off + (size_t)g->n_views * sizeof(float4));
    lv.off_quad = off; off = up256(off + (size_t)g->batch * lv.qw * lv.qw * sizeof(float4));
    float* res = (float*)(ws + off);
    cudaError_t e = launch_setup_rays(*g, lv, ws, st);
    if (e == cudaSuccess)
        e = launch_prep_quad(d_x, g->n, 1, g->batch, (float4*)(ws + lv.off_quad), lv.qw, st);
    if (e == cudaSuccess) {
        FwdArgs a{};
        a.quad = (const float4*)(ws + lv.off_quad);
        a.qw = lv.qw;
        a.quad_stride = (size_t)lv.qw * lv.qw;
        a.rayf = (const float4*)(ws + lv.off_rayf);
        a.rayk = (const int2*)(ws + lv.off_rayk);
        a.n_det = g->n_det;
        a.first_view = 0;
        a.view_step = 1;
        a.n_sub = g->n_views;
        a.batch = g->batch;
        a.step = (float)g->step;
        a.weight = (float)g->step;
        a.b = d_b;
        a.n_views = g->n_views;
        a.out = res;
        e = launch_forward(a, st);
    }
    if (e == cudaSuccess) {
        BackArgs a{};
        a.res = res;
        a.rayf = (const float4*)(ws + lv.off_rayf);
        a.rayi = (const float2*)(ws + lv.off_rayi);
        a.view = (const float4*)(ws + lv.off_view);
        a.rayk = (const int2*)(ws + lv.off_rayk);
        a.ns = g->n;
        a.n_det = g->n_det;
        a.first_view = 0;
        a.view_step = 1;
        a.n_sub = g->n_views;
        a.batch = g->batch;
        a.step = (float)g->step;
        a.mode = kBackGradFine;
        a.s = 1;
        a.n = g->n;
        a.scale = (float)g->step;
        a.out = d_g;
        e = launch_backward(a, st);
    }
    if (e != cudaSuccess) return fail(PNP_ECUDA, "pnp_full_grad_noalloc: %s", cudaGetErrorString(e));
    return PNP_OK;
}
