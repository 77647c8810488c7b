// Deterministic FP64 reductions: power-iteration inner products and norms
// (step size eta = 1/L, Sec. 3), final residual, objective and PSNR.
// Every sum runs in a fixed order (per-thread strided loop, fixed block tree,
// fixed final pass), so results are bitwise repeatable.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdlib>

#include "pnp_internal.cuh"

namespace pnp {

bool pdl_enabled()
{
    static const bool on = [] {
        const char* e = std::getenv("PNP_PDL");
        return !(e && e[0] == '0');
    }();
    return on;
}

bool fuse_quad_enabled()
{
    static const bool on = [] {
        const char* e = std::getenv("PNP_FUSE_QUAD");
        return !(e && e[0] == '0');
    }();
    return on;
}

namespace {

__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double sh[32];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        r = lane < nw ? sh[lane] : 0.0;
        for (int off = 16; off > 0; off >>= 1) r += __shfl_xor_sync(0xffffffffu, r, off);
    }
    return r;  // valid in thread 0
}

// mode: dot a.b | (a-b)^2 | a^2 | isotropic TV of image a (n x n)
__global__ void k_reduce_partial(int mode, const float* __restrict__ a, const float* __restrict__ b,
                                 size_t count, size_t stride, int n, double* __restrict__ partials)
{
    const int inst = blockIdx.y;
    const float* A = a + (size_t)inst * stride;
    const float* B = b ? b + (size_t)inst * stride : nullptr;
    double acc = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (size_t)gridDim.x * blockDim.x) {
        double x = (double)__ldg(A + i);
        switch (mode) {
            case kRedDot: acc += x * (double)__ldg(B + i); break;
            case kRedDiffSq: { double d = x - (double)__ldg(B + i); acc += d * d; } break;
            case kRedSq: acc += x * x; break;
            case kRedWSq: acc += (double)__ldg(B + i) * x * x; break;
            default: {
                const size_t r = i / n, c = i % n;
                double gy = r + 1 < (size_t)n ? (double)__ldg(A + i + n) - x : 0.0;
                double gx = c + 1 < (size_t)n ? (double)__ldg(A + i + 1) - x : 0.0;
                acc += sqrt(gy * gy + gx * gx);
            } break;
        }
    }
    double s = block_sum(acc);
    if (threadIdx.x == 0) partials[(size_t)inst * gridDim.x + blockIdx.x] = s;
}

__global__ void k_reduce_final(const double* __restrict__ partials, int nparts, double* out,
                               int out_stride, int out_off)
{
    const int inst = blockIdx.x;
    double acc = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += partials[(size_t)inst * nparts + i];
    double s = block_sum(acc);
    if (threadIdx.x == 0) out[(size_t)inst * out_stride + out_off] = s;
}

__global__ void k_scale_by_rnorm(const float* __restrict__ w, float* __restrict__ u, size_t count,
                                 const double* __restrict__ norm2)
{
    const double f = 1.0 / sqrt(norm2[0]);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (size_t)gridDim.x * blockDim.x)
        u[i] = (float)((double)w[i] * f);
}

__global__ void k_fill(float* __restrict__ x, size_t count, float v)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (size_t)gridDim.x * blockDim.x)
        x[i] = v;
}

// x[i] = lo + (hi - lo) u_i, u_i in [0, 1) from an integer hash of i (the
// "lowbias32" mixer: xor-shift / multiply rounds): a fixed noisy test image
__global__ void k_fill_hash(float* __restrict__ x, size_t count, float lo, float hi)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (size_t)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)i * 0x9E3779B9u;
        h ^= h >> 16;
        h *= 0x7FEB352Du;
        h ^= h >> 15;
        h *= 0x846CA68Bu;
        h ^= h >> 16;
        x[i] = fmaf((float)(h >> 8) * (1.0f / 16777216.0f), hi - lo, lo);
    }
}

__global__ void k_copy(const float* __restrict__ s, float* __restrict__ d, size_t count)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (size_t)gridDim.x * blockDim.x)
        d[i] = s[i];
}

inline cudaError_t counted(cudaError_t e = cudaGetLastError())
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return e;
}

inline int grid_for(size_t count)
{
    const size_t cap = (size_t)8 * device_sm_count();   // 8 blocks of 256 threads per SM
    size_t g = (count + 255) / 256;
    return (int)(g < cap ? (g < 1 ? 1 : g) : cap);
}

}  // namespace

cudaError_t launch_reduce_partial(int mode, const float* a, const float* b, size_t count,
                                  size_t stride, int batch, int n, double* partials, cudaStream_t st)
{
    dim3 grd(kRedBlocks, batch);
    k_reduce_partial<<<grd, kRedThreads, 0, st>>>(mode, a, b, count, stride, n, partials);
    return counted();
}

cudaError_t launch_reduce_final(const double* partials, int nparts, int batch, double* out,
                                int out_stride, int out_off, cudaStream_t st)
{
    k_reduce_final<<<batch, 256, 0, st>>>(partials, nparts, out, out_stride, out_off);
    return counted();
}

cudaError_t launch_scale_by_rnorm(const float* w, float* u, size_t count, const double* norm2,
                                  cudaStream_t st)
{
    k_scale_by_rnorm<<<grid_for(count), 256, 0, st>>>(w, u, count, norm2);
    return counted();
}

cudaError_t launch_fill(float* x, size_t count, float v, cudaStream_t st)
{
    k_fill<<<grid_for(count), 256, 0, st>>>(x, count, v);
    return counted();
}

cudaError_t launch_fill_hash(float* x, size_t count, float lo, float hi, cudaStream_t st)
{
    k_fill_hash<<<grid_for(count), 256, 0, st>>>(x, count, lo, hi);
    return counted();
}

cudaError_t launch_copy(const float* src, float* dst, size_t count, cudaStream_t st)
{
    k_copy<<<grid_for(count), 256, 0, st>>>(src, dst, count);
    return counted();
}

}  // namespace pnp
