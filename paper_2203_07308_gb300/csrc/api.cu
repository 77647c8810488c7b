// C ABI of libpnp_ms2g.so (declared in include/pnp_ms2g.h): argument checks,
// workspace layout, the (workspace, geometry) registry, and the host side of
// the gradient estimators, the TV denoiser, the power iteration and the
// multi-stage loop of Algorithm 1.  Every step of the numerical path runs in
// the kernels of projector.cu, tv.cu and reduce.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "pnp_internal.cuh"

namespace pnp {

int level_index(int factor)
{
    switch (factor) {
        case 1: return 0;
        case 2: return 1;
        case 4: return 2;
        case 8: return 3;
        default: return -1;
    }
}

int device_sm_count()
{
    constexpr int kMaxDev = 64;
    static std::atomic<int> cache[kMaxDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 1;
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) return 1;
    cache[dev].store(v, std::memory_order_relaxed);
    return v;
}

thread_local std::string t_err;

void clear_error() { t_err.clear(); }

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return code;
}

#define PNP_CUDA(call)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(PNP_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),      \
                        __FILE__, __LINE__);                                             \
    } while (0)

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

}  // namespace

// A level is available when it divides n, keeps at least 4 pixels per side and
// leaves the source far enough outside the image for the backprojector's
// shadow bound (distance >= 4 sqrt(2) level pixels beyond the support).
bool level_ok(const pnp_geom& g, int s)
{
    if (g.n % s != 0 || g.n / s < 4) return false;
    return g.dso >= std::sqrt(2.0) * (0.5 * g.n + 5.5 * s);
}

int validate_geom(const pnp_geom* g)
{
    if (!g) return fail(PNP_EINVAL, "geometry pointer is NULL");
    if (g->n < 4 || g->n > 8192) return fail(PNP_EINVAL, "n=%d outside [4, 8192]", g->n);
    if (g->n_views < 1 || g->n_det < 1 || g->batch < 1)
        return fail(PNP_EINVAL, "n_views, n_det and batch must be >= 1");
    if ((double)g->n_views * g->n_det > (double)(1 << 28))
        return fail(PNP_EINVAL, "n_views * n_det too large");
    if ((double)g->batch * g->n * g->n > 4.0e9 || (double)g->batch * g->n_views * g->n_det > 4.0e9)
        return fail(PNP_EINVAL, "batch too large");
    if (!(std::isfinite(g->dso) && std::isfinite(g->ddo) && std::isfinite(g->det_pitch) &&
          std::isfinite(g->angle0) && std::isfinite(g->angle_span) && std::isfinite(g->step)))
        return fail(PNP_EINVAL, "geometry has a non-finite value");
    if (g->ddo < 0.0 || g->det_pitch <= 0.0 || g->step <= 0.0 || g->step > 4.0)
        return fail(PNP_EINVAL, "need ddo >= 0, det_pitch > 0, 0 < step <= 4");
    if (!level_ok(*g, 1))
        return fail(PNP_EINVAL, "source too close: need dso >= sqrt(2) (n/2 + 5.5) = %g",
                    std::sqrt(2.0) * (0.5 * g->n + 5.5));
    // longest ray inside the image in samples must fit an int comfortably
    if (std::sqrt(2.0) * (g->n + 2) / g->step > 1.0e8) return fail(PNP_EINVAL, "step too small");
    return PNP_OK;
}

namespace {

Layout make_layout(const pnp_geom& g)
{
    Layout L;
    size_t off = 0;
    const size_t nr = (size_t)g.n_views * g.n_det;
    const int factors[kMaxLevels] = {1, 2, 4, 8};
    for (int l = 0; l < kMaxLevels; ++l) {
        const int s = factors[l];
        if (!level_ok(g, s)) continue;
        LevelLayout& v = L.lv[l];
        v.factor = s;
        v.ns = g.n / s;
        v.qw = v.ns + 2 * kPad - 1;
        v.off_rayf = off; off = align_up(off + nr * sizeof(float4));
        v.off_rayi = off; off = align_up(off + nr * sizeof(float2));
        v.off_rayk = off; off = align_up(off + nr * sizeof(int2));
        v.off_view = off; off = align_up(off + (size_t)g.n_views * sizeof(float4));
        v.off_quad = off; off = align_up(off + (size_t)g.batch * v.qw * v.qw * sizeof(float4));
    }
    const size_t img = (size_t)g.batch * g.n * g.n;
    L.off_res = off; off = align_up(off + (size_t)g.batch * nr * sizeof(float));
    L.off_y = off; off = align_up(off + img * sizeof(float));
    L.off_z = off; off = align_up(off + img * sizeof(float));
    L.off_x2 = off; off = align_up(off + 2 * img * sizeof(float));
    L.off_tv = off; off = align_up(off + 8 * img * sizeof(float));
    L.off_pw = off; off = align_up(off + 2 * (size_t)g.n * g.n * sizeof(float));
    L.off_cs = off; off = align_up(off + 2 * (size_t)g.batch * (g.n / 2) * (g.n / 2) * sizeof(float));
    // partials of the largest part count any denoiser shape may use (smallest tile 8, warp tiles)
    const size_t tv_parts = std::max((size_t)tile_tv_parts_for(g.n, g.batch, 8),
                                     (size_t)tile_tv_parts_for(g.n, g.batch, kTvTileWarp));
    const size_t parts = tv_parts > (size_t)kRedBlocks ? tv_parts : (size_t)kRedBlocks;
    L.off_red = off; off = align_up(off + ((size_t)g.batch * parts + (size_t)g.batch * 8) * sizeof(double));
    L.off_log = off; off = align_up(off + (size_t)PNP_MAX_LOG_ITERS * sizeof(double));
    L.total = off;
    return L;
}

inline size_t red_parts(const pnp_geom& g)
{
    const size_t tv_parts = std::max((size_t)tile_tv_parts_for(g.n, g.batch, 8),
                                     (size_t)tile_tv_parts_for(g.n, g.batch, kTvTileWarp));
    return tv_parts > (size_t)kRedBlocks ? tv_parts : (size_t)kRedBlocks;
}

uint64_t fingerprint(const pnp_geom& g)
{
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](const void* p, size_t n) {
        const unsigned char* c = (const unsigned char*)p;
        for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
    };
    mix(&g.n, sizeof g.n); mix(&g.n_views, sizeof g.n_views); mix(&g.n_det, sizeof g.n_det);
    mix(&g.batch, sizeof g.batch); mix(&g.dso, sizeof g.dso); mix(&g.ddo, sizeof g.ddo);
    mix(&g.det_pitch, sizeof g.det_pitch); mix(&g.angle0, sizeof g.angle0);
    mix(&g.angle_span, sizeof g.angle_span); mix(&g.step, sizeof g.step);
    return h;
}

// Launch shapes chosen by pnp_autotune for one prepared workspace (0 = heuristic).
struct Tuned {
    int lanes[kMaxLevels] = {0, 0, 0, 0};    // forward: lanes per ray
    int groups[kMaxLevels] = {0, 0, 0, 0};   // backprojector: view groups per CTA
    int tile = 0;                            // tiled FGP: tile side
};

// Step-size constants L = ||W^{1/2} A_s S||^2 found by pnp_step_sizes (or a
// pnp_run without step sizes), per level and sketch kind; cleared by pnp_setup and
// pnp_set_weights.
struct LCache {
    double L[kMaxLevels][2] = {};
    bool valid[kMaxLevels][2] = {};
};

// Stored gather table registered with pnp_set_gather_table: per level, byte offsets
// of the header, weights and bins in the caller's buffer.
struct GatherTab {
    char* base = nullptr;
    size_t bytes = 0;
    size_t off_hdr[kMaxLevels] = {}, off_w[kMaxLevels] = {}, off_ray[kMaxLevels] = {};
    bool present[kMaxLevels] = {};
};

struct RegEntry {
    const void* ws; uint64_t fp; size_t bytes; Tuned tuned; const float* weights;
    void* vr = nullptr; size_t vr_bytes = 0;     // estimator-state buffer (SVRG / SAGA)
    LCache lc;
    GatherTab tab;
};
std::mutex g_reg_mu;
std::vector<RegEntry> g_reg;

void reg_put(const void* ws, uint64_t fp, size_t bytes)
{
    std::lock_guard<std::mutex> lk(g_reg_mu);
    for (auto& e : g_reg)
        if (e.ws == ws) {
            e.fp = fp; e.bytes = bytes; e.tuned = Tuned(); e.weights = nullptr; e.vr = nullptr; e.vr_bytes = 0;
            e.lc = LCache();
            e.tab = GatherTab();
            return;
        }
    if (g_reg.size() >= 4096) g_reg.erase(g_reg.begin());
    RegEntry e{ws, fp, bytes, Tuned(), nullptr};
    g_reg.push_back(e);
}

void reg_vr(const void* ws, void** buf, size_t* bytes)
{
    std::lock_guard<std::mutex> lk(g_reg_mu);
    *buf = nullptr;
    *bytes = 0;
    for (const auto& e : g_reg)
        if (e.ws == ws) { *buf = e.vr; *bytes = e.vr_bytes; }
}

void reg_set_vr(const void* ws, void* buf, size_t bytes)
{
    std::lock_guard<std::mutex> lk(g_reg_mu);
    for (auto& e : g_reg)
        if (e.ws == ws) { e.vr = buf; e.vr_bytes = buf ? bytes : 0; }
}

// Estimator-state buffer: fine snapshot and difference image, then level-grid
// running sum (SVRG mu / SAGA Phi), combined estimate, raw subset gradient, and
// the SAGA table of P_k level-grid images, each [batch][.][.].
struct VrLayout { size_t off_yt = 0, off_diff = 0, off_acc = 0, off_v = 0, off_G = 0, off_tab = 0, bytes = 0; };

VrLayout vr_layout(const pnp_geom& g, const pnp_stage* st, int n_stages)
{
    VrLayout V;
    bool any = false;
    size_t tab = 0;
    for (int k = 0; k < n_stages; ++k) {
        if (st[k].n_subsets <= 1 || st[k].estimator == PNP_EST_MINIBATCH) continue;
        any = true;
        if (st[k].estimator == PNP_EST_SAGA && st[k].factor > 0) {
            const size_t ns = (size_t)(g.n / st[k].factor);
            tab = std::max(tab, (size_t)st[k].n_subsets * g.batch * ns * ns);
        }
    }
    if (!any) return V;
    const size_t img = (size_t)g.batch * g.n * g.n * sizeof(float);
    size_t off = 0;
    V.off_yt = off; off = align_up(off + img);
    V.off_diff = off; off = align_up(off + img);
    V.off_acc = off; off = align_up(off + img);
    V.off_v = off; off = align_up(off + img);
    V.off_G = off; off = align_up(off + img);
    V.off_tab = off; off = align_up(off + tab * sizeof(float));
    V.bytes = off;
    return V;
}

Tuned reg_tuned(const void* ws)
{
    std::lock_guard<std::mutex> lk(g_reg_mu);
    for (const auto& e : g_reg)
        if (e.ws == ws) return e.tuned;
    return Tuned();
}

const float* reg_weights(const void* ws)
{
    std::lock_guard<std::mutex> lk(g_reg_mu);
    for (const auto& e : g_reg)
        if (e.ws == ws) return e.weights;
    return nullptr;
}

void reg_set_weights(const void* ws, const float* w)
{
    std::lock_guard<std::mutex> lk(g_reg_mu);
    for (auto& e : g_reg)
        if (e.ws == ws) {
            e.weights = w;
            e.lc = LCache();     // L depends on the weights
        }
}

bool reg_get_L(const void* ws, int li, int kind, double* L)
{
    std::lock_guard<std::mutex> lk(g_reg_mu);
    for (const auto& e : g_reg)
        if (e.ws == ws && e.lc.valid[li][kind]) {
            *L = e.lc.L[li][kind];
            return true;
        }
    return false;
}

void reg_put_L(const void* ws, int li, int kind, double L)
{
    std::lock_guard<std::mutex> lk(g_reg_mu);
    for (auto& e : g_reg)
        if (e.ws == ws) {
            e.lc.L[li][kind] = L;
            e.lc.valid[li][kind] = true;
        }
}

GatherTab reg_table(const void* ws)
{
    std::lock_guard<std::mutex> lk(g_reg_mu);
    for (const auto& e : g_reg)
        if (e.ws == ws) return e.tab;
    return GatherTab();
}

void reg_set_table(const void* ws, const GatherTab& t)
{
    std::lock_guard<std::mutex> lk(g_reg_mu);
    for (auto& e : g_reg)
        if (e.ws == ws) e.tab = t;
}

void reg_set_tuned(const void* ws, const Tuned& t)
{
    std::lock_guard<std::mutex> lk(g_reg_mu);
    for (auto& e : g_reg)
        if (e.ws == ws) e.tuned = t;
}

int check_ws(const pnp_geom& g, const void* ws)
{
    if (!ws) return fail(PNP_EINVAL, "workspace pointer is NULL");
    const uint64_t fp = fingerprint(g);
    std::lock_guard<std::mutex> lk(g_reg_mu);
    for (const auto& e : g_reg)
        if (e.ws == ws) {
            if (e.fp != fp) return fail(PNP_ESTATE, "workspace was set up for another geometry");
            return PNP_OK;
        }
    return fail(PNP_ESTATE, "workspace not prepared: call pnp_setup first");
}

int check_level(const pnp_geom& g, int factor, const Layout& L, int* li)
{
    int l = level_index(factor);
    if (l < 0) return fail(PNP_EINVAL, "factor %d not in {1,2,4,8}", factor);
    if (L.lv[l].factor == 0)
        return fail(PNP_EINVAL, "factor %d unavailable for n=%d, dso=%g (needs n %% s == 0, n/s >= 4, "
                    "dso >= sqrt(2)(n/2 + 5.5 s))", factor, g.n, g.dso);
    *li = l;
    return PNP_OK;
}

int check_subset(const pnp_geom& g, int p, int P)
{
    if (P < 1 || P > g.n_views) return fail(PNP_EINVAL, "n_subsets=%d outside [1, n_views]", P);
    if (p < 0 || p >= P) return fail(PNP_EINVAL, "subset=%d outside [0, n_subsets)", p);
    return PNP_OK;
}

inline int subset_views(const pnp_geom& g, int p, int P)
{
    return P <= 1 ? g.n_views : (g.n_views - p + P - 1) / P;
}

inline cudaStream_t S(void* st) { return (cudaStream_t)st; }

// Forward residual r = A_s^{(p)} (level image in quad) - b^{(p)} into the workspace.
// il: the output is a workspace residual that a backprojector of this batch reads
// next (image-interleaved for batches with interleaved coefficient images).
FwdArgs fwd_args(const pnp_geom& g, const LevelLayout& lv, char* ws, int p, int P, const float* b,
                 float* out, int batch, const float* w = nullptr, bool il = false)
{
    FwdArgs a{};
    a.w = w;
    a.out_il = il && quad_interleaved(batch);
    a.quad = (const float4*)(ws + lv.off_quad);
    a.qw = lv.qw;
    a.quad_stride = (size_t)lv.qw * lv.qw;
    a.rayf = (const float4*)(ws + lv.off_rayf);
    a.rayk = (const int2*)(ws + lv.off_rayk);
    a.n_det = g.n_det;
    a.first_view = P <= 1 ? 0 : p;
    a.view_step = P <= 1 ? 1 : P;
    a.n_sub = subset_views(g, p, P);
    a.batch = batch;
    a.step = (float)g.step;
    a.weight = (float)(g.step * lv.factor);
    a.b = b;
    a.n_views = g.n_views;
    a.out = out;
    return a;
}

// Bound on the (ray, sample) terms that one level pixel receives from one view,
// for the fixed-point scatter: the rays whose line passes within sqrt 2 of the
// pixel centre (the hat support is the 2 x 2 square around it; adjacent rays
// are at least delta apart there: their angular spacing, smallest at the
// detector's edge bins, times the distance from the source, at least dso minus
// the image's circumradius and the apron) times the samples of one ray inside
// that square.
float scatter_terms_bound(const pnp_geom& g, int factor)
{
    const double r2 = std::sqrt(2.0);
    double dgam = 0.5 * M_PI;
    if (g.n_det > 1) {
        const double dsd = g.dso + g.ddo;
        const double u1 = 0.5 * (g.n_det - 1) * g.det_pitch, u0 = u1 - g.det_pitch;
        dgam = std::atan(u1 / dsd) - std::atan(u0 / dsd);
    }
    const double dmin = g.dso - (0.5 * g.n + 3.0 * factor) * r2;
    if (!(dmin > 0.0) || !(dgam > 0.0)) return 0.0f;
    const double delta = dmin * std::sin(std::min(dgam, 0.5 * M_PI)) / factor;
    const double rays = std::floor(2.0 * r2 / delta) + 2.0;
    const double samples = std::floor(2.0 * r2 / g.step) + 2.0;
    const double b = rays * samples;
    return b < 1e9 ? (float)b : 0.0f;
}

BackArgs back_args(const pnp_geom& g, const LevelLayout& lv, char* ws, int p, int P, const float* res,
                   int mode, float scale, const float* y, float eta, float* out, int batch, bool il = false)
{
    BackArgs a{};
    a.res_il = il && quad_interleaved(batch);
    a.cmax = scatter_terms_bound(g, lv.factor);
    a.res = res;
    a.rayf = (const float4*)(ws + lv.off_rayf);
    a.rayi = (const float2*)(ws + lv.off_rayi);
    a.view = (const float4*)(ws + lv.off_view);
    a.rayk = (const int2*)(ws + lv.off_rayk);
    a.ns = lv.ns;
    a.n_det = g.n_det;
    a.first_view = P <= 1 ? 0 : p;
    a.view_step = P <= 1 ? 1 : P;
    a.n_sub = subset_views(g, p, P);
    a.batch = batch;
    a.step = (float)g.step;
    a.mode = mode;
    a.s = lv.factor;
    a.n = g.n;
    a.scale = scale;
    a.y = y;
    a.eta = eta;
    a.out = out;
    const int li = level_index(lv.factor);
    const GatherTab tb = reg_table(ws);
    if (li >= 0 && tb.present[li]) {
        a.thdr = (const int2*)(tb.base + tb.off_hdr[li]);
        a.tw = (const float4*)(tb.base + tb.off_w[li]);
        a.tray = (const int*)(tb.base + tb.off_ray[li]);
    }
    return a;
}

// Gradient estimate on the fine grid into `out` (mode GradFine) or the fused
// step z = y - eta * grad (mode Step).  `y` is the fine iterate.
int grad_into(const pnp_geom& g, const Layout& L, int li, char* ws, const float* y, const float* b,
              int p, int P, int mode, float eta, float* out, cudaStream_t st, int kind = PNP_SKETCH_POOL)
{
    const LevelLayout& lv = L.lv[li];
    const Tuned tu = reg_tuned(ws);
    float* res = (float*)(ws + L.off_res);
    if (kind == PNP_SKETCH_BICUBIC && lv.factor > 1) {
        // S y (bicubic) -> A_s -> A_s^T (coarse) -> U = S^T and the step on the fine grid
        float* cimg = (float*)(ws + L.off_cs);
        float* cgrad = cimg + (size_t)g.batch * (g.n / 2) * (g.n / 2);
        PNP_CUDA(launch_bicubic_down(y, cimg, g.n, lv.factor, g.batch, st));
        PNP_CUDA(launch_prep_quad(cimg, lv.ns, 1, g.batch, (float4*)(ws + lv.off_quad), lv.qw, st));
        PNP_CUDA(launch_forward(fwd_args(g, lv, ws, p, P, b, res, g.batch, reg_weights(ws), true), st, tu.lanes[li]));
        const double c = P <= 1 ? 1.0 : (double)P;
        PNP_CUDA(launch_backward(back_args(g, lv, ws, p, P, res, kBackRaw, (float)(g.step * lv.factor * c), nullptr,
                                           0.0f, cgrad, g.batch, true), st, tu.groups[li]));
        PNP_CUDA(launch_bicubic_up(cgrad, mode == kBackStep ? y : nullptr, out, g.n, lv.factor, g.batch, 1.0f, eta,
                                   st));
        return PNP_OK;
    }
    PNP_CUDA(launch_prep_quad(y, g.n, lv.factor, g.batch, (float4*)(ws + lv.off_quad), lv.qw, st));
    PNP_CUDA(launch_forward(fwd_args(g, lv, ws, p, P, b, res, g.batch, reg_weights(ws), true), st, tu.lanes[li]));
    const double c = P <= 1 ? 1.0 : (double)P;
    const float scale = (float)(g.step * lv.factor * c / ((double)lv.factor * lv.factor));
    PNP_CUDA(launch_backward(back_args(g, lv, ws, p, P, res, mode, scale, y, eta, out, g.batch, true), st,
                             tu.groups[li]));
    return PNP_OK;
}

// ------------------------------------------------------------- phase timing
// PNP_RUN_KERNEL_TIMES: one start/stop event pair per phase launch, from a
// process-wide pool; elapsed times are folded into per-phase totals when the
// pool fills up or when pnp_kernel_times asks for them.
struct PhaseTimer {
    std::mutex mu;
    std::vector<cudaEvent_t> ev;
    std::vector<int> phase;       // per pending pair
    size_t used = 0;              // events handed out
    double ms[PNP_N_PHASES] = {};
    int64_t launches[PNP_N_PHASES] = {};
    static constexpr size_t kPool = 1u << 14;

    int fold()   // caller holds mu
    {
        for (size_t k = 0; k < phase.size(); ++k) {
            PNP_CUDA(cudaEventSynchronize(ev[2 * k + 1]));
            float t = 0.0f;
            PNP_CUDA(cudaEventElapsedTime(&t, ev[2 * k], ev[2 * k + 1]));
            ms[phase[k]] += t;
            launches[phase[k]] += 1;
        }
        phase.clear();
        used = 0;
        return PNP_OK;
    }
    int mark(int ph, cudaStream_t st, bool start)
    {
        std::lock_guard<std::mutex> lk(mu);
        if (start) {
            if (used + 2 > kPool)
                if (int e = fold()) return e;
            while (ev.size() < used + 2) {
                cudaEvent_t e;
                PNP_CUDA(cudaEventCreate(&e));
                ev.push_back(e);
            }
            phase.push_back(ph);
            PNP_CUDA(cudaEventRecord(ev[used], st));
            used += 2;
        } else {
            PNP_CUDA(cudaEventRecord(ev[used - 1], st));
        }
        return PNP_OK;
    }
};
PhaseTimer g_timer;

// Raw level-s gradient step*s * A_s^{(p)T} W (A_s^{(p)} S img - b^{(p)}) into
// `out` [batch][ns][ns] (no U, no subset factor); b may be null (no data term).
int coarse_grad(const pnp_geom& g, const Layout& L, int li, char* ws, int kind, const float* img,
                const float* b, int p, int P, float* out, cudaStream_t st)
{
    const LevelLayout& lv = L.lv[li];
    const Tuned tu = reg_tuned(ws);
    float* res = (float*)(ws + L.off_res);
    if (kind == PNP_SKETCH_BICUBIC && lv.factor > 1) {
        float* cimg = (float*)(ws + L.off_cs);
        PNP_CUDA(launch_bicubic_down(img, cimg, g.n, lv.factor, g.batch, st));
        PNP_CUDA(launch_prep_quad(cimg, lv.ns, 1, g.batch, (float4*)(ws + lv.off_quad), lv.qw, st));
    } else {
        PNP_CUDA(launch_prep_quad(img, g.n, lv.factor, g.batch, (float4*)(ws + lv.off_quad), lv.qw, st));
    }
    PNP_CUDA(launch_forward(fwd_args(g, lv, ws, p, P, b, res, g.batch, reg_weights(ws), true), st, tu.lanes[li]));
    PNP_CUDA(launch_backward(back_args(g, lv, ws, p, P, res, kBackRaw, (float)(g.step * lv.factor), nullptr,
                                       0.0f, out, g.batch, true), st, tu.groups[li]));
    return PNP_OK;
}

// One SVRG or SAGA iteration's gradient step z = y - eta U v on subset p of P;
// jj is the iteration's index inside its stage (epoch starts at jj % P == 0).
int vr_step(const pnp_geom& g, const Layout& L, int li, char* ws, char* vb, const VrLayout& V, int est,
            int kind, const float* y, const float* b, int p, int P, int jj, float eta, float* z, cudaStream_t st)
{
    const LevelLayout& lv = L.lv[li];
    const int s = lv.factor, ns = lv.ns;
    const size_t cnt = (size_t)g.batch * ns * ns;
    const size_t img = (size_t)g.batch * g.n * g.n;
    float* yt = (float*)(vb + V.off_yt);
    float* dif = (float*)(vb + V.off_diff);
    float* acc = (float*)(vb + V.off_acc);
    float* v = (float*)(vb + V.off_v);
    float* G = (float*)(vb + V.off_G);
    float* tab = (float*)(vb + V.off_tab);
    const bool bic = kind == PNP_SKETCH_BICUBIC && s > 1;
    if (est == PNP_EST_SVRG) {
        if (jj % P == 0) {      // new epoch: snapshot and its full sketched gradient
            PNP_CUDA(launch_copy(y, yt, img, st));
            if (int e = coarse_grad(g, L, li, ws, kind, yt, b, 0, 1, acc, st)) return e;
        }
        PNP_CUDA(launch_axpby(y, 1.0f, yt, -1.0f, dif, (long)img, st));
        if (int e = coarse_grad(g, L, li, ws, kind, dif, nullptr, p, P, G, st)) return e;
        PNP_CUDA(launch_vr_combine(PNP_EST_SVRG, G, acc, nullptr, (float)P, ns, g.batch, bic ? v : nullptr, y,
                                   bic ? nullptr : z, s, eta, st));
    } else {
        if (jj == 0) {          // table of every subset's gradient at the stage's first iterate
            for (int j = 0; j < P; ++j)
                if (int e = coarse_grad(g, L, li, ws, kind, y, b, j, P, tab + (size_t)j * cnt, st)) return e;
            PNP_CUDA(launch_vr_table_sum(tab, P, (long)cnt, acc, st));
        }
        if (int e = coarse_grad(g, L, li, ws, kind, y, b, p, P, G, st)) return e;
        PNP_CUDA(launch_vr_combine(PNP_EST_SAGA, G, acc, tab + (size_t)p * cnt, (float)P, ns, g.batch,
                                   bic ? v : nullptr, y, bic ? nullptr : z, s, eta, st));
    }
    if (bic) PNP_CUDA(launch_bicubic_up(v, y, z, g.n, s, g.batch, 1.0f, eta, st));
    return PNP_OK;
}

// ---------------------------------------------------------------- CUDA graphs
// pnp_run / pnp_run_many with PNP_RUN_GRAPH capture their launch sequence once
// per distinct call (same pointers, geometry, schedule, step sizes, subset
// sequence and parameters) and replay the instantiated graph afterwards.
struct GraphEntry { uint64_t key; cudaGraphExec_t exec; };
std::mutex g_graph_mu;
std::vector<GraphEntry> g_graphs;
constexpr size_t kMaxGraphs = 16;

struct Hasher {
    uint64_t h = 1469598103934665603ull;
    void add(const void* p, size_t n)
    {
        const unsigned char* c = (const unsigned char*)p;
        for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
    }
    template <class T> void val(const T& v) { add(&v, sizeof v); }
};

cudaGraphExec_t graph_find(uint64_t key)
{
    std::lock_guard<std::mutex> lk(g_graph_mu);
    for (const auto& e : g_graphs)
        if (e.key == key) return e.exec;
    return nullptr;
}

void graph_store(uint64_t key, cudaGraphExec_t exec)
{
    std::lock_guard<std::mutex> lk(g_graph_mu);
    if (g_graphs.size() >= kMaxGraphs) {
        cudaGraphExecDestroy(g_graphs.front().exec);
        g_graphs.erase(g_graphs.begin());
    }
    g_graphs.push_back({key, exec});
}

// Runs `issue` (which enqueues kernels on st) directly, or through a cached
// graph keyed by `key` when use_graph is set and st can be captured.
template <class F>
int run_maybe_graph(bool use_graph, uint64_t key, cudaStream_t st, F&& issue)
{
    if (!use_graph || st == nullptr) return issue();
    if (cudaGraphExec_t ex = graph_find(key)) {
        PNP_CUDA(cudaGraphLaunch(ex, st));
        return PNP_OK;
    }
    PNP_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const int rc = issue();
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(st, &graph);
    if (rc != PNP_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (ec != cudaSuccess) return fail(PNP_ECUDA, "graph capture: %s", cudaGetErrorString(ec));
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&ex, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return fail(PNP_ECUDA, "graph instantiate: %s", cudaGetErrorString(ei));
    graph_store(key, ex);
    PNP_CUDA(cudaGraphLaunch(ex, st));
    return PNP_OK;
}

}  // namespace
}  // namespace pnp

using namespace pnp;

extern "C" {

const char* pnp_last_error(void) { return t_err.c_str(); }

uint64_t pnp_launch_count(void) { return g_launches.load(); }

int pnp_kernel_times(double* h_ms, int64_t* h_launches, int reset)
{
    t_err.clear();
    std::lock_guard<std::mutex> lk(g_timer.mu);
    if (int e = g_timer.fold()) return e;
    for (int k = 0; k < PNP_N_PHASES; ++k) {
        if (h_ms) h_ms[k] = g_timer.ms[k];
        if (h_launches) h_launches[k] = g_timer.launches[k];
        if (reset) {
            g_timer.ms[k] = 0.0;
            g_timer.launches[k] = 0;
        }
    }
    return PNP_OK;
}

// Sizes (tab == nullptr) or builds (tab != nullptr) the stored gather table of
// every level of the layout: per level, slot counts of each (view, block group)
// from the count kernel, a host prefix sum into the header, then the entries.
// The counts go through the workspace's TV state planes, in chunks of views.
static int gather_table(const pnp_geom& g, const Layout& L, char* ws, char* tab, size_t tab_bytes, size_t* need,
                 GatherTab* out, cudaStream_t st)
{
    size_t off = 0;
    int* wd = (int*)(ws + L.off_tv);
    const size_t wd_ints = (size_t)8 * g.batch * g.n * g.n;
    for (int li = 0; li < kMaxLevels; ++li) {
        const LevelLayout& lv = L.lv[li];
        if (lv.factor == 0) continue;
        BackArgs a = back_args(g, lv, ws, 0, 1, nullptr, kBackRaw, 1.0f, nullptr, 0.0f, nullptr, 1);
        const int groups = table_groups(lv.ns);
        const size_t nh = (size_t)g.n_views * groups;
        const int vchunk = (int)std::max<size_t>(1, std::min<size_t>(g.n_views, wd_ints / groups));
        std::vector<int> widths(nh);
        for (int v0 = 0; v0 < g.n_views; v0 += vchunk) {
            const int nv = std::min(vchunk, g.n_views - v0);
            BackArgs av = a;
            av.rayf = a.rayf + (size_t)v0 * g.n_det;
            av.view = a.view + v0;
            PNP_CUDA(launch_table_count(av, nv, wd, st));
            PNP_CUDA(cudaMemcpyAsync(widths.data() + (size_t)v0 * groups, wd, (size_t)nv * groups * sizeof(int),
                                     cudaMemcpyDeviceToHost, st));
            PNP_CUDA(cudaStreamSynchronize(st));
        }
        std::vector<int2> hdr(nh);
        long slots = 0;
        for (size_t i = 0; i < nh; ++i) {
            if (slots > (long)INT32_MAX - widths[i]) return fail(PNP_EINVAL, "gather table exceeds 2^31 slots");
            hdr[i] = make_int2((int)slots, widths[i]);
            slots += widths[i];
        }
        const size_t oh = off;
        off = align_up(off + nh * sizeof(int2));
        const size_t ow = off;
        off = align_up(off + (size_t)slots * 32 * sizeof(float4));
        const size_t orr = off;
        off = align_up(off + (size_t)slots * 32 * sizeof(int));
        if (!tab) continue;
        if (off > tab_bytes) return fail(PNP_EINVAL, "gather table buffer of %zu bytes is too small", tab_bytes);
        PNP_CUDA(cudaMemcpyAsync(tab + oh, hdr.data(), nh * sizeof(int2), cudaMemcpyHostToDevice, st));
        PNP_CUDA(launch_table_fill(a, g.n_views, (const int2*)(tab + oh), (float4*)(tab + ow), (int*)(tab + orr), st));
        PNP_CUDA(cudaStreamSynchronize(st));
        out->off_hdr[li] = oh;
        out->off_w[li] = ow;
        out->off_ray[li] = orr;
        out->present[li] = true;
    }
    *need = off;
    return PNP_OK;
}

int pnp_gather_table_size(const pnp_geom* g, void* d_ws, size_t* bytes, void* stream)
{
    t_err.clear();
    if (int e = validate_geom(g)) return e;
    if (!bytes) return fail(PNP_EINVAL, "bytes pointer is NULL");
    if (int e = check_ws(*g, d_ws)) return e;
    const Layout L = make_layout(*g);
    GatherTab tb;
    return gather_table(*g, L, (char*)d_ws, nullptr, 0, bytes, &tb, S(stream));
}

int pnp_set_gather_table(const pnp_geom* g, void* d_table, size_t bytes, void* d_ws, void* stream)
{
    t_err.clear();
    if (int e = validate_geom(g)) return e;
    if (int e = check_ws(*g, d_ws)) return e;
    if (!d_table) {
        reg_set_table(d_ws, GatherTab());
        return PNP_OK;
    }
    if (reinterpret_cast<uintptr_t>(d_table) % 256) return fail(PNP_EINVAL, "gather table buffer not 256-byte aligned");
    reg_set_table(d_ws, GatherTab());            // the gather stays on the hats while the table is rebuilt
    const Layout L = make_layout(*g);
    GatherTab tb;
    tb.base = (char*)d_table;
    tb.bytes = bytes;
    size_t need = 0;
    if (int e = gather_table(*g, L, (char*)d_ws, (char*)d_table, bytes, &need, &tb, S(stream))) return e;
    reg_set_table(d_ws, tb);
    return PNP_OK;
}

int pnp_workspace_size(const pnp_geom* g, size_t* bytes)
{
    t_err.clear();
    if (int e = validate_geom(g)) return e;
    if (!bytes) return fail(PNP_EINVAL, "bytes pointer is NULL");
    *bytes = make_layout(*g).total;
    return PNP_OK;
}

int pnp_setup(const pnp_geom* g, void* d_ws, size_t ws_bytes, void* stream)
{
    t_err.clear();
    if (int e = validate_geom(g)) return e;
    if (!d_ws) return fail(PNP_EINVAL, "workspace pointer is NULL");
    if ((uintptr_t)d_ws % kAlign) return fail(PNP_EINVAL, "workspace must be 256-byte aligned");
    Layout L = make_layout(*g);
    if (ws_bytes < L.total)
        return fail(PNP_EINVAL, "workspace has %zu bytes, needs %zu", ws_bytes, L.total);
    for (int l = 0; l < kMaxLevels; ++l)
        if (L.lv[l].factor) PNP_CUDA(launch_setup_rays(*g, L.lv[l], (char*)d_ws, S(stream)));
    reg_put(d_ws, fingerprint(*g), ws_bytes);
    return PNP_OK;
}

int pnp_project(const pnp_geom* g, int factor, const float* d_img, const float* d_b, float* d_sino,
                int subset, int n_subsets, void* d_ws, void* stream)
{
    t_err.clear();
    if (int e = validate_geom(g)) return e;
    Layout L = make_layout(*g);
    int li = 0;
    if (int e = check_level(*g, factor, L, &li)) return e;
    if (int e = check_subset(*g, subset, n_subsets)) return e;
    if (!d_img || !d_sino) return fail(PNP_EINVAL, "image or sinogram pointer is NULL");
    if (int e = check_ws(*g, d_ws)) return e;
    char* ws = (char*)d_ws;
    const LevelLayout& lv = L.lv[li];
    PNP_CUDA(launch_prep_quad(d_img, lv.ns, 1, g->batch, (float4*)(ws + lv.off_quad), lv.qw, S(stream)));
    PNP_CUDA(launch_forward(fwd_args(*g, lv, ws, subset, n_subsets, d_b, d_sino, g->batch), S(stream),
                            reg_tuned(d_ws).lanes[li]));
    return PNP_OK;
}

int pnp_backproject(const pnp_geom* g, int factor, const float* d_sino, float* d_img, int subset,
                    int n_subsets, void* d_ws, void* stream)
{
    t_err.clear();
    if (int e = validate_geom(g)) return e;
    Layout L = make_layout(*g);
    int li = 0;
    if (int e = check_level(*g, factor, L, &li)) return e;
    if (int e = check_subset(*g, subset, n_subsets)) return e;
    if (!d_img || !d_sino) return fail(PNP_EINVAL, "image or sinogram pointer is NULL");
    if (int e = check_ws(*g, d_ws)) return e;
    const LevelLayout& lv = L.lv[li];
    PNP_CUDA(launch_backward(back_args(*g, lv, (char*)d_ws, subset, n_subsets, d_sino, kBackRaw,
                                       (float)(g->step * factor), nullptr, 0.0f, d_img, g->batch),
                             S(stream), reg_tuned(d_ws).groups[li]));
    return PNP_OK;
}

int pnp_sketch_kind(const pnp_geom* g, int factor, int kind, const float* d_fine, float* d_coarse, void* stream)
{
    t_err.clear();
    if (int e = validate_geom(g)) return e;
    Layout L = make_layout(*g);
    int li = 0;
    if (int e = check_level(*g, factor, L, &li)) return e;
    if (kind != PNP_SKETCH_POOL && kind != PNP_SKETCH_BICUBIC) return fail(PNP_EINVAL, "unknown sketch kind %d", kind);
    if (!d_fine || !d_coarse) return fail(PNP_EINVAL, "image pointer is NULL");
    if (kind == PNP_SKETCH_BICUBIC)
        PNP_CUDA(launch_bicubic_down(d_fine, d_coarse, g->n, factor, g->batch, S(stream)));
    else
        PNP_CUDA(launch_pool(d_fine, d_coarse, g->n, factor, g->batch, S(stream)));
    return PNP_OK;
}

int pnp_sketch(const pnp_geom* g, int factor, const float* d_fine, float* d_coarse, void* stream)
{
    return pnp_sketch_kind(g, factor, PNP_SKETCH_POOL, d_fine, d_coarse, stream);
}

int pnp_upsample_kind(const pnp_geom* g, int factor, int kind, const float* d_coarse, float* d_fine,
                      void* stream)
{
    t_err.clear();
    if (int e = validate_geom(g)) return e;
    Layout L = make_layout(*g);
    int li = 0;
    if (int e = check_level(*g, factor, L, &li)) return e;
    if (kind != PNP_SKETCH_POOL && kind != PNP_SKETCH_BICUBIC) return fail(PNP_EINVAL, "unknown sketch kind %d", kind);
    if (!d_fine || !d_coarse) return fail(PNP_EINVAL, "image pointer is NULL");
    if (kind == PNP_SKETCH_BICUBIC)
        PNP_CUDA(launch_bicubic_up(d_coarse, nullptr, d_fine, g->n, factor, g->batch, 1.0f, 0.0f, S(stream)));
    else
        PNP_CUDA(launch_unpool(d_coarse, d_fine, g->n, factor, g->batch, S(stream)));
    return PNP_OK;
}

int pnp_upsample(const pnp_geom* g, int factor, const float* d_coarse, float* d_fine, void* stream)
{
    return pnp_upsample_kind(g, factor, PNP_SKETCH_POOL, d_coarse, d_fine, stream);
}

int pnp_sketch_grad(const pnp_geom* g, int factor, const float* d_y, const float* d_b, float* d_g,
                    int subset, int n_subsets, void* d_ws, void* stream)
{
    return pnp_sketch_grad_kind(g, factor, PNP_SKETCH_POOL, d_y, d_b, d_g, subset, n_subsets, d_ws, stream);
}

int pnp_sketch_grad_kind(const pnp_geom* g, int factor, int kind, const float* d_y, const float* d_b, float* d_g,
                         int subset, int n_subsets, void* d_ws, void* stream)
{
    t_err.clear();
    if (kind != PNP_SKETCH_POOL && kind != PNP_SKETCH_BICUBIC) return fail(PNP_EINVAL, "unknown sketch kind %d", kind);
    if (int e = validate_geom(g)) return e;
    Layout L = make_layout(*g);
    int li = 0;
    if (int e = check_level(*g, factor, L, &li)) return e;
    if (int e = check_subset(*g, subset, n_subsets)) return e;
    if (!d_y || !d_b || !d_g) return fail(PNP_EINVAL, "y, b or g pointer is NULL");
    if (d_y == d_g) return fail(PNP_EINVAL, "y and g must not alias");
    if (int e = check_ws(*g, d_ws)) return e;
    return grad_into(*g, L, li, (char*)d_ws, d_y, d_b, subset, n_subsets, kBackGradFine, 0.0f, d_g,
                     S(stream), kind);
}

int pnp_full_grad(const pnp_geom* g, const float* d_x, const float* d_b, float* d_g, void* d_ws,
                  void* stream)
{
    return pnp_sketch_grad(g, 1, d_x, d_b, d_g, 0, 1, d_ws, stream);
}

int pnp_tv_workspace_size(int n, int batch, size_t* bytes)
{
    t_err.clear();
    if (n < 2 || batch < 1 || (double)n * n * batch > 4.0e9) return fail(PNP_EINVAL, "bad n or batch");
    if (!bytes) return fail(PNP_EINVAL, "bytes pointer is NULL");
    *bytes = 8 * (size_t)batch * n * n * sizeof(float);
    return PNP_OK;
}

int pnp_tv_denoise(const float* d_z, float* d_x, int n, int batch, float lambda, int iters,
                   void* d_ws, size_t ws_bytes, void* stream)
{
    t_err.clear();
    size_t need = 0;
    if (int e = pnp_tv_workspace_size(n, batch, &need)) return e;
    if (!d_z || !d_x) return fail(PNP_EINVAL, "z or x pointer is NULL");
    if (d_z == d_x) return fail(PNP_EINVAL, "z and x must not alias");
    if (iters < 0 || iters > 100000) return fail(PNP_EINVAL, "iters outside [0, 100000]");
    if (!(lambda >= 0.0f) || !std::isfinite(lambda)) return fail(PNP_EINVAL, "lambda must be >= 0");
    if (iters > 0 && lambda > 0.0f) {
        // one launch covers up to 8 iterations; more are chained through the workspace
        const bool chained = iters > 8;
        if (chained && (!d_ws || ws_bytes < need))
            return fail(PNP_EINVAL, "TV workspace of %zu bytes needed for %d iterations", need, iters);
        const size_t img = (size_t)batch * n * n;
        float* sa = chained ? (float*)d_ws : nullptr;
        float* sb = chained ? (float*)d_ws + 4 * img : nullptr;
        PNP_CUDA(launch_tv_tiled(d_z, n, batch, lambda, iters, 1.0f, 0.0f, d_x, nullptr, nullptr,
                                 nullptr, sa, sb, S(stream)));
    } else {
        PNP_CUDA(launch_copy(d_z, d_x, (size_t)batch * n * n, S(stream)));
    }
    return PNP_OK;
}

int pnp_power_iter(const pnp_geom* g, int factor, int max_iters, double tol, double* h_L, int* h_iters,
                   void* d_ws, void* stream)
{
    return pnp_power_iter_kind(g, factor, PNP_SKETCH_POOL, max_iters, tol, h_L, h_iters, d_ws, stream);
}

}  // extern "C"

namespace pnp {
namespace {

// L = ||W^{1/2} A_s S||^2 of level li by power iteration on S^T A_s^T W A_s S from
// the normalised all-ones image (FP32 operators, FP64 inner products and norm);
// synchronous.  Arguments already checked.
int power_iter_impl(const pnp_geom& gg, const Layout& L, int li, int kind, int max_iters, double tol, double* h_L,
                    int* h_iters, char* ws, cudaStream_t st)
{
    const pnp_geom* g = &gg;
    pnp_geom g1 = *g;
    g1.batch = 1;
    const LevelLayout& lv = L.lv[li];
    const size_t N = (size_t)g->n * g->n;
    float* u = (float*)(ws + L.off_pw);
    float* w = u + N;
    double* part = (double*)(ws + L.off_red);
    double* outv = part + (size_t)g->batch * red_parts(*g);
    float* res = (float*)(ws + L.off_res);
    PNP_CUDA(launch_fill(u, N, (float)(1.0 / std::sqrt((double)N)), st));
    const float scale = (float)(g->step * lv.factor / ((double)lv.factor * lv.factor));
    double lam = 0.0;
    int it = 0;
    for (it = 1; it <= max_iters; ++it) {
        if (kind == PNP_SKETCH_BICUBIC && lv.factor > 1) {
            float* cimg = (float*)(ws + L.off_cs);
            float* cgrad = cimg + (size_t)g->batch * (g->n / 2) * (g->n / 2);
            PNP_CUDA(launch_bicubic_down(u, cimg, g->n, lv.factor, 1, st));
            PNP_CUDA(launch_prep_quad(cimg, lv.ns, 1, 1, (float4*)(ws + lv.off_quad), lv.qw, st));
            PNP_CUDA(launch_forward(fwd_args(g1, lv, ws, 0, 1, nullptr, res, 1, reg_weights(ws)), st));
            PNP_CUDA(launch_backward(back_args(g1, lv, ws, 0, 1, res, kBackRaw, (float)(g->step * lv.factor), nullptr,
                                               0.0f, cgrad, 1), st));
            PNP_CUDA(launch_bicubic_up(cgrad, nullptr, w, g->n, lv.factor, 1, 1.0f, 0.0f, st));
        } else {
            PNP_CUDA(launch_prep_quad(u, g->n, lv.factor, 1, (float4*)(ws + lv.off_quad), lv.qw, st));
            PNP_CUDA(launch_forward(fwd_args(g1, lv, ws, 0, 1, nullptr, res, 1, reg_weights(ws)), st));
            PNP_CUDA(launch_backward(back_args(g1, lv, ws, 0, 1, res, kBackGradFine, scale, nullptr, 0.0f, w, 1), st));
        }
        PNP_CUDA(launch_reduce_partial(kRedDot, u, w, N, N, 1, g->n, part, st));
        PNP_CUDA(launch_reduce_final(part, kRedBlocks, 1, outv, 1, 0, st));
        PNP_CUDA(launch_reduce_partial(kRedSq, w, nullptr, N, N, 1, g->n, part, st));
        PNP_CUDA(launch_reduce_final(part, kRedBlocks, 1, outv + 1, 1, 0, st));
        PNP_CUDA(launch_scale_by_rnorm(w, u, N, outv + 1, st));
        double hv[2];
        PNP_CUDA(cudaMemcpyAsync(hv, outv, sizeof hv, cudaMemcpyDeviceToHost, st));
        PNP_CUDA(cudaStreamSynchronize(st));
        const double rq = hv[0];
        const bool done = it > 1 && std::fabs(rq - lam) <= tol * std::fabs(rq);
        lam = rq;
        if (done) break;
    }
    *h_L = lam;
    if (h_iters) *h_iters = it > max_iters ? max_iters : it;
    return PNP_OK;
}

// Power-iteration settings of the step sizes the library computes itself.
constexpr int kStepPowerIters = 100;
constexpr double kStepPowerTol = 1e-6;

// eta_k = 1 / L_k for every stage (stages already checked): L_k of the stage's
// level and sketch kind from the workspace's cache, else by power iteration
// (then cached).
int step_sizes(const pnp_geom& g, const Layout& L, const pnp_stage* stages, int n_stages, double* eta, char* ws,
               cudaStream_t st)
{
    for (int k = 0; k < n_stages; ++k) {
        const int li = level_index(stages[k].factor);
        const int kind = stages[k].factor > 1 && stages[k].kind == PNP_SKETCH_BICUBIC ? 1 : 0;
        double Lk = 0.0;
        if (!reg_get_L(ws, li, kind, &Lk)) {
            if (int e = power_iter_impl(g, L, li, kind, kStepPowerIters, kStepPowerTol, &Lk, nullptr, ws, st))
                return e;
            if (!(Lk > 0.0) || !std::isfinite(Lk))
                return fail(PNP_EINVAL, "stage %d: operator norm %g is not positive (no ray meets the image?)", k, Lk);
            reg_put_L(ws, li, kind, Lk);
        }
        eta[k] = 1.0 / Lk;
    }
    return PNP_OK;
}

int check_stages(const pnp_geom& g, const Layout& L, const pnp_stage* stages, int n_stages)
{
    if (!stages || n_stages < 1) return fail(PNP_EINVAL, "stages are required");
    for (int k = 0; k < n_stages; ++k) {
        int li = 0;
        if (int e = check_level(g, stages[k].factor, L, &li)) return e;
        if (stages[k].kind != PNP_SKETCH_POOL && stages[k].kind != PNP_SKETCH_BICUBIC)
            return fail(PNP_EINVAL, "stage %d: unknown sketch kind %d", k, stages[k].kind);
    }
    return PNP_OK;
}

}  // namespace

// a_i of iteration i (Sec. 3: a_i = (i-1)/(i+3); 0 without momentum, Eq. 5).
float momentum_coef(long i, int momentum)
{
    return momentum ? (float)((double)(i - 1) / (double)(i + 3)) : 0.0f;
}

namespace {

// Counter-based SplitMix64 (Steele, Lea & Flood 2014): number t of the stream is
// the generator's finaliser applied to seed + t * golden gamma.
class SplitMixStream {
public:
    explicit SplitMixStream(uint64_t seed) : seed_(seed) {}
    uint64_t next()
    {
        ++count_;
        uint64_t x = seed_ + count_ * 0x9e3779b97f4a7c15ull;
        x ^= x >> 30;
        x *= 0xbf58476d1ce4e5b9ull;
        x ^= x >> 27;
        x *= 0x94d049bb133111ebull;
        return x ^ (x >> 31);
    }
    // uniform in [0, m): redraw the numbers below 2^64 mod m, then reduce
    uint32_t below(uint32_t m)
    {
        const uint64_t lo = (~(uint64_t)0 - (uint64_t)m + 1) % m;  // (2^64 - m) mod m = 2^64 mod m
        uint64_t u;
        do u = next(); while (u < lo);
        return (uint32_t)(u % m);
    }
private:
    uint64_t seed_;
    uint64_t count_ = 0;
};

}  // namespace

// The subset order of a schedule: per stage with P > 1, a Fisher-Yates
// permutation of the subsets per epoch of P iterations; zeros where P = 1.
void subset_order(const pnp_stage* stages, int n_stages, uint64_t seed, int32_t* out)
{
    SplitMixStream rng(seed);
    std::vector<int32_t> perm;
    for (int k = 0; k < n_stages; ++k) {
        const int P = stages[k].n_subsets, T = stages[k].iters;
        if (P <= 1) {
            std::fill(out, out + T, 0);
            out += T;
            continue;
        }
        perm.resize((size_t)P);
        for (int first = 0; first < T; first += P) {
            for (int a = 0; a < P; ++a) perm[(size_t)a] = a;
            for (int j = P - 1; j > 0; --j) std::swap(perm[(size_t)j], perm[rng.below((uint32_t)j + 1)]);
            const int take = std::min(P, T - first);
            std::copy(perm.begin(), perm.begin() + take, out);
            out += take;
        }
    }
}

}  // namespace pnp

extern "C" {

int pnp_power_iter_kind(const pnp_geom* g, int factor, int kind, int max_iters, double tol, double* h_L,
                        int* h_iters, void* d_ws, void* stream)
{
    t_err.clear();
    if (kind != PNP_SKETCH_POOL && kind != PNP_SKETCH_BICUBIC) return fail(PNP_EINVAL, "unknown sketch kind %d", kind);
    if (int e = validate_geom(g)) return e;
    Layout L = make_layout(*g);
    int li = 0;
    if (int e = check_level(*g, factor, L, &li)) return e;
    if (max_iters < 1 || !(tol >= 0.0)) return fail(PNP_EINVAL, "need max_iters >= 1 and tol >= 0");
    if (!h_L) return fail(PNP_EINVAL, "h_L is NULL");
    if (int e = check_ws(*g, d_ws)) return e;
    return power_iter_impl(*g, L, li, kind, max_iters, tol, h_L, h_iters, (char*)d_ws, S(stream));
}

int pnp_step_sizes(const pnp_geom* g, const pnp_stage* stages, int n_stages, double* h_eta, void* d_ws,
                   void* stream)
{
    t_err.clear();
    if (int e = validate_geom(g)) return e;
    Layout L = make_layout(*g);
    if (int e = check_stages(*g, L, stages, n_stages)) return e;
    if (!h_eta) return fail(PNP_EINVAL, "h_eta is NULL");
    if (int e = check_ws(*g, d_ws)) return e;
    return step_sizes(*g, L, stages, n_stages, h_eta, (char*)d_ws, S(stream));
}

int pnp_schedule(const pnp_stage* stages, int n_stages, const int32_t* h_subset_seq, int momentum,
                 int32_t* h_stage, int32_t* h_subset, float* h_amom, int64_t capacity, int64_t* h_total)
{
    t_err.clear();
    if (!stages || n_stages < 1 || !h_total) return fail(PNP_EINVAL, "stages and h_total are required");
    int64_t total = 0;
    bool any_subsets = false;
    for (int k = 0; k < n_stages; ++k) {
        if (stages[k].iters < 0) return fail(PNP_EINVAL, "stage %d has negative iterations", k);
        if (stages[k].n_subsets < 1) return fail(PNP_EINVAL, "stage %d: n_subsets < 1", k);
        any_subsets |= stages[k].n_subsets > 1 && stages[k].iters > 0;
        total += stages[k].iters;
    }
    *h_total = total;
    if (total > capacity) return fail(PNP_EINVAL, "schedule has %lld iterations, capacity %lld", (long long)total,
                                      (long long)capacity);
    if (total > 0 && (!h_stage || !h_subset || !h_amom)) return fail(PNP_EINVAL, "output arrays are required");
    if (any_subsets && !h_subset_seq) return fail(PNP_EINVAL, "subset sequence required");
    int64_t i = 0;
    for (int k = 0; k < n_stages; ++k)
        for (int jj = 0; jj < stages[k].iters; ++jj, ++i) {
            const int P = stages[k].n_subsets;
            const int p = P > 1 ? h_subset_seq[i] : 0;
            if (p < 0 || p >= P)
                return fail(PNP_EINVAL, "subset_seq[%lld]=%d outside stage %d's [0, %d)", (long long)i, p, k, P);
            h_stage[i] = k;
            h_subset[i] = p;
            h_amom[i] = momentum_coef((long)(i + 1), momentum);
        }
    return PNP_OK;
}

int pnp_subset_sequence(const pnp_stage* stages, int n_stages, uint64_t seed, int32_t* h_seq, int64_t capacity,
                        int64_t* h_total)
{
    t_err.clear();
    if (!stages || n_stages < 1 || !h_total) return fail(PNP_EINVAL, "stages and h_total are required");
    int64_t total = 0;
    for (int k = 0; k < n_stages; ++k) {
        if (stages[k].iters < 0) return fail(PNP_EINVAL, "stage %d has negative iterations", k);
        if (stages[k].n_subsets < 1) return fail(PNP_EINVAL, "stage %d: n_subsets < 1", k);
        total += stages[k].iters;
    }
    *h_total = total;
    if (total > capacity) return fail(PNP_EINVAL, "schedule has %lld iterations, capacity %lld", (long long)total,
                                      (long long)capacity);
    if (total > 0 && !h_seq) return fail(PNP_EINVAL, "h_seq is NULL");
    subset_order(stages, n_stages, seed, h_seq);
    return PNP_OK;
}

namespace {

struct ProblemState {
    const pnp_problem* pb;
    Layout L;
    long total;
    int tv_parts;
    Tuned tuned;
    VrLayout vr;
    char* vr_buf = nullptr;
};

int validate_problem(const pnp_problem& q, const pnp_run_params& pr, int idx, ProblemState* out)
{
    const pnp_geom* g = &q.geom;
    if (int e = validate_geom(g)) return e;
    out->pb = &q;
    out->L = make_layout(*g);
    if (!q.stages || q.n_stages < 1 || !q.h_eta || !q.d_b || !q.d_x)
        return fail(PNP_EINVAL, "problem %d: stages, eta, b and x are required", idx);
    if ((q.d_xtrue == nullptr) != (q.h_psnr_log == nullptr))
        return fail(PNP_EINVAL, "problem %d: d_xtrue and h_psnr_log must be given together", idx);
    long total = 0;
    bool any_subsets = false;
    for (int k = 0; k < q.n_stages; ++k) {
        int li = 0;
        if (int e = check_level(*g, q.stages[k].factor, out->L, &li)) return e;
        if (q.stages[k].iters < 0) return fail(PNP_EINVAL, "stage %d has negative iterations", k);
        if (q.stages[k].n_subsets < 1 || q.stages[k].n_subsets > g->n_views)
            return fail(PNP_EINVAL, "stage %d: n_subsets outside [1, n_views]", k);
        if (!(std::isfinite(q.h_eta[k]) && q.h_eta[k] >= 0.0)) return fail(PNP_EINVAL, "eta[%d] invalid", k);
        if (q.stages[k].kind != PNP_SKETCH_POOL && q.stages[k].kind != PNP_SKETCH_BICUBIC)
            return fail(PNP_EINVAL, "stage %d: unknown sketch kind %d", k, q.stages[k].kind);
        if (q.stages[k].estimator < PNP_EST_MINIBATCH || q.stages[k].estimator > PNP_EST_SAGA)
            return fail(PNP_EINVAL, "stage %d: unknown estimator %d", k, q.stages[k].estimator);
        any_subsets |= q.stages[k].n_subsets > 1;
        total += q.stages[k].iters;
    }
    if (total > (1L << 30)) return fail(PNP_EINVAL, "too many iterations");
    if (any_subsets && !q.h_subset_seq) return fail(PNP_EINVAL, "subset sequence required");
    if (q.h_psnr_log && total * g->batch > PNP_MAX_LOG_ITERS)
        return fail(PNP_EINVAL, "PSNR log limited to %d iterations x batch", PNP_MAX_LOG_ITERS);
    if (q.start_iter < 0 || q.start_iter > total)
        return fail(PNP_EINVAL, "problem %d: start_iter %d outside [0, %ld]", idx, q.start_iter, total);
    if (q.d_y && q.d_y == q.d_x) return fail(PNP_EINVAL, "problem %d: d_y must not alias d_x", idx);
    if (int e = check_ws(*g, q.d_ws)) return e;
    long i = 0;
    for (int k = 0; k < q.n_stages; ++k)
        for (int jj = 0; jj < q.stages[k].iters; ++jj, ++i)
            if (q.stages[k].n_subsets > 1 &&
                (q.h_subset_seq[i] < 0 || q.h_subset_seq[i] >= q.stages[k].n_subsets))
                return fail(PNP_EINVAL, "subset_seq[%ld]=%d outside stage %d's [0, %d)", i, q.h_subset_seq[i], k,
                            q.stages[k].n_subsets);
    out->total = total;
    out->tuned = reg_tuned(q.d_ws);
    out->vr = vr_layout(*g, q.stages, q.n_stages);
    if (out->vr.bytes > 0) {
        void* vb;
        size_t vbytes;
        reg_vr(q.d_ws, &vb, &vbytes);
        if (!vb || vbytes < out->vr.bytes)
            return fail(PNP_ESTATE, "problem %d: SVRG/SAGA stages need an estimator buffer of %zu bytes "
                        "(pnp_set_vr_buffer); registered: %zu", idx, out->vr.bytes, vbytes);
        out->vr_buf = (char*)vb;
    }
    const bool do_tv = pr.tv_iters > 0 && pr.lambda > 0.0f;
    out->tv_parts = do_tv ? tile_tv_parts_for(g->n, g->batch, out->tuned.tile)
                          : ((g->n + 31) / 32) * ((g->n + 7) / 8);
    return PNP_OK;
}

int run_many_impl(const pnp_problem* pb_in, int np, const pnp_run_params* params, void* stream)
{
    if (!pb_in || np < 1) return fail(PNP_EINVAL, "no problems");
    if (np > kMaxRunClasses) return fail(PNP_EUNSUPPORTED, "at most %d geometry classes per call", kMaxRunClasses);
    if (!params) return fail(PNP_EINVAL, "params are required");
    // problems without step sizes get eta_k = 1/L_k from the library (cached per
    // workspace; the first computation of a level's L synchronises the stream)
    std::vector<pnp_problem> pbv(pb_in, pb_in + np);
    std::vector<std::vector<double>> etas((size_t)np);
    // problems without a subset sequence get the seeded order of their stages
    std::vector<std::vector<int32_t>> seqs((size_t)np);
    for (int c = 0; c < np; ++c) {
        pnp_problem& q = pbv[c];
        if (q.h_subset_seq || !q.stages || q.n_stages < 1) continue;
        int64_t total = 0;
        bool any_subsets = false;
        for (int k = 0; k < q.n_stages; ++k) {
            if (q.stages[k].iters < 0 || q.stages[k].n_subsets < 1) { total = -1; break; }
            total += q.stages[k].iters;
            any_subsets |= q.stages[k].n_subsets > 1;
        }
        if (!any_subsets || total < 0 || total > (1L << 30)) continue;   // validate_problem reports these
        seqs[c].resize((size_t)std::max<int64_t>(total, 1));
        subset_order(q.stages, q.n_stages, params->subset_seed, seqs[c].data());
        q.h_subset_seq = seqs[c].data();
    }
    for (int c = 0; c < np; ++c) {
        pnp_problem& q = pbv[c];
        if (q.h_eta) continue;
        if (int e = validate_geom(&q.geom)) return e;
        const Layout Lq = make_layout(q.geom);
        if (int e = check_stages(q.geom, Lq, q.stages, q.n_stages)) return e;
        if (int e = check_ws(q.geom, q.d_ws)) return e;
        etas[c].resize((size_t)q.n_stages);
        if (int e = step_sizes(q.geom, Lq, q.stages, q.n_stages, etas[c].data(), (char*)q.d_ws, S(stream))) return e;
        q.h_eta = etas[c].data();
    }
    const pnp_problem* pb = pbv.data();
    const pnp_run_params& pr = *params;
    if (!(pr.alpha > 0.0f && pr.alpha <= 1.0f)) return fail(PNP_EINVAL, "alpha must be in (0, 1]");
    if (!(pr.lambda >= 0.0f) || !std::isfinite(pr.lambda)) return fail(PNP_EINVAL, "lambda must be >= 0");
    if (pr.tv_iters < 0 || pr.tv_iters > 100000) return fail(PNP_EINVAL, "tv_iters outside [0, 100000]");
    if (pr.flags & ~(PNP_RUN_GRAPH | PNP_RUN_KERNEL_TIMES | PNP_RUN_PERSISTENT))
        return fail(PNP_EINVAL, "unknown run flags %d", pr.flags);
    if ((pr.flags & PNP_RUN_GRAPH) && (pr.flags & PNP_RUN_KERNEL_TIMES))
        return fail(PNP_EINVAL, "PNP_RUN_KERNEL_TIMES cannot be combined with PNP_RUN_GRAPH");
    // the phase kernels in their persistent form for this call (restored on return)
    struct PersistentScope {
        bool prev;
        explicit PersistentScope(bool on) : prev(persistent_mode()) { set_persistent_mode(on); }
        ~PersistentScope() { set_persistent_mode(prev); }
    } persistent_scope((pr.flags & PNP_RUN_PERSISTENT) != 0);
    std::vector<ProblemState> ps((size_t)np);
    for (int c = 0; c < np; ++c)
        if (int e = validate_problem(pb[c], pr, c, &ps[c])) return e;
    for (int c = 0; c < np; ++c)
        for (int d = c + 1; d < np; ++d)
            if (pb[c].d_ws == pb[d].d_ws || pb[c].d_x == pb[d].d_x)
                return fail(PNP_EINVAL, "problems %d and %d share a workspace or an output", c, d);
    cudaStream_t st = S(stream);
    const bool do_tv = pr.tv_iters > 0 && pr.lambda > 0.0f;
    // one denoiser launch covers every class, so the classes share its variant:
    // a register-resident one only when every class was tuned to it (the strips
    // then take the first class's CTA height)
    bool same_family = true;
    for (int c = 0; c < np; ++c) same_family = same_family && tv_family(ps[c].tuned.tile) == tv_family(ps[0].tuned.tile);
    const bool all_warp = same_family && ps[0].tuned.tile == kTvTileWarp;
    for (int c = 0; c < np; ++c) {
        if (!same_family && tv_family(ps[c].tuned.tile) != 0) ps[c].tuned.tile = 0;
        if (same_family && tv_is_strip(ps[0].tuned.tile)) ps[c].tuned.tile = ps[0].tuned.tile;
        if (do_tv) ps[c].tv_parts = tile_tv_parts_for(pb[c].geom.n, pb[c].geom.batch, ps[c].tuned.tile);
    }
    const bool all_register = same_family && tv_family(ps[0].tuned.tile) != 0;
    long max_total = 0;
    for (const auto& q : ps) max_total = std::max(max_total, q.total);

    long min_start = max_total;
    for (int c = 0; c < np; ++c) min_start = std::min(min_start, (long)pb[c].start_iter);
    const bool timed = (pr.flags & PNP_RUN_KERNEL_TIMES) != 0;
    // the denoiser's last launch also writes the coefficient image of the next
    // iteration's level (full grid, or the 2x pooled sketch) when that iteration
    // is a mini-batch one (it then needs no coefficient-image kernel)
    const bool fuse_quad = do_tv && !all_register && fuse_quad_enabled();
    (void)all_warp;
    auto issue = [&]() -> int {
        int e0 = PNP_OK;
        for (int c = 0; c < np; ++c) {
            const pnp_geom& g = pb[c].geom;
            char* ws = (char*)pb[c].d_ws;
            const float* y0 = pb[c].d_y ? pb[c].d_y : pb[c].d_x;
            PNP_CUDA(launch_copy(y0, (float*)(ws + ps[c].L.off_y), (size_t)g.batch * g.n * g.n, st));
        }
        std::vector<int> stage((size_t)np, 0), in_stage((size_t)np, 0);
        // per-iteration launch items of the active classes
        std::vector<PrepArgs> v_prep((size_t)np);
        std::vector<FwdArgs> v_fwd((size_t)np);
        std::vector<BackArgs> v_back((size_t)np);
        std::vector<TvItem> v_tv((size_t)np);
        std::vector<int> v_act((size_t)np), v_bic((size_t)np), v_need((size_t)np), v_lvl((size_t)np);
        // x alternates between d_x (even iteration count) and the workspace copy, so
        // that the denoiser can read x_{i-1} around its tile while writing x_i
        std::vector<long> done((size_t)np, 0);
        std::vector<char> quad_ready((size_t)np, 0);
        for (long i = 1; i <= max_total; ++i) {
            if (i <= min_start) {       // resumed runs: advance the schedule cursors only
                for (int c = 0; c < np; ++c) {
                    if (i > ps[c].total) continue;
                    const pnp_problem& q = pb[c];
                    while (in_stage[c] >= q.stages[stage[c]].iters) { ++stage[c]; in_stage[c] = 0; }
                    ++in_stage[c];
                }
                continue;
            }
            PrepArgs* prep = v_prep.data();
            FwdArgs* fwd = v_fwd.data();
            BackArgs* back = v_back.data();
            TvItem* tv = v_tv.data();
            int* act = v_act.data();
            int* bic = v_bic.data();
            int* need_prep = v_need.data();
            int* lvl = v_lvl.data();
            int na = 0;
            const float amom = momentum_coef(i, pr.momentum);
            for (int c = 0; c < np; ++c) {
                if (i > ps[c].total) continue;
                const pnp_problem& q = pb[c];
                while (in_stage[c] >= q.stages[stage[c]].iters) { ++stage[c]; in_stage[c] = 0; }
                const pnp_stage& sk = q.stages[stage[c]];
                ++in_stage[c];
                if (i <= (long)q.start_iter) continue;   // this class resumes later
                const pnp_geom& g = q.geom;
                const Layout& L = ps[c].L;
                const int li = level_index(sk.factor);
                const LevelLayout& lv = L.lv[li];
                char* ws = (char*)q.d_ws;
                const int P = sk.n_subsets;
                const int p = P > 1 ? q.h_subset_seq[i - 1] : 0;
                float* y = (float*)(ws + L.off_y);
                float* z = (float*)(ws + L.off_z);
                float* res = (float*)(ws + L.off_res);
                const int est = P > 1 ? sk.estimator : PNP_EST_MINIBATCH;
                if (est != PNP_EST_MINIBATCH) {
                    // SVRG / SAGA stages run their own gradient launches; the denoiser joins the rest
                    if (int e = vr_step(g, L, li, ws, ps[c].vr_buf, ps[c].vr, est, sk.kind, y, q.d_b, p, P,
                                        in_stage[c] - 1, (float)q.h_eta[stage[c]], z, st))
                        return e;
                    bic[na] = 1;
                } else if (sk.kind == PNP_SKETCH_BICUBIC && lv.factor > 1) {
                    // so do bicubic stages
                    if (int e = grad_into(g, L, li, ws, y, q.d_b, p, P, kBackStep, (float)q.h_eta[stage[c]], z, st,
                                          PNP_SKETCH_BICUBIC))
                        return e;
                    bic[na] = 1;
                } else {
                    bic[na] = 0;
                }
                need_prep[na] = quad_ready[c] != lv.factor;
                lvl[na] = li;
                prep[na] = PrepArgs{y, g.n, lv.factor, g.batch, (float4*)(ws + lv.off_quad), lv.qw};
                fwd[na] = fwd_args(g, lv, ws, p, P, q.d_b, res, g.batch, reg_weights(ws), true);
                const double cs = P <= 1 ? 1.0 : (double)P;
                const float scale = (float)(g.step * lv.factor * cs / ((double)lv.factor * lv.factor));
                back[na] = back_args(g, lv, ws, p, P, res, kBackStep, scale, y, (float)q.h_eta[stage[c]], z, g.batch,
                                     true);
                const size_t img = (size_t)g.batch * g.n * g.n;
                float* tvb = (float*)(ws + L.off_tv);
                float* x2 = (float*)(ws + L.off_x2);
                TvItem t{};
                t.xin = done[c] % 2 == 0 ? q.d_x : x2;
                t.xprev = done[c] % 2 == 0 ? x2 : q.d_x;
                ++done[c];
                quad_ready[c] = 0;
                if (fuse_quad && i < ps[c].total) {
                    // the stage of iteration i + 1 (the cursor skips stages without iterations)
                    int sn = stage[c];
                    if (in_stage[c] >= q.stages[sn].iters)
                        do ++sn; while (q.stages[sn].iters == 0);
                    const pnp_stage& nx = q.stages[sn];
                    const bool minibatch = nx.n_subsets <= 1 || nx.estimator == PNP_EST_MINIBATCH;
                    const bool pooled = nx.factor == 1 || nx.kind == PNP_SKETCH_POOL;
                    if (minibatch && pooled && tv_fuses_quad(ps[c].tuned.tile, g.n, g.batch, nx.factor)) {
                        const LevelLayout& lq = L.lv[level_index(nx.factor)];
                        t.quad = (float4*)(ws + lq.off_quad);
                        t.qw = lq.qw;
                        t.qs = nx.factor;
                        quad_ready[c] = (char)nx.factor;
                    }
                }
                t.z = z; t.y = y; t.xtrue = q.d_xtrue;
                t.mse_part = q.h_psnr_log ? (double*)(ws + L.off_red) : nullptr;
                t.state_a = tvb; t.state_b = tvb + 4 * img;
                t.n = g.n; t.batch = g.batch; t.tile = ps[c].tuned.tile; t.amom = amom;
                tv[na] = t;
                act[na] = c;
                ++na;
                (void)li;
            }
            if (na == 0) break;
            // the active classes in groups of at most kMaxClasses: one launch per
            // phase and group (a single launch per phase for up to kMaxClasses classes)
            for (int a0 = 0; a0 < na; a0 += kMaxClasses) {
                const int a1 = std::min(na, a0 + kMaxClasses);
                // one launch shape per phase: the tuned one of the group's class with the
                // most level pixels in it (the only class when there is one)
                int lanes_sel = 0, groups_sel = 0;
                {
                    double wmax = -1.0;
                    for (int a = a0; a < a1; ++a) {
                        if (bic[a]) continue;
                        const pnp_geom& g = pb[act[a]].geom;
                        const double ns = (double)g.n / (double)(1 << lvl[a]);
                        const double work = (double)g.batch * ns * ns;
                        if (work > wmax) {
                            wmax = work;
                            lanes_sel = ps[act[a]].tuned.lanes[lvl[a]];
                            groups_sel = ps[act[a]].tuned.groups[lvl[a]];
                        }
                    }
                }
                // pooled-sketch classes share one launch per phase
                PrepArgs pp[kMaxClasses];
                FwdArgs ff[kMaxClasses];
                BackArgs bb[kMaxClasses];
                int m = 0, mp = 0;
                for (int a = a0; a < a1; ++a) {
                    if (bic[a]) continue;
                    if (need_prep[a]) pp[mp++] = prep[a];
                    ff[m] = fwd[a];
                    bb[m] = back[a];
                    ++m;
                }
                if (mp > 0) {
                    if (timed && (e0 = g_timer.mark(PNP_PHASE_PREP, st, true))) return e0;
                    PNP_CUDA(launch_prep_multi(pp, mp, st));
                    if (timed && (e0 = g_timer.mark(PNP_PHASE_PREP, st, false))) return e0;
                }
                if (m > 0) {
                    if (timed && (e0 = g_timer.mark(PNP_PHASE_FORWARD, st, true))) return e0;
                    PNP_CUDA(launch_forward_multi(ff, m, st, lanes_sel));
                    if (timed && (e0 = g_timer.mark(PNP_PHASE_FORWARD, st, false))) return e0;
                    if (timed && (e0 = g_timer.mark(PNP_PHASE_BACKWARD, st, true))) return e0;
                    PNP_CUDA(launch_backward_multi(bb, m, st, groups_sel));
                    if (timed && (e0 = g_timer.mark(PNP_PHASE_BACKWARD, st, false))) return e0;
                }
            }
            for (int a0 = 0; a0 < na; a0 += kMaxClasses) {
                const int cnt = std::min(na - a0, kMaxClasses);
                if (do_tv) {
                    if (timed && (e0 = g_timer.mark(PNP_PHASE_DENOISE, st, true))) return e0;
                    PNP_CUDA(launch_tv_tiled_multi(tv + a0, cnt, pr.lambda, pr.tv_iters, pr.alpha, st));
                    if (timed && (e0 = g_timer.mark(PNP_PHASE_DENOISE, st, false))) return e0;
                } else {
                    for (int a = a0; a < a0 + cnt; ++a) {
                        const TvItem& t = tv[a];
                        PNP_CUDA(launch_tv_final(t.z, nullptr, 0, t.n, t.batch, pr.lambda, pr.alpha, t.amom,
                                                 t.xprev, t.y, t.xtrue, t.mse_part, st, t.xin));
                    }
                }
            }
            for (int a = 0; a < na; ++a) {
                const int c = act[a];
                const pnp_problem& q = pb[c];
                if (!q.h_psnr_log) continue;
                char* ws = (char*)q.d_ws;
                double* dlog = (double*)(ws + ps[c].L.off_log);
                PNP_CUDA(launch_reduce_final((double*)(ws + ps[c].L.off_red), ps[c].tv_parts, q.geom.batch,
                                             dlog + (i - 1) * q.geom.batch, 1, 0, st));
            }
        }
        for (int c = 0; c < np; ++c) {
            const pnp_geom& g = pb[c].geom;
            char* ws = (char*)pb[c].d_ws;
            if (done[c] % 2 == 1)
                PNP_CUDA(launch_copy((float*)(ws + ps[c].L.off_x2), pb[c].d_x, (size_t)g.batch * g.n * g.n, st));
        }
        for (int c = 0; c < np; ++c) {
            if (!pb[c].d_y) continue;
            const pnp_geom& g = pb[c].geom;
            char* ws = (char*)pb[c].d_ws;
            PNP_CUDA(launch_copy((float*)(ws + ps[c].L.off_y), pb[c].d_y, (size_t)g.batch * g.n * g.n, st));
        }
        return PNP_OK;
    };

    Hasher h;
    h.val(np);
    h.val(pr.alpha); h.val(pr.lambda); h.val(pr.tv_iters); h.val(pr.momentum); h.val(pr.flags);
    h.val(stream);
    for (int c = 0; c < np; ++c) {
        const pnp_problem& q = pb[c];
        h.val(q.geom);
        h.val(q.d_b); h.val(q.d_x); h.val(q.d_xtrue); h.val(q.d_ws);
        h.val(q.h_psnr_log != nullptr);
        h.val(q.start_iter); h.val(q.d_y);
        h.add(q.stages, sizeof(pnp_stage) * (size_t)q.n_stages);
        h.add(q.h_eta, sizeof(double) * (size_t)q.n_stages);
        if (q.h_subset_seq) h.add(q.h_subset_seq, sizeof(int32_t) * (size_t)ps[c].total);
        h.val(ps[c].tuned);
        h.val(reg_weights(q.d_ws));
        h.val(ps[c].vr_buf);
    }
    if (int e = run_maybe_graph((pr.flags & PNP_RUN_GRAPH) != 0, h.h, st, issue)) return e;

    for (int c = 0; c < np; ++c) {
        const pnp_problem& q = pb[c];
        if (!q.h_psnr_log || ps[c].total == 0) continue;
        char* ws = (char*)q.d_ws;
        const size_t first = (size_t)q.start_iter * q.geom.batch;
        const size_t count = (size_t)ps[c].total * q.geom.batch - first;
        if (count == 0) continue;
        std::vector<double> mse(count);
        PNP_CUDA(cudaMemcpyAsync(mse.data(), (double*)(ws + ps[c].L.off_log) + first, count * sizeof(double),
                                 cudaMemcpyDeviceToHost, st));
        PNP_CUDA(cudaStreamSynchronize(st));
        const double npix = (double)q.geom.n * q.geom.n;
        for (size_t k = 0; k < count; ++k) q.h_psnr_log[first + k] = 10.0 * std::log10(npix / mse[k]);
    }
    return PNP_OK;
}

}  // namespace

int pnp_run(const pnp_geom* g, const pnp_stage* stages, int n_stages, const double* h_eta,
            const int32_t* h_subset_seq, const pnp_run_params* params, const float* d_b, float* d_x,
            const float* d_xtrue, double* h_psnr_log, void* d_ws, void* stream)
{
    t_err.clear();
    if (!g) return fail(PNP_EINVAL, "geometry pointer is NULL");
    pnp_problem q{};
    q.geom = *g;
    q.stages = stages;
    q.n_stages = n_stages;
    q.h_eta = h_eta;
    q.h_subset_seq = h_subset_seq;
    q.d_b = d_b;
    q.d_x = d_x;
    q.d_xtrue = d_xtrue;
    q.h_psnr_log = h_psnr_log;
    q.d_ws = d_ws;
    return run_many_impl(&q, 1, params, stream);
}

int pnp_set_weights(const pnp_geom* g, const float* d_w, void* d_ws)
{
    t_err.clear();
    if (int e = validate_geom(g)) return e;
    if (int e = check_ws(*g, d_ws)) return e;
    reg_set_weights(d_ws, d_w);
    return PNP_OK;
}

int pnp_vr_buffer_size(const pnp_geom* g, const pnp_stage* stages, int n_stages, size_t* bytes)
{
    t_err.clear();
    if (int e = validate_geom(g)) return e;
    if (!stages || n_stages < 1 || !bytes) return fail(PNP_EINVAL, "stages and bytes are required");
    for (int k = 0; k < n_stages; ++k)
        if (stages[k].factor < 1 || g->n % stages[k].factor)
            return fail(PNP_EINVAL, "stage %d: factor %d does not divide n", k, stages[k].factor);
    *bytes = vr_layout(*g, stages, n_stages).bytes;
    return PNP_OK;
}

int pnp_set_vr_buffer(const pnp_geom* g, void* d_buf, size_t bytes, void* d_ws)
{
    t_err.clear();
    if (int e = validate_geom(g)) return e;
    if (int e = check_ws(*g, d_ws)) return e;
    if (d_buf && ((uintptr_t)d_buf & 255u)) return fail(PNP_EINVAL, "estimator buffer must be 256-byte aligned");
    reg_set_vr(d_ws, d_buf, bytes);
    return PNP_OK;
}

int pnp_run_many(const pnp_problem* problems, int n_problems, const pnp_run_params* params, void* stream)
{
    t_err.clear();
    return run_many_impl(problems, n_problems, params, stream);
}

int pnp_autotune(const pnp_geom* g, const pnp_stage* stages, int n_stages, const pnp_run_params* params,
                 void* d_ws, void* stream)
{
    t_err.clear();
    if (int e = validate_geom(g)) return e;
    if (!stages || n_stages < 1 || !params) return fail(PNP_EINVAL, "stages and params are required");
    if (int e = check_ws(*g, d_ws)) return e;
    Layout L = make_layout(*g);
    for (int k = 0; k < n_stages; ++k) {
        int li = 0;
        if (int e = check_level(*g, stages[k].factor, L, &li)) return e;
        if (stages[k].n_subsets < 1 || stages[k].n_subsets > g->n_views)
            return fail(PNP_EINVAL, "stage %d: n_subsets outside [1, n_views]", k);
    }
    cudaStream_t st = S(stream);
    char* ws = (char*)d_ws;
    const size_t img = (size_t)g->batch * g->n * g->n;
    float* y = (float*)(ws + L.off_y);
    float* z = (float*)(ws + L.off_z);
    float* res = (float*)(ws + L.off_res);
    float* tvb = (float*)(ws + L.off_tv);
    PNP_CUDA(launch_fill_hash(y, img, 0.0f, 1.0f, st));   // a noisy image: the denoiser's projections engage
    cudaEvent_t e0, e1;
    PNP_CUDA(cudaEventCreate(&e0));
    PNP_CUDA(cudaEventCreate(&e1));
    // best of five batches of eight launches after two warm-up launches
    auto timeit = [&](auto&& fn, float* ms) -> int {
        for (int rep = 0; rep < 2; ++rep) if (int e = fn()) return e;
        float best = 1e30f;
        for (int trial = 0; trial < 5; ++trial) {
            PNP_CUDA(cudaEventRecord(e0, st));
            for (int rep = 0; rep < 8; ++rep) if (int e = fn()) return e;
            PNP_CUDA(cudaEventRecord(e1, st));
            PNP_CUDA(cudaEventSynchronize(e1));
            float t = 0.0f;
            PNP_CUDA(cudaEventElapsedTime(&t, e0, e1));
            best = std::min(best, t);
        }
        *ms = best;
        return PNP_OK;
    };
    Tuned tu;
    int rc = PNP_OK;
    for (int k = 0; k < n_stages && rc == PNP_OK; ++k) {
        const int li = level_index(stages[k].factor);
        if (tu.lanes[li]) continue;                     // first stage of a level decides
        const LevelLayout& lv = L.lv[li];
        const int P = stages[k].n_subsets;
        rc = launch_prep_quad(y, g->n, lv.factor, g->batch, (float4*)(ws + lv.off_quad), lv.qw, st) == cudaSuccess
                 ? PNP_OK : fail(PNP_ECUDA, "prep failed");
        const FwdArgs fa = fwd_args(*g, lv, ws, 0, P, nullptr, res, g->batch, nullptr, true);
        float best = 1e30f;
        for (int Q : {4, 8, 16}) {
            float ms = 0.0f;
            if (rc == PNP_OK) rc = timeit([&]() -> int { PNP_CUDA(launch_forward(fa, st, Q)); return PNP_OK; }, &ms);
            if (rc == PNP_OK && ms < best) { best = ms; tu.lanes[li] = Q; }
        }
        const BackArgs ba = back_args(*g, lv, ws, 0, P, res, kBackRaw, 1.0f, nullptr, 0.0f, z, g->batch, true);
        best = 1e30f;
        const int nsub = subset_views(*g, 0, P);
        // 8 x 4 blocks with 1..16 view groups; 4 x 4 blocks with 8..64 groups (one,
        // two or a few views per thread; smaller CTAs pack the SMs more evenly)
        std::vector<int> shapes;
        for (int G = 1; G <= 16 && G <= nsub; G *= 2) shapes.push_back(G);
        for (int G : {8, 12, 16, 18, 20, 24, 32, 64, nsub, (nsub + 1) / 2})
            if (G >= 8 && G <= 64 && G <= nsub) shapes.push_back(PNP_BACK_TILE4 | G);
        // batches: the batched gather with 4, 8 or 16 images per thread
        for (int BC : {4, 8, 16}) {
            if (BC > 2 * g->batch || g->batch < 2) continue;
            for (int G : {4, 8, 16, 32})
                if (G <= nsub) shapes.push_back(PNP_BACK_BATCH(BC) | PNP_BACK_TILE4 | G);
            for (int G : {2, 4, 8, 16})
                if (G <= nsub) shapes.push_back(PNP_BACK_BATCH(BC) | G);
        }
        // the stored gather table, when one is registered
        if (ba.thdr) {
            for (int bc : {16, 8, 4}) {
                if (bc > g->batch && bc != 4) continue;     // (one to three images: 4 per thread)
                for (int G : {2, 4, 8, 16})
                    if (G <= nsub) shapes.push_back(PNP_BACK_TABLE | PNP_BACK_BATCH(bc) | G);
            }
        }
        // (the fixed-point scatter is not a candidate: its error depends on the
        // residual's dynamic range; it runs only where pnp_set_launch_shapes pins it)
        for (int shp : shapes) {
            float ms = 0.0f;
            if (rc == PNP_OK)
                rc = timeit([&]() -> int { PNP_CUDA(launch_backward(ba, st, shp)); return PNP_OK; }, &ms);
            if (rc == PNP_OK && ms < best) { best = ms; tu.groups[li] = shp; }
        }
    }
    const pnp_run_params& pr = *params;
    if (rc == PNP_OK && pr.tv_iters > 0 && pr.lambda > 0.0f) {
        // a denoise as the run issues it (up to 20 FGP iterations), momentum, and, when
        // a full-grid mini-batch stage follows, the level-1 coefficient image of y
        // (from the shared-memory tiles' last launch, or a separate kernel after the
        // register-resident variant, which does not write it)
        bool fused = fuse_quad_enabled();
        bool full_minibatch = false;
        for (int k = 0; k < n_stages; ++k)
            full_minibatch |= stages[k].factor == 1 &&
                              (stages[k].n_subsets <= 1 || stages[k].estimator == PNP_EST_MINIBATCH);
        fused = fused && full_minibatch;
        const LevelLayout& l1 = L.lv[level_index(1)];
        float* scratch = (float*)(ws + L.off_x2);       // x_{i-1} and y of the timed denoise
        if (launch_fill_hash(scratch, 2 * img, 0.0f, 1.0f, st) != cudaSuccess) rc = fail(PNP_ECUDA, "fill failed");
        const int T0 = tile_tv_tile(g->n, g->batch);
        const int iters = std::min(pr.tv_iters, 20);   // up to two launches, the last one with the ring
        float best = 1e30f;
        for (int T : {T0 - 6, T0 - 4, T0 - 2, T0, T0 + 2, T0 + 4, T0 + 6, 16, 24, 32, kTvTileWarp, kTvTileStrip8,
                      kTvTileStrip12, kTvTileStrip16}) {
            if (rc != PNP_OK) break;
            if (T != kTvTileWarp && !tv_is_strip(T) && (T < 8 || T > 40)) continue;
            TvItem it{};
            it.z = y; it.xprev = z; it.y = scratch + img; it.xin = scratch;
            it.state_a = tvb; it.state_b = tvb + 4 * img;
            it.n = g->n; it.batch = g->batch; it.tile = T; it.amom = 0.5f;
            const bool own_prep = full_minibatch && tv_family(T) != 0;
            if (fused && !own_prep) {
                it.quad = (float4*)(ws + l1.off_quad);
                it.qw = l1.qw;
            }
            float ms = 0.0f;
            rc = timeit([&]() -> int {
                PNP_CUDA(launch_tv_tiled_multi(&it, 1, pr.lambda, iters, pr.alpha, st));
                if (own_prep || (full_minibatch && !fused))
                    PNP_CUDA(launch_prep_quad(scratch + img, g->n, 1, g->batch, (float4*)(ws + l1.off_quad), l1.qw,
                                              st));
                return PNP_OK;
            }, &ms);
            if (rc != PNP_OK) break;
            if (ms < best) { best = ms; tu.tile = T; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != PNP_OK) return rc;
    reg_set_tuned(d_ws, tu);
    return PNP_OK;
}

int pnp_get_launch_shapes(const pnp_geom* g, pnp_launch_shapes* out, void* d_ws)
{
    t_err.clear();
    if (int e = validate_geom(g)) return e;
    if (!out) return fail(PNP_EINVAL, "output pointer is NULL");
    if (int e = check_ws(*g, d_ws)) return e;
    const Tuned tu = reg_tuned(d_ws);
    for (int k = 0; k < 4; ++k) {
        out->lanes[k] = tu.lanes[k];
        out->back[k] = tu.groups[k];
    }
    out->tile = tu.tile;
    return PNP_OK;
}

int pnp_set_launch_shapes(const pnp_geom* g, const pnp_launch_shapes* in, void* d_ws)
{
    t_err.clear();
    if (int e = validate_geom(g)) return e;
    if (!in) return fail(PNP_EINVAL, "input pointer is NULL");
    if (int e = check_ws(*g, d_ws)) return e;
    Tuned tu;
    for (int k = 0; k < 4; ++k) {
        const int q = in->lanes[k], b = in->back[k];
        if (q != 0 && q != 4 && q != 8 && q != 16) return fail(PNP_EINVAL, "lanes[%d] = %d not in {0, 4, 8, 16}", k, q);
        const int bg = b & 0xff;
        const int bc = back_batch_of(b);
        const bool scatter = (b & ~0xff) == PNP_BACK_SCATTER && (bg == 12 || bg == 16 || bg == 22 || bg == 32);
        const int slots = (b & PNP_BACK_TILE4) ? 16 : 32;
        const bool batch_ok = bc == 0 || bc == 1 || ((bc == 4 || bc == 8 || bc == 16) && bg * slots <= 512);
        const bool table = (b & ~(0xff | PNP_BACK_BATCH(0xff))) == PNP_BACK_TABLE && bg >= 1 && bg <= 16 &&
                           (bc == 0 || bc == 2 || bc == 4 || bc == 8 || bc == 16);
        const bool ok = b == 0 || scatter || table ||
                        ((b & ~(PNP_BACK_TILE4 | 0xff | PNP_BACK_BATCH(0xff))) == 0 && bg >= 1 &&
                         bg <= ((b & PNP_BACK_TILE4) ? 64 : 32) && batch_ok);
        if (!ok) return fail(PNP_EINVAL, "back[%d] = %#x is not a backprojector shape", k, b);
        tu.lanes[k] = q;
        tu.groups[k] = b;
    }
    if (in->tile != 0 && in->tile != kTvTileWarp && !tv_is_strip(in->tile) && (in->tile < 8 || in->tile > 40))
        return fail(PNP_EINVAL, "tile %d is neither 0, 1, 2, 3, 4 nor in [8, 40]", in->tile);
    tu.tile = in->tile;
    reg_set_tuned(d_ws, tu);
    return PNP_OK;
}

int pnp_objective(const pnp_geom* g, const float* d_x, const float* d_b, const float* d_xtrue,
                  double* h_out, void* d_ws, void* stream)
{
    t_err.clear();
    if (int e = validate_geom(g)) return e;
    if (!d_x || !d_b || !h_out) return fail(PNP_EINVAL, "x, b and h_out are required");
    if (int e = check_ws(*g, d_ws)) return e;
    Layout L = make_layout(*g);
    char* ws = (char*)d_ws;
    cudaStream_t st = S(stream);
    const LevelLayout& lv = L.lv[0];
    float* res = (float*)(ws + L.off_res);
    double* part = (double*)(ws + L.off_red);
    double* outv = part + (size_t)g->batch * red_parts(*g);
    const size_t nr = (size_t)g->n_views * g->n_det, N = (size_t)g->n * g->n;
    PNP_CUDA(launch_prep_quad(d_x, g->n, 1, g->batch, (float4*)(ws + lv.off_quad), lv.qw, st));
    PNP_CUDA(launch_forward(fwd_args(*g, lv, ws, 0, 1, d_b, res, g->batch), st));
    if (const float* wts = reg_weights(ws))
        PNP_CUDA(launch_reduce_partial(kRedWSq, res, wts, nr, nr, g->batch, g->n, part, st));
    else
        PNP_CUDA(launch_reduce_partial(kRedSq, res, nullptr, nr, nr, g->batch, g->n, part, st));
    PNP_CUDA(launch_reduce_final(part, kRedBlocks, g->batch, outv, 8, 0, st));
    PNP_CUDA(launch_reduce_partial(kRedTv, d_x, nullptr, N, N, g->batch, g->n, part, st));
    PNP_CUDA(launch_reduce_final(part, kRedBlocks, g->batch, outv, 8, 1, st));
    if (d_xtrue) {
        PNP_CUDA(launch_reduce_partial(kRedDiffSq, d_x, d_xtrue, N, N, g->batch, g->n, part, st));
        PNP_CUDA(launch_reduce_final(part, kRedBlocks, g->batch, outv, 8, 2, st));
    }
    std::vector<double> hv((size_t)g->batch * 8);
    PNP_CUDA(cudaMemcpyAsync(hv.data(), outv, hv.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    PNP_CUDA(cudaStreamSynchronize(st));
    for (int b = 0; b < g->batch; ++b) {
        h_out[3 * b + 0] = 0.5 * hv[8 * b + 0];
        h_out[3 * b + 1] = hv[8 * b + 1];
        h_out[3 * b + 2] = d_xtrue ? 10.0 * std::log10((double)N / hv[8 * b + 2]) : NAN;
    }
    return PNP_OK;
}

int pnp_sample_count(const pnp_geom* g, int factor, int subset, int n_subsets, double* h_count,
                     void* d_ws, void* stream)
{
    t_err.clear();
    if (int e = validate_geom(g)) return e;
    Layout L = make_layout(*g);
    int li = 0;
    if (int e = check_level(*g, factor, L, &li)) return e;
    if (int e = check_subset(*g, subset, n_subsets)) return e;
    if (!h_count) return fail(PNP_EINVAL, "h_count is NULL");
    if (int e = check_ws(*g, d_ws)) return e;
    char* ws = (char*)d_ws;
    cudaStream_t st = S(stream);
    double* outv = (double*)(ws + L.off_red) + (size_t)g->batch * red_parts(*g);
    const LevelLayout& lv = L.lv[li];
    PNP_CUDA(launch_count_samples((const int2*)(ws + lv.off_rayk), g->n_det, n_subsets <= 1 ? 0 : subset,
                                  n_subsets <= 1 ? 1 : n_subsets, subset_views(*g, subset, n_subsets),
                                  outv, st));
    PNP_CUDA(cudaMemcpyAsync(h_count, outv, sizeof(double), cudaMemcpyDeviceToHost, st));
    PNP_CUDA(cudaStreamSynchronize(st));
    return PNP_OK;
}


// ------------------------------------------------------------------ differentiable form
int pnp_tv_vjp_workspace_size(int n, int batch, int iters, size_t* bytes)
{
    t_err.clear();
    if (n < 2 || batch < 1 || iters < 0 || iters > 10000 || (double)n * n * batch * (2.0 * iters + 12) > 4.0e10)
        return fail(PNP_EINVAL, "bad n, batch or iters");
    if (!bytes) return fail(PNP_EINVAL, "bytes pointer is NULL");
    const size_t fl = tv_vjp_workspace_floats(n, batch, iters) * sizeof(float);
    *bytes = align_up(fl) + ((size_t)batch * tv_vjp_partials(n) + (size_t)batch) * sizeof(double);
    return PNP_OK;
}

namespace {
// FGP VJP plus the per-instance dJ/dlambda reduction (into dres[batch]).
int tv_vjp_core(const float* d_z, const float* d_xbar, float* d_zbar, int n, int batch, float lambda,
                int iters, char* vws, double* dres, cudaStream_t st)
{
    const size_t fl = tv_vjp_workspace_floats(n, batch, iters) * sizeof(float);
    double* part = (double*)(vws + align_up(fl));
    const int nparts = (int)tv_vjp_partials(n);
    PNP_CUDA(launch_tv_vjp(d_z, d_xbar, d_zbar, part, n, batch, lambda, iters, (float*)vws, st));
    PNP_CUDA(launch_reduce_final(part, nparts, batch, dres, 1, 0, st));
    return PNP_OK;
}
}  // namespace

int pnp_tv_vjp(const float* d_z, const float* d_xbar, float* d_zbar, double* h_lambar, int n, int batch,
               float lambda, int iters, void* d_ws, size_t ws_bytes, void* stream)
{
    t_err.clear();
    size_t need = 0;
    if (int e = pnp_tv_vjp_workspace_size(n, batch, iters, &need)) return e;
    if (!d_z || !d_xbar || !d_zbar) return fail(PNP_EINVAL, "z, xbar and zbar are required");
    if (iters > 0 && !(lambda > 0.0f && std::isfinite(lambda)))
        return fail(PNP_EINVAL, "lambda must be > 0 to differentiate FGP");
    cudaStream_t st = S(stream);
    const size_t img = (size_t)batch * n * n;
    if (iters == 0) {
        PNP_CUDA(launch_copy(d_xbar, d_zbar, img, st));
        if (h_lambar) for (int b = 0; b < batch; ++b) h_lambar[b] = 0.0;
        return PNP_OK;
    }
    if (!d_ws || ws_bytes < need) return fail(PNP_EINVAL, "VJP workspace needs %zu bytes", need);
    char* vws = (char*)d_ws;
    double* dres = (double*)(vws + need) - batch;
    if (int e = tv_vjp_core(d_z, d_xbar, d_zbar, n, batch, lambda, iters, vws, dres, st)) return e;
    if (h_lambar) {
        PNP_CUDA(cudaMemcpyAsync(h_lambar, dres, sizeof(double) * batch, cudaMemcpyDeviceToHost, st));
        PNP_CUDA(cudaStreamSynchronize(st));
    }
    return PNP_OK;
}

int pnp_vjp_workspace_size(const pnp_geom* g, int tv_iters, size_t* bytes)
{
    t_err.clear();
    if (int e = validate_geom(g)) return e;
    size_t tvb = 0;
    if (int e = pnp_tv_vjp_workspace_size(g->n, g->batch, tv_iters, &tvb)) return e;
    if (!bytes) return fail(PNP_EINVAL, "bytes pointer is NULL");
    *bytes = align_up(tvb) + 3 * align_up((size_t)g->batch * g->n * g->n * sizeof(float));
    return PNP_OK;
}

namespace {
int check_step(const pnp_geom* g, int factor, int subset, int n_subsets, double eta,
               const pnp_run_params* pr, Layout* L, int* li)
{
    if (int e = validate_geom(g)) return e;
    *L = make_layout(*g);
    if (int e = check_level(*g, factor, *L, li)) return e;
    if (int e = check_subset(*g, subset, n_subsets)) return e;
    if (!pr) return fail(PNP_EINVAL, "params are required");
    if (!(std::isfinite(eta) && eta >= 0.0)) return fail(PNP_EINVAL, "eta invalid");
    if (!(pr->alpha > 0.0f && pr->alpha <= 1.0f)) return fail(PNP_EINVAL, "alpha must be in (0, 1]");
    if (!(pr->lambda >= 0.0f) || !std::isfinite(pr->lambda)) return fail(PNP_EINVAL, "lambda must be >= 0");
    if (pr->tv_iters < 0 || pr->tv_iters > 10000) return fail(PNP_EINVAL, "tv_iters outside [0, 10000]");
    return PNP_OK;
}
}  // namespace

namespace {
// One unrolled iteration; z (the gradient step) is also copied to d_zout when given.
int unrolled_step_impl(const pnp_geom* g, int factor, int subset, int n_subsets, double eta,
                       const pnp_run_params* params, float amom, const float* d_y, const float* d_xprev,
                       const float* d_b, float* d_xout, float* d_yout, float* d_zout, void* d_ws, void* stream)
{
    t_err.clear();
    Layout L;
    int li = 0;
    if (int e = check_step(g, factor, subset, n_subsets, eta, params, &L, &li)) return e;
    if (!d_y || !d_xprev || !d_b || !d_xout || !d_yout) return fail(PNP_EINVAL, "y, xprev, b, xout, yout required");
    if (d_xout == d_y || d_yout == d_y || d_xout == d_yout || d_xout == d_xprev)
        return fail(PNP_EINVAL, "outputs must not alias the inputs or each other");
    if (d_zout && (d_zout == d_y || d_zout == d_xprev || d_zout == d_xout || d_zout == d_yout))
        return fail(PNP_EINVAL, "z output must not alias the other arguments");
    if (int e = check_ws(*g, d_ws)) return e;
    char* ws = (char*)d_ws;
    cudaStream_t st = S(stream);
    const size_t img = (size_t)g->batch * g->n * g->n;
    float* z = (float*)(ws + L.off_z);
    float* tvb = (float*)(ws + L.off_tv);
    if (int e = grad_into(*g, L, li, ws, d_y, d_b, subset, n_subsets, kBackStep, (float)eta, z, st)) return e;
    if (d_zout) PNP_CUDA(launch_copy(z, d_zout, img, st));
    PNP_CUDA(launch_copy(d_xprev, d_xout, img, st));
    const pnp_run_params& pr = *params;
    if (pr.tv_iters > 0 && pr.lambda > 0.0f)
        PNP_CUDA(launch_tv_tiled(z, g->n, g->batch, pr.lambda, pr.tv_iters, pr.alpha, amom, d_xout, d_yout,
                                 nullptr, nullptr, tvb, tvb + 4 * img, st));
    else
        PNP_CUDA(launch_tv_final(z, nullptr, 0, g->n, g->batch, pr.lambda, pr.alpha, amom, d_xout, d_yout,
                                 nullptr, nullptr, st));
    return PNP_OK;
}

// VJP of one unrolled iteration; z is recomputed from d_y, or taken from d_zsaved.
int unrolled_step_vjp_impl(const pnp_geom* g, int factor, int subset, int n_subsets, double eta,
                           const pnp_run_params* params, float amom, const float* d_y, const float* d_b,
                           const float* d_zsaved, const float* d_xbar, const float* d_ybar, float* d_ybar_in,
                           float* d_xpbar, double* h_lambar, void* d_ws, void* d_vjp_ws, size_t vjp_ws_bytes,
                           void* stream)
{
    t_err.clear();
    Layout L;
    int li = 0;
    if (int e = check_step(g, factor, subset, n_subsets, eta, params, &L, &li)) return e;
    if (!(d_zsaved || (d_y && d_b)) || !d_xbar || !d_ybar || !d_ybar_in || !d_xpbar)
        return fail(PNP_EINVAL, "z (or y and b), xbar, ybar, ybar_in, xpbar required");
    if (d_ybar_in == d_xpbar) return fail(PNP_EINVAL, "outputs must not alias");
    const pnp_run_params& pr = *params;
    const bool do_tv = pr.tv_iters > 0 && pr.lambda > 0.0f;
    size_t need = 0;
    if (int e = pnp_vjp_workspace_size(g, do_tv ? pr.tv_iters : 0, &need)) return e;
    if (!d_vjp_ws || vjp_ws_bytes < need) return fail(PNP_EINVAL, "VJP workspace needs %zu bytes", need);
    if (int e = check_ws(*g, d_ws)) return e;
    char* ws = (char*)d_ws;
    char* vws = (char*)d_vjp_ws;
    cudaStream_t st = S(stream);
    const size_t img = (size_t)g->batch * g->n * g->n;
    size_t tvb_bytes = 0;
    pnp_tv_vjp_workspace_size(g->n, g->batch, do_tv ? pr.tv_iters : 0, &tvb_bytes);
    float* X = (float*)(vws + align_up(tvb_bytes));
    float* DZ = (float*)((char*)X + align_up(img * sizeof(float)));
    float* ZB = (float*)((char*)DZ + align_up(img * sizeof(float)));
    double* dres = (double*)(vws + tvb_bytes) - g->batch;
    const float* z = d_zsaved;
    if (!z) {   // forward recomputation of z (per-iteration checkpoint: only y is kept)
        float* zw = (float*)(ws + L.off_z);
        if (int e = grad_into(*g, L, li, ws, d_y, d_b, subset, n_subsets, kBackStep, (float)eta, zw, st)) return e;
        z = zw;
    }
    // through y_i = (1 + a) x_i - a x_{i-1}
    PNP_CUDA(launch_axpby(d_xbar, 1.0f, d_ybar, 1.0f + amom, X, (long)img, st));
    PNP_CUDA(launch_axpby(d_ybar, -amom, nullptr, 0.0f, d_xpbar, (long)img, st));
    // through x_i = (1 - alpha) z + alpha D(z)
    if (do_tv) {
        if (int e = tv_vjp_core(z, X, DZ, g->n, g->batch, pr.lambda, pr.tv_iters, vws, dres, st)) return e;
    } else {
        PNP_CUDA(launch_copy(X, DZ, img, st));
    }
    PNP_CUDA(launch_axpby(X, 1.0f - pr.alpha, DZ, pr.alpha, ZB, (long)img, st));
    // through z = y - eta c S^T A_s^T (A_s S y - b): symmetric Jacobian
    if (int e = grad_into(*g, L, li, ws, ZB, nullptr, subset, n_subsets, kBackStep, (float)eta, d_ybar_in, st))
        return e;
    if (h_lambar) {
        if (do_tv) {
            std::vector<double> lb((size_t)g->batch);
            PNP_CUDA(cudaMemcpyAsync(lb.data(), dres, sizeof(double) * g->batch, cudaMemcpyDeviceToHost, st));
            PNP_CUDA(cudaStreamSynchronize(st));
            for (int b = 0; b < g->batch; ++b) h_lambar[b] = pr.alpha * lb[b];
        } else {
            for (int b = 0; b < g->batch; ++b) h_lambar[b] = 0.0;
        }
    }
    return PNP_OK;
}
}  // namespace

int pnp_unrolled_step(const pnp_geom* g, int factor, int subset, int n_subsets, double eta,
                      const pnp_run_params* params, float amom, const float* d_y, const float* d_xprev,
                      const float* d_b, float* d_xout, float* d_yout, void* d_ws, void* stream)
{
    return unrolled_step_impl(g, factor, subset, n_subsets, eta, params, amom, d_y, d_xprev, d_b, d_xout, d_yout,
                              nullptr, d_ws, stream);
}

int pnp_unrolled_step_save(const pnp_geom* g, int factor, int subset, int n_subsets, double eta,
                           const pnp_run_params* params, float amom, const float* d_y, const float* d_xprev,
                           const float* d_b, float* d_xout, float* d_yout, float* d_zout, void* d_ws,
                           void* stream)
{
    if (!d_zout) return fail(PNP_EINVAL, "z output required");
    return unrolled_step_impl(g, factor, subset, n_subsets, eta, params, amom, d_y, d_xprev, d_b, d_xout, d_yout,
                              d_zout, d_ws, stream);
}

int pnp_unrolled_step_vjp(const pnp_geom* g, int factor, int subset, int n_subsets, double eta,
                          const pnp_run_params* params, float amom, const float* d_y, const float* d_b,
                          const float* d_xbar, const float* d_ybar, float* d_ybar_in, float* d_xpbar,
                          double* h_lambar, void* d_ws, void* d_vjp_ws, size_t vjp_ws_bytes, void* stream)
{
    if (!d_y || !d_b) return fail(PNP_EINVAL, "y and b required");
    return unrolled_step_vjp_impl(g, factor, subset, n_subsets, eta, params, amom, d_y, d_b, nullptr, d_xbar,
                                  d_ybar, d_ybar_in, d_xpbar, h_lambar, d_ws, d_vjp_ws, vjp_ws_bytes, stream);
}

int pnp_unrolled_step_vjp_saved(const pnp_geom* g, int factor, int subset, int n_subsets, double eta,
                                const pnp_run_params* params, float amom, const float* d_z,
                                const float* d_xbar, const float* d_ybar, float* d_ybar_in, float* d_xpbar,
                                double* h_lambar, void* d_ws, void* d_vjp_ws, size_t vjp_ws_bytes,
                                void* stream)
{
    if (!d_z) return fail(PNP_EINVAL, "z required");
    return unrolled_step_vjp_impl(g, factor, subset, n_subsets, eta, params, amom, nullptr, nullptr, d_z, d_xbar,
                                  d_ybar, d_ybar_in, d_xpbar, h_lambar, d_ws, d_vjp_ws, vjp_ws_bytes, stream);
}

}  // extern "C"
