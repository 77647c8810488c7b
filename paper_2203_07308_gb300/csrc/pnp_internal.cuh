// Internal declarations shared by the translation units of libpnp_ms2g.so.
//
// Data layout in the caller's workspace (all offsets 256-byte aligned), per
// sketch level s in {1,2,4,8} with n % s == 0 and n/s >= 4:
//   rayf  float4 [n_views*n_det]  (F'_x, F'_y, d_x, d_y): foot point in the
//                                 primed frame (see below), unit direction
//   rayi  float2 [n_views*n_det]  (1/d_x, 1/d_y), clamped away from 0
//   rayk  int2   [n_views*n_det]  first/last sample index k inside the image box
//   view  float4 [n_views]        (cos b, sin b, dso/s, (dso+ddo)/pitch)
//   quad  float4 [batch][(n_s+3)^2] bilinear coefficients of the level image
// then the residual sinogram, the fine-grid loop buffers, the TV buffers, the
// power-iteration vectors and the FP64 reduction scratch.
//
// Index frame: level pixel (ix,iy) has centre index coordinate (ix,iy).  The
// kernels work in the primed frame X' = X - c0 + 1.5 with c0 = n_s/2: its
// origin sits at the image centre (coordinates stay below ~0.71 n_s, which
// halves FP32 position rounding against a corner origin), round(X') + c0 =
// floor(X) + 2 is the column of the 2-pixel-padded coefficient image, and
// X' - round(X') = frac(X) - 1/2.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <cstdint>

#include "../../include/pnp_ms2g.h"

#include <utility>

namespace pnp {

// Programmatic dependent launch.  The loop kernels (coefficient image, forward,
// backprojection, denoiser) are launched with programmatic stream serialisation:
// each one waits for its predecessor's completion (griddepcontrol.wait) before
// touching memory and then lets its own successor be scheduled
// (griddepcontrol.launch_dependents), so the successor's launch and CTA set-up
// overlap this kernel instead of following it.  PNP_PDL=0 in the environment
// launches them the ordinary way (the waits are then no-ops).
__device__ __forceinline__ void pdl_begin()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" :::);
}

bool pdl_enabled();
// PNP_FUSE_QUAD=0 keeps the coefficient-image kernel in every iteration
bool fuse_quad_enabled();

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args&&... args)
{
    if (!pdl_enabled()) {
        kernel<<<grid, block, smem, st>>>(std::forward<Args>(args)...);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}


// Persistent launches (PNP_RUN_PERSISTENT, set by pnp_run / pnp_run_many for the
// duration of the call on the calling thread): the phase kernels then launch in
// their persistent form, as many CTAs as fit on the GPU at once, each walking
// the phase's work table (class, instance, tile) with a stride of the grid.
bool persistent_mode();
void set_persistent_mode(bool on);
int device_sm_count();

// direct: one CTA per work item (grid = items); persistent: the same items walked
// by the CTAs that fit at once (occupancy x SMs), at most one per item
template <typename... KArgs, typename... Args>
cudaError_t launch_items(void (*direct)(KArgs...), void (*persistent)(KArgs...), dim3 grid, dim3 block, size_t smem,
                         cudaStream_t st, Args&&... args)
{
    if (!persistent_mode()) return launch_pdl(direct, grid, block, smem, st, std::forward<Args>(args)...);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent, (int)(block.x * block.y * block.z), smem) !=
            cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const long cap = (long)per_sm * device_sm_count();
    const dim3 pg((unsigned)((long)grid.x < cap ? (long)grid.x : cap), grid.y, grid.z);
    return launch_pdl(persistent, pg, block, smem, st, std::forward<Args>(args)...);
}

constexpr int kMaxLevels = 4;          // factors 1, 2, 4, 8
constexpr int kPad = 2;                // padding of the coefficient image

// Bilinear coefficients (c0, c1, c2, c3) of a cell with corner values a = I(x0,y0),
// b = I(x0+1,y0), c = I(x0,y0+1), d = I(x0+1,y0+1): f = c0 + u c1 + w (c2 + u c3)
// in the centred variables u, w in [-1/2, 1/2].  One definition for every kernel
// that writes the coefficient image, so they agree bit for bit.
__device__ __forceinline__ float4 make_quad(float a, float b, float c, float d)
{
    float4 q;
    q.x = 0.25f * ((a + b) + (c + d));
    q.y = 0.5f * ((b - a) + (d - c));
    q.z = 0.5f * ((c - a) + (d - b));
    q.w = (a - b) - (c - d);
    return q;
}
// FP64 partial-sum blocks per instance: a fixed count (not derived from the
// device) so that the order of every FP64 reduction, and its result, is the same
// on any GPU.
constexpr int kRedBlocks = 304;
constexpr int kRedThreads = 256;

extern std::atomic<uint64_t> g_launches;

struct LevelLayout {
    int factor = 0;   // 0: level not present
    int ns = 0;       // n / factor
    int qw = 0;       // ns + 3 (padded coefficient image side)
    size_t off_rayf = 0, off_rayi = 0, off_rayk = 0, off_view = 0, off_quad = 0;
};

struct Layout {
    LevelLayout lv[kMaxLevels];
    size_t off_res = 0;      // float [batch][n_views][n_det]
    size_t off_y = 0;        // float [batch][n][n]
    size_t off_z = 0;        // float [batch][n][n]
    size_t off_x2 = 0;       // float [2][batch][n][n]  second buffer of the iterate x (odd iterations);
                             // the autotuner's timed denoise uses both images
    size_t off_tv = 0;       // float [8][batch][n][n]  TV state ping/pong (r1 r2 p1 p2)
    size_t off_pw = 0;       // float [2][n][n]   power iteration u, w
    size_t off_cs = 0;       // float [2][batch][(n/2)^2] bicubic coarse image and coarse gradient
    size_t off_red = 0;      // double [batch][kRedBlocks] partials + [batch][8] results
    size_t off_log = 0;      // double [PNP_MAX_LOG_ITERS] (not used when batch grows; see api)
    size_t total = 0;
};

int level_index(int factor);   // 0..3 or -1

// Streaming multiprocessors of the current device (cached per device), for the
// launch-shape heuristics; 1 if the query fails.
int device_sm_count();

// Error reporting and geometry checks shared by the C entry points (api.cu):
// fail() records the message for pnp_last_error() and returns `code`.
int fail(int code, const char* fmt, ...);
void clear_error();
bool level_ok(const pnp_geom& g, int s);
int validate_geom(const pnp_geom* g);

// ---------------------------------------------------------------- kernels (launchers)
cudaError_t launch_setup_rays(const pnp_geom& g, const LevelLayout& L, char* ws, cudaStream_t st);

// Every projector and denoiser kernel takes a table of up to kMaxClasses
// geometry classes (each a uniform batch of images sharing one geometry) and
// covers all of them in one launch; the single-class launchers below are the
// one-entry case.  Autotuned launch shapes (0 = heuristic) ride along.
constexpr int kMaxClasses = 4;
// geometry classes of one pnp_run_many call (launched in groups of kMaxClasses)
constexpr int kMaxRunClasses = 1024;

// Coefficient images of a batch of at least kQuadIlMin images are stored
// image-interleaved, quad[(qy * qw + qx) * batch + image], so that one 128-byte
// line holds a cell of 8 images and the forward projector reads a sample of 8
// images with one line; smaller batches are stored image-major,
// quad[image][qy][qx].  Every writer and reader takes the layout from the batch.
constexpr int kQuadIlMin = 8;
__host__ __device__ inline bool quad_interleaved(int batch) { return batch >= kQuadIlMin; }

struct PrepArgs { const float* fine; int n, s, batch; float4* quad; int qw; };
cudaError_t launch_prep_quad(const float* fine, int n, int s, int batch, float4* quad, int qw,
                             cudaStream_t st);
cudaError_t launch_prep_multi(const PrepArgs* items, int count, cudaStream_t st);

struct FwdArgs {
    const float4* quad; int qw; size_t quad_stride;
    const float4* rayf; const int2* rayk;
    int n_det, first_view, view_step, n_sub, batch;
    float step, weight;
    const float* b; int n_views;     // b: [batch][n_views][n_det] or null
    float* out;                      // [batch][n_sub][n_det], or [n_sub][n_det][batch] with out_il
    const float* w;                  // null or weights [batch][n_views][n_det]: out = w (A x - b)
    int out_il = 0;                  // 1: image-interleaved output (a residual read by the backprojector)
};
cudaError_t launch_forward(const FwdArgs& a, cudaStream_t st, int lanes = 0);
cudaError_t launch_forward_multi(const FwdArgs* items, int count, cudaStream_t st, int lanes = 0);

enum BackMode { kBackRaw = 0, kBackGradFine = 1, kBackStep = 2 };
struct BackArgs {
    const float* res;                // [batch][n_sub][n_det], or [n_sub][n_det][batch] with res_il
    const float4* rayf; const float2* rayi; const float4* view; const int2* rayk;
    int ns, n_det, first_view, view_step, n_sub, batch;
    float step;
    int mode; int s; int n;          // fine side for modes 1, 2
    float scale;                     // multiplies the gathered sum
    const float* y; float eta;       // mode 2: z = y - eta * scale * sum
    float* out;
    float cmax = 0.0f;               // bound on the (ray, sample) terms one pixel receives from one
                                     // view (scatter form; 0: scatter unavailable, gather used)
    int res_il = 0;                  // 1: image-interleaved residual (written with FwdArgs::out_il)
    // stored gather table of this level (all views; null: none): hdr [n_views][groups] of
    // (first slot, slots), weights [slots][32], bins [slots][32]; groups = table_groups(ns)
    const int2* thdr = nullptr; const float4* tw = nullptr; const int* tray = nullptr;
};
// Residual strides: element (image, view row, bin) at image * is + (row * n_det + bin) * js.
__host__ __device__ inline long res_is(const BackArgs& a) { return a.res_il ? 1L : (long)a.n_sub * a.n_det; }
__host__ __device__ inline int res_js(const BackArgs& a) { return a.res_il ? a.batch : 1; }
// `groups`: view groups per CTA of the 2x2-block gather (1..16, 0 = heuristic),
// PNP_BACK_TILE4 | G for 4 x 4-block CTAs, or PNP_BACK_SCATTER | TS for the
// fixed-point scatter form on TS x TS tiles (TS in {12, 16, 22, 32}).
// PNP_BACK_BATCH(BC) | (gather shape) selects the batched gather (BC images per
// thread, BC in {4, 8, 16}; at most 512 threads per CTA).
// PNP_BACK_TABLE | PNP_BACK_BATCH(BC) | G reads the stored gather table (every
// class must have one; BC in {2, 4, 8, 16}, 2 when BC < 2) with G view groups.
inline int back_batch_of(int groups) { return (groups >> 16) & 0xff; }
cudaError_t launch_backward(const BackArgs& a, cudaStream_t st, int groups = 0);
cudaError_t launch_backward_multi(const BackArgs* items, int count, cudaStream_t st, int groups = 0);
// Gather table construction for one level (a: the level's ray tables; all n_views views):
// widths[view][group] = slots of each (view, group of 32 blocks), then the entries.
// groups of 32 blocks = tiles of 8 x 4 blocks (16 x 8 pixels), row-major; lane l of
// group k is the block (8 (k % tiles_x) + l % 8, 4 (k / tiles_x) + l / 8)
__host__ __device__ inline int table_groups(int ns) { const int nb = (ns + 1) / 2; return ((nb + 7) / 8) * ((nb + 3) / 4); }
__host__ __device__ inline void table_block(int ns, int k, int lane, int& bx, int& by)
{
    const int nb = (ns + 1) / 2, tx = (nb + 7) / 8;
    bx = 8 * (k % tx) + (lane & 7);
    by = 4 * (k / tx) + (lane >> 3);
}
cudaError_t launch_table_count(const BackArgs& a, int n_views, int* widths, cudaStream_t st);
cudaError_t launch_table_fill(const BackArgs& a, int n_views, const int2* hdr, float4* tw, int* tray,
                              cudaStream_t st);

cudaError_t launch_pool(const float* fine, float* coarse, int n, int s, int batch, cudaStream_t st);
// Bicubic sketch (kind PNP_SKETCH_BICUBIC) and its adjoint: out = base - eta scale S^T g,
// or scale S^T g when base is null.
cudaError_t launch_bicubic_down(const float* fine, float* coarse, int n, int s, int batch, cudaStream_t st);
cudaError_t launch_bicubic_up(const float* g, const float* base, float* out, int n, int s, int batch,
                              float scale, float eta, cudaStream_t st);
cudaError_t launch_unpool(const float* coarse, float* fine, int n, int s, int batch, cudaStream_t st);

// TV (FGP) --------------------------------------------------------------------
// x = z - lambda L(p) (or z when iters == 0), then relaxation and momentum:
//   xi = (1-alpha) z + alpha x;  y = xi + a (xi - x_{i-1});  xprev <- xi,
// x_{i-1} read from xin (nullptr: from xprev itself).
// With y == nullptr it writes x only (plain denoiser output to xprev).
// If mse_partials != nullptr, accumulates sum (xi - xtrue)^2 per block.
cudaError_t launch_tv_final(const float* z, const float* p, int have_p, int n, int batch, float lambda,
                            float alpha, float a, float* xprev, float* y, const float* xtrue,
                            double* mse_partials, cudaStream_t st, const float* xin = nullptr);

// Temporally blocked FGP: every iteration of the denoiser (iters >= 1) for all
// images, T x T tiles recomputing their halos (launch_tv_tiled chains launches
// of at most 10 iterations through state_a / state_b, each [4][batch][n][n]
// floats).  Then x, the relaxation and momentum as in launch_tv_final; mse
// partials [batch][tile_tv_parts].
constexpr int kTileMaxK = 20;
int tile_tv_tile(int n, int batch);
int tile_tv_parts(int n, int batch);
cudaError_t launch_tv_tiled(const float* z, int n, int batch, float lambda, int iters, float alpha,
                            float amom, float* xprev, float* y, const float* xtrue, double* mse_part,
                            float* state_a, float* state_b, cudaStream_t st, int tile = 0);
// TvItem::tile: 0 = cost model, 8..40 = shared-memory tiles of that side,
// kTvTileWarp = register-resident warp tiles, kTvTileStrip8 / 12 / 16 =
// register-resident strips of 64 columns x 64 / 96 / 128 rows (8 / 12 / 16 warps
// per CTA) (the first item decides the variant).
constexpr int kTvTileWarp = 1;
constexpr int kTvTileStrip8 = 2;
constexpr int kTvTileStrip12 = 3;
constexpr int kTvTileStrip16 = 4;
inline bool tv_is_strip(int tile) { return tile >= kTvTileStrip8 && tile <= kTvTileStrip16; }
inline int tv_strip_warps(int tile) { return tile == kTvTileStrip8 ? 8 : tile == kTvTileStrip12 ? 12 : 16; }
// the denoiser family of a tile code: 0 shared-memory tiles, 1 warp tiles, 2 strips
inline int tv_family(int tile) { return tile == kTvTileWarp ? 1 : tv_is_strip(tile) ? 2 : 0; }
struct TvItem {
    const float* z; float* xprev; float* y; const float* xtrue; double* mse_part;
    float* state_a; float* state_b;        // [4][batch][n][n] each (chained launches only)
    int n, batch, tile;
    float amom;
    const float* xin = nullptr;            // x_{i-1} when it is not xprev (double-buffered x)
    float4* quad = nullptr;                // shared-memory tiles only: also write the coefficient
    int qw = 0;                            // image of S_qs y (qw = n/qs + 2 kPad - 1), qs = 1 or 2
    int qs = 1;                            // (2: pooled; needs an even tile side and n)
};
cudaError_t launch_tv_tiled_multi(const TvItem* items, int count, float lambda, int iters, float alpha,
                                  cudaStream_t st);
int tile_tv_parts_for(int n, int batch, int tile);
// whether the shared-memory tiles' last launch can write the coefficient image of
// S_qs y (qs = 1 always; qs = 2 for an even tile side and n); never for tile = 1
bool tv_fuses_quad(int tile, int n, int batch, int qs);

// Reverse mode (vjp.cu) ----------------------------------------------------------
size_t tv_vjp_workspace_floats(int n, int batch, int iters);
size_t tv_vjp_partials(int n);
// zbar = d<xbar, FGP(z)>/dz; partials[batch][tv_vjp_partials] accumulate dJ/dlambda.
cudaError_t launch_tv_vjp(const float* z, const float* xbar, float* zbar, double* partials, int n,
                          int batch, float lambda, int iters, float* ws, cudaStream_t st);
cudaError_t launch_axpby(const float* a, float c1, const float* b, float c2, float* out, long count,
                         cudaStream_t st);

// Variance-reduced subset estimates (vr.cu) ----------------------------------------
// phi = sum over P planes of `count` values (fixed order).
cudaError_t launch_vr_table_sum(const float* table, int P, long count, float* phi, cudaStream_t st);
// est 1: v = c G + acc; est 2: v = c (G - Tp) + acc, acc += G - Tp, Tp = G.  Level grid
// [batch][ns][ns].  v_out (nullable) receives v; z (nullable) receives y - eta v / s^2
// replicated over each s x s block (the pooled sketch's U = S^T).
cudaError_t launch_vr_combine(int est, const float* G, float* acc, float* Tp, float c, int ns, int batch,
                              float* v_out, const float* y, float* z, int s, float eta, cudaStream_t st);

// Reductions -------------------------------------------------------------------
enum RedMode { kRedDot = 0, kRedDiffSq = 1, kRedSq = 2, kRedTv = 3, kRedWSq = 4 };   // kRedWSq: sum b a^2
// partials[inst][kRedBlocks] for `count` elements per instance (stride `stride`).
cudaError_t launch_reduce_partial(int mode, const float* a, const float* b, size_t count,
                                  size_t stride, int batch, int n, double* partials, cudaStream_t st);
// out[inst * out_stride + out_off] = sum_k partials[inst][k] (fixed order).
cudaError_t launch_reduce_final(const double* partials, int nparts, int batch, double* out,
                                int out_stride, int out_off, cudaStream_t st);
// u = w * factor, where factor = 1 / sqrt(norm2[0]) (device scalar).
cudaError_t launch_scale_by_rnorm(const float* w, float* u, size_t count, const double* norm2,
                                  cudaStream_t st);
cudaError_t launch_fill(float* x, size_t count, float v, cudaStream_t st);
cudaError_t launch_fill_hash(float* x, size_t count, float lo, float hi, cudaStream_t st);
cudaError_t launch_copy(const float* src, float* dst, size_t count, cudaStream_t st);
cudaError_t launch_count_samples(const int2* rayk, int n_det, int first_view, int view_step,
                                 int n_sub, double* partial, cudaStream_t st);

}  // namespace pnp
