// TV-prox denoiser D(z) = argmin 1/2||x - z||^2 + lambda TV_iso(x) by FGP
// (Beck & Teboulle 2009, the paper's reference for the TV prox; the paper
// lists TV-prox among valid denoisers right after Eq. 5), fused with the
// RED-PRO relaxation and FISTA momentum of Alg. 1.
//
// Dual pair (p, q) on the n x n grid: p pairs rows i, i+1 (zero on the last
// row), q pairs columns j, j+1 (zero on the last column).
//   L(p,q)[i][j] = p[i][j] + q[i][j] - p[i-1][j] - q[i][j-1]
//   L^T(x)       = (x[i][j] - x[i+1][j], x[i][j] - x[i][j+1])
// Iteration k:  (p_k, q_k) = Proj[(r_k, s_k) + L^T(z - lambda L(r_k, s_k)) / (8 lambda)]
//               (r_{k+1}, s_{k+1}) = (p_k, q_k) + m_k ((p_k, q_k) - (p_{k-1}, q_{k-1}))
// with Proj the isotropic projection onto unit disks and m_k = (t_k - 1)/t_{k+1}.
// Output x = z - lambda L(p_N, q_N).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "pnp_internal.cuh"


namespace pnp {
namespace {

__host__ __device__ inline int div_up(long a, long b) { return (int)((a + b - 1) / b); }

// Scale of the isotropic projection onto the unit disc, min(1, 1/|a|), from
// |a|^2: PTX rsqrt.approx with subnormal inputs flushed.  For normal inputs it
// gives the bits rsqrtf gives (rsqrtf only adds a rescaling of subnormal
// inputs); a subnormal or zero |a|^2 gives +inf where rsqrtf gives a value
// above 2^63, and the min makes both 1.  NaN stays NaN in both, so the min is 1.
__device__ __forceinline__ float proj_scale(float nrm2)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(nrm2));
    return fminf(1.0f, r);
}

__global__ void k_tv_final(const float* __restrict__ z, const float* __restrict__ p, int have_p,
                           int n, long plane, float lambda, float alpha, float amom,
                           float* __restrict__ xprev, float* __restrict__ y,
                           const float* __restrict__ xtrue, double* __restrict__ mse_part,
                           const float* __restrict__ xin)
{
    pdl_begin();
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    const int inst = blockIdx.z;
    const long img = (long)inst * n * n;
    double e2 = 0.0;
    if (i < n && j < n) {
        const long o = img + (long)i * n + j;
        const float zz = __ldg(z + o);
        float x = zz;
        if (have_p) {
            float l = __ldg(p + o) + __ldg(p + plane + o);
            if (i > 0) l -= __ldg(p + o - n);
            if (j > 0) l -= __ldg(p + plane + o - 1);
            x = zz - lambda * l;
        }
        const float xi = (1.0f - alpha) * zz + alpha * x;
        if (y) {
            const float xp = xin ? xin[o] : xprev[o];
            y[o] = xi + amom * (xi - xp);
        }
        xprev[o] = xi;
        if (xtrue) {
            const double d = (double)xi - (double)__ldg(xtrue + o);
            e2 = d * d;
        }
    }
    if (mse_part) {
        // block sum in a fixed order: warp shuffles, then warp 0
        __shared__ double sh[32];
        for (int off = 16; off > 0; off >>= 1) e2 += __shfl_xor_sync(0xffffffffu, e2, off);
        const int tid = threadIdx.y * blockDim.x + threadIdx.x;
        if ((tid & 31) == 0) sh[tid >> 5] = e2;
        __syncthreads();
        if (tid < 32) {
            const int nw = (blockDim.x * blockDim.y) >> 5;
            double v = tid < nw ? sh[tid] : 0.0;
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (tid == 0)
                mse_part[(long)inst * gridDim.x * gridDim.y + blockIdx.y * gridDim.x + blockIdx.x] = v;
        }
    }
}

// ------------------------------------------------------------------ temporally blocked FGP
// K FGP iterations of a T x T output tile in one CTA, with no communication
// between CTAs: an iteration's dual update at (i, j) reads the momentum point
// r only at Chebyshev distance <= 1, so K iterations on the tile need the
// state on the tile grown by K pixels on every side (plus one row above and one
// column to the left for the final x = z - lambda L(p)).  The CTA loads that
// region once and recomputes the shrinking halo itself; every value it keeps
// is computed by exactly the arithmetic a global iteration would use, so the
// result does not depend on the tiling.  Regions are clipped to the image,
// where the stencil's edge rules apply.
//   R_k (k = 0..K): [i0 - 1 - (K - k), i0 + T + (K - k)) in rows and columns
//   iteration k:  x_tmp on R_k grown by one row/column below/right, from r on
//                 R_{k-1};  then p, r on R_k.
// Launches of K <= kTileMaxK iterations are chained through the state buffers
// (r and p of every tile) when the denoiser needs more iterations.
struct TileTvClass {
    const float* z; const float* sin; float* sout;   // state planes [4][batch][n][n]: r1 r2 p1 p2
    float* xprev; float* y; const float* xtrue; double* mse_part;
    const float* xin;                                 // x_{i-1} (nullptr: xprev)
    float4* quad;                                     // last launch: coefficient image of S_qs y
    int qw, qs, ring;                                 // qs = 1 or 2; ring = qs when quad is written
    int qbatch;                                       // batch of the class (sets the image layout)
    int n, T, tiles_x, tiles;
    long plane;
    float amom;
};

struct TileTvArgs {
    TileTvClass c[kMaxClasses];
    long begin[kMaxClasses + 1];                      // cumulative CTA counts (batch * tiles)
    int count, K, first, last;
    float lambda, alpha;
    float mom[kTileMaxK];
};

// Row stride of the shared arrays, one constant for every region side (S <= 64
// with at most four pixels per thread): congruent to 8 mod 32, so that rows sit
// on distinct bank offsets, and known at compile time, so that the neighbour
// offsets +-1 and +-P fold into the shared-memory instructions.
constexpr int kTilePitch = 72;

// Thread t owns the region pixels with flat index t, t + 1024, ... (NP of
// them) for the whole launch: their z, r and p stay in registers together with
// the pixel's shared-memory offset and two Chebyshev distances that decide in
// which iterations it is inside the shrinking regions.  Shared memory holds
// only what neighbours read: r (phase A; zero outside the image, so that the
// edge rule of L needs no test there), x_tmp (phase B) and, at the end, p.
template <int NP, bool LAST>
__device__ __forceinline__ void k_tv_tile_item(const TileTvArgs& t, const long vb)
{
    int cls = 0;
#pragma unroll
    for (int k = 1; k < kMaxClasses; ++k)
        if (k < t.count && (long)vb >= t.begin[k]) cls = k;
    const TileTvClass& a = t.c[cls];
    const int n = a.n, K = t.K, T = a.T;
    const int tiles_x = a.tiles_x;
    const long local = (long)vb - t.begin[cls];
    const int inst = (int)(local / a.tiles);
    const int tile = (int)(local - (long)inst * a.tiles);
    const int i0 = (tile / tiles_x) * T, j0 = (tile % tiles_x) * T;
    // with ring = 1 or 2 the region (and every R_k) reaches that many rows and
    // columns further below/right, so that y is also known on the ring around the tile
    const int ring = a.ring;
    const int S = T + 1 + 2 * K + ring;          // side of the loaded region
    constexpr int P = kTilePitch;
    const int oi = i0 - 1 - K, oj = j0 - 1 - K;  // its origin (may lie outside the image)
    extern __shared__ float sm[];
    float2* rr = reinterpret_cast<float2*>(sm);          // (r1, r2)   [S][P]
    float* xt = sm + 2 * S * P;                           // x_tmp      [S][P]
    float2* pp = reinterpret_cast<float2*>(sm + 3 * S * P);   // (p1, p2), final step only
    const long img = (long)inst * n * n;
    const float lam = t.lambda, inv8l = 1.0f / (8.0f * t.lambda);
    constexpr int kFar = 1 << 20;

    float z[NP], r1[NP], r2[NP], p1[NP], p2[NP];
    int q[NP], dA[NP], dB[NP], flags[NP];
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        const int f = threadIdx.x + m * blockDim.x;
        const int li = f / S, lj = f - li * S;
        const int i = oi + li, j = oj + lj;
        q[m] = li * P + lj;
        z[m] = r1[m] = r2[m] = p1[m] = p2[m] = 0.0f;
        flags[m] = 0;
        dA[m] = dB[m] = kFar;
        if (f < S * S && i >= 0 && i < n && j >= 0 && j < n) {
            // distance outside the core of R_k ([i0-1, i0+T) x [j0-1, j0+T)) and of
            // the phase-A region (core grown by one row below, one column right)
            dB[m] = max(max(i0 - 1 - i, i - (i0 + T - 1 + ring)), max(max(j0 - 1 - j, j - (j0 + T - 1 + ring)), 0));
            dA[m] = max(max(i0 - 1 - i, i - (i0 + T + ring)), max(max(j0 - 1 - j, j - (j0 + T + ring)), 0));
            flags[m] = (i > 0 ? 1 : 0) | (j > 0 ? 2 : 0) | (i < n - 1 ? 4 : 0) | (j < n - 1 ? 8 : 0) |
                       (i >= i0 && i < i0 + T && j >= j0 && j < j0 + T ? 16 : 0);
            const long g = img + (long)i * n + j;
            z[m] = __ldg(a.z + g);
            if (!t.first) {
                r1[m] = __ldg(a.sin + g);
                r2[m] = __ldg(a.sin + a.plane + g);
                p1[m] = __ldg(a.sin + 2 * a.plane + g);
                p2[m] = __ldg(a.sin + 3 * a.plane + g);
            }
        }
        if (f < S * S) rr[q[m]] = make_float2(r1[m], r2[m]);
    }
    __syncthreads();
    for (int k = 1; k <= K; ++k) {
        const int mg = K - k;
        float x0[NP];
        // phase A: x_tmp = z - lambda L(r)
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            x0[m] = 0.0f;
            if (dA[m] <= mg) {
                float l = r1[m] + r2[m];
                l -= rr[q[m] - P].x;
                l -= rr[q[m] - 1].y;
                x0[m] = z[m] - lam * l;
                xt[q[m]] = x0[m];
            }
        }
        __syncthreads();
        // phase B: dual step, isotropic projection, momentum
        const float mo = t.mom[k - 1];
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            if (dB[m] <= mg) {
                const float g1 = (flags[m] & 4) ? x0[m] - xt[q[m] + P] : 0.0f;
                const float g2 = (flags[m] & 8) ? x0[m] - xt[q[m] + 1] : 0.0f;
                float pa = fmaf(g1, inv8l, r1[m]);
                float pc = fmaf(g2, inv8l, r2[m]);
                // projection onto the unit disc: scale min(1, 1/|a|) without a branch
                const float nrm2 = fmaf(pa, pa, pc * pc);
                const float sc = proj_scale(nrm2);
                pa *= sc;
                pc *= sc;
                r1[m] = fmaf(mo, pa - p1[m], pa);
                r2[m] = fmaf(mo, pc - p2[m], pc);
                p1[m] = pa;
                p2[m] = pc;
                rr[q[m]] = make_float2(r1[m], r2[m]);
            }
        }
        __syncthreads();
    }
    if constexpr (!LAST) {
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            if (flags[m] & 16) {
                const int f = threadIdx.x + m * blockDim.x;
                const int li = f / S, lj = f - li * S;
                const long g = img + (long)(oi + li) * n + (oj + lj);
                a.sout[g] = r1[m];
                a.sout[a.plane + g] = r2[m];
                a.sout[2 * a.plane + g] = p1[m];
                a.sout[3 * a.plane + g] = p2[m];
            }
        }
    } else {
        // x = z - lambda L(p) on the tile (and its ring), relaxation, momentum, squared error
#pragma unroll
        for (int m = 0; m < NP; ++m)
            if (dB[m] == 0) pp[q[m]] = make_float2(p1[m], p2[m]);
        __syncthreads();
        double e2 = 0.0;
        float* ys = xt;                     // y on the tile and its ring, for the coefficient image
        // every x_{i-1} load of this thread is issued before its first store (the
        // stores could alias the loads for the compiler, which would serialise them)
        float xpv[NP];
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            const int f = threadIdx.x + m * blockDim.x;
            const int li = f / S, lj = f - li * S;
            const int i = oi + li, j = oj + lj;
            const bool own = flags[m] & 16;
            const bool rim = ring && f < S * S && !own && i >= i0 && j >= j0 && i < i0 + T + ring &&
                             j < j0 + T + ring && i < n && j < n;
            xpv[m] = 0.0f;
            if (a.y && (own || rim)) {
                const long g = img + (long)i * n + j;
                xpv[m] = a.xin ? a.xin[g] : a.xprev[g];
            }
        }
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            const int f = threadIdx.x + m * blockDim.x;
            const int li = f / S, lj = f - li * S;
            const int i = oi + li, j = oj + lj;
            const bool own = flags[m] & 16;
            const bool rim = ring && f < S * S && !own && i >= i0 && j >= j0 && i < i0 + T + ring &&
                             j < j0 + T + ring && i < n && j < n;
            if (own || rim) {
                float l = p1[m] + p2[m];
                if (flags[m] & 1) l -= pp[q[m] - P].x;
                if (flags[m] & 2) l -= pp[q[m] - 1].y;
                const float x = z[m] - lam * l;
                const float xi = (1.0f - t.alpha) * z[m] + t.alpha * x;
                const long g = img + (long)i * n + j;
                float yv = 0.0f;
                if (a.y) yv = xi + a.amom * (xi - xpv[m]);
                if (own) {
                    if (a.y) a.y[g] = yv;
                    a.xprev[g] = xi;
                    if (a.xtrue) {
                        const double d = (double)xi - (double)__ldg(a.xtrue + g);
                        e2 += d * d;
                    }
                }
                if (ring) ys[q[m]] = yv;
            }
        }
        if (ring) {
            // coefficient cells of the level-qs image whose lower corner lies in the
            // tile; the first tiles of a row/column also take the padding cells before
            // the image, the last ones the cell after it (corners outside are zero).
            // Level pixel (r, c) is the qs x qs average of y, summed in the order of
            // the separate coefficient-image kernel, so the two agree bit for bit.
            __syncthreads();
            const int qs = a.qs, ns = n / qs;
            const int r_lo = i0 == 0 ? -kPad : i0 / qs, r_hi = i0 + T >= n ? ns + 1 : (i0 + T) / qs;
            const int c_lo = j0 == 0 ? -kPad : j0 / qs, c_hi = j0 + T >= n ? ns + 1 : (j0 + T) / qs;
            const int cw = c_hi - c_lo, cells = (r_hi - r_lo) * cw;
            // image-major, or image-interleaved for large batches (quad_interleaved)
            const int qB = a.qbatch;
            const bool qil = quad_interleaved(qB);
            float4* qimg = qil ? a.quad + inst : a.quad + (long)inst * a.qw * a.qw;
            const long qstride = qil ? qB : 1;
            auto inside = [&](int r, int c) { return r >= 0 && c >= 0 && r < ns && c < ns; };
            if (qs == 1) {
                auto Y = [&](int r, int c) -> float { return inside(r, c) ? ys[(r - oi) * P + (c - oj)] : 0.0f; };
                for (int k = threadIdx.x; k < cells; k += blockDim.x) {
                    const int r = r_lo + k / cw, c = c_lo + k % cw;
                    qimg[((long)(r + kPad) * a.qw + (c + kPad)) * qstride] =
                        make_quad(Y(r, c), Y(r, c + 1), Y(r + 1, c), Y(r + 1, c + 1));
                }
            } else {
                auto Y = [&](int r, int c) -> float {
                    if (!inside(r, c)) return 0.0f;
                    const float* p0 = ys + (2 * r - oi) * P + (2 * c - oj);
                    float acc = 0.0f;
                    acc += p0[0];
                    acc += p0[1];
                    acc += p0[P];
                    acc += p0[P + 1];
                    return acc * 0.25f;
                };
                for (int k = threadIdx.x; k < cells; k += blockDim.x) {
                    const int r = r_lo + k / cw, c = c_lo + k % cw;
                    qimg[((long)(r + kPad) * a.qw + (c + kPad)) * qstride] =
                        make_quad(Y(r, c), Y(r, c + 1), Y(r + 1, c), Y(r + 1, c + 1));
                }
            }
        }
        if (a.mse_part) {
            __shared__ double red[32];
            for (int off = 16; off > 0; off >>= 1) e2 += __shfl_xor_sync(0xffffffffu, e2, off);
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e2;
            __syncthreads();
            if (threadIdx.x == 0) {
                double v = 0.0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
                a.mse_part[(long)inst * a.tiles + tile] = v;
            }
        }
    }
}

template <int NP, bool LAST>
__global__ void __launch_bounds__(1024) k_tv_tile(const TileTvArgs t)
{
    pdl_begin();
    k_tv_tile_item<NP, LAST>(t, (long)blockIdx.x);
}

// persistent form (PNP_RUN_PERSISTENT): as many CTAs as fit at once walk the items
template <int NP, bool LAST>
__global__ void __launch_bounds__(1024) k_tv_tile_persistent(const TileTvArgs t)
{
    pdl_begin();
    const long total = t.begin[t.count];
    for (long vb = blockIdx.x; vb < total; vb += gridDim.x) {
        if (vb != (long)blockIdx.x) __syncthreads();   // the previous item's shared memory is free
        k_tv_tile_item<NP, LAST>(t, vb);
    }
}

// ------------------------------------------------------------------ register-resident FGP
// The same K-iteration temporal blocking with no shared memory and no barrier:
// a warp owns a tile of kWarpTvWV x kWarpTvHV output pixels; lane l holds one
// column of the loaded region (the tile grown by K + 1 above/left and K
// below/right) in registers, kWarpTvH rows deep.  Vertical neighbours are the
// lane's own registers, horizontal ones come from the adjacent lanes by warp
// shuffles; values outside the shrinking valid region are computed but never
// reach the output, exactly as in the shared-memory tiles.
constexpr int kWarpTvK = 5;                                  // FGP iterations per launch
constexpr int kWarpTvHV = 10;                                // output rows per warp tile
constexpr int kWarpTvH = kWarpTvHV + 2 * kWarpTvK + 1;       // rows held per lane
constexpr int kWarpTvWV = 31 - 2 * kWarpTvK;                 // output columns per warp tile
constexpr int kWarpTvWarps = 1;                              // warp tiles per CTA

struct WarpTvClass {
    const float* z; const float* sin; float* sout;          // state planes [4][batch][n][n]: r1 r2 p1 p2
    float* xprev; float* y; const float* xtrue; double* mse_part;
    const float* xin;                                        // x_{i-1} (nullptr: xprev)
    int n, tiles_x, tiles;
    long plane;
    float amom;
};

struct WarpTvArgs {
    WarpTvClass c[kMaxClasses];
    long begin[kMaxClasses + 1];                             // cumulative warp tiles (batch * tiles)
    int count, K, first, last;
    float lambda, alpha;
    float mom[kWarpTvK];
};

__device__ __forceinline__ void k_tv_warp_item(const WarpTvArgs& t, const long vb)
{
    constexpr int H = kWarpTvH;
    constexpr unsigned kAll = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long wt = (long)vb * kWarpTvWarps + (threadIdx.x >> 5);
    if (wt >= t.begin[t.count]) return;                      // whole warps only
    int cls = 0;
#pragma unroll
    for (int k = 1; k < kMaxClasses; ++k)
        if (k < t.count && wt >= t.begin[k]) cls = k;
    const WarpTvClass& a = t.c[cls];
    const long local = wt - t.begin[cls];
    const int inst = (int)(local / a.tiles);
    const int tile = (int)(local - (long)inst * a.tiles);
    const int n = a.n;
    const int r0 = (tile / a.tiles_x) * kWarpTvHV, c0 = (tile % a.tiles_x) * kWarpTvWV;
    const int j = c0 - kWarpTvK - 1 + lane;                  // this lane's column
    const int ib = r0 - kWarpTvK - 1;                        // row of register m = 0
    const bool jin = j >= 0 && j < n, jpos = j > 0, jlast = j < n - 1;
    const long img = (long)inst * n * n;
    float z[H], r1[H], r2[H], p1[H], p2[H];
#pragma unroll
    for (int m = 0; m < H; ++m) {
        const int i = ib + m;
        const bool in = jin && i >= 0 && i < n;
        const long g = img + (long)i * n + j;
        z[m] = in ? __ldg(a.z + g) : 0.0f;
        r1[m] = r2[m] = p1[m] = p2[m] = 0.0f;
        if (in && !t.first) {
            r1[m] = __ldg(a.sin + g);
            r2[m] = __ldg(a.sin + a.plane + g);
            p1[m] = __ldg(a.sin + 2 * a.plane + g);
            p2[m] = __ldg(a.sin + 3 * a.plane + g);
        }
    }
    const float lam = t.lambda, inv8l = 1.0f / (8.0f * t.lambda);
    for (int k = 0; k < t.K; ++k) {
        const float mo = t.mom[k];
        float xt[H];
        // x_tmp = z - lambda L(r)
#pragma unroll
        for (int m = 0; m < H; ++m) {
            const float left = __shfl_up_sync(kAll, r2[m], 1);
            float l = r1[m] + r2[m];
            if (m > 0 && ib + m > 0) l -= r1[m - 1];
            if (jpos) l -= left;
            xt[m] = z[m] - lam * l;
        }
        // dual step, isotropic projection, momentum
#pragma unroll
        for (int m = 0; m < H; ++m) {
            const float right = __shfl_down_sync(kAll, xt[m], 1);
            const float g1 = (m + 1 < H && ib + m < n - 1) ? xt[m] - xt[m + 1 < H ? m + 1 : m] : 0.0f;
            const float g2 = jlast ? xt[m] - right : 0.0f;
            float pa = fmaf(g1, inv8l, r1[m]);
            float pc = fmaf(g2, inv8l, r2[m]);
            // projection onto the unit disc: scale min(1, 1/|a|) without a branch
            const float nrm2 = fmaf(pa, pa, pc * pc);
            const float sc = proj_scale(nrm2);
            pa *= sc;
            pc *= sc;
            r1[m] = fmaf(mo, pa - p1[m], pa);
            r2[m] = fmaf(mo, pc - p2[m], pc);
            p1[m] = pa;
            p2[m] = pc;
        }
    }
    // the tile's output pixels: registers [K + 1, K + 1 + HV), lanes [K + 1, K + 1 + WV)
    const bool lane_out = lane >= kWarpTvK + 1 && lane < kWarpTvK + 1 + kWarpTvWV && jin;
    if (!t.last) {
#pragma unroll
        for (int m = kWarpTvK + 1; m < kWarpTvK + 1 + kWarpTvHV; ++m) {
            const int i = ib + m;
            if (lane_out && i < n) {
                const long g = img + (long)i * n + j;
                a.sout[g] = r1[m];
                a.sout[a.plane + g] = r2[m];
                a.sout[2 * a.plane + g] = p1[m];
                a.sout[3 * a.plane + g] = p2[m];
            }
        }
        return;
    }
    // x = z - lambda L(p) on the tile, relaxation, momentum, squared error; every
    // x_{i-1} load is issued before the first store (the stores could alias them)
    double e2 = 0.0;
    float xpv[kWarpTvHV];
#pragma unroll
    for (int m = kWarpTvK + 1; m < kWarpTvK + 1 + kWarpTvHV; ++m) {
        const int i = ib + m;
        const long g = img + (long)i * n + j;
        xpv[m - kWarpTvK - 1] = (a.y && lane_out && i < n) ? (a.xin ? a.xin[g] : a.xprev[g]) : 0.0f;
    }
#pragma unroll
    for (int m = kWarpTvK + 1; m < kWarpTvK + 1 + kWarpTvHV; ++m) {
        const float left = __shfl_up_sync(kAll, p2[m], 1);
        const int i = ib + m;
        if (lane_out && i < n) {
            float l = p1[m] + p2[m];
            if (i > 0) l -= p1[m - 1];
            if (jpos) l -= left;
            const float x = z[m] - lam * l;
            const float xi = (1.0f - t.alpha) * z[m] + t.alpha * x;
            const long g = img + (long)i * n + j;
            if (a.y) a.y[g] = xi + a.amom * (xi - xpv[m - kWarpTvK - 1]);
            a.xprev[g] = xi;
            if (a.xtrue) {
                const double d = (double)xi - (double)__ldg(a.xtrue + g);
                e2 += d * d;
            }
        }
    }
    if (a.mse_part) {
        for (int off = 16; off > 0; off >>= 1) e2 += __shfl_xor_sync(kAll, e2, off);
        if (lane == 0) a.mse_part[(long)inst * a.tiles + tile] = e2;
    }
}

__global__ void __launch_bounds__(32 * kWarpTvWarps) k_tv_warp(const WarpTvArgs t)
{
    pdl_begin();
    k_tv_warp_item(t, (long)blockIdx.x);
}

// persistent form (PNP_RUN_PERSISTENT): as many CTAs as fit at once walk the items
__global__ void __launch_bounds__(32 * kWarpTvWarps) k_tv_warp_persistent(const WarpTvArgs t)
{
    pdl_begin();
    const long total = (t.begin[t.count] + kWarpTvWarps - 1) / kWarpTvWarps;
    for (long vb = blockIdx.x; vb < total; vb += gridDim.x) {
        if (vb != (long)blockIdx.x) __syncthreads();   // the previous item's shared memory is free
        k_tv_warp_item(t, vb);
    }
}

// ------------------------------------------------------------------ register-resident FGP strips
// The same temporal blocking as the tiles above, organised so that almost every
// neighbour is in a register: a CTA owns a region of 64 columns x 8W rows (W
// warps stacked vertically, W = 8, 12 or 16), lane l of warp w holds columns 2l and 2l+1 of the
// warp's 8 rows (z in shared memory; r and p in registers).  Vertical
// neighbours inside a warp are the lane's own registers, horizontal ones the
// lane's other column or the adjacent lane's (one shuffle per row and phase);
// the rows where two warps meet go through a 64-float shared array per warp,
// once per phase.  K <= 10 iterations per launch; the output tile is the region
// minus K + 1 columns/rows on the left/top and K on the right/bottom.
// Edge rules without per-pixel tests: the dual step's differences are set to
// zero outside rows/columns [0, n-2], so p and r stay exactly zero on the last
// row/column and on everything above/left of the image, which is what L(p)
// subtracts there (the same values as the tests of the other variants give);
// other pixels outside the image hold values no output depends on.
constexpr int kStripK = 10;                                  // FGP iterations per launch (at most)
constexpr int kStripR = 8;                                   // rows per warp
constexpr int kStripWO = 64 - 2 * kStripK - 1;               // output columns per tile

struct StripTvClass {
    const float* z; const float* sin; float* sout;          // state [batch][n][n] of float4 (r1, r2, p1, p2)
    float* xprev; float* y; const float* xtrue; double* mse_part;
    const float* xin;                                        // x_{i-1} (nullptr: xprev)
    int n, tiles_x, tiles;
    long plane;
    float amom;
};

struct StripTvArgs {
    StripTvClass c[kMaxClasses];
    long begin[kMaxClasses + 1];                             // cumulative CTAs (batch * tiles)
    int count, K, first, last, W;
    float lambda, alpha;
    float mom[kStripK];
};

// Packed pairs (column 2l in .x, 2l+1 in .y): FP32x2 instructions, each lane
// rounded as the scalar operation would be (a - b as an exact -1 * b + a).
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }

// L2 eviction priorities for the strips' state between their launches: the
// first launch stores it evict-last (it is read back by the next launch while
// the image-sized buffers of the other phases stream through L2), the next
// launch reads it evict-first (dead after that read).  Cache hints only: the
// values are untouched.
__device__ __forceinline__ uint64_t l2_policy_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void st_hint(float4* a, float4 v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(a), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w), "l"(pol) : "memory");
}
__device__ __forceinline__ float4 ld_hint(const float4* a, uint64_t pol)
{
    float4 v;
    asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(a), "l"(pol));
    return v;
}

template <bool LAST, int W>
__device__ __forceinline__ void k_tv_strip_item(const StripTvArgs& t, const long vb)
{
    constexpr int R = kStripR;
    constexpr unsigned kAll = 0xffffffffu;
    const int lane = threadIdx.x, w = threadIdx.y;
    int cls = 0;
#pragma unroll
    for (int k = 1; k < kMaxClasses; ++k)
        if (k < t.count && (long)vb >= t.begin[k]) cls = k;
    const StripTvClass& a = t.c[cls];
    const long local = (long)vb - t.begin[cls];
    const int inst = (int)(local / a.tiles);
    const int tile = (int)(local - (long)inst * a.tiles);
    const int n = a.n;
    const int HO = W * R - 2 * kStripK - 1;                 // output rows per tile
    const int r0 = (tile / a.tiles_x) * HO, c0 = (tile % a.tiles_x) * kStripWO;
    const int rb = r0 - kStripK - 1 + w * R;                 // image row of register row 0
    const int ja = c0 - kStripK - 1 + 2 * lane, jb = ja + 1; // this lane's columns
    const long img = (long)inst * n * n;
    extern __shared__ float2 strip_sm[];
    float2* zs = strip_sm;                                   // [W * R][32]  (z of columns 2l, 2l+1)
    float2* up = zs + W * R * 32;                            // [W][32]      r1 of each warp's last row
    float2* dn = up + W * 32;                                // [W][32]      x_tmp of each warp's first row
    const bool ina = ja >= 0 && ja < n, inb = jb >= 0 && jb < n;
    // the dual step's differences vanish outside rows / columns [0, n-2]
    // (as the step 1/(8 lambda) of the difference, or 0: the same bits as the
    // difference times a 0/1 mask, then times 1/(8 lambda))
    const float inv8l = 1.0f / (8.0f * t.lambda);
    const float2 kcol = make_float2((ja >= 0 && ja < n - 1) ? inv8l : 0.0f, (jb >= 0 && jb < n - 1) ? inv8l : 0.0f);
    float krow[R];
    float2 r1[R], r2[R], p1[R], p2[R];
    const uint64_t polf = l2_policy_first();
#pragma unroll
    for (int m = 0; m < R; ++m) {
        const int i = rb + m;
        krow[m] = (i >= 0 && i < n - 1) ? inv8l : 0.0f;
        const bool ri = i >= 0 && i < n;
        const long g = img + (long)i * n;
        float2 z = make_float2(0.0f, 0.0f);
        r1[m] = r2[m] = p1[m] = p2[m] = z;
        const float4* sin4 = reinterpret_cast<const float4*>(a.sin);
        if (ri && ina) {
            z.x = __ldg(a.z + g + ja);
            if (!t.first) {
                const float4 q = ld_hint(sin4 + g + ja, polf);
                r1[m].x = q.x; r2[m].x = q.y; p1[m].x = q.z; p2[m].x = q.w;
            }
        }
        if (ri && inb) {
            z.y = __ldg(a.z + g + jb);
            if (!t.first) {
                const float4 q = ld_hint(sin4 + g + jb, polf);
                r1[m].y = q.x; r2[m].y = q.y; p1[m].y = q.z; p2[m].y = q.w;
            }
        }
        zs[(w * R + m) * 32 + lane] = z;
    }
    up[w * 32 + lane] = r1[R - 1];
    __syncthreads();
    const float lam = t.lambda;
    const float2 nlam2 = make_float2(-lam, -lam);
    const int wup = w > 0 ? w - 1 : 0, wdn = w + 1 < W ? w + 1 : w;
#pragma unroll 2
    for (int k = 0; k < t.K; ++k) {
        // x_tmp = z - lambda L(r):  L = ((r1 + r2) - r1_up) - r2_left
        float2 x[R];
        {
            float2 u = up[wup * 32 + lane];
#pragma unroll
            for (int m = 0; m < R; ++m) {
                const float2 left = make_float2(__shfl_up_sync(kAll, r2[m].y, 1), r2[m].x);
                float2 l = __fadd2_rn(r1[m], r2[m]);
                l = sub2(l, u);
                l = sub2(l, left);
                x[m] = __ffma2_rn(nlam2, l, zs[(w * R + m) * 32 + lane]);
                u = r1[m];
            }
        }
        dn[w * 32 + lane] = x[0];
        __syncthreads();
        // dual step, isotropic projection, momentum
        const float2 mo = make_float2(t.mom[k], t.mom[k]);
        {
            const float2 d = dn[wdn * 32 + lane];
#pragma unroll
            for (int m = 0; m < R; ++m) {
                const float2 down = m + 1 < R ? x[m + 1 < R ? m + 1 : m] : d;
                const float2 right = make_float2(x[m].y, __shfl_down_sync(kAll, x[m].x, 1));
                float2 pa = __ffma2_rn(sub2(x[m], down), make_float2(krow[m], krow[m]), r1[m]);
                float2 pc = __ffma2_rn(sub2(x[m], right), kcol, r2[m]);
                const float2 nrm2 = __ffma2_rn(pa, pa, __fmul2_rn(pc, pc));
                // projection onto the unit disc without a branch: scale min(1, 1/|a|)
                // (1 for |a| <= 1 up to the last bit of rsqrt at |a| = 1; inf at 0 gives 1)
                const float2 sc = make_float2(proj_scale(nrm2.x), proj_scale(nrm2.y));
                pa = __fmul2_rn(pa, sc);
                pc = __fmul2_rn(pc, sc);
                r1[m] = __ffma2_rn(mo, sub2(pa, p1[m]), pa);
                r2[m] = __ffma2_rn(mo, sub2(pc, p2[m]), pc);
                p1[m] = pa;
                p2[m] = pc;
            }
        }
        up[w * 32 + lane] = r1[R - 1];
        __syncthreads();
    }
    // output pixels of this thread: rows [r0, r0 + HO), columns [c0, c0 + WO), inside the image
    const bool oa = ina && ja >= c0 && ja < c0 + kStripWO, ob = inb && jb >= c0 && jb < c0 + kStripWO;
    if constexpr (!LAST) {
        const uint64_t pol = l2_policy_last();
#pragma unroll
        for (int m = 0; m < R; ++m) {
            const int i = rb + m;
            if (i < r0 || i >= r0 + HO || i >= n) continue;
            const long g = img + (long)i * n;
            float4* sout4 = reinterpret_cast<float4*>(a.sout);
            if (oa) st_hint(sout4 + g + ja, make_float4(r1[m].x, r2[m].x, p1[m].x, p2[m].x), pol);
            if (ob) st_hint(sout4 + g + jb, make_float4(r1[m].y, r2[m].y, p1[m].y, p2[m].y), pol);
        }
    } else {
        // x = z - lambda L(p), relaxation, momentum, squared error.  All of this
        // thread's x values are formed and all its x_{i-1} loads issued before the
        // first store (the stores could alias the loads for the compiler, which
        // would otherwise serialise sixteen round trips to memory).
        up[w * 32 + lane] = p1[R - 1];
        __syncthreads();
        float2 u = up[wup * 32 + lane];
        float2 xv[R];
#pragma unroll
        for (int m = 0; m < R; ++m) {
            const float2 left = make_float2(__shfl_up_sync(kAll, p2[m].y, 1), p2[m].x);
            float2 l = __fadd2_rn(p1[m], p2[m]);
            l = sub2(l, u);
            l = sub2(l, left);
            xv[m] = __ffma2_rn(nlam2, l, zs[(w * R + m) * 32 + lane]);
            u = p1[m];
        }
        const float* __restrict__ xold = a.xin ? a.xin : a.xprev;
        float2 xo[R];
#pragma unroll
        for (int m = 0; m < R; ++m) {
            const int i = rb + m;
            const bool row = i >= r0 && i < r0 + HO && i < n;
            const long g = img + (long)(row ? i : 0) * n;
            xo[m] = make_float2(0.0f, 0.0f);
            if (a.y && row && oa) xo[m].x = xold[g + ja];
            if (a.y && row && ob) xo[m].y = xold[g + jb];
        }
        double e2 = 0.0;
#pragma unroll
        for (int m = 0; m < R; ++m) {
            const int i = rb + m;
            if (i < r0 || i >= r0 + HO || i >= n) continue;
            const long g = img + (long)i * n;
            const float2 z2 = zs[(w * R + m) * 32 + lane];
            const float xva[2] = {xv[m].x, xv[m].y};
            const float xpa[2] = {xo[m].x, xo[m].y};
            const float zv[2] = {z2.x, z2.y};
            const bool ov[2] = {oa, ob};
            const int jv[2] = {ja, jb};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (!ov[h]) continue;
                const long gg = g + jv[h];
                const float xi = (1.0f - t.alpha) * zv[h] + t.alpha * xva[h];
                if (a.y) a.y[gg] = xi + a.amom * (xi - xpa[h]);
                a.xprev[gg] = xi;
                if (a.xtrue) {
                    const double dd = (double)xi - (double)__ldg(a.xtrue + gg);
                    e2 += dd * dd;
                }
            }
        }
        if (a.mse_part) {
            __shared__ double red[16];
            for (int off = 16; off > 0; off >>= 1) e2 += __shfl_xor_sync(kAll, e2, off);
            if (lane == 0) red[w] = e2;
            __syncthreads();
            if (w == 0 && lane == 0) {
                double v = 0.0;
                for (int q = 0; q < W; ++q) v += red[q];
                a.mse_part[(long)inst * a.tiles + tile] = v;
            }
        }
    }
}

template <bool LAST, int W>
__global__ void __launch_bounds__(32 * W, W == 8 ? 2 : 1) k_tv_strip(const StripTvArgs t)   // W = 8, 12 or 16
{
    pdl_begin();
    k_tv_strip_item<LAST, W>(t, (long)blockIdx.x);
}

// persistent form (PNP_RUN_PERSISTENT): as many CTAs as fit at once walk the items
template <bool LAST, int W>
__global__ void __launch_bounds__(32 * W, W == 8 ? 2 : 1) k_tv_strip_persistent(const StripTvArgs t)
{
    pdl_begin();
    const long total = t.begin[t.count];
    for (long vb = blockIdx.x; vb < total; vb += gridDim.x) {
        if (vb != (long)blockIdx.x) __syncthreads();   // the previous item's shared memory is free
        k_tv_strip_item<LAST, W>(t, vb);
    }
}

inline cudaError_t counted(cudaError_t e = cudaGetLastError())
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return e;
}

}  // namespace

cudaError_t launch_tv_final(const float* z, const float* p, int have_p, int n, int batch, float lambda,
                            float alpha, float a, float* xprev, float* y, const float* xtrue,
                            double* mse_partials, cudaStream_t st, const float* xin)
{
    dim3 blk(32, 8), grd(div_up(n, 32), div_up(n, 8), batch);
    long plane = (long)batch * n * n;
    const cudaError_t e = launch_pdl(k_tv_final, grd, blk, 0, st, z, p, have_p, n, plane, lambda, alpha, a, xprev,
                                     y, xtrue, mse_partials, xin);
    if (e != cudaSuccess) return e;
    return counted();
}

}  // namespace pnp

namespace pnp {

namespace {
constexpr int kTileThreads = 1024;
constexpr int kTileKMax = 10;            // iterations per launch (halo recompute vs launches)
constexpr size_t kTileSmemMax = 112 * 1024;

inline size_t tile_smem(int T, int K, int ring = 0)
{
    const int S = T + 1 + 2 * K + ring;
    return (size_t)5 * S * kTilePitch * sizeof(float);
}

// pixels per thread needed to cover the (T + 1 + 2K + ring)^2 region with 1024 threads
inline int tile_np(int T, int K, int ring = 0)
{
    const int S = T + 1 + 2 * K + ring;
    return (S * S + kTileThreads - 1) / kTileThreads;
}

// Tile side: minimises the busiest SM's work, (tiles per SM, rounded up) x
// (work per tile ~ (T + 1 + K)^2); CTAs sharing an SM share its issue slots.
int choose_tile(int n, int batch)
{
    int best = 16;
    double best_cost = 1e300;
    const long sms = device_sm_count();
    for (int T = 8; T <= 40; ++T) {
        if (tile_smem(T, kTileKMax, 2) > kTileSmemMax || tile_np(T, kTileKMax, 2) > 4) break;
        const long tiles = (long)batch * ((n + T - 1) / T) * ((n + T - 1) / T);
        const long waves = (tiles + sms - 1) / sms;
        const double side = (double)std::min(T, n) + 1 + kTileKMax;
        const double cost = (double)waves * side * side;
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best = T;
        }
    }
    return best;
}
}  // namespace

int tile_tv_tile(int n, int batch) { return choose_tile(n, batch); }

// The tile side a launch uses: the requested one when it fits (ring included),
// else the default.
int resolve_tile(int tile, int n, int batch)
{
    if (tile < 4 || tile > 64 || tile_np(tile, kTileKMax, 2) > 4 || tile_smem(tile, kTileKMax, 2) > kTileSmemMax)
        return tile_tv_tile(n, batch);
    return tile;
}

bool tv_fuses_quad(int tile, int n, int batch, int qs)
{
    if (tile == kTvTileWarp || tv_is_strip(tile)) return false;
    if (qs == 1) return true;
    return qs == 2 && n % 2 == 0 && resolve_tile(tile, n, batch) % 2 == 0;
}

int tile_tv_parts_for(int n, int batch, int tile)
{
    if (tile == kTvTileWarp)
        return ((n + kWarpTvWV - 1) / kWarpTvWV) * ((n + kWarpTvHV - 1) / kWarpTvHV);
    if (tv_is_strip(tile)) {
        const int ho = tv_strip_warps(tile) * kStripR - 2 * kStripK - 1;
        return ((n + kStripWO - 1) / kStripWO) * ((n + ho - 1) / ho);
    }
    const int T = resolve_tile(tile, n, batch);
    return ((n + T - 1) / T) * ((n + T - 1) / T);
}

namespace {
// Register-resident variant: warp tiles of kWarpTvWV x kWarpTvHV, kWarpTvK iterations per launch.
cudaError_t launch_tv_warp_multi(const TvItem* items, int count, float lambda, int iters, float alpha,
                                 const std::vector<float>& mom, cudaStream_t st)
{
    WarpTvArgs a{};
    a.count = count;
    a.lambda = lambda;
    a.alpha = alpha;
    a.begin[0] = 0;
    for (int c = 0; c < count; ++c) {
        const TvItem& it = items[c];
        if (iters > kWarpTvK && (!it.state_a || !it.state_b)) return cudaErrorInvalidValue;
        WarpTvClass& wc = a.c[c];
        wc.z = it.z; wc.xprev = it.xprev; wc.y = it.y; wc.xtrue = it.xtrue; wc.mse_part = it.mse_part;
        wc.xin = it.xin;
        wc.n = it.n;
        wc.tiles_x = (it.n + kWarpTvWV - 1) / kWarpTvWV;
        wc.tiles = wc.tiles_x * ((it.n + kWarpTvHV - 1) / kWarpTvHV);
        wc.plane = (long)it.batch * it.n * it.n;
        wc.amom = it.amom;
        a.begin[c + 1] = a.begin[c] + (long)wc.tiles * it.batch;
    }
    const dim3 grd((unsigned)((a.begin[count] + kWarpTvWarps - 1) / kWarpTvWarps)), blk(32 * kWarpTvWarps);
    int k0 = 0, pass = 0;
    cudaError_t e = cudaSuccess;
    do {
        const int K = std::min(kWarpTvK, iters - k0);
        a.K = K;
        a.first = k0 == 0;
        a.last = k0 + K == iters;
        for (int c = 0; c < count; ++c) {
            a.c[c].sin = k0 == 0 ? nullptr : (pass % 2 == 1 ? items[c].state_a : items[c].state_b);
            a.c[c].sout = a.last ? nullptr : (pass % 2 == 0 ? items[c].state_a : items[c].state_b);
        }
        for (int k = 0; k < K; ++k) a.mom[k] = mom[k0 + k];
        e = launch_items(k_tv_warp, k_tv_warp_persistent, grd, blk, 0, st, a);
        g_launches.fetch_add(1, std::memory_order_relaxed);
        if (e != cudaSuccess) return e;
        k0 += K;
        ++pass;
    } while (k0 < iters);
    return e;
}
}  // namespace

// Register-resident strips: 64 x 8W regions, up to kStripK iterations per launch.
cudaError_t launch_tv_strip_multi(const TvItem* items, int count, float lambda, int iters, float alpha,
                                  const std::vector<float>& mom, cudaStream_t st)
{
    StripTvArgs a{};
    a.count = count;
    a.lambda = lambda;
    a.alpha = alpha;
    a.W = tv_strip_warps(items[0].tile);
    a.begin[0] = 0;
    const int ho = a.W * kStripR - 2 * kStripK - 1;
    for (int c = 0; c < count; ++c) {
        const TvItem& it = items[c];
        if (iters > kStripK && (!it.state_a || !it.state_b)) return cudaErrorInvalidValue;
        StripTvClass& sc = a.c[c];
        sc.z = it.z; sc.xprev = it.xprev; sc.y = it.y; sc.xtrue = it.xtrue; sc.mse_part = it.mse_part;
        sc.xin = it.xin;
        sc.n = it.n;
        sc.tiles_x = (it.n + kStripWO - 1) / kStripWO;
        sc.tiles = sc.tiles_x * ((it.n + ho - 1) / ho);
        sc.plane = (long)it.batch * it.n * it.n;
        sc.amom = it.amom;
        a.begin[c + 1] = a.begin[c] + (long)sc.tiles * it.batch;
    }
    const dim3 grd((unsigned)a.begin[count]), blk(32, a.W);
    const size_t smem = (size_t)a.W * 32 * (kStripR + 2) * sizeof(float2);
    int k0 = 0, pass = 0;
    cudaError_t e = cudaSuccess;
    do {
        const int K = std::min(kStripK, iters - k0);
        a.K = K;
        a.first = k0 == 0;
        a.last = k0 + K == iters;
        for (int c = 0; c < count; ++c) {
            a.c[c].sin = k0 == 0 ? nullptr : (pass % 2 == 1 ? items[c].state_a : items[c].state_b);
            a.c[c].sout = a.last ? nullptr : (pass % 2 == 0 ? items[c].state_a : items[c].state_b);
        }
        for (int k = 0; k < K; ++k) a.mom[k] = mom[k0 + k];
        if (a.W == 8)
            e = a.last ? launch_items(k_tv_strip<true, 8>, k_tv_strip_persistent<true, 8>, grd, blk, smem, st, a)
                       : launch_items(k_tv_strip<false, 8>, k_tv_strip_persistent<false, 8>, grd, blk, smem, st, a);
        else if (a.W == 12)
            e = a.last ? launch_items(k_tv_strip<true, 12>, k_tv_strip_persistent<true, 12>, grd, blk, smem, st, a)
                       : launch_items(k_tv_strip<false, 12>, k_tv_strip_persistent<false, 12>, grd, blk, smem, st, a);
        else
            e = a.last ? launch_items(k_tv_strip<true, 16>, k_tv_strip_persistent<true, 16>, grd, blk, smem, st, a)
                       : launch_items(k_tv_strip<false, 16>, k_tv_strip_persistent<false, 16>, grd, blk, smem, st, a);
        g_launches.fetch_add(1, std::memory_order_relaxed);
        if (e != cudaSuccess) return e;
        k0 += K;
        ++pass;
    } while (k0 < iters);
    return e;
}

int tile_tv_parts(int n, int batch) { return tile_tv_parts_for(n, batch, 0); }

cudaError_t launch_tv_tiled_multi(const TvItem* items, int count, float lambda, int iters, float alpha,
                                  cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        const int mx = (int)kTileSmemMax;
        cudaFuncSetAttribute(k_tv_tile<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_tv_tile<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_tv_tile<3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_tv_tile<4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_tv_tile<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_tv_tile<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_tv_tile<3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_tv_tile<4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_tv_tile_persistent<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_tv_tile_persistent<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_tv_tile_persistent<3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_tv_tile_persistent<4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_tv_tile_persistent<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_tv_tile_persistent<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_tv_tile_persistent<3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_tv_tile_persistent<4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        attr = true;
    }
    if (count < 1 || count > kMaxClasses || iters < 1) return cudaErrorInvalidValue;
    std::vector<float> mom((size_t)iters);
    double tt = 1.0;
    for (int k = 0; k < iters; ++k) {
        const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * tt * tt));
        mom[k] = (float)((tt - 1.0) / tn);
        tt = tn;
    }
    if (items[0].tile == kTvTileWarp) return launch_tv_warp_multi(items, count, lambda, iters, alpha, mom, st);
    if (tv_is_strip(items[0].tile)) return launch_tv_strip_multi(items, count, lambda, iters, alpha, mom, st);
    TileTvArgs a{};
    a.count = count;
    a.lambda = lambda;
    a.alpha = alpha;
    a.begin[0] = 0;
    int Tmax = 0;
    for (int c = 0; c < count; ++c) {
        const TvItem& it = items[c];
        const int T = resolve_tile(it.tile, it.n, it.batch);
        if (iters > kTileKMax && (!it.state_a || !it.state_b)) return cudaErrorInvalidValue;   // chaining needs state
        TileTvClass& tc = a.c[c];
        tc.z = it.z; tc.xprev = it.xprev; tc.y = it.y; tc.xtrue = it.xtrue; tc.mse_part = it.mse_part;
        tc.xin = it.xin; tc.quad = it.quad; tc.qw = it.qw; tc.qs = it.qs; tc.qbatch = it.batch;
        tc.n = it.n; tc.T = T; tc.tiles_x = (it.n + T - 1) / T; tc.tiles = tc.tiles_x * tc.tiles_x;
        tc.plane = (long)it.batch * it.n * it.n;
        tc.amom = it.amom;
        a.begin[c + 1] = a.begin[c] + (long)tc.tiles * it.batch;
        Tmax = std::max(Tmax, T);
    }
    int k0 = 0;
    int pass = 0;
    cudaError_t e = cudaSuccess;
    do {
        const int K = std::min(kTileKMax, iters - k0);
        a.K = K;
        a.first = k0 == 0;
        a.last = k0 + K == iters;
        int ring = 0;
        for (int c = 0; c < count; ++c) {
            float* sa = items[c].state_a;
            float* sb = items[c].state_b;
            a.c[c].sin = k0 == 0 ? nullptr : (pass % 2 == 1 ? sa : sb);
            a.c[c].sout = a.last ? nullptr : (pass % 2 == 0 ? sa : sb);
            // the coefficient image needs y on a ring of qs pixels: last launch only
            const bool fuse = a.last && items[c].quad && items[c].y && items[c].xin &&
                              tv_fuses_quad(items[c].tile, items[c].n, items[c].batch, items[c].qs);
            a.c[c].ring = fuse ? items[c].qs : 0;
            a.c[c].qs = items[c].qs;
            ring = std::max(ring, a.c[c].ring);
        }
        for (int k = 0; k < K; ++k) a.mom[k] = mom[k0 + k];
        if (Tmax + 1 + 2 * K + ring > kTilePitch) return cudaErrorInvalidValue;   // rows would overlap
        const dim3 grd((unsigned)a.begin[count]);
        const size_t sm = tile_smem(Tmax, K, ring);
        const dim3 blk(kTileThreads);
        switch (tile_np(Tmax, K, ring)) {
            case 1: e = a.last ? launch_items(k_tv_tile<1, true>, k_tv_tile_persistent<1, true>, grd, blk, sm, st, a)
                               : launch_items(k_tv_tile<1, false>, k_tv_tile_persistent<1, false>, grd, blk, sm, st, a); break;
            case 2: e = a.last ? launch_items(k_tv_tile<2, true>, k_tv_tile_persistent<2, true>, grd, blk, sm, st, a)
                               : launch_items(k_tv_tile<2, false>, k_tv_tile_persistent<2, false>, grd, blk, sm, st, a); break;
            case 3: e = a.last ? launch_items(k_tv_tile<3, true>, k_tv_tile_persistent<3, true>, grd, blk, sm, st, a)
                               : launch_items(k_tv_tile<3, false>, k_tv_tile_persistent<3, false>, grd, blk, sm, st, a); break;
            default: e = a.last ? launch_items(k_tv_tile<4, true>, k_tv_tile_persistent<4, true>, grd, blk, sm, st, a)
                                : launch_items(k_tv_tile<4, false>, k_tv_tile_persistent<4, false>, grd, blk, sm, st, a); break;
        }
        g_launches.fetch_add(1, std::memory_order_relaxed);
        if (e != cudaSuccess) return e;
        k0 += K;
        ++pass;
    } while (k0 < iters);
    return e;
}

cudaError_t launch_tv_tiled(const float* z, int n, int batch, float lambda, int iters, float alpha,
                            float amom, float* xprev, float* y, const float* xtrue, double* mse_part,
                            float* state_a, float* state_b, cudaStream_t st, int tile)
{
    TvItem it{};
    it.z = z; it.xprev = xprev; it.y = y; it.xtrue = xtrue; it.mse_part = mse_part;
    it.state_a = state_a; it.state_b = state_b;
    it.n = n; it.batch = batch; it.tile = tile; it.amom = amom;
    return launch_tv_tiled_multi(&it, 1, lambda, iters, alpha, st);
}

}  // namespace pnp
