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
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cmath>

#include "pnp_internal.cuh"

namespace cg = cooperative_groups;

namespace pnp {
namespace {

__host__ __device__ inline int div_up(long a, long b) { return (int)((a + b - 1) / b); }

// x_tmp(i, j) = z(i, j) - lambda L(r, s)(i, j), from the momentum point r = (r1, r2).
__device__ __forceinline__ float xtmp_at(const float* __restrict__ z, const float* __restrict__ r1,
                                         const float* __restrict__ r2, int n, int i, int j,
                                         float lambda, int first)
{
    const long o = (long)i * n + j;
    float zz = __ldg(z + o);
    if (first) return zz;
    float l = __ldg(r1 + o) + __ldg(r2 + o);
    if (i > 0) l -= __ldg(r1 + o - n);
    if (j > 0) l -= __ldg(r2 + o - 1);
    return zz - lambda * l;
}

__global__ void k_tv_iter(const float* __restrict__ z, float* __restrict__ p,
                          const float* __restrict__ rin, float* __restrict__ rout, int n, long plane,
                          float lambda, float mom, int first)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    const int inst = blockIdx.z;
    if (i >= n || j >= n) return;
    const long img = (long)inst * n * n;
    const float* zi = z + img;
    const float* r1 = rin + img;
    const float* r2 = rin + plane + img;
    const float x0 = xtmp_at(zi, r1, r2, n, i, j, lambda, first);
    float g1 = 0.0f, g2 = 0.0f;
    if (i < n - 1) g1 = x0 - xtmp_at(zi, r1, r2, n, i + 1, j, lambda, first);
    if (j < n - 1) g2 = x0 - xtmp_at(zi, r1, r2, n, i, j + 1, lambda, first);
    const long o = img + (long)i * n + j;
    const float inv8l = 1.0f / (8.0f * lambda);
    float a = (first ? 0.0f : __ldg(r1 + (long)i * n + j)) + g1 * inv8l;
    float c = (first ? 0.0f : __ldg(r2 + (long)i * n + j)) + g2 * inv8l;
    const float nrm = sqrtf(a * a + c * c);
    const float den = fmaxf(nrm, 1.0f);
    a = a / den;
    c = c / den;
    const float pa = first ? 0.0f : p[o];
    const float pc = first ? 0.0f : p[plane + o];
    p[o] = a;
    p[plane + o] = c;
    rout[o] = a + mom * (a - pa);
    rout[plane + o] = c + mom * (c - pc);
}

__global__ void k_tv_final(const float* __restrict__ z, const float* __restrict__ p, int have_p,
                           int n, long plane, float lambda, float alpha, float amom,
                           float* __restrict__ xprev, float* __restrict__ y,
                           const float* __restrict__ xtrue, double* __restrict__ mse_part)
{
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
            const float xp = xprev[o];
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

// ------------------------------------------------------------------ fused cluster FGP
// All FGP iterations of one image in one thread-block cluster: the image rows
// are split into C bands, one per CTA; z and the state of a band live in that
// CTA's shared memory and the neighbour rows are read from the adjacent CTAs
// through distributed shared memory.  The momentum point r is double-buffered,
// so one cluster barrier per iteration suffices:
//   A: x_tmp = z - lambda L(r_cur) on the band plus the first row of the next
//      band (needs r1 of the row above the band and r, z of the row below);
//   B: p = Proj[r_cur + L^T(x_tmp)/(8 lambda)], r_nxt = p + m_k (p - p_prev);
//   cluster barrier (r_nxt complete everywhere; nobody still reads r_cur).
// Then x = z - lambda L(p), the relaxation, the momentum and the optional
// squared-error partial sum are written out.
struct FusedTvArgs {
    const float* z; float* xprev; float* y; const float* xtrue; double* mse_part;
    int n, rows, iters;
    float lambda, alpha, amom;
    float mom[kFusedTvMaxIters];
};

// Walks the band's pixels q = tid, tid + T, ... without a division per step.
struct BandWalk {
    int li, j, dli, dj, n;
    __device__ BandWalk(int tid, int T, int n_) : n(n_)
    {
        li = tid / n_;
        j = tid - li * n_;
        dli = T / n_;
        dj = T - dli * n_;
    }
    __device__ void next()
    {
        li += dli;
        j += dj;
        if (j >= n) { j -= n; ++li; }
    }
};

__global__ void __launch_bounds__(1024) k_tv_fused(const FusedTvArgs a)
{
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int c = (int)cl.block_rank();
    const int inst = blockIdx.x / C;
    const int n = a.n, R = a.rows;
    const int row0 = c * R;
    const int nrows = max(0, min(R, n - row0));
    const bool has_next = c + 1 < C && row0 + nrows < n;
    const int band = R * n;
    extern __shared__ float sm[];
    float* z = sm;
    float* const r1b0 = sm + band;
    float* const r1b1 = sm + 2 * band;
    float* const r2b0 = sm + 3 * band;
    float* const r2b1 = sm + 4 * band;
    float* p1 = sm + 5 * band;
    float* p2 = sm + 6 * band;
    float* xt = sm + 7 * band;                 // (R + 1) rows
    const int T = blockDim.x;
    const long gimg = (long)inst * n * n + (long)row0 * n;
    const int cnt = nrows * n;
    for (int q = threadIdx.x; q < cnt; q += T) {
        z[q] = __ldg(a.z + gimg + q);
        r1b0[q] = 0.0f; r2b0[q] = 0.0f; p1[q] = 0.0f; p2[q] = 0.0f;
    }
    // neighbour bands (valid only when they exist); buffer 1 sits `band` floats
    // after buffer 0 in every CTA
    const float* up_r1 = c > 0 ? cl.map_shared_rank(r1b0, c - 1) : nullptr;
    const float* up_p1 = c > 0 ? cl.map_shared_rank(p1, c - 1) : nullptr;
    const float* dn_r1 = has_next ? cl.map_shared_rank(r1b0, c + 1) : nullptr;
    const float* dn_r2 = has_next ? cl.map_shared_rank(r2b0, c + 1) : nullptr;
    const float* dn_z = has_next ? cl.map_shared_rank(z, c + 1) : nullptr;
    const float inv8l = 1.0f / (8.0f * a.lambda);
    const float lam = a.lambda;
    const int xrows = nrows + (has_next ? 1 : 0);
    const int xcnt = xrows * n;
    cl.sync();
    for (int k = 0; k < a.iters; ++k) {
        const int cur = k & 1;
        const int boff = cur * band;          // offset of the current buffer
        const float* r1 = cur ? r1b1 : r1b0;
        const float* r2 = cur ? r2b1 : r2b0;
        // phase A: x_tmp on the band and on the next band's first row
        BandWalk w(threadIdx.x, T, n);
        for (int q = threadIdx.x; q < xcnt; q += T, w.next()) {
            const int li = w.li, j = w.j;
            float rr1, rr2, zz, up, left;
            if (li < nrows) {
                rr1 = r1[q]; rr2 = r2[q]; zz = z[q];
                left = j > 0 ? r2[q - 1] : 0.0f;
                up = li > 0 ? r1[q - n] : (c > 0 ? up_r1[boff + (R - 1) * n + j] : 0.0f);
            } else {   // first row of band c + 1
                rr1 = dn_r1[boff + j]; rr2 = dn_r2[boff + j]; zz = dn_z[j];
                left = j > 0 ? dn_r2[boff + j - 1] : 0.0f;
                up = r1[q - n];
            }
            xt[q] = zz - lam * (rr1 + rr2 - up - left);
        }
        __syncthreads();
        // phase B: dual step, projection, momentum on the band
        const float m = a.mom[k];
        float* o1 = cur ? r1b0 : r1b1;
        float* o2 = cur ? r2b0 : r2b1;
        BandWalk w2(threadIdx.x, T, n);
        for (int q = threadIdx.x; q < cnt; q += T, w2.next()) {
            const int li = w2.li, j = w2.j;
            const int i = row0 + li;
            const float x0 = xt[q];
            const float g1 = i < n - 1 ? x0 - xt[q + n] : 0.0f;
            const float g2 = j < n - 1 ? x0 - xt[q + 1] : 0.0f;
            float pa = fmaf(g1, inv8l, r1[q]);
            float pc = fmaf(g2, inv8l, r2[q]);
            const float nrm2 = fmaf(pa, pa, pc * pc);
            if (nrm2 > 1.0f) {
                const float sc = rsqrtf(nrm2);
                pa *= sc;
                pc *= sc;
            }
            o1[q] = fmaf(m, pa - p1[q], pa);
            o2[q] = fmaf(m, pc - p2[q], pc);
            p1[q] = pa;
            p2[q] = pc;
        }
        cl.sync();
    }
    double e2 = 0.0;
    BandWalk w3(threadIdx.x, T, n);
    for (int q = threadIdx.x; q < cnt; q += T, w3.next()) {
        const int li = w3.li, j = w3.j;
        const float zz = z[q];
        float x = zz;
        if (a.iters > 0) {
            float l = p1[q] + p2[q];
            if (li > 0) l -= p1[q - n];
            else if (c > 0) l -= up_p1[(R - 1) * n + j];
            if (j > 0) l -= p2[q - 1];
            x = zz - lam * l;
        }
        const float xi = (1.0f - a.alpha) * zz + a.alpha * x;
        const long o = gimg + q;
        if (a.y) {
            const float xp = a.xprev[o];
            a.y[o] = xi + a.amom * (xi - xp);
        }
        a.xprev[o] = xi;
        if (a.xtrue) {
            const double d = (double)xi - (double)__ldg(a.xtrue + o);
            e2 += d * d;
        }
    }
    if (a.mse_part) {
        __shared__ double red[32];
        for (int off = 16; off > 0; off >>= 1) e2 += __shfl_xor_sync(0xffffffffu, e2, off);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e2;
        __syncthreads();
        if (threadIdx.x < 32) {
            const int nw = blockDim.x >> 5;
            double v = threadIdx.x < nw ? red[threadIdx.x] : 0.0;
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (threadIdx.x == 0) a.mse_part[(long)inst * C + c] = v;
        }
    }
    cl.sync();   // keep this CTA's shared memory alive until the neighbours are done
}

// ------------------------------------------------------------------ register-resident cluster FGP
// Same iteration as k_tv_fused, for images whose side n is a multiple of 32 and
// of the cluster size.  Thread (rb, j) of CTA c owns the V rows
// c*R + rb*V ... + V-1 of column j and keeps z, r and p of those pixels in
// registers.  Everything a thread needs from outside its strip comes from
// values its neighbours published at the end of the previous iteration
// (double-buffered, so one cluster barrier per iteration is enough):
//   - the momentum point r of the row above / the column to the left (for
//     x_tmp = z - lambda L(r)),
//   - r of the row below and of the column to the right, from which the thread
//     recomputes the neighbouring x_tmp values it needs for L^T(x_tmp).
// Inside a warp the column neighbours come from shuffles; across warps, row
// blocks and CTAs from shared memory and distributed shared memory.
template <int V>
struct RegTvSmem {
    // double-buffered publications, index [buf][rb][j] or [buf][rb][w][v]
    static __device__ __forceinline__ int row_pub(int buf, int rb, int j, int RB, int n)
    {
        return (buf * RB + rb) * n + j;
    }
    static __device__ __forceinline__ int col_pub(int buf, int rb, int w, int v, int RB, int W)
    {
        return ((buf * RB + rb) * W + w) * V + v;
    }
};

template <int V>
__global__ void __launch_bounds__(1024, 1) k_tv_reg(const FusedTvArgs a)
{
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int c = (int)cl.block_rank();
    const int inst = blockIdx.x / C;
    const int n = a.n, R = a.rows;
    const int RB = R / V;              // row blocks per CTA
    const int W = n >> 5;              // warps per row block
    const int tid = threadIdx.x;
    const int rb = tid / n;
    const int j = tid - rb * n;
    const int lane = tid & 31;
    const int w = j >> 5;
    const int i0 = c * R + rb * V;     // global row of this strip's first row
    typedef RegTvSmem<V> L;

    extern __shared__ float sh[];
    const int rowsz = 2 * RB * n, colsz = 2 * RB * W * V;
    float* last_r1 = sh;                       // r1 of the strip's last row
    float* first_r1 = last_r1 + rowsz;         // r1, r2 of the strip's first row
    float* first_r2 = first_r1 + rowsz;
    float* col0_r1 = first_r2 + rowsz;         // lane 0's column (all V rows)
    float* col0_r2 = col0_r1 + colsz;
    float* col31_r2 = col0_r2 + colsz;         // lane 31's column
    float* zfirst = col31_r2 + colsz;          // [RB][n] z of each strip's first row
    float* zcol0 = zfirst + RB * n;            // [RB][W][V] z of lane 0's column
    float* last_p1 = zcol0 + RB * W * V;       // [RB][n]
    float* col31_p2 = last_p1 + RB * n;        // [RB][W][V]

    const long gimg = (long)inst * n * n;
    float z[V], r1[V], r2[V], p1[V], p2[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        z[v] = __ldg(a.z + gimg + (long)(i0 + v) * n + j);
        r1[v] = r2[v] = p1[v] = p2[v] = 0.0f;
    }
    // static publications and the zero momentum point of iteration 0
    zfirst[rb * n + j] = z[0];
    last_r1[L::row_pub(0, rb, j, RB, n)] = 0.0f;
    first_r1[L::row_pub(0, rb, j, RB, n)] = 0.0f;
    first_r2[L::row_pub(0, rb, j, RB, n)] = 0.0f;
    if (lane == 0) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            zcol0[(rb * W + w) * V + v] = z[v];
            col0_r1[L::col_pub(0, rb, w, v, RB, W)] = 0.0f;
            col0_r2[L::col_pub(0, rb, w, v, RB, W)] = 0.0f;
        }
    }
    if (lane == 31) {
#pragma unroll
        for (int v = 0; v < V; ++v) col31_r2[L::col_pub(0, rb, w, v, RB, W)] = 0.0f;
    }
    // neighbour CTAs (the one above owns row i0 - 1 when rb == 0; the one below
    // owns row i0 + V when rb == RB - 1)
    const bool has_up = c > 0, has_dn = c + 1 < C;
    const float* up_last_r1 = has_up ? cl.map_shared_rank(last_r1, c - 1) : nullptr;
    const float* up_last_p1 = has_up ? cl.map_shared_rank(last_p1, c - 1) : nullptr;
    const float* dn_first_r1 = has_dn ? cl.map_shared_rank(first_r1, c + 1) : nullptr;
    const float* dn_first_r2 = has_dn ? cl.map_shared_rank(first_r2, c + 1) : nullptr;
    const float* dn_zfirst = has_dn ? cl.map_shared_rank(zfirst, c + 1) : nullptr;
    const float lam = a.lambda;
    const float inv8l = 1.0f / (8.0f * a.lambda);
    const bool last_img_row = i0 + V == n;      // the strip ends on the image's last row
    const bool last_col = j == n - 1;
    cl.sync();

    for (int k = 0; k < a.iters; ++k) {
        const int cur = k & 1, nxt = cur ^ 1;
        // r1 of the row above this strip (column j and, for lane 31, column j + 1)
        float r1_up = 0.0f, r1_up_r = 0.0f;
        if (rb > 0) {
            r1_up = last_r1[L::row_pub(cur, rb - 1, j, RB, n)];
            if (lane == 31 && !last_col) r1_up_r = last_r1[L::row_pub(cur, rb - 1, j + 1, RB, n)];
        } else if (has_up) {
            r1_up = up_last_r1[L::row_pub(cur, RB - 1, j, RB, n)];
            if (lane == 31 && !last_col) r1_up_r = up_last_r1[L::row_pub(cur, RB - 1, j + 1, RB, n)];
        }
        // x_tmp on the strip
        float xt[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            float left = __shfl_up_sync(0xffffffffu, r2[v], 1);
            if (lane == 0) left = j > 0 ? col31_r2[L::col_pub(cur, rb, w - 1, v, RB, W)] : 0.0f;
            const float up = v > 0 ? r1[v - 1] : r1_up;
            xt[v] = z[v] - lam * (r1[v] + r2[v] - up - left);
        }
        // x_tmp one row below the strip (same column)
        float xt_dn = 0.0f;
        if (!last_img_row) {
            float rr1, rr2, zz, left;
            if (rb + 1 < RB) {
                rr1 = first_r1[L::row_pub(cur, rb + 1, j, RB, n)];
                rr2 = first_r2[L::row_pub(cur, rb + 1, j, RB, n)];
                left = j > 0 ? first_r2[L::row_pub(cur, rb + 1, j - 1, RB, n)] : 0.0f;
                zz = zfirst[(rb + 1) * n + j];
            } else {
                rr1 = dn_first_r1[L::row_pub(cur, 0, j, RB, n)];
                rr2 = dn_first_r2[L::row_pub(cur, 0, j, RB, n)];
                left = j > 0 ? dn_first_r2[L::row_pub(cur, 0, j - 1, RB, n)] : 0.0f;
                zz = dn_zfirst[j];
            }
            xt_dn = zz - lam * (rr1 + rr2 - r1[V - 1] - left);
        }
        // x_tmp one column to the right (same rows)
        float xt_r[V];
#pragma unroll
        for (int v = 0; v < V; ++v) xt_r[v] = __shfl_down_sync(0xffffffffu, xt[v], 1);
        if (lane == 31 && !last_col) {
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const float rr1 = col0_r1[L::col_pub(cur, rb, w + 1, v, RB, W)];
                const float rr2 = col0_r2[L::col_pub(cur, rb, w + 1, v, RB, W)];
                const float up = v > 0 ? col0_r1[L::col_pub(cur, rb, w + 1, v - 1, RB, W)] : r1_up_r;
                xt_r[v] = zcol0[(rb * W + w + 1) * V + v] - lam * (rr1 + rr2 - up - r2[v]);
            }
        }
        // dual step, projection onto unit disks, momentum
        const float m = a.mom[k];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const float below = v + 1 < V ? xt[v + 1] : xt_dn;
            const float g1 = (v + 1 < V || !last_img_row) ? xt[v] - below : 0.0f;
            const float g2 = last_col ? 0.0f : xt[v] - xt_r[v];
            float pa = fmaf(g1, inv8l, r1[v]);
            float pc = fmaf(g2, inv8l, r2[v]);
            const float nrm2 = fmaf(pa, pa, pc * pc);
            if (nrm2 > 1.0f) {
                const float sc = rsqrtf(nrm2);
                pa *= sc;
                pc *= sc;
            }
            r1[v] = fmaf(m, pa - p1[v], pa);
            r2[v] = fmaf(m, pc - p2[v], pc);
            p1[v] = pa;
            p2[v] = pc;
        }
        // publish for the next iteration
        last_r1[L::row_pub(nxt, rb, j, RB, n)] = r1[V - 1];
        first_r1[L::row_pub(nxt, rb, j, RB, n)] = r1[0];
        first_r2[L::row_pub(nxt, rb, j, RB, n)] = r2[0];
        if (lane == 0) {
#pragma unroll
            for (int v = 0; v < V; ++v) {
                col0_r1[L::col_pub(nxt, rb, w, v, RB, W)] = r1[v];
                col0_r2[L::col_pub(nxt, rb, w, v, RB, W)] = r2[v];
            }
        }
        if (lane == 31) {
#pragma unroll
            for (int v = 0; v < V; ++v) col31_r2[L::col_pub(nxt, rb, w, v, RB, W)] = r2[v];
        }
        if (k + 1 == a.iters) {
            last_p1[rb * n + j] = p1[V - 1];
            if (lane == 31) {
#pragma unroll
                for (int v = 0; v < V; ++v) col31_p2[(rb * W + w) * V + v] = p2[v];
            }
        }
        cl.sync();
    }
    // x = z - lambda L(p), relaxation, momentum, squared error
    float p1_up = 0.0f;
    if (a.iters > 0) {
        if (rb > 0) p1_up = last_p1[(rb - 1) * n + j];
        else if (has_up) p1_up = up_last_p1[(RB - 1) * n + j];
    }
    double e2 = 0.0;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        float x = z[v];
        if (a.iters > 0) {
            float left = __shfl_up_sync(0xffffffffu, p2[v], 1);
            if (lane == 0) left = j > 0 ? col31_p2[(rb * W + w - 1) * V + v] : 0.0f;
            const float up = v > 0 ? p1[v - 1] : p1_up;
            x = z[v] - lam * (p1[v] + p2[v] - up - left);
        }
        const float xi = (1.0f - a.alpha) * z[v] + a.alpha * x;
        const long o = gimg + (long)(i0 + v) * n + j;
        if (a.y) {
            const float xp = a.xprev[o];
            a.y[o] = xi + a.amom * (xi - xp);
        }
        a.xprev[o] = xi;
        if (a.xtrue) {
            const double d = (double)xi - (double)__ldg(a.xtrue + o);
            e2 += d * d;
        }
    }
    if (a.mse_part) {
        __shared__ double red[32];
        for (int off = 16; off > 0; off >>= 1) e2 += __shfl_xor_sync(0xffffffffu, e2, off);
        if (lane == 0) red[tid >> 5] = e2;
        __syncthreads();
        if (tid < 32) {
            const int nw = blockDim.x >> 5;
            double v = tid < nw ? red[tid] : 0.0;
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (tid == 0) a.mse_part[(long)inst * C + c] = v;
        }
    }
    cl.sync();   // keep this CTA's shared memory alive until the neighbours are done
}

inline cudaError_t counted(cudaError_t e = cudaGetLastError())
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return e;
}

}  // namespace

cudaError_t launch_tv_iter(const float* z, TvBuffers b, const float* r_in, float* r_out, int n,
                           int batch, float lambda, float mom, int first, cudaStream_t st)
{
    dim3 blk(32, 8), grd(div_up(n, 32), div_up(n, 8), batch);
    long plane = (long)batch * n * n;
    k_tv_iter<<<grd, blk, 0, st>>>(z, b.p, r_in, r_out, n, plane, lambda, mom, first);
    return counted();
}

cudaError_t launch_tv_final(const float* z, const float* p, int have_p, int n, int batch, float lambda,
                            float alpha, float a, float* xprev, float* y, const float* xtrue,
                            double* mse_partials, cudaStream_t st)
{
    dim3 blk(32, 8), grd(div_up(n, 32), div_up(n, 8), batch);
    long plane = (long)batch * n * n;
    k_tv_final<<<grd, blk, 0, st>>>(z, p, have_p, n, plane, lambda, alpha, a, xprev, y, xtrue,
                                    mse_partials);
    return counted();
}

}  // namespace pnp

namespace pnp {

// Cluster size and band height for the fused kernel, or 0 if the image does
// not fit in the shared memory of one cluster of at most 16 CTAs.
// z, r (2 buffers x 2 components), p (2 components), x_tmp (one extra row)
inline size_t fused_tv_smem(int rows, int n) { return ((size_t)8 * rows + 1) * n * sizeof(float); }

int fused_tv_cluster(int n, int* rows)
{
    static int max_cluster = -1;
    if (max_cluster < 0) {
        // 16-CTA clusters are a non-portable size: use them only if this GPU
        // can schedule one with the largest band this kernel asks for.
        max_cluster = 8;
        cudaFuncSetAttribute(k_tv_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, kFusedTvSmem);
        if (cudaFuncSetAttribute(k_tv_fused, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
            cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = 16;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(16);
            cfg.blockDim = dim3(1024);
            cfg.dynamicSmemBytes = kFusedTvSmem;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int nc = 0;
            if (cudaOccupancyMaxActiveClusters(&nc, k_tv_fused, &cfg) == cudaSuccess && nc > 0)
                max_cluster = 16;
        }
        cudaGetLastError();
    }
    for (int C = max_cluster; C >= 1; C /= 2) {
        const int R = (n + C - 1) / C;
        if ((C - 1) * R >= n) continue;            // every CTA needs at least one row
        if (fused_tv_smem(R, n) > (size_t)kFusedTvSmem) return 0;
        *rows = R;
        return C;
    }
    return 0;
}

// Register-resident variant: V rows per thread, n % 32 == 0, n % C == 0,
// (R / V) * n <= 1024 threads.  Returns V (0 if not applicable).
inline size_t reg_tv_smem(int n, int R, int V)
{
    const size_t RB = R / V, W = n / 32;
    return (6 * RB * n + 6 * RB * W * V + RB * n + RB * W * V + RB * n + RB * W * V) * sizeof(float);
}

int reg_tv_rows_per_thread(int n, int C, int R)
{
    if (n % 32 != 0 || C * R != n) return 0;
    for (int V = 1; V <= 4; V *= 2)
        if (R % V == 0 && (R / V) * n <= 1024 && reg_tv_smem(n, R, V) <= 48 * 1024) return V;
    return 0;
}

template <int V>
cudaError_t launch_reg(cudaLaunchConfig_t& cfg, const FusedTvArgs& a)
{
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_tv_reg<V>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        attr = true;
    }
    return cudaLaunchKernelEx(&cfg, k_tv_reg<V>, a);
}

cudaError_t launch_tv_fused(const float* z, int n, int batch, float lambda, int iters, float alpha,
                            float amom, float* xprev, float* y, const float* xtrue, double* mse_part,
                            int cluster, int rows, cudaStream_t st)
{
    static bool attr_done = false;
    if (!attr_done) {
        cudaFuncSetAttribute(k_tv_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, kFusedTvSmem);
        cudaFuncSetAttribute(k_tv_fused, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        attr_done = true;
    }
    FusedTvArgs a{};
    a.z = z; a.xprev = xprev; a.y = y; a.xtrue = xtrue; a.mse_part = mse_part;
    a.n = n; a.rows = rows; a.iters = iters;
    a.lambda = lambda; a.alpha = alpha; a.amom = amom;
    double t = 1.0;
    for (int k = 0; k < iters; ++k) {
        const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
        a.mom[k] = (float)((t - 1.0) / tn);
        t = tn;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cluster * batch);
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e;
    const int V = reg_tv_rows_per_thread(n, cluster, rows);
    if (V > 0) {
        cfg.blockDim = dim3((rows / V) * n);
        cfg.dynamicSmemBytes = reg_tv_smem(n, rows, V);
        e = V == 1 ? launch_reg<1>(cfg, a) : V == 2 ? launch_reg<2>(cfg, a) : launch_reg<4>(cfg, a);
    } else {
        cfg.blockDim = dim3(1024);
        cfg.dynamicSmemBytes = fused_tv_smem(rows, n);
        e = cudaLaunchKernelEx(&cfg, k_tv_fused, a);
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return e;
}

}  // namespace pnp
