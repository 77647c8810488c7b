// Reverse mode of the PnP-MS2G iteration, for unrolling Algorithm 1 and
// differentiating through it (the paper's Sec. 2 remark that the sketched
// iterations, denoiser and sampling operators can be unrolled and trained end
// to end).  Deterministic: no atomics; reductions go through fixed-order
// per-block partial sums.
//
// FGP with pre-projection points a_k (k = 1..N):
//   a_k = r_k + L^T(z - lambda L r_k)/(8 lambda),  p_k = Proj(a_k),
//   r_{k+1} = (1 + m_k) p_k - m_k p_{k-1},         x = z - lambda L p_N.
// Reverse sweep given xbar:
//   pbar_N = -lambda L^T xbar,  lambar = -<xbar, L p_N>;  for k = N..1:
//   pbar_k += (1 + m_k) rbar_{k+1};  pbar_{k-1} gets -m_k rbar_{k+1};
//   abar_k = J_Proj(a_k)^T pbar_k;   rbar_k = abar_k - L^T L abar_k / 8;
//   zbar += L abar_k / (8 lambda);   lambar -= <L abar_k, z> / (8 lambda^2).
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "pnp_internal.cuh"

namespace pnp {
namespace {

__host__ __device__ inline int div_up(long a, long b) { return (int)((a + b - 1) / b); }

// L(u, v)[i][j] = u[i][j] + v[i][j] - u[i-1][j] - v[i][j-1] (terms outside dropped)
__device__ __forceinline__ float Lop(const float* __restrict__ u, const float* __restrict__ v, int n,
                                     int i, int j)
{
    const long o = (long)i * n + j;
    float l = u[o] + v[o];
    if (i > 0) l -= u[o - n];
    if (j > 0) l -= v[o - 1];
    return l;
}

// One recorded FGP iteration on [batch][n][n]: a_k -> a (2 planes), p, r_out.
__global__ void k_fgp_record(const float* __restrict__ z, const float* __restrict__ rin,
                             float* __restrict__ rout, float* __restrict__ p, float* __restrict__ a_out,
                             int n, long plane, float lambda, float mom, int first)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    const int inst = blockIdx.z;
    if (i >= n || j >= n) return;
    const long img = (long)inst * n * n;
    const float* zi = z + img;
    const float* r1 = rin + img;
    const float* r2 = rin + plane + img;
    auto xt = [&](int ii, int jj) {
        const long o = (long)ii * n + jj;
        return first ? zi[o] : zi[o] - lambda * Lop(r1, r2, n, ii, jj);
    };
    const float x0 = xt(i, j);
    const float g1 = i < n - 1 ? x0 - xt(i + 1, j) : 0.0f;
    const float g2 = j < n - 1 ? x0 - xt(i, j + 1) : 0.0f;
    const long o = img + (long)i * n + j;
    const float inv8l = 1.0f / (8.0f * lambda);
    const float a1 = (first ? 0.0f : r1[(long)i * n + j]) + g1 * inv8l;
    const float a2 = (first ? 0.0f : r2[(long)i * n + j]) + g2 * inv8l;
    a_out[o] = a1;
    a_out[plane + o] = a2;
    const float den = fmaxf(sqrtf(a1 * a1 + a2 * a2), 1.0f);
    const float pa = a1 / den, pc = a2 / den;
    const float po1 = first ? 0.0f : p[o], po2 = first ? 0.0f : p[plane + o];
    p[o] = pa;
    p[plane + o] = pc;
    rout[o] = pa + mom * (pa - po1);
    rout[plane + o] = pc + mom * (pc - po2);
}

// Block sum (256 threads) into partials[inst][block] (+= when accumulate).
__device__ __forceinline__ void block_partial(double v, double* partials, int accumulate)
{
    __shared__ double sh[8];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    if ((tid & 31) == 0) sh[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)((blockDim.x * blockDim.y) >> 5); ++w) s += sh[w];
        const long idx = (long)blockIdx.z * gridDim.x * gridDim.y + blockIdx.y * gridDim.x + blockIdx.x;
        partials[idx] = accumulate ? partials[idx] + s : s;
    }
}

// Start of the sweep: carry = -lambda L^T xbar, rbar = 0, zbar = xbar,
// partials = -<xbar, L p_N>.
__global__ void k_vjp_init(const float* __restrict__ xbar, const float* __restrict__ p,
                           float* __restrict__ carry, float* __restrict__ rbar, float* __restrict__ zbar,
                           double* __restrict__ partials, int n, long plane, float lambda)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    const int inst = blockIdx.z;
    double acc = 0.0;
    if (i < n && j < n) {
        const long img = (long)inst * n * n;
        const long o = img + (long)i * n + j;
        const float* xb = xbar + img;
        const float xv = xb[(long)i * n + j];
        const float lt1 = i < n - 1 ? xv - xb[(long)(i + 1) * n + j] : 0.0f;   // L^T xbar
        const float lt2 = j < n - 1 ? xv - xb[(long)i * n + j + 1] : 0.0f;
        carry[o] = -lambda * lt1;
        carry[plane + o] = -lambda * lt2;
        rbar[o] = 0.0f;
        rbar[plane + o] = 0.0f;
        zbar[o] = xv;
        acc = -(double)xv * (double)Lop(p + img, p + plane + img, n, i, j);
    }
    block_partial(acc, partials, 0);
}

// Reverse step k, part 1 (pointwise): pbar = carry + (1+m) rbar; carry = -m rbar;
// abar = J_Proj(a_k)^T pbar.
__global__ void k_vjp_proj(const float* __restrict__ a_k, float* __restrict__ carry,
                           const float* __restrict__ rbar, float* __restrict__ abar, long count,
                           long plane, float mom)
{
    for (long o = (long)blockIdx.x * blockDim.x + threadIdx.x; o < count; o += (long)gridDim.x * blockDim.x) {
        const float pb1 = carry[o] + (1.0f + mom) * rbar[o];
        const float pb2 = carry[plane + o] + (1.0f + mom) * rbar[plane + o];
        carry[o] = -mom * rbar[o];
        carry[plane + o] = -mom * rbar[plane + o];
        const float a1 = a_k[o], a2 = a_k[plane + o];
        const float nrm = sqrtf(a1 * a1 + a2 * a2);
        if (nrm > 1.0f) {
            const float h1 = a1 / nrm, h2 = a2 / nrm;
            const float d = h1 * pb1 + h2 * pb2;
            abar[o] = (pb1 - h1 * d) / nrm;
            abar[plane + o] = (pb2 - h2 * d) / nrm;
        } else {
            abar[o] = pb1;
            abar[plane + o] = pb2;
        }
    }
}

// Reverse step k, part 2 (stencil): w = L abar; zbar += w / (8 lambda);
// partials += -<w, z> / (8 lambda^2); rbar = abar - L^T w / 8.
__global__ void k_vjp_lap(const float* __restrict__ abar, const float* __restrict__ z,
                          float* __restrict__ rbar, float* __restrict__ zbar, double* __restrict__ partials,
                          int n, long plane, float lambda)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    const int inst = blockIdx.z;
    double acc = 0.0;
    if (i < n && j < n) {
        const long img = (long)inst * n * n;
        const float* u = abar + img;
        const float* v = abar + plane + img;
        const float w0 = Lop(u, v, n, i, j);
        const long o = img + (long)i * n + j;
        zbar[o] += w0 / (8.0f * lambda);
        acc = -(double)w0 * (double)z[o] / (8.0 * (double)lambda * (double)lambda);
        const float lt1 = i < n - 1 ? w0 - Lop(u, v, n, i + 1, j) : 0.0f;
        const float lt2 = j < n - 1 ? w0 - Lop(u, v, n, i, j + 1) : 0.0f;
        rbar[o] = u[(long)i * n + j] - 0.125f * lt1;
        rbar[plane + o] = v[(long)i * n + j] - 0.125f * lt2;
    }
    block_partial(acc, partials, 1);
}

// out = c1 * a + c2 * b (elementwise); b may be null (then out = c1 * a).
__global__ void k_axpby(const float* __restrict__ a, float c1, const float* __restrict__ b, float c2,
                        float* __restrict__ out, long count)
{
    for (long o = (long)blockIdx.x * blockDim.x + threadIdx.x; o < count; o += (long)gridDim.x * blockDim.x)
        out[o] = b ? c1 * a[o] + c2 * b[o] : c1 * a[o];
}

inline cudaError_t counted(cudaError_t e = cudaGetLastError())
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return e;
}

inline int grid1(long count)
{
    long g = (count + 255) / 256;
    return (int)(g < 1216 ? (g < 1 ? 1 : g) : 1216);
}

}  // namespace

size_t tv_vjp_workspace_floats(int n, int batch, int iters)
{
    const size_t img = (size_t)batch * n * n;
    // a_k (2 planes each), r ping/pong (4), p (2), carry (2), rbar (2), abar (2)
    return img * (2 * (size_t)iters + 12);
}

size_t tv_vjp_partials(int n)
{
    return (size_t)div_up(n, 32) * div_up(n, 8);
}

cudaError_t launch_tv_vjp(const float* z, const float* xbar, float* zbar, double* partials, int n,
                          int batch, float lambda, int iters, float* ws, cudaStream_t st)
{
    const size_t img = (size_t)batch * n * n;
    const long plane = (long)img;
    float* a_all = ws;
    float* ra = a_all + 2 * img * (size_t)iters;
    float* rb = ra + 2 * img;
    float* p = rb + 2 * img;
    float* carry = p + 2 * img;
    float* rbar = carry + 2 * img;
    float* abar = rbar + 2 * img;
    dim3 blk(32, 8), grd(div_up(n, 32), div_up(n, 8), batch);
    std::vector<float> mom((size_t)iters);
    double t = 1.0;
    for (int k = 0; k < iters; ++k) {
        const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
        mom[k] = (float)((t - 1.0) / tn);
        t = tn;
    }
    cudaError_t e;
    const float* rin = ra;
    float* rout = rb;
    for (int k = 0; k < iters; ++k) {
        k_fgp_record<<<grd, blk, 0, st>>>(z, rin, rout, p, a_all + 2 * img * (size_t)k, n, plane, lambda,
                                          mom[k], k == 0);
        if ((e = counted()) != cudaSuccess) return e;
        const float* tmp = rout;
        rout = (float*)rin;
        rin = tmp;
    }
    k_vjp_init<<<grd, blk, 0, st>>>(xbar, p, carry, rbar, zbar, partials, n, plane, lambda);
    if ((e = counted()) != cudaSuccess) return e;
    for (int k = iters - 1; k >= 0; --k) {
        k_vjp_proj<<<grid1((long)img), 256, 0, st>>>(a_all + 2 * img * (size_t)k, carry, rbar, abar, (long)img,
                                                     plane, mom[k]);
        if ((e = counted()) != cudaSuccess) return e;
        k_vjp_lap<<<grd, blk, 0, st>>>(abar, z, rbar, zbar, partials, n, plane, lambda);
        if ((e = counted()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_axpby(const float* a, float c1, const float* b, float c2, float* out, long count,
                         cudaStream_t st)
{
    k_axpby<<<grid1(count), 256, 0, st>>>(a, c1, b, c2, out, count);
    return counted();
}

}  // namespace pnp
