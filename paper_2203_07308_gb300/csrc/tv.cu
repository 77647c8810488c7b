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

#include "pnp_internal.cuh"

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
