// Variance-reduced subset estimates for Option 2 of Algorithm 1 (Sec. 2 names
// SVRG and SAGA as replacements for the vanilla minibatch estimate).
//
// Everything here works on raw level-s gradients R = A_s^{(p)T} W (A_s^{(p)} S y - b^{(p)})
// (scaled by the sample weight, before U and the subset factor c = P):
//   SVRG (Johnson & Zhang 2013):  v = P R'_p(y - yt) + R_full(yt), where R' has
//         no data term (G_p(y) - G_p(yt) is linear in y - yt), yt the snapshot;
//   SAGA (Defazio et al. 2014):   v = P (R_p(y) - T_p) + Phi,  Phi = sum_j T_j,
//         then Phi += R_p(y) - T_p and T_p = R_p(y).
// The step z = y - eta U v follows (U = S^T).  All kernels are elementwise over
// the level grid, deterministic and free of atomics.
#include <cuda_runtime.h>

#include "pnp_internal.cuh"

namespace pnp {
namespace {

__host__ __device__ inline int div_up(long a, long b) { return (int)((a + b - 1) / b); }

inline cudaError_t counted(cudaError_t e = cudaGetLastError())
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return e;
}

// Phi = sum_j table[j] over P planes of `count` values, in the order j = 0..P-1.
__global__ void k_vr_table_sum(const float* __restrict__ table, int P, long count, float* __restrict__ phi)
{
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
        float acc = 0.0f;
        for (int j = 0; j < P; ++j) acc += table[(long)j * count + i];
        phi[i] = acc;
    }
}

// Combined estimate v on the level grid [batch][ns][ns]; for the pooled
// sketch (U = replicate / s^2) also the step into z on the fine grid.
//   est 1 (SVRG): v = c G + mu;  est 2 (SAGA): v = c (G - T_p) + Phi, then the table update.
// `v_out` may be null when z is written here.
__global__ void k_vr_combine(int est, const float* __restrict__ G, float* __restrict__ acc_in,
                             float* __restrict__ Tp, float c, int ns, int batch, float* __restrict__ v_out,
                             const float* __restrict__ y, float* __restrict__ z, int s, float eta)
{
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int iy = blockIdx.y * blockDim.y + threadIdx.y;
    const int inst = blockIdx.z;
    if (ix >= ns || iy >= ns || inst >= batch) return;
    const long o = ((long)inst * ns + iy) * ns + ix;
    const float g = G[o];
    float v;
    if (est == 1) {
        v = c * g + acc_in[o];
    } else {
        const float t = Tp[o];
        const float phi = acc_in[o];
        v = c * (g - t) + phi;
        acc_in[o] = phi + (g - t);
        Tp[o] = g;
    }
    if (v_out) v_out[o] = v;
    if (z) {
        const int n = ns * s;
        const float step = eta * v / (float)(s * s);
        for (int b = 0; b < s; ++b) {
            const long row = ((long)inst * n + (long)iy * s + b) * n + (long)ix * s;
            for (int a = 0; a < s; ++a) z[row + a] = __ldg(y + row + a) - step;
        }
    }
}

}  // namespace

cudaError_t launch_vr_table_sum(const float* table, int P, long count, float* phi, cudaStream_t st)
{
    long g = (count + 255) / 256;
    k_vr_table_sum<<<(int)(g < 1216 ? (g < 1 ? 1 : g) : 1216), 256, 0, st>>>(table, P, count, phi);
    return counted();
}

cudaError_t launch_vr_combine(int est, const float* G, float* acc, float* Tp, float c, int ns, int batch,
                              float* v_out, const float* y, float* z, int s, float eta, cudaStream_t st)
{
    dim3 blk(32, 8), grd(div_up(ns, 32), div_up(ns, 8), batch);
    k_vr_combine<<<grd, blk, 0, st>>>(est, G, acc, Tp, c, ns, batch, v_out, y, z, s, eta);
    return counted();
}

}  // namespace pnp
