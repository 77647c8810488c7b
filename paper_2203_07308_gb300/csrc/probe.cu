// pnp_onchip_bandwidth: read bandwidth of the on-chip memory levels the
// projector kernels stream their operands from, measured on the running GPU
// with kernels of this library and CUDA events.  The forward projector gathers
// 16 B of bilinear coefficients per sample from L1 (hits) and L2 (misses), the
// backprojector reads ray tables and residuals from the same levels, and the
// FGP denoiser works in shared memory, so these are the denominators of their
// memory rooflines (the HBM copy bandwidth binds none of them).  Library
// instrumentation; the paper has no counterpart.
//
// Three probes, each a read-only loop of 16-byte loads whose sum is kept alive
// by a store behind a runtime flag that is never set:
//   L2    every thread block streams a buffer of l2_bytes (resident in L2 after
//         the first pass) with loads that bypass L1 (ld.global.cg);
//   L1    every block re-reads a private 16 KB window (L1 hits after the first
//         touch) through the non-coherent path (ld.global.nc);
//   SMEM  every block re-reads 32 KB of shared memory, one 16-byte word per
//         lane, consecutive lanes on consecutive words (no bank conflicts).
#include <cuda_runtime.h>

#include <algorithm>

#include "pnp_internal.cuh"

namespace pnp {
namespace {

__device__ __forceinline__ void add4(float4& a, const float4 b)
{
    a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w;
}

__global__ void __launch_bounds__(512) k_probe_l2(const float4* __restrict__ buf, long n4, int passes, int flag,
                                                  float* __restrict__ sink)
{
    float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0, a2 = a0, a3 = a0;
    const long stride = (long)gridDim.x * blockDim.x;
    const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    for (int p = 0; p < passes; ++p) {
        long i = tid;
        for (; i + 3 * stride < n4; i += 4 * stride) {
            add4(a0, __ldcg(buf + i));
            add4(a1, __ldcg(buf + i + stride));
            add4(a2, __ldcg(buf + i + 2 * stride));
            add4(a3, __ldcg(buf + i + 3 * stride));
        }
        for (; i < n4; i += stride) add4(a0, __ldcg(buf + i));
    }
    add4(a0, a1); add4(a2, a3); add4(a0, a2);
    if (flag) sink[tid] = a0.x + a0.y + a0.z + a0.w;
}

constexpr int kL1Window = 1024;   // float4 per block: 16 KB

__global__ void __launch_bounds__(256) k_probe_l1(const float4* __restrict__ buf, int reps, int flag,
                                                  float* __restrict__ sink)
{
    const float4* base = buf + (long)blockIdx.x * kL1Window;
    float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0, a2 = a0, a3 = a0;
    const int t = threadIdx.x;   // 256 threads: four loads each cover the window once
    for (int r = 0; r < reps; ++r) {
        const int o = (r * 32) & (kL1Window - 1);
        add4(a0, __ldg(base + ((t + o) & (kL1Window - 1))));
        add4(a1, __ldg(base + ((t + 256 + o) & (kL1Window - 1))));
        add4(a2, __ldg(base + ((t + 512 + o) & (kL1Window - 1))));
        add4(a3, __ldg(base + ((t + 768 + o) & (kL1Window - 1))));
    }
    add4(a0, a1); add4(a2, a3); add4(a0, a2);
    if (flag) sink[(long)blockIdx.x * blockDim.x + t] = a0.x + a0.y + a0.z + a0.w;
}

constexpr int kSmemWords = 2048;  // float4: 32 KB

__global__ void __launch_bounds__(256) k_probe_smem(int reps, int flag, float* __restrict__ sink)
{
    __shared__ float4 sm[kSmemWords];
    const int t = threadIdx.x;
    for (int i = t; i < kSmemWords; i += blockDim.x)
        sm[i] = make_float4((float)i, (float)(i + 1), (float)(i + 2), (float)(i + 3));
    __syncthreads();
    float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0, a2 = a0, a3 = a0;
    for (int r = 0; r < reps; ++r) {
        const int o = (r * 32) & (kSmemWords - 1);
        add4(a0, sm[(t + o) & (kSmemWords - 1)]);
        add4(a1, sm[(t + 256 + o) & (kSmemWords - 1)]);
        add4(a2, sm[(t + 512 + o) & (kSmemWords - 1)]);
        add4(a3, sm[(t + 768 + o) & (kSmemWords - 1)]);
    }
    add4(a0, a1); add4(a2, a3); add4(a0, a2);
    if (flag) sink[(long)blockIdx.x * blockDim.x + t] = a0.x + a0.y + a0.z + a0.w;
}

inline cudaError_t counted(cudaError_t e = cudaGetLastError())
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return e;
}

}  // namespace
}  // namespace pnp

using namespace pnp;

#define PROBE_CUDA(call)                                                                        \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) {                                                                \
            rc = fail(PNP_ECUDA, "pnp_onchip_bandwidth: %s: %s", #call, cudaGetErrorString(e_)); \
            goto done;                                                                          \
        }                                                                                       \
    } while (0)

extern "C" int pnp_onchip_bandwidth(void* d_buf, size_t bytes, double* h_gbs, void* stream)
{
    clear_error();
    const size_t l2_bytes = (size_t)24 << 20;
    if (!d_buf || !h_gbs) return fail(PNP_EINVAL, "buffer and output are required");
    if ((uintptr_t)d_buf % 256) return fail(PNP_EINVAL, "buffer must be 256-byte aligned");
    const int sms = device_sm_count();
    const int l1_blocks = 4 * sms;                                 // 4 x 256 threads per SM
    const size_t l1_bytes = (size_t)l1_blocks * kL1Window * sizeof(float4);
    const size_t sink_bytes = (size_t)4 * sms * 512 * sizeof(float);
    const size_t need = std::max(l2_bytes, l1_bytes) + sink_bytes;
    if (bytes < need) return fail(PNP_EINVAL, "buffer has %zu bytes, needs %zu", bytes, need);
    cudaStream_t st = (cudaStream_t)stream;
    const float4* buf = (const float4*)d_buf;
    float* sink = (float*)((char*)d_buf + std::max(l2_bytes, l1_bytes));
    const long n4 = (long)(l2_bytes / sizeof(float4));
    const int l2_passes = 200, l1_reps = 4096, sm_reps = 4096;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = PNP_OK;
    float best[3] = {1e30f, 1e30f, 1e30f};
    PROBE_CUDA(cudaEventCreate(&e0));
    PROBE_CUDA(cudaEventCreate(&e1));
    // contents do not matter (the sums are never stored); fill once so no load reads
    // uninitialised memory
    PROBE_CUDA(cudaMemsetAsync(d_buf, 0, std::max(l2_bytes, l1_bytes), st));
    for (int trial = 0; trial < 4; ++trial) {     // trial 0 warms up
        for (int k = 0; k < 3; ++k) {
            PROBE_CUDA(cudaEventRecord(e0, st));
            if (k == 0)
                k_probe_l2<<<4 * sms, 512, 0, st>>>(buf, n4, l2_passes, 0, sink);
            else if (k == 1)
                k_probe_l1<<<l1_blocks, 256, 0, st>>>(buf, l1_reps, 0, sink);
            else
                k_probe_smem<<<4 * sms, 256, 0, st>>>(sm_reps, 0, sink);
            PROBE_CUDA(counted());
            PROBE_CUDA(cudaEventRecord(e1, st));
            PROBE_CUDA(cudaEventSynchronize(e1));
            float ms = 0.0f;
            PROBE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (trial > 0) best[k] = std::min(best[k], ms);
        }
    }
    h_gbs[0] = (double)l2_bytes * l2_passes / (best[0] * 1e-3) / 1e9;
    h_gbs[1] = (double)l1_blocks * 256.0 * 4.0 * 16.0 * l1_reps / (best[1] * 1e-3) / 1e9;
    h_gbs[2] = (double)(4 * sms) * 256.0 * 4.0 * 16.0 * sm_reps / (best[2] * 1e-3) / 1e9;
done:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}
