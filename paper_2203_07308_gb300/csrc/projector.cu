// Fan-beam projector pair on sm_103a: forward A_s (ray-driven, fixed step,
// bilinear taps) and its exact transpose A_s^T (pixel-driven gather, no
// atomics), plus the image-space sketch S (average pooling) and U = S^T.
//
// Paper: Eq. 1 (b = A x + w), Eq. 4 (A_s acting on S(x)), Eq. 5 (A^T), Alg. 1.
// The discretisation (the paper names only "fan-beam X-ray CT", Sec. 3):
//   ray (v,j) with unit direction d and foot point F (nearest to the origin);
//   samples q_k = F + (k+1/2) step d (level pixels), each weighted by
//   step * s fine pixels; value at q = bilinear interpolant of the level image,
//   zero outside.  The forward sums samples along each ray; the transpose
//   gathers, for each pixel, every (ray, sample) pair whose bilinear hat covers
//   the pixel.  Both visit exactly the samples strictly inside the image box.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "pnp_internal.cuh"

namespace pnp {

std::atomic<uint64_t> g_launches{0};

namespace {
thread_local bool t_persistent = false;
}
bool persistent_mode() { return t_persistent; }
void set_persistent_mode(bool on) { t_persistent = on; }

namespace {

constexpr float kMagic = 12582912.0f;      // 1.5 * 2^23: x + kMagic rounds x to an integer
constexpr int kMagicBits = 0x4B400000;     // bit pattern of kMagic

__host__ __device__ inline int div_up(long a, long b) { return (int)((a + b - 1) / b); }

// ------------------------------------------------------------------ set-up (FP64)
// One thread per (view, bin): the ray's geometry in double precision, rounded once.
__global__ void k_setup_rays(int n, int s, int n_views, int n_det, double dso, double ddo,
                             double pitch, double angle0, double span, double step,
                             float4* __restrict__ rayf, float2* __restrict__ rayi,
                             int2* __restrict__ rayk, float4* __restrict__ view)
{
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)n_views * n_det) return;
    int v = (int)(idx / n_det), j = (int)(idx % n_det);
    const int ns = n / s;
    double beta = angle0 + span * (double)v / (double)n_views;
    double cb = cos(beta), sb = sin(beta);
    double sx = dso * cb, sy = dso * sb;
    double u = ((double)j - 0.5 * (double)(n_det - 1)) * pitch;
    double px = -ddo * cb - u * sb, py = -ddo * sb + u * cb;
    double ex = px - sx, ey = py - sy;
    double len = sqrt(ex * ex + ey * ey);
    double dx = ex / len, dy = ey / len;
    double sd = sx * dx + sy * dy;
    // foot point in level index units (pixel centre ix at ix)
    double fx = (sx - sd * dx) / s + 0.5 * (ns - 1);
    double fy = (sy - sd * dy) / s + 0.5 * (ns - 1);
    const int c0 = ns / 2;   // origin of the primed frame: index column/row c0
    // samples strictly inside the box (-1, ns)^2 of index coordinates
    double tlo = -1e300, thi = 1e300;
    const double lo = -1.0, hi = (double)ns;
    if (fabs(dx) > 0.0) {
        double t1 = (lo - fx) / dx, t2 = (hi - fx) / dx;
        tlo = fmax(tlo, fmin(t1, t2));
        thi = fmin(thi, fmax(t1, t2));
    } else if (!(fx > lo && fx < hi)) {
        thi = tlo;
    }
    if (fabs(dy) > 0.0) {
        double t1 = (lo - fy) / dy, t2 = (hi - fy) / dy;
        tlo = fmax(tlo, fmin(t1, t2));
        thi = fmin(thi, fmax(t1, t2));
    } else if (!(fy > lo && fy < hi)) {
        thi = tlo;
    }
    int klo = 0, khi = -1;
    if (thi > tlo) {
        // (k + 1/2) step > tlo  and  (k + 1/2) step < thi
        klo = (int)floor(tlo / step - 0.5) + 1;
        khi = (int)ceil(thi / step - 0.5) - 1;
        if (khi < klo) { klo = 0; khi = -1; }
    }
    rayf[idx] = make_float4((float)(fx - c0 + 1.5), (float)(fy - c0 + 1.5), (float)dx, (float)dy);
    const double tiny = 1e-12;
    double adx = fabs(dx) < tiny ? copysign(tiny, dx) : dx;
    double ady = fabs(dy) < tiny ? copysign(tiny, dy) : dy;
    rayi[idx] = make_float2((float)(1.0 / adx), (float)(1.0 / ady));
    rayk[idx] = make_int2(klo, khi);
    if (j == 0) view[v] = make_float4((float)cb, (float)sb, (float)(dso / s), (float)((dso + ddo) / pitch));
}

// ------------------------------------------------------------------ coefficient image
// quad[iy0+2][ix0+2] holds the bilinear coefficients of the cell whose lower
// corner is level pixel (ix0, iy0), in the centred variables u, w in [-1/2, 1/2]:
//   f = c0 + u c1 + w (c2 + u c3)
// with a = I(ix0,iy0), b = I(ix0+1,iy0), c = I(ix0,iy0+1), d = I(ix0+1,iy0+1)
// (zero outside), I the s x s average pool of the fine image.
__device__ __forceinline__ float pooled(const float* __restrict__ fine, int n, int s, int ns, int i,
                                        int j)
{
    if (i < 0 || j < 0 || i >= ns || j >= ns) return 0.0f;
    if (s == 1) return __ldg(fine + (long)j * n + i);
    float acc = 0.0f;
    for (int b = 0; b < s; ++b)
        for (int a = 0; a < s; ++a) acc += __ldg(fine + (long)(j * s + b) * n + (i * s + a));
    return acc * (1.0f / (float)(s * s));
}

// pooled() read with one vector load per fine row (float2 / float4 for s = 2 /
// 4), summed in pooled()'s order (rows outer, columns inner, from 0), so the
// same bits.  `vec`: the fine image's base is aligned to the vector (the
// offsets j s n + i s and image strides n^2 are multiples of s floats);
// otherwise, and for other s, pooled() itself.
__device__ __forceinline__ float pooled_rows(const float* __restrict__ fine, int n, int s, int ns, int i, int j,
                                             bool vec)
{
    if (!vec || (s != 2 && s != 4)) return pooled(fine, n, s, ns, i, j);
    if (i < 0 || j < 0 || i >= ns || j >= ns) return 0.0f;
    const float* p = fine + (long)j * s * n + (long)i * s;
    float acc = 0.0f;
    if (s == 2) {
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const float2 v = __ldg(reinterpret_cast<const float2*>(p + (long)b * n));
            acc += v.x;
            acc += v.y;
        }
    } else {
        float4 v[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) v[b] = __ldg(reinterpret_cast<const float4*>(p + (long)b * n));
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            acc += v[b].x;
            acc += v[b].y;
            acc += v[b].z;
            acc += v[b].w;
        }
    }
    return acc * (1.0f / (float)(s * s));
}

struct PrepTable {
    PrepArgs c[kMaxClasses];
    long ibegin[kMaxClasses + 1];  // cumulative image counts
    int count;
};

// grid.x covers the cells of one image (32-bit indices), grid.y the images of
// all classes (strided when there are more than gridDim.y).
__global__ void k_prep_quad(const PrepTable t)
{
    pdl_begin();
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    for (long item = blockIdx.y; item < t.ibegin[t.count]; item += gridDim.y) {
        int c = 0;
#pragma unroll
        for (int k = 1; k < kMaxClasses; ++k)
            if (k < t.count && item >= t.ibegin[k]) c = k;
        const PrepArgs& a = t.c[c];
        const int qw = a.qw;
        if (cell >= qw * qw) continue;
        const long inst = item - t.ibegin[c];
        const int qy = cell / qw, qx = cell - qy * qw;
        const int n = a.n, s = a.s, ns = n / s;
        const float* f = a.fine + inst * n * n;
        const bool vec = (reinterpret_cast<uintptr_t>(a.fine) & (uintptr_t)(4 * min(s, 4) - 1)) == 0;
        const int ix0 = qx - kPad, iy0 = qy - kPad;
        const float pa = pooled_rows(f, n, s, ns, ix0, iy0, vec), pb = pooled_rows(f, n, s, ns, ix0 + 1, iy0, vec);
        const float pc = pooled_rows(f, n, s, ns, ix0, iy0 + 1, vec);
        const float pd = pooled_rows(f, n, s, ns, ix0 + 1, iy0 + 1, vec);
        a.quad[inst * qw * qw + cell] = make_quad(pa, pb, pc, pd);
    }
}

// Image-interleaved coefficient image, quad[(qy * qw + qx) * B + b].  A CTA
// builds ROWS x kIlCells cells for all B images of its class: it stages the
// ROWS + 1 level-image rows those cells read (pooled for s > 1) in shared
// memory, 64 images at a time for ROWS = 1 and 32 for ROWS = 4 (a warp per
// staged row of one image), then writes the cells with the image index
// fastest, so that both the image reads and the cell writes are contiguous.  ROWS = 4 for level images of 256 or more (each staged row serves
// two rows of cells, and a CTA's fixed costs spread over four times the cells:
// 39 -> 29 us at 16 x 512^2), 1 below (enough CTAs for the small images).
constexpr int kIlCells = 32;

struct PrepIlTable {
    PrepArgs c[kMaxClasses];
    long begin[kMaxClasses + 1];   // cumulative CTA counts (row blocks x segments)
    int count;
};

template <int ROWS>
__device__ __forceinline__ void k_prep_quad_il_item(const PrepIlTable& t, const long vb)
{
    constexpr int kIlRows = ROWS;
    constexpr int kIlImages = ROWS == 1 ? 64 : 32;   // images staged at a time
    constexpr int C1 = kIlCells + 1, R1 = kIlRows + 1;
    __shared__ float lv[kIlImages * R1 * C1];              // [image][row][column]
    int c = 0;
#pragma unroll
    for (int k = 1; k < kMaxClasses; ++k)
        if (k < t.count && (long)vb >= t.begin[k]) c = k;
    const PrepArgs& a = t.c[c];
    const int qw = a.qw, B = a.batch;
    const int segs = (qw + kIlCells - 1) / kIlCells;
    const int local = (int)((long)vb - t.begin[c]);
    const int rblk = local / segs;
    const int qy0 = rblk * kIlRows, qx0 = (local - rblk * segs) * kIlCells;
    const int n = a.n, s = a.s, ns = n / s;
    const int cells = min(kIlCells, qw - qx0), rows = min(kIlRows, qw - qy0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
    const bool vec = (reinterpret_cast<uintptr_t>(a.fine) & (uintptr_t)(4 * min(s, 4) - 1)) == 0;
    for (int b0 = 0; b0 < B; b0 += kIlImages) {
        const int nb = min(kIlImages, B - b0);
        if (b0 > 0) __syncthreads();
        // a warp stages columns 0..31 of one level row of one image at a time
        // (lane = column), then one thread per row its 33rd column
        for (int it = warp; it < nb * R1; it += warps) {
            const int b = it / R1, r = it - b * R1;
            lv[it * C1 + lane] = pooled_rows(a.fine + (long)(b0 + b) * n * n, n, s, ns, qx0 - kPad + lane,
                                             qy0 - kPad + r, vec);
        }
        for (int it = threadIdx.x; it < nb * R1; it += blockDim.x) {
            const int b = it / R1, r = it - b * R1;
            lv[it * C1 + kIlCells] = pooled_rows(a.fine + (long)(b0 + b) * n * n, n, s, ns, qx0 - kPad + kIlCells,
                                                 qy0 - kPad + r, vec);
        }
        __syncthreads();
        // thread -> image b = tid % nb (fixed), cells tid / nb, + cstep, ...: two
        // divisions per thread, consecutive threads on consecutive images of a cell
        const int b = threadIdx.x % nb, cstep = blockDim.x / nb;
        if (threadIdx.x < cstep * nb) {
            for (int r = 0; r < rows; ++r) {
                const float* l0 = lv + (b * R1 + r) * C1;
                float4* qrow = a.quad + ((long)(qy0 + r) * qw + qx0) * B + b0 + b;
                for (int cx = threadIdx.x / nb; cx < cells; cx += cstep)
                    qrow[(long)cx * B] = make_quad(l0[cx], l0[cx + 1], l0[C1 + cx], l0[C1 + cx + 1]);
            }
        }
    }
}

template <int ROWS>
__global__ void __launch_bounds__(256, 8) k_prep_quad_il(const PrepIlTable t)
{
    pdl_begin();
    k_prep_quad_il_item<ROWS>(t, (long)blockIdx.x);
}

// persistent form (PNP_RUN_PERSISTENT): as many CTAs as fit at once walk the items
template <int ROWS>
__global__ void __launch_bounds__(256, 8) k_prep_quad_il_persistent(const PrepIlTable t)
{
    pdl_begin();
    const long total = t.begin[t.count];
    for (long vb = blockIdx.x; vb < total; vb += gridDim.x) {
        if (vb != (long)blockIdx.x) __syncthreads();   // the previous item's shared memory is free
        k_prep_quad_il_item<ROWS>(t, vb);
    }
}

// ------------------------------------------------------------------ forward A_s
// Warp = R rays x Q phases (R*Q = 32): lane (r, q) sums the samples k = k_lo + q,
// k_lo + q + Q, ... of ray r into four interleaved partial sums (independent
// chains keep four loads in flight); the four, then the Q lanes' sums, are
// combined in a fixed order, so the result is deterministic.  One 16-byte load
// per sample.  A CTA (8 warps) takes 8R adjacent bins of one view; CTAs are
// numbered from the detector's centre outwards, all views of a rank together,
// so the long central rays go first and the last wave holds the short rays at
// the fan's edges (a shorter tail than in bin order).
struct FwdTable {
    FwdArgs c[kMaxClasses];
    long begin[kMaxClasses + 1];   // cumulative CTA counts (batch * n_sub * bin blocks)
    int count;
};

constexpr int kFwdWarps = 8;       // warps per forward CTA

template <int Q>
__device__ __forceinline__ void k_forward_item(const FwdTable& t, const long vb)
{
    constexpr int R = 32 / Q;
    constexpr int RB = kFwdWarps * R;   // bins per CTA
    const int lane = threadIdx.x & 31;
    const int r = lane / Q, q = lane % Q;
    const long cta = vb;
    int c = 0;
#pragma unroll
    for (int k = 1; k < kMaxClasses; ++k)
        if (k < t.count && cta >= t.begin[k]) c = k;
    const FwdArgs& a = t.c[c];
    const int nb = (a.n_det + RB - 1) / RB;
    const long per_inst = (long)a.n_sub * nb;
    const long local = cta - t.begin[c];
    const int inst = (int)(local / per_inst);
    const int rem = (int)(local - (long)inst * per_inst);
    const int rank = rem / a.n_sub, vs = rem - rank * a.n_sub;
    const int mid = nb >> 1;
    const int blk = (rank & 1) ? mid - ((rank + 1) >> 1) : mid + (rank >> 1);
    const int j = blk * RB + (threadIdx.x >> 5) * R + r;
    const bool active = j < a.n_det;
    float acc = 0.0f;
    long out_idx = 0;
    int v = 0;
    if (active) {
        v = a.first_view + vs * a.view_step;
        out_idx = a.out_il ? ((long)vs * a.n_det + j) * a.batch + inst : ((long)inst * a.n_sub + vs) * a.n_det + j;
        const float4 f = __ldg(a.rayf + (long)v * a.n_det + j);
        const int2 kr = __ldg(a.rayk + (long)v * a.n_det + j);
        const float4* __restrict__ img = a.quad + (long)inst * a.quad_stride;
        const int qw = a.qw;
        // cell iy qw + ix as bits(Y + kMagic) qw + bits(X + kMagic) - bias (qw + 1)
        // modulo 2^32, with ix = bits(X + kMagic) - bias (likewise iy)
        const int bias = kMagicBits - (qw - 3) / 2;   // column = round(X') + c0
        const unsigned cbias = (unsigned)bias * (unsigned)(qw + 1);
        // sample k at F + (k + 1/2) step d, as k (step d) + (F + step d / 2)
        const float sx = a.step * f.z, sy = a.step * f.w;
        const float hx = fmaf(0.5f * a.step, f.z, f.x), hy = fmaf(0.5f * a.step, f.w, f.y);
        float kf = (float)(kr.x + q);                 // sample indices below 2^24: exact
        const float dk = (float)Q;
        float acc2 = 0.0f, acc3 = 0.0f, acc4 = 0.0f;
        auto smp = [&](float kk) {
            const float X = fmaf(kk, sx, hx);
            const float Y = fmaf(kk, sy, hy);
            const float mx = __fadd_rn(X, kMagic);
            const float my = __fadd_rn(Y, kMagic);
            const float u = __fsub_rn(X, __fsub_rn(mx, kMagic));
            const float w = __fsub_rn(Y, __fsub_rn(my, kMagic));
            const unsigned ci = (unsigned)__float_as_int(my) * (unsigned)qw + (unsigned)__float_as_int(mx) - cbias;
            const float4 cq = __ldg(img + ci);
            return fmaf(w, fmaf(u, cq.w, cq.z), fmaf(u, cq.y, cq.x));
        };
        int k = kr.x + q;
#pragma unroll 2
        for (; k + 3 * Q <= kr.y; k += 4 * Q) {
            acc += smp(kf);
            acc2 += smp(kf + dk);
            acc3 += smp(kf + 2.0f * dk);
            acc4 += smp(kf + 3.0f * dk);
            kf += 4.0f * dk;
        }
        for (; k <= kr.y; k += Q) {
            acc += smp(kf);
            kf += dk;
        }
        acc = (acc + acc2) + (acc3 + acc4);
    }
#pragma unroll
    for (int o = Q / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (active && q == 0) {
        const long bi = ((long)inst * a.n_views + v) * a.n_det + j;
        float val = a.weight * acc;
        if (a.b) val -= __ldg(a.b + bi);
        if (a.w) val *= __ldg(a.w + bi);
        a.out[out_idx] = val;
    }
}

template <int Q>
__global__ void __launch_bounds__(32 * kFwdWarps, 4) k_forward(const FwdTable t)
{
    pdl_begin();
    k_forward_item<Q>(t, (long)blockIdx.x);
}

// persistent form (PNP_RUN_PERSISTENT): as many CTAs as fit at once walk the items
template <int Q>
__global__ void __launch_bounds__(32 * kFwdWarps, 4) k_forward_persistent(const FwdTable t)
{
    pdl_begin();
    const long total = t.begin[t.count];
    for (long vb = blockIdx.x; vb < total; vb += gridDim.x) {
        k_forward_item<Q>(t, vb);
    }
}

// Forward projector on an image-interleaved coefficient image.  A warp takes one
// ray for all images of its class: lane (g, i) = (lane / 8, lane % 8) sums the
// samples k = k_lo + g, k_lo + g + 4, ... of images i, i + 8, ..., i + 8 (IPL - 1),
// so the position and cell of a sample are computed once for 8 IPL images and
// each load instruction reads whole 128-byte lines (8 images' cells), 4
// consecutive samples at a time; the four sample groups are joined in a fixed
// order.  A CTA (4 warps) takes 4 adjacent bins of one view, CTAs numbered from
// the detector's centre outwards as in k_forward.
constexpr int kFwdIlWarps = 4;

template <int IPL>
__device__ __forceinline__ void k_forward_il_item(const FwdTable& t, const long vb)
{
    const int lane = threadIdx.x & 31;
    const int sg = lane >> 3, li = lane & 7;
    const long cta = vb;
    int c = 0;
#pragma unroll
    for (int k = 1; k < kMaxClasses; ++k)
        if (k < t.count && cta >= t.begin[k]) c = k;
    const FwdArgs& a = t.c[c];
    const int nb = (a.n_det + kFwdIlWarps - 1) / kFwdIlWarps;
    const int per_chunk = a.n_sub * nb;
    const int local = (int)(cta - t.begin[c]);
    const int chunk = local / per_chunk;                    // images [8 IPL chunk, 8 IPL (chunk + 1))
    const int rem = local - chunk * per_chunk;
    const int rank = rem / a.n_sub, vs = rem - rank * a.n_sub;
    const int mid = nb >> 1;
    const int blk = (rank & 1) ? mid - ((rank + 1) >> 1) : mid + (rank >> 1);
    const int j = blk * kFwdIlWarps + (threadIdx.x >> 5);
    if (j >= a.n_det) return;                                  // whole warps only
    const int v = a.first_view + vs * a.view_step;
    const float4 f = __ldg(a.rayf + (long)v * a.n_det + j);
    const int2 kr = __ldg(a.rayk + (long)v * a.n_det + j);
    const int B = a.batch, qw = a.qw;
    const int i0 = chunk * 8 * IPL + li;                     // this lane's first image
    // cell iy qw + ix with ix = bits(X + kMagic) - bias (likewise iy), formed as
    // bits(Y + kMagic) qw + bits(X + kMagic) - bias (qw + 1) modulo 2^32
    const int bias = kMagicBits - (qw - 3) / 2;             // column = round(X') + c0
    const unsigned cbias = (unsigned)bias * (unsigned)(qw + 1);
    // sample k at F + (k + 1/2) step d, as k (step d) + (F + step d / 2)
    const float sx = a.step * f.z, sy = a.step * f.w;
    const float hx = fmaf(0.5f * a.step, f.z, f.x), hy = fmaf(0.5f * a.step, f.w, f.y);
    bool valid[IPL];
#pragma unroll
    for (int q = 0; q < IPL; ++q) valid[q] = i0 + 8 * q < B;
    float acc[IPL];
#pragma unroll
    for (int q = 0; q < IPL; ++q) acc[q] = 0.0f;
    const float4* __restrict__ img = a.quad + i0;
    auto smp = [&](float kf) {
        const float X = fmaf(kf, sx, hx);
        const float Y = fmaf(kf, sy, hy);
        const float mx = __fadd_rn(X, kMagic);
        const float my = __fadd_rn(Y, kMagic);
        const float u = __fsub_rn(X, __fsub_rn(mx, kMagic));
        const float w = __fsub_rn(Y, __fsub_rn(my, kMagic));
        const unsigned ci = (unsigned)__float_as_int(my) * (unsigned)qw + (unsigned)__float_as_int(mx) - cbias;
        const float4* cell = img + (size_t)ci * (unsigned)B;
#pragma unroll
        for (int q = 0; q < IPL; ++q) {
            if (!valid[q]) continue;
            const float4 cq = __ldg(cell + 8 * q);
            acc[q] += fmaf(w, fmaf(u, cq.w, cq.z), fmaf(u, cq.y, cq.x));
        }
    };
    float kf = (float)(kr.x + sg);
    const float klast = (float)kr.y;                         // sample indices below 2^24: exact
#pragma unroll 1
    for (; kf + 4.0f <= klast; kf += 8.0f) {
        smp(kf);
        smp(kf + 4.0f);
    }
    if (kf <= klast) smp(kf);
#pragma unroll
    for (int q = 0; q < IPL; ++q) {
        acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], 8);
        acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], 16);
    }
    if (sg != 0) return;
    const long out_row = (long)vs * a.n_det + j;
    const long b_row = (long)v * a.n_det + j;
#pragma unroll
    for (int q = 0; q < IPL; ++q) {
        if (!valid[q]) continue;
        const int inst = i0 + 8 * q;
        const long bi = (long)inst * a.n_views * a.n_det + b_row;
        float val = a.weight * acc[q];
        if (a.b) val -= __ldg(a.b + bi);
        if (a.w) val *= __ldg(a.w + bi);
        a.out[a.out_il ? out_row * B + inst : (long)inst * a.n_sub * a.n_det + out_row] = val;
    }
}

template <int IPL>
__global__ void __launch_bounds__(32 * kFwdIlWarps) k_forward_il(const FwdTable t)
{
    pdl_begin();
    k_forward_il_item<IPL>(t, (long)blockIdx.x);
}

// persistent form (PNP_RUN_PERSISTENT): as many CTAs as fit at once walk the items
template <int IPL>
__global__ void __launch_bounds__(32 * kFwdIlWarps) k_forward_il_persistent(const FwdTable t)
{
    pdl_begin();
    const long total = t.begin[t.count];
    for (long vb = blockIdx.x; vb < total; vb += gridDim.x) {
        k_forward_il_item<IPL>(t, vb);
    }
}

// ------------------------------------------------------------------ transpose A_s^T
// Pixel-driven gather.  Thread (2x2 pixel block, g) gathers the views g, g+G,
// g+2G, ... of the subset: for each view, the detector interval that the
// block's hat support can shadow; for every bin in it, a perpendicular-distance
// test of the ray against the support; for each ray that meets it, the hat
// products of the block's four pixels summed over the ray's samples near the
// block.  The G partial sums are added in a fixed order through shared memory,
// so the result is deterministic for a given G (a function of the problem
// size).  CTA = 8 x 4 blocks (16 x 8 pixels) x G view groups, so the 32
// threads of a warp walk the same views in step; or 4 x 4 blocks x G, two view
// groups per warp, which allows up to 64 groups (one view per thread for
// subsets of up to 64 views) and four times as many CTAs, so that the CTAs
// pack the SMs with a smaller partial last wave.
constexpr int kBack2TileX = 8;    // a warp = 8 x 4 blocks of one view group
constexpr int kBack2TileY = 4;
constexpr int kBack2MaxGroups = 16;

// The four pixels share the view set-up and the candidate rays; their union
// support is the 3 x 3 square around the block centre, whose extent across and
// along a ray of direction d is 3 (|d_x| + |d_y|) <= 3 sqrt 2 = 2 rho.  A ray
// meets it only if its distance from the centre is below half that, and then
// only samples whose projection lies within half that of the centre's can touch
// a pixel: floor(3 (|d_x| + |d_y|) / step) + 1 samples (7 to 9 for step 1/2).
// Each sample evaluates the two x hats and two y hats once (saturated 1 - |x|)
// and feeds four products.
struct BackTable {
    BackArgs c[kMaxClasses];
    long begin[kMaxClasses + 1];   // cumulative CTA counts (batch * tiles)
    int count;
};

template <int NWIN, int TX>
__device__ __forceinline__ void k_backward2x2_item(const BackTable& t, const long vb)
{
    const int tx = threadIdx.x, ty = threadIdx.y, g = threadIdx.z, G = blockDim.z;
    int c = 0;
#pragma unroll
    for (int k = 1; k < kMaxClasses; ++k)
        if (k < t.count && (long)vb >= t.begin[k]) c = k;
    const BackArgs& a = t.c[c];
    const int nb = (a.ns + 1) / 2;                             // blocks per side
    const int tiles_x = (nb + TX - 1) / TX;
    const int tiles_y = (nb + kBack2TileY - 1) / kBack2TileY;
    const long local = (long)vb - t.begin[c];
    const int tiles = tiles_x * tiles_y;
    const int inst = (int)(local / tiles);
    const int tile = (int)(local - (long)inst * tiles);
    const int bx = (tile % tiles_x) * TX + tx;
    const int by = (tile / tiles_x) * kBack2TileY + ty;
    const bool inside = bx < nb && by < nb;
    extern __shared__ float4 part[];                           // [G][TX * kBack2TileY]
    float t00 = 0.0f, t10 = 0.0f, t01 = 0.0f, t11 = 0.0f;
    if (inside) {
        const int ix = 2 * bx, iy = 2 * by;
        const float half = 0.5f * (float)(a.ns - 1);
        const float cx = (float)ix + 0.5f - half, cy = (float)iy + 0.5f - half;   // centred, level units
        const int c0 = a.ns / 2;
        const float px = (float)(ix - c0) + 2.0f, py = (float)(iy - c0) + 2.0f;   // primed frame
        const float jc = 0.5f * (float)(a.n_det - 1);
        const float inv_step = 1.0f / a.step;
        const float rho = 2.12132034f;                           // 1.5 sqrt(2)
        const int nwin = NWIN > 0 ? NWIN : (int)floorf(2.0f * rho * inv_step) + 1;
        const int js = res_js(a);
        const float* __restrict__ res = a.res + (long)inst * res_is(a);
        for (int vs = g; vs < a.n_sub; vs += G) {
            const int v = a.first_view + vs * a.view_step;
            const float4 vp = __ldg(a.view + v);   // cos b, sin b, dso/s, (dso+ddo)/pitch
            const float along = cx * vp.x + cy * vp.y;
            const float lat = cy * vp.x - cx * vp.y;
            const float inv = __fdividef(1.0f, vp.z - along);
            const float uj = vp.w * lat * inv + jc;
            // conservative shadow half-width (bins) of the disc of radius rho
            const float invp = inv * (1.0f + 2.0f * rho * inv);
            const float T = (fabsf(lat) + rho) * invp;
            const float hw = rho * vp.w * fmaf(T, T, 1.0f) * invp * 1.01f + 0.02f;
            const int jlo = max(0, (int)ceilf(uj - hw));
            const int jhi = min(a.n_det - 1, (int)floorf(uj + hw));
            const long base = (long)v * a.n_det;
            const float* __restrict__ rrow = res + (long)vs * a.n_det * js;
            float4 fn = make_float4(0.0f, 0.0f, 1.0f, 0.0f);
            float rn = 0.0f;
            if (jlo <= jhi) {
                fn = __ldg(a.rayf + base + jlo);
                rn = __ldg(rrow + (long)jlo * js);
            }
            for (int j = jlo; j <= jhi; ++j) {
                const float4 f = fn;
                const float r = rn;
                if (j < jhi) {
                    fn = __ldg(a.rayf + base + j + 1);
                    rn = __ldg(rrow + (long)(j + 1) * js);
                }
                const float ax = px - f.x, ay = py - f.y;
                const float e = ax * f.w - ay * f.z;
                const float hwid = 1.5f * (fabsf(f.z) + fabsf(f.w));   // half the support's width across / along d
                if (fabsf(e) >= hwid) continue;
                const float tau = fmaf(ax, f.z, ay * f.w);
                const float k0 = ceilf(fmaf(tau - hwid, inv_step, -0.5f));
                const int cnt = (int)(2.0f * hwid * inv_step) + 1;
                const float t0 = (k0 + 0.5f) * a.step;
                const float X0 = fmaf(t0, f.z, -ax), Y0 = fmaf(t0, f.w, -ay);
                const float xa0 = X0 + 0.5f, xb0 = X0 - 0.5f;    // relative to the left / right pixel
                const float ya0 = Y0 + 0.5f, yb0 = Y0 - 0.5f;    // relative to the lower / upper pixel
                const float sx = a.step * f.z, sy = a.step * f.w;
                float w00 = 0.0f, w10 = 0.0f, w01 = 0.0f, w11 = 0.0f;
                auto sample = [&](float fm) {
                    const float hxa = __saturatef(1.0f - fabsf(fmaf(fm, sx, xa0)));
                    const float hxb = __saturatef(1.0f - fabsf(fmaf(fm, sx, xb0)));
                    const float hya = __saturatef(1.0f - fabsf(fmaf(fm, sy, ya0)));
                    const float hyb = __saturatef(1.0f - fabsf(fmaf(fm, sy, yb0)));
                    w00 = fmaf(hxa, hya, w00);
                    w10 = fmaf(hxb, hya, w10);
                    w01 = fmaf(hxa, hyb, w01);
                    w11 = fmaf(hxb, hyb, w11);
                };
                if (NWIN > 0) {
#pragma unroll
                    for (int m = 0; m < (NWIN > 2 ? NWIN - 2 : 1); ++m) sample((float)m);
                    if (cnt > NWIN - 2) sample((float)(NWIN - 2));
                    if (cnt > NWIN - 1) sample((float)(NWIN - 1));
                } else {
                    for (int m = 0; m < min(cnt, nwin); ++m) sample((float)m);
                }
                t00 = fmaf(w00, r, t00);
                t10 = fmaf(w10, r, t10);
                t01 = fmaf(w01, r, t01);
                t11 = fmaf(w11, r, t11);
            }
        }
    }
    constexpr int kSlots = TX * kBack2TileY;
    const int slot = ty * TX + tx;
    part[g * kSlots + slot] = make_float4(t00, t10, t01, t11);
    __syncthreads();
    if (g != 0 || !inside) return;
    float s00 = 0.0f, s10 = 0.0f, s01 = 0.0f, s11 = 0.0f;
    for (int q = 0; q < G; ++q) {
        const float4 pq = part[q * kSlots + slot];
        s00 += pq.x; s10 += pq.y; s01 += pq.z; s11 += pq.w;
    }
    const float vals[4] = {a.scale * s00, a.scale * s10, a.scale * s01, a.scale * s11};
    const int s = a.s;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int ix = 2 * bx + (q & 1), iy = 2 * by + (q >> 1);
        if (ix >= a.ns || iy >= a.ns) continue;
        if (a.mode == kBackRaw) {
            a.out[((long)inst * a.ns + iy) * a.ns + ix] = vals[q];
            continue;
        }
        for (int bb = 0; bb < s; ++bb) {
            const long row = ((long)inst * a.n + (long)iy * s + bb) * a.n + (long)ix * s;
            for (int aa = 0; aa < s; ++aa) {
                if (a.mode == kBackGradFine)
                    a.out[row + aa] = vals[q];
                else
                    a.out[row + aa] = __ldg(a.y + row + aa) - a.eta * vals[q];
            }
        }
    }
}

template <int NWIN, int TX>
__global__ void __launch_bounds__(1024, 1) k_backward2x2(const BackTable t)
{
    pdl_begin();
    k_backward2x2_item<NWIN, TX>(t, (long)blockIdx.x);
}

// persistent form (PNP_RUN_PERSISTENT): as many CTAs as fit at once walk the items
template <int NWIN, int TX>
__global__ void __launch_bounds__(1024, 1) k_backward2x2_persistent(const BackTable t)
{
    pdl_begin();
    const long total = t.begin[t.count];
    for (long vb = blockIdx.x; vb < total; vb += gridDim.x) {
        if (vb != (long)blockIdx.x) __syncthreads();   // the previous item's shared memory is free
        k_backward2x2_item<NWIN, TX>(t, vb);
    }
}

// Batched form of the gather for a class of B images that share one geometry:
// the rays, their samples and therefore every hat product are the same for all
// images; only the residuals differ.  A thread (2x2 pixel block, view group g)
// now covers a chunk of BC images: each (ray, sample) hat product is computed
// once and applied to the BC residuals (BC x 4 accumulators per thread).  The
// view, ray and sample order of every accumulator and the fixed-order sum over
// the G view groups are those of k_backward2x2 with the same TX and G, so the
// result is bitwise the same as the unbatched gather's.  The view-group sums go
// through shared memory in rounds of RB images (RB from the host, so that
// G x RB x slots float4 fit the CTA's shared memory).
struct BackBatchTable {
    BackArgs c[kMaxClasses];
    long begin[kMaxClasses + 1];   // cumulative CTA counts (tiles * chunks of BC images)
    int count;
    int rb;                        // images per reduction round
};

constexpr int kBackBatchThreads = 512;

template <int NWIN, int TX, int BC>
__device__ __forceinline__ void k_backward_batch_item(const BackBatchTable& t, const long vb)
{
    const int tx = threadIdx.x, ty = threadIdx.y, g = threadIdx.z, G = blockDim.z;
    int c = 0;
#pragma unroll
    for (int k = 1; k < kMaxClasses; ++k)
        if (k < t.count && (long)vb >= t.begin[k]) c = k;
    const BackArgs& a = t.c[c];
    const int nb = (a.ns + 1) / 2;                             // blocks per side
    const int tiles_x = (nb + TX - 1) / TX;
    const int tiles_y = (nb + kBack2TileY - 1) / kBack2TileY;
    const long local = (long)vb - t.begin[c];
    const int tiles = tiles_x * tiles_y;
    const int chunk = (int)(local / tiles);
    const int tile = (int)(local - (long)chunk * tiles);
    const int bx0 = (tile % tiles_x) * TX, by0 = (tile / tiles_x) * kBack2TileY;
    const int bx = bx0 + tx, by = by0 + ty;
    const int i0 = chunk * BC;
    const int ni = min(BC, a.batch - i0);                      // images in this chunk
    const bool inside = bx < nb && by < nb;
    const long istride = res_is(a);                            // residual stride between images
    const int js = res_js(a);                                  // ... and between bins
    // image-interleaved residuals of a batch of a multiple of 4: the chunk's
    // residuals of a ray are contiguous and 16-byte aligned
    const bool vec = a.res_il && (a.batch & 3) == 0 && (BC & 3) == 0;
    // accumulators of images (2h, 2h + 1) as FP32x2 pairs: each lane of a packed
    // FMA rounds as the scalar FMA would
    float2 acc2[BC / 2][4];
#pragma unroll
    for (int h = 0; h < BC / 2; ++h) acc2[h][0] = acc2[h][1] = acc2[h][2] = acc2[h][3] = make_float2(0.0f, 0.0f);
    if (inside) {
        const int ix = 2 * bx, iy = 2 * by;
        const float half = 0.5f * (float)(a.ns - 1);
        const float cx = (float)ix + 0.5f - half, cy = (float)iy + 0.5f - half;   // centred, level units
        const int c0 = a.ns / 2;
        const float px = (float)(ix - c0) + 2.0f, py = (float)(iy - c0) + 2.0f;   // primed frame
        const float jc = 0.5f * (float)(a.n_det - 1);
        const float inv_step = 1.0f / a.step;
        const float rho = 2.12132034f;                           // 1.5 sqrt(2)
        const int nwin = NWIN > 0 ? NWIN : (int)floorf(2.0f * rho * inv_step) + 1;
        const float* __restrict__ res = a.res + (long)i0 * istride;
        for (int vs = g; vs < a.n_sub; vs += G) {
            const int v = a.first_view + vs * a.view_step;
            const float4 vp = __ldg(a.view + v);   // cos b, sin b, dso/s, (dso+ddo)/pitch
            const float along = cx * vp.x + cy * vp.y;
            const float lat = cy * vp.x - cx * vp.y;
            const float inv = __fdividef(1.0f, vp.z - along);
            const float uj = vp.w * lat * inv + jc;
            const float invp = inv * (1.0f + 2.0f * rho * inv);
            const float T = (fabsf(lat) + rho) * invp;
            const float hw = rho * vp.w * fmaf(T, T, 1.0f) * invp * 1.01f + 0.02f;
            const int jlo = max(0, (int)ceilf(uj - hw));
            const int jhi = min(a.n_det - 1, (int)floorf(uj + hw));
            const long base = (long)v * a.n_det;
            const float* __restrict__ rrow = res + (long)vs * a.n_det * js;
            float4 fn = make_float4(0.0f, 0.0f, 1.0f, 0.0f);
            if (jlo <= jhi) fn = __ldg(a.rayf + base + jlo);
            for (int j = jlo; j <= jhi; ++j) {
                const float4 f = fn;
                if (j < jhi) fn = __ldg(a.rayf + base + j + 1);
                const float ax = px - f.x, ay = py - f.y;
                const float e = ax * f.w - ay * f.z;
                const float hwid = 1.5f * (fabsf(f.z) + fabsf(f.w));
                if (fabsf(e) >= hwid) continue;
                // the chunk's residuals of this ray, in flight while the hats are computed
                float r[BC];
                if (vec) {
                    const float4* r4 = reinterpret_cast<const float4*>(rrow + (long)j * js);
#pragma unroll
                    for (int b = 0; b < BC; b += 4) {
                        const float4 q = b < ni ? __ldg(r4 + b / 4) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                        r[b] = q.x; r[b + 1] = q.y; r[b + 2] = q.z; r[b + 3] = q.w;
                    }
                } else {
#pragma unroll
                    for (int b = 0; b < BC; ++b) r[b] = b < ni ? __ldg(rrow + b * istride + (long)j * js) : 0.0f;
                }
                const float tau = fmaf(ax, f.z, ay * f.w);
                const float k0 = ceilf(fmaf(tau - hwid, inv_step, -0.5f));
                const int cnt = (int)(2.0f * hwid * inv_step) + 1;
                const float t0 = (k0 + 0.5f) * a.step;
                const float X0 = fmaf(t0, f.z, -ax), Y0 = fmaf(t0, f.w, -ay);
                const float xa0 = X0 + 0.5f, xb0 = X0 - 0.5f;
                const float ya0 = Y0 + 0.5f, yb0 = Y0 - 0.5f;
                const float sx = a.step * f.z, sy = a.step * f.w;
                float w00 = 0.0f, w10 = 0.0f, w01 = 0.0f, w11 = 0.0f;
                auto sample = [&](float fm) {
                    const float hxa = __saturatef(1.0f - fabsf(fmaf(fm, sx, xa0)));
                    const float hxb = __saturatef(1.0f - fabsf(fmaf(fm, sx, xb0)));
                    const float hya = __saturatef(1.0f - fabsf(fmaf(fm, sy, ya0)));
                    const float hyb = __saturatef(1.0f - fabsf(fmaf(fm, sy, yb0)));
                    w00 = fmaf(hxa, hya, w00);
                    w10 = fmaf(hxb, hya, w10);
                    w01 = fmaf(hxa, hyb, w01);
                    w11 = fmaf(hxb, hyb, w11);
                };
                if (NWIN > 0) {
#pragma unroll
                    for (int m = 0; m < (NWIN > 2 ? NWIN - 2 : 1); ++m) sample((float)m);
                    if (cnt > NWIN - 2) sample((float)(NWIN - 2));
                    if (cnt > NWIN - 1) sample((float)(NWIN - 1));
                } else {
                    for (int m = 0; m < min(cnt, nwin); ++m) sample((float)m);
                }
                const float2 v00 = make_float2(w00, w00), v10 = make_float2(w10, w10);
                const float2 v01 = make_float2(w01, w01), v11 = make_float2(w11, w11);
#pragma unroll
                for (int h = 0; h < BC / 2; ++h) {
                    const float2 rr = make_float2(r[2 * h], r[2 * h + 1]);
                    acc2[h][0] = __ffma2_rn(v00, rr, acc2[h][0]);
                    acc2[h][1] = __ffma2_rn(v10, rr, acc2[h][1]);
                    acc2[h][2] = __ffma2_rn(v01, rr, acc2[h][2]);
                    acc2[h][3] = __ffma2_rn(v11, rr, acc2[h][3]);
                }
            }
        }
    }
    // view-group sums in rounds of RB images: part[g][k][slot]
    extern __shared__ float4 part[];
    constexpr int kSlots = TX * kBack2TileY;
    const int slot = ty * TX + tx;
    const int RB = t.rb;
    const int nthr = kSlots * G;
    const int lt = (g * kBack2TileY + ty) * TX + tx;
    const int s = a.s;
    for (int b0 = 0; b0 < ni; b0 += RB) {
        if (b0 > 0) __syncthreads();
#pragma unroll
        for (int b = 0; b < BC; ++b)
            if (b >= b0 && b < b0 + RB)
                part[(g * RB + (b - b0)) * kSlots + slot] =
                    (b & 1) ? make_float4(acc2[b / 2][0].y, acc2[b / 2][1].y, acc2[b / 2][2].y, acc2[b / 2][3].y)
                            : make_float4(acc2[b / 2][0].x, acc2[b / 2][1].x, acc2[b / 2][2].x, acc2[b / 2][3].x);
        __syncthreads();
        for (int idx = lt; idx < RB * kSlots; idx += nthr) {
            const int k = idx / kSlots, sl = idx - k * kSlots;
            const int inst = i0 + b0 + k;
            const int obx = bx0 + sl % TX, oby = by0 + sl / TX;
            if (b0 + k >= ni || obx >= nb || oby >= nb) continue;
            float s00 = 0.0f, s10 = 0.0f, s01 = 0.0f, s11 = 0.0f;
            for (int q = 0; q < G; ++q) {
                const float4 pq = part[(q * RB + k) * kSlots + sl];
                s00 += pq.x; s10 += pq.y; s01 += pq.z; s11 += pq.w;
            }
            const float vals[4] = {a.scale * s00, a.scale * s10, a.scale * s01, a.scale * s11};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int ix = 2 * obx + (q & 1), iy = 2 * oby + (q >> 1);
                if (ix >= a.ns || iy >= a.ns) continue;
                if (a.mode == kBackRaw) {
                    a.out[((long)inst * a.ns + iy) * a.ns + ix] = vals[q];
                    continue;
                }
                for (int bb = 0; bb < s; ++bb) {
                    const long row = ((long)inst * a.n + (long)iy * s + bb) * a.n + (long)ix * s;
                    for (int aa = 0; aa < s; ++aa) {
                        if (a.mode == kBackGradFine)
                            a.out[row + aa] = vals[q];
                        else
                            a.out[row + aa] = __ldg(a.y + row + aa) - a.eta * vals[q];
                    }
                }
            }
        }
    }
}

template <int NWIN, int TX, int BC>
__global__ void __launch_bounds__(kBackBatchThreads, 1) k_backward_batch(const BackBatchTable t)
{
    pdl_begin();
    k_backward_batch_item<NWIN, TX, BC>(t, (long)blockIdx.x);
}

// persistent form (PNP_RUN_PERSISTENT): as many CTAs as fit at once walk the items
template <int NWIN, int TX, int BC>
__global__ void __launch_bounds__(kBackBatchThreads, 1) k_backward_batch_persistent(const BackBatchTable t)
{
    pdl_begin();
    const long total = t.begin[t.count];
    for (long vb = blockIdx.x; vb < total; vb += gridDim.x) {
        if (vb != (long)blockIdx.x) __syncthreads();   // the previous item's shared memory is free
        k_backward_batch_item<NWIN, TX, BC>(t, vb);
    }
}

// ------------------------------------------------------------------ transpose A_s^T from a stored table
// The gather's weights depend on the geometry only, so they can be computed once
// and stored: for every (view, 2x2 block) the bins of the rays that meet the
// block's support (ascending) and the four summed hat products of each, exactly
// as k_backward2x2 / k_backward_batch form them.  Blocks go in groups of 32 (tiles
// of 8 x 4 blocks, whose rays stay close together); the entries of a (view,
// group) are sliced-ELL: slot s
// of the group holds entry s of each of its 32 blocks, so a warp reads one
// slot as 32 consecutive float4 (weights) and 32 ints (bins, -1 past a block's
// own entries), and a group takes as many slots as its block with the most rays.
// Layout per level: hdr int2 [n_views][groups] (first slot, slots), weights
// float4 [slots][32], bins int [slots][32].  The gather then streams the table
// from HBM instead of evaluating the hats (about 2.3 entries of 20 B per block
// and view at 512^2 / 720 x 768); with the same view-group count G its sums are
// the bits of the two gathers (same weights, same view and ray order, same
// fixed-order sum over the view groups).

// per-view candidate bins of the block at (bx, by): the conservative shadow of its support
struct GatherFrame {
    float cx, cy, px, py, jc, inv_step, rho;
    int nwin;
};

template <int NWIN>
__device__ __forceinline__ GatherFrame gather_frame(const BackArgs& a, int bx, int by)
{
    GatherFrame f;
    const int ix = 2 * bx, iy = 2 * by;
    const float half = 0.5f * (float)(a.ns - 1);
    f.cx = (float)ix + 0.5f - half;
    f.cy = (float)iy + 0.5f - half;
    const int c0 = a.ns / 2;
    f.px = (float)(ix - c0) + 2.0f;
    f.py = (float)(iy - c0) + 2.0f;
    f.jc = 0.5f * (float)(a.n_det - 1);
    f.inv_step = 1.0f / a.step;
    f.rho = 2.12132034f;
    f.nwin = NWIN > 0 ? NWIN : (int)floorf(2.0f * f.rho * f.inv_step) + 1;
    return f;
}

__device__ __forceinline__ void gather_bins(const BackArgs& a, const GatherFrame& fr, int v, int& jlo, int& jhi)
{
    const float4 vp = __ldg(a.view + v);
    const float along = fr.cx * vp.x + fr.cy * vp.y;
    const float lat = fr.cy * vp.x - fr.cx * vp.y;
    const float inv = __fdividef(1.0f, vp.z - along);
    const float uj = vp.w * lat * inv + fr.jc;
    const float invp = inv * (1.0f + 2.0f * fr.rho * inv);
    const float T = (fabsf(lat) + fr.rho) * invp;
    const float hw = fr.rho * vp.w * fmaf(T, T, 1.0f) * invp * 1.01f + 0.02f;
    jlo = max(0, (int)ceilf(uj - hw));
    jhi = min(a.n_det - 1, (int)floorf(uj + hw));
}

// the four summed hat products of ray f on the block; false when the ray misses its support
template <int NWIN>
__device__ __forceinline__ bool gather_weights(const BackArgs& a, const GatherFrame& fr, const float4 f, float4& wq)
{
    const float ax = fr.px - f.x, ay = fr.py - f.y;
    const float e = ax * f.w - ay * f.z;
    const float hwid = 1.5f * (fabsf(f.z) + fabsf(f.w));
    if (fabsf(e) >= hwid) return false;
    const float tau = fmaf(ax, f.z, ay * f.w);
    const float k0 = ceilf(fmaf(tau - hwid, fr.inv_step, -0.5f));
    const int cnt = (int)(2.0f * hwid * fr.inv_step) + 1;
    const float t0 = (k0 + 0.5f) * a.step;
    const float X0 = fmaf(t0, f.z, -ax), Y0 = fmaf(t0, f.w, -ay);
    const float xa0 = X0 + 0.5f, xb0 = X0 - 0.5f;
    const float ya0 = Y0 + 0.5f, yb0 = Y0 - 0.5f;
    const float sx = a.step * f.z, sy = a.step * f.w;
    float w00 = 0.0f, w10 = 0.0f, w01 = 0.0f, w11 = 0.0f;
    auto sample = [&](float fm) {
        const float hxa = __saturatef(1.0f - fabsf(fmaf(fm, sx, xa0)));
        const float hxb = __saturatef(1.0f - fabsf(fmaf(fm, sx, xb0)));
        const float hya = __saturatef(1.0f - fabsf(fmaf(fm, sy, ya0)));
        const float hyb = __saturatef(1.0f - fabsf(fmaf(fm, sy, yb0)));
        w00 = fmaf(hxa, hya, w00);
        w10 = fmaf(hxb, hya, w10);
        w01 = fmaf(hxa, hyb, w01);
        w11 = fmaf(hxb, hyb, w11);
    };
    if (NWIN > 0) {
#pragma unroll
        for (int m = 0; m < (NWIN > 2 ? NWIN - 2 : 1); ++m) sample((float)m);
        if (cnt > NWIN - 2) sample((float)(NWIN - 2));
        if (cnt > NWIN - 1) sample((float)(NWIN - 1));
    } else {
        for (int m = 0; m < min(cnt, fr.nwin); ++m) sample((float)m);
    }
    wq = make_float4(w00, w10, w01, w11);
    return true;
}

// one warp per (view, group of 32 blocks): the group's slot count (its largest entry count)
__global__ void __launch_bounds__(256) k_table_count(const BackArgs a, int n_views, int* widths)
{
    const int nb = (a.ns + 1) / 2, groups = table_groups(a.ns);
    const long wid = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= (long)n_views * groups) return;                // whole warps
    const int v = (int)(wid / groups), k = (int)(wid - (long)v * groups);
    int bx, by;
    table_block(a.ns, k, lane, bx, by);
    int cnt = 0;
    if (bx < nb && by < nb) {
        const GatherFrame fr = gather_frame<0>(a, bx, by);
        int jlo, jhi;
        gather_bins(a, fr, v, jlo, jhi);
        const long base = (long)v * a.n_det;
        for (int j = jlo; j <= jhi; ++j) {
            const float4 f = __ldg(a.rayf + base + j);
            const float ax = fr.px - f.x, ay = fr.py - f.y;
            const float e = ax * f.w - ay * f.z;
            const float hwid = 1.5f * (fabsf(f.z) + fabsf(f.w));
            if (fabsf(e) < hwid) ++cnt;
        }
    }
    cnt = __reduce_max_sync(0xffffffffu, cnt);
    if (lane == 0) widths[wid] = cnt;
}

template <int NWIN>
__global__ void __launch_bounds__(256) k_table_fill(const BackArgs a, int n_views, const int2* __restrict__ hdr,
                                                     float4* __restrict__ tw, int* __restrict__ tray)
{
    const int nb = (a.ns + 1) / 2, groups = table_groups(a.ns);
    const long wid = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= (long)n_views * groups) return;                // whole warps
    const int v = (int)(wid / groups), k = (int)(wid - (long)v * groups);
    int bx, by;
    table_block(a.ns, k, lane, bx, by);
    const int2 h = hdr[wid];
    int s = 0;
    if (bx < nb && by < nb) {
        const GatherFrame fr = gather_frame<NWIN>(a, bx, by);
        int jlo, jhi;
        gather_bins(a, fr, v, jlo, jhi);
        const long base = (long)v * a.n_det;
        for (int j = jlo; j <= jhi && s < h.y; ++j) {
            float4 wq;
            if (!gather_weights<NWIN>(a, fr, __ldg(a.rayf + base + j), wq)) continue;
            const long idx = ((long)h.x + s) * 32 + lane;
            tw[idx] = wq;
            tray[idx] = j;
            ++s;
        }
    }
    for (; s < h.y; ++s) {
        const long idx = ((long)h.x + s) * 32 + lane;
        tw[idx] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        tray[idx] = -1;
    }
}

// The table gather: CTA = one group of 32 blocks x G view groups (warp g walks
// the views g, g + G, ... of the subset), BC images per thread as in
// k_backward_batch, whose reduction and epilogue it shares.
template <int BC>
__global__ void __launch_bounds__(512, 1) k_backward_table(const BackBatchTable t)
{
    pdl_begin();
    const int lane = threadIdx.x, g = threadIdx.y, G = blockDim.y;
    int c = 0;
#pragma unroll
    for (int k = 1; k < kMaxClasses; ++k)
        if (k < t.count && (long)blockIdx.x >= t.begin[k]) c = k;
    const BackArgs& a = t.c[c];
    const int nb = (a.ns + 1) / 2, groups = table_groups(a.ns);
    const int chunks = (a.batch + BC - 1) / BC;
    const long local = (long)blockIdx.x - t.begin[c];
    const int k = (int)(local / chunks);                       // the chunks of a group are adjacent
    const int chunk = (int)(local - (long)k * chunks);         // CTAs: their table reads meet in L2
    const int i0 = chunk * BC;
    const int ni = min(BC, a.batch - i0);                      // images in this chunk
    const long istride = res_is(a);
    const int js = res_js(a);
    const bool vec = a.res_il && (a.batch & 3) == 0 && (BC & 3) == 0;
    float2 acc2[BC / 2][4];
#pragma unroll
    for (int h = 0; h < BC / 2; ++h) acc2[h][0] = acc2[h][1] = acc2[h][2] = acc2[h][3] = make_float2(0.0f, 0.0f);
    const float* __restrict__ res = a.res + (long)i0 * istride;
    auto entry = [&](int j, const float4 wq, const float* __restrict__ rrow) {
        float r[BC];
        if (vec) {
            const float4* r4 = reinterpret_cast<const float4*>(rrow + (long)j * js);
#pragma unroll
            for (int b = 0; b < BC; b += 4) {
                const float4 q = b < ni ? __ldg(r4 + b / 4) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                r[b] = q.x; r[b + 1] = q.y; r[b + 2] = q.z; r[b + 3] = q.w;
            }
        } else {
#pragma unroll
            for (int b = 0; b < BC; ++b) r[b] = b < ni ? __ldg(rrow + b * istride + (long)j * js) : 0.0f;
        }
        const float2 v00 = make_float2(wq.x, wq.x), v10 = make_float2(wq.y, wq.y);
        const float2 v01 = make_float2(wq.z, wq.z), v11 = make_float2(wq.w, wq.w);
#pragma unroll
        for (int h = 0; h < BC / 2; ++h) {
            const float2 rr = make_float2(r[2 * h], r[2 * h + 1]);
            acc2[h][0] = __ffma2_rn(v00, rr, acc2[h][0]);
            acc2[h][1] = __ffma2_rn(v10, rr, acc2[h][1]);
            acc2[h][2] = __ffma2_rn(v01, rr, acc2[h][2]);
            acc2[h][3] = __ffma2_rn(v11, rr, acc2[h][3]);
        }
    };
    // headers of the next view fetched one view ahead; the slots of a view in
    // batches of kTabPre (bins and weights loaded together, then used in order)
    constexpr int kTabPre = 4;
    int vs = g;
    int2 hd = make_int2(0, 0);
    if (vs < a.n_sub) hd = __ldg(a.thdr + (long)(a.first_view + vs * a.view_step) * groups + k);
    for (; vs < a.n_sub; vs += G) {
        const int2 cur = hd;
        if (vs + G < a.n_sub) hd = __ldg(a.thdr + (long)(a.first_view + (vs + G) * a.view_step) * groups + k);
        const float* __restrict__ rrow = res + (long)vs * a.n_det * js;
        for (int sl = 0; sl < cur.y; sl += kTabPre) {
            int jj[kTabPre];
            float4 ww[kTabPre];
#pragma unroll
            for (int q = 0; q < kTabPre; ++q) {
                const long idx = ((long)cur.x + sl + q) * 32 + lane;
                jj[q] = sl + q < cur.y ? __ldg(a.tray + idx) : -1;
                ww[q] = sl + q < cur.y ? __ldg(a.tw + idx) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
#pragma unroll
            for (int q = 0; q < kTabPre; ++q)
                if (jj[q] >= 0) entry(jj[q], ww[q], rrow);
        }
    }
    // view-group sums in rounds of RB images: part[g][k][slot]
    extern __shared__ float4 part[];
    constexpr int kSlots = 32;
    const int RB = t.rb;
    const int nthr = kSlots * G;
    const int lt = g * 32 + lane;
    const int s = a.s;
    for (int b0 = 0; b0 < ni; b0 += RB) {
        if (b0 > 0) __syncthreads();
#pragma unroll
        for (int b = 0; b < BC; ++b)
            if (b >= b0 && b < b0 + RB)
                part[(g * RB + (b - b0)) * kSlots + lane] =
                    (b & 1) ? make_float4(acc2[b / 2][0].y, acc2[b / 2][1].y, acc2[b / 2][2].y, acc2[b / 2][3].y)
                            : make_float4(acc2[b / 2][0].x, acc2[b / 2][1].x, acc2[b / 2][2].x, acc2[b / 2][3].x);
        __syncthreads();
        for (int idx = lt; idx < RB * kSlots; idx += nthr) {
            const int kk = idx / kSlots, sl = idx - kk * kSlots;
            const int inst = i0 + b0 + kk;
            int obx, oby;
            table_block(a.ns, k, sl, obx, oby);
            if (b0 + kk >= ni || obx >= nb || oby >= nb) continue;
            float s00 = 0.0f, s10 = 0.0f, s01 = 0.0f, s11 = 0.0f;
            for (int q = 0; q < G; ++q) {
                const float4 pq = part[(q * RB + kk) * kSlots + sl];
                s00 += pq.x; s10 += pq.y; s01 += pq.z; s11 += pq.w;
            }
            const float vals[4] = {a.scale * s00, a.scale * s10, a.scale * s01, a.scale * s11};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int ix = 2 * obx + (q & 1), iy = 2 * oby + (q >> 1);
                if (ix >= a.ns || iy >= a.ns) continue;
                if (a.mode == kBackRaw) {
                    a.out[((long)inst * a.ns + iy) * a.ns + ix] = vals[q];
                    continue;
                }
                for (int bb = 0; bb < s; ++bb) {
                    const long row = ((long)inst * a.n + (long)iy * s + bb) * a.n + (long)ix * s;
                    for (int aa = 0; aa < s; ++aa) {
                        if (a.mode == kBackGradFine)
                            a.out[row + aa] = vals[q];
                        else
                            a.out[row + aa] = __ldg(a.y + row + aa) - a.eta * vals[q];
                    }
                }
            }
        }
    }
}

// ------------------------------------------------------------------ transpose A_s^T, scatter form
// CTA = one TS x TS tile of the level image of one instance, all views of the
// subset.  Every sample of every ray that can touch the tile is splatted with
// the weights of the forward interpolant, (1/2 -+ u)(1/2 -+ w) on the four
// pixels of its cell, as a 32-bit fixed-point shared-memory atomic add: integer
// sums do not depend on the order of the adds, so the result is deterministic.
// Scale: the largest |r| among the rays that reach the tile maps to qmax, small
// enough that no accumulator overflows within a chunk of views (one view per
// warp), given the geometric bound cmax on the terms a pixel receives from one
// view; after each chunk the integers are folded into FP32 totals in a fixed
// order.  A two-pixel apron around the tile takes the terms of neighbouring
// tiles' pixels (those tiles splat the same samples for their own pixels).
// A lane walks the samples of a ray inside the tile grown by the hat support
// (plus one sample each way), so every sample with a weight on the tile is
// visited; tap positions are clamped to the apron, so a sample that float
// rounding lets in from outside lands there.  (Measured and dropped: two rays
// per lane, in two loops or one fused loop, to even out the lanes' sample
// counts, 30 % slower; sample ranges trimmed instead of clamped taps, 15 %
// slower.)
struct BackScTable {
    BackArgs c[kMaxClasses];
    long begin[kMaxClasses + 1];   // cumulative CTA counts (batch * tiles)
    int count;
    float qsum;                    // 2^30 / (views per chunk): qmax = min(2^21, qsum / cmax)
};

template <int TS, int NT>
__global__ void __launch_bounds__(NT) k_backward_scatter(const BackScTable t)
{
    pdl_begin();
    constexpr int AP = TS + 4;                  // accumulator side: the tile and a 2-pixel apron
    constexpr int NW = NT / 32;                 // warps = views per chunk
    constexpr int PPT = (TS * TS + NT - 1) / NT;
    __shared__ int acc[AP * AP];
    __shared__ float wmax[NW];
    int c = 0;
#pragma unroll
    for (int k = 1; k < kMaxClasses; ++k)
        if (k < t.count && (long)blockIdx.x >= t.begin[k]) c = k;
    const BackArgs& a = t.c[c];
    const int ns = a.ns;
    const int tiles_x = (ns + TS - 1) / TS;
    const int tiles = tiles_x * tiles_x;
    const long local = (long)blockIdx.x - t.begin[c];
    const int inst = (int)(local / tiles);
    const int tile = (int)(local - (long)inst * tiles);
    const int tx0 = (tile % tiles_x) * TS, ty0 = (tile / tiles_x) * TS;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < AP * AP; i += NT) acc[i] = 0;
    const int js = res_js(a);
    const float* __restrict__ res = a.res + (long)inst * res_is(a);
    const float half = 0.5f * (float)(ns - 1);
    const float jc = 0.5f * (float)(a.n_det - 1);
    // bins of a view that can reach the tile: the central projection of the
    // corners of the tile grown by the apron (a convex polygon projects onto the
    // flat detector as the interval between its extreme corners), one bin wider
    auto shadow = [&](const float4 vp, int& jlo, int& jhi) {
        float lo = 1e30f, hi = -1e30f;
        bool ok = true;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float x = (float)((q & 1) ? tx0 + TS + 1 : tx0 - 2) - half;
            const float y = (float)((q & 2) ? ty0 + TS + 1 : ty0 - 2) - half;
            const float along = x * vp.x + y * vp.y;
            const float lat = y * vp.x - x * vp.y;
            const float den = vp.z - along;
            ok = ok && den > 1e-3f * vp.z;
            const float uj = vp.w * lat / den + jc;
            lo = fminf(lo, uj);
            hi = fmaxf(hi, uj);
        }
        if (!ok) {
            jlo = 0;
            jhi = a.n_det - 1;
            return;
        }
        jlo = max(0, (int)floorf(fmaxf(lo, -2.0f)) - 1);
        jhi = min(a.n_det - 1, (int)ceilf(fminf(hi, (float)a.n_det + 1.0f)) + 1);
    };
    // the largest |r| that can reach the tile; a non-finite one makes the tile's
    // outputs NaN (fixed point cannot carry it)
    float m = 0.0f;
    int bad = 0;
    for (int vs = wid; vs < a.n_sub; vs += NW) {
        int jlo, jhi;
        shadow(__ldg(a.view + a.first_view + vs * a.view_step), jlo, jhi);
        const float* __restrict__ rrow = res + (long)vs * a.n_det * js;
        for (int j = jlo + lane; j <= jhi; j += 32) {
            const float rv = fabsf(__ldg(rrow + (long)j * js));
            bad |= !(rv <= 3.402823466e38f);
            m = fmaxf(m, rv);
        }
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) wmax[wid] = m;
    const bool nonfinite = __syncthreads_or(bad) != 0;
    float M = 0.0f;
#pragma unroll
    for (int w = 0; w < NW; ++w) M = fmaxf(M, wmax[w]);
    const float qmax = fminf(2097152.0f, t.qsum / a.cmax);
    const float S = M > 0.0f && !nonfinite ? qmax / M : 0.0f;
    const int c0 = ns / 2;
    const int biasx = kMagicBits - c0 + tx0;   // float_as_int(X' + kMagic) - biasx: tap a's column in acc
    const int biasy = kMagicBits - c0 + ty0;
    // sample region in the primed frame: index coordinates (tx0 - 1, tx0 + TS)
    const float xlo = (float)(tx0 - c0) + 0.5f, xhi = (float)(tx0 + TS - c0) + 1.5f;
    const float ylo = (float)(ty0 - c0) + 0.5f, yhi = (float)(ty0 + TS - c0) + 1.5f;
    const float inv_step = 1.0f / a.step;
    float tot[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) tot[q] = 0.0f;
    for (int v0 = 0; v0 < a.n_sub; v0 += NW) {
        const int vs = v0 + wid;
        if (vs < a.n_sub) {
            const int v = a.first_view + vs * a.view_step;
            int jlo, jhi;
            shadow(__ldg(a.view + v), jlo, jhi);
            const long base = (long)v * a.n_det;
            const float* __restrict__ rrow = res + (long)vs * a.n_det * js;
            // lane = ray; lanes start five rays apart, so that the samples of one
            // atomic instruction rarely share a pixel
            for (int j = jlo + ((lane * 5) & 31); j <= jhi; j += 32) {
                const float4 f = __ldg(a.rayf + base + j);
                const float2 ri = __ldg(a.rayi + base + j);
                const int2 kr = __ldg(a.rayk + base + j);
                const float tx1 = (xlo - f.x) * ri.x, tx2 = (xhi - f.x) * ri.x;
                const float ty1 = (ylo - f.y) * ri.y, ty2 = (yhi - f.y) * ri.y;
                const float tlo = fmaxf(fminf(tx1, tx2), fminf(ty1, ty2));
                const float thi = fminf(fmaxf(tx1, tx2), fmaxf(ty1, ty2));
                const float fa = fmaxf(fmaf(tlo, inv_step, -0.5f), (float)kr.x - 2.0f);
                const float fb = fminf(fmaf(thi, inv_step, -0.5f), (float)kr.y + 2.0f);
                const int ka = max(kr.x, (int)ceilf(fa) - 1);
                const int kb = min(kr.y, (int)floorf(fb) + 1);
                const float rS = __ldg(rrow + (long)j * js) * S;
                for (int k = ka; k <= kb; ++k) {
                    const float tt = ((float)k + 0.5f) * a.step;
                    const float X = fmaf(tt, f.z, f.x);
                    const float Y = fmaf(tt, f.w, f.y);
                    const float mx = __fadd_rn(X, kMagic);
                    const float my = __fadd_rn(Y, kMagic);
                    const float u = __fsub_rn(X, __fsub_rn(mx, kMagic));
                    const float w = __fsub_rn(Y, __fsub_rn(my, kMagic));
                    const int lc = min(max(__float_as_int(mx) - biasx, 0), TS + 2);
                    const int lr = min(max(__float_as_int(my) - biasy, 0), TS + 2);
                    int* const p = acc + lr * AP + lc;
                    const float r0 = rS * (0.5f - w), r1 = rS * (0.5f + w);
                    const float ua = 0.5f - u, ub = 0.5f + u;
                    atomicAdd(p, __float_as_int(fmaf(ua, r0, kMagic)) - kMagicBits);
                    atomicAdd(p + 1, __float_as_int(fmaf(ub, r0, kMagic)) - kMagicBits);
                    atomicAdd(p + AP, __float_as_int(fmaf(ua, r1, kMagic)) - kMagicBits);
                    atomicAdd(p + AP + 1, __float_as_int(fmaf(ub, r1, kMagic)) - kMagicBits);
                }
            }
        }
        __syncthreads();
        // fold the chunk into the totals and clear the tile's cells (the apron is never read)
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            const int pix = threadIdx.x + q * NT;
            if (pix < TS * TS) {
                int* const cell = acc + (pix / TS + 2) * AP + (pix % TS) + 2;
                tot[q] += (float)*cell;
                *cell = 0;
            }
        }
        __syncthreads();
    }
    const float inv_s = S > 0.0f ? M / qmax : 0.0f;
    const int s = a.s;
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int pix = threadIdx.x + q * NT;
        const int ix = tx0 + pix % TS, iy = ty0 + pix / TS;
        if (pix >= TS * TS || ix >= ns || iy >= ns) continue;
        const float val = nonfinite ? __int_as_float(0x7FC00000) : a.scale * (tot[q] * inv_s);
        if (a.mode == kBackRaw) {
            a.out[((long)inst * ns + iy) * ns + ix] = val;
            continue;
        }
        for (int bb = 0; bb < s; ++bb) {
            const long row = ((long)inst * a.n + (long)iy * s + bb) * a.n + (long)ix * s;
            for (int aa = 0; aa < s; ++aa) {
                if (a.mode == kBackGradFine)
                    a.out[row + aa] = val;
                else
                    a.out[row + aa] = __ldg(a.y + row + aa) - a.eta * val;
            }
        }
    }
}

// ------------------------------------------------------------------ bicubic S and S^T
// The paper's sketch and upsampler are bicubic resizes (Sec. 3).  Here S is
// separable: coarse pixel I (centre X_I = s I + (s-1)/2 in fine index units)
// averages fine pixels x with weights k((x - X_I)/s) / sum_x' k((x' - X_I)/s),
// k the Keys cubic convolution kernel with a = -1/2, widened by s (so no
// aliasing), the sum running over the fine pixels inside the image.  U = S^T.
__device__ __forceinline__ float keys_kernel(float t)
{
    const float a = -0.5f;
    t = fabsf(t);
    if (t <= 1.0f) return ((a + 2.0f) * t - (a + 3.0f)) * t * t + 1.0f;
    if (t < 2.0f) return ((a * t - 5.0f * a) * t + 8.0f * a) * t - 4.0f * a;
    return 0.0f;
}

// Normalisation of coarse index I's weights (sum over its support inside [0, n)).
__device__ __forceinline__ float bicubic_den(int I, int s, int n)
{
    const float XI = s * I + 0.5f * (s - 1);
    const int x0 = max(0, (int)ceilf(XI - 2.0f * s)), x1 = min(n - 1, (int)floorf(XI + 2.0f * s));
    float den = 0.0f;
    for (int x = x0; x <= x1; ++x) den += keys_kernel(((float)x - XI) / (float)s);
    return den;
}

__global__ void k_bicubic_down(const float* __restrict__ fine, float* __restrict__ coarse, int n, int s)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const int inst = blockIdx.z;
    const int ns = n / s;
    if (I >= ns || J >= ns) return;
    const float XI = s * I + 0.5f * (s - 1), YJ = s * J + 0.5f * (s - 1);
    const int x0 = max(0, (int)ceilf(XI - 2.0f * s)), x1 = min(n - 1, (int)floorf(XI + 2.0f * s));
    const int y0 = max(0, (int)ceilf(YJ - 2.0f * s)), y1 = min(n - 1, (int)floorf(YJ + 2.0f * s));
    const float inv = 1.0f / ((float)s);
    const float* f = fine + (long)inst * n * n;
    float acc = 0.0f;
    for (int y = y0; y <= y1; ++y) {
        const float wy = keys_kernel(((float)y - YJ) * inv);
        float row = 0.0f;
        for (int x = x0; x <= x1; ++x) row = fmaf(keys_kernel(((float)x - XI) * inv), __ldg(f + (long)y * n + x), row);
        acc = fmaf(wy, row, acc);
    }
    coarse[((long)inst * ns + J) * ns + I] = acc / (bicubic_den(I, s, n) * bicubic_den(J, s, n));
}

// out = (base ? base - eta * scale * S^T g : scale * S^T g) on the fine grid.
__global__ void k_bicubic_up(const float* __restrict__ g, const float* __restrict__ base, float* __restrict__ out,
                             int n, int s, float scale, float eta)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int inst = blockIdx.z;
    const int ns = n / s;
    if (x >= n || y >= n) return;
    const float inv = 1.0f / ((float)s);
    const float half = 0.5f * (s - 1);
    const int Ic = (int)floorf(((float)x - half) * inv), Jc = (int)floorf(((float)y - half) * inv);
    const float* gi = g + (long)inst * ns * ns;
    float acc = 0.0f;
    for (int J = max(0, Jc - 2); J <= min(ns - 1, Jc + 2); ++J) {
        const float wy = keys_kernel(((float)y - (s * J + half)) * inv) / bicubic_den(J, s, n);
        if (wy == 0.0f) continue;
        float row = 0.0f;
        for (int I = max(0, Ic - 2); I <= min(ns - 1, Ic + 2); ++I) {
            const float wx = keys_kernel(((float)x - (s * I + half)) * inv);
            if (wx != 0.0f) row = fmaf(wx / bicubic_den(I, s, n), __ldg(gi + (long)J * ns + I), row);
        }
        acc = fmaf(wy, row, acc);
    }
    const long o = ((long)inst * n + y) * n + x;
    out[o] = base ? __ldg(base + o) - eta * scale * acc : scale * acc;
}

// ------------------------------------------------------------------ S and S^T
__global__ void k_pool(const float* __restrict__ fine, float* __restrict__ coarse, int n, int s)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    int inst = blockIdx.z;
    int ns = n / s;
    if (i >= ns || j >= ns) return;
    coarse[((long)inst * ns + j) * ns + i] = pooled(fine + (long)inst * n * n, n, s, ns, i, j);
}

__global__ void k_unpool(const float* __restrict__ coarse, float* __restrict__ fine, int n, int s)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    int inst = blockIdx.z;
    int ns = n / s;
    if (x >= n || y >= n) return;
    fine[((long)inst * n + y) * n + x] =
        __ldg(coarse + ((long)inst * ns + y / s) * ns + x / s) * (1.0f / (float)(s * s));
}

__global__ void k_count_samples(const int2* __restrict__ rayk, int n_det, int first_view,
                                int view_step, int n_sub, double* __restrict__ out)
{
    __shared__ double sh[256];
    double acc = 0.0;
    long total = (long)n_sub * n_det;
    for (long i = threadIdx.x; i < total; i += blockDim.x) {
        int vs = (int)(i / n_det), j = (int)(i % n_det);
        int2 kr = rayk[(long)(first_view + vs * view_step) * n_det + j];
        if (kr.y >= kr.x) acc += (double)(kr.y - kr.x + 1);
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0];
}

inline cudaError_t counted(cudaError_t e = cudaGetLastError())
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return e;
}

}  // namespace

cudaError_t launch_setup_rays(const pnp_geom& g, const LevelLayout& L, char* ws, cudaStream_t st)
{
    long nr = (long)g.n_views * g.n_det;
    k_setup_rays<<<div_up(nr, 128), 128, 0, st>>>(
        g.n, L.factor, g.n_views, g.n_det, g.dso, g.ddo, g.det_pitch, g.angle0, g.angle_span,
        g.step, (float4*)(ws + L.off_rayf), (float2*)(ws + L.off_rayi), (int2*)(ws + L.off_rayk),
        (float4*)(ws + L.off_view));
    return counted();
}

cudaError_t launch_prep_multi(const PrepArgs* items, int count, cudaStream_t st)
{
    if (count < 1 || count > kMaxClasses) return cudaErrorInvalidValue;
    // image-major classes in one launch, image-interleaved ones in another
    PrepTable t{};
    PrepIlTable ti{};
    t.ibegin[0] = 0;
    ti.begin[0] = 0;
    long cells = 0;
    // four cell rows per CTA when the interleaved classes' level images are large
    int il_rows = 1;
    for (int c = 0; c < count; ++c)
        if (quad_interleaved(items[c].batch) && items[c].n / items[c].s >= 256) il_rows = 4;
    for (int c = 0; c < count; ++c) {
        const PrepArgs& it = items[c];
        if (quad_interleaved(it.batch)) {
            ti.c[ti.count] = it;
            ti.begin[ti.count + 1] = ti.begin[ti.count] + (long)div_up(it.qw, il_rows) * div_up(it.qw, kIlCells);
            ++ti.count;
        } else {
            t.c[t.count] = it;
            t.ibegin[t.count + 1] = t.ibegin[t.count] + it.batch;
            ++t.count;
            cells = max(cells, (long)it.qw * it.qw);
        }
    }
    if (t.count > 0) {
        const dim3 grd(div_up(cells, 256), (unsigned)min(t.ibegin[t.count], 65535L));
        const cudaError_t e = launch_pdl(k_prep_quad, grd, dim3(256), 0, st, t);
        if (e != cudaSuccess) return e;
        counted();
    }
    if (ti.count > 0) {
        const dim3 grd((unsigned)ti.begin[ti.count]);
        const cudaError_t e = il_rows == 4 ? launch_items(k_prep_quad_il<4>, k_prep_quad_il_persistent<4>, grd, dim3(256), 0, st, ti)
                                           : launch_items(k_prep_quad_il<1>, k_prep_quad_il_persistent<1>, grd, dim3(256), 0, st, ti);
        if (e != cudaSuccess) return e;
        counted();
    }
    return cudaSuccess;
}

cudaError_t launch_prep_quad(const float* fine, int n, int s, int batch, float4* quad, int qw,
                             cudaStream_t st)
{
    const PrepArgs a{fine, n, s, batch, quad, qw};
    return launch_prep_multi(&a, 1, st);
}

template <int Q>
cudaError_t forward_q(FwdTable t, cudaStream_t st)
{
    constexpr int RB = kFwdWarps * (32 / Q);
    for (int c = 0; c < t.count; ++c)
        t.begin[c + 1] = t.begin[c] + (long)t.c[c].batch * t.c[c].n_sub * div_up(t.c[c].n_det, RB);
    return launch_items(k_forward<Q>, k_forward_persistent<Q>, dim3((unsigned)t.begin[t.count]), dim3(32 * kFwdWarps), 0, st, t);
}

namespace {
template <int IPL>
cudaError_t forward_il(const FwdTable& t, cudaStream_t st)
{
    return launch_items(k_forward_il<IPL>, k_forward_il_persistent<IPL>, dim3((unsigned)t.begin[t.count]), dim3(32 * kFwdIlWarps), 0, st, t);
}
}  // namespace

// Classes with image-interleaved coefficient images (batch >= kQuadIlMin, at
// most 32 images) take k_forward_il, the others k_forward; one launch each.
cudaError_t launch_forward_multi(const FwdArgs* items, int count, cudaStream_t st, int lanes)
{
    if (count < 1 || count > kMaxClasses) return cudaErrorInvalidValue;
    FwdTable ti{};
    ti.begin[0] = 0;
    int maxb = 0;
    FwdArgs rest[kMaxClasses];
    int nrest = 0;
    for (int c = 0; c < count; ++c) {
        if (quad_interleaved(items[c].batch)) {
            ti.c[ti.count] = items[c];
            maxb = max(maxb, items[c].batch);
            ++ti.count;
        } else {
            rest[nrest++] = items[c];
        }
    }
    if (ti.count > 0) {
        // images per lane: 1, 2 or 4 (chunks of 8, 16 or 32 images per warp)
        const int ipl = maxb <= 8 ? 1 : maxb <= 16 ? 2 : 4;
        for (int c = 0; c < ti.count; ++c)
            ti.begin[c + 1] = ti.begin[c] + (long)ti.c[c].n_sub * div_up(ti.c[c].n_det, kFwdIlWarps) *
                                                div_up(ti.c[c].batch, 8 * ipl);
        const cudaError_t e = ipl == 1 ? forward_il<1>(ti, st) : ipl == 2 ? forward_il<2>(ti, st)
                                                                          : forward_il<4>(ti, st);
        if (e != cudaSuccess) return e;
        counted();
    }
    if (nrest == 0) return cudaSuccess;
    items = rest;
    count = nrest;
    FwdTable t{};
    t.count = count;
    t.begin[0] = 0;
    long rays = 0;
    for (int c = 0; c < count; ++c) {
        t.c[c] = items[c];
        rays += (long)items[c].batch * items[c].n_sub * items[c].n_det;
    }
    // lanes per ray: enough threads to fill the GPU (~2 waves of 2048 threads
    // per SM), unless the autotuner chose
    int Q = lanes;
    const long fill = 2L * device_sm_count() * 2048;
    if (Q != 4 && Q != 8 && Q != 16) Q = rays * 4 >= fill ? 4 : rays * 8 >= fill ? 8 : 16;
    const cudaError_t e = Q == 4 ? forward_q<4>(t, st) : Q == 8 ? forward_q<8>(t, st) : forward_q<16>(t, st);
    if (e != cudaSuccess) return e;
    return counted();
}

cudaError_t launch_forward(const FwdArgs& a, cudaStream_t st, int lanes)
{
    return launch_forward_multi(&a, 1, st, lanes);
}

namespace {
template <int TS, int NT>
cudaError_t scatter_launch(const BackArgs* items, int count, cudaStream_t st)
{
    BackScTable t{};
    t.count = count;
    t.begin[0] = 0;
    for (int c = 0; c < count; ++c) {
        t.c[c] = items[c];
        const long tl = div_up(items[c].ns, TS);
        t.begin[c + 1] = t.begin[c] + tl * tl * items[c].batch;
    }
    t.qsum = 1073741824.0f / (float)(NT / 32);
    const cudaError_t e = launch_pdl(k_backward_scatter<TS, NT>, dim3((unsigned)t.begin[count]), dim3(NT), 0, st, t);
    if (e != cudaSuccess) return e;
    return counted();
}

// The scatter needs the geometric term bound of every class and a scale that
// keeps at least 12 bits per term; otherwise the gather runs.
bool scatter_usable(const BackArgs* items, int count, int nt)
{
    for (int c = 0; c < count; ++c) {
        const float cm = items[c].cmax;
        if (!(cm > 0.0f) || 1073741824.0f / (float)(nt / 32) / cm < 4096.0f) return false;
    }
    return true;
}
}  // namespace

namespace {
template <int BC>
cudaError_t batch_launch(const BackBatchTable& t, int TX, bool half_step, dim3 grd, dim3 blk, size_t smem,
                         cudaStream_t st)
{
    if (TX == 4)
        return half_step ? launch_items(k_backward_batch<9, 4, BC>, k_backward_batch_persistent<9, 4, BC>, grd, blk, smem, st, t)
                         : launch_items(k_backward_batch<0, 4, BC>, k_backward_batch_persistent<0, 4, BC>, grd, blk, smem, st, t);
    return half_step ? launch_items(k_backward_batch<9, kBack2TileX, BC>, k_backward_batch_persistent<9, kBack2TileX, BC>, grd, blk, smem, st, t)
                     : launch_items(k_backward_batch<0, kBack2TileX, BC>, k_backward_batch_persistent<0, kBack2TileX, BC>, grd, blk, smem, st, t);
}

// The batched gather: BC in {4, 8, 16} images per thread, TX x 4 blocks x G view
// groups per CTA (at most 512 threads).
cudaError_t launch_backward_batch(const BackArgs* items, int count, cudaStream_t st, int groups)
{
    const int BC = back_batch_of(groups);
    const int TX = (groups & PNP_BACK_TILE4) ? 4 : kBack2TileX;
    int G = groups & 0xff;
    BackBatchTable t{};
    t.count = count;
    t.begin[0] = 0;
    long threads1 = 0;
    int min_views = 1 << 30;
    bool half_step = true;
    for (int c = 0; c < count; ++c) {
        t.c[c] = items[c];
        const int nb = (items[c].ns + 1) / 2;
        const int tiles = div_up(nb, TX) * div_up(nb, kBack2TileY);
        const int chunks = div_up(items[c].batch, BC);
        t.begin[c + 1] = t.begin[c] + (long)tiles * chunks;
        threads1 += (long)tiles * chunks * TX * kBack2TileY;
        min_views = min(min_views, items[c].n_sub);
        half_step = half_step && items[c].step == 0.5f;
    }
    const int gmax = kBackBatchThreads / (TX * kBack2TileY);
    if (G < 1 || G > gmax) {   // about two waves of 1024 threads per SM
        G = 1;
        const long wave = 2L * device_sm_count() * 1024;
        while (G * 2 <= gmax && threads1 * G < wave && G * 2 <= min_views) G *= 2;
    }
    const int slots = TX * kBack2TileY;
    t.rb = max(1, min(BC, (int)(32768 / ((long)G * slots * sizeof(float4)))));
    const size_t smem = (size_t)G * t.rb * slots * sizeof(float4);
    dim3 blk(TX, kBack2TileY, G), grd((unsigned)t.begin[count]);
    cudaError_t e;
    switch (BC) {
        case 4: e = batch_launch<4>(t, TX, half_step, grd, blk, smem, st); break;
        case 8: e = batch_launch<8>(t, TX, half_step, grd, blk, smem, st); break;
        default: e = batch_launch<16>(t, TX, half_step, grd, blk, smem, st); break;
    }
    if (e != cudaSuccess) return e;
    return counted();
}
}  // namespace

namespace {
template <int BC>
cudaError_t table_launch(const BackBatchTable& t, dim3 grd, dim3 blk, size_t smem, cudaStream_t st)
{
    return launch_pdl(k_backward_table<BC>, grd, blk, smem, st, t);
}

// The table gather: BC in {2, 4, 8, 16} images per thread, 32 blocks x G view groups per CTA.
cudaError_t launch_backward_table(const BackArgs* items, int count, cudaStream_t st, int groups)
{
    int BC = back_batch_of(groups);
    BC = BC >= 16 ? 16 : BC >= 8 ? 8 : BC >= 4 ? 4 : 2;
    int G = groups & 0xff;
    BackBatchTable t{};
    t.count = count;
    t.begin[0] = 0;
    int min_views = 1 << 30;
    long warps1 = 0;
    for (int c = 0; c < count; ++c) {
        if (!items[c].thdr || !items[c].tw || !items[c].tray) return cudaErrorInvalidValue;
        t.c[c] = items[c];
        const int chunks = div_up(items[c].batch, BC);
        t.begin[c + 1] = t.begin[c] + (long)table_groups(items[c].ns) * chunks;
        warps1 += (long)table_groups(items[c].ns) * chunks;
        min_views = min(min_views, items[c].n_sub);
    }
    if (G < 1 || G > 16) {   // about two waves of 32 warps per SM
        G = 1;
        const long wave = 2L * device_sm_count() * 32;
        while (G * 2 <= 16 && warps1 * G < wave && G * 2 <= min_views) G *= 2;
    }
    t.rb = max(1, min(BC, (int)(32768 / ((long)G * 32 * sizeof(float4)))));
    const size_t smem = (size_t)G * t.rb * 32 * sizeof(float4);
    dim3 blk(32, G), grd((unsigned)t.begin[count]);
    cudaError_t e;
    switch (BC) {
        case 2: e = table_launch<2>(t, grd, blk, smem, st); break;
        case 4: e = table_launch<4>(t, grd, blk, smem, st); break;
        case 8: e = table_launch<8>(t, grd, blk, smem, st); break;
        default: e = table_launch<16>(t, grd, blk, smem, st); break;
    }
    if (e != cudaSuccess) return e;
    return counted();
}
}  // namespace

cudaError_t launch_table_count(const BackArgs& a, int n_views, int* widths, cudaStream_t st)
{
    const long warps = (long)n_views * table_groups(a.ns);
    k_table_count<<<(unsigned)div_up(warps * 32, 256), 256, 0, st>>>(a, n_views, widths);
    return counted();
}

cudaError_t launch_table_fill(const BackArgs& a, int n_views, const int2* hdr, float4* tw, int* tray,
                              cudaStream_t st)
{
    const long warps = (long)n_views * table_groups(a.ns);
    const unsigned grd = (unsigned)div_up(warps * 32, 256);
    if (a.step == 0.5f)
        k_table_fill<9><<<grd, 256, 0, st>>>(a, n_views, hdr, tw, tray);
    else
        k_table_fill<0><<<grd, 256, 0, st>>>(a, n_views, hdr, tw, tray);
    return counted();
}

cudaError_t launch_backward_multi(const BackArgs* items, int count, cudaStream_t st, int groups)
{
    if (count < 1 || count > kMaxClasses) return cudaErrorInvalidValue;
    if (groups & PNP_BACK_TABLE) {
        bool all = true;
        for (int c = 0; c < count; ++c) all = all && items[c].thdr && items[c].tw && items[c].tray;
        if (all) return launch_backward_table(items, count, st, groups);
        // no table registered: the gather with the same view groups (batched for BC >= 4)
        groups &= ~PNP_BACK_TABLE;
        if (back_batch_of(groups) < 4) groups &= 0xffff;
    }
    if (!(groups & PNP_BACK_SCATTER) && back_batch_of(groups) > 1)
        return launch_backward_batch(items, count, st, groups);
    if (groups & PNP_BACK_SCATTER) {
        const int ts = groups & 0xff;
        const int nt = ts >= 22 ? 512 : 256;
        if (scatter_usable(items, count, nt)) {
            switch (ts) {
                case 12: return scatter_launch<12, 256>(items, count, st);
                case 16: return scatter_launch<16, 256>(items, count, st);
                case 22: return scatter_launch<22, 512>(items, count, st);
                case 32: return scatter_launch<32, 512>(items, count, st);
                default: break;
            }
        }
        groups = 0;
    }
    // CTA shape: TX x 4 blocks x G view groups; PNP_BACK_TILE4 selects TX = 4
    const int TX = (groups & PNP_BACK_TILE4) ? 4 : kBack2TileX;
    int G = groups & 0xff;
    BackTable t{};
    t.count = count;
    t.begin[0] = 0;
    long blocks = 0;
    int min_views = 1 << 30;
    bool half_step = true;
    for (int c = 0; c < count; ++c) {
        t.c[c] = items[c];
        const int nb = (items[c].ns + 1) / 2;
        const int tiles = div_up(nb, TX) * div_up(nb, kBack2TileY);
        t.begin[c + 1] = t.begin[c] + (long)tiles * items[c].batch;
        blocks += (long)nb * nb * items[c].batch;
        min_views = min(min_views, items[c].n_sub);
        half_step = half_step && items[c].step == 0.5f;
    }
    // view groups: about two waves of 2048 threads per SM, at most 16 per CTA,
    // unless the autotuner chose
    if (G < 1 || G * TX * kBack2TileY > 1024) {
        G = 1;
        const long wave = 2L * device_sm_count() * 2048;
        while (G < kBack2MaxGroups && blocks * G < wave && G * 2 <= min_views) G *= 2;
    }
    dim3 blk(TX, kBack2TileY, G), grd((unsigned)t.begin[count]);
    const size_t smem = (size_t)G * TX * kBack2TileY * sizeof(float4);
    cudaError_t e;
    if (TX == 4)
        e = half_step ? launch_items(k_backward2x2<9, 4>, k_backward2x2_persistent<9, 4>, grd, blk, smem, st, t)
                      : launch_items(k_backward2x2<0, 4>, k_backward2x2_persistent<0, 4>, grd, blk, smem, st, t);
    else
        e = half_step ? launch_items(k_backward2x2<9, kBack2TileX>, k_backward2x2_persistent<9, kBack2TileX>, grd, blk, smem, st, t)
                      : launch_items(k_backward2x2<0, kBack2TileX>, k_backward2x2_persistent<0, kBack2TileX>, grd, blk, smem, st, t);
    if (e != cudaSuccess) return e;
    return counted();
}

cudaError_t launch_backward(const BackArgs& a, cudaStream_t st, int groups)
{
    return launch_backward_multi(&a, 1, st, groups);
}

cudaError_t launch_pool(const float* fine, float* coarse, int n, int s, int batch, cudaStream_t st)
{
    int ns = n / s;
    dim3 blk(32, 8), grd(div_up(ns, 32), div_up(ns, 8), batch);
    k_pool<<<grd, blk, 0, st>>>(fine, coarse, n, s);
    return counted();
}

cudaError_t launch_unpool(const float* coarse, float* fine, int n, int s, int batch, cudaStream_t st)
{
    dim3 blk(32, 8), grd(div_up(n, 32), div_up(n, 8), batch);
    k_unpool<<<grd, blk, 0, st>>>(coarse, fine, n, s);
    return counted();
}

cudaError_t launch_bicubic_down(const float* fine, float* coarse, int n, int s, int batch, cudaStream_t st)
{
    const int ns = n / s;
    dim3 blk(16, 16), grd(div_up(ns, 16), div_up(ns, 16), batch);
    k_bicubic_down<<<grd, blk, 0, st>>>(fine, coarse, n, s);
    return counted();
}

cudaError_t launch_bicubic_up(const float* g, const float* base, float* out, int n, int s, int batch,
                              float scale, float eta, cudaStream_t st)
{
    dim3 blk(32, 8), grd(div_up(n, 32), div_up(n, 8), batch);
    k_bicubic_up<<<grd, blk, 0, st>>>(g, base, out, n, s, scale, eta);
    return counted();
}

cudaError_t launch_count_samples(const int2* rayk, int n_det, int first_view, int view_step,
                                 int n_sub, double* partial, cudaStream_t st)
{
    k_count_samples<<<1, 256, 0, st>>>(rayk, n_det, first_view, view_step, n_sub, partial);
    return counted();
}

}  // namespace pnp
