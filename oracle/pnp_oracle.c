/*
 * FP64 CPU oracle of the PnP-MS2G hot path (arXiv 2203.07308).
 *
 * TEST INFRASTRUCTURE ONLY.  The product library never includes, links or calls
 * this file; only the test suite, the smoke check and the benchmark's CPU
 * baseline leg do.  It is written to be read against the paper, not to be fast:
 * double precision everywhere, a naive ray march for A, a naive *scatter* for
 * A^T (the CUDA path uses a pixel-driven gather instead, so the two cannot share
 * a failure mode), and no blocking, fusion or reordering.
 *
 * What it computes
 *   Eq. 1    measurement model b = A x + w: the forward operator A (fan-beam,
 *            ray-driven, fixed step, bilinear taps) and its transpose A^T.
 *   Eq. 4    the sketched objective f(b, A_s S x): S = s x s average pooling,
 *            A_s = the same fan beam on the grid of pixel size s.
 *   Alg. 1   the multi-stage loop: v = S_k(y), G (Option 1 or Option 2 with
 *            angle subsets), z = y - eta U_k G, x = (1-a) z + a D(z),
 *            y = x + a_i (x - x_prev), with U_k = S_k^T.
 *   Eq. 5    the PnP proximal-gradient special case (one stage, s = 1, a_i = 0).
 *   Sec. 3   step size eta = 1/L with L = ||A_s S||^2 (power iteration) and the
 *            convergent-FISTA momentum a_i = (i-1)/(i+3).
 *   Beck & Teboulle 2009 (the paper's TV reference): FGP for the TV-prox
 *            denoiser D(z) = argmin 1/2||x - z||^2 + lambda TV_iso(x).
 *
 * Readings (the paper names fan-beam CT but no discretisation):
 *   grid     level-s image has n_s = n/s pixels per side, pixel size s (fine px),
 *            pixel (ix,iy) centred at ((ix-(n_s-1)/2) s, (iy-(n_s-1)/2) s),
 *            stored row-major img[iy*n_s + ix].
 *   source   view v at beta = angle0 + span*v/n_views, source dso (cos, sin),
 *            flat detector centred at -ddo (cos, sin), axis (-sin, cos), bin j at
 *            u_j = (j - (n_det-1)/2) pitch.
 *   samples  ray (v,j) with unit direction d and foot point F (nearest point to
 *            the origin); samples q_k = F + (k+1/2) delta d for every integer k,
 *            delta = step*s; each sample weighs delta.
 *   interp   bilinear, zero outside the image:
 *            f(q) = sum_p img[p] hat((q_x-c_px)/s) hat((q_y-c_py)/s),
 *            hat(t) = max(0, 1-|t|).
 *   subsets  subset p of P holds views v = p, p+P, p+2P, ...; its sinogram rows
 *            are those views in increasing order; the minibatch gradient is
 *            scaled by P so that its mean over p is the full gradient.
 *   order    the minibatch of each iteration is drawn at random (Sec. 2, the
 *            stochastic gradient of Eq. 6-7); read as sampling the P subsets
 *            without replacement within each epoch of P iterations (a fresh
 *            uniform permutation per epoch), from a seeded SplitMix64 stream.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int n, n_views, n_det, batch;
    double dso, ddo, pitch, angle0, span, step;
} orc_geom;

static double hat(double t)
{
    double a = 1.0 - fabs(t);
    return a > 0.0 ? a : 0.0;
}

/* Source position and unit ray direction of ray (v, j), centred fine-px coords. */
void orc_ray(const orc_geom *g, int v, int j, double out[6])
{
    double beta = g->angle0 + g->span * (double)v / (double)g->n_views;
    double cb = cos(beta), sb = sin(beta);
    double sx = g->dso * cb, sy = g->dso * sb;
    double u = ((double)j - 0.5 * (double)(g->n_det - 1)) * g->pitch;
    double px = -g->ddo * cb - u * sb;
    double py = -g->ddo * sb + u * cb;
    double ex = px - sx, ey = py - sy;
    double len = sqrt(ex * ex + ey * ey);
    double dx = ex / len, dy = ey / len;
    double sd = sx * dx + sy * dy;            /* foot point F = S - (S.d) d */
    out[0] = sx;
    out[1] = sy;
    out[2] = dx;
    out[3] = dy;
    out[4] = sx - sd * dx;
    out[5] = sy - sd * dy;
}

/* Number of views in subset p of P. */
int orc_subset_views(const orc_geom *g, int p, int P)
{
    if (P <= 1) return g->n_views;
    return (g->n_views - p + P - 1) / P;
}

/* Bilinear interpolant of a level-s image at centred point (qx, qy). */
static double interp(const double *img, int ns, double s, double qx, double qy)
{
    double X = qx / s + 0.5 * (ns - 1), Y = qy / s + 0.5 * (ns - 1);
    double fx = floor(X), fy = floor(Y);
    double val = 0.0;
    for (int b = 0; b < 2; ++b) {
        for (int a = 0; a < 2; ++a) {
            double ix = fx + a, iy = fy + b;
            if (ix < 0 || iy < 0 || ix > ns - 1 || iy > ns - 1) continue;
            double w = hat(X - ix) * hat(Y - iy);
            val += w * img[(long)iy * ns + (long)ix];
        }
    }
    return val;
}

/* Adjoint of interp: add wt * hat * hat into the (up to) four taps. */
static void scatter(double *img, int ns, double s, double qx, double qy, double wt)
{
    double X = qx / s + 0.5 * (ns - 1), Y = qy / s + 0.5 * (ns - 1);
    double fx = floor(X), fy = floor(Y);
    for (int b = 0; b < 2; ++b) {
        for (int a = 0; a < 2; ++a) {
            double ix = fx + a, iy = fy + b;
            if (ix < 0 || iy < 0 || ix > ns - 1 || iy > ns - 1) continue;
            double w = hat(X - ix) * hat(Y - iy);
            img[(long)iy * ns + (long)ix] += wt * w;
        }
    }
}

/* Sample index bound: every sample with |k| >= K lies outside the support box
 * (|x|,|y| < (n_s/2 + 1/2) s), where the interpolant is zero. */
static long sample_bound(const orc_geom *g, int s)
{
    int ns = g->n / s;
    double H = (0.5 * ns + 0.5) * s;
    double delta = g->step * s;
    return (long)ceil(sqrt(2.0) * H / delta) + 2;
}

/* One row of A_s applied to img: delta * sum_k f(q_k). */
static double ray_sum(const orc_geom *g, int s, const double *img, int v, int j)
{
    double r[6];
    orc_ray(g, v, j, r);
    int ns = g->n / s;
    double delta = g->step * s;
    long K = sample_bound(g, s);
    double acc = 0.0;
    for (long k = -K; k < K; ++k) {
        double t = ((double)k + 0.5) * delta;
        acc += interp(img, ns, s, r[4] + t * r[2], r[5] + t * r[3]);
    }
    return delta * acc;
}

/* A_s^{(p)} img: sino[vs*n_det + j] for the subset's views in increasing order.
 * P <= 1 means all views.  b (nullable, full sinogram [n_views][n_det]) is
 * subtracted row by row, giving the residual A_s^{(p)} v - b^{(p)}. */
void orc_project(const orc_geom *g, int s, const double *img, const double *b,
                 double *sino, int p, int P)
{
    int nsub = orc_subset_views(g, p, P);
    int step = P <= 1 ? 1 : P;
    int first = P <= 1 ? 0 : p;
#pragma omp parallel for schedule(dynamic, 1)
    for (int vs = 0; vs < nsub; ++vs) {
        int v = first + vs * step;
        for (int j = 0; j < g->n_det; ++j) {
            double val = ray_sum(g, s, img, v, j);
            if (b) val -= b[(long)v * g->n_det + j];
            sino[(long)vs * g->n_det + j] = val;
        }
    }
}

/* A_s^{(p)T} sino by scatter: every sample of every ray adds its weighted ray
 * value into the pixels whose hat functions cover it.  The subset's views are
 * cut into a fixed number of contiguous chunks (set by the view count alone,
 * not by the number of threads); each chunk scatters into an image of its own
 * in view order, and the chunk images are added in chunk order, so the result
 * is the same whatever the thread count. */
void orc_backproject(const orc_geom *g, int s, const double *sino, double *img, int p, int P)
{
    int ns = g->n / s;
    int nsub = orc_subset_views(g, p, P);
    int step = P <= 1 ? 1 : P;
    int first = P <= 1 ? 0 : p;
    double delta = g->step * s;
    long K = sample_bound(g, s);
    size_t N = (size_t)ns * ns;
    int nchunk = nsub < 32 ? nsub : 32;
    memset(img, 0, sizeof(double) * N);
    if (nchunk < 1) return;
    double *part = calloc((size_t)nchunk * N, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < nchunk; ++c) {
        double *im = part + (size_t)c * N;
        int v0 = (int)((long)nsub * c / nchunk), v1 = (int)((long)nsub * (c + 1) / nchunk);
        for (int vs = v0; vs < v1; ++vs) {
            int v = first + vs * step;
            for (int j = 0; j < g->n_det; ++j) {
                double r[6];
                orc_ray(g, v, j, r);
                double val = sino[(long)vs * g->n_det + j];
                if (val == 0.0) continue;
                for (long k = -K; k < K; ++k) {
                    double t = ((double)k + 0.5) * delta;
                    scatter(im, ns, s, r[4] + t * r[2], r[5] + t * r[3], delta * val);
                }
            }
        }
    }
    for (int c = 0; c < nchunk; ++c)
        for (size_t i = 0; i < N; ++i) img[i] += part[(size_t)c * N + i];
    free(part);
}

/* Sketch S: s x s average pooling, fine [n][n] -> coarse [n/s][n/s]. */
void orc_pool(int n, int s, const double *fine, double *coarse)
{
    int ns = n / s;
    for (int cy = 0; cy < ns; ++cy) {
        for (int cx = 0; cx < ns; ++cx) {
            double acc = 0.0;
            for (int b = 0; b < s; ++b)
                for (int a = 0; a < s; ++a)
                    acc += fine[(long)(cy * s + b) * n + (cx * s + a)];
            coarse[(long)cy * ns + cx] = acc / (double)(s * s);
        }
    }
}

/* Upsampler U = S^T: replicate each coarse value over its s x s block, / s^2. */
void orc_unpool(int n, int s, const double *coarse, double *fine)
{
    int ns = n / s;
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x)
            fine[(long)y * n + x] = coarse[(long)(y / s) * ns + (x / s)] / (double)(s * s);
}

/* ---------------- bicubic sketch (Sec. 3 uses bicubic imresize for S and U) --
 * Reading: S is separable; coarse pixel I (centre s I + (s-1)/2 in fine index
 * units) averages fine pixels x with weights k((x - X_I)/s), k the Keys cubic
 * convolution kernel with a = -1/2 (widened by s to avoid aliasing), normalised
 * to sum to one over the fine pixels inside the image.  U = S^T. */
double orc_keys(double t)
{
    const double a = -0.5;
    t = fabs(t);
    if (t <= 1.0) return (a + 2.0) * t * t * t - (a + 3.0) * t * t + 1.0;
    if (t < 2.0) return a * t * t * t - 5.0 * a * t * t + 8.0 * a * t - 4.0 * a;
    return 0.0;
}

/* W[I][x], ns x n, the 1-D bicubic sketch. */
static void bicubic_matrix(int n, int s, double *W)
{
    int ns = n / s;
    for (int I = 0; I < ns; ++I) {
        double XI = s * I + 0.5 * (s - 1);
        double den = 0.0;
        for (int x = 0; x < n; ++x) den += orc_keys((x - XI) / s);
        for (int x = 0; x < n; ++x) W[(long)I * n + x] = orc_keys((x - XI) / s) / den;
    }
}

void orc_bicubic_down(int n, int s, const double *fine, double *coarse)
{
    int ns = n / s;
    double *W = malloc(sizeof(double) * (size_t)ns * n), *tmp = malloc(sizeof(double) * (size_t)n * ns);
    bicubic_matrix(n, s, W);
    /* rows: tmp[y][I] = sum_x W[I][x] fine[y][x] */
    for (int y = 0; y < n; ++y)
        for (int I = 0; I < ns; ++I) {
            double acc = 0.0;
            for (int x = 0; x < n; ++x) acc += W[(long)I * n + x] * fine[(long)y * n + x];
            tmp[(long)y * ns + I] = acc;
        }
    /* columns: coarse[J][I] = sum_y W[J][y] tmp[y][I] */
    for (int J = 0; J < ns; ++J)
        for (int I = 0; I < ns; ++I) {
            double acc = 0.0;
            for (int y = 0; y < n; ++y) acc += W[(long)J * n + y] * tmp[(long)y * ns + I];
            coarse[(long)J * ns + I] = acc;
        }
    free(W);
    free(tmp);
}

void orc_bicubic_up(int n, int s, const double *coarse, double *fine)
{
    int ns = n / s;
    double *W = malloc(sizeof(double) * (size_t)ns * n), *tmp = malloc(sizeof(double) * (size_t)n * ns);
    bicubic_matrix(n, s, W);
    /* tmp[y][I] = sum_J W[J][y] coarse[J][I] */
    for (int y = 0; y < n; ++y)
        for (int I = 0; I < ns; ++I) {
            double acc = 0.0;
            for (int J = 0; J < ns; ++J) acc += W[(long)J * n + y] * coarse[(long)J * ns + I];
            tmp[(long)y * ns + I] = acc;
        }
    /* fine[y][x] = sum_I W[I][x] tmp[y][I] */
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x) {
            double acc = 0.0;
            for (int I = 0; I < ns; ++I) acc += W[(long)I * n + x] * tmp[(long)y * ns + I];
            fine[(long)y * n + x] = acc;
        }
    free(W);
    free(tmp);
}

static void sketch_down(int kind, int n, int s, const double *fine, double *coarse)
{
    if (kind == 1) orc_bicubic_down(n, s, fine, coarse);
    else orc_pool(n, s, fine, coarse);
}

static void sketch_up(int kind, int n, int s, const double *coarse, double *fine)
{
    if (kind == 1) orc_bicubic_up(n, s, coarse, fine);
    else orc_unpool(n, s, coarse, fine);
}

/* Gradient estimate on the fine grid (Alg. 1, Option 1 for P<=1, Option 2 with
 * angle subset p of P otherwise):
 *     g = c * S^T A_s^{(p)T} (A_s^{(p)} S y - b^{(p)}),   c = max(P, 1).
 * For s = 1 and P <= 1 this is the full gradient A^T (A y - b) of Eq. 5. */
static void apply_weights(const orc_geom *g, const double *w, double *res, int p, int P)
{
    if (!w) return;
    int nsub = orc_subset_views(g, p, P);
    int step = P <= 1 ? 1 : P;
    int first = P <= 1 ? 0 : p;
    for (int vs = 0; vs < nsub; ++vs)
        for (int j = 0; j < g->n_det; ++j)
            res[(long)vs * g->n_det + j] *= w[(long)(first + vs * step) * g->n_det + j];
}

/* Weighted variant (w nullable, full [n_views][n_det]): the data fidelity is
 * 1/2 sum_j w_j (A x - b)_j^2, the weighted least squares of transmission CT
 * with Poisson counts (Sec. 3's b ~ Poisson(I0 exp(-A x)) after the log), so
 * the gradient is c S^T A_s^{(p)T} W^{(p)} (A_s^{(p)} S y - b^{(p)}). */
void orc_grad_wk(const orc_geom *g, int s, int kind, const double *y, const double *b, const double *w,
                 double *grad, int p, int P)
{
    int n = g->n, ns = n / s;
    int nsub = orc_subset_views(g, p, P);
    double *v = malloc(sizeof(double) * (size_t)ns * ns);
    double *res = malloc(sizeof(double) * (size_t)nsub * g->n_det);
    double *gc = malloc(sizeof(double) * (size_t)ns * ns);
    sketch_down(kind, n, s, y, v);
    orc_project(g, s, v, b, res, p, P);
    apply_weights(g, w, res, p, P);
    orc_backproject(g, s, res, gc, p, P);
    sketch_up(kind, n, s, gc, grad);
    double c = P <= 1 ? 1.0 : (double)P;
    for (long i = 0; i < (long)n * n; ++i) grad[i] *= c;
    free(v);
    free(res);
    free(gc);
}

void orc_grad_w(const orc_geom *g, int s, const double *y, const double *b, const double *w,
                double *grad, int p, int P)
{
    orc_grad_wk(g, s, 0, y, b, w, grad, p, P);
}

void orc_grad(const orc_geom *g, int s, const double *y, const double *b, double *grad, int p, int P)
{
    orc_grad_wk(g, s, 0, y, b, NULL, grad, p, P);
}

/* ---------------- TV prox by FGP (Beck & Teboulle 2009) -------------------
 * Dual variables (p, q) live on the m x m grid; p[i][j] pairs rows i and i+1
 * (zero on the last row), q[i][j] pairs columns j and j+1 (zero on the last
 * column).  L(p,q)[i][j] = p[i][j] + q[i][j] - p[i-1][j] - q[i][j-1];
 * L^T(x) = (x[i][j] - x[i+1][j], x[i][j] - x[i][j+1]).  Isotropic projection
 * (p,q)/max(1, sqrt(p^2+q^2)).  No box constraint (P_C = identity).         */
static void tv_L(int m, const double *p, const double *q, double *out)
{
    for (int i = 0; i < m; ++i) {
        for (int j = 0; j < m; ++j) {
            double v = p[i * m + j] + q[i * m + j];
            if (i > 0) v -= p[(i - 1) * m + j];
            if (j > 0) v -= q[i * m + j - 1];
            out[i * m + j] = v;
        }
    }
}

static void tv_LT(int m, const double *x, double *p, double *q)
{
    for (int i = 0; i < m; ++i) {
        for (int j = 0; j < m; ++j) {
            p[i * m + j] = i < m - 1 ? x[i * m + j] - x[(i + 1) * m + j] : 0.0;
            q[i * m + j] = j < m - 1 ? x[i * m + j] - x[i * m + j + 1] : 0.0;
        }
    }
}

/* x = FGP_lambda^iters(z) on one m x m image. */
void orc_fgp(int m, const double *z, double lambda, int iters, double *x)
{
    size_t N = (size_t)m * m;
    if (lambda <= 0.0 || iters <= 0) {
        memcpy(x, z, sizeof(double) * N);
        return;
    }
    double *pk = calloc(N, sizeof(double)), *qk = calloc(N, sizeof(double));
    double *pp = calloc(N, sizeof(double)), *qp = calloc(N, sizeof(double));
    double *r = calloc(N, sizeof(double)), *sv = calloc(N, sizeof(double));
    double *w = malloc(sizeof(double) * N), *gp = malloc(sizeof(double) * N),
           *gq = malloc(sizeof(double) * N);
    double t = 1.0;
    for (int k = 1; k <= iters; ++k) {
        /* (p_k, q_k) = P_P[(r_k, s_k) + 1/(8 lambda) L^T(z - lambda L(r_k, s_k))] */
        tv_L(m, r, sv, w);
        for (size_t i = 0; i < N; ++i) w[i] = z[i] - lambda * w[i];
        tv_LT(m, w, gp, gq);
        for (size_t i = 0; i < N; ++i) {
            double a = r[i] + gp[i] / (8.0 * lambda);
            double c = sv[i] + gq[i] / (8.0 * lambda);
            double nrm = sqrt(a * a + c * c);
            double den = nrm > 1.0 ? nrm : 1.0;
            pk[i] = a / den;
            qk[i] = c / den;
        }
        /* t_{k+1} and the momentum point (r_{k+1}, s_{k+1}) */
        double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        double mom = (t - 1.0) / tn;
        for (size_t i = 0; i < N; ++i) {
            r[i] = pk[i] + mom * (pk[i] - pp[i]);
            sv[i] = qk[i] + mom * (qk[i] - qp[i]);
            pp[i] = pk[i];
            qp[i] = qk[i];
        }
        t = tn;
    }
    /* x = z - lambda L(p_N, q_N) */
    tv_L(m, pp, qp, w);
    for (size_t i = 0; i < N; ++i) x[i] = z[i] - lambda * w[i];
    free(pk); free(qk); free(pp); free(qp); free(r); free(sv); free(w); free(gp); free(gq);
}

/* Isotropic TV with forward differences and zero differences past the edge. */
double orc_tv(int m, const double *x)
{
    double acc = 0.0;
    for (int i = 0; i < m; ++i) {
        for (int j = 0; j < m; ++j) {
            double a = i < m - 1 ? x[(i + 1) * m + j] - x[i * m + j] : 0.0;
            double c = j < m - 1 ? x[i * m + j + 1] - x[i * m + j] : 0.0;
            acc += sqrt(a * a + c * c);
        }
    }
    return acc;
}

/* L = ||A_s S||^2 by power iteration on S^T A_s^T A_s S from the normalised
 * all-ones vector; stops when the Rayleigh quotient changes by less than tol
 * (relative) or after max_iters.  Returns L; *iters_out = iterations used. */
double orc_power_iter_w(const orc_geom *g, int s, const double *wts, int max_iters, double tol,
                        int *iters_out);

double orc_power_iter(const orc_geom *g, int s, int max_iters, double tol, int *iters_out)
{
    return orc_power_iter_w(g, s, NULL, max_iters, tol, iters_out);
}

double orc_power_iter_wk(const orc_geom *g, int s, int kind, const double *wts, int max_iters,
                         double tol, int *iters_out);

/* L = ||W^{1/2} A_s S||^2 (wts nullable: W = I). */
double orc_power_iter_w(const orc_geom *g, int s, const double *wts, int max_iters, double tol,
                        int *iters_out)
{
    return orc_power_iter_wk(g, s, 0, wts, max_iters, tol, iters_out);
}

/* The same with the sketch of the given kind (0 average pool, 1 bicubic). */
double orc_power_iter_wk(const orc_geom *g, int s, int kind, const double *wts, int max_iters,
                         double tol, int *iters_out)
{
    int n = g->n, ns = n / s;
    size_t N = (size_t)n * n;
    double *u = malloc(sizeof(double) * N), *w = malloc(sizeof(double) * N);
    double *v = malloc(sizeof(double) * (size_t)ns * ns), *gc = malloc(sizeof(double) * (size_t)ns * ns);
    double *res = malloc(sizeof(double) * (size_t)g->n_views * g->n_det);
    for (size_t i = 0; i < N; ++i) u[i] = 1.0 / sqrt((double)N);
    double lam = 0.0;
    int it = 0;
    for (it = 1; it <= max_iters; ++it) {
        sketch_down(kind, n, s, u, v);
        orc_project(g, s, v, NULL, res, 0, 1);
        apply_weights(g, wts, res, 0, 1);
        orc_backproject(g, s, res, gc, 0, 1);
        sketch_up(kind, n, s, gc, w);
        double rq = 0.0, nw = 0.0;
        for (size_t i = 0; i < N; ++i) {
            rq += u[i] * w[i];
            nw += w[i] * w[i];
        }
        nw = sqrt(nw);
        for (size_t i = 0; i < N; ++i) u[i] = w[i] / nw;
        int done = it > 1 && fabs(rq - lam) <= tol * fabs(rq);
        lam = rq;
        if (done) break;
    }
    if (iters_out) *iters_out = it > max_iters ? max_iters : it;
    free(u); free(w); free(v); free(gc); free(res);
    return lam;
}

double orc_psnr(long count, const double *x, const double *xt)
{
    double mse = 0.0;
    for (long i = 0; i < count; ++i) mse += (x[i] - xt[i]) * (x[i] - xt[i]);
    mse /= (double)count;
    return 10.0 * log10(1.0 / mse);
}

/* Algorithm 1 (PnP-MS2G) on one image.
 *   stages      n_stages records (factor s_k, iterations N_k, subsets P_k, sketch kind:
 *               0 average pool, 1 bicubic; subset estimator: 0 vanilla, 1 SVRG, 2 SAGA)
 *   eta         per-stage step sizes eta_k
 *   seq         subset id of every iteration (length sum N_k)
 *   x           in: x_0 (= y_0); out: x after the last iteration
 *   momentum    0: a_i = 0 (PnP proximal gradient, Eq. 5); 1: a_i = (i-1)/(i+3)
 *   xt, psnr    optional ground truth and per-iteration PSNR log
 * Iteration i = 1, 2, ...:  v = S_k y_{i-1};  G per Option 1/2;
 *   z_i = y_{i-1} - eta_k S_k^T G;  x_i = (1-alpha) z_i + alpha D(z_i);
 *   y_i = x_i + a_i (x_i - x_{i-1}).                                          */
void orc_pnp_run_w(const orc_geom *g, int n_stages, const int *stages, const double *eta,
                   const int *seq, const double *b, const double *w, double *x, double alpha,
                   double lambda, int tv_iters, int momentum, const double *xt, double *psnr);

void orc_pnp_run(const orc_geom *g, int n_stages, const int *stages, const double *eta,
                 const int *seq, const double *b, double *x, double alpha, double lambda,
                 int tv_iters, int momentum, const double *xt, double *psnr)
{
    orc_pnp_run_w(g, n_stages, stages, eta, seq, b, NULL, x, alpha, lambda, tv_iters, momentum, xt, psnr);
}

/* ---------------- variance-reduced subset estimators ----------------------
 * Sec. 2 (after the minibatch form of the sketched step) names SVRG and SAGA
 * as drop-in replacements for the vanilla minibatch estimate.  With
 * G_p(y) = orc_grad_wk(..., p, P) (the vanilla estimate on subset p, already
 * scaled by P so that its mean over p is the full sketched gradient):
 *   SVRG (Johnson & Zhang 2013): snapshot yt and mu = full sketched gradient
 *     at yt taken at the start of every epoch (P iterations);
 *     v = G_p(y) - G_p(yt) + mu.
 *   SAGA (Defazio, Bach & Lacoste-Julien 2014): a table psi_j of the last
 *     G_j evaluated for every subset j, filled at the start of the stage;
 *     v = G_p(y) - psi_p + (1/P) sum_j psi_j, then psi_p = G_p(y).        */
void orc_svrg_estimate(const orc_geom *g, int s, int kind, const double *y, const double *yt,
                       const double *mu, const double *b, const double *w, int p, int P, double *out)
{
    size_t N = (size_t)g->n * g->n;
    double *gt = malloc(sizeof(double) * N);
    orc_grad_wk(g, s, kind, y, b, w, out, p, P);
    orc_grad_wk(g, s, kind, yt, b, w, gt, p, P);
    for (size_t q = 0; q < N; ++q) out[q] = out[q] - gt[q] + mu[q];
    free(gt);
}

void orc_saga_estimate(const orc_geom *g, int s, int kind, const double *y, double *psi,
                       const double *b, const double *w, int p, int P, double *out)
{
    size_t N = (size_t)g->n * g->n;
    double *gp = malloc(sizeof(double) * N);
    orc_grad_wk(g, s, kind, y, b, w, gp, p, P);
    for (size_t q = 0; q < N; ++q) {
        double mean = 0.0;
        for (int j = 0; j < P; ++j) mean += psi[(size_t)j * N + q];
        out[q] = gp[q] - psi[(size_t)p * N + q] + mean / (double)P;
    }
    memcpy(psi + (size_t)p * N, gp, sizeof(double) * N);
    free(gp);
}

/* Algorithm 1 with the weighted data fidelity (w nullable).  Stage records
 * hold 5 ints: factor, iterations, subsets P, sketch kind, estimator
 * (0 vanilla minibatch, 1 SVRG, 2 SAGA; the last two only when P > 1). */
void orc_pnp_run_w(const orc_geom *g, int n_stages, const int *stages, const double *eta,
                   const int *seq, const double *b, const double *w, double *x, double alpha,
                   double lambda, int tv_iters, int momentum, const double *xt, double *psnr)
{
    int n = g->n;
    size_t N = (size_t)n * n;
    double *y = malloc(sizeof(double) * N), *xprev = malloc(sizeof(double) * N);
    double *z = malloc(sizeof(double) * N), *gr = malloc(sizeof(double) * N);
    double *dz = malloc(sizeof(double) * N);
    double *yt = malloc(sizeof(double) * N), *mu = malloc(sizeof(double) * N);
    memcpy(y, x, sizeof(double) * N);
    memcpy(xprev, x, sizeof(double) * N);
    int i = 0;
    for (int k = 0; k < n_stages; ++k) {
        int s = stages[5 * k], Nk = stages[5 * k + 1], P = stages[5 * k + 2], kind = stages[5 * k + 3];
        int est = P > 1 ? stages[5 * k + 4] : 0;
        double *psi = est == 2 ? malloc(sizeof(double) * N * (size_t)P) : NULL;
        for (int jj = 0; jj < Nk; ++jj) {
            i += 1;
            int p = P > 1 ? seq[i - 1] : 0;
            if (est == 1) {
                if (jj % P == 0) {   /* new epoch: snapshot and its full gradient */
                    memcpy(yt, y, sizeof(double) * N);
                    orc_grad_wk(g, s, kind, yt, b, w, mu, 0, 1);
                }
                orc_svrg_estimate(g, s, kind, y, yt, mu, b, w, p, P, gr);
            } else if (est == 2) {
                if (jj == 0)         /* table filled at the stage's first iterate */
                    for (int j = 0; j < P; ++j) orc_grad_wk(g, s, kind, y, b, w, psi + (size_t)j * N, j, P);
                orc_saga_estimate(g, s, kind, y, psi, b, w, p, P, gr);
            } else {
                orc_grad_wk(g, s, kind, y, b, w, gr, p, P);
            }
            for (size_t q = 0; q < N; ++q) z[q] = y[q] - eta[k] * gr[q];
            orc_fgp(n, z, lambda, tv_iters, dz);
            double a = momentum ? (double)(i - 1) / (double)(i + 3) : 0.0;
            for (size_t q = 0; q < N; ++q) {
                double xn = (1.0 - alpha) * z[q] + alpha * dz[q];
                y[q] = xn + a * (xn - xprev[q]);
                xprev[q] = xn;
            }
            if (xt && psnr) psnr[i - 1] = orc_psnr((long)N, xprev, xt);
        }
        free(psi);
    }
    memcpy(x, xprev, sizeof(double) * N);
    free(y); free(xprev); free(z); free(gr); free(dz); free(yt); free(mu);
}

/* Objective terms: 1/2 ||A x - b||^2 and TV(x) (Eq. 2 with f least squares). */
void orc_objective_w(const orc_geom *g, const double *x, const double *b, const double *w,
                     double out[2]);

void orc_objective(const orc_geom *g, const double *x, const double *b, double out[2])
{
    orc_objective_w(g, x, b, NULL, out);
}

/* (1/2 sum_j w_j (A x - b)_j^2, TV(x)); w nullable. */
void orc_objective_w(const orc_geom *g, const double *x, const double *b, const double *w,
                     double out[2])
{
    size_t M = (size_t)g->n_views * g->n_det;
    double *res = malloc(sizeof(double) * M);
    orc_project(g, 1, x, b, res, 0, 1);
    double f = 0.0;
    for (size_t i = 0; i < M; ++i) f += (w ? w[i] : 1.0) * res[i] * res[i];
    out[0] = 0.5 * f;
    out[1] = orc_tv(g->n, x);
    free(res);
}

/* Number of samples with a nonzero-support position along every ray of the
 * subset (the exact Joseph sample count used for GRay-samples/s): samples
 * strictly inside the box |x|,|y| < (n_s/2 + 1/2) s. */
double orc_sample_count(const orc_geom *g, int s, int p, int P)
{
    int ns = g->n / s;
    int nsub = orc_subset_views(g, p, P);
    int step = P <= 1 ? 1 : P;
    int first = P <= 1 ? 0 : p;
    double H = (0.5 * ns + 0.5) * s, delta = g->step * s;
    long K = sample_bound(g, s);
    double count = 0.0;
    for (int vs = 0; vs < nsub; ++vs) {
        for (int j = 0; j < g->n_det; ++j) {
            double r[6];
            orc_ray(g, first + vs * step, j, r);
            for (long k = -K; k < K; ++k) {
                double t = ((double)k + 0.5) * delta;
                double qx = r[4] + t * r[2], qy = r[5] + t * r[3];
                if (fabs(qx) < H && fabs(qy) < H) count += 1.0;
            }
        }
    }
    return count;
}

/* ---------------- differentiable form (reverse mode, FP64) ----------------
 * Vector-Jacobian products for unrolling Algorithm 1 (Sec. 2 notes that the
 * sketched iterations can be unrolled and trained end to end).               */

/* FGP with every pre-projection point a_k = r_k + L^T(z - lambda L r_k)/(8 lambda)
 * kept (a: iters x 2 planes), and p_N (pn: 2 planes).  Same recurrence as
 * orc_fgp. */
static void fgp_record(int m, const double *z, double lambda, int iters, double *a, double *pn)
{
    size_t N = (size_t)m * m;
    double *pp = calloc(2 * N, sizeof(double)), *r = calloc(2 * N, sizeof(double));
    double *w = malloc(sizeof(double) * N), *gp = malloc(sizeof(double) * N), *gq = malloc(sizeof(double) * N);
    double t = 1.0;
    for (int k = 1; k <= iters; ++k) {
        double *ak = a + (size_t)(k - 1) * 2 * N;
        tv_L(m, r, r + N, w);
        for (size_t i = 0; i < N; ++i) w[i] = z[i] - lambda * w[i];
        tv_LT(m, w, gp, gq);
        double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        double mom = (t - 1.0) / tn;
        for (size_t i = 0; i < N; ++i) {
            double a1 = r[i] + gp[i] / (8.0 * lambda);
            double a2 = r[N + i] + gq[i] / (8.0 * lambda);
            ak[i] = a1;
            ak[N + i] = a2;
            double nrm = sqrt(a1 * a1 + a2 * a2);
            double den = nrm > 1.0 ? nrm : 1.0;
            double p1 = a1 / den, p2 = a2 / den;
            r[i] = p1 + mom * (p1 - pp[i]);
            r[N + i] = p2 + mom * (p2 - pp[N + i]);
            pp[i] = p1;
            pp[N + i] = p2;
        }
        t = tn;
    }
    memcpy(pn, pp, sizeof(double) * 2 * N);
    free(pp); free(r); free(w); free(gp); free(gq);
}

/* Reverse sweep of FGP: given xbar = dJ/dx for x = FGP_lambda^iters(z), returns
 * zbar = dJ/dz and dJ/dlambda.  With r_{k+1} = (1+m_k) p_k - m_k p_{k-1},
 * p_k = Proj(a_k), a_k = r_k + L^T z/(8 lambda) - L^T L r_k / 8, x = z - lambda L p_N:
 *   pbar_N = -lambda L^T xbar,  lambar = -<xbar, L p_N>;  for k = N..1:
 *   pbar_k += (1+m_k) rbar_{k+1};  carry -m_k rbar_{k+1} to pbar_{k-1};
 *   abar_k = J_Proj(a_k)^T pbar_k;  rbar_k = abar_k - L^T L abar_k / 8;
 *   zbar += L abar_k / (8 lambda);  lambar -= <L abar_k, z> / (8 lambda^2).
 * J_Proj at a with |a| > 1 is (I - a a^T/|a|^2)/|a|, the identity otherwise.   */
void orc_fgp_vjp(int m, const double *z, double lambda, int iters, const double *xbar,
                 double *zbar, double *lambar)
{
    size_t N = (size_t)m * m;
    memcpy(zbar, xbar, sizeof(double) * N);
    *lambar = 0.0;
    if (lambda <= 0.0 || iters <= 0) return;
    double *a = malloc(sizeof(double) * 2 * N * (size_t)iters), *pn = malloc(sizeof(double) * 2 * N);
    double *pbar = calloc(2 * N, sizeof(double)), *carry = calloc(2 * N, sizeof(double));
    double *rbar = calloc(2 * N, sizeof(double)), *abar = malloc(sizeof(double) * 2 * N);
    double *w = malloc(sizeof(double) * N), *u1 = malloc(sizeof(double) * N), *u2 = malloc(sizeof(double) * N);
    double *mom = malloc(sizeof(double) * (size_t)iters);
    fgp_record(m, z, lambda, iters, a, pn);
    double t = 1.0;
    for (int k = 0; k < iters; ++k) {
        double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        mom[k] = (t - 1.0) / tn;
        t = tn;
    }
    /* x = z - lambda L p_N */
    tv_L(m, pn, pn + N, w);
    double acc = 0.0;
    for (size_t i = 0; i < N; ++i) acc += xbar[i] * w[i];
    *lambar = -acc;
    tv_LT(m, xbar, u1, u2);
    for (size_t i = 0; i < N; ++i) {
        carry[i] = -lambda * u1[i];
        carry[N + i] = -lambda * u2[i];
    }
    for (int k = iters; k >= 1; --k) {
        const double *ak = a + (size_t)(k - 1) * 2 * N;
        double mk = mom[k - 1];
        for (size_t i = 0; i < 2 * N; ++i) {
            pbar[i] = carry[i] + (1.0 + mk) * rbar[i];
            carry[i] = -mk * rbar[i];
        }
        for (size_t i = 0; i < N; ++i) {
            double a1 = ak[i], a2 = ak[N + i];
            double nrm = sqrt(a1 * a1 + a2 * a2);
            if (nrm > 1.0) {
                double h1 = a1 / nrm, h2 = a2 / nrm;
                double d = h1 * pbar[i] + h2 * pbar[N + i];
                abar[i] = (pbar[i] - h1 * d) / nrm;
                abar[N + i] = (pbar[N + i] - h2 * d) / nrm;
            } else {
                abar[i] = pbar[i];
                abar[N + i] = pbar[N + i];
            }
        }
        tv_L(m, abar, abar + N, w);                    /* w = L abar */
        double dz = 0.0;
        for (size_t i = 0; i < N; ++i) {
            zbar[i] += w[i] / (8.0 * lambda);
            dz += w[i] * z[i];
        }
        *lambar -= dz / (8.0 * lambda * lambda);
        tv_LT(m, w, u1, u2);                           /* L^T L abar */
        for (size_t i = 0; i < N; ++i) {
            rbar[i] = abar[i] - u1[i] / 8.0;
            rbar[N + i] = abar[N + i] - u2[i] / 8.0;
        }
    }
    free(a); free(pn); free(pbar); free(carry); free(rbar); free(abar); free(w); free(u1); free(u2); free(mom);
}

/* One iteration of Algorithm 1 as a function of (y_{i-1}, x_{i-1}, lambda):
 *   z = y - eta c S^T A_s^{(p)T}(A_s^{(p)} S y - b^{(p)});  d = FGP(z);
 *   x = (1-alpha) z + alpha d;  y_new = x + a (x - xprev).                    */
void orc_step(const orc_geom *g, int s, int p, int P, double eta, double alpha, double lambda,
              int tv_iters, double amom, const double *y, const double *xprev, const double *b,
              double *xout, double *yout)
{
    size_t N = (size_t)g->n * g->n;
    double *gr = malloc(sizeof(double) * N), *z = malloc(sizeof(double) * N), *d = malloc(sizeof(double) * N);
    orc_grad(g, s, y, b, gr, p, P);
    for (size_t i = 0; i < N; ++i) z[i] = y[i] - eta * gr[i];
    orc_fgp(g->n, z, lambda, tv_iters, d);
    for (size_t i = 0; i < N; ++i) {
        double x = (1.0 - alpha) * z[i] + alpha * d[i];
        xout[i] = x;
        yout[i] = x + amom * (x - xprev[i]);
    }
    free(gr); free(z); free(d);
}

/* VJP of orc_step: given xbar, ybar (gradients of the two outputs), returns
 * ybar_in = dJ/dy_{i-1}, xpbar = dJ/dx_{i-1} and dJ/dlambda.  The data step's
 * Jacobian I - eta c S^T A_s^T A_s S is symmetric, so ybar_in is that matrix
 * applied to zbar. */
void orc_step_vjp(const orc_geom *g, int s, int p, int P, double eta, double alpha, double lambda,
                  int tv_iters, double amom, const double *y, const double *b, const double *xbar,
                  const double *ybar, double *ybar_in, double *xpbar, double *lambar)
{
    size_t N = (size_t)g->n * g->n;
    double *gr = malloc(sizeof(double) * N), *z = malloc(sizeof(double) * N);
    double *xt = malloc(sizeof(double) * N), *dz = malloc(sizeof(double) * N), *zbar = malloc(sizeof(double) * N);
    double *zero = calloc((size_t)g->n_views * g->n_det, sizeof(double));
    orc_grad(g, s, y, b, gr, p, P);
    for (size_t i = 0; i < N; ++i) z[i] = y[i] - eta * gr[i];
    for (size_t i = 0; i < N; ++i) {
        xt[i] = xbar[i] + (1.0 + amom) * ybar[i];
        xpbar[i] = -amom * ybar[i];
    }
    double lb = 0.0;
    orc_fgp_vjp(g->n, z, lambda, tv_iters, xt, dz, &lb);
    *lambar = alpha * lb;
    for (size_t i = 0; i < N; ++i) zbar[i] = (1.0 - alpha) * xt[i] + alpha * dz[i];
    orc_grad(g, s, zbar, zero, gr, p, P);
    for (size_t i = 0; i < N; ++i) ybar_in[i] = zbar[i] - eta * gr[i];
    free(gr); free(z); free(xt); free(dz); free(zbar); free(zero);
}

/* Subset order of Algorithm 1's minibatches.
 *
 * Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), used as a counter-based
 * generator: the t-th number (t = 1, 2, ...) of the stream with seed `seed` is
 * the 64-bit finaliser applied to seed + t * gamma, gamma = 0x9e3779b97f4a7c15. */
uint64_t orc_splitmix64(uint64_t seed, uint64_t t)
{
    uint64_t z = seed + t * 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

/* A uniform integer in [0, m), m >= 1, from the stream: take the next number u,
 * discard it while u < 2^64 mod m (so that the accepted range is a whole number
 * of copies of [0, m)), and return u mod m.  *t counts the numbers taken. */
static uint32_t orc_uniform_below(uint64_t seed, uint64_t *t, uint32_t m)
{
    uint64_t reject_below = (0 - (uint64_t)m) % (uint64_t)m;   /* 2^64 mod m */
    for (;;) {
        *t += 1;
        uint64_t u = orc_splitmix64(seed, *t);
        if (u >= reject_below) return (uint32_t)(u % m);
    }
}

/* The subset id of every iteration of the schedule (stages as orc_pnp_run
 * takes them: 5 ints per stage, {factor, iters, n_subsets, kind, estimator}).
 * Stages in order; a stage with P = n_subsets > 1 runs in epochs of P
 * iterations, each epoch visiting the subsets in the order of a new uniform
 * permutation of 0..P-1 (the last epoch of the stage, when shorter, takes the
 * first entries of its permutation); a stage with P = 1 contributes zeros and
 * draws nothing.  A permutation is Durstenfeld's form of the Fisher-Yates
 * shuffle (Knuth, TAOCP vol. 2, Algorithm 3.4.2P) of the identity: for
 * j = P-1 down to 1, swap entry j with entry r, r uniform in [0, j].  One
 * stream serves the whole schedule, its counter running on across epochs and
 * stages.  Writes sum(iters) entries to seq and returns that count. */
long orc_subset_sequence(int n_stages, const int *stages, uint64_t seed, int *seq)
{
    uint64_t t = 0;
    long i = 0;
    for (int k = 0; k < n_stages; ++k) {
        int iters = stages[5 * k + 1], P = stages[5 * k + 2];
        int *perm = (int *)malloc(sizeof(int) * (size_t)(P > 0 ? P : 1));
        for (int done = 0; done < iters;) {
            if (P <= 1) { seq[i++] = 0; ++done; continue; }
            for (int a = 0; a < P; ++a) perm[a] = a;
            for (int j = P - 1; j >= 1; --j) {
                int r = (int)orc_uniform_below(seed, &t, (uint32_t)(j + 1));
                int tmp = perm[j]; perm[j] = perm[r]; perm[r] = tmp;
            }
            for (int a = 0; a < P && done < iters; ++a, ++done) seq[i++] = perm[a];
        }
        free(perm);
    }
    return i;
}

/* Threads of the OpenMP loops (timing only; results do not depend on it). */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
