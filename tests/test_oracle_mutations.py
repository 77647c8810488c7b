"""Plants plausible mistakes in a copy of the oracle's C source (on the CPU) and
checks that the pins in test_oracle_pins.py and test_oracle_vjp.py catch every one."""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "pnp_oracle.c")

# (name, original text, mutated text)
MUTATIONS = [
    ("transposed image in interp", "val += w * img[(long)iy * ns + (long)ix];",
     "val += w * img[(long)ix * ns + (long)iy];"),
    ("dropped sample weight", "return delta * acc;", "return acc;"),
    ("foot point sign", "out[4] = sx - sd * dx;", "out[4] = sx + sd * dx;"),
    ("detector centre offset", "u = ((double)j - 0.5 * (double)(g->n_det - 1)) * g->pitch;",
     "u = ((double)j - 0.5 * (double)(g->n_det)) * g->pitch;"),
    ("view angle direction", "double beta = g->angle0 + g->span * (double)v / (double)g->n_views;",
     "double beta = g->angle0 - g->span * (double)v / (double)g->n_views;"),
    ("transposed scatter", "img[(long)iy * ns + (long)ix] += wt * w;",
     "img[(long)ix * ns + (long)iy] += wt * w;"),
    ("unpool without 1/s^2", "fine[(long)y * n + x] = coarse[(long)(y / s) * ns + (x / s)] / (double)(s * s);",
     "fine[(long)y * n + x] = coarse[(long)(y / s) * ns + (x / s)];"),
    ("pool index swap", "acc += fine[(long)(cy * s + b) * n + (cx * s + a)];",
     "acc += fine[(long)(cx * s + b) * n + (cy * s + a)];"),
    ("subset scale dropped", "double c = P <= 1 ? 1.0 : (double)P;", "double c = 1.0;"),
    ("fgp dual step", "double a = r[i] + gp[i] / (8.0 * lambda);", "double a = r[i] + gp[i] / (4.0 * lambda);"),
    ("fgp momentum dropped", "r[i] = pk[i] + mom * (pk[i] - pp[i]);", "r[i] = pk[i];"),
    ("fgp divergence sign", "if (i > 0) v -= p[(i - 1) * m + j];", "if (i > 0) v += p[(i - 1) * m + j];"),
    ("fgp anisotropic projection", "double nrm = sqrt(a * a + c * c);", "double nrm = fabs(a) + fabs(c);"),
    ("pnp momentum index", "double a = momentum ? (double)(i - 1) / (double)(i + 3) : 0.0;",
     "double a = momentum ? (double)(i) / (double)(i + 3) : 0.0;"),
    ("relaxation swapped", "double xn = (1.0 - alpha) * z[q] + alpha * dz[q];",
     "double xn = alpha * z[q] + (1.0 - alpha) * dz[q];"),
    ("power iteration unnormalised", "for (size_t i = 0; i < N; ++i) u[i] = w[i] / nw;",
     "for (size_t i = 0; i < N; ++i) u[i] = w[i];"),
    ("fgp vjp momentum carry", "carry[i] = -mk * rbar[i];", "carry[i] = mk * rbar[i];"),
    ("fgp vjp projection jacobian", "abar[i] = (pbar[i] - h1 * d) / nrm;", "abar[i] = (pbar[i] + h1 * d) / nrm;"),
    ("fgp vjp lambda term", "*lambar -= dz / (8.0 * lambda * lambda);", "*lambar += dz / (8.0 * lambda * lambda);"),
    ("step vjp momentum", "xt[i] = xbar[i] + (1.0 + amom) * ybar[i];", "xt[i] = xbar[i] + amom * ybar[i];"),
    ("keys kernel coefficient", "if (t <= 1.0) return (a + 2.0) * t * t * t - (a + 3.0) * t * t + 1.0;",
     "if (t <= 1.0) return (a + 2.0) * t * t * t - (a + 2.0) * t * t + 1.0;"),
    ("bicubic adjoint index", "for (int J = 0; J < ns; ++J) acc += W[(long)J * n + y] * coarse[(long)J * ns + I];",
     "for (int J = 0; J < ns; ++J) acc += W[(long)J * n + y] * coarse[(long)I * ns + J];"),
    ("svrg correction sign", "for (size_t q = 0; q < N; ++q) out[q] = out[q] - gt[q] + mu[q];",
     "for (size_t q = 0; q < N; ++q) out[q] = out[q] + gt[q] + mu[q];"),
    ("svrg snapshot gradient on a subset", "orc_grad_wk(g, s, kind, yt, b, w, mu, 0, 1);",
     "orc_grad_wk(g, s, kind, yt, b, w, mu, 0, P);"),
    ("svrg snapshot never refreshed", "if (jj % P == 0) {   /* new epoch",
     "if (jj == 0) {   /* new epoch"),
    ("saga table mean unscaled", "out[q] = gp[q] - psi[(size_t)p * N + q] + mean / (double)P;",
     "out[q] = gp[q] - psi[(size_t)p * N + q] + mean;"),
    ("saga table not updated", "memcpy(psi + (size_t)p * N, gp, sizeof(double) * N);", "(void)0;"),
    ("sample-count box half a pixel small", "double H = (0.5 * ns + 0.5) * s, delta = g->step * s;",
     "double H = (0.5 * ns) * s, delta = g->step * s;"),
    ("sample-count box edge included", "if (fabs(qx) < H && fabs(qy) < H) count += 1.0;",
     "if (fabs(qx) <= H && fabs(qy) <= H) count += 1.0;"),
    ("splitmix64 finaliser shift", "z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;",
     "z = (z ^ (z >> 31)) * 0xbf58476d1ce4e5b9ull;"),
    ("shuffle draws below j (cyclic orders only)",
     "int r = (int)orc_uniform_below(seed, &t, (uint32_t)(j + 1));",
     "int r = (int)orc_uniform_below(seed, &t, (uint32_t)j);"),
    ("stream restarts at every stage", "        int *perm = (int *)malloc(sizeof(int) * (size_t)(P > 0 ? P : 1));",
     "        int *perm = (int *)malloc(sizeof(int) * (size_t)(P > 0 ? P : 1)); t = 0;"),
    ("naive shuffle over the whole range",
     "int r = (int)orc_uniform_below(seed, &t, (uint32_t)(j + 1));",
     "int r = (int)orc_uniform_below(seed, &t, (uint32_t)P);"),
    ("objective without the 1/2", "out[0] = 0.5 * f;", "out[0] = f;"),
    ("objective TV anisotropic", "acc += sqrt(a * a + c * c);", "acc += fabs(a) + fabs(c);"),
    ("objective TV zero past the last row",
     "double a = i < m - 1 ? x[(i + 1) * m + j] - x[i * m + j] : 0.0;",
     "double a = i < m - 1 ? x[(i + 1) * m + j] - x[i * m + j] : -x[i * m + j];"),
    ("psnr of the summed squared error", "mse /= (double)count;", "(void)count;"),
    ("samples at whole steps (half-step offset dropped)",
     "double t = ((double)k + 0.5) * delta;\n        acc += interp(",
     "double t = (double)k * delta;\n        acc += interp("),
    ("contiguous view blocks as subsets", """    int first = P <= 1 ? 0 : p;
#pragma omp parallel for schedule(dynamic, 1)
    for (int vs = 0; vs < nsub; ++vs) {
        int v = first + vs * step;
        for (int j = 0; j < g->n_det; ++j) {
            double val = ray_sum(g, s, img, v, j);""", """    int first = P <= 1 ? 0 : p;
#pragma omp parallel for schedule(dynamic, 1)
    for (int vs = 0; vs < nsub; ++vs) {
        int v = P <= 1 ? vs : first * nsub + vs; (void)step;
        for (int j = 0; j < g->n_det; ++j) {
            double val = ray_sum(g, s, img, v, j);"""),
    ("fgp momentum sequence without the 4", """        /* t_{k+1} and the momentum point (r_{k+1}, s_{k+1}) */
        double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));""", """        /* t_{k+1} and the momentum point (r_{k+1}, s_{k+1}) */
        double tn = 0.5 * (1.0 + sqrt(1.0 + t * t));"""),
    ("keys kernel a = -3/4", "const double a = -0.5;", "const double a = -0.75;"),
    ("source at the detector distance", "double sx = g->dso * cb, sy = g->dso * sb;",
     "double sx = g->ddo * cb, sy = g->ddo * sb;"),
    ("pixel centres half a pixel off",
     "    double X = qx / s + 0.5 * (ns - 1), Y = qy / s + 0.5 * (ns - 1);\n    double fx = floor(X), fy = floor(Y);\n    double val = 0.0;",
     "    double X = qx / s + 0.5 * ns, Y = qy / s + 0.5 * ns;\n    double fx = floor(X), fy = floor(Y);\n    double val = 0.0;"),
    ("residual sign flipped", "if (b) val -= b[(long)v * g->n_det + j];", "if (b) val = b[(long)v * g->n_det + j] - val;"),
    ("uneven subsets rounded down", "return (g->n_views - p + P - 1) / P;", "return g->n_views / P;"),
    ("weights on the wrong views", "res[(long)vs * g->n_det + j] *= w[(long)(first + vs * step) * g->n_det + j];",
     "res[(long)vs * g->n_det + j] *= w[(long)vs * g->n_det + j];"),
]


@pytest.mark.parametrize("name,orig,mut", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(name, orig, mut, tmp_path):
    src = open(SRC).read()
    assert src.count(orig) == 1, f"mutation anchor not found once: {name}"
    msrc = tmp_path / "mut.c"
    msrc.write_text(src.replace(orig, mut))
    lib = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-o", str(lib),
                    str(msrc), "-lm"], check=True)
    env = dict(os.environ, PNP_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        os.path.join(ROOT, "tests", "test_oracle_vjp.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins did not catch: {name}\n{r.stdout[-2000:]}"
