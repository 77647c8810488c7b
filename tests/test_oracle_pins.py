"""Pins of the FP64 oracle against what mathematics and the paper fix.

None of these compares the oracle with itself: each checks it against a closed
form, a special case, an identity, or a brute-force restatement written here in
a different way (dense matrices, rotation matrices, hat weights over all
pixels, a different TV solver).
"""
import dataclasses
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2203_07308_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers
def rot(beta):
    c, s = math.cos(beta), math.sin(beta)
    return np.array([[c, -s], [s, c]])


def ray_endpoints(g, v, j):
    """Source and detector-bin centre of ray (v, j), via a rotation of the
    view-0 frame (source on +x, detector on the line x = -ddo)."""
    beta = g.angle0 + g.angle_span * v / g.n_views
    u = (j - (g.n_det - 1) / 2.0) * g.det_pitch
    R = rot(beta)
    return R @ np.array([g.dso, 0.0]), R @ np.array([-g.ddo, u])


def line_distance(c, S, P):
    e = P - S
    w = np.asarray(c) - S
    return abs(e[0] * w[1] - e[1] * w[0]) / np.hypot(*e)


def pixel_centres(n, s=1):
    ns = n // s
    c = (np.arange(ns) - (ns - 1) / 2.0) * s
    X, Y = np.meshgrid(c, c, indexing="xy")
    return X, Y


def dense_rows(g, s):
    """Rows of A_s enumerated directly: for every ray, every sample on the
    foot-point grid, the hat weights of *every* pixel (no tap selection)."""
    ns = g.n // s
    X, Y = pixel_centres(g.n, s)
    xs, ys = X.ravel(), Y.ravel()
    delta = g.step * s
    half = (ns / 2 + 0.5) * s
    kmax = int(math.ceil(math.sqrt(2) * half / delta)) + 3
    t = (np.arange(-kmax, kmax) + 0.5) * delta
    rows = []
    for v in range(g.n_views):
        for j in range(g.n_det):
            S, P = ray_endpoints(g, v, j)
            d = (P - S) / np.hypot(*(P - S))
            F = S - np.dot(S, d) * d
            qx = F[0] + t * d[0]
            qy = F[1] + t * d[1]
            wx = np.clip(1 - np.abs(qx[:, None] - xs[None, :]) / s, 0, None)
            wy = np.clip(1 - np.abs(qy[:, None] - ys[None, :]) / s, 0, None)
            rows.append(delta * (wx * wy).sum(axis=0))
    return np.array(rows)


def dense_cols(g, s):
    ns = g.n // s
    cols = []
    for i in range(ns * ns):
        e = np.zeros(ns * ns)
        e[i] = 1.0
        cols.append(oracle.project(g, s, e.reshape(ns, ns)).ravel())
    return np.array(cols).T


def pool_matrix(n, s):
    ns = n // s
    S = np.zeros((ns * ns, n * n))
    for y in range(n):
        for x in range(n):
            S[(y // s) * ns + x // s, y * n + x] = 1.0 / (s * s)
    return S


@pytest.fixture(scope="module")
def g16():
    return synth.make_geometry(16, 12, 24)


@pytest.fixture(scope="module")
def dense16(g16):
    return {s: dense_rows(g16, s) for s in (1, 2)}


# ---------------------------------------------------------------- forward operator A
def test_gaussian_blob_line_integrals():
    """Off-centre Gaussian: the line integral is sigma sqrt(2 pi) exp(-d^2/2 sigma^2),
    d the distance from the blob centre to the ray line (geometry recomputed here)."""
    g = synth.make_geometry(64, 24, 96)
    sig, c = 5.0, (9.0, -6.0)
    X, Y = pixel_centres(64)
    img = np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2) / (2 * sig * sig))
    sino = oracle.project(g, 1, img)
    exact = np.zeros_like(sino)
    for v in range(g.n_views):
        for j in range(g.n_det):
            S, P = ray_endpoints(g, v, j)
            dist = line_distance(c, S, P)
            exact[v, j] = sig * math.sqrt(2 * math.pi) * math.exp(-dist * dist / (2 * sig * sig))
    err = np.abs(sino - exact).max() / exact.max()
    # bilinear interpolation error of a smooth bump: O(h^2 f''/f) = O(1/sigma^2)
    assert err < 0.25 / sig ** 2, err
    # the blob must not be found at the transposed position
    swapped = np.zeros_like(sino)
    for v in range(g.n_views):
        for j in range(g.n_det):
            S, P = ray_endpoints(g, v, j)
            dist = line_distance((c[1], c[0]), S, P)
            swapped[v, j] = sig * math.sqrt(2 * math.pi) * math.exp(-dist * dist / (2 * sig * sig))
    assert np.abs(sino - swapped).max() / exact.max() > 0.1


def test_centred_disk_chord_lengths():
    """Binary disk of radius r (pixels whose centre lies inside): a ray at
    distance p < r from the centre has line integral ~ 2 sqrt(r^2 - p^2), the
    chord.  The pixelised edge moves each end of the chord by at most about one
    pixel, so the error is O(1) pixel-lengths (below 1.5 away from grazing
    rays, under half a pixel on average) and its ratio to the diameter halves
    when the grid is refined with the disk fixed relative to the image."""
    rel_errs = []
    for n in (64, 128):
        g = synth.make_geometry(n, 12, 96)
        r = 0.3 * n
        X, Y = pixel_centres(n)
        img = (X ** 2 + Y ** 2 <= r * r).astype(float)
        sino = oracle.project(g, 1, img)
        errs = []
        for v in range(g.n_views):
            for j in range(g.n_det):
                S, P = ray_endpoints(g, v, j)
                p = line_distance((0.0, 0.0), S, P)
                if p < r - 2.0:
                    errs.append(abs(sino[v, j] - 2.0 * math.sqrt(r * r - p * p)))
        errs = np.array(errs)
        assert errs.size > 100 and errs.max() < 1.5 and errs.mean() < 0.5, (n, errs.max(), errs.mean())
        rel_errs.append(errs.mean() / (2 * r))
    assert rel_errs[1] < 0.7 * rel_errs[0], rel_errs


def test_paraboloid_closed_form_and_order():
    """max(0, r^2 - rho^2) has line integral (4/3)(r^2 - p^2)^{3/2}; the error
    falls at second order when the grid is refined (same physical object)."""
    errs = []
    for n in (32, 64, 128):
        g = synth.make_geometry(n, 8, 64)
        r = 0.3 * n
        X, Y = pixel_centres(n)
        img = np.clip(r * r - X ** 2 - Y ** 2, 0, None) / (r * r)
        sino = oracle.project(g, 1, img)
        exact = np.zeros_like(sino)
        for v in range(g.n_views):
            for j in range(g.n_det):
                S, P = ray_endpoints(g, v, j)
                p = line_distance((0.0, 0.0), S, P)
                exact[v, j] = (4.0 / 3.0) * max(r * r - p * p, 0.0) ** 1.5 / (r * r)
        errs.append(np.abs(sino - exact).max() / exact.max())
    assert errs[1] < 1e-2
    # observed order over two grid doublings (the kink at rho = r makes single
    # doublings irregular)
    assert math.log2(errs[0] / errs[2]) / 2 > 1.6, errs


def test_paraboloid_closed_form_unequal_distances():
    """The paraboloid's closed form again with the source and the detector at
    different distances (source 3n from the centre, detector n on the other
    side), so that each ray's distance from the centre depends on both: an
    exchanged distance or magnification moves every off-centre ray."""
    n = 64
    g = synth.make_geometry(n, 8, 64, dso_ratio=3.0, ddo_ratio=1.0)
    r = 0.3 * n
    X, Y = pixel_centres(n)
    img = np.clip(r * r - X ** 2 - Y ** 2, 0, None) / (r * r)
    sino = oracle.project(g, 1, img)
    exact = np.zeros_like(sino)
    for v in range(g.n_views):
        for j in range(g.n_det):
            S, P = ray_endpoints(g, v, j)
            p = line_distance((0.0, 0.0), S, P)
            exact[v, j] = (4.0 / 3.0) * max(r * r - p * p, 0.0) ** 1.5 / (r * r)
    assert np.abs(sino - exact).max() / exact.max() < 1e-2


def test_axis_rays_are_row_and_column_sums():
    """With an odd grid and an odd detector the central ray of the view at 0 runs
    along the middle row and the one at 90 degrees along the middle column; the
    fixed-step sample sum of the linear interpolant is then the exact row/column sum."""
    n = 33
    g = synth.Geometry(n=n, n_views=4, n_det=31, dso=80.0, ddo=60.0, det_pitch=1.7)
    rng = np.random.default_rng(1)
    img = rng.random((n, n))
    sino = oracle.project(g, 1, img)
    mid = (n - 1) // 2
    jc = (g.n_det - 1) // 2
    assert abs(sino[0, jc] - img[mid, :].sum()) < 1e-11
    assert abs(sino[1, jc] - img[:, mid].sum()) < 1e-11
    assert abs(sino[2, jc] - img[mid, :].sum()) < 1e-11
    # even grid: the axis ray passes between the two middle rows -> their mean
    n2 = 32
    g2 = synth.Geometry(n=n2, n_views=4, n_det=31, dso=80.0, ddo=60.0, det_pitch=1.7)
    img2 = rng.random((n2, n2))
    s2 = oracle.project(g2, 1, img2)
    assert abs(s2[0, jc] - 0.5 * (img2[15, :].sum() + img2[16, :].sum())) < 1e-11


@pytest.mark.parametrize("s", [1, 2])
def test_dense_matrix_two_ways(g16, dense16, s):
    """Columns A_s e_i from the oracle equal the rows enumerated directly."""
    rows = dense16[s]
    cols = dense_cols(g16, s)
    assert rows.shape == cols.shape == (g16.n_views * g16.n_det, (16 // s) ** 2)
    assert np.abs(rows - cols).max() < 1e-13 * np.abs(rows).max()


@pytest.mark.parametrize("s", [1, 2])
def test_backprojection_is_dense_transpose(g16, dense16, s):
    rng = np.random.default_rng(2)
    y = rng.standard_normal((g16.n_views, g16.n_det))
    bp = oracle.backproject(g16, s, y).ravel()
    ref = dense16[s].T @ y.ravel()
    assert np.abs(bp - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("P,p", [(1, 0), (4, 1), (7, 6)])
def test_adjoint_identity(P, p):
    g = synth.make_geometry(48, 30, 64)
    rng = np.random.default_rng(3 + p)
    for s in (1, 2, 4):
        x = rng.random((48 // s, 48 // s))
        nsub = oracle.subset_views(g, p, P)
        y = rng.standard_normal((nsub, g.n_det))
        lhs = np.vdot(oracle.project(g, s, x, None, p, P), y)
        rhs = np.vdot(x, oracle.backproject(g, s, y, p, P))
        assert abs(lhs - rhs) < 1e-12 * max(abs(lhs), 1.0)


def test_subset_rows_are_interleaved_views():
    g = synth.make_geometry(32, 10, 40)
    rng = np.random.default_rng(4)
    x = rng.random((32, 32))
    full = oracle.project(g, 1, x)
    for P in (3, 4):
        for p in range(P):
            sub = oracle.project(g, 1, x, None, p, P)
            assert np.array_equal(sub, full[p::P])
    assert oracle.subset_views(g, 1, 3) == 3 and oracle.subset_views(g, 0, 3) == 4


def test_noise_free_residual_is_zero():
    g = synth.make_geometry(32, 20, 48)
    x = synth.ellipse_phantom(32, 5)
    b = oracle.project(g, 1, x)
    r = oracle.project(g, 1, x, b)
    assert np.abs(r).max() == 0.0


# ---------------------------------------------------------------- sketch S and U = S^T
def test_pool_closed_forms_and_adjoint():
    n = 16
    X, Y = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float), indexing="xy")
    for s in (2, 4):
        v = oracle.pool(X + 3 * Y, s)
        ic = np.arange(n // s)
        CX, CY = np.meshgrid(ic, ic, indexing="xy")
        expect = s * CX + (s - 1) / 2 + 3 * (s * CY + (s - 1) / 2)
        assert np.abs(v - expect).max() < 1e-13
        assert np.abs(oracle.unpool(np.full((n // s, n // s), 2.0), s) - 2.0 / (s * s)).max() == 0
        rng = np.random.default_rng(s)
        x = rng.standard_normal((n, n))
        c = rng.standard_normal((n // s, n // s))
        assert abs(np.vdot(oracle.pool(x, s), c) - np.vdot(x, oracle.unpool(c, s))) < 1e-12
        assert np.abs(oracle.pool(x, s).ravel() - pool_matrix(n, s) @ x.ravel()).max() < 1e-14


def test_sketched_operator_consistent_with_full():
    """A_s S x approximates A x for a smooth object (both near the closed form)."""
    g = synth.make_geometry(64, 16, 96)
    sig, c = 7.0, (-5.0, 8.0)
    X, Y = pixel_centres(64)
    img = np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2) / (2 * sig * sig))
    full = oracle.project(g, 1, img)
    for s in (2, 4):
        sk = oracle.project(g, s, oracle.pool(img, s))
        assert np.abs(sk - full).max() / full.max() < 0.02 * s * s


# ---------------------------------------------------------------- gradient estimates
@pytest.mark.parametrize("s,P,p", [(1, 1, 0), (2, 1, 0), (2, 3, 2), (4, 5, 1)])
def test_gradient_matches_finite_differences(s, P, p):
    """c S^T A_s^{(p)T}(A_s^{(p)} S y - b^{(p)}) is the gradient of
    (c/2)||A_s^{(p)} S y - b^{(p)}||^2; the function is quadratic, so central
    differences are exact up to rounding."""
    g = synth.make_geometry(16, 15, 24)
    rng = np.random.default_rng(10 * s + p)
    y = rng.random((16, 16))
    b = rng.standard_normal((g.n_views, g.n_det)) * 5
    c = max(P, 1)

    def f(yy):
        r = oracle.project(g, s, oracle.pool(yy, s), b, p, P)
        return 0.5 * c * np.vdot(r, r)

    gr = oracle.grad(g, s, y, b, p, P)
    h = 1e-3
    for _ in range(3):
        d = rng.standard_normal((16, 16))
        fd = (f(y + h * d) - f(y - h * d)) / (2 * h)
        assert abs(fd - np.vdot(gr, d)) < 1e-8 * max(abs(fd), 1.0)


@pytest.mark.parametrize("s", [1, 2])
def test_subset_gradients_average_to_full(s):
    g = synth.make_geometry(24, 18, 32)
    rng = np.random.default_rng(20 + s)
    y = rng.random((24, 24))
    b = rng.standard_normal((g.n_views, g.n_det))
    full = oracle.grad(g, s, y, b)
    for P in (4, 7):
        mean = sum(oracle.grad(g, s, y, b, p, P) for p in range(P)) / P
        assert np.abs(mean - full).max() < 1e-12 * np.abs(full).max()


def test_full_gradient_is_dense_normal_equation(g16, dense16):
    rng = np.random.default_rng(30)
    x = rng.random((16, 16))
    b = rng.standard_normal((g16.n_views, g16.n_det))
    A = dense16[1]
    ref = A.T @ (A @ x.ravel() - b.ravel())
    assert np.abs(oracle.grad(g16, 1, x, b).ravel() - ref).max() < 1e-11 * np.abs(ref).max()


# ---------------------------------------------------------------- step size
@pytest.mark.parametrize("s", [1, 2])
def test_power_iteration_matches_dense_eigenvalue(g16, dense16, s):
    M = dense16[s] @ pool_matrix(16, s)
    lmax = np.linalg.eigvalsh(M.T @ M).max()
    L, it = oracle.power_iter(g16, s, max_iters=3000, tol=1e-14)
    assert abs(L - lmax) < 1e-8 * lmax, (L, lmax, it)


# ---------------------------------------------------------------- TV prox (FGP)
def tv_grad_np(x):
    """Forward differences (rows, columns), zero past the last row/column."""
    gy = np.zeros_like(x)
    gx = np.zeros_like(x)
    gy[:-1, :] = np.diff(x, axis=0)
    gx[:, :-1] = np.diff(x, axis=1)
    return gy, gx


def tv_div_np(py, px):
    """Negative adjoint of tv_grad_np (checked by the test below)."""
    d = np.zeros_like(py)
    d[:-1, :] += py[:-1, :]
    d[1:, :] -= py[:-1, :]
    d[:, :-1] += px[:, :-1]
    d[:, 1:] -= px[:, :-1]
    return d


def chambolle_pock_tv(z, lam, iters=20000):
    """Independent TV-prox solve (primal-dual hybrid gradient, tau sigma ||grad||^2 < 1)."""
    x = z.copy()
    xb = z.copy()
    py = np.zeros_like(z)
    px = np.zeros_like(z)
    tau = sig = 1.0 / math.sqrt(8.0) * 0.99
    for _ in range(iters):
        gy, gx = tv_grad_np(xb)
        py, px = py + sig * gy, px + sig * gx
        nrm = np.maximum(1.0, np.sqrt(py ** 2 + px ** 2) / lam)
        py, px = py / nrm, px / nrm
        xn = (x + tau * tv_div_np(py, px) + tau * z) / (1 + tau)
        xb = 2 * xn - x
        x = xn
    return x


def test_tv_div_is_negative_adjoint():
    rng = np.random.default_rng(40)
    x = rng.standard_normal((7, 7))
    py, px = rng.standard_normal((2, 7, 7))
    py[-1, :] = 0
    px[:, -1] = 0
    gy, gx = tv_grad_np(x)
    assert abs(np.vdot(gy, py) + np.vdot(gx, px) + np.vdot(x, tv_div_np(py, px))) < 1e-12


def test_fgp_fixed_points_and_identity():
    z = np.full((12, 12), 0.37)
    assert np.abs(oracle.fgp(z, 0.05, 20) - z).max() < 1e-15
    rng = np.random.default_rng(41)
    z = rng.random((12, 12))
    assert np.abs(oracle.fgp(z, 1e-12, 20) - z).max() < 1e-11
    assert np.array_equal(oracle.fgp(z, 0.05, 0), z)


def test_fgp_converges_to_step_closed_form():
    """An image constant along rows with one jump: the TV prox moves each side by
    lambda / (half width) towards the other (1-D TV prox of a step, per row)."""
    m, lam, a, c = 16, 0.05, 0.8, 0.3
    z = np.full((m, m), c)
    z[:, : m // 2] = a
    x = oracle.fgp(z, lam, 3000)
    expect = np.full((m, m), c + lam / (m // 2))
    expect[:, : m // 2] = a - lam / (m // 2)
    assert np.abs(x - expect).max() < 1e-7


def test_fgp_converges_to_independent_tv_prox():
    rng = np.random.default_rng(42)
    z = rng.random((8, 8))
    lam = 0.08
    ref = chambolle_pock_tv(z, lam)
    x = oracle.fgp(z, lam, 6000)
    assert np.abs(x - ref).max() < 1e-6
    # and it minimises the prox objective better than perturbations of itself
    obj = lambda u: 0.5 * np.sum((u - z) ** 2) + lam * oracle.tv(u)
    for k in range(5):
        d = rng.standard_normal(z.shape) * 1e-3
        assert obj(x) <= obj(x + d) + 1e-12


def test_fgp_twenty_iterations_match_dense_fista():
    """20 FGP iterations equal generic FISTA (Beck & Teboulle 2009) on the dual
    h(p) = ||z - lam L p||^2 over the product of unit disks, with L built densely
    from its definition (the negative adjoint of forward differences)."""
    m, lam, iters = 6, 0.1, 20
    rng = np.random.default_rng(43)
    z = rng.random((m, m))
    N = m * m
    G = np.zeros((2 * N, N))  # forward differences, stacked (rows, columns)
    for i in range(N):
        e = np.zeros(N)
        e[i] = 1
        gy, gx = tv_grad_np(e.reshape(m, m))
        G[:N, i] = gy.ravel()
        G[N:, i] = gx.ravel()
    L = -G.T  # B&T: L^T x = (x[i]-x[i+1], x[j]-x[j+1]) = -grad x

    def proj(v):
        a, c = v[:N], v[N:]
        nrm = np.maximum(1.0, np.hypot(a, c))
        return np.concatenate([a / nrm, c / nrm])

    step = 1.0 / (16 * lam * lam)          # 1 / Lipschitz(grad h), ||L||^2 <= 8
    grad_h = lambda v: -2 * lam * L.T @ (z.ravel() - lam * L @ v)
    xk = np.zeros(2 * N)
    yk = xk.copy()
    t = 1.0
    for _ in range(iters):
        xn = proj(yk - step * grad_h(yk))
        tn = (1 + math.sqrt(1 + 4 * t * t)) / 2
        yk = xn + (t - 1) / tn * (xn - xk)
        xk, t = xn, tn
    ref = z.ravel() - lam * L @ xk
    assert np.abs(oracle.fgp(z, lam, iters).ravel() - ref).max() < 1e-13


def test_tv_of_step_image():
    z = np.zeros((10, 10))
    z[:, 4:] = 2.0
    assert abs(oracle.tv(z) - 10 * 2.0) < 1e-13


def test_tv_of_diagonal_ramp_is_isotropic():
    """Isotropic TV with forward differences and nothing past the last row or
    column (the denoiser's TV_iso): on x[i, j] = i + 2 j every pixel off the last
    row and column has gradient (1, 2), norm sqrt 5 (anisotropic TV would give
    3); the last row has (0, 2), the last column (1, 0), the corner 0:
    TV = (m-1)^2 sqrt 5 + 2 (m-1) + (m-1)."""
    m = 9
    i, j = np.mgrid[0:m, 0:m].astype(np.float64)
    want = (m - 1) ** 2 * np.sqrt(5.0) + 3.0 * (m - 1)
    assert abs(oracle.tv(i + 2.0 * j) - want) < 1e-12


# ---------------------------------------------------------------- Algorithm 1
def dense_alg1(A_by_s, S_by_s, stages, eta, seq, b, x0, alpha, lam, tv_iters, momentum, nv):
    """Algorithm 1 with dense A_s and S matrices (U = S^T, subsets = interleaved rows)."""
    y = x0.ravel().copy()
    xp = y.copy()
    i = 0
    nd = b.shape[1]
    for k, (s, Nk, P) in enumerate(stages):
        A, S = A_by_s[s], S_by_s[s]
        for _ in range(Nk):
            i += 1
            p = seq[i - 1] if P > 1 else 0
            views = np.arange(nv)[p::P] if P > 1 else np.arange(nv)
            rows = (views[:, None] * nd + np.arange(nd)[None, :]).ravel()
            M = A[rows] @ S
            G = max(P, 1) * M.T @ (M @ y - b.ravel()[rows])
            z = y - eta[k] * G
            n = int(round(math.sqrt(z.size)))
            dz = oracle.fgp(z.reshape(n, n), lam, tv_iters).ravel()
            xn = (1 - alpha) * z + alpha * dz
            a = (i - 1) / (i + 3) if momentum else 0.0
            y = xn + a * (xn - xp)
            xp = xn
    return xp


def test_pgd_special_case(g16, dense16):
    """One stage, s = 1, P = 1, a_i = 0, alpha = 1: x_1 = D(x_0 - eta A^T(A x_0 - b)) (Eq. 5)."""
    rng = np.random.default_rng(50)
    A = dense16[1]
    xt = synth.ellipse_phantom(16, 9, (3, 3))
    b = (A @ xt.ravel()).reshape(g16.n_views, g16.n_det)
    x0 = rng.random((16, 16)) * 0.1
    eta = 1.0 / np.linalg.eigvalsh(A.T @ A).max()
    x1, _ = oracle.pnp_run(g16, [synth.Stage(1, 1, 1)], [eta], [0], b, x0,
                           alpha=1.0, lam=0.02, tv_iters=20, momentum=False)
    z = x0.ravel() - eta * A.T @ (A @ x0.ravel() - b.ravel())
    ref = oracle.fgp(z.reshape(16, 16), 0.02, 20)
    assert np.abs(x1 - ref).max() < 1e-12


def test_multistage_subsets_momentum_relaxation(g16, dense16):
    """Four iterations over two stages (2x sketch with 3 subsets, then full grid
    with 2 subsets), FISTA momentum and alpha < 1, against the dense restatement."""
    rng = np.random.default_rng(51)
    Ad = {1: dense16[1], 2: dense16[2]}
    Sd = {1: np.eye(256), 2: pool_matrix(16, 2)}
    xt = synth.ellipse_phantom(16, 11, (4, 4))
    b = (Ad[1] @ xt.ravel()).reshape(g16.n_views, g16.n_det) + 0.05 * rng.standard_normal((12, 24))
    stages = [(2, 2, 3), (1, 2, 2)]
    eta = [0.8 / np.linalg.eigvalsh((Ad[2] @ Sd[2]).T @ (Ad[2] @ Sd[2])).max(),
           0.9 / np.linalg.eigvalsh(Ad[1].T @ Ad[1]).max()]
    seq = [2, 0, 1, 0]
    x0 = rng.random((16, 16)) * 0.2
    x, log = oracle.pnp_run(g16, stages, eta, seq, b, x0, alpha=0.7, lam=0.03, tv_iters=20,
                            momentum=True, xt=xt)
    ref = dense_alg1(Ad, Sd, stages, eta, seq, b, x0, 0.7, 0.03, 20, True, g16.n_views)
    assert np.abs(x.ravel() - ref).max() < 1e-12
    assert log.shape == (4,) and abs(log[-1] - 10 * math.log10(1 / np.mean((ref - xt.ravel()) ** 2))) < 1e-9


# ---------------------------------------------------------------- SVRG / SAGA subset estimators
def _vr_problem():
    g = synth.make_geometry(16, 24, 24)
    rng = np.random.default_rng(70)
    xt = synth.ellipse_phantom(16, 9, (3, 3))
    b = oracle.project(g, 1, xt) + 0.3 * rng.standard_normal((24, 24))
    return g, b, rng


@pytest.mark.parametrize("s,kind", [(1, 0), (2, 0), (4, 1)])
def test_svrg_estimate_unbiased_and_exact_at_snapshot(s, kind):
    """Mean over the P subsets of the SVRG estimate is the full sketched gradient
    at y (each G_p is affine and averages to it); at y = yt every subset returns
    the snapshot gradient itself (zero variance at the snapshot)."""
    g, b, rng = _vr_problem()
    P = 4
    y, yt = rng.random((16, 16)), rng.random((16, 16))
    mu = oracle.grad(g, s, yt, b, kind=kind)
    full = oracle.grad(g, s, y, b, kind=kind)
    mean = sum(oracle.svrg_estimate(g, s, y, yt, mu, b, p, P, kind=kind) for p in range(P)) / P
    assert np.abs(mean - full).max() < 1e-10 * np.abs(full).max()
    for p in range(P):
        v = oracle.svrg_estimate(g, s, yt, yt, mu, b, p, P, kind=kind)
        assert np.abs(v - mu).max() < 1e-10 * np.abs(mu).max()


def test_saga_estimate_unbiased_and_table_update():
    """Mean over p of the SAGA estimate is the full gradient at y for any table;
    the call replaces only row p of the table, with G_p(y)."""
    g, b, rng = _vr_problem()
    P, s = 3, 2
    y = rng.random((16, 16))
    psi = rng.standard_normal((P, 16, 16))
    full = oracle.grad(g, s, y, b)
    vs = [oracle.saga_estimate(g, s, y, psi.copy(), b, p, P) for p in range(P)]
    assert np.abs(sum(vs) / P - full).max() < 1e-10 * np.abs(full).max()
    t = psi.copy()
    oracle.saga_estimate(g, s, y, t, b, 1, P)
    assert np.array_equal(t[0], psi[0]) and np.array_equal(t[2], psi[2])
    gp = oracle.grad(g, s, y, b, 1, P)
    assert np.abs(t[1] - gp).max() < 1e-12 * np.abs(gp).max()


def test_variance_reduction_converges_where_minibatch_stalls():
    """Constant step 0.5/L on the 4x-sketched least-squares problem (16 coarse
    unknowns, noisy data, D = identity, no momentum): the vanilla minibatch
    iteration stalls at a noise floor, SVRG and SAGA converge linearly to the
    least-squares minimiser (relative objective gap below 1e-7 after 600
    iterations; vanilla above 1e-4)."""
    g, b, _ = _vr_problem()
    s = 4
    cols = []
    for k in range(256):
        e = np.zeros(256)
        e[k] = 1.0
        cols.append(oracle.project(g, s, oracle.pool(e.reshape(16, 16), s)).ravel())
    M = np.array(cols).T
    L = np.linalg.eigvalsh(M.T @ M).max()
    c, *_ = np.linalg.lstsq(M, b.ravel(), rcond=None)
    fstar = 0.5 * np.sum((M @ c - b.ravel()) ** 2)
    gaps = {}
    for est in (0, 1, 2):
        stages = [synth.Stage(s, 600, 6, estimator=est)]
        seq = synth.schedule_sequence(stages, 5)
        x, _ = oracle.pnp_run(g, stages, [0.5 / L], seq, b, None, lam=0.0, tv_iters=0, momentum=False)
        gaps[est] = (0.5 * np.sum((M @ x.ravel() - b.ravel()) ** 2) - fstar) / fstar
    assert gaps[0] > 1e-4, gaps
    assert gaps[1] < 1e-7 and gaps[2] < 1e-7, gaps


def dense_vr(A, S, Nk, P, est, eta, seq, b, x0, nv):
    """One stage of Algorithm 1 with an SVRG or SAGA subset estimate, dense
    matrices, D = identity, no momentum."""
    nd = b.shape[1]
    M = A @ S
    rows = [(np.arange(nv)[p::P][:, None] * nd + np.arange(nd)[None, :]).ravel() for p in range(P)]
    Gp = lambda y, p: P * M[rows[p]].T @ (M[rows[p]] @ y - b.ravel()[rows[p]])  # noqa: E731
    y = x0.ravel().copy()
    tab = [Gp(y, j) for j in range(P)] if est == 2 else None
    for jj in range(Nk):
        p = seq[jj]
        if est == 1:
            if jj % P == 0:
                yt = y.copy()
                mu = M.T @ (M @ yt - b.ravel())
            v = Gp(y, p) - Gp(yt, p) + mu
        else:
            gnew = Gp(y, p)
            v = gnew - tab[p] + sum(tab) / P
            tab[p] = gnew
        y = y - eta * v
    return y


@pytest.mark.parametrize("est", [1, 2])
def test_vr_run_matches_dense_restatement(g16, dense16, est):
    """Seven iterations (two epochs and a part) of a 2x-sketched stage with three
    subsets: the oracle's loop against dense matrices."""
    rng = np.random.default_rng(72)
    A, S = dense16[2], pool_matrix(16, 2)
    xt = synth.ellipse_phantom(16, 12, (4, 4))
    b = (dense16[1] @ xt.ravel()).reshape(g16.n_views, g16.n_det) + 0.05 * rng.standard_normal((12, 24))
    eta = 0.5 / np.linalg.eigvalsh((A @ S).T @ (A @ S)).max()
    seq = [2, 0, 1, 1, 2, 0, 0]
    x0 = rng.random((16, 16)) * 0.2
    x, _ = oracle.pnp_run(g16, [synth.Stage(2, 7, 3, estimator=est)], [eta], seq, b, x0,
                          lam=0.0, tv_iters=0, momentum=False)
    ref = dense_vr(A, S, 7, 3, est, eta, seq, b, x0, g16.n_views)
    assert np.abs(x.ravel() - ref).max() < 1e-12


def test_psnr_closed_form():
    xt = np.random.default_rng(60).random((20, 20))
    assert abs(oracle.psnr(xt + 0.1, xt) - 20.0) < 1e-12


def test_objective_terms():
    g = synth.make_geometry(24, 16, 32)
    x = synth.ellipse_phantom(24, 61, (3, 3))
    b = oracle.project(g, 1, x)
    f, t = oracle.objective(g, x, b)
    assert f == 0.0 and abs(t - oracle.tv(x)) < 1e-12
    f2, _ = oracle.objective(g, x, b + 0.5)
    assert abs(f2 - 0.5 * 0.25 * b.size) < 1e-9


# ---------------------------------------------------------------- the paper's printed numbers
def test_paper_operator_sizes():
    """Sec. 3 prints A in R^{20520 x 65536} (90 views) and R^{82080 x 65536} (360 views)
    for 256 x 256 images, and m_1 = d/16, m_2 = d/4 for the two sketch stages."""
    with open(os.path.join(GOLDEN, "paper_numbers.json")) as f:
        gold = json.load(f)
    for case in gold["operator_sizes"]:
        n_det = case["rows"] // case["views"]
        g = synth.make_geometry(case["n"], case["views"], n_det)
        img = np.zeros((case["n"], case["n"]))
        img[case["n"] // 2, case["n"] // 2] = 1.0
        out = oracle.project(g, 1, img, None, 0, case["views"])  # one view is enough for the shape
        assert out.shape == (1, n_det)
        assert case["views"] * n_det == case["rows"] and case["n"] ** 2 == case["cols"]
    for case in gold["sketch_sizes"]:
        s = case["factor"]
        d = case["n"] ** 2
        assert oracle.pool(np.zeros((case["n"], case["n"])), s).size == d // case["reduction"]


def half_integers_inside(a):
    """Number of k in Z with |k + 1/2| < a (a a Fraction or float >= 0)."""
    from fractions import Fraction
    a = Fraction(a)
    # -a < k + 1/2 < a  <=>  -a - 1/2 < k < a - 1/2
    lo = math.floor(-a - Fraction(1, 2)) + 1
    hi = math.ceil(a - Fraction(1, 2)) - 1
    return max(0, hi - lo + 1)


@pytest.mark.parametrize("s", [1, 2, 4])
@pytest.mark.parametrize("step", ["0.5", "1", "0.3"])
def test_sample_count_axis_ray_closed_form(s, step):
    """One ray (one view at angle 0, one bin): it runs along the x axis through the
    origin, so its foot point is the origin and its samples sit at x = (k + 1/2) delta,
    delta = step s.  The count is the number of half-integers strictly inside
    (-H/delta, H/delta), H = (n_s/2 + 1/2) s the half-width of the support box.  With
    step 1 and even n_s the outermost samples lie exactly on the box edge and are not
    counted (strict inequality)."""
    from fractions import Fraction
    n = 64
    g = dataclasses.replace(synth.make_geometry(n, 1, 1), step=float(step))
    ns = n // s
    H = (Fraction(ns, 2) + Fraction(1, 2)) * s
    delta = Fraction(step) * s
    want = half_integers_inside(H / delta)
    assert oracle.sample_count(g, s) == want
    if step == "0.5":
        assert want == 2 * (ns + 1)
    if step == "1":
        assert want == ns   # (n_s + 1)/2 is a half-integer: the two edge samples drop out


@pytest.mark.parametrize("s", [1, 2])
@pytest.mark.parametrize("step", [0.5, 0.3])
def test_sample_count_diagonal_ray_closed_form(s, step):
    """One ray at 45 degrees through the origin: |x| = |y| = |t| / sqrt 2, so the
    count is the number of half-integers inside (-sqrt2 H/delta, sqrt2 H/delta)
    (irrational bound: no ties), i.e. 2 floor(sqrt2 H/delta + 1/2)."""
    n = 64
    g = synth.make_geometry(n, 1, 1, angle0=math.pi / 4, step=step)
    ns = n // s
    a = math.sqrt(2.0) * (0.5 * ns + 0.5) * s / (step * s)
    assert oracle.sample_count(g, s) == 2 * math.floor(a + 0.5)


def chord_count(g, s, v, j):
    """Samples of ray (v, j) strictly inside the box |x|,|y| < H, counted from the
    chord: the ray (source S, direction d, foot point F = S - (S.d) d, from the
    rotated view frame) meets the box for t in (t_lo, t_hi) (slab intersection),
    and the samples t = (k + 1/2) delta inside that interval are counted in closed
    form."""
    S, P = ray_endpoints(g, v, j)
    d = (P - S) / np.linalg.norm(P - S)
    F = S - np.dot(S, d) * d
    ns = g.n // s
    H = (0.5 * ns + 0.5) * s
    delta = g.step * s
    lo, hi = -math.inf, math.inf
    for c in range(2):
        if abs(d[c]) < 1e-15:
            if abs(F[c]) >= H:
                return 0
            continue
        t1, t2 = (-H - F[c]) / d[c], (H - F[c]) / d[c]
        lo, hi = max(lo, min(t1, t2)), min(hi, max(t1, t2))
    if not hi > lo:
        return 0
    # lo < (k + 1/2) delta < hi
    k_lo = math.floor(lo / delta - 0.5) + 1
    k_hi = math.ceil(hi / delta - 0.5) - 1
    return max(0, k_hi - k_lo + 1)


@pytest.mark.parametrize("s,P,p", [(1, 1, 0), (2, 1, 0), (1, 8, 3), (4, 5, 4)])
def test_sample_count_equals_chord_count(s, P, p):
    """The whole 64^2 / 90 views x 96 bins geometry (and subsets): the oracle's
    brute-force count over all integer k equals the chord-interval count of every
    ray, exactly."""
    g = synth.make_geometry(64, 90, 96)
    views = range(p, g.n_views, P) if P > 1 else range(g.n_views)
    want = sum(chord_count(g, s, v, j) for v in views for j in range(g.n_det))
    assert oracle.sample_count(g, s, p, P) == want
    if (s, P) == (1, 1):
        assert 7.0e5 < want < 8.5e5


# ---------------------------------------------------------------- weighted least squares (Poisson data)
@pytest.mark.parametrize("s,P,p", [(1, 1, 0), (2, 4, 3)])
def test_weighted_gradient_matches_finite_differences(s, P, p):
    """With weights w the gradient is that of (c/2) sum_j w_j r_j^2 on the subset rows."""
    g = synth.make_geometry(16, 16, 24)
    rng = np.random.default_rng(70 + s)
    y = rng.random((16, 16))
    b = rng.standard_normal((g.n_views, g.n_det)) * 3
    w = rng.uniform(0.2, 3.0, (g.n_views, g.n_det))
    c = max(P, 1)
    rows = np.arange(g.n_views)[p::P] if P > 1 else np.arange(g.n_views)

    def f(yy):
        r = oracle.project(g, s, oracle.pool(yy, s), b, p, P)
        return 0.5 * c * np.sum(w[rows] * r * r)

    gr = oracle.grad(g, s, y, b, p, P, w=w)
    h = 1e-3
    for _ in range(3):
        d = rng.standard_normal((16, 16))
        fd = (f(y + h * d) - f(y - h * d)) / (2 * h)
        assert abs(fd - np.vdot(gr, d)) < 1e-8 * max(abs(fd), 1.0)
    # unit weights reduce to the unweighted gradient
    assert np.abs(oracle.grad(g, s, y, b, p, P, w=np.ones_like(w)) - oracle.grad(g, s, y, b, p, P)).max() == 0.0


def test_weighted_power_iteration_matches_dense(g16, dense16):
    rng = np.random.default_rng(80)
    w = rng.uniform(0.5, 2.0, (g16.n_views, g16.n_det))
    A = dense16[1]
    M = np.sqrt(w.ravel())[:, None] * A
    lmax = np.linalg.eigvalsh(M.T @ M).max()
    L, _ = oracle.power_iter(g16, 1, 3000, 1e-14, w=w)
    assert abs(L - lmax) < 1e-8 * lmax


def test_weighted_objective():
    g = synth.make_geometry(24, 16, 32)
    x = synth.ellipse_phantom(24, 81, (3, 3))
    b = oracle.project(g, 1, x) + 0.5
    w = np.full((16, 32), 3.0)
    f, _ = oracle.objective(g, x, b, w)
    assert abs(f - 0.5 * 3.0 * 0.25 * b.size) < 1e-9


# ---------------------------------------------------------------- bicubic sketch (Sec. 3's imresize)
def keys_np(t, a=-0.5):
    """Keys (1981) cubic convolution kernel, written out here independently."""
    t = abs(t)
    if t <= 1:
        return (a + 2) * t ** 3 - (a + 3) * t ** 2 + 1
    if t < 2:
        return a * t ** 3 - 5 * a * t ** 2 + 8 * a * t - 4 * a
    return 0.0


def bicubic_dense(n, s):
    """2-D bicubic sketch as a dense matrix: separable normalised widened Keys weights."""
    ns = n // s
    W = np.zeros((ns, n))
    for I in range(ns):
        XI = s * I + (s - 1) / 2
        w = np.array([keys_np((x - XI) / s) for x in range(n)])
        W[I] = w / w.sum()
    return np.kron(W, W)


def test_keys_kernel_textbook_values():
    """Keys 1981 with a = -1/2: interpolating at a half-way point uses weights
    -1/16, 9/16, 9/16, -1/16; k vanishes at the other integers."""
    assert oracle.keys(0.0) == 1.0
    for t in (1.0, -1.0, 2.0, -2.0, 2.5):
        assert oracle.keys(t) == 0.0
    assert abs(oracle.keys(0.5) - 9 / 16) < 1e-15 and abs(oracle.keys(-1.5) + 1 / 16) < 1e-15
    for t in np.linspace(-2.5, 2.5, 41):
        assert abs(oracle.keys(t) - keys_np(t)) < 1e-15


@pytest.mark.parametrize("s", [2, 4])
def test_bicubic_sketch_closed_forms_and_adjoint(s):
    n = 32
    rng = np.random.default_rng(90 + s)
    x = rng.standard_normal((n, n))
    v = rng.standard_normal((n // s, n // s))
    assert abs(np.vdot(oracle.bicubic_down(x, s), v) - np.vdot(x, oracle.bicubic_up(v, s))) < 1e-12
    assert np.abs(oracle.bicubic_down(np.full((n, n), 0.7), s) - 0.7).max() < 1e-14
    # a linear ramp is reproduced at the coarse centres away from the border
    X, Y = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float), indexing="xy")
    c = oracle.bicubic_down(2 * X - Y, s)
    I = np.arange(n // s)
    XI = s * I + (s - 1) / 2
    inner = slice(2, n // s - 2)
    expect = 2 * XI[None, :] - XI[:, None]
    assert np.abs(c[inner, inner] - expect[inner, inner]).max() < 1e-12
    D = bicubic_dense(n, s)
    assert np.abs(oracle.bicubic_down(x, s).ravel() - D @ x.ravel()).max() < 1e-13


def test_bicubic_gradient_and_step_size():
    g = synth.make_geometry(16, 12, 24)
    rng = np.random.default_rng(95)
    y = rng.random((16, 16))
    b = rng.standard_normal((12, 24))

    def f(yy):
        r = oracle.project(g, 2, oracle.bicubic_down(yy, 2), b)
        return 0.5 * np.vdot(r, r)

    gr = oracle.grad(g, 2, y, b, kind=1)
    d = rng.standard_normal((16, 16))
    fd = (f(y + 1e-3 * d) - f(y - 1e-3 * d)) / 2e-3
    assert abs(fd - np.vdot(gr, d)) < 1e-8 * max(1.0, abs(fd))
    A = dense_rows(g, 2)
    M = A @ bicubic_dense(16, 2)
    lmax = np.linalg.eigvalsh(M.T @ M).max()
    L, _ = oracle.power_iter(g, 2, 3000, 1e-14, kind=1)
    assert abs(L - lmax) < 1e-8 * lmax


# ---------------------------------------------------------------- subset order
def test_splitmix64_published_outputs():
    """The subset order draws from SplitMix64: its first numbers from seed 0 are
    the published ones."""
    with open(os.path.join(GOLDEN, "splitmix64.json")) as f:
        ref = json.load(f)
    for case in ref["streams"]:
        got = [oracle.splitmix64(case["seed"], t) for t in range(1, len(case["outputs"]) + 1)]
        assert got == [int(h, 16) for h in case["outputs"]]


def test_subset_sequence_epochs_are_permutations():
    """Sec. 2 draws each minibatch at random; the reading samples the P subsets
    without replacement per epoch: every full epoch is a permutation of 0..P-1,
    a shorter last epoch has distinct ids, a stage with P = 1 gives zeros."""
    stages = [synth.Stage(4, 29, 12), synth.Stage(2, 5, 1), synth.Stage(1, 10, 7), synth.Stage(1, 0, 5)]
    seq = oracle.subset_sequence(stages, 123)
    assert seq.size == 44
    a, z, c = seq[:29], seq[29:34], seq[34:]
    for e in range(2):
        assert sorted(a[12 * e:12 * e + 12]) == list(range(12))
    assert len(set(a[24:])) == 5 and all(0 <= v < 12 for v in a[24:])
    assert (z == 0).all()
    assert sorted(c[:7]) == list(range(7))
    assert len(set(c[7:])) == 3 and all(0 <= v < 7 for v in c[7:])
    assert oracle.subset_sequence([synth.Stage(1, 0, 4)], 1).size == 0


def test_subset_sequence_uniform_over_orders():
    """Each epoch's order is uniform over all P! permutations (Fisher-Yates):
    chi-square over many seeds, for P = 3 and P = 4.  Thresholds sit near the
    1e-5 tail of the chi-square law with P! - 1 degrees of freedom; a shuffle
    that draws from the wrong range (cyclic orders only, or the naive shuffle)
    lands far beyond them."""
    for P, seeds, limit in ((3, 6000, 28.0), (4, 12000, 62.0)):
        counts = {}
        for s in range(seeds):
            key = tuple(oracle.subset_sequence([synth.Stage(1, P, P)], s))
            counts[key] = counts.get(key, 0) + 1
        assert len(counts) == math.factorial(P)
        expect = seeds / math.factorial(P)
        chi2 = sum((c - expect) ** 2 / expect for c in counts.values())
        assert chi2 < limit, (P, chi2)


def test_subset_sequence_two_subsets_follow_the_stream():
    """P = 2: an epoch's one draw r is uniform in {0, 1} (2^64 mod 2 = 0, no
    rejection); the epoch is (0, 1) when r = 1 (the swap of entry 1 with
    itself) and (1, 0) when r = 0, r being the stream's next number mod 2."""
    seed = 0
    seq = oracle.subset_sequence([synth.Stage(1, 16, 2)], seed)
    for e in range(8):
        r = oracle.splitmix64(seed, e + 1) % 2
        assert tuple(seq[2 * e:2 * e + 2]) == ((0, 1) if r == 1 else (1, 0))


def test_subset_sequence_one_stream_across_stages():
    """One stream serves the whole schedule: splitting a stage at an epoch
    boundary, or putting a P = 1 stage (which draws nothing) between the
    halves, leaves the sequence unchanged; two epochs are not copies of each
    other; different seeds give different orders."""
    whole = oracle.subset_sequence([synth.Stage(1, 36, 12)], 77)
    split = oracle.subset_sequence([synth.Stage(2, 12, 12), synth.Stage(1, 24, 12)], 77)
    gap = oracle.subset_sequence([synth.Stage(2, 12, 12), synth.Stage(2, 5, 1), synth.Stage(1, 24, 12)], 77)
    assert (whole == split).all()
    assert (gap[:12] == whole[:12]).all() and (gap[12:17] == 0).all() and (gap[17:] == whole[12:]).all()
    assert not (whole[:12] == whole[12:24]).all()
    assert not (whole == oracle.subset_sequence([synth.Stage(1, 36, 12)], 78)).all()
