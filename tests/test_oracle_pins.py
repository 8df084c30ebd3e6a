"""Pins of the CPU oracle against facts the paper and the mathematics fix.

None of these compare the oracle with itself: each check is a closed form,
an invariant, a textbook/library special case or brute force on tiny inputs.
"""
import math

import numpy as np
import pytest
import scipy.fft
import scipy.linalg

from oracle import heat
from oracle.parareal import async_replay, serial_fine, sync_parareal
from synthetic import preset


# ----------------------------------------------------------------- helpers
def mode_eigs(n, h):
    """mu_j = (4/h^2) sin^2(j pi h / 2), j = 1..n: eigenvalues of the 1D Dirichlet Laplacian."""
    j = np.arange(1, n + 1)
    return 4.0 / h ** 2 * np.sin(j * np.pi * h / 2) ** 2


def grid_mu(n_xyz, h_xyz):
    """Eigenvalue array of the d-dim Laplacian in numpy (z, y, x) order."""
    mus = [mode_eigs(n, h) for n, h in zip(n_xyz, h_xyz)]
    out = np.zeros(tuple(reversed(n_xyz)))
    d = len(n_xyz)
    for a, mu in enumerate(mus):
        shp = [1] * d
        shp[d - 1 - a] = mu.size
        out = out + mu.reshape(shp)
    return out


def sine_mode(n_xyz, j_xyz, h_xyz):
    d = len(n_xyz)
    out = np.ones(tuple(reversed(n_xyz)))
    for a, (n, j, h) in enumerate(zip(n_xyz, j_xyz, h_xyz)):
        x = np.arange(1, n + 1) * h
        shp = [1] * d
        shp[d - 1 - a] = n
        out = out * np.sin(j * np.pi * x).reshape(shp)
    return out


def dense_of(op, shape):
    m = int(np.prod(shape))
    cols = []
    for c in range(m):
        e = np.zeros(m)
        e[c] = 1.0
        cols.append(np.asarray(op(e.reshape(shape))).reshape(-1))
    return np.array(cols).T


def small_prob(dim, n, N, f_steps, dt_h2=0.2, f_scheme="explicit", g_solver=None,
               g_rtol=1e-14, kappa=None, seed=0):
    h = tuple(1.0 / (m + 1) for m in n)
    rng = np.random.default_rng(seed)
    u0 = rng.standard_normal(tuple(reversed(n)))
    return dict(dim=dim, n=n, h=h, N=N, f_steps=f_steps, dt=dt_h2 * min(h) ** 2,
                f_scheme=f_scheme, g_solver=g_solver or ("thomas" if dim == 1 else "cg"),
                g_rtol=g_rtol, g_maxit=5000, kappa=kappa, u0=u0, tol=0.0)


# ----------------------------------------------------- operator A (flux form)
@pytest.mark.parametrize("n,j", [((9,), (3,)), ((7, 5), (2, 4)), ((4, 5, 3), (1, 3, 2))])
def test_A_sine_modes_are_eigenvectors(n, j):
    h = tuple(1.0 / (m + 1) for m in n)
    u = sine_mode(n, j, h)
    mu = sum(4.0 / hh ** 2 * math.sin(jj * math.pi * hh / 2) ** 2 for jj, hh in zip(j, h))
    np.testing.assert_allclose(heat.apply_A(u, h), mu * u, rtol=1e-12, atol=1e-12 * mu)


def test_A_constant_kappa_scales_laplacian():
    n = (6, 7)
    h = (1 / 7, 1 / 8)
    u = np.random.default_rng(1).standard_normal((7, 6))
    kap = np.full((9, 8), 2.5)
    np.testing.assert_allclose(heat.apply_A(u, h, kap), 2.5 * heat.apply_A(u, h), rtol=1e-13)


def test_A_energy_form_and_symmetry():
    """<A u, u> equals the face-sum energy sum_f h^-2 kappa_f (u_p-u_q)^2 (loops over faces)."""
    rng = np.random.default_rng(2)
    nx, ny = 5, 4
    h = (1 / (nx + 1), 1 / (ny + 1))
    kap = np.exp(rng.standard_normal((ny + 2, nx + 2)))
    u = rng.standard_normal((ny, nx))
    v = rng.standard_normal((ny, nx))
    U = np.pad(u, 1)
    E = 0.0
    for y in range(ny + 2):
        for x in range(nx + 2):
            if x + 1 < nx + 2 and 1 <= y <= ny:          # x-face (x, x+1)
                E += 0.5 * (kap[y, x] + kap[y, x + 1]) * (U[y, x] - U[y, x + 1]) ** 2 / h[0] ** 2
            if y + 1 < ny + 2 and 1 <= x <= nx:          # y-face (y, y+1)
                E += 0.5 * (kap[y, x] + kap[y + 1, x]) * (U[y, x] - U[y + 1, x]) ** 2 / h[1] ** 2
    assert np.isclose(np.sum(heat.apply_A(u, h, kap) * u), E, rtol=1e-12)
    assert np.isclose(np.sum(heat.apply_A(u, h, kap) * v), np.sum(u * heat.apply_A(v, h, kap)), rtol=1e-12)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_A_converges_to_div_kappa_grad(dim):
    """Manufactured solution: A_kappa u -> -div(kappa grad u), error O(h^2)."""
    def fields(n):
        h = 1.0 / (n + 1)
        xi = np.arange(1, n + 1) * h
        xr = np.arange(0, n + 2) * h
        g = np.meshgrid(*([xi] * dim), indexing="ij")[::-1]   # (z,y,x) arrays, g[0] = x
        gr = np.meshgrid(*([xr] * dim), indexing="ij")[::-1]
        # u = prod sin(pi x_a), kappa = 1 + x/2 + y^2 ... (smooth, varies per axis)
        def kap_f(c):
            return 1.0 + 0.5 * c[0] + (0.3 * c[1] ** 2 if dim > 1 else 0) + (0.2 * c[2] if dim > 2 else 0)
        grads = [0.5, None, 0.2]
        u = np.ones_like(g[0])
        for a in range(dim):
            u = u * np.sin(np.pi * g[a])
        k = kap_f(g)
        # -div(kappa grad u) = -sum_a (dk/dx_a du/dx_a + k d2u/dx_a^2)
        res = np.zeros_like(u)
        for a in range(dim):
            du = np.pi * np.cos(np.pi * g[a]) * u / np.sin(np.pi * g[a])
            d2u = -np.pi ** 2 * u
            dk = grads[a] if a != 1 else 0.6 * g[1]
            res -= dk * du + k * d2u
        Ah = heat.apply_A(u, tuple([h] * dim), kap_f(gr))
        return np.max(np.abs(Ah - res))
    e1, e2 = fields(15), fields(31)
    assert e2 < e1 / 3.3   # second order: ratio ~4 when h halves


# ------------------------------------------------------------ propagators
@pytest.mark.parametrize("n,j", [((11,), (2,)), ((6, 7), (3, 1)), ((4, 3, 5), (2, 1, 4))])
def test_explicit_euler_mode_decay(n, j):
    h = tuple(1.0 / (m + 1) for m in n)
    dt = 0.15 * min(h) ** 2
    u = sine_mode(n, j, h)
    mu = sum(4.0 / hh ** 2 * math.sin(jj * math.pi * hh / 2) ** 2 for jj, hh in zip(j, h))
    out = heat.explicit_euler(u, dt, h, None, steps=7)
    np.testing.assert_allclose(out, (1 - dt * mu) ** 7 * u, rtol=1e-11, atol=1e-13)


def test_implicit_1d_mode_decay_and_banded():
    n, h = 31, 1 / 32
    dt = 3e-3
    mu = mode_eigs(n, h)
    u = sine_mode((n,), (5,), (h,))
    out = heat.implicit_euler_1d(u, dt, (h,), None, steps=4)
    np.testing.assert_allclose(out, u / (1 + dt * mu[4]) ** 4, rtol=1e-12, atol=1e-14)
    # variable kappa: the Thomas solution satisfies (I + dt A) x = b with A from the flux form,
    # and agrees with LAPACK's banded solver on the same system
    rng = np.random.default_rng(3)
    kap = np.exp(rng.standard_normal(n + 2))
    b = rng.standard_normal(n)
    x = heat.implicit_euler_1d(b, dt, (h,), kap, steps=1)
    np.testing.assert_allclose(x + dt * heat.apply_A(x, (h,), kap), b, rtol=1e-12, atol=1e-12)
    sub, diag, sup = heat.tridiagonal_1d(n, dt, (h,), kap)
    ab = np.zeros((3, n))
    ab[0, 1:] = sup[:-1]
    ab[1] = diag
    ab[2, :-1] = sub[1:]
    np.testing.assert_allclose(x, scipy.linalg.solve_banded((1, 1), ab, b), rtol=1e-12)


@pytest.mark.parametrize("n,j", [((13,), (4,)), ((6, 5), (2, 3)), ((4, 3, 5), (3, 2, 1))])
def test_crank_nicolson_mode_factor(n, j):
    """Trapezoidal rule on a sine mode: factor (1 - dt mu / 2) / (1 + dt mu / 2) per step,
    in 1D (Thomas) and 2D/3D (CG), at a step far beyond the explicit limit."""
    h = tuple(1.0 / (m + 1) for m in n)
    dt = 3.0 * min(h) ** 2
    u = sine_mode(n, j, h)
    mu = sum(4.0 / hh ** 2 * math.sin(jj * math.pi * hh / 2) ** 2 for jj, hh in zip(j, h))
    fac = ((1 - 0.5 * dt * mu) / (1 + 0.5 * dt * mu)) ** 5
    if len(n) == 1:
        out = heat.crank_nicolson_1d(u, dt, h, None, steps=5)
    else:
        out, it = heat.crank_nicolson_cg(u, dt, h, None, steps=5, rtol=1e-14)
        assert it <= 5 * 2   # an eigenvector is solved in one CG iteration (plus rounding)
    np.testing.assert_allclose(out, fac * u, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("dim", [1, 2])
def test_crank_nicolson_variable_kappa_dense(dim):
    """One trapezoidal step equals (I + dt/2 A)^-1 (I - dt/2 A) u with dense matrices of
    the flux-form operator (variable kappa); two steps are the square."""
    n = (9,) if dim == 1 else (5, 4)
    h = tuple(1.0 / (m + 1) for m in n)
    shape = tuple(reversed(n))
    rng = np.random.default_rng(8)
    kap = np.exp(0.5 * rng.standard_normal(tuple(m + 2 for m in shape)))
    u = rng.standard_normal(shape)
    dt = 2.0 * min(h) ** 2
    A = dense_of(lambda v: heat.apply_A(v, h, kap), shape)
    I = np.eye(A.shape[0])
    S = np.linalg.solve(I + 0.5 * dt * A, I - 0.5 * dt * A)
    if dim == 1:
        one = heat.crank_nicolson_1d(u, dt, h, kap, steps=1)
        two = heat.crank_nicolson_1d(u, dt, h, kap, steps=2)
    else:
        one, _ = heat.crank_nicolson_cg(u, dt, h, kap, steps=1, rtol=1e-15, maxit=500)
        two, _ = heat.crank_nicolson_cg(u, dt, h, kap, steps=2, rtol=1e-15, maxit=500)
    np.testing.assert_allclose(one.reshape(-1), S @ u.reshape(-1), rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(two.reshape(-1), S @ S @ u.reshape(-1), rtol=1e-11, atol=1e-12)


def test_crank_nicolson_is_second_order_in_time():
    """Against the exact decay exp(-mu t) of a mode, the error falls ~4x when dt halves
    (backward Euler would give ~2x): the scheme is the trapezoidal rule."""
    n, h = (31,), (1 / 32,)
    u = sine_mode(n, (3,), h)
    mu = 4.0 / h[0] ** 2 * math.sin(3 * math.pi * h[0] / 2) ** 2
    T = 4e-3
    errs = []
    for steps in (8, 16, 32):
        out = heat.crank_nicolson_1d(u, T / steps, h, None, steps=steps)
        errs.append(np.max(np.abs(out - math.exp(-mu * T) * u)))
    assert 3.6 < errs[0] / errs[1] < 4.4 and 3.6 < errs[1] / errs[2] < 4.4


@pytest.mark.parametrize("dim", [2, 3])
def test_cg_solves_backward_euler(dim):
    n = (5, 4) if dim == 2 else (3, 4, 3)
    h = tuple(1.0 / (m + 1) for m in n)
    shape = tuple(reversed(n))
    rng = np.random.default_rng(4)
    kap = np.exp(0.5 * rng.standard_normal(tuple(m + 2 for m in shape)))
    b = rng.standard_normal(shape)
    dT = 40 * min(h) ** 2
    x, it = heat.cg_implicit_euler(b, dT, h, kap, None, rtol=1e-14, maxit=500)
    D = dense_of(lambda v: v + dT * heat.apply_A(v, h, kap), shape)
    np.testing.assert_allclose(x.reshape(-1), np.linalg.solve(D, b.reshape(-1)), rtol=1e-11, atol=1e-12)
    assert 0 < it <= D.shape[0] + 5       # CG terminates in about M steps in exact arithmetic
    # a mode is solved exactly: G(mode) = mode / (1 + dT mu)
    u = sine_mode(n, (2,) * dim, h)
    mu = sum(4.0 / hh ** 2 * math.sin(2 * math.pi * hh / 2) ** 2 for hh in h)
    xm, _ = heat.cg_implicit_euler(u, dT, h, None, None, rtol=1e-14)
    np.testing.assert_allclose(xm, u / (1 + dT * mu), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("n", [(40, 33), (12, 10, 9)])
def test_cg_matches_the_sine_transform_solution(n):
    """Constant kappa: I + dT A is diagonal in the type-I sine basis (each grid
    axis separately), so the exact backward-Euler step of a random right-hand
    side is DST^-1[DST(b) / (1 + dT mu)] (scipy's FFT-based DST-I, an
    independent route).  The oracle's CG meets it at rtol 1e-14."""
    h = tuple(1.0 / (m + 1) for m in n)
    shape = tuple(reversed(n))
    rng = np.random.default_rng(21)
    b = rng.standard_normal(shape)
    dT = 60 * min(h) ** 2
    mu = grid_mu(n, h)
    exact = scipy.fft.idstn(scipy.fft.dstn(b, type=1) / (1 + dT * mu), type=1)
    x, it = heat.cg_implicit_euler(b, dT, h, None, None, rtol=1e-14, maxit=2000)
    assert np.linalg.norm(x - exact) / np.linalg.norm(exact) < 1e-12
    assert it > 10


@pytest.mark.parametrize("n", [(40, 33), (12, 10, 9)])
def test_single_reduction_cg_matches_the_sine_transform_solution(n):
    """The single-reduction (Chronopoulos-Gear) CG of the coarse step meets the
    exact backward-Euler step DST^-1[DST(b) / (1 + dT mu)] at rtol 1e-14."""
    h = tuple(1.0 / (m + 1) for m in n)
    shape = tuple(reversed(n))
    rng = np.random.default_rng(31)
    b = rng.standard_normal(shape)
    dT = 60 * min(h) ** 2
    mu = grid_mu(n, h)
    exact = scipy.fft.idstn(scipy.fft.dstn(b, type=1) / (1 + dT * mu), type=1)
    x, it = heat.cg1_implicit_euler(b, dT, h, None, None, rtol=1e-14, maxit=2000)
    assert np.linalg.norm(x - exact) / np.linalg.norm(exact) < 1e-12
    assert it > 10


@pytest.mark.parametrize("dim", [2, 3])
def test_single_reduction_cg_dense_solve_and_mode(dim):
    """Variable kappa: the dense solve (LAPACK) of I + dT A; constant kappa: a sine
    mode comes out divided by 1 + dT mu."""
    n = (5, 4) if dim == 2 else (3, 4, 3)
    h = tuple(1.0 / (m + 1) for m in n)
    shape = tuple(reversed(n))
    rng = np.random.default_rng(32)
    kap = np.exp(0.5 * rng.standard_normal(tuple(m + 2 for m in shape)))
    b = rng.standard_normal(shape)
    dT = 40 * min(h) ** 2
    x, it = heat.cg1_implicit_euler(b, dT, h, kap, None, rtol=1e-14, maxit=500)
    D = dense_of(lambda v: v + dT * heat.apply_A(v, h, kap), shape)
    np.testing.assert_allclose(x.reshape(-1), np.linalg.solve(D, b.reshape(-1)), rtol=1e-11,
                               atol=1e-12)
    assert 0 < it <= D.shape[0] + 5
    u = sine_mode(n, (2,) * dim, h)
    mu = sum(4.0 / hh ** 2 * math.sin(2 * math.pi * hh / 2) ** 2 for hh in h)
    xm, _ = heat.cg1_implicit_euler(u, dT, h, None, None, rtol=1e-14)
    np.testing.assert_allclose(xm, u / (1 + dT * mu), rtol=1e-12, atol=1e-14)
    # an eigenvector: one step of the Krylov method is exact (to rounding)
    _, itm = heat.cg1_implicit_euler(u, dT, h, None, None, rtol=1e-10)
    assert itm == 1


def test_single_reduction_cg_has_the_krylov_iterates_of_textbook_cg():
    """In exact arithmetic the single-reduction recurrence produces the iterates
    of Hestenes-Stiefel CG (both minimise the B-norm error over the same Krylov
    space).  Brute force on a small dense system: after j iterations both equal
    the B-norm minimiser over x0 + K_j(B, r0), computed here by a dense
    least-squares solve on an orthonormal Krylov basis (an independent route)."""
    n = (6, 5)
    h = tuple(1.0 / (m + 1) for m in n)
    shape = tuple(reversed(n))
    rng = np.random.default_rng(33)
    kap = np.exp(0.4 * rng.standard_normal(tuple(m + 2 for m in shape)))
    b = rng.standard_normal(shape)
    x0 = rng.standard_normal(shape)
    dT = 30 * min(h) ** 2
    D = dense_of(lambda v: v + dT * heat.apply_A(v, h, kap), shape)
    bb, xx0 = b.reshape(-1), x0.reshape(-1)
    r0 = bb - D @ xx0
    xstar = np.linalg.solve(D, bb)
    L = np.linalg.cholesky(D)
    for j in range(1, 7):
        K = np.stack([np.linalg.matrix_power(D, i) @ r0 for i in range(j)], axis=1)
        Q, _ = np.linalg.qr(K)
        # min over c of ||L^T (x0 + Q c - x*)||_2
        c, *_ = np.linalg.lstsq(L.T @ Q, L.T @ (xstar - xx0), rcond=None)
        xj = xx0 + Q @ c
        x1, it1 = heat.cg1_implicit_euler(b, dT, h, kap, x0, rtol=0.0, maxit=j)
        xt, itt = heat.cg_implicit_euler(b, dT, h, kap, x0, rtol=0.0, maxit=j)
        assert it1 == itt == j
        assert np.linalg.norm(x1.reshape(-1) - xj) / np.linalg.norm(xj) < 1e-9, j
        assert np.linalg.norm(xt.reshape(-1) - xj) / np.linalg.norm(xj) < 1e-9, j


def test_single_reduction_cg_zero_rhs_warm_start_and_stop_rule():
    h = (1 / 6, 1 / 6)
    x, it = heat.cg1_implicit_euler(np.zeros((5, 5)), 0.1, h)
    assert it == 0 and not x.any()
    b = np.random.default_rng(34).standard_normal((5, 5))
    xs, _ = heat.cg1_implicit_euler(b, 0.1, h, rtol=1e-14)
    x2, it2 = heat.cg1_implicit_euler(b, 0.1, h, x0=xs, rtol=1e-10)
    assert it2 == 0
    # the stop rule is on the recursively updated residual against rtol ||b||_2,
    # as for textbook CG: same iteration count on a mid-size grid
    n = (40, 33)
    hh = tuple(1.0 / (m + 1) for m in n)
    bb = np.random.default_rng(35).standard_normal(tuple(reversed(n)))
    for rtol in (1e-4, 1e-7, 1e-10):
        _, i1 = heat.cg1_implicit_euler(bb, 60 * min(hh) ** 2, hh, None, None, rtol, 2000)
        _, i0 = heat.cg_implicit_euler(bb, 60 * min(hh) ** 2, hh, None, None, rtol, 2000)
        assert abs(i1 - i0) <= 1, (rtol, i1, i0)


@pytest.mark.parametrize("m", [2, 5, 8])
def test_chebyshev_preconditioner_on_a_mode(m):
    """On an eigenvector of B = I + dT A with eigenvalue lam, m Chebyshev steps give
    (1 - T_m((c - lam)/e) / T_m(c/e)) / lam times the vector (c, e: centre and half
    width of the bounds)."""
    n, j = (7, 6), (3, 2)
    h = tuple(1.0 / (k + 1) for k in n)
    dT = 30 * min(h) ** 2
    u = sine_mode(n, j, h)
    mu = sum(4.0 / hh ** 2 * math.sin(jj * math.pi * hh / 2) ** 2 for jj, hh in zip(j, h))
    lam = 1 + dT * mu
    a, b = heat.coarse_spectrum_bounds(n, h, dT)
    c, e = (a + b) / 2, (b - a) / 2
    T = lambda k, x: np.cosh(k * np.arccosh(x)) if abs(x) >= 1 else np.cos(k * np.arccos(x))
    fac = (1 - T(m, (c - lam) / e) / T(m, c / e)) / lam
    op = lambda v: v + dT * heat.apply_A(v, h, None)
    np.testing.assert_allclose(heat.chebyshev_apply(op, u, m, a, b), fac * u, rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("m", [2, 3, 4, 12])
def test_three_term_chebyshev_form_equals_the_oracles(m):
    """The three-term form the vectorised GPU steps run,
        y_{k+1} = y_k + c1_k (y_k - y_{k-1}) + c2_k (f - B y_k),  y_0 = 0, y_1 = f / c,
    with c1_k = rho_k rho_{k-1} and c2_k = 2 rho_k / e, is the oracle's two-term
    Chebyshev iteration (the same polynomial p_m(B) f), here in FP64 on a random right-hand
    side of a 3D coarse operator; its first two steps use y_1 = f / c and y_0 = 0 only,
    which is what lets the GPU form y_1 from f instead of storing it."""
    n = (6, 5, 4)
    h = tuple(1.0 / (k + 1) for k in n)
    dT = 9.6 * min(h) ** 2
    op = lambda v: v + dT * heat.apply_A(v, h, None)
    a, b = heat.coarse_spectrum_bounds(n, h, dT)
    c, e = 0.5 * (a + b), 0.5 * (b - a)
    f = np.random.default_rng(210).standard_normal(tuple(reversed(n)))
    sigma = c / e
    rho = 1.0 / sigma
    y_prev, y = np.zeros_like(f), f / c
    for _ in range(1, m):
        rho_n = 1.0 / (2.0 * sigma - rho)
        c1, c2 = rho_n * rho, 2.0 * rho_n / e
        y_prev, y = y, y + c1 * (y - y_prev) + c2 * (f - op(y))
        rho = rho_n
    ref = heat.chebyshev_apply(op, f, m, a, b)
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("var", [False, True])
def test_coarse_spectrum_bounds(var):
    """Constant kappa: the bounds are the extreme eigenvalues; variable kappa: they
    enclose the spectrum (dense eigenvalues)."""
    n = (6, 5)
    h = tuple(1.0 / (k + 1) for k in n)
    shape = tuple(reversed(n))
    rng = np.random.default_rng(22)
    kap = np.exp(0.5 * rng.standard_normal(tuple(k + 2 for k in shape))) if var else None
    dT = 25 * min(h) ** 2
    D = dense_of(lambda v: v + dT * heat.apply_A(v, h, kap), shape)
    ev = np.linalg.eigvalsh(0.5 * (D + D.T))
    a, b = heat.coarse_spectrum_bounds(n, h, dT, kap)
    if var:
        assert a <= ev.min() + 1e-12 and ev.max() <= b + 1e-12
    else:
        np.testing.assert_allclose([a, b], [ev.min(), ev.max()], rtol=1e-12)


@pytest.mark.parametrize("var", [False, True])
def test_pcg_solves_backward_euler(var):
    n = (7, 5)
    h = tuple(1.0 / (k + 1) for k in n)
    shape = tuple(reversed(n))
    rng = np.random.default_rng(23)
    kap = np.exp(0.5 * rng.standard_normal(tuple(k + 2 for k in shape))) if var else None
    b = rng.standard_normal(shape)
    dT = 60 * min(h) ** 2
    D = dense_of(lambda v: v + dT * heat.apply_A(v, h, kap), shape)
    x, it = heat.pcg_implicit_euler(b, dT, h, kap, None, rtol=1e-14, maxit=500, m=6)
    np.testing.assert_allclose(x.reshape(-1), np.linalg.solve(D, b.reshape(-1)), rtol=1e-11, atol=1e-12)
    # on a grid large enough for CG to be far from finite termination, the
    # preconditioner cuts the iteration count
    n = (40, 30)
    h = tuple(1.0 / (k + 1) for k in n)
    shape = tuple(reversed(n))
    kap = np.exp(0.5 * rng.standard_normal(tuple(k + 2 for k in shape))) if var else None
    b = rng.standard_normal(shape)
    dT = 60 * min(h) ** 2
    _, it = heat.pcg_implicit_euler(b, dT, h, kap, None, rtol=1e-10, maxit=500, m=6)
    _, it_cg = heat.cg_implicit_euler(b, dT, h, kap, None, rtol=1e-10, maxit=500)
    assert it < 0.8 * it_cg, (it, it_cg)


def test_cg_zero_rhs_and_warm_start():
    h = (1 / 6, 1 / 6)
    x, it = heat.cg_implicit_euler(np.zeros((5, 5)), 0.1, h)
    assert it == 0 and not x.any()
    b = np.random.default_rng(5).standard_normal((5, 5))
    xs, _ = heat.cg_implicit_euler(b, 0.1, h, rtol=1e-14)
    x2, it2 = heat.cg_implicit_euler(b, 0.1, h, x0=xs, rtol=1e-10)
    assert it2 == 0                      # exact start: converged before the first iteration


# ------------------------------------------- Parareal: per-mode closed form
def scalar_parareal(f, g, lam0, N, k):
    """lambda_n^k = sum_{j=0}^{min(k,n)} C(n,j) (f-g)^j g^(n-j) lambda_0 (Pascal induction on Eq. (11))."""
    out = np.zeros((N + 1,) + np.shape(lam0))
    for n in range(N + 1):
        s = 0.0
        for j in range(0, min(k, n) + 1):
            s = s + math.comb(n, j) * (f - g) ** j * g ** (n - j)
        out[n] = s * lam0
    return out


@pytest.mark.parametrize("case", ["1d_implicit", "2d_explicit", "3d_explicit", "1d_cn", "2d_cn",
                                  "2d_explicit_pcg"])
def test_sync_parareal_matches_closed_form_per_mode(case):
    if case == "1d_implicit":
        prob = small_prob(1, (31,), N=8, f_steps=10, dt_h2=2.0, f_scheme="implicit")
    elif case == "1d_cn":
        prob = small_prob(1, (27,), N=7, f_steps=6, dt_h2=3.0, f_scheme="cn")
    elif case == "2d_cn":
        prob = small_prob(2, (8, 6), N=5, f_steps=4, dt_h2=2.5, f_scheme="cn")
        prob["f_rtol"] = 1e-15
    elif case == "2d_explicit":
        prob = small_prob(2, (9, 7), N=6, f_steps=12)
    elif case == "2d_explicit_pcg":
        prob = small_prob(2, (9, 7), N=6, f_steps=12)
        prob["g_cheb"] = 4
    else:
        prob = small_prob(3, (5, 4, 6), N=5, f_steps=8, dt_h2=0.15)
    n, h, N = prob["n"], prob["h"], prob["N"]
    dt = prob["dt"]
    mu = grid_mu(n, h)
    if prob["f_scheme"] == "explicit":
        f = (1 - dt * mu) ** prob["f_steps"]
    elif prob["f_scheme"] == "cn":
        f = ((1 - 0.5 * dt * mu) / (1 + 0.5 * dt * mu)) ** prob["f_steps"]
    else:
        f = (1 + dt * mu) ** (-prob["f_steps"])
    g = 1.0 / (1 + prob["f_steps"] * dt * mu)
    res = sync_parareal(prob, record=True)
    assert res.k == N
    c0 = scipy.fft.dstn(prob["u0"], type=1)          # coefficients in the sine basis
    for k, lam in enumerate(res.iterates):
        coef = scalar_parareal(f, g, c0, N, k)
        expect = np.array([scipy.fft.idstn(c, type=1).reshape(-1) for c in coef])
        scale = np.max(np.abs(expect))
        np.testing.assert_allclose(lam, expect, rtol=0, atol=1e-12 * scale)


def test_finite_termination_with_inexact_coarse():
    """After N iterations Parareal equals the serial fine solution for any G (§3.2)."""
    prob = small_prob(2, (8, 6), N=5, f_steps=9, g_rtol=1e-3)
    res = sync_parareal(prob)
    ref = serial_fine(prob)
    assert res.k == prob["N"]
    np.testing.assert_allclose(res.lam, ref, rtol=0, atol=1e-13 * np.max(np.abs(ref)))


def test_brute_force_block_richardson_variable_kappa():
    """Dense A, M, b of §3.1: lambda* = A^-1 b and lambda^{k+1} = (I - M^-1 A) lambda^k + M^-1 b."""
    n = (4, 3)
    rng = np.random.default_rng(6)
    kap = np.exp(0.6 * rng.standard_normal((5, 6)))
    prob = small_prob(2, n, N=4, f_steps=5, dt_h2=0.05, kappa=kap)
    shape = tuple(reversed(n))
    M_ = int(np.prod(shape))
    N = prob["N"]
    Ad = dense_of(lambda v: heat.apply_A(v, prob["h"], kap), shape)
    I = np.eye(M_)
    Fm = np.linalg.matrix_power(I - prob["dt"] * Ad, prob["f_steps"])
    Gm = np.linalg.inv(I + prob["f_steps"] * prob["dt"] * Ad)
    Ab = np.eye((N + 1) * M_)
    Mb = np.eye((N + 1) * M_)
    for i in range(1, N + 1):
        Ab[i * M_:(i + 1) * M_, (i - 1) * M_:i * M_] = -Fm
        Mb[i * M_:(i + 1) * M_, (i - 1) * M_:i * M_] = -Gm
    b = np.zeros((N + 1) * M_)
    b[:M_] = prob["u0"].reshape(-1)
    lam_star = np.linalg.solve(Ab, b)
    np.testing.assert_allclose(serial_fine(prob).reshape(-1), lam_star, atol=1e-12)
    res = sync_parareal(prob, record=True)
    lam = np.linalg.solve(Mb, b)
    Minv = np.linalg.inv(Mb)
    for it in res.iterates:
        np.testing.assert_allclose(it.reshape(-1), lam, atol=1e-12)
        lam = lam - Minv @ (Ab @ lam) + Minv @ b


def test_stop_rule_is_strict_and_absolute():
    prob = small_prob(1, (15,), N=6, f_steps=5, dt_h2=1.0, f_scheme="implicit")
    full = sync_parareal(prob, tol=0.0, record=True)
    d = [float(np.max(x)) for x in full.deltas]
    # choose tol equal to an attained increment: strict '<' must not stop there
    j = 2
    res = sync_parareal(prob, tol=d[j])
    expect = next(i + 1 for i, x in enumerate(d) if x < d[j])
    assert res.k == expect
    # frozen prefix: after iteration k, slices 1..k no longer change
    for k in range(1, len(full.iterates)):
        for i in range(1, min(k, prob["N"]) + 1):
            if k >= 2 and i <= k - 1:
                assert np.array_equal(full.iterates[k][i], full.iterates[k - 1][i])


def test_single_slice_and_single_point():
    prob = small_prob(1, (1,), N=1, f_steps=3, dt_h2=0.5, f_scheme="implicit")
    res = sync_parareal(prob)
    np.testing.assert_allclose(res.lam, serial_fine(prob), rtol=1e-15)
    assert res.k == 1


# ---------------------------------------------------- asynchronous replay
def test_replay_of_synchronous_schedule_equals_eq11():
    prob = small_prob(1, (23,), N=6, f_steps=8, dt_h2=1.5, f_scheme="implicit")
    K = 4
    events = []
    for k in range(1, K + 1):
        for i in range(1, prob["N"] + 1):
            vG = 0 if i == 1 else k
            vF = 0 if i == 1 else k - 1
            events.append((i, k, vF, vG))
    rep = async_replay(prob, events)
    res = sync_parareal(prob, tol=0.0, max_iter=K, record=True)
    for k in range(K + 1):
        for i in range(prob["N"] + 1):
            np.testing.assert_allclose(rep.versions[(i, k) if i else (0, 0)], res.iterates[k][i],
                                       rtol=0, atol=1e-13)


def random_schedule(N, rng, until_quiescent=True, max_events=400):
    """A random valid asynchronous schedule: each event reads a predecessor
    version no older than the one it read last time."""
    latest = [0] * (N + 1)
    last_vG = [0] * (N + 1)
    last_vF = [0] * (N + 1)
    events = []
    for _ in range(max_events):
        busy = [i for i in range(1, N + 1)
                if not (last_vF[i] == last_vG[i] == latest[i - 1] and latest[i] > 0)]
        if not busy:
            break
        i = int(rng.choice(busy))
        vF = last_vG[i]
        vG = int(rng.integers(vF, latest[i - 1] + 1))
        latest[i] += 1
        events.append((i, latest[i], vF, vG))
        last_vF[i], last_vG[i] = vF, vG
    return events


def test_replay_random_schedule_quiescence_is_serial_fine():
    """Async finite-time termination (§3.2, Proposition 1): quiescent state = lambda*."""
    prob = small_prob(2, (6, 5), N=5, f_steps=6, g_rtol=1e-6)
    rng = np.random.default_rng(7)
    events = random_schedule(prob["N"], rng)
    rep = async_replay(prob, events)
    ref = serial_fine(prob)
    np.testing.assert_allclose(rep.lam, ref, rtol=0, atol=1e-13 * np.max(np.abs(ref)))


def test_replay_per_event_contraction_per_mode():
    """Theorem 4's per-update bound, mode by mode:
    |e_new| <= (|g| + |f-g|) max(|e(x_G)|, |e(x_F)|), e = error vs lambda*."""
    prob = small_prob(1, (19,), N=6, f_steps=10, dt_h2=1.0, f_scheme="implicit")
    mu = grid_mu(prob["n"], prob["h"])
    f = (1 + prob["dt"] * mu) ** (-prob["f_steps"])
    g = 1.0 / (1 + prob["f_steps"] * prob["dt"] * mu)
    alpha = np.abs(g) + np.abs(f - g)
    events = random_schedule(prob["N"], np.random.default_rng(8))
    rep = async_replay(prob, events)
    ref = serial_fine(prob)
    def err(i, v):
        return np.abs(scipy.fft.dst(rep.versions[(i, v)] - ref[i], type=1))
    scale = np.max(np.abs(scipy.fft.dst(ref, type=1, axis=1)))
    for (i, k, vF, vG) in events:
        lhs = err(i, k)
        rhs = alpha * np.maximum(err(i - 1, vF), err(i - 1, vG))
        assert np.all(lhs <= rhs + 1e-12 * scale)


def test_replay_rejects_inconsistent_logs():
    prob = small_prob(1, (7,), N=3, f_steps=3, dt_h2=1.0, f_scheme="implicit")
    with pytest.raises(ValueError):
        async_replay(prob, [(1, 2, 0, 0)])            # version gap
    with pytest.raises(ValueError):
        async_replay(prob, [(2, 1, 0, 1)])            # reads a version never produced
    with pytest.raises(ValueError):
        async_replay(prob, [(1, 1, 0, 0), (2, 1, 0, 1), (2, 2, 0, 1)])  # vF != previous vG


# -------------------------------------------------------------- presets
@pytest.mark.parametrize("name", ["heat1d_thomas", "heat2d_explicit", "heat3d_mixed",
                                  "heat2d_inverse", "heat3d_varkappa_async"])
def test_presets_are_stable_and_shaped(name):
    p = preset(name, "tiny")
    assert p["u0"].shape == tuple(reversed(p["n"]))
    if p["f_scheme"] == "explicit":
        kmax = 1.0 if p["kappa"] is None else float(p["kappa"].max())
        lam_max_bound = sum(4.0 * kmax / hh ** 2 for hh in p["h"])
        assert p["dt"] * lam_max_bound <= 2.0


def test_coarse_solves_follow_algorithm_1():
    """Algorithm 1 solves G only for i-1 > k; slice k+1 reuses w_i^k and slices i <= k are frozen."""
    prob = small_prob(2, (7, 6), N=5, f_steps=6, g_rtol=1e-8)
    res = sync_parareal(prob, tol=0.0)
    assert np.all(res.predictor_cg > 0)
    for k, cg in enumerate(res.cg_iters):
        for i in range(1, prob["N"] + 1):
            if i - 1 > k:
                assert cg[i - 1] > 0, (k, i)
            else:
                assert cg[i - 1] == 0, (k, i)


def test_tridiagonal_propagators_at_1023_points_match_closed_form():
    """The 1D workload (1023 points, u0 = 8 sine modes): 100 implicit-Euler fine
    steps at r = 65.536, one coarse step at r = 6553.6 and 100 trapezoidal
    steps are exact per mode, (1 + dt mu)^-s and ((1 - dt mu/2)/(1 + dt mu/2))^s.
    The oracle must meet them to a few ulps per solve (relative L2 <= 2e-14),
    well inside the 1e-12 the GPU is held to."""
    p = preset("heat1d_thomas", "full")
    n, h = p["n"][0], p["h"][0]
    x = np.arange(1, n + 1) * h
    modes = np.array([np.sin(j * np.pi * x) for j in range(1, 9)])
    coef = np.linalg.lstsq(modes.T, p["u0"].reshape(-1), rcond=None)[0]
    mu = mode_eigs(n, h)[:8]
    dt, dT = p["dt"], p["dt"] * p["f_steps"]
    cases = [(heat.implicit_euler_1d(p["u0"], dt, (h,), None, p["f_steps"]),
              (1 + dt * mu) ** (-p["f_steps"])),
             (heat.implicit_euler_1d(p["u0"], dT, (h,), None, 1), 1 / (1 + dT * mu)),
             (heat.crank_nicolson_1d(p["u0"], dt, (h,), None, p["f_steps"]),
              ((1 - 0.5 * dt * mu) / (1 + 0.5 * dt * mu)) ** p["f_steps"])]
    for got, fac in cases:
        exact = (coef * fac) @ modes
        assert np.linalg.norm(got - exact) / np.linalg.norm(exact) < 2e-14
