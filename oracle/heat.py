"""Discrete heat operator and one-slice propagators, FP64, plain numpy.

Problem (§3.1, Eq. (8)-(9)): u_t = div(kappa grad u) on the unit interval,
square or cube, zero Dirichlet boundary (h(u,s,t) = 0 on the boundary).
Space: uniform grid, interior sizes n per axis, h_a = 1/(n_a+1), finite
volumes in flux form

    (A u)_p = sum_axes h_a^-2 sum_{faces f=(p,q)} kappa_f (u_p - u_q),
    kappa_f = (kappa_p + kappa_q) / 2,   u_q = 0 outside the grid,

with kappa given at every node including the boundary ring (kappa = None
means kappa = 1, the standard 3/5/7-point negative Laplacian).

One slice [T_{i-1}, T_i] is propagated by (§3.1, definitions of F and G;
§5.1, backward Euler and the time steps dT, dt):
  * explicit Euler:  u <- u - dt A u              (fine, n_f steps)
  * implicit Euler:  (I + dt A) u_new = u         (fine in 1D, coarse always)
    solved by the Thomas algorithm (1D, exact) or by conjugate gradients
    (2D/3D) stopped when ||r||_2 <= rtol ||b||_2.
  * trapezoidal rule (Crank-Nicolson), the fine scheme of Table 1:
      (I + dt/2 A) u_new = (I - dt/2 A) u          (fine, n_f steps)
    with the right-hand side formed as u - (dt/2) A u, solved by Thomas (1D)
    or by the same CG (2D/3D) started from the current state u.

Arrays use the layout of ``synthetic.generators``: interior states have
numpy shape (nx,), (ny, nx) or (nz, ny, nx); kappa has n+2 per axis.
"""
from __future__ import annotations

import numpy as np


def _h_of_axis(h, ndim: int, ax: int) -> float:
    # numpy axis 0 is the slowest grid axis (z in 3D, y in 2D); h is (hx, hy, hz)
    return h[ndim - 1 - ax]


def apply_A(u: np.ndarray, h, kappa: np.ndarray | None = None) -> np.ndarray:
    """A_kappa u in flux form (definition above), zero Dirichlet boundary."""
    d = u.ndim
    U = np.pad(u, 1)  # zero boundary ring
    out = np.zeros_like(u)
    for ax in range(d):
        # restrict every other axis to interior indices
        inner = [slice(1, -1)] * d
        inner[ax] = slice(None)
        Ua = U[tuple(inner)]
        hi = [slice(None)] * d
        lo = [slice(None)] * d
        hi[ax] = slice(1, None)
        lo[ax] = slice(None, -1)
        diff = Ua[tuple(hi)] - Ua[tuple(lo)]        # u_{j+1} - u_j on the n+1 faces
        if kappa is None:
            kf = 1.0
        else:
            Ka = kappa[tuple(inner)]
            kf = 0.5 * (Ka[tuple(hi)] + Ka[tuple(lo)])  # face diffusivity
        flux = kf * diff
        # -(flux_{p+1/2} - flux_{p-1/2}) / h^2 at the interior nodes
        out -= (flux[tuple(hi)] - flux[tuple(lo)]) / _h_of_axis(h, d, ax) ** 2
    return out


def explicit_euler(u: np.ndarray, dt: float, h, kappa=None, steps: int = 1) -> np.ndarray:
    """`steps` explicit Euler steps u <- u - dt A u (fine propagator F, §5.1)."""
    u = np.array(u, dtype=np.float64, copy=True)
    for _ in range(steps):
        u = u - dt * apply_A(u, h, kappa)
    return u


def tridiagonal_1d(n: int, dt: float, h, kappa=None):
    """Bands (sub, diag, sup) of I + dt A in 1D (length n each; sub[0], sup[-1] unused)."""
    hx = h[0]
    if kappa is None:
        kf = np.ones(n + 1)
    else:
        kf = 0.5 * (kappa[1:] + kappa[:-1])          # n+1 faces
    r = dt / hx ** 2
    diag = 1.0 + r * (kf[:-1] + kf[1:])
    sub = np.zeros(n)
    sup = np.zeros(n)
    sub[1:] = -r * kf[1:-1]
    sup[:-1] = -r * kf[1:-1]
    return sub, diag, sup


def thomas(sub, diag, sup, rhs: np.ndarray) -> np.ndarray:
    """Thomas algorithm (Gaussian elimination without pivoting) on the last axis.

    rhs may carry leading batch axes; the bands are shared by the batch.
    """
    n = diag.shape[0]
    rhs = np.array(rhs, dtype=np.float64, copy=True)
    c = np.zeros(n)
    d = np.zeros_like(rhs)
    c[0] = sup[0] / diag[0]
    d[..., 0] = rhs[..., 0] / diag[0]
    for m in range(1, n):
        denom = diag[m] - sub[m] * c[m - 1]
        c[m] = sup[m] / denom
        d[..., m] = (rhs[..., m] - sub[m] * d[..., m - 1]) / denom
    x = np.zeros_like(rhs)
    x[..., n - 1] = d[..., n - 1]
    for m in range(n - 2, -1, -1):
        x[..., m] = d[..., m] - c[m] * x[..., m + 1]
    return x


def solve_tridiagonal(sub, diag, sup, rhs: np.ndarray, apply_matrix) -> np.ndarray:
    """x = Mat^-1 rhs for one tridiagonal system (1D, last axis): the Thomas
    algorithm followed by one step of iterative refinement,
        x <- x + Thomas(rhs - Mat x),
    with the residual formed in FP64 by `apply_matrix` (the operator's own
    definition).  Thomas alone accumulates its rounding along the whole chain
    of n rows: on a weakly diagonally dominant system (I + r T with r >> 1) it
    loses about 50 ulps per solve at n = 1023, which 100 steps of F turn into
    5e-13.  One refinement step brings each solve to the accuracy its FP64
    residual allows (a few ulps; the sine-mode closed form pins it)."""
    x = thomas(sub, diag, sup, rhs)
    return x + thomas(sub, diag, sup, rhs - apply_matrix(x))


def implicit_euler_1d(u: np.ndarray, dt: float, h, kappa=None, steps: int = 1) -> np.ndarray:
    """`steps` backward-Euler steps in 1D: (I + dt A) x = u by a direct
    tridiagonal solve (§5.1, LU solve; Thomas with one refinement step)."""
    n = u.shape[-1]
    sub, diag, sup = tridiagonal_1d(n, dt, h, kappa)
    mat = lambda v: v + dt * apply_A(v, h, kappa)
    x = np.array(u, dtype=np.float64, copy=True)
    for _ in range(steps):
        x = solve_tridiagonal(sub, diag, sup, x, mat)
    return x


def crank_nicolson_1d(u: np.ndarray, dt: float, h, kappa=None, steps: int = 1) -> np.ndarray:
    """`steps` trapezoidal-rule steps in 1D (§5.1, Table 1's F): the right-hand
    side (I - dt/2 A) u, then (I + dt/2 A) x = rhs by the tridiagonal solve."""
    n = u.shape[-1]
    sub, diag, sup = tridiagonal_1d(n, 0.5 * dt, h, kappa)
    mat = lambda v: v + (0.5 * dt) * apply_A(v, h, kappa)
    x = np.array(u, dtype=np.float64, copy=True)
    for _ in range(steps):
        rhs = x - (0.5 * dt) * apply_A(x, h, kappa)
        x = solve_tridiagonal(sub, diag, sup, rhs, mat)
    return x


def crank_nicolson_cg(u: np.ndarray, dt: float, h, kappa=None, steps: int = 1,
                      rtol: float = 1e-12, maxit: int = 10000):
    """`steps` trapezoidal-rule steps in 2D/3D; each solve (I + dt/2 A) x = rhs by
    the CG below, started from the current state.  Returns (u, total CG iterations)."""
    x = np.array(u, dtype=np.float64, copy=True)
    total = 0
    for _ in range(steps):
        rhs = x - (0.5 * dt) * apply_A(x, h, kappa)
        x, it = cg_implicit_euler(rhs, 0.5 * dt, h, kappa, x, rtol, maxit)
        total += it
    return x, total


def cg_implicit_euler(b: np.ndarray, dt: float, h, kappa=None, x0=None,
                      rtol: float = 1e-10, maxit: int = 10000):
    """One backward-Euler step (I + dt A) x = b by textbook conjugate gradients.

    Hestenes-Stiefel CG from x0 (x0 = b when None); stops as soon as the
    recursively updated residual satisfies ||r||_2 <= rtol ||b||_2, when the
    residual is exactly zero, or after maxit iterations.  Returns (x, iters).
    """
    b = np.asarray(b, dtype=np.float64)
    x = np.array(b if x0 is None else x0, dtype=np.float64, copy=True)

    def op(v):
        return v + dt * apply_A(v, h, kappa)

    bnorm = np.sqrt(np.sum(b * b))
    r = b - op(x)
    rr = np.sum(r * r)
    it = 0
    if np.sqrt(rr) <= rtol * bnorm or rr == 0.0:
        return x, it
    p = r.copy()
    while it < maxit:
        q = op(p)
        alpha = rr / np.sum(p * q)
        x = x + alpha * p
        r = r - alpha * q
        rr_new = np.sum(r * r)
        it += 1
        if np.sqrt(rr_new) <= rtol * bnorm or rr_new == 0.0:
            break
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
    return x, it


def cg1_implicit_euler(b: np.ndarray, dt: float, h, kappa=None, x0=None,
                       rtol: float = 1e-10, maxit: int = 10000):
    """One backward-Euler step (I + dt A) x = b by single-reduction conjugate
    gradients (Chronopoulos and Gear, 1989): the same Krylov iterates as the
    textbook CG above in exact arithmetic, with both inner products of an
    iteration taken together on the residual,

        r_0 = b - B x_0,  w_0 = B r_0,  gamma_0 = (r_0, r_0),  delta_0 = (w_0, r_0),
        alpha_0 = gamma_0 / delta_0,  beta_0 = 0,  p_{-1} = s_{-1} = 0,
        p_i = r_i + beta_i p_{i-1},      s_i = w_i + beta_i s_{i-1}   (s_i = B p_i)
        x_{i+1} = x_i + alpha_i p_i,     r_{i+1} = r_i - alpha_i s_i
        w_{i+1} = B r_{i+1},  gamma_{i+1} = (r_{i+1}, r_{i+1}),  delta_{i+1} = (w_{i+1}, r_{i+1})
        beta_{i+1} = gamma_{i+1} / gamma_i
        alpha_{i+1} = gamma_{i+1} / (delta_{i+1} - beta_{i+1} gamma_{i+1} / alpha_i)

    (B = I + dt A).  Same start and stopping rule as cg_implicit_euler: x0 = b
    when None; stop as soon as ||r_i||_2 <= rtol ||b||_2 (sqrt(gamma_i)), when
    gamma_i == 0, or after maxit iterations.  Returns (x, iters)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.array(b if x0 is None else x0, dtype=np.float64, copy=True)

    def op(v):
        return v + dt * apply_A(v, h, kappa)

    bnorm = np.sqrt(np.sum(b * b))
    r = b - op(x)
    gamma = np.sum(r * r)
    it = 0
    if np.sqrt(gamma) <= rtol * bnorm or gamma == 0.0:
        return x, it
    w = op(r)
    delta = np.sum(w * r)
    alpha = gamma / delta
    beta = 0.0
    p = np.zeros_like(x)
    s = np.zeros_like(x)
    while it < maxit:
        p = r + beta * p
        s = w + beta * s
        x = x + alpha * p
        r = r - alpha * s
        it += 1
        gamma_new = np.sum(r * r)
        if np.sqrt(gamma_new) <= rtol * bnorm or gamma_new == 0.0:
            break
        w = op(r)
        delta = np.sum(w * r)
        beta = gamma_new / gamma
        alpha = gamma_new / (delta - beta * gamma_new / alpha)
        gamma = gamma_new
    return x, it


def coarse_spectrum_bounds(n, h, dt: float, kappa=None):
    """Interval [a, b] holding the spectrum of I + dt A.

    The eigenvalues of the constant-coefficient A_1 are sums over axes of
    4/h^2 sin^2(j pi h / 2), j = 1..n (discrete sine modes), so for kappa = 1
    the bounds are exact.  For variable kappa the Rayleigh quotient
    <u, A u> = sum_faces kappa_f (Du)_f^2 / h^2 lies between kappa_min and
    kappa_max (over faces) times that of A_1; the upper bound is also capped by
    the largest Gershgorin row bound 1 + 2 dt sum_faces kappa_f / h^2.
    """
    lo1 = sum(4.0 / hh ** 2 * np.sin(np.pi * hh / 2) ** 2 for hh in h)
    hi1 = sum(4.0 / hh ** 2 * np.sin(m * np.pi * hh / 2) ** 2 for m, hh in zip(n, h))
    if kappa is None:
        return 1.0 + dt * lo1, 1.0 + dt * hi1
    d = len(n)
    rows = np.zeros(tuple(reversed(n)))
    kmin, kmax = np.inf, -np.inf
    for ax in range(d):
        inner = [slice(1, -1)] * d
        inner[ax] = slice(None)
        K = kappa[tuple(inner)]
        hi_ = [slice(None)] * d
        lo_ = [slice(None)] * d
        hi_[ax] = slice(1, None)
        lo_[ax] = slice(None, -1)
        kf = 0.5 * (K[tuple(hi_)] + K[tuple(lo_)])        # n+1 faces along ax
        kmin, kmax = min(kmin, float(kf.min())), max(kmax, float(kf.max()))
        a = [slice(None)] * d
        b = [slice(None)] * d
        a[ax] = slice(None, -1)
        b[ax] = slice(1, None)
        rows = rows + (kf[tuple(a)] + kf[tuple(b)]) / _h_of_axis(h, d, ax) ** 2
    gersh = 1.0 + 2.0 * dt * float(rows.max())
    return 1.0 + dt * kmin * lo1, min(gersh, 1.0 + dt * kmax * hi1)


def chebyshev_apply(op, f: np.ndarray, m: int, a: float, b: float) -> np.ndarray:
    """m steps of Chebyshev iteration for op(y) = f from y = 0 on the interval
    [a, b] (three-term recurrence of Chebyshev acceleration): a fixed
    polynomial p_m(B) f with residual polynomial T_m((c - x)/e) / T_m(c/e),
    c = (a+b)/2, e = (b-a)/2, used as the preconditioner z = p_m(B) r."""
    c, e = 0.5 * (b + a), 0.5 * (b - a)
    sigma = c / e
    rho = 1.0 / sigma
    res = np.array(f, dtype=np.float64, copy=True)
    d = res / c
    y = d.copy()
    for _ in range(1, m):
        res = res - op(d)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = (rho_new * rho) * d + (2.0 * rho_new / e) * res
        y = y + d
        rho = rho_new
    return y


def pcg_implicit_euler(b: np.ndarray, dt: float, h, kappa=None, x0=None, rtol: float = 1e-10,
                       maxit: int = 10000, m: int = 8, bounds=None):
    """(I + dt A) x = b by preconditioned conjugate gradients with the degree-m
    Chebyshev polynomial preconditioner above (spectrum bounds from
    coarse_spectrum_bounds unless given).  Same start and stopping rule as
    cg_implicit_euler.  Returns (x, iters)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.array(b if x0 is None else x0, dtype=np.float64, copy=True)
    n = tuple(reversed(b.shape))

    def op(v):
        return v + dt * apply_A(v, h, kappa)

    lo, hi = bounds if bounds is not None else coarse_spectrum_bounds(n, h, dt, kappa)
    bnorm = np.sqrt(np.sum(b * b))
    r = b - op(x)
    rr = np.sum(r * r)
    it = 0
    if np.sqrt(rr) <= rtol * bnorm or rr == 0.0:
        return x, it
    z = chebyshev_apply(op, r, m, lo, hi)
    rz = np.sum(r * z)
    p = z.copy()
    while it < maxit:
        q = op(p)
        alpha = rz / np.sum(p * q)
        x = x + alpha * p
        r = r - alpha * q
        rr = np.sum(r * r)
        it += 1
        if np.sqrt(rr) <= rtol * bnorm or rr == 0.0:
            break
        z = chebyshev_apply(op, r, m, lo, hi)
        rz_new = np.sum(r * z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it


class Propagators:
    """F and G of one problem (§3.1): F accurate, G cheap, both over one slice.

    prob keys: dim, n, h, dt (fine step), f_steps, f_scheme ('explicit',
    'implicit' (1D) or 'cn', the trapezoidal rule), f_rtol/f_maxit (CG of the
    trapezoidal steps in 2D/3D), g_solver ('thomas' or 'cg'), g_steps
    (default 1), g_rtol, g_maxit, g_cheb (0: plain CG; m >= 2: CG preconditioned
    by m Chebyshev steps), g_cg ('textbook', default, or 'single': the
    single-reduction recurrence of cg1_implicit_euler), kappa.  The coarse step
    is dT = f_steps * dt.
    """

    def __init__(self, prob: dict, kappa="from_prob"):
        self.dim = prob["dim"]
        self.n = tuple(prob["n"])
        self.h = tuple(prob["h"])
        self.dt = float(prob["dt"])
        self.f_steps = int(prob["f_steps"])
        self.f_scheme = prob.get("f_scheme", "explicit")
        self.g_solver = prob.get("g_solver", "cg" if self.dim > 1 else "thomas")
        self.g_steps = int(prob.get("g_steps", 1))
        self.g_rtol = float(prob.get("g_rtol", 1e-10))
        self.g_maxit = int(prob.get("g_maxit", 20000))
        self.g_cheb = int(prob.get("g_cheb") or 0)
        self.g_cg = prob.get("g_cg") or "textbook"
        if self.g_cg not in ("textbook", "single"):
            raise ValueError("g_cg must be 'textbook' or 'single'")
        self.f_rtol = float(prob.get("f_rtol") or 1e-12)
        self.f_maxit = int(prob.get("f_maxit") or 10000)
        self.kappa = prob.get("kappa") if isinstance(kappa, str) else kappa
        self.dT = self.f_steps * self.dt
        self.shape = tuple(reversed(self.n))
        if self.g_solver == "cg" and self.g_steps != 1:
            raise ValueError("CG coarse propagator takes one implicit step")

    def F(self, x: np.ndarray) -> np.ndarray:
        x = np.asarray(x, dtype=np.float64).reshape(self.shape)
        if self.f_scheme == "explicit":
            return explicit_euler(x, self.dt, self.h, self.kappa, self.f_steps)
        if self.f_scheme == "cn":
            if self.dim == 1:
                return crank_nicolson_1d(x, self.dt, self.h, self.kappa, self.f_steps)
            return crank_nicolson_cg(x, self.dt, self.h, self.kappa, self.f_steps,
                                     self.f_rtol, self.f_maxit)[0]
        if self.dim != 1:
            raise ValueError("implicit fine propagator is 1D (Thomas) only")
        return implicit_euler_1d(x, self.dt, self.h, self.kappa, self.f_steps)

    def G(self, x: np.ndarray, x0=None):
        """Returns (G(x), cg_iterations); x0 is the CG starting guess."""
        x = np.asarray(x, dtype=np.float64).reshape(self.shape)
        dTg = self.dT / self.g_steps
        if self.g_solver == "thomas":
            if self.dim != 1:
                raise ValueError("Thomas coarse propagator is 1D only")
            return implicit_euler_1d(x, dTg, self.h, self.kappa, self.g_steps), 0
        x0 = None if x0 is None else np.asarray(x0, dtype=np.float64).reshape(self.shape)
        if self.g_cheb:
            return pcg_implicit_euler(x, dTg, self.h, self.kappa, x0, self.g_rtol, self.g_maxit,
                                      self.g_cheb)
        if self.g_cg == "single":
            return cg1_implicit_euler(x, dTg, self.h, self.kappa, x0, self.g_rtol, self.g_maxit)
        return cg_implicit_euler(x, dTg, self.h, self.kappa, x0, self.g_rtol, self.g_maxit)
