"""Pins of the oracle's discrete adjoint: transposition identity, finite
differences, and the finite-termination special case (K = N gives the adjoint
of the serial fine solve, i.e. F applied N times since F is symmetric)."""
import numpy as np
import pytest

from oracle import heat
from oracle.adjoint import adjoint_sync, face_grad, loss_and_forward


def prob2d(var=True, N=4, f_steps=5, n=(6, 5), seed=0, K=None):
    rng = np.random.default_rng(seed)
    h = tuple(1.0 / (m + 1) for m in n)
    shape = tuple(reversed(n))
    kap = np.exp(0.4 * rng.standard_normal(tuple(s + 2 for s in shape))) if var else None
    kmax = 1.0 if kap is None else kap.max()
    dt = 0.8 * min(h) ** 2 / (4 * kmax)
    return dict(dim=2, n=n, h=h, N=N, f_steps=f_steps, dt=dt, f_scheme="explicit",
                g_solver="cg", g_rtol=1e-14, g_maxit=5000, kappa=kap,
                u0=rng.standard_normal(shape), tol=0.0)


def test_face_grad_is_derivative_of_bilinear_form():
    rng = np.random.default_rng(1)
    p = prob2d()
    shape = tuple(reversed(p["n"]))
    a, u = rng.standard_normal(shape), rng.standard_normal(shape)
    g = face_grad(a, u, p["h"], p["kappa"].shape)
    d = rng.standard_normal(p["kappa"].shape)
    eps = 1e-6
    f = lambda k: np.sum(a * heat.apply_A(u, p["h"], k))
    fd = (f(p["kappa"] + eps * d) - f(p["kappa"] - eps * d)) / (2 * eps)
    assert np.isclose(np.sum(g * d), fd, rtol=1e-8)


@pytest.mark.parametrize("K", [1, 2, 4])
def test_u0_adjoint_transposition_identity(K):
    """u0 -> lambda_N^K is linear: <J v, y> = <v, J^T y>."""
    p = prob2d(seed=2)
    rng = np.random.default_rng(3)
    shape = tuple(reversed(p["n"]))
    v, y = rng.standard_normal(shape), rng.standard_normal(shape)
    _, Jv = loss_and_forward(p, K, np.zeros(shape), u0=v)
    gu0, _, _ = adjoint_sync(p, y, K, u0=v)
    lhs, rhs = float(Jv @ y.reshape(-1)), float(np.sum(v * gu0))
    assert abs(lhs - rhs) <= 1e-11 * max(abs(lhs), 1.0)


def test_kappa_and_u0_gradients_match_central_differences():
    p = prob2d(seed=4, N=3, f_steps=4)
    K = 2
    rng = np.random.default_rng(5)
    shape = tuple(reversed(p["n"]))
    u_obs = rng.standard_normal(shape)
    L0, lamN = loss_and_forward(p, K, u_obs)
    gu0, gk, lamN2 = adjoint_sync(p, lamN - u_obs.reshape(-1), K)
    # same map; the CG start differs (warm vs cold), so agree to the solve accuracy
    np.testing.assert_allclose(lamN2.reshape(-1), lamN, rtol=0, atol=1e-12 * np.max(np.abs(lamN)))
    for trial in range(3):
        d = rng.standard_normal(p["kappa"].shape)
        eps = 1e-6 * np.max(np.abs(p["kappa"]))
        Lp, _ = loss_and_forward(dict(p, kappa=p["kappa"] + eps * d), K, u_obs)
        Lm, _ = loss_and_forward(dict(p, kappa=p["kappa"] - eps * d), K, u_obs)
        fd = (Lp - Lm) / (2 * eps)
        assert np.isclose(np.sum(gk * d), fd, rtol=1e-6, atol=1e-12), (trial, np.sum(gk * d), fd)
        du = rng.standard_normal(shape)
        Lp, _ = loss_and_forward(p, K, u_obs, u0=p["u0"] + 1e-6 * du)
        Lm, _ = loss_and_forward(p, K, u_obs, u0=p["u0"] - 1e-6 * du)
        assert np.isclose(np.sum(gu0 * du), (Lp - Lm) / 2e-6, rtol=1e-6)


def test_K_equal_N_is_adjoint_of_serial_fine():
    """After N iterations Parareal is the serial fine map F^N (§3.2), so dL/du0 = F^N g."""
    p = prob2d(seed=6, N=3, f_steps=4)
    rng = np.random.default_rng(7)
    shape = tuple(reversed(p["n"]))
    g = rng.standard_normal(shape)
    gu0, _, _ = adjoint_sync(p, g, p["N"])
    P = heat.Propagators(p)
    ref = g
    for _ in range(p["N"]):
        ref = P.F(ref)
    np.testing.assert_allclose(gu0, ref, rtol=1e-10, atol=1e-12 * np.max(np.abs(ref)))


def test_constant_kappa_has_no_kappa_gradient():
    p = prob2d(var=False, seed=8)
    gu0, gk, _ = adjoint_sync(p, np.ones(tuple(reversed(p["n"]))), 2)
    assert gk is None and np.all(np.isfinite(gu0))


# ------------------------------------------ adjoint of a logged asynchronous run
def sync_schedule(N, K):
    """The synchronous schedule as an event log (each iteration reads the new
    predecessor for G and the old one for F; slice 1 always reads u0)."""
    return [(i, k, 0 if i == 1 else k - 1, 0 if i == 1 else k)
            for k in range(1, K + 1) for i in range(1, N + 1)]


def test_async_adjoint_of_sync_schedule_equals_sync_adjoint():
    """On the synchronous schedule the logged run is the K-iteration Parareal map
    (Eq. (11); the frozen prefix of Algorithm 1 is the same function), so both adjoints
    give the same gradients."""
    from oracle.adjoint import adjoint_async
    p = prob2d(seed=11, N=4, f_steps=4)
    K = 3
    rng = np.random.default_rng(12)
    g = rng.standard_normal(tuple(reversed(p["n"])))
    gu_s, gk_s, lam_s = adjoint_sync(p, g, K)
    gu_a, gk_a, lam_a = adjoint_async(p, sync_schedule(p["N"], K), g)
    np.testing.assert_allclose(lam_a, lam_s, rtol=0, atol=1e-12 * np.max(np.abs(lam_s)))
    np.testing.assert_allclose(gu_a, gu_s, rtol=0, atol=1e-10 * np.max(np.abs(gu_s)))
    np.testing.assert_allclose(gk_a, gk_s, rtol=0, atol=1e-10 * np.max(np.abs(gk_s)))


def test_async_adjoint_transposition_identity_random_schedule():
    """For a fixed log, u0 -> lambda_N is linear: <J v, y> = <v, J^T y>."""
    from oracle.adjoint import adjoint_async
    from oracle.parareal import async_replay
    from .test_oracle_pins import random_schedule
    p = prob2d(seed=13, N=5, f_steps=3)
    events = random_schedule(p["N"], np.random.default_rng(14), until_quiescent=False, max_events=23)
    rng = np.random.default_rng(15)
    shape = tuple(reversed(p["n"]))
    v, y = rng.standard_normal(shape), rng.standard_normal(shape)
    Jv = async_replay(p, events, u0=v).lam[-1]
    gu0, _, _ = adjoint_async(p, events, y, u0=v)
    lhs, rhs = float(Jv @ y.reshape(-1)), float(np.sum(v * gu0))
    assert abs(lhs - rhs) <= 1e-11 * max(abs(lhs), 1.0)


def test_async_adjoint_matches_central_differences():
    from oracle.adjoint import adjoint_async
    from oracle.parareal import async_replay
    from .test_oracle_pins import random_schedule
    p = prob2d(seed=16, N=4, f_steps=3)
    events = random_schedule(p["N"], np.random.default_rng(17), until_quiescent=False, max_events=15)
    rng = np.random.default_rng(18)
    shape = tuple(reversed(p["n"]))
    u_obs = rng.standard_normal(shape).reshape(-1)

    def loss(kap=None, u0=None):
        q = dict(p, kappa=p["kappa"] if kap is None else kap)
        r = async_replay(q, events, u0=u0).lam[-1] - u_obs
        return 0.5 * float(r @ r), r

    _, r = loss()
    gu0, gk, _ = adjoint_async(p, events, r)
    for trial in range(3):
        d = rng.standard_normal(p["kappa"].shape)
        eps = 1e-6 * np.max(np.abs(p["kappa"]))
        fd = (loss(kap=p["kappa"] + eps * d)[0] - loss(kap=p["kappa"] - eps * d)[0]) / (2 * eps)
        assert np.isclose(np.sum(gk * d), fd, rtol=1e-6, atol=1e-12), (trial, np.sum(gk * d), fd)
        du = rng.standard_normal(shape)
        fd = (loss(u0=p["u0"] + 1e-6 * du)[0] - loss(u0=p["u0"] - 1e-6 * du)[0]) / 2e-6
        assert np.isclose(np.sum(gu0 * du), fd, rtol=1e-6)


def test_async_adjoint_at_quiescence_is_adjoint_of_serial_fine():
    """A quiescent log's result is F^N u0 (Proposition 1), so dL/du0 = F^N g."""
    from oracle.adjoint import adjoint_async
    from .test_oracle_pins import random_schedule
    p = prob2d(seed=19, N=4, f_steps=3)
    events = random_schedule(p["N"], np.random.default_rng(20))
    g = np.random.default_rng(21).standard_normal(tuple(reversed(p["n"])))
    gu0, _, _ = adjoint_async(p, events, g)
    P = heat.Propagators(p)
    ref = g
    for _ in range(p["N"]):
        ref = P.F(ref)
    np.testing.assert_allclose(gu0, ref, rtol=0, atol=1e-10 * np.max(np.abs(ref)))


# ------------------------------------------- 1D implicit fine steps, Thomas coarse solve
def prob1d(var=True, N=4, f_steps=5, n=(13,), seed=0):
    rng = np.random.default_rng(seed)
    h = (1.0 / (n[0] + 1),)
    kap = np.exp(0.4 * rng.standard_normal(n[0] + 2)) if var else None
    return dict(dim=1, n=n, h=h, N=N, f_steps=f_steps, dt=2.0 * h[0] ** 2, f_scheme="implicit",
                g_solver="thomas", g_rtol=0.0, kappa=kap, u0=rng.standard_normal(n), tol=0.0)


def test_implicit_1d_adjoint_transposition_and_differences():
    """Tridiagonal solves run backward: <J v, y> = <v, J^T y> for u0, and central
    differences for kappa and u0."""
    p = prob1d(seed=31)
    K = 2
    rng = np.random.default_rng(32)
    v, y = rng.standard_normal(p["n"]), rng.standard_normal(p["n"])
    _, Jv = loss_and_forward(p, K, np.zeros(p["n"]), u0=v)
    gu0, _, _ = adjoint_sync(p, y, K, u0=v)
    lhs, rhs = float(Jv @ y), float(np.sum(v * gu0))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)
    u_obs = rng.standard_normal(p["n"])
    L0, lamN = loss_and_forward(p, K, u_obs)
    gu0, gk, _ = adjoint_sync(p, lamN - u_obs, K)
    for trial in range(3):
        d = rng.standard_normal(p["kappa"].shape)
        eps = 1e-6 * np.max(np.abs(p["kappa"]))
        Lp, _ = loss_and_forward(dict(p, kappa=p["kappa"] + eps * d), K, u_obs)
        Lm, _ = loss_and_forward(dict(p, kappa=p["kappa"] - eps * d), K, u_obs)
        assert np.isclose(np.sum(gk * d), (Lp - Lm) / (2 * eps), rtol=1e-6, atol=1e-12), trial
        du = rng.standard_normal(p["n"])
        Lp, _ = loss_and_forward(p, K, u_obs, u0=p["u0"] + 1e-6 * du)
        Lm, _ = loss_and_forward(p, K, u_obs, u0=p["u0"] - 1e-6 * du)
        assert np.isclose(np.sum(gu0 * du), (Lp - Lm) / 2e-6, rtol=1e-6)
