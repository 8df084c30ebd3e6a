"""GPU discrete adjoint (parareal_adjoint / ParaRealFn) against the oracle's
adjoint, central finite differences and the transposition identity.

Tolerances: 1e-10 relative L2 against the oracle adjoint (the coarse solves
are CG to rtol 1e-13 on both sides, which bounds agreement below 1e-12);
1e-6 relative for central differences.
"""
import numpy as np
import pytest

from oracle.adjoint import adjoint_sync
from synthetic import preset, random_directions

from .gpu_util import Ctx, dev, host, rel_l2, torch

pr = pytest.importorskip("paper_2110_10762_gb300")

pytestmark = pytest.mark.gpu

ADJ_TOL = 1e-10


def small(name="heat2d_inverse", **over):
    p = preset(name, "small")
    p.update(dict(g_rtol=1e-13, f_prec=64, tol=0.0))
    p.update(over)
    return p


def gpu_adjoint(p, g, K, want_kappa=True):
    with Ctx(p) as c:
        gu0 = torch().empty(c.M, dtype=torch().float64, device="cuda")
        gk = None
        if want_kappa and p.get("kappa") is not None:
            gk = torch().empty(p["kappa"].size, dtype=torch().float64, device="cuda")
        pr.parareal_adjoint(c.ctx, dev(g), K, gu0, gk)
        return host(gu0), (host(gk) if gk is not None else None)


def gpu_lamN(p, K, u0=None, kappa=None):
    q = dict(p)
    if u0 is not None:
        q["u0"] = u0
    if kappa is not None:
        q["kappa"] = kappa
    q["max_iter"] = K
    q["tol"] = 0.0
    with Ctx(q) as c:
        lam = c.lam()
        pr.parareal_run_sync(c.ctx, lam)
        return host(lam)[p["N"] * c.M:]


@pytest.mark.parametrize("name,K", [("heat2d_inverse", 3), ("heat3d_varkappa_async", 2),
                                    ("heat2d_explicit", 2)])
def test_adjoint_matches_oracle(name, K):
    p = small(name)
    rng = np.random.default_rng(31)
    g = rng.standard_normal(tuple(reversed(p["n"])))
    ref_u0, ref_k, _ = adjoint_sync(p, g, K)
    gu0, gk = gpu_adjoint(p, g, K)
    assert rel_l2(gu0, ref_u0) < ADJ_TOL
    if ref_k is not None:
        assert rel_l2(gk, ref_k) < ADJ_TOL


def test_adjoint_transposition_identity_on_gpu():
    p = small()
    K = p["K"]
    rng = np.random.default_rng(32)
    shape = tuple(reversed(p["n"]))
    v, y = rng.standard_normal(shape), rng.standard_normal(shape)
    Jv = gpu_lamN(p, K, u0=v)
    q = dict(p, u0=v)
    gu0, _ = gpu_adjoint(q, y, K, want_kappa=False)
    lhs, rhs = float(Jv @ y.reshape(-1)), float(np.sum(v.reshape(-1) * gu0))
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_full_size_kappa_gradient_by_central_differences():
    """512 x 512, N = 32, n_f = 128, K = 6 (the inverse-problem workload)."""
    p = preset("heat2d_inverse", "full")
    p.update(dict(g_rtol=1e-13, f_prec=64, tol=0.0))
    K = p["K"]
    # u_obs: the serial fine solution with kappa* (GPU serial fine)
    q = dict(p, kappa=p["kappa_star"])
    with Ctx(q) as c:
        lam = c.lam()
        pr.parareal_serial_fine(c.ctx, lam)
        u_obs = host(lam)[p["N"] * c.M:]
    lamN = gpu_lamN(p, K)
    g = lamN - u_obs
    gu0, gk = gpu_adjoint(p, g.reshape(tuple(reversed(p["n"]))), K)
    L = lambda lam_end: 0.5 * float(np.sum((lam_end - u_obs) ** 2))
    dirs = random_directions(p["kappa"].shape, 2, seed=42)
    for d in dirs:
        eps = 1e-6 * float(np.max(np.abs(p["kappa"])))
        Lp = L(gpu_lamN(p, K, kappa=p["kappa"] + eps * d))
        Lm = L(gpu_lamN(p, K, kappa=p["kappa"] - eps * d))
        fd = (Lp - Lm) / (2 * eps)
        assert abs(float(np.sum(gk * d.reshape(-1))) - fd) <= 1e-6 * abs(fd), (np.sum(gk * d.reshape(-1)), fd)
    du = random_directions(tuple(reversed(p["n"])), 1, seed=43)[0]
    Lp = L(gpu_lamN(p, K, u0=p["u0"] + 1e-6 * du))
    Lm = L(gpu_lamN(p, K, u0=p["u0"] - 1e-6 * du))
    fd = (Lp - Lm) / 2e-6
    assert abs(float(np.sum(gu0 * du.reshape(-1))) - fd) <= 1e-6 * abs(fd)


def test_autograd_function_matches_adjoint():
    from paper_2110_10762_gb300.autograd import ParaRealFn
    t = torch()
    p = small()
    K = p["K"]
    spec = dict(dim=p["dim"], n=p["n"], T=p["N"] * p["f_steps"] * p["dt"], N=p["N"],
                f_steps=p["f_steps"], K=K, g_rtol=1e-13)
    u0 = dev(p["u0"]).requires_grad_(True)
    kap = dev(p["kappa"]).requires_grad_(True)
    u_obs = t.zeros_like(u0)
    out = ParaRealFn.apply(u0, kap, spec)
    loss = 0.5 * ((out - u_obs) ** 2).sum()
    loss.backward()
    ref_u0, ref_k, lamN = adjoint_sync(p, (host(out) - 0.0), K)
    assert rel_l2(host(out), lamN) < 1e-12
    assert rel_l2(host(u0.grad), ref_u0) < ADJ_TOL
    assert rel_l2(host(kap.grad), ref_k) < ADJ_TOL


def test_adjoint_rejects_unsupported():
    p = small(f_prec=32)
    with Ctx(p) as c:
        gu0 = torch().empty(c.M, dtype=torch().float64, device="cuda")
        with pytest.raises(pr.PararealError):
            pr.parareal_adjoint(c.ctx, gu0, 1, gu0, None)


def test_adjoint_K0_is_the_predictor_chain():
    """K = 0: lambda_N = G^N u0, so dL/du0 = G^N g (G symmetric)."""
    p = small()
    rng = np.random.default_rng(33)
    g = rng.standard_normal(tuple(reversed(p["n"])))
    ref_u0, ref_k, _ = adjoint_sync(p, g, 0)
    gu0, gk = gpu_adjoint(p, g, 0)
    assert rel_l2(gu0, ref_u0) < ADJ_TOL
    assert rel_l2(gk, ref_k) < ADJ_TOL


def test_adjoint_rejects_bad_K_and_constant_kappa_gradient():
    p = small("heat2d_explicit")
    with Ctx(p) as c:
        gu0 = torch().empty(c.M, dtype=torch().float64, device="cuda")
        with pytest.raises(pr.PararealError):
            pr.parareal_adjoint(c.ctx, gu0, p["N"] + 1, gu0, None)
        with pytest.raises(pr.PararealError):
            pr.parareal_adjoint(c.ctx, gu0, 1, gu0, gu0)   # no kappa to differentiate
