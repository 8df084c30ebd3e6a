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

import paper_2110_10762_gb300 as pr  # noqa: E402  (a missing library fails the first call loudly)

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


def test_autograd_function_1d_implicit_thomas():
    """ParaRealFn with 1D implicit fine steps and the Thomas coarse step."""
    from paper_2110_10762_gb300.autograd import ParaRealFn
    p = preset("heat1d_thomas", "small")
    rng = np.random.default_rng(72)
    p["kappa"] = np.exp(0.3 * rng.standard_normal(p["n"][0] + 2))
    K = 2
    spec = dict(dim=1, n=p["n"], T=p["N"] * p["f_steps"] * p["dt"], N=p["N"],
                f_steps=p["f_steps"], K=K, f_scheme="implicit", g_solver="thomas")
    u0 = dev(p["u0"]).requires_grad_(True)
    kap = dev(p["kappa"]).requires_grad_(True)
    out = ParaRealFn.apply(u0, kap, spec)
    (0.5 * (out ** 2).sum()).backward()
    ref_u0, ref_k, lamN = adjoint_sync(dict(p, tol=0.0), host(out), K)
    assert rel_l2(host(out), lamN) < 1e-12
    assert rel_l2(host(u0.grad), ref_u0) < 1e-12
    assert rel_l2(host(kap.grad), ref_k) < 1e-11


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


# ------------------------------------------- adjoint of a logged asynchronous run
def as_events(tuples):
    out = []
    for (i, k, vF, vG) in tuples:
        e = pr.pr_event()
        e.slice, e.version, e.vF, e.vG = i, k, vF, vG
        out.append(e)
    return out


def random_log(N, seed, max_events):
    """A valid asynchronous schedule (same rule as the oracle's replay tests)."""
    rng = np.random.default_rng(seed)
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


def gpu_adjoint_async(p, events, g):
    with Ctx(p) as c:
        gu0 = torch().empty(c.M, dtype=torch().float64, device="cuda")
        gk = (torch().empty(p["kappa"].size, dtype=torch().float64, device="cuda")
              if p.get("kappa") is not None else None)
        lamN = torch().empty(c.M, dtype=torch().float64, device="cuda")
        # any order of the log is accepted
        evs = as_events(events)[::-1]
        pr.parareal_adjoint_async(c.ctx, evs, dev(g), gu0, gk, lamN)
        return host(gu0), (host(gk) if gk is not None else None), host(lamN)


@pytest.mark.parametrize("name,seed", [("heat2d_inverse", 41), ("heat3d_varkappa_async", 42),
                                       ("heat2d_explicit", 43)])
def test_async_adjoint_matches_oracle_random_log(name, seed):
    from oracle.adjoint import adjoint_async
    p = small(name)
    events = random_log(p["N"], seed, max_events=3 * p["N"])
    g = np.random.default_rng(seed + 1).standard_normal(tuple(reversed(p["n"])))
    ref_u0, ref_k, ref_lam = adjoint_async(p, events, g)
    gu0, gk, lamN = gpu_adjoint_async(p, events, g)
    assert rel_l2(lamN, ref_lam) < 1e-12
    assert rel_l2(gu0, ref_u0) < ADJ_TOL
    if ref_k is not None:
        assert rel_l2(gk, ref_k) < ADJ_TOL


def test_async_adjoint_with_more_updates_per_slice_than_slices():
    """A log in which every slice publishes many more versions than there are slices:
    the batched fine propagations and adjoints of one slice's updates are split into
    batches of at most N states (the context's workspaces hold N)."""
    from oracle.adjoint import adjoint_async
    p = small("heat2d_inverse")
    p["N"] = 3
    events = random_log(p["N"], 46, max_events=40)
    per_slice = max(sum(1 for e in events if e[0] == i) for i in range(1, 4))
    assert per_slice > p["N"]
    g = np.random.default_rng(47).standard_normal(tuple(reversed(p["n"])))
    ref_u0, ref_k, ref_lam = adjoint_async(p, events, g)
    gu0, gk, lamN = gpu_adjoint_async(p, events, g)
    assert rel_l2(lamN, ref_lam) < 1e-12
    assert rel_l2(gu0, ref_u0) < ADJ_TOL
    assert rel_l2(gk, ref_k) < ADJ_TOL


def test_async_adjoint_of_sync_schedule_equals_sync_adjoint():
    """The synchronous schedule written as a log: both GPU adjoints agree."""
    p = small("heat2d_inverse")
    K = 3
    events = [(i, k, 0 if i == 1 else k - 1, 0 if i == 1 else k)
              for k in range(1, K + 1) for i in range(1, p["N"] + 1)]
    g = np.random.default_rng(44).standard_normal(tuple(reversed(p["n"])))
    gu_s, gk_s = gpu_adjoint(p, g, K)
    gu_a, gk_a, _ = gpu_adjoint_async(p, events, g)
    assert rel_l2(gu_a, gu_s) < ADJ_TOL
    assert rel_l2(gk_a, gk_s) < ADJ_TOL


def test_async_adjoint_of_a_kernel_log():
    """The log of a real persistent-kernel run: the replayed lambda_N matches the run's,
    and the gradients match the oracle's adjoint of the same log."""
    from oracle.adjoint import adjoint_async
    p = small("heat2d_inverse", tol=1e-9)
    with Ctx(p) as c:
        lam = c.lam()
        code, st, log = pr.parareal_run_async(c.ctx, pr.make_async_opts(timeout_s=60.0), lam,
                                              log_cap=100000)
        run_lamN = host(lam)[p["N"] * c.M:]
    assert code == pr.PR_OK
    events = [(e.slice, e.version, e.vF, e.vG) for e in log]
    g = np.random.default_rng(45).standard_normal(tuple(reversed(p["n"])))
    gu0, gk, lamN = gpu_adjoint_async(p, events, g)
    assert rel_l2(lamN, run_lamN) < 1e-11
    ref_u0, ref_k, _ = adjoint_async(p, events, g)
    assert rel_l2(gu0, ref_u0) < ADJ_TOL
    assert rel_l2(gk, ref_k) < ADJ_TOL


def test_async_adjoint_rejects_invalid_logs():
    p = small("heat2d_inverse")
    g = dev(np.zeros(tuple(reversed(p["n"]))))
    bad = [
        [(1, 2, 0, 0)],                      # versions must start at 1
        [(2, 1, 0, 1)],                      # predecessor version 1 never produced
        [(1, 1, 0, 0), (2, 1, 0, 1), (2, 2, 0, 1)],  # fine input is not the previous coarse input
        [(1, 1, 0, 0), (1, 1, 0, 0)],        # duplicate
    ]
    with Ctx(p) as c:
        gu0 = torch().empty(c.M, dtype=torch().float64, device="cuda")
        for evs in bad:
            with pytest.raises(pr.PararealError) as e:
                pr.parareal_adjoint_async(c.ctx, as_events(evs), g, gu0)
            assert e.value.code == pr.PR_EINVAL


@pytest.mark.parametrize("K", [1, 3])
def test_adjoint_1d_implicit_thomas(K):
    """Tridiagonal solves run backward: 1D implicit fine steps and the Thomas coarse
    step, variable kappa, against the oracle's adjoint."""
    p = preset("heat1d_thomas", "small")
    rng = np.random.default_rng(71)
    p["kappa"] = np.exp(0.4 * rng.standard_normal(p["n"][0] + 2))
    p["tol"] = 0.0
    g = rng.standard_normal(tuple(reversed(p["n"])))
    ref_u0, ref_k, _ = adjoint_sync(p, g, K)
    got_u0, got_k = gpu_adjoint(p, g, K)
    assert rel_l2(got_u0, ref_u0) < 1e-12
    assert rel_l2(got_k, ref_k) < 1e-11
