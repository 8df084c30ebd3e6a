"""Chebyshev-preconditioned coarse CG (option PR_OPT_G_CHEBYSHEV) against the
oracle's PCG with the same preconditioner degree: the FP32 Chebyshev steps on
the GPU perturb z at the 1e-7 level only, so the iteration counts agree within
a few and both solutions meet the FP64 residual bound ||r|| <= rtol ||b||
(I + dT A >= I bounds their distance by 2 rtol ||b||)."""
import numpy as np
import pytest

from oracle import heat
from oracle.parareal import sync_parareal
from synthetic import preset

from .gpu_util import Ctx, dev, host, problem_struct, rel_l2, torch

import paper_2110_10762_gb300 as pr  # noqa: E402  (a missing library fails the first call loudly)

pytestmark = pytest.mark.gpu


def case(name, **over):
    sizes = {k: over.pop(k) for k in ("n", "N", "f_steps") if k in over}
    p = preset(name, "small", **sizes)
    p.update(dict(g_rtol=1e-13, f_prec=64))
    p.update(over)
    return p


@pytest.mark.parametrize("name", ["heat2d_explicit", "heat2d_inverse", "heat3d_mixed",
                                  "heat3d_varkappa_async"])
@pytest.mark.parametrize("m", [2, 8])
def test_pcg_coarse_solve(name, m):
    p = case(name, g_cheb=m)
    rng = np.random.default_rng(61)
    shape = tuple(reversed(p["n"]))
    b = rng.standard_normal(shape)
    x0 = b + 0.1 * rng.standard_normal(shape)
    P = heat.Propagators(p)
    ref, ref_it = P.G(b, x0=x0)
    _, plain_it = heat.Propagators(dict(p, g_cheb=0)).G(b, x0=x0)
    with Ctx(p) as c:
        pr.parareal_set_option(c.ctx, pr.PR_OPT_G_CHEBYSHEV, m)
        out = torch().empty(c.M, dtype=torch().float64, device="cuda")
        it = pr.parareal_coarse(c.ctx, dev(b), dev(x0), out)
        got = host(out).reshape(shape)
    assert abs(it - ref_it) <= 2, (it, ref_it)
    assert rel_l2(got, ref) < 1e-12
    r = b - (got + P.dT * heat.apply_A(got, P.h, P.kappa))
    assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(b)
    if m == 8:
        assert it < plain_it


@pytest.mark.parametrize("n", [(132, 61), (4, 9), (256, 37), (136, 30, 19), (8, 5, 3),
                               (128, 16, 17)])
@pytest.mark.parametrize("m", [2, 3, 12])
def test_pcg_vectorised_steps(n, m):
    """Constant kappa with nx % 4 == 0 takes the vectorised three-term Chebyshev
    steps (128 x per warp, streamed slowest axis): ragged x chunks (a chunk with
    one or two active lanes), ragged plane runs, single-lane rows, m = 2 (the first
    step is also the last) and m = 3 (first and last distinct)."""
    name = "heat2d_explicit" if len(n) == 2 else "heat3d_mixed"
    p = case(name, g_cheb=m, n=n)
    rng = np.random.default_rng(64)
    shape = tuple(reversed(n))
    b = rng.standard_normal(shape)
    x0 = b + 0.1 * rng.standard_normal(shape)
    P = heat.Propagators(p)
    ref, ref_it = P.G(b, x0=x0)
    with Ctx(p) as c:
        pr.parareal_set_option(c.ctx, pr.PR_OPT_G_CHEBYSHEV, m)
        out = torch().empty(c.M, dtype=torch().float64, device="cuda")
        it = pr.parareal_coarse(c.ctx, dev(b), dev(x0), out)
        got = host(out).reshape(shape)
    assert abs(it - ref_it) <= 2, (it, ref_it)
    assert rel_l2(got, ref) < 1e-12
    r = b - (got + P.dT * heat.apply_A(got, P.h, P.kappa))
    assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(b)


def test_pcg_vectorised_sync_parareal_parity():
    n = (132, 61)
    p = case("heat2d_explicit", tol=1e-9, g_cheb=8, n=n)
    ref = sync_parareal(p)
    with Ctx(p) as c:
        pr.parareal_set_option(c.ctx, pr.PR_OPT_G_CHEBYSHEV, 8)
        lam = c.lam()
        code, st = pr.parareal_run_sync(c.ctx, lam)
        got = host(lam).reshape(ref.lam.shape)
    assert code == pr.PR_OK and st.iterations == ref.k
    assert rel_l2(got, ref.lam) < 1e-11


def test_pcg_sync_parareal_parity():
    p = case("heat2d_explicit", tol=1e-9, g_cheb=6)
    ref = sync_parareal(p)
    with Ctx(p) as c:
        pr.parareal_set_option(c.ctx, pr.PR_OPT_G_CHEBYSHEV, 6)
        lam = c.lam()
        code, st = pr.parareal_run_sync(c.ctx, lam)
        got = host(lam).reshape(ref.lam.shape)
    assert code == pr.PR_OK and st.iterations == ref.k
    assert rel_l2(got, ref.lam) < 1e-11


def test_pcg_option_before_problem_and_validation():
    p = case("heat2d_inverse", g_cheb=4)
    ctx = pr.parareal_create(0, torch().cuda.current_stream())
    try:
        for bad in (1, 65, -1):
            with pytest.raises(pr.PararealError) as e:
                pr.parareal_set_option(ctx, pr.PR_OPT_G_CHEBYSHEV, bad)
            assert e.value.code == pr.PR_EINVAL
        pr.parareal_set_option(ctx, pr.PR_OPT_G_CHEBYSHEV, 4)   # before the problem
        u0, kap = dev(p["u0"]), dev(p["kappa"])
        pr.parareal_set_problem(ctx, problem_struct(p, u0, kap))
        rng = np.random.default_rng(62)
        b = rng.standard_normal(tuple(reversed(p["n"])))
        out = torch().empty(b.size, dtype=torch().float64, device="cuda")
        it = pr.parareal_coarse(ctx, dev(b), None, out)
        ref, ref_it = heat.Propagators(p).G(b)
        assert abs(it - ref_it) <= 2 and rel_l2(host(out), ref) < 1e-12
        pr.parareal_set_option(ctx, pr.PR_OPT_G_CHEBYSHEV, 0)    # back to plain CG
        it0 = pr.parareal_coarse(ctx, dev(b), None, out)
        _, plain_it = heat.Propagators(dict(p, g_cheb=0)).G(b)
        assert abs(it0 - plain_it) <= 2
    finally:
        pr.parareal_destroy(ctx)


def test_pcg_adjoint_matches_oracle():
    from oracle.adjoint import adjoint_sync
    p = case("heat2d_inverse", tol=0.0)
    K = 2
    g = np.random.default_rng(63).standard_normal(tuple(reversed(p["n"])))
    ref_u0, ref_k, _ = adjoint_sync(p, g, K)
    with Ctx(p) as c:
        pr.parareal_set_option(c.ctx, pr.PR_OPT_G_CHEBYSHEV, 8)
        gu0 = torch().empty(c.M, dtype=torch().float64, device="cuda")
        gk = torch().empty(p["kappa"].size, dtype=torch().float64, device="cuda")
        pr.parareal_adjoint(c.ctx, dev(g), K, gu0, gk)
        got_u0, got_k = host(gu0), host(gk)
    assert rel_l2(got_u0, ref_u0) < 1e-10
    assert rel_l2(got_k, ref_k) < 1e-10
