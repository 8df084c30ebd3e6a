"""GPU parity of the fine/coarse propagators, the fused correction and
synchronous Parareal (Algorithm 1) against the FP64 CPU oracle.

Tolerances (relative L2 over the compared arrays):
  FP64 path       1e-12  (different rounding order only)
  mixed FP32 fine 1e-5   (FP32 steps, FP64 coarse/correction/test)
  correction      bit-exact (same operation order in IEEE FP64)
"""
import numpy as np
import pytest

from oracle import heat
from oracle.parareal import serial_fine, sync_parareal
from synthetic import preset

from .gpu_util import Ctx, dev, host, rel_l2, torch

import paper_2110_10762_gb300 as pr  # noqa: E402  (a missing library fails the first call loudly)

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = 1e-5


def small(name, **over):
    p = preset(name, "small")
    p.update(over)
    return p


CASES = {
    "1d_thomas": lambda: small("heat1d_thomas"),
    "1d_explicit": lambda: dict(small("heat1d_thomas"), f_scheme="explicit", g_solver="cg",
                                dt=0.3 / 128 ** 2, g_rtol=1e-13),
    "2d_const": lambda: small("heat2d_explicit", g_rtol=1e-13),
    "2d_var": lambda: small("heat2d_inverse", g_rtol=1e-13),
    "3d_const": lambda: small("heat3d_mixed", f_prec=64, g_rtol=1e-13),
    "3d_var": lambda: small("heat3d_varkappa_async", f_prec=64, g_rtol=1e-13),
}


def oracle_props(p):
    return heat.Propagators(p)


@pytest.mark.parametrize("case", list(CASES))
def test_fine_propagator_batched(case):
    p = CASES[case]()
    rng = np.random.default_rng(11)
    shape = tuple(reversed(p["n"]))
    X = rng.standard_normal((p["N"],) + shape)
    P = oracle_props(p)
    with Ctx(p) as c:
        xin = dev(X)
        out = torch().empty_like(xin)
        pr.parareal_fine(c.ctx, xin, out, p["N"])
        got = host(out).reshape(X.shape)
    for s in range(p["N"]):
        assert rel_l2(got[s], P.F(X[s])) < FP64_TOL, s


@pytest.mark.parametrize("case", ["2d_const", "3d_var"])
def test_fine_propagator_mixed_precision(case):
    p = CASES[case]()
    p["f_prec"] = 32
    rng = np.random.default_rng(12)
    shape = tuple(reversed(p["n"]))
    X = rng.standard_normal((p["N"],) + shape)
    P = oracle_props(p)
    with Ctx(p) as c:
        xin = dev(X)
        out = torch().empty_like(xin)
        pr.parareal_fine(c.ctx, xin, out, p["N"])
        got = host(out).reshape(X.shape)
    for s in range(p["N"]):
        err = rel_l2(got[s], P.F(X[s]))
        assert err < MIXED_TOL, (s, err)
        assert err > 1e-12  # the steps really ran in FP32


@pytest.mark.parametrize("n,var", [((68, 12, 9), False), ((68, 12, 9), True),
                                   ((64, 17, 33), False), ((4, 3, 4), True)])
def test_fine_fp32_vectorized_3d(n, var):
    """FP32 3D steps with 4 x-points per thread (nx % 4 == 0): ragged x/y/z tiles."""
    rng = np.random.default_rng(15)
    h = tuple(1.0 / (m + 1) for m in n)
    shape = tuple(reversed(n))
    kap = np.exp(0.3 * rng.standard_normal(tuple(s + 2 for s in shape))) if var else None
    kmax = 1.0 if kap is None else float(kap.max())
    p = dict(dim=3, n=n, h=h, N=3, f_steps=5, dt=0.8 * min(h) ** 2 / (6 * kmax),
             f_scheme="explicit", g_solver="cg", g_rtol=1e-10, f_prec=32, kappa=kap,
             u0=rng.standard_normal(shape), tol=0.0)
    P = oracle_props(p)
    X = rng.standard_normal((3,) + shape)
    with Ctx(p) as c:
        xin = dev(X)
        out = torch().empty_like(xin)
        pr.parareal_fine(c.ctx, xin, out, 3)
        got = host(out).reshape(X.shape)
    for s in range(3):
        err = rel_l2(got[s], P.F(X[s]))
        assert 1e-12 < err < MIXED_TOL, (s, err)


@pytest.mark.parametrize("n,f_steps", [((68, 19, 70), 3), ((68, 19, 70), 4), ((64, 17, 33), 5),
                                        ((132, 9, 37), 8), ((8, 5, 3), 9), ((64, 16, 32), 6)])
def test_fine_fp32_two_steps_per_pass(n, f_steps):
    """TMA-fed FP32 middle steps two per pass (temporal blocking) against one per
    pass: bitwise identical (the same FMA-ordered step, the first step's values on
    the halo recomputed per tile and set to the Dirichlet zero outside the grid),
    and against the FP64 oracle.  Odd and even middle-step counts (a single step
    finishes an odd count), ragged x/y tiles and z chunks, a grid smaller than one
    tile."""
    rng = np.random.default_rng(19)
    h = tuple(1.0 / (m + 1) for m in n)
    shape = tuple(reversed(n))
    p = dict(dim=3, n=n, h=h, N=3, f_steps=f_steps, dt=0.15 * min(h) ** 2, f_scheme="explicit",
             g_solver="cg", g_rtol=1e-10, f_prec=32, kappa=None, u0=rng.standard_normal(shape),
             tol=0.0)
    P = oracle_props(p)
    X = rng.standard_normal((3,) + shape)
    got = {}
    with Ctx(p) as c:
        xin = dev(X)
        for per_pass in (1, 2):
            pr.parareal_set_option(c.ctx, pr.PR_OPT_F_STEPS_PER_PASS, per_pass)
            out = torch().empty_like(xin)
            pr.parareal_fine(c.ctx, xin, out, 3)
            got[per_pass] = host(out).reshape(X.shape)
        with pytest.raises(pr.PararealError):
            pr.parareal_set_option(c.ctx, pr.PR_OPT_F_STEPS_PER_PASS, 3)
    assert np.array_equal(got[1], got[2])
    for s in range(3):
        err = rel_l2(got[2][s], P.F(X[s]))
        assert 1e-12 < err < MIXED_TOL, (s, err)


@pytest.mark.parametrize("n,f_steps", [((37, 19, 70), 2), ((37, 19, 70), 7), ((64, 8, 33), 4),
                                        ((5, 3, 2), 3), ((33, 9, 97), 6)])
def test_fine_fp32_3d_ragged_chunks_and_step_counts(n, f_steps):
    """FP32 3D constant-kappa F: ragged x/y tiles, several and ragged z chunks, nx % 4 != 0
    (scalar kernel) and == 0 (vector kernel), even and odd step counts, two steps (the
    first reads FP64, the last writes FP64)."""
    rng = np.random.default_rng(16)
    h = tuple(1.0 / (m + 1) for m in n)
    shape = tuple(reversed(n))
    p = dict(dim=3, n=n, h=h, N=3, f_steps=f_steps, dt=0.15 * min(h) ** 2, f_scheme="explicit",
             g_solver="cg", g_rtol=1e-10, f_prec=32, kappa=None, u0=rng.standard_normal(shape),
             tol=0.0)
    P = oracle_props(p)
    X = rng.standard_normal((3,) + shape)
    with Ctx(p) as c:
        xin = dev(X)
        out = torch().empty_like(xin)
        pr.parareal_fine(c.ctx, xin, out, 3)
        got = host(out).reshape(X.shape)
    for s in range(3):
        err = rel_l2(got[s], P.F(X[s]))
        assert 1e-12 < err < MIXED_TOL, (s, err)


@pytest.mark.parametrize("case", list(CASES))
def test_coarse_propagator(case):
    p = CASES[case]()
    rng = np.random.default_rng(13)
    shape = tuple(reversed(p["n"]))
    b = rng.standard_normal(shape)
    x0 = b + 0.1 * rng.standard_normal(shape)
    P = oracle_props(p)
    ref, ref_it = P.G(b, x0=x0)
    with Ctx(p) as c:
        out = torch().empty(c.M, dtype=torch().float64, device="cuda")
        it = pr.parareal_coarse(c.ctx, dev(b), dev(x0), out)
        got = host(out)
    assert rel_l2(got, ref) < FP64_TOL
    if p.get("g_solver") != "thomas":
        assert abs(it - ref_it) <= 2, (it, ref_it)
        # residual of the GPU solution, measured by the oracle's operator
        r = b - (got.reshape(shape) + P.dT * heat.apply_A(got.reshape(shape), P.h, P.kappa))
        assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(b) * 10


@pytest.mark.parametrize("case", ["2d_const", "2d_var", "3d_const", "3d_var", "1d_explicit"])
@pytest.mark.parametrize("recurrence", ["textbook", "single"])
def test_coarse_cg_recurrences_match_their_oracle(case, recurrence):
    """PR_OPT_G_CG forces each coarse CG recurrence; each is compared with the
    oracle's CG of the same recurrence (solution at 1e-12, iteration count within
    2) from a warm start and from the right-hand side."""
    p = CASES[case]()
    p["g_cg"] = recurrence
    rng = np.random.default_rng(17)
    shape = tuple(reversed(p["n"]))
    b = rng.standard_normal(shape)
    P = oracle_props(p)
    with Ctx(p) as c:
        pr.parareal_set_option(c.ctx, pr.PR_OPT_G_CG, 1 if recurrence == "textbook" else 2)
        for x0 in (b + 0.1 * rng.standard_normal(shape), None):
            ref, ref_it = P.G(b, x0=x0)
            out = torch().empty(c.M, dtype=torch().float64, device="cuda")
            it = pr.parareal_coarse(c.ctx, dev(b), None if x0 is None else dev(x0), out)
            got = host(out)
            assert rel_l2(got, ref) < FP64_TOL
            assert abs(it - ref_it) <= 2, (it, ref_it)


def test_single_reduction_cg_on_an_hbm_resident_grid():
    """The single-reduction recurrence forced on the 4-blocks/SM instance (2.5 M points)."""
    n = (136, 136, 136)
    rng = np.random.default_rng(18)
    h = tuple(1.0 / (m + 1) for m in n)
    shape = tuple(reversed(n))
    p = dict(dim=3, n=n, h=h, N=1, f_steps=64, dt=0.15 * h[0] ** 2, f_scheme="explicit",
             g_solver="cg", g_rtol=1e-8, u0=np.zeros(shape), tol=0.0, g_cg="single")
    b = rng.standard_normal(shape)
    ref, ref_it = oracle_props(p).G(b)
    with Ctx(p) as c:
        pr.parareal_set_option(c.ctx, pr.PR_OPT_G_CG, 2)
        out = torch().empty(c.M, dtype=torch().float64, device="cuda")
        it = pr.parareal_coarse(c.ctx, dev(b), None, out)
        got = host(out)
    assert abs(it - ref_it) <= 2
    assert rel_l2(got, ref) < 1e-10


@pytest.mark.parametrize("case", ["2d_const", "2d_var"])
def test_sync_parareal_single_reduction_coarse_matches_oracle(case):
    """Algorithm 1 with the single-reduction coarse CG on both sides (the GPU's
    automatic choice on grids that fit in L2), every iterate."""
    p = CASES[case]()
    p["g_cg"] = "single"
    ref = sync_parareal(p, tol=0.0, record=True)
    with Ctx(p) as c:
        pr.parareal_set_option(c.ctx, pr.PR_OPT_G_CG, 2)
        for k in (1, 2, p["N"] // 2, p["N"]):
            c.prob.max_iter = k
            c.prob.tol = 0.0
            pr.parareal_set_problem(c.ctx, c.prob)
            lam = c.lam()
            pr.parareal_run_sync(c.ctx, lam)
            assert rel_l2(host(lam), ref.iterates[k]) < FP64_TOL, k


def test_coarse_propagator_hbm_resident_grid():
    """2.5 M points (the CG instance sized for grids that do not fit in L2)."""
    n = (136, 136, 136)
    rng = np.random.default_rng(16)
    h = tuple(1.0 / (m + 1) for m in n)
    shape = tuple(reversed(n))
    p = dict(dim=3, n=n, h=h, N=1, f_steps=64, dt=0.15 * h[0] ** 2, f_scheme="explicit",
             g_solver="cg", g_rtol=1e-8, u0=np.zeros(shape), tol=0.0)
    b = rng.standard_normal(shape)
    P = oracle_props(p)
    ref, ref_it = P.G(b)
    with Ctx(p) as c:
        out = torch().empty(c.M, dtype=torch().float64, device="cuda")
        it = pr.parareal_coarse(c.ctx, dev(b), None, out)
        got = host(out)
    assert abs(it - ref_it) <= 2
    assert rel_l2(got, ref) < 1e-10


def test_correction_is_bit_exact():
    p = CASES["2d_const"]()
    rng = np.random.default_rng(14)
    M = int(np.prod(p["n"]))
    wn, v, wo, lam = (rng.standard_normal(M) * s for s in (1.0, 1e-3, 1.0, 1.0))
    expect = (wn + v) - wo
    with Ctx(p) as c:
        lam_t = dev(lam)
        d = pr.parareal_correct(c.ctx, dev(wn), dev(v), dev(wo), lam_t)
        got = host(lam_t)
    assert np.array_equal(got, expect)
    assert d == np.max(np.abs(expect - lam))


@pytest.mark.parametrize("case", list(CASES))
def test_sync_parareal_matches_oracle(case):
    p = CASES[case]()
    p["tol"] = 1e-9 if case != "1d_thomas" else 1e-10
    ref = sync_parareal(p)
    with Ctx(p) as c:
        lam = c.lam()
        code, st = pr.parareal_run_sync(c.ctx, lam)
        got = host(lam).reshape(ref.lam.shape)
        ks, ds = pr.parareal_slice_stats(c.ctx, p["N"])
    assert st.iterations == ref.k, (st.iterations, ref.k)
    assert rel_l2(got, ref.lam) < FP64_TOL
    # increments near convergence are differences of O(1) states: compare on the state scale
    np.testing.assert_allclose(st.max_delta, np.max(ref.deltas[-1]), rtol=0,
                               atol=1e-12 * np.max(np.abs(ref.lam)))
    assert st.fine_lups == sum(p["N"] - k for k in range(ref.k)) * int(np.prod(p["n"])) * p["f_steps"]


@pytest.mark.parametrize("case", ["2d_const", "3d_var", "1d_thomas"])
def test_sync_every_iterate_matches_oracle(case):
    """Run with max_iter = k for each k and compare lam^k (iterate-level parity)."""
    p = CASES[case]()
    ref = sync_parareal(p, tol=0.0, record=True)
    with Ctx(p) as c:
        for k in range(1, p["N"] + 1):
            c.prob.max_iter = k
            c.prob.tol = 0.0
            pr.parareal_set_problem(c.ctx, c.prob)
            lam = c.lam()
            pr.parareal_run_sync(c.ctx, lam)
            assert rel_l2(host(lam), ref.iterates[k]) < FP64_TOL, k


@pytest.mark.parametrize("case", ["2d_const", "3d_const"])
def test_sync_mixed_precision_against_fp64_oracle(case):
    p = CASES[case]()
    p["f_prec"] = 32
    p["tol"] = 1e-7
    ref = sync_parareal(p)
    with Ctx(p) as c:
        lam = c.lam()
        pr.parareal_run_sync(c.ctx, lam)
        got = host(lam)
    assert rel_l2(got, ref.lam) < MIXED_TOL


@pytest.mark.parametrize("case", ["2d_var", "1d_thomas", "3d_const"])
def test_finite_termination_equals_serial_fine(case):
    p = CASES[case]()
    p["g_rtol"] = 1e-4   # inexact coarse solves: termination holds for any G
    ref = serial_fine(p)
    with Ctx(p) as c:
        lam = c.lam()
        code, st = pr.parareal_run_sync(c.ctx, lam)
        assert st.iterations == p["N"]
        sf = c.lam()
        pr.parareal_serial_fine(c.ctx, sf)
        assert rel_l2(host(sf), ref) < FP64_TOL
        assert rel_l2(host(lam), ref) < FP64_TOL


def test_run_sync_host_buffers_match_device_run():
    p = CASES["2d_const"]()
    p["tol"] = 1e-8
    with Ctx(p) as c:
        lam = c.lam()
        pr.parareal_run_sync(c.ctx, lam)
        t = torch()
        u0h = t.from_numpy(p["u0"].reshape(-1).copy()).pin_memory()
        out = t.empty((p["N"] + 1) * c.M, dtype=t.float64).pin_memory()
        code, st = pr.parareal_run_sync_host(c.ctx, u0h, out)
        assert np.array_equal(out.numpy(), host(lam))


# ------------------------------------------------------------------ edges
def test_single_slice_single_point_1d():
    p = dict(dim=1, n=(1,), h=(0.5,), N=1, f_steps=3, dt=1e-3, f_scheme="implicit",
             g_solver="thomas", u0=np.array([0.7]), tol=0.0)
    ref = sync_parareal(p)
    with Ctx(p) as c:
        lam = c.lam()
        pr.parareal_run_sync(c.ctx, lam)
        assert rel_l2(host(lam), ref.lam) < FP64_TOL


@pytest.mark.parametrize("n", [(2,), (3,), (5,), (33,), (64,), (65,), (1000,)])
def test_thomas_partition_ragged_sizes(n):
    rng = np.random.default_rng(n[0])
    p = dict(dim=1, n=n, h=(1.0 / (n[0] + 1),), N=3, f_steps=4, dt=2e-3, f_scheme="implicit",
             g_solver="thomas", u0=rng.standard_normal(n), tol=0.0,
             kappa=np.exp(rng.standard_normal(n[0] + 2)))
    P = oracle_props(p)
    X = rng.standard_normal((3,) + n)
    with Ctx(p) as c:
        xin = dev(X)
        out = torch().empty_like(xin)
        pr.parareal_fine(c.ctx, xin, out, 3)
        got = host(out).reshape(X.shape)
    for s in range(3):
        assert rel_l2(got[s], P.F(X[s])) < FP64_TOL


@pytest.mark.parametrize("n", [(1, 1), (33, 1), (1, 40), (31, 33)])
def test_explicit_ragged_tiles_2d(n):
    rng = np.random.default_rng(5)
    p = dict(dim=2, n=n, h=tuple(1.0 / (m + 1) for m in n), N=2, f_steps=5,
             dt=0.2 * min(1.0 / (m + 1) for m in n) ** 2, f_scheme="explicit", g_solver="cg",
             g_rtol=1e-13, u0=rng.standard_normal(tuple(reversed(n))), tol=0.0)
    P = oracle_props(p)
    X = rng.standard_normal((2,) + tuple(reversed(n)))
    with Ctx(p) as c:
        xin = dev(X)
        out = torch().empty_like(xin)
        pr.parareal_fine(c.ctx, xin, out, 2)
        got = host(out).reshape(X.shape)
    for s in range(2):
        assert rel_l2(got[s], P.F(X[s])) < FP64_TOL


def test_invalid_problems_are_rejected():
    p = CASES["2d_const"]()
    t = torch()
    u0 = dev(p["u0"])
    ctx = pr.parareal_create(0, t.cuda.current_stream())
    try:
        lam = t.zeros(10, dtype=t.float64, device="cuda")
        with pytest.raises(pr.PararealError) as e:
            pr.parareal_run_sync(ctx, lam)
        assert e.value.code == pr.PR_ESTATE
        from .gpu_util import problem_struct
        bad = [dict(N=0), dict(dim=4), dict(f_steps=0), dict(T=-1.0),
               dict(f_prec=16), dict(g_solver=pr.PR_SOLVER_THOMAS)]
        for over in bad:
            s = problem_struct(p, u0, None, **over)
            with pytest.raises(pr.PararealError) as e:
                pr.parareal_set_problem(ctx, s)
            assert e.value.code == pr.PR_EINVAL, over
        # unstable explicit step: dt = 0.35 h^2 in 2D gives dt*lambda_max near 2.8 > 2
        s = problem_struct(p, u0, None, T=p["N"] * p["f_steps"] * 0.35 * (1.0 / (p["n"][0] + 1)) ** 2)
        with pytest.raises(pr.PararealError) as e:
            pr.parareal_set_problem(ctx, s)
        assert e.value.code == pr.PR_EINVAL
        # misaligned device pointer
        s = problem_struct(p, u0, None)
        s.u0_dev = s.u0_dev + 8
        with pytest.raises(pr.PararealError):
            pr.parareal_set_problem(ctx, s)
    finally:
        pr.parareal_destroy(ctx)


def test_out_of_memory_problem_leaves_context_usable():
    """A problem whose trajectory cannot be allocated (40000^2 x 64 slices, about
    0.8 TB per array, within the size limits) fails with PR_ENOMEM before anything
    runs; the context then takes an ordinary problem and solves it as usual."""
    p = CASES["2d_const"]()
    t = torch()
    ctx = pr.parareal_create(0, t.cuda.current_stream())
    try:
        u0 = dev(p["u0"])
        huge = pr.make_problem(dim=2, n=(40000, 40000), T0=0.0, T=1e-6, N=64, u0=u0,
                               f_steps=16, g_rtol=1e-10, tol=1e-9)
        with pytest.raises(pr.PararealError) as e:
            pr.parareal_set_problem(ctx, huge)
        assert e.value.code == pr.PR_ENOMEM
        from .gpu_util import problem_struct
        pr.parareal_set_problem(ctx, problem_struct(p, u0, None))
        lam = t.zeros((p["N"] + 1) * u0.numel(), dtype=t.float64, device="cuda")
        code, st = pr.parareal_run_sync(ctx, lam)
        ref = sync_parareal(p)
        assert code == pr.PR_OK and st.iterations == ref.k
        assert rel_l2(host(lam), ref.lam) < FP64_TOL
    finally:
        pr.parareal_destroy(ctx)


def test_set_problem_rejects_sizes_beyond_the_limits_without_overflow():
    """Each axis and the running product are bounded before the next
    multiplication: three axes of 2^21 (product 2^63, which wraps a signed
    64-bit integer), a product just above 2^31 - 1, and a trajectory of more
    than 2^40 points are PR_EINVAL; nothing is allocated or launched."""
    p = CASES["2d_const"]()
    t = torch()
    ctx = pr.parareal_create(0, t.cuda.current_stream())
    try:
        u0 = dev(p["u0"])
        bad = [dict(dim=3, n=(1 << 21, 1 << 21, 1 << 21), N=4),
               dict(dim=2, n=(65536, 32769), N=4),
               dict(dim=3, n=(2048, 2048, 256), N=1100),
               dict(dim=1, n=(16,), N=70000)]
        for kw in bad:
            prob = pr.make_problem(T0=0.0, T=1e-6, u0=u0, f_steps=4, g_rtol=1e-10, tol=1e-9, **kw)
            with pytest.raises(pr.PararealError) as e:
                pr.parareal_set_problem(ctx, prob)
            assert e.value.code == pr.PR_EINVAL, kw
    finally:
        pr.parareal_destroy(ctx)


@pytest.mark.parametrize("case,chunks,bps", [("2d_const", 8, 0), ("2d_var", 3, 1),
                                             ("3d_var", 1, 0), ("1d_thomas", 4, 0),
                                             ("3d_const", 100, 2)])
def test_pipelined_schedule_is_bitwise_identical(case, chunks, bps):
    """Overlapping F of iteration k+1 with the sweep of k changes timing only."""
    p = CASES[case]()
    p["tol"] = 1e-9
    if case == "3d_var":
        p["f_prec"] = 32
    with Ctx(p) as c:
        lam_a = c.lam()
        code_a, st_a = pr.parareal_run_sync(c.ctx, lam_a)
        pr.parareal_set_option(c.ctx, pr.PR_OPT_PIPELINE, 1)
        pr.parareal_set_option(c.ctx, pr.PR_OPT_PIPELINE_CHUNKS, chunks)
        pr.parareal_set_option(c.ctx, pr.PR_OPT_CG_BLOCKS_PER_SM, bps)
        for _ in range(2):
            lam_b = c.lam()
            code_b, st_b = pr.parareal_run_sync(c.ctx, lam_b)
            assert st_b.iterations == st_a.iterations
            assert st_b.fine_lups == st_a.fine_lups
            if bps == 0:
                assert torch().equal(lam_a, lam_b)
            else:   # fewer CG blocks: same arithmetic, another summation order
                assert rel_l2(host(lam_b), host(lam_a)) < FP64_TOL


@pytest.mark.parametrize("case", ["2d_const", "3d_var", "1d_thomas"])
def test_pipelined_schedule_matches_oracle(case):
    """The pipelined schedule against Algorithm 1 in the oracle (not only against
    the plain GPU schedule): the converged run and two capped runs, every point."""
    p = CASES[case]()
    p["tol"] = 1e-9 if case != "1d_thomas" else 1e-10
    ref = sync_parareal(p)
    rec = sync_parareal(p, tol=0.0, record=True)
    with Ctx(p) as c:
        pr.parareal_set_option(c.ctx, pr.PR_OPT_PIPELINE, 1)
        pr.parareal_set_option(c.ctx, pr.PR_OPT_PIPELINE_CHUNKS, 3)
        lam = c.lam()
        code, st = pr.parareal_run_sync(c.ctx, lam)
        assert st.iterations == ref.k
        assert rel_l2(host(lam), ref.lam) < FP64_TOL
        for k in (1, 2):
            c.prob.max_iter = k
            c.prob.tol = 0.0
            pr.parareal_set_problem(c.ctx, c.prob)
            lam = c.lam()
            pr.parareal_run_sync(c.ctx, lam)
            assert rel_l2(host(lam), rec.iterates[k]) < FP64_TOL, k


def test_pipelined_schedule_with_iteration_cap_and_bad_options():
    p = CASES["2d_const"]()
    p["tol"] = 1e-14
    p["max_iter"] = 3
    with Ctx(p) as c:
        lam_a = c.lam()
        code_a, st_a = pr.parareal_run_sync(c.ctx, lam_a)
        pr.parareal_set_option(c.ctx, pr.PR_OPT_PIPELINE, 1)
        lam_b = c.lam()
        code_b, st_b = pr.parareal_run_sync(c.ctx, lam_b)
        assert code_a == code_b == pr.PR_ENOTCONV and st_b.iterations == 3
        assert torch().equal(lam_a, lam_b)
        for opt, val in [(99, 1), (pr.PR_OPT_PIPELINE_CHUNKS, 0), (pr.PR_OPT_CG_BLOCKS_PER_SM, -1)]:
            with pytest.raises(pr.PararealError):
                pr.parareal_set_option(c.ctx, opt, val)


def test_notconv_status_when_max_iter_stops_early():
    p = CASES["2d_const"]()
    p["tol"] = 1e-14
    p["max_iter"] = 2
    with Ctx(p) as c:
        lam = c.lam()
        code, st = pr.parareal_run_sync(c.ctx, lam)
        assert code == pr.PR_ENOTCONV and st.iterations == 2 and not st.converged


@pytest.mark.parametrize("case", ["2d_const", "2d_var", "3d_const", "3d_var"])
def test_fine_and_coarse_are_symmetric(case):
    """Dot-product tests <F x, y> = <x, F y> and <G x, y> = <x, G y> of the GPU
    propagators (F = S^n_f and G = (I + dT A)^-1 are symmetric; the adjoint relies on it)."""
    p = CASES[case]()
    p["f_prec"] = 64
    p["g_rtol"] = 1e-14
    rng = np.random.default_rng(19)
    shape = tuple(reversed(p["n"]))
    x, y = rng.standard_normal(shape), rng.standard_normal(shape)
    with Ctx(p) as c:
        outs = {}
        for name, v in (("x", x), ("y", y)):
            f = torch().empty(c.M, dtype=torch().float64, device="cuda")
            g = torch().empty(c.M, dtype=torch().float64, device="cuda")
            pr.parareal_fine(c.ctx, dev(v), f, 1)
            pr.parareal_coarse(c.ctx, dev(v), None, g)
            outs[name] = (host(f), host(g))
    fx, gx = outs["x"]
    fy, gy = outs["y"]
    xv, yv = x.reshape(-1), y.reshape(-1)
    for a, b in ((fx @ yv, xv @ fy), (gx @ yv, xv @ gy)):
        assert abs(a - b) <= 1e-12 * max(abs(a), np.linalg.norm(xv) * np.linalg.norm(yv) * 1e-3)
