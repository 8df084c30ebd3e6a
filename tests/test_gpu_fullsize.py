"""Parity at the full workload sizes, in the launch configuration bench.py times.

The oracle cannot run a whole Parareal solve at these sizes, so the checks
use outputs it can compute one at a time (one fine propagation, one coarse
residual) and properties that hold at any size:
  * after k >= 1 iterations slice 1 is exact: lambda_1 = F(u0) (§3.2);
  * at convergence lambda_i - F(lambda_{i-1}) is of the order of the last
    increments (Eq. (11) with lambda^k ~ lambda^{k-1});
  * the coarse solve meets its residual bound, measured with the oracle's
    operator;
  * one correction of Eq. (11) / Algorithm 1 element by element: from the
    GPU's own iterates lambda^k and lambda^{k+1} the oracle forms
    (G(lambda_{i-1}^{k+1}) + F(lambda_{i-1}^k)) - G(lambda_{i-1}^k) for sampled
    slices i and compares it with the GPU's lambda_i^{k+1} at every point.
"""
import numpy as np
import pytest

from oracle import heat
from synthetic import preset

from .gpu_util import Ctx, dev, host, rel_l2, torch

import paper_2110_10762_gb300 as pr  # noqa: E402  (a missing library fails the first call loudly)

pytestmark = pytest.mark.gpu


def test_heat2d_bench_workload_sampled_parity():
    """1024^2, N = 64, F = 256 explicit steps, coarse CG rtol 1e-10 preconditioned by
    16 Chebyshev steps, tol 1e-10 (the 2D workload's launch configuration)."""
    p = preset("heat2d_explicit", "full")
    P = heat.Propagators(p)
    shape = tuple(reversed(p["n"]))
    with Ctx(p) as c:
        lam = c.lam()
        code, st = pr.parareal_run_sync(c.ctx, lam)
        L = host(lam).reshape((p["N"] + 1,) + shape)
        # coarse solve on the last state: residual of the GPU solution by the oracle's operator
        out = torch().empty(c.M, dtype=torch().float64, device="cuda")
        pr.parareal_coarse(c.ctx, dev(L[-2]), None, out)
        x = host(out).reshape(shape)
    assert code == pr.PR_OK and st.converged and 1 <= st.iterations < p["N"]
    assert np.array_equal(L[0], p["u0"])
    assert rel_l2(L[1], P.F(p["u0"])) < 1e-12
    for i in (2, p["N"] // 2, p["N"]):
        gap = np.max(np.abs(L[i] - P.F(L[i - 1])))
        assert gap < 20 * p["tol"], (i, gap)
    r = L[-2] - (x + P.dT * heat.apply_A(x, P.h, None))
    assert np.linalg.norm(r) <= 1.01 * p["g_rtol"] * np.linalg.norm(L[-2])


def test_heat3d_mixed_workload_sampled_parity():
    """256^3, N = 128, FP32 fine / FP64 coarse, tol 1e-5: slice 1 and the accuracy target."""
    p = preset("heat3d_mixed", "full")
    p["g_rtol"] = 1e-7
    P64 = heat.Propagators(p)
    shape = tuple(reversed(p["n"]))
    with Ctx(p) as c:
        lam = c.lam()
        code, st = pr.parareal_run_sync(c.ctx, lam)
        l1 = host(lam[c.M:2 * c.M]).reshape(shape)
        lN = host(lam[p["N"] * c.M:]).reshape(shape)
        lNm1 = host(lam[(p["N"] - 1) * c.M:p["N"] * c.M]).reshape(shape)
    assert code == pr.PR_OK and st.converged
    ref1 = P64.F(p["u0"])                      # FP64 oracle
    assert rel_l2(l1, ref1) < 1e-5
    scale = np.max(np.abs(ref1))
    gap = np.max(np.abs(lN - P64.F(lNm1))) / scale
    assert gap < 1e-5, gap


def _iterates(p, k, slices, **over):
    """Slices `slices` of the GPU's lambda^k (max_iter = k, tol = 0) as host arrays."""
    shape = tuple(reversed(p["n"]))
    with Ctx(p, tol=0.0, max_iter=k, **over) as c:   # Ctx applies the preset's coarse options
        lam = c.lam()
        code, st = pr.parareal_run_sync(c.ctx, lam)
        assert st.iterations == k
        out = {i: host(lam[i * c.M:(i + 1) * c.M]).reshape(shape) for i in slices}
    return out


def _correction_parity(p, k, slices, tol, P):
    """lambda_i^{k+1} against (G(lambda_{i-1}^{k+1}) + F(lambda_{i-1}^k)) - G(lambda_{i-1}^k)
    computed by the FP64 oracle from the GPU's lambda^k and lambda^{k+1}, for
    slices i with i - 1 > k (fresh coarse values).  The coarse difference is
    taken as G(lambda_{i-1}^{k+1} - lambda_{i-1}^k) (G is linear), solved to
    rtol 1e-14 of that difference.  Slices i <= k are frozen (Algorithm 1)."""
    need = sorted(set([i - 1 for i in slices] + list(slices) + [1, k]))
    Lk = _iterates(p, k, need)
    Lk1 = _iterates(p, k + 1, need)
    assert np.array_equal(Lk1[k], Lk[k]) and np.array_equal(Lk1[1], Lk[1])   # frozen prefix
    worst = 0.0
    for i in slices:
        assert i - 1 > k
        d = Lk1[i - 1] - Lk[i - 1]
        Gd, _ = heat.cg_implicit_euler(d, P.dT, P.h, P.kappa, None, rtol=1e-14, maxit=20000)
        expect = Gd + P.F(Lk[i - 1])
        err = np.max(np.abs(Lk1[i] - expect)) / np.max(np.abs(expect))
        assert rel_l2(Lk1[i], expect) < tol, (i, rel_l2(Lk1[i], expect))
        assert err < tol, (i, err)
        worst = max(worst, err)
    return worst


def test_heat2d_bench_workload_correction_parity():
    """1024^2, N = 64, F = 256 explicit FP64 steps, coarse CG at the parity
    setting rtol 1e-13: one correction (k = 2 -> 3) at every point of slices 4,
    32 and 64, within 1e-12."""
    p = preset("heat2d_explicit", "full")
    p["g_rtol"] = 1e-13
    _correction_parity(p, 2, (4, p["N"] // 2, p["N"]), 1e-12, heat.Propagators(p))


def test_heat3d_mixed_workload_correction_parity():
    """256^3, N = 128, FP32 fine / FP64 coarse in the bench's coarse configuration:
    one correction (k = 2 -> 3) at every point of slice 64 against the FP64
    oracle, within the mixed-precision tolerance 1e-5."""
    p = preset("heat3d_mixed", "full")
    _correction_parity(p, 2, (p["N"] // 2,), 1e-5, heat.Propagators(dict(p, f_prec=64)))


def test_heat3d_varkappa_fp32_fine_step_full_size():
    """192^3 variable kappa, FP32 vector kernel (one slice, 32 steps) vs the FP64 oracle."""
    p = preset("heat3d_varkappa_async", "full")
    P = heat.Propagators(dict(p, f_prec=64))
    rng = np.random.default_rng(17)
    x0 = p["u0"] + 0.01 * rng.standard_normal(p["u0"].shape)
    with Ctx(p) as c:
        xin = dev(x0)
        out = torch().empty_like(xin)
        pr.parareal_fine(c.ctx, xin, out, 1)
        got = host(out).reshape(x0.shape)
    err = rel_l2(got, P.F(x0))
    assert 1e-12 < err < 1e-5, err


def test_heat1d_thomas_workload_full_size():
    """1023 points, N = 16, F = 100 implicit-Euler steps, G by Thomas, tol 1e-10.
    The oracle runs the first three iterations at full size: the stacked
    (N+1) x M trajectory of every iterate k = 1..3 must match
    within 1e-12 relative L2; the converged run must stop with its last
    increment below tol and sit on the oracle's serial fine solution."""
    from oracle.parareal import serial_fine, sync_parareal

    p = preset("heat1d_thomas", "full")
    K = 3
    ref = sync_parareal(p, tol=0.0, max_iter=K, record=True)
    for k in range(1, K + 1):
        with Ctx(p, tol=0.0, max_iter=k) as c:
            lam = c.lam()
            code, st = pr.parareal_run_sync(c.ctx, lam)
            got = host(lam).reshape(p["N"] + 1, -1)
        assert st.iterations == k
        assert rel_l2(got, ref.iterates[k]) < 1e-12, k
    with Ctx(p) as c:
        lam = c.lam()
        code, st = pr.parareal_run_sync(c.ctx, lam)
        got = host(lam).reshape(p["N"] + 1, -1)
    assert code == pr.PR_OK and st.converged and st.max_delta < p["tol"]
    star = serial_fine(p)
    assert np.max(np.abs(got - star)) < 100 * p["tol"] * max(1.0, np.max(np.abs(star)))
    assert np.array_equal(got[0], p["u0"].reshape(-1))


def test_heat2d_async_workload_full_size():
    """The asynchronous kernel on the 1024^2, N = 64 FP64 workload in the launch
    configuration the benchmark times (automatic teams, no delays, tol 1e-10).
    Checked: the log is a valid asynchronous schedule (consecutive versions,
    fine input = previous coarse input, a coarse solve exactly when the input
    changed); slice 1 is exactly F(u0) by the oracle; and sampled slices sit
    on the fine propagation of their predecessor, lambda_i = F(lambda_{i-1}),
    within the order of the stop tolerance."""
    p = preset("heat2d_explicit", "full")
    P = heat.Propagators(p)
    shape = tuple(reversed(p["n"]))
    with Ctx(p) as c:
        lam = c.lam()
        opts = pr.make_async_opts(timeout_s=120.0)
        code, st, log = pr.parareal_run_async(c.ctx, opts, lam, log_cap=1 << 20)
        L = host(lam).reshape((p["N"] + 1,) + shape)
    assert code == pr.PR_OK and st.converged and st.iterations >= 1
    last = {i: (0, 0) for i in range(1, p["N"] + 1)}
    for e in sorted(log, key=lambda e: (e.slice, e.version)):
        k, vG = last[e.slice]
        assert e.version == k + 1 and e.vF == vG and e.vG >= e.vF
        assert e.cg_iters == 0 or e.vG > e.vF   # no solve when the input did not change
        last[e.slice] = (e.version, e.vG)
    assert all(v >= 1 for v, _ in last.values())
    assert np.array_equal(L[0], p["u0"])
    assert rel_l2(L[1], P.F(p["u0"])) < 1e-12
    for i in (2, p["N"] // 2, p["N"]):
        gap = np.max(np.abs(L[i] - P.F(L[i - 1])))
        assert gap < 20 * p["tol"], (i, gap)


def test_heat3d_varkappa_async_workload_full_size():
    """192^3 variable kappa, N = 256, F = 32 FP32 steps, FP64 coarse CG, seeded
    publication delays of 0-4 units, tol 1e-5: the asynchronous kernel in the
    benchmark's launch configuration (automatic teams; the unit here is 36.6 us,
    the measured duration of one fine step of one slice).  Checked: a valid
    asynchronous log whose delays were honoured, slice 1 against the FP64
    oracle's F(u0) within the mixed-precision bound, and the last slice on the
    FP64 fine propagation of its predecessor within the stop rule's tolerance
    plus the FP32 rounding of F."""
    from synthetic import delay_table

    p = preset("heat3d_varkappa_async", "full")
    P64 = heat.Propagators(dict(p, f_prec=64))
    shape = tuple(reversed(p["n"]))
    unit_ns = 36600.0
    table = delay_table(p["N"], 64, seed=p["delay_seed"])
    with Ctx(p) as c:
        delays = torch().from_numpy(table).cuda()
        opts = pr.make_async_opts(timeout_s=240.0, delays=delays, delay_unit_ns=unit_ns)
        lam = c.lam()
        code, st, log = pr.parareal_run_async(c.ctx, opts, lam, log_cap=1 << 20)
        torch().cuda.synchronize()
        picks = (1, p["N"])
        L = {i: host(lam[i * c.M:(i + 1) * c.M]).reshape(shape) for i in picks}
        L.update({i - 1: host(lam[(i - 1) * c.M:i * c.M]).reshape(shape) for i in picks})
    assert code == pr.PR_OK and st.converged
    last = {i: (0, 0) for i in range(1, p["N"] + 1)}
    for e in sorted(log, key=lambda e: (e.slice, e.version)):
        k, vG = last[e.slice]
        assert e.version == k + 1 and e.vF == vG and e.vG >= e.vF
        # visibility = publication + delay: the update spans at least its delay
        assert e.t_end >= e.t_start + int(table[e.slice - 1, k % 64] * unit_ns) - 1
        last[e.slice] = (e.version, e.vG)
    assert all(v >= 1 for v, _ in last.values())
    ref1 = P64.F(p["u0"])
    assert rel_l2(L[1], ref1) < 1e-5
    scale = np.max(np.abs(ref1))
    gap = np.max(np.abs(L[p["N"]] - P64.F(L[p["N"] - 1])))
    assert gap < 2 * p["tol"] + 1e-5 * scale, gap
