"""Asynchronous Parareal persistent kernel (Eq. (12), Algorithm 2) against the
oracle's replay of the kernel's own event log.

Parity: the oracle recomputes every logged update in FP64 from the logged
input versions; the GPU's final state must match within 1e-12 relative L2
(FP64 fine steps) or 1e-5 (FP32 fine steps).  Run to quiescence, the result
must equal the serial fine solution (async finite termination, §3.2).
"""
import numpy as np
import pytest

from oracle.parareal import async_replay, serial_fine
from synthetic import delay_table, preset

from .gpu_util import Ctx, host, rel_l2, torch

import paper_2110_10762_gb300 as pr  # noqa: E402  (a missing library fails the first call loudly)

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = 1e-5


def case(name, **over):
    p = preset(name, "small")
    p.update(dict(g_rtol=1e-13, f_prec=64))
    p.update(over)
    return p


def events_of(log):
    return [(e.slice, e.version, e.vF, e.vG) for e in log]


def check_log(log, N):
    last = {i: (0, 0) for i in range(1, N + 1)}   # slice -> (version, vG)
    for e in sorted(log, key=lambda e: (e.slice, e.version)):
        k, vG = last[e.slice]
        assert e.version == k + 1
        assert e.vF == vG
        assert e.vG >= e.vF
        assert (e.cg_iters > 0) == (e.vG > e.vF) or e.cg_iters == 0
        last[e.slice] = (e.version, e.vG)


def run_async(c, log_cap=100000, **kw):
    opts = pr.make_async_opts(**kw)
    lam = c.lam()
    code, st, log = pr.parareal_run_async(c.ctx, opts, lam, log_cap=log_cap)
    return code, st, log, host(lam)


@pytest.mark.parametrize("name", ["heat2d_explicit", "heat3d_varkappa_async", "heat2d_inverse"])
def test_async_replay_parity_fp64(name):
    p = case(name, tol=1e-9)
    with Ctx(p) as c:
        code, st, log, lam = run_async(c, timeout_s=60.0)
    assert code == pr.PR_OK and st.converged
    check_log(log, p["N"])
    assert st.iterations == max(e.version for e in log)
    rep = async_replay(p, events_of(log))
    assert rel_l2(lam, rep.lam) < FP64_TOL
    # the stop rule held when the monitor stopped: after some prefix of the log
    # (publication order) every slice had updated and its last update either moved
    # it by less than tol or was settled (fine and coarse inputs both the
    # predecessor's latest version).  Updates already running at the stop still
    # publish, so at most one event per team may follow that prefix.
    assert stop_prefix_length(log, p["N"], p["tol"]) >= len(log) - len({e.team for e in log})


def stop_prefix_length(log, N, tol):
    """Length of the longest log prefix after which the asynchronous stop rule
    holds, or -1 if none does."""
    last, latest, found = {}, {0: 0}, -1
    for n_ev, e in enumerate(log, 1):
        last[e.slice] = e
        latest[e.slice] = e.version
        if len(last) < N:
            continue
        if all(last[i].delta < tol or last[i].vF == last[i].vG == latest[i - 1]
               for i in range(1, N + 1)):
            found = n_ev
    return found


@pytest.mark.parametrize("name", ["heat2d_explicit", "heat3d_mixed"])
def test_async_quiescence_is_serial_fine(name):
    p = case(name, g_rtol=1e-6)   # any coarse accuracy: the fixed point is lambda*
    ref = serial_fine(p)
    with Ctx(p) as c:
        code, st, log, lam = run_async(c, timeout_s=60.0, quiescence=True)
    assert code == pr.PR_OK and st.converged
    check_log(log, p["N"])
    assert rel_l2(lam, ref) < FP64_TOL


@pytest.mark.parametrize("ctas", [1, 3])
def test_async_team_sizes_and_mixed_precision(ctas):
    p = case("heat3d_varkappa_async", f_prec=32, tol=1e-7)
    with Ctx(p) as c:
        code, st, log, lam = run_async(c, timeout_s=60.0, ctas_per_slice=ctas)
    assert code == pr.PR_OK
    check_log(log, p["N"])
    p64 = dict(p, f_prec=64)
    rep = async_replay(p64, events_of(log))
    err = rel_l2(lam, rep.lam)
    assert err < MIXED_TOL, err


def test_async_with_injected_delays():
    p = case("heat2d_explicit", tol=1e-9)
    delays = delay_table(p["N"], 64, seed=51)
    with Ctx(p) as c:
        d = torch().from_numpy(delays).cuda()
        code, st, log, lam = run_async(c, timeout_s=60.0, delays=d, delay_unit_ns=20000.0)
    assert code == pr.PR_OK
    check_log(log, p["N"])
    rep = async_replay(p, events_of(log))
    assert rel_l2(lam, rep.lam) < FP64_TOL
    # every event respects its delay: visible time - start >= delay units
    for e in log:
        dly = delays[e.slice - 1, (e.version - 1) % delays.shape[1]]
        assert e.t_end >= e.t_start + int(dly * 20000.0) - 1


def test_async_one_slice_delayed_far_beyond_the_others():
    """An extreme delay schedule: every publication of slice 3 becomes visible only
    after 200 delay units, the others at once.  The run still terminates (quiescence),
    its log replays, and the result is the serial fine solution."""
    p = case("heat2d_explicit", tol=1e-9)
    delays = np.zeros((p["N"], 8), dtype=np.int32)
    delays[2, :] = 200
    with Ctx(p) as c:
        d = torch().from_numpy(delays).cuda()
        code, st, log, lam = run_async(c, timeout_s=60.0, delays=d, delay_unit_ns=20000.0,
                                       quiescence=True)
    assert code == pr.PR_OK and st.converged
    check_log(log, p["N"])
    rep = async_replay(p, events_of(log))
    assert rel_l2(lam, rep.lam) < FP64_TOL
    assert rel_l2(lam, serial_fine(p)) < FP64_TOL
    # the delayed slice's versions became visible 200 units after their start
    for e in log:
        if e.slice == 3:
            assert e.t_end >= e.t_start + 200 * 20000 - 1


@pytest.mark.parametrize("quiescence", [False, True])
def test_async_lazy_policy(quiescence):
    """Skipping superseded re-updates keeps replay parity and the quiescent fixed point."""
    p = case("heat2d_explicit", tol=1e-9)
    with Ctx(p) as c:
        code, st, log, lam = run_async(c, timeout_s=60.0, lazy=True, quiescence=quiescence)
    assert code == pr.PR_OK and st.converged
    check_log(log, p["N"])
    rep = async_replay(p, events_of(log))
    assert rel_l2(lam, rep.lam) < FP64_TOL
    if quiescence:
        assert rel_l2(lam, serial_fine(p)) < FP64_TOL


@pytest.mark.parametrize("name", ["heat2d_explicit", "heat3d_varkappa_async"])
def test_async_verified_stop(name):
    """Verify mode: the run ends only when the fixed-point residual
    max_i |lam_i - F(lam_{i-1})| of the latest versions is below tol (checked
    here with the oracle's F); the log spans every resumed launch and replays
    to the same state.  One team per slice (lockstep-like schedule)."""
    from oracle import heat

    p = case(name, tol=1e-9)
    with Ctx(p) as c:
        code, st, log, lam = run_async(c, timeout_s=60.0, verify=True, ctas_per_slice=8)
    assert code == pr.PR_OK and st.converged and st.verify_rounds >= 1
    assert st.residual < p["tol"]
    check_log(log, p["N"])
    assert st.events == len(log)
    P = heat.Propagators(p)
    L = lam.reshape((p["N"] + 1,) + tuple(reversed(p["n"])))
    scale = np.max(np.abs(L))
    res = max(np.max(np.abs(L[i] - P.F(L[i - 1]))) for i in range(1, p["N"] + 1))
    assert res < p["tol"] + 1e-13 * scale, res
    rep = async_replay(p, events_of(log))
    assert rel_l2(lam, rep.lam) < FP64_TOL


def test_async_paper_literal_mode():
    p = case("heat2d_explicit", tol=1e-9)
    with Ctx(p) as c:
        code, st, log, lam = run_async(c, timeout_s=60.0, paper_literal=True)
    assert code == pr.PR_OK
    check_log(log, p["N"])
    rep = async_replay(p, events_of(log))
    assert rel_l2(lam, rep.lam) < FP64_TOL


def test_async_wall_clock_limit_returns_timeout_and_context_survives():
    """A run that cannot finish within its limit stops with PR_ETIMEOUT
    (bounded waits, no trap); the context keeps working afterwards."""
    p = case("heat2d_explicit", tol=0.0)
    p["f_steps"] = 512
    with Ctx(p) as c:
        opts = pr.make_async_opts(timeout_s=0.002, quiescence=True)
        lam = c.lam()
        code, st, log = pr.parareal_run_async(c.ctx, opts, lam, log_cap=100000)
        assert code == pr.PR_ETIMEOUT and not st.converged
        lam2 = c.lam()
        code, st = pr.parareal_run_sync(c.ctx, lam2)
        assert st.iterations == p["N"]


def test_async_log_capacity_is_enforced():
    p = case("heat2d_explicit", tol=0.0)
    with Ctx(p) as c:
        opts = pr.make_async_opts(timeout_s=60.0, quiescence=True)
        lam = c.lam()
        code, st, log = pr.parareal_run_async(c.ctx, opts, lam, log_cap=3)
        assert code == pr.PR_ELOGFULL and len(log) == 3


def test_async_rejects_unsupported_problems():
    p = preset("heat1d_thomas", "small")
    with Ctx(p) as c:
        with pytest.raises(pr.PararealError) as e:
            pr.parareal_run_async(c.ctx, pr.make_async_opts(), c.lam(), log_cap=10)
        assert e.value.code == pr.PR_EINVAL


def test_async_single_slice_is_one_fine_solve():
    """N = 1: the only update is lambda_1 = F(u0) (w_new = w_old, no coarse solve)."""
    p = case("heat2d_explicit", tol=1e-9)
    p["N"] = 1
    ref = serial_fine(p)
    with Ctx(p) as c:
        code, st, log, lam = run_async(c, timeout_s=30.0)
    assert code == pr.PR_OK and st.iterations == 1 and len(log) == 1
    assert log[0].vF == 0 and log[0].vG == 0 and log[0].cg_iters == 0
    assert rel_l2(lam, ref) < FP64_TOL


def test_async_one_dimensional_explicit():
    p = case("heat1d_thomas", tol=1e-9)
    p.update(dict(f_scheme="explicit", g_solver="cg", dt=0.3 / 128 ** 2))
    with Ctx(p) as c:
        code, st, log, lam = run_async(c, timeout_s=30.0)
    assert code == pr.PR_OK
    check_log(log, p["N"])
    rep = async_replay(p, events_of(log))
    assert rel_l2(lam, rep.lam) < FP64_TOL
