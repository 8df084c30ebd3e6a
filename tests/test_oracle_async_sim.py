"""Pins of the oracle's discrete-event simulation of asynchronous Parareal.

The expected logs below are derived by hand from the rules of Algorithm 2
(§4.1) on a virtual clock (F costs f_cost units, G costs c_G units, a version
becomes visible after its publication delay); the states are pinned by the
finite-time termination (§3.2), the per-mode contraction of one asynchronous
update (§3.2, the error bound of Eq. (12)) and by the special case that
reduces to Algorithm 1.
"""
import numpy as np
import pytest
import scipy.fft

from oracle.async_sim import async_simulate
from oracle.parareal import async_replay, serial_fine, sync_parareal
from tests.test_oracle_pins import grid_mu, small_prob


def _log(res):
    return [(e.i, e.k, e.vF, e.vG, e.worker, e.t_start, e.t_end, e.t_vis) for e in res.events]


def test_two_slices_no_delay_hand_derived():
    """N = 2, one worker per slice, F = 4 units, G = 1 unit, no delays.
    t=0: both slices start F from the predictor (vF = 0).
    t=4: slice 1 has no newer input (slice 0 is u0): publishes F(u0).
         slice 2 now sees version 1 of slice 1: G costs 1, publishes at 5.
    t=5: slice 2 re-runs F on version 1 (its coarse input), nothing newer at
         t=9, publishes F(lambda_1^1) without a solve: every slice settled."""
    prob = small_prob(1, (9,), N=2, f_steps=4, dt_h2=1.0, f_scheme="implicit")
    res = async_simulate(prob, c_G=1.0, tol=0.0)
    assert _log(res) == [(1, 1, 0, 0, 0, 0, 4, 4), (2, 1, 0, 1, 1, 0, 5, 5),
                         (2, 2, 1, 1, 1, 5, 9, 9)]
    assert res.stop_reason == "quiescent" and res.t_stop == 9 and res.kappa == 2
    ref = serial_fine(prob)
    np.testing.assert_allclose(res.lam, ref, rtol=0, atol=1e-14 * np.max(np.abs(ref)))


def test_two_slices_with_delay_hand_derived():
    """Slice 1's versions become visible 3 units after publication.
    t=4: slice 1 publishes (visible at 7); slice 2 sees nothing new and
         publishes F(lambda_1^0) without a solve, then idles.
    t=7: slice 2 wakes (version 1 visible), F on its held input (version 0)
         until 11, G on version 1 until 12, publishes.
    t=12: F on version 1 until 16, publishes: quiescent."""
    prob = small_prob(1, (9,), N=2, f_steps=4, dt_h2=1.0, f_scheme="implicit")
    res = async_simulate(prob, c_G=1.0, tol=0.0, delays=[[3.0], [0.0]])
    assert _log(res) == [(1, 1, 0, 0, 0, 0, 4, 7), (2, 1, 0, 0, 1, 0, 4, 4),
                         (2, 2, 0, 1, 1, 7, 12, 12), (2, 3, 1, 1, 1, 12, 16, 16)]
    assert res.t_stop == 16 and res.kappa == 3
    ref = serial_fine(prob)
    np.testing.assert_allclose(res.lam, ref, rtol=0, atol=1e-14 * np.max(np.abs(ref)))


def test_one_worker_round_robin_hand_derived():
    """One worker owns both slices and visits them in turn.
    t=0..4 slice 1 (publishes F(u0)); t=4..8 F of slice 2 on version 0, then
    G on version 1 until 9; t=9 slice 1 idle, slice 2 F on version 1 until 13."""
    prob = small_prob(1, (9,), N=2, f_steps=4, dt_h2=1.0, f_scheme="implicit")
    res = async_simulate(prob, workers=1, c_G=1.0, tol=0.0)
    assert _log(res) == [(1, 1, 0, 0, 0, 0, 4, 4), (2, 1, 0, 1, 0, 4, 9, 9),
                         (2, 2, 1, 1, 0, 9, 13, 13)]


def test_no_cost_no_delay_reduces_to_algorithm_1():
    """With G free, equal F costs and no delays every slice reads its
    predecessor's version of the same instant, so version k of slice i is the
    synchronous iterate lambda_i^k (Algorithm 1 with its frozen prefix), bit
    for bit, and the run ends at quiescence with kappa = N."""
    prob = small_prob(2, (7, 6), N=5, f_steps=5, g_rtol=1e-9)
    res = async_simulate(prob, c_G=0.0, f_cost=1.0, tol=0.0)
    syn = sync_parareal(prob, tol=0.0, max_iter=prob["N"], record=True)
    assert res.kappa == prob["N"]
    for i in range(1, prob["N"] + 1):
        assert res.k_i[i - 1] == i
        for k in range(0, i + 1):
            np.testing.assert_array_equal(res.versions[(i, k)], syn.iterates[k][i])


@pytest.mark.parametrize("workers", [1, 2, 5])
def test_random_delays_reach_serial_fine_at_quiescence(workers):
    """Finite-time termination of the asynchronous iteration (§3.2): at
    quiescence lambda_i = F(lambda_{i-1}) for all i, i.e. the serial fine
    solution, whatever the delays, the owners and an inexact coarse solve."""
    prob = small_prob(2, (6, 5), N=5, f_steps=6, g_rtol=1e-6)
    rng = np.random.default_rng(11)
    delays = rng.integers(0, 5, size=(prob["N"], 7)).astype(float)
    res = async_simulate(prob, workers=workers, c_G=2.0, delays=delays, tol=0.0)
    assert res.stop_reason == "quiescent"
    ref = serial_fine(prob)
    np.testing.assert_allclose(res.lam, ref, rtol=0, atol=1e-13 * np.max(np.abs(ref)))
    # the log is a valid asynchronous schedule: the replay accepts it and
    # recomputes the same states bit for bit
    rep = async_replay(prob, res.events)
    np.testing.assert_array_equal(rep.lam, res.lam)


def test_per_event_contraction_per_mode():
    """Each simulated update obeys the per-mode bound of one asynchronous
    Parareal update: |e_new| <= (|g| + |f - g|) max(|e(x_G)|, |e(x_F)|)."""
    prob = small_prob(1, (19,), N=6, f_steps=10, dt_h2=1.0, f_scheme="implicit")
    mu = grid_mu(prob["n"], prob["h"])
    f = (1 + prob["dt"] * mu) ** (-prob["f_steps"])
    g = 1.0 / (1 + prob["f_steps"] * prob["dt"] * mu)
    alpha = np.abs(g) + np.abs(f - g)
    delays = np.random.default_rng(3).integers(0, 25, size=(prob["N"], 5)).astype(float)
    res = async_simulate(prob, workers=3, c_G=3.0, delays=delays, tol=0.0)
    ref = serial_fine(prob)

    def err(i, v):
        return np.abs(scipy.fft.dst(res.versions[(i, v)] - ref[i], type=1))

    scale = np.max(np.abs(scipy.fft.dst(ref, type=1, axis=1)))
    assert len(res.events) > prob["N"]
    for e in res.events:
        lhs = err(e.i, e.k)
        rhs = alpha * np.maximum(err(e.i - 1, e.vF), err(e.i - 1, e.vG))
        assert np.all(lhs <= rhs + 1e-12 * scale)


def test_tolerance_stop_rule():
    """The run stops at the first publication after which every slice has
    updated and is settled or had its last increment below tol; the updates
    in flight at that instant still publish."""
    prob = small_prob(1, (15,), N=12, f_steps=10, dt_h2=4.0, f_scheme="implicit")
    tol = 1e-6
    res = async_simulate(prob, c_G=2.0, tol=tol)
    assert res.stop_reason == "tol"
    N = prob["N"]

    def holds(prefix):
        last, latest = {}, {0: 0}
        for e in prefix:
            last[e.i] = e
            latest[e.i] = e.k
        if sorted(last) != list(range(1, N + 1)):
            return False
        return all((e.vF == e.vG == latest.get(i - 1, 0)) or e.delta < tol
                   for i, e in last.items())

    n_stop = res.n_at_stop
    assert holds(res.events[:n_stop])
    assert not any(holds(res.events[:n]) for n in range(1, n_stop))
    assert all(e.t_start < res.t_stop for e in res.events[n_stop:])
    ref = serial_fine(prob)
    assert np.max(np.abs(res.lam - ref)) < 1e-5 * np.max(np.abs(ref))


def test_paper_literal_repeats_idempotent_updates():
    """Paper-literal mode repeats the loop of Algorithm 2 unconditionally:
    slice 1 re-publishes F(u0) every f_cost units, identical bit for bit."""
    prob = small_prob(1, (9,), N=3, f_steps=4, dt_h2=1.0, f_scheme="implicit")
    res = async_simulate(prob, c_G=1.0, tol=1e-8, paper_literal=True, max_updates=200)
    s1 = [e for e in res.events if e.i == 1]
    assert [e.t_end for e in s1[:4]] == [4, 8, 12, 16]
    assert all(e.vF == e.vG == 0 for e in s1)
    for e in s1[1:]:
        assert e.delta == 0.0
        np.testing.assert_array_equal(res.versions[(1, e.k)], res.versions[(1, 1)])
    assert res.stop_reason == "tol"


def test_rejects_bad_arguments():
    prob = small_prob(1, (5,), N=2, f_steps=2, dt_h2=1.0, f_scheme="implicit")
    with pytest.raises(ValueError):
        async_simulate(prob, c_G=-1.0)
    with pytest.raises(ValueError):
        async_simulate(prob, delays=np.zeros((3, 2)))


def test_verified_stop_closes_the_increment_gap():
    """A delay-free lockstep schedule (one worker per slice) on a slowly
    contracting problem: the per-slice increment rule stops while the state is
    still far from the fixed point (error 100x tol); with the residual check the
    run resumes until max_i |lambda_i - F(lambda_{i-1})| < tol, and the error
    falls to the order of tol."""
    prob = small_prob(1, (31,), N=32, f_steps=20, dt_h2=1.0, f_scheme="implicit")
    tol = 1e-6
    ref = serial_fine(prob)
    scale = np.max(np.abs(ref))
    plain = async_simulate(prob, c_G=0.2, tol=tol)
    assert plain.stop_reason == "tol"
    assert np.max(np.abs(plain.lam - ref)) > 10 * tol * scale
    checked = async_simulate(prob, c_G=0.2, tol=tol, verify=True)
    assert checked.verify_rounds >= 2 and checked.residual < tol
    P = __import__("oracle.heat", fromlist=["Propagators"]).Propagators(prob)
    res = max(np.max(np.abs(checked.lam[i] - P.F(checked.lam[i - 1])))
              for i in range(1, prob["N"] + 1))
    assert res == checked.residual
    assert np.max(np.abs(checked.lam - ref)) < tol * scale
    # the resumed run is still one valid asynchronous schedule
    rep = async_replay(prob, checked.events)
    np.testing.assert_array_equal(rep.lam, checked.lam)
