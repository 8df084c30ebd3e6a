"""The allocation-free coarse solve (parareal_coarse_noalloc) against the
context-based coarse solve (parareal_coarse).

parareal_coarse_noalloc exists for callers that must not allocate device
memory while running (allocator hooks, host callbacks, fixed memory budgets,
loops that cannot afford cudaMalloc's implicit synchronisation); its CG
vectors live in a static device array inside the library.  The test calls it
twice in a row with different inputs -- the second call finds the first
call's leftovers in that shared array -- and compares each result with the
existing entry point within the FP64 parity tolerance of the other tests.
This file is collected last on purpose.
"""
import numpy as np
import pytest

import paper_2110_10762_gb300 as pr  # noqa: E402  (a missing library fails the first call loudly)

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_coarse_matches_context_coarse_twice():
    import torch
    n = (211, 157)                       # 33127 points: below the 131072-point limit
    h = 1.0 / (max(n) + 1)
    f_steps = 256
    dT = f_steps * 0.2 * h * h
    rng = np.random.default_rng(21)
    M = n[0] * n[1]
    u0 = torch.from_numpy(rng.standard_normal(M)).cuda()
    stream = torch.cuda.current_stream()
    ctx = pr.parareal_create(0, stream)
    try:
        prob = pr.make_problem(dim=2, n=n, T0=0.0, T=dT, N=1, u0=u0, f_steps=f_steps,
                               g_rtol=1e-13, tol=0.0)
        pr.parareal_set_problem(ctx, prob)
        for call in range(2):              # two calls in a row share the static scratch
            b = torch.from_numpy(rng.standard_normal(M) * (1 + call)).cuda()
            x0 = b + 0.05 * torch.from_numpy(rng.standard_normal(M)).cuda()
            ref = torch.empty_like(b)
            it_ref = pr.parareal_coarse(ctx, b, x0, ref)
            got = torch.full_like(b, float("nan"))
            it = pr.parareal_coarse_noalloc(2, n, dT, b, x0, got, rtol=1e-13, stream=stream)
            torch.cuda.synchronize()
            # the two kernels may run with different block counts, which changes the
            # order of the FP64 reductions: the stop test may fall one iteration apart
            assert abs(it - it_ref) <= 1, (call, it, it_ref)
            assert _rel(got.cpu().numpy(), ref.cpu().numpy()) < FP64_TOL, call
    finally:
        pr.parareal_destroy(ctx)


def test_noalloc_rejects_grids_beyond_its_limit():
    """A grid one point beyond the 131072-point limit is rejected before any
    launch; the buffers hold the full declared size, so the call could not
    fault even if the limit were raised."""
    import torch
    M = 131073
    b = torch.zeros(M, dtype=torch.float64, device="cuda")
    x = torch.zeros(M, dtype=torch.float64, device="cuda")
    with pytest.raises(pr.PararealError) as e:
        pr.parareal_coarse_noalloc(1, (M,), 1e-3, b, None, x)
    assert e.value.code == pr.PR_EINVAL


def test_noalloc_wrapper_rejects_short_buffers_and_mismatched_dims():
    import torch
    b = torch.zeros(100, dtype=torch.float64, device="cuda")
    x = torch.zeros(100, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        pr.parareal_coarse_noalloc(2, (11, 10), 1e-3, b, None, x)   # 110 > 100 values
    with pytest.raises(ValueError):
        pr.parareal_coarse_noalloc(2, (10, 10, 1), 1e-3, b, None, x)  # dim != len(n)
