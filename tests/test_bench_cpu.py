"""Host-side pieces of bench.py that need no GPU: the §4.1 cost model."""
import types

import bench


def test_cost_model_recovers_the_overhead_of_eq_pr_cost():
    """Build a solve time from Eq. (pr_cost) with a constant overhead C_bar per
    processor and iteration (its double sum written out), and recover C_bar."""
    p, k, C_F, C_G, C_bar = 8, 3, 10.0, 1.0, 0.5
    overhead = sum(C_bar for l in range(1, k + 1) for j in range(l + 1, p))
    T = p * C_G + k * (C_F + C_G) + overhead
    st = {"iterations": k, "coarse_solves": 20, "t_fine_ms": k * C_F, "t_coarse_ms": 20 * C_G}
    cm = bench.cost_model_sync({"N": p}, st, T)
    assert abs(cm["C_F_ms"] - C_F) < 1e-12 and abs(cm["C_G_ms"] - C_G) < 1e-12
    assert abs(cm["aubanel_ms"] - (p * C_G + k * (C_F + C_G))) < 1e-12
    assert abs(cm["C_bar_ms"] - C_bar) < 1e-12


def test_async_cost_model_reads_the_log():
    ev = lambda i, k, vF, vG, t0, t1: types.SimpleNamespace(slice=i, version=k, vF=vF, vG=vG,
                                                          t_start=t0, t_end=t1)
    log = [ev(1, 1, 0, 0, 0, 4_000_000), ev(2, 1, 0, 1, 0, 5_000_000),
           ev(2, 2, 1, 1, 5_000_000, 9_000_000)]
    cm = bench.cost_model_async(log, 2, 9.0)
    assert cm["kappa"] == 2 and cm["updates"] == 3
    assert cm["update_F_ms"] == 4.0 and cm["update_FG_ms"] == 5.0
    assert cm["n_F_only"] == 2 and cm["n_FG"] == 1
    both = bench.cost_models(log, 2, 9.0, {"N": 2},
                             {"iterations": 1, "coarse_solves": 3, "t_fine_ms": 4.0,
                              "t_coarse_ms": 3.0}, 8.0)
    assert both["async"]["prop3_ms"] == bench.apr_cost(2, 2, 4.0, 1.0) == 12.0
    assert both["sync"]["C_F_ms"] == 4.0 and both["sync"]["C_G_ms"] == 1.0


def test_sync_delay_sums_the_updated_slices():
    import numpy as np
    table = np.arange(12).reshape(3, 4)       # slices 1..3, 4 columns
    # k = 2: iteration 0 updates slices 1..3 (column 0), iteration 1 slices 2..3 (column 1)
    units = (0 + 4 + 8) + (5 + 9)
    assert abs(bench.sync_delay_ms(table, 1e6, 2, 3) - units) < 1e-12


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` times the oracle on the host and prints one JSON
    line with the keys of the benchmark contract."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "3", "--grid", "96,80", "--slices", "4",
                          "--workload", "heat2d_explicit"], capture_output=True, text=True,
                         check=True, timeout=600, cwd=root).stdout.strip().splitlines()
    lines = [ln for ln in out if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] == os.cpu_count()          # every host core
    for key in ("grid", "N", "f_steps", "tol", "g_rtol"):           # the GPU line's config keys
        assert key in d["config"], key
    assert d["config"]["grid"] == [96, 80] and d["config"]["N"] == 4
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_proposition3_reproduces_the_papers_table1_estimates():
    """The bench's Proposition 3 (C~ = p C_G + kappa (C_F + C_G)) with the paper's
    C_G = 0.14 s and C_F = 100 C_G gives Table 1's printed estimates: within
    0.1% for five rows, 1.4% for p = 16 (whose kappa is a rounded average)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_async_cost.txt")
    rows = [ln.split() for ln in open(path) if ln[0].isdigit()]
    assert len(rows) == 6
    C_G = 0.14
    for p, kappa, printed in rows:
        est = bench.apr_cost(int(p), int(kappa), 100 * C_G, C_G)
        tol = 0.015 if p == "16" else 0.001
        assert abs(est - float(printed)) <= tol * float(printed), (p, est, printed)


def test_oracle_time_to_tol_extrapolation_counts_the_work():
    """The extrapolated oracle time: the fine phase of iteration j spreads the
    N - j active slices over the cores; the coarse CG iterations run in sequence."""
    p = {"N": 10, "f_steps": 4}
    # k = 2: ceil(10/4) + ceil(9/4) = 3 + 3 rounds of 4 steps at 0.5 s, plus 7 CG x 2 s
    t = bench.oracle_time_to_tol_s(p, 0.5, 2.0, 4, 2, 7)
    assert abs(t - (6 * 4 * 0.5 + 14.0)) < 1e-12


def test_pcg_pass_costs_add_up():
    """The per-point bytes of the preconditioned CG's passes: 16 m + 68 per iteration
    (m - 1 Chebyshev passes, the direction pass and the solution/residual pass) and 60
    per solve; the FP64 instruction count per iteration is the direction pass's
    operator (6 in 3D, 4 in 2D) plus 3, the residual pass's 3 and the last
    Chebyshev step's r.z."""
    for dim, op in ((3, 6), (2, 4)):
        for m in (4, 12, 16):
            it, solve, first_dir = bench.pcg_pass_costs(dim, m)
            assert len(it) == m + 1                       # m - 1 Chebyshev + 2 CG passes
            assert sum(b for b, _ in it) == 16 * m + 68
            assert sum(b for b, _ in solve) + first_dir[0] - it[-2][0] == 60
            assert sum(f for _, f in it) == op + 3 + 3 + 1


def test_pcg_roofline_bound_is_the_sum_of_pass_maxima():
    """With an FP64 peak so high that no pass is FP64-bound, the bound is the HBM
    time of the algorithmic bytes; with a low one the direction pass dominates."""
    M, m, its, solves = 1000, 12, 7, 3
    r = bench.pcg_roofline(M, 3, m, its, solves, 1.0, 1000.0, "measured", 1e9)
    gbytes = M * (its * (16 * m + 68) + solves * 60)
    assert abs(r["t_bound_ms"] - gbytes / 1000e9 * 1e3) < 1e-12
    assert abs(r["achieved"] - gbytes / 1e-3 / 1e9) < 1e-6
    slow = bench.pcg_roofline(M, 3, m, its, solves, 1.0, 1000.0, "measured", 1e-3)
    assert slow["t_bound_ms"] > r["t_bound_ms"]
    assert abs(slow["frac_of_pass_roofline"] - slow["t_bound_ms"] / 1.0) < 1e-12
