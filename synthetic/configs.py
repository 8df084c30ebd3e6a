"""Problem presets: sizes, step counts and tolerances of the five heat workloads.

Each preset returns a plain dict.  `scale` selects the full-size workload
("full") or a reduced variant with the same recipe ("small", "tiny") for
parity tests.  The fine step dt follows the workload's rule; for variable
diffusivity dt = 0.8 h^2 / (2 d max(kappa)), a Gershgorin-stable choice.
"""
from __future__ import annotations

import numpy as np

from . import generators as gen

# name: (dim, full sizes, N, n_f, ...).  Sizes are interior points per axis.
PRESETS = {
    "heat1d_thomas": dict(dim=1, n=(1023,), N=16, f_steps=100, f_scheme="implicit",
                          g_solver="thomas", T=0.1, tol=1e-10, g_rtol=0.0, f_prec=64,
                          small=dict(n=(127,), N=8, f_steps=20),
                          tiny=dict(n=(15,), N=4, f_steps=5)),
    # coarse CG preconditioned by 16 FP32 Chebyshev steps at full size (1.35x on the
    # solve, measured); the reduced parity variants run plain CG
    "heat2d_explicit": dict(dim=2, n=(1024, 1024), N=64, f_steps=256, f_scheme="explicit",
                            g_solver="cg", dt_h2=0.2, tol=1e-10, g_rtol=1e-10, f_prec=64,
                            g_cheb=16,
                            small=dict(n=(70, 61), N=8, f_steps=32, g_cheb=0),
                            tiny=dict(n=(6, 5), N=4, f_steps=4, g_cheb=0)),
    # coarse CG tolerance 1e-7: the FP32 fine steps' rounding noise floor (the workload
    # names no CG tolerance; the same setting serves the FP64 comparison arm); the
    # coarse CG is preconditioned by 12 FP32 Chebyshev steps at full size (the reduced
    # parity variants run plain CG; the preconditioner has parity cases of its own)
    "heat3d_mixed": dict(dim=3, n=(256, 256, 256), N=128, f_steps=64, f_scheme="explicit",
                         g_solver="cg", dt_h2=0.15, tol=1e-5, g_rtol=1e-7, f_prec=32,
                         g_cheb=12,
                         small=dict(n=(37, 30, 26), N=6, f_steps=16, g_cheb=0),
                         tiny=dict(n=(4, 3, 3), N=3, f_steps=3, g_cheb=0)),
    "heat2d_inverse": dict(dim=2, n=(512, 512), N=32, f_steps=128, f_scheme="explicit",
                           g_solver="cg", kappa_seed=40, kappa_star_seed=41, tol=0.0,
                           g_rtol=1e-13, K=6, f_prec=64,
                           small=dict(n=(40, 33), N=6, f_steps=24, K=3),
                           tiny=dict(n=(5, 4), N=3, f_steps=4, K=2)),
    "heat3d_varkappa_async": dict(dim=3, n=(192, 192, 192), N=256, f_steps=32,
                                  f_scheme="explicit", g_solver="cg", kappa_seed=5,
                                  tol=1e-5, g_rtol=1e-10, f_prec=32, delay_seed=51,
                                  small=dict(n=(29, 24, 21), N=8, f_steps=8),
                                  tiny=dict(n=(4, 3, 3), N=3, f_steps=3)),
    # trapezoidal-rule F as in Table 1 (dT / dt = 100, eps = 1e-6), steps of 4 h^2
    "heat2d_cn": dict(dim=2, n=(512, 512), N=32, f_steps=100, f_scheme="cn", g_solver="cg",
                      dt_h2=4.0, tol=1e-6, g_rtol=1e-10, f_rtol=1e-12, f_prec=64,
                      small=dict(n=(48, 40), N=6, f_steps=10),
                      tiny=dict(n=(6, 5), N=4, f_steps=3)),
}

_U0_SEEDS = {"heat1d_thomas": 1, "heat2d_explicit": 2, "heat3d_mixed": 3,
             "heat2d_inverse": 4, "heat3d_varkappa_async": 50, "heat2d_cn": 6}


def _u0(name: str, n) -> np.ndarray:
    seed = _U0_SEEDS[name]
    if name == "heat1d_thomas":
        return gen.sine_modes_1d(n[0], 8, seed)
    if name in ("heat2d_explicit", "heat2d_inverse", "heat2d_cn"):
        return gen.modes_and_bumps_2d(n[0], n[1], seed=seed)
    # 3D families: smoothed noise, shape (nz, ny, nx)
    return gen.smoothed_noise_3d((n[2], n[1], n[0]), seed=seed)


def preset(name: str, scale: str = "full", **override) -> dict:
    """Return the problem dict (sizes, steps, dt, T, u0, kappa) for a workload.

    `override` replaces recipe entries (e.g. n, N, f_steps) before the inputs
    are generated, for profiling the same recipe at another size."""
    base = dict(PRESETS[name])
    small = base.pop("small")
    tiny = base.pop("tiny")
    if scale == "small":
        base.update(small)
    elif scale == "tiny":
        base.update(tiny)
    elif scale != "full":
        raise ValueError(scale)
    base.update(override)
    dim = base["dim"]
    n = tuple(base["n"])
    h = [1.0 / (m + 1) for m in n]
    kappa = None
    if "kappa_seed" in base:
        kappa = gen.lognormal_kappa(n, seed=base["kappa_seed"])
    if "kappa_star_seed" in base:
        base["kappa_star"] = gen.lognormal_kappa(n, seed=base["kappa_star_seed"])
    if "T" in base:
        dt = base["T"] / (base["N"] * base["f_steps"])
    elif kappa is None:
        dt = base["dt_h2"] * min(h) ** 2
    else:
        kmax = float(kappa.max())
        if "kappa_star" in base:
            kmax = max(kmax, float(base["kappa_star"].max()))
        dt = 0.8 * min(h) ** 2 / (2 * dim * kmax)
    base["dt"] = dt
    base["T"] = base["N"] * base["f_steps"] * dt
    base["h"] = tuple(h)
    base["u0"] = _u0(name, n)
    base["kappa"] = kappa
    base["name"] = name
    base["scale"] = scale
    return base
