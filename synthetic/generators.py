"""Seeded input recipes (numpy.random.default_rng).

Array convention used everywhere in this repository: a state on a grid with
interior sizes (nx,), (nx, ny) or (nx, ny, nz) is a C-ordered numpy array of
shape (nx,), (ny, nx) or (nz, ny, nx), so that x is the fastest index once
flattened.  Interior point m (1-based) along an axis with n interior points
sits at coordinate m*h, h = 1/(n+1); the Dirichlet boundary sits at 0 and 1.

Diffusivity fields are given at every node including the boundary ring, i.e.
arrays of shape (n+2,) per axis in the same axis order.
"""
from __future__ import annotations

import numpy as np


def _axis_coords(n: int, ring: bool = False) -> np.ndarray:
    h = 1.0 / (n + 1)
    if ring:
        return np.arange(n + 2, dtype=np.float64) * h
    return np.arange(1, n + 1, dtype=np.float64) * h


def sine_modes_1d(n: int, n_modes: int = 8, seed: int = 1) -> np.ndarray:
    """u0(x) = sum_{j=1..n_modes} a_j sin(j pi x), a_j ~ N(0,1)/j."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(n_modes) / np.arange(1, n_modes + 1)
    x = _axis_coords(n)
    u = np.zeros(n)
    for j in range(1, n_modes + 1):
        u += a[j - 1] * np.sin(j * np.pi * x)
    return u


def modes_and_bumps_2d(nx: int, ny: int | None = None, n_modes: int = 32,
                       max_wavenumber: int = 32, n_bumps: int = 8,
                       width: float = 0.05, seed: int = 2) -> np.ndarray:
    """Sum of random 2D sine modes plus Gaussian bumps.

    Draw order: mode indices j, l ~ U{1..max_wavenumber} (n_modes each),
    amplitudes N(0,1)/sqrt(j^2+l^2); bump centres ~ U[0.2,0.8]^2, bump
    amplitudes N(0,1); bump profile A*exp(-|x-c|^2 / (2 width^2)).
    """
    ny = nx if ny is None else ny
    rng = np.random.default_rng(seed)
    j = rng.integers(1, max_wavenumber + 1, size=n_modes)
    l = rng.integers(1, max_wavenumber + 1, size=n_modes)
    amp = rng.standard_normal(n_modes) / np.sqrt(j.astype(float) ** 2 + l.astype(float) ** 2)
    centres = rng.uniform(0.2, 0.8, size=(n_bumps, 2))
    bump_amp = rng.standard_normal(n_bumps)
    x = _axis_coords(nx)[None, :]
    y = _axis_coords(ny)[:, None]
    u = np.zeros((ny, nx))
    for m in range(n_modes):
        u += amp[m] * np.sin(j[m] * np.pi * x) * np.sin(l[m] * np.pi * y)
    for b in range(n_bumps):
        cx, cy = centres[b]
        u += bump_amp[b] * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * width ** 2))
    return u


def smoothed_noise_3d(shape, sweeps: int = 3, omega: float = 2.0 / 3.0,
                      seed: int = 3) -> np.ndarray:
    """iid N(0,1) field smoothed by damped-Jacobi sweeps with zero boundary.

    Each sweep: u <- u + (omega / (2d)) * (sum of the 2d neighbours - 2d*u),
    neighbours outside the grid read as zero.  Works for any dimension d.
    """
    rng = np.random.default_rng(seed)
    u = rng.standard_normal(tuple(shape))
    d = u.ndim
    for _ in range(sweeps):
        p = np.pad(u, 1)
        nb = np.zeros_like(u)
        for ax in range(d):
            lo = [slice(1, -1)] * d
            hi = [slice(1, -1)] * d
            lo[ax] = slice(0, -2)
            hi[ax] = slice(2, None)
            nb += p[tuple(lo)] + p[tuple(hi)]
        u = u + (omega / (2 * d)) * (nb - 2 * d * u)
    return u


def gaussian_random_field(shape_with_ring, sigma: float = 0.5, corr_len: float = 0.1,
                          seed: int = 40) -> np.ndarray:
    """Gaussian random field with covariance sigma^2 exp(-r^2 / (2 corr_len^2)).

    Synthesis: white noise on a zero-padded box is convolved (FFT) with a
    Gaussian kernel of standard deviation corr_len/sqrt(2), whose
    self-convolution is the requested Gaussian covariance; the box is padded
    by 4*corr_len per side so the periodic wrap does not correlate opposite
    faces.  The cropped field is rescaled to sample mean 0 and sample
    standard deviation sigma.  Node spacing h = 1/(n_ring-1) per axis.
    """
    shape = tuple(int(s) for s in shape_with_ring)
    rng = np.random.default_rng(seed)
    hs = [1.0 / (s - 1) for s in shape]
    pads = [int(np.ceil(4 * corr_len / h)) for h in hs]
    big = tuple(s + 2 * p for s, p in zip(shape, pads))
    w = rng.standard_normal(big)
    s_k = corr_len / np.sqrt(2.0)
    W = np.fft.fftn(w)
    # Fourier transform of the unit-mass Gaussian kernel exp(-x^2/(2 s_k^2))
    K = np.ones(big)
    for ax, (m, h) in enumerate(zip(big, hs)):
        f = np.fft.fftfreq(m, d=h)
        kk = np.exp(-2.0 * (np.pi * f * s_k) ** 2)
        shp = [1] * len(big)
        shp[ax] = m
        K = K * kk.reshape(shp)
    g = np.real(np.fft.ifftn(W * K))
    crop = tuple(slice(p, p + s) for p, s in zip(pads, shape))
    g = g[crop]
    g = g - g.mean()
    g = g * (sigma / g.std())
    return g


def lognormal_kappa(n_interior, sigma: float = 0.5, corr_len: float = 0.1,
                    seed: int = 40) -> np.ndarray:
    """kappa = exp(g) at every node including the boundary ring.

    n_interior is (nx,), (nx, ny) or (nx, ny, nz); the returned array has
    shape (n+2) per axis in (z, y, x) order.
    """
    ring = tuple(int(n) + 2 for n in reversed(tuple(n_interior)))
    return np.exp(gaussian_random_field(ring, sigma, corr_len, seed))


def delay_table(n_slices: int, max_events: int, low: int = 0, high: int = 4,
                seed: int = 51) -> np.ndarray:
    """Per-(slice, event) publish delays, integers in [low, high] (fine-step units).

    Row i-1 belongs to slice i; column e to that slice's e-th update.
    """
    rng = np.random.default_rng(seed)
    return rng.integers(low, high + 1, size=(n_slices, max_events)).astype(np.int32)


def random_directions(shape, count: int, seed: int = 42) -> np.ndarray:
    """count iid N(0,1) directions of the given shape (finite-difference probes)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((count,) + tuple(shape))
