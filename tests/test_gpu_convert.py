"""The integer-pipe FP32 <-> FP64 conversions of the coarse solver's vectorised
passes against the hardware conversions (torch's casts), bit for bit: random
encodings over every exponent, values exactly halfway between two binary32
neighbours (ties to even), the subnormal range and the overflow edge.  NaN
inputs only have to stay NaN (payloads may differ)."""
import numpy as np
import pytest

import paper_2110_10762_gb300 as pr

pytestmark = pytest.mark.gpu


def _f32_cases(rng):
    rand = rng.integers(0, 2**32, size=1 << 21, dtype=np.uint64).astype(np.uint32)
    special = np.array([0, 0x80000000, 1, 0x80000001, 0x007FFFFF, 0x807FFFFF, 0x00800000,
                        0x00400000, 0x7F7FFFFF, 0xFF7FFFFF, 0x7F800000, 0xFF800000, 0x7FC00000,
                        0x3F800000, 0xBF800000, 0x3EAAAAAB], dtype=np.uint32)
    # every subnormal leading-bit position
    sub = np.array([1 << k for k in range(23)] + [(1 << k) | 1 for k in range(1, 23)], dtype=np.uint32)
    return np.concatenate([special, sub, sub | np.uint32(0x80000000), rand]).view(np.float32)


def _f64_cases(rng):
    n = 1 << 20
    sign = rng.integers(0, 2, size=n, dtype=np.uint64) << np.uint64(63)
    mant = rng.integers(0, 2**52, size=n, dtype=np.uint64)
    # exponents: the whole range, and concentrated on binary32's normal and subnormal ranges
    e_all = rng.integers(0, 2048, size=n, dtype=np.uint64)
    e_f32 = rng.integers(860, 1160, size=n, dtype=np.uint64)
    d_all = sign | (e_all << np.uint64(52)) | mant
    d_f32 = sign | (e_f32 << np.uint64(52)) | mant
    # ties: the 29 dropped significand bits exactly one half (both parities of the kept bits),
    # and one unit either side of the tie
    half = np.uint64(1 << 28)
    kept = mant & ~np.uint64((1 << 29) - 1)
    tie = sign | (e_f32 << np.uint64(52)) | kept | half
    near = np.concatenate([tie - np.uint64(1), tie + np.uint64(1)])
    # largest binary32 and the values that round up to infinity or stay finite
    edge = np.array([0x47EFFFFFE0000000, 0x47EFFFFFEFFFFFFF, 0x47EFFFFFF0000000, 0x47F0000000000000,
                     0x36A0000000000000, 0x3690000000000000, 0x3690000000000001, 0x36A8000000000000,
                     0x3810000000000000, 0x380FFFFFF0000000, 0x380FFFFFE8000000, 0,
                     0x8000000000000000, 1, 0x7FF0000000000000, 0x7FF8000000000000],
                    dtype=np.uint64)
    return np.concatenate([edge, d_all, d_f32, tie, near]).view(np.float64)


def test_integer_pipe_conversions_equal_hardware_conversions():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(20211020)
    f32, f64 = _f32_cases(rng), _f64_cases(rng)
    f32 = np.resize(f32, f64.size)   # repeated to the length of the FP64 cases
    f_in = torch.from_numpy(f32).cuda()
    d_in = torch.from_numpy(f64).cuda()
    d_out, f_out = pr.parareal_probe_convert(f_in, d_in)
    torch.cuda.synchronize()
    ref_d = f_in.double()
    ref_f = d_in.float()
    nan_d = torch.isnan(ref_d)
    assert torch.equal(torch.isnan(d_out), nan_d)
    assert torch.equal(d_out[~nan_d].view(torch.int64), ref_d[~nan_d].view(torch.int64))
    nan_f = torch.isnan(ref_f)
    assert torch.equal(torch.isnan(f_out), nan_f)
    bad = (f_out[~nan_f].view(torch.int32) != ref_f[~nan_f].view(torch.int32)).nonzero()
    assert bad.numel() == 0, d_in[~nan_f][bad[:8, 0]].cpu().numpy().view(np.uint64)


def test_probe_convert_rejects_bad_arguments():
    lib = pr._abi.load()
    assert lib.parareal_probe_convert(None, None, None, None, -1, None) == pr.PR_EINVAL
    assert lib.parareal_probe_convert(None, None, None, None, 4, None) == pr.PR_EINVAL
    assert lib.parareal_probe_convert(None, None, None, None, 0, None) == pr.PR_OK
