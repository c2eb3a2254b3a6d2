"""The rollout's own FP32 elementary functions (sin/cos by Cody-Waite
reduction and Taylor series, atan2 by octant reduction and a fitted
polynomial, the MUFU reciprocal and reciprocal square root) against CUDA's
library functions and an
FP64 reference, and the packed two-wide FP32 operations against their scalar
forms, on the GPU through atp_math_check."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def run(a, b):
    from paper_2603_20525_gb300 import atp
    L = atp.load()
    ad = torch.as_tensor(np.asarray(a, np.float32)).cuda()
    bd = torch.as_tensor(np.asarray(b, np.float32)).cuda()
    out = torch.empty((len(a), 14), dtype=torch.float32, device="cuda")
    assert L.atp_math_check(C.c_void_p(ad.data_ptr()), C.c_void_p(bd.data_ptr()), len(a),
                            C.c_void_p(out.data_ptr()), None) == 0
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def test_sincos_against_cuda_and_fp64():
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.uniform(-0.8, 0.8, 200000), rng.uniform(-60, 60, 200000),
                        [0.0, -0.0, 0.785398163, -0.785398163, 1e-30, 3.14159265]]).astype(np.float32)
    o = run(a, np.ones_like(a))
    x = a.astype(np.float64)
    es = np.abs(o[:, 0] - np.sin(x)).max()
    ec = np.abs(o[:, 1] - np.cos(x)).max()
    es_ref = np.abs(o[:, 2] - np.sin(x)).max()
    ec_ref = np.abs(o[:, 3] - np.cos(x)).max()
    print("sin/cos max abs error: library", es, ec, "CUDA", es_ref, ec_ref)
    assert es <= 1.2e-7 and ec <= 1.2e-7
    assert es <= 2.5 * es_ref and ec <= 2.5 * ec_ref


def test_sincos_special_arguments():
    """NaN comes out NaN from the library's reduction, infinities and
    arguments from 2^17 up are CUDA's sincosf bit for bit, and the largest
    argument the reduction takes still meets its bound."""
    big = np.array([131072.0, -131072.0, 1e6, -3.5e7, 3e38, np.inf, -np.inf], np.float32)
    edge = np.array([np.nextafter(np.float32(131072.0), np.float32(0)), -100000.0], np.float32)
    a = np.concatenate([[np.nan, -np.nan], big, edge]).astype(np.float32)
    o = run(a, np.ones_like(a))
    assert np.all(np.isnan(o[:2, :2]))
    nb = 2 + len(big)
    assert np.array_equal(o[2:nb, 0], o[2:nb, 2], equal_nan=True)
    assert np.array_equal(o[2:nb, 1], o[2:nb, 3], equal_nan=True)
    assert np.all(np.isnan(o[nb - 2:nb, :2]))
    x = a[nb:].astype(np.float64)
    assert np.abs(o[nb:, 0] - np.sin(x)).max() <= 2e-6
    assert np.abs(o[nb:, 1] - np.cos(x)).max() <= 2e-6


def test_atan2_against_cuda_and_fp64():
    rng = np.random.default_rng(1)
    n = 300000
    mag = 10.0 ** rng.uniform(-4, 2, n)
    ang = rng.uniform(-np.pi, np.pi, n)
    y = (mag * np.sin(ang)).astype(np.float32)
    x = (mag * np.cos(ang)).astype(np.float32)
    # the common case: a wheel rolling forward, small slip
    y2 = rng.normal(0, 0.5, n).astype(np.float32)
    x2 = rng.uniform(2, 16, n).astype(np.float32)
    y = np.concatenate([y, y2, [0.0, 0.0, 1.0, -1.0]]).astype(np.float32)
    x = np.concatenate([x, x2, [0.0, 1.0, 0.0, 0.0]]).astype(np.float32)
    o = run(y, x)
    ref = np.arctan2(y.astype(np.float64), x.astype(np.float64))
    err = np.abs(o[:, 4] - ref)
    err_ref = np.abs(o[:, 5] - ref)
    tol = 2.5e-7 * np.abs(ref) + 1e-12
    print("atan2 max rel error: library", (err / np.maximum(np.abs(ref), 1e-30)).max(),
          "CUDA", (err_ref / np.maximum(np.abs(ref), 1e-30)).max())
    assert np.all(err <= np.maximum(tol, 4e-7))
    assert o[-4, 4] == 0.0 and o[-3, 4] == 0.0


def test_reciprocal_within_one_ulp():
    rng = np.random.default_rng(2)
    b = np.concatenate([rng.uniform(0.2, 1.5, 100000), -rng.uniform(0.2, 1.5, 100000),
                        10.0 ** rng.uniform(-10, 10, 100000)]).astype(np.float32)
    o = run(np.zeros_like(b), b)
    ref = 1.0 / b.astype(np.float64)
    rel = np.abs(o[:, 6] - ref) / np.abs(ref)
    assert rel.max() <= 1.2e-7
    assert np.array_equal(o[:, 7], (np.float32(1.0) / b).astype(np.float64))


def test_reciprocal_sqrt_within_two_ulp():
    rng = np.random.default_rng(3)
    b = np.concatenate([rng.uniform(0.36, 40.0, 200000), 10.0 ** rng.uniform(-30, 30, 100000),
                        [1.0, 4.0, 0.36]]).astype(np.float32)
    o = run(np.zeros_like(b), b)
    ref = 1.0 / np.sqrt(b.astype(np.float64))
    rel = np.abs(o[:, 8] - ref) / ref
    rel_cuda = np.abs(o[:, 9] - ref) / ref
    print("rsqrt max rel error: library", rel.max(), "CUDA", rel_cuda.max())
    assert rel.max() <= 2.4e-7


def test_packed_fp32_matches_scalar_bits():
    """The packed two-wide FMA and subtraction give the scalar operations'
    bits, over every magnitude including subnormal operands and results."""
    rng = np.random.default_rng(5)
    n = 400000
    a = (rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-44, 30, n)).astype(np.float32)
    b = (rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-44, 30, n)).astype(np.float32)
    tiny = np.float32(1.4e-45)
    extra_a = np.array([0.0, -0.0, tiny, -tiny, 1e-39, 3e-39, 1.0, np.inf, np.nan], np.float32)
    extra_b = np.array([-0.0, 0.0, tiny, tiny, -5e-39, 2e-39, -1.0, 1.0, 2.0], np.float32)
    a = np.concatenate([a, extra_a, rng.uniform(-1, 1, 100000).astype(np.float32)])
    b = np.concatenate([b, extra_b, rng.uniform(-1, 1, 100000).astype(np.float32)])
    from paper_2603_20525_gb300 import atp
    L = atp.load()
    ad = torch.as_tensor(a).cuda()
    bd = torch.as_tensor(b).cuda()
    out = torch.empty((len(a), 14), dtype=torch.float32, device="cuda")
    assert L.atp_math_check(C.c_void_p(ad.data_ptr()), C.c_void_p(bd.data_ptr()), len(a),
                            C.c_void_p(out.data_ptr()), None) == 0
    torch.cuda.synchronize()
    o = out.cpu().numpy().view(np.uint32)
    assert np.array_equal(o[:, 10], o[:, 11])
    assert np.array_equal(o[:, 12], o[:, 13])
