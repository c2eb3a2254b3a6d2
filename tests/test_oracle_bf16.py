"""Pins of the oracle's BF16 terrain format (oracle.bf16_round,
oracle.bf16_terrain), the host restatement the BF16 texel tests compare the
GPU with: the rounding against torch's own float32 -> bfloat16 conversion
(round to nearest even), exact decoding of a constant map, and the error of
every decoded height and slope against the FP32 map within half a bf16 ulp
of its residual from the block plane (plus FP32 rounding)."""
import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(0)
    x = (rng.choice([-1.0, 1.0], 200000) * 10.0 ** rng.uniform(-40, 38, 200000)).astype(np.float32)
    ties = (np.arange(1, 2000, dtype=np.uint32) << 16 | 0x8000).view(np.float32)   # exact halfway cases
    odd = (np.arange(1, 2000, dtype=np.uint32) << 16 | 0x7FFF).view(np.float32)
    special = np.array([0.0, -0.0, np.inf, -np.inf, 1.0, -1.0, 3.0e38, 1e-45], np.float32)
    x = np.concatenate([x, ties, odd, special])
    want = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(oracle.bf16_round(x), want)


def test_constant_map_decodes_exactly():
    h = np.full((37, 45), 2.375, np.float32)
    hd, gx, gy, _, plane = oracle.bf16_terrain(h, 0.1)
    assert np.array_equal(hd, h)
    assert np.all(gx == 0.0) and np.all(gy == 0.0)
    assert np.all(plane[..., 0] == 2.375) and np.all(plane[..., 1:] == 0.0)


def test_decoded_map_within_half_an_ulp_of_the_residuals():
    """Rough fBm with a ragged edge (blocks of fewer than 8 nodes): every
    decoded value differs from the FP32 one by at most half a bf16 ulp of its
    residual from the block plane (2^-8 relative: bf16 keeps 8 significant
    bits) plus FP32 rounding."""
    t = gen.terrain_plain(3)
    h = np.ascontiguousarray(t.heights[:, :-3])
    hd, gx, gy, (wr, wx, wy), plane = oracle.bf16_terrain(h, t.cell)
    ref = oracle.Terrain(h, t.cell)
    u = 2.0 ** -24
    ny, nx = h.shape
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    P = plane[jj // 8, ii // 8].astype(np.float64)
    base = P[..., 0] + P[..., 1] * (ii & 7) + P[..., 2] * (jj & 7)
    res = h.astype(np.float64) - base
    bound = 2.0 ** -8 * np.abs(res) + 4 * u * (np.abs(h) + np.abs(base)) + 1e-30
    assert np.all(np.abs(hd.astype(np.float64) - h) <= bound)
    inv = 1.0 / t.cell
    for dec, full, sl in ((gx, ref.gx, P[..., 1] * inv), (gy, ref.gy, P[..., 2] * inv)):
        r = full - sl
        b = 2.0 ** -8 * np.abs(r) + 4 * u * (np.abs(full) + np.abs(sl)) + 1e-30
        assert np.all(np.abs(dec - full) <= b)
    # the block planes pass through each block's first node
    assert np.array_equal(plane[..., 0], h[::8, ::8])


def test_block_planes_recover_a_linear_map():
    """h = 0.25 + 0.125 i - 0.0625 j (exact in FP32): every block's plane,
    the ragged edge blocks included, has the map's per-node slopes (to the
    FP32 rounding of the division by the block's extent) through its first
    node, and the decoded map is the map to within FP32 rounding."""
    ny, nx = 29, 43                                # ragged blocks on both edges
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    h = (0.25 + 0.125 * ii - 0.0625 * jj).astype(np.float32)
    hd, gx, gy, _, plane = oracle.bf16_terrain(h, 0.5)
    assert np.array_equal(plane[..., 0], h[::8, ::8])
    wide = np.array([min(8, nx - 8 * b) for b in range(plane.shape[1])]) > 1
    tall = np.array([min(8, ny - 8 * b) for b in range(plane.shape[0])]) > 1
    assert np.allclose(plane[:, wide, 1], 0.125, rtol=2 ** -22, atol=0)
    assert np.allclose(plane[tall, :, 2], -0.0625, rtol=2 ** -22, atol=0)
    assert np.allclose(hd, h, rtol=0, atol=4 * 2 ** -24 * np.abs(h).max())
    assert np.allclose(gx, 0.25, rtol=2 ** -20) and np.allclose(gy, -0.125, rtol=2 ** -20)
