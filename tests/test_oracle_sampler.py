"""Pins of the oracle's candidate sampler: its Philox4x64-10 against numpy's
independent implementation of the same published generator, the Box-Muller
normals against their distribution, and the warm-start rule by hand."""
import numpy as np
import pytest
from scipy import stats

import oracle


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_philox_matches_numpy(seed):
    rng = np.random.default_rng(seed)
    for _ in range(20):
        key = rng.integers(0, 2 ** 63, 2, dtype=np.uint64) * 2 + rng.integers(0, 2, 2, dtype=np.uint64)
        ctr = rng.integers(0, 2 ** 63, 4, dtype=np.uint64)
        # numpy's Philox advances its counter by one before each block of 4
        ref = np.random.Philox(key=key, counter=ctr).random_raw(4)
        nxt = ctr.copy()
        nxt[0] += np.uint64(1)
        assert np.array_equal(oracle.philox4x64_10(nxt, key), ref)


def test_sampler_distribution_and_nominal():
    N, H = 4096, 40
    s = oracle.sample(None, 0, 0.2, 0.3, (7, 11), 3, N, H)
    assert np.all(s[:, 0, :] == 0.0)                    # candidate 0 is the nominal
    a = s[:, 1:, 0].ravel() / 0.2
    b = s[:, 1:, 1].ravel() / 0.3
    for x in (a, b):
        assert abs(x.mean()) < 0.01 and abs(x.std() - 1.0) < 0.01
        assert stats.kstest(x, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.01           # the pair is independent
    # distinct nonces give distinct draws, the same nonce the same draws
    s2 = oracle.sample(None, 0, 0.2, 0.3, (7, 11), 4, N, H)
    assert not np.allclose(s[:, 1:], s2[:, 1:])
    assert np.array_equal(s, oracle.sample(None, 0, 0.2, 0.3, (7, 11), 3, N, H))


def test_warm_start_shift_rule():
    prev = np.arange(10, dtype=np.float32).reshape(5, 2)        # 5 steps
    s = oracle.sample(prev, 1, 0.0, 0.0, (1, 2), 0, 3, 8)     # zero noise: nominal only
    want = [prev[min(k + 1, 4)] for k in range(8)]
    for j in range(3):
        assert np.array_equal(s[:, j, :], np.array(want, dtype=np.float64))


def test_draws_follow_the_documented_word_and_bit_map():
    """Each draw from numpy's independent Philox4x64-10 by the documented map:
    one call at counter (j, k // 4, nonce, 0) serves four steps, words (w0, w1)
    for k % 4 in {0, 2} and (w2, w3) for {1, 3}, bits 63..41 of each for
    k % 4 < 2 and bits 31..9 for k % 4 >= 2, then the Box-Muller pair."""
    key, nonce, N, H = (np.uint64(0x1234567), np.uint64(0x89ABCDEF)), 5, 7, 9
    s = oracle.sample(None, 0, 0.2, 0.3, (int(key[0]), int(key[1])), nonce, N, H)
    for j in range(1, N):
        for k in range(H):
            ctr = np.array([j, k // 4, nonce, 0], dtype=np.uint64)
            # numpy's Philox advances its counter by one before each block
            prev = ctr.copy()
            prev[0] -= np.uint64(1)
            w = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=prev).random_raw(4)
            a, b = (w[2], w[3]) if k % 2 else (w[0], w[1])
            if k % 4 >= 2:
                ua, ub = (int(a) >> 9) & 0x7FFFFF, (int(b) >> 9) & 0x7FFFFF
            else:
                ua, ub = int(a) >> 41, int(b) >> 41
            u1, u2 = (ua + 0.5) / 8388608.0, (ub + 0.5) / 8388608.0
            r = np.sqrt(-2.0 * np.log(u1))
            np.testing.assert_allclose(s[k, j], [0.2 * r * np.cos(2 * np.pi * u2), 0.3 * r * np.sin(2 * np.pi * u2)],
                                       rtol=1e-13, atol=1e-15)
