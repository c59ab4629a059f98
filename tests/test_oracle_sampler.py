"""Oracle of the geo-anchor draw (Supp. "TDOM/DSM Reference Crop": valid geo-anchors are
sampled from the crop), pinned on the CPU:

* its generator against the published SplitMix64 test vector (tests/golden/splitmix64.txt)
  and against the generator's defining recurrence written differently (a closed form of the
  j-th state instead of the running sum);
* the draw: exactly min(n, #valid) distinct valid pixels in increasing order, all valid
  pixels when n >= #valid, nothing for n = 0;
* a uniform draw without replacement: every valid pixel is drawn with frequency n / #valid
  over many seeds (chi-square), and each pair of pixels with frequency n(n-1) / (V(V-1));
* the draw depends only on the keys: restricting the mask to a superset of the drawn pixels
  draws the same pixels.
"""
import os

import numpy as np

from oracle import sampler as OS

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")


def test_splitmix64_published_test_vector():
    line = next(l for l in open(GOLDEN) if l.startswith("seed"))
    parts = line.split()
    seed, k, want = int(parts[1]), int(parts[3]), int(parts[4], 16)
    assert OS.splitmix64(seed, k)[k - 1] == want


def test_splitmix64_matches_the_closed_form_state():
    # the j-th state is seed + j * gamma (mod 2^64); mix it directly
    M = (1 << 64) - 1
    for seed in (0, 1, 12345678901234, M):
        outs = OS.splitmix64(seed, 20)
        for j in range(1, 21):
            z = (seed + j * 0x9E3779B97F4A7C15) & M
            z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
            z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
            assert outs[j - 1] == z ^ (z >> 31)


def test_draw_is_a_sorted_subset_of_the_valid_pixels():
    rng = np.random.default_rng(0)
    for n_pix, n in [(100, 10), (1000, 500), (37, 37), (50, 0), (8100, 500)]:
        valid = rng.random(n_pix) < 0.7
        idx = OS.sample_anchors(valid, n, seed=99)
        assert len(idx) == min(n, valid.sum())
        assert np.all(valid[idx])
        assert np.all(np.diff(idx) > 0)


def test_all_valid_pixels_when_n_exceeds_them():
    valid = np.zeros(64, bool)
    valid[[3, 7, 8, 40]] = True
    np.testing.assert_array_equal(OS.sample_anchors(valid, 10, seed=5), [3, 7, 8, 40])
    assert OS.sample_anchors(np.zeros(10, bool), 3, seed=5).size == 0


def test_draw_is_uniform_without_replacement():
    valid = np.zeros(40, bool)
    valid[np.arange(0, 40, 3)] = True            # 14 valid pixels, spread out
    V, n, trials = int(valid.sum()), 4, 3000
    counts = np.zeros(40)
    pair = np.zeros((40, 40))
    for seed in range(trials):
        idx = OS.sample_anchors(valid, n, seed)
        counts[idx] += 1
        pair[np.ix_(idx, idx)] += 1
    exp = trials * n / V
    chi2 = (((counts[valid] - exp) ** 2) / exp).sum()
    assert chi2 < 36.0                            # 13 degrees of freedom: p < 1e-3 above 34.5
    v = np.flatnonzero(valid)
    off = pair[np.ix_(v, v)][~np.eye(V, dtype=bool)]
    exp2 = trials * n * (n - 1) / (V * (V - 1))
    assert abs(off.mean() - exp2) < 0.05 * exp2
    assert counts[~valid].sum() == 0


def test_draw_depends_only_on_the_keys():
    rng = np.random.default_rng(1)
    valid = rng.random(500) < 0.5
    idx = OS.sample_anchors(valid, 30, seed=7)
    sub = np.zeros_like(valid)
    sub[idx] = True
    sub[rng.choice(np.flatnonzero(valid), 60, replace=False)] = True
    np.testing.assert_array_equal(OS.sample_anchors(sub, 30, seed=7), idx)
