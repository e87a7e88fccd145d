"""The seeded input generators that both the oracle and the CUDA path consume.

bf16_round decides which bytes the oracle sees for every BF16-mixed parity
case, so it is pinned to hand-worked round-to-nearest-even cases and to an
independent implementation (torch's own float -> bfloat16 conversion); the
generators are checked for determinism and for the structure they claim.
"""
import numpy as np
import pytest
import torch

from paper_1710_02812_gb300 import workloads as W


def test_bf16_round_ties_go_to_even():
    one = 1.0
    ulp = 2.0 ** -7                       # bfloat16 spacing in [1, 2)
    cases = {
        one: one,
        one + ulp / 2: one,               # tie between 1 and 1 + ulp: even (1)
        one + 3 * ulp / 2: one + 2 * ulp,  # tie between 1 + ulp (odd) and 1 + 2 ulp (even)
        one + ulp / 2 + 2.0 ** -20: one + ulp,  # just above the tie rounds up
        one + ulp / 2 - 2.0 ** -20: one,        # just below rounds down
        -(one + 3 * ulp / 2): -(one + 2 * ulp),
        0.0: 0.0,
        3.4e38: float("inf"),             # past the midpoint between the largest bfloat16 and 2^128
    }
    x = np.array(list(cases.keys()), dtype=np.float32)
    want = np.array(list(cases.values()), dtype=np.float32)
    np.testing.assert_array_equal(W.bf16_round(x), want)
    special = np.array([np.inf, -np.inf, np.nan], dtype=np.float32)
    got = W.bf16_round(special)
    assert got[0] == np.inf and got[1] == -np.inf and np.isnan(got[2])


def test_bf16_round_matches_torch_conversion():
    rng = np.random.default_rng(11)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-30, 30, 20000),
                        rng.standard_normal(1000) * 1e-40]).astype(np.float32)  # includes subnormals
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(W.bf16_round(x), ref)
    # the result is exactly representable: rounding twice changes nothing
    np.testing.assert_array_equal(W.bf16_round(W.bf16_round(x)), W.bf16_round(x))


def test_generators_are_deterministic_per_tag():
    a = W.exp_decay(256, 192, r=64, noise=1e-5, tag=7)
    b = W.exp_decay(256, 192, r=64, noise=1e-5, tag=7)
    c = W.exp_decay(256, 192, r=64, noise=1e-5, tag=8)
    assert a.dtype == np.float32 and a.shape == (256, 192)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_planted_factors_are_what_they_claim():
    s = np.exp(-np.arange(20) / 5.0)
    a, u, s_out, v = W.planted(120, 90, s, noise=0.0, tag=3, dtype=np.float64, return_factors=True)
    np.testing.assert_allclose(u.T @ u, np.eye(20), atol=1e-13)
    np.testing.assert_allclose(v.T @ v, np.eye(20), atol=1e-13)
    np.testing.assert_allclose(a, (u * s_out) @ v.T, atol=1e-13)
    np.testing.assert_allclose(np.linalg.svd(a, compute_uv=False)[:20], np.sort(s)[::-1], rtol=1e-12)


def test_planted_band_is_the_slice_of_the_full_matrix():
    s = (np.arange(40) + 1.0) ** -1.5
    full = W.planted(300, 260, s, noise=1e-6, tag=77, dtype=np.float64)
    band = W.planted_band(300, 260, s, noise=1e-6, tag=77, rows=48, cols=100, dtype=np.float64)
    np.testing.assert_allclose(band, full[:48, :100], rtol=0, atol=1e-15)
