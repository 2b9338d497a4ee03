"""CPU checks of the seeded input generators against the recipe they state:
power-law coordinate frequencies, the rank -> index bijection, distinct
uniform coordinates, round-to-nearest-even 16-bit factors, the integer case,
and determinism under the seed."""
import math

import numpy as np
import pytest

import synth


def test_zipf_frequencies_follow_the_power_law():
    """Sorted coordinate counts against I p(k) with p(k) = k^-s / H (the map
    rank -> index is a bijection, so the sorted counts are the rank counts
    wherever expected counts are far apart): the top ranks within 5 sigma."""
    I, n = 1000, 400_000
    for s in (0.8, 1.2, 2.0):
        idx, _ = synth.coo_zipf([I], n, s, 7)
        cnt = np.sort(np.bincount(idx[0], minlength=I))[::-1]
        p = np.arange(1, I + 1, dtype=np.float64) ** -s
        p /= p.sum()
        for k in range(3):
            mu = n * p[k]
            sd = math.sqrt(n * p[k] * (1 - p[k]))
            assert abs(cnt[k] - mu) <= 5 * sd, (s, k, cnt[k], mu)
        assert cnt.sum() == n


def test_rank_to_index_map_is_a_bijection_and_uniform_case_is_flat():
    I, n = 997, 300_000
    idx, _ = synth.coo_zipf([I], n, 0.0, 3)
    assert idx.min() >= 0 and idx.max() < I
    cnt = np.bincount(idx[0], minlength=I)
    chi2 = ((cnt - n / I) ** 2 / (n / I)).sum()
    assert chi2 < I + 6 * math.sqrt(2 * I)  # chi-square with I-1 degrees of freedom, 6 sigma
    # with s > 0 every index stays in range and the hottest one is not simply 0
    for seed in range(5):
        z, _ = synth.coo_zipf([I], 50_000, 1.5, seed)
        assert z.min() >= 0 and z.max() < I
    hot = {int(np.argmax(np.bincount(synth.coo_zipf([I], 50_000, 1.5, seed)[0][0], minlength=I)))
           for seed in range(5)}
    assert len(hot) > 1


def test_generators_are_deterministic_under_the_seed():
    a = synth.coo_zipf([50, 40, 30], 10_000, (1.1, 0.5, 0.0), 11)
    b = synth.coo_zipf([50, 40, 30], 10_000, (1.1, 0.5, 0.0), 11)
    c = synth.coo_zipf([50, 40, 30], 10_000, (1.1, 0.5, 0.0), 12)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[0], c[0])
    assert a[1].dtype == np.float32 and a[1].min() >= 0 and a[1].max() < 1
    f1 = synth.factor_matrices([50, 40], 12, 4, "normal")
    f2 = synth.factor_matrices([50, 40], 12, 4, "normal")
    assert all(np.array_equal(x, y) for x, y in zip(f1, f2))


def test_distinct_uniform_coordinates_are_distinct():
    dims = (20, 15, 10)
    idx, vals = synth.coo_uniform_distinct(dims, 2500, 0)
    lin = np.ravel_multi_index(tuple(idx.astype(np.int64)), dims)
    assert np.unique(lin).size == 2500
    assert not np.all(np.diff(lin) > 0)  # storage order is the draw's, not sorted


def _rne_bf16(x):
    """fp32 -> bf16 round to nearest even on the bit pattern (finite inputs)."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return r.astype(np.uint16)


def test_bf16_factors_are_round_to_nearest_even():
    rng = np.random.default_rng(0)
    x = rng.standard_normal(100_000).astype(np.float32)
    # exact ties: the low 16 bits equal 0x8000, both even and odd kept halves
    ties = (rng.integers(0x3F800000 >> 16, 0x40800000 >> 16, 1000, dtype=np.uint32) << 16) | 0x8000
    x = np.concatenate([x, ties.view(np.float32), -ties.view(np.float32)])
    got = synth._to_bf16_bits(x)
    assert np.array_equal(got, _rne_bf16(x))
    back = synth.bf16_bits_to_f32(got)
    assert np.all(np.abs(back - x) <= np.abs(x) * 2.0 ** -8)


def test_padding_columns_are_zero_and_16_bit_factors_round_the_fp32_draw():
    f32 = synth.factor_matrices([30, 20], 13, 5, "uniform")
    b16 = synth.factor_matrices([30, 20], 13, 5, "uniform", dtype="bf16")
    h16 = synth.factor_matrices([30, 20], 13, 5, "uniform", dtype="f16")
    for a, b, h in zip(f32, b16, h16):
        assert a.shape[1] == 16 and np.all(a[:, 13:] == 0)
        assert np.array_equal(b, _rne_bf16(a))
        assert np.array_equal(synth.f16_bits_to_f32(h), a.astype(np.float16).astype(np.float32))


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16", "f64"])
def test_integer_case_values_and_factors(dtype):
    idx, vals, facs = synth.small_integer_case((30, 20, 10), 5000, 7, 2, dtype=dtype)
    assert set(np.unique(vals)) <= {1.0, 2.0, 3.0, 4.0}
    for f in facs:
        w = {"f32": lambda a: a, "f64": lambda a: a, "bf16": synth.bf16_bits_to_f32,
             "f16": synth.f16_bits_to_f32}[dtype](f)
        assert set(np.unique(w[:, :7])) <= set(range(-3, 4))
        assert np.all(w[:, 7:] == 0)
