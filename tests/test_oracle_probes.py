"""Pins of the oracle's probe references and of the synthetic generators (CPU only)."""
from fractions import Fraction

import numpy as np

import oracle as O
import synthetic as S


def test_splitmix64_reference_values():
    # First outputs of SplitMix64 with seed 1234567 as published with the
    # generator's reference C code (splitmix64.c test vector).
    z = S.splitmix64(1234567, 5)
    assert [int(v) for v in z] == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                                   4593380528125082431, 16408922859458223821]


def test_uniform_range_and_slicing():
    x = S.uniform_pm1(1, 100000)
    assert x.min() >= -1.0 and x.max() < 1.0
    assert abs(float(x.mean())) < 0.01
    assert np.array_equal(S.uniform_pm1(1, 50, offset=1000), x[1000:1050])
    # spacing 2^-23: (x + 1) * 2^23 is an integer
    assert np.all(np.floor((x.astype(np.float64) + 1.0) * 2 ** 23) == (x.astype(np.float64) + 1.0) * 2 ** 23)


def test_normal_moments():
    x = S.normal(2, 200000).astype(np.float64)
    assert abs(x.mean()) < 0.01 and abs(x.std() - 1.0) < 0.01


def test_triad_single_rounding_exact():
    n = 4000
    b = S.normal(1, n) * np.float32(1e3)
    c = S.uniform_pm1(2, n)
    s = np.float32(3.0)
    a = O.triad_f32(b, c, float(s))
    for i in range(0, n, 7):
        exact = Fraction(float(s)) * Fraction(float(c[i])) + Fraction(float(b[i]))
        # round the exact value to the nearest FP32 (ties to even) via numpy's
        # correctly rounded FP64 -> FP32 conversion of the two bracketing doubles
        lo = np.float32(float(exact))
        cands = [lo, np.nextafter(lo, np.float32(np.inf)), np.nextafter(lo, np.float32(-np.inf))]
        best = min(cands, key=lambda v: (abs(Fraction(float(v)) - exact), int(np.float32(v).view(np.uint32)) & 1))
        assert a[i] == best, (i, a[i], best)


def test_cyclic_permutation_is_one_cycle():
    for n in (1, 2, 3, 17, 1000, 65536):
        nxt = S.cyclic_permutation(n, seed=1)
        assert np.array_equal(np.sort(nxt), np.arange(n, dtype=np.uint32))
        j, seen = 0, 0
        while True:
            j = int(nxt[j]); seen += 1
            if j == 0:
                break
        assert seen == n


def test_pchase_walk():
    n = 4096
    buf = S.pchase_buffer(n, seed=1, stride_bytes=64)
    assert O.pchase(buf, 16, 0, n) == 0                 # one full cycle returns home
    assert O.pchase(buf, 16, 0, 3 * n) == 0
    nxt = S.cyclic_permutation(n, 1)
    j = 5
    for _ in range(123):
        j = int(nxt[j])
    assert O.pchase(buf, 16, 5, 123) == j
    assert O.pchase(buf, 16, 5, 0) == 5


def test_grouped_m_distribution():
    m = S.grouped_m(64, 3)
    assert m.min() >= 16 and m.max() <= 4096 and len(m) == 64
    lm = np.log(S.grouped_m(20000, 3).astype(np.float64))
    # log-uniform on [ln 16, ln 4096]: mean at the midpoint ln 256
    assert abs(lm.mean() - np.log(256.0)) < 0.05


def test_model_config_batch_shapes():
    c = S.model_config_batch(10000, seed=4)
    for f in ("M", "N", "K"):
        assert c[f].min() >= 16 and c[f].max() <= 16384 and np.all(c[f] % 16 == 0)
    assert set(np.unique(c["dtype"])) == {0, 1, 2}
    assert len(S.tile_space(1)) == 180


def test_stencil_fixed_points_and_closed_forms():
    # integer grids keep every intermediate exact: an affine (discrete
    # harmonic) grid is a fixed point, x = i^2 gains 0.125 * 2 per interior point
    rows, cols = 37, 53
    i, j = np.meshgrid(np.arange(rows), np.arange(cols), indexing="ij")
    aff = (3 * i - 2 * j + 7).astype(np.float32)
    assert np.array_equal(O.stencil5_f32(aff), aff)
    quad = (i * i).astype(np.float32)
    out = O.stencil5_f32(quad)
    expect = quad.copy()
    expect[1:-1, 1:-1] += 0.25
    assert np.array_equal(out, expect)
    const = np.full((5, 4), 1.75, np.float32)
    assert np.array_equal(O.stencil5_f32(const), const)


def test_stencil_matches_stepwise_float32_on_random_grid():
    x = S.uniform_pm1(17, 9 * 11).reshape(9, 11)
    out = O.stencil5_f32(x)
    f = np.float32
    for r in range(9):
        for c in range(11):
            if r in (0, 8) or c in (0, 10):
                assert out[r, c] == x[r, c]
                continue
            vert = f(x[r - 1, c]) + f(x[r + 1, c])
            horz = f(x[r, c - 1]) + f(x[r, c + 1])
            want = f(f(0.5) * x[r, c]) + f(f(0.125) * f(vert + horz))
            assert out[r, c] == want, (r, c)
