"""Pins of TMEM strategy B in the oracle (CPU only).

Sec. III-A.1 names two TMEM strategies: (A) only the accumulators live in
tensor memory, both operands are read from shared memory; (B) the A operand
is also staged in tensor memory, which adds TMEM traffic and is covered by
the same T_TMEM term of Eq. 2 (under the measured reading its tcgen05.cp
copies are tensor-pipe instructions and pay L_mma like the MMAs).  The pins: hand-checked capacity boundaries of
the strategy-B tile space, the closed-form time difference B - A when the
K-step is compute-bound, the reduction to strategy A at unbounded TMEM
bandwidth, and the homogeneity / gradient identities on strategy-B rows.
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S

FIELDS = ("M", "N", "K", "BM", "BN", "BK", "stages", "cta_group", "dtype", "kind", "tmem_a")
PRIOR160 = O.prior_theta(160)


def cfgs(rows):
    return {f: np.array([r.get(f, 0) for r in rows], dtype=np.int32) for f in FIELDS}


def one(theta, n_sm=160, **r):
    return float(O.model_batch(cfgs([r]), theta, n_sm)[0])


# (BM, BN, BK, stages, cta_group, dtype, valid under B, reason)
BOUNDARIES = [
    # FP8: 256 accumulator columns (two 128-row blocks x 128) + 4 stages x 2
    # blocks x 32 columns of A (128 one-byte K values = 32 words) = 512
    (256, 128, 128, 4, 1, 2, True, "TMEM exactly full"),
    # FP8: 256 + 6 x 2 x 16 = 448 columns; ring 6 x 64 x 384 B = 144 KiB
    (256, 128, 64, 6, 1, 2, True, "fits"),
    # 256 x 256 accumulators already take all 512 columns
    (256, 256, 64, 2, 1, 2, False, "no room for A"),
    (256, 256, 64, 2, 1, 1, False, "no room for A"),
    # FP32 (hi and lo planes, 4-byte words): 256 + 2 stages x 2 blocks x
    # 2 planes x 32 columns = 512
    (256, 128, 32, 2, 1, 0, True, "TMEM exactly full"),
    # BF16: 128 + 4 x 1 x 32 = 256 columns
    (128, 128, 64, 4, 1, 1, True, "fits"),
    (128, 128, 64, 4, 2, 1, False, "CTA pairs keep strategy A"),
    (64, 128, 64, 4, 1, 1, False, "64-row tiles keep strategy A"),
]


@pytest.mark.parametrize("bm,bn,bk,s,g,dt,ok,why", BOUNDARIES)
def test_strategy_b_capacity_boundaries(bm, bn, bk, s, g, dt, ok, why):
    assert O.cfg_valid(bm, bn, bk, s, g, dt, 1) == ok, why
    assert O.cfg_valid(bm, bn, bk, s, g, dt, 0)          # all of these are valid strategy-A tiles


def test_strategy_b_space_is_a_subset_of_a():
    counts = {}
    for dt in (0, 1, 2):
        b = [t for t in S.tile_space(dt) if O.cfg_valid(*t, dt, 1)]
        assert all(O.cfg_valid(*t, dt, 0) for t in b)
        assert all(t[4] == 1 and t[0] >= 128 for t in b)
        # a valid ring stays valid with one stage fewer
        assert all(O.cfg_valid(t[0], t[1], t[2], t[3] - 1, 1, dt, 1) for t in b if t[3] > 2)
        counts[dt] = len(b)
    assert counts == {0: 9, 1: 28, 2: 45}
    assert not O.cfg_valid(128, 128, 64, 4, 1, 1, 2)      # only strategies 0 and 1 exist


@pytest.mark.parametrize("dt,bk,e,n_p,l", [(1, 64, 2, 1, 1), (2, 128, 1, 1, 1), (0, 32, 4, 3, 2)])
def test_strategy_b_adds_a_tile_traffic_when_compute_bound(reading, dt, bk, e, n_p, l):
    # alpha = 1 (c_alpha = 0) leaves T_io = T_sync, so every K-step costs
    # T_c + T_sync (instant loads keep the measured reading's ring bound
    # (T_tma + T_c + T_sync)/s below it) and the two strategies differ only
    # in T_TMEM:
    #   per K-step   n_p e BM BK / BW_rd  (every pass reads A from TMEM)
    #              + l e BM BK / BW_wr    (the A planes are copied in)
    #              + n_cp L_mma           (measured reading: one tcgen05.cp per
    #                                      128 x 32-byte slice, l * BK e / 32)
    th = PRIOR160.copy()
    th[15] = 0.0
    th[4], th[5] = 0.0, 1e30           # instant loads: the ring bound of the measured reading stays below
    M = N = 1024                       # 8 x 8 = 64 tiles of 128 x 128: one wave on 160 SMs
    K = bk * 50
    base = dict(M=M, N=N, K=K, BM=128, BN=128, BK=bk, stages=2, cta_group=1, dtype=dt)
    t_a = one(th, **base)
    t_b = one(th, tmem_a=1, **base)
    n_cp = l * bk * e // 32 if reading == 1 else 0      # the copies pay L_mma under the measured reading
    per_step = n_p * e * 128 * bk / th[10] + l * e * 128 * bk / th[11] + n_cp * th[9]
    assert t_b - t_a == pytest.approx(50 * per_step, rel=1e-9)


def test_strategy_b_equals_a_at_unbounded_tmem_bandwidth(reading):
    th = PRIOR160.copy()
    th[10] = th[11] = 1e30
    th[9] = 0.0                                        # and free tensor-pipe instructions
    th[17] = 1e30                                      # and a free drain: B's A ring can leave one buffer
    rows = []
    for dt in (0, 1, 2):
        for t in S.tile_space(dt):
            if O.cfg_valid(*t, dt, 1):
                for mnk in ((512, 512, 512), (4096, 2048, 1024), (300, 200, 320)):
                    rows.append(dict(zip(("M", "N", "K"), mnk), BM=t[0], BN=t[1], BK=t[2], stages=t[3],
                                     cta_group=t[4], dtype=dt))
    ca = cfgs(rows)
    cb = cfgs([dict(r, tmem_a=1) for r in rows])
    assert np.allclose(O.model_batch(cb, th, 152), O.model_batch(ca, th, 152), rtol=1e-12, atol=0)


def _b_rows(n=2000, seed=31):
    c = S.model_config_batch(n, seed)
    c["kind"] = np.zeros(n, dtype=np.int32)
    c["tmem_a"] = np.ones(n, dtype=np.int32)
    return c


def test_strategy_b_homogeneity_and_euler_identity(reading):
    c = _b_rows()
    th2 = PRIOR160.copy()
    for j in O.LATENCY_IDX:
        th2[j] *= 2.0
    for j in O.RATE_IDX:
        th2[j] /= 2.0
    assert np.allclose(O.model_batch(c, th2, 152) / O.model_batch(c, PRIOR160, 152), 2.0, rtol=1e-12, atol=0)
    t, g = O.model_batch(c, PRIOR160, 152, grad=True)
    lat = sum(PRIOR160[j] * g[:, j] for j in O.LATENCY_IDX)
    rate = sum(PRIOR160[j] * g[:, j] for j in O.RATE_IDX)
    assert np.allclose(lat - rate, t, rtol=1e-9, atol=0)


def test_strategy_b_tmem_gradient_central_differences(reading):
    # dT/dtheta for the TMEM bandwidths on compute-bound strategy-B rows,
    # against central differences in ln theta
    th = PRIOR160.copy()
    th[15] = 0.0
    rows = [dict(M=1024, N=1024, K=64 * 50, BM=128, BN=128, BK=64, stages=2, cta_group=1, dtype=1, tmem_a=1),
            dict(M=2048, N=1024, K=128 * 30, BM=256, BN=128, BK=128, stages=4, cta_group=1, dtype=2, tmem_a=1)]
    c = cfgs(rows)
    t, g = O.model_batch(c, th, 160, grad=True)
    for j in (9, 10, 11):
        h = 1e-4
        tp, tm = th.copy(), th.copy()
        tp[j] *= np.exp(h)
        tm[j] *= np.exp(-h)
        fd = (O.model_batch(c, tp, 160) - O.model_batch(c, tm, 160)) / (2 * h)
        assert np.allclose(g[:, j] * th[j], fd, rtol=1e-6, atol=0)
