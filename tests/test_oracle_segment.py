"""Pins of the oracle's generic segment model (Sec. III-E generic roofline
path with Eq. 16, host transfers of Eq. 15, synchronisation points, extra
launches of multi-kernel segments, executions).  Each term is checked in
isolation against its closed form, plus one hand-evaluated mixed row and the
model's time homogeneity."""
import numpy as np
import pytest

import oracle as O

N_SM = 152
TH = O.prior_theta(N_SM)
PSI = np.array([1.2, 1.1, 1.3, 1.5, 0.9, 1.0, 0.8, 2.1e11, 3.6e-6, 1.93e11, 3.4e-6, 1e-5,
                0.9, 1.1, 0.6, 0.7, 0.2])


def seg(**kw):
    return {k: np.array([v]) for k, v in kw.items()}


def one(theta=TH, psi=PSI, **kw):
    return float(O.segment_predict(seg(**kw), theta, psi, N_SM)[0])


def test_memory_class_without_working_set_blend():
    th = TH.copy()
    th[3] = 0.0                                   # w0 <= 0: B_eff = B_sus (Eq. 16 disabled)
    t = one(th, bytes=3e9, working_set=1e6, kernels=1, cls=0)
    assert t == pytest.approx(th[0] + PSI[0] * 3e9 / th[1], rel=1e-14)


def test_small_working_set_sees_peak_bandwidth():
    th = TH.copy()
    th[3] = 1e30
    t = one(th, bytes=3e9, working_set=1e6, kernels=1, cls=3)
    assert t == pytest.approx(th[0] + PSI[3] * 3e9 / th[2], rel=1e-12)


@pytest.mark.parametrize("prec,rate_idx", [(0, 6), (1, 7), (2, 8)])
def test_compute_class_uses_precision_rate_and_efficiency(prec, rate_idx):
    t = one(flops=1e15, bytes=1.0, kernels=1, cls=1, precision=prec)
    assert t == pytest.approx(TH[0] + PSI[1] * 1e15 / (N_SM * TH[rate_idx] * PSI[4 + prec]), rel=1e-14)


def test_transfers_and_synchronisation():
    # no kernel: only Eq. 15 per direction and the sync points
    assert one(h2d_bytes=1e9, kernels=0) == pytest.approx(1e9 / PSI[7] + PSI[8], rel=1e-14)
    assert one(d2h_bytes=1e9, kernels=0) == pytest.approx(1e9 / PSI[9] + PSI[10], rel=1e-14)
    assert one(syncs=3, kernels=0) == pytest.approx(3 * PSI[11], rel=1e-14)
    assert one(kernels=0) == 0.0                  # an empty transfer costs nothing, not tau


def test_extra_launches_and_executions():
    base = dict(flops=1e9, bytes=1e8, working_set=1e8, cls=2, precision=1)
    t1 = one(kernels=1, **base)
    assert one(kernels=4, **base) - t1 == pytest.approx(3 * TH[0], rel=1e-9)
    assert one(kernels=1, execs=7, **base) == pytest.approx(7 * t1, rel=1e-14)


def test_hand_evaluated_mixed_row():
    # balanced BF16 segment, 3 kernels, both transfers, 2 syncs, 4 executions;
    # evaluated by hand: B_eff = 6.8e12 (W = 2 GB >> w0), compute 1.690725e-3 s
    # beats memory 1.176471e-3 s, x 1.3, + 3 launches + 2.557143e-3 + 3.6e-6
    # + 1.388601e-3 + 3.4e-6 + 2e-5, all x 4
    t = one(flops=4e12, bytes=8e9, working_set=2e9, h2d_bytes=5.37e8, d2h_bytes=2.68e8, cls=2, precision=1,
            kernels=3, syncs=2, execs=4)
    assert t == pytest.approx(2.474274323e-02, rel=1e-9)


def test_time_homogeneity():
    # latencies x lambda and rates / lambda (theta and psi) scale every time by lambda
    rng = np.random.default_rng(0)
    n = 200
    s = dict(flops=10 ** rng.uniform(6, 15, n), bytes=10 ** rng.uniform(3, 11, n),
             working_set=10 ** rng.uniform(3, 11, n), h2d_bytes=np.where(rng.uniform(size=n) < 0.5, 1e8, 0.0),
             d2h_bytes=np.where(rng.uniform(size=n) < 0.5, 1e7, 0.0), cls=rng.integers(0, 4, n),
             precision=rng.integers(0, 3, n), kernels=rng.integers(0, 5, n), syncs=rng.integers(0, 3, n),
             execs=rng.integers(1, 9, n))
    lam = 3.0
    th = TH.copy()
    for j in O.LATENCY_IDX:
        th[j] *= lam
    for j in O.RATE_IDX:
        th[j] /= lam
    ps = PSI.copy()
    ps[[8, 10, 11]] *= lam
    ps[[7, 9]] /= lam
    t1 = O.segment_predict(s, TH, PSI, N_SM)
    t2 = O.segment_predict(s, th, ps, N_SM)
    assert np.allclose(t2, lam * t1, rtol=1e-12, atol=0)


def test_invalid_records_are_nan():
    for bad in (dict(cls=4), dict(precision=3), dict(kernels=-1), dict(execs=0), dict(bytes=-1.0), dict(syncs=-2)):
        rec = dict(flops=1e9, bytes=1e9, kernels=1)
        rec.update(bad)
        assert np.isnan(one(**rec)), bad


def test_concurrent_streams_add_tau_c():
    # Sec. III-A.6: N_c concurrent copies add (N_c - 1) tau_c, tau_c =
    # kappa_launch x launches + kappa_class x the class-scaled roofline term;
    # one stream (or 0) adds nothing
    base = dict(flops=1e9, bytes=4e9, working_set=4e9, kernels=2, cls=0, precision=1)
    t1 = one(**base)
    assert one(streams=0, **base) == t1 and one(streams=1, **base) == t1
    launches = 2 * TH[0]
    roof = t1 - launches
    for nc in (2, 3, 8):
        assert one(streams=nc, **base) == pytest.approx(t1 + (nc - 1) * (PSI[16] * launches + PSI[12] * roof),
                                                       rel=1e-13)
    comp = dict(flops=1e15, bytes=1.0, kernels=1, cls=1, precision=1)
    c1 = one(**comp)
    assert one(streams=4, **comp) == pytest.approx(c1 + 3 * (PSI[16] * TH[0] + PSI[13] * (c1 - TH[0])), rel=1e-13)
    # transfers and syncs are not multiplied by the streams (they are the host's)
    t_h = one(h2d_bytes=1e8, syncs=2, streams=3, **base)
    assert t_h - one(streams=3, **base) == pytest.approx(1e8 / PSI[7] + PSI[8] + 2 * PSI[11], rel=1e-12)
    assert np.isnan(one(streams=-1, **base))
