"""Host-side calibration logic on the CPU: the fit driver recovers known
parameters when the objective is the oracle's (the GPU objective is the same
driver with pm_model_grad behind it), the split is seeded and disjoint, and
the MAE bookkeeping follows its definition."""
import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S
from paper_2605_04178_gb300 import calibrate as C

N_SM = 152
FIELDS = C.FIELDS


def table(theta):
    """The calibration table's configurations: the BF16/FP8 sweep (every valid BF16 and
    FP8 tile at M = N = K in {1024 .. 16384}, 1,445 rows), the FP32 GEMM at
    512^3 over its 55 tiles and the memory probes (copy and triad 2^20 .. 2^30, the
    five TMA tiles), with the oracle's times under theta as the targets."""
    rows = []
    for s in (1024, 2048, 4096, 8192, 16384):
        for dt in (1, 2):
            for t in S.tile_space(dt):
                if O.cfg_valid(*t, dt):
                    rows.append(dict(zip(FIELDS, (s, s, s, *t, dt, 0))))
    for t in S.tile_space(0):
        if O.cfg_valid(*t, 0):
            rows.append(dict(zip(FIELDS, (512, 512, 512, *t, 0, 0))))
    for k in range(20, 31):
        rows.append(dict(M=2 ** k, N=0, K=0, BM=0, BN=0, BK=0, stages=0, cta_group=0, dtype=0, kind=1))
        rows.append(dict(M=2 ** k, N=0, K=0, BM=0, BN=0, BK=0, stages=0, cta_group=0, dtype=0, kind=2))
    for tr, tc in ((64, 64), (128, 64), (128, 128), (256, 64), (256, 128)):
        rows.append(dict(M=16384, N=16384, K=0, BM=tr, BN=tc, BK=0, stages=0, cta_group=0, dtype=0, kind=3))
    cols = {f: np.array([r.get(f, 0) for r in rows], dtype=np.int32) for f in FIELDS}
    t = O.model_batch(cols, theta, N_SM)
    for r, v in zip(rows, t):
        r["t"] = float(v)
    return rows, cols


class OracleLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, cols, t_meas):
        L, g = O.model_loss_grad(cols, theta.detach().numpy(), N_SM, t_meas)
        ctx.save_for_backward(torch.tensor(g))
        return torch.tensor(L, dtype=torch.float64)

    @staticmethod
    def backward(ctx, go):
        (g,) = ctx.saved_tensors
        return go * g, None, None


@pytest.mark.parametrize("r", [0, 1])
def test_prior_matches_oracle_prior(r):
    assert np.array_equal(C.prior_theta(N_SM, reading=r), O.prior_theta(N_SM, reading=r))


# Parameters the table does not determine one by one at the generating
# point: TMEM read and write bandwidth enter every strategy-A K-step only as
# D (1/BW_rd + 1/BW_wr) (Eq. 2), so only that sum is fixed; the literal
# reading uses neither rho_L2 nor B_drain; under the measured reading the
# ring bound of Eq. 8 sets every K-step of the table at the printed priors,
# so alpha's c_alpha (Eq. 7) is not seen at all.
UNIDENTIFIABLE = {0: {10, 11, 16, 17}, 1: {10, 11, 15}}


def identifiable(cols, theta):
    """Parameters j whose direction has no component in the null space of
    the Jacobian d ln T_hat / d ln theta (singular values below 1e-6 of the
    largest) at theta."""
    t, g = O.model_batch(cols, theta, N_SM, grad=True)
    J = g * theta[None, :] / t[:, None]
    _, sv, Vt = np.linalg.svd(J, full_matrices=False)
    null = Vt[sv < 1e-6 * sv[0]]
    proj = np.sqrt((null ** 2).sum(0)) if len(null) else np.zeros(O.N_PARAMS)
    return proj < 1e-6


def test_fit_recovers_generating_parameters(reading):
    # Targets from a known theta* (the printed priors); the fit starts from
    # theta* exp(N(0, 0.3^2)) (seed 5) and must return ln theta* within 1e-3
    # on every identifiable parameter (Sec. III-D: parameters fitted to
    # measured times; here the times are the model's own, so the fit must
    # find the generating point, not another one that fits as well).
    truth = C.prior_theta(N_SM, reading=reading)
    rows, cols = table(truth)
    assert len(rows) == 1445 + 55 + 27
    ident = identifiable(cols, truth)
    assert set(np.where(~ident)[0]) == UNIDENTIFIABLE[reading]
    t_meas = np.array([r["t"] for r in rows])
    start = truth * np.exp(0.3 * S.normal(5, O.N_PARAMS).astype(np.float64))
    theta, trace = C.fit(lambda th: OracleLoss.apply(th, cols, t_meas), start, reg=0.0)
    err = np.abs(np.log(theta) - np.log(truth))
    assert np.all(err[ident] <= 1e-3), dict(zip(np.where(ident)[0], err[ident]))
    # the unidentified combination is still fitted: 1/BW_rd + 1/BW_wr
    assert 1 / theta[10] + 1 / theta[11] == pytest.approx(1 / truth[10] + 1 / truth[11], rel=1e-6)
    pred = O.model_batch(cols, theta, N_SM)
    assert C.mae_by_family(rows, pred)["all"]["mae_pct"] < 1e-6


def test_fit_leaves_dead_region_of_eq16():
    # A start with B_sus above B_peak: Eq. 16's blend then never beats the
    # B_peak floor, so (literal reading) B_sus and w0 have no gradient.  The
    # fit's ordering penalty moves it out, after which the data fix both.
    truth = C.prior_theta(N_SM)
    rows, cols = table(truth)
    t_meas = np.array([r["t"] for r in rows])
    start = truth.copy()
    start[1], start[2] = 1.4 * truth[2], 0.9 * truth[2]
    theta, _ = C.fit(lambda th: OracleLoss.apply(th, cols, t_meas), start, reg=0.0)
    assert abs(np.log(theta[1] / truth[1])) <= 1e-3 and abs(np.log(theta[3] / truth[3])) <= 1e-3


def test_split_is_seeded_and_disjoint():
    tr, ho = C.split(1000)
    tr2, ho2 = C.split(1000)
    assert np.array_equal(tr, tr2) and not np.any(tr & ho) and np.all(tr | ho)
    assert ho.sum() == 200


def test_mae_definition():
    rows = [dict(kind=0, dtype=1, t=1.0), dict(kind=0, dtype=1, t=2.0), dict(kind=1, dtype=0, t=4.0)]
    m = C.mae_by_family(rows, np.array([1.1, 1.8, 4.0]))
    assert m["bf16"]["mae_pct"] == pytest.approx(10.0)
    assert m["stream"]["mae_pct"] == pytest.approx(0.0)
    assert m["all"]["mae_pct"] == pytest.approx(20.0 / 3)


def test_eq15_fit_recovers_link_parameters():
    # Eq. 15: T = S / B_dir + tau; exact data gives back B and tau
    rows = [dict(bytes=b, h2d_s=b / 2.1e11 + 8e-6, d2h_s=b / 1.93e11 + 9e-6) for b in [2 ** k for k in range(12, 31, 2)]]
    f = C.fit_eq15(rows)
    assert f["h2d"]["B_eff"] == pytest.approx(2.1e11, rel=1e-9) and f["h2d"]["tau_s"] == pytest.approx(8e-6, rel=1e-9)
    assert f["d2h"]["B_eff"] == pytest.approx(1.93e11, rel=1e-9) and f["d2h"]["tau_s"] == pytest.approx(9e-6, rel=1e-9)


def test_probe_priors_replace_only_measured_parameters():
    instr = dict(mma=[dict(dtype=d, cta_group=1, M=128, N=256, tflops=t) for d, t in ((0, 1200.0), (1, 2400.0),
                                                                                        (2, 4800.0))],
                 mbar_round_trip_ns=100.0, tmem_ld_bytes_per_s_per_sm=2e12, tmem_st_bytes_per_s_per_sm=1e12)
    th = C.probe_priors(instr, N_SM)
    base = C.prior_theta(N_SM)
    assert th[6] == pytest.approx(1.2e15 / N_SM) and th[7] == pytest.approx(2.4e15 / N_SM)
    assert th[8] == pytest.approx(4.8e15 / N_SM)
    assert th[12] == pytest.approx(50e-9) and th[10] == 2e12 and th[11] == 1e12
    keep = [j for j in range(16) if j not in (6, 7, 8, 10, 11, 12)]
    assert np.array_equal(th[keep], base[keep])


def test_tau_c_fit_recovers_additive_law():
    # T(N_c) = T1 + (N_c - 1) tau_c exactly: the fit returns tau_c, MAE 0
    counts = C.STREAM_COUNTS
    t = [2e-5 + (n - 1) * 7e-6 for n in counts]
    f = C.fit_tau_c(counts, t)
    assert f["T1_s"] == 2e-5 and f["tau_c_s"] == pytest.approx(7e-6, rel=1e-12) and f["mae_pct"] < 1e-9
    # perfect overlap gives tau_c = 0; full serialisation gives tau_c = T1
    assert C.fit_tau_c(counts, [3e-5] * len(counts))["tau_c_s"] == pytest.approx(0.0, abs=1e-18)
    assert C.fit_tau_c(counts, [3e-5 * n for n in counts])["tau_over_T1"] == pytest.approx(1.0, rel=1e-12)


def test_pchase_levels_takes_medians_inside_each_level():
    W = [16384 * 2 ** k for k in range(17)]
    ns = [20.0 if w <= 128 * 1024 else (140.0 if w <= 64 * 2 ** 20 else 400.0) for w in W]
    ns[3] = 25.0                                   # one noisy L1 point: the median ignores it
    lv = C.pchase_levels([dict(W=w, ns_per_hop=v) for w, v in zip(W, ns)], 256 * 1024, 128 * 2 ** 20)
    assert lv["l1_ns"] == 20.0 and lv["l2_ns"] == 140.0 and lv["dram_ns"] == 400.0
    assert lv["l1_points"] == 4 and lv["dram_points"] == 2


def test_stream_interference_fit_recovers_kappas(monkeypatch):
    # makespans generated by the generic path's own concurrent-stream term
    # (the oracle standing in for pm_segment_predict): the least-squares fit
    # returns the generating kappas, and the MMA probe on an eighth of the SMs
    # is left out (no roofline term describes it)
    monkeypatch.setattr(C, "_seg_predict", lambda rows, th, psi, n: O.segment_predict(
        {f: np.array([r.get(f, 1 if f == "execs" else 0) for r in rows]) for f in C.SEG_FIELDS}, th, psi, n))
    th = O.prior_theta(N_SM)
    psi = np.array([1.0, 1.4, 2.0, 1.2, 0.05, 1.0, 0.9, 2.1e11, 3.6e-6, 1.9e11, 3.4e-6, 3.7e-6, 0, 0, 0, 0, 0])
    truth = psi.copy()
    truth[[12, 13, 14, 15, 16]] = [0.95, 1.1, 1.1, 0.95, 0.18]
    streams = {}
    for name in ("triad_2^24_per_stream", "copy_2^16_per_stream", "mma_bf16_%d_ctas_per_stream" % N_SM,
                 "mma_bf16_%d_ctas_per_stream" % (N_SM // 8)):
        seg = C.stream_segments(name, N_SM)
        if seg is None:
            streams[name] = dict(counts=list(C.STREAM_COUNTS), t_s=[5e-4 * c for c in C.STREAM_COUNTS])
            continue
        t = O.segment_predict({k: np.array([v] * 6) for k, v in seg.items()} | {"streams": np.array(C.STREAM_COUNTS)},
                              th, truth, N_SM)
        streams[name] = dict(counts=list(C.STREAM_COUNTS), t_s=t.tolist())
    f = C.fit_stream_interference(streams, th, psi, N_SM)
    assert f["kappa_launch"] == pytest.approx(0.18, rel=1e-9)
    assert f["kappa_memory"] == pytest.approx(0.95, rel=1e-9) and f["kappa_compute"] == pytest.approx(1.1, rel=1e-9)
    assert set(f["classes"]) == {"triad_2^24_per_stream", "copy_2^16_per_stream", "mma_bf16_%d_ctas_per_stream" % N_SM}
    assert all(v["mae_pct"] < 1e-9 for v in f["classes"].values())
