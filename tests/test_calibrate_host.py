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
    rows = []
    for s in (1024, 4096, 16384):
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
    cols = {f: np.array([r[f] for r in rows], dtype=np.int32) for f in FIELDS}
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


def test_prior_matches_oracle_prior():
    assert np.allclose(C.prior_theta(N_SM), O.prior_theta(N_SM), rtol=0, atol=0)


def test_fit_recovers_generating_parameters():
    prior = C.prior_theta(N_SM)
    noise = S.normal(5, 16).astype(np.float64)
    truth = prior * np.exp(0.3 * noise)
    truth[15] = 0.4                      # keep alpha's clamp inactive at every depth
    rows, cols = table(truth)
    t_meas = np.array([r["t"] for r in rows])
    theta, trace = C.fit(lambda th: OracleLoss.apply(th, cols, t_meas), prior, reg=0.0, iters=600)
    assert trace[-1] < 1e-3 * trace[0]
    pred = O.model_batch(cols, theta, N_SM)
    assert np.max(np.abs(pred - t_meas) / t_meas) < 0.02
    mae = C.mae_by_family(rows, pred)
    assert mae["all"]["mae_pct"] < 0.5


def test_split_is_seeded_and_disjoint():
    tr, ho = C.split(1000)
    tr2, ho2 = C.split(1000)
    assert np.array_equal(tr, tr2) and not np.any(tr & ho) and np.all(tr | ho)
    assert ho.sum() == 200


def test_mae_definition():
    rows = [dict(kind=0, dtype=1, t=1.0), dict(kind=0, dtype=1, t=2.0), dict(kind=1, dtype=0, t=4.0)]
    m = C.mae_by_family(rows, np.array([1.1, 1.8, 4.0]))
    assert m["3_bf16"]["mae_pct"] == pytest.approx(10.0)
    assert m["2a_stream"]["mae_pct"] == pytest.approx(0.0)
    assert m["all"]["mae_pct"] == pytest.approx(20.0 / 3)
