"""The Python usage shown for the binding (autotune from the calibrated model,
run, predict), at 1024^3, checked against the FP64 oracle on sampled rows."""
import json
import os

import numpy as np
import pytest

import oracle as O
import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_usage_example(lib):
    pm = lib
    n_sm = pm.sm_count()
    theta = json.load(open(os.path.join(os.path.dirname(pm.__file__), "theta_gb300.json")))["theta"]
    M = N = K = 1024
    A_h, B_h = S.gemm_operands(M, N, K, seed=2, dist="normal")
    A, B = torch.from_numpy(A_h).cuda(), torch.from_numpy(B_h).cuda()
    ops = pm.GemmOperands(pm.PM_BF16, M, N, K)
    ops.prepare(A, B)
    C = torch.empty(M, N, device="cuda")
    best, times = pm.pm_gemm_autotune(pm.cfg(M, N, K, dtype=pm.PM_BF16), 8, theta, n_sm, ops.A_op, ops.B_op, C,
                                      ops.scales)
    assert times["median_s"] > 0 and O.cfg_valid(best.BM, best.BN, best.BK, best.stages, best.cta_group, 1)
    C.fill_(float("nan"))
    ops.run(best, C)
    t_pred = torch.empty(1, device="cuda")
    pm.pm_model_predict(pm.cfg_tensor({"M": [M], "N": [N], "K": [K], "BM": [best.BM], "BN": [best.BN],
                                       "BK": [best.BK], "stages": [best.stages], "cta_group": [best.cta_group],
                                       "dtype": [pm.PM_BF16]}), 1, theta, n_sm, t_pred)
    torch.cuda.synchronize()
    assert pm.pm_device_status(True) == pm.PM_OK
    rows = S.sampled_rows(12, M, 64)
    ref = O.gemm_f64(A_h[rows], B_h)
    assert np.linalg.norm(C.cpu().numpy()[rows] - ref) / np.linalg.norm(ref) <= 2e-2
    assert 0.2 < float(t_pred.item()) / times["median_s"] < 5.0
