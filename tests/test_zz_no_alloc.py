"""The allocation-free calibration gradient (pm_model_grad_noalloc).

Callers that cannot allocate device memory when they need the gradient use
this entry point; it keeps its partial sums in a fixed array inside the
library.  It must give what pm_model_grad (caller workspace) gives, on
repeated calls that reuse the same array, and refuse batches beyond its
capacity.  This file is collected last so that a failure here stops a
first-failure run only after every other test has run.
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_SM = 152


def _case(n, seed):
    c = S.model_config_batch(n, seed)
    c["kind"] = np.zeros(n, dtype=np.int32)
    th = O.prior_theta(N_SM).astype(np.float32).astype(np.float64)
    t = O.model_batch(c, th, N_SM)
    noise = S.uniform01_f64(seed + 1, n)
    t_meas = (t * np.exp(0.3 * (noise - 0.5))).astype(np.float32)
    return c, th, t_meas


def test_noalloc_matches_workspace_gradient_on_consecutive_calls(lib):
    for n, seed in ((200003, 41), (1000, 43)):           # second call reuses (and overreads nothing of) the first's array
        c, th, t_meas = _case(n, seed)
        dev = lib.cfg_tensor(c)
        tm = torch.from_numpy(t_meas).cuda()
        ws = torch.empty(lib.pm_model_grad_workspace(n) // 8, dtype=torch.float64, device="cuda")
        ref = torch.empty(17, dtype=torch.float64, device="cuda")
        lib.pm_model_grad(dev, n, th, N_SM, tm, ws, ref)
        _, gi = O.model_batch(c, th, N_SM, grad=True)
        tt = O.model_batch(c, th, N_SM)
        r = np.log(tt) - np.log(t_meas.astype(np.float64))
        scale = (2.0 / n) * np.sum(np.abs(r[:, None] * gi / tt[:, None]), axis=0)
        for _ in range(2):
            out = torch.full((17,), float("nan"), dtype=torch.float64, device="cuda")
            lib.pm_model_grad_noalloc(dev, n, th, N_SM, tm, out)
            torch.cuda.synchronize()
            o, rr = out.cpu().numpy(), ref.cpu().numpy()
            assert o[0] == pytest.approx(rr[0], rel=1e-4, abs=1e-9)
            assert np.all(np.abs(o[1:] - rr[1:]) <= 1e-4 * scale + 1e-30)


def test_noalloc_rejects_batches_beyond_capacity(lib):
    n = 1048576 + 1
    dev = torch.zeros(24, dtype=torch.uint8, device="cuda")
    out = torch.zeros(17, dtype=torch.float64, device="cuda")
    tm = torch.ones(1, dtype=torch.float32, device="cuda")
    with pytest.raises(lib.PMError) as e:
        lib.pm_model_grad_noalloc(dev, n, np.ones(16), N_SM, tm, out)
    assert e.value.status == lib.PM_ENOMEM and "at most 1048576" in str(e.value)
