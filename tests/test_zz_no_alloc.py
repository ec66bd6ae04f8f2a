"""The allocation-free calibration gradient (pm_model_grad_noalloc).

Some callers cannot allocate device memory when they need the gradient: a
host program that links only this library and owns no CUDA allocator, or a
runtime held to a fixed device-memory budget.  This entry point keeps its
partial sums in a fixed array inside the library instead of a caller
workspace.  On two calls in a row, which reuse that array, it must give the
FP64 oracle's loss and gradient within the tolerance the other gradient
tests use, and exactly what pm_model_grad gives (same grid, same summation
order); it must refuse batches beyond its capacity.  This file is collected
last so that a failure here stops a first-failure run only after every
other test has run.
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


def test_noalloc_matches_oracle_on_consecutive_calls(lib):
    # the second batch is smaller than the first, so its call reuses (and must
    # not read stale) partial records the first call left in the array
    for n, seed in ((200003, 41), (1000, 43)):
        c, th, t_meas = _case(n, seed)
        dev = lib.cfg_tensor(c)
        tm = torch.from_numpy(t_meas).cuda()
        # the FP64 oracle: loss and gradient, and the scale of the gradient's
        # summands (FP32 per-configuration terms are compared against it)
        L_o, g_o = O.model_loss_grad(c, th, N_SM, t_meas.astype(np.float64))
        _, gi = O.model_batch(c, th, N_SM, grad=True)
        tt = O.model_batch(c, th, N_SM)
        r = np.log(tt) - np.log(t_meas.astype(np.float64))
        scale = (2.0 / n) * np.sum(np.abs(r[:, None] * gi / tt[:, None]), axis=0)
        # the workspace entry point on the same inputs
        ws = torch.empty(lib.pm_model_grad_workspace(n) // 8, dtype=torch.float64, device="cuda")
        ref = torch.empty(lib.N_GRAD_OUT, dtype=torch.float64, device="cuda")
        lib.pm_model_grad(dev, n, th, N_SM, tm, ws, ref)
        rr = ref.cpu().numpy()
        for _ in range(2):
            out = torch.full((lib.N_GRAD_OUT,), float("nan"), dtype=torch.float64, device="cuda")
            lib.pm_model_grad_noalloc(dev, n, th, N_SM, tm, out)
            torch.cuda.synchronize()
            o = out.cpu().numpy()
            assert o[0] == pytest.approx(L_o, rel=1e-4)
            assert np.all(np.abs(o[1:] - g_o) <= 1e-4 * scale + 1e-30)
            assert np.array_equal(o, rr)


def test_noalloc_rejects_batches_beyond_capacity(lib):
    n = 1048576 + 1
    dev = torch.zeros(24, dtype=torch.uint8, device="cuda")
    out = torch.zeros(lib.N_GRAD_OUT, dtype=torch.float64, device="cuda")
    tm = torch.ones(1, dtype=torch.float32, device="cuda")
    with pytest.raises(lib.PMError) as e:
        lib.pm_model_grad_noalloc(dev, n, np.ones(lib.N_PARAMS), N_SM, tm, out)
    assert e.value.status == lib.PM_ENOMEM and "at most 1048576" in str(e.value)
