"""GPU parity of the generic segment model (Sec. III-E generic roofline path,
Eqs. 15-16) against the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_SM = 152


def random_segments(n, seed):
    u = [S.uniform01_f64(seed + k, n) for k in range(11)]
    return dict(flops=10 ** (6 + 9 * u[0]), bytes=10 ** (3 + 8 * u[1]), working_set=10 ** (3 + 8 * u[2]),
                h2d_bytes=np.where(u[3] < 0.5, 10 ** (3 + 7 * u[4]), 0.0),
                d2h_bytes=np.where(u[5] < 0.5, 10 ** (3 + 7 * u[4]), 0.0),
                cls=(4 * u[6]).astype(np.int32), precision=(3 * u[7]).astype(np.int32),
                kernels=(5 * u[8]).astype(np.int32), syncs=(3 * u[9]).astype(np.int32),
                execs=(1 + 8 * u[0]).astype(np.int32), streams=(5 * u[10]).astype(np.int32))


@pytest.mark.parametrize("n", [1, 1000, 100003])
def test_segment_predict_matches_oracle(lib, n):
    th = O.prior_theta(N_SM).astype(np.float32).astype(np.float64)
    psi = np.array([1.2, 1.1, 1.3, 1.5, 0.9, 1.0, 0.8, 2.1e11, 3.6e-6, 1.93e11, 3.4e-6, 1e-5, 0.9, 1.1, 0.6, 0.7, 0.2])
    s = random_segments(n, 40 + n)
    t_gpu = lib.pm_segment_predict(lib.segment_array(s), th, psi, N_SM)
    t_orc = O.segment_predict(s, th, psi, N_SM)
    assert np.all(np.abs(t_gpu - t_orc) <= 1e-12 * t_orc + 1e-300)


def test_segment_invalid_records_are_nan(lib):
    th = O.prior_theta(N_SM)
    s = dict(flops=np.array([1e9, 1e9, 1e9]), bytes=np.array([1e9, -1.0, 1e9]), kernels=np.array([1, 1, 1]),
             cls=np.array([0, 0, 7]))
    t = lib.pm_segment_predict(lib.segment_array(s), th, np.ones(lib.N_PSI), N_SM)
    assert np.isfinite(t[0]) and np.isnan(t[1]) and np.isnan(t[2])
