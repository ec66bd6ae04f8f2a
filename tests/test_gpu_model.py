"""GPU parity of the batched model, its adjoint and the autotuners against the
FP64 CPU oracle (1e-5 relative for predictions)."""
import numpy as np
import pytest

import oracle as O
import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_SM = 152
THETA = O.prior_theta(N_SM)
FIELDS = ("M", "N", "K", "BM", "BN", "BK", "stages", "cta_group", "dtype", "kind", "tmem_a")


def theta32():
    # the GPU takes FP32 parameters; the oracle gets the same rounded values
    return THETA.astype(np.float32).astype(np.float64)


def random_cfgs(n, seed=4, valid_only=False, strategy_b=False):
    c = S.model_config_batch(n, seed)
    c["kind"] = np.zeros(n, dtype=np.int32)
    if strategy_b:
        # half the rows ask for TMEM strategy B (the model evaluates any tile)
        c["tmem_a"] = (S.uniform01_f64(seed + 1000, n) < 0.5).astype(np.int32)
    if valid_only:
        ok = np.array([O.cfg_valid(c["BM"][i], c["BN"][i], c["BK"][i], c["stages"][i], c["cta_group"][i],
                                   c["dtype"][i]) for i in range(n)])
        c = {k: v[ok] for k, v in c.items()}
    return c


def probe_cfgs():
    rows = [dict(M=2 ** k + j, kind=1) for k in range(20, 31) for j in (0, 3)]
    rows += [dict(M=2 ** k, kind=2) for k in range(20, 31)]
    rows += [dict(M=16384, N=16384, BM=r, BN=c, kind=3) for r, c in ((64, 64), (128, 64), (128, 128), (256, 64),
                                                                     (256, 128))]
    return {f: np.array([r.get(f, 0) for r in rows], dtype=np.int32) for f in FIELDS}


def predict_gpu(lib, c, theta):
    n = len(c["M"])
    dev = lib.cfg_tensor(c)
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    lib.pm_model_predict(dev, n, theta, N_SM, out)
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("n", [1, 7, 1000, 100003])
def test_predict_matches_oracle(lib, reading, n):
    c = random_cfgs(n, seed=n, strategy_b=True)
    th = theta32()
    t_gpu = predict_gpu(lib, c, th)
    t_orc = O.model_batch(c, th, N_SM)
    assert np.all(np.abs(t_gpu - t_orc) <= 1e-5 * t_orc)


def test_predict_probes_and_fp32_512(lib, reading):
    th = theta32()
    c = probe_cfgs()
    assert np.all(np.abs(predict_gpu(lib, c, th) - O.model_batch(c, th, N_SM)) <= 1e-5 * O.model_batch(c, th, N_SM))
    one = {f: np.array([v], dtype=np.int32) for f, v in
           zip(FIELDS, (512, 512, 512, 128, 128, 32, 2, 1, 0, 0))}
    assert predict_gpu(lib, one, th)[0] == pytest.approx(O.model_batch(one, th, N_SM)[0], rel=1e-5)


def test_predict_invalid_records_are_nan(lib):
    c = {f: np.array([v], dtype=np.int32) for f, v in zip(FIELDS, (512, 512, 512, 0, 128, 32, 2, 1, 0, 0))}
    assert np.isnan(predict_gpu(lib, c, theta32())[0])


def test_predict_million_configs(lib):
    n = 10 ** 6
    c = random_cfgs(n, seed=4)
    th = theta32()
    t_gpu = predict_gpu(lib, c, th)
    idx = S.sampled_rows(5, n, 20000)
    sub = {k: v[idx] for k, v in c.items()}
    t_orc = O.model_batch(sub, th, N_SM)
    assert np.all(np.abs(t_gpu[idx] - t_orc) <= 1e-5 * t_orc)


def grad_gpu(lib, c, theta, t_meas):
    n = len(c["M"])
    dev = lib.cfg_tensor(c)
    tm = torch.from_numpy(t_meas.astype(np.float32)).cuda()
    ws = torch.empty(lib.pm_model_grad_workspace(n) // 8, dtype=torch.float64, device="cuda")
    out = torch.empty(lib.N_GRAD_OUT, dtype=torch.float64, device="cuda")
    lib.pm_model_grad(dev, n, theta, N_SM, tm, ws, out)
    o = out.cpu().numpy()
    return o[0], o[1:]


@pytest.mark.parametrize("n", [1, 1000, 200000])
def test_grad_matches_oracle(lib, reading, n):
    c = random_cfgs(n, seed=17 + n, strategy_b=True)
    pc = probe_cfgs()
    c = {k: np.concatenate([c[k], pc[k]]) for k in c}
    th = theta32()
    t_true = O.model_batch(c, th, N_SM)
    noise = S.uniform01_f64(23, len(t_true))
    t_meas = (t_true * np.exp(0.3 * (noise - 0.5))).astype(np.float32).astype(np.float64)
    L_gpu, g_gpu = grad_gpu(lib, c, th, t_meas)
    L_orc, g_orc = O.model_loss_grad(c, th, N_SM, t_meas)
    assert L_gpu == pytest.approx(L_orc, rel=1e-4, abs=1e-9)
    # per-component scale: the sum of absolute contributions (FP32 terms)
    _, gi = O.model_batch(c, th, N_SM, grad=True)
    r = np.log(t_true) - np.log(t_meas)
    scale = (2.0 / len(r)) * np.sum(np.abs(r[:, None] * gi / t_true[:, None]), axis=0)
    assert np.all(np.abs(g_gpu - g_orc) <= 1e-4 * scale + 1e-30), (g_gpu, g_orc, scale)


def test_autotune_matches_oracle(lib, reading):
    rng = S.splitmix64(31, 3 * 600)
    MNK = (16 * (1 + (rng >> np.uint64(40)) % np.uint64(1024))).astype(np.int32).reshape(-1, 3)
    MNK = np.concatenate([MNK, np.array([[512, 512, 512], [8192, 8192, 8192], [16384, 16384, 16384]], np.int32)])
    th = theta32()
    for dt in (0, 1, 2):
        n = len(MNK)
        picks = torch.empty(n * 24, dtype=torch.uint8, device="cuda")
        t = torch.empty(n, dtype=torch.float32, device="cuda")
        lib.pm_autotune_pick(torch.from_numpy(MNK.ravel()).cuda(), n, dt, th, N_SM, picks, t)
        p = picks.cpu().numpy().view(lib.CFG_DTYPE)
        pick_o, t_o = O.autotune(MNK, dt, th, N_SM)
        got = np.stack([p["BM"], p["BN"], p["BK"], p["stages"], p["cta_group"]], 1)
        same = np.all(got == pick_o, axis=1)
        # a different pick is allowed only where the oracle's own FP64
        # predictions of the two candidates are within FP32 resolution
        for i in np.nonzero(~same)[0]:
            alt = {f: np.array([v], dtype=np.int32) for f, v in
                   zip(FIELDS, (*MNK[i], *got[i], dt, 0))}
            t_alt = O.model_batch(alt, th, N_SM)[0]
            assert abs(t_alt - t_o[i]) <= 1e-6 * t_o[i], (MNK[i], got[i], pick_o[i])
        assert same.mean() > 0.95
        assert np.all(np.abs(t.cpu().numpy() - t_o) <= 1e-5 * t_o)


def test_autotune_million_configs_per_launch(lib):
    n_shapes = 10 ** 6 // 180 + 1
    c = S.model_config_batch(n_shapes, seed=4)
    MNK = np.stack([c["M"], c["N"], c["K"]], 1).astype(np.int32)
    picks = torch.empty(n_shapes * 24, dtype=torch.uint8, device="cuda")
    t = torch.empty(n_shapes, dtype=torch.float32, device="cuda")
    th = theta32()
    lib.pm_autotune_pick(torch.from_numpy(MNK.ravel()).cuda(), n_shapes, 1, th, N_SM, picks, t)
    idx = S.sampled_rows(3, n_shapes, 200)
    _, t_o = O.autotune(MNK[idx], 1, th, N_SM)
    assert np.all(np.abs(t.cpu().numpy()[idx] - t_o) <= 1e-5 * t_o)


def test_grouped_autotune_matches_oracle(lib, reading):
    Mg = S.grouped_m(64, 3)
    th = theta32()
    t_g, bm_g, bn_g, launch_g = lib.pm_grouped_autotune(Mg, 4096, 4096, 1, th, N_SM)
    t_o, bm_o, bn_o, launch_o = O.grouped_autotune(Mg, 4096, 4096, 1, th, N_SM)
    assert t_g == pytest.approx(t_o, rel=1e-5)
    # the GPU's choice evaluated by the oracle is as good as the oracle's
    t_check = O.grouped_predict(Mg, 4096, 4096, bm_g, bn_g, *launch_g, 1, th, N_SM)
    assert t_check == pytest.approx(t_o, rel=1e-5)


def test_autotune_topk_matches_oracle_order(lib, reading):
    th = theta32()
    MNK = np.array([[512, 512, 512], [1024, 2048, 4096], [8192, 8192, 8192], [300, 5000, 1000]], np.int32)
    k = 8
    for dt in (0, 1, 2):
        n = len(MNK)
        picks = torch.empty(n * k * 24, dtype=torch.uint8, device="cuda")
        t = torch.empty(n * k, dtype=torch.float32, device="cuda")
        lib.pm_autotune_topk(torch.from_numpy(MNK.ravel()).cuda(), n, dt, th, N_SM, k, picks, t)
        p = picks.cpu().numpy().view(lib.CFG_DTYPE).reshape(n, k)
        tg = t.cpu().numpy().reshape(n, k).astype(np.float64)
        for i, (M, N, K) in enumerate(MNK):
            space = [c for c in S.tile_space(dt) if O.cfg_valid(*c, dt)]
            cols = {f: np.array(v, dtype=np.int32) for f, v in zip(("BM", "BN", "BK", "stages", "cta_group"),
                                                                    zip(*space))}
            cols.update(M=np.full(len(space), M), N=np.full(len(space), N), K=np.full(len(space), K),
                        dtype=np.full(len(space), dt), kind=np.zeros(len(space)))
            to = O.model_batch(cols, th, N_SM)
            order = np.argsort(to, kind="stable")[:k]
            assert np.all(np.abs(tg[i] - to[order]) <= 1e-5 * to[order])
            got = [tuple(int(p[i, r][f]) for f in ("BM", "BN", "BK", "stages", "cta_group")) for r in range(k)]
            assert np.all(np.diff(tg[i]) >= 0)
            for r in range(k):   # each pick's own FP64 prediction sits at its rank (up to FP32 resolution)
                j = space.index(got[r])
                assert abs(to[j] - to[order[r]]) <= 2e-6 * to[order[r]]


@pytest.mark.parametrize("n", [1, 1000, 50000])
def test_grad_f64_matches_oracle_tightly(lib, reading, n):
    # the all-FP64 objective agrees with the FP64 oracle to rounding order
    c = random_cfgs(n, seed=29 + n, strategy_b=True)
    pc = probe_cfgs()
    c = {k: np.concatenate([c[k], pc[k]]) for k in c}
    th = THETA.copy()
    t_true = O.model_batch(c, th, N_SM)
    t_meas = t_true * np.exp(0.3 * (S.uniform01_f64(31, len(t_true)) - 0.5))
    dev = lib.cfg_tensor(c)
    m = len(t_meas)
    ws = torch.empty(lib.pm_model_grad_workspace(m) // 8, dtype=torch.float64, device="cuda")
    out = torch.empty(lib.N_GRAD_OUT, dtype=torch.float64, device="cuda")
    lib.pm_model_grad_f64(dev, m, th, N_SM, torch.from_numpy(t_meas).cuda(), ws, out)
    o = out.cpu().numpy()
    L_orc, g_orc = O.model_loss_grad(c, th, N_SM, t_meas)
    assert o[0] == pytest.approx(L_orc, rel=1e-10)
    _, gi = O.model_batch(c, th, N_SM, grad=True)
    r = np.log(t_true) - np.log(t_meas)
    scale = (2.0 / len(r)) * np.sum(np.abs(r[:, None] * gi / t_true[:, None]), axis=0)
    assert np.all(np.abs(o[1:] - g_orc) <= 1e-10 * scale + 1e-300), (o[1:], g_orc)


def test_grouped_predict_matches_oracle(lib, reading):
    Mg = S.grouped_m(64, 3)
    th = theta32()
    G = len(Mg)
    bm = [(64, 128, 256)[q % 3] for q in range(G)]
    bn = [(128, 256, 64)[q % 3] for q in range(G)]
    for launch in ((64, 4, 1), (128, 3, 2), (128, 2, 2)):
        t_g = lib.pm_grouped_predict(Mg, 4096, 4096, bm, bn, *launch, 1, th, N_SM)
        t_o = O.grouped_predict(Mg, 4096, 4096, bm, bn, *launch, 1, th, N_SM)
        assert t_g == pytest.approx(t_o, rel=1e-5)


@pytest.mark.parametrize("launch", [(64, 4, 1), (128, 3, 2), (64, 2, 1)])
def test_grouped_grad_matches_oracle(lib, reading, launch):
    # FP64 makespan and its gradient (the busiest worker's tiles through the
    # tile adjoint) against the oracle's dual numbers, mixed tiles so the
    # launch reorders its groups
    Mg = S.grouped_m(48, 7)
    th = O.prior_theta(N_SM, reading=reading)
    G = len(Mg)
    bm = [(64, 128, 256)[q % 3] for q in range(G)]
    bn = [(128, 256, 64)[(q // 3) % 3] for q in range(G)]
    bm = [b if O.cfg_valid(b, n, *launch, 1) else 64 for b, n in zip(bm, bn)]
    t_g, g_g = lib.pm_grouped_grad(Mg, 2048, 4096, bm, bn, *launch, 1, th, N_SM)
    t_o, g_o = O.grouped_predict_grad(Mg, 2048, 4096, bm, bn, *launch, 1, th, N_SM)
    assert t_g == pytest.approx(t_o, rel=1e-12)
    scale = np.abs(g_o * th).max()
    assert np.all(np.abs((g_g - g_o) * th) <= 1e-10 * scale), (g_g, g_o)


def test_pairs_on_fewer_than_two_sms(lib, reading):
    # one SM: pair records (cta_group 2) are NaN and never picked, as in the
    # oracle; one-SM records match it (every tile its own wave).  Three SMs:
    # one-SM tiles divide by 3, pairs by 2 (the invariant-divisor path)
    th = theta32()
    c = random_cfgs(2000, seed=77, strategy_b=True)
    n = len(c["M"])
    dev = lib.cfg_tensor(c)
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    pair = c["cta_group"] == 2
    for n_sm in (1, 3):
        lib.pm_model_predict(dev, n, th, n_sm, out)
        t_gpu = out.cpu().numpy().astype(np.float64)
        t_orc = O.model_batch(c, th, n_sm)
        if n_sm == 1:
            assert pair.any() and np.all(np.isnan(t_gpu[pair])) and np.all(np.isnan(t_orc[pair]))
            ok = ~pair
        else:
            ok = np.ones(n, dtype=bool)
        assert np.all(np.abs(t_gpu[ok] - t_orc[ok]) <= 1e-5 * t_orc[ok])
    MNK = np.array([[512, 512, 512], [4096, 1024, 2048], [16, 16384, 64]], dtype=np.int32)
    for n_sm in (1, 3):
        picks = torch.empty(3 * 24, dtype=torch.uint8, device="cuda")
        t = torch.empty(3, dtype=torch.float32, device="cuda")
        lib.pm_autotune_pick(torch.from_numpy(MNK.ravel()).cuda(), 3, 1, th, n_sm, picks, t)
        p = picks.cpu().numpy().view(lib.CFG_DTYPE)
        _, t_o = O.autotune(MNK, 1, th, n_sm)
        if n_sm == 1:
            assert np.all(p["cta_group"] == 1)
        assert np.all(np.abs(t.cpu().numpy() - t_o) <= 1e-5 * t_o)
    Mg = S.grouped_m(16, 3)
    t_g, _, _, launch_g = lib.pm_grouped_autotune(Mg, 1024, 1024, 1, th, 1)
    t_o, _, _, launch_o = O.grouped_autotune(Mg, 1024, 1024, 1, th, 1)
    assert launch_g[2] == 1 and launch_o[2] == 1 and t_g == pytest.approx(t_o, rel=1e-5)
    bm = [128] * len(Mg)
    assert np.isnan(lib.pm_grouped_predict(Mg, 1024, 1024, bm, bm, 64, 4, 2, 1, th, 1))
    assert np.isnan(O.grouped_predict(Mg, 1024, 1024, bm, bm, 64, 4, 2, 1, th, 1))
