"""GPU parity of the plain FP32 path against the FP64 oracle (through the
C ABI). Tolerances: bit-exact for integers (coordinates, indices); FP32
single-step forward and gradients within 1e-5 relative (normwise for sums
over the batch, plus the kink allowance of parity.py); PSNR after N seeded
steps within 0.2 dB."""
import math

import numpy as np
import pytest

import parity as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_10516_gb300 import model as dv

    return dv


def _model(dv, c, seed, lo=(0, 0, 0), hi=(64, 64, 64), ghost=0):
    enc = dv.EncodingConfig(c["L"], c["F"], c["log2T"], c["base"], c["growth"])
    mlp = dv.MLPConfig(c["width"], c["hidden"])
    return dv.Model(lo, hi, ghost, enc, mlp, seed=seed)


def test_init_matches_oracle_bit_exact(dv, orc):
    c = P.configs_blobs64()
    m = _model(dv, c, seed=12345)
    w = m.get_weights()
    want = orc.init_params(P.oracle_cfg(c), 12345).astype(np.float32)
    np.testing.assert_array_equal(w, want)


def test_corner_indices_bit_exact(dv, orc):
    c = P.configs_spectral256()
    m = _model(dv, c, seed=1, hi=(256, 256, 256))
    oc = P.oracle_cfg(c)
    rng = np.random.default_rng(3)
    coords = rng.integers(0, (1 << 24) + 1, size=(2000, 3)).astype(np.uint32)
    coords[:8] = [[0, 0, 0], [1 << 24] * 3, [(1 << 24) - 1] * 3, [1 << 23, 0, 1 << 24],
                  [1, 2, 3], [0, 1 << 24, 0], [12345, 678910, 1 << 22], [5, 5, 5]]
    got = m.corner_indices(torch.from_numpy(coords.view(np.int32)).cuda()).cpu().numpy().view(np.uint32)
    for i in range(0, 2000, 7):
        for l in range(oc.L):
            N = oc.N[l]
            b = [min((int(v) * N) >> 24, N - 1) for v in coords[i]]
            for k in range(8):
                want = orc.corner_index(oc, l, b[0] + (k & 1), b[1] + ((k >> 1) & 1), b[2] + ((k >> 2) & 1))
                assert got[i, l, k] == want


@pytest.mark.parametrize("lam,loss", [(0.0, 0), (0.15, 0), (0.0, 1)])
def test_fp32_step_matches_oracle(dv, orc, lam, loss):
    from paper_2304_10516_gb300 import volumes

    c = P.configs_blobs64()
    oc = P.oracle_cfg(c)
    vol = volumes.blobs(64, seed=1001)
    theta = P.random_theta(oc, 21)
    m = _model(dv, c, seed=0)
    m.set_weights(theta)
    lam32 = float(np.float32(lam))
    cfg = dv.TrainConfig(batch=c["batch"], lambda_bnd=lam32, sigma_bnd=0.005, loss=loss, seed=77)
    out = m.train_grad(torch.from_numpy(vol).cuda(), cfg, iteration=3)
    torch.cuda.synchronize()
    # sampling: bit-exact coordinates (uniform and boundary samples)
    qtab = orc.quantile_table(float(np.float32(0.005)))
    coords = orc.sample(77, 0, 3, c["batch"], lam32, qtab)
    np.testing.assert_array_equal(out["coords"].cpu().numpy().view(np.uint32), coords)
    # targets: trilinear of the normalised volume
    t = orc.targets(vol, coords, float(vol.min()), float(vol.max()))
    np.testing.assert_allclose(out["target"].cpu().numpy(), t, atol=2e-6, rtol=0)
    th64 = theta.astype(np.float64)
    r = orc.fwd_bwd(oc, th64, coords, t, loss=loss, want_zabs=True)
    y = out["y"].cpu().numpy()
    np.testing.assert_allclose(y, r["y"], atol=1e-5 * max(1.0, np.abs(r["y"]).max()), rtol=0)
    assert abs(out["loss"].item() - r["loss"]) <= 1e-5 * max(r["loss"], 1e-3)
    a_enc, a_mlp, flagged = P.kink_allowance(oc, th64, coords, t, loss, False, 1.0, c["batch"],
                                             r["zabs"], delta=1e-5)
    keep = np.ones(c["batch"], bool)
    keep[flagged] = False
    assert keep.sum() > 0.95 * c["batch"]
    dx0 = out["dx0"].cpu().numpy()
    P.assert_normwise(dx0[keep], r["dx0"][keep], 1e-5, what="dL/dx0")
    g = out["grad"].cpu().numpy()
    P.assert_normwise(g[: oc.n_enc], r["grad_enc"], 1e-5, a_enc, what="table grad")
    P.assert_normwise(g[oc.n_enc:], r["grad_mlp"], 1e-5, a_mlp, what="mlp grad")


def _oracle_train_psnr(orc, oc, vol, theta, lr, steps, seed, batch):
    th = theta.copy()
    m1, m2 = np.zeros_like(th), np.zeros_like(th)
    tc = orc.TrainConfig(batch=batch, lr=float(np.float32(lr)), seed=seed)
    st = orc.State()
    hist = orc.train(oc, tc, st, th, m1, m2, vol, float(vol.min()), float(vol.max()), steps)
    dec = orc.decode_grid(oc, th, vol.shape[::-1], 0, float(vol.min()), float(vol.max()))
    mse, _ = orc.mse(dec, vol)
    return P.psnr(mse), hist


def _gpu_train_psnr(dv, c, vol, seed_model, lr, steps, seed):
    m = _model(dv, c, seed=seed_model)
    cfg = dv.TrainConfig(batch=c["batch"], steps=steps, lr=lr, seed=seed)
    vt = torch.from_numpy(vol).cuda()
    losses = dv.train([m], [vt], cfg)
    st = m.state()
    assert st["adam_t"] == steps and st["iter"] == steps and st["skipped"] == 0
    sse, _ = dv.error_stats(m.decode_grid(), vt)
    return P.psnr(sse / vol.size), losses[0], m


def test_fp32_training_psnr_matches_oracle(dv, orc):
    # Trajectory parity after 200 seeded steps of the 64^3 workload at
    # lr = 5e-4, where the oracle's own PSNR spreads by 0.013 dB (standard
    # deviation over 1e-7 relative perturbations of its initial weights; at
    # lr = 1e-3 the 200-step point falls in a fast-changing phase of training
    # and the spread is 0.05 dB in FP64 and 0.19 dB with FP16 rounding).
    from paper_2304_10516_gb300 import volumes

    c = P.configs_blobs64()
    oc = P.oracle_cfg(c)
    vol = volumes.blobs(64, seed=1001)
    psnr_gpu, loss_gpu, m = _gpu_train_psnr(dv, c, vol, 4242, 5e-4, 200, 99)
    psnr_orc, hist = _oracle_train_psnr(orc, oc, vol, orc.init_params(oc, 4242), 5e-4, 200, 99,
                                        c["batch"])
    assert abs(psnr_gpu - psnr_orc) < 0.2, (psnr_gpu, psnr_orc)
    assert abs(loss_gpu - hist[-1]) < 0.1 * hist[-1]
    # the learned network gains over its untrained initialisation
    m0 = _model(dv, c, seed=4242)
    sse0, _ = dv.error_stats(m0.decode_grid(), torch.from_numpy(vol).cuda())
    assert psnr_gpu > P.psnr(sse0 / vol.size) + 10.0


def test_fp32_training_chaotic_regime_matches_oracle_ensemble(dv, orc):
    # At lr = 1e-2 (the workload's setting) training is chaotic: a 1e-6
    # relative perturbation of the initial weights moves the 200-step PSNR by
    # several dB, so single runs cannot be compared. Both sides instead train
    # the same K perturbed initialisations (FP32 values, widened exactly for
    # the oracle) and the mean PSNRs of the two ensembles must agree within
    # three standard errors of their difference (a two-sample z-test, floored
    # at 0.5 dB). The runs' PSNRs are draws of one distribution with a heavy
    # lower tail (a run that falls into a bad trajectory ends several dB
    # lower), so single runs are not bounded by the other ensemble's range;
    # the two samples must instead not differ in location by a rank-sum
    # (Mann-Whitney U) test at p >= 1e-3.
    from paper_2304_10516_gb300 import volumes

    K = 12
    c = P.configs_blobs64()
    oc = P.oracle_cfg(c)
    vol = volumes.blobs(64, seed=1001)
    vt = torch.from_numpy(vol).cuda()
    th0 = orc.init_params(oc, 4242)
    rng = np.random.default_rng(1)
    p_gpu, p_orc = [], []
    for _ in range(K):
        th = (th0 * (1 + 1e-6 * rng.standard_normal(th0.size))).astype(np.float32)
        m = _model(dv, c, seed=0)
        m.set_weights(th)
        cfg = dv.TrainConfig(batch=c["batch"], steps=200, lr=1e-2, seed=99)
        dv.train([m], [vt], cfg)
        sse, _ = dv.error_stats(m.decode_grid(), vt)
        p_gpu.append(P.psnr(sse / vol.size))
        m.close()
        p_orc.append(_oracle_train_psnr(orc, oc, vol, th.astype(np.float64), 1e-2, 200, 99,
                                        c["batch"])[0])
    p_gpu, p_orc = np.array(p_gpu), np.array(p_orc)
    se = math.sqrt(p_gpu.var(ddof=1) / K + p_orc.var(ddof=1) / K)
    tol = max(0.5, 3.0 * se)
    assert abs(p_gpu.mean() - p_orc.mean()) <= tol, (p_gpu, p_orc, tol)
    stats = pytest.importorskip("scipy.stats")
    p = stats.mannwhitneyu(p_gpu, p_orc, alternative="two-sided").pvalue
    assert p >= 1e-3, (p, p_gpu, p_orc)


def test_decode_grid_and_points_match_oracle(dv, orc):
    c = P.configs_blobs64()
    oc = P.oracle_cfg(c)
    theta = P.random_theta(oc, 5, table_scale=0.3)
    lo, hi, g = (10, 20, 30), (40, 44, 50), 1
    m = _model(dv, c, seed=0, lo=lo, hi=hi, ghost=g)
    m.set_weights(theta)
    dec = m.decode_grid().cpu().numpy()
    dims = [h - l + 2 * g for l, h in zip(lo, hi)]
    # value range of a fresh model is [0, 1]
    want = orc.decode_grid(oc, theta.astype(np.float64), dims, g, 0.0, 1.0)
    np.testing.assert_allclose(dec, want, atol=1e-5 * max(1.0, np.abs(want).max()), rtol=0)
    # points: global voxel coordinates mapped to the unit domain
    rng = np.random.default_rng(8)
    xyz = np.stack([rng.uniform(l - g, h + g - 1, 3000) for l, h in zip(lo, hi)], 1).astype(np.float32)
    got = m.decode_points(torch.from_numpy(xyz).cuda()).cpu().numpy()
    u = (xyz.astype(np.float64) - (np.array(lo) - g)) / (np.array(dims) - 1)
    mm = np.rint(np.clip(u, 0, 1) * (1 << 24)).astype(np.uint32)
    want_p = orc.decode_unit(oc, theta.astype(np.float64), mm, 0.0, 1.0)
    np.testing.assert_allclose(got, want_p, atol=2e-5 * max(1.0, np.abs(want_p).max()), rtol=0)


def test_render_matches_oracle(dv, orc):
    c = dict(P.configs_blobs64(), width=16, hidden=1)
    oc = P.oracle_cfg(c)
    theta = P.random_theta(oc, 6, table_scale=0.5)
    lo, hi = (0, 0, 0), (32, 32, 32)
    m = _model(dv, c, seed=0, lo=lo, hi=hi)
    m.set_weights(theta)
    tf = dv.make_tf(alpha_max=0.05, v_lo=-0.5, v_hi=0.5)
    img = dv.render([m], tf, 64, 32, 128).cpu().numpy()
    grid = orc.decode_grid(oc, theta.astype(np.float64), (32, 32, 32), 0, 0.0, 1.0)
    tfv = [0.1, 0.2, 0.6, 1.0, 0.9, 0.2, 0.05, -0.5, 0.5]
    want = orc.render([grid], [lo], [hi], [float(np.float32(v)) for v in tfv], 64, 32, 128)
    np.testing.assert_allclose(img, want, atol=2e-4, rtol=0)


def test_render_two_blocks_front_to_back(dv, orc):
    c = dict(P.configs_blobs64(), width=16, hidden=1)
    oc = P.oracle_cfg(c)
    boxes = [((0, 0, 16), (16, 16, 32)), ((0, 0, 0), (16, 16, 16))]
    ms, grids = [], []
    for i, (lo, hi) in enumerate(boxes):
        theta = P.random_theta(oc, 30 + i, table_scale=0.5)
        m = _model(dv, c, seed=0, lo=lo, hi=hi)
        m.set_weights(theta)
        ms.append(m)
        grids.append(orc.decode_grid(oc, theta.astype(np.float64), (16, 16, 16), 0, 0.0, 1.0))
    tf = dv.make_tf(alpha_max=0.1, v_lo=-0.5, v_hi=0.5)
    img = dv.render(ms, tf, 16, 16, 64).cpu().numpy()
    tfv = [0.1, 0.2, 0.6, 1.0, 0.9, 0.2, 0.1, -0.5, 0.5]
    want = orc.render(grids, [b[0] for b in boxes], [b[1] for b in boxes],
                      [float(np.float32(v)) for v in tfv], 16, 16, 64)
    np.testing.assert_allclose(img, want, atol=2e-4, rtol=0)


def test_error_stats_fp64(dv):
    rng = np.random.default_rng(0)
    a = rng.normal(size=1_000_003).astype(np.float32)
    b = (a + rng.normal(scale=1e-3, size=a.size)).astype(np.float32)
    sse, mx = dv.error_stats(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda())
    d = a.astype(np.float64) - b.astype(np.float64)
    assert sse == pytest.approx(float((d * d).sum()), rel=1e-12)
    assert mx == float(np.abs(d).max())


def test_nonfinite_volume_is_reported(dv):
    from paper_2304_10516_gb300 import _abi as A

    c = P.configs_blobs64()
    m = _model(dv, c, seed=0, hi=(16, 16, 16))
    vol = torch.rand((16, 16, 16), device="cuda")
    vol[3, 4, 5] = float("nan")
    with pytest.raises(A.DvnrError) as e:
        dv.train([m], [vol], dv.TrainConfig(batch=256, steps=1))
    assert e.value.status == 4


def test_weights_roundtrip_and_warm_start(dv):
    c = P.configs_blobs64()
    a = _model(dv, c, seed=1, hi=(16, 16, 16))
    b = _model(dv, c, seed=2, hi=(16, 16, 16))
    vol = torch.rand((16, 16, 16), device="cuda")
    dv.train([a], [vol], dv.TrainConfig(batch=512, steps=5))
    b.copy_weights_from(a)
    np.testing.assert_array_equal(a.get_weights(), b.get_weights())
    sb = b.state()
    assert sb["adam_t"] == 0 and sb["iter"] == 0
    assert sb["vmin"] == a.state()["vmin"] and sb["vmax"] == a.state()["vmax"]
    w = np.linspace(-1, 1, a.n_params).astype(np.float32)
    a.set_weights(w)
    np.testing.assert_array_equal(a.get_weights(), w)


def test_fp16_export_import_roundtrip(dv):
    # Sec. 3.4 stores the model as 16-bit floats: export is the binary16
    # rounding of the master weights; importing it gives a model that decodes
    # like the FP16 copy it came from
    c = P.configs_blobs64()
    a = _model(dv, c, seed=3, hi=(16, 16, 16))
    w = a.get_weights()
    w16 = a.export_fp16()
    np.testing.assert_array_equal(w16, w.astype(np.float16))
    b = _model(dv, c, seed=4, hi=(16, 16, 16))
    b.import_fp16(w16)
    np.testing.assert_array_equal(b.get_weights(), w16.astype(np.float32))
    assert a.n_params * 2 == w16.nbytes  # the stored model size in bytes


@pytest.mark.parametrize("fp16", [False, True], ids=["fp32_file", "fp16_file"])
def test_model_file_round_trip(dv, tmp_path, fp16):
    # a trained model saved and loaded decodes bit for bit as the original on
    # the path whose parameters the file holds (FP32 master weights and value
    # range; or the binary16 weights, which the FP16 path computes with), and
    # a value range set by hand de-normalises exactly
    from paper_2304_10516_gb300 import model as M
    from paper_2304_10516_gb300 import volumes

    c = P.configs_blobs64()
    vol = torch.from_numpy(volumes.blobs(64, seed=1001) * 3.0 - 1.0).cuda()  # range [-1, 2]
    m = _model(dv, c, seed=9)
    prec = dv.A.DVNR_FP16 if fp16 else dv.A.DVNR_FP32
    dv.train([m], [vol], dv.TrainConfig(batch=c["batch"], steps=40, lr=1e-2, seed=4, precision=prec))
    f = tmp_path / "m.dvnr"
    m.save(f, fp16=fp16)
    m2 = M.Model.load(f)
    m2.set_precision(prec)
    a, b = m.decode_grid().cpu().numpy(), m2.decode_grid().cpu().numpy()
    np.testing.assert_array_equal(a.view(np.uint32), b.view(np.uint32))
    s1, s2 = m.state(), m2.state()
    assert (s1["vmin"], s1["vmax"]) == (s2["vmin"], s2["vmax"])
    # de-normalisation: out = y (vmax - vmin) + vmin with the set range
    m2.set_value_range(0.0, 1.0)
    y = m2.decode_grid().cpu().numpy()
    m2.set_value_range(-3.0, 5.0)
    z = m2.decode_grid().cpu().numpy()
    np.testing.assert_allclose(z, y * 8.0 - 3.0, rtol=0, atol=1e-5 * max(1.0, np.abs(z).max()))
    with pytest.raises(Exception):
        m2.set_value_range(2.0, 1.0)
    m.close()
    m2.close()
