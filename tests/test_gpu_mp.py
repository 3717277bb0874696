"""GPU parity of the FP16 tensor-core path (tcgen05) against the oracle.

The oracle's mixed mode rounds to binary16 at the points where the GPU keeps
FP16 operands (tables, weights, encoding, hidden activations, scaled output
gradient, hidden-layer gradients); accumulations stay FP64 there and FP32 on
the GPU. Tolerances: bit-exact coordinates; forward and gradients within
2e-3 (normwise for batch sums, plus the kink allowance of parity.py); PSNR
after seeded training within 0.2 dB of the oracle and of the plain FP32 path.
"""
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


@pytest.fixture(scope="module")
def A():
    from paper_2304_10516_gb300 import _abi as A

    return A


def _model(dv, c, seed, lo=(0, 0, 0), hi=(64, 64, 64), ghost=0):
    enc = dv.EncodingConfig(c["L"], c["F"], c["log2T"], c["base"], c["growth"])
    mlp = dv.MLPConfig(c["width"], c["hidden"])
    return dv.Model(lo, hi, ghost, enc, mlp, seed=seed)


def test_umma_operand_layouts(A):
    import ctypes as C

    out = (C.c_int32 * 5)()
    A.call("dvnr_selftest_umma", C.cast(out, C.c_void_p))
    assert list(out) == [0, 0, 0, 0, 0]


CONFIGS = {
    "blobs64": P.configs_blobs64(),
    # the 256^3 model's MLP and encoding width with a smaller table
    "w64d32h3": dict(L=16, F=2, log2T=14, base=16, growth=1.38, width=64, hidden=3, batch=4096),
    "w16d16h1_f4": dict(L=4, F=4, log2T=12, base=4, growth=1.5, width=16, hidden=1, batch=1000),
    # one and eight features per level (the other widths of the grouped kernels)
    "w32d16h2_f1": dict(L=16, F=1, log2T=13, base=4, growth=1.3, width=32, hidden=2, batch=2048),
    "w32d32h2_f8": dict(L=4, F=8, log2T=12, base=6, growth=1.6, width=32, hidden=2, batch=1536),
    # the appendix's NekRS and S3D networks (n_levels 5 and 4, 4 features per
    # level, 16 neurons, base resolution cbrt(T), per-level scale 2): an
    # encoding width of 20 enters layer 0 padded with zeros to 32
    "nekrs_w16d20h3_f4": dict(L=5, F=4, log2T=12, base=16, growth=2.0, width=16, hidden=3, batch=2048),
    "s3d_w16d16h2_f4": dict(L=4, F=4, log2T=11, base=12, growth=2.0, width=16, hidden=2, batch=1500),
    # width 10: padded to 16, and its layer-0 gradient rows are not 16-byte aligned
    "w32d10h2_f2": dict(L=5, F=2, log2T=12, base=8, growth=1.5, width=32, hidden=2, batch=1200),
    # more than 16 levels of two features: the staged gathers take two rounds
    "w64d48h3_l24": dict(L=24, F=2, log2T=14, base=4, growth=1.2, width=64, hidden=3, batch=2048),
}


@pytest.mark.parametrize("name", sorted(CONFIGS))
@pytest.mark.parametrize("lam,loss", [(0.0, 0), (0.15, 0), (0.0, 1)])
def test_fp16_step_matches_oracle(dv, orc, A, name, lam, loss):
    from paper_2304_10516_gb300 import volumes

    c = CONFIGS[name]
    oc = P.oracle_cfg(c)
    vol = volumes.blobs(40, seed=1001)
    theta = P.random_theta(oc, 31, table_scale=0.4)
    m = _model(dv, c, seed=0, hi=(40, 40, 40))
    m.set_weights(theta)
    lam32 = float(np.float32(lam))
    B = c["batch"]
    cfg = dv.TrainConfig(batch=B, lambda_bnd=lam32, sigma_bnd=0.005, loss=loss, seed=78,
                         precision=A.DVNR_FP16)
    out = m.train_grad(torch.from_numpy(vol).cuda(), cfg, iteration=5)
    torch.cuda.synchronize()
    coords = orc.sample(78, 0, 5, B, lam32, orc.quantile_table(float(np.float32(0.005))))
    np.testing.assert_array_equal(out["coords"].cpu().numpy().view(np.uint32), coords)
    t = orc.targets(vol, coords, float(vol.min()), float(vol.max()))
    np.testing.assert_allclose(out["target"].cpu().numpy(), t, atol=2e-6, rtol=0)
    S = float(2 ** round(np.log2(B)))
    th64 = theta.astype(np.float64)
    r = orc.fwd_bwd(oc, th64, coords, t, loss=loss, mixed=True, loss_scale=S, want_zabs=True)
    y = out["y"].cpu().numpy()
    np.testing.assert_allclose(y, r["y"], atol=2e-3 * max(1.0, np.abs(r["y"]).max()), rtol=0)
    a_enc, a_mlp, flagged = P.kink_allowance(oc, th64, coords, t, loss, True, S, B, r["zabs"],
                                             delta=1e-4)
    keep = np.ones(B, bool)
    keep[flagged] = False
    assert keep.sum() > 0.6 * B
    P.assert_normwise(out["dx0"].cpu().numpy()[keep], r["dx0"][keep], 2e-3, what="dL/dx0")
    g = out["grad"].cpu().numpy()
    P.assert_normwise(g[: oc.n_enc], r["grad_enc"], 2e-3, a_enc, what="table grad")
    P.assert_normwise(g[oc.n_enc:], r["grad_mlp"], 2e-3, a_mlp, what="mlp grad")


def test_fp16_ragged_batch_and_tail(dv, orc, A):
    # batch not a multiple of the 128-sample tile: the tail rows must not
    # contribute (compare against the oracle on exactly `batch` samples)
    from paper_2304_10516_gb300 import volumes

    c = dict(P.configs_blobs64(), batch=333)
    oc = P.oracle_cfg(c)
    vol = volumes.blobs(24, seed=1003)
    theta = P.random_theta(oc, 32, table_scale=0.4)
    m = _model(dv, c, seed=0, hi=(24, 24, 24))
    m.set_weights(theta)
    cfg = dv.TrainConfig(batch=333, loss=1, seed=3, precision=A.DVNR_FP16)
    out = m.train_grad(torch.from_numpy(vol).cuda(), cfg, iteration=0)
    coords = orc.sample(3, 0, 0, 333, 0.0, orc.quantile_table(0.005))
    t = orc.targets(vol, coords, float(vol.min()), float(vol.max()))
    S = float(2 ** round(np.log2(333)))
    r = orc.fwd_bwd(oc, theta.astype(np.float64), coords, t, loss=1, mixed=True, loss_scale=S,
                    want_zabs=True)
    a_enc, a_mlp, _ = P.kink_allowance(oc, theta.astype(np.float64), coords, t, 1, True, S, 333,
                                       r["zabs"], delta=1e-4)
    g = out["grad"].cpu().numpy()
    P.assert_normwise(g[: oc.n_enc], r["grad_enc"], 2e-3, a_enc, what="table grad")
    P.assert_normwise(g[oc.n_enc:], r["grad_mlp"], 2e-3, a_mlp, what="mlp grad")
    assert abs(out["loss"].item() - r["loss"]) < 2e-3 * max(r["loss"], 1e-3)


@pytest.mark.parametrize("name", sorted(CONFIGS))
def test_fp16_decode_matches_oracle(dv, orc, A, name):
    # every width / features-per-level / depth of the decode kernel (W = 16
    # reads its outputs as one 16-column chunk, H = 1 forms the output in the
    # first layer's epilogue); 26 048 points = 203.5 tiles (ragged tail)
    c = CONFIGS[name]
    oc = P.oracle_cfg(c)
    theta = P.random_theta(oc, 7, table_scale=0.3)
    lo, hi, g = (3, 5, 7), (40, 37, 29), 1
    m = _model(dv, c, seed=0, lo=lo, hi=hi, ghost=g)
    m.set_weights(theta)
    m.set_precision(A.DVNR_FP16)
    dec = m.decode_grid().cpu().numpy()
    dims = [h - l + 2 * g for l, h in zip(lo, hi)]
    want = orc.decode_grid(oc, theta.astype(np.float64), dims, g, 0.0, 1.0, mixed=True)
    np.testing.assert_allclose(dec, want, atol=2e-3 * max(1.0, np.abs(want).max()), rtol=0)
    # decode_grid equals point inference at the voxel centres (same kernel path)
    zz, yy, xx = np.meshgrid(np.arange(lo[2], hi[2]), np.arange(lo[1], hi[1]), np.arange(lo[0], hi[0]),
                             indexing="ij")
    xyz = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], 1).astype(np.float32)
    pts = m.decode_points(torch.from_numpy(xyz).cuda()).cpu().numpy()
    np.testing.assert_allclose(pts, dec.ravel(), atol=1e-3 * max(1.0, np.abs(want).max()), rtol=0)


def _train_psnr(dv, c, vol, seed_model, lr, steps, seed, precision):
    m = _model(dv, c, seed=seed_model, hi=vol.shape[::-1])
    cfg = dv.TrainConfig(batch=c["batch"], steps=steps, lr=lr, seed=seed, precision=precision)
    vt = torch.from_numpy(vol).cuda()
    losses = dv.train([m], [vt], cfg)
    sse, _ = dv.error_stats(m.decode_grid(), vt)
    return P.psnr(sse / vol.size), losses[0], m


def test_fp16_training_equal_psnr(dv, orc, A):
    # 200 seeded steps of the 64^3 workload at lr 5e-4 (a regime where the
    # oracle's run-to-run spread is 0.013 dB): the FP16 path reaches the PSNR
    # of the oracle's FP16 emulation and of the plain FP32 path within 0.2 dB.
    from paper_2304_10516_gb300 import volumes

    c = P.configs_blobs64()
    oc = P.oracle_cfg(c)
    vol = volumes.blobs(64, seed=1001)
    p16, l16, m16 = _train_psnr(dv, c, vol, 4242, 5e-4, 200, 99, A.DVNR_FP16)
    p32, _, _ = _train_psnr(dv, c, vol, 4242, 5e-4, 200, 99, A.DVNR_FP32)
    st = m16.state()
    assert st["adam_t"] == 200 and st["skipped"] == 0 and st["precision"] == A.DVNR_FP16
    th = orc.init_params(oc, 4242)
    m1, m2 = np.zeros_like(th), np.zeros_like(th)
    tc = orc.TrainConfig(batch=c["batch"], lr=float(np.float32(5e-4)), seed=99, mixed=True)
    ost = orc.State(loss_scale=4096.0)
    orc.train(oc, tc, ost, th, m1, m2, vol, float(vol.min()), float(vol.max()), 200)
    odec = orc.decode_grid(oc, th, (64, 64, 64), 0, float(vol.min()), float(vol.max()), mixed=True)
    po = P.psnr(orc.mse(odec, vol)[0])
    assert abs(p16 - po) < 0.2, (p16, po)
    assert abs(p16 - p32) < 0.2, (p16, p32)


@pytest.mark.parametrize("wave_models", [None, "1", "3", "tiles:7"])
def test_grouped_launch_models_are_independent(dv, A, monkeypatch, wave_models):
    # Four models in one grouped FP16 launch. Compared after one step through
    # the first Adam moment, m1 = (1 - beta1) g: linear in the step's
    # gradient (the weights are not -- Adam's first steps move every entry by
    # about lr sign(g), so an entry whose gradient is at the level of the
    # atomic reordering noise moves by up to 2 lr between runs), and the
    # step's forward is bit-identical between runs (same initial weights).
    # Model 0 trained in the group equals model 0 trained alone (same RNG
    # slot) up to the reordering of atomic sums, and perturbing model 2's
    # volume leaves the other models within that same noise. Then 10 steps:
    # the unperturbed models' PSNRs do not move.
    from paper_2304_10516_gb300 import volumes

    # wave_models: models trained per wave inside the launch (1: one model at
    # a time; 3: waves of 3 + 1); None leaves the library's choice
    # ("tiles:7": waves of 7 tiles, which split the models' tile runs mid-model)
    if wave_models and wave_models.startswith("tiles:"):
        monkeypatch.setenv("DVNR_WAVE_TILES", wave_models[6:])
    elif wave_models:
        monkeypatch.setenv("DVNR_WAVE_MODELS", wave_models)
    c = dict(P.configs_blobs64(), batch=2048)
    vols = [torch.from_numpy(volumes.blobs(32, seed=2000 + i)).cuda() for i in range(4)]

    def group(vs, steps, loss=A.DVNR_LOSS_L1):
        ms = [_model(dv, c, seed=50 + i, hi=(32, 32, 32)) for i in range(4)]
        dv.train(ms, vs, dv.TrainConfig(batch=2048, steps=steps, lr=1e-3, seed=5, loss=loss,
                                        precision=A.DVNR_FP16))
        return ms

    def m1_of(ms):
        return [m.moments()[0] for m in ms]

    # L2: the first step's L1 gradient is sign(y - t) with y ~ 0 at the
    # initial weights, the same for any target, so it could not show the
    # perturbation
    L2 = A.DVNR_LOSS_L2
    base = m1_of(group(vols, 1, L2))
    again = m1_of(group(vols, 1, L2))
    noise = max(np.linalg.norm(a - b) for a, b in zip(base, again))
    pert = list(vols)
    pert[2] = vols[2] ** 2  # a non-affine change (min/max normalisation hides affine ones)
    moved = m1_of(group(pert, 1, L2))
    ref = max(np.linalg.norm(b) for b in base)
    for j in (0, 1, 3):
        assert np.linalg.norm(moved[j] - base[j]) <= 3 * noise + 1e-6 * ref, j
    assert np.linalg.norm(moved[2] - base[2]) > 10 * noise + 1e-4 * ref
    alone = _model(dv, c, seed=50, hi=(32, 32, 32))
    dv.train([alone], [vols[0]], dv.TrainConfig(batch=2048, steps=1, lr=1e-3, seed=5, loss=L2,
                                                precision=A.DVNR_FP16))
    assert np.linalg.norm(alone.moments()[0] - base[0]) <= 3 * noise + 1e-6 * ref

    def psnrs(ms, vs):
        out = []
        for m, v in zip(ms, vs):
            sse, _ = dv.error_stats(m.decode_grid(), v)
            out.append(P.psnr(sse / v.numel()))
        return out

    p_base = psnrs(group(vols, 10), vols)
    p_moved = psnrs(group(pert, 10), pert)
    for j in (0, 1, 3):
        assert abs(p_moved[j] - p_base[j]) < 0.05, (j, p_moved[j], p_base[j])


def test_fp16_overflow_skips_step_and_halves_scale(dv, A):
    c = dict(P.configs_blobs64(), batch=1024)
    m = _model(dv, c, seed=1, hi=(16, 16, 16))
    w = m.get_weights()
    w[: m.n_enc] = 3.0e4  # encoding outputs near the FP16 limit: activations overflow
    w[m.n_enc:] = np.abs(w[m.n_enc:]) * 50
    m.set_weights(w)
    vol = torch.rand((16, 16, 16), device="cuda")
    dv.train([m], [vol], dv.TrainConfig(batch=1024, steps=3, precision=A.DVNR_FP16))
    st = m.state()
    assert st["skipped"] == 3 and st["adam_t"] == 0
    assert st["loss_scale"] == 1024.0 / 8
    np.testing.assert_array_equal(m.get_weights(), w.astype(np.float32))


@pytest.mark.parametrize("name", ["blobs64", "w64d32h3"])
def test_fp16_error_against_plain_fp64_oracle(dv, orc, A, name):
    # The production path against the FP64 oracle without FP16 emulation: the
    # error the FP16 storage and tensor-core operands cost (Sec. 3.4 16-bit
    # weights, Sec. 3.6 tensor-core training). Measured on one GB300, one step
    # of 4096 samples (L1) with tables of the scale training reaches:
    #   forward y         max |err| / max |y|        6.4e-4, 8.4e-4
    #   dL/d(encoding)    normwise (kink-free rows)  4.3e-4, 6.2e-4
    #   MLP gradients     normwise                   5.5e-4, 8.1e-4
    #   table gradients   normwise                   6.2e-3, 2.8e-2 (rows whose
    #                     pre-activations lie within the FP16 rounding of 0
    #                     switch ReLU branch; the emulation comparison of
    #                     test_fp16_step_matches_oracle bounds that part)
    #   decode (grid)     max |err| / value range    4.9e-4, 6.7e-4
    # The bounds are about three times those values.
    from paper_2304_10516_gb300 import volumes

    c = dict(CONFIGS.get(name, P.configs_blobs64()), batch=4096)
    oc = P.oracle_cfg(c)
    vol = volumes.blobs(40, seed=1001)
    theta = orc.init_params(oc, 31).astype(np.float32)
    theta[: oc.n_enc] = np.random.default_rng(3).uniform(-0.1, 0.1, oc.n_enc).astype(np.float32)
    m = _model(dv, c, seed=0, hi=(40, 40, 40))
    m.set_weights(theta)
    out = m.train_grad(torch.from_numpy(vol).cuda(),
                       dv.TrainConfig(batch=4096, loss=0, seed=78, precision=A.DVNR_FP16), iteration=5)
    torch.cuda.synchronize()
    coords = out["coords"].cpu().numpy().view(np.uint32)
    t = orc.targets(vol, coords, float(vol.min()), float(vol.max()))
    th64 = theta.astype(np.float64)
    r = orc.fwd_bwd(oc, th64, coords, t, loss=0, mixed=False, want_zabs=True)
    y = out["y"].cpu().numpy()
    assert np.abs(y - r["y"]).max() <= 3e-3 * np.abs(r["y"]).max()
    keep = r["zabs"].min(axis=1) > 2e-4
    assert keep.sum() > 0.1 * len(keep)
    P.assert_normwise(out["dx0"].cpu().numpy()[keep], r["dx0"][keep], 2e-3, what="dL/dx0 vs FP64")
    g = out["grad"].cpu().numpy()
    P.assert_normwise(g[oc.n_enc:], r["grad_mlp"], 3e-3, what="MLP grad vs FP64")
    P.assert_normwise(g[: oc.n_enc], r["grad_enc"], 0.1, what="table grad vs FP64")
    m.set_precision(A.DVNR_FP16)
    dec = m.decode_grid().cpu().numpy()
    ref = orc.decode_grid(oc, th64, (40, 40, 40), 0, 0.0, 1.0)
    assert np.abs(dec - ref).max() <= 2e-3 * (ref.max() - ref.min())
    m.close()


def test_interleaved_steps_train_like_plain_steps(dv, A, monkeypatch):
    # DVNR_INTERLEAVE=1 runs a step wave by wave with each wave's Adam update
    # before its training launch (here one model per wave); per model the
    # sequence of operations is that of the plain layout, so the counters
    # agree exactly and the models reach the same PSNR (up to the reordering
    # of atomic sums)
    from paper_2304_10516_gb300 import volumes

    c = dict(P.configs_blobs64(), batch=2048)
    vols = [torch.from_numpy(volumes.blobs(32, seed=2100 + i)).cuda() for i in range(4)]

    def run(interleave):
        if interleave:
            monkeypatch.setenv("DVNR_INTERLEAVE", "1")
        else:
            monkeypatch.delenv("DVNR_INTERLEAVE", raising=False)
        monkeypatch.setenv("DVNR_WAVE_MODELS", "1")
        ms = [_model(dv, c, seed=60 + i, hi=(32, 32, 32)) for i in range(4)]
        losses = dv.train(ms, vols, dv.TrainConfig(batch=2048, steps=20, lr=1e-3, seed=9,
                                                  loss=A.DVNR_LOSS_L2, precision=A.DVNR_FP16))
        out = []
        for m, v in zip(ms, vols):
            st = m.state()
            sse, _ = dv.error_stats(m.decode_grid(), v)
            out.append((st["adam_t"], st["iter"], st["skipped"], P.psnr(sse / v.numel())))
            m.close()
        return out, losses

    plain, lp = run(False)
    inter, li = run(True)
    for (a, b) in zip(plain, inter):
        assert a[:3] == b[:3] == (20, 20, 0)
        assert abs(a[3] - b[3]) < 0.05, (a, b)
    np.testing.assert_allclose(li, lp, rtol=2e-3)
