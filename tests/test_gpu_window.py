"""Temporal sliding window (Sec. 4.2), frozen models and partitions with
adaptive table sizes (Sec. 3.2) on the GPU.

Window semantics are exact: the cached range, eviction, which steps are
frozen, the bytes held, and that a frozen step decodes bit for bit as it did
right after its own push (the FP16 parameters it keeps are those it was
decoded from). Warm starting is checked bit for bit on the FP16 copy and, as
training, against the oracle's warm-started sequence (parameters carried,
Adam reset per step) within 0.2 dB at lr 5e-4. Heterogeneous partitions
(each with its own table size and base resolution) trained in one FP16 call
match the oracle's FP16 emulation of each within 0.2 dB.
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


def _series(n, steps, seed=1006):
    from paper_2304_10516_gb300 import volumes

    return [volumes.advected((n, n, n), seed, float(t)) for t in range(steps)]


def test_window_range_eviction_freezing_and_bytes(dv):
    from paper_2304_10516_gb300 import volumes

    c = P.configs_blobs64()
    boxes = [((0, 0, 0), (24, 40, 40)), ((24, 0, 0), (40, 40, 40))]
    glob = 40 ** 3
    encs = [dv.adaptive_encoding((hi[0] - lo[0]) * 40 * 40, glob, 15, 10, 6.0,
                                 base=dv.EncodingConfig(c["L"], c["F"], 15, 4, c["growth"]))
            for lo, hi in boxes]
    assert encs[0].log2_T != encs[1].log2_T  # two configurations in one grouped call
    mlp = dv.MLPConfig(c["width"], c["hidden"])
    w = dv.Window(boxes, 3, encs, mlp, ghost=1, seed=5)
    series = _series(40, 5)
    cfg = dv.TrainConfig(batch=2048, steps=20, lr=1e-3, precision=dv.A.DVNR_FP16, seed=3)
    decoded = {}
    for t, f in enumerate(series):
        vols = [torch.from_numpy(volumes.extract_block(f, lo, hi, 1)).cuda() for lo, hi in boxes]
        tt, losses = w.push(vols, cfg)
        assert tt == t and all(np.isfinite(losses))
        first, last = w.range()
        assert (first, last) == (max(0, t - 2), t)
        for s in range(first, last + 1):
            for part in range(2):
                st = w.model(s, part).state()
                assert st["frozen"] == (1 if s < t else 0)
                assert st["precision"] == dv.A.DVNR_FP16
        decoded[t] = [w.model(t, p_).decode_grid().cpu().numpy() for p_ in range(2)]
        # steps still cached decode exactly as right after their own push
        for s in range(first, last + 1):
            for p_ in range(2):
                np.testing.assert_array_equal(w.model(s, p_).decode_grid().cpu().numpy(),
                                              decoded[s][p_])
        mb, db = w.bytes()
        n_steps = last - first + 1
        per_step = sum(w.model(t, p_).n_params * 2 for p_ in range(2))
        assert mb == n_steps * per_step
        full = db - sum(w.model(s, p_).n_params * 2 for s in range(first, last) for p_ in range(2))
        assert full > 8 * per_step  # only the newest step keeps FP32 weights and Adam state
    with pytest.raises(dv.A.DvnrError):
        w.model(1, 0)  # evicted
    frozen = w.model(3, 0)
    with pytest.raises(dv.A.DvnrError):
        dv.train([frozen], [torch.zeros((42, 42, 42), device="cuda")], cfg)
    with pytest.raises(dv.A.DvnrError):
        frozen.set_precision(dv.A.DVNR_FP32)
    # a push with no iterations warm-starts exactly: the new step holds the
    # previous step's FP16 parameters
    prev = [w.model(4, p_).export_fp16() for p_ in range(2)]
    vols = [torch.from_numpy(volumes.extract_block(series[0], lo, hi, 1)).cuda() for lo, hi in boxes]
    w.push(vols, dv.TrainConfig(batch=2048, steps=0, precision=dv.A.DVNR_FP16))
    for p_ in range(2):
        np.testing.assert_array_equal(w.model(5, p_).export_fp16(), prev[p_])
    w.close()


def test_window_warm_start_sequence_matches_oracle(dv, orc):
    c = dict(P.configs_blobs64(), batch=2048)
    oc = P.oracle_cfg(c)
    enc = dv.EncodingConfig(c["L"], c["F"], c["log2T"], c["base"], c["growth"])
    mlp = dv.MLPConfig(c["width"], c["hidden"])
    n = 32
    series = _series(n, 3, seed=1007)
    w = dv.Window([((0, 0, 0), (n, n, n))], 3, enc, mlp, ghost=0, seed=21)
    cfg = dv.TrainConfig(batch=2048, steps=100, lr=5e-4, seed=9)
    th = orc.init_params(oc, 21)
    for t, f in enumerate(series):
        w.push([torch.from_numpy(f).cuda()], cfg)
        m = w.model(t, 0)
        sse, _ = dv.error_stats(m.decode_grid(), torch.from_numpy(f).cuda())
        p_gpu = P.psnr(sse / f.size)
        # oracle: the parameters carry over, Adam and the step counter restart
        m1, m2 = np.zeros_like(th), np.zeros_like(th)
        tc = orc.TrainConfig(batch=2048, lr=float(np.float32(5e-4)), seed=9)
        orc.train(oc, tc, orc.State(), th, m1, m2, f, float(f.min()), float(f.max()), 100)
        dec = orc.decode_grid(oc, th, (n, n, n), 0, float(f.min()), float(f.max()))
        p_orc = P.psnr(orc.mse(dec, f)[0])
        assert abs(p_gpu - p_orc) < 0.2, (t, p_gpu, p_orc)
    w.close()


def test_adaptive_partitions_in_one_fp16_call_match_oracle(dv, orc):
    from paper_2304_10516_gb300 import volumes

    vol = volumes.blobs(64, seed=1001)
    c = P.configs_blobs64()
    boxes = [((0, 0, 0), (16, 64, 64)), ((16, 0, 0), (40, 64, 64)), ((40, 0, 0), (64, 64, 64))]
    base = dv.EncodingConfig(c["L"], c["F"], 16, 8, c["growth"])
    encs = [dv.adaptive_encoding((hi[0] - lo[0]) * 64 * 64, 64 ** 3, 16, 11, 8.0, base=base)
            for lo, hi in boxes]
    assert len({(e.log2_T, e.base_res) for e in encs}) >= 2
    mlp = dv.MLPConfig(c["width"], c["hidden"])
    models = [dv.Model(lo, hi, 1, e, mlp, seed=30 + i) for i, ((lo, hi), e) in enumerate(zip(boxes, encs))]
    vols = [torch.from_numpy(volumes.extract_block(vol, lo, hi, 1)).cuda() for lo, hi in boxes]
    steps, lr = 150, 5e-4
    dv.train(models, vols, dv.TrainConfig(batch=2048, steps=steps, lr=lr, seed=13,
                                          precision=dv.A.DVNR_FP16))
    for i, ((lo, hi), e, m, v) in enumerate(zip(boxes, encs, models, vols)):
        assert m.state()["iter"] == steps
        oc = orc.Config(e.n_levels, e.n_features, e.log2_T, e.base_res, e.growth, mlp.width,
                        mlp.n_hidden)
        th = orc.init_params(oc, 30 + i)
        m1, m2 = np.zeros_like(th), np.zeros_like(th)
        vn = v.cpu().numpy()
        tc = orc.TrainConfig(batch=2048, lr=float(np.float32(lr)), seed=13, mixed=True, model=i)
        orc.train(oc, tc, orc.State(loss_scale=2048.0), th, m1, m2, vn, float(vn.min()),
                  float(vn.max()), steps)
        dims = [h_ - l_ + 2 for l_, h_ in zip(lo, hi)]
        odec = orc.decode_grid(oc, th, dims, 1, float(vn.min()), float(vn.max()), mixed=True)
        ref = vn[1:-1, 1:-1, 1:-1]
        p_orc = P.psnr(orc.mse(odec, ref)[0])
        sse, _ = dv.error_stats(m.decode_grid(), torch.from_numpy(np.ascontiguousarray(ref)).cuda())
        p_gpu = P.psnr(sse / ref.size)
        assert abs(p_gpu - p_orc) < 0.2, (i, e, p_gpu, p_orc)
