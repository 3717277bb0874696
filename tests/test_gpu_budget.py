"""Iteration budget and early stop of a training call (Sec. 3.2) on the GPU.

Budgets are integers and must equal the oracle's N_train^max exactly, per
model, on both paths; in a grouped FP16 call every model keeps its own
budget. Early stop follows the oracle's moving-average rule: on the FP32
path the stop step equals the oracle's where the oracle's moving average
crosses the threshold with a margin of 0.5% on both sides; on the FP16 path a
model that meets the threshold leaves the grouped launch while the others
train on unaffected.
"""
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


def _model(dv, c, seed, lo, hi, ghost=1):
    enc = dv.EncodingConfig(c["L"], c["F"], c["log2T"], c["base"], c["growth"])
    mlp = dv.MLPConfig(c["width"], c["hidden"])
    return dv.Model(lo, hi, ghost, enc, mlp, seed=seed)


def _blocks():
    # three partitions of the 64^3 blobs field with uneven owned extents
    return [((0, 0, 0), (20, 24, 28)), ((20, 0, 0), (64, 40, 44)), ((0, 24, 28), (37, 64, 64))]


def _nvox(lo, hi):
    return (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2])


def _setup(dv, c, seeds=(11, 12, 13)):
    from paper_2304_10516_gb300 import volumes

    vol = volumes.blobs(64, seed=1001)
    models, vols = [], []
    for (lo, hi), sd in zip(_blocks(), seeds):
        models.append(_model(dv, c, sd, lo, hi))
        vols.append(torch.from_numpy(volumes.extract_block(vol, lo, hi, 1)).cuda())
    return models, vols


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_budget_per_model_equals_oracle(dv, orc, precision):
    c = P.configs_blobs64()
    prec = dv.A.DVNR_FP16 if precision == "fp16" else dv.A.DVNR_FP32
    models, vols = _setup(dv, c)
    B = 2048
    for epochs, min_steps, steps in ((2, 0, 0), (1, 20, 0), (0, 9, 5), (0, 0, 7)):
        for m in models:
            m.set_weights(m.get_weights())  # fresh optimiser state
        cfg = dv.TrainConfig(batch=B, steps=steps, epochs=epochs, min_steps=min_steps, lr=5e-4,
                             precision=prec, seed=3)
        dv.train(models, vols, cfg)
        for m, (lo, hi) in zip(models, _blocks()):
            want = orc.max_iterations(_nvox(lo, hi), B, steps=steps, epochs=epochs,
                                      min_steps=min_steps)
            st = m.state()
            assert st["iter"] == want and st["adam_t"] == want, (epochs, min_steps, steps, st)
            assert st["budget_end"] == want and st["stopped"] == 0
    # the three budgets of the first setting differ, so the grouped launch ran
    # models that had finished beside models that had not
    assert len({orc.max_iterations(_nvox(lo, hi), B, epochs=2) for lo, hi in _blocks()}) == 3


def _ema_seq(L, d):
    m, out = None, []
    for x in L:
        m = x if m is None else d * m + (1 - d) * x
        out.append(m)
    return np.array(out)


def test_fp32_early_stop_step_matches_oracle(dv, orc):
    from paper_2304_10516_gb300 import volumes

    c = P.configs_blobs64()
    oc = P.oracle_cfg(c)
    vol = volumes.blobs(64, seed=1001)
    decay, budget, lr = 0.5, 300, 5e-4
    th0 = orc.init_params(oc, 4242)
    tc = orc.TrainConfig(batch=c["batch"], lr=float(np.float32(lr)), seed=99)
    th = th0.copy()
    hist = orc.train(oc, tc, orc.State(), th, np.zeros_like(th), np.zeros_like(th), vol,
                     float(vol.min()), float(vol.max()), budget)
    ema = _ema_seq(hist, decay)
    # a threshold that the oracle's average crosses with a clear margin: a
    # new low at least 1% below every earlier value
    delta = 5e-3
    pick = None
    for t in range(40, budget):
        prev = ema[:t].min()
        if prev > ema[t] * (1 + delta) / (1 - delta) * 1.0001:
            pick = t
            thr = math.sqrt(prev * ema[t])
            break
    assert pick is not None
    want, want_ema = orc.stop_step(hist, decay, thr)
    assert want == pick + 1
    m = _model(dv, c, 0, (0, 0, 0), (64, 64, 64), ghost=0)
    m.set_weights(th0.astype(np.float32))
    cfg = dv.TrainConfig(batch=c["batch"], steps=budget, lr=lr, seed=99, stop_loss=float(thr),
                         stop_decay=decay)
    dv.train([m], [torch.from_numpy(vol).cuda()], cfg)
    st = m.state()
    assert st["stopped"] == 1 and st["iter"] == want and st["adam_t"] == want, (st, want)
    assert abs(st["loss_ema"] - want_ema) <= 2e-3 * want_ema
    assert st["loss_ema"] < float(np.float32(thr))


def test_fp16_model_that_stops_leaves_the_group(dv, orc):
    # model 1 learns a constant field (its normalised targets are all 0) and
    # meets the threshold within a few steps; models 0 and 2 never do. They
    # run their whole budget, and model 0 ends as it does when trained alone
    # (same RNG slot 0, same budget): the grouped launch after model 1 left
    # computes the same steps up to summation order. FP16 trajectories differ
    # by about 0.1 dB after 150 steps from summation order alone (the
    # rounding of the FP16 weight copy amplifies last-bit differences), so
    # the PSNR bound is 0.25 dB; that the compacted schedule covers every
    # tile of every active model exactly once is checked exactly elsewhere.
    from paper_2304_10516_gb300 import volumes

    c = P.configs_blobs64()
    FP16 = dv.A.DVNR_FP16
    models, vols = _setup(dv, c)
    vols[1] = torch.full_like(vols[1], 0.25)
    cfg = dv.TrainConfig(batch=2048, steps=150, lr=5e-4, precision=FP16, seed=7,
                         stop_loss=2e-3, stop_decay=0.5)
    w0 = [m.get_weights() for m in models]
    dv.train(models, vols, cfg)
    s0, s1, s2 = (m.state() for m in models)
    assert s1["stopped"] == 1 and s1["iter"] < 150 and s1["loss_ema"] < 2e-3
    assert s0["stopped"] == 0 and s0["iter"] == 150 and s2["iter"] == 150
    assert s0["loss_ema"] >= 2e-3 and s2["loss_ema"] >= 2e-3
    assert s1["adam_t"] == s1["iter"]
    alone = _model(dv, c, 11, *_blocks()[0])
    alone.set_weights(w0[0])
    dv.train([alone], [vols[0]], cfg)
    sa = alone.state()
    assert sa["iter"] == 150
    ref = vols[0][1:-1, 1:-1, 1:-1].contiguous()
    p_group = P.psnr(dv.error_stats(models[0].decode_grid(), ref)[0] / ref.numel())
    p_alone = P.psnr(dv.error_stats(alone.decode_grid(), ref)[0] / ref.numel())
    assert abs(p_group - p_alone) < 0.25, (p_group, p_alone)
    # a further call continues model 1 from where it stopped, with a fresh
    # budget and moving average; its first loss is that of the stopped model
    # alone (steps it sat out left no loss or gradient behind)
    dv.train([models[1]], [vols[1]], dv.TrainConfig(batch=2048, steps=1, lr=5e-4, precision=FP16,
                                                     seed=7))
    s1b = models[1].state()
    assert s1b["iter"] == s1["iter"] + 1 and s1b["stopped"] == 0
    assert s1b["last_loss"] < 3 * s1["loss_ema"] + 1e-4, (s1, s1b)
    assert s1b["loss_ema"] == pytest.approx(s1b["last_loss"], rel=1e-6)


@pytest.mark.parametrize("wave_tiles", [None, "5"])
def test_fp16_losses_cover_every_tile_after_a_model_leaves(dv, orc, monkeypatch, wave_tiles):
    # weights frozen (lr 1e-30 moves no FP32 weight), so every step's loss is
    # the loss of the initial network on that step's samples. Model 1 stops
    # after its first step and leaves the middle of the group; from then on
    # models 0 and 2 are tiled over positions 0 and 1. Their losses at the
    # last step must equal the oracle's (mixed-precision forward) on the
    # same samples: a tile lost or counted twice moves the mean by 1/16.
    # wave_tiles "5": waves of 5 tiles, which split every model's 16 tiles
    if wave_tiles:
        monkeypatch.setenv("DVNR_WAVE_TILES", wave_tiles)
    c = P.configs_blobs64()
    oc = P.oracle_cfg(c)
    FP16 = dv.A.DVNR_FP16
    models, vols = _setup(dv, c)
    vols[1] = torch.full_like(vols[1], 0.25)
    B, K = 2048, 40
    th0 = [m.get_weights() for m in models]
    # models 0 and 2 see losses of about the mean normalised value (> 0.1)
    # and never meet the threshold; model 1's targets are all 0 and the
    # initial network's output is far below 1e-2
    cfg = dv.TrainConfig(batch=B, steps=K, lr=1e-30, precision=FP16, seed=5, stop_loss=1e-2,
                         stop_decay=0.5)
    dv.train(models, vols, cfg)
    s = [m.state() for m in models]
    assert s[1]["stopped"] == 1 and s[1]["iter"] == 1
    qtab = orc.quantile_table(0.005)
    for slot in (0, 2):
        assert s[slot]["iter"] == K and s[slot]["stopped"] == 0
        # (an Adam step of lr 1e-30 moves only parameters within ~1e-28 of zero)
        np.testing.assert_allclose(models[slot].get_weights(), th0[slot], rtol=1e-6, atol=1e-25)
        v = vols[slot].cpu().numpy()
        coords = orc.sample(5, slot, K - 1, B, 0.0, qtab)
        t = orc.targets(v, coords, float(v.min()), float(v.max()))
        r = orc.fwd_bwd(oc, th0[slot].astype(np.float64), coords, t, loss=0, mixed=True,
                        loss_scale=float(2 ** round(np.log2(B))), want_grads=False)
        assert abs(s[slot]["last_loss"] - r["loss"]) <= 2e-3 * r["loss"], (slot, s[slot], r["loss"])


@pytest.mark.parametrize("loop", [True, False])
def test_fp16_group_that_stops_ends_the_loop(dv, monkeypatch, loop):
    # every model learns a constant field and meets the threshold within a
    # few steps of a 3000-step budget. The steps of a call with a stop rule
    # run as a conditional loop of 32-step bodies that ends once no model is
    # active, so the call launches a few bodies, not 3000 steps of kernels
    # that find nothing to do; each model's counters stop where it stopped.
    # A second call on the same group (same cached graph) re-arms the loop.
    # loop=False: the fallback for runtimes without conditional nodes, a
    # fixed 32-step graph whose steps do nothing once every model stopped:
    # the same per-model counters, and 3 kernels for every step slot.
    from paper_2304_10516_gb300 import _abi as A

    if not loop:
        monkeypatch.setenv("DVNR_GRAPH_LOOP", "0")

    c = P.configs_blobs64()
    FP16 = dv.A.DVNR_FP16
    models, vols = _setup(dv, c)
    vols = [torch.full_like(v, 0.25) for v in vols]
    cfg = dv.TrainConfig(batch=2048, steps=3000, lr=5e-4, precision=FP16, seed=7,
                         stop_loss=2e-3, stop_decay=0.5)
    lib = A.load()
    dv.train(models, vols, dv.TrainConfig(batch=2048, steps=1, lr=5e-4, precision=FP16, seed=7,
                                          stop_loss=2e-3, stop_decay=0.5))  # launch-shape tuning
    for call in range(2):
        torch.cuda.synchronize()
        n0 = lib.dvnr_launch_count()
        it0 = [m.state()["iter"] for m in models]
        dv.train(models, vols, cfg)
        torch.cuda.synchronize()
        launched = lib.dvnr_launch_count() - n0
        s = [m.state() for m in models]
        ran = [st["iter"] - i0 for st, i0 in zip(s, it0)]
        for st, r in zip(s, ran):
            assert st["stopped"] == 1 and 1 <= r < 100 and st["loss_ema"] < 2e-3, (call, st)
            assert st["adam_t"] == st["iter"] and st["budget_end"] == st["iter"] - r + 3000
        if loop:
            bodies = (max(ran) + 31) // 32
            # begin-call kernels, the arm node, then 97 kernels per 32-step
            # body; the masked schedule launches 3 x 3000
            assert launched <= 16 + 1 + bodies * 97, (call, launched, ran)
            assert launched >= 1 + bodies * 97, (call, launched, ran)
        else:
            assert 3 * 3000 <= launched <= 16 + 3 * 3000, (call, launched, ran)


def test_appendix_nekrs_network_trains_on_fp16_path(dv, orc):
    # the appendix's in situ NekRS network (5 levels x 4 features, 16 neurons,
    # 3 hidden layers, lrate 0.001, 4 epochs, target loss 0.0105) through the
    # appendix-key mapper: the epoch budget is the oracle's N_train^max, the
    # call trains on the FP16 path, and the moving-average stop ends it no
    # later than the budget
    import json
    import os

    from paper_2304_10516_gb300 import config as PC
    from paper_2304_10516_gb300 import volumes

    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "appendix_configs.json")))
    pc = PC.PaperConfig.from_dict(gold["insitu"]["NekRS"])
    vol = torch.from_numpy(volumes.blobs(64, seed=1001)).cuda()
    m = dv.Model((0, 0, 0), (64, 64, 64), 0, pc.encoding(), pc.mlp(), seed=3)
    B = 4096
    cfg = pc.train(batch=B, precision=dv.A.DVNR_FP16, seed=2)
    dv.train([m], [vol], dv.TrainConfig(batch=B, steps=1, lr=1e-30, precision=dv.A.DVNR_FP16))
    sse0, _ = dv.error_stats(m.decode_grid(), vol)  # the untrained network (value range set)
    it0 = m.state()["iter"]
    dv.train([m], [vol], cfg)
    st = m.state()
    budget = orc.max_iterations(64 ** 3, B, epochs=4)
    ran = st["iter"] - it0
    assert st["budget_end"] == it0 + budget
    assert 1 <= ran <= budget and st["adam_t"] + st["skipped"] == st["iter"]
    assert (st["stopped"] == 1) == (ran < budget)
    if st["stopped"]:
        assert st["loss_ema"] < 0.0105
    sse, _ = dv.error_stats(m.decode_grid(), vol)
    assert sse < 0.25 * sse0, (sse, sse0)  # the network has learned the field
