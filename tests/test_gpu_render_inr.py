"""Direct INR ray-marching (Sec. 4.3) on the GPU against the oracle's march.

Both sides use one reading of the camera, samples, block ownership, transfer
function and compositing; they differ only in how the networks' values are
computed (FP32/FP16 kernels vs the FP64 oracle, its mixed mode emulating the
FP16 rounding points). The image tolerance is derived from the value errors
measured at the very samples of the image: with values off by at most dv,
each opacity is off by at most alpha_max dv / (v_hi - v_lo), the opacity of
a ray by at most the sum of those (compositing is 1-Lipschitz in each
opacity) and the colour by at most three times that (colours in [0, 1]).
"""
import numpy as np
import pytest

import parity as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TF = dict(c0=(0.1, 0.2, 0.6), c1=(1.0, 0.9, 0.2), alpha_max=0.05, v_lo=-0.4, v_hi=0.6)


@pytest.fixture(scope="module")
def dv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_10516_gb300 import model as dv

    return dv


def _tf_list():
    f = lambda v: float(np.float32(v))  # noqa: E731 -- the GPU holds the TF in float32
    return [f(v) for v in (*TF["c0"], *TF["c1"], TF["alpha_max"], TF["v_lo"], TF["v_hi"])]


def _model(dv, c, seed, lo, hi, ghost):
    enc = dv.EncodingConfig(c["L"], c["F"], c["log2T"], c["base"], c["growth"])
    mlp = dv.MLPConfig(c["width"], c["hidden"])
    return dv.Model(lo, hi, ghost, enc, mlp, seed=seed)


def _samples(boxes, w, h, spr, pixels):
    """Positions of the samples of the listed pixels, as the kernels compute
    them in float32, with the owning block of each (-1: outside)."""
    f32 = np.float32
    LO = np.array([min(b[0][a] for b in boxes) for a in range(3)], dtype=f32)
    HI = np.array([max(b[1][a] for b in boxes) for a in range(3)], dtype=f32)
    px, py = pixels % w, pixels // w
    X = (LO[0] - f32(0.5)) + ((px.astype(f32) + f32(0.5)) * (HI[0] - LO[0])) / f32(w)
    Y = (LO[1] - f32(0.5)) + ((py.astype(f32) + f32(0.5)) * (HI[1] - LO[1])) / f32(h)
    k = np.arange(spr, dtype=f32)
    Z = (LO[2] - f32(0.5)) + ((k + f32(0.5)) * (HI[2] - LO[2])) / f32(spr)
    P3 = np.stack(np.broadcast_arrays(X[:, None], Y[:, None], Z[None, :]), -1).reshape(-1, 3)
    owner = np.full(P3.shape[0], -1)
    for b, (lo, hi) in enumerate(boxes):
        lo32, hi32 = np.array(lo, f32) - f32(0.5), np.array(hi, f32) - f32(0.5)
        inside = np.all((P3 >= lo32) & (P3 < hi32), axis=1) & (owner < 0)
        owner[inside] = b
    return P3, owner


def _value_error(dv, orc, oc, models, thetas, boxes, ghost, P3, owner, mixed):
    """Max |GPU value - oracle value| over the samples (point decoding at the
    same positions, the same kernels as the ray-marcher)."""
    err = 0.0
    for b, (m, th, (lo, hi)) in enumerate(zip(models, thetas, boxes)):
        pts = P3[owner == b]
        if pts.size == 0:
            continue
        got = m.decode_points(torch.from_numpy(np.ascontiguousarray(pts)).cuda()).cpu().numpy()
        n = np.array([h_ - l_ + 2 * ghost for l_, h_ in zip(lo, hi)], dtype=np.float64)
        u = np.clip((pts.astype(np.float64) - (np.array(lo) - ghost)) / (n - 1), 0.0, 1.0)
        mfix = np.rint(u * 2 ** 24).astype(np.uint32)
        want = orc.decode_unit(oc, th.astype(np.float64), mfix, 0.0, 1.0, mixed=mixed)
        err = max(err, float(np.abs(got - want).max()))
    return err


def _check(dv, orc, c, boxes, ghost, precision, w, h, spr, seed, pixels=None, dv_tol=None):
    oc = P.oracle_cfg(c)
    models, thetas = [], []
    for i, (lo, hi) in enumerate(boxes):
        th = P.random_theta(oc, seed + i, table_scale=0.3)
        m = _model(dv, c, 0, lo, hi, ghost)
        m.set_weights(th)
        m.set_precision(precision)
        models.append(m)
        thetas.append(th)
    tf = dv.make_tf(**TF)
    img = dv.render_inr(models, tf, w, h, spr).cpu().numpy().reshape(-1, 4)
    pix = np.arange(w * h) if pixels is None else np.asarray(pixels)
    mixed = precision == dv.A.DVNR_FP16
    want = orc.render_inr(oc, [t.astype(np.float64) for t in thetas], [b[0] for b in boxes],
                          [b[1] for b in boxes], ghost, 0.0, 1.0, _tf_list(), w, h, spr,
                          pixels=pix, mixed=mixed)
    P3, owner = _samples(boxes, w, h, spr, pix)
    dvmax = _value_error(dv, orc, oc, models, thetas, boxes, ghost, P3, owner, mixed)
    if dv_tol is not None:
        assert dvmax <= dv_tol, dvmax
    n_max = int(np.max(np.sum((owner >= 0).reshape(pix.size, spr), axis=1)))
    bound = TF["alpha_max"] * n_max * dvmax / (TF["v_hi"] - TF["v_lo"]) + 1e-5
    got = img[pix]
    np.testing.assert_allclose(got[:, 3], want[:, 3], atol=bound, rtol=0)
    np.testing.assert_allclose(got[:, :3], want[:, :3], atol=3 * bound, rtol=0)
    return got, want, models


# four blocks: two stacked in z, offset in x; block edges fall inside segments
BOXES = [((0, 0, 0), (20, 18, 33)), ((20, 0, 0), (37, 18, 33)),
         ((0, 0, 33), (20, 18, 61)), ((20, 0, 33), (37, 18, 61))]


def test_render_inr_fp32_matches_oracle(dv, orc):
    c = dict(P.configs_blobs64(), width=16, hidden=1)
    got, want, _ = _check(dv, orc, c, BOXES, 1, dv.A.DVNR_FP32, 23, 17, 300, seed=40,
                          dv_tol=2e-5)
    assert want[:, 3].mean() > 0.01  # the rays see the volume


@pytest.mark.parametrize("c", [
    dict(L=16, F=2, log2T=14, base=16, growth=1.38, width=64, hidden=3, batch=4096),
    # another instantiation of the decode kernel's ray-lattice mode
    dict(L=16, F=1, log2T=13, base=4, growth=1.3, width=32, hidden=2, batch=2048),
    # the appendix's NekRS network: encoding width 20, padded to 32
    dict(L=5, F=4, log2T=12, base=16, growth=2.0, width=16, hidden=3, batch=2048),
], ids=["w64f2h3", "w32f1h2", "nekrs_w16d20h3"])
def test_render_inr_fp16_matches_oracle(dv, orc, c):
    _check(dv, orc, c, BOXES, 1, dv.A.DVNR_FP16, 23, 17, 300, seed=50, dv_tol=2e-3)


def test_render_inr_single_block_no_ghost_and_thin_block(dv, orc):
    # ghost 0 (samples in the outer half voxel clamp to the domain edge) and
    # a block too thin to own any pixel centre next to a regular one
    c = dict(P.configs_blobs64(), width=16, hidden=1)
    boxes = [((0, 0, 0), (30, 12, 20)), ((30, 0, 0), (32, 12, 20))]
    # (pixel centres at x = -0.5 + (px + 0.5) 32/7: the last, 29.2, is left of 29.5)
    _check(dv, orc, c, boxes, 0, dv.A.DVNR_FP32, 7, 5, 129, seed=60, dv_tol=2e-5)


def test_render_inr_rejects_mixed_precisions(dv):
    c = dict(P.configs_blobs64(), width=16, hidden=1)
    a = _model(dv, c, 0, (0, 0, 0), (8, 8, 8), 1)
    b = _model(dv, c, 0, (8, 0, 0), (16, 8, 8), 1)
    b.set_precision(dv.A.DVNR_FP16)
    with pytest.raises(dv.A.DvnrError):
        dv.render_inr([a, b], dv.make_tf(**TF), 8, 8, 16)
