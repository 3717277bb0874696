"""Sort-last compositing (Sec. 4.3) on the GPU: partitions rendered apart in
the global frame and blended in depth order give the image of all of them
rendered together (grid march and network march), whatever the order in
which the images are handed over. The image of all partitions is itself
checked against the oracle by the render tests."""
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


BOXES = [((0, 0, 0), (20, 18, 33)), ((20, 0, 0), (37, 18, 33)),
         ((0, 0, 33), (20, 18, 61)), ((20, 0, 33), (37, 18, 61))]


@pytest.mark.parametrize("from_network", [False, True], ids=["grid", "network"])
def test_partitions_rendered_apart_composite_to_the_whole(dv, from_network):
    c = dict(P.configs_blobs64(), width=16, hidden=1)
    oc = P.oracle_cfg(c)
    enc = dv.EncodingConfig(c["L"], c["F"], c["log2T"], c["base"], c["growth"])
    mlp = dv.MLPConfig(c["width"], c["hidden"])
    models = []
    for i, (lo, hi) in enumerate(BOXES):
        m = dv.Model(lo, hi, 1, enc, mlp, seed=0)
        m.set_weights(P.random_theta(oc, 70 + i, table_scale=0.3))
        models.append(m)
    tf = dv.make_tf(alpha_max=0.05, v_lo=-0.4, v_hi=0.6)
    w, h, spr = 29, 23, 200
    whole = (dv.render_inr(models, tf, w, h, spr) if from_network else dv.render(models, tf, w, h, spr))
    flo, fhi = (0, 0, 0), (37, 18, 61)
    parts = [dv.render_in_frame([m], flo, fhi, tf, w, h, spr, from_network=from_network) for m in models]
    depths = [lo[2] for lo, _ in BOXES]
    got = dv.composite(parts, depths)
    np.testing.assert_allclose(got.cpu().numpy(), whole.cpu().numpy(), atol=2e-6, rtol=0)
    # the blend follows depth, not the order of the images
    perm = [3, 0, 2, 1]
    got2 = dv.composite([parts[i] for i in perm], [depths[i] for i in perm])
    np.testing.assert_allclose(got2.cpu().numpy(), got.cpu().numpy(), atol=1e-7, rtol=0)
    # a part rendered alone is transparent outside its own footprint
    a = parts[1].cpu().numpy()
    assert np.all(a[:, :5] == 0.0) and a[..., 3].max() > 0.0
    # the frame must be a box
    with pytest.raises(dv.A.DvnrError):
        dv.render_in_frame([models[0]], (0, 0, 0), (0, 18, 61), tf, w, h, spr)
