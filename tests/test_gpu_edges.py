"""Edge cases of the hot path against the oracle, on both GPU paths.

- A batch of one sample (one tile whose other 127 rows are padding) and a
  batch of 129 (a full tile and a tile of one).
- The smallest stored block, 2 x 2 x 2 voxels: one cell for the target
  lookup (Sec. 3.2), every encoding level over the same unit cube.
- A constant volume: max = min, so the min/max normalisation's guard sets
  every target to 0.
- Coordinates on the unit cube's faces, u = 0 and u = 1 exactly (fixed point
  0 and 2^24): the lattice clamp puts u = 1 in the last cell with fraction 1.
- Zero points: forward and decode_points return at once; the backward
  rejects n = 0 with DVNR_E_INVALID.
"""
import numpy as np
import pytest

import parity as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32, FP16 = 0, 1


@pytest.fixture(scope="module")
def dv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_10516_gb300 import model as dv

    return dv


def _model(dv, c, dims, seed=0):
    enc = dv.EncodingConfig(c["L"], c["F"], c["log2T"], c["base"], c["growth"])
    return dv.Model((0, 0, 0), dims, 0, enc, dv.MLPConfig(c["width"], c["hidden"]), seed=seed)


def _step_against_oracle(dv, orc, c, vol, prec, seed, it, theta_seed=41):
    """One train_grad step against orc.fwd_bwd on the same samples: bit-exact
    coordinates, targets to 2e-6, y, dL/dx0 and gradients within 1e-5 (FP32)
    or 2e-3 (FP16, against the oracle's binary16 emulation)."""
    oc = P.oracle_cfg(c)
    theta = P.random_theta(oc, theta_seed, table_scale=0.4)
    m = _model(dv, c, vol.shape[::-1])
    m.set_weights(theta)
    B = c["batch"]
    mixed = prec == FP16
    tol = 2e-3 if mixed else 1e-5
    out = m.train_grad(torch.from_numpy(vol).cuda(), dv.TrainConfig(batch=B, loss=0, seed=seed, precision=prec),
                       iteration=it)
    torch.cuda.synchronize()
    coords = orc.sample(seed, 0, it, B, 0.0, orc.quantile_table(0.005))
    np.testing.assert_array_equal(out["coords"].cpu().numpy().view(np.uint32), coords)
    vmin, vmax = float(vol.min()), float(vol.max())
    t = orc.targets(vol, coords, vmin, vmax)
    np.testing.assert_allclose(out["target"].cpu().numpy(), t, atol=2e-6, rtol=0)
    S = float(2 ** round(np.log2(B))) if mixed else 1.0
    th64 = theta.astype(np.float64)
    r = orc.fwd_bwd(oc, th64, coords, t, loss=0, mixed=mixed, loss_scale=S, want_zabs=True)
    y = out["y"].cpu().numpy()
    np.testing.assert_allclose(y, r["y"], atol=tol * max(1.0, np.abs(r["y"]).max()), rtol=0)
    a_enc, a_mlp, flagged = P.kink_allowance(oc, th64, coords, t, 0, mixed, S, B, r["zabs"], delta=1e-4)
    keep = np.ones(B, bool)
    keep[flagged] = False
    if keep.any():
        P.assert_normwise(out["dx0"].cpu().numpy()[keep], r["dx0"][keep], tol, what="dL/dx0")
    g = out["grad"].cpu().numpy()
    P.assert_normwise(g[: oc.n_enc], r["grad_enc"], tol, a_enc, what="table grad")
    P.assert_normwise(g[oc.n_enc:], r["grad_mlp"], tol, a_mlp, what="mlp grad")
    m.close()
    return out


@pytest.mark.parametrize("prec", [FP32, FP16], ids=["fp32", "fp16"])
@pytest.mark.parametrize("batch", [1, 129])
def test_tiny_batches_match_oracle(dv, orc, prec, batch):
    from paper_2304_10516_gb300 import volumes

    c = dict(P.configs_blobs64(), batch=batch)
    _step_against_oracle(dv, orc, c, volumes.blobs(16, seed=1005), prec, seed=11, it=3)


@pytest.mark.parametrize("prec", [FP32, FP16], ids=["fp32", "fp16"])
def test_smallest_block_matches_oracle(dv, orc, prec):
    rng = np.random.default_rng(12)
    vol = rng.uniform(-1.0, 2.0, size=(2, 2, 2)).astype(np.float32)
    c = dict(P.configs_blobs64(), batch=512)
    _step_against_oracle(dv, orc, c, vol, prec, seed=13, it=0)


@pytest.mark.parametrize("prec", [FP32, FP16], ids=["fp32", "fp16"])
def test_constant_volume_targets_are_zero(dv, orc, prec):
    vol = np.full((8, 8, 8), 0.7, dtype=np.float32)
    c = dict(P.configs_blobs64(), batch=256)
    out = _step_against_oracle(dv, orc, c, vol, prec, seed=14, it=1)
    assert not out["target"].any()


@pytest.mark.parametrize("prec", [FP32, FP16], ids=["fp32", "fp16"])
def test_forward_on_the_cube_faces(dv, orc, prec):
    c = P.configs_blobs64()
    oc = P.oracle_cfg(c)
    theta = P.random_theta(oc, 43, table_scale=0.4)
    m = _model(dv, c, (16, 16, 16))
    m.set_weights(theta)
    one = 1 << 24
    corners = np.array([[x, y, z] for z in (0, one) for y in (0, one) for x in (0, one)], dtype=np.uint32)
    rng = np.random.default_rng(15)
    faces = rng.integers(0, one + 1, size=(120, 3)).astype(np.uint32)
    faces[np.arange(120), rng.integers(0, 3, 120)] = rng.choice([0, one], 120).astype(np.uint32)
    coords = np.concatenate([corners, faces])
    y = m.forward(torch.from_numpy(coords.view(np.int32)).cuda(), prec).cpu().numpy()
    want = orc.decode_unit(oc, theta.astype(np.float64), coords, 0.0, 1.0, mixed=prec == FP16)
    tol = 2e-3 if prec == FP16 else 1e-5
    np.testing.assert_allclose(y, want, atol=tol * max(1.0, np.abs(want).max()), rtol=0)
    m.close()


def test_zero_points(dv):
    from paper_2304_10516_gb300 import _abi as A

    c = P.configs_blobs64()
    m = _model(dv, c, (16, 16, 16))
    empty = torch.empty((0, 3), dtype=torch.int32, device="cuda")
    for prec in (FP32, FP16):
        assert m.forward(empty, prec).numel() == 0
    assert m.decode_points(torch.empty((0, 3), dtype=torch.float32, device="cuda")).numel() == 0
    with pytest.raises(A.DvnrError) as ei:
        m.backward(empty, torch.empty(0, device="cuda"), FP16)
    assert ei.value.status == 1  # DVNR_E_INVALID
    m.close()
