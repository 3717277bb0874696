"""Trajectory parity on the 256^3 workload: after 200 seeded training steps of
the 256^3 spectral-field model (L=16, F=2, T=2^19, N_min=16, b=1.38, MLP
32-64-64-64-1), both GPU paths reach the PSNR of the FP64 oracle within
0.2 dB (Sec. 5: PSNR from the mean squared error).

The batch is 2^15 samples per step (the workload's is 2^18) so that the
oracle's 200 steps take well under a minute on the host cores; model, volume,
sampler and Adam are the workload's. The learning rate is 5e-4, where a
200-step point is stable under tiny perturbations (at 1e-2 training is
chaotic, see the 64^3 ensemble test). PSNR is taken over 2^16 seeded voxels of
the 256^3 grid, the same voxels on both sides (the oracle decodes those
points at their exact grid coordinates; the GPU decodes its whole grid).
Both the plain FP32 path and the FP16 tensor-core path are compared with the
plain FP64 oracle (no FP16 emulation): this is the FP16 path's end-to-end
error against FP64.
"""
import numpy as np
import pytest

import parity as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STEPS, BATCH, LR, SEED, INIT = 200, 1 << 15, 5e-4, 99, 4242


@pytest.fixture(scope="module")
def dv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_10516_gb300 import model as dv

    return dv


@pytest.fixture(scope="module")
def setup(orc):
    from paper_2304_10516_gb300 import volumes

    c = dict(P.configs_spectral256(), batch=BATCH)
    oc = P.oracle_cfg(c)
    vol = volumes.spectral((256, 256, 256), seed=1002)
    rng = np.random.default_rng(7)
    idx = rng.integers(0, 256, size=(1 << 16, 3))  # (x, y, z) voxel indices
    coords = np.array([[orc.grid_coord(int(j), 256) for j in row] for row in idx], dtype=np.uint32)
    truth = vol[idx[:, 2], idx[:, 1], idx[:, 0]].astype(np.float64)
    vmin, vmax = float(vol.min()), float(vol.max())
    th = orc.init_params(oc, INIT)
    m1, m2 = np.zeros_like(th), np.zeros_like(th)
    tc = orc.TrainConfig(batch=BATCH, lr=float(np.float32(LR)), seed=SEED)
    st = orc.State()
    hist = orc.train(oc, tc, st, th, m1, m2, vol, vmin, vmax, STEPS)
    dec = orc.decode_unit(oc, th, coords, vmin, vmax)
    psnr_orc = P.psnr(np.mean((dec - truth) ** 2))
    return dict(c=c, oc=oc, vol=vol, idx=idx, truth=truth, psnr_orc=psnr_orc, loss_orc=hist[-1])


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_256_model_200_steps_psnr_matches_fp64_oracle(dv, setup, prec):
    from paper_2304_10516_gb300 import _abi as A

    c, vol, idx = setup["c"], setup["vol"], setup["idx"]
    precision = A.DVNR_FP16 if prec == "fp16" else A.DVNR_FP32
    m = dv.Model((0, 0, 0), (256, 256, 256), 0,
                 dv.EncodingConfig(c["L"], c["F"], c["log2T"], c["base"], c["growth"]),
                 dv.MLPConfig(c["width"], c["hidden"]), seed=INIT)
    vt = torch.from_numpy(vol).cuda()
    losses = dv.train([m], [vt], dv.TrainConfig(batch=BATCH, steps=STEPS, lr=LR, seed=SEED,
                                                 precision=precision))
    st = m.state()
    assert st["adam_t"] == STEPS and st["skipped"] == 0
    grid = m.decode_grid().cpu().numpy().astype(np.float64)
    dec = grid[idx[:, 2], idx[:, 1], idx[:, 0]]
    psnr = P.psnr(np.mean((dec - setup["truth"]) ** 2))
    assert abs(psnr - setup["psnr_orc"]) < 0.2, (prec, psnr, setup["psnr_orc"])
    assert abs(losses[0] - setup["loss_orc"]) < 0.1 * setup["loss_orc"]
    m.close()
