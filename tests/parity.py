"""Helpers shared by the GPU parity tests (test infrastructure only).

The GPU evaluates the network in FP32 (or FP16 operands) and the oracle in
FP64. Where a pre-activation z or the L1 residual y - t lies within rounding
distance of zero, the two may legitimately take different branches (ReLU
derivative 0 or 1, L1 sign -1/0/+1). `kink_allowance` asks the oracle how
much such a flip can change the batch gradient: for every sample with a unit
closer than `delta` to its kink it evaluates that sample alone under every
combination of flips of its near-kink units and adds the largest change.
Per-sample quantities of flagged samples are left out of elementwise checks.
"""
from __future__ import annotations

import itertools

import numpy as np

import oracle as orc


def configs_blobs64():
    """Config of the 64^3 blob workload: L=8, F=2, T=2^15, N_min=4, b=1.5,
    MLP 16->32->32->1, batch 4096."""
    return dict(L=8, F=2, log2T=15, base=4, growth=1.5, width=32, hidden=2, batch=4096)


def configs_spectral256():
    """Config of the 256^3 spectral workload: L=16, F=2, T=2^19, N_min=16,
    b=1.38, MLP 32->64->64->64->1, batch 2^18."""
    return dict(L=16, F=2, log2T=19, base=16, growth=1.38, width=64, hidden=3, batch=1 << 18)


def oracle_cfg(c):
    return orc.Config(c["L"], c["F"], c["log2T"], c["base"], c["growth"], c["width"], c["hidden"])


def random_theta(ocfg, seed, table_scale=0.5):
    """Seeded non-trivial parameters in binary32 (tables U(-s, s), MLP
    Glorot from the oracle's initialiser)."""
    rng = np.random.default_rng(seed)
    th = orc.init_params(ocfg, seed).astype(np.float32)
    th[: ocfg.n_enc] = rng.uniform(-table_scale, table_scale, ocfg.n_enc).astype(np.float32)
    return th


def kink_allowance(ocfg, theta, m, t, loss, mixed, scale, batch, zabs, delta, max_units=6):
    """Bound (norm of the table-gradient change, norm of the MLP-gradient
    change) and the flagged sample indices."""
    W, H = ocfg.width, ocfg.n_hidden
    nunits = H * W + 1
    flagged = np.nonzero((zabs < delta).any(axis=1))[0]
    a_enc = 0.0
    a_mlp = 0.0
    for s in flagged:
        units = np.nonzero(zabs[s] < delta)[0][:max_units]
        base = orc.fwd_bwd(ocfg, theta, m[s:s + 1], t[s:s + 1], loss=loss, mixed=mixed,
                           loss_scale=scale, grad_norm_count=batch)
        worst_e = worst_m = 0.0
        for r in range(1, len(units) + 1):
            for sub in itertools.combinations(units, r):
                fl = np.zeros((1, nunits), np.uint8)
                fl[0, list(sub)] = 1
                g = orc.fwd_bwd(ocfg, theta, m[s:s + 1], t[s:s + 1], loss=loss, mixed=mixed,
                                loss_scale=scale, grad_norm_count=batch, flip=fl)
                worst_e = max(worst_e, np.linalg.norm(g["grad_enc"] - base["grad_enc"]))
                worst_m = max(worst_m, np.linalg.norm(g["grad_mlp"] - base["grad_mlp"]))
        a_enc += worst_e
        a_mlp += worst_m
    return a_enc, a_mlp, flagged


def assert_normwise(got, want, tol, allowance=0.0, what=""):
    err = float(np.linalg.norm(np.asarray(got, np.float64) - want))
    ref = float(np.linalg.norm(want))
    assert err <= tol * ref + allowance, f"{what}: |err| {err:.3e} > {tol:.1e} * {ref:.3e} + {allowance:.3e}"
    return err / max(ref, 1e-300)


def psnr(mse, value_range=1.0):
    return 20 * np.log10(value_range) - 10 * np.log10(mse)
