"""Seeded synthetic volumes and partitions that stand in for the paper's data.

This module only draws inputs: it holds none of the method's arithmetic
(no encoding, network, loss, optimiser, decoding or rendering), so both the
CUDA path and the CPU oracle can be fed from it.

The paper trains on simulation fields (S3D, NekRS, CloverLeaf) and post hoc
volumes that are not available here (Sec. 5). The stand-ins:

* ``blobs``: a sum of 8 seeded Gaussian blobs plus a low-frequency sinusoid,
  normalised to [0, 1] (64^3 workload).
* ``spectral``: a random-phase field whose energy spectrum falls as k^-5/3
  (mode amplitude ~ k^-11/6, k = 0 dropped, Hermitian through an inverse real
  FFT), normalised to [0, 1] -- the turbulence-like 256^3 workload.
* ``advected``: the same spectrum advected by a uniform drift with viscous
  decay of the high modes, for in situ time series.
* ``front``: a thin front across a randomly wrinkled surface (a tanh
  profile about 1.5 voxels thick) over a gentle background, normalised to
  [0, 1] -- a field with a sharp, localised feature, the kind the paper's
  combustion fields have and the spectral field lacks.
* ``uneven_boxes``: a rectangular decomposition into blocks of uneven edge
  (Sec. 3.1 assumes one box per rank), with a ghost layer (Sec. 3.3).
"""
from __future__ import annotations

import numpy as np


def blobs(n: int = 64, seed: int = 1001, n_blobs: int = 8) -> np.ndarray:
    """(n, n, n) float32 indexed [z, y, x]; voxel centre i sits at i/(n-1)."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.15, 0.85, size=(n_blobs, 3))
    s = rng.uniform(0.04, 0.12, size=n_blobs)
    a = rng.uniform(0.5, 1.0, size=n_blobs)
    t = np.linspace(0.0, 1.0, n)
    z, y, x = np.meshgrid(t, t, t, indexing="ij")
    f = 0.3 * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y) * np.sin(2 * np.pi * z)
    for i in range(n_blobs):
        r2 = (x - c[i, 0]) ** 2 + (y - c[i, 1]) ** 2 + (z - c[i, 2]) ** 2
        f += a[i] * np.exp(-r2 / (2 * s[i] ** 2))
    f = (f - f.min()) / (f.max() - f.min())
    return f.astype(np.float32)


def front(shape=(256, 256, 256), seed=1006, width=1.5, modes=6) -> np.ndarray:
    """(nz, ny, nx) float32 indexed [z, y, x]: 0.5 + 0.5 tanh((z - h(x, y)) /
    width) with h a random-phase sum of modes (kx, ky) in [1, modes]^2 of
    amplitude ~ 1/|k| (total excursion about nz/10 voxels) around nz/2, plus a
    background 0.15 sin(2 pi x) cos(2 pi y); normalised to [0, 1]."""
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    x = np.arange(nx) / nx
    y = np.arange(ny) / ny
    X, Y = np.meshgrid(x, y, indexing="xy")  # (ny, nx)
    h = np.full((ny, nx), nz / 2.0)
    amp = nz / 10.0 / modes
    for kx in range(1, modes + 1):
        for ky in range(1, modes + 1):
            a = amp / np.hypot(kx, ky) * rng.uniform(0.5, 1.5)
            h += a * np.sin(2 * np.pi * (kx * X + ky * Y) + rng.uniform(0, 2 * np.pi))
    z = np.arange(nz, dtype=np.float64)[:, None, None]
    f = 0.5 + 0.5 * np.tanh((z - h[None]) / width)
    f += 0.15 * (np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y))[None]
    return _normalise(f).astype(np.float32)


def _spectral_coeffs(shape, seed, slope):
    """Random-phase half-spectrum for a field of ``shape`` = (nz, ny, nx)."""
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    kz = np.fft.fftfreq(nz) * nz
    ky = np.fft.fftfreq(ny) * ny
    kx = np.fft.rfftfreq(nx) * nx
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    k = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    amp = np.zeros_like(k)
    nz_mask = k > 0
    # 3-D energy spectrum E(k) ~ k^slope spread over a shell of area ~ k^2:
    # |a(k)|^2 ~ k^(slope - 2), so |a(k)| ~ k^((slope - 2)/2) = k^-11/6 at -5/3.
    amp[nz_mask] = k[nz_mask] ** ((slope - 2.0) / 2.0)
    phase = rng.uniform(0.0, 2 * np.pi, size=k.shape)
    return amp * np.exp(1j * phase), (KX, KY, KZ, k)


def _normalise(f):
    f = f - f.min()
    m = f.max()
    return (f / m if m > 0 else f).astype(np.float32)


def spectral(shape=(256, 256, 256), seed: int = 1002, slope: float = -5.0 / 3.0) -> np.ndarray:
    """Random-phase k^-5/3 field, float32 [z, y, x], normalised to [0, 1]."""
    coef, _ = _spectral_coeffs(shape, seed, slope)
    f = np.fft.irfftn(coef, s=shape, axes=(0, 1, 2))
    return _normalise(f)


def spectral_torch(shape, seed: int, device="cuda", slope: float = -5.0 / 3.0):
    """The same field family generated with torch.fft in float32 on ``device``
    (for the large partitioned workload); returns a float32 tensor [z, y, x]."""
    import torch

    nz, ny, nx = shape
    g = torch.Generator(device="cpu").manual_seed(seed)
    kz = torch.fft.fftfreq(nz, device=device) * nz
    ky = torch.fft.fftfreq(ny, device=device) * ny
    kx = torch.fft.rfftfreq(nx, device=device) * nx
    k2 = kz.view(-1, 1, 1) ** 2 + ky.view(1, -1, 1) ** 2 + kx.view(1, 1, -1) ** 2
    k = torch.sqrt(k2)
    amp = torch.where(k > 0, k.clamp_min(1e-30) ** ((slope - 2.0) / 2.0), torch.zeros_like(k))
    del k, k2
    phase = torch.rand(amp.shape, generator=g, dtype=torch.float32).to(device) * (2 * np.pi)
    coef = torch.polar(amp, phase)
    del amp, phase
    f = torch.fft.irfftn(coef, s=shape, dim=(0, 1, 2))
    del coef
    f -= f.min()
    f /= f.max()
    return f.contiguous()


def advected(shape, seed: int, t: float, velocity=(3.0, 2.0, 1.0), nu: float | None = None,
             slope: float = -5.0 / 3.0) -> np.ndarray:
    """Spectral field advected by ``velocity`` voxels per step for ``t`` steps,
    with viscous decay exp(-nu |k|^2 t); by default nu halves the top octave
    over 16 steps. Float32 [z, y, x], normalised to [0, 1]."""
    nz, ny, nx = shape
    coef, (KX, KY, KZ, k) = _spectral_coeffs(shape, seed, slope)
    if nu is None:
        kmax = np.sqrt((nx / 2) ** 2 + (ny / 2) ** 2 + (nz / 2) ** 2)
        nu = np.log(2.0) / (16.0 * kmax ** 2)
    vx, vy, vz = velocity
    shift = np.exp(-2j * np.pi * (KX * vx / nx + KY * vy / ny + KZ * vz / nz) * t)
    f = np.fft.irfftn(coef * shift * np.exp(-nu * k ** 2 * t), s=shape, axes=(0, 1, 2))
    return _normalise(f)


def uneven_edges(total: int, parts: int, lo: int, hi: int, rng) -> list[int]:
    """``parts`` integer edges in [lo, hi] that sum to ``total``."""
    if not (parts * lo <= total <= parts * hi):
        raise ValueError("edges cannot tile the extent")
    for _ in range(10000):
        e = rng.integers(lo, hi + 1, size=parts)
        diff = total - int(e.sum())
        i = 0
        while diff != 0 and i < 100 * parts:
            j = i % parts
            step = 1 if diff > 0 else -1
            if lo <= e[j] + step <= hi:
                e[j] += step
                diff -= step
            i += 1
        if diff == 0:
            return [int(v) for v in e]
    raise RuntimeError("no edge split found")


def uneven_boxes(extent=(512, 512, 512), parts=(4, 4, 4), edge=(96, 160), seed: int = 1004):
    """Rectangular decomposition of [0, extent) into parts[0] x parts[1] x
    parts[2] boxes with seeded uneven edges; returns a list of (lo, hi) with
    lo, hi = (x, y, z) integer tuples, x fastest in block order."""
    rng = np.random.default_rng(seed)
    cuts = []
    for a in range(3):
        e = uneven_edges(extent[a], parts[a], edge[0], edge[1], rng)
        cuts.append(np.concatenate([[0], np.cumsum(e)]).astype(int))
    boxes = []
    for kz in range(parts[2]):
        for ky in range(parts[1]):
            for kx in range(parts[0]):
                lo = (int(cuts[0][kx]), int(cuts[1][ky]), int(cuts[2][kz]))
                hi = (int(cuts[0][kx + 1]), int(cuts[1][ky + 1]), int(cuts[2][kz + 1]))
                boxes.append((lo, hi))
    return boxes


def extract_block(field, lo, hi, ghost: int = 1):
    """Stored block of a [z, y, x] field: the owned box plus ``ghost`` layers,
    edge-replicated where the ghost layer leaves the field. Works on numpy
    arrays and torch tensors; returns the same kind, contiguous."""
    idx = []
    for a in (2, 1, 0):  # z, y, x order of the array axes
        n = field.shape[2 - a]
        r = np.clip(np.arange(lo[a] - ghost, hi[a] + ghost), 0, n - 1)
        idx.append(r)
    if hasattr(field, "index_select"):
        import torch

        t = field
        for ax, r in enumerate(idx):
            t = t.index_select(ax, torch.as_tensor(r, device=field.device))
        return t.contiguous()
    return np.ascontiguousarray(field[np.ix_(idx[0], idx[1], idx[2])])


def advected_torch(shape, seed: int, t: float, velocity=(3.0, 2.0, 1.0), nu: float | None = None,
                   device="cuda", slope: float = -5.0 / 3.0):
    """`advected` generated with torch.fft in float32 on ``device`` (for the
    512^3 in situ series); returns a float32 tensor [z, y, x] in [0, 1]."""
    import math

    import torch

    nz, ny, nx = shape
    g = torch.Generator(device="cpu").manual_seed(seed)
    kz = torch.fft.fftfreq(nz, device=device) * nz
    ky = torch.fft.fftfreq(ny, device=device) * ny
    kx = torch.fft.rfftfreq(nx, device=device) * nx
    KZ, KY, KX = kz.view(-1, 1, 1), ky.view(1, -1, 1), kx.view(1, 1, -1)
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    k = torch.sqrt(k2)
    if nu is None:
        kmax2 = (nx / 2) ** 2 + (ny / 2) ** 2 + (nz / 2) ** 2
        nu = math.log(2.0) / (16.0 * kmax2)
    amp = torch.where(k > 0, k.clamp_min(1e-30) ** ((slope - 2.0) / 2.0), torch.zeros_like(k))
    amp = amp * torch.exp(-nu * k2 * t)
    del k
    phase = torch.rand(amp.shape, generator=g, dtype=torch.float32).to(device) * (2 * math.pi)
    vx, vy, vz = velocity
    phase = phase - 2 * math.pi * t * (KX * (vx / nx) + KY * (vy / ny) + KZ * (vz / nz))
    coef = torch.polar(amp, phase)
    del amp, phase, k2
    f = torch.fft.irfftn(coef, s=shape, dim=(0, 1, 2))
    del coef
    f -= f.min()
    f /= f.max()
    return f.contiguous()
