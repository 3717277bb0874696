"""ctypes front end of the FP64 CPU oracle (``dvnr_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
CPU-baseline leg of the benchmark. It never imports the product package and the
product never imports it.

Every function forwards to the C oracle; the docstrings name the passage of the
paper (arXiv 2304.10516) each one follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dvnr_oracle.c")
_HDR = os.path.join(_HERE, "dvnr_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libdvnr_oracle.so")
_lock = threading.Lock()
_lib = None

MAX_LEVELS = 32
MAX_HIDDEN = 8
QTAB = 4096
FIX_ONE = 1 << 24


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, OpenMP on)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Cfg(C.Structure):
    _fields_ = [
        ("L", C.c_int32), ("F", C.c_int32), ("log2T", C.c_int32), ("base_res", C.c_int32),
        ("growth", C.c_double), ("width", C.c_int32), ("n_hidden", C.c_int32),
        ("in_dim", C.c_int32),
        ("N", C.c_int32 * MAX_LEVELS), ("dense", C.c_int32 * MAX_LEVELS),
        ("entries", C.c_int64 * MAX_LEVELS), ("offset", C.c_int64 * MAX_LEVELS),
        ("w_off", C.c_int64 * (MAX_HIDDEN + 1)),
        ("n_enc", C.c_int64), ("n_mlp", C.c_int64), ("n_params", C.c_int64),
    ]


class _TrainCfg(C.Structure):
    _fields_ = [
        ("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double),
        ("weight_decay", C.c_double), ("lambda_bnd", C.c_double), ("sigma_bnd", C.c_double),
        ("batch", C.c_int32), ("loss", C.c_int32), ("mixed", C.c_int32),
        ("growth_interval", C.c_int32), ("seed", C.c_uint64), ("model", C.c_uint32),
    ]


class _State(C.Structure):
    _fields_ = [
        ("loss_scale", C.c_double), ("adam_t", C.c_int64), ("iter", C.c_int64),
        ("good_steps", C.c_int64), ("skipped", C.c_int64),
    ]


_P = C.c_void_p


def _lib_handle():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            lib.orc_cfg_init.argtypes = [C.POINTER(_Cfg), C.c_int32, C.c_int32, C.c_int32,
                                         C.c_int32, C.c_double, C.c_int32, C.c_int32]
            lib.orc_cfg_init.restype = C.c_int
            lib.orc_philox4x32_10.argtypes = [_P, _P, _P]
            lib.orc_round_half.argtypes = [C.c_double]
            lib.orc_round_half.restype = C.c_double
            lib.orc_corner_index.argtypes = [C.POINTER(_Cfg), C.c_int, C.c_int64, C.c_int64, C.c_int64]
            lib.orc_corner_index.restype = C.c_uint32
            lib.orc_init_params.argtypes = [C.POINTER(_Cfg), C.c_uint64, _P]
            lib.orc_quantile_table.argtypes = [C.c_double, _P]
            lib.orc_sample.argtypes = [C.c_uint64, C.c_uint32, C.c_uint64, C.c_int32,
                                       C.c_double, _P, _P]
            lib.orc_sample.restype = C.c_int
            lib.orc_volume_trilinear.argtypes = [_P, C.c_int64, C.c_int64, C.c_int64, _P]
            lib.orc_volume_trilinear.restype = C.c_double
            lib.orc_encode_batch.argtypes = [C.POINTER(_Cfg), _P, C.c_int64, _P, C.c_int, _P]
            lib.orc_targets.argtypes = [_P, C.c_int64, C.c_int64, C.c_int64, C.c_int64, _P,
                                        C.c_double, C.c_double, _P]
            lib.orc_fwd_bwd.argtypes = [C.POINTER(_Cfg), _P, C.c_int64, _P, _P, C.c_int32,
                                        C.c_int32, C.c_double, C.c_int64, _P, _P, _P, _P, _P, _P,
                                        _P]
            lib.orc_fwd_bwd.restype = C.c_double
            lib.orc_adam.argtypes = [C.POINTER(_Cfg), C.POINTER(_TrainCfg), C.POINTER(_State),
                                     _P, _P, _P, _P]
            lib.orc_train.argtypes = [C.POINTER(_Cfg), C.POINTER(_TrainCfg), C.POINTER(_State),
                                      _P, _P, _P, _P, C.c_int64, C.c_int64, C.c_int64,
                                      C.c_double, C.c_double, C.c_int64, _P]
            lib.orc_train.restype = C.c_double
            lib.orc_max_iterations.argtypes = [C.c_int64] * 5
            lib.orc_max_iterations.restype = C.c_int64
            lib.orc_adaptive_encoding.argtypes = [C.c_int64, C.c_int64, C.c_int32, C.c_int32,
                                                  C.c_double, _P, _P]
            lib.orc_stop_step.argtypes = [_P, _P, C.c_int64, C.c_double, C.c_double, _P]
            lib.orc_stop_step.restype = C.c_int64
            lib.orc_train_budget.argtypes = [C.POINTER(_Cfg), C.POINTER(_TrainCfg),
                                             C.POINTER(_State), _P, _P, _P, _P, C.c_int64,
                                             C.c_int64, C.c_int64, C.c_double, C.c_double,
                                             C.c_int64, C.c_double, C.c_double, _P, _P, _P]
            lib.orc_train_budget.restype = C.c_int64
            lib.orc_decode_unit.argtypes = [C.POINTER(_Cfg), _P, C.c_int64, _P, C.c_int,
                                            C.c_double, C.c_double, _P]
            lib.orc_grid_coord.argtypes = [C.c_int64, C.c_int64]
            lib.orc_grid_coord.restype = C.c_uint32
            lib.orc_decode_grid.argtypes = [C.POINTER(_Cfg), _P, _P, C.c_int32, C.c_int,
                                            C.c_double, C.c_double, _P]
            lib.orc_render.argtypes = [C.c_int32, _P, _P, _P, _P, C.c_int32, C.c_int32,
                                       C.c_int32, _P]
            lib.orc_render_inr.argtypes = [C.POINTER(_Cfg), C.c_int32, _P, _P, _P, _P, C.c_int,
                                           _P, _P, _P, C.c_int32, C.c_int32, C.c_int32,
                                           C.c_int64, _P, _P]
            lib.orc_mse.argtypes = [_P, _P, C.c_int64, _P]
            lib.orc_mse.restype = C.c_double
            lib.orc_threads.restype = C.c_int
            lib.orc_set_threads.argtypes = [C.c_int]
            lib.orc_set_threads.restype = C.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _arr(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class Config:
    """Encoding + MLP configuration with the derived parameter layout
    (hash encoding of Sec. 3; level resolution N_l = floor(N_min b^l))."""

    def __init__(self, L, F, log2T, base_res, growth, width, n_hidden):
        self._c = _Cfg()
        rc = _lib_handle().orc_cfg_init(C.byref(self._c), L, F, log2T, base_res, float(growth),
                                        width, n_hidden)
        if rc != 0:
            raise ValueError("invalid oracle configuration")

    def __getattr__(self, name):
        c = self.__dict__["_c"]
        if name in ("N", "dense", "entries", "offset"):
            return [int(v) for v in getattr(c, name)[: c.L]]
        if name == "w_off":
            return [int(v) for v in c.w_off[: c.n_hidden + 1]]
        return getattr(c, name)

    @property
    def ref(self):
        return C.byref(self._c)


def philox4x32_10(ctr, key):
    """Philox-4x32-10 block (Salmon et al. 2011)."""
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _lib_handle().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def round_half(x):
    """binary16 round-to-nearest-even of each element (kept as float64)."""
    f = _lib_handle().orc_round_half
    a = np.asarray(x, dtype=np.float64)
    return np.array([f(float(v)) for v in a.ravel()]).reshape(a.shape)


def corner_index(cfg: Config, level, x, y, z):
    return int(_lib_handle().orc_corner_index(cfg.ref, level, int(x), int(y), int(z)))


def init_params(cfg: Config, seed: int):
    theta = np.zeros(cfg.n_params, dtype=np.float64)
    _lib_handle().orc_init_params(cfg.ref, seed, _ptr(theta))
    return theta


def quantile_table(sigma: float):
    tab = np.zeros(QTAB + 1, dtype=np.int64)
    _lib_handle().orc_quantile_table(float(sigma), _ptr(tab))
    return tab


def sample(seed, model, it, batch, lambda_bnd, qtab):
    """Fixed-point training coordinates of one iteration (Sec. 3.2-3.3)."""
    m = np.zeros((batch, 3), dtype=np.uint32)
    q = _arr(qtab, np.int64)
    _lib_handle().orc_sample(seed, model, it, batch, float(lambda_bnd), _ptr(q), _ptr(m))
    return m


def volume_trilinear(vol, m):
    v = _arr(vol, np.float32)
    mm = _arr(m, np.uint32)
    nz, ny, nx = v.shape
    return _lib_handle().orc_volume_trilinear(_ptr(v), nx, ny, nz, _ptr(mm))


def targets(vol, m, vmin, vmax):
    v = _arr(vol, np.float32)
    mm = _arr(m, np.uint32).reshape(-1, 3)
    nz, ny, nx = v.shape
    out = np.zeros(mm.shape[0], dtype=np.float64)
    _lib_handle().orc_targets(_ptr(v), nx, ny, nz, mm.shape[0], _ptr(mm), float(vmin),
                              float(vmax), _ptr(out))
    return out


def encode(cfg: Config, theta, m, mixed=False):
    th = _arr(theta, np.float64)
    mm = _arr(m, np.uint32).reshape(-1, 3)
    out = np.zeros((mm.shape[0], cfg.in_dim), dtype=np.float64)
    _lib_handle().orc_encode_batch(cfg.ref, _ptr(th), mm.shape[0], _ptr(mm), int(mixed), _ptr(out))
    return out


def fwd_bwd(cfg: Config, theta, m, target, loss=0, mixed=False, loss_scale=1.0,
            grad_norm_count=None, flip=None, want_grads=True, want_zabs=False, want_enc=True):
    """Forward + backward of one batch. Returns a dict with loss, grad_enc,
    grad_mlp, y, dx0, margin and optionally zabs (see the C header)."""
    th = _arr(theta, np.float64)
    mm = _arr(m, np.uint32).reshape(-1, 3)
    n = mm.shape[0]
    t = _arr(target, np.float64)
    ge = np.zeros(cfg.n_enc, dtype=np.float64) if (want_grads and want_enc) else None
    gm = np.zeros(cfg.n_mlp, dtype=np.float64) if want_grads else None
    y = np.zeros(n, dtype=np.float64)
    dx0 = np.zeros((n, cfg.in_dim), dtype=np.float64)
    margin = np.zeros(n, dtype=np.float64)
    fl = None if flip is None else _arr(flip, np.uint8)
    zabs = np.zeros((n, cfg.n_hidden * cfg.width + 1)) if want_zabs else None
    lval = _lib_handle().orc_fwd_bwd(
        cfg.ref, _ptr(th), n, _ptr(mm), _ptr(t), int(loss), int(mixed), float(loss_scale),
        int(grad_norm_count or n), _ptr(fl), _ptr(ge), _ptr(gm), _ptr(y), _ptr(dx0), _ptr(margin),
        _ptr(zabs))
    return dict(loss=lval, grad_enc=ge, grad_mlp=gm, y=y, dx0=dx0, margin=margin, zabs=zabs)


class TrainConfig:
    def __init__(self, batch, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=1e-9,
                 lambda_bnd=0.0, sigma_bnd=0.005, loss=0, mixed=False, growth_interval=2000,
                 seed=0, model=0):
        self._t = _TrainCfg(lr, beta1, beta2, eps, weight_decay, lambda_bnd, sigma_bnd,
                            batch, loss, int(mixed), growth_interval, seed, model)

    @property
    def ref(self):
        return C.byref(self._t)

    def __getattr__(self, name):
        return getattr(self.__dict__["_t"], name)


class State:
    def __init__(self, loss_scale=1.0):
        self._s = _State(loss_scale, 0, 0, 0, 0)

    @property
    def ref(self):
        return C.byref(self._s)

    def __getattr__(self, name):
        return getattr(self.__dict__["_s"], name)


def adam(cfg: Config, tc: TrainConfig, st: State, theta, mom1, mom2, grad):
    """One Adam step in place (Sec. 3.6)."""
    for a in (theta, mom1, mom2):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _arr(grad, np.float64)
    _lib_handle().orc_adam(cfg.ref, tc.ref, st.ref, _ptr(theta), _ptr(mom1), _ptr(mom2), _ptr(g))


def train(cfg: Config, tc: TrainConfig, st: State, theta, mom1, mom2, vol, vmin, vmax, steps):
    """``steps`` training iterations in place (Sec. 3.2); returns the loss history."""
    v = _arr(vol, np.float32)
    nz, ny, nx = v.shape
    hist = np.zeros(steps, dtype=np.float64)
    for a in (theta, mom1, mom2):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    _lib_handle().orc_train(cfg.ref, tc.ref, st.ref, _ptr(theta), _ptr(mom1), _ptr(mom2), _ptr(v),
                            nx, ny, nz, float(vmin), float(vmax), steps, _ptr(hist))
    return hist


def max_iterations(n_vox, batch, steps=0, epochs=0, min_steps=0):
    """N_train^max of one call (Sec. 3.2)."""
    return int(_lib_handle().orc_max_iterations(int(n_vox), int(batch), int(steps), int(epochs),
                                                int(min_steps)))


def adaptive_encoding(n_vox, n_vox_global, log2_T_ref, log2_T_min, R_ref):
    """(log2 T, R_0) of a partition (Sec. 3.2 reading)."""
    a, b = C.c_int32(), C.c_int32()
    _lib_handle().orc_adaptive_encoding(int(n_vox), int(n_vox_global), int(log2_T_ref),
                                        int(log2_T_min), float(R_ref), C.byref(a), C.byref(b))
    return a.value, b.value


def stop_step(losses, decay, stop_loss, finite=None):
    """(steps run, final moving average) of the Sec. 3.2 early stop applied
    to a recorded loss sequence."""
    L = _arr(losses, np.float64)
    fin = None if finite is None else _arr(finite, np.int32)
    ema = C.c_double()
    n = _lib_handle().orc_stop_step(_ptr(L), None if fin is None else _ptr(fin), L.size,
                                    float(decay), float(stop_loss), C.byref(ema))
    return int(n), ema.value


def train_budget(cfg: Config, tc: TrainConfig, st: State, theta, mom1, mom2, vol, vmin, vmax,
                 budget, stop_loss=0.0, decay=0.9):
    """Training under the budget and early stop of one call (Sec. 3.2), in
    place; returns (steps run, loss history, final moving average, stopped)."""
    v = _arr(vol, np.float32)
    nz, ny, nx = v.shape
    hist = np.zeros(max(int(budget), 1), dtype=np.float64)
    for a in (theta, mom1, mom2):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    ema = C.c_double()
    stopped = C.c_int32()
    n = _lib_handle().orc_train_budget(cfg.ref, tc.ref, st.ref, _ptr(theta), _ptr(mom1),
                                       _ptr(mom2), _ptr(v), nx, ny, nz, float(vmin), float(vmax),
                                       int(budget), float(stop_loss), float(decay), _ptr(hist),
                                       C.byref(ema), C.byref(stopped))
    return int(n), hist[:n], ema.value, bool(stopped.value)


def decode_unit(cfg: Config, theta, m, vmin, vmax, mixed=False):
    th = _arr(theta, np.float64)
    mm = _arr(m, np.uint32).reshape(-1, 3)
    out = np.zeros(mm.shape[0], dtype=np.float64)
    _lib_handle().orc_decode_unit(cfg.ref, _ptr(th), mm.shape[0], _ptr(mm), int(mixed),
                                  float(vmin), float(vmax), _ptr(out))
    return out


def grid_coord(j, n):
    return int(_lib_handle().orc_grid_coord(int(j), int(n)))


def decode_grid(cfg: Config, theta, dims_stored, ghost, vmin, vmax, mixed=False):
    """Owned voxels of a block of stored dims (nx, ny, nz); returns (ez, ey, ex)."""
    th = _arr(theta, np.float64)
    n = np.asarray(dims_stored, dtype=np.int64)
    e = n - 2 * ghost
    out = np.zeros(int(e[0] * e[1] * e[2]), dtype=np.float64)
    _lib_handle().orc_decode_grid(cfg.ref, _ptr(th), _ptr(n), int(ghost), int(mixed),
                                  float(vmin), float(vmax), _ptr(out))
    return out.reshape(int(e[2]), int(e[1]), int(e[0]))


def render(grids, lo, hi, tf, w, h, spr):
    """Front-to-back ray march of decoded blocks (Sec. 4.3 reading)."""
    gs = [_arr(g, np.float64) for g in grids]
    ptrs = (C.c_void_p * len(gs))(*[g.ctypes.data for g in gs])
    lo_a = _arr(lo, np.int64).reshape(-1, 3)
    hi_a = _arr(hi, np.int64).reshape(-1, 3)
    tf_a = _arr(tf, np.float64)
    out = np.zeros((h, w, 4), dtype=np.float64)
    _lib_handle().orc_render(len(gs), C.cast(ptrs, C.c_void_p), _ptr(lo_a), _ptr(hi_a), _ptr(tf_a),
                             w, h, spr, _ptr(out))
    return out


def render_inr(cfg: Config, thetas, lo, hi, ghost, vmin, vmax, tf, w, h, spr, pixels=None,
               mixed=False):
    """Ray-march the networks of the blocks directly (Sec. 4.3 reading, the
    conventions of `render`). pixels: indices py * w + px (all if None).
    Returns (h, w, 4) for the whole image, else (len(pixels), 4)."""
    ths = [_arr(t, np.float64) for t in thetas]
    nb = len(ths)
    ptrs = (C.c_void_p * nb)(*[t.ctypes.data for t in ths])
    lo_a = _arr(lo, np.int64).reshape(-1, 3)
    hi_a = _arr(hi, np.int64).reshape(-1, 3)
    g = _arr(np.broadcast_to(np.asarray(ghost), (nb,)), np.int32)
    vmn = _arr(np.broadcast_to(np.asarray(vmin, dtype=np.float64), (nb,)), np.float64)
    vmx = _arr(np.broadcast_to(np.asarray(vmax, dtype=np.float64), (nb,)), np.float64)
    pix = _arr(np.arange(w * h) if pixels is None else pixels, np.int64)
    out = np.zeros((pix.size, 4), dtype=np.float64)
    tfa = _arr(tf, np.float64)
    _lib_handle().orc_render_inr(cfg.ref, nb, C.cast(ptrs, C.c_void_p), _ptr(lo_a), _ptr(hi_a),
                                 _ptr(g), int(mixed), _ptr(vmn), _ptr(vmx), _ptr(tfa), w, h, spr,
                                 pix.size, _ptr(pix), _ptr(out))
    return out.reshape(h, w, 4) if pixels is None else out


def mse(a, b):
    aa = _arr(a, np.float64).ravel()
    bb = _arr(b, np.float32).ravel()
    mx = C.c_double(0.0)
    v = _lib_handle().orc_mse(_ptr(aa), _ptr(bb), aa.size, C.byref(mx))
    return v, mx.value


def threads():
    return int(_lib_handle().orc_threads())


def set_threads(n):
    """Threads of the oracle's parallel loops (timing only); returns the count in effect."""
    return int(_lib_handle().orc_set_threads(int(n)))
