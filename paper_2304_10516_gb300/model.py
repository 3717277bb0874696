"""Python front end of libdvnr: a Model handle and thin wrappers around the
C ABI calls. Tensors are torch tensors on the CUDA device (PyTorch supplies
device memory and streams only); every computation runs in libdvnr.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _abi as A


@dataclass
class EncodingConfig:
    """Hash-grid encoding (the paper's appendix keys n_levels,
    n_features_per_level, log2_hashmap_size, base_resolution, per_level_scale)."""
    n_levels: int = 16
    n_features: int = 2
    log2_T: int = 19
    base_res: int = 16
    growth: float = 1.38


def adaptive_encoding(n_vox: int, n_vox_global: int, log2_T_ref: int = 19, log2_T_min: int = 12,
                      R_ref: float = 16.0, base: EncodingConfig | None = None) -> EncodingConfig:
    """The encoding of a partition with n_vox of n_vox_global voxels: table
    size and base resolution scaled with its share (Sec. 3.2); the other
    fields from `base`."""
    base = base or EncodingConfig()
    ec = A.dvnr_enc_cfg(base.n_levels, base.n_features, base.log2_T, base.base_res, float(base.growth))
    A.call("dvnr_adaptive_encoding", int(n_vox), int(n_vox_global), int(log2_T_ref), int(log2_T_min),
           float(R_ref), C.byref(ec))
    return EncodingConfig(base.n_levels, base.n_features, ec.log2_T, ec.base_res, base.growth)


@dataclass
class MLPConfig:
    """ReLU MLP (appendix keys n_neurons, n_hidden_layers)."""
    width: int = 64
    n_hidden: int = 3


@dataclass
class TrainConfig:
    """Training settings (Sec. 3.2-3.3, 3.6 defaults)."""
    batch: int = 1 << 14
    steps: int = 1
    lr: float = 1e-2
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    weight_decay: float = 1e-9
    lambda_bnd: float = 0.0
    sigma_bnd: float = 0.005
    precision: int = A.DVNR_FP32
    loss: int = A.DVNR_LOSS_L1
    growth_interval: int = 2000
    seed: int = 0
    # Sec. 3.2 iteration budget and early stop (see dvnr_train_cfg)
    epochs: int = 0
    min_steps: int = 0
    stop_loss: float = 0.0
    stop_decay: float = 0.9

    def to_c(self) -> A.dvnr_train_cfg:
        return A.dvnr_train_cfg(self.lr, self.beta1, self.beta2, self.eps, self.weight_decay,
                                self.lambda_bnd, self.sigma_bnd, self.batch, self.precision,
                                self.loss, self.growth_interval, self.steps, self.seed,
                                self.epochs, self.min_steps, self.stop_loss, self.stop_decay)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Model:
    """One INR of a box partition (Sec. 3.1)."""

    def __init__(self, lo, hi, ghost=0, enc: EncodingConfig | None = None,
                 mlp: MLPConfig | None = None, seed: int = 0):
        enc = enc or EncodingConfig()
        mlp = mlp or MLPConfig()
        self.lo, self.hi, self.ghost = tuple(int(v) for v in lo), tuple(int(v) for v in hi), int(ghost)
        self.enc, self.mlp = enc, mlp
        box = A.dvnr_box((C.c_int64 * 3)(*self.lo), (C.c_int64 * 3)(*self.hi), self.ghost)
        ec = A.dvnr_enc_cfg(enc.n_levels, enc.n_features, enc.log2_T, enc.base_res, float(enc.growth))
        mc = A.dvnr_mlp_cfg(mlp.width, mlp.n_hidden)
        h = C.c_void_p()
        A.call("dvnr_create", C.byref(box), C.byref(ec), C.byref(mc), int(seed), C.byref(h))
        self._h = h
        ne, nm = C.c_int64(), C.c_int64()
        A.call("dvnr_param_count", h, C.byref(ne), C.byref(nm))
        self.n_enc, self.n_mlp = ne.value, nm.value
        self.n_params = self.n_enc + self.n_mlp

    @classmethod
    def _borrowed(cls, handle, lo, hi, ghost, enc, mlp):
        """A view of a model owned by the library (e.g. by a Window): closing
        or collecting it does not free the model."""
        m = cls.__new__(cls)
        m.lo, m.hi, m.ghost = tuple(int(v) for v in lo), tuple(int(v) for v in hi), int(ghost)
        m.enc, m.mlp = enc, mlp
        m._h = handle
        m._owned = False
        ne, nm = C.c_int64(), C.c_int64()
        A.call("dvnr_param_count", handle, C.byref(ne), C.byref(nm))
        m.n_enc, m.n_mlp = ne.value, nm.value
        m.n_params = m.n_enc + m.n_mlp
        return m

    # ------------------------------------------------------------ lifecycle
    def close(self):
        if getattr(self, "_h", None):
            if getattr(self, "_owned", True):
                A.load().dvnr_destroy(self._h)
            self._h = None

    def freeze(self, stream=None):
        """Keep only the FP16 parameters and value range (storage form)."""
        A.call("dvnr_freeze", self._h, _stream(stream))

    def set_value_range(self, vmin: float, vmax: float, stream=None):
        """The range decoding de-normalises with (set by training otherwise)."""
        A.call("dvnr_set_value_range", self._h, float(vmin), float(vmax), _stream(stream))

    def save(self, path, fp16: bool = False):
        """Write a versioned model file: box, configuration, value range and
        the parameters as float32 (resume exactly) or binary16 (the paper's
        16-bit storage)."""
        from . import storage

        st = self.state()
        header = {"box": {"lo": list(self.lo), "hi": list(self.hi), "ghost": self.ghost},
                  "encoding": {"n_levels": self.enc.n_levels, "n_features": self.enc.n_features,
                               "log2_T": self.enc.log2_T, "base_res": self.enc.base_res,
                               "growth": float(self.enc.growth)},
                  "mlp": {"width": self.mlp.width, "n_hidden": self.mlp.n_hidden},
                  "value_range": [float(st["vmin"]), float(st["vmax"])],
                  "payload": "fp16" if fp16 else "fp32", "n_enc": self.n_enc, "n_mlp": self.n_mlp}
        storage.write_model_file(path, header,
                                 self.export_fp16().view(np.uint16) if fp16 else self.get_weights())

    @classmethod
    def load(cls, path, seed: int = 0) -> "Model":
        """A model from a file written by save(): weights (an fp16 file sets
        the FP32 weights to the widened binary16 values) and value range; the
        optimiser state starts fresh."""
        from . import storage

        h, params = storage.read_model_file(path)
        b, e, mm = h["box"], h["encoding"], h["mlp"]
        m = cls(b["lo"], b["hi"], b["ghost"],
                EncodingConfig(e["n_levels"], e["n_features"], e["log2_T"], e["base_res"], e["growth"]),
                MLPConfig(mm["width"], mm["n_hidden"]), seed=seed)
        if (m.n_enc, m.n_mlp) != (int(h["n_enc"]), int(h["n_mlp"])):
            m.close()
            raise ValueError("model file parameter counts do not match its configuration")
        if h["payload"] == "fp16":
            m.import_fp16(params.view(np.float16))
        else:
            m.set_weights(params)
        m.set_value_range(*h["value_range"])
        return m

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    @property
    def stored_dims(self):
        return tuple(h - l + 2 * self.ghost for l, h in zip(self.lo, self.hi))

    @property
    def owned_dims(self):
        return tuple(h - l for l, h in zip(self.lo, self.hi))

    # -------------------------------------------------------------- weights
    def get_weights(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        A.call("dvnr_get_weights", self._h, out.ctypes.data, self.n_params)
        return out

    def set_weights(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        assert w.size == self.n_params
        A.call("dvnr_set_weights", self._h, w.ctypes.data, self.n_params)

    def export_fp16(self) -> np.ndarray:
        """The model as 16-bit floats (compact layout), e.g. for storage."""
        out = np.empty(self.n_params, dtype=np.uint16)
        A.call("dvnr_export_fp16", self._h, out.ctypes.data, self.n_params)
        return out.view(np.float16)

    def import_fp16(self, w16):
        w = np.ascontiguousarray(w16, dtype=np.float16).view(np.uint16)
        assert w.size == self.n_params
        A.call("dvnr_import_fp16", self._h, w.ctypes.data, self.n_params)

    def copy_weights_from(self, src: "Model", stream=None):
        A.call("dvnr_copy_weights", self._h, src._h, _stream(stream))

    def set_precision(self, precision: int, stream=None):
        A.call("dvnr_set_precision", self._h, int(precision), _stream(stream))

    def state(self) -> dict:
        s = A.dvnr_state_info()
        A.call("dvnr_get_state", self._h, C.byref(s))
        return {k: getattr(s, k) for k, _ in A.dvnr_state_info._fields_}

    # ------------------------------------------------------------ training
    def train_grad(self, volume, cfg: TrainConfig, iteration: int = 0, stream=None,
                   want=("grad", "y", "target", "dx0", "coords", "loss")):
        """One step's forward+backward without the optimiser; returns the
        requested device tensors (unscaled gradients)."""
        import torch

        dev = volume.device
        B = cfg.batch
        D = self.enc.n_levels * self.enc.n_features
        shapes = {"grad": (self.n_params,), "y": (B,), "target": (B,), "dx0": (B, D),
                  "coords": (B, 3), "loss": (1,)}
        outs = {}
        for k in want:
            dt = torch.int32 if k == "coords" else torch.float32
            outs[k] = torch.empty(shapes[k], dtype=dt, device=dev)
        so = A.dvnr_step_outputs(*[outs[k].data_ptr() if k in outs else None
                                   for k in ("grad", "y", "target", "dx0", "coords", "loss")])
        c = cfg.to_c()
        A.call("dvnr_train_grad", self._h, _ptr(volume), C.byref(c), int(iteration), C.byref(so),
               _stream(stream))
        return outs

    def adam_step(self, grad, cfg: TrainConfig, stream=None):
        """One Adam step (Sec. 3.6) from a caller-given gradient: a float32
        device tensor of n_params values in the compact layout (unscaled)."""
        import torch

        g = grad.detach().to(torch.float32).contiguous().reshape(-1)
        assert g.numel() == self.n_params and g.is_cuda
        c = cfg.to_c()
        A.call("dvnr_adam_step", self._h, _ptr(g), C.byref(c), _stream(stream))

    def params_tensor(self, device="cuda"):
        """The FP32 master weights as a float32 CUDA tensor (compact layout),
        e.g. as the params argument of EncodeMLP."""
        import torch

        return torch.from_numpy(self.get_weights()).to(device)

    def forward(self, coords, precision=A.DVNR_FP32, stream=None):
        """Network output (normalised units) at fixed-point coordinates (n, 3)."""
        import torch

        coords = coords.contiguous()
        y = torch.empty(coords.shape[0], dtype=torch.float32, device=coords.device)
        A.call("dvnr_forward", self._h, _ptr(coords), coords.shape[0], int(precision), _ptr(y),
               _stream(stream))
        return y

    def backward(self, coords, dy, precision=A.DVNR_FP32, loss_scale=0.0, want_dx0=False, stream=None):
        """(gradient of all parameters (compact), dL/d(encoding) or None) for
        the upstream gradient dy at fixed-point coordinates (n, 3)."""
        import torch

        coords = coords.contiguous()
        d = dy.detach().to(torch.float32).contiguous()
        g = torch.empty(self.n_params, dtype=torch.float32, device=coords.device)
        dx0 = (torch.empty((coords.shape[0], self.enc.n_levels * self.enc.n_features),
                           dtype=torch.float32, device=coords.device) if want_dx0 else None)
        A.call("dvnr_backward", self._h, _ptr(coords), coords.shape[0], _ptr(d), int(precision),
               float(loss_scale), _ptr(g), _ptr(dx0), _stream(stream))
        return g, dx0

    def moments(self):
        """(m1, m2): the Adam moments in the compact layout (host arrays)."""
        m1 = np.empty(self.n_params, dtype=np.float32)
        m2 = np.empty(self.n_params, dtype=np.float32)
        A.call("dvnr_get_moments", self._h, m1.ctypes.data, m2.ctypes.data, self.n_params)
        return m1, m2

    # ------------------------------------------------------------ inference
    def decode_points(self, xyz, stream=None):
        import torch

        xyz = xyz.contiguous()
        out = torch.empty(xyz.shape[0], dtype=torch.float32, device=xyz.device)
        A.call("dvnr_decode_points", self._h, _ptr(xyz), xyz.shape[0], _ptr(out), _stream(stream))
        return out

    def decode_grid(self, out=None, stream=None):
        import torch

        ex, ey, ez = self.owned_dims
        if out is None:
            out = torch.empty((ez, ey, ex), dtype=torch.float32, device="cuda")
        A.call("dvnr_decode_grid", self._h, _ptr(out), _stream(stream))
        return out

    def corner_indices(self, coords, stream=None):
        import torch

        coords = coords.contiguous()
        n = coords.shape[0]
        out = torch.empty((n, self.enc.n_levels, 8), dtype=torch.int32, device=coords.device)
        A.call("dvnr_corner_indices", self._h, _ptr(coords), n, _ptr(out), _stream(stream))
        return out


def _encode_mlp_class():
    import torch

    class EncodeMLP(torch.autograd.Function):
        """y = f(params; coords): the hash-grid encoding and ReLU MLP of a
        model (Sec. 3) as a differentiable function of its parameters, run by
        the library's kernels (dvnr_forward / dvnr_backward).

        apply(params, coords, model, precision=DVNR_FP32, loss_scale=0.0)
          params  float32 CUDA tensor of model.n_params values, the compact
                  layout (tables level by level, then W_0 .. W_{H-1}, w_out);
                  loaded into the model before the forward and again before
                  the backward, so it is the source of truth
          coords  int32/uint32 CUDA tensor (n, 3) of fixed-point coordinates
                  m in [0, 2^24] (u = m 2^-24), not differentiable
          returns y, a float32 tensor (n,) in normalised units.
        The gradient with respect to params comes from the fused training
        kernel with the loss replaced by the incoming dL/dy."""

        @staticmethod
        def forward(ctx, params, coords, model, precision=A.DVNR_FP32, loss_scale=0.0):
            assert params.is_cuda and params.dtype == torch.float32 and params.numel() == model.n_params
            coords = coords.contiguous()
            assert coords.is_cuda and coords.dim() == 2 and coords.shape[1] == 3
            p = params.detach().contiguous()
            stream = _stream(None)
            A.call("dvnr_load_params", model.handle, _ptr(p), stream)
            y = torch.empty(coords.shape[0], dtype=torch.float32, device=coords.device)
            A.call("dvnr_forward", model.handle, _ptr(coords), coords.shape[0], int(precision), _ptr(y),
                   stream)
            ctx.save_for_backward(p, coords)
            ctx.model, ctx.precision, ctx.loss_scale = model, int(precision), float(loss_scale)
            return y

        @staticmethod
        def backward(ctx, dy):
            p, coords = ctx.saved_tensors
            m = ctx.model
            stream = _stream(None)
            A.call("dvnr_load_params", m.handle, _ptr(p), stream)
            g = torch.empty(m.n_params, dtype=torch.float32, device=p.device)
            d = dy.detach().to(torch.float32).contiguous()
            A.call("dvnr_backward", m.handle, _ptr(coords), coords.shape[0], _ptr(d), ctx.precision,
                   ctx.loss_scale, _ptr(g), None, stream)
            return g, None, None, None, None

    return EncodeMLP


_ENCODE_MLP = None


def __getattr__(name):
    # EncodeMLP subclasses a torch class: built on first use, so that importing
    # this module does not import torch
    global _ENCODE_MLP
    if name == "EncodeMLP":
        if _ENCODE_MLP is None:
            _ENCODE_MLP = _encode_mlp_class()
        return _ENCODE_MLP
    raise AttributeError(name)


def train(models, volumes, cfg: TrainConfig, stream=None, sync: bool = True):
    """dvnr_train over ``models`` with their stored-block ``volumes``."""
    n = len(models)
    hs = (C.c_void_p * n)(*[m.handle for m in models])
    vs = (C.c_void_p * n)(*[v.data_ptr() for v in volumes])
    c = cfg.to_c()
    losses = (C.c_float * n)() if sync else None
    A.call("dvnr_train", C.cast(hs, C.c_void_p), n, C.cast(vs, C.c_void_p), C.byref(c),
           _stream(stream), C.cast(losses, C.c_void_p) if sync else None)
    return [float(v) for v in losses] if sync else None


def make_tf(c0=(0.1, 0.2, 0.6), c1=(1.0, 0.9, 0.2), alpha_max=0.05, v_lo=0.0, v_hi=1.0):
    return A.dvnr_tf((C.c_float * 3)(*c0), (C.c_float * 3)(*c1), alpha_max, v_lo, v_hi)


def render(models, tf, w, h, spr, out=None, stream=None):
    import torch

    n = len(models)
    hs = (C.c_void_p * n)(*[m.handle for m in models])
    if out is None:
        out = torch.empty((h, w, 4), dtype=torch.float32, device="cuda")
    A.call("dvnr_render", C.cast(hs, C.c_void_p), n, C.byref(tf), w, h, spr, _ptr(out),
           _stream(stream))
    return out


class Window:
    """Temporal sliding window of trained models (Sec. 4.2): one model per
    partition and time step, the newest step trainable, older steps frozen,
    at most `capacity` steps."""

    def __init__(self, boxes, capacity, encs=None, mlp: MLPConfig | None = None, ghost=1,
                 seed: int = 0):
        self.boxes = [(tuple(lo), tuple(hi)) for lo, hi in boxes]
        n = len(self.boxes)
        if encs is None or isinstance(encs, EncodingConfig):
            encs = [encs or EncodingConfig()] * n
        self.encs, self.mlp, self.ghost = list(encs), mlp or MLPConfig(), int(ghost)
        cb = (A.dvnr_box * n)(*[A.dvnr_box((C.c_int64 * 3)(*lo), (C.c_int64 * 3)(*hi), self.ghost)
                                for lo, hi in self.boxes])
        ce = (A.dvnr_enc_cfg * n)(*[A.dvnr_enc_cfg(e.n_levels, e.n_features, e.log2_T, e.base_res,
                                                   float(e.growth)) for e in self.encs])
        mc = A.dvnr_mlp_cfg(self.mlp.width, self.mlp.n_hidden)
        h = C.c_void_p()
        A.call("dvnr_window_create", C.cast(cb, C.c_void_p), n, C.cast(ce, C.c_void_p),
               C.byref(mc), int(capacity), int(seed), C.byref(h))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            A.load().dvnr_window_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def push(self, volumes, cfg: TrainConfig, stream=None, sync: bool = True):
        n = len(self.boxes)
        vs = (C.c_void_p * n)(*[v.data_ptr() for v in volumes])
        c = cfg.to_c()
        losses = (C.c_float * n)() if sync else None
        t = C.c_int64()
        A.call("dvnr_window_push", self._h, C.cast(vs, C.c_void_p), C.byref(c), _stream(stream),
               C.cast(losses, C.c_void_p) if sync else None, C.byref(t))
        return t.value, ([float(v) for v in losses] if sync else None)

    def range(self):
        a, b = C.c_int64(), C.c_int64()
        A.call("dvnr_window_range", self._h, C.byref(a), C.byref(b))
        return a.value, b.value

    def model(self, t: int, part: int = 0) -> Model:
        h = C.c_void_p()
        A.call("dvnr_window_model", self._h, int(t), int(part), C.byref(h))
        lo, hi = self.boxes[part]
        return Model._borrowed(h, lo, hi, self.ghost, self.encs[part], self.mlp)

    def bytes(self):
        a, b = C.c_int64(), C.c_int64()
        A.call("dvnr_window_bytes", self._h, C.byref(a), C.byref(b))
        return a.value, b.value


def render_inr(models, tf, w, h, spr, out=None, stream=None):
    """Ray-march the networks directly (no decoded grids); same image
    conventions as `render`."""
    import torch

    n = len(models)
    hs = (C.c_void_p * n)(*[m.handle for m in models])
    if out is None:
        out = torch.empty((h, w, 4), dtype=torch.float32, device="cuda")
    A.call("dvnr_render_inr", C.cast(hs, C.c_void_p), n, C.byref(tf), w, h, spr, _ptr(out),
           _stream(stream))
    return out


def render_in_frame(models, frame_lo, frame_hi, tf, w, h, spr, from_network=False, out=None,
                    stream=None):
    """Render `models` with the camera spanning [frame_lo, frame_hi) (the
    global domain): images of disjoint partitions rendered apart composite
    into the image of all of them."""
    import torch

    n = len(models)
    hs = (C.c_void_p * n)(*[m.handle for m in models])
    if out is None:
        out = torch.empty((h, w, 4), dtype=torch.float32, device="cuda")
    lo = (C.c_int64 * 3)(*[int(v) for v in frame_lo])
    hi = (C.c_int64 * 3)(*[int(v) for v in frame_hi])
    A.call("dvnr_render_in_frame", C.cast(hs, C.c_void_p), n, lo, hi, C.byref(tf), w, h, spr,
           1 if from_network else 0, _ptr(out), _stream(stream))
    return out


def composite(images, depths, out=None, stream=None):
    """Sort-last blend of premultiplied RGBA images (h, w, 4) in increasing
    depth (front first)."""
    import torch

    n = len(images)
    h, w = images[0].shape[0], images[0].shape[1]
    imgs = [im.contiguous() for im in images]
    ptrs = (C.c_void_p * n)(*[im.data_ptr() for im in imgs])
    dep = (C.c_double * n)(*[float(d) for d in depths])
    if out is None:
        out = torch.empty((h, w, 4), dtype=torch.float32, device=imgs[0].device)
    A.call("dvnr_composite", C.cast(ptrs, C.c_void_p), C.cast(dep, C.c_void_p), n, w, h, _ptr(out),
           _stream(stream))
    return out


def error_stats(a, b, stream=None):
    """(sum of squared differences, max abs difference) in FP64 on the device."""
    out = (C.c_double * 2)()
    A.call("dvnr_error_stats", _ptr(a.contiguous()), _ptr(b.contiguous()), a.numel(),
           C.cast(out, C.c_void_p), _stream(stream))
    return out[0], out[1]
