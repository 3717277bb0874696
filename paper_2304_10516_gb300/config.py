"""Network configurations in the keys of the paper's appendix (the scaling
and in situ experiment listings): lrate, lrate_decay, epochs, n_neurons,
n_hidden_layers, n_levels, n_features_per_level, per_level_scale,
base_resolution, log2_hashmap_size (one value, or a [min, max] range for
per-partition table sizes), target_loss. PaperConfig maps them onto the
library's EncodingConfig, MLPConfig and TrainConfig; weight compression keys
(zfp_mlp, zfp_enc) are accepted and not used (model compression is not part
of this library).
"""
from __future__ import annotations

from dataclasses import dataclass, field

from . import model as M

_KEYS = {"lrate", "lrate_decay", "epochs", "n_neurons", "n_hidden_layers", "n_levels",
         "n_features_per_level", "per_level_scale", "base_resolution", "log2_hashmap_size",
         "target_loss"}
_IGNORED = {"zfp_mlp", "zfp_enc"}


def icbrt(n: int) -> int:
    """Largest r with r^3 <= n (the appendix's base resolution (int)cbrt(T),
    in exact integer arithmetic)."""
    if n < 0:
        raise ValueError("n must be >= 0")
    r = int(round(n ** (1.0 / 3.0)))
    while r * r * r > n:
        r -= 1
    while (r + 1) ** 3 <= n:
        r += 1
    return r


@dataclass
class PaperConfig:
    lrate: float = 1e-2
    lrate_decay: float = -1.0
    epochs: int = 0
    n_neurons: int = 64
    n_hidden_layers: int = 3
    n_levels: int = 16
    n_features_per_level: int = 2
    per_level_scale: float = 2.0
    # an int, or None for (int)cbrt(2^log2_hashmap_size) of each partition's table
    base_resolution: int | None = None
    # one value, or (min, max): a partition's table scales with its share of
    # the domain between 2^min and 2^max (Sec. 3.2)
    log2_hashmap_size: int | tuple = 19
    target_loss: float = 0.0
    ignored: dict = field(default_factory=dict)

    @classmethod
    def from_dict(cls, d: dict) -> "PaperConfig":
        unknown = set(d) - _KEYS - _IGNORED
        if unknown:
            raise ValueError(f"unknown configuration keys {sorted(unknown)}")
        kw = {k: d[k] for k in _KEYS if k in d}
        if "log2_hashmap_size" in kw and isinstance(kw["log2_hashmap_size"], (list, tuple)):
            lo, hi = kw["log2_hashmap_size"]
            if not lo <= hi:
                raise ValueError("log2_hashmap_size range needs min <= max")
            kw["log2_hashmap_size"] = (int(lo), int(hi))
        cfg = cls(**kw, ignored={k: d[k] for k in _IGNORED if k in d})
        if cfg.lrate_decay != -1:
            raise ValueError("only a constant learning rate (lrate_decay -1) is supported")
        return cfg

    def encoding(self, n_vox: int | None = None, n_vox_global: int | None = None) -> M.EncodingConfig:
        """The encoding of a partition holding n_vox of the domain's
        n_vox_global voxels (both needed when log2_hashmap_size is a range)."""
        if isinstance(self.log2_hashmap_size, tuple):
            if n_vox is None or n_vox_global is None:
                raise ValueError("a table-size range needs the partition's and the domain's voxel counts")
            lo, hi = self.log2_hashmap_size
            base = M.EncodingConfig(self.n_levels, self.n_features_per_level, hi, 16,
                                    float(self.per_level_scale))
            enc = M.adaptive_encoding(n_vox, n_vox_global, log2_T_ref=hi, log2_T_min=lo,
                                      R_ref=float(icbrt(1 << hi)), base=base)
            log2_T = min(enc.log2_T, hi)
        else:
            log2_T = int(self.log2_hashmap_size)
        R0 = self.base_resolution if self.base_resolution is not None else icbrt(1 << log2_T)
        return M.EncodingConfig(self.n_levels, self.n_features_per_level, log2_T, int(R0),
                                float(self.per_level_scale))

    def mlp(self) -> M.MLPConfig:
        return M.MLPConfig(self.n_neurons, self.n_hidden_layers)

    def train(self, batch: int, **kw) -> M.TrainConfig:
        """Training settings: lrate, the epoch budget ceil(N_vox / batch) x
        epochs (Sec. 3.2) and target_loss as the moving-average stop."""
        return M.TrainConfig(batch=batch, lr=self.lrate, epochs=self.epochs, stop_loss=self.target_loss,
                             **kw)
