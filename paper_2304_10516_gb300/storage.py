"""Versioned model files (checkpoint / resume of trained partition models;
the paper keeps trained models for later visualisation, Sec. 4.2, and stores
weights as 16-bit floats, Sec. 3.4).

Layout: 8-byte magic b"DVNRMODL", a little-endian uint32 header length, a
UTF-8 JSON header, then the n_enc + n_mlp parameters in the compact layout of
dvnr_get_weights, little-endian float32 ("fp32") or IEEE binary16 bit
patterns ("fp16"). The header holds the format version, the partition box,
the encoding and MLP configuration, the value range and the payload type and
counts. Pure host code: reading and writing need no GPU.
"""
from __future__ import annotations

import json
import struct

import numpy as np

MAGIC = b"DVNRMODL"
VERSION = 1


def write_model_file(path, header: dict, params: np.ndarray) -> None:
    h = dict(header, version=VERSION)
    if h.get("payload") == "fp16":
        params = np.asarray(params)
        if params.dtype != np.uint16:
            raise ValueError("an fp16 payload is passed as binary16 bit patterns (uint16)")
        data = np.ascontiguousarray(params, dtype="<u2")
    elif h.get("payload") == "fp32":
        data = np.ascontiguousarray(params, dtype="<f4")
    else:
        raise ValueError("payload must be 'fp16' or 'fp32'")
    if data.size != int(h["n_enc"]) + int(h["n_mlp"]):
        raise ValueError("parameter count does not match n_enc + n_mlp")
    hb = json.dumps(h, sort_keys=True).encode("utf-8")
    with open(path, "wb") as f:
        f.write(MAGIC)
        f.write(struct.pack("<I", len(hb)))
        f.write(hb)
        f.write(data.tobytes())


def read_model_file(path) -> tuple[dict, np.ndarray]:
    """(header, params): params as float32 or uint16 (binary16 bits)."""
    with open(path, "rb") as f:
        blob = f.read()
    if len(blob) < 12 or blob[:8] != MAGIC:
        raise ValueError("not a model file (bad magic)")
    (hl,) = struct.unpack("<I", blob[8:12])
    if 12 + hl > len(blob):
        raise ValueError("truncated model file (header)")
    try:
        h = json.loads(blob[12:12 + hl].decode("utf-8"))
    except ValueError as e:
        raise ValueError(f"unreadable model file header: {e}") from None
    if h.get("version") != VERSION:
        raise ValueError(f"model file version {h.get('version')} (this library reads {VERSION})")
    for k in ("box", "encoding", "mlp", "value_range", "payload", "n_enc", "n_mlp"):
        if k not in h:
            raise ValueError(f"model file header lacks '{k}'")
    n = int(h["n_enc"]) + int(h["n_mlp"])
    dt = {"fp16": "<u2", "fp32": "<f4"}.get(h["payload"])
    if dt is None:
        raise ValueError(f"unknown payload '{h['payload']}'")
    body = blob[12 + hl:]
    if len(body) != n * np.dtype(dt).itemsize:
        raise ValueError(f"model file holds {len(body)} payload bytes, expected {n * np.dtype(dt).itemsize}")
    params = np.frombuffer(body, dtype=dt).copy()
    return h, params.astype(np.float32) if dt == "<f4" else params.astype(np.uint16)
