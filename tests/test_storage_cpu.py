"""Versioned model files (paper_2304_10516_gb300.storage): the format round
trip, bit for bit, and rejection of damaged or foreign files. Host only."""
import json
import struct

import numpy as np
import pytest

from paper_2304_10516_gb300 import storage as S

HDR = {"box": {"lo": [0, 0, 0], "hi": [8, 9, 10], "ghost": 1},
       "encoding": {"n_levels": 5, "n_features": 4, "log2_T": 12, "base_res": 16, "growth": 2.0},
       "mlp": {"width": 16, "n_hidden": 3}, "value_range": [-0.25, 3.5]}


def _params(n, fp16):
    rng = np.random.default_rng(3)
    x = rng.standard_normal(n).astype(np.float32)
    x[:4] = [0.0, -0.0, np.inf, 1e-30]
    return x.astype(np.float16).view(np.uint16) if fp16 else x


@pytest.mark.parametrize("fp16", [False, True])
def test_round_trip_is_bit_exact(tmp_path, fp16):
    p = _params(1000, fp16)
    h = dict(HDR, payload="fp16" if fp16 else "fp32", n_enc=900, n_mlp=100)
    f = tmp_path / "m.dvnr"
    S.write_model_file(f, h, p)
    h2, p2 = S.read_model_file(f)
    assert h2["version"] == S.VERSION and h2["box"] == HDR["box"] and h2["value_range"] == [-0.25, 3.5]
    assert p2.dtype == (np.uint16 if fp16 else np.float32)
    np.testing.assert_array_equal(p2.view(np.uint16 if fp16 else np.uint32),
                                  p.view(np.uint16 if fp16 else np.uint32))
    # the file is the magic, the header length, the header, then exactly the payload
    blob = f.read_bytes()
    (hl,) = struct.unpack("<I", blob[8:12])
    assert blob[:8] == b"DVNRMODL" and len(blob) == 12 + hl + p.size * (2 if fp16 else 4)


def test_damaged_and_foreign_files_are_rejected(tmp_path):
    p = _params(100, False)
    h = dict(HDR, payload="fp32", n_enc=90, n_mlp=10)
    f = tmp_path / "m.dvnr"
    S.write_model_file(f, h, p)
    good = f.read_bytes()
    cases = {
        "magic": b"XXXXXXXX" + good[8:],
        "truncated payload": good[:-4],
        "extra payload": good + b"\0\0\0\0",
        "truncated header": good[:20],
    }
    (hl,) = struct.unpack("<I", good[8:12])
    hdr = json.loads(good[12:12 + hl])
    for k, v in (("version", 99), ("payload", "bf16")):
        bad = dict(hdr, **{k: v})
        hb = json.dumps(bad).encode()
        cases[k] = good[:8] + struct.pack("<I", len(hb)) + hb + good[12 + hl:]
    missing = {k: v for k, v in hdr.items() if k != "value_range"}
    hb = json.dumps(missing).encode()
    cases["missing key"] = good[:8] + struct.pack("<I", len(hb)) + hb + good[12 + hl:]
    for name, blob in cases.items():
        g = tmp_path / f"bad_{name.replace(' ', '_')}.dvnr"
        g.write_bytes(blob)
        with pytest.raises(ValueError):
            S.read_model_file(g)


def test_writer_checks_its_arguments(tmp_path):
    with pytest.raises(ValueError):
        S.write_model_file(tmp_path / "a", dict(HDR, payload="fp32", n_enc=5, n_mlp=5), np.zeros(9, np.float32))
    with pytest.raises(ValueError):
        S.write_model_file(tmp_path / "b", dict(HDR, payload="fp16", n_enc=5, n_mlp=5), np.zeros(10, np.float16))
    with pytest.raises(ValueError):
        S.write_model_file(tmp_path / "c", dict(HDR, payload="int8", n_enc=5, n_mlp=5), np.zeros(10, np.float32))
