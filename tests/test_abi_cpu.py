"""Host-side tests of the C ABI (no GPU): the library builds for sm_103a,
loads, exports every entry point include/dvnr.h declares, its struct layouts
agree with the ctypes binding, and host argument checks reject bad input
before any device work."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2304_10516_gb300 import _abi as A

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dvnr.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dvnr_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = A.load()
    declared = _declared()
    assert len(declared) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", A.lib_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (dvnr_\w+)", out))
    missing = [d for d in declared if d not in exported]
    assert not missing, missing
    assert set(declared) == set(A.EXPORTS)
    for name in declared:
        assert hasattr(lib, name)
    assert lib.dvnr_abi_version() == 1


def test_struct_layouts_match_binding(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "dvnr.h"
#define S(t) printf(#t " %zu\\n", sizeof(t));
#define O(t, f) printf(#t "." #f " %zu\\n", offsetof(t, f));
int main(void) {
  S(dvnr_box) S(dvnr_enc_cfg) S(dvnr_mlp_cfg) S(dvnr_train_cfg) S(dvnr_state_info)
  S(dvnr_tf) S(dvnr_step_outputs)
  O(dvnr_box, ghost) O(dvnr_enc_cfg, growth) O(dvnr_train_cfg, steps) O(dvnr_train_cfg, seed)
  O(dvnr_train_cfg, growth_interval) O(dvnr_state_info, precision) O(dvnr_tf, v_hi)
  O(dvnr_step_outputs, loss)
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(ln.rsplit(" ", 1) for ln in lines if ln.strip())
    for name in ["dvnr_box", "dvnr_enc_cfg", "dvnr_mlp_cfg", "dvnr_train_cfg", "dvnr_state_info",
                 "dvnr_tf", "dvnr_step_outputs"]:
        assert int(got[name]) == C.sizeof(getattr(A, name)), name
    for key, val in got.items():
        if "." in key:
            t, f = key.split(".")
            assert getattr(getattr(A, t), f).offset == int(val), key


def _enc(**kw):
    d = dict(n_levels=8, n_features=2, log2_T=15, base_res=4, growth=1.5)
    d.update(kw)
    return A.dvnr_enc_cfg(d["n_levels"], d["n_features"], d["log2_T"], d["base_res"], d["growth"])


def _box(lo=(0, 0, 0), hi=(8, 8, 8), ghost=0):
    return A.dvnr_box((C.c_int64 * 3)(*lo), (C.c_int64 * 3)(*hi), ghost)


@pytest.mark.parametrize("bad", [
    dict(box=_box(hi=(0, 8, 8))),                 # empty box
    dict(box=_box(lo=(0, 0, 0), hi=(1, 1, 1))),   # one stored voxel per axis
    dict(box=_box(ghost=-1)),
    dict(enc=_enc(n_levels=0)),
    dict(enc=_enc(n_levels=33)),
    dict(enc=_enc(n_features=3)),
    dict(enc=_enc(log2_T=3)),
    dict(enc=_enc(log2_T=25)),
    dict(enc=_enc(base_res=0)),
    dict(enc=_enc(growth=0.5)),
    dict(enc=_enc(growth=float("nan"))),
    dict(mlp=A.dvnr_mlp_cfg(32, 0)),
    dict(mlp=A.dvnr_mlp_cfg(32, 9)),
])
def test_create_rejects_bad_arguments_on_host(bad):
    lib = A.load()
    box = bad.get("box", _box())
    enc = bad.get("enc", _enc())
    mlp = bad.get("mlp", A.dvnr_mlp_cfg(32, 2))
    h = C.c_void_p()
    rc = lib.dvnr_create(C.byref(box), C.byref(enc), C.byref(mlp), 0, C.byref(h))
    assert rc == 1  # DVNR_E_INVALID
    assert h.value is None
    assert lib.dvnr_last_error()


def test_unsupported_width_is_reported():
    lib = A.load()
    h = C.c_void_p()
    mlp = A.dvnr_mlp_cfg(48, 2)
    rc = lib.dvnr_create(C.byref(_box()), C.byref(_enc()), C.byref(mlp), 0, C.byref(h))
    assert rc == 7  # DVNR_E_UNSUPPORTED


def test_null_arguments_rejected():
    lib = A.load()
    assert lib.dvnr_create(None, None, None, 0, None) == 1
    assert lib.dvnr_train(None, 0, None, None, None, None) == 1
    assert lib.dvnr_render(None, 0, None, 1, 1, 1, None, None) == 1
    assert lib.dvnr_param_count(None, None, None) == 1
    lib.dvnr_destroy(None)  # ignored


def test_python_package_has_no_cpu_fallback():
    # the model module routes every call through libdvnr; no import of the
    # oracle, numpy math or torch ops stands in for a kernel
    src = open(os.path.join(ROOT, "paper_2304_10516_gb300", "model.py")).read()
    assert "oracle" not in src
    assert "import torch.nn" not in src


def test_adaptive_encoding_matches_oracle(orc):
    # host arithmetic of the library (no device work) against the oracle
    from paper_2304_10516_gb300 import model as dv

    rng = np.random.default_rng(11)
    cases = [(512 ** 3, 512 ** 3), (256 ** 3, 512 ** 3), (96 * 130 * 150, 512 ** 3),
             (2 ** 27 + 1, 2 ** 30), (1, 10 ** 9)]
    cases += [(int(v), int(g)) for g, v in
              ((g, rng.integers(1, g + 1)) for g in rng.integers(10 ** 6, 10 ** 10, 100))]
    for n_vox, n_glob in cases:
        for lref, lmin, rref in ((19, 12, 16.0), (17, 10, 20.0), (22, 14, 7.5)):
            e = dv.adaptive_encoding(n_vox, n_glob, lref, lmin, rref)
            assert (e.log2_T, e.base_res) == orc.adaptive_encoding(n_vox, n_glob, lref, lmin, rref), \
                (n_vox, n_glob, lref, lmin, rref)
    with pytest.raises(A.DvnrError):
        dv.adaptive_encoding(10, 5)


def test_null_arguments_rejected_by_newer_entry_points():
    lib = A.load()
    assert lib.dvnr_render_inr(None, 0, None, 1, 1, 1, None, None) == 1
    assert lib.dvnr_render_in_frame(None, 0, None, None, None, 1, 1, 1, 0, None, None) == 1
    assert lib.dvnr_composite(None, None, 0, 1, 1, None, None) == 1
    assert lib.dvnr_freeze(None, None) == 1
    assert lib.dvnr_set_value_range(None, 0.0, 1.0, None) == 1
    assert lib.dvnr_export_fp16(None, None, 0) == 1
    assert lib.dvnr_import_fp16(None, None, 0) == 1
    h = C.c_void_p()
    assert lib.dvnr_window_create(None, 1, None, None, 2, 0, C.byref(h)) == 1 and h.value is None
    box = (A.dvnr_box * 1)(_box())
    enc = (A.dvnr_enc_cfg * 1)(_enc())
    mlp = A.dvnr_mlp_cfg(32, 2)
    assert lib.dvnr_window_create(C.cast(box, C.c_void_p), 1, C.cast(enc, C.c_void_p), C.byref(mlp), 0, 0,
                                  C.byref(h)) == 1  # capacity 0
    assert lib.dvnr_window_push(None, None, None, None, None, None) == 1
    assert lib.dvnr_window_range(None, None, None) == 1
    assert lib.dvnr_window_model(None, 0, 0, None) == 1
    assert lib.dvnr_window_bytes(None, None, None) == 1
    lib.dvnr_window_destroy(None)  # ignored
    assert lib.dvnr_adaptive_encoding(5, 10, 19, 12, 16.0, None) == 1


@pytest.mark.parametrize("field,value", [("stop_decay", 1.0), ("stop_decay", -0.1), ("stop_loss", -1.0),
                                         ("stop_loss", float("inf")), ("epochs", -1), ("min_steps", -3),
                                         ("steps", -1), ("batch", 0)])
def test_train_config_checked_on_host(field, value):
    # the call fails on the configuration before it looks at any model
    from paper_2304_10516_gb300 import model as dv

    lib = A.load()
    cfg = dv.TrainConfig()
    setattr(cfg, field, value)
    c = cfg.to_c()
    hs = (C.c_void_p * 1)()
    vs = (C.c_void_p * 1)()
    rc = lib.dvnr_train(C.cast(hs, C.c_void_p), 1, C.cast(vs, C.c_void_p), C.byref(c), None, None)
    assert rc == 1, (field, value)
    assert lib.dvnr_last_error()
