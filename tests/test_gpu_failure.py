"""Failure handling on the GPU, made to happen without faulting anything.

Every tensor-core wait in the FP16 kernels is bounded; when one runs out the
CTA lets its product finish, frees its tensor memory and returns, the step is
skipped by Adam and the call reports DVNR_E_TIMEOUT. The tests lower the limit
of each CTA's first wait to zero (dvnr_debug_first_wait), so that wait runs
out while its product is still in flight, then restore the default and check
that the model trains and decodes as before.

Also: a model created after another one of a grouped call was destroyed gets
its own training (the grouped-call cache compares model ids, not handle
addresses, which the allocator may hand out again).
"""
import ctypes as C

import numpy as np
import pytest

import parity as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TIMEOUT = 5


@pytest.fixture(scope="module")
def dv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_10516_gb300 import model as dv

    return dv


@pytest.fixture(scope="module")
def A():
    from paper_2304_10516_gb300 import _abi as A

    return A


@pytest.fixture
def short_first_wait(A):
    prev = C.c_int64()
    A.call("dvnr_debug_first_wait", 0, C.byref(prev))
    try:
        yield
    finally:
        A.call("dvnr_debug_first_wait", -1, None)
    assert prev.value > 0


def _state(A, m):
    """(status, state dict) of dvnr_get_state without raising."""
    s = A.dvnr_state_info()
    rc = A.load().dvnr_get_state(m.handle, C.byref(s))
    return rc, {k: getattr(s, k) for k, _ in A.dvnr_state_info._fields_}


def _models(dv, n, seed=40):
    c = P.configs_blobs64()
    enc = dv.EncodingConfig(c["L"], c["F"], c["log2T"], c["base"], c["growth"])
    mlp = dv.MLPConfig(c["width"], c["hidden"])
    return c, [dv.Model((0, 0, 0), (64, 64, 64), 0, enc, mlp, seed=seed + i) for i in range(n)]


def _vol(seed=1001):
    from paper_2304_10516_gb300 import volumes

    return torch.from_numpy(volumes.blobs(64, seed=seed)).cuda()


def _psnr(dv, m, vol):
    sse, _ = dv.error_stats(m.decode_grid(), vol)
    return P.psnr(sse / vol.numel())


def test_training_wait_that_runs_out_skips_the_step(dv, A, short_first_wait):
    c, (a, b) = _models(dv, 2)
    vols = [_vol(1001), _vol(1011)]
    cfg = dv.TrainConfig(batch=c["batch"], steps=1, precision=A.DVNR_FP16, seed=3)
    w0 = [a.get_weights(), b.get_weights()]
    with pytest.raises(A.DvnrError) as ei:
        dv.train([a, b], vols, cfg)
    assert ei.value.status == TIMEOUT
    for m, w in zip((a, b), w0):
        rc, s = _state(A, m)
        assert rc == TIMEOUT
        assert s["adam_t"] == 0 and s["skipped"] == 1 and s["iter"] == 1
        assert s["loss_scale"] == 2.0 ** 12  # an aborted step does not halve the scale
        np.testing.assert_array_equal(m.get_weights(), w)  # parameters untouched
    for m in (a, b):
        m.close()


def test_training_recovers_after_a_timeout(dv, A):
    c, (a, ref) = _models(dv, 2, seed=50)
    ref.set_weights(a.get_weights())
    vol = _vol()
    # lr 5e-4: a stable regime, where a shift of the sample stream by one
    # iteration moves the 200-step PSNR little (at 1e-2 training is chaotic)
    cfg = dv.TrainConfig(batch=c["batch"], steps=1, lr=5e-4, precision=A.DVNR_FP16, seed=3)
    p0 = _psnr(dv, a, vol)
    A.call("dvnr_debug_first_wait", 0, None)
    try:
        with pytest.raises(A.DvnrError):
            dv.train([a], [vol], cfg)
    finally:
        A.call("dvnr_debug_first_wait", -1, None)
    # the next call, at the normal limit, trains: its graph-replayed steps
    # reach the PSNR of a model that never timed out (same initial weights;
    # its sample stream is one iteration ahead)
    cfg.steps = 200
    dv.train([a], [vol], cfg)
    dv.train([ref], [vol], cfg)
    rc, s = _state(A, a)
    assert rc == 0
    assert s["adam_t"] == 200 and s["skipped"] == 1 and s["iter"] == 201
    pa, pr = _psnr(dv, a, vol), _psnr(dv, ref, vol)
    assert abs(pa - pr) < 0.2, (pa, pr)
    assert pa > p0 + 10.0
    a.close()
    ref.close()


def test_decode_wait_that_runs_out_reports_timeout(dv, A):
    c, (m,) = _models(dv, 1, seed=60)
    vol = _vol()
    dv.train([m], [vol], dv.TrainConfig(batch=c["batch"], steps=20, precision=A.DVNR_FP16, seed=3))
    good = m.decode_grid().clone()
    A.call("dvnr_debug_first_wait", 0, None)
    try:
        m.decode_grid()
        torch.cuda.synchronize()
    finally:
        A.call("dvnr_debug_first_wait", -1, None)
    rc, _ = _state(A, m)
    assert rc == TIMEOUT
    # at the normal limit the decoder gives the same grid as before
    again = m.decode_grid()
    torch.cuda.synchronize()
    assert torch.equal(again, good)
    # the timeout count restarts with the next training call
    dv.train([m], [vol], dv.TrainConfig(batch=c["batch"], steps=1, precision=A.DVNR_FP16, seed=3))
    assert _state(A, m)[0] == 0
    m.close()


def test_grouped_call_after_a_model_is_replaced(dv, A):
    c, (a, b) = _models(dv, 2, seed=70)
    vols = [_vol(1001), _vol(1011)]
    cfg = dv.TrainConfig(batch=c["batch"], steps=2, precision=A.DVNR_FP16, seed=3)
    dv.train([a, b], vols, cfg)
    b.close()
    # a new model, possibly at the destroyed model's handle address
    _, (n,) = _models(dv, 1, seed=71)
    w_n = n.get_weights()
    dv.train([a, n], vols, cfg)
    assert a.state()["adam_t"] == 4
    assert n.state()["adam_t"] == 2
    assert not np.array_equal(n.get_weights(), w_n)
    a.close()
    n.close()


def _live(A):
    c, b = C.c_int64(), C.c_int64()
    A.call("dvnr_debug_live_allocs", C.byref(c), C.byref(b))
    return c.value, b.value


def _scenario_models(dv, A):
    """Model lifecycle through every call that allocates device memory:
    creation, a grouped FP16 call (descriptor cache and step graphs), decode,
    grid and network rendering, compositing, the FP64 error reduction, a
    backward at given points, freezing, and the FP32 path's workspaces."""
    enc = dv.EncodingConfig(4, 2, 10, 4, 1.5)
    mlp = dv.MLPConfig(16, 2)
    vol = _vol()[:18, :18, :18].contiguous()
    models = []
    try:
        for lo in ((0, 0, 0), (0, 0, 16)):
            models.append(dv.Model(lo, (16, 16, lo[2] + 16), 1, enc, mlp, seed=3))
        a, b = models
        dv.train([a, b], [vol, vol], dv.TrainConfig(batch=1000, steps=9, precision=A.DVNR_FP16, seed=1))
        g = a.decode_grid()
        tf = dv.make_tf()
        img = dv.render([a, b], tf, 24, 24, 16)
        img2 = dv.render_inr([a, b], tf, 24, 24, 16)
        dv.composite([img, img2], [0.0, 1.0])
        dv.error_stats(g, vol[1:-1, 1:-1, 1:-1].contiguous())
        coords = torch.randint(0, 1 << 24, (300, 3), dtype=torch.int32, device="cuda")
        b.backward(coords, torch.ones(300, device="cuda") / 300, A.DVNR_FP16)
        a.freeze()
        a.decode_grid()
        dv.train([b], [vol], dv.TrainConfig(batch=500, steps=2, precision=A.DVNR_FP32, seed=1))
        b.decode_points(torch.rand(100, 3, device="cuda") * 16)
        dv.render_inr([b], tf, 24, 24, 16)
        b.backward(coords, torch.ones(300, device="cuda") / 300, A.DVNR_FP32)
    finally:
        for m in models:
            m.close()


def _scenario_window(dv, A):
    """A temporal window of two partitions pushed three times into a window
    of two steps: model creation, warm starts, training, freezing, eviction."""
    enc = dv.EncodingConfig(4, 2, 10, 4, 1.5)
    vol = _vol()[:18, :18, :18].contiguous()
    w = dv.Window([((0, 0, 0), (16, 16, 16)), ((0, 0, 16), (16, 16, 32))], 2, enc, dv.MLPConfig(16, 2),
                  ghost=1, seed=5)
    try:
        for _ in range(3):
            w.push([vol, vol], dv.TrainConfig(batch=600, steps=3, precision=A.DVNR_FP16, seed=2))
    finally:
        w.close()


@pytest.mark.parametrize("scenario", [_scenario_models, _scenario_window])
def test_failed_allocations_release_everything(dv, A, scenario):
    # the nth device allocation fails, for n = 1, 2, ... until the scenario
    # runs through: every failure is reported as DVNR_E_OOM and, once the
    # scenario's objects are closed, the library holds no more device memory
    # than before
    scenario(dv, A)  # once without failures (compiles, autotunes)
    torch.cuda.synchronize()
    base = _live(A)
    failures = 0
    for n in range(1, 400):
        A.call("dvnr_debug_fail_alloc", n)
        try:
            scenario(dv, A)
            done = True
        except A.DvnrError as e:
            assert e.status == 2, (n, str(e))  # DVNR_E_OOM
            done = False
            failures += 1
        finally:
            A.call("dvnr_debug_fail_alloc", 0)
        torch.cuda.synchronize()
        assert _live(A) == base, (scenario.__name__, n, _live(A), base)
        if done:
            break
    else:
        pytest.fail("the scenario never ran through")
    assert failures >= 5  # the scenario allocates, and each allocation was made to fail once
