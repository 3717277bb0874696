"""The fused Adam kernel element by element against the oracle's Adam step.

Sec. 3.6: Adam with beta1 0.9, beta2 0.999, eps 1e-8 and L2 weight decay
added to the gradient of every parameter; Kingma & Ba bias correction; FP32
master weights and moments, an FP16 copy for the tensor-core path and dynamic
loss scaling there. dvnr_adam_step feeds the library's own optimiser kernel a
gradient chosen by the test, so a step is compared with orc_adam on identical
inputs: the FP32 weights, both moments and a gradient of FP32 values.

Tolerances (FP32 arithmetic against FP64): each moment and each new weight
within about eight FP32 roundings (1e-6 relative) of the terms it is made of
(see _compare); the FP16 copy bit-exact to binary16 rounding of the FP32
master weight.
"""
import numpy as np
import pytest

import parity as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def f32(v):
    return float(np.float32(v))


def _setup(dv, orc, seed):
    c = P.configs_blobs64()
    oc = P.oracle_cfg(c)
    m = dv.Model((0, 0, 0), (64, 64, 64), 0, dv.EncodingConfig(c["L"], c["F"], c["log2T"], c["base"], c["growth"]),
                 dv.MLPConfig(c["width"], c["hidden"]), seed=seed)
    th = P.random_theta(oc, seed, table_scale=0.3)
    m.set_weights(th)
    return c, oc, m, th


def _grad(rng, n, scale):
    g = (rng.standard_normal(n) * scale).astype(np.float32)
    g[rng.random(n) < 0.3] = 0.0  # entries no sample touched: only the decay moves them
    return g


def _compare(m, prev, g, th, m1, m2, t, hp):
    """GPU state after Adam step t against the oracle's (th, m1, m2), which
    started from the same FP32 values `prev` = (theta, m1, m2). The kernel
    works in FP32, so each result is compared within a few FP32 roundings of
    the terms it is made of (the decayed gradient g + wd theta can cancel, so
    a bound relative to the result itself would not hold):
      m1: beta1 |m1'| + (1 - beta1) (|g| + wd |theta'|)
      m2: twice that with the squares
      theta: |theta'| + |step|, plus the step's response to the moments'
             errors through m^ / (sqrt(v^) + eps)."""
    b1, b2, lr, eps, wd = hp
    th_p, m1_p, m2_p = prev
    got = m.get_weights().astype(np.float64)
    g1, g2 = (a.astype(np.float64) for a in m.moments())
    u = 1e-6  # about eight units in the last place of FP32
    a = np.abs(g) + wd * np.abs(th_p)
    tol1 = u * (b1 * np.abs(m1_p) + (1 - b1) * a)
    tol2 = 2 * u * (b2 * np.abs(m2_p) + (1 - b2) * a * a)
    bc1, bc2 = 1 - b1 ** t, 1 - b2 ** t
    mh, vh = m1 / bc1, m2 / bc2
    rv = np.maximum(np.sqrt(vh), 1e-300)
    den = rv + eps
    step = lr * mh / den
    # the step's own rounding and that of the bias corrections (a few ulps
    # each) are inside u |step|
    tol_th = u * (np.abs(th_p) + 2 * np.abs(step)) + lr * (tol1 / bc1 / den + np.abs(mh) * (tol2 / bc2) / (2 * rv * den * den))

    def check(x, want, tol, what):
        err = np.abs(x - want)
        k = int(np.argmax(err / (tol + 1e-300)))
        assert np.all(err <= tol), f"{what}[{k}]: {x[k]!r} vs {want[k]!r} (tolerance {tol[k]:.3e})"

    check(g1, m1, tol1, "m1")
    check(g2, m2, tol2, "m2")
    check(got, th, tol_th, "theta")
    # the FP16 copy the tensor-core kernels read is binary16 of the new master
    w16 = m.export_fp16()
    np.testing.assert_array_equal(w16.view(np.uint16), got.astype(np.float32).astype(np.float16).view(np.uint16))


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_adam_step_matches_oracle(dv, orc, A, prec):
    precision = A.DVNR_FP16 if prec == "fp16" else A.DVNR_FP32
    c, oc, m, th0 = _setup(dv, orc, 21)
    lr, b1, b2, eps, wd = 1e-2, 0.9, 0.999, 1e-8, 0.05  # decay large enough to see
    cfg = dv.TrainConfig(batch=c["batch"], lr=lr, beta1=b1, beta2=b2, eps=eps, weight_decay=wd,
                         precision=precision, growth_interval=1000)
    # the oracle takes the FP32 values of the hyper-parameters the kernel uses
    tc = orc.TrainConfig(batch=c["batch"], lr=f32(lr), beta1=f32(b1), beta2=f32(b2), eps=f32(eps),
                         weight_decay=f32(wd), mixed=prec == "fp16", growth_interval=1000)
    S0 = float(2 ** round(np.log2(c["batch"]))) if prec == "fp16" else 1.0
    st = orc.State(loss_scale=S0)
    th = th0.astype(np.float64)
    m1 = np.zeros_like(th)
    m2 = np.zeros_like(th)
    rng = np.random.default_rng(5)
    n = oc.n_params
    hp = (f32(b1), f32(b2), f32(lr), f32(eps), f32(wd))
    for k in range(3):
        g = _grad(rng, n, 1e-3 * (k + 1))
        th_prev, m1_prev, m2_prev = th.copy(), m1.copy(), m2.copy()
        orc.adam(oc, tc, st, th, m1, m2, g.astype(np.float64))
        m.adam_step(torch.from_numpy(g).cuda(), cfg)
        torch.cuda.synchronize()
        _compare(m, (th_prev, m1_prev, m2_prev), g.astype(np.float64), th, m1, m2, k + 1, hp)
        s = m.state()
        assert s["adam_t"] == k + 1 and s["skipped"] == 0
        assert s["loss_scale"] == S0
        assert s["iter"] == 0  # no samples were drawn
        # the weights and the moments carry the state of the next step: feed
        # the oracle the GPU's FP32 values so that rounding does not accumulate
        th = m.get_weights().astype(np.float64)
        m1, m2 = (a.astype(np.float64) for a in m.moments())
        assert not np.array_equal(th, th_prev) and not np.array_equal(m1, m1_prev) and not np.array_equal(m2, m2_prev)
    # a non-finite gradient: the step is skipped (weights, moments unchanged),
    # the FP16 path halves its loss scale, and the gradient buffer is cleared
    g = _grad(rng, n, 1e-3)
    g[17] = np.inf
    m.adam_step(torch.from_numpy(g).cuda(), cfg)
    orc.adam(oc, tc, st, th, m1, m2, g.astype(np.float64))
    torch.cuda.synchronize()
    s = m.state()
    assert s["skipped"] == 1 and s["adam_t"] == 3
    assert s["loss_scale"] == (S0 / 2 if prec == "fp16" else 1.0) == st.loss_scale
    np.testing.assert_array_equal(m.get_weights(), th.astype(np.float32))
    # the next step sees only its own gradient (a leftover would show here)
    g = _grad(rng, n, 2e-3)
    prev = (th.copy(), m1.copy(), m2.copy())
    orc.adam(oc, tc, st, th, m1, m2, g.astype(np.float64))
    m.adam_step(torch.from_numpy(g).cuda(), cfg)
    torch.cuda.synchronize()
    _compare(m, prev, g.astype(np.float64), th, m1, m2, 4, hp)
    assert m.state()["adam_t"] == 4
    m.close()


def test_adam_step_rejects_bad_arguments(dv, orc, A):
    c, oc, m, _ = _setup(dv, orc, 3)
    g = torch.zeros(m.n_params, device="cuda")
    with pytest.raises(A.DvnrError):
        m.adam_step(g, dv.TrainConfig(batch=c["batch"], lr=-1.0))
    m.close()
