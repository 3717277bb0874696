"""The fused Adam kernel element by element against the oracle's Adam step.

Sec. 3.6: Adam with beta1 0.9, beta2 0.999, eps 1e-8 and L2 weight decay
added to the gradient of every parameter; Kingma & Ba bias correction; FP32
master weights and moments, an FP16 copy for the tensor-core path and dynamic
loss scaling there. dvnr_adam_step feeds the library's own optimiser kernel a
gradient chosen by the test, so a step is compared with orc_adam on identical
inputs: the FP32 weights, both moments and a gradient of FP32 values.

Tolerances (FP32 arithmetic against FP64): moments within 1e-6 relative; the
new weight within 1e-6 of (|theta| + |step|), the step being lr m^/(sqrt(v^)
+ eps) -- a few FP32 roundings of each term; the FP16 copy bit-exact to
binary16 rounding of the FP32 master weight.
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


def _compare(m, th, m1, m2, step):
    got = m.get_weights().astype(np.float64)
    g1, g2 = (a.astype(np.float64) for a in m.moments())
    np.testing.assert_allclose(g1, m1, rtol=1e-6, atol=1e-30)
    np.testing.assert_allclose(g2, m2, rtol=1e-6, atol=1e-30)
    err = np.abs(got - th)
    bound = 1e-6 * (np.abs(th) + np.abs(step)) + 1e-30
    worst = int(np.argmax(err / bound))
    assert np.all(err <= bound), f"theta[{worst}]: {got[worst]!r} vs {th[worst]!r} (step {step[worst]:.3e})"
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
    for k in range(3):
        g = _grad(rng, n, 1e-3 * (k + 1))
        th_prev, m1_prev, m2_prev = th.copy(), m1.copy(), m2.copy()
        orc.adam(oc, tc, st, th, m1, m2, g.astype(np.float64))
        m.adam_step(torch.from_numpy(g).cuda(), cfg)
        torch.cuda.synchronize()
        _compare(m, th, m1, m2, th - th_prev)
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
    th_prev = th.copy()
    orc.adam(oc, tc, st, th, m1, m2, g.astype(np.float64))
    m.adam_step(torch.from_numpy(g).cuda(), cfg)
    torch.cuda.synchronize()
    _compare(m, th, m1, m2, th - th_prev)
    assert m.state()["adam_t"] == 4
    m.close()


def test_adam_step_rejects_bad_arguments(dv, orc, A):
    c, oc, m, _ = _setup(dv, orc, 3)
    g = torch.zeros(m.n_params, device="cuda")
    with pytest.raises(A.DvnrError):
        m.adam_step(g, dv.TrainConfig(batch=c["batch"], lr=-1.0))
    m.close()
