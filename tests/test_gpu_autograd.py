"""The network as a differentiable function: dvnr_forward / dvnr_backward and
the EncodeMLP autograd Function over them (Sec. 3: hash-grid encoding + ReLU
MLP; Sec. 3.6: trained by back-propagation through both).

1. Finite differences: the gradient EncodeMLP returns equals central
   differences of its own FP32 forward (tiny model, L2 loss, points whose
   pre-activations stay clear of the ReLU kinks under the perturbation).
2. Oracle parity at caller-given points and upstream gradients: forward y,
   dL/d(encoding) and the table and MLP gradients within 1e-5 (FP32) and
   2e-3 (FP16, against the oracle's FP16 emulation) -- normwise for batch
   sums, plus the kink allowance of parity.py.
3. The FP16 kernels on the one-path networks of the oracle's binary16 pins,
   embedded in a width-16 MLP: every output bit-identical to the oracle's
   (whose values are worked out by hand in test_oracle_fp16_points.py).
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


def _model(dv, c, seed=0):
    enc = dv.EncodingConfig(c["L"], c["F"], c["log2T"], c["base"], c["growth"])
    return dv.Model((0, 0, 0), (32, 32, 32), 0, enc, dv.MLPConfig(c["width"], c["hidden"]), seed=seed)


def _coords(rng, n):
    return rng.integers(0, 2 ** 24 + 1, size=(n, 3)).astype(np.uint32)


def _cuda_coords(m):
    return torch.from_numpy(m.view(np.int32)).cuda()


TINY = dict(L=2, F=2, log2T=6, base=4, growth=1.5, width=16, hidden=1)


def test_encode_mlp_gradient_matches_finite_differences(dv, orc, A):
    c = TINY
    oc = P.oracle_cfg(c)
    rng = np.random.default_rng(11)
    theta = P.random_theta(oc, 12, table_scale=0.5)
    m = _model(dv, c)
    n = 256
    coords = _coords(rng, n)
    t = rng.uniform(-0.5, 0.5, n)
    # keep points whose hidden pre-activations all lie more than 5e-3 from
    # the ReLU kink (FP64 oracle): a perturbation h = 2e-3 of one parameter
    # moves a pre-activation by at most h (|W0| < 1, |x0| < 1), so no unit
    # switches and the loss is exactly quadratic along the perturbation
    r = orc.fwd_bwd(oc, theta.astype(np.float64), coords, t, loss=1, want_zabs=True)
    keep = r["zabs"][:, :-1].min(axis=1) > 5e-3
    assert keep.sum() >= 64
    coords, t = coords[keep], t[keep]
    n = len(t)
    mc = _cuda_coords(coords)
    tt = torch.from_numpy(t).cuda()  # FP64: the loss adds no FP32 rounding
    EncodeMLP = dv.EncodeMLP
    params = torch.from_numpy(theta).cuda().requires_grad_(True)

    def loss_of(p):
        y = EncodeMLP.apply(p, mc, m, A.DVNR_FP32)
        return ((y.double() - tt) ** 2).mean()

    L = loss_of(params)
    L.backward()
    g = params.grad.detach().cpu().numpy().astype(np.float64)
    # the oracle's FP64 gradient of the same loss
    r = orc.fwd_bwd(oc, theta.astype(np.float64), coords, t, loss=1)
    want = np.concatenate([r["grad_enc"], r["grad_mlp"]])
    P.assert_normwise(g, want, 1e-5, what="EncodeMLP gradient vs oracle")
    # central differences of the FP32 forward on the largest-gradient table
    # entries and a spread of MLP weights
    h = 2e-3
    idx = list(np.argsort(-np.abs(want[: oc.n_enc]))[:12]) + \
        list(oc.n_enc + rng.choice(oc.n_mlp, 12, replace=False))
    base = params.detach().clone()
    with torch.no_grad():
        for j in idx:
            pp = base.clone()
            pp[j] += h
            lp = float(loss_of(pp))
            pp[j] -= 2 * h
            lm = float(loss_of(pp))
            fd = (lp - lm) / (2 * h)
            # exact for a quadratic up to the FP32 rounding of the outputs y
            # (about 1e-7 |y| each, times 2 |y - t| in the loss, over 2h)
            tol = 1e-5 + 1e-3 * abs(want[j])
            assert abs(fd - g[j]) <= tol, (j, fd, g[j], want[j])
    m.close()


CONFIGS = {
    "blobs64": P.configs_blobs64(),
    "w64d32h3": dict(L=16, F=2, log2T=14, base=16, growth=1.38, width=64, hidden=3),
    "nekrs_w16d20h3_f4": dict(L=5, F=4, log2T=12, base=16, growth=2.0, width=16, hidden=3),
}


@pytest.mark.parametrize("name", sorted(CONFIGS))
@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("n", [4096, 333])
def test_backward_at_given_points_matches_oracle(dv, orc, A, name, prec, n):
    c = CONFIGS[name]
    oc = P.oracle_cfg(c)
    mixed = prec == "fp16"
    precision = A.DVNR_FP16 if mixed else A.DVNR_FP32
    rng = np.random.default_rng(sum(name.encode()) + n)
    theta = P.random_theta(oc, 7, table_scale=0.4)
    th64 = theta.astype(np.float64)
    m = _model(dv, c)
    coords = _coords(rng, n)
    # upstream gradient of a mean L2 loss with targets half a unit away
    y0 = orc.fwd_bwd(oc, th64, coords, np.zeros(n), loss=1, mixed=mixed, want_grads=False)["y"]
    t = y0 + rng.choice([-0.5, 0.5], n)
    dy64 = 2.0 * (y0 - t) / n
    S = float(2 ** round(np.log2(n))) if mixed else 1.0
    r = orc.fwd_bwd(oc, th64, coords, t, loss=1, mixed=mixed, loss_scale=S, want_zabs=True)
    mc = _cuda_coords(coords)
    params = torch.from_numpy(theta).cuda()
    A.call("dvnr_load_params", m.handle, params.data_ptr(), None)
    y = m.forward(mc, precision).cpu().numpy()
    tol = 2e-3 if mixed else 1e-5
    np.testing.assert_allclose(y, r["y"], atol=tol * max(1.0, np.abs(r["y"]).max()), rtol=0)
    g, dx0 = m.backward(mc, torch.from_numpy(dy64.astype(np.float32)).cuda(), precision,
                        loss_scale=S if mixed else 0.0, want_dx0=True)
    torch.cuda.synchronize()
    delta = 1e-4 if mixed else 1e-5
    a_enc, a_mlp, flagged = P.kink_allowance(oc, th64, coords, t, 1, mixed, S, n, r["zabs"], delta=delta)
    keep = np.ones(n, bool)
    keep[flagged] = False
    assert keep.sum() > 0.6 * n
    P.assert_normwise(dx0.cpu().numpy()[keep], r["dx0"][keep], tol, what="dL/dx0")
    g = g.cpu().numpy()
    P.assert_normwise(g[: oc.n_enc], r["grad_enc"], tol, a_enc, what="table grad")
    P.assert_normwise(g[oc.n_enc:], r["grad_mlp"], tol, a_mlp, what="mlp grad")
    # the automatic loss scale (max |dy| S in [1, 2)) gives the oracle's
    # result at that scale
    if mixed:
        e = np.frexp(np.abs(dy64.astype(np.float32)).max())[1]
        S_auto = float(2.0 ** (1 - e))
        g2, _ = m.backward(mc, torch.from_numpy(dy64.astype(np.float32)).cuda(), precision, 0.0)
        r2 = orc.fwd_bwd(oc, th64, coords, t, loss=1, mixed=True, loss_scale=S_auto)
        g2 = g2.cpu().numpy()
        P.assert_normwise(g2[: oc.n_enc], r2["grad_enc"], tol, a_enc, what="table grad, auto scale")
        P.assert_normwise(g2[oc.n_enc:], r2["grad_mlp"], tol, a_mlp, what="mlp grad, auto scale")
    # the model's training state is untouched by forward and backward
    s = m.state()
    assert s["adam_t"] == 0 and s["iter"] == 0
    m.close()


# one-path networks of the oracle's binary16 pins: (t0, t1, W0, W1, wout, frac, target)
E = 1 + 2.0 ** -10
PIN_NETWORKS = [
    ([1 + 2 ** -12, 0], [-(1 - 2 ** -6), 0], [[1, 0], [0, 0]], [[1, 0], [0, 0]], [1, 0], 0.5, 0.0),
    ([1, 0], [0, 0], [[1 + 2 ** -12, 0], [0, 0]], [[1, 0], [0, 0]], [1 + 2 ** -12, 0], 0.0, 0.5),
    ([1, 1], [1 + 2 ** -10, 1], [[1, -1], [0, 1]], [[1, 0], [0, 1]], [1, 1], 0.25, 0.5),
    ([E, E], [0, 0], [[E, 0], [0, 1]], [[1, -1], [0, 1]], [1, 0], 0.0, 2 ** -10 - 0.5),
    ([E, 1], [0, 0], [[1, 0], [0, 1]], [[E, 0], [0, 1]], [1, -1], 0.0, 2 ** -9 - 0.5),
    ([1, 0], [0, 0], [[1, 0], [0, 0]], [[1, 0], [-1, 0]], [0, 1], 0.0, 1 + 2 ** -20),
    ([1, 0], [0, 0], [[1, 0], [0, 0]], [[1, 0], [0, 0]], [E, 0], 0.0, 0.5 + 2 ** -11),
    ([1, 0], [0, 0], [[1, 0], [0, 0]], [[E, 0], [0, 0]], [E, 0], 0.0, E * E - 0.5),
    ([1, 0], [0, 0], [[E, 0], [0, 0]], [[1, 0], [0, 0]], [E, 0], 0.5, E * E / 2 - 0.5),
]


@pytest.mark.parametrize("k", range(len(PIN_NETWORKS)))
@pytest.mark.parametrize("S", [1.0, 64.0])
def test_fp16_kernels_on_the_binary16_pin_networks(dv, orc, A, k, S):
    t0, t1, W0, W1, wout, frac, target = PIN_NETWORKS[k]
    W = 16
    c = dict(L=1, F=2, log2T=4, base=1, growth=1.0, width=W, hidden=2)
    oc16 = P.oracle_cfg(c)
    th = np.zeros(oc16.n_params)
    th[0:2], th[2:4] = t0, t1
    w = oc16.w_off
    W0f = np.zeros((W, 2))
    W0f[:2] = W0
    W1f = np.zeros((W, W))
    W1f[:2, :2] = W1
    wo = np.zeros(W)
    wo[:2] = wout
    th[w[0]:w[0] + 2 * W] = W0f.ravel()
    th[w[1]:w[1] + W * W] = W1f.ravel()
    th[w[2]:w[2] + W] = wo
    coords = np.array([[int(frac * 2 ** 24), 0, 0]], dtype=np.uint32)
    r = orc.fwd_bwd(oc16, th, coords, np.array([target]), loss=1, mixed=True, loss_scale=S,
                    grad_norm_count=1)
    dy = 2.0 * (r["y"][0] - target)  # the upstream gradient the oracle's L2 used
    assert np.float32(dy) == dy
    m = dv.Model((0, 0, 0), (8, 8, 8), 0, dv.EncodingConfig(1, 2, 4, 1, 1.0), dv.MLPConfig(W, 2))
    assert m.n_params == oc16.n_params
    params = torch.from_numpy(th.astype(np.float32)).cuda()  # held until the loads ran
    A.call("dvnr_load_params", m.handle, params.data_ptr(), None)
    mc = _cuda_coords(coords)
    y = m.forward(mc, A.DVNR_FP16).cpu().numpy()
    g, dx0 = m.backward(mc, torch.tensor([dy], dtype=torch.float32, device="cuda"), A.DVNR_FP16,
                        loss_scale=S, want_dx0=True)
    torch.cuda.synchronize()
    assert y[0] == r["y"][0]
    np.testing.assert_array_equal(dx0.cpu().numpy()[0], r["dx0"][0])
    np.testing.assert_array_equal(g.cpu().numpy(), np.concatenate([r["grad_enc"], r["grad_mlp"]]))
    m.close()


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_encode_mlp_trains_under_a_torch_optimizer(dv, A, prec):
    # EncodeMLP as a building block: a torch optimizer fits the network to a
    # smooth target through the library's forward and backward kernels
    c = dict(L=8, F=2, log2T=14, base=4, growth=1.5, width=32, hidden=2)
    m = _model(dv, c, seed=3)
    precision = A.DVNR_FP16 if prec == "fp16" else A.DVNR_FP32
    params = m.params_tensor().requires_grad_(True)
    opt = torch.optim.Adam([params], lr=1e-2)
    gen = torch.Generator(device="cuda").manual_seed(0)
    losses = []
    for step in range(150):
        coords = torch.randint(0, (1 << 24) + 1, (4096, 3), dtype=torch.int32, device="cuda", generator=gen)
        u = coords.double() / (1 << 24)
        target = 0.5 + 0.3 * torch.sin(2 * np.pi * u[:, 0]) * torch.cos(2 * np.pi * u[:, 1]) + 0.1 * u[:, 2]
        y = dv.EncodeMLP.apply(params, coords, m, precision)
        loss = ((y.double() - target) ** 2).mean()
        opt.zero_grad()
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    assert np.isfinite(losses).all()
    assert np.mean(losses[-10:]) < 0.05 * np.mean(losses[:5]), (losses[:5], losses[-10:])
    m.close()
