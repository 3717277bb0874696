"""Pins of the oracle's FP16 emulation (the mixed-precision path's rounding points).

The mixed-precision path stores tables and weights as binary16 and rounds the
encoding output, every hidden activation after the ReLU, the scaled output
gradient in the dW_out product and every hidden-layer gradient dZ to
binary16; dL/dy, dL/d(encoding), the network output and all accumulations stay
wide (the FP16 tensor-core operands with FP32 accumulation of Sec. 3.6; the
paper stores weights as 16-bit floats, Sec. 3.4).

Each test below builds a one-path network (one level, two features, two hidden
layers of two units, one sample, L2 loss) whose values are dyadic rationals
with few bits, so that every rounding point but ONE acts on a value binary16
holds exactly. The expected outputs are worked out by hand for that network,
with numpy's float16 at the one inexact point. Dropping that rounding changes
the outputs of exactly that test; dropping any other rounding changes nothing
there. Two more tests pin values that must NOT be rounded (dL/d(encoding) and
the network output). Every case runs at loss scales 1 and 2^6: power-of-two
scales leave every quantity exact, and the unscaled gradients must not change.

Parameter layout (compact): level 0 is dense (N = 1, 8 vertices, index
x + 2y + 4z), 8 entries x 2 features; W0 [2 x 2], W1 [2 x 2], w_out [2], all
row-major [out][in]. The sample sits on the x edge of the cell: coordinate
(f 2^24, 0, 0) weights corner 0 by 1 - f and corner 1 by f.
"""
import numpy as np
import pytest

Q = 2.0 ** -10  # binary16 quantum on [1, 2)


def f16(v):
    return float(np.float16(v))


def _cfg(orc):
    return orc.Config(1, 2, 4, 1, 1.0, 2, 2)


def _theta(orc, cfg, t0, t1, W0, W1, wout):
    th = np.zeros(cfg.n_params)
    th[0:2] = t0  # corner (0,0,0), features 0 and 1
    th[2:4] = t1  # corner (1,0,0)
    w = cfg.w_off
    th[w[0]:w[0] + 4] = np.ravel(W0)
    th[w[1]:w[1] + 4] = np.ravel(W1)
    th[w[2]:w[2] + 2] = wout
    assert cfg.n_params == w[2] + 2 == 26
    return th


def _run(orc, th, frac_x, target, S, mixed=True):
    cfg = _cfg(orc)
    m = np.array([[int(frac_x * 2 ** 24), 0, 0]], dtype=np.uint32)
    assert m[0, 0] == frac_x * 2 ** 24
    return orc.fwd_bwd(cfg, th, m, np.array([target]), loss=1, mixed=mixed, loss_scale=S,
                       grad_norm_count=1)


def _enc(frac_x, dx0):
    """Table gradient of the sample: corner 0 gets (1 - f) dx0, corner 1 f dx0."""
    g = np.zeros(16)
    g[0:2] = (1 - frac_x) * np.asarray(dx0, dtype=np.float64)
    g[2:4] = frac_x * np.asarray(dx0, dtype=np.float64)
    return g


def _check(r, y, loss, dx0, g_enc, gW0, gW1, gwout):
    assert r["y"][0] == y
    assert r["loss"] == loss
    np.testing.assert_array_equal(r["dx0"][0], dx0)
    np.testing.assert_array_equal(r["grad_enc"], g_enc)
    np.testing.assert_array_equal(r["grad_mlp"], np.concatenate([np.ravel(gW0), np.ravel(gW1), gwout]))


SCALES = [1.0, 2.0 ** 6]


@pytest.mark.parametrize("S", SCALES)
def test_tables_are_read_as_binary16(orc, S):
    t00 = 1 + 2 ** -12                     # rounds to 1 when read
    assert f16(t00) == 1.0
    t10 = -(1 - 2 ** -6)                   # exact
    th = _theta(orc, _cfg(orc), [t00, 0], [t10, 0], [[1, 0], [0, 0]], [[1, 0], [0, 0]], [1, 0])
    r = _run(orc, th, 0.5, 0.0, S)
    x0 = 0.5 * f16(t00) + 0.5 * t10       # 2^-7: exact, so the encoding rounding is idle
    assert x0 == 2 ** -7
    y = x0                                 # one path of unit weights
    gy = 2 * y                             # L2, batch 1; unscaled
    _check(r, y, y * y, [gy, 0], _enc(0.5, [gy, 0]), [[gy * x0, 0], [0, 0]],
           [[gy * x0, 0], [0, 0]], [gy * x0, 0])
    assert _run(orc, th, 0.5, 0.0, S, mixed=False)["y"][0] == 0.5 * t00 + 0.5 * t10 != y


@pytest.mark.parametrize("S", SCALES)
def test_weights_are_read_as_binary16(orc, S):
    a = 1 + 2 ** -12                       # first-layer weight, rounds to 1
    c = 1 + 2 ** -12                       # output weight, rounds to 1
    th = _theta(orc, _cfg(orc), [1, 0], [0, 0], [[a, 0], [0, 0]], [[1, 0], [0, 0]], [c, 0])
    r = _run(orc, th, 0.0, 0.5, S)
    y = f16(c) * 1.0                       # x0 = h1 = h2 = 1 on unit 0
    assert y == 1.0
    gy = 2 * (y - 0.5)                     # = 1
    dx0 = f16(a) * gy                      # dL/dx0 seen through the rounded W0: 1
    _check(r, y, 0.25, [dx0, 0], _enc(0.0, [dx0, 0]), [[1, 0], [0, 0]], [[1, 0], [0, 0]], [1, 0])
    fr = _run(orc, th, 0.0, 0.5, S, mixed=False)
    assert fr["y"][0] == a * c and fr["dx0"][0, 0] != dx0


@pytest.mark.parametrize("S", SCALES)
def test_encoding_output_is_binary16(orc, S):
    # tables exact; the interpolated feature 0 at f = 1/4 is 1 + 2^-12, which
    # rounds to 1; W0 row 0 subtracts feature 1 (= 1) to expose the rounding
    th = _theta(orc, _cfg(orc), [1, 1], [1 + Q, 1], [[1, -1], [0, 1]], [[1, 0], [0, 1]], [1, 1])
    x0_wide = 0.75 * 1 + 0.25 * (1 + Q)
    assert x0_wide == 1 + 2 ** -12
    x0 = f16(x0_wide)
    assert x0 == 1.0
    r = _run(orc, th, 0.25, 0.5, S)
    # z1 = (x0_0 - x0_1, x0_1) = (0, 1): unit 0 off; y = h2_1 = 1
    y = (x0 - 1) + 1
    gy = 2 * (y - 0.5)                     # 1
    gW0 = [[0, 0], [gy * x0, gy * 1]]      # only unit 1 of layer 1 carries gradient
    _check(r, y, 0.25, [0, gy], _enc(0.25, [0, gy]), gW0, [[0, 0], [0, gy]], [0, gy])
    assert _run(orc, th, 0.25, 0.5, S, mixed=False)["y"][0] == 1 + 2 ** -12


@pytest.mark.parametrize("S", SCALES)
def test_first_hidden_activation_is_binary16(orc, S):
    e = 1 + Q
    th = _theta(orc, _cfg(orc), [e, e], [0, 0], [[e, 0], [0, 1]], [[1, -1], [0, 1]], [1, 0])
    r = _run(orc, th, 0.0, 2 ** -10 - 0.5, S)
    h1 = [f16(e * e), e]                   # (1 + 2^-9 + 2^-20) rounds to 1 + 2^-9
    assert h1[0] == 1 + 2 * Q
    h2 = [h1[0] - h1[1], h1[1]]            # (2^-10, 1 + 2^-10), both exact
    y = h2[0]
    assert y == 2 ** -10
    gy = 1.0                               # target y - 1/2
    # dz2 = (gy, 0); dh1 = (gy, -gy); dz1 = (gy, -gy)
    gW1 = [[gy * h1[0], gy * h1[1]], [0, 0]]
    gW0 = [[gy * e, gy * e], [-gy * e, -gy * e]]
    dx0 = [e * gy, -gy]
    _check(r, y, 0.25, dx0, _enc(0.0, dx0), gW0, gW1, [gy * h2[0], gy * h2[1]])
    fr = _run(orc, th, 0.0, 2 ** -10 - 0.5, S, mixed=False)
    assert fr["y"][0] == e * e - e != y


@pytest.mark.parametrize("S", SCALES)
def test_last_hidden_activation_is_binary16(orc, S):
    e = 1 + Q
    th = _theta(orc, _cfg(orc), [e, 1], [0, 0], [[1, 0], [0, 1]], [[e, 0], [0, 1]], [1, -1])
    h1 = [e, 1.0]
    h2 = [f16(e * e), 1.0]                 # 1 + 2^-9
    y = h2[0] - h2[1]                      # 2^-9, not rounded itself
    assert y == 2 ** -9
    r = _run(orc, th, 0.0, y - 0.5, S)
    gy = 1.0
    dz2 = [gy, -gy]
    dz1 = [e * dz2[0], dz2[1]]             # W1^T dz2 = (e, -1): exact
    gW1 = [[dz2[0] * h1[0], dz2[0] * h1[1]], [dz2[1] * h1[0], dz2[1] * h1[1]]]
    gW0 = [[dz1[0] * e, dz1[0] * 1], [dz1[1] * e, dz1[1] * 1]]
    _check(r, y, 0.25, dz1, _enc(0.0, dz1), gW0, gW1, [gy * h2[0], gy * h2[1]])
    assert _run(orc, th, 0.0, y - 0.5, S, mixed=False)["y"][0] == e * e - 1 != y


@pytest.mark.parametrize("S", SCALES)
def test_output_gradient_operand_of_dW_out_is_binary16(orc, S):
    # unit 0 of the last layer has w_out = 0 (so its dZ is an exact 0) but a
    # positive activation, so dW_out[0] = fp16(S dL/dy) h2_0 / S shows the
    # rounding of the scaled output gradient; unit 1 is off
    th = _theta(orc, _cfg(orc), [1, 0], [0, 0], [[1, 0], [0, 0]], [[1, 0], [-1, 0]], [0, 1])
    t = 1 + 2 ** -20
    r = _run(orc, th, 0.0, t, S)
    y = 0.0
    gy = 2 * (y - t)                       # -2 - 2^-19: not a binary16 value
    g_op = f16(gy * S) / S                 # -2
    assert g_op == -2.0 != gy
    _check(r, y, t * t, [0, 0], np.zeros(16), [[0, 0], [0, 0]], [[0, 0], [0, 0]], [g_op * 1.0, 0])
    assert _run(orc, th, 0.0, t, S, mixed=False)["grad_mlp"][8] == gy


@pytest.mark.parametrize("S", SCALES)
def test_top_hidden_gradient_is_binary16(orc, S):
    e = 1 + Q
    th = _theta(orc, _cfg(orc), [1, 0], [0, 0], [[1, 0], [0, 0]], [[1, 0], [0, 0]], [e, 0])
    y = e                                  # h1 = h2 = (1, 0)
    t = 0.5 + 2 ** -11                     # dL/dy = 2 (y - t) = 1 + 2^-10
    r = _run(orc, th, 0.0, t, S)
    gy = 2 * (y - t)
    assert gy == e
    dz2 = f16(gy * S * e) / S              # (1 + 2^-10)^2 rounds to 1 + 2^-9
    assert dz2 == 1 + 2 * Q
    _check(r, y, (y - t) ** 2, [dz2, 0], _enc(0.0, [dz2, 0]), [[dz2, 0], [0, 0]],
           [[dz2, 0], [0, 0]], [gy, 0])
    assert _run(orc, th, 0.0, t, S, mixed=False)["grad_mlp"][4] == e * e


@pytest.mark.parametrize("S", SCALES)
def test_lower_hidden_gradient_is_binary16(orc, S):
    e = 1 + Q
    th = _theta(orc, _cfg(orc), [1, 0], [0, 0], [[1, 0], [0, 0]], [[e, 0], [0, 0]], [e, 0])
    y = e * e                              # the output stays wide: 1 + 2^-9 + 2^-20
    assert f16(y) != y
    r = _run(orc, th, 0.0, y - 0.5, S)
    gy = 1.0
    dz2 = e * gy                           # exact
    dz1 = f16(e * dz2 * S) / S             # (1 + 2^-10)^2 rounds to 1 + 2^-9
    assert dz1 == 1 + 2 * Q
    _check(r, y, 0.25, [dz1, 0], _enc(0.0, [dz1, 0]), [[dz1, 0], [0, 0]], [[dz2, 0], [0, 0]],
           [gy * e, 0])
    assert _run(orc, th, 0.0, y - 0.5, S, mixed=False)["grad_mlp"][0] == e * e


@pytest.mark.parametrize("S", SCALES)
def test_encoding_gradient_stays_wide(orc, S):
    # dL/d(encoding) = W0^T dz1 / S is (1 + 2^-10)^2, which binary16 cannot
    # hold: it must reach the table gradients unrounded
    e = 1 + Q
    th = _theta(orc, _cfg(orc), [1, 0], [0, 0], [[e, 0], [0, 0]], [[1, 0], [0, 0]], [e, 0])
    x0 = 0.5                               # (1 - 1/2) 1 + (1/2) 0 on feature 0; feature 1 is 0
    h1 = e * x0                            # 1/2 + 2^-11: exact, and h2 = h1
    y = e * h1
    r = _run(orc, th, 0.5, y - 0.5, S)
    gy = 1.0
    dz2 = e                                # fp16(gy e): exact
    dz1 = dz2                              # W1 = identity on unit 0
    dx0 = e * dz1                          # not rounded
    assert f16(dx0) != dx0
    _check(r, y, 0.25, [dx0, 0], _enc(0.5, [dx0, 0]), [[dz1 * x0, 0], [0, 0]],
           [[dz2 * h1, 0], [0, 0]], [gy * h1, 0])


def test_mixed_decode_shares_the_forward_rounding_points(orc):
    """The decoder's forward (mixed) gives the hand-derived outputs of the
    networks above: tables, weights, encoding output and both hidden
    activations are rounded, the output is not."""
    cfg = _cfg(orc)
    e = 1 + Q
    cases = [
        # (t0, t1, W0, W1, wout, frac, expected y, FP64 y)
        ([1 + 2 ** -12, 0], [-(1 - 2 ** -6), 0], [[1, 0], [0, 0]], [[1, 0], [0, 0]], [1, 0], 0.5,
         2 ** -7, 2 ** -7 + 2 ** -13),
        ([1, 0], [0, 0], [[1, 0], [0, 0]], [[1, 0], [0, 0]], [1 + 2 ** -12, 0], 0.0, 1.0, 1 + 2 ** -12),
        ([1, 1], [1 + Q, 1], [[1, -1], [0, 1]], [[1, 0], [0, 1]], [1, 1], 0.25, 1.0, 1 + 2 ** -12),
        ([e, e], [0, 0], [[e, 0], [0, 1]], [[1, -1], [0, 1]], [1, 0], 0.0, 2 ** -10, e * e - e),
        ([e, 1], [0, 0], [[1, 0], [0, 1]], [[e, 0], [0, 1]], [1, -1], 0.0, 2 ** -9, e * e - 1),
        ([1, 0], [0, 0], [[1, 0], [0, 0]], [[e, 0], [0, 0]], [e, 0], 0.0, e * e, e * e),
    ]
    for t0, t1, W0, W1, wout, frac, y16, y64 in cases:
        th = _theta(orc, cfg, t0, t1, W0, W1, wout)
        m = np.array([[int(frac * 2 ** 24), 0, 0]], dtype=np.uint32)
        assert orc.decode_unit(cfg, th, m, 0.0, 1.0, mixed=True)[0] == y16
        assert orc.decode_unit(cfg, th, m, 0.0, 1.0, mixed=False)[0] == y64
        # de-normalisation y (vmax - vmin) + vmin after the network
        assert orc.decode_unit(cfg, th, m, -1.0, 3.0, mixed=True)[0] == y16 * 4.0 - 1.0
