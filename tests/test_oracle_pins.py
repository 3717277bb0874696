"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: published
known-answer vectors, closed forms, exact special cases, library routines
(numpy/scipy) for sub-steps that reduce to them, brute force on tiny inputs,
or finite differences. A plausible slip in the oracle (dropped term, wrong
sign or index, transposed operand) fails at least one of them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


# ---------------------------------------------------------------- Philox ----
def test_philox_known_answers(orc):
    for row in _golden_rows("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in row]
        out = orc.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


# --------------------------------------------------------- level layout ----
def _layout_rows():
    rows = []
    with open(os.path.join(GOLDEN, "level_layout.txt")) as f:
        for ln in f:
            if not ln.strip() or ln.startswith("#"):
                continue
            head, ns, nd, npar = [p.split() for p in ln.split("|")]
            rows.append((head, [int(x) for x in ns], int(nd[0]), int(npar[0])))
    return rows


@pytest.mark.parametrize("row", _layout_rows(), ids=lambda r: r[0][0])
def test_level_resolutions_and_sizes(orc, row):
    head, ns, n_dense, n_params = row
    L, F, log2T, base = (int(x) for x in head[1:5])
    b = head[5]
    width, hidden = int(head[6]), int(head[7])
    cfg = orc.Config(L, F, log2T, base, float(b), width, hidden)
    assert cfg.N == ns
    # exact rational evaluation of floor(N_min * b^l): independent of FP pow
    bq = Fraction(b)
    assert [math.floor(base * bq ** l) for l in range(L)] == ns
    T = 1 << log2T
    dense = [(n + 1) ** 3 <= T for n in ns]
    assert sum(dense) == n_dense and cfg.dense == [int(d) for d in dense]
    n_enc = sum(min((n + 1) ** 3, T) * F for n in ns)
    n_mlp = width * L * F + (hidden - 1) * width * width + width
    assert cfg.n_enc == n_enc and cfg.n_mlp == n_mlp
    assert cfg.n_params == n_params == n_enc + n_mlp


# --------------------------------------------------------------- hashing ----
def test_dense_levels_are_bijective(orc):
    cfg = orc.Config(4, 2, 10, 3, 1.5, 16, 1)  # N = 3, 4, 6, 10 ; T = 1024
    for l in range(cfg.L):
        if not cfg.dense[l]:
            continue
        n1 = cfg.N[l] + 1
        seen = set()
        for z in range(n1):
            for y in range(n1):
                for x in range(n1):
                    i = orc.corner_index(cfg, l, x, y, z)
                    assert 0 <= i < cfg.entries[l]
                    seen.add(i)
        assert len(seen) == n1 ** 3  # bijective onto [0, (N+1)^3)


def test_spatial_hash_structure(orc):
    # Hashed level: Mueller et al. Eq. 4 with primes pi_1 = 1,
    # pi_2 = 2654435761, pi_3 = 805459861, arithmetic modulo 2^32, then mod T.
    cfg = orc.Config(2, 2, 6, 8, 2.0, 16, 1)  # N = 8, 16 ; T = 64 -> both hashed
    assert cfg.dense == [0, 0]
    T = 64
    for x in range(0, 200, 7):
        assert orc.corner_index(cfg, 1, x, 0, 0) == x % T  # pi_1 = 1
    assert orc.corner_index(cfg, 1, 0, 1, 0) == 2654435761 % T
    assert orc.corner_index(cfg, 1, 0, 0, 1) == 805459861 % T
    # wrap-around modulo 2^32 (2 * 2654435761 > 2^32) and odd prime * 2^31
    assert orc.corner_index(cfg, 1, 0, 2, 0) == (2 * 2654435761 - 2 ** 32) % T
    rng = np.random.default_rng(0)
    for _ in range(200):
        x, y, z = (int(v) for v in rng.integers(0, 2000, 3))
        h = orc.corner_index(cfg, 1, x, y, z)
        assert h == (orc.corner_index(cfg, 1, x, 0, 0) ^ orc.corner_index(cfg, 1, 0, y, 0)
                     ^ orc.corner_index(cfg, 1, 0, 0, z))


def test_hash_vs_bruteforce_tiny_grids(orc):
    # All vertices of tiny hashed grids against an independent big-integer
    # evaluation of the XOR-of-products hash (T = 2^4 .. 2^8).
    for log2T in (4, 6, 8):
        cfg = orc.Config(1, 1, log2T, 7, 1.0, 16, 1)  # one level, N = 7, 512 vertices
        dense = 8 ** 3 <= (1 << log2T)
        assert cfg.dense[0] == int(dense)
        for z in range(8):
            for y in range(8):
                for x in range(8):
                    if dense:
                        expect = x + 8 * y + 64 * z
                    else:
                        prod = [x * 1, y * 2654435761, z * 805459861]
                        expect = ((prod[0] ^ prod[1] ^ prod[2]) % (1 << 32)) % (1 << log2T)
                    assert orc.corner_index(cfg, 0, x, y, z) == expect


# ---------------------------------------------------------- fp16 rounding ---
def test_round_half_matches_numpy(orc):
    rng = np.random.default_rng(1)
    x = np.concatenate([
        rng.normal(0, 1, 3000), rng.normal(0, 1e-5, 1000), rng.normal(0, 3e4, 500),
        np.array([65504.0, 65519.99, 65520.0, 7e4, -7e4, 0.0, -0.0, 2 ** -24, 2 ** -25,
                  3 * 2 ** -26, 1 + 2 ** -11, 1 + 3 * 2 ** -11]),
    ])
    got = orc.round_half(x)
    with np.errstate(over="ignore"):
        want = x.astype(np.float16).astype(np.float64)
    np.testing.assert_array_equal(got, want)


# ----------------------------------------------------------- initialiser ----
def test_init_params_ranges_and_seed(orc):
    cfg = orc.Config(4, 2, 12, 4, 1.5, 16, 2)
    th = orc.init_params(cfg, 7)
    enc, mlp = th[: cfg.n_enc], th[cfg.n_enc:]
    assert np.all(np.abs(enc) <= 1e-4)
    assert np.all(th == th.astype(np.float32).astype(np.float64))  # binary32 values
    lim0 = math.sqrt(6.0 / (cfg.in_dim + cfg.width))
    w0 = mlp[: cfg.width * cfg.in_dim]
    assert np.all(np.abs(w0) <= lim0) and np.abs(w0).max() > 0.8 * lim0
    wout = th[cfg.w_off[cfg.n_hidden]:]
    assert np.all(np.abs(wout) <= math.sqrt(6.0 / (cfg.width + 1)))
    # uniform: mean ~0 and variance of U(-a, a) = a^2/3 on the tables
    assert abs(enc.mean()) < 3e-6 and abs(enc.var() / (1e-8 / 3) - 1) < 0.05
    assert not np.array_equal(th, orc.init_params(cfg, 8))
    # the i-th value is drawn from Philox block {i, 0, 0, 'INIT'} with key = seed
    r = orc.philox4x32_10([5, 0, 0, 0x494E4954], [7, 0])
    u = (int(r[0]) >> 8) / 2 ** 24
    assert th[5] == float(np.float32(-1e-4 + 2e-4 * u))


# ---------------------------------------------------------------- sampler ---
def test_quantile_table_matches_scipy(orc):
    scipy_stats = pytest.importorskip("scipy.stats")
    sigma = 0.005
    tab = orc.quantile_table(sigma)
    p = np.arange(4097) / 4096.0
    p[-1] = 1 - 2.0 ** -24
    want = scipy_stats.halfnorm.ppf(p) * sigma * 2 ** 24
    assert np.max(np.abs(tab - want)) <= 1.0
    assert tab[0] == 0 and np.all(np.diff(tab) >= 0)


def test_sampler_split_and_uniform_part(orc):
    B, lam = 4096, np.float32(0.15)
    tab = orc.quantile_table(0.005)
    m = orc.sample(11, 3, 5, B, float(lam), tab)
    nb = int(math.floor(float(lam) * B))
    assert nb == 614
    uni = m[nb:]
    assert uni.max() < 2 ** 24
    # uniform part equals (r >> 8) of Philox {i, iter, model, 'SAM\0'}
    r = orc.philox4x32_10([nb + 17, 5, 3, 0x53414D00], [11, 0])
    assert list(uni[17]) == [int(v) >> 8 for v in r[:3]]
    # boundary part: exactly one coordinate within 8 sigma of a face
    bnd = m[:nb].astype(np.int64)
    near = np.minimum(bnd, 2 ** 24 - bnd) <= int(8 * 0.005 * 2 ** 24)
    assert np.all(near.sum(axis=1) >= 1)


def test_sampler_boundary_distribution(orc):
    # Eq. 2 integrated over the two other coordinates gives every coordinate
    # the marginal density  2/3 uniform + 1/3 (half-normal from face 0 or 1,
    # equally likely) -- the normaliser of the six half-Gaussians is
    # 3 sigma sqrt(2 pi). Kolmogorov-Smirnov per axis against that CDF.
    st = pytest.importorskip("scipy.stats")
    sigma = 0.01
    tab = orc.quantile_table(sigma)
    B = 1 << 18
    m = np.concatenate([orc.sample(99, 0, it, B, 1.0, tab) for it in range(4)])
    u = m.astype(np.float64) / 2 ** 24

    def cdf(x):
        hn = st.halfnorm.cdf
        return 2.0 / 3.0 * x + 1.0 / 6.0 * (hn(x / sigma) + 1.0 - hn((1.0 - x) / sigma))

    for a in range(3):
        ks = st.kstest(u[:, a], cdf)
        assert ks.statistic < 1.63 / math.sqrt(u.shape[0]) + 2e-4, (a, ks)
    # exactly one coordinate per sample comes from the half-normal: the mass
    # within 3 sigma of a face is 1/3 * 0.9973 + 2/3 * 6 sigma per axis
    near = np.minimum(u, 1 - u) < 3 * sigma
    frac = near.mean(axis=0)
    np.testing.assert_allclose(frac, 0.9973 / 3 + 2.0 / 3.0 * 6 * sigma, atol=3e-3)


# ------------------------------------------------------ trilinear lookups ---
def test_volume_trilinear_affine_and_nodes(orc):
    nz, ny, nx = 5, 7, 9
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    vol = (0.5 + 0.25 * x + 0.125 * y - 0.0625 * z).astype(np.float32)  # exact in fp32
    rng = np.random.default_rng(3)
    for _ in range(200):
        m = rng.integers(0, 2 ** 24 + 1, 3).astype(np.uint32)
        u = m.astype(np.float64) / 2 ** 24
        pos = u * np.array([nx - 1, ny - 1, nz - 1])
        want = 0.5 + 0.25 * pos[0] + 0.125 * pos[1] - 0.0625 * pos[2]
        assert abs(orc.volume_trilinear(vol, m) - want) < 1e-12
    # a voxel centre returns the voxel value
    rv = rng.normal(size=(nz, ny, nx)).astype(np.float32)
    for (k, j, i) in [(0, 0, 0), (4, 6, 8), (2, 3, 4)]:
        m = np.array([orc.grid_coord(i, nx), orc.grid_coord(j, ny), orc.grid_coord(k, nz)],
                     dtype=np.uint32)
        if all(int(v) * (n - 1) % (1 << 24) == 0 for v, n in zip(m, (nx, ny, nz))):
            assert orc.volume_trilinear(rv, m) == pytest.approx(float(rv[k, j, i]), abs=1e-12)


def test_grid_coord_closed_form(orc):
    assert orc.grid_coord(0, 9) == 0
    assert orc.grid_coord(8, 9) == 1 << 24
    assert orc.grid_coord(4, 9) == 1 << 23
    assert orc.grid_coord(1, 4) == round((1 << 24) / 3)
    assert orc.grid_coord(0, 1) == 0


def _affine_tables(orc, cfg, coef):
    th = np.zeros(cfg.n_params)
    for l in range(cfg.L):
        if not cfg.dense[l]:
            continue
        N = cfg.N[l]
        for z in range(N + 1):
            for y in range(N + 1):
                for x in range(N + 1):
                    i = orc.corner_index(cfg, l, x, y, z)
                    for f in range(cfg.F):
                        a = coef[f]
                        th[cfg.offset[l] + i * cfg.F + f] = a[0] + (a[1] * x + a[2] * y + a[3] * z) / N
    return th


def test_encoding_reproduces_affine_fields_dense(orc):
    cfg = orc.Config(3, 2, 14, 3, 2.0, 16, 1)  # N = 3, 6, 12 all dense for T = 2^14
    assert all(cfg.dense)
    coef = [(0.1, 0.7, -0.3, 0.2), (-0.4, 0.05, 0.9, -0.6)]
    th = _affine_tables(orc, cfg, coef)
    rng = np.random.default_rng(4)
    m = rng.integers(0, 2 ** 24 + 1, size=(300, 3)).astype(np.uint32)
    x0 = orc.encode(cfg, th, m)
    u = m.astype(np.float64) / 2 ** 24
    for l in range(cfg.L):
        for f in range(2):
            a = coef[f]
            want = a[0] + a[1] * u[:, 0] + a[2] * u[:, 1] + a[3] * u[:, 2]
            np.testing.assert_allclose(x0[:, l * 2 + f], want, atol=1e-12, rtol=0)


def test_encoding_affine_within_a_hashed_cell(orc):
    # On a hashed level the affine identity holds inside any cell whose eight
    # vertices do not collide.
    cfg = orc.Config(1, 2, 8, 20, 1.0, 16, 1)  # N = 20, 9261 vertices > T = 256: hashed
    assert cfg.dense == [0]
    rng = np.random.default_rng(5)
    N = 20
    checked = 0
    for _ in range(50):
        c = rng.integers(0, N, 3)
        verts = [(c[0] + (k & 1), c[1] + ((k >> 1) & 1), c[2] + ((k >> 2) & 1)) for k in range(8)]
        idx = [orc.corner_index(cfg, 0, *v) for v in verts]
        if len(set(idx)) < 8:
            continue
        th = np.zeros(cfg.n_params)
        for v, i in zip(verts, idx):
            th[2 * i] = 0.3 + (0.5 * v[0] - 0.2 * v[1] + 0.1 * v[2]) / N
            th[2 * i + 1] = -1.0 + v[2] / N
        fr = rng.integers(0, 2 ** 24, size=(20, 3))
        m = (((c[None, :].astype(np.int64) << 24) + fr) // N).astype(np.uint32)
        # keep only points that fall inside this cell
        p = m.astype(np.int64) * N
        inside = np.all((p >> 24) == c[None, :], axis=1)
        x0 = orc.encode(cfg, th, m[inside])
        u = m[inside].astype(np.float64) / 2 ** 24
        np.testing.assert_allclose(x0[:, 0], 0.3 + 0.5 * u[:, 0] - 0.2 * u[:, 1] + 0.1 * u[:, 2],
                                   atol=1e-12)
        np.testing.assert_allclose(x0[:, 1], -1.0 + u[:, 2], atol=1e-12)
        checked += 1
    assert checked >= 10


def test_encoding_clamps_u_equal_one(orc):
    # u = 1 uses the last cell with frac = 1 (no out-of-range vertex)
    cfg = orc.Config(2, 1, 12, 4, 2.0, 16, 1)
    coef = [(0.0, 1.0, 2.0, 4.0)]
    th = _affine_tables(orc, cfg, coef)
    x0 = orc.encode(cfg, th, np.array([[1 << 24] * 3], dtype=np.uint32))
    np.testing.assert_allclose(x0[0], [7.0, 7.0], atol=1e-12)


# -------------------------------------------------------------------- MLP ---
def _rand_theta(orc, cfg, seed, table_scale=0.5):
    rng = np.random.default_rng(seed)
    th = orc.init_params(cfg, seed)
    th[: cfg.n_enc] = rng.uniform(-table_scale, table_scale, cfg.n_enc)
    return th


def _mlp_mats(cfg, th):
    mats = []
    for k in range(cfg.n_hidden):
        n_in = cfg.in_dim if k == 0 else cfg.width
        off = cfg.w_off[k]
        mats.append(th[off: off + cfg.width * n_in].reshape(cfg.width, n_in))
    wout = th[cfg.w_off[cfg.n_hidden]: cfg.w_off[cfg.n_hidden] + cfg.width]
    return mats, wout


def test_mlp_positive_network_is_matrix_chain(orc):
    # With non-negative weights and inputs every ReLU is the identity and the
    # network reduces to a chain of matrix products (numpy matmul).
    cfg = orc.Config(4, 2, 12, 4, 1.5, 16, 3)
    rng = np.random.default_rng(6)
    th = np.abs(_rand_theta(orc, cfg, 6))
    m = rng.integers(0, 2 ** 24, size=(64, 3)).astype(np.uint32)
    x0 = orc.encode(cfg, th, m)
    mats, wout = _mlp_mats(cfg, th)
    h = x0.T
    for W in mats:
        h = W @ h
    want = wout @ h
    r = orc.fwd_bwd(cfg, th, m, np.zeros(64), loss=1)
    np.testing.assert_allclose(r["y"], want, rtol=1e-12, atol=1e-14)
    # all-negative first layer: every hidden unit is cut, y = 0
    mats[0][:] = -np.abs(mats[0])
    th2 = th.copy()
    th2[cfg.w_off[0]: cfg.w_off[0] + mats[0].size] = mats[0].ravel()
    r2 = orc.fwd_bwd(cfg, th2, m, np.zeros(64), loss=1)
    assert np.all(r2["y"] == 0.0)


def _loss_only(orc, cfg, th, m, t, loss, n):
    return orc.fwd_bwd(cfg, th, m, t, loss=loss, grad_norm_count=n, want_grads=False)["loss"]


@pytest.mark.parametrize("loss", [1, 0])
def test_gradients_match_finite_differences(orc, loss):
    cfg = orc.Config(3, 2, 8, 3, 2.0, 16, 2)  # small: dense and hashed levels
    th = _rand_theta(orc, cfg, 8)
    rng = np.random.default_rng(9)
    n = 32
    m = rng.integers(0, 2 ** 24, size=(n, 3)).astype(np.uint32)
    t = rng.uniform(0, 1, n)
    # samples within 1e-4 of a ReLU or L1 kink are left out (FD crosses it)
    keep = orc.fwd_bwd(cfg, th, m, t, loss=loss, want_grads=False)["margin"] > 1e-4
    assert keep.sum() >= n // 2
    m, t = m[keep], t[keep]
    r = orc.fwd_bwd(cfg, th, m, t, loss=loss, grad_norm_count=n)
    grad = np.concatenate([r["grad_enc"], r["grad_mlp"]])
    # every MLP parameter and every table entry that some sample touches
    touched = np.nonzero(r["grad_enc"])[0]
    idx = np.concatenate([touched, np.arange(cfg.n_enc, cfg.n_params)])
    h = 1e-6
    fd = np.empty(idx.size)
    for j, p in enumerate(idx):
        a = th.copy(); a[p] += h
        b = th.copy(); b[p] -= h
        fd[j] = (_loss_only(orc, cfg, a, m, t, loss, n) - _loss_only(orc, cfg, b, m, t, loss, n)) / (2 * h)
    err = np.abs(fd - grad[idx])
    assert err.max() <= 1e-7 * max(1.0, np.abs(grad[idx]).max())
    assert np.linalg.norm(fd - grad[idx]) <= 1e-7 * np.linalg.norm(grad[idx])
    # untouched table entries have exactly zero gradient
    assert np.count_nonzero(r["grad_enc"]) == touched.size


def test_dx0_is_gradient_wrt_encoding(orc):
    # dL/dx0 against finite differences through the MLP alone: perturbing a
    # dense level-0 table entry that only one sample touches moves x0 by w.
    cfg = orc.Config(2, 2, 12, 2, 2.0, 16, 2)
    th = _rand_theta(orc, cfg, 10)
    m = np.array([[3 << 22, 5 << 21, 7 << 20]], dtype=np.uint32)
    t = np.array([0.25])
    r = orc.fwd_bwd(cfg, th, m, t, loss=1)
    # the table gradient of a touched entry equals w_corner * dx0 (one sample)
    N = cfg.N[0]
    u = m[0].astype(np.float64) / 2 ** 24 * N
    b = np.floor(u).astype(int)
    f = u - b
    w000 = (1 - f[0]) * (1 - f[1]) * (1 - f[2])
    i000 = orc.corner_index(cfg, 0, *b)
    np.testing.assert_allclose(r["grad_enc"][cfg.offset[0] + 2 * i000: cfg.offset[0] + 2 * i000 + 2],
                               w000 * r["dx0"][0, 0:2], rtol=1e-12)


def test_mixed_mode_scale_invariance_and_error(orc):
    cfg = orc.Config(4, 2, 10, 4, 1.5, 32, 2)
    th = _rand_theta(orc, cfg, 12, table_scale=0.3)
    rng = np.random.default_rng(13)
    m = rng.integers(0, 2 ** 24, size=(128, 3)).astype(np.uint32)
    t = rng.uniform(0, 1, 128)
    a = orc.fwd_bwd(cfg, th, m, t, loss=0, mixed=True, loss_scale=2.0 ** 7)
    b = orc.fwd_bwd(cfg, th, m, t, loss=0, mixed=True, loss_scale=2.0 ** 9)
    # power-of-two loss scales leave the unscaled gradients bit-identical
    np.testing.assert_array_equal(a["grad_mlp"], b["grad_mlp"])
    np.testing.assert_array_equal(a["grad_enc"], b["grad_enc"])
    # and the FP16 emulation stays within a few binary16 ulps of FP64
    f = orc.fwd_bwd(cfg, th, m, t, loss=0, mixed=False)
    np.testing.assert_allclose(a["y"], f["y"], atol=2e-3 * np.abs(f["y"]).max() + 1e-4)
    assert np.linalg.norm(a["grad_mlp"] - f["grad_mlp"]) < 0.05 * np.linalg.norm(f["grad_mlp"])
    # FP16 emulation really rounds: some y differs from FP64
    assert np.any(a["y"] != f["y"])


def test_flip_changes_only_the_flipped_sample(orc):
    cfg = orc.Config(2, 2, 10, 4, 1.5, 16, 2)
    th = _rand_theta(orc, cfg, 14)
    rng = np.random.default_rng(15)
    m = rng.integers(0, 2 ** 24, size=(8, 3)).astype(np.uint32)
    t = rng.uniform(0, 1, 8)
    base = orc.fwd_bwd(cfg, th, m, t, loss=0)
    flip = np.zeros((8, 2 * 16 + 1), np.uint8)
    flip[3, 2 * 16] = 1  # invert the L1 sign of sample 3
    fl = orc.fwd_bwd(cfg, th, m, t, loss=0, flip=flip)
    np.testing.assert_array_equal(fl["dx0"][[0, 1, 2, 4, 5, 6, 7]], base["dx0"][[0, 1, 2, 4, 5, 6, 7]])
    np.testing.assert_allclose(fl["dx0"][3], -base["dx0"][3], rtol=1e-15)
    np.testing.assert_array_equal(fl["y"], base["y"])


# ------------------------------------------------------------------- Adam ---
def test_adam_closed_form_two_steps(orc):
    cfg = orc.Config(1, 1, 4, 1, 1.0, 1, 1)  # 8 table params + 2 weights
    P = cfg.n_params
    lr, b1, b2, eps = 0.01, 0.9, 0.999, 1e-8
    tc = orc.TrainConfig(batch=1, lr=lr, beta1=b1, beta2=b2, eps=eps, weight_decay=0.0)
    st = orc.State()
    th = np.linspace(-1, 1, P)
    th0 = th.copy()
    m1, m2 = np.zeros(P), np.zeros(P)
    g1 = np.linspace(0.5, -0.3, P)
    g2 = np.linspace(-0.2, 0.4, P)
    orc.adam(cfg, tc, st, th, m1, m2, g1)
    np.testing.assert_allclose(th, th0 - lr * g1 / (np.abs(g1) + eps), rtol=1e-14)
    th1 = th.copy()
    orc.adam(cfg, tc, st, th, m1, m2, g2)
    mm = (b1 * (1 - b1) * g1 + (1 - b1) * g2) / (1 - b1 ** 2)
    vv = (b2 * (1 - b2) * g1 ** 2 + (1 - b2) * g2 ** 2) / (1 - b2 ** 2)
    np.testing.assert_allclose(th, th1 - lr * mm / (np.sqrt(vv) + eps), rtol=1e-13)
    assert st.adam_t == 2


def test_adam_weight_decay_and_skip(orc):
    cfg = orc.Config(1, 1, 4, 1, 1.0, 1, 1)
    P = cfg.n_params
    tc = orc.TrainConfig(batch=1, lr=0.1, weight_decay=0.5, mixed=True, growth_interval=2)
    st = orc.State(loss_scale=64.0)
    th = np.full(P, 2.0)
    m1, m2 = np.zeros(P), np.zeros(P)
    orc.adam(cfg, tc, st, th, m1, m2, np.full(P, -1.0))  # g + 0.5*2 = 0 -> no move
    np.testing.assert_allclose(th, 2.0)
    g = np.zeros(P); g[3] = np.nan
    before = th.copy()
    orc.adam(cfg, tc, st, th, m1, m2, g)
    np.testing.assert_array_equal(th, before)
    assert st.skipped == 1 and st.adam_t == 1 and st.loss_scale == 32.0
    orc.adam(cfg, tc, st, th, m1, m2, np.zeros(P))
    orc.adam(cfg, tc, st, th, m1, m2, np.zeros(P))
    assert st.loss_scale == 64.0  # doubled after growth_interval finite steps


# --------------------------------------------------------- decode, render ---
def test_decode_grid_reproduces_affine_network(orc):
    # One hidden unit passes a dense level-0 feature through: y = x0[0],
    # so decoding returns the affine table function at the voxel centres.
    cfg = orc.Config(1, 2, 12, 6, 1.0, 16, 1)
    th = _affine_tables(orc, cfg, [(0.2, 0.5, 0.25, 0.125), (0.0, 0.0, 0.0, 0.0)])
    w0 = np.zeros((16, 2)); w0[0, 0] = 1.0
    th[cfg.w_off[0]: cfg.w_off[0] + 32] = w0.ravel()
    th[cfg.w_off[1]] = 1.0
    dims, ghost = (7, 6, 5), 1
    out = orc.decode_grid(cfg, th, dims, ghost, vmin=-1.0, vmax=3.0)
    for z in range(out.shape[0]):
        for y in range(out.shape[1]):
            for x in range(out.shape[2]):
                u = np.array([orc.grid_coord(x + 1, 7), orc.grid_coord(y + 1, 6),
                              orc.grid_coord(z + 1, 5)]) / 2 ** 24
                yv = 0.2 + 0.5 * u[0] + 0.25 * u[1] + 0.125 * u[2]
                assert out[z, y, x] == pytest.approx(yv * 4.0 - 1.0, abs=1e-12)


def test_render_constant_field_closed_form(orc):
    e = 6
    g = np.full((e, e, e), 0.5)
    tf = [0.2, 0.4, 0.6, 1.0, 0.8, 0.0, 0.05, 0.0, 1.0]
    img = orc.render([g], [(0, 0, 0)], [(e, e, e)], tf, 5, 4, 64)
    a = 0.05 * 0.5
    A = 1 - (1 - a) ** 64
    rgb = np.array([0.6, 0.6, 0.3])
    np.testing.assert_allclose(img[..., 3], A, rtol=1e-12)
    np.testing.assert_allclose(img[..., :3], np.broadcast_to(rgb * A, img[..., :3].shape), rtol=1e-12)


def test_render_front_to_back_order(orc):
    # Two stacked blocks: an opaque-ish front (low z) block hides the back one.
    e = 4
    front = np.full((e, e, e), 1.0)
    back = np.full((e, e, e), 0.0)
    tf = [1.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.5, 0.0, 1.0]
    img = orc.render([back, front], [(0, 0, e), (0, 0, 0)], [(e, e, 2 * e), (e, e, e)], tf, 2, 2, 8)
    # front half: 4 samples of alpha 0.5, back half contributes nothing
    np.testing.assert_allclose(img[..., 3], 1 - 0.5 ** 4, rtol=1e-12)
    np.testing.assert_allclose(img[..., 0], 1 - 0.5 ** 4, rtol=1e-12)


def test_mse_closed_form(orc):
    a = np.array([1.0, 2.0, 3.0, 4.0])
    b = np.array([1.0, 2.5, 2.0, 4.0], dtype=np.float32)
    v, mx = orc.mse(a, b)
    assert v == pytest.approx((0.25 + 1.0) / 4) and mx == 1.0


# ---------------------------------------------------------------- training ---
def test_training_reduces_error(orc):
    from paper_2304_10516_gb300 import volumes

    vol = volumes.blobs(24, seed=1001)
    cfg = orc.Config(4, 2, 12, 4, 1.5, 16, 2)
    th = orc.init_params(cfg, 1)
    m1, m2 = np.zeros_like(th), np.zeros_like(th)
    tc = orc.TrainConfig(batch=512, lr=1e-2, seed=3)
    st = orc.State()
    dec0 = orc.decode_grid(cfg, th, vol.shape[::-1], 0, float(vol.min()), float(vol.max()))
    hist = orc.train(cfg, tc, st, th, m1, m2, vol, float(vol.min()), float(vol.max()), 150)
    dec = orc.decode_grid(cfg, th, vol.shape[::-1], 0, float(vol.min()), float(vol.max()))
    e0, _ = orc.mse(dec0, vol)
    e1, _ = orc.mse(dec, vol)
    assert st.adam_t == 150 and st.iter == 150
    assert hist[-10:].mean() < 0.5 * hist[:10].mean()
    assert e1 < 0.1 * e0


# ------------------------------------------- iteration budget, early stop ----
def test_max_iterations_counts_batches_by_brute_force(orc):
    # Sec. 3.2: N_train^max = max(N_min, ceil(N_vox / N_batch) N_epoch); the
    # batch count is checked by covering the voxels one batch at a time
    for n_vox in (1, 4095, 4096, 4097, 64 ** 3, 96 * 97 * 98, 160 ** 3):
        for batch in (1, 4096, 16384):
            k, covered = 0, 0
            while covered < n_vox:
                covered += batch
                k += 1
            for epochs in (1, 16):
                assert orc.max_iterations(n_vox, batch, epochs=epochs) == k * epochs
                assert orc.max_iterations(n_vox, batch, epochs=epochs, min_steps=k * epochs + 7) \
                    == k * epochs + 7
    # the 64^3 workload at batch 4096 and 16 epochs: 64 batches per epoch
    assert orc.max_iterations(64 ** 3, 4096, epochs=16) == 1024
    # epochs = 0 keeps the fixed count, still raised to N_min
    assert orc.max_iterations(10 ** 6, 4096, steps=300) == 300
    assert orc.max_iterations(10 ** 6, 4096, steps=300, min_steps=500) == 500
    assert orc.max_iterations(10 ** 6, 4096, steps=0) == 0


def test_stop_rule_matches_geometric_closed_form(orc):
    # losses L_t = r^t (t = 1, 2, ...): the moving average m_1 = L_1,
    # m_t = d m_{t-1} + (1 - d) L_t has the closed form
    # m_t = d^(t-1) r + (1 - d) r^t (1 - (d/r)^(t-1)) / (1 - d/r)
    r, d = 0.97, 0.9
    n = 400
    L = r ** np.arange(1, n + 1, dtype=np.float64)

    def closed(t):
        q = d / r
        return d ** (t - 1) * r + (1 - d) * r ** t * (1 - q ** (t - 1)) / (1 - q)

    for t in (1, 2, 5, 50, 400):
        steps, ema = orc.stop_step(L[:t], d, 0.0)
        assert steps == t
        assert abs(ema - closed(t)) <= 1e-12 * closed(t)
    # the first t with m_t below a threshold between two consecutive values
    thr = 0.5 * (closed(120) + closed(121))
    steps, ema = orc.stop_step(L, d, thr)
    assert steps == 121 and abs(ema - closed(121)) <= 1e-12
    # no threshold: the whole sequence; threshold above L_1: stop after step 1
    assert orc.stop_step(L, d, 0.0)[0] == n
    assert orc.stop_step(L, d, 1.0)[0] == 1


def test_stop_rule_skips_nonfinite_steps(orc):
    # a skipped (non-finite) step counts against the budget but leaves the
    # average as it was: the average of the finite steps alone, one step later
    L = np.array([1.0, np.inf, 0.5, np.nan, 0.2, 0.1])
    fin = np.array([1, 0, 1, 0, 1, 1], dtype=np.int32)
    d = 0.5
    steps, ema = orc.stop_step(L, d, 0.0, finite=fin)
    m = 1.0
    for x in (0.5, 0.2, 0.1):
        m = d * m + (1 - d) * x
    assert steps == 6 and ema == pytest.approx(m, rel=1e-15)
    # threshold crossed at the 5th step (m = 0.45 after 0.2)
    steps, _ = orc.stop_step(L, d, 0.5, finite=fin)
    assert steps == 5
    # an all-skipped call has no average
    assert orc.stop_step(L[1:2], d, 0.3, finite=fin[1:2]) == (1, -1.0)


def test_train_budget_is_train_stopped_at_the_rule(orc):
    # training under a budget is plain training of the same number of steps,
    # and with a threshold it stops where the rule applied to the full loss
    # history says
    from paper_2304_10516_gb300 import volumes

    vol = volumes.blobs(16, seed=1001)
    cfg = orc.Config(4, 2, 10, 4, 1.5, 16, 2)
    vmin, vmax = float(vol.min()), float(vol.max())
    tc = orc.TrainConfig(batch=256, lr=1e-2, seed=5)

    def fresh():
        th = orc.init_params(cfg, 2)
        return th, np.zeros_like(th), np.zeros_like(th), orc.State()

    th, m1, m2, st = fresh()
    full = orc.train(cfg, tc, st, th, m1, m2, vol, vmin, vmax, 60)
    th_b, m1_b, m2_b, st_b = fresh()
    n, hist, _, stopped = orc.train_budget(cfg, tc, st_b, th_b, m1_b, m2_b, vol, vmin, vmax, 60)
    assert n == 60 and not stopped and st_b.iter == 60
    # (the oracle's threaded loss sum may round differently in the last bit)
    np.testing.assert_allclose(hist, full, rtol=1e-12, atol=0)
    np.testing.assert_allclose(th_b, th, rtol=1e-9, atol=1e-15)
    thr = float(np.median(full))
    want, want_ema = orc.stop_step(full, 0.9, thr)
    assert want < 60
    th_s, m1_s, m2_s, st_s = fresh()
    n, hist, ema, stopped = orc.train_budget(cfg, tc, st_s, th_s, m1_s, m2_s, vol, vmin, vmax, 60,
                                             stop_loss=thr, decay=0.9)
    assert stopped and n == want and st_s.iter == want
    assert ema == pytest.approx(want_ema, rel=1e-12)
    th_r, m1_r, m2_r, st_r = fresh()
    orc.train(cfg, tc, st_r, th_r, m1_r, m2_r, vol, vmin, vmax, want)
    np.testing.assert_allclose(th_s, th_r, rtol=1e-9, atol=1e-15)


# ------------------------------------------------- direct INR ray-marching ----
def _zero_net(cfg):
    return np.zeros(cfg.n_params)


def test_render_inr_constant_network_closed_form(orc):
    # an all-zero network outputs 0, so every sample decodes to vmin: alpha and
    # colour are the same along every ray, A = 1 - (1 - a)^spr, C = rgb A
    cfg = orc.Config(2, 2, 10, 4, 1.5, 16, 1)
    tf = [0.2, 0.4, 0.6, 1.0, 0.8, 0.0, 0.05, 0.0, 1.0]
    img = orc.render_inr(cfg, [_zero_net(cfg)], [(2, 3, 1)], [(8, 9, 7)], 1, 0.5, 1.5, tf, 5, 4, 64)
    a = 0.05 * 0.5
    A = 1 - (1 - a) ** 64
    np.testing.assert_allclose(img[..., 3], A, rtol=1e-12)
    np.testing.assert_allclose(img[..., :3], np.broadcast_to(np.array([0.6, 0.6, 0.3]) * A,
                                                             img[..., :3].shape), rtol=1e-12)
    # a listed subset of pixels gives the same rows
    sub = orc.render_inr(cfg, [_zero_net(cfg)], [(2, 3, 1)], [(8, 9, 7)], 1, 0.5, 1.5, tf, 5, 4, 64,
                         pixels=[3, 17, 0])
    np.testing.assert_array_equal(sub, img.reshape(-1, 4)[[3, 17, 0]])


def test_render_inr_front_to_back_two_blocks(orc):
    # stacked blocks [0,4)^2 x [0,4) (front) and [0,4)^2 x [4,8) (back) with
    # constant values 1 and 0.5; spr = 8 puts samples at z = 0..7, four in
    # each. Input order must not matter (depth order is by position).
    cfg = orc.Config(2, 2, 10, 4, 1.5, 16, 1)
    tf = [1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.5, 0.0, 1.0]
    z = _zero_net(cfg)
    args = ([(0, 0, 4), (0, 0, 0)], [(4, 4, 8), (4, 4, 4)], 1, [0.5, 1.0], [2.0, 2.0], tf, 2, 2, 8)
    img = orc.render_inr(cfg, [z, z], *args)
    a1, a2 = 0.5 * 1.0, 0.5 * 0.5
    rgb1, rgb2 = np.array([0.0, 1.0, 0.0]), np.array([0.5, 0.5, 0.0])
    A1 = 1 - (1 - a1) ** 4
    A = 1 - (1 - a1) ** 4 * (1 - a2) ** 4
    C = rgb1 * A1 + (1 - a1) ** 4 * rgb2 * (1 - (1 - a2) ** 4)
    np.testing.assert_allclose(img[..., 3], A, rtol=1e-12)
    np.testing.assert_allclose(img[..., :3], np.broadcast_to(C, img[..., :3].shape), rtol=1e-12)
    swapped = orc.render_inr(cfg, [z, z], [(0, 0, 0), (0, 0, 4)], [(4, 4, 4), (4, 4, 8)], 1,
                             [1.0, 0.5], [2.0, 2.0], tf, 2, 2, 8)
    np.testing.assert_allclose(swapped, img, rtol=1e-15)


def test_render_inr_equals_grid_march_for_a_network_affine_in_x(orc):
    # y = 0.2 + 0.5 u_x (one dense level with affine tables, one hidden unit
    # passing feature 0 through): the network is affine along x and constant
    # in y and z, so marching it equals marching its decoded grid wherever
    # the grid march interpolates (ray centres between the first and the
    # last voxel centre in x). Checks the position -> unit-domain mapping
    # (origin lo - ghost, stored extent), samples and compositing at once.
    cfg = orc.Config(1, 2, 12, 6, 1.0, 16, 1)
    th = _affine_tables(orc, cfg, [(0.2, 0.5, 0.0, 0.0), (0.0, 0.0, 0.0, 0.0)])
    w0 = np.zeros((16, 2))
    w0[0, 0] = 1.0
    th[cfg.w_off[0]: cfg.w_off[0] + 32] = w0.ravel()
    th[cfg.w_off[1]] = 1.0
    lo, hi, ghost = (3, 1, 2), (13, 7, 10), 2
    dims = [h - l + 2 * ghost for l, h in zip(lo, hi)]
    vmin, vmax = -1.0, 3.0
    grid = orc.decode_grid(cfg, th, dims, ghost, vmin, vmax)
    tf = [0.1, 0.2, 0.6, 1.0, 0.9, 0.2, 0.08, -1.0, 3.0]
    w, h, spr = 40, 6, 50
    inr = orc.render_inr(cfg, [th], [lo], [hi], ghost, vmin, vmax, tf, w, h, spr)
    ref = orc.render([grid], [lo], [hi], tf, w, h, spr)
    X = lo[0] - 0.5 + (np.arange(w) + 0.5) * (hi[0] - lo[0]) / w
    inside = (X >= lo[0]) & (X <= hi[0] - 1)
    assert inside.sum() >= 30 and (~inside).sum() >= 4
    np.testing.assert_allclose(inr[:, inside], ref[:, inside], atol=1e-7, rtol=0)
    # outside that span the grid march clamps to the edge voxel while the
    # network keeps its slope: the images differ there
    assert np.abs(inr[:, ~inside] - ref[:, ~inside]).max() > 1e-4


# ------------------------------------------------- adaptive T and R_0 ----
def test_adaptive_encoding_closed_forms(orc):
    # T_ref N_vox / N_global rounded up to a power of two, floored at T_min;
    # R_0 = floor(R_ref cbrt(T / T_ref)), checked with exact fractions
    Tref, Tmin, Rref = 19, 12, 16
    cases = [
        (512 ** 3, 512 ** 3, 19, 16),                 # one partition: T = T_ref, R_0 = R_ref
        (256 ** 3, 512 ** 3, 16, 8),                  # an eighth: T_ref / 8, R_0 = R_ref / 2
        (128 ** 3, 512 ** 3, 13, 4),                  # 1/64: T_ref / 64, R_0 = R_ref / 4
        (64 ** 3, 512 ** 3, 12, 3),                   # 1/512 -> 2^10, floored at T_min = 2^12
        (96 * 130 * 150, 512 ** 3, 13, 4),            # 2^19 / 71.7 = 7312 -> 2^13; 16 cbrt(1/64) = 4
        (2 ** 27 + 1, 2 ** 30, 17, 10),               # just above 1/8 of 2^30 -> 2^17; 16 cbrt(1/4)
    ]
    for n_vox, n_glob, want_T, want_R in cases:
        assert orc.adaptive_encoding(n_vox, n_glob, Tref, Tmin, Rref) == (want_T, want_R)
    # the general case against exact rational arithmetic
    rng = np.random.default_rng(7)
    for _ in range(200):
        n_glob = int(rng.integers(10 ** 6, 10 ** 9))
        n_vox = int(rng.integers(1, n_glob + 1))
        lt, r0 = orc.adaptive_encoding(n_vox, n_glob, Tref, Tmin, Rref)
        share = Fraction(2 ** Tref * n_vox, n_glob)
        k = 0
        while Fraction(2 ** k) < share:
            k += 1
        k = max(k, Tmin)
        assert lt == k
        ratio = Fraction(2 ** k, 2 ** Tref)
        R = 1
        while Fraction((R + 1) ** 3) <= Rref ** 3 * ratio:
            R += 1
        assert r0 == R, (n_vox, n_glob, k, r0, R)
