"""The appendix's configuration keys mapped onto the library's encoding, MLP
and training settings (paper_2304_10516_gb300.config), on the appendix's own
listings (tests/golden/appendix_configs.json). Host logic only."""
import json
import math
import os

import pytest

from paper_2304_10516_gb300 import config as PC

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "appendix_configs.json")))


def test_icbrt_is_the_integer_cube_root():
    for k in range(0, 40):
        n = 1 << k
        r = PC.icbrt(n)
        assert r ** 3 <= n < (r + 1) ** 3, k
    for n in (0, 1, 7, 8, 26, 27, 28, 999, 1000, 1001):
        r = PC.icbrt(n)
        assert r ** 3 <= n < (r + 1) ** 3, n


def test_insitu_nekrs_listing():
    c = PC.PaperConfig.from_dict(GOLD["insitu"]["NekRS"])
    enc = c.encoding()
    assert (enc.n_levels, enc.n_features, enc.log2_T, enc.base_res, enc.growth) == (5, 4, 12, 16, 2.0)
    mlp = c.mlp()
    assert (mlp.width, mlp.n_hidden) == (16, 3)
    t = c.train(batch=1 << 16)
    assert (t.lr, t.epochs, t.stop_loss, t.batch) == (0.001, 4, 0.0105, 1 << 16)
    assert c.ignored == {"zfp_mlp": 0.005, "zfp_enc": 0.010}
    # 5 levels x 4 features = 20: the FP16 path takes it padded to 32
    assert enc.n_levels * enc.n_features == 20


def test_insitu_s3d_listing():
    enc = PC.PaperConfig.from_dict(GOLD["insitu"]["S3D"]).encoding()
    assert (enc.n_levels, enc.n_features, enc.log2_T, enc.base_res) == (4, 4, 11, 12)  # cbrt(2048) = 12.7


@pytest.mark.parametrize("share,log2_T,base", [(1, 13, 20), (8, 10, 10), (64, 9, 8), (4096, 9, 8)])
def test_scaling_s3d_table_range(share, log2_T, base):
    # a partition with 1/share of the domain's voxels: T = max(2^9, 2^ceil(log2(2^13 / share)))
    # and the cbrt rule for its base resolution
    c = PC.PaperConfig.from_dict(GOLD["scaling"]["S3D"])
    n_global = 324 * 320 * 240
    enc = c.encoding(n_global // share, n_global)
    assert enc.log2_T == max(9, math.ceil(math.log2(2 ** 13 * (n_global // share) / n_global)))
    assert (enc.log2_T, enc.base_res) == (log2_T, base)


def test_scaling_cloverleaf_fixed_base_and_range():
    c = PC.PaperConfig.from_dict(GOLD["scaling"]["CloverLeaf"])
    for share in (1, 2, 16, 1 << 12):
        enc = c.encoding((1 << 24) // share, 1 << 24)
        assert enc.base_res == 8 and 8 <= enc.log2_T <= 16
    assert c.encoding(1 << 24, 1 << 24).log2_T == 16
    assert c.encoding(1, 1 << 24).log2_T == 8


def test_every_listing_parses_and_fits_the_fp16_kernels():
    for group in ("scaling", "insitu"):
        for name, d in GOLD[group].items():
            c = PC.PaperConfig.from_dict(d)
            D = c.n_levels * c.n_features_per_level
            assert D <= 64 and c.n_features_per_level in (1, 2, 4, 8) and c.n_neurons in (16, 32, 64), name


def test_rejected_settings():
    base = dict(GOLD["insitu"]["NekRS"])
    with pytest.raises(ValueError):
        PC.PaperConfig.from_dict(dict(base, lrate_decay=0.5))
    with pytest.raises(ValueError):
        PC.PaperConfig.from_dict(dict(base, optimizer="sgd"))
    with pytest.raises(ValueError):
        PC.PaperConfig.from_dict(dict(base, log2_hashmap_size=[16, 8]))
    with pytest.raises(ValueError):
        PC.PaperConfig.from_dict(GOLD["scaling"]["S3D"]).encoding()
