"""Host side of the batching form: the seeded batch workload and the packing
of many simulations into one walled grid (no GPU)."""
import numpy as np

from paper_1510_03560_gb300 import batch as B
from paper_1510_03560_gb300 import workloads as W


def test_batch_workload_is_seeded_and_in_range():
    a = B.c3_cases(6)
    b = B.c3_cases(6)
    for x, y in zip(a, b):
        assert x["kind"] == y["kind"]
        np.testing.assert_array_equal(x["cell_type"], y["cell_type"])
        np.testing.assert_array_equal(x["rho_init"], y["rho_init"])
        for k in ("nx", "ny", "nz"):
            assert x["params"][k] in B.SIZES
    assert {c["kind"] for c in B.c3_cases(16)} == {"impact", "injection"}


def _small():
    return [W.droplet_impact(n=(32, 48, 32), seed=1), W.porous_injection(n=(48, 32, 32), seed=2, inlet=8, x_free=4),
            W.droplet_impact(n=(32, 32, 48), seed=3), W.porous_injection(n=(32, 32, 32), seed=4, inlet=8, x_free=4)]


def test_packing_places_each_simulation_walled_and_apart():
    cases = _small()
    batch, place = B.pack(cases, width=96)
    ct = batch["cell_type"]
    covered = np.zeros(ct.shape, dtype=bool)
    for c, (x0, y0, z0, nx, ny, nz) in zip(cases, place):
        assert x0 % 8 == y0 % 8 == z0 % 8 == 0
        sl = (slice(z0, z0 + nz), slice(y0, y0 + ny), slice(x0, x0 + nx))
        np.testing.assert_array_equal(ct[sl], c["cell_type"])
        np.testing.assert_array_equal(batch["rho_init"][(slice(None),) + sl], c["rho_init"])
        assert not covered[sl].any()
        covered[sl] = True
    assert np.all(ct[~covered] == W.SOLID)
    assert batch["params"]["max_blocks"] == sum(B.nonsolid_blocks(c["cell_type"]) for c in cases)
    # no non-solid block of one simulation touches (26-neighbourhood) a
    # non-solid block of another: creation can never cross between them
    nz, ny, nx = ct.shape
    owner = -np.ones((nz // 8, ny // 8, nx // 8), dtype=int)
    for k, (x0, y0, z0, sx, sy, sz) in enumerate(place):
        blk = (cases[k]["cell_type"] != W.SOLID).reshape(sz // 8, 8, sy // 8, 8, sx // 8, 8).any(axis=(1, 3, 5))
        owner[z0 // 8:(z0 + sz) // 8, y0 // 8:(y0 + sy) // 8, x0 // 8:(x0 + sx) // 8][blk] = k
    idx = np.argwhere(owner >= 0)
    for z, y, x in idx:
        nb = owner[max(z - 1, 0):z + 2, max(y - 1, 0):y + 2, max(x - 1, 0):x + 2]
        assert set(nb[nb >= 0].tolist()) == {owner[z, y, x]}


def test_split_and_block_map_invert_the_packing():
    cases = _small()
    batch, place = B.pack(cases)
    for c, part in zip(cases, B.split(batch["rho_init"], place)):
        np.testing.assert_array_equal(part, c["rho_init"])
    p = batch["params"]
    nbx, nby = p["nx"] // 8, p["ny"] // 8
    for k, (x0, y0, z0, nx, ny, nz) in enumerate(place):
        ids = B.block_map(p, place, k)
        assert ids.shape == (nz // 8, ny // 8, nx // 8)
        bx, by, bz = ids % nbx, (ids // nbx) % nby, ids // (nbx * nby)
        assert bx.min() == x0 // 8 and by.min() == y0 // 8 and bz.min() == z0 // 8


def test_packing_rejects_mixed_physics():
    a = W.droplet_impact(n=(32, 32, 32), seed=1)
    b = W.droplet_impact(n=(32, 32, 32), seed=2, g_ads=-0.1)
    try:
        B.pack([a, b])
    except ValueError as e:
        assert "g_ads" in str(e)
    else:
        raise AssertionError("mixed physics accepted")
