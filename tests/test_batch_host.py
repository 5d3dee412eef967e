"""Host side of the batching form: the seeded batch workload and the packing
of many simulations into one walled grid (no GPU)."""
import numpy as np
import pytest

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


SHAPES = [(8, 8, 8), (16, 8, 4), (16, 4, 8)]


@pytest.mark.parametrize("block", SHAPES)
def test_packing_places_each_simulation_walled_and_apart(block):
    bx, by, bz = block
    cases = _small()
    batch, place = B.pack(cases, width=96, block=block)
    assert tuple(batch["params"]["block"]) == block
    ct = batch["cell_type"]
    covered = np.zeros(ct.shape, dtype=bool)
    for c, (x0, y0, z0, nx, ny, nz) in zip(cases, place):
        assert x0 % bx == y0 % by == z0 % bz == 0
        sl = (slice(z0, z0 + nz), slice(y0, y0 + ny), slice(x0, x0 + nx))
        np.testing.assert_array_equal(ct[sl], c["cell_type"])
        np.testing.assert_array_equal(batch["rho_init"][(slice(None),) + sl], c["rho_init"])
        assert not covered[sl].any()
        covered[sl] = True
    assert np.all(ct[~covered] == W.SOLID)
    assert batch["params"]["max_blocks"] == sum(B.nonsolid_blocks(c["cell_type"], block) for c in cases)
    # no non-solid block of one simulation touches (26-neighbourhood) a
    # non-solid block of another: creation can never cross between them
    nz, ny, nx = ct.shape
    owner = -np.ones((nz // bz, ny // by, nx // bx), dtype=int)
    for k, (x0, y0, z0, sx, sy, sz) in enumerate(place):
        blk = (cases[k]["cell_type"] != W.SOLID).reshape(sz // bz, bz, sy // by, by, sx // bx, bx).any(axis=(1, 3, 5))
        owner[z0 // bz:(z0 + sz) // bz, y0 // by:(y0 + sy) // by, x0 // bx:(x0 + sx) // bx][blk] = k
    idx = np.argwhere(owner >= 0)
    for z, y, x in idx:
        nb = owner[max(z - 1, 0):z + 2, max(y - 1, 0):y + 2, max(x - 1, 0):x + 2]
        assert set(nb[nb >= 0].tolist()) == {owner[z, y, x]}


@pytest.mark.parametrize("block", SHAPES)
def test_split_and_block_map_invert_the_packing(block):
    bx, by, bz = block
    cases = _small()
    batch, place = B.pack(cases, block=block)
    for c, part in zip(cases, B.split(batch["rho_init"], place)):
        np.testing.assert_array_equal(part, c["rho_init"])
    p = batch["params"]
    nbx, nby = p["nx"] // bx, p["ny"] // by
    for k, (x0, y0, z0, nx, ny, nz) in enumerate(place):
        ids = B.block_map(p, place, k)
        assert ids.shape == (nz // bz, ny // by, nx // bx)
        ix, iy, iz = ids % nbx, (ids // nbx) % nby, ids // (nbx * nby)
        assert ix.min() == x0 // bx and iy.min() == y0 // by and iz.min() == z0 // bz


def test_packing_needs_members_tiled_by_the_block():
    cases = _small()  # x sizes 32 and 48: not all multiples of 32
    assert not B.tiles(cases, (32, 4, 4)) and B.tiles(cases, (16, 8, 4))
    with pytest.raises(ValueError):
        B.pack(cases, block=(32, 4, 4))


def test_packing_rejects_mixed_physics():
    a = W.droplet_impact(n=(32, 32, 32), seed=1)
    b = W.droplet_impact(n=(32, 32, 32), seed=2, g_ads=-0.1)
    try:
        B.pack([a, b])
    except ValueError as e:
        assert "g_ads" in str(e)
    else:
        raise AssertionError("mixed physics accepted")
