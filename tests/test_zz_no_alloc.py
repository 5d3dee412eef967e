"""lbm_mass_noalloc: the mass reduction for callers that cannot allocate
device memory (their GPU memory belongs to another allocator, or they must
not allocate after start-up).  Called through the C ABI on a population pool
the test holds in device memory, it must agree with lbm_mass on the same
state, on two calls in a row.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_1510_03560_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    from paper_1510_03560_gb300 import build as B
    B.build()
    from paper_1510_03560_gb300 import lbm
    assert torch.cuda.is_available()
    return lbm


def solid_bits(cell_type, block_ids):
    nz, ny, nx = cell_type.shape
    nbx, nby = nx // 8, ny // 8
    out = np.zeros((len(block_ids), 16), dtype=np.uint32)
    for r, b in enumerate(block_ids):
        bx, by, bz = b % nbx, (b // nbx) % nby, b // (nbx * nby)
        blk = cell_type[bz * 8:(bz + 1) * 8, by * 8:(by + 1) * 8, bx * 8:(bx + 1) * 8]
        flat = (blk == 1).reshape(-1)  # cell index x + 8 (y + 8 z)
        for c in np.nonzero(flat)[0]:
            out[r, c // 32] |= np.uint32(1) << np.uint32(c % 32)
    return out


@pytest.mark.parametrize("which", ["drop", "porous"])
def test_noalloc_mass_matches_lbm_mass(L, which):
    import torch
    if which == "drop":
        case = W.drop_in_box(progressive=0)
    else:
        case = W.porous_injection(n=(56, 40, 48), seed=1510035603, inlet=16, x_free=6,
                                  r_range=(3.0, 6.0), S=1e-4, progressive=0)
    sim = L.from_case(case)
    sim.step(25)
    want = sim.mass()
    ids = sim.active_blocks()
    pops = np.stack([sim.block_populations(int(b)) for b in ids])  # [n][ncomp][19][512]
    f = torch.from_numpy(pops).cuda()
    solid = torch.from_numpy(solid_bits(case["cell_type"], ids).view(np.int32)).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    first = L.mass_noalloc(f.data_ptr(), solid.data_ptr(), len(ids), sim.ncomp, stream)
    second = L.mass_noalloc(f.data_ptr(), solid.data_ptr(), len(ids), sim.ncomp, stream)
    np.testing.assert_allclose(first, want, rtol=1e-6)
    np.testing.assert_allclose(second, want, rtol=1e-6)
    np.testing.assert_array_equal(first, second)
    if len(ids) == sim.nblocks:
        # every block of the grid, in block order: the same sums in the same
        # order as lbm_mass, bit for bit
        np.testing.assert_array_equal(first, want)
    sim.close()


def test_noalloc_rejects_oversized_pool(L):
    import torch
    f = torch.zeros(16, device="cuda")
    with pytest.raises(L.LBMError) as e:
        L.mass_noalloc(f.data_ptr(), None, L.NOALLOC_MAX_BLOCKS + 1, 2)
    assert e.value.code == L.EINVAL
    assert "nblocks" in str(e.value)
