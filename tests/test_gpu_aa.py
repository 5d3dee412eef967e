"""A-A streaming (one population array updated in place, the pattern Sec. 3
says the paper uses): every observable equals that of the A-B path bit for
bit -- meshed blocks, fields, mass and the populations left by the last
step -- with bounce-back, periodic wrap, held cells, block creation in both
kinds of step and a static mesh, in the stream and graph execution modes;
and the pool holds one population array instead of two."""
import numpy as np
import pytest

from gpu_helpers import compare_active, compare_fields, oracle_of
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


def _porous(progressive=1):
    return W.porous_injection(n=(56, 40, 48), seed=1510035603, inlet=16, x_free=6,
                              r_range=(3.0, 6.0), S=1e-4, progressive=progressive)


CASES = {
    "drop": lambda: W.drop_in_box(),
    "porous": lambda: _porous(),
    "porous_static": lambda: _porous(progressive=0),
    "impact": lambda: W.droplet_impact(n=(48, 32, 40), seed=1510035701),
}
# odd chunks put either kind of step last
CHUNKS = (1, 1, 2, 5, 11, 20)


def _populations(sim, ids):
    return [sim.block_populations(int(b)) for b in ids]


def _compare(ab, aa, case):
    np.testing.assert_array_equal(ab.active_blocks(), aa.active_blocks())
    for a in range(case["params"]["ncomp"]):
        for x, y in zip(ab.macro(a), aa.macro(a)):
            np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(ab.mass(), aa.mass())
    ids = ab.active_blocks()
    pick = ids[np.linspace(0, len(ids) - 1, min(len(ids), 6)).astype(int)]
    ct = case["cell_type"]
    nz, ny, nx = ct.shape
    nbx, nby = nx // 8, ny // 8
    for b, fa, fb in zip(pick, _populations(ab, pick), _populations(aa, pick)):
        bx, by, bz = b % nbx, (b // nbx) % nby, b // (nbx * nby)
        blk = ct[bz * 8:bz * 8 + 8, by * 8:by * 8 + 8, bx * 8:bx * 8 + 8].reshape(-1)
        keep = blk != W.SOLID  # solid cells' stored values are never read
        np.testing.assert_array_equal(fa[..., keep], fb[..., keep])


@pytest.mark.parametrize("which", sorted(CASES))
def test_aa_equals_ab_bit_for_bit(L, which):
    case = CASES[which]()
    ab = L.from_case(case, partials=False)  # A-A pulls in every pass 1
    aa = L.from_case(case, streaming="aa")
    _compare(ab, aa, case)  # the initial layout
    for n in CHUNKS:
        ab.step(n)
        aa.step(n)
        _compare(ab, aa, case)
    sa, sb = ab.stats(), aa.stats()
    assert sa["created_blocks"] == sb["created_blocks"]
    if case["params"].get("progressive", 1):
        assert sb["created_blocks"] > 0
    print(f"A-A {which}: {sum(CHUNKS)} steps, {len(aa.active_blocks())} meshed blocks, "
          f"created {sb['created_blocks']}")
    ab.close()
    aa.close()


def test_aa_graph_mode_equals_stream(L):
    case = _porous()
    runs = []
    for mode in ("stream", "graph"):
        sim = L.from_case(case, streaming="aa")
        sim.set_exec(mode)
        for n in (3, 4, 7, 2):
            sim.step(n)
        runs.append((sim.active_blocks(), [sim.macro(a) for a in range(2)], sim.mass()))
        sim.close()
    np.testing.assert_array_equal(runs[0][0], runs[1][0])
    for a in range(2):
        for x, y in zip(runs[0][1][a], runs[1][1][a]):
            np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(runs[0][2], runs[1][2])


def test_aa_matches_oracle(L):
    """The drop in a box against the FP64 oracle step by step (meshed
    blocks) and after 200 steps (fields, mass), with the A-B path's bounds."""
    case = W.drop_in_box()
    gpu = L.from_case(case, streaming="aa")
    orc = oracle_of(case)
    for t in range(200):
        gpu.step(1)
        orc.step(1)
        compare_active(gpu, orc, t, case["params"]["S"])
    compare_fields(gpu, orc, case, label="A-A drop")
    np.testing.assert_allclose(gpu.mass(), orc.mass(), rtol=1e-6)
    gpu.close()


def test_aa_halves_population_memory_and_refuses_other_modes(L):
    case = _porous()
    ab = L.from_case(case)
    aa = L.from_case(case, streaming="aa")
    st = ab.stats()
    slot_bytes = 2 * 19 * 512 * 4
    one_array = (st["capacity"] + 1) * slot_bytes
    # A-A adds the constant populations of the blocks holding held cells
    ct = case["cell_type"]
    nz, ny, nx = ct.shape
    held_blocks = int((ct == W.HELD).reshape(nz // 8, 8, ny // 8, 8, nx // 8, 8).any(axis=(1, 3, 5)).sum())
    extra = held_blocks * slot_bytes + st["total_blocks"] * 4
    saved = st["device_bytes"] - aa.stats()["device_bytes"]
    print(f"A-A memory: {aa.stats()['device_bytes'] / 2**20:.1f} MiB against "
          f"{st['device_bytes'] / 2**20:.1f} MiB ({held_blocks} blocks with held cells)")
    assert one_array - extra - (1 << 20) <= saved <= one_array, (saved, one_array, extra)
    for mode in ("persistent", "staged"):
        with pytest.raises(L.LBMError) as e:
            aa.set_exec(mode)
        assert e.value.code == L.EINVAL
    ab.close()
    aa.close()


def test_aa_pool_exhaustion_keeps_last_complete_step(L):
    """A pool too small for the blocks a step creates: LBM_ENOMEM, and the
    in-place array still holds the last completed step (the failing step's
    collision never ran), equal to the A-B run stopped there."""
    case = W.drop_in_box()
    small = L.from_case(case, streaming="aa", max_blocks=12)
    ref = L.from_case(case, partials=False)
    failed_at = None
    for t in range(40):
        try:
            small.step(1)
        except L.LBMError as e:
            assert e.code == L.ENOMEM
            failed_at = t
            break
        ref.step(1)
    assert failed_at is not None
    assert small.stats()["steps"] == failed_at
    for a in range(2):
        for x, y in zip(small.macro(a), ref.macro(a)):
            np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(small.mass(), ref.mass())
    with pytest.raises(L.LBMError):
        small.step(1)
    small.close()
    ref.close()
