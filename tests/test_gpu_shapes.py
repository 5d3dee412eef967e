"""Block shapes other than 8^3 (lbm_params.block: 16x8x4, 16x4x8, 32x4x4):
the same method on another sub-domain shape (Sec. 4.1), checked against
the FP64 oracle run with the same blocks (meshed blocks at every step,
fields, mass), with held cells and a single-block periodic axis; A-A
streaming, the execution modes and batching agree bit for bit within a
shape; the shape autotuner times every shape that tiles a batch."""
import numpy as np
import pytest

from gpu_helpers import compare_active, compare_fields, oracle_of
from paper_1510_03560_gb300 import batch as B
from paper_1510_03560_gb300 import workloads as W

pytestmark = pytest.mark.gpu

OTHER = [(16, 8, 4), (16, 4, 8), (32, 4, 4)]


@pytest.fixture(scope="module")
def L():
    import torch
    from paper_1510_03560_gb300 import build as Bld
    Bld.build()
    from paper_1510_03560_gb300 import lbm
    assert torch.cuda.is_available()
    return lbm


def _pair(L, case, steps):
    gpu = L.from_case(case)
    assert gpu.block == tuple(case["params"]["block"])
    orc = oracle_of(case)
    S = case["params"]["S"]
    counts = [compare_active(gpu, orc, -1, S)]
    for t in range(steps):
        gpu.step(1)
        orc.step(1)
        counts.append(compare_active(gpu, orc, t, S))
    compare_fields(gpu, orc, case, label=str(case["params"]["block"]))
    np.testing.assert_allclose(gpu.mass(), orc.mass(), rtol=1e-6)
    gpu.close()
    return counts


@pytest.mark.parametrize("block", OTHER)
def test_drop_matches_oracle(L, block):
    """The drop in a 32^3 periodic-x/y box (with 32x4x4 blocks one block
    spans x, its own neighbour across the periodic wrap)."""
    counts = _pair(L, W.drop_in_box(block=block), 120)
    print(f"drop {block}: meshed blocks {counts[0]} -> {counts[-1]}")
    assert counts[-1] > counts[0]


@pytest.mark.parametrize("block", [(16, 8, 4), (32, 4, 4)])
def test_porous_with_held_cells_matches_oracle(L, block):
    case = W.porous_injection(n=(64, 48, 48), seed=1510035603, inlet=16, x_free=6, r_range=(3.0, 6.0),
                              S=1e-4, block=block)
    counts = _pair(L, case, 30)
    print(f"porous {block}: meshed blocks {counts[0]} -> {counts[-1]}")
    assert counts[-1] > counts[0]


def _state(sim):
    return sim.active_blocks(), [np.stack(sim.macro(a)) for a in range(2)], sim.mass()


def test_streaming_and_modes_agree_within_a_shape(L):
    case = W.porous_injection(n=(64, 48, 48), seed=1510035603, inlet=16, x_free=6, r_range=(3.0, 6.0),
                              S=1e-4, block=(16, 4, 8))
    runs = {}
    for name, kw, mode in [("ab", {}, "stream"), ("aa", {"streaming": "aa"}, "stream"),
                           ("graph", {}, "graph"), ("persistent", {}, "persistent")]:
        sim = L.from_case(case, **kw)
        sim.set_exec(mode)
        for n in (3, 8, 21):
            sim.step(n)
        runs[name] = _state(sim)
        sim.close()
    ref = runs.pop("ab")
    for name, got in runs.items():
        np.testing.assert_array_equal(ref[0], got[0], err_msg=name)
        for a in range(2):
            np.testing.assert_array_equal(ref[1][a], got[1][a], err_msg=name)
        np.testing.assert_array_equal(ref[2], got[2], err_msg=name)


def _members():
    return [W.droplet_impact(n=(32, 48, 32), seed=1), W.porous_injection(n=(48, 32, 32), seed=2, inlet=8, x_free=4),
            W.droplet_impact(n=(32, 32, 48), seed=3), W.porous_injection(n=(32, 32, 32), seed=4, inlet=8, x_free=4)]


def test_batch_members_match_solo_runs_with_a_shape(L):
    block = (16, 8, 4)
    cases = _members()
    batch, place = B.pack(cases, width=96, block=block)
    sim = L.from_case(batch)
    sim.step(40)
    fields = [B.split(np.stack(sim.macro(a)), place) for a in range(2)]
    act = set(sim.active_blocks().tolist())
    for k, c in enumerate(cases):
        solo = L.from_case(c, block=block)
        solo.step(40)
        for a in range(2):
            np.testing.assert_array_equal(fields[a][k], np.stack(solo.macro(a)))
        ids = B.block_map(batch["params"], place, k).reshape(-1)
        mine = np.array(sorted(i for i, b in enumerate(ids) if int(b) in act))
        np.testing.assert_array_equal(mine, solo.active_blocks())
        solo.close()
    sim.close()


def test_shape_autotuner_times_the_tiling_shapes(L):
    best, res = B.autotune_shape(L, _members(), steps=10)
    assert set(res) == {(8, 8, 8), (16, 8, 4), (16, 4, 8)}  # x sizes 48: no 32x4x4
    assert best == min(res, key=lambda k: res[k]["ms_per_step"])
    assert all(r["ms_per_step"] > 0 and r["mlups"] > 0 for r in res.values())
    print("shape autotuner:", res, "->", best)


def test_proposer_needs_8_cubed_blocks(L):
    sim = L.from_case(W.drop_in_box(block=(16, 8, 4)))
    m = L.MLP(1)
    with pytest.raises(L.LBMError) as e:
        sim.set_proposer(m, period=4, threshold=0.5)
    assert e.value.code == L.EINVAL
    m.close()
    sim.close()


def test_static_mesh_is_the_same_in_every_shape(L):
    """A static mesh updates every non-solid cell whatever the block shape,
    from the same neighbours with the same arithmetic: the fields agree bit
    for bit across shapes (the FP64 mass only to rounding: its partial sums
    follow the blocks)."""
    case = W.porous_injection(n=(64, 48, 48), seed=1510035603, inlet=16, x_free=6, r_range=(3.0, 6.0),
                              S=1e-4, progressive=0)
    runs = {}
    for shape in L.SHAPES:
        sim = L.from_case(case, block=shape)
        sim.step(25)
        runs[shape] = ([np.stack(sim.macro(a)) for a in range(2)], sim.mass())
        sim.close()
    ref = runs.pop((8, 8, 8))
    for shape, (fields, mass) in runs.items():
        for a in range(2):
            np.testing.assert_array_equal(ref[0][a], fields[a], err_msg=str(shape))
        np.testing.assert_allclose(ref[1], mass, rtol=1e-13, err_msg=str(shape))


def test_single_component_with_another_shape(L):
    from gpu_helpers import run_pair
    case = W.droplet(n=32, R=9.0, rho_vap=0.42, block=(16, 8, 4))
    gpu, orc, _ = run_pair(L, case, 100)
    assert gpu.block == (16, 8, 4)
    compare_fields(gpu, orc, case, label="droplet 16x8x4")
    np.testing.assert_allclose(gpu.mass(), orc.mass(), rtol=1e-6)
