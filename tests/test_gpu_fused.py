"""The fused step (lbm_set_fusion): the collision of step t and pass 1 of
step t + 1 in one launch, pass 1 reading the new populations from L2.  The
per-cell code is the same as in the two-launch step, so everything must
agree bit for bit with fusion off: meshed blocks, both fields, the FP64 mass
and stored populations, whatever the lag (all pass-1 items deferred to the
end of the launch, or all collisions first), the slot order (block order or
strips of block rows), the execution mode, the block shape and the points
where the slots are renumbered.  Between calls the next step's pass 1 has
already run; every query must still see the state of the last completed
step.  The fused step's pass 1 pulls, so every run here has the density
partials off."""
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


def _porous(**kw):
    return W.porous_injection(n=(64, 48, 48), seed=1510035603, inlet=16, x_free=6, r_range=(3.0, 6.0),
                              S=1e-4, **kw)


def _state(sim, ids=()):
    return (sim.active_blocks(), [np.stack(sim.macro(a)) for a in range(2)], sim.mass(),
            [sim.block_populations(int(b)) for b in ids])


def _assert_same(a, b, ct, label):
    np.testing.assert_array_equal(a[0], b[0], err_msg=f"{label}: meshed blocks")
    for k in range(2):
        np.testing.assert_array_equal(a[1][k], b[1][k], err_msg=f"{label}: fields of component {k}")
    np.testing.assert_array_equal(a[2], b[2], err_msg=f"{label}: FP64 mass")
    nbx, nby = ct.shape[2] // 8, ct.shape[1] // 8
    for blk, x, y in zip(a[0][:: max(1, len(a[0]) // 5)], a[3], b[3]):
        bx, by, bz = blk % nbx, (blk // nbx) % nby, blk // (nbx * nby)
        solid = ct[bz * 8:bz * 8 + 8, by * 8:by * 8 + 8, bx * 8:bx * 8 + 8].reshape(-1) == 1
        np.testing.assert_array_equal(x[:, :, ~solid], y[:, :, ~solid], err_msg=f"{label}: populations")


def _run(L, case, chunks, fusion, mode="stream", strip=None, sort=64, **over):
    # (the strip order is set before from_case applies the geometry)
    sim = L.from_case(case, fusion=fusion, partials=False,
                     **({} if strip is None else {"slot_strip": strip}), **over)
    sim.set_exec(mode)
    sim.set_slot_order(sort)
    out = []
    for n in chunks:
        sim.step(n)
        act = sim.active_blocks()
        out.append(_state(sim, act[:: max(1, len(act) // 5)]))
    st = sim.stats()
    sim.close()
    return out, st


CHUNKS = [1, 6, 13, 1, 24]


@pytest.mark.parametrize("which", ["drop", "porous", "porous_tau", "static"])
def test_fused_equals_two_launches(L, which):
    over = {}
    if which == "drop":
        case = W.drop_in_box()
    elif which == "static":
        case = _porous(progressive=0)
    else:
        case = _porous()
    if which == "porous_tau":
        over["tau"] = 0.8  # the general collision, not the tau = 1 shortcut
    ref, rst = _run(L, case, CHUNKS, (False, 0), **over)
    got, gst = _run(L, case, CHUNKS, (True, 0), **over)
    for k, (a, b) in enumerate(zip(ref, got)):
        _assert_same(a, b, case["cell_type"], f"{which}, after chunk {k}")
    assert gst["steps"] == rst["steps"] and gst["cell_updates"] == rst["cell_updates"]
    # one launch fewer per step (the first step of a call after a
    # renumbering check runs its pass 1 on its own)
    assert gst["launches"] < rst["launches"]


@pytest.mark.parametrize("max_lag", [1, 3, 1 << 30])
def test_any_lag_gives_the_same_result(L, max_lag):
    """max_lag 1: nearly every pass-1 item comes before its neighbours'
    collisions in the work order and is deferred to the end of the launch;
    a huge lag puts every collision first."""
    case = _porous()
    ref, _ = _run(L, case, CHUNKS, (False, 0))
    got, st = _run(L, case, CHUNKS, (True, max_lag))
    for k, (a, b) in enumerate(zip(ref, got)):
        _assert_same(a, b, case["cell_type"], f"max_lag {max_lag}, chunk {k}")
    if max_lag <= 3:
        assert st["fused_deferred"] > 0
    else:
        assert st["fused_deferred"] == 0


@pytest.mark.parametrize("strip", [0, 1, 2])
def test_slot_strips_change_nothing(L, strip):
    """Slots numbered in strips of block rows (each strip z, y, x) instead
    of block order: a different pool layout, the same results."""
    case = _porous()
    ref, _ = _run(L, case, CHUNKS, (False, 0), strip=0)
    got, st = _run(L, case, CHUNKS, (True, 0), strip=strip, sort=4)
    for k, (a, b) in enumerate(zip(ref, got)):
        _assert_same(a, b, case["cell_type"], f"strip {strip}, chunk {k}")
    assert st["slot_sorts"] > 0


@pytest.mark.parametrize("mode", ["graph", "persistent", "staged"])
def test_modes_with_fusion_on(L, mode):
    """GRAPH replays fused pairs of steps; PERSISTENT and STAGED run unfused
    and repeat a pass 1 that ran ahead (its marks are idempotent)."""
    case = _porous()
    ref, _ = _run(L, case, CHUNKS, (False, 0), sort=8)
    sim = L.from_case(case, fusion=(True, 0), partials=False)
    sim.set_slot_order(8)
    got = []
    for k, n in enumerate(CHUNKS):
        # switch between the fused stream and the mode under test call by call
        sim.set_exec(mode if k % 2 else "stream")
        sim.step(n)
        act = sim.active_blocks()
        got.append(_state(sim, act[:: max(1, len(act) // 5)]))
    sim.close()
    for k, (a, b) in enumerate(zip(ref, got)):
        _assert_same(a, b, case["cell_type"], f"{mode}, chunk {k}")


@pytest.mark.parametrize("block", [(16, 8, 4), (32, 4, 4)])
def test_block_shapes(L, block):
    case = W.porous_injection(n=(64, 48, 48), seed=1510035603, inlet=16, x_free=6, r_range=(3.0, 6.0),
                              S=1e-4, block=block)
    out = []
    for fusion in ((False, 0), (True, 0)):
        sim = L.from_case(case, fusion=fusion, partials=False)
        sim.step(30)
        out.append((sim.active_blocks(), [np.stack(sim.macro(a)) for a in range(2)], sim.mass()))
        sim.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    for k in range(2):
        np.testing.assert_array_equal(out[0][1][k], out[1][1][k])
    np.testing.assert_array_equal(out[0][2], out[1][2])


def test_queries_between_calls(L):
    """After a fused call the next step's candidates are already marked:
    they are not meshed yet for any query, and stepping on gives the same
    result as an unfused run."""
    case = W.drop_in_box()
    ref = L.from_case(case, fusion=(False, 0), partials=False)
    sim = L.from_case(case, fusion=(True, 0), partials=False)
    created = False
    for t in range(40):
        ref.step(1)
        sim.step(1)
        ids = sim.active_blocks()
        np.testing.assert_array_equal(ids, ref.active_blocks())
        np.testing.assert_array_equal(sim.activation_steps(), ref.activation_steps())
        # every unmeshed block is refused, including the next step's candidates
        unmeshed = np.setdiff1d(np.arange(sim.nblocks), ids)
        for b in unmeshed:
            with pytest.raises(L.LBMError) as e:
                sim.block_populations(int(b))
            assert e.value.code == L.EINVAL
        created = created or len(ids) > 8
    assert created
    a = _state(ref)
    b = _state(sim)
    _assert_same(a, b, case["cell_type"], "after 40 single steps")
    ref.close()
    sim.close()


def test_fusion_argument_checks(L):
    sim = L.from_case(W.drop_in_box())
    for bad in ((2, 0), (1, -1)):
        with pytest.raises(L.LBMError) as e:
            sim._check(sim.lib.lbm_set_fusion(sim.h, *bad))
        assert e.value.code == L.EINVAL
    with pytest.raises(L.LBMError) as e:
        sim.set_slot_strip(-2)
    assert e.value.code == L.EINVAL
    sim.close()
