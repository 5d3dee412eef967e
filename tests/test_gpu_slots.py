"""Renumbering the meshed slots in block order between steps
(lbm_set_slot_order) changes where blocks live in the pool, not what any
cell computes: meshed blocks, fields, FP64 mass and stored populations equal
those of a run that never renumbers, bit for bit, in the FP32 and FP16
forms and in every execution mode."""
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


def _case():
    return W.porous_injection(n=(64, 48, 48), seed=1510035603, inlet=16, x_free=6, r_range=(3.0, 6.0),
                              S=1e-4)


def _state(sim, ids=None):
    st = (sim.active_blocks(), [np.stack(sim.macro(a)) for a in range(2)], sim.mass())
    if ids is not None:
        st = st + ([sim.block_populations(int(b)) for b in ids],)
    return st


@pytest.mark.parametrize("storage,mode,streaming", [("fp32", "stream", "ab"), ("fp16", "stream", "ab"),
                                                    ("fp32", "graph", "ab"), ("fp32", "persistent", "ab"),
                                                    ("fp32", "stream", "aa"), ("fp32", "graph", "aa")])
def test_renumbering_changes_nothing(L, storage, mode, streaming):
    """(A-A streaming renumbers the order in which the passes visit the
    slots, not the slots.)"""
    case = _case()
    ref = L.from_case(case, storage=storage)
    ref.set_slot_order(0)
    sim = L.from_case(case, storage=storage, streaming=streaming)
    sim.set_slot_order(4)
    sim.set_exec(mode)
    for n in (5, 11, 17, 31):
        ref.step(n)
        sim.step(n)
        ids = ref.active_blocks()[::37] if storage == "fp32" else None
        a, b = _state(ref, ids), _state(sim, ids)
        np.testing.assert_array_equal(a[0], b[0])
        for k in range(2):
            np.testing.assert_array_equal(a[1][k], b[1][k])
        np.testing.assert_array_equal(a[2], b[2])
        if ids is not None:  # non-solid cells (solid cells' stored values are never read)
            ct = case["cell_type"]
            nbx, nby = ct.shape[2] // 8, ct.shape[1] // 8
            for blk, x, y in zip(ids, a[3], b[3]):
                bx, by, bz = blk % nbx, (blk // nbx) % nby, blk // (nbx * nby)
                keep = ct[bz * 8:bz * 8 + 8, by * 8:by * 8 + 8, bx * 8:bx * 8 + 8].reshape(-1) != W.SOLID
                np.testing.assert_array_equal(x[..., keep], y[..., keep])
    sorts = sim.stats()["slot_sorts"]
    print(f"{storage} {mode}: {sorts} renumberings, {len(sim.active_blocks())} meshed blocks")
    assert sorts > 0 and ref.stats()["slot_sorts"] == 0
    ref.close()
    sim.close()


def test_renumbering_with_the_proposer(L):
    from paper_1510_03560_gb300 import proposer as PR
    case = _case()
    base = L.from_case(case)
    base.set_slot_order(0)
    prop = L.from_case(case)
    prop.set_slot_order(8)
    m = PR.load_model(L)
    prop.set_proposer(m, period=4, threshold=0.5)
    base.step(64)
    prop.step(64)
    np.testing.assert_array_equal(base.active_blocks(), prop.active_blocks())
    for a in range(2):
        for x, y in zip(base.macro(a), prop.macro(a)):
            np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(base.mass(), prop.mass())
    assert prop.stats()["slot_sorts"] > 0
    prop.set_proposer(None)
    m.close()
    prop.close()
    base.close()


def test_negative_period_is_refused(L):
    sim = L.from_case(W.drop_in_box())
    with pytest.raises(L.LBMError) as e:
        sim.set_slot_order(-1)
    assert e.value.code == L.EINVAL
    sim.close()
