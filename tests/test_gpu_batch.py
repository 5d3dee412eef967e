"""The batching form on the GPU: every simulation of a batch evolves bit for
bit as it does alone, in every execution mode."""
import numpy as np
import pytest

from paper_1510_03560_gb300 import batch as B
from paper_1510_03560_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    from paper_1510_03560_gb300 import build as Bld
    Bld.build()
    from paper_1510_03560_gb300 import lbm
    assert torch.cuda.is_available()
    return lbm


def _cases():
    return [W.droplet_impact(n=(32, 48, 32), seed=1), W.porous_injection(n=(48, 32, 32), seed=2, inlet=8, x_free=4),
            W.droplet_impact(n=(32, 32, 48), seed=3), W.porous_injection(n=(32, 32, 32), seed=4, inlet=8, x_free=4)]


@pytest.mark.parametrize("mode,slot_order", [("stream", 64), ("graph", 64), ("persistent", 64),
                                             ("stream", 8)])
def test_batch_members_match_solo_runs(L, mode, slot_order):
    """(slot_order 8: the batch's slots are renumbered in block order several
    times on the way; the solo runs keep the default.)"""
    cases = _cases()
    batch, place = B.pack(cases, width=96)
    sim = L.from_case(batch)
    sim.set_exec(mode)
    sim.set_slot_order(slot_order)
    sim.step(60)
    fields = [B.split(np.stack(sim.macro(a)), place) for a in range(2)]
    act = set(sim.active_blocks().tolist())
    for k, c in enumerate(cases):
        solo = L.from_case(c)
        solo.step(60)
        for a in range(2):
            np.testing.assert_array_equal(fields[a][k], np.stack(solo.macro(a)))
        ids = B.block_map(batch["params"], place, k).reshape(-1)
        mine = np.array(sorted(i for i, b in enumerate(ids) if int(b) in act))
        np.testing.assert_array_equal(mine, solo.active_blocks())
        solo.close()
    if slot_order == 8:
        assert sim.stats()["slot_sorts"] > 0
    sim.close()


def test_autotune_reports_every_mode(L):
    batch, _ = B.pack(_cases())
    best, times = B.autotune(L, batch, steps=10)
    assert best in times and set(times) == {"stream", "graph", "persistent", "staged"}
    assert all(t > 0 for t in times.values())
