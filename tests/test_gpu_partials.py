"""Density partials (lbm_set_density_partials): pass 1 sums the densities the
previous collision prepared (each cell's own-half-block terms plus the
entries its neighbour half blocks sent) instead of pulling 38 populations.

Pull streaming (Eq. 10, left) and Eq. 4 fix what the sum must be, so the two
ways of taking it may differ only by rounding order.  Checked here:
  - one step from the same state: the pull and the partials give the same
    densities up to rounding, seen through the forces (Eqs. 6-9) that the
    reported velocity carries; a missing or doubled term moves psi by
    percents and the velocity by 1e-4 or more;
  - long runs with the partials against the FP64 oracle, meshed sets equal at
    every step, on cases with a one-block periodic axis (a half block is its
    own x and y neighbour), held inlet cells, solid spheres and other block
    shapes;
  - switching them off and on between calls keeps the oracle's meshed sets
    and fields; GRAPH and PERSISTENT agree with the three-launch step bit for
    bit, renumbering of the slots included (the partials move with them)."""
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


def _narrow(progressive=1):
    """The 32^3 drop cropped to 8 x 8 cells across x and y (one block, periodic
    in both): every half block is its own x, y and edge neighbour."""
    c = W.drop_in_box(n=32, cube=(13, 19), progressive=progressive)
    sl = (slice(None), slice(12, 20), slice(12, 20))
    p = dict(c["params"], nx=8, ny=8)
    return dict(cell_type=np.ascontiguousarray(c["cell_type"][sl]),
                rho_init=np.ascontiguousarray(c["rho_init"][(slice(None),) + sl]),
                u_init=None, rho_amb=c["rho_amb"], params=p)


def _porous(**kw):
    return W.porous_injection(n=(56, 40, 48), seed=1510035603, inlet=16, x_free=6, r_range=(3.0, 6.0),
                              S=1e-4, **kw)


CASES = {
    "drop": lambda: W.drop_in_box(),
    "drop_static": lambda: W.drop_in_box(progressive=0),
    "narrow": _narrow,
    "narrow_static": lambda: _narrow(progressive=0),
    "porous": _porous,
    "porous_static": lambda: _porous(progressive=0),
    "shape_16x8x4": lambda: W.drop_in_box(block=(16, 8, 4), progressive=0),
    "shape_32x4x4": lambda: W.porous_injection(n=(64, 48, 48), seed=1510035603, inlet=16, x_free=6,
                                               r_range=(3.0, 6.0), S=1e-4, block=(32, 4, 4), progressive=0),
    "shape_16x4x8": lambda: W.drop_in_box(block=(16, 4, 8)),
}


@pytest.mark.parametrize("which", sorted(CASES))
def test_partial_densities_equal_the_pull(L, which):
    """After 40 steps without partials the state is copied into two runs by
    stepping both from the start; one more step, then the reported fields of
    the partials run must equal the pull run's to rounding: density exactly
    (the output pulls it), velocity within 1e-7 (it carries the force built
    from the pass-1 densities of the 18 neighbours)."""
    case = CASES[which]()
    a = L.from_case(case, partials=False)
    b = L.from_case(case, partials=False)
    a.step(40)
    b.step(40)
    b.set_density_partials(True)
    a.step(1)
    b.step(1)  # pulls once more, its collision writes the partials
    np.testing.assert_array_equal(a.active_blocks(), b.active_blocks())
    ncomp = case["params"]["ncomp"]
    worst = 0.0
    for comp in range(ncomp):
        fa, fb = a.macro(comp), b.macro(comp)  # b: pass 1 from the partials
        np.testing.assert_array_equal(fa[0], fb[0])
        for k in (1, 2, 3):
            worst = max(worst, float(np.abs(fa[k] - fb[k]).max()))
    print(f"{which}: max |u_partials - u_pull| = {worst:.3g}")
    assert worst <= 1e-7
    a.close()
    b.close()


@pytest.mark.parametrize("which", ["narrow", "porous", "shape_16x4x8"])
def test_partials_follow_the_oracle(L, which):
    case = CASES[which]()
    gpu = L.from_case(case, partials=True)
    orc = oracle_of(case)
    S = case["params"].get("S", 0.0)
    for t in range(120):
        gpu.step(1)
        orc.step(1)
        compare_active(gpu, orc, t, S)
    compare_fields(gpu, orc, case, label=which)
    gpu.close()


def test_switching_between_calls(L):
    """Partials on, off, on again (the first pass 1 after switching on pulls),
    in GRAPH mode (a plain step writes the partials before the graph's first
    replay): the meshed sets stay the oracle's at every call and the fields
    within the FP32 tolerances."""
    case = _porous()
    gpu = L.from_case(case, partials=True)
    gpu.set_exec("graph")
    orc = oracle_of(case)
    S = case["params"]["S"]
    t = 0
    for on, n in ((True, 9), (False, 4), (True, 1), (True, 12), (False, 7), (True, 30)):
        gpu.set_density_partials(on)
        gpu.step(n)
        orc.step(n)
        t += n
        compare_active(gpu, orc, t, S)
    compare_fields(gpu, orc, case, label="switching")
    gpu.close()


def test_partials_are_off_where_they_do_not_apply(L):
    """FP16 storage and A-A streaming keep the pull: asking for the partials
    there is accepted and changes nothing."""
    case = W.drop_in_box()
    for kw in ({"storage": "fp16"}, {"streaming": "aa"}):
        runs = []
        for on in (False, True):
            sim = L.from_case(case, partials=on, **kw)
            sim.step(25)
            runs.append((sim.active_blocks(), [np.stack(sim.macro(a)) for a in range(2)]))
            sim.close()
        np.testing.assert_array_equal(runs[0][0], runs[1][0])
        for k in range(2):
            np.testing.assert_array_equal(runs[0][1][k], runs[1][1][k])


@pytest.mark.parametrize("mode", ["graph", "persistent"])
def test_modes_agree_with_partials(L, mode):
    """The three-launch step, the replayed graph and the cooperative launch
    sum the partials with the same code: bit for bit, progressive mesh with
    renumbering of the slots (the partials move with their slots)."""
    case = _porous()
    runs = []
    for m, order in (("stream", 0), (mode, 4)):
        sim = L.from_case(case, partials=True)
        sim.set_exec(m)
        sim.set_slot_order(order)
        for n in (1, 6, 13, 2, 25):
            sim.step(n)
        runs.append((sim.active_blocks(), [np.stack(sim.macro(a)) for a in range(2)], sim.mass(),
                     sim.stats()["slot_sorts"]))
        sim.close()
    np.testing.assert_array_equal(runs[0][0], runs[1][0])
    for k in range(2):
        np.testing.assert_array_equal(runs[0][1][k], runs[1][1][k])
    np.testing.assert_array_equal(runs[0][2], runs[1][2])
    assert runs[0][3] == 0 and runs[1][3] > 0


def test_argument_checks(L):
    sim = L.from_case(W.drop_in_box())
    with pytest.raises(L.LBMError) as e:
        sim._check(sim.lib.lbm_set_density_partials(sim.h, 2))
    assert e.value.code == L.EINVAL
    sim.close()
