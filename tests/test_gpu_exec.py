"""Execution modes (lbm_set_exec): the step as three launches, as a replayed
CUDA graph of two steps, and as one cooperative launch per call with grid
barriers.  All run the same per-cell code, so results must agree bit for
bit; the barrier's bounded wait is checked with a barrier that cannot
complete.  (These run with the density partials off, the default; the
TMA-staged kernels have none.  tests/test_gpu_partials.py compares the
modes with them on.)"""
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


def _run(L, case, mode, chunks, **over):
    sim = L.from_case(case, **over)
    sim.set_exec(mode)
    sets = []
    for n in chunks:
        sim.step(n)
        sets.append(sim.active_blocks())
    fields = [sim.macro(a) for a in range(case["params"]["ncomp"])]
    st = sim.stats()
    mass = sim.mass()
    sim.close()
    return sets, fields, st, mass


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
@pytest.mark.parametrize("which", ["drop", "porous"])
def test_modes_agree_bit_for_bit(L, which, storage):
    if which == "drop":
        case = W.drop_in_box()
    else:
        case = W.porous_injection(n=(56, 40, 48), seed=1510035603, inlet=16, x_free=6,
                                  r_range=(3.0, 6.0), S=1e-4)
    chunks = [7, 20, 1, 32]  # odd and even counts: graph pairs plus single steps
    ref = _run(L, case, "stream", chunks, storage=storage)
    for mode in ("graph", "persistent", "staged"):
        got = _run(L, case, mode, chunks, storage=storage)
        for a, b in zip(ref[0], got[0]):
            np.testing.assert_array_equal(a, b)
        for fa, fb in zip(ref[1], got[1]):
            for x, y in zip(fa, fb):
                np.testing.assert_array_equal(x, y)
        assert got[2]["steps"] == ref[2]["steps"] == sum(chunks)
        assert got[2]["cell_updates"] == ref[2]["cell_updates"]
        # new blocks take slots in block order, so even the FP64 mass
        # (summed over slots) is the same bit for bit
        np.testing.assert_array_equal(got[3], ref[3])


@pytest.mark.parametrize("mode", ["persistent", "staged"])
def test_static_mode(L, mode):
    case = W.drop_in_box(progressive=0)
    ref = _run(L, case, "stream", [15])
    got = _run(L, case, mode, [15])
    for fa, fb in zip(ref[1], got[1]):
        for x, y in zip(fa, fb):
            np.testing.assert_array_equal(x, y)


def test_persistent_pool_exhaustion(L):
    """Block creation that overflows the pool stops the cooperative launch
    at the step boundary, as in stream mode."""
    case = W.drop_in_box()
    out = []
    for mode in ("stream", "persistent"):
        sim = L.from_case(case, max_blocks=12)
        sim.set_exec(mode)
        with pytest.raises(L.LBMError) as e:
            sim.step(200)
        assert e.value.code == L.ENOMEM
        out.append((sim.stats()["steps"], sim.active_blocks(), sim.macro(0)[0]))
        sim.close()
    assert out[0][0] == out[1][0]
    np.testing.assert_array_equal(out[0][1], out[1][1])
    np.testing.assert_array_equal(out[0][2], out[1][2])


def test_bounded_barrier_wait(L):
    assert L.barrier_selftest(0, 1 << 20) == L.OK
    # a barrier that expects one CTA too many gives up after the poll limit
    assert L.barrier_selftest(1, 2000) == L.ETIMEOUT
    # the device is still usable afterwards
    assert L.barrier_selftest(0, 1 << 20) == L.OK


def test_unknown_mode_rejected(L):
    sim = L.from_case(W.drop_in_box())
    with pytest.raises(L.LBMError) as e:
        sim.set_exec(7)
    assert e.value.code == L.EINVAL
    sim.close()
