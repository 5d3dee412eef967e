"""The 16-bit deviation storage forms (FP16, BF16) against the FP64 oracle.

Populations are stored as f_i - w_i rho_r in 16 bits and decoded to FP32
for the arithmetic, so these runs are not expected to match the oracle to
the FP32 tolerances.  Each test states the error per field and bounds it:

  FP16 (11-bit significand): density <= 1e-3 relative, velocity <= 5e-4.
  BF16 (8-bit significand, 8x the FP16 rounding step): density <= 1e-3
  relative (the bound the 16-bit forms are specified to) and velocity
  <= 2e-3, except in the first three fluid layers behind the held inlet of
  the porous crop (FRONT): there the injected liquid (rho 6.6, accelerated
  to |v| ~ 0.3 by the forces) meets gas of density 0.34, so the populations
  a gas cell receives are several times its own density whatever reference
  they are stored against, and 8 significant bits of them leave up to
  2e-3 of its density.

With the progressive mesh the 16-bit rounding of the velocity (about 1e-4
near the injected liquid) is close to the criterion threshold S = 3e-4 of
the injection workload, so a block can be created one step earlier or later
than in the oracle; the fields then differ near that block by more than the
storage error.  Those runs are bounded separately (TIMING) and report the
first step at which the meshed sets differ.

Mass: every stored value is rounded once (round to nearest), and the rest
population of each written cell absorbs the rounding of the other 18, so
the total mass drifts only by the rounding of one value per cell and step.
"""
import numpy as np
import pytest

from gpu_helpers import oracle_of, order_map
from paper_1510_03560_gb300 import workloads as W

pytestmark = pytest.mark.gpu

BOUNDS = {"fp16": dict(rho=1e-3, u=5e-4, mass=1e-5),
          "bf16": dict(rho=1e-3, u=2e-3, mass=1e-4)}
FRONT = dict(rho=2e-3, u=2e-3)  # BF16, the first three layers behind the inlet
TIMING = dict(rho=5e-2, u=2e-2)


@pytest.fixture(scope="module")
def L():
    import torch
    from paper_1510_03560_gb300 import build as B
    B.build()
    from paper_1510_03560_gb300 import lbm
    assert torch.cuda.is_available()
    return lbm


def field_errors(gpu, orc, case, region=None):
    """Max relative density error and max absolute velocity error per
    component over the non-solid cells (of `region` when given)."""
    fluid = case["cell_type"] != 1
    if region is not None:
        fluid = fluid & region
    out = []
    for a in range(orc.ncomp):
        g, o = gpu.macro(a), orc.macro(a)
        rel = np.abs(g[0][fluid] - o[0][fluid]) / np.abs(o[0][fluid])
        du = max(np.abs(g[k][fluid] - o[k][fluid]).max() for k in (1, 2, 3))
        out.append((float(rel.max()), float(du)))
        assert np.all(g[0][case["cell_type"] == 1] == 0)
    return out


def check(form, errs, label, b=None):
    b = b or BOUNDS[form]
    print(f"{label} {form}: " + ", ".join(
        f"comp {a}: rho rel {r:.3g}, u abs {u:.3g}" for a, (r, u) in enumerate(errs)))
    for a, (r, u) in enumerate(errs):
        assert r <= b["rho"], f"{label} {form} comp {a}: rho rel err {r:.3g}"
        assert u <= b["u"], f"{label} {form} comp {a}: u abs err {u:.3g}"


@pytest.mark.parametrize("form", ["fp16", "bf16"])
def test_drop_progressive_error_per_field(L, form):
    case = W.drop_in_box()
    gpu = L.from_case(case, storage=form)
    orc = oracle_of(case)
    m0 = np.array(orc.mass())
    gm0 = np.array(gpu.mass())
    np.testing.assert_allclose(gm0, m0, rtol=BOUNDS[form]["mass"])
    gpu.step(200)
    orc.step(200)
    check(form, field_errors(gpu, orc, case), "drop 32^3, 200 steps")
    drift = np.abs(np.array(gpu.mass()) - m0) / m0
    print(f"mass drift {form}: {drift}")
    assert drift.max() <= BOUNDS[form]["mass"]
    ga, oa = gpu.active_blocks(), orc.active_blocks()
    print(f"active blocks {form}: gpu {len(ga)}, oracle {len(oa)}, "
          f"differing {len(np.setxor1d(ga, oa))}")
    gpu.close()


@pytest.mark.parametrize("form", ["fp16", "bf16"])
def test_drop_static_error_per_field(L, form):
    case = W.drop_in_box(progressive=0)
    gpu = L.from_case(case, storage=form)
    orc = oracle_of(case)
    gpu.step(100)
    orc.step(100)
    check(form, field_errors(gpu, orc, case), "drop static, 100 steps")
    gpu.close()


@pytest.mark.parametrize("form", ["fp16", "bf16"])
@pytest.mark.parametrize("progressive", [0, 1])
def test_porous_crop_error_per_field(L, form, progressive):
    """The 384^3 injection recipe cropped to 64^3 (seed 1510035603, inlet
    16^2): held inlet cells, adhesion, solid spheres, block creation."""
    case = W.porous_injection(n=(64, 64, 64), seed=1510035603, inlet=16, x_free=16,
                              progressive=progressive)
    gpu = L.from_case(case, storage=form)
    orc = oracle_of(case)
    first_diff = None
    for t in range(150):
        gpu.step(1)
        orc.step(1)
        if progressive and first_diff is None:
            ga, oa = gpu.active_blocks(), orc.active_blocks()
            if not np.array_equal(ga, oa):
                first_diff = (t, len(np.setxor1d(ga, oa)))
    print(f"porous {form} progressive={progressive}: first active-set difference "
          f"(step, blocks) = {first_diff}")
    label = f"porous 64^3 crop p={progressive}, 150 steps"
    timing = TIMING if first_diff is not None else None
    if form == "bf16":
        # the gas cells just behind the inlet (x < 4) take the liquid front
        # at the 20-fold density contrast: bounded by FRONT, the rest by 1e-3
        x = np.arange(case["cell_type"].shape[2])[None, None, :]
        away = np.broadcast_to(x >= 4, case["cell_type"].shape)
        check(form, field_errors(gpu, orc, case, ~away), label + ", x < 4", timing or FRONT)
        check(form, field_errors(gpu, orc, case, away), label + ", x >= 4", timing)
    else:
        check(form, field_errors(gpu, orc, case), label, timing)
    # held cells keep their state exactly: density from mac, velocity from
    # the stored initial velocity
    held = case["cell_type"] == 2
    for a in range(2):
        g = gpu.macro(a)
        np.testing.assert_array_equal(g[0][held], case["rho_init"][a][held].astype(np.float32))
        for k in range(3):
            np.testing.assert_array_equal(g[k + 1][held],
                                          case["u_init"][a][k][held].astype(np.float32))
    gpu.close()


@pytest.mark.parametrize("form", ["fp16", "bf16"])
def test_block_populations_decode(L, form):
    """Decoded post-collision populations of meshed blocks against the
    oracle's, relative to the local density."""
    case = W.drop_in_box(progressive=0)
    gpu = L.from_case(case, storage=form)
    orc = oracle_of(case)
    gpu.step(30)
    orc.step(30)
    omap = order_map(L)
    nx = case["cell_type"].shape[2]
    f_o = np.stack([orc.get_f(a) for a in range(2)])  # [ncomp][nz][ny][nx][19], oracle order
    worst = 0.0
    for b in gpu.active_blocks()[::3]:
        g = gpu.block_populations(int(b))  # [ncomp][19][512]
        nbx = nx // 8
        bx, by, bz = b % nbx, (b // nbx) % nbx, b // (nbx * nbx)
        sub = f_o[:, bz * 8:(bz + 1) * 8, by * 8:(by + 1) * 8, bx * 8:(bx + 1) * 8, :]
        sub = sub.reshape(2, 512, 19)[:, :, omap].transpose(0, 2, 1)
        solid = case["cell_type"][bz * 8:(bz + 1) * 8, by * 8:(by + 1) * 8,
                                  bx * 8:(bx + 1) * 8].reshape(512) == 1
        rho = np.maximum(sub.sum(axis=1), 1e-30)  # [2][512]
        err = np.abs(g - sub) / rho[:, None, :]
        worst = max(worst, float(err[:, :, ~solid].max()))
        assert np.all(g[:, :, solid] == 0)
    print(f"populations {form}: max |f - f_oracle| / rho = {worst:.3g}")
    assert worst <= BOUNDS[form]["rho"]
    gpu.close()
