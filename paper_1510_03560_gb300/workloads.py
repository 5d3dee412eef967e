"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and
the benchmark.

This module only builds input arrays (cell types, initial densities and
velocities, ambient state) and parameter sets.  It holds none of the
method's arithmetic.  The paper's own geometries (Figs. 10-11: a two
component leakage in a simple box and in channels) are not published, so
these generators stand in for them with the same kind of workload: a
liquid injected into, or relaxing inside, a gas-filled domain, optionally
with a random porous solid.

Cell types: 0 fluid, 1 solid, 2 held (populations kept at the initial
equilibrium: inlets and outlets).  Arrays are [z, y, x] with x fastest;
densities [ncomp, z, y, x]; velocities [ncomp, 3, z, y, x]; all float32.
"""
from __future__ import annotations

import numpy as np

FLUID, SOLID, HELD = 0, 1, 2

# Maxwell equal-area coexistence densities of the Peng-Robinson EOS
# (a = 2/49, b = 2/21, R = 1, acentric factor 0.344) at T = 0.85 Tc.  They
# are inputs (initial liquid / vapour densities); the test suite re-derives
# them from the textbook molar-volume form of the EOS.
RHO_LIQ = 6.629339
RHO_VAP = 0.341309

# Default physics (Sec. 2.2 and the workload description): tau = 1,
# beta = 1.16, Peng-Robinson constants, g_11 = -1, g_12 = 0.1.
PHYSICS = dict(
    tau=1.0, beta=1.16,
    pr_a=2.0 / 49.0, pr_b=2.0 / 21.0, pr_R=1.0, pr_omega=0.344, T_over_Tc=0.85,
    g_self=-1.0, g_cross=0.1,
)


def f32(x):
    return float(np.float32(x))


def _case(cell_type, rho, u, rho_amb, **kw):
    nz, ny, nx = cell_type.shape
    d = dict(cell_type=np.ascontiguousarray(cell_type, dtype=np.uint8),
             rho_init=np.ascontiguousarray(rho, dtype=np.float32),
             u_init=None if u is None else np.ascontiguousarray(u, dtype=np.float32),
             rho_amb=np.asarray(rho_amb, dtype=np.float32),
             params=dict(nx=nx, ny=ny, nz=nz, **kw))
    d["params"].setdefault("rho_ref", tuple(float(r) for r in d["rho_amb"]))
    return d


def drop_in_box(n=32, cube=(13, 19), grav=-1e-5, S=1e-4, progressive=1,
                block=(8, 8, 8), lid=True):
    """Two-component liquid cube relaxing in vapour above a bounce-back floor.

    Grid n^3, periodic in x and y, solid floor at z = 0 (and a solid lid at
    z = n-1).  Component 0: Peng-Robinson, liquid RHO_LIQ inside the cube,
    vapour RHO_VAP outside; component 1: ideal gas, 0.01 inside, 1.0
    outside.  Gravity along -z acts on the density excess over the ambient.
    """
    ct = np.zeros((n, n, n), dtype=np.uint8)
    ct[0] = SOLID
    if lid:
        ct[n - 1] = SOLID
    rho = np.empty((2, n, n, n), dtype=np.float32)
    rho[0] = f32(RHO_VAP)
    rho[1] = 1.0
    a, b = cube
    rho[0, a:b, a:b, a:b] = f32(RHO_LIQ)
    rho[1, a:b, a:b, a:b] = f32(0.01)
    amb = (f32(RHO_VAP), 1.0)
    return _case(ct, rho, None, amb, ncomp=2, periodic=(1, 1, 0), progressive=progressive,
                 block=block, g_ads=(0.0, 0.0), grav=(0.0, 0.0, grav), S=S, **PHYSICS)


def spheres_mask(shape, seed, solid_frac, r_range, x_free):
    """Random overlapping spheres (uniform centres, uniform radii) added one by
    one until the solid fraction of the box reaches solid_frac.  No sphere
    reaches below x = x_free.  Returns a bool [z, y, x] mask."""
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    solid = np.zeros(shape, dtype=bool)
    target = solid_frac * solid.size
    count = 0
    r0, r1 = r_range
    zz = np.arange(nz)
    yy = np.arange(ny)
    xx = np.arange(nx)
    while count < target:
        r = rng.uniform(r0, r1)
        cx = rng.uniform(x_free + r, nx)
        cy = rng.uniform(0, ny)
        cz = rng.uniform(0, nz)
        x0, x1 = max(int(np.floor(cx - r)), 0), min(int(np.ceil(cx + r)) + 1, nx)
        y0, y1 = max(int(np.floor(cy - r)), 0), min(int(np.ceil(cy + r)) + 1, ny)
        z0, z1 = max(int(np.floor(cz - r)), 0), min(int(np.ceil(cz + r)) + 1, nz)
        d2 = ((zz[z0:z1, None, None] + 0.5 - cz) ** 2 +
              (yy[None, y0:y1, None] + 0.5 - cy) ** 2 +
              (xx[None, None, x0:x1] + 0.5 - cx) ** 2)
        inside = d2 <= r * r
        sub = solid[z0:z1, y0:y1, x0:x1]
        count += int(np.count_nonzero(inside & ~sub))
        sub |= inside
    return solid


def porous_injection(n=(256, 256, 256), seed=1510035601, solid_frac=0.30, r_range=(6.0, 12.0),
                     inlet=64, u_in=0.02, g_ads=-0.2, x_free=16, S=3e-4, progressive=1,
                     block=(8, 8, 8), rho_gas_in=0.1):
    """Liquid injected through an inlet patch into a gas-filled porous box.

    Grid nx*ny*nz; seeded random spheres (radius r_range, solid fraction
    solid_frac) kept out of x < x_free; walls at y = 0, ny-1, z = 0, nz-1;
    the x = 0 face is solid except a centred inlet x inlet patch of held
    cells (component 0 at RHO_LIQ, component 1 at rho_gas_in, both moving at
    u_in along +x); the x = nx-1 face is held at the ambient gas state (an
    open outlet).  Gas: component 0 at RHO_VAP, component 1 at 1.0.
    Component 0 wets the solid (g_ads).  The criterion threshold S = 3e-4
    meshes about 58 % of the 256^3 blocks by the end of the run (the paper
    uses S = 0, which in FP32 meshes everything at the first acoustic wave).
    The injected liquid carries some of
    the second component (rho_gas_in = 0.1): with much less (0.01) the
    nearly empty component's velocity F / rho at the inlet grows without
    bound and the run diverges within a hundred steps.
    """
    nx, ny, nz = n
    ct = np.zeros((nz, ny, nx), dtype=np.uint8)
    ct[spheres_mask((nz, ny, nx), seed, solid_frac, r_range, x_free)] = SOLID
    outlet = ct[:, :, nx - 1]
    outlet[outlet != SOLID] = HELD
    ct[:, :, 0] = SOLID
    ct[:, 0, :] = SOLID
    ct[:, ny - 1, :] = SOLID
    ct[0, :, :] = SOLID
    ct[nz - 1, :, :] = SOLID
    y0, z0 = (ny - inlet) // 2, (nz - inlet) // 2
    ct[z0:z0 + inlet, y0:y0 + inlet, 0] = HELD
    rho = np.empty((2, nz, ny, nx), dtype=np.float32)
    rho[0] = f32(RHO_VAP)
    rho[1] = 1.0
    u = np.zeros((2, 3, nz, ny, nx), dtype=np.float32)
    rho[0, z0:z0 + inlet, y0:y0 + inlet, 0] = f32(RHO_LIQ)
    rho[1, z0:z0 + inlet, y0:y0 + inlet, 0] = f32(rho_gas_in)
    u[:, 0, z0:z0 + inlet, y0:y0 + inlet, 0] = f32(u_in)
    amb = (f32(RHO_VAP), 1.0)
    return _case(ct, rho, u, amb, ncomp=2, periodic=(0, 0, 0), progressive=progressive,
                 block=block, g_ads=(g_ads, 0.0), grav=(0.0, 0.0, 0.0), S=S, **PHYSICS)


def droplet_impact(n=(64, 64, 64), seed=1510035700, u_drop=0.03, g_ads=-0.2, S=3e-4,
                   progressive=1, block=(8, 8, 8)):
    """A liquid drop moving towards a wetting floor in a closed gas box.

    Walls on every face; a sphere of radius max(4, min(n) / 6) centred
    near the top (seeded jitter of the centre) holds component 0 at RHO_LIQ
    and component 1 at 0.1, both moving at u_drop along -z; gas elsewhere
    (component 0 at RHO_VAP, component 1 at 1.0).  Physics, ambient and S
    as porous_injection, so that the two kinds of case can share one batch.
    """
    nx, ny, nz = n
    rng = np.random.default_rng(seed)
    ct = np.zeros((nz, ny, nx), dtype=np.uint8)
    ct[:, :, 0] = ct[:, :, nx - 1] = SOLID
    ct[:, 0, :] = ct[:, ny - 1, :] = SOLID
    ct[0, :, :] = ct[nz - 1, :, :] = SOLID
    R = max(4.0, min(n) / 6.0)
    c = (nx / 2 + rng.uniform(-0.1, 0.1) * nx, ny / 2 + rng.uniform(-0.1, 0.1) * ny,
         nz - 2.0 * R - 2.0 + rng.uniform(-1.0, 1.0))
    z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    inside = ((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2 < R * R) & (ct == FLUID)
    rho = np.empty((2, nz, ny, nx), dtype=np.float32)
    rho[0] = f32(RHO_VAP)
    rho[1] = 1.0
    rho[0][inside] = f32(RHO_LIQ)
    rho[1][inside] = f32(0.1)
    u = np.zeros((2, 3, nz, ny, nx), dtype=np.float32)
    u[0, 2][inside] = f32(-u_drop)
    u[1, 2][inside] = f32(-u_drop)
    amb = (f32(RHO_VAP), 1.0)
    return _case(ct, rho, u, amb, ncomp=2, periodic=(0, 0, 0), progressive=progressive,
                 block=block, g_ads=(g_ads, 0.0), grav=(0.0, 0.0, 0.0), S=S, **PHYSICS)


def droplet(n=32, R=8.0, center=None, progressive=0, block=(8, 8, 8), rho_vap=RHO_VAP):
    """Single-component Peng-Robinson droplet of radius R in vapour of
    density rho_vap, fully periodic box (Laplace test)."""
    c = (n / 2.0,) * 3 if center is None else center
    z, y, x = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5, np.arange(n) + 0.5,
                          indexing="ij")
    r = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2)
    rho = np.where(r <= R, f32(RHO_LIQ), f32(rho_vap)).astype(np.float32)[None]
    ct = np.zeros((n, n, n), dtype=np.uint8)
    phys = dict(PHYSICS)
    phys["g_cross"] = 0.0
    return _case(ct, rho, None, (f32(rho_vap),), ncomp=1, periodic=(1, 1, 1),
                 progressive=progressive, block=block, g_ads=(0.0, 0.0), grav=(0.0, 0.0, 0.0),
                 S=0.0, **phys)


def slab(nxy=8, nz=64, frac=0.5, block=(8, 8, 8)):
    """Single-component flat liquid slab across a periodic box (coexistence
    test): liquid for the central frac of z, vapour elsewhere."""
    ct = np.zeros((nz, nxy, nxy), dtype=np.uint8)
    rho = np.full((1, nz, nxy, nxy), f32(RHO_VAP), dtype=np.float32)
    a = int(nz * (1 - frac) / 2)
    rho[0, a:nz - a] = f32(RHO_LIQ)
    phys = dict(PHYSICS)
    phys["g_cross"] = 0.0
    return _case(ct, rho, None, (f32(RHO_VAP),), ncomp=1, periodic=(1, 1, 1), progressive=0,
                 block=block, g_ads=(0.0, 0.0), grav=(0.0, 0.0, 0.0), S=0.0, **phys)


def channel(H=16, nxy=8, gx=1e-6, tau=1.0, block=(8, 8, 8)):
    """Single-component, non-interacting fluid between two solid plates
    (z = 0 and z = H+1, H fluid layers), periodic in x and y, driven by a
    uniform body force density rho * gx along x (Poiseuille test).  The z
    extent is padded with solid up to a multiple of the block height."""
    bz = block[2]
    nz = ((H + 2 + bz - 1) // bz) * bz
    ct = np.zeros((nz, nxy, nxy), dtype=np.uint8)
    ct[0] = SOLID
    ct[H + 1:] = SOLID
    rho = np.ones((1, nz, nxy, nxy), dtype=np.float32)
    phys = dict(PHYSICS)
    phys.update(g_self=0.0, g_cross=0.0, tau=tau)
    return _case(ct, rho, None, (1.0,), ncomp=1, periodic=(1, 1, 0), progressive=0,
                 block=block, g_ads=(0.0, 0.0), grav=(gx, 0.0, 0.0), rho_ref=(0.0,), S=0.0,
                 **phys)


def blob(n=16, block=(4, 4, 4), rho_amb=(RHO_VAP, 1.0), S=0.0, progressive=1, seed=7,
         grav=-1e-5):
    """Small asymmetric two-component liquid blob (an off-centre ellipsoid
    with a seeded random density ripple) in a periodic-x/y box with floor
    and lid; used for the progressive-equals-static test on tiny grids."""
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    inside = (((x - 5.3) / 2.6) ** 2 + ((y - 6.1) / 2.1) ** 2 + ((z - 7.2) / 1.8) ** 2) <= 1.0
    ct = np.zeros((n, n, n), dtype=np.uint8)
    ct[0] = SOLID
    ct[n - 1] = SOLID
    rho = np.empty((2, n, n, n), dtype=np.float32)
    rho[0] = f32(rho_amb[0])
    rho[1] = f32(rho_amb[1])
    ripple = rng.uniform(-0.05, 0.05, size=inside.sum()).astype(np.float32)
    rho[0][inside] = f32(RHO_LIQ) + ripple
    rho[1][inside] = f32(0.01)
    amb = (f32(rho_amb[0]), f32(rho_amb[1]))
    return _case(ct, rho, None, amb, ncomp=2, periodic=(1, 1, 0), progressive=progressive,
                 block=block, g_ads=(0.0, 0.0), grav=(0.0, 0.0, grav), S=S, **PHYSICS)
