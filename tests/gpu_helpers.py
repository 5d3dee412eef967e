"""Shared helpers of the GPU parity tests: run the CUDA library and the FP64
oracle side by side on the same seeded inputs and compare."""
import numpy as np

from oracle import oracle as O

RHO_RTOL = 1e-4   # density, relative (FP32 path vs FP64 oracle)
U_ATOL = 1e-5     # velocity, absolute, lattice units


def oracle_of(case, **over):
    p = dict(case["params"])
    p.update(over)
    return O.OracleSim(case["cell_type"], case["rho_init"], case["u_init"], case["rho_amb"], **p)


def gpu_of(L, case, **over):
    return L.from_case(case, **over)


def compare_fields(gpu, orc, case, rho_rtol=RHO_RTOL, u_atol=U_ATOL, label=""):
    fluid = case["cell_type"] != 1
    worst = {}
    for a in range(orc.ncomp):
        g = gpu.macro(a)
        o = orc.macro(a)
        rel = np.abs(g[0][fluid] - o[0][fluid]) / np.abs(o[0][fluid])
        du = max(np.abs(g[k][fluid] - o[k][fluid]).max() for k in (1, 2, 3))
        worst[a] = (float(rel.max()), float(du))
        assert rel.max() <= rho_rtol, f"{label} comp {a}: rho rel err {rel.max():.3g}"
        assert du <= u_atol, f"{label} comp {a}: u abs err {du:.3g}"
        solid = case["cell_type"] == 1
        assert np.all(g[0][solid] == 0)
    return worst


def compare_active(gpu, orc, step, S):
    ga, oa = gpu.active_blocks(), orc.active_blocks()
    if not np.array_equal(ga, oa):
        diff = np.setxor1d(ga, oa)
        crit = orc.crit()
        info = {int(b): float(np.sqrt(max(crit[b], 0.0))) for b in diff}
        raise AssertionError(
            f"step {step}: active sets differ on blocks {sorted(info)}; oracle max |du| at "
            f"their borders {info} (S = {S})")
    return len(ga)


def run_pair(L, case, steps, check_active=True, **over):
    gpu = gpu_of(L, case, **over)
    orc = oracle_of(case, **over)
    S = dict(case["params"], **over).get("S", 0.0)
    counts = []
    if check_active:
        counts.append(compare_active(gpu, orc, -1, S))
    for t in range(steps):
        gpu.step(1)
        orc.step(1)
        if check_active:
            counts.append(compare_active(gpu, orc, t, S))
    return gpu, orc, counts


def block_cells(nx, ny, nz, b):
    nbx, nby = nx // 8, ny // 8
    bx, by, bz = b % nbx, (b // nbx) % nby, b // (nbx * nby)
    return bx * 8, by * 8, bz * 8


def order_map(L):
    """Index in the oracle's velocity order of each of the library's."""
    eg = L.velocities()
    eo, _, _ = O.lattice()
    return np.array([[tuple(v) for v in eo].index(tuple(u)) for u in eg])
