"""Many independent simulations in one context: one block pool, one set of
launches per step for all of them.

Each simulation is placed at a block-aligned offset of one large walled
grid, with at least one all-solid block between any two of them.  Its
cells then see exactly the neighbourhood they see alone in a box with solid
outside, and no block of one simulation is ever a creation target of
another (the blocks between them are fully solid and never meshed), so each
simulation evolves bit for bit as it does alone.  The library's neighbour
tables cover only meshed blocks, so the empty space of the packing costs
table entries, not work or population memory (the pool capacity is the sum
of the simulations' non-solid blocks).  The simulations must share the
physics and the ambient state.

The execution mode (lbm_set_exec) that suits a batch is chosen by
`autotune`, which times each mode on a scratch context; the block shape by
`autotune_shape`, which packs and times the batch once per shape that tiles
every member.
"""
from __future__ import annotations

import math

import numpy as np

from . import workloads as W

EDGE = 8     # the default block, 8 x 8 x 8 cells
SIZES = tuple(range(32, 129, 16))


def c3_cases(count: int = 64, seed0: int = 1510035700):
    """The batching workload: `count` seeded simulations, each a droplet
    impact or an injection (probability 1/2), with dimensions drawn
    uniformly from the multiples of 16 in [32, 128]."""
    out = []
    for k in range(count):
        rng = np.random.default_rng(seed0 + k)
        dims = tuple(int(v) for v in rng.choice(SIZES, 3))
        if rng.random() < 0.5:
            case = W.droplet_impact(n=dims, seed=seed0 + k)
            kind = "impact"
        else:
            inlet = max(8, min(dims[1], dims[2]) // 4)
            case = W.porous_injection(n=dims, seed=seed0 + k, inlet=inlet, x_free=max(dims[0] // 16, 4))
            kind = "injection"
        case["kind"] = kind
        out.append(case)
    return out


def _shared_params(cases):
    keys = set().union(*(c["params"].keys() for c in cases)) - {"nx", "ny", "nz", "max_blocks", "block"}
    p0 = cases[0]["params"]
    for c in cases[1:]:
        for k in keys:
            if c["params"].get(k) != p0.get(k):
                raise ValueError(f"batched simulations must share parameter {k!r}")
        if not np.array_equal(c["rho_amb"], cases[0]["rho_amb"]):
            raise ValueError("batched simulations must share the ambient state")
    if any(p0.get("periodic", (0, 0, 0))):
        raise ValueError("batched simulations must be walled (non-periodic)")
    return {k: p0[k] for k in keys if k in p0}


def nonsolid_blocks(cell_type, block=(EDGE, EDGE, EDGE)) -> int:
    nz, ny, nx = cell_type.shape
    bx, by, bz = block
    b = (cell_type != W.SOLID).reshape(nz // bz, bz, ny // by, by, nx // bx, bx)
    return int(b.any(axis=(1, 3, 5)).sum())


def tiles(cases, block) -> bool:
    """Whether every simulation's size is a multiple of the block."""
    return all(c["params"][k] % b == 0 for c in cases for k, b in zip(("nx", "ny", "nz"), block))


def pack(cases, width: int | None = None, block=(EDGE, EDGE, EDGE)):
    """One case holding every simulation: shelf packing in x-y (rows of the
    given width, tallest first), one layer in z, one all-solid block between
    neighbours.  Returns (case, placements), placements[k] = (x0, y0, z0,
    nx, ny, nz) of simulation k."""
    shared = _shared_params(cases)
    bx, by, _ = block
    dims = [(c["params"]["nx"], c["params"]["ny"], c["params"]["nz"]) for c in cases]
    if not tiles(cases, block):
        raise ValueError(f"simulation sizes must be multiples of the {block} block")
    if width is None:
        area = sum((d[0] + bx) * (d[1] + by) for d in dims)
        width = max(max(d[0] for d in dims), int(math.ceil(math.sqrt(area) / bx)) * bx)
    order = sorted(range(len(cases)), key=lambda i: (-dims[i][1], -dims[i][0], i))
    place = [None] * len(cases)
    x = y = row_h = 0
    for i in order:
        nx, ny, nz = dims[i]
        if x > 0 and x + nx > width:
            y += row_h + by
            x = row_h = 0
        place[i] = (x, y, 0, nx, ny, nz)
        x += nx + bx
        row_h = max(row_h, ny)
    NX = max(p[0] + p[3] for p in place)
    NY = max(p[1] + p[4] for p in place)
    NZ = max(p[5] for p in place)
    ncomp = cases[0]["rho_init"].shape[0]
    ct = np.full((NZ, NY, NX), W.SOLID, dtype=np.uint8)
    rho = np.empty((ncomp, NZ, NY, NX), dtype=np.float32)
    for a in range(ncomp):
        rho[a] = cases[0]["rho_amb"][a]
    u = np.zeros((ncomp, 3, NZ, NY, NX), dtype=np.float32)
    for c, (x0, y0, z0, nx, ny, nz) in zip(cases, place):
        sl = (slice(z0, z0 + nz), slice(y0, y0 + ny), slice(x0, x0 + nx))
        ct[sl] = c["cell_type"]
        rho[(slice(None),) + sl] = c["rho_init"]
        if c["u_init"] is not None:
            u[(slice(None), slice(None)) + sl] = c["u_init"]
    params = dict(shared, nx=NX, ny=NY, nz=NZ, block=tuple(block),
                  max_blocks=sum(nonsolid_blocks(c["cell_type"], block) for c in cases))
    batch = dict(cell_type=ct, rho_init=rho, u_init=u, rho_amb=cases[0]["rho_amb"].copy(),
                 params=params)
    return batch, place


def split(field, placements):
    """Per-simulation views of a batch field ([..., z, y, x])."""
    return [field[..., z0:z0 + nz, y0:y0 + ny, x0:x0 + nx]
            for (x0, y0, z0, nx, ny, nz) in placements]


def block_map(batch_params, placements, k):
    """Batch block id of every block of simulation k, [nbz][nby][nbx]."""
    ex, ey, ez = batch_params.get("block", (EDGE, EDGE, EDGE))
    NBX, NBY = batch_params["nx"] // ex, batch_params["ny"] // ey
    x0, y0, z0, nx, ny, nz = placements[k]
    bz, by, bx = np.meshgrid(np.arange(nz // ez), np.arange(ny // ey), np.arange(nx // ex),
                             indexing="ij")
    return (x0 // ex + bx) + NBX * ((y0 // ey + by) + NBY * (z0 // ez + bz))


def autotune(L, case, steps: int = 40, modes=("stream", "graph", "persistent", "staged"), storage="fp32"):
    """Time `steps` steps in each execution mode on a scratch context (CUDA
    events on the library's stream) and return (best mode, {mode: ms})."""
    import torch
    times = {}
    for m in modes:
        sim = L.from_case(case, storage=storage)
        sim.set_exec(m)
        sim.step(4)
        stream = sim.torch_stream
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.step_async(steps)
        b.record(stream)
        sim.sync()
        torch.cuda.synchronize()
        times[m] = a.elapsed_time(b)
        sim.close()
    return min(times, key=times.get), times


def autotune_shape(L, cases, shapes=None, steps: int = 40, warmup: int = 4, exec_mode="stream"):
    """Pack the simulations once per block shape that tiles all of them
    (default: every shape of the library), time `steps` steps after
    `warmup` (CUDA events on the library's stream) and return (the shape
    with the least time per step, {shape: {"ms_per_step", "mlups"}}).  The
    time decides, not the cell-update rate: a coarser shape meshes more
    cells for the same simulations."""
    import torch
    res = {}
    for shape in shapes or L.SHAPES:
        if not tiles(cases, shape):
            continue
        batch, _ = pack(cases, block=shape)
        sim = L.from_case(batch)
        sim.set_exec(exec_mode)
        sim.step(warmup)
        st0 = sim.stats()
        stream = sim.torch_stream
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.step_async(steps)
        b.record(stream)
        sim.sync()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        cells = sim.stats()["cell_updates"] - st0["cell_updates"]
        res[tuple(shape)] = {"ms_per_step": ms / steps, "mlups": cells / (ms * 1e-3) / 1e6}
        sim.close()
    return min(res, key=lambda k: res[k]["ms_per_step"]), res
