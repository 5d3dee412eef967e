"""Benchmark: active-cell MLUPS and fraction of the HBM roofline of the
progressive-mesh two-component LBM step, against the static mesh, on one
GB300 (replicas on N GPUs under torchrun).

Workload: 256^3 liquid injection into a gas-filled porous box (seeded
spheres, radius 6-12, solid fraction 0.30, 64^2 inlet at u = 0.02, wetting
g_ads = -0.2, Peng-Robinson component + ideal-gas component), 5000 time
steps in total, during which the meshed fraction grows from about 1 % to
about 60 %.  A "step" is one time step of the whole hot path (streaming,
moments, criterion and block creation, forces, collision).

Every run goes through the whole 5000-step trajectory: W untimed warm-up
steps, then K timed steps spread evenly over the remaining steps (the
centres of K equal stretches), the steps between them untimed.  So the K
timed steps sample the whole run, early and late, whatever K is.

Timing: every timed step is bracketed by CUDA events on the library's
stream, with a synchronize before it and after it; before each one a
256 MiB buffer is written to flush the 129 MB L2, outside the events.
MLUPS counts 512 cells for every meshed block of every timed step (Eq. 16
with the meshed cells as the domain).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import re
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "active-cell MLUPS (D3Q19, 2 comp) & % HBM roofline vs static mesh, same GPU"
# algorithmic bytes per fluid-cell update: 2 components x 19 populations,
# read + write, 4 B each (FP32 storage) or 2 B (16-bit deviation storage)
BYTES_PER_UPDATE = {"fp32": 304, "fp16": 152, "bf16": 152}
WORKLOAD = ("porous injection 256^3 (seeded spheres r 6-12, solid 0.30, 64^2 inlet u=0.02, "
            "g_ads=-0.2, 2 components), 5000 steps, 8^3 blocks")
CPU_SAMPLE = "64^3 crop of the same recipe (seed 1510035603, 16^2 inlet), progressive mesh"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_code_hash(text):
    """sha256 of kernel source without its // comments, trailing blanks and
    empty lines: changes with the code, not with its comments."""
    lines = (re.sub(r"//.*$", "", line).rstrip() for line in text.splitlines())
    return hashlib.sha256("\n".join(line for line in lines if line).encode()).hexdigest()


def kernel_traffic(storage, which="collide"):
    """ncu DRAM bytes per fluid cell of one storage form's kernel ("fused",
    "collide") or of a whole step ("step"), if the committed capture was
    taken on the current kernel code."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    src = os.path.join(ROOT, "paper_1510_03560_gb300", "csrc", "lbm_step.cuh")
    try:
        with open(path) as fh:
            d = json.load(fh)
        with open(src) as fh:
            h = kernel_code_hash(fh.read())
        if d.get("kernels_code_sha256") == h:
            return float(d["forms"][storage][which + "_dram_bytes_per_fluid_cell"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid=None):
        self.proc = None
        self.uuid = device_uuid

    def __enter__(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "100"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def device_uuid(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


# the other injection workloads: the same recipe on a larger grid (the
# 16-bit storage forms are quoted on it) and a longer porous channel (the
# learned form is quoted on it)
WORKLOADS = {
    "injection384": ("porous injection 384^3 (seed 1510035602, spheres r 6-12, solid 0.30, "
                     "96^2 inlet u=0.02, g_ads=-0.2, 2 components), 8^3 blocks",
                     dict(n=(384, 384, 384), seed=1510035602, inlet=96, x_free=24)),
    "channel512": ("porous channel 512x256x256 (seed 1510035604, spheres r 6-12, solid 0.35, "
                   "64^2 inlet u=0.03, g_ads=-0.2, 2 components), 8^3 blocks",
                   dict(n=(512, 256, 256), seed=1510035604, solid_frac=0.35, inlet=64, u_in=0.03,
                        x_free=16)),
}


def make_case(S=None, size=256, workload="injection", block="8x8x8"):
    from paper_1510_03560_gb300 import workloads as W
    kw = {} if S is None else {"S": S}
    kw["block"] = tuple(int(v) for v in block.split("x"))
    if workload in WORKLOADS:
        kw.update(WORKLOADS[workload][1])
    elif size != 256:
        kw.update(n=(size, size, size), inlet=size // 4, x_free=max(size // 16, 4))
    return W.porous_injection(**kw)


TOTAL_STEPS = 5000  # the workload's run length


def sample_steps(total, warmup, k):
    """k step indices spread evenly over [warmup, total): the centres of k
    equal stretches."""
    span = total - warmup
    if k > span:
        raise ValueError(f"{k} timed steps do not fit in {span} steps after the warm-up")
    return [warmup + (2 * i + 1) * span // (2 * k) for i in range(k)]


def run_timed(L, torch, case, sample, total, progressive, flush, uuid, storage="fp32", proposer=None,
              exec_mode="stream", streaming="ab", slot_order=64, partials=False):
    """Run the whole trajectory of `total` steps, timing the steps listed in
    `sample` one by one (L2 flushed before each, a synchronize on both
    sides); the device time of the whole trajectory is recorded too.
    proposer: an lbm MLP to run the activation proposer with (period 16,
    threshold 0.5).  streaming: "ab" or "aa" (one population array)."""
    sim = L.from_case(case, progressive=progressive, storage=storage, streaming=streaming, partials=partials)
    sim.set_exec(exec_mode)
    sim.set_slot_order(slot_order)
    if proposer is not None:
        sim.set_proposer(proposer, period=16, threshold=0.5)
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    timed, untimed, per_step = [], [], []
    acc = dict(cells=0, fluid=0, launches=0, created=0, prepared=0, prepared_hits=0,
               kernel_ms=[0.0] * 4, kernel_launches=[0] * 4)
    t = 0
    torch.cuda.synchronize()
    with ClockSampler(uuid) as clk:
        for s in list(sample) + [total]:
            if s > t:  # untimed stretch (device time kept for the trajectory figure)
                a, b = ev(), ev()
                a.record(stream)
                sim.step_async(s - t)
                b.record(stream)
                untimed.append((a, b))
                t = s
            if s >= total:
                break
            st0 = sim.stats()  # (synchronizes)
            sim.set_profiling(True)
            flush.zero_()
            torch.cuda.synchronize()
            a, b = ev(), ev()
            a.record(stream)
            sim.step_async(1)
            b.record(stream)
            sim.sync()
            torch.cuda.synchronize()
            sim.set_profiling(False)
            st1 = sim.stats()
            t += 1
            timed.append((a, b))
            d = {k: st1[k] - st0[k] for k in ("cell_updates", "fluid_updates", "launches")}
            acc["cells"] += d["cell_updates"]
            acc["fluid"] += d["fluid_updates"]
            acc["launches"] += d["launches"]
            acc["created"] += st1["created_blocks"] - st0["created_blocks"]
            acc["prepared"] += st1["prepared_blocks"] - st0["prepared_blocks"]
            acc["prepared_hits"] += st1["prepared_hits"] - st0["prepared_hits"]
            for k in range(4):
                acc["kernel_ms"][k] += st1["kernel_ms"][k] - st0["kernel_ms"][k]
                acc["kernel_launches"][k] += st1["kernel_launches"][k] - st0["kernel_launches"][k]
            ms = a.elapsed_time(b)
            per_step.append([s, round(d["cell_updates"] / 512 / st1["total_blocks"], 4), round(ms, 4),
                             round(d["cell_updates"] / (ms * 1e-3) / 1e6, 1)])
        sim.sync()
        torch.cuda.synchronize()
    st = sim.stats()
    ms = sum(a.elapsed_time(b) for a, b in timed)
    traj_ms = ms + sum(a.elapsed_time(b) for a, b in untimed)
    out = dict(acc, ms=ms, per_step=per_step, traj_ms=traj_ms, traj_cells=st["cell_updates"],
               active_end=st["active_blocks"], nonsolid_blocks=st["nonsolid_blocks"],
               total_blocks=st["total_blocks"], device_bytes=st["device_bytes"],
               slot_sorts=st["slot_sorts"], fused_deferred=st["fused_deferred"],
               fused_waited=st["fused_waited"], fused_lag_distance=st["fused_lag_distance"],
               clocks=clk.summary())
    sim.close()
    return out


def run_e2e(L, torch, case, steps, storage="fp32", streaming="ab"):
    """End to end through the public API with host buffers: geometry and
    initial state uploaded, `steps` steps, both components' fields read
    back; wall clock around all of it."""
    import numpy as np
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim = L.from_case(case, storage=storage, streaming=streaming)
    sim.step(steps)
    outs = [sim.macro(a) for a in range(2)]
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    st = sim.stats()
    sim.close()
    h2d = case["cell_type"].nbytes + case["rho_init"].nbytes + case["u_init"].nbytes + 8
    d2h = sum(a.nbytes for o in outs for a in o)
    return dict(wall=wall, cells=st["cell_updates"], h2d=h2d, d2h=d2h, steps=steps,
                checksum=float(np.float64(outs[0][0].sum())))


def oracle_sample(budget_s=15.0, max_steps=None):
    """The FP64 oracle on a bounded sample of the workload: active-cell MLUPS."""
    from oracle import oracle as O
    from paper_1510_03560_gb300 import workloads as W
    case = W.porous_injection(n=(64, 64, 64), seed=1510035603, inlet=16, x_free=4)
    p = dict(case["params"])
    sim = O.OracleSim(case["cell_type"], case["rho_init"], case["u_init"], case["rho_amb"], **p)
    cells, steps, t_used = 0, 0, 0.0
    while t_used < budget_s and (max_steps is None or steps < max_steps):
        t0 = time.perf_counter()
        sim.step(1)
        t_used += time.perf_counter() - t0
        cells += 512 * len(sim.active_blocks())
        steps += 1
    sim.close()
    return dict(mlups=cells / t_used / 1e6, steps=steps, seconds=t_used, cores=O.threads())


def oracle_sample_single_thread(budget_s=8.0):
    """oracle_sample with one OpenMP thread, in a fresh interpreter (the
    thread count is fixed when the oracle library loads)."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_sample(budget_s=%r)))" % (ROOT, budget_s))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                           timeout=budget_s * 6 + 60)
        d = json.loads(r.stdout.strip().splitlines()[-1])
    except Exception:
        return None
    return {"value": round(d["mlups"], 4), "unit": "MLUPS", "cores": d["cores"],
            "sample": f"{CPU_SAMPLE}, {d['steps']} steps, {d['seconds']:.1f} s"}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return None, 0, 1
    import torch.distributed as dist
    backend = "nccl"
    dist.init_process_group(backend=backend)
    return dist, dist.get_rank(), ws


def reduce_max_sum(dist, torch, vmax, vsum, device="cuda"):
    """Whole-job figures of N replicas: the slowest rank's time, the sum of
    the work."""
    if dist is None:
        return vmax, vsum
    t = torch.tensor([vmax], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    s = torch.tensor([vsum], dtype=torch.float64, device=device)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    return float(t.item()), float(s.item())


def run_batch(args):
    """The batching workload: 64 seeded simulations (droplet impacts and
    injections, 32^3 to 128^3) in one context.  Times K steps of the batch
    in each execution mode (the one the autotuner picks is the value), and
    the same simulations run one after another as separate contexts."""
    import torch
    from paper_1510_03560_gb300 import batch as BT
    from paper_1510_03560_gb300 import build as B
    B.build()
    from paper_1510_03560_gb300 import lbm as L
    uuid = device_uuid(torch, 0)
    cases = BT.c3_cases(64)
    # a growing mesh: tune over a window like the timed one
    shape, shape_rates = BT.autotune_shape(L, cases, steps=min(args.steps, 100), warmup=args.warmup)
    batch, place = BT.pack(cases, block=shape)
    best, tune_ms = BT.autotune(L, batch, steps=20)

    def timed(case, mode, steps, warmup):
        sim = L.from_case(case)
        sim.set_exec(mode)
        sim.step(warmup)
        st0 = sim.stats()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(sim.torch_stream)
        sim.step_async(steps)
        b.record(sim.torch_stream)
        sim.sync()
        torch.cuda.synchronize()
        st1 = sim.stats()
        sim.close()
        return a.elapsed_time(b), st1["cell_updates"] - st0["cell_updates"], st1["launches"] - st0["launches"]

    modes = {}
    with ClockSampler(uuid) as clk:
        for m in ("stream", "graph", "persistent", "staged"):
            ms, cells, launches = timed(batch, m, args.steps, args.warmup)
            modes[m] = {"mlups": round(cells / (ms * 1e-3) / 1e6, 1), "ms_per_step": round(ms / args.steps, 5),
                        "launches": launches}
    seq_ms = 0.0
    seq_cells = 0
    for c in cases:
        ms, cells, _ = timed(c, "stream", args.steps, args.warmup)
        seq_ms += ms
        seq_cells += cells
    value = modes[best]["mlups"]
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": modes[best]["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {
            "workload": "batch of 64 seeded simulations (droplet impact or porous injection, "
                        "grids drawn from multiples of 16 in [32, 128]) in one shared block pool",
            "grid": [batch["params"][k] for k in ("nx", "ny", "nz")], "block": list(shape),
            "block_autotuned": {"x".join(map(str, k)): {"ms_per_step": round(v["ms_per_step"], 4),
                                                                 "mlups": round(v["mlups"], 1)}
                                         for k, v in shape_rates.items()},
            "pool_blocks": batch["params"]["max_blocks"], "exec_autotuned": best,
            "autotune_ms_20_steps": {k: round(v, 3) for k, v in tune_ms.items()},
            "modes": modes,
            "sequential_contexts_mlups": round(seq_cells / (seq_ms * 1e-3) / 1e6, 1),
            "batch_over_sequential": round(value / (seq_cells / (seq_ms * 1e-3) / 1e6), 3),
            "l2": "no flush: the batch's populations (GB) exceed the 129 MB L2",
            "kinds": {k: sum(1 for c in cases if c["kind"] == k) for k in ("impact", "injection")},
        },
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    # each "step" a bounded sample: a few oracle steps of the 64^3 crop
    per_step = 2
    total_steps = args.warmup + args.steps
    budget = max(20.0, min(150.0, 1.0 * total_steps))
    r = oracle_sample(budget_s=budget, max_steps=per_step * total_steps)
    line = {
        "metric": METRIC, "value": round(r["mlups"], 4), "unit": "MLUPS", "impl": "reference",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * r["seconds"] / max(r["steps"], 1), 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": CPU_SAMPLE, "oracle_steps": r["steps"]},
        "cpu_baseline": {"value": round(r["mlups"], 4), "unit": "MLUPS", "cores": r["cores"],
                         "kind": "oracle",
                         "sample": f"{CPU_SAMPLE}, {r['steps']} steps, {r['seconds']:.1f} s"},
        "e2e": {"value": round(r["mlups"], 4), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20,
                    help="timed steps, spread evenly over the trajectory after the warm-up")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--total", type=int, default=TOTAL_STEPS,
                    help="length of the trajectory every run goes through (the workload's 5000 steps)")
    ap.add_argument("--fusion", default="off", choices=["on", "off"],
                    help="collision and the next step's pass 1 in one launch (FP32, two components, A-B)")
    ap.add_argument("--partials", default="off", choices=["on", "off"],
                    help="density partials: the collision sums the next step's densities, pass 1 adds "
                         "them instead of pulling (FP32, two components, A-B)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--S", type=float, default=None, help="criterion threshold override")
    ap.add_argument("--no-static", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--size", type=int, default=256,
                    help="grid edge (profiling captures use a smaller grid; the metric is 256)")
    ap.add_argument("--static-only", action="store_true",
                    help="time the static mesh only (profiling captures)")
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp16", "bf16"],
                    help="population storage form (arithmetic is FP32 in all)")
    ap.add_argument("--workload", default="injection",
                    choices=["injection", "batch", "injection384", "channel512"],
                    help="injection: the 256^3 headline; batch: 64 small simulations in one pool; "
                         "injection384 / channel512: the grids the 16-bit and learned forms are "
                         "quoted on")
    ap.add_argument("--exec", default="stream", choices=["stream", "graph", "persistent", "staged"],
                    help="how the library enqueues the steps")
    ap.add_argument("--block", default="8x8x8", choices=["8x8x8", "16x8x4", "16x4x8", "32x4x4"],
                    help="cells per block along x, y, z")
    ap.add_argument("--slot-order", type=int, default=64,
                    help="steps between checks for renumbering the meshed slots in block order (0: never)")
    ap.add_argument("--streaming", default="ab", choices=["ab", "aa"],
                    help="population streaming pattern: two arrays (A-B) or one updated in place (A-A)")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip timing the FP16, BF16, A-A and learned-proposer forms")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    import torch
    dist, rank, world = dist_setup()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    from paper_1510_03560_gb300 import build as B
    if rank == 0 or dist is None:
        B.build()
    if dist is not None:
        dist.barrier()
    from paper_1510_03560_gb300 import lbm as L
    uuid = device_uuid(torch, local)
    case = make_case(args.S, args.size, args.workload, args.block)
    case["params"]["fusion"] = (args.fusion == "on", 0)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    sample = sample_steps(args.total, args.warmup, args.steps)
    if args.static_only:
        st = run_timed(L, torch, case, sample, args.total, 0, flush, uuid, args.storage,
                       exec_mode=args.exec, streaming=args.streaming, partials=args.partials == "on")
        if rank == 0:
            print(json.dumps({"static_mlups": st["cells"] / (st["ms"] * 1e-3) / 1e6,
                              "ms": st["ms"], "kernel_ms": st["kernel_ms"],
                              "kernel_launches": st["kernel_launches"], "fusion": args.fusion}), flush=True)
        return 0

    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    prog = run_timed(L, torch, case, sample, args.total, 1, flush, uuid, args.storage,
                     exec_mode=args.exec, streaming=args.streaming, slot_order=args.slot_order,
                     partials=args.partials == "on")
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t_max, cells_sum = reduce_max_sum(dist, torch, prog["ms"], prog["cells"])

    stat = None
    if not args.no_static:
        stat = run_timed(L, torch, case, sample, args.total, 0, flush, uuid, args.storage,
                         streaming=args.streaming, partials=args.partials == "on")
        s_max, s_cells = reduce_max_sum(dist, torch, stat["ms"], stat["cells"])
    forms = {}

    def form_line(r, **extra):
        f_max, f_cells = reduce_max_sum(dist, torch, r["ms"], r["cells"])
        d = {"mlups": round(f_cells / (f_max * 1e-3) / 1e6, 1),
             "fluid_mlups": round(r["fluid"] / (r["ms"] * 1e-3) / 1e6, 1),
             "active_fraction_end": round(r["active_end"] / r["total_blocks"], 4),
             "collide_ms_per_step": round(r["kernel_ms"][2] / args.steps, 5)}
        d.update(extra)
        return d

    if not args.no_forms and args.storage == "fp32" and args.streaming == "ab":
        from paper_1510_03560_gb300 import proposer as PR
        r = run_timed(L, torch, case, sample, args.total, 1, flush, uuid, "fp32", streaming="aa")
        forms["aa"] = form_line(r, macro_ms_per_step=round(r["kernel_ms"][0] / args.steps, 5),
                                device_bytes=r["device_bytes"], device_bytes_ab=prog["device_bytes"],
                                streaming="A-A: one population array updated in place")
        for form in ("fp16", "bf16"):
            r = run_timed(L, torch, case, sample, args.total, 1, flush, uuid, form)
            forms[form] = form_line(r)
            if not args.no_static:
                # the same kernels on the same (static) cells as the FP32 static arm
                r = run_timed(L, torch, case, sample, args.total, 0, flush, uuid, form)
                forms[form + "_static"] = form_line(r)
        mlp = PR.load_model(L)
        r = run_timed(L, torch, case, sample, args.total, 1, flush, uuid, "fp32", proposer=mlp)
        forms["learned"] = form_line(
            r, created=r["created"], prepared=r["prepared"], prepared_hits=r["prepared_hits"],
            activate_ms_per_step=round(r["kernel_ms"][1] / args.steps, 5),
            activate_ms_per_step_without=round(prog["kernel_ms"][1] / args.steps, 5),
            period=16, threshold=0.5, inference="bf16 operands, fp32 accumulation")
        mlp.close()
    e2e = None if args.no_e2e else run_e2e(L, torch, case, args.total, args.storage, args.streaming)
    if e2e is not None:
        e_max, e_cells = reduce_max_sum(dist, torch, e2e["wall"], e2e["cells"])

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    peak, peak_kind = peaks()
    bpu = BYTES_PER_UPDATE[args.storage]
    mlups = cells_sum / (t_max * 1e-3) / 1e6
    # algorithmic bytes: 304 B for every fluid cell updated (solid cells move
    # no data, held cells are read by their neighbours but never written)
    step_frac = prog["fluid"] * bpu / (prog["ms"] * 1e-3) / 1e9 / peak
    # dominant kernel: the collision launch (kind 2); fused, it also runs the
    # next step's pass 1, so its algorithmic bytes are the whole step's
    fused = args.fusion == "on" and args.storage == "fp32" and args.streaming == "ab" and \
        args.exec in ("stream", "graph")
    kms, kn = prog["kernel_ms"][2], prog["kernel_launches"][2]
    coll_gbs = prog["fluid"] * bpu / (kms * 1e-3) / 1e9 if kms > 0 else None
    traffic_pc = kernel_traffic(args.storage, "fused" if fused else "collide") if args.streaming == "ab" else None
    avg_cells = prog["cells"] / max(kn, 1)
    avg_fluid = prog["fluid"] / max(kn, 1)
    roofline = {
        "bound": "hbm", "achieved": round(coll_gbs, 1) if coll_gbs else None,
        "peak": peak, "unit": "GB/s",
        "frac": round(coll_gbs / peak, 4) if coll_gbs else None,
        "traffic": round(traffic_pc * avg_fluid) if traffic_pc else None,
        "kernel": ("k_fused2 (collision of step t: pull, force gather, exact-difference collision; "
                   "pass 1 of step t+1: pull, densities, psi, criterion)" if fused else
                   "k_collide (force gather + exact-difference collision + pull streaming)"
                   if args.streaming == "ab" else
                   "k_collide_aa (force gather + exact-difference collision, A-A in place)"),
        "peak_kind": peak_kind,
        "algorithmic_bytes_per_launch": round(avg_fluid * bpu),
        "avg_launch_ms": round(kms / max(kn, 1), 5),
        "traffic_basis": "ncu dram bytes per fluid cell of the kernel (profiles/traffic.json) x "
                         "the launch's fluid cells",
    }
    share = {name: round(v / max(sum(prog["kernel_ms"]), 1e-9), 4)
             for name, v in zip(("macro", "activate", "collide", "other"), prog["kernel_ms"])}
    config = {
        "workload": (WORKLOADS[args.workload][0] if args.workload in WORKLOADS
                     else WORKLOAD if args.size == 256 else f"{args.size}^3 variant of: {WORKLOAD}"
                     ).replace("8^3 blocks", "8^3 blocks" if args.block == "8x8x8" else f"{args.block} blocks"),
        "mode": "progressive", "grid": [case["params"][k] for k in ("nx", "ny", "nz")],
        "block": list(case["params"]["block"]),
        "storage": args.storage, "exec": args.exec, "streaming": args.streaming, "fusion": args.fusion,
        "density_partials": args.partials,
        "slot_order_period": args.slot_order, "slot_sorts": prog["slot_sorts"],
        "S": case["params"]["S"],
        "trajectory_steps": args.total, "timed_steps": sample,
        "timing": f"{args.steps} steps spread evenly over steps {args.warmup}..{args.total - 1} of the "
                  f"{args.total}-step trajectory (the rest run untimed)",
        "samples": {"columns": ["step", "meshed_fraction", "ms", "mlups"], "rows": prog["per_step"]},
        "active_fraction_end": round(prog["active_end"] / prog["total_blocks"], 4),
        "mean_active_fraction": round(prog["cells"] / 512 / args.steps / prog["total_blocks"], 4),
        "trajectory_mlups": round(prog["traj_cells"] / (prog["traj_ms"] * 1e-3) / 1e6, 1),
        "step_hbm_frac": round(step_frac, 4), "kernel_time_share": share,
        "fluid_mlups": round(prog["fluid"] / (prog["ms"] * 1e-3) / 1e6, 1),
        "fused_deferred_items": prog["fused_deferred"], "fused_waited_items": prog["fused_waited"],
        "fused_lag_distance": prog["fused_lag_distance"],
        "l2": "256 MiB buffer written before every timed step; flush outside the timed events",
        "parallelism": f"replicas x{world}",
    }
    step_traffic = kernel_traffic(args.storage, "step") if args.streaming == "ab" else None
    if step_traffic:
        config["step_dram_bytes_per_fluid_cell"] = step_traffic
    if forms:
        forms["fp32_progressive_mlups"] = round(mlups, 1)
        config["forms"] = forms
    if stat is not None:
        s_mlups = s_cells / (s_max * 1e-3) / 1e6
        config["static_mlups"] = round(s_mlups, 1)
        config["static_step_hbm_frac"] = round(
            stat["fluid"] * bpu / (stat["ms"] * 1e-3) / 1e9 / peak, 4)
        config["progressive_over_static_time"] = round(prog["ms"] / stat["ms"], 4)
    cpu = None
    if not args.no_cpu:
        r = oracle_sample(budget_s=15.0)
        cpu = {"value": round(r["mlups"], 4), "unit": "MLUPS", "cores": r["cores"],
               "kind": "oracle",
               "sample": f"{CPU_SAMPLE}, {r['steps']} steps, {r['seconds']:.1f} s"}
        one = oracle_sample_single_thread(budget_s=8.0)
        if one is not None:
            cpu["single_thread"] = one
    line = {
        "metric": METRIC, "value": round(mlups, 1), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_max / args.steps, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": config, "roofline": roofline, "cpu_baseline": cpu,
        "clocks": prog["clocks"],
        "gpu_launches": prog["launches"],
    }
    if e2e is not None:
        line["e2e"] = {"value": round(e_cells / e_max / 1e6, 1), "unit": "MLUPS",
                       "h2d_bytes_per_step": round(e2e["h2d"] / e2e["steps"], 1),
                       "d2h_bytes_per_step": round(e2e["d2h"] / e2e["steps"], 1)}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
