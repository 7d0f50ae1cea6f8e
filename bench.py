"""Benchmark: batched RVE homogenisation throughput on one GB300 (or N, weak scaling).

Workload (one step): the batched FE^2 evaluation of 4096 macro Gauss points per
GPU, each with its own degradation state (T ~ U(20,60) C, moisture ~ U(0,1.5)
wt%, time = 10^U(0,4) h; one batch of 4096 x N points from seed 2, split over N
ranks into blocks of equal estimated cost), RVE plain-weave grids 16x16x6 / 24x24x8 /
32x32x10 and order p in {1,2} drawn uniformly, periodic BC; each point solves
6 mechanical + 3 thermal + 3 moisture cell problems and returns C, K, D.
Mixed precision: FP32 operator and vectors, FP64 scalars / reductions and
FP64 residual refinement.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
instead (bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import rve_inputs as ri  # noqa: E402

METRIC = "RVE homogenisations/s on 1 GB300: batched PCG vs surrogate at ≤1e-2 rel err"
UNIT = "homogenisations/s"
G_POINTS = 4096
SEED = 2
WORKLOAD = ("batched FE2 evaluation: 4096 macro Gauss points per GPU, plain-weave RVEs on "
            "16x16x6 / 24x24x8 / 32x32x10 Kuhn grids, p in {1,2}, periodic BC, 12 load cases "
            "per RVE (6 mech + 3 thermal + 3 moisture), degradation state per point from the "
            "Sec. 4 law, FP32 operator and inner PCG, double-float true residual, FP64 reductions")
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
RTOL = 1e-5          # FP64 outer (true-residual) tolerance of every cell solve
INNER_RTOL = 5e-6    # FP32 inner PCG tolerance per refinement sweep
WARM_START = 4       # batches start from the energy-optimal combination of the previous batch's solutions
# One ncu capture of the current p = 2 mechanical operator (one launch on the 32x32x10
# weave, 8 RVEs, all 48 columns active): DRAM read + write bytes of that launch against its
# algorithmic bytes.  The bench scales the ratio to its own mean launch of that
# instance (traffic grows with the columns and elements processed); None for other kernels.
TRAFFIC_KERNEL = "k_operator<p=2,mech,f32>"
TRAFFIC_CAPTURE = {"case": "k_operator<2,3,float>, 32x32x10 p=2 periodic, 8 RVEs (48 columns, all active)",
                   "dram_bytes": 116.65e6, "algorithmic_bytes": 104.5e6, "ratio": 116.65 / 104.5}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--points", type=int, default=G_POINTS)
    ap.add_argument("--batch", type=int, default=0)
    ap.add_argument("--warm-start", type=int, default=WARM_START,
                    help="0 cold batches; 1 nearest, 2 line, 3 parabola through previous solutions, "
                         "4 their energy-optimal combination")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-macro", action="store_true", help="skip the coupled macro time-stepping leg")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the transport-once-per-mesh variant measured beside the main line")
    ap.add_argument("--no-autotune", action="store_true",
                    help="built-in batch-size rule instead of the per-mesh autotuner")
    ap.add_argument("--surrogate-points", type=int, default=1 << 20)
    return ap.parse_args()


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return world, rank, local


def max_over_ranks(v: float, world: int) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(v: float, world: int) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for i, n in enumerate(names):
                    if r[5 + i].strip().lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ workload
def build_meshes(ctx, rve):
    """The six mesh classes (3 grids x 2 orders), periodic BC, nominal constituents."""
    meshes, classes = [], []
    for si, grid in enumerate(ri.SIZE_CLASSES):
        xyz, tets, phase, tangent = ri.weave_rve(*grid)
        for p in ri.P_CLASSES:
            m = ctx.mesh_load(xyz, tets, p, phase, tangent)
            m.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
            m.set_bc(rve.BC_PERIODIC)
            meshes.append(m)
            classes.append((si, p))
    return meshes, classes


TUNE_SEED = 1000
KERNEL_NAMES = {1: "cuda_core", 2: "tensor_tf32x3"}
TUNE_MAX_ENTRIES = 64e6      # candidate batch sizes keep one FP64 vector within 512 MB


def autotune(meshes, classes, n_points, rank):
    """Batch size per mesh from rve_autotune_batch, on a tuning sample of the same
    state distribution (its own seed) and about as many points per mesh as the
    timed workload; runs before the warm-up, outside every timed region."""
    T, c, t, size, p = ri.gauss_point_states(n_points, TUNE_SEED + rank)
    mid = mesh_ids(size, p, classes)
    chosen = {}
    for i, (m, (si, q)) in enumerate(zip(meshes, classes)):
        sel = mid == i
        rows = 3 * m.info()["n_scalar_dofs"]
        cand = [b for b in (8, 16, 32, 64, 128, 256) if rows * 6 * b <= TUNE_MAX_ENTRIES] or [8]
        name = "x".join(map(str, ri.SIZE_CLASSES[si])) + f" p={q}"
        if len(cand) == 1 or sel.sum() < 2:
            chosen[name] = {"batch": cand[0], "rates": None}
            continue
        if q >= 2:
            # schedule: batch size and operator kernel (tensor cores or CUDA cores)
            best, kern, rates = m.autotune_schedule(T[sel], c[sel], t[sel], cand)
            chosen[name] = {"batch": best, "kernel": KERNEL_NAMES[kern],
                            "rates": {f"{KERNEL_NAMES[k]} b{b}": round(v, 1) for (k, b), v in rates.items()}}
        else:
            best, rates = m.autotune_batch(T[sel], c[sel], t[sel], cand)
            chosen[name] = {"batch": best, "kernel": "cuda_core (matrix-free)",
                            "rates": {str(k): round(v, 1) for k, v in rates.items()}}
    return chosen


def mesh_ids(size, p, classes):
    lut = {c: i for i, c in enumerate(classes)}
    return np.array([lut[(int(s), int(q))] for s, q in zip(size, p)], np.int32)


def run_ours(args, world, rank, local):
    # the CPU oracle's per-class timings run in spawned worker processes on the
    # host cores while the GPU legs run (started before the first GPU call)
    cpu_pool = cpu_baseline_start() if (rank == 0 and not args.no_cpu_baseline and world == 1) else None
    import torch
    import paper_1610_03484_gb300 as rve
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    ctx = rve.Context(precision=rve.PREC_MIXED, rtol=RTOL, inner_rtol=INNER_RTOL, max_refine=4,
                      batch=args.batch, stream=stream.cuda_stream, device=local,
                      warm_start=args.warm_start)
    meshes, classes = build_meshes(ctx, rve)
    tuned = autotune(meshes, classes, args.points, rank) if not args.no_autotune and args.batch == 0 else None
    # one seeded batch of points x world Gauss points; with several ranks it is split
    # into contiguous blocks of equal estimated cost (DOFs x expected iterations)
    # and every step ends with the gather of the 33 tensor values per point
    G_total = args.points * world
    T, c, t, size, p = ri.gauss_point_states(G_total, SEED)
    mid = mesh_ids(size, p, classes)
    shard = None
    if world > 1:
        from paper_1610_03484_gb300 import sharding
        dofs = [3 * m.info()["n_scalar_dofs"] for m in meshes]
        cost = sharding.point_costs(dofs, [ri.SIZE_CLASSES[si] for si, _ in classes], [q for _, q in classes], mid)
        off, imb = rve.partition_blocks(cost, world)
        lo, hi = int(off[rank]), int(off[rank + 1])
        T, c, t, size, p, mid = T[lo:hi], c[lo:hi], t[lo:hi], size[lo:hi], p[lo:hi], mid[lo:hi]
        shard = {"offsets": off, "imbalance": imb, "module": sharding}
    G = len(T)
    # device-resident inputs / outputs for `value`
    Td = torch.tensor(T, dtype=torch.float64, device=dev)
    cd = torch.tensor(c, dtype=torch.float64, device=dev)
    td = torch.tensor(t, dtype=torch.float64, device=dev)
    Cd = torch.zeros((G, 36), dtype=torch.float64, device=dev)
    Kd = torch.zeros((G, 9), dtype=torch.float64, device=dev)
    Dd = torch.zeros((G, 9), dtype=torch.float64, device=dev)
    Sd = torch.zeros(G, dtype=torch.int32, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2

    def step():
        st, rc = ctx.macro_update_dev(meshes, Td.data_ptr(), cd.data_ptr(), td.data_ptr(), mid,
                                      Cd.data_ptr(), Kd.data_ptr(), Dd.data_ptr(), Sd.data_ptr())
        if shard is not None:   # the data-path collective: every rank gets the whole batch
            sh = shard["module"]
            local = sh.pack(Cd.cpu().numpy(), Kd.cpu().numpy(), Dd.cpu().numpy(), Sd.cpu().numpy())
            shard["result"] = sh.gather_blocks(local, shard["offsets"])
        return st

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    launches = 0
    graph_ms, graphs = 0.0, 0
    times = []
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = step()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        launches += st["kernel_launches"]
        graph_ms += st["graph_host_ms"]
        graphs += st["graphs"]
    barrier(world)
    clk = clocks.stop()
    status = Sd.cpu().numpy()
    if not (status == 0).all():
        raise RuntimeError(f"timed leg: {int((status != 0).sum())} points not converged")
    C_timed, K_timed, D_timed = Cd.cpu().numpy(), Kd.cpu().numpy(), Dd.cpu().numpy()
    # one more step of the same workload with every operator launch bracketed by
    # CUDA events on the launching stream (profile mode replaces the graph
    # replay by direct launches); gives the operator's mean launch duration
    ctx.set_options(profile=1)
    flush.fill_(1.0)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st = step()
    e1.record(stream)
    torch.cuda.synchronize()
    prof_step_ms = e0.elapsed_time(e1)
    ctx.set_options(profile=0)
    op_ms, op_n, op_bytes, op_flops = st["op_ms"], st["op_launches"], st["op_bytes"], st["op_flops"]
    # variant, reported beside `value`: the thermal and moisture cell problems
    # (not degraded, so the same for every point of a mesh) solved once per mesh
    # and call instead of once per point
    variant = None
    if not args.no_variants:
        ctx.set_options(transport_once=1)
        step()
        vt = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            torch.cuda.synchronize()
            vt.append(e0.elapsed_time(e1))
        ctx.set_options(transport_once=0)
        v_s = max_over_ranks(sum(vt) / 1000.0, world)
        variant = {"transport_once_per_mesh": {
            "value": sum_over_ranks(G * args.steps, world) / v_s, "unit": UNIT,
            "what": "3 + 3 transport load cases solved once per mesh and call (they do not depend on the "
                    "degradation state), 6 mechanical load cases per point; same points, same tolerance"}}
    local_s = sum(times) / 1000.0
    job_s = max_over_ranks(local_s, world)
    units = sum_over_ranks(G * args.steps, world)
    value = units / job_s
    if shard is not None and not (shard["result"][:, 33] == 0).all():
        raise RuntimeError("gathered batch: some points not converged")

    # end to end through the host-buffer entry point (pinned host memory)
    Th = torch.tensor(T).pin_memory()
    ch = torch.tensor(c).pin_memory()
    th = torch.tensor(t).pin_memory()
    e2e_times, e2e_ok = [], 0
    for _ in range(max(1, args.steps)):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # a point that did not converge raises here (RVE_ERR_NOT_CONVERGED is not accepted)
        Cc, Kk, Ddd, stt, _, _ = ctx.macro_update(meshes, Th.numpy(), ch.numpy(), th.numpy(), mid)
        e2e_times.append(time.perf_counter() - t0)
        e2e_ok += int((stt == 0).sum())
    if e2e_ok != G * len(e2e_times):
        raise RuntimeError(f"end-to-end leg: {G * len(e2e_times) - e2e_ok} points not converged")
    e2e_s = max_over_ranks(sum(e2e_times), world)
    e2e_value = sum_over_ranks(G * len(e2e_times), world) / e2e_s

    check = self_check(ctx, rve, meshes, classes, T, c, t, size, p, C_timed, K_timed, D_timed)

    pk, pk_kind = peaks()
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": job_s * 1000.0 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "points_per_gpu": G, "points_total": G_total, "seed": SEED,
                   "bc": "periodic",
                   "sharding": (None if shard is None else
                                {"blocks": "contiguous, balanced by DOFs x expected iterations",
                                 "offsets": [int(x) for x in shard["offsets"]],
                                 "cost_imbalance": shard["imbalance"],
                                 "collective": "all_gather of 33 FP64 values + status per point, "
                                               "inside every timed step"}),
                   "precision": "FP32 operator and inner PCG; double-float true residual; FP64 scalars, "
                                "reductions and solution", "rtol": RTOL,
                   "inner_rtol": INNER_RTOL, "warm_start": args.warm_start,
                   "batch_per_mesh": tuned if tuned is not None else "built-in rule",
                   "l2": "256 MB buffer written between timed steps; per-step working set >> 129 MB L2",
                   "status_ok": int((status == 0).sum())},
        "self_check": check,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": G * 3 * 8,
                "d2h_bytes_per_step": G * (36 + 9 + 9) * 8 + G * 4,
                "points_converged": e2e_ok, "points": G * len(e2e_times)},
        "gpu_launches": int(launches),
        "variants": variant,
        "host_overhead": {"graph_build_ms_per_step": graph_ms / args.steps,
                          "graphs_per_step": graphs / args.steps},
        "clocks": clk,
        "roofline": None,
        "cpu_baseline": None,
    }
    if op_n > 0:
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        result["roofline"] = roofline(st, prof_step_ms, pk, pk_kind, clk, n_sm)
    if cpu_pool is not None:
        result["cpu_baseline"] = cpu_baseline_collect(cpu_pool)
    if not args.no_surrogate:
        result["surrogate"] = surrogate_leg(ctx, rve, args.surrogate_points, rank)
    if not args.no_macro:
        result["macro_coupled"] = macro_leg(ctx, rve, rank)
    for m in meshes:
        m.free()
    ctx.close()
    return result


def roofline(st, step_ms, pk, pk_kind, clk, n_sm):
    """Roofline of the step's kernels from one profiled step of the same workload:
    every launch of the PCG iteration is bracketed by CUDA events on its stream
    and its algorithmic bytes (and, for the operator, flops) are counted by the
    library, per operator instance (order p x field).  The dominant kernel (the
    largest share of the step) fills the top-level fields with its HBM fraction:
    algorithmic bytes per launch / mean launch time / the measured copy
    bandwidth.  Its FP32-ALU fraction (against a peak derived from the device's
    SM count and the sampled clock) is reported beside it."""
    hbm_peak = pk["hbm_gbs"]
    mhz = clk.get("sm_mhz") or pk.get("sm_max_mhz", 2070.0)
    fp32_peak = n_sm * 128 * 2 * mhz * 1e6 / 1e12      # FP32 CUDA-core FMA peak at the sampled clock

    def op_entry(ms, n, by, fl, act):
        sec = ms / 1e3
        e = {"launches": n, "mean_launch_ms": ms / n, "share_of_step": ms / step_ms,
             "hbm_gbs": by / sec / 1e9, "hbm_frac": by / sec / 1e9 / hbm_peak,
             "tflops": fl / sec / 1e12, "alu_frac": fl / sec / 1e12 / fp32_peak,
             "bytes_per_launch": by / n, "flops_per_launch": fl / n, "active_column_frac": act}
        e["bound"] = "alu" if e["alu_frac"] >= e["hbm_frac"] else "hbm"
        return e

    kernels = {}
    for k in range(6):
        n = st["op_class_launches"][k]
        if n > 0:
            name = f"k_operator<p={k // 2 + 1},{'mech' if k % 2 == 0 else 'scalar'},f32>"
            kernels[name] = op_entry(st["op_class_ms"][k], n, st["op_class_bytes"][k],
                                     st["op_class_flops"][k], st["op_class_active_frac"][k])
    n = st["op_launches"]
    kernels["k_operator (all instances)"] = op_entry(st["op_ms"], n, st["op_bytes"], st["op_flops"],
                                                     st["op_active_frac"])
    for name, ms, by in (("k_update", st["update_ms"], st["update_bytes"]),
                         ("k_pupdate", st["pupdate_ms"], st["pupdate_bytes"])):
        kernels[name] = {"launches": n, "mean_launch_ms": ms / n, "share_of_step": ms / step_ms,
                         "hbm_gbs": by / (ms / 1e3) / 1e9, "hbm_frac": by / (ms / 1e3) / 1e9 / hbm_peak,
                         "bytes_per_launch": by / n, "bound": "hbm"}
    kernels["finalize (alpha, beta)"] = {"share_of_step": st["finalize_ms"] / step_ms}
    kernels["true residual (double-float)"] = {"launches": st["residual_launches"],
                                               "share_of_step": st["residual_ms"] / step_ms}
    cands = [k for k, v in kernels.items() if "bound" in v and not k.endswith("(all instances)")]
    dom = max(cands, key=lambda k: kernels[k]["share_of_step"])
    out = {"how": "one extra step of the same workload after the timed ones, every PCG-iteration launch "
                  "bracketed by CUDA events on its stream; bytes and flops are algorithmic, counted for "
                  "the columns still iterating; frac = achieved / peak with achieved = bytes_per_launch / "
                  "mean_launch_ms of the dominant kernel (HBM roofline)",
           "profiled_step_ms": step_ms, "kernels": kernels, "kernel": dom,
           "traffic": (TRAFFIC_CAPTURE["ratio"] * kernels[dom]["bytes_per_launch"]
                       if dom == TRAFFIC_KERNEL else None),
           "traffic_capture": TRAFFIC_CAPTURE,
           "peaks": {"hbm_gbs": hbm_peak, "hbm_kind": f"{pk_kind} (copy bandwidth)",
                     "fp32_tflops": fp32_peak,
                     "fp32_kind": f"derived, not measured: {n_sm} SM (device query) x 128 FP32 lanes x 2 x "
                                  f"{mhz:.0f} MHz (sampled median)"}}
    k = kernels[dom]
    out.update({"bound": "hbm", "achieved": k["hbm_gbs"], "peak": hbm_peak, "unit": "GB/s",
                "frac": k["hbm_frac"], "alu_frac_derived": k.get("alu_frac"),
                "binding_roof": k["bound"]})
    return out


# ------------------------------------------------------------ surrogate leg
SURROGATE_FILE = os.path.join(ROOT, "paper_1610_03484_gb300", "surrogate_24x24x8_p2.npz")
SURROGATE_TAU = 5e-3


def surrogate_leg(ctx, rve, n_points, rank):
    """Surrogate + fallback against plain batched PCG on the surrogate's RVE class
    (24x24x8, p = 2, periodic): n_points Gauss points (seed 5 + rank) through
    macro_update_gauss_points_surrogate; the error is measured on a sample solved
    by the plain PCG, and the plain PCG rate on that class is measured beside it."""
    if not os.path.exists(SURROGATE_FILE):
        return {"unavailable": "no trained surrogate weights in the package"}
    import time as _t
    z = np.load(SURROGATE_FILE)
    s = rve.Surrogate(ctx, members=int(z["members"]), seed=0)
    s.set_params(z["params"])
    xyz, tets, phase, tangent = ri.weave_rve(24, 24, 8)
    mesh = ctx.mesh_load(xyz, tets, 2, phase, tangent)
    mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
    mesh.set_bc(rve.BC_PERIODIC)
    T, c, t, _, _ = ri.gauss_point_states(n_points, 5 + rank)
    mid = np.zeros(n_points, np.int32)
    ctx.macro_update_surrogate([mesh], [s], SURROGATE_TAU, T[:4096], c[:4096], t[:4096], mid[:4096])  # warm-up
    t0 = _t.perf_counter()
    Cs, Ks, Ds, st, fb, stats, rc = ctx.macro_update_surrogate([mesh], [s], SURROGATE_TAU, T, c, t, mid)
    sur_s = _t.perf_counter() - t0
    # plain batched PCG on a sample of the same points: rate and the error reference
    ns = min(4096, n_points)
    t0 = _t.perf_counter()
    Cp, Kp, Dp, stp, _, _ = ctx.macro_update([mesh], T[:ns], c[:ns], t[:ns], mid[:ns])
    pcg_s = _t.perf_counter() - t0

    def rel(a, b):
        a = a.reshape(len(a), -1)
        b = b.reshape(len(b), -1)
        return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)
    err = max(rel(Cs[:ns], Cp).max(), rel(Ks[:ns], Kp).max(), rel(Ds[:ns], Dp).max())
    mlp = mlp_inference(ctx, mesh, s, T, c, t, int(z["members"]))
    mesh.free()
    s.free()
    return {"value": n_points / sur_s, "unit": UNIT, "points": n_points, "seconds": sur_s,
            "fallback_frac": float(fb.mean()), "status_ok": int((st == 0).sum()), "gate_tau": SURROGATE_TAU,
            "max_rel_err_vs_pcg": float(err), "err_sample": ns, "mlp_inference": mlp,
            "pcg_same_class": {"value": ns / pcg_s, "unit": UNIT, "sample": ns},
            "workload": "24x24x8 p=2 plain weave, periodic; 4-member BF16 MLP ensemble (8 -> 4x256 SiLU -> 33), "
                        "spread gate -> batched mixed-precision PCG fallback; timed through the host-buffer call"}


def mlp_inference(ctx, mesh, s, T, c, t, members):
    """The ensemble's inference alone on the device (features in, tensors and
    spread out, no host copies), timed with CUDA events: the BF16 tcgen05 GEMMs
    of every member plus the head and ensemble kernels.  Flops count the four
    layers' products of the useful rows (8 -> 256 padded to 64 inputs, 256 x 256
    three times, 256 -> 33 padded to 64 outputs)."""
    import torch
    n = len(T)
    feat = torch.tensor(ctx.features(mesh, T, c, t), dtype=torch.float64, device="cuda")
    Cd = torch.empty((n, 36), dtype=torch.float64, device="cuda")
    Kd = torch.empty((n, 9), dtype=torch.float64, device="cuda")
    Dd = torch.empty((n, 9), dtype=torch.float64, device="cuda")
    sp = torch.empty(n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    args = (n, feat.data_ptr(), Cd.data_ptr(), Kd.data_ptr(), Dd.data_ptr(), sp.data_ptr())
    s.predict_dev(*args)
    torch.cuda.synchronize()
    reps = 5
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        s.predict_dev(*args)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    flops = 2.0 * n * members * (64 * 256 + 3 * 256 * 256 + 256 * 64)
    pk, pk_kind = peaks()
    tf = flops / (ms / 1e3) / 1e12
    return {"points": n, "members": members, "ms": ms, "points_per_s": n / (ms / 1e3), "tflops": tf,
            "peak_tflops": pk["bf16_tflops"], "peak_kind": f"{pk_kind} bf16 burst", "frac": tf / pk["bf16_tflops"],
            "bound": "tensor"}


# ------------------------------------------------------------ coupled macro leg
MACRO_GRID = (200, 40, 10)       # hexes of the 0.5 x 0.1 x 0.01 m plate, 6 tets each
MACRO_DT_H = 100.0               # 100 implicit steps to 1e4 h
MACRO_REFRESH_SAMPLE = 1 << 18   # Gauss points refreshed through the surrogate at the last step
MACRO_TENSION_PA = 1.0e8         # in-plane traction on the plate's end x = L (macro mechanics)
MACRO_PCG_SAMPLE = 4096          # Gauss points refreshed through the plain PCG at the last step


def macro_leg(ctx, rve, rank):
    """Coupled macro time stepping on the composite plate: transient heat and
    moisture transport with the homogenised K and D of the 24x24x8, p = 2 RVE,
    one hot, wet face, 100 implicit steps to 1e4 h with the Gauss-point
    degradation advanced every step; then, at the last (most degraded) state,
    the RVE refresh of the plate's Gauss points through surrogate + fallback
    (timed on a seeded sample, scaled to all 1.92M points) against plain batched
    PCG (timed on a smaller sample); and the macro elastic solve of the nested
    FE^2 step with C_bar at every Gauss point.  C_bar depends on a point's state
    only through its 1 - omega, so every point takes the refreshed C_bar of the
    sampled point nearest in 1 - omega (input preparation for the timed solve).
    The plate is held by symmetry rollers on x = 0, y = 0 and z = 0 and pulled
    by a uniform traction on x = L; the end displacement is compared with the
    undegraded plate's."""
    import time as _t
    ex = ri.PlateExposure()
    xyz, tets, face = ri.plate(*MACRO_GRID)
    rx, rt, ph, tg = ri.weave_rve(24, 24, 8)
    mesh = ctx.mesh_load(rx, rt, 2, ph, tg)
    mesh.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
    mesh.set_bc(rve.BC_PERIODIC)
    hom = mesh.homogenise()
    m = ctx.macro_load(xyz, tets)
    m.set_transport(hom.K, ex.rho_cp, hom.D)
    m.set_face(face, ex.T_face_C, ex.c_face_wt)
    m.reset(ex.T0_C, ex.c0_wt)
    m.step(MACRO_DT_H)                       # warm-up (forms the diagonal)
    m.reset(ex.T0_C, ex.c0_wt)
    its, bad = [], 0
    t0 = _t.perf_counter()
    for _ in range(ex.n_steps):
        st = m.step(MACRO_DT_H, rtol=1e-10)
        its.append(st["iterations_T"] + st["iterations_c"])
        bad += st["gauss_points_unencodable"]
    march_s = _t.perf_counter() - t0
    g = m.get()
    n_gp = g["W"].size
    Tg, cg, teq = g["Tg"].reshape(-1), g["cg"].reshape(-1), g["t_eq"].reshape(-1)
    rng = np.random.default_rng(7 + rank)
    pick = rng.choice(n_gp, size=min(MACRO_REFRESH_SAMPLE, n_gp), replace=False)
    out = {"plate_hexes": list(MACRO_GRID), "tets": int(len(tets)), "gauss_points": int(n_gp),
           "steps": ex.n_steps, "dt_h": MACRO_DT_H,
           "transport_and_degradation_ms_per_step": march_s * 1e3 / ex.n_steps,
           "pcg_iterations_per_step": float(np.mean(its)),
           "t_eq_unencodable_point_steps": int(bad),
           "W_min_last_step": float(g["W"].min()), "W_mean_last_step": float(g["W"].mean())}
    Wg = g["W"].reshape(-1)
    # points whose 1 - omega the closed-form law cannot reproduce at their own (T, c)
    # (degraded, then dried out): t_eq = 0 although W < 1
    unenc = (teq == 0.0) & (Wg < 1.0)
    out["handover"] = {"plain_pcg": "1 - omega passed per point (macro_update_gauss_points_w)",
                       "surrogate": "features from (T, c, t_eq); points that t_eq cannot encode go to the "
                                    "1 - omega route of the plain PCG",
                       "gauss_points_unencodable_last_step_t_eq": int(unenc.sum()),
                       "gauss_points_handed_over_inexactly": 0}
    if os.path.exists(SURROGATE_FILE):
        z = np.load(SURROGATE_FILE)
        s = rve.Surrogate(ctx, members=int(z["members"]), seed=0)
        s.set_params(z["params"])
        ps, pw = pick[~unenc[pick]], pick[unenc[pick]]
        mid = np.zeros(len(pick), np.int32)
        ctx.macro_update_surrogate([mesh], [s], SURROGATE_TAU, Tg[ps[:4096]], cg[ps[:4096]],
                                   teq[ps[:4096]], mid[:min(4096, len(ps))])
        t0 = _t.perf_counter()
        Cs_s, _, _, sst, fb, _, _ = ctx.macro_update_surrogate([mesh], [s], SURROGATE_TAU, Tg[ps], cg[ps],
                                                               teq[ps], mid[:len(ps)])
        if len(pw):
            Cs_w, _, _, wst, _, _ = ctx.macro_update_w([mesh], Wg[pw], mid[:len(pw)])
        sur_s = _t.perf_counter() - t0
        Cs = np.zeros((len(pick), 6, 6))
        Cs[~unenc[pick]] = Cs_s
        if len(pw):
            Cs[unenc[pick]] = Cs_w
            sst = np.concatenate([sst, wst])
        ns = min(MACRO_PCG_SAMPLE, len(pick))
        t0 = _t.perf_counter()
        Cp, _, _, pst, _, _ = ctx.macro_update_w([mesh], Wg[pick[:ns]], mid[:ns])
        pcg_s = _t.perf_counter() - t0
        err = float((np.linalg.norm((Cs[:ns] - Cp).reshape(ns, -1), axis=1) /
                     np.linalg.norm(Cp.reshape(ns, -1), axis=1)).max())
        out["refresh"] = {
            "surrogate_fallback": {"rate": len(pick) / sur_s, "unit": UNIT, "sample": int(len(pick)),
                                   "fallback_frac": float(fb.mean()), "status_ok": int((sst == 0).sum()),
                                   "via_1_minus_omega_route": int(len(pw)),
                                   "s_per_step_all_points": n_gp / (len(pick) / sur_s),
                                   "scaled": f"extrapolated from a seeded sample of {len(pick)} of the "
                                             f"{n_gp} Gauss points at the sample's rate"},
            "plain_pcg": {"rate": ns / pcg_s, "unit": UNIT, "sample": ns,
                          "s_per_step_all_points": n_gp / (ns / pcg_s),
                          "scaled": f"extrapolated from a seeded sample of {ns} of the {n_gp} Gauss points "
                                    f"(one warm-started batched call) at the sample's rate"},
            "max_rel_err_C_vs_pcg": err}
        s.free()
        out["mechanics"] = macro_mech(m, xyz, g["W"].reshape(-1), g["W"].reshape(-1)[pick], Cs, hom.C)
    m.free()
    mesh.free()
    return out


def macro_mech(m, xyz, W_all, W_sample, C_sample, C_nominal):
    import time as _t
    import torch
    order = np.argsort(W_sample)
    Ws = W_sample[order]
    idx = np.clip(np.searchsorted(Ws, W_all), 0, len(Ws) - 1)
    lower = np.clip(idx - 1, 0, len(Ws) - 1)
    idx = np.where(np.abs(Ws[lower] - W_all) < np.abs(Ws[idx] - W_all), lower, idx)
    C_all = np.ascontiguousarray(C_sample[order][idx])
    fixed = np.stack([xyz[:, i] <= 1e-12 for i in range(3)], axis=1)
    end = xyz[:, 0] >= xyz[:, 0].max() * (1 - 1e-12)
    m.mech_set_bc(fixed)
    m.mech_set_traction(end, [MACRO_TENSION_PA, 0.0, 0.0])
    # undegraded plate first (host C_bar), then the degraded one from the device
    C_nom = np.broadcast_to(np.asarray(C_nominal), (len(W_all), 6, 6))
    st0 = m.mech_solve(np.ascontiguousarray(C_nom), rtol=1e-10)
    u0 = m.mech_get()["u"]
    Cd = torch.from_numpy(C_all).cuda()
    torch.cuda.synchronize()
    m.mech_solve(Cd.data_ptr(), rtol=1e-10)            # warm-up
    cold, warm = [], []
    for _ in range(3):
        m.mech_set_u(None)                              # from rest
        cold.append(m.mech_solve(Cd.data_ptr(), rtol=1e-10))
        m.mech_set_u(u0)                                # from the undegraded solution
        warm.append(m.mech_solve(Cd.data_ptr(), rtol=1e-10))
    u = m.mech_get()["u"]
    del Cd
    return {"traction_Pa": MACRO_TENSION_PA, "bc": "symmetry rollers on x = 0, y = 0, z = 0; traction on x = L",
            "dofs": int(u0.size), "rtol": 1e-10, "iterations_undegraded_from_rest": st0["iterations"],
            "solve_ms_from_rest": float(np.median([x["seconds"] for x in cold])) * 1e3,
            "iterations_from_rest": int(np.median([x["iterations"] for x in cold])),
            "solve_ms_from_undegraded": float(np.median([x["seconds"] for x in warm])) * 1e3,
            "iterations_from_undegraded": int(np.median([x["iterations"] for x in warm])),
            "u_end_undegraded_m": float(u0[end, 0].mean()), "u_end_degraded_m": float(u[end, 0].mean()),
            "C_bar_source": "refreshed sample (surrogate + fallback), nearest in 1 - omega"}


# ------------------------------------------------------------------ CPU oracle
def oracle_one(grid, p, T, c, t):
    from oracle import fem
    from oracle import materials as mt
    xyz, tets, phase, tangent = ri.weave_rve(*grid)
    w = float(mt.one_minus_omega(T, c, t))
    m0 = ri.NOMINAL_MATRIX
    mat = ri.MatrixProps(E=m0.E * w, nu=m0.nu, k=m0.k, d=m0.d)
    D, K, Dd = mt.element_tensors(phase, tangent, mat, ri.NOMINAL_YARN)
    return fem.homogenise(xyz, tets, grid, p, fem.BC_PERIODIC, D, K, Dd)


def _oracle_class_worker(si, p, seed_index):
    """One homogenisation (12 load cases) of one class, timed in its own process."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    T, c, t, size, pp = ri.gauss_point_states(256, SEED)
    g = int(np.nonzero((size == si) & (pp == p))[0][seed_index])
    t0 = time.perf_counter()
    oracle_one(ri.SIZE_CLASSES[si], p, T[g], c[g], t[g])
    return si, p, g, time.perf_counter() - t0


def cpu_baseline_start():
    """Starts one single-threaded worker per class (six processes, spawn) that
    times one seeded point of that class through the FP64 oracle."""
    import multiprocessing as mp
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(k, "1")
    pool = mp.get_context("spawn").Pool(len(ri.SIZE_CLASSES) * len(ri.P_CLASSES))
    jobs = [pool.apply_async(_oracle_class_worker, (si, p, 0))
            for si in range(len(ri.SIZE_CLASSES)) for p in ri.P_CLASSES]
    return pool, jobs, time.perf_counter()


def cpu_baseline_collect(handle):
    """Mean oracle time per homogenisation over the workload's uniform class mix
    (one seeded point of each of the six classes, each in its own single-threaded
    process) -> homogenisations/s of one core."""
    pool, jobs, t0 = handle
    per = [j.get() for j in jobs]
    pool.close()
    pool.join()
    secs = {f"{'x'.join(map(str, ri.SIZE_CLASSES[si]))} p={p}": round(dt, 3) for si, p, _, dt in per}
    mean_s = float(np.mean([dt for *_, dt in per]))
    host = os.cpu_count() or 1
    return {"value": 1.0 / mean_s, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "one seeded Gauss point of each of the six size/order classes (12 load cases each), "
                      "FP64 oracle, each class timed in its own single-threaded process (six processes ran "
                      "concurrently beside the GPU legs); value = 1 / mean seconds per homogenisation over "
                      "the uniform class mix, i.e. the rate of one core on the workload's mix",
            "seconds_per_class": secs, "wall_s": time.perf_counter() - t0,
            "ideal_parallel_bound": {"value": host / mean_s, "unit": UNIT, "cores": host,
                                     "note": "the one-core rate times the host's cores: an upper bound for "
                                             "independent points, not measured"}}


SELF_CHECK_PER_CLASS = 8
SELF_CHECK_RTOL = 1e-11


def self_check(ctx, rve, meshes, classes, T, c, t, size, p, C_t, K_t, D_t):
    """Outside every timed region: re-solves a seeded sample of the timed points
    (SELF_CHECK_PER_CLASS per class) on the FP64 path at rtol 1e-11 and compares
    the timed (mixed-precision, rtol 1e-5, warm-started) tensors with them."""
    opts = dict(precision=rve.PREC_FP64, rtol=SELF_CHECK_RTOL, warm_start=0, batch=SELF_CHECK_PER_CLASS)
    saved = ctx.get_options()
    ctx.set_options(**opts)
    worst = {"C": 0.0, "K": 0.0, "D": 0.0}
    per_class = {}
    try:
        for i, (si, q) in enumerate(classes):
            idx = np.nonzero((size == si) & (p == q))[0][:SELF_CHECK_PER_CLASS]
            if len(idx) == 0:
                continue
            Cr, Kr, Dr, st, _, _ = ctx.macro_update([meshes[i]], T[idx], c[idx], t[idx],
                                                   np.zeros(len(idx), np.int32))
            errs = {}
            for name, a, b in (("C", C_t[idx].reshape(len(idx), 36), Cr.reshape(len(idx), 36)),
                               ("K", K_t[idx].reshape(len(idx), 9), Kr.reshape(len(idx), 9)),
                               ("D", D_t[idx].reshape(len(idx), 9), Dr.reshape(len(idx), 9))):
                e = float((np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)).max())
                errs[name] = e
                worst[name] = max(worst[name], e)
            per_class[f"{'x'.join(map(str, ri.SIZE_CLASSES[si]))} p={q}"] = errs
    finally:
        ctx.set_options(**saved)
    return {"max_rel_err_vs_fp64": worst, "per_class": per_class, "points_per_class": SELF_CHECK_PER_CLASS,
            "reference": f"FP64 path, rtol {SELF_CHECK_RTOL:g}, cold batches", "bound": 1e-6,
            "ok": bool(max(worst.values()) <= 1e-6)}


def run_reference(args, world, rank):
    if rank != 0:
        return None
    T, c, t, _, _ = ri.gauss_point_states(64, SEED)
    grid, p = ri.SIZE_CLASSES[0], 1
    for i in range(args.warmup):
        oracle_one(grid, p, T[i % 64], c[i % 64], t[i % 64])
    t0 = time.perf_counter()
    for i in range(args.steps):
        oracle_one(grid, p, T[i % 64], c[i % 64], t[i % 64])
    el = time.perf_counter() - t0
    v = args.steps / el
    sample = ("one homogenisation (12 load cases) per step of the 16x16x6 p=1 class (the cheapest class of "
              "the workload), FP64 CPU oracle, single thread")
    return {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1000 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        res = run_reference(args, world, rank)
    else:
        res = run_ours(args, world, rank, local)
    if rank == 0 and res is not None:
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
