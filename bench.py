#!/usr/bin/env python3
"""Throughput benchmark of the residual-distribution Euler step on GB300.

Default workload: the 4096 x 4096-vertex periodic mesh (33,554,432 triangles)
with the Kelvin-Helmholtz shear-layer state, blended B scheme with the
two-stage update (B2), CFL 0.8, FP64.  One "step" is one full time step of
every triangle (both stages and the CFL reduction); the metric is
triangle-updates per second.  Inputs are synthetic (seeded) and larger than
L2 (537 MB of FP64 vertex state), so no L2 flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the plain FP64 reference of the
method, on the host cores) on a bounded sample of the same workload.
Under torchrun (N > 1) the mesh is split into N vertex parts, one per rank,
with the ghost states moved by NCCL point-to-point before each stage and dt
taken by an all-reduce (min) -- strong scaling; --multi replicas runs N
independent replicas instead (weak scaling).  The batched workload splits its
64 meshes across the ranks.  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "triangle-updates/s FP64/FP32 & % HBM roofline; batched & adjoint vs plain step"
UNIT = "triangle-updates/s"
WORKLOADS = {
    # name: (side, state, scheme, mesh kind)
    "khi4096_B2": (4096, "khi", "B2", "grid"),
    "khi2048_B2": (2048, "khi", "B2", "grid"),
    "sod1024_B2": (1024, "sod", "B2", "grid"),
    "vortex64_N1": (64, "vortex", "N1", "grid"),
    "batch64_B2": (None, "batch", "B2", "grid"),
    # unstructured: jittered vertices, Delaunay diagonals, labels scrambled (seed 6)
    "khi4096j_B2": (4096, "khi", "B2", "jittered"),
    "khi2048j_B2": (2048, "khi", "B2", "jittered"),
    # bounded: periodic in x, reflecting walls at y = 0 and y = 1 (Sec. 3.5)
    "khi4096w_B2": (4096, "khi", "B2", "channel"),
}
# algorithmic HBM bytes of one triangle-update (whole step) for the two-stage
# scheme: W^n, xy, V read and R1, sigma written in the first pass; W^n, R1, V,
# xy read and R2 written in the second; W^n, R1, R2, V read and W^{n+1}
# written in the last: 44 words per vertex and 2 x 12 B of connectivity per
# triangle, N_v = N_t / 2 -> 22 s + 24 bytes (s = word size).
# arithmetic type of each precision mode: df64 keeps the state, the gathers and
# the updates in FP64 and runs the per-triangle algebra in double-float
DTYPES = {"fp64": "f64", "fp32": "f32", "df64": "f64 state; f32x2 double-float triangle algebra"}
ALG_BYTES_STEP = {("B2", 8): 200.0, ("B2", 4): 112.0, ("N1", 8): 112.0, ("N1", 4): 62.0}


def alg_scheme(scheme: str) -> str:
    """Two-stage variants move the same arrays as B2 (the Bx |v| range is reduced
    inside the vertex update)."""
    return "N1" if scheme == "N1" else "B2"


def flop_scheme(scheme: str) -> str:
    """Operation count used for a variant: LDA2 has its own; the blends count as B2
    (their blend weights differ by a few selects; Bx adds its sensor, ~20 flops)."""
    base = scheme[:-3] if scheme.endswith("_SL") else scheme
    return base if base in ("N1", "B2", "LDA2") else "B2"


def kernel_alg_bytes(kernel: str, scheme: str, s: int) -> float:
    """Algorithmic bytes per triangle of one kernel launch: every input read once,
    every output written once; vertex arrays count N_v / N_t = 1/2 per triangle."""
    geo = 11 * s + 12                     # 3 unit normals + 3 half lengths + area + l_max, 3 corner ids
    if kernel == "tri_stage1":
        rec = 16 * s if scheme != "N1" else 0
        return geo + 0.5 * 5 * s + 12 * s + rec + s      # Z, |v|+c in; shares, rec, cfl out
    if kernel == "tri_stage2":
        return geo + 0.5 * 12 * s + 16 * s + 12 * s      # Z*, W^n, W* in; rec in; shares out
    # tiled step: corner slots (3 x uint16) instead of ids, the CSR read once, no share arrays
    tgeo, csr = 11 * s + 6, 0.5 * 4 + 12
    if kernel == "tile_stage1":
        return tgeo + 0.5 * 5 * s + 16 * s + 0.5 * 5 * s + csr   # Z, |v|+c in; rec out; R1 out, V in
    if kernel == "tile_stage2":
        return tgeo + 0.5 * 9 * s + 16 * s + 0.5 * 9 * s + csr   # W^n, R1, V in; rec in; W, Z, |v|+c out
    raise KeyError(kernel)


def design_min_bytes(scheme: str, s: int) -> float:
    """This design's own floor of DRAM bytes per triangle-update of the untiled step:
    the per-triangle arrays it reads and writes (geometry 11 words + 12 B ids per
    triangle kernel, the 12-word shares written and gathered back once, the 16-word
    stage-2 record written and read, the CFL term) plus the vertex arrays at N_v =
    N_t / 2 (stage 1: Z, |v|+c in; gather: R1 out; update: W^n, R1 in, W*, Z* out;
    stage 2: Z*, W^n, W* in; update: W*, W out, Z, |v|+c out)."""
    geo = 11 * s + 12
    if alg_scheme(scheme) == "N1":
        tri = geo + 12 * s + 12 * s + s + s                      # shares out + back, CFL term out + back
        vtx = 0.5 * (5 * s + 4 * s + 4 * s + 9 * s)              # Z, spd in; R1; W, R1 in; W, Z, spd out
        return tri + vtx
    tri = 2 * geo + 2 * (12 * s + 12 * s) + 2 * 16 * s + 2 * s     # two stages: shares, record, CFL term
    vtx = 0.5 * (5 * s + 4 * s + 8 * s + 8 * s + 12 * s + 8 * s + 9 * s)
    return tri + vtx


def parse():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="khi4096_B2")
    ap.add_argument("--precision", choices=["fp64", "fp32", "df64"], default="fp64",
                    help="df64: FP64 state, per-triangle algebra in double-float (FP32 pairs)")
    ap.add_argument("--scheme", default=None,
                    choices=["N1", "B2", "LDA2", "BMAX2", "BMIN2", "BX2", "B2_SL", "LDA2_SL", "BMAX2_SL",
                             "BMIN2_SL", "BX2_SL"],
                    help="override the workload's scheme (suffix _SL: selective lumping)")
    ap.add_argument("--reorder", choices=["none", "morton", "rcm"], default="morton",
                    help="vertex/triangle reordering of the mesh store")
    ap.add_argument("--no-fp32", action="store_true", help="skip the FP32 companion measurement")
    ap.add_argument("--no-df64", action="store_true",
                    help="skip the RD_DF64 companion measurement (FP64 state, double-float triangle algebra)")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the accuracy leg (FP32 L1 density error and DF64 difference against FP64)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-form companion measurement")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tiling", default="auto",
                    help="tiled step: 'auto' (the autotuner's choice), 'none', or TRIANGLESxTHREADS, e.g. 512x128 "
                         "(suffix g: geometry staged in shared memory, e.g. 512x128g)")
    ap.add_argument("--stage-shapes", default=None,
                    help="triangle block and DF64 kernel variant of each stage instead of the autotuner's, "
                         "e.g. 256:5,128:4 (stage 1, stage 2; rd_state_set_stage_shapes)")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint-rollout companion measurement")
    ap.add_argument("--adjoint-only", default=None, metavar="N,STEPS,CKPT",
                    help="run only the adjoint measurement on an N x N mesh with STEPS steps and checkpoints every "
                         "CKPT steps (e.g. 320,8,4 for a profile of the reverse kernels) and print its JSON")
    ap.add_argument("--no-meshgen", action="store_true", help="skip the mesh-generation companion measurement")
    ap.add_argument("--multi", choices=["partition", "replicas"], default="partition",
                    help="with N > 1 ranks: one mesh split into N vertex parts with NCCL ghost exchange "
                         "(strong scaling), or N independent replicas (weak scaling)")
    return ap.parse_args()


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def build_inputs(workload):
    from paper_1705_02028_gb300 import inputs
    side, state, scheme, kind = WORKLOADS[workload]
    if kind == "jittered":
        mesh = inputs.jittered_grid(side, relabel_seed=6)
    elif kind == "channel":
        mesh = inputs.bounded_grid(side, side, periodic_x=True, bc_y="wall")
    else:
        mesh = inputs.periodic_grid(side)
    W0 = {"khi": inputs.khi_state, "sod": inputs.sod_like_state, "vortex": inputs.vortex_state}[state](mesh)
    return mesh, W0, scheme


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"rd_bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop_and_keep(self):
        self.result = self.stop()

    result = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        import statistics
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def kernel_source_hash(precision="fp64"):
    """Hash of the device code of a precision's triangle and tile kernels (the DF64
    kernels add the double-float files), which keys the committed ncu traffic figures."""
    h = hashlib.sha256()
    files = ["rd_kernels.cuh", "rd_tiled.cu"]
    if precision == "df64":
        files += ["rd_dfloat.cuh", "rd_df64_kernels.cuh"]
    for f in files:
        with open(os.path.join(ROOT, "paper_1705_02028_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def tiling_info(t, flags=0):
    """Tiled-step choice of the autotuner (rd_state_get_tiling), None when untiled."""
    if not t or not t[0]:
        return None
    return {"tile_triangles": t[0], "threads": t[1], "boundary_vertices": t[2],
            "geometry_in_shared_memory": bool(flags & 1)}


# ncu captures are taken on a smaller case of the same kernel (full-set captures
# of the 4096^2 workload are too large to replay); DRAM bytes per triangle carry
# over because every per-triangle and per-vertex array is touched once per launch.
TRAFFIC_CAPTURE = {"khi4096_B2": "khi2048_B2", "khi4096j_B2": "khi2048j_B2"}


def ncu_traffic(workload, precision, kernel, nt, variant=None):
    """DRAM bytes per launch of a kernel from the committed ncu summary, scaled to nt
    triangles, with the workload it was captured on; None when missing or taken on a
    different kernel source.  DF64 kernels are looked up by their variant too (the
    register budgets spill, and spills change the traffic)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None
    name = f"{kernel}:v{variant}" if variant is not None else kernel
    cap = workload if f"{workload}:{precision}:{name}" in d else TRAFFIC_CAPTURE.get(workload, workload)
    e = d.get(f"{cap}:{precision}:{name}")
    if not e or e.get("source_hash") != kernel_source_hash(precision):
        return None
    return {"bytes_per_launch": float(e["dram_bytes_per_triangle"]) * nt,
            "bytes_per_triangle": float(e["dram_bytes_per_triangle"]),
            "captured_on": cap, "scaled": cap != workload}


def run_state_timing(binding, mesh_dev, W0, scheme, precision, steps, warmup, ws, clocks=None, autotune=True,
                     tiling="auto", stage_shapes=None):
    import torch
    s = binding.State(mesh_dev, W0, scheme=scheme, precision=precision)
    s.shapes = s.autotune() if autotune else None
    if stage_shapes:
        for k, spec in enumerate(stage_shapes.split(","), start=1):
            tb, var = (int(x) for x in spec.split(":"))
            s.set_stage_shapes(k, tb, var)
    if tiling == "none":
        s.set_tiling(0)
    elif tiling != "auto":
        gs = tiling.lower().endswith("g")
        tt, bt = (int(x) for x in tiling.lower().rstrip("g").split("x"))
        s.set_tiling(tt, bt, stage_geometry=gs)
    s.tiles = s.tiling()
    s.tflags = s.tiling_flags()
    s.sshapes = {f"stage{k}": dict(zip(("tri_block", "df_variant"), s.stage_shapes(k))) for k in (1, 2)}
    s.run(warmup)
    st = mesh_dev.stream
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.start()
    barrier(ws)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    per_kernel, launches = s.profile(steps)
    e1.record(st)
    torch.cuda.synchronize()
    barrier(ws)
    if clocks is not None:
        clocks.stop_and_keep()
    ms_total = e0.elapsed_time(e1)
    return s, ms_total, per_kernel, launches


def ours_batched(args, ws, rank, local):
    import torch
    torch.cuda.set_device(local)
    bt = batched(args, ws, args.steps)
    line = {"metric": METRIC, "value": bt["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": bt["ms_per_step"], "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": DTYPES[args.precision],
            "data": "synthetic (64 seeded periodic meshes, vortex / shear states; whole meshes split across ranks)",
            "config": {"workload": "batch64_B2", "meshes": bt["meshes"], "triangles": bt["triangles"],
                       "scheme": "B2", "cfl": 0.8, "precision": args.precision,
                       "l2": "inputs larger than L2", "steps_per_graph_launch": args.steps},
            "batched": bt, "gpu_launches": 7 * args.steps + 1}
    return line


def ours(args, ws, rank, local):
    import numpy as np
    import torch

    from paper_1705_02028_gb300 import binding

    if args.workload == "batch64_B2":
        return ours_batched(args, ws, rank, local)
    if ws > 1 and args.multi == "partition":
        return ours_partitioned(args, ws, rank, local)
    torch.cuda.set_device(local)
    mesh, W0, scheme = build_inputs(args.workload)
    if args.scheme:
        scheme = args.scheme
    nt, nv = mesh.nt, mesh.nv
    m = binding.Mesh(mesh, reorder=args.reorder)
    s_bytes = 4 if args.precision == "fp32" else 8

    clocks = ClockSampler(local)
    s, ms_total, per_kernel, launches = run_state_timing(binding, m, W0, scheme, args.precision,
                                                         args.steps, args.warmup, ws, clocks,
                                                         autotune=not args.no_autotune, tiling=args.tiling,
                                                         stage_shapes=args.stage_shapes)
    clk = clocks.result
    shapes = s.shapes
    ms_step = max_over_ranks(ms_total / args.steps, ws)
    value = ws * nt / (ms_step * 1e-3)

    # graph-replayed product path (rd_run), same state, for reference
    st = m.stream
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record(st)
    s.run(args.steps)
    g1.record(st)
    torch.cuda.synchronize()
    ms_graph = g0.elapsed_time(g1) / args.steps

    # roofline of the dominant kernel
    dom = max(per_kernel, key=per_kernel.get)
    dom_ms = per_kernel[dom]
    stage = 1 if dom in ("tri_stage1", "tile_stage1") else 2
    if args.precision in ("fp64", "df64") and dom in ("tri_stage1", "tri_stage2", "tile_stage1", "tile_stage2"):
        fl = binding.count_flops(flop_scheme(scheme), stage)["total"]
        peak = binding.probe_fma_peak("fp64")
        achieved = fl * nt / (dom_ms * 1e-3)
        roof = {"bound": "alu", "kernel": dom, "achieved": achieved / 1e12, "peak": peak / 1e12,
                "unit": "TFLOP/s", "frac": achieved / peak, "flops_per_triangle": fl,
                "peak_source": "measured FP64 FMA probe (rd_probe_fma_peak), same GPU, same run",
                "traffic": None}
        if args.precision == "df64":
            roof["note"] = ("FP64-equivalent counted flops against the FP64 FMA peak; the per-triangle algebra "
                            "runs in double-float on the FP32 pipe, so frac can exceed 1")
            roof["measured_fp32_fma_peak_tflops"] = binding.probe_fma_peak("fp32") / 1e12
        var = s.sshapes[f"stage{stage}"]["df_variant"] if args.precision == "df64" else None
        tr = ncu_traffic(args.workload, args.precision, dom, nt, var)
        roof["traffic"] = tr["bytes_per_launch"] if tr else None
        roof["traffic_source"] = tr
    else:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        bpt = kernel_alg_bytes(dom, scheme, s_bytes) if dom.startswith(("tri_", "tile_stage")) else None
        achieved = bpt * nt / (dom_ms * 1e-3) / 1e9 if bpt else None
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm if achieved else None, "bytes_per_triangle": bpt,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback 6.8 TB/s",
                "traffic": None}
        tr = ncu_traffic(args.workload, args.precision, dom, nt)
        roof["traffic"] = tr["bytes_per_launch"] if tr else None
        roof["traffic_source"] = tr
    step_bytes = ALG_BYTES_STEP.get((alg_scheme(scheme), s_bytes))
    hbm_peak = 6765.0
    try:
        hbm_peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        pass
    step_hbm = {"alg_bytes_per_triangle": step_bytes,
                "achieved_gbs": step_bytes * nt / (ms_step * 1e-3) / 1e9 if step_bytes else None,
                "frac_of_measured_hbm": (step_bytes * nt / (ms_step * 1e-3) / 1e9) / hbm_peak if step_bytes else None,
                "note": "alg_bytes_per_triangle is the ideal floor (22 s + 24 B: vertex arrays once per pass, "
                        "geometry recomputed from coordinates); design_min_bytes_per_triangle is this design's own "
                        "floor (precomputed per-triangle geometry, per-triangle shares and stage-2 record, every "
                        "array touched once)",
                "design_min_bytes_per_triangle": design_min_bytes(scheme, s_bytes)}

    # end to end through the public API with host buffers (pinned), every step
    Wh = torch.empty((4, nv), dtype=torch.float64, pin_memory=True).numpy()
    Wo = torch.empty((4, nv), dtype=torch.float64, pin_memory=True).numpy()
    Wh[:] = s.get()
    e2e_steps = max(2, min(args.steps, 5))
    s.set(Wh)
    s.step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        s.set(Wh)
        s.step()
        s.get(out=Wo)
    t_e2e = max_over_ranks((time.perf_counter() - t0) / e2e_steps, ws)
    e2e = {"value": ws * nt / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(Wh.nbytes),
           "d2h_bytes_per_step": int(Wo.nbytes), "ms_per_step": t_e2e * 1e3,
           "path": "rd_state_set (pinned host W) + rd_step + rd_get_state (pinned host W)"}
    s.close()

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPES[args.precision],
            "data": "synthetic (seeded KHI shear layer / generated periodic triangulation)",
            "config": {"workload": args.workload, "triangles": nt, "vertices": nv, "scheme": scheme,
                       "cfl": 0.8, "precision": args.precision, "reorder": args.reorder,
                       "mesh": WORKLOADS[args.workload][3],
                       "l2": "inputs larger than L2 (%.0f MB vertex state)" % (4 * nv * s_bytes / 1e6),
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "ms_per_step_graph": ms_graph, "per_kernel_ms": per_kernel,
            "launch_shapes": {"tri_block": shapes[0], "vtx_block": shapes[1], "per_stage": s.sshapes,
                              "source": "rd_state_autotune"} if shapes else None,
            "tiling": tiling_info(s.tiles, s.tflags),
            "roofline": roof, "step_hbm": step_hbm, "e2e": e2e,
            "gpu_launches": launches * args.steps + 1,
            "clocks": clk}

    # FP32 companion measurement on the same mesh
    if not args.no_fp32 and args.precision == "fp64":
        s32, ms32, pk32, _ = run_state_timing(binding, m, W0, scheme, "fp32", max(args.steps, 20),
                                              args.warmup, ws, autotune=not args.no_autotune, tiling=args.tiling)
        ms32 = max_over_ranks(ms32 / max(args.steps, 20), ws)
        d32 = max(pk32, key=pk32.get)
        hbm = hbm_peak
        b32 = kernel_alg_bytes(d32, scheme, 4) if d32.startswith(("tri_", "tile_stage")) else None
        a32 = b32 * nt / (pk32[d32] * 1e-3) / 1e9 if b32 else None
        sb32 = ALG_BYTES_STEP.get((alg_scheme(scheme), 4))
        line["fp32"] = {"value": ws * nt / (ms32 * 1e-3), "ms_per_step": ms32, "per_kernel_ms": pk32,
                        "tiling": tiling_info(s32.tiles, s32.tflags),
                        "roofline": {"bound": "hbm", "kernel": d32, "achieved": a32, "peak": hbm, "unit": "GB/s",
                                     "frac": a32 / hbm if a32 else None, "bytes_per_triangle": b32,
                                     "traffic": (ncu_traffic(args.workload, "fp32", d32, nt) or {}).get(
                                         "bytes_per_launch"),
                                     "traffic_source": ncu_traffic(args.workload, "fp32", d32, nt)},
                        "step_hbm_frac_of_measured": sb32 * nt / (ms32 * 1e-3) / 1e9 / hbm}
        s32.close()
    # RD_DF64 companion: the same step with the triangle algebra in double-float
    if not args.no_df64 and args.precision == "fp64":
        sdf, msdf, pkdf, _ = run_state_timing(binding, m, W0, scheme, "df64", args.steps, args.warmup, ws,
                                              autotune=not args.no_autotune, tiling="none")
        msdf = max_over_ranks(msdf / args.steps, ws)
        ddf = max(pkdf, key=pkdf.get)
        stage_df = 1 if ddf in ("tri_stage1", "tile_stage1") else 2
        fl_df = binding.count_flops(flop_scheme(scheme), stage_df)["total"] if ddf.startswith("tri_") else None
        fp64_peak = binding.probe_fma_peak("fp64")
        fp32_peak = binding.probe_fma_peak("fp32")
        eq = fl_df * nt / (pkdf[ddf] * 1e-3) if fl_df else None
        line["df64"] = {"value": ws * nt / (msdf * 1e-3), "ms_per_step": msdf, "per_kernel_ms": pkdf,
                        "vs_fp64_step": ms_step / msdf,
                        "launch_shapes": {"vtx_block": sdf.launch_shapes()[1], "per_stage": sdf.sshapes},
                        "dominant_kernel": ddf,
                        "traffic_source": ncu_traffic(args.workload, "df64", ddf, nt,
                                                      sdf.sshapes[f"stage{stage_df}"]["df_variant"]),
                        "counted_fp64_equivalent_tflops": eq / 1e12 if eq else None,
                        "vs_measured_fp64_fma_peak": eq / fp64_peak if eq else None,
                        "measured_fp32_fma_peak_tflops": fp32_peak / 1e12,
                        "note": "FP64 state and vertex kernels; per-triangle algebra in double-float (FP32 pairs) "
                                "on the nodal differences; parity-tested against the oracle at the FP64 bar (1e-12)"}
        sdf.close()

    if not args.no_accuracy and args.precision == "fp64":
        line["accuracy"] = accuracy_leg(binding, m, W0, scheme, nt, mesh)
    m.close()

    if not args.no_batched and args.workload != "batch64_B2":
        bt = batched(args, ws, args.steps)
        bt["vs_plain_step"] = bt["value"] / value
        if "df64" in bt and "df64" in line:
            bt["df64"]["vs_plain_step"] = bt["df64"]["value"] / line["df64"]["value"]
        if "fp32" in bt and "fp32" in line:
            bt["fp32"]["vs_plain_step"] = bt["fp32"]["value"] / line["fp32"]["value"]
        if ws == 1 and args.precision == "fp64":
            bt["small_meshes"] = batched_small(args, ws, args.steps)
        line["batched"] = bt
    if not args.no_adjoint and args.precision == "fp64":
        line["adjoint"] = adjoint_measure(args, ws)
        line["adjoint"]["large_mesh_no_stored_linearisation"] = adjoint_measure(args, ws, n_steps=40, ckpt_every=20,
                                                                                N=2048)
    if not args.no_meshgen:
        line["meshgen"] = meshgen_measure(args)

    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
    return line


def ours_partitioned(args, ws, rank, local):
    """The workload's mesh split into ws vertex parts, one per rank (rd_part_*): ghost
    states through NCCL point-to-point before each stage, dt through an all-reduce
    (min).  Strong scaling: the whole job advances the one mesh."""
    import torch

    from paper_1705_02028_gb300 import binding
    torch.cuda.set_device(local)
    mesh, W0, scheme = build_inputs(args.workload)
    if args.scheme:
        scheme = args.scheme
    m = binding.Mesh(mesh, reorder=args.reorder)
    part = binding.Part(m, ws, rank, W0, scheme=scheme, precision=args.precision)
    binding.run_part_distributed(part, args.warmup)
    clocks = ClockSampler(local)
    clocks.start()
    barrier(ws)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    binding.run_part_distributed(part, args.steps)
    e1.record()
    torch.cuda.synchronize()
    barrier(ws)
    clocks.stop_and_keep()
    ms_step = max_over_ranks(e0.elapsed_time(e1) / args.steps, ws)
    nt = mesh.nt
    line = {"metric": METRIC, "value": nt / (ms_step * 1e-3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": DTYPES[args.precision],
            "data": "synthetic (seeded KHI shear layer / generated periodic triangulation)",
            "config": {"workload": args.workload, "triangles": nt, "vertices": mesh.nv, "scheme": scheme,
                       "cfl": 0.8, "precision": args.precision, "reorder": args.reorder,
                       "parallelism": f"vertex partition x{ws} (NCCL ghost exchange, all-reduce min dt)",
                       "owned_vertices_rank0": part.n_owned, "ghost_vertices_rank0": part.n_ghost,
                       "l2": "inputs larger than L2"},
            "clocks": clocks.result,
            "e2e": None,
            "gpu_launches": None}
    part.close()
    m.close()
    return line


def accuracy_leg(binding, m, W0, scheme, nt, mesh, steps=20):
    """FP32 L1 density error and the RD_DF64 max-norm difference, both against the
    FP64 path (itself held to the oracle at 1e-12 by the parity tests), after
    `steps` steps from the workload's initial state."""
    import numpy as np
    out = {"steps": steps, "reference": "FP64 GPU path, same steps (parity-tested against the oracle at 1e-12)"}
    ref = binding.State(m, W0, scheme=scheme, precision="fp64")
    ref.run(steps)
    W64 = ref.get()
    ref.close()
    # nodal volumes V_i = sum |T| / 3 for the L1 norm of Sec. 5.1.1
    P = mesh.xy[mesh.tri] + (mesh.shift * np.array([mesh.Lx, mesh.Ly]) if mesh.shift is not None else 0.0)
    area = 0.5 * ((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1]) -
                  (P[:, 2, 0] - P[:, 0, 0]) * (P[:, 1, 1] - P[:, 0, 1]))
    V = np.zeros(mesh.nv)
    np.add.at(V, mesh.tri.ravel(), np.repeat(area / 3.0, 3))
    for prec in ("fp32", "df64"):
        s = binding.State(m, W0, scheme=scheme, precision=prec)
        s.run(steps)
        W = s.get()
        s.close()
        if prec == "fp32":
            out["fp32_l1_density_error"] = float(np.sum(V * np.abs(W[0] - W64[0])) / np.sum(V))
        else:
            scale = np.maximum(np.abs(W64).max(axis=1), np.abs(W64[3]).max())
            out["df64_max_rel_difference"] = float((np.abs(W - W64).max(axis=1) / scale).max())
    return out


def _time_batch(binding, torch, meshes, states, scheme, precision, warmup, steps, ws, autotune=True):
    """One batch on the given meshes: autotune, warm up, then `steps` steps as ONE
    graph launch timed with CUDA events; per-kernel ms of two profiled steps."""
    stream = meshes[0].stream
    b = binding.Batch(meshes, states, scheme=scheme, precision=precision)
    nv, nt = b.sizes()
    shapes = b.autotune() if autotune else None
    b.run(warmup)
    torch.cuda.synchronize()
    barrier(ws)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.run(steps)                      # one graph launch of `steps` steps
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    ms = max_over_ranks(e0.elapsed_time(e1) / steps, ws)
    pk = b.profile(2)
    dts = b.dt()
    b.close()
    return {"ms_per_step": ms, "triangles_rank0": nt, "vertices_rank0": nv, "per_kernel_ms": pk,
            "dt_min": float(dts.min()), "dt_max": float(dts.max()),
            "launch_shapes": {"tri_block": shapes[0], "vtx_block": shapes[1], "source": "rd_batch_autotune"}
            if shapes else None}


def batched(args, ws, steps):
    """64 independent periodic meshes, sides ~ U{128..1024} (seed 2), vortex or shear state
    (50/50), B2, each with its own dt, `steps` steps as ONE CUDA-graph launch: FP64 (the
    line's numbers), RD_DF64 and FP32 on the same meshes."""
    import torch

    from paper_1705_02028_gb300 import binding, inputs
    work_all = inputs.batch_workload(n_mesh=64, seed=2)
    nt_all = sum(m.nt for m, _, _ in work_all)
    rank = int(os.environ.get("RANK", "0"))
    work = work_all[rank::ws]          # whole meshes per rank: independent units, no collective
    stream = torch.cuda.Stream()
    meshes = [binding.Mesh(m, stream=stream) for m, _, _ in work]
    states = [W for _, W, _ in work]
    out = {}
    for prec in ("fp64", "df64", "fp32"):
        if prec != "fp64" and args.precision != "fp64":
            continue
        r = _time_batch(binding, torch, meshes, states, "B2", prec if args.precision == "fp64" else args.precision,
                        args.warmup, steps, ws, autotune=not args.no_autotune)
        r["value"] = nt_all / (r["ms_per_step"] * 1e-3)
        out[prec] = r
    for mm in meshes:
        mm.close()
    main = out["fp64"]
    line = {"value": main["value"], "unit": UNIT, "ms_per_step": main["ms_per_step"], "meshes": len(work_all),
            "meshes_per_rank": len(work), "triangles": nt_all, "triangles_rank0": main["triangles_rank0"],
            "vertices_rank0": main["vertices_rank0"], "steps_per_graph_launch": steps,
            "sides": [int(mm.Nx) for mm, _, _ in work], "dt_min": main["dt_min"], "dt_max": main["dt_max"],
            "launch_shapes": main["launch_shapes"], "per_kernel_ms": main["per_kernel_ms"],
            "precision": args.precision}
    if "df64" in out:
        line["df64"] = {k: out["df64"][k] for k in ("value", "ms_per_step", "per_kernel_ms", "launch_shapes")}
    if "fp32" in out:
        line["fp32"] = {k: out["fp32"][k] for k in ("value", "ms_per_step", "per_kernel_ms", "launch_shapes")}
    return line


def batched_small(args, ws, steps, n_mesh=512, smin=32, smax=128):
    """Many small meshes, where launch overhead matters: 512 periodic meshes of sides
    U{32..128} (seed 5), B2 FP64.  The batched form (`steps` steps as one graph
    launch) against the same meshes advanced one by one through their own states
    (rd_run per mesh, each replaying its own two-step graph), and the graph's step
    time against the sum of its kernels' times (the launch overhead left to a
    persistent kernel)."""
    import torch

    from paper_1705_02028_gb300 import binding, inputs
    work = inputs.batch_workload(n_mesh=n_mesh, seed=5, smin=smin, smax=smax)
    nt_all = sum(m.nt for m, _, _ in work)
    stream = torch.cuda.Stream()
    meshes = [binding.Mesh(m, stream=stream) for m, _, _ in work]
    states = [W for _, W, _ in work]
    r = _time_batch(binding, torch, meshes, states, "B2", "fp64", args.warmup, steps, ws,
                    autotune=not args.no_autotune)
    kern = sum(v for k, v in r["per_kernel_ms"].items())
    plain = [binding.State(mm, W, scheme="B2") for mm, W in zip(meshes, states)]
    for s in plain:
        s.run(2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in plain:
        s.run(steps)
    torch.cuda.synchronize()
    t_plain = (time.perf_counter() - t0) / steps
    for s in plain:
        s.close()
    for mm in meshes:
        mm.close()
    return {"meshes": n_mesh, "sides": [smin, smax], "triangles": nt_all, "precision": "fp64",
            "ms_per_step": r["ms_per_step"], "value": nt_all / (r["ms_per_step"] * 1e-3),
            "sum_of_kernel_ms_per_step": kern, "graph_overhead_ms_per_step": r["ms_per_step"] - kern,
            "per_mesh_states_ms_per_step": t_plain * 1e3,
            "per_mesh_states_value": nt_all / t_plain,
            "vs_per_mesh_states": (t_plain * 1e3) / r["ms_per_step"],
            "note": "per-mesh states: rd_run(steps) on each of the 512 states in turn (host wall clock); "
                    "graph overhead = graph-timed step minus the sum of its kernels' event-timed durations"}


def meshgen_measure(args, R=7.3e-4):
    """Delaunay refinement of the periodic unit square to circumradius <= R and
    beta <= sqrt 2 on the GPU (about 1.3 million vertices for R = 7.3e-4, the
    size of the paper's mesh-generation test), timed with CUDA events."""
    import torch
    from paper_1705_02028_gb300 import binding
    binding.meshgen(0.05)          # warm-up: module load, first launches
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mesh, info = binding.meshgen(R)
    wall = time.perf_counter() - t0
    ms = info["ms"]
    return {"vertices": mesh.nv, "triangles": mesh.nt, "max_circumradius": R, "quality_bound": 2.0 ** 0.5,
            "status": info["status"], "rounds": info["rounds"], "flips": info["flips"],
            "device_ms": ms["total"], "wall_s": wall, "vertices_per_s": mesh.nv / (ms["total"] * 1e-3),
            "phase_ms": {k: v for k, v in ms.items() if k != "total"},
            "note": "device time of rd_meshgen_run (CUDA events around the whole run, host control loop included)"}


def adjoint_measure(args, ws, n_steps=200, ckpt_every=20, N=512):
    """Gradient of L = 1/2 sum V (rho - rho_tgt)^2 after an n_steps B2 FP64 rollout on the
    N x N periodic mesh from a smooth density perturbation (amplitude 0.05), checkpoints
    every ckpt_every steps, against n_steps plain steps of the same state.  (At 512^2 a
    segment's linearisations fit in a quarter of the free memory and the backward pass
    reads them; at 2048^2 they do not, and it linearises again.)"""
    import numpy as np
    import torch

    from paper_1705_02028_gb300 import binding, inputs
    mesh = inputs.periodic_grid(N)
    W0 = inputs.smooth_density_state(mesh, seed=3)
    tgt = inputs.smooth_density_state(mesh, seed=4)
    m = binding.Mesh(mesh)
    plain = binding.State(m, W0, scheme="B2")
    plain.run(3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain.run(n_steps)
    t_plain = time.perf_counter() - t0
    plain.close()
    s = binding.State(m, W0, scheme="B2")
    s.adjoint_forward(2, 1)             # warm the adjoint kernels once
    s.adjoint_backward(np.zeros_like(W0))
    s.set(W0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.adjoint_forward(n_steps, ckpt_every)
    t_fwd = time.perf_counter() - t0
    Wf = s.get()
    # L = 1/2 sum V (rho - rho_tgt)^2 with V = |T|/3 summed over the triangles (regular grid: h^2)
    V = np.full(mesh.nv, (1.0 / N) ** 2)
    seed = np.zeros_like(Wf)
    seed[0] = V * (Wf[0] - tgt[0])
    t0 = time.perf_counter()
    g = s.adjoint_backward(seed)
    t_bwd = time.perf_counter() - t0
    s.close()
    m.close()
    nt = mesh.nt
    return {"mesh": f"{N}x{N}", "triangles": nt, "steps": n_steps, "ckpt_every": ckpt_every, "scheme": "B2",
            "precision": "fp64", "plain_s": t_plain, "forward_s": t_fwd, "backward_s": t_bwd,
            "value": nt * n_steps / (t_fwd + t_bwd), "unit": "triangle-updates/s (forward + backward)",
            "plain_value": nt * n_steps / t_plain,
            "cost_vs_plain_step": (t_fwd + t_bwd) / t_plain, "grad_norm": float(np.linalg.norm(g))}


def host_cpu():
    """CPU model and logical core count of the host the oracle runs on."""
    import platform
    import subprocess
    model = None
    try:  # lscpu names Arm cores (/proc/cpuinfo on Arm gives only part numbers)
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip().lower() == "model name":
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    key = line.split(":")[0].strip().lower()
                    if key in ("model name", "cpu part", "hardware"):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"model": model or platform.processor() or platform.machine(), "machine": platform.machine(),
            "logical_cpus": os.cpu_count()}


def sample_mesh(workload):
    """1024^2 periodic mesh of the workload's kind (1/16 of a 4096^2 workload's triangles)."""
    from paper_1705_02028_gb300 import inputs
    if WORKLOADS[workload][3] == "jittered":
        return inputs.jittered_grid(1024, relabel_seed=6)
    if WORKLOADS[workload][3] == "channel":
        return inputs.bounded_grid(1024, 1024, periodic_x=True, bc_y="wall")
    return inputs.periodic_grid(1024)


def oracle_sample_rate(workload, scheme, steps, nthreads):
    """Oracle triangle-updates/s on the sample: the KHI state on a 1024^2 periodic mesh
    of the workload's kind, `steps` full steps."""
    import oracle
    from paper_1705_02028_gb300 import inputs
    mesh = sample_mesh(workload)
    W0 = inputs.khi_state(mesh)
    t0 = time.perf_counter()
    oracle.run(mesh, W0, scheme, nsteps=steps, nthreads=nthreads)
    dt = time.perf_counter() - t0
    return mesh.nt * steps / dt, dt, mesh.nt


def cpu_baseline(args):
    import oracle
    scheme = WORKLOADS[args.workload][2]
    nth = os.cpu_count() or 1
    oracle.build()
    rate, secs, nts = oracle_sample_rate(args.workload, scheme, 2, nth)
    if secs < 8.0:  # aim for ~10-30 s of CPU work
        extra = max(1, int(10.0 / max(secs / 2, 1e-3)))
        rate, secs, nts = oracle_sample_rate(args.workload, scheme, min(extra, 40), nth)
    return {"value": rate, "unit": UNIT, "cores": nth, "kind": "oracle", "seconds": secs, "host": host_cpu(),
            "sample": f"{scheme} steps of the KHI state on a 1024x1024 periodic mesh ({nts} triangles, "
                      f"1/16 of the workload, {WORKLOADS[args.workload][3]} mesh), FP64 C++ oracle, OpenMP over {nth} host threads"}


def reference(args, ws, rank):
    import oracle
    if rank != 0:
        return None
    scheme = WORKLOADS[args.workload][2]
    nth = os.cpu_count() or 1
    oracle.build()
    from paper_1705_02028_gb300 import inputs
    mesh = sample_mesh(args.workload)
    W = inputs.khi_state(mesh)
    for _ in range(args.warmup):
        W, _ = oracle.run(mesh, W, scheme, nsteps=1, nthreads=nth)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        W, _ = oracle.run(mesh, W, scheme, nsteps=1, nthreads=nth)
    secs = time.perf_counter() - t0
    ms_step = secs / args.steps * 1e3
    value = mesh.nt / (ms_step * 1e-3)
    sample = (f"each step: one {scheme} step of the KHI state on a 1024x1024 {WORKLOADS[args.workload][3]} periodic mesh "
              f"({mesh.nt} triangles, 1/16 of the 4096^2 workload), FP64 C++ oracle on {nth} host threads")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "triangles_per_sample_step": mesh.nt, "scheme": scheme},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nth, "kind": "oracle", "sample": sample,
                             "host": host_cpu()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        line = reference(args, ws, rank)
    elif args.adjoint_only:
        n, steps, ckpt = (int(x) for x in args.adjoint_only.split(","))
        line = adjoint_measure(args, ws, n_steps=steps, ckpt_every=ckpt, N=n)
    else:
        line = ours(args, ws, rank, local)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
