"""Benchmark: coloured Q1 stencil sweeps on one large FP64 grid per GPU.

Workload (one "step" = one pass of the op mix over the resident grids):
  3D: 512^3 cells (513^3 vertices, FP64), unit cube, homogeneous Dirichlet boundary,
      u0 ~ U[-1,1] (seed 1), f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z);
  2D: 16384^2 cells (16385^2 vertices, FP64, row pitch padded to 16392), same fields;
  per grid and step: 50 element-wise applies, 50 assembled-stencil applies, one
  coloured Gauss-Seidel call of 50 sweeps, one damped Jacobi call of 50 sweeps
  (omega = 2/3), one residual with norms -- the op mix of the 512^3 configuration
  (100 applies, 50 GS, 50 Jacobi sweeps) on both grids.
Metric: interior-vertex updates per second (Mupdates/s), whole job; one update = one
interior vertex processed by one apply, sweep or residual.
Inputs are larger than L2 (1.08 GB / 2.15 GB per array), so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
                  [--n3 CELLS] [--n2 CELLS]   (smaller grids, e.g. for profiling)

With N > 1 (torchrun), every rank runs its own replica of the workload (independent
problems, no data-path collective); timing takes the max over ranks.
"""
import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

N3 = 512
N2 = 16384
OMEGA = 2.0 / 3.0
HBM_NOMINAL_GBS = 7900.0  # GB300 HBM3e, nominal (the roofline's peak is the measured copy rate)
N_APPLY = 50      # per form
N_SWEEPS = 50     # GS and Jacobi sweeps per call
OPS = ("apply_elementwise", "apply_stencil", "gs_sweep", "jacobi_sweep", "residual")
PASSES = {"apply_elementwise": N_APPLY, "apply_stencil": N_APPLY, "gs_sweep": N_SWEEPS,
          "jacobi_sweep": N_SWEEPS, "residual": 1}
# algorithmic HBM bytes per interior update (compulsory traffic of one pass)
BYTES_PER_UPDATE = {"apply_elementwise": 16, "apply_stencil": 16, "gs_sweep": 24,
                    "jacobi_sweep": 24, "residual": 16}


def bytes_per_update(op, g, fd=False):
    """Compulsory bytes per update and sweep: the Q1 2D Jacobi and Gauss-Seidel calls run
    two sweeps per pass over memory (read u and 3/8 h^2 f, write u once per pair), 12 B
    per sweep."""
    if op in ("jacobi_sweep", "gs_sweep") and g == "2" and not fd:
        return 12
    return BYTES_PER_UPDATE[op]


def pitch2(n2):
    return ((n2 + 1 + 7) // 8) * 8  # rows start on 64-byte boundaries


def launches_per_step(n3, n2):
    """Kernel launches of the library per step (every multi-sweep call has two pre-pass
    launches; 3D: GS two launches per sweep, Jacobi one; 2D: GS and Jacobi one launch per
    two sweeps)."""
    d3 = 2 * N_APPLY + (2 * N_SWEEPS + 2) + (N_SWEEPS + 2) + 1
    d2 = 2 * N_APPLY + (N_SWEEPS // 2 + 2) + (N_SWEEPS // 2 + 2) + 1
    return (d3 if n3 else 0) + (d2 if n2 else 0)


def interior(dim, n):
    return (n - 1) ** dim if n else 0


def updates_per_step(n3, n2):
    return sum(PASSES.values()) * (interior(3, n3) + interior(2, n2))


def max_over_ranks(torch, ms, world, device):
    """The slowest rank's time: every rank runs its own replica of the workload, so
    the job's time is the maximum (all_reduce MAX; the identity on one rank)."""
    if world <= 1:
        return ms
    tt = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
    return float(tt.item())


def whole_job_rate(units_per_rank, world, ms_max):
    """Units of all ranks (weak scaling: each rank does the same work) per second, in
    millions."""
    return units_per_rank * world / (ms_max * 1e-3) / 1e6


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true",
                    help="skip the oracle timings on the host cores (cpu_baseline; the refine "
                         "workload's per-iterate oracle comparison)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="grid workload: keep the built-in launch shapes instead of autotuning them first")
    ap.add_argument("--n3", type=int, default=N3, help="3D cells per edge (0: no 3D grid)")
    ap.add_argument("--n2", type=int, default=N2, help="2D cells per edge (0: no 2D grid)")
    ap.add_argument("--workload", default="grid",
                    choices=["grid", "small", "patches", "refine", "serve", "fd"],
                    help="grid (default): the 512^3 + 16384^2 op mix above; small: 32^3 apply + 10 GS "
                         "sweeps; patches: 4096 uneven patches x 20 sweeps; refine: refinement to 1e-10 "
                         "at 256^3 (FP32 / bf16 inner) vs FP64 inner; serve: request server; fd: the "
                         "grid op mix with the 5/7-point finite-difference operator (red-black GS)")
    ap.add_argument("--requests", type=int, default=10000, help="serve: requests per arrival rate")
    ap.add_argument("--rates", default="200,1000,5000", help="serve: arrival rates (req/s)")
    ap.add_argument("--solver", default="mg", choices=["mg", "refine"],
                    help="serve: SOLVE requests by multigrid V-cycles (mg) or by refinement with FP32 GS")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks sampler
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ GPU arm
class GpuWorkload:
    def __init__(self, torch, st, device, n3, n2, op=0):
        self.torch, self.st, self.dev = torch, st, device
        self.op = op  # st.OP_Q1 or st.OP_FD
        self.n = {"3": n3, "2": n2}
        self.grids = [g for g in ("3", "2") if self.n[g]]
        self.h = {"3": 1.0 / n3 if n3 else 0.0, "2": 1.0 / n2 if n2 else 0.0}
        self.p2 = pitch2(n2) if n2 else 0
        self.p3 = pitch2(n3) if n3 else 0  # rows on 64-byte boundaries (TMA plane loads)
        self.host = {}
        if n3:
            s3 = synth.grid_shape(3, n3)
            self.host["u3"] = self._pad3(torch.from_numpy(synth.uniform_field(s3, 1))).pin_memory()
            self.host["f3"] = self._pad3(torch.from_numpy(synth.sin_rhs(3, n3))).pin_memory()
        if n2:
            s2 = synth.grid_shape(2, n2)
            self.host["u2"] = self._pad2(torch.from_numpy(synth.uniform_field(s2, 1))).pin_memory()
            self.host["f2"] = self._pad2(torch.from_numpy(synth.sin_rhs(2, n2))).pin_memory()
        d = {}
        for g in self.grids:
            d["u" + g] = self.host["u" + g].to(device)
            d["f" + g] = self.host["f" + g].to(device)
            d["y" + g] = torch.empty_like(d["u" + g])
            d["ja" + g] = d["u" + g].clone()
            d["jb" + g] = torch.empty_like(d["u" + g])
            d["n" + g] = torch.zeros(2, dtype=torch.float64, device=device)
        self.d = d

    def _pad2(self, t):
        buf = self.torch.zeros((t.shape[0], self.p2), dtype=t.dtype)
        buf[:, :t.shape[1]] = t
        return buf

    def _pad3(self, t):
        buf = self.torch.zeros((t.shape[0], t.shape[1], self.p3), dtype=t.dtype)
        buf[..., :t.shape[2]] = t
        return buf

    def autotune(self):
        """Tunes the launch shape of every tunable call on each grid (stencil_autotune:
        candidates timed on scratch arrays of the same shape), before any timing; the
        calls then use the recorded shapes.  Returns {grid: {call: [chunk, depth]}}."""
        st = self.st
        calls = (("apply_elementwise", st.CALL_APPLY_ELEMENTWISE, 0), ("apply_stencil", st.CALL_APPLY_STENCIL, 0),
                 ("gs_sweep", st.CALL_SMOOTH_COLOURED, N_SWEEPS), ("jacobi_sweep", st.CALL_SMOOTH_JACOBI, N_SWEEPS))
        out = {}
        for g in self.grids:
            u = self.view("u" + g)
            out[g] = {}
            for name, call, sweeps in calls:
                chunk, depth, _ = st.stencil_autotune(u, self.h[g], call, sweeps)
                out[g][name] = [chunk, depth]
        return out

    def view(self, key):
        t = self.d[key]
        if key.endswith("2"):
            return t[:, :self.n["2"] + 1]
        if key.endswith("3"):
            return t[..., :self.n["3"] + 1]
        return t

    def run_op(self, op, g, stream):
        st = self.st
        h = self.h[g]
        u, f, y = self.view("u" + g), self.view("f" + g), self.view("y" + g)
        k = self.op
        if op == "apply_elementwise":
            for _ in range(N_APPLY):
                st.stencil_apply(u, y, h, st.FORM_ELEMENTWISE, stream=stream)
        elif op == "apply_stencil":
            for _ in range(N_APPLY):
                st.stencil_apply(u, y, h, st.FORM_STENCIL, stream=stream, op=k)
        elif op == "gs_sweep":
            st.stencil_smooth_coloured(u, f, h, N_SWEEPS, stream=stream, op=k)
        elif op == "jacobi_sweep":
            st.stencil_smooth_jacobi(self.view("ja" + g), f, self.view("jb" + g), h, N_SWEEPS, OMEGA,
                                     stream=stream, op=k)
        elif op == "residual":
            st.stencil_residual(u, f, h, norms2=self.d["n" + g], stream=stream, op=k)

    def step(self, stream, events=None, ops=None):
        for g in self.grids:
            for op in (ops or OPS):
                if events is not None:
                    events[(op, g)][0].record(stream)
                self.run_op(op, g, stream)
                if events is not None:
                    events[(op, g)][1].record(stream)


# Kernel sources behind each (op, grid) of the grid workload, beside the shared ones
# (api.cu, which routes the calls, and every header).  The multi-sweep smoothers also
# run the pre-pass kernels of gs_fx.cu; the 3D Jacobi call can fall back to ops_fx.cu.
TRAFFIC_SOURCES = {
    "apply_elementwise_3d": ["ew_fx.cu"],
    "apply_stencil_3d": ["ops_fx.cu"],
    "residual_3d": ["ops_fx.cu"],
    "gs_sweep_3d": ["gs_fx.cu"],
    "jacobi_sweep_3d": ["jac3_fx.cu", "gs_fx.cu", "ops_fx.cu"],
    "apply_elementwise_2d": ["ops2d_fx.cu"],
    "apply_stencil_2d": ["ops2d_fx.cu"],
    "residual_2d": ["ops2d_fx.cu"],
    "gs_sweep_2d": ["ops2d_fx.cu", "gs_fx.cu"],
    "jacobi_sweep_2d": ["ops2d_fx.cu", "gs_fx.cu"],
}


def traffic_source_sha(kernel_key, root=None):
    """First 16 hex digits of sha256 over the sources of one (op, grid): its kernel
    files, api.cu and every header of the library, in sorted order."""
    src = os.path.join(root or ROOT, "paper_1810_04033_gb300", "csrc")
    files = set(TRAFFIC_SOURCES[kernel_key]) | {"api.cu"}
    files |= {fn for fn in os.listdir(src) if fn.endswith((".cuh", ".h"))}
    sha = hashlib.sha256()
    for fn in sorted(files):
        sha.update(fn.encode() + b"\0")
        sha.update(open(os.path.join(src, fn), "rb").read())
    return sha.hexdigest()[:16]


def traffic_from_profiles(kernel_key, units_per_launch):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the
    current sources of that kernel (null otherwise)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path) or kernel_key not in TRAFFIC_SOURCES:
        return None
    cur = traffic_source_sha(kernel_key)
    for line in open(path):
        m = re.match(r"\s*kernel=(\S+)\s+src_sha=(\S+)\s+dram_bytes_per_update=([\d.eE+-]+)", line)
        if m and m.group(1) == kernel_key and m.group(2) == cur:
            return float(m.group(3)) * units_per_launch
    return None


def workload_name(n3, n2):
    parts = []
    if n3:
        parts.append("%d^3-cell 3D" % n3)
    if n2:
        parts.append("%d^2-cell 2D 9-point" % n2)
    return ("FP64 Q1 grids: %s; per step and grid 50+50 applies, 50 GS sweeps, 50 Jacobi sweeps, "
            "1 residual" % " + ".join(parts))


def metric_name(n3, n2):
    parts = []
    if n3:
        parts.append("3D %d^3" % n3)
    if n2:
        parts.append("2D %d^2" % n2)
    return ("Mupdates/s (interior-vertex updates; FP64 Q1: 50 element-wise + 50 stencil applies, "
            "50 coloured GS sweeps, 50 damped Jacobi sweeps, 1 residual per grid; %s)" % " + ".join(parts))


def run_gpu(args, rank, world):
    import torch
    import paper_1810_04033_gb300 as st

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    st.lib()
    n3, n2 = args.n3, args.n2
    wl = GpuWorkload(torch, st, dev, n3, n2)
    stream = torch.cuda.Stream(device=dev)
    tuned = None if args.no_autotune else wl.autotune()
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks else "fallback 6800 GB/s"

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            wl.step(stream)
    stream.synchronize()

    # one pair of events per op, grid and step on the launching stream; read after the
    # timed region only
    ev = [{(op, g): (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for op in OPS for g in wl.grids} for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(dev.index)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    with torch.cuda.stream(stream):
        t0.record(stream)
        for k in range(args.steps):
            wl.step(stream, ev[k])
        t1.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    clock_info = clocks.stop()
    barrier()
    per_op_ms = {key: sum(e[key][0].elapsed_time(e[key][1]) for e in ev) for key in ev[0]}
    ms = t0.elapsed_time(t1)
    ms_max = max_over_ranks(torch, ms, world, dev)
    value = whole_job_rate(updates_per_step(n3, n2) * args.steps, world, ms_max)

    # dominant kernel: the (op, grid) with the largest share of the step; its achieved
    # bandwidth = algorithmic bytes of one pass / average duration of one pass
    top_key = max(per_op_ms, key=per_op_ms.get)
    top_op, top_g = top_key
    nn = n3 if top_g == "3" else n2
    units = interior(int(top_g), nn)
    ms_pass = per_op_ms[top_key] / args.steps / PASSES[top_op]
    achieved = bytes_per_update(top_op, top_g) * units / (ms_pass * 1e-3) / 1e9
    per_pass = {g: {op: round(per_op_ms[(op, g)] / args.steps / PASSES[op], 4) for op in OPS}
                for g in wl.grids}
    gbs = {g: {op: round(bytes_per_update(op, g) * interior(int(g), wl.n[g]) /
                         (per_op_ms[(op, g)] / args.steps / PASSES[op] * 1e-3) / 1e9, 1) for op in OPS}
           for g in wl.grids}
    roofline = {"bound": "hbm", "kernel": "%s (%sD, %d cells per edge)" % (top_op, top_g, nn),
                "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(achieved / hbm_peak, 4), "peak_source": peak_src,
                "nominal_peak": HBM_NOMINAL_GBS, "frac_of_nominal": round(achieved / HBM_NOMINAL_GBS, 4),
                "traffic": traffic_from_profiles("%s_%sd" % (top_op, top_g), units),
                "share_of_step": round(per_op_ms[top_key] / ms, 3),
                "ms_per_pass": per_pass, "algorithmic_gbs": gbs}

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(torch, st, wl, stream, args, world)

    out = {"metric": metric_name(n3, n2),
           "value": round(value, 1), "unit": "Mupdates/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded U[-1,1] u0, manufactured sin RHS)",
           "config": {"workload": workload_name(n3, n2),
                      "grid_3d": [n3 + 1] * 3 if n3 else None,
                      "grid_2d": [n2 + 1, n2 + 1] if n2 else None, "pitch_2d": wl.p2 or None,
                      "pitch_3d": wl.p3 or None,
                      "l2": "inputs larger than L2 (no flush)" if n3 >= 256 or n2 >= 8192
                            else "small case (profiling)",
                      "parallelism": "replicas" if world > 1 else "single GPU",
                      "launch_shapes": {"autotuned": tuned} if tuned else "built-in"},
           "roofline": roofline, "clocks": clock_info,
           "gpu_launches": launches_per_step(n3, n2) * args.steps,
           "e2e": e2e}
    return out


def run_e2e(torch, st, wl, stream, args, world):
    """Same op mix through the public API with host buffers: every step copies u and f
    of each grid from pinned host memory, runs the ops, and reads u and the norms
    back; copies are inside the timed region.  Each grid has a copy-in and a copy-out
    stream and two sets of device inputs (u, f, norms) used in alternate steps, so a
    step's inputs go up while the previous step still computes on, or copies back from,
    the other set; events order each grid's copy-in, compute and copy-out, and a set is
    refilled only after its previous results have left."""
    steps = args.steps
    h_out = {g: torch.empty_like(wl.host["u" + g]).pin_memory() for g in wl.grids}
    h_nrm = torch.empty(4, dtype=torch.float64).pin_memory()
    bi = sum(wl.host[k + g].numel() * 8 for k in ("u", "f") for g in wl.grids)
    bo = sum(h_out[g].numel() * 8 for g in h_out) + 16 * len(wl.grids)
    cin = {g: torch.cuda.Stream(device=wl.dev) for g in wl.grids}
    cout = {g: torch.cuda.Stream(device=wl.dev) for g in wl.grids}
    keys = [k + g for k in ("u", "f", "n") for g in wl.grids]
    home = {k: wl.d[k] for k in keys}
    sets = [home, {k: torch.empty_like(home[k]) for k in keys}]
    freed = {}  # (set, grid) -> event after that set's last copy-out

    def ev():
        return torch.cuda.Event(enable_timing=True)

    marks = []  # per step and grid: events around the copy-in, the compute and the copy-out

    def one(stream, k, rec=None):
        cur = sets[k % 2]
        for i, g in enumerate(wl.grids):
            ci, co = cin[g], cout[g]
            with torch.cuda.stream(ci):
                if (k % 2, g) in freed:
                    ci.wait_event(freed[(k % 2, g)])
                a_in = ev()
                a_in.record(ci)
                cur["u" + g].copy_(wl.host["u" + g], non_blocking=True)
                cur["f" + g].copy_(wl.host["f" + g], non_blocking=True)
                e_in = ev()
                e_in.record(ci)
            stream.wait_event(e_in)
            for key in ("u" + g, "f" + g, "n" + g):
                wl.d[key] = cur[key]
            c0 = ev()
            c0.record(stream)
            for op in OPS:
                wl.run_op(op, g, stream)
            done = ev()
            done.record(stream)
            with torch.cuda.stream(co):
                co.wait_event(done)
                o0 = ev()
                o0.record(co)
                h_out[g].copy_(cur["u" + g], non_blocking=True)
                h_nrm[2 * i:2 * i + 2].copy_(cur["n" + g], non_blocking=True)
                o1 = ev()
                o1.record(co)
            freed[(k % 2, g)] = o1
            if rec is not None:
                rec.append((a_in, e_in, c0, done, o0, o1))

    with torch.cuda.stream(stream):
        one(stream, 1)
        one(stream, 0)
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for g in wl.grids:
            cin[g].wait_event(t0)
        for k in range(steps):
            one(stream, k, marks)
        for g in wl.grids:
            end_copy = ev()
            end_copy.record(cout[g])
            stream.wait_event(end_copy)
        t1.record(stream)
    torch.cuda.synchronize()
    wl.d.update(home)
    ms = max_over_ranks(torch, t0.elapsed_time(t1), world, wl.dev)
    val = whole_job_rate(updates_per_step(args.n3, args.n2) * steps, world, ms)
    # where the time went (read after the timed region): copy durations, and the time the
    # compute stream waited between one grid's ops and the next (for that grid's inputs)
    h2d = sum(a.elapsed_time(b) for a, b, *_ in marks)
    d2h = sum(o0.elapsed_time(o1) for *_, o0, o1 in marks)
    idle = sum(max(0.0, marks[k][2].elapsed_time(marks[k + 1][2]) - marks[k][2].elapsed_time(marks[k][3]))
               for k in range(len(marks) - 1))
    return {"value": round(val, 1), "unit": "Mupdates/s", "h2d_bytes_per_step": bi,
            "d2h_bytes_per_step": bo, "steps": steps, "copies": "a copy-in and a copy-out stream per grid, two sets of device inputs in alternate steps",
            "h2d_ms_per_step": round(h2d / steps, 2), "d2h_ms_per_step": round(d2h / steps, 2),
            "compute_idle_ms_per_step": round(idle / steps, 2)}


# ------------------------------------------------------------------ CPU oracle
def oracle_sample(n3, n2, nthreads):
    """One pass of each op of the mix through the oracle on grids of n3^3 and n2^2
    cells (one apply of each form, one GS sweep, one Jacobi sweep, one residual).
    Returns (updates, seconds)."""
    import oracle
    t_total = 0.0
    upd = 0
    for dim, n in ((3, n3), (2, n2)):
        if n <= 0:
            continue
        h = 1.0 / n
        s = synth.grid_shape(dim, n)
        u = synth.uniform_field(s, 1)
        f = synth.sin_rhs(dim, n)
        t = time.perf_counter()
        oracle.apply_elementwise(u, h, nthreads)
        oracle.apply_stencil(u, h, nthreads)
        oracle.gs_coloured(u, f, h, 1, nthreads)
        oracle.jacobi(u, f, h, OMEGA, 1, nthreads)
        oracle.residual(u, f, h, nthreads)
        t_total += time.perf_counter() - t
        upd += len(OPS) * interior(dim, n)
    return upd, t_total


def cpu_baseline():
    nthreads = os.cpu_count() or 1
    n3, n2 = 384, 12288
    upd, sec = oracle_sample(n3, n2, nthreads)
    return {"value": round(upd / sec / 1e6, 2), "unit": "Mupdates/s", "cores": nthreads,
            "kind": "oracle",
            "sample": "one pass of each op of the mix (element-wise apply, stencil apply, 1 GS "
                      "sweep, 1 Jacobi sweep, residual) on a %d^3 and a %d^2 grid, %.1f s, "
                      "OpenMP colour-pass parallel for" % (n3, n2, sec)}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    nthreads = os.cpu_count() or 1
    n3, n2 = 128, 2048
    for _ in range(args.warmup):
        oracle_sample(n3, n2, nthreads)
    upd_tot, sec_tot = 0, 0.0
    for _ in range(args.steps):
        u, s = oracle_sample(n3, n2, nthreads)
        upd_tot += u
        sec_tot += s
    val = upd_tot / sec_tot / 1e6
    return {"impl": "reference", "metric": metric_name(args.n3, args.n2),
            "value": round(val, 2), "unit": "Mupdates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(sec_tot / args.steps * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "grid op mix, oracle on host cores; "
                                                        "each step a bounded sample: 128^3 + 2048^2"},
            "cpu_baseline": {"value": round(val, 2), "unit": "Mupdates/s", "cores": nthreads,
                             "kind": "oracle", "sample": "per step: op mix on 128^3 and 2048^2"},
            "e2e": {"value": round(val, 2), "unit": "Mupdates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


# ------------------------------------------------------------------ other workloads
def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _hbm_peak():
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    if "hbm_gbs" in peaks:
        return peaks["hbm_gbs"], "measured (MEASURED_PEAKS.json hbm_gbs)"
    return 6800.0, "fallback 6800 GB/s"


def _roofline(bytes_moved, ms, kernel, note=None):
    """HBM roofline of a workload line: algorithmic bytes over the measured time."""
    peak, src = _hbm_peak()
    gbs = bytes_moved / (ms * 1e-3) / 1e9
    r = {"bound": "hbm", "kernel": kernel, "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
         "frac": round(gbs / peak, 4), "peak_source": src, "traffic": None}
    if note:
        r["note"] = note
    return r


def _oracle_rate(fn, updates_per_call, budget_s=10.0):
    """Calls fn (one oracle pass of `updates_per_call` updates) until about budget_s
    seconds have passed; returns (Mupdates/s, calls, seconds)."""
    t0 = time.perf_counter()
    calls = 0
    while True:
        fn()
        calls += 1
        sec = time.perf_counter() - t0
        if sec >= budget_s:
            return updates_per_call * calls / sec / 1e6, calls, sec


def run_small(args):
    """32^3 cells: one element-wise apply on u ~ U[-1,1] (seed 0), then 10 coloured GS
    sweeps on A u = f, f = 3 pi^2 sin sin sin, u0 = 0."""
    import torch
    import paper_1810_04033_gb300 as st
    n, h = 32, 1.0 / 32
    s3 = synth.grid_shape(3, n)
    u = torch.from_numpy(synth.uniform_field(s3, 0)).cuda()
    f = torch.from_numpy(synth.sin_rhs(3, n)).cuda()
    y, g = torch.empty_like(u), torch.zeros_like(u)

    def step():
        st.stencil_apply(u, y, h, st.FORM_ELEMENTWISE)
        g.zero_()
        st.stencil_smooth_coloured(g, f, h, 10)

    # launch-bound size: the step's 24 kernel launches and the memset are captured once
    # into a CUDA graph (workspaces allocated by the warm-up) and replayed per step
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for _ in range(max(1, args.warmup)):
            step()
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        step()
    graph.replay()
    torch.cuda.synchronize()
    steps = max(args.steps, 2000)  # a step is ~25 us: enough steps for the clock record
    clocks = ClockSampler(0)
    clocks.start()
    e0, e1 = _events(torch)
    e0.record()
    for _ in range(steps):
        graph.replay()
    e1.record()
    torch.cuda.synchronize()
    clock_info = clocks.stop()
    ms = e0.elapsed_time(e1) / steps
    upd = 11 * (n - 1) ** 3
    # oracle on the host cores: the same step (apply + 10 sweeps from u0 = 0)
    import oracle
    nt = os.cpu_count() or 1
    un, fn_ = synth.uniform_field(s3, 0), synth.sin_rhs(3, n)

    def ostep():
        oracle.apply_elementwise(un, h, nthreads=nt)
        oracle.gs_coloured(np.zeros_like(fn_), fn_, h, 10, nthreads=nt)

    cpu = None
    if not args.no_cpu:
        rate, calls, sec = _oracle_rate(ostep, upd, budget_s=5.0)
        cpu = {"value": round(rate, 1), "unit": "Mupdates/s", "cores": nt, "kind": "oracle",
               "sample": "the whole step (apply + 10 GS sweeps at 32^3), %d times, %.1f s" % (calls, sec)}
    return {"metric": "Mupdates/s (32^3 Q1: 1 element-wise apply + 10 coloured GS sweeps)", "workload": "small",
            "value": round(upd / ms / 1e3, 1), "unit": "Mupdates/s", "ms_per_step": round(ms, 4),
            "steps": steps, "dtype": "f64", "clocks": clock_info,
            "roofline": _roofline((16 + 10 * 24) * (n - 1) ** 3, ms, "apply + 10 GS sweeps, 33^3",
                                  "launch-bound size: 0.27 MB per array, L2-resident; the fraction is of "
                                  "algorithmic bytes only"),
            "cpu_baseline": cpu,
            "note": "launch-bound size (30K interior vertices); one CUDA graph replay per step"}


def patches_oracle_sample(nthreads, lat=(8, 8, 8), sweeps=20):
    """The oracle's patch iteration (halo fill, then a coloured GS sweep per patch) on a
    bounded lattice of the same edge distribution.  Returns (updates, seconds)."""
    import oracle
    L = synth.PatchLattice(lat=lat, seed=2)
    t = time.perf_counter()
    oracle.patch_smooth(L.lat, L.np_sizes, L.offsets, L.u, L.f, sweeps, nthreads)
    return sweeps * L.interior_updates_per_sweep, time.perf_counter() - t


def run_patches(args):
    """4096 patches in a 16^3 lattice, edges from {8,12,16,24,32} (seed 2), f ~ U[-1,1],
    u0 = 0, 20 coloured GS sweeps with a halo fill before each; launch shape autotuned."""
    import torch
    import paper_1810_04033_gb300 as st
    L = synth.PatchLattice(lat=(16, 16, 16), seed=2)
    b = st.PatchBatch(L.np_sizes, L.offsets, L.neighbours27())
    u = torch.from_numpy(L.u).cuda()
    f = torch.from_numpy(L.f).cuda()
    tuned = b.autotune(u, f)
    for _ in range(args.warmup):
        b.smooth(u, f, 20)
    torch.cuda.synchronize()
    steps = max(args.steps, 1)
    clocks = ClockSampler(0)
    clocks.start()
    e0, e1 = _events(torch)
    e0.record()
    for _ in range(steps):
        b.smooth(u, f, 20)
    e1.record()
    torch.cuda.synchronize()
    clock_info = clocks.stop()
    ms = e0.elapsed_time(e1) / steps
    upd = 20 * L.interior_updates_per_sweep
    return {"metric": "Mupdates/s (4096 uneven patches, 20 GS sweeps with halo fill)", "workload": "patches",
            "value": round(upd / ms / 1e3, 1), "unit": "Mupdates/s", "ms_per_step": round(ms, 3), "steps": steps,
            "clocks": clock_info,
            "roofline": _roofline(24 * upd, ms, "k_patch_gs + k_patch_halo (24 B per update and sweep)"),
            "autotuned_launch": {"threads": tuned[0], "ctas_per_sm": tuned[1]}, "dtype": "f64",
            "patches": int(L.np_sizes.size), "vertices": L.total,
            "cpu_baseline": None if args.no_cpu else patches_cpu_baseline()}


def patches_cpu_baseline():
    nthreads = os.cpu_count() or 1
    upd, sec = patches_oracle_sample(nthreads)
    return {"value": round(upd / sec / 1e6, 2), "unit": "Mupdates/s", "cores": nthreads, "kind": "oracle",
            "sample": "512 patches (8^3 lattice, same edge distribution), 20 sweeps with halo fill, "
                      "%.1f s, OpenMP colour passes inside each patch" % sec}


# FP64 instructions per interior update of the finite-difference kernels (FMA = one):
# the neighbour sum (3D: 5 adds, 2D: 3), then apply: FMA + scale; GS: scale + FMA;
# Jacobi: apply + subtract + FMA; residual: apply + subtract + two FMA for the norms.
FD_FP64_OPS = {"apply_stencil": {"3": 7, "2": 5}, "gs_sweep": {"3": 7, "2": 5},
               "jacobi_sweep": {"3": 9, "2": 7}, "residual": {"3": 10, "2": 8}}
FP64_PER_CLK_SM = 2.0    # FP64 add/FMA/multiply instructions per clock per SM (measured)
SM_CLOCK_MAX_HZ = 2.07e9


def fd_fp64_frac(op, g, updates, ms, sms):
    """Fraction of the FP64 pipe's instruction rate (FP64_PER_CLK_SM x SMs x maximum SM
    clock) that `updates` interior updates of op on grid g in `ms` milliseconds use."""
    return FD_FP64_OPS[op][g] * updates / (ms * 1e-3) / (FP64_PER_CLK_SM * sms * SM_CLOCK_MAX_HZ)


def run_fd(args):
    """The grid workload's op mix (stencil apply x50, one 50-sweep GS call, one 50-sweep
    Jacobi call, 1 residual per grid) with the 5/7-point finite-difference operator;
    GS is red-black.  Per-op CUDA events; fractions of the measured HBM bandwidth with
    16 B (apply, residual) and 24 B (sweeps) per update for a single pass, and of the
    FP64 pipe's instruction rate (these kernels compute in FP64)."""
    import torch
    import paper_1810_04033_gb300 as st
    dev = torch.device("cuda", 0)
    n3, n2 = args.n3, args.n2
    wl = GpuWorkload(torch, st, dev, n3, n2, op=st.OP_FD)
    ops = ["apply_stencil", "gs_sweep", "jacobi_sweep", "residual"]
    stream = torch.cuda.Stream(device=dev)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = peaks.get("hbm_gbs", 6800.0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    with torch.cuda.stream(stream):
        for _ in range(max(1, args.warmup)):
            wl.step(stream, ops=ops)
    stream.synchronize()
    steps = max(1, min(args.steps, 5))
    ev = [{(op, g): (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for op in ops for g in wl.grids} for _ in range(steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(0)
    clocks.start()
    with torch.cuda.stream(stream):
        t0.record(stream)
        for k in range(steps):
            wl.step(stream, ev[k], ops=ops)
        t1.record(stream)
    stream.synchronize()
    clock_info = clocks.stop()
    ms = t0.elapsed_time(t1)
    upd = sum(PASSES[op] * (interior(3, n3) + interior(2, n2)) for op in ops) * steps
    per = {}
    for g in wl.grids:
        nn = wl.n[g]
        for op in ops:
            t = sum(e[(op, g)][0].elapsed_time(e[(op, g)][1]) for e in ev) / steps / PASSES[op]
            b = bytes_per_update(op, g, fd=True) * interior(int(g), nn)
            per["%s_%sd" % (op, g)] = {"ms_per_pass": round(t, 4), "frac": round(b / (t * 1e-3) / 1e9 / peak, 3),
                                       "fp64_frac": round(fd_fp64_frac(op, g, interior(int(g), nn), t, sms), 3)}
    # red-black sweeps: colour passes with barriers vs dependency-driven tasks, and the
    # expensive stencils S(k) (k = 100 everywhere / k = 0..99 linear over the mesh)
    def timed(fn, reps=2):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps
    cmp = {}
    for g in wl.grids:
        nn, hh = wl.n[g], wl.h[g]
        u, f = wl.view("u" + g), wl.view("f" + g)
        tb = timed(lambda: st.stencil_smooth_coloured(u, f, hh, 10, op=st.OP_FD)) / 10
        td = timed(lambda: st.stencil_smooth_depend(u, f, hh, 10)) / 10
        cmp["redblack_%sd" % g] = {"barrier_ms_per_sweep": round(tb, 4), "depend_ms_per_sweep": round(td, 4)}
        ns = 128 if g == "3" else 2048  # S(k): FP64 sin-bound, a smaller grid
        hs = 1.0 / ns
        us = torch.from_numpy(synth.uniform_field(synth.grid_shape(int(g), ns), 1)).to(dev)
        fs = torch.from_numpy(synth.uniform_field(synth.grid_shape(int(g), ns), 2)).to(dev)
        ups = interior(int(g), ns)
        for mode, name in ((st.COST_UNIFORM, "k100"), (st.COST_LINEAR, "k0to99")):
            tb = timed(lambda: st.stencil_smooth_expensive(us, fs, hs, 1, mode, 100))
            td = timed(lambda: st.stencil_smooth_expensive(us, fs, hs, 1, mode, 100, depend={}))
            cmp["expensive_%s_%sd_n%d" % (name, g, ns)] = {
                "barrier_mupd_s": round(ups / tb / 1e3, 1), "depend_mupd_s": round(ups / td / 1e3, 1)}
    return {"metric": "Mupdates/s (5/7-point FD op mix: 50 stencil applies, 50 red-black GS sweeps, "
                      "50 Jacobi sweeps, 1 residual per grid)", "workload": "fd", "redblack_and_expensive": cmp,
            "value": round(upd / (ms * 1e-3) / 1e6, 1), "unit": "Mupdates/s", "steps": steps,
            "ms_per_step": round(ms / steps, 3), "grid_3d": n3, "grid_2d": n2, "dtype": "f64",
            "clocks": clock_info, "per_op": per}


def run_refine(args):
    """256^3, f from u* = sin(2 pi x) sin(3 pi y) sin(pi z): refinement to a relative
    residual of 1e-10 with 8 inner GS sweeps in FP32 and in bf16 storage, against plain
    FP64 coloured GS (inner FP64, same loop) to the same residual; error of each result
    against the closed-form discrete solution."""
    import torch
    import paper_1810_04033_gb300 as st
    n, h = 256, 1.0 / 256
    modes = (2, 3, 1)
    f = synth.sin_rhs(3, n, modes)
    lam = 0.0
    a = [2 - 2 * math.cos(m * math.pi * h) for m in modes]
    mm = [(2 + math.cos(m * math.pi * h)) / 3 for m in modes]
    lam = a[0] * mm[1] * mm[2] + mm[0] * a[1] * mm[2] + mm[0] * mm[1] * a[2]
    uh = h * h * f / lam
    # rows padded to a 64-byte multiple (pitch 264), as in the grid workload: every
    # precision then runs its TMA-staged kernels
    pitch = pitch2(n)

    def padded(a):
        buf = torch.zeros(a.shape[:-1] + (pitch,), dtype=torch.float64, device="cuda")
        v = buf[..., :a.shape[-1]]
        v.copy_(torch.from_numpy(a).cuda())
        return v

    fd = padded(f)
    out = {}
    clocks = ClockSampler(0)
    clocks.start()
    for name, prec in (("fp64", st.F64), ("fp32", st.F32), ("bf16", st.BF16)):
        ud = padded(np.zeros_like(f))
        torch.cuda.synchronize()
        t = time.perf_counter()
        res = st.stencil_solve(ud, fd, h, rel_tol=1e-10, max_outer=20000, inner_sweeps=8, inner_dtype=prec,
                               history=False)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t
        err = float(np.max(np.abs(ud.cpu().numpy() - uh)) / np.max(np.abs(uh)))
        out[name] = {"seconds": round(sec, 3), "corrections": res["iterations"], "sweeps": 8 * res["iterations"],
                     "relres": res["relres"], "converged": res["converged"], "rel_err_vs_closed_form": err}
    # the multigrid solver (FP64 V(2,2) cycles) on the same problem, for comparison
    ud = padded(np.zeros_like(f))
    st.stencil_mg_solve(ud, fd, h, rel_tol=1e-10, max_cycles=50, history=False)  # workspace warm-up
    ud.zero_()
    torch.cuda.synchronize()
    t = time.perf_counter()
    res = st.stencil_mg_solve(ud, fd, h, rel_tol=1e-10, max_cycles=50, history=False)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t
    err = float(np.max(np.abs(ud.cpu().numpy() - uh)) / np.max(np.abs(uh)))
    out["mg"] = {"seconds": round(sec, 4), "cycles": res["cycles"], "levels": res["levels"],
                 "relres": res["relres"], "converged": res["converged"], "rel_err_vs_closed_form": err}
    clock_info = clocks.stop()
    if args.no_cpu:  # timing only (e.g. under a profiler): no oracle runs
        return {"metric": "time to relative residual 1e-10, 256^3 (speedup of mixed precision over FP64)",
                "workload": "refine", "value": round(out["fp64"]["seconds"] / out["fp32"]["seconds"], 3),
                "unit": "x (FP64 time / FP32-inner time)", "pitch": pitch, "runs": out, "clocks": clock_info}
    # error per iterate: the GPU's iterates 1..K of each inner precision against the FP64
    # oracle's iterates (plain FP64 inner sweeps, same loop) and against the oracle of the
    # same precision; K bounded by the oracle's host time (one correction of 8 sweeps
    # at 256^3 is ~1.4e8 updates)
    import oracle
    K = 3
    t = time.perf_counter()
    ref = {}
    for name, po in (("fp64", 0), ("fp32", 1), ("bf16", 2)):
        _, _, _, _, hist = oracle.ir_solve(np.zeros_like(f), f, h, 0.0, K, 8, po, keep_history=True)
        ref[name] = hist
    osec = time.perf_counter() - t
    per_iter = {}
    for name, prec in (("fp64", st.F64), ("fp32", st.F32), ("bf16", st.BF16)):
        rows = []
        for k in range(1, K + 1):
            ud = padded(np.zeros_like(f))
            st.stencil_solve(ud, fd, h, rel_tol=0.0, max_outer=k, inner_sweeps=8, inner_dtype=prec, history=False)
            x = ud.cpu().numpy()
            nrm = float(np.max(np.abs(ref["fp64"][k - 1])))
            rows.append({"iterate": k,
                         "rel_err_vs_fp64_oracle": float(np.max(np.abs(x - ref["fp64"][k - 1])) / nrm),
                         "rel_err_vs_same_precision_oracle":
                             float(np.max(np.abs(x - ref[name][k - 1])) / float(np.max(np.abs(ref[name][k - 1]))))})
        per_iter[name] = rows
    # cpu baseline: the oracle's FP64-inner refinement, per correction (K corrections,
    # timed above together with the other precisions: a third of the time each)
    upd_corr = 8 * (n - 1) ** 3 + (n - 1) ** 3
    orate = upd_corr * K / (osec / 3) / 1e6
    return {"metric": "time to relative residual 1e-10, 256^3 (speedup of mixed precision over FP64)",
            "workload": "refine", "value": round(out["fp64"]["seconds"] / out["fp32"]["seconds"], 3),
            "mg_speedup_over_fp64_refinement": round(out["fp64"]["seconds"] / out["mg"]["seconds"], 1),
            "unit": "x (FP64 time / FP32-inner time)", "bf16_speedup": round(out["fp64"]["seconds"] /
                                                                             out["bf16"]["seconds"], 3),
            "pitch": pitch, "runs": out, "clocks": clock_info, "per_iterate_error": per_iter,
            "cpu_baseline": {"value": round(orate, 2), "unit": "Mupdates/s", "cores": 1, "kind": "oracle",
                             "sample": "%d refinement corrections (8 GS sweeps + a residual each) at 256^3 in each "
                                       "of FP64, FP32, bf16 inner precision, %.1f s in all; rate of one precision"
                                       % (K, osec),
                             "fp64_refinement_to_1e-10_s_extrapolated":
                                 round(out["fp64"]["corrections"] * osec / 3 / K, 1)}}


def run_serve(args):
    """Request server: per arrival rate, `requests` requests from the seeded stream
    (edge log-uniform in [16, 256], SMOOTH = 20 GS sweeps or SOLVE to 1e-8 with FP32
    inner sweeps, f drawn on the device from each request's seed), Poisson arrivals;
    p50 / p99 latency (submit to done) and aggregate Mupdates/s."""
    import torch
    import paper_1810_04033_gb300 as st
    lines = []
    for rate in [float(r) for r in args.rates.split(",")]:
        reqs = synth.request_stream(args.requests, rate, seed=3)
        solver = st.SOLVER_MG if args.solver == "mg" else st.SOLVER_REFINE
        srv = st.Server(64 << 30, streams=8, max_inflight=64, inner_dtype=st.F32, solver=solver)
        torch.cuda.synchronize()
        clocks = ClockSampler(0)
        clocks.start()
        # a client that takes each result as it completes: a collector thread waits on
        # the tickets in submission order and releases each result (its resident grid
        # counts against the HBM budget until then); ctypes calls drop the GIL
        import queue
        inbox = queue.Queue()
        lat, upd = [], [0]

        def collect():
            while True:
                item = inbox.get()
                if item is None:
                    return
                t, r = item
                res = srv.wait(t)
                lat.append(res["t_done"] - res["t_submit"])
                if r["kind"] == "smooth":
                    upd[0] += 20 * (r["edge"] - 1) ** 3
                elif args.solver == "mg":
                    upd[0] += res["iterations"] * mg_cycle_updates(r["edge"])
                else:
                    upd[0] += 8 * res["iterations"] * (r["edge"] - 1) ** 3
                srv.release(t)

        collector = threading.Thread(target=collect, daemon=True)
        collector.start()
        t0 = time.perf_counter()
        for r in reqs:
            while time.perf_counter() - t0 < r["t"]:
                time.sleep(0.0002)
            kind = st.REQ_SOLVE if r["kind"] == "solve" else st.REQ_SMOOTH
            inbox.put((srv.submit(kind, r["edge"], sweeps=20, rel_tol=1e-8, f_seed=r["seed"]), r))
        inbox.put(None)
        collector.join()
        upd = upd[0]
        wall = time.perf_counter() - t0
        clock_info = clocks.stop()
        srv.close()
        lat = np.array(lat)
        lines.append({"rate_req_s": rate, "requests": len(reqs), "clocks": clock_info,
                      "p50_s": round(float(np.percentile(lat, 50)), 4),
                      "p99_s": round(float(np.percentile(lat, 99)), 4), "wall_s": round(wall, 2),
                      "requests_per_s": round(len(reqs) / wall, 1),
                      "aggregate_mupdates_s": round(upd / wall / 1e6, 1)})
    return {"metric": "serving: p50/p99 latency and aggregate Mupdates/s", "workload": "serve",
            "value": lines[0]["aggregate_mupdates_s"], "unit": "Mupdates/s", "solver": args.solver,
            "updates": "GS vertex updates (multigrid: smoothing sweeps on every level)", "per_rate": lines}


def mg_cycle_updates(n, pre=2, post=2, coarse=20):
    """GS vertex updates of one V(pre, post) cycle on an n^3 grid (coarsened while n is
    even and n / 2 >= 2; `coarse` sweeps on the coarsest grid)."""
    tot = 0
    while n % 2 == 0 and n // 2 >= 2:
        tot += (pre + post) * (n - 1) ** 3
        n //= 2
    return tot + coarse * (n - 1) ** 3


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.workload != "grid" and args.impl == "gpu":
        import torch
        torch.cuda.set_device(0)
        fn = {"small": run_small, "patches": run_patches, "refine": run_refine, "serve": run_serve,
              "fd": run_fd}[args.workload]
        if rank == 0:
            print(json.dumps(fn(args)))
        return
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out))
        return
    if world > 1:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        torch.distributed.init_process_group("nccl")
    out = run_gpu(args, rank, world)
    if rank == 0:
        if not args.no_cpu:
            out["cpu_baseline"] = cpu_baseline()
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
