"""Benchmark: coloured Q1 stencil sweeps on one large FP64 grid per GPU.

Workload (one "step" = one pass of the hot path over the resident grids):
  3D: 512^3 cells (513^3 vertices, FP64), unit cube, homogeneous Dirichlet boundary,
      u0 ~ U[-1,1] (seed 1), f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z);
  2D: 16384^2 cells (16385^2 vertices, FP64, row pitch padded to 16392), same fields;
  per grid and step: element-wise apply, stencil apply, 1 coloured Gauss-Seidel sweep,
  1 damped Jacobi sweep (omega = 2/3), residual with norms.
  --steps 50 reproduces 100 applies + 50 GS + 50 Jacobi sweeps per grid.
Metric: interior-vertex updates per second (Mupdates/s), whole job.
Inputs are larger than L2 (1.08 GB / 2.15 GB per array), so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

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
PITCH2 = 16392  # 16385 rounded up to a multiple of 8 doubles (64 B)
OMEGA = 2.0 / 3.0
OPS = ("apply_elementwise", "apply_stencil", "gs_sweep", "jacobi_sweep", "residual")
# algorithmic HBM bytes per interior update (compulsory traffic of one pass)
BYTES_PER_UPDATE = {"apply_elementwise": 16, "apply_stencil": 16, "gs_sweep": 24,
                    "jacobi_sweep": 24, "residual": 16}
# kernel launches of our library per op and grid (3D GS: 4 row phases; 2D: 4 colours)
LAUNCHES_PER_OP = {"apply_elementwise": 1, "apply_stencil": 1, "gs_sweep": 4,
                   "jacobi_sweep": 1, "residual": 1}


def interior(dim, n):
    return (n - 1) ** dim


def updates_per_step():
    return len(OPS) * (interior(3, N3) + interior(2, N2))


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
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
    def __init__(self, torch, st, device):
        self.torch, self.st, self.dev = torch, st, device
        self.h3, self.h2 = 1.0 / N3, 1.0 / N2
        s3 = synth.grid_shape(3, N3)
        self.host = {}
        u3 = synth.uniform_field(s3, 1)
        f3 = synth.sin_rhs(3, N3)
        u2 = synth.uniform_field(synth.grid_shape(2, N2), 1)
        f2 = synth.sin_rhs(2, N2)
        # pinned host copies for the end-to-end leg
        self.host["u3"] = torch.from_numpy(u3).pin_memory()
        self.host["f3"] = torch.from_numpy(f3).pin_memory()
        self.host["u2"] = self._pad2(torch.from_numpy(u2)).pin_memory()
        self.host["f2"] = self._pad2(torch.from_numpy(f2)).pin_memory()
        del u3, f3, u2, f2
        d = {}
        for g in ("3", "2"):
            d["u" + g] = self.host["u" + g].to(device)
            d["f" + g] = self.host["f" + g].to(device)
            d["y" + g] = torch.empty_like(d["u" + g])
            d["ja" + g] = d["u" + g].clone()
            d["jb" + g] = torch.empty_like(d["u" + g])
            d["n" + g] = torch.zeros(2, dtype=torch.float64, device=device)
        self.d = d
        self.jflip = 0

    @staticmethod
    def _pad2(t):
        import torch
        buf = torch.zeros((t.shape[0], PITCH2), dtype=t.dtype)
        buf[:, :t.shape[1]] = t
        return buf

    def view(self, key):
        t = self.d[key]
        return t[:, :N2 + 1] if key.endswith("2") else t

    def run_op(self, op, g, stream):
        st = self.st
        h = self.h3 if g == "3" else self.h2
        u, f, y = self.view("u" + g), self.view("f" + g), self.view("y" + g)
        if op == "apply_elementwise":
            st.stencil_apply(u, y, h, st.FORM_ELEMENTWISE, stream=stream)
        elif op == "apply_stencil":
            st.stencil_apply(u, y, h, st.FORM_STENCIL, stream=stream)
        elif op == "gs_sweep":
            st.stencil_smooth_coloured(u, f, h, 1, stream=stream)
        elif op == "jacobi_sweep":
            a, b = ("ja", "jb") if self.jflip == 0 else ("jb", "ja")
            st.stencil_jacobi_step(self.view(a + g), f, self.view(b + g), h, OMEGA, stream=stream)
        elif op == "residual":
            st.stencil_residual(u, f, h, norms2=self.d["n" + g], stream=stream)

    def step(self, stream, events=None):
        for g in ("3", "2"):
            for op in OPS:
                if events is not None:
                    events[(op, g)][0].record(stream)
                self.run_op(op, g, stream)
                if events is not None:
                    events[(op, g)][1].record(stream)
        self.jflip ^= 1


def traffic_from_profiles(kernel_key, units_per_launch):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the
    current kernel source (null otherwise)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    src = os.path.join(ROOT, "paper_1810_04033_gb300", "csrc")
    if not os.path.exists(path):
        return None
    sha = hashlib.sha256()
    for fn in sorted(os.listdir(src)):
        if fn.endswith((".cu", ".h")):
            sha.update(open(os.path.join(src, fn), "rb").read())
    cur = sha.hexdigest()[:16]
    for line in open(path):
        m = re.match(r"\s*kernel=(\S+)\s+src_sha=(\S+)\s+dram_bytes_per_update=([\d.eE+-]+)", line)
        if m and m.group(1) == kernel_key and m.group(2) == cur:
            return float(m.group(3)) * units_per_launch
    return None


def run_gpu(args, rank, world):
    import torch
    import paper_1810_04033_gb300 as st

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    st.lib()
    wl = GpuWorkload(torch, st, dev)
    stream = torch.cuda.Stream(device=dev)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            wl.step(stream)
    stream.synchronize()

    # one pair of events per op, grid and step; read only after the timed region
    ev = [{(op, g): (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for op in OPS for g in ("3", "2")} for _ in range(args.steps)]
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
    ms_max = ms
    if world > 1:
        tt = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        ms_max = float(tt.item())
    total_updates = updates_per_step() * args.steps * world
    value = total_updates / (ms_max * 1e-3) / 1e6

    # dominant kernel: the op (summed over both grids' launches) with the largest time
    agg = {}
    for (op, g), t in per_op_ms.items():
        agg.setdefault(op, 0.0)
        agg[op] += t
    top = max(agg, key=agg.get)
    top3 = per_op_ms[(top, "3")] / args.steps  # ms per 3D op
    units3 = interior(3, N3)
    launches = LAUNCHES_PER_OP[top]
    achieved = BYTES_PER_UPDATE[top] * units3 / (top3 * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": top + " (3D 513^3)", "achieved": round(achieved, 1),
                "peak": hbm_peak, "unit": "GB/s", "frac": round(achieved / hbm_peak, 4),
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)",
                "traffic": traffic_from_profiles(top + "_3d", units3 / launches),
                "per_op_ms_3d": {op: round(per_op_ms[(op, "3")] / args.steps, 3) for op in OPS},
                "per_op_ms_2d": {op: round(per_op_ms[(op, "2")] / args.steps, 3) for op in OPS}}

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(torch, st, wl, stream, args, world)

    out = {"metric": "Mupdates/s (interior-vertex updates, FP64 Q1 apply x2 + coloured GS + "
                     "damped Jacobi + residual, 3D 512^3 + 2D 16384^2)",
           "value": round(value, 1), "unit": "Mupdates/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded U[-1,1] u0, manufactured sin RHS)",
           "config": {"workload": "configs[1]: 512^3 FP64 Q1 + 2D 9-point 16384^2 FP64; per step "
                                  "apply(element-wise) + apply(stencil) + 1 GS sweep + 1 Jacobi "
                                  "sweep (omega 2/3) + residual on each grid",
                      "grid_3d": [N3 + 1] * 3, "grid_2d": [N2 + 1, N2 + 1], "pitch_2d": PITCH2,
                      "l2": "inputs larger than L2 (1.08 GB / 2.15 GB arrays), no flush",
                      "parallelism": "replicas" if world > 1 else "single GPU"},
           "roofline": roofline, "clocks": clock_info,
           "gpu_launches": sum(LAUNCHES_PER_OP[op] for op in OPS) * 2 * args.steps,
           "e2e": e2e}
    return out


def run_e2e(torch, st, wl, stream, args, world):
    """Same op mix through the public API with host buffers: every step copies u and f
    of both grids from pinned host memory, runs the ops, and reads u and the norms
    back.  Copies are inside the timed region."""
    steps = max(2, min(args.steps, 5))
    h_out = {g: torch.empty_like(wl.host["u" + g]).pin_memory() for g in ("3", "2")}
    h_nrm = torch.empty(4, dtype=torch.float64).pin_memory()
    bi = sum(wl.host[k].numel() * 8 for k in ("u3", "f3", "u2", "f2"))
    bo = sum(h_out[g].numel() * 8 for g in h_out) + 32

    def one(stream):
        for g in ("3", "2"):
            wl.d["u" + g].copy_(wl.host["u" + g], non_blocking=True)
            wl.d["f" + g].copy_(wl.host["f" + g], non_blocking=True)
        wl.step(stream)
        for i, g in enumerate(("3", "2")):
            h_out[g].copy_(wl.d["u" + g], non_blocking=True)
            h_nrm[2 * i:2 * i + 2].copy_(wl.d["n" + g], non_blocking=True)

    with torch.cuda.stream(stream):
        one(stream)
        stream.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(steps):
            one(stream)
        t1.record(stream)
    stream.synchronize()
    ms = t0.elapsed_time(t1)
    if world > 1:
        tt = torch.tensor([ms], device=wl.dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        ms = float(tt.item())
    val = updates_per_step() * steps * world / (ms * 1e-3) / 1e6
    return {"value": round(val, 1), "unit": "Mupdates/s", "h2d_bytes_per_step": bi,
            "d2h_bytes_per_step": bo, "steps": steps}


# ------------------------------------------------------------------ CPU oracle
def oracle_sample(n3, n2, nthreads):
    """One pass of the op mix through the oracle on grids of n3^3 and n2^2 cells.
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
    n3, n2 = 256, 8192
    upd, sec = oracle_sample(n3, n2, nthreads)
    return {"value": round(upd / sec / 1e6, 2), "unit": "Mupdates/s", "cores": nthreads,
            "kind": "oracle",
            "sample": "one pass of the same op mix (element-wise apply, stencil apply, 1 GS "
                      "sweep, 1 Jacobi sweep, residual) on a 256^3 and an 8192^2 grid, "
                      "%.1f s, OpenMP colour-pass parallel for" % sec}


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
    return {"impl": "reference", "metric": "Mupdates/s (interior-vertex updates, FP64 Q1 apply x2 "
                                           "+ coloured GS + damped Jacobi + residual, 3D 512^3 + "
                                           "2D 16384^2)",
            "value": round(val, 2), "unit": "Mupdates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(sec_tot / args.steps * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "configs[1] op mix, oracle on host cores; "
                                                        "each step a bounded sample: 128^3 + 2048^2"},
            "cpu_baseline": {"value": round(val, 2), "unit": "Mupdates/s", "cores": nthreads,
                             "kind": "oracle", "sample": "per step: op mix on 128^3 and 2048^2"},
            "e2e": {"value": round(val, 2), "unit": "Mupdates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
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
