"""The benchmark's host logic on CPU: the reference arm's JSON line (the oracle timed
on the host cores, no host-device copies), alone and under two ranks; the unit counts
the rates divide by; the rule that drops DRAM-traffic figures taken on other sources."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n3", "16", "--n2", "64",
                          "--steps", "1", "--warmup", "0"], cwd=ROOT, capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["higher_is_better"] is True and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    assert "workload" in d["config"]


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_unit_counts():
    """Updates, bytes and rates the benchmark divides by, checked by hand."""
    b = _bench()
    passes = 50 + 50 + 50 + 50 + 1
    assert b.updates_per_step(512, 16384) == passes * (511 ** 3 + 16383 ** 2)
    assert b.updates_per_step(0, 64) == passes * 63 ** 2
    assert b.interior(3, 0) == 0
    assert b.bytes_per_update("jacobi_sweep", "2") == 12      # two sweeps per pass over memory
    assert b.bytes_per_update("jacobi_sweep", "3") == 24
    assert b.bytes_per_update("jacobi_sweep", "2", fd=True) == 24
    assert b.bytes_per_update("gs_sweep", "2") == 12          # two sweeps per pass too
    assert b.bytes_per_update("gs_sweep", "3") == 24
    p = b.pitch2(16384)
    assert p >= 16385 and p % 8 == 0 and p - 16385 < 8       # 64-byte rows, minimal padding
    # V(2,2) on 8^3: levels 8, 4 (2 is the coarsest: 20 sweeps on its single interior vertex)
    assert b.mg_cycle_updates(8) == 4 * 7 ** 3 + 4 * 3 ** 3 + 20 * 1
    # weak scaling: every rank does the same units; the slowest rank's time counts
    assert b.whole_job_rate(1e6, 4, 1000.0) == pytest.approx(4.0)
    # launches per step: 3D 2x50 applies, GS 2 launches per sweep + 2 pre-passes, Jacobi
    # 1 per sweep + 2, residual 1; 2D the same except GS and Jacobi 1 per 2 sweeps
    assert b.launches_per_step(512, 16384) == (100 + 102 + 52 + 1) + (100 + 27 + 27 + 1)
    # FP64-pipe fraction of the finite-difference kernels: 7 FP64 instructions per 3D
    # apply update, 1e6 updates in 1 ms on 152 SMs at 2 per clock and 2.07 GHz
    assert b.fd_fp64_frac("apply_stencil", "3", 1e6, 1.0, 152) == pytest.approx(7e9 / (2 * 152 * 2.07e9))
    assert b.FD_FP64_OPS["residual"]["2"] == 8 and b.FD_FP64_OPS["jacobi_sweep"]["3"] == 9


def test_traffic_is_dropped_when_the_kernel_sources_change(tmp_path, monkeypatch):
    """A committed DRAM-traffic line counts only for the sources of its own kernel: an
    edit to another kernel's file keeps it, an edit to its kernel file, to api.cu or to
    a header drops it."""
    import shutil
    b = _bench()
    csrc = os.path.join(ROOT, "paper_1810_04033_gb300", "csrc")
    for key, files in b.TRAFFIC_SOURCES.items():
        for fn in files:
            assert os.path.exists(os.path.join(csrc, fn)), (key, fn)
    keys = list(b.TRAFFIC_SOURCES)
    got = {k: b.traffic_from_profiles(k, 1000.0) for k in keys}
    assert all(v is None or v > 0 for v in got.values())
    root = tmp_path / "repo"
    shutil.copytree(os.path.join(ROOT, "profiles"), root / "profiles")
    shutil.copytree(csrc, root / "paper_1810_04033_gb300" / "csrc")
    monkeypatch.setattr(b, "ROOT", str(root))
    assert {k: b.traffic_from_profiles(k, 1000.0) for k in keys} == got

    def edit(fn):
        src = root / "paper_1810_04033_gb300" / "csrc" / fn
        src.write_text(src.read_text() + "\n// edited\n")

    edit("patches.cu")  # no grid-workload kernel lives there
    assert {k: b.traffic_from_profiles(k, 1000.0) for k in keys} == got
    edit("gs_fx.cu")    # the 3D GS kernels and the smoothers' pre-passes
    after = {k: b.traffic_from_profiles(k, 1000.0) for k in keys}
    for k in ("gs_sweep_3d", "jacobi_sweep_3d", "gs_sweep_2d", "jacobi_sweep_2d"):
        assert after[k] is None
    for k in ("apply_elementwise_2d", "apply_stencil_2d", "residual_2d", "apply_elementwise_3d"):
        assert after[k] == got[k]
    edit("fixed.cuh")   # shared by every kernel
    assert all(b.traffic_from_profiles(k, 1000.0) is None for k in keys)
    assert b.traffic_from_profiles("no_such_kernel", 1000.0) is None


def test_reference_arm_under_two_ranks_prints_once():
    """Launched like the multi-GPU runs (torchrun, 2 ranks): rank 0 alone times the oracle
    and prints; the other rank exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", "29531", "bench.py", "--impl", "reference",
           "--gpus", "2", "--n3", "16", "--n2", "64", "--steps", "1", "--warmup", "0"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0


def test_patches_oracle_sample_counts_interior_updates():
    """The patch workload's CPU baseline: updates = sweeps x sum over patches of (n-1)^3."""
    import numpy as np
    b = _bench()
    import synth
    upd, sec = b.patches_oracle_sample(1, lat=(2, 2, 1), sweeps=3)
    L = synth.PatchLattice(lat=(2, 2, 1), seed=2)
    assert upd == 3 * int(np.sum((L.np_sizes.astype(np.int64) - 1) ** 3)) and sec > 0
