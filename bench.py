#!/usr/bin/env python3
"""Throughput benchmark of the scattering-graph voxel path on GB300.

A step is one whole scene: set the medium, assemble K and s, solve
(I - K) x = s to a relative FP64 residual of 1e-10 (FP32 SpMV, FP64
refinement), render the 64x64 detector.  The workload is the plume scene of
64x64x32 voxels with the 124-neighbour stencil (16.8M edges).  The graph
structure (per shape) is built once before timing.

Default: 1 GPU, 200 timed steps after 3 warm-up steps; L2 is flushed (256 MB
write) between timed steps, outside the timed interval.  Under torchrun each
rank runs an independent replica (weak scaling; the path has no exchange).

``--impl reference`` times the FP64 CPU oracle on the host cores instead.
``--c-min C`` (coupling selection, scattering graph with C > c_min) and
``--shape NXxNYxNZ`` and ``--aniso`` (the edge unknowns, arrival direction
kept) time variants of the plume scene; their lines are not the
headline and skip the CPU baseline, the adjoint, the cloud and serving.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "scenes/s and edges/s at 64²×32 (rel err ≤1e-4 vs FP64), %HBM roofline; p50/p99 served"
WORKLOAD = "plume 64x64x32 voxels (50x50x100 m), R=2 stencil (124 neighbours), 2 species + gas, SZA 60 VZA 30, " \
           "64x64 detector; FP32 assembly+SpMV, FP64 refinement to rel. residual 1e-10"
RTOL = 1e-10


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--no-cloud", action="store_true")  # skip the cloud scene and the per-config timings
    p.add_argument("--solver", type=int, default=0)
    # variants (not the headline): coupling selection with threshold c_min
    # (Sec. 2, scattering graph C > c_min) and other plume shapes
    p.add_argument("--c-min", type=float, default=0.0)
    p.add_argument("--shape", default="64x64x32")
    p.add_argument("--workload", default="plume", choices=["plume", "cloud"])  # cloud: a variant line
    p.add_argument("--aniso", action="store_true")  # edge unknowns (arrival direction kept)
    # solve tolerance (relative FP64 residual); default 1e-10, and 1e-8 for
    # the edge unknowns (their FP32 coefficients hold the radiances to ~2e-7
    # of the FP64 oracle either way)
    p.add_argument("--rtol", type=float, default=None)
    p.add_argument("--oracle-times", action="store_true", help=argparse.SUPPRESS)  # child: oracle timings
    # the coupling study of the paper on the synthetic plume: radiance against the kept number of couplings
    p.add_argument("--coupling-sweep", action="store_true")
    return p.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# nominal dense TF32 / BF16 tensor rate of this part (1.1 / 2.25 PFLOP/s)
TF32_PER_BF16 = 1.1 / 2.25


def tf32_peak():
    """TF32 tensor peak: the measured sustained BF16 GEMM rate (a kernel timed
    inside a long step) times the nominal TF32 / BF16 ratio."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops_sustained"]) * TF32_PER_BF16, "measured bf16 sustained x nominal tf32/bf16"
    except Exception:
        return 1700.0 * TF32_PER_BF16, "fallback bf16 sustained x nominal tf32/bf16"


# the sources each traffic record depends on
TRAFFIC_SOURCES = {
    "k_tile_OpCheb": ("kernels_solve.cu", "stage.cuh", "kern.h"),
    "assembly": ("kernels_asm.cu", "asm_util.cuh", "stage.cuh", "kern.h"),
    "cloud_gmres_prod": ("kernels_solve.cu", "stage.cuh", "kern.h"),
}


def traffic_record(kernel: str):
    """Per-launch DRAM bytes of a kernel from the committed ncu summary, if the
    summary's source hash matches the kernel source as it is now."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    csrc = os.path.join(ROOT, "paper_2503_16037_gb300", "csrc")
    try:
        h = hashlib.sha256()
        for f in TRAFFIC_SOURCES[kernel]:
            h.update(open(os.path.join(csrc, f), "rb").read())
        sha = h.hexdigest()[:16]
        for line in open(path):
            parts = line.split()
            if len(parts) >= 3 and parts[0] == kernel and parts[1] == sha:
                return float(parts[2])
    except OSError:
        pass
    return None


class NvmlClocks:
    """SM clock and throttle-reason sampling through NVML (read-only queries),
    every ~2 ms in a thread during the timed region."""

    HW_SLOWDOWN, SW_THERMAL, HW_THERMAL, SW_POWER_CAP = 0x8, 0x20, 0x40, 0x4

    def __init__(self, uuid=None, pci=None):
        import ctypes
        self.ok = False
        self.samples = []
        try:
            self.L = ctypes.CDLL("libnvidia-ml.so.1")
        except OSError:
            return
        self.c = ctypes
        if self.L.nvmlInit_v2() != 0:
            return
        self.h = ctypes.c_void_p()
        # the device torch runs on, by UUID (else PCI address): NVML indices
        # need not follow CUDA_VISIBLE_DEVICES
        found = False
        if uuid:
            found = self.L.nvmlDeviceGetHandleByUUID(("GPU-" + uuid).encode(), ctypes.byref(self.h)) == 0
        if not found and pci:
            found = self.L.nvmlDeviceGetHandleByPciBusId_v2(pci.encode(), ctypes.byref(self.h)) == 0
        self.ok = found

    def _one(self):
        c = self.c
        sm, mx, rs = c.c_uint(0), c.c_uint(0), c.c_ulonglong(0)
        if self.L.nvmlDeviceGetClockInfo(self.h, 1, c.byref(sm)) != 0:  # NVML_CLOCK_SM
            return None
        self.L.nvmlDeviceGetMaxClockInfo(self.h, 1, c.byref(mx))
        self.L.nvmlDeviceGetCurrentClocksEventReasons(self.h, c.byref(rs))
        return sm.value, mx.value, rs.value

    def start(self):
        if not self.ok:
            return
        self.stop_flag = False

        def run():
            while not self.stop_flag:
                v = self._one()
                if v:
                    self.samples.append(v)
                time.sleep(0.002)
        self.th = threading.Thread(target=run, daemon=True)
        self.th.start()

    def stop(self):
        if not self.ok:
            return None
        self.stop_flag = True
        self.th.join(timeout=2)
        v = self._one()  # at least one sample taken at the end of the region
        if v:
            self.samples.append(v)
        if not self.samples:
            return None
        reasons = set()
        for _, _, r in self.samples:
            for bit, name in ((self.HW_SLOWDOWN, "hw_slowdown"), (self.HW_THERMAL, "hw_thermal_slowdown"),
                              (self.SW_THERMAL, "sw_thermal_slowdown"), (self.SW_POWER_CAP, "sw_power_cap")):
                if r & bit:
                    reasons.add(name)
        return {"sm_mhz": statistics.median(x[0] for x in self.samples),
                "sm_max_mhz": max(x[1] for x in self.samples), "samples": len(self.samples),
                "reasons": sorted(reasons), "source": "NVML, polled every ~2 ms"}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, bus_id=None):
        self.lines = []
        self.proc = None
        self.bus_id = bus_id

    def start(self):
        cmd = ["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS), "--format=csv,noheader,nounits", "-lms", "50"]
        if self.bus_id:
            cmd += ["--id=" + self.bus_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def max_over_ranks(x, dist=None):
    """The largest x over all ranks (the slowest replica's time); x itself
    when there is one rank.  The all-reduce runs on the GPU under NCCL and on
    the host under gloo."""
    if dist is None:
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, steps, slowest_s):
    """Scenes per second of the whole job: every rank runs `steps` scenes of
    its own replica, and the job ends with the slowest rank."""
    return world * steps / slowest_s


def cpu_baseline(sc, full=True):
    """The FP64 oracle as it stands, on all host cores, on one scene."""
    from oracle import oracle
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    r = oracle.run(sc, threads=cores)
    t = time.perf_counter() - t0
    return r, t, cores


def run_reference(args, rank):
    """Reference arm: the FP64 CPU oracle, timed on the host cores, one full
    plume scene (64x64x32, the headline workload) per step."""
    if rank != 0:
        return
    from paper_2503_16037_gb300 import scenes
    from oracle import oracle
    oracle.build()
    sample = scenes.make_plume()
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.run(sample, threads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.run(sample, threads=cores)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "scenes/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": "one full plume scene 64x64x32 per step (all stages)"},
        "cpu_baseline": {"value": value, "unit": "scenes/s", "cores": cores, "kind": "oracle",
                         "sample": "one full plume scene 64x64x32 per step, FP64 C oracle with OpenMP on all "
                                   "host cores"},
        "e2e": {"value": value, "unit": "scenes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def oracle_times():
    """FP64 oracle wall time per scene for the three workloads of the method
    (8^3 plain, 64x64x32 plume, 128x128x40 cloud), single-threaded and on all
    host cores; run in a child process (bench.py --oracle-times)."""
    from paper_2503_16037_gb300 import scenes
    from oracle import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    out = {"cores": cores}
    for name, sc in (("plain 8x8x8 R1", scenes.make_plain()), ("plume 64x64x32 R2", scenes.make_plume()),
                     ("cloud 128x128x40 R2", scenes.make_cloud())):
        row = {}
        for th, key in ((cores, "all_cores_s"), (1, "one_thread_s")):
            t0 = time.perf_counter()
            r = oracle.run(sc, threads=th)
            row[key] = time.perf_counter() - t0
            row["gmres_iters"] = r["gmres_iters"]
        out[name] = row
        print(json.dumps(out), flush=True)  # partial results survive a timeout


SERVE_SHAPES = [(16, 16, 16), (32, 32, 24), (48, 48, 32), (64, 64, 32), (96, 96, 32)]


def serving(T, scenes, torch, np, n_requests=1024, workers=8, load=0.8, seed=0, batch_solves=False, plain=True):
    """Continuous-batching serving of plume scenes of uneven sizes (uniform
    over SERVE_SHAPES, SZA ~ U(20, 75) deg, FP32 + refinement to 1e-10):
    the saturation rate with all requests queued at once, then an open-loop
    run with Poisson arrivals at `load` x that rate (latency = completion -
    arrival), then the plain FP64 path (one scene at a time, FP64 solve) on a
    subset of the same requests."""
    import threading
    rng = np.random.default_rng(seed)
    nvar = 8
    pool = {sh: [scenes.make_plume(nx=sh[0], ny=sh[1], nz=sh[2], sza=float(rng.uniform(20.0, 75.0)))
                 for _ in range(nvar)] for sh in SERVE_SHAPES}
    fields = {(sh, k): (torch.as_tensor(sc.mu_a, dtype=torch.float32).pin_memory(),
                        torch.as_tensor(sc.mu_s, dtype=torch.float32).pin_memory())
              for sh, l in pool.items() for k, sc in enumerate(l)}
    reqs = [(SERVE_SHAPES[rng.integers(len(SERVE_SHAPES))], int(rng.integers(nvar))) for _ in range(n_requests)]
    outs = [torch.empty((sh[1], sh[0]), dtype=torch.float32).pin_memory() for sh, _ in reqs]
    srv = T.Server(40 << 30, workers, batch_solves=batch_solves)
    for sh in SERVE_SHAPES:  # one warm request per shape builds its first slot
        srv.wait(srv.submit(pool[sh][0], T.FP32_REFINE, 1e-10, fields=fields[(sh, 0)]))

    def closed(sub):
        t0 = time.perf_counter()
        tk = [srv.submit(pool[sh][k], T.FP32_REFINE, 1e-10, fields=fields[(sh, k)], out=outs[j])
              for j, (sh, k) in sub]
        infos = [srv.wait(t)[1] for t in tk]
        return len(sub) / (time.perf_counter() - t0), infos

    sat, _ = closed(list(enumerate(reqs[:256])))
    rate = load * sat
    gaps = rng.exponential(1.0 / rate, size=n_requests)
    tickets = [None] * n_requests

    def submitter():
        t = time.perf_counter()
        for j, (sh, k) in enumerate(reqs):
            t += gaps[j]
            while True:
                d = t - time.perf_counter()
                if d <= 0:
                    break
                time.sleep(min(d, 0.0005) if d > 0.0002 else 0)
            tickets[j] = srv.submit(pool[sh][k], T.FP32_REFINE, 1e-10, fields=fields[(sh, k)], out=outs[j])

    th = threading.Thread(target=submitter)
    t0 = time.perf_counter()
    th.start()
    infos = []
    for j in range(n_requests):
        while tickets[j] is None:
            time.sleep(0.0001)
        infos.append(srv.wait(tickets[j])[1])
    th.join()
    wall = time.perf_counter() - t0
    lat = np.array([i["end_ms"] - i["submit_ms"] for i in infos])
    svc = np.array([i["end_ms"] - i["start_ms"] for i in infos])
    per_shape = {}
    for (sh, _), v in zip(reqs, svc):
        per_shape.setdefault("%dx%dx%d" % sh, []).append(v)
    per_shape = {k: {"requests": len(v), "service_p50_ms": float(np.percentile(v, 50)),
                     "service_p99_ms": float(np.percentile(v, 99))} for k, v in sorted(per_shape.items())}
    subm = np.array([i["submit_ms"] for i in infos])
    st = srv.stats()
    srv.close()
    ok = all(i["status"] == 0 and i["rel_resid64"] <= 1e-10 for i in infos)
    # the plain FP64 path: one scene per call sequence, nothing overlapped
    base = []
    rn_of = {}
    for sh, k in (reqs[:64] if plain else []):
        if sh not in rn_of:
            rn_of[sh] = T.Runner(pool[sh][0], T.FP64)
        rn = rn_of[sh]
        rn.sc = pool[sh][k]
        rn.geom = T.geometry(pool[sh][k])
        a = torch.as_tensor(pool[sh][k].mu_a, dtype=torch.float64).pin_memory()
        m = torch.as_tensor(pool[sh][k].mu_s, dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        rn.run(a, m, rtol=1e-10)
        rn.rad.cpu()
        base.append(1000.0 * (time.perf_counter() - t1))
    for rn in rn_of.values():
        rn.close()
    base = np.array(base if base else [float("nan")])
    return {
        "workload": "1024 plume scenes, shapes uniform over 16^3, 32^2x24, 48^2x32, 64^2x32, 96^2x32 "
                    "(R = 2), SZA ~ U(20, 75) deg, FP32 + FP64 refinement to 1e-10, host inputs (pinned)",
        "workers": workers, "saturation_scenes_per_s": sat,
        "arrivals": "Poisson at %.2f x saturation (%.0f /s requested, %.0f /s achieved)"
                    % (load, rate, (n_requests - 1) / max(1e-9, (subm.max() - subm.min()) / 1000.0)),
        "scenes_per_s": n_requests / wall, "per_shape_service": per_shape, "p50_ms": float(np.percentile(lat, 50)),
        "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(lat.max()), "all_converged": ok,
        "slots_built": st["slots_built"], "peak_device_bytes": st["peak_bytes"], "evictions": st["evictions"],
        "batched_refinements": {"on": batch_solves, "launches": st["batches"],
                                "refinements": st["batched_refinements"], "max_in_one_launch": st["max_batch"]},
        "plain_fp64_one_scene_at_a_time": {
            "requests": int(base.size), "scenes_per_s": 1000.0 / float(base.mean()),
            "p50_ms": float(np.percentile(base, 50)), "p99_ms": float(np.percentile(base, 99)),
            "note": "service time per scene with nothing overlapped (no queueing)"},
    }


def coupling_sweep(args):
    """Synthetic analogue of the paper's study of the result against the
    amount of scattering coupling (Sec. 4): the plume 64x64x32 solved with the
    K largest couplings kept (TURSCA_OPT_MAX_COUPLINGS), K from all of them
    down to 1%; per K the kept fraction, the radiance change against the full
    stencil (mean and max relative, and of the scene mean), the mean
    reflectance and the time per scene (host clock around a synchronised
    scene, median of 5, L2 flushed; the selection included)."""
    import numpy as np
    import torch
    from paper_2503_16037_gb300 import build as B
    B.build()
    from paper_2503_16037_gb300 import scenes
    from paper_2503_16037_gb300 import tursca as T
    torch.cuda.set_device(0)
    sc = scenes.make_plume()
    stream = torch.cuda.current_stream()
    rn = T.Runner(sc, T.FP32_REFINE, stream=stream)
    mu_a, mu_s = rn.fields("cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def timed():
        ts = []
        for k in range(args.warmup + 5):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rn.run(mu_a, mu_s, rtol=RTOL)
            torch.cuda.synchronize()
            if k >= args.warmup:
                ts.append(time.perf_counter() - t0)
        return 1000.0 * statistics.median(ts)

    ms_full = timed()
    full = rn.rad.double().cpu().numpy()
    refl_full = rn.refl.double().cpu().numpy()
    T.tursca_set_option(rn.handle, T.OPT_MAX_COUPLINGS, 1)
    rn.run(mu_a, mu_s, rtol=RTOL)
    n = T.tursca_selection_info(rn.handle)["n_couplings"]
    rows = [{"K": n, "kept": n, "kept_fraction": 1.0, "ms_per_scene": ms_full, "mean_rel_change": 0.0,
             "max_rel_change": 0.0, "mean_radiance": float(full.mean()), "mean_reflectance": float(refl_full.mean())}]
    for frac in (0.75, 0.5, 0.3, 0.2, 0.1, 0.05, 0.02, 0.01):
        K = int(frac * n)
        T.tursca_set_option(rn.handle, T.OPT_MAX_COUPLINGS, K)
        ms = timed()
        info = T.tursca_selection_info(rn.handle)
        rad = rn.rad.double().cpu().numpy()
        rel = np.abs(rad - full) / np.abs(full)
        rows.append({"K": K, "kept": info["n_kept"], "kept_fraction": info["n_kept"] / n, "threshold": info["threshold"],
                     "ms_per_scene": ms, "mean_rel_change": float(rel.mean()), "max_rel_change": float(rel.max()),
                     "mean_radiance": float(rad.mean()), "mean_reflectance": float(rn.refl.double().mean().item()),
                     "solve_iters": rn.info.iters})
    rn.close()
    print(json.dumps({"metric": "radiance against the kept number of couplings (plume 64x64x32, FP32 + refinement)",
                      "unit": "relative radiance change against the full stencil", "data": "synthetic",
                      "couplings": n, "sweep": rows}), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.oracle_times:
        oracle_times()
        return
    if args.coupling_sweep:
        coupling_sweep(args)
        return

    import numpy as np
    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", rank=rank, world_size=world)
    else:
        torch.cuda.set_device(0)
    from paper_2503_16037_gb300 import build as B
    if rank == 0:
        B.build()
    if dist:
        dist.barrier()
    from paper_2503_16037_gb300 import scenes
    from paper_2503_16037_gb300 import tursca as T

    global RTOL
    if args.rtol is not None:
        RTOL = args.rtol
    elif args.aniso:
        RTOL = 1e-8
    nx, ny, nz = (int(v) for v in args.shape.lower().split("x"))
    variant = args.c_min > 0.0 or (nx, ny, nz) != (64, 64, 32) or args.aniso or args.workload != "plume"
    if args.workload == "cloud":
        sc = scenes.make_cloud().replace(c_min=args.c_min)
        nx, ny, nz = sc.nx, sc.ny, sc.nz
    else:
        sc = scenes.make_plume(nx=nx, ny=ny, nz=nz).replace(c_min=args.c_min)
    stream = torch.cuda.current_stream()
    rn = T.Runner(sc, T.FP32_REFINE, stream=stream)
    if args.aniso:
        T.tursca_set_option(rn.handle, T.OPT_ANISO, 1)
    st = rn.stats
    mu_a, mu_s = rn.fields("cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def step():  # set_medium -> assemble -> solve -> render, one library call (tursca_run)
        rn.run(mu_a, mu_s, rtol=RTOL, solver=args.solver)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()

    uuid = pci = None
    try:
        pr = torch.cuda.get_device_properties(torch.cuda.current_device())
        uuid = str(pr.uuid)
        pci = "%08X:%02X:%02X.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
    except Exception:
        pass
    clk = NvmlClocks(uuid, pci)
    if not clk.ok:
        clk = Clocks(pci)
    clk.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # per-kernel CUDA events are recorded on every PROF_EVERY-th timed step only:
    # an event pair around each launch drains the stream between kernels
    # (about 4 us per launch), which would slow every step if always on
    PROF_EVERY = 8
    l0 = rn.launches()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    iters = []
    prof = {}
    prof_steps = []
    for k in range(args.steps):
        profiled = k % PROF_EVERY == 0
        if profiled:
            T.tursca_profile_enable(rn.handle, True)
        flush.zero_()
        ev0[k].record(stream)
        step()
        ev1[k].record(stream)
        if profiled:
            for name, (n, ms) in T.tursca_profile_read(rn.handle).items():
                a = prof.setdefault(name, [0, 0.0])
                a[0] += n
                a[1] += ms
            T.tursca_profile_enable(rn.handle, False)
            prof_steps.append(k)
        iters.append((rn.info.iters, rn.info.refinements, rn.info.rho_est, rn.info.rel_resid64))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = rn.launches() - l0
    clocks = clk.stop()
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    total_ms = sum(step_ms)
    prof_ms = sum(step_ms[k] for k in prof_steps)
    total_ms = max_over_ranks(total_ms, dist)
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(world, args.steps, total_ms / 1000.0)

    # ---- end to end through the C ABI with host buffers (pinned), copies inside
    mu_a_h = mu_a.cpu().pin_memory()
    mu_s_h = mu_s.cpu().pin_memory()
    rad_h = torch.empty((sc.npy, sc.npx), dtype=torch.float32).pin_memory()
    refl_h = torch.empty((sc.npy, sc.npx), dtype=torch.float32).pin_memory()
    e2e_t = []
    for k in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        T.tursca_run(rn.handle, mu_a_h, mu_s_h, list(sc.g), sc.albedo, rn.geom, args.solver, RTOL, 5000, rad_h,
                     refl_h)  # synchronises
        if k >= args.warmup:
            e2e_t.append(time.perf_counter() - t0)
    e2e_total = sum(e2e_t)
    e2e_total = max_over_ranks(e2e_total, dist)
    e2e_value = whole_job_rate(world, args.steps, e2e_total)
    h2d = mu_a_h.numel() * 4 + mu_s_h.numel() * 4
    d2h = rad_h.numel() * 4 + refl_h.numel() * 4

    # ---- adjoint of the same scene (J = sum_p L_p^2, gradient w.r.t. every
    # voxel's absorption), outside the timed region: time per gradient
    adj = None
    try:
        if variant:
            raise RuntimeError("not measured on a variant run")
        rn.run(mu_a, mu_s, rtol=RTOL)
        lbar = 2.0 * rn.rad
        rn.adjoint(lbar)  # first call allocates the K^T copy
        torch.cuda.synchronize()
        ta = []
        for _ in range(10):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            grad = rn.adjoint(lbar)
            ta.append(time.perf_counter() - t0)
        adj = {"ms_per_gradient": 1000.0 * statistics.median(ta), "objective": "J = sum_p L_p^2",
               "wrt": "absorption coefficient of every voxel (131,072)",
               "timing": "host wall clock around tursca_adjoint (synchronising), median of 10, L2 flushed",
               "grad_abs_max": float(grad.abs().max().item())}
    except Exception as e:  # the bench line must still print
        adj = {"error": str(e)[:200]}

    # ---- the broken-cloud configuration (128 x 128 x 40, ~81M edges), a few
    # scenes outside the timed region: scenes/s of the same FP32 + refinement path
    cloud = None
    if rank == 0 and not args.no_cloud and not variant:
        try:
            csc = scenes.make_cloud()
            crn = T.Runner(csc, T.FP32_REFINE, stream=stream)
            ca, cm = crn.fields("cuda")
            crn.run(ca, cm, rtol=RTOL)
            ct = []
            for _ in range(5):
                flush.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                crn.run(ca, cm, rtol=RTOL)
                torch.cuda.synchronize()
                ct.append(time.perf_counter() - t0)
            cloud = {"workload": "broken cloud 128x128x40 (R = 2, %d edges), FP32 + FP64 refinement to 1e-10"
                                 % crn.stats.nnz_edges,
                     "scenes_per_s": 1.0 / statistics.median(ct), "ms_per_scene": 1000.0 * statistics.median(ct),
                     "edges_per_s": crn.stats.nnz_edges / statistics.median(ct),
                     "solve": {"iters": crn.info.iters, "refinements": crn.info.refinements,
                               "solver": crn.info.solver, "rel_resid64": crn.info.rel_resid64},
                     "timing": "host clock around a synchronised scene, median of 5, L2 flushed"}
            # roofline of the passes over K inside GMRES (K = 4 nnz bytes of
            # values, far beyond L2): one profiled scene, events around each
            # Arnoldi step's run of passes (preconditioner and I - K product)
            flush.zero_()
            T.tursca_profile_enable(crn.handle, True)
            crn.run(ca, cm, rtol=RTOL)
            cprof = T.tursca_profile_read(crn.handle)
            T.tursca_profile_enable(crn.handle, False)
            n_gp, ms_gp = cprof.get("gmres_prod", (0, 0.0))
            if n_gp:
                pb = 4 * crn.stats.nnz + 12 * crn.stats.n_nodes
                avg_s = ms_gp / n_gp / 1000.0
                peak, peak_kind = peaks()
                cloud["roofline"] = {
                    "kernel": "passes over K inside GMRES (k_tile<6, OpSpmv/OpImk<float>>: y = b + K x or "
                              "y = x - K x, K read once per pass)", "bound": "hbm",
                    "achieved": pb / avg_s / 1e9, "peak": peak, "unit": "GB/s",
                    "frac": pb / avg_s / 1e9 / peak, "peak_kind": peak_kind + " (hbm_gbs, copy)",
                    "algorithmic_bytes_per_launch": pb, "avg_launch_us": avg_s * 1e6, "launches": n_gp,
                    "traffic": traffic_record("cloud_gmres_prod"),
                    "timing": "CUDA events on the scene stream around each Arnoldi step's passes over K, one "
                              "profiled scene, averaged per pass"}
            crn.close()
        except Exception as e:
            cloud = {"error": str(e)[:200]}

    # ---- the three workloads of the method on this GPU in both precisions
    # (host clock around a synchronised scene, median of 5, L2 flushed) and
    # the FP64 oracle on the host cores, one thread and all cores (a child
    # process, bounded by a timeout)
    configs = None
    if rank == 0 and not args.no_cloud and not variant:
        configs = {}
        try:
            for name, mk in (("plain 8x8x8 R1", lambda p: scenes.make_plain().replace(precision=p)),
                             ("plume 64x64x32 R2", lambda p: scenes.make_plume(precision=p)),
                             ("cloud 128x128x40 R2", lambda p: scenes.make_cloud(precision=p))):
                row = {}
                for prec, key in ((T.FP64, "gpu_fp64_ms"), (T.FP32_REFINE, "gpu_fp32_refine_ms")):
                    xrn = T.Runner(mk(0 if prec == T.FP64 else 1), prec, stream=stream)
                    xa, xm = xrn.fields("cuda")
                    xrn.run(xa, xm, rtol=RTOL)
                    xt = []
                    for _ in range(5):
                        flush.zero_()
                        torch.cuda.synchronize()
                        t0 = time.perf_counter()
                        xrn.run(xa, xm, rtol=RTOL)
                        torch.cuda.synchronize()
                        xt.append(time.perf_counter() - t0)
                    row[key] = 1000.0 * statistics.median(xt)
                    row["edges"] = xrn.stats.nnz_edges
                    xrn.close()
                configs[name] = row
        except Exception as e:
            configs["error"] = str(e)[:200]
        if not args.no_cpu_baseline:
            try:
                r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-times"],
                                   capture_output=True, text=True, timeout=600)
                lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
                if lines:
                    ot = json.loads(lines[-1])
                    for name, row in ot.items():
                        if name != "cores" and name in configs:
                            configs[name].update({"oracle_" + k: v for k, v in row.items()})
                    configs["oracle_cores"] = ot.get("cores")
            except subprocess.TimeoutExpired as e:
                configs["oracle_error"] = "oracle timings exceeded 600 s"
                out = e.stdout.decode() if isinstance(e.stdout, bytes) else (e.stdout or "")
                lines = [x for x in out.splitlines() if x.startswith("{")]
                if lines:
                    ot = json.loads(lines[-1])
                    for name, row in ot.items():
                        if name != "cores" and name in configs:
                            configs[name].update({"oracle_" + k: v for k, v in row.items()})

    # ---- serving (continuous batching over resident slots), rank 0 of one GPU
    serve = None
    if rank == 0 and not args.no_serving and not variant:
        try:
            serve = serving(T, scenes, torch, np)
            # the same requests with the Chebyshev refinements of concurrent
            # requests batched into persistent kernels
            bat = serving(T, scenes, torch, np, batch_solves=True, plain=False)
            serve["batched_refinements_on"] = {k: bat[k] for k in (
                "saturation_scenes_per_s", "scenes_per_s", "p50_ms", "p99_ms", "max_ms", "all_converged",
                "arrivals", "per_shape_service", "batched_refinements")}
        except Exception as e:  # the bench line must still print
            serve = {"error": str(e)[:200]}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel: the Chebyshev step of the inner
    # iterations (q = K p over all slots, then r, d, p updated per row)
    peak, peak_kind = peaks()
    n_sp, ms_sp = prof.get("cheb", (0, 0.0))
    kernels = {}
    for name, (n, ms) in prof.items():
        if n:
            kernels[name] = {"launches": n, "avg_us": 1000.0 * ms / n, "share_of_step": ms / prof_ms}
    # the stages of a step (the solve's own kernels lie inside "solve"): what
    # of the sampled steps' time the event profile accounts for
    stage_names = ("set_medium", "assemble_pre", "select", "assemble_rows", "solve", "render")
    stages = {k: prof[k][1] / prof_ms for k in stage_names if k in prof and prof[k][0]}
    stages["accounted"] = sum(stages.values())
    # 4 B per stored value (columns are implicit), per row: p gathered (4),
    # r read + written (8), d read + written (8), new p written (4)
    spmv_bytes = st.nnz * 4 + st.n_nodes * 24
    roof = None
    if n_sp:
        avg_s = ms_sp / n_sp / 1000.0
        ach = spmv_bytes / avg_s / 1e9
        roof = {"kernel": "k_tile<6, OpCheb<float>> (FP32 Chebyshev step: q = K p over the rows of K with p "
                          "gathered from a shared-memory tile, then r, d, p updated per row)", "bound": "hbm",
                "achieved": ach,
                "peak": peak,
                "unit": "GB/s", "frac": ach / peak, "peak_kind": peak_kind + " (hbm_gbs, copy)",
                "traffic": traffic_record("k_tile_OpCheb") if not variant else None,
                "algorithmic_bytes_per_launch": spmv_bytes,
                "avg_launch_us": avg_s * 1e6}
    # ---- the edge form's terms: the contraction (tcgen05, TF32 split in
    # three products) against the TF32 peak, counting the useful FP32 flops
    # 2 n_atm nd nin S; the transport against HBM, counting P' (4 nnz), the
    # planes of G (4 nd N), b and the previous X read and the new X written
    # (12 nin N).  Per working term: terms launched past convergence return
    # at once and are not counted.
    roof_edge = None
    if args.aniso and prof.get("ani_leave", (0, 0.0))[0] and prof_steps:
        nin = st.n_dirs + st.n_gdirs
        n_terms = max(1, len(prof_steps) * (iters[prof_steps[0]][0] - 1))
        t_leave = prof["ani_leave"][1] / n_terms / 1000.0
        t_move = prof["ani_transport"][1] / n_terms / 1000.0
        flops = 2.0 * st.n_atm * st.n_dirs * nin * sc.n_species
        tpk, tpk_kind = tf32_peak()
        mv_bytes = 4 * st.nnz + 4 * st.n_dirs * st.n_nodes + 12 * nin * st.n_nodes
        roof_edge = {
            "contraction": {"kernel": "k_ani_mma (tcgen05 kind::tf32, A and B split in high and low TF32 parts, "
                                      "three products, persistent warp-specialised, TMA-fed)", "bound": "tensor",
                            "achieved": flops / t_leave / 1e12, "peak": tpk, "unit": "TFLOP/s",
                            "frac": flops / t_leave / 1e12 / tpk, "peak_kind": tpk_kind,
                            "algorithmic_flops_per_term": flops, "tensor_flops_issued_per_term": 3 * flops,
                            "avg_term_us": t_leave * 1e6},
            "transport": {"kernel": "k_ani_transport (gather by arrival direction, P' = P Cf, first-order term b)",
                          "bound": "hbm", "achieved": mv_bytes / t_move / 1e9, "peak": peak, "unit": "GB/s",
                          "frac": mv_bytes / t_move / 1e9 / peak, "peak_kind": peak_kind + " (hbm_gbs, copy)",
                          "algorithmic_bytes_per_term": mv_bytes, "avg_term_us": t_move * 1e6},
            "terms_per_solve": iters[prof_steps[0]][0], "residuals_per_solve": iters[prof_steps[0]][1],
            "residual_ms": prof.get("ani_residual", (1, 0.0))[1] / max(1, prof.get("ani_residual", (1, 0.0))[0]),
        }
        if roof is None:
            roof = dict(roof_edge["contraction"])
            roof["traffic"] = None
    # ---- roofline of the assembly (edge march and edge weights, with the
    # per-scene tables): algorithmic bytes per scene = fields read 4 N (2 + S)
    # + values written 4 nnz + s, e1, g^sun 12 N + tau_inf round trip
    # 8 N n_up, over the summed event time of the table stage and the edge
    # kernel
    roof_asm = None
    n_pre, ms_pre = prof.get("assemble_pre", (0, 0.0))
    n_rows, ms_rows = prof.get("assemble_rows", (0, 0.0))
    if n_pre and n_rows:
        asm_bytes = (4 * st.n_nodes * (2 + sc.n_species) + 4 * st.nnz + 12 * st.n_nodes
                     + 8 * st.n_nodes * st.n_up_dirs)
        t_asm = (ms_pre / n_pre + ms_rows / n_rows) / 1000.0
        roof_asm = {"kernel": "assembly: per-scene tables (k_prep, k_segtau_fixed, k_tinf, k_tinfg, k_sunz on three "
                              "streams; the quadrature tables only when the view changed) + edge kernel k_asm0",
                    "bound": "hbm",
                    "achieved": asm_bytes / t_asm / 1e9, "peak": peak, "unit": "GB/s",
                    "frac": asm_bytes / t_asm / 1e9 / peak, "peak_kind": peak_kind + " (hbm_gbs, copy)",
                    "algorithmic_bytes_per_scene": asm_bytes, "us_per_scene": t_asm * 1e6,
                    "edge_kernel_us": ms_rows / n_rows * 1000.0, "tables_us": ms_pre / n_pre * 1000.0,
                    "edges_per_s": st.nnz_edges / t_asm,
                    "traffic": traffic_record("assembly") if not variant else None}
    # ---- accuracy of this run against the FP64 oracle (also the CPU baseline)
    cpu = None
    parity = None
    if not args.no_cpu_baseline and not variant:
        r, t, cores = cpu_baseline(sc)
        got = rn.rad.float().cpu().numpy().astype(np.float64)
        err = np.abs(got - r["rad"]) / np.abs(r["rad"])
        parity = {"max_rel_err_vs_fp64_oracle": float(err.max()), "mean_rel_err": float(err.mean()),
                  "tolerance": 1e-4, "pixels": int(err.size)}
        cpu = {"value": 1.0 / t, "unit": "scenes/s", "cores": cores, "kind": "oracle",
               "sample": "1 full plume scene 64x64x32 (all stages, FP64 C oracle, OpenMP)", "seconds": t}
    it = iters[-1]
    line = {
        "metric": METRIC, "value": value, "unit": "scenes/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if not variant else
                   "%s %dx%dx%d voxels, R=2, coupling selection c_min = %g%s (variant, not the headline)"
                   % (args.workload, nx, ny, nz, args.c_min,
                      ", edge unknowns (arrival direction kept)" if args.aniso else ""),
                   "nnz_edges": st.nnz_edges, "nnz_stored": st.nnz, "nodes": st.n_nodes, "rtol": RTOL,
                   "l2": "flushed between timed steps (256 MB write, outside the timed interval)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "edges_per_s": value * st.nnz_edges,
        "roofline": roof,
        "roofline_assembly": roof_asm,
        "roofline_edge_form": roof_edge,
        "kernels": kernels,
        "stage_shares": stages,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "scenes/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "kernel_timing": "CUDA events on the scene stream, on every %dth timed step (%d steps): around each launch, and around each run of back-to-back Chebyshev steps or power sweeps (average per launch within the run)"
                         % (PROF_EVERY, len(prof_steps)),
        "clocks": clocks,
        "parity": parity,
        "solve": {"iters": it[0], "refinements": it[1], "rho_est": it[2], "rel_resid64": it[3]},
        "adjoint": adj,
        "serving": serve,
        "cloud": cloud,
        "configs": configs,
        "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms), "max": max(step_ms)},
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
