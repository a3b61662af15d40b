"""Benchmark of the particle-decomposition Gamma-SPH-ALE hot path on GB300.

Workload: the Taylor-bar impact (aluminium rod r 5 mm x 40 mm at dx 0.125 mm, 1,607,680 particles,
200 m/s onto a rigid wall, K = 4 random ownership labels, communication hash every step and the swap
heuristic every step). A step is one pass of the whole hot path: bucket hash, radix sort, reorder,
swap pass, communication hash and MGPU boundary set, interaction loop fused with the integration.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line on rank 0. `value` is particle-steps/s of the FP32-split path with the state resident
in HBM, timed with CUDA events on the launch stream; the FP64 path is measured beside it. Under
torchrun every rank runs its own replica (independent problems: weak scaling, no collective on the
data path). `--impl reference` times the plain FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Algorithmic FP operations (+, -, *, /, sqrt) of one ordered pair evaluation: the pair flux (distance,
# normal, kernel gradient, normal velocities and tractions, acoustic Riemann state, interface state, mass,
# momentum and energy fluxes) plus one end's accumulation of its volume, mass, momentum, energy and
# velocity-gradient rates, as counted by running the oracle's pair function on a counting scalar type
# (a CPU test keeps the two equal).
FLOPS_PER_PAIR = 233
LINK_GBPS = 900.0   # modelled inter-GPU link bandwidth per direction (NVLink 5 class), for the overlap report
SMS, FP32_LANES = 152, 128


def algorithmic_bytes_per_particle_step(key_passes: int, K: int, swap_every: int, record_copy: bool = True) -> dict:
    """Compulsory HBM bytes per particle and step of each kernel (state read/written once). With
    record_copy (split path, linear EOS) the integration writes the next step's 48-byte state record and
    the reorder gathers it with the positions, volume and ids instead of the whole FP64 state."""
    state = 15 * 8 + 6          # FP64 fields + material, label, id
    rec = 64                    # FP32 interaction record (position + state)
    gathered = (4 * 8 + 6 + 48) if record_copy else state
    b = {
        "hash": 24 + 8,                                   # x y z in, key + slot out
        "sort": key_passes * (4 + 8 + 8),                 # histogram read + key/slot in and out
        "reorder": 8 + gathered + 24 + 6 + rec,           # key+perm, gathered input, sorted x, ids, records
        "comm": 4 + 1 + 1 + 4 + 4,                        # key, label, flag, comm hash, list entry
        # own record, key/perm, state in, state out (and the next record)
        "interact": rec + 8 + state + 24 + 6 + state + (48 if record_copy else 0),
    }
    if K > 1 and swap_every > 0:
        # the reorder writes the FP32 positions (12 B); the pass reads them and the labels once for the
        # Cg sums, and per label pair the pair's particles (2/K of all) read position, label, material
        # and id and write their balancing hash
        pairs = K * (K - 1) // 2
        b["swap"] = (12 + 12 + 1 + pairs * (2.0 / K) * (12 + 1 + 1 + 4 + 2)) / swap_every
    b["total"] = sum(b.values())
    return b


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def code_sha256(kernel_src: str) -> str:
    """sha256 of a CUDA source's code: comments removed and runs of blank space collapsed, so that an
    edit of the comments alone keeps a profile's counters valid."""
    src = open(kernel_src).read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return hashlib.sha256(" ".join(src.split()).encode()).hexdigest()


def _traffic_from_profile(kernel_src: str, profile: str, kernel: str):
    """dram bytes per launch of `kernel` recorded in a committed ncu summary, if it was taken on this
    source's code."""
    path = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"code_sha256:\s*([0-9a-f]{16,64})", txt)
    t = re.search(r"dram_bytes_per_launch\.%s:\s*([0-9.eE+]+)" % re.escape(kernel), txt)
    if not m or not t:
        return None
    return float(t.group(1)) if code_sha256(kernel_src).startswith(m.group(1)) else None


class ClockSampler:
    """SM clock and clock-event reasons read during the timed region (reads only; nothing is set).
    NVML through ctypes, sampled every 2 ms by a thread, so that a short timed region still has samples;
    the GPU is found by its UUID. Without NVML, nvidia-smi at its shortest period (samples only when
    the region outlasts it). The summary says why it has no samples when it has none."""

    Q = ("uuid,clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    # NVML clock-event reason bits
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40}

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.why = None
        self.proc = self.thread = None
        self.uuid = None
        try:
            import torch
            u = str(torch.cuda.get_device_properties(index).uuid)
            self.uuid = u if u.startswith("GPU-") else "GPU-" + u
        except Exception:
            pass

    def _nvml(self):
        import ctypes as C
        lib = C.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        h = C.c_void_p()
        ok = -1
        if self.uuid:
            ok = lib.nvmlDeviceGetHandleByUUID(self.uuid.encode(), C.byref(h))
        if ok != 0:
            ok = lib.nvmlDeviceGetHandleByIndex_v2(C.c_uint(self.index), C.byref(h))
        if ok != 0:
            raise RuntimeError("no NVML handle for the device")
        reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        return lib, h, reasons

    def start(self):
        import threading
        try:
            import ctypes as C
            lib, h, reasons = self._nvml()
            self.stop_flag = False

            def run():
                clk, mx, rs = C.c_uint(), C.c_uint(), C.c_ulonglong()
                while not self.stop_flag:
                    if (lib.nvmlDeviceGetClockInfo(h, 1, C.byref(clk)) == 0 and
                            lib.nvmlDeviceGetMaxClockInfo(h, 1, C.byref(mx)) == 0 and reasons(h, C.byref(rs)) == 0):
                        self.rows.append((float(clk.value), float(mx.value), int(rs.value)))
                    time.sleep(0.002)

            self.thread = threading.Thread(target=run, daemon=True)
            self.thread.start()
            return
        except Exception as e:   # no NVML: nvidia-smi
            self.why = f"NVML unavailable ({e}); nvidia-smi"
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "20"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception as e:
            self.proc = None
            self.why = f"no clock source: {e}"

    def stop(self):
        if self.thread is not None:
            self.stop_flag = True
            self.thread.join(timeout=2)
        elif self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 7 or (self.uuid and parts[0] != self.uuid):
                    continue
                try:
                    bits = sum(self.BITS[nm] for nm, v in zip(names, parts[3:7]) if v.lower() == "active")
                    self.rows.append((float(parts[1]), float(parts[2]), bits))
                except ValueError:
                    continue
            os.unlink(self.path)
        if not self.rows:
            return {"samples": 0, "reason_no_samples": self.why or "the timed region ended before the first sample"}
        reasons = sorted({nm for _, _, b in self.rows for nm, bit in self.BITS.items() if b & bit})
        out = {"sm_mhz": statistics.median(r[0] for r in self.rows), "sm_max_mhz": max(r[1] for r in self.rows),
               "reasons": reasons, "samples": len(self.rows)}
        if self.why:
            out["source"] = self.why
        return out


def reduce_max(x: float, dist, device=None) -> float:
    """Maximum of x over the ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: float, seconds_max: float) -> float:
    """Whole-job throughput of independent replicas: all ranks' units over the slowest rank's time."""
    return world * units_per_rank / seconds_max


def workload_config(n: int, K: int, swap_period: int, world: int) -> dict:
    return {"workload": "taylor_bar: Al rod r 5 mm x 40 mm, dx 0.125 mm, 200 m/s onto a rigid wall",
            "particles": n, "labels": K, "swap_period": swap_period, "precision": "fp32-split",
            "l2": f"inputs larger than L2 ({n * 600 / 1e6:.0f} MB of state and records resident)",
            "parallelism": f"{world} independent replica(s)"}


def run_reference(args, rank: int):
    """The plain FP64 CPU oracle on the host cores, one bounded sample of the workload per step."""
    from oracle import orc
    from paper_2310_03596_gb300 import scenes

    if rank != 0:
        return None
    full = scenes.taylor_bar()
    # bounded sample: the base of the rod (on the wall) with about 1/10 of the particles per step, so
    # that warmup + steps finish within a few minutes on the host
    frac = min(0.1, 100.0 / (14.0 * max(1, args.steps + args.warmup)) * 1.0)
    zcut = 40e-3 * frac
    keep = full.pos[:, 2] < zcut
    s = scenes.taylor_bar()
    s.pos, s.vel, s.vol = full.pos[keep], full.vel[keep], full.vol[keep]
    s.material, s.label = full.material[keep], full.label[keep]
    P = orc.params_of(s)
    st = orc.OracleState.from_scene(s)
    orc.lib()
    cores = orc.set_threads(os.cpu_count() or 1)
    for k in range(args.warmup):
        orc.step(P, st, do_swap=True)
    t = time.perf_counter()
    pairs = 0
    for k in range(args.steps):
        out = orc.step(P, st, do_swap=True)
        pairs += int(out["nreal"].sum() + out["nimage"].sum())
    el = time.perf_counter() - t
    value = s.n * args.steps / el
    sample = (f"base {zcut * 1e3:.2f} mm of the Taylor bar ({s.n} of {full.n} particles, wall contact "
              f"included), full step incl. swap pass, {args.steps} steps")
    return {"impl": "reference", "metric": "particle-steps/sec", "value": value, "unit": "particle-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(full.n, full.K, full.swap_period, args.gpus),
            "pair_interactions_per_s": pairs / el,
            "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": cores, "kind": "oracle",
                             "sample": sample + f", per-particle loops on {cores} host threads"},
            "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def cpu_baseline(device: int = 0):
    """One full oracle step of the whole workload on the host cores: on one core, and with its
    per-particle loops on every core (OpenMP). The same step on the GPU's FP32-split path from the same
    initial state gives the per-field error of that path against the FP64 oracle."""
    from oracle import orc
    from paper_2310_03596_gb300 import gsph, scenes

    s = scenes.taylor_bar()
    P = orc.params_of(s)
    orc.lib()
    out = {}
    ncores = os.cpu_count() or 1
    st1 = None
    for threads in (1, ncores):
        used = orc.set_threads(threads)
        st = orc.OracleState.from_scene(s)
        t = time.perf_counter()
        orc.step(P, st, do_swap=True)
        el = time.perf_counter() - t
        out[used] = (s.n / el, el)
        st1 = st
    orc.set_threads(1)
    sol = gsph.Solver.from_scene(s, precision=gsph.FP32_SPLIT, device=device)
    sol.step(1)
    sol.sync()
    g = sol.state()
    sol.close()
    og = np.argsort(g["id"])
    oo = np.argsort(st1.id)
    err = {}
    for f in orc.FIELDS:
        a, b = g[f][og], getattr(st1, f)[oo]
        err[f] = float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
    used_max = max(out)
    v1, el1 = out[min(out)]
    vm, elm = out[used_max]
    return ({"value": vm, "unit": "particle-steps/s", "cores": used_max, "kind": "oracle",
             "sample": f"one full step (hash, sort, swap pass, comm hash, interaction, integration) of the "
                       f"{s.n}-particle Taylor bar: {elm:.1f} s with the per-particle loops on {used_max} "
                       f"host threads (nproc {ncores}); {el1:.1f} s on one core",
             "single_core": {"value": v1, "cores": 1, "seconds": el1}},
            {"what": "FP32-split path after one step of the Taylor bar against the FP64 oracle's step from "
                     "the same state: max-norm relative error per field", "max": max(err.values()),
             "per_field": err})


def _at_least_one(v):
    k = int(v)
    if k < 1:
        raise argparse.ArgumentTypeError("must be at least 1")
    return k


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    # the lines without a switch-off (0 skips the collapse block, the plate and the adjoint)
    ap.add_argument("--fp64-steps", type=_at_least_one, default=5)
    ap.add_argument("--overlap-steps", type=_at_least_one, default=20)
    ap.add_argument("--phase-steps", type=_at_least_one, default=100)
    ap.add_argument("--hvi-steps", type=_at_least_one, default=50)
    ap.add_argument("--heun-steps", type=_at_least_one, default=20)
    ap.add_argument("--muscl-steps", type=_at_least_one, default=20)
    ap.add_argument("--varh-steps", type=_at_least_one, default=20)
    ap.add_argument("--collapse-steps", type=int, default=10)
    ap.add_argument("--plate-steps", type=int, default=50)
    ap.add_argument("--adjoint-steps", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        line = run_reference(args, rank)
        if line is not None:
            print(json.dumps(line), flush=True)
        return

    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__

    if rank == 0 or world == 1:
        __graft_entry__.build()
    if dist is not None:
        dist.barrier()
    from paper_2310_03596_gb300 import gsph, scenes

    s = scenes.taylor_bar()
    stream = torch.cuda.current_stream()
    sol = gsph.Solver.from_scene(s, precision=gsph.FP32_SPLIT, device=local, stream=stream)
    n = s.n
    _, ncell = sol.sizes()
    key_passes = (int(ncell).bit_length() + 8) // 9   # radix passes of at most 9 bits

    sol.step(args.warmup, stream)
    sol.sync(stream)
    st0 = sol.exchange_stats(stream)
    # inside the timed region only the three events per step that bound the pair kernel (its duration
    # for the roofline); the per-phase breakdown comes from a separate run that follows
    sol.set_timing(args.steps, pair_only=True)
    clocks = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    if rank == 0:
        clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sol.step(args.steps, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop() if rank == 0 else None
    ms = reduce_max(e0.elapsed_time(e1), dist, device="cuda")
    sol.sync(stream)
    st1 = sol.exchange_stats(stream)
    tm = sol.timings()
    pairs = st1["pairs_total"] - st0["pairs_total"]
    launches = st1["kernel_launches"] - st0["kernel_launches"]
    # the phase breakdown: every phase's events, over the steps that follow the timed region
    sol.set_timing(args.phase_steps)
    sol.step(args.phase_steps, stream)
    sol.sync(stream)
    tph = sol.timings()
    sol.set_timing(0)
    sec = ms * 1e-3
    value = job_rate(world, n * args.steps, sec)
    pair_rate = job_rate(world, pairs, sec)

    # FP64 path on the same workload, fewer steps (its pair math runs on the FP64 units)
    sol64 = gsph.Solver.from_scene(s, precision=gsph.FP64, device=local, stream=stream)
    sol64.step(3, stream)
    sol64.sync(stream)
    p0 = sol64.exchange_stats(stream)["pairs_total"]
    sol64.set_timing(args.fp64_steps)
    torch.cuda.synchronize()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    sol64.step(args.fp64_steps, stream)
    f1.record(stream)
    torch.cuda.synchronize()
    ms64 = f0.elapsed_time(f1)
    p1 = sol64.exchange_stats(stream)["pairs_total"]
    tm64 = sol64.timings()
    sol64.close()

    # Sec. IV's hypervelocity example at full size: Mie-Gruneisen EOS with spall cut-off
    sh = scenes.hvi_bead_plate()
    solh = gsph.Solver.from_scene(sh, device=local, stream=stream)
    solh.step(3, stream)
    solh.sync(stream)
    solh.set_timing(args.hvi_steps)
    torch.cuda.synchronize()
    h0 = torch.cuda.Event(enable_timing=True)
    h1 = torch.cuda.Event(enable_timing=True)
    h0.record(stream)
    solh.step(args.hvi_steps, stream)
    h1.record(stream)
    torch.cuda.synchronize()
    msh = h0.elapsed_time(h1)
    tmh = solh.timings()
    sth = solh.exchange_stats(stream)
    solh.close()
    hvi = {"workload": "hvi_bead_plate: Al bead r 1.5 mm at 4.05 km/s, 32 deg, onto a 2 mm Al plate, "
                       "dx 0.1 mm, Mie-Gruneisen EOS + spall cut-off, K = 4",
           "particles": sh.n, "value": world * sh.n * args.hvi_steps / (msh * 1e-3), "unit": "particle-steps/s",
           "ms_per_step": msh / args.hvi_steps, "steps": args.hvi_steps,
           "phase_ms_per_step": {k[:-3]: v / max(tmh["steps"], 1) for k, v in tmh.items()
                                 if k.endswith("_ms") and v > 0},
           "exchange_fraction": sth["exchange_fraction"]}

    # the second-order variant: two-stage Heun on the same workload
    s2 = scenes.taylor_bar()
    s2.integrator = 1
    solr = gsph.Solver.from_scene(s2, device=local, stream=stream)
    solr.step(3, stream)
    solr.sync(stream)
    solr.set_timing(args.heun_steps)
    torch.cuda.synchronize()
    r0 = torch.cuda.Event(enable_timing=True)
    r1 = torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    solr.step(args.heun_steps, stream)
    r1.record(stream)
    torch.cuda.synchronize()
    msr = r0.elapsed_time(r1)
    tmr = solr.timings()
    solr.close()
    heun = {"what": "two-stage Heun (SSP-RK2) on the Taylor bar: Euler prediction, record refresh, second "
                    "stage over the step-start lists, conserved-variable average",
            "value": world * n * args.heun_steps / (msr * 1e-3), "unit": "particle-steps/s",
            "ms_per_step": msr / args.heun_steps, "steps": args.heun_steps,
            "phase_ms_per_step": {k[:-3]: v / max(tmr["steps"], 1) for k, v in tmr.items()
                                  if k.endswith("_ms") and v > 0}}

    # MUSCL-reconstructed Riemann states on the same workload: gradient pass, reconstructed fluxes
    s3 = scenes.taylor_bar()
    s3.reconstruction = 1
    solm = gsph.Solver.from_scene(s3, device=local, stream=stream)
    solm.step(3, stream)
    solm.sync(stream)
    solm.set_timing(args.muscl_steps)
    torch.cuda.synchronize()
    m0 = torch.cuda.Event(enable_timing=True)
    m1 = torch.cuda.Event(enable_timing=True)
    m0.record(stream)
    solm.step(args.muscl_steps, stream)
    m1.record(stream)
    torch.cuda.synchronize()
    msm = m0.elapsed_time(m1)
    tmm = solm.timings()
    solm.close()
    muscl = {"what": "MUSCL reconstruction on the Taylor bar: SPH gradients of v and sigma (gradient pass), "
                     "minmod-limited midpoint states of both ends for each Riemann problem",
             "value": world * n * args.muscl_steps / (msm * 1e-3), "unit": "particle-steps/s",
             "ms_per_step": msm / args.muscl_steps, "steps": args.muscl_steps,
             "phase_ms_per_step": {k[:-3]: v / max(tmm["steps"], 1) for k, v in tmm.items()
                                   if k.endswith("_ms") and v > 0}}

    # the largest workload: the 64 M-particle collapse block, K = 16, swap pass every 10 steps (step 0
    # and step 10 of the timed window include one), exchange-volume fraction per step
    collapse = None
    if args.collapse_steps > 0 and world == 1:   # one GPU only: 80 GB of state, a minute of setup
        s5 = scenes.collapse_block()
        solc = gsph.Solver.from_scene(s5, device=local, stream=stream)
        solc.step(1, stream)
        solc.sync(stream)
        solc.set_timing(args.collapse_steps)
        torch.cuda.synchronize()
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        solc.step(args.collapse_steps, stream)
        c1.record(stream)
        torch.cuda.synchronize()
        msc = c0.elapsed_time(c1)
        tmc = solc.timings()
        stc = solc.exchange_stats(stream)
        solc.close()
        collapse = {"workload": "collapse_block: Al block 0.4 x 0.2 x 0.1 m at dx 0.5 mm on a floor under gravity, "
                                "K = 16 random labels, swap every 10 steps",
                    "particles": s5.n, "value": world * s5.n * args.collapse_steps / (msc * 1e-3),
                    "unit": "particle-steps/s", "ms_per_step": msc / args.collapse_steps,
                    "steps": args.collapse_steps,
                    "phase_ms_per_step": {k[:-3]: v / max(tmc["steps"], 1) for k, v in tmc.items()
                                          if k.endswith("_ms") and v > 0},
                    "exchange_fraction": stc["exchange_fraction"], "swap_passes": stc["swap_passes"]}

    # the projectile-on-plate workload: steel sphere into an aluminium plate, two materials, K = 8 x-slab
    # labels with per-type swaps (Sec. III.B) at the scene's period
    plate = None
    if args.plate_steps > 0:
        s6 = scenes.projectile_plate()
        solp = gsph.Solver.from_scene(s6, device=local, stream=stream)
        solp.step(3, stream)
        solp.sync(stream)
        solp.set_timing(args.plate_steps)
        torch.cuda.synchronize()
        pe0 = torch.cuda.Event(enable_timing=True)
        pe1 = torch.cuda.Event(enable_timing=True)
        pe0.record(stream)
        solp.step(args.plate_steps, stream)
        pe1.record(stream)
        torch.cuda.synchronize()
        msp = pe0.elapsed_time(pe1)
        tmp = solp.timings()
        stp = solp.exchange_stats(stream)
        solp.close()
        plate = {"workload": "projectile_plate: steel sphere r 5 mm at 1000 m/s onto an Al plate 60 x 60 x 10 mm, "
                             "dx 0.2 mm, two materials, K = 8 x-slab labels, per-type swaps every "
                             f"{s6.swap_period} steps",
                 "particles": s6.n, "value": world * s6.n * args.plate_steps / (msp * 1e-3),
                 "unit": "particle-steps/s", "ms_per_step": msp / args.plate_steps, "steps": args.plate_steps,
                 "phase_ms_per_step": {k[:-3]: v / max(tmp["steps"], 1) for k, v in tmp.items()
                                       if k.endswith("_ms") and v > 0},
                 "exchange_fraction": stp["exchange_fraction"], "swap_passes": stp["swap_passes"]}

    # the adjoint workload: gradient of the rear-face mean z velocity of the 64^3 cube w.r.t. (Y, G, v0),
    # FP32-split forward of 200 steps with a checkpoint every 20, recompute and FP64 reverse sweep, all in
    # one gsph_adjoint call
    adj = None
    if args.adjoint_steps > 0:
        from paper_2310_03596_gb300 import adjoint as adjm
        sa = scenes.adjoint_cube()
        ids = adjm.rear_face_ids(sa)
        sola = gsph.Solver.from_scene(sa, device=local, stream=stream)
        torch.cuda.synchronize()
        t = time.perf_counter()
        Jf, _, dts = sola.adjoint(args.adjoint_steps, 20, ids, want_gradient=False, stream=stream)
        torch.cuda.synchronize()
        tf = time.perf_counter() - t
        sola.close()
        sola = gsph.Solver.from_scene(sa, device=local, stream=stream)
        torch.cuda.synchronize()
        t = time.perf_counter()
        Ja, ga, _ = sola.adjoint(args.adjoint_steps, 20, ids, stream=stream)
        torch.cuda.synchronize()
        ta = time.perf_counter() - t
        sola.close()
        adj = {"workload": "adjoint_cube: Al cube 64^3 at dx 1 mm, 100 m/s onto a wall; J = rear-face mean v_z",
               "particles": sa.n, "steps": args.adjoint_steps, "checkpoint_every": 20,
               "forward_only_ms_per_step": 1e3 * tf / args.adjoint_steps,
               "forward_and_reverse_ms_per_step": 1e3 * ta / args.adjoint_steps,
               "what": "one gsph_adjoint call: split forward with device checkpoints, segment recompute, FP64 "
                       "reverse steps, dJ/d(Y, G, v0); wall time of the call (host-driven, synchronous)",
               "J": Ja, "grad": list(ga)}

    # per-particle smoothing lengths (Sec. V's varying particle sizes): the rod with a fine impact end,
    # and the cost function per label there
    s4 = scenes.graded_bar()
    solv = gsph.Solver.from_scene(s4, device=local, stream=stream)
    solv.step(3, stream)
    solv.sync(stream)
    solv.set_timing(args.varh_steps)
    torch.cuda.synchronize()
    v0 = torch.cuda.Event(enable_timing=True)
    v1 = torch.cuda.Event(enable_timing=True)
    v0.record(stream)
    solv.step(args.varh_steps, stream)
    v1.record(stream)
    torch.cuda.synchronize()
    msv = v0.elapsed_time(v1)
    tmv = solv.timings()
    stv = solv.exchange_stats()
    solv.close()
    varh = {"workload": "graded_bar: the Taylor bar with spacing 0.125 mm over its 10 mm impact end and 0.25 mm "
                        "over the rest, h_i = 1.3 x spacing, K = 4 random labels",
            "particles": s4.n, "value": world * s4.n * args.varh_steps / (msv * 1e-3), "unit": "particle-steps/s",
            "ms_per_step": msv / args.varh_steps, "steps": args.varh_steps,
            "phase_ms_per_step": {k[:-3]: v / max(tmv["steps"], 1) for k, v in tmv.items()
                                  if k.endswith("_ms") and v > 0},
            "cost_per_label": stv["cost"], "cost_imbalance": stv["cost_imbalance"],
            "pairs_per_particle": float(sum(stv["cost"])) / s4.n}

    # the interaction in the order of Sec. II steps d-f (two passes, halo gather on a second stream)
    solo = gsph.Solver.from_scene(s, device=local, stream=stream, overlap=True)
    solo.step(3, stream)
    solo.sync(stream)
    solo.set_timing(args.overlap_steps)
    solo.step(args.overlap_steps, stream)
    solo.sync(stream)
    tmo = solo.timings()
    sto = solo.exchange_stats(stream)
    solo.close()
    ko = max(tmo["steps"], 1)
    recv = sto["boundary_total"] * (s.K - 1) / s.K * sto["record_bytes"]   # bytes one GPU receives per step
    link_ms = recv / (LINK_GBPS * 1e9) * 1e3
    overlap = {
        "what": "Sec. II steps d-f on one device: pairs within a label while the MGPU boundary set is gathered "
                "into a halo buffer on a second (high-priority) stream, then the boundary particles' pairs "
                "across labels from the halo",
        "local_ms": tmo["local_ms"] / ko, "boundary_ms": tmo["boundary_ms"] / ko,
        "halo_gather_ms": tmo["halo_ms"] / ko,
        "pair_two_pass_ms": tmo["pair_ms"] / ko, "pair_one_pass_ms": tph["pair_ms"] / max(tph["steps"], 1),
        "boundary_total": sto["boundary_total"], "boundary_bytes_received_per_gpu": recv,
        "link_model": f"{LINK_GBPS:.0f} GB/s per direction per GPU (NVLink 5 class)",
        "link_ms_model": link_ms,
        "hidden_fraction_model": min(1.0, (tmo["local_ms"] / ko) / link_ms) if link_ms > 0 else 1.0,
        "steps": args.overlap_steps,
    }

    # end to end through the public API with host buffers: upload the particle set from pinned host
    # memory, run the steps, read the whole state back
    pin = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory()
           for k, v in (("pos", s.pos), ("vel", s.vel), ("vol", s.vol), ("mat", s.material), ("lab", s.label))}
    out_host = torch.empty((15, n), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t = time.perf_counter()
    sol.set_particles(pin["pos"].numpy(), pin["vel"].numpy(), pin["vol"].numpy(), pin["mat"].numpy(),
                      pin["lab"].numpy(), stream=stream)
    sol.step(args.steps, stream)
    outs = out_host.numpy()
    for k, f in enumerate(gsph.FIELDS[:15]):
        sol.get(f, stream, out=outs[k])
    torch.cuda.synchronize()
    e2e_s = reduce_max(time.perf_counter() - t, dist, device="cuda")
    h2d = n * (24 + 24 + 8 + 1 + 1)
    d2h = n * 15 * 8

    if rank != 0:
        sol.close()
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return

    peaks, peaks_kind = _peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = SMS * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12
    kph = max(tph["steps"], 1)
    it_ms = tph["interact_ms"] / kph
    pk_ms = tm["pair_ms"] / max(tm["steps"], 1)   # the timed region's own pair-kernel events
    nl_ms = tph["nbr_list_ms"] / kph
    flops_per_launch = FLOPS_PER_PAIR * pairs / args.steps
    achieved = flops_per_launch / (pk_ms * 1e-3) / 1e12
    traffic = _traffic_from_profile(os.path.join(ROOT, "paper_2310_03596_gb300", "csrc", "k_interact.cu"),
                                    "k_interact_taylor_bar_split.md", "k_pair")
    ab = algorithmic_bytes_per_particle_step(key_passes, s.K, s.swap_period)
    step_ms = ms / args.steps
    hbm_ach = ab["total"] * n / (step_ms * 1e-3) / 1e9
    line = {
        "metric": "particle-steps/sec",
        "value": value,
        "unit": "particle-steps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": step_ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": workload_config(n, s.K, s.swap_period, world),
        "pair_interactions_per_s": pair_rate,
        "pairs_per_step": pairs / args.steps,
        "phase_ms_per_step": {k[:-3]: v / kph for k, v in tph.items() if k.endswith("_ms")},
        "phase_steps": tph["steps"],
        "fp64": {"value": world * n * args.fp64_steps / (ms64 * 1e-3), "unit": "particle-steps/s",
                 "ms_per_step": ms64 / args.fp64_steps,
                 "pair_interactions_per_s": world * (p1 - p0) / (ms64 * 1e-3),
                 "interact_ms": tm64["interact_ms"] / max(tm64["steps"], 1), "steps": args.fp64_steps},
        "roofline": {"kernel": "k_pair<split>: pair fluxes, per-particle sums, integration (one launch per step)",
                     "bound": "alu", "achieved": achieved, "peak": fp32_peak,
                     "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": traffic,
                     "flops_per_launch": flops_per_launch, "launch_ms": pk_ms,
                     "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz (sm_max_mhz, {peaks_kind})",
                     "interaction_phase": {"nbr_list_ms": nl_ms, "pair_ms": tph["pair_ms"] / kph,
                                           "interact_ms": it_ms,
                                           "achieved_over_phase": flops_per_launch / (it_ms * 1e-3) / 1e12}},
        "hbm_step": {"bytes_per_particle_step": ab, "achieved_GBps": hbm_ach, "peak_GBps": peaks["hbm_gbs"],
                     "frac": hbm_ach / peaks["hbm_gbs"], "peak_source": f"hbm_gbs ({peaks_kind})"},
        "e2e": {"value": world * n * args.steps / e2e_s, "unit": "particle-steps/s",
                "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                "what": "upload of the particle set from pinned host memory, the steps, read-back of the "
                        "15 state fields, through the public API"},
        "gpu_launches": launches,
        "overlap": overlap,
        "hvi": hvi,
        "heun": heun,
        "muscl": muscl,
        "varh": varh,
        "collapse": collapse,
        "projectile_plate": plate,
        "adjoint": adj,
        "clocks": ck,
        "exchange": {k: st1[k] for k in ("boundary_total", "exchange_fraction", "bytes_boundary_broadcast",
                                         "swapped_last_pass", "swap_passes", "dt_candidates",
                                         "dt_fp64_evaluations", "swap_fp64_hashes")},
    }
    sol.close()
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"], line["split_path_error"] = cpu_baseline(local)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
