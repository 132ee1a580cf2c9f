#!/usr/bin/env python
"""Throughput benchmark of the full fractional-step MRT-LBE update.

One bench step = one lattice time step over the whole grid: fields and
forces, collision and streaming of both population sets, the three RK3
finite-difference stages, the Picard sweeps of the implicit velocity and the
selective filter.  Workload: the capillary-wave setup (flat interface with a
cosine perturbation of amplitude 0.01 L, density ratio 1000, periodic in x,
no-slip walls in y) on a 4096 x 4096 grid in FP32, synthetic initial fields.
Metric: MLUPS = nodes x steps / seconds / 1e6.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch one process per GPU with torch.distributed.run; every rank
advances its own replica (the method has no cross-replica exchange), the time
is the maximum over ranks and the value counts the nodes of all ranks.
"""
import argparse
import hashlib
import json
import os
import platform
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLUPS (both lattices+FD+filter) FP32 vs mixed, % HBM roofline; adjoint/forward time"
UNIT = "MLUPS"
KERNEL_SRC = os.path.join(ROOT, "paper_1812_02459_gb300", "csrc", "lbm_kernels.cuh")
PROFILES = os.path.join(ROOT, "profiles")

# Algorithmic words (4 bytes in FP32, 8 in FP64) per node and launch of each
# kernel: every persistent plane it needs read once and written once; what
# stays on chip is not counted.  FP32 handles carry phi as phi_hi + phi_lo.
#   collide+stream: read 18 populations + phi, phi_lo, p, u(2), u_prev(2),
#                   u_hat(2); write 18 populations + dbar, p_hat, j(2) -> 49
#     k_collide_pairs (default rates) does not need the rest populations
#     f_0, g_0, whose rate-1 relaxation discards them: reads 16       -> 47
#   RK3 stages over a step: (phi, dbar) -> d1; (phi, d1, dbar) -> d2;
#     (phi, d2, dbar) -> phi^{n+1}, phi_lo: 3 + 4 + 5 words          -> 4 per launch
#   Picard sweep: read phi, p_hat, j(2), u^k(2); write u^{k+1}(2)     -> 8
#   filter: read p_hat, u_hat(2); write p, u(2)                       -> 6
KIND_WORDS = {"k_collide_stream": 49.0, "k_rk_stage": 4.0, "k_picard": 8.0, "k_filter": 6.0}
VARIANT_WORDS = {"k_collide_pairs": 47.0}
# Mixed-precision storage: the 34 population words of k_collide_pairs take 2
# bytes; its 13 scalar words and the other kernels' words stay FP32.
MIXED_COLLIDE_BYTES = 34 * 2 + 13 * 4
# The least a step must move (all intermediates on chip): populations read and
# written once, phi, u^n, u^{n-1} read and phi, u^{n+1} written (8 words).
B_MIN = {"fp32": 18 * 2 * 4 + 8 * 4, "mixed": 18 * 2 * 2 + 8 * 4}


def algo_words(kind, variant):
    return VARIANT_WORDS.get(variant, KIND_WORDS[kind])


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--n", type=int, default=4096, help="grid is n x n")
    ap.add_argument("--adjoint-n", type=int, default=256, help="side of the adjoint side measurement's grid")
    ap.add_argument("--adjoint-steps", type=int, default=200, help="steps of the adjoint side measurement")
    ap.add_argument("--adjoint-sweep", type=int, nargs="*", default=[512, 1024, 2048, 4096],
                    help="grid sides of the adjoint/forward time sweep on the capillary wave")
    ap.add_argument("--precision", default="fp32", choices=("fp32", "fp64"))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the reduced-precision and adjoint side measurements")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# multi-process plumbing (replicas; used for the barrier and max-over-ranks)
# ---------------------------------------------------------------------------
def dist_init(backend="nccl"):
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and not dist.is_initialized():
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(value, world, device=None):
    """Maximum of a float over all ranks (identity for one rank)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_mlups(nodes_per_rank, steps, max_seconds, world):
    """Whole-job throughput: nodes of all replicas x steps / slowest rank's time."""
    return world * nodes_per_rank * steps / max_seconds / 1e6


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi sampled every 200 ms; only samples inside [t0, t1] are kept."""
    QUERY = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id=None):
        self.proc = None
        self.path = None
        self.gpu_id = gpu_id
        self.t0 = self.t1 = None

    def start(self, wait_s=15.0):
        """Start sampling and wait until the first sample arrives (NVML is up)."""
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.gpu_id:
                cmd += ["-i", self.gpu_id]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t_end = time.time() + wait_s
        while time.time() < t_end and os.path.getsize(self.path) == 0 and self.proc.poll() is None:
            time.sleep(0.05)

    def mark(self, which):
        setattr(self, which, time.time())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        import datetime
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                continue
            rows.append((ts, parts))
        os.unlink(self.path)
        inside = [r for ts, r in rows if self.t0 is not None and self.t0 - 0.2 <= ts <= self.t1 + 0.2]
        use = inside if inside else [r for _, r in rows]
        if not use:
            return None
        num = lambda v: float(v) if v.replace(".", "").isdigit() else None
        sm = [num(r[1]) for r in use if num(r[1]) is not None]
        mx = [num(r[2]) for r in use if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in use for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(use), "samples_in_timed_region": len(inside)}


def gpu_uuid(device):
    try:
        import torch
        u = torch.cuda.get_device_properties(device).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        return None


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash():
    return hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()[:16]


def recorded_traffic_per_node(precision, kernel):
    """DRAM bytes per node of a kernel from its committed ncu summary on the
    capillary-wave workload, if taken on the current kernel source; else None."""
    try:
        txt = open(os.path.join(PROFILES, "%s_capillary_wave.md" % kernel)).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_node_%s:\s*([0-9.]+)\s+kernel_source_sha256_16:\s*([0-9a-f]+)" % precision, txt)
    if not m or m.group(2) != kernel_source_hash():
        return None
    return float(m.group(1))


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        m = re.search(r"Model name:\s*(.+)", out)
        if m:
            return m.group(1).strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def oracle_mlups(n, steps, warmup=1):
    """The FP64 oracle, single-threaded, on an n x n capillary wave."""
    import oracle
    from paper_1812_02459_gb300 import inputs
    prm, fields = inputs.capillary_wave(n=n)
    s = oracle.Sim(prm, *fields)
    if warmup:
        s.step(warmup)
    t0 = time.perf_counter()
    s.step(steps)
    dt = time.perf_counter() - t0
    s.close()
    return n * n * steps / dt / 1e6, dt


def _oracle_worker(job):
    n, steps = job
    v, dt = oracle_mlups(n, steps)
    return n * n * steps, dt


def oracle_mlups_all_cores(n, steps):
    """The same oracle in one process per host core, each on its own copy of
    the sample (processes started by spawn, so none inherits a CUDA context):
    node updates of all processes over the wall time of the slowest."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_worker, [(64, 1)] * cores)   # workers up, oracle loaded
        t0 = time.perf_counter()
        res = pool.map(_oracle_worker, [(n, steps)] * cores)
        wall = time.perf_counter() - t0
    return sum(r[0] for r in res) / wall / 1e6, wall, cores


# ---------------------------------------------------------------------------
# reference arm: the oracle as it stands, on the host cores
# ---------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_1812_02459_gb300 import inputs
    n = 256
    prm, fields = inputs.capillary_wave(n=n)
    s = oracle.Sim(prm, *fields)
    s.step(args.warmup)
    t0 = time.perf_counter()
    s.step(args.steps)
    dt = time.perf_counter() - t0
    v = n * n * args.steps / dt / 1e6
    sample = (f"capillary wave {n}x{n} (same parameters as the 4096^2 workload), one oracle step "
              f"per bench step, FP64, single thread on {cpu_model()} ({os.cpu_count()} cores on the host)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"capillary wave {n}x{n} sample of the 4096x4096 workload, rho ratio 1000",
                   "nx": n, "ny": n, "precision": "fp64"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    from paper_1812_02459_gb300 import inputs, lbm

    rank, world, local = dist_init("nccl")
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.n
    prm, fields = inputs.capillary_wave(n=n)
    stream = torch.cuda.current_stream(dev)
    sim = lbm.Sim(prm, *fields, precision=args.precision, stream=stream.cuda_stream)
    N = n * n
    elem = 8 if args.precision == "fp64" else 4
    state_bytes = sim.device_bytes()

    clocks = ClockSampler(gpu_uuid(local))
    clocks.start()
    sim.step(args.warmup)
    torch.cuda.synchronize(dev)

    sim.profile(True)
    barrier(world)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks.mark("t0")
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clocks.mark("t1")
    barrier(world)
    clk = clocks.stop()
    prof = sim.profile_read()
    sim.profile(False)
    ms_total = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms_total, world, dev)
    value = aggregate_mlups(N, args.steps, ms_max / 1e3, world)

    # roofline of the dominant kernel, timed live over the same region
    peak, peak_kind = measured_peaks()
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms, dom_n = prof[dom]
    variants = sim.kernel_variants()
    algo_bytes = algo_words(dom, variants[dom]) * elem * N
    achieved = algo_bytes / (dom_ms / dom_n / 1e3) / 1e9
    tpn = recorded_traffic_per_node(args.precision, variants[dom])
    roofline = {"bound": "hbm", "kernel": variants[dom], "kind": dom, "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": None if tpn is None else round(tpn * N),
                "algorithmic_bytes_per_launch": int(algo_bytes), "peak_source": peak_kind}
    step_words = sum(algo_words(k, variants[k]) * v[1] for k, v in prof.items()) / args.steps
    step_bytes = step_words * elem * N
    kernels = {k: {"kernel": variants[k], "ms_per_launch": round(v[0] / max(v[1], 1), 4), "launches": v[1],
                   "share": round(v[0] / max(sum(x[0] for x in prof.values()), 1e-12), 4)}
               for k, v in prof.items()}
    gpu_launches = sum(v[1] for v in prof.values())

    # end to end through the C ABI with host buffers: upload the initial
    # fields from pinned memory, step, read the diagnostics every step, read
    # the fields back at the end
    e2e = None
    if not args.no_e2e:
        pinned = [torch.empty((n, n), dtype=torch.float64, pin_memory=True) for _ in range(4)]
        for t, a in zip(pinned, fields):
            t.numpy()[...] = a
        outs = [torch.empty((n, n), dtype=torch.float64, pin_memory=True) for _ in range(4)]
        # every step's sums are read back on the host; the read of step i waits
        # for its own copy while step i + 1 is already queued (two page-locked
        # buffers, an event after each copy)
        hd = [torch.empty(lbm.LBM_NDIAG, dtype=torch.float64, pin_memory=True).numpy() for _ in range(2)]
        evs = [torch.cuda.Event() for _ in range(2)]
        hp = [t.numpy() for t in pinned]
        ho = [t.numpy() for t in outs]
        sums = []
        torch.cuda.synchronize(dev)
        barrier(world)
        t0 = time.perf_counter()
        sim.set_fields(*hp)
        for i in range(args.steps):
            sim.step(1)
            sim.diagnostics_async(hd[i % 2])
            evs[i % 2].record(stream)
            if i > 0:
                evs[(i - 1) % 2].synchronize()
                sums.append(float(hd[(i - 1) % 2][0]))
        evs[(args.steps - 1) % 2].synchronize()
        sums.append(float(hd[(args.steps - 1) % 2][0]))
        ph, p_, ux_, uy_ = sim.fields(out=ho)
        t1 = time.perf_counter()
        barrier(world)
        del ph, p_, ux_, uy_, ho
        e2e_s = max_over_ranks(t1 - t0, world, dev)
        e2e = {"value": round(aggregate_mlups(N, args.steps, e2e_s, world), 1), "unit": UNIT,
               "h2d_bytes_per_step": round(4 * 8 * N / args.steps),
               "d2h_bytes_per_step": round(lbm.LBM_NDIAG * 8 + 4 * 8 * N / args.steps),
               "readback": "every step's FP64 sums (lbm_diagnostics_async) read on the host while the next "
                           "step runs; fields uploaded before and downloaded after the steps",
               "sum_phi_first_last": [sums[0], sums[-1]]}

    # side measurements: the same workload with reduced-precision population
    # storage, and the adjoint/forward time ratio on the adjoint workload
    variants = None
    if not args.no_variants:
        variants = {}
        for prec in ("mix_bf16", "mix_fp16"):
            v = lbm.Sim(prm, *fields, precision=prec, stream=stream.cuda_stream)
            v.step(max(3, args.warmup // 2))
            torch.cuda.synchronize(dev)
            k = max(10, args.steps // 2)
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            v.profile(True)
            a0.record(stream)
            v.step(k)
            a1.record(stream)
            torch.cuda.synchronize(dev)
            vprof = v.profile_read()
            v.profile(False)
            vvar = v.kernel_variants()
            ms_v = a0.elapsed_time(a1) / k
            mixed_bytes = MIXED_COLLIDE_BYTES + 4 * sum(algo_words(kk, vvar[kk]) * x[1] for kk, x in vprof.items()
                                                        if kk != "k_collide_stream") / k
            variants[prec] = {"MLUPS": round(N / ms_v / 1e3, 1), "ms_per_step": round(ms_v, 4), "steps": k,
                              "vs_fp32": round((N / ms_v / 1e3) / (N / (ms_max / args.steps) / 1e3), 4),
                              "step_roofline": {"algorithmic_bytes_per_node": mixed_bytes,
                                                "frac": round(mixed_bytes * N / (ms_v / 1e3) / 1e9 / peak, 4),
                                                "b_min_bytes_per_node": B_MIN["mixed"],
                                                "b_min_frac": round(B_MIN["mixed"] * N / (ms_v / 1e3) / 1e9 / peak, 4)},
                              "kernels": {kk: {"kernel": vvar[kk], "ms_per_launch": round(x[0] / max(x[1], 1), 4)}
                                          for kk, x in vprof.items()}}
            v.close()
        an, asteps, aevery = args.adjoint_n, args.adjoint_steps, 22

        def adjoint_run(aprm, afields, nsteps):
            a = lbm.Sim(aprm, *afields, precision="fp32", stream=stream.cuda_stream)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            a.adjoint_begin(nsteps, aevery)
            t1 = time.perf_counter()
            phiT = a.fields()[0]
            a.adjoint_end(phiT - afields[0])
            t2 = time.perf_counter()
            eng = a.adjoint_engine()
            a.close()
            return t1 - t0, t2 - t1, eng
        engines = {1: "compiled level kernels", 0: "tape interpreter"}
        aprm, afields = inputs.translating_drop(n=an, R=an / 8.0, U0=0.01)
        # the first reverse sweep of a tape structure compiles its level
        # kernels (once per process): a short untimed run does that
        _, c_rev, _ = adjoint_run(aprm, afields, 2)
        fw, rv, eng = adjoint_run(aprm, afields, asteps)
        os.environ["LBM_ADJOINT_COMPILED"] = "0"
        try:
            fwi, rvi, engi = adjoint_run(aprm, afields, asteps)
        finally:
            del os.environ["LBM_ADJOINT_COMPILED"]
        variants["adjoint"] = {"workload": f"translating drop {an}x{an}, rho ratio 100, {asteps} steps, "
                                           f"checkpoint every {aevery}, FP32 forward and reverse sweep",
                               "engine": engines.get(eng, "none"),
                               "forward_s": round(fw, 4), "reverse_s": round(rv, 4),
                               "adjoint_over_forward": round(rv / fw, 2),
                               "first_sweep_with_compile_s": round(c_rev, 3),
                               "interpreter": {"engine": engines.get(engi),
                                               "reverse_s": round(rvi, 4), "adjoint_over_forward": round(rvi / fwi, 2)}}
        # the reverse/forward ratio per grid on the capillary wave (walls in
        # y, density ratio 1000), 44 steps in two checkpoint segments
        sweep = []
        for gn in args.adjoint_sweep:
            cprm, cfields = inputs.capillary_wave(n=gn)
            if not sweep:
                adjoint_run(cprm, cfields, 2)   # compiles the walled tape's kernels
            cfw, crv, ceng = adjoint_run(cprm, cfields, 44)
            sweep.append({"n": gn, "forward_s": round(cfw, 4), "reverse_s": round(crv, 4),
                          "adjoint_over_forward": round(crv / cfw, 2), "engine": engines.get(ceng, "none"),
                          # node updates per second of the reverse sweep, and of forward + reverse
                          "reverse_MLUPS": round(gn * gn * 44 / crv / 1e6, 1),
                          "gradient_MLUPS": round(gn * gn * 44 / (cfw + crv) / 1e6, 1)})
        variants["adjoint_sweep"] = {"workload": "capillary wave n x n, walls in y, rho ratio 1000, 44 steps, "
                                                 f"checkpoint every {aevery}, FP32 forward and reverse sweep",
                                     "grids": sweep}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cn, cs = 512, 20
        v, dt = oracle_mlups(cn, cs)
        cpu = {"value": round(v, 3), "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
               "sample": f"capillary wave {cn}x{cn}, same parameters, {cs} steps ({dt:.1f} s), FP64 oracle, "
                         f"single thread on {cpu_model()} ({os.cpu_count()} cores on the host)"}
        va, wall, ncores = oracle_mlups_all_cores(cn, cs)
        cpu["all_cores"] = {"value": round(va, 3), "unit": UNIT, "cores": ncores, "kind": "oracle",
                            "sample": f"the same sample in {ncores} processes at once, one per core "
                                      f"({wall:.1f} s wall): throughput of the whole host, not a parallel oracle"}

    diag = sim.diagnostics()
    ok = diag[10] == 0
    sim.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32", "data": "synthetic",
            "config": {"workload": f"capillary wave {n}x{n}: periodic x, no-slip walls y, rho ratio 1000, "
                                   f"nu 1/30, sigma 0.02, W 4, M 0.05, SF-11 a 0.5, 2 Picard sweeps",
                       "nx": n, "ny": n, "precision": args.precision,
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": f"inputs larger than L2: {state_bytes / 1e9:.2f} GB state, "
                             f"{step_bytes / 1e9:.2f} GB algorithmic traffic per step"},
            "roofline": roofline,
            "step_roofline": {"algorithmic_bytes_per_node": step_bytes / N,
                              "achieved_GBps": round(step_bytes / (ms_max / args.steps / 1e3) / 1e9, 1),
                              "frac": round(step_bytes / (ms_max / args.steps / 1e3) / 1e9 / peak, 4),
                              "b_min_bytes_per_node": B_MIN["fp32"] * elem // 4,
                              "b_min_frac": round(B_MIN["fp32"] * elem // 4 * N / (ms_max / args.steps / 1e3) / 1e9
                                                  / peak, 4)},
            "kernels": kernels,
            "variants": variants,
            "gpu_launches": gpu_launches,
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "finite": bool(ok),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
