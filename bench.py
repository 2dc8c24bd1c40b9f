#!/usr/bin/env python
"""Benchmark of the Galerkin ROM hot path on GB300.

Workload (seeded, synthetic; stands in for the paper's 2D/3D LDC and MFU
operators, which are not available): N = 1024 modes, the CP-structured skew
advection tensor C_ijk = sum_r V_jr (U_ir W_kr - W_ir U_kr) + skew residual at
1e-3 relative norm with R = N, A = diag((i/N)^2), B = I, nu = 1e-2,
dt = 1e-3, initial state u_i ~ N(0,1)/i.

One bench step is one BDF3/EXT3 step (advection term, extrapolation, cached
reduced solve, energy/invariant, history rotation) of one trajectory of the
headline model: the full G-ROM at FP64 tolerance.  Its tensor is stored as
F32X2 (hi = rn32(C), lo = rn32(C - hi): a 48-bit significand in 8 bytes) in
the skew-packed layout (one entry of each pair C_ijk = -C_kji; the same model
as the dense tensor), contracted in double-single FP32 arithmetic (error-free
products and sums) with an FP64 state update; its per-evaluation error
against the FP64 oracle is bounded by 1e-12 and printed in the line.  The
same step is also timed for the other storage types (BF16, FP32, FP64), for
the dense layout and for the CPD-ROM (skew CP factors, rank N) and reported
under "variants"; each result carries its error against the FP64 oracle.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

With --impl reference the FP64 CPU oracle is timed on the host cores for the
same metric and workload.  Under torchrun every rank runs an independent
replica (the path shards by trajectory and needs no collective).
"""
import argparse
import hashlib
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

METRIC = "ROM steps/s at N=1024 (full vs CPD, FP64 vs BF16), HBM/TC roofline %, p99 latency"
UNIT = "steps/s"
NU, DT = 1e-2, 1e-3
HEADLINE_FORM = "full"  # storage and layout: --storage (F32X2) and --layout (skew-packed)
VARIANTS = [("full", "bf16", "skew_packed"), ("full", "f32", "skew_packed"), ("full", "f32x2", "skew_packed"),
            ("full", "f64", "skew_packed"), ("full", "bf16", "dense"), ("full", "f32", "dense"),
            ("full", "f32x2", "dense"), ("full", "f64", "dense"), ("cp_skew", "bf16", "dense"),
            ("cp_skew", "f32", "dense"), ("cp_skew", "f64", "dense")]
TOL = {"f64": 1e-12, "f32x2": 1e-12, "f32": 1e-5, "bf16": 2e-2}
STORAGE_BYTES = {"f64": 8, "f32x2": 8, "f32": 4, "bf16": 2}
L2_BYTES = 129 * 2 ** 20


def parse_args():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="grom", choices=["grom", "reference"])
    p.add_argument("--n", type=int, default=1024)
    p.add_argument("--rank", type=int, default=0, help="CP rank (default N)")
    p.add_argument("--variants", default="all", help="'all', 'none' or comma list like full:f64:skew_packed,cp_skew:bf16,aug (layout defaults to dense; aug = the model with the zeroth mode)")
    p.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the oracle CPU baseline")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--batches", default="16,64,256,1024", help="batched-trajectory sizes ('none' to skip)")
    p.add_argument("--serve-requests", type=int, default=10000, help="serving-mix requests (0 to skip)")
    p.add_argument("--serve-rate", type=float, default=2000.0)
    p.add_argument("--serve-slots", type=int, default=64)
    p.add_argument("--serve-quantum", type=int, default=16, help="steps a pool runs between scheduling decisions")
    p.add_argument("--json-out", default="")
    p.add_argument("--svd-ranks", default="64,256", help="SVD-ROM variant ranks ('none' to skip)")
    p.add_argument("--als-ranks", default="128,512", help="CP fitting (ALS, ALS-skew) ranks ('none' to skip)")
    p.add_argument("--als-iters", type=int, default=5)
    p.add_argument("--als-ridge", type=float, default=1e-5, help="relative ridge of the ALS normal equations")
    p.add_argument("--layout", default="skew_packed", choices=["skew_packed", "dense"],
                   help="stored layout of the headline tensor")
    p.add_argument("--storage", default="f32x2", choices=["f32x2", "f64", "f32", "bf16"],
                   help="storage of the headline tensor (f32x2: FP64 tolerance on the FP32 pipe)")
    p.add_argument("--autotune", action="store_true",
                   help="batched section: also autotune each BF16 batched ROM (grom_autotune) and re-time it")
    return p.parse_args()


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        # wait until nvidia-smi is polling (its start-up must not fall inside
        # the timed region)
        t0 = time.time()
        while self.proc is not None and time.time() - t0 < 10.0:
            with open(self.path) as fh:
                if fh.readline():
                    break
            time.sleep(0.05)
        time.sleep(0.2)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        busy = [r for r in rows if (num(r[8]) or 0) > 0] or rows
        sm = [num(r[0]) for r in busy if num(r[0]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in busy:
            for name, v in zip(names, r[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": num(rows[0][1]),
                "samples": len(busy), "reasons": sorted(reasons)}


# -------------------------------------------------------------- workload
def workload(n, rank, seed, device):
    """FP64 tensor (device), skew CP factors, stiffness and initial state."""
    import synth

    U, V, W, s, _ = synth.cp_workload(n, rank, 2)
    C = synth.cp_tensor_device(U, V, W, seed, s, device)
    a = synth.diag_stiffness(n)
    return C, (U, V, W), a


def svd_of_workload(C, ranks, torch):
    """Truncated SVD of the tensor's matricization over the advecting index
    (the SVD-ROM's offline step, Sec. 4.4.2) in FP64: M M^T on the device, its
    eigenpairs on the host (n x n), U and sigma from them and V = M^T U / sigma
    on the device.  Returns {rank: (U, sigma, V)} with V laid out n x rank x n
    (V[i][r][k])."""
    n = C.shape[0]
    M = C.permute(1, 0, 2).reshape(n, n * n)
    lam_h, vec_h = np.linalg.eigh((M @ M.T).cpu().numpy())
    lam, vec = torch.from_numpy(lam_h).to(C.device), torch.from_numpy(vec_h).to(C.device)
    order = torch.argsort(lam, descending=True)
    out = {}
    for r in ranks:
        idx = order[:r]
        sigma = torch.sqrt(torch.clamp(lam[idx], min=0.0))
        U = vec[:, idx].contiguous()
        V = (M.T @ U) / sigma[None, :]
        out[r] = (U, sigma.contiguous(), V.reshape(n, n, r).permute(0, 2, 1).contiguous())
        del V
    del M
    return out


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), float(d.get("bf16_tflops_sustained", 0) or 0), "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


def kernel_traffic(kernel_key):
    """dram bytes per launch of a kernel from the committed ncu summary, or None
    when the kernel source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh).get(kernel_key)
    if not d:
        return None
    h = hashlib.sha256()
    for f in d["sources"]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return d["bytes_per_launch"] if h.hexdigest() == d["source_sha256"] else None


# ------------------------------------------------------------------ timing
def time_steps(torch, tr, steps, stream):
    """ms per step of `steps` steps of an existing trajectory batch (one
    untimed step first, so captured graphs are rebuilt outside the region)."""
    tr.step(1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    tr.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def autotuned(torch, rom, tr, batch, steps, stream):
    """Autotune the ROM for the batch, then re-time the same trajectories."""
    t = rom.autotune(batch)
    ms = time_steps(torch, tr, steps, stream)
    return {"entry": t, "ms_per_step": ms, "trajectory_steps_per_s": batch * 1e3 / ms}


def flush_l2(buf):
    buf.add_(1.0)


def time_variant(grom, torch, rom, u0, steps, warmup, flush=None):
    """ms per step of grom_step(1) timed with CUDA events on the ROM's stream."""
    tr = grom.Trajectories(rom, u0)
    stream = torch.cuda.current_stream()
    tr.step(warmup)
    torch.cuda.synchronize()
    if flush is None:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tr.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        per = None
    else:
        per = []
        for _ in range(steps):
            flush_l2(flush)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            tr.step(1)
            e1.record(stream)
            per.append((e0, e1))
        torch.cuda.synchronize()
        per = [a.elapsed_time(b) for a, b in per]
        ms = float(np.mean(per))
    code, _ = tr.status()
    tr.close()
    return ms, code, per


def max_over_ranks(ms, device="cuda"):
    """Largest per-step time over all ranks (every rank gets it)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_initial_state(n, seed, rank_id):
    """The trajectory that replica `rank_id` steps (1 x n FP64): the seeded
    initial condition with trajectory index rank_id, so that every rank
    advances its own independent problem of the same workload."""
    import synth

    return synth.initial_condition(n, seed, traj=rank_id)


def replica_throughput(ms, world):
    """Steps per second of all replicas together, each stepping one trajectory."""
    return world * 1e3 / ms


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# ----------------------------------------------------------------- serving
def serving_section(args, grom, synth, torch, a_of):
    """Serving mix: four resident ROMs N = 128, 256, 512, 1024, each with skew
    CP factor sets of rank N and N/2 (the leading N/2 columns) in BF16 and
    FP64, served with continuous batching; compared with plain per-request
    FP64 full G-ROM stepping (one trajectory at a time, measured step times,
    FIFO queue)."""
    seed = synth.seed_for(4)
    ns = [128, 256, 512, 1024]
    roms, keys, streams, fulls = [], [], [], {}
    srv = grom.Server(150 * 2 ** 30, quantum=args.serve_quantum)
    for n in ns:
        U, V, W, resid, _ = synth.cp_workload(n, n, 4)
        a = a_of(n)
        for R in (n // 2, n):
            for storage in ("bf16", "f64"):
                st = torch.cuda.Stream()
                streams.append(st)
                fac = tuple(np.ascontiguousarray(x[:, :R]) for x in (U, V, W))
                rom = grom.Rom(n, "cp_skew", storage, factors=fac, stiffness=a, nu=NU, dt=DT,
                               max_batch=args.serve_slots, stream=st)
                roms.append(rom)
                keys.append((n, R, storage))
                srv.add_rom(rom, args.serve_slots)
        fulls[n] = (U, V, W, resid)
    times, horizons, draws = synth.arrivals(args.serve_requests, args.serve_rate, seed)
    nidx = (draws % 4).astype(int)
    vidx = ((draws // 4) % 4).astype(int)
    models = nidx * 4 + vidx
    u0s = [synth.initial_condition(ns[nidx[q]], seed, traj=q)[0] for q in range(len(models))]
    out = srv.serve(models, horizons, times, u0s, want_final=True)
    lat = out["t_done"] - times
    stats = out["stats"]
    res = {"requests": int(len(models)), "rate_per_s": args.serve_rate, "slots_per_rom": args.serve_slots,
           "roms": len(roms), "quantum_steps": args.serve_quantum, "hbm_budget_gb": 150,
           "status_ok": int(np.sum(out["status"] == 0)),
           "trajectory_steps": int(stats["trajectory_steps"]), "seconds": stats["seconds"],
           "steps_per_s": stats["trajectory_steps"] / stats["seconds"],
           "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
           "peak_active": int(stats["peak_active"]), "peak_gb": stats["peak_bytes"] / 1e9}
    # where the time goes: per resident ROM, the requests' demand and the
    # pool's measured step time with all slots busy (one quantum on random
    # states of the workload), i.e. the GPU time the demand needs at full pools
    per_rom = {}
    for q, (rom, (n_q, R_q, st_q)) in enumerate(zip(roms, keys)):
        mask = models == q
        demand = int(horizons[mask].sum())
        tr = grom.Trajectories(rom, synth.initial_condition(n_q, seed, 50000, args.serve_slots))
        tr.step(16)  # builds the pool's captured step graph outside the timed region
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(streams[q])
        tr.step(16)
        e1.record(streams[q])
        torch.cuda.synchronize()
        pool_ms = e0.elapsed_time(e1) / 16
        tr.close()
        per_rom["N%d_R%s_%s" % (n_q, "N" if R_q == n_q else "N/2", st_q)] = {
            "requests": int(mask.sum()), "demand_trajectory_steps": demand,
            "pool_ms_per_step_all_slots": pool_ms,
            "pool_trajectory_steps_per_s": args.serve_slots * 1e3 / pool_ms,
            "gpu_s_at_full_pools": demand / args.serve_slots * pool_ms * 1e-3}
    res["per_rom"] = per_rom
    res["per_rom_note"] = ("demand_trajectory_steps / slots x the pool's step time with every slot busy: the GPU "
                           "seconds each ROM's requests need if its pool ran alone and full; pools on different "
                           "streams overlap")
    # plain per-request FP64 full G-ROM: single-trajectory step time per N
    step_ms = {}
    finals_full = {}
    sample_s = {}
    order = np.argsort(horizons)
    sample = list(order[:8])
    for n in ns:
        U, V, W, resid = fulls[n]
        Cn = synth.cp_tensor_device(U, V, W, seed, resid, "cuda")
        full_rom = grom.Rom(n, "full", "f64", tensor=Cn, stiffness=a_of(n), nu=NU, dt=DT)
        del Cn
        tr = grom.Trajectories(full_rom, synth.initial_condition(n, seed, 0))
        tr.step(3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(torch.cuda.current_stream())
        tr.step(24)
        e1.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        step_ms[n] = e0.elapsed_time(e1) / 24
        tr.close()
        for q in sample:
            if ns[nidx[q]] == n:
                t1 = grom.Trajectories(full_rom, u0s[q][None, :])
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                t1.step(int(horizons[q]))
                finals_full[q] = t1.get_state()[0][:n]
                sample_s[q] = time.perf_counter() - t0
                t1.close()
        full_rom.close()
        torch.cuda.empty_cache()
    # FIFO queue of one-at-a-time requests with the measured step times
    end = 0.0
    blat = np.empty(len(models))
    for q in np.argsort(times, kind="stable"):
        start = max(times[q], end)
        end = start + horizons[q] * step_ms[ns[nidx[q]]] * 1e-3
        blat[q] = end - times[q]
    res["baseline_fp64_full_per_request"] = {
        "kind": "modelled",
        "steps_per_s": float(horizons.sum() / (end - times.min())),
        "p50_latency_s": float(np.percentile(blat, 50)), "p99_latency_s": float(np.percentile(blat, 99)),
        "step_ms_by_n": {str(k): v for k, v in step_ms.items()},
        "how": "modelled: a FIFO queue of the requests served one at a time in arrival order, each step costing "
               "the measured single-trajectory FP64 full step time of its N",
        "measured_sample": {
            "requests": len(sample_s), "trajectory_steps": int(sum(horizons[q] for q in sample_s)),
            "seconds": float(sum(sample_s.values())),
            "steps_per_s": float(sum(horizons[q] for q in sample_s) / max(sum(sample_s.values()), 1e-9)),
            "modelled_seconds": float(sum(horizons[q] * step_ms[ns[nidx[q]]] * 1e-3 for q in sample_s)),
            "how": "the %d shortest-horizon requests stepped one at a time through grom_step on the FP64 full "
                   "G-ROM (wall clock per request, including the final-state read-back)" % len(sample_s)}}
    errs = {}
    for q, ref in finals_full.items():
        n, R, storage = keys[models[q]]
        errs.setdefault("%s_R%s" % (storage, "N" if R == n else "N/2"), []).append(rel(out["final"][q], ref))
    res["final_state_rel_err_vs_fp64_full"] = {k: float(max(v)) for k, v in errs.items()}
    res["final_state_error_sample"] = "%d shortest-horizon requests, final state vs the same request on the " \
                                      "FP64 full G-ROM (model gap + precision)" % len(finals_full)
    srv.close()
    for rom in roms:
        rom.close()
    return res


# --------------------------------------------------------------- reference
def run_reference(args):
    import oracle
    import synth

    if int(os.environ.get("RANK", "0")) != 0:
        return
    n = args.n
    rank = args.rank or n
    dev = "cuda" if _cuda_ok() else "cpu"
    if dev == "cuda":
        C, _, a = workload(n, rank, synth.seed_for(2), dev)
        Ch = C.cpu().numpy()
        del C
    else:
        U, V, W, s, seed = synth.cp_workload(n, rank, 2)
        Ch = synth.cp_tensor(U, V, W, seed, s)
        a = synth.diag_stiffness(n)
    u0 = synth.initial_condition(n, synth.seed_for(2))[0]
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    rom = oracle.Rom("full", n, a, NU, DT, C=Ch)
    h = rom.initial_history(u0)
    t0 = time.perf_counter()
    rom.step(h, max(1, args.warmup))
    t_w = (time.perf_counter() - t0) / max(1, args.warmup)
    steps = args.steps
    budget = 150.0
    if steps * t_w > budget:
        steps = max(3, int(budget / t_w))
    t0 = time.perf_counter()
    rom.step(h, steps)
    dt = time.perf_counter() - t0
    v = steps / dt
    sample = "%d BDF3/EXT3 steps of the N=%d FP64 full G-ROM (of %d requested)" % (steps, n, args.steps)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": _workload(n, rank),
                   "storage": "FP64 dense tensor, FP64 loops on the host cores (the oracle, OpenMP over the "
                              "test index)", "n": n, "cp_rank": rank, "batch_per_gpu": 1, "nu": NU, "dt": DT,
                   "layout": "dense"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def _cuda_ok():
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:
        return False


def _packed_len(n):
    """Stored elements per row of the skew-packed layout: round_up(max(n//2, 1), 64)."""
    return (max(n // 2, 1) + 63) // 64 * 64


def _row_len(n, layout):
    return _packed_len(n) if layout == "skew_packed" else (n + 63) // 64 * 64


STORAGE_NAME = {"f32x2": "F32X2", "f64": "F64", "f32": "F32", "bf16": "BF16"}
ARITH = {"f32x2": "F32X2 tensor (FP32 hi/lo pair, 48-bit significand), double-single FP32 contraction "
                  "(error-free products and sums), FP64 state; FP64 tolerance (1e-12 per evaluation)",
         "f64": "FP64 tensor, FP64 contraction and state",
         "f32": "FP32 tensor, FP32 accumulation, FP64 state",
         "bf16": "BF16 tensor, FP32 accumulation, FP64 state"}


def _workload(n, rank):
    """The model every arm steps (the same text for the GPU and the reference arm)."""
    return ("N=%d full G-ROM, one BDF3/EXT3 step of one trajectory per GPU; CP-structured skew tensor (R=%d) "
            "+ 1e-3 skew residual, A = diag((i/N)^2), B = I" % (n, rank))


def _config(n, rank, layout, storage):
    how = ("skew-packed layout (one entry of each pair C_ijk = -C_kji)" if layout == "skew_packed"
           else "dense layout")
    return {"workload": _workload(n, rank), "storage": "%s; %s" % (ARITH[storage], how),
            "n": n, "cp_rank": rank, "batch_per_gpu": 1, "nu": NU, "dt": DT, "layout": layout,
            "l2": "inputs larger than L2 (stored tensor %.2f GB per step)" % (
                n * n * _row_len(n, layout) * STORAGE_BYTES[storage] / 1e9)}


# -------------------------------------------------------------------- main
def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch

    import oracle
    import synth
    import paper_2311_03694_gb300 as grom

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank_id = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    grom.build()
    n = args.n
    R = args.rank or n
    seed = synth.seed_for(2)
    C, factors, a = workload(n, R, seed, "cuda")
    u0 = replica_initial_state(n, seed, rank_id)  # one trajectory per replica
    hbm_peak, tc_peak, tc_sustained, peak_kind = peaks()

    def make_rom(form, storage, layout="dense"):
        if form == "full":
            return grom.Rom(n, "full", storage, tensor=C, stiffness=a, nu=NU, dt=DT, layout=layout)
        return grom.Rom(n, form, storage, factors=factors, stiffness=a, nu=NU, dt=DT)

    # ---------------------------------------------------- headline, timed
    rom = make_rom(HEADLINE_FORM, args.storage, args.layout)
    tr = grom.Trajectories(rom, u0)
    stream = torch.cuda.current_stream()
    tr.step(args.warmup)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    tr.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    code, bad = tr.status()
    ms = max_over_ranks(ms)
    value = replica_throughput(ms, world)  # all replicas' steps per second

    # The same K steps again with a CUDA event pair around every streaming
    # launch (event nodes inside the replayed graphs): the kernel's live
    # duration for the roofline.  The event nodes lengthen each step, so the
    # headline value above comes from the run without them.
    rom.profile(True)
    torch.cuda.synchronize()
    e0.record(stream)
    tr.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    profiled_ms = e0.elapsed_time(e1) / args.steps
    k1_ms, k1_launches = rom.profile_read()
    rom.profile(False)

    # roofline of the dominant kernel.  Its algorithmic bytes are the stored
    # tensor per step, N * N rows of round_up(N/2, 64) (skew-packed) or
    # round_up(N, 64) (dense) values of the storage type (8 bytes for F32X2
    # and FP64, 4 for FP32, 2 for BF16), times the steps one launch runs:
    # the persistent stepper runs all K steps (streaming, finalize and step)
    # in one launch, the graph path one streaming launch per step.
    k1_avg_ms = k1_ms / max(1, k1_launches)
    steps_per_launch = args.steps // max(1, k1_launches)
    step_bytes = float(n) * n * _row_len(n, args.layout) * STORAGE_BYTES[args.storage]
    alg_bytes = step_bytes * steps_per_launch
    achieved = alg_bytes / (k1_avg_ms * 1e-3) / 1e9
    persistent = steps_per_launch > 1
    kname = "k1pp" if persistent else ("k1_packed" if args.layout == "skew_packed" else "k1_stream")
    traffic = kernel_traffic("%s_%s_n%d" % (kname, args.storage, n))
    stname = STORAGE_NAME[args.storage]
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": traffic * steps_per_launch if traffic else None,
                "kernel": ("k1pp_kernel<%s> (persistent stepper: streaming, finalize and BDF3/EXT3 step of "
                           "%d steps in one launch)" % (stname, steps_per_launch)) if persistent
                else "%s_kernel<%s> (finalize excluded)" % (kname, stname), "peak_kind": peak_kind,
                "kernel_ms": k1_avg_ms, "kernel_launches": k1_launches, "steps_per_launch": steps_per_launch,
                "algorithmic_bytes_per_launch": alg_bytes,
                "timing": "CUDA events around each launch in a second timed run of the same %d steps "
                          "(%.4f ms per step with the events)" % (args.steps, profiled_ms)}

    # ------------------------------------------------------------- e2e
    pin_in = torch.empty((1, n), dtype=torch.float64).pin_memory()
    tr.step_host(0, None, pin_in.numpy())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2 = [torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
    e2[0].record(stream)
    for _ in range(args.steps):
        tr.step_host(1, pin_in, pin_in)  # state in from pinned host memory, new state back out
    e2[1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    e2e_ms = max(e2[0].elapsed_time(e2[1]), 1e3 * wall) / args.steps
    e2e = {"value": world * 1e3 / e2e_ms, "unit": UNIT, "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n,
           "api": "grom_step_host(traj, 1, u_in=pinned host, u_out=pinned host)"}
    tr.close()
    headline = {"storage": args.storage, "layout": args.layout, "tolerance": TOL[args.storage]}
    # launches in the headline timed region: one persistent launch, or per
    # step the streaming kernel and the fused finalize + step kernel
    timed_launches = 1 if persistent else 2 * args.steps

    # -------------------------------------------- errors vs the FP64 oracle
    cores = os.cpu_count() or 1
    Ch = None
    errors = {}
    cpu_baseline = None
    if rank_id == 0:
        oracle.set_threads(cores)
        Ch = C.cpu().numpy()
        t_ref = time.perf_counter()
        c_full = oracle.nonlinear_full(Ch, u0[0])
        t_ref = time.perf_counter() - t_ref
        c_cp = oracle.nonlinear_cp_skew(*factors, u0[0])
        ud = torch.from_numpy(u0.copy()).cuda()
        cd = torch.empty_like(ud)
        rom.nonlinear(ud, cd)
        torch.cuda.synchronize()
        headline["eval_rel_err_vs_fp64_oracle"] = rel(cd.cpu().numpy()[0], c_full)
        headline["eval_max_abs_err_over_max_abs"] = float(np.max(np.abs(cd.cpu().numpy()[0] - c_full)) /
                                                          np.max(np.abs(c_full)))

    # ------------------------------------------------------------ variants
    wanted = VARIANTS if args.variants == "all" else (
        [] if args.variants == "none" else [tuple((v + ":dense").split(":")[:3]) for v in args.variants.split(",")
                                            if v != "aug"])
    flush = torch.empty(2 * L2_BYTES // 8, dtype=torch.float64, device="cuda")
    variants = {}
    for form, storage, layout in wanted:
        vrom = make_rom(form, storage, layout)
        key = "%s_%s%s" % ("full" if form == "full" else "cpd", storage, "_packed" if layout == "skew_packed" else "")
        vsteps = max(10, min(args.steps, 200))
        if form == "full":
            vms, vcode, _ = time_variant(grom, torch, vrom, u0, vsteps, 8)
            entry = {"ms_per_step": vms, "steps_per_s": 1e3 / vms, "l2": "tensor > L2", "layout": layout}
        else:
            vms, vcode, per = time_variant(grom, torch, vrom, u0, vsteps, 8, flush=flush)
            # warm-up of 8 steps: one call long enough to run (and load) the persistent stepper
            wms, _, _ = time_variant(grom, torch, vrom, u0, vsteps, 8)
            entry = {"ms_per_step": vms, "steps_per_s": 1e3 / vms, "l2": "flushed before every step",
                     "p50_ms": float(np.percentile(per, 50)), "p99_ms": float(np.percentile(per, 99)),
                     "warm_l2_ms_per_step": wms, "warm_l2_steps_per_s": 1e3 / wms}
        if rank_id == 0:
            ud = torch.from_numpy(u0.copy()).cuda()
            cd = torch.empty_like(ud)
            vrom.nonlinear(ud, cd)
            torch.cuda.synchronize()
            ref = c_full if form == "full" else c_cp
            entry["eval_rel_err_vs_fp64_oracle"] = rel(cd.cpu().numpy()[0], ref)
            entry["tolerance"] = TOL[storage]
            if form != "full":
                entry["cp_vs_full_model_gap"] = rel(ref, c_full)
        entry["status"] = grom.ERRORS.get(vcode, "OK") if vcode else "OK"
        variants[key] = entry
        vrom.close()
    # the model including the zeroth mode (Sec. 4.2): skew-packed BF16 core,
    # zeroth-mode terms in the stepper's L and f (dense-L step)
    if args.variants == "all" or "aug" in args.variants.split(","):
        Cbar = synth.augment_tensor_device(C, seed)
        vrom = grom.Rom(n, "full", "bf16", tensor=Cbar, stiffness=a, nu=NU, dt=DT, layout="skew_packed",
                        augmented=True)
        vsteps = max(10, min(args.steps, 200))
        vms, vcode, _ = time_variant(grom, torch, vrom, u0, vsteps, 3)
        entry = {"ms_per_step": vms, "steps_per_s": 1e3 / vms, "l2": "tensor > L2", "layout": "skew_packed",
                 "zeroth_mode": "L += C1 + C2 (dense), f += c0"}
        if rank_id == 0:
            Cbh = Cbar.cpu().numpy()
            ref_rom = oracle.Rom("full_aug", n, a, NU, DT, C=Cbh)
            h = ref_rom.initial_history(u0[0])
            ref_rom.step(h, 3)
            vt = grom.Trajectories(vrom, u0)
            vt.step(3)
            entry["traj_rel_err_after_3_steps_vs_fp64_oracle"] = rel(vt.get_state()[0][:n], h[:n])
            entry["tolerance"] = TOL["bf16"]
            vt.close()
            del Cbh
        entry["status"] = grom.ERRORS.get(vcode, "OK") if vcode else "OK"
        variants["full_bf16_packed_augmented"] = entry
        vrom.close()
        del Cbar
        torch.cuda.empty_cache()
    # SVD-ROM (Sec. 4.4.2) at the requested ranks: skew-packed BF16 slices
    if args.svd_ranks and args.svd_ranks != "none" and args.variants != "none":
        ranks = [int(x) for x in args.svd_ranks.split(",")]
        for r, (Us, ss, Vs) in svd_of_workload(C, ranks, torch).items():
            for storage in ("bf16", "f64"):
                vrom = grom.Rom(n, "svd", storage, factors=(Us, ss, Vs), stiffness=a, nu=NU, dt=DT,
                                layout="skew_packed")
                vsteps = max(10, min(args.steps, 200))
                vms, vcode, per = time_variant(grom, torch, vrom, u0, vsteps, 3, flush=flush)
                wms, _, _ = time_variant(grom, torch, vrom, u0, vsteps, 3)
                entry = {"rank": r, "cr_svd": n / r, "layout": "skew_packed", "ms_per_step": vms,
                         "steps_per_s": 1e3 / vms, "l2": "flushed before every step",
                         "p50_ms": float(np.percentile(per, 50)), "p99_ms": float(np.percentile(per, 99)),
                         "warm_l2_ms_per_step": wms, "warm_l2_steps_per_s": 1e3 / wms,
                         "stored_bytes": n * r * _packed_len(n) * STORAGE_BYTES[storage]}
                if rank_id == 0:
                    ud = torch.from_numpy(u0.copy()).cuda()
                    cd = torch.empty_like(ud)
                    vrom.nonlinear(ud, cd)
                    torch.cuda.synchronize()
                    ref = oracle.nonlinear_svd(Us.cpu().numpy(), ss.cpu().numpy(), Vs.cpu().numpy(), u0[0])
                    entry["eval_rel_err_vs_fp64_oracle"] = rel(cd.cpu().numpy()[0], ref)
                    entry["tolerance"] = TOL[storage]
                    entry["svd_vs_full_model_gap"] = rel(ref, c_full)
                entry["status"] = grom.ERRORS.get(vcode, "OK") if vcode else "OK"
                variants["svd_%s_packed_R%d" % (storage, r)] = entry
                vrom.close()
            del Us, ss, Vs
        torch.cuda.empty_cache()
    del flush

    # ------------------------------------------- batched trajectories (K2)
    batched = {}
    if args.batches and args.batches != "none":
        for B in [int(x) for x in args.batches.split(",")]:
            brom = grom.Rom(n, "full", "bf16", tensor=C, stiffness=a, nu=NU, dt=DT, max_batch=B)
            U0 = synth.initial_condition(n, seed, 0, B)
            btr = grom.Trajectories(brom, U0)
            bsteps = 10
            # warm-up with timing on, so that the captured step graph (which
            # carries the timing nodes) is built outside the timed region
            brom.profile(True)
            btr.step(bsteps)
            brom.profile_read()
            torch.cuda.synchronize()
            e0b, e1b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0b.record(stream)
            btr.step(bsteps)
            e1b.record(stream)
            torch.cuda.synchronize()
            kms, kl = brom.profile_read()
            brom.profile(False)
            bms = e0b.elapsed_time(e1b) / bsteps
            kavg = kms / max(1, kl)
            flops = 2.0 * float(n) ** 3 * B
            entry = {"ms_per_step": bms, "trajectory_steps_per_s": B * 1e3 / bms,
                     "kernel": "k2_tc_kernel (tcgen05, KR hi/lo)" if B > 8 else "k1_stream_kernel",
                     "kernel_ms": kavg, "alg_tflops": flops / (kavg * 1e-3) / 1e12, "alg_flops": "2 N^3 B",
                     "tc_frac_of_sustained_bf16": flops / (kavg * 1e-3) / 1e12 / tc_sustained,
                     "issued_tflops": 2.0 * flops / (kavg * 1e-3) / 1e12,
                     "hbm_frac": float(n) ** 3 * 2 / (kavg * 1e-3) / 1e9 / hbm_peak}
            if rank_id == 0:
                # evaluate the whole batch through the batched kernel, check three trajectories
                uf = torch.from_numpy(U0.copy()).cuda()
                cf = torch.empty_like(uf)
                brom.nonlinear(uf, cf)
                torch.cuda.synchronize()
                errs = [rel(cf[b].cpu().numpy(), oracle.nonlinear_full(Ch, U0[b])) for b in range(min(3, B))]
                entry["eval_rel_err_vs_fp64_oracle_max3"] = max(errs)
            if args.autotune:
                entry["autotuned"] = autotuned(torch, brom, btr, B, bsteps, stream)
            code_b, _ = btr.status()
            entry["status"] = grom.ERRORS.get(code_b, "OK") if code_b else "OK"
            batched["B%d" % B] = entry
            btr.close()
            brom.close()
            # the same batch on the skew-packed tensor: the factored K2P kernel
            prom = grom.Rom(n, "full", "bf16", tensor=C, stiffness=a, nu=NU, dt=DT, max_batch=B,
                            layout="skew_packed")
            ptr = grom.Trajectories(prom, U0)
            prom.profile(True)
            ptr.step(bsteps)
            prom.profile_read()
            torch.cuda.synchronize()
            e0b.record(stream)
            ptr.step(bsteps)
            e1b.record(stream)
            torch.cuda.synchronize()
            kms, kl = prom.profile_read()
            pms = e0b.elapsed_time(e1b) / bsteps
            kavg = kms / max(1, kl)
            pairs = B > 8 and _packed_len(n) > 128  # the rule: SM pairs wherever a row has two blocks
            single_ms = None
            if pairs:
                # the same steps on single CTAs (one 128-row MMA per CTA), for comparison
                prom.set_tuning({"batch": B, "kernel": "tensor", "tile_m": 0, "split_a": 0, "split_b": 1})
                str1 = grom.Trajectories(prom, U0)
                str1.step(bsteps)
                prom.profile_read()
                torch.cuda.synchronize()
                str1.step(bsteps)
                torch.cuda.synchronize()
                sms, sl = prom.profile_read()
                single_ms = sms / max(1, sl)
                str1.close()
                prom.set_tuning({"batch": B, "kernel": "auto", "tile_m": 0, "split_a": 0, "split_b": 0})
            prom.profile(False)
            pbytes = float(n) * n * _packed_len(n) * 2
            # the factored kernel's own work: one multiply-add per stored entry
            # and trajectory (N x N x lp of them, the stored half); the dense
            # contraction's 2 N^3 B is reported beside it as an equivalent rate
            own = 2.0 * n * n * _packed_len(n) * B
            pentry = {"ms_per_step": pms, "trajectory_steps_per_s": B * 1e3 / pms,
                      "kernel": ("k2p_pair_kernel (tcgen05 over SM pairs, cta_group::2, factored, skew-packed)" if pairs
                                 else "k2p_tc_kernel (tcgen05, factored, skew-packed)" if B > 8 else "k1_packed_kernel"),
                      "kernel_ms": kavg, "alg_tflops": own / (kavg * 1e-3) / 1e12,
                      "alg_flops": "2 N N lp B (lp = %d stored positions per row)" % _packed_len(n),
                      "tc_frac_of_sustained_bf16": own / (kavg * 1e-3) / 1e12 / tc_sustained,
                      "dense_equivalent_tflops": flops / (kavg * 1e-3) / 1e12,
                      "issued_tflops": 2.0 * own / (kavg * 1e-3) / 1e12,
                      "issued_note": "twice the own work: the states enter the MMA as BF16 hi and lo parts",
                      "stored_tensor_bytes": pbytes,
                      "hbm_frac_per_tensor_read": pbytes / (kavg * 1e-3) / 1e9 / hbm_peak}
            if single_ms is not None:
                pentry["single_cta_kernel_ms"] = single_ms
                pentry["single_cta_tc_frac_of_sustained_bf16"] = own / (single_ms * 1e-3) / 1e12 / tc_sustained
            if rank_id == 0:
                uf = torch.from_numpy(U0.copy()).cuda()
                cf = torch.empty_like(uf)
                prom.nonlinear(uf, cf)
                torch.cuda.synchronize()
                errs = [rel(cf[b].cpu().numpy(), oracle.nonlinear_full(Ch, U0[b])) for b in range(min(3, B))]
                pentry["eval_rel_err_vs_fp64_oracle_max3"] = max(errs)
            if args.autotune:
                pentry["autotuned"] = autotuned(torch, prom, ptr, B, bsteps, stream)
            code_p, _ = ptr.status()
            pentry["status"] = grom.ERRORS.get(code_p, "OK") if code_p else "OK"
            batched["B%d_packed" % B] = pentry
            ptr.close()
            prom.close()
            # the CPD-ROM (skew CP factors, rank N) on the same batch: BF16
            # factors on the tensor cores, FP64 factors in double-single FP32
            # arithmetic (K3D, FP64 tolerance) and, for reference, in FP64
            # arithmetic (K3g, GROM_KERNEL_STREAM)
            for storage, kernel in (("bf16", "auto"), ("f64", "auto"), ("f64", "tensor"), ("f64", "stream")):
                crom = grom.Rom(n, "cp_skew", storage, factors=factors, stiffness=a, nu=NU, dt=DT, max_batch=B)
                crom.set_kernel(kernel)
                ctr = grom.Trajectories(crom, U0)
                ctr.step(bsteps)  # builds the captured step graph outside the timed region
                torch.cuda.synchronize()
                e0b.record(stream)
                ctr.step(bsteps)
                e1b.record(stream)
                torch.cuda.synchronize()
                cms = e0b.elapsed_time(e1b) / bsteps
                cflops = 2.0 * 5 * n * R * B  # p, q, s projections and two expansions
                key = "B%d_cpd_%s%s" % (B, storage, {"stream": "_fp64_gemm", "tensor": "_tensor"}.get(kernel, ""))
                entry = {
                    "ms_per_step": cms, "trajectory_steps_per_s": B * 1e3 / cms,
                    "alg_tflops": cflops / (cms * 1e-3) / 1e12,
                    "kernel": ("k3t_gemm x2 (tcgen05 projections and expansion)" if storage == "bf16" and B >= 16
                               else ("k3o (tcgen05 GEMMs of digit slices: %s-bit for the projections, 6-bit for the "
                                     "expansion; FP64 tolerance)" % ("7" if n <= 1024 else "6"))
                               if storage == "f64" and B >= 16 and (kernel == "tensor" or (
                                   kernel == "auto" and n * R * B >= 2 ** 24))
                               else "k3d project/expand (double-single FP32 GEMMs, FP64 tolerance)"
                               if storage == "f64" and kernel == "auto" and B >= 16
                               else "k3g project/expand (register-tiled FP64 GEMMs)" if B >= 16
                               else "k3 project/expand")}
                if rank_id == 0:
                    uf = torch.from_numpy(U0.copy()).cuda()
                    cf = torch.empty_like(uf)
                    crom.nonlinear(uf, cf)
                    torch.cuda.synchronize()
                    errs = [rel(cf[b].cpu().numpy(), oracle.nonlinear_cp_skew(*factors, U0[b])) for b in range(min(3, B))]
                    entry["eval_rel_err_vs_fp64_oracle_max3"] = max(errs)
                    entry["tolerance"] = TOL[storage]
                if args.autotune and storage == "bf16":
                    entry["autotuned"] = autotuned(torch, crom, ctr, B, bsteps, stream)
                batched[key] = entry
                ctr.close()
                crom.close()

    # -------------------------------------- CP fitting (ALS, ALS-skew)
    fitting = {}
    if args.als_ranks and args.als_ranks != "none":
        als = grom.Als(C)
        for r in [int(x) for x in args.als_ranks.split(",")]:
            F0 = [synth.normal(seed, 30 + q, 0, n * r).reshape(n, r) / np.sqrt(n) for q in range(3)]
            for method in ("plain", "skew"):
                init = F0 if method == "plain" else (F0[0], F0[1][:, : r // 2])
                als.fit(init, 1, method=method, ridge=args.als_ridge)  # warm-up (allocation, tensor maps)
                als.stats()
                t0 = time.perf_counter()
                _, res = als.fit(init, args.als_iters, method=method, ridge=args.als_ridge)
                wall = (time.perf_counter() - t0) / args.als_iters
                mms, calls, solve = als.stats()
                flops = 2.0 * float(n) ** 3 * r  # one MTTKRP: X_(m) (P kr Q)
                per = mms / max(calls, 1)
                fitting["%s_R%d" % (method, r)] = {
                    "rank": r, "iterations": args.als_iters, "ridge": args.als_ridge, "s_per_iteration": wall,
                    "mttkrp_per_iteration": calls / args.als_iters, "mttkrp_ms": per,
                    "note": "one MTTKRP per iteration is the residual's <X, K>",
                    "mttkrp_alg_tflops": flops / (per * 1e-3) / 1e12,
                    "mttkrp_tc_frac_of_sustained_bf16": flops / (per * 1e-3) / 1e12 / tc_sustained,
                    "solve_ms_per_iteration": solve / args.als_iters,
                    "relative_residual": [float(x) for x in res],
                    "init": "seeded normal factors / sqrt(N) (stream 30-32)"}
        als.close()

    # ---------------------------------------------- CPU baseline (oracle)
    if rank_id == 0 and not args.no_cpu_baseline:
        a_rom = oracle.Rom("full", n, a, NU, DT, C=Ch)
        h = a_rom.initial_history(u0[0])
        t0 = time.perf_counter()
        a_rom.step(h, 1)
        t1 = time.perf_counter() - t0
        k = int(max(1, min(200, args.cpu_seconds / max(t1, 1e-6))))
        t0 = time.perf_counter()
        a_rom.step(h, k)
        tk = time.perf_counter() - t0
        cpu_baseline = {"value": k / tk, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
                        "sample": "%d BDF3/EXT3 steps (after 1 untimed) of the N=%d FP64 full G-ROM on the "
                                  "host cores, OpenMP over the test index" % (k, n)}
        # trajectory error after 1 + k steps: the headline, each full-form
        # storage type and layout, and each CPD variant against the oracle's
        # CPD-ROM (same factors, same steps)
        tkey = "traj_rel_err_after_%d_steps" % (1 + k)
        ht = grom.Trajectories(rom, u0)
        ht.step(1 + k)
        headline[tkey] = rel(ht.get_state()[0][:n], h[:n])
        ht.close()
        for key in [k for k in variants if k.startswith("full_") and "augmented" not in k]:
            storage = key.split("_")[1]
            vrom = make_rom("full", storage, variants[key]["layout"])
            vt = grom.Trajectories(vrom, u0)
            vt.step(1 + k)
            hv = vt.get_state()[0]
            variants[key][tkey] = rel(hv[:n], h[:n])
            vt.close()
            vrom.close()
        cpd_keys = [k for k in variants if k.startswith("cpd_")]
        if cpd_keys:
            cp_ref = oracle.Rom("cp_skew", n, a, NU, DT, factors=factors)
            hc = cp_ref.initial_history(u0[0])
            cp_ref.step(hc, 1 + k)
            for key in cpd_keys:
                vrom = make_rom("cp_skew", key.split("_")[1])
                vt = grom.Trajectories(vrom, u0)
                vt.step(1 + k)
                variants[key][tkey] = rel(vt.get_state()[0][:n], hc[:n])
                variants[key][tkey + "_cpd_vs_full_model_gap"] = rel(hc[:n], h[:n])
                vt.close()
                vrom.close()
        errors["oracle_full_eval_seconds"] = t_ref

    # ------------------------------------------------------ serving mix
    serving = None
    if args.serve_requests > 0 and rank_id == 0:
        del C
        torch.cuda.empty_cache()
        serving = serving_section(args, grom, synth, torch, a_of=synth.diag_stiffness)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
        "config": _config(n, R, args.layout, args.storage),
        "headline": headline,
        "roofline": roofline,
        "cpu_baseline": cpu_baseline,
        "e2e": e2e,
        "gpu_launches": timed_launches,  # in the headline timed region
        "clocks": clocks,
        "status": grom.ERRORS.get(code, "OK") if code else "OK",
        "variants": variants,
        "batched": batched,
        "serving": serving,
        "fitting": fitting,
    }
    if errors:
        line["oracle"] = errors
    rom.close()
    if rank_id == 0:
        out = json.dumps(line)
        print(out)
        if args.json_out:
            with open(args.json_out, "w") as fh:
                fh.write(out + "\n")
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
