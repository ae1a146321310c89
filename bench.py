#!/usr/bin/env python
"""Throughput of the ACE build + apply hot path on GB300.

One step = one pass of the whole hot path over one synthetic system: orbitals
to real space, every pair density and its FFT Poisson solve with the exchange
accumulation, W to reciprocal space, M = Phi^T W, the FP64 Cholesky of -M,
xi = W L^-T, E_x, and one ACE apply K psi = -xi (xi^T psi) on n_occ trial
vectors (an inner MTS step).  Workload: 128 occupied real orbitals of a
32-water-box-shaped cell (18.6 bohr, 96^3 grid, 80 Ry, 8256 pairs), seeded
synthetic Gaussian-sum orbitals.

Prints one JSON line.  value = pair Poisson solves per second (whole job);
the line also carries ACE builds per second, the FP64 GPU form of the same
step, the roofline of the dominant kernel, a CPU-oracle baseline, the
end-to-end number through the public API with host buffers, and the SM
clocks sampled during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pair Poisson solves/sec + ACE builds/sec, mixed vs FP64 GPU at |dE_x|<=1e-6 Ha/atom"
WORKLOAD = "water32: 128 occupied real orbitals, 96^3 grid, cubic 18.6 bohr, 80 Ry, 8256 pairs, alpha 0.25"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
GOLDEN_DIR = os.path.join(ROOT, "tests", "golden")
L2_BYTES = 129 * 1024 * 1024
ALG_BYTES_PER_PAIR_PER_POINT = 16  # FP32: four complex (8-byte) transfers per packed transform of two pairs


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[4 + i] and "Not" not in r[4 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def workload(seed_trials=77):
    import gen
    cfg = gen.config_water32()
    trials = gen.random_trials(cfg["cell"], cfg["ecut"], cfg["psi"].shape[0], seed_trials)
    return cfg, trials


def golden(key):
    """The FP64 oracle's stored results for a full-size workload
    (tests/golden/fullsize_<key>.npz, written by make_fullsize_oracle.py from
    the oracle alone), or None when not stored."""
    path = os.path.join(GOLDEN_DIR, f"fullsize_{key}.npz")
    if not os.path.exists(path):
        return None
    with np.load(path) as z:
        d = {k: z[k] for k in z.files}
    d["E_x"] = float(d["E_x"])
    return d


def parity_vs_oracle(ace, plan, cfg, xi, E, key):
    """The metric's validity gate against the stored oracle results: |dE_x|
    per atom, K psi on the stored trials (max |diff| / max |K psi|), M and the
    quadratic form t^T K t; None when the workload has no stored results."""
    import torch

    import gen
    g = golden(key)
    if g is None:
        return None
    n = len(cfg["psi"])
    T = max(int(g["n_kpsi"]), int(g["n_q"]))
    tr = gen.random_trials(cfg["cell"], cfg["ecut"], T, seed=int(g["trials_seed"]))
    dt = plan.cdtype
    K = ace.ace_apply(plan, xi, torch.from_numpy(tr.astype(np.complex64 if dt == torch.complex64 else np.complex128))
                      .cuda()).cpu().numpy().astype(np.complex128)
    Kg = g["Kpsi"].astype(np.complex128)
    _, M = ace.ace_last_intermediates(plan, n)
    Q = gen.gamma_overlap(tr[:int(g["n_q"])], K[:int(g["n_q"])])
    rows = g["M_rows"]
    return {"dE_x_per_atom_vs_oracle": abs(E - g["E_x"]) / cfg["n_atom"],
            "Kpsi_rel_vs_oracle": float(np.abs(K[:len(Kg)] - Kg).max() / np.abs(Kg).max()),
            "M_rel_vs_oracle": float(np.abs(M[rows] - g["M"]).max() / np.abs(g["M"]).max()),
            "Q_rel_vs_oracle": float(np.abs(Q - g["Q"]).max() / np.abs(g["Q"]).max()),
            "E_x_oracle": g["E_x"], "trials": T, "tolerance": {"dE_x_per_atom": 1e-6, "Kpsi_rel": 1e-6}}


def workload_leg(ace, cfg, key, hbm, steps=2, warmup=1, trial_sets=(), pairs=None, fp64=True):
    """Another configuration of the metric, timed like the headline (CUDA
    events on the call's stream, L2 flushed between steps): a step is one
    ace_build over the listed pairs plus one ace_apply per trial set.  Reports
    pairs/s and builds/s of the mixed form, its pair-pass roofline (16 N bytes
    per pair over the pair wall time), the stored-oracle deltas, and the FP64
    GPU form of the same step (one step, no warm-up: it is slow)."""
    import torch

    n = len(cfg["psi"])
    npairs = n * (n + 1) // 2 if pairs is None else int(pairs[0][-1])
    N = int(np.prod(cfg["grid"]))
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    out = {"workload": cfg["name"], "pairs_per_build": npairs, "apply_calls_per_step": len(trial_sets),
           "apply_trials": int(trial_sets[0].shape[0]) if len(trial_sets) else 0}
    for prec in ("mixed", "fp64") if fp64 else ("mixed",):
        plan = ace.Plan(cfg["grid"], cfg["cell"], cfg["ecut"], n, prec)
        dt = np.complex64 if prec == "mixed" else np.complex128
        psi = torch.from_numpy(cfg["psi"].astype(dt)).cuda()
        trs = [torch.from_numpy(t.astype(dt)).cuda() for t in trial_sets]
        xi = torch.empty_like(psi)
        outs = [torch.empty_like(t) for t in trs]
        E = [None]
        apply_ev = []  # (start, end) events around each step's applies

        def step():
            _, E[0] = ace.ace_build(plan, psi, cfg["alpha"], pairs=pairs, xi=xi)
            if trs:
                a_ = torch.cuda.Event(enable_timing=True)
                b_ = torch.cuda.Event(enable_timing=True)
                a_.record()
                # the outer step's split copy of xi, then its inner steps (timed with them)
                ace.ace_apply_prepare(plan, xi)
                for t, o in zip(trs, outs):
                    ace.ace_apply(plan, xi, t, out=o)
                b_.record()
                apply_ev.append((a_, b_))

        nw, ns = (warmup, steps) if prec == "mixed" else (0, 1)
        for _ in range(nw):
            step()
        torch.cuda.synchronize()
        apply_ev.clear()
        ace.ace_get_stats(plan)
        ace.ace_set_timing(plan, prec == "mixed")
        total = 0.0
        for _ in range(ns):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            step()
            b.record()
            torch.cuda.synchronize()
            total += a.elapsed_time(b)
        st = ace.ace_get_stats(plan)
        ace.ace_set_timing(plan, False)
        ms = total / ns
        rec = {"ms_per_step": ms, "pairs_per_s": npairs / (ms / 1e3), "builds_per_s": 1e3 / ms, "E_x": E[0]}
        if prec == "mixed":
            wall = st["pair_wall_ms"] / ns
            ach = ALG_BYTES_PER_PAIR_PER_POINT * N * npairs / (wall / 1e3) / 1e9 if wall > 0 else 0.0
            apply_ms = sum(a_.elapsed_time(b_) for a_, b_ in apply_ev) / ns if apply_ev else 0.0
            rec.update(pair_wall_ms_per_build=wall, apply_ms_per_step=apply_ms,
                       apply_ms_per_call=apply_ms / len(trs) if trs else None,
                       roofline={"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                                 "count": "16 N bytes per pair over the pair passes' wall time"},
                       pair_kernels=plan.config(),
                       parity=parity_vs_oracle(ace, plan, cfg, xi, E[0], key) if key else None)
            out["mixed"] = rec
        else:
            rec["dE_x_per_atom_mixed_vs_fp64"] = abs(out["mixed"]["E_x"] - E[0]) / cfg["n_atom"]
            out["fp64_gpu"] = rec
        plan.close()
        del psi, trs, xi, outs
    del flush
    torch.cuda.empty_cache()
    return out


def pair_quads(n):
    """Packed transforms of the all-pairs list i <= j, two consecutive pairs each."""
    pairs = [(i, j) for i in range(n) for j in range(i, n)]
    return [(pairs[k], pairs[k + 1] if k + 1 < len(pairs) else None) for k in range(0, len(pairs), 2)]


def pass_bytes(n, N, esz=4, batch=64):
    """Algorithmic HBM bytes of each pair pass over one build (FP32), counted
    per launch of `batch` packed transforms (the library's launch size on this
    workload): P1 writes the half-transformed spectrum (8N per transform) and
    reads each distinct orbital of the launch once (4N); P2 reads and writes
    the spectrum (16N per transform); P3 reads the spectrum (8N per transform),
    each distinct orbital of the launch once (4N) and read-modify-writes each
    distinct W of the launch once (8N).  Returns (bytes per pass, launches)."""
    c = 2 * esz
    tot = {"pair_fwd": 0, "pair_coulomb": 0, "pair_inv": 0}
    quads = pair_quads(n)
    launches = 0
    for s0 in range(0, len(quads), batch):
        chunk = quads[s0:s0 + batch]
        t = len(chunk)
        fs = set()
        for p, q in chunk:
            fs |= {p[0], p[1]} | ({q[0], q[1]} if q else set())
        tot["pair_fwd"] += N * (c * t + esz * len(fs))
        tot["pair_coulomb"] += N * 2 * c * t
        tot["pair_inv"] += N * (c * t + esz * len(fs) + 2 * esz * len(fs))
        launches += 1
    return tot, launches


# DRAM bytes per launch (64 transforms) of the pair passes on this workload,
# from ncu captures (dram__bytes_read.sum + dram__bytes_write.sum; see
# profiles/dram_pair_passes_water32_96cubed.md): the tile-pass forward kernel,
# the plane-kernel forward pass of the hybrid variant, and the Coulomb and
# accumulation kernels both variants share.
MEASURED_TRAFFIC_PER_LAUNCH = {"pair_fwd": None, "pair_fwd_hybrid": 0.5473e9, "pair_coulomb": 0.8473e9,
                               "pair_inv": 0.8595e9}


def cpu_baseline(cfg, rows=5):
    """The FP64 oracle on a bounded sample of the workload's pairs, all host cores."""
    import oracle
    n = cfg["psi"].shape[0]
    # sample: the pairs of the first `rows` rows of the pair list (all of the
    # orbital and W transforms still run; the rate counts the pair-solve time only)
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    cols = []
    for i in range(rows):
        cols.extend(range(i, n))
        row_ptr[i + 1] = len(cols)
    row_ptr[rows + 1:] = len(cols)
    cols = np.array(cols, dtype=np.int32)
    _, _, t = oracle.exchange(cfg["psi"], cfg["cell"], cfg["grid"], cfg["ecut"], cfg["alpha"],
                              pairs=(row_ptr, cols), times=True)
    npairs = len(cols)
    return {"value": npairs / t[1], "unit": "pairs/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"FP64 oracle on {npairs} pairs (rows 0-{rows - 1} of the {n * (n + 1) // 2}-pair list): "
                      f"pair solves {t[1]:.1f} s, orbital transforms {t[0]:.1f} s, "
                      f"W back-transforms {t[2]:.1f} s (not counted)"}


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    cfg, _ = workload()
    # each step a bounded sample: the pairs of the first two rows (about 6 s
    # of oracle work on 16 cores); warm-up steps one row
    for _ in range(args.warmup):
        cpu_baseline(cfg, rows=1)
    vals, walls = [], []
    sample = None
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        cb = cpu_baseline(cfg, rows=2)
        walls.append((time.perf_counter() - t0) * 1e3)
        vals.append(cb["value"])
        sample = cb
    v = statistics.median(vals)
    n = cfg["psi"].shape[0]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "pairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.median(walls),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"water32 sample: the {2 * n - 1} pairs of rows 0-1 of the {n * (n + 1) // 2}-pair "
                                   "list (128 orbitals, 96^3, 18.6 bohr, 80 Ry), all orbital transforms; "
                                   "value = sampled pairs / pair-solve seconds",
                       "sample": sample["sample"]},
            "full_build_ms_extrapolated": n * (n + 1) // 2 / v * 1e3,
            "cpu_baseline": {"value": v, "unit": "pairs/s", "cores": sample["cores"], "kind": "oracle",
                             "sample": sample["sample"]},
            "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch

    import paper_2110_07670_gb300 as ace

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    cfg, trials = workload()
    n = cfg["psi"].shape[0]
    npairs = n * (n + 1) // 2
    N = int(np.prod(cfg["grid"]))

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # N > 1: the pairs of the one build are sharded over the ranks, W_G and E_x
    # summed by one NCCL allreduce, and each rank applies xi to its slice of
    # the trial vectors; N = 1: the plain build and apply
    t_lo, t_hi = trials.shape[0] * rank // world, trials.shape[0] * (rank + 1) // world
    my_trials = trials[t_lo:t_hi]

    def setup(prec):
        plan = ace.Plan(cfg["grid"], cfg["cell"], cfg["ecut"], n, prec,
                        pair_variant=(args.pair_variant or 0) if prec == "mixed" else 0)
        dt = np.complex64 if prec == "mixed" else np.complex128
        psi = torch.from_numpy(cfg["psi"].astype(dt)).cuda()
        tr = torch.from_numpy(my_trials.astype(dt)).cuda()
        xi = torch.empty_like(psi)
        K = torch.empty_like(tr)
        return plan, psi, tr, xi, K

    WG_buf = {}

    def build(plan, psi, xi):
        if world == 1:
            return ace.ace_build(plan, psi, cfg["alpha"], xi=xi)
        from paper_2110_07670_gb300 import shard
        key = id(plan)
        if key not in WG_buf:
            WG_buf[key] = torch.empty_like(psi)
        return shard.build_sharded(plan, psi, cfg["alpha"], xi=xi, W_G=WG_buf[key])

    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    def timed_steps(plan, psi, tr, xi, K, steps, warmup, with_timing=False):
        E = None
        for _ in range(warmup):
            xi, E = build(plan, psi, xi)
            ace.ace_apply(plan, xi, tr, out=K)
        torch.cuda.synchronize()
        ace.ace_get_stats(plan)
        ace.ace_set_timing(plan, with_timing)
        barrier()
        torch.cuda.synchronize()
        total = 0.0
        for _ in range(steps):
            flush.zero_()  # L2 flush between timed steps, outside the timed interval
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            xi, E = build(plan, psi, xi)
            ace.ace_apply(plan, xi, tr, out=K)
            b.record()
            torch.cuda.synchronize()
            total += a.elapsed_time(b)
        barrier()
        torch.cuda.synchronize()
        stats = ace.ace_get_stats(plan)
        ace.ace_set_timing(plan, False)
        return total, E, stats

    # ---- mixed form, device-resident inputs (the headline value)
    plan, psi, tr, xi, K = setup("mixed")
    sampler = ClockSampler(local)
    sampler.start()
    total_ms, E_mixed, stats = timed_steps(plan, psi, tr, xi, K, args.steps, args.warmup, with_timing=True)
    # the metric's validity gate on this build, against the stored FP64 oracle results
    parity = parity_vs_oracle(ace, plan, cfg, xi, E_mixed, "water32") if world == 1 else None
    clocks = sampler.stop()
    t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    # one build of the whole pair list per step, over all ranks
    value = npairs * args.steps / (total_ms / 1e3)
    builds = args.steps / (total_ms / 1e3)

    # ---- roofline.  The pair passes (P1 pair product + XY forward, P2 z /
    # Coulomb / z inverse, P3 XY inverse + W accumulation) take ~90% of the
    # step and run as one pipeline: sub-batches of 32 transforms alternate over
    # two streams, so the passes overlap and the unit measured is the pipeline:
    # its algorithmic bytes (counted per 32-transform launch) over its wall time.
    hbm, peak_kind = peaks()
    kcfg = plan.config()
    variant, streams = kcfg["pair_variant"], kcfg["pair_streams"]
    vname = {1: "tile passes", 2: "transposed-plane passes", 3: "persistent pipeline kernel",
             4: "plane-kernel forward pass, tile passes after it",
             5: "plane passes on clusters of two half-plane blocks"}[variant]
    group = 32 if (variant != 3 and streams == 2) else 64  # transforms per launch (algorithmic count)
    pbg, _ = pass_bytes(n, N, batch=group)
    pipe_bytes = sum(pbg.values())  # per build, counted per launch (orbital reads and W updates included)
    share = 1.0
    if world > 1:  # this rank's shard of the pairs: its share of the transforms
        share = (stats["pair_transforms"] / args.steps) / len(pair_quads(n))
        pipe_bytes *= share
    pair_wall = stats["pair_wall_ms"] / args.steps
    # the roofline unit: 16 N bytes per pair -- the spectrum's four FP32
    # complex HBM transfers (written after the forward plane pass, read and
    # written by the Coulomb pass, read by the accumulation pass) per packed
    # transform of two pairs; orbital reads and W updates are not counted
    alg_bytes = ALG_BYTES_PER_PAIR_PER_POINT * N * npairs * share
    achieved = alg_bytes / (pair_wall / 1e3) / 1e9 if pair_wall > 0 else 0.0
    achieved_launch = pipe_bytes / (pair_wall / 1e3) / 1e9 if pair_wall > 0 else 0.0
    fwd_key = "pair_fwd_hybrid" if variant == 4 else "pair_fwd"
    # the ncu DRAM capture covers the hybrid variant's passes (column-shared
    # packing, row blocks of 4); other variants report no traffic
    traffic_step = None
    if variant == 4:
        traffic_step = (MEASURED_TRAFFIC_PER_LAUNCH[fwd_key] + MEASURED_TRAFFIC_PER_LAUNCH["pair_coulomb"] +
                        MEASURED_TRAFFIC_PER_LAUNCH["pair_inv"]) * (stats["pair_transforms"] / args.steps) / 64
    # each pass alone (one stream, 64-transform launches), timed the same way:
    # the chosen variant's passes, or the tile passes when the choice is the
    # persistent kernel (which has no separate passes)
    per_pass = None
    if world == 1:
        ps = ace.Plan(cfg["grid"], cfg["cell"], cfg["ecut"], n, "mixed", pair_streams=1,
                      pair_variant=variant if variant != 3 else 1)
        xs = torch.empty_like(psi)
        _, _, st1 = timed_steps(ps, psi, tr, xs, K, 2, 1, with_timing=True)
        ps.close()
        pb64, nl64 = pass_bytes(n, N, batch=64)
        per_pass = {}
        per_pass["variant"] = {1: "tile passes", 2: "transposed-plane passes", 3: "tile passes",
                               4: "hybrid", 5: "half-plane pairs"}[variant]
        for k in ("pair_fwd", "pair_coulomb", "pair_inv"):
            ms = st1[k + "_ms"] / 2
            per_pass[k] = {"ms_per_build": ms, "launches_per_build": nl64,
                           "algorithmic_bytes_per_launch": pb64[k] / nl64,
                           "achieved_gbs": pb64[k] / (ms / 1e3) / 1e9 if ms > 0 else 0.0,
                           "frac": (pb64[k] / (ms / 1e3) / 1e9) / hbm if ms > 0 else 0.0,
                           "traffic_per_launch": MEASURED_TRAFFIC_PER_LAUNCH[fwd_key if k == "pair_fwd" else k]
                           if variant == 4 else None}
    layout = ("one launch for all transforms" if variant == 3 else
              "32-transform sub-batches on 2 streams" if streams == 2 else "64-transform launches on one stream")
    roofline = {"bound": "hbm",
                "kernel": f"pair pipeline: P1 + P2 + P3 ({vname}), {layout}",
                "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "peak_kind": peak_kind,
                "traffic": traffic_step if world == 1 else None,
                "traffic_unit": "bytes per build (sum of the three passes' DRAM bytes from the ncu "
                "captures, scaled from 64-transform launches)",
                "algorithmic_bytes_per_build": alg_bytes,
                "algorithmic_count": "16 N bytes per pair (N = 96^3): the spectrum's four FP32 complex HBM "
                                     "transfers per packed transform of two pairs",
                "pair_wall_ms_per_build": pair_wall,
                "share_of_step": pair_wall / max(stats["total_ms"] / args.steps, 1e-9),
                "per_launch_count": {
                    "bytes_per_build": pipe_bytes, "achieved_gbs": achieved_launch, "frac": achieved_launch / hbm,
                    "count": "every distinct orbital read and W read-modify-write of each "
                             f"{group}-transform launch added to the spectrum transfers (depends on launch size)"},
                "per_pass_alone": per_pass}
    # ALU view of the same passes (the FFT/pair path is near the FP32 ridge,
    # about 6 flops per algorithmic byte): the FFT flops of every packed
    # transform -- a forward and an inverse 3D complex FFT of N points, 5 N
    # log2 N flops each, the usual count -- over the pair wall time, against
    # the FP32 peak of SMs x 128 lanes x 2 flops x the highest SM clock seen
    fft_flops = 2 * 5.0 * N * math.log2(N) * (stats["pair_transforms"] / args.steps)
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    fp32_peak = sms * 128 * 2 * mhz * 1e6 / 1e12
    alu_tflops = fft_flops / (pair_wall / 1e3) / 1e12 if pair_wall > 0 else 0.0
    roofline["alu"] = {"flops_per_build": fft_flops, "achieved_tflops": alu_tflops, "peak_tflops_fp32": fp32_peak,
                       "peak_kind": f"derived: {sms} SMs x 128 FP32 lanes x 2 x {mhz:.0f} MHz",
                       "frac": alu_tflops / fp32_peak if fp32_peak > 0 else 0.0}
    # the dominant kernel live: its launches' CUDA-event durations on the
    # stream that ran them, in the timed steps (with two streams each launch
    # shares the GPU with the other stream's passes)
    if variant != 3:
        phase_ms = {"pair_fwd": stats["pair_fwd_ms"], "pair_coulomb": stats["pair_coulomb_ms"],
                    "pair_inv": stats["pair_inv_ms"]}
        dom = max(phase_ms, key=phase_ms.get)
        live_ms = phase_ms[dom] / args.steps
        roofline["dominant_kernel_live"] = {
            "pass": dom, "ms_per_build": live_ms, "bytes_per_build_launch_count": pbg[dom],
            "achieved_gbs": pbg[dom] / (live_ms / 1e3) / 1e9 if live_ms > 0 else 0.0,
            "frac": (pbg[dom] / (live_ms / 1e3) / 1e9) / hbm if live_ms > 0 else 0.0}
    gpu_launches = int(stats["launches"]) + 0

    # ---- s-MTACE on the same workload (Section 2.4): overlap screening at the
    # rho_cut the paper uses for 32 water molecules (Table 3), then the
    # screened build; reported beside the headline, not in it
    s_mtace = None
    if world == 1:
        rho_cut = 2.5e-2
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pairs, _ = ace.ace_overlap_screen(plan, psi, rho_cut)
        ov_ms = (time.perf_counter() - t0) * 1e3  # synchronous call: host wall time
        t0 = time.perf_counter()
        pairs, _ = ace.ace_overlap_screen(plan, psi, rho_cut)
        ov_ms = min(ov_ms, (time.perf_counter() - t0) * 1e3)
        kept = int(pairs[0][-1])
        xs = torch.empty_like(psi)
        ace.ace_build(plan, psi, cfg["alpha"], pairs=pairs, xi=xs)
        sb = []
        for _ in range(2):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            _, E_s = ace.ace_build(plan, psi, cfg["alpha"], pairs=pairs, xi=xs)
            b.record()
            torch.cuda.synchronize()
            sb.append(a.elapsed_time(b))
        s_mtace = {"rho_cut": rho_cut, "overlap_screen_ms": ov_ms, "pairs_kept": kept, "pairs_all": npairs,
                   "build_ms": min(sb), "pairs_per_s": kept / (min(sb) / 1e3), "E_x": E_s,
                   "dE_x_per_atom_vs_all_pairs": abs(E_s - E_mixed) / cfg["n_atom"]}
        del xs
        # MTS (Section 2.3): an inner step applies K_0 to the occupied set (one
        # ACE apply on 128 vectors, xi's split copy made once at the outer step);
        # the exact exchange on it is a full build
        Kp = torch.empty_like(psi)
        ace.ace_apply_prepare(plan, xi)
        ace.ace_apply(plan, xi, psi, out=Kp)
        ts_ = []
        for _ in range(3):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            ace.ace_apply(plan, xi, psi, out=Kp)
            b.record()
            torch.cuda.synchronize()
            ts_.append(a.elapsed_time(b))
        s_mtace["mts_inner_apply_ms"] = min(ts_)
        s_mtace["mts_exact_over_inner"] = ms_per_step / min(ts_)
        # the same inner step replayed from a CUDA graph (an MTS loop captures
        # its inner step once: xi, the orbitals' buffer and the output stay put)
        try:
            g_ = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g_):
                ace.ace_apply(plan, xi, psi, out=Kp)
            g_.replay()
            torch.cuda.synchronize()
            ts_ = []
            for _ in range(5):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record()
                g_.replay()
                b.record()
                torch.cuda.synchronize()
                ts_.append(a.elapsed_time(b))
            del g_
            s_mtace["mts_inner_apply_ms_graph"] = min(ts_)
        except (RuntimeError, ace.AceError) as exc:  # a capture failure is reported, not fatal
            s_mtace["mts_inner_apply_ms_graph"] = None
            s_mtace["mts_inner_apply_graph_error"] = str(exc)[:200]
        del Kp
        # s'-MTACE (Sections 2.4-2.5): SCDM localisation with the density /
        # gradient pre-selection, then the overlap screen and the screened
        # build on the localised orbitals -- the whole outer step
        phi = torch.empty_like(psi)
        ace.ace_scdm(plan, psi, phi_G=phi)
        sc = []
        for _ in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, piv, _, ncand = ace.ace_scdm(plan, psi, phi_G=phi)  # synchronous call: host wall time
            sc.append((time.perf_counter() - t0) * 1e3)
        pairs_l, _ = ace.ace_overlap_screen(plan, phi, rho_cut)
        xs = torch.empty_like(psi)
        ace.ace_build(plan, phi, cfg["alpha"], pairs=pairs_l, xi=xs)
        sb = []
        for _ in range(2):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            _, E_l = ace.ace_build(plan, phi, cfg["alpha"], pairs=pairs_l, xi=xs)
            b.record()
            torch.cuda.synchronize()
            sb.append(a.elapsed_time(b))
        s_mtace["s_prime"] = {"scdm_ms": min(sc), "candidate_points": ncand, "grid_points": int(np.prod(cfg["grid"])),
                              "pairs_kept": int(pairs_l[0][-1]), "screened_build_ms": min(sb),
                              "outer_step_ms": min(sc) + ov_ms + min(sb), "E_x": E_l,
                              "dE_x_per_atom_vs_all_pairs": abs(E_l - E_mixed) / cfg["n_atom"]}
        del xs, phi

    # ---- 16 independent systems of uneven size (n_occ 32..256, 48^3..120^3
    # grids): the eager batched call, and all 16 builds captured as one CUDA
    # graph (each on its own forked stream) and replayed
    batched = None
    if world == 1:
        import gen

        systems = gen.batched_systems()
        bplans = [ace.Plan(s_["grid"], s_["cell"], s_["ecut"], len(s_["psi"]), "mixed") for s_ in systems]
        bpsi = [torch.from_numpy(s_["psi"].astype(np.complex64)).cuda() for s_ in systems]
        bsys = [dict(plan=p_, psi_G=x_, alpha=s_["alpha"]) for p_, x_, s_ in zip(bplans, bpsi, systems)]
        n_pairs_b = sum(len(s_["psi"]) * (len(s_["psi"]) + 1) // 2 for s_ in systems)
        ace.ace_build_batched(bsys)
        te = []
        for _ in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ace.ace_build_batched(bsys)  # synchronous call: host wall time
            te.append((time.perf_counter() - t0) * 1e3)
        bg = ace.BatchedBuildGraph(bsys)
        bg.replay()
        tg = []
        for _ in range(3):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            bg.launch()
            b.record()
            torch.cuda.synchronize()
            tg.append(a.elapsed_time(b))
        batched = {"systems": len(systems), "pairs": n_pairs_b, "eager_ms": min(te), "graph_ms": min(tg),
                   "pairs_per_s_graph": n_pairs_b / (min(tg) / 1e3)}
        del bg
        for p_ in bplans:
            p_.close()
        del bpsi, bsys

    # ---- the other configurations of the metric: 256 orbitals on 120^3 with
    # ten applies on 256 trials per build (an MTS outer step and its inner
    # steps), 512 localised orbitals on 160^3 with the screened pair list, and
    # the 8-orbital 32^3 case (latency)
    legs = None
    if world == 1 and not args.no_legs:
        import gen

        hbm_, _ = peaks()
        legs = {}
        c3 = gen.config_water64(n_trial_sets=10, T=256)
        legs["water64"] = workload_leg(ace, c3, "water64", hbm_, trial_sets=c3["trials"])
        del c3
        c5 = gen.config_localized()
        legs["localized"] = workload_leg(ace, c5, "localized", hbm_, pairs=c5["pairs"])
        del c5
        c1 = gen.config_small()
        legs["small"] = workload_leg(ace, c1, None, hbm_, steps=20, warmup=3,
                                     trial_sets=[gen.random_trials(c1["cell"], c1["ecut"], 8, 2)])

    # ---- the same step replayed from a CUDA graph (build + apply captured once),
    # and on the small 8-orbital / 32^3 case, where launches dominate
    graph = None
    if world == 1:
        def graph_ms(pl, ps, trs, steps):
            xg = torch.empty_like(ps)
            kg = torch.empty_like(trs)
            ace.ace_build_async(pl, ps, cfg["alpha"], xi=xg)
            ace.ace_apply(pl, xg, trs, out=kg)
            ace.ace_build_result(pl)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                ace.ace_build_async(pl, ps, cfg["alpha"], xi=xg)
                ace.ace_apply(pl, xg, trs, out=kg)
            g.replay()
            torch.cuda.synchronize()
            eager, replay = [], []
            for _ in range(steps):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record()
                ace.ace_build(pl, ps, cfg["alpha"], xi=xg)
                ace.ace_apply(pl, xg, trs, out=kg)
                b.record()
                torch.cuda.synchronize()
                eager.append(a.elapsed_time(b))
                a.record()
                g.replay()
                b.record()
                torch.cuda.synchronize()
                ace.ace_build_result(pl)
                replay.append(a.elapsed_time(b))
            del g
            return statistics.median(eager), statistics.median(replay)
        e_ms, r_ms = graph_ms(plan, psi, tr, 3)
        import gen
        small = gen.config_small()
        ps_ = ace.Plan(small["grid"], small["cell"], small["ecut"], 8, "mixed")
        psi_s = torch.from_numpy(small["psi"].astype(np.complex64)).cuda()
        tr_s = torch.from_numpy(gen.random_trials(small["cell"], small["ecut"], 8, 2).astype(np.complex64)).cuda()
        e1, r1 = graph_ms(ps_, psi_s, tr_s, 20)
        ps_.close()
        graph = {"workload_ms_eager": e_ms, "workload_ms_graph": r_ms, "workload_pairs_per_s_graph": npairs / (r_ms / 1e3),
                 "small_8orb_32cubed_ms_eager": e1, "small_8orb_32cubed_ms_graph": r1}

    # ---- end to end through the public API with host buffers
    psi_h = torch.from_numpy(cfg["psi"].astype(np.complex64)).pin_memory()
    tr_h = torch.from_numpy(my_trials.astype(np.complex64)).pin_memory()
    xi_h = torch.empty_like(psi_h).pin_memory()
    K_h = torch.empty_like(tr_h).pin_memory()
    for _ in range(1):
        psi.copy_(psi_h, non_blocking=True)
        xi, _ = build(plan, psi, xi)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        psi.copy_(psi_h, non_blocking=True)
        tr.copy_(tr_h, non_blocking=True)
        xi, _ = build(plan, psi, xi)
        ace.ace_apply(plan, xi, tr, out=K)
        xi_h.copy_(xi, non_blocking=True)
        K_h.copy_(K, non_blocking=True)
        b.record()
        torch.cuda.synchronize()
        e2e_ms += a.elapsed_time(b)
    t = torch.tensor([e2e_ms], dtype=torch.float64, device="cuda")
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e2e_ms = float(t.item())
    h2d = psi_h.numel() * 8 + tr_h.numel() * 8
    d2h = xi_h.numel() * 8 + K_h.numel() * 8 + 8
    e2e = {"value": npairs * args.steps / (e2e_ms / 1e3), "unit": "pairs/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
    plan.close()
    del psi, tr, xi, K

    # ---- plain FP64 GPU form of the same step (comparison point of the metric)
    fp64 = None
    if not args.no_fp64:
        p64, psi64, tr64, xi64, K64 = setup("fp64")
        t64, E64, _ = timed_steps(p64, psi64, tr64, xi64, K64, 1, 1)
        if world > 1:
            import torch.distributed as dist
            t = torch.tensor([t64], dtype=torch.float64, device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            t64 = float(t.item())
        fp64 = {"pairs_per_s": npairs / (t64 / 1e3), "builds_per_s": 1e3 / t64, "ms_per_step": t64,
                "E_x": E64, "dE_x_per_atom_mixed_vs_fp64": abs(E_mixed - E64) / cfg["n_atom"]}
        p64.close()
        del psi64, tr64, xi64, K64

    if rank != 0:
        return
    cb = None if args.no_cpu_baseline or world > 1 else cpu_baseline(cfg)
    line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "mixed (FP32 FFT/pairs/W, FP64 M/Cholesky/xi/E_x)",
                       "apply_trials": int(trials.shape[0]), "l2": "flushed between timed steps",
                       "parallelism": f"pair shards over {world} GPUs, W_G/E_x allreduce (NCCL)" if world > 1
                       else "single GPU",
                       "pair_kernels": kcfg},
            "ace_builds_per_s": builds, "E_x": E_mixed, "fp64_gpu": fp64,
            "phases_ms_per_step": {k: v / args.steps for k, v in stats.items() if k.endswith("_ms")},
            "s_mtace": s_mtace, "cuda_graph": graph, "batched_16_systems": batched,
            "roofline": roofline, "cpu_baseline": cb, "e2e": e2e, "gpu_launches": gpu_launches,
            "parity_vs_oracle": parity, "workloads": legs,
            "clocks": clocks}
    print(json.dumps(line), flush=True)


def profile_case(n_occ, batch=64, pair_variant=1, pair_streams=1):
    """One small ACE build on the 96^3 workload grid (n_occ orbitals): the
    case the ncu captures under profiles/ run."""
    import torch

    import gen
    import paper_2110_07670_gb300 as ace
    psi, _ = gen.water_orbitals(18.6, 80.0, n_occ, 2)
    plan = ace.Plan((96, 96, 96), gen.cubic_cell(18.6), 80.0, n_occ, "mixed", pair_batch=batch,
                    pair_variant=pair_variant, pair_streams=pair_streams)
    xi, E = ace.ace_build(plan, torch.from_numpy(psi.astype(np.complex64)).cuda(), 0.25)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": n_occ, "E_x": E}))


def profile_overlap(n_occ, reps=3):
    """The s-MTACE overlap screen (Section 2.4) of the first n_occ of the 128
    water-box orbitals on the 96^3 grid: the |phi| Gram on tcgen05 that the
    ncu captures under profiles/ run."""
    import torch

    import gen
    import paper_2110_07670_gb300 as ace
    psi, _ = gen.water_orbitals(18.6, 80.0, 128, 2)
    plan = ace.Plan((96, 96, 96), gen.cubic_cell(18.6), 80.0, n_occ, "mixed", pair_variant=1)
    d = torch.from_numpy(psi[:n_occ].astype(np.complex64)).cuda()
    for _ in range(reps):
        t0 = time.perf_counter()
        pairs, _ = ace.ace_overlap_screen(plan, d, 2.5e-2)
        ms = (time.perf_counter() - t0) * 1e3
    print(json.dumps({"profile_overlap": n_occ, "pairs_kept": int(pairs[0][-1]), "ms": ms}))


def profile_scdm(which, reps=2):
    """SCDM localisation with the s'-MTACE pre-selection (Sections 2.4-2.5) on
    the 128 water-box orbitals on 96^3 ("water32") or the 512 localised
    orbitals on 160^3 ("localized"): the kernels the SCDM launch lists under
    profiles/ cover (the first call allocates, the last is the one to read)."""
    import torch

    import gen
    import paper_2110_07670_gb300 as ace
    cfg = gen.config_water32() if which == "water32" else gen.config_localized()
    n = len(cfg["psi"])
    plan = ace.Plan(cfg["grid"], cfg["cell"], cfg["ecut"], n, "mixed", pair_variant=1)
    d = torch.from_numpy(cfg["psi"].astype(np.complex64)).cuda()
    phi = torch.empty_like(d)
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, piv, _, ncand = ace.ace_scdm(plan, d, phi_G=phi)
        ms = (time.perf_counter() - t0) * 1e3
    print(json.dumps({"profile_scdm": which, "n_occ": n, "grid": list(cfg["grid"]), "candidates": ncand, "ms": ms}))


def profile_apply(T, reps=3):
    """ACE applies on T random trials with 256 random ACE vectors in the
    120^3 / 23.5-bohr / 80 Ry basis (78398 plane waves): the tensor-core Gram
    and the apply product the ncu captures under profiles/ run."""
    import torch

    import gen
    import paper_2110_07670_gb300 as ace
    cell = gen.cubic_cell(23.5)
    plan = ace.Plan((120, 120, 120), cell, 80.0, 256, "mixed")
    rng = np.random.default_rng(1)
    npw = plan.n_pw_half
    xi = (rng.standard_normal((256, npw)) + 1j * rng.standard_normal((256, npw))) / np.sqrt(npw)
    xi[:, 0] = xi[:, 0].real
    tr = gen.random_trials(cell, 80.0, T, 2)
    d_xi = torch.from_numpy(xi.astype(np.complex64)).cuda()
    d_tr = torch.from_numpy(tr.astype(np.complex64)).cuda()
    out = torch.empty_like(d_tr)
    ace.ace_apply_prepare(plan, d_xi)  # xi's split copy, as at an outer MTS step
    for _ in range(reps):
        ace.ace_apply(plan, d_xi, d_tr, out=out)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ace.ace_get_stats(plan)
    ace.ace_set_timing(plan, True)
    a.record()
    ace.ace_apply(plan, d_xi, d_tr, out=out)
    b.record()
    torch.cuda.synchronize()
    st = ace.ace_get_stats(plan)
    print(json.dumps({"profile_apply": T, "apply_ms": a.elapsed_time(b), "gram_ms": st["gram_ms"],
                      "product_ms": st["xi_ms"]}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-legs", action="store_true", help="skip the 120^3, 160^3 and 32^3 workloads")
    ap.add_argument("--profile-case", type=int, default=0, help="run one small build with this many orbitals")
    ap.add_argument("--profile-apply", type=int, default=0, help="run ACE applies on this many trial vectors")
    ap.add_argument("--profile-overlap", type=int, default=0, help="run the overlap screen on this many orbitals")
    ap.add_argument("--profile-scdm", default=None, choices=["water32", "localized"],
                    help="run SCDM localisation on this workload")
    ap.add_argument("--pair-variant", type=int, default=None,
                    help="pair-pass kernels (1-4); default: autotuned, and 1 for --profile-case")
    ap.add_argument("--pair-streams", type=int, default=1, help="pair streams of --profile-case")
    args = ap.parse_args()
    if args.profile_case:
        profile_case(args.profile_case, pair_variant=args.pair_variant or 1, pair_streams=args.pair_streams)
        return
    if args.profile_scdm:
        profile_scdm(args.profile_scdm)
        return
    if args.profile_overlap:
        profile_overlap(args.profile_overlap)
        return
    if args.profile_apply:
        profile_apply(args.profile_apply)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)
    if int(os.environ.get("WORLD_SIZE", 1)) > 1:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
