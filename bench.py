#!/usr/bin/env python
"""Benchmark of the Proportional Similarity hot path on one GB300 per rank.

Default workload: 2-way metrics over all pairs of nv=32768 vectors of nf=8192
FP32 fields (seeded zero-inflated -log10 p-value stand-ins), packed FP32
upper-triangular output.  A step is one full pass of the path: FP64 vector
sums + the FP32 min-product kernel with the fused ratio epilogue.

Metric: elementwise comparisons per second (one comparison = one min plus one
add per element pair, the paper's count).  Prints ONE JSON line on rank 0.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Multi-GPU (torchrun): by default the ranks share ONE instance, each
computing the equal-work part ps_partition gives it (the paper's split of
the vector axis, Section 4.1; V replicated, outputs sharded, no collective
on the data path); value = the instance's comparisons / max-over-ranks time
("scaling": "strong").  --scaling weak runs one independent instance per
rank (seed + rank) instead.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "elementwise comparisons/sec (2-way, 3-way) at 1 GB300; % of min+add peak; INT8-TC vs FP32"
UNIT = "comparisons/s"
WORKLOADS = {
    "2way_32768x8192_f32": dict(way=2, nv=32768, nf=8192, number=2),
    "3way_2048x4096_f32": dict(way=3, nv=2048, nf=4096, number=3),
    "2way_1024x512_f64": dict(way=2, nv=1024, nf=512, number=1),
    # small cases of the same kernels for profiler captures
    "2way_8192x8192_f32": dict(way=2, nv=8192, nf=8192, number=2),
    "3way_1024x4096_f32": dict(way=3, nv=1024, nf=4096, number=3),
    # output-bound shapes (few fields), and a small one for profiler captures
    "2way_16384x16_f32": dict(way=2, nv=16384, nf=16, number=2),
    "2way_32768x16_f32": dict(way=2, nv=32768, nf=16, number=2),
    "2way_32768x64_f32": dict(way=2, nv=32768, nf=64, number=2),
    "2way_32768x385_f32": dict(way=2, nv=32768, nf=385, number=2),
    # the single-GPU kernel timing of the paper's Table 1 (n_v = 10,240, n_f = 12,288)
    "2way_10240x12288_f32": dict(way=2, nv=10240, nf=12288, number=2),
}
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")


def comparisons(w):
    nv, nf = w["nv"], w["nf"]
    if w["way"] == 2:
        return nf * nv * (nv - 1) // 2
    return nf * nv * (nv - 1) * (nv - 2) // 6


def packed_pair_index(nv, i, j):
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    return i * (2 * nv - i - 1) // 2 + (j - i - 1)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = os.path.join("/tmp", f"ps_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# DRAM traffic per launch from a committed ncu summary, valid while the
# kernel's sources hash to the value recorded with the capture.
TRAFFIC = {
    "mgemm2": ("profiles/mgemm2_2way_32768x8192_dram.md",
               ["paper_1705_08210_gb300/csrc/ps_mgemm_impl.cuh", "paper_1705_08210_gb300/csrc/ps_mgemm_tma.cu",
                "paper_1705_08210_gb300/csrc/ps_sync.cuh"]),
    "thermo_gemm": ("profiles/thermo_gemm_2way_32768x8192_dram.md",
                    ["paper_1705_08210_gb300/csrc/ps_thermo.cu", "paper_1705_08210_gb300/csrc/ps_sync.cuh"]),
}


def sources_sha256(paths):
    import hashlib
    hsh = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            hsh.update(f.read())
    return hsh.hexdigest()


def profiled_traffic(kernel, workload):
    """Bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of
    `kernel` on `workload`, or None when no capture matches the current
    sources."""
    if kernel not in TRAFFIC:
        return None
    summary, srcs = TRAFFIC[kernel]
    path = os.path.join(ROOT, summary)
    if not os.path.exists(path):
        return None
    rec = {}
    for line in open(path):
        if ":" in line and line.strip().startswith(("traffic_bytes_per_launch", "source_sha256", "workload")):
            k, v = line.strip().split(":", 1)
            rec[k.strip()] = v.strip()
    if rec.get("workload") != workload or rec.get("source_sha256") != sources_sha256(srcs):
        return None
    return float(rec["traffic_bytes_per_launch"]) / 1e9


def cpu_baseline(V_fm: np.ndarray, w, n_sample: int):
    """The plain FP64 oracle on the first n_sample vectors, all host cores."""
    import oracle
    nf = V_fm.shape[0]
    sub = np.ascontiguousarray(V_fm[:, :n_sample].T).astype(np.float64)
    t0 = time.perf_counter()
    if w["way"] == 2:
        oracle.c2_packed(sub)
        cmp = nf * n_sample * (n_sample - 1) // 2
        what = f"c2 over all pairs of the first {n_sample} vectors ({cmp:.3e} comparisons)"
    else:
        oracle.c3_slab(sub, 0, n_sample)
        cmp = nf * n_sample * (n_sample - 1) * (n_sample - 2) // 6
        what = f"c3 over all triples of the first {n_sample} vectors ({cmp:.3e} comparisons)"
    dt = time.perf_counter() - t0
    return {"value": cmp / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": what, "seconds": round(dt, 3)}


def sampled_parity(V_fm: np.ndarray, samples):
    """The second half of the CPU-baseline leg: the FP64 oracle on the sampled
    outputs the GPU sections recorded (pairs, triples, or all pairs of the
    first vectors), with the relative (or absolute) error of each."""
    import oracle
    Vv = None
    res = {}
    for name, (kind, sel, got) in samples.items():
        if kind == "pairs":
            Vv = oracle.to_vector_major(V_fm) if Vv is None else Vv
            ref = oracle.c2_pairs(Vv, sel)
        elif kind == "triples":
            Vv = oracle.to_vector_major(V_fm) if Vv is None else Vv
            ref = oracle.c3_triples(Vv, sel)
        else:
            ref = oracle.c2_packed(oracle.to_vector_major(V_fm[:, :sel]))
        if kind == "first":
            e = np.abs(got - ref)
            res[name] = {"sample": f"all {ref.size} pairs of the first {sel} vectors", "max_abs": float(e.max()),
                         "mean_abs": float(e.mean()), "p99_abs": float(np.percentile(e, 99))}
        else:
            nz = ref != 0
            r = np.abs(got[nz] - ref[nz]) / ref[nz] if nz.any() else np.zeros(1)
            res[name] = {"sample": f"{len(sel)} random {kind}", "max_rel": float(r.max()),
                         "mean_rel": float(r.mean())}
    return res


def run_reference(args, w, ws, rank):
    """--impl reference: the FP64 CPU oracle, timed as it stands."""
    if rank != 0:
        return
    from paper_1705_08210_gb300 import synth
    n_sample = min(2048 if w["way"] == 2 else 128, w["nv"])
    V = synth.zero_inflated(n_sample, w["nf"], synth.seed_for(w["number"]))
    times = []
    cb = None
    for s in range(args.warmup + args.steps):
        cb = cpu_baseline(V, w, n_sample)
        if s >= args.warmup:
            times.append(cb["seconds"])
    cmp = cb["value"] * cb["seconds"]
    ms = 1e3 * statistics.mean(times)
    value = cmp / (ms / 1e3)
    cb["value"] = value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "nv": w["nv"], "nf": w["nf"],
                       "sample_vectors": n_sample, "l2": "CPU run"},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batched_section(ps, synth, h, torch, sptr, peak_cmp, steps=3):
    """The 64 uneven instances (48 2-way with nv ~ U[256, 4096], 16 3-way with
    nv ~ U[256, 1024], nf ~ U[512, 8192], FP32) in one persistent launch
    replayed from a CUDA graph, against one call per instance; the kernel
    variant is the autotuner's choice for this batch shape."""
    shapes = synth.batched_shapes(synth.seed_for(4))
    keep, probs = [], (ps.ps_problem * len(shapes))()
    cmp_total = 0
    for t, (way, nv, nf) in enumerate(shapes):
        V = synth.zero_inflated(nv, nf, synth.seed_for(4, 1 + t))
        ld = (nv + 3) // 4 * 4
        Xp = torch.zeros((nf, ld), dtype=torch.float32, device="cuda")
        Xp[:, :nv] = torch.from_numpy(V).cuda()
        n = nv * (nv - 1) // 2 if way == 2 else ps.ps_slab_size(nv, 0, nv)
        out = torch.empty(n, dtype=torch.float32, device="cuda")
        probs[t].V = ps.matrix(Xp[:, :nv])
        probs[t].way = way
        probs[t].out_dtype = ps.PS_F32
        probs[t].out = out.data_ptr()
        keep.append((Xp, out))
        cmp_total += nf * (nv * (nv - 1) // 2 if way == 2 else nv * (nv - 1) * (nv - 2) // 6)
    choice = ctypes.create_string_buffer(256)
    t0 = time.perf_counter()
    ps.check(ps.ps_autotune_batched(h.h, probs, len(shapes), None, choice, 256, sptr), h.h)
    t_tune = time.perf_counter() - t0
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    res = {}
    for name, mode in (("persistent_graph", ps.PS_BATCH_PERSISTENT), ("per_instance", ps.PS_BATCH_PER_INSTANCE)):
        for _ in range(2):
            ps.check(ps.ps_metrics_batched(h.h, probs, len(shapes), mode, sptr), h.h)
        torch.cuda.synchronize()
        e0.record(torch.cuda.current_stream())
        for _ in range(steps):
            ps.check(ps.ps_metrics_batched(h.h, probs, len(shapes), mode, sptr), h.h)
        e1.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        res[name] = {"ms_per_batch": ms, "value": cmp_total / (ms / 1e3), "unit": UNIT,
                     "frac_of_alu_peak": cmp_total / (ms / 1e3) / peak_cmp}
    del keep, probs
    torch.cuda.empty_cache()
    n2 = sum(1 for w, _, _ in shapes if w == 2)
    return {"workload": f"64 uneven instances ({n2} 2-way nv~U[256,4096], {64 - n2} 3-way nv~U[256,1024], "
                        "nf~U[512,8192], FP32)",
            "comparisons_per_batch": cmp_total, **res,
            "speedup_persistent_vs_per_instance": res["per_instance"]["ms_per_batch"]
            / res["persistent_graph"]["ms_per_batch"],
            "autotuner_choice": choice.value.decode(), "autotune_seconds": t_tune,
            "timing": "CUDA events on the launching stream around each whole batched call (the persistent "
                      "call includes its error-flag read back)"}


def threshold_section(ps, synth, h, torch, sptr, peak_cmp):
    """Exhaustive vs learned vs bound-filtered thresholded 3-way search on
    8192 x 2048 vectors from 64 latent profiles (sigma 0.4), tau = 0.7.

    The encoder is trained on 8 fresh 1024-vector matrices drawn from the
    same latent-profile population (the same 64 profiles, new profile
    assignments, scales and noise: none of the searched vectors), labelled by
    the exact thresholded search, 1500 Adam steps.  A second line trains on 8
    random 1024-vector subsets of the searched matrix itself."""
    nv, nf, tau = 8192, 2048, 0.7
    pseed = synth.seed_for(5)
    V, _ = synth.latent_profiles(nv, nf, pseed, n_profiles=64, sigma=0.4)
    X = torch.from_numpy(V).cuda()
    m = ps.matrix(X)
    cap = 20_000_000
    out = torch.empty((cap, 4), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")

    def run(mode):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ps.check(ps.ps_threshold_3way(h.h, ctypes.byref(m), tau, mode, out.data_ptr(), cap, cnt.data_ptr(),
                                      sptr), h.h)
        dt = time.perf_counter() - t0
        kept = ctypes.c_double()
        nb = ctypes.c_int64()
        ps.check(ps.ps_proposal_last_stats(h.h, ctypes.byref(kept), ctypes.byref(nb)), h.h)
        n = int(cnt.item())
        keys = out[:n, :3].to(torch.int64)
        return dt, n, (keys[:, 0] << 42) | (keys[:, 1] << 21) | keys[:, 2], out[:n, 3].clone(), kept.value

    def train(mats_np, label):
        subs = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in mats_np]
        mats = (ps.ps_matrix * len(subs))(*[ps.matrix(x) for x in subs])
        loss = ctypes.c_double()
        ps.check(ps.ps_proposal_init(h.h, nf, 99), h.h)
        ps.check(ps.ps_timing_enable(h.h, 1), h.h)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ps.check(ps.ps_proposal_train(h.h, mats, len(subs), tau, 1500, 1e-3, 0.995, 99, ctypes.addressof(loss),
                                      sptr), h.h)
        t_train = time.perf_counter() - t0
        n_l, ms_l, n_s, ms_s = ctypes.c_int64(), ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
        ps.check(ps.ps_timing_read(h.h, b"proposal_labels", ctypes.byref(n_l), ctypes.byref(ms_l)), h.h)
        ps.check(ps.ps_timing_read(h.h, b"proposal_steps", ctypes.byref(n_s), ctypes.byref(ms_s)), h.h)
        ps.check(ps.ps_timing_enable(h.h, 0), h.h)
        t_l, n_found, k_l, v_l, kept_l = run(1)
        found = torch.isin(k_l, k_ex)
        exact_vals = bool(torch.equal(v_l, v_ex[torch.isin(k_ex, k_l)]))
        recall = float(found.sum().item()) / max(n_ex, 1)
        del subs
        return {"training_data": label, "train_seconds": t_train, "train_loss": loss.value,
                "train_breakdown": {"exact_label_search_s": ms_l.value / 1e3, "label_searches": n_l.value,
                                    "adam_steps_s": ms_s.value / 1e3, "steps": 1500,
                                    "other_s": t_train - (ms_l.value + ms_s.value) / 1e3},
                "search_seconds": t_l, "triples": n_found, "recall": recall,
                "values_bit_identical": exact_vals, "blocks_searched": kept_l,
                "speedup_search": t_ex / t_l, "speedup_incl_training": t_ex / (t_l + t_train)}

    t_ex, n_ex, k_ex, v_ex, _ = run(0)
    fresh = [synth.latent_profiles(1024, nf, synth.seed_for(5, 100 + t), n_profiles=64, sigma=0.4,
                                   profile_seed=pseed)[0] for t in range(8)]
    held_out = train(fresh, "8 fresh 1024-vector matrices from the same 64 latent profiles (new assignments, "
                            "scales and noise; no searched vector)")
    rng = np.random.default_rng(170508210)
    subsets = [V[:, np.sort(rng.choice(nv, 1024, replace=False))] for _ in range(8)]
    subset = train(subsets, "8 random 1024-vector subsets of the searched matrix")
    t_b, n_b, k_b, v_b, kept_b = run(2)
    exact_b = n_b == n_ex and bool(torch.equal(k_b, k_ex)) and bool(torch.equal(v_b, v_ex))
    del out, X
    torch.cuda.empty_cache()
    return {"workload": "3way threshold 8192x2048 f32, 64 latent profiles, sigma 0.4, tau 0.7",
            "comparisons_exhaustive": nf * nv * (nv - 1) * (nv - 2) // 6,
            "exhaustive": {"seconds": t_ex, "triples": n_ex,
                           "cmp_per_s": nf * nv * (nv - 1) * (nv - 2) // 6 / t_ex,
                           "frac_of_alu_peak": nf * nv * (nv - 1) * (nv - 2) // 6 / t_ex / peak_cmp},
            "learned": held_out, "learned_subset_training": subset,
            "bound_lossless": {"search_seconds": t_b, "triples": n_b, "identical_to_exhaustive": exact_b,
                               "blocks_searched": kept_b, "speedup": t_ex / t_b}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="2way_32768x8192_f32", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-secondary", action="store_true")
    ap.add_argument("--no-thermo", action="store_true")
    ap.add_argument("--no-threshold", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--scaling", default="strong", choices=["strong", "weak"],
                    help="with N > 1 ranks: strong = the ranks share one instance (ps_partition's equal-work "
                         "parts, no collective on the data path); weak = one independent instance per rank")
    ap.add_argument("--ps-config", default="",
                    help="kernel choices for the handle, as ps_config fields: name=value[,name=value...] "
                         "(e.g. tma_schedule=2,tma_meet=32); default: every choice automatic")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, w, ws, rank)
        return

    import torch
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1705_08210_gb300 import ps, synth

    fields = {}
    for item in filter(None, args.ps_config.split(",")):
        k, v = item.split("=", 1)
        fields[k.strip()] = int(v)
    h = ps.Handle(local, **fields)
    nv, nf = w["nv"], w["nf"]
    dtype = np.float64 if args.workload.endswith("f64") else np.float32
    strong = ws > 1 and args.scaling == "strong"
    # strong scaling: every rank holds the same instance and computes its
    # part; weak scaling: rank r computes its own instance (seed + r)
    V = synth.zero_inflated(nv, nf, synth.seed_for(w["number"], 0 if strong else rank), dtype=dtype)
    X = torch.from_numpy(V).cuda()
    m = ps.matrix(X)
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    # this rank's share of the unique outputs (the whole instance unless strong)
    pb, pe, ob, oe = (ctypes.c_int64() for _ in range(4))
    ps.check(ps.ps_partition(nv, w["way"], ws if strong else 1, rank if strong else 0, ctypes.byref(pb),
                             ctypes.byref(pe), ctypes.byref(ob), ctypes.byref(oe)))
    if w["way"] == 2:
        out_dtype = 1 if dtype == np.float64 else 0
        out = torch.empty(nv * (nv - 1) // 2, dtype=torch.float64 if out_dtype else torch.float32, device="cuda")
        main_kernel = "mgemm2"
        # vector sums, (the small-n_f epilogue's sums and range words,) min-product
        launches_per_step = 2 + (1 if nf <= 256 and dtype == np.float32 else 0)
        rows = range(pb.value, pe.value)
        cmp_mine = nf * sum(nv - 1 - i for i in rows) if strong else None

        if strong:
            def step():
                ps.check(ps.ps_metrics_2way_part(h.h, ctypes.byref(m), ws, rank, out.data_ptr(), out_dtype, sptr),
                         h.h)
        else:
            def step():
                ps.check(ps.ps_metrics_2way(h.h, ctypes.byref(m), ps.PS_PATH_FP32, 0, out.data_ptr(), out_dtype,
                                            sptr), h.h)
    else:
        jb, je = pb.value, pe.value
        out = torch.empty(max(ps.ps_slab_size(nv, jb, je), 1), dtype=torch.float32, device="cuda")
        main_kernel = "mgemm3"
        launches_per_step = 5  # sums, n2 table, pivot prefix, item table, 3-way
        cmp_mine = nf * ps.ps_slab_size(nv, jb, je) if strong else None

        def step():
            ps.check(ps.ps_metrics_3way(h.h, ctypes.byref(m), jb, je, out.data_ptr(), sptr), h.h)

    out_bytes = out.numel() * out.element_size()
    cmp_per_step = comparisons(w)
    # comparisons this rank's kernel makes per step (for its roofline)
    cmp_rank = cmp_mine if strong else cmp_per_step
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- device-timed region ----
    ps.check(ps.ps_timing_enable(h.h, 1), h.h)
    clocks = ClockSampler(local)
    clocks.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    n_launch = ctypes.c_int64()
    k_ms = ctypes.c_double()
    ps.check(ps.ps_timing_read(h.h, main_kernel.encode(), ctypes.byref(n_launch), ctypes.byref(k_ms)), h.h)
    ps.check(ps.ps_timing_enable(h.h, 0), h.h)
    if ws > 1:
        t = torch.tensor([ms_total], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_total = float(t.item())
    ms_step = ms_total / args.steps
    # whole-job comparisons per second: one shared instance (strong) or one
    # instance per rank (weak), over the slowest rank's time
    value = (cmp_per_step if strong else ws * cmp_per_step) / (ms_step / 1e3)

    # ---- roofline of the dominant kernel ----
    k_avg_ms = k_ms.value / max(n_launch.value, 1)
    achieved = cmp_rank / (k_avg_ms / 1e3)
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    props = torch.cuda.get_device_properties(local)
    n_sm = props.multi_processor_count
    # ALU-pipe bound of the inner loop: FP32 min (FMNMX) executes on the ALU
    # pipe at 16 lanes per clock per SM sub-partition (two pipe cycles per
    # warp instruction, measured with ncu), so an SM retires at most
    # 4 x 16 = 64 comparisons per clock whatever the add form; the adds run on
    # the FMA pipe in parallel.
    peak_cmp = n_sm * 64 * sm_max * 1e6
    probe = ctypes.c_double()
    ps.check(ps.ps_probe_minadd_peak(h.h, 1, ctypes.byref(probe)), h.h)
    probe0 = ctypes.c_double()
    ps.check(ps.ps_probe_minadd_peak(h.h, 0, ctypes.byref(probe0)), h.h)
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_cmp / 1e12, "unit": "Tcmp/s",
                "frac": achieved / peak_cmp, "traffic": profiled_traffic(main_kernel, args.workload),
                "traffic_unit": "GB per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                "algorithmic_bytes": (V.nbytes + out_bytes) / 1e9,
                "kernel": main_kernel, "kernel_ms": k_avg_ms,
                "peak_basis": f"{n_sm} SMs x 64 FP32 min lanes/clock (ALU pipe) x {sm_max:.0f} MHz max clock",
                "probe_minadd_f32x2": probe.value / 1e12, "probe_minadd_scalar": probe0.value / 1e12}

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        Vh = torch.from_numpy(V).pin_memory()
        mh = ps.matrix(Vh)
        if w["way"] == 2 and strong:
            # the part call writes device memory: copy V in and this rank's
            # packed range out around it (inside the timed region)
            outh = torch.empty(oe.value - ob.value, dtype=out.dtype).pin_memory()

            def hstep():
                X.copy_(Vh, non_blocking=True)
                ps.check(ps.ps_metrics_2way_part(h.h, ctypes.byref(m), ws, rank, out.data_ptr(), out_dtype, sptr),
                         h.h)
                outh.copy_(out[ob.value:oe.value], non_blocking=True)
                torch.cuda.current_stream().synchronize()
        elif w["way"] == 2:
            outh = torch.empty(out.numel(), dtype=out.dtype).pin_memory()

            def hstep():
                ps.check(ps.ps_metrics_2way(h.h, ctypes.byref(mh), ps.PS_PATH_FP32, 0, outh.data_ptr(),
                                            out_dtype, sptr), h.h)
        else:
            outh = torch.empty(out.numel(), dtype=out.dtype).pin_memory()

            def hstep():
                ps.check(ps.ps_metrics_3way(h.h, ctypes.byref(mh), jb, je, outh.data_ptr(), sptr), h.h)
        hstep()
        if ws > 1:
            torch.distributed.barrier()
        # (the library's event pairs around the min-product launches: the
        # kernel's share of the end-to-end step)
        ps.check(ps.ps_timing_enable(h.h, 1), h.h)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            hstep()
        dt = (time.perf_counter() - t0) / args.steps
        n_e, k_e = ctypes.c_int64(), ctypes.c_double()
        ps.check(ps.ps_timing_read(h.h, (b"mgemm3" if w["way"] == 3 else b"mgemm2"), ctypes.byref(n_e),
                                   ctypes.byref(k_e)), h.h)
        ps.check(ps.ps_timing_enable(h.h, 0), h.h)
        # one plain copy of the step's input from the same pinned buffer
        Vd = torch.empty(Vh.shape, dtype=Vh.dtype, device="cuda")
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        Vd.copy_(Vh, non_blocking=True)
        c0.record()
        Vd.copy_(Vh, non_blocking=True)
        c1.record()
        torch.cuda.synchronize()
        h2d_ms = c0.elapsed_time(c1)
        del Vd
        if ws > 1:
            t = torch.tensor([dt], device="cuda", dtype=torch.float64)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            dt = float(t.item())
        e2e = {"value": (cmp_per_step if strong else ws * cmp_per_step) / dt, "unit": UNIT, "ms_per_step": dt * 1e3,
               "kernel_ms_per_step": k_e.value / args.steps, "h2d_copy_ms": h2d_ms,
               "h2d_bytes_per_step": int(Vh.numel() * Vh.element_size()),
               "d2h_bytes_per_step": int(outh.numel() * outh.element_size())}
        if w["way"] == 2 and ws == 1:
            # the same call with one-byte metric codes (PS_U8) as the output
            outu = torch.empty(out.numel(), dtype=torch.uint8).pin_memory()

            def ustep():
                ps.check(ps.ps_metrics_2way(h.h, ctypes.byref(mh), ps.PS_PATH_FP32, 0, outu.data_ptr(),
                                            ps.PS_U8, sptr), h.h)
            ustep()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                ustep()
            du = (time.perf_counter() - t0) / args.steps
            e2e["u8_codes"] = {"value": cmp_per_step / du, "unit": UNIT, "ms_per_step": du * 1e3,
                               "d2h_bytes_per_step": int(outu.numel())}
            del outu
        del Vh, outh

    # ---- sampled outputs of the timed run (checked in the CPU-baseline leg) ----
    samples = {}
    torch.cuda.synchronize()
    if w["way"] == 2:
        pairs = synth.sample_pairs(nv, 2000, seed=11)
        idx = torch.from_numpy(packed_pair_index(nv, pairs[:, 0], pairs[:, 1])).cuda()
        samples["fp32"] = ("pairs", pairs, out[idx].double().cpu().numpy())
    else:
        t3 = synth.sample_triples(nv, 2000, seed=11)
        F = lambda x: (nv - 1) * (x * (x - 1) // 2) - (x - 1) * x * (2 * x - 1) // 6  # noqa: E731
        pos = F(t3[:, 1]) + t3[:, 0] * (nv - 1 - t3[:, 1]) + (t3[:, 2] - t3[:, 1] - 1)
        samples["fp32"] = ("triples", t3, out[torch.from_numpy(pos).cuda()].double().cpu().numpy())

    # ---- packed half2 variant on the same input (2-way only) ----
    half2 = None
    if not args.no_thermo and w["way"] == 2 and ws == 1:
        def hstep2():
            ps.check(ps.ps_metrics_2way(h.h, ctypes.byref(m), ps.PS_PATH_HALF2, 0, out.data_ptr(), out_dtype,
                                        sptr), h.h)
        for _ in range(2):
            hstep2()
        torch.cuda.synchronize()
        ps.check(ps.ps_timing_enable(h.h, 1), h.h)
        e0.record(stream)
        for _ in range(args.steps):
            hstep2()
        e1.record(stream)
        torch.cuda.synchronize()
        hms = e0.elapsed_time(e1) / args.steps
        ps.check(ps.ps_timing_read(h.h, b"mgemm2_half", ctypes.byref(n_launch), ctypes.byref(k_ms)), h.h)
        hk = k_ms.value / max(n_launch.value, 1)
        ps.check(ps.ps_timing_enable(h.h, 0), h.h)
        torch.cuda.synchronize()
        samples["half2"] = ("pairs", pairs, out[idx].double().cpu().numpy())
        # its own peak: the measured register-only rate of its inner
        # operation (one packed FP16 min for two comparisons, two FP32 adds of
        # its halves; ps_probe_minadd_peak variant 2)
        probe_h = ctypes.c_double()
        ps.check(ps.ps_probe_minadd_peak(h.h, 2, ctypes.byref(probe_h)), h.h)
        hach = cmp_per_step / (hk / 1e3)
        half2 = {"value": cmp_per_step / (hms / 1e3), "unit": UNIT, "ms_per_step": hms, "kernel_ms": hk,
                 "speedup_vs_fp32": ms_step / hms,
                 "roofline": {"bound": "alu", "achieved": hach / 1e12, "peak": probe_h.value / 1e12,
                              "unit": "Tcmp/s", "frac": hach / probe_h.value,
                              "peak_basis": "measured register-only rate of min.f16x2 + 2 FP32 adds "
                                            "(ps_probe_minadd_peak variant 2)"},
                 "sampled_error": None,
                 "note": "FP16-rounded inputs (power-of-two scaled), min.f16x2, FP32 accumulation"}

    # ---- thermometer tensor-core path on the same input (2-way only) ----
    thermo = None
    if not args.no_thermo and w["way"] == 2 and ws == 1:
        L = 16
        def tstep():
            ps.check(ps.ps_metrics_2way(h.h, ctypes.byref(m), ps.PS_PATH_THERMO, L, out.data_ptr(), out_dtype,
                                        sptr), h.h)
        for _ in range(2):
            tstep()
        torch.cuda.synchronize()
        ps.check(ps.ps_timing_enable(h.h, 1), h.h)
        e0.record(stream)
        for _ in range(args.steps):
            tstep()
        e1.record(stream)
        torch.cuda.synchronize()
        tms = e0.elapsed_time(e1) / args.steps
        kt = {}
        for name in ("quantize", "thermo_encode", "thermo_gemm"):
            ps.check(ps.ps_timing_read(h.h, name.encode(), ctypes.byref(n_launch), ctypes.byref(k_ms)), h.h)
            kt[name] = k_ms.value / max(n_launch.value, 1)
        ps.check(ps.ps_timing_enable(h.h, 0), h.h)
        flops = 2.0 * nf * (L - 1) * (nv * (nv - 1) // 2)
        fp8_peak = 2.0 * float(peaks.get("bf16_tflops", 1900.0)) * 1e12
        tach = flops / (kt["thermo_gemm"] / 1e3)
        # quantization error against the FP64 oracle on the original values,
        # all pairs of the first 4096 vectors
        ns = 4096
        ii = np.concatenate([np.full(ns - 1 - i, i) for i in range(ns - 1)])
        jj = np.concatenate([np.arange(i + 1, ns) for i in range(ns - 1)])
        gq = out[torch.from_numpy(packed_pair_index(nv, ii, jj)).cuda()].double().cpu().numpy()
        samples["thermo"] = ("first", ns, gq)
        thermo = {"value": cmp_per_step / (tms / 1e3), "unit": UNIT, "ms_per_step": tms, "levels": L,
                  "speedup_vs_fp32": ms_step / tms, "kernel_ms": kt,
                  "roofline": {"bound": "tensor", "achieved": tach / 1e12, "peak": fp8_peak / 1e12,
                               "unit": "TFLOP/s", "frac": tach / fp8_peak,
                               "traffic": profiled_traffic("thermo_gemm", args.workload),
                               "kernel": "thermo_gemm", "dtype": "fp8 e4m3 0/1, fp32 accumulate",
                               "peak_basis": "measured bf16 dense burst x 2 (nominal fp8/bf16 ratio), of measured"},
                  "quantization_error_vs_fp64_oracle": None}

    # ---- secondary: the 3-way workload ----
    secondary = None
    if not args.no_secondary and w["way"] == 2 and ws == 1:
        # thresholded 2-way on the benchmark matrix: every pair with c2 >= tau
        # (tau: the 0.9981 quantile of 10^6 sampled metrics, about 10^6 hits),
        # sorted; device output buffers
        torch.manual_seed(11)
        samp = out[torch.randint(0, out.numel(), (1000000,), device="cuda")]
        tau2 = float(torch.quantile(samp.float(), 0.9981))
        cap2 = 4_000_000
        tp = torch.empty((cap2, 3), dtype=torch.int32, device="cuda")
        tc = torch.empty(1, dtype=torch.int64, device="cuda")
        for _ in range(2):
            ps.check(ps.ps_threshold_2way(h.h, ctypes.byref(m), tau2, tp.data_ptr(), cap2, tc.data_ptr(), sptr), h.h)
        ps.check(ps.ps_timing_enable(h.h, 1), h.h)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            ps.check(ps.ps_threshold_2way(h.h, ctypes.byref(m), tau2, tp.data_ptr(), cap2, tc.data_ptr(), sptr), h.h)
        torch.cuda.synchronize()
        mst = (time.perf_counter() - t0) / 3 * 1e3
        ps.check(ps.ps_timing_read(h.h, b"threshold2", ctypes.byref(n_launch), ctypes.byref(k_ms)), h.h)
        ps.check(ps.ps_timing_enable(h.h, 0), h.h)
        kt2 = k_ms.value / max(n_launch.value, 1)
        thr2 = {
            "tau": tau2, "pairs": int(tc.item()), "ms_per_call": mst, "kernel_ms": kt2,
            "frac_of_alu_peak": cmp_per_step / (kt2 / 1e3) / peak_cmp,
            "note": "ps_threshold_2way with device buffers, sorted (i, j, c2); wall time per call (synchronising)"}
        del tp, tc, samp
        del out
        torch.cuda.empty_cache()
        w3 = WORKLOADS["3way_2048x4096_f32"]
        V3 = synth.zero_inflated(w3["nv"], w3["nf"], synth.seed_for(3))
        X3 = torch.from_numpy(V3).cuda()
        m3 = ps.matrix(X3)
        o3 = torch.empty(ps.ps_slab_size(w3["nv"], 0, w3["nv"]), dtype=torch.float32, device="cuda")
        for _ in range(2):
            ps.check(ps.ps_metrics_3way(h.h, ctypes.byref(m3), 0, w3["nv"], o3.data_ptr(), sptr), h.h)
        ps.check(ps.ps_timing_enable(h.h, 1), h.h)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(3):
            ps.check(ps.ps_metrics_3way(h.h, ctypes.byref(m3), 0, w3["nv"], o3.data_ptr(), sptr), h.h)
        e1.record(stream)
        torch.cuda.synchronize()
        ms3 = e0.elapsed_time(e1) / 3
        ps.check(ps.ps_timing_read(h.h, b"mgemm3", ctypes.byref(n_launch), ctypes.byref(k_ms)), h.h)
        ps.check(ps.ps_timing_enable(h.h, 0), h.h)
        k3 = k_ms.value / max(n_launch.value, 1)
        c3 = comparisons(w3)
        secondary = {"3way_2048x4096_f32": {"value": c3 / (ms3 / 1e3), "unit": UNIT, "ms_per_step": ms3,
                                            "mgemm3_ms": k3, "frac_of_peak": c3 / (k3 / 1e3) / peak_cmp}}
        del o3, X3
        torch.cuda.empty_cache()
        # the shape of the paper's Table 1 kernel timing (10,240 vectors of
        # 12,288 fields, FP32), one more point of the same min-product kernel
        wt = WORKLOADS["2way_10240x12288_f32"]
        Vt = synth.zero_inflated(wt["nv"], wt["nf"], synth.seed_for(2, 1050))
        Xt = torch.from_numpy(Vt).cuda()
        mt = ps.matrix(Xt)
        ot = torch.empty(wt["nv"] * (wt["nv"] - 1) // 2, dtype=torch.float32, device="cuda")
        for _ in range(2):
            ps.check(ps.ps_metrics_2way(h.h, ctypes.byref(mt), ps.PS_PATH_FP32, 0, ot.data_ptr(), 0, sptr), h.h)
        ps.check(ps.ps_timing_enable(h.h, 1), h.h)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(5):
            ps.check(ps.ps_metrics_2way(h.h, ctypes.byref(mt), ps.PS_PATH_FP32, 0, ot.data_ptr(), 0, sptr), h.h)
        e1.record(stream)
        torch.cuda.synchronize()
        mst_ = e0.elapsed_time(e1) / 5
        ps.check(ps.ps_timing_read(h.h, b"mgemm2", ctypes.byref(n_launch), ctypes.byref(k_ms)), h.h)
        ps.check(ps.ps_timing_enable(h.h, 0), h.h)
        kt = k_ms.value / max(n_launch.value, 1)
        ct = comparisons(wt)
        secondary["2way_10240x12288_f32"] = {
            "value": ct / (mst_ / 1e3), "unit": UNIT, "ms_per_step": mst_, "mgemm2_ms": kt,
            "frac_of_peak": ct / (kt / 1e3) / peak_cmp,
            "note": "upper triangle (i < j), the paper's Table 1 shape; inputs larger than L2 (0.50 GB in)"}
        del ot, Xt
        torch.cuda.empty_cache()
        # output-bound shapes: 32768 vectors with few fields, FP32 output
        # (2.15 GB per call) against the measured HBM copy bandwidth
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        nvs = 32768
        os_ = torch.empty(nvs * (nvs - 1) // 2, dtype=torch.float32, device="cuda")
        small = {}
        for nfs in (16, 64, 385):
            Vs = synth.zero_inflated(nvs, nfs, synth.seed_for(2, 1000 + nfs))
            Xs = torch.from_numpy(Vs).cuda()
            ms_ = ps.matrix(Xs)
            for _ in range(3):
                ps.check(ps.ps_metrics_2way(h.h, ctypes.byref(ms_), ps.PS_PATH_FP32, 0, os_.data_ptr(), 0,
                                            sptr), h.h)
            ps.check(ps.ps_timing_enable(h.h, 1), h.h)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(10):
                ps.check(ps.ps_metrics_2way(h.h, ctypes.byref(ms_), ps.PS_PATH_FP32, 0, os_.data_ptr(), 0,
                                            sptr), h.h)
            e1.record(stream)
            torch.cuda.synchronize()
            mss = e0.elapsed_time(e1) / 10
            ps.check(ps.ps_timing_read(h.h, b"mgemm2", ctypes.byref(n_launch), ctypes.byref(k_ms)), h.h)
            ps.check(ps.ps_timing_enable(h.h, 0), h.h)
            ks = k_ms.value / max(n_launch.value, 1)
            byts = Vs.nbytes + os_.numel() * 4
            cs = nfs * nvs * (nvs - 1) // 2
            # the same call with one-byte codes (PS_U8): a quarter of the bytes out
            ou_ = torch.empty(os_.numel(), dtype=torch.uint8, device="cuda")
            for _ in range(3):
                ps.check(ps.ps_metrics_2way(h.h, ctypes.byref(ms_), ps.PS_PATH_FP32, 0, ou_.data_ptr(), ps.PS_U8,
                                            sptr), h.h)
            ps.check(ps.ps_timing_enable(h.h, 1), h.h)
            torch.cuda.synchronize()
            for _ in range(10):
                ps.check(ps.ps_metrics_2way(h.h, ctypes.byref(ms_), ps.PS_PATH_FP32, 0, ou_.data_ptr(), ps.PS_U8,
                                            sptr), h.h)
            torch.cuda.synchronize()
            ps.check(ps.ps_timing_read(h.h, b"mgemm2", ctypes.byref(n_launch), ctypes.byref(k_ms)), h.h)
            ps.check(ps.ps_timing_enable(h.h, 0), h.h)
            ku = k_ms.value / max(n_launch.value, 1)
            bytu = Vs.nbytes + ou_.numel()
            del ou_
            small[f"2way_32768x{nfs}_f32"] = {
                "ms_per_step": mss, "mgemm2_ms": ks, "value": cs / (mss / 1e3), "unit": UNIT,
                "algorithmic_gb": byts / 1e9, "achieved_gbs": byts / (ks / 1e3) / 1e9,
                "frac_of_hbm": byts / (ks / 1e3) / 1e9 / hbm,
                "frac_of_alu_peak": cs / (ks / 1e3) / peak_cmp,
                "u8_codes": {"mgemm2_ms": ku, "algorithmic_gb": bytu / 1e9,
                             "achieved_gbs": bytu / (ku / 1e3) / 1e9, "frac_of_hbm": bytu / (ku / 1e3) / 1e9 / hbm,
                             "frac_of_alu_peak": cs / (ku / 1e3) / peak_cmp}}
            del Xs
        secondary["small_nf_output_bound"] = small
        del os_
        torch.cuda.empty_cache()
        # bit-packed 0/1 input (Sorenson case): bits straight into the tensor
        # cores vs. the FP32 CUDA-core path on the same (unpacked) data
        nvb, nfb = 32768, 8192
        _, words = synth.binary_bits(nvb, nfb, synth.seed_for(7), junk_tail=False)
        Wb = torch.from_numpy(words.view(np.int32)).cuda()
        mb = ps.bit_matrix(Wb, nfb)
        ob = torch.empty(nvb * (nvb - 1) // 2, dtype=torch.float32, device="cuda")
        sor = {}
        for name, path, kern in (("tensor_core_bits", ps.PS_PATH_THERMO, b"thermo_gemm"),
                                 ("fp32_cuda_core", ps.PS_PATH_FP32, b"mgemm2")):
            for _ in range(2):
                ps.check(ps.ps_metrics_2way(h.h, ctypes.byref(mb), path, 0, ob.data_ptr(), 0, sptr), h.h)
            ps.check(ps.ps_timing_enable(h.h, 1), h.h)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(3):
                ps.check(ps.ps_metrics_2way(h.h, ctypes.byref(mb), path, 0, ob.data_ptr(), 0, sptr), h.h)
            e1.record(stream)
            torch.cuda.synchronize()
            msb = e0.elapsed_time(e1) / 3
            ps.check(ps.ps_timing_read(h.h, kern, ctypes.byref(n_launch), ctypes.byref(k_ms)), h.h)
            ps.check(ps.ps_timing_enable(h.h, 0), h.h)
            sor[name] = {"ms_per_step": msb, "kernel_ms": k_ms.value / max(n_launch.value, 1),
                         "value": nfb * nvb * (nvb - 1) // 2 / (msb / 1e3), "unit": UNIT}
        sor["speedup_tensor_vs_fp32"] = sor["fp32_cuda_core"]["ms_per_step"] / sor["tensor_core_bits"]["ms_per_step"]
        sor["input"] = f"{nvb} x {nfb} bit-packed 0/1 (p_one 0.15), {words.nbytes / 1e6:.1f} MB"
        secondary["sorenson_b1_32768x8192"] = sor
        del Wb, ob
        secondary["threshold_2way_32768x8192"] = thr2

    # ---- batched uneven instances (64 problems, one persistent graph launch) ----
    batched = None
    if not args.no_batched and w["way"] == 2 and ws == 1:
        batched = batched_section(ps, synth, h, torch, sptr, peak_cmp)

    # ---- thresholded 3-way search with proposals (8192 x 2048 latent profiles) ----
    thresh = None
    if not args.no_threshold and w["way"] == 2 and ws == 1:
        thresh = threshold_section(ps, synth, h, torch, sptr, peak_cmp)

    # ---- CPU-baseline leg: the oracle timed on a bounded sample, and the
    # oracle's values for the sampled GPU outputs ----
    cb = None
    max_rel = None
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        cb = cpu_baseline(V, w, 8192 if w["way"] == 2 else 256)
        cb["parity_samples"] = sampled_parity(V, samples)
        max_rel = cb["parity_samples"]["fp32"]["max_rel"]
        if half2 is not None:
            half2["sampled_error"] = cb["parity_samples"]["half2"]
        if thermo is not None:
            thermo["quantization_error_vs_fp64_oracle"] = cb["parity_samples"]["thermo"]

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
                "scaling": "strong" if strong else "weak",
                "vs_baseline": None, "dtype": "f32" if dtype == np.float32 else "f64", "data": "synthetic",
                "config": {"workload": args.workload, "nv": nv, "nf": nf, "way": w["way"],
                           "comparisons_per_step": cmp_per_step, "path": "fp32 CUDA-core min+add",
                           "l2": f"inputs larger than L2 ({V.nbytes / 1e9:.2f} GB in, "
                                 f"{out_bytes / 1e9:.2f} GB out)",
                           "parallelism": (f"one instance split over {ws} ranks (ps_partition, no collective)"
                                           if strong else f"independent instance per rank x{ws}")},
                "roofline": roofline, "cpu_baseline": cb, "e2e": e2e, "clocks": clk,
                "gpu_launches": launches_per_step * args.steps,
                "sampled_max_rel_err": max_rel, "half2_variant": half2, "thermo_tensor_core": thermo,
                "secondary": secondary, "batched": batched,
                "threshold_3way": thresh}
        print(json.dumps(line), flush=True)
    h.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
