#!/usr/bin/env python3
"""Benchmark: samples/s of the whole hot path on one GB300 per rank.

One step = one pass of every hot-path stage over the resident batch:
  compress (H D x, mask draw, ELL)  ->  covariance (Gram accumulate, C_n
  finalize)  ->  top-k PCA + un-mix  ->  K-means start (dense y of K seeded
  rows)  ->  `iters` sparsified K-means iterations (one CUDA graph)  ->
  un-mixed centres.
Workload (default): n = 1,000,000, p = 1024, m = 51 (5%), K = 10, 20
iterations; Gaussian mixture with centres N(0,1)*3, noise N(0, 0.5^2), 10% of
rows Student-t(3) (synthetic, generated on the device from the seed).

Multi-GPU: replicas only (the method needs no exchange on one GPU; each rank
runs its own copy of the workload), "scaling": "weak".

--impl reference times the CPU oracle (plain FP64 C) on a bounded row sample
of the same workload on the host cores.
"""
from __future__ import annotations

import os

# the CPU oracle and numpy's LAPACK run single-threaded; say so in the output
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import math
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(workload="kmeans_mixture_n1e6_p1024_m51_K10", n=1_000_000, p=1024, m=51, K=10,
                iters=20, pca_k=10, seed=20240611)
METRIC = "samples/s compress+cov+K-means iter at 1 GB300; %HBM/tensor peak; err vs FP64"

# The paper's own timings (Sec. VII), context only: Matlab + C in float64 on
# two 8-core Xeons at 2.4-3.2 GHz, on MNIST-derived data with p = 784 (not
# this workload).  Rates are the paper's rows divided by its times.
PAPER_CONTEXT = {
    "hardware": "2 x 8-core Xeon, 2.4-3.2 GHz, Matlab + C, float64 (the paper's runs)",
    # table of estimated speedups, n = 9,631,605, gamma = 0.05: one iteration
    # 7.0 s (assignments 1.3 s, centre update 5.7 s)
    "kmeans_iteration_samples_per_s": 9_631_605 / 7.0,
    "kmeans_assign_samples_per_s": 9_631_605 / 1.3,
    # timing table at n = 6e5, gamma = 0.05: preconditioning 33.7 s, sampling 6.0 s
    "precondition_and_sample_samples_per_s": 600_000 / (33.7 + 6.0),
    "workload": "p = 784, m/p = 0.05, K = 10 (MNIST-derived); not comparable sizes",
}
UNIT = "samples/s"

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# dominant kernel from one ncu capture of this workload, valid only while the
# kernel source still has the digest it had when captured.
KERNEL_TRAFFIC = {
    # kmeans_rc_kernel<5, 1> (adaptive pass, incremental): 164.88 MB read +
    # 4.19 MB written per launch at n = 400,000 (422.7 B per row), scaled to
    # n = 10^6
    "kmeans": {"bytes": 422_700_000, "n": 1_000_000, "p": 1024,
               "source": "paper_1511_00152_gb300/csrc/kmeans.cu", "src_sha": "e3f68cf3451fcfb0"},
    # gram_tc_kernel (split-BF16): 178.28 MB read + 9.86 MB written per launch
    # at n = 400,000; the reads (the ELL rows, read once from DRAM by all of a
    # row range's tiles) scaled to n = 10^6, the writes (the float64 Gram's
    # atomics) kept
    "gram": {"bytes": 455_600_000, "n": 1_000_000, "p": 1024,
             "source": "paper_1511_00152_gb300/csrc/gram_tc.cu", "src_sha": "7208d7883a2122bd"},
}


def source_digest(rel: str) -> str:
    import hashlib
    with open(os.path.join(ROOT, rel), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), float(d["bf16_tflops_sustained"]), "measured"
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl != "reference" else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def gpu_local_cpus(index: int):
    """CPUs on the GPU's own NUMA node: the PCI device's local_cpulist in sysfs,
    else the CPU affinity `nvidia-smi topo -m` prints; None if neither says."""
    import torch

    def parse(text):
        cpus = set()
        for part in text.strip().split(","):
            if "-" in part:
                a, b = part.split("-")
                cpus.update(range(int(a), int(b) + 1))
            elif part.strip():
                cpus.add(int(part))
        return cpus or None

    try:
        pr = torch.cuda.get_device_properties(index)
        bus = "%04x:%02x:%02x.0" % (getattr(pr, "pci_domain_id", 0), pr.pci_bus_id,
                                    pr.pci_device_id)
        with open(f"/sys/bus/pci/devices/{bus}/local_cpulist") as fh:
            cpus = parse(fh.read())
        if cpus and len(cpus) < (os.cpu_count() or 0):
            return cpus
    except Exception:
        pass
    try:
        out = subprocess.run(["nvidia-smi", "topo", "-m"], capture_output=True, text=True,
                             timeout=20).stdout.splitlines()
        head = next(line for line in out if "CPU Affinity" in line)
        col = head.split("\t").index("CPU Affinity") if "\t" in head else None
        row = next(line for line in out if line.startswith(f"GPU{index}"))
        fields = row.split("\t") if col is not None else row.split()
        cpus = parse(fields[col] if col is not None else fields[-2])
        if cpus and len(cpus) < (os.cpu_count() or 0):
            return cpus
    except Exception:
        pass
    return None


def max_over_ranks(value: float, pg, device=None) -> float:
    """Max of a per-rank float over all ranks (identity on one rank)."""
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def barrier(pg, device=None):
    if pg is not None:
        if device is not None:
            pg.barrier(device_ids=[device.index])
        else:
            pg.barrier()


# ------------------------------------------------------------------ CPU oracle

def oracle_step(X, cfg, rows_init):
    """One step of the oracle on a row sample (compress, C_n, top-k, K-means);
    returns its results for the accuracy comparison."""
    import oracle
    n, p = X.shape
    m, K = cfg["m"], cfg["K"]
    seed = cfg["seed"]
    pt = oracle.ptilde(p)
    idx, val = oracle.compress(X, m, seed)
    C = oracle.cov(idx, val, pt)
    w, V = oracle.pca_topk(C, cfg["pca_k"])
    oracle.unmix(V.T.copy(), p, seed)
    mu0 = oracle.precondition(X[rows_init], seed)
    labels, mu, _ = oracle.kmeans(idx, val, mu0, pt, cfg["iters"])
    oracle.unmix(mu, p, seed)
    return {"idx": idx, "val": val, "C": C, "evals": w, "V": V, "labels": labels, "mu": mu}


def cpu_sample(cfg, rows: int):
    from paper_1511_00152_gb300 import synth
    X, _, _ = synth.mixture(rows, cfg["p"], cfg["K"], seed=cfg["seed"])
    rows_init = synth.init_rows(rows, cfg["K"], cfg["seed"])
    return X, rows_init


def time_cpu_baseline(cfg, rows=4000):
    X, ri = cpu_sample(cfg, rows)
    oracle_step(X[:200], cfg, synth_rows(200, cfg))  # compile/warm the oracle
    t = time.perf_counter()
    ref = oracle_step(X, cfg, ri)
    dt = time.perf_counter() - t
    return rows / dt, dt, (X, ri, ref)


def accuracy_vs_oracle(sk, pipeline, ctx, mode, topk_iters, gwork, work, sample, cfg, dev):
    """The GPU path on the oracle's row sample (untimed), each result against
    the FP64 oracle's: idx exact, val relative to the row norm, C_n relative
    Frobenius, top-k eigenvalues and principal angles, centres and labels
    after the K-means iterations."""
    import numpy as np
    import torch
    X, ri, ref = sample
    rows, p = X.shape
    m, K, k, iters = cfg["m"], cfg["K"], cfg["pca_k"], cfg["iters"]
    pt = ctx.pt
    Xd = torch.as_tensor(X, device=dev)
    idx, val = sk.sk_compress(ctx, Xd)
    G = torch.empty((pt, pt), dtype=torch.float64, device=dev)
    sk.sk_cov_reset(ctx, G)
    sk.sk_cov_accumulate(ctx, mode, idx, val, G, work=gwork)
    C = torch.empty_like(G)
    sk.sk_cov_finalize(ctx, G, rows, C=C)
    ev = torch.empty(k, dtype=torch.float64, device=dev)
    U = torch.empty((k, pt), dtype=torch.float64, device=dev)
    sk.sk_cov_topk(ctx, C, k, topk_iters, evals=ev, U=U, work=work)
    mu0 = sk.sk_precondition(ctx, Xd[torch.as_tensor(ri, device=dev)].contiguous())
    st = pipeline.KMeansState(ctx, rows, K, device=dev)
    labels, mu = st.run(idx, val, mu0, iters, use_graph=False)
    torch.cuda.synchronize()
    idx_h, val_h = idx.cpu().numpy(), val.cpu().numpy().astype(np.float64)
    norms = np.linalg.norm(X.astype(np.float64), axis=1)
    Co, Cg = ref["C"], C.cpu().numpy()
    Vo, Vg = ref["V"], U.cpu().numpy().T
    Qg, _ = np.linalg.qr(Vg)
    # largest principal angle: sin = ||(I - Vo Vo^T) Qg||_2 (accurate for small angles)
    sin_max = float(np.linalg.norm(Qg - Vo @ (Vo.T @ Qg), 2))
    evo, evg = ref["evals"], ev.cpu().numpy()
    muo, mug = ref["mu"], mu.cpu().numpy().astype(np.float64)
    return {
        "rows": rows, "against": "FP64 oracle on the same rows",
        "idx_rows_exact": float(np.mean(np.all(idx_h == ref["idx"], axis=1))),
        "val_max_err_rel_row_norm": float(np.max(np.abs(val_h - ref["val"]).max(axis=1) / norms)),
        "cov_rel_frobenius": float(np.linalg.norm(Cg - Co) / np.linalg.norm(Co)),
        "topk_eigenvalue_max_rel_err": float(np.max(np.abs(evg - evo) / np.abs(evo))),
        "topk_max_sin_principal_angle": sin_max,
        "kmeans_label_agreement": float(np.mean(labels.cpu().numpy() == ref["labels"])),
        "kmeans_centre_rel_err": float(np.linalg.norm(mug - muo) / np.linalg.norm(muo)),
        "notes": (f"Gram mode {cfg.get('gram', '')}; top-{k} by {topk_iters} subspace iterations "
                  f"(oracle: LAPACK eigh); {iters} K-means iterations end to end (a flipped "
                  "near-tie can move a trajectory, so the label figure is an agreement)"),
    }


def synth_rows(n, cfg):
    from paper_1511_00152_gb300 import synth
    return synth.init_rows(n, cfg["K"], cfg["seed"])


def run_reference(args, cfg):
    world, rank, local, pg = dist_setup(args)
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    rows = args.ref_rows
    X, ri = cpu_sample(cfg, rows)
    for _ in range(args.warmup):
        oracle_step(X, cfg, ri)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(X, cfg, ri)
    dt = (time.perf_counter() - t) / args.steps
    value = rows / dt
    sample = (f"{rows} rows of the workload per step (full p, m, K, iters; compress, C_n, "
              f"top-{cfg['pca_k']}, {cfg['iters']} K-means iterations)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {k: cfg[k] for k in ("workload", "n", "p", "m", "K", "iters")} | {"rows_per_step": rows},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU path

def run_gpu(args, cfg):
    import torch
    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1511_00152_gb300 import build as skbuild
    skbuild.build()
    from paper_1511_00152_gb300 import _lib as sk
    from paper_1511_00152_gb300 import pipeline, synth

    n, p, m, K, iters, k = cfg["n"], cfg["p"], cfg["m"], cfg["K"], cfg["iters"], cfg["pca_k"]
    seed = cfg["seed"] + rank
    mode = {"fp32": sk.SK_GRAM_FP32, "bf16": sk.SK_GRAM_BF16, "bf16x3": sk.SK_GRAM_BF16X3}[args.gram]
    ctx = sk.sk_init(p, m, seed)
    pt = ctx.pt
    X, _, _ = synth.mixture_device(n, p, 10, seed, device=dev)
    rows = synth.init_rows(n, K, seed)
    Xsel = X[torch.as_tensor(rows, device=dev)].contiguous()
    idx = torch.empty((n, m), dtype=torch.int32, device=dev)
    val = torch.empty((n, m), dtype=torch.float32, device=dev)
    G = torch.empty((pt, pt), dtype=torch.float64, device=dev)
    C = torch.empty((pt, pt), dtype=torch.float64, device=dev)
    evals = torch.empty(k, dtype=torch.float64, device=dev)
    U = torch.empty((k, pt), dtype=torch.float64, device=dev)
    Ux = torch.empty((k, p), dtype=torch.float64, device=dev)
    work = torch.empty(sk.sk_cov_topk_workspace(pt, k), dtype=torch.float64, device=dev)
    cen = torch.empty((K, p), dtype=torch.float32, device=dev)
    gwork = torch.empty(max(1, sk.sk_cov_workspace_bytes(ctx, mode, n)), dtype=torch.uint8, device=dev)
    st = pipeline.KMeansState(ctx, n, K, device=dev)
    stream = torch.cuda.current_stream()

    stages = ["compress", "gram", "cov_finalize", "topk", "kmeans_prep", "kmeans", "unmix"]
    # library kernels per step: bucket + Gram for the tensor-core modes; top-k
    # = init + the float32 panels' diagonal shift (more than 2 iterations) +
    # (iters + 1) x panel + iters x (Gram, Cholesky, apply) + Rayleigh-Ritz
    # Gram + Ritz eigenproblem + Ritz vectors + sign fix, then the eigenvector
    # un-mix; K-means = start centres + iters x (pass choice,
    # full-rebuild pass, incremental pass -- one of the two returns at once --,
    # finalize)
    launches = {"compress": 1, "gram": 1 if args.gram == "fp32" else 2, "cov_finalize": 1,
                "topk": 4 * max(args.topk_iters, 1) + 6 + (1 if args.topk_iters > 2 else 0) + 1,
                "kmeans_prep": 1, "kmeans": 3 * iters, "unmix": 1}

    def step(ev=None):
        def mark(i):
            if ev is not None:
                ev[i].record(stream)
        mark(0)
        sk.sk_compress(ctx, X, idx=idx, val=val)
        mark(1)
        sk.sk_cov_reset(ctx, G)
        sk.sk_cov_accumulate(ctx, mode, idx, val, G, work=gwork)
        mark(2)
        sk.sk_cov_finalize(ctx, G, n, C=C)
        mark(3)
        sk.sk_cov_topk(ctx, C, k, args.topk_iters, evals=evals, U=U, work=work)
        sk.sk_unmix(ctx, U, out=Ux)
        mark(4)
        sk.sk_precondition(ctx, Xsel, Y=st.mu)
        mark(5)
        if args.no_graph:
            for it in range(iters):
                st.iteration(idx, val, first=(it == 0))
        else:
            st.graph.replay()
        mark(6)
        sk.sk_unmix(ctx, st.mu, out=cen)
        mark(7)

    # capture the K-means loop once (its own kernels, replayed as one graph)
    mu0 = sk.sk_precondition(ctx, Xsel)
    sk.sk_compress(ctx, X, idx=idx, val=val)
    st.run(idx, val, mu0, iters, use_graph=not args.no_graph)
    torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(pg, dev)
    sampler = ClockSampler(local)
    sampler.start()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(stages) + 1)]
           for _ in range(args.steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier(pg, dev)
    t0.record(stream)
    for s in range(args.steps):
        step(evs[s])
    t1.record(stream)
    torch.cuda.synchronize()
    barrier(pg, dev)
    clocks = sampler.stop()
    ms = t0.elapsed_time(t1) / args.steps
    ms = max_over_ranks(ms, pg, dev)
    stage_ms = {}
    for i, name in enumerate(stages):
        stage_ms[name] = sum(e[i].elapsed_time(e[i + 1]) for e in evs) / args.steps
    assert sk.sk_device_status() == sk.SK_OK

    # accuracy of the timed top-k (outside the timed region): largest relative
    # eigen-residual ||C u - lambda u|| / |lambda| of the returned pairs
    Cu = C @ U.T
    pca_res = float((((Cu - U.T * evals[None, :]) ** 2).sum(0).sqrt() / evals.abs()).max())

    # ---- rooflines (algorithmic bytes or flops per launch / event-timed duration)
    hbm, bf16, bf16s, peak_src = load_peaks()
    kmeans_iter_ms = stage_ms["kmeans"] / iters
    N = 256 if pt >= 256 else pt
    ntiles = sum(pt // N - bi // (N // 128) for bi in range(pt // 128)) if pt >= 128 else 0
    prods = {"fp32": 0, "bf16": 1, "bf16x3": 3}[args.gram]
    roofs = {
        # read X (4p B) + write the ELL row (8m B)
        "compress": {"kernel": "compress_kernel<10,false,true>", "bound": "hbm",
                     "bytes": n * (4 * p + 8 * m), "ms": stage_ms["compress"],
                     "peak": hbm, "unit": "GB/s"},
        # read the ELL row (8m B) and the previous label (4 B), write the label (4 B);
        # the per-iteration time is the graph's / iters, so it includes one
        # finalize launch (and the first, full-sums pass is averaged in)
        "kmeans": {"kernel": "kmeans_rc_kernel (assignment + incremental sums; rebuilds add "
                             "kmeans_sums_kernel)", "bound": "hbm",
                   "bytes": n * (8 * m + 8), "ms": kmeans_iter_ms, "peak": hbm, "unit": "GB/s"},
    }
    if prods:
        # 128 x N upper tiles over n rows, three products per tile when split
        roofs["gram"] = {"kernel": "gram_tc_kernel", "bound": "tensor",
                         "flops": 2.0 * n * 128 * N * ntiles * prods, "ms": stage_ms["gram"],
                         "peak": bf16s, "unit": "TFLOP/s", "tiles": ntiles,
                         "algorithmic_macs": n * m * (m + 1) // 2}
    for r in roofs.values():
        if r["bound"] == "hbm":
            r["achieved"] = r["bytes"] / (r["ms"] * 1e-3) / 1e9
        else:
            r["achieved"] = r["flops"] / (r["ms"] * 1e-3) / 1e12
        r["frac"] = r["achieved"] / r["peak"]
    dom_stage = max((s_ for s_ in roofs), key=lambda s_: roofs[s_]["ms"] *
                    (iters if s_ == "kmeans" else 1))
    d = roofs[dom_stage]
    src = (f"{peak_src} hbm_gbs (burst copy)" if d["bound"] == "hbm"
           else f"{peak_src} bf16_tflops_sustained")
    traffic = KERNEL_TRAFFIC.get(dom_stage)
    if traffic is not None and (traffic["n"] != n or traffic["p"] != p or
                                traffic["src_sha"] != source_digest(traffic["source"])):
        traffic = None  # counters taken on another workload or an older kernel
    roof = {"kernel": d["kernel"], "bound": d["bound"], "achieved": d["achieved"],
            "peak": d["peak"], "unit": d["unit"], "frac": d["frac"],
            "traffic": None if traffic is None else traffic["bytes"],
            "algorithmic": d.get("bytes", d.get("flops")), "peak_source": src,
            "stage": dom_stage}

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        # pinned host buffers on the GPU's own NUMA node (first touch by a
        # thread on a local CPU), so the host link is not crossed twice
        host_cpus = gpu_local_cpus(local)
        if host_cpus:
            os.sched_setaffinity(0, host_cpus)
        Xh = torch.empty((n, p), dtype=torch.float32, pin_memory=True)
        Xh.copy_(X)
        # the seeded start rows, picked on the host (input preparation)
        Xsel_h = Xh[torch.as_tensor(rows)].contiguous().pin_memory()
        lab_h = torch.empty(n, dtype=torch.int32, pin_memory=True)
        cen_h = torch.empty((K, p), dtype=torch.float32, pin_memory=True)
        ux_h = torch.empty((k, p), dtype=torch.float64, pin_memory=True)
        Xsel2 = torch.empty_like(Xsel)
        # X streams to the device in chunks; each chunk is compressed and added
        # to the Gram while the next ones are copied (a ring of three chunk
        # buffers on the device)
        nchunk = max(1, args.e2e_chunks)
        streamer = pipeline.HostStreamer(ctx, (n + nchunk - 1) // nchunk, mode, nbuf=3,
                                         device=dev)

        def e2e_step():
            Xsel2.copy_(Xsel_h, non_blocking=True)
            streamer.run(Xh, idx, val, G)
            sk.sk_cov_finalize(ctx, G, n, C=C)
            sk.sk_cov_topk(ctx, C, k, args.topk_iters, evals=evals, U=U, work=work)
            sk.sk_unmix(ctx, U, out=Ux)
            sk.sk_precondition(ctx, Xsel2, Y=st.mu)
            if args.no_graph:
                for it in range(iters):
                    st.iteration(idx, val, first=(it == 0))
            else:
                st.graph.replay()
            sk.sk_unmix(ctx, st.mu, out=cen)
            lab_h.copy_(st.labels, non_blocking=True)
            cen_h.copy_(cen, non_blocking=True)
            ux_h.copy_(Ux, non_blocking=True)

        for _ in range(max(1, args.warmup)):
            e2e_step()
        torch.cuda.synchronize()
        barrier(pg, dev)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        nst = max(1, min(args.steps, 5))
        for _ in range(nst):
            e2e_step()
        b.record(stream)
        torch.cuda.synchronize()
        ems = max_over_ranks(a.elapsed_time(b) / nst, pg, dev)
        e2e = {"value": world * n / (ems * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": n * p * 4 + K * p * 4,
               "d2h_bytes_per_step": n * 4 + K * p * 4 + k * p * 8,
               "ms_per_step": ems,
               "host_cpus": (f"{min(host_cpus)}-{max(host_cpus)} ({len(host_cpus)}, GPU-local)"
                             if host_cpus else "any")}
        del Xh

    # the plain FP32 GPU form of the covariance pass (shared-memory scatter
    # Gram), timed beside the chosen mode on the same ELL rows
    plain = None
    if mode != sk.SK_GRAM_FP32 and not args.no_plain:
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        sk.sk_cov_reset(ctx, G)
        sk.sk_cov_accumulate(ctx, sk.SK_GRAM_FP32, idx, val, G)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(3):
            sk.sk_cov_reset(ctx, G)
            sk.sk_cov_accumulate(ctx, sk.SK_GRAM_FP32, idx, val, G)
        b.record(stream)
        torch.cuda.synchronize()
        g32 = a.elapsed_time(b) / 3
        plain = {"gram": "fp32", "gram_ms": g32, "chosen_gram_ms": stage_ms["gram"],
                 "speedup": g32 / stage_ms["gram"],
                 "step_value": world * n / ((ms - stage_ms["gram"] + g32) * 1e-3)}
    # the unfused form of the compress pass: the dense y = HDx written to HBM
    # (sk_precondition), then its entries at the same mask stream gathered by
    # sk_compress of a context without preconditioning (pt columns)
    if not args.no_plain and p == pt:
        ctx_raw = sk.sk_init_ex(pt, m, seed, sk.SK_FLAG_NO_PRECONDITION)
        Yd = torch.empty((n, pt), dtype=torch.float32, device=dev)
        idx2 = torch.empty_like(idx)
        val2 = torch.empty_like(val)
        sk.sk_precondition(ctx, X, Y=Yd)
        sk.sk_compress(ctx_raw, Yd, idx=idx2, val=val2)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(3):
            sk.sk_precondition(ctx, X, Y=Yd)
            sk.sk_compress(ctx_raw, Yd, idx=idx2, val=val2)
        b.record(stream)
        torch.cuda.synchronize()
        tu = a.elapsed_time(b) / 3
        unfused = {"form": "sk_precondition (dense y to HBM) + sk_compress of y, no preconditioning",
                   "compress_ms": tu, "fused_compress_ms": stage_ms["compress"],
                   "speedup": tu / stage_ms["compress"],
                   "bytes_per_row": 3 * 4 * pt + 8 * m,
                   "same_output": bool(torch.equal(idx2, idx) and torch.equal(val2, val))}
        plain = dict(plain or {}, compress_unfused=unfused)
        del Yd, idx2, val2

    cpu = None
    accuracy = None
    if rank == 0 and not args.no_cpu:
        try:
            v, dt, sample = time_cpu_baseline(cfg, rows=args.cpu_rows)
            cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"{args.cpu_rows} rows of the workload (full p, m, K, iters), {dt:.1f} s"}
        except Exception as exc:  # report, do not hide
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {exc}"}
            sample = None
        if sample is not None:
            try:
                accuracy = accuracy_vs_oracle(sk, pipeline, ctx, mode, args.topk_iters, gwork, work,
                                              sample, dict(cfg, gram=args.gram), dev)
            except Exception as exc:  # report, do not hide
                accuracy = {"failed": repr(exc)}

    extra = None
    if rank == 0 and world == 1 and not args.no_extra:
        # the other workloads of the path, each timed on its own with its own
        # clock record, after the main step's memory is released
        del X, Xsel, idx, val, G, C, gwork, st, work
        torch.cuda.empty_cache()
        extra = {}
        for name, fn in (("pca", run_pca), ("serving", run_serving), ("batching", run_batching),
                         ("dct", run_dct)):
            try:
                extra[name] = fn(args, standalone=False)
            except Exception as exc:  # report, do not hide
                extra[name] = {"failed": repr(exc)}
            torch.cuda.empty_cache()

    if rank == 0:
        line = {
            "metric": METRIC, "value": world * n / (ms * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.gram == "fp32" else f"f32+{args.gram}",
            "data": "synthetic",
            "config": {"workload": cfg["workload"], "n": n, "p": p, "m": m, "K": K,
                       "kmeans_iters": iters, "pca_k": k, "topk_iters": args.topk_iters,
                       "gram": args.gram, "parallelism": f"replicas{world}",
                       "l2": "inputs larger than L2 (X is 4.1 GB)"},
            "stage_ms": stage_ms, "kmeans_iter_ms": kmeans_iter_ms,
            "pca_max_rel_residual": pca_res,
            "roofline": roof, "stage_rooflines": roofs, "plain_fp32_form": plain,
            "cpu_baseline": cpu, "accuracy_vs_fp64": accuracy, "paper_context": PAPER_CONTEXT,
            "e2e": e2e, "clocks": clocks,
            "gpu_launches": sum(launches.values()) * args.steps,
            "workloads": extra,
        }
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()
    return 0


# ------------------------------------------------------------------ serving

SERVING = dict(workload="serving_lowrank_mixture_p2048_m102_K8", p=2048, m=102, K=8,
               rows=10_000_000, chunk_min=4096, chunk_max=65536, seed=7, slots=4,
               mem_budget=4 << 30)


def run_serving(args, standalone=True):
    """Streaming workload: chunks of 4,096-65,536 rows (log-uniform) of one
    data stream go through the continuous-admission request loop; the Gram
    (BF16 products, FP32 accumulation, FP64 cross-block reduction) and the
    K = 8 centre sums stay resident on the device.
    The chunks' inputs are generated on the device before timing (resident,
    like the main workload).  Two passes: all chunks queued at once
    (throughput), then arrivals paced at half that throughput (latency)."""
    import numpy as np
    import torch
    from paper_1511_00152_gb300 import build as skbuild
    skbuild.build()
    from paper_1511_00152_gb300 import _lib as sk
    from paper_1511_00152_gb300 import serving, synth
    cfg = dict(SERVING)
    if args.n:
        cfg["rows"] = args.n
    P, M, K, seed = cfg["p"], cfg["m"], cfg["K"], cfg["seed"]
    rng = np.random.default_rng(seed)
    chunks, r0 = [], 0
    while r0 < cfg["rows"]:
        n = int(min(cfg["rows"] - r0, np.exp(rng.uniform(np.log(cfg["chunk_min"]),
                                                          np.log(cfg["chunk_max"])))))
        chunks.append((r0, n))
        r0 += n
    xs = [synth.lowrank_mixture_chunk_device(n, P, seed, r0) for (r0, n) in chunks]
    torch.cuda.synchronize()

    def one_pass(pace_rows_per_s=None):
        srv = serving.Server(P, M, seed, slots=cfg["slots"], max_rows=cfg["chunk_max"],
                             mem_budget_bytes=cfg["mem_budget"], mode=sk.SK_GRAM_BF16)
        srv.open_stream(0, sk.sk_precondition(srv.ctx, xs[0][:K].contiguous()))
        reqs, t = [], 0.0
        for (r0, n), x in zip(chunks, xs):
            reqs.append(serving.Request(stream_id=0, row0=r0, n=n, x=x, arrival=t))
            if pace_rows_per_s:
                t += n / pace_rows_per_s
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        done = srv.run(reqs, realtime=pace_rows_per_s is not None)
        wall = time.perf_counter() - t0
        assert sk.sk_device_status() == sk.SK_OK
        return srv, done, wall

    one_pass()  # warm-up (launch configuration, allocator)
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    srv, done, wall = one_pass()
    thr = cfg["rows"] / wall
    srv2, done2, wall2 = one_pass(pace_rows_per_s=0.5 * thr)
    clocks = sampler.stop()
    lat = serving.Server.latency_percentiles(done2)
    lat_sat = serving.Server.latency_percentiles(done)
    line = {
        "metric": "serving samples/s and per-chunk latency (continuous admission)",
        "value": thr, "unit": "samples/s", "n_gpus": 1, "higher_is_better": True,
        "dtype": "f32+bf16", "data": "synthetic",
        "config": {"workload": cfg["workload"], "rows": cfg["rows"], "chunks": len(chunks),
                   "chunk_rows": [cfg["chunk_min"], cfg["chunk_max"]], "p": P, "m": M, "K": K,
                   "slots": cfg["slots"], "mem_budget_bytes": cfg["mem_budget"],
                   "gram": "bf16"},
        "saturated": {"wall_s": wall, "samples_per_s": thr, "p50_ms": lat_sat["p50"],
                      "p99_ms": lat_sat["p99"], "peak_inflight_bytes": srv.peak_bytes},
        "paced_at_half_throughput": {"wall_s": wall2, "p50_ms": lat["p50"], "p99_ms": lat["p99"],
                                     "peak_inflight_bytes": srv2.peak_bytes},
        "latency_note": ("saturated: device time per chunk (all chunks queued at once); paced: "
                         "arrival to completion, queueing included"),
        "clocks": clocks,
    }
    del xs
    if not standalone:
        return line
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ PCA

PCA = dict(workload="pca_lowrank_decay_n1048576_p4096_m205_k20", n=1_048_576, p=4096, m=205,
           k=20, seed=7)


def run_pca(args, standalone=True):
    """Config 3: compress, then the three Gram paths on the same ELL rows
    (split-BF16, BF16, plain FP32 scatter), C_n and the top-20 subspace.
    Reports each path's time and tensor / HBM fraction, each Gram's relative
    Frobenius distance to the FP64 oracle's on a seeded row prefix (and, at
    full size, to the FP32 one), and the top-20 at the iteration count whose
    largest eigen-residual is <= 1e-6, with its time."""
    import numpy as np
    import torch
    from paper_1511_00152_gb300 import build as skbuild
    skbuild.build()
    from paper_1511_00152_gb300 import _lib as sk
    from paper_1511_00152_gb300 import synth
    cfg = dict(PCA)
    n, p, m, k = cfg["n"], cfg["p"], cfg["m"], cfg["k"]
    ctx = sk.sk_init(p, m, cfg["seed"])
    pt = ctx.pt
    X = synth.lowrank_decay_device(n, p, cfg["seed"])
    idx = torch.empty((n, m), dtype=torch.int32, device="cuda")
    val = torch.empty((n, m), dtype=torch.float32, device="cuda")
    hbm, bf16, bf16s, src = load_peaks()
    sampler = ClockSampler(torch.cuda.current_device())

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    reps = 3
    sampler.start()
    t_comp = timed(lambda: sk.sk_compress(ctx, X, idx=idx, val=val), reps)
    n0 = 20_000 if not args.no_cpu else 0
    X0 = X[:n0].cpu().numpy() if n0 else None
    del X
    torch.cuda.empty_cache()
    Gs, times = {}, {}
    N = 256
    ntiles = sum(pt // N - bi // (N // 128) for bi in range(pt // 128))
    for name, mode in (("bf16x3", sk.SK_GRAM_BF16X3), ("bf16", sk.SK_GRAM_BF16),
                       ("fp32", sk.SK_GRAM_FP32)):
        G = torch.zeros((pt, pt), dtype=torch.float64, device="cuda")
        wb = sk.sk_cov_workspace_bytes(ctx, mode, n)
        work = torch.empty(max(wb, 256), dtype=torch.uint8, device="cuda")

        def run(G=G, mode=mode, work=work):
            sk.sk_cov_reset(ctx, G)
            sk.sk_cov_accumulate(ctx, mode, idx, val, G, work=work)
        times[name] = timed(run, 1 if name == "fp32" else reps)
        Gs[name] = G
        del work
    U32 = torch.triu(Gs["fp32"])

    def fro(A):  # plain reduction (torch.linalg needs a library ncu cannot load)
        return float((A * A).sum().sqrt())
    rel32 = {nm: fro(torch.triu(Gs[nm]) - U32) / fro(U32) for nm in ("bf16x3", "bf16")}
    C = sk.sk_cov_finalize(ctx, Gs["bf16x3"], n)
    del Gs, U32
    torch.cuda.empty_cache()

    def residual(ev, U):
        Cu = C @ U.T
        return float((((Cu - U.T * ev[None, :]) ** 2).sum(0).sqrt() / ev.abs()).max())
    # the top-20 at the smallest tried iteration count that converges
    conv = None
    tried = {}
    for it in (20, 40, 60, 80, 120, 160, 240):
        ev, U = sk.sk_cov_topk(ctx, C, k, iters=it)
        tried[it] = residual(ev, U)
        if tried[it] <= 1e-6:
            conv = it
            break
    it_used = conv if conv is not None else max(tried)
    t_topk = timed(lambda: sk.sk_cov_topk(ctx, C, k, iters=it_used), 1)
    clocks = sampler.stop()
    assert sk.sk_device_status() == sk.SK_OK
    fl3 = 2.0 * n * 128 * N * ntiles * 3
    # each Gram path against the FP64 oracle on the first n0 rows (untimed)
    oracle_prefix = None
    if n0:
        import oracle
        oi, ov = oracle.compress(X0, m, cfg["seed"])
        Go = np.triu(oracle.gram(oi, ov, pt))
        nrm = np.linalg.norm(Go)
        oracle_prefix = {"rows": n0, "idx_exact": bool(np.array_equal(oi, idx[:n0].cpu().numpy()))}
        for name, mode in (("bf16x3", sk.SK_GRAM_BF16X3), ("bf16", sk.SK_GRAM_BF16),
                           ("fp32", sk.SK_GRAM_FP32)):
            G = torch.zeros((pt, pt), dtype=torch.float64, device="cuda")
            sk.sk_cov_accumulate(ctx, mode, idx[:n0].contiguous(), val[:n0].contiguous(), G)
            oracle_prefix[f"{name}_rel_frobenius"] = float(
                np.linalg.norm(np.triu(G.cpu().numpy()) - Go) / nrm)
            del G
    line = {
        "metric": "PCA workload: Gram paths (time, %tensor peak), error vs FP64, converged top-20",
        "value": n / ((t_comp + times["bf16x3"]) * 1e-3), "unit": "samples/s (compress + split-BF16 Gram)",
        "n_gpus": 1, "higher_is_better": True, "dtype": "f32+bf16x3", "data": "synthetic",
        "config": {"workload": cfg["workload"], "n": n, "p": p, "m": m, "k": k,
                   "l2": "inputs larger than L2 (X is 17.2 GB)"},
        "compress": {"ms": t_comp, "achieved_gbs": n * (4 * p + 8 * m) / (t_comp * 1e-3) / 1e9,
                     "frac_hbm": n * (4 * p + 8 * m) / (t_comp * 1e-3) / 1e9 / hbm,
                     "target_frac": 0.55},
        "gram_ms": times,
        "gram_tflops_issued": {"bf16x3": fl3 / (times["bf16x3"] * 1e-3) / 1e12,
                               "bf16": fl3 / 3 / (times["bf16"] * 1e-3) / 1e12},
        "gram_frac_sustained_bf16": {"bf16x3": fl3 / (times["bf16x3"] * 1e-3) / 1e12 / bf16s,
                                     "bf16": fl3 / 3 / (times["bf16"] * 1e-3) / 1e12 / bf16s,
                                     "target": 0.60},
        "gram_algorithmic_macs": n * m * (m + 1) // 2,
        "split_bf16_speedup_vs_fp32": times["fp32"] / times["bf16x3"],
        "rel_frobenius_vs_fp32_gram": rel32,
        "vs_fp64_oracle_prefix": oracle_prefix,
        "topk": {"ms": t_topk, "iters": it_used, "converged": conv is not None,
                 "max_rel_residual": tried[it_used], "residual_by_iters": tried},
        "peak_source": src, "clocks": clocks,
    }
    del C, idx, val
    if not standalone:
        return line
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ DCT

DCT = dict(workload="dct_mixture_n1e6_p784_m39_K10", n=1_000_000, p=784, m=39, K=10, iters=10,
           seed=784)


def run_dct(args, standalone=True):
    """The DCT preconditioner (no padding) on the paper's MNIST-sized samples
    (p = 784, gamma = 5%): compress against its HBM roofline (4p + 8m bytes
    per row), beside the Hadamard form of the same rows (zero-padded to 1024),
    and K-means iterations at pt = 784."""
    import torch
    from paper_1511_00152_gb300 import build as skbuild
    skbuild.build()
    from paper_1511_00152_gb300 import _lib as sk
    from paper_1511_00152_gb300 import pipeline, synth
    cfg = dict(DCT)
    n, p, m, K = cfg["n"], cfg["p"], cfg["m"], cfg["K"]
    X, _, _ = synth.mixture_device(n, p, K, cfg["seed"])
    hbm, bf16, bf16s, src = load_peaks()
    sampler = ClockSampler(torch.cuda.current_device())

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    ctx = sk.sk_init_ex(p, m, cfg["seed"], sk.SK_FLAG_DCT)
    ctx_h = sk.sk_init(p, m, cfg["seed"])
    idx = torch.empty((n, m), dtype=torch.int32, device="cuda")
    val = torch.empty((n, m), dtype=torch.float32, device="cuda")
    sampler.start()
    t_dct = timed(lambda: sk.sk_compress(ctx, X, idx=idx, val=val))
    t_had = timed(lambda: sk.sk_compress(ctx_h, X, idx=torch.empty_like(idx),
                                         val=torch.empty_like(val)))
    sk.sk_compress(ctx, X, idx=idx, val=val)
    rows = synth.init_rows(n, K, cfg["seed"])
    mu0 = sk.sk_precondition(ctx, X[torch.as_tensor(rows, device="cuda")].contiguous())
    st = pipeline.KMeansState(ctx, n, K)
    st.run(idx, val, mu0, cfg["iters"], use_graph=True)
    t_km = timed(lambda: st.run(idx, val, mu0, cfg["iters"], use_graph=True), reps=3)
    clocks = sampler.stop()
    assert sk.sk_device_status() == sk.SK_OK
    bytes_row = 4 * p + 8 * m
    line = {
        "metric": "DCT preconditioner (no padding): compress samples/s and %HBM, K-means iteration",
        "value": n / (t_dct * 1e-3), "unit": "samples/s (compress)", "n_gpus": 1,
        "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": cfg["workload"], "n": n, "p": p, "pt": ctx.pt, "m": m, "K": K,
                   "kmeans_iters": cfg["iters"]},
        "compress_dct": {"ms": t_dct, "achieved_gbs": n * bytes_row / (t_dct * 1e-3) / 1e9,
                         "frac_hbm": n * bytes_row / (t_dct * 1e-3) / 1e9 / hbm},
        "compress_hadamard_padded_1024": {"ms": t_had,
                                          "achieved_gbs": n * bytes_row / (t_had * 1e-3) / 1e9},
        "kmeans_iter_ms": t_km / cfg["iters"],
        "kmeans_frac_hbm": n * (8 * m + 8) / (t_km / cfg["iters"] * 1e-3) / 1e9 / hbm,
        "peak_source": src, "clocks": clocks,
    }
    del X, idx, val, st
    if not standalone:
        return line
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ batching

BATCHING = dict(workload="batch64_mixtures_p256-8192_n1e4-5e5", datasets=64, iters=15,
                seed=4242)


def batching_sets(cfg):
    """64 seeded data-set shapes: p from {256, ..., 8192}, n log-uniform in
    [1e4, 5e5], m / p in {2%, 5%, 10%}, K in [5, 50]."""
    import numpy as np
    rng = np.random.default_rng(cfg["seed"])
    out = []
    for d in range(cfg["datasets"]):
        p = int(2 ** rng.integers(8, 14))
        n = int(np.exp(rng.uniform(np.log(1e4), np.log(5e5))))
        gamma = float(rng.choice([0.02, 0.05, 0.10]))
        m = max(2, int(round(gamma * p)))
        K = int(rng.integers(5, 51))
        out.append(dict(n=n, p=p, m=m, K=K, seed=cfg["seed"] * 1000 + d))
    return out


def run_batching(args, standalone=True):
    """Config 4: 64 data sets through compress, BF16 Gram and 15 K-means
    iterations, one launch per stage for all data sets (the K-means loop as a
    CUDA graph), tiles picked by the library's autotuner.  Reports samples/s
    over all rows and the step time against the sum of the per-data-set
    roofline times of the three stages."""
    import torch
    from paper_1511_00152_gb300 import build as skbuild
    skbuild.build()
    from paper_1511_00152_gb300 import _lib as sk
    from paper_1511_00152_gb300 import pipeline, synth
    cfg = dict(BATCHING)
    shapes = batching_sets(cfg)
    ds = []
    for sh in shapes:
        X, _, _ = synth.mixture_device(sh["n"], sh["p"], sh["K"], sh["seed"], heavy_frac=0.0)
        ds.append(dict(X=X, m=sh["m"], K=sh["K"], seed=sh["seed"]))
    torch.cuda.synchronize()
    br = pipeline.BatchRun(ds, mode=sk.SK_GRAM_BF16)
    tuning = br.autotune()
    iters = cfg["iters"]
    stream = torch.cuda.current_stream()

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        br.compress_and_cov()
        if ev is not None:
            ev[1].record(stream)
        br.init_centres()
        br.kmeans(iters, use_graph=True)
        if ev is not None:
            ev[2].record(stream)

    for _ in range(max(args.warmup if standalone else 1, 1)):
        step()
    torch.cuda.synchronize()
    steps = args.steps if standalone else min(args.steps, 3)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(0)
    sampler.start()
    a.record(stream)
    for k in range(steps):
        step(evs[k])
    b.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = a.elapsed_time(b) / steps
    t_cc = sum(e[0].elapsed_time(e[1]) for e in evs) / steps
    t_km = sum(e[1].elapsed_time(e[2]) for e in evs) / steps
    assert sk.sk_device_status() == sk.SK_OK
    hbm, bf16, bf16s, src = load_peaks()
    rows = sum(sh["n"] for sh in shapes)
    # summed roofline times: compress and K-means passes on HBM bytes, the
    # Gram on the tensor-core work it issues (128 x N tiles over all rows)
    tn = tuning[1]
    comp_b = sum(sh["n"] * (4 * sh["p"] + 8 * sh["m"]) for sh in shapes)
    km_b = iters * sum(sh["n"] * (8 * sh["m"] + 8) for sh in shapes)
    flops = 0.0
    for sh in shapes:
        pt = sh["p"]
        N = tn if pt >= tn else pt
        tiles = sum(pt // N - bi // (N // 128) for bi in range(pt // 128))
        flops += 2.0 * sh["n"] * 128 * N * tiles
    t_roof = (comp_b / (hbm * 1e9) + km_b / (hbm * 1e9) + flops / (bf16s * 1e12)) * 1e3
    line = {
        "metric": "samples/s of many data sets, one launch per stage (compress+BF16 Gram+"
                  "15 K-means iters)",
        "value": rows / (ms * 1e-3), "unit": "samples/s", "n_gpus": 1, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "dtype": "f32+bf16", "data": "synthetic",
        "config": {"workload": cfg["workload"], "datasets": len(shapes), "rows": rows,
                   "kmeans_iters": iters, "gram": "bf16", "seed": cfg["seed"],
                   "autotuned": {"compress_units_per_group": tuning[0],
                                 "gram_tile_n": tuning[1]}},
        "stage_ms": {"compress_and_gram": t_cc, "kmeans_start_and_loop": t_km},
        "roofline": {"bound": "mixed (sum of per-data-set rooflines)",
                     "time_ms": t_roof, "achieved_frac": t_roof / ms,
                     "compress_bytes": comp_b, "kmeans_bytes": km_b, "gram_flops": flops,
                     "peak_hbm_gbs": hbm, "peak_bf16_tflops": bf16s, "peak_source": src},
        "clocks": clocks,
        # per K-means iteration: the pass (one launch for the data sets whose
        # centre table fits shared memory, one for the others) and the finalize
        "gpu_launches_per_step": 1 + 2 + len(shapes) + 1 + 3 * iters,
    }
    del br, ds
    if not standalone:
        return line
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--gram", default="bf16x3", choices=["fp32", "bf16", "bf16x3"])
    ap.add_argument("--topk-iters", type=int, default=4)
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--cpu-rows", type=int, default=200_000)
    ap.add_argument("--ref-rows", type=int, default=20_000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-chunks", type=int, default=8,
                    help="chunks of X per end-to-end step (host-to-device copy ring)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-plain", action="store_true",
                    help="skip timing the plain FP32 Gram beside the chosen mode")
    ap.add_argument("--no-extra", action="store_true",
                    help="default run: skip the PCA, serving and batching workloads that "
                         "follow the main step")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch the K-means loop kernel by kernel (for profilers)")
    ap.add_argument("--workload", default="kmeans",
                    choices=["kmeans", "serving", "batching", "pca", "dct"],
                    help="kmeans: the main step (default); serving: the streaming request loop; "
                         "batching: 64 data sets, one launch per stage; pca: the PCA workload; "
                         "dct: the DCT preconditioner at p = 784")
    args = ap.parse_args()
    if args.workload == "serving" and args.impl != "reference":
        return run_serving(args)
    if args.workload == "batching" and args.impl != "reference":
        return run_batching(args)
    if args.workload == "pca" and args.impl != "reference":
        return run_pca(args)
    if args.workload == "dct" and args.impl != "reference":
        return run_dct(args)
    cfg = dict(WORKLOAD)
    if args.n:
        cfg["n"] = args.n
    if args.impl == "reference":
        return run_reference(args, cfg)
    return run_gpu(args, cfg)


if __name__ == "__main__":
    sys.exit(main())
