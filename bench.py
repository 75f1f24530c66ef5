#!/usr/bin/env python3
"""Throughput of the bipartite H|psi> on one GB300 (or N replicas).

Default workload: J1-J2 Heisenberg on the 4x8 torus, J1=1, J2=0.5, Sz=0
(601,080,390 states, 17 blocks, cut 16|16), FP64 storage.  One step = one
H|psi> of the whole sector vector (input and output 4.8 GB each, far larger
than L2, so no flush is needed between steps).  The JSON line also carries
the FP32 H|psi> rate, Lanczos time-to-E0 for plain FP64 vs mixed precision,
an end-to-end rate through the C ABI with host buffers, the roofline of the
apply kernel and the oracle's CPU rate on a bounded sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "H psi/s & HBM GB/s vs peak, 4x8 J1-J2 Sz=0; time-to-E0(1e-10) mixed vs FP64"
UNIT = "Hpsi/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--config", default="j1j2_4x8", choices=list(W.CONFIG_NAMES))
    p.add_argument("--dtype", default="f64", choices=["f64", "f32"])
    p.add_argument("--no-lanczos", action="store_true", help="skip the time-to-E0 comparison")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    p.add_argument("--lanczos-max-iter", type=int, default=400)
    p.add_argument("--no-batched", action="store_true", help="skip the batched and serving measurements")
    p.add_argument("--batch-n", type=int, default=512)
    p.add_argument("--serve-rate", type=float, default=4000.0, help="Poisson arrival rate (requests/s)")
    p.add_argument("--pipes", action="store_true", help="build and run the pipe-rate microbenchmark, then exit")
    p.add_argument("--dense-only", action="store_true",
                   help="run only the dense-block (digit-split tensor-core) measurement and print it")
    p.add_argument("--batched-only", action="store_true",
                   help="run only the batched measurement (no serving sweep) and print it")
    p.add_argument("--no-configs", action="store_true", help="skip the Heis16 / Hub12 / Hub4x4 measurements")
    p.add_argument("--no-entangle", action="store_true", help="skip the entanglement spectrum of the ground state")
    p.add_argument("--no-dense", action="store_true", help="skip the dense-block (DMRG-style) H psi")
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def shard(n: int, rank: int, world: int):
    """Instances handled by `rank` when n independent instances are spread
    over `world` ranks (round robin; no data exchange between ranks)."""
    return list(range(rank, n, world))


def max_over_ranks(value: float, world: int, device: str = "cpu") -> float:
    """Largest value over all ranks (the slowest rank sets the job time)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, world: int, device: str = "cpu") -> float:
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# Digit-split tensor-core GEMM (the dense-block products and the Gram
# matrices): each FP64 product runs as 36 BF16 digit-pair products (digit
# orders p + q <= 7 of 8 digits) on 128 x 64 output tiles with K in steps of
# 64; the BF16 FLOPs it executes are counted on those padded tiles.
OZ_PAIRS = 36

# pieces (and streams) per host<->device copy in the end-to-end pipeline
E2E_CHUNKS = 4


def oz_tensor_flops(M, N, K, tri=False):
    """BF16 FLOPs the tensor cores execute for one digit-split product."""
    tm, tn, tk = -(-M // 128), -(-N // 64), -(-K // 64)
    tiles = sum(min(tn, 2 * (i + 1)) for i in range(tm)) if tri else tm * tn
    return 2.0 * tiles * 128 * 64 * tk * 64 * OZ_PAIRS


def bf16_peak():
    peaks, src = measured_peaks()
    return float(peaks.get("bf16_tflops", 1900.0)), src


def entanglement_section(ed, ctx):
    """Ground state (mixed precision, FP64 vector), then its entanglement
    spectrum across the cut: time, the Gram kernels' FP64 rate against the
    FP64 peak, sector weights W_q and the effective numbers of sectors
    1 / sum_q w_q^2 (by weight and by block dimension)."""
    import torch

    psi = torch.empty(ctx.dim, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = ed.lanczos_ground(ctx, mode="mixed", tol=1e-12, psi0=psi)
    torch.cuda.synchronize()
    t_gs = time.perf_counter() - t0
    t0 = time.perf_counter()
    es = ed.entanglement_spectrum(ctx, psi)
    t_es = time.perf_counter() - t0
    s, dA, dB, _ = ctx.blocks()
    m = np.minimum(dA, dB).astype(np.float64)
    L = np.maximum(dA, dB).astype(np.float64)
    macs = float(np.sum(m * (m + 1) / 2 * L))  # lower triangle with the diagonal
    tflops = sum(oz_tensor_flops(int(a), int(a), int(b), tri=True) for a, b in zip(m, L))
    gram_ms, eig_ms = es.stage_ms
    tot = float(es.weight.sum())
    W = es.weight / tot
    w_dim = (dA * dB) / float(np.sum(dA * dB))
    xi_low = [float(-np.log(l[0] / tot)) if len(l) and l[0] > 0 else None for l in es.lam]
    peak, src = bf16_peak()
    achieved = tflops / (gram_ms * 1e-3) / 1e12 if gram_ms > 0 else None
    # the reduction's dominant traffic: every column's product reads the
    # float-float trailing triangle (8 bytes an entry) once; over the whole
    # stage (every kernel of it in the time) this is a lower bound of the
    # product kernel's rate
    f_bytes = 0.0
    for mb in m:
        n = np.arange(int(mb) - 3, -1, -1, dtype=np.float64) + 2.0 if mb >= 3 else np.zeros(0)  # n = m - c - 1
        f_bytes += float(np.sum(n * (n + 1) / 2)) * 8.0
    peaks, psrc = measured_peaks()
    stream_gbs = f_bytes / (eig_ms * 1e-3) / 1e9 if eig_ms > 0 else None
    eig_stream = {"bytes": f_bytes, "achieved": stream_gbs, "unit": "GB/s", "peak": peaks["hbm_gbs"],
                  "frac": stream_gbs / peaks["hbm_gbs"] if stream_gbs else None, "peak_source": psrc,
                  "note": "float-float triangle bytes the per-column products read, over the whole eigenvalue "
                          "stage's device time (panel kernels and trailing updates included)"}
    return {"ground_state_s": t_gs, "e0": r.e0, "seconds": t_es, "gram_ms": gram_ms, "eigensolver_ms": eig_ms,
            "gram_fp64_equiv_tflops": 2 * macs / (gram_ms * 1e-3) / 1e12 if gram_ms > 0 else None,
            "gram_roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                              "frac": achieved / peak if achieved else None, "flops": tflops,
                              "peak_source": f"{src} BF16 (burst)",
                              "note": "BF16 FLOPs executed by the digit-split products (36 digit pairs, padded "
                                      "tiles, the tiles on or below the diagonal)"},
            "eigensolver_stream": eig_stream,
            "entropy": es.entropy, "s": [int(v) for v in s], "W_q": [float(v) for v in W],
            "xi_lowest_per_sector": xi_low, "n_eff_weights": float(1.0 / np.sum(W ** 2)),
            "n_eff_dims": float(1.0 / np.sum(w_dim ** 2)), "levels": int(sum(len(l) for l in es.lam))}


def dense_blocks_section(ed):
    """Dense-block H|psi> (DMRG-style side operators) on the paper's block-size
    laws chi_q = C e^{-alpha |q - q0|}, sum chi about 4000, 21 sectors, two
    adjoint pairs of cross terms: device time per apply (CUDA events) and the
    FP64 FLOP rate against the FP64 peak (parity is checked by the tests)."""
    import torch

    import workloads.dense as WD

    out = {}
    peak, src = bf16_peak()
    for alpha in (0.95, 0.15, 1.11):
        m = WD.dense_config(alpha)
        op = ed.DenseOperator(m)
        flops = 0.0   # FP64-equivalent (2 M N K per product)
        tflops = 0.0  # BF16 FLOPs the tensor cores execute
        for c in m.chi.astype(np.int64):
            flops += 4.0 * float(c) ** 3
            tflops += 2 * oz_tensor_flops(int(c), int(c), int(c))
        for d, Ls in zip(m.delta, m.Lm):
            for q, l in enumerate(Ls):
                if l is not None:
                    ct, c = l.shape
                    flops += 2.0 * ct * c * c + 2.0 * ct * ct * c
                    tflops += oz_tensor_flops(ct, c, c) + oz_tensor_flops(ct, ct, c)
        rng = np.random.default_rng(3)
        x = rng.standard_normal(m.dim)
        xd = torch.tensor(x, device="cuda")
        yd = torch.empty_like(xd)
        for _ in range(2):
            op.apply(xd, yd)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(5):
            op.apply(xd, yd)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 5
        ach = tflops / (ms * 1e-3) / 1e12
        out[f"alpha_{alpha}"] = {"chi_max": int(m.chi.max()), "sum_chi": int(m.chi.sum()), "states": m.dim,
                                 "ms": ms, "fp64_equiv_tflops": flops / (ms * 1e-3) / 1e12, "fp64_flops": flops,
                                 "roofline": {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                                              "frac": ach / peak, "flops": tflops,
                                              "peak_source": f"{src} BF16 (burst)"}}
        op.close()
        del xd, yd
    return out


def kernel_source_hash():
    h = hashlib.sha256()
    for fn in ("apply3.cu", "apply3.cuh", "ed_internal.h",
               "ops.cpp", "sectors.cpp"):
        with open(os.path.join(ROOT, "paper_2605_07621_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [s.strip() for s in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        load = sorted(sm)
        return {"sm_mhz": float(np.median(load)) if load else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def oracle_row_sample(D: int, n_rows: int, seed: int = 20260507, n_chunks: int = 64):
    """Rows of a bounded oracle sample spread over the whole sector: n_chunks
    runs of consecutive rows (so each run keeps the locality a full pass has)
    starting at seeded random positions, at most n_rows rows in all."""
    n_rows = int(max(1, min(D, n_rows)))
    n_chunks = int(max(1, min(n_chunks, n_rows)))
    clen = max(1, n_rows // n_chunks)
    rng = np.random.default_rng(seed)
    slots = max(1, D // clen)
    starts = np.sort(rng.choice(slots, size=min(n_chunks, slots), replace=False)) * clen
    rows = (starts[:, None] + np.arange(clen)[None, :]).ravel()
    return rows[rows < D].astype(np.int64)


class OracleSample:
    """The oracle's H|psi> on the host cores over a bounded row sample of one
    workload: keys enumerated and the lookup index built once (both timed
    apart from the rows), then listed rows evaluated by all threads."""

    def __init__(self, model, budget_s: float, seed: int = 20260507):
        import oracle

        self.cores = len(os.sched_getaffinity(0))
        t0 = time.time()
        self.keys = oracle.sector_keys(model)
        self.t_keys = time.time() - t0
        self.D = len(self.keys)
        t0 = time.time()
        self.ix = oracle.RowIndex(model, self.keys)
        self.t_index = time.time() - t0
        # x = the key-indexed start vector is not needed for timing; ones keep
        # every term's work identical
        self.x = np.ones(self.D)
        probe = oracle_row_sample(self.D, min(self.D, 20000), seed + 1)
        t0 = time.time()
        self.ix.apply_rows(self.x, probe, nthreads=self.cores)
        rate = len(probe) / max(time.time() - t0, 1e-6)
        self.rows = oracle_row_sample(self.D, int(rate * budget_s), seed)

    def run(self):
        return self.ix.apply_rows(self.x, self.rows, nthreads=self.cores)

    def describe(self):
        return (f"{len(self.rows)} rows of {self.D} ({len(self.rows) / self.D:.2e} of one H psi) in 64 runs of "
                f"consecutive rows at seeded random positions (seed 20260507) across the whole sector; key list "
                f"({self.t_keys:.1f} s) and lookup index ({self.t_index:.2f} s) built once outside the timing; "
                f"{self.cores} threads")


def cpu_baseline(model, budget_s: float = 12.0):
    """The oracle's H|psi> rows on the host cores, bounded sample, scaled to H psi/s."""
    smp = OracleSample(model, budget_s)
    smp.run()  # warm caches and pages
    t0 = time.time()
    smp.run()
    dt = time.time() - t0
    rows_per_s = len(smp.rows) / dt
    value = rows_per_s / smp.D
    # a whole H psi by the oracle would also build its index once
    with_index = 1.0 / (smp.D / rows_per_s + smp.t_index)
    return {"value": value, "unit": UNIT, "cores": smp.cores, "kind": "oracle", "sample": smp.describe(),
            "rows_per_s": rows_per_s, "index_build_s": smp.t_index, "value_with_index_build": with_index}


def batched_and_served(ed, n: int, rate: float, seed: int = 20260507, rank: int = 0, world: int = 1,
                       serve: bool = True):
    """512 independent Hubbard instances (this rank's share when several GPUs
    run): one batched Lanczos solve, then the same instances as a Poisson
    stream of requests to the serving loop."""
    import torch

    all_models = W.batched_hubbard_instances(n, seed)
    models = [all_models[i] for i in shard(n, rank, world)]
    n = len(models)
    t0 = time.perf_counter()
    b = ed.batch_create(models)
    t_create = time.perf_counter() - t0
    modes, tune = b.info()
    # one batched H|psi> over all instances (FP32), device-timed
    x = torch.ones(b.dim, dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    ed.batch_apply(b, x, y)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(5):
        ed.batch_apply(b, x, y)
    e1.record()
    torch.cuda.synchronize()
    apply_ms = e0.elapsed_time(e1) / 5
    # roofline of the batched apply: HBM bytes of read x + write y (FP32),
    # and the tensor-core FLOPs of the dense instances (six BF16 piece
    # products per multiply-add of H_A Psi + Psi H_B^T) over the whole apply
    from math import comb
    dims = [(comb(m.n_sites, m.n_up), comb(m.n_sites, m.n_dw)) for m in models]
    D = sum(a * bb for a, bb in dims)
    dense_flops = sum(6 * 2 * a * bb * (a + bb) for (a, bb), md in zip(dims, modes) if md > 0)
    peaks, peak_src = measured_peaks()
    gbs = 8 * D / (apply_ms * 1e-3) / 1e9
    tfl = dense_flops / (apply_ms * 1e-3) / 1e12
    apply_roof = {"hbm": {"achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
                          "bytes": 8 * D, "peak_source": peak_src},
                  "tensor": {"achieved": tfl, "peak": bf16_peak()[0], "unit": "TFLOP/s",
                             "frac": tfl / bf16_peak()[0], "flops": dense_flops, "peak_source": bf16_peak()[1],
                             "note": "BF16 piece products of the dense instances over the whole apply time"}}
    t0 = time.perf_counter()
    e, it, info = ed.batch_lanczos(b, tol=1e-7)
    t_solve = time.perf_counter() - t0
    batched = {"workload": f"{n} Hubbard instances (8-12 sites, random fillings, U, t', eps)", "states": int(b.dim),
               "create_s": t_create,
               "modes": {"csr": int(np.sum(modes == 0)), "dense_64": int(np.sum(modes == 1)),
                         "dense_128": int(np.sum(modes == 2))},
               "tune_ms": {"all_csr": float(tune[0]), "all_dense_64": float(tune[1]),
                           "all_dense_128": float(tune[2]), "tuned": float(tune[3])},
               "apply_ms": apply_ms, "apply_roofline": apply_roof, "solve_s": t_solve, "instances_per_s": n / t_solve,
               "hpsi_per_s_aggregate": float(np.sum(it)) / t_solve, "steps": info["steps"],
               "all_converged": info["all_converged"], "storage": "f32", "reductions": "f64"}
    del x, y, b
    if not serve:
        return batched, None
    # served: Poisson arrivals, continuous batching, arrival rate swept up to
    # `rate` (the last, highest rate is the headline entry)
    sweep = []
    for k, r_k in enumerate((rate / 8, rate / 4, rate / 2, rate)):
        rng = np.random.default_rng(seed + 1 + k)
        srv = ed.Server(device_bytes=8 << 30, max_slots=512, check_every=5, tol=1e-7)
        gaps = rng.exponential(1.0 / r_k, n)
        tickets = []
        t0 = time.perf_counter()
        nxt = t0
        for m, g in zip(models, gaps):
            nxt += g
            while time.perf_counter() < nxt:
                pass
            tickets.append(srv.submit(m))
        res = [srv.wait(t, 600000) for t in tickets]
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        lat = np.array([r["latency_s"] for r in res])
        same = float(np.max(np.abs(np.array([r["e0"] for r in res]) - e)))
        sweep.append({"arrival_rate_rps": r_k, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                      "p99_ms": 1e3 * float(np.percentile(lat, 99)), "throughput_rps": n / wall,
                      "failed": int(st["failed"]), "max_abs_diff_vs_batched_e0": same})
    served = dict(sweep[-1])
    served.update({"requests": n, "max_slots": 512, "sweep": sweep})
    return batched, served


def other_configs(ed):
    """The other workloads: Heis16 (150 fixed steps), Hub12 (ground state FP64
    and mixed, G on 2048 frequencies), Hub4x4 (H psi rates, ground state FP64
    and mixed to 1e-10, G on 4096 frequencies with 400 steps, eta = 0.05)."""
    import torch

    out = {}

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return r, time.perf_counter() - t0

    # the headline lattice with a coupling that is not a dyadic rational
    # (J2 = 0.3): fixed-point class sums with 64-bit integer weights, exact 128-bit sums
    ctx = ed.build_local_ops(ed.build_sectors(W.j1j2_torus(8, 4, 1.0, 0.3, 16, 0xFFFF)))
    x = torch.empty(ctx.dim, dtype=torch.float64, device="cuda")
    ed.random_vector(ctx, x)
    y = torch.empty_like(x)
    ed.apply_H(ctx, x, y)
    _, t1 = timed(lambda: [ed.apply_H(ctx, x, y) for _ in range(5)])
    out["j1j2_4x8_j2_0.3"] = {"states": ctx.dim, "hpsi_per_s_f64": 5 / t1, "ms_per_hpsi": 1e3 * t1 / 5,
                              "fp64_mode": ctx.fp64_mode()}
    del x, y, ctx
    torch.cuda.empty_cache()
    ctx = ed.build_local_ops(ed.build_sectors(W.config_heis16()))
    r, dt = timed(lambda: ed.lanczos_ground(ctx, mode="f64", max_iter=150, fixed_iter=True))
    out["heis16"] = {"states": ctx.dim, "e0_150": r.e0, "seconds_150_steps": dt, "us_per_step": 1e6 * dt / 150}
    for name, n_om, n_it in (("hub12", 2048, 300), ("hub4x4", 4096, 400), ("qim15", 2048, 300)):
        m = W.config_by_name(name)
        ctx = ed.build_local_ops(ed.build_sectors(m))
        rec = {"states": ctx.dim}
        x = torch.empty(ctx.dim, dtype=torch.float64, device="cuda")
        ed.random_vector(ctx, x)
        for dt_ in (torch.float64, torch.float32):
            xx = x.to(dt_)
            yy = torch.empty_like(xx)
            ed.apply_H(ctx, xx, yy)
            _, t1 = timed(lambda: [ed.apply_H(ctx, xx, yy) for _ in range(5)])
            rec["hpsi_per_s_" + ("f64" if dt_ == torch.float64 else "f32")] = 5 / t1
            del xx, yy
        del x
        for mode in ("f64", "mixed"):
            r, t1 = timed(lambda: ed.lanczos_ground(ctx, mode=mode, tol=1e-12))
            rec[f"e0_{mode}"] = r.e0
            rec[f"time_to_e0_{mode}_s"] = t1
            rec[f"iterations_{mode}"] = r.iterations
        rec["mixed_vs_f64_rel"] = abs(rec["e0_mixed"] - rec["e0_f64"]) / abs(rec["e0_f64"])
        psi = torch.empty(ctx.dim, dtype=torch.float64, device="cuda")
        r, t1 = timed(lambda: ed.lanczos_ground(ctx, mode="mixed", tol=1e-12, psi0=psi))
        rec["ground_vector_s"] = t1
        omega = np.linspace(-15.0, 15.0, n_om)
        (G, co), t2 = timed(lambda: ed.lanczos_gf(ctx, psi, r.e0, omega, 0.05, site=0, spin=0, n_iter=n_it))
        rec["gf"] = {"n_omega": n_om, "n_iter": n_it, "eta": 0.05, "seconds": t2,
                     "sum_rule": co["particle"][0] + co["hole"][0], "max_im_G": float(G.imag.max())}
        out[name] = rec
        del psi, ctx
        torch.cuda.empty_cache()
    return out


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    model = W.config_by_name(args.config)
    # each step: about 4 s of oracle rows, so warm-up + timed steps end in minutes
    smp = OracleSample(model, budget_s=4.0)
    for _ in range(args.warmup):
        smp.run()
    t0 = time.time()
    for _ in range(args.steps):
        smp.run()
    dt = time.time() - t0
    value = args.steps * (len(smp.rows) / smp.D) / dt
    sample = "each step: " + smp.describe() + ", scaled to H psi/s"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": args.config, "states": smp.D, "l2_flush": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": smp.cores, "kind": "oracle", "sample": sample,
                             "index_build_s": smp.t_index},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_pipes():
    src = os.path.join(ROOT, "paper_2605_07621_gb300", "microbench", "pipes.cu")
    exe = os.path.join(tempfile.mkdtemp(), "pipes")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe, src])
    print(subprocess.check_output([exe], text=True).strip(), flush=True)


def main():
    args = parse()
    if args.pipes:
        return run_pipes()
    if args.impl == "reference":
        return run_reference(args)
    import torch

    if args.dense_only:
        import paper_2605_07621_gb300 as ed

        print(json.dumps(dense_blocks_section(ed)), flush=True)
        return
    if args.batched_only:
        import paper_2605_07621_gb300 as ed

        print(json.dumps(batched_and_served(ed, args.batch_n, args.serve_rate, serve=False)[0]), flush=True)
        return
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    import paper_2605_07621_gb300 as ed

    model = W.config_by_name(args.config)
    t0 = time.time()
    ctx = ed.build_local_ops(ed.build_sectors(model))
    t_setup = time.time() - t0
    D = ctx.dim
    tdt = torch.float64 if args.dtype == "f64" else torch.float32
    esz = 8 if args.dtype == "f64" else 4
    stream = torch.cuda.current_stream()
    x = torch.empty(D, dtype=torch.float64, device=dev)
    ed.random_vector(ctx, x, seed=W.DEFAULT_SEED)
    if tdt != torch.float64:
        x = x.to(tdt)
    y = torch.empty_like(x)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    for _ in range(max(args.warmup, 0)):
        ed.apply_H(ctx, x, y)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device() if ws == 1 else local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    ctx.profile(True)
    ctx.profile_read(reset=True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ed.apply_H(ctx, x, y)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    stage_ms, n_prof = ctx.profile_read(reset=True)
    ctx.profile(False)
    stage_ms = stage_ms / max(n_prof, 1)
    t_max = max_over_ranks(ms, ws, device=str(dev))
    ms_per_step = t_max / args.steps
    value = ws * args.steps / (t_max / 1000.0)

    # the other precision, same workload (not part of the headline)
    other = {}
    odt = torch.float32 if tdt == torch.float64 else torch.float64
    xo = x.to(odt)
    yo = torch.empty_like(xo)
    for _ in range(2):
        ed.apply_H(ctx, xo, yo)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(max(3, args.steps // 2)):
        ed.apply_H(ctx, xo, yo)
    e1.record(stream)
    torch.cuda.synchronize()
    oms = e0.elapsed_time(e1) / max(3, args.steps // 2)
    other = {"dtype": "f32" if odt == torch.float32 else "f64", "hpsi_per_s": 1000.0 / oms, "ms_per_hpsi": oms,
             "algorithmic_gbs": 2 * D * (4 if odt == torch.float32 else 8) / (oms * 1e-3) / 1e9}
    del xo, yo

    peaks, peak_src = measured_peaks()
    alg_bytes = 2 * D * esz
    achieved = alg_bytes / (ms_per_step * 1e-3) / 1e9
    traffic = whole_traffic = None
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            tr = json.load(f)
        ent = tr.get(f"{args.config}:{args.dtype}")
        if ent and ent.get("kernel_hash") == kernel_source_hash():
            traffic = ent["dram_bytes_per_launch"]
        ent = tr.get(f"{args.config}:{args.dtype}:whole_apply")
        if ent and ent.get("kernel_hash") == kernel_source_hash():
            whole_traffic = ent["dram_bytes_per_apply"]
    except Exception:
        traffic = whole_traffic = None
    # dominant kernel: the row pass (stage 2) -- reads every row of x once and
    # writes every element of y once, i.e. the algorithmic bytes of H|psi>
    names = ["k_exp_max", "k_to_fixed", ctx.row_pass(tdt), "k_panel4"]
    dom = int(np.argmax(stage_ms))
    dom_ms = float(stage_ms[dom])
    achieved_dom = alg_bytes / (dom_ms * 1e-3) / 1e9 if dom_ms > 0 else None
    roof = {"bound": "hbm", "achieved": achieved_dom, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": (achieved_dom / peaks["hbm_gbs"]) if achieved_dom else None, "traffic": traffic,
            "peak_source": peak_src, "kernel": names[dom], "kernel_ms": dom_ms,
            "algorithmic_bytes_per_launch": alg_bytes,
            "stage_ms": {n: float(v) for n, v in zip(names, stage_ms)},
            "whole_apply": {"achieved": achieved, "frac": achieved / peaks["hbm_gbs"], "ms": ms_per_step,
                            "traffic": whole_traffic,
                            "traffic_vs_algorithmic": (whole_traffic / alg_bytes) if whole_traffic else None}}

    # end to end through the C ABI with host buffers: H2D x, H psi, D2H y
    e2e = None
    if not args.no_e2e:
        xh = torch.empty(D, dtype=tdt, pin_memory=True)
        yh = torch.empty(D, dtype=tdt, pin_memory=True)
        xh.copy_(x)
        n_e2e = max(20, args.steps)  # the three-stream pipeline fills and drains once per run
        # untimed warm-up steps: the first host<->device copies of freshly
        # pinned buffers run at a fraction of the link rate
        for _ in range(max(2, args.warmup)):
            x.copy_(xh, non_blocking=True)
            ed.apply_H(ctx, x, y)
            yh.copy_(y, non_blocking=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0.record(stream)
        for _ in range(n_e2e):
            x.copy_(xh, non_blocking=True)
            ed.apply_H(ctx, x, y)
            yh.copy_(y, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        serial = {"value": n_e2e / wall, "device_ms_per_step": e0.elapsed_time(e1) / n_e2e}
        # the same steps pipelined (H2D of step i+1, H psi of step i and D2H
        # of step i-1 overlap; two device buffer pairs); each copy is split
        # into E2E_CHUNKS pieces on as many streams, since one copy of a large
        # buffer runs on a single copy engine
        xs, ys = [x, torch.empty_like(x)], [y, torch.empty_like(y)]
        s_in = [torch.cuda.Stream() for _ in range(E2E_CHUNKS)]
        s_out = [torch.cuda.Stream() for _ in range(E2E_CHUNKS)]
        s_cmp = torch.cuda.Stream()
        cb = -(-D // E2E_CHUNKS)
        parts = [(q * cb, min(D, (q + 1) * cb)) for q in range(E2E_CHUNKS)]
        ev_in = [[torch.cuda.Event() for _ in range(E2E_CHUNKS)] for _ in range(n_e2e)]
        ev_cmp = [torch.cuda.Event() for _ in range(n_e2e)]
        ev_out = [[torch.cuda.Event() for _ in range(E2E_CHUNKS)] for _ in range(n_e2e)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(n_e2e):
            k = i % 2
            for q, (a, b) in enumerate(parts):
                with torch.cuda.stream(s_in[q]):
                    if i >= 2:
                        s_in[q].wait_event(ev_cmp[i - 2])
                    xs[k][a:b].copy_(xh[a:b], non_blocking=True)
                    ev_in[i][q].record(s_in[q])
            with torch.cuda.stream(s_cmp):
                for q in range(E2E_CHUNKS):
                    s_cmp.wait_event(ev_in[i][q])
                    if i >= 2:
                        s_cmp.wait_event(ev_out[i - 2][q])
                ed.apply_H(ctx, xs[k], ys[k], stream=s_cmp)
                ev_cmp[i].record(s_cmp)
            for q, (a, b) in enumerate(parts):
                with torch.cuda.stream(s_out[q]):
                    s_out[q].wait_event(ev_cmp[i])
                    yh[a:b].copy_(ys[k][a:b], non_blocking=True)
                    ev_out[i][q].record(s_out[q])
        torch.cuda.synchronize()
        wall_p = time.perf_counter() - t0
        e2e = {"value": n_e2e / wall_p, "unit": UNIT, "h2d_bytes_per_step": D * esz, "d2h_bytes_per_step": D * esz,
               "steps": n_e2e,
               "pipelined": f"H2D / H psi / D2H overlapped, two device buffer pairs, each copy in {E2E_CHUNKS} "
                            "pieces on as many streams",
               "serial": serial}
        del xh, yh, xs, ys

    # Lanczos time-to-E0: plain FP64 vs FP32 + FP64 refinement
    lanczos = None
    if not args.no_lanczos and rank == 0:
        del x, y
        torch.cuda.empty_cache()
        lanczos = {}
        for mode in ("f64", "mixed"):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = ed.lanczos_ground(ctx, mode=mode, tol=1e-12, max_iter=args.lanczos_max_iter)
            wall = time.perf_counter() - t0
            lanczos[mode] = {"e0": r.e0, "seconds": wall, "iterations": r.iterations,
                             "iterations_fp32": r.iterations_low, "restarts": r.restarts,
                             "converged": r.converged}
        lanczos["mixed_vs_f64_rel"] = abs(lanczos["mixed"]["e0"] - lanczos["f64"]["e0"]) / abs(lanczos["f64"]["e0"])
        lanczos["speedup_mixed"] = lanczos["f64"]["seconds"] / lanczos["mixed"]["seconds"]
        # the reference energy of "time-to-E0(1e-10)": FP64 Lanczos until the
        # Ritz value changes by less than 1e-14 (relative) over 10 steps, with
        # its Ritz vector's residual ||Hx - Ex|| / |E| checked below 1e-7
        psi = torch.empty(D, dtype=torch.float64, device=dev)
        t0 = time.perf_counter()
        rr = ed.lanczos_ground(ctx, mode="f64", tol=1e-14, check_every=10, max_iter=600, psi0=psi)
        t_ref = time.perf_counter() - t0
        hx = torch.empty_like(psi)
        ed.apply_H(ctx, psi, hx)
        res = float(torch.linalg.norm(hx - rr.e0 * psi) / abs(rr.e0))
        del hx, psi
        torch.cuda.empty_cache()
        e_ref = rr.e0
        lanczos["e_ref"] = {"e0": e_ref, "iterations": rr.iterations, "seconds": t_ref, "residual_rel": res,
                            "converged": rr.converged,
                            "definition": "FP64 Lanczos, Ritz change < 1e-14 over 10 steps; ||Hx-Ex||/|E| of its vector"}
        for mode in ("f64", "mixed"):
            err = abs(lanczos[mode]["e0"] - e_ref) / abs(e_ref)
            lanczos[mode]["rel_err_vs_ref"] = err
            lanczos[mode]["meets_1e-10"] = bool(err <= 1e-10)

    # entanglement spectrum of the ground state across the cut
    entangle = None
    if not args.no_entangle and rank == 0:
        torch.cuda.empty_cache()
        try:
            entangle = entanglement_section(ed, ctx)
        except Exception as exc:
            entangle = {"error": str(exc)}

    dense = None
    if not args.no_dense and rank == 0:
        torch.cuda.empty_cache()
        try:
            dense = dense_blocks_section(ed)
        except Exception as exc:
            dense = {"error": str(exc)}

    batched = served = None
    if not args.no_batched:
        torch.cuda.empty_cache()
        try:
            batched, served = batched_and_served(ed, args.batch_n, args.serve_rate, rank=rank, world=ws)
            # instances are sharded by rank: job time = slowest rank
            t_solve = max_over_ranks(batched["solve_s"], ws, device=str(dev))
            batched["instances_total"] = args.batch_n
            batched["instances_per_s_job"] = args.batch_n / t_solve
            batched["hpsi_per_s_job"] = sum_over_ranks(batched["hpsi_per_s_aggregate"] * batched["solve_s"], ws,
                                                       device=str(dev)) / t_solve
        except Exception as exc:
            batched = {"error": str(exc)}

    configs = None
    if rank == 0 and not args.no_configs:
        torch.cuda.empty_cache()
        try:
            configs = other_configs(ed)
        except Exception as exc:
            configs = {"error": str(exc)}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        try:
            cpu = cpu_baseline(model)
        except Exception as exc:  # the baseline must not hide the GPU line
            cpu = {"value": None, "unit": UNIT, "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
                   "sample": f"failed: {exc}"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
                "config": {"workload": args.config, "states": D, "blocks": ctx.num_blocks,
                           "parallelism": "replicas" if ws > 1 else "single", "l2_flush": "inputs larger than L2",
                           "setup_s": t_setup, "row_pass": ctx.row_pass(tdt)},
                "gpu_launches": args.steps * (4 if args.dtype == "f64" else 2),
                "roofline": roof, "clocks": clk, "e2e": e2e, "other_precision": other, "lanczos": lanczos,
                "entanglement": entangle, "dense_blocks": dense, "batched": batched, "serving": served,
                "configs": configs,
                "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
