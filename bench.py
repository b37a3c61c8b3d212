#!/usr/bin/env python
"""Benchmark of the window solve: converged roots per second on one GB300.

Workload (the configuration the metric is quoted on): one synthetic dot with
nocc = 64, nvir = 256, naux = 768 (particle-hole dimension 16384), seed 1,
perturbative-width density-fitting tensor; one window [omega0, omega0 + 0.1 Ha]
with omega0 at the 20th percentile of diag(A)/diag(S); the k = 8 lowest roots,
second order, mixed precision (BF16 tensor-core sigma, FP64 Krylov/Ritz,
split-BF16 refinement to a residual of 1e-6).

A step is one full window solve (pp_solve_window) on device-resident inputs.
value = roots converged / timed seconds; e2e repeats the step through the C ABI
from host buffers (pp_create with the host B tensor, solve, results to host,
pp_destroy) with the copies inside the timed region.

Run:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = dict(name="dot-64x256x768", nocc=64, nvir=256, naux=768, seed=1, mode="perturbative",
                pct=20.0, delta=0.1, k=8, order=2)
METRIC = "converged roots/s"
# residual |M x - theta Sigma x| / |x^T Sigma x| at which a root counts as converged; the split-
# BF16 refinement reaches it, and the root then lies within |r|^2 / gap (<= 1e-6 Ha) of theta
RES_TOL = 1e-6
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            d = json.load(f)
        return dict(hbm=float(d["hbm_gbs"]), bf16=float(d["bf16_tflops"]),
                    bf16_sustained=float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), src="measured")
    except Exception:
        return dict(hbm=6800.0, bf16=1900.0, bf16_sustained=1700.0, src="fallback")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        out = dict(sm_mhz=None, sm_max_mhz=None, reasons=[])
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except Exception:
                continue
            for n, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(n)
        if sm:
            out["sm_mhz"] = statistics.median(sm)
            out["sm_max_mhz"] = max(mx)
        out["reasons"] = sorted(reasons)
        out["samples"] = len(sm)
        try:
            os.unlink(self.path)
        except Exception:
            pass
        return out


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_over_ranks(dist, ms: float, roots: float, device):
    """Weak scaling: the job's time is the slowest rank's, its roots the sum over ranks."""
    import torch

    ms_t = torch.tensor([float(ms)], device=device)
    roots_t = torch.tensor([float(roots)], device=device)
    if dist is not None:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
        dist.all_reduce(roots_t, op=dist.ReduceOp.SUM)
    return float(ms_t.item()), float(roots_t.item())


def window_for_rank(omega0: float, delta: float, rank: int) -> float:
    """Ranks take consecutive, non-overlapping windows of the same width."""
    return omega0 + rank * delta


def make_dot_inputs():
    from synth.inputs import make_inputs

    w = WORKLOAD
    return make_inputs(w["nocc"], w["nvir"], w["naux"], seed=w["seed"], mode=w["mode"])


# DRAM bytes (read + write) of one slab-GEMM launch from an ncu capture of the bench dot
# (profiles/k_gemm_bf16_dot-64x256x768_sigma8.md); the timed launches mix R and the split form,
# so this is the traffic of the captured launch shape, next to its algorithmic minimum
SLAB_GEMM_CAPTURE = dict(dram_bytes=880.2e6, algorithmic_bytes=570e6,
                         launch="R = 16 half-vectors, BF16 phase: 2048 x 12288 x 16384 (8.25e11 FLOP)")


def sigma_flops(o, v, Q, nvec):
    """Algorithmic FLOPs of one sigma batch (nvec supervectors, both halves)."""
    ov = o * v
    R = 2 * nvec
    small = R * (4 * Q * ov + 2 * Q * o * v * v + 2 * Q * o * o * v + 2 * 2 * Q * o * o * v
                 + 2 * 2 * Q * o * o * v + 2 * Q * o * o * v + 2 * Q * o * v * v + 2 * Q * o * o * v
                 + 4 * (o * o * v + o * v * v))
    ladder = 2.0 * ov * ov * Q * R
    tgen = 2.0 * 2.0 * Q * ov * ov
    return small + ladder + tgen


def run_ours(args, world, rank, local):
    import torch

    import paper_2512_09811_gb300 as pp

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    pp.load()
    stream = torch.cuda.current_stream()
    inp = make_dot_inputs()
    w = WORKLOAD
    opt_kw = dict(prec=pp.PP_BF16, order=w["order"], select=0, res_tol=RES_TOL, block=8, refine=1,
                  cuda_stream=stream.cuda_stream)
    t0 = time.time()
    dot = pp.Dot(inp, **opt_kw)
    create_s = time.time() - t0
    dA, dS = dot.diagonal()
    # every rank solves its own window (independent problems: weak scaling, no collective)
    omega0 = window_for_rank(float(np.percentile((dA / dS).ravel(), w["pct"])), w["delta"], rank)

    def step():
        return dot.solve_window(omega0, w["delta"], w["k"], allow_notconv=True)

    for _ in range(max(args.warmup, 0)):
        step()
    pk = peaks()
    roots = 0
    iters = []
    res_all = []
    pp.pp_profile(dot.ctx, True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    launches0 = pp.pp_kernel_launches()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            out = step()
            ok = out["resid"] <= RES_TOL * 1.0000001
            roots += int(np.count_nonzero(ok))
            res_all.extend(out["resid"].tolist())
            iters.append(dot.stats()["iterations"])
        ev1.record(stream)
        torch.cuda.synchronize()
    launches = pp.pp_kernel_launches() - launches0
    if dist is not None:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    k0 = pp.pp_profile_read(dot.ctx, 0)
    k1 = pp.pp_profile_read(dot.ctx, 1)
    pp.pp_profile(dot.ctx, False)
    stats = dot.stats()
    ms_max, roots_tot = reduce_over_ranks(dist, ms, roots, "cuda")
    value = roots_tot / (ms_max / 1e3)

    # sigma throughput of one BF16 batch of 8 supervectors (device-resident, CUDA events)
    from synth.inputs import random_vectors

    Zh = random_vectors(8, w["nocc"], w["nvir"], seed=5)
    Zd = torch.from_numpy(Zh).cuda()
    for _ in range(2):
        pp.pp_sigma(dot.ctx, Zd, prec=pp.PP_BF16)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    nrep = 3
    for _ in range(nrep):
        pp.pp_sigma(dot.ctx, Zd, prec=pp.PP_BF16)
    e1.record(stream)
    torch.cuda.synchronize()
    sig_ms = e0.elapsed_time(e1) / nrep
    sig_tflops = sigma_flops(w["nocc"], w["nvir"], w["naux"], 8) / (sig_ms / 1e3) / 1e12

    # end to end through the C ABI from host buffers: create (B to the device), solve, results back
    from synth.inputs import DotInputs

    # the host inputs in pinned memory
    pin = {f: torch.from_numpy(np.ascontiguousarray(getattr(inp, f))).pin_memory().numpy() for f in ("eps", "B", "mu")}
    pinned = DotInputs(nocc=inp.nocc, nvir=inp.nvir, naux=inp.naux, sigma_b=inp.sigma_b, seed=inp.seed, **pin)
    h2d = inp.eps.nbytes + inp.B.nbytes + inp.mu.nbytes
    d2h = w["k"] * 3 * 8
    torch.cuda.synchronize()
    t0 = time.time()
    ee = 0
    for _ in range(max(1, min(args.steps, 2))):
        d2 = pp.Dot(pinned, **opt_kw)
        o2 = d2.solve_window(omega0, w["delta"], w["k"], allow_notconv=True)
        ee += int(np.count_nonzero(o2["resid"] <= RES_TOL * 1.0000001))
        d2.close()
    torch.cuda.synchronize()
    e2e_s = time.time() - t0
    e2e_max, ee_tot = reduce_over_ranks(dist, e2e_s, ee, "cuda")
    e2e_val = ee_tot / e2e_max

    achieved = (k0["flops"] / (k0["ms"] / 1e3) / 1e12) if k0["ms"] > 0 else None
    peak = pk["bf16_sustained"]
    cap = SLAB_GEMM_CAPTURE
    roof = dict(bound="tensor", kernel="k_gemm_bf16 (amplitude contraction, tcgen05)",
                achieved=achieved, peak=peak, unit="TFLOP/s",
                frac=(achieved / peak) if achieved else None, traffic=cap["dram_bytes"],
                traffic_launch=cap["launch"], traffic_algorithmic_bytes=cap["algorithmic_bytes"],
                peak_source=f"{pk['src']} bf16 sustained", launches=k0["launches"],
                avg_launch_ms=(k0["ms"] / k0["launches"]) if k0["launches"] else None,
                tgen=dict(launches=k1["launches"], ms=k1["ms"],
                          achieved=(k1["flops"] / (k1["ms"] / 1e3) / 1e12) if k1["ms"] > 0 else None))
    line = dict(
        metric=METRIC, value=value, unit="roots/s", n_gpus=world, steps=args.steps, warmup=args.warmup,
        ms_per_step=ms_max / max(args.steps, 1), higher_is_better=True, scaling="weak", vs_baseline=None,
        dtype="bf16", data="synthetic",
        config=dict(workload=w["name"], nocc=w["nocc"], nvir=w["nvir"], naux=w["naux"], k=w["k"],
                    window_ha=w["delta"], order=w["order"], precision="bf16 tensor cores + fp64 krylov + bf16x3 refine",
                    inputs=w["mode"], l2="inputs larger than L2 (B tensor 630 MB fp64 resident)",
                    parallelism=f"replicas{world}"),
        roofline=roof,
        e2e=dict(value=e2e_val, unit="roots/s", h2d_bytes_per_step=int(h2d), d2h_bytes_per_step=int(d2h)),
        gpu_launches=int(launches),
        clocks=clk.summary(),
        extra=dict(create_s=create_s, iterations=iters, sigma_vectors=stats["sigma_vectors"],
                   sigma_ms_last_solve=stats["sigma_ms"], solve_ms_last=stats["solve_ms"],
                   max_resid=max(res_all) if res_all else None,
                   sigma_batch8_ms=sig_ms, sigma_tflops=sig_tflops),
    )
    dot.close()
    return line


SERVING_SIZES = [(32, 128, 384), (64, 256, 768), (128, 512, 1536)]


def serving_leg(args):
    """Poisson arrivals of window requests over a pool of dots (4 per size), served by the
    continuous-batching loop; latency = finish - submit as the server records it."""
    import paper_2512_09811_gb300 as pp
    from synth.inputs import make_inputs

    rng = np.random.default_rng(3)
    sizes = SERVING_SIZES if args.serving_all_sizes else SERVING_SIZES[:2]
    n_req, rate = args.serving_requests, args.serving_rate
    opts = dict(prec=pp.PP_BF16, order=2, select=0, res_tol=RES_TOL, max_iter=300)
    pool = []  # (size index, inputs, sorted diag(A)/diag(S))
    for si, (o, v, Q) in enumerate(sizes):
        for di in range(4):
            inp = make_inputs(o, v, Q, seed=3000 + 10 * si + di, mode="perturbative")
            d = pp.Dot(inp, **opts)
            dA, dS = d.diagonal()
            d.close()
            pool.append((si, inp, np.sort((dA / dS).ravel())))
    reqs = []
    t = 0.0
    for _ in range(n_req):
        t += rng.exponential(1.0 / rate)
        si = int(rng.integers(len(sizes)))
        di = int(rng.integers(4))
        k = int(rng.choice([4, 8, 16]))
        width = float(rng.uniform(0.05, 0.2))
        r = pool[4 * si + di][2]
        w0 = float(rng.uniform(np.percentile(r, 10), np.percentile(r, 50)))
        reqs.append((t, 4 * si + di, w0, width, k))
    srv = pp.Server(200 << 30, slots_per_dot=4, nworkers=4, **opts)
    try:
        ids = [srv.add_dot(p_[1]) for p_ in pool]
        t0 = time.perf_counter()
        rid = []
        for (ta, dot, w0, width, k) in reqs:
            dt = t0 + ta - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            rid.append((srv.submit(ids[dot], w0, width, k), k, ta))
        lat, roots, finish, notconv = [], 0, 0.0, 0
        for (r_id, k, ta) in rid:
            out = srv.wait(r_id, k, timeout_ms=1_800_000, allow_notconv=True)
            lat.append(out["latency_ms"])
            roots += int(np.count_nonzero(out["resid"] <= RES_TOL * 1.0000001))
            notconv += int(out["status"] != pp.PP_OK)
            finish = max(finish, ta + out["latency_ms"] / 1e3)
        st = srv.stats()
    finally:
        srv.close()
    return dict(requests=n_req, arrival_rate_per_s=rate, sizes=[list(z) for z in sizes], dots_per_size=4,
                k_choices=[4, 8, 16], window_ha=[0.05, 0.2], start="U[pct10, pct50] of diag(A)/diag(S)",
                p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                roots_per_s=roots / finish, roots=roots, wall_s=finish, not_converged=notconv,
                slots_per_dot=4, workers=4, max_concurrent_dots=st["max_concurrent_dots"],
                max_windows_per_step=st["max_windows_per_step"], ctx_created=st["ctx_created"],
                ctx_evicted=st["ctx_evicted"], failed=st["failed"])


def run_reference(args, world, rank):
    """The CPU oracle (plain FP64 NumPy) on this machine's host cores: its matrix-free sigma,
    timed on one trial supervector per step, scaled by the sigma supervectors a window
    solve needs."""
    if rank != 0:
        return None
    from oracle import pp_oracle as po
    from synth.inputs import random_vectors

    inp = make_dot_inputs()
    w = WORKLOAD
    t0 = time.time()
    ref = po.SigmaRef(inp.eps, inp.B, inp.nocc, order=w["order"])
    setup_s = time.time() - t0
    Z = random_vectors(1, w["nocc"], w["nvir"], seed=5)
    ref.sigma(Z)  # warm caches
    times = []
    for _ in range(max(1, args.steps)):
        t0 = time.time()
        ref.sigma(Z)
        times.append(time.time() - t0)
    t_vec = statistics.median(times)
    vecs_per_root = REF_SIGMA_VECTORS_PER_ROOT
    value = 1.0 / (t_vec * vecs_per_root)
    cores = os.cpu_count()
    sample = (f"oracle FP64 sigma of 1 supervector per step at {w['name']} (median {t_vec:.2f} s, "
              f"setup {setup_s:.1f} s), times {vecs_per_root} supervectors per converged root")
    return dict(metric=METRIC, value=value, unit="roots/s", n_gpus=world, steps=args.steps,
                warmup=args.warmup, ms_per_step=t_vec * 1e3, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=w["name"], nocc=w["nocc"], nvir=w["nvir"], naux=w["naux"], k=w["k"]),
                cpu_baseline=dict(value=value, unit="roots/s", cores=cores, kind="oracle", sample=sample),
                e2e=dict(value=value, unit="roots/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))


# sigma supervectors per converged root of the window solve at this workload: the GPU solver
# needed 255-293 supervector products for the 8 roots of one window (bench and trace runs)
REF_SIGMA_VECTORS_PER_ROOT = 33


def cpu_baseline_leg():
    """Bounded oracle sample for the cpu_baseline field (rank 0, N = 1 only)."""
    from oracle import pp_oracle as po
    from synth.inputs import random_vectors

    inp = make_dot_inputs()
    w = WORKLOAD
    t0 = time.time()
    ref = po.SigmaRef(inp.eps, inp.B, inp.nocc, order=w["order"])
    setup = time.time() - t0
    Z = random_vectors(1, w["nocc"], w["nvir"], seed=5)
    t0 = time.time()
    ref.sigma(Z)
    t_vec = time.time() - t0
    return dict(value=1.0 / (t_vec * REF_SIGMA_VECTORS_PER_ROOT), unit="roots/s", cores=os.cpu_count(),
                kind="oracle",
                sample=f"1 oracle FP64 sigma supervector at {w['name']} ({t_vec:.2f} s, setup {setup:.1f} s) "
                       f"x {REF_SIGMA_VECTORS_PER_ROOT} supervectors per root")


def profile_workload(args):
    """Small fixed workloads for ncu captures (no timing, no JSON line)."""
    import torch

    import paper_2512_09811_gb300 as pp
    from synth.inputs import random_vectors

    w = WORKLOAD
    inp = make_dot_inputs()
    if args.profile_sigma:
        dot = pp.Dot(inp, prec=pp.PP_BF16, order=w["order"])
        Z = torch.from_numpy(random_vectors(8, w["nocc"], w["nvir"], seed=5)).cuda()
        for _ in range(2):
            pp.pp_sigma(dot.ctx, Z, prec=pp.PP_BF16)
        torch.cuda.synchronize()
    else:
        dot = pp.Dot(inp, prec=pp.PP_BF16, order=w["order"], select=0, res_tol=RES_TOL,
                     max_iter=args.profile_solve)
        dA, dS = dot.diagonal()
        omega0 = float(np.percentile((dA / dS).ravel(), w["pct"]))
        dot.solve_window(omega0, w["delta"], w["k"], allow_notconv=True)
    dot.close()
    print("profile workload done", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-trace leg")
    ap.add_argument("--serving-requests", type=int, default=48)
    ap.add_argument("--serving-rate", type=float, default=50.0, help="Poisson arrival rate (requests/s)")
    ap.add_argument("--serving-all-sizes", action="store_true",
                    help="include 128/512/1536 dots in the serving mix (minutes per request)")
    ap.add_argument("--profile-sigma", action="store_true",
                    help="profiling workload: create the dot, two BF16 sigma batches of 8 supervectors")
    ap.add_argument("--profile-solve", type=int, default=0,
                    help="profiling workload: one window solve capped at this many iterations")
    args = ap.parse_args()
    if args.profile_sigma or args.profile_solve:
        profile_workload(args)
        return
    world, rank, local = dist_setup()
    if args.impl == "reference":
        line = run_reference(args, world, rank)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    line = run_ours(args, world, rank, local)
    if rank == 0:
        if world == 1 and not args.no_serving:
            line["serving"] = serving_leg(args)
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_leg()
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
