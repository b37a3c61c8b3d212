#!/usr/bin/env python
"""Benchmark of the batched window solver on one GB300.

Workload (default, the large dot): one synthetic dot with nocc = 256, nvir = 1024,
naux = 3072 (particle-hole dimension 262144; 6.9e10 MP2 amplitudes, regenerated per slab),
seed 4, FP32 density-fitting tensor (20 GB) of perturbative width; 4 consecutive windows of
0.05 Ha from the 20th percentile of diag(A)/diag(S), the k = 16 lowest roots of each, block
of 16 trial vectors per window; second order, mixed precision (BF16 tensor-core sigma with
FP32 accumulation, FP64 Krylov basis and projected problems, split-BF16 refinement to a
residual of 1e-6).  --workload batched-128x512x1536 runs the 8-window x k = 8 batch on the
128/512/1536 dot, --workload dot-64x256x768 the single window of the plain-vs-mixed test.

A step is one block iteration of the window batch: the whole hot path once -- Rayleigh-Ritz
and the folded extraction, residuals, weighted-Jacobi directions, block CGS2, and one sigma
batch per precision phase of every window's new vectors (pp_windows_step).  On the large dot
the batch is one window, and the four windows are solved in turn (each starts when the one
before it finishes): a block iteration of one window there takes about 12 s in the BF16
phase and 36 s in the split phase.  value =
algorithmic sigma TFLOP/s of the timed steps (each contraction counted once; the split form's
three products count as one).  With --full-solve (the default for the two smaller workloads)
the solve continues after the timed steps and its converged roots per second are reported
beside the value.  e2e times the sigma batch of one step through the C ABI on pinned host
buffers (pp_sigma with on_device = 0: the host-to-device copy of the trial vectors, the
product, the device-to-host copy of sigma and Sigma z inside the timed region).

Run:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload NAME]
"""

from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    # 8 windows x k = 8, block 16 per window (128 trial supervectors per iteration)
    "batched-128x512x1536": dict(nocc=128, nvir=512, naux=1536, seed=2, mode="perturbative", pct=20.0, nwin=8,
                                 delta=0.05, k=8, block=16, order=2, full_solve=True),
    # one window, k = 8 (the plain-vs-mixed comparison)
    "dot-64x256x768": dict(nocc=64, nvir=256, naux=768, seed=1, mode="perturbative", pct=20.0, nwin=1, delta=0.1,
                           k=8, block=8, order=2, full_solve=True),
    # 4 windows x k = 16, solved one window at a time (the large dot: a block iteration of one
    # window takes about 12 s in the BF16 phase and 36 s in the split phase, a window's solve
    # tens of minutes, so it is not finished by default; the four windows batched together
    # would make one split-phase step about 145 s)
    "dot-256x1024x3072": dict(nocc=256, nvir=1024, naux=3072, seed=4, mode="perturbative", pct=20.0, nwin=4,
                              delta=0.05, k=16, block=16, order=2, full_solve=False, workspace_gb=140.0,
                              in_turn=True),
}
DEFAULT_WORKLOAD = "dot-256x1024x3072"
METRIC = "converged roots/s & sigma TFLOP/s at <=1e-6 Ha vs FP64 oracle; p50/p99 window latency"
# residual |M x - theta Sigma x| / |x^T Sigma x| at which a root counts as converged; the split-
# BF16 refinement reaches it, and an isolated root then lies within |r|^2 / gap of theta
RES_TOL = 1e-6
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# the oracle's bounded sample (its matrix-free sigma at the serving dot; see cpu_sample)
ORACLE_SAMPLE = dict(nocc=32, nvir=128, naux=384, seed=3, mode="perturbative")


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


def reduce_over_ranks(dist, ms: float, amount: float, device):
    """Weak scaling: the job's time is the slowest rank's, its work the sum over ranks."""
    import torch

    ms_t = torch.tensor([float(ms)], device=device)
    am_t = torch.tensor([float(amount)], device=device)
    if dist is not None:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
        dist.all_reduce(am_t, op=dist.ReduceOp.SUM)
    return float(ms_t.item()), float(am_t.item())


def window_for_rank(omega0: float, delta: float, rank: int) -> float:
    """Ranks take consecutive, non-overlapping windows of the same width."""
    return omega0 + rank * delta


def windows_for_rank(omega0: float, delta: float, nwin: int, rank: int):
    """The nwin consecutive windows of this rank (replicas solve disjoint frequency ranges)."""
    return [window_for_rank(omega0, delta, rank * nwin + w) for w in range(nwin)]


def window_batches(w):
    """Which windows are stepped together: all of them in one batch, or (workloads with
    in_turn) one window at a time, the windows taken in turn as each one finishes."""
    n = w["nwin"]
    return [[i] for i in range(n)] if w.get("in_turn") else [list(range(n))]


def next_batch(b: int, nbatches: int) -> int:
    return (b + 1) % nbatches


def make_dot_inputs(w, b_dtype=np.float32):
    from synth.inputs import make_inputs

    return make_inputs(w["nocc"], w["nvir"], w["naux"], seed=w["seed"], mode=w["mode"], b_dtype=b_dtype)


def sigma_flops_per_vector(o, v, Q):
    """Algorithmic FLOPs of sigma for one supervector (both halves), each contraction once:
    J 4 Q ov; U = Boo_Q V and the exchange sum_(Q,b) U_Q Bvv_Q 2 Q o^2 v + 2 Q o v^2;
    E, F and their contraction with [Bov + Gamma; Bov] 8 Q o^2 v; C_Q(V) = V Bvv_Q - U 2 Q o v^2;
    the amplitude contraction P_Q = T C_Q(V) 2 (ov)^2 Q; sum_Q C_Q(P_Q) 2 Q o v^2 + 2 Q o^2 v;
    the A(2) pair-sum products 4 (o^2 v + o v^2)."""
    ov = o * v
    half = (4 * Q * ov + 12 * Q * o * o * v + 6 * Q * o * v * v + 4 * (o * o * v + o * v * v)
            + 2.0 * ov * ov * Q)
    return 2.0 * half


def tgen_flops(o, v, Q):
    """Regeneration of the amplitudes once per sigma batch: one Q-long product per t_ij^cd."""
    return 2.0 * Q * (o * v) ** 2


def step_flops(o, v, Q, nvec, ncalls):
    return nvec * sigma_flops_per_vector(o, v, Q) + ncalls * tgen_flops(o, v, Q)


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
    w = WORKLOADS[args.workload]
    o, v, Q = w["nocc"], w["nvir"], w["naux"]
    inp = make_dot_inputs(w)
    # the large dot holds about 90 GB of integrals and their copies; 140 GB of sigma workspace
    # (about 10 half-vectors per chunk at 14 GB each) fit beside them
    ws = args.workspace_gb if args.workspace_gb > 0 else w.get("workspace_gb", 0.0)
    opt_kw = dict(prec=pp.PP_BF16, order=w["order"], select=0, res_tol=RES_TOL, block=w["block"], refine=1,
                  max_iter=300, cuda_stream=stream.cuda_stream, workspace_gb=ws)
    t0 = time.time()
    dot = pp.Dot(inp, **opt_kw)
    torch.cuda.synchronize()
    create_s = time.time() - t0
    dA, dS = dot.diagonal()
    omega0 = float(np.percentile((dA / dS).ravel(), w["pct"]))
    wins = windows_for_rank(omega0, w["delta"], w["nwin"], rank)
    deltas = [w["delta"]] * w["nwin"]
    ks = [w["k"]] * w["nwin"]

    # ---- the solve, one block iteration per step ------------------------------------------
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    batches = window_batches(w)
    bidx = 0

    def start(b):
        sel = batches[b]
        return dot.windows([wins[i] for i in sel], [deltas[i] for i in sel], [ks[i] for i in sel])

    run = start(0)
    solves = []  # (roots converged, ms, iterations, sigma supervectors, max resid) per completed batch
    cur = dict(ms=0.0, it=0, nv=0)

    def one_step():
        nonlocal run, bidx
        ev0.record(stream)
        un, nv, nc = run.step()
        ev1.record(stream)
        ev1.synchronize()
        ms = ev0.elapsed_time(ev1)
        cur["ms"] += ms
        cur["it"] += 1
        cur["nv"] += nv
        if un == 0:  # the batch is done: collect it and start the next one (or the same again)
            res, st = run.end(allow_notconv=True)
            roots = sum(int(np.count_nonzero(r["resid"] <= RES_TOL * 1.0000001)) for r in res)
            mres = max((float(r["resid"].max()) for r in res if len(r["resid"])), default=None)
            solves.append(dict(roots=roots, ms=cur["ms"], iterations=cur["it"], sigma_vectors=cur["nv"],
                               max_resid=mres, status=int(st), found=[len(r["omega"]) for r in res]))
            cur.update(ms=0.0, it=0, nv=0)
            bidx = next_batch(bidx, len(batches))
            run = start(bidx)
        return ms, step_flops(o, v, Q, nv, nc), nv

    for _ in range(max(args.warmup, 0)):
        one_step()
    pk = peaks()
    pp.pp_profile(dot.ctx, True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = pp.pp_kernel_launches()
    timed_ms, timed_flops, timed_nv = 0.0, 0.0, 0
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            ms, fl, nv = one_step()
            timed_ms += ms
            timed_flops += fl
            timed_nv += nv
        torch.cuda.synchronize()
    launches = pp.pp_kernel_launches() - launches0
    k0 = pp.pp_profile_read(dot.ctx, 0)
    k1 = pp.pp_profile_read(dot.ctx, 1)
    k2 = pp.pp_profile_read(dot.ctx, 2)
    pp.pp_profile(dot.ctx, False)
    if dist is not None:
        dist.barrier()
    ms_max, flops_tot = reduce_over_ranks(dist, timed_ms, timed_flops, "cuda")
    value = flops_tot / (ms_max / 1e3) / 1e12
    # finish the solve that was running when the timed steps ended (at least one full batch)
    roots_obj = None
    full_solve = w["full_solve"] if args.full_solve is None else args.full_solve
    if full_solve:
        while not solves:
            one_step()
        first = solves[0]
        solve_ms_max, roots_tot = reduce_over_ranks(dist, first["ms"], first["roots"], "cuda")
        solve_flops = first["sigma_vectors"] * sigma_flops_per_vector(o, v, Q)
        roots_obj = dict(roots_per_s=roots_tot / (solve_ms_max / 1e3), roots=int(roots_tot),
                         solve_s=solve_ms_max / 1e3, iterations=first["iterations"],
                         sigma_vectors=first["sigma_vectors"], max_resid=first["max_resid"], found=first["found"],
                         status=first["status"], sigma_tflops=solve_flops / (first["ms"] / 1e3) / 1e12)

    # ---- end to end through the C ABI on pinned host buffers: one step's sigma batch -----
    e2e = None
    nv_step = max(1, int(round(timed_nv / max(args.steps, 1))))
    if not args.no_e2e:
        from synth.inputs import random_vectors

        Zh = torch.from_numpy(random_vectors(nv_step, o, v, seed=11)).pin_memory()
        Sh = torch.empty_like(Zh).pin_memory()
        Mh = torch.empty_like(Zh).pin_memory()
        lib = pp.load()
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        t0 = time.time()
        st = lib.pp_sigma(dot.ctx, nv_step, Zh.data_ptr(), Sh.data_ptr(), Mh.data_ptr(), pp.PP_BF16, 0)
        torch.cuda.synchronize()
        e2e_s = time.time() - t0
        pp._check(st, dot.ctx)
        fin = bool(np.isfinite(Sh.numpy()).all())
        e2e_fl = step_flops(o, v, Q, nv_step, 1)
        e2e_max, e2e_flops = reduce_over_ranks(dist, e2e_s * 1e3, e2e_fl, "cuda")
        nb = Zh.numel() * 8
        e2e = dict(value=e2e_flops / (e2e_max / 1e3) / 1e12, unit="TFLOP/s", h2d_bytes_per_step=int(nb),
                   d2h_bytes_per_step=int(2 * nb), supervectors=nv_step, seconds=e2e_max / 1e3, finite=fin,
                   step="pp_sigma through the C ABI on pinned host buffers (on_device = 0): trial vectors "
                        "host->device, BF16 tensor-core sigma and metric, both products device->host")
    dot.close()

    # ---- roofline of the dominant kernel: the amplitude-contraction GEMM -----------------
    achieved = (k0["flops"] / (k0["ms"] / 1e3) / 1e12) if k0["ms"] > 0 else None
    hw = ((k0["flops"] + 2.0 * k2["flops"]) / (k0["ms"] / 1e3) / 1e12) if k0["ms"] > 0 else None
    peak = pk["bf16_sustained"]
    cap = SLAB_GEMM_CAPTURE.get(args.workload)
    roof = dict(bound="tensor", kernel="k_gemm_bf16 amplitude contraction P_Q = T C_Q(V) (tcgen05)",
                achieved=achieved, peak=peak, unit="TFLOP/s", frac=(achieved / peak) if achieved else None,
                traffic=cap["dram_bytes"] if cap else None,
                peak_source=f"{pk['src']} bf16 sustained", launches=k0["launches"],
                avg_launch_ms=(k0["ms"] / k0["launches"]) if k0["launches"] else None,
                hardware_mma_tflops=hw, hardware_frac=(hw / peak) if hw else None,
                split_form_share_of_launch_flops=(k2["flops"] / k0["flops"]) if k0["flops"] else None,
                generator=dict(kernel="k_tgen_p", launches=k1["launches"], ms=k1["ms"],
                               achieved=(k1["flops"] / (k1["ms"] / 1e3) / 1e12) if k1["ms"] > 0 else None))
    if cap:
        roof.update(traffic_launch=cap["launch"], traffic_algorithmic_bytes=cap["algorithmic_bytes"])
    line = dict(
        metric=METRIC, value=value, unit="TFLOP/s", n_gpus=world, steps=args.steps, warmup=args.warmup,
        ms_per_step=ms_max / max(args.steps, 1), higher_is_better=True, scaling="weak", vs_baseline=None,
        dtype="bf16 (fp32 accumulate; fp64 krylov)", data="synthetic",
        config=dict(workload=args.workload, nocc=o, nvir=v, naux=Q, windows=w["nwin"], k=w["k"],
                    window_ha=w["delta"], block=w["block"], order=w["order"],
                    precision="bf16 tensor cores + fp64 krylov + bf16x3 refinement to 1e-6",
                    inputs=w["mode"],
                    step=("one block iteration of the current window (pp_windows_step on a one-window batch; "
                          "the windows solved in turn)") if w.get("in_turn") else
                         "one block iteration of all windows (pp_windows_step)",
                    l2="inputs larger than L2 (FP32 B tensor %.1f GB; slab and operands > 129 MB)" % (inp.B.nbytes / 1e9),
                    parallelism=f"replicas{world}"),
        roots=roots_obj,
        roofline=roof,
        e2e=e2e,
        gpu_launches=int(launches),
        clocks=clk.summary(),
        extra=dict(create_s=create_s, timed_sigma_vectors=timed_nv, omega0=omega0),
    )
    return line


# DRAM bytes (read + write) per launch of the amplitude-contraction GEMM from an ncu capture
SLAB_GEMM_CAPTURE = {}


def mixed_vs_fp64_leg(args):
    """The plain FP64 form against the mixed form on the same single window (64/256/768, k = 8,
    residual 1e-6): converged roots/s of each, one full solve each on device-resident inputs."""
    import torch

    import paper_2512_09811_gb300 as pp

    w = WORKLOADS["dot-64x256x768"]
    inp = make_dot_inputs(w, b_dtype=np.float64)
    out = {}
    for name, prec in (("mixed", pp.PP_BF16), ("fp64", pp.PP_FP64)):
        d = pp.Dot(inp, prec=prec, order=2, select=0, res_tol=RES_TOL, block=w["block"], max_iter=300)
        dA, dS = d.diagonal()
        w0 = float(np.percentile((dA / dS).ravel(), w["pct"]))
        torch.cuda.synchronize()
        t0 = time.time()
        r = d.solve_window(w0, w["delta"], w["k"], allow_notconv=True)
        torch.cuda.synchronize()
        dt = time.time() - t0
        st = d.stats()
        d.close()
        n = int(np.count_nonzero(r["resid"] <= RES_TOL * 1.0000001))
        out[name] = dict(roots=n, seconds=dt, roots_per_s=n / dt, iterations=st["iterations"],
                         sigma_vectors=st["sigma_vectors"], omega=[float(x) for x in r["omega"]])
    out["mixed_over_fp64"] = out["mixed"]["roots_per_s"] / out["fp64"]["roots_per_s"]
    out["max_root_difference_ha"] = float(np.max(np.abs(np.array(out["mixed"]["omega"]) - np.array(out["fp64"]["omega"])))) \
        if len(out["mixed"]["omega"]) == len(out["fp64"]["omega"]) else None
    out["workload"] = "dot-64x256x768, one window [pct20, +0.1 Ha], k = 8, residual 1e-6"
    return out


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
            inp = make_inputs(o, v, Q, seed=3000 + 10 * si + di, mode="perturbative",
                              b_dtype=np.float32 if o >= 128 else np.float64)
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
            rid.append((srv.submit(ids[dot], w0, width, k), k, ta, pool[dot][0]))
        lat, roots, finish, notconv = [], 0, 0.0, 0
        by_size = {si: [] for si in range(len(sizes))}
        for (r_id, k, ta, si) in rid:
            out = srv.wait(r_id, k, timeout_ms=3_600_000, allow_notconv=True)
            lat.append(out["latency_ms"])
            by_size[si].append(out["latency_ms"])
            roots += int(np.count_nonzero(out["resid"] <= RES_TOL * 1.0000001))
            notconv += int(out["status"] != pp.PP_OK)
            finish = max(finish, ta + out["latency_ms"] / 1e3)
        st = srv.stats()
    finally:
        srv.close()
    served = roots / finish
    return dict(requests=n_req, arrival_rate_per_s=rate, arrivals_s=reqs[-1][0], sizes=[list(z) for z in sizes],
                regime="sustained" if reqs[-1][0] >= 0.5 * finish else "burst (arrivals end before half the drain)",
                dots_per_size=4, k_choices=[4, 8, 16], window_ha=[0.05, 0.2],
                start="U[pct10, pct50] of diag(A)/diag(S)",
                p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                p50_ms_by_size={str(list(sizes[s])): float(np.percentile(v_, 50)) for s, v_ in by_size.items() if v_},
                p99_ms_by_size={str(list(sizes[s])): float(np.percentile(v_, 99)) for s, v_ in by_size.items() if v_},
                roots_per_s=served, roots=roots, wall_s=finish, not_converged=notconv,
                slots_per_dot=4, workers=4, max_concurrent_dots=st["max_concurrent_dots"],
                max_windows_per_step=st["max_windows_per_step"], ctx_created=st["ctx_created"],
                ctx_evicted=st["ctx_evicted"], failed=st["failed"])


def host_cpu():
    name = platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                name = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return name


def cpu_sample(nvec: int):
    """The oracle as it stands (plain FP64 NumPy, OpenBLAS threads on every host core): its
    matrix-free sigma of nvec supervectors at the 32/128/384 dot, the largest dot whose
    oracle sigma takes a few seconds per supervector.  Returns (seconds, setup seconds,
    algorithmic FLOPs of the sample, counted as for the GPU)."""
    from oracle import pp_oracle as po
    from synth.inputs import make_inputs, random_vectors

    s = ORACLE_SAMPLE
    inp = make_inputs(s["nocc"], s["nvir"], s["naux"], seed=s["seed"], mode=s["mode"])
    t0 = time.time()
    ref = po.SigmaRef(inp.eps, inp.B, inp.nocc, order=2)
    setup = time.time() - t0
    Z = random_vectors(nvec, s["nocc"], s["nvir"], seed=5)
    return ref, Z, setup, step_flops(s["nocc"], s["nvir"], s["naux"], nvec, 1)


def cpu_baseline_leg():
    """Bounded oracle sample for the cpu_baseline field (rank 0, N = 1 only)."""
    ref, Z, setup, fl = cpu_sample(4)
    t0 = time.time()
    ref.sigma(Z)
    dt = time.time() - t0
    return dict(value=fl / dt / 1e12, unit="TFLOP/s", cores=os.cpu_count(), cpu=host_cpu(), kind="oracle",
                sample=f"oracle FP64 matrix-free sigma of 4 supervectors at the 32/128/384 dot ({dt:.2f} s, setup "
                       f"{setup:.1f} s); algorithmic FLOPs counted as for the GPU")


def run_reference(args, world, rank):
    """The reference arm: the CPU oracle (plain FP64 NumPy) on this machine's host cores, each step
    its matrix-free sigma of 2 supervectors at the 32/128/384 dot (a bounded sample: the oracle
    cannot hold the 128/512/1536 amplitudes, 34 GB, nor finish one of its sigmas in minutes)."""
    if rank != 0:
        return None
    ref, Z, setup, fl = cpu_sample(2)
    for _ in range(max(args.warmup, 0)):
        ref.sigma(Z)
    times = []
    for _ in range(max(1, args.steps)):
        t0 = time.time()
        ref.sigma(Z)
        times.append(time.time() - t0)
    tot = sum(times)
    value = fl * len(times) / tot / 1e12
    cores = os.cpu_count()
    sample = (f"oracle FP64 matrix-free sigma of 2 supervectors per step at the 32/128/384 dot (mean "
              f"{tot / len(times):.2f} s per step, setup {setup:.1f} s); algorithmic FLOPs counted as for the GPU")
    w = WORKLOADS[args.workload]
    return dict(metric=METRIC, value=value, unit="TFLOP/s", n_gpus=world, steps=args.steps,
                warmup=args.warmup, ms_per_step=tot / len(times) * 1e3, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=args.workload, nocc=w["nocc"], nvir=w["nvir"], naux=w["naux"],
                            windows=w["nwin"], k=w["k"], window_ha=w["delta"], block=w["block"], order=w["order"]),
                cpu_baseline=dict(value=value, unit="TFLOP/s", cores=cores, cpu=host_cpu(), kind="oracle",
                                  sample=sample),
                e2e=dict(value=value, unit="TFLOP/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))


def profile_workload(args):
    """Small fixed workloads for ncu captures (no timing, no JSON line).  The sigma workload
    limits the tensor-core workspace (workspace_gb) so that the capture holds a few GB."""
    import torch

    import paper_2512_09811_gb300 as pp
    from synth.inputs import random_vectors

    w = WORKLOADS[args.workload]
    inp = make_dot_inputs(w)
    if args.profile_sigma:  # kernel by kernel (no chunk graphs), for per-launch profiles
        dot = pp.Dot(inp, prec=pp.PP_BF16, order=w["order"], workspace_gb=args.profile_workspace_gb, graphs=0)
        Z = torch.from_numpy(random_vectors(args.profile_sigma, w["nocc"], w["nvir"], seed=5)).cuda()
        for prec in (pp.PP_BF16, pp.PP_BF16X3):
            pp.pp_sigma(dot.ctx, Z, prec=prec)
        torch.cuda.synchronize()
    else:
        dot = pp.Dot(inp, prec=pp.PP_BF16, order=w["order"], select=0, res_tol=RES_TOL, block=w["block"],
                     max_iter=args.profile_solve, graphs=0, workspace_gb=w.get("workspace_gb", 0.0))
        dA, dS = dot.diagonal()
        omega0 = float(np.percentile((dA / dS).ravel(), w["pct"]))
        dot.solve_windows(windows_for_rank(omega0, w["delta"], w["nwin"], 0), [w["delta"]] * w["nwin"],
                          [w["k"]] * w["nwin"], allow_notconv=True)
    dot.close()
    print("profile workload done", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end sigma batch on host buffers")
    ap.add_argument("--full-solve", dest="full_solve", action="store_true", default=None,
                    help="finish the solve after the timed steps and report its converged roots/s (default for "
                         "the two smaller workloads; the large dot's full solve takes tens of minutes)")
    ap.add_argument("--no-full-solve", dest="full_solve", action="store_false")
    ap.add_argument("--workspace-gb", type=float, default=0.0,
                    help="device memory for one chunk of the sigma workspaces (0: automatic)")
    ap.add_argument("--fp64-leg", action="store_true",
                    help="also solve the 64/256/768 window in the plain FP64 form and the mixed form "
                         "(minutes: the FP64 form issues at GB300's FP64 rate)")
    ap.add_argument("--serving", action="store_true", help="run the serving-trace leg")
    ap.add_argument("--serving-requests", type=int, default=48)
    ap.add_argument("--serving-rate", type=float, default=50.0, help="Poisson arrival rate (requests/s)")
    ap.add_argument("--serving-all-sizes", action="store_true",
                    help="include 128/512/1536 dots in the serving mix (minutes per request)")
    ap.add_argument("--profile-sigma", type=int, default=0,
                    help="profiling workload: create the dot, one BF16 and one split sigma of this many supervectors")
    ap.add_argument("--profile-workspace-gb", type=float, default=2.0)
    ap.add_argument("--profile-solve", type=int, default=0,
                    help="profiling workload: the workload's windows solved with this iteration cap")
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
        if world == 1 and args.fp64_leg:
            line["mixed_vs_fp64"] = mixed_vs_fp64_leg(args)
        if world == 1 and args.serving:
            line["serving"] = serving_leg(args)
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_leg()
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
