#!/usr/bin/env python
"""Frequency-solve throughput of reciprocity-aware TLR MDD on GB300.

Workload (the plain-method batched-frequency configuration): nr = ns = 4096
receivers / sources on a 64 x 64 grid (Hilbert-reordered), 64 frequencies,
tile 256, off-diagonal rank rising linearly 4 -> 48 with frequency, low-rank
diagonal tiles (rank < tile/4), D(w) = Q diag(sigma e^{i phi_w}) W^H with sigma
decaying 1 -> 1e-3, U = D X + complex Gaussian noise at 10 dB SNR, X a planted
symmetric TLR Green's function.  One step = one frequency solve (30 L-BFGS
iterations: 3 lambda stages x 2 ADMM iterations x 5) for every frequency,
inputs resident in HBM.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
instead (the only place besides the cpu_baseline leg that runs it).
"""
from __future__ import annotations

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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NR = 4096
GRID = (64, 64)
NFREQ = 64
TILE = 256
RANK_LO, RANK_HI = 4, 48
SNR_DB = 10.0
ITERS_PER_SOLVE = 30
FP32_LANES_PER_SM, SMS, SM_MAX_MHZ = 128, 152, 2070.0


def rank_of(f, nfreq):
    if nfreq == 1:
        return RANK_LO
    return RANK_LO + int(math.floor((RANK_HI - RANK_LO) * f / (nfreq - 1) + 0.5))


def flops_per_iter(nr, ns, tile, k):
    """Algorithmic flops of one L-BFGS iteration (8 real flops per complex MAC):
    compress of the direction and of the residual (8 + 8), the two line-search
    expands (16 + 8) and the gradient projection (16), all x ns x n_LR."""
    n = nr // tile
    n_lr = n * n * tile * k
    return 56.0 * ns * n_lr


def flops_per_solve(nr, ns, tile, k, iters=ITERS_PER_SOLVE):
    n = nr // tile
    n_lr = n * n * tile * k
    return iters * flops_per_iter(nr, ns, tile, k) + 40.0 * ns * n_lr


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def clock_problem(clocks):
    """Why a timed region's clock record disqualifies it, or None: a hardware
    or thermal slowdown reason, or a median SM clock below 80% of the maximum
    with no reason active (a leftover clock lock).  sw_power_cap is normal."""
    bad = [r for r in clocks.get("reasons", []) if r in ("hw_slowdown", "hw_thermal_slowdown",
                                                          "sw_thermal_slowdown")]
    if bad:
        return ",".join(bad)
    sm, mx = clocks.get("sm_mhz"), clocks.get("sm_max_mhz")
    if sm and mx and sm < 0.8 * mx and not clocks.get("reasons"):
        return f"SM clock median {sm} of {mx} MHz with no reason"
    return None


# ---------------------------------------------------------------------------
# synthetic workload on the device (input generation only)
# ---------------------------------------------------------------------------
def make_workload(T, torch, nfreq, seed, device):
    """D, U stacks (paper layout, complex64) and start points theta0 per frequency."""
    g = torch.Generator(device=device).manual_seed(seed)
    n = NR

    def cn(shape):
        re = torch.randn(shape, generator=g, device=device, dtype=torch.float32)
        im = torch.randn(shape, generator=g, device=device, dtype=torch.float32)
        return torch.complex(re, im) * (1.0 / math.sqrt(2.0))

    # exactly unitary random-phase DFT products (tlr_synth recipe), built on the host
    import tlr_synth as synth
    hg = synth.rng(seed)
    Q = torch.from_numpy(synth.phase_dft_unitary(n, hg).astype(np.complex64)).to(device)
    W = torch.from_numpy(synth.phase_dft_unitary(n, hg).astype(np.complex64)).to(device)
    sig = torch.pow(10.0, -3.0 * torch.arange(n, device=device, dtype=torch.float32) / (n - 1))
    perm = torch.empty(n, dtype=torch.int32, device=device)
    T.tlr_mdd_hilbert_perm(GRID[0], GRID[1], perm)
    inv = torch.empty_like(perm)
    inv[perm.long()] = torch.arange(n, dtype=torch.int32, device=device)
    D = torch.empty((nfreq, n, n), dtype=torch.complex64, device=device)
    U = torch.empty_like(D)
    thetas, descs, ranks = [], [], []
    b = TILE
    N = n // b
    pairs = [(i, j) for j in range(N) for i in range(j + 1, N)]
    for f in range(nfreq):
        k = rank_of(f, nfreq)
        ranks.append(k)
        ph = torch.exp(2j * math.pi * torch.rand(n, generator=g, device=device)).to(torch.complex64)
        D[f] = (Q * (sig * ph)[None, :]) @ W.conj().T
        # planted X_h (Hilbert order) from random factors, then X = S X_h S^T
        Xh = torch.zeros((n, n), dtype=torch.complex64, device=device)
        for i in range(N):
            Qi = cn((b, k)) / math.sqrt(b * k)
            Xh[i * b:(i + 1) * b, i * b:(i + 1) * b] = Qi @ Qi.T
        for (i, j) in pairs:
            s = 1.0 / ((1 + abs(i - j)) * math.sqrt(b * k))
            L, R = cn((b, k)) * s, cn((b, k)) * s
            t = L @ R.T
            Xh[i * b:(i + 1) * b, j * b:(j + 1) * b] = t
            Xh[j * b:(j + 1) * b, i * b:(i + 1) * b] = t.T
        X = Xh[inv.long()][:, inv.long()]
        Y = D[f] @ X
        nz = cn((n, n))
        scale = Y.norm() / nz.norm() * 10 ** (-SNR_DB / 20)
        U[f] = Y + scale * nz
        d = T.desc(n, n, b, rank=k, nx=GRID[0], ny=GRID[1], diag_mode=T.TLR_DIAG_RULE)
        descs.append(d)
        nth = T.tlr_mdd_theta_size(d)
        th0 = cn((nth,)) * (0.1 / math.sqrt(b * k))
        thetas.append(th0)
        del Xh, X, Y, nz
    return D, U, thetas, descs, ranks


def measured_bf16_sustained():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            j = json.load(fh)
        return float(j["bf16_tflops_sustained"]), "measured sustained"
    except (OSError, KeyError, ValueError):
        return 1700.0, "fallback sustained"


def percentile(xs, p):
    xs = sorted(xs)
    if not xs:
        return None
    i = min(len(xs) - 1, max(0, int(math.ceil(p / 100.0 * len(xs))) - 1))
    return xs[i]


# ---------------------------------------------------------------------------
# CPU oracle leg (bounded sample)
# ---------------------------------------------------------------------------
def oracle_sample(D0, U0, k, lbfgs_iters):
    """Time the FP64 oracle's TLR-structured solve on one frequency for a few
    L-BFGS iterations; returns (seconds, iterations, theta, threads)."""
    from oracle import hilbert, layout, operator, solver
    perm = hilbert.perm(*GRID)
    lay = layout.make_layout(NR, TILE, k, "rule")
    Dh, Uh, alpha = operator.normalise(D0, U0, perm)
    prob = solver.Problem(lay, Dh.T, Uh.T)
    return prob, lay, perm, alpha


def run_oracle(prob, th0, iters):
    from oracle import solver
    opts = solver.SolveOpts(stages=1, admm_iters=1, lbfgs_iters=iters)
    t0 = time.perf_counter()
    th, z, u, st = solver.admm(prob, th0, opts)
    return time.perf_counter() - t0, th, st


def blas_threads():
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(k):
            return int(os.environ[k])
    return os.cpu_count()


# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16x3", choices=["fp32", "bf16x3"])
    ap.add_argument("--compare-fp32", type=int, default=8,
                    help="frequencies (evenly spaced) re-solved with the FP32 SIMT path for the speedup")
    ap.add_argument("--freqs", type=int, default=NFREQ)
    ap.add_argument("--seed", type=int, default=2412)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--streams", type=int, default=4, help="CUDA streams the frequencies are spread over")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--oracle-iters", type=int, default=3)
    ap.add_argument("--bench-iters", type=int, default=20,
                    help="CG iterations of the eq. (4) benchmark solver timed on frequency 0 (0: skip)")
    ap.add_argument("--general-rank", type=int, default=26,
                    help="rank of one timed solve of the general (non-reciprocal) form on frequency 0 (0: skip)")
    ap.add_argument("--tiles-rank", type=int, default=26,
                    help="rank of one timed solve on a non-uniform partition (tiles of 192 and 320 "
                         "receivers alternating) of frequency 0 (0: skip)")
    ap.add_argument("--serving", type=int, default=0,
                    help="also serve this many per-frequency requests of the serving mix (nr 1024-8192)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return reference_arm(args, world, rank)

    import torch
    import paper_2412_14973_gb300 as T

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    nfreq = args.freqs
    with torch.cuda.stream(stream):
        D, U, th0, descs, ranks = make_workload(T, torch, nfreq, args.seed + 7919 * rank, dev)
    torch.cuda.synchronize()
    prec = T.TLR_PREC_FP32 if args.precision == "fp32" else T.TLR_PREC_BF16X3
    for d in descs:
        d.precision = prec
    theta = [t.clone() for t in th0]
    opts = T.solve_opts()
    lat_ms = []
    # one handle per frequency, kept across steps (workspace and recorded
    # solve); each step re-runs the data step (alpha, reorder, normalise)
    nstream = max(1, min(args.streams, nfreq))
    streams = [torch.cuda.Stream(device=dev) for _ in range(nstream)]
    handles = [T.tlr_mdd_create(descs[f], D[f], U[f], streams[f % nstream]) for f in range(nfreq)]
    main_stream = torch.cuda.current_stream(dev)

    def step(record=False, host=None):
        """One pass over every frequency; returns the device ms between the
        start event (main stream) and the join of all worker streams."""
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(main_stream)
        for s_ in streams:
            s_.wait_event(e0)
        for f in range(nfreq):
            st_ = streams[f % nstream]
            if host is None:
                T.tlr_mdd_set_data(handles[f], D[f], U[f], T.TLR_MEM_DEVICE)
                with torch.cuda.stream(st_):
                    theta[f].copy_(th0[f])
                T.tlr_mdd_solve_async(handles[f], theta[f], opts)
            else:
                Dh_, Uh_, th_h_, out_h_, hopts_ = host
                T.tlr_mdd_set_data(handles[f], Dh_[f], Uh_[f], T.TLR_MEM_HOST)
                out_h_[f].copy_(th_h_[f])
                T.tlr_mdd_solve_async(handles[f], out_h_[f], hopts_)
        for f in range(nfreq):
            st = T.tlr_mdd_solve_wait(handles[f])
            if record:
                lat_ms.append(st.gpu_ms)
        for s_ in streams:
            ev = torch.cuda.Event()
            ev.record(s_)
            main_stream.wait_event(ev)
        e1.record(main_stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    T.tlr_mdd_timing_reset()
    T.tlr_mdd_timing_enable(True)
    step()   # records the solve graphs with the timing events (not timed)
    def timed_region():
        T.tlr_mdd_timing_reset()
        lat_ms.clear()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        n0 = T.tlr_mdd_launch_count()
        clk = ClockSampler(local)
        clk.start()
        ms = 0.0
        for _ in range(args.steps):
            ms += step(record=True)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        return ms, clk.stop(), T.tlr_mdd_launch_count() - n0, T.tlr_mdd_timing_read()

    ms, clocks, launches, timing = timed_region()
    # a timed region that saw a hardware or thermal slowdown, or SM clocks held
    # far below their maximum with no reason given (a clock lock), is measured
    # once more and that second measurement is reported
    bad = clock_problem(clocks)
    if bad:
        ms, clocks, launches, timing = timed_region()
        clocks["remeasured_after"] = bad
        clocks["still_flagged"] = clock_problem(clocks)
    T.tlr_mdd_timing_enable(False)
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    solves = nfreq * args.steps * world
    value = solves / (ms / 1e3)
    total_flops = sum(flops_per_solve(NR, NR, TILE, k) for k in ranks) * args.steps * world

    # roofline of the dominant contraction kernel
    names = ["cgemm_compress", "cgemm_expand", "cgemm_project"]
    dom = max(range(len(timing)), key=lambda c: timing[c][0])
    dms, dfl, dnl = timing[dom]
    achieved = (dfl / max(1, dnl)) / (dms / max(1, dnl) / 1e3) / 1e12 if dnl else 0.0
    if args.precision == "fp32":
        peak = FP32_LANES_PER_SM * SMS * 2 * SM_MAX_MHZ * 1e6 / 1e12
        roof = {"bound": "alu", "kernel": names[dom], "achieved": round(achieved, 3),
                "peak": round(peak, 2), "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": None,
                "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz (unit counts and max clock)"}
    else:
        bf16, src = measured_bf16_sustained()
        # 4M x BF16x3: 12 real BF16 products = 24 flops issued per complex MAC counted as 8
        peak = bf16 * 8.0 / 24.0
        roof = {"bound": "tensor", "kernel": names[dom], "achieved": round(achieved, 3),
                "peak": round(peak, 2), "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": None,
                "bf16_issued_tflops": round(achieved * 24.0 / 8.0, 2),
                "peak_source": f"{src} bf16 {bf16} TFLOP/s x 8/24 (complex flops per issued BF16 flop, 4M x BF16x3)"}
    roof["per_class_ms"] = {names[c]: round(timing[c][0], 2) for c in range(len(timing))}
    # launches of different frequencies overlap on the 4 streams, so a launch's
    # event-timed duration includes time shared with other launches; the
    # device-wide rate below is all contraction flops over the timed wall time
    roof["aggregate_contraction_tflops"] = round(sum(t[1] for t in timing) / (ms / 1e3) / 1e12, 2)
    roof["aggregate_frac"] = round(roof["aggregate_contraction_tflops"] / peak, 4)

    # e2e through the C-ABI with HOST buffers: every step copies each
    # frequency's D, U and start point from pinned host memory inside the
    # timed region and reads the solved factors back
    e2e = None
    if not args.no_e2e:
        Dh = torch.empty((nfreq, NR, NR), dtype=torch.complex64, pin_memory=True)
        Uh = torch.empty_like(Dh, pin_memory=True)
        Dh.copy_(D)
        Uh.copy_(U)
        th_h = [t.cpu().pin_memory() for t in th0]
        out_h = [torch.empty_like(t).pin_memory() for t in th_h]
        hopts = T.solve_opts(theta_memory=T.TLR_MEM_HOST)
        host = (Dh, Uh, th_h, out_h, hopts)
        step(host=host)  # records the host-theta graphs
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(host=host)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        h2d = sum(2 * Dh[f].numel() * 8 + th_h[f].numel() * 8 for f in range(nfreq))
        d2h = sum(out_h[f].numel() * 8 for f in range(nfreq))
        e2e = {"value": round(nfreq * world / te, 4), "unit": "freq-solves/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
        del Dh, Uh

    # the plain FP32 SIMT form on an evenly spaced subset, same subset on tensor cores
    cmp = None
    if args.precision != "fp32" and args.compare_fp32 > 0:
        sub = sorted(set(int(round(i * (nfreq - 1) / max(1, args.compare_fp32 - 1)))
                         for i in range(min(args.compare_fp32, nfreq))))

        def run_subset(prec_):
            hs = []
            for f in sub:
                d = T.desc(NR, NR, TILE, rank=ranks[f], nx=GRID[0], ny=GRID[1], diag_mode=T.TLR_DIAG_RULE,
                           precision=prec_)
                hs.append(T.tlr_mdd_create(d, D[f], U[f], streams[0]))
            ms_tot = 0.0
            for rep in range(2):          # first pass records the graphs
                if rep == 1 and prec_ == prec and prec != T.TLR_PREC_FP32:
                    T.tlr_mdd_timing_reset()
                    T.tlr_mdd_timing_enable(True)
                t0_ = torch.cuda.Event(enable_timing=True)
                t1_ = torch.cuda.Event(enable_timing=True)
                t0_.record(streams[0])
                for h_, f in zip(hs, sub):
                    T.tlr_mdd_set_data(h_, D[f], U[f], T.TLR_MEM_DEVICE)
                    with torch.cuda.stream(streams[0]):
                        theta[f].copy_(th0[f])
                    T.tlr_mdd_solve(h_, theta[f], opts)
                t1_.record(streams[0])
                torch.cuda.synchronize()
                if rep == 1:
                    ms_tot = t0_.elapsed_time(t1_)
                    if T.tlr_mdd_timing_read and prec_ == prec and prec != T.TLR_PREC_FP32:
                        single[:] = T.tlr_mdd_timing_read()
                        T.tlr_mdd_timing_enable(False)
            for h_ in hs:
                T.tlr_mdd_destroy(h_)
            return ms_tot

        single = []
        t_fp32 = run_subset(T.TLR_PREC_FP32)
        t_tc = run_subset(prec)
        if single:
            # one stream, no overlap between launches: per-launch rates of each class
            roof["single_stream_tflops_per_class"] = {
                names[c]: round(single[c][1] / (single[c][0] / 1e3) / 1e12, 1) for c in range(len(single))
                if single[c][0] > 0}
            roof["single_stream_frac_per_class"] = {
                k: round(v / roof["peak"], 4) for k, v in roof["single_stream_tflops_per_class"].items()}
        cmp = {"frequencies": sub, "fp32_simt_freq_solves_per_s": round(len(sub) / (t_fp32 / 1e3), 4),
               "tensor_core_freq_solves_per_s": round(len(sub) / (t_tc / 1e3), 4),
               "speedup_tc_vs_fp32": round(t_fp32 / t_tc, 3),
               "accuracy": "both paths within 1e-5 (FP32) / 1e-5 (BF16x3, measured) of the FP64 oracle per operator; see tests"}

    # the eq. (4) benchmark solver (warm-start stage) on frequency 0's handle:
    # G = D^H D and D^H U once, then one nr^3 complex product per CG iteration
    bsolve = None
    if args.bench_iters > 0 and rank == 0:
        Xb = torch.empty((NR, NR), dtype=torch.complex64, device=dev)
        T.tlr_mdd_set_data(handles[0], D[0], U[0], T.TLR_MEM_DEVICE)
        T.tlr_mdd_benchmark_solve(handles[0], 0.1, 2, 0.0, Xb)          # warm-up
        bst = T.tlr_mdd_benchmark_solve(handles[0], 0.1, args.bench_iters, 0.0, Xb)
        fl = 2 * 8.0 * NR * NR * NR + bst.iters * 8.0 * NR ** 3
        tf = fl / (bst.gpu_ms / 1e3) / 1e12
        bsolve = {"nr": NR, "ns": NR, "lambda": 0.1, "iters": bst.iters, "ms": round(bst.gpu_ms, 2),
                  "ms_per_iter": round(bst.gpu_ms / max(1, bst.iters + 2), 3),
                  "tflops": round(tf, 1), "frac": round(tf / roof["peak"], 4) if args.precision != "fp32" else None,
                  "rel_res": bst.rel_res,
                  "flops": "8 nr^2 ns (D^H D) + 8 nr^2 ns (D^H U) + iters x 8 nr^3, complex-counted"}
        del Xb

    # the general (non-reciprocal) form: one solve of frequency 0's data at a
    # given rank (same contraction flops per iteration as the reciprocal form
    # at that rank, twice the unknowns)
    gsolve = None
    if args.general_rank > 0 and rank == 0:
        kg = args.general_rank
        dg = T.desc(NR, NR, TILE, rank=kg, nx=GRID[0], ny=GRID[1], diag_mode=T.TLR_DIAG_RULE,
                    precision=prec, reciprocity=T.TLR_RECIP_NONE)
        hg = T.tlr_mdd_create(dg, D[0], U[0], streams[0])
        gen = torch.Generator(device=dev).manual_seed(args.seed + 5)
        ntg = T.tlr_mdd_theta_size(dg)
        th_g0 = 0.01 * torch.randn(ntg, dtype=torch.complex64, device=dev, generator=gen)
        th_g = th_g0.clone()
        torch.cuda.synchronize()
        T.tlr_mdd_solve(hg, th_g, opts)                                   # records the graph
        th_g.copy_(th_g0)
        torch.cuda.synchronize()
        gst = T.tlr_mdd_solve(hg, th_g, opts)
        gf = flops_per_solve(NR, NR, TILE, kg)
        gsolve = {"rank": kg, "n_theta": ntg, "ms": round(gst.gpu_ms, 2),
                  "tflops": round(gf / (gst.gpu_ms / 1e3) / 1e12, 1), "iters": gst.iters,
                  "note": "one solve, one stream; flops as for the reciprocal form at this rank"}
        T.tlr_mdd_destroy(hg)

    # a non-uniform partition: 16 tiles of 192 and 320 receivers alternating
    # (sum 4096), the same rank on every tile; with N tiles and rank k the
    # low-rank entries are N k nr, as for equal tiles
    tsolve = None
    if args.tiles_rank > 0 and rank == 0 and NR == 4096:
        kt = args.tiles_rank
        tiles = [192, 320] * 8
        dt = T.desc(NR, NR, 0, rank=kt, nx=GRID[0], ny=GRID[1], diag_mode=T.TLR_DIAG_RULE,
                    precision=prec, tiles=tiles)
        ht = T.tlr_mdd_create(dt, D[0], U[0], streams[0])
        gen = torch.Generator(device=dev).manual_seed(args.seed + 6)
        ntt = T.tlr_mdd_theta_size(dt)
        th_t0 = 0.01 * torch.randn(ntt, dtype=torch.complex64, device=dev, generator=gen)
        th_t = th_t0.clone()
        torch.cuda.synchronize()
        T.tlr_mdd_solve(ht, th_t, opts)                                   # records the graph
        th_t.copy_(th_t0)
        torch.cuda.synchronize()
        tst = T.tlr_mdd_solve(ht, th_t, opts)
        T.tlr_mdd_destroy(ht)
        # the same rank on 16 equal tiles, for comparison
        du = T.desc(NR, NR, NR // 16, rank=kt, nx=GRID[0], ny=GRID[1], diag_mode=T.TLR_DIAG_RULE, precision=prec)
        hu = T.tlr_mdd_create(du, D[0], U[0], streams[0])
        th_u0 = 0.01 * torch.randn(T.tlr_mdd_theta_size(du), dtype=torch.complex64, device=dev, generator=gen)
        th_u = th_u0.clone()
        torch.cuda.synchronize()
        T.tlr_mdd_solve(hu, th_u, opts)
        th_u.copy_(th_u0)
        torch.cuda.synchronize()
        ust = T.tlr_mdd_solve(hu, th_u, opts)
        T.tlr_mdd_destroy(hu)
        tf = (ITERS_PER_SOLVE * 56.0 + 40.0) * NR * ntt
        tsolve = {"tiles": "192,320 alternating x8", "rank": kt, "n_theta": ntt, "ms": round(tst.gpu_ms, 2),
                  "tflops": round(tf / (tst.gpu_ms / 1e3) / 1e12, 1), "iters": tst.iters,
                  "equal_tiles_ms": round(ust.gpu_ms, 2),
                  "note": "one solve, one stream; equal_tiles_ms: 16 tiles of 256 at the same rank "
                          "(same flops); 192- and 320-row blocks fill 75% and 83% of their 128-row MMA tiles"}

    # CPU oracle baseline (rank 0 only, N = 1 only) + accuracy at the sample
    cpu = None
    acc = None
    if rank == 0 and world == 1 and not args.no_cpu:
        f0 = 0
        k0 = ranks[f0]
        D0 = D[f0].cpu().numpy()
        U0 = U[f0].cpu().numpy()
        prob, lay, perm, alpha = oracle_sample(D0, U0, k0, args.oracle_iters)
        th_start = th0[f0].cpu().numpy().astype(np.complex128)
        secs, th_or, st_or = run_oracle(prob, th_start, args.oracle_iters)
        # GPU with the same short schedule for the accuracy check
        h = T.tlr_mdd_create(descs[f0], D[f0], U[f0], stream)
        thg = th0[f0].clone()
        T.tlr_mdd_solve(h, thg, T.solve_opts(stages=1, admm_iters=1, lbfgs_iters=args.oracle_iters))
        T.tlr_mdd_destroy(h)
        from oracle import operator
        Xo = operator.assemble_xh(th_or, lay)
        Xg = operator.assemble_xh(thg.cpu().numpy().astype(np.complex128), lay)
        rel = float(np.linalg.norm(Xg - Xo) / np.linalg.norm(Xo))
        kmean = sum(ranks) / len(ranks)
        per_solve = secs * (ITERS_PER_SOLVE / args.oracle_iters) * (kmean / k0)
        cpu = {"value": round(1.0 / per_solve, 6), "unit": "freq-solves/s", "cores": blas_threads(),
               "kind": "oracle",
               "sample": (f"frequency {f0} (rank {k0}), {args.oracle_iters} L-BFGS iterations of the FP64 "
                          f"TLR-structured oracle in {secs:.1f} s, scaled to a {ITERS_PER_SOLVE}-iteration "
                          f"solve at the mean rank {kmean:.1f} (work grows linearly with rank)")}
        acc = {"frequency": f0, "iters": args.oracle_iters, "rel_err_X_vs_fp64_oracle": rel,
               "within_1e-3": rel <= 1e-3}

    for h_ in handles:
        T.tlr_mdd_destroy(h_)
    serve = None
    if args.serving > 0 and rank == 0:
        del D, U
        torch.cuda.empty_cache()
        serve = serving_leg(T, torch, args.serving, args.seed, dev)
    if rank != 0:
        return
    line = {
        "metric": "freq-solves/s", "value": round(value, 4), "unit": "freq-solves/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms / args.steps, 2), "higher_is_better": True, "scaling": "weak",
        "streams": nstream,
        "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "bf16x3",
        "data": "synthetic",
        "config": {"workload": "plain-method batched frequencies: nr=ns=4096 (64x64 grid, Hilbert order), "
                               "64 frequencies, tile 256, rank 4->48, low-rank diagonal, 10 dB SNR",
                   "nr": NR, "ns": NR, "frequencies_per_gpu": nfreq, "tile": TILE,
                   "ranks": f"{RANK_LO}->{RANK_HI} linear", "iters_per_solve": ITERS_PER_SOLVE,
                   "precision": args.precision,
                   "l2": "inputs larger than L2 (each 4096x4096 complex64 panel is 134 MB; 64 frequencies cycled)",
                   "parallelism": f"frequency sharding x{world}"},
        "gflops": round(total_flops / (ms / 1e3) / 1e9, 1),
        "latency_ms": {"p50": percentile(lat_ms, 50), "p99": percentile(lat_ms, 99)},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
        "gpu_launches": launches, "accuracy": acc, "fp32_comparison": cmp,
    }
    if bsolve is not None:
        line["benchmark_solver"] = bsolve
    if gsolve is not None:
        line["general_form"] = gsolve
    if tsolve is not None:
        line["nonuniform_tiles"] = tsolve
    if serve is not None:
        line["serving"] = serve
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def serving_leg(T, torch, n, seed, dev):
    """The serving mix: per-frequency solve requests with nr = ns uniform over
    {1024, 2048, 4096, 8192}, tile over {128, 256, 512}, rank log-uniform 2-64,
    Poisson arrivals.  Measures one-at-a-time throughput on the FP32 and the
    tensor-core paths, then serves the stream with continuous batching (4
    slots, HBM budget 200 GB) at 90% of the tensor-core one-at-a-time capacity
    and at 0.7x and 1.3x the FP32 one-at-a-time capacity, and reports p50 /
    p99 latency.  One seeded D, U per problem size is shared
    by the requests of that size (work does not depend on the values)."""
    import tlr_synth as synth
    from paper_2412_14973_gb300 import serving
    reqs = synth.request_stream(n, 1.0, seed + 17)
    g = torch.Generator(device=dev).manual_seed(seed + 18)
    pool = {}
    for r in reqs:
        if r.nr not in pool:
            re = torch.randn((r.nr, r.nr), generator=g, device=dev)
            im = torch.randn((r.nr, r.nr), generator=g, device=dev)
            Dm = (torch.complex(re, im) / math.sqrt(2 * r.nr)).to(torch.complex64)
            re = torch.randn((r.nr, r.nr), generator=g, device=dev)
            im = torch.randn((r.nr, r.nr), generator=g, device=dev)
            Um = (torch.complex(re, im) / math.sqrt(2 * r.nr)).to(torch.complex64)
            pool[r.nr] = (Dm, Um)

    def make(prec, arrivals):
        out = []
        for r, t in zip(reqs, arrivals):
            d = T.desc(r.nr, r.nr, r.tile, rank=r.rank, nx=r.nx, ny=r.ny, diag_mode=T.TLR_DIAG_RULE,
                       precision=prec)
            nth = T.tlr_mdd_theta_size(d)
            gg = torch.Generator(device=dev).manual_seed(r.seed)
            th = (torch.randn(nth, generator=gg, device=dev) + 1j * torch.randn(nth, generator=gg, device=dev))
            th = (th * (0.1 / math.sqrt(r.tile * max(1, r.rank)))).to(torch.complex64)
            out.append(serving.SolveRequest(r.rid, t, d, pool[r.nr][0], pool[r.nr][1], th, T.solve_opts()))
        return out

    budget = 200 << 30
    zero = [0.0] * n
    t0 = time.perf_counter()
    res_fp32 = serving.Server(budget, max_active=1).run(make(T.TLR_PREC_FP32, zero), realtime=False)
    t_fp32 = time.perf_counter() - t0
    t0 = time.perf_counter()
    res_tc1 = serving.Server(budget, max_active=1).run(make(T.TLR_PREC_BF16X3, zero), realtime=False)
    t_tc1 = time.perf_counter() - t0
    rate = 0.9 * n / t_tc1
    gg = np.random.default_rng(seed + 19)
    arrivals = list(np.cumsum(gg.exponential(1.0 / rate, n)))
    srv = serving.Server(budget, max_active=4)
    t0 = time.perf_counter()
    res = srv.run(make(T.TLR_PREC_BF16X3, arrivals), realtime=True)
    t_srv = time.perf_counter() - t0
    ok = [r for r in res if r.status == 0]
    pc = serving.percentiles(res)
    same = all(torch.equal(a.theta, b.theta) for a, b in zip(res_tc1, res) if a.status == 0 and b.status == 0)
    # the tensor-core server at 0.7x and 1.3x the FP32 path's one-at-a-time
    # capacity (the FP32 path alone would keep up with the first and not the second)
    loads = []
    for x in (0.7, 1.3):
        rx = x * n / t_fp32
        ax = list(np.cumsum(np.random.default_rng(seed + 20).exponential(1.0 / rx, n)))
        sx = serving.Server(budget, max_active=4)
        t0 = time.perf_counter()
        rs = sx.run(make(T.TLR_PREC_BF16X3, ax), realtime=True)
        tx = time.perf_counter() - t0
        px = serving.percentiles(rs)
        loads.append({"x_fp32_capacity": x, "arrival_rate_hz": round(rx, 3),
                      "completed": sum(1 for r in rs if r.status == 0), "served_solves_per_s": round(n / tx, 3),
                      "p50_ms": round(1e3 * px[50], 1) if px[50] else None,
                      "p99_ms": round(1e3 * px[99], 1) if px[99] else None})
    return {"requests": n, "completed": len(ok), "arrival_rate_hz": round(rate, 3),
            "fp32_one_at_a_time_solves_per_s": round(n / t_fp32, 3),
            "tc_one_at_a_time_solves_per_s": round(n / t_tc1, 3),
            "tc_served_solves_per_s": round(len(ok) / t_srv, 3),
            "p50_ms": round(1e3 * pc[50], 1) if pc[50] else None,
            "p99_ms": round(1e3 * pc[99], 1) if pc[99] else None,
            "peak_active": srv.peak_active, "peak_budget_gb": round(srv.peak_used / 2**30, 1),
            "results_identical_alone_and_in_mix": bool(same),
            "fp32_capacity_load_points": loads,
            "mix": "nr=ns in {1024,2048,4096,8192}, tile in {128,256,512}, rank log-uniform 2-64, Poisson"}


def reference_arm(args, world, rank):
    """The FP64 CPU oracle on this workload's config, a bounded sample per step."""
    if rank != 0:
        return
    import tlr_synth as synth
    from oracle import hilbert
    k0 = rank_of(0, args.freqs)
    # one frequency of the same recipe, generated on the host
    D0 = synth.make_d(NR, NR, 1, args.seed, haar_max=1024)[0]
    lay_perm = hilbert.perm(*GRID)
    from oracle import layout, operator
    lay = layout.make_layout(NR, TILE, k0, "rule")
    th_true = synth.planted_theta(NR, TILE, k0, lay.dense, args.seed + 1)
    X = operator.unpermute(operator.assemble_xh(th_true, lay), lay_perm)
    Y = D0.astype(np.complex128) @ X
    nz = synth.noise(Y.shape, args.seed + 2)
    U0 = (Y + np.linalg.norm(Y) / np.linalg.norm(nz) * 10 ** (-SNR_DB / 20) * nz).astype(np.complex64)
    prob, lay, perm, alpha = oracle_sample(D0, U0, k0, args.oracle_iters)
    th0 = 0.1 * synth.planted_theta(NR, TILE, k0, lay.dense, args.seed + 3)
    for _ in range(args.warmup):
        run_oracle(prob, th0, args.oracle_iters)
    t = 0.0
    for _ in range(args.steps):
        s, _, _ = run_oracle(prob, th0, args.oracle_iters)
        t += s
    ranks = [rank_of(f, args.freqs) for f in range(args.freqs)]
    kmean = sum(ranks) / len(ranks)
    per_solve = (t / args.steps) * (ITERS_PER_SOLVE / args.oracle_iters) * (kmean / k0)
    v = 1.0 / per_solve
    sample = (f"per step: frequency 0 (rank {k0}), {args.oracle_iters} L-BFGS iterations of the FP64 "
              f"TLR-structured oracle, scaled to a {ITERS_PER_SOLVE}-iteration solve at mean rank {kmean:.1f}")
    line = {"impl": "reference", "metric": "freq-solves/s", "value": round(v, 6), "unit": "freq-solves/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * t / args.steps, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "plain-method batched frequencies: nr=ns=4096 (64x64 grid, Hilbert order), "
                                   "64 frequencies, tile 256, rank 4->48, low-rank diagonal, 10 dB SNR",
                       "nr": NR, "ns": NR, "frequencies_per_gpu": args.freqs, "tile": TILE,
                       "ranks": f"{RANK_LO}->{RANK_HI} linear", "iters_per_solve": ITERS_PER_SOLVE,
                       "precision": "fp64 (oracle)", "parallelism": f"frequency sharding x{world}"},
            "cpu_baseline": {"value": round(v, 6), "unit": "freq-solves/s", "cores": blas_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(v, 6), "unit": "freq-solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
