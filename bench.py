#!/usr/bin/env python
"""Frequency-solve throughput of reciprocity-aware TLR MDD on GB300.

Workload (the precision-form configuration, the largest that fits one GPU):
nr = ns = 9216 receivers / sources on a 96 x 96 grid (Hilbert order on the
128 x 128 square), 128 frequencies, tile 384 (24 x 24 tiles), off-diagonal rank
rising linearly 8 -> 64 with frequency, low-rank diagonal tiles (rank < tile/4),
complex contractions as BF16x3 on the tcgen05 tensor cores with FP32
accumulation, FP64 reductions.  D(w) = Q diag(sigma e^{i phi_w}) W^H (sigma
decaying 1 -> 1e-3, Q and W exactly unitary random-phase DFT products),
U = D X + complex Gaussian noise at 10 dB SNR, X a planted symmetric TLR
Green's function.  One frequency solve = 30 L-BFGS iterations (3 lambda stages
x 2 ADMM iterations x 5).  One step = the solves of one batch of 8 of the 128
frequencies (every 16th, so each batch spans the rank range; 16 batches cover
all 128), each from its raw D, U (data step included: Hilbert reorder,
normalisation, packing); inputs resident in HBM.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
instead (the only place besides the cpu_baseline leg that runs it).
``--gpus N`` without a torchrun environment starts the N ranks itself.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import socket
import statistics
import subprocess
import sys
import tempfile
import time
from dataclasses import dataclass

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

ITERS_PER_SOLVE = 30


@dataclass(frozen=True)
class Workload:
    name: str
    nr: int
    grid: tuple
    tile: int
    nfreq: int        # frequencies per GPU
    rank_lo: int
    rank_hi: int
    snr_db: float
    batch: int        # frequencies per step

    def ranks(self, total: int) -> list:
        """k_f = lo + floor((hi - lo) f / (F - 1) + 1/2) over the job's F frequencies."""
        if total == 1:
            return [self.rank_lo]
        return [self.rank_lo + int(math.floor((self.rank_hi - self.rank_lo) * f / (total - 1) + 0.5))
                for f in range(total)]


PRECISION_FORM = Workload(
    "precision form: nr=ns=9216 (96x96 grid, Hilbert order), 128 frequencies, tile 384, rank 8->64, "
    "low-rank diagonal, 10 dB SNR, BF16x3 tensor cores", 9216, (96, 96), 384, 128, 8, 64, 10.0, 8)
BATCHED = Workload(
    "plain-method batched frequencies: nr=ns=4096 (64x64 grid, Hilbert order), 64 frequencies, tile 256, "
    "rank 4->48, low-rank diagonal, 10 dB SNR", 4096, (64, 64), 256, 64, 4, 48, 10.0, 64)


def n_lr(nr, tile, k):
    n = nr // tile
    return n * n * tile * k


def flops_per_iter(nr, ns, tile, k):
    """Algorithmic flops of one L-BFGS iteration (8 real flops per complex MAC):
    compress of the direction and of the residual (8 + 8), the two line-search
    expands (16 + 8) and the gradient projection (16), all x ns x n_LR.  The
    factor products T and the residual are carried between iterations and
    updated in place, so an iteration has no fresh forward product (72 -> 56)."""
    return 56.0 * ns * n_lr(nr, tile, k)


def flops_per_solve(nr, ns, tile, k, iters=ITERS_PER_SOLVE):
    """The iterations plus the solve's first forward product and gradient (40)."""
    return iters * flops_per_iter(nr, ns, tile, k) + 40.0 * ns * n_lr(nr, tile, k)


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


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            j = json.load(fh)
        return float(j["bf16_tflops_sustained"]), float(j.get("hbm_gbs", 6794.1)), "measured"
    except (OSError, KeyError, ValueError):
        return 1700.0, 6800.0, "fallback"


# DRAM bytes per contraction launch (dram__bytes_read.sum + dram__bytes_write.sum,
# mean over the 992 contraction launches of one step of the nr = 9216 workload:
# the 8 frequencies of ranks 8, 15, ..., 57 solved on one stream), from one ncu
# capture of the sources whose SHA-256 is GEMM_TRAFFIC_SHA.  A change to any of
# those sources, another rank mix or another tile voids the figures (traffic null).
GEMM_TRAFFIC_SOURCES = ("k_gemm_tcp.cu", "api.cu", "internal.h")
GEMM_TRAFFIC_SHA = "e581fcb16358b17cf51da7bbe9389e1ba4ced8619b74d2b3ae55e566bada001a"
GEMM_TRAFFIC_CASE = {"nr": 9216, "tile": 384, "ranks": [8, 15, 22, 29, 36, 43, 50, 57], "precision": "bf16x3"}
GEMM_TRAFFIC_BYTES = {"cgemm_compress": 2098697744, "cgemm_expand": 4456706142, "cgemm_project": 4685540407}


def gemm_traffic(kernel, nr, tile, step_ranks, precision):
    """Measured DRAM bytes per launch of `kernel`, or None when the capture does not apply."""
    import hashlib
    h = hashlib.sha256()
    for f in GEMM_TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2412_14973_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    case = {"nr": nr, "tile": tile, "ranks": list(step_ranks), "precision": precision}
    if h.hexdigest() != GEMM_TRAFFIC_SHA or case != GEMM_TRAFFIC_CASE:
        return None
    return GEMM_TRAFFIC_BYTES.get(kernel)


# CTAs per SM of a fused update-and-pack launch when several streams share
# the GPU (beside two contraction CTAs an SM has registers for two; one per
# SM measured best: 4 streams 3.45 freq-solves/s against 3.43 with two and
# 3.32 uncapped)
PASS_CTAS_PER_SM = 1


def log(msg):
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def percentile(xs, p):
    xs = sorted(xs)
    if not xs:
        return None
    i = min(len(xs) - 1, max(0, int(math.ceil(p / 100.0 * len(xs))) - 1))
    return xs[i]


def blas_threads():
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(k):
            return int(os.environ[k])
    return os.cpu_count()


# ---------------------------------------------------------------------------
# synthetic workload on the device (input generation only, not timed)
# ---------------------------------------------------------------------------
def phase_dft_unitary_device(torch, n, g, device):
    """tlr_synth.phase_dft_unitary's matrix F diag(phi) Pi F diag(psi) / n from
    the same draws of g, with the two FFTs done on the device (complex64)."""
    psi = np.exp(2j * np.pi * g.random(n))
    phi = np.exp(2j * np.pi * g.random(n))
    pi = g.permutation(n)
    m = torch.fft.fft(torch.diag(torch.from_numpy(psi.astype(np.complex64)).to(device)), dim=0)
    m = m[torch.from_numpy(pi).to(device), :] * torch.from_numpy(phi.astype(np.complex64)).to(device)[:, None]
    return torch.fft.fft(m, dim=0) / n


class Inputs:
    """D, U (paper layout, complex64, device) and the start point theta0 of
    each of a rank's frequencies, generated on the device from per-frequency
    seeds, so any rank can regenerate any global frequency identically."""

    def __init__(self, T, torch, wl: Workload, freqs, ranks, seed, device):
        import tlr_synth as synth
        self.wl, self.freqs, self.ranks = wl, list(freqs), ranks
        n = wl.nr
        self.dev = device
        hg = synth.rng(seed)
        Q = phase_dft_unitary_device(torch, n, hg, device)
        W = phase_dft_unitary_device(torch, n, hg, device)
        sig = torch.pow(10.0, -3.0 * torch.arange(n, device=device, dtype=torch.float32) / (n - 1))
        perm = torch.empty(n, dtype=torch.int32, device=device)
        T.tlr_mdd_hilbert_perm(wl.grid[0], wl.grid[1], perm)
        inv = torch.empty_like(perm)
        inv[perm.long()] = torch.arange(n, dtype=torch.int32, device=device)
        inv = inv.long()
        self.D = torch.empty((len(freqs), n, n), dtype=torch.complex64, device=device)
        self.U = torch.empty_like(self.D)
        self.th0, self.descs = [], []
        b = wl.tile
        N = n // b
        pairs = [(i, j) for j in range(N) for i in range(j + 1, N)]
        tf32 = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = True   # generation only: far below the 10 dB noise
        try:
            for slot, f in enumerate(freqs):
                k = ranks[f]
                g = torch.Generator(device=device).manual_seed(seed * 1000003 + f)

                def cn(shape):
                    re = torch.randn(shape, generator=g, device=device, dtype=torch.float32)
                    im = torch.randn(shape, generator=g, device=device, dtype=torch.float32)
                    return torch.complex(re, im) * (1.0 / math.sqrt(2.0))

                ph = torch.exp(2j * math.pi * torch.rand(n, generator=g, device=device)).to(torch.complex64)
                Df = (Q * (sig * ph)[None, :]) @ W.conj().T
                self.D[slot] = Df
                Xh = torch.zeros((n, n), dtype=torch.complex64, device=device)
                for i in range(N):
                    Qi = cn((b, k)) / math.sqrt(b * k)
                    Xh[i * b:(i + 1) * b, i * b:(i + 1) * b] = Qi @ Qi.T
                for (i, j) in pairs:
                    s = 1.0 / ((1 + abs(i - j)) * math.sqrt(b * k))
                    t = (cn((b, k)) * s) @ (cn((b, k)) * s).T
                    Xh[i * b:(i + 1) * b, j * b:(j + 1) * b] = t
                    Xh[j * b:(j + 1) * b, i * b:(i + 1) * b] = t.T
                X = Xh[inv][:, inv]
                del Xh
                Y = Df @ X
                del X
                nz = cn((n, n))
                scale = Y.norm() / nz.norm() * 10 ** (-wl.snr_db / 20)
                self.U[slot] = Y + scale * nz
                del Y, nz, Df
                d = T.desc(n, n, b, rank=k, nx=wl.grid[0], ny=wl.grid[1], diag_mode=T.TLR_DIAG_RULE,
                           precision=T.TLR_PREC_BF16X3)
                self.descs.append(d)
                nth = T.tlr_mdd_theta_size(d)
                self.th0.append(cn((nth,)) * (0.1 / math.sqrt(b * k)))
        finally:
            torch.backends.cuda.matmul.allow_tf32 = tf32
        del Q, W
        self.slot_of = {f: s for s, f in enumerate(freqs)}

    def desc(self, T, f, precision):
        d = self.descs[self.slot_of[f]]
        wl = self.wl
        return T.desc(wl.nr, wl.nr, wl.tile, rank=d.rank, nx=wl.grid[0], ny=wl.grid[1],
                      diag_mode=T.TLR_DIAG_RULE, precision=precision)


class Runner:
    """Solves frequencies on S streams.  Each stream slot takes its next
    frequency, creates a handle for it from the raw D, U (receiver order,
    alpha, normalised panels, packed operands, all in the library), enqueues
    the solve, and destroys the handle when the solve has finished; the
    library's workspace pool keeps the freed memory for the next handle."""

    def __init__(self, T, torch, inp: Inputs, nstream, device, opts=None):
        self.T, self.torch, self.inp = T, torch, inp
        self.streams = [torch.cuda.Stream(device=device) for _ in range(nstream)]
        nmax = max(t.numel() for t in inp.th0)
        self.bufs = [torch.empty(nmax, dtype=torch.complex64, device=device) for _ in range(nstream)]
        self.opts = opts if opts is not None else T.solve_opts()
        self.main = torch.cuda.current_stream(device)

    def step(self, freqs, precision, host=None, records=None, lat=None):
        """One pass over ``freqs``; returns the device ms between a start event
        on the main stream and the join of the slot streams."""
        T, torch = self.T, self.torch
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(self.main)
        for s in self.streams:
            s.wait_event(e0)
        queue = list(freqs)
        busy = [None] * len(self.streams)
        while queue or any(b is not None for b in busy):
            progressed = False
            for si, st in enumerate(self.streams):
                if busy[si] is None and queue:
                    f = queue.pop(0)
                    slot = self.inp.slot_of[f]
                    d = self.inp.desc(T, f, precision)
                    if host is None:
                        h = T.tlr_mdd_create(d, self.inp.D[slot], self.inp.U[slot], st)
                        buf = self.bufs[si][:self.inp.th0[slot].numel()]
                        with torch.cuda.stream(st):
                            buf.copy_(self.inp.th0[slot])
                        T.tlr_mdd_solve_async(h, buf, self.opts)
                    else:
                        Dh, Uh, th_h, out_h, hopts = host     # pinned host tensors keyed by frequency
                        d.input_memory = T.TLR_MEM_HOST
                        h = T.tlr_mdd_create(d, Dh[f], Uh[f], st)
                        out_h[f].copy_(th_h[f])
                        T.tlr_mdd_solve_async(h, out_h[f], hopts)
                        buf = out_h[f]
                    busy[si] = (f, h, buf)
                    progressed = True
                elif busy[si] is not None and T.tlr_mdd_solve_query(busy[si][1]):
                    f, h, buf = busy[si]
                    stt = T.tlr_mdd_solve_wait(h)
                    T.tlr_mdd_destroy(h)
                    if lat is not None:
                        lat.append(stt.gpu_ms)
                    if records is not None:
                        records.append({"freq": f, "rank": self.inp.ranks[f], "iters": stt.iters,
                                        "restarts": stt.restarts, "status": stt.status,
                                        "f_final": stt.f_hist[max(0, stt.n_hist - 1)], "f0": stt.f0,
                                        "gpu_ms": round(stt.gpu_ms, 3)})
                    busy[si] = None
                    progressed = True
            if not progressed:
                time.sleep(2e-4)
        for s in self.streams:
            ev = torch.cuda.Event()
            ev.record(s)
            self.main.wait_event(ev)
        e1.record(self.main)
        e1.synchronize()
        return e0.elapsed_time(e1)


# ---------------------------------------------------------------------------
# CPU oracle legs
# ---------------------------------------------------------------------------
def oracle_problem(D0, U0, wl: Workload, k, cols=None):
    """The oracle's own panels (its Hilbert order, alpha = max |D|) for one
    frequency, optionally restricted to some source columns (rows of D, U)."""
    from oracle import hilbert, layout, operator, solver
    perm = hilbert.perm(*wl.grid)
    lay = layout.make_layout(wl.nr, wl.tile, k, "rule")
    alpha = float(np.max(np.abs(D0)))
    Ds, Us = (D0, U0) if cols is None else (D0[cols], U0[cols])
    Dh, Uh, _ = operator.normalise(Ds, Us, perm, alpha=alpha)
    return solver.Problem(lay, Dh.T, Uh.T), lay, alpha


def oracle_solve_rate(prob, th0):
    """Seconds of a 30-iteration oracle solve from one measured iteration:
    the first forward product and gradient are timed apart from the
    iteration (line-search products and the gradient at the new point), so
    the figure is first + 30 x iteration, both measured."""
    calls = []
    fgrad = prob.fgrad

    def timed_fgrad(theta):
        t0 = time.perf_counter()
        r = fgrad(theta)
        calls.append(time.perf_counter() - t0)
        return r

    prob.fgrad = timed_fgrad
    secs, th, st = run_oracle_solve(prob, th0, 1)
    prob.fgrad = fgrad
    t_first = calls[0]
    t_iter = secs - t_first
    return t_first + ITERS_PER_SOLVE * t_iter, secs, t_first, t_iter


def run_oracle_solve(prob, th0, iters):
    from oracle import solver
    opts = solver.SolveOpts(stages=1, admm_iters=1, lbfgs_iters=iters)
    t0 = time.perf_counter()
    th, z, u, st = solver.admm(prob, th0, opts)
    return time.perf_counter() - t0, th, st


# ---------------------------------------------------------------------------
def spawn_ranks(args):
    """``--gpus N`` without a torchrun environment: start N ranks (one process
    per GPU, 127.0.0.1 rendezvous) and wait for them."""
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    procs = []
    for r in range(args.gpus):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(args.gpus),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, os.path.abspath(__file__)] + sys.argv[1:], env=env))
    rc = 0
    for p in procs:
        rc = p.wait() or rc
    return rc


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16x3", choices=["fp32", "bf16x3"])
    ap.add_argument("--workload", default="precision", choices=["precision", "batched"])
    ap.add_argument("--seed", type=int, default=2412)
    ap.add_argument("--streams", type=int, default=4, help="CUDA streams the frequencies of a step are spread over")
    ap.add_argument("--pass-ctas", type=int, default=-1,
                    help="cap on the CTAs of one fused update-and-pack launch in the timed steps "
                         "and the other multi-stream legs (tlr_mdd_set_pass_ctas; -1: PASS_CTAS_PER_SM per SM with "
                         "more than one stream, else 0 = one per tile)")
    ap.add_argument("--secondary-streams", type=int, default=4, help="streams of the nr=4096 workload's steps")
    ap.add_argument("--e2e-steps", type=int, default=4, help="steps of the end-to-end leg (0: skip)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--oracle-cols", type=int, default=512,
                    help="source columns per step of the reference arm's bounded sample")
    ap.add_argument("--accuracy", type=int, default=4, help="frequencies of the precision table (0: skip)")
    ap.add_argument("--freqs", type=int, default=0,
                    help="frequencies per GPU (0: the workload's); fewer than a batch make one step")
    ap.add_argument("--rank", type=int, default=0, help="one rank for every frequency (profiling runs; 0: the schedule)")
    ap.add_argument("--schedule", type=int, default=0,
                    help="with --freqs n: take every (schedule/n)-th rank of a schedule over this many frequencies "
                         "(a profiling run then sees the ranks of one headline step)")
    ap.add_argument("--serving", type=int, default=120,
                    help="requests of the serving mix (nr 1024-8192, tile 128-512, rank 2-64) served with "
                         "continuous batching (0: skip)")
    ap.add_argument("--serving-fp32-loads", default="",
                    help="comma-separated arrival rates as fractions of the FP32 path's one-at-a-time capacity "
                         "(e.g. 0.7,1.3): the serving mix served on the tensor cores at each, Poisson")
    ap.add_argument("--small-configs", type=int, default=200,
                    help="solves timed for each of the nr=256 and nr=1024 workloads (0: skip)")
    ap.add_argument("--secondary", type=int, default=2,
                    help="timed steps of the nr=4096 batched workload reported beside the headline (0: skip)")
    args = ap.parse_args()

    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(spawn_ranks(args))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    wl = PRECISION_FORM if args.workload == "precision" else BATCHED
    if args.freqs or args.rank:
        import dataclasses
        if args.freqs:
            wl = dataclasses.replace(wl, nfreq=args.freqs, batch=min(wl.batch, args.freqs))
        if args.rank:
            wl = dataclasses.replace(wl, rank_lo=args.rank, rank_hi=args.rank)

    if args.impl == "reference":
        return reference_arm(args, wl, world, rank)

    import torch
    import paper_2412_14973_gb300 as T
    from paper_2412_14973_gb300 import sharding

    os.environ["TLR_MDD_GRAPHS"] = "0" if wl.nr >= 8192 else "1"
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    # with several streams a capped pass grid leaves the contraction CTAs of
    # the other streams their SMs
    multi_ctas = args.pass_ctas if args.pass_ctas >= 0 else PASS_CTAS_PER_SM * sms
    pass_ctas = multi_ctas if args.streams > 1 else (args.pass_ctas if args.pass_ctas >= 0 else 0)
    T.tlr_mdd_set_pass_ctas(pass_ctas)
    total = wl.nfreq * world
    ranks = wl.ranks(total)
    if args.schedule and args.freqs and args.schedule % args.freqs == 0:
        full = wl.ranks(args.schedule * world)
        stride = args.schedule // args.freqs
        ranks = [full[g * stride] for g in range(total)]
    mine = sharding.frequency_plan(wl.nfreq, rank, world)
    steps_of = sharding.batches(mine, wl.batch)
    prec = T.TLR_PREC_FP32 if args.precision == "fp32" else T.TLR_PREC_BF16X3
    t_gen = time.perf_counter()
    inp = Inputs(T, torch, wl, mine, ranks, args.seed, dev)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    runner = Runner(T, torch, inp, max(1, args.streams), dev)
    nstream = len(runner.streams)
    lat_ms, records = [], []

    for w in range(args.warmup):
        runner.step(steps_of[w % len(steps_of)], prec)
    torch.cuda.synchronize()

    def timed_region():
        lat_ms.clear()
        records.clear()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        n0 = T.tlr_mdd_launch_count()
        clk = ClockSampler(local)
        clk.start()
        ms = 0.0
        for s in range(args.steps):
            ms += runner.step(steps_of[s % len(steps_of)], prec, records=records, lat=lat_ms)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        return ms, clk.stop(), T.tlr_mdd_launch_count() - n0

    log(f"inputs generated in {t_gen:.1f} s; warm-up done")
    ms, clocks, launches = timed_region()
    log(f"timed region: {ms:.0f} ms for {args.steps} steps")
    # a timed region that saw a hardware or thermal slowdown, or SM clocks held
    # far below their maximum with no reason given (a clock lock), is measured
    # once more and that second measurement is reported
    bad = clock_problem(clocks)
    if bad:
        ms, clocks, launches = timed_region()
        clocks["remeasured_after"] = bad
        clocks["still_flagged"] = clock_problem(clocks)
    ms = sharding.max_over_ranks(ms, dist, dev)
    solved = [f for s in range(args.steps) for f in steps_of[s % len(steps_of)]]
    solves = len(solved) * world
    value = solves / (ms / 1e3)
    my_flops = sum(flops_per_solve(wl.nr, wl.nr, wl.tile, ranks[f]) for f in solved)
    gathered = sharding.gather_results(records, dist)

    # roofline of the dominant contraction class: one step's frequencies on
    # ONE stream with CUDA events around every contraction launch (no overlap
    # with other launches, so an event pair times that launch alone)
    bf16, hbm, peak_src = measured_peaks()
    names = ["cgemm_compress", "cgemm_expand", "cgemm_project"]
    roof = None
    if rank == 0:
        single = Runner(T, torch, inp, 1, dev)
        T.tlr_mdd_set_pass_ctas(0)   # one stream: a CTA per tile
        T.tlr_mdd_timing_reset()
        T.tlr_mdd_timing_enable(True)
        ms1 = single.step(steps_of[0], prec)
        timing = T.tlr_mdd_timing_read()
        T.tlr_mdd_timing_enable(False)
        T.tlr_mdd_set_pass_ctas(pass_ctas)
        del single
        dom = max(range(len(timing)), key=lambda c: timing[c][0])
        dms, dfl, dnl = timing[dom]
        achieved = dfl / (dms / 1e3) / 1e12
        step_flops = sum(flops_per_solve(wl.nr, wl.nr, wl.tile, ranks[f]) for f in steps_of[0])
        if prec == T.TLR_PREC_FP32:
            peak = 152 * 128 * 2 * 2070e6 / 1e12
            roof = {"bound": "alu", "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz"}
        else:
            # 4M x BF16x3: 12 real BF16 products (24 flops) issued per complex
            # multiply-add counted as 8; the 3M form would issue 9 (18 flops)
            peak = bf16 * 8.0 / 24.0
            roof = {"bound": "tensor",
                    "peak_source": (f"{peak_src} sustained bf16 {bf16} TFLOP/s x 8/24: the issue rate of the "
                                    "4M BF16x3 form this kernel runs (12 BF16 products per complex MAC); "
                                    f"against the 3M-effective peak (x 8/18 = {bf16 * 8 / 18:.1f}) the "
                                    "fraction is frac x 0.75")}
        roof.update({"kernel": names[dom], "achieved": round(achieved, 2), "peak": round(peak, 1),
                     "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                     "traffic": gemm_traffic(names[dom], wl.nr, wl.tile, [ranks[f] for f in steps_of[0]],
                                             args.precision),
                     "traffic_note": ("DRAM read + write bytes per launch of this class, mean over one step's "
                                      "launches, from the ncu capture of these GEMM sources (null when the "
                                      "sources or the step's shapes differ from the capture's)"),
                     "launches": dnl, "ms": round(dms, 2),
                     "flops_counted": "8 per complex MAC; per iteration 56 ns n_LR (T and the residual carried "
                                      "between iterations; a fresh forward each iteration would be 72)",
                     "single_stream_step_ms": round(ms1, 1),
                     "single_stream_step_tflops": round(step_flops / (ms1 / 1e3) / 1e12, 1),
                     "share_of_step": round(dms / ms1, 3),
                     "per_class": {names[c]: {"ms": round(timing[c][0], 1), "launches": timing[c][2],
                                              "tflops": round(timing[c][1] / max(1e-9, timing[c][0] / 1e3) / 1e12,
                                                              1)}
                                   for c in range(len(timing)) if timing[c][2]}})

    log("roofline pass done")
    # e2e through the C ABI with HOST buffers: D, U and the start point copied
    # from pinned host memory inside the timed region, the solved factors read back
    e2e = None
    if args.e2e_steps > 0:
        # the first two batches' D and U in pinned host memory (every batch has
        # the same rank mix); e2e step i solves batch i % 2 from there
        e2e_batches = steps_of[:min(2, len(steps_of))]
        hf = [f for fs in e2e_batches for f in fs]
        Dh = {f: inp.D[inp.slot_of[f]].cpu().pin_memory() for f in hf}
        Uh = {f: inp.U[inp.slot_of[f]].cpu().pin_memory() for f in hf}
        th_h = {f: inp.th0[inp.slot_of[f]].cpu().pin_memory() for f in hf}
        out_h = {f: torch.empty_like(th_h[f]).pin_memory() for f in hf}
        hopts = T.solve_opts(theta_memory=T.TLR_MEM_HOST)
        host = (Dh, Uh, th_h, out_h, hopts)
        runner.step(e2e_batches[0], prec, host=host)          # warm-up
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        n_e2e = h2d = d2h = 0
        for i in range(args.e2e_steps):
            fs = e2e_batches[i % len(e2e_batches)]
            runner.step(fs, prec, host=host)
            n_e2e += len(fs)
            h2d += sum(Dh[f].numel() * 8 + Uh[f].numel() * 8 + th_h[f].numel() * 8 for f in fs)
            d2h += sum(out_h[f].numel() * 8 for f in fs)
        torch.cuda.synchronize()
        te = sharding.max_over_ranks(time.perf_counter() - t0, dist, dev)
        e2e = {"value": round(n_e2e * world / te, 4), "unit": "freq-solves/s",
               "h2d_bytes_per_step": h2d // args.e2e_steps, "d2h_bytes_per_step": d2h // args.e2e_steps,
               "steps": args.e2e_steps,
               "host_data": f"D, U and theta0 of {len(hf)} frequencies (two batches) in pinned host memory; "
                            "every step copies its batch's inputs in and its solved factors out"}
        del Dh, Uh, th_h, out_h, host

    # precision table: on frequencies spread over the rank range, the error
    # of one operator application (seeded theta0) against the FP64 oracle on
    # sampled source columns, for both paths, and 30-iteration solves on both
    # paths (time, and the difference of their X and final misfit)
    log("e2e leg done")
    # the legs below run one solve at a time (or their own streams): a CTA per tile
    T.tlr_mdd_set_pass_ctas(0)
    acc = None
    cmp = None
    if rank == 0 and args.accuracy > 0:
        acc, cmp = precision_table(T, torch, inp, wl, mine, args, dev)

    # CPU oracle baseline: one full L-BFGS iteration (the solve's first forward
    # product and gradient, the line-search products, the gradient at the new
    # point) of the FP64 oracle at the mean rank, on the host cores, and the
    # same iteration on the GPU for the error of X and f
    log("precision table done")
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu, solve_acc = cpu_leg(T, torch, inp, wl, mine, ranks, dev)
        if acc is not None:
            acc["oracle_solve"] = solve_acc

    log("cpu leg done")
    secondary = None
    if rank == 0 and args.secondary > 0 and wl.nr == PRECISION_FORM.nr:
        del runner, inp
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        T.tlr_mdd_trim_pool(0)
        T.tlr_mdd_set_pass_ctas(multi_ctas)       # several streams
        secondary = secondary_leg(T, torch, args, dev)
        T.tlr_mdd_set_pass_ctas(0)

    peaks = measure_peaks(torch, dev) if rank == 0 else None
    small = None
    if rank == 0 and args.small_configs > 0:
        small = small_configs_leg(T, torch, args.small_configs, args.seed, dev, cpu=not args.no_cpu)
        log("small workloads done")

    serve = None
    if rank == 0 and args.serving > 0:
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        T.tlr_mdd_trim_pool(0)
        loads = [float(x) for x in args.serving_fp32_loads.split(",") if x.strip()]
        # the server's slots run the passes uncapped: with one CTA per SM the
        # served rate fell (9.9 against 11.5 solves/s at the same arrivals)
        serve = serving_leg(T, torch, args.serving, args.seed, dev, loads, 0)
        log("serving leg done")

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    line = {
        "metric": "freq-solves/s", "value": round(value, 4), "unit": "freq-solves/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms / args.steps, 2), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if prec == T.TLR_PREC_FP32 else "bf16x3",
        "data": "synthetic",
        "config": {"workload": wl.name, "nr": wl.nr, "ns": wl.nr, "grid": list(wl.grid),
                   "frequencies_per_gpu": wl.nfreq, "frequencies_per_step": wl.batch,
                   "tile": wl.tile, "ranks": f"{wl.rank_lo}->{wl.rank_hi} linear",
                   "iters_per_solve": ITERS_PER_SOLVE, "precision": args.precision, "streams": nstream,
                   "pass_ctas": pass_ctas, "pass_ctas_other_multi_stream_legs": multi_ctas,
                   "step": "one batch of frequencies (every nfreq/batch-th), each solved from its raw D, U "
                           "through a handle created for it (data step, packing, solve)",
                   "l2": "inputs larger than L2 (each 9216x9216 complex64 panel is 679 MB; every step reads "
                         "8 frequencies' D and U, 10.9 GB)" if wl.nr == PRECISION_FORM.nr else
                         "inputs larger than L2 (134 MB panels)",
                   "parallelism": f"frequency sharding x{world}", "launches": "plain (no CUDA graph) at nr >= 8192",
                   "generation_s": round(t_gen, 1)},
        "gflops": round(my_flops * world / (ms / 1e3) / 1e9, 1),
        "latency_ms": {"p50": percentile(lat_ms, 50), "p99": percentile(lat_ms, 99)},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
        "gpu_launches": launches, "accuracy": acc, "fp32_comparison": cmp,
        "results": {"frequencies": len(gathered or []), "ranks_gathered": world,
                    "all_ok": all(r["status"] == 0 and r["iters"] == ITERS_PER_SOLVE for r in gathered or []),
                    "f_final_over_f0_median": statistics.median(r["f_final"] / r["f0"] for r in gathered)
                    if gathered else None},
    }
    if secondary is not None:
        line["secondary"] = secondary
    if serve is not None:
        line["serving"] = serve
    if peaks is not None:
        line["peaks_measured"] = peaks
    if small is not None:
        line["small_workloads"] = small
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def precision_table(T, torch, inp, wl, mine, args, dev):
    """Per frequency: relative error of Y = X_h Dfrak and of the column misfit
    at the seeded start point against the FP64 oracle (sampled source columns,
    both paths), and 30-iteration solves on both paths from that start point:
    the relative difference of their X and final misfit, and their times."""
    from oracle import tlr
    import tlr_synth as synth
    pick = sorted({mine[int(round(i * (len(mine) - 1) / max(1, args.accuracy - 1)))]
                   for i in range(args.accuracy)})
    rows = []
    t_path = {"bf16x3": 0.0, "tf32": 0.0, "fp32": 0.0}
    st = torch.cuda.current_stream(dev)
    for f in pick:
        sl = inp.slot_of[f]
        k = inp.ranks[f]
        D0 = inp.D[sl].cpu().numpy()
        U0 = inp.U[sl].cpu().numpy()
        cols = np.sort(synth.rng(f + 1).choice(wl.nr, 32, replace=False))
        prob, lay, alpha = oracle_problem(D0, U0, wl, k, cols=cols)
        th0 = inp.th0[sl]
        th0n = th0.cpu().numpy().astype(np.complex128)
        Yo = tlr.apply(th0n, lay, prob.Dt)
        Ro = Yo - prob.Ut
        fo = 0.5 * float(np.vdot(Ro, Ro).real)
        row = {"freq": f, "rank": k}
        X = {}
        for name, p in (("bf16x3", T.TLR_PREC_BF16X3), ("tf32", T.TLR_PREC_TF32), ("fp32", T.TLR_PREC_FP32)):
            d = inp.desc(T, f, p)
            d.alpha = alpha
            h = T.tlr_mdd_create(d, inp.D[sl], inp.U[sl], st)
            Y = torch.empty((wl.nr, wl.nr), dtype=torch.complex64, device=dev)
            T.tlr_mdd_apply(h, th0, Y)
            Yc = Y[:, torch.from_numpy(cols).to(dev)].cpu().numpy().astype(np.complex128)
            del Y
            Rc = Yc - prob.Ut
            fc = 0.5 * float(np.vdot(Rc, Rc).real)
            row[f"apply_rel_err_{name}"] = float(np.linalg.norm(Yc - Yo) / np.linalg.norm(Yo))
            row[f"column_misfit_rel_err_{name}"] = abs(fc - fo) / fo
            th = th0.clone()
            torch.cuda.synchronize()
            s = T.tlr_mdd_solve(h, th, T.solve_opts())
            row[f"solve_ms_{name}"] = round(s.gpu_ms, 1)
            row[f"f_final_{name}"] = s.f_hist[s.n_hist - 1]
            t_path[name] += s.gpu_ms
            Xd = torch.empty((wl.nr, wl.nr), dtype=torch.complex64, device=dev)
            T.tlr_mdd_unpermute_dense(h, th, Xd)
            X[name] = Xd
            T.tlr_mdd_destroy(h)
        for name in ("bf16x3", "tf32"):
            sfx = "tc" if name == "bf16x3" else name
            row[f"solve_X_rel_diff_{sfx}_vs_fp32"] = float((X[name] - X["fp32"]).norm() / X["fp32"].norm())
            row[f"solve_misfit_rel_diff_{sfx}_vs_fp32"] = abs(row[f"f_final_{name}"] - row["f_final_fp32"]) / \
                row["f_final_fp32"]
        del X
        rows.append(row)
    worst = lambda key: max(r[key] for r in rows)  # noqa: E731
    acc = {"per_frequency": rows,
           "bounds": "per application: 1e-5 (FP32), 1e-3 (tensor cores) relative; final X: 1e-3",
           "worst_apply_rel_err_bf16x3": worst("apply_rel_err_bf16x3"),
           "worst_apply_rel_err_tf32": worst("apply_rel_err_tf32"),
           "worst_apply_rel_err_fp32": worst("apply_rel_err_fp32"),
           "worst_solve_X_rel_diff_tc_vs_fp32": worst("solve_X_rel_diff_tc_vs_fp32"),
           "worst_solve_X_rel_diff_tf32_vs_fp32": worst("solve_X_rel_diff_tf32_vs_fp32"),
           "within_bounds": worst("apply_rel_err_bf16x3") <= 1e-3 and worst("apply_rel_err_fp32") <= 1e-5
           and worst("solve_X_rel_diff_tc_vs_fp32") <= 1e-3,
           "tf32_within_bounds": worst("apply_rel_err_tf32") <= 1e-3 and worst("solve_X_rel_diff_tf32_vs_fp32") <= 1e-3,
           "sample": "32 seeded source columns per frequency for the oracle (its work is per column)"}
    rate = {k: round(len(pick) / (v / 1e3), 4) for k, v in t_path.items()}
    cmp = {"frequencies": pick, "fp32_simt_freq_solves_per_s": rate["fp32"],
           "tensor_core_freq_solves_per_s": rate["bf16x3"], "tf32_freq_solves_per_s": rate["tf32"],
           "speedup_tc_vs_fp32": round(t_path["fp32"] / t_path["bf16x3"], 3),
           "speedup_tf32_vs_fp32": round(t_path["fp32"] / t_path["tf32"], 3),
           "accuracy": {"worst_apply_rel_err_fp32": acc["worst_apply_rel_err_fp32"],
                        "worst_apply_rel_err_bf16x3": acc["worst_apply_rel_err_bf16x3"],
                        "worst_apply_rel_err_tf32": acc["worst_apply_rel_err_tf32"],
                        "worst_solve_X_rel_diff": acc["worst_solve_X_rel_diff_tc_vs_fp32"],
                        "worst_solve_X_rel_diff_tf32": acc["worst_solve_X_rel_diff_tf32_vs_fp32"]},
           "note": "one solve at a time on one stream, device time; equal accuracy: both within the bounds"}
    return acc, cmp


def cpu_leg(T, torch, inp, wl, mine, ranks, dev):
    """One full L-BFGS iteration of the FP64 oracle at the frequency nearest
    the mean rank, timed on the host cores and scaled to a 30-iteration solve
    (every iteration does the same work); the same iteration on the GPU gives
    the relative error of X and of f against the oracle."""
    from oracle import operator
    kmean = sum(ranks[f] for f in mine) / len(mine)
    f = min(mine, key=lambda x: (abs(ranks[x] - kmean), x))
    sl = inp.slot_of[f]
    k = ranks[f]
    D0 = inp.D[sl].cpu().numpy()
    U0 = inp.U[sl].cpu().numpy()
    prob, lay, alpha = oracle_problem(D0, U0, wl, k)
    del D0, U0
    th0 = inp.th0[sl].cpu().numpy().astype(np.complex128)
    # the oracle's own first forward product and gradient are timed apart from
    # the iteration (line-search products + gradient at the new point), so the
    # 30-iteration figure is first + 30 x iteration, both measured
    calls = []
    fgrad = prob.fgrad

    def timed_fgrad(theta):
        t0 = time.perf_counter()
        r = fgrad(theta)
        calls.append(time.perf_counter() - t0)
        return r

    prob.fgrad = timed_fgrad
    secs, th_or, st_or = run_oracle_solve(prob, th0, 1)
    t_first = calls[0]
    t_iter = secs - t_first
    per_solve = t_first + ITERS_PER_SOLVE * t_iter
    cpu = {"value": round(1.0 / per_solve, 7), "unit": "freq-solves/s", "cores": blas_threads(),
           "kind": "oracle",
           "sample": (f"frequency {f} (rank {k}, the mean rank {kmean:.1f}): one full L-BFGS iteration of the "
                      f"FP64 TLR-structured oracle in {secs:.1f} s (first forward product and gradient "
                      f"{t_first:.1f} s, then the iteration {t_iter:.1f} s: line-search products and the "
                      f"gradient at the new point); a {ITERS_PER_SOLVE}-iteration solve = first + "
                      f"{ITERS_PER_SOLVE} x iteration = {per_solve:.0f} s")}
    d = inp.desc(T, f, T.TLR_PREC_BF16X3)
    d.alpha = alpha
    h = T.tlr_mdd_create(d, inp.D[sl], inp.U[sl], torch.cuda.current_stream(dev))
    thg = inp.th0[sl].clone()
    sg = T.tlr_mdd_solve(h, thg, T.solve_opts(stages=1, admm_iters=1, lbfgs_iters=1))
    T.tlr_mdd_destroy(h)
    Xo = operator.assemble_xh(th_or, lay)
    Xg = operator.assemble_xh(thg.cpu().numpy().astype(np.complex128), lay)
    acc = {"frequency": f, "rank": k, "iters": 1, "path": "bf16x3",
           "rel_err_X_vs_fp64_oracle": float(np.linalg.norm(Xg - Xo) / np.linalg.norm(Xo)),
           "rel_err_f_vs_fp64_oracle": abs(sg.f_hist[0] - st_or.f_hist[0]) / st_or.f_hist[0]}
    return cpu, acc


def secondary_leg(T, torch, args, dev):
    """The nr = 4096 batched workload (64 frequencies, rank 4 -> 48), reported
    beside the headline: one handle per frequency kept across steps (its solve
    recorded once as a CUDA graph), every step re-running each frequency's data
    step and solve on 4 streams."""
    os.environ["TLR_MDD_GRAPHS"] = "1"
    wl = BATCHED
    ranks = wl.ranks(wl.nfreq)
    freqs = list(range(wl.nfreq))
    inp = Inputs(T, torch, wl, freqs, ranks, args.seed + 1, dev)
    nst = max(1, args.secondary_streams)
    streams = [torch.cuda.Stream(device=dev) for _ in range(nst)]
    main = torch.cuda.current_stream(dev)
    hs = [T.tlr_mdd_create(inp.desc(T, f, T.TLR_PREC_BF16X3), inp.D[f], inp.U[f], streams[f % nst]) for f in freqs]
    theta = [t.clone() for t in inp.th0]
    opts = T.solve_opts()

    def step(hs=hs, fs=freqs):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(main)
        for s_ in streams:
            s_.wait_event(e0)
        for f in fs:
            T.tlr_mdd_set_data(hs[f], inp.D[f], inp.U[f], T.TLR_MEM_DEVICE)
            with torch.cuda.stream(streams[f % nst]):
                theta[f].copy_(inp.th0[f])
            T.tlr_mdd_solve_async(hs[f], theta[f], opts)
        for f in fs:
            T.tlr_mdd_solve_wait(hs[f])
        for s_ in streams:
            ev = torch.cuda.Event()
            ev.record(s_)
            main.wait_event(ev)
        e1.record(main)
        e1.synchronize()
        return e0.elapsed_time(e1)

    step()          # plain launches (a handle's first solve)
    step()          # records the solve graphs
    ms = sum(step() for _ in range(args.secondary))
    # the same step on every 8th frequency, tensor cores and the FP32 SIMT
    # path, on handles of their own (8 solves on the streams overlap little:
    # the pass grid is left uncapped; a recorded graph keeps the grid it was
    # recorded with)
    sub = freqs[::8]
    prev_cap = T.tlr_mdd_set_pass_ctas(0)
    hs_sub = {}
    for prec in (T.TLR_PREC_BF16X3, T.TLR_PREC_FP32):
        hs_sub[prec] = {f: T.tlr_mdd_create(inp.desc(T, f, prec), inp.D[f], inp.U[f], streams[f % nst]) for f in sub}
        step(hs_sub[prec], sub)     # plain launches
        step(hs_sub[prec], sub)     # records the graphs
    ms_tc_sub = step(hs_sub[T.TLR_PREC_BF16X3], sub)
    ms_fp32_sub = step(hs_sub[T.TLR_PREC_FP32], sub)
    T.tlr_mdd_set_pass_ctas(prev_cap)
    for h in list(hs) + [h for d in hs_sub.values() for h in d.values()]:
        T.tlr_mdd_destroy(h)
    fl = sum(flops_per_solve(wl.nr, wl.nr, wl.tile, k) for k in ranks) * args.secondary
    oracle_cpu = None
    if not args.no_cpu:
        kmean = sum(ranks) / len(ranks)
        f = min(freqs, key=lambda x: (abs(ranks[x] - kmean), x))
        prob, _, _ = oracle_problem(inp.D[f].cpu().numpy(), inp.U[f].cpu().numpy(), wl, ranks[f])
        per_solve, secs, t_first, t_iter = oracle_solve_rate(prob, inp.th0[f].cpu().numpy().astype(np.complex128))
        oracle_cpu = {"value": round(1.0 / per_solve, 6), "unit": "freq-solves/s", "cores": blas_threads(),
                      "kind": "oracle",
                      "sample": (f"frequency {f} (rank {ranks[f]}, the mean rank {kmean:.1f}): one full L-BFGS "
                                 f"iteration of the FP64 oracle in {secs:.1f} s (first forward product and "
                                 f"gradient {t_first:.1f} s, the iteration {t_iter:.1f} s); a "
                                 f"{ITERS_PER_SOLVE}-iteration solve = {per_solve:.0f} s")}

    def one_solve(d, seed_):
        # one timed solve (device time) of frequency 0's data in a given form
        h = T.tlr_mdd_create(d, inp.D[0], inp.U[0], streams[0])
        gen = torch.Generator(device=dev).manual_seed(seed_)
        nth = T.tlr_mdd_theta_size(d)
        th0 = 0.01 * torch.randn(nth, dtype=torch.complex64, device=dev, generator=gen)
        th = th0.clone()
        torch.cuda.synchronize()
        T.tlr_mdd_solve(h, th, opts)
        th.copy_(th0)
        torch.cuda.synchronize()
        st = T.tlr_mdd_solve(h, th, opts)
        T.tlr_mdd_destroy(h)
        return st, nth

    kx = 26
    common = dict(rank=kx, nx=wl.grid[0], ny=wl.grid[1], diag_mode=T.TLR_DIAG_RULE, precision=T.TLR_PREC_BF16X3)
    prev_cap = T.tlr_mdd_set_pass_ctas(0)   # one solve on one stream: a CTA per tile
    gst, gn = one_solve(T.desc(wl.nr, wl.nr, wl.tile, reciprocity=T.TLR_RECIP_NONE, **common), args.seed + 5)
    tst, tn = one_solve(T.desc(wl.nr, wl.nr, 0, tiles=[192, 320] * 8, **common), args.seed + 6)
    ust, un = one_solve(T.desc(wl.nr, wl.nr, wl.nr // 16, **common), args.seed + 6)
    warm = warm_start_stage(T, torch, inp, wl, ranks, dev)
    T.tlr_mdd_set_pass_ctas(prev_cap)
    f_eq = flops_per_solve(wl.nr, wl.nr, wl.tile, kx)
    return {"workload": wl.name, "value": round(wl.nfreq * args.secondary / (ms / 1e3), 3),
            "unit": "freq-solves/s", "ms_per_step": round(ms / args.secondary, 1), "steps": args.secondary,
            "tflops": round(fl / (ms / 1e3) / 1e12, 1), "streams": nst,
            "step": "all 64 frequencies; handles kept across steps, data step and CUDA-graph solve per frequency",
            "fp32_comparison": {"frequencies": sub, "fp32_simt_freq_solves_per_s":
                                round(len(sub) / (ms_fp32_sub / 1e3), 3),
                                "tensor_core_freq_solves_per_s": round(len(sub) / (ms_tc_sub / 1e3), 3),
                                "speedup_tc_vs_fp32": round(ms_fp32_sub / ms_tc_sub, 2),
                                "note": f"one step over every 8th frequency (the same rank mix), {nst} streams"},
            "cpu_oracle": oracle_cpu,
            "general_form": {"rank": kx, "n_theta": gn, "ms": round(gst.gpu_ms, 2),
                             "tflops": round(f_eq / (gst.gpu_ms / 1e3) / 1e12, 1),
                             "note": "one solve, one stream; the same contraction flops as the reciprocal form"},
            "warm_start_stage": warm,
            "nonuniform_tiles": {"tiles": "192,320 alternating x8", "rank": kx, "n_theta": tn,
                                 "ms": round(tst.gpu_ms, 2), "equal_tiles_ms": round(ust.gpu_ms, 2),
                                 "note": "one solve, one stream; 16 equal tiles of 256 at the same rank "
                                         "(the same flops) beside it"}}


def warm_start_stage(T, torch, inp, wl, ranks, dev):
    """The paper's warm-start stage on the frequency of mean rank: the
    benchmark solver of eq. (4) (20 CG iterations, lambda = 1e-2), the tile
    rank rule on its solution (tile 256, eps = 0.01) and the tile-size choice
    among 128 / 256 / 512, the SVD / Takagi warm start of the handle's
    factors, then the 30-iteration solve from it beside the solve from the
    seeded start.  Every call synchronises; wall times on the host."""
    kmean = sum(ranks) / len(ranks)
    f = min(range(len(ranks)), key=lambda x: (abs(ranks[x] - kmean), x))
    nr = wl.nr
    h = T.tlr_mdd_create(inp.desc(T, f, T.TLR_PREC_BF16X3), inp.D[f], inp.U[f], torch.cuda.current_stream(dev))
    X = torch.empty((nr, nr), dtype=torch.complex64, device=dev)
    iters = 20
    T.tlr_mdd_benchmark_solve(h, 1e-2, 2, 0.0, X)        # warm-up (operand packs, workspace)
    bst = T.tlr_mdd_benchmark_solve(h, 1e-2, iters, 0.0, X)
    flops = 8.0 * nr ** 3 * iters + 2 * 8.0 * nr ** 3    # CG products, then D^H D and D^H U (ns = nr)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rk, entries, v0 = T.tlr_mdd_tile_ranks(X, nr, 256, 0.01)
    t_ranks = time.perf_counter() - t0
    t0 = time.perf_counter()
    b_best, e_best = T.tlr_mdd_choose_tile(X, nr, [128, 256, 512], 0.01)
    t_choose = time.perf_counter() - t0
    nth = T.tlr_mdd_theta_size(inp.desc(T, f, T.TLR_PREC_BF16X3))
    th_w = torch.empty(nth, dtype=torch.complex64, device=dev)
    t0 = time.perf_counter()
    T.tlr_mdd_warm_start(h, X, th_w)
    t_warm = time.perf_counter() - t0
    opts = T.solve_opts()
    sw = T.tlr_mdd_solve(h, th_w, opts)
    th_c = inp.th0[f].clone()
    sc = T.tlr_mdd_solve(h, th_c, opts)
    T.tlr_mdd_destroy(h)
    return {"frequency": f, "rank": ranks[f],
            "benchmark_solver": {"iterations": bst.iters, "rel_res": bst.rel_res, "ms": round(bst.gpu_ms, 2),
                                 "tflops": round(flops / (bst.gpu_ms / 1e3) / 1e12, 1),
                                 "flops_counted": "8 per complex MAC: one nr^3 product per CG iteration, "
                                                  "plus D^H D and D^H U"},
            "tile_ranks_b256": {"ms": round(1e3 * t_ranks, 1), "mean_rank": round(sum(rk) / len(rk), 2),
                                "entry_ratio": round(nr * nr / max(1, entries), 2)},
            "choose_tile": {"candidates": [128, 256, 512], "chosen": b_best,
                            "entry_ratio": round(nr * nr / max(1, e_best), 2), "ms": round(1e3 * t_choose, 1)},
            "warm_start_ms": round(1e3 * t_warm, 1),
            "solve_from_warm_start": {"f0": sw.f0, "f_final": sw.f_hist[sw.n_hist - 1], "ms": round(sw.gpu_ms, 2)},
            "solve_from_seeded_start": {"f0": sc.f0, "f_final": sc.f_hist[sc.n_hist - 1], "ms": round(sc.gpu_ms, 2)},
            "note": "benchmark solution at lambda = 1e-2 after 20 CG iterations (not converged): the warm start "
                    "is what the paper's pipeline starts from; every step here runs on the GPU"}


def serving_leg(T, torch, n, seed, dev, fp32_loads=(), multi_ctas=0):
    """The serving mix: n per-frequency solve requests, nr = ns uniform over
    {1024, 2048, 4096, 8192}, tile over {128, 256, 512}, rank log-uniform
    2-64, BF16x3 tensor cores, 30-iteration solves.  Measured: one request at
    a time on the tensor cores (all n) and on the FP32 SIMT path (the first
    m of them), then the whole stream served with continuous batching (4
    slots, 120 GB budget, shape-keyed handle reuse) at Poisson arrivals of 90%
    of the tensor cores' one-at-a-time capacity: solves/s, p50 / p99 latency
    from arrival to result, and whether every served result equals its
    one-at-a-time result bit for bit.  One seeded D, U per size is shared by
    the requests of that size (the work does not depend on the values)."""
    import tlr_synth as synth
    from paper_2412_14973_gb300 import serving
    reqs = synth.request_stream(n, 1.0, seed + 17)
    g = torch.Generator(device=dev).manual_seed(seed + 18)
    pool = {}
    for r in reqs:
        if r.nr not in pool:
            mats = []
            for _ in range(2):
                re = torch.randn((r.nr, r.nr), generator=g, device=dev)
                im = torch.randn((r.nr, r.nr), generator=g, device=dev)
                mats.append((torch.complex(re, im) / math.sqrt(2 * r.nr)).to(torch.complex64))
            pool[r.nr] = tuple(mats)

    def make(prec, arrivals, subset=None):
        out = []
        for r, t in zip(reqs[:subset], arrivals):
            d = T.desc(r.nr, r.nr, r.tile, rank=r.rank, nx=r.nx, ny=r.ny, diag_mode=T.TLR_DIAG_RULE,
                       precision=prec)
            nth = T.tlr_mdd_theta_size(d)
            gg = torch.Generator(device=dev).manual_seed(r.seed)
            th = (torch.randn(nth, generator=gg, device=dev) + 1j * torch.randn(nth, generator=gg, device=dev))
            th = (th * (0.1 / math.sqrt(r.tile * max(1, r.rank)))).to(torch.complex64)
            out.append(serving.SolveRequest(r.rid, t, d, pool[r.nr][0], pool[r.nr][1], th, T.solve_opts()))
        return out

    budget = 120 << 30
    m = min(n, 24)
    zero = [0.0] * n
    s1 = serving.Server(budget, max_active=1, reuse=False)
    t0 = time.perf_counter()
    res_fp32 = s1.run(make(T.TLR_PREC_FP32, zero, m), realtime=False)
    t_fp32 = time.perf_counter() - t0
    t0 = time.perf_counter()
    res_tc1 = s1.run(make(T.TLR_PREC_BF16X3, zero), realtime=False)
    t_tc1 = time.perf_counter() - t0
    t_tc1_m = sum(r.finished - r.admitted for r in res_tc1[:m])
    rate = 0.9 * n / t_tc1
    arrivals = list(np.cumsum(np.random.default_rng(seed + 19).exponential(1.0 / rate, n)))
    # served: several slots share the GPU, so the pass grid is capped (the
    # one-at-a-time runs above use one CTA per tile)
    T.tlr_mdd_set_pass_ctas(multi_ctas)
    srv = serving.Server(budget, max_active=4)
    t0 = time.perf_counter()
    res = srv.run(make(T.TLR_PREC_BF16X3, arrivals), realtime=True)
    t_srv = time.perf_counter() - t0
    ok = [r for r in res if r.status == 0]
    pc = serving.percentiles(res)
    svc = [1e3 * (r.finished - r.admitted) for r in ok]   # admission to result: the solve without queueing
    same = all(a.status == 0 and b.status == 0 and torch.equal(a.theta, b.theta) for a, b in zip(res_tc1, res))
    srv.close()
    # the same stream with lockstep batches of up to 4 same-size requests per slot
    srvb = serving.Server(budget, max_active=4, batch_max=4)
    t0 = time.perf_counter()
    resb = srvb.run(make(T.TLR_PREC_BF16X3, arrivals), realtime=True)
    t_b = time.perf_counter() - t0
    pcb = serving.percentiles(resb)
    sameb = all(a.status == 0 and b.status == 0 and torch.equal(a.theta, b.theta) for a, b in zip(res_tc1, resb))
    srvb.close()
    # and with batch partners of any size
    srvm = serving.Server(budget, max_active=4, batch_max=4, mix_sizes=True)
    t0 = time.perf_counter()
    resm = srvm.run(make(T.TLR_PREC_BF16X3, arrivals), realtime=True)
    t_m = time.perf_counter() - t0
    pcm = serving.percentiles(resm)
    samem = all(a.status == 0 and b.status == 0 and torch.equal(a.theta, b.theta) for a, b in zip(res_tc1, resm))
    srvm.close()
    batched = {"tc_served_solves_per_s": round(sum(1 for r in resb if r.status == 0) / t_b, 3),
               "p50_ms": round(1e3 * pcb[50], 1) if pcb[50] else None,
               "p99_ms": round(1e3 * pcb[99], 1) if pcb[99] else None,
               "batches": srvb.batches, "results_identical_alone_and_in_batches": bool(sameb),
               "note": "same arrivals; requests of one size admitted together share one launch per contraction",
               "any_size": {"tc_served_solves_per_s": round(sum(1 for r in resm if r.status == 0) / t_m, 3),
                            "p50_ms": round(1e3 * pcm[50], 1) if pcm[50] else None,
                            "p99_ms": round(1e3 * pcm[99], 1) if pcm[99] else None,
                            "batches": srvm.batches, "results_identical_alone_and_in_batches": bool(samem)}}
    # the stream at loads relative to the FP32 path's one-at-a-time capacity
    # (a load above 1 is one the FP32 path alone cannot carry)
    at_fp32_loads = []
    for li, load in enumerate(fp32_loads):
        rate_l = load * m / t_fp32
        arr = list(np.cumsum(np.random.default_rng(seed + 23 + li).exponential(1.0 / rate_l, n)))
        srvl = serving.Server(budget, max_active=4)
        t0 = time.perf_counter()
        resl = srvl.run(make(T.TLR_PREC_BF16X3, arr), realtime=True)
        t_l = time.perf_counter() - t0
        pcl = serving.percentiles(resl)
        okl = [r for r in resl if r.status == 0]
        svl = [1e3 * (r.finished - r.admitted) for r in okl]
        samel = all(a.status == 0 and b.status == 0 and torch.equal(a.theta, b.theta)
                    for a, b in zip(res_tc1, resl))
        srvl.close()
        at_fp32_loads.append({"load_of_fp32_capacity": load, "arrival_rate_hz": round(rate_l, 3),
                              "tc_served_solves_per_s": round(len(okl) / t_l, 3),
                              "p50_ms": round(1e3 * pcl[50], 1) if pcl[50] else None,
                              "p99_ms": round(1e3 * pcl[99], 1) if pcl[99] else None,
                              "service_p50_ms": round(percentile(svl, 50), 1) if svl else None,
                              "service_p99_ms": round(percentile(svl, 99), 1) if svl else None,
                              "results_identical_alone_and_in_mix": bool(samel)})
    T.tlr_mdd_set_pass_ctas(0)
    sizes = collections_counter(r.nr for r in reqs)
    return {"requests": n, "completed": len(ok), "arrival_rate_hz": round(rate, 3),
            "pass_ctas_served": multi_ctas,
            "tc_served_solves_per_s": round(len(ok) / t_srv, 3),
            "p50_ms": round(1e3 * pc[50], 1) if pc[50] else None,
            "p99_ms": round(1e3 * pc[99], 1) if pc[99] else None,
            "service_p50_ms": round(percentile(svc, 50), 1) if svc else None,
            "service_p99_ms": round(percentile(svc, 99), 1) if svc else None,
            "tc_one_at_a_time_solves_per_s": round(n / t_tc1, 3),
            "fp32_one_at_a_time_solves_per_s": round(m / t_fp32, 3),
            "tc_one_at_a_time_solves_per_s_same_subset": round(m / t_tc1_m, 3),
            "speedup_tc_vs_fp32_one_at_a_time": round(t_fp32 / t_tc1_m, 2),
            "fp32_subset": m,
            "peak_active": srv.peak_active, "peak_budget_gb": round(srv.peak_used / 2**30, 1),
            "handles_created": srv.created, "handles_reused": srv.reused, "handles_evicted": srv.evicted,
            "results_identical_alone_and_in_mix": bool(same),
            "lockstep_batches": batched,
            "at_fp32_loads": at_fp32_loads,
            "sizes": dict(sorted(sizes.items())),
            "mix": "nr=ns in {1024,2048,4096,8192}, tile in {128,256,512}, rank log-uniform 2-64, Poisson; "
                   "latency = arrival to result on the host clock (queueing included), service = admission to "
                   "result"}


def measure_peaks(torch, dev):
    """FP32 (CUDA cores), TF32 and BF16 (tensor cores) and FP64 matrix-multiply
    rates of this GPU, measured like the driver's peaks: torch.matmul (cuBLAS)
    on square operands, CUDA events, best of several."""
    out = {}
    tf32 = torch.backends.cuda.matmul.allow_tf32
    try:
        for name, dt, n, allow, reps in (("fp32_simt", torch.float32, 8192, False, 3),
                                        ("tf32_tensor", torch.float32, 8192, True, 5),
                                        ("bf16_tensor", torch.bfloat16, 8192, False, 5),
                                        ("fp64", torch.float64, 4096, False, 3)):
            torch.backends.cuda.matmul.allow_tf32 = allow
            a = torch.randn((n, n), device=dev, dtype=dt)
            b = torch.randn((n, n), device=dev, dtype=dt)
            torch.matmul(a, b)
            best = 1e30
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1))
            out[name + "_tflops"] = round(2.0 * n ** 3 / (best / 1e3) / 1e12, 2)
            del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = tf32
    out["method"] = "torch.matmul (cuBLAS), n = 8192 (FP64: 4096), 2 n^3 flops, best of 3-5, CUDA events"
    return out


def small_configs_leg(T, torch, n, seed, dev, cpu=True):
    """The two small workloads, solve by solve (CUDA-graph replays on one
    stream, device time per solve, p50 / p99 over n solves), on both paths:
    the plain method on one frequency (nr = ns = 256, 16 x 16 grid, tile 64,
    rank 8, dense diagonal tiles, 20 dB, 30 iterations: latency bound), and
    the differentiation form's sparse solve (nr = 1024, 32 x 32 grid, tile 128,
    rank 12, low-rank diagonals, 717 of 1024 sources kept, 5 dB, 16
    frequencies cycled)."""
    import tlr_synth as synth
    out = {}
    stream = torch.cuda.Stream(device=dev)
    for name, nx, b, k, mode, snr, nfreq, keep in (
            ("plain_nr256", 16, 64, 8, T.TLR_DIAG_DENSE, 20.0, 1, None),
            ("sparse_nr1024", 32, 128, 12, T.TLR_DIAG_LOWRANK, 5.0, 16, 717)):
        nr = nx * nx
        g = torch.Generator(device=dev).manual_seed(seed + nr)
        hg = synth.rng(seed + nr)
        Q = phase_dft_unitary_device(torch, nr, hg, dev)
        W = phase_dft_unitary_device(torch, nr, hg, dev)
        sig = torch.pow(10.0, -3.0 * torch.arange(nr, device=dev, dtype=torch.float32) / (nr - 1))
        rows = torch.arange(nr, device=dev) if keep is None else \
            torch.from_numpy(synth.source_keep(nr, keep / nr, seed + 5)).to(dev)
        data = []
        for f in range(nfreq):
            ph = torch.exp(2j * math.pi * torch.rand(nr, generator=g, device=dev)).to(torch.complex64)
            D = ((Q * (sig * ph)[None, :]) @ W.conj().T)[rows].contiguous()
            X = torch.complex(torch.randn((nr, nr), generator=g, device=dev),
                              torch.randn((nr, nr), generator=g, device=dev)) / math.sqrt(2 * nr)
            X = ((X + X.T) * 0.5).to(torch.complex64)
            Y = D @ X
            nz = torch.complex(torch.randn(Y.shape, generator=g, device=dev), torch.randn(Y.shape, generator=g,
                                                                                             device=dev))
            U = (Y + nz * (Y.norm() / nz.norm() * 10 ** (-snr / 20))).to(torch.complex64)
            data.append((D, U))
        res = {}
        for pname, prec in (("bf16x3", T.TLR_PREC_BF16X3), ("fp32", T.TLR_PREC_FP32)):
            d = T.desc(nr, rows.numel(), b, rank=k, nx=nx, ny=nx, diag_mode=mode, precision=prec)
            h = T.tlr_mdd_create(d, data[0][0], data[0][1], stream)
            nth = T.tlr_mdd_theta_size(d)
            th0 = (torch.randn(nth, generator=g, device=dev) * (0.1 / math.sqrt(b * k))).to(torch.complex64)
            th = th0.clone()
            opts = T.solve_opts()
            T.tlr_mdd_solve(h, th, opts)            # plain launches (the handle's first solve)
            T.tlr_mdd_solve(h, th, opts)            # records the solve graph
            ms = []
            m = n if prec != T.TLR_PREC_FP32 else max(1, n // 4)
            for i in range(m):
                if nfreq > 1:
                    D, U = data[i % nfreq]
                    T.tlr_mdd_set_data(h, D, U, T.TLR_MEM_DEVICE)
                with torch.cuda.stream(stream):
                    th.copy_(th0)
                st = T.tlr_mdd_solve(h, th, opts)
                ms.append(st.gpu_ms)
            T.tlr_mdd_destroy(h)
            res[pname] = {"solves": m, "solves_per_s": round(1e3 * m / sum(ms), 2),
                          "p50_ms": round(percentile(ms, 50), 3), "p99_ms": round(percentile(ms, 99), 3)}
        res["speedup_tc_vs_fp32"] = round(res["bf16x3"]["solves_per_s"] / res["fp32"]["solves_per_s"], 2)
        if cpu:
            # the FP64 oracle's full solve (3 lambda stages x 2 ADMM x 5 L-BFGS)
            # of the first frequency, from its own panels, on the host cores
            from oracle import hilbert, layout, operator, solver
            lay = layout.make_layout(nr, b, k, "dense" if mode == T.TLR_DIAG_DENSE else "lowrank")
            Dh, Uh, _ = operator.normalise(data[0][0].cpu().numpy(), data[0][1].cpu().numpy(),
                                           hilbert.perm(nx, nx))
            prob = solver.Problem(lay, Dh.T, Uh.T)
            t0 = time.perf_counter()
            solver.admm(prob, th0.cpu().numpy().astype(np.complex128), solver.SolveOpts())
            secs = time.perf_counter() - t0
            res["oracle"] = {"solves_per_s": round(1.0 / secs, 4), "cores": blas_threads(),
                             "sample": f"one full 30-iteration FP64 solve of the first frequency in {secs:.2f} s"}
        res["workload"] = (f"nr={nr} ({nx}x{nx} grid), ns={rows.numel()}, tile {b}, rank {k}, "
                           f"{'dense' if mode == T.TLR_DIAG_DENSE else 'low-rank'} diagonal, {snr:g} dB, "
                           f"{nfreq} frequenc{'y' if nfreq == 1 else 'ies'}, 30 iterations; X a random symmetric "
                           f"matrix (the solve's work does not depend on it)")
        out[name] = res
    out["timing"] = "device time of each solve (CUDA events), CUDA-graph replays one at a time on one stream"
    return out


def collections_counter(xs):
    import collections
    return collections.Counter(xs)


def reference_arm(args, wl, world, rank):
    """The FP64 CPU oracle on this workload's config: each step is a bounded
    sample, the forward product and gradient of one frequency at the mean rank
    restricted to a subset of the source columns (the oracle's work is the
    same for every column), scaled to a 30-iteration solve of the whole
    frequency."""
    if rank != 0:
        return
    import tlr_synth as synth
    from oracle import hilbert, layout, operator, tlr
    ranks = wl.ranks(wl.nfreq)
    kmean = sum(ranks) / len(ranks)
    k0 = min(ranks, key=lambda k: abs(k - kmean))
    n = wl.nr
    cols = args.oracle_cols
    g = synth.rng(args.seed)
    # one frequency of the same recipe on the host, restricted to `cols` sources:
    # those rows of D = Q diag(sigma e^{i phi}) W^H and of U = D X + noise
    Q = synth.phase_dft_unitary(n, g)[:cols]
    W = synth.phase_dft_unitary(n, g)
    sig = synth.singular_decay(n)
    ph = np.exp(2j * np.pi * g.random(n))
    Ds = (Q * (sig * ph)[None, :]) @ W.conj().T
    del Q, W
    lay = layout.make_layout(n, wl.tile, k0, "rule")
    perm = hilbert.perm(*wl.grid)
    th_true = synth.planted_theta(n, wl.tile, k0, lay.dense, args.seed + 1)
    X = operator.unpermute(operator.assemble_xh(th_true, lay), perm)
    Ys = Ds @ X
    del X
    nz = synth.noise(Ys.shape, args.seed + 2)
    Us = (Ys + np.linalg.norm(Ys) / np.linalg.norm(nz) * 10 ** (-wl.snr_db / 20) * nz).astype(np.complex64)
    Ds = Ds.astype(np.complex64)
    Dh, Uh, _ = operator.normalise(Ds, Us, perm)
    Dt, Ut = Dh.T.copy(), Uh.T.copy()
    th0 = 0.1 * synth.planted_theta(n, wl.tile, k0, lay.dense, args.seed + 3)

    from oracle import solver
    prob = solver.Problem(lay, Dt, Ut)
    d = 0.01 * synth.cn(synth.rng(args.seed + 4), lay.size)

    def one():
        t0 = time.perf_counter()
        prob.fgrad(th0)
        t1 = time.perf_counter()
        prob.coefficients(th0, d, 1.0, th0)
        return t1 - t0, time.perf_counter() - t1

    for _ in range(args.warmup):
        one()
    ts = [one() for _ in range(args.steps)]
    t_f = sum(a for a, _ in ts) / len(ts)
    t_c = sum(b for _, b in ts) / len(ts)
    per_step = t_f + t_c
    # the oracle's solve: a first forward product and gradient, then per
    # iteration the line-search products and the gradient at the new point
    scale = n / cols
    per_solve = scale * (t_f + ITERS_PER_SOLVE * (t_f + t_c))
    v = 1.0 / per_solve
    sample = (f"per step: the FP64 TLR-structured oracle's forward product and gradient ({t_f:.2f} s) and "
              f"line-search products ({t_c:.2f} s) at rank {k0} (the mean rank) on {cols} of the {n} source "
              f"columns (its work is the same for every column); a {ITERS_PER_SOLVE}-iteration solve of the "
              f"whole frequency = {n}/{cols} x (first + {ITERS_PER_SOLVE} x iteration)")
    line = {"impl": "reference", "metric": "freq-solves/s", "value": round(v, 7), "unit": "freq-solves/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * per_step, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "nr": wl.nr, "ns": wl.nr, "grid": list(wl.grid),
                       "frequencies_per_gpu": wl.nfreq, "frequencies_per_step": wl.batch, "tile": wl.tile,
                       "ranks": f"{wl.rank_lo}->{wl.rank_hi} linear", "iters_per_solve": ITERS_PER_SOLVE,
                       "precision": "fp64 (oracle)", "parallelism": f"frequency sharding x{world}"},
            "cpu_baseline": {"value": round(v, 7), "unit": "freq-solves/s", "cores": blas_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(v, 7), "unit": "freq-solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
