"""Continuous-batching server for per-frequency TLR-MDD solve requests.

Each request is one frequency's solve (its own nr, tile size and rank).  The
server admits arrived requests in arrival order while the device-memory
budget (the library's own footprint figure, ``tlr_mdd_workspace_bytes``) and
the number of slots allow, runs each admitted solve asynchronously on a
stream of its own (``tlr_mdd_solve_async``: the solve's launch sequence is a
recorded CUDA graph), and, as solves finish, frees their memory and admits
the next requests, so work from requests that arrived at different times
overlaps on the GPU.  A request larger than the whole budget is rejected at
admission (TLR_ERR_NOMEM), never attempted.

Only host-side scheduling lives here; every computation is in the CUDA
library.  Results do not depend on what else is running: the library's
reductions have a fixed order, so a request gives the same bits alone and in
the mix.
"""
from __future__ import annotations

import collections
import json
import time
from dataclasses import dataclass, field

import torch

from . import tlr_mdd as T


@dataclass
class SolveRequest:
    rid: int
    arrival: float              # seconds after the stream starts
    desc: T.Desc                # problem description (device inputs)
    D: torch.Tensor             # complex64 ns x nr, on the device
    U: torch.Tensor
    theta0: torch.Tensor        # complex64 start point, on the device
    opts: T.SolveOpts = field(default_factory=T.solve_opts)


@dataclass
class SolveResult:
    rid: int
    theta: torch.Tensor | None
    status: int                 # 0 or a TLR_ERR_* code
    message: str
    arrival: float
    admitted: float
    finished: float
    gpu_ms: float
    iters: int

    @property
    def latency(self) -> float:
        return self.finished - self.arrival

    @property
    def queue_wait(self) -> float:
        return self.admitted - self.arrival


class Server:
    def __init__(self, hbm_budget_bytes: int, max_active: int = 8, device=None, poll_s: float = 2e-4,
                 stream_factory=None):
        self.budget = int(hbm_budget_bytes)
        self.max_active = max(1, int(max_active))
        self.poll_s = poll_s
        if stream_factory is None:
            dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
            stream_factory = lambda: torch.cuda.Stream(device=dev)  # noqa: E731
        self.streams = [stream_factory() for _ in range(self.max_active)]
        self.used = 0
        self.peak_used = 0
        self.peak_active = 0

    def footprint(self, req: SolveRequest) -> int:
        return T.tlr_mdd_workspace_bytes(req.desc)

    def run(self, requests, realtime: bool = True) -> list:
        """Serve ``requests``; with ``realtime`` a request is not admitted
        before its arrival time (seconds from the call), else all arrive at 0."""
        queue = collections.deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        free = list(range(self.max_active))
        active = {}
        out = []
        t0 = time.perf_counter()
        while queue or active:
            now = time.perf_counter() - t0
            progressed = False
            while queue and free and (not realtime or queue[0].arrival <= now):
                req = queue[0]
                need = self.footprint(req)
                if need < 0 or need > self.budget:
                    queue.popleft()
                    out.append(SolveResult(req.rid, None, -4, "request exceeds the device-memory budget",
                                           req.arrival, now, now, 0.0, 0))
                    progressed = True
                    continue
                if self.used + need > self.budget:
                    break   # first-come first-served: wait for memory to free up
                queue.popleft()
                slot = free.pop()
                stream = self.streams[slot]
                theta = req.theta0.clone() if hasattr(req.theta0, "clone") else req.theta0
                try:
                    h = T.tlr_mdd_create(req.desc, req.D, req.U, stream)
                    T.tlr_mdd_solve_async(h, theta, req.opts)
                except T.TLRError as e:
                    free.append(slot)
                    out.append(SolveResult(req.rid, None, e.code, str(e), req.arrival, now, now, 0.0, 0))
                    progressed = True
                    continue
                self.used += need
                self.peak_used = max(self.peak_used, self.used)
                active[req.rid] = (req, h, slot, theta, need, now)
                self.peak_active = max(self.peak_active, len(active))
                progressed = True
            for rid in list(active):
                req, h, slot, theta, need, t_adm = active[rid]
                if not T.tlr_mdd_solve_query(h):
                    continue
                status, msg, ms, iters = 0, "", 0.0, 0
                try:
                    st = T.tlr_mdd_solve_wait(h)
                    ms, iters = st.gpu_ms, st.iters
                except T.TLRError as e:
                    status, msg = e.code, str(e)
                T.tlr_mdd_destroy(h)
                del active[rid]
                free.append(slot)
                self.used -= need
                out.append(SolveResult(rid, theta, status, msg, req.arrival, t_adm,
                                       time.perf_counter() - t0, ms, iters))
                progressed = True
            if not progressed:
                if realtime and queue and not active:
                    time.sleep(max(0.0, min(queue[0].arrival - (time.perf_counter() - t0), 0.01)))
                else:
                    time.sleep(self.poll_s)
        return sorted(out, key=lambda r: r.rid)


def percentiles(results, ps=(50, 99)):
    lat = sorted(r.latency for r in results if r.status == 0)
    if not lat:
        return {p: None for p in ps}
    out = {}
    for p in ps:
        i = min(len(lat) - 1, max(0, int(-(-p * len(lat) // 100)) - 1))
        out[p] = lat[i]
    return out


def records(requests, results) -> list:
    """One log record per request: its problem (nr, ns, tile or tile count,
    rank, precision), queue wait, latency and device time in ms, solver
    iterations and status.  ``desc`` may be any object with those fields."""
    by_id = {r.rid: r for r in requests}
    out = []
    for res in results:
        d = by_id[res.rid].desc
        tiles = getattr(d, "tiles", None)
        prec = getattr(d, "precision", None)
        out.append({
            "rid": res.rid,
            "nr": int(getattr(d, "nr", 0)), "ns": int(getattr(d, "ns", 0)),
            "tile": None if tiles else int(getattr(d, "tile", 0)),
            "ntiles": int(getattr(d, "ntiles", 0)) if tiles else None,
            "rank": int(getattr(d, "rank", 0)),
            "precision": {T.TLR_PREC_FP32: "fp32", T.TLR_PREC_BF16X3: "bf16x3"}.get(prec),
            "queue_wait_ms": round(1e3 * res.queue_wait, 3),
            "latency_ms": round(1e3 * res.latency, 3),
            "gpu_ms": round(float(res.gpu_ms), 3),
            "iters": int(res.iters),
            "status": int(res.status),
            "message": res.message,
        })
    return out


def write_jsonl(path, recs) -> None:
    """The records, one JSON object per line."""
    with open(path, "w") as fh:
        for r in recs:
            fh.write(json.dumps(r) + "\n")
