"""Continuous-batching server for per-frequency TLR-MDD solve requests.

Each request is one frequency's solve (its own nr, tile size and rank).  The
server admits arrived requests in arrival order while the device-memory
budget (the library's own footprint figure, ``tlr_mdd_workspace_bytes``) and
the number of slots allow, runs each admitted solve asynchronously on a
stream of its own (``tlr_mdd_solve_async``: the solve's launch sequence is a
recorded CUDA graph), and, as solves finish, admits the next requests, so
work from requests that arrived at different times overlaps on the GPU.  A
request larger than the whole budget is rejected at admission
(TLR_ERR_NOMEM), never attempted.

Finished handles are kept, with their workspace and recorded solve, in a
cache keyed by the problem's shape (nr, ns, grid, tiles, ranks, diagonal
modes, precision): a later request of that shape takes one over
(``tlr_mdd_set_stream`` to its slot's stream, ``tlr_mdd_set_data`` for its
D, U), so its admission allocates nothing and records nothing.  Idle cached
handles count against the budget and are destroyed, least recently used
first, when an admission needs their memory.

A queued request can be withdrawn (``Server.cancel``, from any thread) or
carry an admission deadline (``SolveRequest.deadline``, seconds after its
arrival); either ends it before admission with status ``CANCELLED`` or
``EXPIRED`` (server codes outside the library's TLR_ERR_* range).  An
admitted solve always runs to its end: its launch sequence is on the GPU.

Only host-side scheduling lives here; every computation is in the CUDA
library.  Results do not depend on what else is running: the library's
reductions have a fixed order, so a request gives the same bits alone and in
the mix.
"""
from __future__ import annotations

import collections
import json
import threading
import time
from dataclasses import dataclass, field

import torch

from . import tlr_mdd as T


# statuses the server itself gives (the library's codes are -1 .. -8)
CANCELLED = -101   # withdrawn while queued
EXPIRED = -102     # not admitted within its deadline


@dataclass
class SolveRequest:
    rid: int
    arrival: float              # seconds after the stream starts
    desc: T.Desc                # problem description (device inputs)
    D: torch.Tensor             # complex64 ns x nr, on the device
    U: torch.Tensor
    theta0: torch.Tensor        # complex64 start point, on the device
    opts: T.SolveOpts = field(default_factory=T.solve_opts)
    deadline: float | None = None   # seconds after arrival by which it must be admitted


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


def shape_key(d):
    """Cache key of a problem description: every field that shapes the
    handle's layout, workspace and recorded solve (not the data)."""
    if isinstance(d, T.Desc):
        arrays = tuple(tuple(a) for a in getattr(d, "_keep", []))
        return (d.nr, d.ns, d.nx, d.ny, d.tile, d.rank, d.diag_mode, d.reciprocity, d.precision, d.alpha,
                d.input_memory, d.ntiles, bool(d.tiles), bool(d.perm), bool(d.ranks), bool(d.diag_dense), arrays)
    try:
        hash(d)
        return d
    except TypeError:
        return id(d)


class Server:
    def __init__(self, hbm_budget_bytes: int, max_active: int = 8, device=None, poll_s: float = 2e-4,
                 stream_factory=None, reuse: bool = True, batch_max: int = 1, window: int = 32,
                 mix_sizes: bool = False):
        self.budget = int(hbm_budget_bytes)
        self.max_active = max(1, int(max_active))
        self.poll_s = poll_s
        self.reuse = reuse
        self.batch_max = max(1, int(batch_max))   # requests per lockstep batch (1: one per slot)
        self.window = window                      # queued requests scanned for batch partners
        # batch partners of any size (each contraction launch then walks the
        # tiles of problems of several sizes) instead of the head's size only
        self.mix_sizes = bool(mix_sizes)
        self.batches = 0
        if stream_factory is None:
            dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
            stream_factory = lambda: torch.cuda.Stream(device=dev)  # noqa: E731
        self.streams = [stream_factory() for _ in range(self.max_active)]
        self.used = 0
        self.peak_used = 0
        self.peak_active = 0
        self.idle = collections.OrderedDict()   # handle -> (key, bytes), least recently used first
        self.created = 0
        self.reused = 0
        self.evicted = 0
        self._cancelled = set()   # request ids withdrawn by cancel()
        self._cancel_lock = threading.Lock()

    def cancel(self, rid) -> None:
        """Withdraw request ``rid`` of the current or next ``run`` if it is
        still queued (safe to call from another thread while ``run`` serves;
        an admitted request finishes, and ``run`` forgets such cancels when
        it returns)."""
        with self._cancel_lock:
            self._cancelled.add(rid)

    def _drop_withdrawn(self, queue, out, now) -> bool:
        """End the queued requests that were cancelled or whose admission
        deadline has passed; True if any."""
        with self._cancel_lock:
            cancelled = set(self._cancelled)
        dropped = False
        for r in list(queue):
            if r.rid in cancelled:
                queue.remove(r)
                with self._cancel_lock:
                    self._cancelled.discard(r.rid)
                out.append(SolveResult(r.rid, None, CANCELLED, "cancelled before admission", r.arrival, now, now,
                                       0.0, 0))
                dropped = True
            elif r.deadline is not None and now - r.arrival > r.deadline:
                queue.remove(r)
                out.append(SolveResult(r.rid, None, EXPIRED, "admission deadline passed", r.arrival, now, now,
                                       0.0, 0))
                dropped = True
        return dropped

    def footprint(self, req: SolveRequest) -> int:
        return T.tlr_mdd_workspace_bytes(req.desc)

    def _take_idle(self, key):
        for h, (k, need) in reversed(self.idle.items()):
            if k == key:
                del self.idle[h]
                return h, need
        return None, 0

    def _evict_until(self, need) -> None:
        while self.idle and self.used + need > self.budget:
            h, (k, n) = self.idle.popitem(last=False)
            T.tlr_mdd_destroy(h)
            self.used -= n
            self.evicted += 1

    def close(self) -> None:
        """Destroy the cached idle handles and release their memory."""
        while self.idle:
            h, (k, n) = self.idle.popitem(last=False)
            T.tlr_mdd_destroy(h)
            self.used -= n

    def _acquire(self, req, key):
        """A handle for req: a cached one of its shape (no allocation), or the
        budget for a new one (idle handles evicted as needed).  Returns
        (handle or None, bytes, status): status -4 when the request can never
        fit, 1 when it must wait for memory, 0 otherwise."""
        h, need = self._take_idle(key) if self.reuse else (None, 0)
        if h is not None:
            return h, need, 0
        need = self.footprint(req)
        if need < 0 or need > self.budget:
            return None, need, -4
        self._evict_until(need)
        if self.used + need > self.budget:
            return None, need, 1
        return None, need, 0

    def _group(self, queue, realtime, now):
        """The head request and, when batching, later arrived requests of the
        same precision and solver options (lockstep solves end together) and,
        unless ``mix_sizes``, the same size."""
        head = queue[0]
        group = [head]
        if self.batch_max <= 1 or getattr(head.desc, "precision", 0) == T.TLR_PREC_FP32:
            return group

        def key(r):
            nr = None if self.mix_sizes else getattr(r.desc, "nr", None)
            return (nr, getattr(r.desc, "precision", None), _opts_key(r.opts))

        hk = key(head)
        for r in list(queue)[1:self.window]:
            if len(group) >= self.batch_max or (realtime and r.arrival > now):
                break
            if key(r) == hk:
                group.append(r)
        return group

    def run(self, requests, realtime: bool = True) -> list:
        """Serve ``requests``; with ``realtime`` a request is not admitted
        before its arrival time (seconds from the call), else all arrive at 0."""
        queue = collections.deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        free = list(range(self.max_active))
        active = []   # units: (slot, members [(req, h, theta, need, key, t_adm, fresh)], batch or None)
        out = []
        t0 = time.perf_counter()
        while queue or active:
            now = time.perf_counter() - t0
            progressed = self._drop_withdrawn(queue, out, now)
            while queue and free and (not realtime or queue[0].arrival <= now):
                members = []
                blocked = False
                for req in self._group(queue, realtime, now):
                    key = shape_key(req.desc)
                    h, need, st = self._acquire(req, key)
                    if st == -4:
                        if req is queue[0] or not members:
                            queue.remove(req)
                            out.append(SolveResult(req.rid, None, -4, "request exceeds the device-memory budget",
                                                   req.arrival, now, now, 0.0, 0))
                            progressed = True
                        continue
                    if st == 1:
                        blocked = not members   # the head waits for memory; later ones wait their turn
                        break
                    fresh = h is None
                    if fresh:
                        self.used += need
                    members.append([req, h, None, need, key, now, fresh])
                if not members:
                    if blocked:
                        break   # first-come first-served: wait for memory to free up
                    continue
                for m in members:
                    queue.remove(m[0])
                slot = free.pop()
                stream = self.streams[slot]
                unit = self._start(members, stream, out, now)
                if unit is None:
                    free.append(slot)
                else:
                    active.append((slot,) + unit)
                    self.peak_active = max(self.peak_active, sum(len(u[1]) for u in active))
                self.peak_used = max(self.peak_used, self.used)
                progressed = True
            for unit in list(active):
                slot, members, batch = unit
                done = batch.query() if batch is not None else T.tlr_mdd_solve_query(members[0][1])
                if not done:
                    continue
                self._finish(members, batch, out, time.perf_counter() - t0)
                active.remove(unit)
                free.append(slot)
                progressed = True
            if not progressed:
                if realtime and queue and not active:
                    time.sleep(max(0.0, min(queue[0].arrival - (time.perf_counter() - t0), 0.01)))
                else:
                    time.sleep(self.poll_s)
        with self._cancel_lock:
            self._cancelled.clear()   # cancels of requests that were already admitted
        return sorted(out, key=lambda r: r.rid)

    def _start(self, members, stream, out, now):
        """Create or take over the members' handles and enqueue their solve:
        one handle alone, or several as one lockstep batch."""
        started = []
        for m in members:
            req, h, _, need, key, t_adm, fresh = m
            m[2] = req.theta0.clone() if hasattr(req.theta0, "clone") else req.theta0
            try:
                if fresh:
                    m[1] = T.tlr_mdd_create(req.desc, req.D, req.U, stream)
                    self.created += 1
                else:
                    T.tlr_mdd_set_stream(h, stream)
                    T.tlr_mdd_set_data(h, req.D, req.U, getattr(req.desc, "input_memory", 0))
                    self.reused += 1
                started.append(m)
            except T.TLRError as e:
                self.used -= need
                if not fresh:
                    T.tlr_mdd_destroy(h)
                out.append(SolveResult(req.rid, None, e.code, str(e), req.arrival, now, now, 0.0, 0))
        if not started:
            return None
        batch = None
        try:
            if len(started) > 1:
                batch = T.Batch([m[1] for m in started], stream)
                batch.solve_async([m[2] for m in started], started[0][0].opts)
                self.batches += 1
            else:
                T.tlr_mdd_solve_async(started[0][1], started[0][2], started[0][0].opts)
        except T.TLRError as e:
            if batch is not None:
                batch.destroy()
            for m in started:
                self._release(m, ok=False)
                out.append(SolveResult(m[0].rid, None, e.code, str(e), m[0].arrival, now, now, 0.0, 0))
            return None
        return started, batch

    def _release(self, m, ok):
        req, h, theta, need, key, t_adm, fresh = m
        if self.reuse and ok:
            self.idle[h] = (key, need)       # most recently used last
        else:
            T.tlr_mdd_destroy(h)
            self.used -= need

    def _finish(self, members, batch, out, t_end):
        if batch is not None:
            try:
                stats = batch.wait()
                res = [(0, "", st.gpu_ms, st.iters) for st in stats]
            except T.TLRError as e:
                res = [(e.code, str(e), 0.0, 0)] * len(members)
            batch.destroy()
        else:
            try:
                st = T.tlr_mdd_solve_wait(members[0][1])
                res = [(0, "", st.gpu_ms, st.iters)]
            except T.TLRError as e:
                res = [(e.code, str(e), 0.0, 0)]
        for m, (status, msg, ms, iters) in zip(members, res):
            req, h, theta, need, key, t_adm, fresh = m
            self._release(m, ok=status == 0)
            out.append(SolveResult(req.rid, theta if status == 0 else theta, status, msg, req.arrival, t_adm, t_end,
                                   ms, iters))


def _opts_key(o):
    if o is None:
        return None
    try:
        return tuple(getattr(o, f) for f, _ in o._fields_)
    except AttributeError:
        return id(o)


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
