"""ctypes binding of ``include/tlr_mdd.h`` -- argument marshalling only.

Every function mirrors the C entry point of the same name; tensors are passed
as raw device pointers (``tensor.data_ptr()``) and streams as
``torch.cuda.Stream.cuda_stream``.  Errors raise ``TLRError`` carrying the C
status code and the library's message.
"""
from __future__ import annotations

import ctypes as C
import os

__all__ = [
    "TLRError", "Desc", "SolveOpts", "Stats", "lib", "lib_path",
    "TLR_PREC_FP32", "TLR_PREC_BF16X3", "TLR_PREC_TF32", "TLR_DIAG_RULE", "TLR_DIAG_LOWRANK", "TLR_DIAG_DENSE",
    "TLR_DIAG_PER_TILE", "TLR_MEM_DEVICE", "TLR_MEM_HOST", "TLR_RECIP_SYMMETRIC", "TLR_RECIP_NONE",
    "ERR", "desc", "solve_opts", "tlr_mdd_theta_size", "tlr_mdd_theta_layout",
    "tlr_mdd_workspace_bytes", "tlr_mdd_hilbert_perm", "tlr_mdd_create", "tlr_mdd_apply",
    "tlr_mdd_adjoint", "tlr_mdd_grad", "tlr_mdd_solve", "tlr_mdd_unpermute_dense",
    "tlr_mdd_get_data", "tlr_mdd_destroy", "tlr_mdd_last_error", "EXPORTED",
    "tlr_mdd_timing_enable", "tlr_mdd_timing_reset", "tlr_mdd_timing_read", "tlr_mdd_launch_count",
    "tlr_mdd_adjoint_noalloc", "TLR_NOALLOC_SCRATCH_BYTES",
    "tlr_mdd_solve_async", "tlr_mdd_solve_query", "tlr_mdd_solve_wait", "tlr_mdd_set_data",
    "tlr_mdd_benchmark_solve", "BenchStats", "tlr_mdd_tile_ranks", "tlr_mdd_choose_tile", "tlr_mdd_warm_start",
    "tlr_mdd_get_state", "tlr_mdd_set_state", "TLR_SOLVE_RESUME", "TLR_SOLVE_REFRESH",
    "tlr_mdd_time_to_freq", "tlr_mdd_freq_to_time", "tlr_mdd_stack_alpha", "tlr_mdd_wait_selftest",
    "tlr_mdd_trim_pool", "tlr_mdd_set_stream", "tlr_mdd_batch_create", "tlr_mdd_batch_solve_async",
    "tlr_mdd_batch_query", "tlr_mdd_batch_wait", "tlr_mdd_batch_destroy", "Batch", "tlr_mdd_set_pass_ctas",
    "TLR_OK", "TLR_ERR_ARG", "TLR_ERR_SHAPE", "TLR_ERR_UNSUPPORTED", "TLR_ERR_NOMEM", "TLR_ERR_CUDA",
    "TLR_ERR_NONFINITE", "TLR_ERR_TIMEOUT", "TLR_ERR_STATE",
]

TLR_OK, TLR_ERR_ARG, TLR_ERR_SHAPE, TLR_ERR_UNSUPPORTED = 0, -1, -2, -3
TLR_ERR_NOMEM, TLR_ERR_CUDA, TLR_ERR_NONFINITE, TLR_ERR_TIMEOUT, TLR_ERR_STATE = -4, -5, -6, -7, -8
TLR_PREC_FP32, TLR_PREC_BF16X3, TLR_PREC_TF32 = 0, 1, 2
TLR_SOLVE_RESUME, TLR_SOLVE_REFRESH = 1, 2
TLR_DIAG_RULE, TLR_DIAG_LOWRANK, TLR_DIAG_DENSE, TLR_DIAG_PER_TILE = 0, 1, 2, 3
TLR_RECIP_SYMMETRIC, TLR_RECIP_NONE = 0, 1
TLR_MEM_DEVICE, TLR_MEM_HOST = 0, 1
ERR = {0: "OK", -1: "ARG", -2: "SHAPE", -3: "UNSUPPORTED", -4: "NOMEM", -5: "CUDA",
       -6: "NONFINITE", -7: "TIMEOUT", -8: "STATE"}
TLR_MAX_HIST = 1024

EXPORTED = [
    "tlr_mdd_desc_init", "tlr_mdd_solve_opts_init", "tlr_mdd_theta_size", "tlr_mdd_theta_layout",
    "tlr_mdd_workspace_bytes", "tlr_mdd_hilbert_perm", "tlr_mdd_create", "tlr_mdd_apply",
    "tlr_mdd_adjoint", "tlr_mdd_grad", "tlr_mdd_solve", "tlr_mdd_unpermute_dense",
    "tlr_mdd_get_data", "tlr_mdd_stream", "tlr_mdd_set_stream", "tlr_mdd_last_error", "tlr_mdd_destroy",
    "tlr_mdd_timing_enable", "tlr_mdd_timing_reset", "tlr_mdd_timing_read", "tlr_mdd_launch_count",
    "tlr_mdd_adjoint_noalloc", "tlr_mdd_solve_async", "tlr_mdd_solve_query", "tlr_mdd_solve_wait",
    "tlr_mdd_set_data", "tlr_mdd_benchmark_solve", "tlr_mdd_tile_ranks", "tlr_mdd_choose_tile",
    "tlr_mdd_warm_start", "tlr_mdd_get_state", "tlr_mdd_set_state", "tlr_mdd_time_to_freq",
    "tlr_mdd_freq_to_time", "tlr_mdd_stack_alpha", "tlr_mdd_wait_selftest", "tlr_mdd_trim_pool",
    "tlr_mdd_set_stream", "tlr_mdd_batch_create", "tlr_mdd_batch_solve_async", "tlr_mdd_batch_query",
    "tlr_mdd_batch_wait", "tlr_mdd_batch_destroy", "tlr_mdd_set_pass_ctas",
]
TLR_NCLASS = 3
TLR_NOALLOC_SCRATCH_BYTES = 16 << 20


class TLRError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"TLR_ERR_{ERR.get(code, code)} ({code}): {msg}")
        self.code = code


class Desc(C.Structure):
    _fields_ = [
        ("nr", C.c_int64), ("ns", C.c_int64), ("nx", C.c_int32), ("ny", C.c_int32),
        ("perm", C.POINTER(C.c_int32)), ("tile", C.c_int32), ("rank", C.c_int32),
        ("ranks", C.POINTER(C.c_int32)), ("diag_mode", C.c_int32),
        ("diag_dense", C.POINTER(C.c_uint8)), ("reciprocity", C.c_int32),
        ("precision", C.c_int32), ("alpha", C.c_double), ("input_memory", C.c_int32),
        ("ntiles", C.c_int32), ("tiles", C.POINTER(C.c_int32)),
    ]


class SolveOpts(C.Structure):
    _fields_ = [
        ("lam0", C.c_double), ("decay", C.c_double), ("stages", C.c_int32),
        ("admm_iters", C.c_int32), ("lbfgs_iters", C.c_int32), ("memory", C.c_int32),
        ("rho", C.c_double), ("theta_memory", C.c_int32), ("flags", C.c_int32),
    ]


class BenchStats(C.Structure):
    _fields_ = [
        ("iters", C.c_int32),
        ("status", C.c_int32),
        ("rel_res", C.c_double),
        ("gpu_ms", C.c_double),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("iters", C.c_int32), ("restarts", C.c_int32), ("status", C.c_int32), ("n_hist", C.c_int32),
        ("f_hist", C.c_double * TLR_MAX_HIST), ("f0", C.c_double), ("gpu_ms", C.c_double),
    ]


_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def lib_path() -> str:
    return os.path.join(_HERE, "lib", "libtlr_mdd.so")


def lib():
    """The loaded library; raises if it was not built (there is no fallback)."""
    global _LIB
    if _LIB is None:
        p = lib_path()
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build it with __graft_entry__.build() "
                               "(python paper_2412_14973_gb300/build.py)")
        L = C.CDLL(p)
        vp, i32, i64 = C.c_void_p, C.c_int, C.c_int64
        L.tlr_mdd_desc_init.argtypes = [C.POINTER(Desc)]
        L.tlr_mdd_desc_init.restype = None
        L.tlr_mdd_solve_opts_init.argtypes = [C.POINTER(SolveOpts)]
        L.tlr_mdd_solve_opts_init.restype = None
        L.tlr_mdd_theta_size.argtypes = [C.POINTER(Desc), C.POINTER(C.c_int64)]
        L.tlr_mdd_theta_layout.argtypes = [C.POINTER(Desc), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                           C.POINTER(C.c_int64), C.POINTER(C.c_uint8)]
        L.tlr_mdd_workspace_bytes.argtypes = [C.POINTER(Desc)]
        L.tlr_mdd_workspace_bytes.restype = i64
        L.tlr_mdd_hilbert_perm.argtypes = [C.c_int32, C.c_int32, vp, vp]
        L.tlr_mdd_create.argtypes = [C.POINTER(vp), C.POINTER(Desc), vp, vp, vp]
        L.tlr_mdd_apply.argtypes = [vp, vp, vp]
        L.tlr_mdd_adjoint.argtypes = [vp, vp, vp]
        L.tlr_mdd_grad.argtypes = [vp, vp, vp, C.POINTER(C.c_double)]
        L.tlr_mdd_solve.argtypes = [vp, vp, C.POINTER(SolveOpts), C.POINTER(Stats)]
        L.tlr_mdd_unpermute_dense.argtypes = [vp, vp, vp]
        L.tlr_mdd_get_data.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_double), vp, vp]
        L.tlr_mdd_stream.argtypes = [vp]
        L.tlr_mdd_stream.restype = vp
        L.tlr_mdd_set_stream.argtypes = [vp, vp]
        L.tlr_mdd_set_stream.restype = i32
        L.tlr_mdd_batch_create.argtypes = [C.POINTER(vp), C.POINTER(vp), C.c_int32, vp]
        L.tlr_mdd_batch_create.restype = i32
        L.tlr_mdd_batch_solve_async.argtypes = [vp, C.POINTER(vp), C.POINTER(SolveOpts)]
        L.tlr_mdd_batch_solve_async.restype = i32
        L.tlr_mdd_batch_query.argtypes = [vp]
        L.tlr_mdd_batch_query.restype = i32
        L.tlr_mdd_batch_wait.argtypes = [vp, C.POINTER(Stats)]
        L.tlr_mdd_batch_wait.restype = i32
        L.tlr_mdd_batch_destroy.argtypes = [vp]
        L.tlr_mdd_batch_destroy.restype = i32
        L.tlr_mdd_last_error.argtypes = [vp]
        L.tlr_mdd_last_error.restype = C.c_char_p
        L.tlr_mdd_destroy.argtypes = [vp]
        L.tlr_mdd_timing_enable.argtypes = [C.c_int]
        L.tlr_mdd_timing_enable.restype = None
        L.tlr_mdd_timing_reset.argtypes = []
        L.tlr_mdd_timing_reset.restype = None
        L.tlr_mdd_timing_read.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_double),
                                          C.POINTER(C.c_int64), C.c_int]
        L.tlr_mdd_timing_read.restype = i32
        L.tlr_mdd_launch_count.argtypes = []
        L.tlr_mdd_launch_count.restype = i64
        L.tlr_mdd_adjoint_noalloc.argtypes = [vp, vp, C.c_int64, C.c_int64, vp, vp]
        L.tlr_mdd_adjoint_noalloc.restype = i32
        L.tlr_mdd_solve_async.argtypes = [vp, vp, C.POINTER(SolveOpts)]
        L.tlr_mdd_solve_async.restype = i32
        L.tlr_mdd_solve_query.argtypes = [vp]
        L.tlr_mdd_solve_query.restype = i32
        L.tlr_mdd_solve_wait.argtypes = [vp, C.POINTER(Stats)]
        L.tlr_mdd_solve_wait.restype = i32
        L.tlr_mdd_set_data.argtypes = [vp, vp, vp, C.c_int32]
        L.tlr_mdd_benchmark_solve.argtypes = [vp, C.c_double, C.c_int32, C.c_double, vp, C.POINTER(BenchStats)]
        L.tlr_mdd_tile_ranks.argtypes = [vp, C.c_int64, C.c_int64, C.c_double, C.POINTER(C.c_int32),
                                         C.POINTER(C.c_int64), C.POINTER(C.c_double), vp]
        L.tlr_mdd_choose_tile.argtypes = [vp, C.c_int64, C.POINTER(C.c_int64), C.c_int32, C.c_double,
                                          C.POINTER(C.c_int64), C.POINTER(C.c_int64), vp]
        L.tlr_mdd_warm_start.argtypes = [vp, vp, vp]
        L.tlr_mdd_get_state.argtypes = [vp, vp, vp]
        L.tlr_mdd_time_to_freq.argtypes = [vp, C.c_int64, C.c_int64, C.c_int64, C.c_int64, vp, vp]
        L.tlr_mdd_freq_to_time.argtypes = [vp, C.c_int64, C.c_int64, C.c_int64, C.c_int64, vp, vp]
        L.tlr_mdd_stack_alpha.argtypes = [vp, C.c_int64, C.POINTER(C.c_double), vp]
        L.tlr_mdd_wait_selftest.argtypes = [C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_double), vp]
        L.tlr_mdd_set_state.argtypes = [vp, vp, vp]
        L.tlr_mdd_trim_pool.argtypes = [C.c_int64, C.POINTER(C.c_int64)]
        L.tlr_mdd_trim_pool.restype = i32
        L.tlr_mdd_set_pass_ctas.argtypes = [C.c_int64, C.POINTER(C.c_int64)]
        L.tlr_mdd_set_pass_ctas.restype = i32
        L.tlr_mdd_set_data.restype = i32
        for name in ("tlr_mdd_theta_size", "tlr_mdd_theta_layout", "tlr_mdd_hilbert_perm",
                     "tlr_mdd_create", "tlr_mdd_apply", "tlr_mdd_adjoint", "tlr_mdd_grad",
                     "tlr_mdd_solve", "tlr_mdd_unpermute_dense", "tlr_mdd_get_data",
                     "tlr_mdd_destroy"):
            getattr(L, name).restype = i32
        _LIB = L
    return _LIB


def _check(rc: int, h=None):
    if rc != 0:
        msg = lib().tlr_mdd_last_error(h)
        raise TLRError(rc, msg.decode() if msg else "")


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):          # numpy array (host)
        return x.ctypes.data
    raise TypeError(type(x))


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


class _Keep:
    """Keeps the host arrays referenced by a Desc alive."""


def desc(nr, ns, tile, rank=0, nx=0, ny=0, perm=None, ranks=None, diag_mode=TLR_DIAG_RULE,
         diag_dense=None, precision=TLR_PREC_FP32, alpha=0.0, input_memory=TLR_MEM_DEVICE,
         reciprocity=TLR_RECIP_SYMMETRIC, tiles=None) -> Desc:
    """``tiles``: the tile sizes d_i of a non-uniform partition (``tile`` is then ignored)."""
    d = Desc()
    lib().tlr_mdd_desc_init(C.byref(d))
    d.nr, d.ns, d.tile, d.rank, d.nx, d.ny = nr, ns, tile or 0, rank, nx, ny
    d.diag_mode, d.precision, d.alpha, d.input_memory = diag_mode, precision, float(alpha), input_memory
    d.reciprocity = reciprocity
    keep = []
    if tiles is not None:
        a = (C.c_int32 * max(1, len(tiles)))(*[int(v) for v in tiles])
        keep.append(a)
        d.tiles = C.cast(a, C.POINTER(C.c_int32))
        d.ntiles = len(tiles)
    if perm is not None:
        a = (C.c_int32 * len(perm))(*[int(v) for v in perm])
        keep.append(a)
        d.perm = C.cast(a, C.POINTER(C.c_int32))
    if ranks is not None:
        a = (C.c_int32 * len(ranks))(*[int(v) for v in ranks])
        keep.append(a)
        d.ranks = C.cast(a, C.POINTER(C.c_int32))
    if diag_dense is not None:
        a = (C.c_uint8 * len(diag_dense))(*[1 if v else 0 for v in diag_dense])
        keep.append(a)
        d.diag_dense = C.cast(a, C.POINTER(C.c_uint8))
    d._keep = keep
    return d


def solve_opts(**kw) -> SolveOpts:
    o = SolveOpts()
    lib().tlr_mdd_solve_opts_init(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def tlr_mdd_theta_size(d: Desc) -> int:
    n = C.c_int64()
    _check(lib().tlr_mdd_theta_size(C.byref(d), C.byref(n)))
    return n.value


def ntiles(d: Desc) -> int:
    """N, the number of tile rows of the description's partition."""
    return d.ntiles if d.tiles else d.nr // d.tile


def tlr_mdd_theta_layout(d: Desc):
    N = ntiles(d)
    P = N * (N - 1) if d.reciprocity == TLR_RECIP_NONE else N * (N - 1) // 2
    od = (C.c_int64 * max(N, 1))()
    ol = (C.c_int64 * max(P, 1))()
    orr = (C.c_int64 * max(P, 1))()
    dn = (C.c_uint8 * max(N, 1))()
    _check(lib().tlr_mdd_theta_layout(C.byref(d), od, ol, orr, dn))
    return list(od)[:N], list(ol)[:P], list(orr)[:P], [bool(x) for x in list(dn)[:N]]


def tlr_mdd_workspace_bytes(d: Desc) -> int:
    return lib().tlr_mdd_workspace_bytes(C.byref(d))


def tlr_mdd_hilbert_perm(nx, ny, perm_dev, stream=None):
    _check(lib().tlr_mdd_hilbert_perm(nx, ny, _ptr(perm_dev), _stream(stream)))


def tlr_mdd_create(d: Desc, D, U, stream=None) -> int:
    h = C.c_void_p()
    _check(lib().tlr_mdd_create(C.byref(h), C.byref(d), _ptr(D), _ptr(U), _stream(stream)))
    return h.value


def tlr_mdd_apply(h, theta, Y):
    _check(lib().tlr_mdd_apply(h, _ptr(theta), _ptr(Y)), h)


def tlr_mdd_adjoint(h, V, G):
    _check(lib().tlr_mdd_adjoint(h, _ptr(V), _ptr(G)), h)


def tlr_mdd_grad(h, theta, grad, want_f=True):
    f = C.c_double()
    _check(lib().tlr_mdd_grad(h, _ptr(theta), _ptr(grad), C.byref(f) if want_f else None), h)
    return f.value if want_f else None


def tlr_mdd_solve(h, theta, opts: SolveOpts | None = None) -> Stats:
    st = Stats()
    opts = opts if opts is not None else solve_opts()
    _check(lib().tlr_mdd_solve(h, _ptr(theta), C.byref(opts), C.byref(st)), h)
    return st


def tlr_mdd_unpermute_dense(h, theta, X):
    _check(lib().tlr_mdd_unpermute_dense(h, _ptr(theta), _ptr(X)), h)


def tlr_mdd_get_data(h, nr, Dt=None, Ut=None):
    perm = (C.c_int32 * nr)()
    alpha = C.c_double()
    _check(lib().tlr_mdd_get_data(h, perm, C.byref(alpha), _ptr(Dt), _ptr(Ut)), h)
    return list(perm), alpha.value


def tlr_mdd_destroy(h):
    _check(lib().tlr_mdd_destroy(h))


def tlr_mdd_last_error(h=None) -> str:
    m = lib().tlr_mdd_last_error(h)
    return m.decode() if m else ""


def tlr_mdd_timing_enable(on: bool):
    lib().tlr_mdd_timing_enable(1 if on else 0)


def tlr_mdd_timing_reset():
    lib().tlr_mdd_timing_reset()


def tlr_mdd_timing_read():
    """[(ms, flops, launches)] per class: 0 compress, 1 expand, 2 project."""
    ms = (C.c_double * TLR_NCLASS)()
    fl = (C.c_double * TLR_NCLASS)()
    nl = (C.c_int64 * TLR_NCLASS)()
    _check(lib().tlr_mdd_timing_read(ms, fl, nl, TLR_NCLASS))
    return [(ms[c], fl[c], nl[c]) for c in range(TLR_NCLASS)]


def tlr_mdd_launch_count() -> int:
    return lib().tlr_mdd_launch_count()


def tlr_mdd_benchmark_solve(h, lam, iters, tol, X) -> BenchStats:
    """Benchmark solver of eq. (4) on the handle's data; X (nr x nr, Hilbert
    order) receives the symmetric solution."""
    st = BenchStats()
    _check(lib().tlr_mdd_benchmark_solve(h, float(lam), int(iters), float(tol), _ptr(X), C.byref(st)), h)
    return st


def tlr_mdd_tile_ranks(X, nr, b, eps=0.01, stream=None):
    """Numerical ranks of the lower b x b tiles of X (device, nr x nr): returns
    (ranks in the descriptor's order, factor entry count, v0)."""
    N = nr // b if b > 0 and nr % b == 0 else 0
    r = (C.c_int32 * max(1, N * (N + 1) // 2))()
    ent, v0 = C.c_int64(), C.c_double()
    _check(lib().tlr_mdd_tile_ranks(_ptr(X), nr, b, float(eps), r, C.byref(ent), C.byref(v0), _stream(stream)))
    return list(r)[: N * (N + 1) // 2], ent.value, v0.value


def tlr_mdd_choose_tile(X, nr, candidates, eps=0.01, stream=None):
    """Tile size with the fewest factor entries among ``candidates``: (b, entries)."""
    c = (C.c_int64 * len(candidates))(*candidates)
    bb, be = C.c_int64(), C.c_int64()
    _check(lib().tlr_mdd_choose_tile(_ptr(X), nr, c, len(candidates), float(eps), C.byref(bb), C.byref(be),
                                     _stream(stream)))
    return bb.value, be.value


def tlr_mdd_warm_start(h, X, theta):
    """Warm-start factors (device theta) of the handle's layout from X (device, Hilbert order)."""
    _check(lib().tlr_mdd_warm_start(h, _ptr(X), _ptr(theta)), h)


def tlr_mdd_get_state(h, z, u):
    """Copy the handle's ADMM state z, u (device, theta order) out."""
    _check(lib().tlr_mdd_get_state(h, _ptr(z), _ptr(u)), h)


def tlr_mdd_set_state(h, z, u):
    """Load z, u (device, theta order) for a solve with TLR_SOLVE_RESUME."""
    _check(lib().tlr_mdd_set_state(h, _ptr(z), _ptr(u)), h)


def tlr_mdd_time_to_freq(x_t, ntr, nt, f0, nf, X_w, stream=None):
    """Frequency stack [nf][ntr] (device complex64) of trace-major x_t [ntr][nt] (device float)."""
    _check(lib().tlr_mdd_time_to_freq(_ptr(x_t), ntr, nt, f0, nf, _ptr(X_w), _stream(stream)))


def tlr_mdd_freq_to_time(X_w, ntr, nt, f0, nf, x_t, stream=None):
    """Traces [ntr][nt] (device float) from the band [f0, f0 + nf) of a frequency stack."""
    _check(lib().tlr_mdd_freq_to_time(_ptr(X_w), ntr, nt, f0, nf, _ptr(x_t), _stream(stream)))


def tlr_mdd_stack_alpha(D_w, n, stream=None) -> float:
    """max |D| over a whole frequency stack of n complex64 values (device)."""
    a = C.c_double()
    _check(lib().tlr_mdd_stack_alpha(_ptr(D_w), n, C.byref(a), _stream(stream)))
    return a.value


def tlr_mdd_wait_selftest(limit_ns, stream=None):
    """Run the contraction kernels' bounded barrier wait on a barrier that
    nothing completes: (status the kernel recorded, milliseconds it waited)."""
    st, ms = C.c_int32(), C.c_double()
    _check(lib().tlr_mdd_wait_selftest(int(limit_ns), C.byref(st), C.byref(ms), _stream(stream)))
    return st.value, ms.value


def _noalloc_args(V, Dt, nr, ns, G):
    """Checks the buffers of tlr_mdd_adjoint_noalloc before the call: the entry
    point has no handle that knows their sizes, so a short or misplaced buffer
    would be read or written out of bounds on the device.  torch tensors must
    be contiguous complex64 CUDA tensors on the current device holding at least
    nr * ns (V, Dt) and nr * nr (G) values.  Raw integer pointers are passed
    through unchecked (the C entry point still checks each pointer's device)."""
    if V is None or Dt is None or G is None:
        raise TLRError(TLR_ERR_ARG, "V, Dt and G must be given")
    if int(nr) <= 0 or int(ns) <= 0:
        raise TLRError(TLR_ERR_SHAPE, "nr and ns must be positive")
    need = {"V": int(nr) * int(ns), "Dt": int(nr) * int(ns), "G": int(nr) * int(nr)}
    tensors = [(n, t) for n, t in (("V", V), ("Dt", Dt), ("G", G)) if not isinstance(t, int)]
    for name, t in tensors:
        if not hasattr(t, "data_ptr") or not hasattr(t, "is_cuda"):
            raise TLRError(TLR_ERR_ARG, f"{name} must be a torch tensor or a device pointer")
        import torch
        if t.dtype != torch.complex64:
            raise TLRError(TLR_ERR_ARG, f"{name} must be complex64, not {t.dtype}")
        if not t.is_contiguous():
            raise TLRError(TLR_ERR_ARG, f"{name} must be contiguous")
        if t.numel() < need[name]:
            raise TLRError(TLR_ERR_SHAPE, f"{name} holds {t.numel()} values, needs {need[name]}")
    for name, t in tensors:
        import torch
        if not t.is_cuda or t.device.index != torch.cuda.current_device():
            raise TLRError(TLR_ERR_ARG, f"{name} must be on the current CUDA device")


def tlr_mdd_adjoint_noalloc(V, Dt, nr, ns, G, stream=None):
    """G = V Dt^H without any device allocation (fixed in-library scratch)."""
    _noalloc_args(V, Dt, nr, ns, G)
    _check(lib().tlr_mdd_adjoint_noalloc(_ptr(V), _ptr(Dt), nr, ns, _ptr(G), _stream(stream)))


def tlr_mdd_set_stream(h, stream=None):
    """Move a handle (no solve pending) to ``stream``."""
    _check(lib().tlr_mdd_set_stream(h, _stream(stream)), h)


class Batch:
    """A batched solve over handles (binding of tlr_mdd_batch_*): keeps the
    handle list and, while a solve is pending, the theta buffers alive."""

    def __init__(self, handles, stream=None):
        self.handles = list(handles)
        arr = (C.c_void_p * len(self.handles))(*self.handles)
        b = C.c_void_p()
        _check(lib().tlr_mdd_batch_create(C.byref(b), arr, len(self.handles), _stream(stream)))
        self.b = b.value
        self._keep = None

    def solve_async(self, thetas, opts: SolveOpts | None = None):
        opts = opts if opts is not None else solve_opts()
        if len(thetas) != len(self.handles):
            raise TLRError(TLR_ERR_ARG, "one theta per member")
        arr = (C.c_void_p * len(thetas))(*[_ptr(t) for t in thetas])
        self._keep = (list(thetas), arr, opts)
        _check(lib().tlr_mdd_batch_solve_async(self.b, arr, C.byref(opts)))

    def query(self) -> bool:
        rc = lib().tlr_mdd_batch_query(self.b)
        if rc < 0:
            _check(rc)
        return rc == 1

    def wait(self) -> list:
        st = (Stats * len(self.handles))()
        rc = lib().tlr_mdd_batch_wait(self.b, st)
        self._keep = None
        _check(rc)
        return list(st)

    def destroy(self):
        if self.b:
            _check(lib().tlr_mdd_batch_destroy(self.b))
            self.b = None


def tlr_mdd_batch_create(handles, stream=None) -> Batch:
    return Batch(handles, stream)


def tlr_mdd_batch_solve_async(batch: Batch, thetas, opts: SolveOpts | None = None):
    batch.solve_async(thetas, opts)


def tlr_mdd_batch_query(batch: Batch) -> bool:
    return batch.query()


def tlr_mdd_batch_wait(batch: Batch) -> list:
    return batch.wait()


def tlr_mdd_batch_destroy(batch: Batch):
    batch.destroy()


def tlr_mdd_trim_pool(keep_bytes=0) -> int:
    """Release the library's reserved workspace memory on the current device
    down to ``keep_bytes``; returns the bytes still reserved."""
    r = C.c_int64()
    _check(lib().tlr_mdd_trim_pool(int(keep_bytes), C.byref(r)))
    return r.value


def tlr_mdd_set_pass_ctas(ctas: int) -> int:
    """Cap the CTAs of the fused update-and-pack launches (0: one per tile),
    for launches made and graphs recorded from now on; returns the previous cap."""
    prev = C.c_int64()
    _check(lib().tlr_mdd_set_pass_ctas(int(ctas), C.byref(prev)))
    return prev.value


def tlr_mdd_solve_async(h, theta, opts: SolveOpts | None = None):
    """Enqueue a solve; keep ``theta`` (and ``opts``) alive until it finishes."""
    opts = opts if opts is not None else solve_opts()
    _check(lib().tlr_mdd_solve_async(h, _ptr(theta), C.byref(opts)), h)


def tlr_mdd_solve_query(h) -> bool:
    rc = lib().tlr_mdd_solve_query(h)
    if rc < 0:
        _check(rc, h)
    return rc == 1


def tlr_mdd_solve_wait(h) -> Stats:
    st = Stats()
    _check(lib().tlr_mdd_solve_wait(h, C.byref(st)), h)
    return st


def tlr_mdd_set_data(h, D, U, input_memory=TLR_MEM_DEVICE):
    _check(lib().tlr_mdd_set_data(h, _ptr(D), _ptr(U), input_memory), h)
