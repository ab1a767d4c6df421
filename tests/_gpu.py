"""GPU test helpers: run the C-ABI library on torch device buffers (test helper)."""
import numpy as np
import torch

import paper_2412_14973_gb300 as T


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a).astype(np.complex64))).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.complex128)


def abi_desc(lay, ns, nx=0, ny=0, perm=None, alpha=0.0, precision=T.TLR_PREC_FP32,
             input_memory=T.TLR_MEM_DEVICE):
    ranks = list(lay.k_diag) + list(lay.k_pair)
    tiles = None if lay.b is not None else list(lay.d)   # non-uniform partition
    return T.desc(lay.nr, ns, lay.b or 0, ranks=ranks, nx=nx, ny=ny, perm=perm,
                  diag_mode=T.TLR_DIAG_PER_TILE, diag_dense=list(lay.dense),
                  precision=precision, alpha=alpha, input_memory=input_memory, tiles=tiles)


class Gpu:
    """One handle on device copies of D, U (paper layout)."""

    def __init__(self, D, U, lay, nx=0, ny=0, perm=None, alpha=0.0, precision=T.TLR_PREC_FP32,
                 host_inputs=False, stream=None, desc=None):
        self.lay = lay
        self.ns = D.shape[0]
        self.stream = stream
        mem = T.TLR_MEM_HOST if host_inputs else T.TLR_MEM_DEVICE
        self.d = desc if desc is not None else abi_desc(lay, self.ns, nx, ny, perm, alpha, precision, mem)
        if host_inputs:
            self._D = np.ascontiguousarray(D.astype(np.complex64))
            self._U = np.ascontiguousarray(U.astype(np.complex64))
        else:
            self._D, self._U = dev(D), dev(U)
        self.h = T.tlr_mdd_create(self.d, self._D, self._U, stream)

    def close(self):
        if self.h:
            T.tlr_mdd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def data(self):
        nr, ns = self.lay.nr, self.ns
        Dt = torch.empty((nr, ns), dtype=torch.complex64, device="cuda")
        Ut = torch.empty_like(Dt)
        perm, alpha = T.tlr_mdd_get_data(self.h, nr, Dt, Ut)
        return np.array(perm), alpha, Dt.cpu().numpy(), Ut.cpu().numpy()

    def apply(self, theta):
        Y = torch.empty((self.lay.nr, self.ns), dtype=torch.complex64, device="cuda")
        T.tlr_mdd_apply(self.h, dev(theta), Y)
        return host(Y)

    def grad(self, theta):
        g = torch.empty(self.lay.size, dtype=torch.complex64, device="cuda")
        f = T.tlr_mdd_grad(self.h, dev(theta), g)
        return f, host(g)

    def adjoint(self, V):
        G = torch.empty((self.lay.nr, self.lay.nr), dtype=torch.complex64, device="cuda")
        T.tlr_mdd_adjoint(self.h, dev(V), G)
        return host(G)

    def unpermute(self, theta):
        X = torch.empty((self.lay.nr, self.lay.nr), dtype=torch.complex64, device="cuda")
        T.tlr_mdd_unpermute_dense(self.h, dev(theta), X)
        return host(X)

    def benchmark(self, lam, iters, tol):
        X = torch.empty((self.lay.nr, self.lay.nr), dtype=torch.complex64, device="cuda")
        st = T.tlr_mdd_benchmark_solve(self.h, lam, iters, tol, X)
        return host(X), st

    def solve(self, theta0, **opts):
        th = dev(theta0)
        st = T.tlr_mdd_solve(self.h, th, T.solve_opts(**opts))
        return host(th), st


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def elem(a, b):
    """max elementwise error over the rms of the reference."""
    rms = np.linalg.norm(b) / np.sqrt(b.size)
    return float(np.max(np.abs(a - b)) / rms)
