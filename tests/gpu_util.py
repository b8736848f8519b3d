"""Helpers for the GPU tests: move a seeded workload to the device and drive the
C ABI through the Python binding."""
import numpy as np

from paper_2510_16930_gb300 import hoqri

TOL = {hoqri.HOQRI_FP64: 1e-10, hoqri.HOQRI_FP32: 1e-5}


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    if nb == 0:
        return float(np.linalg.norm(a))
    return float(np.linalg.norm(a - b) / nb)


def dtype_of(prec):
    import torch
    return torch.float64 if prec == hoqri.HOQRI_FP64 else torch.float32


class Ctx:
    """One library context built from host arrays copied to the device."""

    def __init__(self, dims, idx, vals, U0, prec, chunk=0, qr_kind=0, host_inputs=False, stream=0, **opts):
        import torch
        self.torch = torch
        self.dims = tuple(int(d) for d in dims)
        self.ranks = tuple(int(u.shape[1]) for u in U0)
        self.prec = prec
        dt = dtype_of(prec)
        npdt = np.float64 if prec == hoqri.HOQRI_FP64 else np.float32
        if host_inputs:
            self._idx = [np.ascontiguousarray(a, dtype=np.int32) for a in idx]
            self._vals = np.ascontiguousarray(vals, dtype=npdt)
            self._U0 = [np.ascontiguousarray(u, dtype=npdt) for u in U0]
        else:
            self._idx = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda() for a in idx]
            self._vals = torch.from_numpy(np.ascontiguousarray(vals, dtype=npdt)).cuda()
            self._U0 = [torch.from_numpy(np.ascontiguousarray(u, dtype=npdt)).cuda() for u in U0]
        opt = hoqri.hoqri_default_options(prec=prec, chunk_nnz=chunk, qr_kind=qr_kind, **opts)
        self.h = hoqri.hoqri_create(self.dims, self.ranks, len(vals), self._idx, self._vals, opt, self._U0, stream)
        self.dt = dt

    def ttmctc(self, n):
        A = self.torch.empty((self.dims[n], self.ranks[n]), dtype=self.dt, device="cuda")
        hoqri.hoqri_ttmctc(self.h, n, A)
        self.torch.cuda.synchronize()
        return A.cpu().double().numpy()

    def core(self):
        G = self.torch.empty(self.ranks, dtype=self.dt, device="cuda")
        hoqri.hoqri_core(self.h, G)
        self.torch.cuda.synchronize()
        return G.cpu().double().numpy()

    def factor(self, n):
        U = self.torch.empty((self.dims[n], self.ranks[n]), dtype=self.dt, device="cuda")
        hoqri.hoqri_get_factor(self.h, n, U)
        self.torch.cuda.synchronize()
        return U.cpu().double().numpy()

    def orthonormalize(self, n, A):
        Ad = self.torch.from_numpy(np.ascontiguousarray(A)).to(self.dt).cuda()
        U = self.torch.empty_like(Ad)
        hoqri.hoqri_orthonormalize(self.h, n, Ad, U)
        self.torch.cuda.synchronize()
        return U.cpu().double().numpy()

    def iterate(self, iters):
        return hoqri.hoqri_iterate(self.h, iters)

    def info(self):
        return hoqri.hoqri_info(self.h, len(self.dims))

    def close(self):
        hoqri.hoqri_destroy(self.h)
        self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
