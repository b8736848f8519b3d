"""Checkpoint and resume of a decomposition.

A checkpoint holds the factors U_1..U_N, the number of sweeps run, the
residual history, the precision and seed, and the tensor's dims and ranks
(``numpy.savez``; the tensor itself is not stored: the caller supplies the same
nonzeros on resume).  Resuming creates a context from the tensor with the saved
factors as its initial factors.  The sorted storage is rebuilt the same way
every time and every reduction of the library has a fixed order, so the sweeps
after a resume equal, bit for bit, the sweeps of a ``hoqri_iterate`` call that
the original context would have made from the same factors (each call starts by
recomputing the core from the factors, Alg. 3).

Argument marshalling only: the factors come from ``hoqri_get_factor`` and go
back through ``hoqri_create``.
"""
from __future__ import annotations

import numpy as np

from . import hoqri

FORMAT = 1


def save(path, factors, *, dims, ranks, prec, sweeps, resid_hist=None, seed=0):
    """Writes a checkpoint; factors are host arrays I_n x K_n."""
    dims = [int(d) for d in dims]
    ranks = [int(k) for k in ranks]
    if len(factors) != len(dims) or len(ranks) != len(dims):
        raise ValueError("one factor, one dimension and one rank per mode")
    for n, U in enumerate(factors):
        if tuple(np.shape(U)) != (dims[n], ranks[n]):
            raise ValueError(f"factor {n} has shape {np.shape(U)}, expected {(dims[n], ranks[n])}")
    arrays = {f"U{n}": np.ascontiguousarray(U) for n, U in enumerate(factors)}
    np.savez(path, format=np.int64(FORMAT), dims=np.array(dims, dtype=np.int64),
             ranks=np.array(ranks, dtype=np.int64), prec=np.int64(prec), sweeps=np.int64(sweeps),
             seed=np.uint64(seed), resid_hist=np.asarray(resid_hist if resid_hist is not None else [], np.float64),
             **arrays)


def load(path):
    """Reads a checkpoint: dict(U, dims, ranks, prec, sweeps, seed, resid_hist)."""
    with np.load(path) as z:
        if int(z["format"]) != FORMAT:
            raise ValueError(f"checkpoint format {int(z['format'])}, expected {FORMAT}")
        dims = [int(d) for d in z["dims"]]
        ranks = [int(k) for k in z["ranks"]]
        U = [np.array(z[f"U{n}"]) for n in range(len(dims))]
        for n, u in enumerate(U):
            if u.shape != (dims[n], ranks[n]):
                raise ValueError(f"factor {n} has shape {u.shape}, expected {(dims[n], ranks[n])}")
        return dict(U=U, dims=dims, ranks=ranks, prec=int(z["prec"]), sweeps=int(z["sweeps"]),
                    seed=int(z["seed"]), resid_hist=np.array(z["resid_hist"]))


def capture(ctx, dims, ranks, prec):
    """The current factors of a context, copied to host arrays."""
    dt = np.float64 if prec == hoqri.HOQRI_FP64 else np.float32
    out = []
    for n, (I, K) in enumerate(zip(dims, ranks)):
        U = np.empty((int(I), int(K)), dtype=dt)
        hoqri.hoqri_get_factor(ctx, n, U)
        out.append(U)
    return out


def resume(ckpt, idx, vals, stream=0, **options):
    """A new context over the same nonzeros (idx, vals: as for hoqri_create),
    starting from the checkpoint's factors, precision and seed; further options
    as for hoqri_default_options."""
    opt = hoqri.hoqri_default_options(prec=ckpt["prec"], seed=ckpt["seed"], **options)
    return hoqri.hoqri_create(ckpt["dims"], ckpt["ranks"], len(vals), idx, vals, opt, ckpt["U"], stream)
