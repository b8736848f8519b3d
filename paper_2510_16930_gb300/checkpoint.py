"""Checkpoint and resume of a decomposition.

A checkpoint holds the factors U_1..U_N, the number of sweeps run, the
residual history, every field of the context's options (precision, QR kind,
task size, autotune, graphs, one-stream form, seed, tolerance, lane tile), and the
tensor's dims and ranks (``numpy.savez``; the tensor itself is not stored: the
caller supplies the same nonzeros on resume).  Resuming creates a context from
the tensor with the saved factors as its initial factors and the saved
options.  The sorted storage is rebuilt the same way every time and every
reduction of the library has a fixed order, so the sweeps after a resume
equal, bit for bit, the sweeps of a ``hoqri_iterate`` call that the original
context would have made from the same factors (each call starts by
recomputing the core from the factors, Alg. 3), provided the nonzero-stream
layout is the same: always with autotune off; with autotune on, when the
resumed process finds the original choices in the tune cache (in memory, or
the file named by HOQRI_TUNE_CACHE), since a fresh timing may pick another
layout.  The residual history is returned by ``load`` but not handed to the
new context: the tolerance stop of ``hoqri_run`` counts from the resume.

Argument marshalling only: the factors come from ``hoqri_get_factor`` and go
back through ``hoqri_create``.
"""
from __future__ import annotations

import numpy as np

from . import hoqri

FORMAT = 2
OPTION_FIELDS = ("prec", "qr_kind", "chunk_nnz", "autotune", "use_graphs", "one_stream", "seed", "tol", "tile_rows",
                 "tile_cols")


def save(path, factors, *, dims, ranks, prec, sweeps, resid_hist=None, seed=0, options=None):
    """Writes a checkpoint; factors are host arrays I_n x K_n.  options: the
    context's hoqri_options (or a dict of its fields); prec and seed override
    its fields of the same name."""
    dims = [int(d) for d in dims]
    ranks = [int(k) for k in ranks]
    if len(factors) != len(dims) or len(ranks) != len(dims):
        raise ValueError("one factor, one dimension and one rank per mode")
    for n, U in enumerate(factors):
        if tuple(np.shape(U)) != (dims[n], ranks[n]):
            raise ValueError(f"factor {n} has shape {np.shape(U)}, expected {(dims[n], ranks[n])}")
    arrays = {f"U{n}": np.ascontiguousarray(U) for n, U in enumerate(factors)}
    opt = {}
    if options is not None:
        opt = dict(options) if isinstance(options, dict) else {f: getattr(options, f) for f in OPTION_FIELDS}
    opt["prec"], opt["seed"] = int(prec), int(seed)
    defaults = hoqri.hoqri_default_options()
    d0 = {f: getattr(defaults, f) for f in OPTION_FIELDS}
    d0.update(opt)
    np.savez(path, format=np.int64(FORMAT), dims=np.array(dims, dtype=np.int64),
             ranks=np.array(ranks, dtype=np.int64), prec=np.int64(prec), sweeps=np.int64(sweeps),
             seed=np.uint64(seed), resid_hist=np.asarray(resid_hist if resid_hist is not None else [], np.float64),
             options=np.array([float(d0[f]) for f in OPTION_FIELDS], dtype=np.float64), **arrays)


def load(path):
    """Reads a checkpoint: dict(U, dims, ranks, prec, sweeps, seed, resid_hist,
    options) with options a dict of the saved hoqri_options fields."""
    with np.load(path) as z:
        if int(z["format"]) != FORMAT:
            raise ValueError(f"checkpoint format {int(z['format'])}, expected {FORMAT}")
        dims = [int(d) for d in z["dims"]]
        ranks = [int(k) for k in z["ranks"]]
        U = [np.array(z[f"U{n}"]) for n in range(len(dims))]
        for n, u in enumerate(U):
            if u.shape != (dims[n], ranks[n]):
                raise ValueError(f"factor {n} has shape {u.shape}, expected {(dims[n], ranks[n])}")
        ov = [float(v) for v in z["options"]]
        options = {f: (v if f == "tol" else int(v)) for f, v in zip(OPTION_FIELDS, ov)}
        options["seed"] = int(z["seed"])
        return dict(U=U, dims=dims, ranks=ranks, prec=int(z["prec"]), sweeps=int(z["sweeps"]),
                    seed=int(z["seed"]), resid_hist=np.array(z["resid_hist"]), options=options)


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
    starting from the checkpoint's factors and options; keyword arguments
    override saved option fields."""
    saved = dict(ckpt.get("options", {}))
    saved.update(prec=ckpt["prec"], seed=ckpt["seed"])
    saved.update(options)
    opt = hoqri.hoqri_default_options(**saved)
    return hoqri.hoqri_create(ckpt["dims"], ckpt["ranks"], len(vals), idx, vals, opt, ckpt["U"], stream)
