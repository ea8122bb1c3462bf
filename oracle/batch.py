"""Oracle reference solutions for a batch of parameters, and the error of given solutions
against them.

TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the benchmark's checking
and CPU-baseline legs, never by the product.  Shares no code with the CUDA library.

Each parameter mu_b is solved independently by the oracle's MGCG (Algorithm 1 with the
V-cycle of Algorithm 2 as preconditioner, oracle.mg) from a zero initial value, on A(mu_b)
assembled directly (orc_assemble_mu), in FP64.  The work is spread over worker processes
started with the "spawn" method (safe after a CUDA context exists in the parent).  Only mu
(and a right-hand side, if any) goes to the workers: no input comes from the solutions under
test.  The solutions under test enter only error_summary(), which measures them.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import time

import numpy as np

from . import Operator, assemble_field, assemble_mu

_STATE = {}


def _init(grid, blocks, submap, Q, kscale=(1.0, 1.0, 1.0), neumann=(0, 0, 0), fields=None):
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    _STATE["grid"], _STATE["blocks"], _STATE["submap"], _STATE["Q"] = grid, blocks, submap, Q
    _STATE["kscale"], _STATE["neumann"] = tuple(kscale), tuple(neumann)
    _STATE["field_op"] = None if fields is None else assemble_field(grid, *fields)


def _operator(mu):
    """A(mu) as a one-term operator: assembled directly, or combined from the face-field terms."""
    fo = _STATE.get("field_op")
    if fo is not None:
        return Operator(fo.grid, 1, fo.row_ptr, fo.col, fo.values(mu)[None, :])
    return assemble_mu(_STATE["grid"], mu, blocks=_STATE["blocks"], submap=_STATE["submap"], Q=_STATE["Q"],
                       kscale=_STATE["kscale"], neumann=_STATE["neumann"])


def _solve(task):
    from . import mg
    mu, f, tol, u0 = task
    op = _operator(mu)
    r = mg.mgcg(op, [1.0], f=f, u0=u0, tol=tol, max_iters=400)
    return r.u, r.iters, r.relres, r.status


def reference_solutions(grid, mus, blocks=None, submap=None, Q=None, f=None, tol=1e-13, processes=None,
                        kscale=(1.0, 1.0, 1.0), neumann=(0, 0, 0), u0=None, fields=None):
    """Oracle FP64 MGCG solutions u_b of A(mu_b) u = f_b (f: None = ones, [n] shared, or [B][n];
    kscale, neumann: the operator's anisotropy and Neumann faces, as oracle.assemble takes them;
    u0: None (zero start) or [B][n] initial values computed by the oracle; fields: None, or the
    face coefficients (kfx, kfy, kfz) of oracle.assemble_field, mus then being the [B][Q]
    coefficients of its terms).
    Returns (U [B][n], iters [B], relres [B], status [B], seconds, processes)."""
    mus = np.atleast_2d(np.asarray(mus, dtype=np.float64))
    B = mus.shape[0]
    if submap is not None:
        submap = np.ascontiguousarray(submap, dtype=np.uint8)
    fb = [None] * B
    if f is not None:
        f = np.asarray(f, dtype=np.float64)
        fb = [f[b] for b in range(B)] if f.ndim == 2 else [f] * B
    if processes is None:
        processes = max(1, min(B, len(os.sched_getaffinity(0))))
    t0 = time.perf_counter()
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
    os.environ.update({"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1"})
    try:
        tasks = [(mus[b], fb[b], tol, None if u0 is None else np.asarray(u0[b], dtype=np.float64)) for b in range(B)]
        if processes == 1:
            _init(tuple(grid), blocks, submap, Q, kscale, neumann, fields)
            out = [_solve(t) for t in tasks]
        else:
            with mp.get_context("spawn").Pool(processes, initializer=_init,
                                              initargs=(tuple(grid), blocks, submap, Q, kscale, neumann,
                                                        fields)) as pool:
                out = pool.map(_solve, tasks, chunksize=1)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    U = np.stack([o[0] for o in out])
    its = np.array([o[1] for o in out])
    rel = np.array([o[2] for o in out])
    st = np.array([o[3] for o in out])
    return U, its, rel, st, time.perf_counter() - t0, processes


def true_relres(grid, mus, U, blocks=None, submap=None, Q=None, f=None, kscale=(1.0, 1.0, 1.0),
                neumann=(0, 0, 0), fields=None) -> np.ndarray:
    """||f_b - A(mu_b) u_b|| / ||f_b|| with the oracle's CSR operator, per instance."""
    mus = np.atleast_2d(np.asarray(mus, dtype=np.float64))
    out = np.empty(mus.shape[0])
    fo = None if fields is None else assemble_field(grid, *fields)
    for b in range(mus.shape[0]):
        if fo is not None:
            op = Operator(fo.grid, 1, fo.row_ptr, fo.col, fo.values(mus[b])[None, :])
        else:
            op = assemble_mu(grid, mus[b], blocks=blocks, submap=submap, Q=Q, kscale=kscale, neumann=neumann)
        fb = np.ones(op.n) if f is None else (f[b] if np.ndim(f) == 2 else f)
        out[b] = np.linalg.norm(fb - op.matvec([1.0], U[b])) / np.linalg.norm(fb)
    return out


def relL2(U, U_ref) -> np.ndarray:
    """||u_b - u_ref_b|| / ||u_ref_b|| per instance."""
    U = np.asarray(U, dtype=np.float64)
    return np.linalg.norm(U - U_ref, axis=1) / np.linalg.norm(U_ref, axis=1)


def error_summary(grid, mus, U, U_ref, blocks=None, submap=None, Q=None, f=None, kscale=(1.0, 1.0, 1.0),
                  neumann=(0, 0, 0), fields=None) -> dict:
    """Per-instance relative L2 error of U against the oracle solutions U_ref and the oracle's
    true relative residual of U; max and mean of each, and the per-instance lists."""
    U = np.asarray(U, dtype=np.float64)
    err = relL2(U, U_ref)
    res = true_relres(grid, mus, U, blocks=blocks, submap=submap, Q=Q, f=f, kscale=kscale, neumann=neumann,
                      fields=fields)
    return {"n": int(U.shape[0]), "relL2_max": float(err.max()), "relL2_mean": float(err.mean()),
            "true_relres_max": float(res.max()), "true_relres_mean": float(res.mean()),
            "relL2": [float(x) for x in err], "true_relres": [float(x) for x in res]}

