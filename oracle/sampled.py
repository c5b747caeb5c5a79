"""ORACLE -- test infrastructure only: the oracle's values on sampled rows of
meshes too large for its dense F, computed by a pool of worker processes.

Each worker builds the oracle mesh (snapped geometry and its own BVH) once
and evaluates, for the rows it is given, the visibility rows (Section 3.2)
and the F rows of Eq. FF-def (``oracle.F_rows``), or the point-sun
insolation (Eq. insolation-for-point-sun, ``oracle.insolation``); nothing
here adds arithmetic of its own.  F rows come back as sparse rows (the
nonzeros of each row), so a 4,096-row sample of a 522,242-facet mesh stays
small.  The pool uses the ``spawn`` start method, so it is safe to create
after CUDA has been initialised in the parent.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

_W: dict = {}


def _init(verts, faces):
    import oracle
    m = oracle.mesh(verts, faces)
    m.bvh()
    _W["m"] = m


def _rows_task(rows):
    import oracle
    Fr = oracle.F_rows(_W["m"], rows)
    out = []
    for r in range(Fr.shape[0]):
        nz = np.nonzero(Fr[r])[0].astype(np.int64)
        out.append((nz, Fr[r, nz]))
    return out


def _sun_task(args):
    import oracle
    dirs, rows, S = args
    E = oracle.insolation(_W["m"], dirs, S)
    return E[rows]


def default_workers() -> int:
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    return max(1, n - 1)  # one core left for the process that drives the GPU


class SampledOracle:
    """F rows and insolation of the oracle on a fixed set of rows."""

    def __init__(self, verts, faces, rows, workers: int | None = None, chunk: int = 8):
        self.rows = np.asarray(rows, dtype=np.int64)
        self.n = int(np.asarray(faces).shape[0])
        self.workers = workers or default_workers()
        self.chunk = chunk
        ctx = mp.get_context("spawn")
        self.pool = ctx.Pool(self.workers, initializer=_init,
                             initargs=(np.ascontiguousarray(verts, dtype=np.float64),
                                       np.ascontiguousarray(faces, dtype=np.int32)))

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()
            self.pool = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def F_rows_async(self):
        """Start the F rows in the pool; pass the result to F_rows_sparse."""
        parts = [self.rows[i:i + self.chunk] for i in range(0, self.rows.size, self.chunk)]
        return self.pool.map_async(_rows_task, parts)

    def F_rows_sparse(self, pending=None):
        """The sampled rows of F as (indptr, indices, data) of a CSR matrix
        (len(rows) x N, FP64)."""
        res = (pending if pending is not None else self.F_rows_async()).get()
        indptr = [0]
        idx, val = [], []
        for chunk in res:
            for nz, v in chunk:
                idx.append(nz)
                val.append(v)
                indptr.append(indptr[-1] + nz.size)
        return (np.asarray(indptr, dtype=np.int64), np.concatenate(idx) if idx else np.zeros(0, np.int64),
                np.concatenate(val) if val else np.zeros(0))

    def insolation_rows(self, dirs, solar_flux: float):
        """E on the sampled rows (len(rows) x R, FP64) for the sun directions dirs (R x 3)."""
        dirs = np.atleast_2d(np.asarray(dirs, dtype=np.float64))
        per = max(1, -(-dirs.shape[0] // self.workers))
        tasks = [(dirs[i:i + per], self.rows, solar_flux) for i in range(0, dirs.shape[0], per)]
        return np.concatenate(self.pool.map(_sun_task, tasks), axis=1)


def csr_matmul(indptr, indices, data, X):
    """(sparse rows) @ X for X of shape (N, R), FP64 (a library sparse product)."""
    import scipy.sparse as sp
    X = np.asarray(X, dtype=np.float64)
    A = sp.csr_matrix((data, indices, indptr), shape=(indptr.size - 1, X.shape[0]))
    return np.asarray(A @ X)
