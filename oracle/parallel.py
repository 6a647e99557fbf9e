"""Process-pool evaluation of the oracle's per-candidate score.  TEST INFRASTRUCTURE.

The oracle scores one candidate at a time in float64 NumPy (single-threaded
FFTs).  Candidates are independent (Sec. 3.2: every node of the grid is
scored on its own), so a pool of worker processes scores a list of nodes in
parallel, one core each, with exactly the arithmetic of ``prnu_oracle.score``.
The pool starts its workers with the ``spawn`` method: a process that has
already touched a GPU must not fork.  The residuals and the fingerprint term
reach the workers through .npy files in a private temporary directory (read
memory-mapped), so large frames are not pickled once per worker.

Only the tests and ``bench.py``'s CPU-baseline legs use it.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import shutil
import tempfile
from concurrent.futures import ProcessPoolExecutor

import numpy as np

from .prnu_oracle import score

__all__ = ["available_cores", "ScorePool"]

_STATE = {}


def available_cores() -> int:
    """Cores this process may run on (its affinity mask), else os.cpu_count()."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _init(d):
    _STATE["R"] = np.load(os.path.join(d, "R.npy"), mmap_mode="r")
    _STATE["K0"] = np.load(os.path.join(d, "K0.npy"), mmap_mode="r")
    _STATE["FK"] = {}


def _score_node(node):
    f, lam, th = node
    K0 = _STATE["K0"]
    kf = f if K0.ndim == 3 else 0          # one fingerprint term per frame, or one for all
    if kf not in _STATE["FK"]:
        _STATE["FK"][kf] = np.fft.rfft2(np.asarray(K0[kf] if K0.ndim == 3 else K0))
    K = np.asarray(K0[kf] if K0.ndim == 3 else K0)
    return score(np.asarray(_STATE["R"][f]), K, lam, th, _STATE["FK"][kf])


class ScorePool:
    """Score candidates of the residual(s) R against K0 in worker processes.

    R is one residual [H, W] or a stack [F, H, W]; K0 one fingerprint term
    [H, W] or one per frame [F, H, W].  ``pool(nodes)`` takes (lam, th) pairs
    (frame 0) or (f, lam, th) triples and returns [score(R[f], K0 (or K0[f]),
    lam, th) ...] in order.  A worker that cannot start or
    dies raises BrokenProcessPool in the caller (it is not replaced and waited
    for)."""

    def __init__(self, R, K0, processes: int | None = None):
        R = np.asarray(R, dtype=np.float64)
        if R.ndim == 2:
            R = R[None]
        self.processes = max(1, processes or available_cores())
        self._dir = tempfile.mkdtemp(prefix="oracle-pool-")
        np.save(os.path.join(self._dir, "R.npy"), R)
        np.save(os.path.join(self._dir, "K0.npy"), np.asarray(K0, dtype=np.float64))
        self._pool = ProcessPoolExecutor(self.processes, mp_context=mp.get_context("spawn"), initializer=_init,
                                         initargs=(self._dir,))

    def __call__(self, nodes):
        nodes = [(0, float(n[0]), float(n[1])) if len(n) == 2 else (int(n[0]), float(n[1]), float(n[2]))
                 for n in nodes]
        if not nodes:
            return []
        chunk = max(1, len(nodes) // (4 * self.processes))
        return list(self._pool.map(_score_node, nodes, chunksize=chunk))

    def close(self):
        if self._pool is not None:
            self._pool.shutdown(wait=True, cancel_futures=True)
            self._pool = None
        if self._dir is not None:
            shutil.rmtree(self._dir, ignore_errors=True)
            self._dir = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
