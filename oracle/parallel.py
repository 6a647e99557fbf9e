"""Process-pool evaluation of the oracle's per-candidate score.  TEST INFRASTRUCTURE.

The oracle scores one candidate at a time in float64 NumPy (single-threaded
FFTs).  Candidates are independent (Sec. 3.2: every node of the grid is
scored on its own), so a pool of worker processes scores a list of nodes in
parallel, one core each, with exactly the arithmetic of ``prnu_oracle.score``.
The pool starts its workers with the ``spawn`` method: a process that has
already touched a GPU must not fork.  Each worker holds one residual and one
fingerprint term (set once, by the pool initializer).

Only the tests and ``bench.py``'s CPU-baseline legs use it.
"""
from __future__ import annotations

import multiprocessing as mp
import os
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


def _init(R, K0):
    _STATE["R"] = np.asarray(R, dtype=np.float64)
    _STATE["K0"] = np.asarray(K0, dtype=np.float64)
    _STATE["FK"] = np.fft.rfft2(_STATE["K0"])


def _score_node(node):
    lam, th = node
    return score(_STATE["R"], _STATE["K0"], lam, th, _STATE["FK"])


class ScorePool:
    """``pool(nodes)`` -> [score(R, K0, lam, th) for (lam, th) in nodes], in order.

    A worker that cannot start or dies raises BrokenProcessPool in the caller
    (rather than being replaced and waited for)."""

    def __init__(self, R, K0, processes: int | None = None):
        self.processes = max(1, processes or available_cores())
        self._pool = ProcessPoolExecutor(self.processes, mp_context=mp.get_context("spawn"), initializer=_init,
                                         initargs=(R, K0))

    def __call__(self, nodes):
        nodes = [(float(l), float(t)) for l, t in nodes]
        if not nodes:
            return []
        chunk = max(1, len(nodes) // (4 * self.processes))
        return list(self._pool.map(_score_node, nodes, chunksize=chunk))

    def close(self):
        if self._pool is not None:
            self._pool.shutdown(wait=True, cancel_futures=True)
            self._pool = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
