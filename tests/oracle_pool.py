"""Run oracle row computations in parallel worker processes (spawn-started,
numpy only), for the full-size parity tests.  Imports nothing but the oracle."""
import multiprocessing as mp
import os

import numpy as np

from oracle import tsk_oracle as o


def _rows(args):
    x, m, excl, rows = args
    return o.mp_rows(x, m, excl, rows)


def pool_rows(jobs, workers=None):
    """jobs: [(x, m, excl, rows)] -> [(P, I)], each job on a worker."""
    workers = workers or max(1, min(16, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_rows, jobs, chunksize=1)


def pool_profiles(streams, m, excl, workers=None, chunk=2048):
    """Whole self-join profiles of several streams, rows split across workers."""
    jobs, index = [], []
    for q, x in enumerate(streams):
        l = len(x) - m + 1
        for r0 in range(0, l, chunk):
            jobs.append((np.asarray(x, dtype=np.float64), m, excl, np.arange(r0, min(l, r0 + chunk))))
            index.append(q)
    res = pool_rows(jobs, workers)
    P = [[] for _ in streams]
    I = [[] for _ in streams]
    for q, (p, i) in zip(index, res):
        P[q].append(p)
        I[q].append(i)
    return np.array([np.concatenate(p) for p in P]), np.array([np.concatenate(i) for i in I])
