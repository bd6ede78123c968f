"""Run independent oracle calls in parallel host processes (test infrastructure).

The processes are spawned, never forked, so that a pool started after the GPU was initialised
in the parent is safe.  Each job is (function name in ``oracle``, positional args, keyword
args); results come back in job order.
"""
from __future__ import annotations

import multiprocessing as mp
import os


def _call(job):
    name, args, kwargs = job
    import oracle
    return getattr(oracle, name)(*args, **kwargs)


def run_parallel(jobs, processes=None):
    jobs = list(jobs)
    if not jobs:
        return []
    n = processes or max(1, min(len(jobs), os.cpu_count() or 1))
    if n == 1:
        return [_call(j) for j in jobs]
    import oracle
    oracle.build()  # compile once before the workers load it
    with mp.get_context("spawn").Pool(n) as pool:
        return pool.map(_call, jobs, chunksize=1)
