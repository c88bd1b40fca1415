"""Oracle runs in worker processes (test infrastructure).

The long-run statistical parity tests simulate seconds of biological time of
networks that the single-threaded oracle needs minutes for; they start the
oracle runs here, in spawned worker processes (safe after the parent has
initialised CUDA), and run the GPU side meanwhile.
"""
from __future__ import annotations

import multiprocessing as mp
import os


def run(job):
    """job = (spec, steps, input_steps, receptors): build the oracle network of
    `spec` (tracking the FP64 sums of the inputs), record the input of the
    first `input_steps` steps on each receptor (exact FP64 sum and summed
    magnitudes), simulate `steps` steps in all and return
    (ids, steps, [(exact, magnitude) per step and receptor])."""
    spec, steps, input_steps, receptors = job
    import oracle
    o = oracle.OracleNet(spec, track_abs=input_steps > 0)
    o.finalize()
    inputs = []
    for _ in range(input_steps):
        for r in range(receptors):
            _, ab, ex = o.input(r, 0)
            inputs.append((ex, ab))
        o.simulate(1)
    o.simulate(steps - input_steps)
    ids, st = o.spikes()
    return ids, st, inputs


def start(jobs):
    """Start the jobs on a spawned pool; returns (pool, AsyncResult of the list of results)."""
    procs = max(1, min(len(jobs), (os.cpu_count() or 2) - 1))
    pool = mp.get_context("spawn").Pool(procs)
    return pool, pool.map_async(run, jobs, chunksize=1)
