"""Helpers shared by the GPU tests: move oracle/generator arrays to column-major CUDA tensors."""
import numpy as np
import torch


def to_dev(a: np.ndarray) -> torch.Tensor:
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        return torch.from_numpy(a.copy()).cuda()
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()


def to_np(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().astype(np.float64)


def rhs_dev(rhs):
    return to_dev(rhs.U), to_dev(rhs.s), to_dev(rhs.V)


def _exact_error_n4095(job):
    import lrp_inputs as li
    from oracle import poisson as po
    seed, U, S, V = job
    r = li.workload_n4095(seed=seed)
    return po.rel_error_vs_exact(U, S, V, po.SpectralSolution(r.U, r.s, r.V))


def exact_errors_n4095(seeds, results, procs=16):
    """Exact relative errors of n = 4095 bench-workload results (U, S, V as CUDA
    tensors, rank columns only) against the oracle's exact solution, computed in
    a pool of spawned worker processes (never forked from this CUDA process)."""
    import multiprocessing as mp
    import os
    jobs = [(sd, to_np(U), to_np(S), to_np(V)) for sd, (U, S, V) in zip(seeds, results)]
    with mp.get_context("spawn").Pool(max(1, min(procs, os.cpu_count() or 1))) as pool:
        return np.array(pool.map(_exact_error_n4095, jobs, chunksize=4))
