"""Writes tests/golden/*.json from the CPU oracle only (no GPU code involved).

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import lrp_inputs as li  # noqa: E402
from oracle import cross_deim as cd  # noqa: E402
from oracle import poisson as po  # noqa: E402


def main():
    out = {}
    runs = [(seed, sel, suffix, what) for seed in (0, 1)
            for sel, suffix, what in (("ls", "", "leverage scores, top-c"),
                                      ("bernoulli", "_bernoulli", "leverage scores, Bernoulli sampling"))]
    for seed, sel, suffix, what in runs:
        rhs = li.workload_single_small(seed)
        U, S, V, info, G = cd.poisson_solve(rhs.U, rhs.s, rhs.V, 1e-10, 32, seed=seed,
                                            m_cap=2 * 32 + 4, selector=sel)
        out[f"n255_seed{seed}{suffix}"] = {
            "workload": f"n=255, 4 Gaussians, tol 1e-10, max rank 32, {what}, m_cap 68",
            "iterations": info.iterations,
            "converged": info.converged,
            "rank": int(S.shape[0]),
            "sigma": [float(v) for v in S],
            "rel_err_vs_exact": po.rel_error_vs_exact(U, S, V, G),
            "I": [int(v) for v in info.I],
            "J": [int(v) for v in info.J],
        }
    with open(os.path.join(HERE, "oracle_n255.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
