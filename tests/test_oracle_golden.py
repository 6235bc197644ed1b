"""Regression pin: the oracle reproduces its stored n = 255 results
(written by tests/golden/make_golden.py, which calls only oracle/)."""
import json
import os

import numpy as np
import pytest

import lrp_inputs as li
from oracle import cross_deim as cd

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_n255.json")


@pytest.mark.parametrize("seed", [0, 1])
@pytest.mark.parametrize("selector,suffix", [("ls", ""), ("bernoulli", "_bernoulli")])
def test_oracle_n255_golden(seed, selector, suffix):
    ref = json.load(open(GOLDEN))[f"n255_seed{seed}{suffix}"]
    rhs = li.workload_single_small(seed)
    U, S, V, info, G = cd.poisson_solve(rhs.U, rhs.s, rhs.V, 1e-10, 32, seed=seed, m_cap=68, selector=selector)
    assert info.iterations == ref["iterations"]
    assert S.shape[0] == ref["rank"]
    assert np.abs(S - np.array(ref["sigma"])).max() < 1e-12 * ref["sigma"][0]
