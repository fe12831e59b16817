"""Regression pin: the oracle still reproduces the fixture written by
tests/golden/make_golden.py (FP64 oracle output for the 3-latent chain workload)."""
import json
import os

import numpy as np

import oracle
from paper_1806_08593_gb300 import workload as wl

GOLD = os.path.join(os.path.dirname(__file__), "golden", "oracle_chain_n3_K4_d2_B8.json")


def test_oracle_matches_stored_fixture():
    ref = json.load(open(GOLD))
    p = wl.chain_config("chain_n3_K4_d2_B8")
    np.testing.assert_allclose(oracle.log_marginal(p), ref["log_phat"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(ref["brute_force"], ref["log_phat"], rtol=0, atol=1e-12)
    g = oracle.grad(p)
    for k in ("dq_mean", "dq_logstd", "dW", "dbias", "dC"):
        np.testing.assert_allclose(g[k], ref[k], rtol=1e-10, atol=1e-12)
