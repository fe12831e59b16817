"""Writes the oracle regression fixtures in this folder.  Calls only the FP64 oracle and the
seeded workload generator; nothing here comes from the CUDA path.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1806_08593_gb300 import workload as wl  # noqa: E402


def main():
    p = wl.chain_config("chain_n3_K4_d2_B8")
    g = oracle.grad(p)
    out = {
        "what": "log P_TMC (Eq. (is)) and its gradient for the 3-latent chain, K=4, d=2, obs=4, "
                "B=8, seed 20181806, from the FP64 oracle (regression fixture)",
        "log_phat": [float(v) for v in oracle.log_marginal(p)],
        "brute_force": [float(v) for v in oracle.brute_force(p)],
        "dq_mean": [float(v) for v in g["dq_mean"]],
        "dq_logstd": [float(v) for v in g["dq_logstd"]],
        "dW": [float(v) for v in g["dW"]],
        "dbias": [float(v) for v in g["dbias"]],
        "dC": [float(v) for v in g["dC"]],
    }
    with open(os.path.join(HERE, "oracle_chain_n3_K4_d2_B8.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
