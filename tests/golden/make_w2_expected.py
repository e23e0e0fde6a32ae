"""Writes tests/golden/w2_oracle.json: FP64 oracle values for the one-pair
3-D workload (random walks, cumulative Exp(1) time gaps, nu = 0.001,
lambda = 1, p = 2) at n = m = 100000, plus its FP32-rounded-input twin.

Calls only the oracle (rolling-row FP64, bit-identical to the full matrix)
and the seeded input generators.  About 1e10 cells per value: minutes.
Run: python tests/golden/make_w2_expected.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2007_16135_gb300 import workloads as W  # noqa: E402


def main():
    n = 100_000
    a, ta, b, tb = W.pair_w2(n)
    out = {"workload": "w2", "n": n, "m": n, "nu": 0.001, "lambda": 1.0, "p": 2,
           "how": "oracle.twed_rolling (FP64), tests/golden/make_w2_expected.py"}
    t0 = time.time()
    out["f64_inputs"] = oracle.twed_rolling(a, ta, b, tb, 0.001, 1.0, 2)
    f = lambda x: np.asarray(x, dtype=np.float32).astype(np.float64)
    out["f32_rounded_inputs"] = oracle.twed_rolling(f(a), f(ta), f(b), f(tb), 0.001, 1.0, 2)
    out["seconds"] = round(time.time() - t0, 1)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "w2_oracle.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(out)


if __name__ == "__main__":
    main()
