"""Writes tests/golden/u2_oracle.json: FP64 oracle values for three pairs of
the long 1-D validation-shaped set (10 series of 100,000 points, nu =
lambda = 1, p = 2), on FP64 inputs and on the FP32-rounded inputs.

Calls only the oracle (rolling-row FP64, threads over pairs) and the seeded
input generators.  About 1e10 cells per value: a few minutes.
Run: python tests/golden/make_u2_expected.py
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

PAIRS = [(0, 1), (3, 7), (5, 9)]


def main():
    S = W.set_u2()
    S32 = S.astype(np.float32).astype(np.float64)
    pairs = np.array(PAIRS, dtype=np.int64)
    t0 = time.time()
    f64 = oracle.twed_pairs(S.as_tuple(), S.as_tuple(), pairs, 1.0, 1.0, 2)
    f32in = oracle.twed_pairs(S32.as_tuple(), S32.as_tuple(), pairs, 1.0, 1.0, 2)
    out = {"workload": "u2", "nseries": S.n, "length": int(S.lengths[0]), "nu": 1.0, "lambda": 1.0,
           "p": 2, "pairs": PAIRS, "f64_inputs": [float(v) for v in f64],
           "f32_rounded_inputs": [float(v) for v in f32in],
           "how": "oracle.twed_pairs (rolling-row FP64), tests/golden/make_u2_expected.py",
           "seconds": round(time.time() - t0, 1)}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "u2_oracle.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(out)


if __name__ == "__main__":
    main()
