"""Write the stored expected values under tests/golden/ from the CPU oracle only.

The paper prints no worked numeric example for its KS evaluation, so every stored value here is
the oracle's, computed on the seeded single-series workload (T=64 steps, m=32 samples, one true
change point at step 40; alpha = 1e-6).  Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402


def main():
    b = synth.generate(1, 0, 1)
    k, num, den, p = oracle.ks_scan(b.samples, b.offsets, b.steps)
    rc, cnt, idx, cnum, cden, cp = oracle.ks_segment(b.samples, b.offsets, b.steps, 1e-6, 1, 8)
    out = {
        "workload": "single series, T=64, m=32, seed 0 (32+Poisson(2) | 210+Poisson(6), 1% U{1000..5000})",
        "samples_sum": int(b.samples.astype(np.uint64).sum()),
        "samples_xor": int(np.bitwise_xor.reduce(b.samples)),
        "scan": {"k": int(k[0]), "num": int(num[0]), "den": int(den[0]), "p": float(p[0])},
        "segment_alpha_1e-6": {"count": int(cnt[0]), "idx": idx[0, :cnt[0]].tolist(),
                               "num": cnum[0, :cnt[0]].tolist(), "den": cden[0, :cnt[0]].tolist(),
                               "p": cp[0, :cnt[0]].tolist()},
    }
    with open(os.path.join(HERE, "single_series_64x32_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
