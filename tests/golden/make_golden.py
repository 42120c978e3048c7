"""Writes the stored expected values under tests/golden/ from the FP64 oracle only.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2310_08770_b300 import synth  # noqa: E402


def main():
    p = synth.single_pair(seed=0)
    out = {}
    for name, method in (("ccu", oracle.CC_U), ("ccsn", oracle.CC_SN)):
        r = oracle.track_one(p.frame, p.ref, u=100, method=method, eps=200.0)
        out[name] = {k: r[k] for k in ("dx", "dy", "peak", "ipy", "ipx", "jy", "jx")}
    out["_source"] = ("FP64 oracle on the single-pair workload: 64x64 float32, sigma 3, "
                      "amplitude 1000, background 10, shift (+0.37, -1.21), seed 0, u = 100")
    with open(os.path.join(HERE, "single_pair_oracle.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
