"""Writes tts_optima.json: the exhaustive optimum (Eq. 2 minimised over all 2^n states by
the oracle's brute force) of every instance of the time-to-solution study with n <= 16,
for each Table 2 family.  It calls only oracle/ (and the seeded input generators).

Instance k of family f at size n is instances.family_instance(f, n, instances.tts_seed(f, n,
k)) -- bench.py's TTS workload draws the same instances."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2407_10205_gb300 import instances as ins  # noqa: E402

SIZES = (8, 16)
INSTANCES = 100
BASE_SEED = 9


def tts_seed(family: str, n: int, k: int) -> int:
    return ins.tts_seed(family, n, k, BASE_SEED)


def main():
    out = {"doc": "exhaustive optima (units of q) of the TTS study's instances with n <= 16; "
                  "written by tests/golden/make_tts_optima.py with the oracle's brute force",
           "instances": INSTANCES, "base_seed": BASE_SEED, "optima": {}}
    for f in sorted(ins.FAMILIES):
        for n in SIZES:
            vals = []
            for k in range(INSTANCES):
                d = ins.family_instance(f, n, tts_seed(f, n, k))
                P = oracle.Instance(d.kh, k=d.k, frac_bits=d.frac_bits)
                vals.append(oracle.brute_force(P)[0])
            out["optima"][f"{f}/{n}"] = vals
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "tts_optima.json"), "w") as fh:
        json.dump(out, fh)


if __name__ == "__main__":
    main()
