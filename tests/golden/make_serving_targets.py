"""Write tests/golden/serving_targets.json: the target energy of every instance of the
serving pool (instances.serving_pool(32, seed=5)), defined as the best energy of a short
oracle run (4 replicas x 200 iterations, schedule from schedules.suggest_schedule).

Only the oracle and the seeded generators are used.  Run from the repository root:
    python tests/golden/make_serving_targets.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2407_10205_gb300 import instances as ins  # noqa: E402
from paper_2407_10205_gb300 import schedules  # noqa: E402

POOL, SEED, REPLICAS, ITERS = 32, 5, 4, 200


def main():
    pool = ins.serving_pool(POOL, SEED)
    out = []
    for k, inst in enumerate(pool):
        t0 = time.time()
        if getattr(inst, "k", None) is not None:
            P = oracle.Instance(inst.kh, k=inst.k, frac_bits=inst.frac_bits)
            kind = "dense"
        else:
            P = oracle.Instance(inst.kh, row_ptr=inst.row_ptr, col=inst.col, val=inst.val, frac_bits=inst.frac_bits)
            kind = "sparse"
        b0, b1, eps, gamma, refresh = schedules.suggest_schedule(inst)
        r = oracle.anneal(P, REPLICAS, ITERS, 1234 + k, k, b0, b1, eps, gamma, refresh=refresh,
                          threads=os.cpu_count(), want_spins=False)
        out.append({"index": k, "kind": kind, "N": inst.n, "target_k": int(r["best_e"].min())})
        print(k, kind, inst.n, out[-1]["target_k"], f"{time.time() - t0:.1f}s", flush=True)
    doc = {"pool_count": POOL, "pool_seed": SEED, "oracle_replicas": REPLICAS, "oracle_iterations": ITERS,
           "definition": "best energy (units of q) of an FP64 oracle run of the instance",
           "entries": out}
    with open(os.path.join(ROOT, "tests", "golden", "serving_targets.json"), "w") as f:
        json.dump(doc, f, indent=1)


if __name__ == "__main__":
    main()
