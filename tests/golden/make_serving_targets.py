"""Write tests/golden/serving_targets.json: the target energy of every instance of the
serving pool (instances.serving_pool(32, seed=5)), defined as the best energy of an
oracle run as long as a budget of 4e11 multiply-adds of the field allows, up to 64
replicas x 5000 iterations (the serving step cap): replicas x iterations x (N^2 dense,
stored couplings sparse) <= 4e11, with at least 16 replicas; schedule from
schedules.suggest_schedule with a final jump of 6, as the serving benchmark runs.

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

POOL, SEED = 32, 5
BUDGET, MAX_REPLICAS, MIN_REPLICAS, MAX_ITERS = 4e11, 64, 16, 5000


def run_size(work_per_iter):
    """(replicas, iterations) within the budget."""
    for R in (MAX_REPLICAS, 32, MIN_REPLICAS):
        T = int(min(MAX_ITERS, BUDGET / (work_per_iter * R)))
        if T >= 1000 or R == MIN_REPLICAS:
            return R, max(T, 1)


def main():
    pool = ins.serving_pool(POOL, SEED)
    out = []
    for k, inst in enumerate(pool):
        t0 = time.time()
        if getattr(inst, "k", None) is not None:
            P = oracle.Instance(inst.kh, k=inst.k, frac_bits=inst.frac_bits)
            kind, work = "dense", float(inst.n) ** 2
        else:
            P = oracle.Instance(inst.kh, row_ptr=inst.row_ptr, col=inst.col, val=inst.val, frac_bits=inst.frac_bits)
            kind, work = "sparse", float(max(inst.nnz, inst.n))
        R, T = run_size(work)
        b0, b1, eps, gamma, refresh = schedules.suggest_schedule(inst, jump=6.0)
        r = oracle.anneal(P, R, T, 1234 + k, k, b0, b1, eps, gamma, refresh=refresh,
                          threads=os.cpu_count(), want_spins=False)
        out.append({"index": k, "kind": kind, "N": inst.n, "oracle_replicas": R, "oracle_iterations": T,
                    "target_k": int(r["best_e"].min())})
        print(k, kind, inst.n, out[-1]["target_k"], f"{time.time() - t0:.1f}s", flush=True)
    doc = {"pool_count": POOL, "pool_seed": SEED, "oracle_budget_macs": BUDGET,
           "definition": "best energy (units of q) of an FP64 oracle run of the instance (replicas and "
                         "iterations per entry)",
           "entries": out}
    with open(os.path.join(ROOT, "tests", "golden", "serving_targets.json"), "w") as f:
        json.dump(doc, f, indent=1)


if __name__ == "__main__":
    main()
