"""Writes batch_complete_ff.json: the oracle's complete first-fail solves of
the 256 seeded models of the uneven 6-10-task family (config-2
distributions otherwise), the batched complete-solve workload.  Calls only
the oracle (plain sequential depth-first branch and bound).

    python tests/golden/make_batch_complete.py   (a few CPU minutes)
"""
import json
import os
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from oracle.rcpsp import rcpsp_model  # noqa: E402
from synthetic import config_instance  # noqa: E402

FAMILY = "mixed6_10"
N_MODELS = 256


def solve(seed):
    inst = config_instance(FAMILY, seed)
    r = oracle.solve(rcpsp_model(inst), strategy=oracle.FIRST_FAIL)
    return {"seed": seed, "n": inst.n, "status": r["status"], "objective": r["objective"],
            "nodes": r["nodes"], "fails": r["fails"], "solutions": r["solutions"],
            "max_depth": r["max_depth"],
            "witness_starts": [int(x) for x in r["witness"][: inst.n]]}


def main():
    oracle.build()
    with ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        rows = list(ex.map(solve, range(N_MODELS)))
    out = {"about": "oracle complete first-fail solves; see make_batch_complete.py",
           "family": FAMILY, "strategy": "first_fail", "models": rows}
    with open(os.path.join(HERE, "batch_complete_ff.json"), "w") as f:
        json.dump(out, f)
        f.write("\n")


if __name__ == "__main__":
    main()
