"""Stored oracle outputs stay the oracle's: the cheapest models of the
batched complete-solve file are solved again and compared field by field
(a stale file after an oracle change fails here, on the CPU)."""
import json
import os

import oracle
from oracle.rcpsp import rcpsp_model
from synthetic import config_instance

HERE = os.path.dirname(os.path.abspath(__file__))


def test_batch_complete_file_matches_live_oracle():
    with open(os.path.join(HERE, "golden", "batch_complete_ff.json")) as f:
        g = json.load(f)
    assert len(g["models"]) == 256 and all(m["status"] == oracle.RES_OPTIMAL for m in g["models"])
    cheap = sorted(g["models"], key=lambda m: m["nodes"])[:40]
    for m in cheap:
        inst = config_instance(g["family"], m["seed"])
        r = oracle.solve(rcpsp_model(inst), strategy=oracle.FIRST_FAIL)
        assert (r["status"], r["objective"], r["nodes"], r["fails"], r["solutions"],
                r["max_depth"]) == (m["status"], m["objective"], m["nodes"], m["fails"],
                                    m["solutions"], m["max_depth"])
        assert [int(x) for x in r["witness"][: inst.n]] == m["witness_starts"]
