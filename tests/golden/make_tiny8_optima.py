"""Writes tiny8_sgs_optima.json: the minimum makespan of the 8-task,
1-resource scheduling family (seeds 0..99) by brute-force serial schedule
generation over every precedence-feasible task list (oracle.brute).  Calls
only oracle/ and synthetic/."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import brute  # noqa: E402
from synthetic import config_instance  # noqa: E402


def main():
    optima = [brute.rcpsp_optimum_sgs(config_instance("tiny8", s)) for s in range(100)]
    out = {
        "what": "minimum makespan, 8 tasks, durations U[1,5], 1 resource capacity 4, "
                "demands U[1,3], precedence edge probability 0.2, seeds 0..99",
        "how": "serial schedule generation over all precedence-feasible task lists "
               "(active schedules contain an optimum; Kolisch 1996)",
        "writer": "tests/golden/make_tiny8_optima.py",
        "optima": optima,
    }
    with open(os.path.join(HERE, "tiny8_sgs_optima.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
