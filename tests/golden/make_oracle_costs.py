"""Write tests/golden/oracle_costs.txt: the CPU oracle's optimal costs of the
large named workloads, too slow to recompute inside a test run.

Calls only ``oracle`` and the seeded input generators; run from the
repository root:  python tests/golden/make_oracle_costs.py [name ...]
Each line: <name> <cost> <algorithm> <seconds> (single thread, this host).
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2005_01182_gb300 import workloads as W  # noqa: E402

CASES = {
    "single_4096_circle_square": lambda: W.single_4096("circle-square"),
    "single_4096_circle_triangle": lambda: W.single_4096("circle-triangle"),
    "single_4096_uniform": lambda: W.single_4096("uniform"),
    "single_16384_grid": W.single_16384,
}


def main(names):
    path = os.path.join(HERE, "oracle_costs.txt")
    have = {}
    if os.path.exists(path):
        for line in open(path):
            if line.strip() and not line.startswith("#"):
                have[line.split()[0]] = line.rstrip("\n")
    for name in names or list(CASES):
        C = CASES[name]()
        t0 = time.perf_counter()
        _, cost, _, _ = oracle.km(C)
        have[name] = f"{name} {cost} oracle_km {time.perf_counter() - t0:.1f}"
        print(have[name], flush=True)
        with open(path, "w") as f:
            f.write("# Optimal costs of the named workloads from the CPU oracle (KM, exact;\n"
                    "# its optimality is pinned in tests/test_oracle.py), written by\n"
                    "# tests/golden/make_oracle_costs.py.  Columns: name cost algorithm seconds.\n")
            for k in CASES:
                if k in have:
                    f.write(have[k] + "\n")


if __name__ == "__main__":
    main(sys.argv[1:])
