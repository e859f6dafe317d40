"""Write tests/golden/pair_counts.json: exact connected-pair counts of the workloads.

Calls only the CPU oracle (oracle/) on the seeded inputs (paper_2501_18185_gb300/
workloads.py).  A "pair" is an ordered (I, J), I != J, both in the list, excitation
degree 1 or 2 (the off-diagonal Slater-Condon elements sigma evaluates, Sec. 2.3),
counted whether or not the element's value is zero.

    python tests/golden/make_golden.py [name ...]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import Oracle  # noqa: E402
from paper_2501_18185_gb300 import workloads as W  # noqa: E402

WORKLOADS = {
    "fci_8o_4a4b": lambda: W.fci_small_8o(),
    "sel_30o_10a10b_M2000000": lambda: W.selected_30o(),
    "sel_64s_14e_M1000000": lambda: W.selected_spinor_64(),
    "sel_30o_10a10b_M20000": lambda: W.selected_30o(M=60000),
}


def main(names):
    path = os.path.join(HERE, "pair_counts.json")
    data = json.load(open(path)) if os.path.exists(path) else {}
    for name in names:
        w = WORKLOADS[name]()
        t = time.time()
        o = Oracle.from_workload(w)
        pairs = o.count_pairs()
        data[w.name] = {"M": w.M, "pairs": pairs, "oracle_seconds": round(time.time() - t, 1),
                        "source": "oracle.Oracle.count_pairs (generation + binary search)"}
        print(w.name, data[w.name], flush=True)
        json.dump(data, open(path, "w"), indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(WORKLOADS))
