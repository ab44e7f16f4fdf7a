"""Write tests/golden/oracle_hashes.json: for each named workload, the sha256
of its seeded input and of the CPU oracle's canonical result, and -- where
the candidate rules are few enough for the pure-Python rule oracle -- of its
association rules at 50% confidence.

Only the oracle computes these values (this script imports nothing from the
GPU path); the GPU tests compare against them when their own input has the
same sha256, and run the oracle live otherwise.

    python tests/golden/make_golden.py [workload ...]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from oracle import rules as orules  # noqa: E402
from paper_2412_19420_gb300 import datagen  # noqa: E402

RULES_PPM = 500_000
RULES_MAX_CANDIDATES = 5_000_000

OUT = os.path.join(HERE, "oracle_hashes.json")


def main(names):
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    for name in names:
        gen, minsup = datagen.WORKLOADS[name]
        c = gen()
        t0 = time.time()
        r = oracle.apriori(c.indptr, c.indices, c.m, minsup)
        data[name] = {"input_sha256": c.sha256(), "minsup": minsup, "n_sets": len(r),
                      "max_len": r.max_level, "result_sha256": r.sha256(),
                      "oracle_seconds": round(time.time() - t0, 1)}
        L = np.diff(r.offsets.astype(np.int64))
        cand = int(((np.int64(1) << L[(L >= 2) & (L <= 20)]) - 2).sum())
        if cand <= RULES_MAX_CANDIDATES:
            rules = orules.rules(r, c.n, RULES_PPM)
            data[name]["rules_min_conf_ppm"] = RULES_PPM
            data[name]["n_rules"] = len(rules)
            data[name]["rules_sha256"] = rules.sha256()
        print(name, data[name], flush=True)
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["grocery_like_10k_169", "quest_1M_1000", "planted_100k_2000"])
