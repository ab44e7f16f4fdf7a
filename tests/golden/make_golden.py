"""Write tests/golden/oracle_hashes.json: for each named workload, the sha256
of its seeded input and of the CPU oracle's canonical result, and -- where
the candidate rules are few enough for the pure-Python rule oracle -- of its
association rules at 50% confidence.  For the 4,096-database batch
("batched_4096") the input digest covers every database's input sha256 and
threshold, and the result digest every database's result sha256, in order.

Only the oracle computes these values (this script imports nothing from the
GPU path); the GPU tests compare against them when their own input has the
same sha256, and run the oracle live otherwise.

    python tests/golden/make_golden.py [workload ...]
"""
import hashlib
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


def batched_digests(dbs, minsups, results):
    """(input digest, result digest) of a batch: sha256 over the databases'
    input sha256 and threshold, and over their result sha256, in order."""
    hi, hr = hashlib.sha256(), hashlib.sha256()
    for c, ms, r in zip(dbs, minsups, results):
        hi.update(f"{c.sha256()}:{int(ms)};".encode())
        hr.update(f"{r}".encode() if isinstance(r, str) else r.sha256().encode())
    return hi.hexdigest(), hr.hexdigest()


def batched_entry():
    dbs = datagen.batched_dbs(datagen.batched_specs(4096))
    minsups = [datagen.minsup_from_ppm(c.n, 20_000) for c in dbs]
    t0 = time.time()
    res = [oracle.apriori(c.indptr, c.indices, c.m, ms) for c, ms in zip(dbs, minsups)]
    di, dr = batched_digests(dbs, minsups, res)
    return {"input_sha256": di, "minsup_ppm": 20_000, "n_db": len(dbs),
            "n_sets": int(sum(len(r) for r in res)), "max_len": int(max(r.max_level for r in res)),
            "result_sha256": dr, "oracle_seconds": round(time.time() - t0, 1)}


def main(names):
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    for name in names:
        if name == "batched_4096":
            data[name] = batched_entry()
            print(name, data[name], flush=True)
            continue
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
    main(sys.argv[1:] or ["grocery_like_10k_169", "quest_1M_1000", "planted_100k_2000",
                          "quest_10M_5000", "batched_4096"])
