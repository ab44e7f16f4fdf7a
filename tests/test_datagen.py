"""The seeded input generators are deterministic: each named workload
regenerates the CSR whose sha256 tests/golden/oracle_hashes.json records
(the oracle's stored results refer to exactly these inputs)."""
import json
import os

import pytest

from paper_2412_19420_gb300 import datagen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_hashes.json")


@pytest.mark.parametrize("name", ["grocery_like_10k_169", "quest_1M_1000", "planted_100k_2000"])
def test_workload_inputs_are_reproducible(name):
    with open(GOLDEN) as f:
        g = json.load(f)[name]
    gen, minsup = datagen.WORKLOADS[name]
    c = gen()
    assert minsup == g["minsup"]
    assert c.sha256() == g["input_sha256"]
    # well-formed CSR: indptr starts at 0, never decreases, items in range
    assert int(c.indptr[0]) == 0 and (c.indptr[1:] >= c.indptr[:-1]).all()
    assert int(c.indptr[-1]) == c.indices.shape[0]
    assert c.indices.min() >= 0 and c.indices.max() < c.m
