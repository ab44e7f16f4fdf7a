"""The paper's Table 1 / Table 2 columns for a mine on this library: the
number of frequent itemsets, their average support as a percentage of the
transactions (Table 2), and the device memory the miner held (Table 1's
memory column).  Host arithmetic on fetched results and fim_get_stats; no
mining happens here."""
from __future__ import annotations

import numpy as np


def table_columns(supports, n_trans: int, stats: dict) -> dict:
    """supports: the fetched supports (numpy or torch, any device); n_trans:
    the database's transactions; stats: fim_get_stats after the mine."""
    if hasattr(supports, "detach"):
        total = int(supports.detach().to("cpu").numpy().astype(np.int64).sum())
    else:
        total = int(np.asarray(supports, dtype=np.int64).sum())
    k = int(len(supports))
    avg = 100.0 * total / k / max(1, int(n_trans)) if k else 0.0
    return {"frequent_itemsets": k, "avg_support_pct": avg,
            "peak_device_mib": stats["peak_device_bytes"] / 2**20}
