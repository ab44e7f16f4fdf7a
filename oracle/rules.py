"""Association rules from frequent itemsets -- TEST INFRASTRUCTURE (oracle).

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this module; the product path never does.

Section IV.A names confidence and lift, beside support, as the measures the
mined itemsets are evaluated with, and prints no formula for them.  The
definitions here are the textbook ones (confidence: Agrawal, Imielinski and
Swami, 1993; lift, called "interest" there: Brin, Motwani, Ullman and Tsur,
1997).  For a frequent set Z, a nonempty proper subset X of Z and Y = Z \\ X:

    conf(X -> Y) = S(Z) / S(X)
    lift(X -> Y) = conf(X -> Y) / (S(Y) / n) = S(Z) * n / (S(X) * S(Y))

with S the supports of Eq. 3 and n the number of transactions.

Output convention (the library's): rules are listed set by set in the
canonical order of the itemsets (size, then items lexicographic), and inside
a set by antecedent mask ascending, where bit i of the mask says that the i-th
item of Z (items ascending) belongs to X.  A rule is kept when
S(Z) * 10^6 >= min_conf_ppm * S(X), decided in integers.  conf is the double
S(Z) / S(X); lift is the double quotient of the two exact integer products
S(Z) * n and S(X) * S(Y), each rounded once to double.  Sets longer than
max_len give no rules.

Parity status: pinned in tests/test_oracle_rules.py by brute force from the
transactions (supports recounted by scanning, independently of the itemset
list) and by closed forms (a database of all 2^m subsets, where every rule has
conf 2^-|Y| and lift 1; an all-ones database; disjoint co-occurring blocks).
"""
from __future__ import annotations

import dataclasses

import numpy as np

RULES_MAX_LEN = 20


@dataclasses.dataclass
class Rules:
    set_index: np.ndarray  # uint64[N]: index of Z among the itemsets
    ante_mask: np.ndarray  # uint32[N]: bit i = i-th item of Z is in X
    conf: np.ndarray       # float64[N]
    lift: np.ndarray       # float64[N]

    def __len__(self) -> int:
        return int(self.set_index.shape[0])

    def canonical_bytes(self) -> bytes:
        """Byte stream for bit-exact comparison: set indices, masks, conf, lift."""
        return (np.ascontiguousarray(self.set_index, dtype="<u8").tobytes()
                + np.ascontiguousarray(self.ante_mask, dtype="<u4").tobytes()
                + np.ascontiguousarray(self.conf, dtype="<f8").tobytes()
                + np.ascontiguousarray(self.lift, dtype="<f8").tobytes())

    def sha256(self) -> str:
        import hashlib
        return hashlib.sha256(self.canonical_bytes()).hexdigest()


def rule_of(z_items, z_sup: int, mask: int, support_of, n: int, min_conf_ppm: int,
            _mutant: int = 0):
    """(keep, conf, lift) of the rule X -> Z \\ X picked by ``mask``.

    ``support_of`` maps an ascending item tuple to its support.  ``_mutant`` > 0
    plants one mistake (only the tests that check the pins ask for it):
    1 divides by S(Y) in conf, 2 drops n from lift, 3 reads the mask from the
    last item, 4 keeps a rule only above the threshold, 5 uses S(X) for S(Y)
    in lift."""
    L = len(z_items)
    bit = (lambda i: (mask >> (L - 1 - i)) & 1) if _mutant == 3 else (lambda i: (mask >> i) & 1)
    x = tuple(v for i, v in enumerate(z_items) if bit(i))
    y = tuple(v for i, v in enumerate(z_items) if not bit(i))
    s_z, s_x, s_y = int(z_sup), int(support_of[x]), int(support_of[y])
    if _mutant == 5:
        s_y = s_x
    keep = s_z * 1_000_000 >= int(min_conf_ppm) * s_x
    if _mutant == 4:
        keep = s_z * 1_000_000 > int(min_conf_ppm) * s_x
    conf = float(s_z) / float(s_y if _mutant == 1 else s_x)
    lift = float(s_z * (1 if _mutant == 2 else int(n))) / float(s_x * s_y)
    return keep, conf, lift


def rules(itemsets, n_trans: int, min_conf_ppm: int, max_len: int = 0, _mutant: int = 0) -> Rules:
    """Every kept rule of the canonical ``itemsets`` (offsets, items, supports),
    in the output convention above."""
    if not 0 <= int(min_conf_ppm) <= 1_000_000:
        raise ValueError("min_conf_ppm must lie in [0, 10^6]")
    max_len = RULES_MAX_LEN if max_len == 0 else int(max_len)
    if not 2 <= max_len <= RULES_MAX_LEN:
        raise ValueError("max_len must be 0 or lie in [2, 20]")
    off, items, sup = itemsets.offsets, itemsets.items, itemsets.supports
    support_of = {}
    for q in range(len(sup)):
        support_of[tuple(int(v) for v in items[off[q]:off[q + 1]])] = int(sup[q])
    si, am, cf, lf = [], [], [], []
    for q in range(len(sup)):
        z = tuple(int(v) for v in items[off[q]:off[q + 1]])
        L = len(z)
        if L < 2 or L > max_len:
            continue
        for mask in range(1, (1 << L) - 1):
            keep, conf, lift = rule_of(z, sup[q], mask, support_of, n_trans, min_conf_ppm, _mutant)
            if keep:
                si.append(q)
                am.append(mask)
                cf.append(conf)
                lf.append(lift)
    return Rules(np.asarray(si, np.uint64), np.asarray(am, np.uint32),
                 np.asarray(cf, np.float64), np.asarray(lf, np.float64))
