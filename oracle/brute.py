"""Per-individual brute-force contingency counting (test infrastructure only).

An independent second way to obtain the 3^k x 2 tables: no bit masks, no
words, no prefix reuse.  Each individual i falls in cell
x(i) = sum_t G[s_t][i] * 3^(k-1-t) (first SNP most significant, the row
order of a combined genotype table, Section 2.1) and is counted in the case
column when y_i = 1, the control column otherwise.  Used only on tiny inputs
to pin the C oracle.
"""
from __future__ import annotations

import itertools

import numpy as np


def table(geno: np.ndarray, pheno: np.ndarray, comb) -> np.ndarray:
    k = len(comb)
    cells = 3 ** k
    out = np.zeros((2, cells), dtype=np.int64)
    for i in range(geno.shape[1]):
        x = 0
        for s in comb:
            x = 3 * x + int(geno[s, i])
        out[0 if pheno[i] == 1 else 1, x] += 1
    return out


def all_combinations(n: int, k: int):
    return list(itertools.combinations(range(n), k))
