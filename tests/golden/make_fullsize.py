"""Writes the oracle's top-N of the full-size named workloads to text files.

The expected values of the full-size parity tests come from the CPU oracle
alone (exhaustive search, Section 2.4 / Algorithm 1, MI in double precision by
Eq. 1-3) run on the seeded synthetic dataset of each workload; nothing here
touches the CUDA library.  Each file records a fingerprint of the dataset
(SHA-256 of the genotype and phenotype bytes) so that a test can tell a
changed generator from a changed search.

    python tests/golden/make_fullsize.py order3_2000snp_4000 [order4_500snp_8192 ...]

Format: '#'-prefixed header lines (workload, order, top_n, sizes, sha256,
oracle seconds), then one line per record: rank-in-top, the k SNP indices,
the MI as a float64 hex string, then the 2 x 3^k counts (cases, then controls).
"""
from __future__ import annotations

import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2201_02460_gb300 import synth  # noqa: E402


def fingerprint(geno: np.ndarray, pheno: np.ndarray) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(geno, dtype=np.uint8).tobytes())
    h.update(np.ascontiguousarray(pheno, dtype=np.uint8).tobytes())
    return h.hexdigest()


def path_of(name: str) -> str:
    return os.path.join(HERE, f"{name}_top.txt")


def write(name: str) -> str:
    d, k, top_n = synth.make_workload(name)
    t0 = time.time()
    combs, mi, counts = O.search(d.geno, d.pheno, k, top_n)
    secs = time.time() - t0
    out = path_of(name)
    with open(out, "w") as f:
        f.write(f"# workload {name}\n# order {k}\n# top_n {top_n}\n")
        f.write(f"# n_snps {d.n_snps}\n# n_samples {d.n_samples}\n# n_cases {d.n_cases}\n")
        f.write(f"# sha256 {fingerprint(d.geno, d.pheno)}\n")
        f.write(f"# oracle_seconds {secs:.1f} threads {O.max_threads()}\n")
        for i in range(len(mi)):
            cells = " ".join(str(int(x)) for x in counts[i].reshape(-1))
            snps = " ".join(str(int(x)) for x in combs[i])
            f.write(f"{i} {snps} {float(mi[i]).hex()} {cells}\n")
    return out


def read(name: str) -> dict:
    """The stored top-N: dict(order, top_n, sha256, combs [r, k], mi [r],
    counts [r, 2, 3^k])."""
    meta = {}
    rows = []
    with open(path_of(name)) as f:
        for line in f:
            if line.startswith("#"):
                parts = line[1:].split()
                meta[parts[0]] = parts[1]
                continue
            rows.append(line.split())
    k = int(meta["order"])
    combs = np.array([[int(x) for x in r[1:1 + k]] for r in rows], dtype=np.int64)
    mi = np.array([float.fromhex(r[1 + k]) for r in rows], dtype=np.float64)
    counts = np.array([[int(x) for x in r[2 + k:]] for r in rows], dtype=np.uint32).reshape(len(rows), 2, 3 ** k)
    return dict(order=k, top_n=int(meta["top_n"]), sha256=meta["sha256"], combs=combs, mi=mi, counts=counts)


if __name__ == "__main__":
    for nm in sys.argv[1:]:
        print(write(nm))
