"""ctypes binding of the C oracle (test infrastructure only).

Builds `epi_oracle.c` with the host C compiler on first use.  Every function
validates its numpy inputs and returns numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "epi_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libepi_oracle.so")
_lock = threading.Lock()
_lib = None

MAX_K = 8


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-Wall", "-Wno-unused-variable",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            i64, u64, i32 = C.c_int64, C.c_uint64, C.c_int
            lib.eo_binom.restype = u64
            lib.eo_binom.argtypes = [i64, i64]
            lib.eo_unrank.restype = i32
            lib.eo_unrank.argtypes = [i64, i32, u64, P]
            lib.eo_rank.restype = u64
            lib.eo_rank.argtypes = [i64, i32, P]
            lib.eo_mi.restype = C.c_double
            lib.eo_mi.argtypes = [P, P, i64, i64]
            lib.eo_genotype_table.restype = i32
            lib.eo_genotype_table.argtypes = [P, P, i64, i64, i32, P, P, P]
            lib.eo_tables.restype = i32
            lib.eo_tables.argtypes = [P, P, i64, i64, i32, P, i64, P]
            lib.eo_search.restype = i32
            lib.eo_search.argtypes = [P, P, i64, i64, i32, i64, u64, u64, i32, P, P, P, P]
            lib.eo_max_threads.restype = i32
            lib.eo_max_threads.argtypes = []
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _inputs(geno, pheno):
    geno = np.ascontiguousarray(geno, dtype=np.uint8)
    pheno = np.ascontiguousarray(pheno, dtype=np.uint8)
    if geno.ndim != 2 or pheno.ndim != 1 or geno.shape[1] != pheno.shape[0]:
        raise ValueError("geno must be [n_snps, n_samples] and pheno [n_samples]")
    return geno, pheno


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


def binom(n: int, k: int) -> int:
    return int(_load().eo_binom(n, k))


def unrank(n: int, k: int, r: int) -> tuple:
    out = np.zeros(k, dtype=np.int32)
    _check(_load().eo_unrank(n, k, r, _ptr(out)), "unrank")
    return tuple(int(x) for x in out)


def rank(n: int, k: int, comb) -> int:
    c = np.ascontiguousarray(comb, dtype=np.int32)
    return int(_load().eo_rank(n, k, _ptr(c)))


def mi(ct_case, ct_ctrl, m: int) -> float:
    a = np.ascontiguousarray(ct_case, dtype=np.uint32)
    b = np.ascontiguousarray(ct_ctrl, dtype=np.uint32)
    return float(_load().eo_mi(_ptr(a), _ptr(b), a.size, m))


def genotype_table(geno, pheno, comb):
    """Genotype table of one combination: (case rows, control rows), each a
    uint64 array [3^k, words] with individual 64 w + b at bit b of word w."""
    geno, pheno = _inputs(geno, pheno)
    k = len(comb)
    c = np.ascontiguousarray(comb, dtype=np.int32)
    n, m = geno.shape
    m1 = int(pheno.sum())
    w = (m1 + 63) // 64 + (m - m1 + 63) // 64
    out = np.zeros((3 ** k, max(w, 1)), dtype=np.uint64)
    wo = np.zeros(2, dtype=np.int64)
    _check(_load().eo_genotype_table(_ptr(geno), _ptr(pheno), n, m, k, _ptr(c), _ptr(out), _ptr(wo)),
           "genotype_table")
    return out[:, : wo[0]], out[:, wo[0]: wo[0] + wo[1]]


def tables(geno, pheno, combs) -> np.ndarray:
    """Contingency tables [count, 2, 3^k] (0 = cases, 1 = controls)."""
    geno, pheno = _inputs(geno, pheno)
    combs = np.ascontiguousarray(combs, dtype=np.int32)
    if combs.ndim != 2:
        raise ValueError("combs must be [count, k]")
    count, k = combs.shape
    out = np.zeros((count, 2, 3 ** k), dtype=np.uint32)
    n, m = geno.shape
    _check(_load().eo_tables(_ptr(geno), _ptr(pheno), n, m, k, _ptr(combs), count, _ptr(out)), "tables")
    return out


def search(geno, pheno, k: int, top_n: int, rank_begin: int = 0, rank_end: int | None = None,
           threads: int = 0, with_counts: bool = True):
    """Exhaustive search over lexicographic ranks [rank_begin, rank_end):
    returns (combs [r, k] int32, mi [r] float64, counts [r, 2, 3^k] or None)."""
    geno, pheno = _inputs(geno, pheno)
    n, m = geno.shape
    if rank_end is None:
        rank_end = (1 << 64) - 1
    combs = np.zeros((top_n, k), dtype=np.int32)
    mis = np.zeros(top_n, dtype=np.float64)
    counts = np.zeros((top_n, 2, 3 ** k), dtype=np.uint32) if with_counts else None
    n_out = np.zeros(1, dtype=np.int64)
    rc = _load().eo_search(_ptr(geno), _ptr(pheno), n, m, k, top_n, rank_begin, rank_end, threads,
                           _ptr(combs), _ptr(mis), _ptr(counts) if with_counts else None, _ptr(n_out))
    _check(rc, "search")
    r = int(n_out[0])
    return combs[:r], mis[:r], (counts[:r] if with_counts else None)


def max_threads() -> int:
    return int(_load().eo_max_threads())
