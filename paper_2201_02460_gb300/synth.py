"""Seeded synthetic case/control genotype data.

This module draws the inputs that every search runs on: a genotype matrix
G[n_snps][n_samples] with values in {0, 1, 2} (minor-allele count, the three
rows of a genotype table, Section 2.1) and a phenotype vector y[n_samples] with
1 = case and 0 = control.  It holds none of the search's arithmetic (no masks,
no counting, no scoring); both the CUDA library and the CPU oracle receive its
arrays as plain inputs.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based
generator: draw i of stream s is mix64(s + (i + 1) * 0x9E3779B97F4A7C15).
Every stream is a pure function of (seed, purpose, index), so the arrays are
identical on every machine and numpy version.

Recipe (the paper names no dataset; its evaluation only fixes n, m and the
order, Tables 2 and 3):
  * per-SNP minor-allele frequency p ~ U[maf_lo, maf_hi];
  * genotypes under Hardy-Weinberg: P(0) = (1-p)^2, P(1) = 2p(1-p), P(2) = p^2;
  * optionally q planted SNPs with p = 0.5 exactly and a parity penetrance
    P(case | g) = 0.5 + e if sum(g) is odd else 0.5 - e.  At p = 0.5 every
    proper subset of the planted SNPs carries no information about the parity,
    so no marginal or lower-order effect exists;
  * retrospective (case/control) sampling: individuals are drawn one after the
    other, each gets its phenotype from the penetrance, and is kept while its
    class quota (n_cases, n_controls) is not yet full.  Samples keep the order
    in which they were accepted, so cases and controls are interleaved.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# purpose tags for independent streams
_P_MAF = 1
_P_GENO = 2
_P_PLANT_POS = 3
_P_POOL_GENO = 4
_P_POOL_PHENO = 5
_P_BATCH = 6


def _mix64(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def stream_seed(seed: int, purpose: int, sub: int = 0) -> np.uint64:
    """Seed of an independent stream for (seed, purpose, sub)."""
    with np.errstate(over="ignore"):
        a = _mix64(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
        b = _mix64(np.array([a ^ np.uint64(purpose * 0x100000001B3 + sub)], dtype=np.uint64))[0]
    return b


def raw64(s: np.uint64, start: int, count: int) -> np.ndarray:
    """Draws start .. start+count-1 of the SplitMix64 stream with seed s."""
    idx = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(np.uint64(s) + idx * _GAMMA)


def uniform(s: np.uint64, start: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    return (raw64(s, start, count) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _hwe_genotypes(p: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Genotype from a uniform draw under Hardy-Weinberg, p = per-row MAF."""
    q = 1.0 - p
    t0 = q * q
    t1 = t0 + 2.0 * p * q
    return (u >= t0).astype(np.uint8) + (u >= t1).astype(np.uint8)


@dataclass
class Dataset:
    geno: np.ndarray          # uint8 [n_snps, n_samples], values 0/1/2
    pheno: np.ndarray         # uint8 [n_samples], 1 = case, 0 = control
    maf: np.ndarray           # float64 [n_snps]
    planted: tuple = ()       # sorted SNP indices of the planted interaction
    seed: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n_snps(self) -> int:
        return int(self.geno.shape[0])

    @property
    def n_samples(self) -> int:
        return int(self.geno.shape[1])

    @property
    def n_cases(self) -> int:
        return int(self.pheno.sum())


def make_dataset(n_snps: int, n_cases: int, n_controls: int, *, seed: int,
                 maf_lo: float = 0.05, maf_hi: float = 0.5,
                 plant_q: int = 0, plant_e: float = 0.0) -> Dataset:
    """Draw one case/control dataset (see the module docstring for the recipe)."""
    if n_snps < 0 or n_cases < 0 or n_controls < 0:
        raise ValueError("sizes must be non-negative")
    if plant_q > n_snps:
        raise ValueError("cannot plant more SNPs than exist")
    if not (0.0 <= plant_e <= 0.5):
        raise ValueError("penetrance offset must lie in [0, 0.5]")
    m = n_cases + n_controls
    maf = maf_lo + (maf_hi - maf_lo) * uniform(stream_seed(seed, _P_MAF), 0, n_snps)

    planted: tuple = ()
    if plant_q > 0:
        keys = raw64(stream_seed(seed, _P_PLANT_POS), 0, n_snps)
        planted = tuple(sorted(int(i) for i in np.argsort(keys, kind="stable")[:plant_q]))
        maf[list(planted)] = 0.5

    # retrospective sampling of individuals: only the planted SNPs influence
    # the phenotype, so only they have to be drawn for the candidate pool
    s_pg = stream_seed(seed, _P_POOL_GENO)
    s_pp = stream_seed(seed, _P_POOL_PHENO)
    pool_geno = []
    accepted_rows = []
    accepted_y = []
    need = {1: n_cases, 0: n_controls}
    drawn = 0
    chunk = max(64, 4 * m)
    while need[0] > 0 or need[1] > 0:
        if plant_q > 0:
            g = np.empty((plant_q, chunk), dtype=np.uint8)
            for t, snp in enumerate(planted):
                g[t] = _hwe_genotypes(np.full(chunk, 0.5),
                                      uniform(s_pg, (snp * (1 << 40)) + drawn, chunk))
            odd = (g.astype(np.int64).sum(axis=0) & 1).astype(bool)
            f = np.where(odd, 0.5 + plant_e, 0.5 - plant_e)
        else:
            g = np.empty((0, chunk), dtype=np.uint8)
            f = np.full(chunk, 0.5)
        y = (uniform(s_pp, drawn, chunk) < f).astype(np.uint8)
        # accept in draw order while the class quota lasts
        for cls in (1, 0):
            idx = np.nonzero(y == cls)[0][: need[cls]]
            need[cls] -= len(idx)
            if len(idx):
                accepted_rows.append(drawn + idx)
                accepted_y.append(np.full(len(idx), cls, dtype=np.uint8))
        pool_geno.append(g)
        drawn += chunk
    if m:
        order_idx = np.concatenate(accepted_rows)
        yy = np.concatenate(accepted_y)
        perm = np.argsort(order_idx, kind="stable")
        order_idx = order_idx[perm]
        pheno = yy[perm]
        pool = np.concatenate(pool_geno, axis=1) if pool_geno else np.empty((0, 0), np.uint8)
    else:
        order_idx = np.empty(0, dtype=np.int64)
        pheno = np.empty(0, dtype=np.uint8)
        pool = np.empty((plant_q, 0), np.uint8)

    geno = np.empty((n_snps, m), dtype=np.uint8)
    s_g = stream_seed(seed, _P_GENO)
    for j in range(n_snps):
        geno[j] = _hwe_genotypes(np.full(m, maf[j]), uniform(s_g, j * m, m))
    for t, snp in enumerate(planted):
        geno[snp] = pool[t, order_idx]
    return Dataset(geno=geno, pheno=pheno, maf=maf, planted=planted, seed=seed,
                   meta=dict(n_snps=n_snps, n_cases=n_cases, n_controls=n_controls,
                             maf_lo=maf_lo, maf_hi=maf_hi, plant_q=plant_q, plant_e=plant_e))


# ---------------------------------------------------------------------------
# Named workloads.  Sizes follow the evaluated configurations; seeds are
# 2201024600 + configuration number.
# ---------------------------------------------------------------------------
BASE_SEED = 2201024600

WORKLOADS = {
    # order-2 search, 200 SNPs x 1600 samples, one planted XOR-like pair
    "order2_200snp_1600": dict(n_snps=200, n_cases=800, n_controls=800, maf_lo=0.05,
                               plant_q=2, plant_e=0.25, order=2, top_n=10, seed=BASE_SEED + 1),
    # order-3 search, 2000 SNPs x 4000 samples, one planted 3-way parity table
    "order3_2000snp_4000": dict(n_snps=2000, n_cases=2000, n_controls=2000, maf_lo=0.05,
                                plant_q=3, plant_e=0.3, order=3, top_n=100, seed=BASE_SEED + 2),
    # order-4 search, 500 SNPs x 8192 samples, no plant
    "order4_500snp_8192": dict(n_snps=500, n_cases=4096, n_controls=4096, maf_lo=0.1,
                               plant_q=0, plant_e=0.0, order=4, top_n=100, seed=BASE_SEED + 3),
    # order-8 search, 23 SNPs x 2048 samples (the order-8 row of Table 2), no plant
    "order8_23snp_2048": dict(n_snps=23, n_cases=1024, n_controls=1024, maf_lo=0.05,
                              plant_q=0, plant_e=0.0, order=8, top_n=100, seed=BASE_SEED + 8),
}


def make_workload(name: str, **overrides) -> tuple[Dataset, int, int]:
    """Dataset, order and top-N of a named workload (overrides e.g. n_snps)."""
    cfg = dict(WORKLOADS[name])
    cfg.update(overrides)
    order = cfg.pop("order")
    top_n = cfg.pop("top_n")
    return make_dataset(**cfg), order, top_n


def batch_specs(count: int = 64, seed: int = BASE_SEED + 4) -> list[dict]:
    """Shapes of the heterogeneous batch: n ~ U{100..1000}, m ~ U{1000..16000},
    case fraction ~ U[0.3, 0.7], order ~ U{2, 3, 4}; dataset d uses seed + 1000 d."""
    s = stream_seed(seed, _P_BATCH)
    u = uniform(s, 0, 4 * count).reshape(count, 4)
    specs = []
    for d in range(count):
        n = 100 + int(u[d, 0] * 901)
        m = 1000 + int(u[d, 1] * 15001)
        frac = 0.3 + 0.4 * u[d, 2]
        m1 = int(round(m * frac))
        order = 2 + int(u[d, 3] * 3)
        specs.append(dict(n_snps=n, n_cases=m1, n_controls=m - m1, order=order,
                          top_n=20, seed=seed + 1000 * d, maf_lo=0.05))
    return specs
