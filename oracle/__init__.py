"""CPU oracle of the exhaustive k-SNP mutual-information search.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg are the only callers.  The product library never imports this
package and this package never imports the product library.

`epi_oracle.c` is the plain C search (genotype tables, Section 2.1; fused
last-level count, Section 2.2; MI in double precision, Section 2.3, Eq. 1-3;
exhaustive enumeration with prefix reuse, Section 2.4, Algorithm 1).
`brute.py` is a second, independent per-individual counter used to pin it.
`mlp.py` is a float64 reference of the proposer network (forward, analytic
backward, AdamW step) used to pin the GPU training kernels.
"""
from .oracle import (binom, build, genotype_table, max_threads, mi, rank, search,  # noqa: F401
                     tables, unrank)
