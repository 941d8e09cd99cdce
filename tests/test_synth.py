"""The seeded input generator: determinism, class quotas, HWE frequencies and
the zero-marginal property of the planted parity penetrance."""
import numpy as np
import pytest

from paper_2201_02460_gb300 import synth


def test_splitmix64_reference_values():
    # SplitMix64 with seed 0: the first outputs of the published generator
    s = np.uint64(0)
    got = synth.raw64(s, 0, 3).tolist()
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_deterministic_and_quota():
    a = synth.make_dataset(50, 37, 41, seed=9, plant_q=2, plant_e=0.25)
    b = synth.make_dataset(50, 37, 41, seed=9, plant_q=2, plant_e=0.25)
    assert (a.geno == b.geno).all() and (a.pheno == b.pheno).all()
    assert a.pheno.sum() == 37 and (a.pheno == 0).sum() == 41
    assert a.geno.max() <= 2 and a.geno.dtype == np.uint8
    c = synth.make_dataset(50, 37, 41, seed=10, plant_q=2, plant_e=0.25)
    assert (a.geno != c.geno).any()
    # cases and controls are interleaved in acceptance order
    assert 0 < np.argmin(a.pheno) < 78 or 0 < np.argmax(a.pheno) < 78


def test_hwe_frequencies():
    d = synth.make_dataset(40, 5000, 5000, seed=3, maf_lo=0.2, maf_hi=0.4)
    for j in range(40):
        p = d.maf[j]
        f = np.bincount(d.geno[j], minlength=3) / d.n_samples
        want = np.array([(1 - p) ** 2, 2 * p * (1 - p), p * p])
        assert np.abs(f - want).max() < 0.02


def test_planted_parity_has_no_marginal_effect():
    d = synth.make_dataset(10, 20000, 20000, seed=4, plant_q=3, plant_e=0.3)
    case = d.pheno == 1
    for s in d.planted:
        f1 = np.bincount(d.geno[s][case], minlength=3) / case.sum()
        f0 = np.bincount(d.geno[s][~case], minlength=3) / (~case).sum()
        assert np.abs(f1 - f0).max() < 0.02
    par = d.geno[list(d.planted)].astype(int).sum(axis=0) & 1
    # strong effect of the joint parity
    assert par[case].mean() - par[~case].mean() > 0.4


@pytest.mark.parametrize("name", list(synth.WORKLOADS))
def test_workload_shapes(name):
    cfg = synth.WORKLOADS[name]
    if cfg["n_snps"] * (cfg["n_cases"] + cfg["n_controls"]) > 5_000_000:
        d, k, n = synth.make_workload(name, n_snps=20)
    else:
        d, k, n = synth.make_workload(name)
    assert d.n_cases == cfg["n_cases"]
    assert d.n_samples == cfg["n_cases"] + cfg["n_controls"]


def test_batch_specs():
    specs = synth.batch_specs()
    assert len(specs) == 64
    for s in specs:
        assert 100 <= s["n_snps"] <= 1000
        m = s["n_cases"] + s["n_controls"]
        assert 1000 <= m <= 16000
        assert 0.29 <= s["n_cases"] / m <= 0.71
        assert s["order"] in (2, 3, 4)
    assert synth.batch_specs() == specs
