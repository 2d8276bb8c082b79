"""Seeded input generators of the Table 2 families (no GPU): well-formed Ising instances
(symmetric int8 couplings, zero diagonal), the structure each family promises, the
planted optimum of nae_3_sat against exhaustive enumeration, and the stored exhaustive
optima of the TTS study against a fresh enumeration on a sample."""
import json
import os

import numpy as np
import pytest

import oracle as o
from conftest import GOLDEN
from paper_2407_10205_gb300 import instances as ins


@pytest.mark.parametrize("family", sorted(ins.FAMILIES))
@pytest.mark.parametrize("n", [8, 16, 64])
def test_family_instances_are_well_formed(family, n):
    d = ins.family_instance(family, n, 5)
    assert d.k.dtype == np.int8 and d.k.shape == (n, n) and d.kh.shape == (n,)
    assert np.array_equal(d.k, d.k.T) and not np.diag(d.k).any()
    nz = d.k[np.triu_indices(n, 1)]
    if family in ("maxcut_dense", "maxcut_d3", "sk_bool"):
        assert set(np.unique(nz)) <= {-1, 0} and not d.kh.any() and d.frac_bits == 0
    if family == "sk_ising":
        assert set(np.unique(nz)) == {-1, 1} and not d.kh.any()
    if family == "maxcut_d3":
        assert (np.count_nonzero(d.k, axis=1) == 3).all()
    if family == "sk_uniform":
        assert nz.max() <= 0 and nz.min() >= -127 and d.frac_bits == 7 and not d.kh.any()
        assert 0.3 < np.mean(nz != 0) < 0.7
    if family == "spin_model":
        assert d.frac_bits == 7 and np.abs(d.kh).max() <= 127 and nz.min() < 0 < nz.max()


@pytest.mark.parametrize("n,seed", [(6, 1), (9, 2), (12, 3), (14, 4)])
def test_planted_nae_3_sat_optimum_is_exact(n, seed):
    d = ins.nae_3_sat(n, seed)
    P = o.Instance(d.kh, k=d.k)
    e, _, _ = o.brute_force(P)
    assert e == d.optimum_k == -int(round(2.1 * n))


def test_stored_tts_optima_match_enumeration():
    with open(os.path.join(GOLDEN, "tts_optima.json")) as f:
        doc = json.load(f)
    import importlib.util
    spec = importlib.util.spec_from_file_location("mk", os.path.join(GOLDEN, "make_tts_optima.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    for fam in sorted(ins.FAMILIES):
        for n in (8, 16):
            vals = doc["optima"][f"{fam}/{n}"]
            assert len(vals) == doc["instances"] == 100
            for k in (0, 37, 99):
                d = ins.family_instance(fam, n, mk.tts_seed(fam, n, k))
                assert o.brute_force(o.Instance(d.kh, k=d.k, frac_bits=d.frac_bits))[0] == vals[k]
