"""Host-side schedule heuristic (not from the paper): the field scale it uses and the
shape of the schedule it suggests (CPU only)."""
import math

import numpy as np
import pytest

from paper_2407_10205_gb300 import instances as ins
from paper_2407_10205_gb300 import schedules


def test_field_scale_sk_closed_form():
    # J in {-1,+1}, complete graph: rms(k) = 1, n - 1 couplings per spin
    for n in (16, 100, 512):
        d = ins.sk_pm1(n, 3)
        assert schedules.field_scale(d) == pytest.approx(math.sqrt(n - 1))


def test_field_scale_same_for_dense_and_csr_forms():
    c = ins.erdos_renyi(200, 0.05, 127, 31, 4, seed=6)
    k = np.zeros((c.n, c.n), dtype=np.int8)
    for i in range(c.n):
        for p in range(c.row_ptr[i], c.row_ptr[i + 1]):
            k[i, c.col[p]] = c.val[p]
    class Dense:
        pass
    dense = Dense()
    dense.k, dense.kh, dense.frac_bits = k, c.kh, c.frac_bits
    if np.count_nonzero(c.val) == len(c.val):      # no stored zeros: the two forms agree
        assert schedules.field_scale(dense) == pytest.approx(schedules.field_scale(c))
    # fixed point: the scale carries q = 2^-f
    dense.frac_bits = 0
    assert schedules.field_scale(dense) == pytest.approx(16 * schedules.field_scale(c), rel=1e-2)


def test_suggested_schedule_shape():
    d = ins.sk_pm1(64, 1)
    b0, b1, eps, gamma, refresh = schedules.suggest_schedule(d)
    assert b1 == pytest.approx(6.0 / math.sqrt(63)) and b0 == pytest.approx(b1 / 20)
    assert (eps, gamma, refresh) == (0.1, 2.0, 50)
    b0j, b1j, *_ = schedules.suggest_schedule(d, jump=12.0)
    assert b1j == pytest.approx(2 * b1)
