"""Batches of many instances of uneven N (phia_batch_*): small dense members run on the
resident tcgen05 kernel over a table of CTAs (all iterations in one launch per operand
and tile-count group), the others on the CSR path in one persistent cooperative launch
(or one launch per iteration).  Each instance's result must not depend on the batch or
on the launch form: every member equals the same instance run alone, bit for bit, and
its returned energies equal Eq. 2 (oracle) on its returned spins."""
import numpy as np
import pytest

import oracle as o
from paper_2407_10205_gb300 import instances as ins

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

R, T = 64, 90


def _sched(phia):
    return phia.schedule(0.01, 0.25, 0.1, 2.0, refresh=20)


def _mixed():
    """Small dense members of each (operand, spin-tile) group -- e4m3 with 1, 2 and 3 tiles,
    bf16 with 1 and 2 -- a dense member too large for the resident kernel (run as CSR) and
    two sparse members."""
    return [ins.dense_int(50, 7, 7, seed=1), ins.sk_pm1(130, 2), ins.dense_int(260, 16, 31, seed=3),
            ins.dense_int(100, 100, 50, seed=4), ins.dense_int(200, 127, 9, seed=5), ins.sk_pm1(450, 6),
            ins.erdos_renyi(300, 0.05, 127, 31, 4, seed=7), ins.erdos_renyi(90, 0.2, 127, 31, 4, seed=8),
            ins.dense_int(33, 7, 7, seed=9, frac_bits=3)]


@pytest.mark.parametrize("csr_mode", [1, 2])
def test_dense_members_equal_the_resident_kernel_alone(gpu_lib, csr_mode):
    """csr_mode 1: the CSR part in one persistent launch; 2: one launch per iteration."""
    phia = gpu_lib
    insts = _mixed()
    ids = [40 + k for k in range(len(insts))]
    sched = _sched(phia)
    with phia.Batch(insts, instance_ids=ids, csr_mode=csr_mode) as B:
        B.anneal(sched, R, T, seed=11)
        mix = [B.replica_results(k, R) for k in range(len(insts))]
        st = B.stats()
    assert st.spin_updates == R * T * sum(c.n for c in insts)
    for k, c in enumerate(insts):
        if getattr(c, "k", None) is not None and c.n <= 260:
            # the same instance alone on the resident kernel: 8 replicas per CTA, J in shared memory
            with phia.Annealer(c.k, c.kh, frac_bits=c.frac_bits, path=phia.PATH_TC, tc_kernel=phia.KERNEL_RESIDENT,
                               tile_replicas=8, coupling_mem=phia.MEM_SHARED, instance_id=ids[k]) as A:
                A.anneal(sched, R, T, seed=11)
                alone = phia.replica_results(A.h, R, c.n)
        else:
            with phia.Batch([c], instance_ids=[ids[k]]) as A:
                A.anneal(sched, R, T, seed=11)
                alone = A.replica_results(0, R)
        for u, w in zip(mix[k], alone):
            assert np.array_equal(u, w), f"instance {k} (N = {c.n}) differs alone and in the batch"
        if getattr(c, "k", None) is not None:
            P = o.Instance(c.kh, k=c.k, frac_bits=c.frac_bits)
        else:
            P = o.Instance(c.kh, row_ptr=c.row_ptr, col=c.col, val=c.val, frac_bits=c.frac_bits)
        S = phia.unpack_bits(mix[k][3], c.n)
        for r in range(0, R, 9):
            assert o.energy_exact(P, S[r]) == mix[k][0][r]


def test_persistent_and_per_iteration_csr_launches_agree(gpu_lib):
    """The CSR part in one persistent cooperative launch (grid barrier per iteration, work
    units from a counter) and in one launch per iteration: bit-identical records."""
    phia = gpu_lib
    insts = ins.batched_er(12, seed=3, n_lo=80, n_hi=900)
    sched = _sched(phia)
    outs = []
    for mode in (1, 2):
        with phia.Batch(insts, csr_mode=mode) as B:
            B.anneal(sched, 256, 150, seed=5)
            outs.append([B.replica_results(k, 256) for k in range(len(insts))])
    for a, b in zip(outs[0], outs[1]):
        for u, w in zip(a, b):
            assert np.array_equal(u, w)


def test_batch_autotune_picks_a_mode(gpu_lib):
    phia = gpu_lib
    insts = ins.batched_er(6, seed=5, n_lo=100, n_hi=600) + [ins.sk_pm1(100, 1)]
    with phia.Batch(insts) as B:
        tr = B.autotune(_sched(phia), 256, probe_iters=30)
        assert tr.tc_kernel in (1, 2) and tr.candidates == 2 and 0 < tr.best_us_per_iter <= tr.worst_us_per_iter
        B.anneal(_sched(phia), 256, 40, seed=2)
        be, _, _, _ = B.replica_results(6, 256)
        assert (be < 0).any()

