"""GPU parity tests of the sparse batched path (CSR gather over bit-packed spins)."""
import numpy as np
import pytest

import oracle as o
from paper_2407_10205_gb300 import instances as ins

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _csr_handle(phia, c):
    return phia.Annealer(h_k=c.kh, frac_bits=c.frac_bits, csr=(c.row_ptr, c.col, c.val), path=phia.PATH_CSR)


@pytest.mark.parametrize("N,density,R", [(5, 0.9, 3), (100, 0.06, 40), (700, 0.01, 256), (1500, 0.02, 33)])
def test_csr_field_bit_exact(gpu_lib, N, density, R):
    phia = gpu_lib
    c = ins.erdos_renyi(N, density, 127, 31, 4, seed=N)
    S = ins.random_spins(R, N, seed=N + 1)
    with _csr_handle(phia, c) as A:
        f = torch.empty((R, N), dtype=torch.int32, device="cuda")
        e = torch.empty(R, dtype=torch.int64, device="cuda")
        phia.field(A.h, torch.from_numpy(S).cuda(), f, e)
        torch.cuda.synchronize()
    P = o.Instance(c.kh, row_ptr=c.row_ptr, col=c.col, val=c.val, frac_bits=4)
    I, E = o.field_batch(P, S)
    assert np.array_equal(f.cpu().numpy(), I) and np.array_equal(e.cpu().numpy(), E)


def test_csr_single_step_matches_oracle(gpu_lib):
    phia = gpu_lib
    N, R, eps, gamma, beta = 900, 256, 0.1, 2.0, 0.3
    c = ins.erdos_renyi(N, 0.03, 127, 31, 4, seed=3)
    P = o.Instance(c.kh, row_ptr=c.row_ptr, col=c.col, val=c.val, frac_bits=4)
    x, v = ins.random_state(R, N, seed=4)
    xn = x.astype(np.float64) + eps * v.astype(np.float64)
    bad = np.abs(xn) < 1e-3
    x[bad] = np.where(xn[bad] >= 0, 0.01, -0.01).astype(np.float32)
    v[bad] = 0.0
    with _csr_handle(phia, c) as A:
        xt, vt = torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda()
        phia.run(A.h, phia.schedule(beta, beta, eps, gamma), R, 0, 1, 1, 5, xt, vt)
        be, bs, _, bits = phia.replica_results(A.h, R, N)
        xg, vg = xt.cpu().numpy(), vt.cpu().numpy()
    S = phia.unpack_bits(bits, N)
    for r in range(0, R, 7):
        xo, vo, so, Io, eo = o.step(P, x[r].astype(np.float64), v[r].astype(np.float64), beta, eps, gamma)
        assert np.array_equal(S[r], so) and be[r] == eo and bs[r] == 0
        assert np.allclose(xg[r], xo, rtol=1e-6, atol=1e-7)
        scale = np.abs(v[r]) + eps * (beta * gamma * P.q * np.abs(Io) + np.abs(xo))
        assert np.all(np.abs(vg[r] - vo) <= 1e-5 * np.maximum(scale, 1e-3))


def test_csr_equals_tensor_core_path(gpu_lib):
    """The CSR and tensor-core paths compute the same exact field and the same FP32
    update per replica: on one instance their runs are bit-identical."""
    phia = gpu_lib
    N, R, T = 230, 256, 80
    d = ins.dense_int(N, 7, 7, seed=12)
    rows, cols = np.nonzero(d.k)
    rp = np.zeros(N + 1, dtype=np.int32)
    np.add.at(rp, rows + 1, 1)
    rp = np.cumsum(rp).astype(np.int32)
    sched = phia.schedule(0.01, 0.2, 0.1, 2.0, refresh=20)
    outs = []
    with phia.Annealer(h_k=d.kh, csr=(rp, cols.astype(np.int32), d.k[rows, cols]), path=phia.PATH_CSR) as A:
        A.anneal(sched, R, T, seed=3)
        outs.append(phia.replica_results(A.h, R, N))
    with phia.Annealer(d.k, d.kh, path=phia.PATH_TC) as B:
        B.anneal(sched, R, T, seed=3)
        outs.append(phia.replica_results(B.h, R, N))
    for u, w in zip(outs[0], outs[1]):
        assert np.array_equal(u, w)


def test_batch_results_same_alone_and_in_the_mix(gpu_lib):
    """Each instance of a ragged batch gives bit-identical records to the same instance
    annealed on its own (its Philox id, couplings and replicas are its own)."""
    phia = gpu_lib
    insts = ins.batched_er(5, seed=2, n_lo=60, n_hi=700)
    R, T = 256, 60
    sched = phia.schedule(0.01, 0.3, 0.1, 2.0, refresh=25)
    with phia.Batch(insts, instance_ids=[10 + k for k in range(5)]) as B:
        B.anneal(sched, R, T, seed=9)
        mix = [B.replica_results(k, R) for k in range(5)]
        st = B.stats()
    assert st.spin_updates == R * T * sum(c.n for c in insts)
    for k, c in enumerate(insts):
        with phia.Batch([c], instance_ids=[10 + k]) as A:
            A.anneal(sched, R, T, seed=9)
            alone = A.replica_results(0, R)
        for u, w in zip(mix[k], alone):
            assert np.array_equal(u, w)
        P = o.Instance(c.kh, row_ptr=c.row_ptr, col=c.col, val=c.val, frac_bits=c.frac_bits)
        S = phia.unpack_bits(mix[k][3], c.n)
        for r in range(0, R, 17):
            assert o.energy_exact(P, S[r]) == mix[k][0][r]


def test_padded_replicas_do_not_change_results(gpu_lib):
    phia = gpu_lib
    c = ins.erdos_renyi(300, 0.05, 127, 31, 4, seed=5)
    sched = phia.schedule(0.01, 0.3, 0.1, 2.0)
    with phia.Batch([c]) as A:
        A.anneal(sched, 256, 40, seed=1)
        full = A.replica_results(0, 256)
        A.anneal(sched, 100, 40, seed=1)
        part = A.replica_results(0, 100)
    for u, w in zip(full, part):
        assert np.array_equal(u[:100], w)
