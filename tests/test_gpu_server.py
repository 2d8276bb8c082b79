"""GPU tests of the continuous-batching server (phia_server_*)."""
import numpy as np
import pytest

import oracle as o
from paper_2407_10205_gb300 import instances as ins

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _requests():
    """A mix of small dense (resident kernel), larger dense (per-iteration kernel) and
    sparse (CSR) instances; small ones carry a target from a short oracle run."""
    out = []
    for k in range(10):
        if k % 3 == 0:
            inst = ins.sk_pm1(24 + 7 * k, 100 + k)
            P = o.Instance(inst.kh, k=inst.k)
            tgt = int(o.anneal(P, 4, 60, 5, 0, 0.05, 2.0, 0.2, 2.0)["best_e"].min())
        elif k % 3 == 1:
            inst = ins.dense_int(420 + 10 * k, 7, 7, 200 + k)
            tgt = None
        else:
            inst = ins.erdos_renyi(300 + 40 * k, 0.03, 127, 127, 8, 300 + k)
            P = o.Instance(inst.kh, row_ptr=inst.row_ptr, col=inst.col, val=inst.val, frac_bits=8)
            tgt = int(o.anneal(P, 4, 60, 5, k, 0.02, 0.5, 0.1, 2.0)["best_e"].min())
        out.append((inst, tgt))
    return out


def _serve(phia, reqs, max_inflight, budget):
    sched = phia.schedule(0.02, 0.5, 0.1, 2.0, refresh=40)
    res = []
    with phia.Server(max_inflight=max_inflight, hbm_budget_bytes=budget, chunk_iters=25) as S:
        ids = [S.submit(inst, sched, 64, 200, seed=1000 + k, instance_id=k, target=tgt)
               for k, (inst, tgt) in enumerate(reqs)]
        S.wait_all()
        for rid in ids:
            st, spins = S.poll(rid, want_spins=True)
            res.append((st.state, st.hit, st.energy_k, st.hit_step, st.steps_run, spins.copy(), st))
        stats = S.stats()
    return res, stats


def test_results_same_alone_and_in_the_mix(gpu_lib):
    phia = gpu_lib
    reqs = _requests()
    alone, _ = _serve(phia, reqs, max_inflight=1, budget=64 << 30)
    mix, stats = _serve(phia, reqs, max_inflight=8, budget=96 << 20)   # tight budget forces queueing
    assert stats.completed == len(reqs)
    for (inst, tgt), a, m in zip(reqs, alone, mix):
        assert a[0] == 2 and m[0] == 2
        assert a[1:5] == m[1:5], "result differs between alone and in the mix"
        assert np.array_equal(a[5], m[5])
        # returned energy is Eq. 2 on the returned spins
        if hasattr(inst, "k"):
            P = o.Instance(inst.kh, k=inst.k)
        else:
            P = o.Instance(inst.kh, row_ptr=inst.row_ptr, col=inst.col, val=inst.val, frac_bits=inst.frac_bits)
        assert o.energy_exact(P, m[5]) == m[2]
        if tgt is not None and m[1]:
            assert m[2] <= tgt and m[4] <= 200
    hits = sum(1 for m in mix if m[1])
    assert stats.hits == hits and hits >= 1
    assert stats.ttt_p50_s > 0 and stats.ttt_p99_s >= stats.ttt_p50_s


def test_requests_overlap_under_a_budget(gpu_lib):
    """Several requests are admitted at once (continuous batching) within the budget,
    and later arrivals take freed slots."""
    phia = gpu_lib
    sched = phia.schedule(0.02, 0.5, 0.1, 2.0)
    insts = [ins.dense_int(500, 7, 7, 40 + k) for k in range(6)]
    with phia.Server(max_inflight=3, hbm_budget_bytes=64 << 30, chunk_iters=50) as S:
        ids = [S.submit(inst, sched, 128, 300, seed=k, instance_id=k) for k, inst in enumerate(insts)]
        S.wait_all()
        sts = [S.poll(r)[0] for r in ids]
    # the first three were admitted before any finished; the last three after a slot freed
    first_done = min(s.t_done_s for s in sts[:3])
    assert all(s.t_admit_s < first_done for s in sts[:3])
    assert all(s.t_admit_s >= first_done - 1e-3 for s in sts[3:])
    assert all(s.state == 2 and s.steps_run == 300 for s in sts)


def test_bad_requests_fail_alone(gpu_lib):
    """An invalid instance ends its own request with an error code; the others finish;
    a request bigger than the whole budget is refused at submission."""
    phia = gpu_lib
    sched = phia.schedule(0.02, 0.5, 0.1, 2.0)
    good = ins.dense_int(64, 7, 7, 1)
    bad = ins.dense_int(64, 7, 7, 2)
    bad.k[3, 5] += 1                           # asymmetric J
    with phia.Server(max_inflight=2, hbm_budget_bytes=256 << 20, chunk_iters=20) as S:
        r1 = S.submit(good, sched, 32, 40, seed=1)
        r2 = S.submit(bad, sched, 32, 40, seed=2)
        r3 = S.submit(good, sched, 32, 40, seed=3)
        S.wait_all()
        assert S.poll(r1)[0].state == 2 and S.poll(r3)[0].state == 2
        assert S.poll(r2)[0].state == phia.EINVAL
        with pytest.raises(phia.PhiaError) as ei:
            S.submit(ins.dense_int(8000, 7, 7, 3), sched, 4096, 10, seed=4)
        assert ei.value.code == phia.ENOMEM
