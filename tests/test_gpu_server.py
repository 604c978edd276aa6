"""The serving loop (kcm_server_*): jobs admitted in waves while others run, each result the same
as the job run alone, per-job convergence and caps, admission under a memory budget."""
import time

import numpy as np
import pytest

from paper_1712_05012_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kcm():
    import torch
    assert torch.cuda.is_available()
    from paper_1712_05012_b300 import kcm as K
    K.load()
    return K


def jobs(n, seed0=31):
    out = []
    for i in range(n):
        m = [1, 3, 12, 40, 25, 7, 60, 18][i % 8]
        seq = synth.sequence(m, seed0 + i)
        th = synth.theta_uniform(m, seed0 + i) * 0.05  # near the extended chain: smooth trajectories
        out.append((seq, th))
    return out


def run_server(kcm, table, p, items, caps, budget=8 << 30, max_chains=4, chunk=7, waves=3, admission=None):
    """Submit the jobs in `waves` groups with ticks in between (later jobs arrive while earlier ones
    run), then tick until every job is done."""
    res = {}
    with kcm.Server(p, budget, max_chains, chunk) as s:
        if admission:
            s.set_admission(*admission)
        ids = []
        per = (len(items) + waves - 1) // waves
        for w in range(waves):
            for (seq, th), cap in zip(items[w * per:(w + 1) * per], caps[w * per:(w + 1) * per]):
                ids.append(s.submit(seq, table, th, cap))
            for _ in range(3):
                s.tick()
                time.sleep(0.002)
        t0 = time.time()
        while True:
            wt, rn = s.tick()
            if wt == 0 and rn == 0:
                break
            assert time.time() - t0 < 120
            time.sleep(0.001)
        done = set(s.poll())
        assert done == set(ids)
        for jid in ids:
            res[jid] = s.job(jid)
        assert s.device_bytes() == 0  # every batch freed
    return [res[j] for j in ids]


def alone(kcm, table, p, seq, th, n):
    with kcm.Chain(seq, table, p) as ch:
        ch.set_theta(th)
        it, dm = ch.step(n)
        return it, dm, ch.get_theta()


def test_server_results_equal_alone(kcm, table):
    """FP64: every job's theta after up to 30 iterations (caps spanning several chunks) equals the
    job run alone to 1e-9 rad."""
    p = synth.RunParams(precision=synth.PRECISION_FP64, solvation=0)
    items = jobs(10)
    caps = [20, 15, 30, 20, 9, 20, 25, 14, 20, 17]
    got = run_server(kcm, table, p, items, caps)
    for (seq, th), cap, r in zip(items, caps, got):
        it, dm, th1 = alone(kcm, table, p, seq, th, cap)
        assert r["state"] == kcm.JOB_DONE and r["error"] == 0
        assert r["iters"] == it
        assert np.max(np.abs(r["theta"] - th1)) < 1e-9
        assert r["t_submit"] <= r["t_admit"] <= r["t_done"]


def test_server_admission_waves(kcm, table):
    """Admission in waves (at least 5 waiting jobs, or 30 ms, or nothing running): every job still
    runs and equals the job alone; bad settings are refused."""
    p = synth.RunParams(precision=synth.PRECISION_FP64, solvation=0)
    items = jobs(9, seed0=81)
    caps = [12, 9, 20, 7, 15, 20, 11, 8, 14]
    got = run_server(kcm, table, p, items, caps, admission=(5, 0.03))
    for (seq, th), cap, r in zip(items, caps, got):
        it, dm, th1 = alone(kcm, table, p, seq, th, cap)
        assert r["state"] == kcm.JOB_DONE and r["error"] == 0
        assert r["iters"] == it
        assert np.max(np.abs(r["theta"] - th1)) < 1e-9
    with kcm.Server(p, 1 << 30, 4, 5) as s:
        for bad in ((0, 0.0), (1, -1.0), (1, float("inf"))):
            with pytest.raises(kcm.KcmError):
                s.set_admission(*bad)


def test_server_side_joints_equal_alone(kcm, table):
    """With side-chain joints on, every job's side groups start at chi = 0 and are stepped with its
    main chain, in the mix as alone (FP64, 1e-9 rad on the main-chain angles it reports)."""
    p = synth.RunParams(precision=synth.PRECISION_FP64, solvation=0, side_joints=1)
    items = jobs(8, seed0=71)
    caps = [12, 20, 7, 20, 15, 9, 20, 11]
    got = run_server(kcm, table, p, items, caps)
    for (seq, th), cap, r in zip(items, caps, got):
        it, dm, th1 = alone(kcm, table, p, seq, th, cap)
        assert r["state"] == kcm.JOB_DONE and r["error"] == 0
        assert r["iters"] == it
        assert np.max(np.abs(r["theta"] - th1)) < 1e-9


def test_server_mixed_steps_equal_alone(kcm, table):
    """Mixed mode, within its per-iteration tolerance: the torques of a job in the mix and alone may
    differ by 1e-4 of the largest (rounding of the double-float kinematics depends on where the
    chain sits in its batch), so after k clamped steps theta agrees to k kappa 1e-4 max|tau|."""
    p = synth.RunParams(precision=synth.PRECISION_MIXED, solvation=1)
    items = jobs(10, seed0=91)
    caps = [2, 1, 2, 2, 1, 2, 2, 1, 2, 2]
    got = run_server(kcm, table, p, items, caps, chunk=1)
    for (seq, th), cap, r in zip(items, caps, got):
        with kcm.Chain(seq, table, p) as ch:
            ch.set_theta(th)
            tmax = np.max(np.abs(ch.torques()))
        it, dm, th1 = alone(kcm, table, p, seq, th, cap)
        assert r["iters"] == it
        assert np.max(np.abs(r["theta"] - th1)) <= cap * p.kappa * 1e-4 * tmax + 1e-12


def test_server_convergence_per_job(kcm, table):
    p = synth.RunParams(precision=synth.PRECISION_FP64, solvation=0, kappa=2e-5, conv_tol=2e-3)
    items = jobs(8, seed0=57)
    caps = [200] * 8
    got = run_server(kcm, table, p, items, caps, chunk=5)
    its = set()
    for (seq, th), r in zip(items, got):
        it, dm, th1 = alone(kcm, table, p, seq, th, 200)
        assert r["iters"] == it
        assert bool(r["converged"]) == (it < 200)
        assert np.max(np.abs(r["theta"] - th1)) < 1e-9
        its.add(it)
    assert len(its) > 1


def test_server_budget(kcm, table):
    """Device memory of the server's batches stays within the budget; a job that can never fit is
    refused with KCM_E_NOMEM while the others complete, with results equal to the jobs alone."""
    p = synth.RunParams(precision=synth.PRECISION_FP64, solvation=0)
    small = jobs(3, seed0=77)
    budget = 24 << 20  # 8 MB per batch plus a few small chains
    with kcm.Server(p, budget, 8, 5) as s:
        ids = [s.submit(seq, table, th, 10) for seq, th in small]
        big = synth.sequence(2000, 5)
        bid = s.submit(big, table, synth.theta_extended(2000), 10)
        peak = 0
        t0 = time.time()
        while True:
            wt, rn = s.tick()
            peak = max(peak, s.device_bytes())
            if wt == 0 and rn == 0:
                break
            assert time.time() - t0 < 60
        assert peak <= budget
        assert s.job(bid, with_theta=False)["error"] == kcm.KCM_E_NOMEM
        for jid, (seq, th) in zip(ids, small):
            r = s.job(jid)
            assert r["error"] == 0 and r["iters"] == 10
            it, dm, th1 = alone(kcm, table, p, seq, th, 10)
            assert np.max(np.abs(r["theta"] - th1)) < 1e-9


def test_served_fp64_surrogate_follows_oracle_loop(kcm, table):
    """Served FP64 jobs with the pairwise solvation surrogate (smooth, solvation = 2), several sharing
    batches, 25 iterations each: theta against the oracle's own loop from the same start to 1e-8 rad."""
    from oracle import oracle as O
    p = synth.RunParams(precision=synth.PRECISION_FP64, solvation=2)
    items = []
    for i, m in enumerate((15, 30, 40, 9, 22, 33)):
        items.append((synth.sequence(m, 71 + i), synth.theta_extended(m)))
    caps = [25] * len(items)
    got = run_server(kcm, table, p, items, caps, max_chains=3, chunk=6, waves=2)
    for (seq, th), r in zip(items, got):
        assert r["state"] == kcm.JOB_DONE and r["error"] == 0 and r["iters"] == 25
        th_ref, it_ref, _, _ = O.OracleChain(seq, table, synth.GEOMETRY).run(p, th, 25)
        assert it_ref == 25
        assert np.max(np.abs(r["theta"] - th_ref)) < 1e-8


def test_served_mixed_enumeration_torque_parity(kcm, table):
    """Served mixed-precision jobs with Algorithm 1 (solvation = 1) from compact starts, in a mix, 20
    iterations each: at the conformation each served job reached, the mixed torques agree with the FP64
    oracle's to 1e-4 (per-iteration parity; the trajectories themselves are chaotic from compact starts)."""
    from oracle import oracle as O
    p = synth.RunParams(precision=synth.PRECISION_MIXED, solvation=1)
    items, ochs = [], []
    for i, m in enumerate((24, 60, 37, 12, 80)):
        seq = synth.sequence(m, 91 + i)
        och = O.OracleChain(seq, table, synth.GEOMETRY)
        items.append((seq, synth.theta_from_codes(och.grow_start(91 + i))))
        ochs.append(och)
    caps = [20] * len(items)
    got = run_server(kcm, table, p, items, caps, max_chains=3, chunk=7, waves=2)
    pf = synth.RunParams(precision=synth.PRECISION_FP64, solvation=1)
    for (seq, _), och, r in zip(items, ochs, got):
        assert r["state"] == kcm.JOB_DONE and r["error"] == 0 and r["iters"] == 20
        ref = och.evaluate(pf, r["theta"])
        with kcm.Chain(seq, table, p) as ch:
            ch.set_theta(r["theta"])
            tau = ch.torques()
        assert np.max(np.abs(tau - ref["tau"])) / np.max(np.abs(ref["tau"])) < 1e-4


def drive(s, ids, on_tick=None, limit=120):
    """Tick until every job is done; on_tick(s) runs after every tick."""
    t0 = time.time()
    while True:
        wt, rn = s.tick()
        if on_tick:
            on_tick(s)
        if wt == 0 and rn == 0 and set(ids) <= set(j for j in ids if s.job(j, with_theta=False)["state"] == 2):
            break
        assert time.time() - t0 < limit
        time.sleep(0.0005)


def test_freed_slots_are_refilled(kcm, table):
    """Slots, not waves: two jobs arrive while a batch of four runs and wait (the admission wave asks for
    three); when the batch's first two jobs retire after one chunk, the next batch takes the two waiting
    jobs into the freed slots together with the batch's two running jobs, which move over with the angles
    they reached, and the old batch is freed. Every job, moved or admitted into a freed slot, equals the
    job run alone (FP64, 1e-9 rad), and the device memory held falls when jobs retire."""
    p = synth.RunParams(precision=synth.PRECISION_FP64, solvation=0)
    items = jobs(6, seed0=51)
    caps = [5, 5, 40, 40, 30, 30]
    with kcm.Server(p, 8 << 30, 4, 5) as s:
        s.set_admission(3, 30.0)
        ids = [s.submit(seq, table, th, cap) for (seq, th), cap in zip(items[:4], caps[:4])]
        while s.tick()[1] == 0:  # the first batch is made on the worker thread (nothing ran: admitted)
            time.sleep(0.0005)
        first = s.device_bytes()
        assert first > 0
        ids += [s.submit(seq, table, th, cap) for (seq, th), cap in zip(items[4:], caps[4:])]
        seen = []
        for _ in range(200):  # the new jobs wait while all four slots are taken
            w, r = s.tick()
            if s.job(ids[0], with_theta=False)["state"] == kcm.JOB_DONE:
                break
            assert w == 2 and r == 4
            time.sleep(0.0005)
        seen = []
        drive(s, ids, on_tick=lambda srv: seen.append(srv.device_bytes()))
        assert s.device_bytes() == 0
        # memory returns while jobs still run (a compacted batch replaces one with retired slots)
        assert any(0 < b < a for a, b in zip(seen, seen[1:]))
        got = [s.job(j) for j in ids]
    for (seq, th), cap, r in zip(items, caps, got):
        it, dm, th1 = alone(kcm, table, p, seq, th, cap)
        assert r["state"] == kcm.JOB_DONE and r["error"] == 0 and r["iters"] == it == cap
        assert np.max(np.abs(r["theta"] - th1)) < 1e-9


def test_cancel(kcm, table):
    """kcm_server_cancel: a waiting job retires at once, a running job at the end of its chunk, both with
    KCM_E_CANCELLED; the other jobs are unaffected (equal to alone, FP64, 1e-9 rad)."""
    p = synth.RunParams(precision=synth.PRECISION_FP64, solvation=0)
    items = jobs(5, seed0=61)
    caps = [30, 30, 30, 30, 30]
    with kcm.Server(p, 8 << 30, 3, 4) as s:
        ids = [s.submit(seq, table, th, cap) for (seq, th), cap in zip(items, caps)]
        s.cancel(ids[4])  # still waiting
        assert s.job(ids[4], with_theta=False)["error"] == kcm.KCM_E_CANCELLED
        while s.job(ids[1], with_theta=False)["state"] != kcm.JOB_RUNNING:
            s.tick()
            time.sleep(0.0005)
        s.cancel(ids[1])  # running: stops at the end of its chunk
        with pytest.raises(kcm.KcmError):
            s.cancel(ids[4])  # already finished
        drive(s, ids)
        got = [s.job(j) for j in ids]
    c = got[1]
    assert c["state"] == kcm.JOB_DONE and c["error"] == kcm.KCM_E_CANCELLED and 0 < c["iters"] < caps[1]
    seq, th = items[1]
    _, _, th_c = alone(kcm, table, p, seq, th, c["iters"])  # the angles it had reached
    assert np.max(np.abs(c["theta"] - th_c)) < 1e-9
    for k in (0, 2, 3):
        seq, th = items[k]
        it, dm, th1 = alone(kcm, table, p, seq, th, caps[k])
        assert got[k]["error"] == 0 and got[k]["iters"] == it
        assert np.max(np.abs(got[k]["theta"] - th1)) < 1e-9
