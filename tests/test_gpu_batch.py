"""Batches of chains (kcm_create_batch) against the same chains alone and against the oracle.

A batch concatenates its chains; every scan is segmented at chain boundaries and every chain has
its own cell grid, so each chain's results must equal its results alone up to rounding order
(the scan blocks fall differently), and its iteration count and convergence must be its own."""
import os
import numpy as np
import pytest

from oracle import oracle as O
from paper_1712_05012_b300 import synth

from kcm_testutil import SPARSE_KINKS, rel_inf, tol_positions

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kcm():
    import torch
    assert torch.cuda.is_available()
    from paper_1712_05012_b300 import kcm as K
    K.load()
    return K

# lengths from one residue up, starts of both kinds
CASES = [(1, 11, "uniform"), (2, 12, "uniform"), (3, 13, "compact"), (17, 14, "compact"), (40, 15, "extended"),
         (97, 16, "compact"), (5, 17, "uniform")]


def chain_inputs(table):
    seqs, thetas = [], []
    for m, seed, kind in CASES:
        seq = synth.sequence(m, seed)
        if kind == "compact":
            th = synth.theta_from_codes(O.OracleChain(seq, table, synth.GEOMETRY).grow_start(seed))
        elif kind == "extended":
            th = synth.theta_extended(m)
        else:
            th = synth.theta_uniform(m, seed)
        seqs.append(seq)
        thetas.append(th)
    return seqs, thetas


def alone(kcm, seq, table, p, th):
    with kcm.Chain(seq, table, p) as ch:
        ch.set_theta(th)
        return dict(xyz=ch.positions(), tau=ch.torques(), E=ch.energy(), F=ch.forces())


@pytest.mark.parametrize("precision", [synth.PRECISION_FP64, synth.PRECISION_MIXED])
def test_batch_matches_alone(kcm, table, precision):
    seqs, thetas = chain_inputs(table)
    p = synth.RunParams(precision=precision)
    with kcm.Batch(seqs, table, p) as b:
        assert b.nchains == len(seqs)
        b.set_theta(np.concatenate(thetas))
        xyz = b.split(b.positions())
        tau = b.split(b.torques(), per="joint")
        F = b.split(b.forces())
        E = b.chain_energies()
        Etot = b.energy()
    tol = 1e-10 if precision == synth.PRECISION_FP64 else 1e-9
    for c, (seq, th) in enumerate(zip(seqs, thetas)):
        ref = alone(kcm, seq, table, p, th)
        assert np.max(np.abs(xyz[c] - ref["xyz"])) < 1e-9
        assert rel_inf(tau[c], ref["tau"]) < tol, c
        assert rel_inf(F[c], ref["F"]) < tol, c
        np.testing.assert_allclose(E[c], ref["E"], rtol=1e-6 if precision else 1e-10, atol=1e-6)
    # two evaluations: mixed-mode energies are FP32 per warp, summed by atomics in any order
    np.testing.assert_allclose(Etot, E.sum(0), rtol=1e-12 if precision == synth.PRECISION_FP64 else 1e-6, atol=1e-9)


def test_batch_fp64_matches_oracle(kcm, table):
    seqs, thetas = chain_inputs(table)
    p = synth.RunParams(precision=synth.PRECISION_FP64)
    with kcm.Batch(seqs, table, p) as b:
        b.set_theta(np.concatenate(thetas))
        tau = b.split(b.torques(), per="joint")
        xyz = b.split(b.positions())
    for c in (2, 5):  # a 3-residue and the 97-residue compact chain
        och = O.OracleChain(seqs[c], table, synth.GEOMETRY)
        ref = och.evaluate(p, thetas[c])
        assert np.max(np.abs(xyz[c] - ref["xyz"])) < tol_positions(och.l)
        assert rel_inf(tau[c], ref["tau"]) < 1e-10


def test_batch_steps_and_convergence_per_chain(kcm, table):
    """Every chain stops when its own max |dtheta| falls below conv_tol; the batch loop ends when all
    have. The iterations, theta and last step of each chain equal those of the chain stepped alone."""
    seqs, thetas = chain_inputs(table)
    p = synth.RunParams(precision=synth.PRECISION_FP64, solvation=0, kappa=2e-5, conv_tol=2e-3)
    n = 60
    with kcm.Batch(seqs, table, p) as b:
        b.set_theta(np.concatenate(thetas))
        it_b, _ = b.step(n)
        th_b = b.split(b.get_theta(), per="joint")
        iters, conv, dm = b.chain_state()
    its = []
    for c, (seq, th) in enumerate(zip(seqs, thetas)):
        with kcm.Chain(seq, table, p) as ch:
            ch.set_theta(th)
            it, d1 = ch.step(n)
            its.append(it)
            assert iters[c] == it, c
            assert conv[c] == (it < n or d1 < p.conv_tol), c
            assert np.max(np.abs(th_b[c] - ch.get_theta())) < 1e-9, c
            assert abs(dm[c] - d1) < 1e-9
    assert it_b == max(its)
    assert len(set(its)) > 1  # the chains converge at different iterations


def test_batch_mixed_steps_match_alone(kcm, table):
    """Mixed mode, three iterations: the double-float kinematics round differently in the batch
    (its scan blocks fall elsewhere), by ~1e-13 A, which can move an FP32 rounding of the next
    iteration's cell offsets and so the torques by ~1e-7 relative; kappa = 1e-3 makes that ~1e-7 rad
    per step. The bound, 1e-5 rad after three steps, is far inside the mixed torque tolerance
    (1e-4 of max |tau| per step)."""
    seqs, thetas = chain_inputs(table)
    p = synth.RunParams(precision=synth.PRECISION_MIXED)
    with kcm.Batch(seqs, table, p) as b:
        b.set_theta(np.concatenate(thetas))
        b.step(3)
        th_b = b.split(b.get_theta(), per="joint")
    for c, (seq, th) in enumerate(zip(seqs, thetas)):
        with kcm.Chain(seq, table, p) as ch:
            ch.set_theta(th)
            ch.step(3)
            assert np.max(np.abs(th_b[c] - ch.get_theta())) < 1e-5, c


def test_batch512_mixed_vs_fp64_and_oracle(kcm, table):
    """The 512-chain batch workload from its stored compact starts: every chain's mixed torques
    within 1e-4 (relative to the chain's largest) of the FP64 batch, and three chains (the shortest,
    a middle one and the longest) against the oracle."""
    import json
    import os
    here = os.path.dirname(os.path.abspath(__file__))
    wl = synth.workload(4)
    seqs = [synth.sequence(m, synth.chain_seed(wl.seed, i)) for i, m in enumerate(wl.m)]
    theta = synth.theta_from_codes(np.load(os.path.join(here, "golden", "start_batch512.npy")))
    man = json.load(open(os.path.join(here, "golden", "starts.json")))["batch512"]
    tau = {}
    for prec in (synth.PRECISION_MIXED, synth.PRECISION_FP64):
        with kcm.Batch(seqs, table, synth.RunParams(precision=prec)) as b:
            assert b.n == man["atoms"]
            b.set_theta(theta)
            tau[prec] = b.split(b.torques(), per="joint")
            joff = b.joint_off
    worst = max(rel_inf(tm, tf) for tm, tf in zip(tau[synth.PRECISION_MIXED], tau[synth.PRECISION_FP64]))
    assert worst < 1e-4
    order = np.argsort(wl.m)
    for c in (order[0], order[len(order) // 2], order[-1]):
        och = O.OracleChain(seqs[c], table, synth.GEOMETRY)
        ref = och.evaluate(synth.RunParams(precision=synth.PRECISION_FP64), theta[joff[c]:joff[c + 1]])
        assert rel_inf(tau[synth.PRECISION_FP64][c], ref["tau"]) < 1e-10
        assert rel_inf(tau[synth.PRECISION_MIXED][c], ref["tau"]) < 1e-4


def test_batch_chain_fails_alone(kcm, table):
    """A chain whose solvation lists overflow (a compact ~1,000-atom chain with probe radius 9 A: far
    more neighbours than the list holds) stops with KCM_E_OVERFLOW; a 3-residue chain in the same batch
    (fewer atoms than the list holds, it cannot overflow) takes all its iterations and ends where it
    ends alone."""
    big = synth.sequence(97, 9)
    small = synth.sequence(3, 13)
    th_big = synth.theta_from_codes(O.OracleChain(big, table, synth.GEOMETRY).grow_start(9))
    th_small = synth.theta_uniform(3, 13)
    p = synth.RunParams(precision=synth.PRECISION_FP64, r_probe=9.0)
    with kcm.Batch([big, small], table, p) as b:
        b.set_theta(np.concatenate([th_big, th_small]))
        with pytest.raises(kcm.KcmError) as e:
            b.step(4)
        assert e.value.code == kcm.KCM_E_OVERFLOW
        iters, stopped, dm, err = b.chain_state(with_errors=True)
        th = b.split(b.get_theta(), per="joint")
    assert err[0] == kcm.KCM_E_OVERFLOW and err[1] == kcm.KCM_OK
    assert iters[1] == 4
    with kcm.Chain(small, table, p) as ch:
        ch.set_theta(th_small)
        ch.step(4)
        assert np.max(np.abs(th[1] - ch.get_theta())) < 1e-9



def test_batch_binning_large_grid(kcm, table):
    """Mixed batches bin each chain in one block, counting its cells in shared memory up to 8,192 cells
    and in global memory beyond. A 600-residue chain kinked into three straight segments (its grid is
    coarsened to its cap of 8 x 6,290 cells, far above 8,192) beside two compact chains: the mixed batch
    finds the FP64 batch's pair set and covered counts exactly (and a superset of its solvation lists), and every chain's torques agree with
    the FP64 batch within the mixed bar; the compact chains also match their evaluation alone."""
    m = 600
    seq_k = synth.sequence(m, 77)
    th_k = synth.theta_extended(m).copy()
    for j, v in SPARSE_KINKS:
        th_k[j] = v
    seqs, thetas = [seq_k], [th_k]
    for mm, seed in ((97, 16), (17, 14)):
        s = synth.sequence(mm, seed)
        seqs.append(s)
        thetas.append(synth.theta_from_codes(O.OracleChain(s, table, synth.GEOMETRY).grow_start(seed)))
    out = {}
    for prec in (synth.PRECISION_FP64, synth.PRECISION_MIXED):
        p = synth.RunParams(precision=prec)
        with kcm.Batch(seqs, table, p) as b:
            b.set_theta(np.concatenate(thetas))
            out[prec] = dict(tau=b.split(b.torques(), per="joint"), covered=b.sasa_counts(), stats=b.stats())
    mix, f64 = out[synth.PRECISION_MIXED], out[synth.PRECISION_FP64]
    assert mix["stats"]["cells"] > 8192
    assert mix["stats"]["pairs"] == f64["stats"]["pairs"]
    assert mix["stats"]["sasa_neighbors"] >= f64["stats"]["sasa_neighbors"]  # FP32 lists keep a margin
    assert np.array_equal(mix["covered"], f64["covered"])
    for c in range(len(seqs)):
        assert rel_inf(mix["tau"][c], f64["tau"][c]) < 1e-4, c
    pm = synth.RunParams(precision=synth.PRECISION_MIXED)
    for c in (1, 2):
        ref = alone(kcm, seqs[c], table, pm, thetas[c])
        assert rel_inf(mix["tau"][c], ref["tau"]) < 1e-9, c


def test_mixed_trajectory_reproducible_through_clashes(kcm, table):
    """Chain 216 of the 512-chain batch workload (425 residues), alone: its clamped
    steps drive atoms into clashes whose pair terms exceed the 2^-23 fixed point's range (2^22). Those
    terms are summed in exact integer units of 2^-1, so every run from the same start gives the same
    angles, bit for bit (a float sum of them varied with the order of the atomics and, through
    Algorithm 1's coverage decisions, moved joints by whole steps in some runs)."""
    wl = synth.workload(4)
    i = 216
    seq = synth.sequence(wl.m[i], synth.chain_seed(wl.seed, i))
    codes = np.load(os.path.join(os.path.dirname(__file__), "golden", "start_batch512.npy"))
    off = 2 * int(np.sum(wl.m[:i]))
    th = synth.theta_from_codes(codes[off:off + 2 * wl.m[i]])
    p = synth.RunParams(precision=synth.PRECISION_MIXED)
    with kcm.Chain(seq, table, p) as c:
        runs = []
        for _ in range(6):
            c.set_theta(th)
            c.step(8)
            runs.append(np.asarray(c.get_theta()).copy())
    for r in runs[1:]:
        assert np.array_equal(r, runs[0])
