"""Side-chain joints (eq. kin_05, r2: up to four rotations chi_k per residue about successive side-chain
bonds; the branch torques of Sec. 3.5) through the C ABI against the oracle: positions, side- and
main-chain torques, FP64 loops that step both kinds of joint as one vector (clamped and normalised),
the mixed path against FP64, and batches against chains alone."""
import json
import os

import numpy as np
import pytest

from kcm_testutil import rel_inf, tol_positions
from oracle import oracle as O
from paper_1712_05012_b300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TOL_FP64 = 1e-10
TOL_MIXED = 1e-4


@pytest.fixture(scope="module")
def kcm():
    import torch
    assert torch.cuda.is_available()
    from paper_1712_05012_b300 import kcm as K
    K.load()
    return K


def case(table, m, seed, spread):
    seq = synth.sequence(m, seed)
    och = O.OracleChain(seq, table, synth.GEOMETRY)
    th = synth.theta_from_codes(och.grow_start(seed))
    chi = np.random.default_rng(seed).uniform(-spread, spread, och.nside_joints)
    return seq, och, th, chi


def gpu_eval(kcm, seq, table, p, th, chi):
    with kcm.Chain(seq, table, p) as ch:
        ch.set_theta(th)
        ch.set_side_theta(chi)
        out = dict(xyz=ch.positions(), tau=ch.torques(), tau_side=ch.side_torques(), E=ch.energy())
        out["F_pair"], out["F_cav"] = ch.force_terms()
        return out


@pytest.mark.parametrize("m,seed", [(1, 41), (7, 42), (40, 1235), (97, 43)])
def test_positions_vs_oracle(kcm, table, m, seed):
    """Atom centres at random main-chain and side-chain angles (chi uniform over the full turn)."""
    seq, och, th, chi = case(table, m, seed, np.pi)
    want, _, _ = och.fk(th, side=chi)
    for prec, tol in ((synth.PRECISION_FP64, tol_positions(och.l)), (synth.PRECISION_MIXED, 1e-5)):
        with kcm.Chain(seq, table, synth.RunParams(precision=prec, side_joints=1)) as ch:
            assert ch.ls == och.nside_joints
            ch.set_theta(th)
            ch.set_side_theta(chi)
            assert np.array_equal(ch.get_side_theta(), chi)
            got = ch.positions()
        assert np.max(np.abs(got - want)) < tol


@pytest.mark.parametrize("solv", [0, 1, 2])
@pytest.mark.parametrize("m,seed", [(7, 44), (40, 1235)])
def test_fp64_torques_vs_oracle(kcm, table, m, seed, solv):
    """Side- and main-chain torques, forces and energies in FP64 with every solvation mode."""
    seq, och, th, chi = case(table, m, seed, 0.3)  # no clashes: |tau| stays below ~1e4
    p = synth.RunParams(precision=synth.PRECISION_FP64, solvation=solv, side_joints=1)
    ref = och.evaluate(p, th, side=chi)
    got = gpu_eval(kcm, seq, table, p, th, chi)
    assert rel_inf(got["F_pair"], ref["F_pair"]) < TOL_FP64
    if solv:
        assert rel_inf(got["F_cav"], ref["F_cav"]) < TOL_FP64
    assert rel_inf(got["tau_side"], ref["tau_side"]) < TOL_FP64
    assert rel_inf(got["tau"], ref["tau"]) < TOL_FP64
    np.testing.assert_allclose(got["E"], ref["E"], rtol=TOL_FP64, atol=1e-9)


def test_chain1000_side_joints(kcm, table):
    """The 1,000-residue compact workload with small random side-chain angles (+-0.1 rad, a state without
    clashes: |tau| below ~3e4), both precisions."""
    man = json.load(open(os.path.join(GOLDEN, "starts.json")))["chain1000"]
    seq = synth.sequence(man["residues"], man["sequence_seed"])
    th = synth.theta_from_codes(np.load(os.path.join(GOLDEN, "start_chain1000.npy")))
    och = O.OracleChain(seq, table, synth.GEOMETRY)
    chi = np.random.default_rng(6).uniform(-0.1, 0.1, och.nside_joints)
    pf = synth.RunParams(precision=synth.PRECISION_FP64, solvation=2, side_joints=1)
    ref = och.evaluate(pf, th, side=chi)
    f64 = gpu_eval(kcm, seq, table, pf, th, chi)
    assert rel_inf(f64["tau_side"], ref["tau_side"]) < TOL_FP64
    assert rel_inf(f64["tau"], ref["tau"]) < TOL_FP64
    mix = gpu_eval(kcm, seq, table, synth.RunParams(precision=synth.PRECISION_MIXED, solvation=2, side_joints=1),
                   th, chi)
    assert rel_inf(mix["tau_side"], ref["tau_side"]) < TOL_MIXED
    assert rel_inf(mix["tau"], ref["tau"]) < TOL_MIXED


@pytest.mark.parametrize("mode", [0, 1])  # per-joint clamp, the paper's normalised step
def test_fp64_trajectory_vs_oracle(kcm, table, mode):
    """40 FP64 iterations of the 40-residue chain from the extended start with the surrogate solvation
    (smooth), main and side joints stepped together, against the oracle's loop."""
    seq = synth.sequence(40, synth.chain_seed(synth.workload(1).seed, 0))
    och = O.OracleChain(seq, table, synth.GEOMETRY)
    p = synth.RunParams(precision=synth.PRECISION_FP64, solvation=2, side_joints=1, step_mode=mode,
                        kappa=0.05 if mode else 1e-3)
    th0 = synth.theta_extended(40)
    chi0 = np.zeros(och.nside_joints)
    th_ref, chi_ref, it_ref, _, dm_ref = och.run(p, th0, 40, side=chi0)
    with kcm.Chain(seq, table, p) as ch:
        ch.set_theta(th0)
        it, dm = ch.step(40)
        th, chi = ch.get_theta(), ch.get_side_theta()
    assert it == it_ref
    assert np.max(np.abs(th - th_ref)) < 1e-8
    assert np.max(np.abs(chi - chi_ref)) < 1e-8
    assert np.max(np.abs(chi)) > 1e-3  # the side groups turned
    assert abs(dm - dm_ref[-1]) < 1e-8


def test_mixed_trajectory_rmsd(kcm, table):
    """All-atom RMSD of the mixed path against FP64 after 100 iterations with side-chain joints."""
    seq = synth.sequence(40, synth.chain_seed(synth.workload(1).seed, 0))
    xyz = {}
    for prec in (synth.PRECISION_MIXED, synth.PRECISION_FP64):
        with kcm.Chain(seq, table, synth.RunParams(precision=prec, solvation=2, side_joints=1)) as ch:
            ch.set_theta(synth.theta_extended(40))
            it, _ = ch.step(100)
            assert it == 100
            xyz[prec] = ch.positions()
    d = xyz[synth.PRECISION_MIXED] - xyz[synth.PRECISION_FP64]
    assert np.sqrt((d ** 2).sum(1).mean()) <= 1e-3


def test_batch_matches_alone(kcm, table):
    cases = [(3, 51), (17, 52), (40, 53)]
    seqs, ths, chis = [], [], []
    for m, seed in cases:
        seq, och, th, chi = case(table, m, seed, 0.3)
        seqs.append(seq)
        ths.append(th)
        chis.append(chi)
    for prec, tol in ((synth.PRECISION_FP64, 1e-8), (synth.PRECISION_MIXED, 1e-4)):
        p = synth.RunParams(precision=prec, solvation=2, side_joints=1)
        with kcm.Batch(seqs, table, p) as b:
            assert b.ls == sum(len(c) for c in chis)
            b.set_theta(np.concatenate(ths))
            b.set_side_theta(np.concatenate(chis))
            ts = b.split(b.side_torques(), per="side")
            b.step(8)
            th = b.split(b.get_theta(), per="joint")
            chi = b.split(b.get_side_theta(), per="side")
        for c in range(len(cases)):
            with kcm.Chain(seqs[c], table, p) as one:
                one.set_theta(ths[c])
                one.set_side_theta(chis[c])
                assert rel_inf(ts[c], one.side_torques()) < (TOL_FP64 if prec == synth.PRECISION_FP64 else 1e-5)
                one.step(8)
                assert np.max(np.abs(th[c] - one.get_theta())) < tol
                assert np.max(np.abs(chi[c] - one.get_side_theta())) < tol


def test_zero_side_angles_and_arguments(kcm, table):
    """chi = 0 gives the rigid side groups of side_joints = 0; wrong lengths are refused."""
    seq, och, th, _ = case(table, 12, 61, 0.0)
    with kcm.Chain(seq, table, synth.RunParams(side_joints=1)) as a, kcm.Chain(seq, table, synth.RunParams()) as b:
        assert b.ls == 0 and a.ls == och.nside_joints
        a.set_theta(th)
        b.set_theta(th)
        assert np.max(np.abs(a.positions() - b.positions())) < 1e-13
        assert rel_inf(a.torques(), b.torques()) < 1e-12
        L = kcm.load()
        x = np.zeros(a.ls + 1)
        assert L.kcm_set_side_theta(a.handle, x.ctypes.data_as(kcm._dp), a.ls + 1) == kcm.KCM_E_INVAL
        assert L.kcm_side_torques(a.handle, x.ctypes.data_as(kcm._dp), a.ls - 1) == kcm.KCM_E_INVAL
        x[:] = np.nan
        assert L.kcm_set_side_theta(a.handle, x.ctypes.data_as(kcm._dp), a.ls) == kcm.KCM_E_INVAL
        assert b.get_side_theta().shape == (0,)
        b.set_side_theta(np.zeros(0))


def test_side_theta_device_pointers(kcm, table):
    import torch
    seq, och, th, chi = case(table, 9, 62, 1.0)
    with kcm.Chain(seq, table, synth.RunParams(side_joints=1)) as ch:
        src = torch.tensor(chi, dtype=torch.float64, device="cuda")
        dst = torch.zeros_like(src)
        torch.cuda.synchronize()
        ch.set_side_theta_dev(src.data_ptr())
        ch.get_side_theta_dev(dst.data_ptr())
        torch.cuda.synchronize()
        assert np.array_equal(ch.get_side_theta(), chi)
        assert np.array_equal(dst.cpu().numpy(), chi)



def test_degenerate_side_joint_sets(kcm, table):
    """side_joints = 1 on a chain whose groups are all single atoms (no side-chain joint: the path runs
    as with the joints off) and on one residue with the largest group (four joints, nine moved atoms)."""
    one = [t for t in range(len(table.n_side)) if table.n_side[t] == 1]
    seq = np.array([one[i % len(one)] for i in range(9)], dtype=np.int32)
    th = synth.theta_uniform(9, 4)
    p = synth.RunParams(precision=synth.PRECISION_FP64, side_joints=1)
    with kcm.Chain(seq, table, p) as a, kcm.Chain(seq, table, synth.RunParams(precision=synth.PRECISION_FP64)) as b:
        assert a.ls == 0
        a.set_theta(th)
        b.set_theta(th)
        assert np.array_equal(a.positions(), b.positions())
        assert rel_inf(a.torques(), b.torques()) < 1e-12
        assert a.side_torques().shape == (0,)
        it, _ = a.step(3)
        assert it == 3
    big = int(np.argmax(table.n_side))
    seq1 = np.array([big], dtype=np.int32)
    och = O.OracleChain(seq1, table, synth.GEOMETRY)
    assert och.nside_joints == 4
    th1 = synth.theta_uniform(1, 5)
    chi = np.array([0.7, -1.1, 2.0, -0.4])
    ref = och.evaluate(p, th1, side=chi)
    with kcm.Chain(seq1, table, p) as c:
        c.set_theta(th1)
        c.set_side_theta(chi)
        assert np.max(np.abs(c.positions() - ref["xyz"])) < 1e-12
        assert rel_inf(c.side_torques(), ref["tau_side"]) < TOL_FP64
