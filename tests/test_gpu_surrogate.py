"""The pairwise solvation surrogate (solvation = 2; Sec. 3.4, the smooth pairwise area formulae that
preceded surface enumeration) through the C ABI against the oracle. Being smooth, it gives the
trajectory parity that the piecewise-constant enumeration cannot: FP64 runs follow the oracle's loop
and mixed runs follow FP64 runs."""
import json
import os

import numpy as np
import pytest

from kcm_testutil import rel_inf
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


def gpu_eval(kcm, seq, table, p, theta):
    with kcm.Chain(seq, table, p) as ch:
        ch.set_theta(theta)
        out = dict(tau=ch.torques(), E=ch.energy(), stats=ch.stats())
        out["F_pair"], out["F_cav"] = ch.force_terms()
        return out


@pytest.mark.parametrize("m,seed,kind", [(1, 1, "uniform"), (3, 3, "compact"), (40, 1235, "compact"),
                                         (97, 9, "compact")])
def test_fp64_surrogate_vs_oracle(kcm, table, m, seed, kind):
    seq = synth.sequence(m, seed)
    och = O.OracleChain(seq, table, synth.GEOMETRY)
    th = synth.theta_from_codes(och.grow_start(seed)) if kind == "compact" else synth.theta_uniform(m, seed)
    p = synth.RunParams(precision=synth.PRECISION_FP64, solvation=2)
    ref = och.evaluate(p, th)
    got = gpu_eval(kcm, seq, table, p, th)
    assert rel_inf(got["F_cav"], ref["F_cav"]) < TOL_FP64
    assert rel_inf(got["tau"], ref["tau"]) < TOL_FP64
    np.testing.assert_allclose(got["E"], ref["E"], rtol=TOL_FP64, atol=1e-9)
    # the pair terms cancel exactly in the integer sums
    assert np.abs(got["F_cav"].sum(axis=0)).max() < 1e-9


def test_chain1000_surrogate(kcm, table):
    """The 1,000-residue compact workload with the surrogate, both precisions, against the oracle."""
    man = json.load(open(os.path.join(GOLDEN, "starts.json")))["chain1000"]
    seq = synth.sequence(man["residues"], man["sequence_seed"])
    th = synth.theta_from_codes(np.load(os.path.join(GOLDEN, "start_chain1000.npy")))
    och = O.OracleChain(seq, table, synth.GEOMETRY)
    pf = synth.RunParams(precision=synth.PRECISION_FP64, solvation=2)
    ref = och.evaluate(pf, th)
    f64 = gpu_eval(kcm, seq, table, pf, th)
    mix = gpu_eval(kcm, seq, table, synth.RunParams(precision=synth.PRECISION_MIXED, solvation=2), th)
    assert rel_inf(f64["tau"], ref["tau"]) < TOL_FP64
    assert rel_inf(f64["F_cav"], ref["F_cav"]) < TOL_FP64
    assert rel_inf(mix["tau"], ref["tau"]) < TOL_MIXED
    assert rel_inf(mix["F_cav"], ref["F_cav"]) < 1e-5
    assert mix["E"][2] == pytest.approx(ref["E"][2], rel=1e-6)


def test_fp64_surrogate_trajectory_chain40(kcm, table):
    """100 FP64 iterations of the 40-residue extended chain with the surrogate on, against the oracle's
    loop (with the enumeration on, such runs diverge: its force is piecewise constant)."""
    seq = synth.sequence(40, synth.chain_seed(synth.workload(1).seed, 0))
    och = O.OracleChain(seq, table, synth.GEOMETRY)
    p = synth.RunParams(precision=synth.PRECISION_FP64, solvation=2)
    th_ref, it_ref, _, dm_ref = och.run(p, synth.theta_extended(40), 100)
    with kcm.Chain(seq, table, p) as ch:
        it, dm = ch.step(100)
        th = ch.get_theta()
    assert it == it_ref
    assert np.max(np.abs(th - th_ref)) < 1e-8
    assert abs(dm - dm_ref[-1]) < 1e-8


def test_mixed_surrogate_trajectory_rmsd_chain40(kcm, table):
    """The trajectory gate with solvation on, which the surrogate makes attainable: backbone RMSD of the
    mixed path against FP64 after 100 iterations of the 40-residue extended chain."""
    seq = synth.sequence(40, synth.chain_seed(synth.workload(1).seed, 0))
    och = O.OracleChain(seq, table, synth.GEOMETRY)
    bb = np.isin(och.kind, (0, 2, 3))  # backbone N, CA, C
    xyz = {}
    for prec in (synth.PRECISION_MIXED, synth.PRECISION_FP64):
        with kcm.Chain(seq, table, synth.RunParams(precision=prec, solvation=2)) as ch:
            ch.set_theta(synth.theta_extended(40))
            it, _ = ch.step(100)
            assert it == 100
            xyz[prec] = ch.positions()
    d = xyz[synth.PRECISION_MIXED][bb] - xyz[synth.PRECISION_FP64][bb]
    assert np.sqrt((d ** 2).sum(1).mean()) <= 1e-3


def test_batch_surrogate_matches_alone(kcm, table):
    cases = [(3, 13), (17, 14), (40, 15)]
    seqs, ths = [], []
    for m, seed in cases:
        seq = synth.sequence(m, seed)
        seqs.append(seq)
        ths.append(synth.theta_from_codes(O.OracleChain(seq, table, synth.GEOMETRY).grow_start(seed)))
    for prec, tol in ((synth.PRECISION_FP64, TOL_FP64), (synth.PRECISION_MIXED, 1e-5)):
        p = synth.RunParams(precision=prec, solvation=2)
        with kcm.Batch(seqs, table, p) as b:
            b.set_theta(np.concatenate(ths))
            tau = b.split(b.torques(), per="joint")
            E = b.chain_energies()
        for c in range(len(cases)):
            one = gpu_eval(kcm, seqs[c], table, p, ths[c])
            assert rel_inf(tau[c], one["tau"]) < tol
            assert E[c][2] == pytest.approx(one["E"][2], rel=1e-9 if prec == synth.PRECISION_FP64 else 1e-6)
