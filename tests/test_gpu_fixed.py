"""Fixed joints (Sec. 4.1: dihedral angles held fixed so that groups of residues move as rigid bodies)
through the C ABI, against the oracle's masked loop and against the kinematic invariant."""
import json
import os

import numpy as np
import pytest

from kcm_testutil import rel_inf
from oracle import oracle as O
from paper_1712_05012_b300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def kcm():
    import torch
    assert torch.cuda.is_available()
    from paper_1712_05012_b300 import kcm as K
    K.load()
    return K


def pair_distances(x):
    return np.linalg.norm(x[:, None] - x[None], axis=-1)


@pytest.mark.parametrize("mode", [0, 1])  # per-joint clamp, the paper's normalised step
def test_fp64_masked_trajectory_chain40(kcm, table, mode):
    """The 40-residue workload with residues 10-24 held as one rigid body: FP64 loop against the
    oracle's masked loop, fixed angles bitwise unchanged."""
    seq = synth.sequence(40, synth.chain_seed(synth.workload(1).seed, 0))
    och = O.OracleChain(seq, table, synth.GEOMETRY)
    fixed = np.zeros(och.l, dtype=np.uint8)
    fixed[20:50] = 1
    th0 = synth.theta_extended(40)
    p = synth.RunParams(precision=synth.PRECISION_FP64, solvation=0, step_mode=mode)
    th_ref, it_ref, _, dm_ref = och.run(p, th0, 40, fixed=fixed)
    with kcm.Chain(seq, table, p) as ch:
        ch.set_fixed_joints(fixed)
        it, dm = ch.step(40)
        th = ch.get_theta()
    assert it == it_ref
    assert np.max(np.abs(th - th_ref)) < 1e-8
    assert abs(dm - dm_ref[-1]) < 1e-8
    assert np.array_equal(th[20:50], th0[20:50])


def test_mixed_fixed_domain_chain1000(kcm, table):
    """The 1,000-residue workload with residues 300-499 held fixed: the domain moves as one rigid
    body, the free joints move, and the mask changes only the step (torques at the same theta are
    those of the unmasked chain)."""
    man = json.load(open(os.path.join(GOLDEN, "starts.json")))["chain1000"]
    seq = synth.sequence(man["residues"], man["sequence_seed"])
    th0 = synth.theta_from_codes(np.load(os.path.join(GOLDEN, "start_chain1000.npy")))
    p = synth.RunParams(precision=synth.PRECISION_MIXED)
    fixed = np.zeros(2 * man["residues"], dtype=np.uint8)
    fixed[600:1000] = 1  # joints 600 .. 999 join links 600 .. 1000
    with kcm.Chain(seq, table, p) as ch, kcm.Chain(seq, table, p) as ref:
        ch.set_theta(th0)
        ref.set_theta(th0)
        ch.set_fixed_joints(fixed)
        assert np.array_equal(ch.torques(), ref.torques())
        x0 = ch.positions()
        ch.step(3)
        th = ch.get_theta()
        x1 = ch.positions()
    assert np.array_equal(th[600:1000], th0[600:1000])
    assert np.max(np.abs(th - th0)) > 1e-4
    och = O.OracleChain(seq, table, synth.GEOMETRY)
    g = (och.link >= 600) & (och.link <= 1000)
    assert np.max(np.abs(pair_distances(x1[g]) - pair_distances(x0[g]))) < 1e-8


def test_batch_masks_match_alone(kcm, table):
    """A batch with per-chain masks (one chain entirely fixed: it converges at once) against the
    chains alone with their masks."""
    cases = [(12, 31), (25, 32), (40, 33)]
    seqs, ths, masks = [], [], []
    for k, (m, seed) in enumerate(cases):
        seq = synth.sequence(m, seed)
        seqs.append(seq)
        ths.append(synth.theta_from_codes(O.OracleChain(seq, table, synth.GEOMETRY).grow_start(seed)))
        f = np.zeros(2 * m, dtype=np.uint8)
        if k == 0:
            f[:] = 1
        else:
            f[4:2 * m:3] = 1
        masks.append(f)
    p = synth.RunParams(precision=synth.PRECISION_FP64)
    with kcm.Batch(seqs, table, p) as b:
        b.set_theta(np.concatenate(ths))
        b.set_fixed_joints(np.concatenate(masks))
        b.step(8)
        th = b.split(b.get_theta(), per="joint")
        iters, conv, _ = b.chain_state()
    assert iters[0] == 1 and conv[0]  # nothing moves: max |dtheta| = 0 < tol
    assert np.array_equal(th[0], ths[0])
    for c in range(1, len(cases)):
        with kcm.Chain(seqs[c], table, p) as one:
            one.set_theta(ths[c])
            one.set_fixed_joints(masks[c])
            one.step(8)
            assert np.max(np.abs(th[c] - one.get_theta())) < 1e-8
        assert np.array_equal(th[c][masks[c] == 1], ths[c][masks[c] == 1])


def test_fixed_joints_arguments(kcm, table):
    with kcm.Chain(synth.sequence(5, 3), table, synth.RunParams()) as ch:
        with pytest.raises(ValueError):
            ch.set_fixed_joints(np.zeros(3))
        L = kcm.load()
        m = np.zeros(3, dtype=np.uint8)
        assert L.kcm_set_fixed_joints(ch.handle, m.ctypes.data, 3) == kcm.KCM_E_INVAL
        ch.set_fixed_joints(np.ones(ch.l))
        th0 = ch.get_theta()
        it, dm = ch.step(5)
        assert it == 1 and dm == 0.0 and np.array_equal(ch.get_theta(), th0)
        ch.set_fixed_joints(None)
        it, dm = ch.step(1)
        assert dm > 0.0
