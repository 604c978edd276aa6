"""The cluster binning kernel (KCM_BIN_CLUSTER: the counting sort of a single mixed-precision chain in
one launch of one thread-block cluster) against the count and placement kernels (KCM_BIN_BLOCKS) and
against the FP64 oracle.

Both run after the same kinematics and form the cells and the cell-relative offsets with the same
double-float arithmetic (kcm_cells.cuh), so only the order of the atoms within a cell differs (ranks
from atomics). The pair sums are exact integer sums and Algorithm 1 does not depend on the order of a
list, so positions, pair and solvation forces, torques and whole trajectories are equal bit for bit;
energies are FP32 sums in another order (1e-5), and so is the pairwise surrogate's product over a list
(compared per evaluation, 1e-5). The cluster shapes cover the two ways the CTAs are
counted: by atoms (512 per CTA, at most 16; chains of up to 32,768 atoms) and by the cell cap (at most
53,248 cells per CTA); then which handles take which kernel."""
import json
import os

import numpy as np
import pytest

from kcm_testutil import rel_inf, tol_positions
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


def start(name):
    man = json.load(open(os.path.join(GOLDEN, "starts.json")))[name]
    codes = np.load(os.path.join(GOLDEN, f"start_{name}.npy"))
    return synth.sequence(man["residues"], man["sequence_seed"]), synth.theta_from_codes(codes)


def expected_ctas(n, cap):
    return min(16, max(1, -(-n // 512), -(-cap // 53248)))


def run(kcm, seq, table, p, th, kind, cell=None, steps=3):
    with kcm.Chain(seq, table, p) as ch:
        ch.set_binning_kernel(kind)
        if cell is not None:
            ch.autotune_cell(candidates=(cell,), reps=1)
        ch.set_theta(th)
        out = dict(kind=ch.get_binning_kernel(), n=ch.n, xyz=ch.positions(), tau=ch.torques(), E=ch.energy(),
                   stats=ch.stats(), covered=ch.sasa_counts())
        if steps:
            out["it"], _ = ch.step(steps)
            out["theta"] = ch.get_theta()
        return out


def check(kcm, table, seq, th, och=None, cell=None, steps=3, p=None):
    p = p or synth.RunParams(precision=synth.PRECISION_MIXED)
    order_free = p.solvation != 2  # the surrogate's FP32 product over a list follows the list's order
    steps = steps if order_free else 0
    c = run(kcm, seq, table, p, th, kcm.BIN_CLUSTER, cell, steps)
    b = run(kcm, seq, table, p, th, kcm.BIN_BLOCKS, cell, steps)
    n = c["n"]
    cap = max(8 * n, 65536) * (8 if cell is not None and cell < 10.0 else 1)
    assert c["kind"] == (kcm.BIN_CLUSTER, expected_ctas(n, cap))
    assert b["kind"] == (kcm.BIN_BLOCKS, 0)
    assert np.array_equal(c["xyz"], b["xyz"])
    for k in ("pairs", "sasa_neighbors", "max_neighbors"):
        assert c["stats"][k] == b["stats"][k], k
    assert np.array_equal(c["covered"], b["covered"])
    if order_free:
        assert np.array_equal(c["tau"], b["tau"])
    else:
        assert rel_inf(c["tau"], b["tau"]) < 1e-5
    np.testing.assert_allclose(c["E"], b["E"], rtol=1e-5, atol=1e-6)
    if steps:
        assert c["it"] == b["it"]
        assert np.array_equal(c["theta"], b["theta"])
    if och is not None:
        ref = och.evaluate(synth.RunParams(precision=synth.PRECISION_FP64, solvation=p.solvation), th)
        assert np.max(np.abs(c["xyz"] - ref["xyz"])) < tol_positions(len(th))
        assert c["stats"]["pairs"] == ref["stats"]["pairs"]
        assert rel_inf(c["tau"], ref["tau"]) < 1e-4
    return c


# residues: two CTAs by the cell cap (a single atom's residue up to ~2,000 atoms), more by the atoms
@pytest.mark.parametrize("m,solvation", [(1, 1), (2, 0), (40, 2), (97, 1), (300, 1), (450, 1)])
def test_cluster_binning_shapes(kcm, table, m, solvation):
    seq = synth.sequence(m, 100 + m)
    och = O.OracleChain(seq, table, synth.GEOMETRY)
    th = synth.theta_from_codes(och.grow_start(100 + m)) if m > 2 else synth.theta_uniform(m, m)
    check(kcm, table, seq, th, och, p=synth.RunParams(precision=synth.PRECISION_MIXED, solvation=solvation))


@pytest.mark.parametrize("cell", [None, 5.0])
def test_cluster_binning_chain1000(kcm, table, cell):
    """The benchmark's workload (10,506 atoms: 16 CTAs), at the default edge and at 5 A (the 125-cell
    stencil: a cap of 672,384 cells, 16 CTAs of 42,024)."""
    seq, th = start("chain1000")
    och = O.OracleChain(seq, table, synth.GEOMETRY)
    check(kcm, table, seq, th, och, cell=cell)


def test_cluster_binning_limits(kcm, table):
    """The largest chains it takes: 3,100 residues (about 32,000 atoms, 16 CTAs of two atoms per thread);
    the 8,000-residue chain (83,746 atoms) and a 5 A edge on it go to the blocks."""
    m = 3100
    seq = synth.sequence(m, 31)
    with kcm.Chain(seq, table, synth.RunParams(precision=synth.PRECISION_MIXED)) as ch:
        assert 32000 < ch.n <= 32768  # 32,701 atoms
    th = synth.theta_extended(m)
    check(kcm, table, seq, th, steps=0)
    seq8, th8 = start("chain8000")
    p = synth.RunParams(precision=synth.PRECISION_MIXED, cutoff=12.0)
    with kcm.Chain(seq8, table, p) as ch:
        assert ch.get_binning_kernel() == (kcm.BIN_BLOCKS, 0)


def test_binning_choice_rules(kcm, table):
    seq = synth.sequence(6, 3)
    th = synth.theta_uniform(6, 3)
    mixed = synth.RunParams(precision=synth.PRECISION_MIXED)
    with kcm.Chain(seq, table, mixed) as ch:
        assert ch.get_binning_kernel() == (kcm.BIN_CLUSTER, 2)
        with pytest.raises(kcm.KcmError) as e:
            ch.set_binning_kernel(2)
        assert e.value.code == kcm.KCM_E_INVAL
        ch.set_binning_kernel(kcm.BIN_BLOCKS)
        assert ch.get_binning_kernel() == (kcm.BIN_BLOCKS, 0)
        ch.set_binning_kernel(kcm.BIN_CLUSTER)
        ch.set_theta(th)
        assert ch.get_binning_kernel() == (kcm.BIN_CLUSTER, 2)
    # FP64 and batches take the count and placement kernels; side-chain joints do not matter
    with kcm.Chain(seq, table, synth.RunParams(precision=synth.PRECISION_FP64)) as ch:
        assert ch.get_binning_kernel() == (kcm.BIN_BLOCKS, 0)
    with kcm.Chain(seq, table, synth.RunParams(precision=synth.PRECISION_MIXED, side_joints=1)) as ch:
        assert ch.get_binning_kernel() == (kcm.BIN_CLUSTER, 2)
    with kcm.Batch([seq, seq], table, mixed) as b:
        assert b.get_binning_kernel() == (kcm.BIN_BLOCKS, 0)
