"""Binning cell edges and the cell-edge autotuner against the oracle and against each other.

The pair set does not depend on the cell edge (Sec. 3.2 only restricts the search to nearby cells):
every edge, with the 27-cell stencil (edge >= the largest interaction range) or the 125-cell one
(edge down to half of it), must give the oracle's pair count and sample-point classifications
exactly, FP64 results within the FP64 bar and mixed results within the mixed bar. What may change
with the edge is only the rounding of the FP32 cell offsets and the order of floating-point sums.
"""
import dataclasses

import numpy as np
import pytest

from kcm_testutil import SPARSE_KINKS, rel_inf
from oracle import oracle as O
from paper_1712_05012_b300 import synth

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10
TOL_MIXED = 1e-4
# requested edges: 0 (smallest 27-cell edge), 27-cell above it, 125-cell ones, and one below the
# 125-cell minimum (raised to it)
EDGES = (0.0, 12.0, 8.0, 6.0, 5.0)


@pytest.fixture(scope="module")
def kcm():
    import torch
    assert torch.cuda.is_available()
    from paper_1712_05012_b300 import kcm as K
    K.load()
    return K


def evaluate(kcm, seq, table, p, th):
    with kcm.Chain(seq, table, p) as ch:
        ch.set_theta(th)
        out = dict(xyz=ch.positions(), tau=ch.torques(), E=ch.energy(), covered=ch.sasa_counts(), stats=ch.stats())
        out["F_pair"], out["F_cav"] = ch.force_terms()
        return out


@pytest.mark.parametrize("edge", EDGES)
@pytest.mark.parametrize("m,seed", [(40, 1235), (97, 9)])
def test_fp64_edges_vs_oracle(kcm, table, edge, m, seed):
    seq = synth.sequence(m, seed)
    och = O.OracleChain(seq, table, synth.GEOMETRY)
    th = synth.theta_from_codes(och.grow_start(seed))
    p = synth.RunParams(precision=synth.PRECISION_FP64, cell_size=edge)
    ref = och.evaluate(p, th)
    got = evaluate(kcm, seq, table, p, th)
    assert got["stats"]["pairs"] == ref["stats"]["pairs"]
    g = och.gamma != 0
    assert np.array_equal(got["covered"][g], ref["covered"][g])
    assert rel_inf(got["F_pair"], ref["F_pair"]) < TOL_FP64
    assert rel_inf(got["tau"], ref["tau"]) < TOL_FP64
    np.testing.assert_allclose(got["E"], ref["E"], rtol=TOL_FP64, atol=1e-9)
    assert got["stats"]["cell_size"] >= edge


@pytest.fixture(scope="module")
def chain1000(table):
    from test_gpu_parity import start
    seq, th = start("chain1000")
    och = O.OracleChain(seq, table, synth.GEOMETRY)
    ref = och.evaluate(synth.RunParams(precision=synth.PRECISION_FP64), th)
    return seq, th, ref


@pytest.mark.parametrize("edge", EDGES[1:])
def test_chain1000_edges(kcm, table, chain1000, edge):
    """The 1,000-residue compact workload at every edge, both precisions, against the oracle."""
    seq, th, ref = chain1000
    f64 = evaluate(kcm, seq, table, synth.RunParams(precision=synth.PRECISION_FP64, cell_size=edge), th)
    mix = evaluate(kcm, seq, table, synth.RunParams(precision=synth.PRECISION_MIXED, cell_size=edge), th)
    assert f64["stats"]["pairs"] == mix["stats"]["pairs"] == ref["stats"]["pairs"]
    # the FP32 neighbour test is padded (a superset; the overlap tests decide exactly)
    assert mix["stats"]["sasa_neighbors"] >= f64["stats"]["sasa_neighbors"]
    assert rel_inf(f64["tau"], ref["tau"]) < TOL_FP64
    assert rel_inf(mix["tau"], ref["tau"]) < TOL_MIXED
    assert np.array_equal(mix["covered"], f64["covered"])
    assert np.array_equal(mix["F_cav"], f64["F_cav"])
    for o in (f64, mix):
        s = o["stats"]["cell_size"]
        assert s >= edge
        if edge < 10.0:  # 125-cell stencil: raised to about half the largest range at most
            assert s < 10.0
    if edge >= 6.0:
        assert f64["stats"]["cell_size"] == pytest.approx(edge, abs=1e-3)


def test_batch_edges_match_alone(kcm, table):
    """A batch with the 125-cell stencil: every chain equals itself alone with the default edge."""
    cases = [(3, 13), (17, 14), (40, 15), (97, 16)]
    seqs, ths = [], []
    for m, seed in cases:
        seq = synth.sequence(m, seed)
        seqs.append(seq)
        ths.append(synth.theta_from_codes(O.OracleChain(seq, table, synth.GEOMETRY).grow_start(seed)))
    for prec, tol in ((synth.PRECISION_FP64, TOL_FP64), (synth.PRECISION_MIXED, 1e-5)):
        p = synth.RunParams(precision=prec, cell_size=6.0)
        with kcm.Batch(seqs, table, p) as b:
            b.set_theta(np.concatenate(ths))
            tau = b.split(b.torques(), per="joint")
        for c in range(len(seqs)):
            one = evaluate(kcm, seqs[c], table, dataclasses.replace(p, cell_size=0.0), ths[c])
            assert rel_inf(tau[c], one["tau"]) < tol


def test_autotune_keeps_theta_and_matches_fixed_edge(kcm, table):
    from test_gpu_parity import start
    seq, th = start("chain1000")
    p = synth.RunParams(precision=synth.PRECISION_MIXED)
    with kcm.Chain(seq, table, p) as ch:
        ch.set_theta(th)
        chosen, times = ch.autotune_cell(reps=2)
        assert chosen in kcm.CELL_CANDIDATES
        assert times.shape == (len(kcm.CELL_CANDIDATES),)
        assert np.all(np.isfinite(times)) and np.all(times > 0)
        assert times[list(kcm.CELL_CANDIDATES).index(chosen)] == times.min()
        assert np.array_equal(ch.get_theta(), th)  # evaluations only: theta untouched
        ch.step(3)
        th_tuned = ch.get_theta()
    with kcm.Chain(seq, table, dataclasses.replace(p, cell_size=chosen)) as ref:
        ref.set_theta(th)
        ref.step(3)
        # the same edge gives the same launches and fixed-order (or integer) sums: bitwise equal
        assert np.array_equal(ref.get_theta(), th_tuned)


def test_autotune_rejects_bad_arguments(kcm, table):
    with kcm.Chain(synth.sequence(5, 3), table, synth.RunParams()) as ch:
        for cand, reps in (([], 1), ([0.0], 0), ([-1.0], 1), ([float("nan")], 1), ([0.0] * 65, 1)):
            with pytest.raises(kcm.KcmError) as e:
                ch.autotune_cell(cand, reps=reps)
            assert e.value.code == kcm.KCM_E_INVAL
        ch.autotune_cell([0.0, 6.0], reps=1)  # still usable
        ch.step(1)


@pytest.mark.parametrize("prec,solv", [(synth.PRECISION_MIXED, 1), (synth.PRECISION_FP64, 1),
                                       (synth.PRECISION_MIXED, 2)])
def test_tile_shapes_give_identical_results(kcm, table, prec, solv):
    """Every tile shape (atoms per block of the pair kernel and of the solvation kernel) gives the same
    torques: each atom's work is its own warp's. Mixed mode with Algorithm 1: bitwise, trajectory
    included (its shared sums are integers and its result does not depend on the order of a
    neighbour list). To rounding otherwise: in FP64 mode the order of the atoms within a cell (drawn
    by atomic counters) orders the force sums, and the surrogate's product over a neighbour list
    follows the list's order (drawn by atomic counters too)."""
    from test_gpu_parity import start
    seq, th = start("chain1000")
    p = synth.RunParams(precision=prec, solvation=solv)
    ref_tau = ref_th = None
    shapes = [(pw, sw, 0) for pw in kcm.TILE_CHOICES for sw in kcm.TILE_CHOICES] + \
             [(pw, 1, 1) for pw in kcm.TILE_CHOICES]
    with kcm.Chain(seq, table, p) as ch:
        assert ch.get_tiles() == (1, 1, 0)
        for pw, sw, pp in shapes:
            ch.set_tiles(pw, sw, pp)
            assert ch.get_tiles() == (pw, sw, pp)
            ch.set_theta(th)
            tau = ch.torques()
            if prec == synth.PRECISION_MIXED:
                ch.step(2)
                tt = ch.get_theta()
            if ref_tau is None:
                ref_tau = tau
                ref_th = tt if prec == synth.PRECISION_MIXED else None
                continue
            if prec == synth.PRECISION_MIXED and solv == 1:
                assert np.array_equal(tau, ref_tau), (pw, sw, pp)
                assert np.array_equal(tt, ref_th), (pw, sw, pp)
            else:
                assert rel_inf(tau, ref_tau) < (1e-12 if prec == synth.PRECISION_FP64 else 1e-5), (pw, sw, pp)


def test_autotune_tiles(kcm, table):
    from test_gpu_parity import start
    seq, th = start("chain1000")
    with kcm.Chain(seq, table, synth.RunParams(precision=synth.PRECISION_MIXED)) as ch:
        ch.set_theta(th)
        tau0 = ch.torques()
        (pw, sw, pp), times = ch.autotune_tiles(reps=2)
        assert times.shape == (2, 3, 3) and np.all(np.isfinite(times)) and np.all(times > 0)
        i, j = kcm.TILE_CHOICES.index(pw), kcm.TILE_CHOICES.index(sw)
        assert times[pp, i, j] == times.min()
        assert ch.get_tiles() == (pw, sw, pp)
        assert np.array_equal(ch.get_theta(), th)  # evaluations only
        assert np.array_equal(ch.torques(), tau0)
        L = kcm.load()
        for bad in ((3, 1, 0), (1, 0, 0), (8, 4, 0), (1, 1, 2)):
            assert L.kcm_set_tiles(ch.handle, *bad) == kcm.KCM_E_INVAL
        assert ch.get_tiles() == (pw, sw, pp)
        with pytest.raises(kcm.KcmError):
            ch.autotune_tiles(reps=0)




def test_sparse_box_coarsens(kcm, table):
    """The coarsening path of both grid forms (FP64, and the mixed one in double-float and integer
    arithmetic): the cell edge grows until the cells fit the cap, the pair set and the classification
    stay the oracle's, torques within each precision's bar, and the mixed path's two binning kernels
    (each forming the same grid) agree bit for bit."""
    m = 600
    seq = synth.sequence(m, 77)
    th = synth.theta_extended(m).copy()
    for j, v in SPARSE_KINKS:
        th[j] = v
    och = O.OracleChain(seq, table, synth.GEOMETRY)
    ref = och.evaluate(synth.RunParams(precision=synth.PRECISION_FP64), th)
    f64 = evaluate(kcm, seq, table, synth.RunParams(precision=synth.PRECISION_FP64), th)
    mix = evaluate(kcm, seq, table, synth.RunParams(precision=synth.PRECISION_MIXED), th)
    for o in (f64, mix):
        assert o["stats"]["pairs"] == ref["stats"]["pairs"]
        assert o["stats"]["cell_size"] > 15.0  # coarsened from ~10 A
        assert o["stats"]["cells"] <= 65536
    g = och.gamma != 0
    assert np.array_equal(f64["covered"][g], ref["covered"][g])
    assert np.array_equal(mix["covered"], f64["covered"])
    assert rel_inf(f64["tau"], ref["tau"]) < TOL_FP64
    assert rel_inf(mix["tau"], ref["tau"]) < TOL_MIXED
    p = synth.RunParams(precision=synth.PRECISION_MIXED)
    res = []
    for kind in (kcm.BIN_CLUSTER, kcm.BIN_BLOCKS):
        with kcm.Chain(seq, table, p) as ch:
            ch.set_binning_kernel(kind)
            ch.set_theta(th)
            res.append((ch.torques(), ch.stats()["cell_size"], ch.stats()["cells"]))
    assert np.array_equal(res[0][0], res[1][0]) and res[0][1:] == res[1][1:]
