"""The cell-pair tile kernel of the mixed path (KCM_PAIR_CELL_TILES, the default from 65,536 atoms on) against the
warp-per-atom kernel (KCM_PAIR_WARP_PER_ATOM) on the same inputs, and against the FP64 oracle.

Both kernels form every pair term with the same explicitly rounded FP32 operations and add it to both
atoms in exact fixed point, so the pair forces must be equal bit for bit, and with them the solvation
lists (as sets: Algorithm 1 does not depend on a list's order), the covered counts, the solvation
forces, the torques and whole trajectories. Energies are FP32 sums in a different order: 1e-5.
Workloads: chains of 1 to 97 residues, the 1,000-residue compact start with the 27-cell stencil and
with the 125-cell stencil (a 5 A cell edge), the 8,000-residue start with its 12 A cutoff, cells of
more than 32 atoms (several home chunks), and a batch of uneven chains."""
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


def start(name):
    man = json.load(open(os.path.join(GOLDEN, "starts.json")))[name]
    codes = np.load(os.path.join(GOLDEN, f"start_{name}.npy"))
    return synth.sequence(man["residues"], man["sequence_seed"]), synth.theta_from_codes(codes)


def small(table, m, seed, kind):
    seq = synth.sequence(m, seed)
    och = O.OracleChain(seq, table, synth.GEOMETRY)
    if kind == "compact":
        th = synth.theta_from_codes(och.grow_start(seed))
    elif kind == "extended":
        th = synth.theta_extended(m)
    else:
        th = synth.theta_uniform(m, seed)
    return seq, och, th


def evaluate(kcm, make, kind, theta, cell=None, steps=0, split=1):
    with make() as ch:
        ch.set_pair_kernel(kind)
        assert ch.get_pair_kernel() == kind
        ch.set_tiles(split, 1, 0)  # the tile kernel's split: warps per window and stencil row
        if cell is not None:
            ch.autotune_cell(candidates=(cell,), reps=1)
        ch.set_theta(theta)
        out = dict(tau=ch.torques(), E=ch.energy(), covered=ch.sasa_counts(), stats=ch.stats())
        out["F_pair"], out["F_cav"] = ch.force_terms()
        if steps:
            out["it"], out["dm"] = ch.step(steps)
            out["theta"] = ch.get_theta()
        return out


def compare(a, b, list_order_free=True):
    """list_order_free: the solvation result does not depend on the order of a neighbour list
    (Algorithm 1); the pairwise surrogate's FP32 product over a list does, to rounding."""
    assert np.array_equal(a["F_pair"], b["F_pair"])
    assert np.array_equal(a["covered"], b["covered"])
    for k in ("pairs", "sasa_neighbors", "max_neighbors", "guard_rechecks", "sasa_tests"):
        assert a["stats"][k] == b["stats"][k], k
    np.testing.assert_allclose(a["E"], b["E"], rtol=1e-5, atol=1e-6)
    if list_order_free:
        assert np.array_equal(a["F_cav"], b["F_cav"])
        assert np.array_equal(a["tau"], b["tau"])
    else:
        assert rel_inf(a["F_cav"], b["F_cav"]) < 1e-5
        assert rel_inf(a["tau"], b["tau"]) < 1e-5
    if "theta" in a:
        assert a["it"] == b["it"]
        assert a["dm"] == b["dm"]
        assert np.array_equal(a["theta"], b["theta"])


@pytest.mark.parametrize("m,seed,kind", [(1, 1, "uniform"), (2, 2, "uniform"), (3, 3, "compact"),
                                         (40, 1235, "extended"), (40, 1235, "compact"), (97, 9, "compact")])
@pytest.mark.parametrize("solvation", [0, 1, 2])
def test_tiles_equal_warp_kernel_small(kcm, table, m, seed, kind, solvation):
    seq, och, th = small(table, m, seed, kind)
    p = synth.RunParams(precision=synth.PRECISION_MIXED, solvation=solvation)
    mk = lambda: kcm.Chain(seq, table, p)  # noqa: E731
    # the surrogate's products follow a list's order, so its trajectories part to rounding and then grow
    # apart (chaotically from compact starts): it is compared per evaluation only
    steps = 5 if solvation != 2 else 0
    t = evaluate(kcm, mk, kcm.PAIR_CELL_TILES, th, steps=steps)
    w = evaluate(kcm, mk, kcm.PAIR_WARP_PER_ATOM, th, steps=steps)
    compare(t, w, list_order_free=solvation != 2)
    ref = och.evaluate(synth.RunParams(precision=synth.PRECISION_FP64, solvation=solvation), th)
    assert t["stats"]["pairs"] == ref["stats"]["pairs"]
    assert rel_inf(t["tau"], ref["tau"]) < 1e-4


@pytest.mark.parametrize("cell,split", [(None, 1), (None, 2), (None, 4), (5.0, 1), (5.0, 4)])
def test_tiles_equal_warp_kernel_chain1000(kcm, table, cell, split):
    """The benchmark's workload, with the 27-cell stencil (the default edge) and the 125-cell one, and
    the tile kernel's rows split over one, two or four warps."""
    seq, th = start("chain1000")
    p = synth.RunParams(precision=synth.PRECISION_MIXED)
    mk = lambda: kcm.Chain(seq, table, p)  # noqa: E731
    t = evaluate(kcm, mk, kcm.PAIR_CELL_TILES, th, cell=cell, steps=3, split=split)
    w = evaluate(kcm, mk, kcm.PAIR_WARP_PER_ATOM, th, cell=cell, steps=3)
    compare(t, w)
    och = O.OracleChain(seq, table, synth.GEOMETRY)
    ref = och.evaluate(synth.RunParams(precision=synth.PRECISION_FP64), th)
    assert t["stats"]["pairs"] == ref["stats"]["pairs"]
    assert rel_inf(t["tau"], ref["tau"]) < 1e-4
    np.testing.assert_allclose(t["E"], ref["E"], rtol=1e-5, atol=1e-3)


def test_tiles_equal_warp_kernel_chain8000(kcm, table):
    """The 8,000-residue workload (12 A cutoff) at the default edge (125-cell stencil below the range)."""
    seq, th = start("chain8000")
    p = synth.RunParams(precision=synth.PRECISION_MIXED, cutoff=12.0)
    mk = lambda: kcm.Chain(seq, table, p)  # noqa: E731
    compare(evaluate(kcm, mk, kcm.PAIR_CELL_TILES, th, cell=10.0),
            evaluate(kcm, mk, kcm.PAIR_WARP_PER_ATOM, th, cell=10.0))


def test_tiles_dense_cells(kcm, table):
    """A compact 97-residue chain on a coarse 24 A grid: cells of well over 64 atoms (three and more
    home chunks, with flushes of the home sums between staged rows) and the 1,000-residue start with a
    3.2 A probe (lists longer than the solvation kernels stage)."""
    seq, och, th = small(table, 97, 9, "compact")
    p = synth.RunParams(precision=synth.PRECISION_MIXED)
    mk = lambda: kcm.Chain(seq, table, p)  # noqa: E731
    compare(evaluate(kcm, mk, kcm.PAIR_CELL_TILES, th, cell=24.0, steps=2),
            evaluate(kcm, mk, kcm.PAIR_WARP_PER_ATOM, th, cell=24.0, steps=2))
    seq, th = start("chain1000")
    p = synth.RunParams(precision=synth.PRECISION_MIXED, r_probe=3.2)
    mk = lambda: kcm.Chain(seq, table, p)  # noqa: E731
    t = evaluate(kcm, mk, kcm.PAIR_CELL_TILES, th)
    compare(t, evaluate(kcm, mk, kcm.PAIR_WARP_PER_ATOM, th))
    assert t["stats"]["max_neighbors"] == 168


def test_tiles_batch(kcm, table):
    cases = [(1, 11, "uniform"), (3, 13, "compact"), (17, 14, "compact"), (40, 15, "extended"), (97, 16, "compact"),
             (5, 17, "uniform"), (60, 18, "compact")]
    seqs, thetas = [], []
    for m, seed, kind in cases:
        seq, _, th = small(table, m, seed, kind)
        seqs.append(seq)
        thetas.append(th)
    p = synth.RunParams(precision=synth.PRECISION_MIXED)
    mk = lambda: kcm.Batch(seqs, table, p)  # noqa: E731
    th = np.concatenate(thetas)
    compare(evaluate(kcm, mk, kcm.PAIR_CELL_TILES, th, steps=4, split=2),
            evaluate(kcm, mk, kcm.PAIR_WARP_PER_ATOM, th, steps=4))


def test_pair_kernel_choice_rules(kcm, table):
    seq, _, th = small(table, 5, 3, "uniform")
    with kcm.Chain(seq, table, synth.RunParams(precision=synth.PRECISION_MIXED)) as ch:
        assert ch.get_pair_kernel() == kcm.PAIR_WARP_PER_ATOM  # small handles: the warp-per-atom kernel
        ch.set_pair_kernel(kcm.PAIR_CELL_TILES)
        assert ch.get_pair_kernel() == kcm.PAIR_CELL_TILES
        with pytest.raises(kcm.KcmError) as e:
            ch.set_pair_kernel(7)
        assert e.value.code == kcm.KCM_E_INVAL
    with kcm.Chain(seq, table, synth.RunParams(precision=synth.PRECISION_FP64)) as ch:
        assert ch.get_pair_kernel() == kcm.PAIR_WARP_PER_ATOM
        with pytest.raises(kcm.KcmError) as e:
            ch.set_pair_kernel(kcm.PAIR_CELL_TILES)
        assert e.value.code == kcm.KCM_E_INVAL
    # from 65,536 atoms on (the 8,000-residue chain: 83,746; a batch of eight of them) the tile kernel
    seq8, _ = start("chain8000")
    mixed = synth.RunParams(precision=synth.PRECISION_MIXED, cutoff=12.0)
    with kcm.Chain(seq8, table, mixed) as ch:
        assert ch.n >= 65536 and ch.get_pair_kernel() == kcm.PAIR_CELL_TILES
    with kcm.Chain(seq8, table, synth.RunParams(precision=synth.PRECISION_FP64, cutoff=12.0)) as ch:
        assert ch.get_pair_kernel() == kcm.PAIR_WARP_PER_ATOM
    with kcm.Batch([seq8[:3000]] * 3, table, mixed) as b:  # 3 x ~31,000 atoms
        assert b.get_pair_kernel() == kcm.PAIR_CELL_TILES
    with kcm.Batch([seq8[:3000]] * 2, table, mixed) as b:  # ~63,000 atoms
        assert b.get_pair_kernel() == kcm.PAIR_WARP_PER_ATOM
