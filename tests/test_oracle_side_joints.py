"""Pins of the oracle's side-chain joints (eq. kin_05, r2: up to four rotations chi_k per residue about
successive side-chain bonds, each moving the side atoms beyond its bond; torques on the branches of
the chain, Sec. 3.5): the ZP at chi = 0, full turns, preserved bond lengths and angles, and the side-
and main-chain torques against central differences of the energy."""
import numpy as np
import pytest

from kcm_testutil import rel_inf
from oracle import oracle as O
from paper_1712_05012_b300 import synth


def chain(table, m, seed):
    seq = synth.sequence(m, seed)
    ch = O.OracleChain(seq, table, synth.GEOMETRY)
    return seq, ch


def test_chi_counts(table):
    """min(4, side atoms - 1) joints per residue: a joint turns about the bond to a side atom and
    must move at least the next one."""
    seq, ch = chain(table, 20, 11)
    want = sum(min(4, max(0, table.n_side[t] - 1)) for t in seq)
    assert ch.nside_joints == want


def test_zero_and_full_turn(table):
    seq, ch = chain(table, 8, 12)
    rng = np.random.default_rng(1)
    th = synth.theta_uniform(8, 12)
    x0, _, _ = ch.fk(th)
    x1, _, _ = ch.fk(th, side=np.zeros(ch.nside_joints))
    assert np.max(np.abs(x1 - x0)) < 1e-13
    s = rng.uniform(-np.pi, np.pi, ch.nside_joints)
    xa, _, _ = ch.fk(th, side=s)
    xb, _, _ = ch.fk(th, side=s + 2 * np.pi * rng.integers(-2, 3, ch.nside_joints))
    assert np.max(np.abs(xa - xb)) < 1e-11
    assert np.max(np.abs(xa - x0)) > 0.1  # the side groups did move


def test_bond_geometry_preserved(table):
    """Every bond length and every angle between two bonds of an atom is that of the ZP, for random
    main- and side-chain angles: the joints only turn about bonds."""
    seq, ch = chain(table, 10, 13)
    rng = np.random.default_rng(2)
    z, _, _ = ch.fk(np.zeros(ch.l))
    x, _, _ = ch.fk(synth.theta_uniform(10, 13), side=rng.uniform(-np.pi, np.pi, ch.nside_joints))
    bonds = ch.bonds()
    lz = np.linalg.norm(z[bonds[:, 0]] - z[bonds[:, 1]], axis=1)
    lx = np.linalg.norm(x[bonds[:, 0]] - x[bonds[:, 1]], axis=1)
    assert np.max(np.abs(lx - lz)) < 1e-12
    adj = [[] for _ in range(ch.n)]
    for a, b in bonds:
        adj[a].append(b)
        adj[b].append(a)
    for a in range(ch.n):
        for i in range(len(adj[a])):
            for j in range(i + 1, len(adj[a])):
                def ang(p):
                    u, v = p[adj[a][i]] - p[a], p[adj[a][j]] - p[a]
                    return np.arccos(np.dot(u, v) / np.linalg.norm(u) / np.linalg.norm(v))
                assert abs(ang(x) - ang(z)) < 1e-10


@pytest.mark.parametrize("m,seed", [(4, 14), (7, 15)])
def test_torques_are_minus_energy_gradient(table, m, seed):
    """tau = -dE/dtheta for every joint, main and side (Sec. 2.3); solvation off and a cutoff that
    covers every pair, so the pair set does not change under the differences."""
    seq, ch = chain(table, m, seed)
    th = synth.theta_from_codes(ch.grow_start(seed))
    rng = np.random.default_rng(seed)
    s = rng.uniform(-0.4, 0.4, ch.nside_joints)
    p = synth.RunParams(cutoff=500.0, solvation=0)
    r = ch.evaluate(p, th, side=s)
    h = 1e-6
    gs = np.zeros(ch.nside_joints)
    for k in range(ch.nside_joints):
        sp = s.copy(); sp[k] += h
        sm = s.copy(); sm[k] -= h
        gs[k] = (ch.evaluate(p, th, side=sp)["E"].sum() - ch.evaluate(p, th, side=sm)["E"].sum()) / (2 * h)
    assert rel_inf(r["tau_side"], -gs) < 1e-5
    gm = np.zeros(ch.l)
    for k in range(ch.l):
        tp = th.copy(); tp[k] += h
        tm = th.copy(); tm[k] -= h
        gm[k] = (ch.evaluate(p, tp, side=s)["E"].sum() - ch.evaluate(p, tm, side=s)["E"].sum()) / (2 * h)
    assert rel_inf(r["tau"], -gm) < 1e-5


def test_run_steps_side_joints(table):
    """The loop steps main and side joints as one vector: with a tiny gain every joint moves by
    kappa tau, the side joints included."""
    seq, ch = chain(table, 6, 16)
    th = synth.theta_from_codes(ch.grow_start(16))
    s = np.zeros(ch.nside_joints)
    p = synth.RunParams(solvation=0, kappa=1e-9, dtheta_max=1.0)
    r = ch.evaluate(p, th, side=s)
    th1, s1, it, _, _ = ch.run(p, th, 1, side=s)
    assert it == 1
    assert np.max(np.abs(s1 - (s + 1e-9 * r["tau_side"]))) < 1e-15
    assert np.max(np.abs(th1 - (th + 1e-9 * r["tau"]))) < 1e-14
    assert np.max(np.abs(s1 - s)) > 1e-9


def test_side_torques_with_surrogate_solvation(table):
    """With the smooth pairwise solvation surrogate on (solvation = 2) the side-chain torques still equal
    -dE/dchi, solvation energy included: the branch sums take the solvation forces too."""
    seq, ch = chain(table, 5, 17)
    th = synth.theta_from_codes(ch.grow_start(17))
    s = np.random.default_rng(17).uniform(-0.3, 0.3, ch.nside_joints)
    p = synth.RunParams(cutoff=500.0, solvation=2)
    r = ch.evaluate(p, th, side=s)
    assert np.abs(r["F_cav"]).max() > 0
    h = 1e-6
    g = np.zeros(ch.nside_joints)
    for k in range(ch.nside_joints):
        sp = s.copy(); sp[k] += h
        sm = s.copy(); sm[k] -= h
        g[k] = (ch.evaluate(p, th, side=sp)["E"].sum() - ch.evaluate(p, th, side=sm)["E"].sum()) / (2 * h)
    assert rel_inf(r["tau_side"], -g) < 1e-5


def test_no_side_joints_for_one_atom_groups(table):
    """Residue types whose side group is a single atom have no side-chain joint (nothing beyond the
    first bond to turn): a chain of them has none, and its side atoms do not move with chi."""
    one = [t for t in range(len(table.n_side)) if table.n_side[t] == 1]
    assert one
    seq = np.array([one[i % len(one)] for i in range(6)], dtype=np.int32)
    ch = O.OracleChain(seq, table, synth.GEOMETRY)
    assert ch.nside_joints == 0
    th = synth.theta_uniform(6, 3)
    x0, _, _ = ch.fk(th)
    x1, _, _ = ch.fk(th, side=np.zeros(0))
    assert np.array_equal(x0, x1)
