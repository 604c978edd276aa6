"""Pins of the oracle's chain geometry and forward kinematics (Sec. 2.1, eq. kin_02..05, r1, r2)
against geometric definitions that do not use the oracle's formulation: bond lengths and angles of
the input geometry, IUPAC dihedrals, the L-chirality (CORN) rule, and rigidity of the links."""
import math

import numpy as np
import pytest

from kcm_testutil import Index, angle, dihedral, wrap
from oracle import oracle as O
from paper_1712_05012_b300 import synth

G = synth.GEOMETRY


def chain(m, seed, table):
    seq = synth.sequence(m, seed)
    return seq, O.OracleChain(seq, table, G), Index(seq)


def expected_bond_length(ix, kind_a, kind_b):
    ks = {kind_a, kind_b}
    # kinds: 0 N, 1 H, 2 CA, 3 C, 4 O, 5 side
    if ks == {0, 1}:
        return G["b_n_h"]
    if ks == {0, 2}:
        return G["b_n_ca"]
    if ks == {2, 3}:
        return G["b_ca_c"]
    if ks == {3, 4}:
        return G["b_c_o"]
    if ks == {3, 0}:
        return G["b_c_n"]
    if 5 in ks:
        return G["b_side"]
    raise AssertionError(ks)


@pytest.mark.parametrize("start", ["zp", "random"])
def test_bond_lengths_kept(table, start):
    seq, ch, ix = chain(12, 7, table)
    th = synth.theta_extended(12) if start == "zp" else synth.theta_uniform(12, 11)
    xyz, _, _ = ch.fk(th)
    bonds = ch.bonds()
    assert len(bonds) == ch.n - 1  # the bond graph of these chains is a tree
    for a, b in bonds:
        d = np.linalg.norm(xyz[a] - xyz[b])
        assert abs(d - expected_bond_length(ix, ch.kind[a], ch.kind[b])) < 1e-12


@pytest.mark.parametrize("seed", [3, 4])
def test_bond_angles_kept(table, seed):
    seq, ch, ix = chain(10, seed, table)
    xyz, _, _ = ch.fk(synth.theta_uniform(10, seed + 100))
    r = lambda a: xyz[a]
    deg = math.radians
    ext = deg((360.0 - G["a_c_n_ca"]) / 2.0)  # H on the bisector of the external C-N-CA angle
    for i in range(ix.m):
        assert abs(angle(r(ix.N(i)), r(ix.CA(i)), r(ix.C(i))) - deg(G["a_n_ca_c"])) < 1e-12
        assert abs(angle(r(ix.CA(i)), r(ix.C(i)), r(ix.O(i))) - deg(G["a_ca_c_o"])) < 1e-12
        assert abs(angle(r(ix.H(i)), r(ix.N(i)), r(ix.CA(i))) - ext) < 1e-12
        if i + 1 < ix.m:
            assert abs(angle(r(ix.CA(i)), r(ix.C(i)), r(ix.N(i + 1))) - deg(G["a_ca_c_n"])) < 1e-12
            assert abs(angle(r(ix.C(i)), r(ix.N(i + 1)), r(ix.CA(i + 1))) - deg(G["a_c_n_ca"])) < 1e-12
            assert abs(angle(r(ix.C(i)), r(ix.N(i + 1)), r(ix.H(i + 1))) - ext) < 1e-12
            # O on the far side of C from N(i+1): the three angles at C add to 360 deg (planar sp2)
            tot = angle(r(ix.CA(i)), r(ix.C(i)), r(ix.N(i + 1))) + angle(r(ix.CA(i)), r(ix.C(i)), r(ix.O(i))) + \
                angle(r(ix.O(i)), r(ix.C(i)), r(ix.N(i + 1)))
            assert abs(tot - 2 * math.pi) < 1e-12
        k = ix.nside[i]
        # CB: bisector of N-CA-C turned out of the plane by half the tetrahedral angle
        cb = ix.S(i, 0)
        nh = (r(ix.N(i)) - r(ix.CA(i))) / G["b_n_ca"]
        chh = (r(ix.C(i)) - r(ix.CA(i))) / G["b_ca_c"]
        bis = -(nh + chh) / np.linalg.norm(nh + chh)
        dcb = (r(cb) - r(ix.CA(i))) / G["b_side"]
        assert abs(math.acos(np.dot(bis, dcb)) - deg(G["a_side"]) / 2) < 1e-12
        assert abs(angle(r(ix.N(i)), r(ix.CA(i)), r(cb)) - angle(r(ix.C(i)), r(ix.CA(i)), r(cb))) < 1e-12
        prev2, prev1 = ix.CA(i), cb
        for t in range(1, k):
            assert abs(angle(r(prev2), r(prev1), r(ix.S(i, t))) - deg(G["a_side"])) < 1e-12
            prev2, prev1 = prev1, ix.S(i, t)


def test_dihedrals_follow_theta(table):
    """phi_i = theta_{2i-1} - 180 deg and psi_i = theta_{2i} - 180 deg (eq. theta_1, theta_2) as
    IUPAC dihedrals; omega stays trans; side groups stay all-trans; O and H turn with the plane."""
    m = 9
    seq, ch, ix = chain(m, 5, table)
    th = synth.theta_uniform(m, 21)
    xyz, _, _ = ch.fk(th)
    r = lambda a: xyz[a]
    for i in range(m):
        if i > 0:
            phi = dihedral(r(ix.C(i - 1)), r(ix.N(i)), r(ix.CA(i)), r(ix.C(i)))
            assert abs(wrap(phi - (th[2 * i] - math.pi))) < 1e-11
            omega = dihedral(r(ix.CA(i - 1)), r(ix.C(i - 1)), r(ix.N(i)), r(ix.CA(i)))
            assert abs(wrap(omega - math.pi)) < 1e-11
        if i + 1 < m:
            psi = dihedral(r(ix.N(i)), r(ix.CA(i)), r(ix.C(i)), r(ix.N(i + 1)))
            assert abs(wrap(psi - (th[2 * i + 1] - math.pi))) < 1e-11
        # O anti to N(i+1): dihedral N-CA-C-O = psi + 180 deg = theta_psi
        d_o = dihedral(r(ix.N(i)), r(ix.CA(i)), r(ix.C(i)), r(ix.O(i)))
        assert abs(wrap(d_o - th[2 * i + 1])) < 1e-11
        # H cis to C across N-CA when phi = 180: dihedral H-N-CA-C = phi + 180 deg = theta_phi
        d_h = dihedral(r(ix.H(i)), r(ix.N(i)), r(ix.CA(i)), r(ix.C(i)))
        assert abs(wrap(d_h - th[2 * i])) < 1e-11
        a, b, c = ix.N(i), ix.CA(i), ix.S(i, 0)
        for t in range(1, ix.nside[i]):
            d = dihedral(r(a), r(b), r(c), r(ix.S(i, t)))
            assert abs(wrap(d - math.pi)) < 1e-11
            a, b, c = b, c, ix.S(i, t)


def test_zero_position_frame(table):
    """ZP (all theta = 0): planar backbone in the xy-plane, N_1 at the origin, CA_1 on +x, C_1 at y > 0."""
    seq, ch, ix = chain(6, 9, table)
    xyz, _, _ = ch.fk(synth.theta_extended(6))
    assert np.max(np.abs(xyz - ch.zp())) < 1e-12
    assert np.all(xyz[ix.N(0)] == 0.0)
    assert np.allclose(xyz[ix.CA(0)], [G["b_n_ca"], 0, 0], atol=0, rtol=0)
    assert xyz[ix.C(0)][1] > 0 and xyz[ix.C(0)][2] == 0.0
    for i in range(6):
        for a in (ix.N(i), ix.H(i), ix.CA(i), ix.C(i), ix.O(i)):
            assert abs(xyz[a][2]) < 1e-12


def test_cb_is_l_chirality(table):
    """CORN rule: looking from H-alpha towards CA, CO -> R -> N runs clockwise (L amino acids)."""
    seq, ch, ix = chain(5, 13, table)
    xyz, _, _ = ch.fk(synth.theta_uniform(5, 3))
    for i in range(5):
        ca = xyz[ix.CA(i)]
        dn = xyz[ix.N(i)] - ca
        dc = xyz[ix.C(i)] - ca
        dr = xyz[ix.S(i, 0)] - ca
        dn, dc, dr = (v / np.linalg.norm(v) for v in (dn, dc, dr))
        ha = -(dn + dc + dr)  # the fourth tetrahedral direction
        view = -ha / np.linalg.norm(ha)  # from H-alpha towards CA
        # clockwise seen along `view` <=> (a x b) . view > 0 for successive members
        for a, b in ((dc, dr), (dr, dn), (dn, dc)):
            assert np.dot(np.cross(a, b), view) > 0


def test_only_distal_links_move(table):
    """Turning joint k moves exactly the links k..l (Sec. 2.1; the N-terminus is anchored)."""
    m = 6
    seq, ch, ix = chain(m, 17, table)
    th = synth.theta_uniform(m, 5)
    base, _, _ = ch.fk(th)
    for k in range(2 * m):
        t2 = th.copy()
        t2[k] += 0.3
        moved, _, _ = ch.fk(t2)
        diff = np.linalg.norm(moved - base, axis=1)
        for a in range(ch.n):
            if ch.link[a] < k + 1:
                assert diff[a] == 0.0
        # atoms off the axis in distal links do move
        far = [a for a in range(ch.n) if ch.link[a] > k + 1]
        if far:
            assert max(diff[a] for a in far) > 1e-3


def test_rigid_links(table):
    m = 8
    seq, ch, ix = chain(m, 19, table)
    x0 = ch.zp()
    x1, _, _ = ch.fk(synth.theta_uniform(m, 23))
    for h in range(2 * m + 1):
        at = np.where(ch.link == h)[0]
        d0 = np.linalg.norm(x0[at, None] - x0[None, at], axis=-1)
        d1 = np.linalg.norm(x1[at, None] - x1[None, at], axis=-1)
        assert np.max(np.abs(d0 - d1)) < 1e-12


def test_axes_are_current_bonds(table):
    m = 5
    seq, ch, ix = chain(m, 29, table)
    th = synth.theta_uniform(m, 31)
    xyz, u, p = ch.fk(th)
    for i in range(m):
        e = xyz[ix.CA(i)] - xyz[ix.N(i)]
        assert np.allclose(u[2 * i], e / np.linalg.norm(e), atol=1e-14)
        assert np.allclose(p[2 * i], xyz[ix.N(i)], atol=1e-14)
        e = xyz[ix.C(i)] - xyz[ix.CA(i)]
        assert np.allclose(u[2 * i + 1], e / np.linalg.norm(e), atol=1e-14)
        assert np.allclose(p[2 * i + 1], xyz[ix.CA(i)], atol=1e-14)
