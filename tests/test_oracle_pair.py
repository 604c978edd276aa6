"""Pins of the oracle's pairwise Coulomb (eps = 4 d) and Lennard-Jones forces (eq. 02_2, 03_2, 03_8,
03_9) and of its 1-2/1-3/1-4 classification (Sec. 3.3), by properties that do not restate the
force formula: F = -grad E by central differences, Newton's third law, the LJ minimum, 1/d^2
scaling, cutoff inclusion, and the paper's parent-pointer tree rule for interaction types."""
import numpy as np
import pytest

from kcm_testutil import Index
from oracle import oracle as O
from paper_1712_05012_b300 import synth


def random_cluster(n, seed, box=7.0, dmin=2.2):
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < n:
        p = rng.uniform(0, box, 3)
        if all(np.linalg.norm(p - q) > dmin for q in pts):
            pts.append(p)
    xyz = np.array(pts)
    q = rng.uniform(-0.6, 0.6, n)
    eps = rng.uniform(0.02, 0.2, n)
    R = rng.uniform(1.4, 2.0, n)
    return xyz, q, eps, R


def energy_free(xyz, q, eps, R, p):
    _, E, _ = O.pair_forces_free(xyz, q, eps, R, p)
    return E.sum()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_free_force_is_minus_gradient(seed):
    xyz, q, eps, R = random_cluster(8, seed)
    p = synth.RunParams(cutoff=50.0)
    F, E, _ = O.pair_forces_free(xyz, q, eps, R, p)
    h = 1e-6
    G = np.zeros_like(xyz)
    for a in range(len(xyz)):
        for x in range(3):
            xp = xyz.copy(); xp[a, x] += h
            xm = xyz.copy(); xm[a, x] -= h
            G[a, x] = (energy_free(xp, q, eps, R, p) - energy_free(xm, q, eps, R, p)) / (2 * h)
    assert np.max(np.abs(F + G)) / np.max(np.abs(F)) < 1e-6


def test_chain_force_is_minus_gradient(table):
    """Cartesian gradient on a bonded chain: exclusions and 1-4 weights enter E and F alike."""
    m = 4
    seq = synth.sequence(m, 41)
    ch = O.OracleChain(seq, table, synth.GEOMETRY)
    codes = ch.grow_start(5)
    xyz, _, _ = ch.fk(synth.theta_from_codes(codes))
    p = synth.RunParams(cutoff=80.0, w14_elec=0.4, w14_vdw=0.7)
    F, E, _ = ch.pair_forces(xyz, p)
    h = 1e-6
    rng = np.random.default_rng(0)
    for a in rng.choice(ch.n, 12, replace=False):
        for x in range(3):
            xp = xyz.copy(); xp[a, x] += h
            xm = xyz.copy(); xm[a, x] -= h
            g = (ch.pair_forces(xp, p)[1].sum() - ch.pair_forces(xm, p)[1].sum()) / (2 * h)
            assert abs(F[a, x] + g) <= 1e-6 * max(1.0, np.max(np.abs(F)))


def test_newton_third_law(table):
    m = 30
    seq = synth.sequence(m, 43)
    ch = O.OracleChain(seq, table, synth.GEOMETRY)
    xyz, _, _ = ch.fk(synth.theta_from_codes(ch.grow_start(7)))
    F, E, npairs = ch.pair_forces(xyz, synth.RunParams())
    scale = np.max(np.abs(F))
    assert np.max(np.abs(F.sum(0))) < 1e-12 * scale * ch.n
    torque = np.cross(xyz, F).sum(0)
    assert np.max(np.abs(torque)) < 1e-11 * scale * ch.n * np.max(np.abs(xyz))
    assert npairs > 0


def test_lj_minimum_at_D():
    """eq. 03: eps [(D/d)^12 - 2 (D/d)^6] has its minimum -eps at d = D = R_i + R_j."""
    R = np.array([1.6, 1.85])
    eps = np.array([0.05, 0.18])
    q = np.zeros(2)
    p = synth.RunParams(cutoff=20.0)
    D = R.sum()
    xyz = np.array([[0.0, 0, 0], [D, 0, 0]])
    F, E, _ = O.pair_forces_free(xyz, q, eps, R, p)
    assert abs(E[1] + np.sqrt(eps[0] * eps[1])) < 1e-15
    assert np.max(np.abs(F)) < 1e-13
    for d, sign in ((0.9 * D, 1), (1.2 * D, -1)):  # repulsive inside, attractive outside
        xyz = np.array([[0.0, 0, 0], [d, 0, 0]])
        F, E, _ = O.pair_forces_free(xyz, q, eps, R, p)
        assert np.sign(F[1, 0]) == sign and np.sign(F[0, 0]) == -sign


def test_coulomb_distance_dependent_dielectric_scaling():
    """With eps_ij = 4 d the energy goes as 1/d^2 and the force as 1/d^3; like charges repel."""
    q = np.array([0.4, 0.3])
    eps = np.zeros(2)
    R = np.array([1.5, 1.5])
    p = synth.RunParams(cutoff=50.0)
    out = []
    for d in (3.0, 6.0):
        F, E, _ = O.pair_forces_free(np.array([[0.0, 0, 0], [d, 0, 0]]), q, eps, R, p)
        out.append((E[0], F[1, 0]))
    assert abs(out[1][0] * 4 - out[0][0]) < 1e-14 * abs(out[0][0])
    assert abs(out[1][1] * 8 - out[0][1]) < 1e-14 * abs(out[0][1])
    assert out[0][1] > 0
    # the paper's constant in kcal/mol units: K q q / (4 d^2) at d = 1 A is K q q / 4
    F, E, _ = O.pair_forces_free(np.array([[0.0, 0, 0], [1.0, 0, 0]]), q, eps, R, p)
    assert abs(E[0] - 332.0636 * 0.12 / 4) < 1e-12


def test_cutoff_is_inclusive():
    """eq. 02_2 neighbourhood: d <= d_cut is kept, d > d_cut dropped."""
    q = np.array([0.5, -0.5])
    eps = np.array([0.1, 0.1])
    R = np.array([1.5, 1.5])
    p = synth.RunParams(cutoff=10.0)
    F, E, n = O.pair_forces_free(np.array([[0.0, 0, 0], [10.0, 0, 0]]), q, eps, R, p)
    assert n == 1 and E[0] != 0.0
    F, E, n = O.pair_forces_free(np.array([[0.0, 0, 0], [10.000000001, 0, 0]]), q, eps, R, p)
    assert n == 0 and E[0] == 0.0 and np.all(F == 0)


def tree_rule_class(parent, a, b):
    """Sec. 3.3: 1-2 if one is the other's parent; 1-3 if grandparent or sibling; 1-4 if
    great-grandparent or sibling of the parent; otherwise farther. Checked both ways round."""
    def anc(x, k):
        for _ in range(k):
            x = parent[x]
            if x < 0:
                return -2
        return x

    def one_way(x, y):
        if anc(x, 1) == y:
            return 1
        if anc(x, 2) == y or (parent[x] >= 0 and parent[x] == parent[y]):
            return 2
        if anc(x, 3) == y or (anc(x, 2) >= 0 and parent[y] == anc(x, 2) and y != parent[x]):
            return 3
        return 4

    return min(one_way(a, b), one_way(b, a))


def test_bfs_classes_match_tree_rule(table):
    m = 7
    seq = synth.sequence(m, 47)
    ch = O.OracleChain(seq, table, synth.GEOMETRY)
    ix = Index(seq)
    # parent pointers of the bond tree rooted at N_1
    adj = {a: [] for a in range(ch.n)}
    for a, b in ch.bonds():
        adj[a].append(b)
        adj[b].append(a)
    parent = [-1] * ch.n
    seen = {ix.N(0)}
    stack = [ix.N(0)]
    while stack:
        x = stack.pop()
        for y in adj[x]:
            if y not in seen:
                seen.add(y)
                parent[y] = x
                stack.append(y)
    assert len(seen) == ch.n
    for a in range(ch.n):
        for b in range(a + 1, ch.n):
            if abs(ch.res[a] - ch.res[b]) > 1:
                assert ch.bond_distance(a, b) == 4  # the paper's shortcut: w = 1
                continue
            assert tree_rule_class(parent, a, b) == ch.bond_distance(a, b), (a, b)


@pytest.mark.parametrize("slots,cls", [((0, 2), 1), ((0, 3), 2), ((0, 4), 3), ((0, 7), 4), ((1, 5), 3)])
def test_excluded_and_14_weights(table, slots, cls):
    """Only two atoms of the middle residue carry charge and well depth: the chain energy is then
    exactly that pair's energy times w (0 for 1-2 and 1-3, w14 for 1-4, 1 beyond; eq. 03_8/9).
    Slots: 0 N, 1 H, 2 CA, 3 C, 4 O, 5.. side atoms (type 3 has four)."""
    import copy
    t2 = copy.deepcopy(table)
    t2.q[:] = 0.0
    t2.eps[:] = 0.0
    a_slot, b_slot = slots
    t2.q[3, a_slot], t2.q[3, b_slot] = 0.37, -0.52
    t2.eps[3, a_slot], t2.eps[3, b_slot] = 0.11, 0.17
    seq = np.array([0, 3, 5], dtype=np.int32)
    ch = O.OracleChain(seq, t2, synth.GEOMETRY)
    ix = Index(seq)
    slot_atom = {0: ix.N(1), 1: ix.H(1), 2: ix.CA(1), 3: ix.C(1), 4: ix.O(1)}
    for t in range(4):
        slot_atom[5 + t] = ix.S(1, t)
    a, b = slot_atom[a_slot], slot_atom[b_slot]
    assert ch.bond_distance(a, b) == cls
    xyz, _, _ = ch.fk(synth.theta_uniform(3, 3))
    p = synth.RunParams(cutoff=50, w14_elec=0.3, w14_vdw=0.6)
    _, Ec, _ = ch.pair_forces(xyz, p)
    sel = [a, b]
    _, Ef, _ = O.pair_forces_free(xyz[sel], ch.q[sel], ch.eps[sel], ch.R[sel], p)
    w_e, w_v = {1: (0, 0), 2: (0, 0), 3: (0.3, 0.6), 4: (1, 1)}[cls]
    assert Ec[0] == pytest.approx(w_e * Ef[0], rel=1e-13, abs=1e-300)
    assert Ec[1] == pytest.approx(w_v * Ef[1], rel=1e-13, abs=1e-300)
