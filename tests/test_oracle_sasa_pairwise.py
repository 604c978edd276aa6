"""Pins of the oracle's pairwise solvation surrogate (the smooth pairwise approximation of the
solvent-accessible area that preceded surface enumeration, Sec. 3.4): the buried area of two spheres
against the spherical-cap formula, the forces against central differences of the energy, Newton's
third law, and the joint torques against central differences of the total energy through the
kinematics (the surrogate is smooth, unlike the enumeration)."""
import numpy as np
import pytest

from kcm_testutil import rel_inf
from oracle import oracle as O
from paper_1712_05012_b300 import synth


def cap_area(Ri, Rj, d):
    """Area of the sphere of radius Ri (centre 0) inside the sphere of radius Rj (centre at d): a
    spherical cap of height h = (Rj^2 - (d - Ri)^2) / (2 d), area 2 pi Ri h; 0 and the whole sphere
    at the containment limits."""
    if d >= Ri + Rj or d + Rj <= Ri:
        return 0.0
    if d + Ri <= Rj:
        return 4 * np.pi * Ri ** 2
    return 2 * np.pi * Ri * (Rj ** 2 - (d - Ri) ** 2) / (2 * d)


@pytest.mark.parametrize("Ri,Rj,d", [(3.0, 3.0, 2.0), (3.2, 2.9, 4.1), (2.9, 3.4, 1.2), (3.0, 3.0, 5.999),
                                     (3.0, 3.0, 6.5), (3.4, 2.9, 0.3), (2.9, 3.4, 0.3)])
def test_two_spheres_exact(Ri, Rj, d):
    """With one neighbour the surrogate is exact: A_i = S_i - (area of sphere i inside sphere j)."""
    xyz = np.array([[0.0, 0.0, 0.0], [d, 0.0, 0.0]])
    g = np.array([0.7, 0.0])
    _, E = O.sasa_pairwise(xyz, np.array([Ri, Rj]), g)
    want = 0.7 * (4 * np.pi * Ri ** 2 - cap_area(Ri, Rj, d))
    assert E[0] == pytest.approx(want, rel=1e-13, abs=1e-12)
    assert E[1] == 0.0


def test_lone_atom_fully_exposed():
    _, E = O.sasa_pairwise(np.zeros((1, 3)), np.array([3.1]), np.array([0.012]))
    assert E[0] == pytest.approx(0.012 * 4 * np.pi * 3.1 ** 2, rel=1e-15)


def cluster(n, seed, box=7.0):
    """Random atoms at least 1.2 A apart (no offset sphere contains another)."""
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < n:
        p = rng.uniform(0, box, 3)
        if all(np.linalg.norm(p - q) > 1.2 for q in pts):
            pts.append(p)
    return np.array(pts), rng.uniform(2.8, 3.4, n), rng.uniform(-0.2, 0.02, n)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_forces_are_minus_energy_gradient(seed):
    xyz, Roff, g = cluster(12, seed)
    F, _ = O.sasa_pairwise(xyz, Roff, g)
    h = 1e-6
    G = np.zeros_like(xyz)
    for a in range(len(xyz)):
        for x in range(3):
            xp = xyz.copy(); xp[a, x] += h
            xm = xyz.copy(); xm[a, x] -= h
            G[a, x] = (O.sasa_pairwise(xp, Roff, g)[1].sum() - O.sasa_pairwise(xm, Roff, g)[1].sum()) / (2 * h)
    assert rel_inf(F, -G) < 1e-6


@pytest.mark.parametrize("seed", [4, 5])
def test_newton_third_law(seed):
    xyz, Roff, g = cluster(15, seed)
    F, _ = O.sasa_pairwise(xyz, Roff, g)
    scale = np.abs(F).max()
    assert np.abs(F.sum(axis=0)).max() < 1e-12 * scale * len(xyz)
    assert np.abs(np.cross(xyz, F).sum(axis=0)).max() < 1e-11 * scale * len(xyz)


@pytest.mark.parametrize("m,seed", [(5, 1), (9, 2)])
def test_torques_are_minus_energy_gradient(table, m, seed):
    """tau_k = -dE/dtheta_k with the surrogate on (Sec. 2.3): the pair cutoff covers every pair, so
    only the surrogate's overlap boundaries (d = Roff_i + Roff_j, where its derivative jumps) could
    disturb the central differences; none is crossed at these steps."""
    seq = synth.sequence(m, 200 + seed)
    ch = O.OracleChain(seq, table, synth.GEOMETRY)
    th = synth.theta_from_codes(ch.grow_start(seed))
    p = synth.RunParams(cutoff=500.0, solvation=2)
    r = ch.evaluate(p, th)
    h = 1e-6
    g = np.zeros(ch.l)
    for k in range(ch.l):
        tp = th.copy(); tp[k] += h
        tm = th.copy(); tm[k] -= h
        g[k] = (ch.evaluate(p, tp)["E"].sum() - ch.evaluate(p, tm)["E"].sum()) / (2 * h)
    assert rel_inf(r["tau"], -g) < 1e-5
    assert r["E"][2] != 0.0
