"""Pins of the oracle's surface enumeration (Sec. 3.4, Algorithm 1, eq. G_cav_patch, F_cav_patch,
finitediff): the sample set's geometry, an isolated sphere, the closed-form exposed area of two
overlapping spheres, the closed-form derivative of that area, exact equality of Algorithm 1's
count rules with the brute-force definition, and the zero net solvation force."""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1712_05012_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("N", [1, 7, 64, 256, 1000, 4096])
def test_sample_set_on_unit_sphere(N):
    Q = O.sample_points(N)
    assert Q.shape == (N, 3)
    assert np.max(np.abs(np.linalg.norm(Q, axis=1) - 1.0)) < 1e-15
    assert len(np.unique(np.round(Q, 12), axis=0)) == N
    if N >= 64:
        assert np.linalg.norm(Q.mean(0)) < 0.02
        # quasi-uniform: the fraction inside a polar cap of half-angle b is its area fraction
        K = round(math.sqrt(math.pi * N / 4))
        for b in (0.5, 1.0, 1.7, 2.5):
            frac = np.mean(Q[:, 2] >= math.cos(b))
            assert abs(frac - (1 - math.cos(b)) / 2) < 1.5 / K


def test_isolated_sphere_fully_exposed():
    Q = O.sample_points(256)
    r = O.sasa(np.array([[1.0, 2.0, 3.0]]), np.array([3.1]), np.array([0.012]), Q, 0.02)
    assert r["covered"][0] == 0
    assert r["E_atom"][0] == pytest.approx(4 * math.pi * 0.012 * 3.1 ** 2, rel=1e-15)
    assert np.all(r["F"] == 0)


def cap_exposed_area(Ri, Rj, d):
    """Exposed area of sphere i (radius Ri) next to sphere j at distance d (|Ri-Rj| < d < Ri+Rj)."""
    x = (d * d + Ri * Ri - Rj * Rj) / (2 * d)
    return 2 * math.pi * Ri * (Ri + x)


@pytest.mark.parametrize("d", [2.0, 4.0, 5.5])
def test_two_sphere_area_converges(d):
    Ri, Rj = 3.1, 2.7
    xyz = np.array([[0.0, 0, 0], [d * 0.6, d * 0.64, d * 0.48]])  # unit direction (0.6, 0.64, 0.48)
    exact = cap_exposed_area(Ri, Rj, d)
    errs = []
    for N in (256, 4096, 65536):
        Q = O.sample_points(N)
        r = O.sasa(xyz, np.array([Ri, Rj]), np.array([1.0, 1.0]), Q, 0.01)
        area = 4 * math.pi * Ri * Ri * (1 - r["covered"][0] / N)
        errs.append(abs(area - exact) / exact)
    assert errs[-1] < 2e-3
    assert errs[-1] < errs[0]


def test_two_sphere_force_matches_cap_derivative():
    """F = -dE/dd along the line of centres, E = gamma_i A_i(d) + gamma_j A_j(d), with
    dA_i/dd = pi Ri (1 - (Ri^2 - Rj^2)/d^2). The forward difference of Algorithm 1 with many
    samples approaches it."""
    Ri, Rj, d = 3.2, 2.9, 4.3
    gi, gj = 0.012, -0.116
    e = np.array([0.48, -0.6, 0.64])
    xyz = np.array([[0.0, 0, 0], d * e])
    N, dr = 200000, 0.02
    Q = O.sample_points(N)
    r = O.sasa(xyz, np.array([Ri, Rj]), np.array([gi, gj]), Q, dr)
    dAi = math.pi * Ri * (1 - (Ri * Ri - Rj * Rj) / (d * d))
    dAj = math.pi * Rj * (1 - (Rj * Rj - Ri * Ri) / (d * d))
    dE = gi * dAi + gj * dAj
    Fj_along = np.dot(r["F"][1], e)
    assert Fj_along == pytest.approx(-dE, rel=0.05)
    assert np.dot(r["F"][0], e) == pytest.approx(dE, rel=0.05)
    np.testing.assert_allclose(r["F"][0], -r["F"][1], rtol=0, atol=1e-12)


def random_spheres(n, seed, box=6.0):
    rng = np.random.default_rng(seed)
    xyz = rng.uniform(0, box, (n, 3))
    Roff = rng.uniform(2.8, 3.4, n)
    gamma = rng.choice([0.012, -0.116, -0.018, -0.175, -0.186, 0.0], n)
    return xyz, Roff, gamma


@pytest.mark.parametrize("seed,N,dr", [(1, 128, 0.1), (2, 96, 0.3), (3, 200, 0.05), (4, 64, 0.5)])
def test_count_rules_equal_bruteforce(seed, N, dr):
    """Algorithm 1's three-state counts (C = 0, 1, >= 2) give exactly the forward differences
    f_{i,j,s} - f_i of the definition (eq. finitediff), re-enumerated by brute force."""
    xyz, Roff, gamma = random_spheres(7, seed)
    Q = O.sample_points(N)
    a = O.sasa(xyz, Roff, gamma, Q, dr, want_counts=True)
    b = O.sasa_bruteforce(xyz, Roff, gamma, Q, dr)
    assert np.array_equal(a["covered"], b["covered"])
    n = len(xyz)
    full = np.zeros((n, n, 3), dtype=np.int64)
    cs, cand, cnt = a["cand_start"], a["cand"], a["counts"]
    for i in range(n):
        for slot in range(cs[i], cs[i + 1]):
            full[i, cand[slot]] = cnt[slot]
    assert np.array_equal(full, -b["dcount"])
    assert np.any(full != 0)
    np.testing.assert_allclose(a["F"], b["F"], rtol=0, atol=1e-12 * max(1, np.max(np.abs(b["F"]))))
    np.testing.assert_allclose(a["E_atom"], b["E_atom"], rtol=1e-15, atol=0)


def test_literal_break_drops_exchanges():
    """The printed break in the C = 0 branch stops after the first newly covering neighbour, so
    it records no more exchanges than the definition (comparison variant only)."""
    xyz, Roff, gamma = random_spheres(9, 11, box=5.0)
    Q = O.sample_points(256)
    a = O.sasa(xyz, Roff, gamma, Q, 0.3, want_counts=True)
    b = O.sasa(xyz, Roff, gamma, Q, 0.3, literal_break=True, want_counts=True)
    pos_a = np.clip(a["counts"], 0, None).sum()
    pos_b = np.clip(b["counts"], 0, None).sum()
    assert pos_b <= pos_a
    assert np.array_equal(a["covered"], b["covered"])


def test_solvation_forces_sum_to_zero(table):
    m = 25
    seq = synth.sequence(m, 61)
    ch = O.OracleChain(seq, table, synth.GEOMETRY)
    xyz, _, _ = ch.fk(synth.theta_from_codes(ch.grow_start(3)))
    p = synth.RunParams()
    r = O.sasa(xyz, ch.roff(p), ch.gamma, O.sample_points(256), p.delta_r)
    assert np.max(np.abs(r["F"])) > 0
    assert np.max(np.abs(r["F"].sum(0))) < 1e-10


def test_table3_gamma_fixture(table):
    """Atomic solvation parameters of Table 3 (Sharp et al. adjustment) per class."""
    rows = {}
    with open(os.path.join(GOLDEN, "table3_gamma.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                rows[k] = float(v)
    seq = synth.sequence(60, 71)
    ch = O.OracleChain(seq, table, synth.GEOMETRY)
    names = {synth.CLS_C: "C", synth.CLS_ON: "O/N", synth.CLS_S: "S", synth.CLS_OMINUS: "O-",
             synth.CLS_NPLUS: "N+", synth.CLS_H: "H"}
    from kcm_testutil import Index
    ix = Index(seq)
    seen = set()
    for i, t in enumerate(seq):
        slots = [0, 1, 2, 3, 4] + [5 + s for s in range(ix.nside[i])]
        atoms = [ix.N(i), ix.H(i), ix.CA(i), ix.C(i), ix.O(i)] + [ix.S(i, s) for s in range(ix.nside[i])]
        for sl, a in zip(slots, atoms):
            name = names[int(table.cls[t, sl])]
            assert ch.gamma[a] == rows[name]
            seen.add(name)
    assert {"C", "O/N", "O-", "N+", "H"} <= seen
