"""Helpers shared by the tests: atom indexing of the documented atom order and independent
geometric definitions (IUPAC dihedral, bond angle) used to pin the oracle and the library."""
from __future__ import annotations

import numpy as np

from paper_1712_05012_b300 import synth


class Index:
    """Atom order per residue: N, H, CA, side 1..k, C, O (links are contiguous in this order)."""

    def __init__(self, res_type):
        self.m = len(res_type)
        self.nside = [synth.n_side_of_type(int(t)) for t in res_type]
        self.first = np.cumsum([0] + [5 + k for k in self.nside])[:-1].tolist()
        self.n = int(sum(5 + k for k in self.nside))

    def N(self, i):
        return self.first[i]

    def H(self, i):
        return self.first[i] + 1

    def CA(self, i):
        return self.first[i] + 2

    def S(self, i, t):
        return self.first[i] + 3 + t

    def C(self, i):
        return self.first[i] + 3 + self.nside[i]

    def O(self, i):
        return self.first[i] + 4 + self.nside[i]


def dihedral(p0, p1, p2, p3):
    """IUPAC dihedral angle (radians, (-pi, pi]): positive when, looking from p1 to p2, the bond
    p1->p0 turns clockwise to eclipse p2->p3."""
    b0 = p0 - p1
    b1 = p2 - p1
    b2 = p3 - p2
    b1 = b1 / np.linalg.norm(b1)
    v = b0 - np.dot(b0, b1) * b1
    w = b2 - np.dot(b2, b1) * b1
    x = np.dot(v, w)
    y = np.dot(np.cross(b1, v), w)
    return np.arctan2(y, x)


def angle(p0, p1, p2):
    a = p0 - p1
    b = p2 - p1
    return np.arccos(np.clip(np.dot(a, b) / (np.linalg.norm(a) * np.linalg.norm(b)), -1, 1))


def wrap(a):
    """wrap to (-pi, pi]"""
    return (a + np.pi) % (2 * np.pi) - np.pi


def rel_inf(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / den) if den > 0 else float(np.max(np.abs(a - b)))


def tol_positions(l):
    """Parity bound (A) on atom centres after l joints. Each FP64 rotation product adds a relative
    error of a few ulp; accumulated over k products it behaves like a random walk, ~eps sqrt(k), and
    the centre at the end of the chain sums such errors times body vectors of about 1.5 A, ~eps
    l^1.5 A. Measured against an 80-bit evaluation of the same definition (tests/
    test_oracle_precision.py): the oracle 1.64 eps l^1.5 at 2,000 joints and 1.04 eps l^1.5 at 16,000
    (4.7e-10 A), the library 3e-10 A at 16,000. The bound is 4 eps l^1.5 + 1e-12: about twice the
    largest measured error, and above the sum of the two implementations' errors, which bounds their
    difference."""
    eps = 2.0 ** -52
    return 1e-12 + 4.0 * eps * l ** 1.5


def fk_extended(och, theta):
    """Atom centres of an oracle chain evaluated in 80-bit long double, in the paper's form:
    M_j = R_1 ... R_j about the ZP axes (eq. kin_04), centres as sums of rotated ZP body vectors
    (eq. kin_03, r1, r2), starting from the oracle's ZP short vectors. A higher-precision evaluation
    of the same definition, used to bound the FP64 rounding of both implementations."""
    LD = np.longdouble
    loc, nstep = och.zp_local()
    loc = loc.astype(LD)
    nstep = nstep.astype(LD)
    res = och.res
    first = np.searchsorted(res, np.arange(och.m))
    last = np.append(first[1:], och.n)
    out = np.zeros((och.n, 3), dtype=LD)

    def rot(u, th):
        th = LD(th)
        c, s = np.cos(th), np.sin(th)
        C = LD(1) - c
        return np.array([[c + u[0] * u[0] * C, u[0] * u[1] * C - u[2] * s, u[0] * u[2] * C + u[1] * s],
                         [u[1] * u[0] * C + u[2] * s, c + u[1] * u[1] * C, u[1] * u[2] * C - u[0] * s],
                         [u[2] * u[0] * C - u[1] * s, u[2] * u[1] * C + u[0] * s, c + u[2] * u[2] * C]], dtype=LD)

    M = np.eye(3, dtype=LD)
    rN = np.zeros(3, dtype=LD)
    out[first[0]] = loc[first[0]]          # N_1
    out[first[0] + 1] = loc[first[0] + 1]  # H_1
    for i in range(och.m):
        f, e = first[i], last[i]
        aCA, aC, aO = f + 2, e - 2, e - 1
        b = loc[aCA]
        M = M @ rot(b / np.sqrt(np.sum(b * b)), theta[2 * i])
        rCA = rN + M @ b
        out[aCA] = rCA
        side = np.arange(f + 3, aC)
        out[side] = rCA + (M @ (loc[side] - loc[aCA]).T).T
        v = loc[aC] - loc[aCA]
        M = M @ rot(v / np.sqrt(np.sum(v * v)), theta[2 * i + 1])
        out[aC] = rCA + M @ v
        out[aO] = rCA + M @ (loc[aO] - loc[aCA])
        if i + 1 < och.m:
            g = first[i + 1]
            out[g] = rCA + M @ (nstep[i] - loc[aCA])
            out[g + 1] = rCA + M @ (nstep[i] + loc[g + 1] - loc[aCA])
            rN = out[g]
    return out


# A 600-residue chain, extended but for two kinks of three residues each, so that its three straight
# segments point in different directions: its box (about 1,100 x 1,300 x 940 A) needs ~1.35 M cells of
# the default edge against the chain's cap of 65,536, and the grid is coarsened (edge x 1.25 per step)
# until it fits. (joint index, angle in rad) of the kinks; every other joint at the extended value.
SPARSE_KINKS = [(400, -0.9104), (401, -0.0214), (402, -0.6128), (403, -0.2325), (404, 2.2295), (405, -0.5433),
                (800, 1.5295), (801, 2.2393), (802, -0.5749), (803, -1.0016), (804, -2.5707), (805, 1.0907)]
