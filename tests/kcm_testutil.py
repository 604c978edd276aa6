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
    """Parity bound (A) on atom centres after l joints. The oracle multiplies l rotation matrices in
    sequence (eq. kin_04) and sums body vectors of about 1.5 A (eq. r1); each product adds a
    relative error of a few ulp, so the rotation after k joints is off by up to ~3 k eps and the
    centre at the end of the chain by up to ~sum_k 3 k eps * 1.5 A = 2.25 eps l^2 A. The bound
    takes twice that, plus 1e-12 A."""
    eps = 2.0 ** -52
    return 1e-12 + 4.5 * eps * l * l


def fk_extended(och, theta):
    """Atom centres of an oracle chain evaluated in 80-bit long double, in the paper's form:
    M_j = R_1 ... R_j about the ZP axes (eq. kin_04), centres as sums of rotated ZP offsets
    (eq. r1, r2). A higher-precision evaluation of the same definition, used to bound the FP64
    rounding of both implementations."""
    LD = np.longdouble
    zp = och.zp().astype(LD)
    link = och.link
    l = och.l
    byl = [[] for _ in range(l + 1)]
    for a in range(och.n):
        byl[link[a]].append(a)
    # the first atom of link h >= 1 lies on joint h's axis (CA for phi links, C for psi links)
    out = np.zeros_like(zp)
    out[byl[0]] = zp[byl[0]]
    M = np.eye(3, dtype=LD)
    prev_anchor_zp = zp[byl[0][0]]     # N_1
    prev_anchor_now = out[byl[0][0]]
    for h in range(1, l + 1):
        at = byl[h]
        # the axis of joint h runs from the previous link's anchor to this link's first atom
        first = at[0]
        if h % 2 == 1:   # phi: N_i -> CA_i ; the N_i of residue i belongs to the previous link
            axis_from = zp[first - 2]  # N_i (order N, H, CA)
        else:            # psi: CA_i -> C_i
            axis_from = zp[first - 1 - (len(byl[h - 1]) - 1)]  # CA_i, first atom of the previous link
        u = zp[first] - axis_from
        u = u / np.sqrt(np.sum(u * u))
        th = LD(theta[h - 1])
        c, s = np.cos(th), np.sin(th)
        C = LD(1) - c
        R = np.array([[c + u[0] * u[0] * C, u[0] * u[1] * C - u[2] * s, u[0] * u[2] * C + u[1] * s],
                      [u[1] * u[0] * C + u[2] * s, c + u[1] * u[1] * C, u[1] * u[2] * C - u[0] * s],
                      [u[2] * u[0] * C - u[1] * s, u[2] * u[1] * C + u[0] * s, c + u[2] * u[2] * C]], dtype=LD)
        # the anchor (a point on the axis, fixed by the rotation) moves with the previous links
        anchor_now = prev_anchor_now + M @ (axis_from - prev_anchor_zp)
        M = M @ R
        out[at] = anchor_now + (M @ (zp[at] - axis_from).T).T
        prev_anchor_zp, prev_anchor_now = axis_from, anchor_now
    return out
