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
