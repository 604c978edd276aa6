"""ctypes wrapper of the C oracle (orc.c) — TEST INFRASTRUCTURE ONLY.

Only the tests, the package smoke check and the benchmark's CPU-baseline leg import this module.
It takes its inputs from the synthetic generator (plain arrays) and shares nothing with the CUDA
library. See orc.c for what each function computes and which passage of the paper it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "orc.c")
LIB = os.path.join(HERE, "liborc.so")

_lock = threading.Lock()
_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile orc.c into liborc.so beside it (gcc, OpenMP)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-o", LIB, SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            L.orc_chain_new.restype = C.c_void_p
            L.orc_chain_new.argtypes = [C.c_int, _ip, _ip, _dp, _dp, _dp, _ip, _dp]
            L.orc_chain_free.argtypes = [C.c_void_p]
            L.orc_natoms.argtypes = [C.c_void_p]
            L.orc_natoms.restype = C.c_int
            L.orc_atom_info.argtypes = [C.c_void_p, _ip, _ip, _ip, _dp, _dp, _dp, _dp]
            L.orc_zp.argtypes = [C.c_void_p, _dp]
            L.orc_zp_local.argtypes = [C.c_void_p, _dp, _dp]
            L.orc_bond_distance.argtypes = [C.c_void_p, C.c_int, C.c_int]
            L.orc_bond_distance.restype = C.c_int
            L.orc_bonds.argtypes = [C.c_void_p, C.c_void_p]
            L.orc_bonds.restype = C.c_int
            L.orc_fk.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp]
            L.orc_pair_forces_chain.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp]
            L.orc_pair_forces_chain.restype = C.c_longlong
            L.orc_pair_forces_free.argtypes = [C.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
            L.orc_pair_forces_free.restype = C.c_longlong
            L.orc_sample_points.argtypes = [C.c_int, _dp]
            L.orc_sample_points.restype = C.c_int
            L.orc_sasa.argtypes = [C.c_int, _dp, _dp, _dp, C.c_int, _dp, C.c_double, C.c_int, _dp, _dp, _ip,
                                   _lp, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_sasa_ncand.argtypes = [C.c_int, _dp, _dp, C.c_double]
            L.orc_sasa_ncand.restype = C.c_int
            L.orc_sasa_bruteforce.argtypes = [C.c_int, _dp, _dp, _dp, C.c_int, _dp, C.c_double, _dp, _dp, _ip, _ip]
            L.orc_torques_columns.argtypes = [C.c_int, C.c_int, _ip, _dp, _dp, _dp, _dp, _dp]
            L.orc_torques_rowscan.argtypes = [C.c_int, C.c_int, _ip, _dp, _dp, _dp, _dp, _dp]
            L.orc_sasa_pairwise.argtypes = [C.c_int, _dp, _dp, _dp, _dp, _dp]
            L.orc_sasa_pairwise.restype = None
            L.orc_step.argtypes = [C.c_int, _dp, _dp, C.c_double, C.c_double, C.c_int, C.c_void_p, C.c_void_p]
            L.orc_step.restype = C.c_double
            L.orc_evaluate.argtypes = [C.c_void_p, _dp, _dp, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_run.argtypes = [C.c_void_p, _dp, _dp, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_run.restype = C.c_int
            L.orc_fk_x.argtypes = [C.c_void_p, _dp, C.c_void_p, _dp, C.c_void_p, C.c_void_p]
            L.orc_nside_joints.argtypes = [C.c_void_p]
            L.orc_nside_joints.restype = C.c_int
            L.orc_side_torques.argtypes = [C.c_void_p, _dp, _dp, _dp]
            L.orc_evaluate_x.argtypes = [C.c_void_p, _dp, _dp, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_run_x.argtypes = [C.c_void_p, _dp, _dp, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_run_x.restype = C.c_int
            L.orc_grow_start.argtypes = [C.c_void_p, C.c_ulonglong, C.c_double, C.c_int, C.c_int, C.c_void_p]
            L.orc_grow_start.restype = C.c_int
            L.orc_num_threads.restype = C.c_int
            L.orc_set_threads.argtypes = [C.c_int]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def set_threads(t: int) -> None:
    lib().orc_set_threads(int(t))


def num_threads() -> int:
    return int(lib().orc_num_threads())


def sample_points(N: int) -> np.ndarray:
    Q = np.zeros((N, 3))
    k = lib().orc_sample_points(N, Q.reshape(-1))
    assert k == N
    return Q


def pair_params(p) -> np.ndarray:
    return np.array([p.cutoff, p.vdw_cutoff, p.coulomb_k, p.w14_elec, p.w14_vdw], dtype=np.float64)


def run_params(p) -> np.ndarray:
    return np.array([p.cutoff, p.vdw_cutoff, p.coulomb_k, p.w14_elec, p.w14_vdw, p.r_probe, p.delta_r,
                     p.kappa, p.dtheta_max, p.conv_tol, float(p.solvation), float(p.n_sample),
                     float(p.step_mode)], dtype=np.float64)


def pair_forces_free(xyz, q, eps, R, p):
    """Pair forces/energies of free (unbonded) atoms: returns F [n,3], (E_elec, E_vdw), npairs."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    n = xyz.shape[0]
    F = np.zeros((n, 3))
    E = np.zeros(2)
    npairs = lib().orc_pair_forces_free(n, xyz.reshape(-1), np.ascontiguousarray(q, dtype=np.float64),
                                        np.ascontiguousarray(eps, dtype=np.float64),
                                        np.ascontiguousarray(R, dtype=np.float64), pair_params(p), F.reshape(-1), E)
    return F, E, int(npairs)


def sasa(xyz, Roff, gamma, Q, dr, literal_break=False, want_counts=False):
    """Algorithm 1. Returns dict with F [n,3], E_atom [n], covered [n], stats, and optionally the
    candidate lists and per-(i, candidate, s) net exchange counts."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    n = xyz.shape[0]
    Roff = np.ascontiguousarray(Roff, dtype=np.float64)
    gamma = np.ascontiguousarray(gamma, dtype=np.float64)
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    F = np.zeros((n, 3))
    Ea = np.zeros(n)
    cov = np.zeros(n, dtype=np.int32)
    stats = np.zeros(3, dtype=np.int64)
    out = {}
    cs = cand = cnt = None
    if want_counts:
        nc = lib().orc_sasa_ncand(n, xyz.reshape(-1), Roff, dr)
        cs = np.zeros(n + 1, dtype=np.int32)
        cand = np.zeros(max(nc, 1), dtype=np.int32)
        cnt = np.zeros(max(3 * nc, 1), dtype=np.int32)
    lib().orc_sasa(n, xyz.reshape(-1), Roff, gamma, Q.shape[0], Q.reshape(-1), float(dr), int(literal_break),
                   F.reshape(-1), Ea, cov, stats, _ptr(cs), _ptr(cand), _ptr(cnt))
    out.update(F=F, E_atom=Ea, covered=cov, stats=stats)
    if want_counts:
        out.update(cand_start=cs, cand=cand[:cs[-1]], counts=cnt[:3 * cs[-1]].reshape(-1, 3))
    return out


def sasa_pairwise(xyz, Roff, gamma):
    """The pairwise solvation surrogate: returns (F [n,3], E_atom [n])."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    n = xyz.shape[0]
    F = np.zeros((n, 3))
    Ea = np.zeros(n)
    lib().orc_sasa_pairwise(n, xyz.reshape(-1), np.ascontiguousarray(Roff, dtype=np.float64),
                            np.ascontiguousarray(gamma, dtype=np.float64), F.reshape(-1), Ea)
    return F, Ea


def sasa_bruteforce(xyz, Roff, gamma, Q, dr):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    n = xyz.shape[0]
    F = np.zeros((n, 3))
    Ea = np.zeros(n)
    cov = np.zeros(n, dtype=np.int32)
    dcount = np.zeros(n * n * 3, dtype=np.int32)
    lib().orc_sasa_bruteforce(n, xyz.reshape(-1), np.ascontiguousarray(Roff, dtype=np.float64),
                              np.ascontiguousarray(gamma, dtype=np.float64), Q.shape[0],
                              np.ascontiguousarray(Q).reshape(-1), float(dr), F.reshape(-1), Ea, cov, dcount)
    return dict(F=F, E_atom=Ea, covered=cov, dcount=dcount.reshape(n, n, 3))


def _mask(fixed, l):
    """Joints held fixed as a uint8 array [l] (None: none), kept alive by the caller."""
    if fixed is None:
        return None
    m = np.ascontiguousarray(fixed, dtype=np.uint8)
    assert m.shape == (l,)
    return m


def step(theta, tau, kappa, dmax, mode=0, fixed=None):
    th = np.array(theta, dtype=np.float64)
    d = np.zeros_like(th)
    m = _mask(fixed, len(th))
    dm = lib().orc_step(len(th), th, np.ascontiguousarray(tau, dtype=np.float64), kappa, dmax, mode, _ptr(d),
                        None if m is None else _ptr(m))
    return th, d, dm


class OracleChain:
    """One chain built by the oracle from a sequence, a residue-type table and geometry constants."""

    def __init__(self, res_type, table, geometry: dict):
        from paper_1712_05012_b300 import synth  # input tables only

        self.m = int(len(res_type))
        self._res_type = np.ascontiguousarray(res_type, dtype=np.int32)
        geom = np.array([geometry[k] for k in synth.GEOMETRY_KEYS], dtype=np.float64)
        self._h = lib().orc_chain_new(self.m, self._res_type, np.ascontiguousarray(table.n_side, dtype=np.int32),
                                      np.ascontiguousarray(table.q, dtype=np.float64).reshape(-1),
                                      np.ascontiguousarray(table.eps, dtype=np.float64).reshape(-1),
                                      np.ascontiguousarray(table.sigma, dtype=np.float64).reshape(-1),
                                      np.ascontiguousarray(table.cls, dtype=np.int32).reshape(-1), geom)
        self.n = int(lib().orc_natoms(self._h))
        self.l = 2 * self.m
        self.nside_joints = int(lib().orc_nside_joints(self._h))  # chi joints, residue by residue
        self.res = np.zeros(self.n, dtype=np.int32)
        self.kind = np.zeros(self.n, dtype=np.int32)
        self.link = np.zeros(self.n, dtype=np.int32)
        self.q = np.zeros(self.n)
        self.eps = np.zeros(self.n)
        self.R = np.zeros(self.n)
        self.gamma = np.zeros(self.n)
        lib().orc_atom_info(self._h, self.res, self.kind, self.link, self.q, self.eps, self.R, self.gamma)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_chain_free(h)
            self._h = None

    def zp(self):
        x = np.zeros((self.n, 3))
        lib().orc_zp(self._h, x.reshape(-1))
        return x

    def zp_local(self):
        """ZP as short vectors: (offset of each atom from its residue's N [n,3], N_i -> N_{i+1} [m,3])."""
        loc = np.zeros((self.n, 3))
        nstep = np.zeros((self.m, 3))
        lib().orc_zp_local(self._h, loc.reshape(-1), nstep.reshape(-1))
        return loc, nstep

    def bonds(self):
        nb = lib().orc_bonds(self._h, None)
        out = np.zeros(2 * nb, dtype=np.int32)
        lib().orc_bonds(self._h, out.ctypes.data_as(C.c_void_p))
        return out.reshape(nb, 2)

    def bond_distance(self, a, b):
        return int(lib().orc_bond_distance(self._h, int(a), int(b)))

    def _side(self, side):
        if side is None:
            return None
        s = np.ascontiguousarray(side, dtype=np.float64)
        assert s.shape == (self.nside_joints,)
        return s

    def fk(self, theta, side=None):
        """eq. kin_04/05 + eq. r1/r2: returns (xyz [n,3], u [l,3] current axes, p [l,3] axis points) of
        the main-chain joints; side: the side-chain joint angles (None: the ZP side groups)."""
        th = np.ascontiguousarray(theta, dtype=np.float64)
        assert th.shape == (self.l,)
        s = self._side(side)
        xyz = np.zeros((self.n, 3))
        u = np.zeros((self.l, 3))
        p = np.zeros((self.l, 3))
        lib().orc_fk_x(self._h, th, _ptr(s), xyz.reshape(-1), _ptr(u), _ptr(p))
        return xyz, u, p

    def side_torques(self, xyz, F):
        t = np.zeros(self.nside_joints)
        lib().orc_side_torques(self._h, np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1),
                               np.ascontiguousarray(F, dtype=np.float64).reshape(-1), t)
        return t

    def pair_forces(self, xyz, params):
        F = np.zeros((self.n, 3))
        E = np.zeros(2)
        npairs = lib().orc_pair_forces_chain(self._h, np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1),
                                             pair_params(params), F.reshape(-1), E)
        return F, E, int(npairs)

    def roff(self, params):
        return self.R + params.r_probe

    def torques(self, xyz, F, u, p, form="columns"):
        tau = np.zeros(self.l)
        fn = lib().orc_torques_columns if form == "columns" else lib().orc_torques_rowscan
        fn(self.n, self.l, self.link, np.ascontiguousarray(xyz).reshape(-1), np.ascontiguousarray(F).reshape(-1),
           np.ascontiguousarray(u).reshape(-1), np.ascontiguousarray(p).reshape(-1), tau)
        return tau

    def evaluate(self, params, theta, side=None):
        """Everything at theta: dict(xyz, F_pair, F_cav, tau, E[3], covered, stats); with side (the
        side-chain joint angles) also tau_side."""
        th = np.ascontiguousarray(theta, dtype=np.float64)
        s = self._side(side)
        ts = None if s is None else np.zeros(self.nside_joints)
        xyz = np.zeros((self.n, 3))
        Fp = np.zeros((self.n, 3))
        Fc = np.zeros((self.n, 3))
        tau = np.zeros(self.l)
        E = np.zeros(3)
        cov = np.zeros(self.n, dtype=np.int32)
        stats = np.zeros(4, dtype=np.int64)
        lib().orc_evaluate_x(self._h, run_params(params), th, _ptr(s), _ptr(xyz), _ptr(Fp), _ptr(Fc), _ptr(tau),
                             _ptr(ts), _ptr(E), _ptr(cov), _ptr(stats))
        out = dict(xyz=xyz, F_pair=Fp, F_cav=Fc, tau=tau, E=E, covered=cov,
                   stats=dict(pairs=int(stats[0]), sasa_tests1=int(stats[1]), sasa_tests2=int(stats[2]),
                              sasa_cand=int(stats[3])))
        if ts is not None:
            out["tau_side"] = ts
        return out

    def grow_start(self, seed, min_dist=2.5, max_retries=100, backtrack=5):
        """Compact self-avoiding random-walk start as 16-bit angle codes [2m] (input generation)."""
        codes = np.zeros(self.l, dtype=np.uint16)
        rc = lib().orc_grow_start(self._h, int(seed), float(min_dist), int(max_retries), int(backtrack),
                                  codes.ctypes.data_as(C.c_void_p))
        if rc != 0:
            raise RuntimeError("start growth ran out of attempts")
        return codes

    def run(self, params, theta, n_iters, fixed=None, side=None):
        """The KCM loop; returns (theta, iterations taken, E trace [it,3], max|dtheta| trace), and with
        side (the side-chain joint angles, stepped together with theta) (theta, side, it, Et, dt).
        fixed: main-chain joints held fixed (uint8 [l]), None for none."""
        th = np.array(theta, dtype=np.float64)
        s = None if side is None else np.array(side, dtype=np.float64)
        if s is not None:
            assert s.shape == (self.nside_joints,)
        Et = np.zeros((n_iters, 3))
        dt = np.zeros(n_iters)
        m = _mask(fixed, self.l)
        it = lib().orc_run_x(self._h, run_params(params), th, _ptr(s), int(n_iters), _ptr(Et), _ptr(dt),
                             None if m is None else _ptr(m))
        if s is not None:
            return th, s, int(it), Et[:it], dt[:it]
        return th, int(it), Et[:it], dt[:it]
