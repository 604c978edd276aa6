"""Thin ctypes binding of libkcm.so (include/kcm.h). Argument marshalling only: every step of the
KCM iteration runs in the library's CUDA kernels. Importing this module loads the library and
raises if it is missing; there is no fallback path."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkcm.so")

KCM_OK = 0
KCM_E_INVAL = -1
KCM_E_NOMEM = -2
KCM_E_CUDA = -3
KCM_E_TIMEOUT = -4
KCM_E_NONFINITE = -5
KCM_E_OVERFLOW = -6
KCM_E_NODEVICE = -8
KCM_E_CANCELLED = -9
KCM_FP64 = 0
KCM_MIXED = 1
KCM_STEP_CLAMP = 0
KCM_STEP_NORMALIZED = 1
MAX_SIDE = 10


class KcmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"kcm error {code}: {msg}")
        self.code = code


class AtomParam(C.Structure):
    _fields_ = [("q", C.c_double), ("eps", C.c_double), ("sigma", C.c_double), ("solv_class", C.c_int32),
                ("reserved", C.c_int32)]


class ResType(C.Structure):
    _fields_ = [("n_side", C.c_int32), ("reserved", C.c_int32), ("backbone", AtomParam * 5),
                ("side", AtomParam * MAX_SIDE)]


class Geometry(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("b_n_ca", "b_ca_c", "b_c_n", "b_c_o", "b_n_h", "b_side", "a_n_ca_c",
                                          "a_ca_c_n", "a_c_n_ca", "a_ca_c_o", "a_side")]


class Topology(C.Structure):
    _fields_ = [("n_res", C.c_int32), ("n_types", C.c_int32), ("res_type", C.POINTER(C.c_int32)),
                ("types", C.POINTER(ResType)), ("geometry", C.POINTER(Geometry))]


class Params(C.Structure):
    _fields_ = [("cutoff", C.c_double), ("vdw_cutoff", C.c_double), ("kappa", C.c_double),
                ("dtheta_max", C.c_double), ("w14_elec", C.c_double), ("w14_vdw", C.c_double),
                ("r_probe", C.c_double), ("delta_r", C.c_double), ("coulomb_k", C.c_double),
                ("conv_tol", C.c_double), ("cell_size", C.c_double), ("n_sample", C.c_int32),
                ("solvation", C.c_int32), ("precision", C.c_int32), ("step_mode", C.c_int32),
                ("side_joints", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("pairs", C.c_int64), ("sasa_neighbors", C.c_int64), ("max_neighbors", C.c_int64),
                ("guard_rechecks", C.c_int64), ("cells", C.c_int64), ("cell_size", C.c_double),
                ("iterations", C.c_int64), ("sasa_tests", C.c_int64)]


EXPORTS = [
    "kcm_params_default", "kcm_create", "kcm_destroy", "kcm_natoms", "kcm_njoints", "kcm_set_theta",
    "kcm_get_theta", "kcm_set_theta_dev", "kcm_get_theta_dev", "kcm_positions", "kcm_forces", "kcm_force_terms",
    "kcm_torques", "kcm_torques_dev", "kcm_energy", "kcm_sasa_counts", "kcm_step", "kcm_step_async",
    "kcm_step_status", "kcm_get_stats", "kcm_stream", "kcm_sample_points", "kcm_build_zp", "kcm_pair_class",
    "kcm_topology_natoms", "kcm_strerror", "kcm_last_error", "kcm_step_timed", "kcm_torques_noalloc",
    "kcm_create_batch", "kcm_nchains", "kcm_chain_offsets", "kcm_chain_energies", "kcm_chain_state",
    "kcm_set_chain_max_iters", "kcm_device_bytes", "kcm_server_create", "kcm_server_destroy", "kcm_server_submit",
    "kcm_server_tick", "kcm_server_poll", "kcm_server_job", "kcm_server_device_bytes", "kcm_autotune_cell",
    "kcm_set_fixed_joints", "kcm_nside_joints", "kcm_set_side_theta", "kcm_get_side_theta", "kcm_side_torques",
    "kcm_side_offsets", "kcm_set_side_theta_dev", "kcm_get_side_theta_dev", "kcm_step_host",
    "kcm_set_tiles", "kcm_get_tiles", "kcm_autotune_tiles", "kcm_server_set_admission",
    "kcm_set_pair_kernel", "kcm_get_pair_kernel", "kcm_autotune_pair_kernel", "kcm_server_cancel",
    "kcm_set_test_withhold", "kcm_set_binning_kernel", "kcm_get_binning_kernel", "kcm_set_graph_overlap",
]
PAIR_WARP_PER_ATOM, PAIR_CELL_TILES = 0, 1
BIN_BLOCKS, BIN_CLUSTER = 0, 1
TILE_CHOICES = (1, 2, 4)
AUTOTUNE_MAX = 64
# candidate cell edges of the autotuner (A): 0 is the smallest 27-cell edge; edges below the largest
# interaction range use the 125-cell stencil and are raised to the smallest legal edge for it
CELL_CANDIDATES = (0.0, 12.0, 9.0, 8.0, 7.0, 6.0, 5.0)
JOB_WAITING, JOB_RUNNING, JOB_DONE = 0, 1, 2
NOALLOC_MAX_LINKS = 32768
NUM_STAGES = 5
STAGES = ("kinematics", "binning", "pairs", "solvation", "torques_step")

_lib = None
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


def load():
    """Load libkcm.so (built in-tree by build.py); raises OSError when it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"{LIB_PATH} is missing: run `python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        h = C.c_void_p
        sig = {
            "kcm_params_default": (C.c_int, [C.POINTER(Params)]),
            "kcm_create": (C.c_int, [C.POINTER(Topology), C.POINTER(Params), C.c_void_p, C.POINTER(C.c_void_p)]),
            "kcm_destroy": (None, [h]),
            "kcm_natoms": (C.c_int64, [h]),
            "kcm_njoints": (C.c_int64, [h]),
            "kcm_set_theta": (C.c_int, [h, _dp, C.c_int64]),
            "kcm_get_theta": (C.c_int, [h, _dp, C.c_int64]),
            "kcm_set_theta_dev": (C.c_int, [h, C.c_void_p, C.c_int64]),
            "kcm_get_theta_dev": (C.c_int, [h, C.c_void_p, C.c_int64]),
            "kcm_positions": (C.c_int, [h, _dp, C.c_int64]),
            "kcm_forces": (C.c_int, [h, _dp, C.c_int64]),
            "kcm_force_terms": (C.c_int, [h, _dp, _dp, C.c_int64]),
            "kcm_torques": (C.c_int, [h, _dp, C.c_int64]),
            "kcm_torques_dev": (C.c_int, [h, C.c_void_p, C.c_int64]),
            "kcm_energy": (C.c_int, [h, _dp]),
            "kcm_sasa_counts": (C.c_int, [h, _ip, C.c_int64]),
            "kcm_step": (C.c_int, [h, C.c_int32, _ip, _dp]),
            "kcm_step_async": (C.c_int, [h, C.c_int32]),
            "kcm_step_host": (C.c_int, [h, _dp, _dp, C.c_int64, C.c_int32, _ip, _dp]),
            "kcm_step_status": (C.c_int, [h, _ip, _dp]),
            "kcm_get_stats": (C.c_int, [h, C.POINTER(Stats)]),
            "kcm_autotune_cell": (C.c_int, [h, _dp, C.c_int32, C.c_int32, _dp, _dp]),
            "kcm_set_tiles": (C.c_int, [h, C.c_int32, C.c_int32, C.c_int32]),
            "kcm_get_tiles": (C.c_int, [h, _ip, _ip, _ip]),
            "kcm_autotune_tiles": (C.c_int, [h, C.c_int32, _dp, _ip, _ip, _ip]),
            "kcm_set_pair_kernel": (C.c_int, [h, C.c_int32]),
            "kcm_get_pair_kernel": (C.c_int, [h, _ip]),
            "kcm_autotune_pair_kernel": (C.c_int, [h, C.c_int32, _dp, _ip]),
            "kcm_set_test_withhold": (C.c_int, [h, C.c_int32]),
            "kcm_set_binning_kernel": (C.c_int, [h, C.c_int32]),
            "kcm_set_graph_overlap": (C.c_int, [h, C.c_int32]),
            "kcm_get_binning_kernel": (C.c_int, [h, _ip, _ip]),
            "kcm_set_fixed_joints": (C.c_int, [h, C.c_void_p, C.c_int64]),
            "kcm_nside_joints": (C.c_int64, [h]),
            "kcm_set_side_theta": (C.c_int, [h, _dp, C.c_int64]),
            "kcm_get_side_theta": (C.c_int, [h, _dp, C.c_int64]),
            "kcm_side_torques": (C.c_int, [h, _dp, C.c_int64]),
            "kcm_set_side_theta_dev": (C.c_int, [h, C.c_void_p, C.c_int64]),
            "kcm_get_side_theta_dev": (C.c_int, [h, C.c_void_p, C.c_int64]),
            "kcm_side_offsets": (C.c_int, [h, C.POINTER(C.c_int64)]),
            "kcm_stream": (C.c_void_p, [h]),
            "kcm_sample_points": (C.c_int, [C.c_int32, _dp]),
            "kcm_build_zp": (C.c_int, [C.POINTER(Topology), _dp, _ip, C.c_int64]),
            "kcm_pair_class": (C.c_int, [C.POINTER(Topology), _ip, _ip, C.c_int64, _ip]),
            "kcm_topology_natoms": (C.c_int64, [C.POINTER(Topology)]),
            "kcm_step_timed": (C.c_int, [h, C.POINTER(C.c_float), C.c_int32, C.POINTER(C.c_float)]),
            "kcm_torques_noalloc": (C.c_int, [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                             C.c_void_p, C.c_void_p]),
            "kcm_strerror": (C.c_char_p, [C.c_int]),
            "kcm_last_error": (C.c_char_p, [h]),
            "kcm_create_batch": (C.c_int, [C.POINTER(Topology), C.c_int32, C.POINTER(Params), C.c_void_p,
                                           C.POINTER(C.c_void_p)]),
            "kcm_nchains": (C.c_int32, [h]),
            "kcm_chain_offsets": (C.c_int, [h, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
            "kcm_chain_energies": (C.c_int, [h, _dp]),
            "kcm_chain_state": (C.c_int, [h, _ip, _ip, _dp, _ip]),
            "kcm_set_chain_max_iters": (C.c_int, [h, _ip]),
            "kcm_device_bytes": (C.c_int64, [h]),
            "kcm_server_create": (C.c_int, [C.POINTER(Params), C.c_int64, C.c_int32, C.c_int32,
                                            C.POINTER(C.c_void_p)]),
            "kcm_server_destroy": (None, [C.c_void_p]),
            "kcm_server_submit": (C.c_int, [C.c_void_p, C.POINTER(Topology), _dp, C.c_int64, C.c_int32,
                                            C.POINTER(C.c_int64)]),
            "kcm_server_tick": (C.c_int, [C.c_void_p, _ip, _ip]),
            "kcm_server_poll": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.c_int32, _ip]),
            "kcm_server_job": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(JobInfo), _dp, C.c_int64]),
            "kcm_server_device_bytes": (C.c_int64, [C.c_void_p]),
            "kcm_server_set_admission": (C.c_int, [C.c_void_p, C.c_int32, C.c_double]),
            "kcm_server_cancel": (C.c_int, [C.c_void_p, C.c_int64]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc, h=None):
    if rc != KCM_OK:
        L = load()
        raise KcmError(rc, (L.kcm_last_error(h) or b"").decode() or L.kcm_strerror(rc).decode())


def _dptr(a):
    return a.ctypes.data_as(_dp)


def _iptr(a):
    return a.ctypes.data_as(_ip)


def params_struct(p) -> Params:
    """A kcm_params from any object with the same field names (e.g. synth.RunParams)."""
    s = Params()
    for name, _ in Params._fields_:
        setattr(s, name, getattr(p, name))
    return s


class JobInfo(C.Structure):
    _fields_ = [("state", C.c_int32), ("error", C.c_int32), ("iters", C.c_int32), ("converged", C.c_int32),
                ("max_dtheta", C.c_double), ("natoms", C.c_int64), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double)]


class TopologyArgs:
    """kcm_topology plus the buffers it points to (kept alive together)."""

    def __init__(self, res_type, table, geometry=None):
        self.res = np.ascontiguousarray(res_type, dtype=np.int32)
        nt = len(table.n_side)
        self.types = (ResType * nt)()
        for t in range(nt):
            rt = self.types[t]
            rt.n_side = int(table.n_side[t])
            for s in range(5):
                rt.backbone[s] = AtomParam(float(table.q[t, s]), float(table.eps[t, s]), float(table.sigma[t, s]),
                                           int(table.cls[t, s]), 0)
            for s in range(int(table.n_side[t])):
                rt.side[s] = AtomParam(float(table.q[t, 5 + s]), float(table.eps[t, 5 + s]),
                                       float(table.sigma[t, 5 + s]), int(table.cls[t, 5 + s]), 0)
        self.geom = None
        if geometry is not None:
            self.geom = Geometry(**{k: float(geometry[k]) for k, _ in Geometry._fields_})
        self.top = Topology(len(self.res), nt, _iptr(self.res), self.types,
                            C.pointer(self.geom) if self.geom is not None else None)

    def ptr(self):
        return C.byref(self.top)


def sample_points(N: int) -> np.ndarray:
    Q = np.zeros((N, 3))
    _check(load().kcm_sample_points(int(N), _dptr(Q)))
    return Q


def topology_natoms(res_type, table, geometry=None) -> int:
    t = TopologyArgs(res_type, table, geometry)
    n = load().kcm_topology_natoms(t.ptr())
    if n < 0:
        _check(int(n))
    return int(n)


def build_zp(res_type, table, geometry=None):
    t = TopologyArgs(res_type, table, geometry)
    n = topology_natoms(res_type, table, geometry)
    xyz = np.zeros((n, 3))
    link = np.zeros(n, dtype=np.int32)
    _check(load().kcm_build_zp(t.ptr(), _dptr(xyz), _iptr(link), n))
    return xyz, link


def pair_class(res_type, table, a, b, geometry=None):
    t = TopologyArgs(res_type, table, geometry)
    a = np.ascontiguousarray(a, dtype=np.int32)
    b = np.ascontiguousarray(b, dtype=np.int32)
    out = np.zeros(len(a), dtype=np.int32)
    _check(load().kcm_pair_class(t.ptr(), _iptr(a), _iptr(b), len(a), _iptr(out)))
    return out


def torques_noalloc(n_links: int, link_start_ptr: int, xyz_ptr: int, F_ptr: int, axis_ptr: int, point_ptr: int,
                    tau_ptr: int, stream: int = 0) -> None:
    """kcm_torques_noalloc on device pointers (stream-ordered; synchronise before reading tau)."""
    rc = load().kcm_torques_noalloc(int(n_links), C.c_void_p(link_start_ptr), C.c_void_p(xyz_ptr), C.c_void_p(F_ptr),
                                    C.c_void_p(axis_ptr), C.c_void_p(point_ptr), C.c_void_p(tau_ptr),
                                    C.c_void_p(stream) if stream else None)
    if rc != KCM_OK:
        raise KcmError(rc, load().kcm_strerror(rc).decode())


class Chain:
    """One chain on the current CUDA device (kcm_create ... kcm_destroy)."""

    def __init__(self, res_type, table, params, geometry=None, stream=None):
        L = load()
        self._t = TopologyArgs(res_type, table, geometry)
        self._p = params_struct(params)
        h = C.c_void_p()
        rc = L.kcm_create(self._t.ptr(), C.byref(self._p), C.c_void_p(stream) if stream else None, C.byref(h))
        if rc != KCM_OK:
            raise KcmError(rc, (L.kcm_last_error(None) or b"").decode())
        self._init_handle(h)

    def _init_handle(self, h):
        L = load()
        self._h = h
        self.n = int(L.kcm_natoms(h))
        self.l = int(L.kcm_njoints(h))
        self.nchains = int(L.kcm_nchains(h))
        ao = np.zeros(self.nchains + 1, dtype=np.int64)
        jo = np.zeros(self.nchains + 1, dtype=np.int64)
        _check(L.kcm_chain_offsets(h, ao.ctypes.data_as(C.POINTER(C.c_int64)), jo.ctypes.data_as(C.POINTER(C.c_int64))), h)
        self.atom_off, self.joint_off = ao, jo
        self.ls = int(L.kcm_nside_joints(h))
        so = np.zeros(self.nchains + 1, dtype=np.int64)
        _check(L.kcm_side_offsets(h, so.ctypes.data_as(C.POINTER(C.c_int64))), h)
        self.side_off = so

    def close(self):
        if getattr(self, "_h", None):
            load().kcm_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    def stream(self) -> int:
        return int(load().kcm_stream(self._h) or 0)

    def set_theta(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        _check(load().kcm_set_theta(self._h, _dptr(th), len(th)), self._h)

    def get_theta(self):
        th = np.zeros(self.l)
        _check(load().kcm_get_theta(self._h, _dptr(th), self.l), self._h)
        return th

    def set_side_theta(self, chi):
        """Side-chain joint angles chi [ls] (params.side_joints = 1)."""
        c = np.ascontiguousarray(chi, dtype=np.float64)
        _check(load().kcm_set_side_theta(self._h, _dptr(c), len(c)), self._h)

    def get_side_theta(self):
        c = np.zeros(self.ls)
        _check(load().kcm_get_side_theta(self._h, _dptr(c), self.ls), self._h)
        return c

    def set_side_theta_dev(self, ptr: int):
        _check(load().kcm_set_side_theta_dev(self._h, C.c_void_p(ptr), self.ls), self._h)

    def get_side_theta_dev(self, ptr: int):
        _check(load().kcm_get_side_theta_dev(self._h, C.c_void_p(ptr), self.ls), self._h)

    def side_torques(self):
        t = np.zeros(self.ls)
        _check(load().kcm_side_torques(self._h, _dptr(t), self.ls), self._h)
        return t

    def set_theta_dev(self, ptr: int, l: int):
        _check(load().kcm_set_theta_dev(self._h, C.c_void_p(ptr), l), self._h)

    def get_theta_dev(self, ptr: int, l: int):
        _check(load().kcm_get_theta_dev(self._h, C.c_void_p(ptr), l), self._h)

    def positions(self):
        x = np.zeros((self.n, 3))
        _check(load().kcm_positions(self._h, _dptr(x), self.n), self._h)
        return x

    def forces(self):
        F = np.zeros((self.n, 3))
        _check(load().kcm_forces(self._h, _dptr(F), self.n), self._h)
        return F

    def force_terms(self):
        Fp = np.zeros((self.n, 3))
        Fc = np.zeros((self.n, 3))
        _check(load().kcm_force_terms(self._h, _dptr(Fp), _dptr(Fc), self.n), self._h)
        return Fp, Fc

    def torques(self):
        t = np.zeros(self.l)
        _check(load().kcm_torques(self._h, _dptr(t), self.l), self._h)
        return t

    def torques_dev(self, ptr: int):
        _check(load().kcm_torques_dev(self._h, C.c_void_p(ptr), self.l), self._h)

    def energy(self):
        E = np.zeros(3)
        _check(load().kcm_energy(self._h, _dptr(E)), self._h)
        return E

    def sasa_counts(self):
        c = np.zeros(self.n, dtype=np.int32)
        _check(load().kcm_sasa_counts(self._h, _iptr(c), self.n), self._h)
        return c

    def step(self, n_iters: int):
        it = np.zeros(1, dtype=np.int32)
        dm = np.zeros(1)
        _check(load().kcm_step(self._h, int(n_iters), _iptr(it), _dptr(dm)), self._h)
        return int(it[0]), float(dm[0])

    def step_host(self, theta, n_iters: int):
        """From theta (host) run up to n_iters iterations and return (theta after, iterations, max
        |dtheta|), with one wait."""
        th = np.ascontiguousarray(theta, dtype=np.float64)
        out = np.zeros(self.l)
        it = np.zeros(1, dtype=np.int32)
        dm = np.zeros(1)
        _check(load().kcm_step_host(self._h, _dptr(th), _dptr(out), len(th), int(n_iters), _iptr(it), _dptr(dm)),
               self._h)
        return out, int(it[0]), float(dm[0])

    def step_async(self, n_iters: int):
        _check(load().kcm_step_async(self._h, int(n_iters)), self._h)

    def step_status(self):
        it = np.zeros(1, dtype=np.int32)
        dm = np.zeros(1)
        _check(load().kcm_step_status(self._h, _iptr(it), _dptr(dm)), self._h)
        return int(it[0]), float(dm[0])

    def step_timed(self):
        """One iteration with CUDA-event timing: (total_ms, {stage: ms})."""
        st = (C.c_float * NUM_STAGES)()
        tot = C.c_float()
        _check(load().kcm_step_timed(self._h, st, NUM_STAGES, C.byref(tot)), self._h)
        return float(tot.value), dict(zip(STAGES, [float(x) for x in st]))

    def set_fixed_joints(self, fixed=None):
        """Hold the joints flagged in fixed [l] (None releases all): they take no step."""
        if fixed is None:
            _check(load().kcm_set_fixed_joints(self._h, None, self.l), self._h)
        else:
            m = np.ascontiguousarray(fixed, dtype=np.uint8)
            if m.shape != (self.l,):
                raise ValueError(f"fixed must have {self.l} entries")
            _check(load().kcm_set_fixed_joints(self._h, m.ctypes.data_as(C.c_void_p), self.l), self._h)

    def autotune_cell(self, candidates=CELL_CANDIDATES, reps: int = 3):
        """Time an evaluation at each candidate cell edge and keep the fastest: (chosen, times_ms)."""
        cand = np.ascontiguousarray(candidates, dtype=np.float64)
        t = np.zeros(len(cand))
        ch = np.zeros(1)
        _check(load().kcm_autotune_cell(self._h, _dptr(cand), len(cand), int(reps), _dptr(t), _dptr(ch)), self._h)
        return float(ch[0]), t

    def set_tiles(self, pair_warps: int, sasa_warps: int, pair_persistent: int = 0):
        """Atoms per thread block of the pair kernel and of the solvation kernel (1, 2 or 4), and whether
        the pair kernel runs on a persistent grid."""
        _check(load().kcm_set_tiles(self._h, int(pair_warps), int(sasa_warps), int(pair_persistent)), self._h)

    def set_pair_kernel(self, kind: int):
        """PAIR_CELL_TILES or PAIR_WARP_PER_ATOM (the default of mixed handles below 65,536 atoms and of
        FP64 handles)."""
        _check(load().kcm_set_pair_kernel(self._h, int(kind)), self._h)

    def autotune_pair_kernel(self, reps: int = 3):
        """Both pair kernels (mixed precision), each with its best tile shapes; keeps the fastest:
        (kind, times_ms[2] indexed by kind)."""
        t = np.zeros(2)
        k = np.zeros(1, dtype=np.int32)
        _check(load().kcm_autotune_pair_kernel(self._h, int(reps), _dptr(t), _iptr(k)), self._h)
        return int(k[0]), t

    def set_test_withhold(self, tile: int):
        """Test only: the torque kernel never publishes this link tile's total (-1: none), so the
        waits on it time out and calls report KCM_E_TIMEOUT."""
        _check(load().kcm_set_test_withhold(self._h, int(tile)), self._h)

    def get_pair_kernel(self) -> int:
        p = np.zeros(1, dtype=np.int32)
        _check(load().kcm_get_pair_kernel(self._h, _iptr(p)), self._h)
        return int(p[0])

    def set_graph_overlap(self, on: bool):
        """Programmatic dependent launch in the captured step graphs (default on; off for handles that
        share the GPU with other streams' kernels)."""
        _check(load().kcm_set_graph_overlap(self._h, int(bool(on))), self._h)

    def set_binning_kernel(self, kind: int):
        """BIN_CLUSTER (default: the binning in one cluster launch where the chain qualifies) or
        BIN_BLOCKS (the count and placement kernels)."""
        _check(load().kcm_set_binning_kernel(self._h, int(kind)), self._h)

    def get_binning_kernel(self):
        """(kind in use, CTAs of the cluster or 0)."""
        p = np.zeros(2, dtype=np.int32)
        _check(load().kcm_get_binning_kernel(self._h, _iptr(p[:1]), _iptr(p[1:])), self._h)
        return int(p[0]), int(p[1])

    def get_tiles(self):
        """(pair_warps, sasa_warps, pair_persistent)."""
        p = np.zeros(3, dtype=np.int32)
        _check(load().kcm_get_tiles(self._h, _iptr(p[0:1]), _iptr(p[1:2]), _iptr(p[2:3])), self._h)
        return int(p[0]), int(p[1]), int(p[2])

    def autotune_tiles(self, reps: int = 3):
        """Time an evaluation with every combination of tile shapes and keep the fastest:
        ((pair_warps, sasa_warps, pair_persistent), times_ms[2, 3, 3] indexed [persistent][pair shape]
        [solvation shape], shapes by their positions in TILE_CHOICES)."""
        nt = len(TILE_CHOICES)
        t = np.zeros(2 * nt * nt)
        p = np.zeros(3, dtype=np.int32)
        _check(load().kcm_autotune_tiles(self._h, int(reps), _dptr(t), _iptr(p[0:1]), _iptr(p[1:2]), _iptr(p[2:3])),
               self._h)
        return (int(p[0]), int(p[1]), int(p[2])), t.reshape(2, nt, nt)

    def stats(self) -> dict:
        s = Stats()
        _check(load().kcm_get_stats(self._h, C.byref(s)), self._h)
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def chain_energies(self):
        """Coulomb, LJ and solvation energies of every chain at the current theta: [nchains, 3]."""
        E = np.zeros((self.nchains, 3))
        _check(load().kcm_chain_energies(self._h, _dptr(E)), self._h)
        return E

    def set_chain_max_iters(self, caps=None):
        """Per-chain iteration caps for later step calls (None removes them)."""
        if caps is None:
            _check(load().kcm_set_chain_max_iters(self._h, None), self._h)
        else:
            a = np.ascontiguousarray(caps, dtype=np.int32)
            _check(load().kcm_set_chain_max_iters(self._h, _iptr(a)), self._h)

    def device_bytes(self) -> int:
        return int(load().kcm_device_bytes(self._h))

    def chain_state(self, with_errors=False):
        """(iterations, stopped, max |dtheta| of the last step[, status]) per chain since the last step
        call."""
        it = np.zeros(self.nchains, dtype=np.int32)
        cv = np.zeros(self.nchains, dtype=np.int32)
        dm = np.zeros(self.nchains)
        er = np.zeros(self.nchains, dtype=np.int32)
        _check(load().kcm_chain_state(self._h, _iptr(it), _iptr(cv), _dptr(dm), _iptr(er)), self._h)
        return (it, cv.astype(bool), dm, er) if with_errors else (it, cv.astype(bool), dm)


class Batch(Chain):
    """Independent chains stepped together in one handle (kcm_create_batch): atoms and joints of the
    chains are concatenated in order (atom_off, joint_off); every per-atom or per-joint method of
    Chain covers the whole batch."""

    def __init__(self, seqs, table, params, geometry=None, stream=None):
        L = load()
        self._ts = [TopologyArgs(s, table, geometry) for s in seqs]
        tops = (Topology * len(self._ts))(*[t.top for t in self._ts])
        self._tops = tops
        self._p = params_struct(params)
        h = C.c_void_p()
        rc = L.kcm_create_batch(tops, len(self._ts), C.byref(self._p), C.c_void_p(stream) if stream else None,
                                C.byref(h))
        if rc != KCM_OK:
            raise KcmError(rc, (L.kcm_last_error(None) or b"").decode())
        self._init_handle(h)

    def split(self, x, per="atom"):
        """The per-chain pieces of a batch array (per atom, joint or side-chain joint)."""
        off = {"atom": self.atom_off, "joint": self.joint_off, "side": self.side_off}[per]
        return [x[off[c]:off[c + 1]] for c in range(self.nchains)]


class Server:
    """The serving loop (kcm_server_*): submit jobs, tick, poll retired jobs, read their results."""

    def __init__(self, params, hbm_budget_bytes: int, max_chains_per_batch: int = 512, chunk_iters: int = 50):
        L = load()
        self._p = params_struct(params)
        s = C.c_void_p()
        _check(L.kcm_server_create(C.byref(self._p), int(hbm_budget_bytes), int(max_chains_per_batch),
                                   int(chunk_iters), C.byref(s)))
        self._s = s
        self._tops = {}

    def close(self):
        if getattr(self, "_s", None):
            load().kcm_server_destroy(self._s)
            self._s = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit(self, res_type, table, theta0, max_iters: int, geometry=None) -> int:
        t = TopologyArgs(res_type, table, geometry)
        th = np.ascontiguousarray(theta0, dtype=np.float64)
        jid = C.c_int64()
        _check(load().kcm_server_submit(self._s, t.ptr(), _dptr(th), len(th), int(max_iters), C.byref(jid)))
        self._tops[int(jid.value)] = len(th)
        return int(jid.value)

    def set_admission(self, min_jobs: int = 1, max_wait_s: float = 0.0):
        """Admit waiting jobs once min_jobs wait or the oldest has waited max_wait_s (or nothing runs)."""
        _check(load().kcm_server_set_admission(self._s, int(min_jobs), float(max_wait_s)))

    def cancel(self, job_id: int):
        """Cancel a waiting or running job (it ends with KCM_E_CANCELLED)."""
        _check(load().kcm_server_cancel(self._s, int(job_id)))

    def tick(self):
        w = np.zeros(1, dtype=np.int32)
        r = np.zeros(1, dtype=np.int32)
        _check(load().kcm_server_tick(self._s, _iptr(w), _iptr(r)))
        return int(w[0]), int(r[0])

    def poll(self, capacity: int = 4096):
        ids = np.zeros(capacity, dtype=np.int64)
        n = np.zeros(1, dtype=np.int32)
        _check(load().kcm_server_poll(self._s, ids.ctypes.data_as(C.POINTER(C.c_int64)), capacity, _iptr(n)))
        return [int(x) for x in ids[:n[0]]]

    def job(self, job_id: int, with_theta: bool = True):
        info = JobInfo()
        l = self._tops[job_id]
        th = np.zeros(l) if with_theta else None
        _check(load().kcm_server_job(self._s, int(job_id), C.byref(info), _dptr(th) if with_theta else None,
                                     l if with_theta else 0))
        d = {k: getattr(info, k) for k, _ in JobInfo._fields_}
        if with_theta:
            d["theta"] = th
        return d

    def device_bytes(self) -> int:
        return int(load().kcm_server_device_bytes(self._s))

