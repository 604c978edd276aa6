"""Seeded synthetic inputs for the KCM step: sequences, residue-type tables, geometry constants,
start angles and run parameters.

This module draws random numbers and states constants. It holds none of the method's arithmetic:
it builds no coordinates, forces, torques or sample sets. Both the CUDA path and the oracle take
what it returns as plain inputs.

Workload shape. The paper times polyalanine chains and random Ala/Cys/Ser chains (Sec. 5.2); the
generator below keeps that shape (a backbone N, H, CA, C, O per residue plus a rigid side-chain
group hung on CA) with 20 synthetic residue types whose side-group sizes span 1 to 10 atoms.

Recipe (all draws from numpy's PCG64):
  * residue type t in 0..19 has a side group of 1 + (t mod 10) atoms;
  * backbone charges N -0.40, H +0.25, CA +0.10, C +0.55, O -0.50 (net 0);
  * side-chain charges are uniform in [-0.5, 0.5], then shifted so that the residue's net charge is
    0 for types 0..15, +1 for 16..17 and -1 for 18..19;
  * LJ well depth eps ~ U[0.02, 0.2] kcal/mol and size sigma ~ U[2.8, 4.0] A per atom type
    (one draw per backbone kind, shared by all residue types; one per side-chain slot per type);
  * solvation classes (Table 3 rows plus H): backbone N, O -> O/N; CA, C -> C; H -> H; side atoms
    are C for types 0..9 and O/N for 10..15; charged types carry an N+ (16, 17) or O- (18, 19)
    atom at the tip of the group, the rest C;
  * sequences draw each residue type uniformly; the type table uses seed 1234, the workloads
    1234 + k for k = 1..5.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

N_TYPES = 20
MAX_SIDE = 10
SLOTS = 5 + MAX_SIDE  # backbone N, H, CA, C, O then side slots 1..10

# Solvation class codes (Table 3 rows, plus H which the table does not list).
CLS_C, CLS_ON, CLS_S, CLS_OMINUS, CLS_NPLUS, CLS_H = 0, 1, 2, 3, 4, 5

TYPE_TABLE_SEED = 1234

# Backbone bond lengths (A) and angles (degrees) of the synthetic chains; omega is trans (180 deg).
GEOMETRY = {
    "b_n_ca": 1.458,
    "b_ca_c": 1.525,
    "b_c_n": 1.329,
    "b_c_o": 1.231,
    "b_n_h": 1.0,
    "b_side": 1.53,
    "a_n_ca_c": 111.2,
    "a_ca_c_n": 116.2,
    "a_c_n_ca": 121.7,
    "a_ca_c_o": 120.8,
    "a_side": 109.47122063449069,  # tetrahedral, acos(-1/3) in degrees
}
GEOMETRY_KEYS = tuple(GEOMETRY.keys())

BACKBONE_Q = (-0.40, 0.25, 0.10, 0.55, -0.50)
BACKBONE_CLS = (CLS_ON, CLS_H, CLS_C, CLS_C, CLS_ON)


def n_side_of_type(t: int) -> int:
    return 1 + (t % 10)


def net_charge_of_type(t: int) -> float:
    if t < 16:
        return 0.0
    return 1.0 if t < 18 else -1.0


@dataclass
class TypeTable:
    """Per residue type: side-group size and per-slot (q, eps, sigma, solvation class).

    Slot order: 0 N, 1 H, 2 CA, 3 C, 4 O, 5.. side atoms 1..n_side (unused slots are zero).
    """

    n_side: np.ndarray  # [20] int32
    q: np.ndarray  # [20, 15] float64, e
    eps: np.ndarray  # [20, 15] float64, kcal/mol
    sigma: np.ndarray  # [20, 15] float64, A
    cls: np.ndarray  # [20, 15] int32


def type_table(seed: int = TYPE_TABLE_SEED) -> TypeTable:
    rng = np.random.default_rng(seed)
    n_side = np.array([n_side_of_type(t) for t in range(N_TYPES)], dtype=np.int32)
    q = np.zeros((N_TYPES, SLOTS))
    eps = np.zeros((N_TYPES, SLOTS))
    sigma = np.zeros((N_TYPES, SLOTS))
    cls = np.zeros((N_TYPES, SLOTS), dtype=np.int32)
    bb_eps = rng.uniform(0.02, 0.2, size=5)
    bb_sigma = rng.uniform(2.8, 4.0, size=5)
    for t in range(N_TYPES):
        q[t, :5] = BACKBONE_Q
        eps[t, :5] = bb_eps
        sigma[t, :5] = bb_sigma
        cls[t, :5] = BACKBONE_CLS
        k = int(n_side[t])
        side_q = rng.uniform(-0.5, 0.5, size=k)
        side_q += (net_charge_of_type(t) - side_q.sum()) / k
        q[t, 5:5 + k] = side_q
        eps[t, 5:5 + k] = rng.uniform(0.02, 0.2, size=k)
        sigma[t, 5:5 + k] = rng.uniform(2.8, 4.0, size=k)
        if t < 10:
            cls[t, 5:5 + k] = CLS_C
        elif t < 16:
            cls[t, 5:5 + k] = CLS_ON
        else:
            cls[t, 5:5 + k] = CLS_C
            cls[t, 5 + k - 1] = CLS_NPLUS if t < 18 else CLS_OMINUS
    return TypeTable(n_side, q, eps, sigma, cls)


def sequence(m: int, seed: int) -> np.ndarray:
    """m residue types drawn uniformly from 0..19."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, N_TYPES, size=m).astype(np.int32)


def n_atoms(res_type: np.ndarray) -> int:
    """Atom count of a chain: 5 backbone atoms plus the side group per residue."""
    return int(5 * len(res_type) + sum(n_side_of_type(int(t)) for t in res_type))


def theta_extended(m: int) -> np.ndarray:
    """The zero position: every joint angle 0, i.e. phi = psi = 180 deg (eq. theta_1, theta_2)."""
    return np.zeros(2 * m)


def theta_uniform(m: int, seed: int) -> np.ndarray:
    """Joint angles uniform in [0, 2 pi), i.e. phi, psi uniform in [-pi, pi)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 2.0 * math.pi, size=2 * m)


# Angle code used by the stored compact starts: theta = code * 2 pi / 65536, exact in float64.
ANGLE_CODE_SCALE = 2.0 * math.pi / 65536.0


def theta_from_codes(codes: np.ndarray) -> np.ndarray:
    return codes.astype(np.float64) * ANGLE_CODE_SCALE


@dataclass
class RunParams:
    cutoff: float = 10.0  # A; Coulomb and LJ unless vdw_cutoff > 0
    vdw_cutoff: float = 0.0  # A; 0 means "same as cutoff"
    kappa: float = 1e-3  # rad per kcal/mol
    dtheta_max: float = 0.02  # rad
    w14_elec: float = 0.5
    w14_vdw: float = 0.5
    r_probe: float = 1.4  # A
    delta_r: float = 0.02  # A
    coulomb_k: float = 332.0636  # kcal A / (mol e^2)
    conv_tol: float = 1e-4  # rad
    cell_size: float = 0.0  # A; 0 picks the smallest legal cell
    n_sample: int = 256
    solvation: int = 1
    precision: int = 0  # 0 = FP64, 1 = mixed (FP32 pair/solvation arithmetic, FP64 scans)
    step_mode: int = 0  # 0 = per-joint clamp of kappa*tau, 1 = the paper's kappa*tau/max|tau|
    side_joints: int = 0  # 1 = side-chain joints chi_1..chi_4 (eq. kin_05), stepped with the main chain


PRECISION_FP64 = 0
PRECISION_MIXED = 1


@dataclass
class Workload:
    name: str
    m: list  # residues per chain
    seed: int
    params: RunParams = field(default_factory=RunParams)
    iterations: int = 1
    start: str = "extended"  # extended | compact | uniform


def workload(k: int) -> Workload:
    """The five synthetic workloads (k = 1..5)."""
    seed = TYPE_TABLE_SEED + k
    if k == 1:
        return Workload("chain40_fp64_extended", [40], seed, RunParams(), 100, "extended")
    if k == 2:
        return Workload("chain1000_compact_cut10", [1000], seed, RunParams(precision=PRECISION_MIXED),
                        1000, "compact")
    if k == 3:
        return Workload("chain8000_compact_cut12", [8000], seed,
                        RunParams(cutoff=12.0, precision=PRECISION_MIXED), 500, "compact")
    if k == 4:
        rng = np.random.default_rng(seed)
        ms = rng.integers(30, 601, size=512).tolist()
        return Workload("batch512_m30_600", ms, seed, RunParams(precision=PRECISION_MIXED), 1000, "compact")
    if k == 5:
        return Workload("serve_poisson200", [], seed, RunParams(precision=PRECISION_MIXED), 5000, "compact")
    raise ValueError(k)


def chain_seed(workload_seed: int, chain_index: int) -> int:
    """Seed of chain `chain_index`'s sequence within a workload."""
    return workload_seed * 1000003 + chain_index
