"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same seeded inputs.

Tolerances:
  * positions: FP64 kinematics in both. The oracle multiplies the l rotations in sequence, whose
    rounding grows with l (bound: kcm_testutil.tol_positions, 4 eps l^1.5 A, checked against an
    80-bit evaluation); the library composes local link-frame transforms in a chunked scan and is
    checked against the 80-bit evaluation directly, to the same bound (measured: 3e-10 A at 16,000
    joints, where the oracle itself is 5e-10 A from it).
  * FP64 mode: forces, energies and torques to 1e-10 relative (max-norm), the library's stated
    FP64 bar; sample-point classifications and pair sets are compared exactly (integers).
  * mixed mode (FP32 pair and solvation arithmetic, FP64 kinematics/scans): torques to 1e-4
    relative per evaluation, the bar stated for the 1,000-residue workload; classifications
    are re-decided in FP64 inside a guard band, so covered counts and the pair set must equal
    the FP64 mode's exactly.
"""
import json
import os

import numpy as np
import pytest

from kcm_testutil import fk_extended, rel_inf, tol_positions
from oracle import oracle as O
from paper_1712_05012_b300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TOL_FP64 = 1e-10
TOL_MIXED = 1e-4


@pytest.fixture(scope="module")
def kcm():
    import torch
    assert torch.cuda.is_available()
    from paper_1712_05012_b300 import kcm as K
    K.load()
    return K


def start(name):
    man = json.load(open(os.path.join(GOLDEN, "starts.json")))[name]
    codes = np.load(os.path.join(GOLDEN, f"start_{name}.npy"))
    seq = synth.sequence(man["residues"], man["sequence_seed"])
    return seq, synth.theta_from_codes(codes)


def small_case(table, m, seed, kind="compact"):
    seq = synth.sequence(m, seed)
    och = O.OracleChain(seq, table, synth.GEOMETRY)
    if kind == "compact":
        th = synth.theta_from_codes(och.grow_start(seed))
    elif kind == "extended":
        th = synth.theta_extended(m)
    else:
        th = synth.theta_uniform(m, seed)
    return seq, och, th


def gpu_eval(kcm, seq, table, p, theta):
    with kcm.Chain(seq, table, p) as ch:
        ch.set_theta(theta)
        out = dict(xyz=ch.positions(), tau=ch.torques(), E=ch.energy(), covered=ch.sasa_counts(),
                   stats=ch.stats())
        out["F_pair"], out["F_cav"] = ch.force_terms()
        return out


@pytest.mark.parametrize("m,seed,kind", [(1, 1, "uniform"), (2, 2, "uniform"), (3, 3, "compact"),
                                         (40, 1235, "extended"), (40, 1235, "compact"), (97, 9, "compact")])
def test_fp64_parity_small(kcm, table, m, seed, kind):
    seq, och, th = small_case(table, m, seed, kind)
    p = synth.RunParams(precision=synth.PRECISION_FP64)
    ref = och.evaluate(p, th)
    got = gpu_eval(kcm, seq, table, p, th)
    assert np.max(np.abs(got["xyz"] - ref["xyz"])) < tol_positions(och.l)
    assert rel_inf(got["F_pair"], ref["F_pair"]) < TOL_FP64
    g = och.gamma != 0
    assert np.array_equal(got["covered"][g], ref["covered"][g])
    if np.any(ref["F_cav"]):
        assert rel_inf(got["F_cav"], ref["F_cav"]) < TOL_FP64
    assert rel_inf(got["tau"], ref["tau"]) < TOL_FP64
    np.testing.assert_allclose(got["E"], ref["E"], rtol=TOL_FP64, atol=1e-9)
    assert got["stats"]["pairs"] == ref["stats"]["pairs"]


@pytest.mark.parametrize("m,seed,kind", [(1, 1, "uniform"), (2, 2, "uniform"), (3, 3, "compact"),
                                         (40, 1235, "compact")])
def test_mixed_solvation_small(kcm, table, m, seed, kind):
    """Algorithm 1 in the mixed kernel on chains whose atoms have from one to a few dozen solvation
    neighbours (odd and even list lengths; step 1 takes the neighbours two at a time): classifications,
    exchange counts and forces equal the FP64 kernel's bit for bit, and the oracle's."""
    seq, och, th = small_case(table, m, seed, kind)
    pf = synth.RunParams(precision=synth.PRECISION_FP64)
    ref = och.evaluate(pf, th)
    mixed = gpu_eval(kcm, seq, table, synth.RunParams(precision=synth.PRECISION_MIXED), th)
    fp64 = gpu_eval(kcm, seq, table, pf, th)
    # the mixed lists also hold the pairs within the guard band of the range test (decided later)
    assert mixed["stats"]["sasa_neighbors"] >= fp64["stats"]["sasa_neighbors"] > 0
    assert np.array_equal(mixed["covered"], fp64["covered"])
    assert np.array_equal(mixed["F_cav"], fp64["F_cav"])
    g = och.gamma != 0
    assert np.array_equal(mixed["covered"][g], ref["covered"][g])
    if np.any(ref["F_cav"]):
        assert rel_inf(mixed["F_cav"], ref["F_cav"]) < TOL_FP64


@pytest.mark.parametrize("solvation", [0, 1])
def test_mixed_parity_chain1000(kcm, table, solvation):
    """The 1,000-residue compact workload in the launch configuration the benchmark times."""
    seq, th = start("chain1000")
    och = O.OracleChain(seq, table, synth.GEOMETRY)
    pm = synth.RunParams(precision=synth.PRECISION_MIXED, solvation=solvation)
    pf = synth.RunParams(precision=synth.PRECISION_FP64, solvation=solvation)
    ref = och.evaluate(pf, th)
    mixed = gpu_eval(kcm, seq, table, pm, th)
    fp64 = gpu_eval(kcm, seq, table, pf, th)
    assert rel_inf(fp64["tau"], ref["tau"]) < TOL_FP64
    assert rel_inf(mixed["tau"], ref["tau"]) < TOL_MIXED
    assert np.max(np.abs(fp64["xyz"] - fk_extended(och, th))) < tol_positions(och.l)
    assert np.max(np.abs(fp64["xyz"] - ref["xyz"])) < tol_positions(och.l)
    # mixed-mode kinematics runs in double-float (about 48 bits): within 1e-9 A of FP64 at ~300 A
    assert np.max(np.abs(mixed["xyz"] - fp64["xyz"])) < 1e-9
    assert mixed["stats"]["pairs"] == fp64["stats"]["pairs"] == ref["stats"]["pairs"]
    assert np.array_equal(mixed["covered"], fp64["covered"])
    # identical classifications and integer exchange counts: bitwise-equal solvation forces
    assert np.array_equal(mixed["F_cav"], fp64["F_cav"])
    np.testing.assert_allclose(mixed["E"], ref["E"], rtol=1e-5, atol=1e-3)
    if solvation:
        g = och.gamma != 0
        assert np.array_equal(fp64["covered"][g], ref["covered"][g])
        assert rel_inf(fp64["F_cav"], ref["F_cav"]) < TOL_FP64


def test_fp64_trajectory_chain40(kcm, table):
    """The 40-residue extended-start workload: 100 FP64 iterations against the oracle's loop."""
    seq = synth.sequence(40, synth.chain_seed(synth.workload(1).seed, 0))
    och = O.OracleChain(seq, table, synth.GEOMETRY)
    for solvation in (0, 1):
        p = synth.RunParams(precision=synth.PRECISION_FP64, solvation=solvation)
        th_ref, it_ref, _, dm_ref = och.run(p, synth.theta_extended(40), 100)
        with kcm.Chain(seq, table, p) as ch:
            it, dm = ch.step(100)
            th = ch.get_theta()
        assert it == it_ref
        assert np.max(np.abs(th - th_ref)) < 1e-8
        assert abs(dm - dm_ref[-1]) < 1e-8


def test_mixed_trajectory_rmsd_chain40(kcm, table):
    """Trajectory gate of the mixed path: backbone (N, CA, C) RMSD against the FP64 path after 100
    iterations of the 40-residue extended chain with solvation off (a smooth trajectory; measured
    1.4e-4 A). From the compact 1,000-residue start the trajectory is chaotic: two FP64 runs that
    differ only in the order of the pair sums already differ by 0.06 A after two iterations and by
    hundreds of A after ten, so there the gate is per-iteration torque parity (same theta in)."""
    seq = synth.sequence(40, synth.chain_seed(synth.workload(1).seed, 0))
    och = O.OracleChain(seq, table, synth.GEOMETRY)
    bb = np.isin(och.kind, (0, 2, 3))  # backbone N, CA, C
    xyz = {}
    for prec in (synth.PRECISION_MIXED, synth.PRECISION_FP64):
        p = synth.RunParams(precision=prec, solvation=0)
        with kcm.Chain(seq, table, p) as ch:
            ch.set_theta(synth.theta_extended(40))
            it, _ = ch.step(100)
            assert it == 100
            xyz[prec] = ch.positions()
    d = xyz[synth.PRECISION_MIXED][bb] - xyz[synth.PRECISION_FP64][bb]
    assert np.sqrt((d ** 2).sum(1).mean()) <= 1e-3


def test_step_rules(kcm, table):
    seq, och, th = small_case(table, 10, 5)
    p = synth.RunParams(precision=synth.PRECISION_FP64)
    ref = och.evaluate(p, th)
    for mode in (0, 1):
        p = synth.RunParams(precision=synth.PRECISION_FP64, step_mode=mode, kappa=0.05 if mode else 1e-3)
        want, _, dmax = O.step(th, ref["tau"], p.kappa, p.dtheta_max, mode)
        with kcm.Chain(seq, table, p) as ch:
            ch.set_theta(th)
            it, dm = ch.step(1)
            got = ch.get_theta()
        assert it == 1
        assert np.max(np.abs(got - want)) < 1e-12
        assert abs(dm - dmax) < 1e-12
    # convergence: a tiny gain stops after the first iteration
    p = synth.RunParams(precision=synth.PRECISION_FP64, kappa=1e-14)
    with kcm.Chain(seq, table, p) as ch:
        ch.set_theta(th)
        it, dm = ch.step(50)
    assert it == 1 and dm < p.conv_tol


def test_deterministic(kcm, table):
    seq, th = start("chain1000")
    p = synth.RunParams(precision=synth.PRECISION_MIXED)
    with kcm.Chain(seq, table, p) as ch:
        ch.set_theta(th)
        t1 = ch.torques()
        t2 = ch.torques()
        ch.step(5)
        a = ch.get_theta()
        ch.set_theta(th)
        ch.step(5)
        b = ch.get_theta()
    assert np.array_equal(t1, t2)
    assert np.array_equal(a, b)


def test_overflow_is_reported(kcm, table):
    """A huge probe radius gives the atoms of a compact ~1,000-atom chain far more solvation neighbours
    than the list holds."""
    seq, och, th = small_case(table, 97, 9, "compact")
    p = synth.RunParams(r_probe=9.0)
    with kcm.Chain(seq, table, p) as ch:
        ch.set_theta(th)
        with pytest.raises(kcm.KcmError) as e:
            ch.torques()
        assert e.value.code == kcm.KCM_E_OVERFLOW


def test_invalid_theta_rejected(kcm, table):
    seq, och, th = small_case(table, 4, 2)
    with kcm.Chain(seq, table, synth.RunParams()) as ch:
        bad = th.copy()
        bad[1] = np.nan
        with pytest.raises(kcm.KcmError) as e:
            ch.set_theta(bad)
        assert e.value.code == kcm.KCM_E_INVAL
        with pytest.raises(kcm.KcmError):
            ch.set_theta(th[:-1])


def test_step_host_round_trip(kcm, table):
    """kcm_step_host (theta in, iterations, theta out, one wait) equals kcm_set_theta + kcm_step +
    kcm_get_theta (bitwise: the mixed path sums its forces in fixed point), and refuses a non-finite
    theta."""
    import torch
    seq, och, th = small_case(table, 20, 7)
    p = synth.RunParams(precision=synth.PRECISION_MIXED)
    with kcm.Chain(seq, table, p) as a, kcm.Chain(seq, table, p) as b:
        pin = torch.tensor(th, dtype=torch.float64).pin_memory()
        out, it, dm = a.step_host(pin.numpy(), 5)
        b.set_theta(th)
        it2, dm2 = b.step(5)
        assert (it, dm) == (it2, dm2)
        assert np.array_equal(out, b.get_theta())
        assert np.array_equal(a.get_theta(), out)
        bad = th.copy()
        bad[3] = np.inf
        with pytest.raises(kcm.KcmError) as e:
            a.step_host(bad, 1)
        assert e.value.code == kcm.KCM_E_INVAL


def host_vs_device(kcm, make, theta, n_iters, prepare=None):
    """kcm_step_host with both buffers (the angles and the status record through page-locked mapped
    memory, no copies on the stream) against kcm_set_theta + kcm_step + kcm_get_theta on a second handle:
    theta, iterations and max |dtheta| bitwise; then the first handle's device state agrees."""
    with make() as a, make() as b:
        if prepare:
            prepare(a)
            prepare(b)
        out, it, dm = a.step_host(theta, n_iters)
        b.set_theta(theta)
        it2, dm2 = b.step(n_iters)
        assert (it, dm) == (it2, dm2)
        assert np.array_equal(out, b.get_theta())
        assert np.array_equal(a.get_theta(), out)
        assert np.array_equal(a.torques(), b.torques())
        # the ordinary graphs after the exchange graphs, and the exchange graphs again
        a.set_theta(theta)
        assert a.step(n_iters) == (it2, dm2)
        assert np.array_equal(a.get_theta(), out)
        out2, it3, dm3 = a.step_host(theta, n_iters)
        assert (it3, dm3) == (it2, dm2) and np.array_equal(out2, out)
        return it


@pytest.mark.parametrize("precision,step_mode,n_iters", [(synth.PRECISION_MIXED, 0, 1),
                                                         (synth.PRECISION_FP64, 1, 4),
                                                         (synth.PRECISION_MIXED, 1, 3)])
def test_step_host_exchange(kcm, table, precision, step_mode, n_iters):
    """Both step rules and precisions, with fixed joints (they take no step: their angle in the
    exchange buffer is the one read in)."""
    seq, och, th = small_case(table, 30, 11)
    p = synth.RunParams(precision=precision, step_mode=step_mode)
    fixed = (np.arange(len(th)) % 5 == 0).astype(np.uint8)
    host_vs_device(kcm, lambda: kcm.Chain(seq, table, p), th, n_iters, lambda c: c.set_fixed_joints(fixed))


def test_step_host_exchange_side_joints(kcm, table):
    """With side-chain joints the exchange carries the main-chain angles only; the side-chain angles
    stay on the device and step with them (equal to the device loop's, bitwise)."""
    seq, och, th = small_case(table, 25, 12)
    p = synth.RunParams(precision=synth.PRECISION_MIXED, side_joints=1)
    with kcm.Chain(seq, table, p) as a, kcm.Chain(seq, table, p) as b:
        chi = np.linspace(-0.3, 0.3, a.ls)
        a.set_side_theta(chi)
        b.set_side_theta(chi)
        out, it, dm = a.step_host(th, 3)
        b.set_theta(th)
        assert b.step(3) == (it, dm)
        assert np.array_equal(out, b.get_theta())
        assert np.array_equal(a.get_side_theta(), b.get_side_theta())
        assert not np.array_equal(a.get_side_theta(), chi)  # the side-chain joints took steps
        out0, it0, _ = a.step_host(th, 0)  # no iteration: the copies' path, theta back unchanged
        assert it0 == 0 and np.array_equal(out0, th)


def test_step_host_exchange_batch_convergence(kcm, table):
    """A batch whose chains stop at different iterations of one call (iteration caps and convergence):
    a stopped chain's angles stay as its last step left them, and the call's iteration count and max
    |dtheta| are those of the device loop; a call whose chains all stop early reports the iterations
    taken."""
    seqs, ths = [], []
    for m, seed in ((12, 3), (25, 4), (40, 5)):
        seq, och, th = small_case(table, m, seed)
        seqs.append(seq)
        ths.append(th)
    th = np.concatenate(ths)
    p = synth.RunParams(precision=synth.PRECISION_MIXED, solvation=0, conv_tol=1e-6)
    it = host_vs_device(kcm, lambda: kcm.Batch(seqs, table, p), th, 6,
                        lambda c: c.set_chain_max_iters(np.array([2, 6, 4], dtype=np.int32)))
    assert it == 6
    it = host_vs_device(kcm, lambda: kcm.Batch(seqs, table, p), th, 8,
                        lambda c: c.set_chain_max_iters(np.array([1, 3, 2], dtype=np.int32)))
    assert it == 3  # every chain at its cap after three iterations; the rest of the call is no-ops
    # a single chain that converges in the call (conv_tol above the first steps' max |dtheta|)
    seq, och, th1 = small_case(table, 15, 9)
    pc = synth.RunParams(precision=synth.PRECISION_MIXED, solvation=0, conv_tol=0.05)
    it = host_vs_device(kcm, lambda: kcm.Chain(seq, table, pc), th1, 5)
    assert it == 1


def test_device_pointer_calls(kcm, table):
    import torch
    seq, och, th = small_case(table, 20, 6)
    p = synth.RunParams()
    ref = och.evaluate(p, th)
    with kcm.Chain(seq, table, p) as ch:
        t = torch.tensor(th, dtype=torch.float64, device="cuda")
        out = torch.zeros(ch.l, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        ch.set_theta_dev(t.data_ptr(), ch.l)
        ch.torques_dev(out.data_ptr())
        ch.step_status()  # synchronises the library's stream
        assert rel_inf(out.cpu().numpy(), ref["tau"]) < TOL_FP64


def test_chain8000_cut12_sampled(kcm, table):
    """The 8,000-residue workload (12 A cutoff): positions everywhere and torques against the
    oracle's full evaluation."""
    seq, th = start("chain8000")
    och = O.OracleChain(seq, table, synth.GEOMETRY)
    pm = synth.RunParams(cutoff=12.0, precision=synth.PRECISION_MIXED)
    ref = och.evaluate(synth.RunParams(cutoff=12.0), th)
    got = gpu_eval(kcm, seq, table, pm, th)
    f64 = gpu_eval(kcm, seq, table, synth.RunParams(cutoff=12.0), th)
    g = och.gamma != 0
    # FP32 overlap tests are re-decided in FP64 inside the guard band: identical classifications
    assert np.array_equal(got["covered"], f64["covered"])
    assert np.array_equal(got["F_cav"], f64["F_cav"])
    assert np.array_equal(f64["covered"][g], ref["covered"][g])
    assert got["stats"]["guard_rechecks"] > 0
    assert np.max(np.abs(got["xyz"] - fk_extended(och, th))) < tol_positions(och.l)
    assert np.max(np.abs(got["xyz"] - ref["xyz"])) < tol_positions(och.l)
    assert rel_inf(got["tau"], ref["tau"]) < TOL_MIXED
    assert got["stats"]["pairs"] == ref["stats"]["pairs"]


def test_long_neighbour_lists(kcm, table):
    """Lists longer than the solvation kernels stage in shared memory (128): the 1,000-residue compact
    start with a 3.2 A solvent probe gives 88 atoms with gamma != 0 more than 128 solvation neighbours
    (largest 168). They are taken by the long-list kernels beside the main ones. FP64 against the
    oracle; mixed classifications and exchange sums equal to FP64's."""
    seq, th = start("chain1000")
    och = O.OracleChain(seq, table, synth.GEOMETRY)
    pf = synth.RunParams(precision=synth.PRECISION_FP64, r_probe=3.2)
    pm = synth.RunParams(precision=synth.PRECISION_MIXED, r_probe=3.2)
    ref = och.evaluate(pf, th)
    f64 = gpu_eval(kcm, seq, table, pf, th)
    mix = gpu_eval(kcm, seq, table, pm, th)
    assert f64["stats"]["max_neighbors"] == 168
    g = och.gamma != 0
    assert np.array_equal(f64["covered"][g], ref["covered"][g])
    assert rel_inf(f64["F_cav"], ref["F_cav"]) < TOL_FP64
    assert rel_inf(f64["tau"], ref["tau"]) < TOL_FP64
    np.testing.assert_allclose(f64["E"], ref["E"], rtol=TOL_FP64, atol=1e-9)
    assert np.array_equal(mix["covered"], f64["covered"])
    assert np.array_equal(mix["F_cav"], f64["F_cav"])
    assert rel_inf(mix["tau"], ref["tau"]) < TOL_MIXED


def clash_conformation(table, target=0.05):
    """A 6-residue chain bent until two atoms (CA of residue 1 and an atom of residue 6) are `target` A
    apart (oracle kinematics: a Nelder-Mead walk to the overlap, then bisection back along the path)."""
    from scipy.optimize import minimize
    seq = synth.sequence(6, 7)
    och = O.OracleChain(seq, table, synth.GEOMETRY)
    th0 = np.random.default_rng(3).uniform(-np.pi, np.pi, och.l)
    i, j = 2, och.n - 2

    def dist(th):
        x, _, _ = och.fk(th)
        return float(np.linalg.norm(x[i] - x[j]))

    r = minimize(lambda th: dist(th) ** 2, th0, method="Nelder-Mead",
                 options={"maxiter": 4000, "xatol": 1e-10, "fatol": 1e-14})
    lo, hi = 0.0, 1.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if dist(th0 + mid * (r.x - th0)) > target:
            lo = mid
        else:
            hi = mid
    th = th0 + hi * (r.x - th0)
    assert abs(dist(th) - target) < 1e-6 * max(target, 1.0)
    return seq, och, th


def test_near_coincident_atoms_stay_finite(kcm, table):
    """Atoms 0.003 A apart: the FP32 pair term overflows (measured: without a bound the mixed torques
    come out non-finite, KCM_E_NONFINITE, from about this distance down); the mixed path holds it at a
    large finite repulsion, so its torques stay finite and the clamped step goes ahead, like the FP64
    path's (whose terms stay finite in double)."""
    seq, och, th = clash_conformation(table, 0.003)
    for prec in (synth.PRECISION_MIXED, synth.PRECISION_FP64):
        with kcm.Chain(seq, table, synth.RunParams(precision=prec)) as ch:
            ch.set_theta(th)
            tau = ch.torques()
            assert np.all(np.isfinite(tau)) and np.abs(tau).max() > 1e10
            it, dm = ch.step(1)
            assert it == 1 and dm == pytest.approx(0.02)


def test_deterministic_fp64(kcm, table):
    """FP64 mode puts each cell's atoms in atom order (a stable counting sort), so its floating-point
    pair sums, the torques and a trajectory are bitwise the same from run to run and handle to handle."""
    seq, th = start("chain1000")
    p = synth.RunParams(precision=synth.PRECISION_FP64)
    runs = []
    for _ in range(2):
        with kcm.Chain(seq, table, p) as ch:
            ch.set_theta(th)
            t1 = ch.torques()
            t2 = ch.torques()
            ch.step(5)
            runs.append((t1, t2, ch.get_theta()))
    (a1, a2, ath), (b1, b2, bth) = runs
    assert np.array_equal(a1, a2) and np.array_equal(a1, b1) and np.array_equal(b1, b2)
    assert np.array_equal(ath, bth)


@pytest.mark.parametrize("precision", [synth.PRECISION_MIXED, synth.PRECISION_FP64])
def test_graph_overlap_changes_nothing(kcm, table, precision):
    """Programmatic dependent launch in the step graphs (kcm_set_graph_overlap, on by default) only lets
    each kernel's launch overlap the previous kernel's run: the trajectory is bitwise that of the graphs
    without it, on a single chain and on a batch."""
    seq, th = start("chain1000")
    p = synth.RunParams(precision=precision)
    out = []
    for on in (True, False):
        with kcm.Chain(seq, table, p) as ch:
            ch.set_graph_overlap(on)
            ch.set_theta(th)
            it, dm = ch.step(4)
            out.append((it, dm, ch.get_theta()))
    assert out[0][:2] == out[1][:2]
    assert np.array_equal(out[0][2], out[1][2])
    seqs = [synth.sequence(m, 7 + m) for m in (5, 40, 97)]
    ths = [synth.theta_uniform(len(q), 3) for q in seqs]
    res = []
    for on in (True, False):
        with kcm.Batch(seqs, table, p) as b:
            b.set_graph_overlap(on)
            b.set_theta(np.concatenate(ths))
            b.step(3)
            res.append(b.get_theta())
    assert np.array_equal(res[0], res[1])
    with kcm.Chain(seq, table, p) as ch:
        assert kcm.load().kcm_set_graph_overlap(ch.handle, 2) == kcm.KCM_E_INVAL


def test_bounded_wait_times_out(kcm, table):
    """The torque kernel's blocks wait for the totals of later link tiles with a bounded wait. With the
    last tile's publication withheld (test hook) every other block gives up after its bound and the
    call reports KCM_E_TIMEOUT, without hanging; the handle and the context stay usable, and the next
    evaluation is correct again."""
    seq, och, th = small_case(table, 40, 1235, "compact")  # 81 links: three tiles of 32
    p = synth.RunParams(precision=synth.PRECISION_FP64)
    ref = och.evaluate(p, th)
    with kcm.Chain(seq, table, p) as ch:
        ch.set_theta(th)
        ch.set_test_withhold(2)
        with pytest.raises(kcm.KcmError) as e:
            ch.torques()
        assert e.value.code == kcm.KCM_E_TIMEOUT
        with pytest.raises(kcm.KcmError) as e:
            ch.step(3)
        assert e.value.code == kcm.KCM_E_TIMEOUT
        with pytest.raises(kcm.KcmError) as e:  # the status record exported by the timed-out iteration
            ch.step_host(th, 3)
        assert e.value.code == kcm.KCM_E_TIMEOUT
        ch.set_test_withhold(-1)
        ch.set_theta(th)
        assert rel_inf(ch.torques(), ref["tau"]) < TOL_FP64
        with pytest.raises(kcm.KcmError):
            ch.set_test_withhold(3)  # out of range
