"""Pins of the oracle's joint torques (eq. KCM_01..06, 04_9, Sec. 3.5) and kinetostatic step
(eq. KCM_07): tau_k = -dE/dtheta_k by central differences of the energy through the kinematics,
equality of the O(l^2) column form with the row-scan form, and the step rules."""
import numpy as np
import pytest

from kcm_testutil import rel_inf
from oracle import oracle as O
from paper_1712_05012_b300 import synth


def pair_energy_at(ch, theta, p):
    xyz, _, _ = ch.fk(theta)
    _, E, _ = ch.pair_forces(xyz, p)
    return E.sum()


@pytest.mark.parametrize("m,seed", [(4, 1), (7, 2), (12, 3)])
def test_torque_is_minus_energy_gradient(table, m, seed):
    """KCM is steepest descent in angle space: tau_k = -dE/dtheta_k (Sec. 2.3). Solvation is off
    (its enumerated energy is piecewise constant) and the cutoff covers every pair, so the pair
    set does not change under the finite differences."""
    seq = synth.sequence(m, 100 + seed)
    ch = O.OracleChain(seq, table, synth.GEOMETRY)
    th = synth.theta_from_codes(ch.grow_start(seed))
    p = synth.RunParams(cutoff=500.0, solvation=0)
    r = ch.evaluate(p, th)
    h = 1e-5
    g = np.zeros(ch.l)
    for k in range(ch.l):
        tp = th.copy(); tp[k] += h
        tm = th.copy(); tm[k] -= h
        g[k] = (pair_energy_at(ch, tp, p) - pair_energy_at(ch, tm, p)) / (2 * h)
    assert rel_inf(r["tau"], -g) < 1e-6


def test_columns_equal_rowscan(table):
    m = 30
    seq = synth.sequence(m, 5)
    ch = O.OracleChain(seq, table, synth.GEOMETRY)
    th = synth.theta_from_codes(ch.grow_start(9))
    p = synth.RunParams()
    r = ch.evaluate(p, th)
    xyz, u, pk = ch.fk(th)
    F = r["F_pair"] + r["F_cav"]
    t1 = ch.torques(xyz, F, u, pk, "columns")
    t2 = ch.torques(xyz, F, u, pk, "rowscan")
    assert rel_inf(t2, t1) < 1e-12
    assert np.array_equal(t1, r["tau"])


def test_base_link_forces_do_not_matter(table):
    """No joint precedes the anchored base link (N_1, H_1), so forces on it give no torque."""
    m = 5
    seq = synth.sequence(m, 6)
    ch = O.OracleChain(seq, table, synth.GEOMETRY)
    th = synth.theta_uniform(m, 2)
    xyz, u, pk = ch.fk(th)
    rng = np.random.default_rng(1)
    F = rng.normal(size=(ch.n, 3))
    t1 = ch.torques(xyz, F, u, pk)
    F2 = F.copy()
    F2[ch.link == 0] += rng.normal(size=(int((ch.link == 0).sum()), 3))
    assert np.array_equal(ch.torques(xyz, F2, u, pk), t1)


def test_step_clamp_and_normalised():
    tau = np.array([5.0, -40.0, 0.001, 100.0, -3.0])
    th0 = np.array([0.1, 0.2, 0.3, 0.4, 0.5])
    th, d, dm = O.step(th0, tau, 1e-3, 0.02, mode=0)
    assert np.allclose(d, [0.005, -0.02, 1e-6, 0.02, -0.003], rtol=0, atol=1e-18)
    assert np.allclose(th, th0 + d, rtol=0, atol=0)
    assert dm == 0.02
    th, d, dm = O.step(th0, tau, 0.05, 0.02, mode=1)  # eq. KCM_07: kappa tau / max|tau|
    assert np.allclose(d, 0.05 * tau / 100.0, rtol=1e-15)
    assert dm == pytest.approx(0.05)


def test_step_with_fixed_joints():
    """Sec. 4.1: fixed dihedral angles take no step, and the normalised step's max |tau| runs over
    the free joints only (here 5.0, not 100.0)."""
    tau = np.array([5.0, -40.0, 0.001, 100.0, -3.0])
    th0 = np.array([0.1, 0.2, 0.3, 0.4, 0.5])
    fixed = [0, 1, 0, 1, 0]
    th, d, dm = O.step(th0, tau, 1e-3, 0.02, mode=0, fixed=fixed)
    assert np.array_equal(d, [0.005, 0.0, 1e-6, 0.0, -0.003])
    assert th[1] == th0[1] and th[3] == th0[3]
    assert dm == 0.005
    th, d, dm = O.step(th0, tau, 0.05, 0.02, mode=1, fixed=fixed)
    assert np.allclose(d, [0.05, 0.0, 1e-5, 0.0, -0.03], rtol=1e-15, atol=0)
    assert dm == pytest.approx(0.05)


def test_fixed_domain_moves_rigidly(table):
    """Fixing every joint between links 8 and 20 makes those links one rigid body: after a run the
    distances between their atoms are unchanged, while the free joints moved. A property of the
    kinematics, independent of the step rule."""
    m = 15
    seq = synth.sequence(m, 21)
    ch = O.OracleChain(seq, table, synth.GEOMETRY)
    th0 = synth.theta_from_codes(ch.grow_start(5))
    fixed = np.zeros(ch.l, dtype=np.uint8)
    fixed[8:20] = 1  # joints 8 .. 19 join links 8 .. 20
    p = synth.RunParams(solvation=0)
    th, it, _, _ = ch.run(p, th0, 10, fixed=fixed)
    assert it == 10
    assert np.array_equal(th[8:20], th0[8:20])
    assert np.max(np.abs(th - th0)) > 1e-4
    x0, _, _ = ch.fk(th0)
    x1, _, _ = ch.fk(th)
    g = (ch.link >= 8) & (ch.link <= 20)
    d0 = np.linalg.norm(x0[g][:, None] - x0[g][None], axis=-1)
    d1 = np.linalg.norm(x1[g][:, None] - x1[g][None], axis=-1)
    assert np.max(np.abs(d1 - d0)) < 1e-10
    # without the mask the same links deform
    th2, _, _, _ = ch.run(p, th0, 10)
    x2, _, _ = ch.fk(th2)
    d2 = np.linalg.norm(x2[g][:, None] - x2[g][None], axis=-1)
    assert np.max(np.abs(d2 - d0)) > 1e-3


def test_run_stops_on_convergence(table):
    m = 6
    seq = synth.sequence(m, 8)
    ch = O.OracleChain(seq, table, synth.GEOMETRY)
    th0 = synth.theta_from_codes(ch.grow_start(4))
    p = synth.RunParams(kappa=1e-12, conv_tol=1e-4)
    th, it, Et, dt = ch.run(p, th0, 50)
    assert it == 1 and dt[0] < 1e-4
    p = synth.RunParams()
    th, it, Et, dt = ch.run(p, th0, 20)
    assert it == 20 and np.all(dt <= p.dtheta_max)


def test_oracle_thread_count_invariant(table):
    """Per-atom work is reduced in a fixed order: results do not depend on the thread count."""
    seq = synth.sequence(40, 1235)
    ch = O.OracleChain(seq, table, synth.GEOMETRY)
    th = synth.theta_from_codes(ch.grow_start(1))
    p = synth.RunParams()
    n0 = O.num_threads()
    O.set_threads(1)
    a = ch.evaluate(p, th)
    O.set_threads(max(2, n0))
    b = ch.evaluate(p, th)
    O.set_threads(n0)
    for k in ("F_pair", "F_cav", "tau", "E", "covered"):
        assert np.array_equal(a[k], b[k]), k
