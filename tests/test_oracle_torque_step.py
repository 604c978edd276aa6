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
