"""The oracle's FP64 kinematics against the same definition evaluated in 80-bit long double: its
accumulated rounding stays within the bound the parity tests use (kcm_testutil.tol_positions)."""
import json
import os

import numpy as np
import pytest

from kcm_testutil import fk_extended, tol_positions
from oracle import oracle as O
from paper_1712_05012_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_extended_reference_is_the_same_definition(table):
    seq = synth.sequence(9, 3)
    och = O.OracleChain(seq, table, synth.GEOMETRY)
    th = synth.theta_uniform(9, 4)
    x, _, _ = och.fk(th)
    assert np.max(np.abs(fk_extended(och, th).astype(np.float64) - x)) < 1e-13


@pytest.mark.parametrize("name", ["chain1000", "chain8000"])
def test_oracle_rounding_long_chains(table, name):
    man = json.load(open(os.path.join(GOLDEN, "starts.json")))[name]
    seq = synth.sequence(man["residues"], man["sequence_seed"])
    th = synth.theta_from_codes(np.load(os.path.join(GOLDEN, f"start_{name}.npy")))
    och = O.OracleChain(seq, table, synth.GEOMETRY)
    x, _, _ = och.fk(th)
    err = float(np.max(np.abs(fk_extended(och, th) - x)))
    assert err < tol_positions(och.l)
