"""The stored compact starts are reproducible from the oracle and clash-free."""
import json
import os

import numpy as np

from oracle import oracle as O
from paper_1712_05012_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_chain1000_start_reproducible_and_clash_free(table):
    man = json.load(open(os.path.join(GOLDEN, "starts.json")))["chain1000"]
    codes = np.load(os.path.join(GOLDEN, "start_chain1000.npy"))
    seq = synth.sequence(man["residues"], man["sequence_seed"])
    ch = O.OracleChain(seq, table, synth.GEOMETRY)
    assert ch.n == man["atoms"]
    again = ch.grow_start(man["grow_seed"], man["min_dist"], man["max_retries"], man["backtrack"])
    assert np.array_equal(again, codes)
    xyz, _, _ = ch.fk(synth.theta_from_codes(codes))
    heavy = np.where(ch.kind != 1)[0]
    X = xyz[heavy]
    for a in range(0, len(heavy), 1024):
        d = np.linalg.norm(X[a:a + 1024, None, :] - X[None, :, :], axis=-1)
        ii, jj = np.nonzero(d < man["min_dist"])
        for i, j in zip(ii + a, jj):
            if heavy[i] < heavy[j]:
                assert ch.bond_distance(heavy[i], heavy[j]) <= 3
