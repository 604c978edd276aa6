"""Write the compact self-avoiding random-walk starts of the long-chain and batch workloads.

Run from the repository root:  python tests/golden/make_starts.py
Each start is the oracle's residue-by-residue growth (phi, psi uniform, redrawn until no heavy-atom
pair more than three bonds apart is closer than 2.5 A, backing up five residues after 100 failed
draws), stored as 16-bit angle codes (theta = code * 2 pi / 65536, exact in float64). Only the
oracle and the input generator are called.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_1712_05012_b300 import synth  # noqa: E402

STARTS = [
    # name, workload index, residues
    ("chain1000", 2, 1000),
    ("chain8000", 3, 8000),
]


def main():
    table = synth.type_table()
    manifest = {}
    for name, k, m in STARTS:
        wl = synth.workload(k)
        seed = synth.chain_seed(wl.seed, 0)
        seq = synth.sequence(m, seed)
        ch = O.OracleChain(seq, table, synth.GEOMETRY)
        codes = ch.grow_start(seed, min_dist=2.5, max_retries=100, backtrack=5)
        np.save(os.path.join(HERE, f"start_{name}.npy"), codes)
        manifest[name] = {"workload": k, "residues": m, "sequence_seed": seed, "grow_seed": seed,
                          "min_dist": 2.5, "max_retries": 100, "backtrack": 5, "atoms": ch.n}
        print(name, ch.n, "atoms")
    # the batch workload: every chain grown the same way, codes concatenated in chain order
    wl = synth.workload(4)
    codes_all = []
    natoms = 0
    for i, m in enumerate(wl.m):
        seed = synth.chain_seed(wl.seed, i)
        ch = O.OracleChain(synth.sequence(m, seed), table, synth.GEOMETRY)
        codes_all.append(ch.grow_start(seed, min_dist=2.5, max_retries=100, backtrack=5))
        natoms += ch.n
    np.save(os.path.join(HERE, "start_batch512.npy"), np.concatenate(codes_all))
    manifest["batch512"] = {"workload": 4, "chains": len(wl.m), "residues_total": int(sum(wl.m)),
                            "sequence_seed": "chain_seed(workload seed, chain index)", "grow_seed": "the same",
                            "min_dist": 2.5, "max_retries": 100, "backtrack": 5, "atoms": natoms}
    print("batch512", len(wl.m), "chains", natoms, "atoms")
    # a pool of serving jobs: lengths log-uniform in 20..2000 residues, each grown the same way
    wl = synth.workload(5)
    rng = np.random.default_rng(wl.seed)
    lens = np.exp(rng.uniform(np.log(20), np.log(2000), size=256)).astype(int).tolist()
    codes_all = []
    for i, m in enumerate(lens):
        seed = synth.chain_seed(wl.seed, i)
        ch = O.OracleChain(synth.sequence(m, seed), table, synth.GEOMETRY)
        codes_all.append(ch.grow_start(seed, min_dist=2.5, max_retries=100, backtrack=5))
    np.save(os.path.join(HERE, "start_serve256.npy"), np.concatenate(codes_all))
    manifest["serve256"] = {"workload": 5, "residues": lens, "sequence_seed": "chain_seed(workload seed, index)",
                            "grow_seed": "the same", "min_dist": 2.5, "max_retries": 100, "backtrack": 5}
    print("serve256", len(lens), "chains", sum(lens), "residues")
    with open(os.path.join(HERE, "starts.json"), "w") as f:
        json.dump(manifest, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
