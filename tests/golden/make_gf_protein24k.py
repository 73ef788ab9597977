"""Write the FP64 oracle's graph-family result at 24,000 atoms for the GPU tests.

    python -m tests.golden.make_gf_protein24k      # a few minutes per 8 cores

The graph family's six layers reach 36 A, so a force needs nearly the whole
24,000-atom box and no sampled evaluation is cheaper than the whole system.
This script runs ``oracle.gf_compute`` once on the seeded protein-in-water
system with the seeded weights and stores, in ``gf_protein24k.json``: the
energy, the virial, the force RMS over all 3N components, and the forces and
atomic energies of 200 atoms chosen by seed (plus the blob's and the most
crowded atom).  A SHA-256 of the inputs (coordinates, species, box, weights)
lets the test refuse a stale file.  Only ``oracle`` and ``synth`` are used.
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from synth import configs as C, normal_blob  # noqa: E402

OUT = os.path.join(HERE, "gf_protein24k.json")
SAMPLE_SEED = 20260204          # the graph-family workload's seed
N_SAMPLE = 200


def inputs():
    m, s = C.GRAPH_MODEL, C.protein24k()
    w = normal_blob(oracle.gf_weight_count(m), C.WEIGHT_SEED)
    return m, s, w


def digest(s, w) -> str:
    h = hashlib.sha256()
    for a in (np.ascontiguousarray(s.coords, np.float64), np.ascontiguousarray(s.types, np.int32),
              np.ascontiguousarray(s.box, np.float64), np.ascontiguousarray(w, np.float64)):
        h.update(a.tobytes())
    return h.hexdigest()


def sample(s, m) -> np.ndarray:
    rng = np.random.default_rng(SAMPLE_SEED)
    cnt = oracle.neighbours(s.coords, s.box, m.rc, 1)[0]
    pick = rng.choice(s.n, N_SAMPLE - 2, replace=False)
    extra = [int(rng.integers(0, s.blob_atoms)), int(np.argmax(cnt))]
    return np.unique(np.concatenate([pick, extra])).astype(np.int64)


def main():
    m, s, w = inputs()
    idx = sample(s, m)
    t0 = time.time()
    E, ae, F, V = oracle.gf_compute(m, w, s.types, s.coords, s.box)
    out = {
        "what": "oracle.gf_compute, graph family (6 layers, node 128, edge 64, angles < 4 A), "
                "24,000-atom protein-in-water system, seeded weights",
        "inputs_sha256": digest(s, w),
        "energy": E,
        "virial": V.tolist(),
        "force_rms": float(np.sqrt(np.mean(F ** 2))),
        "net_force": F.sum(0).tolist(),
        "sample": idx.tolist(),
        "forces": F[idx].tolist(),
        "atom_energies": ae[idx].tolist(),
        "oracle_seconds": time.time() - t0,
    }
    with open(OUT, "w") as f:
        json.dump(out, f, indent=0)
    print(OUT, out["energy"], out["oracle_seconds"])


if __name__ == "__main__":
    main()
