"""Write the oracle's reference values for the full-size H-LU workloads.

    python tests/golden/make_golden.py laplace3d_32 [laplace3d_64 ...]

For each workload this runs the CPU oracle (``oracle/``, serial FP64,
accumulated H-LU of Section 6 with the accumulators of Section 4) on the
seeded input of ``hmat_synth`` and writes ``oracle_<workload>.json`` next to
this file.  Nothing here touches the CUDA path: every stored value comes from
the oracle alone.  The stored values are

  * the block tree's structure: counts of dense and admissible leaves and a
    SHA-256 of the node arrays (row cluster, column cluster, kind, in the
    pre-order of Section 2's block tree, as little-endian int32), and the
    hash of the cluster tree's permutation;
  * the preconditioner error ||I - (LU)^{-1} A||_2 (Section 7) by the power
    iteration of the oracle from the N(0,1) start vector of seed 0 (50 steps
    at most, relative change 1e-3);
  * the truncation count and the rank histogram of the admissible leaves.

The 64^3 run is long (hours on one core) and needs tens of GB of host memory.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

sys.path.insert(0, os.path.dirname(HERE))
import golden  # noqa: E402  (tests/golden.py: the hashes the GPU tests compare)
import hmat_synth as hs  # noqa: E402
import oracle  # noqa: E402

WORKLOADS = {"laplace3d_32": hs.laplace3d_32, "laplace3d_64": hs.laplace3d_64, "laplace2d_64": hs.laplace2d_64}


def oracle_values(name: str) -> dict:
    p = WORKLOADS[name]()
    ct, bt, csr, H = oracle.setup(p)
    nodes = bt.nodes()
    oracle.stats_reset()
    t0 = time.perf_counter()
    H.lu(p.eps, True)
    lu_s = time.perf_counter() - t0
    st = oracle.stats()
    perm = ct.perm()
    err, iters = H.precond_error(csr, hs.start_vector(p.n, 0)[perm])
    ranks = H.ranks()
    adm = ranks[nodes["kind"] == 2]
    hist = np.bincount(adm, minlength=1)
    return {
        "workload": name, "n": p.n, "leaf": p.leaf, "eta": p.eta, "eps": p.eps,
        "blocks": int(len(nodes["t"])), "dense_leaves": int(np.sum(nodes["kind"] == 1)),
        "lowrank_leaves": int(np.sum(nodes["kind"] == 2)),
        "blocktree_sha256": golden.tree_hash(nodes), "perm_sha256": golden.perm_hash(perm),
        "precond_error": err, "power_iterations": iters,
        "truncations": int(st["truncations"]), "mean_rank": float(adm.mean()) if adm.size else 0.0,
        "max_rank": int(adm.max()) if adm.size else 0,
        "rank_histogram": [int(x) for x in hist],
        "oracle_lu_seconds": lu_s, "oracle_cores": 1,
        "made_by": "tests/golden/make_golden.py (oracle only)",
    }


def main(argv):
    for name in argv or ["laplace3d_32"]:
        out = oracle_values(name)
        path = os.path.join(HERE, f"oracle_{name}.json")
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
            f.write("\n")
        print(json.dumps({k: out[k] for k in ("workload", "precond_error", "truncations", "mean_rank",
                                               "oracle_lu_seconds")}), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
