"""Writes cfg3_mini_N3.npz: the oracle's clustered-LTS run of the small layered
graded scenario (`inputs.cfg3_mini_scenario`: 12,288 tets, N = 3, rate-2
clusters capped at 6, explosive source, 8 LOHp receivers, 20 steps of the
largest cluster).  Everything stored comes from `oracle/` only.

The run takes ~40 min of one host core, so the GPU test reads its result
from this file instead of re-running it.

Stored: the cluster of every element, dt_min, the seismogram (times and the
13 quantities) of every receiver, the final DOFs of 96 elements spread over
the mesh (every cluster represented) and the L2 norm of every element's
final DOFs.

  python tests/golden/make_cfg3_mini.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import corrector  # noqa: E402
from paper_2108_10565_gb300 import inputs  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cfg3_mini_N3.npz")


def sample_elements(ne, k=96):
    return np.unique(np.linspace(0, ne - 1, k).round().astype(np.int64))


def main():
    sc = inputs.cfg3_mini_scenario()
    t0 = time.time()
    sim = corrector.LTSSimulation(sc["mesh"], sc["materials"], sc["N"], sc["max_clusters"],
                                  source=sc["source"], receivers=sc["receivers"])
    Q, seis = sim.run(sc["Q0"], sc["n_cycles"])
    ne = Q.shape[0]
    idx = sample_elements(ne)
    out = dict(cluster=sim.cl.astype(np.int32), dt_min=np.array(sim.dt_min), sample=idx, Q_sample=Q[idx],
               Q_norm=np.linalg.norm(Q.reshape(ne, -1), axis=1))
    for r, (t, q) in enumerate(seis):
        out[f"t{r}"] = t
        out[f"q{r}"] = q
    np.savez_compressed(OUT, **out)
    print(f"wrote {OUT}: {ne} elements, clusters {np.bincount(sim.cl).tolist()}, {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
