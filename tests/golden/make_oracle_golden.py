"""Write oracle-computed expected values for marches too long to recompute
inside a test.

Calls only the FP64 CPU oracle (oracle/) and the seeded input module; no
value here comes from the CUDA path.  Output: tests/golden/<name>.npz with
the flat node indices, the oracle's u^0 at those nodes, and the workload
description.  Run from the repository root:

    python tests/golden/make_oracle_golden.py [threads] [workload ...]

(default: every workload below).
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import fk_inputs  # noqa: E402
from oracle import fk_oracle as O  # noqa: E402

FAM = {"const_drift": O.CONST_DRIFT, "cellular_flow": O.CELLULAR_FLOW,
       "paper_cellular": O.PAPER_CELLULAR}
WORKLOADS = ("cellular_1025x513", "paper_2d_1025x257", "graded_1025x513",
             "cellular_4097x2049")
# workloads whose full march is too long for the oracle: a march of this many
# steps on the same mesh and rule instead (the file name says so)
TRUNCATED = {"cellular_4097x2049": 50}


def make(name: str, threads: int, samples: int = 20000, seed: int = 99):
    w = fk_inputs.workload(name, precision="fp64")
    tag = name
    if name in TRUNCATED:
        w["n_steps"] = TRUNCATED[name]
        tag = f"{name}_{w['n_steps']}steps"
    g = O.Grid(tuple(w["n"]), tuple(w["lo"]), tuple(w["hi"]), int(w.get("periodic_x", False)),
               fk_inputs.axes_of(w))
    t = time.time()
    u = O.march(g, FAM[w["family"]], list(w["params"]), w["q"], w["dt"], w["n_steps"], 0,
                nthreads=threads)
    elapsed = time.time() - t
    shape = g.shape
    nodes = fk_inputs.sample_nodes(shape, samples, seed)
    # add every node of the rows and columns next to the boundary (with
    # periodic x, of the two seam columns as well)
    ny, nx = shape
    strips = np.concatenate([np.arange(nx) + nx * 1, np.arange(nx) + nx * (ny - 2),
                             np.arange(ny) * nx + 1, np.arange(ny) * nx + nx - 2,
                             np.arange(ny) * nx, np.arange(ny) * nx + nx - 1])
    nodes = np.unique(np.concatenate([nodes, strips])).astype(np.int64)
    vals = u.reshape(-1)[nodes]
    out = os.path.join(HERE, f"{tag}_oracle_u0.npz")
    np.savez_compressed(out, nodes=nodes, u0=vals, n=np.array(w["n"]), q=w["q"], dt=w["dt"],
                        n_steps=w["n_steps"], params=np.array(w["params"]),
                        umin=u.min(), umax=u.max(), umean=u.mean())
    print(f"{out}: {nodes.size} nodes, march {elapsed:.0f} s on {threads} threads")


if __name__ == "__main__":
    threads = int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1)
    for name in (sys.argv[2:] or WORKLOADS):
        make(name, threads)
