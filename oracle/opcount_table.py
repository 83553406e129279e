"""Write profiles/fp64_opcount.json: the FP64 arithmetic of one stage per
interior cell, counted by the op-counting build of the oracle (opcount.cpp),
for the FP64 roofline of the benchmark.  Measurement infrastructure: it calls
only the oracle.

Counted: additions/subtractions, multiplications, divisions, square roots,
minima/maxima and comparisons (one flop each; the oracle has no fused
multiply-add), over the stage's faces, sources and update.  The boundary and
primitive update is left out: the oracle inverts the closure by bisection,
where the stage kernels use the closed-form root (the primitive pass, not
the stage kernel, does it there).  Transcendental calls are listed apart.

    python oracle/opcount_table.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
from paper_2304_00140_gb300 import workloads as wl  # noqa: E402

FLOP_CLASSES = ("add", "mul", "div", "sqrt", "minmax", "cmp")


def count(w, inflow_u=None):
    o = oracle.Oracle(w, inflow_u=inflow_u)
    q = o.prim_to_cons(w.primitives())
    dt = 0.3 * o.dt(q, 1.0)
    _, stage, box = oracle.opcount_stage(o, 1, dt, q, q)
    net = {k: (stage[k] - box[k]) / w.cells for k in stage}
    return dict(flops_per_cell=sum(net[k] for k in FLOP_CLASSES), classes=net,
                sample=f"{w.name}, stage 1 from the initial state, CFL 0.3")


def main():
    # each benchmark workload's scheme and state, on a smaller grid of the
    # same layout (the key is the workload as the benchmark runs it).  Only
    # schemes whose oracle stage does each operation once per face or cell:
    # with CSF or the App. D switch the oracle re-smooths the fraction at
    # every vertex of every cell, and with Peng-Robinson it brackets the
    # cubic's root by bisection, so its counts there (jet 11338, droplet
    # 1637, rising bubble 1674, Peng-Robinson 4535 a cell) are not the
    # algorithm's
    table = {
        "shock_bubble_2048x1024": count(wl.shock_bubble(nx=256, ny=128)),
        "advection_128x128": count(wl.advection(n=128)),
        "vapour_bubble_collapse_1000x1000": count(wl.bubble_collapse("vapour", n=(125, 125))),
        "gas_bubble_collapse_1000x1000": count(wl.bubble_collapse("gas", n=(125, 125))),
    }
    out = os.path.join(os.path.dirname(HERE), "profiles", "fp64_opcount.json")
    json.dump(dict(note=__doc__.split("\n\n")[1].replace("\n", " "), workloads=table), open(out, "w"), indent=1,
              sort_keys=True)
    print(json.dumps({k: round(v["flops_per_cell"], 1) for k, v in table.items()}))


if __name__ == "__main__":
    main()
