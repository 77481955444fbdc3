"""Write opt_values.txt: exact optima of the seeded image-pair workloads (oracle O1 only).

Each line: k seed spike_frac OPT pivots.  OPT is the optimal value of the Kantorovich LP
(Section 2.1) with squared-Euclidean pixel cost, from the oracle's network simplex, certified by
its dual potentials (zero gap, dual feasibility over all pairs).  Run from the repository root:
    python tests/golden/make_opt_values.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import certificate, costs, netsimplex  # noqa: E402
from paper_2206_11009_gb300 import synth  # noqa: E402

CASES = [(8, s, 0.0) for s in range(3)] + [(16, s, 0.0) for s in range(5)] + [(16, 0, 0.05)] + \
        [(32, s, 0.0) for s in range(2)] + [(32, 0, 0.05), (64, 0, 0.0)]


def main():
    lines = ["# k seed spike_frac OPT pivots   (oracle network simplex, certified)"]
    for k, s, sp in CASES:
        inst = synth.image_pair(k, s, spike_frac=sp)
        c = costs.square_grid(k)
        r = netsimplex.solve(c, inst.a, inst.b)
        gap = abs(inst.a @ r.u + inst.b @ r.v - r.obj) / r.obj
        assert gap < 1e-10 and certificate.min_reduced_cost(c, r.u, r.v) >= 0.0
        lines.append(f"{k} {s} {sp} {r.obj!r} {r.pivots}")
        print(lines[-1], flush=True)
    with open(os.path.join(HERE, "opt_values.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
