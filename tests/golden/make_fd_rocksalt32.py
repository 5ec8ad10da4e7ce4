"""Writes fd_rocksalt32.txt: central differences of the FP64 oracle's MSM energy
on the 32^3 rock-salt supercell (262,144 atoms, lattice constant 5.64 A,
Gaussian displacements sigma = 0.1 A, charges +/-(1 + 0.1 N(0,1)) shifted to
zero sum; p = 4, h = 2 A, a = 8 A), for 64 seeded atoms:

  dE/dr_i,d   = (E(r_i,d + delta) - E(r_i,d - delta)) / (2 delta),  delta = 1e-4 A
  dE/dq_i     = (E(q_i + delta) - E(q_i - delta)) / (2 delta),      delta = 1e-4
  W_ab        = -dE/d eps_ab under r -> (1 + eps) r, cell rows -> (1 + eps) rows,
                eps symmetric, central difference with |eps_ab + eps_ba| = 1e-6

These are the derivatives of Sec. 3.2.2 (forces, charge gradients) and the cell
virial, taken numerically from the energy alone, so they check the analytic
gradients independently of how they are computed. Only the oracle is called;
the inputs come from the seeded workload generator. The oracle evaluates on the
float32 inputs promoted to float64 (the values the GPU reads).

Run from the repository root:  python tests/golden/make_fd_rocksalt32.py
(about 10 minutes on 8 cores).
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2510_05961_gb300 import workloads as W  # noqa: E402

NPICK = 64
SEED = 4064
DR = 1e-4
DQ = 1e-4
DEPS = 1e-6
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fd_rocksalt32.txt")


def main():
    O.build()
    w = W.rocksalt(ncell=32)
    pos = w.pos.astype(np.float64)
    q = w.q.astype(np.float64)
    L = w.cell[0]
    M = 64  # the planner's grid for h = 2 A at L = 180.48 A, fixed so strained cells keep it
    P = O.make_plan(w.cell, w.pbc, w.h, w.a, w.p, grid_override=(M, M, M))

    def energy(P_, p_, q_):
        return O.msm(P_, p_, q_, forces=False, virial=False)["E"]

    idx = np.sort(np.random.default_rng(SEED).choice(w.n, NPICK, replace=False))
    rows = []
    for i in idx:
        g = []
        for d in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, d] += DR
            pm[i, d] -= DR
            g.append((energy(P, pp, q) - energy(P, pm, q)) / (2 * DR))
        qp, qm = q.copy(), q.copy()
        qp[i] += DQ
        qm[i] -= DQ
        g.append((energy(P, pos, qp) - energy(P, pos, qm)) / (2 * DQ))
        rows.append((int(i), *g))
        print(i, g, flush=True)
    A = np.diag([L, L, L])
    wv = []
    for a, b in [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]:
        es = []
        for sg in (1, -1):
            eps = np.zeros((3, 3))
            eps[a, b] += 0.5 * DEPS * sg
            eps[b, a] += 0.5 * DEPS * sg
            Fm = np.eye(3) + eps
            cell = A @ Fm.T
            if a == b:  # still rectangular
                P2 = O.make_plan(np.diag(cell).copy(), w.pbc, w.h, w.a, w.p, grid_override=(M, M, M))
            else:
                P2 = O.make_plan(cell, w.pbc, w.h, w.a, w.p, grid_override=(M, M, M))
            es.append(energy(P2, pos @ Fm.T, q))
        wv.append(-(es[0] - es[1]) / (2 * DEPS))
        print((a, b), wv[-1], flush=True)
    with open(OUT, "w") as f:
        f.write("# Central differences of the FP64 oracle MSM energy, 32^3 rock-salt supercell\n")
        f.write("# (workloads.rocksalt(ncell=32): 262144 atoms, a0 = 5.64 A, sigma = 0.1 A,\n")
        f.write("# q = +/-(1 + 0.1 N(0,1)) minus the mean; p = 4, h = 2 A (M = 64), a = 8 A).\n")
        f.write("# Derivatives of Sec. 3.2.2 and the cell virial, from the energy alone.\n")
        f.write("# Written by tests/golden/make_fd_rocksalt32.py (oracle only).\n")
        f.write("# delta_r = %g A, delta_q = %g, delta_eps = %g; atoms drawn with seed %d\n" % (DR, DQ, DEPS, SEED))
        f.write("# E = %.17g\n" % energy(P, pos, q))
        f.write("# virial W_xx W_yy W_zz W_xy W_xz W_yz (W = -dE/d eps)\n")
        f.write("virial " + " ".join("%.17g" % v for v in wv) + "\n")
        f.write("# atom dE/dx dE/dy dE/dz dE/dq\n")
        for r in rows:
            f.write("%d %s\n" % (r[0], " ".join("%.17g" % v for v in r[1:])))


if __name__ == "__main__":
    main()
