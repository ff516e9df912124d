"""Writes the stored expected values under tests/golden/ from the CPU oracle
alone (no CUDA code is imported).

c1_fullgrid_20steps.txt: the C1 workload (d=4, n=24, nu=0.05, mean sin x,
sigma=0.3, ell=1.0) advanced 20 classical RK4 steps of dt=1e-3 on the full
n^d grid with no truncation (the plain definition of the discretised PDE,
Eq. (hyper1) with the RK4 increment of Eq. (discrete-flow-intro)); Phi at 12
seeded grid points near a = 0 and the finite-difference moments at a = 0 (Sec. 1:
moments are functional derivatives at theta = 0).  Also the same 20 steps of
the TT oracle (step truncation, tol 1e-10, rank cap 16, App. A Alg. 1/2
mirrored) from the TT-SVD of Phi0: the rank chosen by every rounding and Phi
at the same points, so that a solver can replay the ranks and be compared
entry by entry.

  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import fullgrid, model, tt  # noqa: E402
import synthetic  # noqa: E402

NSTEPS, NPTS, SEED = 20, 12, 7


def c1_fullgrid():
    w = synthetic.C1
    m0, C0 = model.cell_moments(w.d, w.alpha, w.beta, w.sigma, w.ell)
    L = model.default_L(C0)
    F = fullgrid.solve(fullgrid.phi0_grid(m0, C0, w.n, L), w.dt, NSTEPS, w.d, w.n, L, w.nu)
    # seeded points within 3 grid steps of a = 0, where Phi is of order one
    idx = w.n // 2 - 3 + synthetic.random_probe_indices(w.d, 7, NPTS, SEED)
    vals = np.array([F[tuple(i)] for i in idx])
    mean, cov = fullgrid.moments(F, w.n, L)
    return L, idx, vals, mean, cov


def c1_tt(L, idx):
    w = synthetic.C1
    m0, C0 = model.cell_moments(w.d, w.alpha, w.beta, w.sigma, w.ell)
    cores = tt.tt_svd(fullgrid.phi0_grid(m0, C0, w.n, L), w.tol, w.cap)
    W, bond = model.mpo_blocks(w.d, w.n, L, w.nu), model.mpo_bond_dims(w.d)
    log = []
    for _ in range(NSTEPS):
        cores, _ = tt.rk4_step(cores, w.dt, W, bond, w.tol, w.cap, record=log)
    return np.array(log, dtype=int), tt.evaluate(cores, idx)


def main():
    L, idx, vals, mean, cov = c1_fullgrid()
    ranks, tvals = c1_tt(L, idx)
    path = os.path.join(HERE, "c1_fullgrid_20steps.txt")
    with open(path, "w") as f:
        f.write("# C1 (d=4, n=24, nu=0.05, mean sin x, sigma=0.3, ell=1.0), 20 RK4 steps of dt=1e-3\n")
        f.write("# on the full grid, no truncation: Eq. (hyper1) for 1-D Burgers, classical RK4\n")
        f.write("# (Eq. discrete-flow-intro); moments by central differences at a = 0 (Sec. 1).\n")
        f.write("# Then the TT oracle (tol 1e-10, cap 16): 'ttranks' = ranks of each rounding,\n")
        f.write("# 'ttphi' = its Phi at the same points.  Written by tests/golden/make_golden.py\n")
        f.write("# from oracle.fullgrid and oracle.tt only.\n")
        f.write(f"L {float(L)!r}\n")
        for i, v in zip(idx, vals):
            f.write("phi " + " ".join(str(int(x)) for x in i) + f" {float(v.real)!r} {float(v.imag)!r}\n")
        f.write("mean " + " ".join(repr(float(x)) for x in mean) + "\n")
        for row in cov:
            f.write("cov " + " ".join(repr(float(x)) for x in row) + "\n")
        for row in ranks:
            f.write("ttranks " + " ".join(str(int(x)) for x in row) + "\n")
        for v in tvals:
            f.write(f"ttphi {float(v.real)!r} {float(v.imag)!r}\n")
    print("wrote", path)


def read_c1():
    """(L, idx, full-grid Phi, mean, cov, TT rank log, TT Phi) as stored."""
    idx, vals, mean, cov, L, ranks, tvals = [], [], None, [], None, [], []
    for line in open(os.path.join(HERE, "c1_fullgrid_20steps.txt")):
        if line.startswith("#"):
            continue
        tag, *rest = line.split()
        if tag == "L":
            L = float(rest[0])
        elif tag == "phi":
            idx.append([int(x) for x in rest[:4]])
            vals.append(complex(float(rest[4]), float(rest[5])))
        elif tag == "mean":
            mean = np.array([float(x) for x in rest])
        elif tag == "cov":
            cov.append([float(x) for x in rest])
        elif tag == "ttranks":
            ranks.append([int(x) for x in rest])
        elif tag == "ttphi":
            tvals.append(complex(float(rest[0]), float(rest[1])))
    return (L, np.array(idx, dtype=np.int32), np.array(vals), mean, np.array(cov),
            np.array(ranks, dtype=np.int32), np.array(tvals))


if __name__ == "__main__":
    main()
