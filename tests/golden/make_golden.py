"""Writes tests/golden/ed_observables.json: exact steady-state observables of the workloads' problems
(Ising and XYZ chains, the Heisenberg chain with fields, the 2D Ising torus), computed by the oracle only
(dense LU for N <= 6, RK4 propagation of Eq. VecLin for N = 8 and 10).  Every propagated state also
stores its certificate: the residual ||Lhat rho|| / ||rho||, the Hermiticity error and the smallest
eigenvalue of rho (unit trace by construction).

    python tests/golden/make_golden.py             # every case
    python tests/golden/make_golden.py heis_n10_By0.5   # the named cases, merged into the file
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import lindblad  # noqa: E402
from paper_2502_20723_gb300 import synth  # noqa: E402


def observables(problem, rho):
    n = problem["n_sites"]
    out = {}
    for p in "XYZ":
        A = sum(lindblad.site_op(lindblad.PAULI[p], i, n, sparse=True) for i in range(n)) / n
        out["s" + p.lower()] = float((A @ rho).trace().real / np.trace(rho).real)
    out["purity"] = float(np.trace(rho @ rho).real / np.trace(rho).real ** 2)
    return out


CASES = {
    "ising_n4_V2_g1": (synth.ising_chain, dict(n=4, V=2.0, g=1.0, gamma=1.0)),
    "ising_n6_V2_g1": (synth.ising_chain, dict(n=6, V=2.0, g=1.0, gamma=1.0)),
    "ising_n6_V2_g4": (synth.ising_chain, dict(n=6, V=2.0, g=4.0, gamma=1.0)),
    "ising_n8_V2_g1": (synth.ising_chain, dict(n=8, V=2.0, g=1.0, gamma=1.0)),
    "xyz_n4_Jx0.9": (synth.xyz_chain, dict(n=4, Jx=0.9, Jy=1.0, Jz=1.0, gamma=1.0)),
    "xyz_n8_Jx0.9": (synth.xyz_chain, dict(n=8, Jx=0.9, Jy=1.0, Jz=1.0, gamma=1.0)),
    # Heisenberg chain with fields (J = (1.4, 2.0, 1.0), B = (-1.0, B_y, 0.1)) and the 2D Ising torus
    "heis_n5_By0.5": (synth.xyz_chain, dict(n=5, Jx=1.4, Jy=2.0, Jz=1.0, Bx=-1.0, By=0.5, Bz=0.1, gamma=1.0)),
    "heis_n10_By0.5": (synth.xyz_chain, dict(n=10, Jx=1.4, Jy=2.0, Jz=1.0, Bx=-1.0, By=0.5, Bz=0.1, gamma=1.0)),
    "ising2d_2x2_V2_g1": (synth.ising_2d, dict(mx=2, ny=2, V=2.0, g=1.0, gamma=1.0)),
    "ising2d_2x3_V2_g1": (synth.ising_2d, dict(mx=2, ny=3, V=2.0, g=1.0, gamma=1.0)),
}


def certificate(problem, rho):
    """||Lhat rho|| / ||rho|| (vectorised), the Hermiticity error and the smallest eigenvalue of rho."""
    Lh = lindblad.lindbladian_sparse(problem)
    v = rho.reshape(-1)
    return {"residual": float(np.linalg.norm(Lh @ v) / np.linalg.norm(v)),
            "herm_err": float(np.abs(rho - rho.conj().T).max()),
            "min_eig": float(np.linalg.eigvalsh(0.5 * (rho + rho.conj().T)).min()),
            "trace": float(np.trace(rho).real)}


def main(names=None):
    path = os.path.join(HERE, "ed_observables.json")
    res = {}
    if names and os.path.exists(path):
        with open(path) as f:
            res = json.load(f)
    for name, (fn, kw) in CASES.items():
        if names and name not in names:
            continue
        p = fn(**kw)
        dense = p["n_sites"] <= 6
        rho = lindblad.steady_state_dense(p) if dense else lindblad.steady_state_propagate(p)
        res[name] = {"problem": kw, "method": "dense LU" if dense else "RK4 dt=0.02 to 1e-12",
                     **observables(p, rho)}
        if not dense:
            res[name]["certificate"] = certificate(p, rho)
        print(name, res[name], flush=True)
    with open(path, "w") as f:
        json.dump(res, f, indent=1)


if __name__ == "__main__":
    main(sys.argv[1:] or None)
