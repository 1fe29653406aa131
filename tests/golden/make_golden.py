"""Writes tests/golden/ed_observables.json: exact steady-state observables of the workloads' problems
(Ising and XYZ chains, the Heisenberg chain with fields, the 2D Ising torus), computed by the oracle only
(dense LU for N <= 6, RK4 propagation of Eq. VecLin for N = 8).

    python tests/golden/make_golden.py
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
    "ising2d_2x2_V2_g1": (synth.ising_2d, dict(mx=2, ny=2, V=2.0, g=1.0, gamma=1.0)),
    "ising2d_2x3_V2_g1": (synth.ising_2d, dict(mx=2, ny=3, V=2.0, g=1.0, gamma=1.0)),
}


def main():
    res = {}
    for name, (fn, kw) in CASES.items():
        p = fn(**kw)
        rho = lindblad.steady_state_dense(p) if p["n_sites"] <= 6 else lindblad.steady_state_propagate(p)
        res[name] = {"problem": kw, "method": "dense LU" if p["n_sites"] <= 6 else "RK4 dt=0.02 to 1e-12",
                     **observables(p, rho)}
        print(name, res[name], flush=True)
    with open(os.path.join(HERE, "ed_observables.json"), "w") as f:
        json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
