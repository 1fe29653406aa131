"""Pins of the oracle's Lindbladian and exact steady states against what the paper and the mathematics fix."""
import numpy as np
import pytest

from oracle import lindblad
from paper_2502_20723_gb300 import synth


def _general_problem():
    """3 sites, all Pauli kinds, a two-site YX string, a non-Hermitian general jump and sigma^-."""
    rng = np.random.default_rng(3)
    Lgen = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
    return {"n_sites": 3,
            "terms": [(0.7, ((0, "X"), (1, "X"))), (-0.3, ((1, "Y"), (2, "Y"))), (0.5, ((2, "Z"), (0, "Z"))),
                      (0.2, ((0, "Y"), (2, "X"))), (0.9, ((1, "X"),)), (-0.4, ((2, "Y"),)), (0.25, ((0, "Z"),))],
            "jumps": [(0, synth.SIGMA_MINUS, 1.0), (1, synth.SIGMA_MINUS, 0.5), (2, Lgen, 0.3)]}


@pytest.mark.parametrize("g", [0.5, 1.0, 2.0])
def test_single_qubit_closed_form(g):
    """Null vector of the N=1 Lindbladian = the closed-form driven-dissipative qubit (large-g section)."""
    p = {"n_sites": 1, "terms": [(g / 2, ((0, "X"),))], "jumps": [(0, synth.SIGMA_MINUS, 1.0)]}
    rho = lindblad.steady_state_dense(p)
    assert np.abs(rho - lindblad.single_qubit_steady_state(g)).max() < 1e-13


def test_vectorisation_matches_master_equation():
    """Lhat |rho>> (Kronecker form of Eq. VecLin) == vec(-i[H,rho] + sum gamma (L rho L^+ - {L^+L,rho}/2))."""
    p = _general_problem()
    m = 1 << p["n_sites"]
    rng = np.random.default_rng(0)
    rho = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    lhs = lindblad.lindbladian_dense(p) @ rho.reshape(-1)
    rhs = lindblad.master_equation_rhs(p, rho).reshape(-1)
    assert np.abs(lhs - rhs).max() < 1e-12


def test_sigma_minus_convention():
    """sigma^- = (X - iY)/2 = |1><0| lowers bit 0 -> 1 (|0> = spin up)."""
    sm = (lindblad.PAULI["X"] - 1j * lindblad.PAULI["Y"]) / 2
    assert np.allclose(sm, synth.SIGMA_MINUS)
    op = lindblad.site_op(synth.SIGMA_MINUS, 2, 3)
    v = np.zeros(8); v[0b000] = 1
    assert np.argmax(np.abs(op @ v)) == 0b100


@pytest.mark.parametrize("kind", ["ising", "xyz", "general"])
def test_trace_preservation(kind):
    """<<I| Lhat = 0 (GKSL property (iii))."""
    p = {"ising": synth.ising_chain(4), "xyz": synth.xyz_chain(4, Bx=-1.0, By=0.3, Bz=0.1),
         "general": _general_problem()}[kind]
    m = 1 << p["n_sites"]
    tr = np.eye(m).reshape(-1)
    assert np.abs(tr @ lindblad.lindbladian_dense(p)).max() < 1e-12


@pytest.mark.parametrize("kind", ["ising", "xyz_field", "general"])
def test_row_elements_match_dense(kind):
    """Element-wise rows (used for the sample-based estimator) == rows of the Kronecker-built Lhat."""
    p = {"ising": synth.ising_chain(4, g=1.3), "xyz_field": synth.xyz_chain(4, 1.4, 2.0, 1.0, -1.0, 0.5, 0.1),
         "general": _general_problem()}[kind]
    n = p["n_sites"]
    L = lindblad.lindbladian_dense(p)
    for x in range(4 ** n):
        a, b = x >> n, x & ((1 << n) - 1)
        row = lindblad.lindbladian_row(p, a, b)
        dense = {(int(y) >> n, int(y) & ((1 << n) - 1)): L[x, y] for y in np.nonzero(L[x])[0]}
        for k in set(row) | set(dense):
            assert abs(row.get(k, 0) - dense.get(k, 0)) < 1e-12, (x, k)


def test_steady_state_properties():
    """rho_ss is Hermitian, positive semidefinite, unit trace, and Lhat rho_ss = 0; the gap is open."""
    p = synth.ising_chain(4)
    rho = lindblad.steady_state_dense(p)
    assert np.abs(rho - rho.conj().T).max() < 1e-12
    assert np.linalg.eigvalsh((rho + rho.conj().T) / 2).min() > -1e-12
    assert abs(np.trace(rho) - 1) < 1e-12
    L = lindblad.lindbladian_dense(p)
    assert np.linalg.norm(L @ rho.reshape(-1)) < 1e-11
    ev = np.sort(np.abs(np.linalg.eigvals(L)))
    assert ev[0] < 1e-10 and ev[1] > 1e-3       # unique null vector


def test_dark_state_ising_g0():
    """g = 0: |1...1><1...1| is the steady state, purity 1 (purity section)."""
    p = synth.ising_chain(5, g=0.0)
    rho = lindblad.steady_state_dense(p)
    assert abs(rho[-1, -1] - 1) < 1e-12
    assert abs(np.trace(rho @ rho).real - 1) < 1e-12


def test_dark_state_xyz_isotropic_xy():
    """XYZ with Jx = Jy conserves total sigma^z, and sigma^- kills |1>: the all-|1> state is dark."""
    p = synth.xyz_chain(4, Jx=1.0, Jy=1.0, Jz=1.0)
    rho = lindblad.steady_state_propagate(p, tol=1e-11)
    assert abs(rho[-1, -1] - 1) < 1e-8


@pytest.mark.parametrize("g", [0.7, 3.0])
def test_decoupled_limit_is_product_state(g):
    """V = 0: the sites decouple and rho_ss is the tensor product of single-qubit steady states;
    purity -> 1/2^N as g -> infinity (large-g limit in the purity section)."""
    n = 3
    p = synth.ising_chain(n, V=0.0, g=g)
    rho = lindblad.steady_state_dense(p)
    r1 = lindblad.single_qubit_steady_state(g)
    prod = np.array([[1.0]])
    for _ in range(n):
        prod = np.kron(r1, prod)
    assert np.abs(rho - prod).max() < 1e-12
    big = lindblad.steady_state_dense(synth.ising_chain(n, V=0.0, g=200.0))
    assert abs(np.trace(big @ big).real - 1 / 2 ** n) < 1e-3


@pytest.mark.parametrize("n,g", [(4, 1.0), (4, 2.5), (5, 1.6)])
def test_ising_sum_rule(n, g):
    """d<sigma^z>/dt = g <sigma^y> - gamma (1 + <sigma^z>) = 0 in the steady state (site-averaged).
    Derived from the Ising H and sigma^- jumps; it also fixes the signs of the observables."""
    p = synth.ising_chain(n, V=2.0, g=g)
    rho = lindblad.steady_state_dense(p)
    sy = np.mean([np.trace(lindblad.site_op(lindblad.PAULI["Y"], i, n) @ rho).real for i in range(n)])
    sz = np.mean([np.trace(lindblad.site_op(lindblad.PAULI["Z"], i, n) @ rho).real for i in range(n)])
    assert abs(g * sy - (1 + sz)) < 1e-11


def test_propagation_matches_dense():
    p = synth.xyz_chain(4, Jx=0.9)
    a = lindblad.steady_state_dense(p)
    b = lindblad.steady_state_propagate(p, tol=1e-12)
    assert np.abs(a - b).max() < 1e-10


def test_golden_ed_observables_are_consistent():
    """The stored exact steady states (tests/golden/ed_observables.json, written by
    tests/golden/make_golden.py from the oracle): every Ising entry, chain or 2D torus, obeys the
    site-averaged sum rule g <sigma^y> = gamma (1 + <sigma^z>) (the sigma^z sigma^z bonds commute with
    sigma^z_i, so the rule holds on any lattice); the 2 x 2 torus is the 4-site ring; purities lie in
    [2^-N, 1]."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "ed_observables.json")))
    assert {"heis_n5_By0.5", "ising2d_2x2_V2_g1", "ising2d_2x3_V2_g1"} <= set(gold)
    for name, e in gold.items():
        pr = e["problem"]
        n = pr["n"] if "n" in pr else pr["mx"] * pr["ny"]
        assert 2.0 ** -n - 1e-9 <= e["purity"] <= 1.0 + 1e-9, name
        if name.startswith("ising"):
            assert pr["g"] * e["sy"] == pytest.approx(pr["gamma"] * (1.0 + e["sz"]), abs=1e-8), name
    for q in ("sx", "sy", "sz", "purity"):
        assert gold["ising2d_2x2_V2_g1"][q] == pytest.approx(gold["ising_n4_V2_g1"][q], abs=1e-10)


def test_golden_propagated_states_carry_their_certificates():
    """Steady states too large for the dense LU (N = 8 and the 10-site Heisenberg chain with fields of the
    Heisenberg section) come from RK4 propagation; each stores the certificate computed from the state
    itself: ||Lhat rho|| / ||rho|| below 1e-10 (the steady-state equation), rho Hermitian and positive
    semidefinite to 1e-10, unit trace."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "ed_observables.json")))
    assert "heis_n10_By0.5" in gold
    for name, e in gold.items():
        if e["method"].startswith("RK4"):
            c = e["certificate"]
            assert c["residual"] < 1e-10, name
            assert c["herm_err"] < 1e-10, name
            assert c["min_eig"] > -1e-10, name
            assert abs(c["trace"] - 1.0) < 1e-12, name
            for q in ("sx", "sy", "sz"):
                assert -1.0 <= e[q] <= 1.0, name
