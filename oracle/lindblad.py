"""Vectorised Lindbladian and exact steady states (oracle; test infrastructure only).

Follows the paper's vectorisation appendix: |rho>> = sum rho(a,b)|a>|b>, A rho B -> (A (x) B^T)|rho>>,
and Eq. VecLin:
  Lhat = -i(H (x) I - I (x) H^T) + sum_i gamma_i [L_i (x) L_i^* - 1/2 (L_i^dag L_i (x) I + I (x) L_i^T L_i^*)].
Basis index of a configuration: s = sum_i bit_i 2^i (bit i = site i). Doubled index x = sigma*2^N + sigma'.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

PAULI = {
    "I": np.eye(2, dtype=np.complex128),
    "X": np.array([[0, 1], [1, 0]], dtype=np.complex128),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    "Z": np.array([[1, 0], [0, -1]], dtype=np.complex128),
}


def site_op(op: np.ndarray, site: int, n: int, sparse: bool = False):
    """Embed a single-site 2x2 operator on `site` of an n-site register (bit `site` of the index)."""
    if sparse:
        hi = sp.identity(1 << (n - 1 - site), dtype=np.complex128, format="csr")
        lo = sp.identity(1 << site, dtype=np.complex128, format="csr")
        return sp.kron(sp.kron(hi, sp.csr_matrix(op)), lo, format="csr")
    return np.kron(np.kron(np.eye(1 << (n - 1 - site)), op), np.eye(1 << site))


def hamiltonian(problem: dict, sparse: bool = False):
    """H = sum_terms coef * prod_sites Pauli (the Ising / Heisenberg Hamiltonians as term lists)."""
    n = problem["n_sites"]
    dim = 1 << n
    H = sp.csr_matrix((dim, dim), dtype=np.complex128) if sparse else np.zeros((dim, dim), np.complex128)
    for coef, ops in problem["terms"]:
        P = sp.identity(dim, dtype=np.complex128, format="csr") if sparse else np.eye(dim, dtype=np.complex128)
        for site, p in ops:
            P = P @ site_op(PAULI[p], site, n, sparse)
        H = H + coef * P
    return H


def jump_ops(problem: dict, sparse: bool = False):
    n = problem["n_sites"]
    return [(site_op(np.asarray(L, np.complex128), s, n, sparse), rate) for s, L, rate in problem["jumps"]]


def lindbladian_dense(problem: dict) -> np.ndarray:
    """Dense vectorised Lindbladian, Eq. VecLin written out with Kronecker products (N <= 6)."""
    n = problem["n_sites"]
    assert n <= 6, "dense Lindbladian is for N <= 6"
    H = hamiltonian(problem)
    I = np.eye(1 << n, dtype=np.complex128)
    Lh = -1j * (np.kron(H, I) - np.kron(I, H.T))
    for L, g in jump_ops(problem):
        LdL = L.conj().T @ L
        Lh = Lh + g * (np.kron(L, L.conj()) - 0.5 * (np.kron(LdL, I) + np.kron(I, L.T @ L.conj())))
    return Lh


def lindbladian_sparse(problem: dict):
    """Same operator as lindbladian_dense, as a scipy CSR matrix (N <= 10)."""
    n = problem["n_sites"]
    H = hamiltonian(problem, sparse=True)
    I = sp.identity(1 << n, dtype=np.complex128, format="csr")
    Lh = -1j * (sp.kron(H, I) - sp.kron(I, H.T))
    for L, g in jump_ops(problem, sparse=True):
        LdL = L.conj().T @ L
        Lh = Lh + g * (sp.kron(L, L.conj()) - 0.5 * (sp.kron(LdL, I) + sp.kron(I, L.T @ L.conj())))
    return sp.csr_matrix(Lh)


def master_equation_rhs(problem: dict, rho: np.ndarray) -> np.ndarray:
    """d rho/dt = -i[H, rho] + sum gamma (L rho L^dag - 1/2 {L^dag L, rho}) in matrix form (Eq. Lindblad, hbar=1)."""
    H = hamiltonian(problem)
    out = -1j * (H @ rho - rho @ H)
    for L, g in jump_ops(problem):
        LdL = L.conj().T @ L
        out = out + g * (L @ rho @ L.conj().T - 0.5 * (LdL @ rho + rho @ LdL))
    return out


# ------------------------------------------------------------------ single-row elements
def _local_elem(ops: dict, n: int, bra: int, ket: int) -> complex:
    """<bra| prod_site ops[site] |ket> for single-site 2x2 operators on a subset of sites (identity elsewhere)."""
    val = 1.0 + 0j
    for i in range(n):
        b, k = (bra >> i) & 1, (ket >> i) & 1
        if i in ops:
            val *= ops[i][b, k]
        elif b != k:
            return 0j
        if val == 0:
            return 0j
    return val


def lindbladian_row(problem: dict, sig: int, sigp: int) -> dict:
    """Nonzero elements Lhat_{(sig,sigp),(eta,eta')} of one row, element by element:
        -i H_{sig,eta} d_{sigp,eta'} + i H_{eta',sigp} d_{sig,eta}
        + sum gamma [L_{sig,eta} L*_{sigp,eta'} - 1/2 (L^dag L)_{sig,eta} d_{sigp,eta'} - 1/2 (L^dag L)_{eta',sigp} d_{sig,eta}]
    (Eq. VecLin with the index map A rho B -> A (x) B^T). Returns {(eta, eta'): value}."""
    n = problem["n_sites"]
    out: dict = {(sig, sigp): 0j}

    def add(key, v):
        if v != 0:
            out[key] = out.get(key, 0j) + v

    for coef, ops in problem["terms"]:
        d = {}
        for site, p in ops:
            d[site] = d[site] @ PAULI[p] if site in d else PAULI[p]
        # candidate kets: only sites in the term may differ
        sites = sorted(d)
        for mask in range(1 << len(sites)):
            eta = sig
            etap = sigp
            for j, s in enumerate(sites):
                if (mask >> j) & 1:
                    eta ^= 1 << s
                    etap ^= 1 << s
            add((eta, sigp), -1j * coef * _local_elem(d, n, sig, eta))
            add((sig, etap), 1j * coef * _local_elem(d, n, etap, sigp))
    for site, L, g in problem["jumps"]:
        L = np.asarray(L, np.complex128)
        LdL = L.conj().T @ L
        for a in range(2):
            eta = (sig & ~(1 << site)) | (a << site)
            etap_ = (sigp & ~(1 << site)) | (a << site)
            add((eta, sigp), -0.5 * g * LdL[(sig >> site) & 1, a])
            add((sig, etap_), -0.5 * g * LdL[a, (sigp >> site) & 1])
            for b in range(2):
                etap = (sigp & ~(1 << site)) | (b << site)
                add((eta, etap), g * L[(sig >> site) & 1, a] * np.conj(L[(sigp >> site) & 1, b]))
    return out


# ------------------------------------------------------------------ exact steady state
def steady_state_dense(problem: dict) -> np.ndarray:
    """Null vector of Lhat (Lhat rho_ss = 0) for N <= 6, normalised to Tr rho = 1.
    The steady state is assumed unique (paper, steady-state section), so replacing the row of the
    diagonal element (0,0) by the trace functional <<I| (a left null vector: trace preservation)
    gives a nonsingular system with right-hand side e_0. Returns rho as a 2^N x 2^N matrix."""
    n = problem["n_sites"]
    m = 1 << n
    A = lindbladian_dense(problem).copy()
    tr = np.zeros(m * m, np.complex128)
    tr[np.arange(m) * m + np.arange(m)] = 1.0
    A[0, :] = tr
    b = np.zeros(m * m, np.complex128)
    b[0] = 1.0
    v = np.linalg.solve(A, b)
    return v.reshape(m, m)


def steady_state_propagate(problem: dict, dt: float = 0.02, tol: float = 1e-12, max_steps: int = 200000,
                           check_every: int = 50) -> np.ndarray:
    """Steady state as the t -> infinity limit of d|rho>>/dt = Lhat|rho>> (classical RK4, FP64),
    from the maximally mixed state, until ||Lhat rho|| / ||rho|| < tol. For N up to ~10."""
    n = problem["n_sites"]
    m = 1 << n
    Lh = lindbladian_sparse(problem)
    v = (np.eye(m, dtype=np.complex128) / m).reshape(-1)
    for step in range(max_steps):
        k1 = Lh @ v
        if step % check_every == 0:
            res = np.linalg.norm(k1) / np.linalg.norm(v)
            if res < tol:
                break
        k2 = Lh @ (v + 0.5 * dt * k1)
        k3 = Lh @ (v + 0.5 * dt * k2)
        k4 = Lh @ (v + dt * k3)
        v = v + (dt / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
    rho = v.reshape(m, m)
    return rho / np.trace(rho)


def single_qubit_steady_state(g: float) -> np.ndarray:
    """Closed form of the driven-dissipative qubit (gamma = 1), large-g section of the paper:
    rho = [[g^2, -i g], [i g, 1 + g^2]] / (1 + 2 g^2)."""
    return np.array([[g * g, -1j * g], [1j * g, 1 + g * g]], dtype=np.complex128) / (1 + 2 * g * g)
