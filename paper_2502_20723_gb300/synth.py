"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds no arithmetic of the method: it only writes down problem statements
(Pauli-string Hamiltonian terms and jump operators, as the paper states its models) and
draws seeded random parameters and configurations.

Problem statement format (a plain dict):
    n_sites: int                      chain length N (1..32)
    terms:   list of (coef, ((site, pauli), ...))   real coef times a Pauli string on <=2 sites
    jumps:   list of (site, L, rate)  L a 2x2 complex matrix in the basis (|0>, |1>)

Basis convention: bit i of a configuration word is site i; bit value 0 is |0> (sigma^z=+1),
1 is |1> (sigma^z=-1); sigma^- = |1><0| (Ising/Heisenberg sections of the paper: the
lowering operator annihilates |1>, so |1...1> is the dark state at g=0).
"""
from __future__ import annotations

import numpy as np

SIGMA_MINUS = np.array([[0.0, 0.0], [1.0, 0.0]], dtype=np.complex128)


def ising_chain(n: int, V: float = 2.0, g: float = 1.0, gamma: float = 1.0, pbc: bool = True) -> dict:
    """Dissipative transverse-field Ising chain: H = (V/4) sum_i Z_i Z_{i+1} + (g/2) sum_i X_i,
    jump sigma^-_i at rate gamma on every site (Ising section, H and L_i definitions)."""
    terms = []
    nb = n if pbc else n - 1
    for i in range(nb):
        terms.append((V / 4.0, ((i, "Z"), ((i + 1) % n, "Z"))))
    for i in range(n):
        terms.append((g / 2.0, ((i, "X"),)))
    jumps = [(i, SIGMA_MINUS.copy(), gamma) for i in range(n)]
    return {"n_sites": n, "terms": terms, "jumps": jumps}


def xyz_chain(n: int, Jx: float = 0.9, Jy: float = 1.0, Jz: float = 1.0,
              Bx: float = 0.0, By: float = 0.0, Bz: float = 0.0,
              gamma: float = 1.0, pbc: bool = True) -> dict:
    """Dissipative XYZ Heisenberg chain: H = sum_i sum_k (J_k s^k_i s^k_{i+1} + B_k s^k_i),
    jump sigma^-_i at rate gamma (Heisenberg section, H definition)."""
    terms = []
    nb = n if pbc else n - 1
    for i in range(nb):
        j = (i + 1) % n
        for J, p in ((Jx, "X"), (Jy, "Y"), (Jz, "Z")):
            if J != 0.0:
                terms.append((J, ((i, p), (j, p))))
    for i in range(n):
        for B, p in ((Bx, "X"), (By, "Y"), (Bz, "Z")):
            if B != 0.0:
                terms.append((B, ((i, p),)))
    jumps = [(i, SIGMA_MINUS.copy(), gamma) for i in range(n)]
    return {"n_sites": n, "terms": terms, "jumps": jumps}


def ising_2d(mx: int, ny: int, V: float = 2.0, g: float = 1.0, gamma: float = 1.0) -> dict:
    """2D dissipative Ising model on an mx x ny torus, sites numbered i*ny + j
    (2D Ising section: nearest-neighbour ZZ bonds, transverse field, sigma^- jumps)."""
    n = mx * ny
    bonds = set()
    for i in range(mx):
        for j in range(ny):
            a = i * ny + j
            for b in (((i + 1) % mx) * ny + j, i * ny + (j + 1) % ny):
                if a != b:
                    bonds.add((min(a, b), max(a, b)))
    terms = [(V / 4.0, ((a, "Z"), (b, "Z"))) for (a, b) in sorted(bonds)]
    terms += [(g / 2.0, ((i, "X"),)) for i in range(n)]
    jumps = [(i, SIGMA_MINUS.copy(), gamma) for i in range(n)]
    return {"n_sites": n, "terms": terms, "jumps": jumps}


# ---------------------------------------------------------------- transformer shapes
def model_spec(d_model: int, n_heads: int, n_layers: int, mlp_ratio: int = 0,
               embed: str = "token", conv_channels: int = 0) -> dict:
    """Hyper-parameters of the ansatz (no weights)."""
    assert d_model % n_heads == 0
    return {"d_model": d_model, "n_heads": n_heads, "n_layers": n_layers,
            "mlp_ratio": mlp_ratio, "embed": embed, "conv_channels": conv_channels}


def param_shapes(spec: dict) -> list[tuple[str, tuple[int, ...]]]:
    """Flat parameter order shared (as a written convention, not code) by both sides:
    embedding, then per layer Wq, Wk, Wv, Wo [d][d] (row = input feature), then the optional
    MLP W1 [d][r*d], b1, W2 [r*d][d], b2, then the head Wh [d][2], bh [2].
    Token embedding: E [4][d], token = 2*bit(first channel) + bit(second channel).
    Conv embedding: Wc1 [2 offsets][2 channels][C1], bc1 [C1], Wc2 [2][C1][d], bc2 [d]."""
    d, r = spec["d_model"], spec["mlp_ratio"]
    out = []
    if spec["embed"] == "token":
        out.append(("E", (4, d)))
    else:
        c1 = spec["conv_channels"]
        out += [("Wc1", (2, 2, c1)), ("bc1", (c1,)), ("Wc2", (2, c1, d)), ("bc2", (d,))]
    for l in range(spec["n_layers"]):
        for nm in ("Wq", "Wk", "Wv", "Wo"):
            out.append((f"{nm}{l}", (d, d)))
        if r > 0:
            out += [(f"W1_{l}", (d, r * d)), (f"b1_{l}", (r * d,)),
                    (f"W2_{l}", (r * d, d)), (f"b2_{l}", (d,))]
    out += [("Wh", (d, 2)), ("bh", (2,))]
    return out


def num_params(spec: dict) -> int:
    return int(sum(int(np.prod(s)) for _, s in param_shapes(spec)))


def init_params(spec: dict, seed: int = 0, std: float = 0.02) -> np.ndarray:
    """theta ~ N(0, std^2), FP64, in the flat order of param_shapes."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, std, size=num_params(spec)).astype(np.float64)


def random_configs(n_sites: int, count: int, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Uniform random doubled configurations (sigma, sigma') as uint32 bit words."""
    rng = np.random.default_rng(seed)
    mask = np.uint64((1 << n_sites) - 1)
    a = (rng.integers(0, 1 << 32, size=count, dtype=np.uint64) & mask).astype(np.uint32)
    b = (rng.integers(0, 1 << 32, size=count, dtype=np.uint64) & mask).astype(np.uint32)
    return a, b


def all_configs(n_sites: int) -> tuple[np.ndarray, np.ndarray]:
    """Every doubled configuration, index = sigma * 2^N + sigma' (4^N of them)."""
    m = 1 << n_sites
    idx = np.arange(m * m, dtype=np.uint64)
    return (idx >> np.uint64(n_sites)).astype(np.uint32), (idx & np.uint64(m - 1)).astype(np.uint32)


def random_matrix(rows: int, cols: int, seed: int = 0, scale: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((rows, cols)) * scale)


# Workloads (shapes of the paper's dissipative chains, seeded)
WORKLOADS = {
    "ising_n4_d16_l1": dict(problem=("ising", dict(n=4, V=2.0, g=1.0, gamma=1.0)),
                            model=dict(d_model=16, n_heads=2, n_layers=1, mlp_ratio=0)),
    "ising_n8_d32_l2": dict(problem=("ising", dict(n=8, V=2.0, g=1.0, gamma=1.0)),
                            model=dict(d_model=32, n_heads=4, n_layers=2, mlp_ratio=0),
                            chains=64, sweeps=64),
    "xyz_n8_d32_l2": dict(problem=("xyz", dict(n=8, Jx=0.9, Jy=1.0, Jz=1.0, gamma=1.0)),
                          model=dict(d_model=32, n_heads=4, n_layers=2, mlp_ratio=0),
                          samples=4096),
    "ising_n16_d64_l4_mlp4": dict(problem=("ising", dict(n=16, V=2.0, g=1.0, gamma=1.0)),
                                  model=dict(d_model=64, n_heads=8, n_layers=4, mlp_ratio=4),
                                  samples=16384),
}


def make_problem(kind: str, **kw) -> dict:
    return {"ising": ising_chain, "xyz": xyz_chain}[kind](**kw)
