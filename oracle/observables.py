"""Mixed-state observables and purity (supplement, "Mixed-State Observables"; the magnetisation figures).

Oracle copy in FP64; test infrastructure only (tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline leg may import it; the product path never does).

<A> = Tr(rho A) / Tr(rho) is a classical average over P(alpha) = rho(alpha, alpha) / Tr(rho) of the local
estimator A~(alpha) = sum_beta rho(alpha, beta) / rho(alpha, alpha) <beta|A|alpha>.  The ansatz does not
force rho(alpha, alpha) >= 0, so the samples are drawn from |rho(alpha, alpha)| and every term carries
s(alpha) = sign rho(alpha, alpha):  <A> = E[s A~] / E[s].

Written conventions both sides implement (no shared code):
  bit i of a configuration word is site i, bit value 0 = |0> (sigma^z = +1);
  rho(alpha, beta) = <alpha|rho|beta> = exp(log rho(sigma = alpha, sigma' = beta));
  A = (1/N) sum_i sigma^a_i with <alpha ^ e_i|sigma^x_i|alpha> = 1,
  <alpha ^ e_i|sigma^y_i|alpha> = i (1 - 2 alpha_i), <alpha|sigma^z_i|alpha> = 1 - 2 alpha_i;
  diagonal Metropolis: the Philox stream of the |rho|^2 sampler with N choices per draw,
  bit k = ((x0 >> 8) * N) >> 24 flips site k of alpha, u = (x1 >> 8) 2^-24, accept iff
  u < exp(min(0, Re log rho(alpha', alpha') - Re log rho(alpha, alpha))); a sweep is N proposals,
  t = counter + sweep * N + j.
Purity: with (sigma, sigma') drawn from |rho|^2 / Tr(rho^2) (the main sampler),
  E[rho(sigma, sigma) rho(sigma', sigma') / |rho(sigma, sigma')|^2] = Tr(rho)^2 / Tr(rho^2),
so Tr(rho^2) / Tr(rho)^2 is the inverse of that mean.
"""
from __future__ import annotations

import numpy as np

from .lindblad import PAULI, site_op
from .philox import philox4x32_10
from .transformer import log_rho_np


def draws_diag(seed: int, chains: np.ndarray, t: int, n_sites: int):
    """Proposal t of every chain: (site k < N, uniform u)."""
    t = np.uint64(t)
    x0, x1, _, _ = philox4x32_10(chains, t & np.uint64(0xFFFFFFFF), t >> np.uint64(32), 0,
                                 seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    k = ((x0.astype(np.uint64) >> np.uint64(8)) * np.uint64(n_sites)) >> np.uint64(24)
    u = (x1 >> np.uint32(8)).astype(np.float64) * 2.0 ** -24
    return k.astype(np.int64), u


def metropolis_diag(spec: dict, theta, alpha, n_sites: int, n_sweeps: int, seed: int, counter: int,
                    record: bool = False):
    """Chains on P(alpha) ~ |rho(alpha, alpha)|.  Returns (alpha, accepted, per-sweep samples, min margin
    |Re dlog rho - log u| of every chain's accept decisions)."""
    a = np.array(alpha, dtype=np.uint32)
    nc = len(a)
    chains = np.arange(nc, dtype=np.uint64)
    lr = log_rho_np(spec, theta, a, a, n_sites)
    acc = 0
    samples = []
    margin = np.full(nc, np.inf)
    for sw in range(n_sweeps):
        for j in range(n_sites):
            k, u = draws_diag(seed, chains, counter + sw * n_sites + j, n_sites)
            na = a ^ (np.uint32(1) << k.astype(np.uint32))
            lrn = log_rho_np(spec, theta, na, na, n_sites)
            delta = lrn.real - lr.real
            with np.errstate(divide="ignore"):
                margin = np.minimum(margin, np.abs(np.minimum(delta, 0.0) - np.log(u)))
            ok = u < np.exp(np.minimum(0.0, delta))
            a[ok], lr[ok] = na[ok], lrn[ok]
            acc += int(ok.sum())
        if record:
            samples.append(a.copy())
    return a, acc, samples, margin


def magnetisation_local(spec: dict, theta, alpha, n_sites: int):
    """Per sample: s = sign rho(alpha, alpha) and the local estimators (A~x, A~y, A~z) (complex [Ns, 3])."""
    a = np.asarray(alpha, dtype=np.uint32)
    lr0 = log_rho_np(spec, theta, a, a, n_sites)
    s = np.where(np.cos(lr0.imag) < 0.0, -1.0, 1.0)
    A = np.zeros((len(a), 3), dtype=np.complex128)
    for i in range(n_sites):
        b = a ^ np.uint32(1 << i)
        ratio = np.exp(log_rho_np(spec, theta, a, b, n_sites) - lr0)
        zi = 1.0 - 2.0 * ((a >> np.uint32(i)) & np.uint32(1)).astype(np.float64)
        A[:, 0] += ratio
        A[:, 1] += ratio * 1j * zi
        A[:, 2] += zi
    return s, A / n_sites


def magnetisation_estimate(s: np.ndarray, A: np.ndarray) -> np.ndarray:
    """(<sigma^x>, <sigma^y>, <sigma^z>) = Re sum s A~ / sum s."""
    return (np.asarray(s)[:, None] * A).sum(axis=0).real / np.sum(s)


def density_matrix(spec: dict, theta, n_sites: int) -> np.ndarray:
    """rho[a, b] = rho(sigma = a, sigma' = b) of the model, scaled by a positive constant."""
    dim = 1 << n_sites
    a = np.repeat(np.arange(dim, dtype=np.uint32), dim)
    b = np.tile(np.arange(dim, dtype=np.uint32), dim)
    lr = log_rho_np(spec, theta, a, b, n_sites)
    return np.exp(lr - lr.real.max()).reshape(dim, dim)


def exact_magnetisation(spec: dict, theta, n_sites: int) -> np.ndarray:
    """Tr(rho A) / Tr(rho) for A = (1/N) sum_i sigma^{x,y,z}_i, by dense matrices."""
    rho = density_matrix(spec, theta, n_sites)
    tr = np.trace(rho)
    out = []
    for p in ("X", "Y", "Z"):
        A = sum(site_op(PAULI[p], i, n_sites) for i in range(n_sites)) / n_sites
        out.append((np.trace(rho @ A) / tr).real)
    return np.array(out)


def purity_local(spec: dict, theta, sig, sigp, n_sites: int) -> np.ndarray:
    """Per sample (sigma, sigma'): Re rho(sigma, sigma) rho(sigma', sigma') / |rho(sigma, sigma')|^2."""
    s0 = np.asarray(sig, dtype=np.uint32)
    s1 = np.asarray(sigp, dtype=np.uint32)
    la = log_rho_np(spec, theta, s0, s0, n_sites)
    lb = log_rho_np(spec, theta, s1, s1, n_sites)
    lc = log_rho_np(spec, theta, s0, s1, n_sites)
    return np.exp(la + lb - 2.0 * lc.real).real


def exact_purity(spec: dict, theta, n_sites: int) -> float:
    """Tr(rho^2) / Tr(rho)^2 of the model, by its dense matrix (Tr(rho^2) = sum |rho(a, b)|^2 for the
    Hermitian rho of the symmetrised ansatz)."""
    rho = density_matrix(spec, theta, n_sites)
    return float((np.trace(rho @ rho) / np.trace(rho) ** 2).real)
