"""Metropolis-Hastings sampling of P(sigma, sigma') ~ |rho|^2 with single-bit proposals
("Efficient Sampling Strategy" section: symmetric local proposal, acceptance min(1, P'/P)).
Oracle copy, FP64 log rho (test infrastructure only).

Random stream (a written convention both sides implement): proposal number t (64-bit, running over
calls) of chain c uses Philox4x32-10 with key (seed_lo, seed_hi) and counter (c, t_lo, t_hi, 0); output
x0 picks the bit k = ((x0 >> 8) * 2N) >> 24 (k < N flips sigma_k, else sigma'_{k-N}), and
u = (x1 >> 8) * 2^-24; the move is accepted iff u < exp(min(0, 2 (Re log rho' - Re log rho))).
A sweep is 2N proposals.
"""
from __future__ import annotations

import numpy as np

from .philox import philox4x32_10
from .transformer import log_rho_np


def draws(seed: int, chains: np.ndarray, t: int, n_sites: int):
    t = np.uint64(t)
    x0, x1, _, _ = philox4x32_10(chains, t & np.uint64(0xFFFFFFFF), t >> np.uint64(32), 0,
                                 seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    k = ((x0.astype(np.uint64) >> np.uint64(8)) * np.uint64(2 * n_sites)) >> np.uint64(24)
    u = (x1 >> np.uint32(8)).astype(np.float64) * 2.0 ** -24
    return k.astype(np.int64), u


def metropolis(spec: dict, theta, sig, sigp, n_sites: int, n_sweeps: int, seed: int, counter: int,
               record: bool = False):
    """Run n_sweeps sweeps on every chain. Returns (sig, sigp, accepted_count, per-sweep samples,
    min |2 Re dlogrho - log u| margin per chain)."""
    sig = np.array(sig, dtype=np.uint32)
    sigp = np.array(sigp, dtype=np.uint32)
    nc = len(sig)
    chains = np.arange(nc, dtype=np.uint64)
    lr = log_rho_np(spec, theta, sig, sigp, n_sites)
    acc = 0
    samples = []
    margin = np.full(nc, np.inf)
    for sw in range(n_sweeps):
        for j in range(2 * n_sites):
            t = counter + sw * 2 * n_sites + j
            k, u = draws(seed, chains, t, n_sites)
            ns, nsp = sig.copy(), sigp.copy()
            left = k < n_sites
            ns[left] ^= (np.uint32(1) << k[left].astype(np.uint32))
            nsp[~left] ^= (np.uint32(1) << (k[~left] - n_sites).astype(np.uint32))
            lrn = log_rho_np(spec, theta, ns, nsp, n_sites)
            delta = 2.0 * (lrn.real - lr.real)
            with np.errstate(divide="ignore"):
                margin = np.minimum(margin, np.abs(np.minimum(delta, 0.0) - np.log(u)))
            a = u < np.exp(np.minimum(0.0, delta))
            sig[a], sigp[a], lr[a] = ns[a], nsp[a], lrn[a]
            acc += int(a.sum())
        if record:
            samples.append((sig.copy(), sigp.copy()))
    return sig, sigp, acc, samples, margin
