"""The transformer density-operator ansatz in plain FP64 PyTorch CPU ops (oracle; test infrastructure only).

Follows the architecture appendix step by step:
  * two-channel input: channel 1 = sigma (x^l), channel 2 = sigma' (x^r)          (Feature Embedding)
  * embedding: either the paper's two circular convolutions with kernel spanning sites (i, i+1 mod N),
    each followed by the activation (Eq. circ-conv and the next equation), or a 4-entry token table
    indexed by 2*bit(channel 1) + bit(channel 2)
  * per layer: Q = X Wq, K = X Wk, V = X Wv (no bias), per head softmax(Q_h K_h^T / sqrt(d/h)) V_h
    (Eq. attn-head-appendix), concat, X' = concat Wo + X; optional MLP X'' = X' + act(X' W1 + b1) W2 + b2
  * global mean pooling over sites (Eq. global-pool-final), dense layer to [F0, F1], z = F0 + i F1
  * Hermitian symmetrisation log rho(a,b) = log(exp z(a,b) + conj(exp z(b,a))) (Eq. log_sum_exp_conjugate),
    principal branch of the complex logarithm.
Readings where the paper is silent: activation = GELU (tanh form); bit 0 -> spin +1 for the conv inputs;
no bias on Q/K/V/O; biases on conv, MLP and head; no LayerNorm.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from paper_2502_20723_gb300.synth import param_shapes

DT = torch.float64


def unflatten(spec: dict, theta) -> dict:
    """Split the flat parameter vector into named tensors (order of synth.param_shapes)."""
    th = theta if isinstance(theta, torch.Tensor) else torch.as_tensor(np.asarray(theta), dtype=DT)
    out, off = {}, 0
    for name, shape in param_shapes(spec):
        n = int(np.prod(shape))
        out[name] = th[off:off + n].reshape(shape)
        off += n
    assert off == th.numel(), (off, th.numel())
    return out


def gelu(u: torch.Tensor) -> torch.Tensor:
    """GELU, tanh form: 0.5 u (1 + tanh(sqrt(2/pi) (u + 0.044715 u^3)))."""
    return 0.5 * u * (1.0 + torch.tanh(math.sqrt(2.0 / math.pi) * (u + 0.044715 * u ** 3)))


def bits(words: np.ndarray, n: int) -> torch.Tensor:
    """[B] uint32 words -> [B, n] float64 bits (bit i = site i)."""
    w = np.asarray(words, dtype=np.uint64)
    b = (w[:, None] >> np.arange(n, dtype=np.uint64)[None, :]) & np.uint64(1)
    return torch.as_tensor(b.astype(np.float64), dtype=DT)


def embed(spec: dict, P: dict, b1: torch.Tensor, b2: torch.Tensor) -> torch.Tensor:
    """Embedding of sequences whose channel-1 bits are b1 and channel-2 bits b2 ([S, N] each) -> [S, N, d]."""
    if spec["embed"] == "token":
        tok = (2 * b1 + b2).long()
        return P["E"][tok]
    # paper: spins as +-1, circular convolution over sites (i, i+1 mod N), 2 -> C1 -> d channels
    x = torch.stack([1.0 - 2.0 * b1, 1.0 - 2.0 * b2], dim=-1)          # [S, N, 2]
    xs = torch.roll(x, shifts=-1, dims=1)                                # site i+1 (circular)
    h1 = torch.einsum("snc,cf->snf", x, P["Wc1"][0]) + torch.einsum("snc,cf->snf", xs, P["Wc1"][1]) + P["bc1"]
    h1 = gelu(h1)
    h1s = torch.roll(h1, shifts=-1, dims=1)
    h2 = torch.einsum("snc,cf->snf", h1, P["Wc2"][0]) + torch.einsum("snc,cf->snf", h1s, P["Wc2"][1]) + P["bc2"]
    return gelu(h2)


def encoder(spec: dict, P: dict, X: torch.Tensor) -> torch.Tensor:
    """Attention layers (+ optional MLP), each with its residual connection."""
    S, N, d = X.shape
    h = spec["n_heads"]
    dh = d // h
    for l in range(spec["n_layers"]):
        Q = X @ P[f"Wq{l}"]
        K = X @ P[f"Wk{l}"]
        V = X @ P[f"Wv{l}"]
        heads = []
        for j in range(h):
            sl = slice(j * dh, (j + 1) * dh)
            scores = Q[:, :, sl] @ K[:, :, sl].transpose(1, 2) / math.sqrt(dh)
            A = torch.softmax(scores, dim=-1)
            heads.append(A @ V[:, :, sl])
        X = torch.cat(heads, dim=-1) @ P[f"Wo{l}"] + X
        if spec["mlp_ratio"] > 0:
            X = gelu(X @ P[f"W1_{l}"] + P[f"b1_{l}"]) @ P[f"W2_{l}"] + P[f"b2_{l}"] + X
    return X


def z_of(spec: dict, P: dict, b1: torch.Tensor, b2: torch.Tensor) -> torch.Tensor:
    """[F0, F1] of one ordering of the two channels ([S, 2] real); z = F0 + i F1."""
    X = encoder(spec, P, embed(spec, P, b1, b2))
    hpool = X.mean(dim=1)
    return hpool @ P["Wh"] + P["bh"]


def log_rho_parts(spec: dict, theta, sig: np.ndarray, sigp: np.ndarray, n_sites: int):
    """(Re, Im) of log rho(sigma, sigma') = log(exp z(sigma,sigma') + conj exp z(sigma',sigma)), principal
    branch, written in real arithmetic: with w = z(sigma,sigma'), v = conj z(sigma',sigma) and m = max(Re w, Re v),
    s = e^{Re w - m} e^{i Im w} + e^{Re v - m} e^{i Im v}, log rho = m + log|s| + i arg(s)."""
    P = unflatten(spec, theta)
    bs, bp = bits(sig, n_sites), bits(sigp, n_sites)
    FA = z_of(spec, P, bs, bp)
    FB = z_of(spec, P, bp, bs)
    wr, wi = FA[:, 0], FA[:, 1]
    vr, vi = FB[:, 0], -FB[:, 1]
    m = torch.maximum(wr, vr).detach()
    ea, eb = torch.exp(wr - m), torch.exp(vr - m)
    sr = ea * torch.cos(wi) + eb * torch.cos(vi)
    si = ea * torch.sin(wi) + eb * torch.sin(vi)
    return m + 0.5 * torch.log(sr * sr + si * si), torch.atan2(si, sr)


def log_rho(spec: dict, theta, sig: np.ndarray, sigp: np.ndarray, n_sites: int) -> torch.Tensor:
    """log rho for a batch of doubled configurations ([B] complex128). Differentiable in theta."""
    re, im = log_rho_parts(spec, theta, sig, sigp, n_sites)
    return torch.complex(re, im)


def log_rho_np(spec: dict, theta, sig, sigp, n_sites: int) -> np.ndarray:
    with torch.no_grad():
        return log_rho(spec, theta, sig, sigp, n_sites).numpy()
