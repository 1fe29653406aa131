"""Pins of the oracle's transformer ansatz: library routines for each stage, special cases and the
symmetries the paper states (Hermiticity, translation invariance)."""
import math

import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import transformer as T
from paper_2502_20723_gb300 import synth

torch.set_default_dtype(torch.float64)


def _spec(embed="token", mlp=0, layers=2, d=16, h=4):
    return synth.model_spec(d, h, layers, mlp, embed=embed, conv_channels=6 if embed == "conv" else 0)


def test_gelu_is_torch_tanh_gelu():
    u = torch.linspace(-6, 6, 1001)
    assert torch.allclose(T.gelu(u), F.gelu(u, approximate="tanh"), atol=1e-15, rtol=0)


def test_attention_layer_is_torch_multihead_attention():
    """One layer without MLP == torch.nn.MultiheadAttention (no bias) + residual."""
    spec = _spec(layers=1, d=16, h=4)
    th = torch.as_tensor(synth.init_params(spec, 1, std=0.3))
    P = T.unflatten(spec, th)
    X = torch.randn(5, 7, 16, generator=torch.Generator().manual_seed(0))
    mha = torch.nn.MultiheadAttention(16, 4, bias=False, batch_first=True).double()
    with torch.no_grad():
        mha.in_proj_weight.copy_(torch.cat([P["Wq0"].T, P["Wk0"].T, P["Wv0"].T], 0))
        mha.out_proj.weight.copy_(P["Wo0"].T)
        ref = mha(X, X, X, need_weights=False)[0] + X
    assert torch.allclose(T.encoder(spec, P, X), ref, atol=1e-13)


def test_mlp_sublayer_is_linear_gelu_linear():
    spec = _spec(layers=1, mlp=4, d=8, h=2)
    th = torch.as_tensor(synth.init_params(spec, 2, std=0.3))
    P = T.unflatten(spec, th)
    zero_o = dict(P)
    zero_o["Wo0"] = torch.zeros_like(P["Wo0"])        # attention drops out
    X = torch.randn(3, 5, 8, generator=torch.Generator().manual_seed(1))
    lin1 = F.linear(X, P["W1_0"].T, P["b1_0"])
    ref = F.linear(F.gelu(lin1, approximate="tanh"), P["W2_0"].T, P["b2_0"]) + X
    assert torch.allclose(T.encoder(spec, zero_o, X), ref, atol=1e-13)


def test_conv_embedding_is_circular_conv1d():
    """Two kernel-2 convolutions with circular padding over sites (channels sigma, sigma'), each + GELU."""
    spec = _spec(embed="conv", layers=1, d=8, h=2)
    th = torch.as_tensor(synth.init_params(spec, 3, std=0.5))
    P = T.unflatten(spec, th)
    a, b = synth.random_configs(6, 10, seed=4)
    b1, b2 = T.bits(a, 6), T.bits(b, 6)
    x = torch.stack([1 - 2 * b1, 1 - 2 * b2], dim=1)                      # [S, 2, N]
    w1 = P["Wc1"].permute(2, 1, 0)                                        # [C1, 2, k]
    h1 = F.gelu(F.conv1d(F.pad(x, (0, 1), mode="circular"), w1, P["bc1"]), approximate="tanh")
    w2 = P["Wc2"].permute(2, 1, 0)
    h2 = F.gelu(F.conv1d(F.pad(h1, (0, 1), mode="circular"), w2, P["bc2"]), approximate="tanh")
    assert torch.allclose(T.embed(spec, P, b1, b2), h2.transpose(1, 2), atol=1e-14)


def test_attention_free_case_by_hand():
    """Wo = 0, no MLP: X stays the embedding, z = mean_i E[token_i] Wh + bh, and log rho is the
    symmetrised log-sum-exp of the two orders."""
    spec = _spec(layers=2, d=4, h=2)
    th = synth.init_params(spec, 5, std=0.4)
    P = {k: v.numpy().copy() for k, v in T.unflatten(spec, torch.as_tensor(th)).items()}
    for l in range(2):
        P[f"Wo{l}"][:] = 0
    flat = np.concatenate([P[k].reshape(-1) for k, _ in synth.param_shapes(spec)])
    sig, sigp = 0b1011, 0b0110
    n = 4
    tA = [2 * ((sig >> i) & 1) + ((sigp >> i) & 1) for i in range(n)]
    tB = [2 * ((sigp >> i) & 1) + ((sig >> i) & 1) for i in range(n)]
    hA = np.mean([P["E"][t] for t in tA], axis=0)
    hB = np.mean([P["E"][t] for t in tB], axis=0)
    zA = complex(*(hA @ P["Wh"] + P["bh"]))
    zB = complex(*(hB @ P["Wh"] + P["bh"]))
    expect = np.log(np.exp(zA) + np.conj(np.exp(zB)))
    got = T.log_rho_np(spec, flat, np.array([sig], np.uint32), np.array([sigp], np.uint32), n)[0]
    assert abs(got - expect) < 1e-14


@pytest.mark.parametrize("embed,mlp", [("token", 0), ("token", 4), ("conv", 0)])
def test_hermiticity(embed, mlp):
    """log rho(b, a) = conj log rho(a, b) modulo 2 pi i (Eq. log_sum_exp_conjugate)."""
    spec = _spec(embed, mlp)
    th = synth.init_params(spec, 0, std=0.3)
    a, b = synth.random_configs(7, 64, seed=1)
    x = T.log_rho_np(spec, th, a, b, 7)
    y = T.log_rho_np(spec, th, b, a, 7)
    d = x - np.conj(y)
    assert np.abs(d.real).max() < 1e-13
    assert np.abs(np.angle(np.exp(1j * d.imag))).max() < 1e-13


@pytest.mark.parametrize("embed,mlp", [("token", 0), ("token", 4), ("conv", 2)])
def test_translation_invariance(embed, mlp):
    """Cyclic shift of both sigma and sigma' leaves log rho unchanged (pooling + circular conv)."""
    spec = _spec(embed, mlp)
    th = synth.init_params(spec, 0, std=0.3)
    n = 9
    a, b = synth.random_configs(n, 32, seed=2)
    rot = lambda w, s: ((w.astype(np.uint64) << np.uint64(s)) | (w.astype(np.uint64) >> np.uint64(n - s))) & np.uint64((1 << n) - 1)
    x = T.log_rho_np(spec, th, a, b, n)
    for s in (1, 4):
        y = T.log_rho_np(spec, th, rot(a, s).astype(np.uint32), rot(b, s).astype(np.uint32), n)
        d = x - y
        assert np.abs(d.real).max() < 1e-13
        assert np.abs(np.angle(np.exp(1j * d.imag))).max() < 1e-13     # phase modulo 2 pi


def test_diagonal_elements():
    """sigma = sigma': both orders coincide, rho(a,a) = 2 exp(Re z) cos(Im z) (real)."""
    spec = _spec("token", 0)
    th = synth.init_params(spec, 0, std=0.5)
    a, _ = synth.random_configs(6, 32, seed=5)
    lr = T.log_rho_np(spec, th, a, a, 6)
    P = T.unflatten(spec, torch.as_tensor(th))
    F_ = T.z_of(spec, P, T.bits(a, 6), T.bits(a, 6)).numpy()
    z = F_[:, 0] + 1j * F_[:, 1]
    assert np.allclose(np.exp(lr), 2 * np.exp(z.real) * np.cos(z.imag), atol=1e-14, rtol=1e-13)


def test_parameter_count():
    spec = synth.model_spec(64, 8, 4, 4)
    assert synth.num_params(spec) == 4 * 64 + 4 * (4 * 64 * 64 + 2 * 64 * 256 + 256 + 64) + 130
