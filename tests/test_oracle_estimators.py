"""Pins of the oracle's cost, local estimator, gradient, log-derivatives and SR solve."""
import numpy as np
import pytest
import torch

from oracle import estimators as E, lindblad, transformer as T
from paper_2502_20723_gb300 import synth


def _setup(n=4, d=16, h=2, layers=1, mlp=0, std=0.2, seed=0, kind="ising"):
    p = synth.ising_chain(n, g=1.0) if kind == "ising" else synth.xyz_chain(n, Jx=0.9)
    spec = synth.model_spec(d, h, layers, mlp)
    th = synth.init_params(spec, seed, std=std)
    return p, spec, th


def test_cost_zero_at_steady_state_and_positive_elsewhere():
    """Cost >= 0 and = 0 iff Lhat rho = 0 (loss section)."""
    p = synth.ising_chain(4)
    rho = lindblad.steady_state_dense(p)
    assert E.cost_of_vector(p, rho.reshape(-1)) < 1e-24
    rng = np.random.default_rng(0)
    v = rng.standard_normal(256) + 1j * rng.standard_normal(256)
    assert E.cost_of_vector(p, v) > 1e-2
    assert abs(E.cost_of_vector(p, 3.7j * v) - E.cost_of_vector(p, v)) < 1e-12   # scale invariant


def test_cost_equals_expectation_of_squared_lindbladian():
    """||Lhat rho||^2/||rho||^2 == <<rho| Lhat^+ Lhat |rho>> / <<rho|rho>> with the explicit Hermitian operator."""
    p = synth.xyz_chain(3, Jx=0.6, Bz=0.4)
    L = lindblad.lindbladian_dense(p)
    frakL = L.conj().T @ L
    assert np.abs(frakL - frakL.conj().T).max() < 1e-12
    assert np.linalg.eigvalsh(frakL).min() > -1e-10
    rng = np.random.default_rng(1)
    v = rng.standard_normal(64) + 1j * rng.standard_normal(64)
    assert abs((v.conj() @ frakL @ v).real / (v.conj() @ v).real - E.cost_of_vector(p, v)) < 1e-12


def test_local_estimator_vanishes_at_exact_steady_state():
    """At rho = rho_ss, L_loc(x) = (Lhat rho)_x / rho_x = 0 for every x (zero-variance property)."""
    p = synth.ising_chain(4, g=1.5)
    rho = lindblad.steady_state_dense(p)
    fn = lambda a, b: np.log(rho[a.astype(np.int64), b.astype(np.int64)].astype(np.complex128))
    a, b = synth.all_configs(4)
    keep = np.abs(rho[a.astype(np.int64), b.astype(np.int64)]) > 1e-8
    ll = E.local_estimator_fn(p, fn, a[keep], b[keep])
    assert np.abs(ll).max() < 1e-9


@pytest.mark.parametrize("kind", ["ising", "xyz"])
def test_weighted_local_estimator_is_full_sum_cost(kind):
    """sum_x P(x) |L_loc(x)|^2 over all 4^N configurations == Eq. lossnetk with the dense Lhat."""
    p, spec, th = _setup(kind=kind)
    a, b, w = E.full_sum_weights(p, spec, th)
    ll = E.local_estimator(p, spec, th, a, b)
    assert abs(E.cost_mc(ll, w)[0] - E.full_sum_cost(p, spec, th)) < 1e-12 * max(1, E.full_sum_cost(p, spec, th))


def test_full_sum_gradient_autograd_vs_finite_differences():
    """Autograd of the full-sum cost == central finite differences (h = 1e-6, FP64)."""
    p, spec, th = _setup(std=0.3)
    t = torch.as_tensor(th).clone().requires_grad_(True)
    (g,) = torch.autograd.grad(E.full_sum_cost(p, spec, t, torch_out=True), t)
    rng = np.random.default_rng(0)
    h = 1e-6
    for k in rng.choice(len(th), 12, replace=False):
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (E.full_sum_cost(p, spec, tp) - E.full_sum_cost(p, spec, tm)) / (2 * h)
        assert abs(fd - g[k].item()) < 1e-6 * max(1.0, abs(fd))


@pytest.mark.parametrize("kind", ["ising", "xyz"])
def test_gradient_estimator_with_exact_weights_is_exact_gradient(kind):
    """The local-estimator gradient formula, weighted by the exact P(x) over all configurations,
    equals d(full-sum cost)/d theta: pins the cotangents, the -Cost O(x) term and the factor 2."""
    p, spec, th = _setup(kind=kind, std=0.3)
    t = torch.as_tensor(th).clone().requires_grad_(True)
    (gx,) = torch.autograd.grad(E.full_sum_cost(p, spec, t, torch_out=True), t)
    a, b, w = E.full_sum_weights(p, spec, th)
    g, cost, _, _ = E.grad_estimator(p, spec, th, a, b, weights=w)
    assert abs(cost - E.full_sum_cost(p, spec, th)) < 1e-12 * max(1, cost)
    assert np.abs(g - gx.numpy()).max() < 1e-10 * max(1, np.abs(g).max())


def test_jacobian_vs_finite_differences():
    """O_k = d log rho / d theta_k (complex) == central differences of the forward."""
    p, spec, th = _setup(n=5, d=8, h=2, layers=2, mlp=2, std=0.3)
    a, b = synth.random_configs(5, 6, seed=3)
    O = E.jacobian(spec, th, a, b, 5)
    h = 1e-6
    rng = np.random.default_rng(1)
    for k in rng.choice(len(th), 10, replace=False):
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        d = T.log_rho_np(spec, tp, a, b, 5) - T.log_rho_np(spec, tm, a, b, 5)
        d = d.real + 1j * np.angle(np.exp(1j * d.imag))
        assert np.abs(d / (2 * h) - O[:, k]).max() < 1e-6


def test_mc_estimates_converge_to_full_sum():
    """Samples drawn exactly from P(x): the Monte Carlo cost lies within 5 standard errors of Eq. lossnetk."""
    p, spec, th = _setup(std=0.3)
    a, b, w = E.full_sum_weights(p, spec, th)
    rng = np.random.default_rng(7)
    idx = rng.choice(len(w), size=4000, p=w)
    ll = E.local_estimator(p, spec, th, a[idx], b[idx])
    c, se = E.cost_mc(ll)
    assert abs(c - E.full_sum_cost(p, spec, th)) < 5 * se


def test_sr_constant_O_gives_scaled_gradient():
    """If O is the same for every sample, S = 0 and delta = grad / lambda."""
    rng = np.random.default_rng(0)
    row = rng.standard_normal(7) + 1j * rng.standard_normal(7)
    O = np.tile(row, (11, 1))
    g = rng.standard_normal(7)
    assert np.abs(E.sr_solve(O, g, 0.01) - g / 0.01).max() < 1e-9


def test_sr_matrix_brute_force_and_solve_residual():
    """Re S by the double sum of the metric-tensor section, and ||(S + lambda I) delta - grad|| ~ 0."""
    rng = np.random.default_rng(2)
    O = rng.standard_normal((9, 5)) + 1j * rng.standard_normal((9, 5))
    S = np.zeros((5, 5))
    for i in range(5):
        for j in range(5):
            a = np.mean(np.conj(O[:, i]) * O[:, j])
            b = np.mean(np.conj(O[:, i])) * np.mean(O[:, j])
            S[i, j] = (a - b).real
    assert np.abs(S - E.sr_matrix(O)).max() < 1e-13
    g = rng.standard_normal(5)
    d = E.sr_solve(O, g, 1e-3)
    assert np.linalg.norm((S + 1e-3 * np.eye(5)) @ d - g) < 1e-10 * np.linalg.norm(g) / 1e-3


def test_sr_product_is_the_brute_force_matrix_times_v():
    """The matrix-free product against the double-sum S of the metric-tensor section times v, with a
    mean far from zero (the centring must cancel it) and a shift."""
    rng = np.random.default_rng(4)
    O = 3.0 + rng.standard_normal((13, 6)) + 1j * (rng.standard_normal((13, 6)) - 2.0)
    S = np.zeros((6, 6))
    for i in range(6):
        for j in range(6):
            S[i, j] = (np.mean(np.conj(O[:, i]) * O[:, j]) - np.mean(np.conj(O[:, i])) * np.mean(O[:, j])).real
    v = rng.standard_normal(6)
    assert np.abs(E.sr_product(O, v, 0.25) - (S @ v + 0.25 * v)).max() < 1e-12


def test_connections_structure_ising():
    """Ising row: diagonal + N sigma flips + N sigma' flips + one jump per site with both bits = 1."""
    p = synth.ising_chain(6, g=1.0)
    a, b = synth.random_configs(6, 20, seed=9)
    rows = E.connections(p, a, b)
    for s, r in zip(zip(a, b), rows):
        assert r[0][0] == (int(s[0]), int(s[1]))
        both = bin(int(s[0]) & int(s[1])).count("1")
        assert len(r) == 1 + 12 + both


def test_lr_schedule():
    assert E.lr_schedule(0) == 0.0061
    assert abs(E.lr_schedule(30000) - 0.0061 * (1 + 0.001)) < 1e-15
    assert abs(E.lr_schedule(70000) - 0.0061 * 0.001) < 1e-15


def test_adam_step_matches_torch_and_first_step_closed_form():
    """The oracle's Adam (Kingma and Ba, Algorithm 1) against torch.optim.Adam fed the same directions, and
    its first step: m_hat = delta, v_hat = delta^2, so theta moves by lr delta / (|delta| + eps)."""
    import torch
    rng = np.random.default_rng(4)
    th0 = rng.standard_normal(7)
    deltas = [rng.standard_normal(7) * s for s in (1.0, 0.1, 3.0, 1e-4)]
    lr, b1, b2, eps = 0.02, 0.85, 0.995, 1e-6
    th, m, v = th0.copy(), np.zeros(7), np.zeros(7)
    p = torch.nn.Parameter(torch.as_tensor(th0.copy()))
    opt = torch.optim.Adam([p], lr=lr, betas=(b1, b2), eps=eps)
    for t, d in enumerate(deltas, start=1):
        th, m, v = E.adam_step(th, d, m, v, t, lr, b1, b2, eps)
        opt.zero_grad()
        p.grad = torch.as_tensor(d)
        opt.step()
        assert np.abs(th - p.detach().numpy()).max() < 1e-13
    th1, _, _ = E.adam_step(th0, deltas[0], np.zeros(7), np.zeros(7), 1, lr, b1, b2, eps)
    assert np.allclose(th0 - th1, lr * deltas[0] / (np.abs(deltas[0]) + eps), rtol=0, atol=1e-15)
