"""Cost, local estimator, gradient, log-derivatives and stochastic reconfiguration (oracle; test infrastructure only).

Cost (Eq. lossnetk): Cost = ||Lhat rho||^2 / ||rho||^2.
Local estimator (optimisation-procedure section): L_loc(x) = sum_y Lhat_{xy} rho(y) / rho(x).
With P(x) = |rho(x)|^2 / sum |rho|^2, Cost = E_P |L_loc|^2, and for real parameters
  dCost/dtheta_k = 2 Re E_P[ conj(L_loc(x)) sum_y Lhat_{xy} (rho_y/rho_x) O_k(y) - Cost O_k(x) ],
  O_k = d log rho / d theta_k.
The paper prints this gradient in a garbled form (no centring, ambiguous conjugation); the form above is
the derivative of Eq. lossnetk itself, and test_oracle_estimators pins it against autograd and finite
differences of the full-sum cost.
SR (metric-tensor and regularisation sections): S_ij = <dO_i^* dO_j> - <dO_i^*><dO_j>, real part for real
parameters, S' = S + lambda I, delta = S'^{-1} grad, theta <- theta - eta delta.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import torch

from . import lindblad
from .transformer import log_rho, log_rho_np, log_rho_parts, DT
from paper_2502_20723_gb300.synth import all_configs


def connections(problem: dict, sig, sigp, drop_zero: bool = True):
    """Per sample: list of ((eta, eta'), Lhat element); the diagonal (x itself) always first."""
    rows = []
    for a, b in zip(np.asarray(sig).tolist(), np.asarray(sigp).tolist()):
        r = lindblad.lindbladian_row(problem, int(a), int(b))
        diag = ((a, b), r.pop((a, b), 0j))
        rest = [(k, v) for k, v in r.items() if (not drop_zero) or abs(v) > 0]
        rest.sort(key=lambda kv: (kv[0][0], kv[0][1]))
        rows.append([diag] + rest)
    return rows


def full_sum_cost(problem: dict, spec: dict, theta, torch_out: bool = False):
    """Cost by summation over all 4^N doubled configurations with the dense Lindbladian (N <= 6)."""
    n = problem["n_sites"]
    sig, sigp = all_configs(n)
    lr = log_rho(spec, theta, sig, sigp, n)
    lr = lr - lr.real.max().detach()
    rho = torch.exp(lr)
    Lh = torch.as_tensor(lindblad.lindbladian_dense(problem))
    Lrho = Lh @ rho
    cost = (Lrho.abs() ** 2).sum() / (rho.abs() ** 2).sum()
    return cost if torch_out else float(cost.detach())


def full_sum_weights(problem: dict, spec: dict, theta):
    """Exact P(x) = |rho_x|^2 / sum |rho|^2 over all doubled configurations."""
    n = problem["n_sites"]
    sig, sigp = all_configs(n)
    lr = log_rho_np(spec, theta, sig, sigp, n)
    w = np.exp(2 * (lr.real - lr.real.max()))
    return sig, sigp, w / w.sum()


def local_estimator_fn(problem: dict, logrho_fn, sig, sigp, rows=None):
    """L_loc for each given configuration, by the row sum over connected configurations (FP64);
    logrho_fn(sig, sigp) -> complex log rho of any ansatz (or of an exact state)."""
    if rows is None:
        rows = connections(problem, sig, sigp)
    ys = np.array([[k[0], k[1]] for r in rows for k, _ in r], dtype=np.uint32).reshape(-1, 2)
    lr = logrho_fn(ys[:, 0], ys[:, 1])
    out, off = np.zeros(len(rows), np.complex128), 0
    for s, r in enumerate(rows):
        lx = lr[off]
        for j, (_, v) in enumerate(r):
            out[s] += v * np.exp(lr[off + j] - lx)
        off += len(r)
    return out


def local_estimator(problem: dict, spec: dict, theta, sig, sigp, rows=None):
    """L_loc of the transformer ansatz with parameters theta."""
    n = problem["n_sites"]
    return local_estimator_fn(problem, lambda a, b: log_rho_np(spec, theta, a, b, n), sig, sigp, rows)


def cost_of_vector(problem: dict, rho_vec):
    """Eq. lossnetk for an explicit vectorised rho (length 4^N, index sigma*2^N + sigma'), dense Lhat."""
    Lh = lindblad.lindbladian_dense(problem)
    v = np.asarray(rho_vec)
    return float(np.linalg.norm(Lh @ v) ** 2 / np.linalg.norm(v) ** 2)


def cost_mc(lloc: np.ndarray, weights=None):
    """Cost estimate E|L_loc|^2 and its standard error (uniform weights = Monte Carlo average)."""
    a = np.abs(lloc) ** 2
    if weights is None:
        return float(a.mean()), float(a.std(ddof=0) / np.sqrt(len(a)))
    return float((weights * a).sum()), 0.0


def grad_estimator(problem: dict, spec: dict, theta, sig, sigp, weights=None, rows=None):
    """dCost/dtheta from samples (weights None: uniform 1/N_s) or exact weights P(x).
    Uses the surrogate sum_rows Re(c_row * log rho_row) with constant cotangents
    c = w_x conj(L_loc(x)) Lhat_xy rho_y/rho_x (and -w_x Cost on the row y = x), times 2."""
    n = problem["n_sites"]
    if rows is None:
        rows = connections(problem, sig, sigp)
    lloc = local_estimator(problem, spec, theta, sig, sigp, rows)
    ns = len(rows)
    w = np.full(ns, 1.0 / ns) if weights is None else np.asarray(weights)
    cost = float((w * np.abs(lloc) ** 2).sum())
    ys = np.array([[k[0], k[1]] for r in rows for k, _ in r], dtype=np.uint32).reshape(-1, 2)
    th = torch.as_tensor(np.asarray(theta, np.float64), dtype=DT).clone().requires_grad_(True)
    lr = log_rho(spec, th, ys[:, 0], ys[:, 1], n)
    lrn = lr.detach().numpy()
    cot = np.zeros(len(ys), np.complex128)
    off = 0
    for s, r in enumerate(rows):
        lx = lrn[off]
        for j, (_, v) in enumerate(r):
            cot[off + j] = w[s] * np.conj(lloc[s]) * v * np.exp(lrn[off + j] - lx)
        cot[off] -= w[s] * cost
        off += len(r)
    c = torch.as_tensor(cot)
    surrogate = 2.0 * (c.real * lr.real - c.imag * lr.imag).sum()
    (g,) = torch.autograd.grad(surrogate, th)
    return g.numpy(), cost, lloc, cot


def jacobian(spec: dict, theta, sig, sigp, n_sites: int, chunk: int = 256) -> np.ndarray:
    """O[s, k] = d log rho(x_s) / d theta_k, complex, via reverse-mode autodiff in FP64."""
    th = torch.as_tensor(np.asarray(theta, np.float64), dtype=DT)
    out = []
    sig = np.asarray(sig)
    sigp = np.asarray(sigp)
    for a in range(0, len(sig), chunk):
        def f(t):
            return torch.stack(log_rho_parts(spec, t, sig[a:a + chunk], sigp[a:a + chunk], n_sites), dim=0)
        J = torch.func.jacrev(f)(th)              # [2, b, P]
        out.append((J[0] + 1j * J[1]).numpy())
    return np.concatenate(out, axis=0)


def sr_matrix(O: np.ndarray) -> np.ndarray:
    """Re S with S_ij = <O_i^* O_j> - <O_i^*><O_j> over the samples (rows of O)."""
    Oc = O - O.mean(axis=0, keepdims=True)
    return (Oc.conj().T @ Oc).real / O.shape[0]


def sr_product(O: np.ndarray, v: np.ndarray, diag_shift: float) -> np.ndarray:
    """(Re S + lambda I) v without forming S: (1/Ns) Re[Oc^H (Oc v)] + lambda v, Oc = O - mean(O) (the
    metric-tensor section's S applied to a vector; v real)."""
    Oc = O - O.mean(axis=0, keepdims=True)
    return (Oc.conj().T @ (Oc @ v)).real / O.shape[0] + diag_shift * v


def sr_solve(O: np.ndarray, grad: np.ndarray, diag_shift: float) -> np.ndarray:
    """delta = (Re S + lambda I)^{-1} grad by Cholesky (S' symmetric positive definite)."""
    S = sr_matrix(O) + diag_shift * np.eye(O.shape[1])
    c = sla.cho_factor(S, lower=True)
    return sla.cho_solve(c, grad)


def sr_step(problem: dict, spec: dict, theta, sig, sigp, lr_eta: float, diag_shift: float):
    """One optimisation-workflow step on a given sample set: cost, gradient, S, shift, solve, update."""
    n = problem["n_sites"]
    g, cost, lloc, _ = grad_estimator(problem, spec, theta, sig, sigp)
    O = jacobian(spec, theta, sig, sigp, n)
    delta = sr_solve(O, g, diag_shift)
    return np.asarray(theta) - lr_eta * delta, cost, g, delta


def adam_step(theta, delta, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam step (Kingma and Ba 2014, Algorithm 1) with the SR direction delta as the gradient, as the
    optimisation-procedure section combines Adam with stochastic reconfiguration; t = this step's number
    (1 for the first).  Returns (theta, m, v)."""
    m = b1 * np.asarray(m) + (1.0 - b1) * np.asarray(delta)
    v = b2 * np.asarray(v) + (1.0 - b2) * np.asarray(delta) ** 2
    m_hat = m / (1.0 - b1 ** t)
    v_hat = v / (1.0 - b2 ** t)
    return np.asarray(theta) - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def lr_schedule(i: int, eta0: float = 0.0061, i_switch: int = 30000, i_decay: int = 40000, alpha: float = 0.001):
    """Learning-rate schedule of the scheduling section: constant, then cosine decay plus a floor."""
    if i < i_switch:
        return eta0
    return eta0 * (1 + np.cos(np.pi * (i - i_switch) / i_decay)) / 2 + alpha * eta0
