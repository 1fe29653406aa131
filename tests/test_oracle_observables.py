"""Pins of the oracle's mixed-state observables, purity and diagonal Metropolis chains (supplement,
"Mixed-State Observables").  The local estimators are checked against dense-matrix traces of the same
model, against the closed form of the all-zero-parameter model, and the chains against the exact
diagonal distribution."""
import numpy as np
import pytest
from scipy import stats

from oracle import estimators as E, observables as OB
from paper_2502_20723_gb300 import synth


def _model(n, std, seed=0, d=8, h=2):
    spec = synth.model_spec(d, h, 1, 0)
    return spec, synth.init_params(spec, seed, std=std)


def test_diag_draws_uniform():
    k, u = OB.draws_diag(5, np.arange(30000, dtype=np.uint64), 3, 7)
    assert k.min() == 0 and k.max() == 6
    assert stats.chisquare(np.bincount(k, minlength=7)).pvalue > 1e-4
    assert 0 <= u.min() and u.max() < 1 and abs(u.mean() - 0.5) < 0.01


def test_zero_parameters_closed_form():
    """theta = 0: z = 0 for every pair, so rho is proportional to the all-ones matrix, the pure state
    |+><+| (up to normalisation): <sigma^x> = 1, <sigma^y> = <sigma^z> = 0, purity 1, and every local
    x estimator is exactly 1."""
    n = 4
    spec = synth.model_spec(8, 2, 1, 0)
    th = np.zeros(synth.num_params(spec))
    assert np.allclose(OB.exact_magnetisation(spec, th, n), [1.0, 0.0, 0.0], atol=1e-12)
    assert OB.exact_purity(spec, th, n) == pytest.approx(1.0, abs=1e-12)
    a = np.arange(16, dtype=np.uint32)
    s, A = OB.magnetisation_local(spec, th, a, n)
    assert np.all(s == 1.0)
    assert np.allclose(A[:, 0], 1.0, atol=1e-12)
    bits = (a[:, None] >> np.arange(n)) & 1
    assert np.allclose(A[:, 2], (1 - 2 * bits).mean(axis=1), atol=1e-12)
    assert np.allclose(A[:, 1], 1j * (1 - 2 * bits).mean(axis=1), atol=1e-12)
    s0, s1 = synth.random_configs(n, 50, seed=3)
    assert np.allclose(OB.purity_local(spec, th, s0, s1, n), 1.0, atol=1e-12)


@pytest.mark.parametrize("n,std,seed", [(3, 0.6, 0), (4, 0.8, 2)])
def test_estimator_expectation_equals_trace(n, std, seed):
    """Sum over every alpha of |rho(alpha, alpha)|-weighted s A~ / s: exactly Tr(rho A) / Tr(rho) from the
    dense matrix (a dropped ratio, a wrong sigma^y phase or a missing sign reweighting breaks it)."""
    spec, th = _model(n, std, seed)
    rho = OB.density_matrix(spec, th, n)
    a = np.arange(1 << n, dtype=np.uint32)
    s, A = OB.magnetisation_local(spec, th, a, n)
    w = np.abs(np.diag(rho).real)
    got = (w[:, None] * s[:, None] * A).sum(axis=0).real / np.sum(w * s)
    assert np.allclose(got, OB.exact_magnetisation(spec, th, n), atol=1e-10)


def test_sign_reweighting_is_exercised():
    """The model of the test above at N = 4 has diagonal entries of both signs, so the reweighting is
    what makes the estimator exact there."""
    spec, th = _model(4, 0.8, 2)
    d = np.diag(OB.density_matrix(spec, th, 4)).real
    assert (d < 0).any() and (d > 0).any()


@pytest.mark.parametrize("n,std", [(3, 0.6), (4, 0.5)])
def test_purity_estimator_expectation(n, std):
    """|rho|^2-weighted mean of the purity estimator = Tr(rho)^2 / Tr(rho^2) from the dense matrix."""
    spec, th = _model(n, std)
    prob = synth.ising_chain(n)
    a, b, w = E.full_sum_weights(prob, spec, th)
    f = OB.purity_local(spec, th, a, b, n)
    assert np.sum(w * f) == pytest.approx(1.0 / OB.exact_purity(spec, th, n), rel=1e-10)


def test_diag_chains_sample_abs_diagonal():
    """Chain-end states of many chains follow |rho(alpha, alpha)| / sum |rho(alpha, alpha)| (chi-square)."""
    n = 3
    spec, th = _model(n, 0.6)
    w = np.abs(np.diag(OB.density_matrix(spec, th, n)).real)
    w = w / w.sum()
    chains = 4000
    a0, _ = synth.random_configs(n, chains, seed=4)
    a, acc, samples, _ = OB.metropolis_diag(spec, th, a0, n, 25, seed=9, counter=5, record=True)
    end = np.bincount(a.astype(np.int64), minlength=1 << n)
    assert stats.chisquare(end, w * chains).pvalue > 1e-4
    allc = np.bincount(np.concatenate(samples[10:]).astype(np.int64), minlength=1 << n)
    assert np.abs(allc / allc.sum() - w).max() < 0.01
    assert 0 < acc < chains * 25 * n
