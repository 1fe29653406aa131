"""Pins of the oracle's Philox stream and Metropolis sampler."""
import numpy as np
import pytest
from scipy import stats

from oracle import estimators as E, philox, sampler
from paper_2502_20723_gb300 import synth


@pytest.mark.parametrize("ctr,key,expect", [
    ((0, 0, 0, 0), (0, 0), (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
    ((0xffffffff,) * 4, (0xffffffff,) * 2, (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
    ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
     (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
])
def test_philox_known_answers(ctr, key, expect):
    """Known-answer vectors published with the Random123 library for Philox4x32-10."""
    out = philox.philox4x32_10(*ctr, *key)
    assert tuple(int(x) for x in out) == expect


def test_draws_are_uniform():
    k, u = sampler.draws(11, np.arange(20000, dtype=np.uint64), 5, 6)
    assert k.min() == 0 and k.max() == 11
    assert stats.chisquare(np.bincount(k, minlength=12)).pvalue > 1e-4
    assert 0 <= u.min() and u.max() < 1 and abs(u.mean() - 0.5) < 0.01


def test_metropolis_samples_rho_squared():
    """N=3 (64 doubled configurations): chain histogram vs the exact |rho|^2 / sum |rho|^2 (chi-square)."""
    n = 3
    spec = synth.model_spec(8, 2, 1, 0)
    th = synth.init_params(spec, 0, std=0.6)
    p = synth.ising_chain(n)
    a, b, w = E.full_sum_weights(p, spec, th)
    chains = 4000
    s0, s1 = synth.random_configs(n, chains, seed=1)
    s0, s1, acc, samples, _ = sampler.metropolis(spec, th, s0, s1, n, 30, seed=3, counter=0, record=True)
    idx = np.concatenate([(x.astype(np.int64) << n) | y.astype(np.int64) for x, y in samples[15:]])
    counts = np.bincount(idx, minlength=64)
    expected = w * counts.sum()
    # samples of one chain are correlated across sweeps: use the chain-end states only for the p-value
    end = np.bincount((s0.astype(np.int64) << n) | s1.astype(np.int64), minlength=64)
    assert stats.chisquare(end, w * chains).pvalue > 1e-4
    assert np.abs(counts / counts.sum() - w).max() < 0.01
    assert 0 < acc < chains * 30 * 2 * n
