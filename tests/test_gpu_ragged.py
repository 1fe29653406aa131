"""Chains of different lengths in one batch (tdo_log_rho_ragged): every configuration against the FP64 oracle
at its own chain length, and bit for bit against the same context's uniform-length forward (the ragged
launch runs the same per-tile evaluation; only the tiles' grouping and schedule differ)."""
import numpy as np
import pytest

from oracle import transformer as T
from paper_2502_20723_gb300 import synth
from tests.gpu_common import logrho_err, problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MIX = (8, 12, 16, 17, 20, 21, 24, 29, 32, 1, 5, 13)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_20723_gb300 import build
    build.build()


def dev(a, dtype=torch.int32):
    return torch.as_tensor(np.asarray(a).astype(np.int64)).to(dtype).cuda()


def ragged_batch(per_n: int, seed: int):
    rng = np.random.default_rng(seed)
    ns, ss, ps = [], [], []
    for i, n in enumerate(MIX):
        a, b = synth.random_configs(n, per_n + i, seed=seed + n)
        ns.append(np.full(len(a), n, np.int32))
        ss.append(a)
        ps.append(b)
    n_all, s_all, p_all = np.concatenate(ns), np.concatenate(ss), np.concatenate(ps)
    order = rng.permutation(len(n_all))   # interleaved lengths
    return n_all[order], s_all[order], p_all[order]


@pytest.mark.parametrize("prec,L,r", [("fp32", 2, 2), ("fp16", 2, 2), ("bf16", 2, 2), ("fp16", 4, 4)])
def test_ragged_matches_oracle_and_uniform_forward(prec, L, r):
    from paper_2502_20723_gb300 import tdo
    spec = synth.model_spec(64, 8, L, r)
    th = synth.init_params(spec, seed=31, std=0.05)
    ctx = tdo.Context(problem("ising", 16), spec, th, prec)
    n_all, s_all, p_all = ragged_batch(40, 7)
    out = ctx.log_rho_ragged(dev(n_all), dev(s_all), dev(p_all)).cpu().numpy()
    for n in MIX:
        sel = n_all == n
        ref = T.log_rho_np(spec, th, s_all[sel], p_all[sel], n)
        err = logrho_err(out[sel], ref)
        if prec == "fp32":
            assert np.all(err <= 1e-6 * np.abs(ref)), (n, err.max())
        else:
            assert err.max() <= 2e-2, (n, err.max())
        uni = tdo.Context(problem("ising", n), spec, th, prec).log_rho(dev(s_all[sel]), dev(p_all[sel])).cpu().numpy()
        assert np.array_equal(uni, out[sel]), n
    # a second call with the same mix reuses the tuned shape and gives the same bits
    mix = sum(1 << (n - 1) for n in MIX)
    if prec != "fp32":
        cps, desc, dyn = ctx.ragged_tuning(mix)
        assert cps in (1, 2) and desc in (0, 1) and dyn in (0, 1)
    again = ctx.log_rho_ragged(dev(n_all), dev(s_all), dev(p_all)).cpu().numpy()
    assert np.array_equal(again, out)


def test_ragged_rejects_lengths_outside_1_to_32():
    from paper_2502_20723_gb300 import tdo
    spec = synth.model_spec(64, 8, 1, 0)
    ctx = tdo.Context(problem("ising", 8), spec, synth.init_params(spec), "fp16")
    n = np.array([8, 33, 8], np.int32)
    s, p = synth.random_configs(8, 3, seed=1)
    with pytest.raises(tdo.TdoError, match="EUNSUPPORTED"):
        ctx.log_rho_ragged(dev(n), dev(s), dev(p))
    empty = ctx.log_rho_ragged(dev([]), dev([]), dev([]))
    assert empty.shape == (0, 2)
