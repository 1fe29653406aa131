"""Thirty optimisation steps at the headline model (N = 16 Ising chain, d = 64, 8 heads, 4 layers, MLP 4d)
with the paper's initial rate and shift (eta_0 = 0.0061, lambda_0 = 0.004): one Metropolis sweep and one
tdo_sr_step per step on 2048 chains, for an FP32 context and an FP16 tensor-core context from the same
parameters and chains.  Every step must finish (no breakdown, no non-finite value, a converged or
iteration-capped CG), the cost must fall, and the FP16 optimisation must follow the FP32 one: its cost
within 3 % of the FP32 cost at every step (a BF16 backward's rounding, amplified by 1 / lambda, made the
BF16 optimisation leave the FP32 trajectory after a few steps)."""
import numpy as np
import pytest

from paper_2502_20723_gb300 import synth
from tests.gpu_common import problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

STEPS, CHAINS, LR, SHIFT = 30, 2048, 0.0061, 0.004


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_20723_gb300 import build
    build.build()


def run(prec: str):
    from paper_2502_20723_gb300 import tdo
    n = 16
    spec = synth.model_spec(64, 8, 4, 4)
    ctx = tdo.Context(problem("ising", n), spec, synth.init_params(spec, seed=0), prec)
    s0, s1 = synth.random_configs(n, CHAINS, seed=1000)
    sig = torch.as_tensor(s0.astype(np.int64)).to(torch.int32).cuda()
    sigp = torch.as_tensor(s1.astype(np.int64)).to(torch.int32).cuda()
    ctx.sample(sig, sigp, 4, 7, 0)
    counter = 4 * 2 * n
    costs, iters = [], []
    for _ in range(STEPS):
        ctx.sample(sig, sigp, 1, 7, counter)
        counter += 2 * n
        costs.append(ctx.sr_step(sig, sigp, LR, SHIFT))
        outcome, pap, restarts = ctx.sr_report()
        assert outcome in (0, 1) and restarts == 0 and np.isfinite(pap) and pap > 0
        iters.append(ctx.sr_info()[0])
    assert np.all(np.isfinite(ctx.get_params()))
    return np.array(costs), iters


def test_thirty_sr_steps_fp16_follow_fp32():
    c32, it32 = run("fp32")
    c16, it16 = run("fp16")
    print("fp32 costs", np.round(c32, 4).tolist(), "CG iterations", it32)
    print("fp16 costs", np.round(c16, 4).tolist(), "CG iterations", it16)
    assert c32[-1] < 0.5 * c32[0] and c16[-1] < 0.5 * c16[0]
    assert np.all(np.abs(c16 - c32) <= 0.03 * c32), np.abs(c16 - c32) / c32
