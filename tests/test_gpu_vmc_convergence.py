"""Variational steady state on the GPU path vs exact diagonalisation (results section: VMC reaches the
exact steady-state magnetisations of small dissipative chains).

The dissipative transverse-field Ising chain (V=2, g=1, gamma=1, PBC) is trained with Metropolis samples
from tdo_sample and stochastic-reconfiguration updates from tdo_sr_step, with the paper's circular-conv
embedding.  The magnetisations <sigma^a> = Tr(rho A)/Tr(rho), A = (1/N) sum_i sigma^a_i, are then formed
exactly from the model: the trace needs rho on the 2^N diagonal configurations and on the N 2^N
configurations one flip away, evaluated by tdo_log_rho.  The exact values come from the oracle's
dense steady state (tests/golden/ed_observables.json, written by tests/golden/make_golden.py).

Persistent chains need several sweeps per step: with one sweep (2N proposals) the samples lag the
parameters they are used with, and the run stalls near an error of 0.011 whatever the sample count;
four sweeps reach 0.003 in 600 steps at N = 4.

The token embedding cannot pass this test: with no positional information the transformer is
invariant under every permutation of the sites, and the steady state of the chain is only translation
invariant (a VMC run with it stalls near an error of 0.06 in <sigma^y>)."""
import json
import os

import numpy as np
import pytest

from paper_2502_20723_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "ed_observables.json")))


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_20723_gb300 import build
    build.build()


def magnetisations(ctx, n):
    """Exact <sigma^{x,y,z}> of the (unnormalised) model density matrix, rho[a, b] = rho(sigma=a, sigma'=b)."""
    dim = 1 << n
    a = np.arange(dim, dtype=np.int64)
    bit = lambda v, i: (v >> i) & 1
    rows_s, rows_p = [a], [a]
    for i in range(n):
        rows_s.append(a)
        rows_p.append(a ^ (1 << i))
    s = np.concatenate(rows_s).astype(np.uint32)
    p = np.concatenate(rows_p).astype(np.uint32)
    lr = ctx.log_rho(s, p).astype(np.float64)
    z = lr[:, 0] + 1j * lr[:, 1]
    rho = np.exp(z - z.real.max())
    diag = rho[:dim]
    tr = diag.sum()
    sz = sum(np.sum(diag * (1 - 2 * bit(a, i))) for i in range(n)) / n
    # Tr(rho A) = sum_{a,b} rho[a,b] <b|A|a>; for A = X_i or Y_i only b = a ^ e_i contributes:
    # <b|X|a> = 1, <b|Y|a> = i (-1)^{a_i}  (bit 0 = |0> = sigma^z +1)
    sx = sy = 0
    for i in range(n):
        off = rho[dim * (i + 1):dim * (i + 2)]
        sx += np.sum(off)
        sy += np.sum(off * 1j * (1 - 2 * bit(a, i)))
    return {"sx": (sx / tr).real / n, "sy": (sy / tr).real / n, "sz": (sz / tr).real}


def train(n, spec, steps, chains, lr, shift, sweeps, seed=0):
    from paper_2502_20723_gb300 import tdo
    prob = synth.ising_chain(n, V=2.0, g=1.0, gamma=1.0)
    ctx = tdo.Context(prob, spec, synth.init_params(spec, seed), "fp32")
    s0, s1 = synth.random_configs(n, chains, seed=seed + 1)
    sig = torch.as_tensor(s0.astype(np.int64)).to(torch.int32).cuda()
    sigp = torch.as_tensor(s1.astype(np.int64)).to(torch.int32).cuda()
    ctr = 0
    ctx.sample(sig, sigp, 10, 7, ctr)
    ctr += 10 * 2 * n
    for _ in range(steps):
        ctx.sample(sig, sigp, sweeps, 7, ctr)
        ctr += sweeps * 2 * n
        ctx.sr_step(sig, sigp, lr, shift)
    return ctx


@pytest.mark.parametrize("n,d,h,L,c1,steps,chains,lr,shift,sweeps", [
    (4, 16, 2, 1, 8, 600, 8192, 0.03, 1e-3, 4),
    (8, 16, 2, 1, 8, 1500, 8192, 0.03, 1e-2, 4),   # at N = 8 a shift of 1e-3 diverges
])
def test_vmc_reaches_exact_magnetisations(n, d, h, L, c1, steps, chains, lr, shift, sweeps):
    spec = synth.model_spec(d, h, L, 0, embed="conv", conv_channels=c1)
    ctx = train(n, spec, steps, chains, lr, shift, sweeps)
    got = magnetisations(ctx, n)
    ref = GOLD[f"ising_n{n}_V2_g1"]
    err = {k: abs(got[k] - ref[k]) for k in ("sx", "sy", "sz")}
    print(f"N={n}: " + " ".join(f"{k} {got[k]:+.4f} (exact {ref[k]:+.4f})" for k in err))
    assert max(err.values()) <= 1e-2, err
