"""Mixed-state observables, purity and the diagonal Metropolis chains on the GPU vs the FP64 oracle,
through the C ABI (supplement, "Mixed-State Observables").

Tolerances: FP32 contexts (log rho within 1e-6 relative): local estimators within 1e-4 (1 + |A~|), the
purity within 1e-4 relative, chain decisions identical wherever the oracle's margin |Re dlogrho - log u|
exceeds 1e-3; BF16 contexts (log rho within 2e-2 absolute, so a ratio of two values within about 4 %):
local estimators within 5e-2 (1 + |A~|), the purity within 10 % relative, the diagonal distribution within
0.03 per state."""
import numpy as np
import pytest

from oracle import observables as OB
from paper_2502_20723_gb300 import synth
from tests.gpu_common import problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_20723_gb300 import build
    build.build()


def ctx_for(prob, spec, theta, precision="fp32"):
    from paper_2502_20723_gb300 import tdo
    return tdo.Context(prob, spec, theta, precision)


def dev(a):
    return torch.as_tensor(np.asarray(a).astype(np.int64)).to(torch.int32).cuda()


def host(t):
    return t.cpu().numpy().astype(np.int64) & 0xFFFFFFFF


def test_diag_chains_replay_oracle():
    """Same Philox stream, N choices per draw: every chain whose decisions all clear 1e-3 in log space
    follows the oracle's trajectory exactly, sample by sample."""
    n = 6
    spec = synth.model_spec(16, 2, 1, 0)
    th = synth.init_params(spec, 0, std=0.5)
    a0, _ = synth.random_configs(n, 128, seed=2)
    ctx = ctx_for(problem("ising", n), spec, th)
    a = dev(a0)
    acc, ss = ctx.sample_diag(a, 5, seed=4321, counter=11, samples=True)
    oa, oacc, osamp, margin = OB.metropolis_diag(spec, th, a0, n, 5, 4321, 11, record=True)
    ok = margin > 1e-3
    assert ok.mean() > 0.9
    assert np.array_equal(host(a)[ok], oa[ok].astype(np.int64))
    for sw in range(5):
        assert np.array_equal(host(ss[sw])[ok], osamp[sw][ok].astype(np.int64))
    if ok.all():
        assert acc == oacc


@pytest.mark.parametrize("precision,d,h", [("fp32", 16, 2), ("bf16", 64, 8)])
def test_diag_chains_follow_abs_diagonal(precision, d, h):
    """Chain-end states of 8192 chains after 30 sweeps vs |rho(alpha, alpha)| / sum (N = 4)."""
    n = 4
    spec = synth.model_spec(d, h, 1, 0)
    th = synth.init_params(spec, 0, std=0.3 if d == 16 else 0.1)
    w = np.abs(np.diag(OB.density_matrix(spec, th, n)).real)
    w = w / w.sum()
    a0, _ = synth.random_configs(n, 8192, seed=5)
    ctx = ctx_for(problem("ising", n), spec, th, precision)
    a = dev(a0)
    ctx.sample_diag(a, 30, seed=7, counter=0)
    hist = np.bincount(host(a), minlength=1 << n) / 8192.0
    assert np.abs(hist - w).max() < 0.03


@pytest.mark.parametrize("precision,d,h,n,std,tol", [("fp32", 16, 2, 6, 0.5, 1e-4), ("fp32", 32, 4, 9, 0.3, 1e-4),
                                                      ("bf16", 64, 8, 16, 0.05, 5e-2), ("bf16", 64, 8, 7, 0.05, 5e-2)])
def test_magnetisation_local_matches_oracle(precision, d, h, n, std, tol):
    """Per-sample sign and local estimators (A~x, A~y, A~z) and the reweighted estimate, same samples."""
    spec = synth.model_spec(d, h, 2, 4 if precision == "bf16" else 0)
    th = synth.init_params(spec, 1, std=std)
    a0, _ = synth.random_configs(n, 300, seed=6)
    ctx = ctx_for(problem("ising", n), spec, th, precision)
    mag, sm, loc = ctx.magnetisation(dev(a0), local=True)
    s, A = OB.magnetisation_local(spec, th, a0, n)
    assert np.array_equal(loc[:, 0].real, s)
    assert (np.abs(loc[:, 1:] - A) <= tol * (1.0 + np.abs(A))).all()
    # the estimate divides by sum s: its error bound scales with the largest term and with Ns / |sum s|
    bound = tol * (1.0 + np.abs(A).max()) * len(s) / abs(s.sum())
    assert np.abs(mag - OB.magnetisation_estimate(s, A)).max() <= bound
    assert sm == pytest.approx(s.mean())


def test_magnetisation_estimate_converges_to_trace():
    """Diagonal chains + local estimator on the GPU: the estimate approaches the dense-matrix trace
    Tr(rho A) / Tr(rho) of the same model (N = 4, 16384 chains, statistical tolerance)."""
    n = 4
    spec = synth.model_spec(16, 2, 1, 0)
    th = synth.init_params(spec, 0, std=0.3)   # mean sign 0.96; statistical error <= 0.004 per component
    exact = OB.exact_magnetisation(spec, th, n)
    a0, _ = synth.random_configs(n, 16384, seed=8)
    ctx = ctx_for(problem("ising", n), spec, th)
    a = dev(a0)
    ctx.sample_diag(a, 20, seed=3, counter=0)
    mag, sm, _ = ctx.magnetisation(a)
    assert np.abs(mag - exact).max() < 0.02, (mag, exact)


@pytest.mark.parametrize("precision,d,h,n,tol", [("fp32", 16, 2, 5, 1e-4), ("bf16", 64, 8, 16, 0.1)])
def test_purity_matches_oracle(precision, d, h, n, tol):
    """Purity estimate on fixed samples vs the oracle's estimator on the same samples; the all-zero model
    (rho proportional to the all-ones matrix, a pure state) gives exactly 1."""
    spec = synth.model_spec(d, h, 1, 0)
    th = synth.init_params(spec, 2, std=0.3 if d == 16 else 0.05)
    s0, s1 = synth.random_configs(n, 400, seed=9)
    ctx = ctx_for(problem("ising", n), spec, th, precision)
    pu, se = ctx.purity(dev(s0), dev(s1))
    ref = 1.0 / OB.purity_local(spec, th, s0, s1, n).mean()
    assert abs(pu - ref) <= tol * abs(ref)
    assert se >= 0.0
    z = ctx_for(problem("ising", n), spec, np.zeros_like(th), precision)
    p1, se1 = z.purity(dev(s0), dev(s1))
    assert p1 == pytest.approx(1.0, abs=1e-6) and se1 == pytest.approx(0.0, abs=1e-6)


def test_vmc_step_is_sample_then_scheduled_sr_step():
    """tdo_vmc_step = tdo_sample (counter advanced by sweeps * 2N) + tdo_sr_step with the scheduled rate
    and shift: identical chains and cost, and parameters equal to the rounding of the gradient's float
    atomics (within 1e-5); each step starts both contexts from the same parameters."""
    from paper_2502_20723_gb300 import tdo
    n = 4
    spec = synth.model_spec(16, 2, 1, 0)
    th = synth.init_params(spec, 0, std=0.2)
    s0, s1 = synth.random_configs(n, 256, seed=1)
    sched = tdo.Schedule(eta0=0.01, i_switch=2, i_decay=10, alpha=0.001, lambda0=0.05, i_switch_sr=1, i_decay_sr=8,
                         alpha_sr=0.01)
    a = ctx_for(problem("ising", n), spec, th)
    b = ctx_for(problem("ising", n), spec, th)
    sa, pa, sb, pb = dev(s0), dev(s1), dev(s0), dev(s1)
    ctr = 5
    for k, step in enumerate((0, 6)):   # before the switch, and on the cosine part of both schedules
        cost_a, ctr_new = a.vmc_step(sa, pa, 2, 99, ctr, step, sched)
        b.sample(sb, pb, 2, 99, ctr)
        cost_b = b.sr_step(sb, pb, tdo.schedule_value(step, 0.01, 2, 10, 0.001),
                           tdo.schedule_value(step, 0.05, 1, 8, 0.01))
        assert ctr_new == ctr + 2 * 2 * n
        ctr = ctr_new
        assert np.array_equal(host(sa), host(sb)) and np.array_equal(host(pa), host(pb))
        assert cost_a == pytest.approx(cost_b, rel=1e-12)
        pa_, pb_ = a.get_params(), b.get_params()
        assert np.abs(pa_ - pb_).max() <= 1e-5 * max(1.0, np.abs(pb_).max())
        # the next step from one shared state (set_params also drops both warm starts)
        a.set_params(pa_)
        b.set_params(pa_)
