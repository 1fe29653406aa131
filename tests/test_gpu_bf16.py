"""Tensor-core path (tcgen05; BF16 contexts, and FP16 contexts where named) vs the FP64 oracle, through the C ABI.

Tolerances: log rho within 2e-2 absolute (phase modulo 2 pi), cost within 1e-3 relative on the same
samples, Metropolis decisions identical wherever the oracle's margin |2 Re dlogrho - log u| exceeds
twice the log rho tolerance."""
import numpy as np
import pytest

from oracle import estimators as E, sampler as OS, transformer as T
from paper_2502_20723_gb300 import synth
from tests.gpu_common import block_errors, logrho_err, problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_20723_gb300 import build
    build.build()


def ctx_for(prob, spec, theta):
    from paper_2502_20723_gb300 import tdo
    return tdo.Context(prob, spec, theta, "bf16")


def dev(a):
    return torch.as_tensor(np.asarray(a).astype(np.int64)).to(torch.int32).cuda()


@pytest.mark.parametrize("n,d,h,L,r,B,std", [
    (16, 64, 8, 4, 4, 2000, 0.02),    # headline shape, default init
    (16, 64, 8, 4, 4, 301, 0.05),
    (8, 32, 4, 2, 0, 777, 0.1),       # N=8 / XYZ workload shapes (no MLP)
    (8, 32, 4, 2, 4, 129, 0.1),
    (13, 64, 8, 2, 2, 97, 0.05),      # ragged tile (9 sequences of 13 tokens)
    (32, 64, 8, 1, 4, 33, 0.05),
    (1, 64, 8, 2, 0, 5, 0.05),
])
def test_log_rho_bf16(n, d, h, L, r, B, std):
    spec = synth.model_spec(d, h, L, r)
    th = synth.init_params(spec, seed=5 + n, std=std)
    sig, sigp = synth.random_configs(n, B, seed=B)
    ref = T.log_rho_np(spec, th, sig, sigp, n)
    out = ctx_for(problem("ising", n), spec, th).log_rho(dev(sig), dev(sigp)).cpu().numpy()
    err = logrho_err(out, ref)
    assert err.max() <= 2e-2, err.max()


@pytest.mark.parametrize("kind,n,d,h,L,r,Ns", [("ising", 16, 64, 8, 4, 4, 512), ("xyz", 8, 32, 4, 2, 0, 1024)])
def test_cost_bf16(kind, n, d, h, L, r, Ns):
    prob = problem(kind, n)
    spec = synth.model_spec(d, h, L, r)
    th = synth.init_params(spec, seed=3, std=0.02 if d == 64 else 0.1)
    sig, sigp = synth.random_configs(n, Ns, seed=7)
    _, cost, _ = ctx_for(prob, spec, th).local_estimator(dev(sig), dev(sigp))
    ref = E.local_estimator(prob, spec, th, sig, sigp)
    c_ref, _ = E.cost_mc(ref)
    assert abs(cost - c_ref) <= 1e-3 * c_ref, (cost, c_ref)


def test_metropolis_bf16_replays_decided_chains():
    """One sweep (12 proposals) per chain; a chain counts as decided when every one of its proposals has
    an oracle margin above 4e-2 (about 60% of chains for uniform u)."""
    n = 6
    spec = synth.model_spec(32, 4, 1, 0)
    th = synth.init_params(spec, 0, std=0.3)
    s0, s1 = synth.random_configs(n, 1024, seed=3)
    a, b = dev(s0), dev(s1)
    ctx_for(problem("ising", n), spec, th).sample(a, b, 1, seed=99, counter=5)
    o0, o1, _, _, margin = OS.metropolis(spec, th, s0, s1, n, 1, 99, 5)
    ok = margin > 4e-2
    assert ok.sum() >= 300, ok.sum()
    g0 = a.cpu().numpy().astype(np.int64) & 0xFFFFFFFF
    g1 = b.cpu().numpy().astype(np.int64) & 0xFFFFFFFF
    assert np.array_equal(g0[ok], o0[ok].astype(np.int64))
    assert np.array_equal(g1[ok], o1[ok].astype(np.int64))


def test_bf16_unsupported_shapes():
    from paper_2502_20723_gb300 import tdo
    spec = synth.model_spec(16, 2, 1, 0)
    with pytest.raises(tdo.TdoError, match="EUNSUPPORTED"):
        ctx_for(problem("ising", 4), spec, synth.init_params(spec))


# Bounds per named parameter block (max |g - ref| / max |ref| over the block) and in norm, about three times
# the errors measured on GB300: FP16 operands at most 1.3e-2 (weights) and 1.7e-2 (biases), 5.3e-4 in norm;
# BF16 operands 1.9e-2 (weights) and 0.16 (the hidden bias b1, a 16-bit ones-MMA sum over every row),
# 3.6e-3 in norm.  Chains of 17 to 32 sites take the 32-token attention unit of attention pass 1.
GRAD_BOUNDS = {"fp16": (4e-2, 5e-2, 2e-3), "bf16": (5e-2, 0.5, 1e-2)}


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("kind,n,h,L,r,Ns", [("ising", 16, 8, 4, 4, 96), ("xyz", 13, 4, 2, 2, 64), ("ising", 8, 8, 2, 0, 128),
                                              ("ising", 20, 8, 1, 2, 24), ("xyz", 5, 4, 1, 4, 40),
                                              ("xyz", 24, 8, 2, 4, 48), ("ising", 32, 8, 1, 4, 64),
                                              ("xyz", 17, 4, 1, 0, 20), ("ising", 21, 8, 2, 2, 20)])
def test_cost_gradient_tensor_core(prec, kind, n, h, L, r, Ns):
    """tdo_grad on a tensor-core context runs the tensor-core backward (16-bit activations, FP32
    accumulation, softmax attention by warp-level FP16 MMAs) for every N <= 32: one 16-token block per
    (sequence, head) up to N = 16, two query and two key blocks from N = 17 (N = 21 reads the deepest
    staged row, 5 x 21 + 31 = 136).  The bias block b1 is a 16-bit sum over every row whose terms cancel;
    with a dozen samples at N = 32 its relative error reaches 0.15 (FP16) against 0.05 with 48, for every
    N, so the long chains get enough samples for the bounds to measure the kernels, not the cancellation."""
    from paper_2502_20723_gb300 import tdo
    prob = problem(kind, n)
    spec = synth.model_spec(64, h, L, r)
    th = synth.init_params(spec, seed=21, std=0.05)
    sig, sigp = synth.random_configs(n, Ns, seed=9)
    g, cost = tdo.Context(prob, spec, th, prec).grad(dev(sig), dev(sigp))
    g = g.cpu().numpy()
    ref, c_ref, _, _ = E.grad_estimator(prob, spec, th, sig, sigp)
    rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    blocks = block_errors(spec, g, ref)
    print(f"{prec} gradient: relative error {rel:.3e}, worst block {max(blocks, key=blocks.get)} "
          f"{max(blocks.values()):.2e}")
    w_tol, b_tol, n_tol = GRAD_BOUNDS[prec]
    assert abs(cost - c_ref) <= 1e-3 * c_ref
    bad = {k: v for k, v in blocks.items() if v > (b_tol if k.startswith("b") else w_tol)}
    assert not bad, bad
    assert rel <= n_tol


@pytest.mark.parametrize("prec,tol", [("bf16", 5e-2), ("fp16", 1e-2)])
@pytest.mark.parametrize("kind,n,d,h,L,r,Ns", [("xyz", 6, 32, 4, 1, 0, 256), ("ising", 8, 32, 4, 1, 0, 40)])
def test_sr_step_bf16(prec, tol, kind, n, d, h, L, r, Ns):
    """One SR step of a tensor-core context: 16-bit forward and backward, the SR matrix's log-derivatives
    stored in BF16 (shifted by their mean over the first 64 samples), FP64 CG.  The parameter update is
    within tol of the oracle's FP64 step in norm (measured values are reported)."""
    from paper_2502_20723_gb300 import tdo
    prob = problem(kind, n)
    spec = synth.model_spec(d, h, L, r)
    th = synth.init_params(spec, 0, std=0.1 if d == 32 else 0.05)
    sig, sigp = synth.random_configs(n, Ns, seed=8)
    ctx = tdo.Context(prob, spec, th, prec)
    cost = ctx.sr_step(dev(sig), dev(sigp), 0.01, 0.1)
    new = ctx.get_params()
    ref_new, c_ref, _, _ = E.sr_step(prob, spec, th, sig, sigp, 0.01, 0.1)
    rel = np.linalg.norm((new - th) - (ref_new - th)) / np.linalg.norm(ref_new - th)
    print(f"{prec} SR update relative error {rel:.3e}, cost {cost:.6f} vs {c_ref:.6f}")
    assert abs(cost - c_ref) <= 1e-3 * c_ref
    assert rel <= tol


@pytest.mark.parametrize("prec,tol", [("bf16", 3e-2), ("fp16", 3e-3)])
@pytest.mark.parametrize("kind,n,h,L,r,B,std", [("ising", 16, 8, 2, 4, 7, 0.05), ("xyz", 16, 4, 1, 2, 10, 0.05),
                                                 ("ising", 16, 8, 4, 4, 3, 0.02), ("ising", 24, 8, 2, 4, 5, 0.05),
                                                 ("xyz", 24, 4, 1, 2, 6, 0.05), ("ising", 32, 8, 2, 4, 5, 0.05),
                                                 ("xyz", 32, 8, 4, 4, 3, 0.02)])
def test_jacobian_tensor_core(prec, tol, kind, n, h, L, r, B, std):
    """tdo_jacobian on a 16-bit context at N = 16, 24 and 32: two virtual configurations per sample (one
    per real cotangent seed) through the tensor-core forward and backward with per-configuration
    weight-gradient MMAs over each configuration's 2N rows (N = 16: four configurations per tile, so an
    odd sample count leaves a half-empty last tile; N = 24: two, 96 of the tile's 128 rows; N = 32: two,
    all 128 rows).  Within the bound of the oracle's log-derivatives in norm, per sample (measured
    values are reported)."""
    spec = synth.model_spec(64, h, L, r)
    th = synth.init_params(spec, seed=13, std=std)
    sig, sigp = synth.random_configs(n, B, seed=3)
    from paper_2502_20723_gb300 import tdo
    O = tdo.Context(problem(kind, n), spec, th, prec).jacobian(dev(sig), dev(sigp)).cpu().numpy()
    got = O[..., 0].astype(np.float64) + 1j * O[..., 1]
    ref = E.jacobian(spec, th, sig, sigp, n)
    rel = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    print(f"{prec} tensor-core log-derivatives: relative error per sample max {rel.max():.3e}")
    assert rel.max() <= tol


@pytest.mark.parametrize("n,Ns", [(16, 70), (16, 37), (24, 41), (32, 33)])
def test_sr_step_bf16_log_derivative_storage(n, Ns):
    """At N = 16, 24 and 32 a BF16 context's SR step stores the tensor-core log-derivatives as BF16 pairs
    of O - ō (written by the staged per-configuration flushes).  Its update must equal, within 2e-3 in
    norm, the solve of the same system from the FP32 log-derivatives of tdo_jacobian (same gradient,
    shift and CG tolerance): the only difference is the BF16 rounding of the centred values."""
    prob = problem("ising", n)
    spec = synth.model_spec(64, 8, 2, 4)
    th = synth.init_params(spec, 4, std=0.05)
    sig, sigp = synth.random_configs(n, Ns, seed=12)
    lr, shift = 0.01, 0.004
    ref_ctx = ctx_for(prob, spec, th)
    g, _ = ref_ctx.grad(dev(sig), dev(sigp))
    O = ref_ctx.jacobian(dev(sig), dev(sigp))
    x, it, res = ref_ctx.sr_solve(O, g, shift, tol=1e-6, max_iter=100)
    ctx = ctx_for(prob, spec, th)
    ctx.sr_step(dev(sig), dev(sigp), lr, shift)
    delta = (th - ctx.get_params()) / lr
    x = x.cpu().numpy()
    rel = np.linalg.norm(delta - x) / np.linalg.norm(x)
    print(f"SR update from BF16-stored log-derivatives: relative difference {rel:.3e} ({it} CG iterations)")
    assert rel <= 2e-3
