"""GPU (FP32 path) vs the FP64 oracle on identical seeded inputs, through the C ABI.

Tolerances (FP32 path): log rho within 1e-6 relative (phase modulo 2 pi); connection coefficients
within FP32 rounding of the FP64 sums; L_loc, cost, gradient, log-derivatives within the accumulated
FP32 rounding of their terms (bounds stated per test)."""
import numpy as np
import pytest

from oracle import estimators as E, lindblad, sampler as OS, transformer as T
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


def ctx_for(prob, spec, theta, precision="fp32"):
    from paper_2502_20723_gb300 import tdo
    return tdo.Context(prob, spec, theta, precision)


def dev(a):
    return torch.as_tensor(np.asarray(a).astype(np.int64)).to(torch.int32).cuda()


# ------------------------------------------------------------------ log rho (forward)
FWD_CASES = [
    # (N, d, heads, layers, mlp, B)
    (4, 16, 2, 1, 0, 256),     # the N=4 Ising workload shape, every doubled configuration
    (8, 32, 4, 2, 0, 1000),    # N=8 workload shape, ragged last tile
    (16, 64, 8, 4, 4, 333),    # N=16 headline shape
    (1, 16, 4, 2, 2, 7),
    (3, 16, 1, 1, 0, 50),
    (7, 32, 8, 3, 1, 77),
    (13, 64, 4, 2, 0, 41),
    (24, 64, 16, 1, 2, 19),
    (32, 64, 8, 2, 4, 11),
]


@pytest.mark.parametrize("n,d,h,L,r,B", FWD_CASES)
def test_log_rho_fp32(n, d, h, L, r, B):
    spec = synth.model_spec(d, h, L, r)
    th = synth.init_params(spec, seed=n + d, std=0.1 if d * L * (1 + r) < 256 else 0.04)
    prob = problem("ising", n)
    if B == 4 ** n:
        sig, sigp = synth.all_configs(n)
    else:
        sig, sigp = synth.random_configs(n, B, seed=B)
    ref = T.log_rho_np(spec, th, sig, sigp, n)
    ctx = ctx_for(prob, spec, th)
    out = ctx.log_rho(dev(sig), dev(sigp)).cpu().numpy()
    err = logrho_err(out, ref)
    # relative to each element's |log rho| (measured at most 2.6e-7; |log rho| >= 0.55 in these cases)
    assert np.all(err <= 1e-6 * np.abs(ref)), ((err / np.abs(ref)).max(), np.abs(ref).min())
    # host pointers give the same bits
    host = ctx.log_rho(sig.astype(np.uint32), sigp.astype(np.uint32))
    assert np.array_equal(host, out)


def test_log_rho_std_init_relative():
    """Default N(0, 0.02) parameters at the headline shape: within 1e-6 of |log rho| (relative)."""
    spec = synth.model_spec(64, 8, 4, 4)
    th = synth.init_params(spec, 0)
    sig, sigp = synth.random_configs(16, 512, seed=3)
    ref = T.log_rho_np(spec, th, sig, sigp, 16)
    out = ctx_for(problem("ising", 16), spec, th).log_rho(dev(sig), dev(sigp)).cpu().numpy()
    assert np.all(logrho_err(out, ref) <= 1e-6 * np.abs(ref))


def test_log_rho_empty_and_single():
    spec = synth.model_spec(16, 2, 1, 0)
    ctx = ctx_for(problem("ising", 4), spec, synth.init_params(spec))
    out = ctx.log_rho(dev([]), dev([]))
    assert out.shape == (0, 2)
    one = ctx.log_rho(dev([5]), dev([9])).cpu().numpy()
    ref = T.log_rho_np(spec, synth.init_params(spec), np.array([5], np.uint32), np.array([9], np.uint32), 4)
    assert logrho_err(one, ref)[0] < 1e-6


def test_set_params_roundtrip_and_autograd():
    from paper_2502_20723_gb300 import tdo
    spec = synth.model_spec(32, 4, 2, 2)
    th = synth.init_params(spec, 1, std=0.1)
    ctx = ctx_for(problem("ising", 8), spec, th)
    assert np.array_equal(ctx.get_params(), th)
    th2 = synth.init_params(spec, 2, std=0.1)
    ctx.set_params(torch.as_tensor(th2).cuda())
    assert np.array_equal(ctx.get_params(), th2)
    sig, sigp = synth.random_configs(8, 37, seed=1)
    # autograd.Function: d/dtheta of sum(w . (Re, Im) log rho) vs the oracle's autograd
    LogRho = tdo.log_rho_autograd()
    t = torch.as_tensor(th2).cuda().requires_grad_(True)
    y = LogRho.apply(t, dev(sig), dev(sigp), ctx)
    w = torch.as_tensor(np.random.default_rng(0).standard_normal((37, 2))).float().cuda()
    (y * w).sum().backward()
    tt = torch.as_tensor(th2).requires_grad_(True)
    re, im = T.log_rho_parts(spec, tt, sig, sigp, 8)
    wc = w.cpu().double()
    ((re * wc[:, 0]) + (im * wc[:, 1])).sum().backward()
    g_ref = tt.grad.numpy()
    g = t.grad.cpu().numpy()
    assert np.abs(g - g_ref).max() <= 1e-5 * max(1.0, np.abs(g_ref).max())


# ------------------------------------------------------------------ connections (rows of Lhat)
@pytest.mark.parametrize("kind,n,kw", [
    ("ising", 4, {}), ("ising", 16, dict(g=0.5)), ("xyz", 8, dict(Jx=0.9)), ("xyz", 8, dict(Jx=1.0)),
    ("xyz", 5, dict(Jx=1.4, Jy=2.0, Jz=1.0, Bx=-1.0, By=0.7, Bz=0.1)), ("ising", 32, {}), ("ising", 1, {}),
    ("heis", 10, {}), ("ising2d", 4, {}), ("ising2d", 6, {}),
])
def test_connections_match_oracle_rows(kind, n, kw):
    prob = problem(kind, n, **kw)
    spec = synth.model_spec(16, 2, 1, 0)
    ctx = ctx_for(prob, spec, synth.init_params(spec))
    sig, sigp = synth.random_configs(n, 200, seed=n)
    cnt, cs, cp, cc = [x.cpu().numpy() for x in ctx.connections(dev(sig), dev(sigp))]
    rows = E.connections(prob, sig, sigp)
    for s in range(len(sig)):
        k = int(cnt[s])
        assert (int(cs[s, 0]) & 0xFFFFFFFF, int(cp[s, 0]) & 0xFFFFFFFF) == (int(sig[s]), int(sigp[s]))
        got = {}
        for j in range(k):
            key = (int(cs[s, j]) & 0xFFFFFFFF, int(cp[s, j]) & 0xFFFFFFFF)
            assert key not in got, "duplicate connection"
            got[key] = complex(cc[s, j, 0], cc[s, j, 1])
        ref = {key: v for key, v in rows[s]}
        keys = set(got) | set(ref)
        for key in keys:
            a, b = got.get(key, 0j), ref.get(key, 0j)
            assert abs(a - b) <= 1e-6 * max(1.0, abs(b)), (s, key, a, b)
        # nonzero entries appear on both sides (zero diagonal allowed)
        assert {k2 for k2, v in ref.items() if abs(v) > 1e-9} <= set(got)


# ------------------------------------------------------------------ L_loc, cost
@pytest.mark.parametrize("kind,n,d,h,L,r,Ns", [
    ("ising", 4, 16, 2, 1, 0, 256), ("ising", 8, 32, 4, 2, 0, 300), ("xyz", 8, 32, 4, 2, 0, 300),
    ("ising", 16, 64, 8, 4, 4, 64), ("heis", 5, 32, 4, 2, 0, 300), ("heis", 10, 32, 4, 2, 0, 200),
    ("ising2d", 6, 32, 4, 2, 0, 300),
])
def test_local_estimator_and_cost(kind, n, d, h, L, r, Ns):
    prob = problem(kind, n)
    spec = synth.model_spec(d, h, L, r)
    th = synth.init_params(spec, seed=3, std=0.2 if d < 64 else 0.04)
    if Ns == 4 ** n:
        sig, sigp = synth.all_configs(n)
    else:
        sig, sigp = synth.random_configs(n, Ns, seed=5)
    ctx = ctx_for(prob, spec, th)
    lloc, cost, se = ctx.local_estimator(dev(sig), dev(sigp))
    lloc = lloc.cpu().numpy()
    ref = E.local_estimator(prob, spec, th, sig, sigp)
    # each term coef * rho_y/rho_x carries FP32 rounding of log rho (<= 1e-6 rel) and of exp: bound by
    # 1e-5 of the sum of |terms| (computed from the oracle rows)
    rows = E.connections(prob, sig, sigp)
    scale = np.array([sum(abs(v) for _, v in r_) for r_ in rows]) * 3
    got = lloc[:, 0] + 1j * lloc[:, 1]
    assert np.all(np.abs(got - ref) <= 1e-5 * scale)
    c_ref, se_ref = E.cost_mc(ref)
    assert abs(cost - c_ref) <= 1e-5 * c_ref
    assert abs(se - se_ref) <= 1e-3 * se_ref + 1e-12


def test_cost_full_sum_n4():
    """All 256 configurations weighted by the exact P(x): the GPU L_loc reproduce the full-sum cost."""
    prob = problem("ising", 4)
    spec = synth.model_spec(16, 2, 1, 0)
    th = synth.init_params(spec, 0)
    a, b, w = E.full_sum_weights(prob, spec, th)
    lloc, _, _ = ctx_for(prob, spec, th).local_estimator(dev(a), dev(b))
    lloc = lloc.cpu().numpy()
    c = float((w * (lloc[:, 0] ** 2 + lloc[:, 1] ** 2)).sum())
    ref = E.full_sum_cost(prob, spec, th)
    assert abs(c - ref) <= 1e-5 * ref


# ------------------------------------------------------------------ Jacobian, VJP, gradient
@pytest.mark.parametrize("n,d,h,L,r,B", [(4, 16, 2, 1, 0, 40), (8, 32, 4, 2, 0, 33), (16, 64, 8, 4, 4, 6),
                                         (5, 16, 4, 2, 2, 9), (32, 64, 8, 1, 1, 3)])
def test_jacobian(n, d, h, L, r, B):
    spec = synth.model_spec(d, h, L, r)
    th = synth.init_params(spec, seed=7, std=0.2 if d < 64 else 0.04)
    sig, sigp = synth.random_configs(n, B, seed=2)
    O = ctx_for(problem("ising", n), spec, th).jacobian(dev(sig), dev(sigp)).cpu().numpy()
    ref = E.jacobian(spec, th, sig, sigp, n)
    got = O[..., 0] + 1j * O[..., 1]
    scale = max(1.0, np.abs(ref).max())
    assert np.abs(got - ref).max() <= 2e-5 * scale, np.abs(got - ref).max()


@pytest.mark.parametrize("n,d,h,L,r,B", [(8, 32, 4, 2, 0, 500), (16, 64, 8, 4, 4, 40),
                                         (6, 16, 2, 1, 0, 300), (13, 64, 8, 2, 2, 50), (5, 32, 4, 1, 4, 77)])
def test_vjp_random_cotangents(n, d, h, L, r, B):
    """Includes ragged tiles (N not dividing the 64/128-row tile): padding rows must not leak into the
    weight-gradient sums."""
    spec = synth.model_spec(d, h, L, r)
    th = synth.init_params(spec, seed=9, std=0.2 if d < 64 else 0.04)
    sig, sigp = synth.random_configs(n, B, seed=4)
    cot = np.random.default_rng(1).standard_normal((B, 2)).astype(np.float32)
    grad = torch.zeros(synth.num_params(spec), dtype=torch.float64, device="cuda")
    ctx_for(problem("ising", n), spec, th).log_rho_vjp(dev(sig), dev(sigp), torch.as_tensor(cot).cuda(), grad)
    tt = torch.as_tensor(th).requires_grad_(True)
    lr = T.log_rho(spec, tt, sig, sigp, n)
    c = torch.as_tensor(cot.astype(np.float64))
    (c[:, 0] * lr.real - c[:, 1] * lr.imag).sum().backward()
    ref = tt.grad.numpy()
    g = grad.cpu().numpy()
    assert np.abs(g - ref).max() <= 1e-4 * np.abs(ref).max()
    assert np.linalg.norm(g - ref) <= 2e-5 * np.linalg.norm(ref)


@pytest.mark.parametrize("kind,n,d,h,L,r,Ns", [("ising", 8, 32, 4, 2, 0, 256), ("xyz", 8, 32, 4, 2, 0, 256),
                                               ("ising", 16, 64, 8, 4, 4, 48), ("heis", 5, 32, 4, 2, 0, 200),
                                               ("ising2d", 6, 32, 4, 2, 0, 200)])
def test_cost_gradient(kind, n, d, h, L, r, Ns):
    prob = problem(kind, n)
    spec = synth.model_spec(d, h, L, r)
    th = synth.init_params(spec, seed=11, std=0.2 if d < 64 else 0.04)
    sig, sigp = synth.random_configs(n, Ns, seed=6)
    g, cost = ctx_for(prob, spec, th).grad(dev(sig), dev(sigp))
    g = g.cpu().numpy()
    ref, c_ref, _, _ = E.grad_estimator(prob, spec, th, sig, sigp)
    assert abs(cost - c_ref) <= 1e-5 * c_ref
    # element by element per named block (a wrong small block shows even where the norm would hide it):
    # measured at most 1.8e-4 of the block's largest entry (the MLP biases of the 4-layer case, sums over
    # every connected row), 5e-6 in norm
    worst = {k: v for k, v in block_errors(spec, g, ref).items() if v > 1e-3}
    assert not worst, worst
    assert np.linalg.norm(g - ref) <= 2e-5 * np.linalg.norm(ref), np.linalg.norm(g - ref) / np.linalg.norm(ref)


# ------------------------------------------------------------------ SR
def _re_s_norm(O):
    """||Re S||_2 for S = Obar^H Obar / Ns (O: [Ns][P][2] FP32), from the 2Ns x 2Ns Gram matrix of the
    centred real and imaginary parts; also returns those centred parts (FP64)."""
    Ns = O.shape[0]
    Or = O[..., 0].astype(np.float64)
    Oi = O[..., 1].astype(np.float64)
    Or -= Or.mean(axis=0)
    Oi -= Oi.mean(axis=0)
    A = np.concatenate([Or, Oi], axis=0)
    return float(np.linalg.eigvalsh(A @ A.T).max()) / Ns, (Or, Oi)


def test_sr_solve_matches_cholesky():
    """Identical FP32 O on both sides: FP64 CG (GPU) vs FP64 Cholesky (oracle)."""
    spec = synth.model_spec(16, 2, 1, 0)
    th = synth.init_params(spec)
    ctx = ctx_for(problem("ising", 4), spec, th)
    P = ctx.P
    rng = np.random.default_rng(0)
    O = (rng.standard_normal((300, P, 2)) * 0.3).astype(np.float32)
    O[:, :, 0] += rng.standard_normal(P).astype(np.float32)   # nonzero mean, removed by the centring
    rhs = rng.standard_normal(P)
    x, it, res = ctx.sr_solve(torch.as_tensor(O).cuda(), torch.as_tensor(rhs).cuda(), 1e-2, tol=1e-12, max_iter=2000)
    ref = E.sr_solve(O[..., 0].astype(np.float64) + 1j * O[..., 1].astype(np.float64), rhs, 1e-2)
    assert res < 1e-10
    # FP32 products in the matvec: forward error within cond(Re S + lambda I) x 4 FP32 units
    norm_s, _ = _re_s_norm(O)
    cond = (norm_s + 1e-2) / 1e-2
    err = np.linalg.norm(x.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err <= 4 * 2.0 ** -24 * cond, (err, cond)


@pytest.mark.parametrize("d,h,L,r,Ns", [(32, 4, 2, 0, 301), (64, 8, 2, 4, 77), (64, 8, 4, 4, 69),
                                         (64, 8, 6, 4, 37), (64, 8, 8, 4, 45)])
def test_sr_solve_residual_any_size(d, h, L, r, Ns):
    """P from 8k to 396k parameters (one to six parameters per thread of the one-pass matvec on 152
    SMs), Ns not a multiple of the row block: the true residual of (Re S + lambda I) x = rhs, formed in
    FP64 from the same FP32 O, is at the FP32-product level."""
    spec = synth.model_spec(d, h, L, r)
    ctx = ctx_for(problem("ising", 4), spec, synth.init_params(spec))
    P = ctx.P
    rng = np.random.default_rng(P)
    O = (rng.standard_normal((Ns, P, 2)) * 0.3).astype(np.float32)
    O[:, :, 1] += rng.standard_normal(P).astype(np.float32)
    rhs = rng.standard_normal(P)
    lam = 1e-2
    x, it, res = ctx.sr_solve(torch.as_tensor(O).cuda(), torch.as_tensor(rhs).cuda(), lam, tol=1e-8, max_iter=500)
    x = x.cpu().numpy()
    norm_s, (Or, Oi) = _re_s_norm(O)
    Sx = (Or.T @ (Or @ x) + Oi.T @ (Oi @ x)) / Ns + lam * x
    assert res <= 1e-8 and it < 500
    # normwise backward error of the computed x at the FP32-product level
    eta = np.linalg.norm(Sx - rhs) / ((norm_s + lam) * np.linalg.norm(x) + np.linalg.norm(rhs))
    assert eta <= 1e-6, eta


def test_sr_step_matches_oracle():
    prob = problem("xyz", 6, Jx=0.9)
    spec = synth.model_spec(16, 2, 1, 0)
    th = synth.init_params(spec, 0, std=0.1)
    sig, sigp = synth.random_configs(6, 256, seed=8)
    ctx = ctx_for(prob, spec, th)
    cost = ctx.sr_step(dev(sig), dev(sigp), 0.01, 0.1)
    new = ctx.get_params()
    ref_new, c_ref, g_ref, d_ref = E.sr_step(prob, spec, th, sig, sigp, 0.01, 0.1)
    assert abs(cost - c_ref) <= 1e-5 * c_ref
    assert np.linalg.norm((new - th) - (ref_new - th)) <= 1e-3 * np.linalg.norm(ref_new - th)


def test_sr_step_adam_three_steps_match_oracle():
    """Adam on the SR direction (tdo_set_optimizer): three steps on the same samples, each compared element by
    element with the oracle's Cholesky SR direction fed to its Adam (Kingma and Ba).  The CG runs to 1e-12, so
    the FP32 context's direction agrees with the oracle's to about 1e-5 of max|delta| (the FP32 rounding of
    the log-derivatives and gradient); one Adam update moves by at most lr / eps per unit change of delta,
    which bounds the parameter difference after t steps by t lr / eps 2e-5 max|delta|."""
    prob = problem("ising", 4)
    spec = synth.model_spec(16, 2, 1, 0)
    th = synth.init_params(spec, 3, std=0.1)
    sig, sigp = synth.random_configs(4, 200, seed=5)
    ctx = ctx_for(prob, spec, th)
    ctx.set_sr_options(1e-12, 4000)
    lr, shift, eps = 0.01, 0.01, 0.1
    ctx.set_optimizer("adam", 0.9, 0.999, eps)
    ref, m, v = th.copy(), np.zeros_like(th), np.zeros_like(th)
    dmax = 0.0
    for t in range(1, 4):
        ctx.sr_step(dev(sig), dev(sigp), lr, shift)
        _, _, _, delta = E.sr_step(prob, spec, ref, sig, sigp, lr, shift)
        dmax = max(dmax, np.abs(delta).max())
        ref, m, v = E.adam_step(ref, delta, m, v, t, lr, 0.9, 0.999, eps)
        got = ctx.get_params()
        err = np.abs(got - ref).max()
        assert err <= t * lr / eps * 2e-5 * dmax, (t, err, dmax)
        assert np.abs(got - th).max() > 0.5 * lr   # the steps moved the parameters by order lr


# ------------------------------------------------------------------ Metropolis
def test_metropolis_replays_oracle_chains():
    """Same Philox stream on both sides: every chain whose accept decisions are all decided by more than
    1e-3 in log space follows exactly the oracle's trajectory."""
    n = 6
    spec = synth.model_spec(16, 2, 1, 0)
    th = synth.init_params(spec, 0, std=0.5)
    s0, s1 = synth.random_configs(n, 128, seed=1)
    ctx = ctx_for(problem("ising", n), spec, th)
    a, b = dev(s0), dev(s1)
    acc, (ss, sp) = ctx.sample(a, b, 5, seed=1234, counter=77, samples=True)
    o0, o1, oacc, osamp, margin = OS.metropolis(spec, th, s0, s1, n, 5, 1234, 77, record=True)
    ok = margin > 1e-3
    assert ok.mean() > 0.9
    g0 = (a.cpu().numpy().astype(np.int64) & 0xFFFFFFFF)
    g1 = (b.cpu().numpy().astype(np.int64) & 0xFFFFFFFF)
    assert np.array_equal(g0[ok], o0[ok].astype(np.int64)) and np.array_equal(g1[ok], o1[ok].astype(np.int64))
    for sw in range(5):
        assert np.array_equal(ss[sw].cpu().numpy().astype(np.int64)[ok] & 0xFFFFFFFF, osamp[sw][0][ok].astype(np.int64))
    if ok.all():
        assert acc == oacc


def test_metropolis_histogram_n3():
    """Chain-end states of many chains follow |rho|^2 / sum |rho|^2 (chi-square), N = 3.  (A much
    larger init scale concentrates |rho|^2 on diagonal states that single-bit moves connect only through
    tiny off-diagonal weights; the oracle's own chains then do not mix either.)"""
    from scipy import stats
    n = 3
    spec = synth.model_spec(16, 2, 1, 0)
    th = synth.init_params(spec, 0, std=0.3)
    prob = problem("ising", n)
    _, _, w = E.full_sum_weights(prob, spec, th)
    chains = 20000
    s0, s1 = synth.random_configs(n, chains, seed=2)
    a, b = dev(s0), dev(s1)
    ctx_for(prob, spec, th).sample(a, b, 40, seed=5, counter=0)
    idx = (a.cpu().numpy().astype(np.int64) << n) | b.cpu().numpy().astype(np.int64)
    counts = np.bincount(idx, minlength=64)
    assert stats.chisquare(counts, w * chains).pvalue > 1e-4


# ------------------------------------------------------------------ errors
def test_invalid_arguments():
    from paper_2502_20723_gb300 import tdo
    spec = synth.model_spec(16, 2, 1, 0)
    th = synth.init_params(spec)
    with pytest.raises(tdo.TdoError, match="EUNSUPPORTED"):
        tdo.Context({"n_sites": 33, "terms": [], "jumps": []}, spec, th)
    with pytest.raises(tdo.TdoError, match="EINVAL"):
        tdo.Context(problem("ising", 4), spec, th[:-1])
    with pytest.raises(tdo.TdoError, match="EINVAL"):
        tdo.Context({"n_sites": 4, "terms": [(1.0, ((5, "X"),))], "jumps": []}, spec, th)


def test_nan_parameters_raise_numeric():
    from paper_2502_20723_gb300 import tdo
    spec = synth.model_spec(16, 2, 1, 0)
    th = synth.init_params(spec)
    th[3] = np.nan
    ctx = ctx_for(problem("ising", 4), spec, th)
    sig, sigp = synth.random_configs(4, 10)
    with pytest.raises(tdo.TdoError, match="ENUMERIC"):
        ctx.local_estimator(dev(sig), dev(sigp))


# ------------------------------------------------------------------ conv embedding (Eq. circ-conv)
CONV_CASES = [
    # (N, d, heads, layers, mlp, C1, B)
    (4, 16, 2, 1, 0, 4, 40),
    (8, 32, 4, 2, 0, 8, 33),
    (13, 64, 8, 2, 2, 16, 21),    # ragged tile
    (3, 16, 4, 1, 1, 3, 17),      # sites i+1, i+2 wrap twice
]


def _conv(d, h, L, r, c1, seed):
    spec = synth.model_spec(d, h, L, r, embed="conv", conv_channels=c1)
    return spec, synth.init_params(spec, seed=seed, std=0.2 if d < 64 else 0.05)


@pytest.mark.parametrize("n,d,h,L,r,c1,B", CONV_CASES)
def test_conv_log_rho(n, d, h, L, r, c1, B):
    spec, th = _conv(d, h, L, r, c1, 3)
    sig, sigp = synth.random_configs(n, B, seed=5)
    out = ctx_for(problem("ising", n), spec, th).log_rho(dev(sig), dev(sigp)).cpu().numpy()
    ref = T.log_rho_np(spec, th, sig, sigp, n)
    assert np.all(logrho_err(out, ref) <= 1e-6 * np.maximum(np.abs(ref), 1.0))


@pytest.mark.parametrize("n,d,h,L,r,c1,B", CONV_CASES)
def test_conv_jacobian(n, d, h, L, r, c1, B):
    """Per-configuration log-derivatives including the two conv layers (table gradient per pattern,
    then back through both convolutions and GELUs)."""
    spec, th = _conv(d, h, L, r, c1, 4)
    sig, sigp = synth.random_configs(n, B, seed=6)
    O = ctx_for(problem("ising", n), spec, th).jacobian(dev(sig), dev(sigp)).cpu().numpy()
    ref = E.jacobian(spec, th, sig, sigp, n)
    got = O[..., 0] + 1j * O[..., 1]
    scale = max(1.0, np.abs(ref).max())
    assert np.abs(got - ref).max() <= 2e-5 * scale, np.abs(got - ref).max()


@pytest.mark.parametrize("n,d,h,L,r,c1,B", CONV_CASES)
def test_conv_vjp(n, d, h, L, r, c1, B):
    spec, th = _conv(d, h, L, r, c1, 5)
    sig, sigp = synth.random_configs(n, B, seed=7)
    cot = np.random.default_rng(2).standard_normal((B, 2)).astype(np.float32)
    grad = torch.zeros(synth.num_params(spec), dtype=torch.float64, device="cuda")
    ctx_for(problem("ising", n), spec, th).log_rho_vjp(dev(sig), dev(sigp), torch.as_tensor(cot).cuda(), grad)
    tt = torch.as_tensor(th).requires_grad_(True)
    lr = T.log_rho(spec, tt, sig, sigp, n)
    c = torch.as_tensor(cot.astype(np.float64))
    (c[:, 0] * lr.real - c[:, 1] * lr.imag).sum().backward()
    ref = tt.grad.numpy()
    g = grad.cpu().numpy()
    assert np.abs(g - ref).max() <= 1e-4 * np.abs(ref).max()
    assert np.linalg.norm(g - ref) <= 2e-5 * np.linalg.norm(ref)


@pytest.mark.parametrize("kind,n", [("ising", 8), ("xyz", 6)])
def test_conv_cost_gradient(kind, n):
    prob = problem(kind, n)
    spec, th = _conv(32, 4, 2, 0, 8, 8)
    sig, sigp = synth.random_configs(n, 200, seed=9)
    g, cost = ctx_for(prob, spec, th).grad(dev(sig), dev(sigp))
    ref, c_ref, _, _ = E.grad_estimator(prob, spec, th, sig, sigp)
    assert abs(cost - c_ref) <= 1e-5 * c_ref
    assert np.linalg.norm(g.cpu().numpy() - ref) <= 1e-4 * np.linalg.norm(ref)
