"""The whole optimisation-workflow step as one CUDA graph (tdo_set_step_graph) against the same step run call
by call (tdo_vmc_step without the graph), through the C ABI.

The graph runs the same kernels in the same order; what differs is where the host's mid-step decisions
live: the connected-row count is read by the kernels from device memory (buffers and grids sized for
Ns x n_pat rows), the CG iterations are a conditional while node, the sampler's counter and Adam's bias
corrections come from device memory.  The only numerical difference is the order of the float atomics
of the gradient sums, which differs between any two runs of either mode: measured on GB300 at N = 16,
two call-by-call runs differ by 3.8e-6 in the first gradient and by 6.7e-7, 2.1e-5, 1.7e-4 of the
update theta_k - theta_0 after steps 1, 2, 3; graph against call-by-call: 4.0e-6 and 9.4e-7, 3.7e-5,
2.1e-4.  The growth is the optimisation's, not the graph's: each step's gradient depends on the last
step's parameters, a CG that crosses its tolerance one iteration earlier changes the update by about
that tolerance, and Adam divides by the square root of small second moments (2.2e-3 after two Adam
steps, and 9.2e-3 after one, have been seen between the modes: Adam's own bounds are 2e-2, 5e-2, 1e-1 of
the update).  So, from the same parameters and chains:
  - the first step is deterministic up to the first gradient's atomics: the same cost bit for bit, the
    parameters within 2e-5 of the update;
  - over three steps the chains stay equal (the Metropolis decisions replay; a decision whose margin is
    below the atomics' rounding could flip, so at most 2 chains may differ and the count is printed), the
    costs agree to 2e-3 relative, the parameters to 1e-2 and 5e-2 of the update after steps 2 and 3, and
    the CG iteration counts within two;
  - one more step from the same parameters and chains in both modes (a later counter, the graph recorded
    again for the new chain buffers, the solve started cold after tdo_set_params) gives the same cost bit
    for bit and parameters within 5e-4 of its update (measured up to 7.5e-5: from these later parameters
    the CG runs longer and amplifies the first gradient's atomics more than at step 1).
Also: the graph is recorded once for a fixed schedule and again whenever lr or the shift changes; Adam's
bias corrections replay; host chain buffers are staged; a non-finite L_loc leaves every finite parameter
unchanged and reports TDO_ENUMERIC as the call-by-call step does; an FP32 context refuses graph mode."""
import numpy as np
import pytest

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


def dev(a):
    return torch.as_tensor(np.asarray(a).astype(np.int64)).to(torch.int32).cuda()


def run(ctx, s0, s1, steps, sched, graph, host=False, counter=7):
    ctx.set_step_graph(graph)
    if host:
        a, b = s0.astype(np.uint32).copy(), s1.astype(np.uint32).copy()
    else:
        a, b = dev(s0), dev(s1)
    out = []
    for k in range(steps):
        cost, counter = ctx.vmc_step(a, b, 1, 1234, counter, k, sched)
        chains = (a.copy(), b.copy()) if host else (a.cpu().numpy().copy(), b.cpu().numpy().copy())
        out.append((cost, counter, ctx.sr_info()[0], chains, ctx.get_params().copy()))
    return out


PARAM_BOUND = (2e-5, 1e-2, 5e-2)
# Adam divides each component of the SR direction by its own magnitude (plus eps), so a component within
# the gradient atomics' noise of zero moves by up to 2 lr between any two runs: measured 9.2e-3 of the update
# norm after step 1 at P = 49,858 (one such component).  A wrong bias correction 1 - beta^t changes every
# component by tens of per cent, far above these bounds.
ADAM_PARAM_BOUND = (2e-2, 5e-2, 1e-1)


def compare(eager, graph, theta0, bounds=PARAM_BOUND):
    differing = 0
    for k, ((ce, ke, ie, he, pe), (cg, kg, ig, hg, pg)) in enumerate(zip(eager, graph)):
        assert ke == kg
        differing = max(differing, int(np.sum((he[0] != hg[0]) | (he[1] != hg[1]))))
        if k == 0:
            assert cg == ce, (cg, ce)
        assert abs(cg - ce) <= 2e-3 * abs(ce), (cg, ce)
        rel = np.linalg.norm(pg - pe) / np.linalg.norm(pe - theta0)
        print(f"step {k + 1}: cost {cg:.8f} vs {ce:.8f}, CG iterations {ig} vs {ie}, parameters differ by "
              f"{rel:.3e} of the update")
        assert rel <= bounds[k], rel
        assert abs(ig - ie) <= 2, (ig, ie)
    return differing


@pytest.mark.parametrize("prec,kind,n,L,Ns", [("fp16", "ising", 16, 2, 512), ("bf16", "xyz", 16, 1, 300),
                                              ("fp16", "ising", 24, 1, 256), ("fp16", "xyz", 8, 2, 400),
                                              ("fp8", "ising", 16, 1, 256)])
def test_graph_step_matches_call_by_call(prec, kind, n, L, Ns):
    from paper_2502_20723_gb300 import tdo
    spec = synth.model_spec(64, 8, L, 4)
    th = synth.init_params(spec, seed=21)
    s0, s1 = synth.random_configs(n, Ns, seed=5)
    sched = tdo.Schedule(eta0=0.0061, lambda0=0.004)   # constant over these steps (i_switch 30000)
    eager = run(tdo.Context(problem(kind, n), spec, th, prec), s0, s1, 3, sched, False)
    gctx = tdo.Context(problem(kind, n), spec, th, prec)
    graph = run(gctx, s0, s1, 3, sched, True)
    differing = compare(eager, graph, th)
    # one more step from the eager run's final parameters and chains in both modes
    th3, (c0, c1), ctr = eager[-1][4], eager[-1][3], eager[-1][1]
    ectx = tdo.Context(problem(kind, n), spec, th3, prec)
    ce, _ = ectx.vmc_step(dev(c0), dev(c1), 1, 1234, ctr, 3, sched)
    gctx.set_params(th3)
    cg, _ = gctx.vmc_step(dev(c0), dev(c1), 1, 1234, ctr, 3, sched)
    pe, pg = ectx.get_params(), gctx.get_params()
    rel = np.linalg.norm(pg - pe) / np.linalg.norm(pe - th3)
    rec, launches = gctx.step_graph_stats()
    print(f"{prec} {kind} N={n} L={L} Ns={Ns}: costs {[round(g[0], 6) for g in graph]}, CG iterations "
          f"{[g[2] for g in graph]}, chains differing {differing}; step 4 from equal states: cost {cg:.8f} vs "
          f"{ce:.8f}, parameters within {rel:.2e} of the update; recorded {rec}, launched {launches}")
    assert differing <= 2
    assert cg == ce and rel <= 5e-4, (cg, ce, rel)
    assert (rec, launches) == (2, 4)   # new chain buffers: recorded again


def test_graph_recorded_again_when_the_schedule_moves():
    """i_switch = 0: lr and the shift change every step, so every step is recorded again (and still equals
    the call-by-call step)."""
    from paper_2502_20723_gb300 import tdo
    n, spec = 16, synth.model_spec(64, 8, 1, 4)
    th = synth.init_params(spec, seed=2)
    s0, s1 = synth.random_configs(n, 256, seed=9)
    sched = tdo.Schedule(eta0=0.0061, i_switch=0, i_decay=4, lambda0=0.004, i_switch_sr=0, i_decay_sr=4)
    eager = run(tdo.Context(problem("ising", n), spec, th, "fp16"), s0, s1, 3, sched, False)
    gctx = tdo.Context(problem("ising", n), spec, th, "fp16")
    graph = run(gctx, s0, s1, 3, sched, True)
    assert compare(eager, graph, th) <= 2
    assert gctx.step_graph_stats() == (3, 3)


def test_graph_adam_and_host_chains():
    """Adam's bias corrections (1 - beta^t for t = 1, 2, 3) are uploaded per launch; host numpy chains are
    staged into the recorded device buffers and copied back."""
    from paper_2502_20723_gb300 import tdo
    n, spec = 16, synth.model_spec(64, 8, 1, 4)
    th = synth.init_params(spec, seed=3)
    s0, s1 = synth.random_configs(n, 256, seed=10)
    sched = tdo.Schedule(eta0=1e-3, lambda0=0.004)
    res = []
    for graph in (False, True):
        ctx = tdo.Context(problem("ising", n), spec, th, "fp16")
        ctx.set_optimizer("adam")
        res.append(run(ctx, s0, s1, 3, sched, graph, host=graph))
    assert compare(res[0], res[1], th, ADAM_PARAM_BOUND) <= 2


def test_graph_nonfinite_parameters_leave_the_rest_unchanged():
    from paper_2502_20723_gb300 import tdo
    n, spec = 16, synth.model_spec(64, 8, 1, 4)
    th = synth.init_params(spec, seed=4)
    th_bad = th.copy()
    th_bad[-1] = np.nan   # the head bias: every log rho, hence L_loc, is NaN
    s0, s1 = synth.random_configs(n, 128, seed=11)
    errs = []
    for graph in (False, True):
        ctx = tdo.Context(problem("ising", n), spec, th_bad, "fp16")
        ctx.set_step_graph(graph)
        with pytest.raises(tdo.TdoError) as e:
            ctx.vmc_step(dev(s0), dev(s1), 1, 5, 0, 0, tdo.Schedule())
        errs.append(str(e.value))
        after = ctx.get_params()
        assert np.array_equal(after[:-1], th_bad[:-1])
        # and the context still works once the parameters are finite
        ctx.set_params(th)
        cost, _ = ctx.vmc_step(dev(s0), dev(s1), 1, 5, 0, 0, tdo.Schedule())
        assert np.isfinite(cost)
    print(errs)
    assert all("non-finite" in e for e in errs)


def test_graph_needs_the_tensor_core_gradient():
    from paper_2502_20723_gb300 import tdo
    spec = synth.model_spec(32, 4, 1, 0)
    ctx = tdo.Context(problem("ising", 8), spec, synth.init_params(spec, seed=0), "fp32")
    with pytest.raises(tdo.TdoError):
        ctx.set_step_graph(True)
