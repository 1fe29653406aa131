"""tdo_local_estimator_noalloc: the local estimator for callers that may not allocate device memory while
they run (their memory belongs to another allocator, or they cannot afford the synchronisation that
cudaMalloc / cudaFree may imply).  It must give the same L_loc and cost as tdo_local_estimator, on two
calls in a row (its fixed scratch keeps the previous call's contents), and reject sizes beyond its
fixed scratch.  This file runs last (pytest collects files in name order)."""
import ctypes as C

import numpy as np
import pytest

from paper_2502_20723_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_20723_gb300 import build, tdo
    build.build()
    return tdo


def _dev(a):
    return torch.as_tensor(np.asarray(a).astype(np.int64)).to(torch.int32).cuda()


def _noalloc(tdo, ctx, sig, sigp):
    lloc = torch.empty((len(sig), 2), dtype=torch.float64, device="cuda")
    cost, se = C.c_double(), C.c_double()
    rc = tdo.lib().tdo_local_estimator_noalloc(ctx.h, sig.data_ptr(), sigp.data_ptr(), len(sig), lloc.data_ptr(),
                                              C.byref(cost), C.byref(se))
    return rc, lloc, cost.value, se.value


@pytest.mark.parametrize("precision,n,d,h,L,r", [("fp32", 16, 64, 8, 4, 4), ("bf16", 16, 64, 8, 4, 4),
                                                 ("fp32", 8, 32, 4, 2, 0)])
def test_noalloc_matches_local_estimator_twice(lib, precision, n, d, h, L, r):
    tdo = lib
    prob = synth.ising_chain(n)
    spec = synth.model_spec(d, h, L, r)
    ctx = tdo.Context(prob, spec, synth.init_params(spec, 0), precision)
    for call, ns in enumerate((1500, 700)):          # second call smaller: stale scratch must not leak in
        s0, s1 = synth.random_configs(n, ns, seed=10 + call)
        sig, sigp = _dev(s0), _dev(s1)
        ref_lloc, ref_cost, ref_se = ctx.local_estimator(sig, sigp)
        rc, lloc, cost, se = _noalloc(tdo, ctx, sig, sigp)
        assert rc == 0, tdo.lib().tdo_last_error(ctx.h)
        np.testing.assert_allclose(lloc.cpu().numpy(), ref_lloc.cpu().numpy(), rtol=1e-5, atol=1e-8)
        assert abs(cost - ref_cost) <= 1e-5 * ref_cost
        assert abs(se - ref_se) <= 1e-3 * ref_se + 1e-12


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    tdo = lib
    prob = synth.ising_chain(16)
    spec = synth.model_spec(16, 2, 1, 0)
    ctx = tdo.Context(prob, spec, synth.init_params(spec, 0))
    s0, s1 = synth.random_configs(16, 6000, seed=1)    # 6000 x 49 connections > 262144
    rc, _, _, _ = _noalloc(tdo, ctx, _dev(s0), _dev(s1))
    assert rc == -1
    assert b"exceeds its fixed scratch" in tdo.lib().tdo_last_error(ctx.h)
