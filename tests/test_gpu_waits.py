"""The bounded device waits of the tensor-core kernels: a wait that nothing completes gives up after its
poll limit, the kernel raises the context's error flag, frees its tensor memory and returns, and the call
reports TDO_ETIMEOUT; the context then keeps working (no GPU fault, no reset)."""
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


def test_wait_that_never_completes_reports_timeout_and_context_survives():
    from paper_2502_20723_gb300 import tdo
    spec = synth.model_spec(32, 4, 1, 0)
    th = synth.init_params(spec, 0, std=0.1)
    ctx = tdo.Context(problem("ising", 8), spec, th, "bf16")
    sig, sigp = synth.random_configs(8, 200, seed=2)
    a = torch.as_tensor(sig.astype(np.int64)).to(torch.int32).cuda()
    b = torch.as_tensor(sigp.astype(np.int64)).to(torch.int32).cuda()
    before = ctx.log_rho(a, b).cpu().numpy()
    for limit in (1, 1000, 1 << 16):
        assert ctx.wait_selftest(limit) == -5      # TDO_ETIMEOUT, twice in a row included
    assert "bounded wait" in tdo.lib().tdo_last_error(ctx.h).decode()
    after = ctx.log_rho(a, b).cpu().numpy()        # the flag was cleared and the kernels still run
    assert np.array_equal(before, after)
    assert ctx.wait_selftest(0) == -1              # limit out of range
    assert ctx.wait_selftest(1 << 21) == -1
    f32 = tdo.Context(problem("ising", 8), spec, th, "fp32")
    assert f32.wait_selftest(100) == -6            # BF16 contexts only
