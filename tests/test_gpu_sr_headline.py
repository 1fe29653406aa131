"""The SR step at the headline model width (N = 16, d = 64, 8 heads) against the FP64 oracle.

tdo_sr_step's update delta = (theta_old - theta_new) / eta is checked through the residual of the oracle's
own system, ||(Re S_oracle + lambda I) delta - grad_oracle|| / ||grad_oracle||, formed matrix-free from
the oracle's log-derivatives and gradient estimator (no P x P matrix, no Cholesky).  The step uses the
paper's initial rate and shift (eta_0 = 0.0061, lambda_0 = 0.004) and CG to 1e-10, so the residual
measures the context's arithmetic: FP32 rounding for the FP32 path; for the tensor-core paths the
16-bit operands of the backward and the BF16 storage of O - obar, amplified by the condition number of
S + lambda I.  Bounds: about three times the errors measured on GB300."""
import numpy as np
import pytest

from oracle import estimators as E
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


@pytest.mark.parametrize("prec,L,r,tol", [
    ("fp32", 1, 0, 6e-6), ("fp32", 2, 4, 6e-6),       # measured 1.8e-6, 8.6e-7
    ("fp16", 1, 0, 5e-4), ("fp16", 2, 4, 1e-3),       # measured 1.4e-4, 3.2e-4
    ("bf16", 1, 0, 5e-4), ("bf16", 2, 4, 1e-2),       # measured 1.6e-4, 2.9e-3
])
def test_sr_step_solves_the_oracle_system(prec, L, r, tol):
    from paper_2502_20723_gb300 import tdo
    n, Ns, lr, shift = 16, 64, 0.0061, 0.004
    prob = problem("ising", n)
    spec = synth.model_spec(64, 8, L, r)
    th = synth.init_params(spec, seed=0)
    sig, sigp = synth.random_configs(n, Ns, seed=17)
    ctx = tdo.Context(prob, spec, th, prec)
    ctx.set_sr_options(1e-10, 500)
    ctx.sr_step(dev(sig), dev(sigp), lr, shift)
    assert ctx.sr_report()[0] == 1          # converged
    delta = (th - ctx.get_params()) / lr
    g_ref, _, _, _ = E.grad_estimator(prob, spec, th, sig, sigp)
    O = E.jacobian(spec, th, sig, sigp, n)
    Oc = O - O.mean(axis=0, keepdims=True)
    Sd = (Oc.conj().T @ (Oc @ delta)).real / Ns + shift * delta
    res = np.linalg.norm(Sd - g_ref) / np.linalg.norm(g_ref)
    print(f"{prec} L={L} r={r}: relative residual {res:.3e}")
    assert res <= tol
