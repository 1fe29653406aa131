"""Helpers for the GPU parity tests: build contexts from the shared seeded inputs and compare with the oracle."""
import numpy as np

from paper_2502_20723_gb300 import synth


def problem(kind: str, n: int, **kw):
    """"ising": the dissipative Ising chain; "xyz": the XYZ chain; "heis": the XYZ chain with the fields of the
    Heisenberg figures (J = (1.4, 2.0, 1.0), B = (-1.0, 0.5, 0.1)); "ising2d": the 2D Ising model on a
    2 x (n / 2) torus."""
    if kind == "ising":
        return synth.ising_chain(n, **kw)
    if kind == "heis":
        return synth.xyz_chain(n, Jx=1.4, Jy=2.0, Jz=1.0, Bx=-1.0, By=0.5, Bz=0.1, **kw)
    if kind == "ising2d":
        return synth.ising_2d(2, n // 2, **kw)
    return synth.xyz_chain(n, **kw)


def wrap_phase(d):
    """Imaginary parts compared modulo 2 pi."""
    return np.angle(np.exp(1j * np.asarray(d)))


def logrho_err(gpu_f2: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """|log rho_gpu - log rho_ref| with the phase difference wrapped to (-pi, pi]."""
    dr = gpu_f2[:, 0].astype(np.float64) - ref.real
    di = wrap_phase(gpu_f2[:, 1].astype(np.float64) - ref.imag)
    return np.hypot(dr, di)


def block_errors(spec: dict, g: np.ndarray, ref: np.ndarray) -> dict:
    """Per named parameter block (synth.param_shapes order): max |g - ref| / max |ref| over the block, so
    that a wrong small block (the head, the embedding table, one bias) shows even when the gradient's
    norm is dominated by the large weight matrices."""
    out, off = {}, 0
    for name, shape in synth.param_shapes(spec):
        n = int(np.prod(shape))
        gb, rb = np.asarray(g[off:off + n]), np.asarray(ref[off:off + n])
        out[name] = float(np.abs(gb - rb).max() / max(np.abs(rb).max(), 1e-300))
        off += n
    return out
