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
