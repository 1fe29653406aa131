"""Helpers for the GPU parity tests: build contexts from the shared seeded inputs and compare with the oracle."""
import numpy as np

from paper_2502_20723_gb300 import synth


def problem(kind: str, n: int, **kw):
    return synth.ising_chain(n, **kw) if kind == "ising" else synth.xyz_chain(n, **kw)


def wrap_phase(d):
    """Imaginary parts compared modulo 2 pi."""
    return np.angle(np.exp(1j * np.asarray(d)))


def logrho_err(gpu_f2: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """|log rho_gpu - log rho_ref| with the phase difference wrapped to (-pi, pi]."""
    dr = gpu_f2[:, 0].astype(np.float64) - ref.real
    di = wrap_phase(gpu_f2[:, 1].astype(np.float64) - ref.imag)
    return np.hypot(dr, di)
