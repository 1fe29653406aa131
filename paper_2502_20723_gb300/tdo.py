"""Python binding of libtdo.so (include/tdo.h): argument marshalling only.

Every computation runs in the library's CUDA kernels; this module converts problem statements and
model specs to the C structs, passes device (torch CUDA tensors) or host (numpy arrays) pointers, and
raises TdoError on a non-zero status.  There is no CPU fallback: if libtdo.so is missing or a CUDA
device is absent the calls fail loudly.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libtdo.so")

TDO_EMBED_TOKEN, TDO_EMBED_CONV = 0, 1
TDO_FP32, TDO_BF16, TDO_FP16, TDO_FP8 = 0, 1, 2, 3
PRECISIONS = {"fp32": TDO_FP32, "bf16": TDO_BF16, "fp16": TDO_FP16, "fp8": TDO_FP8}
STATUS = {0: "TDO_OK", -1: "TDO_EINVAL", -2: "TDO_ENOMEM", -3: "TDO_ECUDA", -4: "TDO_ENUMERIC",
          -5: "TDO_ETIMEOUT", -6: "TDO_EUNSUPPORTED"}

EXPORTS = ["tdo_model_num_params", "tdo_create", "tdo_destroy", "tdo_num_params", "tdo_max_connections",
           "tdo_set_params", "tdo_get_params", "tdo_log_rho", "tdo_log_rho_vjp", "tdo_jacobian",
           "tdo_connections", "tdo_local_estimator", "tdo_local_estimator_noalloc", "tdo_sample", "tdo_grad", "tdo_sr_solve", "tdo_set_sr_options", "tdo_sr_step",
           "tdo_timing", "tdo_timing_read", "tdo_sr_info", "tdo_sr_report", "tdo_set_sr_product", "tdo_sr_product_shape", "tdo_sr_apply", "tdo_wait_selftest", "tdo_set_optimizer", "tdo_log_rho_ragged", "tdo_ragged_tuning", "tdo_measure_peak", "tdo_last_error", "tdo_sample_diag", "tdo_magnetisation",
           "tdo_purity", "tdo_schedule_value", "tdo_vmc_step", "tdo_set_step_graph", "tdo_step_graph_stats"]


class TdoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Problem(C.Structure):
    _fields_ = [("n_sites", C.c_int), ("n_terms", C.c_int), ("term_sites", C.POINTER(C.c_int)),
                ("term_paulis", C.c_char_p), ("term_coef", C.POINTER(C.c_double)), ("n_jumps", C.c_int),
                ("jump_site", C.POINTER(C.c_int)), ("jump_op", C.POINTER(C.c_double)),
                ("jump_rate", C.POINTER(C.c_double))]


class Model(C.Structure):
    _fields_ = [("embed", C.c_int), ("conv_channels", C.c_int), ("d_model", C.c_int), ("n_heads", C.c_int),
                ("n_layers", C.c_int), ("mlp_ratio", C.c_int), ("precision", C.c_int)]


class Schedule(C.Structure):
    """tdo_schedule: learning-rate and SR-shift schedules (defaults: the paper's values)."""
    _fields_ = [("eta0", C.c_double), ("i_switch", C.c_longlong), ("i_decay", C.c_longlong), ("alpha", C.c_double),
                ("lambda0", C.c_double), ("i_switch_sr", C.c_longlong), ("i_decay_sr", C.c_longlong),
                ("alpha_sr", C.c_double)]

    def __init__(self, eta0=0.0061, i_switch=30000, i_decay=40000, alpha=0.001, lambda0=0.004, i_switch_sr=30000,
                 i_decay_sr=40000, alpha_sr=0.01):
        super().__init__(eta0, i_switch, i_decay, alpha, lambda0, i_switch_sr, i_decay_sr, alpha_sr)


def measure_peak(kind: str = "fp32", stream=None) -> float:
    """tdo_measure_peak: measured FMA peak of the current device in TFLOP/s ("fp32" or "fp64")."""
    t = C.c_double()
    rc = lib().tdo_measure_peak(0 if kind == "fp32" else 1, stream, C.byref(t))
    if rc != 0:
        raise TdoError(rc, "tdo_measure_peak failed")
    return t.value


def schedule_value(step: int, v0: float, i_switch: int, i_decay: int, alpha: float) -> float:
    """tdo_schedule_value: v0 before i_switch, then cosine decay to a floor alpha v0."""
    return lib().tdo_schedule_value(step, v0, i_switch, i_decay, alpha)


_lib = None


def lib() -> C.CDLL:
    """Load libtdo.so (built by paper_2502_20723_gb300.build); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"libtdo.so not found at {_LIB_PATH}: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(_LIB_PATH)
        vp, sz, u64, i32 = C.c_void_p, C.c_size_t, C.c_uint64, C.c_int
        dp = C.POINTER(C.c_double)
        L.tdo_model_num_params.argtypes = [C.POINTER(Model)]
        L.tdo_model_num_params.restype = sz
        L.tdo_create.argtypes = [C.POINTER(Problem), C.POINTER(Model), vp, sz, vp, C.POINTER(vp)]
        L.tdo_destroy.argtypes = [vp]
        L.tdo_num_params.argtypes = [vp]
        L.tdo_num_params.restype = sz
        L.tdo_max_connections.argtypes = [vp]
        L.tdo_max_connections.restype = i32
        L.tdo_set_params.argtypes = [vp, vp]
        L.tdo_get_params.argtypes = [vp, vp]
        L.tdo_log_rho.argtypes = [vp, vp, vp, sz, vp]
        L.tdo_log_rho_ragged.argtypes = [vp, vp, vp, vp, sz, vp]
        L.tdo_ragged_tuning.argtypes = [vp, C.c_uint32, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
        L.tdo_log_rho_vjp.argtypes = [vp, vp, vp, sz, vp, vp]
        L.tdo_jacobian.argtypes = [vp, vp, vp, sz, vp]
        L.tdo_connections.argtypes = [vp, vp, vp, sz, vp, vp, vp, vp]
        L.tdo_local_estimator.argtypes = [vp, vp, vp, sz, vp, dp, dp]
        L.tdo_local_estimator_noalloc.argtypes = [vp, vp, vp, sz, vp, dp, dp]
        L.tdo_sample.argtypes = [vp, sz, sz, u64, u64, vp, vp, vp, vp, C.POINTER(u64)]
        L.tdo_sample_diag.argtypes = [vp, sz, sz, u64, u64, vp, vp, C.POINTER(u64)]
        L.tdo_magnetisation.argtypes = [vp, vp, sz, vp, dp, vp]
        L.tdo_purity.argtypes = [vp, vp, vp, sz, dp, dp]
        L.tdo_schedule_value.argtypes = [C.c_longlong, C.c_double, C.c_longlong, C.c_longlong, C.c_double]
        L.tdo_schedule_value.restype = C.c_double
        L.tdo_vmc_step.argtypes = [vp, vp, vp, sz, sz, u64, C.POINTER(u64), C.c_longlong, C.POINTER(Schedule), dp]
        L.tdo_set_step_graph.argtypes = [vp, i32]
        L.tdo_step_graph_stats.argtypes = [vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
        L.tdo_grad.argtypes = [vp, vp, vp, sz, vp, dp, vp]
        L.tdo_sr_solve.argtypes = [vp, vp, sz, vp, C.c_double, C.c_double, i32, vp, C.POINTER(i32), dp]
        L.tdo_sr_step.argtypes = [vp, vp, vp, sz, C.c_double, C.c_double, dp]
        L.tdo_set_sr_options.argtypes = [vp, C.c_double, i32]
        L.tdo_set_optimizer.argtypes = [vp, i32, C.c_double, C.c_double, C.c_double]
        L.tdo_timing.argtypes = [vp, i32]
        L.tdo_timing_read.argtypes = [vp, C.c_char_p, dp, C.POINTER(C.c_longlong)]
        L.tdo_sr_info.argtypes = [vp, C.POINTER(i32), dp]
        L.tdo_sr_report.argtypes = [vp, C.POINTER(i32), dp, C.POINTER(i32)]
        L.tdo_set_sr_product.argtypes = [vp, i32]
        L.tdo_sr_product_shape.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
        L.tdo_sr_apply.argtypes = [vp, vp, sz, sz, vp, C.c_double, vp]
        L.tdo_wait_selftest.argtypes = [vp, C.c_longlong]
        L.tdo_measure_peak.argtypes = [i32, vp, dp]
        L.tdo_last_error.argtypes = [vp]
        L.tdo_last_error.restype = C.c_char_p
        for name in EXPORTS:
            if name not in ("tdo_model_num_params", "tdo_num_params", "tdo_max_connections", "tdo_last_error",
                            "tdo_schedule_value"):
                getattr(L, name).restype = i32
        _lib = L
    return _lib


def _ptr(x):
    """Raw pointer of a torch tensor (device or host) or a contiguous numpy array; None -> NULL."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"], "arrays must be C-contiguous"
        return x.ctypes.data
    assert x.is_contiguous(), "tensors must be contiguous"
    return x.data_ptr()


def make_model(spec: dict, precision: str = "fp32") -> Model:
    return Model(TDO_EMBED_TOKEN if spec.get("embed", "token") == "token" else TDO_EMBED_CONV,
                 int(spec.get("conv_channels", 0)), int(spec["d_model"]), int(spec["n_heads"]),
                 int(spec["n_layers"]), int(spec.get("mlp_ratio", 0)),
                 PRECISIONS[precision])


def model_num_params(spec: dict) -> int:
    m = make_model(spec)
    return int(lib().tdo_model_num_params(C.byref(m)))


class _ProblemArrays:
    """Keeps the ctypes arrays of a problem statement alive while the C struct points at them."""

    def __init__(self, problem: dict):
        terms = problem["terms"]
        jumps = problem["jumps"]
        sites, paulis, coef = [], [], []
        for c, ops in terms:
            ops = list(ops)
            assert 1 <= len(ops) <= 2, "Pauli strings on one or two sites"
            s = [ops[0][0], ops[1][0] if len(ops) > 1 else -1]
            p = ops[0][1] + (ops[1][1] if len(ops) > 1 else "I")
            sites += s
            paulis.append(p)
            coef.append(float(c))
        self.sites = np.asarray(sites or [0], dtype=np.int32)
        self.paulis = ("".join(paulis) or "II").encode()
        self.coef = np.asarray(coef or [0.0], dtype=np.float64)
        self.jsite = np.asarray([j[0] for j in jumps] or [0], dtype=np.int32)
        ops = np.zeros((max(len(jumps), 1), 2, 2, 2), dtype=np.float64)
        for q, (_, Lm, _) in enumerate(jumps):
            Lm = np.asarray(Lm, dtype=np.complex128)
            ops[q, :, :, 0] = Lm.real
            ops[q, :, :, 1] = Lm.imag
        self.jop = np.ascontiguousarray(ops)
        self.jrate = np.asarray([float(j[2]) for j in jumps] or [0.0], dtype=np.float64)
        ip, dpp = C.POINTER(C.c_int), C.POINTER(C.c_double)
        self.struct = Problem(int(problem["n_sites"]), len(terms), self.sites.ctypes.data_as(ip), self.paulis,
                              self.coef.ctypes.data_as(dpp), len(jumps), self.jsite.ctypes.data_as(ip),
                              self.jop.ctypes.data_as(dpp), self.jrate.ctypes.data_as(dpp))


class Context:
    """One tdo_ctx: a problem, a transformer model and its parameters on the current CUDA device."""

    def __init__(self, problem: dict, spec: dict, theta, precision: str = "fp32", stream=None):
        L = lib()
        self._pa = _ProblemArrays(problem)
        self._model = make_model(spec, precision)
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
        h = C.c_void_p()
        st = 0 if stream is None else int(stream)
        self.n_sites = int(problem["n_sites"])
        rc = L.tdo_create(C.byref(self._pa.struct), C.byref(self._model), th.ctypes.data, th.size, st, C.byref(h))
        if rc != 0:
            raise TdoError(rc, L.tdo_last_error(None).decode())
        self.h = h
        self.P = int(L.tdo_num_params(h))
        self.M = int(L.tdo_max_connections(h))

    def _chk(self, rc):
        if rc != 0:
            raise TdoError(rc, lib().tdo_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib().tdo_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- parameters
    def set_params(self, theta):
        self._chk(lib().tdo_set_params(self.h, _ptr(theta)))

    def get_params(self, out=None):
        out = np.empty(self.P, np.float64) if out is None else out
        self._chk(lib().tdo_get_params(self.h, _ptr(out)))
        return out

    # -- calls (outputs allocated like the inputs: torch CUDA in -> torch CUDA out, numpy in -> numpy out)
    @staticmethod
    def _like(x, shape, dtype):
        if isinstance(x, np.ndarray):
            return np.empty(shape, dtype=dtype)
        import torch
        tdt = {np.float32: torch.float32, np.float64: torch.float64, np.uint32: torch.int32,
               np.int32: torch.int32}[dtype]
        return torch.empty(shape, dtype=tdt, device=x.device)

    def log_rho(self, sig, sigp, out=None):
        B = len(sig)
        out = self._like(sig, (B, 2), np.float32) if out is None else out
        self._chk(lib().tdo_log_rho(self.h, _ptr(sig), _ptr(sigp), B, _ptr(out)))
        return out

    def log_rho_ragged(self, n_sites, sig, sigp, out=None):
        """tdo_log_rho_ragged: log rho of configurations of chains of lengths n_sites[b] (int32)."""
        B = len(sig)
        out = self._like(sig, (B, 2), np.float32) if out is None else out
        self._chk(lib().tdo_log_rho_ragged(self.h, _ptr(n_sites), _ptr(sig), _ptr(sigp), B, _ptr(out)))
        return out

    def ragged_tuning(self, mix: int):
        """(CTAs per SM, descending order, dynamic schedule) kept by the autotuner for a mix of lengths."""
        a, b, d = C.c_int(), C.c_int(), C.c_int()
        self._chk(lib().tdo_ragged_tuning(self.h, mix, C.byref(a), C.byref(b), C.byref(d)))
        return a.value, b.value, d.value

    def log_rho_vjp(self, sig, sigp, cot, grad):
        self._chk(lib().tdo_log_rho_vjp(self.h, _ptr(sig), _ptr(sigp), len(sig), _ptr(cot), _ptr(grad)))
        return grad

    def jacobian(self, sig, sigp, out=None):
        B = len(sig)
        out = self._like(sig, (B, self.P, 2), np.float32) if out is None else out
        self._chk(lib().tdo_jacobian(self.h, _ptr(sig), _ptr(sigp), B, _ptr(out)))
        return out

    def connections(self, sig, sigp):
        Ns, M = len(sig), self.M
        cnt = self._like(sig, (Ns,), np.int32)
        cs = self._like(sig, (Ns, M), np.uint32)
        cp = self._like(sig, (Ns, M), np.uint32)
        cc = self._like(sig, (Ns, M, 2), np.float32)
        self._chk(lib().tdo_connections(self.h, _ptr(sig), _ptr(sigp), Ns, _ptr(cnt), _ptr(cs), _ptr(cp), _ptr(cc)))
        return cnt, cs, cp, cc

    def local_estimator(self, sig, sigp, lloc=None):
        Ns = len(sig)
        lloc = self._like(sig, (Ns, 2), np.float64) if lloc is None else lloc
        cost, se = C.c_double(), C.c_double()
        self._chk(lib().tdo_local_estimator(self.h, _ptr(sig), _ptr(sigp), Ns, _ptr(lloc), C.byref(cost), C.byref(se)))
        return lloc, cost.value, se.value

    def sample(self, sig, sigp, n_sweeps: int, seed: int, counter: int, samples=False):
        """Metropolis sweeps in place on the chains (sig, sigp); returns (accepted, samples or None)."""
        nc = len(sig)
        ss = sp = None
        if samples:
            ss = self._like(sig, (n_sweeps, nc), np.uint32)
            sp = self._like(sig, (n_sweeps, nc), np.uint32)
        acc = C.c_uint64()
        self._chk(lib().tdo_sample(self.h, nc, n_sweeps, seed, counter, _ptr(sig), _ptr(sigp), _ptr(ss), _ptr(sp),
                                   C.byref(acc)))
        return acc.value, ((ss, sp) if samples else None)

    def sample_diag(self, alpha, n_sweeps: int, seed: int, counter: int, samples=False):
        """Metropolis sweeps on |rho(alpha, alpha)| in place on the chains alpha; returns (accepted, samples
        [n_sweeps][chains] or None)."""
        nc = len(alpha)
        ss = self._like(alpha, (n_sweeps, nc), np.uint32) if samples else None
        acc = C.c_uint64()
        self._chk(lib().tdo_sample_diag(self.h, nc, n_sweeps, seed, counter, _ptr(alpha), _ptr(ss), C.byref(acc)))
        return acc.value, ss

    def magnetisation(self, alpha, local: bool = False):
        """(<sigma^x>, <sigma^y>, <sigma^z>) from samples alpha of |rho(alpha, alpha)|; returns (mag [3],
        mean sign, per-sample (s, A~x, A~y, A~z) as complex [Ns, 4] or None)."""
        mag = np.zeros(3)
        sm = C.c_double()
        loc = np.zeros((len(alpha), 8)) if local else None
        self._chk(lib().tdo_magnetisation(self.h, _ptr(alpha), len(alpha), mag.ctypes.data, C.byref(sm), _ptr(loc)))
        return mag, sm.value, (loc.view(np.complex128) if local else None)

    def purity(self, sig, sigp):
        """Tr(rho^2) / Tr(rho)^2 from samples of |rho|^2; returns (purity, standard error)."""
        pu, se = C.c_double(), C.c_double()
        self._chk(lib().tdo_purity(self.h, _ptr(sig), _ptr(sigp), len(sig), C.byref(pu), C.byref(se)))
        return pu.value, se.value

    def vmc_step(self, sig, sigp, n_sweeps: int, seed: int, counter: int, step: int, schedule=None):
        """Sweeps of the chains, then an SR step with the scheduled rate and shift; returns (cost, counter)."""
        ctr = C.c_uint64(counter)
        cost = C.c_double()
        sched = C.byref(schedule) if schedule is not None else None
        self._chk(lib().tdo_vmc_step(self.h, _ptr(sig), _ptr(sigp), len(sig), n_sweeps, seed, C.byref(ctr), step,
                                     sched, C.byref(cost)))
        return cost.value, ctr.value

    def set_step_graph(self, enable: bool):
        """tdo_set_step_graph: vmc_step records its whole step into a CUDA graph once and replays it."""
        self._chk(lib().tdo_set_step_graph(self.h, 1 if enable else 0))

    def step_graph_stats(self):
        """(recordings, launches) of the step graph (tdo_step_graph_stats)."""
        a, b = C.c_longlong(), C.c_longlong()
        self._chk(lib().tdo_step_graph_stats(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def grad(self, sig, sigp, grad=None, O=None):
        Ns = len(sig)
        grad = self._like(sig, (self.P,), np.float64) if grad is None else grad
        cost = C.c_double()
        self._chk(lib().tdo_grad(self.h, _ptr(sig), _ptr(sigp), Ns, _ptr(grad), C.byref(cost), _ptr(O)))
        return grad, cost.value

    def sr_solve(self, O, rhs, diag_shift: float, tol: float = 1e-10, max_iter: int = 1000, x=None):
        Ns = O.shape[0]
        x = self._like(rhs, (self.P,), np.float64) if x is None else x
        it, res = C.c_int(), C.c_double()
        self._chk(lib().tdo_sr_solve(self.h, _ptr(O), Ns, _ptr(rhs), float(diag_shift), float(tol), int(max_iter),
                                     _ptr(x), C.byref(it), C.byref(res)))
        return x, it.value, res.value

    def timing(self, enable: bool):
        self._chk(lib().tdo_timing(self.h, 1 if enable else 0))

    def timing_read(self, group: str = "all"):
        ms, n = C.c_double(), C.c_longlong()
        self._chk(lib().tdo_timing_read(self.h, group.encode(), C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def sr_info(self):
        it, res = C.c_int(), C.c_double()
        self._chk(lib().tdo_sr_info(self.h, C.byref(it), C.byref(res)))
        return it.value, res.value

    def sr_report(self):
        """(outcome, last p.S'p, restarts) of the last SR step's CG solve (tdo_sr_report)."""
        o, pap, r = C.c_int(), C.c_double(), C.c_int()
        self._chk(lib().tdo_sr_report(self.h, C.byref(o), C.byref(pap), C.byref(r)))
        return o.value, pap.value, r.value

    def set_sr_product(self, mode: str):
        """tdo_set_sr_product: "two_pass" (default), "one_pass" (thread-block clusters) or "grid" (one pass
        over the whole grid), the last two where the log-derivatives' storage allows it."""
        self._chk(lib().tdo_set_sr_product(self.h, {"two_pass": 0, "one_pass": 1, "grid": 2}[mode]))

    def sr_apply(self, O_pairs, v, shift: float, out=None):
        """tdo_sr_apply: (Re S + shift I) v for log-derivatives O given as BF16 pairs (a device int32 / uint32
        tensor [Ns][ldo], ldo >= P), v FP64 [P] on the device."""
        Ns, ldo = O_pairs.shape
        out = self._like(v, (self.P,), np.float64) if out is None else out
        self._chk(lib().tdo_sr_apply(self.h, _ptr(O_pairs), Ns, ldo, _ptr(v), float(shift), _ptr(out)))
        return out

    def sr_product_shape(self):
        """(product used: 0 two passes, 1 clusters, 2 grid; CTAs per cluster; clusters or CTAs) of the last SR
        step's products (tdo_sr_product_shape)."""
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        self._chk(lib().tdo_sr_product_shape(self.h, C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value

    def wait_selftest(self, spin_limit: int) -> int:
        """tdo_wait_selftest: status of a bounded device wait that nothing completes (TDO_ETIMEOUT = -5)."""
        return lib().tdo_wait_selftest(self.h, int(spin_limit))

    def set_optimizer(self, kind: str = "sgd", beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        """tdo_set_optimizer: "sgd" or "adam" on the SR direction (resets Adam's moments)."""
        self._chk(lib().tdo_set_optimizer(self.h, {"sgd": 0, "adam": 1}[kind], float(beta1), float(beta2), float(eps)))

    def set_sr_options(self, tol: float, max_iter: int):
        self._chk(lib().tdo_set_sr_options(self.h, float(tol), int(max_iter)))

    def sr_step(self, sig, sigp, lr: float, diag_shift: float) -> float:
        cost = C.c_double()
        self._chk(lib().tdo_sr_step(self.h, _ptr(sig), _ptr(sigp), len(sig), float(lr), float(diag_shift),
                                    C.byref(cost)))
        return cost.value


def log_rho_autograd():
    """torch.autograd.Function over tdo_log_rho / tdo_log_rho_vjp: y = (Re, Im) log rho [B, 2] as a
    differentiable function of theta (FP64 CUDA tensor)."""
    import torch

    class LogRho(torch.autograd.Function):
        @staticmethod
        def forward(ctx, theta, sig, sigp, context):
            context.set_params(theta.detach().contiguous())
            ctx.save_for_backward(sig, sigp)
            ctx.context = context
            return context.log_rho(sig, sigp)

        @staticmethod
        def backward(ctx, g):
            sig, sigp = ctx.saved_tensors
            # d L = sum_b g0 dRe + g1 dIm = Re((g0 - i g1) d log rho)
            cot = torch.stack([g[:, 0], -g[:, 1]], dim=1).float().contiguous()
            grad = torch.zeros(ctx.context.P, dtype=torch.float64, device=g.device)
            ctx.context.log_rho_vjp(sig, sigp, cot, grad)
            return grad, None, None, None

    return LogRho
