"""CPU-side checks of the C ABI: the library loads and exports every function include/tdo.h declares,
and the pure host entry points (no GPU needed) behave."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tdo.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tdo_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libtdo():
    from paper_2502_20723_gb300 import build, tdo
    build.build()
    return tdo.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("tdo_create", "tdo_log_rho", "tdo_local_estimator", "tdo_sample", "tdo_grad", "tdo_sr_step"):
        assert n in names


def test_library_exports_every_declared_symbol(libtdo):
    for name in _declared():
        assert hasattr(libtdo, name), name


def test_binding_lists_every_export():
    from paper_2502_20723_gb300 import tdo
    assert sorted(tdo.EXPORTS) == _declared()


def test_model_num_params_matches_shapes(libtdo):
    from paper_2502_20723_gb300 import synth, tdo
    for spec in (synth.model_spec(64, 8, 4, 4), synth.model_spec(16, 2, 1, 0),
                 synth.model_spec(32, 4, 2, 0, embed="conv", conv_channels=5)):
        assert tdo.model_num_params(spec) == synth.num_params(spec)
    bad = tdo.Model(0, 0, 48, 8, 4, 4, 0)   # d_model 48 unsupported
    assert libtdo.tdo_model_num_params(ctypes.byref(bad)) == 0


def test_create_without_device_fails_cleanly(libtdo):
    """Without a GPU, tdo_create must return an error status (never crash, never fall back to the CPU)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2502_20723_gb300 import synth, tdo
    spec = synth.model_spec(16, 2, 1, 0)
    with pytest.raises(tdo.TdoError):
        tdo.Context(synth.ising_chain(4), spec, synth.init_params(spec))


def test_null_context_is_rejected_without_a_device(libtdo):
    """Entry points given no context return TDO_EINVAL before touching CUDA (pure host checks)."""
    from paper_2502_20723_gb300 import tdo
    einval = -1
    assert [k for k, v in tdo.STATUS.items() if v == "TDO_EINVAL"] == [einval]
    u64 = ctypes.c_uint64(0)
    d = ctypes.c_double(0.0)
    mag = (ctypes.c_double * 3)()
    assert libtdo.tdo_sample(None, 4, 1, 0, 0, None, None, None, None, None) == einval
    assert libtdo.tdo_sample_diag(None, 4, 1, 0, 0, None, None, None) == einval
    assert libtdo.tdo_magnetisation(None, None, 4, mag, None, None) == einval
    assert libtdo.tdo_purity(None, None, None, 4, ctypes.byref(d), None) == einval
    assert libtdo.tdo_vmc_step(None, None, None, 4, 1, 0, ctypes.byref(u64), 0, None, None) == einval
    assert libtdo.tdo_sr_step(None, None, None, 4, 0.1, 0.1, None) == einval
    assert libtdo.tdo_local_estimator_noalloc(None, None, None, 4, None, None, None) == einval
    assert libtdo.tdo_sr_report(None, None, None, None) == einval
    assert libtdo.tdo_set_sr_product(None, 0) == einval
    assert libtdo.tdo_sr_product_shape(None, None, None, None) == einval
    assert libtdo.tdo_sr_apply(None, None, 4, 4, None, ctypes.c_double(0.1), None) == einval
    assert libtdo.tdo_wait_selftest(None, 16) == einval
    assert libtdo.tdo_set_step_graph(None, 1) == einval
    assert libtdo.tdo_step_graph_stats(None, None, None) == einval
    assert libtdo.tdo_set_optimizer(None, 1, 0.9, 0.999, 1e-8) == einval
    assert libtdo.tdo_log_rho_ragged(None, None, None, None, 4, None) == einval
    assert libtdo.tdo_ragged_tuning(None, 1, None, None, None) == einval
    assert libtdo.tdo_measure_peak(2, None, ctypes.byref(d)) == einval
    assert libtdo.tdo_measure_peak(0, None, None) == einval
