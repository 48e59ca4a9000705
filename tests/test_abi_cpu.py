"""Host-side checks of the C ABI that need no GPU: the library builds, loads,
exports every function include/kirin.h declares, and refuses bad arguments
without touching a device."""
import ctypes

import pytest

from paper_0707_0438_gb300 import abi, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return abi.lib()


def test_header_declares_the_paper_calls():
    names = abi.header_functions()
    # the GRAPE-6 style sequence of Appendix A
    for n in ("kirin_init", "kirin_finalize", "kirin_query", "kirin_set_j_particles", "kirin_predict",
              "kirin_compute_forces", "kirin_get_acc_jerk_pot", "kirin_energy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    names = abi.header_functions()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding declares a signature for each of them
    assert sorted(abi._SIGS) == names


def test_strerror_names_every_code(lib):
    for code in (abi.KIRIN_OK, abi.KIRIN_EINVAL, abi.KIRIN_ENOMEM, abi.KIRIN_ECUDA, abi.KIRIN_ENONFINITE,
                 abi.KIRIN_ETIMEOUT, abi.KIRIN_ESTATE, abi.KIRIN_EEXCHANGE):
        s = lib.kirin_strerror(code).decode()
        assert s and s != "unknown error"
    assert lib.kirin_strerror(-99).decode() == "unknown error"


def test_init_rejects_bad_arguments_before_any_device_call(lib):
    h = ctypes.c_void_p()
    ok_cfg = abi.kirin_config(0.01, 1.0, 0.0, abi.KIRIN_MIXED, 0, None)
    assert lib.kirin_init(None, 16, ctypes.byref(ok_cfg)) == abi.KIRIN_EINVAL
    assert lib.kirin_init(ctypes.byref(h), 16, None) == abi.KIRIN_EINVAL
    assert lib.kirin_init(ctypes.byref(h), 0, ctypes.byref(ok_cfg)) == abi.KIRIN_EINVAL
    bad_eps = abi.kirin_config(-1.0, 1.0, 0.0, abi.KIRIN_MIXED, 0, None)
    assert lib.kirin_init(ctypes.byref(h), 16, ctypes.byref(bad_eps)) == abi.KIRIN_EINVAL
    bad_prec = abi.kirin_config(0.01, 1.0, 0.0, 7, 0, None)
    assert lib.kirin_init(ctypes.byref(h), 16, ctypes.byref(bad_prec)) == abi.KIRIN_EINVAL
    bad_rmin = abi.kirin_config(0.01, 1.0, float("nan"), abi.KIRIN_MIXED, 0, None)
    assert lib.kirin_init(ctypes.byref(h), 16, ctypes.byref(bad_rmin)) == abi.KIRIN_EINVAL


def test_null_context_is_rejected(lib):
    assert lib.kirin_finalize(None) == abi.KIRIN_OK
    assert lib.kirin_compute_forces(None, 1, None) == abi.KIRIN_EINVAL
    assert lib.kirin_get_acc_jerk_pot(None, None, None, None) == abi.KIRIN_EINVAL
    assert lib.kirin_predict(None, 0.0) == abi.KIRIN_EINVAL
    assert lib.kirin_sync(None) == abi.KIRIN_EINVAL
    assert lib.kirin_batch_leapfrog(None, 0.1, 1, 0) == abi.KIRIN_EINVAL
    assert lib.kirin_batch_set_launch(None, 1, 0) == abi.KIRIN_EINVAL
    assert lib.kirin_batch_set_state_dev(None, None, None, None) == abi.KIRIN_EINVAL
    assert lib.kirin_batch_get_state_dev(None, None, None) == abi.KIRIN_EINVAL
    assert lib.kirin_batch_accel_dev(None, None) == abi.KIRIN_EINVAL
    assert lib.kirin_batch_get_launch(None, None, None, None) == abi.KIRIN_EINVAL
    assert lib.kirin_hermite_init(None, 0.0, 0.01, 2.0 ** -20, 2.0 ** -3) == abi.KIRIN_EINVAL
    assert lib.kirin_hermite_shared_run(None, 0.1, 1) == abi.KIRIN_EINVAL
    assert lib.kirin_set_shared_persistent(None, 1) == abi.KIRIN_EINVAL
    assert lib.kirin_get_shared_persistent(None, None) == abi.KIRIN_EINVAL
    assert lib.kirin_set_tracing(None, 1) == abi.KIRIN_EINVAL
    assert lib.kirin_get_trace(None, None, None) == abi.KIRIN_EINVAL
    assert lib.kirin_selftest_arrival_timeout(None, 1000) == abi.KIRIN_EINVAL
    assert lib.kirin_selftest_wait_timeout(None, 1000) == abi.KIRIN_EINVAL
    assert lib.kirin_last_error(None).decode() == "no context"


def test_batch_create_validates_offsets(lib):
    b = ctypes.c_void_p()
    off = (ctypes.c_int64 * 3)(0, 10, 5)  # decreasing
    eps = (ctypes.c_double * 2)(0.1, 0.1)
    assert lib.kirin_batch_create(ctypes.byref(b), 2, off, eps, 1.0, 0, None) == abi.KIRIN_EINVAL
    off2 = (ctypes.c_int64 * 3)(1, 10, 20)  # does not start at 0
    assert lib.kirin_batch_create(ctypes.byref(b), 2, off2, eps, 1.0, 0, None) == abi.KIRIN_EINVAL


def test_no_gpu_means_a_clean_error_not_a_crash(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    cfg = abi.kirin_config(0.01, 1.0, 0.0, abi.KIRIN_MIXED, 0, None)
    assert lib.kirin_init(ctypes.byref(h), 16, ctypes.byref(cfg)) == abi.KIRIN_ECUDA
    with pytest.raises(abi.KirinError):
        abi.Kirin(16, 0.01)
