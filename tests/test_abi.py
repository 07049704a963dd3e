"""CPU checks of the C-ABI boundary: the shared library builds for sm_103a,
loads, and exports every symbol include/filterreg.h declares; host-only entry
points behave; nothing here launches a kernel."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "filterreg.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"FR_API\s+[\w\s\*]+?\b(fr_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import paper_1811_10136_gb300 as fr
    from paper_1811_10136_gb300 import build
    build.build()
    return fr.load()


def test_header_declares_the_binding_names():
    import paper_1811_10136_gb300 as fr
    assert declared_symbols() == sorted(fr.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_library_targets_sm_103a_only():
    # The build passes exactly one -gencode (compute_103a / sm_103a).
    from paper_1811_10136_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_host_only_entry_points(lib):
    import paper_1811_10136_gb300 as fr
    o = fr.options()
    assert (o.residual, o.blur, o.iters, o.storage, o.use_graph) == (0, 0, 30, 0, 1)
    assert abs(o.sigma_start - 0.02) < 1e-9 and abs(o.w - 0.1) < 1e-7
    assert lib.fr_status_string(0) == b"ok"
    assert lib.fr_status_string(4) == b"lattice capacity exceeded"
    with pytest.raises(TypeError):
        fr.options(no_such_option=1)


def test_null_arguments_rejected_without_gpu(lib):
    # Argument validation happens before any device work.
    assert lib.fr_ctx_create(0, None, None) == 1          # FR_EINVAL
    assert lib.fr_register_rigid(None, None, 0, None, None, 0, None, None, None) == 1
    assert lib.fr_ctx_kernel_launches(None) == 0
    assert lib.fr_register_articulated_batch(None, None, None, 1, None, None) == 1


def test_fault_injection_arguments(lib):
    import paper_1811_10136_gb300 as fr
    assert lib.fr_debug_fail_allocations(-1, 1) == 1      # FR_EINVAL
    assert lib.fr_debug_fail_allocations(0, -1) == 1
    with pytest.raises(fr.FilterRegError):
        fr.debug_fail_allocations(-1, 1)
    fr.debug_fail_allocations(3, 2)
    fr.debug_fail_allocations(0, 0)                        # clears


def test_no_device_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.fr_ctx_create(0, None, ctypes.byref(h)) == 3   # FR_ECUDA
    assert not h.value
