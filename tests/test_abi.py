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


STRUCTS = ["fr_options", "fr_report", "fr_profile", "fr_kintree", "fr_articulated_item", "fr_batch_item",
           "fr_tune_params", "fr_request", "fr_result"]


def test_struct_layouts_match_the_header(tmp_path):
    # A probe compiled against include/filterreg.h prints every field's offset
    # and every struct's size; the ctypes mirrors of the binding must agree.
    import shutil
    import subprocess
    import paper_1811_10136_gb300 as fr
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "filterreg.h"', 'int main(void) {']
    for name in STRUCTS:
        lines.append(f'    printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in getattr(fr, name)._fields_:
            lines.append(f'    printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ['    return 0;', '}']
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "probe"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in filter(None, out):
        name, field, value = line.split()
        got[(name, field)] = int(value)
    for name in STRUCTS:
        cls = getattr(fr, name)
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)


def test_batch_items_marshalled_by_field():
    # The binding fills fr_batch_item through a numpy record view: every
    # field of every item lands where the C struct has it.
    import numpy as np
    import paper_1811_10136_gb300 as fr
    ctx = fr.Context.__new__(fr.Context)   # marshalling only: no device needed
    pairs = [(np.ones((5 + b, 4), np.float32), np.ones((7 + b, 4), np.float32),
              np.ones((7 + b, 4), np.float32) if b % 2 else None) for b in range(4)]
    o = fr.options(sigma_start=0.04, sigma_end=0.01, w=0.2)
    T0s = [np.arange(16.0).reshape(4, 4) + b for b in range(4)]
    items, keep = ctx._batch_items(pairs, [(0.03, 0.02)] * 4, [0.1, 0.2, 0.3, 0.4], T0s, True, o)
    for b in range(4):
        it = items[b]
        assert (it.M, it.N) == (5 + b, 7 + b)
        assert it.d_X == keep[b][0].ctypes.data and it.d_Y == keep[b][1].ctypes.data
        assert (it.d_Yn or 0) == (keep[b][2].ctypes.data if keep[b][2] is not None else 0)
        assert it.sigma_start == np.float32(0.03) and it.sigma_end == np.float32(0.02)
        assert it.w == np.float32(0.1 * (b + 1))
        assert list(it.T) == list(T0s[b].ravel())
    items, _ = ctx._batch_items(pairs, None, None, None, True, o)
    for b in range(4):
        it = items[b]
        assert it.sigma_start == np.float32(0.04) and it.w == np.float32(0.2)
        assert list(it.T) == list(np.eye(4).ravel())
    ro = np.ones((3, 4), np.float32)
    ro.setflags(write=False)
    assert fr._host_ptr(ro) == ro.ctypes.data
