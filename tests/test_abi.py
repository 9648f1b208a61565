"""The C ABI: the library builds and loads, exports every symbol that
include/*.h declares, the Python structures match the C layout, and argument
errors are reported as statuses (no GPU needed)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2401_08260_gb300 import build, slk
    build.build()
    return slk.load()


def _declared_functions():
    names = set()
    for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(slk_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    from paper_2401_08260_gb300 import slk
    declared = _declared_functions()
    assert "slk_plan_create" in declared and "slk_sum" in declared and "slk_grad" in declared
    out = subprocess.run(["nm", "-D", "--defined-only", slk.LIB_PATH], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (slk_[a-z0-9_]+)", out))
    missing = [n for n in declared if n not in exported]
    assert not missing, missing
    for n in declared:
        assert hasattr(lib, n)


def test_struct_layout_matches_header(tmp_path):
    """Compile a probe against include/slk.h with gcc and compare sizes and offsets."""
    from paper_2401_08260_gb300 import slk
    src = tmp_path / "probe.c"
    structs = [("slk_plan_desc", slk.PlanDesc), ("slk_plan_info", slk.PlanInfo), ("slk_kernel_time", slk.KernelTime),
               ("slk_serve_desc", slk.ServeDesc), ("slk_request", slk.RequestDesc), ("slk_result", slk.RequestResult),
               ("slk_rff_desc", slk.RffDesc)]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "slk_serve.h"', "int main(void){"]
    expect = []
    for cname, py in structs:
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        expect.append(ctypes.sizeof(py))
        for f, _ in py._fields_:
            lines.append(f'printf("%zu\\n", offsetof({cname}, {f}));')
            expect.append(getattr(py, f).offset)
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert vals == expect


def test_status_strings_and_version(lib):
    assert lib.slk_version() == 1
    assert lib.slk_status_string(0) == b"ok"
    assert lib.slk_status_string(4) == b"accuracy target cannot be met"
    assert lib.slk_status_string(99) == b"unknown status"


def test_invalid_descriptors_are_rejected_without_a_device(lib):
    from paper_2401_08260_gb300 import slk
    h = ctypes.c_void_p()
    buf = (ctypes.c_float * 64)()
    assert lib.slk_plan_create(ctypes.byref(h), None, buf, 4, 4, buf, None) == 1
    assert b"descriptor" in lib.slk_last_error()
    desc = slk.PlanDesc()
    desc.kernel, desc.precision, desc.param, desc.d, desc.P = 0, 1, 1.0, 4, 8
    for field, bad in [("kernel", 7), ("precision", 9), ("d", 0), ("P", 0), ("param", -1.0), ("n_coeff", 3),
                       ("method", 5), ("tol", -1.0)]:
        d2 = slk.PlanDesc.from_buffer_copy(desc)
        setattr(d2, field, bad)
        assert lib.slk_plan_create(ctypes.byref(h), ctypes.byref(d2), buf, 4, 4, buf, None) == 1, field
    # N < 1 and ldx < d
    assert lib.slk_plan_create(ctypes.byref(h), ctypes.byref(desc), buf, 0, 4, buf, None) == 1
    assert lib.slk_plan_create(ctypes.byref(h), ctypes.byref(desc), buf, 4, 3, buf, None) == 1
    # NULL plan handles
    assert lib.slk_sum(None, buf, 1, 4, buf, None) == 1
    assert lib.slk_grad(None, buf, 1, 4, None, buf, 4, None) == 1
    assert lib.slk_sum_derivs(None, buf, 1, 4, buf, buf, 1, None) == 1
    assert lib.slk_grad_derivs(None, buf, 1, 1, None, buf, 4, None) == 1
    assert lib.slk_plan_sync(None) == 1
    assert lib.slk_plan_destroy(None) == 0


def test_python_binding_fails_loudly_without_library(tmp_path):
    from paper_2401_08260_gb300 import slk
    with pytest.raises(slk.SlkError):
        slk._lib_saved = slk._lib
        try:
            slk._lib = None
            slk.load(str(tmp_path / "nope.so"))
        finally:
            slk._lib = slk._lib_saved


def test_request_bytes_estimate_is_monotone(lib):
    """The serving admission estimate (host-only) grows with every size and rejects bad input."""
    from paper_2401_08260_gb300 import slk
    base = dict(kernel="negdist", param=0.0, d=64, P=128, precision="f32")
    b0 = slk.request_bytes(slk.make_desc(**base), 10000, 10000)
    assert b0 > 0
    for key, val in [("d", 128), ("P", 256)]:
        assert slk.request_bytes(slk.make_desc(**dict(base, **{key: val})), 10000, 10000) > b0
    assert slk.request_bytes(slk.make_desc(**base), 20000, 10000) > b0
    # peak over phases (plan build, then plan + sum): non-decreasing in M, growing once the sum dominates
    assert slk.request_bytes(slk.make_desc(**base), 10000, 20000) >= b0
    assert slk.request_bytes(slk.make_desc(**base), 10000, 10 ** 6) > b0
    assert slk.request_bytes(slk.make_desc(**base), -1, 10) == -1
    # a cached plan needs only the target side
    assert slk.request_bytes(slk.make_desc(**base), 0, 10000) < b0


def test_serve_calls_report_errors_without_a_device(lib):
    from paper_2401_08260_gb300 import slk
    sl = slk._serve_lib()
    res = slk.RequestResult()
    assert sl.slk_serve_poll(None, 1, 0, ctypes.byref(res)) == 1
    assert sl.slk_serve_submit(None, None, None) == 1
    assert sl.slk_serve_destroy(None) == 0
