"""The C-ABI library loads and exports every entry point its header declares (no GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2601_16637_gb300 import binding as b
from paper_2601_16637_gb300 import build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "sbd.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(sbd_[a-z_0-9]+)\s*\(", text))
    return sorted(n for n in names if not n.endswith("_fn"))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return b.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(b._SIGNATURES) == set(names)


def test_struct_layouts_match_header():
    # sbd_options: double, int, int, size_t, double, int, int, fn, fn, void*, int (+4), double, int, int
    assert ctypes.sizeof(b.sbd_options) == 8 + 4 + 4 + 8 + 8 + 4 + 4 + 8 + 8 + 8 + 4 + 4 + 8 + 4 + 4
    assert ctypes.sizeof(b.sbd_report) == 7 * 4 + 4 + 4 * 8  # 7 ints, padding, 4 doubles


def test_struct_layouts_match_the_compiled_header(tmp_path):
    """sizeof and every field offset of the header's structs, as the C compiler lays them out, equal
    the binding's ctypes mirrors."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"sbd_options": b.sbd_options, "sbd_report": b.sbd_report,
               "sbd_engine_options": b.sbd_engine_options, "sbd_job_result": b.sbd_job_result,
               "sbd_engine_stats": b.sbd_engine_stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sbd.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.split("\n") if l)
    for name, cls in structs.items():
        assert int(out[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(out[f"{name}.{f}"]) == getattr(cls, f).offset, f"{name}.{f}"


def test_engine_defaults_and_argument_errors_need_no_gpu(lib):
    o = b.sbd_engine_default_options()
    assert (o.max_slots, o.max_subspace, o.max_iter, o.max_norb, o.max_strings) == (64, 12, 200, 64, 20000)
    assert o.rows_per_item == 0 and o.delta == 1e-4 and o.hbm_budget_bytes == 0
    out = ctypes.c_void_p()
    bad = b.sbd_engine_default_options()
    bad.max_subspace = 33
    assert lib.sbd_engine_create(ctypes.byref(out), ctypes.byref(bad), None) == -1
    bad = b.sbd_engine_default_options()
    bad.rows_per_item = 3
    assert lib.sbd_engine_create(ctypes.byref(out), ctypes.byref(bad), None) == -1
    # schedule: 0 fair share by cost (default), 1 lockstep; anything else is refused
    assert o.schedule == b.SCHEDULE["fair"] == 0 and b.SCHEDULE["lockstep"] == 1
    bad = b.sbd_engine_default_options()
    bad.schedule = 2
    assert lib.sbd_engine_create(ctypes.byref(out), ctypes.byref(bad), None) == -1
    with pytest.raises(ValueError):
        b.Engine(schedule="round-robin")
    assert lib.sbd_engine_create(None, None, None) == -1
    assert lib.sbd_engine_destroy(None) == -1
    assert lib.sbd_engine_step(None, None) == -1
    assert lib.sbd_engine_run(None) == -1
    r = b.sbd_job_result()
    assert lib.sbd_engine_result(None, 0, ctypes.byref(r)) == -1
    assert lib.sbd_sigma_batched(-1, None, None, None, 0, 0, None) == -1
    assert lib.sbd_sigma_batched(0, None, None, None, 0, 0, None) == 0
    assert b.sbd_status_string(2) == "pending"


def test_defaults_and_status_strings(lib):
    o = b.sbd_default_options()
    assert o.delta == 1e-4 and o.max_iter == 200 and o.max_subspace == 0 and not o.alloc
    assert b.sbd_status_string(0) == "ok"
    assert b.sbd_status_string(-3) == "duplicate string"


def test_host_side_argument_errors_need_no_gpu(lib):
    z = np.zeros(1)
    s = np.ones(1, dtype=np.uint64)
    with pytest.raises(b.SbdError) as e:
        b.sbd_create(65, 1, 1, z, z, s, s, stream=0)
    assert e.value.code == -4
    with pytest.raises(b.SbdError) as e:
        b.sbd_create(4, 5, 1, z, z, s, s, stream=0)
    assert e.value.code == -1
    out = ctypes.c_void_p()
    assert lib.sbd_create(None, 4, 1, 1, None, None, None, 1, None, 1, None, None) == -1
    assert lib.sbd_create(ctypes.byref(out), 4, 1, 1, None, None, None, 1, None, 1, None, None) == -1
    assert lib.sbd_destroy(None) == -1
    assert lib.sbd_sigma(None, None, None, 1, 0, None) == -1
    assert lib.sbd_davidson(None, 1, 1e-8, 0, None, None, None, None) == -1
