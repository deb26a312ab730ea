"""The C-ABI library loads and exports every symbol include/sosfilt.h declares; host-side
argument checks that need no GPU."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sosfilt.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sos_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2607_23763_gb300 import build
    build.build()
    from paper_2607_23763_gb300 import load_library
    return load_library()


def test_header_declares_the_abi():
    assert _declared() == sorted([
        "sos_filter_create", "sos_filter_destroy", "sos_filter_run", "sos_filter_run_batch",
        "sos_filter_stream_push", "sos_filter_stream_state", "sos_filter_sync_status", "sos_filter_trace",
        "sos_filter_run_host", "sos_filter_run_noalloc", "sos_filter_run_batch_ex", "sos_batch_sync_status",
        "sos_server_create", "sos_server_destroy", "sos_server_add_stream", "sos_server_submit", "sos_server_poll",
        "sos_server_drain", "sos_server_stream_state", "sos_server_get_stats", "sos_server_replay",
        "sos_autotune", "sos_autotune_choice", "sos_batch_plan_create", "sos_batch_plan_launch",
        "sos_batch_plan_status", "sos_batch_plan_destroy", "sos_status_string"])


def test_library_exports_every_declared_symbol(lib):
    from paper_2607_23763_gb300 import LIB_PATH, EXPORTED
    out = subprocess.run(["nm", "-D", "--defined-only", LIB_PATH], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (sos_[a-z_]+)", out))
    for name in _declared():
        assert name in exported, name
        assert hasattr(lib, name)
    assert set(EXPORTED) == set(_declared())


def test_status_strings(lib):
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert lib.sos_status_string(code).decode().startswith("SOS_")


def test_create_rejects_bad_arguments_before_touching_a_device(lib):
    h = ctypes.c_void_p()
    sos = np.array([[1.0, 0.0, 0.0, -0.5, 0.25]])
    assert lib.sos_filter_create(1, None, None, None, ctypes.byref(h)) == -1
    assert lib.sos_filter_create(0, sos.ctypes.data, None, None, ctypes.byref(h)) == -1
    assert lib.sos_filter_create(1, sos.ctypes.data, None, None, None) == -1
    unstable = np.array([[1.0, 0.0, 0.0, -2.5, 1.2]])
    assert lib.sos_filter_create(1, unstable.ctypes.data, None, None, ctypes.byref(h)) == -5
    nonfinite = np.array([[np.nan, 0.0, 0.0, -0.5, 0.25]])
    assert lib.sos_filter_create(1, nonfinite.ctypes.data, None, None, ctypes.byref(h)) == -5
    assert h.value is None
    from paper_2607_23763_gb300._binding import Tuning
    bad = Tuning(N=24)
    assert lib.sos_filter_create(1, sos.ctypes.data, None, ctypes.byref(bad), ctypes.byref(h)) == -1
    # NULL filter handles are argument errors, not crashes
    assert lib.sos_filter_run(None, None, None, 0, None, None, None) == -1
    assert lib.sos_filter_sync_status(None) == -1
    assert lib.sos_filter_trace(None, None, 0) == -1
    assert lib.sos_filter_run_host(None, None, None, 0, None, None, 0) == -1
    assert lib.sos_filter_run_noalloc(None, None, None, 0, None, None, None) == -1
    assert lib.sos_filter_destroy(None) == 0
    assert lib.sos_filter_run_batch(0, None, None, None, None, None) == 0
    assert lib.sos_filter_run_batch(-1, None, None, None, None, None) == -1


def test_ctypes_structures_match_the_header_layout():
    """Every struct the binding mirrors has the header's size and field offsets (compiled with the
    host C compiler from include/sosfilt.h, no device needed)."""
    import shutil
    import subprocess
    from paper_2607_23763_gb300 import _binding as B
    if not shutil.which("gcc"):
        pytest.skip("no host C compiler")
    structs = {"sos_tuning": B.Tuning, "sos_server_config": B.ServerConfig, "sos_completion": B.Completion,
               "sos_server_stats": B.ServerStats}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "sosfilt.h"', 'int main(void) {']
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0; }")
    build_dir = os.path.join(ROOT, "tests", "_build")
    os.makedirs(build_dir, exist_ok=True)
    src = os.path.join(build_dir, "layout.c")
    with open(src, "w") as fh:
        fh.write("\n".join(lines))
    exe = os.path.join(build_dir, "layout")
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", exe, src], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
