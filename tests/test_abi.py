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
        "sos_autotune", "sos_autotune_choice", "sos_autotune_choice_ex", "sos_autotune_batch",
        "sos_autotune_batch_choice", "sos_batch_plan_create",
        "sos_batch_plan_launch",
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


def _tuning_valid(N, carry, solver, lw, det):
    """sos_filter_create's verdict on a tuning, written from the sos_tuning documentation in
    include/sosfilt.h (not from the implementation)."""
    if N not in (0, 32, 64, 128) or carry not in (0, 1, 2) or solver not in (0, 1, 2, 3, 4):
        return False
    if lw not in (0, 1, 2, 4, 8, 16) or det not in (0, 1):
        return False
    if carry in (0, 1) and N not in (0, 32, 64):  # the cascade carry (also the default) takes 32 or 64
        return False
    if solver == 2 and (N == 128 or carry == 2 or lw):
        return False
    if solver == 3 and (N not in (0, 64) or carry == 2 or lw):  # double-thread-group: N = 64, cascade carry
        return False
    if solver == 4 and (N not in (0, 64) or carry == 2 or lw):  # tensor cores: N = 64, cascade carry
        return False
    if det and (solver in (1, 3) or carry or lw or N == 128):
        return False
    return True


def _create_verdict(lib, sos, tuning):
    h = ctypes.c_void_p()
    rc = lib.sos_filter_create(sos.shape[0], sos.ctypes.data, None, ctypes.byref(tuning), ctypes.byref(h))
    if rc == 0:
        lib.sos_filter_destroy(h)
    else:
        assert h.value is None
    return rc


def test_tuning_validation_matches_the_header(lib):
    """Every combination of the tuning's selector fields: argument errors come back as SOS_EINVAL
    before a device is touched; the rest pass validation (and then fail, without a GPU, only at the
    first CUDA call, or succeed on a GPU)."""
    from paper_2607_23763_gb300._binding import Tuning
    sos = np.array([[1.0, 0.5, 0.25, -0.5, 0.25], [0.5, 0.0, -0.5, 0.1, 0.2]])
    seen = {True: 0, False: 0}
    for N in (0, 24, 32, 64, 128):
        for carry in (0, 1, 2, 3):
            for solver in (0, 1, 2, 3, 4):
                for lw in (0, 1, 3, 16):
                    for det in (0, 1, 2):
                        t = Tuning(N=N, carry=carry, solver=solver, lookback_width=lw, deterministic=det)
                        want = _tuning_valid(N, carry, solver, lw, det)
                        rc = _create_verdict(lib, sos, t)
                        assert (rc != -1) == want, (N, carry, solver, lw, det, rc)
                        assert rc in ((0, -2, -3) if want else (-1,)), rc
                        seen[want] += 1
    assert seen[True] > 50 and seen[False] > 500
    # the reserved and fixed fields
    for t in (Tuning(L=16), Tuning(threads_per_group=64), Tuning(groups_per_cta=2), Tuning(fp64_carry=1),
              Tuning(spin_budget_cycles=-1), Tuning(groups_per_cta=10, N=32), Tuning(groups_per_cta=7, solver=1),
              Tuning(groups_per_cta=10, solver=3), Tuning(groups_per_cta=7, carry=2), Tuning(groups_per_cta=8, solver=4),
              Tuning(groups_per_cta=7, solver=4)):
        assert _create_verdict(lib, sos, t) == -1
    # groups per tile of the PH solver: 7, or 10 at N = 64 (the default solver is PH)
    for t in (Tuning(groups_per_cta=7), Tuning(groups_per_cta=10), Tuning(groups_per_cta=10, solver=2, N=64),
              Tuning(groups_per_cta=7, solver=2, N=32)):
        assert _create_verdict(lib, sos, t) != -1
    for t in (Tuning(L=32), Tuning(threads_per_group=32), Tuning(spin_budget_cycles=1 << 20)):
        assert _create_verdict(lib, sos, t) != -1


def test_stability_triangle_is_the_unit_circle(lib):
    """A section is accepted exactly when both roots of z^2 + a1 z + a2 lie inside the unit circle
    (np.roots), on a seeded scatter over and around the stability triangle, away from its edges."""
    rng = np.random.default_rng(7)
    n_in = n_out = 0
    for a1, a2 in rng.uniform([-2.6, -1.4], [2.6, 1.4], size=(3000, 2)):
        margin = min(abs(abs(a2) - 1.0), abs(abs(a1) - (1.0 + a2)))
        if margin < 1e-6:
            continue
        stable = float(np.max(np.abs(np.roots([1.0, a1, a2])))) < 1.0
        sos = np.array([[1.0, 2.0, 1.0, a1, a2]])
        h = ctypes.c_void_p()
        rc = lib.sos_filter_create(1, sos.ctypes.data, None, None, ctypes.byref(h))
        if rc == 0:
            lib.sos_filter_destroy(h)
        assert (rc != -5) == stable, (a1, a2, rc)
        n_in += stable
        n_out += not stable
    assert n_in > 500 and n_out > 500
    # on the edges: a pole on the unit circle is rejected
    for a1, a2 in ((0.0, 1.0), (0.0, -1.0), (1.5, 0.5), (-1.5, 0.5), (2.0, 1.0)):
        sos = np.array([[1.0, 2.0, 1.0, a1, a2]])
        h = ctypes.c_void_p()
        assert lib.sos_filter_create(1, sos.ctypes.data, None, None, ctypes.byref(h)) == -5


def test_no_cpu_fallback_without_a_gpu_or_the_library(tmp_path):
    """The binding fails loudly: a missing library raises, and without a GPU creating a filter
    raises SosError (SOS_ECUDA) instead of computing on the CPU."""
    import torch

    from paper_2607_23763_gb300 import _binding as B
    with pytest.raises(RuntimeError, match="missing"):
        saved = B._lib
        B._lib = None
        try:
            B.load_library(str(tmp_path / "libsosfilt_absent.so"))
        finally:
            B._lib = saved
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the GPU tests cover the library's device path")
    from paper_2607_23763_gb300 import SosError, SosFilter
    with pytest.raises(SosError) as e:
        SosFilter(np.array([[1.0, 2.0, 1.0, -0.5, 0.25]]))
    assert e.value.code == -3 and "SOS_ECUDA" in str(e.value)
