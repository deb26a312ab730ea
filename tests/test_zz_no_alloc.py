"""sos_filter_run_noalloc, the entry point for callers that cannot allocate device memory while
they filter (for instance a real-time receive thread, where cudaMalloc/cudaFree may block and
synchronize the device): it runs the same PH kernel as sos_filter_run with its scratch in the
library's fixed device array, so its output and final state must equal sos_filter_run's bit for
bit, call after call, and match the float64 oracle within the stated bound.

Collected last on purpose (file name), so a run that stops at the first failure has already run
every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads
from workloads import designs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SOLVER_PH = 2
MAX_SAMPLES = 1 << 28  # SOS_NOALLOC_MAX_SAMPLES


def _call(f, x, y, zi=None, zf=None):
    # straight through the C ABI
    lib = f._lib
    rc = lib.sos_filter_run_noalloc(f.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                    x.numel(), None if zi is None else ctypes.c_void_p(zi.data_ptr()),
                                    None if zf is None else ctypes.c_void_p(zf.data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, rc


def _sos(kind):
    if kind == "butter16":
        return designs.butter_lowpass(16, 0.05)
    if kind == "butter2":
        return designs.butter_lowpass(2, 0.2)
    # twelve sections: two passes (8 + 4) through the fixed array
    return designs.butter_lowpass(24, 0.1)


@pytest.mark.parametrize("kind,n", [("butter16", 3 * 14336 + 4099), ("butter2", 1 << 20), ("butter16", 1 << 22),
                                    ("butter24", 5 * 14336 + 77)])
def test_noalloc_matches_run_two_calls(kind, n):
    from paper_2607_23763_gb300 import SosFilter, build
    build.build()
    dev = torch.device("cuda:0")
    sos = _sos(kind)
    K = sos.shape[0]
    # sos_filter_run with the PH solver at its default N = 64: the kernel the no-alloc path runs
    f = SosFilter(sos, tuning={"solver": SOLVER_PH})
    xh = workloads.normal_f32(7 + K, n)
    x = torch.from_numpy(xh).to(dev)
    zih = (np.random.default_rng(K).standard_normal((K, 2)) * 0.01).astype(np.float32)
    zi = torch.from_numpy(zih).to(dev)
    zf_ref = torch.empty(K, 2, device=dev)
    y_ref = f.run(x, zi=zi, zf=zf_ref)
    yo, zo = oracle.sosfilt(sos, xh, zi=zih.astype(np.float64), return_state=True)
    tol = designs.tolerance_for(sos)
    for _ in range(2):  # two calls in a row share the same device array
        y = torch.full_like(x, float("nan"))
        zf = torch.full((K, 2), float("nan"), device=dev)
        _call(f, x, y, zi, zf)
        torch.cuda.synchronize()
        assert f.sync_status() == 0
        assert torch.equal(y, y_ref)
        assert torch.equal(zf, zf_ref)
        err = oracle.rel_err(y.cpu().numpy(), yo)
        zerr = float(np.abs(zf.cpu().numpy() - zo).max() / max(1e-30, np.abs(zo).max()))
        print(f"{kind} n={n}: output error {err:.3e}, final-state error {zerr:.3e}, bound {tol}")
        assert err < tol and zerr < tol
    f.close()


def test_noalloc_at_the_size_limit():
    """n = SOS_NOALLOC_MAX_SAMPLES fills the array's descriptor space to its last tile: the same
    output as sos_filter_run bit for bit, and sampled windows against the oracle."""
    from paper_2607_23763_gb300 import SosFilter, build
    build.build()
    dev = torch.device("cuda:0")
    sos = designs.butter_lowpass(16, 0.05)
    xh = workloads.normal_f32(1, MAX_SAMPLES)
    x = torch.from_numpy(xh).to(dev)
    f = SosFilter(sos, tuning={"solver": SOLVER_PH})
    y_ref = f.run(x)
    y = torch.full_like(x, float("nan"))
    _call(f, x, y)
    torch.cuda.synchronize()
    assert f.sync_status() == 0
    assert torch.equal(y, y_ref)
    del y_ref
    settle = 4000  # r_max^4000 < 1e-20 for r_max < 0.99
    worst = 0.0
    for a in [0, MAX_SAMPLES - 4096, MAX_SAMPLES // 2 + 123]:
        a0 = max(0, a - settle)
        ref = oracle.sosfilt(sos, xh[a0:a + 4096])[a - a0:]
        got = y[a:a + 4096].cpu().numpy()
        worst = max(worst, float(np.abs(got - ref).max() / np.abs(ref).max()))
    assert worst < designs.tolerance_for(sos), worst
    f.close()


def test_noalloc_rejects_oversized_request():
    from paper_2607_23763_gb300 import SosFilter
    f = SosFilter(designs.butter_lowpass(2, 0.2))
    lib = f._lib
    rc = lib.sos_filter_run_noalloc(f.handle, ctypes.c_void_p(16), ctypes.c_void_p(16), MAX_SAMPLES + 1, None, None,
                                    None)
    assert rc == -6  # SOS_EBUDGET, before any device work
    f.close()
