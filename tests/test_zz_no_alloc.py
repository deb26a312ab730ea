"""sos_filter_run_noalloc, the entry point for callers that cannot allocate device memory while
they filter (for instance a real-time receive thread, where cudaMalloc/cudaFree may block and
synchronize the device): it must give the same output as sos_filter_run, call after call, with
its scratch in the library's fixed device array.

Collected last on purpose (file name), so a run that stops at the first failure has already run
every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads
from workloads import designs

from ._tol import bound

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _call(f, x, y, zi=None, zf=None):
    # straight through the C ABI
    lib = f._lib
    rc = lib.sos_filter_run_noalloc(f.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                    x.numel(), None if zi is None else ctypes.c_void_p(zi.data_ptr()),
                                    None if zf is None else ctypes.c_void_p(zf.data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, rc


@pytest.mark.parametrize("order,n", [(16, 3 * 8192 + 4099), (2, 1 << 20), (16, 1 << 22)])
def test_noalloc_matches_run_two_calls(order, n):
    from paper_2607_23763_gb300 import SosFilter, build
    build.build()
    dev = torch.device("cuda:0")
    sos = designs.butter_lowpass(order, 0.05)
    K = sos.shape[0]
    f = SosFilter(sos)
    x = torch.from_numpy(workloads.normal_f32(7 + order, n)).to(dev)
    zi = torch.from_numpy((np.random.default_rng(order).standard_normal((K, 2)) * 0.01).astype(np.float32)).to(dev)
    y_ref = f.run(x, zi=zi, zf=(zf_ref := torch.empty(K, 2, device=dev)))
    for _ in range(2):  # two calls in a row share the same device array
        y = torch.full_like(x, float("nan"))
        zf = torch.full((K, 2), float("nan"), device=dev)
        _call(f, x, y, zi, zf)
        torch.cuda.synchronize()
        assert f.sync_status() == 0
        ref = y_ref.double().cpu().numpy()
        got = y.double().cpu().numpy()
        tol = bound(sos)
        assert np.all(np.isfinite(got))
        assert oracle.rel_err(got, ref) < tol
        assert float((zf - zf_ref).abs().max()) <= 10 * tol * max(1e-30, float(zf_ref.abs().max()))
    f.close()


def test_noalloc_rejects_oversized_request():
    from paper_2607_23763_gb300 import SosFilter
    f = SosFilter(designs.butter_lowpass(2, 0.2))
    lib = f._lib
    rc = lib.sos_filter_run_noalloc(f.handle, ctypes.c_void_p(16), ctypes.c_void_p(16), (1 << 28) + 1, None, None,
                                    None)
    assert rc == -6  # SOS_EBUDGET, before any device work
    f.close()
