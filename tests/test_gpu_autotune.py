"""GPU test of the autotuner: it measures every candidate, its choices are valid launch
configurations, and filters created with default tuning then run the chosen kernels correctly."""
import numpy as np
import pytest

import oracle
import workloads
from workloads import designs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_autotune_choices_and_parity():
    from paper_2607_23763_gb300 import build
    build.build()
    from paper_2607_23763_gb300 import SosFilter, autotune, autotune_choice
    dev = torch.device("cuda:0")
    rep = autotune(max_log2n=22)
    assert rep.shape == (8, 4, 6)
    assert np.all(rep[:, :3, :] > 0)  # lengths up to 2^24 (2^22 cap: the last bucket repeats the third)
    for K in (1, 2, 4, 8):
        for n in (1000, 1 << 16, 3 << 20, 1 << 27):
            solver, N, W = autotune_choice(K, n, with_groups=True)
            assert (solver, N, W) in ((1, 32, 0), (1, 64, 0), (2, 64, 7), (3, 64, 0), (2, 64, 10), (4, 64, 8)), \
                (K, n, solver, N, W)
    for K, n in ((1, 70001), (2, 1 << 16), (4, 300000), (8, 1 << 20)):
        sos = designs.butter_lowpass(2 * K, 0.05 if K > 1 else 0.2)
        x = workloads.normal_f32(K, n)
        f = SosFilter(sos)
        y = f.run(torch.from_numpy(x).to(dev))
        torch.cuda.synchronize()
        assert f.sync_status() == 0
        assert oracle.rel_err(y.cpu().numpy(), oracle.sosfilt(sos, x)) < designs.tolerance_for(sos), (K, n)
        f.close()
