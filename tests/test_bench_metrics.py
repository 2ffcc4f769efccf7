"""The bench's torch quality metrics (PSNR, 3D SSIM) agree with the oracle's on the CPU."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_psnr_ssim_match_oracle():
    import torch
    import oracle
    sys.path.insert(0, ROOT)
    import bench
    rng = np.random.default_rng(0)
    ref = rng.uniform(0, 1, (17, 20, 23))
    x = np.clip(ref + rng.normal(0, 0.05, ref.shape), 0, 1)
    tx, tr = torch.as_tensor(x), torch.as_tensor(ref)
    assert abs(bench.psnr_t(tx, tr) - oracle.psnr(x, ref)) < 1e-9
    assert abs(bench.ssim3d_t(tx, tr) - oracle.ssim3d(x, ref)) < 1e-9
    assert abs(bench.ssim3d_t(tr, tr) - 1.0) < 1e-12
