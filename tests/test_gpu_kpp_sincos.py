"""The sine and cosine of the KPP flux (cvweno_kpp_sincos, the forms the stage kernels
use): against FP64 and against CUDA's own FP32 sine and cosine on |d| <= 12 (the KPP
datum jumps by 3.25 pi, so deviations inside a cell stay well within that range).
  * sin d and cos d - 1 within 5e-7 absolutely (a few FP32 ulps at 1);
  * up to |d| = 1, cos d - 1 within 1e-6 relatively: the series has no cancellation;
  * within 6e-7 of torch.sin and torch.cos - 1 on the same FP32 arguments.
"""
import numpy as np
import pytest
import torch

from paper_2601_16911_gb300 import cvweno as cv

pytestmark = pytest.mark.gpu


def test_kpp_sincos_against_fp64_and_cuda():
    d = torch.linspace(-12.0, 12.0, 400001, device="cuda", dtype=torch.float32)
    s, cm1 = cv.cvweno_kpp_sincos(d)
    torch.cuda.synchronize()
    x = d.cpu().numpy().astype(np.float64)
    s64, c64 = np.sin(x), -2.0 * np.sin(0.5 * x) ** 2  # cos x - 1 without cancellation
    s_, c_ = s.cpu().numpy().astype(np.float64), cm1.cpu().numpy().astype(np.float64)
    assert np.abs(s_ - s64).max() <= 5e-7
    assert np.abs(c_ - c64).max() <= 5e-7
    small = (np.abs(x) <= 1.0) & (np.abs(c64) > 1e-30)
    assert (np.abs(c_ - c64)[small] / np.abs(c64[small])).max() <= 1e-6
    assert (s - torch.sin(d)).abs().max().item() <= 6e-7
    assert (cm1 - (torch.cos(d) - 1.0)).abs().max().item() <= 6e-7


def test_kpp_sincos_arguments():
    with pytest.raises(cv.CvwenoError) as e:
        cv._check(cv.load().cvweno_kpp_sincos(None, None, -1, None), "cvweno_kpp_sincos")
    assert e.value.code == cv.ERR_ARG
    s, cm1 = cv.cvweno_kpp_sincos(torch.empty(0, device="cuda"))
    assert s.numel() == 0 and cm1.numel() == 0
