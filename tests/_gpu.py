"""Helpers of the GPU tests: moving seeded workloads to the device and comparing results
with the oracle. Every GPU call goes through the library's C ABI."""
import numpy as np
import pytest
import torch

from paper_2111_12238_gb300 import sparsefusion as sf

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


def need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev_csr(csr):
    return sf.DeviceCsr.from_host(csr)


def t(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(x):
    return x.detach().double().cpu().numpy()


def col_rel_err(got, ref):
    """max over right-hand-side columns of ||got - ref||_inf / ||ref||_inf."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if ref.ndim == 1:
        ref = ref[:, None]
        got = got.reshape(ref.shape)
    worst = 0.0
    for c in range(ref.shape[1]):
        den = np.max(np.abs(ref[:, c]))
        num = np.max(np.abs(got[:, c] - ref[:, c]))
        worst = max(worst, num / den if den > 0 else num)
    return worst


def vec_rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    den = np.max(np.abs(ref)) if ref.size else 0.0
    num = np.max(np.abs(got - ref)) if ref.size else 0.0
    return num / den if den > 0 else num


def order_to_vid(order, n):
    o = order.view(np.uint32).astype(np.int64)
    return (o >> 31) * n + (o & 0x7FFFFFFF)
