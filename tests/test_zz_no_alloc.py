"""The allocation-free entry point sf_trsv_spmv_noalloc, called through the C ABI, must give
the same y = M L^-1 b as the scheduled path (sf_inspect + sf_execute) and as the FP64 oracle,
on two calls in a row (the second call checks that the shared device scratch is cleared
between calls), without allocating device memory. It serves callers that cannot allocate at
the point of the call: a custom allocator's own callbacks, applications whose device memory is
all handed out in advance by their own pool, latency-critical loops that cannot wait for the
synchronisation an allocation can imply. Collected last, so that a failure here leaves every
other test already run."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
from paper_2111_12238_gb300 import inputs as I
from paper_2111_12238_gb300 import sparsefusion as sf
from tests._gpu import TOL, col_rel_err, dev_csr, host, need_cuda, t
from tests._mats import dense_to_csr

pytestmark = pytest.mark.gpu

MAX_ROWS = 1048576


def _entry():
    lib = sf.load_library()
    f = lib.sf_trsv_spmv_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_int, C.POINTER(sf.SfCsr), C.POINTER(sf.SfCsr), C.c_void_p, C.c_void_p, C.c_void_p,
                  C.c_void_p, C.c_void_p]
    return f


def _call(f, dt, Ld, Md, Lv, Mv, b, y):
    Ls, Ms = Ld.struct(), Md.struct()
    return f(dt, C.byref(Ls), C.byref(Ms), Lv.data_ptr(), Mv.data_ptr(), b.data_ptr(), y.data_ptr(),
             torch.cuda.current_stream().cuda_stream)


def _free_bytes():
    free, _ = torch.cuda.mem_get_info()
    return free


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("make", [lambda: I.trsv_spmv_lap2d(64, seed=1),
                                  lambda: I.trsv_spmv_lap3d_band(24, per_row=8, halfband=1000, seed=2)])
def test_noalloc_matches_scheduled_path_and_oracle_twice(dtype, make):
    need_cuda()
    f = _entry()
    w = make()
    Ld, Md = dev_csr(w.L), dev_csr(w.M)
    Lv, Mv, b = t(w.L.vals, dtype), t(w.M.vals, dtype), t(w.b, dtype)
    sch = sf.inspect("trsv_spmv", Ld, Md)
    y_ref = sch.execute(Lv, Mv, b=b)
    sch.check()
    _, y_orc = oracle.trsv_spmv(w.L, w.M, w.b)
    dt = 0 if dtype == torch.float64 else 1
    ys = [torch.full_like(b, 7.0) for _ in range(3)]
    assert _call(f, dt, Ld, Md, Lv, Mv, b, ys[0]) == 0        # first call on the device: set-up
    torch.cuda.synchronize()
    alloc0, free0 = torch.cuda.memory_allocated(), _free_bytes()
    for y in ys[1:]:
        assert _call(f, dt, Ld, Md, Lv, Mv, b, y) == 0
    torch.cuda.synchronize()
    # nothing was allocated by the two calls
    assert torch.cuda.memory_allocated() == alloc0 and _free_bytes() == free0
    for y in ys:
        assert col_rel_err(host(y), host(y_ref)) < TOL[dtype]
        assert col_rel_err(host(y), y_orc) < TOL[dtype]


def test_noalloc_zero_diagonal_is_reported_and_the_next_call_works():
    need_cuda()
    f = _entry()
    # L = [[2, 0], [1, 0]]: the zero L_11 is used as a divisor
    L = dense_to_csr(np.array([[2.0, 0.0], [1.0, 0.0]]), pattern=np.array([[True, False], [True, True]]))
    M = dense_to_csr(np.eye(2))
    Ld, Md = dev_csr(L), dev_csr(M)
    y = torch.zeros((2, 1), dtype=torch.float64, device="cuda")
    assert _call(f, 0, Ld, Md, t(L.vals), t(M.vals), t(np.ones((2, 1))), y) == 7      # SF_ERR_NONFINITE
    w = I.trsv_spmv_lap2d(16, seed=3)
    y2 = torch.empty((w.n, 1), dtype=torch.float64, device="cuda")
    assert _call(f, 0, dev_csr(w.L), dev_csr(w.M), t(w.L.vals), t(w.M.vals), t(w.b), y2) == 0
    assert col_rel_err(host(y2), oracle.trsv_spmv(w.L, w.M, w.b)[1]) < 1e-12


def test_noalloc_rejects_oversize_and_bad_patterns():
    need_cuda()
    f = _entry()
    lib = sf.load_library()
    one = torch.ones(4, dtype=torch.int32, device="cuda")
    big = sf.SfCsr(MAX_ROWS + 1, MAX_ROWS + 1, MAX_ROWS + 1, one.data_ptr(), one.data_ptr())
    v = torch.ones(4, dtype=torch.float64, device="cuda")
    st = f(0, C.byref(big), C.byref(big), v.data_ptr(), v.data_ptr(), v.data_ptr(), v.data_ptr(),
           torch.cuda.current_stream().cuda_stream)
    assert st == 1
    buf = C.create_string_buffer(256)
    lib.sf_last_error_detail(buf, 256)
    assert b"SF_NOALLOC_MAX_ROWS" in buf.value
    # an upper entry in L: reported, nothing computed from it
    rp = torch.tensor([0, 2, 3], dtype=torch.int32, device="cuda")
    ci = torch.tensor([0, 1, 1], dtype=torch.int32, device="cuda")
    bad = sf.DeviceCsr(2, 2, rp, ci)
    Md = sf.DeviceCsr(2, 2, torch.tensor([0, 1, 2], dtype=torch.int32, device="cuda"),
                      torch.tensor([0, 1], dtype=torch.int32, device="cuda"))
    vals = torch.ones(3, dtype=torch.float64, device="cuda")
    y = torch.zeros((2, 1), dtype=torch.float64, device="cuda")
    assert _call(f, 0, bad, Md, vals, vals, torch.ones((2, 1), dtype=torch.float64, device="cuda"), y) == 2
    # the next valid call still works
    w = I.trsv_spmv_lap2d(16, seed=3)
    Ld, Mdd = dev_csr(w.L), dev_csr(w.M)
    sch = sf.inspect("trsv_spmv", Ld, Mdd)
    y_ref = sch.execute(t(w.L.vals), t(w.M.vals), b=t(w.b))
    y2 = torch.empty_like(y_ref)
    assert _call(f, 0, Ld, Mdd, t(w.L.vals), t(w.M.vals), t(w.b), y2) == 0
    assert col_rel_err(host(y2), host(y_ref)) < 1e-12
