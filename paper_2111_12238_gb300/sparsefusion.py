"""Python binding of libsparsefusion.so (ctypes): argument marshalling only.

Every step of the inspector and the executor runs in the library's CUDA kernels; this
module turns torch tensors into device pointers and streams, raises on error statuses,
and wraps the fused pairs in ``torch.autograd.Function``s whose backward is the library's
fused adjoint pass. There is no CPU fallback: if the library is missing or no CUDA device
is present, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import _build

PAIRS = {"trsv_spmv": 0, "ic0_trsv": 1, "spmv_trsv": 2, "trsv": 3, "ic0": 4, "trsv_trsv": 5, "ilu0_trsv": 6}
SF_WANT_ADJOINT = 0x1
SF_EPOCH_FLAGS = 0x2
SF_DYNAMIC_QUEUE = 0x4
STATUS = {0: "SF_OK", 1: "SF_ERR_INVALID_ARG", 2: "SF_ERR_BAD_PATTERN", 3: "SF_ERR_CUDA", 4: "SF_ERR_OOM",
          5: "SF_ERR_TIMEOUT", 6: "SF_ERR_BREAKDOWN", 7: "SF_ERR_NONFINITE", 8: "SF_ERR_UNSUPPORTED"}


class SfCsr(C.Structure):
    _fields_ = [("n_rows", C.c_int32), ("n_cols", C.c_int32), ("nnz", C.c_int64),
                ("rowptr", C.c_void_p), ("colidx", C.c_void_p)]


class SfOptions(C.Structure):
    _fields_ = [("part_cost_target", C.c_int64), ("lanes_per_row", C.c_int32), ("rhs_tile", C.c_int32),
                ("g2_placement", C.c_int32), ("blocks_per_sm", C.c_int32), ("timeout_ns", C.c_uint64),
                ("flags", C.c_uint32), ("team_lanes", C.c_int32), ("block_rows", C.c_int32),
                ("exec_mode", C.c_int32)]


class SfInfo(C.Structure):
    _fields_ = [("pair", C.c_int32), ("n", C.c_int32), ("k_hint", C.c_int32), ("instances", C.c_int32),
                ("depth", C.c_int32), ("n_parts", C.c_int32), ("n_items", C.c_int64),
                ("adj_depth", C.c_int32), ("adj_n_parts", C.c_int32), ("adj_n_items", C.c_int64),
                ("lanes_per_row", C.c_int32), ("rhs_tile", C.c_int32),
                ("part_cost_target", C.c_int64), ("adj_part_cost_target", C.c_int64),
                ("packing", C.c_int32), ("blocks_per_sm", C.c_int32), ("epoch_flags", C.c_int32),
                ("dynamic_queue", C.c_int32),
                ("reuse_ratio", C.c_double), ("inspect_ms", C.c_double),
                ("wide_cost", C.c_int64), ("adj_wide_cost", C.c_int64),
                ("cost_total", C.c_int64), ("adj_cost_total", C.c_int64),
                ("adj_lanes_per_row", C.c_int32), ("reserved2", C.c_int32),
                ("team_lanes", C.c_int32), ("adj_team_lanes", C.c_int32),
                ("block_rows", C.c_int32), ("n_blocks", C.c_int32), ("adj_block_rows", C.c_int32),
                ("adj_n_blocks", C.c_int32), ("exec_mode", C.c_int32), ("adj_exec_mode", C.c_int32),
                ("block_lanes", C.c_int32), ("adj_block_lanes", C.c_int32),
                ("block_segments", C.c_int32), ("adj_block_segments", C.c_int32),
                ("block_threads", C.c_int32), ("adj_block_threads", C.c_int32),
                ("parts_class0", C.c_int32), ("adj_parts_class0", C.c_int32),
                ("split_pct", C.c_int32), ("adj_split_pct", C.c_int32),
                ("g2_placement", C.c_int32), ("adj_g2_placement", C.c_int32),
                ("min_blocks", C.c_int32), ("adj_min_blocks", C.c_int32),
                ("ic0_pairs", C.c_int64), ("ic0_use_pairs", C.c_int32), ("reserved3", C.c_int32),
                ("slice_cost", C.c_int64), ("adj_slice_cost", C.c_int64),
                ("slice_units", C.c_int32), ("adj_slice_units", C.c_int32),
                ("max_slices", C.c_int32), ("adj_max_slices", C.c_int32),
                ("fwd_rhs_tile", C.c_int32), ("adj_rhs_tile", C.c_int32)]


class SparseFusionError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        super().__init__(f"{what}: {STATUS.get(status, status)}{(' - ' + detail) if detail else ''}")
        self.status = status
        self.detail = detail


_lib = None
_lock = threading.Lock()

_P = C.c_void_p
_SIGS = {
    "sf_inspect": (C.c_int, [C.c_int, C.POINTER(SfCsr), C.POINTER(SfCsr), C.POINTER(SfOptions), _P, C.POINTER(_P)]),
    "sf_inspect_batched": (C.c_int, [C.c_int, C.c_int32, C.POINTER(SfCsr), C.POINTER(SfCsr), C.POINTER(SfOptions),
                                     _P, C.POINTER(_P)]),
    "sf_execute": (C.c_int, [_P, C.c_int, C.c_int32, _P, _P, _P, _P, _P, _P, _P]),
    "sf_adjoint": (C.c_int, [_P, C.c_int, C.c_int32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "sf_spmv": (C.c_int, [C.c_int, C.c_int32, C.POINTER(SfCsr), _P, _P, _P, _P, _P]),
    "sf_schedule_check": (C.c_int, [_P, _P, C.POINTER(C.c_int32)]),
    "sf_validate": (C.c_int, [_P]),
    "sf_schedule_info": (C.c_int, [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int64)]),
    "sf_schedule_query": (C.c_int, [_P, C.POINTER(SfInfo)]),
    "sf_schedule_export": (C.c_int, [_P, C.c_int32, _P, _P, _P]),
    "sf_schedule_set_launch": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32, C.c_int32]),
    "sf_schedule_set_timeout": (C.c_int, [_P, C.c_uint64]),
    "sf_schedule_recut": (C.c_int, [_P, C.c_int32, C.c_int64, C.c_int32, C.c_int32, _P]),
    "sf_schedule_reblock": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _P]),
    "sf_schedule_export_blocks": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P]),
    "sf_schedule_set_split": (C.c_int, [_P, C.c_int32, C.c_int32]),
    "sf_schedule_set_slices": (C.c_int, [_P, C.c_int32, C.c_int64, _P]),
    "sf_schedule_set_rhs_tile": (C.c_int, [_P, C.c_int32, C.c_int32]),
    "sf_schedule_set_packing": (C.c_int, [_P, C.c_int32]),
    "sf_schedule_replace": (C.c_int, [_P, C.c_int32, C.c_int32, _P]),
    "sf_schedule_set_occupancy": (C.c_int, [_P, C.c_int32, C.c_int32]),
    "sf_schedule_set_ic0_pairs": (C.c_int, [_P, C.c_int32]),
    "sf_schedule_set_exec_events": (C.c_int, [_P, C.c_int32, _P, _P]),
    "sf_schedule_launches": (C.c_int, [_P, C.c_int32, C.c_int32, C.POINTER(C.c_int32)]),
    "sf_schedule_debug_swap": (C.c_int, [_P, C.c_int64, C.c_int64]),
    "sf_schedule_destroy": (None, [_P]),
    "sf_bench_fma": (C.c_int, [C.c_int, C.c_int32, C.c_int32, _P, _P]),
    "sf_bench_hop": (C.c_int, [C.c_int32, _P, _P, _P]),
    "sf_status_string": (C.c_char_p, [C.c_int]),
    "sf_last_error_detail": (C.c_int, [C.c_char_p, C.c_size_t]),
}


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Loads libsparsefusion.so (building it first when absent and nvcc is available)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB):
                if not build_if_missing:
                    raise RuntimeError(f"{_build.LIB} is missing; build it with "
                                       "`python -m paper_2111_12238_gb300._build`")
                _build.build()
            lib = C.CDLL(_build.LIB)
            for name, (res, args) in _SIGS.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _detail() -> str:
    buf = C.create_string_buffer(512)
    load_library().sf_last_error_detail(buf, 512)
    return buf.value.decode(errors="replace")


def _check(st: int, what: str):
    if st != 0:
        raise SparseFusionError(st, what, _detail())


def _require_cuda(t: torch.Tensor, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (no CPU path exists)")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _ptr(t: Optional[torch.Tensor], name: str = "tensor"):
    if t is None:
        return None
    _require_cuda(t, name)
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dtype_code(dt: torch.dtype) -> int:
    if dt == torch.float64:
        return 0
    if dt == torch.float32:
        return 1
    raise ValueError(f"unsupported dtype {dt}: float64 or float32")


def _k_of(t: torch.Tensor) -> int:
    return 1 if t.dim() == 1 else int(t.shape[1])


@dataclass
class DeviceCsr:
    """A CSR pattern resident on the GPU (int32 rowptr / colidx)."""
    n_rows: int
    n_cols: int
    rowptr: torch.Tensor
    colidx: torch.Tensor

    @property
    def nnz(self) -> int:
        return int(self.colidx.numel())

    @classmethod
    def from_host(cls, csr, device="cuda") -> "DeviceCsr":
        rp = torch.from_numpy(np.ascontiguousarray(csr.rowptr, dtype=np.int32)).to(device)
        ci = torch.from_numpy(np.ascontiguousarray(csr.colidx, dtype=np.int32)).to(device)
        return cls(int(csr.n_rows), int(csr.n_cols), rp, ci)

    def struct(self) -> SfCsr:
        _require_cuda(self.rowptr, "rowptr")
        _require_cuda(self.colidx, "colidx")
        return SfCsr(self.n_rows, self.n_cols, self.nnz, self.rowptr.data_ptr(),
                     self.colidx.data_ptr() if self.nnz else 0)


def _options(want_adjoint, part_cost_target, lanes_per_row, rhs_tile, timeout_ns, blocks_per_sm=0,
             epoch_flags=False, dynamic_queue=False, team_lanes=0, block_rows=0, exec_mode=0,
             g2_placement=0) -> SfOptions:
    o = SfOptions()
    o.g2_placement = int(g2_placement)
    o.part_cost_target = int(part_cost_target)
    o.lanes_per_row = int(lanes_per_row)
    o.rhs_tile = int(rhs_tile)
    o.timeout_ns = int(timeout_ns)
    o.blocks_per_sm = int(blocks_per_sm)
    o.team_lanes = int(team_lanes)
    o.block_rows = int(block_rows)
    o.exec_mode = int(exec_mode)
    o.flags = ((SF_WANT_ADJOINT if want_adjoint else 0) | (SF_EPOCH_FLAGS if epoch_flags else 0)
               | (SF_DYNAMIC_QUEUE if dynamic_queue else 0))
    return o


class Schedule:
    """A fused schedule built by the GPU inspector; owns the library handle."""

    def __init__(self, handle: C.c_void_p, pair: str, n: int, keep=()):
        self._h = handle
        self.pair = pair
        self.n = n
        self._keep = keep

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("schedule destroyed")
        return self._h

    def close(self):
        if self._h:
            load_library().sf_schedule_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- introspection
    def info(self) -> dict:
        inf = SfInfo()
        _check(load_library().sf_schedule_query(self.handle, C.byref(inf)), "sf_schedule_query")
        return {f: getattr(inf, f) for f, _ in SfInfo._fields_}

    def export(self, which: int = 0) -> dict:
        inf = self.info()
        nv = inf["n_items"] if which == 0 else inf["adj_n_items"]
        P = inf["n_parts"] if which == 0 else inf["adj_n_parts"]
        level = np.zeros(nv, dtype=np.int32)
        order = np.zeros(nv, dtype=np.int32)
        pp = np.zeros(P + 1, dtype=np.int32)
        _check(load_library().sf_schedule_export(self.handle, which, level.ctypes.data, order.ctypes.data,
                                                 pp.ctypes.data), "sf_schedule_export")
        depth = inf["depth"] if which == 0 else inf["adj_depth"]
        return dict(level=level, order=order, part_ptr=pp, depth=depth)

    def validate(self):
        _check(load_library().sf_validate(self.handle), "sf_validate")

    def check(self, stream=None):
        """Synchronises and raises the first device-side failure recorded by executions."""
        row = C.c_int32(-1)
        st = load_library().sf_schedule_check(self.handle, _stream(stream), C.byref(row))
        if st != 0:
            raise SparseFusionError(st, "execution", _detail())

    def check_status(self, stream=None):
        row = C.c_int32(-1)
        st = load_library().sf_schedule_check(self.handle, _stream(stream), C.byref(row))
        return st, row.value

    def set_launch(self, lanes_per_row=0, rhs_tile=0, blocks_per_sm=0, epoch_flags=-1):
        _check(load_library().sf_schedule_set_launch(self.handle, int(lanes_per_row), int(rhs_tile),
                                                     int(blocks_per_sm), int(epoch_flags)),
               "sf_schedule_set_launch")

    def recut(self, which=-1, part_cost_target=0, lanes_per_row=0, team_lanes=0, stream=None):
        """Re-cuts the partitions for a new cost target and lane counts (levels and order kept)."""
        _check(load_library().sf_schedule_recut(self.handle, int(which), int(part_cost_target), int(lanes_per_row),
                                                int(team_lanes), _stream(stream)), "sf_schedule_recut")

    def reblock(self, which=-1, block_rows=0, exec_mode=-1, lanes_per_row=0, stream=None):
        """Rebuilds the row-block order for `block_rows` rows per block and/or selects the
        executor (exec_mode 0 automatic, 1 partitions, 2-4 row blocks, 5 one CTA per instance;
        for 5, block_rows must be 0 and lanes_per_row is the number of CTAs per SM)."""
        _check(load_library().sf_schedule_reblock(self.handle, int(which), int(block_rows), int(exec_mode),
                                                  int(lanes_per_row), _stream(stream)), "sf_schedule_reblock")

    def export_blocks(self, which=0) -> dict:
        inf = self.info()
        nv = inf["n_items"] if which == 0 else inf["adj_n_items"]
        nb = inf["n_blocks"] if which == 0 else inf["adj_n_blocks"]
        ns = inf["block_segments"] if which == 0 else inf["adj_block_segments"]
        order = np.zeros(nv, dtype=np.int32)
        bp = np.zeros(nb + 1, dtype=np.int32)
        sp = np.zeros(ns + 1, dtype=np.int32)
        bs = np.zeros(nb + 1, dtype=np.int32)
        _check(load_library().sf_schedule_export_blocks(self.handle, which, order.ctypes.data, bp.ctypes.data,
                                                        sp.ctypes.data, bs.ctypes.data),
               "sf_schedule_export_blocks")
        return dict(order=order, block_ptr=bp, seg_ptr=sp, block_seg=bs,
                    block_rows=inf["block_rows"] if which == 0 else inf["adj_block_rows"])

    def launches(self, which=0, k=1) -> int:
        """Kernel launches of one execute (0) or adjoint with both gradients (1)."""
        n = C.c_int32(0)
        _check(load_library().sf_schedule_launches(self.handle, int(which), int(k), C.byref(n)),
               "sf_schedule_launches")
        return n.value

    def set_exec_events(self, which, start=None, stop=None):
        """Records torch.cuda.Event pair (start, stop) around the next launches of the fused
        executor kernel of direction `which`; None, None stops recording."""
        hs = int(start.cuda_event) if start is not None else 0
        he = int(stop.cuda_event) if stop is not None else 0
        if (start is not None) and (hs == 0 or he == 0):
            raise ValueError("record each event once before passing it (torch creates events lazily)")
        _check(load_library().sf_schedule_set_exec_events(self.handle, int(which), hs or None, he or None),
               "sf_schedule_set_exec_events")

    def replace(self, which=-1, g2_placement=0, stream=None):
        """Re-places the second kernel's vertices of a separated schedule (0 earliest
        wavefront, -1 last, d > 0 delayed by d) and rebuilds order, cut and row blocks."""
        _check(load_library().sf_schedule_replace(self.handle, int(which), int(g2_placement), _stream(stream)),
               "sf_schedule_replace")

    def set_occupancy(self, which=-1, min_blocks=0):
        """Executor kernels budgeted for min_blocks resident blocks per SM (1 default, 3 for
        schedules bound by rows in flight)."""
        _check(load_library().sf_schedule_set_occupancy(self.handle, int(which), int(min_blocks)),
               "sf_schedule_set_occupancy")

    def set_ic0_pairs(self, use: bool):
        """IC0 schedules: read the inspector's intersection pairs (True) or search the common
        columns on every call (False)."""
        _check(load_library().sf_schedule_set_ic0_pairs(self.handle, int(bool(use))), "sf_schedule_set_ic0_pairs")

    def set_split(self, which=-1, class0_pct=0):
        """Runs the partitions that open with a first-kernel row on class0_pct percent of the
        teams (separated schedules; 0 = one class)."""
        _check(load_library().sf_schedule_set_split(self.handle, int(which), int(class0_pct)),
               "sf_schedule_set_split")

    def set_slices(self, which=-1, cost_per_slice=0, stream=None):
        """Split rows costlier than cost_per_slice over several teams (0: off)."""
        _check(load_library().sf_schedule_set_slices(self.handle, which, int(cost_per_slice), _stream(stream)),
               "sf_schedule_set_slices")

    def set_rhs_tile(self, which=-1, rhs_tile=0):
        """Right-hand-side columns a row's lanes handle side by side (0: automatic)."""
        _check(load_library().sf_schedule_set_rhs_tile(self.handle, which, int(rhs_tile)), "sf_schedule_set_rhs_tile")

    def set_packing(self, packing: int):
        """SpMV -> SpTRSV forward: 1 interleaved (paired rows), 0 separated (r first)."""
        _check(load_library().sf_schedule_set_packing(self.handle, int(packing)), "sf_schedule_set_packing")

    def set_timeout(self, ns: int):
        _check(load_library().sf_schedule_set_timeout(self.handle, int(ns)), "sf_schedule_set_timeout")

    def debug_swap(self, q1: int, q2: int):
        _check(load_library().sf_schedule_debug_swap(self.handle, int(q1), int(q2)), "sf_schedule_debug_swap")

    # -- executor
    def execute(self, L_vals, M_vals=None, b=None, x_in=None, y=None, x_save=None, stream=None):
        """Runs the fused pair; returns y (allocated when not given)."""
        ref = b if b is not None else L_vals
        dt = _dtype_code(ref.dtype)
        if self.pair == "ic0":
            k = 1
        else:
            k = _k_of(b)
            if y is None:
                y = torch.empty_like(b)
        st = load_library().sf_execute(self.handle, dt, k, _ptr(L_vals, "L_vals"), _ptr(M_vals, "M_vals"),
                                       _ptr(x_in, "x_in"), _ptr(b, "b"), _ptr(y, "y"), _ptr(x_save, "x_save"),
                                       _stream(stream))
        _check(st, "sf_execute")
        return y if self.pair != "ic0" else x_save

    def adjoint(self, L_vals, M_vals, gy, saved=None, x_in=None, gb=None, gx=None, gL=None, gM=None, stream=None):
        dt = _dtype_code(gy.dtype)
        k = _k_of(gy)
        if gb is None:
            gb = torch.empty_like(gy)
        st = load_library().sf_adjoint(self.handle, dt, k, _ptr(L_vals, "L_vals"), _ptr(M_vals, "M_vals"),
                                       _ptr(x_in, "x_in"), _ptr(saved, "saved"), _ptr(gy, "gy"), _ptr(gb, "gb"),
                                       _ptr(gx, "gx"), _ptr(gL, "gL"), _ptr(gM, "gM"), _stream(stream))
        _check(st, "sf_adjoint")
        return gb


def inspect(pair: str, L: DeviceCsr, M: Optional[DeviceCsr] = None, *, want_adjoint=False, part_cost_target=0,
            lanes_per_row=0, rhs_tile=0, timeout_ns=0, blocks_per_sm=0, epoch_flags=False,
            dynamic_queue=False, team_lanes=0, block_rows=0, exec_mode=0, g2_placement=0,
            stream=None) -> Schedule:
    lib = load_library()
    o = _options(want_adjoint, part_cost_target, lanes_per_row, rhs_tile, timeout_ns, blocks_per_sm, epoch_flags,
                 dynamic_queue, team_lanes, block_rows, exec_mode, g2_placement)
    Ls = L.struct()
    Ms = M.struct() if M is not None else None
    h = C.c_void_p()
    st = lib.sf_inspect(PAIRS[pair], C.byref(Ls), C.byref(Ms) if Ms is not None else None, C.byref(o),
                        _stream(stream), C.byref(h))
    _check(st, "sf_inspect")
    return Schedule(h, pair, L.n_rows)


def inspect_batched(pair: str, Ls: Sequence[DeviceCsr], Ms: Optional[Sequence[DeviceCsr]] = None, *,
                    want_adjoint=False, part_cost_target=0, lanes_per_row=0, rhs_tile=0, timeout_ns=0,
                    blocks_per_sm=0, epoch_flags=False, dynamic_queue=False, team_lanes=0, block_rows=0,
                    exec_mode=0, g2_placement=0, stream=None) -> Schedule:
    lib = load_library()
    o = _options(want_adjoint, part_cost_target, lanes_per_row, rhs_tile, timeout_ns, blocks_per_sm, epoch_flags,
                 dynamic_queue, team_lanes, block_rows, exec_mode, g2_placement)
    cnt = len(Ls)
    la = (SfCsr * cnt)(*[x.struct() for x in Ls])
    ma = (SfCsr * cnt)(*[x.struct() for x in Ms]) if Ms is not None else None
    h = C.c_void_p()
    st = lib.sf_inspect_batched(PAIRS[pair], cnt, la, ma, C.byref(o), _stream(stream), C.byref(h))
    _check(st, "sf_inspect_batched")
    return Schedule(h, pair, sum(x.n_rows for x in Ls))


def spmv(M: DeviceCsr, vals: torch.Tensor, x: torch.Tensor, b: Optional[torch.Tensor] = None,
         y: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """y = M x, or y = b - M x when b is given (the unfused SpMV launch)."""
    lib = load_library()
    k = _k_of(x)
    if y is None:
        y = torch.empty((M.n_rows,) + tuple(x.shape[1:]), dtype=x.dtype, device=x.device)
    Ms = M.struct()
    _check(lib.sf_spmv(_dtype_code(x.dtype), k, C.byref(Ms), _ptr(vals, "vals"), _ptr(x, "x"), _ptr(b, "b"),
                       _ptr(y, "y"), _stream(stream)), "sf_spmv")
    return y


# ------------------------------------------------------------------------------ measurement
def bench_fma_tflops(dtype=torch.float64, iters=4096, reps=5, stream=None) -> float:
    """Measured fused multiply-add rate of the current GPU (TFLOP/s, best of `reps`)."""
    lib = load_library()
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    blocks = props.multi_processor_count * 8
    sink = torch.empty(256, dtype=dtype, device="cuda")
    best = 0.0
    for _ in range(reps + 1):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        _check(lib.sf_bench_fma(_dtype_code(dtype), blocks, iters, _ptr(sink), _stream(stream)), "sf_bench_fma")
        b.record()
        b.synchronize()
        ms = a.elapsed_time(b)
        best = max(best, blocks * 256 * 16 * iters / (ms * 1e-3) / 1e12)
    return best


def bench_hop_ns(hops=20000, stream=None) -> float:
    """Measured latency (ns) of one value handed between two SMs through L2."""
    lib = load_library()
    word = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    _check(lib.sf_bench_hop(int(hops), _ptr(word), _ptr(out), _stream(stream)), "sf_bench_hop")
    o = out.cpu().tolist()
    if o[1]:
        raise SparseFusionError(5, "sf_bench_hop", "a poll gave up")
    return o[0] / hops


# ------------------------------------------------------------------------------ autograd
class TrsvSpmv(torch.autograd.Function):
    """y = M L^-1 b as one fused pass; backward is one fused adjoint pass."""

    @staticmethod
    def forward(ctx, sched: Schedule, L_vals, M_vals, b):
        x = torch.empty_like(b)
        y = sched.execute(L_vals, M_vals, b=b, x_save=x)
        ctx.sched = sched
        ctx.save_for_backward(L_vals, M_vals, x)
        return y

    @staticmethod
    def backward(ctx, gy):
        L_vals, M_vals, x = ctx.saved_tensors
        gy = gy.contiguous()
        need_L, need_M = ctx.needs_input_grad[1], ctx.needs_input_grad[2]
        gL = torch.empty_like(L_vals) if need_L else None
        gM = torch.empty_like(M_vals) if need_M else None
        gb = ctx.sched.adjoint(L_vals, M_vals, gy, saved=x, gL=gL, gM=gM)
        return None, gL, gM, gb


class SpmvTrsv(torch.autograd.Function):
    """z = L^-1 (b - A x_in) as one fused pass; backward is one fused adjoint pass."""

    @staticmethod
    def forward(ctx, sched: Schedule, L_vals, A_vals, x_in, b):
        z = sched.execute(L_vals, A_vals, b=b, x_in=x_in)
        ctx.sched = sched
        ctx.save_for_backward(L_vals, A_vals, x_in, z)
        return z

    @staticmethod
    def backward(ctx, gz):
        L_vals, A_vals, x_in, z = ctx.saved_tensors
        gz = gz.contiguous()
        gL = torch.empty_like(L_vals) if ctx.needs_input_grad[1] else None
        gA = torch.empty_like(A_vals) if ctx.needs_input_grad[2] else None
        gx = torch.empty_like(x_in) if ctx.needs_input_grad[3] else None
        gb = ctx.sched.adjoint(L_vals, A_vals, gz, saved=z, x_in=x_in, gx=gx, gL=gL, gM=gA)
        return None, gL, gA, gx, gb


def fused(sched: Schedule, *args):
    """Differentiable fused pair: fused(sched, L_vals, M_vals, b) for 'trsv_spmv',
    fused(sched, L_vals, A_vals, x_in, b) for 'spmv_trsv'."""
    if sched.pair == "trsv_spmv":
        return TrsvSpmv.apply(sched, *args)
    if sched.pair == "spmv_trsv":
        return SpmvTrsv.apply(sched, *args)
    raise ValueError(f"no differentiable form for {sched.pair}")


class GraphedExecute:
    """One fused execution captured in a CUDA graph with static tensors: replay() re-runs
    the persistent launch (the schedule's device-side epoch advances inside the graph)."""

    def __init__(self, sched: Schedule, **static):
        self.sched = sched
        self.static = static
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            sched.execute(**static)          # first call allocates any library scratch
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.out = sched.execute(**static)

    def replay(self):
        self.graph.replay()
        return self.out
