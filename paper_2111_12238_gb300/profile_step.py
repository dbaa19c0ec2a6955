"""One step of a workload in a fixed launch shape, for profilers:

    python -m paper_2111_12238_gb300.profile_step [n] [steps]
    python -m paper_2111_12238_gb300.profile_step lap2d [nx] [steps]
    python -m paper_2111_12238_gb300.profile_step lap3d [nx] [steps]

The first form runs the power-law SpMV -> SpTRSV workload: the fused forward with L read from
A's rows, then the fused adjoint with both value gradients. n = 4,194,304 is the powerlaw4m
workload of bench.py; a smaller n draws from the same generator (mean 16, max 2000, +-5000
band, k = 16, seed 5). The shapes are those the autotuner picks for that workload: forward 16
lanes per row, cost target 26, rows costlier than 64 split over teams; adjoint 16 lanes per
row, cost target 14, two-block kernels.

The second form runs the SpTRSV -> SpMV pair on the nx x nx 5-point grid (nx = 64 is the
lap2d64 workload, seed 1) on the single-CTA executor, the shape the autotuner picks there.

The third runs the SpTRSV -> SpMV pair on nx^3 (nx = 128 is the lap3d128 workload: lower
7-point L, banded M, seed 2), forward and adjoint with both value gradients, in the shapes the
autotuner picks there: forward on partitions (one lane per row, cost target 112, second-kernel
rows 32 wavefronts late), adjoint on the warp-specialised row blocks of 16384 rows."""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _powerlaw(n, steps, sf, I, dev):
    w = I.spmv_trsv_powerlaw(n=n, k=16, seed=5)
    sch = sf.inspect("spmv_trsv", sf.DeviceCsr.from_host(w.L), sf.DeviceCsr.from_host(w.M), want_adjoint=True)
    sch.recut(0, 26, 16, 32)
    sch.set_slices(0, 64)
    sch.recut(1, 14, 16, 32)
    sch.set_occupancy(1, 2)
    Lv, Av, xin, b, gz = dev(w.L.vals), dev(w.M.vals), dev(w.x_in), dev(w.b), dev(w.gy)
    z, gb, gx = torch.empty_like(b), torch.empty_like(b), torch.empty_like(b)
    gL, gA = torch.empty_like(Lv), torch.empty_like(Av)
    for _ in range(steps):
        sch.execute(None, Av, b=b, x_in=xin, y=z)
        sch.adjoint(Lv, Av, gz, saved=z, x_in=xin, gb=gb, gx=gx, gL=gL, gM=gA)
    return sch


def _lap2d(nx, steps, sf, I, dev):
    w = I.trsv_spmv_lap2d(nx, seed=1)
    sch = sf.inspect("trsv_spmv", sf.DeviceCsr.from_host(w.L), sf.DeviceCsr.from_host(w.M))
    sch.reblock(0, 0, 5, 0)
    Lv, Mv, b = dev(w.L.vals), dev(w.M.vals), dev(w.b)
    xs, y = torch.empty_like(b), torch.empty_like(b)
    for _ in range(steps):
        sch.execute(Lv, Mv, b=b, x_save=xs, y=y)
    return sch


def _lap3d(nx, steps, sf, I, dev):
    w = I.trsv_spmv_lap3d_band(nx)
    sch = sf.inspect("trsv_spmv", sf.DeviceCsr.from_host(w.L), sf.DeviceCsr.from_host(w.M), want_adjoint=True,
                     g2_placement=32)
    sch.recut(0, 112, 1, 32)
    sch.reblock(1, 16384, 3, 0)
    Lv, Mv, b, gy = dev(w.L.vals), dev(w.M.vals), dev(w.b), dev(w.gy)
    xs, y, gb = torch.empty_like(b), torch.empty_like(b), torch.empty_like(b)
    gL, gM = torch.empty_like(Lv), torch.empty_like(Mv)
    for _ in range(steps):
        sch.execute(Lv, Mv, b=b, x_save=xs, y=y)
        sch.adjoint(Lv, Mv, gy, saved=xs, gb=gb, gL=gL, gM=gM)
    return sch


def main():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2111_12238_gb300 import inputs as I
    from paper_2111_12238_gb300 import sparsefusion as sf
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()   # noqa: E731
    args = sys.argv[1:]
    if args and args[0] in ("lap2d", "lap3d"):
        size = int(args[1]) if len(args) > 1 else (64 if args[0] == "lap2d" else 128)
        steps = int(args[2]) if len(args) > 2 else 1
        sch = (_lap2d if args[0] == "lap2d" else _lap3d)(size, steps, sf, I, dev)
    else:
        size = int(args[0]) if args else (1 << 22)
        steps = int(args[1]) if len(args) > 1 else 1
        sch = _powerlaw(size, steps, sf, I, dev)
    torch.cuda.synchronize()
    sch.check()
    print("profile step done", size, steps)


if __name__ == "__main__":
    main()
