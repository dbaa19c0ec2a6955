"""Benchmark of the fused sparse-fusion hot path on its synthetic workloads (GB300, one GPU).

The default run measures every workload, each as one "step" of its fused passes, and prints
ONE JSON line: the headline workload, the 4M-row power-law SpMV -> SpTRSV Gauss-Seidel
half-sweep with 16 right-hand sides (fused forward, L = tril(A) read from A's rows, plus
the fused adjoint with both value gradients; FP64), whose object carries the complete lines
of the other workloads under "workloads" (each line is also printed to stderr as it
finishes):
  lap2d64      SpTRSV -> SpMV on the 64x64 5-point grid, forward (k = 1)
  lap3d128     SpTRSV -> SpMV on 128^3 (L lower 7-point, M banded), forward + adjoint
  aniso100     SpIC0 -> SpTRSV on the anisotropic 100^3 Laplacian, 32 right-hand sides
  batched512   512 power-law SpTRSV -> SpMV instances in one launch, forward + adjoint,
               FP64 and FP32 (two lines)
  powerlaw4m   the headline
  trsv_trsv    SpTRSV -> SpTRSV with the 128^3 lower 7-point L (Table 2 combination 1)
  ilu0_trsv    SpILU0 -> SpTRSV on the anisotropic 100^3 matrix, 32 right-hand sides
               (Table 2 combination 6)
`--workload NAME` measures one workload and prints its line alone.

For each workload: `value` = steps per second with inputs resident in HBM (L2 flushed by a
256 MB write before every step, outside the timed launches); `e2e` = the same steps through
the public calls with the right-hand sides copied in from pinned host memory and the results
(and value gradients) copied back; `roofline` = the longer fused executor kernel, timed live
with CUDA events the library records around it, against the measured HBM copy bandwidth, with
the measured FP64 rate and the measured SM-to-SM hand-off latency as further lower bounds;
the unfused two-launch paths (forward and adjoint) timed on the same GPU; `cpu_baseline` =
the sequential FP64 oracle on the host (a bounded sample). `--impl reference` times the
oracle alone on the headline workload (a bounded leading-rows sample per step).
For N > 1 (torchrun) every rank runs an independent replica (a single triangular system does
not shard); the value is the sum over ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fused-pair solves/s, HBM GB/s (% peak) vs unfused same GPU; adjoint/fwd ratio"
HEADLINE = "powerlaw4m"
ORDER = ["lap2d64", "lap3d128", "aniso100", "batched512", "batched512_f32", "powerlaw4m", "trsv_trsv", "ilu0_trsv"]
FP64_NOMINAL_TFLOPS = 1.25   # GB300 nominal FP64 rate, used only when no measured rate is given


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def _csrc_hash(files=None):
    """Hash of the named sources under csrc/ (all of them when `files` is None)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2111_12238_gb300", "csrc")
    paths = sorted(glob.glob(os.path.join(csrc, "*"))) if files is None else \
        [os.path.join(csrc, f) for f in sorted(files)]
    for f in paths:
        with open(f, "rb") as fh:
            h.update(os.path.basename(f).encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def _recorded_traffic(workload, kernel):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current
    sources of that kernel (the files the record lists, else every source); else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(workload, {}).get(kernel)
    if not e:
        return None
    try:
        if e.get("csrc_hash") != _csrc_hash(e.get("sources")):
            return None
    except OSError:
        return None
    return e.get("bytes_per_launch")


# ----------------------------------------------------------------------------- workloads
def csr_bytes(nnz, n, es):
    return (es + 4) * nnz + 4 * (n + 1)


_GENERATED = {}


def _generate(name):
    """The seeded inputs of a workload (generated once per process; the FP32 line of the
    batched workload reuses the FP64 line's instances)."""
    base = name[:-4] if name.endswith("_f32") else name
    if base not in _GENERATED:
        _GENERATED[base] = _generate_new(base)
    return _GENERATED[base]


def _generate_new(base):
    from paper_2111_12238_gb300 import inputs as I
    if base == "lap2d64":
        return I.trsv_spmv_lap2d(64, seed=1), False
    if base == "lap3d128":
        return I.trsv_spmv_lap3d_band(128, seed=2), True
    if base == "aniso100":
        return I.ic0_trsv_aniso3d(100, k=32, seed=3), False
    if base == "batched512":
        return I.batched_trsv_spmv(512, seed=4), True
    if base == "powerlaw4m":
        return I.spmv_trsv_powerlaw(seed=5), True
    if base == "trsv_trsv":
        # Table 2 combination 1 on the 128^3 lower 7-point L of lap3d128
        w = I.trsv_spmv_lap3d_band(128, seed=2)
        return I.Workload("trsv_trsv_lap3d_128^3", "trsv_trsv", w.n, 1, w.L, None, w.b), False
    if base == "ilu0_trsv":
        # Table 2 combination 6 on the anisotropic 100^3 matrix (the full A, not its lower part)
        A = I.aniso_laplacian_3d((100, 100, 100))
        b = I.dense_vectors(A.n_rows, 32, 3, I.S_RHS)
        w = I.Workload("ilu0_trsv_aniso3d_100^3_k32", "ilu0_trsv", A.n_rows, 32, I.lower_part(A), A, b)
        return w, False
    raise SystemExit(f"unknown workload {base}")


def make_workload(name, dtype_name="f64"):
    """The workload's inputs and the algorithmic bytes and flops of its passes (each array
    touched once; value arrays es bytes per entry, patterns 4 bytes per entry and row)."""
    if name.endswith("_f32"):
        dtype_name = "f32"
    w, adj = _generate(name)
    es = 8 if dtype_name == "f64" else 4
    n, k = w.n, w.k
    if w.instances:
        nnzL = sum(x.L.nnz for x in w.instances)
        nnzM = sum(x.M.nnz for x in w.instances)
    else:
        nnzL = w.L.nnz
        nnzM = w.M.nnz if w.M is not None else 0
    vec = es * n * k
    adj_bytes = adj_exec_bytes = adj_flops = 0
    if w.pair == "trsv_spmv":
        fwd_bytes = csr_bytes(nnzL, n, es) + csr_bytes(nnzM, n, es) + 3 * vec      # b in, x and y out
        adj_bytes = csr_bytes(nnzL, n, es) + csr_bytes(nnzM, n, es) + 3 * vec + es * (nnzL + nnzM)
        # fused adjoint kernel alone: L^T and M^T (pattern, values), gy in, lam out
        adj_exec_bytes = csr_bytes(nnzL, n, es) + csr_bytes(nnzM, n, es) + 2 * vec
        fwd_flops = 2 * (nnzL + nnzM) * k + n * k                                # + one division per row
        adj_flops = 2 * (nnzL + nnzM) * k + n * k
    elif w.pair == "spmv_trsv":
        # forward with L = tril(A) read from A's rows: A (pattern, values, diagonal positions),
        # x_in and b in, z out
        fwd_bytes = csr_bytes(nnzM, n, es) + 4 * n + 3 * vec
        adj_bytes = csr_bytes(nnzL, n, es) + csr_bytes(nnzM, n, es) + 5 * vec + es * (nnzL + nnzM)
        # fused adjoint kernel alone: L^T and A^T (pattern, values), gz in, lam and gx out
        adj_exec_bytes = csr_bytes(nnzL, n, es) + csr_bytes(nnzM, n, es) + 3 * vec
        fwd_flops = 2 * (nnzL + nnzM) * k + n * k
        adj_flops = 2 * (nnzL + nnzM) * k + n * k
    elif w.pair == "ic0_trsv":
        # read tril(A) values + pattern, write factor values, b in, y out
        fwd_bytes = csr_bytes(nnzL, n, es) + es * nnzL + 2 * vec
        fwd_flops = 2 * nnzL * k + n * k + 4 * nnzL    # solve; factor: divide, square, sum per entry
    elif w.pair == "trsv_trsv":
        fwd_bytes = csr_bytes(nnzL, n, es) + 3 * vec                           # b in, x and z out
        fwd_flops = 4 * nnzL * k + 2 * n * k
    else:  # ilu0_trsv: A (pattern, values, diagonal positions) in, factor out, b in, y out
        fwd_bytes = csr_bytes(nnzM, n, es) + 4 * n + es * nnzM + 2 * vec
        fwd_flops = 2 * nnzL * k + 2 * nnzM
    return dict(w=w, name=name, pair=w.pair, n=n, k=k, nnzL=nnzL, nnzM=nnzM, adj=adj, es=es, dtype=dtype_name,
                fwd_bytes=fwd_bytes, adj_bytes=adj_bytes, adj_exec_bytes=adj_exec_bytes, fwd_flops=fwd_flops,
                adj_flops=adj_flops, fits_l2=(fwd_bytes < 129e6))


def _concat(instances, which):
    """Block-diagonal concatenation of the instances' patterns (host)."""
    from paper_2111_12238_gb300 import inputs as I
    rp, ci, off, offn = [np.zeros(1, dtype=np.int64)], [], 0, 0
    for x in instances:
        m = getattr(x, which)
        rp.append(m.rowptr[1:].astype(np.int64) + off)
        ci.append(m.colidx.astype(np.int64) + offn)
        off += m.nnz
        offn += x.n
    vals = np.concatenate([getattr(x, which).vals for x in instances])
    return I.Csr(offn, offn, np.concatenate(rp).astype(np.int32), np.concatenate(ci).astype(np.int32), vals)


def _transposed(torch, rp, ci, vals, n, rev_rows, rev_cols):
    """CSR of the transpose of (rp, ci, vals) on the device, rows and/or columns reversed
    (i -> n - 1 - i): the reversed transpose of a lower-triangular L is lower triangular
    again, so the unfused adjoint can run its upper solve as a forward solve."""
    dev = rp.device
    rows = torch.repeat_interleave(torch.arange(n, device=dev), (rp[1:] - rp[:-1]).long())
    nr = ci.long()
    nc = rows
    if rev_rows:
        nr = (n - 1) - nr
    if rev_cols:
        nc = (n - 1) - nc
    order = torch.argsort(nr * n + nc)
    counts = torch.bincount(nr, minlength=n)
    trp = torch.zeros(n + 1, dtype=torch.int32, device=dev)
    trp[1:] = torch.cumsum(counts, 0).to(torch.int32)
    return trp, nc[order].to(torch.int32), vals[order]


class Gpu:
    """Device state of one workload: the fused schedule, resident inputs and outputs, and the
    unfused two-launch paths of its forward and adjoint passes."""

    def __init__(self, wl, device, launch_opts=None):
        import torch
        from paper_2111_12238_gb300 import sparsefusion as sf
        launch_opts = launch_opts or {}
        self.torch, self.sf, self.wl = torch, sf, wl
        w = wl["w"]
        dt = torch.float64 if wl["dtype"] == "f64" else torch.float32
        self.dt = dt
        T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device=device, dtype=dt)
        pair = self.pair = w.pair
        n = self.n = w.n
        if w.instances:
            L, M = _concat(w.instances, "L"), _concat(w.instances, "M")
        else:
            L, M = w.L, w.M
        self.L_dev = sf.DeviceCsr.from_host(L, device)
        self.M_dev = sf.DeviceCsr.from_host(M, device) if M is not None else None
        t0 = time.perf_counter()
        if w.instances:
            Ls = [sf.DeviceCsr.from_host(x.L, device) for x in w.instances]
            Ms = [sf.DeviceCsr.from_host(x.M, device) for x in w.instances]
            self.sched = sf.inspect_batched(pair, Ls, Ms, want_adjoint=wl["adj"], **launch_opts)
        else:
            self.sched = sf.inspect(pair, self.L_dev, self.M_dev, want_adjoint=wl["adj"], **launch_opts)
        torch.cuda.synchronize()
        self.inspect_s = time.perf_counter() - t0
        self.Lv = T(L.vals)
        self.Mv = T(M.vals) if M is not None else None
        self.b = T(w.b)
        self.x_in = T(w.x_in) if w.x_in is not None else None
        self.gy = T(w.gy) if w.gy is not None else None
        self.y = torch.empty_like(self.b)
        self.xs = {"trsv_spmv": lambda: torch.empty_like(self.b), "trsv_trsv": lambda: torch.empty_like(self.b),
                   "ic0_trsv": lambda: torch.empty(self.Lv.numel(), device=device, dtype=dt),
                   "ilu0_trsv": lambda: torch.empty(self.Mv.numel(), device=device, dtype=dt)}.get(pair,
                                                                                              lambda: None)()
        self.tmp = torch.empty_like(self.b)
        self.tmp2 = torch.empty_like(self.b)
        # unfused forward: the single-kernel schedules (none for SpILU0 -> SpTRSV)
        self.un_sched = None
        if pair in ("trsv_spmv", "spmv_trsv", "trsv_trsv"):
            self.un_sched = sf.inspect("trsv", self.L_dev, **launch_opts)
        elif pair == "ic0_trsv":
            self.un_sched = sf.inspect("ic0", self.L_dev, **launch_opts)
            self.un_sched2 = sf.inspect("trsv", self.L_dev, **launch_opts)
        if wl["adj"]:
            self.gb = torch.empty_like(self.b)
            self.gL = torch.empty_like(self.Lv)
            self.gM = torch.empty_like(self.Mv)
            self.gx = torch.empty_like(self.x_in) if self.x_in is not None else None
            self._unfused_adjoint_setup(device, launch_opts)

    def _unfused_adjoint_setup(self, device, launch_opts):
        """The adjoint's solve as two launches: L^T's upper solve runs as a forward solve of the
        reversed transpose Ur = P L^T P (P reverses the row order), whose right-hand side and
        solution are kept in reversed order; the SpMV with M^T (A^T) reads or writes that order
        through a transpose with reversed rows (columns)."""
        torch, sf = self.torch, self.sf
        n = self.n
        L = self.L_dev
        urp, uci, uv = _transposed(torch, L.rowptr, L.colidx, self.Lv, n, True, True)
        self.Ur = sf.DeviceCsr(n, n, urp, uci)
        self.Urv = uv
        M = self.M_dev
        rev_rows = self.pair == "trsv_spmv"     # u_r = (P M^T) gy; gx = -(A^T P) lam_r
        trp, tci, tv = _transposed(torch, M.rowptr, M.colidx, self.Mv, n, rev_rows, not rev_rows)
        self.MT = sf.DeviceCsr(n, n, trp, tci)
        self.MTv = tv
        self.un_adj = sf.inspect("trsv", self.Ur, **launch_opts)
        self.gy_rev = torch.flip(self.gy, [0]).contiguous()
        self.zero = torch.zeros_like(self.b)
        self.lam_r = torch.empty_like(self.b)
        self.u_r = torch.empty_like(self.b)
        self.gx_u = torch.empty_like(self.b)
        torch.cuda.synchronize()

    def fwd(self):
        # SpMV -> SpTRSV reads L = tril(A) from A's rows (shared storage)
        Lv = None if self.pair in ("spmv_trsv", "ilu0_trsv") else self.Lv
        self.sched.execute(Lv, self.Mv, b=self.b, x_in=self.x_in, y=self.y, x_save=self.xs)

    def adj(self, grads=True):
        s = self.sched
        gL, gM = (self.gL, self.gM) if grads else (None, None)
        if self.pair == "trsv_spmv":
            s.adjoint(self.Lv, self.Mv, self.gy, saved=self.xs, gb=self.gb, gL=gL, gM=gM)
        else:
            s.adjoint(self.Lv, self.Mv, self.gy, saved=self.y, x_in=self.x_in, gb=self.gb, gx=self.gx, gL=gL, gM=gM)

    def adj_solve(self):
        """The fused adjoint without the value gradients (what the unfused adjoint computes)."""
        self.adj(grads=False)

    def unfused(self):
        sf = self.sf
        if self.pair == "trsv_spmv":
            self.un_sched.execute(self.Lv, b=self.b, y=self.tmp)
            sf.spmv(self.M_dev, self.Mv, self.tmp, y=self.tmp2)
        elif self.pair == "spmv_trsv":
            sf.spmv(self.M_dev, self.Mv, self.x_in, b=self.b, y=self.tmp)
            self.un_sched.execute(self.Lv, b=self.tmp, y=self.tmp2)
        elif self.pair == "trsv_trsv":
            self.un_sched.execute(self.Lv, b=self.b, y=self.tmp)
            self.un_sched.execute(self.Lv, b=self.tmp, y=self.tmp2)
        elif self.pair == "ic0_trsv":
            self.un_sched.execute(self.Lv, x_save=self.xs)
            self.un_sched2.execute(self.xs, b=self.b, y=self.tmp2)

    def unfused_adj(self):
        sf = self.sf
        if self.pair == "trsv_spmv":     # u = M^T gy, then lam = L^-T u
            sf.spmv(self.MT, self.MTv, self.gy, y=self.u_r)
            self.un_adj.execute(self.Urv, b=self.u_r, y=self.lam_r)
        else:                            # lam = L^-T gz, then gx = -A^T lam
            self.un_adj.execute(self.Urv, b=self.gy_rev, y=self.lam_r)
            sf.spmv(self.MT, self.MTv, self.lam_r, b=self.zero, y=self.gx_u)

    def check(self):
        self.sched.check()
        for s in (self.un_sched, getattr(self, "un_sched2", None), getattr(self, "un_adj", None)):
            if s is not None:
                s.check()


def _time_loop(torch, fns, steps, flush=None, before=None):
    """Runs `steps` iterations of the launches in `fns` on the current stream with CUDA
    events around each launch; returns (total_ms, [per-fn total ms]). flush() runs before
    every step outside the events; before(s), when given, runs on the host before step s."""
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(fns) + 1)] for _ in range(steps)]
    torch.cuda.synchronize()
    for s in range(steps):
        if flush is not None:
            flush()
        if before is not None:
            before(s)
        ev[s][0].record()
        for i, f in enumerate(fns):
            f()
            ev[s][i + 1].record()
    torch.cuda.synchronize()
    per = [0.0] * len(fns)
    total = 0.0
    for s in range(steps):
        for i in range(len(fns)):
            dtm = ev[s][i].elapsed_time(ev[s][i + 1])
            per[i] += dtm
            total += dtm
    return total, per


def _gpu_id(torch, local):
    """nvidia-smi id of this process's GPU (its UUID), falling back to the ordinal."""
    try:
        u = str(torch.cuda.get_device_properties(local).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(local)


class ClockSampler:
    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                s_, m_ = float(r[1]), float(r[2])
            except (ValueError, IndexError):
                continue
            sm.append(s_)
            mx.append(m_)
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- bounds
def roofline_bounds(depth, t_hop_ns, nbytes, hbm_gbs, flops, dtype, kernel_ms, fp64_tflops=None):
    """Lower bounds on one launch of the executor kernel, in ms: the dependence chain (depth x
    one hand-off), the HBM stream of its algorithmic bytes and, for FP64, its algorithmic flops
    at the FP64 rate (measured when given, else the nominal 1.25 TFLOP/s); the tightest of them
    and the fraction of it achieved."""
    b = {"latency": depth * t_hop_ns * 1e-6, "hbm": nbytes / (hbm_gbs * 1e9) * 1e3}
    rate = fp64_tflops if fp64_tflops else FP64_NOMINAL_TFLOPS
    if dtype == "f64" and flops:
        b["fp64"] = flops / (rate * 1e12) * 1e3
    tight = max(b, key=b.get)
    return {"latency_bound_ms": b["latency"], "hbm_bound_ms": b["hbm"], "fp64_bound_ms": b.get("fp64"),
            "fp64_peak_tflops": rate if "fp64" in b else None,
            "fp64_peak_source": ("measured (FMA kernel)" if fp64_tflops else "nominal") if "fp64" in b else None,
            "algorithmic_flops_per_launch": flops, "tightest_bound": tight,
            "frac_of_tightest_bound": b[tight] / kernel_ms if kernel_ms > 0 else None}


# ----------------------------------------------------------------------------- ranks
def max_over_ranks(x, world, device):
    """The largest of one float per rank, on every rank (torch.distributed, any backend);
    x itself when there is one rank."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(world, steps, slowest_ms):
    """Whole-job throughput: every rank ran `steps` solves; the job took the slowest rank's
    time."""
    return world * steps / (slowest_ms / 1e3)


# ----------------------------------------------------------------------------- one workload
def measure(wl, args, device, world, rank, hw):
    """Times one workload on this GPU and returns its JSON line (rank 0) or None."""
    import torch
    from paper_2111_12238_gb300 import autotune
    g = Gpu(wl, device, dict(epoch_flags=args.epoch_flags, dynamic_queue=args.dynamic_queue))
    adj = wl["adj"]
    fns = [g.fwd] + ([g.adj] if adj else [])
    flush_buf = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=device)
    flush = lambda: flush_buf.zero_()   # noqa: E731  (L2 is 129 MB: every step starts cold)
    for _ in range(args.warmup):
        for f in fns:
            f()
        if g.un_sched is not None:
            g.unfused()
        if adj:
            g.unfused_adj()
    g.check()
    tuned = {}
    packing_ablation = None
    if not args.no_tune:
        # the project's autotuner picks each pass's launch shape, the unfused paths included
        kw = dict(dtype=g.dt, k=wl["k"], budget_s=args.tune_seconds, use_cache=False)
        tuned["fwd"] = autotune.tune(g.sched, g.fwd, which=0, **kw)
        if adj:
            tuned["adj"] = autotune.tune(g.sched, g.adj, which=1, **kw)
        if g.un_sched is not None:
            tuned["unfused"] = autotune.tune(g.un_sched, g.unfused, which=0, **kw)
        if adj:
            tuned["unfused_adj"] = autotune.tune(g.un_adj, g.unfused_adj, which=0, **kw)
        # packing ablation (§3.2.3, Fig. 7): the forward's best interleaved and separated trials
        if wl["pair"] == "spmv_trsv":
            tr = tuned["fwd"]["trials"]
            inter = [t["ms"] for t in tr if t.get("packing", 1) == 1]
            sep = [t["ms"] for t in tr if t.get("packing", 1) == 0]
            packing_ablation = {"interleaved_ms": min(inter) if inter else None,
                                "separated_ms": min(sep) if sep else None,
                                "how": "autotuner trials of the fused forward, same launch shape, median of 3"}
        for v in tuned.values():
            v.pop("trials", None)
    steps = args.steps
    if steps is None:   # about a second of device time, 20 to 2000 steps
        one, _ = _time_loop(torch, fns, 3, flush)
        steps = int(min(2000, max(20, 1000.0 / max(one / 3, 1e-3))))

    # ---- timed region (device-resident inputs); the fused executor kernel of each pass is
    # also timed alone with events the library records around it on the launch stream
    dirs = [0] + ([1] if adj else [])
    kev = {d: [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)] for d in dirs}
    for pairs in kev.values():      # torch creates an event at its first record
        for a_, b_ in pairs:
            a_.record()
            b_.record()

    def before(s):
        for d in dirs:
            g.sched.set_exec_events(d, *kev[d][s])

    clk = ClockSampler(_gpu_id(torch, int(str(device).split(":")[-1])))
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    total_ms, per = _time_loop(torch, fns, steps, flush, before)
    clocks = clk.stop()
    for d in dirs:
        g.sched.set_exec_events(d, None, None)
    exec_ms = {d: sum(a_.elapsed_time(b_) for a_, b_ in kev[d]) / steps for d in dirs}
    g.check()
    total_ms = max_over_ranks(total_ms, world, device)
    value = job_value(world, steps, total_ms)
    fwd_ms = per[0] / steps
    adj_ms = per[1] / steps if adj else None

    # ---- unfused two-launch paths and the fused adjoint's solve alone, same GPU
    reps = max(10, steps // 4)
    un_ms = un_adj_ms = adj_solve_ms = None
    if g.un_sched is not None:
        un_ms = _time_loop(torch, [g.unfused], reps, flush)[0] / reps
    if adj:
        un_adj_ms = _time_loop(torch, [g.unfused_adj], reps, flush)[0] / reps
        adj_solve_ms = _time_loop(torch, [g.adj_solve], reps, flush)[0] / reps
    g.check()

    # ---- end to end through the public calls with host buffers
    pin_in = [g.b.cpu().pin_memory()] + ([g.gy.cpu().pin_memory()] if adj else [])
    dev_in = [g.b] + ([g.gy] if adj else [])
    dev_out = [g.y] + ([g.gb, g.gL, g.gM] + ([g.gx] if g.gx is not None else []) if adj else [])
    pin_out = [torch.empty(t_.shape, dtype=t_.dtype, pin_memory=True) for t_ in dev_out]

    def e2e_step():
        for d_, h_ in zip(dev_in, pin_in):
            d_.copy_(h_, non_blocking=True)
        for f in fns:
            f()
        for h_, d_ in zip(pin_out, dev_out):
            h_.copy_(d_, non_blocking=True)
        torch.cuda.current_stream().synchronize()

    e2e_steps = max(5, steps // 10)
    for _ in range(2):
        e2e_step()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, device)
    g.check()
    h2d = sum(t_.numel() * t_.element_size() for t_ in pin_in)
    d2h = sum(t_.numel() * t_.element_size() for t_ in pin_out)
    if rank != 0:
        return None

    hbm, peak_src = _peaks()
    info = g.sched.info()
    dom = "fwd" if (1 not in exec_ms or exec_ms[0] >= exec_ms[1]) else "adj"
    dom_ms = exec_ms[0] if dom == "fwd" else exec_ms[1]
    dom_bytes = wl["fwd_bytes"] if dom == "fwd" else wl["adj_exec_bytes"]
    dom_flops = wl["fwd_flops"] if dom == "fwd" else wl["adj_flops"]
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9
    depth = info["depth"] if dom == "fwd" else info["adj_depth"]
    mode = info["exec_mode" if dom == "fwd" else "adj_exec_mode"]
    w = wl["w"]
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "solves/s",
        "n_gpus": world,
        "steps": steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": wl["dtype"],
        "data": "synthetic (seeded generators standing in for the paper's SuiteSparse matrices)",
        "config": {
            "workload": w.name,
            "pair": wl["pair"],
            "n": wl["n"], "k": wl["k"], "nnz_L": wl["nnzL"], "nnz_M": wl["nnzM"],
            "step": "one fused forward pass" + (" + one fused adjoint pass with both value gradients" if adj else ""),
            "l2": "flushed (256 MB write) before every step, outside the timed launches",
            "parallelism": "replicas" if world > 1 else "single GPU",
            "instances": len(w.instances) or 1,
        },
        "roofline": {
            "kernel": ("fused forward executor kernel" if dom == "fwd" else "fused adjoint executor kernel") +
                      {2: " (row blocks)", 3: " (warp-specialised row blocks)", 4: " (packed row blocks)",
                       5: " (single CTA per instance)"}.get(mode, " (partitions)"),
            "kernel_ms": dom_ms,
            "bound": "hbm",
            "achieved": achieved,
            "peak": hbm,
            "unit": "GB/s",
            "frac": achieved / hbm,
            "traffic": _recorded_traffic(wl["name"], dom),
            "peak_source": peak_src,
            "algorithmic_bytes_per_launch": dom_bytes,
            "hop_ns_measured": hw["hop_ns"],
            "executor_ns_per_wavefront": dom_ms * 1e6 / max(depth, 1),
            **roofline_bounds(depth, hw["hop_ns"], dom_bytes, hbm, dom_flops, wl["dtype"], dom_ms,
                              hw["fp64_tflops"]),
        },
        "fwd_ms": fwd_ms,
        "fwd_exec_ms": exec_ms[0],
        "fwd_gbs": wl["fwd_bytes"] / (exec_ms[0] / 1e3) / 1e9,
        "unfused_fwd_ms": un_ms,
        "fused_speedup_vs_unfused": (un_ms / fwd_ms) if un_ms else None,
        "adj_ms": adj_ms,
        "adj_exec_ms": exec_ms.get(1),
        "adj_solve_ms": adj_solve_ms,
        "unfused_adj_solve_ms": un_adj_ms,
        "adj_fused_speedup_vs_unfused": (un_adj_ms / adj_solve_ms) if adj else None,
        "adjoint_fwd_ratio": (adj_ms / fwd_ms) if adj else None,
        "adj_gbs": (wl["adj_bytes"] / (adj_ms / 1e3) / 1e9) if adj else None,
        "depth": info["depth"], "adj_depth": info["adj_depth"],
        "inspect_ms": g.inspect_s * 1e3,
        "ner_vs_unfused": (g.inspect_s * 1e3 / (un_ms - fwd_ms)) if (un_ms and un_ms > fwd_ms) else None,
        "tuned": tuned,
        "packing_ablation": packing_ablation,
        "e2e": {"value": job_value(world, e2e_steps, e2e_s * 1e3), "unit": "solves/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        # our kernels per step, as the library counts them for the tuned launch shapes:
        # pre-passes, value gathers, fused kernels and gradient passes
        "gpu_launches": steps * (g.sched.launches(0, wl["k"]) + (g.sched.launches(1, wl["k"]) if adj else 0)),
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, args.cpu_seconds)
    del g
    torch.cuda.empty_cache()
    return line


# ----------------------------------------------------------------------------- the oracle
def _oracle_step(w, adj):
    import oracle
    items = w.instances if w.instances else [w]

    def step():
        for x in items:
            if x.pair == "trsv_spmv":
                xx, _ = oracle.trsv_spmv(x.L, x.M, x.b)
                if adj:
                    oracle.adj_trsv_spmv(x.L, x.M, xx, x.gy)
            elif x.pair == "spmv_trsv":
                z = oracle.spmv_trsv(x.M, x.L, x.x_in, x.b)
                if adj:
                    oracle.adj_spmv_trsv(x.M, x.L, x.x_in, z, x.gy)
            elif x.pair == "ic0_trsv":
                oracle.ic0_trsv(x.L, x.b)
            elif x.pair == "trsv_trsv":
                oracle.trsv_trsv(x.L, x.b)
            else:
                oracle.ilu0_trsv(x.M, x.b)
    return step


def cpu_baseline(wl, seconds):
    """The sequential FP64 oracle (one host core) on the same workload, whole steps repeated
    for about `seconds` (at least one step)."""
    step = _oracle_step(wl["w"], wl["adj"])
    t0 = time.perf_counter()
    reps = 0
    while True:
        step()
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return {"value": reps / el, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"{reps} full step(s) of the workload ({el:.1f} s), single-threaded C FP64, "
                      f"host has {os.cpu_count()} cores"}


def _leading_rows(w, m):
    """The leading m rows (and columns) of a SpMV -> SpTRSV workload: the oracle's bounded
    sample for the reference arm (entries of A in columns >= m are dropped)."""
    from paper_2111_12238_gb300 import inputs as I

    def lead(M):
        rp = M.rowptr[:m + 1].astype(np.int64)
        ci = M.colidx[:rp[-1]]
        vv = M.vals[:rp[-1]]
        keep = ci < m
        rows = np.repeat(np.arange(m), np.diff(rp))
        lengths = np.bincount(rows[keep], minlength=m)
        nrp = np.zeros(m + 1, dtype=np.int64)
        nrp[1:] = np.cumsum(lengths)
        return I.Csr(m, m, nrp.astype(np.int32), ci[keep].astype(np.int32), vv[keep])

    return I.Workload(w.name + f"_leading_{m}", w.pair, m, w.k, lead(w.L), lead(w.M), w.b[:m], x_in=w.x_in[:m],
                      gy=w.gy[:m])


# ----------------------------------------------------------------------------- arms
def hardware_bounds(torch):
    """Measured once per run: the FP64 FMA rate and the SM-to-SM hand-off latency of this
    GPU, by the library's measurement kernels."""
    from paper_2111_12238_gb300 import sparsefusion as sf
    fp64 = sf.bench_fma_tflops(torch.float64)
    fp32 = sf.bench_fma_tflops(torch.float32)
    hops = [sf.bench_hop_ns(20000) for _ in range(3)]
    return {"fp64_tflops": fp64, "fp32_tflops": fp32, "hop_ns": min(hops),
            "how": "FMA rate: 8 independent FMA chains per thread, 8 blocks of 256 threads per SM, best of 5 "
                   "(CUDA events); hop: one uint32 handed 20,000 times between two SMs through L2 (relaxed "
                   "store, polling relaxed load), best of 3"}


def run_gpu(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    device = f"cuda:{local}"
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(device))
    import __graft_entry__
    __graft_entry__.build()
    hw = hardware_bounds(torch)
    names = ORDER if args.workload == "all" else [args.workload]
    lines = {}
    for name in names:
        wl = make_workload(name, args.dtype)
        line = measure(wl, args, device, world, rank, hw)
        if rank == 0:
            print(json.dumps(line), file=sys.stderr, flush=True)
            lines[name] = line
    if rank == 0:
        if len(names) == 1:
            out = lines[names[0]]
        else:
            out = lines[HEADLINE]
            out["workloads"] = [lines[nm] for nm in names if nm != HEADLINE]
        out["hardware"] = hw
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_reference(args):
    """The oracle alone (sequential FP64 C, one host core) on the headline workload: every
    step is the forward and adjoint of the leading eighth of its rows, the value scaled to
    whole solves per second."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    name = HEADLINE if args.workload == "all" else args.workload
    wl = make_workload(name, "f64")
    w = wl["w"]
    frac = 1.0
    if w.pair == "spmv_trsv" and not w.instances and w.n >= (1 << 20):
        frac = 0.125
        w = _leading_rows(w, int(w.n * frac))
    step = _oracle_step(w, wl["adj"])
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = time.perf_counter() - t0
    v = args.steps / el * frac
    sample = (f"{args.steps} steps on the leading {w.n} of {wl['n']} rows (value scaled by {frac})" if frac < 1
              else f"{args.steps} full steps") + ", single-threaded C FP64"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded generators standing in for the paper's SuiteSparse matrices)",
            "config": {"workload": wl["w"].name, "pair": wl["pair"], "n": wl["n"], "k": wl["k"],
                       "step": "oracle forward" + (" + adjoint" if wl["adj"] else "")},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=None)
    ap.add_argument("--impl", default="fused", choices=["fused", "reference"])
    ap.add_argument("--workload", default="all", choices=["all"] + ORDER)
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32"])
    ap.add_argument("--cpu-seconds", type=float, default=4.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--epoch-flags", action="store_true", help="publish through epoch flags even for k = 1")
    ap.add_argument("--dynamic-queue", action="store_true", help="draw partitions from a ticket counter")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (use the default launch shape)")
    ap.add_argument("--tune-seconds", type=float, default=3.0, help="time budget of each autotuning search")
    args = ap.parse_args()
    if args.impl == "reference":
        args.steps = args.steps if args.steps is not None else 20
        args.warmup = args.warmup if args.warmup is not None else 3
        run_reference(args)
        return
    args.warmup = max(3, args.warmup if args.warmup is not None else 5)
    run_gpu(args)


if __name__ == "__main__":
    main()
