"""Sequential FP64 CPU oracle for the sparse-fusion hot path (ctypes over sf_oracle.c).

TEST INFRASTRUCTURE. Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The library in ``paper_2111_12238_gb300`` never
does, and nothing here imports the library: the only code both sides share is the seeded
input generator module, which holds none of the method's arithmetic.

Every routine is the plain definition run unfused in program order (see the header of
sf_oracle.c). Functions take and return numpy arrays; CSR arguments are any object with
``n_rows``, ``n_cols``, ``rowptr`` (int32), ``colidx`` (int32) and ``vals`` (float64).

Pins: the oracle is checked against dense solves, dense Cholesky, closed forms, exact
integer arithmetic and invariants in tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sf_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libsforacle.so")
_lock = threading.Lock()
_lib = None

# schedule kinds of sf_oracle.c
SEP, PAIRED, PAIRED_T, SEP_T = 0, 1, 2, 3
# cost formulas of orc_costs
(COST_SEP, COST_PAIRED_T, COST_SEP_T, COST_SPMV_TRSV, COST_IC0_TRSV, COST_TRSV, COST_IC0, COST_TRSV_TRSV,
 COST_ILU0_TRSV) = range(9)


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: oracle status {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile sf_oracle.c with gcc into oracle/_lib/libsforacle.so. Floating-point
    contraction is off so every operation rounds exactly as written."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            for name in ("orc_trsv_lower", "orc_spmv", "orc_residual", "orc_ic0", "orc_trsv_lower_T",
                         "orc_spmv_T", "orc_trsv_spmv", "orc_spmv_trsv", "orc_ic0_trsv",
                         "orc_adj_trsv_spmv", "orc_adj_spmv_trsv", "orc_levels", "orc_costs",
                         "orc_order", "orc_validate", "orc_trsv_trsv", "orc_ilu0", "orc_ilu0_trsv"):
                getattr(lib, name).restype = C.c_int
            lib.orc_partition.restype = C.c_int64
            lib.orc_block_order.restype = C.c_int64
            lib.orc_block_order_instances.restype = C.c_int64
            lib.orc_block_segments.restype = C.c_int64
            lib.orc_reuse_ratio.restype = C.c_double
            lib.orc_reuse_ratio.argtypes = [C.c_int32, C.c_int64, C.c_int64, C.c_int64]
            _lib = lib
    return _lib


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(C.c_void_p)


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.c_void_p)


def _out(shape, dtype=np.float64):
    a = np.zeros(shape, dtype=dtype)
    return a, a.ctypes.data_as(C.c_void_p)


def _csr(M):
    rp, prp = _i32(M.rowptr)
    ci, pci = _i32(M.colidx)
    v, pv = _f64(M.vals)
    return (rp, ci, v), prp, pci, pv


def _block(x, n):
    x = np.asarray(x, dtype=np.float64)
    if x.ndim == 1:
        x = x.reshape(n, 1)
    return x


def _check(rc, what):
    if rc != 0:
        raise OracleError(rc, what)


# ---------------------------------------------------------------------- kernels
def trsv_lower(L, b):
    """x = L^-1 b by forward substitution."""
    lib = _load()
    b = _block(b, L.n_rows)
    keep, rp, ci, v = _csr(L)
    bb, pb = _f64(b)
    x, px = _out(b.shape)
    _check(lib.orc_trsv_lower(C.c_int32(L.n_rows), C.c_int32(b.shape[1]), rp, ci, v, pb, px), "trsv")
    return x


def spmv(M, x):
    lib = _load()
    x = _block(x, M.n_cols)
    keep, rp, ci, v = _csr(M)
    xx, px = _f64(x)
    y, py = _out((M.n_rows, x.shape[1]))
    lib.orc_spmv(C.c_int32(M.n_rows), C.c_int32(x.shape[1]), rp, ci, v, px, py)
    return y


def residual(M, x, b):
    lib = _load()
    x = _block(x, M.n_cols)
    b = _block(b, M.n_rows)
    keep, rp, ci, v = _csr(M)
    xx, px = _f64(x)
    bb, pb = _f64(b)
    r, pr = _out(b.shape)
    lib.orc_residual(C.c_int32(M.n_rows), C.c_int32(x.shape[1]), rp, ci, v, px, pb, pr)
    return r


def ic0(L):
    """Zero fill-in incomplete Cholesky factor values on the pattern of L = tril(A)."""
    lib = _load()
    keep, rp, ci, v = _csr(L)
    lf, pl = _out(L.nnz)
    _check(lib.orc_ic0(C.c_int32(L.n_rows), rp, ci, v, pl), "ic0")
    return lf


def trsv_lower_T(L, u):
    lib = _load()
    u = _block(u, L.n_rows)
    keep, rp, ci, v = _csr(L)
    uu, pu = _f64(u)
    lam, pl = _out(u.shape)
    _check(lib.orc_trsv_lower_T(C.c_int32(L.n_rows), C.c_int32(u.shape[1]), rp, ci, v, pu, pl),
           "trsv_T")
    return lam


def spmv_T(M, g):
    lib = _load()
    g = _block(g, M.n_rows)
    keep, rp, ci, v = _csr(M)
    gg, pg = _f64(g)
    u, pu = _out((M.n_cols, g.shape[1]))
    lib.orc_spmv_T(C.c_int32(M.n_rows), C.c_int32(M.n_cols), C.c_int32(g.shape[1]), rp, ci, v, pg, pu)
    return u


# ---------------------------------------------------------------------- pairs
def trsv_spmv(L, M, b):
    """(x, y) with x = L^-1 b and y = M x."""
    lib = _load()
    b = _block(b, L.n_rows)
    kl, lrp, lci, lv = _csr(L)
    km, mrp, mci, mv = _csr(M)
    bb, pb = _f64(b)
    x, px = _out(b.shape)
    y, py = _out(b.shape)
    _check(lib.orc_trsv_spmv(C.c_int32(L.n_rows), C.c_int32(b.shape[1]), lrp, lci, lv, mrp, mci, mv,
                             pb, px, py), "trsv_spmv")
    return x, y


def spmv_trsv(A, L, x_in, b):
    """z = L^-1 (b - A x_in)."""
    lib = _load()
    b = _block(b, L.n_rows)
    x_in = _block(x_in, A.n_cols)
    ka, arp, aci, av = _csr(A)
    kl, lrp, lci, lv = _csr(L)
    xx, px = _f64(x_in)
    bb, pb = _f64(b)
    z, pz = _out(b.shape)
    _check(lib.orc_spmv_trsv(C.c_int32(L.n_rows), C.c_int32(b.shape[1]), arp, aci, av, lrp, lci, lv,
                             px, pb, pz), "spmv_trsv")
    return z


def ic0_trsv(L, b):
    """(lfac, y): zero fill-in IC factor of tril(A) (values on L's pattern), y = lfac^-1 b."""
    lib = _load()
    b = _block(b, L.n_rows)
    kl, rp, ci, v = _csr(L)
    bb, pb = _f64(b)
    lf, pl = _out(L.nnz)
    y, py = _out(b.shape)
    _check(lib.orc_ic0_trsv(C.c_int32(L.n_rows), C.c_int32(b.shape[1]), rp, ci, v, pb, pl, py),
           "ic0_trsv")
    return lf, y


def trsv_trsv(L, b):
    """(x, z): x = L^-1 b, then z = L^-1 x (Table 2 combination 1)."""
    lib = _load()
    b = _block(b, L.n_rows)
    keep, rp, ci, v = _csr(L)
    bb, pb = _f64(b)
    x, px = _out(b.shape)
    z, pz = _out(b.shape)
    _check(lib.orc_trsv_trsv(C.c_int32(L.n_rows), C.c_int32(b.shape[1]), rp, ci, v, pb, px, pz), "trsv_trsv")
    return x, z


def ilu0(A):
    """Zero fill-in incomplete LU of A on A's pattern: the strictly lower part of the unit
    lower factor and the upper factor with its diagonal (Table 2 combination 6)."""
    lib = _load()
    keep, rp, ci, v = _csr(A)
    lu, pl = _out(A.nnz)
    _check(lib.orc_ilu0(C.c_int32(A.n_rows), rp, ci, v, pl), "ilu0")
    return lu


def ilu0_trsv(A, b):
    """(lu, y): ILU0 of A, then y = L^-1 b with its unit lower factor."""
    lib = _load()
    b = _block(b, A.n_rows)
    keep, rp, ci, v = _csr(A)
    bb, pb = _f64(b)
    lu, pl = _out(A.nnz)
    y, py = _out(b.shape)
    _check(lib.orc_ilu0_trsv(C.c_int32(A.n_rows), C.c_int32(b.shape[1]), rp, ci, v, pb, pl, py), "ilu0_trsv")
    return lu, y


def adj_trsv_spmv(L, M, x, gy):
    """(gb, gL, gM) for y = M L^-1 b with x = L^-1 b."""
    lib = _load()
    n = L.n_rows
    x = _block(x, n)
    gy = _block(gy, n)
    kl, lrp, lci, lv = _csr(L)
    km, mrp, mci, mv = _csr(M)
    xx, px = _f64(x)
    gg, pg = _f64(gy)
    gb, pgb = _out(x.shape)
    gL, pgL = _out(L.nnz)
    gM, pgM = _out(M.nnz)
    _check(lib.orc_adj_trsv_spmv(C.c_int32(n), C.c_int32(x.shape[1]), lrp, lci, lv, mrp, mci, mv,
                                 px, pg, pgb, pgL, pgM), "adj_trsv_spmv")
    return gb, gL, gM


def adj_spmv_trsv(A, L, x_in, z, gz):
    """(gb, gx, gL, gA) for z = L^-1 (b - A x_in)."""
    lib = _load()
    n = L.n_rows
    x_in = _block(x_in, n)
    z = _block(z, n)
    gz = _block(gz, n)
    ka, arp, aci, av = _csr(A)
    kl, lrp, lci, lv = _csr(L)
    xx, px = _f64(x_in)
    zz, pz = _f64(z)
    gg, pg = _f64(gz)
    gb, pgb = _out(z.shape)
    gx, pgx = _out(z.shape)
    gL, pgL = _out(L.nnz)
    gA, pgA = _out(A.nnz)
    _check(lib.orc_adj_spmv_trsv(C.c_int32(n), C.c_int32(z.shape[1]), arp, aci, av, lrp, lci, lv,
                                 px, pz, pg, pgb, pgx, pgL, pgA), "adj_spmv_trsv")
    return gb, gx, gL, gA


# ---------------------------------------------------------------------- schedules
def n_vertices(kind, n):
    return 2 * n if kind in (SEP, SEP_T) else n


def levels(kind, L, M=None, g2=0):
    """Wavefront of every joint-DAG vertex; g2 places the second kernel's vertices of a
    separated schedule (0 earliest, -1 last wavefront, d > 0 delayed by d)."""
    lib = _load()
    n = L.n_rows
    kl, lrp, lci, _ = _csr(L)
    if M is not None:
        km, mrp, mci, _ = _csr(M)
    else:
        mrp = mci = None
    lev, pl = _out(n_vertices(kind, n), np.int32)
    _check(lib.orc_levels(C.c_int32(kind), C.c_int32(n), lrp, lci, mrp, mci, pl), "levels")
    if g2:
        lib.orc_place_g2(C.c_int32(kind), C.c_int32(n), pl, C.c_int32(int(g2)))
    return lev


def costs(what, L, M=None):
    lib = _load()
    n = L.n_rows
    kl, lrp, lci, _ = _csr(L)
    if M is not None:
        km, mrp, mci, _ = _csr(M)
    else:
        mrp = mci = None
    nv = 2 * n if what in (COST_SEP, COST_SEP_T) else n
    c, pc = _out(nv, np.int64)
    _check(lib.orc_costs(C.c_int32(what), C.c_int32(n), lrp, lci, mrp, mci, pc), "costs")
    return c


def order(level, n):
    """(order, depth): vertices sorted by (level, tag, row), encoded row | tag << 31."""
    lib = _load()
    lev, pl = _i32(level)
    o, po = _out(len(lev), np.int32)
    depth = lib.orc_order(C.c_int64(len(lev)), C.c_int32(n), pl, po)
    if depth < 0:
        raise OracleError(depth, "order")
    return o, depth


def partition(order_, n, cost, target, wide=0):
    """Partition pointers of the cut (items of cost > wide, if wide > 0, stand alone)."""
    lib = _load()
    o, po = _i32(order_)
    c = np.ascontiguousarray(cost, dtype=np.int64)
    pp, ppp = _out(len(o) + 1, np.int32)
    P = lib.orc_partition(C.c_int64(len(o)), C.c_int32(n), po, c.ctypes.data_as(C.c_void_p),
                          C.c_int64(int(target)), C.c_int64(int(wide)), ppp)
    return pp[: P + 1].copy()


def block_order(kind, L, M, level, B):
    """(order, block_ptr) of the row-block schedule with blocks of B rows."""
    lib = _load()
    n = L.n_rows
    kl, lrp, lci, _ = _csr(L)
    if M is not None:
        km, mrp, mci, _ = _csr(M)
    else:
        mrp = mci = None
    lev, pl = _i32(level)
    o, po = _out(len(lev), np.int32)
    nb = -(-n // int(B))
    bp, pbp = _out(nb + 1, np.int32)
    got = lib.orc_block_order(C.c_int32(kind), C.c_int32(n), lrp, lci, mrp, mci, pl, C.c_int64(int(B)), po, pbp)
    if got < 0:
        raise OracleError(got, "block_order")
    return o, bp


def block_order_instances(kind, n, level, inst_ptr):
    """(order, block_ptr) with one block per instance of a block-diagonal system."""
    lib = _load()
    lev, pl = _i32(level)
    ip, pip = _i32(inst_ptr)
    o, po = _out(len(lev), np.int32)
    bp, pbp = _out(len(ip), np.int32)
    got = lib.orc_block_order_instances(C.c_int32(kind), C.c_int32(int(n)), pl, C.c_int32(len(ip) - 1), pip, po, pbp)
    if got < 0:
        raise OracleError(got, "block_order_instances")
    return o, bp


def block_segments(kind, n, order_, block_ptr, level):
    """(seg_ptr, block_seg) of a row-block order: runs of positions with one block and level."""
    lib = _load()
    o, po = _i32(order_)
    bp, pbp = _i32(block_ptr)
    lev, pl = _i32(level)
    nb = len(bp) - 1
    sp, psp = _out(len(o) + 1, np.int32)
    bs, pbs = _out(nb + 1, np.int32)
    ns = lib.orc_block_segments(C.c_int32(kind), C.c_int32(n), C.c_int64(nb), po, pbp, pl, psp, pbs)
    if ns < 0:
        raise OracleError(ns, "block_segments")
    return sp[:ns + 1].copy(), bs


def validate(kind, L, M, order_, part_ptr):
    lib = _load()
    n = L.n_rows
    kl, lrp, lci, _ = _csr(L)
    if M is not None:
        km, mrp, mci, _ = _csr(M)
    else:
        mrp = mci = None
    o, po = _i32(order_)
    pp, ppp = _i32(part_ptr)
    return lib.orc_validate(C.c_int32(kind), C.c_int32(n), lrp, lci, mrp, mci, po, C.c_int64(len(o)),
                            ppp, C.c_int64(len(pp) - 1))


def schedule(kind, what, L, M, target, wide=0, g2=0):
    """Levels, order and partition pointers of one schedule, as the inspector must build
    them: returns dict(level, order, part_ptr, depth, cost)."""
    lev = levels(kind, L, M, g2)
    o, depth = order(lev, L.n_rows)
    c = costs(what, L, M)
    pp = partition(o, L.n_rows, c, target, wide)
    return dict(level=lev, order=o, part_ptr=pp, depth=depth, cost=c)


def reuse_ratio(pair, n, size_L, size_M):
    return _load().orc_reuse_ratio(int(pair), int(n), int(size_L), int(size_M))
