"""Small-matrix helpers for the tests: dense <-> CSR conversion and tiny structured
patterns. Structural only; no solver arithmetic lives here."""
import numpy as np

from paper_2111_12238_gb300.inputs import Csr, uniform_pm1, uniform_below


def dense_to_csr(D, pattern=None):
    """CSR of D keeping entries where ``pattern`` (default D != 0) is true."""
    D = np.asarray(D, dtype=np.float64)
    P = (D != 0) if pattern is None else np.asarray(pattern, dtype=bool)
    n, m = D.shape
    rowptr = np.zeros(n + 1, dtype=np.int32)
    cols, vals = [], []
    for i in range(n):
        js = np.nonzero(P[i])[0]
        cols.extend(js.tolist())
        vals.extend(D[i, js].tolist())
        rowptr[i + 1] = len(cols)
    return Csr(n, m, rowptr, np.asarray(cols, dtype=np.int32), np.asarray(vals, dtype=np.float64))


def csr_to_dense(M, vals=None):
    v = M.vals if vals is None else vals
    D = np.zeros((M.n_rows, M.n_cols))
    for i in range(M.n_rows):
        for e in range(M.rowptr[i], M.rowptr[i + 1]):
            D[i, M.colidx[e]] = v[e]
    return D


def pattern_dense(M):
    P = np.zeros((M.n_rows, M.n_cols), dtype=bool)
    for i in range(M.n_rows):
        P[i, M.colidx[M.rowptr[i]:M.rowptr[i + 1]]] = True
    return P


def random_lower(n, density, seed, unit_int=False):
    """Random sparse lower-triangular dense matrix with a nonzero diagonal. With
    ``unit_int`` the strict part is in {-1, 0, 1} and the diagonal is 1."""
    idx = np.arange(n * n)
    u = (uniform_pm1(seed, 11, idx).reshape(n, n) + 1) / 2
    keep = np.tril(u < density, -1)
    if unit_int:
        s = uniform_below(seed, 12, idx, 2).reshape(n, n) * 2 - 1
        D = np.where(keep, s, 0).astype(np.float64)
        np.fill_diagonal(D, 1.0)
        return D
    v = uniform_pm1(seed, 13, idx).reshape(n, n)
    D = np.where(keep, v, 0.0)
    np.fill_diagonal(D, 1.0 + np.abs(D).sum(axis=1))
    return D


def random_square(n, density, seed):
    idx = np.arange(n * n)
    u = (uniform_pm1(seed, 21, idx).reshape(n, n) + 1) / 2
    v = uniform_pm1(seed, 22, idx).reshape(n, n)
    return np.where(u < density, v, 0.0)


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.max(np.abs(b)) if b.size else 0.0
    return float(np.max(np.abs(a - b)) / den) if den > 0 else float(np.max(np.abs(a - b), initial=0.0))
