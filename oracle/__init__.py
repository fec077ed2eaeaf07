"""CPU oracle for the embedded-ensemble diffusion problem.

TEST INFRASTRUCTURE ONLY: only `tests/`, `__graft_entry__.smoke()` and the
benchmark's CPU-baseline leg may import this package.  It shares no code with
the CUDA library.  The arithmetic lives in `ens_oracle.c` (plain sequential
FP64 C, per sample); this module builds it with gcc and wraps it with numpy.

Per-sample functions follow the paper (Fig. 2 CRS SpMV, Algorithm 2 assembly,
Sect. 4 KL expansion, CG of Sect. 3.4).  The ensemble helpers at the end only
re-order per-sample results into the commuted layout of Eq. 3
(value of member e of entry i at [i*s + e]); they do no arithmetic.

Every function is pinned by `tests/test_oracle_*.py` against closed forms,
brute force, invariants or published values; none is "parity unpinned".
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ens_oracle.c")
_HDR = os.path.join(_HERE, "ens_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

STATUS_OK, STATUS_NOT_CONVERGED, STATUS_BREAKDOWN = 0, 5, 6


def build(force=False):
    """Compile ens_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fPIC", "-shared",
            _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def _declare(L):
    I, D, I64 = ctypes.c_int, ctypes.c_double, ctypes.c_int64
    L.or_num_rows.restype = I64; L.or_num_rows.argtypes = [I]
    L.or_num_cells.restype = I64; L.or_num_cells.argtypes = [I]
    L.or_node_index.restype = None; L.or_node_index.argtypes = [I, _i32p]
    L.or_graph.restype = I64; L.or_graph.argtypes = [I, _i32p, _i32p]
    L.or_elem_graph.restype = I; L.or_elem_graph.argtypes = [I, _i32p, _i32p, _i32p]
    L.or_bmask.restype = None; L.or_bmask.argtypes = [I, _u8p]
    L.or_kl_1d.restype = I; L.or_kl_1d.argtypes = [I, D, _f64p, _f64p]
    L.or_kl_phi1d.restype = D; L.or_kl_phi1d.argtypes = [I, D, D, D]
    L.or_kl_modes.restype = I; L.or_kl_modes.argtypes = [I, D, _i32p, _f64p]
    L.or_kl_coeff_at.restype = D
    L.or_kl_coeff_at.argtypes = [I, D, D, D, _i32p, _f64p, _f64p, _f64p, _f64p]
    L.or_kl_coeff_qp.restype = I; L.or_kl_coeff_qp.argtypes = [I, I, D, D, D, _f64p, _f64p]
    L.or_element_matrix.restype = None; L.or_element_matrix.argtypes = [D, _f64p, _f64p]
    L.or_element_load.restype = None; L.or_element_load.argtypes = [D, _f64p]
    L.or_assemble.restype = I
    L.or_assemble.argtypes = [I, I, D, D, D, _f64p, _i32p, _i32p, _f64p, _f64p]
    L.or_spmv.restype = None; L.or_spmv.argtypes = [I64, _i32p, _i32p, _f64p, _f64p, _f64p]
    L.or_dot.restype = D; L.or_dot.argtypes = [I64, _f64p, _f64p]
    L.or_cg.restype = I
    L.or_cg.argtypes = [I64, _i32p, _i32p, _f64p, _f64p, _f64p, D, I, _i32p, _f64p]
    L.or_solve_samples.restype = I
    L.or_solve_samples.argtypes = [I, I, D, D, D, I, _f64p, D, I, I, _f64p, _i32p, _f64p, _i32p]
    L.or_max_threads.restype = I; L.or_max_threads.argtypes = []


def _p(a, t):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# ------------------------------------------------------------------ mesh
def num_rows(N):
    return int(lib().or_num_rows(N))


def node_index(N):
    out = np.empty(N ** 3 * 8, np.int32)
    lib().or_node_index(N, _p(out, _i32p))
    return out.reshape(N ** 3, 8)


def graph(N):
    """CRS graph (row_map int32[n+1], col_entry int32[nnz]) of the Q1 hex mesh."""
    n = num_rows(N)
    row_map = np.empty(n + 1, np.int32)
    lib().or_graph(N, _p(row_map, _i32p), None)
    col = np.empty(int(row_map[-1]), np.int32)
    lib().or_graph(N, _p(row_map, _i32p), _p(col, _i32p))
    return row_map, col


def elem_graph(N, row_map, col_entry):
    row_map, col_entry = _i32(row_map), _i32(col_entry)
    out = np.empty(N ** 3 * 64, np.int32)
    rc = lib().or_elem_graph(N, _p(row_map, _i32p), _p(col_entry, _i32p), _p(out, _i32p))
    if rc:
        raise RuntimeError(f"or_elem_graph failed ({rc})")
    return out


def bmask(N):
    out = np.empty(num_rows(N), np.uint8)
    lib().or_bmask(N, _p(out, _u8p))
    return out


# -------------------------------------------------------------------- KL
def kl_1d(P, L=1.0):
    om, la = np.empty(P), np.empty(P)
    lib().or_kl_1d(P, L, _p(om, _f64p), _p(la, _f64p))
    return om, la


def kl_phi1d(p, omega, x, L=1.0):
    f = lib().or_kl_phi1d
    return np.array([f(int(p), L, float(omega), float(t)) for t in np.atleast_1d(x)])


def kl_modes(M, L=1.0):
    pqr = np.empty(3 * max(M, 1), np.int32)
    lam = np.empty(max(M, 1))
    lib().or_kl_modes(M, L, _p(pqr, _i32p), _p(lam, _f64p))
    return pqr[: 3 * M].reshape(M, 3), lam[:M]


def kl_coeff_at(M, xi, x, L=1.0, sigma=0.1, kappa0=1.0):
    pqr, lam = kl_modes(M, L)
    om, _ = kl_1d(max(M, 1), L)
    pqr, lam, xi = _i32(pqr), _f64(lam), _f64(xi)
    x = _f64(x)
    return lib().or_kl_coeff_at(M, L, sigma, kappa0, _p(pqr, _i32p), _p(lam, _f64p),
                                _p(om, _f64p), _p(xi, _f64p), _p(x, _f64p))


def kl_coeff_qp(N, M, xi, L=1.0, sigma=0.1, kappa0=1.0):
    xi = _f64(xi) if M > 0 else np.zeros(1)
    out = np.empty(N ** 3 * 8)
    lib().or_kl_coeff_qp(N, M, L, sigma, kappa0, _p(xi, _f64p), _p(out, _f64p))
    return out.reshape(N ** 3, 8)


def coeff_min(N, M, xi, L=1.0, sigma=0.1, kappa0=1.0):
    """Smallest coefficient a(x_q) over every Gauss point of the N^3 mesh."""
    return float(np.min(kl_coeff_qp(N, M, xi, L=L, sigma=sigma, kappa0=kappa0)))


# -------------------------------------------------------------- assembly
def element_matrix(h, a_q):
    a_q = _f64(a_q)
    K = np.empty(64)
    lib().or_element_matrix(h, _p(a_q, _f64p), _p(K, _f64p))
    return K.reshape(8, 8)


def element_load(h):
    f = np.empty(8)
    lib().or_element_load(h, _p(f, _f64p))
    return f


NONPOS_COEFF = 7   # or_assemble's status for a coefficient <= 0 (the library's ENS_ERR_NONPOS_COEFF)


class NonPositiveCoefficient(ValueError):
    """The sample's coefficient a(x_q) is not positive at some Gauss point."""


def assemble(N, M, xi, row_map, col_entry, L=1.0, sigma=0.1, kappa0=1.0, check=True):
    """values float64[nnz], b float64[n] of one sample (Algorithm 2).
    check: raise NonPositiveCoefficient when a(x_q) <= 0 at a Gauss point."""
    row_map, col_entry = _i32(row_map), _i32(col_entry)
    xi = _f64(xi) if M > 0 else np.zeros(1)
    vals = np.empty(len(col_entry))
    b = np.empty(len(row_map) - 1)
    rc = lib().or_assemble(N, M, L, sigma, kappa0, _p(xi, _f64p), _p(row_map, _i32p),
                           _p(col_entry, _i32p), _p(vals, _f64p), _p(b, _f64p))
    if rc == NONPOS_COEFF:
        if check:
            raise NonPositiveCoefficient(f"coefficient not positive at some Gauss point (N={N}, M={M})")
    elif rc:
        raise RuntimeError(f"or_assemble failed ({rc})")
    return vals, b


# ------------------------------------------------------- linear algebra
def spmv(row_map, col_entry, values, x):
    row_map, col_entry, values, x = _i32(row_map), _i32(col_entry), _f64(values), _f64(x)
    z = np.empty(len(row_map) - 1)
    lib().or_spmv(len(z), _p(row_map, _i32p), _p(col_entry, _i32p), _p(values, _f64p),
                  _p(x, _f64p), _p(z, _f64p))
    return z


def dot(u, v):
    u, v = _f64(u), _f64(v)
    return lib().or_dot(len(u), _p(u, _f64p), _p(v, _f64p))


def cg(row_map, col_entry, values, b, x0=None, tol=1e-10, max_iter=10000):
    """Returns (x, iters, relres_true, status)."""
    row_map, col_entry, values, b = _i32(row_map), _i32(col_entry), _f64(values), _f64(b)
    x = np.zeros(len(b)) if x0 is None else _f64(x0).copy()
    it = np.zeros(1, np.int32)
    rr = np.zeros(1)
    st = lib().or_cg(len(b), _p(row_map, _i32p), _p(col_entry, _i32p), _p(values, _f64p),
                     _p(b, _f64p), _p(x, _f64p), tol, max_iter, _p(it, _i32p), _p(rr, _f64p))
    return x, int(it[0]), float(rr[0]), int(st)


def max_threads():
    return int(lib().or_max_threads())


def solve_samples(N, M, xi, tol, max_iter=10000, nthreads=1, want_x=False, L=1.0, sigma=0.1,
                  kappa0=1.0):
    """Assemble + CG for each row of xi (shape (num_samples, M)), per sample.

    Returns (x or None, iters, relres, status) with x shape (num_samples, n).
    """
    xi = _f64(np.asarray(xi).reshape(-1, max(M, 1)))
    ns = xi.shape[0]
    n = num_rows(N)
    x = np.empty((ns, n)) if want_x else None
    it = np.zeros(ns, np.int32)
    rr = np.zeros(ns)
    st = np.zeros(ns, np.int32)
    rc = lib().or_solve_samples(N, M, L, sigma, kappa0, ns, _p(xi, _f64p), tol, max_iter,
                                nthreads, _p(x, _f64p) if want_x else None, _p(it, _i32p),
                                _p(rr, _f64p), _p(st, _i32p))
    if rc:
        raise RuntimeError(f"or_solve_samples failed ({rc})")
    return x, it, rr, st


# ------------------------------------------ ensemble re-ordering helpers
def to_ensemble(per_sample):
    """list of s per-sample arrays of length m -> commuted layout [m*s] (Eq. 3)."""
    return np.ascontiguousarray(np.stack([_f64(a) for a in per_sample], axis=1)).reshape(-1)


def from_ensemble(flat, s):
    """commuted layout [m*s] -> array (s, m) of per-sample vectors."""
    return np.ascontiguousarray(np.asarray(flat).reshape(-1, s).T)
