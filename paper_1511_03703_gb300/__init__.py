"""Embedded ensemble propagation on one GB300: Python binding of libens.so.

A thin ctypes layer over the C ABI declared in include/ens.h.  Every function
here only marshals arguments (torch tensors -> device pointers, the current
CUDA stream) and turns status codes into EnsError; every step of the
computation runs in the library's CUDA kernels.  PyTorch is used for device
memory and streams only.  There is no CPU fallback: if libens.so cannot be
built or loaded, or no GPU is present, calls raise.
"""
import ctypes
import os
import threading

__all__ = ["EnsError", "lib", "Graph", "Mesh", "mesh_sizes", "graph_build", "kl_table_size",
           "kl_setup", "mode_matrices", "assemble", "spmv", "dot", "dot_workspace_size", "dot_static", "cg",
           "cg_workspace_size", "CgStats", "Batch", "convert_values", "cg_mixed", "cg_mixed_workspace_size", "F64", "F32", "BF16", "CG_COUPLED", "CG_GRAPH",
           "CG_TIME_SPMV", "CG_DF64", "CG_SPLIT64", "CG_GUESS_FALLBACK", "CG_X0_ZERO", "F64_DF", "F64_SPLIT",
           "snapshots_put", "pod", "pod_workspace_size", "pod_targets", "to_f32", "mlp_param_count",
           "mlp_init", "mlp_workspace_size", "mlp_forward", "mlp_grad", "mlp_adam", "mlp_train",
           "guess", "guess_workspace_size", "MLP_DIMS", "pcg", "pcg_workspace_size", "PC_JACOBI",
           "PC_CHEBYSHEV", "PC_LANCZOS", "Multigrid", "mg_level_sizes"]

F64, F32, BF16, F64_DF, F64_SPLIT = 0, 1, 2, 3, 4
CG_COUPLED, CG_GRAPH, CG_TIME_SPMV, CG_DF64, CG_SPLIT64, CG_GUESS_FALLBACK, CG_X0_ZERO = 1, 2, 4, 8, 16, 32, 64
CG_K1_CHUNKS_SHIFT = 16
CG_BATCH_K1_WIDE = 1 << 19
CG_K1_DEFER = 1 << 20


def cg_k1_chunks(chunks):
    """ens_cg flags for the CG SpMV's mapping: `chunks` (1, 2, 4 or 8) chunks of
    32 rows per CTA (ENS_CG_K1_CHUNKS), or "defer" for one chunk per CTA with
    the upper levels of p.q's tree in a second kernel (ENS_CG_K1_DEFER); 0 or
    None leaves the library's default."""
    if not chunks:
        return 0
    if chunks == "defer":
        return CG_K1_DEFER
    k = {1: 0, 2: 1, 4: 2, 8: 3}[chunks]
    return (k + 1) << CG_K1_CHUNKS_SHIFT
MLP_DIMS = (10, 256, 256, 64)
OK, ERR_NOT_CONVERGED, ERR_BREAKDOWN = 0, 5, 6
ERR_ARG, ERR_WORKSPACE = 1, 9

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None
_lock = threading.Lock()


class EnsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[ens status {code}] {msg}")
        self.code = code


class EnsGraphC(ctypes.Structure):
    _fields_ = [("num_rows", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("num_entries", ctypes.c_int64), ("row_map", ctypes.c_void_p),
                ("col_entry", ctypes.c_void_p)]


class BatchItemC(ctypes.Structure):
    _fields_ = [("graph", EnsGraphC), ("s", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("values", ctypes.c_void_p), ("b", ctypes.c_void_p), ("x", ctypes.c_void_p),
                ("iters_host", ctypes.c_void_p), ("relres_host", ctypes.c_void_p),
                ("status_host", ctypes.c_void_p), ("values_df", ctypes.c_void_p)]


class MgLevelC(ctypes.Structure):
    _fields_ = [("graph", EnsGraphC), ("N", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("values", ctypes.c_void_p), ("power_start", ctypes.c_void_p), ("values_df", ctypes.c_void_p),
                ("values_f32", ctypes.c_void_p)]


class NewtonParamsC(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("tol", ctypes.c_double),
                ("lin_tol", ctypes.c_double), ("max_newton", ctypes.c_int32), ("restart", ctypes.c_int32),
                ("max_lin", ctypes.c_int32), ("precond", ctypes.c_int32), ("degree", ctypes.c_int32),
                ("power_iters", ctypes.c_int32), ("check_every", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("ratio", ctypes.c_double), ("boost", ctypes.c_double)]


class CgStats(ctypes.Structure):
    _fields_ = [("spmv_ms", ctypes.c_double), ("spmv_launches", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("host_checks", ctypes.c_int32), ("guess_fallbacks", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def library_path():
    return os.path.join(_HERE, "_build", "libens.so")


def lib(build_if_missing=True):
    """Load libens.so (building it with nvcc if it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                if not build_if_missing:
                    raise EnsError(-1, f"{path} missing: run paper_1511_03703_gb300.build.build()")
                from . import build as _b
                _b.build()
            _lib = ctypes.CDLL(path)
            _declare(_lib)
    return _lib


def _declare(L):
    vp, i32, i64, d, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
    I = ctypes.c_int
    P = ctypes.POINTER
    sig = {
        "ens_last_error": (ctypes.c_char_p, []),
        "ens_status_string": (ctypes.c_char_p, [I]),
        "ens_version": (I, []),
        "ens_mesh_sizes": (I, [I, P(i32), P(i64), P(i64)]),
        "ens_graph_build": (I, [I, vp, vp, vp, vp, vp]),
        "ens_kl_table_size": (I, [I, I, P(i64)]),
        "ens_kl_setup": (I, [I, I, d, vp, vp, vp, vp]),
        "ens_mode_matrices": (I, [I, P(EnsGraphC), I, vp, vp, vp, vp]),
        "ens_assemble": (I, [P(EnsGraphC), vp, I, I, vp, vp, vp, vp, d, d, vp, vp, vp]),
        "ens_assemble_df": (I, [P(EnsGraphC), vp, I, I, vp, vp, vp, vp, d, d, vp, vp, vp, vp]),
        "ens_spmv": (I, [P(EnsGraphC), I, I, vp, vp, vp, vp]),
        "ens_spmv_df": (I, [P(EnsGraphC), I, vp, vp, vp, vp, vp]),
        "ens_dot_workspace_size": (I, [i64, I, P(sz)]),
        "ens_dot": (I, [i64, I, vp, vp, vp, vp, sz, vp]),
        "ens_dot_static": (I, [i64, I, vp, vp, vp, vp]),
        "ens_cg_workspace_size": (I, [i32, I, P(sz)]),
        "ens_cg": (I, [P(EnsGraphC), I, vp, vp, vp, d, I, I, I, vp, sz, vp, vp, vp, P(CgStats), vp]),
        "ens_cg_df": (I, [P(EnsGraphC), I, vp, vp, vp, vp, d, I, I, I, vp, sz, vp, vp, vp, P(CgStats), vp]),
        "ens_pcg_workspace_size": (I, [i32, I, P(sz)]),
        "ens_mg_workspace_size": (I, [I, P(MgLevelC), I, P(sz)]),
        "ens_mg_pcg": (I, [I, P(MgLevelC), I, vp, vp, d, I, I, d, d, I, I, I, vp, sz, vp, vp, vp, P(CgStats), vp]),
        "ens_pcg": (I, [P(EnsGraphC), I, vp, vp, vp, d, I, I, I, d, d, I, vp, I, I, vp, sz, vp, vp, vp, vp,
                        P(CgStats), vp]),
        "ens_convert_values": (I, [P(EnsGraphC), I, vp, I, vp, vp, vp]),
        "ens_cg_batched_workspace_size": (I, [I, P(BatchItemC), P(sz)]),
        "ens_cg_batched": (I, [I, P(BatchItemC), d, I, I, I, vp, sz, P(CgStats), vp]),
        "ens_cg_mixed_workspace_size": (I, [i32, I, P(sz)]),
        "ens_cg_mixed": (I, [P(EnsGraphC), I, vp, vp, I, vp, vp, vp, d, I, d, I, I, I, vp, sz, vp, vp,
                             vp, vp, P(CgStats), vp]),
        "ens_snapshots_put": (I, [i64, i32, vp, vp, i64, i64, vp]),
        "ens_pod_workspace_size": (I, [i64, i32, i32, P(sz)]),
        "ens_pod": (I, [i64, i32, vp, i64, i32, i32, vp, i32, vp, vp, vp, vp, sz, vp]),
        "ens_pod_targets_workspace_size": (I, [i64, i32, i32, P(sz)]),
        "ens_pod_targets": (I, [i64, i32, vp, i64, i32, vp, vp, vp, vp, vp, sz, vp]),
        "ens_to_f32": (I, [i64, vp, vp, vp]),
        "ens_mlp_param_count": (I, [P(i32), P(i64)]),
        "ens_mlp_init": (I, [P(i32), vp, vp, vp]),
        "ens_mlp_workspace_size": (I, [P(i32), i32, P(sz)]),
        "ens_mlp_forward": (I, [P(i32), vp, i32, vp, vp, vp, sz, vp]),
        "ens_mlp_grad": (I, [P(i32), vp, i32, vp, vp, vp, vp, vp, sz, vp]),
        "ens_mlp_adam": (I, [i64, vp, vp, vp, vp, vp, i64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                             ctypes.c_float, vp]),
        "ens_mlp_train": (I, [P(i32), vp, vp, vp, vp, i64, vp, vp, i32, i32, i64, ctypes.c_float,
                              ctypes.c_float, ctypes.c_float, ctypes.c_float, vp, i32, vp, sz, vp]),
        "ens_nl_advection": (I, [P(EnsGraphC), i32, vp, vp, vp]),
        "ens_nl_jacobian_workspace_size": (I, [P(sz)]),
        "ens_nl_jacobian": (I, [P(EnsGraphC), i32, I, vp, vp, d, d, vp, vp, vp, vp, vp, vp]),
        "ens_gmres_workspace_size": (I, [I, P(MgLevelC), I, I, I, P(sz)]),
        "ens_gmres": (I, [I, P(MgLevelC), I, vp, vp, vp, d, I, I, I, I, d, d, I, I, vp, sz, vp, vp, vp,
                          P(CgStats), vp]),
        "ens_newton_workspace_size": (I, [I, P(MgLevelC), I, P(NewtonParamsC), P(sz)]),
        "ens_newton": (I, [I, P(MgLevelC), I, vp, vp, vp, P(NewtonParamsC), vp, sz, vp, vp, vp, vp, P(CgStats),
                           vp]),
        "ens_guess_workspace_size": (I, [P(i32), i32, P(sz)]),
        "ens_guess": (I, [P(i32), vp, i64, i32, vp, vp, vp, vp, vp, vp, vp, sz, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def exported_symbols():
    """Names declared in include/ens.h (used by the load/export test)."""
    import re
    hdr = os.path.join(os.path.dirname(_HERE), "include", "ens.h")
    txt = open(hdr).read()
    return sorted(set(re.findall(r"^(?:int|const char \*)\s*\*?\s*(ens_\w+)\s*\(", txt, re.M)))


def _check(rc):
    if rc != 0:
        msg = lib().ens_last_error()
        raise EnsError(rc, msg.decode() if msg else "")
    return rc


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _require_cuda(*tensors):
    for t in tensors:
        if t is not None and not t.is_cuda:
            raise EnsError(1, "tensor arguments must live on the GPU (no CPU path)")


# ------------------------------------------------------------- mesh / graph
def mesh_sizes(N):
    n, nnz, nc = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().ens_mesh_sizes(N, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(nc)))
    return n.value, nnz.value, nc.value


class Graph:
    """CRS graph of the ensemble matrix (Fig. 2); keeps its tensors alive."""

    def __init__(self, row_map, col_entry):
        _require_cuda(row_map, col_entry)
        self.row_map, self.col_entry = row_map, col_entry
        self.num_rows = row_map.numel() - 1
        self.num_entries = col_entry.numel()
        self.c = EnsGraphC(self.num_rows, 0, self.num_entries, row_map.data_ptr(),
                           col_entry.data_ptr())

    def ref(self):
        return ctypes.byref(self.c)


def graph_build(N, row_map, col_entry, elem_graph=None, bmask=None, stream=None):
    _require_cuda(row_map, col_entry, elem_graph, bmask)
    _check(lib().ens_graph_build(N, _ptr(row_map), _ptr(col_entry), _ptr(elem_graph), _ptr(bmask),
                                 _stream(stream)))


# ---------------------------------------------------------------------- KL
def kl_table_size(N, M):
    v = ctypes.c_int64()
    _check(lib().ens_kl_table_size(N, M, ctypes.byref(v)))
    return v.value


def kl_setup(N, M, L, kl_table, want_host=True, stream=None):
    """Returns (lambda[M], pqr[M][3]) as Python lists when want_host."""
    _require_cuda(kl_table)
    if want_host:
        lam = (ctypes.c_double * M)()
        pqr = (ctypes.c_int32 * (3 * M))()
        _check(lib().ens_kl_setup(N, M, L, _ptr(kl_table), lam, pqr, _stream(stream)))
        return list(lam), [list(pqr[3 * k:3 * k + 3]) for k in range(M)]
    _check(lib().ens_kl_setup(N, M, L, _ptr(kl_table), None, None, _stream(stream)))
    return None, None


def mode_matrices(N, graph, M, kl_table, modes, load, stream=None):
    _require_cuda(kl_table, modes, load)
    _check(lib().ens_mode_matrices(N, graph.ref(), M, _ptr(kl_table), _ptr(modes), _ptr(load),
                                   _stream(stream)))


def assemble(graph, bmask, s, M, modes, load, xi, sigma, kappa0, values, b, stream=None, df=False,
             values_df=None, kl_table=None):
    """ens_assemble; df=True (or a values_df tensor, 2*nnz*s float32) runs
    ens_assemble_df, which also writes the pre-split copy into values_df.
    kl_table (the mesh's ens_kl_setup table) turns on the coefficient
    positivity check: EnsError(7) when a member's a(x_q) <= 0 somewhere (the
    values are still written)."""
    _require_cuda(bmask, modes, load, xi, values, b, values_df, kl_table)
    if df or values_df is not None:
        _check(lib().ens_assemble_df(graph.ref(), _ptr(bmask), s, M, _ptr(kl_table), _ptr(modes), _ptr(load),
                                     _ptr(xi), sigma, kappa0, _ptr(values), _ptr(values_df), _ptr(b),
                                     _stream(stream)))
    else:
        _check(lib().ens_assemble(graph.ref(), _ptr(bmask), s, M, _ptr(kl_table), _ptr(modes), _ptr(load),
                                  _ptr(xi), sigma, kappa0, _ptr(values), _ptr(b), _stream(stream)))


# ------------------------------------------------------------ linear algebra
_DT = {"float64": F64, "float32": F32, "bfloat16": BF16}


def spmv(graph, s, values, x, y, stream=None, df=False, split=False, values_df=None):
    """y = A_c x.  float64 values: df=True -> double-float arithmetic (ENS_F64_DF),
    split=True -> alternate entries FP64 / double-float (ENS_F64_SPLIT),
    values_df (the ENS_F64_DF split copy of values) -> ens_spmv_df."""
    _require_cuda(values, x, y, values_df)
    if values_df is not None:
        _check(lib().ens_spmv_df(graph.ref(), s, _ptr(values), _ptr(values_df), _ptr(x), _ptr(y),
                                 _stream(stream)))
        return
    dt = _DT[str(values.dtype).replace("torch.", "")]
    if df or split:
        if dt != F64:
            raise EnsError(2, "df / split arithmetic needs float64 values")
        dt = F64_SPLIT if split else F64_DF
    _check(lib().ens_spmv(graph.ref(), s, dt, _ptr(values), _ptr(x), _ptr(y), _stream(stream)))


def dot_workspace_size(n, s):
    v = ctypes.c_size_t()
    _check(lib().ens_dot_workspace_size(n, s, ctypes.byref(v)))
    return v.value


def dot(n, s, u, v, out, work, stream=None):
    _require_cuda(u, v, out, work)
    _check(lib().ens_dot(n, s, _ptr(u), _ptr(v), _ptr(out), _ptr(work), work.numel() * work.element_size(),
                         _stream(stream)))


def dot_static(n, s, u, v, out, stream=None):
    """ens_dot without a workspace: scratch comes from the library's static array."""
    _require_cuda(u, v, out)
    _check(lib().ens_dot_static(n, s, _ptr(u), _ptr(v), _ptr(out), _stream(stream)))


def cg_workspace_size(n, s):
    v = ctypes.c_size_t()
    _check(lib().ens_cg_workspace_size(n, s, ctypes.byref(v)))
    return v.value


def cg(graph, s, values, b, x, tol, max_iter, work, flags=0, check_every=8, stream=None,
       raise_on_failure=False, values_df=None):
    """Runs ens_cg (or ens_cg_df when values_df, the ENS_F64_DF split copy of
    values, is given); returns (iters[s], relres[s], status[s], CgStats).
    Synchronises."""
    _require_cuda(values, b, x, work, values_df)
    it = (ctypes.c_int32 * s)()
    rr = (ctypes.c_double * s)()
    stt = (ctypes.c_int32 * s)()
    stats = CgStats()
    if values_df is None:
        rc = lib().ens_cg(graph.ref(), s, _ptr(values), _ptr(b), _ptr(x), tol, max_iter, flags,
                          check_every, _ptr(work), work.numel() * work.element_size(), it, rr, stt,
                          ctypes.byref(stats), _stream(stream))
    else:
        rc = lib().ens_cg_df(graph.ref(), s, _ptr(values), _ptr(values_df), _ptr(b), _ptr(x), tol, max_iter,
                             flags, check_every, _ptr(work), work.numel() * work.element_size(), it, rr, stt,
                             ctypes.byref(stats), _stream(stream))
    if rc not in (0, ERR_NOT_CONVERGED, ERR_BREAKDOWN) or (rc and raise_on_failure):
        _check(rc)
    return list(it), list(rr), list(stt), stats


# ------------------------------------------------------ preconditioned CG
PC_JACOBI, PC_CHEBYSHEV = 1, 2
PC_LANCZOS = 1 << 24   # flags of pcg and Multigrid.solve: the eigenvalue bound by Lanczos steps


def pcg_workspace_size(n, s):
    v = ctypes.c_size_t()
    _check(lib().ens_pcg_workspace_size(n, s, ctypes.byref(v)))
    return v.value


def pcg(graph, s, values, b, x, tol, max_iter, work, precond=PC_JACOBI, degree=2, ratio=30.0, boost=1.1,
        power_iters=10, power_start=None, flags=0, check_every=8, stream=None):
    """Runs ens_pcg; returns (iters[s], relres[s], status[s], lam[s], CgStats).  Synchronises."""
    _require_cuda(values, b, x, work, power_start)
    it = (ctypes.c_int32 * s)()
    rr = (ctypes.c_double * s)()
    stt = (ctypes.c_int32 * s)()
    lam = (ctypes.c_double * s)()
    stats = CgStats()
    rc = lib().ens_pcg(graph.ref(), s, _ptr(values), _ptr(b), _ptr(x), tol, max_iter, precond, degree, ratio,
                       boost, power_iters, _ptr(power_start), flags, check_every, _ptr(work),
                       work.numel() * work.element_size(), it, rr, stt, lam, ctypes.byref(stats), _stream(stream))
    if rc not in (0, ERR_NOT_CONVERGED, ERR_BREAKDOWN):
        _check(rc)
    return list(it), list(rr), list(stt), list(lam), stats


# ------------------------------------------------ multigrid-preconditioned CG
def _per_level(values_df, nlevels):
    """values_df as a per-level list: None, one tensor (level 0) or a list."""
    if values_df is None:
        return [None] * nlevels
    if isinstance(values_df, (list, tuple)):
        return list(values_df) + [None] * (nlevels - len(values_df))
    return [values_df] + [None] * (nlevels - 1)


def mg_level_sizes(N):
    """N, N/2, ... while the size is even and above 4 (the coarsest has <= 125 rows)."""
    out = [N]
    while out[-1] % 2 == 0 and out[-1] > 4:
        out.append(out[-1] // 2)
    return out


class Multigrid:
    """The nested meshes of a V-cycle (set-up per mesh, on the GPU), and the
    per-ensemble assembly and MG-PCG solve (ens_mg_pcg)."""

    def __init__(self, N, M, L=1.0, device="cuda"):
        self.sizes = mg_level_sizes(N)
        if len(self.sizes) < 2 or self.sizes[-1] > 4:
            raise EnsError(1, f"N={N}: no nested hierarchy down to N <= 4 by halving")
        self.meshes = [Mesh(n, M, L=L, device=device) for n in self.sizes]
        self.N, self.M = N, M

    def assemble(self, s, xi_ens, sigma=0.1, kappa0=1.0, df=False, values_df=None):
        """Values of every level and the level-0 right-hand side (df: the
        double-float assembly, see assemble(); values_df: a 2*nnz*s float32
        tensor that receives level 0's pre-split values, or a list of such
        tensors (or None) per level, for solve())."""
        vdfs = _per_level(values_df, len(self.meshes))
        vals, b0 = [], None
        for l, mesh in enumerate(self.meshes):
            v, b = mesh.assemble(s, xi_ens, sigma=sigma, kappa0=kappa0, df=df, values_df=vdfs[l])
            vals.append(v)
            if l == 0:
                b0 = b
        return vals, b0

    def _levels(self, s, values, power_starts, values_df=None, values_f32=None):
        c = (MgLevelC * len(self.meshes))()
        for l, mesh in enumerate(self.meshes):
            _require_cuda(values[l], power_starts[l])
            c[l].graph = mesh.graph.c
            c[l].N = mesh.N
            c[l].values = values[l].data_ptr()
            c[l].power_start = power_starts[l].data_ptr()
        for l, v in enumerate(_per_level(values_df, len(self.meshes))):
            if v is not None:
                _require_cuda(v)
                c[l].values_df = v.data_ptr()
        if values_f32 is not None:
            for l, v in enumerate(values_f32):
                _require_cuda(v)
                c[l].values_f32 = v.data_ptr()
        return c

    def to_f32(self, s, values, out=None, stream=None):
        """FP32 copies of every level's values (for the FP32 V-cycle of solve())."""
        import torch
        out = out or [torch.empty(v.numel(), dtype=torch.float32, device=v.device) for v in values]
        for l, mesh in enumerate(self.meshes):
            convert_values(mesh.graph, s, values[l], out[l], stream=stream)
        return out

    def workspace_size(self, s, values, power_starts, values_df=None, values_f32=None):
        v = ctypes.c_size_t()
        c = self._levels(s, values, power_starts, values_df, values_f32)
        _check(lib().ens_mg_workspace_size(len(self.meshes), c, s, ctypes.byref(v)))
        return v.value

    def solve(self, s, values, b, x, tol, max_iter, work, power_starts, degree=2, ratio=5.0, boost=1.1,
              power_iters=10, flags=0, check_every=8, stream=None, values_df=None, values_f32=None):
        """Returns (iters[s], relres[s], status[s], CgStats).  values_df: pre-split
        values (level 0's, or a list per level: those SpMVs in double-float);
        values_f32: FP32 values of every level (to_f32): the V-cycle in FP32.
        Synchronises."""
        _require_cuda(b, x, work)
        c = self._levels(s, values, power_starts, values_df, values_f32)
        it = (ctypes.c_int32 * s)()
        rr = (ctypes.c_double * s)()
        stt = (ctypes.c_int32 * s)()
        stats = CgStats()
        rc = lib().ens_mg_pcg(len(self.meshes), c, s, _ptr(b), _ptr(x), tol, max_iter, degree, ratio, boost,
                              power_iters, flags, check_every, _ptr(work), work.numel() * work.element_size(),
                              it, rr, stt, ctypes.byref(stats), _stream(stream))
        if rc not in (0, ERR_NOT_CONVERGED, ERR_BREAKDOWN):
            _check(rc)
        return list(it), list(rr), list(stt), stats


# ------------------------------------------ nonlinear advection-diffusion
NL_PRECOND_NONE, NL_PRECOND_MG = 0, 1


def nl_advection(mesh, v=(1.0, 1.0, 1.0), out=None, stream=None):
    """C (nnz float64) of the advection term int phi_i v.grad(phi_j), constant v."""
    import torch
    C = out if out is not None else torch.empty(mesh.nnz, dtype=torch.float64, device=mesh.row_map.device)
    _require_cuda(C)
    vh = (ctypes.c_double * 3)(*[float(t) for t in v])
    _check(lib().ens_nl_advection(mesh.graph.ref(), mesh.N, vh, _ptr(C), _stream(stream)))
    return C


def nl_jacobian(mesh, s, A, C, alpha, beta, b, u, J=None, F=None, stream=None):
    """(J, F) = (J(u), F(u)) of the nonlinear problem (ens_nl_jacobian).  Synchronises."""
    import torch
    _require_cuda(A, C, b, u, J, F)
    dev = A.device
    J = J if J is not None else torch.empty(mesh.nnz * s, dtype=torch.float64, device=dev)
    F = F if F is not None else torch.empty(mesh.n * s, dtype=torch.float64, device=dev)
    nb = ctypes.c_size_t()
    _check(lib().ens_nl_jacobian_workspace_size(ctypes.byref(nb)))
    work = torch.empty(nb.value, dtype=torch.uint8, device=dev)
    _check(lib().ens_nl_jacobian(mesh.graph.ref(), mesh.N, s, _ptr(A), _ptr(C), alpha, beta, _ptr(b), _ptr(u),
                                 _ptr(J), _ptr(F), _ptr(work), _stream(stream)))
    return J, F


class Nonlinear:
    """Newton-GMRES for the nonlinear advection-diffusion problem on the
    N^3 mesh (ens_newton): the advection matrix of the velocity v, and the
    hierarchy of the multigrid preconditioner (or the single mesh)."""

    def __init__(self, N, M, v=(1.0, 1.0, 1.0), precond=NL_PRECOND_MG, L=1.0, device="cuda"):
        self.precond = precond
        if precond == NL_PRECOND_MG:
            self.mg = Multigrid(N, M, L=L, device=device)
            self.meshes = self.mg.meshes
        else:
            self.mg = None
            self.meshes = [Mesh(N, M, L=L, device=device)]
        self.mesh = self.meshes[0]
        self.N, self.M = N, M
        self.v = tuple(float(t) for t in v)
        self.C = nl_advection(self.mesh, self.v)

    def assemble(self, s, xi_ens, sigma=0.1, kappa0=1.0, df=False, values_df=None):
        """Diffusion values of every level and the load (see Multigrid.assemble)."""
        if self.mg is not None:
            return self.mg.assemble(s, xi_ens, sigma=sigma, kappa0=kappa0, df=df, values_df=values_df)
        v, b = self.mesh.assemble(s, xi_ens, sigma=sigma, kappa0=kappa0, df=df,
                                  values_df=_per_level(values_df, 1)[0])
        return [v], b

    def _levels(self, values, power_starts, values_df=None, values_f32=None):
        c = (MgLevelC * len(self.meshes))()
        for l, mesh in enumerate(self.meshes):
            _require_cuda(values[l])
            c[l].graph = mesh.graph.c
            c[l].N = mesh.N
            c[l].values = values[l].data_ptr()
            c[l].power_start = power_starts[l].data_ptr() if power_starts is not None else None
        for l, v in enumerate(_per_level(values_df, len(self.meshes))):
            if v is not None:
                _require_cuda(v)
                c[l].values_df = v.data_ptr()
        if values_f32 is not None:
            for l, v in enumerate(values_f32):
                _require_cuda(v)
                c[l].values_f32 = v.data_ptr()
        return c

    def params(self, alpha, beta, tol=1e-8, lin_tol=1e-10, max_newton=20, restart=30, max_lin=500, degree=2,
               ratio=5.0, boost=1.1, power_iters=10, check_every=4, flags=0):
        """flags: 0 or PC_LANCZOS (the V-cycle's eigenvalue bounds by power_iters Lanczos steps)."""
        p = NewtonParamsC()
        p.alpha, p.beta, p.tol, p.lin_tol = alpha, beta, tol, lin_tol
        p.max_newton, p.restart, p.max_lin, p.precond = max_newton, restart, max_lin, self.precond
        p.degree, p.power_iters, p.check_every, p.flags = degree, power_iters, check_every, flags
        p.ratio, p.boost = ratio, boost
        return p

    def workspace_size(self, s, values, power_starts, params, values_df=None, values_f32=None):
        v = ctypes.c_size_t()
        _check(lib().ens_newton_workspace_size(len(self.meshes),
                                               self._levels(values, power_starts, values_df, values_f32), s,
                                               ctypes.byref(params), ctypes.byref(v)))
        return v.value

    def solve(self, s, values, b, u, work, power_starts, params, stream=None, values_df=None, values_f32=None):
        """Newton from the given u (values_df: level 0's pre-split values for
        the preconditioner).  Returns (newton_iters[s], lin_iters[s],
        relres[s], status[s], CgStats).  Synchronises."""
        _require_cuda(b, u, work)
        ni = (ctypes.c_int32 * s)()
        li = (ctypes.c_int32 * s)()
        rr = (ctypes.c_double * s)()
        stt = (ctypes.c_int32 * s)()
        stats = CgStats()
        rc = lib().ens_newton(len(self.meshes), self._levels(values, power_starts, values_df, values_f32), s,
                              _ptr(self.C), _ptr(b), _ptr(u), ctypes.byref(params), _ptr(work),
                              work.numel() * work.element_size(), ni, li, rr, stt, ctypes.byref(stats),
                              _stream(stream))
        if rc not in (0, ERR_NOT_CONVERGED, ERR_BREAKDOWN):
            _check(rc)
        return list(ni), list(li), list(rr), list(stt), stats

    def gmres_workspace_size(self, s, values, power_starts, restart):
        v = ctypes.c_size_t()
        _check(lib().ens_gmres_workspace_size(len(self.meshes), self._levels(values, power_starts), s, restart,
                                              self.precond, ctypes.byref(v)))
        return v.value

    def gmres(self, s, values, J, b, x, work, power_starts, tol, restart=30, max_iter=500, degree=2, ratio=5.0,
              boost=1.1, power_iters=10, check_every=4, stream=None):
        """ens_gmres for J x = b (values: the preconditioner's levels).
        Returns (iters[s], relres[s], status[s], CgStats).  Synchronises."""
        _require_cuda(J, b, x, work)
        it = (ctypes.c_int32 * s)()
        rr = (ctypes.c_double * s)()
        stt = (ctypes.c_int32 * s)()
        stats = CgStats()
        rc = lib().ens_gmres(len(self.meshes), self._levels(values, power_starts), s, _ptr(J), _ptr(b), _ptr(x),
                             tol, restart, max_iter, self.precond, degree, ratio, boost, power_iters, check_every,
                             _ptr(work), work.numel() * work.element_size(), it, rr, stt, ctypes.byref(stats),
                             _stream(stream))
        if rc not in (0, ERR_NOT_CONVERGED, ERR_BREAKDOWN):
            _check(rc)
        return list(it), list(rr), list(stt), stats


# ------------------------------------------------------------- batched CG
class Batch:
    """A batch of ensembles (graph, s, values, b, x[, values_df]) solved by
    ens_cg_batched; with values_df (pre-split values, on every item) the batch
    runs the pre-split double-float SpMV of ens_cg_df."""

    def __init__(self, items):
        """items: list of (graph, s, values, b, x) or (graph, s, values, b, x,
        values_df) with device tensors."""
        self.items = list(items)
        n = len(self.items)
        self.c = (BatchItemC * n)()
        self.iters = [(ctypes.c_int32 * it[1])() for it in self.items]
        self.relres = [(ctypes.c_double * it[1])() for it in self.items]
        self.status = [(ctypes.c_int32 * it[1])() for it in self.items]
        for i, item in enumerate(self.items):
            graph, s, values, b, x = item[:5]
            vdf = item[5] if len(item) > 5 else None
            _require_cuda(values, b, x, vdf)
            self.c[i].graph = graph.c
            self.c[i].s = s
            self.c[i].values, self.c[i].b, self.c[i].x = values.data_ptr(), b.data_ptr(), x.data_ptr()
            self.c[i].values_df = vdf.data_ptr() if vdf is not None else None
            self.c[i].iters_host = ctypes.cast(self.iters[i], ctypes.c_void_p)
            self.c[i].relres_host = ctypes.cast(self.relres[i], ctypes.c_void_p)
            self.c[i].status_host = ctypes.cast(self.status[i], ctypes.c_void_p)

    def workspace_size(self):
        v = ctypes.c_size_t()
        _check(lib().ens_cg_batched_workspace_size(len(self.items), self.c, ctypes.byref(v)))
        return v.value

    def solve(self, tol, max_iter, work, flags=0, check_every=8, stream=None):
        """Returns (iters, relres, status) lists per item, and CgStats."""
        _require_cuda(work)
        stats = CgStats()
        rc = lib().ens_cg_batched(len(self.items), self.c, tol, max_iter, flags, check_every,
                                  _ptr(work), work.numel() * work.element_size(), ctypes.byref(stats),
                                  _stream(stream))
        if rc not in (0, ERR_NOT_CONVERGED, ERR_BREAKDOWN):
            _check(rc)
        return ([list(a) for a in self.iters], [list(a) for a in self.relres],
                [list(a) for a in self.status], stats)


# --------------------------------------------------------- mixed precision
def convert_values(graph, s, values, values_lo, diag_lo=None, stream=None, dtype=None):
    """FP64 values -> values_lo (float32 or bfloat16 tensor); diag_lo (float32)
    optional.  dtype=F64_DF: values_lo holds 2*nnz*s float32 (the split pairs)."""
    _require_cuda(values, values_lo, diag_lo)
    dt = _DT[str(values_lo.dtype).replace("torch.", "")] if dtype is None else dtype
    _check(lib().ens_convert_values(graph.ref(), s, _ptr(values), dt, _ptr(values_lo), _ptr(diag_lo),
                                    _stream(stream)))


def cg_mixed_workspace_size(n, s):
    v = ctypes.c_size_t()
    _check(lib().ens_cg_mixed_workspace_size(n, s, ctypes.byref(v)))
    return v.value


def cg_mixed(graph, s, values, values_lo, b, x, tol, work, diag_lo=None, max_outer=20,
             inner_tol=1e-4, max_inner=2000, check_every=8, flags=0, stream=None):
    """FP64 iterative refinement around an FP32 inner CG; synchronises.

    Returns (outer_iters[s], inner_iters[s], relres[s], status[s], CgStats)."""
    _require_cuda(values, values_lo, b, x, work, diag_lo)
    dt = _DT[str(values_lo.dtype).replace("torch.", "")]
    oi = (ctypes.c_int32 * s)()
    ii = (ctypes.c_int32 * s)()
    rr = (ctypes.c_double * s)()
    stt = (ctypes.c_int32 * s)()
    stats = CgStats()
    rc = lib().ens_cg_mixed(graph.ref(), s, _ptr(values), _ptr(values_lo), dt, _ptr(diag_lo), _ptr(b),
                            _ptr(x), tol, max_outer, inner_tol, max_inner, check_every, flags, _ptr(work),
                            work.numel() * work.element_size(), oi, ii, rr, stt, ctypes.byref(stats),
                            _stream(stream))
    if rc not in (0, ERR_NOT_CONVERGED, ERR_BREAKDOWN):
        _check(rc)
    return list(oi), list(ii), list(rr), list(stt), stats


# ------------------------------------------------- learned initial guess
def _nbytes(t):
    return t.numel() * t.element_size()


def _dims(dims):
    return (ctypes.c_int32 * 4)(*dims)


def snapshots_put(x, X, col0, s, stream=None):
    """Copy ensemble solution x (n*s, commuted layout) into columns col0.. of X (n x m)."""
    _require_cuda(x, X)
    n, ldx = X.shape
    _check(lib().ens_snapshots_put(n, s, _ptr(x), _ptr(X), ldx, col0, _stream(stream)))


def pod_workspace_size(n, m, l):
    v = ctypes.c_size_t()
    _check(lib().ens_pod_workspace_size(n, m, l, ctypes.byref(v)))
    return v.value


def pod(X, k, l, Omega, mean, Phi, sigma, work, power_iters=1, m=None, stream=None):
    """POD basis of the snapshot columns of X (centred in place); synchronises."""
    _require_cuda(X, Omega, mean, Phi, sigma, work)
    n, ldx = X.shape
    m = ldx if m is None else m
    _check(lib().ens_pod(n, m, _ptr(X), ldx, k, l, _ptr(Omega), power_iters, _ptr(mean), _ptr(Phi),
                         _ptr(sigma), _ptr(work), _nbytes(work), _stream(stream)))


def pod_targets(X, Phi, coef_mean, coef_scale, T, work=None, m=None, stream=None):
    """Standardised coefficients T (float32 m x k) of the centred snapshots X."""
    import torch
    _require_cuda(X, Phi, coef_mean, coef_scale, T)
    n, ldx = X.shape
    m = ldx if m is None else m
    k = Phi.shape[1]
    if work is None:
        v = ctypes.c_size_t()
        _check(lib().ens_pod_targets_workspace_size(n, m, k, ctypes.byref(v)))
        work = torch.empty(v.value, dtype=torch.uint8, device=X.device)
    _check(lib().ens_pod_targets(n, m, _ptr(X), ldx, k, _ptr(Phi), _ptr(coef_mean), _ptr(coef_scale),
                                 _ptr(T), _ptr(work), _nbytes(work), _stream(stream)))


def to_f32(src, dst, stream=None):
    _require_cuda(src, dst)
    _check(lib().ens_to_f32(src.numel(), _ptr(src), _ptr(dst), _stream(stream)))


def mlp_param_count(dims=MLP_DIMS):
    v = ctypes.c_int64()
    _check(lib().ens_mlp_param_count(_dims(dims), ctypes.byref(v)))
    return v.value


def mlp_init(u, params, dims=MLP_DIMS, stream=None):
    _require_cuda(u, params)
    _check(lib().ens_mlp_init(_dims(dims), _ptr(u), _ptr(params), _stream(stream)))


def mlp_workspace_size(batch, dims=MLP_DIMS):
    v = ctypes.c_size_t()
    _check(lib().ens_mlp_workspace_size(_dims(dims), batch, ctypes.byref(v)))
    return v.value


def mlp_forward(params, xin, y, work, dims=MLP_DIMS, stream=None):
    _require_cuda(params, xin, y, work)
    _check(lib().ens_mlp_forward(_dims(dims), _ptr(params), xin.shape[0], _ptr(xin), _ptr(y), _ptr(work),
                                 _nbytes(work), _stream(stream)))


def mlp_grad(params, xin, target, grad, work, loss=None, dims=MLP_DIMS, stream=None):
    _require_cuda(params, xin, target, grad, work, loss)
    _check(lib().ens_mlp_grad(_dims(dims), _ptr(params), xin.shape[0], _ptr(xin), _ptr(target), _ptr(grad),
                              _ptr(loss), _ptr(work), _nbytes(work), _stream(stream)))


def mlp_adam(params, grad, m, v, step, total_steps, lr0=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
             stream=None):
    """step: int64 device tensor of 2 (step count, scratch 0)."""
    _require_cuda(params, grad, m, v, step)
    _check(lib().ens_mlp_adam(params.numel(), _ptr(params), _ptr(grad), _ptr(m), _ptr(v), _ptr(step),
                              total_steps, lr0, beta1, beta2, eps, _stream(stream)))


def mlp_train(params, m, v, step, xin, target, batch, epochs, total_steps, work, lr0=1e-3, beta1=0.9,
              beta2=0.999, eps=1e-8, epoch_loss=None, use_graph=True, dims=MLP_DIMS, stream=None):
    _require_cuda(params, m, v, step, xin, target, work, epoch_loss)
    _check(lib().ens_mlp_train(_dims(dims), _ptr(params), _ptr(m), _ptr(v), _ptr(step), xin.shape[0],
                               _ptr(xin), _ptr(target), batch, epochs, total_steps, lr0, beta1, beta2, eps,
                               _ptr(epoch_loss), 1 if use_graph else 0, _ptr(work), _nbytes(work),
                               _stream(stream)))


def guess_workspace_size(s, dims=MLP_DIMS):
    v = ctypes.c_size_t()
    _check(lib().ens_guess_workspace_size(_dims(dims), s, ctypes.byref(v)))
    return v.value


def guess(params, s, xi, mean, Phi32, coef_mean, coef_scale, x0, work, dims=MLP_DIMS, stream=None):
    """x0 (n*s, commuted layout) = mean + Phi (coef_mean + coef_scale * MLP(xi))."""
    _require_cuda(params, xi, mean, Phi32, coef_mean, coef_scale, x0, work)
    _check(lib().ens_guess(_dims(dims), _ptr(params), mean.numel(), s, _ptr(xi), _ptr(mean), _ptr(Phi32),
                           _ptr(coef_mean), _ptr(coef_scale), _ptr(x0), _ptr(work), _nbytes(work),
                           _stream(stream)))


# ------------------------------------------------------------ convenience
class Mesh:
    """Per-mesh, sample-independent set-up on the GPU: graph, boundary mask,
    KL tables and mode matrices (all computed by library kernels)."""

    def __init__(self, N, M, L=1.0, device="cuda", with_elem_graph=False, stream=None):
        import torch
        self.N, self.M, self.L = N, M, L
        n, nnz, nc = mesh_sizes(N)
        self.n, self.nnz, self.ncells = n, nnz, nc
        dev = torch.device(device)
        self.row_map = torch.empty(n + 1, dtype=torch.int32, device=dev)
        self.col_entry = torch.empty(nnz, dtype=torch.int32, device=dev)
        self.bmask = torch.empty(n, dtype=torch.uint8, device=dev)
        self.elem_graph = torch.empty(nc * 64, dtype=torch.int32, device=dev) if with_elem_graph else None
        graph_build(N, self.row_map, self.col_entry, self.elem_graph, self.bmask, stream)
        self.graph = Graph(self.row_map, self.col_entry)
        self.kl_table = torch.empty(kl_table_size(N, M), dtype=torch.float64, device=dev)
        self.kl_lambda, self.kl_pqr = kl_setup(N, M, L, self.kl_table, True, stream)
        self.modes = torch.empty((M + 1) * nnz, dtype=torch.float64, device=dev)
        self.load = torch.empty(n, dtype=torch.float64, device=dev)
        mode_matrices(N, self.graph, M, self.kl_table, self.modes, self.load, stream)

    def assemble(self, s, xi_ens, sigma=0.1, kappa0=1.0, values=None, b=None, stream=None, df=False,
                 values_df=None, check=True):
        """xi_ens: device float64[M*s] (commuted layout).  Returns (values, b).
        df / values_df: see assemble().  check: the coefficient positivity
        check with this mesh's KL table (synchronises the stream)."""
        import torch
        dev = self.row_map.device
        if values is None:
            values = torch.empty(self.nnz * s, dtype=torch.float64, device=dev)
        if b is None:
            b = torch.empty(self.n * s, dtype=torch.float64, device=dev)
        assemble(self.graph, self.bmask, s, self.M, self.modes, self.load, xi_ens, sigma, kappa0,
                 values, b, stream, df=df, values_df=values_df, kl_table=self.kl_table if check else None)
        return values, b
