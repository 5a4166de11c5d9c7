"""GB300 (sm_103a) column-block SVD of sparse short-and-fat matrices.

Implements the data-parallel path of Ranky (Tugay & Gunduz Oguducu, arXiv
2009.09767, section III, Algorithm 1): column blocks, lonely-node detection
and RandomChecker insertion (Algorithm 2), block SVDs (Eq. 1) through block
cross products and a Jacobi eigensolver, the proxy matrix and its SVD
(Eqs. 2-3), and right vectors V = A'^T U S^-1.

This module is the thin Python binding of the C ABI in ``include/ranky.h``
(``libranky.so``): it only marshals arguments.  Every step runs in the CUDA
kernels of the library; there is no CPU fallback.  PyTorch supplies device
memory and streams.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libranky.so")

SVD_OK = 0
STATUS_NAMES = {
    0: "SVD_OK", 1: "SVD_ERR_INVALID_ARG", 2: "SVD_ERR_INVALID_CSC", 3: "SVD_ERR_OOM",
    4: "SVD_ERR_BUDGET", 5: "SVD_ERR_CUDA", 6: "SVD_ERR_NOT_CONVERGED", 7: "SVD_ERR_TIMEOUT",
    8: "SVD_ERR_UNSUPPORTED",
}
PREC = {"fp64": 0, "mixed": 1}
RANKFIX = {"truncate": 0, "random": 1, "neighbor": 2, "neighbor_random": 3}
VALUE = {"f32": 0, "f64": 1}
FLAG_CHECK_CSC = 1
FLAG_SKIP_V = 2
FLAG_TIMING = 4
FLAG_DENSE_REFINE = 8
FLAG_FP64_PRODUCTS = 16
FLAG_TALL = 32
FLAG_LEGACY_MMA = 64
STAGES = ["partition", "gram", "block_jacobi", "block_refine", "sort_proxy", "merge_gram",
          "merge_eig", "finalize", "spmm"]

Q_BLOCK_BOUNDS, Q_LONELY, Q_ROW_NONEMPTY, Q_BLOCK_RANKS, Q_BLOCK_SIGMA = 1, 2, 3, 4, 5
Q_BLOCK_GRAM, Q_PROXY_COLS, Q_PROXY, Q_SWEEPS, Q_LAUNCHES, Q_MERGE_GRAM = 6, 7, 8, 9, 10, 11
Q_STAGE_MS = 12
Q_STAGE_TOTAL = 13


class RankyError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)}")


class SvdDesc(ctypes.Structure):
    _fields_ = [
        ("M", ctypes.c_int32), ("N", ctypes.c_int64), ("nnz", ctypes.c_int64),
        ("value_type", ctypes.c_int32), ("num_blocks", ctypes.c_int32),
        ("block_col_bounds", ctypes.c_void_p), ("k", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("rank_fix", ctypes.c_int32),
        ("seed", ctypes.c_uint64), ("rank_tol", ctypes.c_double),
        ("max_sweeps", ctypes.c_int32), ("jacobi_tol", ctypes.c_double),
        ("refine_iters", ctypes.c_int32), ("flags", ctypes.c_int32),
        ("merge_arity", ctypes.c_int32), ("jacobi_cluster", ctypes.c_int32),
        ("merge_rank", ctypes.c_int32),
    ]


class SvdPatch(ctypes.Structure):
    _fields_ = [("row", ctypes.c_int32), ("block", ctypes.c_int32), ("col", ctypes.c_int64)]


_lib = None


def load_library():
    """Load ``libranky.so``; raise if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, I64, U64, D, SZ = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                               ctypes.c_double, ctypes.c_size_t)
    sigs = {
        "svd_plan": ([ctypes.POINTER(SvdDesc), ctypes.POINTER(P), ctypes.POINTER(SZ)], I32),
        "svd_plan_bytes": ([ctypes.POINTER(SvdDesc), ctypes.POINTER(SZ)], I32),
        "svd_run": ([P] * 10 + [P], I32),
        "svd_run_host": ([P] * 10 + [P], I32),
        "svd_sync": ([P], I32),
        "svd_check_csc": ([I32, I64, I64, P, P, P], I32),
        "svd_query": ([P, I32, I64, P, SZ], I32),
        "svd_free": ([P], None),
        "svd_status_str": ([I32], ctypes.c_char_p),
        "svd_version": ([], I32),
    }
    for name, (args, res) in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(status: int, what: str):
    if status != SVD_OK:
        raise RankyError(status, what)


def make_desc(M, N, nnz, num_blocks, *, bounds=None, k=0, precision="mixed",
              rank_fix="truncate", seed=0, value_type="f32", rank_tol=0.0, max_sweeps=0,
              jacobi_tol=0.0, refine_iters=-1, flags=0, merge_arity=0, merge_rank=0,
              jacobi_cluster=0):
    d = SvdDesc()
    d.M, d.N, d.nnz = int(M), int(N), int(nnz)
    d.value_type = VALUE[value_type] if isinstance(value_type, str) else int(value_type)
    d.num_blocks = int(num_blocks)
    keep = None
    if bounds is not None:
        keep = np.ascontiguousarray(bounds, dtype=np.int64)
        d.block_col_bounds = keep.ctypes.data
    d.k = int(k)
    d.precision = PREC[precision] if isinstance(precision, str) else int(precision)
    d.rank_fix = RANKFIX[rank_fix] if isinstance(rank_fix, str) else int(rank_fix)
    d.seed = int(seed)
    d.rank_tol = float(rank_tol)
    d.max_sweeps = int(max_sweeps)
    d.jacobi_tol = float(jacobi_tol)
    d.refine_iters = int(refine_iters)
    d.flags = int(flags)
    d.merge_arity = int(merge_arity)
    d.merge_rank = int(merge_rank)
    d.jacobi_cluster = int(jacobi_cluster)
    return d, keep


def plan_bytes(M, N, nnz, num_blocks, **kw) -> int:
    lib = load_library()
    d, keep = make_desc(M, N, nnz, num_blocks, **kw)
    out = ctypes.c_size_t(0)
    _check(lib.svd_plan_bytes(ctypes.byref(d), ctypes.byref(out)), "svd_plan_bytes")
    del keep
    return int(out.value)


def _ptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return ctypes.c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray):
        return ctypes.c_void_p(t.ctypes.data)
    return ctypes.c_void_p(int(t))


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


class Plan:
    """One svd_plan: fixed shapes, owns its device workspace."""

    def __init__(self, M, N, nnz, num_blocks, **kw):
        lib = load_library()
        self.M, self.N, self.nnz, self.D = int(M), int(N), int(nnz), int(num_blocks)
        self.precision = kw.get("precision", "mixed")
        self.rank_fix = kw.get("rank_fix", "truncate")
        self.value_type = kw.get("value_type", "f32")
        k = int(kw.get("k", 0))
        self.k = k if k > 0 else min(self.M, self.N)
        # tall plans (FLAG_TALL): the problem solved is A^T; its short side is N
        self.tall = bool(int(kw.get("flags", 0)) & FLAG_TALL)
        self.Ms = self.N if self.tall else self.M
        d, keep = make_desc(M, N, nnz, num_blocks, **kw)
        h = ctypes.c_void_p()
        nbytes = ctypes.c_size_t(0)
        _check(lib.svd_plan(ctypes.byref(d), ctypes.byref(h), ctypes.byref(nbytes)), "svd_plan")
        del keep
        self._h = h
        self.workspace_bytes = int(nbytes.value)

    @property
    def handle(self):
        return self._h

    def run(self, col_ptr, row_idx, vals, sigma, U, V, rank, patches=None, npatches=None,
            stream=None):
        """Enqueue the SVD on device tensors (see svd_run in include/ranky.h)."""
        lib = load_library()
        st = lib.svd_run(self._h, _ptr(col_ptr), _ptr(row_idx), _ptr(vals), _ptr(sigma), _ptr(U),
                         _ptr(V), _ptr(rank), _ptr(patches), _ptr(npatches),
                         _stream_handle(stream))
        _check(st, "svd_run")

    def run_host(self, col_ptr, row_idx, vals, sigma, U, V, rank, patches=None, npatches=None,
                 stream=None):
        """Same from host arrays (numpy or pinned torch CPU tensors); synchronous."""
        lib = load_library()
        st = lib.svd_run_host(self._h, _ptr(col_ptr), _ptr(row_idx), _ptr(vals), _ptr(sigma),
                              _ptr(U), _ptr(V), _ptr(rank), _ptr(patches), _ptr(npatches),
                              _stream_handle(stream))
        _check(st, "svd_run_host")

    def sync(self):
        _check(load_library().svd_sync(self._h), "svd_sync")

    def query(self, what: int, index: int = 0):
        lib = load_library()
        D, M = self.D, self.Ms
        if what == Q_BLOCK_BOUNDS:
            out = np.zeros(D + 1, np.int64)
        elif what == Q_LONELY:
            out = np.zeros((D, M), np.uint8)
        elif what == Q_ROW_NONEMPTY:
            out = np.zeros(M, np.uint8)
        elif what == Q_BLOCK_RANKS:
            out = np.zeros(D, np.int32)
        elif what == Q_BLOCK_SIGMA:
            out = np.zeros((D, M), np.float64)
        elif what in (Q_BLOCK_GRAM, Q_MERGE_GRAM):
            out = np.zeros((M, M), np.float64)
        elif what in (Q_PROXY_COLS, Q_LAUNCHES):
            out = np.zeros(1, np.int64)
        elif what == Q_PROXY:
            R = int(self.query(Q_PROXY_COLS)[0])
            out = np.zeros((R, M), np.float64)  # column-major M x R
        elif what == Q_SWEEPS:
            out = np.zeros(D + 1, np.int32)
        elif what == Q_STAGE_MS:
            out = np.zeros(len(STAGES), np.float32)
        elif what == Q_STAGE_TOTAL:
            out = np.zeros(len(STAGES) + 1, np.float64)
        else:
            raise ValueError(what)
        _check(lib.svd_query(self._h, int(what), int(index), _ptr(out), out.nbytes), "svd_query")
        if what == Q_PROXY:
            return out.T.copy()
        return out

    def free(self):
        if getattr(self, "_h", None):
            load_library().svd_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def alloc_outputs(plan: Plan, device="cuda", with_patches=True):
    """Device output tensors for a plan (torch).  Short-fat plans: U column-major
    M x k FP64 (stored k x M), V row-major N x k.  Tall plans: U row-major M x k
    in the long-side type, V column-major N x k FP64 (stored k x N)."""
    import torch
    vdt = torch.float32 if plan.precision == "mixed" else torch.float64
    if plan.tall:
        U = torch.empty(plan.M, plan.k, dtype=vdt, device=device)
        V = torch.empty(plan.k, plan.N, dtype=torch.float64, device=device)
    else:
        U = torch.empty(plan.k, plan.M, dtype=torch.float64, device=device)
        V = torch.empty(plan.N, plan.k, dtype=vdt, device=device)
    out = {
        "sigma": torch.empty(plan.k, dtype=torch.float64, device=device),
        "U": U,
        "V": V,
        "rank": torch.zeros(1, dtype=torch.int32, device=device),
    }
    if with_patches:
        out["patches"] = torch.zeros(plan.D * plan.Ms, 2, dtype=torch.int64, device=device)
        out["npatches"] = torch.zeros(1, dtype=torch.int64, device=device)
    return out


def svd(col_ptr, row_idx, vals, M, N, num_blocks, *, stream=None, plan: Plan | None = None,
        **kw):
    """SVD of a device CSC matrix.  Returns (plan, outputs) with outputs
    sigma (k), U (M x k), V (N x k), rank, patches (P x 2: row, col) as torch
    tensors; U and V are views in the natural orientation."""
    import torch
    vt = "f32" if vals.dtype == torch.float32 else "f64"
    if plan is None:
        plan = Plan(M, N, int(row_idx.numel()), num_blocks, value_type=vt, **kw)
    out = alloc_outputs(plan, device=vals.device)
    plan.run(col_ptr, row_idx, vals, out["sigma"], out["U"], out["V"], out["rank"],
             out["patches"], out["npatches"], stream=stream)
    plan.sync()
    n = int(out["npatches"].item())
    pr = out["patches"].view(-1)[: 2 * plan.D * plan.Ms].view(-1, 2)[:n]
    # svd_patch = {int32 row, int32 block, int64 col}: decode the two int64 words
    row = (pr[:, 0] & 0xFFFFFFFF).to(torch.int64)
    blk = (pr[:, 0] >> 32).to(torch.int64)
    col = pr[:, 1]
    res = {
        "sigma": out["sigma"],
        "U": out["U"] if plan.tall else out["U"].t(),
        "V": out["V"].t() if plan.tall else out["V"],
        "rank": int(out["rank"].item()),
        "patches": torch.stack([row, col], dim=1),
        "patch_blocks": blk,
    }
    return plan, res


def right_vectors_static(M, N, col_ptr, row_idx, vals, sigma, U, V, *, k=None, rank_tol=0.0,
                         patches=None, npatches=None, max_patches=0, stream=None):
    """V = A'^T U_k S_k^-1 through svd_right_vectors_static: no device
    allocation; the weights live in the library's static 4 MiB device array
    (see include/ranky.h for the sharing rules)."""
    lib = load_library()
    f = lib.svd_right_vectors_static
    if f.argtypes is None:
        P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        f.argtypes = [I32, I64, I64, I32, P, P, P, I32, P, P, ctypes.c_double, P, P, I64, I32,
                      P, P]
        f.restype = I32
    import torch
    kk = int(sigma.numel()) if k is None else int(k)
    vt = 0 if vals.dtype == torch.float32 else 1
    vv = 0 if V.dtype == torch.float32 else 1
    st = f(int(M), int(N), int(row_idx.numel()), vt, _ptr(col_ptr), _ptr(row_idx), _ptr(vals), kk,
           _ptr(sigma), _ptr(U), float(rank_tol), _ptr(patches), _ptr(npatches), int(max_patches),
           vv, _ptr(V), _stream_handle(stream))
    _check(st, "svd_right_vectors_static")


PRODUCT_SYM = 1
PRODUCT_LEGACY_MMA = 2


def exact_product(A, B=None, *, slices=5, legacy=False, out=None, err=None, stream=None):
    """C = A B^T (B = A when None: symmetric, upper tiles mirrored) for FP64
    device tensors, through svd_exact_product: exact 8-bit slices on the bf16
    tensor cores (tcgen05 with TMEM accumulators, or mma.sync when legacy).
    The workspace is a torch allocation; err, when given, is a device int32
    tensor that a timed-out wait sets to 1."""
    import torch
    lib = load_library()
    f = lib.svd_exact_product
    if f.argtypes is None:
        P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        f.argtypes = [I32, I32, I64, P, I64, P, I64, P, I64, I32, I32, P, ctypes.c_size_t, P, P]
        f.restype = I32
        g = lib.svd_exact_product_bytes
        g.argtypes = [I32, I32, I64, I32]
        g.restype = ctypes.c_size_t
    sym = B is None
    m, k = A.shape
    n = m if sym else B.shape[0]
    nbytes = lib.svd_exact_product_bytes(m, n, k, slices)
    work = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=A.device)
    C = torch.empty(m, n, dtype=torch.float64, device=A.device) if out is None else out
    flags = (PRODUCT_SYM if sym else 0) | (PRODUCT_LEGACY_MMA if legacy else 0)
    st = f(m, n, k, _ptr(A), A.stride(0), None if sym else _ptr(B), 0 if sym else B.stride(0),
           _ptr(C), C.stride(0), slices, flags, _ptr(work), int(nbytes), _ptr(err),
           _stream_handle(stream))
    _check(st, "svd_exact_product")
    return C


class SvdIo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("col_ptr", "row_idx", "vals", "sigma", "U", "V",
                                                "rank", "patches", "npatches")]


BATCH_GRAPH = 1


class Batch:
    """svd_batch_*: many plans in one pass (see include/ranky.h)."""

    def __init__(self, plans, graph: bool = False):
        lib = load_library()
        for name, args, res in (
            ("svd_batch_create", [ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                  ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int32),
            ("svd_batch_run", [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int32),
            ("svd_batch_sync", [ctypes.c_void_p], ctypes.c_int32),
            ("svd_batch_launches", [ctypes.c_void_p], ctypes.c_int64),
            ("svd_batch_free", [ctypes.c_void_p], None),
        ):
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p.handle.value for p in self.plans])
        h = ctypes.c_void_p()
        _check(lib.svd_batch_create(len(self.plans), arr, BATCH_GRAPH if graph else 0,
                                    ctypes.byref(h)), "svd_batch_create")
        self._h = h
        self._ios = None

    def run(self, inputs, outputs, stream=None):
        """inputs[i] = (col_ptr, row_idx, vals); outputs[i] = alloc_outputs(plan i)."""
        lib = load_library()
        ios = (SvdIo * len(self.plans))()
        for i, ((cp, ri, va), o) in enumerate(zip(inputs, outputs)):
            ios[i] = SvdIo(cp.data_ptr(), ri.data_ptr() if ri.numel() else None,
                           va.data_ptr() if va.numel() else None, o["sigma"].data_ptr(),
                           o["U"].data_ptr(), o["V"].data_ptr(), o["rank"].data_ptr(),
                           o["patches"].data_ptr() if "patches" in o else None,
                           o["npatches"].data_ptr() if "npatches" in o else None)
        self._ios = ios
        _check(lib.svd_batch_run(self._h, ctypes.byref(ios), _stream_handle(stream)),
               "svd_batch_run")

    def sync(self):
        _check(load_library().svd_batch_sync(self._h), "svd_batch_sync")

    def launches(self) -> int:
        return int(load_library().svd_batch_launches(self._h))

    def free(self):
        if getattr(self, "_h", None):
            load_library().svd_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class SvdRequest(ctypes.Structure):
    _fields_ = [("desc", SvdDesc), ("col_ptr", ctypes.c_void_p), ("row_idx", ctypes.c_void_p),
                ("vals", ctypes.c_void_p), ("sigma", ctypes.c_void_p), ("U", ctypes.c_void_p),
                ("V", ctypes.c_void_p), ("rank", ctypes.c_void_p)]


INJECT_ALLOC = 1
INJECT_BAD_CSC = 2


class Server:
    """svd_server_*: continuous-batching service (see include/ranky.h).  Host
    arrays passed to submit() are kept alive here until release()."""

    def __init__(self, budget_bytes: int, max_inflight: int = 8):
        lib = load_library()
        P, I32, U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64
        for name, args, res in (
            ("svd_server_create", [ctypes.c_size_t, I32, ctypes.POINTER(P)], I32),
            ("svd_server_submit", [P, ctypes.POINTER(SvdRequest), ctypes.POINTER(U64)], I32),
            ("svd_server_poll", [P, U64, ctypes.POINTER(I32), ctypes.POINTER(I32)], I32),
            ("svd_server_wait", [P, U64, ctypes.c_double, ctypes.POINTER(I32)], I32),
            ("svd_server_cancel", [P, U64], I32),
            ("svd_server_times", [P, U64, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], I32),
            ("svd_server_release", [P, U64], I32),
            ("svd_server_stats", [P, P], I32),
            ("svd_server_inject", [P, I32, U64], I32),
            ("svd_server_destroy", [P], None),
        ):
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        h = ctypes.c_void_p()
        _check(lib.svd_server_create(int(budget_bytes), int(max_inflight), ctypes.byref(h)),
               "svd_server_create")
        self._h = h
        self._keep = {}

    def submit(self, M, N, col_ptr, row_idx, vals, num_blocks, outputs, **kw) -> int:
        """Host arrays in (numpy or pinned torch CPU tensors); outputs = dict with
        host 'sigma', 'U' (k x M), 'V' (N x k, or None) and 'rank'."""
        vt = "f32" if vals.dtype in (np.float32,) or str(vals.dtype).endswith("float32") else "f64"
        d, keep = make_desc(M, N, len(row_idx), num_blocks, value_type=vt, **kw)
        req = SvdRequest(d, _ptr(col_ptr), _ptr(row_idx) if len(row_idx) else None,
                         _ptr(vals) if len(vals) else None, _ptr(outputs["sigma"]),
                         _ptr(outputs["U"]), _ptr(outputs.get("V")), _ptr(outputs["rank"]))
        t = ctypes.c_uint64(0)
        _check(load_library().svd_server_submit(self._h, ctypes.byref(req), ctypes.byref(t)),
               "svd_server_submit")
        self._keep[t.value] = (col_ptr, row_idx, vals, outputs, keep)
        return int(t.value)

    def wait(self, ticket: int, timeout: float = 60.0) -> int:
        """Returns the request's status (0 = ok); raises on timeout."""
        res = ctypes.c_int32(0)
        _check(load_library().svd_server_wait(self._h, ticket, float(timeout), ctypes.byref(res)),
               "svd_server_wait")
        return int(res.value)

    def wait_status(self, ticket: int, timeout: float):
        """(call status, request status) without raising."""
        res = ctypes.c_int32(-1)
        st = load_library().svd_server_wait(self._h, ticket, float(timeout), ctypes.byref(res))
        return int(st), int(res.value)

    def poll(self, ticket: int):
        done, res = ctypes.c_int32(0), ctypes.c_int32(0)
        _check(load_library().svd_server_poll(self._h, ticket, ctypes.byref(done), ctypes.byref(res)),
               "svd_server_poll")
        return bool(done.value), int(res.value)

    def cancel(self, ticket: int) -> int:
        return int(load_library().svd_server_cancel(self._h, ticket))

    def times(self, ticket: int):
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(load_library().svd_server_times(self._h, ticket, ctypes.byref(a), ctypes.byref(b),
                                               ctypes.byref(c)), "svd_server_times")
        return a.value, b.value, c.value

    def release(self, ticket: int):
        _check(load_library().svd_server_release(self._h, ticket), "svd_server_release")
        self._keep.pop(ticket, None)

    def stats(self) -> dict:
        out = np.zeros(8, np.int64)
        _check(load_library().svd_server_stats(self._h, _ptr(out)), "svd_server_stats")
        keys = ["submitted", "completed", "failed", "rejected", "running", "queued", "pool_used",
                "pool_peak"]
        return dict(zip(keys, (int(x) for x in out)))

    def inject(self, what: int, ticket: int):
        _check(load_library().svd_server_inject(self._h, int(what), int(ticket)), "svd_server_inject")

    def close(self):
        if getattr(self, "_h", None):
            load_library().svd_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def host_outputs(M, N, k, precision="mixed", with_v=True, pinned=False):
    """Host output buffers for Server.submit / Plan.run_host."""
    vdt = np.float32 if precision == "mixed" else np.float64
    out = {"sigma": np.zeros(k), "U": np.zeros((k, M)), "rank": np.zeros(1, np.int32),
           "V": np.zeros((N, k), vdt) if with_v else None}
    if pinned:
        import torch
        for key in ("sigma", "U", "rank", "V"):
            if out[key] is not None:
                t = torch.from_numpy(out[key]).pin_memory()
                out[key] = t.numpy()
                out[key + "_pinned"] = t
    return out
