"""Thin Python binding of the C ABI in include/lsp.h (argument marshalling only).

Every step of the stencil setup runs in liblsp.so's CUDA kernels; this module only converts
arrays to pointers and status codes to exceptions. Device buffers are torch CUDA tensors
(PyTorch provides device memory and the stream); host buffers are numpy arrays. There is no
CPU fallback: without liblsp.so or a CUDA device the calls raise.
"""

from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# LSP_LIBRARY selects another build of the library (e.g. the bounds-checked liblsp_checks.so)
LIB_PATH = os.environ.get("LSP_LIBRARY") or os.path.join(HERE, "liblsp.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "lsp.h")

LSP_OK = 0
STATUS = {0: "LSP_OK", 1: "LSP_ERR_ARG", 2: "LSP_ERR_STATE", 3: "LSP_ERR_RESONANT_SHIFT",
          4: "LSP_ERR_CUDA", 5: "LSP_ERR_OOM", 6: "LSP_ERR_TIMEOUT", 7: "LSP_ERR_DEGENERATE",
          8: "LSP_ERR_UNSUPPORTED"}
POLICY = {"paper": 0, "local": 1, "list": 2, "mean": 3}
MODE = {"fp64": 0, "mixed": 1, "learned": 2, "dword": 3}
EIG = {"symmetric": 0, "full": 1}
FLAG_DEGENERATE, FLAG_NONSYMMETRIC, FLAG_NOT_CONVERGED = 1, 2, 4


class LspError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class StencilOpts(ctypes.Structure):
    _fields_ = [("t", ctypes.c_int), ("policy", ctypes.c_int), ("nshifts", ctypes.c_int),
                ("shifts", ctypes.POINTER(ctypes.c_double)), ("mode", ctypes.c_int),
                ("refine_steps", ctypes.c_int), ("eig_method", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("nd_leaf", ctypes.c_int),
                ("learned_gate", ctypes.c_double)]


class NdOpts(ctypes.Structure):
    _fields_ = [("leaf", ctypes.c_int), ("refine_steps", ctypes.c_int)]


class NdInfo(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("leaf", ctypes.c_int), ("max_front", ctypes.c_int),
                ("factored", ctypes.c_int), ("fronts", ctypes.c_int64),
                ("front_bytes", ctypes.c_int64), ("solve_bytes", ctypes.c_int64),
                ("flops", ctypes.c_double), ("flops_lu", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class GmresOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("restart", ctypes.c_int),
                ("max_cycles", ctypes.c_int), ("precond", ctypes.c_int)]


class GmresResult(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int),
                ("resid_precond", ctypes.c_double), ("resid_true", ctypes.c_double)]


_lib = None


def declared_symbols() -> list[str]:
    """Names of the functions declared in include/lsp.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lsp_[a-z_0-9]+)\s*\(", text)))


def lib() -> ctypes.CDLL:
    """Load liblsp.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run paper_1607_02560_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)
    sig = {
        "lsp_default_opts": (None, [ctypes.POINTER(StencilOpts)]),
        "lsp_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, vp, ctypes.POINTER(vp)]),
        "lsp_destroy": (ctypes.c_int, [vp]),
        "lsp_set_potential": (ctypes.c_int, [vp, vp, ctypes.c_int]),
        "lsp_build_stencils": (ctypes.c_int, [vp, ctypes.POINTER(StencilOpts)]),
        "lsp_apply_operator": (ctypes.c_int, [vp, vp, vp]),
        "lsp_get_rows": (ctypes.c_int, [vp, ctypes.c_char, vp, ctypes.c_int]),
        "lsp_get_rows_async": (ctypes.c_int, [vp, ctypes.c_char, vp]),
        "lsp_wait_rows": (ctypes.c_int, [vp]),
        "lsp_export_sparse_rows": (ctypes.c_int, [vp, ctypes.c_char, vp, vp, vp, i64p]),
        "lsp_get_shift_table": (ctypes.c_int, [vp, i64p, vp, vp, vp, vp, vp, vp]),
        "lsp_get_sizes": (ctypes.c_int, [vp, i64p, ctypes.POINTER(ctypes.c_int)]),
        "lsp_synchronize": (ctypes.c_int, [vp]),
        "lsp_kernel_timing": (ctypes.c_int, [vp, ctypes.c_int]),
        "lsp_kernel_times": (ctypes.c_int, [vp, ctypes.c_int, vp, vp, vp,
                                             ctypes.POINTER(ctypes.c_int)]),
        "lsp_last_error": (ctypes.c_char_p, [vp]),
        "lsp_apply_operator_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, vp, vp, vp,
                                                       vp]),
        "lsp_mlp_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_uint64, vp, ctypes.POINTER(vp)]),
        "lsp_mlp_destroy": (ctypes.c_int, [vp]),
        "lsp_mlp_param_count": (ctypes.c_int, [vp, i64p, i64p]),
        "lsp_mlp_get_params": (ctypes.c_int, [vp, vp]),
        "lsp_mlp_set_params": (ctypes.c_int, [vp, vp]),
        "lsp_mlp_training_pairs": (ctypes.c_int, [vp, vp, ctypes.c_int64, ctypes.c_uint64, vp,
                                                   vp]),
        "lsp_mlp_fit_normalization": (ctypes.c_int, [vp, vp, vp, ctypes.c_int64]),
        "lsp_mlp_forward": (ctypes.c_int, [vp, vp, ctypes.c_int64, vp]),
        "lsp_mlp_train_step": (ctypes.c_int, [vp, vp, vp, ctypes.c_int64, ctypes.c_float,
                                               ctypes.c_int, ctypes.POINTER(ctypes.c_float), vp]),
        "lsp_mlp_last_error": (ctypes.c_char_p, [vp]),
        "lsp_mlp_set_wait_limit": (ctypes.c_int, [vp, ctypes.c_uint64]),
        "lsp_mlp_set_schedule": (ctypes.c_int, [vp, ctypes.c_int]),
        "lsp_inject_alloc_failure": (None, [ctypes.c_int]),
        "lsp_set_mlp": (ctypes.c_int, [vp, vp]),
        "lsp_get_mode_used": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int)]),
        "lsp_get_gate_stats": (ctypes.c_int, [vp, i64p, vp]),
        "lsp_set_autotune": (ctypes.c_int, [vp, ctypes.c_int]),
        "lsp_get_tuning": (ctypes.c_int, [vp, ctypes.c_char_p, ctypes.c_int64]),
        "lsp_default_nd_opts": (None, [ctypes.POINTER(NdOpts)]),
        "lsp_nd_factor": (ctypes.c_int, [vp, ctypes.POINTER(NdOpts)]),
        "lsp_nd_get_info": (ctypes.c_int, [vp, ctypes.POINTER(NdInfo)]),
        "lsp_nd_plan_info": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_int, ctypes.POINTER(NdInfo),
                                             ctypes.c_int, vp, vp, vp, ctypes.c_char_p,
                                             ctypes.c_int]),
        "lsp_nd_solve": (ctypes.c_int, [vp, vp, vp]),
        "lsp_apply_rows": (ctypes.c_int, [vp, ctypes.c_char, vp, vp]),
        "lsp_default_gmres_opts": (None, [ctypes.POINTER(GmresOpts)]),
        "lsp_gmres": (ctypes.c_int, [vp, ctypes.POINTER(GmresOpts), vp, vp, ctypes.c_int,
                                      ctypes.POINTER(GmresResult)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def inject_alloc_failure(after: int) -> None:
    """The library's next `after` device allocations succeed and the one after them fails
    (LSP_ERR_OOM); a negative value clears the injection."""
    lib().lsp_inject_alloc_failure(int(after))


def _ptr(a) -> int | None:
    """Address of a torch tensor's or numpy array's storage (None passes NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(type(a))


def _on_device(a) -> int:
    return int(hasattr(a, "is_cuda") and a.is_cuda)


def apply_operator_noalloc(d: int, n: int, v, u, y, stream=None) -> None:
    """y = (L + diag v) u through lsp_apply_operator_noalloc (no device allocation).

    v, u, y: torch CUDA tensors of n^d float64. Asynchronous on `stream` (default: torch's
    current stream).
    """
    import torch

    for a in (v, u, y):
        if not _on_device(a):
            raise ValueError("apply_operator_noalloc takes device tensors")
    if stream is None:
        stream = torch.cuda.current_stream()
    st = lib().lsp_apply_operator_noalloc(d, n, _ptr(v), _ptr(u), _ptr(y),
                                          ctypes.c_void_p(stream.cuda_stream))
    if st != LSP_OK:
        raise LspError(st, f"lsp_apply_operator_noalloc(d={d}, n={n}) failed")


def nd_plan_info(n: int, leaf: int = 8, t: int = 1, nd_leaf: int = 0, d: int = 2) -> dict:
    """Host-only plan of the nested dissection (lsp_nd_plan_info): sizes, flop counts and the
    (count, |E|, |R|) of every depth, depth 0 being the root separator."""
    info = NdInfo()
    cap = 64
    cnt = np.zeros(cap, dtype=np.int32)
    s = np.zeros(cap, dtype=np.int32)
    r = np.zeros(cap, dtype=np.int32)
    err = ctypes.create_string_buffer(256)
    st = lib().lsp_nd_plan_info(d, n, leaf, t, nd_leaf, ctypes.byref(info), cap, _ptr(cnt),
                                _ptr(s), _ptr(r), err, 256)
    if st != LSP_OK:
        raise LspError(st, err.value.decode())
    out = info.as_dict()
    L = info.levels
    out["depths"] = [(int(cnt[d]), int(s[d]), int(r[d])) for d in range(min(L, cap))]
    return out


def default_opts() -> StencilOpts:
    o = StencilOpts()
    lib().lsp_default_opts(ctypes.byref(o))
    return o


class Context:
    """An lsp_ctx: one grid (d, n) on one CUDA stream."""

    def __init__(self, d: int, n: int, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        st = lib().lsp_create(d, n, ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h))
        if st != LSP_OK:
            raise LspError(st, f"lsp_create(d={d}, n={n}) failed")
        self.h = h
        self.d, self.n = d, n
        N = ctypes.c_int64()
        mu = ctypes.c_int()
        lib().lsp_get_sizes(self.h, ctypes.byref(N), ctypes.byref(mu))
        self.N = N.value
        self._keep = None
        self._pending_rows = []  # host buffers of copies in flight (get_rows_async)

    @property
    def mu(self) -> int:
        """Row width (2t+1)^d of the last build (3^d before any build)."""
        N, mu = ctypes.c_int64(), ctypes.c_int()
        self._check(lib().lsp_get_sizes(self.h, ctypes.byref(N), ctypes.byref(mu)), "get_sizes")
        return mu.value

    def _check(self, st: int, what: str):
        if st != LSP_OK:
            msg = lib().lsp_last_error(self.h)
            raise LspError(st, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "h", None):
            lib().lsp_destroy(self.h)  # waits for the copies in flight
            self.h = None
            self._pending_rows = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- the calls of include/lsp.h ----
    def set_potential(self, v):
        """v: torch CUDA tensor or numpy array, n^d float64 (a1)."""
        if getattr(v, "dtype", None) not in (np.float64,) and str(getattr(v, "dtype", "")) != "torch.float64":
            raise TypeError("v must be float64")
        if int(np.prod(v.shape)) != self.N:
            raise ValueError("v has the wrong size")
        self._check(lib().lsp_set_potential(self.h, _ptr(v), _on_device(v)), "set_potential")

    def build_stencils(self, policy="local", nshifts=0, shifts=None, mode="fp64",
                       refine_steps=0, eig_method="symmetric", use_graph=False, t=1,
                       nd_leaf=0, learned_gate=0.0):
        """Steps a2-a7 (asynchronous on the context stream). t = 2 builds 5^d-wide rows;
        nd_leaf > 0 gives each point t_j from a nested dissection with that leaf width;
        learned_gate = tau > 0 checks every learned stencil against its optimum and gives the
        points above tau the eigen path's rows."""
        o = StencilOpts()
        o.t = t
        o.learned_gate = float(learned_gate)
        o.nd_leaf = int(nd_leaf)
        o.policy = POLICY[policy] if isinstance(policy, str) else int(policy)
        o.mode = MODE[mode] if isinstance(mode, str) else int(mode)
        o.refine_steps = refine_steps
        o.eig_method = EIG[eig_method] if isinstance(eig_method, str) else int(eig_method)
        o.use_graph = int(bool(use_graph))
        o.nshifts = int(nshifts)
        if shifts is not None:
            arr = np.ascontiguousarray(shifts, dtype=np.float64)
            self._keep = arr
            o.shifts = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            o.nshifts = len(arr)
        self._check(lib().lsp_build_stencils(self.h, ctypes.byref(o)), "build_stencils")

    def apply_operator(self, u, y):
        """y = (L + diag v) u for torch CUDA tensors u, y (n^d float64).

        Asynchronous on the context's stream: order it after the producer of u and before any
        reader of y (e.g. with synchronize()).
        """
        if not (_on_device(u) and _on_device(y)):
            raise ValueError("apply_operator takes device tensors")
        self._check(lib().lsp_apply_operator(self.h, _ptr(u), _ptr(y)), "apply_operator")

    def get_rows(self, which: str, out=None):
        """Dense [n^d, |mu|] rows of Q, C or P into `out` (torch CUDA tensor or numpy array)."""
        if out is None:
            out = np.empty((self.N, self.mu), dtype=np.float64)
        self._check(lib().lsp_get_rows(self.h, which.encode(), _ptr(out), _on_device(out)),
                    "get_rows")
        return out

    def get_rows_async(self, which: str, out):
        """Start copying the rows of Q, C or P into the host array `out` (numpy array or CPU
        torch tensor of n^d x |mu| float64; pinned memory for the copy to overlap the next
        build) and return at once. `out` is kept alive until wait_rows()."""
        if _on_device(out):
            raise ValueError("get_rows_async copies into host memory; use get_rows for device")
        nbytes = out.nbytes if isinstance(out, np.ndarray) else out.numel() * out.element_size()
        if nbytes < 8 * self.N * self.mu:
            raise ValueError(f"out holds {nbytes} bytes, the rows need {8 * self.N * self.mu}")
        self._check(lib().lsp_get_rows_async(self.h, which.encode(), _ptr(out)),
                    "get_rows_async")
        self._pending_rows.append(out)
        return out

    def wait_rows(self):
        """Wait until every copy started by get_rows_async() has landed."""
        self._check(lib().lsp_wait_rows(self.h), "wait_rows")
        self._pending_rows.clear()

    def export_sparse_rows(self, which: str):
        """(rowptr int64, colidx int32, vals float64) in host memory."""
        nnz = ctypes.c_int64()
        self._check(lib().lsp_export_sparse_rows(self.h, which.encode(), None, None, None,
                                                 ctypes.byref(nnz)), "export size")
        rowptr = np.empty(self.N + 1, dtype=np.int64)
        colidx = np.empty(nnz.value, dtype=np.int32)
        vals = np.empty(nnz.value, dtype=np.float64)
        self._check(lib().lsp_export_sparse_rows(self.h, which.encode(), _ptr(rowptr),
                                                 _ptr(colidx), _ptr(vals), ctypes.byref(nnz)),
                    "export_sparse_rows")
        return rowptr, colidx, vals

    def get_shift_table(self, with_sidx=True):
        ns = ctypes.c_int64()
        self._check(lib().lsp_get_shift_table(self.h, ctypes.byref(ns), None, None, None, None,
                                              None, None), "shift table size")
        k = ns.value
        out = dict(s=np.empty(k), alpha=np.empty((k, self.mu)), c=np.empty((k, self.mu)),
                   lam=np.empty((k, 2)), flags=np.empty(k, dtype=np.int32),
                   s_idx=np.empty(self.N, dtype=np.int32) if with_sidx else None)
        self._check(lib().lsp_get_shift_table(self.h, ctypes.byref(ns), _ptr(out["s"]),
                                              _ptr(out["alpha"]), _ptr(out["c"]),
                                              _ptr(out["lam"]), _ptr(out["flags"]),
                                              _ptr(out["s_idx"])), "get_shift_table")
        return out

    def synchronize(self):
        self._check(lib().lsp_synchronize(self.h), "synchronize")

    # ---- applying the preconditioner: nested dissection of P, GMRES ----
    def nd_factor(self, leaf: int = 0, refine_steps: int = 0):
        """Factorise the current P rows by nested dissection (returns when done); every later
        solve adds `refine_steps` steps of iterative refinement."""
        o = NdOpts()
        o.leaf = int(leaf)
        o.refine_steps = int(refine_steps)
        self._check(lib().lsp_nd_factor(self.h, ctypes.byref(o)), "nd_factor")

    def nd_info(self) -> dict:
        info = NdInfo()
        self._check(lib().lsp_nd_get_info(self.h, ctypes.byref(info)), "nd_get_info")
        return info.as_dict()

    def nd_solve(self, y, x):
        """x = P^-1 y for torch CUDA tensors (n^d float64; x may be y). Stream-ordered."""
        if not (_on_device(y) and _on_device(x)):
            raise ValueError("nd_solve takes device tensors")
        self._check(lib().lsp_nd_solve(self.h, _ptr(y), _ptr(x)), "nd_solve")

    def apply_rows(self, which: str, u, y):
        """y = M u for M = Q, C or P of the last build (torch CUDA tensors). Stream-ordered."""
        if not (_on_device(u) and _on_device(y)):
            raise ValueError("apply_rows takes device tensors")
        self._check(lib().lsp_apply_rows(self.h, which.encode(), _ptr(u), _ptr(y)), "apply_rows")

    def gmres(self, f, u=None, rtol: float = 1e-6, restart: int = 40, max_cycles: int = 50,
              precond: bool = True):
        """Solve (L + diag v) u = f by GMRES preconditioned with P^-1 C (Sec. 5 settings by
        default). f and u: both numpy arrays or both torch CUDA tensors of n^d float64.
        Returns (u, result dict with iterations, converged, resid_precond, resid_true)."""
        if u is None:
            if _on_device(f):
                import torch
                u = torch.empty_like(f)
            else:
                u = np.empty_like(np.ascontiguousarray(f, dtype=np.float64))
        if _on_device(f) != _on_device(u):
            raise ValueError("f and u must both be on the device or both on the host")
        if not _on_device(f):
            f = np.ascontiguousarray(f, dtype=np.float64)
        o = GmresOpts()
        lib().lsp_default_gmres_opts(ctypes.byref(o))
        o.rtol, o.restart, o.max_cycles, o.precond = rtol, restart, max_cycles, int(bool(precond))
        res = GmresResult()
        self._check(lib().lsp_gmres(self.h, ctypes.byref(o), _ptr(f), _ptr(u), _on_device(f),
                                    ctypes.byref(res)), "gmres")
        return u, {name: getattr(res, name) for name, _ in res._fields_}

    def set_mlp(self, mlp):
        """Attach a trained Mlp for mode="learned" builds (None detaches)."""
        self._mlp = mlp
        self._check(lib().lsp_set_mlp(self.h, mlp.h if mlp is not None else None), "set_mlp")

    def mode_used(self) -> str:
        """Mode the last build actually ran ("learned" falls back to "fp64" out of range)."""
        m = ctypes.c_int()
        self._check(lib().lsp_get_mode_used(self.h, ctypes.byref(m)), "get_mode_used")
        return {v: k for k, v in MODE.items()}.get(m.value, str(m.value))

    def set_autotune(self, on: bool = True):
        """Tune launch shapes on the first build of each configuration (bit-identical rows)."""
        self._check(lib().lsp_set_autotune(self.h, int(bool(on))), "set_autotune")

    def tuning(self) -> dict:
        """{kernel key: (threads, CTAs per SM, ms with the default shape, ms tuned)}."""
        buf = ctypes.create_string_buffer(1 << 16)
        self._check(lib().lsp_get_tuning(self.h, buf, len(buf)), "get_tuning")
        out = {}
        for line in buf.value.decode().splitlines():
            k, th, ps, md, mb, _ = line.split()
            out[k] = (int(th), int(ps), float(md), float(mb))
        return out

    def gate_stats(self, with_rho: bool = True):
        """(points that fell back to the eigen path, per-point residual ratio or None) of the
        last gated learned build."""
        nf = ctypes.c_int64()
        rho = np.empty(self.N, dtype=np.float32) if with_rho else None
        self._check(lib().lsp_get_gate_stats(self.h, ctypes.byref(nf), _ptr(rho)),
                    "get_gate_stats")
        return int(nf.value), rho

    def kernel_timing(self, enable: bool):
        self._check(lib().lsp_kernel_timing(self.h, int(bool(enable))), "kernel_timing")

    def kernel_times(self) -> dict:
        cap = 512
        names = (ctypes.c_char * 32 * cap)()
        ms = np.zeros(cap)
        launches = np.zeros(cap, dtype=np.int64)
        cnt = ctypes.c_int()
        self._check(lib().lsp_kernel_times(self.h, cap, names, _ptr(ms), _ptr(launches),
                                           ctypes.byref(cnt)), "kernel_times")
        return {names[i].value.decode(): (float(ms[i]), int(launches[i]))
                for i in range(min(cnt.value, cap))}


class Mlp:
    """An lsp_mlp: the learned-stencil network (see include/lsp.h)."""

    def __init__(self, d: int, seed: int = 0, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        st = lib().lsp_mlp_create(d, seed, ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h))
        if st != LSP_OK:
            raise LspError(st, f"lsp_mlp_create(d={d}) failed")
        self.h = h
        self.d = d
        self.mu = 9 if d == 2 else 27
        self.nf = 26 if d == 2 else 126  # 5^d patch of h^2 v + the snapped shift h^2 s_j
        self.out = 2 * self.mu
        self.outp = 32 if d == 2 else 64
        self.k0 = 32 if d == 2 else 128
        tot, nw = ctypes.c_int64(), ctypes.c_int64()
        lib().lsp_mlp_param_count(self.h, ctypes.byref(tot), ctypes.byref(nw))
        self.nparams_total, self.nweights = tot.value, nw.value

    def _check(self, st: int, what: str):
        if st != LSP_OK:
            msg = lib().lsp_mlp_last_error(self.h)
            raise LspError(st, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "h", None):
            lib().lsp_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        out = np.empty(self.nparams_total, dtype=np.float32)
        self._check(lib().lsp_mlp_get_params(self.h, _ptr(out)), "get_params")
        return out

    def set_params(self, flat: np.ndarray):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        if flat.size != self.nparams_total:
            raise ValueError("wrong parameter count")
        self._check(lib().lsp_mlp_set_params(self.h, _ptr(flat)), "set_params")

    def training_pairs(self, ctx: Context, n: int, seed: int, X, T):
        """Raw (features, targets) of n random points of ctx's last eigen-path build."""
        self._check(lib().lsp_mlp_training_pairs(ctx.h, self.h, n, seed, _ptr(X), _ptr(T)),
                    "training_pairs")

    def fit_normalization(self, X, T, n: int):
        self._check(lib().lsp_mlp_fit_normalization(self.h, _ptr(X), _ptr(T), n),
                    "fit_normalization")

    def forward(self, X, n: int, Y):
        self._check(lib().lsp_mlp_forward(self.h, _ptr(X), n, _ptr(Y)), "forward")

    def train_step(self, X, T, batch: int, lr: float, apply: bool = True, grads=None) -> float:
        loss = ctypes.c_float()
        self._check(lib().lsp_mlp_train_step(self.h, _ptr(X), _ptr(T), batch, lr, int(apply),
                                             ctypes.byref(loss), _ptr(grads)), "train_step")
        return loss.value

    def set_schedule(self, schedule: int = 1):
        """2D inference: 1 = two tiles in flight per SM (default), 0 = one tile at a time,
        2 = two 256-row tiles in flight per CTA pair (rows only; slower, kept for comparison)."""
        self._check(lib().lsp_mlp_set_schedule(self.h, int(schedule)), "set_schedule")

    def set_wait_limit(self, ns: int = 0):
        """Limit (ns) of the fused kernel's operand waits; 0 restores the default (1 s)."""
        self._check(lib().lsp_mlp_set_wait_limit(self.h, int(ns)), "set_wait_limit")

    def save(self, path: str):
        np.save(path, self.get_params())

    def load(self, path: str):
        self.set_params(np.load(path))
