"""Python binding of the GB300 dashSVD library (libdashsvd.so).

Thin ctypes marshalling over the C ABI declared in include/dashsvd.h; every
step of the computation runs in the library's CUDA kernels. The functions
``dashsvd_*`` take plain ints (device or host addresses) exactly like the C
entry points. ``Handle`` and ``CsrDevice`` add argument marshalling for torch
tensors (PyTorch provides device memory and streams only).

The library must have been built (``python paper_2404_09276_gb300/build.py``
or ``__graft_entry__.build()``); importing this module without it raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdashsvd.so")

# ---- status codes (dashsvd_status) -------------------------------------------
DASHSVD_OK = 0
DASHSVD_MAX_PASSES = 1
DASHSVD_LEARNED_STOP = 2
DASHSVD_EINVAL = -1
DASHSVD_ENOMEM = -2
DASHSVD_ECUDA = -3
DASHSVD_ENONFINITE = -4
DASHSVD_ETIMEOUT = -5
DASHSVD_ENOTIMPL = -6
DASHSVD_ENOCONV = -7
DASHSVD_FORM_PLAIN = 0
DASHSVD_FORM_PRECISION = 1
DASHSVD_MAX_L = 256

# every entry point the header declares (checked by the ABI test)
EXPORTS = (
    "dashsvd_options_init", "dashsvd_create", "dashsvd_destroy", "dashsvd_run", "dashsvd_get_trace",
    "dashsvd_load_mlp", "dashsvd_status_string", "dashsvd_last_error", "dashsvd_gaussian",
    "dashsvd_csr_transpose", "dashsvd_spmm", "dashsvd_spmm_shift", "dashsvd_spmm_bf16", "dashsvd_gram",
    "dashsvd_gram_bf16x3",
    "dashsvd_project", "dashsvd_project_bf16x3", "dashsvd_eigsvd", "dashsvd_gram_noalloc",
    "dashsvd_mlp_features", "dashsvd_mlp_forward", "dashsvd_mlp_loss_grad", "dashsvd_mlp_adam",
    "dashsvd_get_tuning", "dashsvd_spmm_fused", "dashsvd_metrics", "dashsvd_selftest_bounded_wait",
    "dashsvd_selftest_fail_alloc", "dashsvd_csr_check", "dashsvd_eig_fp64", "dashsvd_get_profile",
    "dashsvd_run_host",
)
MLP_PARAMS = 1218
MLP_IN = 16


class dashsvd_csr(C.Structure):
    _fields_ = [
        ("m", C.c_int64), ("n", C.c_int64), ("nnz", C.c_int64),
        ("rowptr", C.c_void_p), ("colidx", C.c_void_p), ("val", C.c_void_p),
    ]


class dashsvd_options(C.Structure):
    _fields_ = [
        ("form", C.c_int32), ("learned", C.c_int32), ("seed", C.c_uint64),
        ("alpha_prev_mode", C.c_int32), ("use_graph", C.c_int32), ("spmm_variant", C.c_int32),
        ("record_trace", C.c_int32), ("shift", C.c_int32), ("gather_bf16", C.c_int32),
        ("pve_mode", C.c_int32), ("trust_csr", C.c_int32), ("deterministic", C.c_int32),
        ("profile", C.c_int32), ("overlap", C.c_int32), ("reserved", C.c_int32 * 1),
    ]


class dashsvd_info(C.Structure):
    _fields_ = [
        ("passes", C.c_int32), ("status", C.c_int32), ("transposed", C.c_int32),
        ("spmm_variant", C.c_int32), ("alpha", C.c_double), ("pve_ratio", C.c_double),
        ("workspace_bytes", C.c_int64), ("eig_sweeps", C.c_int32), ("setup_reused", C.c_int32),
        ("reserved", C.c_int32 * 4),
    ]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`"
        )
    lib = C.CDLL(LIB_PATH)
    P, I, I64, D, U64 = C.c_void_p, C.c_int, C.c_int64, C.c_double, C.c_uint64
    sig = {
        "dashsvd_options_init": (I, [P]),
        "dashsvd_create": (I, [P, P, P]),
        "dashsvd_destroy": (I, [P]),
        "dashsvd_run": (I, [P, P, I, I, I, D, P, P, P, P]),
        "dashsvd_get_trace": (I, [P, P, I64, P, P]),
        "dashsvd_load_mlp": (I, [P, P, I64]),
        "dashsvd_status_string": (C.c_char_p, [I]),
        "dashsvd_last_error": (C.c_char_p, []),
        "dashsvd_gaussian": (I, [P, U64, I64, I, I64, P, I64]),
        "dashsvd_csr_transpose": (I, [P, P, P, P, P]),
        "dashsvd_spmm": (I, [P, P, P, I64, I, P, I64, I]),
        "dashsvd_spmm_shift": (I, [P, P, P, I64, I, P, P, I64, P, I64, I]),
        "dashsvd_spmm_bf16": (I, [P, P, P, I64, I, P, I, I64, P, P, I64, I]),
        "dashsvd_gram": (I, [P, P, I64, I, I64, P, I64]),
        "dashsvd_gram_bf16x3": (I, [P, P, I64, I, I64, P, I64]),
        "dashsvd_project": (I, [P, P, I64, I, I64, P, I64, I, P, I64]),
        "dashsvd_project_bf16x3": (I, [P, P, I64, I, I64, P, I64, I, P, I64]),
        "dashsvd_eigsvd": (I, [P, P, I64, I, I64, P, I64, P, P, I]),
        "dashsvd_gram_noalloc": (I, [P, I64, I, I64, P, I64, P]),
        "dashsvd_mlp_features": (I, [P, P, I64, I, I, I, D, P]),
        "dashsvd_get_tuning": (I, [P, P, I64]),
        "dashsvd_spmm_fused": (I, [P, P, P, I64, I, P, P, I64]),
        "dashsvd_metrics": (I, [P, P, I, P, I64, P, P, I64, P, I, I, U64, P]),
        "dashsvd_selftest_bounded_wait": (I, [P, C.c_uint32]),
        "dashsvd_selftest_fail_alloc": (I, [I]),
        "dashsvd_csr_check": (I, [P, P, P]),
        "dashsvd_eig_fp64": (I, [P, P, I64, I, I, P, P]),
        "dashsvd_get_profile": (I, [P, P, I64]),
        "dashsvd_run_host": (I, [P, P, I, I, I, D, P, P, P, P]),
        "dashsvd_mlp_forward": (I, [P, P, P, I64, P]),
        "dashsvd_mlp_loss_grad": (I, [P, P, P, P, P, I64, P, P]),
        "dashsvd_mlp_adam": (I, [P, P, P, P, P, I, C.c_float, C.c_float, C.c_float, C.c_float]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def _export(name):
    fn = getattr(_lib, name)
    fn.__doc__ = f"C entry point {name} (see include/dashsvd.h)."
    return fn


dashsvd_options_init = _export("dashsvd_options_init")
dashsvd_create = _export("dashsvd_create")
dashsvd_destroy = _export("dashsvd_destroy")
dashsvd_run = _export("dashsvd_run")
dashsvd_get_trace = _export("dashsvd_get_trace")
dashsvd_load_mlp = _export("dashsvd_load_mlp")
dashsvd_status_string = _export("dashsvd_status_string")
dashsvd_last_error = _export("dashsvd_last_error")
dashsvd_gaussian = _export("dashsvd_gaussian")
dashsvd_csr_transpose = _export("dashsvd_csr_transpose")
dashsvd_spmm = _export("dashsvd_spmm")
dashsvd_spmm_shift = _export("dashsvd_spmm_shift")
dashsvd_spmm_bf16 = _export("dashsvd_spmm_bf16")
dashsvd_gram = _export("dashsvd_gram")
dashsvd_gram_bf16x3 = _export("dashsvd_gram_bf16x3")
dashsvd_project = _export("dashsvd_project")
dashsvd_project_bf16x3 = _export("dashsvd_project_bf16x3")
dashsvd_eigsvd = _export("dashsvd_eigsvd")
dashsvd_gram_noalloc = _export("dashsvd_gram_noalloc")
dashsvd_mlp_features = _export("dashsvd_mlp_features")
dashsvd_get_tuning = _export("dashsvd_get_tuning")
dashsvd_spmm_fused = _export("dashsvd_spmm_fused")
dashsvd_metrics = _export("dashsvd_metrics")
dashsvd_selftest_bounded_wait = _export("dashsvd_selftest_bounded_wait")
dashsvd_selftest_fail_alloc = _export("dashsvd_selftest_fail_alloc")
dashsvd_csr_check = _export("dashsvd_csr_check")
dashsvd_eig_fp64 = _export("dashsvd_eig_fp64")
dashsvd_get_profile = _export("dashsvd_get_profile")
dashsvd_run_host = _export("dashsvd_run_host")
PROFILE_CATEGORIES = ("gaussian", "spmm_fwd", "spmm_bwd", "gram", "eig", "project", "host_gap",
                      "spmm_fwd_overlapped", "eig_jacobi", "eig_refine")
DASHSVD_CSR_BAD_FIRST, DASHSVD_CSR_BAD_ORDER, DASHSVD_CSR_BAD_LAST, DASHSVD_CSR_BAD_COL = 1, 2, 4, 8
dashsvd_mlp_forward = _export("dashsvd_mlp_forward")
dashsvd_mlp_loss_grad = _export("dashsvd_mlp_loss_grad")
dashsvd_mlp_adam = _export("dashsvd_mlp_adam")


class DashSvdError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        msg = dashsvd_status_string(status).decode()
        if status == DASHSVD_ECUDA:
            msg += ": " + dashsvd_last_error().decode()
        super().__init__(f"{what}: status {status} ({msg})")
        self.status = status


def check(status: int, what: str = "dashsvd", ok=(DASHSVD_OK,)) -> int:
    if status not in ok:
        raise DashSvdError(status, what)
    return status


def options(**kw) -> dashsvd_options:
    o = dashsvd_options()
    check(dashsvd_options_init(C.byref(o)), "dashsvd_options_init")
    names = {f[0] for f in o._fields_}
    for k, v in kw.items():
        if k not in names or k == "reserved":
            raise TypeError(f"unknown dashsvd option {k!r}")
        setattr(o, k, v)
    return o


def ld_for(l: int) -> int:
    """Leading dimension the library uses for n x l FP32 blocks (l rounded up to 8)."""
    return (l + 7) // 8 * 8


@dataclass
class CsrDevice:
    """A CSR matrix whose three arrays are torch tensors on the GPU."""

    m: int
    n: int
    rowptr: "object"
    colidx: "object"
    val: "object"

    @property
    def nnz(self) -> int:
        return int(self.colidx.numel())

    def struct(self) -> dashsvd_csr:
        return dashsvd_csr(self.m, self.n, self.nnz, self.rowptr.data_ptr(), self.colidx.data_ptr(),
                           self.val.data_ptr())

    @staticmethod
    def from_host(A, device="cuda") -> "CsrDevice":
        """Copy a host CSR (any object with m, n, rowptr, colidx, val numpy arrays)."""
        import torch

        return CsrDevice(
            int(A.m), int(A.n),
            torch.as_tensor(A.rowptr, dtype=torch.int32).to(device),
            torch.as_tensor(A.colidx, dtype=torch.int32).to(device),
            torch.as_tensor(A.val, dtype=torch.float32).to(device),
        )


class Handle:
    """Owns a dashsvd_handle on the current CUDA device and stream."""

    def __init__(self, stream=None, **opts):
        import torch

        self.opts = options(**opts)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.h = C.c_void_p()
        check(dashsvd_create(C.byref(self.h), C.byref(self.opts), C.c_void_p(self.stream.cuda_stream)),
              "dashsvd_create")

    def close(self):
        if self.h:
            dashsvd_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- Alg. 5 ----------------------------------------------------------------
    def run(self, A: CsrDevice, k: int, s: int, max_passes: int, pve_tol: float, U=None, S=None, V=None):
        """dashSVD of A; returns (U m x k, S k, V n x k, info) as torch tensors on the GPU."""
        import torch

        dev = A.rowptr.device
        U = torch.empty((A.m, k), dtype=torch.float32, device=dev) if U is None else U
        S = torch.empty((k,), dtype=torch.float32, device=dev) if S is None else S
        V = torch.empty((A.n, k), dtype=torch.float32, device=dev) if V is None else V
        info = dashsvd_info()
        st = dashsvd_run(self.h, C.byref(A.struct()), k, s, max_passes, float(pve_tol), U.data_ptr(),
                         S.data_ptr(), V.data_ptr(), C.byref(info))
        check(st, "dashsvd_run", ok=(DASHSVD_OK, DASHSVD_MAX_PASSES, DASHSVD_LEARNED_STOP))
        return U, S, V, info

    def csr_check(self, A: CsrDevice) -> tuple[int, int]:
        """Device check of A's structure: (status, failed-condition bits)."""
        flags = C.c_uint32()
        st = dashsvd_csr_check(self.h, C.byref(A.struct()), C.byref(flags))
        return st, flags.value

    def eig_fp64(self, G, l: int, iters: int = 3):
        """FP64 eigenpairs (D descending, V columns) of an l x l FP64 device matrix."""
        import torch

        D = torch.empty((l,), dtype=torch.float64, device=G.device)
        V = torch.empty((l, l), dtype=torch.float64, device=G.device)
        check(dashsvd_eig_fp64(self.h, G.data_ptr(), G.stride(0), l, iters, D.data_ptr(), V.data_ptr()),
              "dashsvd_eig_fp64")
        return D, V

    def run_host(self, A, k: int, s: int, max_passes: int, pve_tol: float, U, S, V):
        """dashSVD of a HOST CSR (object with m, n and numpy rowptr / colidx / val,
        or torch CPU tensors) into HOST outputs U (m x k), S (k), V (n x k) (torch
        CPU float32 tensors, pinned for DMA copies); returns info."""
        import torch

        def ptr(x):
            return x.data_ptr() if isinstance(x, torch.Tensor) else x.ctypes.data

        nnz = int(A.colidx.shape[0])
        csr = dashsvd_csr(int(A.m), int(A.n), nnz, ptr(A.rowptr), ptr(A.colidx), ptr(A.val))
        info = dashsvd_info()
        st = dashsvd_run_host(self.h, C.byref(csr), k, s, max_passes, float(pve_tol), U.data_ptr(), S.data_ptr(),
                              V.data_ptr(), C.byref(info))
        check(st, "dashsvd_run_host", ok=(DASHSVD_OK, DASHSVD_MAX_PASSES, DASHSVD_LEARNED_STOP))
        return info

    def trace(self):
        """Per-pass records of the last run: list of (j, alpha_used, ratio, alpha_next, sweeps, Shat[l])."""
        import numpy as np

        cnt = C.c_int64()
        l = C.c_int()
        check(dashsvd_get_trace(self.h, None, 0, C.byref(cnt), C.byref(l)), "dashsvd_get_trace")
        buf = np.zeros(max(1, cnt.value * (5 + l.value)), dtype=np.float64)
        check(dashsvd_get_trace(self.h, buf.ctypes.data, buf.size, C.byref(cnt), C.byref(l)), "dashsvd_get_trace")
        rec = buf[: cnt.value * (5 + l.value)].reshape(cnt.value, 5 + l.value)
        return [(int(r[0]), r[1], r[2], r[3], int(r[4]), r[5:]) for r in rec]

    # -- step-level entry points ----------------------------------------------
    def gaussian(self, seed: int, rows: int, l: int, row0: int = 0, out=None):
        import torch

        ld = ld_for(l)
        out = torch.empty((rows, ld), dtype=torch.float32, device="cuda") if out is None else out
        check(dashsvd_gaussian(self.h, seed, rows, l, row0, out.data_ptr(), out.stride(0)), "dashsvd_gaussian")
        return out

    def csr_transpose(self, A: CsrDevice) -> CsrDevice:
        import torch

        dev = A.rowptr.device
        rp = torch.empty(A.n + 1, dtype=torch.int32, device=dev)
        ci = torch.empty(max(1, A.nnz), dtype=torch.int32, device=dev)
        va = torch.empty(max(1, A.nnz), dtype=torch.float32, device=dev)
        check(dashsvd_csr_transpose(self.h, C.byref(A.struct()), rp.data_ptr(), ci.data_ptr(), va.data_ptr()),
              "dashsvd_csr_transpose")
        return CsrDevice(A.n, A.m, rp, ci[: A.nnz], va[: A.nnz])

    def spmm(self, A: CsrDevice, X, l: int, out=None, variant: int = -1):
        import torch

        out = torch.empty((A.m, X.shape[1]), dtype=torch.float32, device=X.device) if out is None else out
        check(dashsvd_spmm(self.h, C.byref(A.struct()), X.data_ptr(), X.stride(0), l, out.data_ptr(),
                           out.stride(0), variant), "dashsvd_spmm")
        return out

    def spmm_shift(self, At: CsrDevice, Y, l: int, alpha_dev, Q, out=None, variant: int = -1):
        import torch

        out = torch.empty((At.m, Y.shape[1]), dtype=torch.float32, device=Y.device) if out is None else out
        check(dashsvd_spmm_shift(self.h, C.byref(At.struct()), Y.data_ptr(), Y.stride(0), l,
                                 alpha_dev.data_ptr() if alpha_dev is not None else None,
                                 Q.data_ptr() if Q is not None else None, Q.stride(0) if Q is not None else 0,
                                 out.data_ptr(), out.stride(0), variant), "dashsvd_spmm_shift")
        return out

    def spmm_bf16(self, A: CsrDevice, X, l: int, out, alpha_dev=None, Q=None, variant: int = -1):
        """BF16 X (and Q); out is BF16 or FP32 (torch tensors)."""
        import torch

        check(dashsvd_spmm_bf16(self.h, C.byref(A.struct()), X.data_ptr(), X.stride(0), l, out.data_ptr(),
                                1 if out.dtype == torch.bfloat16 else 0, out.stride(0),
                                alpha_dev.data_ptr() if alpha_dev is not None else None,
                                Q.data_ptr() if Q is not None else None, Q.stride(0) if Q is not None else 0,
                                variant), "dashsvd_spmm_bf16")
        return out

    def gram(self, Cm, l: int, out=None):
        import torch

        out = torch.empty((l, l), dtype=torch.float32, device=Cm.device) if out is None else out
        check(dashsvd_gram(self.h, Cm.data_ptr(), Cm.shape[0], l, Cm.stride(0), out.data_ptr(), out.stride(0)),
              "dashsvd_gram")
        return out

    def gram_bf16x3(self, Cm, l: int, out=None):
        import torch

        out = torch.empty((l, l), dtype=torch.float64, device=Cm.device) if out is None else out
        check(dashsvd_gram_bf16x3(self.h, Cm.data_ptr(), Cm.shape[0], l, Cm.stride(0), out.data_ptr(),
                                  out.stride(0)), "dashsvd_gram_bf16x3")
        return out

    def project(self, Cm, l: int, W, cols: int, out=None, ldo: int | None = None):
        import torch

        ldo = cols if ldo is None else ldo
        out = torch.empty((Cm.shape[0], ldo), dtype=torch.float32, device=Cm.device) if out is None else out
        check(dashsvd_project(self.h, Cm.data_ptr(), Cm.shape[0], l, Cm.stride(0), W.data_ptr(), W.stride(0),
                              cols, out.data_ptr(), out.stride(0)), "dashsvd_project")
        return out

    def project_bf16x3(self, Cm, l: int, W, cols: int, out=None, ldo: int | None = None):
        import torch

        ldo = cols if ldo is None else ldo
        out = torch.empty((Cm.shape[0], ldo), dtype=torch.float32, device=Cm.device) if out is None else out
        check(dashsvd_project_bf16x3(self.h, Cm.data_ptr(), Cm.shape[0], l, Cm.stride(0), W.data_ptr(), W.stride(0),
                                     cols, out.data_ptr(), out.stride(0)), "dashsvd_project_bf16x3")
        return out

    def profile(self) -> dict:
        """Per-step device milliseconds (and launch-group counts) of the last
        run made with profile=1."""
        import numpy as np

        n = len(PROFILE_CATEGORIES)
        buf = np.zeros(2 * n, dtype=np.float64)
        check(dashsvd_get_profile(self.h, buf.ctypes.data, buf.size), "dashsvd_get_profile")
        return {c: (float(buf[i]), int(buf[n + i])) for i, c in enumerate(PROFILE_CATEGORIES)}

    def tuning(self):
        """The autotuner's last measurements: (5 products x 20 variants) ms, 0 = not
        timed; variants 10..19 are 0..9 with L2 hints."""
        import numpy as np

        buf = np.zeros(100, dtype=np.float32)
        check(dashsvd_get_tuning(self.h, buf.ctypes.data, buf.size), "dashsvd_get_tuning")
        return buf.reshape(5, 20)

    def spmm_fused(self, A: CsrDevice, Q, l: int, alpha_dev=None, out=None):
        """Z = A^T (A Q) - alpha Q in one read of A (atomic scatter)."""
        import torch

        out = torch.empty((A.n, Q.shape[1]), dtype=torch.float32, device=Q.device) if out is None else out
        check(dashsvd_spmm_fused(self.h, C.byref(A.struct()), Q.data_ptr(), Q.stride(0), l,
                                 alpha_dev.data_ptr() if alpha_dev is not None else None, out.data_ptr(),
                                 out.stride(0)), "dashsvd_spmm_fused")
        return out

    # -- learned form ------------------------------------------------------------
    def load_mlp(self, weights):
        """Load the shift/stop network (1218 values, any array-like) into the handle."""
        import numpy as np

        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32).ravel())
        check(dashsvd_load_mlp(self.h, w.ctypes.data, w.size), "dashsvd_load_mlp")

    def mlp_features(self, records, l: int, k: int, max_passes: int, pve_tol: float):
        """records: torch float64 tensor (count x (5 + l)) on the GPU -> features (count x 16)."""
        import torch

        X = torch.empty((records.shape[0], MLP_IN), dtype=torch.float32, device=records.device)
        check(dashsvd_mlp_features(self.h, records.data_ptr(), records.shape[0], l, k, max_passes, pve_tol,
                                   X.data_ptr()), "dashsvd_mlp_features")
        return X

    def mlp_forward(self, W, X):
        import torch

        out = torch.empty((X.shape[0], 2), dtype=torch.float32, device=X.device)
        check(dashsvd_mlp_forward(self.h, W.data_ptr(), X.data_ptr(), X.shape[0], out.data_ptr()),
              "dashsvd_mlp_forward")
        return out

    def mlp_loss_grad(self, W, X, T, M, grad=None, loss=None):
        import torch

        grad = torch.empty((MLP_PARAMS,), dtype=torch.float32, device=X.device) if grad is None else grad
        loss = torch.empty((1,), dtype=torch.float32, device=X.device) if loss is None else loss
        check(dashsvd_mlp_loss_grad(self.h, W.data_ptr(), X.data_ptr(), T.data_ptr(), M.data_ptr(), X.shape[0],
                                    grad.data_ptr(), loss.data_ptr()), "dashsvd_mlp_loss_grad")
        return grad, loss

    def mlp_adam(self, W, grad, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
        check(dashsvd_mlp_adam(self.h, W.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(), step, lr, beta1,
                               beta2, eps), "dashsvd_mlp_adam")

    def metrics(self, A: CsrDevice, U, S, V, sigma_ref, spec_block: int = 16, spec_iters: int = 30,
                seed: int = 0x5EED) -> dict:
        """Accuracy metrics of Sec. 4 of a computed SVD (U, S, V device FP32 tensors)
        against reference singular values sigma_ref (k + 1 host values)."""
        import numpy as np

        import torch

        k = S.shape[0]
        if U.stride(0) % 4 or U.stride(1) != 1 or U.data_ptr() % 16:  # the SpMM wants 16-byte rows
            Up = torch.zeros((U.shape[0], (k + 3) // 4 * 4), dtype=torch.float32, device=U.device)
            Up[:, :k] = U[:, :k]
            U = Up
        sig = np.ascontiguousarray(np.asarray(sigma_ref, dtype=np.float64)[: k + 1])
        if sig.shape[0] != k + 1:
            raise ValueError("sigma_ref needs k + 1 values")
        out = (C.c_double * 5)()
        check(dashsvd_metrics(self.h, C.byref(A.struct()), k, U.data_ptr(), U.stride(0), S.data_ptr(),
                              V.data_ptr(), V.stride(0), sig.ctypes.data, spec_block, spec_iters, seed, out),
              "dashsvd_metrics")
        return {"eps_pve": out[0], "eps_res": out[1], "eps_sigma": out[2], "eps_spec": out[3], "spec_norm": out[4]}

    def eigsvd(self, Cm, l: int, form: int = DASHSVD_FORM_PLAIN):
        import torch

        U = torch.empty((Cm.shape[0], l), dtype=torch.float32, device=Cm.device)
        S = torch.empty((l,), dtype=torch.float32, device=Cm.device)
        V = torch.empty((l, l), dtype=torch.float32, device=Cm.device)
        check(dashsvd_eigsvd(self.h, Cm.data_ptr(), Cm.shape[0], l, Cm.stride(0), U.data_ptr(), U.stride(0),
                             S.data_ptr(), V.data_ptr(), form), "dashsvd_eigsvd")
        return U, S, V
