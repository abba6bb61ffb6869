"""Python binding of libtsk, the GB300 tensor-based sketching library.

Thin ctypes marshalling over the C ABI of include/tsk.h: every function here
only turns PyTorch CUDA tensors into pointers and sizes, calls the library and
returns tensors.  Every step of the method runs in the library's CUDA
kernels.  There is no CPU fallback: without the built library (or without a
CUDA device) the calls raise.

Names follow the paper: A_d are stream matrices (m x n), S is the k x m
sketch (Section 3.1), W the l x n second sketch (Eq. 3.6), r the target rank,
and the SCW outputs are US = U_r Sigma_r (m x r), Vt = (Q V_r)^T (r x n) with
B = US @ Vt (Algorithm 1).
"""
from __future__ import annotations

import ctypes as C
import os
import sys
from typing import List, Optional, Sequence

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtsk.so")

FP64, FP32, BF16 = 0, 1, 2
KERNEL_AUTO, KERNEL_SIMT, KERNEL_TC = 0, 1, 2
REFINE_NEVER, REFINE_ALWAYS, REFINE_AUTO = 0, 1, 2
MAX_K = 64

STATUS = {0: "TSK_OK", 1: "TSK_EINVAL", 2: "TSK_ENOMEM", 3: "TSK_ECUDA",
          4: "TSK_ENOCONV", 5: "TSK_ETIMEOUT", 6: "TSK_ERANKDEF",
          7: "TSK_EUNSUPPORTED"}

_DTYPE_PREC = {torch.float64: FP64, torch.float32: FP32, torch.bfloat16: BF16}
_PREC_COMPUTE = {FP64: torch.float64, FP32: torch.float32, BF16: torch.float32}


class TskError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Options(C.Structure):
    _fields_ = [("kernel", C.c_int32), ("refine_q", C.c_int32),
                ("max_iter", C.c_int32), ("err_mode", C.c_int32),
                ("eig_tol", C.c_double), ("spin_limit", C.c_int64),
                ("small_fp64", C.c_int32), ("gram_tile", C.c_int32)]


class MatDesc(C.Structure):
    _fields_ = [("A", C.c_void_p), ("S", C.c_void_p), ("m", C.c_int64),
                ("n", C.c_int64), ("lda", C.c_int64), ("k", C.c_int32),
                ("r", C.c_int32)]


class MatOut(C.Structure):
    _fields_ = [("US", C.c_void_p), ("Vt", C.c_void_p), ("sigma", C.c_void_p)]


class Mat2Desc(C.Structure):
    _fields_ = [("A", C.c_void_p), ("S", C.c_void_p), ("W", C.c_void_p),
                ("m", C.c_int64), ("n", C.c_int64), ("lda", C.c_int64),
                ("k", C.c_int32), ("l", C.c_int32), ("r", C.c_int32),
                ("reserved", C.c_int32)]


class RefineOpts(C.Structure):
    _fields_ = [("steps", C.c_int32), ("batch", C.c_int32), ("lr", C.c_double),
                ("eval_every", C.c_int32), ("reserved", C.c_int32),
                ("seed", C.c_uint64), ("order", C.POINTER(C.c_int32))]


class _RefineStateC(C.Structure):
    _fields_ = [("step", C.c_int32), ("reserved", C.c_int32),
                ("best_loss", C.c_double), ("best", C.c_void_p)]


class RefineState:
    """Where a resumable refiner run stands: the SGD steps taken, the best
    validated dS so far (a device tensor, k x m) and its validation loss."""

    def __init__(self, best: torch.Tensor, step: int = 0, best_loss: float = 0.0):
        self.best, self.step, self.best_loss = best, int(step), float(best_loss)


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libtsk.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build it with "
            "`python -m paper_2209_14637_gb300.build` (needs nvcc)")
    lib = C.CDLL(path)
    P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "tsk_create": ([C.POINTER(P), C.POINTER(Options)], I32),
        "tsk_destroy": ([P], I32),
        "tsk_last_error": ([P], C.c_char_p),
        "tsk_default_options": ([C.POINTER(Options)], None),
        "tsk_sync_status": ([P, P], I32),
        "tsk_gram": ([P, C.POINTER(P), I64, I64, I64, I64, I32, I32, P, I32, P], I32),
        "tsk_sketch_from_gram": ([P, P, I64, I32, I32, P, P, P], I32),
        "tsk_train_sketch": ([P, C.POINTER(P), I64, I64, I64, I64, I32, I32, I32,
                              P, P, P, P], I32),
        "tsk_approx_batch": ([P, I64, C.POINTER(MatDesc), I32, C.POINTER(MatOut),
                              P, P, P], I32),
        "tsk_plan_create": ([P, I64, C.POINTER(MatDesc), I32, C.POINTER(MatOut),
                             P, P, C.POINTER(P)], I32),
        "tsk_plan_execute": ([P, P], I32),
        "tsk_plan_destroy": ([P], I32),
        "tsk_plan_info": ([P, C.POINTER(I64), C.POINTER(I32)], I32),
        "tsk_plan_set_probe": ([P, P, P], I32),
        "tsk_error": ([P, I64, C.POINTER(MatDesc), I32, C.POINTER(MatOut), P, P], I32),
        "tsk_ivy_grad": ([P, I64, C.POINTER(MatDesc), I32, P, P, P, P], I32),
        "tsk_approx_noalloc": ([C.POINTER(MatDesc), I32, P, P, P, P], I32),
        "tsk_quantize_e4m3": ([P, C.POINTER(P), I64, I64, I64, I64, I32, C.POINTER(P), I64,
                               P, P], I32),
        "tsk_gram_e4m3": ([P, C.POINTER(P), P, I64, I64, I64, I64, P, I32, P], I32),
        "tsk_autotune": ([P, I64, C.POINTER(MatDesc), I32, I32, P], I32),
        "tsk_autotune_save": ([P, C.c_char_p], I32),
        "tsk_autotune_load": ([P, C.c_char_p], I32),
        "tsk_approx_two_sided": ([P, I64, C.POINTER(Mat2Desc), I32, C.POINTER(MatOut),
                                  P, P, P], I32),
        "tsk_train_two_sided": ([P, C.POINTER(P), I64, I64, I64, I64, I32, I32, I32, I32,
                                 D, P, P, C.POINTER(D), C.POINTER(I32), P], I32),
        "tsk_default_refine_options": ([C.POINTER(RefineOpts)], None),
        "tsk_refine_sketch": ([P, C.POINTER(MatDesc), I64, C.POINTER(MatDesc), I64, I32,
                               C.POINTER(RefineOpts), P, P, C.POINTER(D), P], I32),
        "tsk_refine_sketch_steps": ([P, C.POINTER(MatDesc), I64, C.POINTER(MatDesc), I64,
                                     I32, C.POINTER(RefineOpts), P, P,
                                     C.POINTER(_RefineStateC), I32, C.POINTER(D), P], I32),
        "tsk_array_save": ([C.c_char_p, P, I32, I64, I64], I32),
        "tsk_array_load": ([C.c_char_p, P, I64, C.POINTER(I32), C.POINTER(I64),
                            C.POINTER(I64)], I32),
        "tsk_refine_save": ([C.c_char_p, I32, I64, I64, C.POINTER(RefineOpts),
                             C.POINTER(_RefineStateC), P, P], I32),
        "tsk_refine_load": ([C.c_char_p, C.POINTER(I32), C.POINTER(I64), C.POINTER(I64),
                             C.POINTER(RefineOpts), C.POINTER(I32),
                             C.POINTER(_RefineStateC), P, P, I64], I32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _require_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("libtsk takes CUDA tensors only (no CPU fallback)")


def default_options() -> Options:
    o = Options()
    load_library().tsk_default_options(C.byref(o))
    return o


class Handle:
    """A library handle bound to the current CUDA device."""

    def __init__(self, kernel: Optional[int] = None, refine_q: Optional[int] = None,
                 max_iter: Optional[int] = None, eig_tol: Optional[float] = None,
                 spin_limit: Optional[int] = None, err_mode: Optional[int] = None,
                 small_fp64: Optional[bool] = None, gram_tile: Optional[int] = None):
        """Options left as None take the library's defaults
        (tsk_default_options, which the TSK_* environment variables can
        change): KERNEL_AUTO, REFINE_AUTO, max_iter 300, eig_tol 0 (the
        precision's own), spin_limit 2^24, err_mode 0, small_fp64 off,
        gram_tile 0."""
        lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("libtsk needs a CUDA device; none is available")
        o = default_options()
        if kernel is not None:
            o.kernel = int(kernel)
        if refine_q is not None:
            o.refine_q = int(refine_q)
        if max_iter is not None:
            o.max_iter = int(max_iter)
        if eig_tol is not None:
            o.eig_tol = float(eig_tol)
        if spin_limit is not None:
            o.spin_limit = int(spin_limit)
        if err_mode is not None:
            o.err_mode = int(err_mode)
        if small_fp64 is not None:
            o.small_fp64 = int(bool(small_fp64))
        if gram_tile is not None:
            o.gram_tile = int(gram_tile)
        h = C.c_void_p()
        st = lib.tsk_create(C.byref(h), C.byref(o))
        if st != 0:
            raise TskError(st, lib.tsk_last_error(None).decode())
        self._lib, self._h = lib, h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.tsk_destroy(self._h)
            self._h = None

    def __del__(self):
        # At interpreter exit the CUDA runtime may already be torn down;
        # the process is ending anyway, so leave the handle alone then.
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, allow=()):
        if st != 0 and st not in allow:
            raise TskError(st, self._lib.tsk_last_error(self._h).decode())
        return st

    def sync_status(self, stream=None) -> int:
        return self._lib.tsk_sync_status(self._h, _stream(stream))

    # ---- training side -------------------------------------------------
    def gram(self, As, mode: int = 1, out: Optional[torch.Tensor] = None,
             accumulate: bool = False, stream=None) -> torch.Tensor:
        """Mode-1 (sum A A^T) or mode-2 (sum A^T A) Gram matrix, float64.
        As: a (D, m, n) CUDA tensor (its matrices' addresses are computed,
        not looked up one by one) or a sequence of (m, n) CUDA tensors."""
        ptrs, D, m, n, ld, dtype, dev = _matrix_pointers(As)
        prec = _DTYPE_PREC[dtype]
        dim = m if mode == 1 else n
        if out is None:
            out = torch.zeros(dim, dim, dtype=torch.float64, device=dev)
        self._check(self._lib.tsk_gram(self._h, ptrs, D, m, n, ld, prec, mode, _ptr(out),
                                       int(accumulate), _stream(stream)))
        return out

    def quantize_e4m3(self, As, out=None, stream=None):
        """E4M3 copies of FP32 / BF16 training matrices with one power-of-two
        scale per row and group of eight matrices.  Returns (A8 uint8 of
        shape (D, m, ld8) with ld8 = n rounded up to 16, scales float32 of
        shape (ceil(D / 8), m)); `out` = such a pair from an earlier call
        with the same shapes is written in place."""
        src, D, m, n, lda, dtype, dev = _matrix_pointers(As)
        ld8 = (n + 15) // 16 * 16
        if out is None:
            A8 = torch.zeros(D, m, ld8, dtype=torch.uint8, device=dev)
            scales = torch.empty((D + 7) // 8, m, dtype=torch.float32, device=dev)
        else:
            A8, scales = out
            if tuple(A8.shape) != (D, m, ld8) or tuple(scales.shape) != ((D + 7) // 8, m):
                raise ValueError("out does not have the shapes of these matrices")
        if not A8.is_contiguous():
            raise ValueError("A8 must be contiguous")
        dst, _, _, _, _, _, _ = _matrix_pointers(A8)
        self._check(self._lib.tsk_quantize_e4m3(self._h, src, D, m, n, lda, _DTYPE_PREC[dtype],
                                                dst, ld8, _ptr(scales), _stream(stream)))
        return A8, scales

    def gram_e4m3(self, A8: torch.Tensor, scales: torch.Tensor, n: int,
                  out: Optional[torch.Tensor] = None, accumulate: bool = False, stream=None):
        """Mode-1 Gram of E4M3 matrices (from quantize_e4m3) on the tensor
        cores, scaled back to the stored values; float64 (m x m)."""
        _require_cuda(A8, scales)
        D, m, ld8 = A8.shape
        if out is None:
            out = torch.zeros(m, m, dtype=torch.float64, device=A8.device)
        ptrs, _, _, _, _, _, _ = _matrix_pointers(A8)
        self._check(self._lib.tsk_gram_e4m3(self._h, ptrs, _ptr(scales), D, m, n, ld8, _ptr(out),
                                            int(accumulate), _stream(stream)))
        return out

    def sketch_from_gram(self, G: torch.Tensor, k: int, prec: int = FP32,
                         stream=None):
        _require_cuda(G)
        dim = G.shape[0]
        S = torch.empty(k, dim, dtype=_PREC_COMPUTE[prec], device=G.device)
        eig = torch.empty(k, dtype=torch.float64, device=G.device)
        st = self._check(self._lib.tsk_sketch_from_gram(
            self._h, _ptr(G.contiguous()), dim, k, prec, _ptr(S), _ptr(eig),
            _stream(stream)), allow=(4,))
        return S, eig, st

    def train_sketch(self, As, k: int, l: int = 0, stream=None):
        """Algorithm 2 lines 1-2: S (k x m) and, with l > 0, W (l x n).

        As: a (D, m, n) CUDA tensor or a list of (m, n) CUDA tensors.
        Returns (S, W or None, eig (k + l,), status).
        """
        if isinstance(As, torch.Tensor):
            mats = [As[i] for i in range(As.shape[0])]
        else:
            mats = list(As)
        _require_cuda(*mats)
        m, n = mats[0].shape
        prec = _DTYPE_PREC[mats[0].dtype]
        dev = mats[0].device
        S = torch.empty(k, m, dtype=_PREC_COMPUTE[prec], device=dev)
        W = torch.empty(l, n, dtype=_PREC_COMPUTE[prec], device=dev) if l > 0 else None
        eig = torch.empty(k + l, dtype=torch.float64, device=dev)
        ptrs = (C.c_void_p * len(mats))(*[a.data_ptr() for a in mats])
        st = self._check(self._lib.tsk_train_sketch(
            self._h, ptrs, len(mats), m, n, mats[0].stride(0), prec, k, l,
            _ptr(S), _ptr(W), _ptr(eig), _stream(stream)), allow=(4,))
        return S, W, eig, st

    # ---- test side -----------------------------------------------------
    @staticmethod
    def _descs(As, Ss, ks, rs):
        n = len(As)
        descs = (MatDesc * n)()
        for i in range(n):
            A, S = As[i], Ss[i]
            descs[i] = MatDesc(A.data_ptr(), S.data_ptr(), A.shape[0], A.shape[1],
                               A.stride(0), int(ks[i]), int(rs[i]))
        return descs

    def approx_batch(self, As, Ss, r, outputs: bool = False, stream=None):
        """SCW (Algorithm 1, QR form) for every matrix of the batch.

        As: (count, m, n) tensor or list of (m, n) tensors (float64, float32
        or bfloat16, all the same type).  Ss: one (k, m) sketch for all, or a
        list (float64 for float64 A, float32 otherwise).  r: int or list.
        Returns dict(err, normA2[, US, Vt, sigma]).
        """
        As = [As[i] for i in range(As.shape[0])] if isinstance(As, torch.Tensor) else list(As)
        count = len(As)
        Ss = [Ss] * count if isinstance(Ss, torch.Tensor) else list(Ss)
        rs = [r] * count if isinstance(r, int) else list(r)
        ks = [S.shape[0] for S in Ss]
        _require_cuda(*As, *Ss)
        prec = _DTYPE_PREC[As[0].dtype]
        dev = As[0].device
        err = torch.empty(count, dtype=torch.float64, device=dev)
        normA2 = torch.empty(count, dtype=torch.float64, device=dev)
        res = {"err": err, "normA2": normA2}
        outs = None
        if outputs:
            cd = _PREC_COMPUTE[prec]
            US = [torch.empty(A.shape[0], rr, dtype=cd, device=dev) for A, rr in zip(As, rs)]
            Vt = [torch.empty(rr, A.shape[1], dtype=cd, device=dev) for A, rr in zip(As, rs)]
            sg = [torch.empty(k, dtype=cd, device=dev) for k in ks]
            outs = (MatOut * count)(*[MatOut(u.data_ptr(), v.data_ptr(), s.data_ptr())
                                      for u, v, s in zip(US, Vt, sg)])
            res.update(US=US, Vt=Vt, sigma=sg)
        descs = self._descs(As, Ss, ks, rs)
        self._check(self._lib.tsk_approx_batch(self._h, count, descs, prec, outs,
                                               _ptr(err), _ptr(normA2), _stream(stream)))
        res["_keep"] = (As, Ss, descs, outs)
        return res

    def plan(self, As, Ss, r, err: torch.Tensor, normA2: Optional[torch.Tensor] = None,
             outs=None) -> "Plan":
        As = [As[i] for i in range(As.shape[0])] if isinstance(As, torch.Tensor) else list(As)
        count = len(As)
        Ss = [Ss] * count if isinstance(Ss, torch.Tensor) else list(Ss)
        rs = [r] * count if isinstance(r, int) else list(r)
        ks = [S.shape[0] for S in Ss]
        _require_cuda(*As, *Ss, err)
        prec = _DTYPE_PREC[As[0].dtype]
        descs = self._descs(As, Ss, ks, rs)
        p = C.c_void_p()
        self._check(self._lib.tsk_plan_create(self._h, count, descs, prec, outs,
                                              _ptr(err), _ptr(normA2), C.byref(p)))
        return Plan(self, p, (As, Ss, descs, err, normA2))

    def error(self, As, Ss, r, US, Vt, stream=None) -> torch.Tensor:
        """Direct ||A - US Vt||_F per matrix (one more pass over A)."""
        As = [As[i] for i in range(As.shape[0])] if isinstance(As, torch.Tensor) else list(As)
        count = len(As)
        Ss = [Ss] * count if isinstance(Ss, torch.Tensor) else list(Ss)
        rs = [r] * count if isinstance(r, int) else list(r)
        ks = [S.shape[0] for S in Ss]
        prec = _DTYPE_PREC[As[0].dtype]
        err = torch.empty(count, dtype=torch.float64, device=As[0].device)
        outs = (MatOut * count)(*[MatOut(u.data_ptr(), v.data_ptr(), None)
                                  for u, v in zip(US, Vt)])
        descs = self._descs(As, Ss, ks, rs)
        self._check(self._lib.tsk_error(self._h, count, descs, prec, outs, _ptr(err),
                                        _stream(stream)))
        return err


    def autotune(self, As, Ss, r, reps: int = 5, stream=None):
        """Times the tensor-core sketch pass's two cluster shapes per size
        class of this batch and keeps the faster in the handle."""
        As = [As[i] for i in range(As.shape[0])] if isinstance(As, torch.Tensor) else list(As)
        count = len(As)
        Ss = [Ss] * count if isinstance(Ss, torch.Tensor) else list(Ss)
        rs = [r] * count if isinstance(r, int) else list(r)
        _require_cuda(*As, *Ss)
        descs = self._descs(As, Ss, [S.shape[0] for S in Ss], rs)
        self._check(self._lib.tsk_autotune(self._h, count, descs, _DTYPE_PREC[As[0].dtype],
                                           reps, _stream(stream)))

    def autotune_save(self, path: str):
        self._check(self._lib.tsk_autotune_save(self._h, os.fsencode(path)))

    def autotune_load(self, path: str):
        self._check(self._lib.tsk_autotune_load(self._h, os.fsencode(path)))

    # ---- two-sided sketching (Algorithms 3 and 5) -----------------------
    def train_two_sided(self, As, k: int, l: int, max_sweeps: int = 50, tol: float = 0.0,
                        stream=None):
        """Tucker2 sketches (S k x m, W l x n) of the training matrices by
        HOOI from the HOSVD start; returns (S, W, core_energy, sweeps, status)."""
        mats = [As[i] for i in range(As.shape[0])] if isinstance(As, torch.Tensor) else list(As)
        _require_cuda(*mats)
        m, n = mats[0].shape
        prec = _DTYPE_PREC[mats[0].dtype]
        dev = mats[0].device
        S = torch.empty(k, m, dtype=_PREC_COMPUTE[prec], device=dev)
        W = torch.empty(l, n, dtype=_PREC_COMPUTE[prec], device=dev)
        energy, sweeps = C.c_double(), C.c_int32()
        ptrs = (C.c_void_p * len(mats))(*[a.data_ptr() for a in mats])
        st = self._check(self._lib.tsk_train_two_sided(
            self._h, ptrs, len(mats), m, n, mats[0].stride(0), prec, k, l, max_sweeps, tol,
            _ptr(S), _ptr(W), C.byref(energy), C.byref(sweeps), _stream(stream)), allow=(4,))
        return S, W, energy.value, sweeps.value, st

    def approx_two_sided(self, As, Ss, Ws, r, outputs: bool = False, stream=None):
        """Two-sided SCW (Algorithm 3) for every matrix; returns
        dict(err, normA2[, US, Vt, sigma])."""
        As = [As[i] for i in range(As.shape[0])] if isinstance(As, torch.Tensor) else list(As)
        count = len(As)
        Ss = [Ss] * count if isinstance(Ss, torch.Tensor) else list(Ss)
        Ws = [Ws] * count if isinstance(Ws, torch.Tensor) else list(Ws)
        rs = [r] * count if isinstance(r, int) else list(r)
        _require_cuda(*As, *Ss, *Ws)
        prec = _DTYPE_PREC[As[0].dtype]
        dev = As[0].device
        err = torch.empty(count, dtype=torch.float64, device=dev)
        normA2 = torch.empty(count, dtype=torch.float64, device=dev)
        res = {"err": err, "normA2": normA2}
        outs = None
        if outputs:
            cd = _PREC_COMPUTE[prec]
            US = [torch.empty(A.shape[0], rr, dtype=cd, device=dev) for A, rr in zip(As, rs)]
            Vt = [torch.empty(rr, A.shape[1], dtype=cd, device=dev) for A, rr in zip(As, rs)]
            sg = [torch.empty(S.shape[0], dtype=cd, device=dev) for S in Ss]
            outs = (MatOut * count)(*[MatOut(u.data_ptr(), v.data_ptr(), g.data_ptr())
                                      for u, v, g in zip(US, Vt, sg)])
            res.update(US=US, Vt=Vt, sigma=sg)
        descs = (Mat2Desc * count)()
        for i in range(count):
            A, S, W = As[i], Ss[i], Ws[i]
            descs[i] = Mat2Desc(A.data_ptr(), S.data_ptr(), W.data_ptr(), A.shape[0],
                                A.shape[1], A.stride(0), S.shape[0], W.shape[0], int(rs[i]), 0)
        self._check(self._lib.tsk_approx_two_sided(self._h, count, descs, prec, outs,
                                                   _ptr(err), _ptr(normA2), _stream(stream)))
        return res

    # ---- learned refiner ------------------------------------------------
    def ivy_grad(self, As, S, r: int, stream=None):
        """IVY loss (Eq. 2.1, per-sample normalised) and dL/dS for a batch."""
        As = [As[i] for i in range(As.shape[0])] if isinstance(As, torch.Tensor) else list(As)
        _require_cuda(*As, S)
        prec = _DTYPE_PREC[As[0].dtype]
        descs = self._descs(As, [S] * len(As), [S.shape[0]] * len(As), [r] * len(As))
        grad = torch.empty_like(S)
        loss = torch.empty(1, dtype=torch.float64, device=S.device)
        self._check(self._lib.tsk_ivy_grad(self._h, len(As), descs, prec, _ptr(S),
                                           _ptr(grad), _ptr(loss), _stream(stream)))
        return grad, float(loss.item())

    def _refine_args(self, train, val, S_tensor, r, steps, batch, lr, eval_every, seed,
                     order):
        train = [train[i] for i in range(train.shape[0])] if isinstance(train, torch.Tensor) else list(train)
        val = [val[i] for i in range(val.shape[0])] if isinstance(val, torch.Tensor) else list(val)
        _require_cuda(*train, *val, S_tensor)
        prec = _DTYPE_PREC[train[0].dtype]
        k = S_tensor.shape[0]
        td = self._descs(train, [S_tensor] * len(train), [k] * len(train), [r] * len(train))
        vd = self._descs(val, [S_tensor] * len(val), [k] * len(val), [r] * len(val))
        o = _refine_opts(steps, batch, lr, eval_every, seed, order)
        return td, len(train), vd, len(val), prec, o

    def refine_sketch(self, train, val, S_tensor, r: int, steps: int = 2000,
                      batch: int = 16, lr: float = 1e-3, eval_every: int = 100,
                      seed: int = 20220929, order=None, dS=None, stream=None):
        """SGD on S_theta = S_tensor + dS; returns (dS, validation history)."""
        td, nt, vd, nv, prec, o = self._refine_args(train, val, S_tensor, r, steps, batch,
                                                    lr, eval_every, seed, order)
        dS = torch.zeros_like(S_tensor) if dS is None else dS
        hist = (C.c_double * (steps // eval_every + 1))()
        self._check(self._lib.tsk_refine_sketch(self._h, td, nt, vd, nv, prec, C.byref(o),
                                                _ptr(S_tensor), _ptr(dS), hist,
                                                _stream(stream)))
        return dS, list(hist)

    def refine_sketch_steps(self, train, val, S_tensor, r: int, dS, state: RefineState,
                            stop: int, steps: int = 2000, batch: int = 16, lr: float = 1e-3,
                            eval_every: int = 100, seed: int = 20220929, order=None,
                            history=None, stream=None):
        """Steps state.step .. stop - 1 of the SGD run that the options
        describe (the same batches whether or not the run was stopped before):
        dS, the current iterate, is updated in place and state advanced.
        history: the run's steps // eval_every + 1 validation losses, NaN
        where not yet computed; the entries this call computes are filled in
        and the list is returned."""
        td, nt, vd, nv, prec, o = self._refine_args(train, val, S_tensor, r, steps, batch,
                                                    lr, eval_every, seed, order)
        _require_cuda(dS, state.best)
        nh = steps // eval_every + 1
        hist = list(history) if history is not None else [float("nan")] * nh
        if len(hist) != nh:
            raise ValueError(f"history must have {nh} entries")
        ch = (C.c_double * nh)(*hist)
        sc = _RefineStateC(state.step, 0, state.best_loss, state.best.data_ptr())
        st = self._lib.tsk_refine_sketch_steps(self._h, td, nt, vd, nv, prec, C.byref(o),
                                               _ptr(S_tensor), _ptr(dS), C.byref(sc),
                                               int(stop), ch, _stream(stream))
        state.step, state.best_loss = int(sc.step), float(sc.best_loss)
        self._check(st)
        return list(ch)


class Plan:
    """A built test-side plan (workspace + schedule + CUDA graph)."""

    def __init__(self, handle: Handle, p, keep):
        self._h, self._p, self._keep = handle, p, keep

    def execute(self, stream=None):
        self._h._check(self._h._lib.tsk_plan_execute(self._p, _stream(stream)))

    def set_probe(self, ev_begin, ev_end):
        """Record ev_begin/ev_end (torch.cuda.Event with timing) around the
        sketch pass on every later execute(); (None, None) removes the probe.
        The plan keeps the events alive while its graph refers to them."""
        if ev_begin is None and ev_end is None:
            self._h._check(self._h._lib.tsk_plan_set_probe(self._p, None, None))
            self._probe = None
            return
        self._h._check(self._h._lib.tsk_plan_set_probe(
            self._p, C.c_void_p(ev_begin.cuda_event), C.c_void_p(ev_end.cuda_event)))
        self._probe = (ev_begin, ev_end)

    def info(self):
        ws, nl = C.c_int64(), C.c_int32()
        self._h._check(self._h._lib.tsk_plan_info(self._p, C.byref(ws), C.byref(nl)))
        return {"workspace_bytes": ws.value, "launches": nl.value}

    def close(self):
        if self._p:
            self._h._lib.tsk_plan_destroy(self._p)
            self._p = None

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


def _matrix_pointers(As):
    """(ctypes array of device pointers, D, m, n, row stride, dtype, device)
    for a (D, m, n) CUDA tensor with unit column stride (addresses computed
    from its strides) or a sequence of equally shaped (m, n) CUDA tensors."""
    if isinstance(As, torch.Tensor):
        if As.dim() != 3:
            raise ValueError("expected a (D, m, n) tensor or a sequence of (m, n) tensors")
        _require_cuda(As)
        D, m, n = As.shape
        if As.stride(2) != 1:
            raise ValueError("the matrices' rows must be contiguous")
        step = As.stride(0) * As.element_size()
        base = As.data_ptr()
        ptrs = (C.c_void_p * D)(*range(base, base + D * step, step)) if step else \
            (C.c_void_p * D)(*([base] * D))
        return ptrs, D, m, n, As.stride(1), As.dtype, As.device
    mats = list(As)
    if not mats:
        raise ValueError("no matrices")
    _require_cuda(*mats)
    m, n = mats[0].shape
    ptrs = (C.c_void_p * len(mats))(*[a.data_ptr() for a in mats])
    return ptrs, len(mats), m, n, mats[0].stride(0), mats[0].dtype, mats[0].device


def _refine_opts(steps, batch, lr, eval_every, seed, order):
    o = RefineOpts()
    load_library().tsk_default_refine_options(C.byref(o))
    o.steps, o.batch, o.lr, o.eval_every, o.seed = steps, batch, lr, eval_every, seed
    if order is not None:
        o._keep = (C.c_int32 * max(1, len(order)))(*[int(x) for x in order])
        o.order = C.cast(o._keep, C.POINTER(C.c_int32))
    return o


def _check_host(st: int):
    if st != 0:
        raise TskError(st, load_library().tsk_last_error(None).decode())


def save_array(path: str, t: torch.Tensor) -> None:
    """Writes a 2-D tensor (S, W, a refiner's dS; float64, float32 or
    bfloat16) to a tsk array file (tsk_array_save: little-endian, with a
    header giving the precision and shape)."""
    if t.dim() != 2 or t.dtype not in _DTYPE_PREC:
        raise ValueError("save_array takes a 2-D float64, float32 or bfloat16 tensor")
    h = t.detach().to("cpu").contiguous()
    _check_host(load_library().tsk_array_save(os.fsencode(path), C.c_void_p(h.data_ptr()),
                                              _DTYPE_PREC[h.dtype], h.shape[0], h.shape[1]))


def load_array(path: str, device="cpu") -> torch.Tensor:
    """Reads a tsk array file into a tensor on `device`."""
    lib = load_library()
    p, rows, cols = C.c_int32(), C.c_int64(), C.c_int64()
    _check_host(lib.tsk_array_load(os.fsencode(path), None, 0, C.byref(p), C.byref(rows),
                                   C.byref(cols)))
    dtype = {v: k for k, v in _DTYPE_PREC.items()}[p.value]
    h = torch.empty((rows.value, cols.value), dtype=dtype)
    _check_host(lib.tsk_array_load(os.fsencode(path), C.c_void_p(h.data_ptr()),
                                   h.numel() * h.element_size(), C.byref(p), C.byref(rows),
                                   C.byref(cols)))
    return h.to(device)


def save_refine_checkpoint(path: str, dS: torch.Tensor, state: RefineState, steps: int,
                           batch: int = 16, lr: float = 1e-3, eval_every: int = 100,
                           seed: int = 20220929, order=None) -> None:
    """Writes a resumable refiner run (tsk_refine_save): the run's options,
    the steps taken, the current dS, the best validated dS and its loss."""
    if dS.dtype not in (torch.float64, torch.float32) or dS.dim() != 2:
        raise ValueError("dS must be a 2-D float64 or float32 tensor")
    o = _refine_opts(steps, batch, lr, eval_every, seed, order)
    d = dS.detach().to("cpu").contiguous()
    b = state.best.detach().to("cpu", dS.dtype).contiguous()
    sc = _RefineStateC(state.step, 0, state.best_loss, None)
    _check_host(load_library().tsk_refine_save(
        os.fsencode(path), _DTYPE_PREC[d.dtype], d.shape[0], d.shape[1], C.byref(o),
        C.byref(sc), C.c_void_p(d.data_ptr()), C.c_void_p(b.data_ptr())))


def load_refine_checkpoint(path: str, device="cuda") -> dict:
    """Reads a refiner checkpoint: {"dS", "state" (a RefineState whose best
    is on `device`), "steps", "batch", "lr", "eval_every", "seed",
    "order_given"}; a run with order_given must be passed its order again."""
    lib = load_library()
    p, k, m, og = C.c_int32(), C.c_int64(), C.c_int64(), C.c_int32()
    o, sc = RefineOpts(), _RefineStateC()
    _check_host(lib.tsk_refine_load(os.fsencode(path), C.byref(p), C.byref(k), C.byref(m),
                                    C.byref(o), C.byref(og), C.byref(sc), None, None, 0))
    dtype = torch.float64 if p.value == FP64 else torch.float32
    d = torch.empty((k.value, m.value), dtype=dtype)
    b = torch.empty_like(d)
    _check_host(lib.tsk_refine_load(os.fsencode(path), C.byref(p), C.byref(k), C.byref(m),
                                    C.byref(o), C.byref(og), C.byref(sc),
                                    C.c_void_p(d.data_ptr()), C.c_void_p(b.data_ptr()),
                                    d.numel() * d.element_size()))
    return {"dS": d.to(device), "state": RefineState(b.to(device), sc.step, sc.best_loss),
            "steps": int(o.steps), "batch": int(o.batch), "lr": float(o.lr),
            "eval_every": int(o.eval_every), "seed": int(o.seed),
            "order_given": bool(og.value)}


def header_functions(path: Optional[str] = None) -> List[str]:
    """Names of the functions include/tsk.h declares."""
    import re
    path = path or os.path.join(os.path.dirname(_PKG), "include", "tsk.h")
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tsk_[a-z0-9_]+)\s*\(", text)))
