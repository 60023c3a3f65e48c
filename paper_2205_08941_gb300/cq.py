"""Thin ctypes binding of libcq.so: the C-ABI calls under the same names, plus small
wrappers that marshal torch CUDA tensors (device memory, streams) into them.

No arithmetic of the method happens here: every step runs in the library's CUDA kernels.
If libcq.so is missing the import fails loudly; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import weakref

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcq.so")

CQ_OK = 0
CQ_FP64 = 0
CQ_SPLIT_BF16X3 = 1
CQ_FP64_EMU = 2
STATUS = {0: "CQ_OK", 1: "CQ_ERR_INVALID", 2: "CQ_ERR_PATTERN", 3: "CQ_ERR_NOMEM",
          4: "CQ_ERR_CUDA", 5: "CQ_ERR_NUMERIC", 6: "CQ_ERR_TIMEOUT", 7: "CQ_ERR_NOT_CONVERGED"}


class CQError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class LnvReport(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("n_elec", ctypes.c_double),
                ("mu", ctypes.c_double), ("gnorm", ctypes.c_double),
                ("alpha", ctypes.c_double), ("restart", ctypes.c_int32),
                ("fallback", ctypes.c_int32), ("n_corr", ctypes.c_int32),
                ("n_products", ctypes.c_int32), ("flops", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_vp = ctypes.c_void_p
_d = ctypes.c_double
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_st = ctypes.c_int

# name -> (restype, argtypes): one line per entry point declared in include/cq.h
SIGNATURES = {
    "cq_ctx_create": (_st, [ctypes.c_int, _vp, ctypes.POINTER(_vp)]),
    "cq_ctx_destroy": (None, [_vp]),
    "cq_last_error": (ctypes.c_char_p, [_vp]),
    "cq_ctx_sync": (_st, [_vp]),
    "cq_ctx_set_mem_limit": (_st, [_vp, _i64]),
    "cq_ctx_mem_used": (_i64, [_vp]),
    "cq_pattern_build": (_st, [_vp, _i32, _vp, ctypes.POINTER(_d), _vp, _d,
                               ctypes.POINTER(_vp)]),
    "cq_pattern_info": (_st, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "cq_pattern_export": (_st, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "cq_pattern_destroy": (None, [_vp]),
    "cq_pattern_scatter": (_st, [_vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp]),
    "cq_bsmm": (_st, [_vp, _d, _vp, _vp, _vp, _vp, _d, _vp, _vp, ctypes.c_int]),
    "cq_bsmm_work": (_st, [_vp, _vp, _vp, _vp, ctypes.POINTER(_i64), ctypes.POINTER(_d)]),
    "cq_trace_prod": (_st, [_vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_d)]),
    "cq_dot": (_st, [_vp, _vp, _vp, _vp, ctypes.POINTER(_d)]),
    "cq_hotelling_init": (_st, [_vp, _vp, _vp, _vp, _vp]),
    "cq_hotelling_step": (_st, [_vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_d)]),
    "cq_overlap_inverse_cg": (_st, [_vp, _vp, _vp, _vp, _vp, _i32, _d, _vp, _vp,
                                    ctypes.POINTER(_i32)]),
    "cq_pm_guess": (_st, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _d]),
    "cq_mcweeny_step": (_st, [_vp, _vp, _vp, _vp, _vp]),
    "cq_lnv_create": (_st, [_vp, _vp, _vp, _vp, _vp, _vp, _d, ctypes.c_int,
                            ctypes.POINTER(_vp)]),
    "cq_lnv_step": (_st, [_vp, _vp]),
    "cq_lnv_set_precision": (_st, [_vp, ctypes.c_int]),
    "cq_lnv_set_preconditioner": (_st, [_vp, _vp, _vp]),
    "cq_lnv_state": (_st, [_vp, _vp]),
    "cq_lnv_step_flops": (_st, [_vp, ctypes.POINTER(_d)]),
    "cq_lnv_destroy": (None, [_vp]),
    "cq_kernel_launches": (_i64, []),
    "cq_ctx_set_timing": (_st, [_vp, ctypes.c_int]),
    "cq_ctx_kernel_stats": (_st, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_d),
                                  ctypes.POINTER(_d), ctypes.POINTER(_d)]),
    "cq_peak_fp64": (_st, [_vp, ctypes.POINTER(_d)]),
    "cq_pattern_build_batch": (_st, [_vp, _i32, _vp, _vp, _vp, _vp, _vp,
                                     ctypes.POINTER(_vp)]),
    "cq_pattern_cells": (_i32, [_vp]),
    "cq_pm_guess_cells": (_st, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "cq_lnv_create_cells": (_st, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int,
                                  ctypes.POINTER(_vp)]),
    "cq_lnv_cells": (_i32, [_vp]),
    "cq_ctx_set_autotune": (_st, [_vp, ctypes.c_int]),
    "cq_ctx_set_graphs": (_st, [_vp, ctypes.c_int]),
    "cq_bsmm_config": (_st, [_vp, _vp, _vp, _vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "cq_guess_create": (_st, [_vp, ctypes.c_uint64, _i32, ctypes.POINTER(_vp)]),
    "cq_guess_destroy": (None, [_vp]),
    "cq_guess_pairs": (_st, [_vp, _vp, ctypes.POINTER(_i64)]),
    "cq_guess_descriptors": (_st, [_vp, _vp, _vp, _vp, _vp]),
    "cq_guess_targets": (_st, [_vp, _vp, _vp, _vp, _vp]),
    "cq_guess_fit_scale": (_st, [_vp, _vp, _vp, _i64]),
    "cq_guess_set_scale": (_st, [_vp, _vp, _vp, _vp, _vp]),
    "cq_guess_params": (_st, [_vp, _vp, _vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), _i32]),
    "cq_guess_train_step": (_st, [_vp, _vp, _vp, _i64, ctypes.c_float,
                                  ctypes.POINTER(ctypes.c_float), _vp, _vp]),
    "cq_guess_loss_sum": (_st, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                ctypes.c_int32]),
    "cq_guess_forward": (_st, [_vp, _vp, _i64, _vp]),
    "cq_guess_apply": (_st, [_vp, _vp, _vp]),
    "cq_ctx_set_test_wait": (_st, [_vp, _i64]),
    "cq_ctx_release_cache": (_st, [_vp]),
    "cq_trace_prod_static": (_st, [_vp, _vp, _vp, _vp, _vp, _vp,
                                   ctypes.POINTER(ctypes.c_char_p)]),
}


def trace_prod_static(pA, A, pB, B, out, stream=None):
    """cq_trace_prod_static: Tr(A.B) into the device tensor `out` (one float64) without any
    device allocation; asynchronous on `stream` (a torch.cuda.Stream, default: current)."""
    st = stream or torch.cuda.current_stream()
    msg = ctypes.c_char_p()
    status = lib().cq_trace_prod_static(pA.h, _ptr(A), pB.h, _ptr(B), _ptr(out),
                                        ctypes.c_void_p(st.cuda_stream), ctypes.byref(msg))
    if status != CQ_OK:
        raise CQError(status, msg.value.decode() if msg.value else "")
    return out


def _host_f64(values):
    arr = (ctypes.c_double * len(values))(*[float(v) for v in values])
    return arr


def _host_i32(values):
    return (ctypes.c_int32 * len(values))(*[int(v) for v in values])

_lib = None


def lib():
    """Load libcq.so (raises if it was not built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} missing: run python -m paper_2205_08941_gb300.build")
        h = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(h, name)
            fn.restype = res
            fn.argtypes = args
        _lib = h
    return _lib


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """A libcq context bound to a device and a torch CUDA stream."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        self.device = device
        self.stream = stream or torch.cuda.current_stream(device)
        h = ctypes.c_void_p()
        self._check(lib().cq_ctx_create(device, ctypes.c_void_p(self.stream.cuda_stream),
                                        ctypes.byref(h)), ctx=None)
        self.h = h

    def _check(self, st, ctx="self"):
        if st != CQ_OK:
            msg = lib().cq_last_error(self.h if ctx == "self" else None)
            raise CQError(st, msg.decode() if msg else "")

    def close(self):
        """Destroy the context; LNV objects and patterns made from it are closed first."""
        if getattr(self, "h", None):
            kids = list(self._children)
            for child in [k for k in kids if isinstance(k, Lnv)] + \
                    [k for k in kids if not isinstance(k, Lnv)]:
                child.close()
            lib().cq_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def _children(self):
        if "_kids" not in self.__dict__:
            self.__dict__["_kids"] = weakref.WeakSet()
        return self.__dict__["_kids"]

    def sync(self):
        self._check(lib().cq_ctx_sync(self.h))

    def set_mem_limit(self, nbytes: int):
        self._check(lib().cq_ctx_set_mem_limit(self.h, int(nbytes)))

    def mem_used(self) -> int:
        return int(lib().cq_ctx_mem_used(self.h))

    def set_timing(self, on: bool):
        self._check(lib().cq_ctx_set_timing(self.h, 1 if on else 0))

    def set_autotune(self, on: bool):
        self._check(lib().cq_ctx_set_autotune(self.h, 1 if on else 0))

    def release_cache(self):
        """Free cached task lists, maps, tile plans and scratch (rebuilt on demand)."""
        self._check(lib().cq_ctx_release_cache(self.h))

    def set_test_wait(self, cycles: int):
        """Test hook: split kernels make their first wait run out after `cycles` (0: off)."""
        self._check(lib().cq_ctx_set_test_wait(self.h, int(cycles)))

    def set_graphs(self, on: bool):
        self._check(lib().cq_ctx_set_graphs(self.h, 1 if on else 0))

    def bsmm_config(self, pA, pB, pC):
        q, tuned = ctypes.c_int32(), ctypes.c_int32()
        self._check(lib().cq_bsmm_config(self.h, pA.h, pB.h, pC.h, ctypes.byref(q),
                                         ctypes.byref(tuned)))
        return int(q.value), bool(tuned.value)

    def kernel_stats(self):
        n, ms, fl, mf = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(lib().cq_ctx_kernel_stats(self.h, ctypes.byref(n), ctypes.byref(ms),
                                              ctypes.byref(fl), ctypes.byref(mf)))
        return int(n.value), float(ms.value), float(fl.value), float(mf.value)

    def peak_fp64(self) -> float:
        out = ctypes.c_double()
        self._check(lib().cq_peak_fp64(self.h, ctypes.byref(out)))
        return float(out.value)

    # ------------------------------------------------------------ patterns
    def pattern(self, pos: torch.Tensor, box, nb: torch.Tensor, rng: float) -> "Pattern":
        return Pattern(self, pos, box, nb, rng)

    def zeros(self, p: "Pattern") -> torch.Tensor:
        return torch.zeros(p.n_values, dtype=torch.float64, device=f"cuda:{self.device}")

    def empty(self, p: "Pattern") -> torch.Tensor:
        return torch.empty(p.n_values, dtype=torch.float64, device=f"cuda:{self.device}")

    def scatter(self, p: "Pattern", i, j, off, values, out=None) -> torch.Tensor:
        out = self.empty(p) if out is None else out
        self._check(lib().cq_pattern_scatter(self.h, p.h, int(i.shape[0]), _ptr(i), _ptr(j),
                                             _ptr(off), _ptr(values), _ptr(out)))
        return out

    # ------------------------------------------------------------ products and traces
    def bsmm(self, alpha, pA, A, pB, B, beta, pC, C, prec=CQ_FP64):
        self._check(lib().cq_bsmm(self.h, float(alpha), pA.h, _ptr(A), pB.h, _ptr(B),
                                  float(beta), pC.h, _ptr(C), int(prec)))
        return C

    def bsmm_work(self, pA, pB, pC):
        t, f = ctypes.c_int64(), ctypes.c_double()
        self._check(lib().cq_bsmm_work(self.h, pA.h, pB.h, pC.h, ctypes.byref(t),
                                       ctypes.byref(f)))
        return int(t.value), float(f.value)

    def trace_prod(self, pA, A, pB, B) -> float:
        out = ctypes.c_double()
        self._check(lib().cq_trace_prod(self.h, pA.h, _ptr(A), pB.h, _ptr(B),
                                        ctypes.byref(out)))
        return float(out.value)

    def dot(self, p, A, B) -> float:
        out = ctypes.c_double()
        self._check(lib().cq_dot(self.h, p.h, _ptr(A), _ptr(B), ctypes.byref(out)))
        return float(out.value)

    # ------------------------------------------------------------ drivers
    def hotelling_init(self, pS, S, pT, T):
        self._check(lib().cq_hotelling_init(self.h, pS.h, _ptr(S), pT.h, _ptr(T)))
        return T

    def hotelling_step(self, pS, S, pT, T) -> float:
        r = ctypes.c_double()
        self._check(lib().cq_hotelling_step(self.h, pS.h, _ptr(S), pT.h, _ptr(T),
                                            ctypes.byref(r)))
        return float(r.value)

    def overlap_inverse_cg(self, pS, S, pT, T, max_iter: int, gtol: float = 0.0):
        """Least-squares inverse on P_T by CG from T (updated in place).  Returns
        (resid, gnorm): ||I - S T_k||_F and ||G_k||_F for the start and every iterate."""
        r = (_d * (max_iter + 1))()
        g = (_d * (max_iter + 1))()
        k = ctypes.c_int32()
        self._check(lib().cq_overlap_inverse_cg(self.h, pS.h, _ptr(S), pT.h, _ptr(T),
                                                int(max_iter), float(gtol), r, g,
                                                ctypes.byref(k)))
        n = int(k.value) + 1
        return list(r[:n]), list(g[:n])

    def pm_guess(self, pS, S, H, pT, T, pL, L, n_occ: float):
        self._check(lib().cq_pm_guess(self.h, pS.h, _ptr(S), _ptr(H), pT.h, _ptr(T), pL.h,
                                      _ptr(L), float(n_occ)))
        return L

    def mcweeny_step(self, pS, S, pL, L):
        self._check(lib().cq_mcweeny_step(self.h, pS.h, _ptr(S), pL.h, _ptr(L)))
        return L

    def lnv(self, pS, S, H, pL, L, n_electrons, prec=CQ_FP64) -> "Lnv":
        return Lnv(self, pS, S, H, pL, L, n_electrons, prec)

    # ------------------------------------------------------------ batches
    def pattern_batch(self, pos, cell_start, boxes, nb, ranges) -> "Pattern":
        """Pattern over several cells (atoms of cell c: cell_start[c]..cell_start[c+1]-1)."""
        return Pattern(self, pos, None, nb, None, batch=(cell_start, boxes, ranges))

    def pm_guess_cells(self, pS, S, H, pT, T, pL, L, n_occ):
        self._check(lib().cq_pm_guess_cells(self.h, pS.h, _ptr(S), _ptr(H), pT.h, _ptr(T),
                                            pL.h, _ptr(L), _host_f64(n_occ)))
        return L

    def lnv_cells(self, pS, S, H, pL, L, n_electrons, prec=CQ_FP64) -> "Lnv":
        return Lnv(self, pS, S, H, pL, L, list(n_electrons), prec)


class Pattern:
    """Range-cutoff pattern built on the device by cq_pattern_build."""

    def __init__(self, ctx: Context, pos: torch.Tensor, box, nb: torch.Tensor, rng,
                 batch=None):
        self.ctx = ctx
        self._pos, self._nb = pos, nb
        h = ctypes.c_void_p()
        if batch is None:
            box_arr = (ctypes.c_double * 3)(*[float(b) for b in box])
            ctx._check(lib().cq_pattern_build(ctx.h, int(pos.shape[0]), _ptr(pos), box_arr,
                                              _ptr(nb), float(rng), ctypes.byref(h)))
            self.range = float(rng)
        else:
            cell_start, boxes, ranges = batch
            n_cells = len(ranges)
            flat_boxes = [float(x) for b in boxes for x in b]
            ctx._check(lib().cq_pattern_build_batch(
                ctx.h, n_cells, _host_i32(cell_start), _ptr(pos), _host_f64(flat_boxes),
                _ptr(nb), _host_f64(ranges), ctypes.byref(h)))
            self.range = [float(r) for r in ranges]
        self.h = h
        ctx._children.add(self)
        self.n_cells = int(lib().cq_pattern_cells(h))
        nbk, nv = ctypes.c_int64(), ctypes.c_int64()
        lib().cq_pattern_info(h, ctypes.byref(nbk), ctypes.byref(nv))
        self.n_blocks, self.n_values = int(nbk.value), int(nv.value)
        self.n_atoms = int(pos.shape[0])

    def export(self):
        """(row_ptr, col, val_off, transpose) as CUDA tensors."""
        dev = self._pos.device
        rp = torch.empty(self.n_atoms + 1, dtype=torch.int64, device=dev)
        col = torch.empty(max(self.n_blocks, 1), dtype=torch.int32, device=dev)
        off = torch.empty(max(self.n_blocks, 1), dtype=torch.int64, device=dev)
        tr = torch.empty(max(self.n_blocks, 1), dtype=torch.int64, device=dev)
        self.ctx._check(lib().cq_pattern_export(self.ctx.h, self.h, _ptr(rp), _ptr(col),
                                                _ptr(off), _ptr(tr)))
        self.ctx.sync()
        n = self.n_blocks
        return rp, col[:n], off[:n], tr[:n]

    def close(self):
        if getattr(self, "h", None):
            lib().cq_pattern_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Lnv:
    """LNV minimisation state (cq_lnv_create(_cells) / cq_lnv_step).

    For a single cell, step() and state() return one dict; for a batch (n_electrons given
    as a list) they return one dict per cell."""

    def __init__(self, ctx, pS, S, H, pL, L, n_electrons, prec=CQ_FP64):
        self.ctx = ctx
        self._keep = (pS, S, H, pL, L)
        h = ctypes.c_void_p()
        self.batch = isinstance(n_electrons, (list, tuple))
        if self.batch:
            ctx._check(lib().cq_lnv_create_cells(ctx.h, pS.h, _ptr(S), _ptr(H), pL.h, _ptr(L),
                                                 _host_f64(n_electrons), int(prec),
                                                 ctypes.byref(h)))
        else:
            ctx._check(lib().cq_lnv_create(ctx.h, pS.h, _ptr(S), _ptr(H), pL.h, _ptr(L),
                                           float(n_electrons), int(prec), ctypes.byref(h)))
        self.h = h
        ctx._children.add(self)
        self.n_cells = int(lib().cq_lnv_cells(h))

    def _reports(self, fn):
        reps = (LnvReport * self.n_cells)()
        self.ctx._check(fn(self.h, reps))
        out = [r.as_dict() for r in reps]
        return out if self.batch else out[0]

    def step(self):
        return self._reports(lib().cq_lnv_step)

    def set_precision(self, prec: int):
        self.ctx._check(lib().cq_lnv_set_precision(self.h, int(prec)))

    def set_preconditioner(self, pT=None, T=None):
        """Precondition later search directions with T (an approximate S^-1 on pT, e.g. from
        hotelling()); None switches back to the plain gradient.  T is copied; pT must stay
        alive while the preconditioner is set."""
        self._keep_T = pT
        self.ctx._check(lib().cq_lnv_set_preconditioner(
            self.h, pT.h if pT is not None else None, _ptr(T) if T is not None else None))

    def state(self):
        return self._reports(lib().cq_lnv_state)

    def step_flops(self) -> float:
        f = ctypes.c_double()
        self.ctx._check(lib().cq_lnv_step_flops(self.h, ctypes.byref(f)))
        return float(f.value)

    def close(self):
        if getattr(self, "h", None):
            lib().cq_lnv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Guess:
    """Learned initial guess (cq_guess_*): descriptors, targets, training, apply."""

    N_IN, N_OUT = 64, 81

    def __init__(self, ctx: Context, seed: int = 0, fp32_weights: bool = False):
        self.ctx = ctx
        h = ctypes.c_void_p()
        ctx._check(lib().cq_guess_create(ctx.h, int(seed), 1 if fp32_weights else 0,
                                         ctypes.byref(h)))
        self.h = h
        ctx._children.add(self)

    def pairs(self, pL) -> int:
        n = ctypes.c_int64()
        self.ctx._check(lib().cq_guess_pairs(self.ctx.h, pL.h, ctypes.byref(n)))
        return int(n.value)

    def descriptors(self, pL):
        n = self.pairs(pL)
        dev = f"cuda:{self.ctx.device}"
        desc = torch.empty((max(n, 1), self.N_IN), dtype=torch.float32, device=dev)
        frames = torch.empty((max(n, 1), 9), dtype=torch.float32, device=dev)
        pairs = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        self.ctx._check(lib().cq_guess_descriptors(self.ctx.h, pL.h, _ptr(desc), _ptr(frames),
                                                   _ptr(pairs)))
        self.ctx.sync()
        return desc[:n], frames[:n], pairs[:n]

    def targets(self, pL, L, frames):
        t = torch.empty((max(frames.shape[0], 1), self.N_OUT), dtype=torch.float32,
                        device=frames.device)
        self.ctx._check(lib().cq_guess_targets(self.ctx.h, pL.h, _ptr(L), _ptr(frames), _ptr(t)))
        self.ctx.sync()
        return t[:frames.shape[0]]

    def fit_scale(self, desc, targets):
        self.ctx._check(lib().cq_guess_fit_scale(self.h, _ptr(desc), _ptr(targets),
                                                 int(desc.shape[0])))

    def set_scale(self, in_mean, in_scale, out_mean, out_scale):
        f = lambda a: (ctypes.c_float * len(a))(*[float(x) for x in a])
        self.ctx._check(lib().cq_guess_set_scale(self.h, f(in_mean), f(in_scale), f(out_mean),
                                                 f(out_scale)))

    def params(self):
        nw, nb = ctypes.c_int64(), ctypes.c_int64()
        self.ctx._check(lib().cq_guess_params(self.h, None, None, ctypes.byref(nw),
                                              ctypes.byref(nb), 0))
        import numpy as np
        w = np.zeros(nw.value, dtype=np.float32)
        b = np.zeros(nb.value, dtype=np.float32)
        self.ctx._check(lib().cq_guess_params(self.h, w.ctypes.data, b.ctypes.data, None, None, 0))
        return w, b

    def set_params(self, w, b):
        import numpy as np
        w = np.ascontiguousarray(w, dtype=np.float32)
        b = np.ascontiguousarray(b, dtype=np.float32)
        self.ctx._check(lib().cq_guess_params(self.h, w.ctypes.data, b.ctypes.data, None, None, 1))

    def train_step(self, desc, targets, lr, grads=False, loss=True):
        """One Adam step; returns the batch loss (and the gradients with grads=True).  With
        loss=False and grads=False nothing is read back and the step stays asynchronous."""
        import numpy as np
        lv = ctypes.c_float()
        gw = gb = None
        if grads:
            w, b = self.params()
            gw, gb = np.zeros_like(w), np.zeros_like(b)
        self.ctx._check(lib().cq_guess_train_step(
            self.h, _ptr(desc), _ptr(targets), int(desc.shape[0]), float(lr),
            ctypes.byref(lv) if (loss or grads) else None,
            None if gw is None else gw.ctypes.data, None if gb is None else gb.ctypes.data))
        if grads:
            return float(lv.value), gw, gb
        return float(lv.value) if loss else None

    def loss_sum(self, reset=True):
        """(squared-error sum, rows) of the training steps since the last reset."""
        sq = ctypes.c_double()
        rows = ctypes.c_int64()
        self.ctx._check(lib().cq_guess_loss_sum(self.h, ctypes.byref(sq), ctypes.byref(rows),
                                                1 if reset else 0))
        return float(sq.value), int(rows.value)

    def forward(self, desc):
        out = torch.empty((max(desc.shape[0], 1), self.N_OUT), dtype=torch.float32,
                          device=desc.device)
        self.ctx._check(lib().cq_guess_forward(self.h, _ptr(desc), int(desc.shape[0]), _ptr(out)))
        self.ctx.sync()
        return out[:desc.shape[0]]

    def apply(self, pL, L):
        self.ctx._check(lib().cq_guess_apply(self.h, pL.h, _ptr(L)))
        return L

    def close(self):
        if getattr(self, "h", None):
            lib().cq_guess_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kernel_launches() -> int:
    return int(lib().cq_kernel_launches())
