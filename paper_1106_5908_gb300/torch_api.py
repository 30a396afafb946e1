"""Torch-facing wrappers over the C ABI (argument marshalling only).

PyTorch supplies device memory, streams and autograd; every operation runs in
``libspmv.so`` through ``_abi``.  There is no CPU path: without the built
library every call raises.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np
import torch

from . import _abi as abi

_DT = {torch.float64: abi.SPMV_F64, torch.float32: abi.SPMV_F32}


def _stream(stream: Optional[torch.cuda.Stream] = None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t: Optional[torch.Tensor]) -> Optional[ctypes.c_void_p]:
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a: np.ndarray) -> ctypes.c_void_p:
    return a.ctypes.data_as(ctypes.c_void_p)


class Matrix:
    """A CRS matrix held by the library (``spmv_handle``)."""

    def __init__(self, handle: ctypes.c_void_p, n_rows: int, n_cols: int, nnz: int,
                 dtype: torch.dtype, device: torch.device):
        self._h = handle
        self.n_rows, self.n_cols, self.nnz = n_rows, n_cols, nnz
        self.dtype = dtype
        self.device = device

    @classmethod
    def from_csr(cls, row_ptr, col_idx, val, n_cols: int, dtype: Optional[torch.dtype] = None,
                 device="cuda") -> "Matrix":
        """Create from CRS arrays (numpy arrays on the host, or CUDA tensors).
        ``dtype`` selects the stored value type (default: that of ``val``)."""
        device = torch.device(device)
        if isinstance(row_ptr, torch.Tensor) and row_ptr.is_cuda:
            rp = row_ptr.to(torch.int32).contiguous()
            ci = col_idx.to(torch.int32).contiguous()
            v = val.contiguous()
            vt = _DT[v.dtype]
            n_rows, nnz = rp.numel() - 1, ci.numel()
            ptrs = (_dptr(rp), _dptr(ci) if nnz else None, _dptr(v) if nnz else None)
            is_dev = 1
            keep = (rp, ci, v)
        else:
            rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
            ci = np.ascontiguousarray(col_idx, dtype=np.int32)
            v = np.ascontiguousarray(val)
            if v.dtype not in (np.float64, np.float32):
                v = v.astype(np.float64)
            vt = abi.SPMV_F64 if v.dtype == np.float64 else abi.SPMV_F32
            n_rows, nnz = rp.size - 1, ci.size
            ptrs = (_hptr(rp), _hptr(ci) if nnz else None, _hptr(v) if nnz else None)
            is_dev = 0
            keep = (rp, ci, v)
        store = vt if dtype is None else _DT[dtype]
        if store != vt:
            # store the requested value type: convert the values before the copy
            if is_dev:
                v = v.to(torch.float64 if store == abi.SPMV_F64 else torch.float32)
                ptrs = (ptrs[0], ptrs[1], _dptr(v) if nnz else None)
            else:
                v = v.astype(np.float64 if store == abi.SPMV_F64 else np.float32)
                ptrs = (ptrs[0], ptrs[1], _hptr(v) if nnz else None)
            keep = (rp, ci, v)
        h = ctypes.c_void_p()
        with torch.cuda.device(device):
            abi.check(abi.spmv_create(ctypes.byref(h), n_rows, n_cols, nnz, ptrs[0], ptrs[1],
                                      ptrs[2], store, is_dev, _stream()), "spmv_create")
        del keep
        return cls(h, n_rows, n_cols, nnz,
                   torch.float64 if store == abi.SPMV_F64 else torch.float32, device)

    @classmethod
    def from_symmetric_upper(cls, row_ptr, col_idx, val, dtype: Optional[torch.dtype] = None,
                             device="cuda") -> "Matrix":
        """Symmetric CRS: a symmetric n x n matrix from its upper triangle with
        the diagonal (host numpy arrays; every column >= its row).  apply()
        computes y = alpha*A*x + beta*y with each off-diagonal value stored once."""
        device = torch.device(device)
        rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
        ci = np.ascontiguousarray(col_idx, dtype=np.int32)
        v = np.ascontiguousarray(val)
        if v.dtype not in (np.float64, np.float32):
            v = v.astype(np.float64)
        if dtype is not None:
            v = v.astype(np.float64 if dtype == torch.float64 else np.float32)
        vt = abi.SPMV_F64 if v.dtype == np.float64 else abi.SPMV_F32
        n, nnz = rp.size - 1, ci.size
        h = ctypes.c_void_p()
        with torch.cuda.device(device):
            abi.check(abi.spmv_create_symmetric(ctypes.byref(h), n, nnz, _hptr(rp), _hptr(ci) if nnz else None,
                                                _hptr(v) if nnz else None, vt, 0, _stream()),
                      "spmv_create_symmetric")
        return cls(h, n, n, nnz, torch.float64 if vt == abi.SPMV_F64 else torch.float32, device)

    # -- lifetime ---------------------------------------------------------------
    def close(self):
        if self._h is not None and self._h.value:
            abi.spmv_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    # -- queries ----------------------------------------------------------------
    def info(self) -> dict:
        plan = (ctypes.c_int32 * 8)()
        abi.check(abi.spmv_get_info(self._h, None, None, None, plan), "spmv_get_info")
        keys = ("family", "E", "threads", "tiles", "rowcap", "T", "long_rows", "dtype")
        return dict(zip(keys, list(plan)))

    def histogram(self, nbins: int) -> np.ndarray:
        out = np.zeros(nbins, np.int64)
        abi.check(abi.spmv_row_histogram(self._h, nbins, _hptr(out)), "spmv_row_histogram")
        return out

    def set_plan(self, family: int, param: int = 0) -> None:
        abi.check(abi.spmv_set_plan(self._h, family, param), "spmv_set_plan")

    def set_accumulator(self, acc: str) -> None:
        """FP32 storage only: "f64" (one FP64 FMA per entry) or "ff" (float-float)."""
        abi.check(abi.spmv_set_accumulator(self._h, {"f64": 0, "ff": 1}[acc]), "spmv_set_accumulator")

    def set_values(self, val: torch.Tensor, stream=None) -> None:
        self._values_token = None
        abi.check(abi.spmv_set_values(self._h, _dptr(val.contiguous()), _DT[val.dtype],
                                      _stream(stream)), "spmv_set_values")

    def check_device_error(self, stream=None) -> None:
        abi.check(abi.spmv_check_device_error(self._h, _stream(stream)), "device error word")

    # -- products ---------------------------------------------------------------
    def apply(self, x: torch.Tensor, y: Optional[torch.Tensor] = None, alpha: float = 1.0,
              beta: float = 0.0, out_dtype: Optional[torch.dtype] = None, stream=None) -> torch.Tensor:
        """y = alpha*A*x + beta*y (Listing 1 generalised)."""
        if y is None:
            y = torch.empty(self.n_rows, dtype=out_dtype or x.dtype, device=x.device)
        abi.check(abi.spmv_apply(self._h, float(alpha), _dptr(x), _DT[x.dtype], float(beta),
                                 _dptr(y), _DT[y.dtype], _stream(stream)), "spmv_apply")
        return y

    def spmm(self, X: torch.Tensor, Y: Optional[torch.Tensor] = None, alpha: float = 1.0,
             beta: float = 0.0, stream=None) -> torch.Tensor:
        """Block vectors stored interleaved: X (n_cols, nrhs), Y (n_rows, nrhs)."""
        nrhs = X.shape[1]
        if Y is None:
            Y = torch.empty(self.n_rows, nrhs, dtype=X.dtype, device=X.device)
        abi.check(abi.spmm_apply(self._h, nrhs, float(alpha), _dptr(X), float(beta), _dptr(Y),
                                 _DT[X.dtype], _stream(stream)), "spmm_apply")
        return Y

    def backward(self, g: torch.Tensor, x: torch.Tensor, alpha: float = 1.0, need_x: bool = True,
                 need_val: bool = True, stream=None):
        """(grad_x, grad_val) of g^T (alpha*A x)."""
        gx = torch.empty(self.n_cols, dtype=g.dtype, device=g.device) if need_x else None
        gv = torch.empty(self.nnz, dtype=g.dtype, device=g.device) if need_val else None
        abi.check(abi.spmv_backward(self._h, float(alpha), _dptr(g), _dptr(x),
                                    _dptr(gx) if gx is not None and gx.numel() else None,
                                    _dptr(gv) if gv is not None and gv.numel() else None,
                                    _stream(stream)), "spmv_backward")
        return gx, gv

    def transpose_structure(self):
        rp = np.zeros(self.n_cols + 1, np.int32)
        ci = np.zeros(max(self.nnz, 1), np.int32)
        pm = np.zeros(max(self.nnz, 1), np.int32)
        abi.check(abi.spmv_get_transpose(self._h, _hptr(rp), _hptr(ci), _hptr(pm), _stream()),
                  "spmv_get_transpose")
        return rp, ci[: self.nnz], pm[: self.nnz]

    def split(self, nblocks: int = 8, block_row_start: Optional[Sequence[int]] = None,
              equal_rows: bool = False) -> "Split":
        """Local/nonlocal split over ``nblocks`` contiguous row blocks: balanced
        nonzeros by default, ``equal_rows`` for blocks of floor(b*n/nblocks)
        rows (Fig. 6's constant-rows case), or explicit ``block_row_start``."""
        if equal_rows and block_row_start is None:
            block_row_start = [b * self.n_rows // nblocks for b in range(nblocks + 1)]
        return Split(self, nblocks, block_row_start)


class Split:
    """Local/nonlocal split plan of a square FP64 matrix (``spmv_split_handle``)."""

    def __init__(self, A: Matrix, nblocks: int, block_row_start=None):
        self.A = A
        self.nblocks = nblocks
        h = ctypes.c_void_p()
        counts = np.zeros(nblocks, np.int32)
        bs = None
        if block_row_start is not None:
            bs_arr = np.ascontiguousarray(block_row_start, dtype=np.int32)
            bs = _hptr(bs_arr)
        abi.check(abi.spmv_split_create(ctypes.byref(h), A.handle, nblocks, bs, _hptr(counts)),
                  "spmv_split_create")
        self._h = h
        self.halo_count = counts

    def close(self):
        if self._h is not None and self._h.value:
            abi.spmv_split_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def plan(self) -> dict:
        nb = ctypes.c_int32()
        tot = ctypes.c_int64()
        abi.check(abi.spmv_split_get_plan(self._h, ctypes.byref(nb), None, None, ctypes.byref(tot),
                                          None, None, None), "spmv_split_get_plan")
        n = nb.value
        bs = np.zeros(n + 1, np.int32)
        hc = np.zeros(n, np.int32)
        hm = np.zeros(max(tot.value, 1), np.int32)
        nl = np.zeros(n, np.int64)
        nn = np.zeros(n, np.int64)
        abi.check(abi.spmv_split_get_plan(self._h, None, _hptr(bs), _hptr(hc), None, _hptr(hm),
                                          _hptr(nl), _hptr(nn)), "spmv_split_get_plan")
        return dict(block_start=bs, halo_count=hc, total_halo=tot.value, halo_map=hm[: tot.value],
                    nnz_local=nl, nnz_nonlocal=nn)

    def apply(self, x: torch.Tensor, y: Optional[torch.Tensor] = None, alpha: float = 1.0,
              beta: float = 0.0, s_compute=None, s_comm=None) -> torch.Tensor:
        if y is None:
            y = torch.empty(self.A.n_rows, dtype=torch.float64, device=x.device)
        sc = _stream(s_compute)
        sm = _stream(s_comm) if s_comm is not None else sc
        abi.check(abi.spmv_apply_split(self._h, float(alpha), _dptr(x), float(beta), _dptr(y), sc, sm),
                  "spmv_apply_split")
        return y

    def apply_vector(self, x: torch.Tensor, y: Optional[torch.Tensor] = None, alpha: float = 1.0,
                     beta: float = 0.0, stream=None) -> torch.Tensor:
        """Vector mode: gather the whole halo, then one pass over the full matrix."""
        if y is None:
            y = torch.empty(self.A.n_rows, dtype=torch.float64, device=x.device)
        abi.check(abi.spmv_apply_split_vector(self._h, float(alpha), _dptr(x), float(beta), _dptr(y),
                                              _stream(stream)), "spmv_apply_split_vector")
        return y

    def halo(self, stream=None) -> np.ndarray:
        tot = int(self.plan()["total_halo"])
        out = np.zeros(max(tot, 1), np.float64)
        abi.check(abi.spmv_split_get_halo(self._h, _hptr(out), _stream(stream)), "spmv_split_get_halo")
        return out[:tot]


class Batch:
    """Many matrices applied in one persistent launch replayed from a CUDA graph."""

    def __init__(self, mats: Sequence[Matrix]):
        self.mats = list(mats)
        arr = (ctypes.c_void_p * len(self.mats))(*[m.handle.value for m in self.mats])
        h = ctypes.c_void_p()
        abi.check(abi.spmv_batched_create(ctypes.byref(h), len(self.mats), arr), "spmv_batched_create")
        self._h = h

    def close(self):
        if self._h is not None and self._h.value:
            abi.spmv_batched_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        plan = (ctypes.c_int32 * 4)()
        abi.check(abi.spmv_batched_get_info(self._h, plan), "spmv_batched_get_info")
        out = dict(zip(("E", "threads", "tiles", "grid"), list(plan)))
        per = (ctypes.c_int32 * len(self.mats))()
        abi.check(abi.spmv_batched_get_member_plan(self._h, per), "spmv_batched_get_member_plan")
        out["member_E"] = list(per)
        return out

    def apply(self, xs: Sequence[torch.Tensor], ys: Sequence[torch.Tensor], alpha: float = 1.0,
              beta: float = 0.0, stream=None) -> None:
        n = len(self.mats)
        xa = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
        ya = (ctypes.c_void_p * n)(*[y.data_ptr() for y in ys])
        abi.check(abi.spmv_batched_apply(self._h, float(alpha), xa, float(beta), ya, _stream(stream)),
                  "spmv_batched_apply")


class SpMVFunction(torch.autograd.Function):
    """y = alpha*A(val)*x with the hand-written reverse pass of the library:
    grad_x = alpha*A^T g (transposed CRS built once on the device) and
    grad_val[k] = alpha*g[row k]*x[col k]."""

    @staticmethod
    def forward(ctx, val: torch.Tensor, x: torch.Tensor, A: Matrix, alpha: float = 1.0):
        A.set_values(val.detach())
        ctx.token = object()
        A._values_token = ctx.token  # the handle holds this forward's values
        y = A.apply(x.detach(), alpha=alpha)
        ctx.save_for_backward(val.detach(), x.detach())
        ctx.A = A
        ctx.alpha = alpha
        return y

    @staticmethod
    def backward(ctx, gy: torch.Tensor):
        val, x = ctx.saved_tensors
        need_val, need_x = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if need_x and getattr(ctx.A, "_values_token", None) is not ctx.token:
            # another forward (or set_values) replaced the handle's values since
            ctx.A.set_values(val)
            ctx.A._values_token = ctx.token
        gx, gv = ctx.A.backward(gy.contiguous(), x, ctx.alpha, need_x=need_x, need_val=need_val)
        return gv, gx, None, None


def spmv(A: Matrix, val: torch.Tensor, x: torch.Tensor, alpha: float = 1.0) -> torch.Tensor:
    """Differentiable y = alpha*A(val)*x."""
    return SpMVFunction.apply(val, x, A, alpha)


def ir_cg(A: Matrix, b: torch.Tensor, outer_tol: float = 1e-12, max_outer: int = 50,
          inner_tol: float = 1e-3, max_inner: int = 500, stream=None):
    """Mixed-precision iterative-refinement CG (FP64 outer, FP32-storage inner).
    The default inner rule (relative residual 1e-3, at most 500 iterations) took
    4 outer and 1040 inner iterations on the 160^3 7-point matrix, 0.83 of the
    FP64 CG time; 1e-4 with 200 took 7 and 1400 (1.12).  Returns (x, stats dict);
    raises unless converged."""
    x = torch.empty_like(b)
    st = np.zeros(4, np.float64)
    status = abi.spmv_ir_cg(A.handle, _dptr(b), _dptr(x), float(outer_tol), int(max_outer),
                            float(inner_tol), int(max_inner), _hptr(st), _stream(stream))
    stats = dict(outer=int(st[0]), inner=int(st[1]), relres=float(st[2]), seconds=float(st[3]),
                 converged=status == abi.SPMV_OK)
    if status not in (abi.SPMV_OK, abi.SPMV_ERR_NOT_CONVERGED):
        abi.check(status, "spmv_ir_cg")
    return x, stats


def cg(A: Matrix, b: torch.Tensor, tol: float = 1e-12, max_iter: int = 10000, stream=None):
    """FP64 CG on the device (comparison solver)."""
    x = torch.empty_like(b)
    st = np.zeros(4, np.float64)
    status = abi.spmv_cg(A.handle, _dptr(b), _dptr(x), float(tol), int(max_iter), _hptr(st),
                         _stream(stream))
    stats = dict(outer=int(st[0]), inner=int(st[1]), relres=float(st[2]), seconds=float(st[3]),
                 converged=status == abi.SPMV_OK)
    if status not in (abi.SPMV_OK, abi.SPMV_ERR_NOT_CONVERGED):
        abi.check(status, "spmv_cg")
    return x, stats
