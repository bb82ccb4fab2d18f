"""Python binding of the C-ABI in include/lrugb.h (argument marshalling only).

Every computation runs in the CUDA library ``liblrugb.so``; this module passes
device pointers of torch tensors and torch's current CUDA stream.  Importing
it raises ImportError when the library has not been built, and there is no
CPU fallback.

Notation (Sec. 2.1 and 3.1 of arXiv 2602.05255, restated with U, V, B, C):
determinant ``A' = A + U V`` with ratio ``det(I + V A^{-1} U)``; Pfaffian
``A' = A + B C B^T`` with ratio ``pf(C^{-1} + B^T A^{-1} B) / pf(C^{-1})``.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# LRUGB_DEBUG=1 loads the debug build (device-side index checks that record a
# sticky error instead of reading out of range, canary-guarded state buffers)
DEBUG = os.environ.get("LRUGB_DEBUG", "") not in ("", "0")
LIB_PATH = os.path.join(_HERE, "liblrugb_debug.so" if DEBUG else "liblrugb.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
        "(there is no CPU fallback)")
_lib = C.CDLL(LIB_PATH)

F64, C128, F32, C64 = 0, 1, 2, 3
DET, PF = 0, 1
FLUSH_NATIVE, FLUSH_TF32X3, FLUSH_TF32, FLUSH_BF16, FLUSH_BF16X3, FLUSH_DF, FLUSH_SPLIT = 0, 1, 2, 3, 4, 5, 6
ARITH_NATIVE, ARITH_DF = 0, 1
REFRESH_AUTO, REFRESH_FP64, REFRESH_TENSOR = 0, 1, 2
WALKER_OK, WALKER_SINGULAR, WALKER_NONFINITE, WALKER_BAD_INDEX = 0, 1, 2, 3

_DTYPES = {torch.float64: F64, torch.complex128: C128, torch.float32: F32, torch.complex64: C64}
_TORCH = {v: k for k, v in _DTYPES.items()}

_STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA runtime error", 3: "device allocation failed",
           4: "call out of order", 5: "singular matrix", 6: "not skew-symmetric",
           7: "bounded device wait gave up", 8: "combination not supported"}


class LRUError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {_lib.lru_status_string(code).decode()} (status {code})")


class _Config(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dtype", C.c_int32), ("walkers", C.c_int64), ("n", C.c_int32),
                ("n_per_walker", C.POINTER(C.c_int32)), ("k", C.c_int32),
                ("k_per_walker", C.POINTER(C.c_int32)), ("delay", C.c_int32), ("flush", C.c_int32),
                ("device", C.c_int32), ("arith", C.c_int32), ("tile_chunks", C.c_int32),
                ("refresh", C.c_int32)]


class _Operand(C.Structure):
    _fields_ = [("dense", C.c_void_p), ("idx", C.c_void_p), ("onehot_mask", C.c_uint32)]


_vp, _i32, _i64, _sz = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t
_H = C.c_void_p
_SIGS = {
    "lru_create": [C.POINTER(_Config), C.POINTER(_H)],
    "lru_destroy": [_H],
    "lru_set_stream": [_H, _vp],
    "lru_device_bytes": [_H, C.POINTER(_sz)],
    "lru_init_det": [_H, _vp, _vp, _vp],
    "lru_init_pf": [_H, _vp, _vp, _vp],
    "lru_refresh_from_scratch": [_H, _vp, _vp, _vp],
    "lru_propose_det": [_H, C.POINTER(_Operand), C.POINTER(_Operand), _vp, _vp],
    "lru_propose_pf": [_H, C.POINTER(_Operand), _vp, _vp, _vp],
    "lru_accept": [_H, _vp],
    "lru_step_persistent": [_H, C.POINTER(_Operand), C.POINTER(_Operand), _vp, _i32, _vp, _vp, _vp, _vp, _vp],
    "lru_flush_delayed": [_H, _vp],
    "lru_get_inverse": [_H, _vp],
    "lru_get_logvalue": [_H, _vp, _vp],
    "lru_get_delay": [_H, _vp],
    "lru_state_bytes": [_H, C.POINTER(_sz)],
    "lru_save_state": [_H, _vp],
    "lru_load_state": [_H, _vp],
    "lru_check_device_error": [_H],
    "lru_wait_selftest": [_H, _i64],
    "lru_form_row_moves": [_H, _vp, _i32, _vp, _vp, _vp, _vp, _vp],
    "lru_form_pf_moves": [_H, _vp, _i32, _vp, _vp, _vp, _vp, _vp],
    "lru_commit_moves": [_H, _vp, _vp, _vp, _vp],
    "lru_gather_rows": [_H, _vp, _i32, _vp, _vp],
    "lru_gather_pairs": [_H, _vp, _i32, _vp, _vp],
    "lru_log_ratio": [_H, _vp],
    "lru_backward_det": [_H, _vp, _vp, _vp, _vp],
    "lru_backward_pf": [_H, _vp, _vp, _vp, _vp],
    "lru_backward_logvalue": [_H, _vp, _vp],
    "lru_scatter_rows_add": [_H, _vp, _vp, _i32, _vp],
    "lru_profile_enable": [_H, _i32],
    "lru_profile_read": [_H, _i32, C.POINTER(C.c_double), C.POINTER(_i64)],
    "lru_launch_count": [_H, C.POINTER(_i64)],
    "lru_slogdet_batched": [_i32, _i64, _i32, _vp, _vp, _vp, _vp],
    "lru_slogpf_batched": [_i32, _i64, _i32, _vp, _vp, _vp, _vp],
    "lru_slogdet_batched_noalloc": [_i32, _i64, _i32, _vp, _vp, _vp, _vp],
    "lru_slogdet_backward": [_i32, _i64, _i32, _vp, _vp, _vp, _vp, _vp, _vp],
    "lru_slogpf_backward": [_i32, _i64, _i32, _vp, _vp, _vp, _vp, _vp, _vp],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int
_lib.lru_status_string.argtypes = [C.c_int]
_lib.lru_status_string.restype = C.c_char_p
_lib.lru_version.argtypes = []
_lib.lru_version.restype = C.c_char_p


def exported_symbols():
    """Names declared by include/lrugb.h that the loaded library resolves."""
    return sorted(list(_SIGS) + ["lru_status_string", "lru_version"])


def version() -> str:
    return _lib.lru_version().decode()


def _check(code: int, where: str):
    if code != 0:
        raise LRUError(code, where)


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _mask_ptr(mask):
    if mask is None:
        return None
    if mask.dtype != torch.uint8:
        raise ValueError("mask must be uint8")
    return _ptr(mask)


@dataclass
class Operand:
    """One proposal operand (kmax vector slots per walker).

    dense: (W, kmax, n) tensor of the handle dtype, slot a = column a of U,
    row a of V or column a of B; idx: (W, kmax) int32 one-hot indices;
    onehot_mask: bit a set means slot a is e_{idx[w, a]} (Sec. 2.2 / 3.2)."""
    dense: Optional[torch.Tensor] = None
    idx: Optional[torch.Tensor] = None
    onehot_mask: int = 0

    def _c(self):
        if self.idx is not None and self.idx.dtype != torch.int32:
            raise ValueError("idx must be int32")
        return _Operand(_ptr(self.dense), _ptr(self.idx), self.onehot_mask)


class LowRankState:
    """Per-walker state of the batched low-rank update (one C-ABI handle).

    kind: "det" or "pf"; k: update rank (det: U has k columns; pf: B has 2k);
    delay: K of the delayed form (0/1 = plain); flush: precision of the
    delayed flush (FLUSH_*)."""

    def __init__(self, kind: str, walkers: int, n, k: int = 1, dtype=torch.float64, delay: int = 0,
                 flush: int = FLUSH_NATIVE, k_per_walker=None, device: Optional[int] = None,
                 arith: int = ARITH_NATIVE, tile_chunks: int = 0, refresh: int = 0):
        self.kind = {"det": DET, "pf": PF}[kind]
        self.dtype = dtype
        self.W = int(walkers)
        self.k = int(k)
        self.delay = int(delay)
        dev = torch.cuda.current_device() if device is None else int(device)
        self.device = torch.device("cuda", dev)
        cfg = _Config()
        cfg.kind = self.kind
        cfg.dtype = _DTYPES[dtype]
        cfg.walkers = self.W
        self._keep = []
        if isinstance(n, int):
            cfg.n = n
            self.n_list = [n] * self.W
        else:
            self.n_list = [int(x) for x in n]
            arr = (C.c_int32 * self.W)(*self.n_list)
            self._keep.append(arr)
            cfg.n = 0
            cfg.n_per_walker = arr
        cfg.k = self.k
        if k_per_walker is not None:
            arr = (C.c_int32 * self.W)(*[int(x) for x in k_per_walker])
            self._keep.append(arr)
            cfg.k_per_walker = arr
        cfg.delay = self.delay
        cfg.flush = int(flush)
        cfg.device = dev
        cfg.arith = int(arith)
        cfg.tile_chunks = int(tile_chunks)
        cfg.refresh = int(refresh)
        h = _H()
        _check(_lib.lru_create(C.byref(cfg), C.byref(h)), "lru_create")
        self._h = h
        self.kmax = self.k if self.kind == DET else 2 * self.k

    def close(self):
        if getattr(self, "_h", None):
            _lib.lru_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _bind(self):
        _check(_lib.lru_set_stream(self._h, _stream()), "lru_set_stream")

    def _vec_out(self, dtype):
        return torch.empty(self.W, dtype=dtype, device=self.device)

    # ---- init / refresh ---------------------------------------------------
    def init(self, A: torch.Tensor):
        """A: all walkers' matrices, row-major, concatenated (uniform: (W, n, n))."""
        self._bind()
        logabs = self._vec_out(torch.float64)
        sign = self._vec_out(self.dtype)
        f = _lib.lru_init_det if self.kind == DET else _lib.lru_init_pf
        _check(f(self._h, _ptr(A), _ptr(logabs), _ptr(sign)), "lru_init")
        return logabs, sign

    def refresh(self, A: torch.Tensor, mask: Optional[torch.Tensor] = None, want_drift: bool = True):
        self._bind()
        drift = torch.full((self.W,), float("nan"), dtype=torch.float64, device=self.device) if want_drift else None
        _check(_lib.lru_refresh_from_scratch(self._h, _ptr(A), _mask_ptr(mask), _ptr(drift)), "lru_refresh")
        return drift

    # ---- propose / accept -------------------------------------------------
    def propose_det(self, U: Operand, V: Operand, ratio=None, status=None):
        self._bind()
        ratio = self._vec_out(self.dtype) if ratio is None else ratio
        status = torch.empty(self.W, dtype=torch.int32, device=self.device) if status is None else status
        self._last = (U, V)   # the accept pass reads V
        u, v = U._c(), V._c()
        _check(_lib.lru_propose_det(self._h, C.byref(u), C.byref(v), _ptr(ratio), _ptr(status)), "lru_propose_det")
        return ratio, status

    def propose_pf(self, B: Operand, Cmat: Optional[torch.Tensor] = None, ratio=None, status=None):
        self._bind()
        ratio = self._vec_out(self.dtype) if ratio is None else ratio
        status = torch.empty(self.W, dtype=torch.int32, device=self.device) if status is None else status
        self._last = (B, Cmat)
        b = B._c()
        _check(_lib.lru_propose_pf(self._h, C.byref(b), _ptr(Cmat), _ptr(ratio), _ptr(status)), "lru_propose_pf")
        return ratio, status

    def step_persistent(self, U: Operand, V: Optional[Operand] = None, Cmat: Optional[torch.Tensor] = None,
                        accept: bool = True, mask=None, u=None, ratio=None, status=None, acc=None):
        """One persistent fused propose(+accept) launch over all walkers (ragged n, k
        allowed); graph-capturable.  Returns (ratio, status, accepted)."""
        self._bind()
        ratio = self._vec_out(self.dtype) if ratio is None else ratio
        status = torch.empty(self.W, dtype=torch.int32, device=self.device) if status is None else status
        acc = torch.empty(self.W, dtype=torch.uint8, device=self.device) if acc is None else acc
        self._last = (U, V, Cmat)
        u_c = U._c()
        v_c = (V or U)._c()
        _check(_lib.lru_step_persistent(self._h, C.byref(u_c), C.byref(v_c), _ptr(Cmat), 1 if accept else 0,
                                        _mask_ptr(mask), _ptr(u), _ptr(ratio), _ptr(status), _ptr(acc)),
               "lru_step_persistent")
        return ratio, status, acc

    def accept(self, mask: Optional[torch.Tensor] = None):
        self._bind()
        _check(_lib.lru_accept(self._h, _mask_ptr(mask)), "lru_accept")

    def flush(self, mask: Optional[torch.Tensor] = None):
        self._bind()
        _check(_lib.lru_flush_delayed(self._h, _mask_ptr(mask)), "lru_flush_delayed")

    # ---- state access -----------------------------------------------------
    def inverse(self) -> torch.Tensor:
        self._bind()
        total = sum(n * n for n in self.n_list)
        out = torch.empty(total, dtype=self.dtype, device=self.device)
        _check(_lib.lru_get_inverse(self._h, _ptr(out)), "lru_get_inverse")
        if len(set(self.n_list)) == 1:
            n = self.n_list[0]
            return out.view(self.W, n, n)
        return out

    def logvalue(self):
        self._bind()
        logabs = self._vec_out(torch.float64)
        sign = self._vec_out(self.dtype)
        _check(_lib.lru_get_logvalue(self._h, _ptr(logabs), _ptr(sign)), "lru_get_logvalue")
        return logabs, sign

    def tau(self):
        self._bind()
        t = torch.empty(self.W, dtype=torch.int32, device=self.device)
        _check(_lib.lru_get_delay(self._h, _ptr(t)), "lru_get_delay")
        return t

    def state_bytes(self) -> int:
        b = _sz()
        _check(_lib.lru_state_bytes(self._h, C.byref(b)), "lru_state_bytes")
        return b.value

    def device_bytes(self) -> int:
        b = _sz()
        _check(_lib.lru_device_bytes(self._h, C.byref(b)), "lru_device_bytes")
        return b.value

    def save(self) -> torch.Tensor:
        self._bind()
        buf = torch.empty(self.state_bytes(), dtype=torch.uint8, device=self.device)
        _check(_lib.lru_save_state(self._h, _ptr(buf)), "lru_save_state")
        return buf

    def load(self, buf: torch.Tensor):
        self._bind()
        _check(_lib.lru_load_state(self._h, _ptr(buf)), "lru_load_state")

    def check_device_error(self):
        self._bind()
        _check(_lib.lru_check_device_error(self._h), "lru_check_device_error")

    def wait_selftest(self, polls: int):
        """Enqueue a bounded wait on a flag nothing sets (see lru_wait_selftest)."""
        self._bind()
        _check(_lib.lru_wait_selftest(self._h, int(polls)), "lru_wait_selftest")

    # ---- reverse mode --------------------------------------------------------
    def log_ratio(self) -> torch.Tensor:
        """log of the pending proposal's ratios (real: log|r|, complex: log r)."""
        self._bind()
        out = self._vec_out(self.dtype)
        _check(_lib.lru_log_ratio(self._h, _ptr(out)), "lru_log_ratio")
        return out

    @property
    def uniform(self) -> bool:
        return len(set(self.n_list)) == 1

    def _ops_like(self):
        """Zeros in the operand vector layout: (W, kmax, n), or flat sum(n) * kmax when n varies."""
        if self.uniform:
            return torch.zeros(self.W, self.kmax, self.n_list[0], dtype=self.dtype, device=self.device)
        return torch.zeros(sum(self.n_list) * self.kmax, dtype=self.dtype, device=self.device)

    def _mats_like(self):
        """Matrices of every walker: (W, n, n), or flat sum(n^2) when n varies."""
        if self.uniform:
            n = self.n_list[0]
            return torch.empty(self.W, n, n, dtype=self.dtype, device=self.device)
        return torch.empty(sum(x * x for x in self.n_list), dtype=self.dtype, device=self.device)

    def backward_det(self, g: torch.Tensor, want_U=True, want_V=True, want_A=True):
        """(gU, gV, gA): vector-Jacobian product of the pending proposal's log ratio."""
        self._bind()
        gU = self._ops_like() if want_U else None
        gV = self._ops_like() if want_V else None
        gA = self._mats_like() if want_A else None
        _check(_lib.lru_backward_det(self._h, _ptr(g.contiguous()), _ptr(gU), _ptr(gV), _ptr(gA)), "lru_backward_det")
        return gU, gV, gA

    def backward_pf(self, g: torch.Tensor, want_B=True, want_C=True, want_A=True):
        """(gB, gC, gA) for the pending Pfaffian proposal (skew parts of A and C)."""
        self._bind()
        gB = self._ops_like() if want_B else None
        gC = torch.empty(self.W, self.kmax, self.kmax, dtype=self.dtype, device=self.device) if want_C else None
        gA = self._mats_like() if want_A else None
        _check(_lib.lru_backward_pf(self._h, _ptr(g.contiguous()), _ptr(gB), _ptr(gC), _ptr(gA)), "lru_backward_pf")
        return gB, gC, gA

    def backward_logvalue(self, g: torch.Tensor) -> torch.Tensor:
        self._bind()
        gA = self._mats_like()
        _check(_lib.lru_backward_logvalue(self._h, _ptr(g.contiguous()), _ptr(gA)), "lru_backward_logvalue")
        return gA

    def scatter_rows_add(self, gA: torch.Tensor, rows: torch.Tensor, gPhi: torch.Tensor):
        self._bind()
        _check(_lib.lru_scatter_rows_add(self._h, _ptr(gA), _ptr(rows), gPhi.shape[0], _ptr(gPhi)),
               "lru_scatter_rows_add")
        return gPhi

    # ---- profiling ---------------------------------------------------------
    PROF_PROPOSE, PROF_ACCEPT, PROF_FLUSH, PROF_REFRESH = 0, 1, 2, 3

    def profile(self, on: bool = True):
        _check(_lib.lru_profile_enable(self._h, 1 if on else 0), "lru_profile_enable")

    def profile_read(self, cls: int):
        """(total ms, launches) of kernel class cls since the last read."""
        self._bind()
        ms, cnt = C.c_double(), _i64()
        _check(_lib.lru_profile_read(self._h, cls, C.byref(ms), C.byref(cnt)), "lru_profile_read")
        return ms.value, cnt.value

    def launch_count(self) -> int:
        cnt = _i64()
        _check(_lib.lru_launch_count(self._h, C.byref(cnt)), "lru_launch_count")
        return cnt.value

    # ---- QMC move operands -------------------------------------------------
    def form_row_moves(self, Phi, occ, slot, new_row, V_out=None, idx_out=None):
        self._bind()
        n = self.n_list[0]
        V_out = torch.empty(self.W, self.k, n, dtype=self.dtype, device=self.device) if V_out is None else V_out
        idx_out = torch.empty(self.W, self.k, dtype=torch.int32, device=self.device) if idx_out is None else idx_out
        _check(_lib.lru_form_row_moves(self._h, _ptr(Phi), Phi.shape[0], _ptr(occ), _ptr(slot), _ptr(new_row),
                                       _ptr(V_out), _ptr(idx_out)), "lru_form_row_moves")
        return V_out, idx_out

    def form_pf_moves(self, F, pos, slot, new_site, B_out=None, idx_out=None):
        self._bind()
        n = self.n_list[0]
        kk = self.kmax        # 2 (one particle) or 4 (two particles at once)
        B_out = torch.empty(self.W, kk, n, dtype=self.dtype, device=self.device) if B_out is None else B_out
        idx_out = torch.empty(self.W, kk, dtype=torch.int32, device=self.device) if idx_out is None else idx_out
        _check(_lib.lru_form_pf_moves(self._h, _ptr(F), F.shape[0], _ptr(pos), _ptr(slot), _ptr(new_site),
                                      _ptr(B_out), _ptr(idx_out)), "lru_form_pf_moves")
        return B_out, idx_out

    def commit_moves(self, occ, slot, new_row, mask=None):
        self._bind()
        _check(_lib.lru_commit_moves(self._h, _ptr(occ), _ptr(slot), _ptr(new_row), _mask_ptr(mask)),
               "lru_commit_moves")


def _gather(self, which, src, occ, out=None):
    self._bind()
    n = self.n_list[0]
    out = torch.empty(self.W, n, n, dtype=self.dtype, device=self.device) if out is None else out
    f = _lib.lru_gather_rows if which == "rows" else _lib.lru_gather_pairs
    _check(f(self._h, _ptr(src), src.shape[0], _ptr(occ), _ptr(out)), "lru_gather")
    return out


LowRankState.gather_rows = lambda self, Phi, occ, out=None: _gather(self, "rows", Phi, occ, out)
LowRankState.gather_pairs = lambda self, F, pos, out=None: _gather(self, "pairs", F, pos, out)


def slogdet_batched(A: torch.Tensor):
    """(sign, log|det|) of W row-major n x n matrices (Gauss-Jordan, handle dtype)."""
    W, n = A.shape[0], A.shape[-1]
    logabs = torch.empty(W, dtype=torch.float64, device=A.device)
    sign = torch.empty(W, dtype=A.dtype, device=A.device)
    _check(_lib.lru_slogdet_batched(_DTYPES[A.dtype], W, n, _ptr(A), _ptr(logabs), _ptr(sign), _stream()),
           "lru_slogdet_batched")
    return sign, logabs


def slogdet_batched_noalloc(A: torch.Tensor, logabs=None, sign=None):
    """slogdet_batched without any device allocation by the library: the
    workspace is a fixed 64 MiB array in the library's device memory, shared by
    all calls (overlapping calls race; the first call on a device should come
    before any stream capture).  Pass logabs / sign to avoid allocations here too."""
    W, n = A.shape[0], A.shape[-1]
    logabs = torch.empty(W, dtype=torch.float64, device=A.device) if logabs is None else logabs
    sign = torch.empty(W, dtype=A.dtype, device=A.device) if sign is None else sign
    _check(_lib.lru_slogdet_batched_noalloc(_DTYPES[A.dtype], W, n, _ptr(A), _ptr(logabs), _ptr(sign), _stream()),
           "lru_slogdet_batched_noalloc")
    return sign, logabs


def slogpf_batched(A: torch.Tensor):
    """(sign/phase, log|pf|) of W skew-symmetric n x n matrices (App. A.1 slogpf;
    Parlett-Reid elimination with pivoting)."""
    W, n = A.shape[0], A.shape[-1]
    logabs = torch.empty(W, dtype=torch.float64, device=A.device)
    sign = torch.empty(W, dtype=A.dtype, device=A.device)
    _check(_lib.lru_slogpf_batched(_DTYPES[A.dtype], W, n, _ptr(A), _ptr(logabs), _ptr(sign), _stream()),
           "lru_slogpf_batched")
    return sign, logabs


class _SlogBatched(torch.autograd.Function):
    """(sign, log|det A|) or (sign, log|pf A|) of a batch, differentiable: the
    forward is lru_slogdet_batched / lru_slogpf_batched, the backward
    lru_slogdet_backward / lru_slogpf_backward (App. A.3)."""

    @staticmethod
    def forward(ctx, A, pf):
        A = A.contiguous()
        sign, logabs = (slogpf_batched if pf else slogdet_batched)(A)
        ctx.save_for_backward(A, sign)
        ctx.pf = pf
        if not A.is_complex():
            ctx.mark_non_differentiable(sign)
        return sign, logabs

    @staticmethod
    def backward(ctx, g_sign, g_logabs):
        A, sign = ctx.saved_tensors
        W, n = A.shape[0], A.shape[-1]
        gA = torch.empty_like(A)
        g_l = g_logabs.contiguous().to(torch.float64) if g_logabs is not None else None
        g_s = g_sign.contiguous() if (g_sign is not None and A.is_complex()) else None
        f = _lib.lru_slogpf_backward if ctx.pf else _lib.lru_slogdet_backward
        _check(f(_DTYPES[A.dtype], W, n, _ptr(A), _ptr(g_l), _ptr(g_s), _ptr(sign), _ptr(gA), _stream()),
               "lru_slog_backward")
        return gA, None


def slogdet(A: torch.Tensor):
    """Differentiable (sign, log|det|) of W matrices (W, n, n) on the device."""
    return _SlogBatched.apply(A, False)


def slogpf(A: torch.Tensor):
    """Differentiable (sign, log|pf|) of W skew matrices (W, n, n); the
    gradient is taken through the skew projection (A - A^T) / 2 (App. A.3)."""
    return _SlogBatched.apply(A, True)


# ---------------------------------------------------------------------------
# torch.autograd.Function wrappers: the forward is a propose through the
# C-ABI, the backward the adjoint kernel.  Call loss.backward() before
# accepting the proposal (accept changes the state the adjoint reads).
# ---------------------------------------------------------------------------
class _DetLogRatio(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, V, A, state):
        state.propose_det(Operand(dense=U.contiguous()), Operand(dense=V.contiguous()))
        ctx.state = state
        ctx.want = (ctx.needs_input_grad[0], ctx.needs_input_grad[1], A is not None and ctx.needs_input_grad[2])
        return state.log_ratio()

    @staticmethod
    def backward(ctx, g):
        gU, gV, gA = ctx.state.backward_det(g, *ctx.want)
        return gU, gV, gA, None


def det_log_ratio(state: LowRankState, U: torch.Tensor, V: torch.Tensor, A: Optional[torch.Tensor] = None):
    """log det(I + V A^{-1} U) per walker (Sec. 2.1), differentiable in U, V
    ((W, k, n) dense tensors) and A (the matrices whose inverses the state
    holds).  Real dtypes give log|r|, complex the principal log r."""
    return _DetLogRatio.apply(U, V, A, state)


class _PfLogRatio(torch.autograd.Function):
    @staticmethod
    def forward(ctx, B, Cm, A, state):
        state.propose_pf(Operand(dense=B.contiguous()), None if Cm is None else Cm.contiguous())
        ctx.state = state
        ctx.want = (ctx.needs_input_grad[0], Cm is not None and ctx.needs_input_grad[1],
                    A is not None and ctx.needs_input_grad[2])
        return state.log_ratio()

    @staticmethod
    def backward(ctx, g):
        gB, gC, gA = ctx.state.backward_pf(g, *ctx.want)
        return gB, gC, gA, None


def pf_log_ratio(state: LowRankState, B: torch.Tensor, Cm: Optional[torch.Tensor] = None,
                 A: Optional[torch.Tensor] = None):
    """log [pf(C^{-1} + B^T A^{-1} B) / pf(C^{-1})] per walker (App. A.2), differentiable
    in B ((W, 2k, n)), C ((W, 2k, 2k); None = -J) and A, with A and C entering
    through their skew parts (App. A.3)."""
    return _PfLogRatio.apply(B, Cm, A, state)


class _OrbitalLogRatio(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Phi, U, V, state, rows):
        state.propose_det(Operand(dense=U.contiguous()), Operand(dense=V.contiguous()))
        ctx.state, ctx.rows, ctx.m = state, rows, Phi.shape[0]
        ctx.save_for_backward(Phi)
        return state.log_ratio()

    @staticmethod
    def backward(ctx, g):
        (Phi,) = ctx.saved_tensors
        gU, gV, gA = ctx.state.backward_det(g, True, True, True)
        gPhi = torch.zeros_like(Phi)
        ctx.state.scatter_rows_add(gA, ctx.rows, gPhi)
        return gPhi, gU, gV, None, None


def orbital_log_ratio(state: LowRankState, Phi: torch.Tensor, rows: torch.Tensor, U: torch.Tensor,
                      V: torch.Tensor):
    """log det(I + V A^{-1} U) with A_w = Phi[rows_w] (the state holds A^{-1}),
    differentiable in the orbital matrix Phi (through A), U and V."""
    return _OrbitalLogRatio.apply(Phi, U, V, state, rows)
