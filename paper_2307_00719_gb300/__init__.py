"""Python binding of the GB300 streaming tensor-ring library (libstrtr.so).

Argument marshalling only: every step of an update runs in the library's CUDA
kernels behind the C ABI of ``include/strtr.h``.  The functions below carry
the C names (``str_init``, ``str_update``, ``rstr_update``, ``tr_reconstruct``,
``tr_fit_error``, ...); ``Stream`` wraps one context.  There is no CPU
fallback: if the library is missing or no GPU is present, calls raise.

Array conventions
-----------------
* A tensor is indexed ``X[i_1, ..., i_N]`` with i_1 fastest in memory (the
  paper's linear index): a numpy array in Fortran order, or a torch tensor
  whose strides are Fortran-contiguous (see ``paper_layout``).
* A core ``G_n`` is a float64 array of shape ``(R_n, I_n, R_{n+1})``.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import (POINTER, Structure, byref, c_char_p, c_double, c_int, c_int64, c_size_t,
                    c_uint32, c_uint64, c_void_p)
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libstrtr.so")

STR_BF16, STR_F32, STR_F64 = 0, 1, 2
SKETCH_NONE, SKETCH_UNIFORM, SKETCH_LEVERAGE, SKETCH_KSRFT = -1, 0, 1, 2
SKETCH_NAMES = {"none": SKETCH_NONE, "uniform": SKETCH_UNIFORM, "leverage": SKETCH_LEVERAGE,
                "ksrft": SKETCH_KSRFT}
STATUS = {0: "STR_OK", 1: "STR_ERR_INVALID_ARG", 2: "STR_ERR_SHAPE", 3: "STR_ERR_DTYPE",
          4: "STR_ERR_SINGULAR", 5: "STR_ERR_NONFINITE", 6: "STR_ERR_CAPACITY", 7: "STR_ERR_OOM",
          8: "STR_ERR_CUDA", 9: "STR_ERR_TIMEOUT", 10: "STR_ERR_STATE"}


class StrOptions(Structure):
    _fields_ = [("compute", c_int), ("sweeps", c_int), ("rescale", c_int), ("t_capacity", c_int64),
                ("init_max_it", c_int), ("init_tol", c_double), ("sketch", c_int), ("m", c_int64),
                ("seed", c_uint64), ("stream_id", c_uint32), ("check_finite", c_int),
                ("async_status", c_int), ("profile", c_int), ("mttkrp_path", c_int),
                ("graphs", c_int)]


class StrTensor(Structure):
    _fields_ = [("data", c_void_p), ("dtype", c_int), ("order", c_int), ("dims", POINTER(c_int64)),
                ("on_host", c_int)]


class StrStats(Structure):
    _fields_ = [("steps", c_int64), ("time_rows", c_int64), ("kernel_launches", c_int64),
                ("device_bytes", c_int64), ("min_pivot_ratio", c_double),
                ("class_launches", c_int64 * 9), ("class_ms", c_double * 9), ("fp64_fallbacks", c_int64)]


KERNEL_CLASSES = ("mttkrp", "reduce", "gram", "factor", "solve", "sketch", "dft", "other", "contract")


class _SaveHeader(Structure):
    """Leading fields of the library's checkpoint blob."""
    _fields_ = [("magic", c_uint64), ("N", ctypes.c_int32), ("compute", ctypes.c_int32),
                ("I", c_int64 * 8), ("R", ctypes.c_int32 * 9), ("opt", StrOptions)]


class StrError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = f"{where}: {STATUS.get(status, status)}"
        try:
            s = lib().str_status_string(status).decode()
            last = lib().str_last_error().decode()
            msg += f" ({s})" + (f" [{last}]" if last else "")
        except Exception:  # pragma: no cover - message decoration only
            pass
        super().__init__(msg)


_lib = None

# (name, restype, argtypes) for every entry point of strtr.h
_SIGS = [
    ("str_default_options", c_int, [POINTER(StrOptions)]),
    ("str_init", c_int, [POINTER(c_void_p), POINTER(StrTensor), POINTER(c_int), POINTER(c_void_p),
                         POINTER(StrOptions), c_void_p]),
    ("str_init_cores", c_int, [POINTER(c_void_p), c_int, POINTER(c_int64), POINTER(c_int), c_int64,
                               POINTER(c_void_p), POINTER(StrTensor), POINTER(StrOptions), c_void_p]),
    ("str_update", c_int, [c_void_p, POINTER(StrTensor), c_void_p]),
    ("rstr_update", c_int, [c_void_p, POINTER(StrTensor), c_int, c_int64, c_uint64, c_void_p]),
    ("str_update_batch", c_int, [POINTER(c_void_p), POINTER(POINTER(StrTensor)), c_int, c_int, c_void_p]),
    ("tr_reconstruct", c_int, [c_void_p, c_int64, c_int64, c_void_p, c_int, c_void_p]),
    ("tr_fit_error", c_int, [c_void_p, POINTER(StrTensor), c_int64, POINTER(c_double), c_void_p]),
    ("str_get_core", c_int, [c_void_p, c_int, c_void_p]),
    ("str_num_time_rows", c_int64, [c_void_p]),
    ("str_get_pq", c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    ("str_get_samples", c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    ("str_save", c_int, [c_void_p, c_void_p, POINTER(c_size_t)]),
    ("str_load", c_int, [POINTER(c_void_p), c_void_p, c_size_t, c_void_p]),
    ("str_get_stats", c_int, [c_void_p, POINTER(StrStats)]),
    ("str_sync", c_int, [c_void_p]),
    ("str_status_string", c_char_p, [c_int]),
    ("str_last_error", c_char_p, []),
    ("str_destroy", None, [c_void_p]),
    ("tr_masked_loss_fwd", c_int, [c_int, POINTER(c_int64), POINTER(c_int), c_int, POINTER(c_void_p),
                                   c_void_p, c_void_p, c_void_p, c_void_p]),
    ("tr_masked_loss_bwd", c_int, [c_int, POINTER(c_int64), POINTER(c_int), c_int, POINTER(c_void_p),
                                   c_void_p, c_void_p, c_double, POINTER(c_void_p), c_void_p]),
    ("tr_masked_loss_fwd_noalloc", c_int, [c_int, POINTER(c_int64), POINTER(c_int), c_int,
                                           POINTER(c_void_p), c_void_p, c_void_p, c_void_p, c_void_p]),
    ("str_fma_probe", c_int, [c_int, c_int, c_int64, c_void_p, POINTER(c_double), c_void_p]),
]


def lib():
    """Load libstrtr.so (built in-tree by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int, where: str):
    if status != 0:
        raise StrError(status, where)


def _torch():
    import torch
    return torch


def _stream_handle(stream=None):
    if stream is not None:
        return c_void_p(int(stream))
    try:
        torch = _torch()
        if torch.cuda.is_available():
            return c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return c_void_p(0)


def default_options(**kw) -> StrOptions:
    o = StrOptions()
    _check(lib().str_default_options(byref(o)), "str_default_options")
    for k, v in kw.items():
        if k == "sketch" and isinstance(v, str):
            v = SKETCH_NAMES[v]
        if k == "compute" and isinstance(v, str):
            v = {"f64": STR_F64, "f32": STR_F32}[v]
        setattr(o, k, v)
    return o


def paper_layout(x):
    """Return a view/copy of torch tensor ``x`` (indexed [i_1..i_N]) with i_1 fastest."""
    rev = list(range(x.dim() - 1, -1, -1))
    return x.permute(rev).contiguous().permute(rev)


def _is_fortran(x) -> bool:
    expected = 1
    for size, stride in zip(x.shape, x.stride()):
        if size != 1 and stride != expected:
            return False
        expected *= size
    return True


class _TensorArg:
    """A StrTensor plus the objects that must stay alive during the call."""

    def __init__(self, x):
        self.keep = [x]
        try:
            torch = _torch()
            is_torch = isinstance(x, torch.Tensor)
        except ImportError:  # pragma: no cover
            is_torch = False
        if is_torch:
            dt = {torch.float64: STR_F64, torch.float32: STR_F32, torch.bfloat16: STR_BF16}.get(x.dtype)
            if dt is None:
                raise TypeError(f"unsupported dtype {x.dtype}")
            if not _is_fortran(x):
                raise ValueError("tensor must have i_1-fastest (Fortran) strides; use paper_layout()")
            ptr = x.data_ptr()
            on_host = 0 if x.is_cuda else 1
            shape = tuple(x.shape)
        else:
            a = np.asfortranarray(x)
            if a.dtype == np.float64:
                dt = STR_F64
            elif a.dtype == np.float32:
                dt = STR_F32
            else:
                raise TypeError(f"unsupported dtype {a.dtype}")
            self.keep.append(a)
            ptr = a.ctypes.data
            on_host = 1
            shape = a.shape
        self.dims = (c_int64 * len(shape))(*shape)
        self.struct = StrTensor(c_void_p(ptr), dt, len(shape), self.dims, on_host)
        self.shape = shape


def cores_to_abi(cores: Sequence[np.ndarray]) -> List[np.ndarray]:
    """(R_n, I_n, R_{n+1}) arrays -> G_{n(2)} row-major buffers (offset i*R_nR_{n+1} + b*R_n + a)."""
    return [np.ascontiguousarray(np.asarray(G, dtype=np.float64).transpose(1, 2, 0)) for G in cores]


def abi_to_core(buf: np.ndarray, Ra: int, rows: int, Rb: int) -> np.ndarray:
    return np.ascontiguousarray(buf.reshape(rows, Rb, Ra).transpose(2, 0, 1))


def _opts(options, **kw) -> StrOptions:
    if options is None:
        return default_options(**kw)
    if isinstance(options, dict):
        d = dict(options)
        d.update(kw)
        return default_options(**d)
    return options


class Stream:
    """One streaming TR context (owns its device state)."""

    def __init__(self, handle: c_void_p, N: int, dims, ranks, options: StrOptions):
        self._h = handle
        self.N = N
        self.dims = tuple(int(d) for d in dims)     # spatial I_1..I_{N-1}
        self.ranks = tuple(int(r) for r in ranks)
        self.options = options

    # ---- lifetime -----------------------------------------------------------
    def close(self):
        if self._h is not None and self._h.value:
            lib().str_destroy(self._h)
        self._h = None

    def __del__(self):  # pragma: no cover - best effort
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self) -> c_void_p:
        if self._h is None or not self._h.value:
            raise RuntimeError("stream is closed")
        return self._h

    # ---- state access -------------------------------------------------------
    def time_rows(self) -> int:
        return int(lib().str_num_time_rows(self.handle))

    def core(self, n: int) -> np.ndarray:
        """Core n (1-based) as (R_n, rows, R_{n+1}) float64."""
        Ra, Rb = self.ranks[n - 1], self.ranks[n % self.N]
        rows = self.time_rows() if n == self.N else self.dims[n - 1]
        buf = np.empty(rows * Ra * Rb, dtype=np.float64)
        _check(lib().str_get_core(self.handle, n, buf.ctypes.data), "str_get_core")
        return abi_to_core(buf, Ra, rows, Rb)

    def cores(self) -> List[np.ndarray]:
        return [self.core(n) for n in range(1, self.N + 1)]

    def pq(self, n: int):
        Ra, Rb = self.ranks[n - 1], self.ranks[n % self.N]
        P = np.empty((self.dims[n - 1], Ra * Rb))
        Q = np.empty((Ra * Rb, Ra * Rb))
        _check(lib().str_get_pq(self.handle, n, P.ctypes.data, Q.ctypes.data), "str_get_pq")
        return P, Q

    def samples(self, k: int, with_p: bool = False, p_rows: Optional[int] = None):
        m = int(self.options.m)
        idx = np.empty(m, dtype=np.int64)
        p = None
        if with_p:
            rows = p_rows if p_rows is not None else (self.dims[k - 1] if k < self.N else self.time_rows())
            p = np.empty(rows, dtype=np.float64)
        _check(lib().str_get_samples(self.handle, k, idx.ctypes.data, p.ctypes.data if p is not None else None),
               "str_get_samples")
        return (idx, p) if with_p else idx

    def stats(self) -> dict:
        s = StrStats()
        _check(lib().str_get_stats(self.handle, byref(s)), "str_get_stats")
        out = {f: getattr(s, f) for f, _ in StrStats._fields_[:5]}
        out["class_launches"] = dict(zip(KERNEL_CLASSES, list(s.class_launches)))
        out["class_ms"] = dict(zip(KERNEL_CLASSES, list(s.class_ms)))
        out["fp64_fallbacks"] = int(s.fp64_fallbacks)
        return out

    def sync(self):
        _check(lib().str_sync(self.handle), "str_sync")

    def save(self) -> bytes:
        n = c_size_t(0)
        _check(lib().str_save(self.handle, None, byref(n)), "str_save")
        buf = ctypes.create_string_buffer(n.value)
        _check(lib().str_save(self.handle, buf, byref(n)), "str_save")
        return buf.raw[: n.value]

    @classmethod
    def load(cls, blob: bytes, stream=None) -> "Stream":
        h = c_void_p()
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(lib().str_load(byref(h), buf, len(blob), _stream_handle(stream)), "str_load")
        hdr = _SaveHeader.from_buffer_copy(blob[: ctypes.sizeof(_SaveHeader)])
        N = int(hdr.N)
        opts = StrOptions.from_buffer_copy(bytes(hdr.opt))
        return cls(h, N, list(hdr.I)[: N - 1], list(hdr.R)[:N], opts)

    # ---- updates (thin wrappers over the C calls) ---------------------------
    def update(self, X, stream=None):
        str_update(self, X, stream)

    def rupdate(self, X, stream=None):
        o = self.options
        rstr_update(self, X, int(o.sketch), int(o.m), int(o.seed), stream)

    def fit_error(self, X, t0: int = 0, stream=None) -> float:
        return tr_fit_error(self, X, t0, stream)

    def reconstruct(self, t0: int, t1: int, dtype=None, stream=None):
        return tr_reconstruct(self, t0, t1, dtype, stream)


# ---------------------------------------------------------------------------
# C-named entry points
# ---------------------------------------------------------------------------
def str_init_cores(cores: Sequence[np.ndarray], X0=None, options=None, stream=None, **kw) -> Stream:
    """Context from given initial cores (Alg. 4/5 initialisation stage)."""
    opts = _opts(options, **kw)
    N = len(cores)
    ranks = [int(G.shape[0]) for G in cores]
    dims = [int(G.shape[1]) for G in cores]
    abi = cores_to_abi(cores)
    ptrs = (c_void_p * N)(*[a.ctypes.data for a in abi])
    d = (c_int64 * N)(*dims)
    r = (c_int * N)(*ranks)
    h = c_void_p()
    xarg = _TensorArg(X0) if X0 is not None else None
    _check(lib().str_init_cores(byref(h), N, d, r, dims[-1], ptrs,
                                byref(xarg.struct) if xarg else None, byref(opts), _stream_handle(stream)),
           "str_init_cores")
    return Stream(h, N, dims[:-1], ranks, opts)


def str_init(X0, ranks: Sequence[int], guess: Sequence[np.ndarray], options=None, stream=None, **kw) -> Stream:
    """Context whose initial cores are computed by TR-ALS-NE (Alg. 2) on X0 from `guess`."""
    opts = _opts(options, **kw)
    xarg = _TensorArg(X0)
    N = len(xarg.shape)
    abi = cores_to_abi(guess)
    ptrs = (c_void_p * N)(*[a.ctypes.data for a in abi])
    r = (c_int * N)(*[int(v) for v in ranks])
    h = c_void_p()
    _check(lib().str_init(byref(h), byref(xarg.struct), r, ptrs, byref(opts), _stream_handle(stream)), "str_init")
    return Stream(h, N, xarg.shape[:-1], ranks, opts)


def str_update(ctx: Stream, X, stream=None):
    x = _TensorArg(X)
    _check(lib().str_update(ctx.handle, byref(x.struct), _stream_handle(stream)), "str_update")


def rstr_update(ctx: Stream, X, sketch, m: int, seed: int, stream=None):
    if isinstance(sketch, str):
        sketch = SKETCH_NAMES[sketch]
    x = _TensorArg(X)
    _check(lib().rstr_update(ctx.handle, byref(x.struct), int(sketch), int(m), int(seed), _stream_handle(stream)),
           "rstr_update")


def str_update_batch(ctxs: Sequence[Stream], Xs: Sequence, randomized: bool = False, stream=None):
    args = [_TensorArg(x) for x in Xs]
    n = len(ctxs)
    hs = (c_void_p * n)(*[c.handle.value for c in ctxs])
    ts = (POINTER(StrTensor) * n)(*[ctypes.pointer(a.struct) for a in args])
    _check(lib().str_update_batch(hs, ts, n, int(bool(randomized)), _stream_handle(stream)), "str_update_batch")


def tr_fit_error(ctx: Stream, X, t0: int = 0, stream=None) -> float:
    x = _TensorArg(X)
    out = c_double(0.0)
    _check(lib().tr_fit_error(ctx.handle, byref(x.struct), int(t0), byref(out), _stream_handle(stream)),
           "tr_fit_error")
    return float(out.value)


def tr_reconstruct(ctx: Stream, t0: int, t1: int, dtype=None, stream=None):
    """TR(G) over temporal rows [t0, t1) as a CUDA torch tensor indexed [i_1..i_N]."""
    torch = _torch()
    dtype = dtype or torch.float64
    shape = list(ctx.dims) + [t1 - t0]
    out = torch.empty(list(reversed(shape)), dtype=dtype, device="cuda")
    code = STR_F64 if dtype == torch.float64 else STR_F32
    _check(lib().tr_reconstruct(ctx.handle, int(t0), int(t1), c_void_p(out.data_ptr()), code,
                                _stream_handle(stream)), "tr_reconstruct")
    return out.permute(list(range(len(shape) - 1, -1, -1)))


def _loss_args(cores, X):
    torch = _torch()
    N = len(cores)
    dims = (c_int64 * N)(*[int(G.shape[1]) for G in cores])
    ranks = (c_int * N)(*[int(G.shape[0]) for G in cores])
    dt = {torch.float64: STR_F64, torch.float32: STR_F32}[X.dtype]
    return N, dims, ranks, dt


def tr_masked_loss_fwd(cores_abi, X, mask_bits=None, stream=None):
    """Masked loss 1/2 sum M (X - TR(G))^2; cores_abi are CUDA tensors in the ABI core layout
    (shape (I_n, R_{n+1}, R_n)); returns a 0-dim float64 CUDA tensor."""
    torch = _torch()
    N = len(cores_abi)
    dims = (c_int64 * N)(*[int(G.shape[0]) for G in cores_abi])
    ranks = (c_int * N)(*[int(G.shape[2]) for G in cores_abi])
    dt = {torch.float64: STR_F64, torch.float32: STR_F32}[X.dtype]
    ptrs = (c_void_p * N)(*[G.data_ptr() for G in cores_abi])
    loss = torch.zeros((), dtype=torch.float64, device=X.device)
    _check(lib().tr_masked_loss_fwd(N, dims, ranks, dt, ptrs, c_void_p(X.data_ptr()),
                                    c_void_p(mask_bits.data_ptr()) if mask_bits is not None else None,
                                    c_void_p(loss.data_ptr()), _stream_handle(stream)), "tr_masked_loss_fwd")
    return loss


def tr_masked_loss_bwd(cores_abi, X, mask_bits=None, grad_scale: float = 1.0, stream=None):
    torch = _torch()
    N = len(cores_abi)
    dims = (c_int64 * N)(*[int(G.shape[0]) for G in cores_abi])
    ranks = (c_int * N)(*[int(G.shape[2]) for G in cores_abi])
    dt = {torch.float64: STR_F64, torch.float32: STR_F32}[X.dtype]
    ptrs = (c_void_p * N)(*[G.data_ptr() for G in cores_abi])
    grads = [torch.empty_like(G) for G in cores_abi]
    gptrs = (c_void_p * N)(*[g.data_ptr() for g in grads])
    _check(lib().tr_masked_loss_bwd(N, dims, ranks, dt, ptrs, c_void_p(X.data_ptr()),
                                    c_void_p(mask_bits.data_ptr()) if mask_bits is not None else None,
                                    float(grad_scale), gptrs, _stream_handle(stream)), "tr_masked_loss_bwd")
    return grads


def fma_probe(dtype: str, ctas: int, iters: int, out, stream=None) -> float:
    """Enqueue the library's FMA-rate probe (``str_fma_probe``) writing into the
    CUDA tensor ``out`` (``ctas`` elements of ``dtype``, "f32" or "f64");
    returns the launch's floating-point operations."""
    code = {"f32": STR_F32, "f64": STR_F64}[dtype]
    flop = c_double(0.0)
    _check(lib().str_fma_probe(code, int(ctas), int(iters), c_void_p(out.data_ptr()), byref(flop),
                               _stream_handle(stream)), "str_fma_probe")
    return float(flop.value)


def _make_loss_fn():
    torch = _torch()

    class TRFitLoss(torch.autograd.Function):
        """Masked TR fit loss L = 1/2 sum_i M(i) (X(i) - TR(G)(i))^2.

        Inputs: X (CUDA, i_1-fastest layout), mask bits (int32 CUDA tensor or None)
        and the cores in the ABI layout (CUDA tensors of shape (I_n, R_{n+1}, R_n)).
        The backward is the subchain MTTKRP of the masked residual,
        -(M .* (X - TR(G)))_[n] G^{!=n}_[2], computed by the library; subchains are
        recomputed, nothing but the inputs is saved."""

        @staticmethod
        def forward(ctx, X, mask_bits, *cores):
            ctx.save_for_backward(X, *cores)
            ctx.mask_bits = mask_bits
            return tr_masked_loss_fwd(list(cores), X, mask_bits)

        @staticmethod
        def backward(ctx, g):
            X, *cores = ctx.saved_tensors
            grads = tr_masked_loss_bwd(cores, X, ctx.mask_bits, float(g))
            return (None, None) + tuple(grads)

    return TRFitLoss


def __getattr__(name):
    if name == "TRFitLoss":
        fn = _make_loss_fn()
        globals()["TRFitLoss"] = fn
        return fn
    raise AttributeError(name)
