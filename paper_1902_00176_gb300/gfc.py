"""Python binding of the GFC C ABI (``include/gfc.h``): argument marshalling only.

Every step of the solve runs in the CUDA library ``libgfc.so`` built in-tree
by ``__graft_entry__.build()``; this module only checks tensors, passes their
device pointers and the current torch stream, and maps status codes to
exceptions. If the library is missing it raises: there is no CPU fallback.

Layout: fields are ``[batch, C, H, W]`` contiguous CUDA tensors (a ``[H, W]``
or ``[C, H, W]`` tensor is read as batch 1 / C 1), in float32, float16 or
bfloat16 storage; arithmetic is FP32.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgfc.so")

GFC_F32, GFC_F16, GFC_BF16 = 0, 1, 2
_DTYPES = {torch.float32: GFC_F32, torch.float16: GFC_F16, torch.bfloat16: GFC_BF16}
_STATUS = {0: "GFC_OK", 1: "GFC_ERR_INVALID_ARG", 2: "GFC_ERR_UNSUPPORTED", 3: "GFC_ERR_ALLOC",
           4: "GFC_ERR_CUDA", 5: "GFC_ERR_TIMEOUT"}


class GFCError(RuntimeError):
    """A non-OK gfc_status, with the library's message."""

    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class _Opts(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("C", ctypes.c_int), ("batch", ctypes.c_int),
                ("dtype", ctypes.c_int), ("pad", ctypes.c_int), ("size_policy", ctypes.c_int),
                ("chunk", ctypes.c_int), ("stream", ctypes.c_void_p), ("streams", ctypes.c_int),
                ("column_solver", ctypes.c_int), ("block_items", ctypes.c_int)]


class Item(ctypes.Structure):
    """Mirror of gfc_item: C fields of H x W at `offset` elements into the packed arrays."""
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("C", ctypes.c_int), ("offset", ctypes.c_longlong)]


class _Edit(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("frac", ctypes.c_float), ("ref", ctypes.c_float),
                ("alpha", ctypes.c_float), ("edges", ctypes.c_void_p)]


EDIT_KINDS = {"none": 0, "threshold": 1, "merge": 2}


class TuneResult(ctypes.Structure):
    """Mirror of gfc_tune_result."""
    _fields_ = [("column_solver", ctypes.c_int), ("block_items", ctypes.c_int), ("chunk", ctypes.c_int),
                ("streams", ctypes.c_int), ("rag_streams", ctypes.c_int), ("ms", ctypes.c_double),
                ("candidates", ctypes.c_int), ("from_cache", ctypes.c_int), ("l2_resident", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Profile(ctypes.Structure):
    """Mirror of gfc_profile: per-pass device time (ms) and launch counts."""
    _fields_ = [("pass_ms", ctypes.c_double * 4), ("launches", ctypes.c_long * 4), ("calls", ctypes.c_long),
                ("dropped", ctypes.c_long)]

    def as_dict(self):
        return {"pass_ms": list(self.pass_ms), "launches": list(self.launches), "calls": self.calls,
                "dropped": self.dropped}


_lib = None
_lib_lock = threading.Lock()

# (name, argtypes) of every function declared in include/gfc.h
_SIGNATURES = {
    "gfc_padded_size": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
    "gfc_row_lengths": [ctypes.POINTER(ctypes.c_int), ctypes.c_int],
    "gfc_plan_l2_resident": [ctypes.c_void_p],
    "gfc_plan_create": [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                        ctypes.c_int],
    "gfc_plan_create_ex": [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(_Opts)],
    "gfc_plan_create_ragged": [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p, ctypes.c_int],
    "gfc_plan_set_stream": [ctypes.c_void_p, ctypes.c_void_p],
    "gfc_plan_padded_size": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                             ctypes.POINTER(ctypes.c_int)],
    "gfc_plan_copy_green": [ctypes.c_void_p, ctypes.c_void_p],
    "gfc_solve_from_gradient": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "gfc_solve_edited": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(_Edit), ctypes.c_void_p],
    "gfc_solve_corrected": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(_Edit),
                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "gfc_solve_from_laplacian": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "gfc_backward": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "gfc_fft_c2c": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "gfc_solve_from_gradient_host": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "gfc_plan_set_profiling": [ctypes.c_void_p, ctypes.c_int],
    "gfc_plan_get_profile": [ctypes.c_void_p, ctypes.POINTER(Profile), ctypes.c_int],
    "gfc_solve_from_gradient_noalloc": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p],
    "gfc_field_stats": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "gfc_color_correct": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "gfc_gradient_threshold": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float, ctypes.c_float,
                               ctypes.c_void_p, ctypes.c_void_p],
    "gfc_gradient_merge": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float,
                           ctypes.c_void_p, ctypes.c_void_p],
    "gfc_boundary_offset": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p],
    "gfc_graph_create": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                         ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)],
    "gfc_graph_launch": [ctypes.c_void_p, ctypes.c_void_p],
    "gfc_graph_destroy": [ctypes.c_void_p],
    "gfc_plan_selftest_wait": [ctypes.c_void_p, ctypes.c_int],
    "gfc_plan_sync": [ctypes.c_void_p],
    "gfc_destroy": [ctypes.c_void_p],
    "gfc_plan_autotune": [ctypes.c_void_p, ctypes.c_char_p, ctypes.POINTER(TuneResult)],
    "gfc_plan_tune_key": [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int],
    "gfc_tune_cache_get": [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int],
    "gfc_tune_cache_put": [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_char_p],
    "gfc_last_error": [],
    "gfc_status_string": [ctypes.c_int],
}


def lib() -> ctypes.CDLL:
    """Load ``libgfc.so`` (raises if it has not been built)."""
    global _lib
    with _lib_lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"GFC CUDA library not built ({LIB_PATH} missing): "
                                   "run __graft_entry__.build() first")
            L = ctypes.CDLL(LIB_PATH)
            for name, argt in _SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = argt
                fn.restype = ctypes.c_char_p if name in ("gfc_last_error", "gfc_status_string") else ctypes.c_int
            _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        raise GFCError(status, lib().gfc_last_error().decode(errors="replace"))


def padded_size(H: int, W: int, pad: int = 4, exact: bool = False):
    """(M, N) of the padded torus for an H x W image (host-only, no GPU needed)."""
    M, N = ctypes.c_int(), ctypes.c_int()
    _check(lib().gfc_padded_size(H, W, pad, 1 if exact else 0, ctypes.byref(M), ctypes.byref(N)))
    return M.value, N.value


def row_lengths():
    """Row lengths N with register-resident row passes, ascending (host-only)."""
    n = lib().gfc_row_lengths(None, 0)
    buf = (ctypes.c_int * n)()
    lib().gfc_row_lengths(buf, n)
    return list(buf)


def tune_cache_get(path: str, key: str):
    """The cached tuning value for ``key`` in the cache file, or None."""
    buf = ctypes.create_string_buffer(512)
    r = lib().gfc_tune_cache_get(path.encode(), key.encode(), buf, len(buf))
    if r < 0:
        raise GFCError(1, lib().gfc_last_error().decode(errors="replace"))
    return buf.value.decode() if r == 1 else None


def tune_cache_put(path: str, key: str, value: str):
    _check(lib().gfc_tune_cache_put(path.encode(), key.encode(), value.encode()))


def _autotune(handle, device, bind, cache):
    r = TuneResult()
    bind()
    with torch.cuda.device(device):
        _check(lib().gfc_plan_autotune(handle, cache.encode() if cache else None, ctypes.byref(r)))
    return r.as_dict()


def _tune_key(handle):
    buf = ctypes.create_string_buffer(1024)
    _check(lib().gfc_plan_tune_key(handle, buf, len(buf)))
    return buf.value.decode()


def _stream_ptr(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _as_bchw(t: torch.Tensor) -> torch.Tensor:
    if t.dim() == 2:
        return t.view(1, 1, *t.shape)
    if t.dim() == 3:
        return t.view(1, *t.shape)
    if t.dim() == 4:
        return t
    raise ValueError(f"expected a [H,W], [C,H,W] or [B,C,H,W] tensor, got shape {tuple(t.shape)}")


class Plan:
    """A GFC plan: Green spectrum, transform tables and scratch for one problem shape."""

    def __init__(self, H: int, W: int, C: int = 1, batch: int = 1, dtype=torch.float32, pad: int = 4,
                 chunk: int = 0, device=None, streams: int = 0, exact: bool = False, column_fft: bool = False,
                 block_items: bool = False):
        """``exact=True`` solves on Algorithm A's own padded size (H + 2p) x (W + 2p)
        instead of the next even 7-smooth size. ``column_fft=True`` applies the column
        direction of the Green multiply by column FFTs instead of the recursive
        (tridiagonal) column solve (register-resident sizes; same operator)."""
        if dtype not in _DTYPES:
            raise ValueError(f"unsupported dtype {dtype}")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        self.H, self.W, self.C, self.batch, self.dtype = H, W, C, batch, dtype
        o = _Opts(H, W, C, batch, _DTYPES[dtype], pad, 1 if exact else 0, chunk, None, streams,
                  1 if column_fft else 0, 1 if block_items else 0)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib().gfc_plan_create_ex(ctypes.byref(h), ctypes.byref(o)))
        self._h = h
        M, N, p = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().gfc_plan_padded_size(h, ctypes.byref(M), ctypes.byref(N), ctypes.byref(p)))
        self.M, self.N, self.pad = M.value, N.value, p.value

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().gfc_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _bind_stream(self):
        _check(lib().gfc_plan_set_stream(self._h, ctypes.c_void_p(_stream_ptr(self.device))))

    def _check_field(self, t: torch.Tensor, name: str) -> torch.Tensor:
        t = _as_bchw(t)
        if not t.is_cuda or t.device != self.device:
            raise ValueError(f"{name} must be a CUDA tensor on {self.device}")
        if t.dtype != self.dtype:
            raise ValueError(f"{name} has dtype {t.dtype}, plan expects {self.dtype}")
        if tuple(t.shape) != (self.batch, self.C, self.H, self.W):
            raise ValueError(f"{name} has shape {tuple(t.shape)}, plan expects "
                             f"{(self.batch, self.C, self.H, self.W)}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        return t

    def _empty(self):
        return torch.empty((self.batch, self.C, self.H, self.W), dtype=self.dtype, device=self.device)

    def solve_from_gradient(self, gx, gy, out=None):
        gx, gy = self._check_field(gx, "gx"), self._check_field(gy, "gy")
        out = self._empty() if out is None else self._check_field(out, "out")
        self._bind_stream()
        _check(lib().gfc_solve_from_gradient(self._h, gx.data_ptr(), gy.data_ptr(), out.data_ptr()))
        return out

    def solve_edited(self, gx, gy, edit="threshold", frac=0.1, ref=0.0, alpha=0.5, edges=None, out=None):
        """Solve from the gradient with an edit applied as it is loaded: ``edit`` is
        "threshold" (Sec. 3.2.3: |E| < frac * r set to 0) or "merge" (Eq. 26 with
        the edge map ``edges`` and weight ``alpha``)."""
        gx, gy = self._check_field(gx, "gx"), self._check_field(gy, "gy")
        if edit not in EDIT_KINDS:
            raise ValueError(f"unknown edit {edit!r}")
        eptr = None
        if edit == "merge":
            if edges is None:
                raise ValueError("merge needs an edge map")
            edges = self._check_field(edges, "edges")
            eptr = edges.data_ptr()
        out = self._empty() if out is None else self._check_field(out, "out")
        e = _Edit(EDIT_KINDS[edit], float(frac), float(ref), float(alpha), eptr)
        self._bind_stream()
        _check(lib().gfc_solve_edited(self._h, gx.data_ptr(), gy.data_ptr(), ctypes.byref(e), out.data_ptr()))
        return out

    def solve_corrected(self, gx, gy, ref_mean, ref_std, edit="none", frac=0.1, ref=0.0, alpha=0.5, edges=None,
                        out=None):
        """Edit (optional), solve and colour-correct (Eq. 25) in one call: each field is
        rescaled to ``ref_mean`` / ``ref_std`` ([batch, C] float32, e.g. from field_stats
        of the original image)."""
        gx, gy = self._check_field(gx, "gx"), self._check_field(gy, "gy")
        ref_mean, ref_std = self._stats_tensor(ref_mean, "ref_mean"), self._stats_tensor(ref_std, "ref_std")
        if edit not in EDIT_KINDS:
            raise ValueError(f"unknown edit {edit!r}")
        eptr = None
        if edit == "merge":
            if edges is None:
                raise ValueError("merge needs an edge map")
            edges = self._check_field(edges, "edges")
            eptr = edges.data_ptr()
        out = self._empty() if out is None else self._check_field(out, "out")
        e = _Edit(EDIT_KINDS[edit], float(frac), float(ref), float(alpha), eptr)
        self._bind_stream()
        _check(lib().gfc_solve_corrected(self._h, gx.data_ptr(), gy.data_ptr(), ctypes.byref(e), ref_mean.data_ptr(),
                                         ref_std.data_ptr(), out.data_ptr()))
        return out

    def solve_from_laplacian(self, lap, out=None):
        lap = self._check_field(lap, "lap")
        out = self._empty() if out is None else self._check_field(out, "out")
        self._bind_stream()
        _check(lib().gfc_solve_from_laplacian(self._h, lap.data_ptr(), out.data_ptr()))
        return out

    def backward(self, grad_out, grad_gx=None, grad_gy=None):
        grad_out = self._check_field(grad_out, "grad_out")
        grad_gx = self._empty() if grad_gx is None else self._check_field(grad_gx, "grad_gx")
        grad_gy = self._empty() if grad_gy is None else self._check_field(grad_gy, "grad_gy")
        self._bind_stream()
        _check(lib().gfc_backward(self._h, grad_out.data_ptr(), grad_gx.data_ptr(), grad_gy.data_ptr()))
        return grad_gx, grad_gy

    def solve_from_gradient_host(self, gx, gy, out):
        """Host-memory solve through the C ABI: CPU tensors (pinned for overlap), result in ``out``.
        Asynchronous on the current stream; synchronize before reading ``out``."""
        for t, n in ((gx, "gx"), (gy, "gy"), (out, "out")):
            if t.is_cuda or t.dtype != self.dtype or not t.is_contiguous() or \
                    t.numel() != self.batch * self.C * self.H * self.W:
                raise ValueError(f"{n} must be a contiguous CPU tensor of {self.batch}x{self.C}x{self.H}x{self.W} "
                                 f"{self.dtype}")
        self._bind_stream()
        _check(lib().gfc_solve_from_gradient_host(self._h, gx.data_ptr(), gy.data_ptr(), out.data_ptr()))
        return out

    # ---- gradient-domain editing (Sec. 2.3.2, Sec. 3.2) ----
    def _stats_tensor(self, t, name):
        if t is None:
            return torch.empty((self.batch, self.C), dtype=torch.float32, device=self.device)
        if not t.is_cuda or t.device != self.device or t.dtype != torch.float32 or not t.is_contiguous() or \
                t.numel() != self.batch * self.C:
            raise ValueError(f"{name} must be a contiguous float32 CUDA tensor of {self.batch * self.C} values")
        return t

    def field_stats(self, x, mean=None, std=None):
        """Per-field mean and population standard deviation, each [batch, C] float32."""
        x = self._check_field(x, "x")
        mean, std = self._stats_tensor(mean, "mean"), self._stats_tensor(std, "std")
        self._bind_stream()
        _check(lib().gfc_field_stats(self._h, x.data_ptr(), mean.data_ptr(), std.data_ptr()))
        return mean, std

    def color_correct(self, out, ref_mean, ref_std):
        """Eq. 25 in place on ``out``: rescale each field to the original's mean and contrast."""
        out = self._check_field(out, "out")
        ref_mean, ref_std = self._stats_tensor(ref_mean, "ref_mean"), self._stats_tensor(ref_std, "ref_std")
        self._bind_stream()
        _check(lib().gfc_color_correct(self._h, out.data_ptr(), ref_mean.data_ptr(), ref_std.data_ptr()))
        return out

    def gradient_threshold(self, gx, gy, frac, ref=0.0, gx_out=None, gy_out=None):
        """Zero the gradient where |E| < frac * r (r = ref if ref > 0, else the field's largest |E|)."""
        gx, gy = self._check_field(gx, "gx"), self._check_field(gy, "gy")
        gx_out = self._empty() if gx_out is None else self._check_field(gx_out, "gx_out")
        gy_out = self._empty() if gy_out is None else self._check_field(gy_out, "gy_out")
        self._bind_stream()
        _check(lib().gfc_gradient_threshold(self._h, gx.data_ptr(), gy.data_ptr(), float(frac), float(ref),
                                            gx_out.data_ptr(), gy_out.data_ptr()))
        return gx_out, gy_out

    def gradient_merge(self, gx, gy, edges, alpha, gx_out=None, gy_out=None):
        """Eq. 26: |Ep| = |E|^(1-alpha) C^alpha with the orientation of E kept."""
        gx, gy = self._check_field(gx, "gx"), self._check_field(gy, "gy")
        edges = self._check_field(edges, "edges")
        gx_out = self._empty() if gx_out is None else self._check_field(gx_out, "gx_out")
        gy_out = self._empty() if gy_out is None else self._check_field(gy_out, "gy_out")
        self._bind_stream()
        _check(lib().gfc_gradient_merge(self._h, gx.data_ptr(), gy.data_ptr(), edges.data_ptr(), float(alpha),
                                        gx_out.data_ptr(), gy_out.data_ptr()))
        return gx_out, gy_out

    def boundary_offset(self, out, ring=3, inner=None):
        """Sec. 2.3.2: subtract the ring's mean from a solved field and crop the ring."""
        out = self._check_field(out, "out")
        shape = (self.batch, self.C, self.H - 2 * ring, self.W - 2 * ring)
        if inner is None:
            inner = torch.empty(shape, dtype=self.dtype, device=self.device)
        elif tuple(inner.shape) != shape or inner.dtype != self.dtype or not inner.is_contiguous() or \
                inner.device != self.device:
            raise ValueError(f"inner must be a contiguous {self.dtype} tensor of shape {shape} on {self.device}")
        self._bind_stream()
        _check(lib().gfc_boundary_offset(self._h, out.data_ptr(), int(ring), inner.data_ptr()))
        return inner

    def set_profiling(self, enable: bool = True):
        _check(lib().gfc_plan_set_profiling(self._h, 1 if enable else 0))

    def profile(self, reset: bool = True) -> dict:
        """Synchronize and return accumulated per-pass times and launch counts."""
        pr = Profile()
        self._bind_stream()
        _check(lib().gfc_plan_get_profile(self._h, ctypes.byref(pr), 1 if reset else 0))
        return pr.as_dict()

    def autotune(self, cache=None) -> dict:
        """Time the plan's candidate splits and keep the fastest (gfc_plan_autotune);
        ``cache`` is an optional path of the tuning cache file."""
        return _autotune(self._h, self.device, self._bind_stream, cache)

    def tune_key(self) -> str:
        return _tune_key(self._h)

    @property
    def l2_resident(self) -> bool:
        """Whether the plan keeps its spectrum hand-off in L2 (gfc_plan_l2_resident)."""
        return lib().gfc_plan_l2_resident(self._h) == 1

    def green(self):
        """The plan's FP32 Green spectrum, M x (N/2+1), as a CPU tensor (1/(MN) folded in)."""
        g = torch.empty((self.M, self.N // 2 + 1), dtype=torch.float32)
        self._bind_stream()
        _check(lib().gfc_plan_copy_green(self._h, g.data_ptr()))
        return g

    def sync(self):
        _check(lib().gfc_plan_sync(self._h))

    def selftest_wait(self, timeout_ms: int = 50):
        """Queue a device wait that runs out after ``timeout_ms``; the next ``sync``
        raises with GFC_ERR_TIMEOUT (checks the bounded-wait failure path)."""
        self._bind_stream()
        _check(lib().gfc_plan_selftest_wait(self._h, int(timeout_ms)))


_plans: dict = {}


def get_plan(H, W, C, batch, dtype, device) -> Plan:
    """Cached plan for a problem shape on a device."""
    dev = torch.device(device)
    key = (H, W, C, batch, dtype, dev.index)
    p = _plans.get(key)
    if p is None:
        p = Plan(H, W, C, batch, dtype, device=dev)
        _plans[key] = p
    return p


def solve(gx: torch.Tensor, gy: torch.Tensor) -> torch.Tensor:
    """GFC solve from a gradient field; returns a tensor shaped like gx."""
    b = _as_bchw(gx)
    p = get_plan(b.shape[2], b.shape[3], b.shape[1], b.shape[0], gx.dtype, gx.device)
    return p.solve_from_gradient(gx, gy).view(gx.shape)


def solve_laplacian(lap: torch.Tensor) -> torch.Tensor:
    """GFC solve from a Laplacian; returns a tensor shaped like lap."""
    b = _as_bchw(lap)
    p = get_plan(b.shape[2], b.shape[3], b.shape[1], b.shape[0], lap.dtype, lap.device)
    return p.solve_from_laplacian(lap).view(lap.shape)


def solve_noalloc(gx: torch.Tensor, gy: torch.Tensor, out: torch.Tensor) -> torch.Tensor:
    """FP32 solve through the allocation-free entry point (no plan; ``out`` preallocated by the caller).

    The three tensors must live on one CUDA device; the call runs with that
    device current and on its current torch stream."""
    b = _as_bchw(gx)
    for t in (gx, gy, out):
        if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() or t.shape != gx.shape:
            raise ValueError("gx, gy, out must be contiguous float32 CUDA tensors of one shape")
    if gy.device != gx.device or out.device != gx.device:
        raise ValueError(f"gx, gy, out must be on one device (got {gx.device}, {gy.device}, {out.device})")
    with torch.cuda.device(gx.device):
        _check(lib().gfc_solve_from_gradient_noalloc(b.shape[2], b.shape[3], b.shape[0] * b.shape[1],
                                                     gx.data_ptr(), gy.data_ptr(), out.data_ptr(),
                                                     ctypes.c_void_p(_stream_ptr(gx.device))))
    return out


def fft_c2c(x: torch.Tensor, inverse: bool = False) -> torch.Tensor:
    """Batched complex transform along the last axis with the library's own FFT engine."""
    if x.dtype != torch.complex64 or not x.is_cuda:
        raise ValueError("fft_c2c expects a complex64 CUDA tensor")
    x = x.contiguous()
    out = torch.empty_like(x)
    n = x.shape[-1]
    count = x.numel() // n if n else 0
    _check(lib().gfc_fft_c2c(n, count, 1 if inverse else -1, x.data_ptr(), out.data_ptr(),
                             ctypes.c_void_p(_stream_ptr(x.device))))
    return out


class GFCFunction(torch.autograd.Function):
    """GFC as a differentiable layer: forward solves from (gx, gy), backward runs the
    hand-written adjoint kernels. Nothing but the plan is saved between the two."""

    @staticmethod
    def forward(ctx, gx, gy):
        b = _as_bchw(gx)
        p = get_plan(b.shape[2], b.shape[3], b.shape[1], b.shape[0], gx.dtype, gx.device)
        ctx.plan = p
        ctx.shape = gx.shape
        return p.solve_from_gradient(gx.contiguous(), gy.contiguous()).view(gx.shape)

    @staticmethod
    def backward(ctx, grad_out):
        ggx, ggy = ctx.plan.backward(grad_out.contiguous())
        return ggx.view(ctx.shape), ggy.view(ctx.shape)


def gfc_layer(gx: torch.Tensor, gy: torch.Tensor) -> torch.Tensor:
    """Differentiable GFC solve (see GFCFunction)."""
    return GFCFunction.apply(gx, gy)


class RaggedPlan:
    """A plan for a ragged batch: items of different sizes packed into one flat array.

    ``items`` is a list of ``(C, H, W)``; item i occupies ``C*H*W`` contiguous
    elements ([C, H, W]) starting at ``offsets[i]`` of the packed arrays.
    """

    def __init__(self, items, dtype=torch.float32, device=None):
        if dtype not in _DTYPES:
            raise ValueError(f"unsupported dtype {dtype}")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        self.items = [tuple(int(v) for v in it) for it in items]
        self.dtype = dtype
        self.offsets, off = [], 0
        for (C, H, W) in self.items:
            self.offsets.append(off)
            off += C * H * W
            off = (off + 7) // 8 * 8  # keep every item 16-byte aligned in any dtype
        self.total = off
        arr = (Item * len(self.items))(*[Item(H, W, C, o) for (C, H, W), o in zip(self.items, self.offsets)])
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib().gfc_plan_create_ragged(ctypes.byref(h), len(self.items), ctypes.cast(arr, ctypes.c_void_p),
                                                _DTYPES[dtype]))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().gfc_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def empty(self):
        return torch.zeros(self.total, dtype=self.dtype, device=self.device)

    def pack(self, tensors):
        """Pack a list of [C, H, W] tensors (one per item) into a flat array."""
        flat = self.empty()
        for t, (C, H, W), o in zip(tensors, self.items, self.offsets):
            flat[o:o + C * H * W] = t.reshape(-1).to(self.device, self.dtype)
        return flat

    def unpack(self, flat):
        return [flat[o:o + C * H * W].view(C, H, W) for (C, H, W), o in zip(self.items, self.offsets)]

    def autotune(self, cache=None) -> dict:
        """Time 1, 2, 4 and 8 internal streams for the per-item sub-plans and keep the fastest."""
        return _autotune(self._h, self.device, self._bind_stream, cache)

    def tune_key(self) -> str:
        return _tune_key(self._h)

    def _check_flat(self, t, name):
        if not t.is_cuda or t.device != self.device or t.dtype != self.dtype or t.numel() != self.total \
                or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {self.dtype} CUDA tensor of {self.total} elements")
        return t

    def _bind_stream(self):
        _check(lib().gfc_plan_set_stream(self._h, ctypes.c_void_p(_stream_ptr(self.device))))

    def solve_from_gradient(self, gx, gy, out=None):
        gx, gy = self._check_flat(gx, "gx"), self._check_flat(gy, "gy")
        out = self.empty() if out is None else self._check_flat(out, "out")
        self._bind_stream()
        _check(lib().gfc_solve_from_gradient(self._h, gx.data_ptr(), gy.data_ptr(), out.data_ptr()))
        return out

    def solve_from_laplacian(self, lap, out=None):
        lap = self._check_flat(lap, "lap")
        out = self.empty() if out is None else self._check_flat(out, "out")
        self._bind_stream()
        _check(lib().gfc_solve_from_laplacian(self._h, lap.data_ptr(), out.data_ptr()))
        return out

    def backward(self, grad_out, grad_gx=None, grad_gy=None):
        grad_out = self._check_flat(grad_out, "grad_out")
        grad_gx = self.empty() if grad_gx is None else self._check_flat(grad_gx, "grad_gx")
        grad_gy = self.empty() if grad_gy is None else self._check_flat(grad_gy, "grad_gy")
        self._bind_stream()
        _check(lib().gfc_backward(self._h, grad_out.data_ptr(), grad_gx.data_ptr(), grad_gy.data_ptr()))
        return grad_gx, grad_gy


class Graph:
    """A captured solve call (see gfc_graph_create): ``launch()`` replays it with one launch
    on the current stream, reading and writing the buffers given at capture."""

    OPS = {"gradient": 0, "laplacian": 1, "backward": 2}

    def __init__(self, plan, op, in0, in1=None, out0=None, out1=None):
        self.plan = plan
        self._keep = (in0, in1, out0, out1)
        ptr = lambda t: None if t is None else t.data_ptr()
        plan._bind_stream()
        h = ctypes.c_void_p()
        _check(lib().gfc_graph_create(plan.handle if hasattr(plan, "handle") else plan._h, self.OPS[op], ptr(in0),
                                      ptr(in1), ptr(out0), ptr(out1), ctypes.byref(h)))
        self._h = h
        self.device = plan.device

    def launch(self):
        _check(lib().gfc_graph_launch(self._h, ctypes.c_void_p(_stream_ptr(self.device))))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().gfc_graph_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
