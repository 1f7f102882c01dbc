"""ctypes binding of libfdkod.so (include/fdkod.h), argument marshalling only.

Functions carry the C names; ``Plan`` bundles them for a plan's lifetime.
Tensors are torch CUDA tensors; the stream defaults to torch's current
stream on the tensor's device.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(HERE, "libfdkod.so")
_lock = threading.Lock()
_lib = None

FDKOD_F32, FDKOD_BF16, FDKOD_F16 = 0, 1, 2
_DTYPES = {"f32": FDKOD_F32, "bf16": FDKOD_BF16, "f16": FDKOD_F16}


class FdkodError(RuntimeError):
    def __init__(self, status: int, what: str):
        msg = _load().fdkod_strerror(status).decode() if _lib is not None else str(status)
        super().__init__(f"{what}: {msg} ({status})")
        self.status = status


class Geometry(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double), ("N", ctypes.c_int32), ("Nu", ctypes.c_int32), ("Nv", ctypes.c_int32),
                ("P", ctypes.c_int32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("s", ctypes.c_int32), ("D", ctypes.c_int32), ("Pd", ctypes.c_int32), ("n_squares", ctypes.c_int32),
                ("T_stride", ctypes.c_int32), ("fft_length", ctypes.c_int32), ("decomposed_elems", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64)]


def lib_path() -> str:
    return _LIB_PATH


def load():
    """Load libfdkod.so (built by __graft_entry__.build()); raise if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise RuntimeError(f"{_LIB_PATH} is not built; the CUDA library is required (no CPU fallback)")
            lib = ctypes.CDLL(_LIB_PATH)
            vp, i, u = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
            sig = {
                "fdkod_plan": (i, [ctypes.POINTER(Geometry), i, i, i, ctypes.POINTER(vp)]),
                "fdkod_plan_ex": (i, [ctypes.POINTER(Geometry), i, i, i, i, ctypes.POINTER(vp)]),
                "fdkod_slab_rows": (i, [vp, i, i, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
                "fdkod_filter_rows": (i, [vp, vp, i, i, vp, u]),
                "fdkod_backproject_slab": (i, [vp, vp, i, i, vp, i, i, vp, u]),
                "fdkod_destroy": (None, [vp]),
                "fdkod_get_info": (i, [vp, ctypes.POINTER(PlanInfo)]),
                "fdkod_filter": (i, [vp, vp, vp, u]),
                "fdkod_backproject": (i, [vp, vp, vp, u]),
                "fdk_backproject_plain": (i, [vp, vp, vp, u]),
                "fdkod_decompose": (i, [vp, vp, vp, u]),
                "fdkod_backproject_decomposed": (i, [vp, vp, vp, u]),
                "fdkod_compute_bounds": (i, [vp, u]),
                "fdkod_backproject_noalloc": (i, [ctypes.POINTER(Geometry), i, i, vp, vp, u]),
                "fdkod_noalloc_device_status": (i, [u]),
                "fdkod_set_test_fault": (i, [vp, i, ctypes.c_int64]),
                "fdkod_get_bounds": (i, [vp, vp, vp, vp, vp, vp, vp]),
                "fdkod_last_device_status": (i, [vp, u]),
                "fdkod_strerror": (ctypes.c_char_p, [i]),
                "fdkod_set_decimation_taps": (i, [vp, vp, i]),
                "fdkod_get_decimation_taps": (i, [vp, vp, i]),
                "fdkod_sinc_taps": (i, [i, i, vp]),
                "fdkod_reconstruct_slabs": (i, [vp, vp, vp, i, u, ctypes.POINTER(ctypes.c_int64)]),
                "fdkod_reconstruct": (i, [vp, vp, vp, u]),
                "fdkod_set_decimation_net": (i, [vp, vp, i]),
                "fdkod_get_decimation_net": (i, [vp, vp, i]),
                "fdkod_net_adjoint": (i, [vp, vp, vp, i, vp, vp, u]),
                "fdkod_net_backward": (i, [vp, vp, vp, vp, i, i, vp, u]),
                "fdkod_batch_create": (i, [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), i,
                                           ctypes.POINTER(vp)]),
                "fdkod_batch_backproject": (i, [vp, u]),
                "fdkod_batch_destroy": (None, [vp]),
                "fdkod_set_tile": (i, [vp, i]),
                "fdkod_get_tile": (i, [vp, ctypes.POINTER(i), ctypes.POINTER(i)]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


_load = load


def _check(rc: int, what: str):
    if rc != 0:
        raise FdkodError(rc, what)


def _stream(t, stream):
    if stream is not None:
        return int(stream)
    import torch
    return int(torch.cuda.current_stream(t.device).cuda_stream)


def _dev_ptr(t, what):
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{what} must be a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _expect(t, shape, dtype, what, at_least=False):
    """The checks the C interface cannot make (it takes bare pointers): t is
    a contiguous CUDA tensor of `dtype` whose shape is `shape` (None entries
    match any extent), or, with at_least, a flat buffer of at least
    `shape` elements.  Raises ValueError."""
    if not getattr(t, "is_cuda", False) or not t.is_contiguous():
        raise ValueError(f"{what} must be a contiguous CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{what} must be {dtype}, not {t.dtype}")
    if at_least:
        if t.numel() < int(shape):
            raise ValueError(f"{what} holds {t.numel()} elements, needs {int(shape)}")
    elif len(t.shape) != len(shape) or any(e is not None and int(g) != int(e) for g, e in zip(t.shape, shape)):
        raise ValueError(f"{what} must have shape {tuple(shape)}, not {tuple(t.shape)}")
    return t


# ---- C-named functions -------------------------------------------------------

FDKOD_PLAN_NO_WORKSPACE = 1
FDKOD_PLAN_SINC_TAPS = 2
FDKOD_NET_SIZE = 1440


def fdkod_plan(R: float, N: int, Nu: int, Nv: int, P: int, s: int, D: int, qtype: int = FDKOD_F32,
               flags: int = 0) -> int:
    g = Geometry(float(R), int(N), int(Nu), int(Nv), int(P))
    out = ctypes.c_void_p()
    _check(load().fdkod_plan_ex(ctypes.byref(g), int(s), int(D), int(qtype), int(flags), ctypes.byref(out)),
           "fdkod_plan")
    return out.value


def fdkod_filter(plan: int, proj, Q, stream=None) -> None:
    _check(load().fdkod_filter(plan, _dev_ptr(proj, "proj"), _dev_ptr(Q, "Q"), _stream(proj, stream)),
           "fdkod_filter")


def fdkod_backproject(plan: int, Q, vol, stream=None) -> None:
    _check(load().fdkod_backproject(plan, _dev_ptr(Q, "Q"), _dev_ptr(vol, "vol"), _stream(Q, stream)),
           "fdkod_backproject")


def fdk_backproject_plain(plan: int, Q, vol, stream=None) -> None:
    _check(load().fdk_backproject_plain(plan, _dev_ptr(Q, "Q"), _dev_ptr(vol, "vol"), _stream(Q, stream)),
           "fdk_backproject_plain")


def fdkod_decompose(plan: int, Q, out, stream=None) -> None:
    _check(load().fdkod_decompose(plan, _dev_ptr(Q, "Q"), _dev_ptr(out, "out"), _stream(Q, stream)),
           "fdkod_decompose")


def fdkod_backproject_decomposed(plan: int, S, vol, stream=None) -> None:
    _check(load().fdkod_backproject_decomposed(plan, _dev_ptr(S, "S"), _dev_ptr(vol, "vol"), _stream(S, stream)),
           "fdkod_backproject_decomposed")


def fdkod_compute_bounds(plan: int, stream) -> None:
    _check(load().fdkod_compute_bounds(plan, int(stream)), "fdkod_compute_bounds")


def fdkod_backproject_noalloc(R: float, N: int, Nu: int, Nv: int, P: int, s: int, D: int, Q, vol,
                              stream=None) -> None:
    """FDK-OD backprojection without any allocation (scratch in the library's
    fixed device array); Q float32 [P][Nv][Nu], vol float32 [N][N][N]."""
    import torch
    _expect(Q, (P, Nv, Nu), torch.float32, "Q")
    _expect(vol, (N, N, N), torch.float32, "vol")
    g = Geometry(float(R), int(N), int(Nu), int(Nv), int(P))
    _check(load().fdkod_backproject_noalloc(ctypes.byref(g), int(s), int(D), _dev_ptr(Q, "Q"), _dev_ptr(vol, "vol"),
                                            _stream(Q, stream)), "fdkod_backproject_noalloc")


def fdkod_noalloc_device_status(stream=None) -> int:
    """Status of the last fdkod_backproject_noalloc call on the current
    device (read and cleared after the stream's work): 0, -5 (a bounded wait
    gave up) or -6 (a window or the shifted-row width bound was too small)."""
    import torch
    st = int(torch.cuda.current_stream().cuda_stream) if stream is None else int(stream)
    return int(load().fdkod_noalloc_device_status(st))


FDKOD_TEST_NONE, FDKOD_TEST_SKIP_COPY, FDKOD_TEST_SMALL_WINDOW = 0, 1, 2


def fdkod_set_test_fault(plan: int, kind: int, wait_ns: int = 0) -> None:
    """Test hook of the backprojection's failure paths (see include/fdkod.h)."""
    _check(load().fdkod_set_test_fault(plan, int(kind), int(wait_ns)), "fdkod_set_test_fault")


def fdkod_get_bounds(plan: int, n_squares: int, P: int) -> dict:
    lo = np.empty((n_squares, P), np.int32)
    hi = np.empty((n_squares, P), np.int32)
    crop = np.empty((n_squares, P), np.int32)
    phi = np.empty((n_squares, P), np.float64)
    w0 = np.empty(n_squares, np.int32)
    T = np.empty(n_squares, np.int32)
    p = [ctypes.c_void_p(a.ctypes.data) for a in (lo, hi, crop, phi, w0, T)]
    _check(load().fdkod_get_bounds(plan, *p), "fdkod_get_bounds")
    return {"lo": lo, "hi": hi, "crop": crop, "phi": phi, "w0": w0, "T": T}


def fdkod_sinc_taps(D: int, H: int = 2) -> np.ndarray:
    """The library's Hann-windowed sinc taps h[|i|], |i| < H D (host only)."""
    h = np.empty(max(1, H * D), np.float64)
    _check(load().fdkod_sinc_taps(int(D), int(H), ctypes.c_void_p(h.ctypes.data)), "fdkod_sinc_taps")
    return h


def fdkod_set_decimation_taps(plan: int, taps) -> None:
    h = np.ascontiguousarray(taps, dtype=np.float64).reshape(-1)
    _check(load().fdkod_set_decimation_taps(plan, ctypes.c_void_p(h.ctypes.data), h.size),
           "fdkod_set_decimation_taps")


def fdkod_get_decimation_taps(plan: int) -> np.ndarray:
    n = load().fdkod_get_decimation_taps(plan, None, 0)
    _check(min(n, 0), "fdkod_get_decimation_taps")
    h = np.empty(n, np.float64)
    load().fdkod_get_decimation_taps(plan, ctypes.c_void_p(h.ctypes.data), n)
    return h


def fdkod_set_decimation_net(plan: int, w) -> None:
    """Set (w: FDKOD_NET_SIZE values) or remove (w None) the learned decimation."""
    if w is None:
        _check(load().fdkod_set_decimation_net(plan, None, 0), "fdkod_set_decimation_net")
        return
    a = np.ascontiguousarray(w, dtype=np.float32).reshape(-1)
    _check(load().fdkod_set_decimation_net(plan, ctypes.c_void_p(a.ctypes.data), a.size),
           "fdkod_set_decimation_net")


def fdkod_get_decimation_net(plan: int):
    """The plan's BF16-rounded net weights (float32), or None without a net."""
    a = np.empty(FDKOD_NET_SIZE, np.float32)
    n = load().fdkod_get_decimation_net(plan, ctypes.c_void_p(a.ctypes.data), a.size)
    _check(min(n, 0), "fdkod_get_decimation_net")
    return a if n > 0 else None


def fdkod_net_adjoint(plan: int, vol_slice, ref_slice, z: int, dS, sq_err, stream=None) -> None:
    _check(load().fdkod_net_adjoint(plan, _dev_ptr(vol_slice, "vol_slice"), _dev_ptr(ref_slice, "ref_slice"), int(z),
                                    _dev_ptr(dS, "dS"), _dev_ptr(sq_err, "sq_err"), _stream(dS, stream)),
           "fdkod_net_adjoint")


def fdkod_net_backward(plan: int, Q, w, dS, row_lo: int, row_hi: int, dW, stream=None) -> None:
    _check(load().fdkod_net_backward(plan, _dev_ptr(Q, "Q"), _dev_ptr(w, "w"), _dev_ptr(dS, "dS"), int(row_lo),
                                     int(row_hi), _dev_ptr(dW, "dW"), _stream(dS, stream)), "fdkod_net_backward")


class BatchBackprojection:
    """fdkod_batch_create / fdkod_batch_backproject: the backprojections of
    many plans in one persistent launch.  srcs[i]: Q (torch CUDA float32) for
    a plan with D = 1, the decomposed data or None (the plan's workspace) for
    D > 1; vols[i]: torch CUDA float32 [N][N][N].  Raises FdkodError
    (status -2) when a plan cannot take the persistent path."""

    def __init__(self, plans, srcs, vols):
        import torch
        n = len(plans)
        if len(srcs) != n or len(vols) != n:
            raise ValueError("one source and one volume per plan")
        for p, src, vol in zip(plans, srcs, vols):
            _expect(vol, p.vol_shape, torch.float32, "vol")
            if src is not None:
                if p.D == 1:
                    _expect(src, p.q_shape, p.q_torch_dtype, "src (Q)")
                else:
                    _expect(src, p.decomposed_shape, torch.float32, "src (decomposed data)")
        arr = ctypes.c_void_p * n
        P = arr(*[p.handle for p in plans])
        S = arr(*[None if s is None else _dev_ptr(s, "src").value for s in srcs])
        V = arr(*[_dev_ptr(v, "vol").value for v in vols])
        out = ctypes.c_void_p()
        _check(load().fdkod_batch_create(P, S, V, n, ctypes.byref(out)), "fdkod_batch_create")
        self.handle = out.value
        self._keep = (list(plans), list(srcs), list(vols))

    def run(self, stream=None):
        import torch
        st = int(torch.cuda.current_stream().cuda_stream) if stream is None else int(stream)
        _check(load().fdkod_batch_backproject(self.handle, st), "fdkod_batch_backproject")

    def close(self):
        if getattr(self, "handle", None):
            load().fdkod_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- convenience wrapper --------------------------------------------------

class Plan:
    """A plan for one geometry, decomposition level s and decimation D."""

    def __init__(self, R: float, N: int, Nu: int, Nv: int, P: int, s: int, D: int, qtype: str = "f32",
                 workspace: bool = True, taps="triangle"):
        """taps: the angular low-pass of the decomposition -- "triangle"
        (default), "sinc" (Hann-windowed sinc, half-width 2D) or an array
        h[|i|] of D or 2D values."""
        self.R, self.N, self.Nu, self.Nv, self.P, self.s, self.D = float(R), N, Nu, Nv, P, s, D
        self.qtype = qtype
        flags = 0 if workspace else FDKOD_PLAN_NO_WORKSPACE
        if isinstance(taps, str):
            if taps not in ("triangle", "sinc"):
                raise ValueError(f"unknown taps {taps!r}")
            if taps == "sinc":
                flags |= FDKOD_PLAN_SINC_TAPS
        self.handle = fdkod_plan(R, N, Nu, Nv, P, s, D, _DTYPES[qtype], flags)
        if not isinstance(taps, str):
            try:
                fdkod_set_decimation_taps(self.handle, taps)
            except Exception:
                self.close()
                raise
        info = PlanInfo()
        _check(load().fdkod_get_info(self.handle, ctypes.byref(info)), "fdkod_get_info")
        self.info = {f: getattr(info, f) for f, _ in PlanInfo._fields_}

    def close(self):
        if getattr(self, "handle", None):
            load().fdkod_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def q_torch_dtype(self):
        import torch
        return {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[self.qtype]

    # shapes of the device arrays the entry points read and write
    @property
    def q_shape(self):
        return (self.P, self.Nv, self.Nu)

    @property
    def vol_shape(self):
        return (self.N, self.N, self.N)

    @property
    def decomposed_shape(self):
        return (self.info["n_squares"], self.info["Pd"], self.Nv, self.info["T_stride"])

    def _q(self, Q, what="Q"):
        return _expect(Q, self.q_shape, self.q_torch_dtype, what)

    def filter(self, proj, Q=None, stream=None):
        import torch
        _expect(proj, self.q_shape, torch.float32, "proj")
        if Q is None:
            Q = torch.empty(self.q_shape, dtype=self.q_torch_dtype, device=proj.device)
        fdkod_filter(self.handle, proj, self._q(Q), stream)
        return Q

    def _vol(self, Q, vol):
        import torch
        if vol is None:
            vol = torch.empty(self.vol_shape, dtype=torch.float32, device=Q.device)
        return _expect(vol, self.vol_shape, torch.float32, "vol")

    def backproject(self, Q, vol=None, stream=None):
        vol = self._vol(self._q(Q), vol)
        fdkod_backproject(self.handle, Q, vol, stream)
        return vol

    def backproject_plain(self, Q, vol=None, stream=None):
        vol = self._vol(self._q(Q), vol)
        fdk_backproject_plain(self.handle, Q, vol, stream)
        return vol

    def decompose_to_workspace(self, Q, stream=None):
        """fdkod_decompose into the plan's own workspace (D > 1)."""
        _check(load().fdkod_decompose(self.handle, _dev_ptr(self._q(Q), "Q"), None, _stream(Q, stream)),
               "fdkod_decompose")

    def decompose(self, Q, out=None, stream=None):
        import torch
        self._q(Q)
        if out is None:
            out = torch.empty(self.decomposed_shape, dtype=torch.float32, device=Q.device)
        fdkod_decompose(self.handle, Q, _expect(out, self.decomposed_shape, torch.float32, "out"), stream)
        return out

    def backproject_decomposed_workspace(self, vol, stream=None):
        """The FDK-OD backprojection of the plan's own decomposed workspace
        (what fdkod_backproject runs after its decomposition)."""
        import torch
        _expect(vol, self.vol_shape, torch.float32, "vol")
        _check(load().fdkod_backproject_decomposed(self.handle, None, _dev_ptr(vol, "vol"), _stream(vol, stream)),
               "fdkod_backproject_decomposed")
        return vol

    def backproject_decomposed(self, S, vol=None, stream=None):
        import torch
        _expect(S, self.decomposed_shape, torch.float32, "S")
        vol = self._vol(S, vol)
        fdkod_backproject_decomposed(self.handle, S, vol, stream)
        return vol

    def compute_bounds(self, stream=None):
        import torch
        fdkod_compute_bounds(self.handle, torch.cuda.current_stream().cuda_stream if stream is None else stream)

    # -- piecemeal (slab-wise) reconstruction --
    def slab_rows(self, z0: int, nz: int) -> tuple[int, int]:
        v0, n = ctypes.c_int32(), ctypes.c_int32()
        _check(load().fdkod_slab_rows(self.handle, int(z0), int(nz), ctypes.byref(v0), ctypes.byref(n)),
               "fdkod_slab_rows")
        return v0.value, n.value

    def filter_rows(self, proj_rows, v0: int, Q=None, stream=None):
        import torch
        _expect(proj_rows, (self.P, None, self.Nu), torch.float32, "proj_rows")
        if Q is None:
            Q = torch.empty(proj_rows.shape, dtype=self.q_torch_dtype, device=proj_rows.device)
        _expect(Q, tuple(proj_rows.shape), self.q_torch_dtype, "Q_rows")
        _check(load().fdkod_filter_rows(self.handle, _dev_ptr(proj_rows, "proj_rows"), int(v0), int(proj_rows.shape[1]),
                                        _dev_ptr(Q, "Q_rows"), _stream(proj_rows, stream)), "fdkod_filter_rows")
        return Q

    def slab_workspace_elems(self, nrows: int) -> int:
        return 0 if self.D == 1 else self.info["n_squares"] * self.info["Pd"] * int(nrows) * self.info["T_stride"]

    def backproject_slab(self, Q_rows, v0: int, S_work, z0: int, nz: int, vol=None, stream=None):
        import torch
        _expect(Q_rows, (self.P, None, self.Nu), self.q_torch_dtype, "Q_rows")
        if S_work is not None:
            _expect(S_work, self.slab_workspace_elems(Q_rows.shape[1]), torch.float32, "S_work", at_least=True)
        if vol is None:
            vol = torch.empty((nz, self.N, self.N), dtype=torch.float32, device=Q_rows.device)
        _expect(vol, (nz, self.N, self.N), torch.float32, "vol_slab")
        sw = _dev_ptr(S_work, "S_work") if S_work is not None else ctypes.c_void_p()
        _check(load().fdkod_backproject_slab(self.handle, _dev_ptr(Q_rows, "Q_rows"), int(v0), int(Q_rows.shape[1]), sw,
                                             int(z0), int(nz), _dev_ptr(vol, "vol_slab"), _stream(Q_rows, stream)),
               "fdkod_backproject_slab")
        return vol

    @property
    def taps(self) -> np.ndarray:
        """The angular low-pass taps h[|i|] in use."""
        return fdkod_get_decimation_taps(self.handle)

    def set_taps(self, taps) -> None:
        """Replace the angular low-pass taps (D or 2D values h[|i|])."""
        fdkod_set_decimation_taps(self.handle, taps)

    @property
    def tile(self) -> tuple[int, int]:
        """(window columns in use, narrowest valid) of the FDK-OD backprojection."""
        w, m = ctypes.c_int(), ctypes.c_int()
        _check(load().fdkod_get_tile(self.handle, ctypes.byref(w), ctypes.byref(m)), "fdkod_get_tile")
        return w.value, m.value

    def set_tile(self, window_cols: int) -> None:
        """Select the backprojection's staging-window width (0: default)."""
        _check(load().fdkod_set_tile(self.handle, int(window_cols)), "fdkod_set_tile")

    @property
    def net(self):
        """The learned decimation's weights (BF16-rounded), or None."""
        return fdkod_get_decimation_net(self.handle)

    def set_net(self, w) -> None:
        """Set (FDKOD_NET_SIZE weights) or remove (None) the learned decimation."""
        fdkod_set_decimation_net(self.handle, w)

    def net_adjoint(self, vol_slice, ref_slice, z: int, dS, sq_err, stream=None) -> None:
        import torch
        _expect(vol_slice, (self.N, self.N), torch.float32, "vol_slice")
        _expect(ref_slice, (self.N, self.N), torch.float32, "ref_slice")
        _expect(dS, self.decomposed_shape, torch.float32, "dS")
        _expect(sq_err, 1, torch.float32, "sq_err", at_least=True)
        fdkod_net_adjoint(self.handle, vol_slice, ref_slice, z, dS, sq_err, stream)

    def net_backward(self, Q, w, dS, row_lo: int, row_hi: int, dW, stream=None) -> None:
        import torch
        self._q(Q)
        _expect(w, (FDKOD_NET_SIZE,), torch.float32, "w")
        _expect(dS, self.decomposed_shape, torch.float32, "dS")
        _expect(dW, (FDKOD_NET_SIZE,), torch.float32, "dW")
        fdkod_net_backward(self.handle, Q, w, dS, row_lo, row_hi, dW, stream)

    def bounds(self) -> dict:
        return fdkod_get_bounds(self.handle, self.info["n_squares"], self.P)

    def device_status(self, stream=None) -> int:
        import torch
        st = int(torch.cuda.current_stream().cuda_stream) if stream is None else int(stream)
        return int(load().fdkod_last_device_status(self.handle, st))


def _host_ptr(a, what, shape):
    """Pointer of a C-contiguous float32 host array (numpy or torch CPU
    tensor) of the given shape; ValueError otherwise."""
    if hasattr(a, "data_ptr"):   # torch CPU tensor
        if a.is_cuda or not a.is_contiguous() or str(a.dtype) != "torch.float32" or tuple(a.shape) != shape:
            raise ValueError(f"{what} must be a contiguous float32 CPU tensor of shape {shape}")
        return ctypes.c_void_p(a.data_ptr())
    if a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"] or a.shape != shape:
        raise ValueError(f"{what} must be a C-contiguous float32 array of shape {shape}")
    return ctypes.c_void_p(a.ctypes.data)


def reconstruct(plan: Plan, proj_host, out=None, stream=None):
    """One whole reconstruction from host memory through fdkod_reconstruct:
    filter, bounds, FDK-OD backprojection, with the upload of the
    projections (in bands of detector rows, each filtered and decomposed as
    it lands) and the read-back of the volume (in groups of slices)
    overlapping the compute.  proj_host: float32 [P][Nv][Nu]
    (numpy or torch CPU; page-locked memory lets the copies overlap); returns
    the float32 [N][N][N] volume (numpy, or `out`, numpy or torch CPU)."""
    N = plan.N
    if not hasattr(proj_host, "data_ptr"):
        proj_host = np.ascontiguousarray(proj_host, dtype=np.float32)
    if out is None:
        out = np.empty((N, N, N), dtype=np.float32)
    src = _host_ptr(proj_host, "proj_host", (plan.P, plan.Nv, plan.Nu))
    dst = _host_ptr(out, "out", (N, N, N))
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    _check(load().fdkod_reconstruct(plan.handle, src, dst, int(stream)), "fdkod_reconstruct")
    return out


def reconstruct_slabs(plan: Plan, proj_host, slab: int, out=None, stream=None):
    """Piecemeal FDK-OD (Sec. 2.2) through fdkod_reconstruct_slabs: the
    library uploads, for each slab of `slab` slices, only the detector rows it
    needs, filters, decomposes and backprojects them and copies the slab
    back, pipelined over three streams.  proj_host: float32 [P][Nv][Nu] host
    array (numpy, or a torch CPU tensor -- page-locked memory lets the copies
    overlap the compute); returns the float32 [N][N][N] volume (numpy, or
    `out`, numpy or torch CPU).  plan.last_slab_device_bytes records the
    device memory the call used."""
    import numpy as np
    N = plan.N

    def host_ptr(a, what, shape):
        if hasattr(a, "data_ptr"):   # torch CPU tensor
            if a.is_cuda or not a.is_contiguous() or str(a.dtype) != "torch.float32" or tuple(a.shape) != shape:
                raise ValueError(f"{what} must be a contiguous float32 CPU tensor of shape {shape}")
            return ctypes.c_void_p(a.data_ptr())
        if a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"] or a.shape != shape:
            raise ValueError(f"{what} must be a C-contiguous float32 array of shape {shape}")
        return ctypes.c_void_p(a.ctypes.data)

    if not hasattr(proj_host, "data_ptr"):
        proj_host = np.ascontiguousarray(proj_host, dtype=np.float32)
    if out is None:
        out = np.empty((N, N, N), dtype=np.float32)
    src = host_ptr(proj_host, "proj_host", (plan.P, plan.Nv, plan.Nu))
    dst = host_ptr(out, "out", (N, N, N))
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    used = ctypes.c_int64(0)
    _check(load().fdkod_reconstruct_slabs(plan.handle, src, dst, int(slab), int(stream), ctypes.byref(used)),
           "fdkod_reconstruct_slabs")
    plan.last_slab_device_bytes = int(used.value)
    return out
