"""FP64 CPU oracle for FDK and FDK-OD -- test infrastructure only.

Only the test-suite, the smoke check and the benchmark's CPU-baseline leg use
this package.  It shares no code with the CUDA library: the arithmetic lives
in ``oracle.c`` (plain C, FP64, OpenMP over independent outputs, compiled
with -ffp-contract=off), and this module only marshals numpy arrays.

Functions and the passages they follow:
  filter / filter_rows   cosine weight + Ram-Lak convolution (Sec. 1, "initial
                         convolution" of Sec. 3), direct sums in C
  filter_fft             the same convolution through numpy's FP64 FFT
  fdk / fdk_slices       FDK backprojection, a weighted sum of P samples per
                         voxel (Sec. 2.1)
  bounds                 Eq. 1 at the four vertices of each square (Sec. 2.1)
                         for the 4^s squares of Sec. 2.2
  shift_decimate         shift + angular low-pass + downsample (Sec. 2.1)
  triangle_taps / sinc_taps   the angular low-pass kernels (default / windowed sinc)
  fdkod / fdkod_slices   FDK-OD (Sec. 2.2)
  shift_rows             the shifted rows of one square at the full view rate
                         (step 1 of Sec. 2.1 alone)
  bp_square / bp_square_adjoint   backprojection of given decomposed data of
                         one square (Sec. 2.2) and its adjoint
  fdkod_net_slices       FDK-OD with the learned decimation of net.py

Every function here has at least one pin in tests/test_oracle_*.py that does
not go through the oracle itself.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None

ERRORS = {0: "ok", -1: "invalid argument", -2: "out of memory", -3: "crop window violated"}


def build(force: bool = False) -> str:
    """Compile oracle.c (gcc, FP64, no FP contraction, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_c_int, _c_long, _c_double, _vp = ctypes.c_int, ctypes.c_long, ctypes.c_double, ctypes.c_void_p


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            sig = {
                "oracle_set_threads": (None, [_c_int]),
                "oracle_max_threads": (_c_int, []),
                "oracle_filter_rows": (_c_int, [_c_double, _c_int, _c_int, _c_int, _vp, _c_long, _vp, _vp]),
                "oracle_filter": (_c_int, [_c_double, _c_int, _c_int, _c_int, _vp, _vp]),
                "oracle_fdk_slices": (_c_int, [_c_double, _c_int, _c_int, _c_int, _c_int, _vp, _c_int, _c_int,
                                               _vp, _vp]),
                "oracle_fdk": (_c_int, [_c_double, _c_int, _c_int, _c_int, _c_int, _vp, _c_int, _vp]),
                "oracle_bounds": (_c_int, [_c_double, _c_int, _c_int, _c_int, _c_int, _vp, _vp, _vp, _vp, _vp,
                                           _vp]),
                "oracle_shift_decimate": (_c_int, [_c_double, _c_int, _c_int, _c_int, _c_int, _c_int, _c_int, _vp,
                                                   _c_int, _c_int, _vp, _vp, _c_int]),
                "oracle_fdkod_slices": (_c_int, [_c_double, _c_int, _c_int, _c_int, _c_int, _c_int, _c_int, _vp,
                                                 _c_int, _c_int, _vp, _vp, _vp, _c_int]),
                "oracle_fdkod": (_c_int, [_c_double, _c_int, _c_int, _c_int, _c_int, _c_int, _c_int, _vp, _c_int,
                                          _vp, _vp, _c_int]),
                "oracle_shift_rows": (_c_int, [_c_double, _c_int, _c_int, _c_int, _c_int, _c_int, _vp, _c_int,
                                               _c_int, _c_int, _c_int, _vp]),
                "oracle_bp_square": (_c_int, [_c_double, _c_int, _c_int, _c_int, _c_int, _c_int, _c_int, _vp, _c_int,
                                              _c_int, _vp, _vp]),
                "oracle_bp_square_adjoint": (_c_int, [_c_double, _c_int, _c_int, _c_int, _c_int, _c_int, _c_int,
                                                      _vp, _c_int, _c_int, _vp, _vp]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what}: {ERRORS.get(rc, rc)}")


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _qarg(Q: np.ndarray):
    if Q.dtype == np.float64:
        return np.ascontiguousarray(Q), 1
    return np.ascontiguousarray(Q, dtype=np.float32), 0


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def filter_rows(proj: np.ndarray, R: float, rows) -> np.ndarray:
    """Filtered rows (flat index k*Nv + v) of proj[P][Nv][Nu] (float32)."""
    proj = np.ascontiguousarray(proj, dtype=np.float32)
    P, Nv, Nu = proj.shape
    rows = np.ascontiguousarray(rows, dtype=np.int64).reshape(-1)
    out = np.empty((rows.size, Nu), dtype=np.float64)
    _check(_load().oracle_filter_rows(R, Nu, Nv, P, _ptr(proj), rows.size, _ptr(rows), _ptr(out)), "filter_rows")
    return out


def filter(proj: np.ndarray, R: float) -> np.ndarray:
    proj = np.ascontiguousarray(proj, dtype=np.float32)
    P, Nv, Nu = proj.shape
    out = np.empty((P, Nv, Nu), dtype=np.float64)
    _check(_load().oracle_filter(R, Nu, Nv, P, _ptr(proj), _ptr(out)), "filter")
    return out


def filter_fft(proj: np.ndarray, R: float, v0: int = 0, Nv_det: int | None = None) -> np.ndarray:
    """The same filter as ``filter`` (cosine weight + linear Ram-Lak
    convolution, zero padding), computed with numpy's FP64 FFT: the kernel
    is wrapped onto a circle of length L >= 2 Nu, where every lag of the
    linear convolution keeps its own tap.  Fast enough for full-size views.
    proj may hold a band of rows v0 .. v0 + proj.shape[1] - 1 of a detector
    with Nv_det rows (default: the whole detector); rows are filtered
    independently, each with its own cosine weight."""
    proj = np.asarray(proj)
    P, nb, Nu = proj.shape
    Nv = nb if Nv_det is None else int(Nv_det)
    if v0 < 0 or v0 + nb > Nv:
        raise ValueError("row band outside the detector")
    L = 1
    while L < 2 * Nu:
        L *= 2
    lag = np.minimum(np.arange(L), L - np.arange(L))
    h = np.zeros(L)
    h[lag == 0] = 0.25
    odd = lag % 2 == 1
    h[odd] = -1.0 / (np.pi ** 2 * lag[odd].astype(np.float64) ** 2)
    H = np.fft.rfft(h).real
    a = np.arange(Nu) - (Nu - 1) / 2
    b = np.arange(v0, v0 + nb) - (Nv - 1) / 2
    w = R / np.sqrt(R * R + a[None, :] ** 2 + b[:, None] ** 2)
    out = np.empty((P, nb, Nu), dtype=np.float64)
    for k in range(P):
        q = proj[k].astype(np.float64) * w
        out[k] = np.fft.irfft(np.fft.rfft(q, n=L, axis=-1) * H, n=L, axis=-1)[:, :Nu]
    return out


def fdk_slices(Q: np.ndarray, R: float, N: int, zs) -> np.ndarray:
    Q, f64 = _qarg(Q)
    P, Nv, Nu = Q.shape
    zs = np.ascontiguousarray(zs, dtype=np.int32).reshape(-1)
    out = np.empty((zs.size, N, N), dtype=np.float64)
    _check(_load().oracle_fdk_slices(R, N, Nu, Nv, P, _ptr(Q), f64, zs.size, _ptr(zs), _ptr(out)), "fdk_slices")
    return out


def fdk(Q: np.ndarray, R: float, N: int) -> np.ndarray:
    Q, f64 = _qarg(Q)
    P, Nv, Nu = Q.shape
    out = np.empty((N, N, N), dtype=np.float64)
    _check(_load().oracle_fdk(R, N, Nu, Nv, P, _ptr(Q), f64, _ptr(out)), "fdk")
    return out


def bounds(R: float, N: int, Nu: int, P: int, s: int) -> dict:
    """Crop bounds per (square, angle): lo, hi, crop, phi [4^s][P]; w0, T [4^s]."""
    nsq = 4 ** s
    lo = np.empty((nsq, P), np.int32)
    hi = np.empty((nsq, P), np.int32)
    crop = np.empty((nsq, P), np.int32)
    phi = np.empty((nsq, P), np.float64)
    w0 = np.empty(nsq, np.int32)
    T = np.empty(nsq, np.int32)
    _check(_load().oracle_bounds(R, N, Nu, P, s, _ptr(lo), _ptr(hi), _ptr(crop), _ptr(phi), _ptr(w0), _ptr(T)),
           "bounds")
    return {"lo": lo, "hi": hi, "crop": crop, "phi": phi, "w0": w0, "T": T}


def triangle_taps(D: int) -> np.ndarray:
    """The default angular low-pass of Sec. 2.1 (its kernel is left open; the
    reading here is the triangle): h[|i|] = (D - |i|) / D^2, |i| < D."""
    i = np.arange(D, dtype=np.float64)
    return (D - i) / float(D * D)


def sinc_taps(D: int, H: int = 2) -> np.ndarray:
    """Hann-windowed sinc low-pass with its cutoff at the decimated Nyquist
    frequency pi / D (Sec. 2.1 says the low-pass filter sets the quality):
    g_i = sinc(i / D) (1 + cos(pi i / (H D))) / 2 for |i| < H D, scaled to
    unit gain at zero frequency.  Returns h[|i|], |i| = 0 .. H D - 1."""
    i = np.arange(H * D, dtype=np.float64)
    g = np.sinc(i / D) * 0.5 * (1.0 + np.cos(np.pi * i / (H * D)))
    return g / (g[0] + 2.0 * g[1:].sum())


def _taps_arg(taps, D: int):
    """(pointer, H) for the C oracle: None is the triangle."""
    if taps is None:
        return None, 1, None
    h = np.ascontiguousarray(taps, dtype=np.float64).reshape(-1)
    if h.size % D != 0 or h.size == 0:
        raise ValueError("taps must hold H D values h[0 .. H D - 1]")
    return _ptr(h), h.size // D, h


def shift_decimate(Q: np.ndarray, R: float, N: int, s: int, D: int, q: int, taps=None) -> np.ndarray:
    """Decomposed data S'_q[j][v][t] of square q (D > 1); taps: h[|i|] of
    the angular low-pass (None: the triangle)."""
    Q, f64 = _qarg(Q)
    P, Nv, Nu = Q.shape
    T = int(bounds(R, N, Nu, P, s)["T"][q])
    out = np.empty((P // D, Nv, T), dtype=np.float64)
    hp, H, _keep = _taps_arg(taps, D)
    _check(_load().oracle_shift_decimate(R, N, Nu, Nv, P, s, D, _ptr(Q), f64, q, _ptr(out), hp, H),
           "shift_decimate")
    return out


def fdkod_slices(Q: np.ndarray, R: float, N: int, s: int, D: int, zs, taps=None) -> np.ndarray:
    Q, f64 = _qarg(Q)
    P, Nv, Nu = Q.shape
    zs = np.ascontiguousarray(zs, dtype=np.int32).reshape(-1)
    out = np.empty((zs.size, N, N), dtype=np.float64)
    hp, H, _keep = _taps_arg(taps, D)
    _check(_load().oracle_fdkod_slices(R, N, Nu, Nv, P, s, D, _ptr(Q), f64, zs.size, _ptr(zs), _ptr(out), hp, H),
           "fdkod_slices")
    return out


def fdkod(Q: np.ndarray, R: float, N: int, s: int, D: int, taps=None) -> np.ndarray:
    Q, f64 = _qarg(Q)
    P, Nv, Nu = Q.shape
    out = np.empty((N, N, N), dtype=np.float64)
    hp, H, _keep = _taps_arg(taps, D)
    _check(_load().oracle_fdkod(R, N, Nu, Nv, P, s, D, _ptr(Q), f64, _ptr(out), hp, H), "fdkod")
    return out


def shift_rows(Q: np.ndarray, R: float, N: int, s: int, q: int, v0: int = 0, nv=None) -> np.ndarray:
    """S_q[k][v - v0][t] at the full view rate (no low-pass), rows v0 .. v0 + nv - 1."""
    Q, f64 = _qarg(Q)
    P, Nv, Nu = Q.shape
    nv = Nv - v0 if nv is None else nv
    T = int(bounds(R, N, Nu, P, s)["T"][q])
    out = np.empty((P, nv, T), dtype=np.float64)
    _check(_load().oracle_shift_rows(R, N, Nu, Nv, P, s, _ptr(Q), f64, q, v0, nv, _ptr(out)), "shift_rows")
    return out


def bp_square(Sp: np.ndarray, R: float, N: int, Nu: int, P: int, s: int, D: int, q: int, zs) -> np.ndarray:
    """Backprojection of decomposed data Sp[P/D][Nv][T_q] into square q's
    voxels on slices zs; other voxels of the returned [nz][N][N] are 0."""
    Sp = np.ascontiguousarray(Sp, dtype=np.float64)
    Nv = Sp.shape[1]
    zs = np.ascontiguousarray(zs, dtype=np.int32).reshape(-1)
    out = np.zeros((zs.size, N, N), dtype=np.float64)
    _check(_load().oracle_bp_square(R, N, Nu, Nv, P, s, D, _ptr(Sp), q, zs.size, _ptr(zs), _ptr(out)), "bp_square")
    return out


def bp_square_adjoint(E: np.ndarray, R: float, N: int, Nu: int, Nv: int, P: int, s: int, D: int, q: int,
                      zs) -> np.ndarray:
    """Adjoint of bp_square: [P/D][Nv][T_q] from E[nz][N][N] (only square q's
    voxels are read)."""
    E = np.ascontiguousarray(E, dtype=np.float64)
    zs = np.ascontiguousarray(zs, dtype=np.int32).reshape(-1)
    T = int(bounds(R, N, Nu, P, s)["T"][q])
    out = np.empty((P // D, Nv, T), dtype=np.float64)
    _check(_load().oracle_bp_square_adjoint(R, N, Nu, Nv, P, s, D, _ptr(E), q, zs.size, _ptr(zs), _ptr(out)),
           "bp_square_adjoint")
    return out


def triangle_or(taps, D: int) -> np.ndarray:
    return triangle_taps(D) if taps is None else np.asarray(taps, dtype=np.float64).reshape(-1)


def slice_rows(R: float, N: int, Nv: int, zs) -> tuple[int, int]:
    """First detector row and row count that slices zs can touch: U lies in
    [1 - r/R, 1 + r/R] with r the largest in-slice radius (the rows the C
    oracle's FDK-OD computes)."""
    vc = 0.5 * (Nv - 1)
    rmax = np.sqrt(2.0) * 0.5 * (N - 1)
    lo, hi = Nv, -1
    for z in np.asarray(zs).reshape(-1):
        zc = float(z) - 0.5 * (N - 1)
        va, vb = zc / (1.0 - rmax / R) + vc, zc / (1.0 + rmax / R) + vc
        lo = min(lo, int(np.floor(min(va, vb))) - 1)
        hi = max(hi, int(np.floor(max(va, vb))) + 2)
    lo, hi = max(lo, 0), min(hi, Nv - 1)
    return lo, max(0, hi - lo + 1)


def net_decomposed(Q: np.ndarray, R: float, N: int, s: int, D: int, q: int, w, taps=None,
                   act_round=None, rows=None) -> np.ndarray:
    """Decomposed data of square q with the learned decimation: the plain
    low-pass plus the net's output on the shifted rows (act_round: see
    net.net_forward).  rows = (v0, nv) computes only those detector rows
    (the rest of the returned [P/D][Nv][T_q] is 0), with the plain low-pass
    taken as the circular FIR of the shifted rows (equal to shift_decimate,
    tests/test_oracle_net.py)."""
    from .net import net_forward
    P, Nv, _ = np.shape(Q)
    if rows is None:
        S = shift_rows(Q, R, N, s, q)                  # [P][Nv][T]
        return shift_decimate(Q, R, N, s, D, q, taps) + net_forward(S, D, w, act_round)
    v0, nv = rows
    S = shift_rows(Q, R, N, s, q, v0, nv)
    h = triangle_or(taps, D)
    lin = sum(h[abs(i)] * np.roll(S, -i, axis=0)[::D] for i in range(-(h.size - 1), h.size))
    out = np.zeros((P // D, Nv, S.shape[2]))
    out[:, v0:v0 + nv] = lin + net_forward(S, D, w, act_round)
    return out


def fdkod_net_slices(Q: np.ndarray, R: float, N: int, s: int, D: int, w, zs, taps=None,
                     act_round=None, squares=None) -> np.ndarray:
    """FDK-OD slices with the learned decimation (D > 1); only the detector
    rows the slices touch are decomposed.  squares: compute only these
    squares' voxels (the others stay 0), for sampled checks at large N."""
    P, Nv, Nu = np.shape(Q)
    zs = np.asarray(zs).reshape(-1)
    rows = slice_rows(R, N, Nv, zs)
    vol = np.zeros((zs.size, N, N))
    for q in (range(4 ** s) if squares is None else squares):
        vol += bp_square(net_decomposed(Q, R, N, s, D, q, w, taps, act_round, rows), R, N, Nu, P, s, D, q, zs)
    return vol


def square_mask(N: int, s: int, squares) -> np.ndarray:
    """[N][N] boolean mask (y, x) of the voxels of the given squares (voxel i
    belongs to square floor(i 2^s / N))."""
    m = 1 << s
    sq = (np.arange(N) * m) // N
    q = sq[:, None] * m + sq[None, :]
    return np.isin(q, np.asarray(list(squares)))
