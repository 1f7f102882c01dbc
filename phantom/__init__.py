"""Seeded synthetic inputs: random-ellipsoid phantoms and their exact cone-beam
projections.

This module is the one input source shared by the FP64 oracle and the CUDA
path.  It holds none of the reconstruction method's arithmetic: it draws
phantom parameters with numpy's PCG64 and evaluates closed-form chord lengths
(``project.c``), which stand in for the paper's Shepp-Logan and scanner data
(Sec. 3), not included here.

Geometry: beta_k = 2*pi*k/P, source at -R (cos beta, sin beta, 0), a virtual
flat detector through the isocentre with unit pitch, detector coordinates
a = u - (Nu-1)/2, b = v - (Nv-1)/2, voxel centres x_i = i - (N-1)/2.  With
this convention the column of a point (x, y) is the paper's Eq. 1 and its row
is the b formula of Sec. 2.2.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "project.c")
_SO = os.path.join(_HERE, "_phantom.so")
_lock = threading.Lock()
_lib = None

NPAR = 16


def build(force: bool = False) -> str:
    """Compile project.c into an in-tree shared object (gcc, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_SRC_GPU = os.path.join(_HERE, "project_gpu.cu")
_SO_GPU = os.path.join(_HERE, "_phantom_gpu.so")
_lib_gpu = None


def build_gpu(force: bool = False) -> str:
    """Compile the GPU projector (nvcc, sm_103a) into an in-tree shared object."""
    if force or not os.path.exists(_SO_GPU) or os.path.getmtime(_SO_GPU) < os.path.getmtime(_SRC_GPU):
        tmp = _SO_GPU + f".{os.getpid()}.tmp"
        nvcc = os.environ.get("NVCC") or "nvcc"
        if not os.path.exists(nvcc) and os.path.exists("/usr/local/cuda/bin/nvcc"):
            nvcc = "/usr/local/cuda/bin/nvcc"
        subprocess.check_call([nvcc, "-O3", "-gencode", "arch=compute_103a,code=sm_103a", "-Xcompiler", "-fPIC",
                               "-shared", "-o", tmp, _SRC_GPU])
        os.replace(tmp, _SO_GPU)
    return _SO_GPU


def project_gpu(ell: np.ndarray, R: float, Nu: int, Nv: int, P: int, out=None, k0: int = 0, k1: int | None = None):
    """The same line integrals as `project`, computed on the current CUDA
    device in FP32 (input generation for large workloads); returns a torch
    float32 tensor [k1-k0][Nv][Nu] on the device."""
    global _lib_gpu
    import torch
    with _lock:
        if _lib_gpu is None:
            lib = ctypes.CDLL(build_gpu())
            lib.phantom_project_gpu.restype = ctypes.c_int
            lib.phantom_project_gpu.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_void_p, ctypes.c_size_t]
            _lib_gpu = lib
    k1 = P if k1 is None else k1
    e32 = np.ascontiguousarray(ell, dtype=np.float32).reshape(-1, NPAR)
    if out is None:
        out = torch.empty((k1 - k0, Nv, Nu), dtype=torch.float32, device="cuda")
    rc = _lib_gpu.phantom_project_gpu(e32.shape[0], e32.ctypes.data, float(R), Nu, Nv, P, k0, k1,
                                      out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    if rc != 0:
        raise RuntimeError(f"GPU projector failed ({rc})")
    return out


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            for name, ptr in (("phantom_project_f64", ctypes.c_double), ("phantom_project_f32", ctypes.c_float)):
                fn = getattr(lib, name)
                fn.restype = ctypes.c_int
                fn.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                               ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               ctypes.POINTER(ptr)]
            fn = lib.phantom_project_band_f32
            fn.restype = ctypes.c_int
            fn.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_double, ctypes.c_int,
                           ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                           ctypes.POINTER(ctypes.c_float)]
            _lib = lib
    return _lib


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform rotation on SO(3) from a normalised Gaussian quaternion."""
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def ellipsoid(centre, semi_axes, rot, rho) -> np.ndarray:
    e = np.zeros(NPAR)
    e[0:3] = centre
    e[3:6] = semi_axes
    e[6:15] = np.asarray(rot, dtype=np.float64).reshape(9)
    e[15] = rho
    return e


def make_phantom(seed: int, N: int, n_ell: int) -> np.ndarray:
    """n_ell random ellipsoids for an N^3 volume, shape (n_ell, 16).

    Centres uniform in the ball of radius 0.7*N/2, semi-axes independent
    U(0.05N, 0.3N), orientation uniform on SO(3), densities U(0.1, 1),
    additive.  Objects may extend past the field of view; both the oracle
    and the GPU path see the same truncated data.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.zeros((n_ell, NPAR))
    rmax = 0.7 * N / 2.0
    for i in range(n_ell):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        c = d * rmax * rng.random() ** (1.0 / 3.0)
        ax = rng.uniform(0.05 * N, 0.3 * N, size=3)
        rot = random_rotation(rng)
        rho = rng.uniform(0.1, 1.0)
        out[i] = ellipsoid(c, ax, rot, rho)
    return out


def project(ell: np.ndarray, R: float, Nu: int, Nv: int, P: int, k0: int = 0, k1: int | None = None,
            dtype=np.float32, rows: tuple[int, int] | None = None) -> np.ndarray:
    """Exact line integrals, array [k1-k0][Nv][Nu] of dtype float32 or float64;
    with rows = (v0, v1) only detector rows v0..v1-1, [k1-k0][v1-v0][Nu]
    (float32)."""
    lib = _load()
    k1 = P if k1 is None else k1
    ell = np.ascontiguousarray(ell, dtype=np.float64).reshape(-1, NPAR)
    n = ell.shape[0]
    ep = ell.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    if rows is not None:
        if dtype != np.float32:
            raise ValueError("row bands are float32")
        v0, v1 = int(rows[0]), int(rows[1])
        out = np.empty((k1 - k0, max(0, v1 - v0), Nu), dtype=np.float32)
        rc = lib.phantom_project_band_f32(n, ep, R, Nu, Nv, P, k0, k1, v0, v1,
                                          out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
        if rc != 0:
            raise RuntimeError(f"phantom projector failed ({rc})")
        return out
    out = np.empty((k1 - k0, Nv, Nu), dtype=dtype)
    if dtype == np.float64:
        rc = lib.phantom_project_f64(n, ep, R, Nu, Nv, P, k0, k1, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    elif dtype == np.float32:
        rc = lib.phantom_project_f32(n, ep, R, Nu, Nv, P, k0, k1, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    else:
        raise ValueError("dtype must be float32 or float64")
    if rc != 0:
        raise RuntimeError(f"phantom projector failed ({rc})")
    return out


def add_noise(p: np.ndarray, sigma_frac: float, seed: int) -> np.ndarray:
    """Add N(0, sigma^2), sigma = sigma_frac * max line integral, in place."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    sigma = sigma_frac * float(np.max(p))
    chunk = 1 << 24
    flat = p.reshape(-1)
    for i in range(0, flat.size, chunk):
        n = min(chunk, flat.size - i)
        flat[i:i + n] += (sigma * rng.standard_normal(n)).astype(p.dtype)
    return p


@dataclass(frozen=True)
class Workload:
    """One synthetic workload: geometry, decomposition and phantom recipe."""
    name: str
    N: int
    P: int
    s: int
    D: int
    n_ell: int
    noise: float
    seed: int

    @property
    def Nu(self) -> int:
        return self.N

    @property
    def Nv(self) -> int:
        return self.N

    @property
    def R(self) -> float:
        # source-to-isocentre 4N voxels; source-to-detector 8N only rescales
        # the physical pitch and cancels on the virtual detector
        return 4.0 * self.N


# Workloads shaped like the paper's (N = 256..2500, P = 720, s up to 5).
WORKLOADS = {
    "fdkod_128": Workload("fdkod_128^3_P128_s2_D2", 128, 128, 2, 2, 10, 0.0, 1000),
    # small case of the 512 workload's square size (64) and D, for profiling
    "fdkod_256": Workload("fdkod_256^3_P360_s2_D4", 256, 360, 2, 4, 20, 0.01, 1500),
    "fdkod_512": Workload("fdkod_512^3_P720_s3_D4", 512, 720, 3, 4, 40, 0.01, 2000),
    # the 512 workload's detector and squares with a quarter of its views, for profiling
    "fdkod_512_p180": Workload("fdkod_512^3_P180_s3_D4", 512, 180, 3, 4, 40, 0.01, 2000),
    "fdkod_1024": Workload("fdkod_1024^3_P720_s4_D8", 1024, 720, 4, 8, 80, 0.0, 3000),
    "fdkod_2000": Workload("fdkod_2000^3_P720_s5_D16", 2000, 720, 5, 16, 150, 0.01, 5000),
}


def batched_workload(seed: int = 4000, count: int = 64, sizes=(64, 96, 128, 192, 256, 384), n_ell: int = 20):
    """Many volumes of uneven size: N drawn (seeded) from `sizes`,
    P = round(1.4 N) views, R = 4N, `n_ell` ellipsoids each.
    Returns a list of (N, P, R, seed_i)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        N = int(rng.choice(sizes))
        out.append((N, int(round(1.4 * N)), 4.0 * N, seed + 1 + i))
    return out


def make_projections(w: Workload, dtype=np.float32) -> np.ndarray:
    ell = make_phantom(w.seed, w.N, w.n_ell)
    p = project(ell, w.R, w.Nu, w.Nv, w.P, dtype=dtype)
    if w.noise > 0:
        add_noise(p, w.noise, w.seed)
    return p
