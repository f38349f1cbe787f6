"""FP64 CPU oracle for the free-energy hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares
no code with the CUDA path (``paper_1412_8754_gb300``) and imports nothing
from it; the two meet only through the seeded input generators in
``paper_1412_8754_gb300.workloads``, which hold none of the method's
arithmetic.

Layout:
  ffe_oracle.c   Eq. freeene / Eq. enequasiparticle / App. A in plain C (FP64)
  search.py      grid argmin, golden-section search and phase labels (Alg. 1)
  threeband.py   the three-band model of App. B (eigvalsh of its 3x3 matrix + the C k-sum)
  chi.py         the static Cooper pair susceptibility of App. C
  mlp.py         FP64 reference of the surrogate MLP (forward, backward, Adam)

Parity status of each function is listed in the module docstrings; every
function here is pinned by a ``-m "not gpu"`` test in tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ffe_oracle.c")
_LIB = os.path.join(_HERE, "libffe_oracle.so")
_lock = threading.Lock()
_lib = None

# App. A: hopping parameters of the two-band model and the chemical potential
# that gives two electrons per site (half filling), in units of |t1|.
RAGHU2 = dict(t1=-1.0, t2=1.3, t3=-0.85, t4=-0.85, mu=1.54)


class Model(ctypes.Structure):
    _fields_ = [
        ("t1", ctypes.c_double),
        ("t2", ctypes.c_double),
        ("t3", ctypes.c_double),
        ("t4", ctypes.c_double),
        ("mu", ctypes.c_double),
        ("eta_amp", ctypes.c_double),
        ("U", ctypes.c_double),
        ("U_band", ctypes.c_double * 2),   # per-band coupling; 0 = U
    ]


def make_model(U: float = 2.0, eta_amp: float = 1.0, U_band=(0.0, 0.0), **over) -> Model:
    p = dict(RAGHU2)
    p.update(over)
    return Model(p["t1"], p["t2"], p["t3"], p["t4"], p["mu"], eta_amp, U, (ctypes.c_double * 2)(*U_band))


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math, no FP contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-std=c11", "-D_DEFAULT_SOURCE", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int32)
            mp = ctypes.POINTER(Model)
            L.ffeo_band_energies.argtypes = [mp, ctypes.c_double, ctypes.c_double, dp]
            L.ffeo_band_energies.restype = None
            L.ffeo_quasiparticle.argtypes = [ctypes.c_double] * 3 + [dp, dp]
            L.ffeo_quasiparticle.restype = None
            L.ffeo_F.argtypes = [ctypes.c_double, ctypes.c_double]
            L.ffeo_F.restype = ctypes.c_double
            L.ffeo_omega.argtypes = [mp, ctypes.c_int] + [ctypes.c_double] * 5 + [dp, dp]
            L.ffeo_omega.restype = None
            L.ffeo_omega_batch.argtypes = [mp, ctypes.c_int64, ip] + [dp] * 7 + [ctypes.c_int]
            L.ffeo_omega_batch.restype = ctypes.c_int
            L.ffeo_band_grid.argtypes = [mp, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp]
            L.ffeo_band_grid.restype = None
            L.ffeo_omega_given.argtypes = ([ctypes.c_int, ctypes.c_int, dp, dp] + [ctypes.c_double] * 2 + [dp]
                                           + [ctypes.c_double] * 3 + [dp, dp])
            L.ffeo_omega_given.restype = None
            L.ffeo_omega_given_batch.argtypes = ([ctypes.c_int, ctypes.c_int, dp, dp] + [ctypes.c_double] * 2
                                                 + [dp, ctypes.c_int64] + [dp] * 5 + [ctypes.c_int])
            L.ffeo_omega_given_batch.restype = ctypes.c_int
            L.ffeo_chi_given.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp] + [ctypes.c_double] * 3 + [dp]
            L.ffeo_chi_given.restype = None
            L.ffeo_max_threads.argtypes = []
            L.ffeo_max_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def band_energies(model: Model, kx: float, ky: float) -> np.ndarray:
    """App. A closed form: [E_-(k), E_+(k)]."""
    out = np.zeros(2)
    lib().ffeo_band_energies(ctypes.byref(model), kx, ky, _dp(out))
    return out


def band_grid(model: Model, N: int, qx: float = 0.0, qy: float = 0.0) -> np.ndarray:
    """[N, N, 2] array of E_eps(k + Q/2) over the lattice k = 2 pi (i, j) / N, index [j, i, eps]."""
    out = np.zeros((N, N, 2))
    lib().ffeo_band_grid(ctypes.byref(model), N, qx, qy, _dp(out))
    return out


def quasiparticle(e_up: float, e_dn: float, gap: float):
    """Eq. enequasiparticle: (E^+, E^-)."""
    ep = ctypes.c_double()
    em = ctypes.c_double()
    lib().ffeo_quasiparticle(e_up, e_dn, gap, ctypes.byref(ep), ctypes.byref(em))
    return ep.value, em.value


def F(E: float, T: float) -> float:
    """-T ln(1 + exp(-E/T))."""
    return lib().ffeo_F(E, T)


def omega(model: Model, N: int, qx: float, qy: float, h: float, T: float, delta: float,
          bands: bool = False):
    """Eq. freeene summed over both bands; with bands=True also returns [Omega_-, Omega_+]."""
    out = ctypes.c_double()
    ob = np.zeros(2)
    lib().ffeo_omega(ctypes.byref(model), N, qx, qy, h, T, delta, ctypes.byref(out), _dp(ob))
    return (out.value, ob) if bands else out.value


def omega_batch(model: Model, N, qx, qy, h, T, delta, nthreads: int = 0, bands: bool = False):
    """Many independent points (broadcast to a common length), OpenMP over points.

    Returns (omega[n], omega_band[n,2] or None, threads_used)."""
    arrs = np.broadcast_arrays(np.asarray(N), np.asarray(qx, float), np.asarray(qy, float),
                               np.asarray(h, float), np.asarray(T, float), np.asarray(delta, float))
    n = arrs[0].size
    Na = np.ascontiguousarray(arrs[0].ravel(), dtype=np.int32)
    cols = [np.ascontiguousarray(a.ravel(), dtype=np.float64) for a in arrs[1:]]
    om = np.zeros(n)
    ob = np.zeros((n, 2)) if bands else None
    used = lib().ffeo_omega_batch(
        ctypes.byref(model), n, Na.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
        *[_dp(c) for c in cols], _dp(om), _dp(ob) if bands else None, int(nthreads))
    return om, ob, used


def max_threads() -> int:
    return lib().ffeo_max_threads()
