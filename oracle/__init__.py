"""FP64 CPU oracle for finite-frequency traveltime tomography (arXiv:1908.03302).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.
The product path (``paper_1908_03302_gb300``) never imports it and shares no code with
it: the two meet only at the seeded inputs of ``workloads``.

Contents:

* ``fft_oracle.c`` (built with gcc + OpenMP into ``_liboracle.so`` next to this file):
  the Phi table by quadrature, the detour time, K0, J, J^T, the squared Frobenius norm,
  damped CGLS and Hessian PSFs, all in double precision (see that file's header for the
  section / equation each function follows).
* ``lowrank.py``: the low-rank posterior covariance and resolution diagonals (randomized
  subspace iteration over the oracle's J and J^T, numpy QR and eigh), FP64.
* ``closed_form.py``: independent closed forms used to pin the C code: the Gaussian
  spectrum's Phi in closed form, prolate-spheroidal quadrature of the uniform-perturbation
  invariant, and a brute-force Born cross-correlation traveltime for a point scatterer.

Parity status: every function here is pinned by a test under ``tests/`` marked
``not gpu`` (closed forms, invariants, brute force, dense linear algebra); see the test
module docstrings for which pin covers which function.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fft_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with the host gcc (portable flags: no -march=native)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            d, i32, i64, vp = ctypes.c_double, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
            geom = [vp, vp, vp, vp, vp, i32, i32, i32, i32, d, vp, d, vp]
            L.oracle_phi_table.argtypes = [ctypes.c_int, d, d, vp, vp, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, d, vp]
            L.oracle_phi_table.restype = ctypes.c_int
            L.oracle_phi.argtypes = [vp, ctypes.c_int, d, d]
            L.oracle_phi.restype = d
            L.oracle_trig_coefs.argtypes = [d, d, d, ctypes.c_int, ctypes.c_int, vp, vp, vp]
            L.oracle_trig_coefs.restype = ctypes.c_int
            L.oracle_phi_trig.argtypes = [vp, ctypes.c_int, d, d, d]
            L.oracle_phi_trig.restype = d
            L.oracle_detour.argtypes = [vp, vp, vp, vp, vp, vp, vp]
            L.oracle_detour_naive.argtypes = [vp, vp, vp]
            L.oracle_detour_naive.restype = d
            L.oracle_k0.argtypes = [vp, vp, vp, d, vp, ctypes.c_int, d]
            L.oracle_k0.restype = d
            L.oracle_J_entry.argtypes = geom + [i64, i64]
            L.oracle_J_entry.restype = d
            L.oracle_J.argtypes = geom + [i64, vp, i64, vp, vp]
            L.oracle_JT.argtypes = geom + [i64, vp, vp, i64, vp]
            L.oracle_coverage.argtypes = geom + [i64, vp, vp, i64, vp]
            L.oracle_J2d.argtypes = geom + [i64, vp, i64, vp, vp]
            L.oracle_JT2d.argtypes = geom + [i64, vp, vp, i64, vp]
            L.oracle_k2_midpoint.argtypes = [vp, vp, d, d, d, d, ctypes.c_int, d, vp, ctypes.c_int, d]
            L.oracle_k2_midpoint.restype = d
            L.oracle_count_support.argtypes = geom + [i64, vp, i64]
            L.oracle_count_support.restype = i64
            L.oracle_frob2.argtypes = geom + [i64]
            L.oracle_frob2.restype = d
            L.oracle_cgls.argtypes = geom + [i64, vp, d, i32, vp, vp]
            L.oracle_cgls.restype = ctypes.c_int
            L.oracle_psf.argtypes = geom + [i64, vp, i32, vp, i32, vp, vp, i64, vp]
            L.oracle_n_threads.restype = ctypes.c_int
            L.oracle_set_threads.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def n_threads() -> int:
    return lib().oracle_n_threads()


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


# --------------------------------------------------------------------------- Phi

def phi_table_gauss(f_center: float, f_sigma: float, n: int, dt_max: float, n_quad: int = 40000) -> np.ndarray:
    """Phi_k (1/s) for the Gaussian power spectrum by composite Simpson quadrature."""
    out = np.empty(n)
    rc = lib().oracle_phi_table(0, f_center, f_sigma, None, None, 0, n_quad, n, dt_max, _p(out))
    if rc != 0:
        raise ValueError("oracle_phi_table rejected its arguments")
    return out


def phi_table_sampled(omega: np.ndarray, weight: np.ndarray, n: int, dt_max: float) -> np.ndarray:
    """Phi_k (1/s) for a sampled power spectrum W(omega_j) by the trapezoid rule."""
    om = np.ascontiguousarray(omega, dtype=np.float64)
    w = np.ascontiguousarray(weight, dtype=np.float64)
    out = np.empty(n)
    rc = lib().oracle_phi_table(1, 0.0, 0.0, _p(om), _p(w), len(om), 0, n, dt_max, _p(out))
    if rc != 0:
        raise ValueError("oracle_phi_table rejected its arguments")
    return out


def phi_lookup(table: np.ndarray, dt_max: float, dt: float) -> float:
    t = np.ascontiguousarray(table, dtype=np.float64)
    return lib().oracle_phi(_p(t), len(t), dt_max, float(dt))


def trig_coefs(f_center: float, f_sigma: float, dt_max: float, n_terms: int = 0,
               n_quad: int = 40000) -> Tuple[np.ndarray, float]:
    """Sine-series form of Phi for the Gaussian power spectrum: (a_j for j = 1..n, dw), with
    Phi(dt) = sum_j a_j sin(j dw dt) (n chosen by the oracle's rule unless n_terms > 0)."""
    a = np.empty(4096)
    dw = ctypes.c_double()
    n = ctypes.c_int()
    rc = lib().oracle_trig_coefs(f_center, f_sigma, dt_max, int(n_terms), n_quad, _p(a), ctypes.byref(dw),
                                 ctypes.byref(n))
    if rc != 0:
        raise ValueError("oracle_trig_coefs rejected its arguments")
    return a[:n.value].copy(), dw.value


def phi_trig(a: np.ndarray, dw: float, dt_max: float, dt: float) -> float:
    """The truncated sine series at one dt (FP64, term by term)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    return lib().oracle_phi_trig(_p(a), len(a), float(dw), float(dt_max), float(dt))


def k2_midpoint(xs, xr, x: float, y: float, z0: float, hz: float, nz: int, c0: float, table: np.ndarray,
                dt_max: float) -> float:
    """int K0(x, y, z) dz over [z0, z0 + nz hz] by the midpoint rule (s^2 / m^3)."""
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (xs, xr)]
    t = np.ascontiguousarray(table, dtype=np.float64)
    return lib().oracle_k2_midpoint(_p(a[0]), _p(a[1]), float(x), float(y), float(z0), float(hz), int(nz), c0,
                                    _p(t), len(t), dt_max)


def detour(xs, xr, x):
    """(R, R_xs, R_xr, L) in metres by the cancellation-free form."""
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (xs, xr, x)]
    out = [ctypes.c_double() for _ in range(4)]
    lib().oracle_detour(*[_p(v) for v in a], *[ctypes.byref(o) for o in out])
    return tuple(o.value for o in out)


def detour_naive(xs, xr, x) -> float:
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (xs, xr, x)]
    return lib().oracle_detour_naive(*[_p(v) for v in a])


def k0(xs, xr, x, c0: float, table: np.ndarray, dt_max: float) -> float:
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (xs, xr, x)]
    t = np.ascontiguousarray(table, dtype=np.float64)
    return lib().oracle_k0(*[_p(v) for v in a], c0, _p(t), len(t), dt_max)


# --------------------------------------------------------------------------- operator

class Geometry:
    """Arrays describing rows, voxels and tables, held as contiguous numpy buffers."""

    def __init__(self, tx: np.ndarray, rows: np.ndarray, band: Optional[np.ndarray],
                 tables: Sequence[np.ndarray], dt_max: Sequence[float], grid, c0: float,
                 trig_dw: Optional[Sequence[float]] = None):
        """tables: per band either a sampled Phi table (trig_dw None) or the coefficients of the
        sine series with node spacing trig_dw[band] (bands of different lengths are zero-padded)."""
        self.tx = np.ascontiguousarray(tx, dtype=np.float64)
        self.rows = np.ascontiguousarray(rows, dtype=np.int32)
        self.M = int(self.rows.shape[0])
        self.band = None if band is None else np.ascontiguousarray(band, dtype=np.int32)
        n = max(len(t) for t in tables)
        self.tables = np.zeros((len(tables), n))
        for b, t in enumerate(tables):
            self.tables[b, :len(t)] = t
        self.trig_dw = None if trig_dw is None else np.ascontiguousarray(trig_dw, dtype=np.float64)
        self.dt_max = np.ascontiguousarray(dt_max, dtype=np.float64)
        self.grid = grid
        self.org = np.ascontiguousarray(grid.origin, dtype=np.float64)
        self.c0 = float(c0)
        self.V = grid.n_vox

    @staticmethod
    def from_workload(w, tables: Optional[Sequence[np.ndarray]] = None, phi: str = "table",
                      n_terms: int = 0) -> "Geometry":
        """phi = "table" (sampled, linear interpolation) or "trig" (sine series)."""
        if phi == "trig":
            series = [trig_coefs(b.f_center_hz, b.f_sigma_hz, b.dt_max, n_terms) for b in w.bands]
            return Geometry(w.tx, w.row_pairs(), w.band_of_row, [a for a, _ in series],
                            [b.dt_max for b in w.bands], w.grid, w.c0, trig_dw=[dw for _, dw in series])
        if tables is None:
            tables = [phi_table_gauss(b.f_center_hz, b.f_sigma_hz, b.n_samples, b.dt_max) for b in w.bands]
        return Geometry(w.tx, w.row_pairs(), w.band_of_row, tables, [b.dt_max for b in w.bands],
                        w.grid, w.c0)

    def _args(self):
        g = self.grid
        return (_p(self.tx), _p(self.rows), _p(self.band), _p(self.tables), _p(self.dt_max),
                int(self.tables.shape[1]), g.nx, g.ny, g.nz, g.h, _p(self.org), self.c0, _p(self.trig_dw))

    def entry(self, p: int, v: int) -> float:
        return lib().oracle_J_entry(*self._args(), int(p), int(v))

    def J(self, m: np.ndarray, rows: Optional[np.ndarray] = None) -> np.ndarray:
        m = np.ascontiguousarray(m, dtype=np.float64)
        assert m.shape == (self.V,)
        if rows is None:
            out = np.empty(self.M)
            lib().oracle_J(*self._args(), self.M, None, 0, _p(m), _p(out))
        else:
            idx = np.ascontiguousarray(rows, dtype=np.int64)
            out = np.empty(len(idx))
            lib().oracle_J(*self._args(), self.M, _p(idx), len(idx), _p(m), _p(out))
        return out

    def JT(self, d: np.ndarray, voxels: Optional[np.ndarray] = None) -> np.ndarray:
        d = np.ascontiguousarray(d, dtype=np.float64)
        assert d.shape == (self.M,)
        if voxels is None:
            out = np.empty(self.V)
            lib().oracle_JT(*self._args(), self.M, _p(d), None, 0, _p(out))
        else:
            idx = np.ascontiguousarray(voxels, dtype=np.int64)
            out = np.empty(len(idx))
            lib().oracle_JT(*self._args(), self.M, _p(d), _p(idx), len(idx), _p(out))
        return out

    def J2d(self, m2: np.ndarray, rows: Optional[np.ndarray] = None) -> np.ndarray:
        """d = J2 m2: the operator integrated over the grid's z layers (Eq. forward_2D)."""
        m2 = np.ascontiguousarray(m2, dtype=np.float64)
        assert m2.shape == (self.grid.nx * self.grid.ny,)
        idx = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
        out = np.empty(self.M if idx is None else len(idx))
        lib().oracle_J2d(*self._args(), self.M, _p(idx), 0 if idx is None else len(idx), _p(m2), _p(out))
        return out

    def JT2d(self, d: np.ndarray, pixels: Optional[np.ndarray] = None) -> np.ndarray:
        d = np.ascontiguousarray(d, dtype=np.float64)
        assert d.shape == (self.M,)
        idx = None if pixels is None else np.ascontiguousarray(pixels, dtype=np.int64)
        out = np.empty(self.grid.nx * self.grid.ny if idx is None else len(idx))
        lib().oracle_JT2d(*self._args(), self.M, _p(d), _p(idx), 0 if idx is None else len(idx), _p(out))
        return out

    def coverage(self, w: Optional[np.ndarray] = None, voxels: Optional[np.ndarray] = None) -> np.ndarray:
        """sum_p |J[p, v] w_p| for every voxel (or the given ones); w None: all ones."""
        wp = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
        if wp is not None:
            assert wp.shape == (self.M,)
        if voxels is None:
            out = np.empty(self.V)
            lib().oracle_coverage(*self._args(), self.M, _p(wp), None, 0, _p(out))
        else:
            idx = np.ascontiguousarray(voxels, dtype=np.int64)
            out = np.empty(len(idx))
            lib().oracle_coverage(*self._args(), self.M, _p(wp), _p(idx), len(idx), _p(out))
        return out

    def count_support(self, rows: Optional[np.ndarray] = None) -> int:
        if rows is None:
            return int(lib().oracle_count_support(*self._args(), self.M, None, 0))
        idx = np.ascontiguousarray(rows, dtype=np.int64)
        return int(lib().oracle_count_support(*self._args(), self.M, _p(idx), len(idx)))

    def frob2(self) -> float:
        return float(lib().oracle_frob2(*self._args(), self.M))

    def lambda_abs(self, lambda_rel: float) -> float:
        """Damping lambda = lambda_rel * |J|_F^2 / N (mean diagonal of J^T J)."""
        return lambda_rel * self.frob2() / self.V

    def cgls(self, d: np.ndarray, lam: float, n_iter: int, m0: Optional[np.ndarray] = None):
        d = np.ascontiguousarray(d, dtype=np.float64)
        m = np.zeros(self.V) if m0 is None else np.array(m0, dtype=np.float64)
        hist = np.empty(n_iter + 1)
        rc = lib().oracle_cgls(*self._args(), self.M, _p(d), float(lam), int(n_iter), _p(m), _p(hist))
        return m, hist, rc

    def psf(self, spikes: np.ndarray, subsets: Sequence[np.ndarray], voxels: Optional[np.ndarray] = None):
        sp = np.ascontiguousarray(spikes, dtype=np.int64)
        off = np.zeros(len(subsets) + 1, dtype=np.int32)
        off[1:] = np.cumsum([len(s) for s in subsets])
        idx = np.ascontiguousarray(np.concatenate(subsets) if subsets else np.zeros(0), dtype=np.int32)
        nv = self.V if voxels is None else len(voxels)
        vx = None if voxels is None else np.ascontiguousarray(voxels, dtype=np.int64)
        out = np.empty((len(subsets), len(sp), nv))
        lib().oracle_psf(*self._args(), self.M, _p(sp), len(sp), _p(off), len(subsets), _p(idx),
                         _p(vx), nv, _p(out))
        return out

    def dense(self) -> np.ndarray:
        """Explicit J (M x V) by entry evaluation; tiny problems only."""
        F = np.zeros((self.M, self.V))
        eye = np.zeros(self.V)
        for v in range(self.V):
            eye[v] = 1.0
            F[:, v] = self.J(eye)
            eye[v] = 0.0
        return F
