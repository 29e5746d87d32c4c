"""GB300-native finite-frequency traveltime tomography (arXiv:1908.03302).

Python face of the CUDA library ``libfft_gb300.so`` (C ABI in ``include/fft_gb300.h``).
PyTorch supplies device memory and the current stream; the computation itself runs in the
library's kernels. The functions mirror the C entry points:

* ``fft_table_build``  - sample the Phi function of a source spectrum (Eq. Kernel_freq)
* ``fft_geom_create``  - rows, voxel grid and tables -> an operator handle (Eq. forward_compact)
* ``fft_J_apply`` / ``fft_JT_apply`` - d = J m and g = J^T d, entries rebuilt on the fly
* ``fft_cg_solve``     - damped least squares by CGLS (Eq. leastSquare_misfit);
  ``fft_cg_continue``, ``fft_cg_save`` / ``fft_cg_load`` resume a solve or checkpoint it
* ``fft_psf_batch``    - Hessian point-spread functions J_S^T J_S e_k (Eq. resolution_2)

``Table`` and ``Geometry`` wrap the handles; ``JFunction`` / ``jacobian_apply`` put J behind
``torch.autograd`` with J^T as its backward.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np

from . import _lib
from ._lib import (FFT_DT_FP64, FFT_DT_NAIVE, FFT_DT_STABLE, FFTError, check, fft_geom_info_t,
                   fft_grid, fft_spectrum)

__all__ = [
    "Table", "TrigTable", "Geometry", "JFunction", "jacobian_apply", "FFTError",
    "fft_table_build", "fft_trig_build", "fft_geom_create", "fft_J_apply", "fft_JT_apply", "fft_cg_solve", "fft_psf_batch",
    "FFT_DT_STABLE", "FFT_DT_NAIVE", "FFT_DT_FP64", "fresnel_width", "build",
]


def build(force: bool = False) -> str:
    """Compile libfft_gb300.so for sm_103a (no-op when up to date)."""
    from . import _buildlib
    return _buildlib.build(force=force)


def _torch():
    import torch
    return torch


def _stream_handle(stream=None) -> int:
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


def _dev_ptr(t, n: Optional[int] = None, name: str = "tensor") -> int:
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} must have {n} elements, got {t.numel()}")
    return int(t.data_ptr())


def fresnel_width(c0: float, length: float, f_center: float) -> float:
    """Width sqrt(c0 L / f) of the first Fresnel zone of a pair of length L (Sec. IV)."""
    return float(np.sqrt(c0 * length / f_center))


# --------------------------------------------------------------------------- tables

class Table:
    """Sampled Phi(dt_k), dt_k = k dt_max / (n - 1), built on the device in FP64."""

    def __init__(self, f_center: Optional[float] = None, f_sigma: Optional[float] = None, n: int = 4096,
                 dt_max: Optional[float] = None, omega: Optional[np.ndarray] = None,
                 weight: Optional[np.ndarray] = None, keep_host: bool = False):
        L = _lib.load()
        spec = fft_spectrum()
        self._keep = []
        if omega is None:
            spec.kind, spec.f_center_hz, spec.f_sigma_hz = 0, float(f_center), float(f_sigma)
            spec.omega = spec.weight = None
            spec.n_omega = 0
        else:
            om = np.ascontiguousarray(omega, dtype=np.float64)
            w = np.ascontiguousarray(weight, dtype=np.float64)
            self._keep = [om, w]
            spec.kind, spec.f_center_hz, spec.f_sigma_hz = 1, 0.0, 0.0
            spec.omega, spec.weight, spec.n_omega = om.ctypes.data, w.ctypes.data, len(om)
        if dt_max is None:
            dt_max = 3.0 / float(f_center)
        self.n = int(n)
        self.dt_max = float(dt_max)
        host = np.empty(self.n) if keep_host else None
        h = ctypes.c_void_p()
        check(L.fft_table_build(ctypes.byref(spec), self.n, self.dt_max,
                                None if host is None else host.ctypes.data, ctypes.byref(h)))
        self.handle = h
        self.host = host

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            _lib.load().fft_table_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class TrigTable(Table):
    """Phi as a short sine series (the form Sec. II-C stores): Phi(dt) = sum_j a_j sin(j dw dt)
    for a Gaussian power spectrum; ``n_terms`` 0 picks the count automatically. ``coef``,
    ``dw`` and ``n`` are the series the library built (host copies)."""

    def __init__(self, f_center: float, f_sigma: float, dt_max: Optional[float] = None, n_terms: int = 0):
        L = _lib.load()
        spec = fft_spectrum()
        spec.kind, spec.f_center_hz, spec.f_sigma_hz = 0, float(f_center), float(f_sigma)
        spec.omega = spec.weight = None
        spec.n_omega = 0
        self._keep = []
        self.dt_max = float(3.0 / float(f_center) if dt_max is None else dt_max)
        coef = np.empty(256)
        dw = ctypes.c_double()
        n = ctypes.c_int32()
        h = ctypes.c_void_p()
        check(L.fft_trig_build(ctypes.byref(spec), self.dt_max, int(n_terms), coef.ctypes.data,
                               ctypes.byref(dw), ctypes.byref(n), ctypes.byref(h)))
        self.handle = h
        self.n = int(n.value)
        self.dw = float(dw.value)
        self.coef = coef[:self.n].copy()
        self.host = None


def fft_table_build(f_center=None, f_sigma=None, n=4096, dt_max=None, omega=None, weight=None,
                    keep_host=False) -> Table:
    return Table(f_center, f_sigma, n, dt_max, omega, weight, keep_host)


# --------------------------------------------------------------------------- geometry

class Geometry:
    """Operator handle: rows (emitter, receiver, band), voxel grid, c0 and Phi tables."""

    def __init__(self, tx: np.ndarray, rows: np.ndarray, grid, c0: float, tables: Sequence[Table],
                 band_of_row: Optional[np.ndarray] = None, dt_mode: int = FFT_DT_STABLE):
        L = _lib.load()
        self._tx = np.ascontiguousarray(tx, dtype=np.float64).reshape(-1, 3)
        self._rows = np.ascontiguousarray(rows, dtype=np.int32).reshape(-1, 2)
        self._band = None if band_of_row is None else np.ascontiguousarray(band_of_row, dtype=np.int32)
        g = fft_grid()
        g.nx, g.ny, g.nz, g.h = int(grid.nx), int(grid.ny), int(grid.nz), float(grid.h)
        for a in range(3):
            g.origin[a] = float(grid.origin[a])
        self.grid = grid
        self.tables = list(tables)
        arr = (ctypes.c_void_p * len(self.tables))(*[t.handle.value for t in self.tables])
        h = ctypes.c_void_p()
        check(L.fft_geom_create(self._tx.ctypes.data, len(self._tx), self._rows.ctypes.data, len(self._rows),
                                None if self._band is None else self._band.ctypes.data, ctypes.byref(g),
                                float(c0), ctypes.cast(arr, ctypes.c_void_p), len(self.tables), int(dt_mode),
                                ctypes.byref(h)))
        self.handle = h
        self.c0 = float(c0)
        info = self.info()
        self.M = int(info.n_rows)
        self.V = int(info.n_vox)
        self._grid_nz = int(grid.nz)

    def info(self) -> fft_geom_info_t:
        out = fft_geom_info_t()
        check(_lib.load().fft_geom_info(self.handle, ctypes.byref(out)))
        return out

    def autotune(self, stream=None) -> dict:
        """Time J and J^T for twelve work decompositions (items per CTA x CTAs per SM) and keep
        the fastest (fft_geom_autotune)."""
        out = _lib.fft_tune_info_t()
        check(_lib.load().fft_geom_autotune(self.handle, _stream_handle(stream), ctypes.byref(out)))
        return {"items_per_cta": out.items_per_cta, "ctas_per_sm": out.ctas_per_sm, "ms_J": out.ms_J,
                "ms_JT": out.ms_JT, "candidates": out.n_tried}

    @property
    def support_evals(self) -> int:
        return int(self.info().support_evals)

    def J(self, m, out=None, stream=None):
        torch = _torch()
        if out is None:
            out = torch.empty(self.M, device=m.device, dtype=torch.float32)
        check(_lib.load().fft_J_apply(self.handle, _dev_ptr(m, self.V, "m"), _dev_ptr(out, self.M, "d"),
                                      _stream_handle(stream)))
        return out

    def JT(self, d, out=None, stream=None):
        torch = _torch()
        if out is None:
            out = torch.empty(self.V, device=d.device, dtype=torch.float32)
        check(_lib.load().fft_JT_apply(self.handle, _dev_ptr(d, self.M, "d"), _dev_ptr(out, self.V, "g"),
                                       _stream_handle(stream)))
        return out

    def J_batch(self, m, out=None, stream=None):
        """d[c] = J m[c] for the rows of m ((n, V) float32 CUDA tensor) -> (n, M)."""
        torch = _torch()
        if m.dim() != 2 or m.shape[1] != self.V:
            raise ValueError("m must be an (n, V) tensor")
        n = int(m.shape[0])
        if out is None:
            out = torch.empty((n, self.M), device=m.device, dtype=torch.float32)
        check(_lib.load().fft_J_apply_batch(self.handle, _dev_ptr(m), n, _dev_ptr(out, n * self.M, "d"),
                                            _stream_handle(stream)))
        return out

    def JT_batch(self, d, out=None, stream=None):
        """g[c] = J^T d[c] for the rows of d ((n, M) float32 CUDA tensor) -> (n, V)."""
        torch = _torch()
        if d.dim() != 2 or d.shape[1] != self.M:
            raise ValueError("d must be an (n, M) tensor")
        n = int(d.shape[0])
        if out is None:
            out = torch.empty((n, self.V), device=d.device, dtype=torch.float32)
        check(_lib.load().fft_JT_apply_batch(self.handle, _dev_ptr(d), n, _dev_ptr(out, n * self.V, "g"),
                                             _stream_handle(stream)))
        return out

    @property
    def V2(self) -> int:
        """Pixels of the plane (nx * ny) for the 2-D approximation."""
        return self.V // self._grid_nz

    def J2d(self, m2, out=None, stream=None):
        """d = J2 m2 (Eq. forward_2D): the operator integrated over the grid's z layers."""
        torch = _torch()
        if out is None:
            out = torch.empty(self.M, device=m2.device, dtype=torch.float32)
        check(_lib.load().fft_J2d_apply(self.handle, _dev_ptr(m2, self.V2, "m2"), _dev_ptr(out, self.M, "d"),
                                        _stream_handle(stream)))
        return out

    def JT2d(self, d, out=None, stream=None):
        """g2 = J2^T d: J^T summed over the grid's z layers per pixel."""
        torch = _torch()
        if out is None:
            out = torch.empty(self.V2, device=d.device, dtype=torch.float32)
        check(_lib.load().fft_JT2d_apply(self.handle, _dev_ptr(d, self.M, "d"), _dev_ptr(out, self.V2, "g2"),
                                         _stream_handle(stream)))
        return out

    def hessian_lowrank(self, omega, k: int, n_power: int = 1, sigma: float = 1.0, stream=None):
        """k dominant eigenpairs of H = J^T J / sigma^2 by randomized subspace iteration from the
        starting block omega (ell x V float32 CUDA tensor, one column per row). Returns
        (eigenvalues as a numpy array, descending; eigenvectors as a k x V tensor)."""
        torch = _torch()
        if omega.dim() != 2 or omega.shape[1] != self.V:
            raise ValueError("omega must be an (ell, V) tensor")
        ell = int(omega.shape[0])
        vecs = torch.empty((k, self.V), device=omega.device, dtype=torch.float32)
        lam = np.empty(k)
        check(_lib.load().fft_hessian_lowrank(self.handle, _dev_ptr(omega), ell, int(k), int(n_power), float(sigma),
                                              _dev_ptr(vecs), lam.ctypes.data, _stream_handle(stream)))
        return lam, vecs

    def lowrank_diag(self, vecs, eigvals, alpha: float, stream=None):
        """(diag of the low-rank posterior covariance, diag of the resolution matrix)."""
        torch = _torch()
        lam = np.ascontiguousarray(eigvals, dtype=np.float64)
        post = torch.empty(self.V, device=vecs.device, dtype=torch.float32)
        res = torch.empty(self.V, device=vecs.device, dtype=torch.float32)
        check(_lib.load().fft_lowrank_diag(self.handle, _dev_ptr(vecs), lam.ctypes.data, len(lam), float(alpha),
                                           _dev_ptr(post), _dev_ptr(res), _stream_handle(stream)))
        return post, res

    def coverage(self, w=None, out=None, device=None, stream=None):
        """Sensitivity coverage sum_p |J[p, v] w_p| per voxel (w: optional row weights)."""
        torch = _torch()
        if out is None:
            dev = w.device if w is not None else (device or torch.device("cuda", torch.cuda.current_device()))
            out = torch.empty(self.V, device=dev, dtype=torch.float32)
        check(_lib.load().fft_coverage(self.handle, None if w is None else _dev_ptr(w, self.M, "w"),
                                       _dev_ptr(out, self.V, "cov"), _stream_handle(stream)))
        return out

    def frob2(self) -> float:
        v = ctypes.c_double()
        check(_lib.load().fft_frob2(self.handle, ctypes.byref(v)))
        return v.value

    def cg_solve(self, d, lambda_rel: float, n_iter: int, m=None, with_history: bool = False, stream=None,
                 check_status: bool = True):
        """CGLS on the damped normal equations (fft_cg_solve). The library call is asynchronous
        without a history; check_status then waits for the solve (fft_cg_status) and raises
        FFTError on a breakdown. check_status=False leaves the solve in flight: call
        cg_status() later."""
        torch = _torch()
        if m is None:
            m = torch.zeros(self.V, device=d.device, dtype=torch.float32)
        hist = np.empty(n_iter + 1) if with_history else None
        check(_lib.load().fft_cg_solve(self.handle, _dev_ptr(d, self.M, "d"), float(lambda_rel), int(n_iter),
                                       _dev_ptr(m, self.V, "m"), None if hist is None else hist.ctypes.data,
                                       _stream_handle(stream)))
        if hist is None and check_status:
            self.cg_status(stream)
        return (m, hist) if with_history else m

    def cg_status(self, stream=None) -> None:
        """Wait for the last solve on `stream` and raise FFTError if it broke down."""
        check(_lib.load().fft_cg_status(self.handle, _stream_handle(stream)))

    def cg_continue(self, n_iter: int, m=None, with_history: bool = False, stream=None, check_status: bool = True):
        """n_iter more CGLS iterations from the handle's state (fft_cg_continue); returns the
        model (written into `m` when given)."""
        torch = _torch()
        if m is None:
            m = torch.empty(self.V, device="cuda", dtype=torch.float32)
        hist = np.empty(n_iter + 1) if with_history else None
        check(_lib.load().fft_cg_continue(self.handle, int(n_iter), _dev_ptr(m, self.V, "m"),
                                          None if hist is None else hist.ctypes.data, _stream_handle(stream)))
        if hist is None and check_status:
            self.cg_status(stream)
        return (m, hist) if with_history else m

    def cg_save(self, stream=None) -> np.ndarray:
        """The handle's CG state as a host byte array (fft_cg_save), e.g. to write to a file."""
        n = ctypes.c_int64()
        check(_lib.load().fft_cg_state_bytes(self.handle, ctypes.byref(n)))
        buf = np.empty(n.value, dtype=np.uint8)
        check(_lib.load().fft_cg_save(self.handle, buf.ctypes.data, n.value, _stream_handle(stream)))
        return buf

    def cg_load(self, state, stream=None) -> None:
        """Replace the handle's CG state by one saved with cg_save (fft_cg_load)."""
        buf = np.ascontiguousarray(state, dtype=np.uint8)
        check(_lib.load().fft_cg_load(self.handle, buf.ctypes.data, buf.size, _stream_handle(stream)))

    def psf_batch(self, spikes: Sequence[int], subsets: Sequence[np.ndarray], mode: int = 0, out=None, stream=None):
        torch = _torch()
        sp = np.ascontiguousarray(spikes, dtype=np.int64)
        off = np.zeros(len(subsets) + 1, dtype=np.int32)
        off[1:] = np.cumsum([len(s) for s in subsets])
        idx = np.ascontiguousarray(np.concatenate([np.asarray(s, dtype=np.int32) for s in subsets])
                                   if len(subsets) else np.zeros(0, np.int32), dtype=np.int32)
        n = len(subsets) * len(sp) * self.V
        if out is None:
            out = torch.empty(n, device="cuda", dtype=torch.float32)
        check(_lib.load().fft_psf_batch(self.handle, sp.ctypes.data, len(sp), off.ctypes.data, len(subsets),
                                        idx.ctypes.data if len(idx) else None, int(mode), _dev_ptr(out, n, "out"),
                                        _stream_handle(stream)))
        return out.view(len(subsets), len(sp), self.V)

    def psf_noalloc(self, spike: int, rows_dev, out=None, stream=None):
        """One PSF (spike, row subset given as a device int32 tensor) with no device allocation
        inside the library; the result tensor is allocated here unless `out` is given."""
        torch = _torch()
        if not (isinstance(rows_dev, torch.Tensor) and rows_dev.is_cuda and rows_dev.dtype == torch.int32
                and rows_dev.is_contiguous()):
            raise TypeError("rows_dev must be a contiguous int32 CUDA tensor")
        if out is None:
            out = torch.empty(self.V, device=rows_dev.device, dtype=torch.float32)
        check(_lib.load().fft_psf_noalloc(self.handle, int(spike), int(rows_dev.data_ptr()), int(rows_dev.numel()),
                                          _dev_ptr(out, self.V, "out"), _stream_handle(stream)))
        return out

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            _lib.load().fft_geom_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fft_trig_build(f_center, f_sigma, dt_max=None, n_terms=0) -> TrigTable:
    return TrigTable(f_center, f_sigma, dt_max, n_terms)


def fft_geom_create(tx, rows, grid, c0, tables, band_of_row=None, dt_mode=FFT_DT_STABLE) -> Geometry:
    return Geometry(tx, rows, grid, c0, tables, band_of_row, dt_mode)


def fft_J_apply(geom: Geometry, m, d=None, stream=None):
    return geom.J(m, d, stream)


def fft_JT_apply(geom: Geometry, d, g=None, stream=None):
    return geom.JT(d, g, stream)


def fft_cg_solve(geom: Geometry, d, lambda_rel: float, n_iter: int, m=None, with_history=False, stream=None):
    return geom.cg_solve(d, lambda_rel, n_iter, m, with_history, stream)


def fft_psf_batch(geom: Geometry, spikes, subsets, mode=0, out=None, stream=None):
    return geom.psf_batch(spikes, subsets, mode, out, stream)


def psf_row_groups(n_rows: int, subsets: Sequence[np.ndarray]):
    """Rows grouped by the set of subsets that hold them (fft_psf_row_groups, host only):
    returns (grp, gmask) with grp[p] the group of row p (255: in no subset) and gmask[g] the
    subsets of group g as a bit mask, or (None, None) for more than 32 groups."""
    off = np.zeros(len(subsets) + 1, dtype=np.int32)
    off[1:] = np.cumsum([len(s) for s in subsets])
    idx = np.ascontiguousarray(np.concatenate([np.asarray(s, dtype=np.int32) for s in subsets])
                               if len(subsets) else np.zeros(0, np.int32), dtype=np.int32)
    grp = np.empty(int(n_rows), dtype=np.uint8)
    gmask = np.zeros(32, dtype=np.uint32)
    ng = ctypes.c_int32()
    check(_lib.load().fft_psf_row_groups(int(n_rows), off.ctypes.data, len(subsets),
                                         idx.ctypes.data if len(idx) else None, grp.ctypes.data,
                                         gmask.ctypes.data, ctypes.byref(ng)))
    if ng.value < 0:
        return None, None
    return grp, gmask[: ng.value].copy()


def tc_selftest(n: int = 128, k: int = 64) -> float:
    """Largest absolute error of a 128 x n x k BF16 tensor-core product against the exact one."""
    err = ctypes.c_double()
    check(_lib.load().fft_tc_selftest(int(n), int(k), ctypes.byref(err)))
    return err.value


# --------------------------------------------------------------------------- autograd

def _make_jfunction():
    torch = _torch()

    class JFunction(torch.autograd.Function):
        """d = J m with the hand-written adjoint as backward: grad_m = J^T grad_d."""

        @staticmethod
        def forward(ctx, m, geom):
            ctx.geom = geom
            return geom.J(m.contiguous())

        @staticmethod
        def backward(ctx, grad_d):
            return ctx.geom.JT(grad_d.contiguous()), None

    return JFunction


_JF = None


def __getattr__(name):
    global _JF
    if name == "JFunction":
        if _JF is None:
            _JF = _make_jfunction()
        return _JF
    raise AttributeError(name)


def jacobian_apply(m, geom: Geometry):
    """Differentiable d = J m (backward runs the J^T kernel)."""
    global _JF
    if _JF is None:
        _JF = _make_jfunction()
    return _JF.apply(m, geom)
