"""Helpers for the GPU parity tests: build both sides from the same seeded workload."""
from __future__ import annotations

import functools

import numpy as np

import oracle
import workloads as wl


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@functools.lru_cache(maxsize=None)
def oracle_geometry(name: str):
    w = wl.by_name(name) if name != "tiny" else wl.tiny()
    return w, oracle.Geometry.from_workload(w)


def gpu_geometry(w, dt_mode=0, tables=None):
    import paper_1908_03302_gb300 as fg
    if tables is None:
        tables = [fg.Table(b.f_center_hz, b.f_sigma_hz, b.n_samples, b.dt_max) for b in w.bands]
    geo = fg.Geometry(w.tx, w.row_pairs(), w.grid, w.c0, tables,
                      band_of_row=w.band_of_row if len(w.bands) > 1 else None, dt_mode=dt_mode)
    return geo, tables


def to_dev(x):
    import torch
    return torch.as_tensor(np.asarray(x, dtype=np.float32), device="cuda").contiguous()


def to_np(t):
    return t.detach().double().cpu().numpy()
