"""Pins for the oracle's detour, K0, J and J^T (Sec. II-B/C, Eqs. Linearized_sensitivity,
Kernel_freq, forward_ffttt, forward_compact).

* detour: the cancellation-free form against the textbook sum of distances in FP64, exact
  zeros on the ray, and the closed value 2(|p| - L/2) on the axis beyond the transducers;
* K0: zero on the ray, reciprocity bit for bit, negative first Fresnel zone, alternating
  signs further out;
* the ray-theory limit: a uniform perturbation gives dT = -L dc / c0^2, checked by
  prolate-spheroidal quadrature of K0 (exact up to the truncated Phi mass) and by the voxel
  sum of J on a fine grid;
* brute force: the cross-correlation traveltime of Born-scattered waveforms from a single
  point scatterer, with the Phi table built from that wavelet's own spectrum;
* J^T is the transpose of J (dense matrix and dot-product test).
"""
import math

import numpy as np
import pytest

import oracle
import workloads as wl
from oracle import closed_form as cf

C0 = 1500.0


def _tab(fc=1e6, fs=0.3e6, n=4096):
    return oracle.phi_table_gauss(fc, fs, n, 3.0 / fc), 3.0 / fc


def test_detour_forms_agree_fp64():
    rng = np.random.default_rng(3)
    for _ in range(200):
        xs, xr = rng.uniform(-0.1, 0.1, 3), rng.uniform(-0.1, 0.1, 3)
        x = rng.uniform(-0.1, 0.1, 3)
        R, rs, rr, L = oracle.detour(xs, xr, x)
        assert R >= 0.0
        assert abs(R - oracle.detour_naive(xs, xr, x)) < 1e-15
        assert rs == pytest.approx(np.linalg.norm(x - xs), rel=1e-14)
        assert rr == pytest.approx(np.linalg.norm(x - xr), rel=1e-14)
        assert L == pytest.approx(np.linalg.norm(xr - xs), rel=1e-14)


def test_detour_on_and_beyond_the_ray():
    # exactly on the segment (axis-aligned pair): R is exactly 0
    xa, xb = np.array([-0.05, 0.01, 0.0]), np.array([0.05, 0.01, 0.0])
    for t in (0.0, 0.1, 0.5, 0.77, 1.0):
        R, *_ = oracle.detour(xa, xb, xa + t * (xb - xa))
        assert R == 0.0
    # oblique segment: the point is on the ray up to its own rounding, R at rounding level
    xs, xr = np.array([-0.05, 0.01, 0.0]), np.array([0.05, -0.02, 0.003])
    for t in (0.0, 0.1, 0.5, 0.77, 1.0):
        R, *_ = oracle.detour(xs, xr, xs + t * (xr - xs))
        assert 0.0 <= R < 1e-18
    e = (xr - xs) / np.linalg.norm(xr - xs)
    for beyond in (1e-3, 2e-2):
        R, *_ = oracle.detour(xs, xr, xr + beyond * e)
        assert R == pytest.approx(2 * beyond, rel=1e-12)


def test_k0_zero_on_ray_and_reciprocal():
    tab, dtm = _tab()
    xs, xr = np.array([-0.095, 0.0, 0.0]), np.array([0.095, 0.0, 0.0])
    for t in np.linspace(0.01, 0.99, 17):
        assert oracle.k0(xs, xr, xs + t * (xr - xs), C0, tab, dtm) == 0.0
    rng = np.random.default_rng(5)
    for _ in range(100):
        x = np.array([rng.uniform(-0.09, 0.09), rng.uniform(-0.01, 0.01), rng.uniform(-0.01, 0.01)])
        assert oracle.k0(xs, xr, x, C0, tab, dtm) == oracle.k0(xr, xs, x, C0, tab, dtm)


def test_fresnel_zone_signs():
    # Fig. 1: negative first Fresnel zone, alternating signs further out, decaying.
    tab, dtm = _tab()
    xs, xr = np.array([-0.095, 0.0, 0.0]), np.array([0.095, 0.0, 0.0])
    L = 0.19
    vals = []
    for R in np.linspace(1e-5, C0 * dtm * 0.999, 600):
        # point in the mid-plane with detour R: 2 sqrt((L/2)^2 + y^2) - L = R
        y = math.sqrt((0.5 * (L + R)) ** 2 - (0.5 * L) ** 2)
        vals.append(oracle.k0(xs, xr, np.array([0.0, y, 0.0]), C0, tab, dtm))
    vals = np.array(vals)
    assert np.all(vals[:20] < 0)
    signs = np.sign(vals[np.abs(vals) > 1e-3 * np.abs(vals).max()])
    changes = np.count_nonzero(np.diff(signs) != 0)
    assert changes >= 3
    assert np.abs(vals[-100:]).max() < 0.2 * np.abs(vals).max()


@pytest.mark.parametrize("xs,xr", [((-0.05, 0.0, 0.0), (0.05, 0.0, 0.0)),
                                   ((-0.07, 0.02, 0.01), (0.03, -0.06, -0.01))])
def test_uniform_dc_prolate_quadrature(xs, xr):
    tab, dtm = _tab()
    xs, xr = np.array(xs), np.array(xr)
    L = np.linalg.norm(xr - xs)
    got = cf.uniform_dc_prolate(lambda x: oracle.k0(xs, xr, x, C0, tab, dtm), xs, xr, C0, dtm,
                                len(tab), n_tau=3, n_phi=3, sub=1)
    mass = np.trapezoid(tab, dx=dtm / (len(tab) - 1))
    assert got == pytest.approx(-(L / C0 ** 2) * mass, rel=1e-9)
    assert got == pytest.approx(-L / C0 ** 2, rel=1e-5)


def test_uniform_dc_voxel_sum():
    # J applied to a uniform 1 m/s perturbation on a 0.5 mm grid enclosing the whole support
    # of one 100 mm pair gives the ray-theory traveltime -L / c0^2 to within 1 %.
    tab, dtm = _tab()
    xs, xr = np.array([-0.05, 0.0, 0.0]), np.array([0.05, 0.0, 0.0])
    h = 0.5e-3
    grid = wl.Grid.centred(216, 68, 68, h)
    geo = oracle.Geometry(np.stack([xs, xr]), np.array([[0, 1]]), None, [tab], [dtm], grid, C0)
    dT = geo.J(np.ones(grid.n_vox))[0]
    assert dT == pytest.approx(-0.1 / C0 ** 2, rel=1e-2)


@pytest.mark.parametrize("zone_R", [0.2e-3, 0.6e-3, 1.2e-3, 2.1e-3])
def test_born_brute_force(zone_R):
    """CC traveltime of p0 + dp (point scatterer) equals K0(x') dc dV to O(dc)."""
    fc, rel_sig = 1.0e6, 0.3
    w0 = 2 * math.pi * fc
    a = (2 * math.pi * rel_sig * fc) ** 2           # |F|^2 has std sqrt(a) in omega
    om = np.linspace(0.0, w0 + 14 * math.sqrt(a), 24001)
    W = cf.wavelet_spectrum(om, a, w0) ** 2
    dtm = 3.0 / fc
    tab = oracle.phi_table_sampled(om, W, 4096, dtm)
    xs, xr = np.array([-0.05, 0.0, 0.0]), np.array([0.05, 0.0, 0.0])
    L = 0.1
    # a point with the requested detour, off the mid-plane and off the z = 0 plane
    px, ang = 0.013, 0.7
    # solve |x-xs| + |x-xr| = L + R for the radius q at axial position px
    lo, hi = 0.0, 0.05
    for _ in range(200):
        q = 0.5 * (lo + hi)
        x = np.array([px, q * math.cos(ang), q * math.sin(ang)])
        if np.linalg.norm(x - xs) + np.linalg.norm(x - xr) - L < zone_R:
            lo = q
        else:
            hi = q
    K = oracle.k0(xs, xr, x, C0, tab, dtm)
    errs = []
    for frac in (1e-3, 1e-4):
        eps = frac * C0 * 1e-9          # dc * dV with dV = 1 mm^3
        dT = cf.born_cc_traveltime(xs, xr, x, eps, C0, a, w0, om)
        errs.append(abs(dT / eps - K))
    scale = abs(K) + 1e-3 * 7e-3        # guard near a zero crossing of Phi
    assert errs[1] / scale < 1e-3
    # the remaining error is the linearisation: it falls with the perturbation strength
    assert errs[1] < 0.5 * errs[0] or errs[1] / scale < 1e-5


def test_J_JT_transpose_and_dot_product():
    w = wl.tiny()
    geo = oracle.Geometry.from_workload(w)
    F = geo.dense()
    rng = np.random.default_rng(11)
    m = rng.normal(size=geo.V)
    d = rng.normal(size=geo.M)
    assert np.allclose(geo.J(m), F @ m, rtol=1e-12, atol=1e-12 * np.abs(F @ m).max())
    jt = geo.JT(d)
    ref = F.T @ d
    assert np.max(np.abs(jt - ref)) <= 1e-12 * np.max(np.abs(ref))
    lhs, rhs = np.dot(geo.J(m), d), np.dot(m, jt)
    assert abs(lhs - rhs) <= 1e-14 * np.linalg.norm(geo.J(m)) * np.linalg.norm(d)
    # entries: reciprocity of the rows, and row sums of J are the ray traveltime scale
    assert geo.entry(0, 100) == F[0, 100]
    # selected rows / voxels equal the full products
    rows = np.array([3, 0, 17], dtype=np.int64)
    assert np.array_equal(geo.J(m, rows), geo.J(m)[rows])
    vox = np.array([5, 600, 1000], dtype=np.int64)
    assert np.array_equal(geo.JT(d, vox), jt[vox])


def test_support_count_matches_ellipsoid_volume():
    # One pair well inside the grid: the number of voxels with dt < dt_max approaches the
    # prolate-spheroid volume (4/3) pi a b^2 / h^3, a = (L + R)/2, b^2 = a^2 - (L/2)^2.
    tab, dtm = _tab()
    xs, xr = np.array([-0.02, 0.0, 0.0]), np.array([0.02, 0.0, 0.0])
    h = 0.25e-3
    grid = wl.Grid.centred(184, 84, 84, h)   # encloses a = 22.25 mm, b = 9.75 mm
    geo = oracle.Geometry(np.stack([xs, xr]), np.array([[0, 1]]), None, [tab], [dtm], grid, C0)
    Rm = C0 * dtm
    a = 0.5 * (0.04 + Rm)
    b2 = a * a - 0.02 ** 2
    vol = 4.0 / 3.0 * math.pi * a * b2 / h ** 3
    assert geo.count_support() == pytest.approx(vol, rel=5e-3)


def test_k0_zero_exactly_at_the_transducers():
    # K0 has no single limit at a transducer; the definition sets it to 0 there. For oblique
    # pairs the pair-frame distance rounds to ~1e-18 m instead of 0, so the rule must look at
    # the coordinates themselves.
    tab, dtm = _tab()
    rng = np.random.default_rng(12)
    for _ in range(50):
        xs, xr = rng.uniform(-0.05, 0.05, 3), rng.uniform(-0.05, 0.05, 3)
        assert oracle.k0(xs, xr, xs, C0, tab, dtm) == 0.0
        assert oracle.k0(xs, xr, xr.copy(), C0, tab, dtm) == 0.0
        # a point 1 um away has a finite, non-zero value of at most the scale near the emitter
        x = xs + 1e-6 * (xr - xs) / np.linalg.norm(xr - xs)
        assert np.isfinite(oracle.k0(xs, xr, x, C0, tab, dtm))


def test_multi_band_rows_use_their_own_band():
    # Rows of band b use band b's table and cut-off (Sec. VI: measurements in several frequency
    # bands): a two-band operator equals, row by row, the single-band operators, and its
    # adjoint is the sum of theirs over each band's rows.
    w = wl.tiny()
    rows = w.row_pairs()
    bor = (np.arange(len(rows)) % 2).astype(np.int32)
    bands = [(1.0e6, 0.3e6), (1.4e6, 0.2e6)]
    dtm = [3.0 / fc for fc, _ in bands]
    tabs = [oracle.phi_table_gauss(fc, fs, 1024, d) for (fc, fs), d in zip(bands, dtm)]
    two = oracle.Geometry(w.tx, rows, bor, tabs, dtm, w.grid, w.c0)
    one = [oracle.Geometry(w.tx, rows, None, [tabs[b]], [dtm[b]], w.grid, w.c0) for b in range(2)]
    rng = np.random.default_rng(21)
    m = rng.normal(size=two.V)
    d = rng.normal(size=two.M)
    J2 = two.J(m)
    for b in range(2):
        sel = bor == b
        assert np.array_equal(J2[sel], one[b].J(m)[sel])
    ref = one[0].JT(np.where(bor == 0, d, 0.0)) + one[1].JT(np.where(bor == 1, d, 0.0))
    assert np.max(np.abs(two.JT(d) - ref)) <= 1e-12 * np.max(np.abs(ref))
    # the bands differ, so a mix-up of tables would show
    J0, J1 = one[0].J(m), one[1].J(m)
    assert np.linalg.norm(J0 - J1) > 0.1 * np.linalg.norm(J0)
