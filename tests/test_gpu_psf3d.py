"""Parity of the tensor-core PSF batch at the full size of the slice-by-slice workload, in the
launch configuration the benchmark times: 128 seeded spikes x 3 nested ring subsets (every
4th / 2nd / every element of each of the 16 rings, all 3 bands) over 1566720 rows and
256 x 256 x 96 voxels. The FP64 oracle computes the PSF values one by one at sampled voxels
around a few spikes (where the PSFs are large), for every subset; the bar is the BF16 path's
relative L2 <= 1e-2."""
import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_common import gpu_geometry, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_psf3d_tensor_cores_sampled_voxels():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = wl.slices3d()
    geo, _ = gpu_geometry(w)
    og = oracle.Geometry.from_workload(w)
    spikes = wl.random_voxels(w.grid, 128, 8)
    subsets = wl.ring_subsets(n_slices=16, n_bands=3)
    out = geo.psf_batch(spikes, subsets, mode=1)          # (3, 128, V) on the device
    rng = np.random.default_rng(34)
    g = w.grid
    for k in (0, 63, 127):
        vk = int(spikes[k])
        i, j, z = vk % g.nx, (vk // g.nx) % g.ny, vk // (g.nx * g.ny)
        off = rng.integers(-20, 21, size=(255, 3))
        ii = np.clip(i + off[:, 0], 0, g.nx - 1)
        jj = np.clip(j + off[:, 1], 0, g.ny - 1)
        zz = np.clip(z + off[:, 2], 0, g.nz - 1)
        vox = np.unique(np.concatenate([[vk], (zz * g.ny + jj) * g.nx + ii])).astype(np.int64)
        vt = torch.as_tensor(vox, device="cuda")
        for s in range(len(subsets)):
            ref = og.psf(np.array([vk]), [subsets[s]], vox)[0, 0]
            got = out[s, k][vt].double().cpu().numpy()
            assert np.linalg.norm(ref) > 0
            assert rel_l2(got, ref) <= 1e-2
    del out
    geo.close()
