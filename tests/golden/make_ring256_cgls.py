"""Write the stored expected result of the 30-iteration damped least-squares solve on the
full-size single-ring workload (256 transducers on a 100 mm ring, 32640 pairs, 200 x 200 x 40
voxels at 1 mm, nested cylinders +40 / -25 / +15 m/s, noise N(0, 5 ns) with seed 3, relative
damping 1e-3).

Everything comes from the FP64 oracle (Sec. II-D, Eq. leastSquare_misfit: CGLS on the damped
normal equations, m0 = 0, 30 iterations, no early stop; the damping is relative to the mean
diagonal of J^T J, computed by the oracle's own Frobenius norm) on the seeded inputs of
``workloads``. The oracle applies J and J^T 31 times each over 1.6 M voxels: about an hour and
a half on 8 host cores.

Stored in ``ring256_cgls30.npz``:
  d       float64[M]  the data the solve was given (J m_true + noise, oracle J)
  m       float32[V]  the model after 30 iterations
  hist    float64[31] |J^T r - lambda m|^2 before each iteration and after the last
  lam     float64     the absolute damping lambda
  frob2   float64     |J|_F^2

Usage: python tests/golden/make_ring256_cgls.py [threads]
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as wl  # noqa: E402


def main():
    if len(sys.argv) > 1:
        oracle.set_threads(int(sys.argv[1]))
    w = wl.ring256()
    og = oracle.Geometry.from_workload(w)
    t0 = time.time()
    d = og.J(wl.model_for(w)) + wl.noise(og.M, w.noise_seed)
    frob2 = og.frob2()
    lam = w.lambda_rel * frob2 / og.V
    print(f"data and |J|_F^2 in {time.time() - t0:.0f} s; lambda {lam:.6e}", flush=True)
    m, hist, rc = og.cgls(d, lam, w.cg_iters)
    if rc != 0:
        raise SystemExit(f"oracle CGLS status {rc}")
    print(f"CGLS in {time.time() - t0:.0f} s; |m| {np.linalg.norm(m):.6e}", flush=True)
    np.savez_compressed(os.path.join(HERE, "ring256_cgls30.npz"), d=d, m=m.astype(np.float32), hist=hist,
                        lam=np.float64(lam), frob2=np.float64(frob2))


if __name__ == "__main__":
    main()
