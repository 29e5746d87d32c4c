"""Write the stored expected results of the damped least-squares solves on the full-size
single-ring workload (256 transducers on a 100 mm ring, 32640 pairs, 200 x 200 x 40 voxels at
1 mm, nested cylinders +40 / -25 / +15 m/s, noise N(0, 5 ns) with seed 3, relative damping
1e-3).

Everything comes from the FP64 oracle (Sec. II-D, Eq. leastSquare_misfit: CGLS on the damped
normal equations, m0 = 0, a fixed number of iterations, no early stop; the damping is relative
to the mean diagonal of J^T J, computed by the oracle's own Frobenius norm) on the seeded
inputs of ``workloads``. The oracle applies J and J^T over 1.6 M voxels for every iteration:
the 30-iteration solve takes about an hour and a half on 8 host cores.

Stored in ``ring256_cgls30.npz``:
  d       float64[M]  the data the solves were given (J m_true + noise, oracle J)
  m       float32[V]  the model after 30 iterations
  hist    float64[31] |J^T r - lambda m|^2 before each iteration and after the last
  lam     float64     the absolute damping lambda
  frob2   float64     |J|_F^2
  m6      float32[V]  the model after 6 iterations
  hist6   float64[7]  its history
  Jm      float64[M]  J m (oracle) of the stored 30-iteration model (the predicted data)
  f       float64     the damped misfit 1/2 |J m - d|^2 + 1/2 lambda |m|^2 of that model

Usage: python tests/golden/make_ring256_cgls.py [threads] [--extend]
  --extend  keep d, m, hist, lam and frob2 of an existing file and add the other fields.
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

PATH = os.path.join(HERE, "ring256_cgls30.npz")


def main():
    args = [a for a in sys.argv[1:] if not a.startswith("--")]
    if args:
        oracle.set_threads(int(args[0]))
    w = wl.ring256()
    og = oracle.Geometry.from_workload(w)
    t0 = time.time()
    if "--extend" in sys.argv:
        old = np.load(PATH)
        out = {k: old[k] for k in ("d", "m", "hist", "lam", "frob2")}
        d, lam = out["d"], float(out["lam"])
    else:
        d = og.J(wl.model_for(w)) + wl.noise(og.M, w.noise_seed)
        frob2 = og.frob2()
        lam = w.lambda_rel * frob2 / og.V
        print(f"data and |J|_F^2 in {time.time() - t0:.0f} s; lambda {lam:.6e}", flush=True)
        m, hist, rc = og.cgls(d, lam, w.cg_iters)
        if rc != 0:
            raise SystemExit(f"oracle CGLS status {rc}")
        out = {"d": d, "m": m.astype(np.float32), "hist": hist, "lam": np.float64(lam), "frob2": np.float64(frob2)}
        print(f"CGLS({w.cg_iters}) in {time.time() - t0:.0f} s", flush=True)
    m6, hist6, rc = og.cgls(d, lam, 6)
    if rc != 0:
        raise SystemExit(f"oracle CGLS status {rc}")
    out["m6"] = m6.astype(np.float32)
    out["hist6"] = hist6
    m30 = out["m"].astype(np.float64)
    Jm = og.J(m30)
    out["Jm"] = Jm
    out["f"] = np.float64(0.5 * np.sum((Jm - d) ** 2) + 0.5 * lam * np.sum(m30 ** 2))
    print(f"CGLS(6), J m and the misfit in {time.time() - t0:.0f} s", flush=True)
    np.savez_compressed(PATH, **out)


if __name__ == "__main__":
    main()
