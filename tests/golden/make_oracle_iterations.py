"""Write oracle_iterations.json: the CPU oracle's Jacobi-PCG iteration count on the benchmark's two
large workloads, to each workload's tolerance.

  c1: 256^3 hot-spot workload (rho = T0/T, 20k hot spots, density ratio 4, seed 2), tol 1e-10
      (about 5 minutes on 8 cores);
  c2: 512^3 hot-spot workload (200k hot spots, density ratio capped at 10, seed 3), tol 1e-8
      (about an hour on 8 cores, 10 GB of memory).

Only oracle/ and the seeded input recipes are used.  bench.py scales the oracle's measured time
per iteration on a bounded sample by these counts to report the CPU baseline in solves/s.
Run: python tests/golden/make_oracle_iterations.py [c1] [c2]   (default: both; an entry that is
not recomputed is kept)
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import vdp_inputs as V  # noqa: E402

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_iterations.json")
WORKLOADS = {
    "c1": (V.config1, "256^3 periodic, rho=T0/T with 20k hot spots (ratio 4, seed 2), FP64 Jacobi-PCG, tol 1e-10"),
    "c2": (V.config2, "512^3 periodic, rho=T0/T with 200k hot spots (ratio capped at 10, seed 3), FP64 Jacobi-PCG, "
                      "tol 1e-8"),
}


def main(keys):
    out = {}
    if os.path.exists(PATH):
        with open(PATH) as fh:
            out = json.load(fh)
    for key in keys:
        make, text = WORKLOADS[key]
        prob = make()
        t0 = time.time()
        _, info = oracle.solve_cg(prob.rho, prob.f, prob.L, tol=prob.tol)
        out[key] = {
            "workload": text,
            "oracle_iterations": info["iters"],
            "oracle_rel_res": info["rel_res"],
            "status": info["status"],
            "ratio": prob.info["ratio"],
            "seconds": round(time.time() - t0, 1),
            "threads": oracle.num_threads(),
        }
        with open(PATH, "w") as fh:
            json.dump(out, fh, indent=1)
        print(json.dumps(out[key]), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(WORKLOADS))
