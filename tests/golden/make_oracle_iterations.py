"""Write oracle_iterations.json: the CPU oracle's Jacobi-PCG iteration count to relative residual
1e-10 on the 256^3 hot-spot workload (rho = T0/T, 20k hot spots, density ratio 4, seed 2).

Only oracle/ and the seeded input recipes are used.  bench.py scales the oracle's measured time
per iteration on a bounded sample by this count to report the CPU baseline in solves/s.
Run: python tests/golden/make_oracle_iterations.py   (about 5 minutes on 8 cores)
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import vdp_inputs as V  # noqa: E402


def main():
    prob = V.config1()
    t0 = time.time()
    _, info = oracle.solve_cg(prob.rho, prob.f, prob.L, tol=prob.tol)
    out = {
        "workload": "256^3 periodic, rho=T0/T with 20k hot spots (ratio 4, seed 2), FP64 Jacobi-PCG, tol 1e-10",
        "oracle_iterations": info["iters"],
        "oracle_rel_res": info["rel_res"],
        "status": info["status"],
        "ratio": prob.info["ratio"],
        "seconds": round(time.time() - t0, 1),
        "threads": oracle.num_threads(),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_iterations.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
