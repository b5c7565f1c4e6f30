"""Writes tests/golden/kerr_batch_golden.json: FP64 oracle results (oracle.mapping, the
paper's mapping method step by step) for sampled instances of the seeded 4096-instance
driven damped Kerr batch at the full horizon (T = 100 ns, dt = 0.002 ns, 50 000 RK4 steps).

Only the oracle is called.  Usage: python tests/golden/make_kerr_batch_golden.py [n_proc]
"""

import json
import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

SAMPLES = list(range(0, 4096, 256)) + [4095]


def one(i):
    from oracle import mapping
    from workloads import configs
    p = configs.kerr_batch(B=i + 1)[i]
    A = mapping.rk4_mapped(p).fock_matrix()
    blk = A[:3, :3]
    return {"index": i, "N": p.N[0], "tr_rho0_A": [A[0, 0].real, A[0, 0].imag],
            "block_re": blk.real.tolist(), "block_im": blk.imag.tolist()}


if __name__ == "__main__":
    n_proc = int(sys.argv[1]) if len(sys.argv) > 1 else 8
    ctx = mp.get_context("spawn")
    with ctx.Pool(n_proc) as pool:
        res = pool.map(one, SAMPLES)
    out = {"source": "oracle.mapping.rk4_mapped (FP64), workloads.configs.kerr_batch seed 20220311, "
                     "T=100 ns, dt=0.002 ns, grid = Fock truncation N", "results": res}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "kerr_batch_golden.json"), "w") as fh:
        json.dump(out, fh, indent=1)
