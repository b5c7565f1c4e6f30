"""Writes tests/golden/two_mode_golden.json: FP64 oracle results for the two exchange-coupled
Kerr modes (workloads.configs.two_mode: Eq. 301 network with two modes, N = 12 per mode,
T = 100 ns, dt = 0.01 ns, 10 000 RK4 steps) at the full horizon, for both methods:

* number basis (oracle.fock.rk4_adjoint, O1): the 9 x 9 low block (every mode index < 3, the
  paper's epsilon_r block), Tr(rho0 A(T)), and 256 elements of the 144 x 144 operator at
  seeded positions;
* mapping (oracle.mapping.rk4_mapped, O2): G_x and G_y of the single initial condition
  (144 coefficients each), 256 elements of R at seeded positions, the low block and
  Tr(rho0 A(T)) of the reconstructed operator.

Only the oracle is called.  Usage: python tests/golden/make_two_mode_golden.py
"""

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

N_SAMPLES = 256
SEED = 12


def cpl(a):
    a = np.asarray(a)
    return [a.real.tolist(), a.imag.tolist()]


def main():
    from oracle import fock, mapping
    from workloads import configs
    p = configs.two_mode()
    d = int(np.prod(p.N))
    rng = np.random.default_rng(SEED)
    pos = rng.choice(d * d, size=N_SAMPLES, replace=False)
    pos = sorted(int(x) for x in pos)
    A = fock.rk4_adjoint(p)
    rho = fock.operator_matrix(p.rho0_items(), p.N)
    direct = {"block": cpl(fock.low_block(A, p.N)), "tr_rho0_A": [float(np.trace(rho @ A).real), float(np.trace(rho @ A).imag)],
              "positions": pos, "values": cpl(A.reshape(-1)[pos])}
    run = mapping.rk4_mapped(p)
    assert len(run.ics) == 1
    _, _, w, C, Gx, Gy, R = run.ics[0]
    Am = run.fock_matrix()
    mapped = {"weight": [w.real, w.imag], "C": [C.real, C.imag], "gx": cpl(Gx), "gy": cpl(Gy),
              "r_positions": pos, "r_values": cpl(R.reshape(-1)[pos]),
              "block": cpl(fock.low_block(Am, p.N)),
              "tr_rho0_A": [float(np.trace(rho @ Am).real), float(np.trace(rho @ Am).imag)]}
    out = {"source": "oracle.fock.rk4_adjoint and oracle.mapping.rk4_mapped (FP64), workloads.configs.two_mode(): "
                     "N = 12 per mode, T = 100 ns, dt = 0.01 ns, 10000 RK4 steps; sample positions from "
                     f"numpy default_rng({SEED}).choice(144 * 144, {N_SAMPLES}, replace=False), sorted",
           "direct": direct, "mapped": mapped}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "two_mode_golden.json"), "w") as fh:
        json.dump(out, fh, indent=0)


if __name__ == "__main__":
    main()
