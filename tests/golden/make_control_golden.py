"""Writes tests/golden/control_golden.json: loss and gradient of the two-mode control problem
(workloads.configs.two_mode_control: 64 piecewise-constant drive segments, seed 5526,
T = 200 ns, dt = 200/64/320 ns, 20 480 RK4 steps) from the FP64 oracle's discrete adjoint
(oracle.grad.loss_and_grad, checkpoint interval 160).  Only the oracle is called.

Usage: python tests/golden/make_control_golden.py
"""

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

if __name__ == "__main__":
    from oracle import grad
    from workloads import configs
    p = configs.two_mode_control()
    loss, gt, gp = grad.loss_and_grad(p, checkpoint_every=160)
    out = {"source": "oracle.grad.loss_and_grad (FP64), workloads.configs.two_mode_control() defaults",
           "loss": loss, "grad_theta": list(map(float, gt)),
           "grad_pwc": [list(map(float, row)) for row in gp[0]],
           "params": list(p.params)}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "control_golden.json"), "w") as fh:
        json.dump(out, fh, indent=1)
