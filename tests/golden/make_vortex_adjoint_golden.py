"""Write the oracle's kinetic-energy gradient for the 8^3 warped p=4 isentropic-vortex workload.

Calls only the CPU oracle (autograd through 50 fixed DP5 steps, one checkpoint per residual) and
the seeded input module.  Output: vortex_8cubed_p4_50steps_oracle_grad.json with the time step,
KE(q_50), d KE/d mu and d KE/d q_0 . u for the seeded directions used by the GPU test.
Run: python tests/golden/make_vortex_adjoint_golden.py   (a few minutes on CPU)
"""
import json
import math
import os
import sys
import time

import torch
import torch.utils.checkpoint as ckp

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
from oracle import esdc_oracle as O  # noqa: E402
from paper_1911_10966_gb300 import inputs as I  # noqa: E402

P, K, STEPS, MA, RE = 4, 8, 50, 0.5, 1000.0
SEEDS = (1234, 99)


def main():
    t0 = time.time()
    s = O.sbp_operator(P)
    x = I.box_coords(s.xi.numpy(), K, K, K, [-5.0] * 3, [5.0] * 3, warp=0.1, seed=1)
    mesh = O.make_mesh(P, x, K, K, K)
    gas = O.Gas.from_mach(MA, RE)
    q0 = torch.tensor(I.isentropic_vortex(x, Ma=MA, u_inf=(1 / math.sqrt(2), -1 / math.sqrt(2), 0.0)))
    dt = O.cfl_dt(q0, mesh, gas, 0.5)
    qq = q0.clone().requires_grad_(True)
    mu = torch.tensor(gas.mu, dtype=torch.float64, requires_grad=True)
    g2 = O.Gas(gas.gamma, gas.R, mu, gas.Pr)
    f = lambda st: ckp.checkpoint(lambda a: O.rhs(a, mesh, g2), st, use_reentrant=False)
    ke = O.kinetic_energy(O.rk_step(qq, f, dt, STEPS), mesh)
    gq, gmu = torch.autograd.grad(ke, (qq, mu))
    out = {"workload": "isentropic vortex, 8^3 warped (0.1h, seed 1) p=4 on [-5,5]^3, Ma 0.5, Re 1000, 50 DP5 steps",
           "dt": dt, "ke_final": float(ke.detach()), "dke_dmu": float(gmu), "directional": {}}
    for seed in SEEDS:
        g = torch.Generator().manual_seed(seed)
        u = torch.randn(q0.shape, generator=g, dtype=torch.float64) * q0.abs().amax(dim=(0, 2, 3, 4), keepdim=True)
        out["directional"][str(seed)] = float((gq * u).sum())
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "vortex_8cubed_p4_50steps_oracle_grad.json")
    json.dump(out, open(path, "w"), indent=1)
    print(json.dumps(out), f"{time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
