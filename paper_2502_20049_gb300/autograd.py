"""torch.autograd.Function around the PSM forward run and its discrete adjoint.

PSMTorque.apply(eps_delta, omega, u_in, case, steps, K) runs `steps` PSM steps
of `case` (libpsm) with body 0 rotating at `omega`, inflow `u_in` and the
per-cell solid-fraction perturbation `eps_delta`, from f^eq(rho0, u_in), and
returns J = mean torque about z on body 0.  Its backward calls psm_backward
(checkpoint every K steps, recompute, adjoint sweep) and returns dJ/d eps_delta
(per cell), dJ/d omega (the geometry sequence held fixed) and dJ/d u_in.
"""

from __future__ import annotations

import numpy as np
import torch

from . import psm
from . import workloads as W


class PSMTorque(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps_delta, omega, u_in, case: "W.Case", steps: int, K: int):
        om = tuple(float(v) for v in omega.detach().cpu().tolist())
        ui = tuple(float(v) for v in u_in.detach().cpu().tolist())
        bodies = list(case.bodies)
        b0 = bodies[0]
        bodies[0] = W.BodyCase(b0.kind, b0.params, b0.s, b0.R0, omega=om, v=b0.v, Q0=b0.Q0)
        c = case.with_(u_in=ui, bodies=bodies)
        sol = psm.Solver.from_case(c)
        sol.set_eps_delta(eps_delta)
        n0 = sol.step_count
        sol.record(K, init_from_inflow=True)
        sol.step(steps)
        ft = sol.force_torque(0, n0, steps)
        ctx.sol = sol
        ctx.device = eps_delta.device
        ctx.dtype = eps_delta.dtype
        return torch.tensor(float(ft[:, 5].mean()), dtype=torch.float64, device=eps_delta.device)

    @staticmethod
    def backward(ctx, gJ):
        # the eps gradient is written straight into a tensor on eps_delta's
        # device (HBM for a CUDA tensor: no host round trip)
        c = ctx.sol.cfg
        ge = torch.empty((c.nz, c.ny, c.nx), dtype=torch.float64, device=ctx.device)
        _, gw, gu = ctx.sol.backward(grad_eps=ge)
        g = float(gJ)
        ctx.sol.close()
        grad_eps = (ge * g).to(dtype=ctx.dtype)
        grad_omega = torch.from_numpy(np.asarray(gw[0]) * g)
        grad_u = torch.from_numpy(np.asarray(gu) * g)
        return grad_eps, grad_omega, grad_u, None, None, None
