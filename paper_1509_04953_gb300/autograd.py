"""torch.autograd.Function around the adjoint of the mechanical increments.

StressStrainCurve.apply(theta, setup) runs T recorded increments of the GPU solver with the
hardening / rate parameters theta = (k1, k2, tau0, n) and returns the macroscopic stress curve
<sigma33>_t (a float64 CPU tensor of length T). Its backward is the library's checkpointed discrete
adjoint (evp_adjoint_end): one adjoint Green-operator solve per increment, no finite differences.
Nucleation and phase-field steps are not part of this path.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import evp


@dataclasses.dataclass
class CurveSetup:
    n: int
    grains: int
    grain_id: np.ndarray
    quat: np.ndarray
    material: object
    seed: int
    increments: int
    dE33: float
    dt: float
    precision: str = "fp64"
    tol: float = 1e-12
    max_iter: int = 20000
    checkpoint_every: int = 0        # 0 = about sqrt(increments)
    adjoint_tol: float = 1e-10
    newton_tol: float | None = None


PARAMS = ("k1", "k2", "tau0", "n")


class StressStrainCurve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, setup: CurveSetup):
        th = theta.detach().cpu().double().numpy()
        mat = dataclasses.replace(setup.material, **{k: float(v) for k, v in zip(PARAMS, th)})
        kw = dict(tol=setup.tol, max_iter=setup.max_iter)
        if setup.newton_tol is not None:
            kw["newton_tol"] = setup.newton_tol
        s = evp.Solver(setup.n, setup.grains, setup.grain_id, setup.quat, mat, setup.seed,
                       precision=setup.precision, **kw)
        ck = setup.checkpoint_every or max(1, int(round(setup.increments ** 0.5)))
        s.adjoint_begin(setup.increments, ck)
        curve = [s.adjoint_step(setup.dE33, setup.dt).sig_mean[2] for _ in range(setup.increments)]
        ctx.solver = s
        ctx.setup = setup
        return torch.tensor(curve, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_curve):
        g = np.zeros((ctx.setup.increments, 6))
        g[:, 2] = grad_curve.detach().cpu().double().numpy()
        grad = ctx.solver.adjoint_end(g, tol=ctx.setup.adjoint_tol)
        ctx.solver.close()
        return torch.tensor(grad, dtype=torch.float64), None


def stress_strain_curve(theta, setup: CurveSetup):
    return StressStrainCurve.apply(theta, setup)
