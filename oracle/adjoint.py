"""Oracle reverse mode: the float64 oracle step differentiated by PyTorch
autograd, for the adjoint parity tests.

TEST INFRASTRUCTURE ONLY.  The objective is the running x momentum of one
material's volume fraction, J = sum_n dt_n sum_cells phi_l (rho u) dx dy over
the states after each step, plus an optional linear functional <qbar, q_N> of
the final conservative state.  Each dt_n is the oracle's own CFL step
(Section 3: a fraction of the largest stable step), or a prescribed value,
and is held fixed under differentiation (it is a Python float).
"""
from __future__ import annotations

import torch

from .closures import history_material, phases, prim_to_cons
from .scheme import cons_from_array, cons_to_array, grid_of, prim_from_array, step

PARAM_KEYS = ("G", "sigma_y", "Q")


def rollout(init, kind, dim, mats, patch, opts, steps, material=-1, qbar=None, dts=None):
    """Returns (J, final conservative array, dts) as differentiable tensors.

    init: (nfields, ny, nx) primitive (kind "prim") or conservative array;
    mats: oracle material dicts whose G, sigma_y, Q entries may be tensors.
    """
    reactive = history_material(mats) is not None
    if kind == "prim":
        q = prim_to_cons(prim_from_array(init, dim, reactive), mats)
    else:
        q = cons_from_array(init, dim, reactive)
    grid = grid_of(patch, dim, opts.get("geometry", "planar"))
    dA = patch.dx * (patch.dy if dim == 2 else 1.0)
    J = torch.zeros((), dtype=torch.float64)
    used = []
    for n in range(steps):
        q, dt = step(q, grid, mats, opts, None if dts is None else dts[n])
        used.append(dt)
        if material >= 0:
            J = J + dt * dA * (phases(q["phi1"])[material] * q["mom"][..., 0]).sum()
    qN = cons_to_array(q, dim, reactive)
    if qbar is not None:
        J = J + (torch.as_tensor(qbar, dtype=torch.float64) * qN).sum()
    return J, qN, used


def with_params(mats, theta):
    """Copies of the material dicts with G, sigma_y, Q taken from the tensor
    theta[3 l + k] (k over G, sigma_y, Q)."""
    out = []
    for l, m in enumerate(mats):
        m2 = dict(m)
        for k, key in enumerate(PARAM_KEYS):
            m2[key] = theta[3 * l + k]
        out.append(m2)
    return out
