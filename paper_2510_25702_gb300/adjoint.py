"""Gradients of the outlet mass flux with respect to an inlet velocity profile.

`OutletFlux` is a torch.autograd.Function over a differentiated window of
the C-ABI library: its forward runs sph_adjoint_forward (the window's
steps with checkpoints) and returns J; its backward runs the hand-written
reverse (sph_adjoint_backward) and returns dJ/dtheta scaled by the incoming
gradient.  All the arithmetic of both passes runs in the library's CUDA
kernels; this module only marshals arguments.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Sequence

import numpy as np


@dataclass
class Window:
    """A differentiated window: `steps` advection steps of `instance`,
    profile of velocity buffer `profile_buffer`, flux out of the `outlets`
    buffers normalised by `slab`, a snapshot every `checkpoint_every` steps.
    The window starts from the simulation's state at the start slot."""

    sim: object
    instance: int
    profile_buffer: int
    outlets: Sequence[int]
    steps: int
    checkpoint_every: int
    slab: float

    def forward(self, theta) -> float:
        return self.sim.adjoint_forward(theta, self.instance, self.profile_buffer, self.outlets, self.steps,
                                        self.checkpoint_every, self.slab)

    def backward(self) -> np.ndarray:
        return self.sim.adjoint_backward()


def _torch():
    import torch

    return torch


class OutletFlux:
    """theta (torch float64 tensor, n_theta) -> J (0-d tensor); call
    OutletFlux.apply(theta, window)."""

    _fn = None

    @classmethod
    def apply(cls, theta, window: Window):
        if cls._fn is None:
            torch = _torch()

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(ctx, th, win):
                    J = win.forward(th.detach().cpu().numpy().astype(np.float64))
                    ctx.win = win
                    return th.new_tensor(J)

                @staticmethod
                def backward(ctx, gJ):
                    g = ctx.win.backward()
                    return gJ * gJ.new_tensor(g), None

            cls._fn = _F
        return cls._fn.apply(theta, window)


def fd_gradient(window: Window, theta, start_slot: int, rel_step: float = 1e-6, directions=None):
    """Central finite differences of the window's J, each run from the state
    saved in start_slot.  directions: None (every theta component) or an
    array of unit directions (rows); returns the derivatives along them."""
    sim = window.sim
    theta = np.asarray(theta, np.float64)
    dirs = np.eye(theta.size) if directions is None else np.atleast_2d(np.asarray(directions, np.float64))
    h = rel_step * max(np.abs(theta).max(), 1e-12)
    out = np.zeros(len(dirs))
    once = Window(sim, window.instance, window.profile_buffer, window.outlets, window.steps, window.steps,
                  window.slab)
    for q, u in enumerate(dirs):
        sim.restore_state(start_slot)
        jp = once.forward(theta + h * u)
        sim.restore_state(start_slot)
        jm = once.forward(theta - h * u)
        out[q] = (jp - jm) / (2 * h)
    sim.restore_state(start_slot)
    sim.adjoint_release()
    return out
