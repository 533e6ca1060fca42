"""torch.autograd.Function for the absorption efficiency Q_abs.

The forward pass is a DDA solve on the GPU for one incident plane wave,
with the dielectric function given per dipole; the backward pass returns
dQ_abs/d(eps_j) for every dipole from one adjoint solve through the same
FFT matvec (the interaction matrix is complex symmetric, so A^T nu = W P^*
is solved with A itself).  All of it runs in the CUDA library (dda_grad_qabs).

Dipoles with equal eps share one composition of the C ABI (at most 255
distinct values per call); each dipole's gradient is still its own.
Gradient convention (PyTorch, real loss of a complex input):
    eps.grad = dQ/dRe(eps) + i dQ/dIm(eps).
"""
from __future__ import annotations

import numpy as np
import torch

from . import Context, Precision


class DipoleTarget:
    """Geometry, size parameter and incident wave of the Q_abs objective.

    occupancy: bool/uint8 grid [nz, ny, nx]; x: size parameter 2 pi a_eff/lambda
    (a_eff from the number of dipoles); khat (3,), ehat (3,) complex.
    """

    def __init__(self, occupancy, x: float, khat, ehat, precision: int = Precision.FP64, device: int = 0,
                 tol: float = 1e-8, maxit: int = 2000):
        self.occ = np.asarray(occupancy).astype(bool)
        self.x = float(x)
        self.khat = np.asarray(khat, dtype=np.float64).reshape(1, 3)
        self.ehat = np.asarray(ehat, dtype=np.complex128).reshape(1, 3)
        self.precision = precision
        self.tol = tol
        self.maxit = maxit
        self.ctx = Context(device)
        self.N = int(self.occ.sum())

    def qabs_and_grad(self, eps: np.ndarray):
        eps = np.asarray(eps, dtype=np.complex128).ravel()
        if eps.size != self.N:
            raise ValueError(f"eps has {eps.size} entries, the target has {self.N} dipoles")
        vals, inv = np.unique(eps, return_inverse=True)
        if vals.size > 255:
            raise ValueError("at most 255 distinct dielectric functions per call")
        grid = np.zeros(self.occ.shape, dtype=np.uint8)
        grid[self.occ] = (inv + 1).astype(np.uint8)        # x-fastest scan order == site order
        self.ctx.set_target(grid)
        self.ctx.set_materials(np.sqrt(vals))
        prep = Precision.FP32_REFINED if self.precision != Precision.FP64 else Precision.FP64
        self.ctx.prepare_size_parameter(self.x, prep)
        g_re, g_im, P, (rf, ra) = self.ctx.grad_qabs(self.precision, self.khat, self.ehat, tol=self.tol,
                                                     maxit=self.maxit)
        return rf["qabs"], g_re + 1j * g_im

    def close(self):
        self.ctx.close()


class QabsFn(torch.autograd.Function):
    """Q_abs(eps) for a DipoleTarget; eps is a complex128 tensor of N entries."""

    @staticmethod
    def forward(ctx, eps: torch.Tensor, target: DipoleTarget):
        q, g = target.qabs_and_grad(eps.detach().cpu().numpy())
        ctx.save_for_backward(torch.from_numpy(g).to(eps.device))
        return torch.tensor(q, dtype=torch.float64, device=eps.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None
