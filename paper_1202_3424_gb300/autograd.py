"""torch.autograd.Function for the absorption efficiency Q_abs.

The forward pass is a DDA solve on the GPU for one incident plane wave,
with the dielectric function given per dipole (every dipole its own value:
the C ABI's per-site materials, no limit on distinct values).  The backward
pass returns dQ_abs/d(eps_j) for every dipole from one adjoint solve through
the same FFT matvec (the interaction matrix is complex symmetric, so
A^T nu = W P^* is solved with A itself); it runs only when a gradient is
asked for, and its forward solve starts from the saved polarization, so it
takes no iterations.  All of it runs in the CUDA library (dda_solve,
dda_grad_qabs).

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
    (a_eff from the number of dipoles); khat (3,), ehat (3,) complex.  The
    dipoles are the occupied sites in x-fastest scan order.
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
        self.ctx.set_target(self.occ.astype(np.uint8))
        self.N = int(self.occ.sum())
        self._eps = None

    def _set_eps(self, eps: np.ndarray):
        eps = np.asarray(eps, dtype=np.complex128).ravel()
        if eps.size != self.N:
            raise ValueError(f"eps has {eps.size} entries, the target has {self.N} dipoles")
        if self._eps is not None and np.array_equal(eps, self._eps):
            return
        # the library squares the index again, so either square root will do
        self.ctx.set_site_materials(np.sqrt(eps))
        prep = Precision.FP32_REFINED if self.precision != Precision.FP64 else Precision.FP64
        self.ctx.prepare_size_parameter(self.x, prep)
        self._eps = eps.copy()

    def qabs(self, eps: np.ndarray):
        """(Q_abs, P [3, N]) from one forward solve."""
        self._set_eps(eps)
        res, P, st = self.ctx.solve(self.precision, self.khat, self.ehat, tol=self.tol, maxit=self.maxit)
        if st != 0:
            raise RuntimeError(f"forward solve failed: {res[0]['status_name']}")
        return res[0]["qabs"], P[0]

    def grad(self, eps: np.ndarray, P=None):
        """dQ_abs/dRe(eps) + i dQ_abs/dIm(eps) per dipole; P (from qabs) warm-starts the forward solve."""
        self._set_eps(eps)
        opts = {} if P is None else {"x0": np.asarray(P, dtype=np.complex128).reshape(1, 3, self.N)}
        g_re, g_im, _, (rf, ra) = self.ctx.grad_qabs(self.precision, self.khat, self.ehat, tol=self.tol,
                                                     maxit=self.maxit, **opts)
        return g_re + 1j * g_im

    def qabs_and_grad(self, eps: np.ndarray):
        q, P = self.qabs(eps)
        return q, self.grad(eps, P)

    def close(self):
        self.ctx.close()


class QabsFn(torch.autograd.Function):
    """Q_abs(eps) for a DipoleTarget; eps is a complex128 tensor of N entries."""

    @staticmethod
    def forward(ctx, eps: torch.Tensor, target: DipoleTarget):
        e = eps.detach().cpu().numpy()
        q, P = target.qabs(e)
        ctx.target = target
        if ctx.needs_input_grad[0]:
            ctx.eps, ctx.P = e, P
        return torch.tensor(q, dtype=torch.float64, device=eps.device)

    @staticmethod
    def backward(ctx, grad_out):
        g = ctx.target.grad(ctx.eps, ctx.P)
        return grad_out * torch.from_numpy(g).to(grad_out.device), None
