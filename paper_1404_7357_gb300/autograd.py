"""torch.autograd.Function around the reduced-matrix fill.

``ReducedMatrix.apply(pos, eps_h, problem)`` returns the dense reduced matrix
Z'(positions, eps_r, h) of an array of identical elements (the fill of the
C-FFT table, Section III-B-3).  Its backward pass calls ``cfft_fill_backward``
(the hand-written adjoint of the interpolation fill) after re-tabulating the
table together with its substrate derivatives -- the table is recomputed,
not stored between forward and backward.  The contour (nodes, height, beta_p,
beta_max) is held fixed while eps_r and h vary, so the gradient is that of
the discretised C-FFT integral.
"""
import torch

from . import cfft


class FillProblem:
    """Everything of a fill except the differentiated inputs: element, contour,
    harmonics, rho grid, precision, rotations, and the CUDA context."""

    def __init__(self, element, k0, contour, q_max, rho_max, n_rho, precision="fp64",
                 rot=None, device=0):
        self.ctx = cfft.Context(device)
        self.element = element
        self.k0 = k0
        self.contour = contour
        self.q_max = q_max
        self.rho_max = rho_max
        self.n_rho = n_rho
        self.precision = cfft.CFFT_FP64 if precision == "fp64" else cfft.CFFT_FP32_MIXED
        self.rot = rot
        self.classes = 4 if rot is not None else 1
        self.device = device

    def tabulate(self, eps_r, h, derivatives):
        c, el = self.contour, self.element
        self.ctx.set_substrate(eps_r, h, self.k0)
        if el.kind == "strip":
            self.ctx.set_mbf_spectra_strip(el.length, el.strip_width)
        else:
            import numpy as np
            self.ctx.set_mbf_spectra(np.stack([el.cx, el.cy], 1), el.direction, el.half_len,
                                     el.width, el.q)
        self.ctx.build_contour(c.n, c.beta_max, c.beta_p, c.height, -1)
        self.ctx.set_option(cfft.OPT_DERIVATIVES, 1 if derivatives else 0)
        self.ctx.tabulate_reactions(self.q_max, self.rho_max, self.n_rho, self.precision,
                                    self.classes)

    @property
    def dtype(self):
        return torch.complex128 if self.precision == cfft.CFFT_FP64 else torch.complex64


class ReducedMatrix(torch.autograd.Function):
    @staticmethod
    def forward(fctx, pos, eps_h, problem):
        eps_r, h = (float(v) for v in eps_h.detach().cpu())
        problem.tabulate(eps_r, h, derivatives=False)
        a = pos.shape[0]
        m = problem.element.n_mbf
        z = torch.empty((a * m, a * m), dtype=problem.dtype, device=pos.device)
        problem.ctx.fill_reduced_matrix(pos.detach().contiguous(), problem.rot, z)
        fctx.save_for_backward(pos.detach(), eps_h.detach())
        fctx.problem = problem
        return z

    @staticmethod
    def backward(fctx, grad_z):
        pos, eps_h = fctx.saved_tensors
        problem = fctx.problem
        eps_r, h = (float(v) for v in eps_h.cpu())
        problem.tabulate(eps_r, h, derivatives=True)   # recomputed, with d/d eps_r, d/d h
        g = grad_z.contiguous()
        if g.dtype != problem.dtype:
            g = g.to(problem.dtype)
        grad_pos, grad_th = problem.ctx.fill_backward(pos.contiguous(), problem.rot, g)
        return grad_pos.to(pos.dtype), grad_th.to(eps_h.dtype).to(eps_h.device), None
