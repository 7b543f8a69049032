"""torch.autograd.Function over the Bragg-spot sum and its hand-written
adjoint (nb_adjoint): diffBragg-style gradients of any scalar image loss
with respect to three small crystal rotations, the cell lengths a, b, c,
Na, Nb, Nc, the scale and every structure factor.

The forward and the backward both run in libnbgb's kernels; torch holds
the tensors and applies the upstream gradient.  Parameters follow the
library's convention: lab axes = rows of Rx(tx) Ry(ty) Rz(tz) U diag(a,b,c).
"""
from __future__ import annotations

import numpy as np
import torch

from . import nbgb

PARAM_NAMES = ("tx", "ty", "tz", "a", "b", "c", "Na", "Nb", "Nc", "scale")


class BraggImage(torch.autograd.Function):
    """image = BraggImage.apply(params, F, sim, U)

    params: float64 tensor of 10 (PARAM_NAMES order); F: float32 tensor of
    the structure-factor table (uploaded when it changes; its gradient is
    float64 on the image's device); sim: an nbgb.Sim set up for a shot with
    NB_MIXED and a Gaussian shape (nearest or tricubic lookup); U: 3x3
    orientation.
    Returns the image as a float64 CUDA tensor of nb_num_pixels values.
    """

    @staticmethod
    def forward(ctx, params, F, sim, U):
        p = params.detach().to("cpu", torch.float64).numpy()
        if F is not None:
            sim.upload_F(F.detach().to("cpu", torch.float32).numpy())
        sim.set_params(U, p[3:6], p[0:3], p[6:9], p[9])
        sim.zero()
        sim.add_spots()
        dev = torch.device("cuda", sim.device)
        img = torch.empty(sim.npix, dtype=torch.float64, device=dev)
        torch.cuda.current_stream(dev).synchronize()
        sim.image_to_device(img.data_ptr(), sim.npix, nbgb.NB_DTYPE_F64)
        ctx.sim = sim
        ctx.F_shape = None if F is None else tuple(F.shape)
        ctx.F_device = None if F is None else F.device
        return img

    @staticmethod
    def backward(ctx, grad_img):
        sim = ctx.sim
        g = grad_img.detach().to(torch.float64).contiguous()
        gradF = None
        ptrF = 0
        if ctx.F_shape is not None and ctx.needs_input_grad[1]:
            gradF = torch.zeros(ctx.F_shape, dtype=torch.float64,
                                device=g.device)
            ptrF = gradF.data_ptr()
        torch.cuda.current_stream(g.device).synchronize()
        g10 = sim.adjoint(g.data_ptr(), ptrF)
        gp = torch.from_numpy(g10).to(torch.float64)
        if gradF is not None and ctx.F_device is not None:
            gradF = gradF.to(ctx.F_device)
        return gp, gradF, None, None


def bragg_image(params, F, sim, U):
    return BraggImage.apply(params, F, sim, U)
