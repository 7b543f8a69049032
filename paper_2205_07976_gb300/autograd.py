"""torch.autograd.Function over the Bragg-spot sum and its hand-written
adjoint (nb_adjoint): diffBragg-style gradients of any scalar image loss
with respect to three small crystal rotations, the cell lengths a, b, c,
Na, Nb, Nc, the scale and every structure factor.

The forward and the backward both run in libnbgb's kernels; torch holds
the tensors and applies the upstream gradient.  Parameters follow the
library's convention: lab axes = rows of Rx(tx) Ry(ty) Rz(tz) U diag(a,b,c).

The adjoint recomputes the forward sum, so backward needs the handle in the
state of its own forward.  Each call therefore keeps its parameters, and
backward sets them (and the structure factors, if another call replaced
them) on the handle again before it runs: several forwards may share one
handle before their backwards run.
"""
from __future__ import annotations

import weakref

import numpy as np
import torch

from . import nbgb

PARAM_NAMES = ("tx", "ty", "tz", "a", "b", "c", "Na", "Nb", "Nc", "scale")


def _ensure_F(sim, F):
    """Make the handle's resident table hold F's values.  Skipped when the
    handle already holds this tensor at its current version (in-place
    changes bump the version).  A CUDA tensor on the handle's device is
    copied device to device on the handle's stream; any other tensor goes
    through the host."""
    ref = getattr(sim, "_F_ref", None)
    held = ref() if ref is not None else None
    # the tensor last uploaded, still alive (so its memory is its own), or
    # a tensor on the same memory (as backward's saved copy of it), with no
    # in-place change since
    if held is not None and (held is F or (
            held.data_ptr() == F.data_ptr() and held.dtype == F.dtype
            and held.shape == F.shape and held.device == F.device)) and (
            held._version == sim._F_version == F._version):
        return
    Fd = F.detach()
    if Fd.is_cuda and Fd.device.index == sim.device:
        Fc = Fd.to(torch.float32).contiguous()
        # F is produced on torch's current stream; the handle's stream reads
        # it next
        torch.cuda.current_stream(Fc.device).synchronize()
        sim.set_fcell_device(Fc.data_ptr(), Fc.numel())
        # the copy is queued: keep the source alive until it has run
        sim.synchronize()
    else:
        sim.upload_F(Fd.to("cpu", torch.float32).numpy())
    sim._F_ref = weakref.ref(F)
    sim._F_version = F._version
    sim.F_uploads = getattr(sim, "F_uploads", 0) + 1


def _set_params(sim, U, p):
    sim.set_params(U, p[3:6], p[0:3], p[6:9], p[9])


class BraggImage(torch.autograd.Function):
    """image = BraggImage.apply(params, F, sim, U)

    params: tensor of 10 values (PARAM_NAMES order) on any device; its
    gradient comes back on the same device and dtype.  F: float32 tensor of
    the structure-factor table, or None to keep the handle's table (a CUDA
    tensor on the handle's device is uploaded device to device, and only
    when it is a different tensor or was changed in place since the last
    upload; its gradient is float64 on F's device).  sim: an nbgb.Sim set
    up for a shot with NB_MIXED and a Gaussian shape (nearest or tricubic
    lookup).  U: 3x3 orientation.
    Returns the image as a float64 CUDA tensor of nb_num_pixels values.
    """

    @staticmethod
    def forward(ctx, params, F, sim, U):
        p = params.detach().to("cpu", torch.float64).numpy().copy()
        Uh = np.array(U, dtype=np.float64).reshape(3, 3).copy()
        if F is not None:
            _ensure_F(sim, F)
        _set_params(sim, Uh, p)
        sim.zero()
        sim.add_spots()
        dev = torch.device("cuda", sim.device)
        img = torch.empty(sim.npix, dtype=torch.float64, device=dev)
        torch.cuda.current_stream(dev).synchronize()
        sim.image_to_device(img.data_ptr(), sim.npix, nbgb.NB_DTYPE_F64)
        ctx.sim = sim
        ctx.p = p
        ctx.U = Uh
        ctx.p_device, ctx.p_dtype = params.device, params.dtype
        ctx.has_F = F is not None
        # saved so that an in-place change of F before backward is caught
        ctx.save_for_backward(F)
        return img

    @staticmethod
    def backward(ctx, grad_img):
        sim = ctx.sim
        (F,) = ctx.saved_tensors
        if ctx.has_F:
            _ensure_F(sim, F)
        _set_params(sim, ctx.U, ctx.p)
        g = grad_img.detach().to(torch.float64).contiguous()
        gradF = None
        ptrF = 0
        if ctx.has_F and ctx.needs_input_grad[1]:
            gradF = torch.zeros(tuple(F.shape), dtype=torch.float64,
                                device=g.device)
            ptrF = gradF.data_ptr()
        torch.cuda.current_stream(g.device).synchronize()
        g10 = sim.adjoint(g.data_ptr(), ptrF)
        gp = torch.from_numpy(g10).to(device=ctx.p_device, dtype=ctx.p_dtype)
        if gradF is not None:
            gradF = gradF.to(F.device)
        return gp, gradF, None, None


def bragg_image(params, F, sim, U):
    return BraggImage.apply(params, F, sim, U)
