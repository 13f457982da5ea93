"""torch.autograd.Function wrappers over the C ABI: every forward and backward is a library call.

Gradient convention: PyTorch's gradient of a real loss with respect to a complex tensor is
dL/dRe + i dL/dIm, the convention of the library's *_backward entry points, so the adjoints pass
through unchanged. Distances and element parameters are float64 CUDA tensors (read by the kernels
at run time, so the same code serves a captured CUDA graph); phase masks are float32 (complex64
fields) or float64 (complex128 fields).
"""
from __future__ import annotations

import torch

from . import xl


def _dev_z(z: torch.Tensor, batch: int) -> torch.Tensor:
    z = z.reshape(-1)
    if z.numel() == 1 and batch > 1:
        z = z.expand(batch)
    return z.contiguous()


class RSPropagate(torch.autograd.Function):
    """u [B][ny][nx] -> RS(u, z); z: float64 CUDA tensor [B] (or [1]). phase_invariant: the loss
    ignores a constant phase on the output (intensity losses behind linear optics), which lets
    the distance derivative drop an exactly-zero, noise-prone term (XL_PHASE_INVARIANT).
    checkpoint: for the distance gradient keep the input field (one plane) instead of the 2D
    spectrum of the zero-padded input (four planes), which the adjoint then recomputes."""

    @staticmethod
    def forward(ctx, u, z, grid, wavelength, phase_invariant=False, checkpoint=False):
        zz = _dev_z(z.detach(), u.shape[0])
        u = u.contiguous()
        need_z = ctx.needs_input_grad[1]
        # a distance gradient needs the input's spectrum: kept by the forward, or recomputed
        saved = xl.save_buffer(u) if need_z and not checkpoint else u.new_empty(0)
        ctx.save_for_backward(saved, zz, u if need_z and checkpoint else u.new_empty(0))
        ctx.grid, ctx.wl, ctx.zshape, ctx.pinv = grid, wavelength, z.shape, phase_invariant
        return xl.rs_propagate(u, grid, wavelength, zz, saved=saved if saved.numel() else None)

    @staticmethod
    def backward(ctx, g):
        saved, zz, u = ctx.saved_tensors
        need_u, need_z = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        g_in, g_z = xl.rs_propagate_backward(g.contiguous(), u if u.numel() else None, ctx.grid,
                                             ctx.wl, zz, want_field=need_u, want_dz=need_z,
                                             phase_invariant=ctx.pinv,
                                             saved=saved if need_z and saved.numel() else None)
        if g_z is not None:
            g_z = g_z.reshape(-1).sum().reshape(ctx.zshape) if ctx.zshape.numel() == 1 else g_z.reshape(ctx.zshape)
        return g_in, g_z, None, None, None, None


class VRSPropagate(torch.autograd.Function):
    """exy [B][2][ny][nx] -> [B][3][ny][nx] (phase_invariant and checkpoint as in RSPropagate:
    two input planes kept instead of eight spectrum planes)."""

    @staticmethod
    def forward(ctx, exy, z, grid, wavelength, phase_invariant=False, checkpoint=False):
        zz = _dev_z(z.detach(), exy.shape[0])
        exy = exy.contiguous()
        need_z = ctx.needs_input_grad[1]
        saved = xl.save_buffer(exy, 2) if need_z and not checkpoint else exy.new_empty(0)
        ctx.save_for_backward(saved, zz, exy if need_z and checkpoint else exy.new_empty(0))
        ctx.grid, ctx.wl, ctx.zshape, ctx.pinv = grid, wavelength, z.shape, phase_invariant
        return xl.vrs_propagate(exy, grid, wavelength, zz, saved=saved if saved.numel() else None)

    @staticmethod
    def backward(ctx, g):
        saved, zz, exy = ctx.saved_tensors
        need_u, need_z = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        g_in, g_z = xl.vrs_propagate_backward(g.contiguous(), exy if exy.numel() else None, ctx.grid,
                                              ctx.wl, zz, want_field=need_u, want_dz=need_z,
                                              phase_invariant=ctx.pinv,
                                              saved=saved if need_z and saved.numel() else None)
        if g_z is not None:
            g_z = g_z.reshape(-1).sum().reshape(ctx.zshape) if ctx.zshape.numel() == 1 else g_z.reshape(ctx.zshape)
        return g_in, g_z, None, None, None, None


class CZTPropagate(torch.autograd.Function):
    """CZT onto a window (scalar [B][ny][nx] or vectorial [B][2][ny][nx]); z: float64 CUDA
    tensor [B] (or [1]). When z requires a gradient the forward saves the sums the distance
    gradient needs (xl_czt_propagate_save) and keeps its input. phase_invariant as in
    RSPropagate."""

    @staticmethod
    def forward(ctx, u, z, grid, window, wavelength, vectorial, phase_invariant=False):
        zz = _dev_z(z.detach(), u.shape[0])
        u = u.contiguous()
        need_z = ctx.needs_input_grad[1]
        saved = xl.czt_save_buffer(u, grid, window, vectorial) if need_z else u.new_empty(0)
        ctx.save_for_backward(zz, saved, u if need_z else u.new_empty(0))
        ctx.grid, ctx.window, ctx.wl, ctx.vec = grid, window, wavelength, vectorial
        ctx.zshape, ctx.pinv = z.shape, phase_invariant
        return xl.czt_propagate(u, grid, window, wavelength, zz, vectorial=vectorial,
                                saved=saved if need_z else None)

    @staticmethod
    def backward(ctx, g):
        zz, saved, u = ctx.saved_tensors
        need_u, need_z = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not need_z:
            g_in = xl.czt_propagate_backward(g.contiguous(), ctx.grid, ctx.window, ctx.wl, zz,
                                             vectorial=ctx.vec)
            return g_in, None, None, None, None, None, None
        g_in, g_z = xl.czt_propagate_backward(g.contiguous(), ctx.grid, ctx.window, ctx.wl, zz,
                                              vectorial=ctx.vec, u_in=u, want_dz=True,
                                              want_field=need_u, phase_invariant=ctx.pinv,
                                              saved=saved)
        g_z = g_z.reshape(-1).sum().reshape(ctx.zshape) if ctx.zshape.numel() == 1 else g_z.reshape(ctx.zshape)
        return g_in, g_z, None, None, None, None, None


class BeamSplitter(torch.autograd.Function):
    """(a, b, R) -> (out_t, out_r): lossless beam splitter of reflectance R (float64 CUDA [B]);
    a and b are fields of the same shape [B][...]."""

    @staticmethod
    def forward(ctx, a, b, R):
        a, b, Rc = a.contiguous(), b.contiguous(), R.detach().contiguous()
        ctx.save_for_backward(a, b, Rc)
        return xl.beam_splitter(a, b, Rc)

    @staticmethod
    def backward(ctx, g_t, g_r):
        a, b, R = ctx.saved_tensors
        need_a, need_b, need_R = ctx.needs_input_grad
        g_a, g_b, g_R = xl.beam_splitter_backward(g_t.contiguous(), g_r.contiguous(), a, b, R,
                                                  want_a=need_a, want_b=need_b, want_R=need_R)
        return g_a, g_b, g_R


class Elements(torch.autograd.Function):
    """Element chain. kinds: list of element kinds; masks: list (per element) of (phi_x, phi_y)
    tensors or None; params: float64 CUDA [B][n][4] {f, alpha, eta, theta} (differentiable)."""

    @staticmethod
    def forward(ctx, field, params, grid, wavelength, kinds, comps_in, *masks):
        mk = [m if m.numel() else None for m in masks]
        els = [dict(kind=k, phi_x=mk[2 * i], phi_y=mk[2 * i + 1]) for i, k in enumerate(kinds)]
        ctx.save_for_backward(field, params, *[m for m in masks])
        ctx.grid, ctx.wl, ctx.kinds, ctx.comps_in, ctx.els_n = grid, wavelength, kinds, comps_in, len(kinds)
        return xl.apply_elements(field.contiguous(), grid, wavelength, els, comps_in=comps_in,
                                 params=params.detach().contiguous())

    @staticmethod
    def backward(ctx, g):
        field, params, *masks = ctx.saved_tensors
        masks = [m if m.numel() else None for m in masks]
        els = [dict(kind=k, phi_x=masks[2 * i], phi_y=masks[2 * i + 1]) for i, k in enumerate(ctx.kinds)]
        g_in, gpx, gpy, gp = xl.apply_elements_backward(
            g.contiguous(), field, ctx.grid, ctx.wl, els, comps_in=ctx.comps_in,
            params=params.detach().contiguous(), want_field=ctx.needs_input_grad[0],
            want_phi=any(ctx.needs_input_grad[6:]), want_params=ctx.needs_input_grad[1])
        gmasks = []
        for i in range(len(ctx.kinds)):
            gmasks += [gpx[i], gpy[i]]
        return (g_in, gp, None, None, None, None, *gmasks)


def elements(field, grid, wavelength, kinds, masks, params, comps_in):
    """Applies an element chain; masks[i] = (phi_x or None, phi_y or None)."""
    flat = []
    for mx, my in masks:
        for m in (mx, my):
            flat.append(m if m is not None else torch.empty(0, device=field.device))
    return Elements.apply(field, params, grid, wavelength, list(kinds), comps_in, *flat)


class IntensityLoss(torch.autograd.Function):
    """field [B][C][ny][nx] -> loss [B] (float64)."""

    @staticmethod
    def forward(ctx, field, grid, comp_mask, mode, eps):
        ctx.save_for_backward(field)
        ctx.grid, ctx.mask, ctx.mode, ctx.eps = grid, comp_mask, mode, eps
        loss, _ = xl.intensity_loss(field.contiguous(), grid, comp_mask, mode, eps)
        return loss

    @staticmethod
    def backward(ctx, g_loss):
        (field,) = ctx.saved_tensors
        g = xl.intensity_loss_backward(field, ctx.grid, ctx.mask, ctx.mode, ctx.eps,
                                       g_loss=g_loss.contiguous())
        return g, None, None, None, None
