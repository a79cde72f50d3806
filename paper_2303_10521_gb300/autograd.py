"""The field stage as a differentiable function (``torch.autograd.Function``).

``EMFieldFn.apply(eps_r, sigma, tx_pos, scene, paths, freq)`` returns the
coherent channel sums h[tx, rx] = (Re, Im) of a frozen path set (the face-ID
sequences in ``paths``) at frequency ``freq``, as a function of the complex
permittivity parameters of every material (eps_r, sigma) and of the
transmitter positions; the reflection points, Fresnel coefficients, spreading
and phase follow the parameters (emrt_channel).  Its backward is the
hand-written adjoint kernel (emrt_channel_backward): reflection points are
recomputed, not stored, and the path topology stays fixed.

The scene keeps float32 transmitter positions (as every frame does); a
``tx_pos`` that differs from the scene's moves its transmitters first
(``Scene.set_transmitters``), so finite differences in tx_pos are taken at
float32 resolution.
"""
import torch

from .engine import Paths, Scene


class EMFieldFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps_r: torch.Tensor, sigma: torch.Tensor, tx_pos: torch.Tensor,
                scene: Scene, paths: Paths, freq: float) -> torch.Tensor:
        e = eps_r.detach().to(device=scene.device, dtype=torch.float64).contiguous()
        s = sigma.detach().to(device=scene.device, dtype=torch.float64).contiguous()
        scene.set_transmitters(tx_pos.detach())
        ch = scene.channel(paths, float(freq), eps_r=e, sigma=s)
        ctx.scene, ctx.paths, ctx.freq = scene, paths, float(freq)
        ctx.save_for_backward(e, s)
        return ch.pair[..., :2].clone()

    @staticmethod
    def backward(ctx, grad_h: torch.Tensor):
        e, s = ctx.saved_tensors
        ge, gs, gt = ctx.scene.channel_backward(ctx.paths, ctx.freq, grad_h.contiguous(),
                                                eps_r=e, sigma=s)
        return ge, gs, gt, None, None, None


def field(eps_r, sigma, tx_pos, scene: Scene, paths: Paths, freq: float) -> torch.Tensor:
    """h[tx, rx, 2] of the frozen path set, differentiable in eps_r, sigma and
    tx_pos (see EMFieldFn)."""
    return EMFieldFn.apply(eps_r, sigma, tx_pos, scene, paths, freq)
