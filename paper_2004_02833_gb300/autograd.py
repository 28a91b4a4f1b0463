"""torch.autograd.Function over the library's detector functional and its discrete adjoint.

    J = detector_response(context, sigma_a, sigma_s, q, u_init, w, k, ckpt_every=20)
    J.backward()   # or torch.autograd.grad(J, (sigma_a, sigma_s, q))

Forward: the media (per-cell sigma_a, sigma_s, q, [z][y][x]) and the initial state u_init (interface
order [c][z][y][x]) go to the context, k steps of Eq. (6) run in the library's kernels, and the
library's rtpn_detector returns J = sum w u_0 as a 0-dim float64 CUDA tensor (no host wait).
Backward: the same media and u_init go back to the context and rtpn_adjoint runs the discrete
adjoint (checkpoints every ckpt_every steps) into float64 CUDA tensors dJ/dsigma_a, dJ/dsigma_s,
dJ/dq; autograd's chain rule multiplies them by the incoming gradient of J.  Both directions run on
PyTorch's current stream.  Every value of the method comes from the library: this module only
moves tensors in and out (the one multiplication is autograd's scaling by grad_output).  After
forward the context holds u(k); after backward it holds u(k) again (rtpn_adjoint leaves it there).
"""
from __future__ import annotations

import torch

from . import rtpn


class DetectorResponse(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sigma_a, sigma_s, q, context, u_init, w, k, ckpt_every):
        for t in (sigma_a, sigma_s, q, u_init, w):
            if not (isinstance(t, torch.Tensor) and t.is_cuda):
                raise TypeError("media, initial state and weights must be CUDA tensors")
        stream = torch.cuda.current_stream(sigma_a.device)
        context.set_stream(stream)
        context.set_media(sigma_a.detach().contiguous(), sigma_s.detach().contiguous(), q.detach().contiguous())
        context.set_moments(u_init.detach().contiguous())
        context.step(int(k))
        J = torch.empty(1, dtype=torch.float64, device=sigma_a.device)
        context.detector(w.detach().contiguous(), out=J)
        ctx.context = context
        ctx.k = int(k)
        ctx.ckpt_every = int(ckpt_every)
        ctx.save_for_backward(sigma_a, sigma_s, q, u_init, w)
        return J.reshape(())

    @staticmethod
    def backward(ctx, grad_J):
        sigma_a, sigma_s, q, u_init, w = ctx.saved_tensors
        c = ctx.context
        c.set_stream(torch.cuda.current_stream(sigma_a.device))
        c.set_media(sigma_a.detach().contiguous(), sigma_s.detach().contiguous(), q.detach().contiguous())
        c.set_moments(u_init.detach().contiguous())
        grads = tuple(torch.empty(sigma_a.shape, dtype=torch.float64, device=sigma_a.device) for _ in range(3))
        c.adjoint(w.detach().contiguous(), ctx.k, ckpt_every=ctx.ckpt_every, out=grads)
        out = []
        for g, x, need in zip(grads, (sigma_a, sigma_s, q), ctx.needs_input_grad[:3]):
            out.append((g * grad_J).to(x.dtype) if need else None)
        return out[0], out[1], out[2], None, None, None, None, None


def detector_response(context: rtpn.Context, sigma_a: torch.Tensor, sigma_s: torch.Tensor, q: torch.Tensor,
                      u_init: torch.Tensor, w: torch.Tensor, k: int, ckpt_every: int = 20) -> torch.Tensor:
    """J = sum w u_0 after k steps from u_init with media (sigma_a, sigma_s, q); differentiable in the
    three media tensors (gradients by the library's discrete adjoint)."""
    return DetectorResponse.apply(sigma_a, sigma_s, q, context, u_init, w, k, ckpt_every)
