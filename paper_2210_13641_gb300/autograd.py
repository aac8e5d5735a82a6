"""torch.autograd integration of the mapping loss.

`MappingLoss.apply(params, m, n_rays, seed)` returns the mapping loss L_M of one
batch as a 0-d CUDA tensor whose gradient with respect to the flat FP32 parameter
tensor `params` (layout of include/nerfmap.h) is the library's own fused backward:
the forward call runs one map_step without the Adam update (the loss and, in the
same fused pass, the gradient, with per-sample activations recomputed rather than
stored) and keeps the gradient; backward() scales it by the incoming gradient.
Argument marshalling only - every computation runs in the CUDA kernels.
"""

from __future__ import annotations

import torch


class MappingLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params: torch.Tensor, m, n_rays: int, seed: int):
        if not (params.is_cuda and params.dtype == torch.float32 and params.is_contiguous()):
            raise ValueError("params must be a contiguous float32 CUDA tensor")
        stream = torch.cuda.current_stream()
        m.set_params(params.detach(), stream=stream)
        loss = m.step(n_rays, seed, no_update=True, want_loss=True, stream=stream)
        grads = torch.empty_like(params)
        m.get_grads(out=grads, stream=stream)
        ctx.save_for_backward(grads)
        return torch.tensor(loss, dtype=torch.float32, device=params.device)

    @staticmethod
    def backward(ctx, grad_out):
        (grads,) = ctx.saved_tensors
        return grad_out * grads, None, None, None


def mapping_loss(params: torch.Tensor, m, n_rays: int, seed: int) -> torch.Tensor:
    return MappingLoss.apply(params, m, n_rays, seed)
