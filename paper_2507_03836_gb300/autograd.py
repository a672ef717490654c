"""torch.autograd wrapper of the encoding: forward is fhash_encode, backward is fhash_encode_backward.

The embedding tables live in the library (up to billions of parameters), so they are not torch
tensors.  Their gradient accumulates in the model's own gradient buffer, the way a parameter's
.grad accumulates, and fhash_apply_adam consumes it.  A zero-size `anchor` tensor that requires
grad ties the encoding into torch's graph even when the coordinates do not require grad; its
gradient is always zero.  Coordinates get no gradient (the cell location is piecewise constant in
the integer rows and the method never differentiates through it).
"""
import torch

from . import fhash_encode, fhash_encode_backward, fhash_get_info


class _Encode(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coords, anchor, model, width):
        enc = torch.empty((coords.shape[0], width), dtype=torch.float32, device=coords.device)
        fhash_encode(model, coords, enc)
        ctx.model = model
        ctx.save_for_backward(coords)
        return enc

    @staticmethod
    def backward(ctx, d_enc):
        (coords,) = ctx.saved_tensors
        fhash_encode_backward(ctx.model, coords, d_enc.contiguous())
        return None, None, None, None


class Encoding(torch.nn.Module):
    """Multi-resolution Tesseract encoding of a library model as a torch module: [n][4] -> [n][L*F]."""

    def __init__(self, model):
        super().__init__()
        self.model = model
        info = fhash_get_info(model)
        self.width = info["n_levels"] * info["F"]
        self.anchor = torch.nn.Parameter(torch.zeros(0), requires_grad=True)

    def forward(self, coords):
        if coords.dtype != torch.float32 or not coords.is_cuda or coords.dim() != 2 or coords.shape[1] != 4:
            raise ValueError("coords must be a float32 CUDA tensor of shape [n, 4]")
        return _Encode.apply(coords.contiguous(), self.anchor, self.model, self.width)
