"""torch.autograd.Function wrappers around the op-level C ABI.

``EncoderMLP`` and ``InfoNCELoss`` run their forward and their hand-written
backward in the library's CUDA kernels (``crl_mlp_forward/backward`` and
``crl_infonce_forward/backward``); torch only allocates and records the graph.

Precision: FP32 / FP64 parameters take the plain SIMT kernels in that dtype.
``precision="bf16"`` (FP32 parameters) takes the tensor-core path: BF16 GEMMs
with FP32 accumulation for the encoder, and with ``path="fused"`` the fused
energy + InfoNCE + penalty kernels (BF16 operands, FP32 logsumexps and loss;
the B x B logits are never written).  Every workspace the backward needs is
saved with the graph, so several forwards may precede their backwards.
"""

from ctypes import byref, c_size_t

import torch

from . import api


def _dtype_code(t, precision=None):
    if precision == "bf16":
        if t.dtype != torch.float32:
            raise TypeError("the BF16 path takes float32 parameters and representations")
        return api.PREC["bf16"]
    if t.dtype == torch.float64:
        return api.PREC["fp64"]
    if t.dtype == torch.float32:
        return api.PREC["fp32"]
    raise TypeError("parameters must be float32 or float64")


class EncoderMLP(torch.autograd.Function):
    """y = MLP(concat(x0, x1)) with params in the flat layout of include/crl.h.

    x0 / x1 are float32 inputs (x1 may be None); params and y share one dtype.
    Gradients flow to params, x0 and x1.  precision "bf16": float32 params on the
    tensor-core path.
    """

    @staticmethod
    def forward(ctx, params, x0, x1, in0, in1, hidden, layers, out, layernorm, precision=None):
        L = api.lib()
        desc = api.CrlMlpDesc(in0, in1, hidden, layers, out, int(layernorm), _dtype_code(params, precision))
        M = x0.shape[0]
        nbytes = c_size_t()
        api.check(L.crl_mlp_saved_bytes(byref(desc), M, byref(nbytes)))
        saved = torch.empty(nbytes.value, dtype=torch.uint8, device=params.device)
        y = torch.empty(M, out, dtype=params.dtype, device=params.device)
        x0c = x0.detach().contiguous().float()
        x1c = None if x1 is None else x1.detach().contiguous().float()
        api.check(L.crl_mlp_forward(byref(desc), params.data_ptr(), x0c.data_ptr(),
                                    None if x1c is None else x1c.data_ptr(), M, y.data_ptr(), saved.data_ptr(),
                                    api.stream_handle()))
        ctx.desc = (in0, in1, hidden, layers, out, int(layernorm))
        ctx.precision = precision
        ctx.has_x1 = x1 is not None
        ctx.save_for_backward(params, x0c, x1c if x1c is not None else x0c, saved)
        return y

    @staticmethod
    def backward(ctx, dy):
        L = api.lib()
        params, x0c, x1c, saved = ctx.saved_tensors
        if not ctx.has_x1:
            x1c = None
        desc = api.CrlMlpDesc(*ctx.desc, _dtype_code(params, ctx.precision))
        M = x0c.shape[0]
        dparams = torch.zeros_like(params) if ctx.needs_input_grad[0] else None
        dx0 = torch.empty(M, ctx.desc[0], dtype=params.dtype, device=params.device) if ctx.needs_input_grad[1] else None
        dx1 = (torch.empty(M, ctx.desc[1], dtype=params.dtype, device=params.device)
               if (x1c is not None and ctx.needs_input_grad[2]) else None)
        dyc = dy.contiguous().to(params.dtype)
        api.check(L.crl_mlp_backward(byref(desc), params.data_ptr(), x0c.data_ptr(),
                                     None if x1c is None else x1c.data_ptr(), M, saved.data_ptr(), dyc.data_ptr(),
                                     api.ptr(dparams), api.ptr(dx0), api.ptr(dx1), api.stream_handle()))
        return dparams, dx0, dx1, None, None, None, None, None, None, None


class InfoNCELoss(torch.autograd.Function):
    """Critic loss (energy + InfoNCE + logsumexp penalty); returns (total, parts[4]).

    parts = {total, InfoNCE-fwd, InfoNCE-bwd, penalty} (not differentiable).
    The backward takes the incoming gradient of ``total`` as a host scalar.
    path "fused": float32 representations on the BF16 fused kernels (B a
    multiple of 8, repr 64 / 128 / 192 / 256; the L1 energy runs on FP32 SIMT
    tiles, the others on the tensor cores).
    """

    @staticmethod
    def forward(ctx, phi, psi, energy, loss, sym_reduction, penalty_axis, temperature, beta, path):
        L = api.lib()
        dtype = _dtype_code(phi, "bf16" if path == "fused" else None)
        desc = api.CrlLossDesc(api.ENERGY[energy], api.LOSS[loss], api.SYM[sym_reduction],
                               api.PENALTY[penalty_axis], temperature, beta, dtype, api.PATH[path])
        B, R = phi.shape
        nbytes = c_size_t()
        api.check(L.crl_infonce_workspace_bytes(byref(desc), B, R, byref(nbytes)))
        ws = torch.empty(nbytes.value, dtype=torch.uint8, device=phi.device)
        phi_c, psi_c = phi.detach().contiguous(), psi.detach().contiguous()
        parts = torch.empty(4, dtype=phi.dtype, device=phi.device)
        r = torch.empty(B, dtype=phi.dtype, device=phi.device)
        c = torch.empty(B, dtype=phi.dtype, device=phi.device)
        api.check(L.crl_infonce_forward(byref(desc), phi_c.data_ptr(), psi_c.data_ptr(), B, R, parts.data_ptr(),
                                        r.data_ptr(), c.data_ptr(), ws.data_ptr(), nbytes.value, api.stream_handle()))
        ctx.desc = desc
        ctx.ws_bytes = nbytes.value
        ctx.save_for_backward(phi_c, psi_c, r, c, ws)
        ctx.mark_non_differentiable(parts)
        return parts[0].clone(), parts

    @staticmethod
    def backward(ctx, dtotal, _dparts):
        L = api.lib()
        phi, psi, r, c, ws = ctx.saved_tensors
        B, R = phi.shape
        dphi = torch.empty_like(phi)
        dpsi = torch.empty_like(psi)
        api.check(L.crl_infonce_backward(byref(ctx.desc), phi.data_ptr(), psi.data_ptr(), B, R, r.data_ptr(),
                                         c.data_ptr(), float(dtotal.item()), dphi.data_ptr(), dpsi.data_ptr(),
                                         ws.data_ptr(), ctx.ws_bytes, api.stream_handle()))
        return dphi, dpsi, None, None, None, None, None, None, None


def encoder(params, x0, x1, in0, in1, hidden, layers, out, layernorm=False, precision=None):
    """precision None: the dtype of params (FP32 / FP64 plain kernels); "bf16": tensor cores."""
    return EncoderMLP.apply(params, x0, x1, in0, in1, hidden, layers, out, layernorm, precision)


def infonce_loss(phi, psi, energy="l2", loss="sym", sym_reduction="mean", penalty_axis="row", temperature=1.0,
                 beta=0.1, path="plain"):
    return InfoNCELoss.apply(phi, psi, energy, loss, sym_reduction, penalty_axis, temperature, beta, path)
