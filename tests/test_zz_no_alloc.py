"""The allocation-free critic-loss forward (crl_infonce_forward_noalloc).

It serves callers that cannot allocate device memory when they evaluate the
loss (a host that fixes its device memory at start-up, a plugin inside a
runtime that owns the device allocator).  Here it is called through the C ABI
and compared with crl_infonce_forward, which takes a caller-allocated
workspace, on two calls in a row.  Both run the same kernels on the same
inputs, so the results must be bit-identical: the shared fixed scratch must
not leak state from one call into the next.  This file is collected last
so that a run stopping at the first failure has already run everything else.
"""

import ctypes

import numpy as np
import pytest
import torch

from paper_2408_11052_gb300 import api, workload

pytestmark = pytest.mark.gpu


def forward_with_workspace(desc, phi, psi, dtype):
    L = api.lib()
    B, R = phi.shape
    nbytes = ctypes.c_size_t()
    api.check(L.crl_infonce_workspace_bytes(ctypes.byref(desc), B, R, ctypes.byref(nbytes)))
    ws = torch.empty(nbytes.value, dtype=torch.uint8, device=phi.device)
    out = [torch.empty(n, dtype=dtype, device=phi.device) for n in (4, B, B)]
    api.check(L.crl_infonce_forward(ctypes.byref(desc), phi.data_ptr(), psi.data_ptr(), B, R, out[0].data_ptr(),
                                    out[1].data_ptr(), out[2].data_ptr(), ws.data_ptr(), nbytes.value,
                                    api.stream_handle()))
    return out


def forward_noalloc(desc, phi, psi, dtype):
    L = api.lib()
    B, R = phi.shape
    out = [torch.empty(n, dtype=dtype, device=phi.device) for n in (4, B, B)]
    api.check(L.crl_infonce_forward_noalloc(ctypes.byref(desc), phi.data_ptr(), psi.data_ptr(), B, R,
                                            out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(),
                                            api.stream_handle()))
    return out


@pytest.mark.parametrize("energy", ["l2", "cos", "dot"])
def test_noalloc_forward_matches_workspace_forward_twice(energy):
    dev = torch.device("cuda")
    desc = api.CrlLossDesc(api.ENERGY[energy], api.LOSS["sym"], api.SYM["mean"], api.PENALTY["row"], 0.9, 0.1,
                           api.PREC["fp32"], api.PATH["plain"])
    for call, (B, R, seed) in enumerate(((256, 64, 1), (97, 33, 2))):   # two calls in a row, new sizes
        phi, psi = (torch.from_numpy(x).to(dev) for x in workload.representations(B, R, seed))
        ref = forward_with_workspace(desc, phi, psi, torch.float32)
        got = forward_noalloc(desc, phi, psi, torch.float32)
        torch.cuda.synchronize()
        for r, g in zip(ref, got):
            np.testing.assert_array_equal(g.cpu().numpy(), r.cpu().numpy(), err_msg=f"call {call}")


def test_noalloc_rejects_sizes_beyond_its_scratch():
    dev = torch.device("cuda")
    desc = api.CrlLossDesc(api.ENERGY["l2"], api.LOSS["sym"], api.SYM["mean"], api.PENALTY["row"], 1.0, 0.1,
                           api.PREC["fp32"], api.PATH["plain"])
    B, R = 2048, 64                                    # 16 MiB of scratch needed
    phi = torch.zeros(B, R, device=dev)
    outs = [torch.empty(n, device=dev) for n in (4, B, B)]
    rc = api.lib().crl_infonce_forward_noalloc(ctypes.byref(desc), phi.data_ptr(), phi.data_ptr(), B, R,
                                               outs[0].data_ptr(), outs[1].data_ptr(), outs[2].data_ptr(),
                                               api.stream_handle())
    assert rc == api.E_SHAPE
    assert b"4 MiB" in api.lib().crl_last_error(None)


def test_noalloc_validates_like_the_workspace_forward():
    """One descriptor check for both entry points: the forward-backward objective
    with B < 2 is a shape error on both, an unknown energy an argument error, and
    a path the allocation-free forward does not take is unsupported."""
    dev = torch.device("cuda")
    L = api.lib()
    phi = torch.zeros(1, 8, device=dev)
    outs = [torch.empty(n, device=dev) for n in (4, 1, 1)]
    ws = torch.empty(1 << 16, dtype=torch.uint8, device=dev)

    def both(desc):
        rc_ws = L.crl_infonce_forward(ctypes.byref(desc), phi.data_ptr(), phi.data_ptr(), 1, 8, outs[0].data_ptr(),
                                      outs[1].data_ptr(), outs[2].data_ptr(), ws.data_ptr(), ws.numel(),
                                      api.stream_handle())
        rc_na = L.crl_infonce_forward_noalloc(ctypes.byref(desc), phi.data_ptr(), phi.data_ptr(), 1, 8,
                                              outs[0].data_ptr(), outs[1].data_ptr(), outs[2].data_ptr(),
                                              api.stream_handle())
        return rc_ws, rc_na

    fb = api.CrlLossDesc(api.ENERGY["l2"], api.LOSS["fb"], api.SYM["mean"], api.PENALTY["row"], 1.0, 0.1,
                         api.PREC["fp32"], api.PATH["plain"])
    assert both(fb) == (api.E_SHAPE, api.E_SHAPE)
    bad = api.CrlLossDesc(99, api.LOSS["sym"], api.SYM["mean"], api.PENALTY["row"], 1.0, 0.1,
                          api.PREC["fp32"], api.PATH["plain"])
    assert both(bad) == (api.E_INVALID_ARG, api.E_INVALID_ARG)
    fused = api.CrlLossDesc(api.ENERGY["l2"], api.LOSS["sym"], api.SYM["mean"], api.PENALTY["row"], 1.0, 0.1,
                            api.PREC["fp32"], api.PATH["fused"])
    assert both(fused)[1] == api.E_UNSUPPORTED
