"""Checkpoint / resume of the library-owned state (crl_save_state / crl_load_state):
a context rebuilt from a saved blob plus the caller's parameters and Adam moments
continues bit-identically to the one that saved it -- relabel draws, Adam step
counts, the tuned entropy coefficient and the collection stub's environments
included -- and the blob checks reject foreign, corrupt and truncated input."""

import struct

import numpy as np
import pytest
import torch

from paper_2408_11052_gb300 import api, workload

from parity_helpers import setup, small

pytestmark = pytest.mark.gpu

NETS = ("phi", "psi", "pi")


def run_steps(ctx, inserts, collect):
    loss = torch.zeros(6, dtype=torch.float32, device=ctx.device)
    hist = []
    for ins in inserts:
        if collect:
            ctx.collect(2, 5)
        ctx.update_step(*(torch.from_numpy(x).to(ctx.device) for x in ins), loss_out=loss)
        hist.append(loss.cpu().numpy().copy())
    torch.cuda.synchronize()
    return np.array(hist)


def snapshot(ctx):
    return {n: {k: ctx.store[n][k].clone() for k in ("params", "grads", "adam_m", "adam_v")} for n in NETS}


@pytest.mark.parametrize("precision,path", [("fp64", "plain"), ("fp32", "plain"), ("bf16", "plain"),
                                            ("bf16", "fused")])
@pytest.mark.parametrize("collect", [False, True])
def test_resume_is_bit_identical(precision, path, collect):
    w = small(B=64, repr=64, alpha_autotune=True, target_entropy=-3.0, lr_alpha=0.05)
    a, _, _ = setup(w, precision=precision, path=path, n=30)
    extra = workload.buffer_contents(w, n=6, mean_len=9.0, seed_offset=5)
    inserts = [tuple(x[i:i + 1] for x in extra) for i in range(6)]
    run_steps(a, inserts[:3], collect)
    blob = a.save_state()
    saved = snapshot(a)
    want_step, want_size, want_alpha = a.get_step(), a.buffer_size(), a.get_alpha()
    want = run_steps(a, inserts[3:], collect)
    want_params = {n: a.store[n]["params"].cpu().numpy() for n in NETS}

    b = api.CRLContext(w, precision=precision, path=path)
    for n in NETS:
        for k, v in saved[n].items():
            b.store[n][k].copy_(v)
    b.load_state(blob)
    assert (b.get_step(), b.buffer_size(), b.get_alpha()) == (want_step, want_size, want_alpha)
    got = run_steps(b, inserts[3:], collect)
    np.testing.assert_array_equal(got, want)
    for n in NETS:
        np.testing.assert_array_equal(b.store[n]["params"].cpu().numpy(), want_params[n])
    assert a.get_alpha() == b.get_alpha()
    assert a.buffer_size() == b.buffer_size()
    assert a.sync_status() == (0, 0) and b.sync_status() == (0, 0)


def test_state_size_grows_with_the_environments():
    w = small(E=4, T=20, B=16)
    ctx = api.CRLContext(w)
    for k, v in workload.init_agent(w).items():
        ctx.load_network(k, v)
    n0 = len(ctx.save_state())
    ctx.collect(1, 5)
    n1 = len(ctx.save_state())
    assert n1 - n0 == w.E * (w.D + w.G + 1) * 4 + 8


def test_load_into_an_unused_context_restores_the_buffer():
    """A blob loaded into a fresh context: the buffer relabels to the same batch."""
    w = small(B=48)
    a, _, _ = setup(w, n=25)
    a.set_step(17)
    blob = a.save_state()
    b = api.CRLContext(w)
    b.load_state(blob)
    assert b.get_step() == 17 and b.buffer_size() == a.buffer_size()
    sa, sb = a.sample(step=3, B=w.B), b.sample(step=3, B=w.B)
    for x, y in zip(sa, sb):
        np.testing.assert_array_equal(x.cpu().numpy(), y.cpu().numpy())


def test_load_rejects_foreign_corrupt_and_truncated_blobs():
    w = small(E=4, T=20, B=16)
    ctx = api.CRLContext(w)
    blob = ctx.save_state()
    other = api.CRLContext(small(E=5, T=20, B=16))
    with pytest.raises(api.CRLError) as e:
        other.load_state(blob)
    assert e.value.code == api.E_SHAPE
    bad = b"x" + blob[1:]
    with pytest.raises(api.CRLError) as e:
        ctx.load_state(bad)
    assert e.value.code == api.E_INVALID_ARG
    with pytest.raises(api.CRLError) as e:
        ctx.load_state(blob[:-4])
    assert e.value.code == api.E_SHAPE
    with pytest.raises(api.CRLError) as e:
        ctx.load_state(blob[:8])
    assert e.value.code == api.E_SHAPE
    # header: magic (8 B), 8 int32, then size_host, total_host (int64)
    fill = struct.unpack_from("<q", blob, 8 + 8 * 4)[0]
    assert fill == 0
    corrupt = bytearray(blob)
    struct.pack_into("<q", corrupt, 8 + 8 * 4, w.T + 1)
    with pytest.raises(api.CRLError) as e:
        ctx.load_state(bytes(corrupt))
    assert e.value.code == api.E_INVALID_ARG


def test_load_rejects_a_device_fill_that_disagrees_with_the_header():
    """The blob's copy of the device fill {size, total} feeds the sampler's ring-row
    addresses unchecked, so a blob whose copy disagrees with its validated header
    (here total < size, which would address rows before the ring) is refused, and
    so is a header whose fill is not min(total, T)."""
    w = small(E=4, T=20, B=16)
    ctx = api.CRLContext(w)
    blob = ctx.save_state()
    # header: magic (8 B), 8 int32, size_host, total_host (int64) = 56 B; counters 72 B;
    # episode starts E int32; then the device fill {size, total} (int32)
    off = 56 + 72 + 4 * w.E
    assert struct.unpack_from("<ii", blob, off) == (0, 0)
    corrupt = bytearray(blob)
    struct.pack_into("<ii", corrupt, off, w.T, 3)
    with pytest.raises(api.CRLError) as e:
        ctx.load_state(bytes(corrupt))
    assert e.value.code == api.E_INVALID_ARG
    corrupt = bytearray(blob)
    struct.pack_into("<qq", corrupt, 8 + 8 * 4, w.T, w.T - 1)
    with pytest.raises(api.CRLError) as e:
        ctx.load_state(bytes(corrupt))
    assert e.value.code == api.E_INVALID_ARG
    ctx.load_state(blob)
