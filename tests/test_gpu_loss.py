"""Masked TR fit loss and its hand-written backward on the GPU."""
import numpy as np
import pytest

import synth
from oracle.loss import closed_form_grad, masked_loss, masked_loss_grad
from gpu_util import dev, lib, rel

pytestmark = pytest.mark.gpu


def _abi_cores(G, dtype):
    import torch
    import paper_2307_00719_gb300 as p
    return [torch.from_numpy(a).to("cuda", dtype) for a in p.cores_to_abi(G)]


def _abi_to_paper(g, Ra, Rb):
    g = g.detach().double().cpu().numpy()
    return g.transpose(2, 0, 1)


@pytest.mark.parametrize("dtype_name,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_masked_loss_fwd_bwd(dtype_name, tol):
    import torch
    p = lib()
    dt = torch.float64 if dtype_name == "f64" else torch.float32
    dims, ranks = (8, 8, 8, 8, 5), (3, 3, 3, 3, 3)
    G = synth.gaussian_cores(dims, ranks, 3)
    X = synth.gaussian_tensor(dims, 4)
    mask = synth.bernoulli_keep_mask(dims, 0.3, 3)
    bits = torch.from_numpy(synth.pack_mask_bits(mask).view(np.int32)).cuda()
    cores = _abi_cores(G, dt)
    for use_mask in (True, False):
        mb = bits if use_mask else None
        mk = mask if use_mask else None
        loss = p.tr_masked_loss_fwd(cores, dev(X, dt), mb).item()
        ref = masked_loss(X, G, mk)
        assert abs(loss - ref) <= tol * ref
        grads = p.tr_masked_loss_bwd(cores, dev(X, dt), mb, 1.0)
        gref = masked_loss_grad(X, G, mk)
        for n in range(5):
            assert rel(_abi_to_paper(grads[n], 0, 0), gref[n]) <= tol
    cf = closed_form_grad(X, G)
    grads = p.tr_masked_loss_bwd(cores, dev(X, dt), None, 1.0)
    for n in range(5):
        assert rel(_abi_to_paper(grads[n], 0, 0), cf[n]) <= tol


def test_autograd_function():
    import torch
    p = lib()
    dims, ranks = (6, 5, 4, 7), (2, 3, 2, 2)
    G = synth.gaussian_cores(dims, ranks, 5)
    X = synth.gaussian_tensor(dims, 6)
    mask = synth.bernoulli_keep_mask(dims, 0.3, 7)
    bits = torch.from_numpy(synth.pack_mask_bits(mask).view(np.int32)).cuda()
    cores = [c.requires_grad_(True) for c in _abi_cores(G, torch.float64)]
    loss = p.TRFitLoss.apply(dev(X), bits, *cores)
    (2.0 * loss).backward()
    gref = masked_loss_grad(X, G, mask)
    for n in range(4):
        assert rel(_abi_to_paper(cores[n].grad, 0, 0), 2.0 * gref[n]) <= 1e-12


# Shapes for the fused loss pass: ragged 64-row / 64-column tiles, a prefix of one
# core (order 3 and order 4), a two-core prefix of 1600 rows over 9 columns (many
# row groups, one column block), and a mid-size order-5 tensor.  For the FP32
# tensor-core passes (128 x 128 tiles): K = R_1 R_2 = 64 over 260 rows and 792
# columns (three row tiles, seven column tiles, ragged); K = 36 over 131 rows (an
# odd row count: unaligned columns of X) and 1050 columns; and 4096 rows over 2304
# columns (576 tiles: each CTA walks several tiles and lane tiles).
@pytest.mark.parametrize("dims,ranks", [
    ((70, 9, 13), (2, 3, 4)),
    ((31, 33, 5, 7), (3, 2, 4, 3)),
    ((40, 40, 3, 3), (2, 8, 2, 2)),
    ((16, 16, 16, 16, 12), (4, 4, 4, 4, 4)),
    ((260, 24, 33), (8, 8, 3)),
    ((131, 7, 150), (6, 6, 5)),
    ((64, 64, 48, 48), (3, 2, 3, 2)),
])
@pytest.mark.parametrize("dtype_name,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_masked_loss_tiles_and_groups(dims, ranks, dtype_name, tol):
    import torch
    p = lib()
    dt = torch.float64 if dtype_name == "f64" else torch.float32
    G = synth.gaussian_cores(dims, ranks, 11)
    X = synth.gaussian_tensor(dims, 12)
    mask = synth.bernoulli_keep_mask(dims, 0.3, 13)
    bits = torch.from_numpy(synth.pack_mask_bits(mask).view(np.int32)).cuda()
    cores = _abi_cores(G, dt)
    Xd = dev(X, dt)
    for mb, mk in ((bits, mask), (None, None)):
        loss = p.tr_masked_loss_fwd(cores, Xd, mb).item()
        ref = masked_loss(X, G, mk)
        assert abs(loss - ref) <= tol * ref
        grads = p.tr_masked_loss_bwd(cores, Xd, mb, 0.5)
        gref = masked_loss_grad(X, G, mk)
        for n in range(len(dims)):
            assert rel(_abi_to_paper(grads[n], 0, 0), 0.5 * gref[n]) <= tol, n


def test_loss_calls_replay_from_a_captured_graph():
    """The FP32 tensor-core forward and backward captured into a CUDA graph on a
    side stream (after one eager call has grown the library's workspace): the
    backward's per-core MTTKRPs on the library's side streams become branches of
    the graph, and a replay gives the eager results bit for bit (fixed-order
    reductions)."""
    import torch
    p = lib()
    dims, ranks = (16, 16, 16, 16, 12), (4, 4, 4, 4, 4)
    G = synth.gaussian_cores(dims, ranks, 21)
    X = synth.gaussian_tensor(dims, 22)
    mask = synth.bernoulli_keep_mask(dims, 0.3, 23)
    bits = torch.from_numpy(synth.pack_mask_bits(mask).view(np.int32)).cuda()
    cores = _abi_cores(G, torch.float32)
    Xd = dev(X, torch.float32)
    ref_loss = p.tr_masked_loss_fwd(cores, Xd, bits).item()
    ref_grads = [g.clone() for g in p.tr_masked_loss_bwd(cores, Xd, bits, 1.0)]
    torch.cuda.synchronize()
    st = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=st):
        loss = p.tr_masked_loss_fwd(cores, Xd, bits)
        grads = p.tr_masked_loss_bwd(cores, Xd, bits, 1.0)
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        assert loss.item() == ref_loss
        for g, r in zip(grads, ref_grads):
            assert torch.equal(g, r)
    assert abs(ref_loss - masked_loss(X, G, mask)) <= 1e-5 * ref_loss
