"""The masked-loss forward that allocates no device memory.

Some callers cannot call cudaMalloc (code whose framework allocator owns the
device memory, loops that cannot take cudaMalloc's synchronisation).
tr_masked_loss_fwd_noalloc serves them from a fixed 32 MiB device array; here
it is called through the C ABI and must give the same loss as
tr_masked_loss_fwd on two calls in a row, leave the device's free memory
unchanged on the second call, and reject a problem whose scratch does not fit.
This file is collected last on purpose.
"""
from ctypes import c_int, c_int64, c_void_p

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _lib():
    import __graft_entry__ as g
    g.build()
    import paper_2307_00719_gb300 as p
    return p


def _args(p, G, X, dtype):
    import torch
    N = len(G)
    cores = [torch.from_numpy(a).to("cuda", dtype) for a in p.cores_to_abi(G)]
    rev = list(range(X.ndim - 1, -1, -1))
    Xd = torch.from_numpy(np.ascontiguousarray(X.transpose(rev))).to("cuda", dtype)
    dims = (c_int64 * N)(*[g.shape[1] for g in G])
    ranks = (c_int * N)(*[g.shape[0] for g in G])
    ptrs = (c_void_p * N)(*[c.data_ptr() for c in cores])
    code = p.STR_F64 if dtype == torch.float64 else p.STR_F32
    return N, dims, ranks, code, ptrs, Xd, cores


@pytest.mark.parametrize("dtype_name,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_noalloc_loss_matches_allocating_entry_point(dtype_name, tol):
    import torch
    p = _lib()
    L = p.lib()
    dtype = torch.float64 if dtype_name == "f64" else torch.float32
    dims, ranks = (9, 7, 8, 6, 5), (3, 2, 3, 2, 3)
    G = synth.gaussian_cores(dims, ranks, 21)
    X = synth.gaussian_tensor(dims, 22)
    bits = torch.from_numpy(synth.pack_mask_bits(synth.bernoulli_keep_mask(dims, 0.3, 23)).view(np.int32)).cuda()
    N, d, r, code, ptrs, Xd, keep = _args(p, G, X, dtype)
    stream = c_void_p(torch.cuda.current_stream().cuda_stream)
    ref = torch.zeros((), dtype=torch.float64, device="cuda")
    assert L.tr_masked_loss_fwd(N, d, r, code, ptrs, c_void_p(Xd.data_ptr()), c_void_p(bits.data_ptr()),
                                c_void_p(ref.data_ptr()), stream) == 0
    outs = [torch.full((), -1.0, dtype=torch.float64, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    free = []
    for out in outs:
        assert L.tr_masked_loss_fwd_noalloc(N, d, r, code, ptrs, c_void_p(Xd.data_ptr()),
                                            c_void_p(bits.data_ptr()), c_void_p(out.data_ptr()), stream) == 0
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        assert abs(out.item() - ref.item()) <= tol * abs(ref.item())
    # the first call may load the array's module and kernels; the second allocates nothing
    assert free[1] == free[0]


def test_noalloc_rejects_scratch_beyond_its_limit():
    import torch
    p = _lib()
    L = p.lib()
    dims, ranks = (4, 4, 64, 64, 32), (6, 6, 6, 6, 6)   # suffix table alone > 32 MiB in FP64
    G = synth.gaussian_cores(dims, ranks, 24)
    X = np.zeros(dims)
    N, d, r, code, ptrs, Xd, keep = _args(p, G, X, torch.float64)
    out = torch.full((), -1.0, dtype=torch.float64, device="cuda")
    st = L.tr_masked_loss_fwd_noalloc(N, d, r, code, ptrs, c_void_p(Xd.data_ptr()), None,
                                      c_void_p(out.data_ptr()), c_void_p(0))
    assert st == 2
    assert b"bytes of scratch" in L.str_last_error()
    torch.cuda.synchronize()
    assert out.item() == -1.0
