"""STR core solves when the normal-equation matrix Q_n is ill conditioned.

Core 2's slices get two rows equal up to delta = 1e-3, so two groups of
columns of mode 1's subchain G^{!=1}_[2] nearly coincide and Q_1 (their Gram,
Sec. 3.1) has a condition number near 1e7.  The core solve
G_{1(2)} = P_1 Q_1^dagger (Alg. 4) must still be an FP64-accurate solve of the
library's own P_1, Q_1: its normwise backward error
||G_1 Q_1 - P_1|| / (||G_1|| ||Q_1||) stays at FP64 rounding level.  With FP32
slab arithmetic the FP32 inverse cannot seed a converging refinement at this
condition number (cond(Q) u_32 is above 1), so the solve must go through the
FP64 fallback, which the context's statistics count."""
import numpy as np
import pytest

import synth
from oracle import stream as ost
from oracle import tr as otr
from gpu_util import dev, lib, rel

pytestmark = pytest.mark.gpu


def _problem(delta):
    dims, T, ranks = (12, 10), 16, (3, 3, 3)
    G = synth.gaussian_cores(dims + (T,), ranks, 40)
    rng = np.random.default_rng(41)
    G[1][1] = G[1][0] + delta * rng.standard_normal(G[1][0].shape)
    X = synth.add_noise(otr.tr_full(G), synth.gaussian_tensor(dims + (T,), 42), 1e-3)
    init = [G[0], G[1], G[2][:, :8, :]]
    return X, init


@pytest.mark.parametrize("compute", ["f64", "f32"])
def test_ill_conditioned_q_is_solved_to_fp64_accuracy(compute):
    import torch
    p = lib()
    X, init = _problem(1e-3)
    dt = torch.float64 if compute == "f64" else torch.float32
    if compute == "f32":
        X = X.astype(np.float32).astype(np.float64)
    ctx = p.str_init_cores(init, X0=dev(X[..., :8], dt), compute=compute)
    ctx.update(dev(X[..., 8:14], dt))
    P1, Q1 = ctx.pq(1)
    ev = np.linalg.eigvalsh(Q1)
    assert ev[-1] / ev[0] > 1e6                     # the case is as ill conditioned as intended
    G1 = otr.core_unfold2(ctx.core(1))
    back = np.linalg.norm(G1 @ Q1 - P1) / (np.linalg.norm(G1) * np.linalg.norm(Q1))
    assert back <= 1e-13, back
    st = ctx.stats()
    if compute == "f32":
        assert st["fp64_fallbacks"] > 0
    # against the oracle on the same values.  FP64: the solution moves by about
    # cond(Q_1) n u (1.6e7 x 9 x 1.1e-16 = 1.6e-8), so cores and fit agree to 1e-7.
    # FP32: P_1 carries the FP32 MTTKRP's rounding (u_32 relative), which the
    # solve moves along the weak direction of Q_1 by 1 / sigma_min; its effect on
    # the reconstruction is at most u_32 sqrt(cond(Q_1)) of ||X||, which bounds
    # the change of the relative fit error.
    ref = ost.str_init(X[..., :8], init)
    ost.str_update(ref, X[..., 8:14])
    e_gpu = ctx.fit_error(dev(X[..., :14], dt))
    e_ref = otr.fit_error(X[..., :14], ref.cores)
    kappa = ev[-1] / ev[0]
    if compute == "f64":
        assert abs(e_gpu - e_ref) <= 1e-7 * e_ref
        for n in (1, 2, 3):
            assert rel(ctx.core(n), ref.cores[n - 1]) <= 1e-7
    else:
        assert abs(e_gpu - e_ref) <= 2 * 2.0 ** -24 * np.sqrt(kappa)
    ctx.close()
