"""The benchmark's host-side input builder and roofline arithmetic (CPU only).

bench.py builds every input tensor on the host in FP64 so that the GPU arm and
the FP64 oracle read the same bytes; its TR builder is checked here against the
oracle's TR format (the trace formula, Sec. 1) on small shapes."""
import numpy as np
import pytest

import bench
import synth
from oracle import tr as otr


@pytest.mark.parametrize("dims,ranks", [((4, 5, 6), (2, 3, 2)), ((3, 4, 2, 5), (2, 1, 3, 2)),
                                        ((2, 3, 2, 2, 3), (3, 2, 2, 1, 2))])
def test_host_tr_tensor_is_the_tr_format(dims, ranks):
    G = synth.gaussian_cores(dims, ranks, 31)
    X = bench.host_tr_tensor(G)
    np.testing.assert_allclose(X, otr.tr_full(G), rtol=1e-12, atol=1e-12)
    i = tuple(d - 1 for d in dims)
    assert abs(X[i] - otr.tr_entry(G, i)) <= 1e-12 * max(1.0, abs(X[i]))
    # a temporal window [t0, t1) is the same window of the whole tensor
    Xw = bench.host_tr_tensor(G, 1, dims[-1] - 1)
    np.testing.assert_allclose(Xw, X[..., 1:dims[-1] - 1], rtol=1e-12, atol=1e-12)


def test_host_workload_noise_level_and_init():
    w = synth.Workload("t", (6, 5), 12, (2, 3, 2), 4, 1e-2, 4, 2)
    G, X, init = bench.host_workload(w, w.seed)
    Xt = otr.tr_full(G)
    assert abs(np.linalg.norm(X - Xt) / np.linalg.norm(Xt) - 1e-2) < 1e-12
    assert init[-1].shape[1] == w.t_init
    assert all(np.linalg.norm(a[:, :b.shape[1]] - b) > 0 for a, b in zip(G, init))


def test_step_roofline_takes_the_larger_bound():
    r = bench.step_roofline(1.0, 2e12, 1000.0, 1e6, 5000.0, "tf32")     # 2 ms of flop, 0.2 us of bytes
    assert r["bound"] == "tf32" and r["t_bound_us"] == pytest.approx(2000.0) and r["frac_step"] == pytest.approx(2.0)
    r = bench.step_roofline(1.0, 1e6, 1000.0, 5e9, 5000.0, "tf32")      # 1 ms of bytes
    assert r["bound"] == "hbm" and r["frac_step"] == pytest.approx(1.0)
    assert bench.str_flop((4, 5), 3, (2, 3, 4), 2) == 2.0 * 60 * (6 + 12 + 8) * 2
