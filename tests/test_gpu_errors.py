"""Error paths of the C ABI on the GPU: numerical and argument failures leave
the state unchanged (no GPU fault is involved in any of them)."""
import numpy as np
import pytest

from gpu_util import dev, lib, perturbed_init, problem

pytestmark = pytest.mark.gpu


def test_singular_normal_equations_leave_state_unchanged():
    """A zero spatial core makes every Q_n increment of the other modes zero
    and Q_n singular: the update reports STR_ERR_SINGULAR, nothing changes."""
    p = lib()
    G, X = problem((6, 5), 10, (2, 2, 2), 0)
    init = perturbed_init(G, 5, 0)
    init[1] = np.zeros_like(init[1])
    ctx = p.str_init_cores(init, X0=None)
    before = [ctx.core(n) for n in (1, 2, 3)]
    with pytest.raises(p.StrError) as e:
        ctx.update(dev(X[..., 5:7]))
    assert e.value.status == 4
    assert ctx.time_rows() == 5
    for n in (1, 2, 3):
        assert np.array_equal(ctx.core(n), before[n - 1])


def test_capacity_shape_dtype_and_nonfinite():
    import torch
    p = lib()
    G, X = problem((6, 5), 12, (2, 2, 2), 1)
    init = perturbed_init(G, 6, 1)
    ctx = p.str_init_cores(init, X0=dev(X[..., :6]), t_capacity=8, check_finite=1)
    with pytest.raises(p.StrError) as e:
        ctx.update(dev(X[..., 6:9]))
    assert e.value.status == 6
    with pytest.raises(p.StrError) as e:
        ctx.update(dev(X[:5, :, 6:8]))
    assert e.value.status == 2
    bad = X[..., 6:8].copy()
    bad[1, 2, 0] = np.nan
    with pytest.raises(p.StrError) as e:
        ctx.update(dev(bad))
    assert e.value.status == 5
    assert ctx.time_rows() == 6
    ctx.update(dev(X[..., 6:8]))
    assert ctx.time_rows() == 8
    with pytest.raises(p.StrError) as e:
        ctx.rupdate(dev(X[..., 8:9]))
    assert e.value.status == 10
