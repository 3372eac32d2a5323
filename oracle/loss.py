"""Masked tensor-ring fit loss and its gradient, by definition (FP64, CPU).

Test infrastructure only: see the package docstring.

Reading: the paper has no masked loss.  The loss is
    L = 1/2 * sum_i M(i) (X(i) - TR(G)(i))^2
with M(i) in {0, 1} (1 = observed), and by the chain rule through the TR format
(Sec. 1) and Eq. tr_als,
    dL/dG_{n(2)} = -(M .* (X - TR(G)))_[n] G^{!=n}_[2].
With M == 1 this equals G_{n(2)} Q_n - P_n, P_n = X_[n] G^{!=n}_[2],
Q_n = (G^{!=n}_[2])^T G^{!=n}_[2] (Eq. partial).
"""
from __future__ import annotations

from typing import List, Optional, Sequence

import numpy as np

from .tr import core_fold2, core_unfold2, gram_explicit, mttkrp, subchain_unfold, tr_full, unfold_cyclic


def masked_loss(X: np.ndarray, cores: Sequence[np.ndarray], mask: Optional[np.ndarray]) -> float:
    res = X - tr_full(cores)
    if mask is not None:
        res = res * mask
    return 0.5 * float(np.sum(res * res))


def masked_loss_grad(X: np.ndarray, cores: Sequence[np.ndarray],
                     mask: Optional[np.ndarray]) -> List[np.ndarray]:
    """Gradient of masked_loss with respect to every core, shaped like the cores."""
    res = X - tr_full(cores)
    if mask is not None:
        res = res * mask
    N = len(cores)
    out = []
    for n in range(1, N + 1):
        g = -(unfold_cyclic(res, n) @ subchain_unfold(cores, n))
        out.append(core_fold2(g, cores[n - 1].shape[0], cores[n % N].shape[0]))
    return out


def closed_form_grad(X: np.ndarray, cores: Sequence[np.ndarray]) -> List[np.ndarray]:
    """G_{n(2)} Q_n - P_n for every n (unmasked case)."""
    N = len(cores)
    out = []
    for n in range(1, N + 1):
        g = core_unfold2(cores[n - 1]) @ gram_explicit(cores, n) - mttkrp(X, cores, n)
        out.append(core_fold2(g, cores[n - 1].shape[0], cores[n % N].shape[0]))
    return out
