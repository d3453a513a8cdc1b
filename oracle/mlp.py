"""FP64 reference of the parameter selector (features and network); TEST INFRASTRUCTURE ONLY.

The arithmetic is in ``mlp_oracle.c``; this module marshals numpy arrays.

* :func:`features`  -- the 64 selector inputs of a tree (its partition rectangles, Section 4)
* :func:`forward`   -- class probabilities of the 64 -> 128 -> 128 -> 225 network
* :func:`loss_grad` -- mean softmax cross-entropy and its gradient (textbook backward pass)
* :func:`nparams`   -- 53,857
"""
from __future__ import annotations

import numpy as np

from . import _f64, _load, _ptr

N_IN, N_HIDDEN, N_OUT = 64, 128, 225


def nparams() -> int:
    return int(_load().orc_mlp_nparams())


def features(rects, L: int, n: int, tol: float) -> np.ndarray:
    r = _f64(rects).reshape(-1)
    assert r.size == 4 * ((4 ** (L + 1) - 1) // 3)
    out = np.empty(N_IN, np.float64)
    _load().orc_features(_ptr(r), int(L), int(n), float(tol), _ptr(out))
    return out


def forward(params, X) -> np.ndarray:
    p = _f64(params)
    assert p.size == nparams()
    X = _f64(X).reshape(-1, N_IN)
    out = np.empty((X.shape[0], N_OUT), np.float64)
    _load().orc_mlp_forward(_ptr(p), _ptr(X), X.shape[0], _ptr(out))
    return out


def loss_grad(params, X, labels):
    p = _f64(params)
    assert p.size == nparams()
    X = _f64(X).reshape(-1, N_IN)
    y = np.ascontiguousarray(labels, np.int32)
    assert y.shape == (X.shape[0],) and y.min() >= 0 and y.max() < N_OUT
    g = np.empty(p.size, np.float64)
    loss = _load().orc_mlp_loss_grad(_ptr(p), _ptr(X), _ptr(y), X.shape[0], _ptr(g))
    return float(loss), g
