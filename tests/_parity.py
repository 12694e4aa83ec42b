"""Entry-wise comparison used by the GPU parity tests (not collected: no test_ prefix).

A column-norm check (max_j ||Y_j - Yref_j|| / ||Yref_j||) can miss errors confined to a few
small entries of a column, such as modes at the kinetic-energy cutoff.  assert_entrywise
bounds every entry on its own:

    |Y_ij - Yref_ij| <= rtol |Yref_ij| + floor max_i |Yref_ij|

rtol is the relative tolerance of the precision under test; floor is the absolute error of
that precision's arithmetic, relative to the column's largest entry (the rounding of the
transforms does not shrink with an entry that is small by cancellation).
"""
import numpy as np


def assert_entrywise(Y, Yref, rtol, floor, what=""):
    Y = np.asarray(Y)
    Yref = np.asarray(Yref)
    assert Y.shape == Yref.shape, (Y.shape, Yref.shape)
    if Yref.ndim == 1:
        Y, Yref = Y[:, None], Yref[:, None]
    Y2 = Y.reshape(Y.shape[0], -1)
    R2 = Yref.reshape(Yref.shape[0], -1)
    scale = np.abs(R2).max(axis=0, keepdims=True)
    bound = rtol * np.abs(R2) + floor * scale
    d = np.abs(Y2 - R2)
    bad = d > bound
    if bad.any():
        worst = np.unravel_index(np.argmax(d / np.maximum(bound, 1e-300)), d.shape)
        raise AssertionError(
            f"{what}: {int(bad.sum())} of {d.size} entries beyond |d| <= {rtol:g}|ref| + {floor:g} max|ref|;"
            f" worst at {worst}: |d| = {d[worst]:.3e}, |ref| = {abs(R2[worst]):.3e},"
            f" column max {scale[0, worst[1]]:.3e}")


def worst_ratios(Y, Yref):
    """(max |d_ij| / |ref_ij| over entries with |ref_ij| >= 1e-3 max, max |d_ij| / max|ref_:j|):
    the relative and absolute error scales an entry-wise bound has to cover."""
    Y = np.asarray(Y).reshape(np.asarray(Y).shape[0], -1)
    R = np.asarray(Yref).reshape(Y.shape)
    scale = np.abs(R).max(axis=0, keepdims=True)
    d = np.abs(Y - R)
    big = np.abs(R) >= 1e-3 * scale
    rel = float((d[big] / np.abs(R[big])).max()) if big.any() else 0.0
    return rel, float((d / scale).max())
