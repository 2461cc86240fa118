"""Acceptance test of an integrator result against the oracle.  TEST
INFRASTRUCTURE ONLY (imported by ``tests/`` and ``__graft_entry__.smoke()``);
it compares arrays and computes no chemistry.

Two bars, both per cell:

* absolute (the acceptance bar of the chemistry substep): |T - T_or| <= 1e-3 K
  and max_k |Y_k - Y_or,k| <= 1e-7 max_k Y_or,k;
* relative to the oracle's own change over the step: |T - T_or| <= rel |T_or - T_in|
  + floor_T and max_k |Y_k - Y_or,k| <= rel max_k |Y_or,k - Y_in,k| + floor_Y max_k Y_or,k,
  with rel = 1e-3.  Over one dt = 1 us the change of a cell can be far below the
  absolute bar (on the 0D H2/air field it is 1e-5 .. 2e-4 K), so the absolute bar
  alone would accept a kernel that returns its input; the relative bar does not.
  The floors (2e-7 K, 1e-10 of the largest mass fraction) are the truncation
  error the integrator's default tolerances leave (at most 1e-7 K and 4e-11 of
  the largest mass fraction on the 9- and 50-species fields): cells that barely
  move are held to that, not to 1e-3 of a change of 1e-6 K.  They sit 50x
  (T) and 20x (Y) below the smallest change of a cell of the 0D H2/air field.

The state must also have moved: the largest change over the cells is at least
``moved`` (100) times the largest error, in T and in Y.
"""
from __future__ import annotations

import numpy as np


def integrator_errors(T_in, Y_in, T, Y, T_or, Y_or):
    """Per-cell errors and changes: (err_T, chg_T, err_Y, chg_Y, maxY), the Y
    figures as maxima over species.  Y arrays are [N, ncells]."""
    T_in, T, T_or = (np.asarray(a, np.float64) for a in (T_in, T, T_or))
    Y_in, Y, Y_or = (np.asarray(a, np.float64) for a in (Y_in, Y, Y_or))
    err_T = np.abs(T - T_or)
    chg_T = np.abs(T_or - T_in)
    err_Y = np.abs(Y - Y_or).max(axis=0)
    chg_Y = np.abs(Y_or - Y_in).max(axis=0)
    return err_T, chg_T, err_Y, chg_Y, np.abs(Y_or).max(axis=0)


def check_integrator(T_in, Y_in, T, Y, T_or, Y_or, tol_T=1e-3, tol_Y=1e-7, rel=1e-3, floor_T=2e-7,
                     floor_Y=1e-10, moved=100.0):
    """Raise AssertionError unless (T, Y) passes both bars against the oracle's
    (T_or, Y_or) from the same inputs (T_in, Y_in).  Returns the figures."""
    err_T, chg_T, err_Y, chg_Y, maxY = integrator_errors(T_in, Y_in, T, Y, T_or, Y_or)
    stats = {"max_err_T": float(err_T.max()), "max_err_Y_rel_maxY": float((err_Y / maxY).max()),
             "max_err_T_over_change": float((err_T / np.maximum(chg_T, 1e-300)).max()),
             "max_err_Y_over_change": float((err_Y / np.maximum(chg_Y, 1e-300)).max()),
             "max_change_T": float(chg_T.max()), "max_change_Y_rel_maxY": float((chg_Y / maxY).max())}
    assert np.all(err_T <= tol_T), ("absolute T", stats, int(err_T.argmax()))
    assert np.all(err_Y <= tol_Y * maxY), ("absolute Y", stats, int((err_Y / maxY).argmax()))
    bad_T = err_T > rel * chg_T + floor_T
    bad_Y = err_Y > rel * chg_Y + floor_Y * maxY
    assert not bad_T.any(), ("T relative to the change", stats, int(np.argmax(bad_T)))
    assert not bad_Y.any(), ("Y relative to the change", stats, int(np.argmax(bad_Y)))
    assert chg_T.max() >= moved * err_T.max() and chg_T.max() > 10 * floor_T, ("T did not move", stats)
    assert (chg_Y / maxY).max() >= moved * (err_Y / maxY).max() and (chg_Y / maxY).max() > 10 * floor_Y, \
        ("Y did not move", stats)
    return stats
