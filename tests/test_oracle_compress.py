"""Pins of the oracle's track-model compression (step 10): on an exact helix
fitted exactly every residual code is 0; a cluster moved by k quantisation
steps (16 u in y, 20 u in zeta: the steps are whole multiples of u) gets code
k; one moved beyond 127 steps is escaped; every other cluster keeps code 0."""
import math

import numpy as np
import pytest

import oracle
from synth import Geom, U_CM, helix_points, make_clusters


class _Res:
    def __init__(self, clusters, cl2trk, fits):
        self.clusters, self.cl2trk, self.fits = clusters, cl2trk, fits


def one_track(shift_row=None, dY=0, dZ=0):
    g = Geom(n_sectors=1, n_time_bins=1000)
    rows = np.arange(20, 120)
    x = g.row_x[rows] * 0.05
    y, z = helix_points(x, 2.0, 100.0, 0.1, 0.3, -1.5)
    Y = (np.round(y / U_CM / 2) * 2).astype(np.int64)
    Z = (np.round(z / U_CM / 5) * 5).astype(np.int64)
    cl, order = make_clusters(g, [(0, int(r), int(a), int(b)) for r, a, b in zip(rows, Y, Z)])
    X, Yc, Zc = oracle.coords(g, cl)
    fit = oracle.fit_points(X * U_CM, Yc * U_CM, Zc * U_CM)   # the unshifted track model
    if shift_row is not None:
        pts = [(0, int(r), int(a) + (dY if r == shift_row else 0), int(b) + (dZ if r == shift_row else 0))
               for r, a, b in zip(rows, Y, Z)]
        cl, order = make_clusters(g, pts)
    fits = np.zeros(1, dtype=oracle.FIT_DTYPE)
    fits[0] = fit
    return g, _Res(cl, np.zeros(len(cl), np.int32), fits), cl


def test_exact_helix_codes_are_zero():
    g, r, cl = one_track()
    cy, cz, st = oracle.compress(g, r)
    assert np.all(st == 1) and np.all(cy == 0) and np.all(cz == 0)


@pytest.mark.parametrize("k", [1, -3, 17, 127, -127])
def test_moved_cluster_gets_its_step_count(k):
    g, r, cl = one_track(shift_row=60, dY=16 * k, dZ=-20 * k)
    cy, cz, st = oracle.compress(g, r)
    i = int(np.nonzero(cl["row"] == 60)[0][0])
    assert st[i] == 1 and cy[i] == k and cz[i] == -k
    others = np.arange(len(cl)) != i
    assert np.all(st[others] == 1) and np.all(cy[others] == 0) and np.all(cz[others] == 0)


def test_cluster_beyond_127_steps_is_escaped():
    g, r, cl = one_track(shift_row=60, dY=16 * 128)
    cy, cz, st = oracle.compress(g, r)
    i = int(np.nonzero(cl["row"] == 60)[0][0])
    assert st[i] == 2
    assert np.all(st[np.arange(len(cl)) != i] == 1)
