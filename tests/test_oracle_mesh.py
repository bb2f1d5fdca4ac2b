"""Pins of oracle.mesh: painting by hand, FKP factors, shell assignment."""
import math

import numpy as np

from oracle import mesh


def test_cic_by_hand():
    # one particle, w = 2, at u = (1.25, 2.5, 3.75) on a 4^3 mesh with h = 1
    d = mesh.paint(np.array([[1.25, 2.5, 3.75, 2.0]]), 1.0, 4, [0, 0, 0], 4.0, 2)
    wx = {1: 0.75, 2: 0.25}
    wy = {2: 0.5, 3: 0.5}
    wz = {3: 0.25, 0: 0.75}          # node 4 wraps to node 0
    want = np.zeros((4, 4, 4))
    for i, a in wx.items():
        for j, b in wy.items():
            for k, c in wz.items():
                want[i, j, k] = 2.0 * a * b * c
    np.testing.assert_allclose(d, want, atol=1e-15)
    assert d.sum() == 2.0


def test_tsc_by_hand():
    # u = (1.2, 0.0, 3.6): nearest nodes 1, 0, 0 (3.6 -> 4 -> wraps to 0), offsets 0.2, 0.0, -0.4
    d = mesh.paint(np.array([[1.2, 0.0, 3.6, 1.0]]), 1.0, 4, [0, 0, 0], 4.0, 3)
    wx = {0: 0.5 * 0.3 ** 2, 1: 0.75 - 0.2 ** 2, 2: 0.5 * 0.7 ** 2}
    wy = {3: 0.125, 0: 0.75, 1: 0.125}
    wz = {3: 0.5 * 0.9 ** 2, 0: 0.75 - 0.4 ** 2, 1: 0.5 * 0.1 ** 2}
    want = np.zeros((4, 4, 4))
    for i, a in wx.items():
        for j, b in wy.items():
            for k, c in wz.items():
                want[i, j, k] += a * b * c
    np.testing.assert_allclose(d, want, atol=1e-15)
    assert abs(d.sum() - 1.0) < 1e-14


def test_snapped_particle_deposits_on_one_node():
    d = mesh.paint(np.array([[10.0 + 3 * 2.0, 10.0, 10.0 + 7 * 2.0, 1.5]]), 1.0, 8, [10, 10, 10], 16.0, 2)
    assert d[3, 0, 7] == 1.5 and np.count_nonzero(d) == 1


def test_norm_factors_by_hand():
    gal = np.array([[0, 0, 0, 1.0], [0, 0, 0, 2.0]])
    ran = np.array([[0, 0, 0, 1.0], [0, 0, 0, 1.0], [0, 0, 0, 2.0]])
    alpha, A = mesh.norm_factors(gal, ran, np.array([0.5, 0.5, 1.0]))
    assert alpha == 0.75
    assert A == 0.75 * (0.5 + 0.5 + 4.0)
    assert mesh.norm_factors(gal, None, None) == (0.0, None)


def test_shell_index_half_open():
    b = mesh.shell_index(np.array([0.0, 0.5, 1.0, 2.999, 3.0, -1.0]), np.array([0.0, 1.0, 2.0, 3.0]))
    assert b.tolist() == [0, 0, 1, 2, -1, -1]


def test_compensation_window():
    W = mesh.compensation(8, 2)
    assert W[0, 0, 0] == 1.0
    assert math.isclose(W[4, 0, 0], (2 / math.pi) ** 2, rel_tol=1e-14)   # label -4, |x| = pi/2
    np.testing.assert_allclose(W[1, 2, 3], W[-1, -2, -3])
    assert math.isclose(mesh.compensation(8, 3)[4, 4, 4], (2 / math.pi) ** 9, rel_tol=1e-13)


def test_grids_labels():
    assert mesh.fft_labels(6).tolist() == [0, 1, 2, -3, -2, -1]
    km = mesh.k_magnitude(4, 2 * math.pi)
    assert km[1, 2, 3] == math.sqrt(1 + 4 + 1)
