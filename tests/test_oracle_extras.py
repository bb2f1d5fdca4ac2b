"""Pins of the oracle's LOS-independent extras (Sec. 2): the random-random
normalised correlation function (norm=2), the FKP shot-noise level and
interlaced transforms.

- Randoms on every node of the mesh make RR_0(r) the same in every bin, and
  with nbar V_cell = alpha_r the RR-normalised xi_ell equals the FKP-normalised
  one exactly (A V_cell = alpha_r^2 N^3 = RR_0): a closed form that fails if
  alpha_r^2, the ell of RR or its line of sight were wrong.
- xi with norm=2 does not change when the randoms' weights are all scaled (the
  FKP-normalised xi does): alpha_r n_r and alpha_r^2 RR are unchanged.
- Parseval: for galaxies and randoms on distinct nodes (CIC puts each on one
  node), the mean of |delta(k)|^2 over all k != 0 is N^3 / (N^3 - 1) times
  sum_g w^2 + alpha_r^2 sum_r w^2 (delta(k=0) = 0 by the choice of alpha_r), so
  P_0 with one bin over every mode equals that multiple of the shot noise.
- Interlacing: the interlaced transform of one particle off the nodes, written out
  per axis by hand on both meshes (which fixes the direction of the shift and the
  sign of its phase); real fields keep Hermitian transforms; on a smooth density the
  interlaced CIC monopole at high k lies closer to a 4x finer mesh than the plain one.
"""
import math

import numpy as np
import pytest

from oracle import estimators as E

N = 16
BOX_LO = np.array([512.0, 512.0, 512.0])
BOX = 1024.0                      # h = 64: node positions are exact in float32


def _nodes(idx):
    h = BOX / N
    x = BOX_LO[None, :] + np.asarray(idx, dtype=np.float64) * h
    return np.concatenate([x, np.ones((len(idx), 1))], axis=1).astype(np.float32)


def _flat_to_idx(flat):
    return np.stack([flat // (N * N), (flat // N) % N, flat % N], axis=1)


@pytest.fixture(scope="module")
def full_randoms():
    rng = np.random.default_rng(11)
    gal = _nodes(_flat_to_idx(rng.integers(0, N ** 3, size=300)))
    ran = _nodes(_flat_to_idx(np.arange(N ** 3)))
    nbar = len(gal) / BOX ** 3                      # nbar V_cell = alpha_r
    return gal, ran, np.full(len(ran), nbar, np.float32)


@pytest.mark.parametrize("los,K", [("yamamoto", 0), ("midpoint", 2), ("bisector", 2)])
def test_rr_normalisation_equals_fkp_for_node_filling_randoms(full_randoms, los, K):
    gal, ran, nbar = full_randoms
    redges = np.linspace(0.0, 400.0, 6)
    kw = dict(N=N, box_lo=BOX_LO, box_len=BOX, assign=2, ell_max=2, los=los, order=K, redges=redges)
    fkp = E.xi_multipoles(gal, ran, nbar, norm=1, **kw)["xi"]
    rr = E.xi_multipoles(gal, ran, nbar, norm=2, **kw)["xi"]
    np.testing.assert_allclose(rr, fkp, rtol=1e-12, atol=1e-12 * np.abs(fkp).max())


def test_rr_normalisation_ignores_random_weight_scale():
    rng = np.random.default_rng(5)
    gal = _nodes(rng.integers(4, 12, size=(200, 3)))
    ran = _nodes(rng.integers(3, 13, size=(2000, 3)))
    ran_w = ran.copy()
    ran_w[:, 3] *= 3.0
    nbar = np.full(len(ran), 1e-6, np.float32)
    redges = np.linspace(0.0, 400.0, 6)
    kw = dict(N=N, box_lo=BOX_LO, box_len=BOX, assign=2, ell_max=2, los="midpoint", order=2, redges=redges)
    a = E.xi_multipoles(gal, ran, nbar, norm=2, **kw)["xi"]
    b = E.xi_multipoles(gal, ran_w, nbar, norm=2, **kw)["xi"]
    np.testing.assert_allclose(b, a, rtol=1e-10, atol=1e-12 * np.abs(a).max())
    f1 = E.xi_multipoles(gal, ran, nbar, norm=1, **kw)["xi"]
    f3 = E.xi_multipoles(gal, ran_w, nbar, norm=1, **kw)["xi"]
    assert np.abs(f3 - f1).max() > 0.1 * np.abs(f1).max()


def test_shot_noise_parseval_on_distinct_nodes():
    rng = np.random.default_rng(7)
    flat = rng.choice(N ** 3, size=900, replace=False)
    gal = _nodes(_flat_to_idx(flat[:300]))
    ran = _nodes(_flat_to_idx(flat[300:]))
    gal[:, 3] = rng.uniform(0.5, 1.5, size=len(gal)).astype(np.float32)   # weights enter as w^2
    ran[:, 3] = rng.uniform(0.5, 1.5, size=len(ran)).astype(np.float32)
    nbar = np.full(len(ran), 2e-7, np.float32)
    kedges = np.array([1e-9, 1e9])
    for norm in (0, 1):
        p0 = E.pk_multipoles(gal, ran, nbar, N=N, box_lo=BOX_LO, box_len=BOX, assign=2, ell_max=0,
                             los="yamamoto", order=0, kedges=kedges, norm=norm)["pk"][0, 0]
        sn = E.shot_noise(gal, ran, nbar, norm=norm)
        assert math.isclose(p0, N ** 3 / (N ** 3 - 1) * sn, rel_tol=1e-11), (norm, p0, sn)


def test_shot_noise_of_one_particle_is_its_power():
    # one galaxy on a node, no randoms, raw normalisation: |delta(k)|^2 = w^2 for every k
    gal = _nodes(np.array([[5, 9, 2]]))
    gal[0, 3] = 1.75
    kedges = np.linspace(0.0, math.pi / (BOX / N), 5)
    p0 = E.pk_multipoles(gal, None, None, N=N, box_lo=BOX_LO, box_len=BOX, assign=2, ell_max=0, los="yamamoto",
                         order=0, kedges=kedges, norm=0)["pk"][0]
    np.testing.assert_allclose(p0[1:], E.shot_noise(gal, None, None, norm=0), rtol=1e-12)


# ---------------------------------------------------------------- interlacing
def test_interlaced_transform_of_one_particle():
    # one particle a quarter cell past a node along every axis, CIC, no compensation: on the
    # mesh the per-axis factor is 3/4 + 1/4 e^{-i theta}; on the mesh shifted by +h/2 the
    # particle sits 3/4 cell past node i0 - 1, giving (1/4 e^{i theta} + 3/4) in the mesh's
    # frame and (1/4 e^{i theta/2} + 3/4 e^{-i theta/2}) after the shift's phase; theta = k_d h
    from oracle import mesh
    i0 = np.array([5, 9, 2])
    h = BOX / N
    gal = np.concatenate([BOX_LO + (i0 + 0.25) * h, [1.0]])[None, :].astype(np.float32)
    kedges = np.linspace(1e-6, math.pi / h * math.sqrt(3.0) * 1.001, 7)
    got = E.pk_multipoles(gal, None, None, N=N, box_lo=BOX_LO, box_len=BOX, assign=2, ell_max=0, los="yamamoto",
                          order=0, kedges=kedges, norm=0, interlace=True)
    n = mesh.fft_labels(N).astype(np.float64)
    th = 2 * math.pi * n / N
    f1 = 0.75 + 0.25 * np.exp(-1j * th)
    f2 = 0.25 * np.exp(0.5j * th) + 0.75 * np.exp(-0.5j * th)
    f2 = np.where(n == -N // 2, 0.0, f2)       # the Nyquist index carries no shifted term
    F = 0.5 * (f1[:, None, None] * f1[None, :, None] * f1[None, None, :]
               + f2[:, None, None] * f2[None, :, None] * f2[None, None, :])
    kmag = mesh.k_magnitude(N, BOX)
    want = [np.mean(np.abs(F[(kmag >= a) & (kmag < b)]) ** 2) for a, b in zip(kedges[:-1], kedges[1:])]
    np.testing.assert_allclose(got["pk"][0], want, rtol=1e-12)
    # without interlacing: |f1|^2 per axis
    plain = E.pk_multipoles(gal, None, None, N=N, box_lo=BOX_LO, box_len=BOX, assign=2, ell_max=0, los="yamamoto",
                            order=0, kedges=kedges, norm=0)
    F1 = f1[:, None, None] * f1[None, :, None] * f1[None, None, :]
    want1 = [np.mean(np.abs(F1[(kmag >= a) & (kmag < b)]) ** 2) for a, b in zip(kedges[:-1], kedges[1:])]
    np.testing.assert_allclose(plain["pk"][0], want1, rtol=1e-12)


def test_interlaced_transforms_are_hermitian():
    rng = np.random.default_rng(2)
    gal = _nodes(rng.uniform(3, 12, size=(500, 3)))
    _, _, _, _, _, tr = E._prepare(gal, None, None, N, BOX_LO, BOX, 3, 0, True, interlace=True)
    from oracle.special import ylm
    for wfun in (None, lambda x: ylm(2, 0, x).real, lambda x: ylm(4, -3, x).real):   # real weights
        F = tr.fwd(wfun)
        np.testing.assert_allclose(E._flip_k(F), np.conj(F), atol=1e-12 * np.abs(F).max())


def test_interlacing_reduces_aliasing():
    # a smooth (band-limited) density of many particles: the interlaced CIC monopole at high k
    # lies closer to the alias-free result (the same particles with a 4x finer mesh, cut to
    # the same k) than the plain one
    rng = np.random.default_rng(8)
    pts = rng.uniform(0.0, 1.0, size=(20000, 3))
    gal = np.concatenate([BOX_LO + pts * BOX, np.ones((len(pts), 1))], 1).astype(np.float32)
    kedges = np.linspace(0.5, 0.95, 4) * math.pi / (BOX / N)
    kw = dict(box_lo=BOX_LO, box_len=BOX, assign=2, ell_max=0, los="yamamoto", order=0, kedges=kedges, norm=0,
              compensate=True)
    fine = E.pk_multipoles(gal, None, None, N=4 * N, **kw)["pk"][0]
    plain = E.pk_multipoles(gal, None, None, N=N, **kw)["pk"][0]
    inter = E.pk_multipoles(gal, None, None, N=N, interlace=True, **kw)["pk"][0]
    assert np.all(np.abs(inter - fine) < np.abs(plain - fine)), (plain, inter, fine)
