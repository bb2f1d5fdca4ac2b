"""Synthetic catalogs with the shapes of the paper's workloads (Sec. 7.2).

The paper measures on MultiDark-Patchy BOSS DR12 NGC mocks (Sec. 7.2), which
are not available here.  Two seeded stand-ins are generated instead:

* ``uniform_cube_catalog`` -- uniform points in a cube at a fixed distance
  from the observer, with uniform randoms (the small FP64 workload);
* ``lognormal_cap_catalog`` -- a survey-like sample: a lognormal density with
  a power-law spectrum, Poisson-sampled inside a spherical cap, Kaiser
  redshift-space displacements along each galaxy's own radial direction,
  uniform-in-volume randoms and FKP weights.

Positions and weights are returned as float32 (n, 4) arrays (x, y, z, w) with
float32 nbar per object, exactly the values both the library and the oracle
consume.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Catalog:
    gal: np.ndarray            # (n_g, 4) float32: x, y, z, w
    ran: np.ndarray            # (n_r, 4) float32
    gal_nbar: np.ndarray       # (n_g,) float32
    ran_nbar: np.ndarray       # (n_r,) float32
    box_lo: np.ndarray         # (3,) float64, mesh node 0
    box_len: float             # cubic box side
    meta: dict


def _rotation_to(pole: np.ndarray) -> np.ndarray:
    """Rotation matrix taking +z to the unit vector ``pole``."""
    z = np.array([0.0, 0.0, 1.0])
    p = pole / np.linalg.norm(pole)
    v = np.cross(z, p)
    s = np.linalg.norm(v)
    c = float(z @ p)
    if s < 1e-15:
        return np.eye(3) if c > 0 else np.diag([1.0, -1.0, -1.0])
    vx = np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])
    return np.eye(3) + vx + vx @ vx * ((1 - c) / s ** 2)


def uniform_cube_catalog(seed: int = 0, n_gal: int = 4096, n_ran: int = 40960,
                         side: float = 500.0, distance: float = 1000.0,
                         box_factor: float = 2.0) -> Catalog:
    """Uniform galaxies and randoms in a cube of the given side whose centre
    sits ``distance`` from the observer along (1,1,1)/sqrt(3); unit weights,
    nbar = n_gal / side^3; the mesh box is the cube ``box_factor`` times wider
    with the same centre."""
    rng = np.random.default_rng(seed)
    centre = distance * np.ones(3) / math.sqrt(3.0)
    gal = rng.uniform(-0.5, 0.5, size=(n_gal, 3)) * side + centre
    ran = rng.uniform(-0.5, 0.5, size=(n_ran, 3)) * side + centre
    nbar = n_gal / side ** 3
    g = np.concatenate([gal, np.ones((n_gal, 1))], axis=1).astype(np.float32)
    r = np.concatenate([ran, np.ones((n_ran, 1))], axis=1).astype(np.float32)
    box_len = box_factor * side
    return Catalog(g, r, np.full(n_gal, nbar, np.float32), np.full(n_ran, nbar, np.float32),
                   centre - 0.5 * box_len, box_len,
                   {"kind": "uniform_cube", "seed": seed, "side": side, "distance": distance})


def snapped_catalog(seed: int, n_gal: int, N: int, box_lo, box_len: float,
                    fill: float = 0.4, n_ran: int = 0) -> Catalog:
    """Points placed exactly on mesh nodes (node-snapped), inside the central
    ``fill`` fraction of the box, unit weights.  box_lo and box_len/N should be
    exactly representable in float32 so that each point is a node."""
    rng = np.random.default_rng(seed)
    h = box_len / N
    lo = int(round(N * (0.5 - fill / 2)))
    hi = int(round(N * (0.5 + fill / 2)))
    box_lo = np.asarray(box_lo, dtype=np.float64)

    def draw(n):
        idx = rng.integers(lo, hi, size=(n, 3))
        x = box_lo[None, :] + idx * h
        return np.concatenate([x, np.ones((n, 1))], axis=1).astype(np.float32)

    g = draw(n_gal)
    r = draw(n_ran) if n_ran else np.zeros((0, 4), np.float32)
    nbar = n_gal / ((hi - lo) * h) ** 3
    return Catalog(g, r, np.full(len(g), nbar, np.float32), np.full(len(r), nbar, np.float32),
                   box_lo, float(box_len), {"kind": "snapped", "seed": seed})


def _cap_directions(rng, n, cos_max):
    mu = rng.uniform(cos_max, 1.0, size=n)
    ph = rng.uniform(0.0, 2 * math.pi, size=n)
    s = np.sqrt(np.maximum(0.0, 1 - mu * mu))
    return np.stack([s * np.cos(ph), s * np.sin(ph), mu], axis=1)


def lognormal_cap_catalog(seed: int = 1, n_gal: int = 1_000_000, ran_factor: float = 10.0,
                          half_angle_deg: float = 30.0, r_min: float = 800.0,
                          r_max: float = 1600.0, pk_amp: float = 2e4, pk_slope: float = -1.5,
                          k0: float = 0.1, f_growth: float = 0.7, bias: float = 2.0,
                          P0: float = 1e4, gen_mesh: int = 256, box_factor: float = 2.0,
                          pole=(1.0, 1.0, 1.0)) -> Catalog:
    """Survey-like mock.  Steps:
    1. Gaussian field G on ``gen_mesh``^3 over a cube (pole-aligned frame)
       enclosing the cap, with power P(k) = pk_amp (k/k0)^pk_slope;
    2. lognormal density 1 + delta_LN = exp(G - sigma^2/2);
    3. Poisson counts nbar V_cell (1 + delta_LN) per cell, uniform jitter in
       the cell, kept inside the cap (half-angle, r_min..r_max);
    4. Kaiser displacement: psi(k) = i k delta_m(k)/k^2 with delta_m = G/bias,
       each galaxy moved by f (psi . rhat) rhat along its own radial direction;
    5. ran_factor * n_gal uniform-in-volume randoms in the cap;
    6. nbar = n_gal / V_cap, FKP weights w = 1/(1 + nbar P0);
    7. rotate the pole-aligned frame onto ``pole``; the mesh box is the
       axis-aligned bounding cube of the randoms widened by ``box_factor``."""
    rng = np.random.default_rng(seed)
    cos_max = math.cos(math.radians(half_angle_deg))
    sin_max = math.sin(math.radians(half_angle_deg))
    v_cap = 2 * math.pi * (1 - cos_max) * (r_max ** 3 - r_min ** 3) / 3.0
    nbar = n_gal / v_cap

    # pole-aligned generation cube
    zlo = r_min * cos_max
    side = max(r_max - zlo, 2 * r_max * sin_max) * 1.02
    g_lo = np.array([-side / 2, -side / 2, 0.5 * (zlo + r_max) - side / 2])
    Ng = int(gen_mesh)
    hg = side / Ng
    kf = 2 * math.pi / side
    n1 = np.fft.fftfreq(Ng, d=1.0 / Ng)
    nz = np.fft.rfftfreq(Ng, d=1.0 / Ng)
    kx = (n1 * kf)[:, None, None]
    ky = (n1 * kf)[None, :, None]
    kz = (nz * kf)[None, None, :]
    k2 = kx * kx + ky * ky + kz * kz
    kk = np.sqrt(k2)
    with np.errstate(divide="ignore"):
        pk = np.where(kk > 0, pk_amp * (np.where(kk > 0, kk, 1.0) / k0) ** pk_slope, 0.0)
    white = rng.standard_normal((Ng, Ng, Ng))
    Gk = np.fft.rfftn(white) * np.sqrt(pk / hg ** 3)
    G = np.fft.irfftn(Gk, s=(Ng, Ng, Ng))
    var = float(G.var())
    dln = np.exp(G - var / 2.0)                 # 1 + delta_LN

    # Poisson sampling inside the cap
    counts = rng.poisson(nbar * hg ** 3 * dln)
    cells = np.repeat(np.arange(Ng ** 3), counts.ravel())
    ci = np.stack(np.unravel_index(cells, (Ng, Ng, Ng)), axis=1)
    pos = g_lo[None, :] + (ci + rng.uniform(0, 1, size=ci.shape)) * hg
    rr = np.linalg.norm(pos, axis=1)
    keep = (rr >= r_min) & (rr <= r_max) & (pos[:, 2] >= rr * cos_max)
    pos, ci = pos[keep], ci[keep]

    # Kaiser displacement along the radial direction
    dm_k = Gk / bias
    with np.errstate(invalid="ignore", divide="ignore"):
        inv_k2 = np.where(k2 > 0, 1.0 / np.where(k2 > 0, k2, 1.0), 0.0)
    psi = [np.fft.irfftn(1j * kc * dm_k * inv_k2, s=(Ng, Ng, Ng)) for kc in (kx, ky, kz)]
    ps = np.stack([p[ci[:, 0], ci[:, 1], ci[:, 2]] for p in psi], axis=1)
    rhat = pos / np.linalg.norm(pos, axis=1, keepdims=True)
    pos = pos + f_growth * np.sum(ps * rhat, axis=1, keepdims=True) * rhat

    # randoms
    n_ran = int(round(ran_factor * n_gal))
    u = rng.uniform(0, 1, size=n_ran)
    rad = (r_min ** 3 + u * (r_max ** 3 - r_min ** 3)) ** (1.0 / 3.0)
    ran = _cap_directions(rng, n_ran, cos_max) * rad[:, None]

    R = _rotation_to(np.asarray(pole, dtype=np.float64))
    pos = pos @ R.T
    ran = ran @ R.T
    w = 1.0 / (1.0 + nbar * P0)
    g = np.concatenate([pos, np.full((len(pos), 1), w)], axis=1).astype(np.float32)
    r = np.concatenate([ran, np.full((n_ran, 1), w)], axis=1).astype(np.float32)

    lo = r[:, :3].min(axis=0).astype(np.float64)
    hi = r[:, :3].max(axis=0).astype(np.float64)
    lo = np.minimum(lo, g[:, :3].min(axis=0))
    hi = np.maximum(hi, g[:, :3].max(axis=0))
    centre = 0.5 * (lo + hi)
    extent = float(np.max(hi - lo))
    box_len = box_factor * extent
    return Catalog(g, r, np.full(len(g), nbar, np.float32), np.full(n_ran, nbar, np.float32),
                   centre - 0.5 * box_len, box_len,
                   {"kind": "lognormal_cap", "seed": seed, "n_gal": len(g), "n_ran": n_ran,
                    "half_angle_deg": half_angle_deg, "r_min": r_min, "r_max": r_max,
                    "nbar": nbar, "P0": P0, "f": f_growth, "b": bias, "pole": tuple(float(v) for v in pole)})
