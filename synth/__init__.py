"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only makes inputs: triangle meshes (vertices + faces), sun
directions and right-hand-side columns.  It holds none of the method's
arithmetic (no geometry, visibility, view factors, trees or solves), so the
oracle and the CUDA library can both consume its output without sharing code.

The paper measures on a LOLA DEM of de Gerlache crater, a 67P shape model and
Triangle-meshed spherical caps (Sections 6-8); none of those data sets are
available, so the seeded surfaces below stand in for them with the same kind
of geometry: a bowl-shaped crater, rough fBm terrain with an embedded crater,
and a closed irregular body.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "cap_bowl_mesh",
    "fbm_dem_mesh",
    "dem_to_mesh",
    "fbm_heights",
    "gaussian_sphere_mesh",
    "sun_directions",
    "uniform_columns",
    "batch_mesh_specs",
    "tiny_meshes",
]


def _orient_ccw_from_above(pts2d: np.ndarray, tris: np.ndarray) -> np.ndarray:
    a, b, c = pts2d[tris[:, 0]], pts2d[tris[:, 1]], pts2d[tris[:, 2]]
    cross = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    out = tris.copy()
    flip = cross < 0
    out[flip, 1], out[flip, 2] = tris[flip, 2], tris[flip, 1]
    return out


def cap_bowl_mesh(n_rim: int = 60, n_interior: int = 570, seed: int = 0,
                  diameter: float = 1.0, depth_ratio: float = 0.2):
    """Spherical-cap crater bowl (no surrounding plain).

    Unit diameter and depth/diameter 0.2 by default, rim at z = 0, the bowl
    below it.  ``n_rim`` equally spaced rim points plus about ``n_interior``
    jittered-hexagonal interior points, triangulated by a 2-D Delaunay
    triangulation (scipy/Qhull) and oriented counter-clockwise seen from
    above, so normals point up/into the bowl.  Returns (verts[nv,3] f64,
    faces[nf,3] i32).
    """
    from scipy.spatial import Delaunay

    rng = np.random.default_rng(seed)
    a = 0.5 * diameter
    d = depth_ratio * diameter
    rs = (a * a + d * d) / (2.0 * d)
    # hexagonal lattice spacing giving ~n_interior points inside r < a - s/2
    s = math.sqrt(math.pi * a * a * 2.0 / (math.sqrt(3.0) * n_interior))
    for _ in range(20):
        s = math.sqrt(math.pi * (a - 0.5 * s) ** 2 * 2.0 / (math.sqrt(3.0) * n_interior))
    pts = []
    ny = int(math.ceil(2 * a / (s * math.sqrt(3) / 2))) + 2
    nx = int(math.ceil(2 * a / s)) + 2
    for iy in range(-ny, ny + 1):
        y = iy * s * math.sqrt(3) / 2
        off = 0.5 * s if (iy % 2) else 0.0
        for ix in range(-nx, nx + 1):
            x = ix * s + off
            pts.append((x, y))
    pts = np.asarray(pts)
    pts = pts + rng.uniform(-0.2 * s, 0.2 * s, size=pts.shape)
    r = np.hypot(pts[:, 0], pts[:, 1])
    pts = pts[r < a - 0.5 * s]
    th = 2 * math.pi * np.arange(n_rim) / n_rim
    rim = np.stack([a * np.cos(th), a * np.sin(th)], axis=1)
    p2 = np.concatenate([rim, pts], axis=0)
    tri = Delaunay(p2).simplices.astype(np.int32)
    tri = _orient_ccw_from_above(p2, tri)
    rr = np.minimum(np.hypot(p2[:, 0], p2[:, 1]), a)
    z = (rs - d) - np.sqrt(rs * rs - rr * rr)
    z[:n_rim] = 0.0
    verts = np.concatenate([p2, z[:, None]], axis=1)
    return verts.astype(np.float64), tri


def fbm_heights(n: int, spacing: float, hurst: float, seed: int,
                rms_slope_deg: float = 15.0) -> np.ndarray:
    """n x n fractional-Brownian heights by FFT spectral synthesis.

    Amplitude |k|^-(H+1), uniform random phases from default_rng(seed), real
    part, mean removed, scaled so the RMS gradient magnitude (central
    differences) equals tan(rms_slope_deg)."""
    rng = np.random.default_rng(seed)
    kx = np.fft.fftfreq(n)
    ky = np.fft.fftfreq(n)
    kk = np.hypot(kx[:, None], ky[None, :])
    amp = np.zeros_like(kk)
    nz = kk > 0
    amp[nz] = kk[nz] ** (-(hurst + 1.0))
    phase = rng.uniform(0.0, 2.0 * np.pi, size=kk.shape)
    z = np.real(np.fft.ifft2(amp * np.exp(1j * phase)))
    z -= z.mean()
    gy, gx = np.gradient(z, spacing)
    rms = math.sqrt(float(np.mean(gx * gx + gy * gy)))
    z *= math.tan(math.radians(rms_slope_deg)) / rms
    return z


def dem_to_mesh(z: np.ndarray, spacing: float):
    """Triangulate an n x n height grid: every cell split on its
    (i,j)-(i+1,j+1) diagonal, counter-clockwise from above; 2(n-1)^2 faces."""
    n0, n1 = z.shape
    ii, jj = np.meshgrid(np.arange(n0), np.arange(n1), indexing="ij")
    verts = np.stack([jj.ravel() * spacing, ii.ravel() * spacing, z.ravel()], axis=1)
    idx = np.arange(n0 * n1).reshape(n0, n1)
    v00 = idx[:-1, :-1].ravel()
    v01 = idx[:-1, 1:].ravel()
    v10 = idx[1:, :-1].ravel()
    v11 = idx[1:, 1:].ravel()
    # x runs along columns (j), y along rows (i): (v00, v01, v11) and (v00, v11, v10) are CCW
    t1 = np.stack([v00, v01, v11], axis=1)
    t2 = np.stack([v00, v11, v10], axis=1)
    faces = np.empty((2 * t1.shape[0], 3), dtype=np.int32)
    faces[0::2] = t1
    faces[1::2] = t2
    return verts.astype(np.float64), faces


def _add_crater(z: np.ndarray, spacing: float, diameter: float, depth_ratio: float):
    n0, n1 = z.shape
    cx = 0.5 * (n1 - 1) * spacing
    cy = 0.5 * (n0 - 1) * spacing
    ii, jj = np.meshgrid(np.arange(n0), np.arange(n1), indexing="ij")
    r = np.hypot(jj * spacing - cx, ii * spacing - cy)
    a = 0.5 * diameter
    d = depth_ratio * diameter
    rs = (a * a + d * d) / (2.0 * d)
    cap = np.where(r < a, (rs - d) - np.sqrt(np.maximum(rs * rs - r * r, 0.0)), 0.0)
    return z + np.minimum(0.0, cap)


def fbm_dem_mesh(n: int = 200, spacing: float = 10.0, hurst: float = 0.8, seed: int = 1,
                 rms_slope_deg: float = 15.0, crater_diameter: float | None = 1000.0,
                 crater_depth_ratio: float = 0.2):
    """Rough fBm terrain, optionally with a spherical-cap crater at the centre.

    Default: 200 x 200 nodes at 10 m, Hurst 0.8, RMS slope 15 deg, seed 1, a
    1 km crater of depth/diameter 0.2 -> 79,202 triangles."""
    z = fbm_heights(n, spacing, hurst, seed, rms_slope_deg)
    if crater_diameter:
        z = _add_crater(z, spacing, crater_diameter, crater_depth_ratio)
    return dem_to_mesh(z, spacing)


def _icosphere(level: int):
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
         (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
         (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
         (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.asarray(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    faces = list(f)
    for _ in range(level):
        cache = {}
        nf = []

        def mid(i, j):
            key = (min(i, j), max(i, j))
            if key not in cache:
                m = verts[i] + verts[j]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        for (a, b, c) in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    return np.asarray(verts), np.asarray(faces, dtype=np.int32)


def gaussian_sphere_mesh(level: int = 6, sigma: float = 0.1, max_degree: int = 10,
                         seed: int = 4, radius: float = 1000.0):
    """Gaussian random sphere: an icosphere (20*4^level faces, outward
    normals) whose log-radius is a seeded real spherical-harmonic-like series
    of degree <= max_degree (products of Legendre functions and cos/sin of
    longitude with Gaussian coefficients), scaled to standard deviation
    ``sigma``."""
    from scipy.special import lpmv

    rng = np.random.default_rng(seed)
    u, faces = _icosphere(level)
    ct = u[:, 2]
    ph = np.arctan2(u[:, 1], u[:, 0])
    s = np.zeros(u.shape[0])
    for l in range(1, max_degree + 1):
        for m in range(0, l + 1):
            p = lpmv(m, l, ct)
            p = p / (np.max(np.abs(p)) + 1e-300)
            a, b = rng.standard_normal(2)
            s += (a * np.cos(m * ph) + (b * np.sin(m * ph) if m else 0.0)) * p / (1.0 + l)
    s = s / (np.std(s) + 1e-300) * sigma
    verts = u * (radius * np.exp(s))[:, None]
    return verts, faces


def sun_directions(n: int, elevation_deg: float, azimuth0_deg: float = 0.0):
    """n unit vectors at fixed elevation, azimuth sweeping 2*pi*k/n."""
    e = math.radians(elevation_deg)
    az = math.radians(azimuth0_deg) + 2.0 * np.pi * np.arange(n) / n
    return np.stack([math.cos(e) * np.cos(az), math.cos(e) * np.sin(az),
                     np.full(n, math.sin(e))], axis=1)


def uniform_columns(n: int, r: int, seed: int = 11) -> np.ndarray:
    """n x r column-major-friendly block of U[0,1) values (float64)."""
    return np.random.default_rng(seed).uniform(0.0, 1.0, size=(n, r))


def batch_mesh_specs(count: int = 32, seed0: int = 100):
    """The batching workload's meshes: sides round(51 + 149 k/(count-1)), 10 m
    spacing, seeds seed0+k, a crater of half the domain width on even seeds."""
    specs = []
    for k in range(count):
        n = int(round(51 + 149 * k / max(count - 1, 1)))
        seed = seed0 + k
        crater = 0.5 * (n - 1) * 10.0 if seed % 2 == 0 else None
        specs.append(dict(n=n, spacing=10.0, hurst=0.8, seed=seed, crater_diameter=crater))
    return specs


def tiny_meshes():
    """Hand-made tiny meshes for brute-force checks (name -> (verts, faces))."""
    out = {}
    # two facing unit right triangles 1 apart (z=0 facing up, z=1 facing down)
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 0, 1], [0, 1, 1]], dtype=np.float64)
    f = np.array([[0, 1, 2], [3, 5, 4]], dtype=np.int32)
    out["facing_pair"] = (v, f)
    # same pair plus an occluding wall triangle between them
    v2 = np.concatenate([v, np.array([[-1, -1, 0.5], [3, -1, 0.5], [-1, 3, 0.5]])], axis=0)
    f2 = np.concatenate([f, np.array([[6, 7, 8]], dtype=np.int32)], axis=0)
    out["pair_with_wall"] = (v2, f2)
    # an open box (floor + 4 walls, 2 triangles each), normals inward
    bv = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
                   [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]], dtype=np.float64)
    quads = [(0, 1, 2, 3), (0, 4, 5, 1), (1, 5, 6, 2), (2, 6, 7, 3), (3, 7, 4, 0)]
    tris = []
    for (a, b, c, d) in quads:
        tris += [(a, b, c), (a, c, d)]
    out["open_box"] = (bv, np.asarray(tris, dtype=np.int32))
    return out
