"""Pins for the oracle's iso-surface extraction and depth rasterisation
(oracle/isosurface.py; the paper's Fig. 3 shows Q iso-surfaces).

* The zero set of cos z is two horizontal planes: each crossed cube holds 8
  triangles (2 single-corner tetrahedra of each crossing type, 2 quads), so
  the count is 2 * 8 N^2 and the area 2 (N h)^2 = 2 (2 pi)^2, exactly.
* A sphere of radius R: every edge of the surface is shared by exactly two
  triangles (closed), and the area converges to 4 pi R^2 at second order.
* The depth image of the planes along +z is the lower plane's height (the
  linear zero of cos between its two cell rows, to single precision) on the
  covered square and +inf elsewhere; the sphere's image approaches
  c - sqrt(R^2 - r^2).
"""
import math
from collections import Counter

import numpy as np

from oracle import isosurface as iso


def centres(N):
    h = 2 * math.pi / N
    c = (np.arange(N) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    return h, x, y, z


def test_planes_count_and_area_exact():
    for N in (8, 12):
        h, x, y, z = centres(N)
        T, area = iso.extract(np.cos(z), 0.0, h)
        assert len(T) == 2 * 8 * N * N
        assert abs(area - 2 * (N * h) ** 2) < 1e-12 * area
        # every vertex of the lower sheet sits at the linear zero of cos between its rows
        k0 = int(np.floor((math.pi / 2) / h - 0.5))
        zl, zh = (k0 + 0.5) * h, (k0 + 1.5) * h
        zs = zl + (0.0 - math.cos(zl)) / (math.cos(zh) - math.cos(zl)) * (zh - zl)
        low = T[:, :, 2][T[:, :, 2] < math.pi]
        assert np.max(np.abs(low - zs)) < 1e-14


def _sphere(N, R=1.5):
    h, x, y, z = centres(N)
    c = math.pi
    return iso.extract(R * R - ((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2), 0.0, h), h


def test_sphere_closed_and_second_order_area():
    (T, area), h = _sphere(16)
    edges = Counter()
    for tri in T:
        v = [tuple(p) for p in tri]
        for a, b in ((0, 1), (1, 2), (2, 0)):
            edges[tuple(sorted((v[a], v[b])))] += 1
    assert set(edges.values()) == {2}
    exact = 4 * math.pi * 1.5 ** 2
    (T2, area2), _ = _sphere(32)
    e1, e2 = abs(area - exact), abs(area2 - exact)
    assert e1 < 0.05 * exact
    assert 3.0 < e1 / e2 < 5.0, (e1, e2)


def test_depth_image_of_planes_and_sphere():
    N = 8
    h, x, y, z = centres(N)
    T, _ = iso.extract(np.cos(z), 0.0, h)
    W, L = 2 * N, (N + 1) * h
    img = iso.raster_depth(T, W, L)
    k0 = int(np.floor((math.pi / 2) / h - 0.5))
    zl, zh = (k0 + 0.5) * h, (k0 + 1.5) * h
    zs = zl + (0.0 - math.cos(zl)) / (math.cos(zh) - math.cos(zl)) * (zh - zl)
    pc = (np.arange(W) + 0.5) * L / W
    inside = (pc >= 0.5 * h) & (pc <= (N + 0.5) * h)
    for py in range(W):
        for px in range(W):
            if inside[px] and inside[py]:
                assert abs(img[py, px] - zs) < 1e-6 * zs  # single-precision depth
            elif not (inside[px] or inside[py]):
                assert img[py, px] == np.inf
    (Ts, _), hs = _sphere(16)
    W, L = 32, 17 * hs
    img = iso.raster_depth(Ts, W, L)
    pc = (np.arange(W) + 0.5) * L / W
    X, Y = np.meshgrid(pc, pc)
    r2 = (X - math.pi) ** 2 + (Y - math.pi) ** 2
    core = r2 < (1.5 - 2 * hs) ** 2
    exact = math.pi - np.sqrt(1.5 ** 2 - r2[core])
    assert np.max(np.abs(img[core] - exact)) < 0.05
    assert np.all(np.isinf(img[r2 > (1.5 + 2 * hs) ** 2]))


def test_cube_counts_agree_with_the_extraction():
    """The vectorised per-cube count equals the triangles cube_triangles emits."""
    from paper_1404_0959_gb300.inputs import smooth_field
    N = 10
    h = 2 * math.pi / N
    f = smooth_field(N, 4, 1.0)
    counts = iso.cube_counts(f, 0.1)
    T, _ = iso.extract(f, 0.1, h)
    assert counts.sum() == len(T)
    for flat in (0, 17, 345, 999):
        k, rem = divmod(flat, N * N)
        j, i = divmod(rem, N)
        assert counts[k, j, i] == len(iso.cube_triangles(f, i, j, k, 0.1, h))
