"""Iso-surface extraction and headless depth rasterisation (FP64).

Test infrastructure (see ``oracle/__init__``).

Fig. 3 of the paper shows iso-surfaces of the Q criterion of a 256^3 run.  The
rendering itself (a graphics API) is not reproduced; what it computes is:

* Extraction by marching tetrahedra on the cell-centre lattice: the cube with
  corners at cells (i + dx, j + dy, k + dz), dx, dy, dz in {0, 1} (values read
  with periodic wrap, coordinates unwrapped: corner b = dx + 2 dy + 4 dz at
  ((i + dx + 1/2) h, (j + dy + 1/2) h, (k + dz + 1/2) h)), is split into the
  six tetrahedra of the Freudenthal triangulation, the paths 0 -> e_a ->
  e_a + e_b -> 7 over the orders (a, b, c) of the axes:
      (0,1,3,7) (0,1,5,7) (0,2,3,7) (0,2,6,7) (0,4,5,7) (0,4,6,7).
  The split is the same in every cube, so neighbouring cubes agree on their
  shared faces and the surface is closed.  A corner is inside when
  f > iso.  A tetrahedron with one corner apart (one inside or one outside)
  gives the triangle (P(a,b), P(a,c), P(a,d)), a the lone corner and b, c, d
  the others in tetrahedron order; two inside (a, b) and two outside (c, d)
  give (P(a,c), P(a,d), P(b,d)) and (P(a,c), P(b,d), P(b,c)).  The edge point
  P is the linear zero of f - iso along the edge, always computed from the
  edge's lower corner (smaller b): p = p_lo + t (p_hi - p_lo),
  t = (iso - f_lo) / (f_hi - f_lo).  Triangles are listed cube by cube (flat
  cube index i + N (j + N k)), tetrahedra in the order above.
* Rasterisation (single precision, as rasterisers work): orthographic view
  along +z of the square [0, L)^2 on W x W pixels (pixel centres
  c = (p + 1/2) L / W in double), z-buffer keeping the smallest z.  Per
  triangle the corners relative to the first one are rounded to FP32
  (X_q = f32(x_q - x_0), Y_q likewise, X_0 = Y_0 = 0; Z_q = f32(z_q)), and
  per pixel the centre likewise (CX = f32(c_x - x_0), CY = f32(c_y - y_0)).
  With E_ab = (X_b - X_a)(CY - Y_a) - (Y_b - Y_a)(CX - X_a) in FP32, the pixel
  is covered when E_12, E_20, E_01 are all >= 0 or all <= 0 and the doubled
  area (X_1 Y_2 - Y_1 X_2, FP32) is not zero; its depth is
  ((E_12 Z_0 + E_20 Z_1) + E_01 Z_2) / ((E_12 + E_20) + E_01) in FP32.
  Empty pixels hold +inf.  Every step is one IEEE operation in this order, so
  an implementation that rounds each operation gives the same bits.

Parity pins (tests/test_oracle_isosurface.py): the zero set of cos z (two
horizontal planes: 8 N^2 triangles each, area (N h)^2 each, exact), a sphere
(area -> 4 pi R^2 at second order, every edge shared by exactly two
triangles), and the depth image of the planes (the lower plane's height on
the covered square, +inf outside).
"""
import numpy as np

TETS = [(0, 1, 3, 7), (0, 1, 5, 7), (0, 2, 3, 7), (0, 2, 6, 7), (0, 4, 5, 7), (0, 4, 6, 7)]


def corner(i, j, k, b, h):
    return ((i + (b & 1) + 0.5) * h, (j + ((b >> 1) & 1) + 0.5) * h, (k + ((b >> 2) & 1) + 0.5) * h)


def edge_point(pa, fa, pb, fb, iso, a, b):
    """Zero of f - iso on edge (a, b), computed from the lower corner."""
    if b < a:
        pa, fa, pb, fb = pb, fb, pa, fa
    t = (iso - fa) / (fb - fa)
    return tuple(pa[q] + t * (pb[q] - pa[q]) for q in range(3))


def cube_triangles(f, i, j, k, iso, h):
    """Triangles of one cube (list of 3-tuples of points), in definition order."""
    N = f.shape[0]
    val = {}
    pos = {}
    for b in range(8):
        ii, jj, kk = i + (b & 1), j + ((b >> 1) & 1), k + ((b >> 2) & 1)
        val[b] = f[kk % N, jj % N, ii % N]
        pos[b] = corner(i, j, k, b, h)
    out = []
    for tet in TETS:
        ins = [v for v in tet if val[v] > iso]
        outs = [v for v in tet if not val[v] > iso]
        P = lambda a, b: edge_point(pos[a], val[a], pos[b], val[b], iso, a, b)
        if len(ins) == 1 or len(ins) == 3:
            lone = ins[0] if len(ins) == 1 else outs[0]
            rest = [v for v in tet if v != lone]
            out.append((P(lone, rest[0]), P(lone, rest[1]), P(lone, rest[2])))
        elif len(ins) == 2:
            a, b = ins
            c, d = outs
            out.append((P(a, c), P(a, d), P(b, d)))
            out.append((P(a, c), P(b, d), P(b, c)))
    return out


def extract(f, iso, h):
    """All triangles (M, 3, 3) array in definition order, and the total area."""
    N = f.shape[0]
    # cubes with corners on both sides of iso (the others have no triangles), in flat order
    ins = f > iso
    corners = [np.roll(ins, (-((b >> 2) & 1), -((b >> 1) & 1), -(b & 1)), axis=(0, 1, 2)) for b in range(8)]
    cut = np.logical_or.reduce(corners) & ~np.logical_and.reduce(corners)
    tris = []
    for flat in np.flatnonzero(cut.reshape(-1)):
        k, rem = divmod(int(flat), N * N)
        j, i = divmod(rem, N)
        tris.extend(cube_triangles(f, i, j, k, iso, h))
    T = np.array(tris, dtype=np.float64).reshape(-1, 3, 3)
    if len(T) == 0:
        return T, 0.0
    e1 = T[:, 1] - T[:, 0]
    e2 = T[:, 2] - T[:, 0]
    area = 0.5 * np.linalg.norm(np.cross(e1, e2), axis=1)
    return T, float(np.sum(area))


def _edge(xa, ya, xb, yb, px, py):
    return (xb - xa) * (py - ya) - (yb - ya) * (px - xa)


def raster_depth(T, width, extent):
    """z-buffer depth image (width x width, [y, x], float32) of triangles T viewed along +z."""
    f32 = np.float32
    img = np.full((width, width), np.inf, dtype=np.float32)
    step = extent / width
    zero = f32(0.0)
    for tri in T:
        x0, y0, z0 = (float(v) for v in tri[0])
        X1, Y1 = f32(tri[1][0] - x0), f32(tri[1][1] - y0)
        X2, Y2 = f32(tri[2][0] - x0), f32(tri[2][1] - y0)
        Z0, Z1, Z2 = f32(tri[0][2]), f32(tri[1][2]), f32(tri[2][2])
        if X1 * Y2 - Y1 * X2 == zero:
            continue
        xs = (tri[0][0], tri[1][0], tri[2][0])
        ys = (tri[0][1], tri[1][1], tri[2][1])
        lo_x = max(int(np.floor(min(xs) / step - 0.5)) - 1, 0)
        hi_x = min(int(np.ceil(max(xs) / step - 0.5)) + 1, width - 1)
        lo_y = max(int(np.floor(min(ys) / step - 0.5)) - 1, 0)
        hi_y = min(int(np.ceil(max(ys) / step - 0.5)) + 1, width - 1)
        for py in range(lo_y, hi_y + 1):
            CY = f32((py + 0.5) * step - y0)
            for px in range(lo_x, hi_x + 1):
                CX = f32((px + 0.5) * step - x0)
                e12 = _edge(X1, Y1, X2, Y2, CX, CY)
                e20 = _edge(X2, Y2, zero, zero, CX, CY)
                e01 = _edge(zero, zero, X1, Y1, CX, CY)
                if (e12 >= 0 and e20 >= 0 and e01 >= 0) or (e12 <= 0 and e20 <= 0 and e01 <= 0):
                    z = ((e12 * Z0 + e20 * Z1) + e01 * Z2) / ((e12 + e20) + e01)
                    if z < img[py, px]:
                        img[py, px] = z
    return img


def cube_counts(f, iso):
    """Triangles per cube (N^3 array [k, j, i]): per tetrahedron 1 for one corner
    apart, 2 for two and two, summed over the six tetrahedra."""
    ins = (f > iso).astype(np.int64)
    corners = [np.roll(ins, (-((b >> 2) & 1), -((b >> 1) & 1), -(b & 1)), axis=(0, 1, 2)) for b in range(8)]
    total = np.zeros_like(ins)
    for tet in TETS:
        n = corners[tet[0]] + corners[tet[1]] + corners[tet[2]] + corners[tet[3]]
        total += np.where((n == 1) | (n == 3), 1, np.where(n == 2, 2, 0))
    return total
