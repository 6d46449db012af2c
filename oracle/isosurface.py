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
* Rasterisation: orthographic view along +z of the square [0, L)^2 on W x W
  pixels (pixel centres ((p + 1/2) L / W)), z-buffer keeping the smallest z.
  A pixel centre P is covered when the three edge functions
  E_ab(P) = (x_b - x_a)(P_y - y_a) - (y_b - y_a)(P_x - x_a) are all >= 0 or
  all <= 0 and the triangle's doubled area E_01(p2) is not zero; its depth is
  (E_12 z_0 + E_20 z_1 + E_01 z_2) / (E_12 + E_20 + E_01).  Empty pixels hold
  +inf.  Every step is a sequence of single IEEE operations in this order, so
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
    """z-buffer depth image (width x width, [y, x]) of triangles T viewed along +z."""
    img = np.full((width, width), np.inf)
    step = extent / width
    for tri in T:
        x0, y0, z0 = tri[0]
        x1, y1, z1 = tri[1]
        x2, y2, z2 = tri[2]
        den = _edge(x0, y0, x1, y1, x2, y2)
        if den == 0.0:
            continue
        lo_x = max(int(np.floor(min(x0, x1, x2) / step - 0.5)) - 1, 0)
        hi_x = min(int(np.ceil(max(x0, x1, x2) / step - 0.5)) + 1, width - 1)
        lo_y = max(int(np.floor(min(y0, y1, y2) / step - 0.5)) - 1, 0)
        hi_y = min(int(np.ceil(max(y0, y1, y2) / step - 0.5)) + 1, width - 1)
        for py in range(lo_y, hi_y + 1):
            cy = (py + 0.5) * step
            for px in range(lo_x, hi_x + 1):
                cx = (px + 0.5) * step
                e12 = _edge(x1, y1, x2, y2, cx, cy)
                e20 = _edge(x2, y2, x0, y0, cx, cy)
                e01 = _edge(x0, y0, x1, y1, cx, cy)
                if (e12 >= 0 and e20 >= 0 and e01 >= 0) or (e12 <= 0 and e20 <= 0 and e01 <= 0):
                    z = (e12 * z0 + e20 * z1 + e01 * z2) / (e12 + e20 + e01)
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
