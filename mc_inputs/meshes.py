"""Closed triangulated surfaces (the paper's CAD objects, Sec. II-A: "CAD surface
model using triangular elements"; Sec. III: "closed triangulated surfaces").

A mesh phantom is a set of bodies, each a closed, outward-oriented triangle
surface with one material and density, and optionally a parent body it sits
inside (it replaces the parent's material there); outside every body is
vacuum.  Arrays:

  vertices       float32 [n_v][3]   (mm, volume coordinates: rotation axis = z)
  triangles      int32   [n_t][3]   (counter-clockwise seen from outside)
  tri_body       int32   [n_t]
  body_material  int32   [n_b]
  body_density   float32 [n_b]      (g/cm^3)
  body_parent    int32   [n_b]      (-1: in vacuum)

The CAD files of the paper's objects are not available; these generators
build the stand-ins (a cylinder with a rod, boxes, spheres).
"""

from __future__ import annotations

import numpy as np

from .tables import MAT_AL, MAT_WATER


def box_mesh(half, center=(0.0, 0.0, 0.0)):
    """Axis-aligned box, 12 outward triangles."""
    hx, hy, hz = half
    cx, cy, cz = center
    v = np.array([[cx + sx * hx, cy + sy * hy, cz + sz * hz]
                  for sz in (-1, 1) for sy in (-1, 1) for sx in (-1, 1)], dtype=np.float64)
    # vertex index = x + 2 y + 4 z (bits)
    quads = [(0, 2, 3, 1), (4, 5, 7, 6), (0, 1, 5, 4), (2, 6, 7, 3), (0, 4, 6, 2), (1, 3, 7, 5)]
    tris = []
    for a, b, c, d in quads:
        tris += [(a, b, c), (a, c, d)]
    return _orient_outward(v, np.array(tris, dtype=np.int64))


def cylinder_mesh(radius, height, n_seg=64, center=(0.0, 0.0, 0.0)):
    """Cylinder along z: n_seg side quads (2 triangles each) and two fan caps."""
    cx, cy, cz = center
    ang = 2.0 * np.pi * np.arange(n_seg) / n_seg
    ring = np.stack([cx + radius * np.cos(ang), cy + radius * np.sin(ang)], axis=1)
    bot = np.column_stack([ring, np.full(n_seg, cz - height / 2)])
    top = np.column_stack([ring, np.full(n_seg, cz + height / 2)])
    v = np.vstack([bot, top, [[cx, cy, cz - height / 2]], [[cx, cy, cz + height / 2]]])
    cb, ct = 2 * n_seg, 2 * n_seg + 1
    tris = []
    for i in range(n_seg):
        j = (i + 1) % n_seg
        tris += [(i, j, n_seg + j), (i, n_seg + j, n_seg + i)]  # side
        tris += [(cb, j, i), (ct, n_seg + i, n_seg + j)]        # caps
    return _orient_outward(v, np.array(tris, dtype=np.int64))


def sphere_mesh(radius, subdiv=3, center=(0.0, 0.0, 0.0)):
    """Icosphere: an icosahedron subdivided `subdiv` times, vertices pushed to the sphere."""
    t = (1.0 + 5 ** 0.5) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6),
         (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10),
         (8, 6, 7), (9, 8, 1)]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    for _ in range(subdiv):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        f = nf
    vv = np.array(verts) * radius + np.asarray(center, dtype=np.float64)
    return _orient_outward(vv, np.array(f, dtype=np.int64))


def _orient_outward(v, tris):
    """Flip triangles whose normal points toward the body's centroid (convex bodies)."""
    c = v.mean(axis=0)
    a, b, d = v[tris[:, 0]], v[tris[:, 1]], v[tris[:, 2]]
    n = np.cross(b - a, d - a)
    flip = np.einsum("ij,ij->i", n, (a + b + d) / 3.0 - c) < 0
    tris = tris.copy()
    tris[flip] = tris[flip][:, [0, 2, 1]]
    return v, tris


def assemble(bodies):
    """bodies: list of (vertices, triangles, material, density, parent index or -1) -> mesh phantom dict."""
    vs, ts, tb = [], [], []
    off = 0
    mats, dens, par = [], [], []
    for k, (v, t, m, rho, parent) in enumerate(bodies):
        vs.append(np.asarray(v, dtype=np.float64))
        ts.append(np.asarray(t, dtype=np.int64) + off)
        tb.append(np.full(len(t), k, dtype=np.int32))
        off += len(v)
        mats.append(m)
        dens.append(rho)
        par.append(parent)
    return dict(vertices=np.vstack(vs).astype(np.float32), triangles=np.vstack(ts).astype(np.int32),
                tri_body=np.concatenate(tb), body_material=np.array(mats, dtype=np.int32),
                body_density=np.array(dens, dtype=np.float32), body_parent=np.array(par, dtype=np.int32))


def cylinder_rod_mesh(n_seg=96):
    """The 64^3 cylinder phantom as surfaces: water cylinder r = 25 mm, h = 60 mm, with an aluminium rod
    r = 5 mm at x = 10 mm inside it (same height)."""
    cyl = cylinder_mesh(25.0, 60.0, n_seg)
    rod = cylinder_mesh(5.0, 60.0, max(16, n_seg // 3), center=(10.0, 0.0, 0.0))
    return assemble([(cyl[0], cyl[1], MAT_WATER, 1.0, -1), (rod[0], rod[1], MAT_AL, 2.7, 0)])


# Nested boxes whose faces lie on the planes of a 2 mm voxel grid centred on the origin: a water box with an
# aluminium box inside it that shares the water box's top face (coincident surfaces of two bodies).
NESTED_OUTER = ((-30.0, -24.0, -20.0), (30.0, 24.0, 20.0))
NESTED_INNER = ((-2.0, -10.0, -8.0), (14.0, 2.0, 20.0))
NESTED_RHO_AL = 2.69921875  # 2.7 g/cm^3 rounded to binary16 (exact in binary32)


def nested_boxes_mesh():
    def box(b):
        (a0, a1, a2), (b0, b1, b2) = b
        return box_mesh(((b0 - a0) / 2, (b1 - a1) / 2, (b2 - a2) / 2), center=((a0 + b0) / 2, (a1 + b1) / 2, (a2 + b2) / 2))

    vo, to = box(NESTED_OUTER)
    vi, ti = box(NESTED_INNER)
    return assemble([(vo, to, MAT_WATER, 1.0, -1), (vi, ti, MAT_AL, NESTED_RHO_AL, 0)])
