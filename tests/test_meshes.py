"""The CAD stand-in generators build closed, outward-oriented triangle surfaces:
every edge is shared by exactly two triangles that traverse it in opposite
directions, and the signed volume (divergence theorem) is positive and equals
the body's volume (exactly for boxes and prisms, converging for spheres)."""

import numpy as np
import pytest

from mc_inputs.meshes import (NESTED_INNER, NESTED_OUTER, assemble, box_mesh, cylinder_mesh, cylinder_rod_mesh,
                              nested_boxes_mesh, sphere_mesh)


def _closed_outward(v, t):
    edges = {}
    for a, b, c in t:
        for e in ((a, b), (b, c), (c, a)):
            edges[e] = edges.get(e, 0) + 1
    assert all(n == 1 for n in edges.values()), "an edge is traversed twice in the same direction"
    assert all((b, a) in edges for (a, b) in edges), "an edge has no opposite"
    p0, p1, p2 = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    return np.einsum("ij,ij->i", p0, np.cross(p1, p2)).sum() / 6.0


def test_box_is_closed_with_exact_volume():
    v, t = box_mesh((3.0, 2.0, 1.5), center=(1.0, -2.0, 0.5))
    assert len(t) == 12
    assert abs(_closed_outward(v, t) - 6.0 * 4.0 * 3.0) < 1e-12


@pytest.mark.parametrize("n_seg", [3, 16, 97])
def test_cylinder_is_a_closed_prism(n_seg):
    r, h = 5.0, 7.0
    v, t = cylinder_mesh(r, h, n_seg, center=(2.0, 1.0, -1.0))
    area = 0.5 * n_seg * r * r * np.sin(2 * np.pi / n_seg)  # the inscribed polygon
    assert abs(_closed_outward(v, t) - area * h) < 1e-9 * area * h


def test_sphere_volume_converges():
    errs = []
    for sub in (1, 2, 3, 4):
        v, t = sphere_mesh(10.0, sub)
        errs.append(abs(_closed_outward(v, t) / (4.0 / 3.0 * np.pi * 1000.0) - 1.0))
    assert errs[-1] < 0.01 and all(b < a for a, b in zip(errs, errs[1:])), errs


def test_assembled_phantoms():
    m = cylinder_rod_mesh(48)
    for b in range(len(m["body_material"])):
        sel = m["tri_body"] == b
        assert _closed_outward(m["vertices"].astype(np.float64), m["triangles"][sel]) > 0
    assert list(m["body_parent"]) == [-1, 0]
    n = nested_boxes_mesh()
    (lo, hi), (li, hi2) = NESTED_OUTER, NESTED_INNER
    vols = [np.prod(np.subtract(hi, lo)), np.prod(np.subtract(hi2, li))]
    for b in range(2):
        sel = n["tri_body"] == b
        assert abs(_closed_outward(n["vertices"].astype(np.float64), n["triangles"][sel]) - vols[b]) < 1e-6 * vols[b]
    with pytest.raises(Exception):
        assemble([])
