"""Icosahedral sphere mesh (paper Sec. 3: icosahedral grids, N_C = 20 * 4**r cells).

Canonical construction (the paper leaves numbering unstated; this is the
reading both implementations follow):

* the 12 icosahedron vertices (0, +-1, +-phi), (+-1, +-phi, 0), (+-phi, 0, +-1)
  are sorted lexicographically by (x, y, z) and scaled to radius R;
* faces are the triples of mutually adjacent vertices, oriented
  counter-clockwise seen from outside, rotated so the smallest index comes
  first, then sorted;
* each refinement visits faces in order and, for face (a, b, c), edges in the
  order ab, bc, ca, creating the radially projected midpoint on first
  encounter; children are (a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca);
* edges are the sorted (low, high) vertex pairs in lexicographic order,
  oriented low -> high; local edge i of a cell is the one opposite its local
  vertex i.

Plain Python loops: obviously correct, slow, fine for r <= 7.
"""

import math

import numpy as np


class Mesh:
    """Vertices, cells, edges and their incidence for one refinement level."""

    def __init__(self, verts, cells, radius):
        self.radius = float(radius)
        self.verts = np.asarray(verts, dtype=np.float64)          # (V, 3)
        self.cells = np.asarray(cells, dtype=np.int64)            # (F, 3) ccw from outside
        edge_set = set()
        for a, b, c in self.cells:
            for p, q in ((b, c), (c, a), (a, b)):
                edge_set.add((min(p, q), max(p, q)))
        edges = sorted(edge_set)
        self.edges = np.array(edges, dtype=np.int64)              # (E, 2) low, high
        index = {e: i for i, e in enumerate(edges)}
        F = len(self.cells)
        self.cell_edges = np.zeros((F, 3), dtype=np.int64)
        # +1 when the cell's counter-clockwise traversal of the local edge runs low -> high
        self.cell_edge_aligned = np.zeros((F, 3), dtype=bool)
        for c, (v0, v1, v2) in enumerate(self.cells):
            for i, (p, q) in enumerate(((v1, v2), (v2, v0), (v0, v1))):
                self.cell_edges[c, i] = index[(min(p, q), max(p, q))]
                self.cell_edge_aligned[c, i] = p < q
        E = len(edges)
        # plus cell: the one traversing the edge low -> high; minus cell: the other
        self.edge_cells = -np.ones((E, 2), dtype=np.int64)
        self.edge_local = -np.ones((E, 2), dtype=np.int64)
        for c in range(F):
            for i in range(3):
                e = self.cell_edges[c, i]
                side = 0 if self.cell_edge_aligned[c, i] else 1
                assert self.edge_cells[e, side] < 0, "edge traversed twice in one direction"
                self.edge_cells[e, side] = c
                self.edge_local[e, side] = i
        assert (self.edge_cells >= 0).all(), "open edge: mesh is not a closed oriented surface"

    @property
    def n_cells(self):
        return len(self.cells)

    @property
    def n_edges(self):
        return len(self.edges)

    @property
    def n_verts(self):
        return len(self.verts)


def _scale_to(p, radius):
    x, y, z = p
    nrm = math.sqrt(x * x + y * y + z * z)
    s = radius / nrm
    return (x * s, y * s, z * s)


def icosahedron(radius):
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    raw = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            raw.append((0.0, s1, s2 * phi))
            raw.append((s1, s2 * phi, 0.0))
            raw.append((s1 * phi, 0.0, s2))
    raw.sort()
    faces = []
    n = len(raw)

    def d2(i, j):
        return sum((raw[i][k] - raw[j][k]) ** 2 for k in range(3))

    for i in range(n):
        for j in range(i + 1, n):
            for k in range(j + 1, n):
                if abs(d2(i, j) - 4) < 1e-9 and abs(d2(j, k) - 4) < 1e-9 and abs(d2(i, k) - 4) < 1e-9:
                    a, b, c = np.array(raw[i]), np.array(raw[j]), np.array(raw[k])
                    if np.dot(a, np.cross(b, c)) > 0:
                        faces.append((i, j, k))
                    else:
                        faces.append((i, k, j))
    rotated = []
    for f in faces:
        m = f.index(min(f))
        rotated.append(tuple(f[m:] + f[:m]))
    rotated.sort()
    assert len(rotated) == 20
    verts = [_scale_to(p, radius) for p in raw]
    return verts, rotated


def refine(verts, faces, radius):
    verts = list(verts)
    mids = {}

    def midpoint(a, b):
        key = (min(a, b), max(a, b))
        if key not in mids:
            pa, pb = verts[a], verts[b]
            m = (pa[0] + pb[0], pa[1] + pb[1], pa[2] + pb[2])
            verts.append(_scale_to(m, radius))
            mids[key] = len(verts) - 1
        return mids[key]

    out = []
    for a, b, c in faces:
        ab = midpoint(a, b)
        bc = midpoint(b, c)
        ca = midpoint(c, a)
        out.extend([(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)])
    return verts, out


def build_mesh(refinement, radius):
    verts, faces = icosahedron(radius)
    for _ in range(refinement):
        verts, faces = refine(verts, faces, radius)
    return Mesh(verts, faces, radius)


def cell_centre_distances(mesh):
    """Great-circle distances between centres of edge-adjacent cells.

    A cell centre is the radial projection of its vertex mean onto the sphere.
    """
    c = mesh.verts[mesh.cells].sum(axis=1)
    c = c / np.linalg.norm(c, axis=1, keepdims=True)
    a = c[mesh.edge_cells[:, 0]]
    b = c[mesh.edge_cells[:, 1]]
    cosang = np.clip((a * b).sum(axis=1), -1.0, 1.0)
    return mesh.radius * np.arccos(cosang)
