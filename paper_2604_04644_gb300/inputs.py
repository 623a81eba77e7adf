"""Seeded synthetic inputs: slab meshes and modal coefficients.

This module holds none of the operator arithmetic. It only builds mesh
topology and vertex coordinates (integers and grid coordinates) and draws
counter-based random numbers, so that the CUDA library and the CPU oracle
can be fed the same inputs.

Mesh recipe (the four-slab construction): the unit cube [0,1]^3 is divided
into nx*ny*nz cells and the cell layers along z are split into four equal
slabs.  From the bottom: each cell of slab 0 is one hexahedron, of slab 1 two
prisms (cut by the cell's y=z diagonal plane, prism axis along x), of slab 2
six pyramids (one per cell face, apex at the cell centre) and of slab 3 six
Kuhn tetrahedra around the cell's (0,0,0)-(1,1,1) diagonal.  Every element is
an affine image of its reference element; ``curved`` marks the elements to
which the smooth deformation x_i += 0.05 sin(pi x_j) sin(pi x_k) is applied.

Reference vertex order (xi coordinates) used for ``vert``:

* hex   : (-1,-1,-1) (1,-1,-1) (1,1,-1) (-1,1,-1) (-1,-1,1) (1,-1,1) (1,1,1) (-1,1,1)
* prism : (-1,-1,-1) (1,-1,-1) (1,1,-1) (-1,1,-1) (-1,-1,1) (-1,1,1)
* pyr   : (-1,-1,-1) (1,-1,-1) (1,1,-1) (-1,1,-1) (-1,-1,1)
* tet   : (-1,-1,-1) (1,-1,-1) (-1,1,-1) (-1,-1,1)

Shape ids: 0 hex, 1 prism, 2 pyramid, 3 tetrahedron.
"""
from __future__ import annotations

import itertools

import numpy as np

HEX, PRISM, PYR, TET = 0, 1, 2, 3
SHAPE_NAMES = ("hex", "prism", "pyr", "tet")
N_VERTS = (8, 6, 5, 4)
# reference vertices adjacent to vertex 0 along xi_1, xi_2, xi_3
AXIS_VERTS = ((1, 3, 4), (1, 3, 4), (1, 3, 4), (1, 2, 3))


def _det3(a, b, c):
    return float(np.dot(a, np.cross(b, c)))


def _orient(shape, X):
    """Reorder a vertex list so the affine reference map has positive volume."""
    v1, v2, v3 = AXIS_VERTS[shape]
    d = _det3(X[v1] - X[0], X[v2] - X[0], X[v3] - X[0])
    if d > 0:
        return X, [0, 1, 2, 3, 4, 5, 6, 7][: len(X)]
    if shape == TET:
        perm = [0, 2, 1, 3]
    elif shape == PYR:
        perm = [0, 3, 2, 1, 4]
    elif shape == PRISM:
        # swap the roles of xi_1 and xi_3 inside the triangle
        perm = [0, 4, 5, 3, 1, 2]
    else:
        perm = [0, 3, 2, 1, 4, 7, 6, 5]
    return X[perm], perm


def slab_mesh(nx, ny, nz, order, *, curved=True, deformation=1, slabs=(HEX, PRISM, PYR, TET),
              order_seed=None, curved_rule=None):
    """Four-slab mixed mesh of the unit cube.

    order: int (uniform P) or a (lo, hi) tuple meaning P ~ U{lo..hi} per element,
      drawn with ``order_seed``.
    curved: bool applied to every element, unless ``curved_rule == 'x_half'``
      (elements whose cell centre has x < 0.5 are affine, the others curved).
    Returns a dict with the mesh descriptor arrays (user element order).
    """
    if nz % len(slabs):
        raise ValueError("nz must be divisible by the number of slabs")
    per = nz // len(slabs)
    h = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
    gid = lambda i, j, k: (k * (ny + 1) + j) * (nx + 1) + i
    n_grid = (nx + 1) * (ny + 1) * (nz + 1)
    grid = np.zeros((n_grid, 3))
    for k in range(nz + 1):
        for j in range(ny + 1):
            for i in range(nx + 1):
                grid[gid(i, j, k)] = (i * h[0], j * h[1], k * h[2])
    centres = []
    shapes, verts, cell_centre = [], [], []

    def emit(shape, ids, coords, cc):
        coords = np.asarray(coords, dtype=np.float64)
        _, perm = _orient(shape, coords)
        ids = [ids[p] for p in perm]
        row = np.full(8, -1, dtype=np.int64)
        row[: len(ids)] = ids
        shapes.append(shape)
        verts.append(row)
        cell_centre.append(cc)

    for s, shape in enumerate(slabs):
        for k in range(s * per, (s + 1) * per):
            for j in range(ny):
                for i in range(nx):
                    c = {(dx, dy, dz): gid(i + dx, j + dy, k + dz)
                         for dx in (0, 1) for dy in (0, 1) for dz in (0, 1)}
                    cc = (np.array([i, j, k]) + 0.5) * h
                    P = lambda key: grid[c[key]]
                    if shape == HEX:
                        keys = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0),
                                (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]
                        emit(HEX, [c[q] for q in keys], [P(q) for q in keys], cc)
                    elif shape == PRISM:
                        # triangles in the (y, z) square split by its y = z diagonal
                        for tri in (((1, 0), (0, 0), (1, 1)), ((0, 1), (1, 1), (0, 0))):
                            A, B, C = tri
                            keys = [(0,) + A, (0,) + B, (1,) + B, (1,) + A, (0,) + C, (1,) + C]
                            emit(PRISM, [c[q] for q in keys], [P(q) for q in keys], cc)
                    elif shape == PYR:
                        centres.append(cc)
                        cid = n_grid + len(centres) - 1
                        faces = [
                            [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0)],
                            [(0, 0, 1), (0, 1, 1), (1, 1, 1), (1, 0, 1)],
                            [(0, 0, 0), (0, 0, 1), (1, 0, 1), (1, 0, 0)],
                            [(0, 1, 0), (1, 1, 0), (1, 1, 1), (0, 1, 1)],
                            [(0, 0, 0), (0, 1, 0), (0, 1, 1), (0, 0, 1)],
                            [(1, 0, 0), (1, 0, 1), (1, 1, 1), (1, 1, 0)],
                        ]
                        for f in faces:
                            emit(PYR, [c[q] for q in f] + [cid], [P(q) for q in f] + [cc], cc)
                    else:
                        for perm in itertools.permutations(range(3)):
                            p = [0, 0, 0]
                            path = [tuple(p)]
                            for ax in perm[:2]:
                                p[ax] = 1
                                path.append(tuple(p))
                            path.append((1, 1, 1))
                            emit(TET, [c[q] for q in path], [P(q) for q in path], cc)
    xyz = np.concatenate([grid, np.array(centres).reshape(-1, 3)], axis=0)
    n_elem = len(shapes)
    shape_arr = np.array(shapes, dtype=np.uint8)
    if isinstance(order, tuple):
        rng = np.random.default_rng(order_seed)
        P_arr = rng.integers(order[0], order[1] + 1, size=n_elem).astype(np.uint8)
    else:
        P_arr = np.full(n_elem, int(order), dtype=np.uint8)
    Q_arr = (P_arr + 2).astype(np.uint8)
    cc = np.array(cell_centre)
    if curved_rule == "x_half":
        curved_arr = (cc[:, 0] >= 0.5).astype(np.uint8)
    else:
        curved_arr = np.full(n_elem, 1 if curved else 0, dtype=np.uint8)
    return dict(
        n_elem=n_elem,
        shape=shape_arr,
        P=P_arr,
        Q=Q_arr,
        vert=np.array(verts, dtype=np.int64),
        xyz=np.ascontiguousarray(xyz, dtype=np.float64),
        n_vert=xyz.shape[0],
        curved=curved_arr,
        deformation=int(deformation),
    )


def hex_cube_mesh(n, order, *, curved=False, deformation=1):
    """n*n*n affine hexahedra filling the unit cube (one slab of hexes)."""
    return slab_mesh(n, n, n, order, curved=curved, deformation=deformation, slabs=(HEX,))


def single_element_mesh(shape, order, *, curved=False, deformation=1, scale=1.0, shift=(0.0, 0.0, 0.0),
                        cell=0):
    """One element of the given shape taken from a one-cell slab, optionally moved."""
    m = slab_mesh(1, 1, 1, order, curved=curved, deformation=deformation, slabs=(shape,))
    keep = min(cell, m["n_elem"] - 1)
    m["xyz"] = m["xyz"] * scale + np.asarray(shift)
    for key in ("shape", "P", "Q", "curved", "vert"):
        m[key] = m[key][keep:keep + 1].copy()
    m["n_elem"] = 1
    return m


def subset_mesh(mesh, elems):
    """Mesh made of the listed elements (vertex array shared, order kept)."""
    elems = np.asarray(elems, dtype=np.int64)
    out = dict(mesh)
    for key in ("shape", "P", "Q", "curved", "vert"):
        out[key] = mesh[key][elems].copy()
    out["n_elem"] = int(len(elems))
    return out


def replicated_mesh(shape, order, n_elem, *, curved=True, deformation=1):
    """n_elem elements of one shape: copies of a one-cell slab's elements on a
    cubic grid of cells inside [0,1]^3 (vertices not shared; element-local
    operators only).  Fast for large n_elem (vectorised)."""
    cell = slab_mesh(1, 1, 1, order, curved=curved, deformation=deformation, slabs=(shape,))
    per = cell["n_elem"]
    nv = N_VERTS[shape]
    n_cells = -(-n_elem // per)
    m = int(np.ceil(n_cells ** (1.0 / 3.0)))
    h = 1.0 / m
    c = np.arange(n_cells)
    offs = np.stack([c % m, (c // m) % m, c // (m * m)], axis=1) * h            # (n_cells, 3)
    tmpl = cell["xyz"][cell["vert"][:, :nv]] * h                                  # (per, nv, 3)
    X = (offs[:, None, None, :] + tmpl[None]).reshape(-1, nv, 3)[:n_elem]        # (n_elem, nv, 3)
    vert = np.full((n_elem, 8), -1, dtype=np.int64)
    vert[:, :nv] = np.arange(n_elem * nv, dtype=np.int64).reshape(n_elem, nv)
    P = np.full(n_elem, int(order), dtype=np.uint8)
    return dict(n_elem=int(n_elem), shape=np.full(n_elem, shape, dtype=np.uint8), P=P, Q=(P + 2).astype(np.uint8),
                vert=vert, xyz=np.ascontiguousarray(X.reshape(-1, 3)), n_vert=n_elem * nv,
                curved=np.full(n_elem, 1 if curved else 0, dtype=np.uint8), deformation=int(deformation))


# ---------------------------------------------------------------------------
# two-dimensional meshes (quadrilaterals and triangles)
# ---------------------------------------------------------------------------
QUAD, TRI = 4, 5


def square_mesh_2d(nx, ny, order, *, cells="checker", curved=True, deformation=1, order_seed=None,
                   curved_rule=None):
    """nx*ny cells of the unit square; a cell is one quadrilateral or two
    triangles (cut along its (1,0)-(0,1) diagonal): ``cells`` = "checker"
    (quadrilateral where i + j is even), "quad" or "tri".  Vertex order:
    quadrilateral (0,0) (1,0) (1,1) (0,1) of the cell; triangles (0,0) (1,0)
    (0,1) and (1,1) (0,1) (1,0) -- vertex 0 and its neighbours along xi_1 and
    xi_2 come first, counter-clockwise.  order / order_seed / curved /
    curved_rule as for slab_mesh (x_half: cell centre x >= 0.5 curved)."""
    gid = lambda i, j: j * (nx + 1) + i
    xs, ys = np.meshgrid(np.arange(nx + 1) / nx, np.arange(ny + 1) / ny, indexing="xy")
    xy = np.stack([xs.ravel(), ys.ravel()], axis=1)
    shapes, verts, cc = [], [], []
    for j in range(ny):
        for i in range(nx):
            c = ((i + 0.5) / nx, (j + 0.5) / ny)
            quad = cells == "quad" or (cells == "checker" and (i + j) % 2 == 0)
            if quad:
                shapes.append(QUAD)
                verts.append([gid(i, j), gid(i + 1, j), gid(i + 1, j + 1), gid(i, j + 1)])
                cc.append(c)
            else:
                for t in ([gid(i, j), gid(i + 1, j), gid(i, j + 1), -1],
                          [gid(i + 1, j + 1), gid(i, j + 1), gid(i + 1, j), -1]):
                    shapes.append(TRI)
                    verts.append(t)
                    cc.append(c)
    n_elem = len(shapes)
    if isinstance(order, tuple):
        rng = np.random.default_rng(order_seed)
        P_arr = rng.integers(order[0], order[1] + 1, size=n_elem).astype(np.uint8)
    else:
        P_arr = np.full(n_elem, int(order), dtype=np.uint8)
    cc = np.array(cc)
    if curved_rule == "x_half":
        curved_arr = (cc[:, 0] >= 0.5).astype(np.uint8)
    else:
        curved_arr = np.full(n_elem, 1 if curved else 0, dtype=np.uint8)
    return dict(n_elem=n_elem, shape=np.array(shapes, dtype=np.uint8), P=P_arr,
                vert=np.array(verts, dtype=np.int64), xy=np.ascontiguousarray(xy, dtype=np.float64),
                n_vert=int(xy.shape[0]), curved=curved_arr, deformation=int(deformation))


# ---------------------------------------------------------------------------
# counter-based random numbers (SplitMix64, Steele, Lea & Flood 2014)
# ---------------------------------------------------------------------------
_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x):
    """SplitMix64 output function applied to a uint64 array of counters."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed, elem, mode):
    """U[-1,1) value for (seed, element id, mode index); layout independent."""
    elem = np.asarray(elem, dtype=np.uint64)
    mode = np.asarray(mode, dtype=np.uint64)
    with np.errstate(over="ignore"):
        key = (np.uint64(seed) << np.uint64(44)) ^ (elem << np.uint64(12)) ^ mode
    z = splitmix64(key)
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return 2.0 * u - 1.0


def random_coefficients(seed, offsets):
    """Ragged modal coefficient vector: element e owns [offsets[e], offsets[e+1])."""
    offsets = np.asarray(offsets, dtype=np.int64)
    n_elem = len(offsets) - 1
    counts = np.diff(offsets)
    elem = np.repeat(np.arange(n_elem, dtype=np.int64), counts)
    mode = np.arange(offsets[-1], dtype=np.int64) - np.repeat(offsets[:-1], counts)
    return uniform_pm1(seed, elem, mode)


def random_phys(seed, offsets, ncomp=1):
    """Values at quadrature points, ncomp component vectors stacked (component-major)."""
    offsets = np.asarray(offsets, dtype=np.int64)
    out = [random_coefficients(seed * 7 + 3 + c, offsets) for c in range(ncomp)]
    return np.concatenate(out) if ncomp > 1 else out[0]


# ---------------------------------------------------------------------------
# conforming four-slab mesh (for C0 assembly)
# ---------------------------------------------------------------------------
def _kuhn_split(face):
    """Two triangles of a cube face given as 4 corner (ids, local xyz) in cyclic
    order, split by the diagonal joining the corners of smallest and largest
    local x+y+z (the diagonal the Kuhn tetrahedra of both adjacent cubes use)."""
    sums = [sum(c[1]) for c in face]
    lo = int(np.argmin(sums))
    hi = (lo + 2) % 4
    a, b = (lo + 1) % 4, (lo + 3) % 4
    return [(face[lo][0], face[a][0], face[hi][0]), (face[lo][0], face[b][0], face[hi][0])]


def c0_slab_mesh(n, order, *, curved=True, deformation=1, nx=None, ny=None):
    """Conforming mixed mesh of the unit cube in n*n*n cells (n divisible by 4):
    slabs of hexes, prisms, pyramids and tetrahedra along z as in slab_mesh, plus
    a transition layer (the first tet-slab layer) where each cube holds the
    pyramid on its bottom face and ten tetrahedra: the other five faces split by
    their Kuhn diagonal, each half joined to the cube centre.  Local vertex
    orders make shared faces agree for a C0 modal basis: every tetrahedron has
    its two largest global ids at local vertices 2 and 3 (vertex 3 largest), every
    prism triangle has its largest id at the collapsed local vertices (4, 5), and
    pyramid apexes (cube centres) have ids above all grid vertices.  Element
    orientation is made positive by swapping local vertices 0 and 1 (tets) or the
    two non-collapsed triangle vertices (prisms)."""
    if n % 4:
        raise ValueError("n must be divisible by 4")
    nx = n if nx is None else nx
    ny = n if ny is None else ny
    per = n // 4
    hv = np.array([1.0 / nx, 1.0 / ny, 1.0 / n])
    NX, NY, NZ = nx + 1, ny + 1, n + 1
    gid = lambda i, j, k: (k * NY + j) * NX + i
    I, J, K = np.meshgrid(np.arange(NX), np.arange(NY), np.arange(NZ), indexing="ij")
    grid = np.zeros((NX * NY * NZ, 3))
    grid[gid(I, J, K).ravel()] = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1) * hv
    shapes, verts = [], []
    centres = []

    def cells(k0, k1):
        i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(k0, k1), indexing="ij")
        return i.ravel(), j.ravel(), k.ravel()

    def corner(i, j, k, d):
        return gid(i + d[0], j + d[1], k + d[2])

    def add(shape, V):
        V = np.asarray(V, dtype=np.int64)
        row = np.full((V.shape[0], 8), -1, dtype=np.int64)
        row[:, :V.shape[1]] = V
        shapes.append(np.full(V.shape[0], shape, dtype=np.uint8))
        verts.append(row)

    # hexes
    i, j, k = cells(0, per)
    keys = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]
    add(HEX, np.stack([corner(i, j, k, d) for d in keys], axis=1))
    # prisms: triangles in the (y, z) square split by the y = z diagonal; the
    # collapsed vertex is the triangle's corner of largest id, here (y, z) = (1, 1)
    i, j, k = cells(per, 2 * per)
    for A, B in (((1, 0), (0, 0)), ((0, 1), (0, 0))):
        C = (1, 1)
        V = np.stack([corner(i, j, k, (0,) + A), corner(i, j, k, (0,) + B), corner(i, j, k, (1,) + B),
                      corner(i, j, k, (1,) + A), corner(i, j, k, (0,) + C), corner(i, j, k, (1,) + C)], axis=1)
        add(PRISM, V)
    # pyramids: 6 per cube around the centre; centres numbered after the grid
    pyr_faces = [
        [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0)], [(0, 0, 1), (0, 1, 1), (1, 1, 1), (1, 0, 1)],
        [(0, 0, 0), (0, 0, 1), (1, 0, 1), (1, 0, 0)], [(0, 1, 0), (1, 1, 0), (1, 1, 1), (0, 1, 1)],
        [(0, 0, 0), (0, 1, 0), (0, 1, 1), (0, 0, 1)], [(1, 0, 0), (1, 0, 1), (1, 1, 1), (1, 1, 0)]]
    i, j, k = cells(2 * per, 3 * per)
    c0 = NX * NY * NZ
    cid = c0 + np.arange(len(i))
    centres.append(np.stack([i + 0.5, j + 0.5, k + 0.5], axis=1) * hv)
    for f in pyr_faces:
        add(PYR, np.stack([corner(i, j, k, d) for d in f] + [cid], axis=1))
    # transition layer: bottom pyramid + 10 tets per cube
    i, j, k = cells(3 * per, 3 * per + 1)
    c0 = NX * NY * NZ + sum(len(c) for c in centres)
    cid = c0 + np.arange(len(i))
    centres.append(np.stack([i + 0.5, j + 0.5, k + 0.5], axis=1) * hv)
    add(PYR, np.stack([corner(i, j, k, d) for d in pyr_faces[0]] + [cid], axis=1))
    tets = []
    for f in pyr_faces[1:]:
        face = [(d, d) for d in f]
        for tri in _kuhn_split(face):
            tets.append(np.stack([corner(i, j, k, d) for d in tri] + [cid], axis=1))
    # Kuhn tets in the remaining layers
    i, j, k = cells(3 * per + 1, n)
    for perm in itertools.permutations(range(3)):
        p = [0, 0, 0]
        path = [tuple(p)]
        for ax in perm[:2]:
            p[ax] = 1
            path.append(tuple(p))
        path.append((1, 1, 1))
        tets.append(np.stack([corner(i, j, k, d) for d in path], axis=1))
    xyz = np.concatenate([grid] + centres, axis=0)
    T = np.concatenate(tets, axis=0)
    T = np.sort(T, axis=1)                          # ascending ids: vertex 3 largest, 2 second
    X = xyz[T]
    det = np.einsum("ij,ij->i", X[:, 1] - X[:, 0], np.cross(X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]))
    swap = det < 0
    T[swap, 0], T[swap, 1] = T[swap, 1].copy(), T[swap, 0].copy()
    add(TET, T)
    shape = np.concatenate(shapes)
    vert = np.concatenate(verts)
    # positive orientation for the other shapes: prisms swap the two
    # non-collapsed triangle vertices (0<->1, 3<->2), pyramids reverse the base
    Xv = lambda e, v: xyz[vert[e, v]]
    for s, v1, v2, v3, perm in ((PRISM, 1, 3, 4, [1, 0, 3, 2, 4, 5, 6, 7]), (PYR, 1, 3, 4, [0, 3, 2, 1, 4, 5, 6, 7]),
                                (HEX, 1, 3, 4, [0, 3, 2, 1, 4, 7, 6, 5])):
        e = np.nonzero(shape == s)[0]
        if len(e) == 0:
            continue
        d = np.einsum("ij,ij->i", Xv(e, v1) - Xv(e, 0), np.cross(Xv(e, v3) - Xv(e, 0), Xv(e, v2) - Xv(e, 0)))
        # d = (E1 . (E3 x E2)) = -det(E1, E2, E3)
        bad = e[d > 0]
        vert[bad] = vert[bad][:, perm]
    n_elem = len(shape)
    P = np.full(n_elem, int(order), dtype=np.uint8)
    return dict(n_elem=n_elem, shape=shape, P=P, Q=(P + 2).astype(np.uint8), vert=vert,
                xyz=np.ascontiguousarray(xyz), n_vert=xyz.shape[0],
                curved=np.full(n_elem, 1 if curved else 0, dtype=np.uint8), deformation=int(deformation))
