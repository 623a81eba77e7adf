"""C0 global numbering of the library, checked on the CPU with the oracle's
own basis evaluation: every global vector, gathered to elements, must give a
function that is continuous across every shared face, vanishes on the
boundary when the boundary DOFs are zero, and the number of global DOFs must
equal the entity count of the mesh (vertices + (P-1) per edge + face and
interior modes)."""
import itertools

import numpy as np
import pytest

from oracle import basis, operators as ops
from paper_2604_04644_gb300 import inputs

FACES = {0: [(0, 1, 2, 3), (4, 5, 6, 7), (0, 1, 5, 4), (1, 2, 6, 5), (3, 2, 6, 7), (3, 0, 4, 7)],
         1: [(0, 1, 4), (3, 2, 5), (0, 1, 2, 3), (0, 3, 5, 4), (1, 2, 5, 4)],
         2: [(0, 1, 2, 3), (0, 1, 4), (1, 2, 4), (2, 3, 4), (3, 0, 4)],
         3: [(0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3)]}
EDGES = {0: 12, 1: 9, 2: 8, 3: 6}


@pytest.fixture(scope="module")
def hp():
    from paper_2604_04644_gb300 import build
    build.build()
    from paper_2604_04644_gb300 import hp as _hp
    return _hp


def _faces(mesh):
    out = {}
    for e in range(mesh["n_elem"]):
        s = int(mesh["shape"][e])
        for f in FACES[s]:
            ids = tuple(sorted(int(mesh["vert"][e][v]) for v in f))
            out.setdefault(ids, []).append(e)
    return out


def _eval_at(mesh, e, x, uloc):
    """u_e at physical points x (n, 3) of an affine element, by the oracle's basis."""
    s = int(mesh["shape"][e])
    nv = inputs.N_VERTS[s]
    X = mesh["xyz"][mesh["vert"][e][:nv]]
    v = inputs.AXIS_VERTS[s]
    E = np.stack([X[v[d]] - X[0] for d in range(3)], axis=1)
    xi = 2.0 * np.linalg.solve(E, (x - X[0]).T) - 1.0
    B = basis.evaluate(s, int(mesh["P"][e]), xi[0], xi[1], xi[2])
    return B @ uloc


def _face_points(mesh, ids, rng, k=6):
    V = mesh["xyz"][list(ids)]
    w = rng.dirichlet(np.ones(len(ids)), size=k) * 0.9 + 0.1 / len(ids)
    if len(ids) == 4:
        # a quad face: convex combinations of its corners stay on the (planar) face
        pass
    return w @ V


def _entity_count(mesh, P):
    verts = set()
    edges = set()
    tri, quad = set(), set()
    interior = 0
    EDGE_LIST = {0: [(0, 1), (1, 2), (3, 2), (0, 3), (4, 5), (5, 6), (7, 6), (4, 7), (0, 4), (1, 5), (2, 6), (3, 7)],
                 1: [(0, 1), (1, 2), (3, 2), (0, 3), (0, 4), (1, 4), (3, 5), (2, 5), (4, 5)],
                 2: [(0, 1), (1, 2), (3, 2), (0, 3), (0, 4), (1, 4), (2, 4), (3, 4)],
                 3: [(0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3)]}
    for e in range(mesh["n_elem"]):
        s = int(mesh["shape"][e])
        g = mesh["vert"][e]
        verts.update(int(g[v]) for v in range(inputs.N_VERTS[s]))
        for a, b in EDGE_LIST[s]:
            edges.add(tuple(sorted((int(g[a]), int(g[b])))))
        for f in FACES[s]:
            (tri if len(f) == 3 else quad).add(tuple(sorted(int(g[v]) for v in f)))
        # interior modes: total minus boundary-entity modes of this element
        nf3 = sum(1 for f in FACES[s] if len(f) == 3)
        nf4 = len(FACES[s]) - nf3
        boundary_modes = inputs.N_VERTS[s] + EDGES[s] * (P - 1) + nf4 * (P - 1) ** 2 + nf3 * (P - 1) * (P - 2) // 2
        interior += basis.n_modes(s, P) - boundary_modes
    return len(verts) + len(edges) * (P - 1) + len(quad) * (P - 1) ** 2 + len(tri) * (P - 1) * (P - 2) // 2 + interior


@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_c0_map_gives_continuous_functions(hp, P):
    mesh = inputs.c0_slab_mesh(4, P, curved=False)
    co, _ = ops.layout(mesh)
    gid, sign, bnd, ng = hp.hp_c0_map_host(mesh, co[-1])
    assert ng == _entity_count(mesh, P)
    assert gid.min() == 0 and gid.max() == ng - 1 and len(np.unique(gid)) == ng
    assert set(np.unique(sign)) <= {-1, 1}
    for e in range(mesh["n_elem"]):          # distinct global DOFs within an element
        assert len(np.unique(gid[co[e]:co[e + 1]])) == co[e + 1] - co[e]
    rng = np.random.default_rng(P)
    g = rng.uniform(-1, 1, ng)
    uloc = sign * g[gid]
    worst = 0.0
    faces = _faces(mesh)
    shared = [(f, el) for f, el in faces.items() if len(el) == 2]
    for f, (e1, e2) in shared[:: max(1, len(shared) // 300)]:
        x = _face_points(mesh, f, rng)
        a = _eval_at(mesh, e1, x, uloc[co[e1]:co[e1 + 1]])
        b = _eval_at(mesh, e2, x, uloc[co[e2]:co[e2 + 1]])
        worst = max(worst, np.abs(a - b).max())
    assert worst < 1e-11, worst
    # zero boundary DOFs -> zero trace on every boundary face
    g0 = np.where(bnd > 0, 0.0, g)
    u0 = sign * g0[gid]
    for f, el in list(faces.items())[::7]:
        if len(el) == 1:
            e = el[0]
            x = _face_points(mesh, f, rng)
            assert np.abs(_eval_at(mesh, e, x, u0[co[e]:co[e + 1]])).max() < 1e-11
    # and every boundary DOF is nonzero somewhere on the boundary: count matches
    assert bnd.sum() > 0


def test_c0_map_rejects_mixed_orders(hp):
    mesh = inputs.c0_slab_mesh(4, 2, curved=False)
    mesh["P"] = mesh["P"].copy()
    mesh["P"][0] = 3
    mesh["Q"] = (mesh["P"] + 2).astype(np.uint8)
    co, _ = ops.layout(mesh)
    with pytest.raises(hp.HpError) as ei:
        hp.hp_c0_map_host(mesh, co[-1])
    assert ei.value.status == hp.HP_ERR_UNSUPPORTED


def test_c0_map_needs_conforming_triangle_orientation(hp):
    """A tetrahedron whose shared face does not collapse at the face's largest
    vertex id gives traces that are no signed permutation: refused (from P = 4 on;
    at P = 3 the only triangle face mode is the symmetric cubic bubble)."""
    mesh = inputs.c0_slab_mesh(4, 4, curved=False)
    tets = np.nonzero(mesh["shape"] == 3)[0]
    v = mesh["vert"].copy()
    e = tets[0]
    v[e, [1, 2]] = v[e, [2, 1]]            # moves the collapse vertex of face (0,1,2)
    v[e, [0, 3]] = v[e, [3, 0]]            # keep the orientation positive
    mesh["vert"] = v
    co, _ = ops.layout(mesh)
    with pytest.raises(hp.HpError) as ei:
        hp.hp_c0_map_host(mesh, co[-1])
    assert ei.value.status == hp.HP_ERR_UNSUPPORTED
