"""Pins of the oracle's assembled solve: the dimension of its constraint null
space equals the number of interior C0 functions counted from the mesh
topology, and the discrete solution of a manufactured problem converges
spectrally in P to the exact solution."""
import numpy as np
import pytest

from oracle import assembly, operators as ops
from paper_2604_04644_gb300 import inputs

EDGE_LIST = {0: [(0, 1), (1, 2), (3, 2), (0, 3), (4, 5), (5, 6), (7, 6), (4, 7), (0, 4), (1, 5), (2, 6), (3, 7)],
             1: [(0, 1), (1, 2), (3, 2), (0, 3), (0, 4), (1, 4), (3, 5), (2, 5), (4, 5)],
             2: [(0, 1), (1, 2), (3, 2), (0, 3), (0, 4), (1, 4), (2, 4), (3, 4)],
             3: [(0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3)]}


def interior_c0_dim(mesh, P):
    """Topological count of C0 functions vanishing on the boundary."""
    from oracle.basis import n_modes
    faces, edges, verts = {}, {}, {}
    interior = 0
    for e in range(mesh["n_elem"]):
        s = int(mesh["shape"][e])
        g = mesh["vert"][e]
        for f in assembly.FACES[s]:
            k = tuple(sorted(int(g[v]) for v in f))
            faces[k] = faces.get(k, 0) + 1
        for a, b in EDGE_LIST[s]:
            edges[tuple(sorted((int(g[a]), int(g[b]))))] = 1
        for v in range(assembly.NV[s]):
            verts[int(g[v])] = 1
        nf3 = sum(1 for f in assembly.FACES[s] if len(f) == 3)
        nf4 = len(assembly.FACES[s]) - nf3
        interior += n_modes(s, P) - (assembly.NV[s] + len(EDGE_LIST[s]) * (P - 1) + nf4 * (P - 1) ** 2
                                     + nf3 * (P - 1) * (P - 2) // 2)
    bverts, bedges = set(), set()
    for k, c in faces.items():
        if c == 1:
            bverts.update(k)
            kk = list(k)
            for a in kk:
                for b in kk:
                    if a < b and (a, b) in edges:
                        bedges.add((a, b))
    nq = sum(1 for k, c in faces.items() if c == 2 and len(k) == 4)
    nt = sum(1 for k, c in faces.items() if c == 2 and len(k) == 3)
    return ((len(verts) - len(bverts)) + (len(edges) - len(bedges)) * (P - 1) + nq * (P - 1) ** 2
            + nt * (P - 1) * (P - 2) // 2 + interior)


@pytest.mark.parametrize("P", [1, 2, 3])
def test_null_space_dimension_matches_topology(P):
    mesh = inputs.c0_slab_mesh(8, P, curved=True, nx=1, ny=1)
    Z = assembly.c0_space(mesh)
    assert Z.shape[1] == interior_c0_dim(mesh, P)


def test_manufactured_solution_converges_spectrally():
    lam = 1.0
    u = lambda x, y, z: np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
    f = lambda x, y, z: (3 * np.pi ** 2 + lam) * u(x, y, z)
    errs = []
    for P in (2, 3, 4):
        mesh = inputs.c0_slab_mesh(8, P, curved=False, nx=1, ny=1)
        ul = assembly.solve(mesh, lam, f)
        co, po = ops.layout(mesh)
        vals = ops.apply("bwd_trans", mesh, ul)
        # exact values at the quadrature points (affine maps)
        err = 0.0
        for e in range(mesh["n_elem"]):
            s, Pe, Q = int(mesh["shape"][e]), int(mesh["P"][e]), int(mesh["Q"][e])
            ref = ops.reference(s, Pe, Q)
            X = mesh["xyz"][mesh["vert"][e][:assembly.NV[s]]]
            x = assembly.element_map(s, X, False, 0)(*ref["xi"])
            err = max(err, np.abs(vals[po[e]:po[e + 1]] - u(*x)).max())
        errs.append(err)
    assert errs[0] < 0.6 and errs[1] < errs[0] / 3 and errs[2] < errs[1] / 3, errs
