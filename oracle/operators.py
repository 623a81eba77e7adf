"""Element-local operators by their plain definitions.

Paper Sec. 2.1: the discrete elemental Helmholtz operator
  H[m][n] = sum_l w_l |J_l| [ lambda phi_n phi_m + (J_l^-T grad phi_n).(J_l^-T grad phi_m) ],
its split H = lambda M + L, and Eq. (mass) M = B^T W B with B[l][m] = phi_m(xi_l)
and W = diag(w_l |J_l|).  Everything is evaluated at the tensor quadrature
points of the collapsed coordinates (Sec. 2.3), with phi and grad_xi phi in
closed form / complex step (see basis.py) and J from geometry.py.  Sums over
modes and points are dense matrix products (numpy matmul/einsum): no sum
factorisation, no collocation.

Building blocks (the paper's BwdTrans, IProductWRTBase, PhysDeriv and
IProductWRTDerivBase, Sec. 3.3 algorithms for the two Helmholtz forms):
  bwd_trans            u_l = sum_m B[l][m] uhat_m
  iproduct_wrt_base    out_m = sum_l phi_m(l) w_l |J_l| f_l
  phys_deriv           (du/dx_i)_l of the tensor Lagrange interpolant (in eta) of u_l
  iproduct_wrt_deriv   out_m = sum_i sum_l (d phi_m / d x_i)(l) w_l |J_l| f_i(l)

``helmholtz_collocated`` evaluates Eq. (helm1) -- B^T { sum D^T Lambda W Lambda D
+ lambda W } B with Lagrange differentiation at the points -- and exists only
to pin the paper's claim that the collocated form equals the plain one.

Point order inside an element: (i, j, k) over (eta_1, eta_2, eta_3) with k
fastest.  Physical-space vectors: Q^3 values per element, elements in user
order; vector fields are component-major (3 whole vectors).
"""
from functools import lru_cache

import numpy as np

from . import basis, quadrature
from .basis import complex_step_gradient
from .geometry import AXIS_VERTS, deform


@lru_cache(maxsize=None)
def reference(shape, P, Q, reduced=0):
    """Reference-element data at the quadrature points of (shape, P, Q);
    reduced = 1: Q - 1 points in the collapsed directions."""
    rule = quadrature.shape_rule(shape, Q, reduced)
    (x1, w1), (x2, w2), (x3, w3) = rule
    e1, e2, e3 = np.meshgrid(x1, x2, x3, indexing="ij")
    eta = np.stack([e1.ravel(), e2.ravel(), e3.ravel()])
    W = np.einsum("i,j,k->ijk", w1, w2, w3).ravel()
    xi = np.stack(basis.xi_from_eta(shape, *eta))
    ml = basis.modes(shape, P)
    B = basis.evaluate(shape, P, *xi, mode_list=ml)
    Dxi = complex_step_gradient(lambda a, b, c: basis.evaluate(shape, P, a, b, c, mode_list=ml), xi)
    # T[l, d, a] = d eta_d / d xi_a (complex step on the collapse map)
    T = np.stack(complex_step_gradient(lambda a, b, c: np.stack(basis.eta_from_xi(shape, a, b, c)), xi),
                 axis=-1).transpose(1, 0, 2)
    D1 = [lagrange_derivative_matrix(x) for x in (x1, x2, x3)]
    return dict(eta=eta, xi=xi, W=W, B=B, Dxi=Dxi, T=T, nodes=(x1, x2, x3), D1=D1,
                NP=B.shape[1], NQ=B.shape[0], Q=Q, dims=(len(x1), len(x2), len(x3)))


def lagrange_derivative_matrix(x):
    """D[i][j] = h_j'(x_i) for the Lagrange basis on nodes x: D = V' V^{-1},
    V[i][k] = P_k(x_i) (Legendre), V' by complex step."""
    from .jacobi import jacobi
    n = len(x)
    V = np.stack([jacobi(k, 0.0, 0.0, x) for k in range(n)], axis=1)
    h = 1e-30
    Vd = np.stack([np.imag(jacobi(k, 0.0, 0.0, x + 1j * h)) / h for k in range(n)], axis=1)
    return Vd @ np.linalg.inv(V)


# ---------------------------------------------------------------------------
# geometry over a block of elements of one shape
# ---------------------------------------------------------------------------
def block_jacobian(shape, X, curved, kind, xi):
    """J[e, l, i, d] = d x_i / d xi_d for vertex arrays X (Ne, nv, 3)."""
    v = AXIS_VERTS[shape]
    X0 = X[:, 0, :]
    E = np.stack([X[:, v[d], :] - X0 for d in range(3)], axis=-1)   # (Ne, 3 (i), 3 (d))

    def chi(a, b, c):
        t = [(a + 1.0) / 2.0, (b + 1.0) / 2.0, (c + 1.0) / 2.0]
        y = [X0[:, i:i + 1] + E[:, i, 0:1] * t[0][None, :] + E[:, i, 1:2] * t[1][None, :]
             + E[:, i, 2:3] * t[2][None, :] for i in range(3)]
        y = np.stack(y)                                   # (3, Ne, NQ)
        if curved:
            y = np.stack(deform(y[0], y[1], y[2], kind))
        return y
    g = complex_step_gradient(chi, xi)                    # d: (3, Ne, NQ)
    return np.stack(g, axis=-1).transpose(1, 2, 0, 3)


def block_points(shape, X, curved, kind, xi):
    """x[i, e, l] = chi^e(xi_l) for vertex arrays X (Ne, nv, 3)."""
    v = AXIS_VERTS[shape]
    X0 = X[:, 0, :]
    E = np.stack([X[:, v[d], :] - X0 for d in range(3)], axis=-1)
    t = [(xi[d] + 1.0) / 2.0 for d in range(3)]
    y = np.stack([X0[:, i:i + 1] + E[:, i, 0:1] * t[0][None, :] + E[:, i, 1:2] * t[1][None, :]
                  + E[:, i, 2:3] * t[2][None, :] for i in range(3)])
    if curved:
        y = np.stack(deform(y[0], y[1], y[2], kind))
    return y


def projection_operator(shape, P, Q):
    """Pi (NQ, NQ): point values -> values at the same points of their L2
    projection onto the element's expansion on the reference element,
    Pi = B (B^T W B)^{-1} B^T W, taken through the Householder QR
    W^{1/2} B = Qo R as Pi = W^{-1/2} Qo Qo^T W^{1/2}: the orthonormal Qo keeps
    it well conditioned, where the normal equations of the modal basis (or
    R^{-1}) lose many digits at high order."""
    ref = reference(shape, P, Q)
    B, W = ref["B"], ref["W"]
    sw = np.sqrt(W)
    Qo, _ = np.linalg.qr(sw[:, None] * B)
    return (Qo / sw[:, None]) @ (Qo.T * sw[None, :])


def isoparametric_jacobian(shape, P, Q, X, curved, kind):
    """J[e, l, i, d] = d x_i / d xi_d of the iso-parametric map at the points:
    each coordinate of the element map (its values at the points) projected
    onto the element's own degree-P expansion (the paper's benchmarks use
    curved elements whose geometry has the degree of the solution, Sec. 4; no
    construction is given; reading: the L2 projection on the reference
    element with the element's quadrature, Pi of projection_operator), then
    differentiated at the points.  The projection is a polynomial of degree
    <= P < Q in each collapsed coordinate eta_d, so the Lagrange collocation
    derivative along each eta line is exact; d x / d xi = (d x / d eta)(d eta / d xi)."""
    ref = reference(shape, P, Q)
    x = block_points(shape, X, curved, kind, ref["xi"])             # (3, Ne, NQ)
    xp = np.einsum("cel,ml->cem", x, projection_operator(shape, P, Q))
    U = xp.reshape(3, -1, Q, Q, Q)
    D1, D2, D3 = ref["D1"]
    v = np.stack([np.einsum("am,cemjk->ceajk", D1, U), np.einsum("bm,ceimk->ceibk", D2, U),
                  np.einsum("km,ceijm->ceijk", D3, U)])               # (d, c, e, Q, Q, Q)
    Jeta = v.reshape(3, 3, X.shape[0], -1).transpose(2, 3, 1, 0)     # [e, l, c, d] = d x_c / d eta_d
    return np.einsum("elcd,lda->elca", Jeta, ref["T"])


def block_metrics(shape, P, Q, X, curved, kind, geometry=0, reduced=0):
    """J, det J, J^{-1} and w|J| at the points; geometry 1 takes J from the
    iso-parametric map of curved elements (affine maps are in the span of
    every expansion, so their iso-parametric map is the map itself)."""
    ref = reference(shape, P, Q, reduced)
    if geometry == 1 and curved and reduced:
        raise ValueError("the iso-parametric geometry is defined on the full rule")
    if geometry == 1 and curved:
        J = isoparametric_jacobian(shape, P, Q, X, curved, kind)
    else:
        J = block_jacobian(shape, X, curved, kind, ref["xi"])
    detJ = np.linalg.det(J)
    Jinv = np.linalg.inv(J)                               # [e, l, d, i] = d xi_d / d x_i
    wJ = ref["W"][None, :] * detJ
    return dict(J=J, detJ=detJ, Jinv=Jinv, wJ=wJ)


# ---------------------------------------------------------------------------
# block operators (uh: (Ne, NP), phys: (Ne, NQ))
# ---------------------------------------------------------------------------
def _grad_x(ref, g, uh):
    """gradient in x at the points of u = sum uh_m phi_m: (3 (i), Ne, NQ)."""
    gxi = np.stack([uh @ ref["Dxi"][d].T for d in range(3)])           # (d, Ne, NQ)
    return np.einsum("eldi,del->iel", g["Jinv"], gxi)


def _iprod_grad(ref, g, f):
    """sum_i (d phi_m / d x_i, f_i) with f (3 (i), Ne, NQ)."""
    t = np.einsum("eldi,el,iel->del", g["Jinv"], g["wJ"], f)
    return sum(t[d] @ ref["Dxi"][d] for d in range(3))


def apply_block(op, shape, P, Q, X, curved, kind, data, lam=1.0, geometry=0, adv=None, reduced=0):
    ref = reference(shape, P, Q, reduced)
    g = block_metrics(shape, P, Q, X, curved, kind, geometry, reduced)
    B = ref["B"]
    if op == "adr":
        return (lam * ((g["wJ"] * (data @ B.T)) @ B) + _iprod_grad(ref, g, _grad_x(ref, g, data))
                + advection_block(ref, g, data, adv))
    if op == "bwd_trans":
        return data @ B.T
    if op == "iproduct_wrt_base":
        return (g["wJ"] * data) @ B
    if op == "mass":
        return (g["wJ"] * (data @ B.T)) @ B
    if op == "laplacian":
        return _iprod_grad(ref, g, _grad_x(ref, g, data))
    if op == "helmholtz":
        return lam * ((g["wJ"] * (data @ B.T)) @ B) + _iprod_grad(ref, g, _grad_x(ref, g, data))
    if op == "phys_deriv":
        return phys_deriv_block(ref, g, data)
    if op == "iproduct_wrt_deriv":
        return _iprod_grad(ref, g, data)
    if op == "helmholtz_collocated":
        return helmholtz_collocated_block(ref, g, data, lam)
    raise ValueError(op)


def advection_block(ref, g, uh, adv):
    """The advection part of the linear advection-diffusion-reaction operator
    (Sec. 2.2: the B^T {pointwise} B decomposition applies to any operator
    tested against the basis or its derivatives, the paper names this one):
    out_m = sum_l w_l |J_l| phi_m(l) (a . grad_x u)(l), a constant velocity."""
    a = np.zeros(3) if adv is None else np.asarray(adv, dtype=np.float64)
    gx = _grad_x(ref, g, uh)                                           # (3, Ne, NQ)
    return (g["wJ"] * np.einsum("i,iel->el", a, gx)) @ ref["B"]


def element_advection_matrices(shape, P, Q, X, curved, kind, adv, geometry=0):
    """Explicit C[e][m][n] = sum_l w|J| phi_m (a . grad_x phi_n) of each element."""
    ref = reference(shape, P, Q)
    g = block_metrics(shape, P, Q, X, curved, kind, geometry)
    Gx = np.einsum("eldi,dlm->eilm", g["Jinv"], np.stack(ref["Dxi"]))    # d phi_m / d x_i at l
    return np.einsum("lm,el,i,eiln->emn", ref["B"], g["wJ"], np.asarray(adv, dtype=np.float64), Gx)


def _eta_derivs(ref, u):
    """d u / d eta_d of the tensor Lagrange interpolant: (3, Ne, NQ)."""
    U = u.reshape(-1, *ref["dims"])
    D1, D2, D3 = ref["D1"]
    v1 = np.einsum("im,emjk->eijk", D1, U)
    v2 = np.einsum("jm,eimk->eijk", D2, U)
    v3 = np.einsum("km,eijm->eijk", D3, U)
    return np.stack([v.reshape(u.shape) for v in (v1, v2, v3)])


def _deta_dx(ref, g):
    """[e, l, d, i] = d eta_d / d x_i = sum_a (d eta_d / d xi_a)(d xi_a / d x_i)."""
    return np.einsum("lda,elai->eldi", ref["T"], g["Jinv"])


def phys_deriv_block(ref, g, u):
    v = _eta_derivs(ref, u)
    return np.einsum("eldi,del->iel", _deta_dx(ref, g), v)


def helmholtz_collocated_block(ref, g, uh, lam):
    """Eq. (helm1): B^T { sum_i [sum_d D_d^T Lam_di] W [sum_d' Lam_d'i D_d'] + lam W } B."""
    u = uh @ ref["B"].T
    v = _eta_derivs(ref, u)
    Gx = _deta_dx(ref, g)
    G = np.einsum("el,eldi,elki->eldk", g["wJ"], Gx, Gx)        # (Ne, NQ, 3, 3)
    # w_d = sum_d' G_dd' v_d'
    w = np.stack([sum(G[:, :, d, e] * v[e] for e in range(3)) for d in range(3)])
    D1, D2, D3 = ref["D1"]
    W1, W2, W3 = (x.reshape(-1, *ref["dims"]) for x in w)
    up = (np.einsum("mi,emjk->eijk", D1, W1) + np.einsum("mj,eimk->eijk", D2, W2)
          + np.einsum("mk,eijm->eijk", D3, W3)).reshape(u.shape)
    up = up + lam * g["wJ"] * u
    return up @ ref["B"]


def element_matrices(shape, P, Q, X, curved, kind, geometry=0, reduced=0):
    """Explicit (M, L) of each element of the block: (Ne, NP, NP) each."""
    ref = reference(shape, P, Q, reduced)
    g = block_metrics(shape, P, Q, X, curved, kind, geometry, reduced)
    B = ref["B"]
    M = np.einsum("lm,el,ln->emn", B, g["wJ"], B)
    Gx = np.einsum("eldi,dlm->eilm", g["Jinv"], np.stack(ref["Dxi"]))    # d phi_m / d x_i at l
    L = np.einsum("eilm,el,eiln->emn", Gx, g["wJ"], Gx)
    return M, L


def geometric_factors_block(shape, P, Q, X, curved, kind, geometry=0, reduced=0):
    """Per point: G_dd' = w|J| sum_i (d eta_d/dx_i)(d eta_d'/dx_i) (6: 11,12,13,22,23,33),
    w|J|, and d eta_d / d x_i (9, row-major d then i)."""
    ref = reference(shape, P, Q, reduced)
    g = block_metrics(shape, P, Q, X, curved, kind, geometry, reduced)
    Gx = _deta_dx(ref, g)
    G = np.einsum("el,eldi,elki->eldk", g["wJ"], Gx, Gx)
    six = np.stack([G[:, :, 0, 0], G[:, :, 0, 1], G[:, :, 0, 2], G[:, :, 1, 1], G[:, :, 1, 2], G[:, :, 2, 2],
                    g["wJ"]], axis=1)                                  # (Ne, 7, NQ)
    nine = Gx.transpose(0, 2, 3, 1).reshape(Gx.shape[0], 9, -1)        # (Ne, 9, NQ)
    return six, nine


# ---------------------------------------------------------------------------
# mesh level (ragged vectors in user element order)
# ---------------------------------------------------------------------------
def n_points(shape, Q, reduced=0):
    """Quadrature points of an element: Q^3, or with the reduced rule Q - 1 in
    the collapsed directions (prism and pyramid eta_3, tetrahedron eta_2 and eta_3)."""
    Q = int(Q)
    if not reduced or shape == 0:
        return Q ** 3
    return Q * Q * (Q - 1) if shape in (1, 2) else Q * (Q - 1) ** 2


def layout(mesh):
    shape = mesh["shape"].astype(int)
    P = mesh["P"].astype(int)
    Q = mesh["Q"].astype(int)
    npm = np.array([basis.n_modes(s, p) for s, p in zip(shape, P)], dtype=np.int64)
    coeff = np.concatenate([[0], np.cumsum(npm)]).astype(np.int64)
    phys = np.concatenate([[0], np.cumsum([n_points(s, q, mesh.get("quadrature", 0))
                                           for s, q in zip(shape, Q)])]).astype(np.int64)
    return coeff, phys


def _blocks(mesh, elems=None):
    n = mesh["n_elem"]
    elems = np.arange(n) if elems is None else np.asarray(elems)
    keys = {}
    for e in elems:
        k = (int(mesh["shape"][e]), int(mesh["P"][e]), int(mesh["Q"][e]), int(mesh["curved"][e]))
        keys.setdefault(k, []).append(int(e))
    return keys


def _verts(mesh, shape, elems):
    nv = (8, 6, 5, 4)[shape]
    return mesh["xyz"][mesh["vert"][elems][:, :nv]]


IN_KIND = {"bwd_trans": "coeff", "iproduct_wrt_base": "phys", "mass": "coeff", "laplacian": "coeff",
           "helmholtz": "coeff", "phys_deriv": "phys", "iproduct_wrt_deriv": "phys3",
           "helmholtz_collocated": "coeff", "adr": "coeff"}
OUT_KIND = {"bwd_trans": "phys", "iproduct_wrt_base": "coeff", "mass": "coeff", "laplacian": "coeff",
            "helmholtz": "coeff", "phys_deriv": "phys3", "iproduct_wrt_deriv": "coeff",
            "helmholtz_collocated": "coeff", "adr": "coeff"}


def apply(op, mesh, data, lam=1.0, elems=None, adv=None):
    """Apply ``op`` to the ragged vector ``data``; with ``elems``, only those
    elements' outputs are computed (others left zero).  ``adv``: the constant
    velocity of the advection-diffusion-reaction operator ("adr":
    -div grad u + a . grad u + lam u, tested against the basis)."""
    coeff, phys = layout(mesh)
    offs = {"coeff": coeff, "phys": phys, "phys3": phys}
    ik, ok = IN_KIND[op], OUT_KIND[op]
    n_out = offs[ok][-1] * (3 if ok == "phys3" else 1)
    out = np.zeros(n_out)
    n_in_vec = offs[ik][-1]
    kind = mesh["deformation"]
    for (shape, P, Q, cv), el in _blocks(mesh, elems).items():
        el = np.array(el)
        X = _verts(mesh, shape, el)
        oi, oo = offs[ik], offs[ok]
        ni = (oi[el + 1] - oi[el])[0]
        no = (oo[el + 1] - oo[el])[0]
        idx_in = oi[el][:, None] + np.arange(ni)[None, :]
        if ik == "phys3":
            x = np.stack([data[c * n_in_vec + idx_in] for c in range(3)])
        else:
            x = data[idx_in]
        y = apply_block(op, shape, P, Q, X, bool(cv), kind, x, lam, mesh.get("geometry", 0), adv,
                        mesh.get("quadrature", 0))
        idx_out = oo[el][:, None] + np.arange(no)[None, :]
        if ok == "phys3":
            for c in range(3):
                out[c * oo[-1] + idx_out] = y[c]
        else:
            out[idx_out] = y
    return out


def geometric_factors(mesh, elems=None):
    """(six+wJ, nine) per element in user order: lists of (7, NQ) and (9, NQ) arrays."""
    n = mesh["n_elem"]
    six = [None] * n
    nine = [None] * n
    kind = mesh["deformation"]
    for (shape, P, Q, cv), el in _blocks(mesh, elems).items():
        el = np.array(el)
        s7, s9 = geometric_factors_block(shape, P, Q, _verts(mesh, shape, el), bool(cv), kind,
                                         mesh.get("geometry", 0), mesh.get("quadrature", 0))
        for t, e in enumerate(el):
            six[e] = s7[t]
            nine[e] = s9[t]
    return six, nine
