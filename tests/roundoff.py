"""Per-output rounding-error bounds of the reduced-precision operators, built
from the oracle's matrices (test infrastructure).

Standard first-order bound: an output that is a sum of products, each product
of k rounded factors (relative error <= u each) and the sum accumulated with
relative error <= gamma, satisfies |y_m - exact_m| <= (k u + gamma) S_m with
S_m the same sum with every factor and term replaced by its absolute value.

Tensor-core elemental matrix (TF32 / BF16), which evaluates
out = sum_c sum_c' A_c^T M_cc' A_c' uhat with dense reference matrices A_c =
B, dB/d eta_1..3 at the points and the per-point metric M (lambda w|J| for
c = c' = 0, G_dd' for c, c' >= 1): each term carries k = 5 roundings to the
operand type (the coefficient, the two reference entries, the metric-weighted
point value V', and the metric factor itself in FP16 after its power-of-two
scale, whose 11 significant bits round at most by 2^-11 <= u), and FP32
accumulates N_P terms forward and 4 N_Q backward:
    bound_m = (5 u + (N_P + 4 N_Q) 2^-24) (|A|^T |M| |A| |uhat|)_m.

FP32 sum factorisation, which evaluates the same operator as the chain
B^T [ sum_d D_d^T G_dd' D_d' + lambda w|J| ] B uhat of 1-D passes: along the
longest chain an output accumulates the 3 passes of B (n = P + 1 terms
each), one collocation derivative (Q terms), the metric (3 terms), the
transposed derivatives (3 Q terms) and the 3 passes of B^T (Q terms each),
so k <= 3 n + 7 Q + 3 products and sums, all in FP32:
    bound_m = 2 (3 n + 7 Q + 3) 2^-24 (|B|^T [sum_d |D_d|^T |G| |D_d'| + |lambda w|J||] |B| |uhat|)_m,
with |B| |uhat| taken per point as the sum over modes of |phi_m| |uhat_m|
(a tensor product of 1-D factors: the same sum the passes accumulate) and
|D_d| applied along direction d of the Q^3 point tensor.  The factor 2: the
eta_1 passes use the table {1/2, -z/2} on the sum and the difference of the
two vertex coefficients (L = 1/2 - z/2, R = 1/2 + z/2), whose absolute chain
(1/2 + |z|/2)(|u_L| + |u_R|) is at most twice |L| |u_L| + |R| |u_R|.
Tensor-core hybrid (TF32 / BF16), which evaluates the same chain with B and
B^T as tensor-core products and the collocated core in FP32: four roundings
to the operand type (the coefficient and the entry of B in u = B uhat, the
point value u' and the entry of B in B^T u'), and FP32 along the rest of the
chain (N_P terms forward, Q + 3 + 3 Q in the core, N_Q backward, and the FP32
factors and collocation tables):
    bound_m = (4 u + (N_P + N_Q + 4 Q + 10) 2^-24) (the chain of the sum factorisation)_m.
All three are slightly enlarged (x 1.1) for second-order terms.
"""
import numpy as np

from oracle import operators as ops

U32 = 2.0 ** -24


def eta_matrices(shape, P, Q, reduced=0):
    """A[c] (4, NQ, NP): B and d B / d eta_d at the points."""
    ref = ops.reference(shape, P, Q, reduced)
    Tinv = np.linalg.inv(ref["T"])                                   # [l, a, d] = d xi_a / d eta_d
    Deta = np.einsum("alm,lad->dlm", np.stack(ref["Dxi"]), Tinv)
    return np.concatenate([ref["B"][None], Deta])


def _metric_abs(six, lam, kind):
    """|M| as (Ne, 4, 4, NQ) from the oracle's factors (G11 G12 G13 G22 G23 G33 w|J|)."""
    Ne, _, NQ = six.shape
    M = np.zeros((Ne, 4, 4, NQ))
    if kind in ("mass", "helmholtz"):
        M[:, 0, 0] = np.abs((lam if kind == "helmholtz" else 1.0) * six[:, 6])
    if kind in ("laplacian", "helmholtz"):
        idx = {(0, 0): 0, (0, 1): 1, (0, 2): 2, (1, 1): 3, (1, 2): 4, (2, 2): 5}
        for (a, b), f in idx.items():
            M[:, 1 + a, 1 + b] = np.abs(six[:, f])
            M[:, 1 + b, 1 + a] = np.abs(six[:, f])
    return M


def tc_chain(mesh, x, lam, kind):
    """(|A|^T |M| |A| |x|)_m for every output coefficient."""
    co, _ = ops.layout(mesh)
    out = np.zeros(co[-1])
    geometry, rq = mesh.get("geometry", 0), mesh.get("quadrature", 0)
    for (shape, P, Q, cv), el in ops._blocks(mesh).items():
        el = np.array(el)
        X = ops._verts(mesh, shape, el)
        A = np.abs(eta_matrices(shape, P, Q, rq))
        six, _ = ops.geometric_factors_block(shape, P, Q, X, bool(cv), mesh["deformation"], geometry, rq)
        M = _metric_abs(six, lam, kind)
        idx = co[el][:, None] + np.arange(co[el[0] + 1] - co[el[0]])[None, :]
        v = np.einsum("cln,en->ecl", A, np.abs(x[idx]))              # (Ne, 4, NQ)
        w = np.einsum("ecdl,edl->ecl", M, v)
        out[idx] = np.einsum("clm,ecl->em", A, w)
    return out


def sf_chain(mesh, x, lam, kind):
    """The absolute chain of the sum-factorised passes for every output coefficient."""
    co, _ = ops.layout(mesh)
    out = np.zeros(co[-1])
    geometry = mesh.get("geometry", 0)
    for (shape, P, Q, cv), el in ops._blocks(mesh).items():
        el = np.array(el)
        X = ops._verts(mesh, shape, el)
        ref = ops.reference(shape, P, Q)
        B = np.abs(ref["B"])
        D = [np.abs(d) for d in ref["D1"]]
        six, _ = ops.geometric_factors_block(shape, P, Q, X, bool(cv), mesh["deformation"], geometry)
        M = _metric_abs(six, lam, kind)
        idx = co[el][:, None] + np.arange(co[el[0] + 1] - co[el[0]])[None, :]
        u = np.abs(x[idx]) @ B.T                                      # (Ne, NQ)
        U = u.reshape(-1, Q, Q, Q)
        v = np.stack([np.einsum("im,emjk->eijk", D[0], U), np.einsum("jm,eimk->eijk", D[1], U),
                      np.einsum("km,eijm->eijk", D[2], U)]).reshape(3, len(el), -1)
        t = M[:, 0, 0] * u                                            # (Ne, NQ)
        w = np.einsum("edfl,fel->del", M[:, 1:, 1:], v)               # (3, Ne, NQ)
        W = w.reshape(3, len(el), Q, Q, Q)
        back = (np.einsum("mi,emjk->eijk", D[0], W[0]) + np.einsum("mj,eimk->eijk", D[1], W[1])
                + np.einsum("mk,eijm->eijk", D[2], W[2])).reshape(len(el), -1)
        out[idx] = (t + back) @ B
    return out


def tc_bound(mesh, x, lam, kind, u):
    co, _ = ops.layout(mesh)
    out = np.zeros(co[-1])
    chain = tc_chain(mesh, x, lam, kind)
    for e in range(mesh["n_elem"]):
        NP = co[e + 1] - co[e]
        NQ = ops.n_points(int(mesh["shape"][e]), int(mesh["Q"][e]), mesh.get("quadrature", 0))
        out[co[e]:co[e + 1]] = 1.1 * (5 * u + (NP + 4 * NQ) * U32) * chain[co[e]:co[e + 1]]
    return out


def sf32_bound(mesh, x, lam, kind):
    co, _ = ops.layout(mesh)
    out = np.zeros(co[-1])
    chain = sf_chain(mesh, x, lam, kind)
    for e in range(mesh["n_elem"]):
        P = int(mesh["P"][e])
        out[co[e]:co[e + 1]] = 1.1 * 2 * (3 * (P + 1) + 7 * (P + 2) + 3) * U32 * chain[co[e]:co[e + 1]]
    return out


def hyb_bound(mesh, x, lam, kind, u):
    co, _ = ops.layout(mesh)
    out = np.zeros(co[-1])
    chain = sf_chain(mesh, x, lam, kind)
    for e in range(mesh["n_elem"]):
        NP = co[e + 1] - co[e]
        Q = int(mesh["Q"][e])
        out[co[e]:co[e + 1]] = 1.1 * (4 * u + (NP + Q ** 3 + 4 * Q + 10) * U32) * chain[co[e]:co[e + 1]]
    return out
