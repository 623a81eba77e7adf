"""Modified C0 modal bases of the four 3-D shapes on collapsed coordinates.

The paper builds its prism, pyramid and tetrahedron expansions as generalised
tensor products on the collapsed coordinates of repeated Duffy
transformations (Sec. 2.3, Eq. for eta_1 and the triangle product
psi^a_p(eta_1) psi^b_pq(eta_2) with p + q <= P, read with the index fix
a_p, b_pq) and refers the 3-D details to Karniadakis & Sherwin.  Each mode
here is written out as a product of three 1-D factors, one per collapsed
coordinate (a, b, c) = (eta_1, eta_2, eta_3); a factor ('1',) means the mode
is constant in that coordinate (the "collapsed vertex" modes).

Collapsed coordinates (xi in the reference element, eta in [-1,1]^3):
  hex     eta = xi
  prism   eta1 = 2(1+xi1)/(1-xi3) - 1, eta2 = xi2, eta3 = xi3
  pyramid eta1 = 2(1+xi1)/(1-xi3) - 1, eta2 = 2(1+xi2)/(1-xi3) - 1, eta3 = xi3
  tet     eta1 = 2(1+xi1)/(-xi2-xi3) - 1, eta2 = 2(1+xi2)/(1-xi3) - 1, eta3 = xi3

Mode order (an interface convention shared with the CUDA library, written
independently on each side): every mode gets a slot key (ka, kb, kc) and the
modes are sorted by that key, kc fastest.  ka: L or constant -> 0, R -> 1,
psi_n -> n+1.  kb: if the a-factor has weight 0 (L, R or constant) or the
shape is not a tetrahedron, the same rule on the b-factor; for a tetrahedron
with a-factor psi_p the b-factor is W_{p,q} and kb = q.  kc: the c-factor
belongs to the family of weight s (prism s = w(a), pyramid s = max(w(a),
w(b)), tet s = w(a) + w(b), hex s = 0); s = 0 uses the L/R/psi rule, s >= 1
has factors W_{s,r} and kc = r.  Weights: w(L) = w(R) = w(1) = 0,
w(psi_n) = n, w(W_{s,q}) = q.
"""
import numpy as np

from .jacobi import factor

HEX, PRISM, PYR, TET = 0, 1, 2, 3

REF_VERTS = {
    HEX: [(-1, -1, -1), (1, -1, -1), (1, 1, -1), (-1, 1, -1), (-1, -1, 1), (1, -1, 1), (1, 1, 1), (-1, 1, 1)],
    PRISM: [(-1, -1, -1), (1, -1, -1), (1, 1, -1), (-1, 1, -1), (-1, -1, 1), (-1, 1, 1)],
    PYR: [(-1, -1, -1), (1, -1, -1), (1, 1, -1), (-1, 1, -1), (-1, -1, 1)],
    TET: [(-1, -1, -1), (1, -1, -1), (-1, 1, -1), (-1, -1, 1)],
}
REF_VOLUME = {HEX: 8.0, PRISM: 4.0, PYR: 8.0 / 3.0, TET: 4.0 / 3.0}


def n_modes(shape, P):
    """Closed-form mode counts of the four shapes."""
    if shape == HEX:
        return (P + 1) ** 3
    if shape == PRISM:
        return (P + 1) ** 2 * (P + 2) // 2
    if shape == PYR:
        return (P + 1) * (P + 2) * (2 * P + 3) // 6
    return (P + 1) * (P + 2) * (P + 3) // 6


def _A(P):
    """The full 1-D family: L, R and the P-1 bubbles."""
    return [("L",), ("R",)] + [("psi", n) for n in range(1, P)]


def _weight(f):
    if f[0] == "psi":
        return f[1]
    if f[0] == "W":
        return f[2]
    return 0


def _a_key(f):
    if f[0] in ("1", "L"):
        return 0
    if f[0] == "R":
        return 1
    return f[1] + 1


def _mode_list_unsorted(shape, P):
    A = _A(P)
    out = []
    if shape == HEX:
        for fa in A:
            for fb in A:
                for fc in A:
                    out.append((fa, fb, fc))
        return out
    if shape == PRISM:
        tri = [(("L",), ("L",)), (("R",), ("L",)), (("1",), ("R",))]
        tri += [(("psi", p), ("W", p, 0)) for p in range(1, P)]
        tri += [(("L",), ("psi", r)) for r in range(1, P)]
        tri += [(("R",), ("psi", r)) for r in range(1, P)]
        tri += [(("psi", p), ("W", p, r)) for p in range(1, P) for r in range(1, P) if p + r < P]
        for fa, fc in tri:
            for fb in A:
                out.append((fa, fb, fc))
        return out
    if shape == PYR:
        LR = [("L",), ("R",)]
        out += [(fa, fb, ("L",)) for fa in LR for fb in LR]
        out.append((("1",), ("1",), ("R",)))
        for p in range(1, P):
            for g in LR:
                out.append((("psi", p), g, ("W", p, 0)))
                out.append((g, ("psi", p), ("W", p, 0)))
        for r in range(1, P):
            out += [(fa, fb, ("psi", r)) for fa in LR for fb in LR]
        for p in range(1, P):
            for q in range(1, P):
                out.append((("psi", p), ("psi", q), ("W", max(p, q), 0)))
        for q in range(1, P):
            for r in range(1, P):
                if q + r < P:
                    for g in LR:
                        out.append((g, ("psi", q), ("W", q, r)))
                        out.append((("psi", q), g, ("W", q, r)))
        for p in range(1, P):
            for q in range(1, P):
                m = max(p, q)
                for r in range(1, P):
                    if m + r < P:
                        out.append((("psi", p), ("psi", q), ("W", m, r)))
        return out
    if shape == TET:
        # vertices A, B, C, D
        out += [(("L",), ("L",), ("L",)), (("R",), ("L",), ("L",)),
                (("1",), ("R",), ("L",)), (("1",), ("1",), ("R",))]
        for n in range(1, P):
            out.append((("psi", n), ("W", n, 0), ("W", n, 0)))      # edge AB
            out.append((("L",), ("psi", n), ("W", n, 0)))           # edge AC
            out.append((("R",), ("psi", n), ("W", n, 0)))           # edge BC
            out.append((("L",), ("L",), ("psi", n)))                # edge AD
            out.append((("R",), ("L",), ("psi", n)))                # edge BD
            out.append((("1",), ("R",), ("psi", n)))                # edge CD
        for p in range(1, P):
            for q in range(1, P):
                if p + q < P:
                    out.append((("psi", p), ("W", p, q), ("W", p + q, 0)))   # face ABC
        for p in range(1, P):
            for r in range(1, P):
                if p + r < P:
                    out.append((("psi", p), ("W", p, 0), ("W", p, r)))       # face ABD
        for q in range(1, P):
            for r in range(1, P):
                if q + r < P:
                    out.append((("L",), ("psi", q), ("W", q, r)))            # face ACD
                    out.append((("R",), ("psi", q), ("W", q, r)))            # face BCD
        for p in range(1, P):
            for q in range(1, P):
                for r in range(1, P):
                    if p + q + r < P:
                        out.append((("psi", p), ("W", p, q), ("W", p + q, r)))  # interior
        return out
    raise ValueError(shape)


def slot_key(shape, mode):
    fa, fb, fc = mode
    ka = _a_key(fa)
    if shape == TET and fa[0] == "psi":
        kb = fb[2]
    else:
        kb = _a_key(fb)
    if shape == HEX:
        s = 0
    elif shape == PRISM:
        s = _weight(fa)
    elif shape == PYR:
        s = max(_weight(fa), _weight(fb))
    else:
        s = _weight(fa) + _weight(fb)
    kc = _a_key(fc) if s == 0 else fc[2]
    return (ka, kb, kc)


def modes(shape, P):
    """Mode list of (shape, P) in the canonical order."""
    ms = _mode_list_unsorted(shape, P)
    return sorted(ms, key=lambda m: slot_key(shape, m))


def eta_from_xi(shape, xi1, xi2, xi3):
    if shape == HEX:
        return xi1, xi2, xi3
    if shape == PRISM:
        return 2.0 * (1.0 + xi1) / (1.0 - xi3) - 1.0, xi2, xi3
    if shape == PYR:
        return (2.0 * (1.0 + xi1) / (1.0 - xi3) - 1.0,
                2.0 * (1.0 + xi2) / (1.0 - xi3) - 1.0, xi3)
    return (2.0 * (1.0 + xi1) / (-xi2 - xi3) - 1.0,
            2.0 * (1.0 + xi2) / (1.0 - xi3) - 1.0, xi3)


def xi_from_eta(shape, e1, e2, e3):
    if shape == HEX:
        return e1, e2, e3
    if shape == PRISM:
        return (1.0 + e1) * (1.0 - e3) / 2.0 - 1.0, e2, e3
    if shape == PYR:
        return ((1.0 + e1) * (1.0 - e3) / 2.0 - 1.0,
                (1.0 + e2) * (1.0 - e3) / 2.0 - 1.0, e3)
    return ((1.0 + e1) * (1.0 - e2) * (1.0 - e3) / 4.0 - 1.0,
            (1.0 + e2) * (1.0 - e3) / 2.0 - 1.0, e3)


def evaluate(shape, P, xi1, xi2, xi3, mode_list=None):
    """phi_m(xi) for all modes: array (n_points, n_modes); complex inputs allowed."""
    if mode_list is None:
        mode_list = modes(shape, P)
    a, b, c = eta_from_xi(shape, np.asarray(xi1), np.asarray(xi2), np.asarray(xi3))
    cols = [factor(fa, a) * factor(fb, b) * factor(fc, c) for fa, fb, fc in mode_list]
    return np.stack(cols, axis=-1)


def complex_step_gradient(fun, xi, h=1e-30):
    """d fun / d xi_d for d = 0..2 by the complex-step method (Squire & Trapp 1998).

    fun maps three coordinate arrays to an array; xi is a (3, n) real array.
    Returns a list of three arrays, each exact to rounding for analytic fun.
    """
    out = []
    for d in range(3):
        z = [np.asarray(xi[k], dtype=np.complex128) for k in range(3)]
        z[d] = z[d] + 1j * h
        out.append(np.imag(fun(*z)) / h)
    return out
