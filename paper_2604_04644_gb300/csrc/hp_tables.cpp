// Reference-element tables: quadrature, 1-D modal families, Lagrange
// differentiation and the slot <-> mode maps of the four shapes.
//
// Quadrature (paper Sec. 2.1: tensor rules with P+2 Gauss-Lobatto points; Sec.
// 2.3: tensor rules on the collapsed coordinates of the Duffy map).  Zeros of
// Jacobi polynomials by Newton's method with deflation; Gauss-Lobatto weights
// from their closed form 2/(Q(Q-1) P_{Q-1}(x)^2); Gauss-Radau-Jacobi weights as
// integrals of the Lagrange polynomials, computed with a Gauss-Jacobi rule of
// Q+1 points whose weights use the closed form
//   w_j = 2^{a+b+1} G(n+a+1) G(n+b+1) / (G(n+a+b+1) n! (1-x_j^2) P_n'(x_j)^2).
// The Duffy Jacobian is absorbed into the collapsed directions (GRJ with
// alpha = 1 halved, alpha = 2 quartered).
//
// Modal families (modified C0 basis of Karniadakis & Sherwin, cited by the
// paper for its 3-D expansions): family 0 = {L, R, psi_1..psi_{P-1}},
// psi_n = L R P^{(1,1)}_{n-1}; family s >= 1 = W_s with W_{s,0} = L^{s+1},
// W_{s,r} = L^{s+1} R P^{(2s+1,1)}_{r-1} (r = 1..P-1-s).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <stdexcept>

#include "hp_internal.h"

namespace hp {
namespace {

double jac(int n, double a, double b, double x) {
    if (n == 0) return 1.0;
    double p0 = 1.0, p1 = 0.5 * (a - b + (a + b + 2.0) * x);
    for (int k = 2; k <= n; ++k) {
        double c = 2.0 * k + a + b;
        double a1 = 2.0 * k * (k + a + b) * (c - 2.0);
        double a2 = (c - 1.0) * (a * a - b * b);
        double a3 = (c - 2.0) * (c - 1.0) * c;
        double a4 = 2.0 * (k + a - 1.0) * (k + b - 1.0) * c;
        double p2 = ((a2 + a3 * x) * p1 - a4 * p0) / a1;
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

// d/dx P_n^{(a,b)} = (n + a + b + 1)/2 P_{n-1}^{(a+1,b+1)}
double jac_d(int n, double a, double b, double x) {
    if (n == 0) return 0.0;
    return 0.5 * (n + a + b + 1.0) * jac(n - 1, a + 1.0, b + 1.0, x);
}

std::vector<double> jac_zeros(int n, double a, double b) {
    std::vector<double> x(n);
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < n; ++k) {
        double r = -std::cos((2.0 * k + 1.0) * pi / (2.0 * n));
        if (k > 0) r = 0.5 * (r + x[k - 1]);
        for (int it = 0; it < 200; ++it) {
            double s = 0.0;
            for (int j = 0; j < k; ++j) s += 1.0 / (r - x[j]);
            double p = jac(n, a, b, r);
            double delta = -p / (jac_d(n, a, b, r) - s * p);
            r += delta;
            if (std::fabs(delta) < 1e-16) break;
        }
        x[k] = r;
    }
    std::sort(x.begin(), x.end());
    return x;
}

void gauss_jacobi(int n, double a, double b, std::vector<double>& x, std::vector<double>& w) {
    x = jac_zeros(n, a, b);
    w.resize(n);
    double c = std::pow(2.0, a + b + 1.0) * std::tgamma(n + a + 1.0) * std::tgamma(n + b + 1.0) /
               (std::tgamma(n + a + b + 1.0) * std::tgamma(n + 1.0));
    for (int j = 0; j < n; ++j) {
        double d = jac_d(n, a, b, x[j]);
        w[j] = c / ((1.0 - x[j] * x[j]) * d * d);
    }
}

void gll_rule(int Q, std::vector<double>& x, std::vector<double>& w) {
    std::vector<double> in = jac_zeros(Q - 2, 1.0, 1.0);
    x.clear();
    x.push_back(-1.0);
    x.insert(x.end(), in.begin(), in.end());
    x.push_back(1.0);
    w.resize(Q);
    for (int i = 0; i < Q; ++i) {
        double p = jac(Q - 1, 0.0, 0.0, x[i]);
        w[i] = 2.0 / (Q * (Q - 1.0) * p * p);
    }
    // exact symmetry about 0 (the even-odd passes rely on z_{Q-1-i} = -z_i)
    for (int i = 0; i < Q / 2; ++i) {
        double a = 0.5 * (x[Q - 1 - i] - x[i]), b = 0.5 * (w[i] + w[Q - 1 - i]);
        x[i] = -a; x[Q - 1 - i] = a; w[i] = b; w[Q - 1 - i] = b;
    }
    if (Q % 2) x[Q / 2] = 0.0;
}

void grj_rule(int Q, int alpha, std::vector<double>& x, std::vector<double>& w) {
    std::vector<double> in = jac_zeros(Q - 1, (double)alpha, 1.0);
    x.clear();
    x.push_back(-1.0);
    x.insert(x.end(), in.begin(), in.end());
    std::vector<double> gx, gw;
    gauss_jacobi(Q + 1, (double)alpha, 0.0, gx, gw);
    w.assign(Q, 0.0);
    for (int l = 0; l < Q; ++l) {
        for (size_t g = 0; g < gx.size(); ++g) {
            double ell = 1.0;
            for (int k = 0; k < Q; ++k)
                if (k != l) ell *= (gx[g] - x[k]) / (x[l] - x[k]);
            w[l] += gw[g] * ell;
        }
    }
}

// D[i][j] = h_j'(x_i): barycentric form, diagonal by the negative-sum rule
std::vector<double> lagrange_d(const std::vector<double>& x) {
    int n = (int)x.size();
    std::vector<double> c(n, 1.0), D(n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k)
            if (k != i) c[i] *= (x[i] - x[k]);
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            D[i * n + j] = c[i] / (c[j] * (x[i] - x[j]));
            s += D[i * n + j];
        }
        D[i * n + i] = -s;
    }
    return D;
}

double fL(double z) { return 0.5 * (1.0 - z); }
double fR(double z) { return 0.5 * (1.0 + z); }

// member m of family s at z (zero past the end of the family)
double family(int P, int s, int m, double z) {
    if (s == 0) {
        if (m == 0) return fL(z);
        if (m == 1) return fR(z);
        if (m <= P) return fL(z) * fR(z) * jac(m - 2, 1.0, 1.0, z);
        return 0.0;
    }
    if (s >= P || m >= P - s) return 0.0;
    double l = std::pow(fL(z), s + 1);
    if (m == 0) return l;
    return l * fR(z) * jac(m - 1, 2.0 * s + 1.0, 1.0, z);
}

int wA(int a) { return a <= 1 ? 0 : a - 1; }   // weight of member a of family 0

RefTables build(int shape, int P) {
    RefTables t;
    t.shape = shape;
    t.P = P;
    t.Q = P + 2;
    t.n = P + 1;
    const int Q = t.Q, n = t.n;
    t.NQ = Q * Q * Q;
    // points per direction
    std::vector<double> gx, gw, r1x, r1w, r2x, r2w;
    gll_rule(Q, gx, gw);
    grj_rule(Q, 1, r1x, r1w);
    for (double& v : r1w) v *= 0.5;
    grj_rule(Q, 2, r2x, r2w);
    for (double& v : r2w) v *= 0.25;
    t.z[0] = gx; t.w[0] = gw;
    if (shape == HP_HEX) { t.z[1] = gx; t.w[1] = gw; t.z[2] = gx; t.w[2] = gw; }
    if (shape == HP_PRISM) { t.z[1] = gx; t.w[1] = gw; t.z[2] = r1x; t.w[2] = r1w; }
    if (shape == HP_PYR) { t.z[1] = gx; t.w[1] = gw; t.z[2] = r2x; t.w[2] = r2w; }
    if (shape == HP_TET) { t.z[1] = r1x; t.w[1] = r1w; t.z[2] = r2x; t.w[2] = r2w; }
    for (int d = 0; d < 3; ++d) t.D[d] = lagrange_d(t.z[d]);
    // 1-D tables
    t.Ta.assign(n * Q, 0.0);
    for (int a = 0; a < n; ++a)
        for (int i = 0; i < Q; ++i) t.Ta[a * Q + i] = family(P, 0, a, t.z[0][i]);
    // parity form of the eta1 table (GLL points, symmetric about 0): the vertex
    // pair {L, R} becomes {1/2, -z/2} (the coefficients of the slots a = 0, 1
    // enter as their sum and difference), so row a has parity (-1)^a; Td is
    // its derivative, row a of parity (-1)^(a+1).  Mirrored entries are set
    // from the first half, entries of the wrong parity at z = 0 are exact zeros.
    {
        const int Qh = (Q + 1) / 2;
        t.Tp.assign(n * Q, 0.0);
        t.Td.assign(n * Q, 0.0);
        for (int i = 0; i < Q; ++i) {
            t.Tp[0 * Q + i] = 0.5;
            t.Tp[1 * Q + i] = -0.5 * t.z[0][i];
            for (int a = 2; a < n; ++a) t.Tp[a * Q + i] = t.Ta[a * Q + i];
        }
        for (int a = 0; a < n; ++a)
            for (int i = 0; i < Q; ++i) {
                double d = 0.0;
                for (int m = 0; m < Q; ++m) d += t.D[0][i * Q + m] * t.Tp[a * Q + m];
                t.Td[a * Q + i] = a == 0 ? 0.0 : (a == 1 ? -0.5 : d);
            }
        for (int a = 0; a < n; ++a) {
            const double sp = (a % 2) ? -1.0 : 1.0;          // parity of Tp row a; Td has -sp
            for (int i = 0; i < Qh; ++i) {
                const int i2 = Q - 1 - i;
                double tp = 0.5 * (t.Tp[a * Q + i] + sp * t.Tp[a * Q + i2]);
                double td = 0.5 * (t.Td[a * Q + i] - sp * t.Td[a * Q + i2]);
                if (i == i2) { if (sp < 0) tp = 0.0; else td = 0.0; }
                t.Tp[a * Q + i] = tp; t.Tp[a * Q + i2] = sp * tp;
                t.Td[a * Q + i] = td; t.Td[a * Q + i2] = -sp * td;
            }
        }
    }
    t.Tb.assign((P + 1) * n * Q, 0.0);
    t.Tc.assign((P + 1) * n * Q, 0.0);
    for (int s = 0; s <= P; ++s)
        for (int m = 0; m < n; ++m)
            for (int q = 0; q < Q; ++q) {
                t.Tb[(s * n + m) * Q + q] = family(P, s, m, t.z[1][q]);
                t.Tc[(s * n + m) * Q + q] = family(P, s, m, t.z[2][q]);
            }
    // their derivatives at the points: every family member has degree <= P < Q
    // in its variable, so the collocation derivative of its values is exact
    t.Tbd.assign(t.Tb.size(), 0.0);
    t.Tcd.assign(t.Tc.size(), 0.0);
    for (int r = 0; r < (P + 1) * n; ++r)
        for (int q = 0; q < Q; ++q) {
            double db = 0.0, dc = 0.0;
            for (int m = 0; m < Q; ++m) {
                db += t.D[1][q * Q + m] * t.Tb[r * Q + m];
                dc += t.D[2][q * Q + m] * t.Tc[r * Q + m];
            }
            t.Tbd[r * Q + q] = db;
            t.Tcd[r * Q + q] = dc;
        }
    // families and slot validity
    t.famb.assign(n, 0);
    t.famc.assign(n * n, 0);
    for (int a = 0; a < n; ++a) {
        if (shape == HP_TET) t.famb[a] = (uint8_t)wA(a);
        for (int b = 0; b < n; ++b) {
            int s = 0;
            if (shape == HP_PRISM) s = wA(a);
            if (shape == HP_PYR) s = std::max(wA(a), wA(b));
            if (shape == HP_TET) {
                if (a <= 1) s = wA(b);
                else s = (b < P - wA(a)) ? wA(a) + b : P;
            }
            t.famc[a * n + b] = (uint8_t)s;
        }
    }
    // canonical slot of each valid slot (merges of the collapsed modes)
    std::vector<int> canon(n * n * n, -1);
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
            int s = t.famc[a * n + b];
            bool bvalid = true;
            if (shape == HP_TET && a >= 2) bvalid = b < P - wA(a);
            for (int c = 0; c < n; ++c) {
                bool cvalid = bvalid && (s == 0 ? true : (s < P && c < P - s));
                if (!cvalid) continue;
                int ca = a, cb = b, cc = c;
                if (shape == HP_PRISM && s == 0 && c == 1 && a <= 1) ca = 0;
                if (shape == HP_PYR && s == 0 && c == 1 && a <= 1 && b <= 1) { ca = 0; cb = 0; }
                if (shape == HP_TET && a <= 1) {
                    if (b <= 1 && c == 1) { ca = 0; cb = 0; }
                    else if (b == 1) ca = 0;
                }
                canon[(a * n + b) * n + c] = (ca * n + cb) * n + cc;
            }
        }
    std::vector<int> mode_of(n * n * n, -1);
    int m = 0;
    for (int sl = 0; sl < n * n * n; ++sl)
        if (canon[sl] == sl) mode_of[sl] = m++;
    t.NP = m;
    t.slot2mode.assign(n * n * n, -1);
    t.mode_slots.assign(m * 4, -1);
    std::vector<int> cnt(m, 0);
    for (int sl = 0; sl < n * n * n; ++sl) {
        if (canon[sl] < 0) continue;
        int md = mode_of[canon[sl]];
        if (md < 0 || cnt[md] >= 4) throw std::runtime_error("slot map");
        t.slot2mode[sl] = (int16_t)md;
        t.mode_slots[md * 4 + cnt[md]++] = (int16_t)sl;
    }
    if (t.NP != n_modes(shape, P)) throw std::runtime_error("mode count");
    return t;
}

std::mutex g_mu;
std::map<int, RefTables> g_tables;

}  // namespace

int n_modes(int shape, int P) {
    switch (shape) {
        case HP_HEX: return (P + 1) * (P + 1) * (P + 1);
        case HP_PRISM: return (P + 1) * (P + 1) * (P + 2) / 2;
        case HP_PYR: return (P + 1) * (P + 2) * (2 * P + 3) / 6;
        default: return (P + 1) * (P + 2) * (P + 3) / 6;
    }
}

const RefTables& ref_tables(int shape, int P) {
    std::lock_guard<std::mutex> lk(g_mu);
    int key = shape * 16 + P;
    auto it = g_tables.find(key);
    if (it == g_tables.end()) it = g_tables.emplace(key, build(shape, P)).first;
    return it->second;
}

double family_value(int P, int s, int m, double z) { return family(P, s, m, z); }

void eval_modes(int shape, int P, const double xi[3], double* out) {
    // eta(xi) of the collapsed coordinates, then the generalised tensor product
    double e1 = xi[0], e2 = xi[1], e3 = xi[2];
    if (shape == HP_PRISM) e1 = 2.0 * (1.0 + xi[0]) / (1.0 - xi[2]) - 1.0;
    if (shape == HP_PYR) {
        e1 = 2.0 * (1.0 + xi[0]) / (1.0 - xi[2]) - 1.0;
        e2 = 2.0 * (1.0 + xi[1]) / (1.0 - xi[2]) - 1.0;
    }
    if (shape == HP_TET) {
        e1 = 2.0 * (1.0 + xi[0]) / (-xi[1] - xi[2]) - 1.0;
        e2 = 2.0 * (1.0 + xi[1]) / (1.0 - xi[2]) - 1.0;
    }
    const RefTables& t = ref_tables(shape, P);
    const int n = t.n;
    for (int m = 0; m < t.NP; ++m) out[m] = 0.0;
    for (int sl = 0; sl < n * n * n; ++sl) {
        int m = t.slot2mode[sl];
        if (m < 0) continue;
        int a = sl / (n * n), b = (sl / n) % n, c = sl % n;
        out[m] += family(P, 0, a, e1) * family(P, t.famb[a], b, e2) * family(P, t.famc[a * n + b], c, e3);
    }
}

std::vector<double> dense_matrices(int shape, int P) {
    // A4[q][l][m], q = 0: B = phi_m at point l; q = d + 1: d phi_m / d eta_d at l,
    // obtained as D_d B (exact: each phi_m lies in the Lagrange span of the points)
    const RefTables& t = ref_tables(shape, P);
    const int n = t.n, Q = t.Q, NQ = t.NQ, NP = t.NP;
    std::vector<double> A(4 * (size_t)NQ * NP, 0.0);
    for (int m = 0; m < NP; ++m) {
        for (int q = 0; q < 4; ++q) {
            int sl = t.mode_slots[m * 4 + q];
            if (sl < 0) continue;
            int a = sl / (n * n), b = (sl / n) % n, c = sl % n;
            int tb = t.famb[a], sc = t.famc[a * n + b];
            for (int i = 0; i < Q; ++i)
                for (int j = 0; j < Q; ++j)
                    for (int k = 0; k < Q; ++k)
                        A[((size_t)((i * Q + j) * Q + k)) * NP + m] +=
                            t.Ta[a * Q + i] * t.Tb[(tb * n + b) * Q + j] * t.Tc[(sc * n + c) * Q + k];
        }
    }
    for (int d = 0; d < 3; ++d) {
        const std::vector<double>& D = t.D[d];
        for (int i = 0; i < Q; ++i)
            for (int j = 0; j < Q; ++j)
                for (int k = 0; k < Q; ++k) {
                    int l = (i * Q + j) * Q + k;
                    for (int mm = 0; mm < Q; ++mm) {
                        int src = d == 0 ? (mm * Q + j) * Q + k : d == 1 ? (i * Q + mm) * Q + k : (i * Q + j) * Q + mm;
                        double dv = D[(d == 0 ? i : d == 1 ? j : k) * Q + mm];
                        const double* from = &A[(size_t)src * NP];
                        double* to = &A[((size_t)(d + 1) * NQ + l) * NP];
                        for (int m = 0; m < NP; ++m) to[m] += dv * from[m];
                    }
                }
    }
    return A;
}

std::vector<unsigned char> make_blob(const RefTables& t, size_t vs) {
    BlobLayout L = blob_layout_c(t.shape, t.P, (int)vs);
    std::vector<unsigned char> out(L.total_bytes, 0);
    auto put = [&](int off, const std::vector<double>& v) {
        for (size_t i = 0; i < v.size(); ++i) {
            if (vs == 8) {
                double d = v[i];
                std::memcpy(&out[(off + i) * 8], &d, 8);
            } else {
                float f = (float)v[i];
                std::memcpy(&out[(off + i) * 4], &f, 4);
            }
        }
    };
    put(L.Ta, t.Tp);
    put(L.Td, t.Td);
    put(L.Tb, t.Tb);
    put(L.Tc, t.Tc);
    for (int d = 0; d < 3; ++d) {
        std::vector<double> tmp(t.D[d]);
        put(L.D + d * t.Q * t.Q, tmp);
        put(L.z + d * t.Q, t.z[d]);
        put(L.w + d * t.Q, t.w[d]);
        // reciprocals of the collapse factors 1 - z (the Duffy chain rule of
        // affine elements); the GLL end point z = 1 never collapses: 0
        std::vector<double> rz(t.Q);
        for (int i = 0; i < t.Q; ++i) rz[i] = t.z[d][i] < 1.0 ? 1.0 / (1.0 - t.z[d][i]) : 0.0;
        put(L.rz + d * t.Q, rz);
    }
    std::memcpy(&out[L.famb], t.famb.data(), t.famb.size());
    std::memcpy(&out[L.famc], t.famc.data(), t.famc.size());
    std::memcpy(&out[L.slot2mode], t.slot2mode.data(), 2 * t.slot2mode.size());
    std::memcpy(&out[L.mode_slots], t.mode_slots.data(), 2 * t.mode_slots.size());
    // Valid index sets of the collapsed shapes, for passes that skip the
    // padding: pairs (a-major, b ascending) = ab | famc << 16 | family length
    // << 24; slots = ab*n + c | pair << 11 | famc << 18 | c << 22; poff[a] =
    // first pair of a; porder = pairs by decreasing family length.
    std::vector<int32_t> pairs, valid;
    std::vector<int16_t> poff;
    const int n = t.n;
    for (int a = 0; a < n; ++a) {
        poff.push_back((int16_t)pairs.size());
        for (int b = 0; b < lenb_c(t.shape, t.P, a); ++b) {
            int sc = famc_c(t.shape, t.P, a, b), len = famlen_c(t.P, sc);
            if (sc != t.famc[a * n + b]) throw std::runtime_error("family table mismatch");
            int p = (int)pairs.size();
            pairs.push_back((a * n + b) | (sc << 16) | (len << 24));
            for (int c = 0; c < len; ++c) valid.push_back(((a * n + b) * n + c) | (p << 11) | (sc << 18) | (c << 22));
        }
    }
    poff.push_back((int16_t)pairs.size());
    if ((int)pairs.size() != npairs_c(t.shape, t.P) || (int)valid.size() != nvalid_c(t.shape, t.P))
        throw std::runtime_error("valid slot count mismatch");
    std::vector<char> is_valid(n * n * n, 0);
    for (int32_t v : valid) is_valid[v & 2047] = 1;
    for (int sl = 0; sl < n * n * n; ++sl)   // every mode slot is a valid slot
        if (t.slot2mode[sl] >= 0 && !is_valid[sl]) throw std::runtime_error("mode slot outside the valid range");
    std::vector<uint8_t> porder(pairs.size());
    for (size_t p = 0; p < pairs.size(); ++p) porder[p] = (uint8_t)p;
    std::stable_sort(porder.begin(), porder.end(), [&](uint8_t x, uint8_t y) { return (pairs[x] >> 24) > (pairs[y] >> 24); });
    if (t.shape == HP_HEX) return out;
    std::memcpy(&out[L.pairs], pairs.data(), 4 * pairs.size());
    std::memcpy(&out[L.valid], valid.data(), 4 * valid.size());
    std::memcpy(&out[L.poff], poff.data(), 2 * poff.size());
    std::memcpy(&out[L.porder], porder.data(), porder.size());
    return out;
}

// Reduced rule (reading of the quadrature option): Q - 1 Gauss-Radau-Jacobi
// points in the collapsed directions, which integrate degree 2Q - 4 = 2P
// exactly against their Jacobi weight, the Gauss-Lobatto-Legendre Q points
// elsewhere.
void rule_points(int shape, int P, int rq, std::vector<double> z[3], std::vector<double> w[3]) {
    const int Q = P + 2, Qc = rq ? Q - 1 : Q;
    std::vector<double> gx, gw, r1x, r1w, r2x, r2w;
    gll_rule(Q, gx, gw);
    grj_rule(Qc, 1, r1x, r1w);
    for (double& v : r1w) v *= 0.5;
    grj_rule(Qc, 2, r2x, r2w);
    for (double& v : r2w) v *= 0.25;
    z[0] = gx; w[0] = gw;
    z[1] = gx; w[1] = gw;
    z[2] = gx; w[2] = gw;
    if (shape == HP_PRISM) { z[2] = r1x; w[2] = r1w; }
    if (shape == HP_PYR) { z[2] = r2x; w[2] = r2w; }
    if (shape == HP_TET) { z[1] = r1x; w[1] = r1w; z[2] = r2x; w[2] = r2w; }
}

int n_points(int shape, int P, int rq) {
    const int Q = P + 2;
    if (!rq || shape == HP_HEX) return Q * Q * Q;
    return shape == HP_TET ? Q * (Q - 1) * (Q - 1) : Q * Q * (Q - 1);
}

std::vector<double> dense_matrices_rq(int shape, int P) {
    // B at the reduced rule's points from the 1-D factors, then D_d B with the
    // Lagrange derivatives of each direction's points (exact: every factor has
    // degree <= P below the direction's point count)
    const RefTables& t = ref_tables(shape, P);
    std::vector<double> z[3], w[3];
    rule_points(shape, P, 1, z, w);
    const int n = t.n, NP = t.NP;
    const int q1 = (int)z[0].size(), q2 = (int)z[1].size(), q3 = (int)z[2].size(), NQ = q1 * q2 * q3;
    std::vector<double> A(4 * (size_t)NQ * NP, 0.0);
    for (int m = 0; m < NP; ++m)
        for (int q = 0; q < 4; ++q) {
            const int sl = t.mode_slots[m * 4 + q];
            if (sl < 0) continue;
            const int a = sl / (n * n), b = (sl / n) % n, c = sl % n;
            const int tb = t.famb[a], sc = t.famc[a * n + b];
            for (int i = 0; i < q1; ++i)
                for (int j = 0; j < q2; ++j)
                    for (int k = 0; k < q3; ++k)
                        A[((size_t)((i * q2 + j) * q3 + k)) * NP + m] +=
                            family(P, 0, a, z[0][i]) * family(P, tb, b, z[1][j]) * family(P, sc, c, z[2][k]);
        }
    const int qd[3] = {q1, q2, q3};
    for (int d = 0; d < 3; ++d) {
        const std::vector<double> D = lagrange_d(z[d]);
        const int qq = qd[d];
        for (int i = 0; i < q1; ++i)
            for (int j = 0; j < q2; ++j)
                for (int k = 0; k < q3; ++k) {
                    const int l = (i * q2 + j) * q3 + k, own = d == 0 ? i : d == 1 ? j : k;
                    for (int mm = 0; mm < qq; ++mm) {
                        const int src = d == 0 ? (mm * q2 + j) * q3 + k : d == 1 ? (i * q2 + mm) * q3 + k : (i * q2 + j) * q3 + mm;
                        const double dv = D[own * qq + mm];
                        const double* from = &A[(size_t)src * NP];
                        double* to = &A[((size_t)(d + 1) * NQ + l) * NP];
                        for (int m = 0; m < NP; ++m) to[m] += dv * from[m];
                    }
                }
    }
    return A;
}

}  // namespace hp
