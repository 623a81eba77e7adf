// C0 global numbering of the modal bases on a conforming mesh (the assembled
// problem behind the paper's Helmholtz weak form, Sec. 2.1: one global
// function per vertex, per edge mode, per face mode, plus element interiors).
//
// Each element's modes are classified by where they live (vertex, edge, face,
// interior) by evaluating them near the reference vertices, edges and faces.
// Every edge and face of the mesh has a canonical basis defined from the global
// vertex ids: edges psi_n(s), s from the smaller to the larger id; quad faces
// psi_p(s) psi_q(t) with the origin at the smallest id and s towards its
// smaller-id neighbour; triangles psi_p(a) W_{p,q}(b) with the collapse at the
// largest id and a from the smallest to the middle id.  An element's trace
// modes on an edge or face are matched numerically to that canonical basis
// (a signed permutation when the local orientation is conforming: triangle
// collapse vertices at the largest id); the matches depend only on (shape,
// local entity, permutation of its vertex ids) and are cached.  Boundary DOFs
// are those on faces that belong to one element.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "hp_internal.h"

namespace hp {
namespace {

const double kRefV[4][8][3] = {
    {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1}, {-1, -1, 1}, {1, -1, 1}, {1, 1, 1}, {-1, 1, 1}},
    {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1}, {-1, -1, 1}, {-1, 1, 1}},
    {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1}, {-1, -1, 1}},
    {{-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}}};
const int kNVert[4] = {8, 6, 5, 4};

struct Topo {
    std::vector<std::array<int, 2>> edges;
    std::vector<std::vector<int>> faces;   // cyclic vertex order
};

const Topo& topo(int shape) {
    static Topo t[4];
    static std::once_flag once;
    std::call_once(once, [] {
        t[HP_HEX].edges = {{0, 1}, {1, 2}, {3, 2}, {0, 3}, {4, 5}, {5, 6}, {7, 6}, {4, 7}, {0, 4}, {1, 5}, {2, 6}, {3, 7}};
        t[HP_HEX].faces = {{0, 1, 2, 3}, {4, 5, 6, 7}, {0, 1, 5, 4}, {1, 2, 6, 5}, {3, 2, 6, 7}, {0, 3, 7, 4}};
        t[HP_PRISM].edges = {{0, 1}, {1, 2}, {3, 2}, {0, 3}, {0, 4}, {1, 4}, {3, 5}, {2, 5}, {4, 5}};
        t[HP_PRISM].faces = {{0, 1, 4}, {3, 2, 5}, {0, 1, 2, 3}, {0, 3, 5, 4}, {1, 2, 5, 4}};
        t[HP_PYR].edges = {{0, 1}, {1, 2}, {3, 2}, {0, 3}, {0, 4}, {1, 4}, {2, 4}, {3, 4}};
        t[HP_PYR].faces = {{0, 1, 2, 3}, {0, 1, 4}, {1, 2, 4}, {2, 3, 4}, {3, 0, 4}};
        t[HP_TET].edges = {{0, 1}, {1, 2}, {0, 2}, {0, 3}, {1, 3}, {2, 3}};
        t[HP_TET].faces = {{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {0, 2, 3}};
    });
    return t[shape];
}

// reference point from vertex weights, nudged towards the centroid so that no
// sample sits on a collapse point of the eta map
void point_from_weights(int shape, const std::vector<int>& lv, const std::vector<double>& w, double* xi) {
    double c[3] = {0, 0, 0};
    for (int v = 0; v < kNVert[shape]; ++v)
        for (int d = 0; d < 3; ++d) c[d] += kRefV[shape][v][d] / kNVert[shape];
    for (int d = 0; d < 3; ++d) {
        double x = 0;
        for (size_t i = 0; i < lv.size(); ++i) x += w[i] * kRefV[shape][lv[i]][d];
        xi[d] = x + 1e-9 * (c[d] - x);
    }
}

// ---------------------------------------------------------------- mode classes
struct Classes {
    std::vector<int> kind;        // 0 vertex, 1 edge, 2 face, 3 interior
    std::vector<int> entity;      // vertex / edge / face index
    std::vector<std::vector<int>> edge_modes, face_modes, vertex_mode;
};

Classes classify(int shape, int P) {
    const Topo& T = topo(shape);
    const int NP = n_modes(shape, P);
    Classes C;
    C.kind.assign(NP, 3);
    C.entity.assign(NP, -1);
    std::vector<double> val(NP);
    const double tol = 1e-6;
    auto eval = [&](const std::vector<int>& lv, const std::vector<double>& w) {
        double xi[3];
        point_from_weights(shape, lv, w, xi);
        eval_modes(shape, P, xi, val.data());
    };
    // vertices
    C.vertex_mode.assign(kNVert[shape], {});
    for (int v = 0; v < kNVert[shape]; ++v) {
        eval({v}, {1.0});
        for (int m = 0; m < NP; ++m)
            if (std::fabs(val[m] - 1.0) < tol) {
                C.kind[m] = 0;
                C.entity[m] = v;
                C.vertex_mode[v].push_back(m);
            }
    }
    auto nonzero_on = [&](const std::vector<int>& lv, const std::vector<std::vector<double>>& ws) {
        std::vector<char> nz(NP, 0);
        for (const auto& w : ws) {
            eval(lv, w);
            for (int m = 0; m < NP; ++m)
                if (std::fabs(val[m]) > tol) nz[m] = 1;
        }
        return nz;
    };
    C.edge_modes.assign(T.edges.size(), {});
    for (size_t e = 0; e < T.edges.size(); ++e) {
        std::vector<int> lv = {T.edges[e][0], T.edges[e][1]};
        auto nz = nonzero_on(lv, {{0.83, 0.17}, {0.41, 0.59}, {0.22, 0.78}});
        for (int m = 0; m < NP; ++m)
            if (nz[m] && C.kind[m] == 3) {
                C.kind[m] = 1;
                C.entity[m] = (int)e;
                C.edge_modes[e].push_back(m);
            }
    }
    C.face_modes.assign(T.faces.size(), {});
    for (size_t f = 0; f < T.faces.size(); ++f) {
        const auto& lv = T.faces[f];
        std::vector<std::vector<double>> ws;
        if (lv.size() == 4) ws = {{0.31, 0.24, 0.19, 0.26}, {0.1, 0.4, 0.3, 0.2}, {0.45, 0.05, 0.35, 0.15}};
        else ws = {{0.2, 0.3, 0.5}, {0.6, 0.25, 0.15}, {0.15, 0.7, 0.15}};
        auto nz = nonzero_on(lv, ws);
        for (int m = 0; m < NP; ++m)
            if (nz[m] && C.kind[m] == 3) {
                C.kind[m] = 2;
                C.entity[m] = (int)f;
                C.face_modes[f].push_back(m);
            }
    }
    return C;
}

// ---------------------------------------------------------------- matching
struct Match {
    bool ok = false;
    std::vector<int> mode, canon;   // local mode -> canonical index
    std::vector<int> sign;
};

double psi(int P, int n, double z) { return family_value(P, 0, n + 1, z); }   // bubble n >= 1

// Canonical functions of an entity at sample points; the sample points' vertex
// weights are given in canonical vertex order.
void canonical_samples(int P, int kind, std::vector<std::vector<double>>& W, std::vector<std::vector<double>>& F) {
    W.clear();
    F.clear();
    const int K = P + 3;
    std::vector<double> z(K);
    for (int k = 0; k < K; ++k) z[k] = -std::cos((k + 0.37) * 3.14159265358979 / (K + 0.1));
    if (kind == 0) {   // edge: s from canonical vertex 0 to 1
        for (int k = 0; k < K; ++k) {
            double s = z[k];
            W.push_back({0.5 * (1 - s), 0.5 * (1 + s)});
            std::vector<double> f;
            for (int n = 1; n < P; ++n) f.push_back(psi(P, n, s));
            F.push_back(f);
        }
    } else if (kind == 1) {   // quad: canonical vertices o, s-neighbour, opposite, t-neighbour (cyclic)
        for (int a = 0; a < K; ++a)
            for (int b = 0; b < K; ++b) {
                double s = z[a], t = z[(b * 3 + 1) % K] * 0.97;
                W.push_back({0.25 * (1 - s) * (1 - t), 0.25 * (1 + s) * (1 - t), 0.25 * (1 + s) * (1 + t),
                             0.25 * (1 - s) * (1 + t)});
                std::vector<double> f;
                for (int p = 1; p < P; ++p)
                    for (int q = 1; q < P; ++q) f.push_back(psi(P, p, s) * psi(P, q, t));
                F.push_back(f);
            }
    } else {   // triangle: canonical vertices A (smallest id), B, C (collapse, largest id)
        for (int i = 0; i < K; ++i)
            for (int j = 0; j < K; ++j) {
                double a = z[i], b = z[(j * 3 + 2) % K] * 0.95;
                double x1 = 0.5 * (1 + a) * (1 - b) - 1, x2 = b;
                double lb = 0.5 * (1 + x1), lc = 0.5 * (1 + x2), la = 1 - lb - lc;
                W.push_back({la, lb, lc});
                std::vector<double> f;
                for (int p = 1; p < P; ++p)
                    for (int q = 1; p + q < P; ++q) f.push_back(psi(P, p, a) * family_value(P, p, q, b));
                F.push_back(f);
            }
    }
}

Match match_entity(int shape, int P, int kind, const std::vector<int>& local_verts_in_canon_order,
                   const std::vector<int>& modes) {
    Match M;
    std::vector<std::vector<double>> W, F;
    canonical_samples(P, kind, W, F);
    const int NP = n_modes(shape, P);
    const size_t K = W.size(), nc = F.empty() ? 0 : F[0].size();
    if (nc != modes.size()) return M;
    std::vector<double> val(NP), tr(K * modes.size());
    for (size_t k = 0; k < K; ++k) {
        double xi[3];
        point_from_weights(shape, local_verts_in_canon_order, W[k], xi);
        eval_modes(shape, P, xi, val.data());
        for (size_t i = 0; i < modes.size(); ++i) tr[k * modes.size() + i] = val[modes[i]];
    }
    std::vector<char> used(nc, 0);
    for (size_t i = 0; i < modes.size(); ++i) {
        int best = -1;
        double best_sign = 0;
        for (size_t j = 0; j < nc; ++j) {
            double dp = 0, dm = 0, ref = 0;
            for (size_t k = 0; k < K; ++k) {
                double t = tr[k * modes.size() + i], c = F[k][j];
                dp = std::max(dp, std::fabs(t - c));
                dm = std::max(dm, std::fabs(t + c));
                ref = std::max(ref, std::fabs(c));
            }
            if (dp < 1e-6 * std::max(ref, 1e-3)) { best = (int)j; best_sign = 1; break; }
            if (dm < 1e-6 * std::max(ref, 1e-3)) { best = (int)j; best_sign = -1; break; }
        }
        if (best < 0 || used[best]) return M;
        used[best] = 1;
        M.mode.push_back(modes[i]);
        M.canon.push_back(best);
        M.sign.push_back((int)best_sign);
    }
    M.ok = true;
    return M;
}

std::mutex g_mu;
std::map<std::vector<int>, Classes> g_classes;
std::map<std::vector<int>, Match> g_matches;

const Classes& classes_of(int shape, int P) {
    std::vector<int> key = {shape, P};
    auto it = g_classes.find(key);
    if (it == g_classes.end()) it = g_classes.emplace(key, classify(shape, P)).first;
    return it->second;
}

const Match& match_of(int shape, int P, int kind, int ent, const std::vector<int>& lv_canon,
                      const std::vector<int>& modes) {
    std::vector<int> key = {shape, P, kind, ent};
    key.insert(key.end(), lv_canon.begin(), lv_canon.end());
    auto it = g_matches.find(key);
    if (it == g_matches.end()) it = g_matches.emplace(key, match_entity(shape, P, kind, lv_canon, modes)).first;
    return it->second;
}

// integer key of (shape, entity kind, local entity, canonical local vertex
// order): 2 + 2 + 4 bits, then up to four 3-bit vertex ids and their count
uint32_t match_key(int shape, int kind, int ent, const int* lv, int n) {
    uint32_t k = (uint32_t)shape | ((uint32_t)kind << 2) | ((uint32_t)ent << 4) | ((uint32_t)n << 8);
    for (int i = 0; i < n; ++i) k |= (uint32_t)lv[i] << (11 + 3 * i);
    return k;
}

struct ArrHash {
    size_t operator()(const std::array<int64_t, 4>& a) const {
        uint64_t h = 1469598103934665603ull;
        for (int64_t v : a) {
            h ^= (uint64_t)v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
            h *= 1099511628211ull;
        }
        return (size_t)h;
    }
};

// Open-addressing hash map from up to four int64 ids to the index of first
// insertion (linear probing, capacity a power of two, at most half full):
// entities are numbered in order of first appearance, as with any map.
class EntityMap {
public:
    explicit EntityMap(size_t expect) { rehash(std::max<size_t>(64, 2 * expect)); }
    int64_t size() const { return n_; }
    // index of `k`, inserting it with the next index when absent; *fresh tells which
    int64_t find_or_insert(const std::array<int64_t, 4>& k, bool* fresh) {
        if (2 * (n_ + 1) > cap_) rehash(2 * cap_);
        size_t i = slot(k);
        while (used_[i]) {
            if (keys_[i] == k) { *fresh = false; return vals_[i]; }
            i = (i + 1) & (cap_ - 1);
        }
        used_[i] = 1;
        keys_[i] = k;
        vals_[i] = n_;
        *fresh = true;
        return n_++;
    }

private:
    size_t slot(const std::array<int64_t, 4>& k) const { return ArrHash()(k) & (cap_ - 1); }
    void rehash(size_t want) {
        size_t c = 64;
        while (c < want) c <<= 1;
        std::vector<std::array<int64_t, 4>> ok = std::move(keys_);
        std::vector<int64_t> ov = std::move(vals_);
        std::vector<uint8_t> ou = std::move(used_);
        cap_ = c;
        keys_.assign(cap_, {});
        vals_.assign(cap_, 0);
        used_.assign(cap_, 0);
        for (size_t j = 0; j < ou.size(); ++j)
            if (ou[j]) {
                size_t i = slot(ok[j]);
                while (used_[i]) i = (i + 1) & (cap_ - 1);
                used_[i] = 1;
                keys_[i] = ok[j];
                vals_[i] = ov[j];
            }
    }
    size_t cap_ = 0;
    int64_t n_ = 0;
    std::vector<std::array<int64_t, 4>> keys_;
    std::vector<int64_t> vals_;
    std::vector<uint8_t> used_;
};

}  // namespace

// Build the map; see the header of this file.  Fills gid/sign (per local
// coefficient), boundary (per global DOF) and returns the global count.
hp_status build_c0(const hp_mesh m, const std::vector<int64_t>& vert, std::vector<int64_t>& gid,
                   std::vector<int8_t>& sign, std::vector<uint8_t>& boundary, int64_t& n_global) {
    std::lock_guard<std::mutex> lk(g_mu);
    const int64_t ne = m->n_elem;
    const int P = m->P[0];
    for (int64_t e = 0; e < ne; ++e)
        if (m->P[e] != P) {
            set_error("hp_c0_create: the C0 map needs one order P on all elements");
            return HP_ERR_UNSUPPORTED;
        }
    const int64_t n_local = m->coeff_off.back();
    gid.assign(n_local, -1);
    sign.assign(n_local, 1);
    // entity numbering
    EntityMap vmap((size_t)ne * 2), emap((size_t)ne * 4), fmap((size_t)ne * 4);
    std::vector<int> fcount;
    std::vector<int> ftype;    // 0 quad, 1 tri
    // per local coefficient: (class 0..3, entity index, canonical index)
    std::vector<int8_t> lclass(n_local, 3);
    std::vector<int64_t> lent(n_local, -1);
    std::vector<int32_t> lcan(n_local, 0);
    int64_t n_interior = 0;
    // per call: the classes of each shape and the matches seen so far by integer key
    // (the shared caches are keyed by vectors in ordered maps, slow for every element)
    const Classes* cls[4] = {nullptr, nullptr, nullptr, nullptr};
    std::unordered_map<uint32_t, const Match*> fast;
    auto match_fast = [&](int s, int kind, int ent, const int* lv, int n, const std::vector<int>& modes) -> const Match& {
        const uint32_t k = match_key(s, kind, ent, lv, n);
        auto it = fast.find(k);
        if (it != fast.end()) return *it->second;
        const Match& M = match_of(s, P, kind, ent, std::vector<int>(lv, lv + n), modes);
        fast.emplace(k, &M);
        return M;
    };
    // face index of (element, local face), for the boundary pass
    std::vector<int64_t> elem_face((size_t)ne * 6, -1);
    for (int64_t e = 0; e < ne; ++e) {
        const int s = m->shape[e];
        if (!cls[s]) cls[s] = &classes_of(s, P);
        const Classes& C = *cls[s];
        const Topo& T = topo(s);
        const int64_t base = m->coeff_off[e];
        const int64_t* g = &vert[e * 8];
        for (int v = 0; v < kNVert[s]; ++v) {
            if (C.vertex_mode[v].size() != 1) { set_error("hp_c0_create: vertex mode classification failed"); return HP_ERR_UNSUPPORTED; }
            bool fresh;
            const int64_t vi = vmap.find_or_insert({g[v], -1, -1, -1}, &fresh);
            int mm = C.vertex_mode[v][0];
            lclass[base + mm] = 0;
            lent[base + mm] = vi;
        }
        for (size_t ed = 0; ed < T.edges.size(); ++ed) {
            int la = T.edges[ed][0], lb = T.edges[ed][1];
            if (g[la] > g[lb]) std::swap(la, lb);
            bool fresh;
            const int64_t ei = emap.find_or_insert({g[la], g[lb], -1, -1}, &fresh);
            const int lvq[2] = {la, lb};
            const Match& M = match_fast(s, 0, (int)ed, lvq, 2, C.edge_modes[ed]);
            if (!M.ok) { set_error("hp_c0_create: edge trace is not a signed permutation"); return HP_ERR_UNSUPPORTED; }
            for (size_t i = 0; i < M.mode.size(); ++i) {
                lclass[base + M.mode[i]] = 1;
                lent[base + M.mode[i]] = ei;
                lcan[base + M.mode[i]] = M.canon[i];
                sign[base + M.mode[i]] = (int8_t)M.sign[i];
            }
        }
        for (size_t f = 0; f < T.faces.size(); ++f) {
            const auto& lvf = T.faces[f];
            int canon[4];
            const int nfv = (int)lvf.size();
            std::array<int64_t, 4> key = {-1, -1, -1, -1};
            if (nfv == 3) {
                for (int i = 0; i < 3; ++i) canon[i] = lvf[i];
                std::sort(canon, canon + 3, [&](int x, int y) { return g[x] < g[y]; });
                for (int i = 0; i < 3; ++i) key[i] = g[canon[i]];
            } else {
                int o = 0;
                for (int i = 1; i < 4; ++i)
                    if (g[lvf[i]] < g[lvf[o]]) o = i;
                int nA = lvf[(o + 1) % 4], nB = lvf[(o + 3) % 4];
                int sN = g[nA] < g[nB] ? nA : nB, tN = g[nA] < g[nB] ? nB : nA;
                canon[0] = lvf[o]; canon[1] = sN; canon[2] = lvf[(o + 2) % 4]; canon[3] = tN;
                std::array<int64_t, 4> ids = {g[lvf[0]], g[lvf[1]], g[lvf[2]], g[lvf[3]]};
                std::sort(ids.begin(), ids.end());
                key = ids;
            }
            bool fresh;
            const int64_t fi = fmap.find_or_insert(key, &fresh);
            if (fresh) {
                fcount.push_back(0);
                ftype.push_back(nfv == 3 ? 1 : 0);
            }
            fcount[fi] += 1;
            elem_face[(size_t)e * 6 + f] = fi;
            const Match& M = match_fast(s, nfv == 3 ? 2 : 1, (int)f, canon, nfv, C.face_modes[f]);
            if (!M.ok) {
                set_error("hp_c0_create: face trace is not a signed permutation (triangle faces need their "
                          "collapsed vertex at the largest global id)");
                return HP_ERR_UNSUPPORTED;
            }
            for (size_t i = 0; i < M.mode.size(); ++i) {
                lclass[base + M.mode[i]] = 2;
                lent[base + M.mode[i]] = fi;
                lcan[base + M.mode[i]] = M.canon[i];
                sign[base + M.mode[i]] = (int8_t)M.sign[i];
            }
        }
        for (int64_t mm = 0; mm < m->coeff_off[e + 1] - base; ++mm)
            if (lclass[base + mm] == 3) lent[base + mm] = n_interior++;
    }
    for (int c : fcount)
        if (c > 2) { set_error("hp_c0_create: a face is shared by more than two elements"); return HP_ERR_GEOM; }
    // global layout: vertices, edges, faces (each with its own size), interiors
    const int64_t nv = vmap.size(), nedge = emap.size(), nface = fmap.size();
    const int per_edge = P - 1, per_quad = (P - 1) * (P - 1), per_tri = (P - 1) * (P - 2) / 2;
    std::vector<int64_t> face_base(nface + 1, 0);
    for (int64_t f = 0; f < nface; ++f) face_base[f + 1] = face_base[f] + (ftype[f] ? per_tri : per_quad);
    const int64_t off_e = nv, off_f = nv + nedge * per_edge, off_i = off_f + face_base[nface];
    n_global = off_i + n_interior;
    for (int64_t i = 0; i < n_local; ++i) {
        switch (lclass[i]) {
            case 0: gid[i] = lent[i]; break;
            case 1: gid[i] = off_e + lent[i] * per_edge + lcan[i]; break;
            case 2: gid[i] = off_f + face_base[lent[i]] + lcan[i]; break;
            default: gid[i] = off_i + lent[i];
        }
    }
    // boundary: everything on faces that belong to one element
    boundary.assign(n_global, 0);
    for (int64_t e = 0; e < ne; ++e) {
        const int s = m->shape[e];
        const Topo& T = topo(s);
        const Classes& C = *cls[s];
        const int64_t base = m->coeff_off[e];
        for (size_t f = 0; f < T.faces.size(); ++f) {
            const auto& lvf = T.faces[f];
            if (fcount[elem_face[(size_t)e * 6 + f]] != 1) continue;
            for (int mm : C.face_modes[f]) boundary[gid[base + mm]] = 1;
            for (int v : lvf) boundary[gid[base + C.vertex_mode[v][0]]] = 1;
            for (size_t ed = 0; ed < T.edges.size(); ++ed) {
                int la = T.edges[ed][0], lb = T.edges[ed][1];
                if (std::find(lvf.begin(), lvf.end(), la) != lvf.end() && std::find(lvf.begin(), lvf.end(), lb) != lvf.end())
                    for (int mm : C.edge_modes[ed]) boundary[gid[base + mm]] = 1;
            }
        }
    }
    return HP_OK;
}

}  // namespace hp
