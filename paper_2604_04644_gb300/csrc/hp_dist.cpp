// Host side of the multi-GPU layout (no CUDA): element partitions balanced by
// predicted cost, the halo plan of the assembled solve (the sum over the
// interface DOFs that partitions share), and exact dot products whose
// cross-rank reduction is an integer sum.
//
// The element-local operators of Sec. 2 need no exchange: a partition of the
// elements is a partition of the work.  The assembled problem
// (grad u, grad v) + lambda (u, v) = (f, v) of Sec. 2.1 couples elements
// through shared global DOFs; each CG iteration then needs one halo sum
// (local copies of each interface DOF reduced to its owner, the owner's value
// sent back to every rank that holds a copy) and two dot products.
//
// Reproducibility by construction:
// - the owner adds the copies of each DOF, its own and the received ones, in
//   the single-rank order (increasing index in the single-rank local
//   coefficient layout, starting from 0), so an assembled entry has the same
//   bits as the one-rank assembly (hp_c0_assemble) for any partition;
// - dot products accumulate each product x_i y_i exactly (its rounded value
//   and the rounding error from one FMA) into a fixed-point accumulator of
//   32-bit limbs spanning the whole double range, and ranks add their
//   accumulators as integers; the sum is exact and rounded once, so it does
//   not depend on the partition or on the order of the terms.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "hp_internal.h"

using namespace hp;

namespace {

constexpr int kLimbs = 68;   // 68 x 32 bits from 2^-1074: every finite double and 2^31 carries of headroom

// -------------------------------------------------------------- exact accumulator
void xacc_normalise(int64_t* a) {
    for (int j = 0; j < kLimbs - 1; ++j) {
        const int64_t c = a[j] >> 32;   // floor division by 2^32
        a[j] -= c * ((int64_t)1 << 32);
        a[j + 1] += c;
    }
}

void xacc_add(int64_t* a, double d) {
    if (d == 0.0 || !std::isfinite(d)) return;
    int E = 0;
    const double f = std::frexp(d, &E);                 // d = f 2^E, 0.5 <= |f| < 1
    int64_t M = (int64_t)std::ldexp(f, 53);              // exact: 53-bit integer
    int B = E - 53 + 1074;                               // bit offset of M's least bit above 2^-1074
    if (B < 0) {                                         // subnormal: M has -B trailing zero bits
        M /= ((int64_t)1 << (-B));
        B = 0;
    }
    const bool neg = M < 0;
    const unsigned __int128 v = (unsigned __int128)(uint64_t)(neg ? -M : M) << (B & 31);
    const int j = B >> 5;
    const int64_t p0 = (int64_t)(uint64_t)(v & 0xffffffffu), p1 = (int64_t)(uint64_t)((v >> 32) & 0xffffffffu),
                  p2 = (int64_t)(uint64_t)(v >> 64);
    if (neg) { a[j] -= p0; a[j + 1] -= p1; a[j + 2] -= p2; }
    else { a[j] += p0; a[j + 1] += p1; a[j + 2] += p2; }
}

// the accumulated value rounded to the nearest double (ties to even)
double xacc_round(const int64_t* in) {
    int64_t a[kLimbs];
    std::memcpy(a, in, sizeof(a));
    xacc_normalise(a);
    const bool neg = a[kLimbs - 1] < 0;
    if (neg) {
        for (int j = 0; j < kLimbs; ++j) a[j] = -a[j];
        xacc_normalise(a);
    }
    int h = kLimbs - 1;
    while (h >= 0 && a[h] == 0) --h;
    if (h < 0) return 0.0;
    const int lo = h >= 2 ? h - 2 : 0;
    unsigned __int128 m = 0;
    for (int j = h; j >= lo; --j) m = (m << 32) | (uint64_t)a[j];
    bool sticky = false;
    for (int j = 0; j < lo; ++j) sticky |= a[j] != 0;
    int nb = 0;
    for (unsigned __int128 t = m; t; t >>= 1) ++nb;
    int e = 32 * lo - 1074;                              // weight of m's least bit
    uint64_t q;
    if (nb <= 53) {
        q = (uint64_t)m;
    } else {
        const int sh = nb - 53;
        q = (uint64_t)(m >> sh);
        const unsigned __int128 rem = m & (((unsigned __int128)1 << sh) - 1), half = (unsigned __int128)1 << (sh - 1);
        if (rem > half || (rem == half && (sticky || (q & 1)))) ++q;
        e += sh;
    }
    const double r = std::ldexp((double)q, e);
    return neg ? -r : r;
}

}  // namespace

// ------------------------------------------------------------------ halo plan
struct hp_halo_s {
    int nparts = 1, rank = 0;
    std::vector<int64_t> local_index;        // [n_local] index in the single-rank coefficient layout
    std::vector<int64_t> touched_gid;        // [n_touched] global DOFs this rank holds copies of, ascending
    std::vector<int32_t> lmap;               // [n_local] touched index t (sign +) or ~t (sign -)
    std::vector<int64_t> owned_t;            // [n_owned] touched index of each owned DOF (ascending gid)
    std::vector<int64_t> rsend_off, rsend;   // reduce: per peer, rank-local coefficient indices (signed values sent)
    std::vector<int64_t> rrecv_off;          // reduce: per peer, values received
    std::vector<int64_t> asm_ptr, asm_src;   // owner sum: sources in single-rank order, index into [own | received]
    std::vector<int64_t> bsend_off, bsend;   // broadcast: per peer, owned indices
    std::vector<int64_t> brecv_off, brecv;   // broadcast: per peer, touched indices filled
};

extern "C" {

hp_status hp_partition(const hp_mesh_desc* d, const double* cost, int nparts, int method, int32_t* part) {
    if (!d || !part || d->n_elem < 1 || nparts < 1 || nparts > 65536 || (method != 0 && method != 1) || !d->shape ||
        !d->P || !d->curved || (method == 1 && (!d->vert || !d->xyz))) {
        set_error("hp_partition: bad argument");
        return HP_ERR_ARG;
    }
    const int64_t n = d->n_elem;
    std::vector<double> c(n);
    for (int64_t e = 0; e < n; ++e) {
        if (cost) c[e] = cost[e];
        else if (d->shape[e] > 3 || d->P[e] < 1 || d->P[e] > PMAX) { set_error("hp_partition: bad shape or order"); return HP_ERR_ARG; }
        else c[e] = elem_flops_helmholtz(d->shape[e], d->P[e]);   // the FP64 path is bound by its flops
        if (!(c[e] >= 0.0) || !std::isfinite(c[e])) { set_error("hp_partition: costs must be finite and >= 0"); return HP_ERR_ARG; }
    }
    std::vector<int64_t> order(n);
    std::iota(order.begin(), order.end(), 0);
    auto cut = [&](const std::vector<int64_t>& ord, int64_t b, int64_t en, int p0, int np) {
        // element ord[i] -> part p0 + floor(np * (prefix before it + half its cost) / total)
        double tot = 0;
        for (int64_t i = b; i < en; ++i) tot += c[ord[i]];
        double pre = 0;
        for (int64_t i = b; i < en; ++i) {
            const double mid = pre + 0.5 * c[ord[i]];
            int p = tot > 0 ? (int)std::floor(np * mid / tot) : (int)((i - b) * np / std::max<int64_t>(en - b, 1));
            part[ord[i]] = p0 + std::min(std::max(p, 0), np - 1);
            pre += c[ord[i]];
        }
    };
    if (method == 0) {
        // ranges of the block order: blocks of equal (shape, P, curved) in order
        // of first appearance, user order inside a block (the library's blocks)
        std::vector<int> key(n), first;
        std::map<int, int> rank_of;
        for (int64_t e = 0; e < n; ++e) {
            const int k = d->shape[e] * 4096 + d->P[e] * 2 + (d->curved[e] ? 1 : 0);
            auto it = rank_of.find(k);
            if (it == rank_of.end()) it = rank_of.emplace(k, (int)rank_of.size()).first;
            key[e] = it->second;
        }
        std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) { return key[x] < key[y]; });
        cut(order, 0, n, 0, nparts);
        return HP_OK;
    }
    // recursive coordinate bisection of the element centroids, cost-weighted:
    // each range of parts splits its elements along the axis of largest extent
    // at the cost fraction of its two halves of parts
    std::vector<double> X(3 * n, 0.0);
    for (int64_t e = 0; e < n; ++e) {
        int nv = 0;
        for (int v = 0; v < 8; ++v) {
            const int64_t id = d->vert[8 * e + v];
            if (id < 0) continue;
            if (id >= d->n_vert) { set_error("hp_partition: vertex id out of range"); return HP_ERR_ARG; }
            for (int i = 0; i < 3; ++i) X[3 * e + i] += d->xyz[3 * id + i];
            ++nv;
        }
        for (int i = 0; i < 3; ++i) X[3 * e + i] /= std::max(nv, 1);
    }
    struct Job { int64_t b, en; int p0, np; };
    std::vector<Job> st{{0, n, 0, nparts}};
    while (!st.empty()) {
        Job j = st.back();
        st.pop_back();
        if (j.np == 1) {
            for (int64_t i = j.b; i < j.en; ++i) part[order[i]] = j.p0;
            continue;
        }
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int64_t i = j.b; i < j.en; ++i)
            for (int a = 0; a < 3; ++a) {
                lo[a] = std::min(lo[a], X[3 * order[i] + a]);
                hi[a] = std::max(hi[a], X[3 * order[i] + a]);
            }
        int ax = 0;
        for (int a = 1; a < 3; ++a) if (hi[a] - lo[a] > hi[ax] - lo[ax]) ax = a;
        std::stable_sort(order.begin() + j.b, order.begin() + j.en, [&](int64_t x, int64_t y) {
            return X[3 * x + ax] < X[3 * y + ax] || (X[3 * x + ax] == X[3 * y + ax] && x < y);
        });
        const int nl = j.np / 2;
        double tot = 0;
        for (int64_t i = j.b; i < j.en; ++i) tot += c[order[i]];
        const double target = tot * nl / j.np;
        double pre = 0;
        int64_t m = j.b;
        while (m < j.en && pre + 0.5 * c[order[m]] < target) pre += c[order[m++]];
        st.push_back({m, j.en, j.p0 + nl, j.np - nl});
        st.push_back({j.b, m, j.p0, nl});
    }
    return HP_OK;
}

hp_status hp_halo_create(const int64_t* gid, const int8_t* sign, const int64_t* coeff_off, int64_t n_elem,
                         int64_t n_global, const int32_t* part, int nparts, int rank, hp_halo* out) {
    if (!gid || !sign || !coeff_off || !part || !out || n_elem < 1 || n_global < 1 || nparts < 1 || rank < 0 ||
        rank >= nparts) {
        set_error("hp_halo_create: bad argument");
        return HP_ERR_ARG;
    }
    *out = nullptr;
    const int64_t n_coeff = coeff_off[n_elem];
    // ranks holding a copy of each global DOF (sorted, unique) and each DOF's owner (the lowest)
    std::vector<std::vector<int32_t>> holders(n_global);
    for (int64_t e = 0; e < n_elem; ++e) {
        if (part[e] < 0 || part[e] >= nparts) { set_error("hp_halo_create: part id out of range"); return HP_ERR_ARG; }
        for (int64_t i = coeff_off[e]; i < coeff_off[e + 1]; ++i) {
            if (gid[i] < 0 || gid[i] >= n_global || (sign[i] != 1 && sign[i] != -1)) {
                set_error("hp_halo_create: gid or sign out of range");
                return HP_ERR_ARG;
            }
            auto& h = holders[gid[i]];
            if (std::find(h.begin(), h.end(), part[e]) == h.end()) h.push_back(part[e]);
        }
    }
    for (auto& h : holders) std::sort(h.begin(), h.end());
    auto H = new hp_halo_s();
    H->nparts = nparts;
    H->rank = rank;
    for (int64_t e = 0; e < n_elem; ++e)
        if (part[e] == rank)
            for (int64_t i = coeff_off[e]; i < coeff_off[e + 1]; ++i) H->local_index.push_back(i);
    const int64_t nl = (int64_t)H->local_index.size();
    // touched DOFs and the local -> touched map
    for (int64_t g = 0; g < n_global; ++g)
        if (std::binary_search(holders[g].begin(), holders[g].end(), rank)) H->touched_gid.push_back(g);
    std::vector<int64_t> tpos(n_global, -1);
    for (size_t t = 0; t < H->touched_gid.size(); ++t) tpos[H->touched_gid[t]] = (int64_t)t;
    H->lmap.resize(nl);
    for (int64_t i = 0; i < nl; ++i) {
        const int64_t li = H->local_index[i], t = tpos[gid[li]];
        H->lmap[i] = sign[li] > 0 ? (int32_t)t : ~(int32_t)t;
    }
    for (size_t t = 0; t < H->touched_gid.size(); ++t)
        if (holders[H->touched_gid[t]][0] == rank) H->owned_t.push_back((int64_t)t);
    // copies of every DOF in single-rank local order, with their rank and rank-local index
    std::vector<int64_t> rank_local(n_coeff, -1);
    {
        std::vector<int64_t> cnt(nparts, 0);
        for (int64_t e = 0; e < n_elem; ++e)
            for (int64_t i = coeff_off[e]; i < coeff_off[e + 1]; ++i) rank_local[i] = cnt[part[e]]++;
    }
    std::vector<int32_t> rank_of_coeff(n_coeff);
    for (int64_t e = 0; e < n_elem; ++e)
        for (int64_t i = coeff_off[e]; i < coeff_off[e + 1]; ++i) rank_of_coeff[i] = part[e];
    std::vector<int64_t> rowptr(n_global + 1, 0), col(n_coeff);
    for (int64_t i = 0; i < n_coeff; ++i) rowptr[gid[i] + 1]++;
    for (int64_t g = 0; g < n_global; ++g) rowptr[g + 1] += rowptr[g];
    {
        std::vector<int64_t> fill(rowptr.begin(), rowptr.end() - 1);
        for (int64_t i = 0; i < n_coeff; ++i) col[fill[gid[i]]++] = i;
    }
    // reduce messages: rank q sends to owner o its copies of every DOF o owns
    // that q holds, ordered by (gid, single-rank local index); this rank's side
    H->rsend_off.assign(nparts + 1, 0);
    H->rrecv_off.assign(nparts + 1, 0);
    std::vector<std::vector<int64_t>> rs(nparts);
    std::vector<int64_t> recv_cnt(nparts, 0);
    for (int64_t g = 0; g < n_global; ++g) {
        const int owner = holders[g][0];
        for (int64_t k = rowptr[g]; k < rowptr[g + 1]; ++k) {
            const int64_t li = col[k];
            const int q = rank_of_coeff[li];
            if (q == owner) continue;
            if (q == rank) rs[owner].push_back(rank_local[li]);
            if (owner == rank) recv_cnt[q]++;
        }
    }
    for (int q = 0; q < nparts; ++q) {
        H->rsend_off[q + 1] = H->rsend_off[q] + (int64_t)rs[q].size();
        H->rrecv_off[q + 1] = H->rrecv_off[q] + recv_cnt[q];
        H->rsend.insert(H->rsend.end(), rs[q].begin(), rs[q].end());
    }
    // owner sums: sources in single-rank order; own copies index [0, nl), copies
    // received from q index nl + rrecv_off[q] + (their position in q's message)
    std::vector<int64_t> rpos(nparts, 0);
    H->asm_ptr.assign(1, 0);
    for (int64_t t : H->owned_t) {
        const int64_t g = H->touched_gid[t];
        for (int64_t k = rowptr[g]; k < rowptr[g + 1]; ++k) {
            const int64_t li = col[k];
            const int q = rank_of_coeff[li];
            H->asm_src.push_back(q == rank ? rank_local[li] : nl + H->rrecv_off[q] + rpos[q]++);
        }
        H->asm_ptr.push_back((int64_t)H->asm_src.size());
    }
    // broadcast: the owner sends each owned DOF's value to every other holder, ascending gid
    H->bsend_off.assign(nparts + 1, 0);
    H->brecv_off.assign(nparts + 1, 0);
    std::vector<std::vector<int64_t>> bs(nparts), br(nparts);
    for (size_t o = 0; o < H->owned_t.size(); ++o) {
        const auto& h = holders[H->touched_gid[H->owned_t[o]]];
        for (size_t x = 1; x < h.size(); ++x) bs[h[x]].push_back((int64_t)o);
    }
    for (size_t t = 0; t < H->touched_gid.size(); ++t) {
        const auto& h = holders[H->touched_gid[t]];
        if (h[0] != rank) br[h[0]].push_back((int64_t)t);
    }
    for (int q = 0; q < nparts; ++q) {
        H->bsend_off[q + 1] = H->bsend_off[q] + (int64_t)bs[q].size();
        H->brecv_off[q + 1] = H->brecv_off[q] + (int64_t)br[q].size();
        H->bsend.insert(H->bsend.end(), bs[q].begin(), bs[q].end());
        H->brecv.insert(H->brecv.end(), br[q].begin(), br[q].end());
    }
    *out = H;
    return HP_OK;
}

hp_status hp_halo_info(hp_halo h, int64_t* n_local, int64_t* n_touched, int64_t* n_owned) {
    if (!h) { set_error("hp_halo_info: null handle"); return HP_ERR_ARG; }
    if (n_local) *n_local = (int64_t)h->local_index.size();
    if (n_touched) *n_touched = (int64_t)h->touched_gid.size();
    if (n_owned) *n_owned = (int64_t)h->owned_t.size();
    return HP_OK;
}

hp_status hp_halo_counts(hp_halo h, int64_t* reduce_send, int64_t* reduce_recv, int64_t* bcast_send,
                         int64_t* bcast_recv) {
    if (!h) { set_error("hp_halo_counts: null handle"); return HP_ERR_ARG; }
    for (int q = 0; q < h->nparts; ++q) {
        if (reduce_send) reduce_send[q] = h->rsend_off[q + 1] - h->rsend_off[q];
        if (reduce_recv) reduce_recv[q] = h->rrecv_off[q + 1] - h->rrecv_off[q];
        if (bcast_send) bcast_send[q] = h->bsend_off[q + 1] - h->bsend_off[q];
        if (bcast_recv) bcast_recv[q] = h->brecv_off[q + 1] - h->brecv_off[q];
    }
    return HP_OK;
}

hp_status hp_halo_maps(hp_halo h, int64_t* local_index, int64_t* touched_gid, int64_t* owned_gid) {
    if (!h) { set_error("hp_halo_maps: null handle"); return HP_ERR_ARG; }
    if (local_index) std::copy(h->local_index.begin(), h->local_index.end(), local_index);
    if (touched_gid) std::copy(h->touched_gid.begin(), h->touched_gid.end(), touched_gid);
    if (owned_gid)
        for (size_t o = 0; o < h->owned_t.size(); ++o) owned_gid[o] = h->touched_gid[h->owned_t[o]];
    return HP_OK;
}

hp_status hp_halo_gather(hp_halo h, const double* touched, double* local) {
    if (!h || !touched || !local) { set_error("hp_halo_gather: null argument"); return HP_ERR_ARG; }
    for (size_t i = 0; i < h->lmap.size(); ++i) {
        const int32_t t = h->lmap[i];
        local[i] = t >= 0 ? touched[t] : -touched[~t];
    }
    return HP_OK;
}

hp_status hp_halo_reduce_pack(hp_halo h, const double* local, double* send) {
    if (!h || !local || (!send && !h->rsend.empty())) { set_error("hp_halo_reduce_pack: null argument"); return HP_ERR_ARG; }
    for (size_t k = 0; k < h->rsend.size(); ++k) {
        const int64_t i = h->rsend[k];
        send[k] = h->lmap[i] >= 0 ? local[i] : -local[i];
    }
    return HP_OK;
}

hp_status hp_halo_reduce_sum(hp_halo h, const double* local, const double* recv, double* owned) {
    if (!h || !local || !owned || (!recv && h->rrecv_off.back() > 0)) {
        set_error("hp_halo_reduce_sum: null argument");
        return HP_ERR_ARG;
    }
    const int64_t nl = (int64_t)h->lmap.size();
    for (size_t o = 0; o < h->owned_t.size(); ++o) {
        double acc = 0.0;
        for (int64_t k = h->asm_ptr[o]; k < h->asm_ptr[o + 1]; ++k) {
            const int64_t s = h->asm_src[k];
            acc += s < nl ? (h->lmap[s] >= 0 ? local[s] : -local[s]) : recv[s - nl];
        }
        owned[o] = acc;
    }
    return HP_OK;
}

hp_status hp_halo_bcast_pack(hp_halo h, const double* owned, double* send) {
    if (!h || !owned || (!send && !h->bsend.empty())) { set_error("hp_halo_bcast_pack: null argument"); return HP_ERR_ARG; }
    for (size_t k = 0; k < h->bsend.size(); ++k) send[k] = owned[h->bsend[k]];
    return HP_OK;
}

hp_status hp_halo_bcast_unpack(hp_halo h, const double* owned, const double* recv, double* touched) {
    if (!h || !owned || !touched || (!recv && !h->brecv.empty())) {
        set_error("hp_halo_bcast_unpack: null argument");
        return HP_ERR_ARG;
    }
    for (size_t o = 0; o < h->owned_t.size(); ++o) touched[h->owned_t[o]] = owned[o];
    for (size_t k = 0; k < h->brecv.size(); ++k) touched[h->brecv[k]] = recv[k];
    return HP_OK;
}

void hp_halo_destroy(hp_halo h) { delete h; }

hp_status hp_xdot_acc(const double* x, const double* y, int64_t n, int64_t* acc) {
    if (!acc || n < 0 || (n > 0 && (!x || !y))) { set_error("hp_xdot_acc: bad argument"); return HP_ERR_ARG; }
    int64_t since = 0;
    for (int64_t i = 0; i < n; ++i) {
        const double p = x[i] * y[i];
        const double e = std::fma(x[i], y[i], -p);     // x y = p + e exactly (no underflow)
        xacc_add(acc, p);
        xacc_add(acc, e);
        if (++since == ((int64_t)1 << 28)) { xacc_normalise(acc); since = 0; }
    }
    xacc_normalise(acc);
    return HP_OK;
}

hp_status hp_xacc_round(const int64_t* acc, double* out) {
    if (!acc || !out) { set_error("hp_xacc_round: null argument"); return HP_ERR_ARG; }
    *out = xacc_round(acc);
    return HP_OK;
}

int hp_xacc_limbs(void) { return kLimbs; }

}  // extern "C"
