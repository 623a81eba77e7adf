// Layout of the per-(shape, P) reference-table blob copied to shared memory
// by the kernels (host and device agree at compile time).
#pragma once

namespace hp {

__host__ __device__ constexpr int n_modes_c(int shape, int P) {
    return shape == 0 ? (P + 1) * (P + 1) * (P + 1)
         : shape == 1 ? (P + 1) * (P + 1) * (P + 2) / 2
         : shape == 2 ? (P + 1) * (P + 2) * (2 * P + 3) / 6
                      : (P + 1) * (P + 2) * (P + 3) / 6;
}

// Index structure of the collapsed shapes at compile time: weight of member a
// of family 0, family of the eta2 factor of slot (a, .), family of the eta3
// factor of slot (a, b, .), family lengths, and the number of valid (a, b)
// pairs and valid slots (the triangular / pyramidal index ranges).
__host__ __device__ constexpr int wA_c(int a) { return a <= 1 ? 0 : a - 1; }
__host__ __device__ constexpr int famlen_c(int P, int s) { return s == 0 ? P + 1 : (s >= P ? 0 : P - s); }
__host__ __device__ constexpr int famb_c(int shape, int a) { return shape == 3 ? wA_c(a) : 0; }
__host__ __device__ constexpr int lenb_c(int shape, int P, int a) { return famlen_c(P, famb_c(shape, a)); }
__host__ __device__ constexpr int famc_c(int shape, int P, int a, int b) {
    return shape == 0 ? 0
         : shape == 1 ? wA_c(a)
         : shape == 2 ? (wA_c(a) > wA_c(b) ? wA_c(a) : wA_c(b))
         : (a <= 1 ? wA_c(b) : (b < P - wA_c(a) ? wA_c(a) + b : P));
}
__host__ __device__ constexpr int npairs_c(int shape, int P) {
    int t = 0;
    for (int a = 0; a <= P; ++a) t += lenb_c(shape, P, a);
    return t;
}
__host__ __device__ constexpr int nvalid_c(int shape, int P) {
    int t = 0;
    for (int a = 0; a <= P; ++a)
        for (int b = 0; b < lenb_c(shape, P, a); ++b) t += famlen_c(P, famc_c(shape, P, a, b));
    return t;
}

struct BlobLayout {
    int Ta, Td, Tb, Tc, D, z, w, rz, total_vals;          // offsets in values (Ta: parity form;
                                                          // rz[d][i] = 1 / (1 - z_d[i]), 0 at z = 1)
    int famb, famc, slot2mode, mode_slots;                // offsets in bytes
    int pairs, valid, poff, porder, total_bytes;          // valid (a,b) pairs and slots (int32), pair
                                                          // offset per a (int16), pairs by length (uint8)
};

__host__ __device__ constexpr int align16c(int x) { return (x + 15) & ~15; }

__host__ __device__ constexpr BlobLayout blob_layout_c(int shape, int P, int vs) {
    BlobLayout L{};
    const int n = P + 1, Q = P + 2;
    int o = 0;
    L.Ta = o; o += n * Q;
    L.Td = o; o += n * Q;
    L.Tb = o; o += (P + 1) * n * Q;
    L.Tc = o; o += (P + 1) * n * Q;
    L.D = o; o += 3 * Q * Q;
    L.z = o; o += 3 * Q;
    L.w = o; o += 3 * Q;
    L.rz = o; o += 3 * Q;
    L.total_vals = o;
    int b = align16c(o * vs);
    L.famb = b; b += n;
    L.famc = b; b += n * n;
    b = (b + 1) & ~1;
    L.slot2mode = b; b += 2 * n * n * n;
    L.mode_slots = b; b += 2 * 4 * n_modes_c(shape, P);
    b = (b + 3) & ~3;
    const bool lists = shape != 0;                  // the hexahedron has no padding to skip
    L.pairs = b; b += lists ? 4 * npairs_c(shape, P) : 0;
    L.valid = b; b += lists ? 4 * nvalid_c(shape, P) : 0;
    L.poff = b; b += lists ? 2 * (n + 1) : 0;
    L.porder = b; b += lists ? npairs_c(shape, P) : 0;
    L.total_bytes = align16c(b);
    return L;
}

}  // namespace hp
