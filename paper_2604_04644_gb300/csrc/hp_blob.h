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

struct BlobLayout {
    int Ta, Tb, Tc, D, z, w, total_vals;                  // offsets in values
    int famb, famc, slot2mode, mode_slots, total_bytes;   // offsets in bytes
};

__host__ __device__ constexpr int align16c(int x) { return (x + 15) & ~15; }

__host__ __device__ constexpr BlobLayout blob_layout_c(int shape, int P, int vs) {
    BlobLayout L{};
    const int n = P + 1, Q = P + 2;
    int o = 0;
    L.Ta = o; o += n * Q;
    L.Tb = o; o += (P + 1) * n * Q;
    L.Tc = o; o += (P + 1) * n * Q;
    L.D = o; o += 3 * Q * Q;
    L.z = o; o += 3 * Q;
    L.w = o; o += 3 * Q;
    L.total_vals = o;
    int b = align16c(o * vs);
    L.famb = b; b += n;
    L.famc = b; b += n * n;
    b = (b + 1) & ~1;
    L.slot2mode = b; b += 2 * n * n * n;
    L.mode_slots = b; b += 2 * 4 * n_modes_c(shape, P);
    L.total_bytes = align16c(b);
    return L;
}

}  // namespace hp
