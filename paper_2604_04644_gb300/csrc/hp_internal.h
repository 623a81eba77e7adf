// Internal data structures of libhp (not part of the C ABI).
#pragma once
#include <cstdint>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/hp.h"
#include "hp_blob.h"

namespace hp {

constexpr int PMAX = 10;

// ---------------------------------------------------------------- tables
// Reference data of one (shape, P) with Q = P + 2, built on the host in FP64.
// Slot space: the padded (P+1)^3 tensor of 1-D factors (a, b, c), c fastest.
// Family index of the eta_2 factor of slot (a, .): famb[a]; of the eta_3 factor
// of slot (a, b, .): famc[a*n+b]; family 0 is {L, R, psi_1..psi_{P-1}}, family
// s >= 1 the warped W_s, family P is empty (all zero).
struct RefTables {
    int shape = 0, P = 0, Q = 0, n = 0, NP = 0, NQ = 0;
    std::vector<double> z[3], w[3];        // points / weights per direction (Duffy-scaled)
    std::vector<double> Ta;                // [a][i]        n*Q
    std::vector<double> Tp, Td;            // [a][i]        n*Q, eta1 table in parity form and its derivative
    std::vector<double> Tb;                // [t][b][j]     (P+1)*n*Q
    std::vector<double> Tc;                // [s][c][k]     (P+1)*n*Q
    std::vector<double> Tbd, Tcd;          // d/d eta_2 of Tb, d/d eta_3 of Tc at the points (same layout)
    std::vector<double> D[3];              // [i][m]        Q*Q, d/d eta of Lagrange basis
    std::vector<uint8_t> famb, famc;       // n, n*n
    std::vector<int16_t> slot2mode;        // n^3, -1 = empty slot
    std::vector<int16_t> mode_slots;       // NP*4, -1 padded
};

const RefTables& ref_tables(int shape, int P);
int n_modes(int shape, int P);
// flops of the collocated sum-factorised Helmholtz operator per element (FMA = 2)
double elem_flops_helmholtz(int shape, int P);

// All modes of (shape, P) at one reference point xi (not at a collapse point).
void eval_modes(int shape, int P, const double xi[3], double* out);
// Member m of 1-D family s (0: L, R, psi; s >= 1: warped W_s) at z.
double family_value(int P, int s, int m, double z);

// Dense reference matrices A4[q][l][m] (q = 0: B, q = 1..3: d/d eta_q of B), FP64.
std::vector<double> dense_matrices(int shape, int P);
// Points and weights per direction of the full (rq = 0) or reduced (rq = 1:
// Q - 1 Gauss-Radau-Jacobi points in the collapsed directions) rule.
void rule_points(int shape, int P, int rq, std::vector<double> z[3], std::vector<double> w[3]);
// A4 at the points of the reduced rule (layout as dense_matrices, N_Q = q1 q2 q3).
std::vector<double> dense_matrices_rq(int shape, int P);
int n_points(int shape, int P, int rq);   // points per element of the rule

// Serialise the tables in value type T (double or float) into bytes.
std::vector<unsigned char> make_blob(const RefTables& t, size_t value_size);

// ---------------------------------------------------------------- mesh
struct Block {
    int shape, P, Q, curved;
    int64_t n_elem;
    // quadrature points per direction and per element (Q, Q, Q and Q^3 for the
    // full rule; the reduced rule has Q - 1 in the collapsed directions, and
    // its blocks keep per-point factors: curved = 1, map_curved = the user flag)
    int q[3] = {0, 0, 0};
    int nq = 0;
    int map_curved = 0;
    std::vector<int64_t> elems;           // user element ids (host)
    int64_t* d_coeff_off = nullptr;       // [n_elem] coefficient offset of each element
    int64_t* d_phys_off = nullptr;        // [n_elem] phys offset of each element
    double* d_frame = nullptr;            // [n_elem][12] X0 (3) + E (3x3, E[i][d])
    double* d_geom = nullptr;             // curved: [n_elem][7][NQp]; affine: [n_elem][16]
    double* d_dgeom = nullptr;            // curved only: [n_elem][9][NQp] d eta_d / d x_i
    float* d_geom32 = nullptr;            // FP32 copies (created on demand)
    float* d_dgeom32 = nullptr;
    double* d_geom_pts = nullptr;         // affine only: per-point factors [n_elem][7][NQp] (FP64 Laplacian /
                                          // Helmholtz read these like curved factors)
    uint16_t* d_geom_tc = nullptr;        // tensor-core operator: tile-major FP16 factors (curved and affine)
    float* d_gscale_tc = nullptr;         // and their per-element scales (Laplacian factors, w|J|)
    int64_t coeff_total = 0, phys_total = 0;   // per-block totals (work accounting)
};

struct DeviceBlobs {
    double* rq_zw = nullptr;    // reduced rule: z1 w1 z2 w2 z3 w3 (per-direction counts of the blocks)
    void* d64 = nullptr;
    void* d32 = nullptr;
    int bytes64 = 0, bytes32 = 0;
    // dense reference matrices (created for elemental-matrix / hybrid operators):
    // A4 [4][NQ][NP] and A4T [NP][4][NQ], in FP64 and FP32
    double* A4_64 = nullptr;
    double* A4T_64 = nullptr;
    float* A4_32 = nullptr;
    float* A4T_32 = nullptr;
    // tensor-core reference tiles (TF32, tensor-core shared-memory order), see TCArgs
    unsigned char* tc_img = nullptr;            // TF32 tiles
    unsigned char* tc_img16 = nullptr;          // BF16 tiles (same order, 2-byte elements)
    int tc_KP16 = 0, tc_fwd16 = 0, tc_bwd16 = 0;
    int64_t tc_chunk16 = 0;
    int tc_KP = 0, tc_NPpad = 0, tc_nch = 0, tc_fwd = 0, tc_bwd = 0;
    int64_t tc_chunk = 0;
    // derivative tables [Tbd | Tcd] in FP64, for the non-collocated sum-factorisation kernel
    double* d_nc64 = nullptr;
    // iso-parametric geometry (FP64): point values -> coefficients of the projection in
    // reference-orthonormal functions, S^T [point][mode], and their values VT [mode][point]
    double* iso_RT = nullptr;
    double* iso_VT = nullptr;
};

}  // namespace hp

struct hp_mesh_s {
    int device = 0;
    int64_t n_elem = 0;
    int deformation = 0;
    int geometry = 0;                           // 0 analytic map, 1 iso-parametric (curved elements)
    int quadrature = 0;                         // 1: Q - 1 points in the collapsed directions
    std::vector<uint8_t> shape, P, Q, curved;
    std::vector<int64_t> coeff_off, phys_off;   // n_elem + 1
    std::vector<int64_t> vert;                  // n_elem * 8 global vertex ids (for the C0 map)
    std::vector<hp::Block> blocks;
    std::map<int, hp::DeviceBlobs> blobs;       // key shape*16 + P
    bool geom_ready = false, dgeom_ready = false, geom32_ready = false;
    unsigned int* d_err = nullptr;              // device error word
};

struct hp_op_s {
    hp_mesh mesh = nullptr;
    hp_opkind kind;
    hp_strategy strategy;
    hp_dtype dtype;
    unsigned int* d_err = nullptr;
    std::vector<int> tile;                      // tile variant per block
    std::vector<int> strat;                     // hp_strategy per block (SUMFAC, ELEMAT, HYBRID)
    int collocated = 1;                         // 0: FP64 sum-factorised Laplacian/Helmholtz in the non-collocated form
    int deterministic = 0;                      // 1: tensor-core split tiles summed in a fixed order
    double adv[3] = {0.0, 0.0, 0.0};            // advection velocity of an advection-diffusion-reaction op
    // batching 1: every block in one persistent work-list launch (FP64 sum factorisation)
    int batching = 0;
    void* d_desc = nullptr;                     // SFDesc per block (plain applies)
    void* d_desc_graph = nullptr;               // the same for the captured graph
    void* d_items = nullptr;                    // WorkItem list, by decreasing cost
    int* d_next = nullptr;                      // work-list counter
    int n_items = 0, wl_smem = 0, wl_grid = 0;
    // while a graph of all blocks is captured: each tensor-core elemental-matrix
    // block's share of the GPU (its tiles x chunks x (K_P + N_P) over all such
    // blocks'), for which it splits its tiles; empty otherwise
    std::vector<double> tc_share;
    // tensor-core hybrid blocks: u = B uhat and u' at every point of the mesh's
    // point layout (two FP32 vectors; blocks write disjoint ranges)
    float* hyb_u = nullptr;
    float* hyb_v = nullptr;
    std::vector<float*> part_buf;               // their partial outputs, per block (grown on demand)
    std::vector<int64_t> part_cap;
    // matrix-based blocks: stored H^e as Ht[n][e][m] (FP64 or FP32, the op's I/O type), built on
    // the first apply, and again when lambda changes (Helmholtz)
    std::vector<void*> mat;
    std::vector<double> mat_lambda;
    // CUDA graph of one apply (blocks as independent nodes), for fixed (lambda, in, out)
    cudaGraphExec_t graph = nullptr;
    const void* g_in = nullptr;
    void* g_out = nullptr;
    double g_lambda = 0.0;
    std::vector<cudaStream_t> pool;             // fork streams used while capturing
};

namespace hp {
void set_error(const std::string& msg);
hp_status cuda_fail(cudaError_t e, const char* what);
int nqp(int Q);   // padded points per element (multiple of 4)

// device-side error codes (latched in the error word)
constexpr unsigned int DERR_TIMEOUT = 1u;
constexpr unsigned int DERR_BOUNDS = 2u;
constexpr unsigned int DERR_GEOM = 4u;

// launch of the geometry kernel over one block (hp_geom.cu)
cudaError_t launch_geom(const Block& b, const DeviceBlobs& blob, int deformation, bool want_deriv,
                        unsigned int* d_err, int* d_bad_elem, cudaStream_t s);
// per-point factors of an affine block, expanded from its records (FP64, curved layout)
cudaError_t launch_affine_points(const Block& b, const DeviceBlobs& blob, double* out, cudaStream_t s);
// iso-parametric geometric factors of a curved block (needs blob.iso_RT and blob.iso_VT)
cudaError_t launch_geom_iso(const Block& b, const DeviceBlobs& blob, int deformation, bool want_deriv,
                            unsigned int* d_err, int* d_bad_elem, cudaStream_t s);
cudaError_t launch_to_f32(const double* src, float* dst, int64_t n, cudaStream_t s);
// physical coordinates of the quadrature points of a block, xyz[c*n_phys_total + phys_off + l]
cudaError_t launch_points(const Block& b, const DeviceBlobs& blob, int deformation, double* xyz,
                          int64_t n_phys_total, cudaStream_t s);
// element diagonals of lambda M + L (FP64) into local coefficient slots
cudaError_t launch_elem_diag(const Block& b, const DeviceBlobs& blob, double lambda, double* diag, cudaStream_t s);
// C0 numbering (hp_c0.cpp)
hp_status build_c0(const hp_mesh m, const std::vector<int64_t>& vert, std::vector<int64_t>& gid,
                   std::vector<int8_t>& sign, std::vector<uint8_t>& boundary, int64_t& n_global);

// arguments of the sum-factorisation kernels
template <typename T>
struct SFArgs {
    int op;                      // hp_opkind
    int64_t n_elem;
    T lambda;
    T adv[3];                    // advection velocity (HP_ADVECTION_DIFFUSION_REACTION)
    const int64_t* coeff_off;    // per block element
    const int64_t* phys_off;
    const T* in;
    T* out;
    int64_t n_phys_total;        // stride between vector-field components
    const T* geom;               // curved [e][7][NQp], affine [e][16]
    const T* dgeom;              // curved [e][9][NQp] (deriv ops), affine: unused
    const unsigned char* blob;   // table blob (16-byte aligned)
    int blob_bytes;
    unsigned int* err;
    // FP32 only: 1 = the point-space core of mass / Laplacian / Helmholtz (in and
    // out are point values in the phys layout; no B, no B^T), the middle kernel
    // of the tensor-core hybrid
    int point_io;
    // differentiation matrices D_d[i][m] and the eta1 table A[a][i] of the block,
    // read by the kernels as constant-bank operands (Q <= 12, n <= 11)
    T cD[3][144];
    T cTa[132];
};

// arguments of the elemental-matrix / hybrid kernels (hp_emat.cu)
template <typename T>
struct EMArgs {
    int op, shape, P, Q, NQ, NP, NQp;
    int64_t n_elem;
    T lambda;
    const int64_t* coeff_off;
    const int64_t* phys_off;
    const T* in;
    T* out;
    const T* geom;               // as SFArgs
    const T* A4;                 // [4][NQ][NP]
    const T* A4T;                // [NP][4][NQ]
    const unsigned char* blob;   // table blob (for D, z, w)
    unsigned int* err;
};
cudaError_t emat_launch_f64(bool hybrid, bool affine, const EMArgs<double>& a, cudaStream_t s);

// tensor-core (tcgen05, TF32) elemental-matrix operator, hp_tc_emat.cu
struct TCArgs {
    int op, Q, NQ, NQp, NP, KP, NPpad, nch, c0, c1;   // components [c0, c1) of {B, dB/deta_1..3}
    int64_t n_elem;
    float lambda;
    const int64_t* coeff_off;
    const float* in;
    float* out;
    const uint16_t* geom16;            // tile-major FP16 factors, scaled per element (tc_geom_layout16)
    const float* gscale;               // [tiles x 128][2] 2^-k of element e's Laplacian factors and of its w|J|
    const unsigned char* img;          // per chunk of points: 4 forward then 4 backward tiles
    int64_t chunk_bytes;
    int fwd_bytes, bwd_bytes, stage_bytes;
    int es;                            // operand bytes: 4 TF32, 2 BF16
    int nsplit, stages, ubufs;         // set by the launcher
    double slot_share;                 // share of the GPU's CTA slots for this block in a concurrent graph (0: all)
    int variant;                       // BF16 past 256 modes (tc_variant): 2 lean (two forward accumulators,
                                       // one V' tile), 1 streamed backward tiles; 0 otherwise
    int nmpart, mwidth;                // output-mode parts of a tile and their width (set by the launcher)
    float* part_out;                   // nullptr: split tiles add with atomics; else [nsplit][n_elem][NP]
                                       // partial outputs summed in part order (deterministic)
    unsigned int* err;
};
// parts per tile the launcher will use (0 on error): part_out needs nsplit * n_elem * NP floats
int tc_emat_nsplit(const TCArgs& a);
int tc_variant(int KP, int NPpad, int fwd_bytes, int es);   // TCArgs::variant of a block
// hybrid strategy on the tensor cores (hp_tc_emat.cu): mode 0 u = B uhat
// (coefficients -> the block's points in the phys layout), mode 1 out = B^T u'
struct HybArgs {
    int NQ, NP, KP, NPpad, nch, es;
    int64_t n_elem;
    const int64_t* coeff_off;
    const int64_t* phys_off;
    const float* in;
    float* out;
    const unsigned char* img;          // the elemental-matrix operator's reference image
    int64_t chunk_bytes;
    int fwd_bytes, bwd_bytes;
    int stages, stage_bytes;           // set by the launcher
    unsigned int* err;
};
cudaError_t tc_hyb_launch(const HybArgs& a, int mode, cudaStream_t s);
constexpr int kTcMaxModes = 256;
constexpr int kTcMaxModes16 = 512;      // BF16 elemental matrix with streamed backward tiles (mode parts of <= 320)
constexpr int kTcDefaultMaxModes16 = 320;   // BF16 blocks an elemental-matrix operator starts on the tensor cores
// the tensor-core hybrid: BF16 up to 512 modes; TF32 up to 352 (its U tile,
// 128 x K_P x 4 bytes, and two ring stages must fit in shared memory)
constexpr int kTcHybMaxModes = 512, kTcHybMaxModesTF32 = 352;
int tc_hyb_smem(int mode, int es, int KP, int NPpad, int bwd_bytes, int* stages_out, int* stage_bytes_out);
int tc_chunk_points();
int64_t tc_geom_halves(int64_t n_elem, int nch);
cudaError_t tc_geom_layout16(int shape, bool curved, const double* g, int NQp, int NQ, const double* z, const double* w, int Q,
                             uint16_t* out, float* isc, int64_t n_elem, int nch, cudaStream_t s);
cudaError_t tc_emat_launch(const TCArgs& a, cudaStream_t s);
cudaError_t emat_launch_f32(bool hybrid, bool affine, const EMArgs<float>& a, cudaStream_t s);

// persistent work-list form of the FP64 sum-factorised operators (hp_sf_worklist.cu):
// one launch in which CTAs take work items (a block and a range of its element
// groups) from a device counter and run that block's (shape, P, affine) body
struct SFDesc {                  // the fields of SFArgs<double> the FP64 bodies read
    int op;
    int64_t n_elem;
    double lambda;
    double adv[3];
    const int64_t* coeff_off;
    const int64_t* phys_off;
    const double* in;
    double* out;
    int64_t n_phys_total;
    const double* geom;
    const double* dgeom;
    const unsigned char* blob;
    int blob_bytes;
    unsigned int* err;
};
struct WorkItem {
    int32_t block, key;          // key = shape * 32 + P * 2 + affine
    int64_t g0, g1;              // element groups [g0, g1) of the block
};
constexpr int kWorklistMaxP = 8;
int sf_worklist_epb(int P);                       // elements per group (tile 0)
int sf_worklist_smem(int shape, int P);           // dynamic shared memory of that body
cudaError_t sf_worklist_grid(int smem, int* grid);   // CTAs resident on the device at that smem
cudaError_t sf_worklist_launch(const SFDesc* desc, const WorkItem* items, int n_items, int* next, int smem, int grid,
                               unsigned int* err, cudaStream_t s);

// per-shape launchers (hp_sf_<shape>.cu)
cudaError_t sf_launch_f64(int shape, int P, bool affine, int tile, const SFArgs<double>& a, cudaStream_t s);
cudaError_t sf_launch_f32(int shape, int P, bool affine, int tile, const SFArgs<float>& a, cudaStream_t s);
int sf_epb_host(int P, int tile, bool f64);
// non-collocated FP64 sum factorisation (hp_sf_nc.cu): the derivatives by
// sum-factorisation passes with the derivative tables dtab = [Tbd | Tcd]
cudaError_t sf_nc_launch(int shape, int P, bool affine, const SFArgs<double>& a, const double* dtab, cudaStream_t s);
// matrix-based strategy (hp_mat.cu)
constexpr int kMatMaxModes = 256;
cudaError_t mat_unit(double* x, const int64_t* coeff_off, int64_t ne, int NP, int m, cudaStream_t s);
cudaError_t mat_collect(const double* y, const int64_t* coeff_off, int64_t ne, int NP, int m, void* Ht, bool f64,
                        cudaStream_t s);
cudaError_t mat_apply(const void* Ht, const int64_t* coeff_off, int64_t ne, int NP, const void* in, void* out, bool f64,
                      cudaStream_t s);
constexpr int kTiles = 3;
constexpr int kDefaultTile = 1;      // the 20 KB shared-memory budget of kTileBudget

}  // namespace hp
