/*
 * hp.h -- C ABI of libhp: element-local spectral/hp operators on mixed
 * hexahedral / prismatic / pyramidal / tetrahedral meshes, on one NVIDIA GPU.
 *
 * The operators are those of Sec. 2 of "Architecture-aware h-to-p
 * optimisation: spectral/hp element operators for mixed-element meshes":
 * the elemental mass matrix M = B^T W B (Eq. mass), the Laplacian L of
 * Eq. (Lap) and the Helmholtz operator H = lambda M + L (Sec. 2.1), evaluated
 * matrix-free in the collocated form of Eq. (helm1) (Sec. 2.2, Alg. "Helmholtz
 * implementation by collocated approach"): BwdTrans to the quadrature
 * points, collocated derivative, pointwise metric, transposed derivative,
 * and one restriction B^T back to modes.  Prisms, pyramids and tetrahedra
 * use tensorial modified-Jacobi expansions on collapsed coordinates
 * (Sec. 2.3, Duffy transformation).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns an hp_status; nothing throws or exits.  A failed
 *   call leaves its outputs untouched unless stated otherwise.
 *   hp_last_error() gives a message for the last failure on this thread.
 * - Device pointers are plain CUDA device addresses on the mesh's device;
 *   the caller owns them (allocate them with any allocator, e.g. PyTorch).
 *   Host pointers are read during the call only.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Operator applications are asynchronous on that stream.
 * - Element order is the caller's ("user order").  The coefficient vector is
 *   ragged: element e owns [coeff_offset[e], coeff_offset[e+1]).  A
 *   physical-space vector holds Q^3 values per element at
 *   [phys_offset[e], phys_offset[e+1]), point (i,j,k) of the collapsed
 *   coordinates (eta_1, eta_2, eta_3) at i*Q*Q + j*Q + k.  Vector fields
 *   (three components) are three whole physical-space vectors back to back.
 * - Mode order inside an element: each mode is a product of 1-D factors
 *   in (eta_1, eta_2, eta_3) and has a slot key (ka, kb, kc); modes are sorted
 *   by that key, kc fastest.  ka/kb/kc index the 1-D family of their
 *   direction: L = (1-z)/2 -> 0, R = (1+z)/2 -> 1, bubble psi_n -> n+1; in a
 *   warped family W_s (factors L^{s+1} and L^{s+1} R P^{(2s+1,1)}_{r-1}) the
 *   member index r.  Modes constant in a direction (collapsed vertex, edge
 *   and face modes) take key 0 there.  The families are those of the
 *   modified C0 basis of Karniadakis & Sherwin, to which the paper refers
 *   its 3-D expansions (Sec. 2.3).
 * - Quadrature: Q = P + 2 points per direction (Sec. 2.1 asks for at least
 *   P + 2); Gauss-Lobatto-Legendre in non-collapsed directions,
 *   Gauss-Radau-Jacobi (node -1 included) in collapsed ones.
 */
#ifndef HP_H
#define HP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hp_mesh_s* hp_mesh;
typedef struct hp_op_s* hp_op;

typedef enum {
    HP_OK = 0,
    HP_ERR_ARG = 1,            /* bad argument: null pointer, size or enum out of range */
    HP_ERR_OOM = 2,            /* device or host allocation failed */
    HP_ERR_CUDA = 3,           /* a CUDA runtime call failed */
    HP_ERR_GEOM = 4,           /* element with |J| <= 0 or vertices that are not an affine image */
    HP_ERR_UNSUPPORTED = 5,    /* valid request that this build does not implement */
    HP_ERR_TIMEOUT = 6,        /* a bounded device wait gave up (error word set by a kernel) */
    HP_ERR_DEVICE_BOUNDS = 7,  /* a kernel saw an index outside its tables */
    HP_ERR_NOT_CONVERGED = 8   /* iterative solve stopped before its tolerance */
} hp_status;

typedef enum { HP_HEX = 0, HP_PRISM = 1, HP_PYR = 2, HP_TET = 3 } hp_shape;

typedef enum {
    HP_MASS = 0,                    /* coeff -> coeff : M uhat                                   */
    HP_LAPLACIAN = 1,               /* coeff -> coeff : L uhat                                   */
    HP_HELMHOLTZ = 2,               /* coeff -> coeff : (lambda M + L) uhat                      */
    HP_BWDTRANS = 3,                /* coeff -> phys  : u = B uhat                               */
    HP_IPRODUCT_WRT_BASE = 4,       /* phys  -> coeff : B^T W f                                  */
    HP_PHYSDERIV = 5,               /* phys  -> 3 phys: du/dx_i of the Lagrange interpolant      */
    HP_IPRODUCT_WRT_DERIV_BASE = 6, /* 3 phys -> coeff: sum_i (d phi/d x_i, f_i)                 */
    HP_ADVECTION_DIFFUSION_REACTION = 7  /* coeff -> coeff: (grad phi_m, grad u) + (phi_m, a . grad u)
                                            + lambda (phi_m, u), a constant velocity set by
                                            hp_op_set_advection (Sec. 2.2 names this operator among those
                                            the B^T {pointwise} B decomposition covers); the Helmholtz
                                            passes with the advection term added at the points */
} hp_opkind;

typedef enum {
    HP_STRAT_SUMFAC = 0,   /* fused sum-factorised collocated kernel (Alg. collocated Helmholtz)  */
    HP_STRAT_ELEMAT = 1,   /* reference-element dense matrices, non-collocated (StdMat, Sec. 3.3.1) */
    HP_STRAT_HYBRID = 2,   /* dense B / B^T with collocated derivatives                           */
    HP_STRAT_AUTO = 3,     /* the library chooses per block                                       */
    HP_STRAT_MATRIX = 4    /* stored per-element dense H^e (matrix-based, Sec. 3.3 implementation
                              strategies): mass, Laplacian, Helmholtz; HP_FP64 / HP_FP32; blocks of
                              at most 256 modes (larger blocks run HP_STRAT_SUMFAC)               */
} hp_strategy;

/* Compute type.  HP_FP64: IEEE double throughout (the oracle-parity form).
 * HP_FP32: single precision (CUDA cores), float arrays.  HP_TF32 / HP_BF16:
 * the elemental-matrix and hybrid strategies on the tensor cores (tcgen05,
 * Blackwell).  Elemental matrix: coefficients, reference matrices and
 * metric-weighted point values rounded to TF32 (10-bit mantissa) or BF16
 * (7-bit mantissa), products accumulated in FP32 in tensor memory, metric
 * factors kept in FP16 with one power-of-two scale per element (11
 * significant bits).  Hybrid: u = B uhat and B^T u' on the tensor cores
 * (coefficients, B and u' rounded to TF32 / BF16, FP32 accumulation), the
 * collocated derivatives and the FP32 metric between them on the CUDA cores.
 * Float arrays; relative error a few units of 2^-11 (TF32) or 2^-8 (BF16). */
typedef enum { HP_FP64 = 0, HP_FP32 = 1, HP_TF32 = 2, HP_BF16 = 3 } hp_dtype;

/* Mesh description (all host arrays, copied by hp_mesh_create).
 *   n_elem               number of elements (>= 1)
 *   shape[n_elem]        hp_shape of each element
 *   P[n_elem], Q[n_elem] expansion order (1..10) and points per direction (must be P + 2)
 *   vert[n_elem*8]       global vertex ids in reference-vertex order, unused slots -1:
 *                        hex (-1,-1,-1)(1,-1,-1)(1,1,-1)(-1,1,-1)(-1,-1,1)(1,-1,1)(1,1,1)(-1,1,1)
 *                        prism (-1,-1,-1)(1,-1,-1)(1,1,-1)(-1,1,-1)(-1,-1,1)(-1,1,1)
 *                        pyramid (-1,-1,-1)(1,-1,-1)(1,1,-1)(-1,1,-1)(-1,-1,1)
 *                        tet (-1,-1,-1)(1,-1,-1)(-1,1,-1)(-1,-1,1)
 *   xyz[3*n_vert]        vertex coordinates, x y z per vertex
 *   curved[n_elem]       0: the element map is the affine vertex map; 1: apply `deformation`
 *   deformation          0 none; 1: x_i += 0.05 sin(pi x_j) sin(pi x_k), (i,j,k) cyclic;
 *                        2: x_i += 0.1 x_j x_k (a quadratic map, for tests of the geometry)
 *   geometry             0: curved elements use the map itself (analytic Jacobian);
 *                        1: iso-parametric: each coordinate of a curved element's map is
 *                        projected onto the element's own degree-P expansion (L2 projection on
 *                        the reference element with its quadrature rule) and the Jacobian is
 *                        that of the expansion (the iso-parametric curved elements of the
 *                        paper's benchmarks, Sec. 4).  Affine elements are exact either way.
 *   quadrature           0: Q = P + 2 points in every direction; 1 (reduced rule): Q - 1
 *                        Gauss-Radau-Jacobi points in the collapsed directions (prism and
 *                        pyramid eta_3, tetrahedron eta_2 and eta_3), which still integrates
 *                        the mass and Laplacian matrices of affine elements exactly and cuts
 *                        the points, so the metric factors, of a tetrahedron by (2Q - 1)/Q^2.
 *                        The point vectors then hold q1 q2 q3 values per element in the same
 *                        (i, j, k) order.  A reduced-rule mesh has the elemental-matrix
 *                        operators of mass, Laplacian and Helmholtz (HP_STRAT_ELEMAT in every
 *                        dtype: FP64 / FP32 CUDA cores, TF32 / BF16 tensor cores); geometry 1,
 *                        the sum-factorised kernels, the C0 space and hp_mesh_points are for
 *                        the full rule (HP_ERR_UNSUPPORTED).
 * Every element must be an affine image of its reference element (all vertices
 * are checked); curved elements are that affine map followed by the deformation. */
typedef struct {
    int64_t n_elem;
    const uint8_t* shape;
    const uint8_t* P;
    const uint8_t* Q;
    const int64_t* vert;
    const double* xyz;
    int64_t n_vert;
    const uint8_t* curved;
    int32_t deformation;
    int32_t geometry;
    int32_t quadrature;
} hp_mesh_desc;

/* Create a mesh on CUDA device `device`: validates and copies the description,
 * groups elements into blocks of equal (shape, P, Q, curved) (paper Sec. 3.3:
 * blocks of identically structured elements with constant stride), and
 * builds the reference tables.  Errors: HP_ERR_ARG (bad sizes or ids),
 * HP_ERR_GEOM (non-affine vertex set or non-positive volume, message names
 * the element), HP_ERR_UNSUPPORTED (P > 10 or Q != P + 2), HP_ERR_CUDA/OOM. */
hp_status hp_mesh_create(const hp_mesh_desc* desc, int device, hp_mesh* out);

/* Ragged layout in user order.  Any output pointer may be NULL.
 *   coeff_offset[n_elem+1], phys_offset[n_elem+1]; n_coeff / n_phys = totals. */
hp_status hp_mesh_layout(hp_mesh mesh, int64_t* coeff_offset, int64_t* phys_offset,
                         int64_t* n_coeff, int64_t* n_phys);

/* Geometric factors in FP64 on the device (paper Sec. 2.1 chain rule; Sec. 4 names these
 * six metric terms and the Jacobian as the geometric data of deformed elements): for curved
 * elements, at every quadrature point G_dd' = w|J| sum_i (d eta_d/d x_i)
 * (d eta_d'/d x_i) (d <= d') and w|J|; for affine elements per element
 * |J| (d xi/d x)(d xi/d x)^T, |J| and d xi/d x.  Idempotent: the first call
 * computes, later calls return HP_OK at once.  Synchronises `stream`.
 * With geometry = 1 the curved elements' factors come from the iso-parametric
 * map (one kernel per block: the map at the points, its projection, the
 * derivatives of the expansion), computed in FP64 on the device; the FP32 and
 * tensor-core copies and every operator then use them.  hp_mesh_points still
 * gives the points of the map itself.
 * Errors: HP_ERR_GEOM if some |J| <= 0 at a quadrature point (message names
 * the first such element), HP_ERR_CUDA. */
hp_status hp_geom_factors(hp_mesh mesh, void* stream);

/* Copy the per-point factors of every element to host memory, in user order:
 * out7[phys_offset[e]*7 + f*Q^3 + l] for f = G11,G12,G13,G22,G23,G33,w|J|,
 * and (if out9 != NULL) out9[phys_offset[e]*9 + (3d+i)*Q^3 + l] = d eta_d/d x_i.
 * Affine elements are expanded to points.  Computes the factors if needed.
 * Meant for tests; synchronises the device. */
hp_status hp_geom_copy(hp_mesh mesh, double* out7, double* out9);

/* Create an operator of kind `kind` over all blocks of `mesh`, computing in
 * `dtype` with `strategy`.  HP_FP64 and HP_FP32 apply to every kind with
 * HP_STRAT_SUMFAC (the only strategy of the derivative building blocks and of
 * HP_ADVECTION_DIFFUSION_REACTION); arrays passed to hp_op_apply are double (HP_FP64) or
 * float (HP_FP32, HP_TF32, HP_BF16).  HP_TF32 and HP_BF16 take HP_STRAT_ELEMAT (or AUTO)
 * or HP_STRAT_HYBRID and the kinds HP_MASS, HP_LAPLACIAN, HP_HELMHOLTZ: blocks
 * with at most 256 modes per element (elemental matrix; BF16: 320, past 256
 * with the backward tiles streamed and the output in two MMAs) or 512 (BF16
 * hybrid) / 352 (TF32 hybrid) run the tensor-core form, larger ones FP32 sum
 * factorisation (hp_op_strategies reports which).  BF16 also builds the
 * elemental matrix for blocks of 321..512 modes (the output in parts of a
 * tile that each repeat the forward); those blocks start on FP32 sum
 * factorisation, measured faster on them, and hp_op_strategies or the
 * schedulers can move them.  Errors: HP_ERR_ARG,
 * HP_ERR_UNSUPPORTED (combination not built), HP_ERR_GEOM / HP_ERR_CUDA from
 * the geometric factors it needs. */
hp_status hp_op_create(hp_mesh mesh, hp_opkind kind, hp_strategy strategy, hp_dtype dtype,
                       hp_op* out);

/* out = op(in) on `stream`, asynchronously (one kernel launch per block).
 * `in`/`out`: device arrays sized by hp_mesh_layout for the op's spaces
 * (see hp_opkind); they must not overlap.  lambda is used by HP_HELMHOLTZ.
 * Errors detected before launch: HP_ERR_ARG; launch failure: HP_ERR_CUDA.
 * Device-side errors latch in the op and are returned by hp_op_sync.
 * HP_STRAT_MATRIX blocks build their stored matrices on the first apply (N_P
 * sum-factorised applies of the block, then a synchronisation of `stream`),
 * and again on a Helmholtz apply with a different lambda; device memory for
 * them is allocated there (HP_ERR_CUDA if it is not available).  Later applies
 * are asynchronous.  A rebuild for a new lambda overwrites the matrices in
 * place: it first waits for all work already queued on the device (applies
 * and graph replays of this op on any stream finish before it), and it drops
 * the op's captured graph.  The caller must not queue applies of the same op
 * on other streams while such a call runs. */
hp_status hp_op_apply(hp_op op, double lambda, const void* in, void* out, void* stream);

/* Batched apply for meshes with many blocks (p-adaptive / mixed meshes): the
 * same result as hp_op_apply, launched as one CUDA graph in which every block's
 * kernel is an independent node, so blocks of different (shape, P, curved) run
 * concurrently on the GPU.  The graph is built on the first call for a given
 * (lambda, in, out) -- that call also runs the apply once uncaptured -- and
 * replayed by later calls with the same arguments; other arguments rebuild it.
 * Do not call it while `stream` is being captured.  Errors as hp_op_apply. */
hp_status hp_op_apply_graph(hp_op op, double lambda, const void* in, void* out, void* stream);

/* How hp_op_apply and hp_op_apply_graph launch the blocks (a p-adaptive mesh
 * has many blocks, each too small to fill the GPU).  mode 0 (the default):
 * one kernel per block (hp_op_apply: one after another; hp_op_apply_graph: a
 * CUDA graph with the blocks as concurrent nodes).  mode 1: one persistent
 * launch over a device work list.  The blocks' element groups are cut into
 * work items of about a quarter of a CTA's fair share of the FP64 operation
 * count, ordered by decreasing cost.  Each CTA takes the next item from a
 * device counter, stages that block's reference tables and runs its
 * sum-factorisation body; hp_op_apply_graph captures the counter reset and
 * that one launch.  Results are bitwise those of mode 0 (the same body per
 * element).  Mode 1 needs an HP_FP64 operator in the collocated form whose
 * blocks all use HP_STRAT_SUMFAC with P <= 8 (HP_ERR_UNSUPPORTED otherwise);
 * writing other strategies, the non-collocated form or running a schedule
 * search returns the op to mode 0.  Drops the op's captured graph.
 * Errors: HP_ERR_ARG, HP_ERR_UNSUPPORTED, HP_ERR_CUDA / HP_ERR_OOM. */
hp_status hp_op_set_batching(hp_op op, int mode);

/* Autotune: time each block's kernel with each tile variant (elements per CTA
 * chosen from shared-memory budgets of 56, 20 and 110 KB) on the given arrays
 * (their contents are overwritten as by hp_op_apply) and keep the fastest per
 * block.  Synchronises `stream`.  Results are bitwise identical for every tile. */
hp_status hp_op_tune(hp_op op, double lambda, const void* in, void* out, void* stream);

/* Read (set = 0) or write (set = 1) the tile variant (0..2: the 56, 20 and
 * 110 KB budgets of hp_op_tune) of each of the op's n_blocks blocks (blocks in
 * order of first appearance of (shape, P, curved) in user element order).  A
 * new operator starts every block on tile 1.  HP_ERR_ARG if n_blocks does not
 * match or a tile is out of range. */
hp_status hp_op_tiles(hp_op op, int* tiles, int64_t n_blocks, int set);

/* Read (set = 0) or write (set = 1) the implementation strategy of each block
 * (HP_STRAT_SUMFAC, HP_STRAT_ELEMAT, HP_STRAT_HYBRID or HP_STRAT_MATRIX).
 * Writing builds the dense reference matrices if a block needs them.
 * HP_STRAT_MATRIX is accepted for HP_FP64 / HP_FP32 mass, Laplacian and
 * Helmholtz operators on blocks of at most 256 modes (its matrices are built
 * by the next apply); a block that leaves HP_STRAT_MATRIX frees its stored
 * matrices at once.  HP_ERR_UNSUPPORTED for a dense strategy on a derivative
 * building block, for HP_STRAT_MATRIX outside those limits, and for an
 * HP_TF32 / HP_BF16 operator for anything but HP_STRAT_SUMFAC (FP32),
 * HP_STRAT_ELEMAT (tensor core, blocks of at most 256 modes; BF16: 512) or
 * HP_STRAT_HYBRID (tensor core, at most 512 modes in BF16, 352 in TF32).
 * Writing drops the op's captured graph. */
hp_status hp_op_strategies(hp_op op, int* strategies, int64_t n_blocks, int set);

/* Form of the sum-factorised Laplacian and Helmholtz blocks of an HP_FP64
 * operator (the two forms of the paper's collocation study, Sec. 5 "Maximising
 * collocation-based operations"; Sec. 3.3 for the collocated algorithm).
 * collocated = 1 (the default): BwdTrans to the points, the derivatives by
 * collocation differentiation there, and their transposes (Sec. 3.3).
 * collocated = 0: the derivatives d phi / d eta_d by sum-factorisation passes
 * with the 1-D derivative tables, and the transposed inner products the same
 * way (the non-collocated approach).  Both compute (lambda M + L) uhat; they
 * agree up to rounding.  Blocks with other strategies and other operator
 * kinds are unaffected.  HP_ERR_ARG unless collocated is 0 or 1;
 * HP_ERR_UNSUPPORTED for collocated = 0 on an operator that is not HP_FP64.
 * Drops the op's captured graph when the form changes.  hp_op_work and
 * hp_op_block_work keep reporting the collocated form's operation counts. */
hp_status hp_op_set_collocated(hp_op op, int collocated);

/* Advection velocity a (host array of 3 doubles, x y z) of an
 * HP_ADVECTION_DIFFUSION_REACTION operator (0 at creation): its applies then
 * compute (grad phi_m, grad u) + (phi_m, a . grad u) + lambda (phi_m, u).  At
 * each point the velocity enters in collapsed coordinates, c_d = sum_i a_i
 * d eta_d / d x_i (curved elements: the stored d eta / d x; affine ones:
 * d eta / d xi times the element's d xi / d x).  Drops the op's captured graph.
 * Errors: HP_ERR_ARG (null arguments, another operator kind). */
hp_status hp_op_set_advection(hp_op op, const double* velocity);

/* Summation order of the tensor-core operators' split tiles (HP_TF32 /
 * HP_BF16; not in the paper).  A block with fewer 128-element tiles than the
 * GPU has CTA slots splits each tile's point chunks over several CTAs, whose
 * partial outputs are added.  deterministic = 0 (the default): FP32 atomics
 * into the zeroed output, so results differ run to run at FP32 rounding
 * (far below the form's own error); 1: each part writes its partial output
 * to a scratch buffer of the op (parts x elements x modes floats per split
 * block, allocated by the first apply that needs it) and one more kernel
 * adds the parts in part order, so results are bitwise reproducible.  Other
 * dtypes are always reproducible and ignore the flag.  hp_solve sets it on
 * its inner tensor-core operator.  Drops the op's captured graph when the
 * setting changes.  Errors: HP_ERR_ARG. */
hp_status hp_op_set_deterministic(hp_op op, int deterministic);

/* ---------------------------------------------------------------- cost model
 * Not in the paper (which picks a strategy by a fixed rule per operator):
 * a small MLP, trained by the library's own kernels on timings the library
 * generates, predicts the log run time of each strategy of a block. */
typedef struct hp_mlp_s* hp_mlp;

/* Features of each block of an op, 5 floats per block:
 * shape/3, P/10, curved (0/1), log10(elements)/6, dtype/2 (FP64 = 0). */
hp_status hp_op_block_features(hp_op op, float* features, int64_t n_blocks);

/* MLP n_in -> n_hidden -> n_hidden -> n_out with ReLU, FP32 parameters on
 * `device`, He-uniform weights drawn from SplitMix64(seed), zero biases.
 * Limits: n_in 1..16, n_hidden 32..256 (multiple of 32), n_out 1..8. */
hp_status hp_mlp_create(int n_in, int n_hidden, int n_out, uint64_t seed, int device, hp_mlp* out);
/* Sizes of a network (any pointer may be NULL). */
hp_status hp_mlp_info(hp_mlp mlp, int* n_in, int* n_hidden, int* n_out, int64_t* n_params);
/* Copy the flat parameter vector (W1[H][n_in], b1[H], W2[H][H], b2[H],
 * W3[n_out][H], b3[n_out]) to (set = 0) or from (set = 1, resets Adam) host memory. */
hp_status hp_mlp_params(hp_mlp mlp, float* host, int64_t n_params, int set);
/* y[batch][n_out] = MLP(x[batch][n_in]); device arrays, 1 <= batch <= 65535. */
hp_status hp_mlp_forward(hp_mlp mlp, const float* x, int64_t batch, float* y, void* stream);
/* Gradient of L = mean over batch and outputs of (y - t)^2 w.r.t. the flat
 * parameters into grad[n_params] (device), and L into loss[1] (device, may be NULL).
 * Deterministic: per-sample rows summed in sample order. */
hp_status hp_mlp_grad(hp_mlp mlp, const float* x, const float* t, int64_t batch, float* grad, float* loss,
                      void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on that loss. */
hp_status hp_mlp_adam_step(hp_mlp mlp, const float* x, const float* t, int64_t batch, float lr, float* loss,
                           void* stream);
void hp_mlp_destroy(hp_mlp mlp);

/* The gradient of hp_mlp_grad for callers that cannot allocate device memory
 * (no counterpart in the paper).  Such callers are, for example, programs whose
 * device memory is owned by a pool or framework allocator that forbids
 * cudaMalloc/cudaFree outside it, or loops that must not pay the device-wide
 * synchronisation cudaFree implies.  The caller passes everything as device
 * arrays on the current device: the flat parameters (layout of hp_mlp_params),
 * x[batch][n_in], t[batch][n_out], and the outputs grad[n_params] and loss[1]
 * (loss may be NULL); sizes obey the limits of hp_mlp_create.  The call
 * allocates nothing: its scratch is one fixed device array of 2^20 floats
 * (4 MiB, held by every GPU that loads the library until the process exits),
 * so batch * (n_params + 2 n_hidden + n_out + 1) must not exceed 2^20, else
 * HP_ERR_ARG with a message.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  Every call uses the same array:
 * calls that overlap on the GPU (other streams, other threads) race and must
 * be serialised by the caller.  Each call writes every scratch entry it
 * reads, so the previous call's contents do not matter.  Results equal
 * hp_mlp_grad's for the same parameters and data. */
hp_status hp_mlp_grad_noalloc(const float* params, int n_in, int n_hidden, int n_out, const float* x,
                              const float* t, int64_t batch, float* grad, float* loss, void* stream);

/* Pick each block's strategy as the argmin of the network's 3 outputs (the
 * predicted log times of SUMFAC, ELEMAT, HYBRID) on the block's features.
 * Derivative building blocks stay SUMFAC.  Same as hp_op_schedule_mlp with
 * graph_launch = 0. */
hp_status hp_op_schedule(hp_op op, hp_mlp mlp, void* stream);

/* Pick each block's strategy as the argmin, over the strategies built for the
 * block, of the network's predicted log times.  The network maps 5 or 6
 * features to 3 or 4 outputs: the features of hp_op_block_features, then (6
 * inputs) graph_launch: 1 when the blocks will run as the concurrent graph of
 * hp_op_apply_graph, 0 when one after another (hp_op_apply); the outputs are
 * the predicted log times of SUMFAC, ELEMAT, HYBRID and (4 outputs) MATRIX.
 * For an HP_TF32 / HP_BF16 operator output 0 is its FP32 sum factorisation,
 * output 1 its tensor-core elemental matrix and output 2 its tensor-core
 * hybrid; stored matrices are not built for it and never chosen.  Derivative building blocks stay SUMFAC.
 * Drops the op's captured graph.  Errors: HP_ERR_ARG (null arguments,
 * graph_launch not 0 or 1, network of another shape), HP_ERR_CUDA. */
hp_status hp_op_schedule_mlp(hp_op op, hp_mlp mlp, int graph_launch, void* stream);

/* Exhaustive schedule: time every strategy of every block on the given arrays
 * (contents overwritten; each block launched alone, one warm-up launch, which
 * also builds stored matrices, and two timed) and keep the fastest;
 * times_ms[4*block + k] (may be NULL) receives the timings for k = 0..3 =
 * HP_STRAT_SUMFAC, HP_STRAT_ELEMAT, HP_STRAT_HYBRID, HP_STRAT_MATRIX (1e30 for
 * strategies not built for the block, and for stored matrices that would not
 * fit in half of the free device memory).  Stored matrices of trials that are
 * not kept are freed.  Synchronises `stream`.  hp_op_schedule_graph searches
 * on the time of the whole concurrent graph instead. */
hp_status hp_op_schedule_exhaustive(hp_op op, double lambda, const void* in, void* out, float* times_ms,
                                    void* stream);

/* Graph-aware schedule (not in the paper): coordinate descent on the time of
 * the whole concurrent graph launch of hp_op_apply_graph.  Starting from the
 * current strategies, each block in turn tries every other strategy built for
 * it (HP_FP64 / HP_FP32 mass, Laplacian and Helmholtz: sum factorisation,
 * elemental matrix, hybrid and, for blocks of at most 256 modes whose matrices
 * fit in half of the free device memory, stored matrices; HP_TF32 / HP_BF16:
 * FP32 sum factorisation, the tensor-core elemental matrix and the
 * tensor-core hybrid) and keeps one
 * only if the graph's median time over `reps` timed launches
 * (after a warm-up) drops by more than 1 %; `passes` sweeps over the blocks.
 * Per-block times taken alone (hp_op_schedule_exhaustive) miss the overlap of
 * the blocks that run concurrently in the graph.  in/out as for
 * hp_op_apply_graph (contents overwritten); *ms (may be NULL) receives the
 * final median graph time.  Errors: HP_ERR_ARG (reps outside 1..64, passes
 * outside 1..8, null or aliasing arrays), HP_ERR_CUDA. */
hp_status hp_op_schedule_graph(hp_op op, double lambda, const void* in, void* out, int reps, int passes, float* ms,
                               void* stream);

/* Physical coordinates of every quadrature point (device array 3*n_phys,
 * component-major: xyz[c*n_phys + phys_offset[e] + l]); the affine vertex map
 * followed, for curved elements, by the mesh's deformation. */
hp_status hp_mesh_points(hp_mesh mesh, double* xyz, void* stream);

/* ---------------------------------------------------------------- assembled solve
 * The global C0 problem behind the weak form of Sec. 2.1:
 * (grad u, grad v) + lambda (u, v) = (f, v), homogeneous Dirichlet conditions
 * on the boundary faces (faces that belong to one element). */
typedef struct hp_c0_s* hp_c0;

/* Global C0 numbering of a conforming mesh with one order P on all elements:
 * one DOF per vertex, P-1 per edge, (P-1)^2 per quad face, (P-1)(P-2)/2 per
 * triangular face, and the element interiors; global order vertices, edges,
 * faces, interiors.  Each local coefficient maps to (gid, sign): u_local =
 * sign * u_global[gid].  Triangular faces must have their collapsed vertex at
 * the face's largest global vertex id (the slab generator ensures it).
 * HP_ERR_UNSUPPORTED for mixed orders or non-conforming orientations. */
hp_status hp_c0_create(hp_mesh mesh, hp_c0* out);
hp_status hp_c0_info(hp_c0 c0, int64_t* n_global, int64_t* n_boundary);
/* The same numbering computed on the host from a mesh description, without a
 * GPU: gid[n_coeff], sign[n_coeff] and boundary[n_global] (the caller sizes
 * boundary with n_coeff entries, an upper bound of n_global). */
hp_status hp_c0_map_host(const hp_mesh_desc* desc, int64_t* gid, int8_t* sign, uint8_t* boundary, int64_t* n_global);
/* Host copies of the maps: gid[n_coeff], sign[n_coeff], boundary[n_global] (any may be NULL). */
hp_status hp_c0_maps(hp_c0 c0, int64_t* gid, int8_t* sign, uint8_t* boundary);
/* local = A global (device FP64 arrays). */
hp_status hp_c0_gather(hp_c0 c0, const double* global, double* local, void* stream);
/* global = A^T local, summing the local copies of each global DOF in a fixed
 * order (deterministic); Dirichlet entries set to 0 if mask_boundary. */
hp_status hp_c0_assemble(hp_c0 c0, const double* local, double* global, int mask_boundary, void* stream);

/* Diagonal of lambda M + L: assembled (the Jacobi preconditioner; local = 0,
 * diag[n_global], Dirichlet entries included) or per element (local = 1,
 * diag[n_coeff], the diagonals of the element matrices in the coefficient layout). */
hp_status hp_c0_diagonal(hp_c0 c0, double lambda, double* diag, int local, void* stream);

typedef struct {
    double tol;            /* stop at ||b - A x|| <= tol ||b|| (FP64 residual)                 */
    int max_iter;          /* FP64 CG: iteration limit                                          */
    int mixed;             /* 0: Jacobi-PCG in FP64; 1: FP64 refinement of FP32 Jacobi-PCG      *
                            * (sum-factorised FP32 operator); 2 / 3: the same with the TF32 /   *
                            * BF16 tensor-core operator inside (HP_TF32 / HP_BF16)               */
    double inner_tol;      /* mixed: relative tolerance of each FP32 solve                      */
    int inner_max_iter;    /* mixed: iteration limit of each FP32 solve                         */
    int max_refinements;   /* mixed: refinement steps                                           */
    int schedule;          /* 1: before the first solve, choose each block's strategy for the   *
                            * FP64 operator and the inner operator with hp_op_schedule_graph    *
                            * (sum factorisation, elemental matrix, hybrid, stored matrices;    *
                            * tensor-core inner operators: FP32 sum factorisation or the        *
                            * tensor-core elemental matrix), kept for later solves with         *
                            * schedule = 1; 0: the operators' default strategies               */
} hp_solve_opts;

typedef struct {
    int iterations;        /* CG iterations (mixed: total FP32 iterations)                      */
    int inner_iterations;  /* mixed: total FP32 iterations                                      */
    int refinements;       /* mixed: FP64 residual evaluations used                             */
    double rel_residual;   /* final ||b - A x|| / ||b||, in FP64                                */
} hp_solve_stats;

/* Solve A x = rhs for the assembled lambda M + L (lambda >= 0) with the
 * element operators of this library.  rhs, x: device FP64 global vectors
 * (x holds the initial guess; its Dirichlet entries are set to 0).  The first
 * solve for a lambda builds the Jacobi diagonal (element diagonals summed).
 * Synchronises `stream`.  HP_ERR_NOT_CONVERGED if the tolerance is not met
 * (x holds the last iterate, stats the residual). */
hp_status hp_solve(hp_c0 c0, double lambda, const double* rhs, double* x, const hp_solve_opts* opts,
                   hp_solve_stats* stats, void* stream);
void hp_c0_destroy(hp_c0 c0);

/* ---------------------------------------------------------------- multi-GPU layout (host only)
 * The element-local operators of Sec. 2 need no exchange: a partition of the
 * elements is a partition of the work.  The assembled problem couples
 * elements through shared global DOFs: each CG iteration needs one sum over
 * the interface DOFs that partitions share and two dot products.  These calls
 * build that layout on the host, with no GPU; the data moves between ranks by
 * the caller's transport (e.g. torch.distributed). */

/* Partition the elements of `desc` into nparts parts (part[n_elem] in
 * 0..nparts-1) balanced by predicted cost: cost[n_elem] (NULL: each element's
 * floating-point operations in the collocated sum-factorised Helmholtz
 * operator, which sets the time of the FP64 path).  method 0: ranges of the block order (blocks of
 * equal shape, order and curvature in order of first appearance, user order
 * inside a block), cut where the cost prefix crosses k/nparts of the total, so
 * each part keeps few, large blocks (element-local operators); method 1:
 * recursive coordinate bisection of the element centroids, each split along
 * the axis of largest extent at the cost fraction of its halves (compact
 * parts, small interfaces: the assembled solve).  Deterministic.  Errors:
 * HP_ERR_ARG (null arrays, nparts outside 1..65536, bad method, negative or
 * non-finite cost, vertex id out of range, bad shape or order). */
hp_status hp_partition(const hp_mesh_desc* desc, const double* cost, int nparts, int method, int32_t* part);

/* Halo plan of one rank for the assembled solve, from the one-rank C0 map
 * (gid, sign over the one-rank coefficient layout coeff_offset[n_elem+1], as
 * hp_c0_maps / hp_c0_map_host give) and an element partition.  The rank's
 * local coefficients are those of its elements in user order; it holds
 * copies of its "touched" global DOFs (ascending gid), of which it owns those
 * whose lowest holding rank it is.  One halo sum = reduce (each rank sends
 * the signed local copies of DOFs owned elsewhere to their owner; the owner
 * adds every copy, its own and the received ones, in the one-rank local order
 * starting from 0, so the assembled value has the same bits as
 * hp_c0_assemble's for any partition) then broadcast (the owner sends each
 * owned value to every other holder).  Messages between two ranks are in
 * ascending gid order.  Errors: HP_ERR_ARG (bad sizes, ids, signs or parts),
 * HP_ERR_OOM. */
typedef struct hp_halo_s* hp_halo;
hp_status hp_halo_create(const int64_t* gid, const int8_t* sign, const int64_t* coeff_offset, int64_t n_elem,
                         int64_t n_global, const int32_t* part, int nparts, int rank, hp_halo* out);
/* Sizes: local coefficients, touched and owned global DOFs (any pointer may be NULL). */
hp_status hp_halo_info(hp_halo h, int64_t* n_local, int64_t* n_touched, int64_t* n_owned);
/* Message sizes (values) per peer rank, arrays of nparts (any may be NULL):
 * reduce sent / received, broadcast sent / received. */
hp_status hp_halo_counts(hp_halo h, int64_t* reduce_send, int64_t* reduce_recv, int64_t* bcast_send,
                         int64_t* bcast_recv);
/* Maps (any may be NULL): local_index[n_local] = index of each local
 * coefficient in the one-rank layout; touched_gid[n_touched]; owned_gid[n_owned]. */
hp_status hp_halo_maps(hp_halo h, int64_t* local_index, int64_t* touched_gid, int64_t* owned_gid);
/* local[n_local] = sign * touched[...] (the rank's part of u_local = A u_global). */
hp_status hp_halo_gather(hp_halo h, const double* touched, double* local);
/* Reduce step, sender side: send[...] = signed local copies for each peer,
 * peer q's message at the offset given by the prefix of reduce_send counts. */
hp_status hp_halo_reduce_pack(hp_halo h, const double* local, double* send);
/* Reduce step, owner side: owned[n_owned] = sum of the copies of each owned
 * DOF (own signed local values and recv, the peers' messages back to back in
 * rank order), in the one-rank order. */
hp_status hp_halo_reduce_sum(hp_halo h, const double* local, const double* recv, double* owned);
/* Broadcast step: send[...] = owned values for each peer (prefix of
 * bcast_send counts); unpack writes touched[n_touched] from the rank's owned
 * values and recv (the peers' messages back to back in rank order). */
hp_status hp_halo_bcast_pack(hp_halo h, const double* owned, double* send);
hp_status hp_halo_bcast_unpack(hp_halo h, const double* owned, const double* recv, double* touched);
void hp_halo_destroy(hp_halo h);

/* Exact dot products (not in the paper; what makes a multi-rank CG take the
 * same iterates as a one-rank CG).  hp_xdot_acc adds sum_i x[i] y[i] exactly
 * into acc[hp_xacc_limbs()] (zero it first): each product as its rounded
 * value and its FMA rounding error, in a fixed-point accumulator of 32-bit
 * limbs (int64 each) from 2^-1074 up, carries normalised on return.  Ranks
 * combine accumulators by an integer sum of the limbs (an all-reduce); the
 * sum is exact and associative, so the result does not depend on the
 * partition or the order of terms.  hp_xacc_round rounds an accumulator (or
 * such a sum of at most 2^30 of them) to the nearest double, ties to even.
 * Products whose error term underflows (|x y| < 2^-969) carry that one
 * rounding, identically on every partition.  Errors: HP_ERR_ARG. */
hp_status hp_xdot_acc(const double* x, const double* y, int64_t n, int64_t* acc);
hp_status hp_xacc_round(const int64_t* acc, double* out);
int hp_xacc_limbs(void);

/* Synchronise `stream` and report any error latched by the op's kernels
 * (HP_ERR_TIMEOUT, HP_ERR_DEVICE_BOUNDS) or by CUDA. */
hp_status hp_op_sync(hp_op op, void* stream);

/* Measured FP64 fused multiply-add rate of GPU `device` (not in the paper: the
 * denominator of the FP64 roofline).  Launches a kernel in which every thread
 * of a full-occupancy grid runs 8 independent FMA recurrences for `iters`
 * steps (1..2^24; 20 000 takes a few tens of milliseconds on a GB300), on
 * `stream`, once to warm up and three times timed with CUDA events; *tflops
 * receives 2 x FMAs / fastest time, *ms (may be NULL) that time.  Allocates a
 * small device buffer for the results and synchronises `stream`.
 * Errors: HP_ERR_ARG, HP_ERR_CUDA. */
hp_status hp_peak_fp64(int device, int iters, double* tflops, double* ms, void* stream);

/* Algorithmic work of one hp_op_apply: output DOFs (sum of N_P, or of Q^3 for
 * physical-space outputs), flops of the sum-factorised collocated algorithm
 * and the minimum HBM bytes (inputs, outputs, geometric factors), for the
 * roofline.  Any pointer may be NULL. */
hp_status hp_op_work(hp_op op, int64_t* out_dofs, double* flops, double* bytes);

/* The same accounting for one block (block >= 0; -1 = the whole operator, as
 * hp_op_work), plus its element count and exec_flops: the floating-point
 * operations the block's kernel issues (FMA = 2), which the FP64
 * sum-factorised kernel brings below the collocated count `flops` by the
 * even-odd symmetry of the GLL direction and by skipping the padding of the
 * collapsed index ranges.  Blocks are numbered as in hp_op_tiles.  Any output
 * pointer may be NULL.  Errors: HP_ERR_ARG. */
hp_status hp_op_block_work(hp_op op, int64_t block, int64_t* n_elem, int64_t* out_dofs, double* flops,
                           double* exec_flops, double* bytes);

/* Apply the operator to the elements of one block only (one kernel launch,
 * as hp_op_apply does for every block in turn); outputs of other blocks are
 * left untouched.  Launching every block in order is hp_op_apply; used to time
 * the kernels one by one.  Errors as hp_op_apply, HP_ERR_ARG for a bad block. */
hp_status hp_op_apply_block(hp_op op, int64_t block, double lambda, const void* in, void* out, void* stream);

/* ------------------------------------------------------------------------
 * Two-dimensional formulation (paper Sec. 2.2): quadrilaterals (HP_QUAD) and
 * triangles (HP_TRI) with the modified C0 basis on (collapsed) coordinates
 * -- quadrilateral A_a(xi_1) A_b(xi_2), triangle A_a(eta_1) W_{w(a),b}(eta_2)
 * on eta_1 = 2 (1 + xi_1)/(1 - xi_2) - 1 -- Q = P + 2 points per direction
 * (Gauss-Lobatto-Legendre; Gauss-Radau-Jacobi alpha = 1 in the triangle's
 * eta_2), and the mass, Laplacian and Helmholtz operators by the collocated
 * algorithm (Eq. helm1 in two dimensions): two sum-factorised passes for B
 * and B^T, collocation derivatives along the point lines, pointwise metric.
 * Mode order: by the slot key (a, b), b fastest (a: L or 1 -> 0, R -> 1,
 * psi_n -> n + 1; b the same on the second factor, or the warped-family
 * index r when a is a bubble of the triangle).  Points (i, j), j fastest.
 * ------------------------------------------------------------------------ */
typedef struct hp_mesh2d_s* hp_mesh2d;
enum { HP_QUAD = 4, HP_TRI = 5 };

/* Two-dimensional mesh (copied by hp_mesh2d_create):
 *   shape[n_elem]        HP_QUAD or HP_TRI
 *   P[n_elem]            polynomial order 1..10 (Q = P + 2)
 *   vert[n_elem * 4]     vertex ids; vertex 0 and its neighbours along xi_1 and
 *                        xi_2 are ids 0, 1 and 3 (quadrilateral, a parallelogram:
 *                        id 2 is not read by the affine map) or 0, 1, 2 (triangle;
 *                        id 3 ignored)
 *   xy[2 * n_vert]       vertex coordinates
 *   curved[n_elem]       1: apply the deformation to the element map
 *   deformation          0 none, 1 x_i += 0.05 sin(pi x_1) sin(pi x_2) (i = 1, 2;
 *                        fixes the boundary of the unit square) */
typedef struct {
    int64_t n_elem;
    const uint8_t* shape;
    const uint8_t* P;
    const int64_t* vert;
    const double* xy;
    int64_t n_vert;
    const uint8_t* curved;
    int32_t deformation;
} hp_mesh2d_desc;

/* Build the mesh on `device`: blocks of equal (shape, P, curved), reference
 * tables, and the FP64 metric factors G11, G12, G22, w|J| at every point (FP32
 * copy).  Synchronises the device.  Errors: HP_ERR_ARG (null or empty arrays,
 * shape, order or vertex id out of range, deformation not 0 / 1),
 * HP_ERR_GEOM (|J| <= 0 at a point), HP_ERR_CUDA / HP_ERR_OOM. */
hp_status hp_mesh2d_create(const hp_mesh2d_desc* desc, int device, hp_mesh2d* out);

/* Element offsets (n_elem + 1 each, may be NULL) of the modal vectors (N_P =
 * (P+1)^2 or (P+1)(P+2)/2 per element) and of the point vectors (Q^2). */
hp_status hp_mesh2d_layout(hp_mesh2d mesh, int64_t* coeff_offset, int64_t* phys_offset);

/* out = operator(in) for kind HP_MASS, HP_LAPLACIAN or HP_HELMHOLTZ (lambda:
 * the Helmholtz constant), dtype HP_FP64 (double arrays) or HP_FP32 (float
 * arrays, FP32 factors and tables); in and out are device modal vectors of
 * the layout above, caller-owned, not aliased.  Asynchronous on `stream`
 * (NULL: the legacy default stream).  Errors: HP_ERR_ARG, HP_ERR_UNSUPPORTED
 * (another kind or dtype), HP_ERR_CUDA. */
hp_status hp_op2d_apply(hp_mesh2d mesh, hp_opkind kind, hp_dtype dtype, double lambda, const void* in, void* out,
                        void* stream);

/* Copy the FP64 metric factors to host memory: host_out[4 * phys_offset[e] +
 * f * Q^2 + l] for factor f = G11, G12, G22, w|J| of element e at point l.
 * Synchronous.  Errors: HP_ERR_ARG, HP_ERR_CUDA. */
hp_status hp_mesh2d_factors(hp_mesh2d mesh, double* host_out);

/* Wait for `stream` and report an asynchronous CUDA error.  Errors: HP_ERR_ARG, HP_ERR_CUDA. */
hp_status hp_mesh2d_sync(hp_mesh2d mesh, void* stream);
void hp_mesh2d_destroy(hp_mesh2d mesh);

void hp_op_destroy(hp_op op);
void hp_mesh_destroy(hp_mesh mesh);
const char* hp_status_str(hp_status s);
const char* hp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HP_H */
