/*
 * lam.h -- C ABI of the GB300 (sm_103a) stiffness-assembly library for 3D
 * layered solids built on an extruded tensor-product discretisation.
 *
 * Method: P. Antolin, "Fast assembly of Galerkin matrices for 3D solid
 * laminated composites using finite element and isogeometric
 * discretizations" (2019). The library assembles the FP64 stiffness matrix
 *     K^{ij} = sum_l int_{Omega_l} B^{iT} D_l B^j |DF| dxi      (Eq. Km_0)
 * of linear elasticity (Eq. a, Section 2.1) in CSR form, two ways:
 *   - lam_assemble_split:    the split 2D x 1D method of Section 3,
 *                            K = sum_m sum_{ab} P_{m,ab} (x) Q_{m,ab} (Eq. Km_2),
 *                            one in-plane operator set per distinct
 *                            (material, angle) configuration m;
 *   - lam_assemble_standard: element-by-element 3D Gauss quadrature
 *                            (Section 2.4), the comparison path.
 * Both produce the same matrix up to rounding (Section 3, after Eq. Q).
 *
 * Discretisation (Assumption 1, Eq. basis_functions): 3D functions are
 * products S^{i_s}(xi^1, xi^2) T^{i_t}(z) of an in-plane function and a
 * thickness function.
 *   - In-plane: tensor-product B-spline (optionally NURBS) or Lagrange Q_p basis
 *     on [knots], with n_x * n_y functions, i_s = iy * n_x + ix; the in-plane
 *     map is x(xi) = sum_i S^i(xi) X_i from the control points X_i.
 *   - Thickness: B-spline or Lagrange basis in the extrusion coordinate xi^3
 *     of Eq. extrusion, F = S(xi^1, xi^2) + xi^3 a (physical z for the plate,
 *     a = e_z; any constant direction a for a general extrusion, see
 *     lam_inplane). DF does not depend on xi^3, so Assumption 2 holds by
 *     construction.
 *   - 3D function index i = i_t * n_s + i_s (0-based form of Assumption 1);
 *     DOF index 3*i + c, c in {x, y, z}.
 * Plies (Eq. C_layers, Assumption 3): ply 0 starts at the first thickness
 * knot, plies stack upwards; each ply has a thickness, a material and an
 * in-plane angle; the ply thicknesses must add up to the thickness-knot range
 * (to 1e-10 relative). A ply interface closer than 1e-10 of a thickness
 * element's length to an end of that element is taken to coincide with it.
 * Materials: 21 Voigt constants (upper triangle, row-major, order
 * 11,22,33,12,13,23, engineering shear, Eq. D) in the material frame; a ply
 * of angle theta has its fibre axis 1 at +theta about +z from global x.
 *
 * Sparsity (bit-exact, independent of the values): one 3x3 block for every
 * pair of 3D functions whose supports share a 3D element (an in-plane
 * element times a thickness element); all 9 entries are stored, explicit
 * zeros included; columns ascending; int64 row pointers, int32 columns.
 *
 * Conventions for every call:
 *   - Errors are returned as lam_status; nothing traps or aborts. The last
 *     error message of the calling thread is available from lam_last_error().
 *   - Host pointers (struct fields of lam_plan_create) are read during the
 *     call only; the plan copies what it needs.
 *   - Device pointers (the d_ arguments) are caller-owned device memory of the
 *     plan's device; the library never frees them.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Every device
 *     call is stream-ordered and asynchronous unless stated otherwise. A plan
 *     must not be used on two streams at the same time.
 *   - The plan owns its device workspace (allocated with cudaMalloc on the
 *     first device call, on the device current at that time). A failed
 *     allocation returns LAM_ERR_OOM and releases what the call had allocated;
 *     the plan stays usable. For tests of these paths, LAM_FAIL_ALLOC=n in the
 *     environment makes the n-th device allocation counted from the moment the
 *     variable took its value fail as out of memory (host side; no device
 *     fault is involved).
 */
#ifndef LAM_H
#define LAM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LAM_OK = 0,
  LAM_ERR_INVALID_ARG = 1,  /* malformed input (degree, knots, plies, sizes) */
  LAM_ERR_UNSUPPORTED = 2,  /* valid input outside what the library handles */
  LAM_ERR_OOM = 3,          /* host or device allocation failed */
  LAM_ERR_CUDA = 4,         /* a CUDA runtime call failed */
  LAM_ERR_TIMEOUT = 5       /* reserved: no call waits on the device with a bound, none returns it */
} lam_status;

typedef enum { LAM_BSPLINE = 0, LAM_LAGRANGE = 1 } lam_basis_kind;

/* A 1D basis (Section 2.2). B-spline: `knots` is a non-decreasing open knot
 * vector of length n_knots (functions: n_knots - degree - 1; interior knot
 * multiplicity <= degree). Lagrange: `knots` holds the n_knots increasing
 * element breakpoints; each element carries degree + 1 equispaced nodes
 * (functions: degree * (n_knots - 1) + 1). 1 <= degree <= 7. */
typedef struct {
  int32_t kind;          /* lam_basis_kind */
  int32_t degree;
  int32_t n_knots;
  const double* knots;   /* host */
} lam_basis1d;

/* In-plane discretisation and map (Section 2.2, Eq. gradient, Eq. extrusion).
 * The solid is the extrusion F(xi) = S(xi^1, xi^2) + xi^3 a of a surface S,
 * given by its control points, along a constant direction a (Assumption 1:
 * DF does not depend on xi^3); xi^3 runs over the thickness knots. A planar
 * S = (x, y, 0) with a = e_z (ctrl_dim 2, extrusion zero) is the plate case
 * of the split kernels; any other S or a (a "shell") is a general extrusion,
 * assembled by the split and standard paths (lam_assemble_split,
 * lam_assemble_split_host, lam_assemble_standard, lam_inplane_operators, and
 * in batches, one by one), differentiated by lam_adjoint, and refused with
 * LAM_ERR_UNSUPPORTED by lam_assemble_split_noalloc. DF = [dS/dxi1 |
 * dS/dxi2 | a] must be regular. */
typedef struct {
  lam_basis1d u;          /* xi^1 direction, index ix */
  lam_basis1d v;          /* xi^2 direction, index iy */
  const double* ctrl;     /* host, n_s x ctrl_dim ((x, y) or (x, y, z)), row i_s = iy * n_x + ix */
  const double* weights;  /* host, n_s NURBS weights (> 0), or NULL (polynomial) */
  int32_t ctrl_dim;       /* 2 (0 reads as 2): planar S; 3: S is a surface in R^3 */
  double extrusion[3];    /* the extrusion direction a; (0, 0, 0) reads as e_z */
} lam_inplane;

/* One ply (Eq. C_layers): thickness > 0, material index, angle in radians. */
typedef struct {
  double thickness;
  int32_t material;
  double angle_rad;
} lam_ply;

/* Material-frame Voigt constants (Eq. D), upper triangle row-major. */
typedef struct {
  double C[21];
} lam_material;

/* Arithmetic of the split path (lam_options.arith). The paper's claim is
 * agreement of the split and standard matrices to machine precision (Section
 * 3, after Eq. Q), so FP64 is the default.
 *   LAM_ARITH_FP64          every product and sum of the in-plane integrals
 *                           (K-a, Eq. P), the thickness integrals (K-b, Eq. Q)
 *                           and the combine (K-c, Eq. Km_2) is an IEEE FP64
 *                           operation (DFMA / DADD);
 *   LAM_ARITH_DOUBLE_FLOAT  opt-in: the in-plane point values and Gram products
 *                           and the combine's slice arithmetic run in
 *                           double-float arithmetic (pairs of floats, error-free
 *                           products and two-sums) on the FP32 pipes, about
 *                           2^-44 relative per term instead of 2^-53, with an
 *                           FP64 re-pass when a value leaves float range.
 * Sums of partial results over elements, the thickness integrals and every
 * stored value are FP64 in both. lam_assemble_standard and
 * lam_assemble_split_noalloc are FP64 whatever this says. */
#define LAM_ARITH_FP64 0
#define LAM_ARITH_DOUBLE_FLOAT 1

/* Options; pass NULL for the defaults. */
typedef struct {
  int32_t nq_u, nq_v, nq_t; /* Gauss points per element direction; 0 = degree + 1 (Section 2.4) */
  double class_tol;         /* thickness pairs whose Q vectors (Eq. Q) agree to class_tol times the
                               largest |Q| of the same (a, b) term share one combine slice; < 0 = 1e-13,
                               0 = exact equality only */
  int32_t arith;            /* LAM_ARITH_FP64 (default) or LAM_ARITH_DOUBLE_FLOAT */
} lam_options;

/* Sizes and structure of a plan. */
typedef struct {
  int64_t n_dof;          /* 3 * n_s * n_t */
  int64_t nnz;            /* stored entries of K */
  int64_t n_s, n_t;       /* in-plane and thickness function counts */
  int64_t nnz_inplane;    /* in-plane neighbour pairs (sum over i_s of its neighbours) */
  int64_t nnz_thickness;  /* thickness neighbour pairs */
  int32_t n_configs;      /* distinct (material, angle) pairs, m-bar of Section 3.1 */
  int32_t n_classes;      /* distinct thickness slices used by the combine */
  int32_t monoclinic;     /* 1 if every configuration has D[I][J] == 0 for I < 4 <= J */
  int32_t n_pieces;       /* (thickness element, ply) pieces */
  int32_t combine_streaming; /* form of the combine: 1 streaming (one CTA per in-plane row, class slices in
                                shared memory, CSR written in address order), 0 class-major (rows of more
                                than 56 in-plane neighbours) */
  int32_t combine_chunks;    /* streaming: chunks of thickness rows whose classes fit in shared memory */
  int32_t shell;             /* 1: a general extrusion (surface in R^3 or a != e_z), see lam_inplane */
  int32_t arith;             /* LAM_ARITH_FP64 or LAM_ARITH_DOUBLE_FLOAT (lam_options.arith) */
  int32_t combine_terms;     /* streaming: (slot, configuration) terms over all chunks */
  int32_t combine_source_terms; /* ... of them evaluated by the FP64 combine of a monoclinic plate: a slot
                                   whose classes agree on the Q terms of an entry kind (Q_11, Q_22 or
                                   Q_12, Q_21) with an earlier slot of its chunk is copied from it, counted
                                   once per kind (so up to 2 combine_terms) */
  int32_t combine_block_terms; /* ... of the source terms, those of the block kind (Q_11, Q_22: entries
                                  (c, d) with c and d both in-plane or both z); the rest are off kind */
} lam_plan_info;

typedef struct lam_plan lam_plan;

/* Build a plan: validates the input, builds the 1D tables, Gauss rules,
 * (material, angle) configurations (Section 3, the reuse of P per distinct
 * configuration), thickness pieces and pair classes, and the sparsity sizes.
 * Host work only: no device memory is touched until the first device call.
 * `out` receives the plan (NULL on error). */
lam_status lam_plan_create(lam_plan** out, const lam_inplane* inplane, const lam_basis1d* thickness,
                           const lam_ply* plies, int32_t n_plies, const lam_material* materials,
                           int32_t n_materials, const lam_options* options);

/* Release the plan and its device workspace. NULL is accepted. Synchronises
 * the plan's device before freeing. */
lam_status lam_plan_destroy(lam_plan* plan);

/* Sizes of the plan (host only). */
lam_status lam_plan_get_info(const lam_plan* plan, lam_plan_info* info);

/* Sparsity pattern of K (see above). With d_row_ptr == NULL and
 * d_col_ind == NULL only *nnz_out is written (host only, no device work).
 * Otherwise d_row_ptr (n_dof + 1 int64) and d_col_ind (nnz int32) are device
 * buffers written on `stream`. nnz_out may be NULL. */
lam_status lam_pattern(lam_plan* plan, int64_t* nnz_out, int64_t* d_row_ptr, int32_t* d_col_ind, void* stream);

/* Split assembly (Section 3, Eq. Km_2 with Eq. P and Eq. Q): writes all nnz
 * FP64 values of K, in the order of lam_pattern, to the device buffer
 * d_values (nnz doubles), in the plan's arithmetic (lam_options.arith).
 * Recomputes the in-plane integrals on every call; the thickness integrals
 * (Eq. Q) depend on the plies only and are computed by the first call and by
 * the first call after each lam_plan_update. Asynchronous on `stream`. */
lam_status lam_assemble_split(lam_plan* plan, double* d_values, void* stream);

/* Standard assembly (Section 2.4, Eq. Km_0): the same matrix by
 * element-by-element 3D Gauss quadrature, into d_values (nnz doubles, device).
 * Asynchronous on `stream`. */
lam_status lam_assemble_standard(lam_plan* plan, double* d_values, void* stream);

/* Split assembly into HOST memory: the values are assembled slab by slab of
 * thickness rows in plan-owned device staging buffers and copied to h_values
 * (nnz doubles, host; pinned memory gives full copy speed) while the next
 * slab is assembled. Synchronous: returns when h_values is complete. */
lam_status lam_assemble_split_host(lam_plan* plan, double* h_values, void* stream);

/* Split assembly that allocates nothing. The paper has no counterpart: this is
 * a deployment variant of lam_assemble_split for callers that cannot call
 * cudaMalloc -- for example a host application whose device memory all comes
 * from its own pool allocator, or code that must not grow the device
 * footprint while it runs. The result equals lam_assemble_split's.
 *   - Instead of plan-owned cudaMalloc memory, the plan's tables and the
 *     in-plane and thickness workspace are placed in ONE fixed array of static
 *     device memory inside the library, LAM_NOALLOC_SCRATCH_BYTES (32 MiB)
 *     long. Every GPU that loads the library holds this array until the
 *     process exits.
 *   - The call uploads the plan's tables into the array each time (plain
 *     stream-ordered copies) and clears the part that must start at zero. It
 *     calls no cudaMalloc, cudaFree or other allocating routine.
 *   - A plan whose tables and workspace need more than the array holds is
 *     rejected with LAM_ERR_UNSUPPORTED (the message gives both sizes); the
 *     64x64 cubic 48-ply plate needs about 16 MB.
 *   - The first call on a device looks up the array's device address for that
 *     device (once per device, with that device current); make that first
 *     call before any stream capture. The address is kept for the life of the
 *     process: it does not survive cudaDeviceReset (or the destruction of the
 *     device's primary context), after which this entry point must not be
 *     called again in that process.
 *   - All calls on a device share the one array and it keeps the last call's
 *     contents: calls that overlap on the GPU (two streams, or two host
 *     threads) race and corrupt each other's results, so serialise them.
 *   - The plan's own device workspace is neither used nor created.
 * d_values: nnz doubles of caller-owned device memory. Asynchronous on `stream`. */
#define LAM_NOALLOC_SCRATCH_BYTES (32u << 20)
lam_status lam_assemble_split_noalloc(const lam_plan* plan, double* d_values, void* stream);

/* Replace the ply angles (radians, n_plies values) and material constants
 * (n_materials x 21, NULL = keep) of an existing plan, as a design loop does
 * between assemblies. Host only; the configuration table and thickness
 * classes are rebuilt. Returns LAM_ERR_INVALID_ARG if a count does not match. */
lam_status lam_plan_update(lam_plan* plan, const double* ply_angle_rad, int32_t n_plies,
                           const lam_material* materials, int32_t n_materials);

/* Cotangent of a scalar L(K) for lam_adjoint: the gradient of L with respect
 * to the stored entries of K, given either on the pattern or as a low-rank
 * product. */
typedef enum {
  LAM_COTANGENT_CSR = 0,     /* L = sum over stored (r, s) of values[k(r, s)] * K_rs */
  LAM_COTANGENT_LOWRANK = 1  /* L = sum_{q < rank} u_q^T K v_q */
} lam_cotangent_kind;

/* lam_cotangent.flags (0 = the default FP64 evaluation; the two flags exclude each other) */
#define LAM_ADJOINT_FP64 1          /* low-rank cotangents: the generic FP64 pass instead of the factorised one */
#define LAM_ADJOINT_DOUBLE_FLOAT 2  /* CSR cotangents: opt in to the double-float pass (see lam_adjoint) */

typedef struct {
  int32_t kind;          /* lam_cotangent_kind */
  int32_t rank;          /* LOWRANK: number of vector pairs, >= 1 */
  int32_t flags;         /* 0, LAM_ADJOINT_FP64 or LAM_ADJOINT_DOUBLE_FLOAT */
  int32_t reserved;      /* 0 */
  const double* values;  /* CSR: nnz doubles (device), in the order of lam_pattern */
  const double* u;       /* LOWRANK: rank x n_dof doubles (device), row-major */
  const double* v;       /* LOWRANK: rank x n_dof doubles (device), row-major */
} lam_cotangent;

/* Adjoint of the assembly: gradients of L (see lam_cotangent) with respect to
 * the material constants and the ply angles. The paper assembles K only; the
 * gradient follows from its structure: K is linear in every ply's Voigt matrix
 * D_l (Eq. Km_0), and with the split of Section 3 (Eq. Km_2, Eq. P, Eq. Q)
 *   dL/dD_l[V(c,a)][V(d,b)] += sum over stored entries of
 *       gbar^{(i_t i_s c)(j_t j_s d)} * G_ab^{i_s j_s} * Q_{l,ab}^{i_t j_t},
 * where G_ab = int g_a g_b |DF| (g = (dS/dx, dS/dy, S)) is the in-plane Gram
 * block and Q_{l,ab} Eq. Q restricted to ply l. Then, with D_l = M C_m M^T
 * (Eq. D; M the Bond matrix of the ply angle theta_l),
 *   dL/dC_m  = sum_{plies l of material m} M^T (dL/dD_l) M, folded onto the
 *              21 constants (an off-diagonal constant takes both entries);
 *   dL/dtheta_l = < dL/dD_l, M' C_m M^T + M C_m M'^T >.
 * Outputs (device, caller-owned; any of them may be NULL):
 *   d_dC      n_materials x 21 doubles, the layout of lam_material.C;
 *   d_dtheta  n_plies doubles, per radian;
 *   d_dD      n_plies x 36 doubles, dL/dD_l[I][J] row-major, every entry of
 *             D_l taken as independent.
 * Arithmetic: FP64 by default (every product and sum an FP64 operation).
 * Low-rank cotangents are contracted in factorised form (G v per thickness
 * function, then u^T (G v) per thickness pair); LAM_ADJOINT_FP64 takes them
 * through the generic pass instead. CSR cotangents take one FP64 pass over the
 * cotangent. With LAM_ADJOINT_DOUBLE_FLOAT (opt-in, CSR only) the products
 * and sums run in double-float arithmetic on the FP32 pipes (about 2^-44
 * relative per term) with FP64 partial sums, and the whole gradient is
 * recomputed in FP64 on the same stream when a partial result is not finite (a
 * cotangent entry beyond float range, an infinity or a NaN) or when no
 * cotangent entry reaches 2^-60 in magnitude; entries below 2^-80 next to
 * larger ones then contribute with an absolute error below 2^-100 of their own
 * size.
 * A general extrusion (lam_inplane.shell): every (a, b) of D_l meets all four
 * thickness types through the 6 x 6 Gram blocks G_(alpha a)(beta b); CSR
 * cotangents opting in to double-float take that pass (with the same FP64
 * re-pass rules) unless a ply meets more than 32 thickness pairs; everything
 * else takes the FP64 pass (workspace 16 * 36 * nnz_inplane bytes more).
 * The in-plane Gram blocks depend on the plan's geometry only, which never
 * changes: the first call computes them and later calls reuse them
 * (lam_inplane_operators with LAM_P_FROM_GRAM discards the copy). Workspace: about
 * 16 * 9 * nnz_inplane + 648 * n_plies * ceil(n_s / 16) bytes, plan-owned.
 * Errors: LAM_ERR_INVALID_ARG for a NULL plan or cotangent, an unknown kind, a
 * missing vector or rank < 1; LAM_ERR_UNSUPPORTED when a ply meets more than
 * 1024 thickness pairs. Asynchronous on `stream`. */
lam_status lam_adjoint(lam_plan* plan, const lam_cotangent* cotangent, double* d_dC, double* d_dtheta,
                       double* d_dD, void* stream);

/* ---------------------------------------------------------------------------
 * Batches: many laminates assembled together (the paper assembles one
 * laminate; this is the batched form of lam_assemble_split for design loops
 * over stack-ups). Instances whose in-plane discretisation is identical (basis
 * kinds, degrees, knots, control points, weights, Gauss orders) share one set
 * of in-plane Gram blocks, so K-a runs once per distinct mesh whatever the
 * materials, angles or ply counts. One launch computes Eq. Q for every
 * instance, one launch the Gram blocks of every mesh, and one persistent
 * launch combines every in-plane row of every instance from an atomic work
 * queue (largest instances first). The first lam_batch_assemble times the
 * whole sequence for every triple (thickness-chunk depth: chunks sized for 4,
 * 3 or 2 CTAs per SM; CTAs per SM 1..4 that the chunks leave room for;
 * in-plane rows per work item 1, 2 or 4), keeps the fastest, and captures it in
 * a CUDA graph that later calls replay. The chunk depth is applied to the
 * plans themselves (their thickness rows are regrouped), so their own
 * lam_assemble_split uses it too and gives the batch's values bit for bit;
 * against the default grouping the values move by rounding only (a chunk
 * shares a slice between thickness pairs whose Q agree up to rounding).
 * ------------------------------------------------------------------------- */
typedef struct lam_batch lam_batch;

typedef struct {
  int32_t n_plans;
  int32_t n_meshes;        /* distinct planar in-plane discretisations (K-a runs once for each) */
  int64_t nnz_total;       /* stored entries over all instances */
  int32_t n_persistent;    /* instances combined by the persistent launch (the others -- class-major rows,
                              general extrusions -- by lam_assemble_split after it) */
  int32_t ctas_per_sm;     /* chosen by the autotuner, 0 before the first lam_batch_assemble */
  int32_t graph;           /* 1 once the launches are replayed from a CUDA graph */
  int32_t rows_per_item;   /* chosen by the autotuner: in-plane rows of one instance per work item */
  int32_t chunk_ctas;      /* chosen by the autotuner: the CTAs per SM the thickness chunks are sized for */
  double tuned_ms[36];     /* autotuner: one assembly per candidate, [(h * 3 + r) * 4 + c - 1] for chunks
                              sized for 4, 3, 2 CTAs per SM (h = 0, 1, 2), 1, 2, 4 rows per item (r = 0, 1, 2)
                              and c CTAs per SM; 0 = not tried */
} lam_batch_info;

/* Batch of n_plans plans (borrowed: they must outlive the batch, all on the
 * current device). The batch holds their configuration as of this call: after
 * lam_plan_update on one of them, lam_batch_assemble returns
 * LAM_ERR_INVALID_ARG (recreate the batch). Allocates the shared Gram blocks
 * and the launch tables on the device. */
lam_status lam_batch_create(lam_batch** out, lam_plan* const* plans, int32_t n_plans);

/* Assembles every instance: d_values is a HOST array of n_plans device
 * pointers, entry k receiving plan k's nnz values (the order of lam_pattern).
 * Asynchronous on `stream`. The first call tunes and captures the graph with
 * the device synchronised, then replays the graph on `stream` like every later
 * call (so its values come from the configuration chosen). If the first call
 * fails while tuning (e.g. LAM_ERR_OOM when re-uploading a plan's tables), the
 * batch refuses every later call with LAM_ERR_INVALID_ARG: destroy it and
 * create a new one (the plans stay usable). */
lam_status lam_batch_assemble(lam_batch* batch, double* const* d_values, void* stream);

lam_status lam_batch_get_info(const lam_batch* batch, lam_batch_info* info);

/* Releases the batch (not its plans). Synchronises the device. */
lam_status lam_batch_destroy(lam_batch* batch);

/* In-plane operators of Eq. P for the material and angle of ply `ply`:
 * d_P receives nnz_inplane x 4 x 3 x 3 doubles (device), pair (i_s, k_s) at
 * row i_s's neighbour k_s (neighbours j_y major, j_x minor, as in the
 * pattern), blocks 11, 12, 21, 22 of Eq. P (B_1 from (S_x, S_y, 0), B_2 from
 * (0, 0, S)), each 3x3 row-major in (c, d). Two constructions:
 *   LAM_P_FROM_GRAM   the split path's: D contracted with the configuration-free
 *                     in-plane Gram blocks of K-a;
 *   LAM_P_VOIGT_FREE  Appendix A: per Gauss point, the bracket C{e_i, e_j} of
 *                     the rotated 4th-order tensor is pulled back with the
 *                     contravariant basis (C~_ab) and integrated against
 *                     parametric gradients, with no Voigt matrix and no B.
 * They agree to rounding; the second is a cross-check (FP64, one CTA per element,
 * plan-owned workspace of 288 (p+1)^4 bytes per in-plane element).
 * Asynchronous on `stream`. */
#define LAM_P_FROM_GRAM 0
#define LAM_P_VOIGT_FREE 1
lam_status lam_inplane_operators(lam_plan* plan, int32_t ply, int32_t method, double* d_P, void* stream);

/* Kernel kinds counted by the profiler. */
typedef enum {
  LAM_KERNEL_PATTERN = 0,   /* kp_row_ptr, kp_col_ind */
  LAM_KERNEL_THICKNESS = 1, /* K-b: Eq. Q per thickness pair */
  LAM_KERNEL_INPLANE = 2,   /* K-a: in-plane Gram blocks (Eq. P without D) */
  LAM_KERNEL_COMBINE = 3,   /* K-c: Eq. Km_2 into the CSR values */
  LAM_KERNEL_STANDARD = 4,  /* K-d: Section 2.4 element quadrature */
  LAM_KERNEL_ADJOINT = 5,   /* lam_adjoint: the cotangent contraction per (rows, ply) */
  LAM_KERNEL_ADJOINT_AUX = 6, /* lam_adjoint: Gram gather and scaling, FP64 re-pass check, chain rule */
  LAM_KERNEL_KINDS = 7
} lam_kernel_kind;

/* Per-plan profile: device time of every kernel launch, measured with CUDA
 * events recorded on the launching stream around each launch, plus the bytes
 * the plan moved between host and device. */
typedef struct {
  int32_t enabled;
  int64_t launches[LAM_KERNEL_KINDS];
  double ms[LAM_KERNEL_KINDS];
  int64_t h2d_bytes;
  int64_t d2h_bytes;
} lam_profile;

/* Enable (1) or disable (0) profiling of a plan's launches; either way the
 * counters restart from zero. Host only. */
lam_status lam_profile_enable(lam_plan* plan, int32_t enable);

/* Read the counters. Waits for the recorded events of pending launches (so it
 * synchronises with the streams they were recorded on). */
lam_status lam_profile_get(lam_plan* plan, lam_profile* out);

/* Message of the last error on the calling thread ("" if none). */
const char* lam_last_error(void);

/* Library version string. */
const char* lam_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LAM_H */
