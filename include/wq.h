/*
 * wq.h -- C ABI of the GB300 weighted-quadrature (WQ) library.
 *
 * Weighted quadrature on bicubic unstructured splines (Sheng, Wei, Chen,
 * "Weighted Quadrature on Unstructured Splines"): per test function N_i a
 * quadrature rule with points in the physical domain and weights fitted to the
 * Gauss-integrated moments by a truncated SVD (Sec. 4), then row-wise assembly
 *      A_ij = sum_q sum_c w^c_iq coef^c(x_q) D_c N_j(x_q)          (Eqs. 9, 11, 12)
 * into CSR.  Everything after wq_build_basis runs in hand-written CUDA kernels
 * for sm_103a on one GPU.
 *
 * Conventions
 *   - Every call returns wq_status; WQ_OK == 0.  On failure a message is
 *     available from wq_last_error(ctx) (valid until the next call on ctx).
 *     The library never traps or aborts; device-side problems (a Jacobi sweep
 *     cap, a non-finite value) come back as status codes.
 *   - Pointers named h_* are host memory, d_* device memory of the context's
 *     device.  The library copies host inputs; it never keeps or frees caller
 *     pointers.  Device views returned by the library (d_x, d_row_ptr, ...)
 *     stay valid until the owning handle is destroyed.
 *   - Indices are 0-based; CSR columns are sorted; the pattern of row i is the
 *     exactness set S_i (Eq. 10), numerically zero entries are kept.
 *   - Streams are passed as void* (a cudaStream_t; NULL = legacy default stream).
 *   - Handles are not thread-safe; use one context per host thread.
 *   - Handles may be destroyed in any order (a rule or batch keeps its device id
 *     and does not read its context when destroyed); calls on a handle whose
 *     context was destroyed are not allowed.  A CUDA error left pending by other
 *     code is cleared, not reported, by the next call that launches work.
 */
#ifndef WQ_H
#define WQ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WQ_OK = 0,
    WQ_ERR_ARG = 1,            /* bad pointer, size or option */
    WQ_ERR_MESH = 2,           /* non-quad / non-manifold mesh, EP in the boundary 1-ring, folded map */
    WQ_ERR_ILLPOSED = 3,       /* r_i < n_i after the min-max repair (Sec. 4.2) */
    WQ_ERR_NOT_CONVERGED = 4,  /* a Jacobi SVD hit its sweep cap (Sec. 4.3 solve) */
    WQ_ERR_NONFINITE = 5,      /* NaN/Inf met on the device */
    WQ_ERR_CUDA = 6,           /* a CUDA runtime call failed */
    WQ_ERR_OOM = 7,            /* device allocation failed */
    WQ_ERR_NO_DEVICE = 8       /* the context was created without a device */
} wq_status;

/* Operators (Eqs. 9, 11, 12 and the symmetric heat tangent, Eq. S). */
typedef enum {
    WQ_OP_MASS = 0,    /* sum_q w_iq c_q N_j(x_q)                                     */
    WQ_OP_STIFF = 1,   /* sum_q c_q sum_d w^d_iq d_d N_j(x_q), d over x,y (,z)         */
    WQ_OP_BIHARM = 2,  /* sum_q w^lap_iq c_q lap N_j(x_q)                              */
    WQ_OP_HEAT_S = 3,  /* alpha * MASS(c = 1) + STIFF(c), alpha = 1/(theta dt)           */
    WQ_OP_HEAT_J = 4   /* HEAT_S + sum_d sum_q w^d_iq c_{1+d,q} N_j(x_q): the exact Newton
                          tangent of the WQ heat residual (Sec. 5.2), with coefficient rows
                          c_0 = k(u), c_{1+d} = k'(u) d_d u (see wq_heat_fields)           */
} wq_op;

/* Weight / table components. */
typedef enum { WQ_COMP_N = 0, WQ_COMP_X = 1, WQ_COMP_Y = 2, WQ_COMP_Z = 3, WQ_COMP_LAP = 4 } wq_comp;

/* Precision of the assembly contraction. */
typedef enum {
    WQ_PREC_F64 = 0,      /* FP64 weights, tables and accumulation; CSR values double */
    WQ_PREC_F32 = 1,      /* FP32 split (hi/lo) products, error-free (TwoSum) accumulation; float values */
    WQ_PREC_F32_FAST = 2, /* FP32 split products, plain FP32 sums; float values; its error depends on
                             the cancellation in the rows -- measure it (wq_rule_autotune does) */
    WQ_PREC_TC = 3,       /* element blocks on the tensor cores: both operands scaled per row /
                             element and split into five 8-bit bf16 slices, slice pairs up to level 4
                             summed exactly in FP32 (integers below 2^24; error-free transformation
                             of Ozaki et al.), per-entry sums as WQ_PREC_F32; float values, error
                             ~2^-40 of each tile's largest |s| |T| K; needs <= 64 points per element */
    WQ_PREC_AUTO = 4      /* the float mode wq_rule_autotune chose for this operator and quadrature
                             (WQ_PREC_F32 until it has run); float values */
} wq_prec;

/* Kernels of the float modes (WQ_PREC_F32, WQ_PREC_F32_FAST), all with the same
 * arithmetic per element block and the same per-entry sum order: the tile engine stages
 * each 16 x 16 element block's data by bulk copies, in chunks of up to 12 points for
 * operators of one or two terms (TILE12; 8 / 4 points for 3-4 / 5-8 terms, the chunks of
 * SLOTMAP, so the values are bitwise those of SLOTMAP) or up to 16 points (TILE16; one
 * chunk per block for 4 x 4 points, so other extraction constants and values within the
 * FP32 rounding of TILE12's), then sums each CSR row from a row-major slot layout;
 * SLOTMAP is the earlier kernel pair (per-lane staged copies, blocks scattered through a
 * slot map, per-entry sums). */
typedef enum { WQ_VARIANT_TILE12 = 0, WQ_VARIANT_TILE16 = 1, WQ_VARIANT_SLOTMAP = 2 } wq_variant;

/* Point-count rule (Sec. 4.2). */
/* Per-element point counts (Sec. 4.2): the min-max rule of eq. qp_allocation, or
 * Table 2's fixed values by element type (3 x 3 / 4 x 4 near high-valence or
 * clustered EPs); both followed by the well-posedness repair. */
typedef enum { WQ_COUNT_MINMAX = 0, WQ_COUNT_TABLE2 = 1 } wq_count_mode;

typedef struct wq_ctx wq_ctx;
typedef struct wq_basis wq_basis;
typedef struct wq_rule wq_rule;
typedef struct wq_batch wq_batch;
typedef struct wq_refine wq_refine;

/* Control mesh (host arrays, copied by wq_build_basis).
 *   dim          2 = planar domain (z ignored), 3 = surface in R^3
 *   xyz          [n_vertices][3] control points of the vertex-based functions
 *   quads        [n_faces][4] vertex ids, counter-clockwise
 *   level0_face  [n_faces] index of the initial-mesh face each face descends
 *                from (-1: none), or NULL when the mesh is itself the initial
 *                mesh.  Enriched elements = descendants of initial irregular
 *                faces (Sec. 3 terminology).
 *   face_xyz     [n_face_xyz][3] positions of the face-based control points:
 *                4 per enriched face (enriched faces in ascending face order,
 *                one per corner in corner order), e.g. from wq_refine_apply;
 *                n_face_xyz must be 4 x the number of enriched faces
 *                (WQ_ERR_ARG otherwise).  NULL: each is placed at the B-spline
 *                inner Bezier point of its face (the legs between the face's
 *                vertices divided in the ratio of the knot spans), which makes
 *                the geometry away from EPs the bicubic B-spline of the vertex
 *                control points. */
typedef struct {
    int32_t dim;
    int64_t n_vertices;
    const double* xyz;
    int64_t n_faces;
    const int32_t* quads;
    const int32_t* level0_face;
    int64_t n_face_xyz;
    const double* face_xyz;
} wq_mesh_desc;

typedef struct {
    int64_t n_functions;      /* n: spline functions with support on active elements */
    int64_t n_elements;       /* E: active (non-passive) elements */
    int64_t n_irregular;      /* split 2x2 elements */
    int64_t nnz;              /* sum_i n_i = #S_i summed (Eq. 10) */
    int32_t max_m;            /* max functions on one element */
    int32_t max_n_i;          /* max #S_i */
    int64_t type_count[7];    /* passive, boundary, irregular, enriched transition,
                                 transition, enriched regular, regular (faces) */
} wq_basis_info;

typedef struct {
    uint32_t comps;           /* bit mask of (1 << wq_comp) weight sets to build */
    int32_t count_mode;       /* wq_count_mode */
    double tsvd_rel_tol;      /* keep sigma_k >= tol * sigma_max (paper: tiny sigma dropped); 1e-12 */
    int32_t max_sweeps;       /* Jacobi sweep cap (default 40 when 0) */
    void* stream;             /* stream for the build (NULL: legacy default) */
    uint32_t skip_plans;      /* wq_plan bits: assembly plans not to build (0: all) */
} wq_rule_opts;

/* Assembly plans a rule may leave out to save device memory (wq_rule_opts.skip_plans):
 * WQ_PLAN_NO_TC drops the tensor-core slices (WQ_PREC_TC then returns WQ_ERR_ARG; about
 * 15 KB per regular element), WQ_PLAN_NO_TILE the tile engine's element-major packs (the
 * float modes then use WQ_VARIANT_SLOTMAP; about 20 KB per regular element). */
typedef enum { WQ_PLAN_NO_TC = 1, WQ_PLAN_NO_TILE = 2 } wq_plan;

typedef struct {
    int64_t n_points;         /* Q: WQ points (Sec. 4.1 placement) */
    int64_t n_gauss;          /* Gauss points (4x4 per element, 4x4x4 per irregular element) */
    int64_t sum_r;            /* sum_i r_i (weights per component) */
    int32_t max_r;            /* max r_i */
    int32_t n_truncated[5];   /* per component: systems with t < n_i (rank-deficient) */
    int32_t n_z_identity[5];  /* per component: systems that used Z = I (N_i vanishes on a sub-element) */
    double setup_ms;          /* device time of the rule build */
    double tsvd_ms;           /* device time of the truncated-SVD weight solves (0 for a loaded rule) */
    double tsvd_gflop;        /* their FP64 operations, counted by the kernel (1e9) */
} wq_rule_info;

/* --- context ------------------------------------------------------------ */

/* device >= 0: bind the context to that CUDA device.  device = -1: host-only
 * context (basis construction and host queries; rule builds return
 * WQ_ERR_NO_DEVICE).  *out receives the handle, owned by the caller until
 * wq_destroy.  Errors: WQ_ERR_ARG (null out), WQ_ERR_NO_DEVICE (no such device),
 * WQ_ERR_CUDA (cudaSetDevice or the scratch lookup failed), WQ_ERR_OOM (host
 * allocation). */
wq_status wq_create(int device, wq_ctx** out);
/* Frees the context (NULL is ignored). */
void wq_destroy(wq_ctx* ctx);
/* Message of the last failed call on ctx ("null context" for NULL); the string
 * belongs to ctx and stays valid until the next call on it. */
const char* wq_last_error(const wq_ctx* ctx);

/* --- spline space (host, Sec. 3) ------------------------------------------ */

/* Classify the mesh (Sec. 3 terminology and assumptions), build the bicubic
 * unstructured spline space element by element (Bezier extraction with
 * face-based enrichment, truncation, 2x2 split and D-patch treatment at EPs,
 * Sec. 3 / Fig. 2) and the exactness-set pattern (Eq. 10).  Host only.
 * Errors: WQ_ERR_ARG (null/size), WQ_ERR_MESH (assumptions violated). */
wq_status wq_build_basis(wq_ctx* ctx, const wq_mesh_desc* mesh, wq_basis** out);
/* Frees the basis (NULL is ignored); rules built on it must be destroyed first. */
void wq_basis_destroy(wq_basis* basis);
/* Sizes and Table 1-style counts of the space (wq_basis_info).  Errors: WQ_ERR_ARG. */
wq_status wq_basis_info_get(const wq_basis* basis, wq_basis_info* info);

/* Element e (0 <= e < E) as host arrays: its face id, type (wq_basis_info order),
 * m (functions), nsub (1 or 4); fns [m] function ids ascending; coef
 * [m][nsub][4][4] Bernstein coefficients (index i along corner0->corner1,
 * j along corner0->corner3; sub-element s = su + 2 sv; the Bezier form of Sec. 3
 * / Fig. 2).  Pass NULL for arrays not wanted; call once with NULL arrays to learn
 * m and nsub.  Host arrays, caller-owned.  Errors: WQ_ERR_ARG (null basis, e out
 * of range). */
wq_status wq_basis_element(const wq_basis* basis, int64_t e, int32_t* face, int32_t* type,
                           int32_t* m, int32_t* nsub, int32_t* h_fns, double* h_coef);

/* Host copies (caller-owned arrays): control points of the functions [n][3]
 * (x = sum_j P_j N_j, Sec. 3); the exactness-set pattern (Eq. 10) row_ptr [n+1],
 * col [nnz] (NULL arrays skipped).  Errors: WQ_ERR_ARG (null basis; null h_xyz). */
wq_status wq_basis_ctrl(const wq_basis* basis, double* h_xyz);
wq_status wq_basis_pattern(const wq_basis* basis, int64_t* h_row_ptr, int32_t* h_col);

/* Positions of the face-based control points (Sec. 3, the extra DOFs of enriched
 * faces), as used by the basis (given in wq_mesh_desc.face_xyz or placed by the
 * default rule): *n_face_xyz = 4 x the number of enriched faces; h_face_xyz
 * [n_face_xyz][3] host, caller-owned (NULL: count only).  Errors: WQ_ERR_ARG. */
wq_status wq_basis_face_ctrl(const wq_basis* basis, int64_t* n_face_xyz, double* h_face_xyz);

/* Min-max point counts (Sec. 4.2, Eq. qp_allocation), or Table 2's fixed counts
 * (count_mode): side s_e of the s x s grid of every element, h_side [E] (host,
 * caller-owned).  Host only.  Errors: WQ_ERR_ARG (null argument, unknown mode),
 * WQ_ERR_ILLPOSED (r_i < n_i after the repair). */
wq_status wq_point_counts(const wq_basis* basis, int32_t count_mode, int32_t* h_side);

/* --- quadrature rule (device, Sec. 4) ---------------------------------------- */

/* Place the points (Sec. 4.1), evaluate the functions and their physical /
 * surface derivatives at WQ and Gauss points (Eqs. 13-17), build the Gauss
 * moments (Sec. 2: b precomputed) and solve every truncated-SVD weight system
 * (Sec. 4.3) on the device.  The basis must outlive the rule.
 * Errors: WQ_ERR_NO_DEVICE, WQ_ERR_OOM, WQ_ERR_CUDA, WQ_ERR_ILLPOSED,
 * WQ_ERR_NOT_CONVERGED, WQ_ERR_NONFINITE. */
wq_status wq_rule_build(wq_basis* basis, const wq_rule_opts* opts, wq_rule** out);
/* The rules of k >= 1 bases (independent mesh instances on one device) with the same
 * options, their truncated-SVD systems (Sec. 4.3) -- every row of every built
 * component of every instance -- solved in ONE persistent launch whose CTAs take
 * the systems from a queue ordered by estimated Jacobi work (n_i^2 r_i, largest
 * first), so that the uneven systems next to extraordinary points spread over the
 * GPU.  Each system is solved by the same code as in wq_rule_build, so the weights
 * are bitwise those of k separate builds.  out [k] (host, caller-owned array)
 * receives the rules, each freed by wq_rule_destroy; on error every entry is NULL
 * and nothing is kept.  wq_rule_info.tsvd_ms and tsvd_gflop of each rule report the
 * shared launch; setup_ms runs from the rule's first device step to its last.
 * The paper builds one mesh at a time; this is the batching of many.  Errors: those
 * of wq_rule_build, WQ_ERR_ARG (k < 1, null base, bases on different devices). */
wq_status wq_rule_build_batched(int32_t k, wq_basis* const* bases, const wq_rule_opts* opts, wq_rule** out);
/* Frees the rule and its device arrays (NULL is ignored). */
void wq_rule_destroy(wq_rule* rule);
/* Sizes and weight statistics (wq_rule_info).  Errors: WQ_ERR_ARG. */
wq_status wq_rule_info_get(const wq_rule* rule, wq_rule_info* info);

/* Device views owned by the rule: WQ point coordinates [Q][3] (Sec. 4.1; the
 * caller evaluates c(x_q) there), Gauss point coordinates [G][3].  Errors:
 * WQ_ERR_ARG (null rule). */
wq_status wq_rule_points(const wq_rule* rule, const double** d_x, int64_t* n_points);
wq_status wq_rule_gauss_points(const wq_rule* rule, const double** d_x, int64_t* n_gauss);

/* Device view, owned by the rule, of the CSR pattern S_i (Eq. 10; int32 row_ptr
 * [n+1], col [nnz]).  Errors: WQ_ERR_ARG (null rule). */
wq_status wq_pattern(const wq_rule* rule, int64_t* n, int64_t* nnz,
                     const int32_t** d_row_ptr, const int32_t** d_col);

/* Device view of the weights of component comp: w [sum_r], with row i's
 * weights at [w_ptr[i], w_ptr[i+1]) ordered by support element (ascending) then
 * by point (u fastest); w_ptr int64 [n+1] (Sec. 4.3 truncated-SVD weights; owned
 * by the rule).  Errors: WQ_ERR_ARG (component not built). */
wq_status wq_rule_weights(const wq_rule* rule, int32_t comp, const double** d_w, const int64_t** d_w_ptr);

/* Device view of the point tables (Sec. 4.1 evaluation): gauss = 0 for the WQ
 * points, 1 for the Gauss points.  Element e's block starts at table +
 * off[e] and is laid out [point][comp][m_e] with comp = N, d_x, d_y, (d_z),
 * lap (ncomp = dim + 2); points of e are [pt_ptr[e], pt_ptr[e+1]); Gauss
 * weights (w_g times the area element) d_gw [G] (gauss = 1 only).  Owned by the
 * rule.  Errors: WQ_ERR_ARG (null rule). */
wq_status wq_rule_table(const wq_rule* rule, int32_t gauss, const double** d_table, const int64_t** d_off,
                        const int64_t** d_pt_ptr, const double** d_gw, int32_t* ncomp);

/* Device copy of the Gauss component matrix G^c (c = 1), the moments b of
 * component comp (Sec. 2: b precomputed), into the caller's d_vals [nnz]
 * (asynchronous on stream).  Errors: WQ_ERR_ARG (component not built, null
 * d_vals), WQ_ERR_CUDA. */
wq_status wq_moments(const wq_rule* rule, int32_t comp, double* d_vals, void* stream);

/* WQ assembly (Eqs. 9, 11, 12, S):
 *   d_coef  coefficient at the WQ points (device): [Q], or [1 + dim][Q] rows for
 *           WQ_OP_HEAT_J (row 0: k(u), row 1 + d: k'(u) d_d u); null means 1
 *   alpha   scalar of WQ_OP_HEAT_S / WQ_OP_HEAT_J (ignored otherwise)
 *   prec    wq_prec; d_vals [nnz] double (F64) or float (F32), caller-owned.
 * No allocation, no host synchronisation; asynchronous on stream.  The FP32
 * modes launch two kernels (element blocks, then per-entry sums) through a
 * rule-owned slot buffer, so FP32 assemblies on one rule must not overlap on the
 * GPU.  Errors: WQ_ERR_ARG (null rule or d_vals, op not built into this rule,
 * unknown precision, WQ_PREC_TC on a rule with more than 64 points in an
 * element), WQ_ERR_CUDA (launch). */
wq_status wq_assemble(const wq_rule* rule, int32_t op, const void* d_coef, double alpha,
                      int32_t prec, void* d_vals, void* stream);

/* Same operator by element-wise 4x4 Gauss quadrature (the paper's reference,
 * Table 2 right column), coefficient at the Gauss points d_coef [G] (rows of G
 * for WQ_OP_HEAT_J); layout, ownership and errors as wq_assemble. */
wq_status wq_gq_assemble(const wq_rule* rule, int32_t op, const void* d_coef, double alpha,
                         int32_t prec, void* d_vals, void* stream);

/* u_h and grad u_h at the WQ points (Sec. 5): d_u [n] -> d_uq [Q], d_grad [Q][3]
 * (caller-owned device arrays; asynchronous on stream).  Errors: WQ_ERR_ARG (null
 * rule, d_u or d_uq), WQ_ERR_CUDA. */
wq_status wq_interp(const wq_rule* rule, const double* d_u, double* d_uq, double* d_grad, void* stream);

/* Matrix-free WQ functional (the residual form of Sec. 5; NEXT: operator apply):
 *   y_i = sum_t sum_{q in pts(supp N_i)} w^{comps[t]}_iq * g_t(x_q)
 * h_comps [n_terms] (host, wq_comp, 1 <= n_terms <= 4); d_g [n_terms][Q] point
 * data (term-major); d_y [n] (caller-owned device arrays).  No allocation;
 * asynchronous on stream.  Errors: WQ_ERR_ARG (null pointer, n_terms outside
 * 1..4, a component not built), WQ_ERR_CUDA. */
wq_status wq_apply(const wq_rule* rule, int32_t n_terms, const int32_t* h_comps, const double* d_g, double* d_y,
                   void* stream);

/* Point fields of the nonlinear heat problem (Sec. 5, theta = 1) from control
 * variables d_u, d_u_old [n]:  d_kappa [Q] = k0 + k2 u(x_q)^2 (the coefficient
 * of the tangent S, Eq. S), d_g [1 + dim][Q] with g_0 = (u - u_old)/dt - f and
 * g_{1+d} = kappa d_d u, so that wq_apply(N, x, y[, z]) gives the residual R_A
 * of Eq. heat_residual_discrete.  With jacobian != 0, d_kappa is [1 + dim][Q]
 * and rows 1 + d hold k'(u) d_d u = 2 k2 u d_d u: the coefficient rows of
 * WQ_OP_HEAT_J.  Caller-owned device arrays; no allocation; asynchronous on
 * stream.  Errors: WQ_ERR_ARG (null pointer, dt <= 0), WQ_ERR_CUDA. */
wq_status wq_heat_fields(const wq_rule* rule, const double* d_u, const double* d_u_old, double dt, double k0,
                         double k2, double f, int32_t jacobian, double* d_kappa, double* d_g, void* stream);

/* Control-variable id of every function (host) [n]: < n_vertices: the vertex
 * of a vertex-based function; otherwise n_vertices + 4 * (rank of the enriched
 * face) + corner for a face-based function (the control variables of Sec. 3).
 * Host array, caller-owned.  Errors: WQ_ERR_ARG. */
wq_status wq_basis_functions(const wq_basis* basis, int64_t* h_raw_ids);

/* Host-buffer round trip for end-to-end use: copies h_coef [Q] to the device,
 * assembles, and returns the CSR values in h_vals [nnz] (double or float by prec),
 * synchronising on stream.  When h_vals is page-locked host memory mapped into the
 * device's address space (cudaHostAlloc / cudaHostRegister under unified
 * addressing), the per-entry sums write it directly over the host link, 8 or 16
 * bytes per store where h_vals is so aligned; otherwise the values go through a
 * library-owned device buffer and one copy.  Operators with one coefficient row
 * only (not WQ_OP_HEAT_J); the operators of Eqs. 9, 11, 12, S.  Errors: those of
 * wq_assemble, WQ_ERR_ARG for WQ_OP_HEAT_J, WQ_ERR_CUDA (copies). */
wq_status wq_assemble_host(const wq_rule* rule, int32_t op, const double* h_coef, double alpha,
                           int32_t prec, void* h_vals, void* stream);

/* Batched assembly of several independent rules (many mesh
 * instances of uneven size).  wq_batch_create concatenates the element tiles of
 * k <= 256 rules (which must share the device, the weight components and the
 * dimension; the rules must outlive the batch) and uploads that plan once.
 * wq_assemble_batched then assembles operator `op` for all of them with ONE
 * launch of the element kernel and ONE launch of the per-entry sums (FP32
 * modes), reading h_coefs[r] (device pointer to rule r's coefficient at its WQ
 * points, or null) and writing h_vals[r] (device pointer, float [nnz_r]); both
 * pointer arrays are host arrays, read during the call (their contents go into
 * the launch parameters, so the call allocates nothing and may be captured in a
 * CUDA graph).  WQ_PREC_F64 and WQ_PREC_TC run one wq_assemble per rule.  The paper
 * treats one mesh at a time; this entry point is the batching of many.  Errors:
 * WQ_ERR_ARG (k out of range, mixed rules, null output, operator not built),
 * WQ_ERR_OOM, WQ_ERR_CUDA. */
wq_status wq_batch_create(int32_t k, const wq_rule* const* rules, wq_batch** out);
/* Frees the batch plan (NULL is ignored); the rules stay. */
void wq_batch_destroy(wq_batch* batch);
wq_status wq_assemble_batched(const wq_batch* batch, int32_t op, const void* const* h_coefs, double alpha,
                              int32_t prec, void* const* h_vals, void* stream);

/* Checkpoint of a rule's expensive part.  wq_rule_save writes the FP64 weights
 * of every built component, the Gauss moments and the weight statistics to a
 * binary file (native byte order), with the build options and a fingerprint of
 * the mesh (coordinates and quads).  wq_rule_load rebuilds the point plan and
 * the basis tables for `basis` (seconds less: no moment assembly and no SVD) and
 * takes the weights and moments from the file; it synchronises on the legacy
 * default stream.  The paper computes weights once and reuses them (Sec. 4.3);
 * the file format is this library's own.  Errors: WQ_ERR_ARG (cannot open or
 * write the file, not a rule file, saved for a different mesh, truncated),
 * WQ_ERR_CUDA, and the errors of wq_rule_build. */
wq_status wq_rule_save(const wq_rule* rule, const char* path);
wq_status wq_rule_load(wq_basis* basis, const char* path, wq_rule** out);

/* Kernel timing of the assembly calls.  Instrumentation with no counterpart in
 * the paper (it serves the benchmark's per-kernel roofline): capacity > 0 makes
 * the next `capacity` calls of wq_assemble / wq_gq_assemble on this rule record
 * CUDA events on their stream before the first, between the two and after the
 * second kernel they launch (FP32 paths: element blocks, then the per-entry sums;
 * FP64 paths: the single row kernel, reported as the first with a zero second).
 * Calls beyond the capacity are not recorded; capacity 0 turns recording off and
 * frees the events.  Not for calls inside a stream capture.  Errors: WQ_ERR_ARG,
 * WQ_ERR_CUDA (event creation). */
wq_status wq_rule_set_timing(wq_rule* rule, int32_t capacity);

/* Kernel choice by measurement (autotuner; no counterpart in the paper).  For
 * operator op on this rule (gauss = 0: WQ assembly, 1: Gauss assembly) and the
 * coefficient d_coef (as for wq_assemble / wq_gq_assemble): assembles once in FP64
 * and once with each candidate -- the tensor-core slices (WQ_PREC_TC), and WQ_PREC_F32
 * and WQ_PREC_F32_FAST each with every kernel variant (wq_variant) -- measures each
 * candidate's normwise error max|A - A_64| / max|A_64|, times the candidates within
 * tol on the device (CUDA events on stream; two warm-ups, then `reps` assemblies, no
 * cache flush), and records the fastest as the rule's WQ_PREC_AUTO choice for
 * (op, gauss) together with its variant (the variant the float modes then use, unless
 * wq_rule_set_variant overrides it).  *chosen = that mode, or -1 when no candidate is
 * within tol (WQ_PREC_AUTO then stays WQ_PREC_F32 with WQ_VARIANT_SLOTMAP).  h_err[3]
 * and h_ms[3] (optional) receive, per mode in the order TC, F32, F32_FAST, the error and
 * the mean time of its fastest variant (error -1: the mode is not available for this
 * rule or operator; time -1: not timed); wq_rule_autotune_report gives every candidate.
 * Allocates temporary device buffers and synchronises stream.  Errors: WQ_ERR_ARG,
 * WQ_ERR_OOM, WQ_ERR_CUDA. */
wq_status wq_rule_autotune(wq_rule* rule, int32_t op, const void* d_coef, double alpha, int32_t gauss, double tol,
                           int32_t reps, void* stream, int32_t* chosen, double* h_err, float* h_ms);

/* Kernel variant (wq_variant) of the float modes for operator op (gauss = 0: WQ
 * assembly, 1: Gauss assembly): variant -1 returns to the autotuner's choice
 * (WQ_VARIANT_TILE12 until wq_rule_autotune has run).  Host-side setting, no device
 * work.  Errors: WQ_ERR_ARG (bad op / gauss / variant; a tile variant on a rule whose
 * elements exceed the tile engine's limits: more than 240 functions or 255 points). */
wq_status wq_rule_set_variant(wq_rule* rule, int32_t op, int32_t gauss, int32_t variant);
/* The variant the float modes use now for (op, gauss).  Errors: WQ_ERR_ARG. */
wq_status wq_rule_get_variant(const wq_rule* rule, int32_t op, int32_t gauss, int32_t* variant);

/* Candidates of the last wq_rule_autotune for (op, gauss): *n = their number (0 before
 * any), and for the first `capacity` of them the mode (wq_prec), the kernel variant
 * (wq_variant; -1 for WQ_PREC_TC), the normwise error against FP64 (-1: not
 * available) and the mean time in ms (-1: not timed, its error above tol).  Host arrays,
 * caller-owned; NULL ones are skipped.  Errors: WQ_ERR_ARG. */
wq_status wq_rule_autotune_report(const wq_rule* rule, int32_t op, int32_t gauss, int32_t capacity, int32_t* n,
                                  int32_t* h_mode, int32_t* h_variant, double* h_err, float* h_ms);

/* Durations of the recorded calls in call order: h_ms[2k] and h_ms[2k + 1] are
 * the first and second kernel of call k (milliseconds); *n_calls = number of
 * recorded calls (at most max_calls are written).  Waits for the recorded events,
 * then clears the record (the capacity stays).  Errors: WQ_ERR_ARG, WQ_ERR_CUDA. */
wq_status wq_rule_kernel_times(wq_rule* rule, int32_t max_calls, float* h_ms, int32_t* n_calls);

/* Truncated-SVD weights of component comp of an existing rule, recomputed into
 * caller memory d_w [sum_r] (row i at [w_ptr[i], w_ptr[i+1]), the layout of
 * wq_rule_weights but contiguous), WITHOUT allocating: the solve's workspace is
 * a fixed 32 MiB array compiled into the library (every device that loads the
 * library holds it until exit).  The paper has no counterpart; this entry point
 * serves callers that cannot allocate device memory while they run (a host
 * program whose own pool allocator owns the free device memory, or a
 * time-critical loop where cudaMalloc's implicit synchronisation is not
 * acceptable).  wq_create, when it binds a context to a device, looks up the
 * array's device address with that device current; under lazy module loading this
 * is also when the array's memory is committed on the device, so create the context
 * before handing the free memory to another allocator.  Every call uses the same
 * array, which keeps the last call's contents; calls that overlap on the GPU race.
 * The call synchronises on stream to report the solve's status.  Errors: WQ_ERR_ARG
 * (component not built; a system needing more than 32 MiB of workspace), WQ_ERR_CUDA,
 * WQ_ERR_NOT_CONVERGED, WQ_ERR_NONFINITE. */
wq_status wq_rule_weights_noalloc(const wq_rule* rule, int32_t comp, double* d_w, void* stream);

/* --- global refinement (Sec. 3) ------------------------------------------------ */

typedef struct {
    int64_t n_vertices;          /* fine mesh vertices */
    int64_t n_faces;             /* fine mesh faces */
    int64_t n_face_xyz;          /* fine face-based control points (4 per fine enriched face) */
    int64_t n_coarse_vertices;   /* the basis's mesh vertices */
    int64_t n_coarse_face_xyz;   /* its face-based control points */
    int64_t n_stencil;           /* non-zeros of the vertex stencils */
    int64_t n_face_jobs;         /* coarse enriched faces (one de Casteljau split each) */
    int64_t n_face_fns;          /* functions over all of them (control points each job reads) */
    int64_t n_face_coef;         /* their Bezier coefficients (16 or 64 per function) */
    int64_t n_face_terms;        /* non-zero (function, fine point) terms: the de Casteljau split
                                    folded into the coefficients, 16 fine points per face */
    int64_t n_face_ell;          /* their padded device copy (16 points x an even count per face) */
} wq_refine_info;

/* Plan one global refinement of the basis's control mesh (Sec. 3: the enriched
 * region keeps its size; vertex-based control points by knot insertion,
 * face-based ones by de Casteljau's algorithm).  Host work: the fine topology,
 * the knot-insertion stencil of every fine vertex and the coefficient tables of
 * the coarse enriched elements; with a device context these are copied to the
 * device.  The plan does not keep a pointer to the basis.
 *   Topology: a face is halved in every direction whose knot span is non-zero
 *   (active faces 2 x 2, faces of the passive ring 1 x 2 along the boundary,
 *   passive corner faces whole).  Fine vertices: the coarse vertices [0, V),
 *   then one per split edge in the order the edges are first met scanning faces
 *   f = 0..F-1 and their edges k = 0..3 (edge k joins corners k and k+1), then one
 *   per 2 x 2-split face centre in face order.  Fine faces in coarse face order;
 *   the children of a 2 x 2 split are listed by the coarse corner they contain
 *   (0, 1, 2, 3), those of a 1 x 2 split by increasing coordinate; each child
 *   keeps its parent's orientation and initial-mesh face (level0_face, or the
 *   coarse face index when the basis had none).
 *   Vertex-based points: the midpoints of the non-zero knot spans are inserted
 *   along both lines of the tensor chart of the fine vertex's parent (coarse
 *   vertex, edge or face), the spans beyond the chart being the cross spans of
 *   the neighbouring faces (0 beyond the boundary); a fine vertex at an EP keeps
 *   the coarse position (the EP function is eliminated).
 *   Face-based points: the four children of an enriched face carry the inner
 *   points of the face's Bezier net split at 1/2 (for a 2 x 2-split irregular
 *   face, of its sub-nets after the D-patch treatment); fine face-based point
 *   16 r + 4 k + c is corner c of child k of the r-th coarse enriched face.
 * Where the coarse geometry is a bicubic spline with the C1 rules of the Bezier
 * nets (faces without an EP corner) the fine geometry equals the coarse one.
 * Errors: WQ_ERR_ARG, WQ_ERR_MESH (a boundary vertex without exactly two
 * boundary edges, an interior valence-4 chart that does not close, a split that
 * needs a face beyond the boundary), WQ_ERR_OOM, WQ_ERR_CUDA. */
wq_status wq_refine_create(const wq_basis* basis, wq_refine** out);
/* Frees the plan and its device tables (NULL is ignored). */
void wq_refine_destroy(wq_refine* r);
/* Sizes of the plan (wq_refine_info).  Errors: WQ_ERR_ARG (null argument). */
wq_status wq_refine_info_get(const wq_refine* r, wq_refine_info* info);

/* Host copies of the fine topology (Sec. 3 refinement, numbering as described at
 * wq_refine_create): h_quads [n_faces][4] (counter-clockwise like the coarse
 * faces), h_level0_face [n_faces]; caller-owned host arrays, NULL ones are
 * skipped.  Errors: WQ_ERR_ARG (null plan). */
wq_status wq_refine_mesh(const wq_refine* r, int32_t* h_quads, int32_t* h_level0_face);

/* Host copies of the knot-insertion stencils (Sec. 3): fine vertex w = sum over k
 * in [h_ptr[w], h_ptr[w+1]) of h_w[k] x coarse vertex h_src[k].  h_ptr
 * [n_vertices+1], h_src / h_w [n_stencil]; caller-owned host arrays, NULL ones are
 * skipped.  Errors: WQ_ERR_ARG (null plan). */
wq_status wq_refine_stencils(const wq_refine* r, int64_t* h_ptr, int32_t* h_src, double* h_w);

/* Apply the refinement on the device (one kernel on stream, no allocation, no
 * synchronisation; each fine face-based point is a short sum over the non-zero
 * terms listed at plan creation): d_xyz [n_coarse_vertices][3] and d_face_xyz
 * [n_coarse_face_xyz][3] are the coarse control points (the basis's own, or any
 * other values: the map is linear), d_xyz_fine [n_vertices][3] and
 * d_face_xyz_fine [n_face_xyz][3] receive the fine ones, ready for
 * wq_mesh_desc.xyz / face_xyz of the fine mesh.  All four are device arrays owned
 * by the caller; the face arrays may be NULL when there is no enriched face.
 * Errors: WQ_ERR_ARG, WQ_ERR_NO_DEVICE, WQ_ERR_CUDA (launch). */
wq_status wq_refine_apply(const wq_refine* r, const double* d_xyz, const double* d_face_xyz, double* d_xyz_fine,
                          double* d_face_xyz_fine, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* WQ_H */
