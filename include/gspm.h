/*
 * gspm.h - C ABI of the GB300 (sm_103a) finite-element GSPM micromagnetics library.
 *
 * The library advances the Landau-Lifshitz equation on an unstructured, periodic mesh of linear
 * tetrahedra with the Gauss-Seidel projection method (arXiv 2510.09812, App. B, Algorithm B.1),
 * coupled to magnetostatics (Sec. 2.1, Eq. demag, weak form (a)) and to mechanical equilibrium
 * with magnetostrictive eigenstrain (Eq. elasticity, weak form (b), Table A.1).  Every step of the
 * path runs in the library's own CUDA kernels; there is no CPU fallback.
 *
 * Conventions
 * -----------
 * - Every function returns an int status (GSPM_OK = 0 or one of GSPM_E*); nothing throws across
 *   the ABI.  gspm_last_error() returns a human-readable message for the calling thread's most
 *   recent failure.
 * - "Node order" in this header is the library's unique-node numbering: after the periodic wrap
 *   (Sec. 2.5) each set of matching stored nodes becomes one unique node, numbered in order of
 *   first appearance in the stored-node array.  Internally the library may renumber nodes
 *   (reverse Cuthill-McKee); that order never crosses the ABI.
 * - Nodal vector fields are arrays of structures: [n_unique][3] (m, u, fields), float64.
 * - `where` = GSPM_HOST for host pointers (the library stages the copy) or GSPM_DEVICE for device
 *   pointers visible to the context's device.  Device-pointer calls are asynchronous on the
 *   context's stream unless stated otherwise; host-pointer calls synchronise that stream.
 * - The library owns all device memory it allocates; the caller owns every pointer it passes
 *   and may free it once the call returns (host) or once the stream has passed the call (device).
 * - A context is not thread-safe: one host thread at a time per context.
 */
#ifndef GSPM_H
#define GSPM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GSPM_API __attribute__((visibility("default")))
#else
#define GSPM_API
#endif

/* ---- status codes ---------------------------------------------------------------------- */
#define GSPM_OK 0
#define GSPM_EINVAL 1    /* bad argument (null pointer, size, enum)                            */
#define GSPM_EMESH 2     /* invalid mesh: index out of range, det(J) <= 0, non-finite coords,
                            a tetrahedron collapsed by the periodic wrap                        */
#define GSPM_ENOMEM 3    /* device or host allocation failed                                    */
#define GSPM_ECUDA 4     /* a CUDA runtime call failed (message has the CUDA error string)      */
#define GSPM_ENOCONV 5   /* a CG solve hit max_iter; the state was still advanced (best iterate) */
#define GSPM_ETIMEOUT 6  /* a bounded device-side wait gave up                                  */
#define GSPM_ESTATE 7    /* call not valid for this context (e.g. host-only context)           */
#define GSPM_ENUMERIC 8  /* a step produced a non-finite or zero m** at a magnetic node (for
                            example from non-finite input); the state is not valid             */

/* ---- enums ------------------------------------------------------------------------------ */
#define GSPM_HOST 0
#define GSPM_DEVICE 1

#define GSPM_PREC_F64 0    /* plain double precision everywhere                               */
#define GSPM_PREC_MIXED 1  /* FP32 matrices, vectors, SpMV, assembly and pointwise work; FP64
                              CG scalars (inner products, residual norms, alpha, beta) and
                              volume averages                                                   */

#define GSPM_ORDER_NONE 0  /* keep the unique-node numbering                                   */
#define GSPM_ORDER_RCM 1   /* reverse Cuthill-McKee renumbering (tie-breaks documented below)  */
#define GSPM_ORDER_AGGREGATE 2 /* nodes grouped by the aggregates of the two-level preconditioner
                              (coordinate bins of coarse_nodes nodes, see gspm_options): bins in
                              x-fastest order, unique index ascending within a bin.  Each
                              aggregate is then a contiguous range of rows, which the
                              restriction reads in order                                       */

#define GSPM_FLAG_HOST_ONLY 1u        /* build host structures only (mesh, node graph,
                                         assembly and, unless PINNED_CG or PLAIN_CG, the
                                         two-level preconditioner's coarse operators and their
                                         inverses); no CUDA call is made                      */
#define GSPM_FLAG_ROW2_PRINTED 2u     /* Algorithm B.1 second row exactly as printed (m^n_1,
                                         g^n_1) instead of the Gauss-Seidel sweep (m*_1, g*_1)  */
#define GSPM_FLAG_NO_AUTOTUNE 4u      /* skip the SpMV schedule autotuner (schedule 0)          */
#define GSPM_FLAG_GRAPH 8u            /* gspm_step / gspm_batch_step replay one captured CUDA
                                         graph per step (see gspm_set_graph)                    */
#define GSPM_FLAG_RESOLVE_AT_MSTAR 32u /* Algorithm B.1 step 3: solve the magnetostatic and
                                         mechanical equilibria again at m* (x0 = the step-n
                                         solutions) so that h[m*] is the whole effective field
                                         of m*.  Default: h~_d and E held from step n.  With
                                         the flag, the state's U and u after a step are the
                                         solutions at m*, it_ms / it_mech count both solves of
                                         a step and *_last report the solves at m*          */
#define GSPM_FLAG_PLAIN_CG 64u        /* unpreconditioned CG for K^ms and K^mech, as in the paper
                                         (Sec. 3.1).  Default (singular form only): CG with the
                                         two-level preconditioner z = D^-1 r + P A_c^-1 P^T r,
                                         D = diag(K), P = plain aggregation of the nodes into
                                         coordinate bins of max(512, n/6000) nodes (the same
                                         for each component), A_c = P^T K P made definite on
                                         the constants and inverted densely at load.  The
                                         stopping test stays ||r|| < rtol ||b||, so the
                                         solution is the unpreconditioned one to tolerance.
                                         The GSPM solves (M + c eps K) g = M f use Jacobi
                                         (z = D^-1 r) unless this flag or PINNED_CG is set    */
#define GSPM_FLAG_PINNED_CG 16u       /* solve K^ms U = b and K^mech u = b as the pinned systems of
                                         Sec. 2.5 (node 0's rows and columns replaced by the
                                         identity, its right-hand side zeroed).  Default: the
                                         equivalent consistent singular systems on the periodic
                                         mesh (b minus its mean per component, CG on the
                                         unpinned K, then the constant that makes the pinned
                                         node zero subtracted): the same solution in exact
                                         arithmetic, with far fewer CG iterations, since
                                         pinning one node of a periodic body leaves an
                                         eigenvalue of order 1/n.  The singular form runs
                                         projected off the constants (x0, r.r and every search
                                         direction without their per-component means), which
                                         keeps FP32 rounding of K 1 from steering the iteration
                                         along the constants.  Stopping test of either form:
                                         ||r|| < rtol ||b||, with its own r and b (the
                                         projected r for the singular form)                   */

/* ---- inputs ----------------------------------------------------------------------------- */
typedef struct gspm_mesh_desc {
  int64_t n_nodes;               /* stored nodes (periodic images included)                    */
  const double* coords;          /* host, [n_nodes][3], nm                                      */
  int64_t n_tets;                /* elements                                                    */
  const int32_t* tets;           /* host, [n_tets][nodes_per_elem], stored-node indices         */
  const uint8_t* elem_magnetic;  /* host, [n_tets]: 1 ferromagnetic host, 0 defect; NULL = all 1 */
  double box_lo[3], box_hi[3];   /* periodic box (nm); faces at box_hi wrap onto box_lo         */
  double wrap_tol;               /* nm; <= 0 selects 1e-6 x the shortest element edge           */
  int32_t nodes_per_elem;        /* 4 (or 0): linear tetrahedra, det J > 0; 8: linear
                                    (trilinear) hexahedra, vertices at reference corners
                                    (-,-,-) (+,-,-) (+,+,-) (-,+,-) (-,-,+) (+,-,+) (+,+,+)
                                    (-,+,+) in that order, det J > 0 at the 2x2x2 Gauss points,
                                    integrals by 2x2x2 Gauss quadrature (Sec. 2.4)             */
} gspm_mesh_desc;

typedef struct gspm_material {
  double Ms;          /* saturation magnetisation m_s, A/m                                     */
  double A;           /* exchange coefficient, J/m                                              */
  double K1;          /* cubic anisotropy kappa_1, J/m^3                                        */
  double lambda100;   /* magnetostriction constants (Table A.1)                                */
  double lambda111;
  double C11, C12, C44;  /* cubic elastic stiffness, Pa                                         */
  double Nd[9];       /* demagnetising tensor of the enclosing ellipsoid (row-major)           */
  double sigma_ext[6];/* external stress, Voigt order 11,22,33,23,13,12, Pa                     */
  double gamma0;      /* mu0 * gyromagnetic ratio, m/(A s); <= 0 selects 2.2127615e5            */
  double mu0;         /* H/m; <= 0 selects 1.25663706212e-6                                     */
  double l_d;         /* model length scale (m) = unit of the mesh coordinates; <= 0 -> 1e-9   */
  double R[9];        /* App. D rotated crystal: v_mesh = R v_crystal (row-major; the rows are
                         the crystal directions of the mesh axes, e.g. <111>, <-110>, <11-2>).
                         All zero = identity (mesh axes = cube axes).  Must be a proper rotation
                         to 1e-12, else GSPM_EINVAL.  C, E0(m), the anisotropy and the
                         magnetoelastic field are then evaluated as Algorithm D.1 states;
                         H_ext, N_d, sigma_ext and all fields at the ABI are in the mesh axes  */
} gspm_material;

typedef struct gspm_options {
  int precision;      /* GSPM_PREC_*                                                           */
  int ordering;       /* GSPM_ORDER_*                                                          */
  double dt;          /* time step, s (Delta tau = gamma0 m_s dt)                              */
  double alpha;       /* damping constant                                                       */
  double rtol_gs;     /* relative residual targets of the three CG families (Sec. 3.1: 1e-7) */
  double rtol_ms;
  double rtol_mech;
  int max_iter;       /* per CG solve; exceeding it returns GSPM_ENOCONV                       */
  unsigned flags;     /* GSPM_FLAG_*                                                           */
  int64_t coarse_nodes; /* nodes per aggregate of the two-level preconditioner (0: the default
                         max(512, n / 6000), n the mesh's nodes); sets the coarse problem size
                         (3 n / coarse_nodes for K^mech), whose dense inverse is formed at load:
                         smaller aggregates cut CG iterations, cost load time (cubic in the
                         coarse size) and coarse-product traffic per iteration (quadratic)   */
  void* stream;       /* cudaStream_t for all work of the context; NULL = legacy default stream */
} gspm_options;

/* ---- outputs ---------------------------------------------------------------------------- */
#define GSPM_SPMV_SCHEDULES 4

typedef struct gspm_mesh_info {
  int64_t n_stored, n_unique, n_tets, n_magnetic_nodes, n_magnetic_tets;
  int64_t nnz;             /* node-graph nonzeros (self included)                              */
  int64_t sell_entries;    /* padded SELL-32 entries                                           */
  double volume;           /* V(Omega_c), nm^3                                                 */
  double volume_magnetic;  /* V(Omega_m), nm^3                                                 */
  double eps;              /* A* Delta tau (nm^2), operator (1 - eps Lap) of Algorithm B.1     */
  double dtau;             /* gamma0 m_s dt                                                    */
  int64_t device_bytes;    /* device memory held by the context                               */
  int n_segments;          /* meshes in the context (1 unless loaded with gspm_batch_load)     */
  int item_slices;         /* slices per work item of a reducing kernel at one block per SM   */
  int spmv_schedule_block; /* SpMV schedule the autotuner chose for the 3x3-block operator:
                              0 thread per row, 1 thread per row with 5-deep load prefetch,
                              2 two threads per row, 3 = 1 with registers capped for three
                              resident blocks per SM                                            */
  int spmv_schedule_scalar;/* ... and for K^ms                                                */
  double spmv_ms_block[GSPM_SPMV_SCHEDULES]; /* ms per launch of each schedule as the CG loop
                              runs it (product fused with p.Ap; 0 = not tuned)                 */
  double spmv_ms_scalar[GSPM_SPMV_SCHEDULES];
  int64_t n_aggregates;    /* aggregates of the two-level preconditioner, all meshes (0: none) */
  double coarse_shift_ms, coarse_shift_mech;
                           /* diagonal shift added to the coarse inverses before their rounding
                              to the device storage to keep them positive definite (largest over
                              the meshes; 0 when the rounded inverse is positive definite as it
                              is, see gspm_coarse_round)                                      */
  int spmv_schedule_gs;    /* schedule chosen for the GSPM operators M + c eps K               */
  double spmv_ms_gs[GSPM_SPMV_SCHEDULES]; /* summed ms of one launch with 1, 2 and 3 right-hand
                              sides, per schedule                                              */
} gspm_mesh_info;

typedef struct gspm_step_stats {
  int64_t steps;           /* steps taken by the call                                          */
  int64_t it_ms, it_mech;  /* CG iterations summed over the call                               */
  int64_t it_gs;           /* summed over the seven GSPM solves of every step                  */
  int it_ms_last, it_mech_last;
  int it_gs_last[8];       /* per GSPM solve of the last step, in solve order (7 for the
                              Gauss-Seidel sweep, 8 with GSPM_FLAG_ROW2_PRINTED)            */
  double res_ms_last, res_mech_last;  /* final recursive relative residuals of the last step   */
  double dm_last;          /* <|m^{n+1} - m^n|> over magnetic nodes, last step                 */
  double m_bar[3];         /* volume average of m over Omega_c before the last step            */
  int noconv;              /* number of solves that hit max_iter                               */
  double true_res_ms_last, true_res_mech_last;
                           /* true relative residuals ||b - K x|| / ||b|| of the last K^ms and
                              K^mech solves, recomputed from b and the final x after the solve
                              (rows other than the pinned one, K x accumulated in FP64 against the
                              operator as stored: FP32 under GSPM_PREC_MIXED); -1 unless enabled
                              with gspm_set_true_residual                                       */
} gspm_step_stats;

/* mesh export selectors (host copies of host-side structures; see gspm_mesh_export) */
#define GSPM_EXPORT_UNIQUE_OF_STORED 0  /* int64 [n_stored]                                    */
#define GSPM_EXPORT_ROWPTR 1            /* int64 [n_unique + 1], unique-node order             */
#define GSPM_EXPORT_COLS 2              /* int64 [nnz], ascending per row, unique-node order   */
#define GSPM_EXPORT_PERM 3              /* int64 [n_unique], perm[internal] = unique index     */
#define GSPM_EXPORT_NODE_MAGNETIC 4     /* uint8 [n_unique]                                    */
#define GSPM_EXPORT_LUMPED_MASS 5       /* double [n_unique], M_L,i = sum_e int_e N_i (V_e / 4
                                           on a tetrahedron, a 2x2x2 Gauss sum on a hexahedron) */
#define GSPM_EXPORT_AGGREGATES 6        /* int32 [n_unique] preconditioner aggregate per node   */
#define GSPM_EXPORT_COARSE_K_MS 7       /* double [n_agg^2] P^T K^ms P (unpinned K), row-major  */
#define GSPM_EXPORT_COARSE_K_MECH 8     /* double [(3 n_agg)^2] P^T K^mech P, index 3 I + a     */
#define GSPM_EXPORT_COARSE_INV_MS 9     /* double [n_agg^2] inverse of P^T K^ms P + rho 1 1^T    */
#define GSPM_EXPORT_COARSE_INV_MECH 10  /* double [(3 n_agg)^2] inverse of P^T K^mech P plus rho
                                           on each component's constants (rho = trace / (3 n_agg)
                                           / n_agg); the FP64 inverses before rounding to the
                                           device storage, kept by host-only contexts only     */
#define GSPM_EXPORT_COARSE_STORED_MS 11   /* double [n_agg^2] the K^ms coarse inverse as the device
                                           stores it (gspm_coarse_round of the inverse: BF16
                                           values under GSPM_PREC_MIXED), widened to FP64;
                                           host-only contexts only                             */
#define GSPM_EXPORT_COARSE_STORED_MECH 12 /* double [(3 n_agg)^2] the same for K^mech          */

/* fields readable / writable with gspm_get_field / gspm_set_field (unique-node order) */
#define GSPM_FIELD_M 0       /* [n][3] magnetisation m (non-magnetic nodes forced to 0)       */
#define GSPM_FIELD_U 1       /* [n]    reduced magnetostatic potential U = U~/m_s (nm)         */
#define GSPM_FIELD_DISP 2    /* [n][3] displacement u (nm)                                     */
#define GSPM_FIELD_HD 3      /* [n][3] local demagnetising field -grad U (reduced), read only  */
#define GSPM_FIELD_STRAIN 4  /* [n][6] total strain E, Voigt 11,22,33,23,13,12 (tensor shear), read only */
#define GSPM_FIELD_H 5       /* [n][3] local field h(m^n) of the last step (reduced), read only */
#define GSPM_FIELD_DISP_PREV 6 /* [n][3] displacement of the solve before the last (history of
                                  the extrapolated and learned initial guesses)                 */

/* initial guess of the mechanical CG inside gspm_step (gspm_set_x0_mode) */
#define GSPM_X0_PREV 0         /* previous step's displacement (default)                      */
#define GSPM_X0_ZERO 1         /* cold start                                                   */
#define GSPM_X0_EXTRAPOLATE 2  /* 2 u_prev - u_prev2                                           */
#define GSPM_X0_LEARNED 3      /* 2 u_prev - u_prev2 + u_s * MPNN(features), see gspm_mpnn_*   */

/* operators for gspm_apply (per-kernel access; y = Op x in unique-node order, host or device) */
#define GSPM_OP_K_MS 0       /* pinned K^ms (Eq. LHS), scalar                                  */
#define GSPM_OP_A_EPS 1      /* M + eps K over Omega_m (identity rows off Omega_m), scalar     */
#define GSPM_OP_A_AEPS 2     /* M + alpha eps K over Omega_m, scalar                          */
#define GSPM_OP_M 3          /* consistent mass over Omega_m (F^GS of Eq. RHS_F), scalar      */
#define GSPM_OP_K_MECH 4     /* pinned K^mech (Eq. LHS), x and y [n][3]                        */
#define GSPM_OP_DIV 5        /* b_i = F^ms_{ij,a} x_{j,a}: x [n][3] -> y [n] (pinned entry 0)  */
#define GSPM_OP_GRAD 6       /* y_{i,a} = (F^ms_a x)_i / M_L,i = -(d_a x)_i: x [n] -> y [n][3] */

/* ---- lifecycle -------------------------------------------------------------------------- */

/* Validate the mesh, apply the periodic wrap (Sec. 2.5: a node on a maximum face is identified
 * with the node at the matching minimum-face position through a hash map of quantised wrapped
 * coordinates floor((x - lo)/tol + 0.5)), build the node graph, optionally renumber it (RCM: start
 * at the unvisited node of smallest degree, lowest index on ties; breadth-first, neighbours in
 * (degree, index) order; all components; reversed), compute element geometry, assemble
 * K^ms, K^mech, K^GS = M + eps K, F^ms, F^mech, F^GS (Eqs. LHS, RHS_F) in SELL-32 form, pin node 0
 * (one DOF of K^ms, three of K^mech), upload everything to the current CUDA device, and set
 * m = 0, U = 0, u = 0.  Errors: GSPM_EINVAL (null/size), GSPM_EMESH, GSPM_ENOMEM, GSPM_ECUDA. */
GSPM_API int gspm_mesh_load(const gspm_mesh_desc* mesh, const gspm_material* mat,
                            const gspm_options* opt, struct gspm_ctx** out);

/* Load several meshes into one context (a batch, e.g. meshes of uneven size or defect
 * geometry): each mesh is prepared as by gspm_mesh_load and the batch is stored slice-aligned in
 * one structure, so that one kernel sequence advances every mesh.  All meshes share the
 * material and options; each keeps its own pin, volume averages, applied field and CG
 * convergence (a mesh whose CG converged stops iterating while the others continue).
 * Node numbering of the batch at the ABI: mesh 0's unique nodes, then mesh 1's, and so on
 * (gspm_batch_segment gives each mesh's offset and count); fields are [sum n][...].
 * gspm_volume_avg returns n_meshes x ncomp values; gspm_step applies one field to every mesh
 * and its stats argument points to n_meshes structures; gspm_mesh_export is single-mesh only;
 * the learned initial guess is single-mesh only. */
GSPM_API int gspm_batch_load(const gspm_mesh_desc* meshes, int n_meshes, const gspm_material* mat,
                             const gspm_options* opt, struct gspm_ctx** out);

/* First ABI node and node count of mesh `seg` of a batch. */
GSPM_API int gspm_batch_segment(const struct gspm_ctx* ctx, int seg, int64_t* node_offset,
                                int64_t* n_nodes);

/* gspm_step with one applied field per mesh: H_ext = [n_meshes][3] (A/m, host); stats (may be
 * NULL) = [n_meshes]. */
GSPM_API int gspm_batch_step(struct gspm_ctx* ctx, int n_steps, const double* H_ext,
                             gspm_step_stats* stats);

/* Free every resource of the context (waits for its stream). NULL is a no-op. */
GSPM_API void gspm_destroy(struct gspm_ctx* ctx);

/* Message of the calling thread's most recent failure ("" if none). */
GSPM_API const char* gspm_last_error(void);

GSPM_API int gspm_mesh_info_get(const struct gspm_ctx* ctx, gspm_mesh_info* out);

/* Copy a host-side structure (GSPM_EXPORT_*) into host memory `out` of `count` elements; count
 * must equal the structure's length.  Works on host-only contexts. */
GSPM_API int gspm_mesh_export(const struct gspm_ctx* ctx, int what, void* out, int64_t count);

/* ---- state ------------------------------------------------------------------------------ */

/* Set / read a nodal field (GSPM_FIELD_*), float64, unique-node order.  Setting M forces m = 0
 * at nodes outside Omega_m (the caller supplies unit vectors elsewhere). */
GSPM_API int gspm_set_field(struct gspm_ctx* ctx, int field, const double* data, int where);
GSPM_API int gspm_get_field(struct gspm_ctx* ctx, int field, double* data, int where);

/* ---- the hot path ----------------------------------------------------------------------- */

/* Advance n_steps GSPM steps in place under the applied field H_ext (A/m, host array of 3).
 * One step (App. B, Algorithm B.1, with Sec. 2.1-2.4):
 *   m_bar (Sec. 2.4) -> b^ms = F^ms m (Eq. RHS_b) -> CG for K^ms U = b^ms with U = 0 at the
 *   pinned node (GSPM_FLAG_PINNED_CG says how), x0 = previous U
 *   -> h~_d = -grad U (F^ms / lumped mass) -> E0(m) (Table A.1), E_bar = <E0> + C^-1 sigma_ext
 *   -> b^mech = F^mech E0 -> CG for K^mech u = b^mech, u = 0 at the pinned node, x0 = previous
 *   u -> E = E_bar + sym grad u
 *   -> h(m^n) = h_anis + H/m_s + h_me + h~_d - N_d m_bar
 *   -> Gauss-Seidel stages with (M + eps K) g = M f (x0 = f), giving m*
 *   -> h(m*) (local terms and far field at m*, h~_d and E held) -> (M + alpha eps K) m** = M f
 *   -> m = m** / |m**| on magnetic nodes.
 * The call synchronises with its stream before returning.  Returns GSPM_ENOCONV if any solve
 * hit max_iter (the state is still advanced), GSPM_ENUMERIC if a projection met a non-finite or
 * zero m** at a magnetic node (the state is then not valid). */
GSPM_API int gspm_step(struct gspm_ctx* ctx, int n_steps, const double H_ext[3],
                       gspm_step_stats* stats);

/* Mechanical equilibrium alone (steps E0 .. strain of gspm_step) for magnetisation m ([n][3],
 * `where`); writes the displacement to u ([n][3], `where`, may be NULL) and keeps it as the
 * context's u (the former u becomes u_prev2).  x0_mode: 0 = zero, 1 = the context's u, 2 = the
 * array x0 ([n][3], `where`), 3 = extrapolation 2u - u_prev2, 4 = learned (gspm_mpnn_*).  rtol
 * <= 0 uses the context's rtol_mech.  iters / relres may be NULL.  Does not change the context's
 * m.  Synchronises the stream. */
GSPM_API int gspm_solve_elastic(struct gspm_ctx* ctx, const double* m, double* u, int where,
                                int x0_mode, const double* x0, double rtol, int* iters,
                                double* relres);

/* Volume average over Omega_c (Sec. 2.4) of a nodal field with ncomp (1..9) interleaved
 * components, [n][ncomp] float64 at `where`; result in out_host[ncomp] (per mesh of a batch:
 * out_host[n_meshes][ncomp]).  Quadrature of the P1
 * interpolant: sum_e V_e (1/4) sum_{k in e} g_k / V = sum_i (M_L,i / V) g_i.  FP64 accumulation
 * with a fixed reduction order (bitwise reproducible for a given device).  Synchronises. */
GSPM_API int gspm_volume_avg(struct gspm_ctx* ctx, const double* field, int where, int ncomp,
                             double* out_host);

/* y = Op x for one assembled operator (GSPM_OP_*), in the context's precision.  Synchronises
 * when where = GSPM_HOST. */
GSPM_API int gspm_apply(struct gspm_ctx* ctx, int op, const double* x, double* y, int where);

/* Number of CUDA kernels the context has launched since creation (host-side counter). */
GSPM_API int64_t gspm_launch_count(const struct gspm_ctx* ctx);

/* Storage rule of the two-level preconditioner's dense coarse inverse (host code, no GPU): the
 * symmetric part of A ([n][n] row-major, symmetric positive definite) rounded entry by entry to
 * bfloat16 (bf16 = 1: round to nearest even of the FP32 value; mixed precision) or kept in FP64
 * (bf16 = 0), into out [n][n] as FP64 values.  The rounded matrix is accepted only if a Cholesky
 * factorisation of it (in FP64) succeeds, so the preconditioner stays symmetric positive
 * definite and the CG's r.z stays positive; otherwise a diagonal shift s is added before
 * rounding (2^-8 max_i A_ii, doubled until accepted, at most max_i A_ii) and returned in *shift
 * (0 if none was needed; may be NULL).  mesh_load applies this rule to every coarse inverse.
 * The paper has no coarse level; this is part of the library's preconditioner (its Sec. 5 names
 * preconditioning as the next step).  Errors: GSPM_EINVAL (null pointer, n < 1, bf16 not 0/1),
 * GSPM_EMESH (no shift up to max_i A_ii is accepted: A is not positive definite). */
GSPM_API int gspm_coarse_round(const double* A, int64_t n, int bf16, double* out, double* shift);

/* ---- allocation-free variant ------------------------------------------------------------ */

/* Volume average without any device allocation, for callers that cannot call cudaMalloc (for
 * example code confined to another framework's fixed memory pool, or real-time loops and host
 * callbacks that must not take cudaMalloc's implicit device synchronisation).  The paper has no
 * counterpart; this is the reduction of gspm_volume_avg with caller-supplied weights.
 *
 * out[c] = sum_i weights[i] * field[i*ncomp + c], c < ncomp, accumulated in FP64 with a fixed
 * reduction order.  field ([n][ncomp]), weights ([n]) and out ([ncomp]) are float64 DEVICE
 * pointers owned by the caller; weights = M_L,i / V(Omega_c) (GSPM_EXPORT_LUMPED_MASS divided
 * by gspm_mesh_info.volume) gives the Sec. 2.4 volume average.  The call is asynchronous on
 * `stream` (a cudaStream_t, NULL = legacy default stream); it allocates nothing and calls no
 * cudaMalloc/cudaFree.
 *
 * Scratch: a file-scope __device__ array of GSPM_NOALLOC_MAX_BLOCKS x 16 doubles plus a counter
 * (about 256 KiB) that every GPU loading the library holds until the process exits.  The first
 * call on a device looks up that array's device address (cudaGetSymbolAddress, with the device
 * current) and caches it; make that first call before any stream capture.  Every call shares the
 * array and it keeps the last call's partial sums; the arrival counter is cleared on `stream` at
 * the start of each call.  Calls whose kernels overlap on the GPU (different streams, or
 * different host threads) race on the scratch and give wrong results: serialise them.
 * Errors: GSPM_EINVAL for null pointers, n <= 0 or ncomp outside 1..GSPM_NOALLOC_MAX_COMP;
 * GSPM_ECUDA if the symbol lookup, the counter clear or the launch fails. */
#define GSPM_NOALLOC_MAX_COMP 9
#define GSPM_NOALLOC_MAX_BLOCKS 2048
GSPM_API int gspm_volume_avg_noalloc(const double* field, const double* weights, int64_t n,
                                     int ncomp, double* out, void* stream);

/* ---- learned warm start of the mechanical CG ------------------------------------------- */
/* A message-passing network over the mesh (the paper has none; this is the library's learned
 * initial guess, checked against its own FP64 CPU definition).  Per node, 16 features:
 * m (3), E0(m) in Voigt order / lambda_s (6), u_prev / u_s (3), (u_prev - u_prev2) / u_s (3), 1,
 * with lambda_s = max(|lambda100|, |lambda111|) and u_s = lambda_s * (V(Omega_c)/n)^(1/3).
 * h0 = relu(f W_in + b_in); three layers h_l = relu([h, A h] W_l + b_l) with A the
 * element-message average (A_ij = sum_{e containing i,j} V_e / k over sum_{e containing i} V_e,
 * k the element's vertices; V_e / (16 M_L,i) on tetrahedra); y = h3 W_out + b_out.
 * Prediction x0 = 2 u_prev - u_prev2 + u_s y.  Inference runs on the tcgen05 tensor cores (BF16
 * weights and activations, FP32 accumulation in tensor memory); a layer whose wait for its
 * accumulator gives up makes the call (or the step that used the guess) return GSPM_ETIMEOUT.
 * Training (backward, Adam) runs in FP32.  CG still runs to the same residual, so the
 * prediction only changes the iteration count.
 * Parameter layout (float32, GSPM_MPNN_PARAMS values): W_in [16][64], b_in [64],
 * {W_l [128][64], b_l [64]} for l = 1..3, W_out [64][3], b_out [3]; all row-major [in][out]. */
#define GSPM_MPNN_PARAMS 26051

/* Graph replay of the time step (on != 0) or direct launches (0, the default unless the context
 * was loaded with GSPM_FLAG_GRAPH).  The paper has no counterpart: it is how the step is issued,
 * not what it computes; results are bitwise those of direct launches.  In graph mode the first
 * gspm_step / gspm_batch_step (and the first after a change of initial-guess mode) captures one
 * step into a CUDA graph on private streams; each CG loop is a conditional WHILE node whose
 * body (SpMV with p.q, update with r.r, p-update) repeats until the device-side count of
 * unconverged meshes reaches zero, with max_iter + 2 iterations as a hard limit.  A call of n
 * steps is then n graph launches on the context's stream and one synchronisation at the end,
 * with no host round trip inside a step.  The graph holds the context's buffers and stream
 * ordering only, so it stays valid across gspm_set_field calls.  While kernel-class profiling is
 * enabled (gspm_profile_enable) steps run directly.  Capture does not allocate device memory
 * beyond a few counters made at the first capture.  Errors: GSPM_ESTATE for host-only contexts,
 * GSPM_ECUDA if capture or instantiation fails (the step is then not run). */
GSPM_API int gspm_set_graph(struct gspm_ctx* ctx, int on);

/* Recompute the true residual ||b - K x|| / ||b|| of every K^ms and K^mech solve after it ends
 * (on != 0) and report the last ones in gspm_step_stats; off (0) by default.  The CG stopping test
 * (Sec. 2.5, relative residual 1e-7 in Sec. 3.1) uses the residual that the CG recursion
 * carries, which drifts from b - K x in finite precision; this call measures the drift.  It adds
 * one FP64-accumulated product with K per solve.  In graph mode the next step captures the graph
 * again.  Errors: GSPM_ESTATE for host-only contexts. */
GSPM_API int gspm_set_true_residual(struct gspm_ctx* ctx, int on);

/* Change the relative residual targets of the GSPM, K^ms and K^mech solves (gspm_options.rtol_*;
 * Sec. 3.1 uses 1e-7) for the following steps; a value <= 0 keeps that tolerance.  In graph mode
 * the next step captures the graph again.  Errors: GSPM_EINVAL for a tolerance >= 1,
 * GSPM_ESTATE for host-only contexts. */
GSPM_API int gspm_set_rtol(struct gspm_ctx* ctx, double rtol_gs, double rtol_ms, double rtol_mech);

/* Select the mechanical CG's initial guess for gspm_step (GSPM_X0_*); GSPM_X0_LEARNED needs
 * parameters (GSPM_ESTATE otherwise). */
GSPM_API int gspm_set_x0_mode(struct gspm_ctx* ctx, int mode);

/* Copy the network parameters in (host float32 [GSPM_MPNN_PARAMS]; resets Adam) or out. */
GSPM_API int gspm_mpnn_set_params(struct gspm_ctx* ctx, const float* params, int64_t count);
GSPM_API int gspm_mpnn_get_params(struct gspm_ctx* ctx, float* params, int64_t count);

/* Run the network on m, u_prev, u_prev2 ([n][3] float64 at `where`; the u's may be NULL = 0).
 * what = 0: raw output y [n][3]; what = 1: initial guess x0 = 2 u_prev - u_prev2 + u_s y. */
GSPM_API int gspm_mpnn_predict(struct gspm_ctx* ctx, const double* m, const double* u_prev,
                               const double* u_prev2, double* out, int what, int where);

/* Device-resident training set of this mesh: reserve `capacity` pairs, then add pairs
 * (m, u_prev, u_prev2) -> u* (u* = the displacement the plain solver found for m); the target
 * stored is t = (u* - (2 u_prev - u_prev2)) / u_s.  index (may be NULL) receives the slot. */
GSPM_API int gspm_mpnn_dataset_reserve(struct gspm_ctx* ctx, int capacity);
GSPM_API int gspm_mpnn_dataset_add(struct gspm_ctx* ctx, const double* m, const double* u_prev,
                                   const double* u_prev2, const double* u_star, int where,
                                   int* index);

/* Loss mean((y - t)^2) over nodes and components on stored pair `pair`, and its gradient with
 * respect to every parameter (host float32 [GSPM_MPNN_PARAMS], may be NULL). */
GSPM_API int gspm_mpnn_loss_grad(struct gspm_ctx* ctx, int pair, double* loss, float* grad);

/* `iterations` Adam steps (lr, beta = 0.9 / 0.999, eps 1e-8), each on one stored pair drawn by a
 * splitmix64 stream of `seed`; loss_first / loss_last (may be NULL) receive the losses of the first
 * and last step (before their update). */
GSPM_API int gspm_mpnn_train(struct gspm_ctx* ctx, int iterations, double lr, uint64_t seed,
                             double* loss_first, double* loss_last);

/* ---- measurement ------------------------------------------------------------------------ */

/* kernel classes for gspm_profile_* */
#define GSPM_KCLASS_SPMV_MECH 0  /* 3x3-block SpMV + fused p.q of the mechanical CG (K^mech)  */
#define GSPM_KCLASS_SPMV_GS 1    /* scalar multi-RHS SpMV + p.q of the GSPM CG solves         */
#define GSPM_KCLASS_SPMV_MS 2    /* scalar SpMV + p.q of the magnetostatic CG (K^ms)          */
#define GSPM_KCLASS_CG_VEC 3     /* CG vector updates (x, r with r.r; p)                       */
#define GSPM_KCLASS_CG_INIT 4    /* CG start-up (residual, norms)                              */
#define GSPM_KCLASS_RHS_MS 5     /* demagnetisation right-hand side b^ms = F^ms m (Eq. RHS_b)   */
#define GSPM_KCLASS_POINTWISE 6  /* E0, h(m), GSPM stages, projection, volume averages         */
#define GSPM_KCLASS_LEARNED 7    /* learned warm start inference (features, 4 layers, output)  */
#define GSPM_KCLASS_GRAD_MS 8    /* h~_d = -grad U through F^ms and the lumped mass (Sec. 2.3) */
#define GSPM_KCLASS_RHS_MECH 9   /* mechanical right-hand side F^mech E0 (Eq. RHS_b)           */
#define GSPM_KCLASS_STRAIN 10    /* strain E = E_bar + sym grad u (Sec. 2.3)                   */
#define GSPM_KCLASS_COUNT 11

/* Record CUDA events on the context's stream around every subsequent launch of the classes in
 * class_mask (bit k = class k); 0 stops recording.  Each call clears the accumulated times. */
GSPM_API int gspm_profile_enable(struct gspm_ctx* ctx, unsigned class_mask);

/* Total device time (ms) and launch count recorded for one class since the last enable;
 * synchronises the context's stream. */
GSPM_API int gspm_profile_read(struct gspm_ctx* ctx, int kclass, double* total_ms,
                               int64_t* launches);

#ifdef __cplusplus
}
#endif
#endif /* GSPM_H */
