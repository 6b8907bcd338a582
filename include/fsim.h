/*
 * fsim.h -- C ABI of the GB300 actuated-face PD + IPC solver.
 *
 * The library solves the quasi-static problem of "Efficient Incremental
 * Potential Contact for Actuated Face Simulation" (Li, Yang, Solenthaler,
 * SIGGRAPH Asia 2023 Technical Communications): minimise
 *     E-hat(x) = E(x) + B(x),
 * E the shape-targeting elastic energy of Eq. 1-2 and B the IPC barrier of
 * Eq. 3, by the loop of Algorithm 1.  Every iteration runs on the GPU:
 * the per-tet local step (Sec. 2.1), the constraint set, barrier gradient and
 * PSD Hessian (Sec. 2.2), the global step of Eq. 4 through the prefactored
 * PD matrix, the Schur complement of Eq. 8-9 and the low-rank update of
 * Eq. 10-11 (Sec. 3.1-3.2), the CCD step bound and the backtracking line
 * search.
 *
 * Conventions
 * -----------
 * - All pointers in this header are HOST pointers unless the name ends in
 *   "_dev" (device pointers, on the context's device).  The library copies
 *   every input it keeps; output buffers are owned by the caller.
 * - Positions are AoS float64 arrays "xyz" of length 3*n (x0,y0,z0,x1,...).
 * - Index arrays are int32 (vertex/triangle ids) or int64 (row pointers).
 * - Every entry point returns an fsim_status: 0 on success, a negative code
 *   on failure.  No entry point traps, asserts or throws; a failed call
 *   leaves the context usable unless it returns FSIM_ECUDA.
 * - Calls on one context are serialised on the context's CUDA stream and
 *   return when their result is on the host (solve_frame is synchronous).
 *   A context must not be used from two host threads at once.
 */
#ifndef FSIM_H
#define FSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fsim_ctx_s* fsim_ctx_t;
typedef int fsim_status;

enum {
  FSIM_OK = 0,
  FSIM_EINVAL = -1,            /* bad argument (null pointer, size, id)        */
  FSIM_ENOMEM = -2,            /* device allocation failed                      */
  FSIM_ECUDA = -3,             /* CUDA runtime error; context state undefined   */
  FSIM_ENOT_SPD = -4,          /* PD matrix or Schur complement not SPD         */
  FSIM_ENOT_CONVERGED = -5,    /* iteration cap hit; positions still readable   */
  FSIM_ELS_FAIL = -6,          /* line search made no acceptable step           */
  FSIM_ECONTACT_OVERFLOW = -7, /* more contact/CCD pairs than the capacity      */
  FSIM_ENONFINITE = -8,        /* NaN/Inf in inputs or iterates                 */
  FSIM_EINTERSECTING = -9,     /* proxy primitives touch (d <= 0) at the start  */
  FSIM_ENOT_READY = -10        /* mesh not prefactored / no actuation set       */
};

/* Arithmetic of solve_frame (Sec. 3 global step and the local step). */
enum {
  FSIM_FP64 = 0,   /* every per-iteration quantity in float64                  */
  FSIM_MIXED = 1   /* float32 SVD, triangular panels and reduced system; the
                      gradient, energies, distances and CCD stay float64       */
};

/* Solver constants (Sec. 2.1-2.2, Algorithm 1). */
typedef struct {
  double weight_scale;    /* w_i = weight_scale * rest volume of tet i (Eq. 2)  */
  double dhat;            /* barrier activation distance d0 (Sec. 2.2)          */
  double kappa;           /* barrier stiffness of Eq. 3; <= 0 selects the mean
                             diagonal entry of H over the free DOFs             */
  double tol_abs;         /* stop when ||g-hat_free||_2 <= max(tol_abs,         */
  double tol_rel;         /*   tol_rel * ||g-hat_free(x_t)||_2)  (Algorithm 1)  */
  int32_t max_iters;      /* iteration cap (FSIM_ENOT_CONVERGED beyond)         */
  int32_t max_ls;         /* line-search halvings before FSIM_ELS_FAIL          */
  double ccd_s;           /* additive-CCD gap ratio s (pairs keep >= s*d0)      */
  int32_t accd_max_iters; /* additive-CCD advancement cap per pair              */
  int32_t coop_ctas;      /* CTAs of the cooperative reduced-system kernel;
                             0 = one per SM (a tuning knob: fewer CTAs make
                             its grid-wide barriers cheaper)                   */
  int64_t contact_capacity; /* max near pairs (within 2 d0 in the float32
                               prefilter) and CCD candidates per pass; <= 0
                               selects max(2^20, 256 * proxy triangles)        */
  int64_t active_capacity;  /* max |C| (pairs with d < d0, each holding a
                               12-vector and a 12x12 block); <= 0 selects
                               max(2^16, 16 * proxy triangles), at most
                               contact_capacity.  More pairs than either
                               capacity return FSIM_ECONTACT_OVERFLOW         */
  double skin;              /* width of the contact candidate list: pairs within
                               d0 + skin are kept and the all-pairs sweep is
                               repeated only after proxy vertices moved about
                               skin / 2 (results are the same as sweeping
                               every time); <= 0 selects max(10 d0, a quarter
                               of the mean proxy edge length at rest)        */
  int32_t solver;           /* global step: FSIM_SOLVER_WOODBURY (Eq. 8-11, the
                               paper's method), FSIM_SOLVER_PCG (conjugate
                               gradients preconditioned with H, the paper's
                               comparison configuration; float64) or
                               FSIM_SOLVER_SCHUR (Sec. 3.1 alone: the dense
                               3 n2 x 3 n2 Sigma-hat of Eq. 9 assembled and
                               Cholesky-factored every iteration; float64, or
                               a float32 factor with two float64 refinement
                               steps in the mixed precision; needs
                               108 n2^2 bytes more workspace per slot)        */
  int32_t cg_max_iters;     /* CG iteration cap per global step                */
  double cg_tol;            /* CG stop: ||r|| <= cg_tol ||g-hat||              */
  int32_t adaptive_kappa;   /* nonzero: IPC's adaptive barrier stiffness, as the
                               paper uses it: within a frame kappa doubles
                               when the smallest active pair distance is below
                               0.1 d0 and smaller than at the previous iterate,
                               up to 100 times its start value; every frame
                               starts from the mesh's kappa                   */
  int32_t ee_mollifier;     /* nonzero: IPC's edge-edge mollifier -- each EE
                               term becomes kappa m(c) b(d) with c = |e_a x
                               e_b|^2, m(c) = (2 - c/eps) c/eps below
                               eps = 1e-3 |E_a|^2 |E_b|^2 (rest proxy edges),
                               1 above; 0 (default): plain b(d)              */
  int32_t reduced_one_cta_max; /* mixed precision: the largest n_c whose reduced
                               system one CTA solves; larger n_c up to 128 go
                               to a 4-CTA cluster, beyond that to the
                               cooperative kernel.  <= 0 selects 96 (the most
                               one CTA's shared memory holds); a tuning knob */
  int32_t sigma_product_simt; /* lock-step batches (fsim_solve_batch, server
                               batch mode): 0 (default) forms u = Sigma^-1 y2
                               for all frames on the tensor cores (tcgen05,
                               TF32 head/tail split, about 22 significant
                               bits); nonzero: float32 SIMT product          */
  int32_t barrier_lane_per_pair; /* single-frame solves: nonzero forms the pair
                               gradients and PSD Hessians with one lane per pair,
                               the form batches always use; 0 (default): one
                               warp per pair, faster for a single frame's few
                               hundred pairs                                  */
} fsim_params;
#define FSIM_SOLVER_WOODBURY 0
#define FSIM_SOLVER_PCG 1
#define FSIM_SOLVER_SCHUR 2

/* Per-frame statistics filled by fsim_solve_frame. */
typedef struct {
  int32_t status;         /* same code as the return value                       */
  int32_t iterations;     /* accepted Newton-like iterations of Algorithm 1      */
  int32_t ls_trials;      /* energy evaluations spent in line searches           */
  int32_t n_c;            /* contact-affected vertices at the last iteration     */
  int32_t n_c_max;        /* largest n_c over the frame                          */
  int32_t kappa_doublings; /* adaptive_kappa: times kappa doubled in the frame    */
  int64_t contacts;       /* |C| at the returned positions                       */
  double grad_norm;       /* ||g-hat_free||_2 at the returned positions           */
  double grad_norm0;      /* ||g-hat_free||_2 at x_t                              */
  double energy;          /* E-hat at the returned positions                      */
  double alpha_min;       /* smallest accepted step of the frame                  */
  double sum_nc3;         /* sum of n_c^3 over the frame's global steps (the
                             reduced system's work scales with it)            */
  int64_t cg_iterations;  /* CG iterations of the frame (FSIM_SOLVER_PCG)       */
  int32_t reduced_steps[4]; /* global steps of the frame by the path that solved
                               the reduced system (index = FSIM_REDUCED_*)    */
  int32_t fp64_steps;       /* FSIM_MIXED: global steps taken with the float64
                               factors because a float32 factor of the reduced
                               (or Schur) system lost positive definiteness:
                               the failed step is redone in float64 and every
                               later global step of the frame stays there   */
} fsim_frame_stats;

/* Path that solves the reduced contact system of Eq. 11 in one global step
 * (chosen from n_c and the precision): */
enum {
  FSIM_REDUCED_UNUSED = -1,     /* no reduced system (PCG or Schur-only solver)   */
  FSIM_REDUCED_COOPERATIVE = 0, /* grid-wide blocked Cholesky (float64 form, and
                                   the mixed form for n_c > 128)                   */
  FSIM_REDUCED_NONE = 1,        /* mixed form, n_c = 0: dx2 = Sigma^-1 y2          */
  FSIM_REDUCED_ONE_CTA = 2,     /* mixed form, 0 < n_c <= reduced_one_cta_max
                                   (96 by default): one CTA                       */
  FSIM_REDUCED_CLUSTER = 3      /* mixed form, above that up to 128: 4-CTA cluster */
};

/* Fill *p with the defaults: weight_scale 1e3, kappa auto, tol_abs 1e-8,
 * tol_rel 0, max_iters 500, max_ls 40, ccd_s 0.1, accd_max_iters 2000,
 * coop_ctas 0, contact_capacity, active_capacity and skin auto, solver
 * Woodbury, cg_max_iters 2000, cg_tol 1e-8, adaptive_kappa off.  dhat must
 * still be set by the caller. */
fsim_status fsim_default_params(fsim_params* p);

/* Create a context on CUDA device `device`; it owns one CUDA stream and all
 * device memory of the meshes uploaded to it. */
fsim_status fsim_create(fsim_ctx_t* out, int device);

/* Release the context and every device buffer it owns. */
fsim_status fsim_destroy(fsim_ctx_t ctx);

/* Number of kernel launches this context issued so far (instrumentation). */
fsim_status fsim_launch_count(fsim_ctx_t ctx, int64_t* count);

/*
 * Upload one simulation mesh and its collision proxy (Sec. 2.1, Sec. 3.1).
 *   rest_xyz   [3n]    rest positions (also the initial state)
 *   tets       [4T]    vertex ids per tetrahedron
 *   pinned     [n]     1 = Dirichlet vertex kept at its rest position
 *   proxy_tris [3Nt]   proxy triangles, ids into the Ns proxy vertices
 *   W_rowptr [Ns+1], W_col [nnz], W_val [nnz]:  CSR rows of the embedding
 *              s = W x (Sec. 3.1, Fig. 2a); at most 4 entries per row
 *   region     [n] or NULL: 1 marks the collision-aware set x2 (Sec. 3.1);
 *              NULL selects the free vertices in the support of W
 * Writes the new mesh id to *mesh_id.  Proxy edges are derived from the
 * triangles.  Errors: FSIM_EINVAL for ids out of range or empty sizes.
 */
fsim_status fsim_mesh_upload(fsim_ctx_t ctx, int* mesh_id,
                             const double* rest_xyz, int64_t n,
                             const int32_t* tets, int64_t T,
                             const uint8_t* pinned,
                             const int32_t* proxy_tris, int64_t Nt,
                             const int64_t* W_rowptr, const int32_t* W_col,
                             const double* W_val, int64_t Ns,
                             const uint8_t* region);

/*
 * One-time precomputation of the PD global step (Eq. 2 and Sec. 3.1-3.2):
 * w_i and shape gradients; the scalar PD matrix K (H = K (x) I_3 over the
 * free DOFs); a nested-dissection ordering of x1; the supernodal Cholesky
 * factor of K11 (H11 = L1 L1^T); the Schur complement Sigma of Eq. 9 and its
 * explicit inverse (Sec. 3.2).  Errors: FSIM_ENOT_SPD if K11 or Sigma is not
 * positive definite (a free component without a pinned vertex).
 */
fsim_status fsim_prefactor(fsim_ctx_t ctx, int mesh_id, const fsim_params* p);

/*
 * Per-tet actuation (Sec. 2.1): unit fibre f_i [3T] and stretch a_i [T]
 * give the symmetric A_i = a f f^T + a^(-1/2) (I - f f^T).  The factor is
 * untouched (H does not depend on actuation, Sec. 2.1).
 */
fsim_status fsim_set_actuation(fsim_ctx_t ctx, int mesh_id,
                               const double* fiber, const double* stretch);

/*
 * Solve one frame with Algorithm 1 from x_t = x_init [3n] (NULL: the
 * positions resident from the previous frame, or the rest state).  Pinned
 * vertices are reset to rest.  precision is FSIM_FP64 or FSIM_MIXED.  The
 * result stays resident (read it with fsim_read_positions).  stats may be
 * NULL.  Returns FSIM_ENOT_CONVERGED / FSIM_ELS_FAIL with the last iterate
 * resident, FSIM_EINTERSECTING if the proxy touches at x_init.
 */
fsim_status fsim_solve_frame(fsim_ctx_t ctx, int mesh_id, const double* x_init,
                             int precision, fsim_frame_stats* stats);

/* Same as fsim_solve_frame with x_init_dev a DEVICE pointer [3n] (or NULL). */
fsim_status fsim_solve_frame_dev(fsim_ctx_t ctx, int mesh_id,
                                 const double* x_init_dev, int precision,
                                 fsim_frame_stats* stats);

/* Copy the resident positions [3n] to host memory. */
fsim_status fsim_read_positions(fsim_ctx_t ctx, int mesh_id, double* xyz_out);

/* Device-to-device copy of the resident positions [3n]. */
fsim_status fsim_read_positions_dev(fsim_ctx_t ctx, int mesh_id, double* xyz_out_dev);

/*
 * The constraint set C at the resident positions (Sec. 2.2), sorted by
 * (type, i, j): keys [3*cap] receive triples (type, i, j) with type 0 =
 * point-triangle (proxy vertex i, proxy triangle j) and type 1 = edge-edge
 * (proxy edges i < j, edges numbered as the sorted unique (lo, hi) pairs of
 * the triangles).  *count receives |C|; FSIM_ECONTACT_OVERFLOW if |C| > cap.
 */
fsim_status fsim_read_contacts(fsim_ctx_t ctx, int mesh_id, int32_t* keys,
                               int64_t cap, int64_t* count);

/* ---- step-level entry points (one row of the iteration each) ----------- */
/* They evaluate one step at the given positions x [3n] (host) with the     */
/* mesh's current actuation and parameters, without changing the resident   */
/* state.  Precision follows `precision` where the step has two forms.      */

/* Local step (Eq. 1, Sec. 2.1): elastic energy E and its gradient
 * sum_i w_i G_i^T (G_i x - p_i) [3n] (zero rows for pinned vertices);
 * proj_out [9T] (may be NULL) receives p_i = vec(R_i A_i), row-major. */
fsim_status fsim_eval_elastic(fsim_ctx_t ctx, int mesh_id, const double* x,
                              int precision, double* energy_out,
                              double* grad_out, double* proj_out);

/* Proxy positions s = W x [3Ns] (Sec. 3.1). */
fsim_status fsim_eval_proxy(fsim_ctx_t ctx, int mesh_id, const double* x,
                            double* s_out);

/* UpdateConstraintSet (Algorithm 1): C at x as in fsim_read_contacts, and
 * the barrier energy kappa * sum b(d_k) (Eq. 3). */
fsim_status fsim_eval_contacts(fsim_ctx_t ctx, int mesh_id, const double* x,
                               int32_t* keys, int64_t cap, int64_t* count,
                               double* barrier_energy_out);

/* Barrier terms at x (Algorithm 1, Sec. 3.1): grad_out [3n] = W^T grad B(s)
 * over the free vertices; *n_c and c_out [n2] (may be NULL) the sorted x2
 * indices of the contact-affected vertices; bcheck_out [(3 n_c)^2] (may be
 * NULL, row-major) the reduced PSD block B-check of Eq. 10. */
fsim_status fsim_eval_barrier(fsim_ctx_t ctx, int mesh_id, const double* x,
                              double* grad_out, int32_t* n_c, int32_t* c_out,
                              double* bcheck_out, int64_t bcheck_cap);

/* Index checks of a bounds-checked build (compiled with -DFSIM_CHECK; the
 * build's check variant is libfsim_check.so).  *enabled is 1 in such a build,
 * else 0.  *word is 0 when no checked index has failed since the last call;
 * otherwise the first failure seen, site << 48 | index (site 1: force
 * gather tet slot, 2: supernodal-solve row, 3: contact-list entry).  A
 * failing index is skipped, not trapped.  Synchronises the device, then
 * resets the words. */
fsim_status fsim_check_status(fsim_ctx_t ctx, int32_t* enabled, uint64_t* word);

/* The explicit Sigma^-1 of Sec. 3.2 applied to ncols right-hand sides at
 * once, as the lock-step batches form u = Sigma^-1 y2 (Eq. 9) for all their
 * frames: y [n2 x ncols] and u_out [n2 x ncols] are row-major host arrays in
 * x2 order (the free x2 vertices in increasing mesh order), 1 <= ncols <=
 * 192.  y is rounded to float32 on the device.  tensor_cores nonzero: the
 * tcgen05 product with TF32 head/tail operands (FSIM_EINVAL where it is not
 * available); 0: the float32 SIMT product.  Needs a prefactored mesh only;
 * allocates and frees its own device buffers.  FSIM_ECUDA if a bounded wait
 * of the tensor-core kernel ran out. */
fsim_status fsim_eval_sigma_inv_mr(fsim_ctx_t ctx, int mesh_id, const double* y, int32_t ncols,
                                   int32_t tensor_cores, double* u_out);

/* Global step (Eq. 4 through Eq. 8-11): dx_out [3n] solves
 * (H + PositiveDefinite(B)) dx = -g-hat at x (zero on pinned vertices).
 * path_out (may be NULL) receives the FSIM_REDUCED_* path that solved the
 * reduced system. */
fsim_status fsim_eval_global_step(fsim_ctx_t ctx, int mesh_id, const double* x,
                                  int precision, double* dx_out, int32_t* path_out);

/* CCD step bound (Algorithm 1): alpha_m = min(1, min TOI) over the pairs
 * whose swept boxes of s -> s + W dx, inflated by dhat, overlap. */
fsim_status fsim_eval_ccd(fsim_ctx_t ctx, int mesh_id, const double* x,
                          const double* dx, double* alpha_out);

/* Line-search objective E-hat(x) = E(x) + B(x) (Sec. 2.2) and the gradient
 * norm ||g-hat_free||_2 at x (the convergence test of Algorithm 1). */
fsim_status fsim_eval_energy(fsim_ctx_t ctx, int mesh_id, const double* x,
                             int precision, double* energy_out,
                             double* grad_norm_out);

/* Same as fsim_set_actuation with DEVICE pointers fiber_dev [3T] and
 * stretch_dev [T] (no host copy; the inputs are not validated on the host). */
fsim_status fsim_set_actuation_dev(fsim_ctx_t ctx, int mesh_id,
                                   const double* fiber_dev, const double* stretch_dev);

/* The context's CUDA stream (a cudaStream_t) in *stream, so that callers
 * can order their own work or record timing events on it. */
fsim_status fsim_get_stream(fsim_ctx_t ctx, void** stream);

/* Kernel timing by CUDA events recorded around every launch of the kernel
 * classes whose bits are set in class_mask (0 disables): 0 local step,
 * 1 contact detection, 2 forward and 3 backward supernodal solves, 4 dense
 * Cholesky, 5 barrier pairs, 6 CCD, 7 Sigma^-1 product, 8 whole reduced
 * system.  fsim_profile_read synchronises and returns the launch count and
 * summed milliseconds of one class since the last fsim_profile_reset. */
fsim_status fsim_profile(fsim_ctx_t ctx, uint32_t class_mask);
fsim_status fsim_profile_read(fsim_ctx_t ctx, int kernel_class, int64_t* launches,
                              double* total_ms);
fsim_status fsim_profile_reset(fsim_ctx_t ctx);

/*
 * CCD step bound that allocates no device memory.  The paper has no
 * counterpart to this entry point; it exists for callers that cannot let a
 * library allocate GPU memory on its own: engines that reserve all device
 * memory up front in their own pool, or applications held to a fixed memory
 * budget.
 *
 * Computes alpha_m = min(1, min over candidate pairs of the additive-CCD time
 * of impact) exactly as the solver's CCD stage (fsim_eval_ccd) does, for
 * proxy positions s_dev [3 Ns] and step ds_dev [3 Ns], triangles
 * tris_dev [3 Nt] and edges edges_dev [2 Ne] (the sorted unique (lo, hi)
 * pairs of the triangles' edges), all DEVICE pointers owned by the caller;
 * the result is written to the device double *alpha_dev.  Work is queued on
 * `stream` (a cudaStream_t, NULL = default stream); the call then reads its
 * status words back and synchronises that stream, so it returns after the
 * stream has finished the work.  The candidate search tests every
 * point-triangle and edge-edge pair (O(Ns Nt + Ne^2) box tests: meant for the
 * few thousand primitives of a contact region); Nt and Ne are limited to
 * 65535 * 128.  Every entry of tris_dev and edges_dev must lie in [0, Ns):
 * primitives that break this are skipped and the call returns FSIM_EINVAL.
 *
 * Scratch: a fixed static device array of 2^20 candidate pairs (about 8 MiB),
 * present on every GPU that loads the library until the process exits.  More
 * candidates than that return FSIM_ECONTACT_OVERFLOW (alpha_dev then holds a
 * bound over the first 2^20 candidates only and must not be used).  The first
 * call on a device looks up the array's device address; make that first call
 * before any stream capture.  All calls share the array, so calls that
 * overlap on the GPU (other streams, other host threads) race: serialise them.
 * Errors: FSIM_EINVAL for null pointers, negative or too large sizes,
 * dhat <= 0, ccd_s outside (0, 1), accd_max_iters <= 0 or a primitive index
 * outside [0, Ns); FSIM_ECUDA for a CUDA error.
 */
fsim_status fsim_ccd_noalloc(const double* s_dev, const double* ds_dev, int64_t Ns,
                             const int32_t* tris_dev, int64_t Nt,
                             const int32_t* edges_dev, int64_t Ne, double dhat,
                             double ccd_s, int32_t accd_max_iters, double* alpha_dev,
                             void* stream);

/*
 * Automatic collision region.  The paper takes the collision-aware region x2
 * and its proxy surface from the user (Sec. 3.1, Fig. 2a) and names their
 * automatic selection as future work (Sec. 5); this selects them from the
 * rest geometry: a boundary vertex can take part in contact when another
 * boundary vertex lies closer than `radius` at rest (float64 squared
 * distance, strict) but more than `rings` surface edges away (two sides of
 * a slit, two bodies across a gap).  The proxy is every boundary triangle
 * (a tet face met once) whose three vertices can take part in contact and
 * are not all pinned (pinned may be NULL); W is the selection of its
 * vertices, so the result feeds fsim_mesh_upload as proxy_tris (local
 * numbering) with W_rowptr = 0..Nv, W_col = proxy_verts, W_val = 1.
 *   rest_xyz [3n], tets [4T] (ids in [0, n)), pinned [n] or NULL
 *   proxy_tris [3 tris_cap] <- sorted triangles in proxy-vertex numbering
 *   proxy_verts [verts_cap] <- proxy vertex ids (mesh numbering, increasing)
 * *n_tris and *n_verts receive the counts; with both caps 0 only the counts
 * are returned (call again with buffers that large).  Host only (no GPU).
 * Errors: FSIM_EINVAL for bad sizes or ids, radius <= 0, rings < 0, or caps
 * smaller than the counts.
 */
fsim_status fsim_select_region(const double* rest_xyz, int64_t n, const int32_t* tets, int64_t T,
                               const uint8_t* pinned, double radius, int32_t rings,
                               int32_t* proxy_tris, int64_t tris_cap, int64_t* n_tris,
                               int32_t* proxy_verts, int64_t verts_cap, int64_t* n_verts);

/* Sizes of a mesh (n, T, Ns, Nt, Ne, free / x1 / x2 vertex counts), the
 * scalar factor's stored entries and supernode / level counts, the bytes of
 * one per-solve workspace (what each request-server slot of this mesh
 * allocates, before its reduced-system buffers grow), and the barrier
 * stiffness kappa in use (after fsim_prefactor). */
typedef struct {
  int64_t n, T, Ns, Nt, Ne, n_free, n1, n2, factor_nnz, n_supernodes, n_levels;
  int64_t workspace_bytes;
  double kappa;
} fsim_mesh_info;
fsim_status fsim_mesh_info_get(fsim_ctx_t ctx, int mesh_id, fsim_mesh_info* info);

/* ---- request server: continuous batching of frame solves -----------------
 * The paper solves one frame at a time; this server is the serving layer on
 * top of Algorithm 1.  Several frame solves run at once, each on its own
 * host thread, CUDA stream and workspace slot (a private copy of the
 * per-solve buffers of its mesh; the factor of K11, Sigma^-1 and the mesh
 * topology stay shared and resident).  A request that arrives while others
 * are on the GPU starts as soon as a worker is idle and a slot fits in the
 * memory budget; idle slots of other meshes are evicted least recently used
 * first.  Every request carries its own actuation and start positions, so
 * its result is the same whether it runs alone or among others (up to the
 * order of floating-point atomics, as for any two runs).
 */
typedef struct fsim_server_s* fsim_server_t;

typedef struct {
  int32_t mesh_id;        /* a prefactored mesh of the server's context        */
  int32_t precision;      /* FSIM_FP64 or FSIM_MIXED                            */
  const double* fiber;    /* 3T: per-tet fiber direction                        */
  const double* stretch;  /* T: per-tet stretch a > 0                           */
  const double* x_init;   /* 3n start positions, or NULL for the rest pose      */
  int32_t flags;          /* 0: fiber, stretch and x_init are host arrays,
                             copied (and checked) at submit.
                             FSIM_REQ_DEVICE: they are device arrays, read when
                             the request runs; they must stay valid and
                             unchanged until it completes and are not checked
                             on the host (a non-positive stretch surfaces as
                             FSIM_ENONFINITE)                                 */
  int32_t reserved0;
  double* x_out_dev;      /* device, 3n, or NULL: receives the converged
                             positions before the request completes; with
                             FSIM_REQ_DEVICE the positions are returned only
                             here (fsim_server_wait's x_out is then unused)   */
} fsim_request;
#define FSIM_REQ_DEVICE 1

typedef struct {
  int32_t workers;          /* concurrent solves (batch_frames < 2) or
                               concurrent batches (batch_frames >= 2), 1..16   */
  int32_t batch_frames;     /* 0 or 1: every request is its own solve on its own
                               worker.  2..64: each worker runs a lock-step
                               batch of up to this many frames of one mesh (as
                               fsim_solve_batch), and at every iteration
                               boundary takes the oldest queued requests of its
                               mesh into the slots of finished frames; such a
                               server accepts FSIM_MIXED requests of meshes
                               using FSIM_SOLVER_WOODBURY (FSIM_EINVAL at
                               submit otherwise)                              */
  int64_t mem_budget_bytes; /* cap on the bytes of all workspace slots (and
                               batches); <= 0 means no cap                     */
} fsim_server_config;

typedef struct {
  int32_t workers, slots, peak_slots, peak_running;
  int64_t queued, completed, bytes_in_use;
} fsim_server_info;

/* Start the worker threads.  The context must outlive the server; meshes
 * must be uploaded and prefactored before their requests are submitted.
 * Errors: FSIM_EINVAL (workers outside 1..16), FSIM_ENOMEM. */
fsim_status fsim_server_create(fsim_ctx_t ctx, const fsim_server_config* cfg, fsim_server_t* out);
/* Queue one frame solve; host inputs are copied before return.  *ticket
 * names it for fsim_server_wait.  Errors: FSIM_EINVAL, FSIM_ENOT_READY (mesh
 * not prefactored), FSIM_ENONFINITE (stretch <= 0 or a zero / non-finite
 * fiber), FSIM_ENOMEM (one workspace of this mesh, see fsim_mesh_info's
 * workspace_bytes, is larger than the memory budget). */
fsim_status fsim_server_submit(fsim_server_t srv, const fsim_request* req, int64_t* ticket);
/* *done = 1 once the request has finished (0 while queued or running). */
fsim_status fsim_server_poll(fsim_server_t srv, int64_t ticket, int32_t* done);
/* Block until the request finishes; copy its positions (3n, may be NULL) and
 * statistics, its latency from submit to completion and its queueing time
 * (submit to start), in milliseconds.  Each ticket is waited for once.
 * Returns the solve's status (as fsim_solve_frame would; FSIM_ENOMEM when
 * its slot's reduced-system buffers had to grow, because n_c rose, beyond
 * the memory budget).  Must not race with fsim_server_destroy. */
fsim_status fsim_server_wait(fsim_server_t srv, int64_t ticket, double* x_out,
                             fsim_frame_stats* stats, double* latency_ms, double* queue_ms);
fsim_status fsim_server_info_get(fsim_server_t srv, fsim_server_info* info);
/* Finish the running solves, drop queued ones and free every slot. */
fsim_status fsim_server_destroy(fsim_server_t srv);

/* Batched form: solve n_req independent frames on a temporary server with
 * `workers` concurrent solves; x_out[i] (3n of request i's mesh) and
 * stats[i] receive the results (either may be NULL).  Returns the first
 * non-OK status (each stats[i].status has its own). */
fsim_status fsim_solve_frames(fsim_ctx_t ctx, int32_t n_req, const fsim_request* reqs,
                              int32_t workers, double* const* x_out, fsim_frame_stats* stats);

/*
 * Lock-step batched form: solve n_req frames of ONE mesh (all requests must
 * name the same prefactored mesh, FSIM_MIXED precision, and the mesh must use
 * FSIM_SOLVER_WOODBURY) with up to max_frames (1..64) of them advancing
 * together through Algorithm 1.  Every stage of an iteration is one launch
 * for all frames in the batch: the local step, constraint set, barrier
 * derivatives, CCD and line-search trials over a table of per-frame
 * workspaces; the triangular solves of Eq. 8 as one pass over the factor for
 * the right-hand sides of all frames; the reduced systems of Eq. 11 side by
 * side.  A frame that converges leaves the batch after its iteration and the
 * next request takes its place.  Each frame's result is that of the same
 * request solved alone (fsim_solve_frame) up to the order of floating-point
 * atomics.  Requests are fsim_request as for the server (host or
 * FSIM_REQ_DEVICE inputs; x_out_dev, when set, receives the positions);
 * x_out[i] (host, 3n, may be NULL) and stats[i] (may be NULL) receive the
 * results.  Runs on the context's stream; returns after all requests have
 * finished, with the first non-OK status (each stats[i].status has its own).
 * Errors: FSIM_EINVAL (mixed meshes or precisions, another solver,
 * max_frames outside 1..64, or a mesh whose largest supernode does not fit
 * the batched solves), FSIM_ENOT_READY, FSIM_ENOMEM.
 */
fsim_status fsim_solve_batch(fsim_ctx_t ctx, int32_t n_req, const fsim_request* reqs,
                             int32_t max_frames, double* const* x_out, fsim_frame_stats* stats);

#ifdef __cplusplus
}
#endif
#endif /* FSIM_H */
