/*
 * emu.h: C ABI of the GB300 quasi-static muscle solver (EMU, arXiv 2006.08821).
 *
 * The library solves the quasi-static problem of Sec. 3 (Eq. 1) in EMU's
 * variable-separated form (Eq. 5). Each tet carries its own deformation
 * gradient F_i. On the device it is stored as a rotation R_i and a
 * symmetric stretch S_i (six coordinates s_i), F_i = R_i S_i. Positions q
 * are the "nearest continuous mesh" of Eq. 4. Each Newton iteration:
 *
 *   - evaluates the exact gradient of Eqs. 6-7 per tet;
 *   - builds the elastic Hessian in rotation/stretch coordinates (rotation
 *     block zero because Psi is rotation invariant; 6x6 stretch block with a
 *     definiteness fix, Sec. 3.2.1);
 *   - forms the low-rank Woodbury direction of Eqs. 9-12 (k = 48);
 *   - solves the constant ACAP system of Eq. 4 on the device in FP64;
 *   - runs the backtracking Armijo line search of Algorithm 1;
 *   - re-extracts R_i, S_i from F_i + sigma d_i by a polar decomposition.
 *
 * Conventions, shared by every entry point:
 *   - Return value 0 (EMU_OK) on success, a negative emu_status otherwise.
 *     No C++ exception crosses this boundary. emu_last_error() returns a
 *     thread-local message for the last failure.
 *   - Host input buffers are read during the call and copied; the caller
 *     keeps ownership. Output buffers are caller-owned.
 *   - Device state is owned by the handle. It is allocated through the
 *     optional allocator callback at create time, or with cudaMalloc when
 *     the allocator is NULL, and released by emu_destroy.
 *   - All device work is enqueued on the stream given at create time
 *     (NULL = the legacy default stream). Calls that return host-visible
 *     results synchronise that stream only.
 *   - A handle is not thread-safe. Distinct handles may be used from
 *     distinct threads.
 *   - Units: SI (metres, pascals). Positions are row-major (n, 3) float64.
 */
#ifndef EMU_H_
#define EMU_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------------- */
typedef enum {
  EMU_OK = 0,
  EMU_ERR_INVALID_ARG = -1,     /* bad pointer, size, index or parameter      */
  EMU_ERR_DEGENERATE_TET = -2,  /* |det D_m| below 1e-14 h^3 (Eq. 2)          */
  EMU_ERR_OOM = -3,             /* allocator or device memory failure          */
  EMU_ERR_NOT_CONVERGED = -4,   /* max_newton reached; state kept and usable   */
  EMU_ERR_LINESEARCH = -5,      /* no Armijo step within ls_max_trials         */
  EMU_ERR_PCG = -6,             /* ACAP solve did not reach pcg_tol            */
  EMU_ERR_INVERTED = -7,        /* non-finite gradient / inverted element      */
  EMU_ERR_TIMEOUT = -8,         /* a bounded device wait ran out               */
  EMU_ERR_CUDA = -9,            /* CUDA runtime error                          */
  EMU_ERR_NOT_IMPLEMENTED = -10
} emu_status;

typedef enum { EMU_PRECISION_FP64 = 0, EMU_PRECISION_MIXED = 1 } emu_precision;
/* Variables of the Newton iteration (emu_params.form): the rotation-stretch
 * chart F_i = R_i S(s_i) with its 6 x 6 stretch Hessian, or the paper's own
 * F-form (Sec. 3.2.1, Eqs. 10-12) with one free F_i and a 9 x 9 block per
 * tet. Both reach the same equilibrium. */
typedef enum { EMU_FORM_RS = 0, EMU_FORM_F = 1 } emu_form;

/* Opaque solver handle (library-owned). */
typedef struct emu_handle emu_handle;

/* Device allocator callback. alloc returns a device pointer aligned to at
 * least 256 bytes, or NULL on failure; free releases it. ``stream`` is the
 * handle's cudaStream_t. The PyTorch binding routes these to torch's caching
 * allocator. */
typedef struct {
  void* ctx;
  void* (*alloc)(void* ctx, size_t bytes, void* stream);
  void (*free)(void* ctx, void* ptr, size_t bytes, void* stream);
} emu_allocator;

/* Mesh, materials, fibers and pins (Eq. 1; Sec. 3.1, 3.6).
 *   rest_pos     n_verts x 3 rest positions Q (m). Copied.
 *   tets         n_tets x 4 vertex indices; corner 3 is the reference corner
 *                of Eq. 2. Negatively oriented tets are re-oriented by
 *                swapping corners 1 and 2. Copied.
 *   youngs, poisson   n_materials entries (Pa, dimensionless).
 *   material_id  n_tets entries in [0, n_materials).
 *   fiber_dir    n_tets x 3 fiber directions u_i; normalised on copy. NULL =
 *                no fiber term.
 *   fixed_verts  n_fixed vertex indices pinned (Sec. 3.1 removes the rigid
 *                null space by pinning). Must be non-empty.
 *   fixed_pos    n_fixed x 3 prescribed positions of the pinned vertices;
 *                NULL pins them at their rest positions. */
typedef struct {
  int64_t n_verts;
  int64_t n_tets;
  const double* rest_pos;
  const int32_t* tets;
  int32_t n_materials;
  const double* youngs;
  const double* poisson;
  const uint8_t* material_id;
  const double* fiber_dir;
  int64_t n_fixed;
  const int32_t* fixed_verts;
  const double* fixed_pos;
  /* Bones and joints (Sec. 3.3). bone_id (n_tets; -1 = deformable, b >= 0
   * = bone b, ids contiguous from 0) may be NULL. Every tet of a bone shares
   * the bone's single deformation gradient F_b; all of a bone's tets have one
   * material and no vertex belongs to two bones. A bone's vertices are either
   * all pinned (the bone stays put, F_b = I) or none (a free bone, at most 4;
   * k_modes must be 48). Activations must be 0 on bone tets.
   * n_joints joints, each with a type (0 ball, 1 hinge), two bone ids (at
   * least one free), a point (metres) and, for a hinge, an axis (normalised
   * on copy) and the half-length of its two axis points (at most 16 joint
   * points). At each joint point the least-squares affine fits of the two
   * bones' vertex positions coincide: hard during Newton, a penalty in the
   * final solve (see eps_bone, eps_joint in emu_params). After a solve the
   * positions are those of the final coupling solve: each free bone's
   * vertices are exactly F_b Q_v + t_b. All may be NULL / 0. */
  const int32_t* bone_id;
  int32_t n_joints;
  const int32_t* joint_type;        /* n_joints */
  const int32_t* joint_bones;       /* n_joints x 2 */
  const double* joint_point;        /* n_joints x 3 */
  const double* joint_axis;         /* n_joints x 3 */
  const double* joint_half_length;  /* n_joints */
} emu_mesh_desc;

/* Solver parameters. emu_default_params fills the defaults shown.
 *   alpha_rel       ACAP weight alpha of Eq. 5 as a multiple of mu_ref, the
 *                   smallest shear modulus in the mesh (default 1).
 *   weight_mode     0: w_i = V_i (Eq. 3 up to the volume measure, default);
 *                   1: w_i = V_i max(1, mu_i/mu_ref) (the stiffness-weighted
 *                   variant of Sec. 3.3).
 *   k_modes         low-rank size of Eq. 9; a multiple of 3 in [3, 48]
 *                   (default 48 = 16 scalar modes x 3 coordinates).
 *   fiber_scale     kappa = fiber_scale * mu_ref multiplies a_i u^T C u.
 *   tol_rel_residual stop when ||dE/dF||_2 / ||dE/dF at F=I||_2 <= tol.
 *   max_newton      Newton iteration cap per solve.
 *   ls_sigma0, ls_c, ls_rho, ls_max_trials   Armijo backtracking
 *                   (Algorithm 1 uses 10, 1e-4, 0.5; defaults 4, 1e-4,
 *                   0.5, 40). Each pass evaluates 4 trial steps
 *                   sigma * rho^j together and takes, among those meeting
 *                   the Armijo condition, the one with the largest energy
 *                   decrease.
 *   pcg_tol         relative residual of the exact coupling solve q = q*(F)
 *                   (Eq. 4); the solve used is min(pcg_tol, 1e-2 * tol),
 *                   floored at 1e-13.
 *   pcg_max         CG iteration cap per ACAP solve.
 *   precision       EMU_PRECISION_FP64 or EMU_PRECISION_MIXED (per-tet
 *                   Hessian/Woodbury work in FP32; state, gradient,
 *                   residual, line-search sums and ACAP solve in FP64).
 *                   MIXED is for tol_rel_residual >= 1e-6 or so: its FP32
 *                   rounding floor can lie above a tighter tolerance, and a
 *                   solve then runs to max_newton; use FP64 there.
 *   mode_iters      subspace iterations used to build the low-rank basis
 *                   (default 8).
 *   seed            seeds the random start of the subspace iteration.
 *   dq_tol          relative residual of the per-iteration solve for the
 *                   change of q along the search direction (q*(F + s d) =
 *                   q + s dq, q* being affine); q itself is then updated by
 *                   linearity (default 8e-2). After a line search fails,
 *                   q is re-solved and dq is solved to the exact-solve
 *                   tolerance for the rest of the call.
 *   q_refresh       every q_refresh iterations, and before convergence is
 *                   declared, q is re-solved exactly from the current F
 *                   (default 32).
 *   eps_bone        slack of the bone rows during Newton (Sec. 3.3, < 0;
 *                   default -1e-3): each bone tet's ACAP weight grows by
 *                   Vbar / |eps_bone| (Vbar the mean rest volume).
 *   eps_joint       slack of the joint rows in the final coupling solve
 *                   (Sec. 3.3, < 0; default -1e-4): the joints become the
 *                   penalty Vbar^(1/3) / |eps_joint| |J q|^2 while every
 *                   bone's vertices follow its affine map exactly.
 *   cg_local_degree degree (1..8) of the block-local Chebyshev polynomial in
 *                   the preconditioner of the mixed path's loose coupling
 *                   solves (the dq solves): each CUDA block applies it to its
 *                   own spatially compact part of the ACAP Laplacian of
 *                   Eq. 4, next to the coarse space on the low-rank basis
 *                   (a two-level additive Schwarz preconditioner). 1 is plain
 *                   Jacobi; higher degrees cost more per CG iteration and
 *                   take fewer iterations (default 4).
 *   form            EMU_FORM_RS (default) or EMU_FORM_F. The F-form keeps one
 *                   deformation gradient F_i per tet, builds the 9 x 9 block
 *                   H_i = PSD(V Psi_iso''(F_i)) + V Psi_fiber''(F_i)
 *                   + alpha w_i I (the definiteness fix on the isotropic
 *                   term, through its analytic eigen-system) and updates
 *                   F <- F + sigma d directly (no polar re-extraction). It
 *                   runs in FP64 (precision must be EMU_PRECISION_FP64) on
 *                   meshes without bones or joints; otherwise emu_create
 *                   returns EMU_ERR_NOT_IMPLEMENTED. emu_get_element_state
 *                   then returns F and its polar factors R, s;
 *                   emu_set_element_state sets F = R S.
 *   autotune        0 (default) or 1: emu_create times candidate settings of
 *                   the coupling solves on the mesh's own matrix and keeps
 *                   the fastest: the local polynomial's degree (2, 3, 4, 6,
 *                   8; overrides cg_local_degree) for the mixed path's dq
 *                   solves, and the rows per block (64, 128, 256) of the
 *                   FP64 CG. Each choice is kept for the process per device
 *                   and mesh size, so handles of one mesh run the same
 *                   settings; another process may choose differently, and
 *                   its results then differ in rounding. emu_get_tuning
 *                   reports the settings in use. */
typedef struct {
  double alpha_rel;
  int32_t weight_mode;
  int32_t k_modes;
  double fiber_scale;
  double tol_rel_residual;
  int32_t max_newton;
  double ls_sigma0;
  double ls_c;
  double ls_rho;
  int32_t ls_max_trials;
  double pcg_tol;
  int32_t pcg_max;
  int32_t precision;
  int32_t mode_iters;
  uint64_t seed;
  double dq_tol;
  int32_t q_refresh;
  double eps_bone;
  double eps_joint;
  int32_t cg_local_degree;
  int32_t form;
  int32_t autotune;
} emu_params;

/* Per-solve statistics. */
typedef struct {
  int32_t newton_iters;     /* Newton iterations taken                         */
  int32_t ls_trials;        /* line-search energy evaluations                  */
  int32_t pcg_iters;        /* CG iterations summed over all ACAP solves       */
  int32_t status;           /* emu_status of the solve                         */
  double rel_residual;      /* final ||g|| / ||g(I)||                          */
  double energy_change;     /* E(final) - E(start), summed line-search deltas  */
  double ms;                /* wall time of the solve (host clock)             */
} emu_solve_stats;

void emu_default_params(emu_params* p);
const char* emu_status_string(int status);
const char* emu_last_error(void);

/* Builds the solver for one mesh (Sec. 3.1 setup): D_m^-1 and V_i (Eq. 2),
 * ACAP weights, the scalar ACAP Laplacian (G^T W G = L x I_3 with full-vertex
 * pins, Eq. 4), its Jacobi preconditioner and the low-rank basis of Eq. 9.
 * The state starts at rest (R = I, S = I, q = q*(I)). ``stream`` is a
 * cudaStream_t (NULL = default stream). Returns EMU_ERR_DEGENERATE_TET,
 * EMU_ERR_INVALID_ARG or EMU_ERR_OOM on the corresponding failure. */
int emu_create(const emu_mesh_desc* mesh, const emu_params* params, const emu_allocator* alloc,
               void* stream, emu_handle** out);

/* Releases all device memory of the handle. NULL is accepted. */
int emu_destroy(emu_handle* h);

/* Sets a_i(t) of Sec. 3.1 (Psi_fiber = kappa a_i u_i^T F_i^T F_i u_i).
 * ``a`` is a host array of n_tets entries, each finite and >= 0. */
int emu_set_activation(emu_handle* h, const double* a, int64_t count);

/* Same as emu_set_activation with ``a`` a device pointer (n_tets float64). */
int emu_set_activation_device(emu_handle* h, const double* a_device, int64_t count);

/* Constant external forces (Sec. 3.4, Eq. external-forces), such as gravity:
 * f is a host array of n_verts x 3 newtons (per vertex, row-major), or NULL
 * to remove them. The force does the work q*(F)^T f through the coupling
 * solve of Eq. 4, so on the deformation gradients it acts as the generalized
 * force nu = W G K^-1 f (forces on pinned vertices are taken by the pins),
 * computed here once on the device (an FP64 CG solve to 1e-13 and a per-tet
 * kernel): every solve then minimises E(F) - <F, nu>. The handle keeps nu
 * (9 n_tets doubles, plus as many floats on the mixed path, allocated on
 * the first call, not counted by emu_required_bytes) until the next call.
 * EMU_ERR_NOT_IMPLEMENTED on meshes with bones; EMU_ERR_INVALID_ARG for a
 * count other than n_verts or a non-finite value; EMU_ERR_PCG if the solve
 * does not converge. Synchronous. */
int emu_set_external_forces(emu_handle* h, const double* f, int64_t n_verts);

/* Runs Newton iterations from the resident state (warm start) until the
 * relative residual reaches tol_rel_residual (Algorithm 1, Newton part).
 * ``stats`` may be NULL. Returns EMU_ERR_NOT_CONVERGED when max_newton is
 * reached, or when the residual has stalled within 10x of the tolerance
 * for 200 iterations; the state is then kept and stats->rel_residual tells
 * how close it got. Before that, a solve stalled there for 50 iterations
 * tries three remedies in turn: the first trial step drops from ls_sigma0
 * to 1 (longer steps can make the gradient zig-zag), a mixed solve
 * finishes on the FP64 kernels (the rounding floor of FP32 per-tet
 * arithmetic can sit above the tolerance for activations near 0), then dq
 * is solved to 1e-2 * dq_tol (q drifts from q*(F) between exact re-solves
 * when dq is loose). The first and last hold for every later solve on the
 * handle until emu_reset. */
int emu_solve_quasistatic(emu_handle* h, emu_solve_stats* stats);

/* Solves ``count`` independent meshes (the c3 batch: Algorithm 1 per mesh,
 * each from its own resident state and activation). Every handle's work is
 * enqueued on its own stream; the host interleaves the handles' Newton
 * loops (each waits for its device results without blocking the others),
 * so meshes given distinct streams overlap on the device. The result of
 * each mesh is the one emu_solve_quasistatic would give it.
 *   hs      ``count`` distinct handles (host array, caller-owned).
 *   stats   NULL or ``count`` entries, filled per handle (status included).
 * Returns EMU_OK when every solve succeeded, else the first failing status
 * in handle order (the others still ran to completion). Not thread-safe
 * with other calls on the same handles. */
int emu_batch_solve(emu_handle* const* hs, int32_t count, emu_solve_stats* stats);

/* Upper bound of the device memory (bytes) that emu_create allocates for
 * this mesh and these parameters (the Laplacian is bounded by 16 entries per
 * tet). Validates like emu_create; needs a current CUDA device. Used by the
 * server's admission control. A mixed-precision solve that escalates to the
 * FP64 kernels (see emu_solve_quasistatic) allocates 960 more bytes per tet
 * on first use. */
int emu_required_bytes(const emu_mesh_desc* desc, const emu_params* params, size_t* bytes);

/* ---------------------------------------------------------------- serving
 * A persistent request loop on the current device (the c4 stream): each
 * request is one mesh and n_frames activation vectors, solved frame by frame
 * from its own resident state (warm starts). A worker thread admits queued
 * requests in arrival order while their device memory (emu_required_bytes)
 * fits in the budget and fewer than 32 are in flight, and interleaves the
 * active requests' Newton loops, each on its own stream, so that their work
 * overlaps on the device (continuous batching: a request that arrives while
 * others run is admitted as soon as memory and a slot free up). Four
 * set-up threads build admitted requests' handles (emu_create, including the
 * low-rank basis) and destroy finished ones, so requests in flight keep
 * advancing while others are set up or released. Without an allocator the
 * handles' memory is stream-ordered (cudaMallocAsync / cudaFreeAsync on the
 * request's stream). A request's memory returns to the budget once its
 * handle is released after its last frame; its result is published before
 * that. The result of a request does not depend on what else is in flight
 * (every kernel is deterministic and touches only its own handle's memory).
 * Submit, poll and result may be called from any thread. */
typedef struct emu_server emu_server;

typedef struct {
  uint64_t id;
  int32_t status;         /* EMU_OK, or the status of the frame that failed */
  int32_t frames_done;    /* frames solved (all of them when status is OK)  */
  int32_t newton_iters;   /* summed over frames                            */
  int32_t pcg_iters;      /* summed over frames                            */
  double rel_residual;    /* of the last frame solved                      */
  double queue_ms;        /* submit -> admitted                            */
  double setup_ms;        /* emu_create of the request                     */
  double solve_ms;        /* frames, after setup                           */
  double latency_ms;      /* submit -> last frame done (host clock)        */
  uint64_t device_bytes;  /* memory reserved against the budget            */
} emu_request_stats;

/* Starts the worker thread. budget_bytes: device memory the active
 * requests may hold in total. params: NULL for defaults (copied). alloc:
 * NULL for cudaMalloc (the worker thread calls it). */
int emu_server_create(size_t budget_bytes, const emu_params* params, const emu_allocator* alloc,
                      emu_server** out);

/* Queues a request. The mesh arrays and activations (n_frames x n_tets,
 * row-major, each finite and >= 0) are copied; request_id must not be in
 * use. EMU_ERR_OOM if the mesh alone exceeds the budget. */
int emu_server_submit(emu_server* srv, const emu_mesh_desc* mesh, const double* activations, int32_t n_frames,
                      uint64_t request_id);

/* Writes up to cap ids of finished requests not reported before. */
int emu_server_poll(emu_server* srv, uint64_t* done_ids, int32_t cap, int32_t* n_done);

/* Copies a finished request's positions (n_frames x n_verts x 3 float64,
 * the converged q of every frame; NULL to skip) and stats (NULL to skip),
 * then forgets the request. EMU_ERR_INVALID_ARG if the id is unknown or
 * not finished. */
int emu_server_result(emu_server* srv, uint64_t request_id, double* positions, emu_request_stats* stats);

/* Stops the threads: device work already enqueued is waited for, requests
 * not finished are dropped, and everything is freed. */
int emu_server_destroy(emu_server* srv);

/* Copies q (n_verts x 3 float64, row-major) to ``out``: a host pointer when
 * out_is_device == 0, a device pointer otherwise. */
int emu_get_positions(emu_handle* h, double* out, int32_t out_is_device);

/* Copies the per-tet state to host arrays (any may be NULL):
 * R n_tets x 9 row-major, s n_tets x 6 in the order (xx, yy, zz, yz, xz, xy)
 * with off-diagonals scaled by sqrt(2) so that |s| = ||S||_F, and
 * F = R S, n_tets x 9 row-major. */
int emu_get_element_state(emu_handle* h, double* R, double* s, double* F);

/* Overwrites the per-tet stretch/rotation state and positions from host
 * arrays (R n_tets x 9, s n_tets x 6, q n_verts x 3). R must be a rotation
 * and S(s) positive definite. Used for warm starts and resume. */
int emu_set_element_state(emu_handle* h, const double* R, const double* s, const double* q);

/* Resets the state to rest (R = I, S = I, q = q*(I)). */
int emu_reset(emu_handle* h);

/* Sizes of the mesh held by the handle. */
int emu_get_sizes(emu_handle* h, int64_t* n_verts, int64_t* n_tets, int32_t* k_modes);

/* Evaluates, on the device, the per-element stretch terms that the solver
 * uses (Sec. 3.1 energy with F = S, Sec. 3.2.1 Hessian):
 *   psi[i]  = V_i Psi(S_i),
 *   grad[i] = V_i dPsi/ds (6),
 *   hess[i] = V_i d2Psi/ds2 (6x6 row-major) with the definiteness fix
 *             (the coefficient mu - lambda ln J of the S^-1 dS S^-1 term
 *             clamped at zero).
 * All pointers are device pointers: s (n x 6), params (n x 8: V, mu,
 * lambda, kappa*a, u_x, u_y, u_z, unused), outputs psi (n), grad (n x 6),
 * hess (n x 36). FP64 when mixed == 0, else the FP32 code path with FP64
 * inputs and outputs. */
int emu_eval_stretch_terms(const double* s, const double* params, int64_t n, int32_t mixed,
                           double* psi, double* grad, double* hess, void* stream);

/* Launch settings of the coupling solves in use: the local polynomial's
 * degree of the mixed path's pipelined CG (0 where that CG is not used),
 * the rows per block of the FP64 CG, and whether emu_create ran the
 * autotuner. Any pointer may be NULL. */
int emu_get_tuning(emu_handle* h, int32_t* cg_local_degree, int32_t* cg64_rows_per_block, int32_t* tuned);

/* Evaluates, on the device, the F-form's element terms (Sec. 3.1 energy,
 * Sec. 3.2.1 Hessian):
 *   psi[i]  = V_i Psi(F_i)  (1e40 V_i when det F_i <= 0),
 *   grad[i] = V_i P(F_i), the first Piola stress (9, row-major F index),
 *   hess[i] = V_i [PSD(Psi_iso''(F_i)) + Psi_fiber''(F_i)] (9 x 9
 *             row-major over the row-major F index): the neo-Hookean
 *             Hessian with its negative eigenvalues clamped at zero, from
 *             its analytic eigen-system in the singular-value frame of F,
 *             plus 2 kappa a I (x) u u^T. NaN where det F_i <= 0.
 * Device pointers: F (n x 9), params (n x 8: V, mu, lambda, kappa*a, u_x,
 * u_y, u_z, unused), outputs psi (n), grad (n x 9), hess (n x 81); any
 * output may be NULL. Synchronises ``stream``. */
int emu_eval_fform_terms(const double* F, const double* params, int64_t n, double* psi, double* grad, double* hess,
                         void* stream);

/* Self-check of the bounded device waits (no counterpart in the paper).
 * Every spin-wait in this library's kernels (the grid barriers of the
 * persistent CG kernels) gives up after about 2 s of GPU time, raises an
 * error word and lets the kernel return, so a solve reports
 * EMU_ERR_TIMEOUT instead of hanging, and the context stays usable. This
 * call runs the same barrier in a two-block cooperative launch in which one
 * block never arrives, with a wait limit of ``wait_ns`` nanoseconds (1e3 to
 * 1e10): it returns EMU_ERR_TIMEOUT when the wait ran out as designed (the
 * expected result), EMU_OK would mean it did not. It allocates 256 bytes of
 * device memory for the duration of the call and synchronises ``stream``. */
int emu_check_bounded_wait(int64_t wait_ns, void* stream);

/* The alpha heuristic of Sec. 3.7: for alpha_rel = alpha0 * factor^k
 * (k = 0 .. max_steps - 1, at most 64; the paper starts at 1 and its table
 * goes by decades) create a solver with *params (NULL: defaults) and that
 * alpha_rel, solve once from the rest state at ``activation`` (n_tets
 * values) and tally the Newton iterations; stop at the first count above
 * jump times the previous one (a solve ending EMU_ERR_NOT_CONVERGED or
 * EMU_ERR_LINESEARCH counts as such an increase) and return in *alpha_out
 * the value before it, else the last value tried. newton_iters (may be
 * NULL; max_steps entries) receives each count (-1: did not converge),
 * *n_tried the number of solves. Each step builds and destroys a handle on
 * ``stream`` (the set-up of Eq. 9 included). EMU_ERR_NOT_CONVERGED if the
 * first value does not converge. */
int emu_alpha_sweep(const emu_mesh_desc* desc, const emu_params* params, const double* activation, double alpha0,
                    double factor, int32_t max_steps, double jump, double* alpha_out, int32_t* newton_iters,
                    int32_t* n_tried, void* stream);

/* Fiber directions from the heat equation (Sec. 3.6, "Modeling"): the P1
 * harmonic field f (the discrete Laplace equation with the rest-volume
 * weighted Laplacian L_ab = sum_i V_i gradN_a . gradN_b) with f = -1 on the
 * origin vertices and +1 on the insertion vertices, then per tet the unit
 * fiber u_i = grad f_i / |grad f_i| (the zero vector where the gradient
 * vanishes). rest_pos: n_verts x 3; tets: n_tets x 4 (either orientation);
 * origin, insertion: vertex indices (disjoint, at least one each); fibers:
 * host output, n_tets x 3 (row-major). The solve runs on the device (FP64 CG
 * to a relative residual of 1e-13). Allocates device memory for the call and
 * synchronises ``stream``. EMU_ERR_INVALID_ARG for bad indices or a
 * degenerate tet; EMU_ERR_PCG if the solve does not converge. Use the result
 * as emu_mesh_desc.fiber_dir. */
int emu_fiber_field(int64_t n_verts, const double* rest_pos, int64_t n_tets, const int32_t* tets,
                    const int32_t* origin, int64_t n_origin, const int32_t* insertion, int64_t n_insertion,
                    double* fibers, void* stream);

/* The capacitance of the Woodbury direction in its Gram form (Eq. 12) from
 * per-tet factors, on the device kernels of the mixed path:
 *   C  = sum_i Yh_i^T Yh_i,  Yh_i = sqrt(w_i) U_i (I3 (x) Gamma_i)   (48 x 48)
 *   By = sum_i w_i (I3 (x) Gamma_i)^T y_i                           (48)
 * with U_i the 6 x 9 chart factor (N_i = U_i^T U_i), Gamma_i the 3 x 16
 * gradients of the 16 scalar modes on tet i (column j = 16 d + l of
 * I3 (x) Gamma_i is e_d (x) Gamma_i[:, l]) and y_i a 9-vector (row-major
 * 3 x 3). Host inputs, component-major over the m tets: U[(9 r + c) m + i]
 * (U_i[r][c]), gamma[(3 l + b) m + i] (Gamma_i[b][l]), y[k m + i], w[i].
 * kernel: 0 = the one a solve on these sizes uses, 1 = tcgen05 tensor
 * cores (m a multiple of 4), 2 = mma.sync tensor cores. Yh is rounded to
 * TF32 and the sums run in FP32 per block, FP64 across blocks. Outputs (host):
 * C row-major, By. Allocates device memory for the call and synchronises
 * ``stream``; EMU_ERR_INVALID_ARG for bad sizes or kernel 1 with m % 4 != 0. */
int emu_eval_capacitance(int64_t m, const float* U, const float* gamma, const float* y, const float* w,
                         int32_t kernel, double* C, double* By, void* stream);

/* Polar decomposition F = R S (R proper rotation, S symmetric positive
 * definite) of n row-major 3x3 matrices with det F > 0, on the device.
 * Outputs R (n x 9) and s (n x 6, ordering as emu_get_element_state). */
int emu_eval_polar(const double* F, int64_t n, double* R, double* s, void* stream);

/* Coupling solve without device allocation. The paper has no counterpart;
 * this exists for callers that cannot call cudaMalloc or any allocating
 * library routine, for instance code running inside a memory pool it does
 * not own, or a host that forbids allocations after start-up.
 *
 * Solves q = q*(F) of Eq. 4 (pinned vertices held as at emu_create) with the
 * handle's ACAP operator, for a per-tet F given by the caller. The iteration
 * starts from the rest-state solution q*(I) and stops at the handle's
 * coupling-solve tolerance min(pcg_tol, 1e-2 tol_rel_residual).
 *   F_device  n_tets x 9 float64 on the device, row-major F per tet (input).
 *   q_device  n_verts x 3 float64 on the device (output).
 *   stream    cudaStream_t the work is enqueued on; the call synchronises it.
 * All scratch memory is one fixed 32 MiB device array inside the library,
 * reserved on every GPU that loads the library until the process exits. A
 * mesh needs 96 n_tets + 144 n_verts bytes plus a few KB; larger meshes are
 * rejected with EMU_ERR_INVALID_ARG. The first call on a device looks up the
 * array's device address (later calls outside stream capture look it up
 * again); make that first call before any stream capture. The device current
 * at the call must be the one the handle was created on (else
 * EMU_ERR_INVALID_ARG). A device reset (cudaDeviceReset) invalidates every
 * handle, this one included. Every call uses the same array and it keeps the
 * last call's contents, so calls that overlap on the GPU (other streams,
 * other threads, other handles) race: serialise them. Returns EMU_ERR_PCG if
 * the CG iteration cap is reached, EMU_ERR_TIMEOUT if a bounded device wait
 * ran out; every failure leaves its reason in emu_last_error(). A handle
 * whose mesh has joints is refused with EMU_ERR_NOT_IMPLEMENTED. */
int emu_acap_solve_noalloc(emu_handle* h, const double* F_device, double* q_device, void* stream);

/* ---- profiling ----------------------------------------------------------
 * Kernel phases of one Newton iteration, in launch order. When profiling is
 * on, every launch of a phase is bracketed by CUDA events on the handle's
 * stream and its device time is accumulated; this adds event records but no
 * synchronisation inside an iteration. */
typedef enum {
  EMU_PHASE_RHS = 0,      /* per tet: corner terms of G^T W (R S) (Eq. 4 RHS)   */
  EMU_PHASE_ASSEMBLE = 1, /* per vertex: gather of corner terms (both solves)  */
  EMU_PHASE_PCG = 2,      /* ACAP conjugate-gradient solves (Eq. 4)            */
  EMU_PHASE_GRAD = 3,     /* per tet: gradient (Eqs. 6-7), chart factor, y      */
  EMU_PHASE_SYRK = 4,     /* capacitance and B y partial sums (Eqs. 11-12)      */
  EMU_PHASE_SMALL = 5,    /* single-block reductions, 48x48 Cholesky, Armijo   */
  EMU_PHASE_DIR = 6,      /* per tet: Woodbury direction and its RHS terms      */
  EMU_PHASE_LS = 7,       /* per tet: line-search energy differences           */
  EMU_PHASE_UPDATE = 8,   /* per tet polar update and per vertex q update       */
  EMU_N_PHASES = 9
} emu_phase;

/* Turns per-phase event timing on (enable != 0) or off and clears the
 * accumulated times and launch counts. */
int emu_set_profiling(emu_handle* h, int32_t enable);

/* Reads the accumulated device milliseconds and launch counts per phase
 * (arrays of n_phases <= EMU_N_PHASES entries, either may be NULL) and the
 * total number of kernel launches the handle issued since profiling was
 * last enabled (counted whether or not timing is on). */
int emu_get_profile(emu_handle* h, double* phase_ms, int32_t* phase_launches, int32_t n_phases,
                    int64_t* total_launches);

#ifdef __cplusplus
}
#endif

#endif /* EMU_H_ */
