/*
 * bodex.h -- C ABI of the GB300 (sm_103a) BODex coarse-stage hot path.
 *
 * BODex (arXiv 2412.16490) synthesises dexterous grasps by a bilevel
 * program (Sec. IV-A, Eqs. (3)-(9)): an upper level does gradient descent
 * on the hand pose x, and at every iteration each of s lower-level QPs
 * finds contact forces that best realise a desired wrench.  One upper
 * iteration of the coarse stage (Secs. IV-B, IV-C) is:
 *
 *   forward kinematics -> fingertip contact points c_i
 *   -> SDF nearest-point query: object point p_i, inward normal n_i
 *   -> grasp matrix G = [G_1 .. G_m] (Eq. (2))
 *   -> s QPs  Q_j = min |beta t_j - G y|^2  over the friction pyramids (Eqs. (7)-(9))
 *   -> energy E = w_Q sum_j Q_j + w_d sum_i (phi_i - alpha - delta)^2
 *   -> dE/dx (envelope theorem) -> Adam step on x, clamp to limits (Eq. (4)).
 *
 * Conventions for every entry point:
 *   - Return value is a status code (BODEX_OK on success).  No C++
 *     exception and no process exit crosses this boundary.
 *     bodex_last_error() returns a message for the calling thread's last
 *     failure.
 *   - Array arguments are CALLER-OWNED DEVICE pointers (e.g. PyTorch CUDA
 *     tensors), contiguous, row-major, float32 unless the comment says
 *     int32.  The library neither frees nor keeps them after the call.
 *     Work is enqueued on `stream` (a cudaStream_t passed as void*; NULL is
 *     the legacy default stream) and is asynchronous.  Launch errors are
 *     reported by the call; faults during execution surface at the next
 *     synchronising call (bodex_sync).
 *   - Descriptor structs (bodex_hand_desc, bodex_object_desc) point to HOST
 *     memory and are copied during the create call.
 *   - Handles own their device memory until *_destroy.
 *   - Per-instance problems (non-finite input, a QP that did not reach the
 *     residual target, a degenerate SDF normal) are written to the optional
 *     `status` outputs and do not fail the call.
 *
 * Notation: B grasps, m contacts, n revolute joints, D = 6 + n pose
 * entries, s desired wrenches, nv = 3m QP variables, nc = 9m + 1 QP rows.
 */
#ifndef BODEX_H
#define BODEX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define BODEX_OK 0
#define BODEX_ERR_INVALID 1        /* bad argument (null pointer, size, unsupported shape) */
#define BODEX_ERR_CUDA 2           /* a CUDA runtime call failed */
#define BODEX_ERR_OOM 3            /* device allocation failed */
#define BODEX_ERR_INFEASIBLE 4     /* gamma > m, gamma < 0, or inverted limits */
#define BODEX_ERR_TIMEOUT 5        /* a bounded device wait gave up */
#define BODEX_ERR_NOT_CONVERGED 6  /* strict mode only: some QP missed eps_abs */

/* per-instance status bits (status outputs) */
#define BODEX_ST_NONFINITE 1       /* non-finite input or result */
#define BODEX_ST_NOT_CONVERGED 2   /* QP residual above eps_abs after max_iter */
#define BODEX_ST_DEGENERATE_NORMAL 4 /* |grad phi| < 1e-12 at a contact */
#define BODEX_ST_POLISHED 8        /* QP result replaced by its polished solution (qp.polish) */

/* ---------------------------------------------------------------- limits */
#define BODEX_MAX_JOINTS 32   /* revolute joints per hand */
#define BODEX_MAX_CONTACTS 5  /* m in {3, 4, 5} are compiled */
#define BODEX_MAX_CHAIN 8     /* joints between the root and a contact link */
#define BODEX_MAX_JOBS 64     /* jobs per bodex_step_multi launch */
#define BODEX_MAX_SPHERES 48  /* collision spheres per hand */

typedef struct bodex_hand_s* bodex_hand_t;
typedef struct bodex_object_s* bodex_object_t;
typedef struct bodex_state_s* bodex_state_t;

/* ---------------------------------------------------------------- hand
 * Hand kinematic tree under a 6-DoF floating base (Sec. IV-B).  Pose
 * reading: x = [tx, ty, tz, rx, ry, rz, q_1 .. q_n]; the root frame is
 * Trans(t) Rx(rx) Ry(ry) Rz(rz).  Joint j's frame is
 *   T_j = T_parent(j) * offset_j * Rot(axis_j, q_j),
 * with parent(j) < j or -1 for the root.  Contact i is the centre of the
 * first fingertip sphere (Sec. IV-C), c_{i,l} in the frame of joint
 * contact_link[i]; its world position is c_{i,w} = R c_{i,l} + T.
 */
typedef struct bodex_hand_desc {
  int n_joints;                /* n, 1..BODEX_MAX_JOINTS */
  int n_contacts;              /* m, 3..BODEX_MAX_CONTACTS */
  const int32_t* parent;       /* [n] */
  const float* offset;         /* [n,12] row-major 3x4 [R | t], parent -> joint */
  const float* axis;           /* [n,3] unit axis in the joint frame */
  const float* qmin;           /* [6+n] lower limits, virtual joints first */
  const float* qmax;           /* [6+n] upper limits */
  const int32_t* contact_link; /* [m] */
  const float* contact_local;  /* [m,3] c_{i,l} */
  float contact_radius;        /* alpha, sphere radius (m) */
  int n_tip_samples;           /* S for the refinement epilogue, 0 if unused */
  const float* tip_samples;    /* [m,S,3] fingertip surface samples, link frame */
  /* Collision spheres for the penetration and self-penetration energies
   * (0..BODEX_MAX_SPHERES; 0 if unused).  Sphere k sits on link
   * sphere_link[k] (-1 = the root/palm frame) at sphere_local[k] with radius
   * sphere_radius[k] > 0.  Self-penetration pairs are all spheres on
   * different links except a link and its nearest ancestor link that
   * carries spheres (the root counts), which touch by construction. */
  int n_spheres;
  const int32_t* sphere_link;  /* [K] */
  const float* sphere_local;   /* [K,3] */
  const float* sphere_radius;  /* [K] */
} bodex_hand_desc;

/* Copies the template to the device.  Errors: BODEX_ERR_INVALID for sizes
 * out of range, a parent index >= its joint, a contact chain longer than
 * BODEX_MAX_CHAIN; BODEX_ERR_INFEASIBLE when qmin > qmax. */
int bodex_hand_create(const bodex_hand_desc* desc, bodex_hand_t* out);
int bodex_hand_destroy(bodex_hand_t hand);

/* ---------------------------------------------------------------- object
 * The object the nearest-point query runs against (Sec. IV-B): an analytic
 * sphere (kind 0) or a signed distance field sampled at the nodes of an
 * N^3 grid (kind 1): node (ix, iy, iz) at origin + h (ix, iy, iz), value
 * index (iz*N + iy)*N + ix, trilinear between nodes; outside the node box
 * phi(c) = phi(clamp(c)) + |c - clamp(c)|.  The object frame's origin for
 * G is the gravity centre (Sec. III): the sphere's centre, or for a grid
 * the mean position of the nodes with negative value, computed in double
 * precision at creation.
 */
typedef struct bodex_object_desc {
  int kind;             /* 0 = sphere, 1 = grid */
  float center[3];      /* sphere */
  float radius;         /* sphere */
  int n;                /* grid nodes per axis, >= 2 */
  float h;              /* grid spacing (m) */
  float origin[3];      /* grid node (0,0,0) */
  const float* values;  /* HOST pointer, [n^3] */
} bodex_object_desc;

/* Uploads the grid on `stream`.  Errors: BODEX_ERR_INVALID, BODEX_ERR_OOM. */
int bodex_object_create(const bodex_object_desc* desc, void* stream, bodex_object_t* out);
int bodex_object_destroy(bodex_object_t obj);
/* Host copy of the gravity centre (object-frame origin). */
int bodex_object_gravity_centre(bodex_object_t obj, float out[3]);

/* ---------------------------------------------------------------- parameters */
/* Lower-level QP (Sec. IV-A).  The friction cone of Eq. (1) is replaced by
 * an inscribed pyramid with 8 edges (1, mu cos(k pi/4), mu sin(k pi/4)) in
 * the contact's (n, d, e) frame; per contact the rows are
 *   0 <= f_n <= 1,  cos(phi_k) f_d + sin(phi_k) f_e - mu cos(pi/8) f_n <= 0,
 *   phi_k = (2k+1) pi/8, k = 0..7,
 * followed by one row  sum_i f_{i,n} >= gamma.  Solved by ADMM in the
 * operator-splitting form of Stellato et al. (OSQP, 2020), batched as in
 * ReLU-QP (Bishop et al., 2024): one explicit K^-1 per grasp shared by its
 * s wrenches, K = P + sigma I + rho A^T A, P = 2 G^T G. */
typedef struct bodex_qp_params {
  float mu;          /* friction coefficient */
  float beta;        /* desired-wrench scale (Eq. (7)) */
  float gamma;       /* minimum total normal force (Eq. (9)), 0 <= gamma <= m */
  float rho;         /* ADMM penalty */
  float sigma;       /* ADMM proximal weight */
  float alpha;       /* ADMM relaxation, in (0, 2) */
  float eps_abs;     /* stop when |A y - z|_inf and |P y + q + A^T lam|_inf <= eps_abs;
                        0 runs exactly max_iter iterations */
  float eps_reg;     /* optional eps |y|^2 added to the objective (0 = off) */
  int max_iter;      /* iteration cap per QP solve */
  int check_every;   /* residual check period (iterations) */
  int warm;          /* 1: start from the y/z/lam passed in, 0: from zero */
  int strict;        /* 1: return BODEX_ERR_NOT_CONVERGED if any QP missed eps_abs
                        (forces a stream synchronisation) */
  int cone;          /* BODEX_CONE_PYRAMID: the 8-facet pyramid of Sec. IV-A (a QP);
                        BODEX_CONE_ELLIPTIC: the unlinearised cone |(f_d, f_e)| <= mu f_n
                        (a second-order-cone program, solved by ADMM with the cone's
                        projection).  ADMM rows, for z and lam: per contact f_n, then
                        8 facets (pyramid, 9m+1 rows in all) or the cone rows
                        (mu f_n, f_d, f_e) (elliptic, 4m+1 rows in all); the sum row last. */
  int adaptive_rho;  /* 1: with eps_abs > 0, adapt rho per grasp by residual balancing
                        (OSQP, Stellato et al. 2020, Sec. 5.2): every check_every
                        iterations each unconverged QP proposes
                        sqrt((|r_p| / s_p) / (|r_d| / s_d)), with s_p = max(|A y|, |z|)
                        and s_d = max(|P y|, |A^T lam|, |q|); when the geometric mean of
                        the grasp's proposals exceeds 5 or 1/5, rho (clamped to
                        [1e-6, 1e6]) is multiplied by it and K^-1 rebuilt.  The
                        returned lam = rho (w - z) uses the grasp's final rho; a warm
                        start reads lam with params->rho.  Results are unchanged up to
                        the residual target; 0: fixed rho.  Ignored when eps_abs == 0
                        (fixed iteration counts). */
  int polish;        /* pyramid cone, eps_reg = 0; bodex_qp_solve_batch only.
                        1: after the ADMM run, solve every QP exactly in FP64 by Wolfe's
                        minimum-norm-point method (the QP is the nearest point of the
                        wrench polytope G C to beta t; Wolfe 1976) and replace y and Q by
                        that minimiser and optimum (Q to FP64 rounding, y rounded to
                        float).  2 (with eps_abs > 0 and a status array): solve exactly,
                        by the float32 method of BODEX_QP_EXACT, only the QPs that ADMM
                        left above eps_abs after max_iter iterations; the others keep
                        their ADMM results bit for bit.  A replaced QP carries
                        BODEX_ST_POLISHED and not BODEX_ST_NOT_CONVERGED; z, lam, res and
                        iters stay those of the ADMM run.  A QP the exact solve gives up
                        on (200 oracle calls in FP64, 64 in float32) keeps its ADMM
                        result.  0: off. */
  int solver;        /* lower-level method.  BODEX_QP_ADMM: the OSQP-form ADMM above.
                        BODEX_QP_EXACT (pyramid cone, eps_reg = 0): the exact optimum by
                        Wolfe's minimum-norm-point method in float32, one QP per thread
                        (the QP is the nearest point of the wrench polytope G C to beta t);
                        it stops when the Frank-Wolfe gap, an upper bound on Q - Q*, is
                        <= 1e-5 Q + 1e-7, when float32 offers no further progress (the
                        oracle's vertex is already in the working set or affinely
                        dependent on it; the gap bound may then be looser than the
                        actual error), or after max_iter oracle calls.  Outputs y, Q;
                        iters = oracle calls; res = (0, the final gap); z = A y clamped
                        to the row bounds and lam = 0 (the method gives no multipliers);
                        BODEX_ST_NOT_CONVERGED when the oracle-call cap stopped it.  rho, sigma, alpha, eps_abs, check_every, warm, polish and
                        adaptive_rho do not apply.  bodex_qp_solve_batch only. */
} bodex_qp_params;

#define BODEX_QP_ADMM 0
#define BODEX_QP_EXACT 1

#define BODEX_CONE_PYRAMID 0
#define BODEX_CONE_ELLIPTIC 1

/* Energy weights (Sec. IV-C): E = w_q sum_j Q_j + w_d sum_i (phi_i - alpha - delta)^2;
 * delta is the 1 cm pre-grasp margin of Sec. IV-D in the coarse stage. */
/* Grasp energies.  BODEX_ENERGY_QP: w_q sum_j Q_j, the lower-level QPs of
 * Eqs. (7)-(9) (with qp.beta = 0 this is the QP baseline of Sec. V-C).
 * BODEX_ENERGY_DFC: the force-closure energy of DFC (Liu et al. 2021, the
 * comparison of Sec. V-C): frictionless contacts pushing with equal unit
 * forces, w_q |sum_i [n_i; p_i x n_i]|^2; no QP is solved (Q and y outputs
 * are 0).  Both add the distance term w_d sum_i (phi_i - alpha - delta)^2. */
#define BODEX_ENERGY_QP 0
#define BODEX_ENERGY_DFC 1

/* Upper-level constraint energies in the style of cuRobo (Sec. IV-B: joint
 * limits, Eq. (4), and no hand-hand / hand-object collision), on the hand's
 * collision spheres (c_k, r_k), all off at weight 0:
 *   w_pen  sum_k h(r_k + eta_pen - phi(c_k)),  h(p) = 0 (p <= 0),
 *          p^2 / (2 eta_pen) (0 < p <= eta_pen), p - eta_pen / 2 (p > eta_pen);
 *   w_self sum_pairs max(0, r_a + r_b - |c_a - c_b|)^2;
 *   w_lim  sum_{k >= 6} max(0, x_k - x_max,k + eta_lim)^2 + max(0, x_min,k + eta_lim - x_k)^2. */
typedef struct bodex_energy_params {
  float w_q;
  float w_d;
  float delta;
  int kind;  /* BODEX_ENERGY_QP or BODEX_ENERGY_DFC */
  float w_pen, w_self, w_lim;
  float eta_pen;  /* activation distance of the penetration hinge (m), >= 0 */
  float eta_lim;  /* margin inside the joint limits (rad), >= 0 */
} bodex_energy_params;

/* Upper-level step: Adam (lr_t for the 3 translations, lr_r for all
 * angles), then clamp x to [qmin, qmax] (Eq. (4)). */
typedef struct bodex_step_params {
  float lr_t, lr_r, b1, b2, adam_eps;
  bodex_energy_params energy;
  bodex_qp_params qp;
  int grasps_per_cta;  /* CTA tile: grasps per thread block (0 = default, 96 / s); an
                          autotuner knob that changes speed, never results */
  int work_pulling;    /* bodex_step_multi only.  0: one thread block per tile (a job's
                          grasps_per_cta grasps), the jobs' tiles in the caller's order,
                          scheduled onto the SMs by the hardware.  1: a persistent grid of
                          as many blocks as fit on the GPU at once; each block takes the
                          next tile from one atomic counter, the tiles of the costliest
                          jobs first, until none is left.  Results equal the jobs' own
                          launches bitwise with 0; with 1, bitwise for fixed-iteration
                          ADMM and within float32 rounding otherwise (the item loop
                          changes the compiler's multiply-add contraction).  1 was
                          measured slower on the mixed-template batch; 0 is the default. */
} bodex_step_params;

/* ---------------------------------------------------------------- calls */

/* FK + nearest-point query + grasp matrix for B poses (Secs. III, IV-B).
 *   x     [B,D]     poses
 *   c_w   [B,m,3]   contact points in the world           (out, may be NULL)
 *   p     [B,m,3]   nearest object points                   (out, may be NULL)
 *   n     [B,m,3]   inward unit normals                     (out, may be NULL)
 *   phi   [B,m]     signed distance of c_w                  (out, may be NULL)
 *   G     [B,6,3m]  grasp matrix, contact i = columns 3i..3i+2 = (n, d, e),
 *                   p measured from the gravity centre     (out, may be NULL)
 *   cell  [B,m,3]   int32 voxel cell of each query (0 for a sphere) (out, may be NULL)
 *   status [B]      int32 per-grasp status bits             (out, may be NULL)
 * Errors: BODEX_ERR_INVALID (null handles or x, B < 0), BODEX_ERR_CUDA. */
int bodex_fk_contacts(bodex_hand_t hand, bodex_object_t obj, const float* x, int B, float* c_w, float* p,
                      float* n, float* phi, float* G, int32_t* cell, int32_t* status, void* stream);

/* Batched lower-level QPs (Sec. IV-A, Eqs. (7)-(9)) for B grasps x s wrenches.
 *   G      [B,6,3m]     grasp matrices
 *   T      [s,6]        desired unit wrenches t_j
 *   y      [B,s,3m]     forces (in: warm start when params->warm, out: solution)
 *   z      [B,s,9m+1]   ADMM constraint copy (in/out, same rule)
 *   lam    [B,s,9m+1]   ADMM multipliers (in/out, same rule)
 *   Q      [B,s]        |beta t_j - G y_j|^2 (+ eps_reg |y_j|^2) at the returned y (out)
 *   iters  [B,s]        int32 iterations used (out, may be NULL)
 *   status [B,s]        int32 status bits (out, may be NULL)
 *   res    [B,s,2]      final (primal, dual) inf-norm residuals (out, may be NULL)
 * m must be 3, 4 or 5; s in 1..16.  Errors: BODEX_ERR_INVALID,
 * BODEX_ERR_INFEASIBLE (gamma outside [0, m]), BODEX_ERR_CUDA,
 * BODEX_ERR_NOT_CONVERGED (strict mode). */
int bodex_qp_solve_batch(const float* G, int B, int m, const float* T, int s, const bodex_qp_params* params,
                         float* y, float* z, float* lam, float* Q, int32_t* iters, int32_t* status, float* res,
                         void* stream);

/* Optimiser state for B grasps and s wrenches: pose x [B,D], Adam moments
 * [B,D], step counter, and the ADMM warm start of every QP.  Owns its
 * device memory.  Errors: BODEX_ERR_INVALID, BODEX_ERR_OOM. */
int bodex_state_create(bodex_hand_t hand, int B, int s, bodex_state_t* out);
int bodex_state_destroy(bodex_state_t state);
/* Sets the pose from a device array [B,D] and resets Adam, the step
 * counter and the ADMM warm start.  Asynchronous on `stream`. */
int bodex_state_set_pose(bodex_state_t state, const float* x, void* stream);
/* Copies the pose to a device array [B,D]. */
int bodex_state_get_pose(bodex_state_t state, float* x, void* stream);
/* Copies, for each grasp, the largest ADMM residual (max of the primal and
 * dual inf-norms over its s QPs) at the last upper iteration of the last
 * bodex_step / bodex_step_multi launch into res [B] (device). */
int bodex_state_get_residual(bodex_state_t state, float* res, void* stream);
/* Copies the Adam moments m, v [B,D] (either may be NULL) and returns the step count. */
int bodex_state_get_adam(bodex_state_t state, float* m, float* v, int* step, void* stream);

/* Energy and gradient at B poses: E [B], dE/dx [B,D] (envelope theorem,
 * Sec. IV-A: the feasible set of the QPs does not depend on x, so
 * dQ_j/dG = -2 r_j y_j^T with r_j = beta t_j - G y_j).
 *   T      [s,6] desired wrenches
 *   warm   optional state whose ADMM warm start is used and updated
 *          (must have been created for the same B and s), or NULL
 *   E      [B]   (out)      dEdx [B,D] (out, may be NULL)
 *   Q      [B,s] (out, may be NULL)   y [B,s,3m] (out, may be NULL)
 *   status [B]   int32 (out, may be NULL)
 * Errors: BODEX_ERR_INVALID, BODEX_ERR_INFEASIBLE, BODEX_ERR_CUDA. */
int bodex_energy_grad(bodex_hand_t hand, bodex_object_t obj, const float* x, int B, const float* T, int s,
                      const bodex_step_params* params, bodex_state_t warm, float* E, float* dEdx, float* Q,
                      float* y, int32_t* status, void* stream);

/* One launch of fused upper iterations for several jobs at once: jobs may
 * use different hand templates (m = 3, 4, 5), objects, batch sizes, wrench
 * sets and step counts.  Each CTA runs one job's tile of grasps; a grasp's
 * result is the same as with bodex_step on its own state (the per-grasp
 * arithmetic does not depend on the other jobs).  The job table travels in
 * the kernel parameters: the call allocates no device memory.  Jobs with
 * B = 0 or n_steps = 0 are skipped; each state's step counter advances by
 * its job's n_steps.
 * Errors: BODEX_ERR_INVALID (n_jobs outside 0..BODEX_MAX_JOBS, null handle,
 * shape mismatch), BODEX_ERR_INFEASIBLE, BODEX_ERR_CUDA. */
typedef struct bodex_job {
  bodex_hand_t hand;
  bodex_object_t obj;
  bodex_state_t state;  /* created for this hand and s */
  const float* T;       /* [s,6] device */
  int s;
  int n_steps;          /* upper iterations for this job in this launch */
  float* E_last;        /* [B] or NULL */
  int32_t* status;      /* [B] or NULL */
} bodex_job;
int bodex_step_multi(const bodex_job* jobs, int n_jobs, const bodex_step_params* params, void* stream);

/* The CTA tile the fused step kernel uses for m contacts and s wrenches:
 * `requested` grasps per thread block (0: the default, 96 / s), capped by
 * 96 lanes and by the shared memory of one block.  A job of B grasps then
 * occupies ceil(B / tile) thread blocks, which is how a scheduler fills one
 * wave of the GPU (4 blocks per SM).  Host-only: touches no device.
 * Errors: BODEX_ERR_INVALID (m outside 3..5, s outside 1..16,
 * requested < 0, null output). */
int bodex_step_tile(int m, int s, int requested, int* grasps_per_cta);

/* Backward pass of the energy for forces y from an earlier solve (the
 * hand-written adjoint behind the autograd binding): recomputes FK, the SDF
 * query and G at x, forms r_j = beta t_j - G y_j, Q_j = |r_j|^2 and E, and
 * applies the envelope-theorem chain dQ_j/dG = -2 r_j y_j^T through the
 * contact frames, the SDF Hessian and the kinematic chain (Secs. III, IV-A,
 * IV-B).  No QP is solved.
 *   x [B,D], T [s,6], y [B,s,3m] (in); E [B] (out, may be NULL), dEdx [B,D]
 *   (out), status [B] (out, may be NULL).
 * Errors: BODEX_ERR_INVALID, BODEX_ERR_INFEASIBLE, BODEX_ERR_CUDA. */
int bodex_energy_adjoint(bodex_hand_t hand, bodex_object_t obj, const float* x, int B, const float* T, int s,
                         const bodex_step_params* params, const float* y, float* E, float* dEdx, int32_t* status,
                         void* stream);

/* n_steps upper-level iterations on the state, fused into one kernel launch:
 * each iteration evaluates E and dE/dx at the current pose (ADMM warm
 * started from the previous iteration, params->qp.max_iter iterations),
 * takes an Adam step and clamps.  E_last [B] (may be NULL) receives E at
 * the last evaluated pose; status [B] (may be NULL) ORs the per-grasp bits.
 * Errors: BODEX_ERR_INVALID, BODEX_ERR_INFEASIBLE, BODEX_ERR_CUDA. */
int bodex_step(bodex_hand_t hand, bodex_object_t obj, bodex_state_t state, const float* T, int s, int n_steps,
               const bodex_step_params* params, float* E_last, int32_t* status, void* stream);

/* Refinement epilogue (fine / final stages, Sec. IV-C, Eqs. (10)-(11), in
 * SDF form; no QP).  n_steps upper iterations on the state (Adam continues
 * from the coarse stage) with the energy
 *   E = w_d sum_i |c'_i - (p^f_i + delta n_out,i)|^2 + w_qp sum_i |c'_i - p^c_i|^2,
 * where c^f_i is the fingertip surface sample (hand desc tip_samples) with
 * the smallest SDF value (lowest index on ties), p^f_i its nearest object
 * point, c'_i = R_i s_{i,k*} + T_i with the sample's link coordinates held
 * fixed (the paper's Detach), and p^c the object points at the end of the
 * coarse stage.  delta = 0.01 gives the pre-grasp pose of the fine stage,
 * delta = 0 the final stage.
 *   p_coarse [B,m,3] (in), E_last [B] (out, may be NULL, energy at the last
 *   evaluated pose), kstar [B,m] int32 (out, may be NULL, the samples chosen
 *   at the last evaluated pose), status [B] (out, may be NULL).
 * Errors: BODEX_ERR_INVALID (no tip samples, shape mismatch), BODEX_ERR_CUDA. */
int bodex_refine(bodex_hand_t hand, bodex_object_t obj, bodex_state_t state, const float* p_coarse, int n_steps,
                 float delta, float w_qp, const bodex_step_params* params, float* E_last, int32_t* kstar,
                 int32_t* status, void* stream);

/* Contact Distance Consistency (Sec. V-B): the spread between the largest
 * and the smallest signed fingertip distance of a grasp.  The signed
 * distance of fingertip i is the smallest SDF value over its surface samples
 * (hand desc tip_samples), or phi(c_i) - alpha for a hand without samples.
 *   x [B,D] (in, device); d [B,m] (out, device, metres); cdc [B] (out,
 *   device, metres, may be NULL): cdc_b = max_i d_bi - min_i d_bi.
 * Asynchronous on `stream`; reads nothing but x, the hand and the object.
 * Errors: BODEX_ERR_INVALID (null handle, B < 0, null x or d), BODEX_ERR_CUDA. */
int bodex_contact_metrics(bodex_hand_t hand, bodex_object_t obj, const float* x, int B, float* d, float* cdc,
                          void* stream);

/* Squeeze pose x_s = 2 x - x_p (Sec. IV-D): the execution target, from the
 * final-stage grasp pose x and the fine-stage pre-grasp pose x_p.
 *   x, x_p [B,D] (in, device, row-major float32); x_s [B,D] (out, device;
 *   may alias x or x_p).  Elementwise, no clamp to the joint limits (the
 *   paper applies none: the squeeze target presses past the grasp).
 * Asynchronous on `stream`.
 * Errors: BODEX_ERR_INVALID (B < 0, D < 1, null array with B > 0),
 * BODEX_ERR_CUDA. */
int bodex_squeeze_pose(const float* x, const float* x_p, int B, int D, float* x_s, void* stream);

/* Allocation-free variant of bodex_step (the paper has no counterpart: this
 * serves callers that cannot allocate device memory while they run, such as
 * real-time control loops that reserve all memory at start-up, or processes
 * whose memory pool owns the device).  It runs n_steps upper iterations on
 * the caller's poses x [B,D] (device, updated in place) exactly as
 * bodex_state_set_pose + bodex_step would, starting from zero Adam moments
 * and a cold ADMM start; those per-grasp states live in a fixed 4 MiB
 * device array inside the library (held by every GPU that loads it until
 * the process exits) instead of a bodex_state_t.
 *   - Allocates nothing: no cudaMalloc or cudaFree, no allocating library
 *     routine.  The caller passes inputs and outputs (E_last [B] and
 *     status [B] may be NULL).
 *   - Size limit: B * (2 (6+n) + s (12 m + 1)) floats, each of the four
 *     regions rounded up to 64 floats, must fit in 1048576 floats (e.g.
 *     B <= 1330 for m = 5, s = 12, n = 22); larger batches return
 *     BODEX_ERR_INVALID before any device work.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.  Under CUDA's default lazy module loading
 *     that first call (and the first call with a hand of a new contact
 *     count m, whose kernel lives in another module) also loads the
 *     library's code and the array onto the device, which does allocate
 *     device memory: a caller with a no-allocation phase makes one warm-up
 *     call per device and per hand template at start-up, before that phase.
 *     Calls after the warm-up allocate nothing.
 *   - All calls share the array and each clears what it uses before its
 *     kernel runs: calls that overlap on the GPU (other streams, other host
 *     threads) race and must be serialised by the caller.
 * Errors: as bodex_step. */
int bodex_step_noalloc(bodex_hand_t hand, bodex_object_t obj, float* x, int B, const float* T, int s, int n_steps,
                       const bodex_step_params* params, float* E_last, int32_t* status, void* stream);

/* Blocks until `stream` is idle; BODEX_ERR_CUDA if a fault occurred. */
int bodex_sync(void* stream);
/* Message for the calling thread's last non-OK status ("" if none). */
const char* bodex_last_error(void);
/* Library version string. */
const char* bodex_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BODEX_H */
