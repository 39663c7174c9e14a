/*
 * qpat.h -- C ABI of the GB300 hot path of QPAT reconstruction with
 * total-variation-type priors (priorconditioned LSQR, lagged diffusivity,
 * matrix-free Jacobians of the diffusion approximation).
 *
 * Paper references below are to its sections, equations, Algorithm 1 and
 * Appendix.  Conventions common to every call:
 *
 *  - Units follow the caller (the paper uses mm and mm^-1).
 *  - Node vectors have length N and are in the CALLER's node order; the
 *    library permutes to its own locality order internally.  Stacked
 *    per-illumination vectors are K x N row-major (illumination k is the
 *    contiguous row k), as in the stacking rule of Sec. 4.
 *  - Parameter vectors of the derivative calls are beta = [kappa_tilde; mu_tilde]
 *    in R^{2N} (log parameters, Eq. (4)); kappa, mu are the nodal (P1)
 *    coefficients kappa_n = kappa_0 exp(kappa_tilde_n), mu_n = mu_0 exp(mu_tilde_n).
 *  - Boundary faces are numbered in the canonical order: each face written
 *    with its three caller node ids ascending, faces sorted lexicographically.
 *    Per-face flux arrays (K x F) use this order.
 *  - Plain calls take HOST pointers, copy in, compute on the GPU and copy
 *    out before returning.  *_dev calls take DEVICE pointers (any CUDA
 *    allocation of the current device) and a cudaStream_t passed as void*;
 *    they are asynchronous with respect to the host except where noted.
 *  - The caller owns every array it passes.  The mesh handle owns the device
 *    copy of the mesh and a workspace that grows on demand (cudaMalloc);
 *    both are released by qpat_mesh_free.
 *  - Every int-returning call returns QPAT_OK (0) or a negative code; the
 *    outputs are then undefined and qpat_last_error() (thread-local) says why.
 *  - A mesh handle must not be used by two host threads at once.
 */
#ifndef QPAT_H
#define QPAT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    QPAT_OK = 0,
    QPAT_EINVAL = -1,      /* bad argument: sizes, NULL, degenerate tet, ... */
    QPAT_ENOCONV = -2,     /* a linear solve hit its iteration cap */
    QPAT_EBREAKDOWN = -3,  /* PCG breakdown: p.Ap <= 0 or a NaN/Inf scalar */
    QPAT_ETIMEOUT = -4,    /* a bounded grid barrier gave up waiting */
    QPAT_ECUDA = -5,       /* a CUDA runtime call failed */
    QPAT_ENOMEM = -6
};

typedef struct qpat_mesh_s* qpat_mesh_t;

/* Solver and Algorithm 1 parameters.  Defaults (qpat_default_params):
 * T = 5e-3, b/a = 1, delta = 1e-6, m0 = 10, tau = 1e-2 (Sec. 4, end),
 * 5 linearisations including step 0 and 50 LSQR rounds as caps,
 * FP64 PCG to a relative residual of 1e-13. */
typedef struct {
    double T;              /* Perona-Malik edge scale, Eq. (10) */
    double b_over_a;       /* prior weight ratio, Eq. (16) */
    double delta;          /* M_delta = M + delta I, Eq. (19) */
    double tau;            /* stopping threshold, Eq. (22) */
    int m0;                /* stopping window, Eq. (22) */
    int max_lin;           /* linearisations, step 0 counted (Sec. 5) */
    int max_lsqr;          /* LSQR rounds per linearisation */
    int fixed_counts;      /* 1: run exactly max_lin x max_lsqr, no Eq. (22) stop
                              (the step-4 acceptance of Algorithm 1 stays active) */
    int precision;         /* 0: FP64 PCG; 1: FP32 PCG inside FP64 refinement for
                              the K solves (M_delta solves always run in FP64:
                              their conditioning, set by delta, is beyond FP32) */
    int max_pcg_iter;      /* cap per PCG run (inner run for precision 1) */
    double pcg_rtol;       /* |b - A x| / |b| target of every K and M_delta solve */
    int fit_grid;          /* (kappa_0, mu_0) search grid per axis (Algorithm 1) */
    int fit_gn_steps;      /* Gauss-Newton polish steps of that search */
    int patch_nodes;       /* owned nodes per CTA patch (0 = library choice) */
    int fp32_operator;     /* FP32 inner operator of precision 1: 0 = matrix-free
                              element recomputation, 1 = assembled FP32 values */
    int pcg_variant;       /* PCG on assembled operators: 0 = library choice
                              (currently 1, the fastest measured), 1 = two grid
                              reductions per iteration (textbook order),
                              2 = one grid reduction per iteration
                              (Chronopoulos-Gear recurrences; the same iterates
                              in exact arithmetic, more vector traffic),
                              3 = as 1 with the operator streamed through a
                              shared-memory ring by bulk copies (QPAT_EINVAL
                              if the ring does not fit).  Matrix-free FP32
                              runs always use 1. */
    int prior;             /* r(t) of the prior R(u) = integral r(|grad u|), Eq. (9):
                              0 = Perona-Malik, Eq. (10) (the paper's examples);
                              1 = smoothed TV^q, r(t) = (t^2 + T^2)^(q/2) / q, one
                              of the alternatives named after Eq. (10) (q = 1:
                              smoothed total variation).  The lagged step
                              weights each tet by r'(t)/t (Eq. (14)). */
    int mixed_restart;     /* precision 1: 0 = reliable updates (each FP32 inner run
                              continues the previous search direction, rescaled,
                              after r is replaced by the true FP64 residual);
                              1 = restart the inner PCG at every refinement sweep */
    int poly_degree;       /* preconditioner of the K solves on assembled operators
                              with pcg_variant 0/1: 0 = Jacobi (D^-1); 1..8 = block
                              Jacobi over the CTA patches, each block's inverse
                              approximated by a Chebyshev polynomial of this degree
                              in D^-1 A_pp (A_pp: the couplings among the patch's
                              owned nodes), on [hi / 50, hi] with hi the Gershgorin
                              bound of D^-1 A.  A fixed symmetric positive definite
                              operator, so PCG converges to the same solution in
                              fewer (and costlier) iterations.  Other variants and
                              the matrix-free FP32 operator use Jacobi.  Default 2. */
    int prior_poly_degree; /* the same for the M_delta solves (default 2) */
    int step_halvings;     /* Algorithm 1, not in the paper (default 0 = the
                              paper's rule): before rejecting a step in step 4,
                              try beta + 2^-j (beta_new - beta), j = 1..this;
                              step 0's update is then kept only if one of
                              x, x/2, ... lowers the residual.  In [0, 16]. */
    double prior_q;        /* q of prior 1, in (0, 2] */
    int lsqr_reorth;       /* LSQR of Algorithm 1 (step 0 and step 3): 1 (default) =
                              with full reorthogonalisation of both Golub-Kahan
                              bases (classical Gram-Schmidt, twice), which gives
                              the iterates of exact arithmetic to rounding;
                              0 = the plain recurrence.  The same method in exact
                              arithmetic; in floating point the plain recurrence
                              loses orthogonality after a few tens of rounds (the
                              1/delta mode of M_delta^-1 re-enters), and one
                              50-round sweep then moves by percents under 1e-13
                              perturbations of the solves.  Keeps
                              (max_lsqr + 1) x (K N + 4 N) doubles on the device. */
    int64_t barrier_spin_limit; /* bounded grid-barrier waits of the persistent
                              PCG kernels: polls (each ~32 ns of sleep) before a
                              waiting CTA gives up with QPAT_ETIMEOUT;
                              0 = library default (about 2 s). */
    int multigrid;         /* preconditioner of the K and M_delta solves (not in the
                              paper, which prescribes no linear solver; every choice
                              reaches the same pcg_rtol):
                              0 = the persistent PCG above (poly_degree,
                              prior_poly_degree);
                              1 = conjugate gradients with one V-cycle of
                              smoothed-aggregation algebraic multigrid per
                              iteration (Vanek, Mandel, Brezina 1996: aggregates
                              of the matrix graph, P = (I - 4/(3 hi) D^-1 A) P_tent,
                              Galerkin coarse operators P^T A P, Chebyshev
                              smoothing in D^-1 A, an exact dense solve on the
                              coarsest level of <= 128 rows), all in FP64; the K
                              solves then run FP64 iterates whatever `precision`
                              says;
                              2 = as 1 with the V-cycle of the K solves in FP32
                              (the CG iterates stay FP64 and take the flexible
                              beta = r.(z - z_old) / (r.z)_old); M_delta keeps the
                              FP64 cycle.
                              The hierarchy's patterns are built on the host on the
                              first such solve of a mesh (seconds at 2 M nodes),
                              its values on the device once per prepared operator. */
    int mg_degree;         /* Chebyshev degree of each multigrid smoothing, 1..8
                              (default and 0: 1, i.e. one damped-Jacobi step
                              before and after each coarse correction; on GB300
                              every fine-level step is an FP64 sparse product,
                              and degree 1 was the fastest measured) */
    double mg_ratio;       /* the smoothing polynomial targets [hi / mg_ratio, hi] of
                              the spectrum of D^-1 A, hi its Gershgorin bound
                              (> 1; 0 = 30) */
} qpat_params;

/* Report of qpat_reconstruct (Algorithm 1). */
typedef struct {
    double kappa0, mu0;            /* background fit or the given values */
    int linearisations;            /* step 0 counted */
    int accepted_last;             /* 0 if step 4 rejected the last LSQR result */
    int lsqr_iters[32];            /* rounds run in each linearisation */
    double residuals[33];          /* |Gamma^-1/2 (chi - h)| after each accepted step */
    int64_t pcg_iters;             /* total PCG iterations (all solves) */
    int64_t solves;                /* total linear solves (RHS counted) */
    int64_t refinements;           /* FP64 refinement sweeps (precision 1) */
    double ms_total;               /* device wall time of the call */
} qpat_report;

void qpat_default_params(qpat_params* p);

/* Thread-local message describing the last error of this thread. */
const char* qpat_last_error(void);

/* Number of CUDA kernels this library has launched in this process (every
 * launch statement counts; a replayed batch graph counts its one kernel).
 * Host-side counter, never reset; take differences around a region.  Not in
 * the paper. */
int64_t qpat_launch_count(void);

/* ---------------------------------------------------------------- mesh */

/* Builds a mesh handle from N node coordinates (xyz, N x 3, row-major) and
 * E tetrahedra (tets, E x 4, 0-based caller node ids, any orientation).
 * The P1 basis of Eq. (5) lives on this mesh.  Copies both arrays; extracts
 * the boundary faces (faces owned by one tet), orders nodes for locality,
 * splits them into CTA patches and uploads everything to the current
 * device.  Fails with QPAT_EINVAL on ids out of range or a degenerate tet. */
int qpat_mesh(const double* xyz, int64_t N, const int32_t* tets, int64_t E,
              qpat_mesh_t* out);

/* Same, with the owned-node patch size chosen by the caller (>= 32). */
int qpat_mesh_ex(const double* xyz, int64_t N, const int32_t* tets, int64_t E,
                 int patch_nodes, qpat_mesh_t* out);

void qpat_mesh_free(qpat_mesh_t mesh);

/* Host-only preparation check (needs no GPU): builds the mesh structures of
 * qpat_mesh_ex and verifies them.  info8 (11 entries) receives F, patches,
 * max touched nodes per patch, max owned nodes, max tets per patch, max faces
 * per patch, total patch-tet entries (>= E; the excess is the tets duplicated
 * on patch borders), total patch-face entries, the stored nonzeros of the
 * assembled K pattern, those of the prior's stiffness-only pattern (pairs
 * with a non-zero gradient coupling in a shared tet), and the largest number
 * of tet colours in a patch (the element kernels sum colour by colour; no two
 * tets of a colour share an owned node, which is checked).  faces (F x 3) and
 * perm (N) are filled when not NULL.  Returns QPAT_EINVAL with a message if a
 * check fails. */
int qpat_mesh_host_info(const double* xyz, int64_t N, const int32_t* tets, int64_t E,
                        int patch_nodes, int64_t* info8, int32_t* faces, int32_t* perm);

/* Host-only check (needs no GPU) of the multigrid hierarchy that
 * qpat_params.multigrid builds for the K pattern (prior = 0) or the prior's
 * pattern (prior = 1) of the mesh qpat_mesh_ex would prepare: builds the
 * aggregates, the level patterns and the index plans of the device set-up
 * and verifies every invariant the device relies on (P rows, R = P^T, the
 * slots of A P and P^T A P, symmetric coarse patterns, a coarsest level of
 * at most 128 rows).  Writes the rows of each level (finest first, up to
 * max_levels) and returns the level count, or QPAT_EINVAL with a message. */
int qpat_multigrid_host_info(const double* xyz, int64_t N, const int32_t* tets, int64_t E,
                             int patch_nodes, int prior, int64_t* rows, int max_levels);

/* Counters of the linear solves run with this mesh since creation or the
 * last reset: out4 = {PCG iterations, solves (RHS), FP64 refinement sweeps,
 * PCG launches}. */
int qpat_mesh_stats(qpat_mesh_t mesh, int64_t* out4);
/* Precision-1 solves of K whose FP32 inner PCG broke down, or whose FP64
 * refinement stalled, and that were therefore solved again by the FP64 PCG
 * (since the last reset); -1 for a NULL mesh. */
int64_t qpat_mesh_fp64_fallbacks(qpat_mesh_t mesh);
int qpat_mesh_reset_stats(qpat_mesh_t mesh);
/* Sum over the PCG launches since the last reset of iterations times the
 * right-hand sides of the launch (a block solve may run as several launches
 * when one launch's shared memory cannot hold all its right-hand sides);
 * -1 for a NULL mesh.  Not in the paper (diagnostics). */
int64_t qpat_mesh_rhs_iterations(qpat_mesh_t mesh);

/* Rows of every level of the multigrid hierarchy built for the K pattern
 * (prior = 0) or the prior's pattern (prior = 1), finest first, into rows
 * (up to max_levels); returns the number of levels (0 before the first
 * multigrid solve of that kind).  Not in the paper (diagnostics). */
int qpat_mesh_multigrid_levels(qpat_mesh_t mesh, int prior, int64_t* rows, int max_levels);

/* With timing on (qpat_mesh_set_timing): the summed device time (ms) and
 * the count of the fine-level Chebyshev smoothing launches of the multigrid
 * cycles since the last reset (the cycle's dominant kernel; each launch
 * bracketed by CUDA events on its stream).  Not in the paper (diagnostics). */
int qpat_mesh_multigrid_fine_time(qpat_mesh_t mesh, double* ms, int64_t* launches);

/* When on, every PCG launch is bracketed by CUDA events recorded on the
 * stream it is launched on; qpat_mesh_pcg_time returns the summed device
 * time (ms) of those launches since the last reset. */
int qpat_mesh_set_timing(qpat_mesh_t mesh, int on);
int qpat_mesh_pcg_time(qpat_mesh_t mesh, double* ms);

int64_t qpat_mesh_num_nodes(qpat_mesh_t mesh);
int64_t qpat_mesh_num_tets(qpat_mesh_t mesh);
int64_t qpat_mesh_num_faces(qpat_mesh_t mesh);
int64_t qpat_mesh_num_patches(qpat_mesh_t mesh);
/* Stored entries of the assembled operators (node pairs sharing a tet,
 * the diagonal included), without the sliced-ELLPACK padding. */
int64_t qpat_mesh_num_entries(qpat_mesh_t mesh);
/* Stored entries of each assembled prior block (M(u) of Eq. (14) plus
 * delta I): the node pairs whose gradient coupling is non-zero in a shared
 * tet, the diagonal included (7 per interior row on Kuhn meshes). */
int64_t qpat_mesh_num_prior_entries(qpat_mesh_t mesh);

/* Stored nonzeros that couple two nodes owned by the same patch, in the K
 * pattern (prior = 0) or the prior pattern (prior = 1): the entries the
 * patch-local Chebyshev preconditioner applies (poly_degree).  -1 if mesh
 * is NULL. */
int64_t qpat_mesh_num_local_entries(qpat_mesh_t mesh, int prior);

/* Boundary faces in canonical order (F x 3 caller node ids, ascending). */
int qpat_mesh_faces(qpat_mesh_t mesh, int32_t* faces);

/* Library node order: perm[i] = caller id of library node i (N entries). */
int qpat_mesh_permutation(qpat_mesh_t mesh, int32_t* perm);

/* Face-constant flux of a square boundary patch (Sec. 5, Test 2 uses such
 * characteristic functions): flux_face[f] = amp if all three vertices of
 * face f lie on the plane through c with unit normal n (to 1e-9 of the mesh
 * extent) and its centroid lies in the closed square of half width half_w
 * about c (infinity norm over the in-plane axes), else 0.  F entries. */
int qpat_flux_patch(qpat_mesh_t mesh, const double c[3], const double n[3],
                    double half_w, double amp, double* flux_face);

/* Face-constant flux through the curved side of a cylinder (Sec. 5, Test 1),
 * canonical face order: Phi = amp cos(pi/2 (theta - theta0) / half_w) for
 * |theta - theta0| <= half_w, else 0 (half_w = pi/8 gives the paper's
 * cos(4 (theta - theta0))), homogeneous along the axis.  A face is on the
 * side iff its three vertices lie at distance `radius` (within 1e-9 of the
 * mesh extent) from the axis line through c along `axis`; it takes Phi at
 * the polar angle of its centroid, measured about the axis from `ref`
 * (projected off the axis).  flux_face: F doubles, caller-owned.
 * QPAT_EINVAL for NULL pointers, a zero axis, ref parallel to the axis, or
 * radius, half_w <= 0. */
int qpat_flux_side(qpat_mesh_t mesh, const double c[3], const double axis[3], const double ref[3],
                   double radius, double theta0, double half_w, double amp, double* flux_face);

/* ------------------------------------------------------- operator apply */

/* y = K(kappa, mu) x for R right-hand sides: the FE matrix of the weak form
 * of Eq. (1) (Appendix): integral kappa grad x . grad v + mu x v plus
 * 1/2 integral over the boundary of x v, with P1 nodal kappa and mu.
 * x, y: N x R node-major (x[n*R + r]), caller order, device pointers.
 * mode 0: FP64 matrix-free element apply; 1: FP32 matrix-free; 2: FP64
 * assembled (sliced ELLPACK) values; 3: FP32 assembled values.  Inputs and
 * outputs stay FP64 in every mode. */
int qpat_apply_K_dev(qpat_mesh_t mesh, int precision, const double* kappa,
                     const double* mu, int R, const double* x, double* y,
                     void* stream);

/* -------------------------------------------------------- forward model */

/* phi^(k) = K^{-1} f^(k), h^(k) = mu * phi^(k) for K illuminations
 * (Appendix; Eq. (2) and (7)), f_i = 2 integral Phi lambda_i over the
 * boundary with face-constant Phi.  flux_face: K x F; phi, h: K x N.
 * Either output may be NULL.  Solved as one K-RHS block PCG. */
int qpat_forward(qpat_mesh_t mesh, const qpat_params* prm, const double* kappa,
                 const double* mu, int K, const double* flux_face,
                 double* phi, double* h);
int qpat_forward_dev(qpat_mesh_t mesh, const qpat_params* prm, const double* kappa,
                     const double* mu, int K, const double* flux_face,
                     double* phi, double* h, void* stream);

/* qpat_forward_dev started from an initial guess phi0 (K x N, caller order,
 * device; NULL = zero), e.g. a learned prediction.  The solve stops at the
 * same absolute residual |f - K phi| <= pcg_rtol |f| as from zero, so the
 * guess changes only the work, not the accuracy. */
int qpat_forward_guess_dev(qpat_mesh_t mesh, const qpat_params* prm, const double* kappa,
                           const double* mu, int K, const double* flux_face,
                           const double* phi0, double* phi, double* h, void* stream);

/* Allocation-free forward solve, for callers that cannot allocate device
 * memory when they need a solve: real-time pipelines that forbid allocator
 * calls after start-up (cudaMalloc may block on the driver), and hosts that
 * budget every byte of GPU memory themselves.  The paper has no counterpart;
 * it computes the same phi = K^-1 f and h = mu * phi as qpat_forward_dev in
 * FP64 (matrix-free operator, Jacobi PCG to a relative residual rtol, at most
 * max_iter iterations), with every scratch vector in one fixed file-scope
 * device array of 4,835,488 doubles (about 39 MB) that each GPU using the
 * library keeps until the process exits.
 *  - Limit: N x R <= 524,288, R = K rounded up to 1, 2, 4, 8 or 16;
 *    larger problems return QPAT_EINVAL without touching the GPU.
 *  - kappa, mu: N; flux_face: K x F; phi, h: K x N (either may be NULL);
 *    all device pointers owned by the caller; stream is a cudaStream_t.
 *  - The mesh handle must already exist (qpat_mesh allocates).
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress, with that device current; the driver may load
 *    the library's device code then); make that first call before any
 *    stream capture.  No call allocates or frees device memory.
 *  - Every call shares the one array, which keeps the last call's contents
 *    (the call zeroes what must start at zero): calls that overlap on the
 *    GPU (other streams, other threads, other meshes) race and must be
 *    serialised by the caller.  The call synchronises the stream before
 *    returning (it reads the solver status). */
int qpat_forward_noalloc_dev(qpat_mesh_t mesh, const double* kappa, const double* mu,
                             int K, const double* flux_face, double rtol, int max_iter,
                             double* phi, double* h, void* stream);

/* out = w o (J s), stacked over K illuminations (Appendix):
 *   J s = diag(mu) K^{-1} (G1 diag(kappa) s1 + G2 diag(mu) s2) + diag(phi) diag(mu) s2
 * with G1_ij = -integral phi_j grad(varphi).grad(phi_i), G2_ij = -integral phi_j varphi phi_i.
 * phi: K x N forward solutions at (kappa, mu); w: K x N whitening weights
 * Gamma^{-1/2} (NULL = 1); s: 2N; out: K x N.  The G matrices are never formed. */
int qpat_jvp(qpat_mesh_t mesh, const qpat_params* prm, const double* kappa,
             const double* mu, int K, const double* phi, const double* w,
             const double* s, double* out);
int qpat_jvp_dev(qpat_mesh_t mesh, const qpat_params* prm, const double* kappa,
                 const double* mu, int K, const double* phi, const double* w,
                 const double* s, double* out, void* stream);

/* out = J^T (w o t) summed over the K illuminations (Appendix):
 *   J^T t = blkdiag(kappa, mu) ([G1^T; G2] K^{-1} diag(mu) t + [0; diag(phi) t]).
 * t: K x N; out: 2N. */
int qpat_vjp(qpat_mesh_t mesh, const qpat_params* prm, const double* kappa,
             const double* mu, int K, const double* phi, const double* w,
             const double* t, double* out);
int qpat_vjp_dev(qpat_mesh_t mesh, const qpat_params* prm, const double* kappa,
                 const double* mu, int K, const double* phi, const double* w,
                 const double* t, double* out, void* stream);

/* One Jv and one J^T w of independent inputs solved together as a single
 * 2K-RHS block PCG (the K solves of each are independent): out_jv = w o (J s)
 * (K x N) and out_vjp = J^T (w o t) (2N). */
int qpat_jvp_vjp_pair_dev(qpat_mesh_t mesh, const qpat_params* prm,
                          const double* kappa, const double* mu, int K,
                          const double* phi, const double* w, const double* s,
                          const double* t, double* out_jv, double* out_vjp,
                          void* stream);
/* The same with host pointers (copied to and from the device on the mesh's
 * stream; returns when out_jv and out_vjp are written).  K in [1, 8]. */
int qpat_jvp_vjp_pair(qpat_mesh_t mesh, const qpat_params* prm,
                      const double* kappa, const double* mu, int K,
                      const double* phi, const double* w, const double* s,
                      const double* t, double* out_jv, double* out_vjp);

/* ------------------------------------------------ learned initial guess */

/* A 3D U-Net that predicts the fluence of one illumination on an n^3 Kuhn
 * grid (node index = voxel index), used as the initial guess of
 * qpat_forward_guess_dev.  Not in the paper: the forward solve it feeds is
 * the Appendix's K^-1 f and still runs to the same tolerance.  Four levels
 * with 16, 32, 64, 128 channels, two 3x3x3 ReLU convolutions per level,
 * 2x2x2 average pooling, nearest upsampling with skip concatenation and a
 * linear output convolution.  Every convolution, forward and backward, runs
 * on hand-written BF16 tensor-core kernels (fp32 accumulation); Adam keeps
 * fp32 master weights.  n must be a multiple of 16 in [32, 512].
 * Features (qpat_unet_features_dev): per voxel [log(mu/0.01),
 * log(kappa/0.33), f_k / h^2] with f_k the load vector of illumination k
 * (2 integral Phi_k lambda_i) -- x is K x N x 3 float.
 * predict: x (B x n^3 x 3 float) -> y (B x n^3 float).
 * train: one Adam step on the mean-squared error of B samples (targets t,
 * B x n^3 float, e.g. forward solutions); *loss (host, may be NULL) gets the
 * mean loss before the step.  Device pointers, asynchronous on stream except
 * when loss is requested.  Parameters: per convolution the fp32 weights
 * [27][c_out][c_in] then the bias [c_out]. */
typedef struct qpat_unet_s* qpat_unet_t;
int qpat_unet_create(int n, uint64_t seed, qpat_unet_t* out);
void qpat_unet_free(qpat_unet_t unet);
int64_t qpat_unet_num_params(qpat_unet_t unet);
int qpat_unet_get_params(qpat_unet_t unet, float* host);
int qpat_unet_set_params(qpat_unet_t unet, const float* host);
int qpat_unet_features_dev(qpat_mesh_t mesh, const double* kappa, const double* mu, int K,
                           const double* flux_face, double h, float* x, void* stream);
int qpat_unet_predict_dev(qpat_unet_t unet, const float* x, int B, float* y, void* stream);
int qpat_unet_train_dev(qpat_unet_t unet, const float* x, const float* t, int B, float lr,
                        float* loss, void* stream);
/* Output mode: floor > 0 makes the network learn log(max(phi, floor)) of its
 * targets (training loss in log space) and predict the exponential of its
 * output, so that fields spanning decades are fitted relative to their size;
 * floor = 0 (default) fits and predicts phi itself.  QPAT_EINVAL for a NULL
 * network or a negative or non-finite floor. */
int qpat_unet_set_log_output(qpat_unet_t unet, double floor);
/* The training loss of those B samples and its gradient with respect to
 * every parameter (summed over the samples, no update): grad (HOST,
 * qpat_unet_num_params floats, the layout of qpat_unet_get_params), *loss
 * (host, may be NULL).  Synchronous. */
int qpat_unet_grad_dev(qpat_unet_t unet, const float* x, const float* t, int B, float* grad,
                       float* loss, void* stream);
/* y (float) -> out (double), count entries (the guess handed to the solve). */
int qpat_unet_to_double_dev(const float* y, int64_t count, double* out, void* stream);

/* The BF16 tensor-core 3x3x3 convolution of the U-Net on its own (tests and
 * users of the kernels): in [n^3][Cin] bf16 (Cin % 16 == 0), w
 * [27][Cout][Cin] bf16 (Cout % 8 == 0), bias fp32 (NULL = 0), zero padding;
 * out bf16 [n^3][Cout], out_f32 (optional) the fp32 values before rounding.
 * wgrad: dw [27][Cout][Cin] and db [Cout] (fp32) of that convolution for an
 * output gradient dy [n^3][Cout] bf16 (Cin % 8 == 0, Cout % 16 == 0,
 * n^3 % 16 == 0); partial: scratch of qpat_conv3d_bf16_wgrad_scratch floats. */
int qpat_conv3d_bf16_dev(const void* in, int Cin, const void* w, const float* bias, int Cout,
                         int relu, int n, void* out, float* out_f32, void* stream);
int qpat_conv3d_bf16_wgrad_dev(const void* in, int Cin, const void* dy, int Cout, int n,
                               float* dw, float* db, float* partial, void* stream);
int64_t qpat_conv3d_bf16_wgrad_scratch(int n, int Cin, int Cout);
/* Convolution engine of qpat_conv3d_bf16_dev and of the U-Net (process-wide):
 * 0 (default) = tcgen05 tensor cores with a tensor-memory accumulator where
 * the shape allows (Cout % 16 == 0, 16 <= Cout <= 256), else mma.sync;
 * 1 = mma.sync only.  QPAT_EINVAL for other values.  Not in the paper. */
int qpat_conv3d_set_engine(int engine);
/* Bounded waits of the tcgen05 convolution that gave up since the library
 * was loaded (their tiles are written as NaN); 0 in normal operation. */
int qpat_conv3d_tc_timeouts(void);

/* ---------------------------------------------------------- autotuner */

/* Times `iters` FP32 PCG iterations (K right-hand sides, host kappa and mu
 * in caller order) for each candidate patch size {library default, 128,
 * 256, 512, 1024 owned nodes per CTA} and each FP32 operator form
 * {matrix-free, assembled}, building a mesh per candidate; returns the
 * fastest pair (best_patch_nodes 0 = the default of qpat_mesh) and, if not
 * NULL, the microseconds per iteration of all candidates in that order
 * (us_per_iter needs 10 entries; *ncand receives the count).  Pass the
 * winners to qpat_mesh_ex / qpat_params.fp32_operator.  Not in the paper. */
int qpat_autotune(const double* xyz, int64_t N, const int32_t* tets, int64_t E,
                  const double* kappa, const double* mu, int K, int iters,
                  int* best_patch_nodes, int* best_fp32_operator,
                  double* us_per_iter, int* ncand);

/* ---------------------------------------------------- uneven batches */

/* A batch of forward solves (as qpat_forward_dev, FP64, assembled K) on
 * several meshes of different sizes.  All solves run in ONE cooperative
 * launch: each problem gets CTAs in proportion to its node count (at least
 * one, at most one per patch) and synchronises only those.  The whole
 * sequence (layout changes, assembly of K, load vectors, the batched PCG,
 * the output layout) is recorded into a CUDA graph on the first
 * qpat_batch_forward and replayed afterwards.  Illuminations are padded to
 * a common R = K_max rounded up to 1, 2, 4 or 8 (K_j <= 8).  FP64 PCG to
 * pcg_rtol with prm->poly_degree's preconditioner (Jacobi if 0).  Stacked
 * illuminations follow Sec. 4; the solve is the Appendix's K^-1 f.
 * Ownership: the batch allocates (at creation) and owns per problem j the
 * device buffers kappa_j, mu_j (N_j), flux_j (K_j x F_j, canonical faces)
 * and phi_j (K_j x N_j) returned by qpat_batch_buffers; the caller fills
 * the inputs, runs qpat_batch_forward(stream) and reads phi_j after the
 * stream completes.  The meshes must outlive the batch. */
typedef struct qpat_batch_s* qpat_batch_t;
int qpat_batch_create(int nprob, const qpat_mesh_t* meshes, const int* K,
                      const qpat_params* prm, qpat_batch_t* out);
int qpat_batch_buffers(qpat_batch_t batch, int j, double** kappa, double** mu,
                       double** flux, double** phi);
/* Asynchronous on `stream` (a cudaStream_t); the first call records the graph. */
int qpat_batch_forward(qpat_batch_t batch, void* stream);
/* Per problem: PCG status (QPAT_OK, QPAT_ENOCONV, ...), iterations and CTAs
 * of the last run (synchronous; any array may be NULL). */
int qpat_batch_status(qpat_batch_t batch, int* status, int* iters, int* ctas);
void qpat_batch_free(qpat_batch_t batch);

/* ------------------------------------------------------------- prior */

/* out = M_delta^{-1} rhs with M_delta = blkdiag(M(kt), (b/a) M(mt)) + delta I
 * (Eqs. (14), (16), (19)); M(u) is the FE matrix of -div(c_u grad) with
 * natural boundary condition and the Perona-Malik lagged diffusivity
 * c_u = r'(|grad u|)/|grad u| = 1/(1 + |grad u|^2/T^2) per tet (Eq. (10)).
 * kt, mt: N; rhs, out: 2N.  Uses prm->T, b_over_a, delta. */
int qpat_prior_solve(qpat_mesh_t mesh, const qpat_params* prm, const double* kt,
                     const double* mt, const double* rhs, double* out);
int qpat_prior_solve_dev(qpat_mesh_t mesh, const qpat_params* prm, const double* kt,
                         const double* mt, const double* rhs, double* out,
                         void* stream);

/* ------------------------------------------------------- Algorithm 1 */

/* Algorithm 1 with step 0 (Sec. 5) and K stacked illuminations (Sec. 4):
 * background fit (unless kappa0_mu0 != NULL), mu_tilde initialisation,
 * step 0 (kappa-only LSQR), then linearise / lagged diffusivity /
 * priorconditioned LSQR (Eqs. (21)-(22)) / acceptance until max_lin
 * linearisations or a rejected step.  flux_face: K x F; chi, sigma: K x N
 * (Gamma = diag(sigma^2)); kappa, mu: N outputs; rep may be NULL.
 * Host pointers; blocks until done. */
int qpat_reconstruct(qpat_mesh_t mesh, const qpat_params* prm, int K,
                     const double* flux_face, const double* chi,
                     const double* sigma, const double* kappa0_mu0,
                     double* kappa, double* mu, qpat_report* rep);

/* Checkpoint / resume of Algorithm 1.  The state between linearisations is
 * the background pair (kappa_0, mu_0), beta^(l) = (kappa_tilde, mu_tilde) and
 * the count l (step 1 of Algorithm 1 restarts from beta^(l) alone).
 * beta_out (2N, caller order: kappa_tilde then mu_tilde; may be NULL)
 * receives the final beta; with beta_in == NULL this is qpat_reconstruct.
 * With beta_in != NULL the run resumes at step 1 from beta^(l) = beta_in
 * after lin_done >= 1 linearisations (step 0 counted), kappa0_mu0 required,
 * and continues until max_lin or a rejected step; rep->linearisations then
 * counts from lin_done, and rep->residuals[0] is the residual at beta_in.
 * Everything on the device sums in a fixed order, so a run stopped at
 * max_lin = l and resumed from its kappa0/mu0, beta_out and
 * rep->linearisations gives the same bits as one uninterrupted run.
 * QPAT_EINVAL if beta_in is given without kappa0_mu0 or with lin_done < 1. */
int qpat_reconstruct_ex(qpat_mesh_t mesh, const qpat_params* prm, int K,
                        const double* flux_face, const double* chi,
                        const double* sigma, const double* kappa0_mu0,
                        const double* beta_in, int lin_done, double* kappa,
                        double* mu, double* beta_out, qpat_report* rep);

#ifdef __cplusplus
}
#endif

#endif /* QPAT_H */
