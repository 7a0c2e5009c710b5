/*
 * stst.h -- C ABI of the GB300 space-time least-squares Schroedinger solver.
 *
 * The library solves the Hermitian positive definite linear system A u = f of
 * the space-time isogeometric least-squares discretization of
 *     i d_t u - nu Delta u (+ V(x) u) = f  in (0,T) x (0,1)^d,
 *     u = 0 on (0,T) x boundary,  u(0) = u0,
 * (Bressan, Kushova, Sangalli, Tani, arXiv 2311.18461: Sec. 2, Sec. 4.2-4.3)
 * by conjugate gradients preconditioned with the paper's P-hat, applied by
 * Fast Diagonalization (Sec. 5, Algorithm 1). Every numerical step runs in
 * the library's CUDA kernels on the device the handle was created on.
 *
 * Conventions shared by all calls
 *  - Directions: index 0 is time, 1..d are the spatial directions.
 *  - Discretization: uniform open knot vectors with n_el[l] elements, degree
 *    p[l], maximal regularity (Sec. 3.1); time basis without its first
 *    function (n_t = n_el[0] + p[0] - 1), spatial bases without the two end
 *    functions (n_l = n_el[l] + p[l] - 2) (Sec. 3.2, Eq. all_basis).
 *  - Vectors: complex128 stored as interleaved (re, im) doubles, ordered by the
 *    vec operator of Sec. 3.3 with time as the FASTEST index:
 *      index = i_t + n_t * (i_1 + n_1 * (i_2 + n_2 * i_3)),  length N_dof = n_t * prod n_l.
 *  - Quadrature: (p[l] + 2) Gauss-Legendre points per element in every
 *    direction, element by element from left to right.
 *  - Memory: every vector argument is a DEVICE pointer owned by the caller,
 *    16-byte aligned; calls are ordered on the handle's CUDA stream. The
 *    library owns all factors and workspaces of a handle; no call after
 *    stst_create allocates device memory, except stst_set_potential (which
 *    re-plans), stst_set_geometry and stst_batch_create.
 *  - Return value: STST_OK (0); a positive value is a numerical outcome, a
 *    negative value is a usage or CUDA error (see stst_strerror).
 */
#ifndef STST_H
#define STST_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  STST_OK = 0,
  STST_NOT_CONVERGED = 1, /* maxit reached before the tolerance                          */
  STST_BREAKDOWN = 2,     /* <p, A p> <= 0 or not finite in CG                            */
  STST_NOT_HPD = 3,       /* a factorization met a non-positive pivot                     */
  STST_TIMEOUT = 4,       /* a bounded device-side wait expired                           */
  STST_ERR_ARG = -1,      /* invalid argument (null pointer, size out of range, ...)      */
  STST_ERR_HANDLE = -2,   /* null or destroyed handle                                     */
  STST_ERR_OOM = -3,      /* device allocation failed                                     */
  STST_ERR_CUDA = -4,     /* a CUDA runtime call failed                                   */
  STST_ERR_STATE = -5     /* call out of order (e.g. apply_prec before build_fd)          */
};

/* Precision of the preconditioner's Fast Diagonalization (the system
 * mat-vec, residuals, inner products and updates are always FP64). */
enum {
  STST_PREC_FP64 = 0, /* mode products and time solves in FP64                        */
  STST_PREC_FP32 = 1, /* mode products and time solves in FP32                        */
  STST_PREC_BF16 = 2  /* mode products on tensor cores, BF16 operands, FP32 accumulate */
};

/* Formulation (stst_create2). STST_FORM_LS: the least-squares method (Sec. 4.3): unknowns on the time
 * basis without its first function, the initial datum enters by lifting. STST_FORM_UW: the ultraweak
 * method (Sec. 4.4, Eq. uw-discrete-system): the same matrix (S B_j, S B_i) on the time basis without
 * its last function (final conditions at T); the initial datum enters the right-hand side and the
 * discrete solution is u_h = S z_h for the computed z_h. */
enum {
  STST_FORM_LS = 0,
  STST_FORM_UW = 1
};

typedef struct stst_problem *stst_handle;

/*
 * stst_create: set up a discretization (Sec. 3-4) on the unit box (0,1)^d in
 * space and (0,T) in time, with coefficient nu > 0 (Eq. problem).
 *   d          number of spatial directions, 1..3
 *   n_el[d+1]  elements per direction (time first), each >= 1
 *   p[d+1]     degrees per direction (time first); p[0] in 1..8, p[l] in 2..8
 *              (C^1 in space, Assumption 2); n_l = n_el[l]+p[l]-2 <= 128
 *   T, nu      final time and diffusion coefficient, > 0
 *   prec_mode  STST_PREC_*
 *   stream     cudaStream_t used by every call of the handle (NULL: legacy default stream)
 * Assembles the 1D matrices on the device (Eq. time_mat, Eq. space_mat).
 * Allocates the handle's device memory. Errors: ERR_ARG, ERR_OOM, ERR_CUDA.
 * stst_create is stst_create2 with formulation STST_FORM_LS; every other call works for both
 * formulations (stst_rhs computes each one's right-hand side).
 */
int stst_create2(stst_handle *h, int d, const int *n_el, const int *p, double T, double nu, int prec_mode,
                 int formulation, void *stream);
int stst_create(stst_handle *h, int d, const int *n_el, const int *p, double T, double nu, int prec_mode,
                void *stream);

/* stst_destroy: free the handle and all its device memory (synchronizes its stream). */
int stst_destroy(stst_handle h);

/* stst_strerror: static description of a status code. */
const char *stst_strerror(int status);

/* stst_sizes: n_dof (unknowns) and the reduced sizes n[0..d] (time first). Host outputs. */
int stst_sizes(stst_handle h, long long *n_dof, int *n);

/*
 * stst_quadrature_points: the n_el[dir]*(p[dir]+2) Gauss points of direction
 * dir (0 = time on (0,T), else (0,1)), written to the device array pts.
 * Callers sample potentials, forcing and initial data at these points.
 */
int stst_quadrature_points(stst_handle h, int dir, double *pts);

/*
 * stst_assemble_1d: univariate Galerkin matrices of Eq. time_mat / Eq. space_mat
 * for degree p, n_el uniform elements on (0, length):
 *   M = int b_i b_j, L = int b'_j b'_i, J = int b''_i b''_j, K = int b'_j b_i,
 *   K2 = int b''_j b_i  (times the weight w(x) if weight != NULL).
 * bc: 0 keep all m = n_el+p functions, 1 drop the first (time), 2 drop the
 * first and last (space). weight: NULL or a device array with the weight at
 * the n_el*(p+2) quadrature points of (0, length).
 * Outputs (device, any may be NULL): band storage, row-major n x (2p+1),
 * out[i*(2p+1) + (j-i+p)] = A[i][j] for |i-j| <= p (zero outside the matrix).
 * n_out (host, may be NULL) receives the number of rows n. Ordered on `stream`.
 */
int stst_assemble_1d(int p, int n_el, double length, int bc, const double *weight, double *M, double *L, double *J,
                     double *K, double *K2, int *n_out, void *stream);

/*
 * stst_set_potential: a separable potential V(x) = sum_{r<rank} prod_l v_{r,l}(x_l)
 * added to the operator, S_V = i d_t - nu Delta + V (an extension; the paper
 * treats V = 0). v_qp (device) packs, for r = 0..rank-1 and l = 1..d, the values
 * of v_{r,l} at the quadrature points of direction l (stst_quadrature_points).
 * rank = 0 removes the potential. The preconditioner stays the V-free P-hat
 * (Eq. prec_definition). Re-plans the mat-vec; may allocate. rank <= 3.
 * Errors: STST_ERR_ARG (bad rank, NULL samples, or a sample that is not finite:
 * the handle keeps its previous potential); STST_ERR_OOM / STST_ERR_CUDA part-way:
 * the potential is removed (V = 0), and if even that operator cannot be planned,
 * every call that applies the matrix returns STST_ERR_STATE until a later
 * stst_set_potential succeeds. Batches (stst_batch_create) captured the previous
 * operator: destroy and re-create them after changing the potential.
 * A factor identically 1 at every quadrature point counts as absent. When each
 * term r has exactly one factor different from 1 and no two terms share a
 * direction (V = sum_l v_l(x_l), e.g. a harmonic potential), the mat-vec groups
 * the operator as i d_t + sum_l H_l and costs as many band applications as V = 0.
 */
int stst_set_potential(stst_handle h, int rank, const double *v_qp);

/*
 * stst_set_geometry: the system on a mapped domain Omega = F((0,1)^d) (Sec. 3.2: the isoparametric
 * push-forward through G(tau, eta) = (T tau, F(eta)); Eq. syst_mat with the spatial matrices of
 * Eq. space_mat integrated over Omega). The matrix keeps the form M_s (x) L_t + nu^2 B_s (x) M_t +
 * nu L_s (x) (W_t + W_t^*) with the parametric time matrices; M_s, L_s, B_s are assembled by quadrature
 * from the map's derivatives: jac[q][m][a] = dF_m / d eta_a and hess[q][m][a][b] = d^2 F_m / (d eta_a
 * d eta_b) (device, row-major per point) at the spatial quadrature points q, the tensor grid of the
 * directions' points (stst_quadrature_points) with direction 1 fastest: q = q_1 + Q_1 (q_2 + Q_2 q_3),
 * Q_l = n_el[l] (p[l] + 2). The library keeps the three matrices as stencils of (2 p_l + 1) entries per
 * direction and row and applies them in place of the parametric mat-vec (stst_apply_sys, stst_pcg_solve,
 * FP64). The preconditioner keeps the structure of the parametric P-hat (the paper's fast solver is
 * for F = id only, Sec. 5), with one change: the eigenvalues of direction l (Algorithm 1 step 1) are
 * multiplied by s_l = int |det J| G^{ll} / int |det J| (G = J^{-1} J^{-T}), the mean scale of the physical
 * Laplacian along l. For an affine map with sides a_l, s_l = 1 / a_l^2 and the scaled P-hat is the box's own
 * preconditioner up to a constant factor; without the scales the parametric P-hat mismatches the
 * operator's time-space balance and PCG needs more iterations the finer the mesh. Setting or removing a
 * geometry marks the preconditioner stale: call stst_build_fd again. jac = NULL removes the geometry.
 * A handle with a geometry cannot join a batch (stst_batch_create: STST_ERR_STATE). Least-squares formulation without potential only; stst_rhs, stst_rhs_lift and
 * stst_rhs_noalloc (parametric integrals) and stst_ir_solve (FP32 mat-vec) return STST_ERR_STATE while a
 * geometry is set: the caller supplies the mapped-domain load vector. Allocates (about
 * 3 N_s (2p+1)^d doubles and three vectors) and synchronizes the handle's stream.
 * Errors: STST_ERR_ARG (hess NULL, (2p+1)^d > 729, or a map whose Jacobian determinant vanishes or
 * changes sign at a quadrature point: the previous operator stays); STST_ERR_STATE (a potential is set,
 * or the ultraweak formulation); STST_ERR_OOM.
 * stst_geometry_info: whether a geometry is set, the stored entries per row, and the d eigenvalue scales
 * s_l (host outputs, each may be NULL; the scales are 1 without a geometry).
 */
int stst_set_geometry(stst_handle h, const double *jac, const double *hess);
int stst_geometry_info(stst_handle h, int *mapped, int *entries_per_row, double *prec_scales);

/*
 * stst_set_prec_operator: the spatial operator the preconditioner is built from (an extension).
 *   0  the paper's P-hat (Eq. prec_definition): the potential-free stiffness nu L_l (default);
 *   1  P_V: for a potential that is a sum of one-direction factors (see stst_set_potential), the
 *      Galerkin matrices G_l = nu L_l + M_{v_l} of H_l = -nu d_ll + v_l in place of nu L_l. Algorithm 1
 *      is unchanged with the eigenpairs of (G_l, M_l) and H_i = L_t + lambda_i^2 M_t + lambda_i (W_t + W_t^*).
 *      With V = 0 it is P-hat.
 * ERR_ARG for another op, or for 1 while the potential is not such a sum. A change takes effect at the
 * next stst_build_fd (apply_prec and the solves return ERR_STATE until then). With 1 selected,
 * stst_set_potential invalidates the preconditioner as well (P_V depends on V), and stst_build_fd
 * returns ERR_STATE if the potential it installed is not such a sum.
 */
int stst_set_prec_operator(stst_handle h, int op);

/*
 * stst_build_fd: preconditioner setup, step 1 of Algorithm 1 plus the
 * per-eigenvalue time operators H_i = L_t + nu^2 lambda_i^2 M_t + nu lambda_i (W_t + W_t^*)
 * (Sec. 5.2). Generalized eigenpairs of (L_l, M_l) with U_l^T M_l U_l = I
 * (Eq. space_eig), banded Cholesky factors of every H_i. Returns STST_NOT_HPD
 * if a factorization meets a non-positive pivot.
 */
int stst_build_fd(stst_handle h);

/* stst_apply_sys: y = A x, Eq. syst_mat (+ potential terms). x, y: device, N_dof complex, distinct. */
int stst_apply_sys(stst_handle h, const double *x, double *y);

/* stst_apply_prec: s = P-hat^{-1} r by Algorithm 1 steps 2-4 in the handle's precision. Needs build_fd. */
int stst_apply_prec(stst_handle h, const double *r, double *s);

/*
 * stst_rhs: right-hand side of the reduced system (Sec. 4.3, Sec. 2.2):
 *   rhs_i = int f conj(S_V B_i)  -  sum_j A_full(b_1 B_j, S_V B_i) c_j,
 * where c = M_s^{-1} (u0, B_j) is the L2 projection of u0 onto the spatial
 * space and b_1 the first time basis function (the lifting of the initial datum).
 *   f_qp   NULL (f = 0) or device complex array on the space-time quadrature
 *          grid, time fastest: f_qp[q_t + Q_t*(q_1 + Q_1*(q_2 + ...))]
 *   u0_qp  NULL (u0 = 0) or device complex array on the spatial grid, x_1 fastest
 *   rhs    device, N_dof complex (output)
 *   c0     NULL or device, N_s complex: receives c (the lifted initial datum;
 *          the discrete solution is u_h = u_bar + b_1(t) sum_j c_j B_j(x)).
 * For STST_FORM_UW handles (Sec. 4.4): rhs_i = int f conj(B_i) + i (u0, B_i(., 0)); the initial term
 * sits on time index 0 (the only time function nonzero at t = 0) and nothing is lifted; c0 still
 * receives M_s^{-1} (u0, B_j). The potential does not enter this right-hand side.
 */
int stst_rhs(stst_handle h, const double *f_qp, const double *u0_qp, double *rhs, double *c0);

/*
 * stst_rhs_lift: right-hand side with general (non-homogeneous) Dirichlet and initial data, the
 * lifting of Sec. 2.2 with the data taken from a function u given on the whole space-time cylinder
 * (as in the experiments of Sec. 6, whose exact solutions supply their boundary values):
 *   G = (M_t^{-1} x M_1^{-1} x ... x M_d^{-1}) (u, B)  over ALL basis functions (no boundary conditions),
 *   g_h = the part of G on the basis functions nonzero at t = 0 or on the spatial boundary
 *         (time index 0, spatial indices 0 and m_l - 1; zero elsewhere),
 *   rhs_i = (f - S_V g_h, S_V B_i), i.e. int f conj(S_V B_i) - sum_j A_full(B_j, B_i) g_j.
 * The discrete solution is u_h = u_bar + g_h (u_bar the reduced solution on the interior functions).
 *   f_qp  NULL (f = 0) or device complex array on the space-time quadrature grid (layout of stst_rhs)
 *   u_qp  device complex array on the same grid: the function whose boundary and initial values are
 *         imposed (required)
 *   rhs   device, N_dof complex (output)
 *   xd    NULL or device complex array of prod_l m_l entries, m_l = n_el_l + p_l the full number of
 *         basis functions per direction, time fastest: receives g_h's coefficients on the full basis.
 * Least-squares handles only (STST_ERR_ARG for STST_FORM_UW or u_qp == NULL). Allocates stream-ordered
 * temporaries of a few grid-sized arrays (STST_ERR_OOM if that fails); stream-ordered, returns
 * without waiting.
 */
int stst_rhs_lift(stst_handle h, const double *f_qp, const double *u_qp, double *rhs, double *xd);

/*
 * stst_rhs_noalloc: the same right-hand side as stst_rhs, computed without
 * taking any device memory at call time. (The paper has no counterpart: this
 * is an interface for callers that cannot allocate.) stst_rhs with a forcing
 * grid allocates temporaries for every call; some callers cannot let it:
 * code that records the call while a CUDA stream is being captured into a
 * graph, where cudaMalloc and cudaFree are not allowed, and programs whose
 * device memory is already claimed by their own pool or a fixed budget, where
 * an allocation inside the solver could fail or fragment that pool. This
 * variant keeps its temporaries in one static device array of 16 MiB
 * (2^20 complex128 values) built into the library: every GPU that loads the
 * library holds it until the process exits. The first call on a device looks
 * up the array's device address (with that device current); make that first
 * call before any stream capture. The lookup is repeated when the device's
 * context has changed (after cudaDeviceReset the module is loaded again): the
 * first call in a new context is again a set-up call. The forcing path needs
 * 3 n_t prod_l Q_l complex values of it for the ultraweak load, 4 for the
 * least-squares load and 5 for the least-squares load with a potential
 * (Q_l = n_el[l]*(p[l]+2)); larger problems return STST_ERR_ARG and do nothing.
 * The initial-datum path uses the
 * handle's own workspaces. All calls share the array: calls whose work may
 * overlap on the GPU (other streams, other host threads, other handles on the
 * same device) race on it and must be serialized by the caller. Nothing in it
 * has to start at zero. Arguments and outputs as for stst_rhs.
 */
int stst_rhs_noalloc(stst_handle h, const double *f_qp, const double *u0_qp, double *rhs, double *c0);

/*
 * stst_pcg_solve: P-hat-preconditioned conjugate gradients (Sec. 5.3, Sec. 6)
 * from the initial guess in x (x is overwritten by the solution). Stops when
 * ||rhs - A x_k||_2 <= tol ||rhs||_2 (recursive residual) or after maxit
 * iterations. With the FP64 preconditioner this is the paper's PCG. With a
 * low-precision one (STST_PREC_FP32 / BF16, a slightly different operator at
 * every application) it is the flexible CG of Notay (2000) with one kept
 * direction: complex alpha = <r, p> / <p, A p> (exact line search) and
 * complex beta = -<z, A p> / <p, A p> (each direction A-orthogonal to the
 * previous one); for a fixed Hermitian preconditioner both give the same
 * iterates. iters, relres: host outputs (may be NULL).
 * Needs build_fd. Returns OK, NOT_CONVERGED or BREAKDOWN, or TIMEOUT when a
 * bounded device-side wait expired since the last solve (the BF16 tensor-core
 * mode products wait on their MMAs' completion barrier; the flag is then
 * cleared). The loop runs as one CUDA graph with a device-side while
 * condition: the host waits once.
 */
int stst_pcg_solve(stst_handle h, const double *rhs, double *x, double tol, int maxit, int *iters, double *relres);

/*
 * stst_ir_solve: mixed-precision iterative refinement (an extension): FP64
 * residual rhs - A x and FP64 update x += d around an inner FP32 flexible CG on
 * A d = r (FP32 mat-vec, FP32/BF16 preconditioner, inner tolerance inner_tol).
 * Stops when the FP64 relative residual <= tol or after maxit outer steps.
 * iters receives the total inner iterations, outer the outer steps. Returns
 * as stst_pcg_solve (TIMEOUT included).
 */
int stst_ir_solve(stst_handle h, const double *rhs, double *x, double tol, int maxit, double inner_tol,
                  int inner_maxit, int *iters, int *outer, double *relres);

/*
 * Batched solves (an extension; the paper solves one problem at a time).
 * stst_batch_create: builds ONE CUDA graph that solves `count` independent problems, each given by
 * its own handle (any sizes, degrees, potentials, precision modes), its right-hand side rhs[i] and
 * its solution array x[i] (device pointers, fixed at creation; x[i] holds the initial guess on
 * input). Each problem is a separate branch of the graph: preconditioner setup as in
 * stst_build_fd, then PCG as in stst_pcg_solve with its loop as a conditional WHILE node; the
 * branches share nothing, so the GPU runs them concurrently. Handles must be distinct and must not
 * be used by other calls while a batch solve runs. stream: NULL creates a stream for the batch.
 * Allocates; the handles keep their own workspaces. STST_ERR_STATE for a handle with a geometry
 * (stst_set_geometry): mapped-domain problems are solved one at a time.
 * stst_batch_solve: one graph launch solving every problem to ||rhs - A x|| <= tol ||rhs|| within
 * maxit iterations; waits for completion. iters, relres, status (host arrays of length count, may be
 * NULL) receive each problem's outcome; the return value is STST_OK or the first non-OK status.
 */
typedef struct stst_batch_s *stst_batch;
int stst_batch_create(stst_batch *b, int count, const stst_handle *handles, const double *const *rhs,
                      double *const *x, void *stream);
int stst_batch_solve(stst_batch b, double tol, int maxit, int *iters, double *relres, int *status);
int stst_batch_destroy(stst_batch b);

/*
 * stst_set_autotune: mode 1 (the default) makes stst_build_fd and stst_batch_create time the candidate
 * tiles of the SIMT mode products (8 cpt columns with cpt in {2, 4}, 32 rpt output rows with rpt in 1..4,
 * per CTA; with the FP32 preconditioner also a wide tile of 256 columns x 32 rows, 8 rows x 4 columns
 * per thread) once per problem shape and precision, keeping the fastest (cached for the process); mode 0
 * uses the fixed default (32 columns, all rows of the mode up to 128 per CTA); mode 10 rpt + cpt forces
 * that tile, mode 132 the wide one (FP32 preconditioner), where it fits in shared memory. Results do not depend on the tile (each output is summed in the
 * same order); the grouping of the PCG dot-product partials does. Process-wide, for handles whose
 * preconditioner is built afterwards. STST_ERR_ARG for other modes.
 * stst_tile_info: the tile of direction dir (1..d) of the handle: columns and output rows per CTA
 * (host, may be NULL) and its measured microseconds per launch (0 when not measured).
 */
int stst_set_autotune(int mode);
/*
 * stst_set_time_solver: the kernel of Algorithm 1 step 3 (the N_s banded time solves): mode 0 (default)
 * chooses per problem shape when the preconditioner is built (timed under autotune mode 1, else the
 * segmented kernel when the sequential one would leave SMs idle); 1 = sequential recurrences (one thread
 * per system); 2 = segmented, parallel in time where its shared memory fits: the time axis is cut into
 * S <= 8 segments that run concurrently, with P x P transfer matrices (precomputed from the factors by
 * stst_build_fd) carrying the recurrence state across segments. The two give the same solves up to
 * rounding. Process-wide, for handles whose preconditioner is built afterwards. STST_ERR_ARG otherwise.
 * stst_time_solver_info: for precision STST_PREC_FP64 (0) or STST_PREC_FP32 (1) factors: the number of
 * segments (0 when the segmented kernel does not fit), their length, and whether it is used (host).
 */
int stst_set_time_solver(int mode);
/*
 * stst_set_fused_transforms: for d = 2 or 3 with the FP32 preconditioner and n_1, n_2 <= 80, the mode
 * products of directions 1 and 2 in Algorithm 1 steps 2 and 4 can run as one kernel (S CTAs per slab
 * (t, i_3) take its n_1 x n_2 slab through both products in shared memory; the forward transform is
 * split by rows, the backward one by columns) instead of two mode-product kernels; direction 3 stays
 * a mode-product kernel. Mode 0 (default) chooses per shape when the
 * preconditioner is built (separate kernels or fused, timed under autotune mode 1; fused, the forward
 * and the backward transform each take the split S = 1..4 that times fastest for it; else fused with
 * the smallest S that gives two CTAs per SM); 1 = separate kernels; 2 = fused with that default split;
 * 11..14 = fused with S = mode - 10 for both transforms (the default split where S would leave a part
 * empty). All give bitwise equal preconditioner outputs (same summation order and FP32
 * intermediate). Process-wide, for handles whose preconditioner is built afterwards; STST_ERR_ARG for
 * other modes. stst_fused_transforms_info: S of the handle's forward transform, 0 when it uses separate
 * kernels.
 */
int stst_set_fused_transforms(int mode);
/*
 * stst_set_pencil: the last spatial direction's steps of Algorithm 1 with the FP32 preconditioner. After
 * the forward products of directions 1..d-1, every pencil (fixed eigen-indices j_1..j_{d-1}) holds complete
 * time series of n_d eigen-systems, so the forward product along direction d (step 2), the n_d banded time
 * solves (step 3, Eq. independent_problems) and the backward product along d (step 4) can run in one kernel
 * with the pencil in shared memory: one CTA per pencil, or a cluster of two CTAs that split its rows and
 * exchange the solved halves through distributed shared memory. The time-solve kernel and one transform
 * launch per application disappear. Mode 0 (default) chooses per shape when the preconditioner is built
 * (whole applications timed under autotune mode 1, else the cluster of two where it fits); 1 = off (separate
 * kernels); 2 = one CTA per pencil; 3 = a cluster of two. Needs p[0] <= 4 and the pencil in shared memory;
 * elsewhere the separate kernels run. Same results up to rounding (the sums of each product run in the same
 * order; the time solves are the sequential recurrences). Process-wide, for handles whose preconditioner is
 * built afterwards; STST_ERR_ARG for other modes. stst_pencil_info: CTAs per pencil of the handle, 0 when the
 * pencil kernel is not used.
 */
int stst_set_pencil(int mode);
int stst_pencil_info(stst_handle h, int *ctas_per_pencil);
/*
 * stst_set_tensor_products: mode products of Algorithm 1 (steps 2 and 4) on the tensor cores with the FP32
 * preconditioner. Per direction l the product with U_l (or U_l^T) is a real GEMM whose rows are the real
 * and imaginary parts of 64 complex columns; the TMA unit copies each 64-column tile (all n_l rows of one
 * outer index) into shared memory, every value is split into two TF32 parts, and three tcgen05 TF32
 * products (high x high, high x low, low x high; FP32 accumulation in tensor memory) give about the
 * accuracy of the FP32 SIMT products. It applies where the input is FP32 with an even inner extent (the row
 * pitch of the copy must be a multiple of 16 bytes) and n_l <= 80 (its shared memory); elsewhere the SIMT
 * tile runs. Mode 0 (default): a candidate of the tile autotuner (autotune mode 1), kept per direction when
 * faster; 1 = off; 2 = used wherever it applies. Results agree with the SIMT products up to rounding (the
 * sums run in another order). Process-wide, for handles whose preconditioner is built afterwards;
 * STST_ERR_ARG for other modes. stst_tensor_products_info: bit l of *dirs (host) is set when direction l's
 * mode products use the tensor cores (FP32 preconditioner; where they run as separate products, not inside
 * the fused 2D transforms or the pencil kernel, see stst_set_fused_transforms and stst_set_pencil; a mode
 * product whose input is not 16-byte aligned runs on the SIMT tile).
 */
int stst_set_tensor_products(int mode);
/*
 * stst_set_fused_matvec: the levels of the sum-factorised mat-vec (Eq. kron_vec_multi applied as a few
 * passes of banded one-direction products) in one launch, with a grid barrier between levels, instead of
 * one launch per level. Mode 0 (default): one launch per level; 1: one launch wherever the last level's
 * 512-thread partial-sum grid fits the GPU at once (measured on c2: 112.7 us per mat-vec against 108.6 us
 * for the separate launches, the two barriers cost more than the launch ramps they remove; kept as an
 * option). FP64 mat-vecs only (the FP32 one of
 * stst_ir_solve's inner solve keeps one launch per level). The outputs and the PCG's partial sums are
 * bitwise those of the unfused launches. Handles in a batch (stst_batch_create) never fuse: their
 * branches run concurrently. A barrier that waits too long sets a flag that the solve reports as
 * STST_TIMEOUT. Process-wide, read at every mat-vec; captured solver graphs keep the form they were
 * captured with. STST_ERR_ARG for other modes.
 */
int stst_set_fused_matvec(int mode);

/*
 * stst_persistent_solve: the PCG of Sec. 5.3 and Sec. 6 (P-hat preconditioner, x_0 = 0, relative residual
 * tol, at most maxit iterations) for `count` problems in ONE kernel launch: problem i is solved from start
 * to end by one thread-block cluster of cluster_ctas CTAs (1, 2, 4, 8 or 16; 0 = 8), whose threads share
 * every phase of the loop (the mat-vec's levels, <p, A p>, the updates, Algorithm 1 steps 2-4 with the
 * sequential banded time solves, <r, z>) and meet at the cluster's hardware barrier between phases; the
 * vectors stay in L2. For small problems, where a solve of separate kernels pays each kernel's latency
 * (Table 1 sizes), and for many problems at once. Handles: distinct, built (stst_build_fd) with the FP64
 * preconditioner (STST_PREC_FP64: plain CG, the paper's method), no geometry, degrees up to 4; any
 * potential, formulation and sizes (a larger problem only takes longer: one cluster per problem).
 * Measured (2D+t, p = 3): about 70 us per iteration at n_el = 8, below the graph solve's cost; at
 * n_el = 16 and above the graph solve (the whole GPU per problem) is faster; the cluster's phases are
 * bound by their L2 round trips and the FP64 rate of a few SMs. rhs[i], x[i]:
 * device vectors of handle i (x[i] receives the solution). iters, status, relres: host arrays of count
 * (may be NULL). Uses the handles' work vectors, synchronizes their streams, launches on `stream`
 * (NULL: the first handle's stream), allocates and frees about 7 KB per problem, and returns when the
 * solves are done: the largest per-problem status (STST_OK, STST_NOT_CONVERGED, STST_BREAKDOWN), or
 * STST_ERR_ARG / STST_ERR_HANDLE / STST_ERR_STATE (a handle not built, not FP64, with a geometry, with a
 * degree above 4, or with a plan of more than four levels) / STST_ERR_CUDA. Results equal stst_pcg_solve's up to rounding (its
 * sums run in another order).
 */
int stst_persistent_solve(int count, const stst_handle *handles, const double *const *rhs, double *const *x,
                          double tol, int maxit, int cluster_ctas, int *iters, int *status, double *relres,
                          void *stream);
int stst_tensor_products_info(stst_handle h, int *dirs);
int stst_fused_transforms_info(stst_handle h, int *fused);
/* The splits S of the handle's fused forward and backward transforms (both 0: separate kernels); either
 * pointer may be NULL. STST_ERR_HANDLE for an invalid handle. */
int stst_fused_transforms_split(stst_handle h, int *forward, int *backward);
int stst_time_solver_info(stst_handle h, int precision, int *segments, int *segment_len, int *segmented);
/* Name and description of the CUDA error behind the calling thread's last STST_ERR_CUDA (static string). */
const char *stst_last_cuda_error(void);
int stst_tile_info(stst_handle h, int dir, int *cols_per_cta, int *rows_per_cta, double *us);

/*
 * stst_profile: enable (1) or disable (0) per-kernel timing for the handle's
 * calls. Enabling clears previous records. While enabled every kernel launch
 * of a call is bracketed by CUDA events on the handle's stream and the call
 * synchronizes on return; stst_pcg_solve then runs its loop as plain launches
 * with one host check per iteration instead of the CUDA graph.
 * stst_profile_read: record idx (0-based) -> kernel name (NUL-terminated, at
 * most name_len bytes), kernel launch count and total device milliseconds (a
 * record may time a short run of kernels as one: the count is of kernels, the
 * time of the run). Returns STST_ERR_ARG past the last record. Host outputs.
 */
int stst_profile(stst_handle h, int enable);

/*
 * stst_plan_info: the sum-factorised mat-vec chosen for this handle.
 * n_passes (host, may be NULL): kernel launches per stst_apply_sys.
 * band_apps (host, may be NULL): banded 1D applications per unknown (each is
 * 2p+1 complex-by-real multiply-adds, 4(2p+1) flops).
 * flops_per_dof (host, may be NULL): the algorithmic flops of one apply_sys per unknown.
 */
int stst_plan_info(stst_handle h, int *n_passes, int *band_apps, double *flops_per_dof);

/*
 * stst_pcg_graph_info: the CUDA graph that runs the PCG loop of stst_pcg_solve (Sec. 6 solves
 * with P-hat, Algorithm 1, as the preconditioner): a device-side WHILE node whose body holds
 * iterations_per_body iterations of the loop in kernels_per_body kernel nodes (host outputs, may be
 * NULL). A solve that takes k iterations launches ceil(k / iterations_per_body) bodies; every
 * kernel of a body launched after convergence returns at once. STST_ERR_STATE before the first
 * unprofiled stst_pcg_solve on the handle (the graph is built then).
 */
int stst_pcg_graph_info(stst_handle h, int *kernels_per_body, int *iterations_per_body);
int stst_profile_read(stst_handle h, int idx, char *name, int name_len, long long *count, double *total_ms);

/* ======================================================================================
 * Learned warm start. The paper has no learned component: these calls are an extension.
 * A network maps a problem's data parameters to coordinates c in a basis Q of the solution
 * space; x0 = Q^T c starts PCG (stst_pcg_solve_guarded), which stays the arbiter of the result.
 * All arrays are device memory owned by the caller unless stated; calls are ordered on the
 * given stream (the network's own stream for stst_ws_*).
 * ====================================================================================== */

/*
 * stst_ws_create: a fully connected network sizes[0] -> sizes[1] -> ... -> sizes[n_layers]
 * (1 <= n_layers <= 8) with tanh after every layer but the last. Parameters are packed layer by
 * layer: W_l (sizes[l+1] x sizes[l], row-major) then b_l (sizes[l+1]). Weights are kept as an
 * FP32 master copy (with the Adam moments) and as a BF16 copy that every product reads; biases
 * are read in FP32; products accumulate in FP32. Weights start as N(0, 1/sizes[l]) drawn from a
 * counter-based generator seeded by `seed`, biases at 0. max_batch bounds the batch of every
 * later call. stream: the stream of every later call on this network (NULL: the legacy default
 * stream). Allocates all workspace here.
 * Errors: STST_ERR_ARG for bad sizes, STST_ERR_OOM.
 */
typedef struct stst_ws_s *stst_ws;
int stst_ws_create(stst_ws *w, int n_layers, const int *sizes, int max_batch, unsigned long long seed,
                   void *stream);
int stst_ws_destroy(stst_ws w);
/* number of parameters (host output) */
int stst_ws_num_params(stst_ws w, long long *n);
/* the effective parameters (weights as the BF16 copy widened to FP32, biases FP32) -> params
 * (device, n floats); synchronizes. stst_ws_set_params: params (device) become the master copy,
 * the BF16 copy is rounded from it, the Adam state is reset; synchronizes. */
int stst_ws_get_params(stst_ws w, float *params);
int stst_ws_set_params(stst_ws w, const float *params);
/* Y (batch x sizes[n_layers], row-major) = s (.) network(X) + beta Y for X (batch x sizes[0], row-major),
 * s the output scale (all ones unless set); beta = 0 does not read Y. 1 <= batch <= max_batch; batches of
 * at most 8 rows run one warp per weight row. Stream-ordered, no synchronization. */
int stst_ws_forward(stst_ws w, const float *X, int batch, float *Y, float beta);
/* Per-output scale s used by stst_ws_forward only (training sees the unscaled outputs); scale: sizes[n_layers]
 * floats (host or device), NULL removes it. Synchronizes. */
int stst_ws_set_output_scale(stst_ws w, const float *scale);
/*
 * Loss L = (1/batch) sum_n w_n ||network(X_n) - T_n||^2 over the batch and its gradient with
 * respect to the effective parameters (backpropagation through the BF16 weights).
 * X: rows x sizes[0], T: rows x sizes[n_layers] (row-major), weight: per-row w_n (NULL: all 1).
 * idx (device int array of length batch, may be NULL): the batch is rows idx[0..batch-1] of X, T
 * and weight; NULL: the first batch rows. grad (device, n_params floats, may be NULL) receives the
 * gradient; loss (host, may be NULL) receives L, and when given the call synchronizes.
 */
int stst_ws_grad(stst_ws w, const float *X, const float *T, const float *weight, const int *idx, int batch,
                 float *grad, double *loss);
/* The same loss and gradient, then one Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected,
 * learning rate lr) on the master copy and a fresh BF16 copy. */
int stst_ws_train_step(stst_ws w, const float *X, const float *T, const float *weight, const int *idx, int batch,
                       float lr, double *loss);

/*
 * stst_pod_basis: rows of Q (K x m, row-major, FP32) = an orthonormal basis of the dominant row
 * space of the snapshot matrix Y (n x m, row-major, FP64; each row one solution viewed as m reals,
 * e.g. m = 2 N_dof for complex128 vectors). Randomized subspace iteration (Halko, Martinsson and
 * Tropp 2011, Alg. 4.4): Q = orth(Omega^T Y), then power_its times Q = orth((Q Y^T) Y) with the
 * intermediate orthonormalized too. orth = CholeskyQR2 with the Gram matrices accumulated in FP64.
 * Omega (n x K, row-major, FP32) is the caller's Gaussian test matrix. Requires 1 <= K <= min(n, m),
 * K <= 4096, m < 2^31, 0 <= power_its <= 8. Allocates stream-ordered temporaries ((K + 2 K) x max
 * of m, n floats and (slices + 2) K^2 doubles) and synchronizes. STST_NOT_HPD when a Gram matrix
 * is numerically singular (the snapshots span fewer than K directions).
 */
int stst_pod_basis(const double *Y, int n, long long m, const float *Omega, int K, int power_its, float *Q,
                   void *stream);
/* C (n x K, row-major, FP32) = Y Q^T: coordinates of the snapshot rows in the basis. Products in FP32,
 * sums in FP32 over at most 32 terms and then in FP64. Stream-ordered, no allocation. */
int stst_pod_project(const double *Y, int n, long long m, const float *Q, int K, float *C, void *stream);
/* X (n x m, row-major, FP64) = alpha C Q + beta X (C: n x K row-major FP32; beta = 0 does not read X),
 * accumulated like stst_pod_project. When phase (device, n doubles) is given, m must be even and row r
 * (m/2 complex values) is then multiplied by e^{i phase[r]}. Stream-ordered, no allocation. */
int stst_pod_expand(const float *Q, int K, long long m, const float *C, int n, float alpha, float beta,
                    const double *phase, double *X, void *stream);

/*
 * Training-data preparation of the warm start (the arithmetic between the snapshot basis and the network):
 * stst_ws_whiten: Cholesky whitening of features F (n x K row-major FP32, e.g. coordinates of the initial
 * data in an input basis): G = F^T F / n accumulated in FP64, plus 1e-10 of its largest diagonal entry,
 * G = R^T R (R upper triangular), W = R^{-1}; Fw = F W (n x K, so that the features have the identity as
 * their training covariance: W^T G W = I), and when Q is given (K x m row-major FP32, the rows of the input
 * basis), Q <- W^T Q in place, so that projecting a new datum on Q gives its whitened features directly.
 * Allocates stream-ordered temporaries and synchronizes; STST_NOT_HPD when a Cholesky pivot collapses
 * (features that are linearly dependent beyond the shift).
 * stst_ws_target_scale: for targets T (n x K row-major FP32): so[k] = max(sqrt(mean_n T[n][k]^2), 1e-300)
 * (FP64, the RMS of every output coordinate), Ts = T / so column by column (FP32), and per-sample weights
 * w[n] = mean_r ||T_r||^2 / max(||T_n||^2, 1e-300) (FP32: the loss then weighs relative errors).
 * stst_ws_cascade: the training targets of one stage of the cascade (resid n x K FP64, kept across calls):
 * with T0 (the first stage): resid = T0, scale = 1; otherwise resid -= Y (.) scale_prev column by column
 * (Y: the previous stage's outputs on every training row, n x K FP32) and scale[k] = max(sqrt(mean_n
 * resid[n][k]^2), 1e-30). Then targets = resid / scale (FP32) and out_scale = so (.) scale (FP32, the
 * stage's output scale for stst_ws_set_output_scale). scale, scale_prev, so: K doubles.
 * All arrays are device memory; stream-ordered (stst_ws_whiten synchronizes).
 */
int stst_ws_whiten(const float *F, int n, int K, float *Fw, float *Q, long long m, void *stream);
int stst_ws_target_scale(const float *T, int n, int K, float *Ts, double *so, float *w, void *stream);
int stst_ws_cascade(const float *T0, const float *Y, const double *scale_prev, double *resid, int n, int K,
                    double *scale, float *targets, const double *so, float *out_scale, void *stream);

/*
 * stst_pcg_solve_guarded: stst_pcg_solve from the initial guess in x, after a device-side check:
 * if ||rhs - A x|| >= ||rhs|| or is not finite, x is set to 0 first (the cold start of Sec. 6).
 * used_warm (host, may be NULL) = 1 when the given guess was kept. Same outputs and errors as
 * stst_pcg_solve.
 */
int stst_pcg_solve_guarded(stst_handle h, const double *rhs, double *x, double tol, int maxit, int *iters,
                           double *relres, int *used_warm);

#ifdef __cplusplus
}
#endif

#endif /* STST_H */
