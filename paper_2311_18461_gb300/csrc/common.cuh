// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <vector>
#include "../../include/stst.h"
#include "prof.cuh"

#define STST_MAXD 3
#define STST_MAXP 8
#define STST_MAXN_SPACE 128
#define STST_MAXPART 65536  // per-CTA partial sums per component (the grids of the reducing kernels stay below)

// ---- error handling -------------------------------------------------------------------------
#define STST_CUDA(call)                                   \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) { stst_last_cuda = e_; return STST_ERR_CUDA; } \
  } while (0)
#define STST_TRY(call)                  \
  do {                                  \
    int s_ = (call);                    \
    if (s_ != STST_OK) return s_;       \
  } while (0)

extern thread_local cudaError_t stst_last_cuda;

// ---- matrix kinds assembled on the device (band storage n x (2p+1), row-major) ----------------
enum MatKind { MK_M = 0, MK_L = 1, MK_J = 2, MK_K = 3, MK_K2 = 4, MK_KA = 5, MK_K2S = 6 };
// MK_KA = K - K^T (time advection, W + W^* = i KA); MK_K2S = K2 + K2^T.

struct DirInfo {
  int p, n_el, nq, m, n;  // degree, elements, quad points / element, full size, reduced size
  double len;              // T for time, 1 for space
  int off;                 // first kept full index (1 for time and space)
  int Q() const { return n_el * nq; }
};

struct BandMat {
  double *d = nullptr;  // n x (2p+1)
  int n = 0, p = 0;
};

// ---- sum-factorised mat-vec plan --------------------------------------------------------------
#define PASS_MAXIN 24
#define PASS_MAXAPP 48
#define PASS_MAXOUT 24

struct PassParams {
  int mode;                  // 0 = time, l >= 1 spatial direction
  int p;                     // half bandwidth of this mode's matrices
  int n_in, n_app, n_out;
  int n_mode_out, n_mode_in, row_off;  // output / input extent along the mode; input index = j + row_off - p + k
  long long inner, outer;    // tensor = (outer, n_mode, inner) complex elements
  const void *in[PASS_MAXIN];
  void *out[PASS_MAXOUT];
  const double *mat[PASS_MAXAPP];    // FP64 band matrices (n_mode_out rows x (2p+1))
  const float *mat32[PASS_MAXAPP];   // FP32 copies
  int app_in[PASS_MAXAPP];
  int app_imag[PASS_MAXAPP];         // multiply by i
  float coef32[PASS_MAXAPP][PASS_MAXOUT];
  double coef[PASS_MAXAPP][PASS_MAXOUT];
  // coef * mat, prepared by the planner, so that kernels accumulate band sums without a multiply
  const double *cmat[PASS_MAXAPP][PASS_MAXOUT];
  const float *cmat32[PASS_MAXAPP][PASS_MAXOUT];
  // epilogue (final pass only, n_out == 1)
  int epi;                    // 0 store, 1 out = b - v
  const void *b;
  const void *dotvec;         // if non-null: partial sums of Re(conj(dotvec) . out) per CTA
  double *dot_partials;
  const void *dot2vec;        // second partial: ||out||^2 when dot2vec == out sentinel (see kernel)
  double *dot2_partials;
  const int *done;            // if non-null and *done: skip
};

struct GeoOp;  // the mapped-domain operator (geometry.cu)

struct Plan {
  std::vector<PassParams> passes;
  int n_levels = 0;
  const GeoOp *geo = nullptr;  // set: run_plan applies the mapped-domain operator instead of the passes
  // one launch for all levels with grid barriers between them (k_pass_fused): allowed (the handle is not
  // in a batch, whose branches run concurrently), the barrier state (count, generation) and its error flag
  int fuse = 0;
  unsigned *gbar = nullptr;
  int *gerr = nullptr;
};

// ---- inner products in the epilogue of a preconditioner application -------------------------------
// The last kernel of s = P^{-1} r sums, per output element v = s[idx] (complex), the products the CG
// update needs next, so no kernel reads s again for them:
//   component 0: Re sum conj(a) v                (a = r: <r, s> of the plain CG, real for Hermitian P)
//   component 1: Im sum conj(a) v                (cplx: the complex <s, r>)
//   components 2, 3: Re, Im sum conj(b) v        (cplx with b: <s, b>, b = A p for the flexible CG)
// a and b have the output's type (double2 or float2). A CTA writes component c of its sums to
// part[c * STST_MAXPART + slot]; the slot is the CTA's index in its grid.
struct EpiDot {
  const void *a = nullptr, *b = nullptr;
  double *part = nullptr;
  int cplx = 0;
  __host__ __device__ int ncomp() const { return !part ? 0 : (!cplx ? 1 : (b ? 4 : 2)); }
};

template <typename TO>
__device__ __forceinline__ void epi_dot_acc(double (&acc)[4], const EpiDot &ed, long long idx, double vx, double vy) {
  // chains of fused multiply-adds (two FP64 operations per term, not a product, a fused product and a sum)
  const TO av = ((const TO *)ed.a)[idx];
  const double ax = av.x, ay = av.y;
  acc[0] = __fma_rn(ax, vx, __fma_rn(ay, vy, acc[0]));
  if (ed.cplx) {
    acc[1] = __fma_rn(ax, vy, __fma_rn(-ay, vx, acc[1]));
    if (ed.b) {
      const TO bv = ((const TO *)ed.b)[idx];
      const double bx = bv.x, by = bv.y;
      acc[2] = __fma_rn(bx, vx, __fma_rn(by, vy, acc[2]));
      acc[3] = __fma_rn(bx, vy, __fma_rn(-by, vx, acc[3]));
    }
  }
}

// Deterministic sum over the CTA (blockDim.x a multiple of 32, <= 1024); valid in thread 0.
__device__ __forceinline__ double epi_block_sum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;
}

// Every thread of the CTA calls this (it synchronizes); sh holds 32 doubles.
__device__ __forceinline__ void epi_dot_store(const double (&acc)[4], const EpiDot &ed, long long slot, double *sh) {
  const int nc = ed.ncomp();
  for (int c = 0; c < nc; ++c) {
    const double t = epi_block_sum(acc[c], sh);
    if (threadIdx.x == 0) ed.part[(long long)c * STST_MAXPART + slot] = t;
  }
}

// ---- PCG control block (device) ---------------------------------------------------------------
// Tile of the SIMT mode product: cpt columns per thread (8 cpt per CTA), rpt groups of 32 output rows;
// tc = 1: the TF32 tensor-core kernel instead, where the shape and the input allow it (FP32 preconditioner).
struct MpCfg {
  int cpt, rpt;
  int tc;
};

// Plain CG (FP64 preconditioner): rho = <r, z> real, alpha = rho / pq, beta = rho_new / rho.
// Flexible CG (low-precision preconditioners, flexible = 1): complex alpha = sigma / pq with
// sigma = <r, p>, complex beta = -<z, A p> / pq (directions A-orthogonalized), sigma_new = <r, z> +
// conj(beta) <r, p_old>.
struct PcgCtl {
  double ff, rr, rho, pq, alpha, beta, tol2;
  double sig_re, sig_im, alpha_im, beta_im;
  int it, maxit, done, status;
  int flexible;
  int x0_zero;  // 1 until a nonzero entry of the initial guess is seen (the host and the batch set it to 1)
};

// Slots of the handle's partial-sum buffer (units of STST_MAXPART doubles): the preconditioner's epilogue
// components (EpiDot, up to 4), ||r||^2, <r_new, p> (flexible CG: real and imaginary part, two halves
// used by alternate iterations; ||f||^2 at the start), <p, A p>.
enum { PS_Z = 0, PS_RR = 4, PS_RP = 5, PS_PQ = 9, PS_COUNT = 10 };

// ---- handle -------------------------------------------------------------------------------------
struct stst_problem {
  int magic;
  int d;
  DirInfo dir[STST_MAXD + 1];
  double T, nu;
  int prec_mode;
  int formulation;                 // STST_FORM_LS (least squares) or STST_FORM_UW (ultraweak)
  cudaStream_t stream;
  int own_stream;                  // stream created by the handle (caller passed NULL)
  long long N_s, N_dof;
  int n_t() const { return dir[0].n; }

  // 1D matrices: per direction, list indexed by matrix id (0 M, 1 L, 2 J, then weighted ones)
  std::vector<BandMat> mats[STST_MAXD + 1];
  std::vector<float *> mats32[STST_MAXD + 1];
  // time: KA = K - K^T (id 2 in mats[0]: 0 L? see capi: time ids 0 L, 1 M, 2 KA)
  BandMat tfull[3];  // full-basis time L, M, KA (rows 1..p of the full matrices used by the lifting)
  float *tfull32[3];
  // quadrature and basis tables per direction
  double *qpts[STST_MAXD + 1];
  double *qwts[STST_MAXD + 1];
  double *tab[STST_MAXD + 1];     // Q x (p+1) x 3 : value, d1, d2 of functions e..e+p (full index) at each point
  double *mchol[STST_MAXD + 1];   // banded Cholesky of the reduced mass, n x (p+1)

  // potential
  int pot_rank;
  // potential-aware preconditioner: G_l = nu L_l + M_{v_l} (band ids in mats[l]), recorded by
  // stst_set_potential for sums of one-direction factors; prec_op 1 builds the FD from them
  int g_valid;
  int g_mat[STST_MAXD + 1];
  int g_share[STST_MAXD + 1];  // direction whose eigendecomposition of (G_l, M_l) this one reuses (itself if none)
  int prec_op;
  std::vector<double *> pot_bufs;  // device buffers of weights (owned)

  // FD
  int fd_ready;
  MpCfg mp_cfg[STST_MAXD + 1];     // mode-product tile per direction (autotuned or default)
  float mp_us[STST_MAXD + 1];      // its measured time per launch (0: not measured)
  int tuned;
  int fd2d;                        // CTAs per slab of the fused transforms (FP32 preconditioner, d = 2 or 3), 0: separate
  int fd2d_b;                      // CTAs per slab of the fused backward transform (timed apart from the forward one)
  int eig_src[STST_MAXD + 1];
  double *U[STST_MAXD + 1];
  float *U32[STST_MAXD + 1];
  __nv_bfloat16 *Ubf[STST_MAXD + 1];
  float *Utf[STST_MAXD + 1];       // TF32 planes of U' (FP32 preconditioner): [fwd hi | bwd hi | fwd lo | bwd lo]
  double *lam[STST_MAXD + 1];
  double *oa_work;                 // refinement workspace
  void *Hg;                        // FP64 factors: n_t x p x N_s complex
  double *Hd;                      // FP64 inverse diagonals n_t x N_s
  void *Hg32;                      // FP32 factors
  float *Hd32;
  void *Gp32;                      // FP32 factors in the pencil order (pencil kernel), or null
  float *Dp32;
  int pencil;                      // CTAs per pencil of the pencil kernel (FP32 preconditioner), 0: not used
  // parallel-in-time time solves, [0] FP32 factors, [1] FP64 factors: segments, segment length,
  // forward / backward transfer matrices, and whether the segmented kernel is used
  int ts_S[2], ts_L[2], ts_seg[2];
  void *Tf[2], *Tb[2];
  int *flags;                      // device status flags: [0] factorization pivots, [1] bounded waits
  int *flags_host;                 // pinned copy

  // plans
  Plan sys_plan, lift_plan;
  GeoOp *geo;                      // mapped-domain operator (stst_set_geometry), or null: the parametric one
  unsigned *gbar;                  // grid-barrier state of the fused mat-vec: arrival count, generation
  int no_fuse;                     // set by stst_batch_create: the handle's kernels may run concurrently
  std::vector<void *> pool;        // intermediate tensors of the plans (FP64 sized)
  std::vector<void *> scaled;      // coefficient-scaled band matrices of the plans

  // workspaces (N_dof complex FP64 each)
  double *w_x, *w_r, *w_z, *w_zold, *w_p, *w_q, *w_f, *w_t1, *w_t2;
  float *v_d, *v_r, *v_z, *v_p, *v_q;  // FP32 inner-solver vectors (N_dof complex each)
  PcgCtl *ctl2;                        // inner-solver control block
  double *partials;                // 4 x MAXPART
  PcgCtl *ctl;
  PcgCtl *ctl_host;                // pinned
  double *proj_work;               // rhs / projection workspace
  size_t proj_work_bytes;

  // PCG graph
  cudaGraphExec_t pcg_exec;
  int pcg_graph_valid;
  int pcg_body_kernels;  // kernel nodes in the WHILE node's body (two iterations)
  int pcg_graph_flexible;
  cudaGraphExec_t ir_exec;
  int ir_graph_valid;

  // tracing
  int prof_on;
  Profiler *prof;
};

// Installs the handle's profiler for the duration of an API call and flushes it on exit.
struct ApiScope {
  stst_problem *h;
  explicit ApiScope(stst_problem *hh) : h(hh) { g_prof = (h && h->prof_on) ? h->prof : nullptr; }
  ~ApiScope() {
    // records are resolved lazily (stst_profile_read) so that queued calls are not serialized
    if (g_prof && g_prof->pending.size() > 4096) prof_flush(g_prof);
    g_prof = nullptr;
  }
};

#define STST_MAGIC 0x57575354

// ---- kernels / launchers (defined in the .cu files) ------------------------------------------
int launch_assemble_band(int kind, int p, int n_el, double len, int nq, int off, int n_rows, int n_cols,
                         const double *weight, double *out, cudaStream_t s);
int launch_quadrature(int p, int n_el, double len, int nq, double *pts, double *wts, double *tab, cudaStream_t s);
int launch_mass_cholesky(const BandMat &M, double *chol, int *flags, cudaStream_t s);
int launch_to_f32(const double *src, float *dst, long long n, cudaStream_t s);
int launch_weight_product(const double *a, const double *b, double *out, int n, cudaStream_t s);
int launch_scale(const double *a, double c, double *out, float *out32, int n, cudaStream_t s);
int launch_band_axpby(const double *a, double ca, const double *b, double cb, double *out, float *out32, int n,
                      cudaStream_t s);

int run_plan(const Plan &plan, const void *x, void *y, int precision, int epi, const void *b, const void *dotvec,
             double *dot_partials, const int *done, cudaStream_t s, const void *dot2vec = nullptr,
             double *dot2_partials = nullptr);
int fd_setup(stst_problem *h);
int fd_setup_launch(stst_problem *h);
int pcg_init(stst_problem *h);
int pcg_body(stst_problem *h, cudaGraphConditionalHandle cond, int use_cond);
int reduction_grid(long long total);
// ed: inner products of the output taken by the last kernel (EpiDot); its vectors are FP64 (double2)
// when the output is FP64, FP32 (float2) when out32 is given.
int fd_apply(stst_problem *h, const double *r, double *s, int precision, const EpiDot &ed, const int *done,
             void *f32_scratch_a, void *f32_scratch_b, float *out32 = nullptr, const float *in32 = nullptr);
int rhs_compute(stst_problem *h, const double *f_qp, const double *u0_qp, double *rhs, double *c0);
int rhs_lift_compute(stst_problem *h, const double *f_qp, const double *u_qp, double *rhs, double *xd);

int pcg_run(stst_problem *h, const double *rhs, double *x, double tol, int maxit, int *iters, double *relres);
int ir_run(stst_problem *h, const double *rhs, double *x, double tol, int maxit, double inner_tol,
           int inner_maxit, int *iters, int *outer, double *relres);

int grid_for(long long n, int block);
int fd_partials_count(stst_problem *h);
void ts_segments(int nt, int P, size_t rsize, int *S, int *L);
template <typename R>
int launch_time_transfer(const void *G, const R *D, int nt, long long Ns, int P, int S, int L, void *Tf, void *Tb,
                         cudaStream_t s);
// Opts kernel `kern` into `bytes` of dynamic shared memory (with its static shared memory the default
// limit is 48 KB in total); remembers the largest size set per kernel, so repeated launches skip the call.
int ensure_dyn_smem(const void *kern, size_t bytes);
MpCfg modeprod_default(int n);
int tune_modeprod(stst_problem *h);  // times the mode-product tiles once per shape (outside graph capture)
extern int g_fused_matvec;  // 0: one launch per mat-vec level (default), 1: all levels in one launch
extern int g_tune_enabled;
extern int g_ts_mode;
extern int g_fd2d_mode;
bool fd2d_fits(const stst_problem *h);

// tensor-core mode products (modeprod_tc.cu)
int launch_u_to_bf16(const double *U, int n, __nv_bfloat16 *out, cudaStream_t s);
template <typename TI, typename TO>
int launch_modeprod_tc(const TI *X, TO *Y, const __nv_bfloat16 *Bk, long long lo_stride, int split, int n,
                       long long inner, long long outer, const EpiDot &ed, const int *done, int *errflag,
                       cudaStream_t s);
int tc_partials_count(long long ncols);

// mapped-domain operator (geometry.cu)
int run_geo(const GeoOp &g, const void *x, void *y, int precision, int epi, const void *b, const void *dotvec,
            double *dot_partials, const int *done, cudaStream_t s, double *dot2_partials);
void free_geo(GeoOp *g);
double geo_prec_scale(const GeoOp *g, int l);  // P-hat's eigenvalue scale of direction l (1 without a geometry)
int launch_scale_vec(double *a, double c, long long n, cudaStream_t s);  // a *= c in place

// TF32 tensor-core mode products fed by TMA (modeprod_tf32.cu)
int launch_u_to_tf32(const double *U, int n, float *out, cudaStream_t s);
size_t tf32_planes_floats(int n);
bool tf32_eligible(int n, long long inner, long long outer, const void *X);
template <typename TO>
int launch_modeprod_tf32(const float2 *X, TO *Y, const float *planes, int backward, int n, long long inner,
                         long long outer, const EpiDot &ed, const int *done, int *errflag, cudaStream_t s);
int tf32_partials_count(int n, long long inner, long long outer);

// pencil kernel (pencil.cu): steps 2-4 of Algorithm 1 along the last spatial direction with the time solves
bool pencil_fits(const stst_problem *h, int CL);
size_t pencil_smem(int n, int nt, int P, int CL);
int launch_factor_pencil(stst_problem *h, cudaStream_t s);
template <typename TI, typename TO>
int launch_pencil(const TI *X, TO *Y, const stst_problem *h, int CL, const EpiDot &ed, const int *done,
                  cudaStream_t s);
extern int g_pencil_mode;
inline int pad16(int n) { return (n + 15) / 16 * 16; }
