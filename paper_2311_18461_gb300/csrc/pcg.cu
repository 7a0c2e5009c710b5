// Preconditioned conjugate gradients for the HPD system A u = f (Sec. 5.3, Sec. 6), and a mixed
// precision iterative-refinement driver around an FP32 inner PCG.
//
// Inner products <a, b> = b^H a; all reductions are deterministic (per-CTA partials reduced in a
// fixed order by one CTA). The iteration runs as one CUDA graph: an init segment, then a
// conditional WHILE node whose body is one iteration. A one-CTA control kernel in the body
// increments the iteration counter, decides convergence / maxit / breakdown and sets the graph
// condition, so the loop always ends after at most maxit bodies and the host waits once.
#include "common.cuh"

int fd_partials_count(stst_problem *h);

__device__ __forceinline__ double block_sum_d(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    int nw = blockDim.x >> 5;
    t = (l < nw) ? sh[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;
}

// sum of nparts partials by one CTA (fixed order => deterministic)
__device__ double reduce_partials(const double *part, int nparts, double *sh) {
  double v = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) v += part[i];
  double t = block_sum_d(v, sh);
  __shared__ double bc;
  if (threadIdx.x == 0) bc = t;
  __syncthreads();
  double r = bc;
  __syncthreads();
  return r;
}

// Reductions for the FP64-poor GB300 (2 FP64 FMA per clock per SM): a butterfly shuffle tree makes all
// 32 lanes of every warp do every addition, so sums that every CTA of a 304-CTA kernel repeats cost as
// much FP64 issue as the vector arithmetic itself. Here warp c alone sums component c (NC <= number of
// warps); the other warps only load and store. The order of the additions is fixed: deterministic.

// NC sums over the CTA of one value per thread, valid in every thread on return. sh: at least
// NC * blockDim.x + NC doubles (checked against 256 threads at compile time; the callers run 256).
template <int NC, int SZ>
__device__ __forceinline__ void block_sum_all(double (&v)[NC], double (&sh)[SZ]) {
  static_assert(SZ >= NC * 256 + NC, "block_sum_all: shared buffer too small for 256 threads");
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nt = blockDim.x;
  __syncthreads();  // sh may still be read by an earlier reduction
#pragma unroll
  for (int c = 0; c < NC; ++c) sh[c * nt + threadIdx.x] = v[c];
  __syncthreads();
  if (w < NC) {
    double t = 0.0;
    for (int i = l; i < nt; i += 32) t += sh[w * nt + i];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (l == 0) sh[NC * nt + w] = t;
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < NC; ++c) v[c] = sh[NC * nt + c];
}

// The sums of NC sets of per-CTA partials (set c: part[c][0 .. n[c])), warp c summing set c; valid in
// every thread on return. sh: at least 33 doubles.
template <int NC, int SZ>
__device__ __forceinline__ void reduce_partials_all(const double *const (&part)[NC], const int (&n)[NC],
                                                    double (&out)[NC], double (&sh)[SZ]) {
  static_assert(SZ >= 33 && NC <= 8, "reduce_partials_all: shared buffer too small or too many sets");
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();  // sh may still be read by an earlier reduction
  if (w < NC) {
    const double *pc = part[0];
    int nc = n[0];
#pragma unroll
    for (int c = 1; c < NC; ++c)
      if (w == c) {
        pc = part[c];
        nc = n[c];
      }
    double t = 0.0;
#pragma unroll 4
    for (int i = l; i < nc; i += 32) t += pc[i];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (l == 0) sh[w] = t;
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < NC; ++c) out[c] = sh[c];
}

template <typename T>
__global__ void k_norm2(const T *__restrict__ v, long long n, double *part) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    T a = v[i];
    acc += (double)a.x * a.x + (double)a.y * a.y;
  }
  double s = block_sum_d(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// init: ff, rr and rho (plain) or sigma = <r, p> = <r, z> (flexible) from partials; done if converged.
// The preconditioner's epilogue summed conj(r) z, i.e. conj(<r, z>) (component 1: its imaginary part).
__global__ void k_pcg_init(PcgCtl *ctl, const double *pf, int nf, const double *pr, int nr, const double *pz, int nz) {
  __shared__ double sh[32];
  const int flexible = ctl->flexible;
  const double ff = reduce_partials(pf, nf, sh);
  const double rr = reduce_partials(pr, nr, sh);
  const double rz = reduce_partials(pz, nz, sh);
  const double rz_im = flexible ? -reduce_partials(pz + STST_MAXPART, nz, sh) : 0.0;
  if (threadIdx.x == 0) {
    ctl->ff = ff;
    ctl->rr = rr;
    ctl->rho = rz;
    ctl->sig_re = rz;
    ctl->sig_im = rz_im;
    ctl->it = 0;
    ctl->status = STST_OK;
    ctl->done = (ff == 0.0 || rr <= ctl->tol2 * ff) ? 1 : 0;
    if (!ctl->done && !(rz > 0.0 && isfinite(rz) && isfinite(rz_im))) { ctl->done = 1; ctl->status = STST_BREAKDOWN; }
  }
}

template <typename T>
__global__ void k_copy_vec(const T *__restrict__ a, T *__restrict__ b, long long n, const int *done) {
  if (done && *done) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = a[i];
}

// Vector updates: UPT elements per thread per pass (indices i0 + 256 u). The first pass's operands
// are loaded before the scalar reductions, so the latency of the vector loads overlaps that of the
// partial sums. Every CTA reduces the same partials, so the grid stays at two CTAs per SM: measured
// on the 2D p = 3 64^2 x 64 solve, one pass over the vector with 545 CTAs cost 10 us more per
// iteration than 304 CTAs looping twice.
#define UPT 2
int update_grid(long long n) {
  long long g = (n + 256 * UPT - 1) / (256 * UPT);
  if (g > 2 * 152) g = 2 * 152;
  return g < 1 ? 1 : (int)g;
}

// pq = <p, q> with q = A p (every CTA reduces the same partials in the same order; CTA 0 records it).
// Plain (FLEX false): alpha = rho / pq, rho = <r, z> reduced from the latest preconditioner application
// (pz, component 0). Flexible: alpha = sigma / pq, complex, sigma = <r, p>; at the first iteration the
// start kernel recorded it, afterwards sigma = <r, z> + conj(beta) <r, p_old> from the preconditioner's
// epilogue (pz components 0, 1: conj(<r, z>)), this kernel's previous partials of <r, p_old> (prp) and
// the beta recorded by k_update_p. Then x += alpha p, r -= alpha q, partials of ||r||^2 (prr) and,
// flexible, of conj(p) r_new = <r_new, p>. No CTA of this kernel reads a scalar or partial that another
// CTA of it writes: the <r, p_old> partials are double-buffered by iteration parity (iteration k writes
// half k & 1 of prp and reads the other half, written by iteration k - 1).
__device__ __forceinline__ double dfma(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T, bool FLEX>
__global__ void __launch_bounds__(256) k_update_xr(T *__restrict__ x, T *__restrict__ r, const T *__restrict__ p,
                                                   const T *__restrict__ q, PcgCtl *ctl, long long n, double *prr,
                                                   double *prp, int nrp, const double *ppq, int npq,
                                                   const double *pz, int nz) {
  if (ctl->done) return;
  __shared__ double sh[3 * 256 + 3];
  const long long stride = (long long)gridDim.x * 256 * UPT;
  long long i0 = (long long)blockIdx.x * 256 * UPT + threadIdx.x;
  T pv[UPT], qv[UPT], xv[UPT], rv[UPT];
  auto load = [&](long long base) {
#pragma unroll
    for (int u = 0; u < UPT; ++u) {
      const long long i = base + 256 * u;
      if (i < n) {
        pv[u] = p[i];
        qv[u] = q[i];
        xv[u] = x[i];
        rv[u] = r[i];
      }
    }
  };
  if (i0 < n) load(i0);
  double pq, num_re, num_im = 0.0;
  double *prp_out = prp;
  if constexpr (FLEX) {
    const int it = ctl->it;
    const double *prp_in = prp + ((it + 1) & 1) * 2 * STST_MAXPART;
    prp_out = prp + (it & 1) * 2 * STST_MAXPART;
    const double *sp[5] = {ppq, pz, pz + STST_MAXPART, prp_in, prp_in + STST_MAXPART};
    const int sn[5] = {npq, it ? nz : 0, it ? nz : 0, it ? nrp : 0, it ? nrp : 0};
    double v[5];
    reduce_partials_all(sp, sn, v, sh);
    pq = v[0];
    if (it == 0) {
      num_re = ctl->sig_re;
      num_im = ctl->sig_im;
    } else {
      // <r, z> = conj(e), e = (v[1], v[2]); conj(beta) tau = (b_re - i b_im)(t_re + i t_im)
      const double b_re = ctl->beta, b_im = ctl->beta_im;
      num_re = v[1] + (b_re * v[3] + b_im * v[4]);
      num_im = -v[2] + (b_re * v[4] - b_im * v[3]);
    }
  } else {
    const double *sp[2] = {ppq, pz};
    const int sn[2] = {npq, nz};
    double v[2];
    reduce_partials_all(sp, sn, v, sh);
    pq = v[0];
    num_re = v[1];
  }
  // alpha by thread 0 alone and broadcast: a division is a sequence of FP64 operations, and 256 threads of
  // every CTA repeating it cost FP64 issue comparable to a quarter of the vector arithmetic
  if (threadIdx.x == 0) {
    const bool bad = !(pq > 0.0) || !isfinite(pq) || !isfinite(num_re) || !isfinite(num_im);
    sh[8] = bad ? 0.0 : num_re / pq;
    sh[9] = bad ? 0.0 : num_im / pq;
    if (blockIdx.x == 0) {
      ctl->pq = pq;
      ctl->rho = num_re;
      ctl->sig_re = num_re;
      ctl->sig_im = num_im;
      ctl->alpha = sh[8];
      ctl->alpha_im = sh[9];
      if (bad) ctl->status = STST_BREAKDOWN;  // the check kernel ends the loop
    }
  }
  __syncthreads();
  const double a_re = sh[8], a_im = sh[9];
  double arr = 0.0, arp_re = 0.0, arp_im = 0.0;
  for (; i0 < n; i0 += stride) {
#pragma unroll
    for (int u = 0; u < UPT; ++u) {
      const long long i = i0 + 256 * u;
      if (i < n) {
        // chains of fused multiply-adds: two FP64 operations per real term instead of a product, a fused
        // product and an addition
        if constexpr (FLEX) {
          xv[u].x = dfma(a_re, pv[u].x, dfma(-a_im, pv[u].y, xv[u].x));
          xv[u].y = dfma(a_re, pv[u].y, dfma(a_im, pv[u].x, xv[u].y));
          rv[u].x = dfma(-a_re, qv[u].x, dfma(a_im, qv[u].y, rv[u].x));
          rv[u].y = dfma(-a_re, qv[u].y, dfma(-a_im, qv[u].x, rv[u].y));
        } else {
          xv[u].x += a_re * pv[u].x;
          xv[u].y += a_re * pv[u].y;
          rv[u].x -= a_re * qv[u].x;
          rv[u].y -= a_re * qv[u].y;
        }
        x[i] = xv[u];
        r[i] = rv[u];
        const double rx = rv[u].x, ry = rv[u].y;
        arr = dfma(rx, rx, dfma(ry, ry, arr));
        if constexpr (FLEX) {
          const double px = pv[u].x, py = pv[u].y;
          arp_re = dfma(px, rx, dfma(py, ry, arp_re));
          arp_im = dfma(px, ry, dfma(-py, rx, arp_im));
        }
      }
    }
    if (i0 + stride < n) load(i0 + stride);
  }
  if constexpr (FLEX) {
    double v[3] = {arr, arp_re, arp_im};
    block_sum_all(v, sh);
    if (threadIdx.x == 0) {
      prr[blockIdx.x] = v[0];
      prp_out[blockIdx.x] = v[1];
      prp_out[STST_MAXPART + blockIdx.x] = v[2];
    }
  } else {
    double v[1] = {arr};
    block_sum_all(v, sh);
    if (threadIdx.x == 0) prr[blockIdx.x] = v[0];
  }
}

// control: count the iteration, test ||r|| <= tol ||f||, maxit; set the WHILE condition.
__global__ void k_pcg_check(PcgCtl *ctl, const double *prr, int nrr, cudaGraphConditionalHandle cond, int use_cond) {
  __shared__ double sh[32];
  int was_done = ctl->done;
  double rr = reduce_partials(prr, nrr, sh);
  if (threadIdx.x == 0) {
    if (!was_done) {
      ctl->it += 1;
      ctl->rr = rr;
      if (ctl->status == STST_BREAKDOWN) {
        ctl->done = 1;
      } else if (!isfinite(rr)) {
        ctl->done = 1;
        ctl->status = STST_BREAKDOWN;
      } else if (rr <= ctl->tol2 * ctl->ff) {
        ctl->done = 1;
        ctl->status = STST_OK;
      } else if (ctl->it >= ctl->maxit) {
        ctl->done = 1;
        ctl->status = STST_NOT_CONVERGED;
      }
    }
    if (ctl->it >= ctl->maxit) ctl->done = 1;  // hard bound on the number of bodies
    if (use_cond) cudaGraphSetConditional(cond, ctl->done ? 0u : 1u);
  }
}

// p = z + beta p; CTA 0 records beta.
// Plain: beta = rho_new / rho (Fletcher-Reeves with the preconditioner), rho_new = <r, z> from the
// epilogue of the preconditioner application (component 0); rho was recorded by k_update_xr.
// Flexible: beta = -<z, q> / pq with q = A p_old (epilogue components 2, 3 hold sum conj(q) z = <z, q>),
// which makes the new direction A-orthogonal to the old one whatever the preconditioner did.
template <typename T, bool FLEX>
__global__ void __launch_bounds__(256) k_update_p(T *__restrict__ p, const T *__restrict__ z, PcgCtl *ctl, long long n,
                                                  const double *pz, int nz) {
  if (ctl->done) return;
  __shared__ double sh[33];
  const long long stride = (long long)gridDim.x * 256 * UPT;
  long long i0 = (long long)blockIdx.x * 256 * UPT + threadIdx.x;
  T pv[UPT], zv[UPT];
  auto load = [&](long long base) {
#pragma unroll
    for (int u = 0; u < UPT; ++u) {
      const long long i = base + 256 * u;
      if (i < n) {
        pv[u] = p[i];
        zv[u] = z[i];
      }
    }
  };
  if (i0 < n) load(i0);
  double b_re, b_im = 0.0;
  // beta by thread 0 alone and broadcast (one division per CTA, not per thread)
  if constexpr (FLEX) {
    const double *gp[2] = {pz + 2 * STST_MAXPART, pz + 3 * STST_MAXPART};
    const int gn[2] = {nz, nz};
    double g[2];
    reduce_partials_all(gp, gn, g, sh);
    if (threadIdx.x == 0) {
      const double pq = ctl->pq;
      b_re = -g[0] / pq;
      b_im = -g[1] / pq;
      const bool bad = !isfinite(b_re) || !isfinite(b_im);
      sh[8] = bad ? 0.0 : b_re;
      sh[9] = bad ? 0.0 : b_im;
      if (bad && blockIdx.x == 0) ctl->status = STST_BREAKDOWN;
    }
  } else {
    const double *rp[1] = {pz};
    const int rn[1] = {nz};
    double rv[1];
    reduce_partials_all(rp, rn, rv, sh);
    if (threadIdx.x == 0) {
      const double rho_old = ctl->rho, rho_new = rv[0];
      const bool bad = !(rho_new > 0.0) || !isfinite(rho_new);
      sh[8] = bad ? 0.0 : rho_new / rho_old;
      sh[9] = 0.0;
      if (bad && blockIdx.x == 0) ctl->status = STST_BREAKDOWN;
    }
  }
  __syncthreads();
  b_re = sh[8];
  b_im = sh[9];
  for (; i0 < n; i0 += stride) {
#pragma unroll
    for (int u = 0; u < UPT; ++u) {
      const long long i = i0 + 256 * u;
      if (i < n) {
        const double px = pv[u].x, py = pv[u].y;
        if constexpr (FLEX) {
          pv[u].x = dfma(b_re, px, dfma(-b_im, py, (double)zv[u].x));
          pv[u].y = dfma(b_re, py, dfma(b_im, px, (double)zv[u].y));
        } else {
          pv[u].x = dfma(b_re, px, (double)zv[u].x);
          pv[u].y = dfma(b_re, py, (double)zv[u].y);
        }
        p[i] = pv[u];
      }
    }
    if (i0 + stride < n) load(i0 + stride);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->beta = b_re;
    ctl->beta_im = b_im;
  }
}

// ------------------------------------------------------------------------------------------------
// FP64 PCG
// ------------------------------------------------------------------------------------------------
// The vectors of one PCG iteration: FP64 work vectors of the handle, or the FP32 ones of the inner solver.
template <typename T>
static int pcg_iteration(stst_problem *h, PcgCtl *ctl, T *x, T *r, T *z, T *p, T *q, int flexible, int fd_prec,
                         cudaGraphConditionalHandle cond, int use_cond) {
  cudaStream_t st = h->stream;
  const long long N = h->N_dof;
  const int g = reduction_grid(N), gu = update_grid(N);
  double *P = h->partials;
  double *pZ = P + PS_Z * STST_MAXPART, *pRR = P + PS_RR * STST_MAXPART, *pRP = P + PS_RP * STST_MAXPART,
         *pPQ = P + PS_PQ * STST_MAXPART;
  const int *done = &ctl->done;
  const int nz = fd_partials_count(h);
  const bool f32 = sizeof(T) == sizeof(float2);
  // q = A p, partials <p, q>
  STST_TRY(run_plan(h->sys_plan, p, q, f32 ? 1 : 0, 0, nullptr, p, pPQ, done, st));
  // alpha; x, r update (+ <r_new, p> for the flexible sigma)
  {
    STST_PROF("pcg_update_xr", st);
    if (flexible) k_update_xr<T, true><<<gu, 256, 0, st>>>(x, r, p, q, ctl, N, pRR, pRP, gu, pPQ, g, pZ, nz);
    else k_update_xr<T, false><<<gu, 256, 0, st>>>(x, r, p, q, ctl, N, pRR, pRP, gu, pPQ, g, pZ, nz);
  }
  // 1024 threads: each loads at most one of the (at most 2 x 152) partials, so the loads are one L2 round
  // trip; one warp looping over them measured slower (9.2 against 7.2 us per iteration on the 2D p = 3
  // 64^2 x 64 solve) despite its fewer FP64 additions
  { STST_PROF("pcg_scalar", st); k_pcg_check<<<1, 1024, 0, st>>>(ctl, pRR, gu, cond, use_cond); }
  // z = P^{-1} r with the epilogue's inner products: <r, z> (plain: real part; flexible: complex, and <z, q>)
  EpiDot ed;
  ed.a = r;
  ed.b = flexible ? q : nullptr;
  ed.part = pZ;
  ed.cplx = flexible;
  if (f32) STST_TRY(fd_apply(h, nullptr, nullptr, fd_prec, ed, done, h->w_t1, h->w_t2, (float *)z, (const float *)r));
  else STST_TRY(fd_apply(h, (const double *)r, (double *)z, fd_prec, ed, done, h->w_t1, h->w_t2));
  {
    STST_PROF("pcg_update_p", st);
    if (flexible) k_update_p<T, true><<<gu, 256, 0, st>>>(p, z, ctl, N, pZ, nz);
    else k_update_p<T, false><<<gu, 256, 0, st>>>(p, z, ctl, N, pZ, nz);
  }
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}

int pcg_body(stst_problem *h, cudaGraphConditionalHandle cond, int use_cond) {
  // STST_PREC_* equals fd_apply's precision code; the low-precision preconditioners run the flexible CG
  return pcg_iteration<double2>(h, h->ctl, (double2 *)h->w_x, (double2 *)h->w_r, (double2 *)h->w_z, (double2 *)h->w_p,
                                (double2 *)h->w_q, h->prec_mode != STST_PREC_FP64, h->prec_mode, cond, use_cond);
}

// Clears ctl->x0_zero if any entry of the initial guess is nonzero (benign race: every writer stores 0).
__global__ void k_x0_zero_check(const double2 *__restrict__ x, long long n, PcgCtl *ctl) {
  bool nz = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 v = x[i];
    nz = nz || v.x != 0.0 || v.y != 0.0;
  }
  if (__syncthreads_or(nz) && threadIdx.x == 0) ctl->x0_zero = 0;
}

// For a zero initial guess: r = f and the per-CTA partials of ||r||^2, in the launch shape and order of
// the residual mat-vec's final level (512 threads, the same grid), which is skipped then.
__global__ void __launch_bounds__(512) k_resid_from_zero(const PcgCtl *ctl, const double2 *__restrict__ f,
                                                         double2 *__restrict__ r, long long n, double *prr) {
  if (!ctl->x0_zero) return;
  __shared__ double sh[32];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 v = f[i];
    r[i] = v;
    acc += (double)v.x * v.x + (double)v.y * v.y;
  }
  const double s = block_sum_d(acc, sh);
  if (threadIdx.x == 0) prr[blockIdx.x] = s;
}

int pcg_init(stst_problem *h) {
  cudaStream_t st = h->stream;
  const long long N = h->N_dof;
  const int g = reduction_grid(N);
  const int prec = h->prec_mode;  // STST_PREC_* equals fd_apply's precision code
  double *P = h->partials;
  double *pZ = P + PS_Z * STST_MAXPART, *pRR = P + PS_RR * STST_MAXPART, *pF = P + PS_RP * STST_MAXPART;
  // r = f - A x, partials ||r||^2 ; ||f||^2. From x0 = 0 (the paper's start, Sec. 6) r = f needs no
  // mat-vec: a device check of x0 makes the residual's passes skip themselves and a copy takes over.
  { STST_PROF("pcg_init", st); k_x0_zero_check<<<g, 256, 0, st>>>((const double2 *)h->w_x, N, h->ctl); }
  STST_TRY(run_plan(h->sys_plan, h->w_x, h->w_r, 0, 1, h->w_f, nullptr, nullptr, &h->ctl->x0_zero, st, nullptr, pRR));
  {
    STST_PROF_N("pcg_init", st, 2);
    k_resid_from_zero<<<g, 512, 0, st>>>(h->ctl, (const double2 *)h->w_f, (double2 *)h->w_r, N, pRR);
    k_norm2<double2><<<g, 256, 0, st>>>((const double2 *)h->w_f, N, pF);
  }
  // z = P^{-1} r with <r, z> (complex for the flexible CG)
  EpiDot ed;
  ed.a = h->w_r;
  ed.part = pZ;
  ed.cplx = prec != STST_PREC_FP64;
  STST_TRY(fd_apply(h, h->w_r, h->w_z, prec, ed, nullptr, h->w_t1, h->w_t2));
  {
    STST_PROF_N("pcg_init", st, 2);
    k_pcg_init<<<1, 1024, 0, st>>>(h->ctl, pF, g, pRR, g, pZ, fd_partials_count(h));
    k_copy_vec<double2><<<g, 256, 0, st>>>((const double2 *)h->w_z, (double2 *)h->w_p, N, &h->ctl->done);
  }
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}

static int build_pcg_graph(stst_problem *h) {
  cudaStream_t st = h->stream;
  cudaGraph_t graph;
  STST_CUDA(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle cond;
  cudaError_t e = cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    stst_last_cuda = e;
    return STST_ERR_CUDA;
  }
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    stst_last_cuda = e;
    return STST_ERR_CUDA;
  }
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  Profiler *saved = g_prof;
  g_prof = nullptr;
  e = cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    stst_last_cuda = e;
    return STST_ERR_CUDA;
  }
  // two iterations per body: half the conditional node's per-body cost (measured ~2.5 us an iteration);
  // every kernel skips once the loop is done, so the iteration count and the maxit bound are unchanged
  int s = pcg_body(h, cond, 1);
  if (s == STST_OK) s = pcg_body(h, cond, 1);
  cudaGraph_t captured = nullptr;
  e = cudaStreamEndCapture(st, &captured);
  g_prof = saved;
  if (s != STST_OK || e != cudaSuccess) {
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) stst_last_cuda = e;
    return s != STST_OK ? s : STST_ERR_CUDA;
  }
  size_t n_nodes = 0;
  e = cudaGraphGetNodes(body, nullptr, &n_nodes);
  std::vector<cudaGraphNode_t> nodes(n_nodes);
  if (e == cudaSuccess && n_nodes) e = cudaGraphGetNodes(body, nodes.data(), &n_nodes);
  int kernels = 0;
  for (size_t i = 0; e == cudaSuccess && i < n_nodes; ++i) {
    cudaGraphNodeType t;
    e = cudaGraphNodeGetType(nodes[i], &t);
    kernels += (e == cudaSuccess && t == cudaGraphNodeTypeKernel);
  }
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    stst_last_cuda = e;
    return STST_ERR_CUDA;
  }
  h->pcg_body_kernels = kernels;
  e = cudaGraphInstantiate(&h->pcg_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    stst_last_cuda = e;
    return STST_ERR_CUDA;
  }
  h->pcg_graph_valid = 1;
  return STST_OK;
}

// Waits for the stream and reads the handle's bounded-wait flag (flags[1], bit 2: a tensor-core mode
// product gave up waiting for its copies or MMAs; bit 3: a grid barrier of the fused mat-vec gave up)
// into flags_host[1], clearing it on the device for the next call.
static int take_timeout_flag(stst_problem *h) {
  cudaStream_t st = h->stream;
  STST_CUDA(cudaMemcpyAsync(h->flags_host + 1, h->flags + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
  STST_CUDA(cudaMemsetAsync(h->flags + 1, 0, sizeof(int), st));
  STST_CUDA(cudaStreamSynchronize(st));
  return STST_OK;
}

int pcg_run(stst_problem *h, const double *rhs, double *x, double tol, int maxit, int *iters, double *relres) {
  cudaStream_t st = h->stream;
  const size_t bytes = sizeof(double) * 2 * (size_t)h->N_dof;
  PcgCtl c0 = {};
  c0.tol2 = tol * tol;
  c0.maxit = maxit;
  c0.x0_zero = 1;  // cleared on the device if x holds a nonzero entry
  c0.flexible = h->prec_mode != STST_PREC_FP64;
  *h->ctl_host = c0;
  STST_CUDA(cudaMemcpyAsync(h->ctl, h->ctl_host, sizeof(PcgCtl), cudaMemcpyHostToDevice, st));
  STST_CUDA(cudaMemcpyAsync(h->w_f, rhs, bytes, cudaMemcpyDeviceToDevice, st));
  STST_CUDA(cudaMemcpyAsync(h->w_x, x, bytes, cudaMemcpyDeviceToDevice, st));
  STST_TRY(pcg_init(h));
  if (maxit > 0) {
    if (g_prof) {
      // profiled run: plain launches, one host check per iteration (events cannot sit in a graph body)
      for (int k = 0; k < maxit; ++k) {
        STST_TRY(pcg_body(h, cudaGraphConditionalHandle(), 0));
        STST_CUDA(cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(PcgCtl), cudaMemcpyDeviceToHost, st));
        STST_CUDA(cudaStreamSynchronize(st));
        if (h->ctl_host->done) break;
      }
    } else {
      if (!h->pcg_graph_valid) STST_TRY(build_pcg_graph(h));
      STST_CUDA(cudaGraphLaunch(h->pcg_exec, st));
    }
  }
  STST_CUDA(cudaMemcpyAsync(x, h->w_x, bytes, cudaMemcpyDeviceToDevice, st));
  STST_CUDA(cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(PcgCtl), cudaMemcpyDeviceToHost, st));
  STST_TRY(take_timeout_flag(h));
  const PcgCtl &c = *h->ctl_host;
  if (iters) *iters = c.it;
  if (relres) *relres = c.ff > 0 ? sqrt(c.rr / c.ff) : 0.0;
  if (h->flags_host[1] & 12) return STST_TIMEOUT;  // bit 2: tensor-core waits, bit 3: grid barriers
  if (c.status != STST_OK) return c.status;
  if (!c.done) return STST_NOT_CONVERGED;
  return STST_OK;
}

// ------------------------------------------------------------------------------------------------
// Mixed-precision iterative refinement: FP64 residual r = b - A x and FP64 update x += ||r|| d around
// an inner FP32 PCG on A d = r / ||r|| (FP32 mat-vec, FP32 preconditioner, flexible beta).
// ------------------------------------------------------------------------------------------------
__global__ void k_ir_outer(PcgCtl *ctl, const double *prr, int nrr, int first) {
  __shared__ double sh[32];
  double rr = reduce_partials(prr, nrr, sh);
  if (threadIdx.x == 0) {
    ctl->rr = rr;
    if (first) ctl->ff = rr;  // x0 = 0 on the first step would give rr = ||b||^2; ff is set by the caller otherwise
    ctl->done = (ctl->ff == 0.0 || rr <= ctl->tol2 * ctl->ff) ? 1 : 0;
    if (!isfinite(rr)) { ctl->done = 1; ctl->status = STST_BREAKDOWN; }
  }
}

__global__ void k_set_ff(PcgCtl *ctl, const double *pf, int nf) {
  __shared__ double sh[32];
  double ff = reduce_partials(pf, nf, sh);
  if (threadIdx.x == 0) ctl->ff = ff;
}

__global__ void k_r_to_f32(const double2 *__restrict__ r, float2 *__restrict__ r32, const PcgCtl *ctl, long long n) {
  if (ctl->done) return;
  const double sc = 1.0 / sqrt(ctl->rr);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double2 v = r[i];
    r32[i] = make_float2((float)(v.x * sc), (float)(v.y * sc));
  }
}

__global__ void k_x_from_f32(double2 *__restrict__ x, const float2 *__restrict__ d, const PcgCtl *ctl, long long n) {
  if (ctl->done) return;
  const double sc = sqrt(ctl->rr);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float2 v = d[i];
    double2 xv = x[i];
    xv.x += sc * (double)v.x;
    xv.y += sc * (double)v.y;
    x[i] = xv;
  }
}

static int inner_body(stst_problem *h, cudaGraphConditionalHandle cond, int use_cond) {
  // FP32 mat-vec, FP32 (or BF16 tensor-core) preconditioner, flexible CG on the FP32 vectors
  return pcg_iteration<float2>(h, h->ctl2, (float2 *)h->v_d, (float2 *)h->v_r, (float2 *)h->v_z, (float2 *)h->v_p,
                               (float2 *)h->v_q, 1, h->prec_mode == STST_PREC_BF16 ? 2 : 1, cond, use_cond);
}

static int build_ir_graph(stst_problem *h) {
  cudaStream_t st = h->stream;
  cudaGraph_t graph;
  STST_CUDA(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle cond;
  cudaError_t e = cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams cp = {};
  cudaGraphNode_t node;
  if (e == cudaSuccess) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
  }
  Profiler *saved = g_prof;
  g_prof = nullptr;
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(st, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                          cudaStreamCaptureModeRelaxed);
  int s = STST_OK;
  if (e == cudaSuccess) {
    s = inner_body(h, cond, 1);
    if (s == STST_OK) s = inner_body(h, cond, 1);  // two iterations per body, as in the PCG graph
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(st, &captured);
  }
  g_prof = saved;
  if (e == cudaSuccess && s == STST_OK) e = cudaGraphInstantiate(&h->ir_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    stst_last_cuda = e;
    return STST_ERR_CUDA;
  }
  if (s != STST_OK) return s;
  h->ir_graph_valid = 1;
  return STST_OK;
}

int ir_run(stst_problem *h, const double *rhs, double *x, double tol, int maxit, double inner_tol, int inner_maxit,
           int *iters, int *outer, double *relres) {
  cudaStream_t st = h->stream;
  const long long N = h->N_dof;
  const int g = reduction_grid(N);
  const size_t bytes = sizeof(double2) * (size_t)N;
  double *P = h->partials;
  double *pZ = P + PS_Z * STST_MAXPART, *pRR = P + PS_RR * STST_MAXPART, *pF = P + PS_RP * STST_MAXPART;
  PcgCtl c0 = {};
  c0.tol2 = tol * tol;
  c0.maxit = maxit;
  PcgCtl c2 = {};
  c2.tol2 = inner_tol * inner_tol;
  c2.maxit = inner_maxit;
  c2.flexible = 1;
  h->ctl_host[0] = c0;
  STST_CUDA(cudaMemcpyAsync(h->ctl, h->ctl_host, sizeof(PcgCtl), cudaMemcpyHostToDevice, st));
  STST_CUDA(cudaMemcpyAsync(h->w_f, rhs, bytes, cudaMemcpyDeviceToDevice, st));
  STST_CUDA(cudaMemcpyAsync(h->w_x, x, bytes, cudaMemcpyDeviceToDevice, st));
  { STST_PROF("norm2", st); k_norm2<double2><<<g, 256, 0, st>>>((const double2 *)h->w_f, N, pF); }
  { STST_PROF("pcg_scalar", st); k_set_ff<<<1, 1024, 0, st>>>(h->ctl, pF, g); }
  int total_inner = 0, k = 0, status = STST_NOT_CONVERGED;
  PcgCtl hc2 = {};
  for (k = 0; k <= maxit; ++k) {
    // FP64 residual
    STST_TRY(run_plan(h->sys_plan, h->w_x, h->w_r, 0, 1, h->w_f, nullptr, nullptr, nullptr, st, nullptr, pRR));
    { STST_PROF("pcg_scalar", st); k_ir_outer<<<1, 1024, 0, st>>>(h->ctl, pRR, g, 0); }
    STST_CUDA(cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(PcgCtl), cudaMemcpyDeviceToHost, st));
    if (k > 0) STST_CUDA(cudaMemcpyAsync(&h->ctl_host[1], h->ctl2, sizeof(PcgCtl), cudaMemcpyDeviceToHost, st));
    STST_CUDA(cudaStreamSynchronize(st));
    if (k > 0) total_inner += h->ctl_host[1].it;
    if (h->ctl_host[0].status == STST_BREAKDOWN) { status = STST_BREAKDOWN; break; }
    if (h->ctl_host[0].done) { status = STST_OK; break; }
    if (k == maxit) break;
    // inner FP32 PCG on A d = r / ||r||
    { STST_PROF("ir_convert", st); k_r_to_f32<<<g, 256, 0, st>>>((const double2 *)h->w_r, (float2 *)h->v_r, h->ctl, N); }
    STST_CUDA(cudaMemsetAsync(h->v_d, 0, sizeof(float2) * N, st));
    hc2 = c2;
    h->ctl_host[1] = hc2;
    STST_CUDA(cudaMemcpyAsync(h->ctl2, &h->ctl_host[1], sizeof(PcgCtl), cudaMemcpyHostToDevice, st));
    { STST_PROF("norm2", st); k_norm2<float2><<<g, 256, 0, st>>>((const float2 *)h->v_r, N, pF); }
    {
      EpiDot ed;  // the inner solve is the flexible CG: complex <r, z>
      ed.a = h->v_r;
      ed.part = pZ;
      ed.cplx = 1;
      STST_TRY(fd_apply(h, nullptr, nullptr, h->prec_mode == STST_PREC_BF16 ? 2 : 1, ed, nullptr, h->w_t1, h->w_t2,
                        h->v_z, h->v_r));
    }
    { STST_PROF("pcg_scalar", st);
      k_pcg_init<<<1, 1024, 0, st>>>(h->ctl2, pF, g, pF, g, pZ, fd_partials_count(h)); }
    { STST_PROF("copy", st);
      k_copy_vec<float2><<<g, 256, 0, st>>>((const float2 *)h->v_z, (float2 *)h->v_p, N, &h->ctl2->done); }
    if (g_prof) {
      for (int j = 0; j < inner_maxit; ++j) {
        STST_TRY(inner_body(h, cudaGraphConditionalHandle(), 0));
        STST_CUDA(cudaMemcpyAsync(&h->ctl_host[1], h->ctl2, sizeof(PcgCtl), cudaMemcpyDeviceToHost, st));
        STST_CUDA(cudaStreamSynchronize(st));
        if (h->ctl_host[1].done) break;
      }
    } else {
      if (!h->ir_graph_valid) STST_TRY(build_ir_graph(h));
      STST_CUDA(cudaGraphLaunch(h->ir_exec, st));
    }
    { STST_PROF("ir_update", st); k_x_from_f32<<<g, 256, 0, st>>>((double2 *)h->w_x, (const float2 *)h->v_d, h->ctl, N); }
  }
  STST_CUDA(cudaMemcpyAsync(x, h->w_x, bytes, cudaMemcpyDeviceToDevice, st));
  STST_TRY(take_timeout_flag(h));
  const PcgCtl &c = h->ctl_host[0];
  if (iters) *iters = total_inner;
  if (outer) *outer = k;
  if (relres) *relres = c.ff > 0 ? sqrt(c.rr / c.ff) : 0.0;
  if (h->flags_host[1] & 12) return STST_TIMEOUT;  // bit 2: tensor-core waits, bit 3: grid barriers
  return status;
}
