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

enum { PART_A = 0, PART_B = 1, PART_C = 2, PART_D = 3 };

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

// init: ff, rr, rho from partials; done if converged already
__global__ void k_pcg_init(PcgCtl *ctl, const double *pf, int nf, const double *pr, int nr, const double *prz, int nrz) {
  __shared__ double sh[32];
  double ff = reduce_partials(pf, nf, sh);
  double rr = reduce_partials(pr, nr, sh);
  double rz = reduce_partials(prz, nrz, sh);
  if (threadIdx.x == 0) {
    ctl->ff = ff;
    ctl->rr = rr;
    ctl->rho = rz;
    ctl->it = 0;
    ctl->status = STST_OK;
    ctl->done = (ff == 0.0 || rr <= ctl->tol2 * ff) ? 1 : 0;
    if (!ctl->done && !(rz > 0.0 && isfinite(rz))) { ctl->done = 1; ctl->status = STST_BREAKDOWN; }
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

// alpha = rho / <p, q> (every CTA reduces the same partials in the same order; CTA 0 records it),
// then x += alpha p; r -= alpha q; partials of ||r||^2 and (flexible) Re<r, z_old>
// rho = <r, z> is reduced from the partials of the latest preconditioner application (prz_in), so no
// CTA of this kernel reads a scalar that another CTA of it writes.
template <typename T>
__global__ void __launch_bounds__(256) k_update_xr(T *__restrict__ x, T *__restrict__ r, const T *__restrict__ p,
                                                   const T *__restrict__ q, const T *__restrict__ zold, PcgCtl *ctl,
                                                   long long n, double *prr, double *prz, const double *ppq, int npq,
                                                   const double *prz_in, int nrz_in) {
  if (ctl->done) return;
  __shared__ double sh[32];
  const long long stride = (long long)gridDim.x * 256 * UPT;
  long long i0 = (long long)blockIdx.x * 256 * UPT + threadIdx.x;
  T pv[UPT], qv[UPT], xv[UPT], rv[UPT], zv[UPT];
  auto load = [&](long long base) {
#pragma unroll
    for (int u = 0; u < UPT; ++u) {
      const long long i = base + 256 * u;
      if (i < n) {
        pv[u] = p[i];
        qv[u] = q[i];
        xv[u] = x[i];
        rv[u] = r[i];
        if (zold) zv[u] = zold[i];
      }
    }
  };
  if (i0 < n) load(i0);
  const double pq = reduce_partials(ppq, npq, sh);
  const double rho = reduce_partials(prz_in, nrz_in, sh);
  const bool bad = !(pq > 0.0) || !isfinite(pq);
  const double alpha = bad ? 0.0 : rho / pq;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->pq = pq;
    ctl->rho = rho;
    ctl->alpha = alpha;
    if (bad) ctl->status = STST_BREAKDOWN;  // the check kernel ends the loop
  }
  double arr = 0.0, arz = 0.0;
  for (; i0 < n; i0 += stride) {
#pragma unroll
    for (int u = 0; u < UPT; ++u) {
      const long long i = i0 + 256 * u;
      if (i < n) {
        xv[u].x += alpha * pv[u].x;
        xv[u].y += alpha * pv[u].y;
        rv[u].x -= alpha * qv[u].x;
        rv[u].y -= alpha * qv[u].y;
        x[i] = xv[u];
        r[i] = rv[u];
        arr += (double)rv[u].x * rv[u].x + (double)rv[u].y * rv[u].y;
        if (zold) arz += (double)zv[u].x * rv[u].x + (double)zv[u].y * rv[u].y;
      }
    }
    if (i0 + stride < n) load(i0 + stride);
  }
  double s = block_sum_d(arr, sh);
  if (threadIdx.x == 0) prr[blockIdx.x] = s;
  if (zold) {
    double t = block_sum_d(arz, sh);
    if (threadIdx.x == 0) prz[blockIdx.x] = t;
  }
}

// control: count the iteration, test ||r|| <= tol ||f||, maxit; set the WHILE condition.
__global__ void k_pcg_check(PcgCtl *ctl, const double *prr, int nrr, const double *prz, int nrz,
                            cudaGraphConditionalHandle cond, int use_cond) {
  __shared__ double sh[32];
  int was_done = ctl->done;
  double rr = reduce_partials(prr, nrr, sh);
  double rz = (prz && nrz > 0) ? reduce_partials(prz, nrz, sh) : 0.0;
  if (threadIdx.x == 0) {
    if (!was_done) {
      ctl->it += 1;
      ctl->rr = rr;
      ctl->rz_old = rz;
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

// beta from the new <r, z> partials (Fletcher-Reeves, or Polak-Ribiere when flexible), p = z + beta p.
// rho_old (written by k_update_xr) and rz_old (written by the check kernel) come from earlier
// kernels; this kernel writes no scalar that its own CTAs read.
template <typename T>
__global__ void __launch_bounds__(256) k_update_p(T *__restrict__ p, const T *__restrict__ z, PcgCtl *ctl, long long n,
                                                  const double *prz, int nrz) {
  if (ctl->done) return;
  __shared__ double sh[32];
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
  const double rho_old = ctl->rho, rz_old = ctl->rz_old;
  const int flexible = ctl->flexible;
  const double rho_new = reduce_partials(prz, nrz, sh);
  const bool bad = !(rho_new > 0.0) || !isfinite(rho_new);
  const double beta = bad ? 0.0 : (flexible ? (rho_new - rz_old) / rho_old : rho_new / rho_old);
  if (bad && blockIdx.x == 0 && threadIdx.x == 0) ctl->status = STST_BREAKDOWN;
  for (; i0 < n; i0 += stride) {
#pragma unroll
    for (int u = 0; u < UPT; ++u) {
      const long long i = i0 + 256 * u;
      if (i < n) {
        pv[u].x = zv[u].x + beta * pv[u].x;
        pv[u].y = zv[u].y + beta * pv[u].y;
        p[i] = pv[u];
      }
    }
    if (i0 + stride < n) load(i0 + stride);
  }
}

// ------------------------------------------------------------------------------------------------
// FP64 PCG
// ------------------------------------------------------------------------------------------------
int pcg_body(stst_problem *h, cudaGraphConditionalHandle cond, int use_cond) {
  cudaStream_t st = h->stream;
  const long long N = h->N_dof;
  const int g = reduction_grid(N), gu = update_grid(N);
  const int prec = h->prec_mode;  // STST_PREC_* equals fd_apply's precision code
  double *P = h->partials;
  double *pA = P, *pB = P + STST_MAXPART, *pC = P + 2 * STST_MAXPART, *pD = P + 3 * STST_MAXPART;
  const int *done = &h->ctl->done;
  const int flexible = prec != 0;
  const int nrz = fd_partials_count(h);
  // q = A p, partials <p, q>
  STST_TRY(run_plan(h->sys_plan, h->w_p, h->w_q, 0, 0, nullptr, h->w_p, pD, done, st));
  // alpha; x, r update (+ Re<r_new, z_old> for the flexible beta)
  { STST_PROF("pcg_update_xr", st); k_update_xr<double2><<<gu, 256, 0, st>>>((double2 *)h->w_x, (double2 *)h->w_r, (const double2 *)h->w_p,
                                          (const double2 *)h->w_q, flexible ? (const double2 *)h->w_z : nullptr,
                                          h->ctl, N, pB, pC, pD, g, pA, nrz); }
  { STST_PROF("pcg_scalar", st); k_pcg_check<<<1, 1024, 0, st>>>(h->ctl, pB, gu, flexible ? pC : nullptr, flexible ? gu : 0, cond, use_cond); }
  // z = P^{-1} r, partials <r, z>
  STST_TRY(fd_apply(h, h->w_r, h->w_z, prec, h->w_r, pA, done, h->w_t1, h->w_t2));
  { STST_PROF("pcg_update_p", st); k_update_p<double2><<<gu, 256, 0, st>>>((double2 *)h->w_p, (const double2 *)h->w_z, h->ctl, N, pA, nrz); }
  STST_CUDA(cudaGetLastError());
  return STST_OK;
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
  double *pA = P, *pB = P + STST_MAXPART, *pC = P + 2 * STST_MAXPART;
  // r = f - A x, partials ||r||^2 ; ||f||^2. From x0 = 0 (the paper's start, Sec. 6) r = f needs no
  // mat-vec: a device check of x0 makes the residual's passes skip themselves and a copy takes over.
  { STST_PROF("pcg_init", st); k_x0_zero_check<<<g, 256, 0, st>>>((const double2 *)h->w_x, N, h->ctl); }
  STST_TRY(run_plan(h->sys_plan, h->w_x, h->w_r, 0, 1, h->w_f, nullptr, nullptr, &h->ctl->x0_zero, st, nullptr, pB));
  {
    STST_PROF_N("pcg_init", st, 2);
    k_resid_from_zero<<<g, 512, 0, st>>>(h->ctl, (const double2 *)h->w_f, (double2 *)h->w_r, N, pB);
    k_norm2<double2><<<g, 256, 0, st>>>((const double2 *)h->w_f, N, pC);
  }
  // z = P^{-1} r with <r, z>
  STST_TRY(fd_apply(h, h->w_r, h->w_z, prec, h->w_r, pA, nullptr, h->w_t1, h->w_t2));
  {
    STST_PROF_N("pcg_init", st, 2);
    k_pcg_init<<<1, 1024, 0, st>>>(h->ctl, pC, g, pB, g, pA, fd_partials_count(h));
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

// Waits for the stream and reads the handle's bounded-wait flag (flags[1], bit 2: the tensor-core mode
// product gave up waiting for its MMAs) into flags_host[1], clearing it on the device for the next call.
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
  if (h->flags_host[1] & 4) return STST_TIMEOUT;
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
  cudaStream_t st = h->stream;
  const long long N = h->N_dof;
  const int g = reduction_grid(N), gu = update_grid(N);
  double *P = h->partials;
  double *pA = P, *pB = P + STST_MAXPART, *pC = P + 2 * STST_MAXPART, *pD = P + 3 * STST_MAXPART;
  const int *done = &h->ctl2->done;
  const int nrz = fd_partials_count(h);
  STST_TRY(run_plan(h->sys_plan, h->v_p, h->v_q, 1, 0, nullptr, h->v_p, pD, done, st));
  { STST_PROF("pcg_update_xr", st);
    k_update_xr<float2><<<gu, 256, 0, st>>>((float2 *)h->v_d, (float2 *)h->v_r, (const float2 *)h->v_p,
                                            (const float2 *)h->v_q, (const float2 *)h->v_z, h->ctl2, N, pB, pC,
                                            pD, g, pA, nrz); }
  { STST_PROF("pcg_scalar", st); k_pcg_check<<<1, 1024, 0, st>>>(h->ctl2, pB, gu, pC, gu, cond, use_cond); }
  STST_TRY(fd_apply(h, nullptr, nullptr, h->prec_mode == STST_PREC_BF16 ? 2 : 1, h->v_r, pA, done, h->w_t1, h->w_t2, h->v_z, h->v_r));
  { STST_PROF("pcg_update_p", st);
    k_update_p<float2><<<gu, 256, 0, st>>>((float2 *)h->v_p, (const float2 *)h->v_z, h->ctl2, N, pA, nrz); }
  STST_CUDA(cudaGetLastError());
  return STST_OK;
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
  double *pA = P, *pB = P + STST_MAXPART, *pC = P + 2 * STST_MAXPART;
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
  { STST_PROF("norm2", st); k_norm2<double2><<<g, 256, 0, st>>>((const double2 *)h->w_f, N, pC); }
  { STST_PROF("pcg_scalar", st); k_set_ff<<<1, 1024, 0, st>>>(h->ctl, pC, g); }
  int total_inner = 0, k = 0, status = STST_NOT_CONVERGED;
  PcgCtl hc2 = {};
  for (k = 0; k <= maxit; ++k) {
    // FP64 residual
    STST_TRY(run_plan(h->sys_plan, h->w_x, h->w_r, 0, 1, h->w_f, nullptr, nullptr, nullptr, st, nullptr, pB));
    { STST_PROF("pcg_scalar", st); k_ir_outer<<<1, 1024, 0, st>>>(h->ctl, pB, g, 0); }
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
    { STST_PROF("norm2", st); k_norm2<float2><<<g, 256, 0, st>>>((const float2 *)h->v_r, N, pC); }
    STST_TRY(fd_apply(h, nullptr, nullptr, h->prec_mode == STST_PREC_BF16 ? 2 : 1, h->v_r, pA, nullptr, h->w_t1, h->w_t2, h->v_z, h->v_r));
    { STST_PROF("pcg_scalar", st);
      k_pcg_init<<<1, 1024, 0, st>>>(h->ctl2, pC, g, pC, g, pA, fd_partials_count(h)); }
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
  if (h->flags_host[1] & 4) return STST_TIMEOUT;
  return status;
}
