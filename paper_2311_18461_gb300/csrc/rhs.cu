// Right-hand side of the reduced system (Sec. 4.3) and the lifting of the initial datum (Sec. 2.2):
//   rhs_i = int f conj(S_V B_i) - sum_j A_full(b_1 B_j, S_V B_i) c_j,  c = M_s^{-1} (u0, B_j);
// for the ultraweak formulation (Sec. 4.4): rhs_i = int f conj(B_i) + i (u0, B_i(., 0)).
// Integrals are tensor Gauss sums evaluated as mode-by-mode contractions of the sampled data with
// the basis tables; M_s^{-1} is applied mode by mode with the banded Cholesky factor of M_l; the
// lifting is the Kronecker operator applied to c placed on the first (removed) time function.
#include "common.cuh"

// out[o, i, c] = scale * sum_{q in supp(b_I)} w_q d^der b_I(x_q) in[o, q, c]  (+ out if accumulate)
template <typename TI>
__global__ void k_contract(const TI *__restrict__ in, double2 *__restrict__ out, const double *__restrict__ tab,
                           const double *__restrict__ wts, int p, int nq, int n_el, int off, int n_out, int Q,
                           long long inner, long long outer, int der, double sre, double sim, int accumulate) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long total = outer * n_out * inner;
  if (idx >= total) return;
  long long c = idx % inner;
  long long t = idx / inner;
  int i = (int)(t % n_out);
  long long o = t / n_out;
  int I = i + off;
  double ax = 0.0, ay = 0.0;
  for (int e = max(I - p, 0); e <= min(I, n_el - 1); ++e) {
    for (int g = 0; g < nq; ++g) {
      int q = e * nq + g;
      double b = tab[((long long)q * (p + 1) + (I - e)) * 3 + der] * wts[q];
      TI v = in[(o * Q + q) * inner + c];
      ax += b * (double)v.x;
      ay += b * (double)v.y;
    }
  }
  double rx = sre * ax - sim * ay, ry = sre * ay + sim * ax;
  if (accumulate) {
    double2 prev = out[idx];
    rx += prev.x;
    ry += prev.y;
  }
  out[idx] = make_double2(rx, ry);
}

// Ultraweak initial term: rhs[(t = 0, j)] += i g_j (time fastest: index j n_t)
__global__ void k_add_initial_uw(double2 *__restrict__ rhs, const double2 *__restrict__ g, int nt, long long Ns) {
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= Ns) return;
  double2 r = rhs[j * nt];
  const double2 v = g[j];
  r.x -= v.y;
  r.y += v.x;
  rhs[j * nt] = r;
}

// Solve M_l y = g along mode l in place (lines of length n with stride inner), banded Cholesky.
__global__ void k_mass_solve(double2 *__restrict__ g, const double *__restrict__ chol, int n, int p, long long inner,
                             long long outer) {
  long long line = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (line >= inner * outer) return;
  long long o = line / inner, c = line % inner;
  double2 *v = g + o * n * inner + c;
  // forward C y = g
  for (int i = 0; i < n; ++i) {
    double2 s = v[(long long)i * inner];
    for (int m = max(i - p, 0); m < i; ++m) {
      double cm = chol[i * (p + 1) + (m - i + p)];
      double2 ym = v[(long long)m * inner];
      s.x -= cm * ym.x;
      s.y -= cm * ym.y;
    }
    double di = 1.0 / chol[i * (p + 1) + p];
    v[(long long)i * inner] = make_double2(s.x * di, s.y * di);
  }
  // backward C^T x = y
  for (int i = n - 1; i >= 0; --i) {
    double2 s = v[(long long)i * inner];
    for (int m = i + 1; m <= min(i + p, n - 1); ++m) {
      double cm = chol[m * (p + 1) + (i - m + p)];
      double2 xm = v[(long long)m * inner];
      s.x -= cm * xm.x;
      s.y -= cm * xm.y;
    }
    double di = 1.0 / chol[i * (p + 1) + p];
    v[(long long)i * inner] = make_double2(s.x * di, s.y * di);
  }
}

// F[q_t, q_s] *= V(x_{q_s}) with V = sum_r prod_l v_{r,l}(x_l) (time fastest, spatial grid flattened x_1 fastest)
__global__ void k_mul_potential(const double2 *__restrict__ F, double2 *__restrict__ out, long long Qt, int d,
                                int Q1, int Q2, int Q3, int rank, const double *__restrict__ v, long long total) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= total) return;
  long long s = idx / Qt;
  int q1 = (int)(s % Q1);
  long long r2 = s / Q1;
  int q2 = d >= 2 ? (int)(r2 % Q2) : 0;
  int q3 = d >= 3 ? (int)(r2 / Q2) : 0;
  const int stride = Q1 + (d >= 2 ? Q2 : 0) + (d >= 3 ? Q3 : 0);
  double V = 0.0;
  for (int r = 0; r < rank; ++r) {
    const double *vr = v + (long long)r * stride;
    double t = vr[q1];
    if (d >= 2) t *= vr[Q1 + q2];
    if (d >= 3) t *= vr[Q1 + Q2 + q3];
    V += t;
  }
  double2 f = F[idx];
  out[idx] = make_double2(f.x * V, f.y * V);
}

template <typename TI>
static int contract(stst_problem *h, int l, const TI *in, double2 *out, long long inner, long long outer, int der,
                    double sre, double sim, int acc) {
  const DirInfo &D = h->dir[l];
  long long total = outer * D.n * inner;
  if (total == 0) return STST_OK;
  k_contract<TI><<<grid_for(total, 128), 128, 0, h->stream>>>(in, out, h->tab[l], h->qwts[l], D.p, D.nq, D.n_el,
                                                               D.off, D.n, D.Q(), inner, outer, der, sre, sim, acc);
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}

int rhs_compute(stst_problem *h, const double *f_qp, const double *u0_qp, double *rhs, double *c0) {
  cudaStream_t st = h->stream;
  const int d = h->d;
  const long long N = h->N_dof;
  int Q[STST_MAXD + 1], n[STST_MAXD + 1];
  for (int l = 0; l <= d; ++l) {
    Q[l] = h->dir[l].Q();
    n[l] = h->dir[l].n;
  }
  STST_CUDA(cudaMemsetAsync(rhs, 0, sizeof(double2) * N, st));
  if (f_qp) {
    // temporaries: after the time contraction the tensor is n_t x prod Q_l
    long long sz = (long long)n[0];
    for (int l = 1; l <= d; ++l) sz *= Q[l];
    long long szF = (long long)Q[0];
    for (int l = 1; l <= d; ++l) szF *= Q[l];
    double2 *T1, *T0, *W1, *W2, *FV = nullptr;
    STST_CUDA(cudaMallocAsync(&T1, sizeof(double2) * sz, st));
    STST_CUDA(cudaMallocAsync(&T0, sizeof(double2) * sz, st));
    STST_CUDA(cudaMallocAsync(&W1, sizeof(double2) * sz, st));
    STST_CUDA(cudaMallocAsync(&W2, sizeof(double2) * sz, st));
    const long long Qs = szF / Q[0];
    const bool uw = h->formulation == STST_FORM_UW;  // ultraweak: plain load int f conj(B_i)
    // time contractions (mode 0: inner 1, outer prod Q_l): T1 = -i int f b'_t, T0 = int f b_t
    if (!uw) STST_TRY(contract(h, 0, (const double2 *)f_qp, T1, 1, Qs, 1, 0.0, -1.0, 0));
    STST_TRY(contract(h, 0, (const double2 *)f_qp, T0, 1, Qs, 0, 1.0, 0.0, 0));
    // spatial contractions. term list: (src, ders per mode, scale)
    struct Term { double2 *src; int der[STST_MAXD + 1]; double s; };
    std::vector<Term> terms;
    if (uw) {
      Term t0 = {T0, {0, 0, 0, 0}, 1.0};
      terms.push_back(t0);
    } else {
      Term t1 = {T1, {0, 0, 0, 0}, 1.0};
      terms.push_back(t1);
      for (int l = 1; l <= d; ++l) {
        Term t = {T0, {0, 0, 0, 0}, -h->nu};
        t.der[l] = 2;
        terms.push_back(t);
      }
    }
    double2 *T0V = nullptr;
    if (h->pot_rank > 0 && !uw) {
      STST_CUDA(cudaMallocAsync(&FV, sizeof(double2) * szF, st));
      STST_CUDA(cudaMallocAsync(&T0V, sizeof(double2) * sz, st));
      k_mul_potential<<<grid_for(szF, 256), 256, 0, st>>>((const double2 *)f_qp, FV, Q[0], d, Q[1],
                                                           d >= 2 ? Q[2] : 1, d >= 3 ? Q[3] : 1, h->pot_rank,
                                                           h->pot_bufs[0], szF);
      STST_CUDA(cudaGetLastError());
      STST_TRY(contract(h, 0, (const double2 *)FV, T0V, 1, Qs, 0, 1.0, 0.0, 0));
      Term tv = {T0V, {0, 0, 0, 0}, 1.0};
      terms.push_back(tv);
    }
    for (const Term &t : terms) {
      const double2 *src = t.src;
      long long ext[STST_MAXD + 1];
      ext[0] = n[0];
      for (int l = 1; l <= d; ++l) ext[l] = Q[l];
      double2 *bufs[2] = {W1, W2};
      int cur = 0;
      for (int l = 1; l <= d; ++l) {
        long long inner = 1, outer = 1;
        for (int k = 0; k < l; ++k) inner *= ext[k];
        for (int k = l + 1; k <= d; ++k) outer *= ext[k];
        bool last = (l == d);
        double2 *dst = last ? (double2 *)rhs : bufs[cur];
        STST_TRY(contract(h, l, src, dst, inner, outer, t.der[l], last ? t.s : 1.0, 0.0, last ? 1 : 0));
        ext[l] = n[l];
        src = dst;
        cur ^= 1;
      }
    }
    cudaFreeAsync(T1, st);
    cudaFreeAsync(T0, st);
    cudaFreeAsync(W1, st);
    cudaFreeAsync(W2, st);
    if (FV) cudaFreeAsync(FV, st);
    if (T0V) cudaFreeAsync(T0V, st);
  }
  if (u0_qp) {
    // g = (u0, B_j) by spatial contractions, then c = M_s^{-1} g mode by mode
    double2 *W1 = (double2 *)h->proj_work;
    double2 *W2 = W1 + h->proj_work_bytes / sizeof(double2) / 3;
    double2 *C = W2 + h->proj_work_bytes / sizeof(double2) / 3;
    long long ext[STST_MAXD + 1];
    for (int l = 1; l <= d; ++l) ext[l] = Q[l];
    const double2 *src = (const double2 *)u0_qp;
    double2 *bufs[2] = {W1, W2};
    int cur = 0;
    for (int l = 1; l <= d; ++l) {
      long long inner = 1, outer = 1;
      for (int k = 1; k < l; ++k) inner *= ext[k];
      for (int k = l + 1; k <= d; ++k) outer *= ext[k];
      double2 *dst = (l == d) ? C : bufs[cur];
      STST_TRY(contract(h, l, src, dst, inner, outer, 0, 1.0, 0.0, 0));
      ext[l] = n[l];
      src = dst;
      cur ^= 1;
    }
    if (h->formulation == STST_FORM_UW) {  // rhs += i (u0, B_j) on time index 0
      k_add_initial_uw<<<grid_for(h->N_s, 256), 256, 0, st>>>((double2 *)rhs, C, n[0], h->N_s);
      STST_CUDA(cudaGetLastError());
    }
    for (int l = 1; l <= d; ++l) {
      long long inner = 1, outer = 1;
      for (int k = 1; k < l; ++k) inner *= n[k];
      for (int k = l + 1; k <= d; ++k) outer *= n[k];
      k_mass_solve<<<grid_for(inner * outer, 128), 128, 0, st>>>(C, h->mchol[l], n[l], h->dir[l].p, inner, outer);
      STST_CUDA(cudaGetLastError());
    }
    if (c0) STST_CUDA(cudaMemcpyAsync(c0, C, sizeof(double2) * h->N_s, cudaMemcpyDeviceToDevice, st));
    // least squares: rhs -= A_full[:, (1, j)] c_j
    if (h->formulation == STST_FORM_LS)
      STST_TRY(run_plan(h->lift_plan, C, rhs, 0, 1, rhs, nullptr, nullptr, nullptr, st));
  } else if (c0) {
    STST_CUDA(cudaMemsetAsync(c0, 0, sizeof(double2) * h->N_s, st));
  }
  return STST_OK;
}

// ------------------------------------------------------------------------------------------------
// Allocation-free variant of stst_rhs (stst_rhs_noalloc). Its temporaries live in one file-scope
// device array of fixed size instead of memory taken from the allocator at call time. The array is
// part of the module: every GPU that loads this library holds it until the process exits. All calls
// on a device share it, so calls whose work overlaps on the GPU (different streams, or different
// host threads) race on it; calls ordered on one stream do not. Every word of the array that a call
// reads it has written earlier in the same call, so nothing needs clearing between calls.
// ------------------------------------------------------------------------------------------------
#include <mutex>

#define STST_RHS_SCRATCH_ELEMS (1 << 20)  // complex128 elements: 16 MiB
static __device__ __align__(256) double2 g_rhs_scratch[STST_RHS_SCRATCH_ELEMS];

// Device address of g_rhs_scratch, looked up once per device with that device current.
static int rhs_scratch_address(double2 **out) {
  static std::mutex mu;
  static double2 *addr[256];
  static bool ready[256];
  int dev = 0;
  STST_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return STST_ERR_ARG;
  std::lock_guard<std::mutex> lock(mu);
  if (!ready[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_rhs_scratch);
    if (e != cudaSuccess || p == nullptr) {
      stst_last_cuda = e;
      return STST_ERR_CUDA;
    }
    addr[dev] = (double2 *)p;
    ready[dev] = true;
  }
  *out = addr[dev];
  return STST_OK;
}

// out[s, i] = sum_{q in supp(b_I)} w_q b_I(t_q) (f[s, q] * V(x_s)): the time contraction of f V without
// forming f V on the grid.
__global__ void k_contract_time_pot(const double2 *__restrict__ in, double2 *__restrict__ out,
                                    const double *__restrict__ tab, const double *__restrict__ wts, int p, int nq,
                                    int n_el, int off, int n_out, int Q, long long Qs, int d, int Q1, int Q2, int Q3,
                                    int rank, const double *__restrict__ v) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= Qs * n_out) return;
  int i = (int)(idx % n_out);
  long long s = idx / n_out;
  int q1 = (int)(s % Q1);
  long long r2 = s / Q1;
  int q2 = d >= 2 ? (int)(r2 % Q2) : 0;
  int q3 = d >= 3 ? (int)(r2 / Q2) : 0;
  const int stride = Q1 + (d >= 2 ? Q2 : 0) + (d >= 3 ? Q3 : 0);
  double V = 0.0;
  for (int r = 0; r < rank; ++r) {
    const double *vr = v + (long long)r * stride;
    double t = vr[q1];
    if (d >= 2) t *= vr[Q1 + q2];
    if (d >= 3) t *= vr[Q1 + Q2 + q3];
    V += t;
  }
  int I = i + off;
  double ax = 0.0, ay = 0.0;
  for (int e = max(I - p, 0); e <= min(I, n_el - 1); ++e) {
    for (int g = 0; g < nq; ++g) {
      int q = e * nq + g;
      double b = tab[((long long)q * (p + 1) + (I - e)) * 3] * wts[q];
      double2 f = in[s * Q + q];
      double fx = f.x * V, fy = f.y * V;
      ax += b * fx;
      ay += b * fy;
    }
  }
  out[idx] = make_double2(ax, ay);
}

extern "C" int stst_rhs_noalloc(stst_handle h, const double *f_qp, const double *u0_qp, double *rhs, double *c0) {
  if (!h || h->magic != STST_MAGIC) return STST_ERR_HANDLE;
  if (!rhs) return STST_ERR_ARG;
  ApiScope scope(h);
  cudaStream_t st = h->stream;
  const int d = h->d;
  int Q[STST_MAXD + 1], n[STST_MAXD + 1];
  for (int l = 0; l <= d; ++l) {
    Q[l] = h->dir[l].Q();
    n[l] = h->dir[l].n;
  }
  double2 *scratch = nullptr;
  STST_TRY(rhs_scratch_address(&scratch));
  long long sz = n[0];
  for (int l = 1; l <= d; ++l) sz *= Q[l];
  const long long need = (h->pot_rank > 0 ? 5 : 4) * sz;
  if (f_qp && need > STST_RHS_SCRATCH_ELEMS) return STST_ERR_ARG;  // forcing grid too large for the static scratch
  STST_CUDA(cudaMemsetAsync(rhs, 0, sizeof(double2) * h->N_dof, st));
  if (f_qp) {
    double2 *T1 = scratch, *T0 = scratch + sz, *W1 = scratch + 2 * sz, *W2 = scratch + 3 * sz;
    double2 *T0V = h->pot_rank > 0 ? scratch + 4 * sz : nullptr;
    long long Qs = 1;
    for (int l = 1; l <= d; ++l) Qs *= Q[l];
    const bool uw = h->formulation == STST_FORM_UW;  // ultraweak: plain load int f conj(B_i)
    if (!uw) STST_TRY(contract(h, 0, (const double2 *)f_qp, T1, 1, Qs, 1, 0.0, -1.0, 0));
    STST_TRY(contract(h, 0, (const double2 *)f_qp, T0, 1, Qs, 0, 1.0, 0.0, 0));
    struct Term { double2 *src; int der[STST_MAXD + 1]; double s; };
    std::vector<Term> terms;
    if (uw) {
      Term t0 = {T0, {0, 0, 0, 0}, 1.0};
      terms.push_back(t0);
    } else {
      Term t1 = {T1, {0, 0, 0, 0}, 1.0};
      terms.push_back(t1);
      for (int l = 1; l <= d; ++l) {
        Term t = {T0, {0, 0, 0, 0}, -h->nu};
        t.der[l] = 2;
        terms.push_back(t);
      }
    }
    if (T0V && !uw) {
      const DirInfo &D = h->dir[0];
      long long tot = Qs * D.n;
      k_contract_time_pot<<<grid_for(tot, 128), 128, 0, st>>>((const double2 *)f_qp, T0V, h->tab[0], h->qwts[0], D.p,
                                                               D.nq, D.n_el, D.off, D.n, D.Q(), Qs, d, Q[1],
                                                               d >= 2 ? Q[2] : 1, d >= 3 ? Q[3] : 1, h->pot_rank,
                                                               h->pot_bufs[0]);
      STST_CUDA(cudaGetLastError());
      Term tv = {T0V, {0, 0, 0, 0}, 1.0};
      terms.push_back(tv);
    }
    for (const Term &t : terms) {
      const double2 *src = t.src;
      long long ext[STST_MAXD + 1];
      ext[0] = n[0];
      for (int l = 1; l <= d; ++l) ext[l] = Q[l];
      double2 *bufs[2] = {W1, W2};
      int cur = 0;
      for (int l = 1; l <= d; ++l) {
        long long inner = 1, outer = 1;
        for (int k = 0; k < l; ++k) inner *= ext[k];
        for (int k = l + 1; k <= d; ++k) outer *= ext[k];
        bool last = (l == d);
        double2 *dst = last ? (double2 *)rhs : bufs[cur];
        STST_TRY(contract(h, l, src, dst, inner, outer, t.der[l], last ? t.s : 1.0, 0.0, last ? 1 : 0));
        ext[l] = n[l];
        src = dst;
        cur ^= 1;
      }
    }
  }
  if (u0_qp) {
    // the initial datum uses the handle's projection workspace (allocated by stst_create)
    double2 *W1 = (double2 *)h->proj_work;
    double2 *W2 = W1 + h->proj_work_bytes / sizeof(double2) / 3;
    double2 *C = W2 + h->proj_work_bytes / sizeof(double2) / 3;
    long long ext[STST_MAXD + 1];
    for (int l = 1; l <= d; ++l) ext[l] = Q[l];
    const double2 *src = (const double2 *)u0_qp;
    double2 *bufs[2] = {W1, W2};
    int cur = 0;
    for (int l = 1; l <= d; ++l) {
      long long inner = 1, outer = 1;
      for (int k = 1; k < l; ++k) inner *= ext[k];
      for (int k = l + 1; k <= d; ++k) outer *= ext[k];
      double2 *dst = (l == d) ? C : bufs[cur];
      STST_TRY(contract(h, l, src, dst, inner, outer, 0, 1.0, 0.0, 0));
      ext[l] = n[l];
      src = dst;
      cur ^= 1;
    }
    if (h->formulation == STST_FORM_UW) {  // rhs += i (u0, B_j) on time index 0
      k_add_initial_uw<<<grid_for(h->N_s, 256), 256, 0, st>>>((double2 *)rhs, C, n[0], h->N_s);
      STST_CUDA(cudaGetLastError());
    }
    for (int l = 1; l <= d; ++l) {
      long long inner = 1, outer = 1;
      for (int k = 1; k < l; ++k) inner *= n[k];
      for (int k = l + 1; k <= d; ++k) outer *= n[k];
      k_mass_solve<<<grid_for(inner * outer, 128), 128, 0, st>>>(C, h->mchol[l], n[l], h->dir[l].p, inner, outer);
      STST_CUDA(cudaGetLastError());
    }
    if (c0) STST_CUDA(cudaMemcpyAsync(c0, C, sizeof(double2) * h->N_s, cudaMemcpyDeviceToDevice, st));
    if (h->formulation == STST_FORM_LS)
      STST_TRY(run_plan(h->lift_plan, C, rhs, 0, 1, rhs, nullptr, nullptr, nullptr, st));
  } else if (c0) {
    STST_CUDA(cudaMemsetAsync(c0, 0, sizeof(double2) * h->N_s, st));
  }
  return STST_OK;
}
