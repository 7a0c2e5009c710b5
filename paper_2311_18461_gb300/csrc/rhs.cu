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
// Right-hand side with general Dirichlet and initial data (the lifting of Sec. 2.2, with the data taken
// from a function u given on the whole space-time cylinder, as in the experiments of Sec. 6):
//   G = (M_t^{-1} x M_1^{-1} x ... x M_d^{-1}) (u, B)   the L2 projection of u onto the full tensor
//       spline space (all basis functions, no boundary conditions);
//   g_h keeps the coefficients of G on the basis functions that do not vanish at t = 0 or on the
//       spatial boundary (time index 0, spatial indices 0 and m_l - 1), zero elsewhere;
//   rhs_i = (f - S_V g_h, S_V B_i), i.e. the load of f minus the method's bilinear form between the
//       lifting and the test functions.
// S_V g_h is evaluated at the tensor Gauss points of the load and integrated by the load's own rule,
// which is exact for these piecewise polynomials (the potential uses that rule in the system matrices
// too), so the result equals the load minus the full-basis Kronecker operator applied to g_h.
// ------------------------------------------------------------------------------------------------

// out[o, q, c] = (sre + i sim) sum_{a = 0..p} d^der b_{e(q)+a}(x_q) in[o, e(q)+a, c]  (+ out if accumulate);
// the input runs over all m = n_el + p basis functions of the mode, the output over its Q points.
__global__ void k_eval_mode(const double2 *__restrict__ in, double2 *__restrict__ out, const double *__restrict__ tab,
                            int p, int nq, int m, int Q, long long inner, long long outer, int der, double sre,
                            double sim, int accumulate) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= outer * Q * inner) return;
  const long long c = idx % inner;
  const long long t = idx / inner;
  const int q = (int)(t % Q);
  const long long o = t / Q;
  const int e = q / nq;
  double ax = 0.0, ay = 0.0;
  for (int a = 0; a <= p; ++a) {
    const double b = tab[((long long)q * (p + 1) + a) * 3 + der];
    const double2 v = in[(o * m + e + a) * inner + c];
    ax += b * v.x;
    ay += b * v.y;
  }
  double rx = sre * ax - sim * ay, ry = sre * ay + sim * ax;
  if (accumulate) {
    const double2 prev = out[idx];
    rx += prev.x;
    ry += prev.y;
  }
  out[idx] = make_double2(rx, ry);
}

// keep the coefficients of the basis functions that are nonzero at t = 0 or on the spatial boundary
__global__ void k_mask_lift(double2 *__restrict__ G, int d, int m0, int m1, int m2, int m3, long long total) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= total) return;
  long long r = idx;
  const int it = (int)(r % m0);
  r /= m0;
  bool keep = it == 0;
  const int ms[3] = {m1, m2, m3};
  for (int l = 0; l < d; ++l) {
    const int i = (int)(r % ms[l]);
    r /= ms[l];
    keep = keep || i == 0 || i == ms[l] - 1;
  }
  if (!keep) G[idx] = make_double2(0.0, 0.0);
}

// out += s a
__global__ void k_axpy_c(double2 *__restrict__ out, const double2 *__restrict__ a, double s, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double2 o = out[i];
  const double2 v = a[i];
  o.x += s * v.x;
  o.y += s * v.y;
  out[i] = o;
}

int rhs_lift_compute(stst_problem *h, const double *f_qp, const double *u_qp, double *rhs, double *xd) {
  if (h->formulation != STST_FORM_LS || !u_qp || !rhs) return STST_ERR_ARG;
  cudaStream_t st = h->stream;
  const int d = h->d;
  int Q[STST_MAXD + 1], m[STST_MAXD + 1];
  long long Qtot = 1, Mtot = 1;
  for (int l = 0; l <= d; ++l) {
    Q[l] = h->dir[l].Q();
    m[l] = h->dir[l].m;
    Qtot *= Q[l];
    Mtot *= m[l];
  }
  // every intermediate tensor has at most Qtot entries (m_l <= Q_l: at least p + 1 points per element)
  std::vector<void *> owned;
  auto get = [&](void **ptr, size_t bytes) -> int {
    cudaError_t e = cudaMallocAsync(ptr, bytes, st);
    if (e != cudaSuccess) {
      stst_last_cuda = e;
      return STST_ERR_OOM;
    }
    owned.push_back(*ptr);
    return STST_OK;
  };
  auto release = [&]() {
    for (void *q : owned) cudaFreeAsync(q, st);
  };
  int status = STST_OK;
  do {
    double2 *A, *B, *G, *SG;
    if ((status = get((void **)&A, sizeof(double2) * Qtot)) != STST_OK) break;
    if ((status = get((void **)&B, sizeof(double2) * Qtot)) != STST_OK) break;
    if ((status = get((void **)&G, sizeof(double2) * Mtot)) != STST_OK) break;
    if ((status = get((void **)&SG, sizeof(double2) * Qtot)) != STST_OK) break;
    double *Mf[STST_MAXD + 1], *Cf[STST_MAXD + 1];
    for (int l = 0; l <= d && status == STST_OK; ++l) {
      const DirInfo &D = h->dir[l];
      if ((status = get((void **)&Mf[l], sizeof(double) * D.m * (2 * D.p + 1))) != STST_OK) break;
      if ((status = get((void **)&Cf[l], sizeof(double) * D.m * (D.p + 1))) != STST_OK) break;
      if ((status = launch_assemble_band(MK_M, D.p, D.n_el, D.len, D.nq, 0, D.m, D.m, nullptr, Mf[l], st)) != STST_OK)
        break;
      BandMat bm;
      bm.d = Mf[l];
      bm.n = D.m;
      bm.p = D.p;
      status = launch_mass_cholesky(bm, Cf[l], h->flags, st);
    }
    if (status != STST_OK) break;
    // (u, B) over all basis functions, mode by mode
    long long ext[STST_MAXD + 1];
    for (int l = 0; l <= d; ++l) ext[l] = Q[l];
    const double2 *src = (const double2 *)u_qp;
    double2 *bufs[2] = {A, B};
    int cur = 0;
    for (int l = 0; l <= d && status == STST_OK; ++l) {
      long long inner = 1, outer = 1;
      for (int k = 0; k < l; ++k) inner *= ext[k];
      for (int k = l + 1; k <= d; ++k) outer *= ext[k];
      double2 *dst = (l == d) ? G : bufs[cur];
      const DirInfo &D = h->dir[l];
      const long long total = outer * D.m * inner;
      k_contract<double2><<<grid_for(total, 128), 128, 0, st>>>(src, dst, h->tab[l], h->qwts[l], D.p, D.nq, D.n_el,
                                                                 0, D.m, D.Q(), inner, outer, 0, 1.0, 0.0, 0);
      if (cudaGetLastError() != cudaSuccess) status = STST_ERR_CUDA;
      ext[l] = D.m;
      src = dst;
      cur ^= 1;
    }
    if (status != STST_OK) break;
    // G = M^{-1} (u, B) with the full mass matrix of every direction
    for (int l = 0; l <= d; ++l) {
      long long inner = 1, outer = 1;
      for (int k = 0; k < l; ++k) inner *= m[k];
      for (int k = l + 1; k <= d; ++k) outer *= m[k];
      k_mass_solve<<<grid_for(inner * outer, 128), 128, 0, st>>>(G, Cf[l], m[l], h->dir[l].p, inner, outer);
    }
    k_mask_lift<<<grid_for(Mtot, 256), 256, 0, st>>>(G, d, m[0], d >= 1 ? m[1] : 1, d >= 2 ? m[2] : 1,
                                                     d >= 3 ? m[3] : 1, Mtot);
    if (cudaGetLastError() != cudaSuccess) {
      status = STST_ERR_CUDA;
      break;
    }
    if (xd) {
      const cudaError_t e = cudaMemcpyAsync(xd, G, sizeof(double2) * Mtot, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) {
        stst_last_cuda = e;
        status = STST_ERR_CUDA;
        break;
      }
    }
    // SG = -S_V g_h at the quadrature points: -i d_t g + nu sum_l d_l^2 g - V g
    struct EvalTerm { int der[STST_MAXD + 1]; double sre, sim; bool pot; };
    std::vector<EvalTerm> terms;
    terms.push_back({{1, 0, 0, 0}, 0.0, -1.0, false});
    for (int l = 1; l <= d; ++l) {
      EvalTerm t = {{0, 0, 0, 0}, h->nu, 0.0, false};
      t.der[l] = 2;
      terms.push_back(t);
    }
    if (h->pot_rank > 0) terms.push_back({{0, 0, 0, 0}, 1.0, 0.0, true});
    for (size_t k = 0; k < terms.size() && status == STST_OK; ++k) {
      const EvalTerm &t = terms[k];
      for (int l = 0; l <= d; ++l) ext[l] = m[l];
      const double2 *s2 = G;
      int c2 = 0;
      for (int l = 0; l <= d && status == STST_OK; ++l) {
        long long inner = 1, outer = 1;
        for (int j = 0; j < l; ++j) inner *= ext[j];
        for (int j = l + 1; j <= d; ++j) outer *= ext[j];
        const bool last = l == d;
        double2 *dst = (last && !t.pot) ? SG : bufs[c2];
        const DirInfo &D = h->dir[l];
        const long long total = outer * D.Q() * inner;
        k_eval_mode<<<grid_for(total, 128), 128, 0, st>>>(s2, dst, h->tab[l], D.p, D.nq, D.m, D.Q(), inner, outer,
                                                          t.der[l], last ? t.sre : 1.0, last ? t.sim : 0.0,
                                                          (last && !t.pot && k > 0) ? 1 : 0);
        if (cudaGetLastError() != cudaSuccess) status = STST_ERR_CUDA;
        ext[l] = D.Q();
        s2 = dst;
        c2 ^= 1;
      }
      if (t.pot && status == STST_OK) {  // SG -= V g_h
        double2 *E0 = (double2 *)s2, *FV = bufs[c2];
        k_mul_potential<<<grid_for(Qtot, 256), 256, 0, st>>>(E0, FV, Q[0], d, Q[1], d >= 2 ? Q[2] : 1,
                                                              d >= 3 ? Q[3] : 1, h->pot_rank, h->pot_bufs[0], Qtot);
        k_axpy_c<<<grid_for(Qtot, 256), 256, 0, st>>>(SG, FV, -1.0, Qtot);
        if (cudaGetLastError() != cudaSuccess) status = STST_ERR_CUDA;
      }
    }
    if (status != STST_OK) break;
    if (f_qp) {
      k_axpy_c<<<grid_for(Qtot, 256), 256, 0, st>>>(SG, (const double2 *)f_qp, 1.0, Qtot);
      if (cudaGetLastError() != cudaSuccess) {
        status = STST_ERR_CUDA;
        break;
      }
    }
    status = rhs_compute(h, (const double *)SG, nullptr, rhs, nullptr);
  } while (false);
  release();
  return status;
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

// Device address of g_rhs_scratch, looked up once per device with that device current. The lookup is
// keyed on the device's current context as well: a device reset (cudaDeviceReset) ends the context and
// the module is loaded again in the next one, possibly at another address, so a new context id makes
// the lookup run again.
typedef int (*CtxGetIdFn)(void *ctx, unsigned long long *id);

static unsigned long long current_context_id() {
  static CtxGetIdFn fn = nullptr;
  static bool looked = false;
  if (!looked) {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (CtxGetIdFn)f;
    looked = true;
  }
  unsigned long long id = 0;
  if (!fn || fn(nullptr, &id) != 0) return 0;  // 0: unknown (no entry point, or no current context yet)
  return id;
}

static int rhs_scratch_address(double2 **out) {
  static std::mutex mu;
  static double2 *addr[256];
  static unsigned long long ctx[256];
  static bool ready[256];
  int dev = 0;
  STST_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return STST_ERR_ARG;
  std::lock_guard<std::mutex> lock(mu);
  const unsigned long long id = current_context_id();
  if (!ready[dev] || id == 0 || id != ctx[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_rhs_scratch);
    if (e != cudaSuccess || p == nullptr) {
      stst_last_cuda = e;
      return STST_ERR_CUDA;
    }
    addr[dev] = (double2 *)p;
    ctx[dev] = id ? id : current_context_id();  // the lookup above has made the primary context current
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
  if (h->geo) return STST_ERR_STATE;  // parametric integrals (as stst_rhs)
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
  // slices of the scratch in the order they are needed: T0, W1, W2 for every load; T1 for the
  // least-squares load; T0V for the least-squares load with a potential (the ultraweak load has no V term)
  const bool uw = h->formulation == STST_FORM_UW;  // ultraweak: plain load int f conj(B_i)
  const long long need = (uw ? 3 : (h->pot_rank > 0 ? 5 : 4)) * sz;
  if (f_qp && need > STST_RHS_SCRATCH_ELEMS) return STST_ERR_ARG;  // forcing grid too large for the static scratch
  STST_CUDA(cudaMemsetAsync(rhs, 0, sizeof(double2) * h->N_dof, st));
  if (f_qp) {
    double2 *T0 = scratch, *W1 = scratch + sz, *W2 = scratch + 2 * sz;
    double2 *T1 = uw ? nullptr : scratch + 3 * sz;
    double2 *T0V = (h->pot_rank > 0 && !uw) ? scratch + 4 * sz : nullptr;
    long long Qs = 1;
    for (int l = 1; l <= d; ++l) Qs *= Q[l];
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
    if (T0V) {
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
