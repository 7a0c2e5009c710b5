// The least-squares system on a mapped domain Omega = F((0,1)^d) (Sec. 3.2, Eq. syst_mat, Eq. space_mat).
//
// With the push-forward basis B_i = B-hat_i o F^{-1} the system keeps the form of Eq. syst_mat,
//     A = M_s (x) L_t + nu^2 B_s (x) M_t + nu L_s (x) (W_t + W_t^*),
// with the parametric time matrices, but M_s, L_s, B_s are integrals over the physical domain and do not split
// into one-direction factors. Pulled back to the parametric box (J = dF/d eta, G = J^{-1} J^{-T}):
//     M_s[i,j] = int |det J| B-hat_i B-hat_j,   L_s[i,j] = int |det J| grad B-hat_i^T G grad B-hat_j,
//     B_s[i,j] = int |det J| (Delta B_i)(Delta B_j),
//     Delta u = sum_ab G^{ab} d_a d_b u-hat + sum_a h^a d_a u-hat,  h^a = - sum_m (J^{-1})_{am} sum_bc F_{m,bc} G^{bc}.
// The caller gives J and the second derivatives of F at the spatial quadrature points (the tensor grid of the
// directions' points, p + 2 Gauss points per element, direction 1 fastest). Setup (stst_set_geometry):
//   k_geo_metric   per point: |det J| times the quadrature weight, G, h (and a check that det J keeps one sign);
//   k_geo_assemble per stored entry (row i, offset o in [-p, p]^d): the three quadrature sums over the
//                  elements the two basis functions share, from the one-direction basis tables;
// the matrices are kept as stencils S_k[i][o], k = 0: M_s, 1: nu^2 B_s, 2: nu L_s ((2p+1)^d entries per row).
// Mat-vec (run_geo, in place of the sum-factorised plan): the time bands first, z_k = T_k x along t for the
// three time matrices (L_t, M_t, i (K - K^T) = W_t + W_t^*), then y[i, t] = sum_k sum_o S_k[i][o] z_k[i + o, t]
// with the plan's epilogue (b - A x, the dot-product partials of the PCG). The parametric P-hat stays the
// preconditioner (the paper's fast solver is for F = id only, Sec. 5). FP64 only; no potential.
#include "common.cuh"
#include <vector>

#define GEO_MAXW 729  // stored entries per row: (2p+1)^d <= 729 (d = 3 with p <= 4, d = 2 with p <= 13)

struct GeoOp {
  int d;
  int p[STST_MAXD + 1], n[STST_MAXD + 1], nel[STST_MAXD + 1], nq[STST_MAXD + 1], Q[STST_MAXD + 1];
  int W;            // stored entries per row
  long long N_s, N_qs;
  int n_t, p_t;
  double scale[STST_MAXD + 1];  // P-hat's eigenvalue scales s_l = int |det J| G^{ll} / int |det J|
  double *S;        // 3 x N_s x W
  double2 *z;       // 3 x N_dof: the time-band products
  const double *Lt, *Mt, *KAt;  // time bands (n_t x (2 p_t + 1)), reduced
};

namespace {

constexpr int NCOEF = 16;  // per point: wdet, G (6), h (3), K = wdet G (6)

__device__ __forceinline__ int sym_index(int a, int b, int d) {
  // packed upper triangle of a symmetric d x d matrix, row-major: (0,0) (0,1) .. (0,d-1) (1,1) ..
  if (a > b) {
    const int t = a;
    a = b;
    b = t;
  }
  return a * d - a * (a - 1) / 2 + (b - a);
}

__global__ void k_geo_metric(int d, long long N_qs, const int *Qd, const double *w1, const double *w2,
                             const double *w3, const double *__restrict__ jac, const double *__restrict__ hess,
                             double *coef, int *flags) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= N_qs) return;
  // the point's 1D indices (direction 1 fastest) and weight
  long long r = q;
  double w = 1.0;
  const double *ws[3] = {w1, w2, w3};
  for (int l = 0; l < d; ++l) {
    const int ql = (int)(r % Qd[l]);
    r /= Qd[l];
    w *= ws[l][ql];
  }
  double J[3][3], Ji[3][3];
  for (int m = 0; m < d; ++m)
    for (int a = 0; a < d; ++a) J[m][a] = jac[(q * d + m) * d + a];
  double det;
  if (d == 1) {
    det = J[0][0];
    Ji[0][0] = 1.0 / det;
  } else if (d == 2) {
    det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    Ji[0][0] = J[1][1] / det;
    Ji[0][1] = -J[0][1] / det;
    Ji[1][0] = -J[1][0] / det;
    Ji[1][1] = J[0][0] / det;
  } else {
    // inverse by cofactors: Ji[a][m] = C[m][a] / det
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1], c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2],
                 c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const double c10 = J[0][2] * J[2][1] - J[0][1] * J[2][2], c11 = J[0][0] * J[2][2] - J[0][2] * J[2][0],
                 c12 = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    const double c20 = J[0][1] * J[1][2] - J[0][2] * J[1][1], c21 = J[0][2] * J[1][0] - J[0][0] * J[1][2],
                 c22 = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    Ji[0][0] = c00 / det, Ji[0][1] = c10 / det, Ji[0][2] = c20 / det;
    Ji[1][0] = c01 / det, Ji[1][1] = c11 / det, Ji[1][2] = c21 / det;
    Ji[2][0] = c02 / det, Ji[2][1] = c12 / det, Ji[2][2] = c22 / det;
  }
  if (!(fabs(det) > 1e-300) || !isfinite(det)) atomicOr(flags, 1);
  atomicOr(flags, det > 0.0 ? 2 : 4);  // both bits: the map folds (det J changes sign)
  // G = Ji Ji^T; tr_m = sum_bc H[m][b][c] G[b][c]; h_a = - sum_m Ji[a][m] tr_m
  double G[3][3];
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) {
      double s = 0.0;
      for (int k = 0; k < d; ++k) s += Ji[a][k] * Ji[b][k];
      G[a][b] = s;
    }
  double tr[3];
  for (int m = 0; m < d; ++m) {
    double s = 0.0;
    for (int b = 0; b < d; ++b)
      for (int c = 0; c < d; ++c) s += hess[((q * d + m) * d + b) * d + c] * G[b][c];
    tr[m] = s;
  }
  double *out = coef + q * NCOEF;
  const double wdet = w * fabs(det);
  out[0] = wdet;
  for (int a = 0; a < d; ++a) {
    double s = 0.0;
    for (int m = 0; m < d; ++m) s -= Ji[a][m] * tr[m];
    out[7 + a] = s;
    for (int b = a; b < d; ++b) {
      const int k = sym_index(a, b, d);
      out[1 + k] = G[a][b];
      out[10 + k] = wdet * G[a][b];
    }
  }
}

struct AsmArgs {
  int d, p[3], n[3], nel[3], nq[3], Q[3], W;
  long long N_s;
  const double *tab[3];  // per direction: Q x (p+1) x 3 (value, first, second derivative of functions e..e+p)
  const double *coef;
  double *S;             // 3 x N_s x W
};

// One thread per stored entry (row i, offset o): M, B, L by quadrature over the shared elements
__global__ void k_geo_assemble(const AsmArgs A) {
  const long long e_id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e_id >= A.N_s * A.W) return;
  const int d = A.d;
  const long long row = e_id / A.W;
  const int o = (int)(e_id - row * A.W);
  int il[3], jl[3], lo[3], cnt[3];
  bool valid = true;
  {
    long long r = row;
    int oo = o;
    for (int l = 0; l < d; ++l) {
      il[l] = (int)(r % A.n[l]);
      r /= A.n[l];
      const int w = 2 * A.p[l] + 1;
      jl[l] = il[l] + (oo % w) - A.p[l];
      oo /= w;
      if (jl[l] < 0 || jl[l] >= A.n[l]) valid = false;
    }
  }
  double sm = 0.0, sb = 0.0, sl = 0.0;
  if (valid) {
    // full indices f = i + 1, g = j + 1; shared elements e in [max(f,g) - p, min(f,g)] within the mesh
    long long total = 1;
    for (int l = 0; l < d; ++l) {
      const int f = il[l] + 1, g = jl[l] + 1;
      int e0 = max(f, g) - A.p[l], e1 = min(f, g);
      if (e0 < 0) e0 = 0;
      if (e1 > A.nel[l] - 1) e1 = A.nel[l] - 1;
      lo[l] = e0 * A.nq[l];
      cnt[l] = (e1 - e0 + 1) * A.nq[l];
      if (cnt[l] <= 0) total = 0;
      total *= cnt[l] > 0 ? cnt[l] : 0;
    }
    for (long long t = 0; t < total; ++t) {
      // the point: 1D indices (direction 1 fastest within the shared box), element, function slots
      long long r = t;
      double vi[3][3], vj[3][3];  // [direction][derivative order]
      long long q = 0, stride = 1;
      for (int l = 0; l < d; ++l) {
        const int ql = lo[l] + (int)(r % cnt[l]);
        r /= cnt[l];
        q += ql * stride;
        stride *= A.Q[l];
        const int e = ql / A.nq[l];
        const int pp1 = A.p[l] + 1;
        const double *ti = A.tab[l] + ((long long)ql * pp1 + (il[l] + 1 - e)) * 3;
        const double *tj = A.tab[l] + ((long long)ql * pp1 + (jl[l] + 1 - e)) * 3;
        for (int s = 0; s < 3; ++s) {
          vi[l][s] = ti[s];
          vj[l][s] = tj[s];
        }
      }
      const double *c = A.coef + q * NCOEF;
      // values, first and second derivatives of the two tensor-product functions
      double fi = 1.0, fj = 1.0, di[3], dj[3], ddi[6], ddj[6];
      for (int l = 0; l < d; ++l) {
        fi *= vi[l][0];
        fj *= vj[l][0];
      }
      for (int a = 0; a < d; ++a) {
        double pi = 1.0, pj = 1.0;
        for (int l = 0; l < d; ++l) {
          pi *= vi[l][l == a ? 1 : 0];
          pj *= vj[l][l == a ? 1 : 0];
        }
        di[a] = pi;
        dj[a] = pj;
        for (int b = a; b < d; ++b) {
          double qi = 1.0, qj = 1.0;
          for (int l = 0; l < d; ++l) {
            const int ord = (l == a) + (l == b);
            qi *= vi[l][ord];
            qj *= vj[l][ord];
          }
          ddi[sym_index(a, b, d)] = qi;
          ddj[sym_index(a, b, d)] = qj;
        }
      }
      const double wdet = c[0];
      sm += wdet * fi * fj;
      double lapi = 0.0, lapj = 0.0, gl = 0.0;
      for (int a = 0; a < d; ++a) {
        lapi += c[7 + a] * di[a];
        lapj += c[7 + a] * dj[a];
        for (int b = 0; b < d; ++b) {
          const int k = sym_index(a, b, d);
          lapi += c[1 + k] * ddi[k];
          lapj += c[1 + k] * ddj[k];
          gl += c[10 + k] * di[a] * dj[b];
        }
      }
      sb += wdet * lapi * lapj;
      sl += gl;
    }
  }
  A.S[e_id] = sm;
  A.S[A.N_s * A.W + e_id] = sb;
  A.S[2 * A.N_s * A.W + e_id] = sl;
}

// sums over the points of |det J| w and of |det J| w G^{ll} (one CTA; setup only)
__global__ void k_geo_means(const double *__restrict__ coef, long long N_qs, int d, double *out) {
  __shared__ double sh[32];
  for (int c = 0; c <= d; ++c) {
    const int k = c == 0 ? 0 : 10 + sym_index(c - 1, c - 1, d);
    double s = 0.0;
    for (long long q = threadIdx.x; q < N_qs; q += blockDim.x) s += coef[q * NCOEF + k];
    s = epi_block_sum(s, sh);
    if (threadIdx.x == 0) out[c] = s;
    __syncthreads();
  }
}

__global__ void k_geo_scale(double *S, long long n, double c) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) S[i] *= c;
}

// z_k[j, t] = sum_t' T_k[t][t'] x[j, t'] for the three time bands (k = 2 multiplied by i)
__global__ void k_geo_time(const double2 *__restrict__ x, double2 *__restrict__ z, const double *__restrict__ Lt,
                           const double *__restrict__ Mt, const double *__restrict__ KAt, int n_t, int p_t,
                           long long N, const int *done) {
  if (done && *done) return;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= N) return;
  const long long j = idx / n_t;
  const int t = (int)(idx - j * n_t);
  const int bw = 2 * p_t + 1;
  double2 a0 = make_double2(0.0, 0.0), a1 = a0, a2 = a0;
  for (int k = -p_t; k <= p_t; ++k) {
    const int tt = t + k;
    if (tt < 0 || tt >= n_t) continue;
    const double2 v = x[j * n_t + tt];
    const int off = t * bw + k + p_t;
    const double l = Lt[off], m = Mt[off], ka = KAt[off];
    a0.x += l * v.x;
    a0.y += l * v.y;
    a1.x += m * v.x;
    a1.y += m * v.y;
    a2.x -= ka * v.y;  // i (KA v)
    a2.y += ka * v.x;
  }
  z[idx] = a0;
  z[N + idx] = a1;
  z[2 * N + idx] = a2;
}

struct SpaceArgs {
  int d, p[3], n[3], W, n_t;
  long long N_s, N;
  const double *S;
  const double2 *z;
  double2 *y;
  int epi;
  const double2 *b, *dotvec;
  double *dot_partials, *dot2_partials;
  const int *done;
};

// y[i, t] = sum_k sum_o S_k[i][o] z_k[i + o, t] over the neighbours inside the mesh, with the plan's epilogue
__global__ void __launch_bounds__(256) k_geo_space(const __grid_constant__ SpaceArgs A) {
  if (A.done && *A.done) return;
  __shared__ double sh[32];
  double dacc = 0.0, d2acc = 0.0;
  const int d = A.d;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < A.N;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long i = idx / A.n_t;
    const int t = (int)(idx - i * A.n_t);
    int il[3] = {0, 0, 0}, a0[3] = {0, 0, 0}, a1[3] = {0, 0, 0};
    long long stride[3] = {1, 1, 1};
    {
      long long r = i, s = 1;
      for (int l = 0; l < d; ++l) {
        il[l] = (int)(r % A.n[l]);
        r /= A.n[l];
        stride[l] = s;
        s *= A.n[l];
        a0[l] = max(-A.p[l], -il[l]);
        a1[l] = min(A.p[l], A.n[l] - 1 - il[l]);
      }
    }
    const int w0 = 2 * A.p[0] + 1, w1 = d > 1 ? 2 * A.p[1] + 1 : 1;
    double yx = 0.0, yy = 0.0;
    const double *S0 = A.S + i * A.W, *S1 = S0 + A.N_s * A.W, *S2 = S1 + A.N_s * A.W;
    const long long N = A.N;
    for (int o3 = (d > 2 ? a0[2] : 0); o3 <= (d > 2 ? a1[2] : 0); ++o3)
      for (int o2 = (d > 1 ? a0[1] : 0); o2 <= (d > 1 ? a1[1] : 0); ++o2)
        for (int o1 = a0[0]; o1 <= a1[0]; ++o1) {
          const int o = (o1 + A.p[0]) + w0 * ((d > 1 ? o2 + A.p[1] : 0) + w1 * (d > 2 ? o3 + A.p[2] : 0));
          const long long jz = (i + o1 + o2 * stride[1] + o3 * stride[2]) * A.n_t + t;
          const double2 z0 = A.z[jz], z1 = A.z[N + jz], z2 = A.z[2 * N + jz];
          const double s0 = S0[o], s1 = S1[o], s2 = S2[o];
          yx += s0 * z0.x + s1 * z1.x + s2 * z2.x;
          yy += s0 * z0.y + s1 * z1.y + s2 * z2.y;
        }
    if (A.epi == 1) {
      const double2 bv = A.b[idx];
      yx = bv.x - yx;
      yy = bv.y - yy;
    }
    A.y[idx] = make_double2(yx, yy);
    if (A.dotvec) {
      const double2 dv = A.dotvec[idx];
      dacc += dv.x * yx + dv.y * yy;  // Re(conj(d) y)
    }
    if (A.dot2_partials) d2acc += yx * yx + yy * yy;
  }
  if (A.dot_partials) {
    const double s = epi_block_sum(dacc, sh);
    if (threadIdx.x == 0) A.dot_partials[blockIdx.x] = s;
  }
  if (A.dot2_partials) {
    const double s = epi_block_sum(d2acc, sh);
    if (threadIdx.x == 0) A.dot2_partials[blockIdx.x] = s;
  }
}

}  // namespace

int reduction_grid(long long total);

int run_geo(const GeoOp &g, const void *x, void *y, int precision, int epi, const void *b, const void *dotvec,
            double *dot_partials, const int *done, cudaStream_t s, double *dot2_partials) {
  if (precision != 0) return STST_ERR_STATE;  // the mapped-domain operator is FP64 only
  const long long N = g.N_s * g.n_t;
  {
    STST_PROF("geo_time_f64", s);
    k_geo_time<<<grid_for(N, 256), 256, 0, s>>>((const double2 *)x, g.z, g.Lt, g.Mt, g.KAt, g.n_t, g.p_t, N, done);
    STST_CUDA(cudaGetLastError());
  }
  SpaceArgs A;
  A.d = g.d;
  for (int l = 0; l < 3; ++l) {
    A.p[l] = l < g.d ? g.p[l + 1] : 0;
    A.n[l] = l < g.d ? g.n[l + 1] : 1;
  }
  A.W = g.W;
  A.n_t = g.n_t;
  A.N_s = g.N_s;
  A.N = N;
  A.S = g.S;
  A.z = g.z;
  A.y = (double2 *)y;
  A.epi = epi;
  A.b = (const double2 *)b;
  A.dotvec = (const double2 *)dotvec;
  A.dot_partials = dot_partials;
  A.dot2_partials = dot2_partials;
  A.done = done;
  STST_PROF("geo_space_f64", s);
  k_geo_space<<<reduction_grid(N), 256, 0, s>>>(A);
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}

void free_geo(GeoOp *g) {
  if (!g) return;
  cudaFree(g->S);
  cudaFree(g->z);
  delete g;
}

void invalidate_solver_graphs(stst_problem *h);

extern "C" int stst_set_geometry(stst_handle h, const double *jac, const double *hess) {
  if (!h || h->magic != STST_MAGIC) return STST_ERR_HANDLE;
  ApiScope scope(h);
  if (!jac) {  // back to the parametric operator
    STST_CUDA(cudaStreamSynchronize(h->stream));
    free_geo(h->geo);
    h->geo = nullptr;
    h->sys_plan.geo = nullptr;
    h->fd_ready = 0;
    invalidate_solver_graphs(h);
    return STST_OK;
  }
  if (!hess) return STST_ERR_ARG;
  if (h->pot_rank > 0 || h->formulation != STST_FORM_LS) return STST_ERR_STATE;
  const int d = h->d;
  int W = 1;
  for (int l = 1; l <= d; ++l) W *= 2 * h->dir[l].p + 1;
  if (W > GEO_MAXW) return STST_ERR_ARG;
  cudaStream_t st = h->stream;
  GeoOp *g = new (std::nothrow) GeoOp();
  if (!g) return STST_ERR_OOM;
  g->d = d;
  g->W = W;
  g->N_s = h->N_s;
  g->N_qs = 1;
  for (int l = 1; l <= d; ++l) {
    g->p[l] = h->dir[l].p;
    g->n[l] = h->dir[l].n;
    g->nel[l] = h->dir[l].n_el;
    g->nq[l] = h->dir[l].nq;
    g->Q[l] = h->dir[l].Q();
    g->N_qs *= g->Q[l];
  }
  g->n_t = h->dir[0].n;
  g->p_t = h->dir[0].p;
  g->Lt = h->mats[0][0].d;
  g->Mt = h->mats[0][1].d;
  g->KAt = h->mats[0][2].d;
  double *coef = nullptr;
  int *dflags = nullptr, *dQ = nullptr;
  auto fail = [&](int s) {
    cudaFree(coef);
    cudaFree(dflags);
    cudaFree(dQ);
    free_geo(g);
    return s;
  };
  double *dmeans = nullptr;
  if (cudaMalloc(&g->S, sizeof(double) * 3 * (size_t)g->N_s * W) != cudaSuccess ||
      cudaMalloc(&g->z, sizeof(double2) * 3 * (size_t)h->N_dof) != cudaSuccess ||
      cudaMalloc(&coef, sizeof(double) * NCOEF * (size_t)g->N_qs) != cudaSuccess ||
      cudaMalloc(&dflags, sizeof(int)) != cudaSuccess || cudaMalloc(&dQ, sizeof(int) * 3) != cudaSuccess ||
      cudaMalloc(&dmeans, sizeof(double) * (STST_MAXD + 1)) != cudaSuccess) {
    cudaFree(dmeans);
    return fail(STST_ERR_OOM);
  }
  int hQ[3] = {g->Q[1], d > 1 ? g->Q[2] : 1, d > 2 ? g->Q[3] : 1};
  if (cudaMemcpyAsync(dQ, hQ, sizeof(hQ), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(dflags, 0, sizeof(int), st) != cudaSuccess)
    return fail(STST_ERR_CUDA);
  {
    STST_PROF("geo_metric", st);
    k_geo_metric<<<grid_for(g->N_qs, 128), 128, 0, st>>>(d, g->N_qs, dQ, h->qwts[1], d > 1 ? h->qwts[2] : nullptr,
                                                          d > 2 ? h->qwts[3] : nullptr, jac, hess, coef, dflags);
  }
  if (cudaGetLastError() != cudaSuccess) return fail(STST_ERR_CUDA);
  AsmArgs A;
  A.d = d;
  A.W = W;
  A.N_s = g->N_s;
  for (int l = 0; l < 3; ++l) {
    const int L = l + 1;
    A.p[l] = l < d ? g->p[L] : 0;
    A.n[l] = l < d ? g->n[L] : 1;
    A.nel[l] = l < d ? g->nel[L] : 1;
    A.nq[l] = l < d ? g->nq[L] : 1;
    A.Q[l] = l < d ? g->Q[L] : 1;
    A.tab[l] = l < d ? h->tab[L] : nullptr;
  }
  A.coef = coef;
  A.S = g->S;
  {
    STST_PROF("geo_assemble", st);
    k_geo_assemble<<<grid_for(g->N_s * W, 128), 128, 0, st>>>(A);
  }
  if (cudaGetLastError() != cudaSuccess) return fail(STST_ERR_CUDA);
  const long long nS = g->N_s * W;
  k_geo_scale<<<grid_for(nS, 256), 256, 0, st>>>(g->S + nS, nS, h->nu * h->nu);
  k_geo_scale<<<grid_for(nS, 256), 256, 0, st>>>(g->S + 2 * nS, nS, h->nu);
  k_geo_means<<<1, 1024, 0, st>>>(coef, g->N_qs, d, dmeans);
  int hf = 0;
  double means[STST_MAXD + 1] = {0.0, 0.0, 0.0, 0.0};
  const bool ok = cudaGetLastError() == cudaSuccess &&
                  cudaMemcpyAsync(&hf, dflags, sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
                  cudaMemcpyAsync(means, dmeans, sizeof(double) * (d + 1), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
                  cudaStreamSynchronize(st) == cudaSuccess;
  cudaFree(dmeans);
  if (!ok) return fail(STST_ERR_CUDA);
  g->scale[0] = 1.0;
  for (int l = 1; l <= d; ++l) g->scale[l] = means[0] > 0.0 ? means[l] / means[0] : 1.0;
  cudaFree(coef);
  cudaFree(dflags);
  cudaFree(dQ);
  coef = nullptr;
  dflags = nullptr;
  dQ = nullptr;
  if ((hf & 1) || (hf & 6) == 6) return fail(STST_ERR_ARG);  // a singular or folding map
  free_geo(h->geo);
  h->geo = g;
  h->sys_plan.geo = g;
  h->fd_ready = 0;  // the preconditioner's eigenvalue scales changed: stst_build_fd again
  invalidate_solver_graphs(h);
  return STST_OK;
}

double geo_prec_scale(const GeoOp *g, int l) { return g ? g->scale[l] : 1.0; }

int launch_scale_vec(double *a, double c, long long n, cudaStream_t s) {
  k_geo_scale<<<grid_for(n, 256), 256, 0, s>>>(a, n, c);
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}

extern "C" int stst_geometry_info(stst_handle h, int *mapped, int *entries_per_row, double *prec_scales) {
  if (!h || h->magic != STST_MAGIC) return STST_ERR_HANDLE;
  if (mapped) *mapped = h->geo ? 1 : 0;
  if (entries_per_row) *entries_per_row = h->geo ? h->geo->W : 0;
  if (prec_scales)
    for (int l = 1; l <= h->d; ++l) prec_scales[l - 1] = geo_prec_scale(h->geo, l);
  return STST_OK;
}
