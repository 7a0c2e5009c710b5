// Pencil kernel: Algorithm 1 steps 2-4 along the last spatial direction, with the time solves of step 3
// in between, for the FP32 Fast Diagonalization.
//
// After the forward products of directions 1..d-1 the tensor holds, for every pencil
// jp = (j_1, ..., j_{d-1}) (Pd = N_s / n_d pencils), the n_d x n_t block
//   B[i][t] = X[t + n_t (jp + Pd i)],
// whose rows are n_t contiguous complex values. Everything that follows for these values stays inside
// the pencil: the last forward product C[j][t] = sum_i U_d[i][j] B[i][t] (step 2), the banded solves
// H_s x_s = C[j][.] of the systems s = jp + Pd j (step 3, Eq. independent_problems), and the backward
// product D[i][t] = sum_j U_d[i][j] x_j[t] (step 4). One CTA, or a cluster of two CTAs that split the
// rows and exchange their solved halves through distributed shared memory, does all three, so the last
// direction costs one kernel and no global exchange: the tensor is read and written once, with
// coalesced rows, and the time solve needs no launch of its own.
//
// The factors are read in the pencil order s' = j + n_d jp (written once at setup by k_factor_pencil),
// so a CTA's systems are consecutive in memory; all of them are requested with cp.async before the
// forward product starts and arrive while it runs.
#include "common.cuh"
#include "async.cuh"
#include <cooperative_groups.h>

namespace cg = cooperative_groups;

template <typename T> struct PencilIO;
template <> struct PencilIO<float2> {
  static __device__ __forceinline__ float2 ld(const float2 *p) { return *p; }
  static __device__ __forceinline__ void st(float2 *p, float x, float y) { *p = make_float2(x, y); }
};
template <> struct PencilIO<double2> {
  static __device__ __forceinline__ float2 ld(const double2 *p) {
    const double2 v = *p;
    return make_float2((float)v.x, (float)v.y);
  }
  static __device__ __forceinline__ void st(double2 *p, float x, float y) { *p = make_double2((double)x, (double)y); }
};

// o(a, b) = sum_k R(k, a) C(k, b), R(k, a) = sR[k rs + a] real, C(k, b) = sC[k cs + b] complex; this thread's
// outputs a = a0 + Ra q (q < 4) and b = 4 g + c (c < 4). Every output is summed over k in ascending order.
__device__ __forceinline__ void pencil_contract(const float *__restrict__ sR, int rs, int A, const float2 *__restrict__ sC,
                                                int cs, int B, int K, int a0, int Ra, int g, float ax[4][4],
                                                float ay[4][4]) {
  int ra[4], cb[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) ra[q] = min(a0 + Ra * q, A - 1);  // clamped: results past A are not stored
#pragma unroll
  for (int c = 0; c < 4; ++c) cb[c] = min(4 * g + c, B - 1);
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int c = 0; c < 4; ++c) { ax[q][c] = 0.f; ay[q][c] = 0.f; }
  for (int k = 0; k < K; ++k) {
    const float *rk = sR + k * rs;
    const float2 *ck = sC + k * cs;
    float u[4];
    float2 x[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) u[q] = rk[ra[q]];
#pragma unroll
    for (int c = 0; c < 4; ++c) x[c] = ck[cb[c]];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        ax[q][c] += u[q] * x[c].x;
        ay[q][c] += u[q] * x[c].y;
      }
  }
}

// Shared-memory plan of the kernel (floats): U (n x n), U^T (n x n), block (n rows x ntp), own solved rows
// (h x ntp), factors (n_t P h complex), inverse diagonals (n_t h). ntp = n_t | 1 (an odd row stride keeps the
// row-per-thread accesses of the time solve free of bank conflicts).
struct PencilShape {
  int n, nt, ntp, h, P, CL;
  __host__ __device__ size_t off_Ub() const { return (size_t)n * n; }
  __host__ __device__ size_t off_B() const { return ((2 * (size_t)n * n + 3) / 4) * 4; }
  __host__ __device__ size_t off_C() const { return off_B() + 2 * (size_t)n * ntp; }
  __host__ __device__ size_t off_G() const { return off_C() + 2 * (size_t)h * ntp; }
  __host__ __device__ size_t off_D() const { return off_G() + 2 * (size_t)nt * P * h; }
  __host__ __device__ size_t floats() const { return off_D() + (size_t)nt * h; }
};

template <typename TI, typename TO, int P, int CL>
__global__ void __launch_bounds__(256) k_pencil(const TI *__restrict__ X, TO *__restrict__ Y, const float *__restrict__ U,
                                                int n, int nt, long long Pd, long long Ns,
                                                const float2 *__restrict__ Gp, const float *__restrict__ Dp,
                                                const EpiDot ed, const int *done) {
  if (done && *done) return;
  extern __shared__ __align__(16) float pc_smem[];
  __shared__ double sh[32];
  PencilShape ps;
  ps.n = n;
  ps.nt = nt;
  ps.ntp = nt | 1;
  ps.h = (n + CL - 1) / CL;
  ps.P = P;
  ps.CL = CL;
  const int ntp = ps.ntp, h = ps.h;
  const int rank = (CL > 1) ? (int)(blockIdx.x % CL) : 0;
  const long long jp = blockIdx.x / CL;
  const int j0 = rank * h, hown = min(h, n - j0);  // this CTA's rows (systems) j0 .. j0 + hown - 1
  float *sUf = pc_smem;                              // U[i][j] at i n + j
  float *sUb = pc_smem + ps.off_Ub();                // U[i][j] at j n + i
  float2 *sB = (float2 *)(pc_smem + ps.off_B());     // block rows i (n x ntp); reused for the solved rows
  float2 *sC = (float2 *)(pc_smem + ps.off_C());     // own rows of the forward product (h x ntp)
  float2 *sG = (float2 *)(pc_smem + ps.off_G());     // factors of the own systems [t][k][s]
  float *sD = pc_smem + ps.off_D();                  // inverse diagonals [t][s]
  const int tid = threadIdx.x, nth = blockDim.x;
  // U and the block (rows of n_t contiguous values) first, then the factors of this CTA's systems (pencil
  // order s' = j + n jp): two groups of copies, all in flight at once; the factors arrive while the
  // forward product runs
  for (int e = tid; e < n * n; e += nth) cp_async<4>(&sUf[e], &U[e]);
  const long long rstride = (long long)nt * Pd;  // distance between consecutive rows i of the block
  const long long base = (long long)nt * jp;
  if constexpr (sizeof(TI) == sizeof(float2)) {
    for (int e = tid; e < n * nt; e += nth) {
      const int i = e / nt, t = e - (e / nt) * nt;
      cp_async<8>(&sB[i * ntp + t], X + base + i * rstride + t);
    }
  }
  cp_async_commit();
  {
    const long long sp0 = j0 + (long long)n * jp;
    for (int e = tid; e < nt * P * hown; e += nth) {
      const int s = e % hown, tk = e / hown;
      cp_async<8>(&sG[tk * h + s], &Gp[(long long)tk * Ns + sp0 + s]);
    }
    for (int e = tid; e < nt * hown; e += nth) {
      const int s = e % hown, t = e / hown;
      cp_async<4>(&sD[t * h + s], &Dp[(long long)t * Ns + sp0 + s]);
    }
    cp_async_commit();
  }
  if constexpr (sizeof(TI) != sizeof(float2)) {  // FP64 input: batches of independent loads, rounded to FP32
    for (int e0 = tid; e0 < n * nt; e0 += 8 * nth) {
      float2 v[8];
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const int e = e0 + b * nth;
        if (e < n * nt) v[b] = PencilIO<TI>::ld(X + base + (e / nt) * rstride + e % nt);
      }
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const int e = e0 + b * nth;
        if (e < n * nt) sB[(e / nt) * ntp + e % nt] = v[b];
      }
    }
  }
  cp_async_wait_group<1>();  // U and the block (the factors may still be in flight)
  __syncthreads();
  for (int e = tid; e < n * n; e += nth) sUb[(e % n) * n + e / n] = sUf[e];
  __syncthreads();
  // step 2 along direction d: C[j][t] = sum_i U[i][j] B[i][t] for the own rows j = j0 + a
  {
    const int Ra = (hown + 3) / 4, items = Ra * ((nt + 3) / 4);
    for (int it = tid; it < items; it += nth) {
      const int a0 = it % Ra, g = it / Ra;
      float ax[4][4], ay[4][4];
      pencil_contract(sUf + j0, n, hown, sB, ntp, nt, n, a0, Ra, g, ax, ay);
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int a = a0 + Ra * q, t = 4 * g + c;
          if (a < hown && t < nt) sC[a * ntp + t] = make_float2(ax[q][c], ay[q][c]);
        }
    }
  }
  cp_async_wait_all();  // the factors
  // the other CTA of the cluster no longer reads its block once this sync is passed: the solved rows can
  // be written into both CTAs' block buffers
  if constexpr (CL > 1) cg::this_cluster().sync();
  else __syncthreads();
  // step 3: the banded Hermitian solves (G G^H) x = c of the own systems, one thread per system, in place:
  // forward G w = c, then backward G^H x = w (factor layout as in k_timesolve: sG[(t P + k - 1) h + s] =
  // G[t][t-k], sD[t h + s] = 1 / G[t][t])
  if (tid < hown) {
    const int s = tid;
    float2 *row = sC + s * ntp;
    // solved values go to the block buffers of every CTA of the cluster (row j0 + s)
    float2 *dst[CL];
#pragma unroll
    for (int r = 0; r < CL; ++r) {
      float2 *b = sB + (j0 + s) * ntp;
      if constexpr (CL > 1) dst[r] = (r == rank) ? b : cg::this_cluster().map_shared_rank(b, r);
      else dst[r] = b;
    }
    constexpr int CH = 8;  // time steps whose operands are loaded ahead of their recurrence steps
    float2 zw[P];
#pragma unroll
    for (int a = 0; a < P; ++a) zw[a] = make_float2(0.f, 0.f);
    for (int t0 = 0; t0 < nt; t0 += CH) {
      float2 yv[CH], gv[CH][P];
      float dv[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int t = min(t0 + u, nt - 1);
        yv[u] = row[t];
        dv[u] = sD[t * h + s];
#pragma unroll
        for (int k = 0; k < P; ++k) gv[u][k] = sG[(t * P + k) * h + s];
      }
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        if (t0 + u < nt) {
          float ax = yv[u].x, ay = yv[u].y;
#pragma unroll
          for (int k = 1; k <= P; ++k) {
            const float2 gk = gv[u][k - 1];
            const float2 z = zw[k - 1];
            ax -= gk.x * z.x - gk.y * z.y;
            ay -= gk.x * z.y + gk.y * z.x;
          }
          const float2 z = make_float2(ax * dv[u], ay * dv[u]);
#pragma unroll
          for (int a = P - 1; a > 0; --a) zw[a] = zw[a - 1];
          zw[0] = z;
          row[t0 + u] = z;
        }
      }
    }
    // backward: x_t = (w_t - sum_k conj(G[t+k][t]) x_{t+k}) / G[t][t]
    float2 xw[P];
#pragma unroll
    for (int a = 0; a < P; ++a) xw[a] = make_float2(0.f, 0.f);
    for (int t1 = nt - 1; t1 >= 0; t1 -= CH) {
      float2 wv[CH], gv[CH][P];
      float dv[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int t = max(t1 - u, 0);
        wv[u] = row[t];
        dv[u] = sD[t * h + s];
#pragma unroll
        for (int k = 1; k <= P; ++k)  // G[t+k][t], zero past the end
          gv[u][k - 1] = (t + k < nt) ? sG[((t + k) * P + (k - 1)) * h + s] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int t = t1 - u;
        if (t >= 0) {
          float ax = wv[u].x, ay = wv[u].y;
#pragma unroll
          for (int k = 1; k <= P; ++k) {
            const float2 gk = gv[u][k - 1];
            const float2 xv = xw[k - 1];
            ax -= gk.x * xv.x + gk.y * xv.y;
            ay -= gk.x * xv.y - gk.y * xv.x;
          }
          const float2 x = make_float2(ax * dv[u], ay * dv[u]);
#pragma unroll
          for (int a = P - 1; a > 0; --a) xw[a] = xw[a - 1];
          xw[0] = x;
#pragma unroll
          for (int r = 0; r < CL; ++r) dst[r][t] = x;
        }
      }
    }
  }
  // every CTA's block buffer now receives all solved rows; after this barrier no CTA touches another's
  // shared memory again (each exits only after its own backward product)
  if constexpr (CL > 1) cg::this_cluster().sync();
  else __syncthreads();
  const float2 *sX = sB;
  // step 4 along direction d: D[i][t] = sum_j U[i][j] x_j[t] for the own rows i = j0 + a, straight to Y
  double dacc[4] = {0.0, 0.0, 0.0, 0.0};
  {
    const int Ra = (hown + 3) / 4, items = Ra * ((nt + 3) / 4);
    for (int it = tid; it < items; it += nth) {
      const int a0 = it % Ra, g = it / Ra;
      float ax[4][4], ay[4][4];
      pencil_contract(sUb + j0, n, hown, sX, ntp, nt, n, a0, Ra, g, ax, ay);
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int a = a0 + Ra * q, t = 4 * g + c;
          if (a < hown && t < nt) {
            const long long idx = base + (long long)(j0 + a) * rstride + t;
            PencilIO<TO>::st(Y + idx, ax[q][c], ay[q][c]);
            if (ed.part) epi_dot_acc<TO>(dacc, ed, idx, (double)ax[q][c], (double)ay[q][c]);
          }
        }
    }
  }
  if (ed.part) epi_dot_store(dacc, ed, blockIdx.x, sh);
}

// Factors in the pencil order: Gp[(t P + k) Ns + s'] = G[(t P + k) Ns + s], Dp[t Ns + s'] = D[t Ns + s],
// s' = j + n jp for s = jp + Pd j.
__global__ void k_factor_pencil(const float2 *__restrict__ G, const float *__restrict__ D, float2 *__restrict__ Gp,
                                float *__restrict__ Dp, int nt, int P, long long Ns, int n) {
  const long long Pd = Ns / n;
  const long long total = (long long)nt * (P + 1) * Ns;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long sp = e % Ns, row = e / Ns;
    const long long jp = sp / n, j = sp - jp * n, s = jp + Pd * j;
    if (row < (long long)nt * P) Gp[row * Ns + sp] = G[row * Ns + s];
    else Dp[(row - (long long)nt * P) * Ns + sp] = D[(row - (long long)nt * P) * Ns + s];
  }
}

size_t pencil_smem(int n, int nt, int P, int CL) {
  PencilShape ps;
  ps.n = n;
  ps.nt = nt;
  ps.ntp = nt | 1;
  ps.h = (n + CL - 1) / CL;
  ps.P = P;
  ps.CL = CL;
  return ps.floats() * sizeof(float);
}

bool pencil_fits(const stst_problem *h, int CL) {
  const int n = h->dir[h->d].n, P = h->dir[0].p;
  if (P < 1 || P > 4 || (CL != 1 && CL != 2) || n < CL) return false;
  if ((long long)(h->N_s / n) * CL > 0x7fffffffLL) return false;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return pencil_smem(n, h->n_t(), P, CL) <= (size_t)optin;
}

int launch_factor_pencil(stst_problem *h, cudaStream_t s) {
  const long long total = (long long)h->n_t() * (h->dir[0].p + 1) * h->N_s;
  STST_PROF("factor_pencil", s);
  k_factor_pencil<<<grid_for(total, 256), 256, 0, s>>>((const float2 *)h->Hg32, h->Hd32, (float2 *)h->Gp32, h->Dp32,
                                                       h->n_t(), h->dir[0].p, h->N_s, h->dir[h->d].n);
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}

template <typename TI, typename TO, int P, int CL>
static int go_pencil(const TI *X, TO *Y, const stst_problem *h, const EpiDot &ed, const int *done, cudaStream_t s) {
  const int d = h->d, n = h->dir[d].n, nt = h->n_t();
  const long long Pd = h->N_s / n;
  const size_t sm = pencil_smem(n, nt, P, CL);
  auto kern = k_pencil<TI, TO, P, CL>;
  STST_TRY(ensure_dyn_smem((const void *)kern, sm));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(Pd * CL));
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = CL > 1 ? 1 : 0;
  STST_CUDA(cudaLaunchKernelEx(&cfg, kern, X, Y, (const float *)h->U32[d], n, nt, Pd, h->N_s,
                               (const float2 *)h->Gp32, (const float *)h->Dp32, ed, done));
  return STST_OK;
}

// Steps 2-4 of Algorithm 1 along direction d for every pencil (see the file comment); CL CTAs per pencil.
template <typename TI, typename TO>
int launch_pencil(const TI *X, TO *Y, const stst_problem *h, int CL, const EpiDot &ed, const int *done,
                  cudaStream_t s) {
  const long long Pd = h->N_s / h->dir[h->d].n;
  if (!pencil_fits(h, CL) || (ed.part && Pd * CL > STST_MAXPART)) return STST_ERR_ARG;
  STST_PROF("pencil_f32", s);
  switch (h->dir[0].p * 10 + CL) {
#define CASE(PP, CC) case PP * 10 + CC: return go_pencil<TI, TO, PP, CC>(X, Y, h, ed, done, s);
    CASE(1, 1) CASE(1, 2) CASE(2, 1) CASE(2, 2) CASE(3, 1) CASE(3, 2) CASE(4, 1) CASE(4, 2)
#undef CASE
    default: return STST_ERR_ARG;
  }
}

template int launch_pencil<float2, float2>(const float2 *, float2 *, const stst_problem *, int, const EpiDot &,
                                           const int *, cudaStream_t);
template int launch_pencil<double2, double2>(const double2 *, double2 *, const stst_problem *, int, const EpiDot &,
                                             const int *, cudaStream_t);
template int launch_pencil<float2, double2>(const float2 *, double2 *, const stst_problem *, int, const EpiDot &,
                                            const int *, cudaStream_t);
template int launch_pencil<double2, float2>(const double2 *, float2 *, const stst_problem *, int, const EpiDot &,
                                            const int *, cudaStream_t);
