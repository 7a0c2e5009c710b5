// Preconditioner setup (Algorithm 1 step 1, Eq. space_eig, Sec. 5.2):
//  * generalized eigenpairs of the pencil (L_l, M_l): U^T M U = I, U^T L U = Lambda.
//    A first approximation comes from a cyclic Jacobi method in FP32 on C^{-1} L C^{-T}
//    (M = C C^T banded Cholesky), computed by one CTA in shared memory; it is then refined
//    to FP64 accuracy by the Ogita-Aishima iteration for symmetric(-definite) eigenproblems
//    (R = I - X^T M X, S = X^T L X, X <- X + X E), whose products run on many CTAs because
//    FP64 throughput per SM is low on this GPU.
//  * the per-eigenvalue time operators H_i = L_t + nu^2 lam_i^2 M_t + nu lam_i (W_t + W_t^*)
//    with lam_i = sum_l lam_{l,i_l}, and their banded Cholesky factors G_i G_i^H = H_i,
//    one thread per system (Eq. independent_problems).
#include "common.cuh"
#include <cmath>

// ------------------------------------------------------------------------------------------------
// FP32 Jacobi on one CTA. Outputs U0 (row-major n x n, column j = eigenvector j, M-orthonormal to
// FP32 accuracy) and lam0, sorted ascending.
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_eig_jacobi(const double *__restrict__ Mb, const double *__restrict__ Lb, int n,
                                                    int p, double *U0, double *lam0, int *flags) {
  extern __shared__ __align__(16) float sm[];
  const int ld = n + 1;
  float *A = sm;                   // n x ld
  float *V = A + n * ld;           // n x ld
  float *C = V + n * ld;           // n x (p+1): C[i*(p+1)+k] = C_{i, i-p+k}
  float *rot = C + n * (p + 1);    // 4 x 64: c, s, p, q (as float bits)
  int *rpq = (int *)(rot + 2 * 64);
  __shared__ float red[32];
  __shared__ int conv;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int bw = 2 * p + 1;
  // 1. banded Cholesky of M (FP32, thread 0)
  if (tid == 0) {
    for (int i = 0; i < n; ++i) {
      for (int k = 0; k <= p; ++k) {
        int j = i - p + k;
        if (j < 0) { C[i * (p + 1) + k] = 0.f; continue; }
        float s = (float)Mb[i * bw + k];
        for (int m = max(i - p, 0); m < j; ++m) s -= C[i * (p + 1) + (m - i + p)] * C[j * (p + 1) + (m - j + p)];
        if (j < i) C[i * (p + 1) + k] = s / C[j * (p + 1) + p];
        else {
          if (!(s > 0.f)) { atomicOr(flags, 1); s = 1.f; }
          C[i * (p + 1) + p] = sqrtf(s);
        }
      }
    }
  }
  __syncthreads();
  // 2. Y = C^{-1} L, column j by thread j (stored in V as Y[i][j])
  for (int j = tid; j < n; j += nth) {
    for (int i = 0; i < n; ++i) {
      float s = (abs(i - j) <= p) ? (float)Lb[i * bw + (j - i + p)] : 0.f;
      for (int m = max(i - p, 0); m < i; ++m) s -= C[i * (p + 1) + (m - i + p)] * V[m * ld + j];
      V[i * ld + j] = s / C[i * (p + 1) + p];
    }
  }
  __syncthreads();
  // 3. A = C^{-1} Y^T : column j = C^{-1} (row j of Y)
  for (int j = tid; j < n; j += nth) {
    for (int i = 0; i < n; ++i) {
      float s = V[j * ld + i];
      for (int m = max(i - p, 0); m < i; ++m) s -= C[i * (p + 1) + (m - i + p)] * A[m * ld + j];
      A[i * ld + j] = s / C[i * (p + 1) + p];
    }
  }
  __syncthreads();
  for (int e = tid; e < n * n; e += nth) {
    int i = e / n, j = e % n;
    if (i < j) {
      float a = 0.5f * (A[i * ld + j] + A[j * ld + i]);
      A[i * ld + j] = a;
      A[j * ld + i] = a;
    }
  }
  for (int e = tid; e < n * n; e += nth) {
    int i = e / n, j = e % n;
    V[i * ld + j] = (i == j) ? 1.f : 0.f;
  }
  __syncthreads();
  // 4. cyclic Jacobi, round-robin pairing; all pairs of a round are disjoint
  const int np = n + (n & 1);
  const int half = np / 2;
  for (int sweep = 0; sweep < 40; ++sweep) {
    for (int r = 0; r < np - 1; ++r) {
      if (tid < half) {
        int a, b;
        if (tid == 0) { a = np - 1; b = r; }
        else { a = (r + tid) % (np - 1); b = (r - tid + np - 1) % (np - 1); }
        int pp = min(a, b), qq = max(a, b);
        float c = 1.f, s = 0.f;
        if (qq < n) {
          float apq = A[pp * ld + qq];
          float app = A[pp * ld + pp], aqq = A[qq * ld + qq];
          if (fabsf(apq) > 1e-30f * (fabsf(app) + fabsf(aqq)) && apq != 0.f) {
            float th = (aqq - app) / (2.f * apq);
            float t = (fabsf(th) > 1e15f) ? 0.5f / th : copysignf(1.f, th) / (fabsf(th) + sqrtf(th * th + 1.f));
            c = rsqrtf(t * t + 1.f);
            s = t * c;
          }
        } else { pp = -1; }
        rot[tid] = c;
        rot[64 + tid] = s;
        rpq[tid] = pp;
        rpq[64 + tid] = qq;
      }
      __syncthreads();
      for (int e = tid; e < half * n; e += nth) {  // rows
        int k = e / n, col = e % n;
        int pp = rpq[k];
        if (pp < 0) continue;
        int qq = rpq[64 + k];
        float c = rot[k], s = rot[64 + k];
        float ap = A[pp * ld + col], aq = A[qq * ld + col];
        A[pp * ld + col] = c * ap - s * aq;
        A[qq * ld + col] = s * ap + c * aq;
      }
      __syncthreads();
      for (int e = tid; e < half * n; e += nth) {  // columns of A and V
        int k = e / n, row = e % n;
        int pp = rpq[k];
        if (pp < 0) continue;
        int qq = rpq[64 + k];
        float c = rot[k], s = rot[64 + k];
        float ap = A[row * ld + pp], aq = A[row * ld + qq];
        A[row * ld + pp] = c * ap - s * aq;
        A[row * ld + qq] = s * ap + c * aq;
        float vp = V[row * ld + pp], vq = V[row * ld + qq];
        V[row * ld + pp] = c * vp - s * vq;
        V[row * ld + qq] = s * vp + c * vq;
      }
      __syncthreads();
    }
    // convergence: off-diagonal mass relative to the diagonal
    float off = 0.f, dia = 0.f;
    for (int e = tid; e < n * n; e += nth) {
      int i = e / n, j = e % n;
      float v = A[i * ld + j];
      if (i == j) dia += v * v; else off += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      dia += __shfl_xor_sync(0xffffffffu, dia, o);
    }
    if ((tid & 31) == 0) { red[tid >> 5] = off; }
    __syncthreads();
    if (tid == 0) {
      float o2 = 0.f;
      for (int w = 0; w < nth / 32; ++w) o2 += red[w];
      red[31] = o2;
    }
    __syncthreads();
    float offt = red[31];
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = dia;
    __syncthreads();
    if (tid == 0) {
      float d2 = 0.f;
      for (int w = 0; w < nth / 32; ++w) d2 += red[w];
      conv = (offt <= 1e-11f * d2) ? 1 : 0;  // FP32 accuracy; the FP64 refinement does the rest
    }
    __syncthreads();
    if (conv) break;
  }
  // 5. U = C^{-T} V (column j by thread j: back substitution), sort by eigenvalue
  for (int j = tid; j < n; j += nth) {
    float lj = A[j * ld + j];
    int rank = 0;
    for (int k = 0; k < n; ++k) {
      float lk = A[k * ld + k];
      rank += (lk < lj || (lk == lj && k < j)) ? 1 : 0;
    }
    lam0[rank] = (double)lj;
    // solve C^T u = v_j : u_i = (v_i - sum_{m=i+1}^{i+p} C[m][i] u_m) / C[i][i]; store u in column j of A? use V column in place
    for (int i = n - 1; i >= 0; --i) {
      float s = V[i * ld + j];
      for (int m = i + 1; m <= min(i + p, n - 1); ++m) s -= C[m * (p + 1) + (i - m + p)] * V[m * ld + j];
      V[i * ld + j] = s / C[i * (p + 1) + p];
    }
    for (int i = 0; i < n; ++i) U0[i * n + rank] = (double)V[i * ld + j];
  }
}

// ---- Ogita-Aishima refinement (FP64) ------------------------------------------------------------
// PM = M X, PL = L X for banded M, L and dense X (row-major).
__global__ void k_oa_band(const double *__restrict__ Mb, const double *__restrict__ Lb, const double *__restrict__ X,
                          int n, int p, double *PM, double *PL) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  int i = e / n, j = e % n, bw = 2 * p + 1;
  double sm = 0.0, sl = 0.0;
  for (int k = 0; k < bw; ++k) {
    int m = i - p + k;
    if (m >= 0 && m < n) {
      double x = X[m * n + j];
      sm += Mb[i * bw + k] * x;
      sl += Lb[i * bw + k] * x;
    }
  }
  PM[e] = sm;
  PL[e] = sl;
}

// R = I - X^T PM, S = X^T PL
__global__ void k_oa_gram(const double *__restrict__ X, const double *__restrict__ PM, const double *__restrict__ PL,
                          int n, double *R, double *S) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  int i = e / n, j = e % n;
  double r = 0.0, s = 0.0;
  for (int k = 0; k < n; ++k) {
    double x = X[k * n + i];
    r += x * PM[k * n + j];
    s += x * PL[k * n + j];
  }
  R[e] = (i == j ? 1.0 : 0.0) - r;
  S[e] = s;
}

// lam_j = S_jj / (1 - R_jj); E_kj = (S_kj + lam_j R_kj) / (lam_j - lam_k) (k != j, separated), R_kj / 2 otherwise.
__global__ void k_oa_E(const double *__restrict__ R, const double *__restrict__ S, int n, double *E, double *lam) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  int k = e / n, j = e % n;
  double lj = S[j * n + j] / (1.0 - R[j * n + j]);
  double lk = S[k * n + k] / (1.0 - R[k * n + k]);
  double v;
  double gap = fabs(lj - lk);
  if (k == j || !(gap > 1e-10 * (fabs(lj) + fabs(lk)))) v = 0.5 * R[e];
  else v = (S[e] + lj * R[e]) / (lj - lk);
  E[e] = v;
  if (k == j) lam[j] = lj;
}

// Xn = X + X E
__global__ void k_oa_update(const double *__restrict__ X, const double *__restrict__ E, int n, double *Xn) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  int i = e / n, j = e % n;
  double s = X[e];
  for (int k = 0; k < n; ++k) s += X[i * n + k] * E[k * n + j];
  Xn[e] = s;
}

// ---- H_i factorization ----------------------------------------------------------------------------
template <int P>
__global__ void k_hfactor(const double *__restrict__ Lt, const double *__restrict__ Mt, const double *__restrict__ KAt,
                          int nt, double nu, int d, const double *__restrict__ lam1, const double *__restrict__ lam2,
                          const double *__restrict__ lam3, int n1, int n2, long long Ns, double2 *G, double *D,
                          float2 *G32, float *D32, int *flags) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= Ns) return;
  double lam;
  {
    long long r = i;
    int i1 = (int)(r % n1);
    r /= n1;
    lam = lam1[i1];
    if (d >= 2) {
      int i2 = (int)(r % n2);
      r /= n2;
      lam += lam2[i2];
      if (d >= 3) lam += lam3[(int)r];
    }
  }
  const double a2 = nu * nu * lam * lam, a1 = nu * lam;
  const int bw = 2 * P + 1;
  double2 rw[P][P];
  double dw[P];
#pragma unroll
  for (int a = 0; a < P; ++a) {
    dw[a] = 1.0;
#pragma unroll
    for (int k = 0; k < P; ++k) rw[a][k] = make_double2(0.0, 0.0);
  }
  for (int t = 0; t < nt; ++t) {
    double2 g[P + 1];
#pragma unroll
    for (int k = P; k >= 1; --k) {
      int s = t - k;
      if (s < 0) { g[k] = make_double2(0.0, 0.0); continue; }
      int off = s - t + P;  // = P - k
      double hr = Lt[t * bw + off] + a2 * Mt[t * bw + off];
      double hi = a1 * KAt[t * bw + off];
      double sr = hr, si = hi;
#pragma unroll
      for (int j = k + 1; j <= P; ++j) {
        double2 gj = g[j];
        double2 c = rw[k - 1][j - k - 1];  // G[s][s-(j-k)]
        // gj * conj(c)
        sr -= gj.x * c.x + gj.y * c.y;
        si -= gj.y * c.x - gj.x * c.y;
      }
      double inv = 1.0 / dw[k - 1];
      g[k] = make_double2(sr * inv, si * inv);
    }
    double dd = Lt[t * bw + P] + a2 * Mt[t * bw + P];
#pragma unroll
    for (int k = 1; k <= P; ++k) dd -= g[k].x * g[k].x + g[k].y * g[k].y;
    if (!(dd > 0.0)) {
      atomicOr(flags, 2);
      dd = 1.0;
    }
    double gd = sqrt(dd);
#pragma unroll
    for (int k = 1; k <= P; ++k) {
      long long ofs = ((long long)t * P + (k - 1)) * Ns + i;
      G[ofs] = g[k];
      G32[ofs] = make_float2((float)g[k].x, (float)g[k].y);
    }
    D[(long long)t * Ns + i] = 1.0 / gd;
    D32[(long long)t * Ns + i] = (float)(1.0 / gd);
#pragma unroll
    for (int a = P - 1; a > 0; --a) {
      dw[a] = dw[a - 1];
#pragma unroll
      for (int k = 0; k < P; ++k) rw[a][k] = rw[a - 1][k];
    }
    dw[0] = gd;
#pragma unroll
    for (int k = 0; k < P; ++k) rw[0][k] = g[k + 1];
  }
}

int fd_setup(stst_problem *h) {
  cudaStream_t st = h->stream;
  const int d = h->d;
  STST_CUDA(cudaMemsetAsync(h->flags, 0, sizeof(int) * 4, st));
  for (int l = 1; l <= d; ++l) {
    int src = l;
    for (int k = 1; k < l; ++k)
      if (h->dir[k].p == h->dir[l].p && h->dir[k].n_el == h->dir[l].n_el) { src = k; break; }
    h->eig_src[l] = src;
    if (src != l) continue;
    const int n = h->dir[l].n, p = h->dir[l].p;
    const BandMat &M = h->mats[l][0], &L = h->mats[l][1];
    size_t sm = (2 * (size_t)n * (n + 1) + (size_t)n * (p + 1) + 4 * 64) * sizeof(float);
    STST_CUDA(cudaFuncSetAttribute(k_eig_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    { STST_PROF("eig_jacobi_f32", st);
    k_eig_jacobi<<<1, 512, sm, st>>>(M.d, L.d, n, p, h->U[l], h->lam[l], h->flags); }
    STST_CUDA(cudaGetLastError());
    double *X = h->U[l], *PM = h->oa_work, *PL = PM + n * n, *R = PL + n * n, *S = R + n * n, *E = S + n * n,
           *Xn = E + n * n;
    int g = grid_for((long long)n * n, 64);
    for (int it = 0; it < 3; ++it) {
      STST_PROF("eig_refine_f64", st);
      k_oa_band<<<g, 64, 0, st>>>(M.d, L.d, X, n, p, PM, PL);
      k_oa_gram<<<g, 64, 0, st>>>(X, PM, PL, n, R, S);
      k_oa_E<<<g, 64, 0, st>>>(R, S, n, E, h->lam[l]);
      k_oa_update<<<g, 64, 0, st>>>(X, E, n, Xn);
      STST_CUDA(cudaMemcpyAsync(X, Xn, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, st));
    }
    STST_CUDA(cudaGetLastError());
  }
  for (int l = 1; l <= d; ++l) {
    int src = h->eig_src[l];
    if (src != l) {
      int n = h->dir[l].n;
      STST_CUDA(cudaMemcpyAsync(h->U[l], h->U[src], sizeof(double) * n * n, cudaMemcpyDeviceToDevice, st));
      STST_CUDA(cudaMemcpyAsync(h->lam[l], h->lam[src], sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    }
    STST_TRY(launch_to_f32(h->U[l], h->U32[l], (long long)h->dir[l].n * h->dir[l].n, st));
  }
  const BandMat &Lt = h->mats[0][0], &Mt = h->mats[0][1], &KAt = h->mats[0][2];
  int n1 = h->dir[1].n, n2 = d >= 2 ? h->dir[2].n : 1;
  const double *l1 = h->lam[1], *l2 = d >= 2 ? h->lam[2] : nullptr, *l3 = d >= 3 ? h->lam[3] : nullptr;
  int grid = grid_for(h->N_s, 64);
  STST_PROF("hfactor_f64", st);
  switch (h->dir[0].p) {
#define CASE(PP)                                                                                                    \
  case PP:                                                                                                          \
    k_hfactor<PP><<<grid, 64, 0, st>>>(Lt.d, Mt.d, KAt.d, h->n_t(), h->nu, d, l1, l2, l3, n1, n2, h->N_s,         \
                                       (double2 *)h->Hg, h->Hd, (float2 *)h->Hg32, h->Hd32, h->flags);             \
    break;
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
    default: return STST_ERR_ARG;
  }
  STST_CUDA(cudaGetLastError());
  int hflags[4];
  STST_CUDA(cudaMemcpyAsync(hflags, h->flags, sizeof(hflags), cudaMemcpyDeviceToHost, st));
  STST_CUDA(cudaStreamSynchronize(st));
  if (hflags[0] & 3) return STST_NOT_HPD;
  h->fd_ready = 1;
  return STST_OK;
}
