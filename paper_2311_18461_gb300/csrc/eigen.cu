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
#include <type_traits>

// ------------------------------------------------------------------------------------------------
// FP32 first approximation (n <= 128) in three kernels. With M = C C^T (banded Cholesky) the pencil
// becomes the symmetric matrix A = C^{-1} L C^{-T}; Householder reflections reduce A to tridiagonal T
// (k_eig_tridiag, one CTA: the reduction is a chain of dependent steps). Every eigenvalue of T is then
// found by multisection on Sturm counts, one warp per eigenvalue (k_eig_values), and every eigenvector
// by inverse iteration with partial pivoting, the reflections applied back and U0 = C^{-T} Q, one warp
// per eigenvalue or cluster of close eigenvalues (k_eig_vectors): these steps are independent across
// the eigenvalues, so they run on ceil(n / 4) CTAs at once.
// Scratch (floats, EigScratch): the reflectors (column k holds v_k on rows k+1..), the diagonal and
// off-diagonal of T, the betas, the band of C, the eigenvalues of T and the eigenvectors of T.
// ------------------------------------------------------------------------------------------------
// C C^T = M for the band of M (n x (2P+1), row-major) into C (n x (P+1), C[i(P+1)+k] = C_{i,i-P+k}),
// one thread; rows i-1 .. i-P of C stay in registers (W[r] = row i-1-r), so the recurrence runs on
// register operands. A non-positive pivot sets bit 0 of *flags.
template <int P>
__device__ void eig_band_cholesky(const float *Ms, float *C, int n, int *flags) {
  constexpr int BW = 2 * P + 1;
  float W[P][P + 1];
#pragma unroll
  for (int r = 0; r < P; ++r)
#pragma unroll
    for (int k = 0; k <= P; ++k) W[r][k] = 0.f;
  for (int i = 0; i < n; ++i) {
    float row[P + 1];
    float mrow[P + 1];
#pragma unroll
    for (int k = 0; k <= P; ++k) mrow[k] = Ms[i * BW + k];
#pragma unroll
    for (int k = 0; k <= P; ++k) {
      const int j = i - P + k;  // column of entry k
      float s = mrow[k];
      // s -= sum_{m < j} C[i][m] C[j][m]: entry kk of row i is column i-P+kk, row j is W[P-1-k] there
#pragma unroll
      for (int kk = 0; kk < k; ++kk) {
        const int e = kk - k + P;  // index of column i-P+kk in row j's band
        if (k < P && e >= 0) s -= row[kk] * W[P - 1 - k][e];
        if (k == P) s -= row[kk] * row[kk];
      }
      if (j < 0) {
        row[k] = 0.f;
      } else if (k < P) {
        row[k] = s / W[P - 1 - k][P];
      } else {
        if (!(s > 0.f)) {
          atomicOr(flags, 1);
          s = 1.f;
        }
        row[P] = sqrtf(s);
      }
    }
#pragma unroll
    for (int k = 0; k <= P; ++k) C[i * (P + 1) + k] = row[k];
#pragma unroll
    for (int r = P - 1; r > 0; --r)
#pragma unroll
      for (int k = 0; k <= P; ++k) W[r][k] = W[r - 1][k];
#pragma unroll
    for (int k = 0; k <= P; ++k) W[0][k] = row[k];
  }
}

// Column of Z = C^{-1} B by forward substitution (C lower banded, C[i(P+1)+k] = C_{i,i-P+k}), the last P
// values in registers; B's entry in row i is bval(i), Z's row i goes to out[i * ostride].
template <int P, typename F>
__device__ void eig_lower_solve(const float *C, const float *rinv, int n, F bval, float *out, int ostride) {
  float win[P];  // win[r] = z_{i-1-r}
#pragma unroll
  for (int r = 0; r < P; ++r) win[r] = 0.f;
  for (int i = 0; i < n; ++i) {
    float s = bval(i);
#pragma unroll
    for (int r = 0; r < P; ++r)
      if (i - 1 - r >= 0) s -= C[i * (P + 1) + (P - 1 - r)] * win[r];
    const float z = s * rinv[i];
    out[i * ostride] = z;
#pragma unroll
    for (int r = P - 1; r > 0; --r) win[r] = win[r - 1];
    win[0] = z;
  }
}

// x <- C^{-T} x by back substitution in place, the last P solved values in registers.
template <int P>
__device__ void eig_upper_solve(const float *C, const float *rinv, int n, float *x) {
  float win[P];  // win[r] = x_{i+1+r} (solved)
#pragma unroll
  for (int r = 0; r < P; ++r) win[r] = 0.f;
  for (int i = n - 1; i >= 0; --i) {
    float t = x[i];
#pragma unroll
    for (int r = 0; r < P; ++r)
      if (i + 1 + r < n) t -= C[(i + 1 + r) * (P + 1) + (P - 1 - r)] * win[r];
    const float xi = t * rinv[i];
    x[i] = xi;
#pragma unroll
    for (int r = P - 1; r > 0; --r) win[r] = win[r - 1];
    win[0] = xi;
  }
}

struct EigScratch {
  float *H, *dg, *od, *bet, *C, *pv, *Xt;
  __host__ __device__ EigScratch(float *base, int n, int p) {
    H = base;
    dg = H + n * n;
    od = dg + n;
    bet = od + n;
    C = bet + n;
    pv = C + n * (p + 1);
    Xt = pv + n;
  }
  static size_t floats(int n, int p) { return 2 * (size_t)n * n + 4 * (size_t)n + (size_t)n * (p + 1); }
};

__global__ void __launch_bounds__(512) k_eig_tridiag(const double *__restrict__ Mb, const double *__restrict__ Lb,
                                                     int n, int p, float *scratch, int *flags) {
  extern __shared__ __align__(16) float sm[];
  const int ld = n + 1;
  float *A = sm;                   // n x ld: matrix, then Householder vectors below the diagonal
  float *X = A + n * ld;           // n x ld: scratch, then eigenvectors (column j)
  float *C = X + n * ld;           // n x (p+1): C[i*(p+1)+k] = C_{i, i-p+k}
  float *dg = C + n * (p + 1);     // diagonal of T
  float *od = dg + n;              // off-diagonal of T (od[k] = T[k+1][k])
  float *bet = od + n;             // Householder beta_k
  float *pv = bet + n;             // work vector p
  float *wv = pv + n;              // reciprocal diagonal of C
  float *Ms = wv + n;              // n x (2p+1): the bands of M and L, staged once
  float *Ls = Ms + n * (2 * p + 1);
  __shared__ float bc[4];
  const int tid = threadIdx.x, nth = blockDim.x;
  const int bw = 2 * p + 1;
  for (int e = tid; e < n * bw; e += nth) {  // the serial steps below then read shared memory only
    Ms[e] = (float)Mb[e];
    Ls[e] = (float)Lb[e];
  }
  __syncthreads();
  // 1. banded Cholesky of M (thread 0, the last P rows of C in registers)
  if (tid == 0) {
    switch (p) {
#define CASE(PP) case PP: eig_band_cholesky<PP>(Ms, C, n, flags); break;
      CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
      default: atomicOr(flags, 1);
    }
  }
  __syncthreads();
  // 2. Y = C^{-1} L (column j by thread j, into X), A = C^{-1} Y^T, symmetrized; the recurrences keep
  //    the last p values in registers and multiply by reciprocal diagonals (wv holds them here)
  for (int i = tid; i < n; i += nth) wv[i] = 1.f / C[i * (p + 1) + p];
  __syncthreads();
  for (int j = tid; j < n; j += nth) {
    auto lval = [&](int i) { return (abs(i - j) <= p) ? Ls[i * bw + (j - i + p)] : 0.f; };
    switch (p) {
#define CASE(PP) case PP: eig_lower_solve<PP>(C, wv, n, lval, X + j, ld); break;
      CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
    }
  }
  __syncthreads();
  for (int j = tid; j < n; j += nth) {
    auto yval = [&](int i) { return X[j * ld + i]; };
    switch (p) {
#define CASE(PP) case PP: eig_lower_solve<PP>(C, wv, n, yval, A + j, ld); break;
      CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
    }
  }
  __syncthreads();
  for (int i = tid; i < n; i += nth)
    for (int j = i + 1; j < n; ++j) {
      float a = 0.5f * (A[i * ld + j] + A[j * ld + i]);
      A[i * ld + j] = a;
      A[j * ld + i] = a;
    }
  __syncthreads();
  // 3. Householder tridiagonalization: step k zeroes column k below the subdiagonal. Three barriers a
  //    step: the reflector (warp 0), p = beta A v (eight lanes per row), then every warp forms
  //    k = beta p.v / 2 itself and the rank-2 update uses w = p - k v on the fly.
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;  // length of x = A[k+1.., k]
    if (tid < 32) {
      float s = 0.f;
      for (int i = tid; i < m; i += 32) {
        float v = A[(k + 1 + i) * ld + k];
        s += v * v;
      }
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (tid == 0) {
        float x0 = A[(k + 1) * ld + k];
        float nx = sqrtf(s);
        float alpha = (x0 >= 0.f) ? -nx : nx;
        float vtv = s - x0 * x0 + (x0 - alpha) * (x0 - alpha);
        const float beta = (nx > 0.f && vtv > 0.f) ? 2.f / vtv : 0.f;
        bc[1] = beta;
        dg[k] = A[k * ld + k];
        od[k] = (beta > 0.f) ? alpha : x0;
        bet[k] = beta;
        A[(k + 1) * ld + k] = x0 - alpha;  // v_0 (the rest of v is the column itself)
      }
    }
    __syncthreads();
    const float beta = bc[1];
    if (beta > 0.f) {
      // p = beta * A_sub v: eight lanes per row, combined by shuffles within each group of eight
      for (int base = 0; base < m; base += nth >> 3) {
        const int i = base + (tid >> 3), q = tid & 7;
        float s = 0.f;
        if (i < m)
          for (int j = q; j < m; j += 8) s += A[(k + 1 + i) * ld + (k + 1 + j)] * A[(k + 1 + j) * ld + k];
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        s += __shfl_xor_sync(0xffffffffu, s, 4);
        if (q == 0 && i < m) pv[i] = beta * s;
      }
      __syncthreads();
      float s = 0.f;
      for (int i = (tid & 31); i < m; i += 32) s += pv[i] * A[(k + 1 + i) * ld + k];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      const float kk = 0.5f * beta * s;
      // rank-2 update, a row per warp and a column per lane: v_i and w_i are warp-uniform (broadcast
      // reads) and no thread divides to find its element
      for (int i = tid >> 5; i < m; i += nth >> 5) {
        const float vi = A[(k + 1 + i) * ld + k];
        const float wi = pv[i] - kk * vi;
        for (int j = tid & 31; j < m; j += 32) {
          const float vj = A[(k + 1 + j) * ld + k];
          const float wj = pv[j] - kk * vj;
          A[(k + 1 + i) * ld + (k + 1 + j)] -= vi * wj + wi * vj;
        }
      }
    }
    __syncthreads();  // also when beta = 0: bc[1] is rewritten by the next step
  }
  if (tid == 0) {
    if (n >= 2) {
      dg[n - 2] = A[(n - 2) * ld + (n - 2)];
      od[n - 2] = A[(n - 1) * ld + (n - 2)];
      if (n - 2 >= 0) bet[n - 2] = 0.f;
    }
    dg[n - 1] = A[(n - 1) * ld + (n - 1)];
  }
  __syncthreads();
  // hand T, the reflectors and C to the eigenvector kernels
  EigScratch sc(scratch, n, p);
  for (int e = tid; e < n * n; e += nth) {  // column-major: H[k n + i] = (v_k)_i
    const int k = e / n, i = e - (e / n) * n;
    sc.H[e] = (i > k) ? A[i * ld + k] : 0.f;
  }
  for (int i = tid; i < n; i += nth) {
    sc.dg[i] = dg[i];
    sc.od[i] = od[i];
    sc.bet[i] = bet[i];
  }
  for (int e = tid; e < n * (p + 1); e += nth) sc.C[e] = C[e];
}

// Gershgorin interval of T, widened by 1e-3 of its span (every lane returns it)
__device__ void eig_bounds(const float *dg, const float *od, int n, float *lo, float *hi) {
  const int lane = threadIdx.x & 31;
  float glo = 1e30f, ghi = -1e30f;
  for (int i = lane; i < n; i += 32) {
    const float r = (i > 0 ? fabsf(od[i - 1]) : 0.f) + (i < n - 1 ? fabsf(od[i]) : 0.f);
    glo = fminf(glo, dg[i] - r);
    ghi = fmaxf(ghi, dg[i] + r);
  }
  for (int o = 16; o > 0; o >>= 1) {
    glo = fminf(glo, __shfl_xor_sync(0xffffffffu, glo, o));
    ghi = fmaxf(ghi, __shfl_xor_sync(0xffffffffu, ghi, o));
  }
  const float span = fmaxf(ghi - glo, 1e-30f);
  *lo = glo - 1e-3f * span;
  *hi = ghi + 1e-3f * span;
}

// Eigenvalue j of T (ascending) for warp j: its 32 lanes count at 32 shifts per step (Sturm counts of
// T - sigma I), shrinking the bracket 33-fold, until it is 2e-7 relative.
__global__ void __launch_bounds__(128) k_eig_values(float *scratch, int n, int p, double *lam0) {
  EigScratch sc(scratch, n, p);
  __shared__ float sd[128], so[128];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    sd[i] = sc.dg[i];
    so[i] = sc.od[i];
  }
  __syncthreads();
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (j >= n) return;
  float lo, hi;
  eig_bounds(sd, so, n, &lo, &hi);
  for (int step = 0; step < 12; ++step) {
    if (!(hi - lo > 2e-7f * fmaxf(fabsf(lo), fabsf(hi)))) break;
    const float w = (hi - lo) / 33.f;
    const float sig = lo + (lane + 1) * w;
    int cnt = 0;
    float q = sd[0] - sig;
    cnt += (q < 0.f);
    for (int i = 1; i < n; ++i) {
      if (fabsf(q) < 1e-30f) q = -1e-30f;
      q = sd[i] - sig - __fdividef(so[i - 1] * so[i - 1], q);
      cnt += (q < 0.f);
    }
    // first lane whose shift has more than j eigenvalues below it brackets eigenvalue j
    const unsigned above = __ballot_sync(0xffffffffu, cnt > j);
    const int l = above ? (__ffs(above) - 1) : 32;
    const float nlo = (l == 0) ? lo : lo + l * w;
    const float nhi = (l == 32) ? hi : lo + (l + 1) * w;
    lo = nlo;
    hi = nhi;
  }
  if (lane == 0) {
    const float v = 0.5f * (lo + hi);
    sc.pv[j] = v;
    lam0[j] = (double)v;
  }
}

// sum over the warp (every lane returns it)
__device__ __forceinline__ float warp_sum_f(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Eigenvectors. Eigenvalues closer than 1e-5 * span to their predecessor form a cluster (the boundary
// outlier modes of the B-spline pencils come in nearly degenerate symmetric / antisymmetric pairs); the
// warp of the cluster's first eigenvalue computes all its vectors in turn, orthogonalizing each sweep
// against the ones already found, so the cluster's subspace is spanned rather than one vector twice.
// Inverse iteration on T - lam I (LU with partial pivoting, 2 sweeps) runs on lane 0 (a serial
// recurrence); normalization, orthogonalization, the back-transform X <- H_0 ... H_{n-3} X and the
// final C^{-T} solve use the whole warp or registers. Shared memory: the reflectors (n x n), T and the
// reciprocal diagonal of C, staged once per CTA, plus 4n floats per warp (the vector and the LU rows).
__global__ void __launch_bounds__(128) k_eig_vectors(float *scratch, int n, int p, double *U0) {
  EigScratch sc(scratch, n, p);
  extern __shared__ __align__(16) float es[];
  float *H = es;                      // n x n reflectors, column-major (H[k n + i] = (v_k)_i)
  float *dg = H + n * n, *od = dg + n, *bet = od + n, *pv = bet + n, *rinv = pv + n;
  float *C = rinv + n;                // n x (p+1)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float *x = C + n * (p + 1) + warp * 4 * n;  // this warp's vector
  float *U = x + n;                           // and its LU rows (3 per row)
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) H[e] = sc.H[e];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    dg[i] = sc.dg[i];
    od[i] = sc.od[i];
    bet[i] = sc.bet[i];
    pv[i] = sc.pv[i];
  }
  for (int e = threadIdx.x; e < n * (p + 1); e += blockDim.x) C[e] = sc.C[e];
  for (int i = threadIdx.x; i < n; i += blockDim.x) rinv[i] = 1.f / sc.C[i * (p + 1) + p];
  __syncthreads();
  const int j = blockIdx.x * (blockDim.x >> 5) + warp;
  if (j >= n) return;
  float glo, ghi;
  eig_bounds(dg, od, n, &glo, &ghi);
  const float span = (ghi - glo) / 1.002f;
  const float ctol = 1e-5f * span;
  if (j > 0 && pv[j] - pv[j - 1] <= ctol) return;  // not the first of its cluster
  int e = j + 1;
  while (e < n && pv[e] - pv[e - 1] <= ctol) ++e;
  for (int a = j; a < e; ++a) {
    const float sh = pv[a] + ((a & 1) ? 1e-7f : -1e-7f) * span;
    for (int i = lane; i < n; i += 32) x[i] = 1.f + 0.01f * (float)((i * 7 + a * 13) % 17);
    __syncwarp();
    for (int sweep = 0; sweep < 2; ++sweep) {
      if (lane == 0) {
        // factor and forward-solve together; row i of U is (a0, a1, a2) on columns i, i+1, i+2.
        // The next row's entries are read one iteration ahead (before this row's stores), so the
        // loads overlap the recurrence.
        float a0 = dg[0] - sh, a1 = (n > 1) ? od[0] : 0.f, a2 = 0.f;
        float rhs = x[0];
        float psub = (n > 1) ? od[0] : 0.f, pdia = (n > 1) ? dg[1] - sh : 0.f;
        float psup = (n > 2) ? od[1] : 0.f, prhs = (n > 1) ? x[1] : 0.f;
        for (int i = 0; i < n; ++i) {
          const bool has_next = (i + 1 < n);
          float nsub = psub, ndia = pdia, nsup = psup, nrhs = prhs;
          if (i + 2 < n) {
            psub = od[i + 1];
            pdia = dg[i + 2] - sh;
            psup = (i + 3 < n) ? od[i + 2] : 0.f;
            prhs = x[i + 2];
          }
          if (has_next && fabsf(nsub) > fabsf(a0)) {  // partial pivoting on column i
            float t0 = a0, t1 = a1, t2 = a2, tr = rhs;
            a0 = nsub; a1 = ndia; a2 = nsup; rhs = nrhs;
            nsub = t0; ndia = t1; nsup = t2; nrhs = tr;
          }
          if (fabsf(a0) < 1e-30f) a0 = 1e-30f;
          U[3 * i + 0] = a0;
          U[3 * i + 1] = a1;
          U[3 * i + 2] = a2;
          x[i] = rhs;
          if (has_next) {
            const float f = __fdividef(nsub, a0);
            const float na0 = ndia - f * a1, na1 = nsup - f * a2, nr = nrhs - f * rhs;
            a0 = na0; a1 = na1; a2 = 0.f; rhs = nr;
          }
        }
        float x1 = 0.f, x2 = 0.f;
        float qx = x[n - 1], q0 = U[3 * (n - 1)], q1 = U[3 * (n - 1) + 1], q2 = U[3 * (n - 1) + 2];
        for (int i = n - 1; i >= 0; --i) {
          const float cx = qx, c0 = q0, c1 = q1, c2 = q2;
          if (i > 0) {
            qx = x[i - 1];
            q0 = U[3 * (i - 1)];
            q1 = U[3 * (i - 1) + 1];
            q2 = U[3 * (i - 1) + 2];
          }
          const float xi = __fdividef(cx - c1 * x1 - c2 * x2, c0);
          x[i] = xi;
          x2 = x1;
          x1 = xi;
        }
      }
      __syncwarp();
      // normalize (max-norm first, against overflow), orthogonalize against the cluster's earlier
      // vectors (columns j.. a-1 of Xt), normalize in the 2-norm
      float mx = 0.f;
      for (int i = lane; i < n; i += 32) mx = fmaxf(mx, fabsf(x[i]));
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const float scl = mx > 0.f ? 1.f / mx : 1.f;
      for (int i = lane; i < n; i += 32) x[i] *= scl;
      __syncwarp();
      for (int b2 = j; b2 < a; ++b2) {
        float dot = 0.f;
        for (int i = lane; i < n; i += 32) dot += x[i] * sc.Xt[(size_t)b2 * n + i];
        dot = warp_sum_f(dot);
        for (int i = lane; i < n; i += 32) x[i] -= dot * sc.Xt[(size_t)b2 * n + i];
        __syncwarp();
      }
      float nr2 = 0.f;
      for (int i = lane; i < n; i += 32) nr2 += x[i] * x[i];
      nr2 = warp_sum_f(nr2);
      const float inv = nr2 > 0.f ? rsqrtf(nr2) : 1.f;
      for (int i = lane; i < n; i += 32) x[i] *= inv;
      __syncwarp();
    }
    for (int i = lane; i < n; i += 32) sc.Xt[(size_t)a * n + i] = x[i];  // for the cluster's later vectors
    // back-transform: x <- H_0 H_1 ... H_{n-3} x, H_k = I - beta_k v_k v_k^T on rows k+1.., with x in
    // registers (lane holds rows lane + 32 r) and v_k read as consecutive words
    float xr[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) xr[r] = (lane + 32 * r < n) ? x[lane + 32 * r] : 0.f;
    for (int k = n - 3; k >= 0; --k) {
      const float b = bet[k];
      if (b == 0.f) continue;
      const float *vk = H + k * n;
      float s = 0.f;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int i = lane + 32 * r;
        if (i > k && i < n) s += vk[i] * xr[r];
      }
      s = b * warp_sum_f(s);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int i = lane + 32 * r;
        if (i > k && i < n) xr[r] -= s * vk[i];
      }
    }
    // normalize (2-norm) and U0 = C^{-T} x by back substitution (lane 0: a serial recurrence)
    float s2 = 0.f;
#pragma unroll
    for (int r = 0; r < 4; ++r) s2 += xr[r] * xr[r];
    s2 = warp_sum_f(s2);
    const float inv2 = rsqrtf(fmaxf(s2, 1e-30f));
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (lane + 32 * r < n) x[lane + 32 * r] = xr[r] * inv2;
    __syncwarp();
    if (lane == 0) {
      switch (p) {
#define CASE(PP) case PP: eig_upper_solve<PP>(C, rinv, n, x); break;
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
      }
    }
    __syncwarp();
    for (int i = lane; i < n; i += 32) U0[(size_t)i * n + a] = (double)x[i];
    __syncwarp();
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

// lam_j = S_jj / (1 - R_jj); E_kj = (S_kj + lam_j R_kj) / (lam_j - lam_k) for well separated pairs,
// R_kj / 2 otherwise. Pairs closer than 1e-3 relative are treated as a cluster: dividing the O(eps)
// error of an FP32 starting vector by a tiny gap would amplify it; such clusters are only
// orthonormalized here and diagonalized exactly afterwards (k_oa_cluster).
#define OA_CLUSTER_GAP 1e-3
__global__ void k_oa_E(const double *__restrict__ R, const double *__restrict__ S, int n, double *E, double *lam) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  int k = e / n, j = e % n;
  double lj = S[j * n + j] / (1.0 - R[j * n + j]);
  double lk = S[k * n + k] / (1.0 - R[k * n + k]);
  double v;
  double gap = fabs(lj - lk);
  if (k == j || !(gap > OA_CLUSTER_GAP * fmax(fabs(lj), fabs(lk)))) v = 0.5 * R[e];
  else v = (S[e] + lj * R[e]) / (lj - lk);
  E[e] = v;
  if (k == j) lam[j] = lj;
}

// Exact diagonalization inside clusters of close eigenvalues (one CTA): for each run of columns whose
// eigenvalues are within OA_CLUSTER_GAP (relative), cyclic Jacobi rotations on the block X_c^T L X_c.
// The columns are already M-orthonormal and rotations keep them so. Y = L X_c is updated alongside.
__global__ void k_oa_cluster(const double *__restrict__ Lb, int n, int p, double *X, double *lam, double *Y) {
  __shared__ int cs, ce;
  __shared__ double red[32];
  __shared__ double rot[3];
  const int tid = threadIdx.x, bw = 2 * p + 1;
  int start = 0;
  while (true) {
    if (tid == 0) {
      int s0 = start;
      while (s0 + 1 < n && !(fabs(lam[s0 + 1] - lam[s0]) <= OA_CLUSTER_GAP * fmax(fabs(lam[s0]), fabs(lam[s0 + 1]))))
        ++s0;
      int e0 = s0 + 1;
      while (e0 < n && fabs(lam[e0] - lam[e0 - 1]) <= OA_CLUSTER_GAP * fmax(fabs(lam[e0]), fabs(lam[e0 - 1]))) ++e0;
      cs = s0;
      ce = (s0 + 1 < n) ? e0 : n;
    }
    __syncthreads();
    const int c0 = cs, c1 = ce;
    __syncthreads();
    if (c1 - c0 < 2) break;
    // Y[:, c] = L X[:, c] for the cluster's columns
    for (int e = tid; e < n * (c1 - c0); e += blockDim.x) {
      const int i = e / (c1 - c0), c = c0 + e % (c1 - c0);
      double acc = 0.0;
      for (int k = 0; k < bw; ++k) {
        const int m = i - p + k;
        if (m >= 0 && m < n) acc += Lb[i * bw + k] * X[m * n + c];
      }
      Y[i * n + c] = acc;
    }
    __syncthreads();
    for (int sweep = 0; sweep < 8; ++sweep) {
      if (tid == 0) rot[2] = 0.0;  // set when a rotation of this sweep is not the identity
      for (int a = c0; a < c1; ++a)
        for (int b = a + 1; b < c1; ++b) {
          // block entries S_aa, S_bb, S_ab
          double saa = 0.0, sbb = 0.0, sab = 0.0;
          for (int i = tid; i < n; i += blockDim.x) {
            saa += X[i * n + a] * Y[i * n + a];
            sbb += X[i * n + b] * Y[i * n + b];
            sab += X[i * n + a] * Y[i * n + b];
          }
          double vals[3] = {saa, sbb, sab};
          for (int q = 0; q < 3; ++q) {
            double v = vals[q];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if ((tid & 31) == 0) red[(tid >> 5) + 8 * q] = v;
          }
          __syncthreads();
          if (tid == 0) {
            double A = 0, B = 0, C = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
              A += red[w];
              B += red[w + 8];
              C += red[w + 16];
            }
            double c = 1.0, sn = 0.0;
            // converged pairs (off-diagonal at rounding level) keep the identity
            if (fabs(C) > 1e-15 * sqrt(fabs(A * B)) + 1e-300) {
              rot[2] = 1.0;
              const double th = (B - A) / (2.0 * C);
              const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
              c = 1.0 / sqrt(t * t + 1.0);
              sn = t * c;
            }
            rot[0] = c;
            rot[1] = sn;
          }
          __syncthreads();
          const double c = rot[0], sn = rot[1];
          for (int i = tid; i < n; i += blockDim.x) {
            const double xa = X[i * n + a], xb = X[i * n + b], ya = Y[i * n + a], yb = Y[i * n + b];
            X[i * n + a] = c * xa - sn * xb;
            X[i * n + b] = sn * xa + c * xb;
            Y[i * n + a] = c * ya - sn * yb;
            Y[i * n + b] = sn * ya + c * yb;
          }
          __syncthreads();
        }
      if (rot[2] == 0.0) break;  // a sweep without rotations: the block is diagonal (uniform: shared)
      __syncthreads();           // every thread has read rot[2] before the next sweep resets it
    }
    // eigenvalues of the rotated columns: lam_c = x_c^T L x_c
    for (int c = c0; c < c1; ++c) {
      double v = 0.0;
      for (int i = tid; i < n; i += blockDim.x) v += X[i * n + c] * Y[i * n + c];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if ((tid & 31) == 0) red[tid >> 5] = v;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        lam[c] = t;
      }
      __syncthreads();
    }
    start = c1;
    if (start >= n - 1) break;
  }
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
// One thread per system i: lam_i = sum_l lam_{l, i_l}; rows of H_i = L_t + nu^2 lam^2 M_t + i nu lam KA_t
// are formed on the fly and factored by banded Cholesky G G^H = H with a register window of the last
// P rows. R = double writes the FP64 factors (and FP32 copies); R = float factors in FP32 only.
template <typename R, int P>
__global__ void k_hfactor(const R *__restrict__ Lt, const R *__restrict__ Mt, const R *__restrict__ KAt, int nt,
                          double nu, int d, const double *__restrict__ lam1, const double *__restrict__ lam2,
                          const double *__restrict__ lam3, int n1, int n2, long long Ns, double2 *G, double *D,
                          float2 *G32, float *D32, int *flags, int stage) {
  using T = typename std::conditional<sizeof(R) == 8, double2, float2>::type;
  extern __shared__ __align__(16) unsigned char hf_smem[];
  const int bw = 2 * P + 1;
  if (stage) {  // the three time bands are read by every thread at every step: keep them on chip
    R *sL = (R *)hf_smem, *sM = sL + nt * bw, *sK = sM + nt * bw;
    for (int e = threadIdx.x; e < nt * bw; e += blockDim.x) {
      sL[e] = Lt[e];
      sM[e] = Mt[e];
      sK[e] = KAt[e];
    }
    __syncthreads();
    Lt = sL;
    Mt = sM;
    KAt = sK;
  }
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
  const R a2 = (R)(nu * nu * lam * lam), a1 = (R)(nu * lam);
  T rw[P][P];
  R dw[P];
#pragma unroll
  for (int a = 0; a < P; ++a) {
    dw[a] = 1;
#pragma unroll
    for (int k = 0; k < P; ++k) { rw[a][k].x = 0; rw[a][k].y = 0; }
  }
  for (int t = 0; t < nt; ++t) {
    T g[P + 1];
#pragma unroll
    for (int k = P; k >= 1; --k) {
      int s = t - k;
      if (s < 0) { g[k].x = 0; g[k].y = 0; continue; }
      int off = s - t + P;  // = P - k
      R sr = Lt[t * bw + off] + a2 * Mt[t * bw + off];
      R si = a1 * KAt[t * bw + off];
#pragma unroll
      for (int j = k + 1; j <= P; ++j) {
        T gj = g[j];
        T c = rw[k - 1][j - k - 1];  // G[s][s-(j-k)]
        sr -= gj.x * c.x + gj.y * c.y;   // gj * conj(c)
        si -= gj.y * c.x - gj.x * c.y;
      }
      R inv = (R)1 / dw[k - 1];
      g[k].x = sr * inv;
      g[k].y = si * inv;
    }
    R dd = Lt[t * bw + P] + a2 * Mt[t * bw + P];
#pragma unroll
    for (int k = 1; k <= P; ++k) dd -= g[k].x * g[k].x + g[k].y * g[k].y;
    if (!(dd > (R)0)) {
      atomicOr(flags, 2);
      dd = 1;
    }
    R gd = sqrt(dd);
#pragma unroll
    for (int k = 1; k <= P; ++k) {
      long long ofs = ((long long)t * P + (k - 1)) * Ns + i;
      if constexpr (sizeof(R) == 8) G[ofs] = make_double2(g[k].x, g[k].y);
      G32[ofs] = make_float2((float)g[k].x, (float)g[k].y);
    }
    if constexpr (sizeof(R) == 8) D[(long long)t * Ns + i] = 1.0 / gd;
    D32[(long long)t * Ns + i] = (float)((R)1 / gd);
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

// Launches the whole setup on the handle's stream without waiting (capturable into a graph).
int fd_setup_launch(stst_problem *h) {
  cudaStream_t st = h->stream;
  const int d = h->d;
  STST_CUDA(cudaMemsetAsync(h->flags, 0, sizeof(int) * 4, st));
  // potential-aware operator: eigenpairs of (G_l, M_l), G_l = nu L_l + M_{v_l}; nu is inside G_l
  const bool pv = h->prec_op == 1 && h->pot_rank > 0 && h->g_valid;
  for (int l = 1; l <= d; ++l) {
    // directions with the same degree and mesh share one eigendecomposition (P_V: and the same G_l)
    int src = pv ? h->g_share[l] : l;
    for (int k = 1; k < l && !pv; ++k)
      if (h->dir[k].p == h->dir[l].p && h->dir[k].n_el == h->dir[l].n_el) { src = k; break; }
    h->eig_src[l] = src;
    if (src != l) continue;
    const int n = h->dir[l].n, p = h->dir[l].p;
    const BandMat &M = h->mats[l][0], &L = pv ? h->mats[l][h->g_mat[l]] : h->mats[l][1];
    const size_t sm = (2 * (size_t)n * (n + 1) + (size_t)n * (p + 1) + 5 * (size_t)n + 2 * (size_t)n * (2 * p + 1)) *
                      sizeof(float);
    float *scratch = (float *)h->oa_work;  // the refinement's 6 n_max^2 doubles hold EigScratch
    int nmax = 1;
    for (int k = 1; k <= d; ++k) nmax = std::max(nmax, h->dir[k].n);
    if (EigScratch::floats(n, p) > 12 * (size_t)nmax * nmax) return STST_ERR_ARG;
    STST_TRY(ensure_dyn_smem((const void *)k_eig_tridiag, sm));
    { STST_PROF("eig_tridiag_f32", st);
    k_eig_tridiag<<<1, 512, sm, st>>>(M.d, L.d, n, p, scratch, h->flags); }
    STST_CUDA(cudaGetLastError());
    const int eg = (n + 3) / 4;  // four warps (eigenvalues) per CTA
    { STST_PROF("eig_values_f32", st); k_eig_values<<<eg, 128, 0, st>>>(scratch, n, p, h->lam[l]); }
    const size_t smv = ((size_t)n * n + 5 * (size_t)n + (size_t)n * (p + 1) + 16 * (size_t)n) * sizeof(float);
    STST_TRY(ensure_dyn_smem((const void *)k_eig_vectors, smv));
    { STST_PROF("eig_vectors_f32", st); k_eig_vectors<<<eg, 128, smv, st>>>(scratch, n, p, h->U[l]); }
    STST_CUDA(cudaGetLastError());
    double *X = h->U[l], *PM = h->oa_work, *PL = PM + n * n, *R = PL + n * n, *S = R + n * n, *E = S + n * n,
           *Xn = E + n * n;
    int g = grid_for((long long)n * n, 64);
    // FP64 factors need full accuracy; the FP32 preconditioner needs FP32 accuracy only
    const int refine = (h->prec_mode == STST_PREC_FP64) ? 3 : 1;
    for (int it = 0; it < refine; ++it) {
      STST_PROF_N("eig_refine_f64", st, 4);
      k_oa_band<<<g, 64, 0, st>>>(M.d, L.d, X, n, p, PM, PL);
      k_oa_gram<<<g, 64, 0, st>>>(X, PM, PL, n, R, S);
      k_oa_E<<<g, 64, 0, st>>>(R, S, n, E, h->lam[l]);
      k_oa_update<<<g, 64, 0, st>>>(X, E, n, Xn);
      STST_CUDA(cudaMemcpyAsync(X, Xn, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, st));
    }
    { STST_PROF("eig_cluster_f64", st); k_oa_cluster<<<1, 256, 0, st>>>(L.d, n, p, X, h->lam[l], PL); }
    STST_CUDA(cudaGetLastError());
  }
  for (int l = 1; l <= d; ++l) {
    int src = h->eig_src[l];
    if (src != l) {
      int n = h->dir[l].n;
      STST_CUDA(cudaMemcpyAsync(h->U[l], h->U[src], sizeof(double) * n * n, cudaMemcpyDeviceToDevice, st));
      STST_CUDA(cudaMemcpyAsync(h->lam[l], h->lam[src], sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    }
    { STST_PROF("to_f32", st); STST_TRY(launch_to_f32(h->U[l], h->U32[l], (long long)h->dir[l].n * h->dir[l].n, st)); }
    if (h->prec_mode == STST_PREC_BF16) {
      STST_PROF("u_to_bf16", st);
      STST_TRY(launch_u_to_bf16(h->U[l], h->dir[l].n, h->Ubf[l], st));
    }
    if (h->prec_mode == STST_PREC_FP32) {
      STST_PROF("u_to_tf32", st);
      STST_TRY(launch_u_to_tf32(h->U[l], h->dir[l].n, h->Utf[l], st));
    }
  }
  // a mapped domain: the eigenvalues scaled per direction by the mean of the metric's diagonal
  // (stst_set_geometry), after any sharing of eigenpairs between directions
  if (h->geo)
    for (int l = 1; l <= d; ++l) {
      const double sc = geo_prec_scale(h->geo, l);
      if (sc != 1.0) STST_TRY(launch_scale_vec(h->lam[l], sc, h->dir[l].n, st));
    }
  const BandMat &Lt = h->mats[0][0], &Mt = h->mats[0][1], &KAt = h->mats[0][2];
  const float *Lt32 = h->mats32[0][0], *Mt32 = h->mats32[0][1], *KAt32 = h->mats32[0][2];
  int n1 = h->dir[1].n, n2 = d >= 2 ? h->dir[2].n : 1;
  const double *l1 = h->lam[1], *l2 = d >= 2 ? h->lam[2] : nullptr, *l3 = d >= 3 ? h->lam[3] : nullptr;
  int grid = grid_for(h->N_s, 64);
  const bool f64 = h->prec_mode == STST_PREC_FP64;
  const double nu_h = pv ? 1.0 : h->nu;
  size_t hsm = 3 * (size_t)h->n_t() * (2 * h->dir[0].p + 1) * (f64 ? sizeof(double) : sizeof(float));
  const int stage = hsm <= 48 * 1024;  // otherwise the bands are read from global memory
  if (!stage) hsm = 0;
  {
  STST_PROF(f64 ? "hfactor_f64" : "hfactor_f32", st);
  switch (h->dir[0].p) {
#define CASE(PP)                                                                                                 \
  case PP:                                                                                                       \
    if (f64)                                                                                                     \
      k_hfactor<double, PP><<<grid, 64, hsm, st>>>(Lt.d, Mt.d, KAt.d, h->n_t(), nu_h, d, l1, l2, l3, n1, n2,     \
                                                 h->N_s, (double2 *)h->Hg, h->Hd, (float2 *)h->Hg32, h->Hd32,    \
                                                 h->flags, stage);                                                      \
    else                                                                                                         \
      k_hfactor<float, PP><<<grid, 64, hsm, st>>>(Lt32, Mt32, KAt32, h->n_t(), nu_h, d, l1, l2, l3, n1, n2,      \
                                                h->N_s, nullptr, nullptr, (float2 *)h->Hg32, h->Hd32, h->flags,  \
                                                stage);                                                         \
    break;
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
    default: return STST_ERR_ARG;
  }
  STST_CUDA(cudaGetLastError());
  }  // profiler scopes do not nest: the hfactor record ends here
  // the FP32 factors in the pencil order as well, when the pencil kernel runs (or before the tuner decides)
  if (h->Gp32 && (!h->tuned || h->pencil)) STST_TRY(launch_factor_pencil(h, st));
  // transfer matrices of the segmented (parallel-in-time) time solves
  STST_TRY(launch_time_transfer<float>(h->Hg32, h->Hd32, h->n_t(), h->N_s, h->dir[0].p, h->ts_S[0], h->ts_L[0],
                                       h->Tf[0], h->Tb[0], st));
  if (f64)
    STST_TRY(launch_time_transfer<double>(h->Hg, h->Hd, h->n_t(), h->N_s, h->dir[0].p, h->ts_S[1], h->ts_L[1],
                                          h->Tf[1], h->Tb[1], st));
  return STST_OK;
}

int fd_setup(stst_problem *h) {
  STST_TRY(fd_setup_launch(h));
  int hflags[4];
  STST_CUDA(cudaMemcpyAsync(hflags, h->flags, sizeof(hflags), cudaMemcpyDeviceToHost, h->stream));
  STST_CUDA(cudaStreamSynchronize(h->stream));
  if (hflags[0] & 3) return STST_NOT_HPD;
  h->fd_ready = 1;
  return STST_OK;
}
