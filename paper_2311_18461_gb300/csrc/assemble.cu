// Univariate assembly on the device: Gauss-Legendre rules, B-spline evaluation by the
// Cox-de Boor recursion (Sec. 3.1), band storage of the Galerkin matrices of
// Eq. time_mat / Eq. space_mat (optionally weighted), basis tables at the quadrature
// points, and the banded Cholesky factor of the reduced mass matrix.
#include "common.cuh"
#include <mutex>
#include <unordered_map>
#include <cmath>

thread_local cudaError_t stst_last_cuda = cudaSuccess;

int grid_for(long long n, int block) { return (int)((n + block - 1) / block); }

int ensure_dyn_smem(const void *kern, size_t bytes) {
  static std::mutex mu;
  static std::unordered_map<const void *, size_t> done;
  if (bytes <= 32 * 1024) return STST_OK;  // below the default limit whatever the static part (< 16 KB here)
  std::lock_guard<std::mutex> lk(mu);
  auto it = done.find(kern);
  if (it != done.end() && it->second >= bytes) return STST_OK;
  STST_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  done[kern] = bytes;
  return STST_OK;
}

// Knot xi_j of the open uniform knot vector on [0,1] (degree p, n_el elements), 0-based j.
__device__ __forceinline__ double knot(int j, int p, int n_el) {
  if (j <= p) return 0.0;
  if (j >= n_el + p) return 1.0;
  return (double)(j - p) / (double)n_el;
}

// Node k (ascending) and weight of the n-point Gauss-Legendre rule on [-1,1]:
// Newton's method on P_n with the three-term recurrence (a fixed, bounded number of steps).
__device__ void gauss_node(int n, int k, double *x, double *w) {
  int j = n - 1 - k;  // the cosine guess orders the roots descending in j
  double z = cos(3.14159265358979323846 * (j + 0.75) / (n + 0.5));
  double p0 = 1.0, p1 = z, dp = 1.0;
  for (int it = 0; it < 60; ++it) {
    p0 = 1.0;
    p1 = z;
    for (int m = 2; m <= n; ++m) {
      double p2 = ((2.0 * m - 1.0) * z * p1 - (m - 1.0) * p0) / m;
      p0 = p1;
      p1 = p2;
    }
    dp = (n == 1) ? 1.0 : n * (z * p1 - p0) / (z * z - 1.0);
    double dz = p1 / dp;
    z -= dz;
    if (fabs(dz) <= 1e-16) break;
  }
  p0 = 1.0;
  p1 = z;
  for (int m = 2; m <= n; ++m) {
    double p2 = ((2.0 * m - 1.0) * z * p1 - (m - 1.0) * p0) / m;
    p0 = p1;
    p1 = p2;
  }
  dp = (n == 1) ? 1.0 : n * (z * p1 - p0) / (z * z - 1.0);
  *x = z;
  *w = 2.0 / ((1.0 - z * z) * dp * dp);
}

// Values, first and second derivatives (reference coordinate) of the p+1 B-splines that
// are nonzero on element e (full indices e..e+p) at the reference point x in element e.
// out[s][a] = d^s b_{e+a}(x).
__device__ void element_basis(int p, int n_el, int e, double x, double out[3][STST_MAXP + 1]) {
  double tab[STST_MAXP + 1][STST_MAXP + 1];  // tab[k][a]: degree-k function with index s-k+a, span s = e+p
  const int s = e + p;
  tab[0][0] = 1.0;
  for (int k = 1; k <= p; ++k) {
    for (int a = 0; a <= k; ++a) {
      int j = s - k + a;
      double v = 0.0;
      if (a >= 1) {
        double den = knot(j + k, p, n_el) - knot(j, p, n_el);
        if (den > 0.0) v += (x - knot(j, p, n_el)) / den * tab[k - 1][a - 1];
      }
      if (a <= k - 1) {
        double den = knot(j + k + 1, p, n_el) - knot(j + 1, p, n_el);
        if (den > 0.0) v += (knot(j + k + 1, p, n_el) - x) / den * tab[k - 1][a];
      }
      tab[k][a] = v;
    }
  }
  // first derivatives of the degree-(p-1) functions (needed for the second derivative)
  double d1m[STST_MAXP + 1];
  for (int b = 0; b <= p - 1; ++b) {
    d1m[b] = 0.0;
    if (p - 1 >= 1) {
      int j = s - (p - 1) + b;
      double v = 0.0;
      if (b >= 1) {
        double den = knot(j + p - 1, p, n_el) - knot(j, p, n_el);
        if (den > 0.0) v += tab[p - 2][b - 1] / den;
      }
      if (b <= p - 2) {
        double den = knot(j + p, p, n_el) - knot(j + 1, p, n_el);
        if (den > 0.0) v -= tab[p - 2][b] / den;
      }
      d1m[b] = (p - 1) * v;
    }
  }
  for (int a = 0; a <= p; ++a) {
    int j = s - p + a;
    double v1 = 0.0, v2 = 0.0;
    if (a >= 1) {
      double den = knot(j + p, p, n_el) - knot(j, p, n_el);
      if (den > 0.0) {
        v1 += tab[p - 1][a - 1] / den;
        v2 += d1m[a - 1] / den;
      }
    }
    if (a <= p - 1) {
      double den = knot(j + p + 1, p, n_el) - knot(j + 1, p, n_el);
      if (den > 0.0) {
        v1 -= tab[p - 1][a] / den;
        v2 -= d1m[a] / den;
      }
    }
    out[0][a] = tab[p][a];
    out[1][a] = p * v1;
    out[2][a] = p * v2;
  }
}

// One thread per band entry (i, k) of the output: row i (full index I = i + off), column
// J = I - p + k. Sums w * integrand over the elements shared by b_I and b_J.
__global__ void k_assemble_band(int kind, int p, int n_el, double len, int nq, int off, int n_rows, int n_cols,
                                const double *__restrict__ weight, double *__restrict__ out) {
  __shared__ double sg[32], sw[32];  // Gauss rule, computed once per block (nq <= p + 2 <= 10)
  if (threadIdx.x < nq) gauss_node(nq, threadIdx.x, &sg[threadIdx.x], &sw[threadIdx.x]);
  __syncthreads();
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int bw = 2 * p + 1;
  if (idx >= n_rows * bw) return;
  int i = idx / bw, k = idx % bw;
  int jr = i - p + k;  // column in the output numbering
  double acc = 0.0;
  if (jr >= 0 && jr < n_cols) {
    int I = i + off, J = jr + off;
    int e0 = max(max(I, J) - p, 0), e1 = min(min(I, J), n_el - 1);
    double h = 1.0 / n_el;
    double s1 = 1.0 / len, s2 = 1.0 / (len * len);
    for (int e = e0; e <= e1; ++e) {
      for (int q = 0; q < nq; ++q) {
        double g = sg[q], gw = sw[q];
        double x = (e + 0.5 * (g + 1.0)) * h;  // reference coordinate in [0,1]
        double wq = 0.5 * h * gw * len;          // weight in physical coordinates
        if (weight) wq *= weight[e * nq + q];
        double B[3][STST_MAXP + 1];
        element_basis(p, n_el, e, x, B);
        int a = I - e, b = J - e;
        double bi = B[0][a], bj = B[0][b];
        double di = B[1][a] * s1, dj = B[1][b] * s1;
        double ei = B[2][a] * s2, ej = B[2][b] * s2;
        double v;
        switch (kind) {
          case MK_M: v = bi * bj; break;
          case MK_L: v = di * dj; break;
          case MK_J: v = ei * ej; break;
          case MK_K: v = bi * dj; break;            // int b'_J b_I
          case MK_K2: v = bi * ej; break;           // int b''_J b_I
          case MK_KA: v = bi * dj - bj * di; break; // K - K^T
          case MK_K2S: v = bi * ej + bj * ei; break;// K2 + K2^T
          default: v = 0.0;
        }
        acc += wq * v;
      }
    }
  }
  out[idx] = acc;
}

int launch_assemble_band(int kind, int p, int n_el, double len, int nq, int off, int n_rows, int n_cols,
                         const double *weight, double *out, cudaStream_t s) {
  long long n = (long long)n_rows * (2 * p + 1);
  if (n == 0) return STST_OK;
  k_assemble_band<<<grid_for(n, 128), 128, 0, s>>>(kind, p, n_el, len, nq, off, n_rows, n_cols, weight, out);
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}

// Quadrature points / weights of direction (physical coordinates) and basis tables:
// tab[(q*(p+1) + a)*3 + s] = d^s b_{e+a}(x_q) in physical scaling (e = element of q).
__global__ void k_quadrature(int p, int n_el, double len, int nq, double *pts, double *wts, double *tab) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_el * nq) return;
  int e = q / nq, g = q % nq;
  double z, w;
  gauss_node(nq, g, &z, &w);
  double h = 1.0 / n_el;
  double x = (e + 0.5 * (z + 1.0)) * h;
  if (pts) pts[q] = x * len;
  if (wts) wts[q] = 0.5 * h * w * len;
  if (tab) {
    double B[3][STST_MAXP + 1];
    element_basis(p, n_el, e, x, B);
    for (int a = 0; a <= p; ++a) {
      tab[(q * (p + 1) + a) * 3 + 0] = B[0][a];
      tab[(q * (p + 1) + a) * 3 + 1] = B[1][a] / len;
      tab[(q * (p + 1) + a) * 3 + 2] = B[2][a] / (len * len);
    }
  }
}

int launch_quadrature(int p, int n_el, double len, int nq, double *pts, double *wts, double *tab, cudaStream_t s) {
  int Q = n_el * nq;
  k_quadrature<<<grid_for(Q, 128), 128, 0, s>>>(p, n_el, len, nq, pts, wts, tab);
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}

// Banded Cholesky M = C C^T of the reduced mass (band p): chol[i*(p+1) + k] = C[i][i-p+k], k = p is the diagonal.
__global__ void k_mass_cholesky(const double *__restrict__ M, int n, int p, double *chol, int *flags) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int bw = 2 * p + 1;
  for (int i = 0; i < n; ++i) {
    for (int k = 0; k <= p; ++k) {
      int j = i - p + k;
      if (j < 0) { chol[i * (p + 1) + k] = 0.0; continue; }
      double s = M[i * bw + k];  // M[i][j]
      for (int m = max(i - p, 0); m < j; ++m) {
        // C[i][m] * C[j][m]
        s -= chol[i * (p + 1) + (m - i + p)] * chol[j * (p + 1) + (m - j + p)];
      }
      if (j < i) {
        chol[i * (p + 1) + k] = s / chol[j * (p + 1) + p];
      } else {
        if (!(s > 0.0)) { if (flags) atomicOr(flags, 1); s = 1.0; }
        chol[i * (p + 1) + p] = sqrt(s);
      }
    }
  }
}

int launch_mass_cholesky(const BandMat &M, double *chol, int *flags, cudaStream_t s) {
  k_mass_cholesky<<<1, 32, 0, s>>>(M.d, M.n, M.p, chol, flags);
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}

__global__ void k_to_f32(const double *__restrict__ a, float *__restrict__ b, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

int launch_to_f32(const double *src, float *dst, long long n, cudaStream_t s) {
  if (n == 0) return STST_OK;
  k_to_f32<<<grid_for(n, 256), 256, 0, s>>>(src, dst, n);
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}

__global__ void k_wprod(const double *a, const double *b, double *o, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) o[i] = a[i] * b[i];
}

int launch_weight_product(const double *a, const double *b, double *out, int n, cudaStream_t s) {
  k_wprod<<<grid_for(n, 128), 128, 0, s>>>(a, b, out, n);
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}

__global__ void k_scale(const double *a, double c, double *o, float *o32, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    double v = c * a[i];
    o[i] = v;
    o32[i] = (float)v;
  }
}

int launch_scale(const double *a, double c, double *out, float *out32, int n, cudaStream_t s) {
  k_scale<<<grid_for(n, 128), 128, 0, s>>>(a, c, out, out32, n);
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}

__global__ void k_band_axpby(const double *a, double ca, const double *b, double cb, double *o, float *o32, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    double v = ca * a[i] + cb * b[i];
    o[i] = v;
    o32[i] = (float)v;
  }
}

int launch_band_axpby(const double *a, double ca, const double *b, double cb, double *out, float *out32, int n,
                      cudaStream_t s) {
  k_band_axpby<<<grid_for(n, 128), 128, 0, s>>>(a, ca, b, cb, out, out32, n);
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}
