// Learned warm start (an extension: the paper has no learned component).
//
// A fully connected network maps a problem's data parameters (e.g. a wavepacket's centre, width and
// momentum) to coordinates c in a real orthonormal basis of the solution space; x0 = Q^T c (optionally times
// a per-problem complex phase) starts PCG, which stays the arbiter of the result.
//   * basis: randomized subspace iteration on the snapshot matrix Y whose rows are solutions the solver
//     produced (Halko, Martinsson and Tropp 2011, Alg. 4.4); every orthonormalization is CholeskyQR2 with the
//     Gram matrices accumulated in FP64;
//   * network: tanh hidden layers, weights kept as an FP32 master copy (Adam moments beside it) and a BF16
//     copy that every product reads; products accumulate in FP32; loss = mean weighted squared error;
//     backpropagation and Adam (Kingma and Ba 2015) run in the kernels below;
//   * solve: PCG from x0 behind a device-side guard that restarts from x0 = 0 when ||f - A x0|| >= ||f||.
#include "common.cuh"
#include <cmath>
#include <new>
#include <vector>

// ---- generic tiled product: C = alpha op(A) op(B) + beta C --------------------------------------------
// A(m, k) = A[m sam + k sak], B(k, n) = B[k sbk + n sbn], C(m, n) = C[m scm + n scn] with any strides.
// 64 x 64 output tile per CTA, k in chunks of 16 staged through shared memory (each operand loaded along
// its contiguous index), 4 x 4 outputs per thread, accumulation in TACC.
// Split-K: blockIdx.y = slice z covers k in [z kchunk, (z + 1) kchunk) and writes C + z scz.
template <typename TA, typename TB, typename TC>
struct GemmArgs {
  int M, N, K;
  float alpha, beta;
  const TA *A;
  long long sam, sak;
  const TB *B;
  long long sbk, sbn;
  TC *C;
  long long scm, scn;
  int kchunk;
  long long scz;
};

template <typename T>
__device__ __forceinline__ T ws_cvt(float v) { return (T)v; }
template <typename T>
__device__ __forceinline__ T ws_cvt(double v) { return (T)v; }
template <typename T>
__device__ __forceinline__ T ws_cvt(__nv_bfloat16 v) { return (T)__bfloat162float(v); }

// Accumulation modes: float, double, or MixedAcc = FP32 products summed in FP32 over each 16-term chunk
// of k and the chunk sums added in FP64 (FP64 throughput on this GPU is ~1/60 of FP32, so full FP64 FMAs
// are kept for the Gram matrices whose accuracy CholeskyQR needs).
struct MixedAcc {};
template <typename T>
struct AccT {
  typedef T smem_t;
  typedef T acc_t;
  static constexpr bool mixed = false;
};
template <>
struct AccT<MixedAcc> {
  typedef float smem_t;
  typedef double acc_t;
  static constexpr bool mixed = true;
};

template <typename TA, typename TB, typename TACC, typename TC>
__global__ void __launch_bounds__(256) k_ws_gemm(GemmArgs<TA, TB, TC> g) {
  typedef typename AccT<TACC>::smem_t TS;
  typedef typename AccT<TACC>::acc_t TR;
  __shared__ TS sA[16][65];
  __shared__ TS sB[16][65];
  const int tid = threadIdx.x;
  const int tiles_m = (g.M + 63) >> 6;
  const int m0 = (int)(blockIdx.x % tiles_m) * 64, n0 = (int)(blockIdx.x / tiles_m) * 64;
  const int kb = blockIdx.y * g.kchunk, ke = min(g.K, kb + g.kchunk);
  const int tm = (tid >> 4) * 4, tn = (tid & 15) * 4;
  const bool a_kfast = g.sak == 1, b_kfast = g.sbk == 1;
  TR acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = (TR)0;
  for (int k0 = kb; k0 < ke; k0 += 16) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + 256 * q;
      int kk = a_kfast ? (e & 15) : (e >> 6);
      const int mm = a_kfast ? (e >> 4) : (e & 63);
      const int m = m0 + mm;
      int k = k0 + kk;
      sA[kk][mm] = (m < g.M && k < ke) ? ws_cvt<TS>(g.A[(long long)m * g.sam + (long long)k * g.sak]) : (TS)0;
      kk = b_kfast ? (e & 15) : (e >> 6);
      const int nn = b_kfast ? (e >> 4) : (e & 63);
      const int n = n0 + nn;
      k = k0 + kk;
      sB[kk][nn] = (n < g.N && k < ke) ? ws_cvt<TS>(g.B[(long long)k * g.sbk + (long long)n * g.sbn]) : (TS)0;
    }
    __syncthreads();
    TS part[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) part[i][j] = (TS)0;
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      TS a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = sA[kk][tm + q];
        b[q] = sB[kk][tn + q];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) part[i][j] += a[i] * b[j];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] += (TR)part[i][j];
    __syncthreads();
  }
  TC *C = g.C + (long long)blockIdx.y * g.scz;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + tm + i, n = n0 + tn + j;
      if (m < g.M && n < g.N) {
        TC *c = &C[(long long)m * g.scm + (long long)n * g.scn];
        TR v = (TR)g.alpha * acc[i][j];
        if (g.beta != 0.f) v += (TR)g.beta * (TR)*c;
        *c = (TC)v;
      }
    }
}

template <typename TACC, typename TA, typename TB, typename TC>
static int ws_gemm(int M, int N, int K, float alpha, const TA *A, long long sam, long long sak, const TB *B,
                   long long sbk, long long sbn, float beta, TC *C, long long scm, long long scn, cudaStream_t s,
                   int kslices = 1, long long scz = 0) {
  if (M <= 0 || N <= 0) return STST_OK;
  const long long tiles = (long long)((M + 63) / 64) * ((N + 63) / 64);
  if (tiles > 0x7fffffffLL || kslices < 1 || kslices > 65535 || K < 0) return STST_ERR_ARG;
  GemmArgs<TA, TB, TC> g;
  g.M = M;
  g.N = N;
  g.K = K;
  g.alpha = alpha;
  g.beta = beta;
  g.A = A;
  g.sam = sam;
  g.sak = sak;
  g.B = B;
  g.sbk = sbk;
  g.sbn = sbn;
  g.C = C;
  g.scm = scm;
  g.scn = scn;
  g.kchunk = ((K + kslices - 1) / kslices + 15) / 16 * 16;
  g.scz = scz;
  dim3 grid((unsigned)tiles, (unsigned)kslices);
  STST_PROF("ws_gemm", s);
  k_ws_gemm<TA, TB, TACC, TC><<<grid, 256, 0, s>>>(g);
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}

// ---- elementwise pieces of the network -----------------------------------------------------------
// Z(m, n) += b[m] (feature-major, row stride N), then tanh in place when act
__global__ void k_ws_bias_act(float *Z, const float *b, int M, int N, int act) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)M * N) return;
  const float v = Z[e] + b[(int)(e / N)];
  Z[e] = act ? tanhf(v) : v;
}

// rows idx[n] of X (.. x dx), T (.. x dt) and of the weights -> the contiguous batch
__global__ void k_ws_gather(const float *X, int dx, const float *T, int dt, const float *w, const int *idx, int batch,
                            float *Xb, float *Tb, float *wb) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nx = (long long)batch * dx, nt = (long long)batch * dt;
  if (e < nx) {
    const int n = (int)(e / dx), j = (int)(e % dx);
    Xb[e] = X[(long long)idx[n] * dx + j];
  } else if (e < nx + nt) {
    const long long f = e - nx;
    const int n = (int)(f / dt), j = (int)(f % dt);
    Tb[f] = T[(long long)idx[n] * dt + j];
  } else if (e < nx + nt + batch) {
    const int n = (int)(e - nx - nt);
    wb[n] = w ? w[idx[n]] : 1.f;
  }
}

__device__ __forceinline__ double ws_block_sum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
  return t;  // valid in thread 0
}

// Y: D x B (feature-major), T: B x D (row-major). dY = 2 w_n (Y - T) / B; per-CTA partials of w_n (Y - T)^2
__global__ void k_ws_loss(const float *Y, const float *T, const float *w, int D, int B, float *dY, double *part) {
  __shared__ double sh[32];
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double v = 0.0;
  if (e < (long long)D * B) {
    const int k = (int)(e / B), n = (int)(e % B);
    const float wn = w ? w[n] : 1.f;
    const float r = Y[e] - T[(long long)n * D + k];
    dY[e] = 2.f * wn * r / (float)B;
    v = (double)wn * (double)r * (double)r;
  }
  v = ws_block_sum(v, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = v;
}

__global__ void k_ws_loss_final(const double *part, int nparts, int B, double *loss) {
  __shared__ double sh[32];
  double v = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) v += part[i];
  v = ws_block_sum(v, sh);
  if (threadIdx.x == 0) *loss = v / B;
}

// dH <- dH (1 - H^2): the derivative of tanh through its output
__global__ void k_ws_tanh_back(float *dH, const float *H, long long n) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e < n) dH[e] *= 1.f - H[e] * H[e];
}

// db[m] = sum_n dZ[m, n]: one warp per row, fixed order
__global__ void k_ws_rowsum(const float *dZ, int M, int N, float *db) {
  const int m = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (m >= M) return;
  float s = 0.f;
  for (int n = lane; n < N; n += 32) s += dZ[(long long)m * N + n];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) db[m] = s;
}

// Adam on the FP32 master copy, then the BF16 copy of the weights (bias slots of the copy stay 0)
__global__ void k_ws_adam(float *w, __nv_bfloat16 *wb, const unsigned char *is_weight, const float *g, float *m,
                          float *v, long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float gi = g[e];
  const float mi = b1 * m[e] + (1.f - b1) * gi;
  const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
  m[e] = mi;
  v[e] = vi;
  const float wi = w[e] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[e] = wi;
  wb[e] = __float2bfloat16(is_weight[e] ? wi : 0.f);
}

// effective parameters: weights from the BF16 copy, biases from the master copy
__global__ void k_ws_effective(const float *w, const __nv_bfloat16 *wb, const unsigned char *is_weight, float *out,
                               long long n) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e < n) out[e] = is_weight[e] ? __bfloat162float(wb[e]) : w[e];
}

__global__ void k_ws_set(const float *in, float *w, __nv_bfloat16 *wb, const unsigned char *is_weight, long long n) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float v = in[e];
  w[e] = v;
  wb[e] = __float2bfloat16(is_weight[e] ? v : 0.f);
}

// N(0, scale^2) numbers: Box-Muller transform of a counter-based hash (the splitmix64 finalizer)
__host__ __device__ __forceinline__ unsigned long long ws_mix(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
__global__ void k_ws_gauss(float *out, long long n, unsigned long long seed, float scale) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const unsigned long long h1 = ws_mix(seed ^ ws_mix(2ull * e)), h2 = ws_mix(seed ^ ws_mix(2ull * e + 1));
  const double u1 = ((double)(h1 >> 11) + 1.0) * (1.0 / 9007199254740992.0);  // (0, 1]
  const double u2 = (double)(h2 >> 11) * (1.0 / 9007199254740992.0);          // [0, 1)
  out[e] = (float)(scale * sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
}

// ---- CholeskyQR pieces (FP64) ------------------------------------------------------------------------
// G = R^T R in place (K x K row-major): upper triangle out, lower zeroed. flag |= 1 when a pivot falls to
// 1e-12 of its diagonal entry or below (a row of Z within ~1e-6 of the span of the rows before it: below
// the FP32 resolution of Z, so the directions are not independent). dorig: K doubles of scratch.
__global__ void __launch_bounds__(1024) k_ws_cholesky(double *G, int K, double *dorig, int *flag) {
  __shared__ double piv;
  __shared__ int bad;
  for (int j = threadIdx.x; j < K; j += blockDim.x) dorig[j] = G[(long long)j * K + j];
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < K; ++j) {
    if (threadIdx.x == 0) {
      double d = G[(long long)j * K + j];
      if (!(d > 1e-12 * dorig[j]) || bad) {
        bad = 1;
        d = 1.0;
      }
      piv = sqrt(d);
      G[(long long)j * K + j] = piv;
    }
    __syncthreads();
    const double pj = piv;
    for (int c = j + 1 + threadIdx.x; c < K; c += blockDim.x) G[(long long)j * K + c] /= pj;
    __syncthreads();
    const int rem = K - j - 1;
    for (long long e = threadIdx.x; e < (long long)rem * rem; e += blockDim.x) {
      const int r = j + 1 + (int)(e / rem), c = j + 1 + (int)(e % rem);
      if (c >= r) G[(long long)r * K + c] -= G[(long long)j * K + r] * G[(long long)j * K + c];
    }
    __syncthreads();
  }
  for (long long e = threadIdx.x; e < (long long)K * K; e += blockDim.x)
    if (e / K > e % K) G[e] = 0.0;
  if (threadIdx.x == 0 && bad) atomicOr(flag, 1);
}

// X = R^{-1} for upper triangular R (K x K row-major): one thread per column, back substitution
__global__ void k_ws_trinv(const double *R, int K, double *X) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= K) return;
  for (int i = K - 1; i >= 0; --i) {
    double v = 0.0;
    if (i == j) {
      v = 1.0 / R[(long long)j * K + j];
    } else if (i < j) {
      double s = 0.0;
      for (int k = i + 1; k <= j; ++k) s += R[(long long)i * K + k] * X[(long long)k * K + j];
      v = -s / R[(long long)i * K + i];
    }
    X[(long long)i * K + j] = v;
  }
}

// G = sum over the split-K slices (upper triangle mirrored to make G exactly symmetric)
__global__ void k_ws_sum_slices(const double *S, int slices, int K, double *G) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)K * K) return;
  const int r = (int)(e / K), c = (int)(e % K);
  const long long src = r <= c ? e : (long long)c * K + r;
  double s = 0.0;
  for (int z = 0; z < slices; ++z) s += S[(long long)z * K * K + src];
  G[e] = s;
}

static int gram_slices(int K, long long m) {
  const long long tiles = (long long)((K + 63) / 64) * ((K + 63) / 64);
  long long s = (4 * 152 + tiles - 1) / tiles;
  const long long smax = (m + 1023) / 1024;
  if (s > smax) s = smax;
  if (s < 1) s = 1;
  if (s > 64) s = 64;
  return (int)s;
}

// Rows of Z (K x m FP32, row-major) made orthonormal by two CholeskyQR passes (Gram in FP64); Zb is a
// second K x m buffer; the result ends in Z. work: >= slices K^2 + 2 K^2 + K doubles.
static int ws_orth_rows(float *Z, float *Zb, int K, long long m, double *work, int *flag, cudaStream_t s) {
  if (m > 0x7fffffffLL) return STST_ERR_ARG;
  const int slices = gram_slices(K, m);
  double *S = work, *G = work + (long long)slices * K * K, *Ri = G + (long long)K * K, *dg = Ri + (long long)K * K;
  float *src = Z, *dst = Zb;
  for (int pass = 0; pass < 2; ++pass) {
    STST_TRY(ws_gemm<double>(K, K, (int)m, 1.f, src, m, 1, src, 1, m, 0.f, S, K, 1, s, slices, (long long)K * K));
    k_ws_sum_slices<<<grid_for((long long)K * K, 256), 256, 0, s>>>(S, slices, K, G);
    k_ws_cholesky<<<1, 1024, 0, s>>>(G, K, dg, flag);
    k_ws_trinv<<<(K + 127) / 128, 128, 0, s>>>(G, K, Ri);
    // dst(k, j) = sum_i Ri[i][k] src(i, j), i.e. dst = R^{-T} src
    STST_TRY(ws_gemm<double>(K, (int)m, K, 1.f, Ri, 1, K, src, m, 1, 0.f, dst, m, 1, s));
    float *t = src;
    src = dst;
    dst = t;
  }
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}

// ---- guarded warm start --------------------------------------------------------------------------------
__global__ void k_ws_sqnorm(const double2 *v, long long n, double *part) {
  __shared__ double sh[32];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s += v[i].x * v[i].x + v[i].y * v[i].y;
  s = ws_block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// keep = (||f - A x0||^2 < ||f||^2 and finite); the partials are reduced in a fixed order
__global__ void k_ws_guard(const double *prr, const double *pff, int np, int *keep) {
  __shared__ double sh[32];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    a += prr[i];
    b += pff[i];
  }
  a = ws_block_sum(a, sh);
  __syncthreads();
  b = ws_block_sum(b, sh);
  if (threadIdx.x == 0) *keep = (isfinite(a) && a < b) ? 1 : 0;
}

__global__ void k_ws_zero_unless(double2 *x, long long n, const int *keep) {
  if (*keep) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = make_double2(0.0, 0.0);
}

// rows of X (m reals = m/2 complex values each) times e^{i phase[row]}
__global__ void k_ws_rotate(double *X, int rows, long long half, const double *phase) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)rows * half) return;
  double sn, cs;
  sincos(phase[e / half], &sn, &cs);
  double2 *p = reinterpret_cast<double2 *>(X) + e;
  const double2 v = *p;
  *p = make_double2(cs * v.x - sn * v.y, sn * v.x + cs * v.y);
}

// ---- small-batch layer product (inference) ------------------------------------------------------------------
#define WS_GEMV_MAXB 8
// Z (dout x B, feature-major) = W (dout x din, BF16 row-major) x, with x(k, b) = X[k sxk + b sxb]:
// one warp per output row reads its weights once (coalesced, 8 BF16 per lane per step), FP32 sums.
__global__ void __launch_bounds__(256) k_ws_gemv(const __nv_bfloat16 *__restrict__ W, int dout, int din,
                                                 const float *__restrict__ X, long long sxk, long long sxb, int B,
                                                 float *Z) {
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= dout) return;
  const __nv_bfloat16 *w = W + (long long)row * din;
  float acc[WS_GEMV_MAXB];
#pragma unroll
  for (int b = 0; b < WS_GEMV_MAXB; ++b) acc[b] = 0.f;
  for (int k = lane; k < din; k += 32) {
    const float wk = __bfloat162float(w[k]);
#pragma unroll
    for (int b = 0; b < WS_GEMV_MAXB; ++b)
      if (b < B) acc[b] += wk * __ldg(&X[(long long)k * sxk + (long long)b * sxb]);
  }
#pragma unroll
  for (int b = 0; b < WS_GEMV_MAXB; ++b) {
    float v = acc[b];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0 && b < B) Z[(long long)row * B + b] = v;
  }
}

// Y (B x D, row-major) = scale (.) H (D x B, feature-major) + beta Y
__global__ void k_ws_output(const float *H, int D, int B, const float *scale, float beta, float *Y) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)D * B) return;
  const int n = (int)(e / D), k = (int)(e % D);
  float v = H[(long long)k * B + n];
  if (scale) v *= scale[k];
  Y[e] = v + (beta != 0.f ? beta * Y[e] : 0.f);
}

// ---- few-row projection and expansion (inference of a handful of problems) -------------------------------
// The tiled product wastes 63/64 of its work when n = 1; these read the basis once (HBM-bound).
#define WS_ROWS_PROJ 8
#define WS_ROWS_EXP 8

// C (n x K) = Y (n x m) Q^T: one warp per basis row, lanes over pairs of columns (float2 / double2 loads:
// m even, 16-byte aligned bases); FP32 products summed in FP32 over 64 pairs per lane, then in FP64.
template <int NR>
__global__ void __launch_bounds__(256) k_pod_project_rows(const double *__restrict__ Y, int n, long long m,
                                                          const float *__restrict__ Q, int K, float *C) {
  const int k = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (k >= K) return;
  const long long half = m >> 1;
  const float2 *q = reinterpret_cast<const float2 *>(Q + (long long)k * m);
  double acc[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) acc[r] = 0.0;
  for (long long j0 = lane; j0 < half; j0 += 32 * 64) {
    float part[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) part[r] = 0.f;
    const long long j1 = min(half, j0 + 32 * 64);
#pragma unroll 4
    for (long long j = j0; j < j1; j += 32) {
      const float2 qv = __ldg(q + j);
#pragma unroll
      for (int r = 0; r < NR; ++r)
        if (r < n) {
          const double2 y = __ldg(reinterpret_cast<const double2 *>(Y + (long long)r * m) + j);
          part[r] += (float)y.x * qv.x + (float)y.y * qv.y;
        }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] += (double)part[r];
  }
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    double v = acc[r];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0 && r < n) C[(long long)r * K + k] = (float)v;
  }
}

// X (n x m) = alpha C (n x K) Q (K x m) + beta X: one thread per 4 columns (float4 loads of Q, 8 or 16
// basis rows in flight), C in shared memory; FP32 products summed in FP32 over 32 basis rows, then in FP64.
template <int NR>
__global__ void __launch_bounds__(256) k_pod_expand_rows(const float *__restrict__ Q, int K, long long m,
                                                         const float *__restrict__ C, int n, float alpha, float beta,
                                                         double *X) {
  extern __shared__ float sC[];  // n x K
  for (int e = threadIdx.x; e < n * K; e += blockDim.x) sC[e] = C[e];
  __syncthreads();
  const long long c4 = blockIdx.x * 256LL + threadIdx.x;  // column quad
  if (c4 * 4 >= m) return;
  const float4 *q = reinterpret_cast<const float4 *>(Q) + c4;
  const long long step = m >> 2;  // float4 per basis row
  double acc[NR][4];
#pragma unroll
  for (int r = 0; r < NR; ++r)
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[r][i] = 0.0;
  for (int k0 = 0; k0 < K; k0 += 32) {
    const int k1 = min(K, k0 + 32);
    float part[NR][4];
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int i = 0; i < 4; ++i) part[r][i] = 0.f;
    // UNR basis rows in flight per thread: the grid has only m/1024 CTAs, so the loads of one thread
    // must cover the HBM latency (16 rows of 16 bytes for one or two right-hand sides)
    constexpr int UNR = NR <= 2 ? 16 : 8;
    int k = k0;
    for (; k + UNR <= k1; k += UNR) {
      float4 qv[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) qv[u] = __ldg(q + (long long)(k + u) * step);
#pragma unroll
      for (int u = 0; u < UNR; ++u)
#pragma unroll
        for (int r = 0; r < NR; ++r)
          if (r < n) {
            const float c = sC[r * K + k + u];
            part[r][0] += c * qv[u].x;
            part[r][1] += c * qv[u].y;
            part[r][2] += c * qv[u].z;
            part[r][3] += c * qv[u].w;
          }
    }
    for (; k < k1; ++k) {
      const float4 qv = __ldg(q + (long long)k * step);
#pragma unroll
      for (int r = 0; r < NR; ++r)
        if (r < n) {
          const float c = sC[r * K + k];
          part[r][0] += c * qv.x;
          part[r][1] += c * qv.y;
          part[r][2] += c * qv.z;
          part[r][3] += c * qv.w;
        }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[r][i] += (double)part[r][i];
  }
#pragma unroll
  for (int r = 0; r < NR; ++r)
    if (r < n) {
      double2 *x = reinterpret_cast<double2 *>(X + (long long)r * m + c4 * 4);
      double2 a = make_double2((double)alpha * acc[r][0], (double)alpha * acc[r][1]);
      double2 b = make_double2((double)alpha * acc[r][2], (double)alpha * acc[r][3]);
      if (beta != 0.f) {
        const double2 xa = x[0], xb = x[1];
        a.x += (double)beta * xa.x;
        a.y += (double)beta * xa.y;
        b.x += (double)beta * xb.x;
        b.y += (double)beta * xb.y;
      }
      x[0] = a;
      x[1] = b;
    }
}

static bool aligned16(const void *p) { return ((unsigned long long)p & 15ull) == 0; }

// ---- network state -------------------------------------------------------------------------------------
#define STST_WS_MAXL 8
#define STST_WS_MAGIC 0x57534D44

struct stst_ws_s {
  int magic;
  int L;
  int sizes[STST_WS_MAXL + 1];
  int max_batch;
  cudaStream_t stream;
  int own_stream;
  long long woff[STST_WS_MAXL], boff[STST_WS_MAXL], n_params;
  float *w, *g, *am, *av;       // master parameters, gradient, Adam moments
  __nv_bfloat16 *wb;            // BF16 copy read by the products (bias slots hold 0)
  unsigned char *is_weight;     // 1 for weight entries, 0 for biases
  int step;                     // Adam step count
  float *H[STST_WS_MAXL + 1];   // activations, feature-major (width x batch); H[L] is the output
  float *dA, *dB;               // back-propagated signals (ping-pong)
  float *Xb, *Tb, *wbatch;      // the gathered batch
  double *part, *loss_dev, *loss_host;
  float *out_scale;             // per-output scale of stst_ws_forward (NULL: none)
};

static void ws_free(stst_ws_s *w) {
  if (!w) return;
  if (w->stream) cudaStreamSynchronize(w->stream);
  void *ptrs[] = {w->w, w->g, w->am, w->av, w->wb, w->is_weight, w->dA, w->dB, w->Xb, w->Tb, w->wbatch, w->part,
                  w->loss_dev, w->out_scale};
  for (void *p : ptrs) cudaFree(p);
  for (int l = 1; l <= w->L; ++l) cudaFree(w->H[l]);
  if (w->loss_host) cudaFreeHost(w->loss_host);
  if (w->own_stream) cudaStreamDestroy(w->stream);
  w->magic = 0;
  delete w;
}

static bool ws_ok(const stst_ws_s *w) { return w && w->magic == STST_WS_MAGIC; }

// forward pass for X (B x sizes[0], row-major); the output lands in H[L] (sizes[L] x B)
static int ws_forward(stst_ws_s *w, const float *X, int B) {
  cudaStream_t s = w->stream;
  for (int l = 0; l < w->L; ++l) {
    const int din = w->sizes[l], dout = w->sizes[l + 1];
    const __nv_bfloat16 *W = w->wb + w->woff[l];
    const float *x = l == 0 ? X : w->H[l];
    const long long sxk = l == 0 ? 1 : B, sxb = l == 0 ? din : 1;
    if (B <= WS_GEMV_MAXB) {
      k_ws_gemv<<<(dout + 7) / 8, 256, 0, s>>>(W, dout, din, x, sxk, sxb, B, w->H[l + 1]);
    } else {
      STST_TRY(ws_gemm<float>(dout, B, din, 1.f, W, din, 1, x, sxk, sxb, 0.f, w->H[l + 1], B, 1, s));
    }
    k_ws_bias_act<<<grid_for((long long)dout * B, 256), 256, 0, s>>>(w->H[l + 1], w->w + w->boff[l], dout, B,
                                                                    l + 1 < w->L);
  }
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}

// loss into loss_dev and dL/d(effective parameters) into g, for the batch (X, T, wt) after a forward pass
static int ws_backward(stst_ws_s *w, const float *X, const float *T, const float *wt, int B) {
  cudaStream_t s = w->stream;
  const int L = w->L, Dout = w->sizes[L];
  const int nb = grid_for((long long)Dout * B, 256);
  if (nb > STST_MAXPART) return STST_ERR_ARG;
  k_ws_loss<<<nb, 256, 0, s>>>(w->H[L], T, wt, Dout, B, w->dA, w->part);
  k_ws_loss_final<<<1, 1024, 0, s>>>(w->part, nb, B, w->loss_dev);
  float *dZ = w->dA, *dN = w->dB;
  for (int l = L - 1; l >= 0; --l) {
    const int din = w->sizes[l], dout = w->sizes[l + 1];
    float *gW = w->g + w->woff[l], *gb = w->g + w->boff[l];
    // gW = dZ H_l^T (dout x din), reduction over the batch
    if (l == 0)
      STST_TRY(ws_gemm<float>(dout, din, B, 1.f, dZ, B, 1, X, din, 1, 0.f, gW, din, 1, s));
    else
      STST_TRY(ws_gemm<float>(dout, din, B, 1.f, dZ, B, 1, w->H[l], 1, B, 0.f, gW, din, 1, s));
    k_ws_rowsum<<<(dout + 7) / 8, 256, 0, s>>>(dZ, dout, B, gb);
    if (l > 0) {
      // dH_l = W_l^T dZ (din x B), then through tanh
      const __nv_bfloat16 *W = w->wb + w->woff[l];
      STST_TRY(ws_gemm<float>(din, B, dout, 1.f, W, 1, din, dZ, B, 1, 0.f, dN, B, 1, s));
      k_ws_tanh_back<<<grid_for((long long)din * B, 256), 256, 0, s>>>(dN, w->H[l], (long long)din * B);
      float *t = dZ;
      dZ = dN;
      dN = t;
    }
  }
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}

static int ws_loss_grad(stst_ws_s *w, const float *X, const float *T, const float *wt, const int *idx, int B) {
  if (B < 1 || B > w->max_batch || !X || !T) return STST_ERR_ARG;
  const float *Xu = X, *Tu = T, *wu = wt;
  if (idx) {
    const int dx = w->sizes[0], dt = w->sizes[w->L];
    const long long tot = (long long)B * (dx + dt + 1);
    k_ws_gather<<<grid_for(tot, 256), 256, 0, w->stream>>>(X, dx, T, dt, wt, idx, B, w->Xb, w->Tb, w->wbatch);
    Xu = w->Xb;
    Tu = w->Tb;
    wu = w->wbatch;
  }
  STST_TRY(ws_forward(w, Xu, B));
  return ws_backward(w, Xu, Tu, wu, B);
}

static int ws_read_loss(stst_ws_s *w, double *loss) {
  if (!loss) return STST_OK;
  STST_CUDA(cudaMemcpyAsync(w->loss_host, w->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, w->stream));
  STST_CUDA(cudaStreamSynchronize(w->stream));
  *loss = *w->loss_host;
  return STST_OK;
}

// ---- training-data preparation (the cascade of a9: whitening, scalings, residual targets) ----------------
// Per-column sums of squares of X (n x K row-major FP32 or FP64), one thread per column, rows in order (FP64):
// colss[k] = sum_n X[n][k]^2.
template <typename T>
__global__ void k_ws_colss(const T *X, int n, int K, double *colss) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  double s = 0.0;
  for (int r = 0; r < n; ++r) {
    const double v = (double)X[(long long)r * K + k];
    s += v * v;
  }
  colss[k] = s;
}

// Per-row sums of squares: one warp per row, lanes over the columns, then a fixed shuffle order.
__global__ void k_ws_rowss(const float *X, int n, int K, double *rowss) {
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (r >= n) return;
  double s = 0.0;
  for (int k = lane; k < K; k += 32) {
    const double v = (double)X[(long long)r * K + k];
    s += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) rowss[r] = s;
}

// so[k] = max(sqrt(colss[k] / n), 1e-300); w[r] = mean(rowss) / max(rowss[r], 1e-300) (one CTA: the mean is
// summed in a fixed order).
__global__ void k_ws_target_scale(int n, int K, const double *colss, const double *rowss, double *so, float *w) {
  __shared__ double part[1024];
  __shared__ double mean;
  double acc = 0.0;
  for (int r = threadIdx.x; r < n; r += blockDim.x) acc += rowss[r];
  part[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) t += part[i];
    mean = t / n;
  }
  for (int k = threadIdx.x; k < K; k += blockDim.x) so[k] = fmax(sqrt(colss[k] / n), 1e-300);
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += blockDim.x) w[r] = (float)(mean / fmax(rowss[r], 1e-300));
}

// Ts = T / so, column by column (n x K row-major)
__global__ void k_ws_scale_cols(const float *T, int n, int K, const double *so, float *Ts) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * K;
       e += (long long)gridDim.x * blockDim.x)
    Ts[e] = (float)((double)T[e] / so[e % K]);
}

// G += shift I, shift = rel * max_k G[k][k] (a symmetric positive semidefinite Gram matrix becomes definite)
__global__ void k_ws_shift_diag(double *G, int K, double rel) {
  __shared__ double mx;
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int k = 0; k < K; ++k) m = fmax(m, G[(long long)k * K + k]);
    mx = m;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += blockDim.x) G[(long long)k * K + k] += rel * mx;
}

// One stage of the cascade, elementwise (resid: n x K FP64): with T0, resid = T0 and scale = 1; otherwise
// resid -= Y (.) scale_prev. Then targets = resid / scale (scale from k_ws_cascade_scale).
__global__ void k_ws_cascade_resid(double *resid, const float *T0, const float *Y, const double *scale_prev, int n,
                                   int K) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * K;
       e += (long long)gridDim.x * blockDim.x) {
    if (T0) resid[e] = (double)T0[e];
    else resid[e] -= (double)Y[e] * scale_prev[e % K];
  }
}

__global__ void k_ws_cascade_out(const double *resid, const double *colss, int n, int K, int first, double *scale,
                                 float *targets, const double *so, float *out_scale) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * K;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e % K);
    const double sc = first ? 1.0 : fmax(sqrt(colss[k] / n), 1e-30);
    targets[e] = (float)(resid[e] / sc);
    if (e < K) {
      scale[e] = first ? 1.0 : fmax(sqrt(colss[e] / n), 1e-30);
      out_scale[e] = (float)(so[e] * scale[e]);
    }
  }
}

struct DevTemp {  // stream-ordered temporaries of the offline basis construction
  cudaStream_t s;
  std::vector<void *> ptrs;
  explicit DevTemp(cudaStream_t st) : s(st) {}
  void *get(size_t bytes) {
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes ? bytes : 16, s) != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    return p;
  }
  ~DevTemp() {
    for (void *p : ptrs) cudaFreeAsync(p, s);
  }
};

extern "C" {

int stst_ws_create(stst_ws *out, int n_layers, const int *sizes, int max_batch, unsigned long long seed,
                   void *stream) {
  if (!out || !sizes || n_layers < 1 || n_layers > STST_WS_MAXL || max_batch < 1) return STST_ERR_ARG;
  *out = nullptr;
  int maxw = 0;
  for (int l = 0; l <= n_layers; ++l) {
    if (sizes[l] < 1 || sizes[l] > (1 << 20)) return STST_ERR_ARG;
    maxw = sizes[l] > maxw ? sizes[l] : maxw;
  }
  if ((long long)maxw * max_batch > (1LL << 31)) return STST_ERR_ARG;
  stst_ws_s *w = new (std::nothrow) stst_ws_s();
  if (!w) return STST_ERR_OOM;
  w->magic = STST_WS_MAGIC;
  w->L = n_layers;
  for (int l = 0; l <= n_layers; ++l) w->sizes[l] = sizes[l];
  w->max_batch = max_batch;
  w->stream = (cudaStream_t)stream;  // NULL: the legacy default stream
  long long tot = 0;
  for (int l = 0; l < n_layers; ++l) {
    w->woff[l] = tot;
    tot += (long long)sizes[l + 1] * sizes[l];
    w->boff[l] = tot;
    tot += sizes[l + 1];
  }
  w->n_params = tot;
  bool ok = true;
  auto al = [&](void **p, size_t bytes) {
    if (ok && cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) ok = false;
  };
  al((void **)&w->w, sizeof(float) * tot);
  al((void **)&w->g, sizeof(float) * tot);
  al((void **)&w->am, sizeof(float) * tot);
  al((void **)&w->av, sizeof(float) * tot);
  al((void **)&w->wb, sizeof(__nv_bfloat16) * tot);
  al((void **)&w->is_weight, (size_t)tot);
  for (int l = 1; l <= n_layers; ++l) al((void **)&w->H[l], sizeof(float) * (size_t)sizes[l] * max_batch);
  al((void **)&w->dA, sizeof(float) * (size_t)maxw * max_batch);
  al((void **)&w->dB, sizeof(float) * (size_t)maxw * max_batch);
  al((void **)&w->Xb, sizeof(float) * (size_t)sizes[0] * max_batch);
  al((void **)&w->Tb, sizeof(float) * (size_t)sizes[n_layers] * max_batch);
  al((void **)&w->wbatch, sizeof(float) * (size_t)max_batch);
  al((void **)&w->part, sizeof(double) * STST_MAXPART);
  al((void **)&w->loss_dev, sizeof(double));
  if (ok && cudaMallocHost(&w->loss_host, sizeof(double)) != cudaSuccess) ok = false;
  if (!ok) {
    stst_last_cuda = cudaErrorMemoryAllocation;
    ws_free(w);
    return STST_ERR_OOM;
  }
  cudaStream_t s = w->stream;
  std::vector<unsigned char> isw((size_t)tot, 0);
  for (int l = 0; l < n_layers; ++l)
    for (long long e = w->woff[l]; e < w->boff[l]; ++e) isw[(size_t)e] = 1;
  int st = STST_OK;
  if (cudaMemcpyAsync(w->is_weight, isw.data(), (size_t)tot, cudaMemcpyHostToDevice, s) != cudaSuccess)
    st = STST_ERR_CUDA;
  cudaMemsetAsync(w->w, 0, sizeof(float) * tot, s);
  cudaMemsetAsync(w->g, 0, sizeof(float) * tot, s);
  cudaMemsetAsync(w->am, 0, sizeof(float) * tot, s);
  cudaMemsetAsync(w->av, 0, sizeof(float) * tot, s);
  // weights ~ N(0, 1 / fan_in), biases 0
  for (int l = 0; l < n_layers; ++l) {
    const long long n = (long long)sizes[l + 1] * sizes[l];
    k_ws_gauss<<<grid_for(n, 256), 256, 0, s>>>(w->w + w->woff[l], n, ws_mix(seed) + (unsigned long long)l,
                                                (float)(1.0 / sqrt((double)sizes[l])));
  }
  k_ws_set<<<grid_for(tot, 256), 256, 0, s>>>(w->w, w->w, w->wb, w->is_weight, tot);
  if (st == STST_OK && (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess))
    st = STST_ERR_CUDA;
  if (st != STST_OK) {
    ws_free(w);
    return st;
  }
  *out = w;
  return STST_OK;
}

int stst_ws_destroy(stst_ws w) {
  if (!ws_ok(w)) return STST_ERR_HANDLE;
  ws_free(w);
  return STST_OK;
}

int stst_ws_num_params(stst_ws w, long long *n) {
  if (!ws_ok(w)) return STST_ERR_HANDLE;
  if (!n) return STST_ERR_ARG;
  *n = w->n_params;
  return STST_OK;
}

int stst_ws_get_params(stst_ws w, float *params) {
  if (!ws_ok(w)) return STST_ERR_HANDLE;
  if (!params) return STST_ERR_ARG;
  k_ws_effective<<<grid_for(w->n_params, 256), 256, 0, w->stream>>>(w->w, w->wb, w->is_weight, params, w->n_params);
  STST_CUDA(cudaGetLastError());
  STST_CUDA(cudaStreamSynchronize(w->stream));
  return STST_OK;
}

int stst_ws_set_params(stst_ws w, const float *params) {
  if (!ws_ok(w)) return STST_ERR_HANDLE;
  if (!params) return STST_ERR_ARG;
  cudaStream_t s = w->stream;
  k_ws_set<<<grid_for(w->n_params, 256), 256, 0, s>>>(params, w->w, w->wb, w->is_weight, w->n_params);
  STST_CUDA(cudaGetLastError());
  STST_CUDA(cudaMemsetAsync(w->am, 0, sizeof(float) * w->n_params, s));
  STST_CUDA(cudaMemsetAsync(w->av, 0, sizeof(float) * w->n_params, s));
  w->step = 0;
  STST_CUDA(cudaStreamSynchronize(s));
  return STST_OK;
}

int stst_ws_set_output_scale(stst_ws w, const float *scale) {
  if (!ws_ok(w)) return STST_ERR_HANDLE;
  const int D = w->sizes[w->L];
  if (!scale) {
    cudaFree(w->out_scale);
    w->out_scale = nullptr;
    return STST_OK;
  }
  if (!w->out_scale && cudaMalloc(&w->out_scale, sizeof(float) * D) != cudaSuccess) {
    w->out_scale = nullptr;
    stst_last_cuda = cudaErrorMemoryAllocation;
    return STST_ERR_OOM;
  }
  STST_CUDA(cudaMemcpyAsync(w->out_scale, scale, sizeof(float) * D, cudaMemcpyDefault, w->stream));
  STST_CUDA(cudaStreamSynchronize(w->stream));
  return STST_OK;
}

int stst_ws_forward(stst_ws w, const float *X, int batch, float *Y, float beta) {
  if (!ws_ok(w)) return STST_ERR_HANDLE;
  if (!X || !Y || batch < 1 || batch > w->max_batch) return STST_ERR_ARG;
  STST_TRY(ws_forward(w, X, batch));
  const int D = w->sizes[w->L];
  k_ws_output<<<grid_for((long long)D * batch, 256), 256, 0, w->stream>>>(w->H[w->L], D, batch, w->out_scale, beta,
                                                                          Y);
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}

int stst_ws_grad(stst_ws w, const float *X, const float *T, const float *weight, const int *idx, int batch,
                 float *grad, double *loss) {
  if (!ws_ok(w)) return STST_ERR_HANDLE;
  STST_TRY(ws_loss_grad(w, X, T, weight, idx, batch));
  if (grad)
    STST_CUDA(cudaMemcpyAsync(grad, w->g, sizeof(float) * w->n_params, cudaMemcpyDeviceToDevice, w->stream));
  return ws_read_loss(w, loss);
}

int stst_ws_train_step(stst_ws w, const float *X, const float *T, const float *weight, const int *idx, int batch,
                       float lr, double *loss) {
  if (!ws_ok(w)) return STST_ERR_HANDLE;
  if (!(lr >= 0.f)) return STST_ERR_ARG;
  STST_TRY(ws_loss_grad(w, X, T, weight, idx, batch));
  const double b1 = 0.9, b2 = 0.999;
  w->step += 1;
  const float c1 = (float)(1.0 - pow(b1, w->step)), c2 = (float)(1.0 - pow(b2, w->step));
  k_ws_adam<<<grid_for(w->n_params, 256), 256, 0, w->stream>>>(w->w, w->wb, w->is_weight, w->g, w->am, w->av,
                                                               w->n_params, lr, (float)b1, (float)b2, 1e-8f, c1, c2);
  STST_CUDA(cudaGetLastError());
  return ws_read_loss(w, loss);
}

int stst_pod_basis(const double *Y, int n, long long m, const float *Omega, int K, int power_its, float *Q,
                   void *stream) {
  if (!Y || !Omega || !Q || n < 1 || K < 1 || K > n || m < K || m > 0x7fffffffLL || power_its < 0 ||
      power_its > 8 || K > 4096)
    return STST_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int st = STST_OK;
  {
    DevTemp tmp(s);
    const int slices = gram_slices(K, m > n ? m : n);
    float *Zb = (float *)tmp.get(sizeof(float) * (size_t)K * m);
    float *Pt = power_its ? (float *)tmp.get(sizeof(float) * (size_t)K * n) : nullptr;
    float *Pb = power_its ? (float *)tmp.get(sizeof(float) * (size_t)K * n) : nullptr;
    double *work = (double *)tmp.get(sizeof(double) * (((size_t)slices + 2) * K * K + K));
    int *flag = (int *)tmp.get(sizeof(int));
    int flag_host = 0;
    if (!Zb || !work || !flag || (power_its && (!Pt || !Pb))) {
      stst_last_cuda = cudaErrorMemoryAllocation;
      st = STST_ERR_OOM;
    }
    if (st == STST_OK && cudaMemsetAsync(flag, 0, sizeof(int), s) != cudaSuccess) st = STST_ERR_CUDA;
    // Q = Omega^T Y (K x m), reduction over the n snapshots
    if (st == STST_OK) st = ws_gemm<float>(K, (int)m, n, 1.f, Omega, 1, K, Y, m, 1, 0.f, Q, m, 1, s);
    if (st == STST_OK) st = ws_orth_rows(Q, Zb, K, m, work, flag, s);
    for (int it = 0; st == STST_OK && it < power_its; ++it) {
      // Pt = Q Y^T (K x n), orthonormalized; Q = Pt Y (K x m), orthonormalized
      st = ws_gemm<float>(K, n, (int)m, 1.f, Q, m, 1, Y, 1, m, 0.f, Pt, n, 1, s);
      if (st == STST_OK) st = ws_orth_rows(Pt, Pb, K, n, work, flag, s);
      if (st == STST_OK) st = ws_gemm<float>(K, (int)m, n, 1.f, Pt, n, 1, Y, m, 1, 0.f, Q, m, 1, s);
      if (st == STST_OK) st = ws_orth_rows(Q, Zb, K, m, work, flag, s);
    }
    if (st == STST_OK && cudaMemcpyAsync(&flag_host, flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      st = STST_ERR_CUDA;
    if (st == STST_OK && cudaStreamSynchronize(s) != cudaSuccess) st = STST_ERR_CUDA;
    if (st == STST_OK && flag_host) st = STST_NOT_HPD;
  }
  if (st == STST_ERR_CUDA) stst_last_cuda = cudaGetLastError();
  return st;
}

int stst_pod_project(const double *Y, int n, long long m, const float *Q, int K, float *C, void *stream) {
  if (!Y || !Q || !C || n < 1 || K < 1 || m < 1 || m > 0x7fffffffLL) return STST_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (n <= WS_ROWS_PROJ && (m & 1) == 0 && aligned16(Y) && aligned16(Q)) {
    STST_PROF("pod_project_rows", s);
    const unsigned grid = (unsigned)((K + 7) / 8);
    if (n == 1)
      k_pod_project_rows<1><<<grid, 256, 0, s>>>(Y, n, m, Q, K, C);
    else if (n <= 2)
      k_pod_project_rows<2><<<grid, 256, 0, s>>>(Y, n, m, Q, K, C);
    else if (n <= 4)
      k_pod_project_rows<4><<<grid, 256, 0, s>>>(Y, n, m, Q, K, C);
    else
      k_pod_project_rows<8><<<grid, 256, 0, s>>>(Y, n, m, Q, K, C);
    STST_CUDA(cudaGetLastError());
    return STST_OK;
  }
  return ws_gemm<MixedAcc>(n, K, (int)m, 1.f, Y, m, 1, Q, 1, m, 0.f, C, K, 1, s);
}

int stst_pod_expand(const float *Q, int K, long long m, const float *C, int n, float alpha, float beta,
                    const double *phase, double *X, void *stream) {
  if (!Q || !C || !X || n < 1 || K < 1 || m < 1 || m > 0x7fffffffLL || (phase && (m & 1))) return STST_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t smem = sizeof(float) * (size_t)n * K;
  if (n <= WS_ROWS_EXP && smem <= 48 * 1024 && (m & 3) == 0 && aligned16(Q) && aligned16(X)) {
    STST_PROF("pod_expand_rows", s);
    const unsigned grid = (unsigned)((m / 4 + 255) / 256);
    if (n == 1)
      k_pod_expand_rows<1><<<grid, 256, smem, s>>>(Q, K, m, C, n, alpha, beta, X);
    else if (n <= 2)
      k_pod_expand_rows<2><<<grid, 256, smem, s>>>(Q, K, m, C, n, alpha, beta, X);
    else if (n <= 4)
      k_pod_expand_rows<4><<<grid, 256, smem, s>>>(Q, K, m, C, n, alpha, beta, X);
    else
      k_pod_expand_rows<8><<<grid, 256, smem, s>>>(Q, K, m, C, n, alpha, beta, X);
    STST_CUDA(cudaGetLastError());
  } else {
    STST_TRY(ws_gemm<MixedAcc>(n, (int)m, K, alpha, C, K, 1, Q, m, 1, beta, X, m, 1, s));
  }
  if (phase) {
    const long long half = m / 2;
    k_ws_rotate<<<grid_for((long long)n * half, 256), 256, 0, s>>>(X, n, half, phase);
    STST_CUDA(cudaGetLastError());
  }
  return STST_OK;
}

int stst_ws_whiten(const float *F, int n, int K, float *Fw, float *Q, long long m, void *stream) {
  if (!F || !Fw || n < 1 || K < 1 || K > 4096 || (Q && (m < 1 || m > 0x7fffffffLL))) return STST_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  DevTemp tmp(s);
  const int slices = gram_slices(K, n);
  double *S = (double *)tmp.get(sizeof(double) * (size_t)slices * K * K);
  double *G = (double *)tmp.get(sizeof(double) * (size_t)K * K);
  double *Ri = (double *)tmp.get(sizeof(double) * (size_t)K * K);
  double *dg = (double *)tmp.get(sizeof(double) * K);
  int *flag = (int *)tmp.get(sizeof(int));
  float *Qn = Q ? (float *)tmp.get(sizeof(float) * (size_t)K * m) : nullptr;
  if (!S || !G || !Ri || !dg || !flag || (Q && !Qn)) return STST_ERR_OOM;
  STST_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s));
  // G = F^T F / n in FP64 (split-K slices summed in a fixed order), a relative shift of 1e-10 of the largest
  // diagonal entry, G = R^T R, W = R^{-1}
  STST_TRY(ws_gemm<double>(K, K, n, 1.f / n, F, 1, K, F, K, 1, 0.f, S, K, 1, s, slices, (long long)K * K));
  k_ws_sum_slices<<<grid_for((long long)K * K, 256), 256, 0, s>>>(S, slices, K, G);
  k_ws_shift_diag<<<1, 256, 0, s>>>(G, K, 1e-10);
  k_ws_cholesky<<<1, 1024, 0, s>>>(G, K, dg, flag);
  k_ws_trinv<<<(K + 127) / 128, 128, 0, s>>>(G, K, Ri);
  // Fw(r, j) = sum_k F(r, k) W(k, j); Q(k, :) <- sum_i W(i, k) Q(i, :) (W^T Q)
  STST_TRY(ws_gemm<double>(n, K, K, 1.f, F, K, 1, Ri, K, 1, 0.f, Fw, K, 1, s));
  if (Q) {
    STST_TRY(ws_gemm<double>(K, (int)m, K, 1.f, Ri, 1, K, Q, m, 1, 0.f, Qn, m, 1, s));
    STST_CUDA(cudaMemcpyAsync(Q, Qn, sizeof(float) * (size_t)K * m, cudaMemcpyDeviceToDevice, s));
  }
  int hflag = 0;
  STST_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  STST_CUDA(cudaStreamSynchronize(s));
  return hflag ? STST_NOT_HPD : STST_OK;
}

int stst_ws_target_scale(const float *T, int n, int K, float *Ts, double *so, float *w, void *stream) {
  if (!T || !Ts || !so || !w || n < 1 || K < 1) return STST_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  DevTemp tmp(s);
  double *colss = (double *)tmp.get(sizeof(double) * K), *rowss = (double *)tmp.get(sizeof(double) * n);
  if (!colss || !rowss) return STST_ERR_OOM;
  k_ws_colss<float><<<(K + 127) / 128, 128, 0, s>>>(T, n, K, colss);
  k_ws_rowss<<<(n + 7) / 8, 256, 0, s>>>(T, n, K, rowss);
  k_ws_target_scale<<<1, 1024, 0, s>>>(n, K, colss, rowss, so, w);
  k_ws_scale_cols<<<grid_for((long long)n * K, 256), 256, 0, s>>>(T, n, K, so, Ts);
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}

int stst_ws_cascade(const float *T0, const float *Y, const double *scale_prev, double *resid, int n, int K,
                    double *scale, float *targets, const double *so, float *out_scale, void *stream) {
  if (!resid || !scale || !targets || !so || !out_scale || n < 1 || K < 1) return STST_ERR_ARG;
  if (!T0 && (!Y || !scale_prev)) return STST_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  DevTemp tmp(s);
  double *colss = (double *)tmp.get(sizeof(double) * K);
  if (!colss) return STST_ERR_OOM;
  const int g = grid_for((long long)n * K, 256);
  k_ws_cascade_resid<<<g, 256, 0, s>>>(resid, T0, Y, scale_prev, n, K);
  k_ws_colss<double><<<(K + 127) / 128, 128, 0, s>>>(resid, n, K, colss);
  k_ws_cascade_out<<<g, 256, 0, s>>>(resid, colss, n, K, T0 ? 1 : 0, scale, targets, so, out_scale);
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}

int stst_pcg_solve_guarded(stst_handle h, const double *rhs, double *x, double tol, int maxit, int *iters,
                           double *relres, int *used_warm) {
  if (!h || h->magic != STST_MAGIC) return STST_ERR_HANDLE;
  if (!rhs || !x || !(tol >= 0.0) || maxit < 0) return STST_ERR_ARG;
  if (!h->fd_ready) return STST_ERR_STATE;
  {
    ApiScope scope(h);
    cudaStream_t st = h->stream;
    const long long N = h->N_dof;
    const int g = reduction_grid(N);
    double *pr = h->partials + STST_MAXPART, *pf = h->partials + 2 * STST_MAXPART;
    // w_r = f - A x0 with partials of ||w_r||^2; partials of ||f||^2
    STST_TRY(run_plan(h->sys_plan, x, h->w_r, 0, 1, rhs, nullptr, nullptr, nullptr, st, nullptr, pr));
    k_ws_sqnorm<<<g, 256, 0, st>>>((const double2 *)rhs, N, pf);
    k_ws_guard<<<1, 1024, 0, st>>>(pr, pf, g, h->flags + 2);
    k_ws_zero_unless<<<g, 256, 0, st>>>((double2 *)x, N, h->flags + 2);
    STST_CUDA(cudaGetLastError());
  }
  const int status = stst_pcg_solve(h, rhs, x, tol, maxit, iters, relres);
  if (used_warm) {
    int keep = 0;
    STST_CUDA(cudaMemcpyAsync(h->flags_host + 2, h->flags + 2, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    STST_CUDA(cudaStreamSynchronize(h->stream));
    keep = h->flags_host[2];
    *used_warm = keep;
  }
  return status;
}

}  // extern "C"
