// Operator applications on the device.
//  * k_pass: one level of the sum-factorised Kronecker mat-vec (Eq. syst_mat applied matrix-free
//    through Eq. kron_vec_multi): banded 1D matrices applied along one tensor mode, several inputs
//    combined into several outputs with real (or imaginary) coefficients.
//  * k_modeprod: dense mode-n product with a spatial eigenvector matrix (Algorithm 1, steps 2 and 4).
//  * k_timesolve: the N_s independent banded Hermitian solves H_i x_i = y_i (Algorithm 1, step 3,
//    Eq. independent_problems) with precomputed Cholesky factors, one thread per system.
#include "common.cuh"
#include <type_traits>
#include <map>
#include <mutex>
#include <tuple>
#include "async.cuh"

template <typename R> struct C2;
template <> struct C2<double> { using T = double2; };
template <> struct C2<float> { using T = float2; };

template <typename T> __device__ __forceinline__ double2 to_d2(T v) { return make_double2((double)v.x, (double)v.y); }
template <typename T> __device__ __forceinline__ T from_d2(double2 v);
template <> __device__ __forceinline__ double2 from_d2<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 from_d2<float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }

// Deterministic block reduction of one double (blockDim.x multiple of 32, <= 1024).
__device__ __forceinline__ double block_sum(double v, double *sh) {
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
  return t;  // valid in thread 0
}

// ------------------------------------------------------------------------------------------------
// Pass kernel. Output element (o, j, c) of output b = sum over its contributions (input a,
// matrix m, coefficient s): s * sum_k m[j][k] * in_a[o, j + row_off - P + k, c].
// ------------------------------------------------------------------------------------------------
struct PassK {
  int n_out;
  int c_start[PASS_MAXOUT + 1];
  int c_in[PASS_MAXAPP];
  int c_imag[PASS_MAXAPP];
  double c_coef[PASS_MAXAPP];
  const void *c_mat[PASS_MAXAPP];
  const void *in[PASS_MAXIN];
  void *out[PASS_MAXOUT];
  int n_mode_out, n_mode_in, row_off;
  long long inner, outer;
  int epi;
  const void *b;
  const void *dotvec;
  double *dot_partials;
  double *dot2_partials;
  const int *done;
  int balanced;  // 1: CTA b takes the contiguous range [b total / grid, (b + 1) total / grid); 0: grid-stride
};

// One output element idx of every output of the level (index arithmetic in I: 32-bit when the tensor has
// fewer than 2^31 elements, which saves the long software sequence of a 64-bit division).
template <typename R, int P, typename I>
__device__ __forceinline__ void pass_element(const PassK &k, I idx, double &dacc, double &d2acc) {
  using T = typename C2<R>::T;
  const I inner = (I)k.inner, nmo = (I)k.n_mode_out;
  const I c = idx % inner;
  const I t = idx / inner;
  const int j = (int)(t % nmo);
  const I o = t / nmo;
  const long long base = (long long)o * k.n_mode_in * k.inner + c;
  for (int b = 0; b < k.n_out; ++b) {
    R ax = 0, ay = 0;
    for (int ci = k.c_start[b]; ci < k.c_start[b + 1]; ++ci) {
      // the matrix already carries the contribution's coefficient
      const T *in = (const T *)k.in[k.c_in[ci]];
      const R *m = (const R *)k.c_mat[ci] + j * (2 * P + 1);
      if (k.c_imag[ci]) {  // + i * (m x)
#pragma unroll
        for (int q = 0; q <= 2 * P; ++q) {
          int jj = j + k.row_off - P + q;
          if (jj >= 0 && jj < k.n_mode_in) {
            T xv = in[base + (long long)jj * k.inner];
            R mv = m[q];
            ax -= mv * xv.y;
            ay += mv * xv.x;
          }
        }
      } else {
#pragma unroll
        for (int q = 0; q <= 2 * P; ++q) {
          int jj = j + k.row_off - P + q;
          if (jj >= 0 && jj < k.n_mode_in) {
            T xv = in[base + (long long)jj * k.inner];
            R mv = m[q];
            ax += mv * xv.x;
            ay += mv * xv.y;
          }
        }
      }
    }
    T *out = (T *)k.out[b];
    if (k.epi == 1) {  // out = b - v
      T bv = ((const T *)k.b)[idx];
      ax = bv.x - ax;
      ay = bv.y - ay;
    }
    T res;
    res.x = ax;
    res.y = ay;
    out[idx] = res;
    if (k.dotvec) {
      T dv = ((const T *)k.dotvec)[idx];
      dacc += (double)dv.x * (double)ax + (double)dv.y * (double)ay;  // Re(conj(d) * out)
    }
    if (k.dot2_partials) d2acc += (double)ax * ax + (double)ay * ay;
  }
}

template <typename R, int P>
__global__ void __launch_bounds__(512) k_pass(const __grid_constant__ PassK k) {
  if (k.done && *k.done) return;
  __shared__ double sh[32];
  const long long total = k.outer * k.n_mode_out * k.inner;
  double dacc = 0.0, d2acc = 0.0;
  // balanced: equal contiguous ranges per CTA (no SM left with a lighter share when a launch holds only one or
  // two elements per resident thread); otherwise the grid-stride order, whose shared sweep keeps the window of
  // concurrently read inputs compact when every thread handles many elements
  const long long first = k.balanced ? (blockIdx.x * total) / gridDim.x + threadIdx.x
                                     : blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long last = k.balanced ? ((blockIdx.x + 1) * total) / gridDim.x : total;
  const long long step = k.balanced ? (long long)blockDim.x : (long long)gridDim.x * blockDim.x;
  // 32-bit indices: run_plan only launches levels whose elements, plus one step past the end, fit (a 2^31
  // element complex128 tensor is 34 GB, and a solve keeps about ten vectors)
  for (int idx = (int)first; idx < (int)last; idx += (int)step) pass_element<R, P, int>(k, idx, dacc, d2acc);
  if (k.dot_partials) {
    double s = block_sum(dacc, sh);
    if (threadIdx.x == 0) k.dot_partials[blockIdx.x] = s;
  }
  if (k.dot2_partials) {
    double s = block_sum(d2acc, sh);
    if (threadIdx.x == 0) k.dot2_partials[blockIdx.x] = s;
  }
}

// resident CTAs of k_pass<R, P> with `threads` threads on the whole GPU (occupancy API, cached)
template <typename R>
static int pass_resident(int p, int threads) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int>, int> cache;
  const auto key = std::make_tuple((int)sizeof(R), p, threads);
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int per_sm = 0, dev = 0, sms = 152;
  cudaError_t e = cudaErrorInvalidValue;
  switch (p) {
#define CASE(PP) case PP: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pass<R, PP>, threads, 0); break;
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
    default: break;
  }
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int r = (e == cudaSuccess && per_sm > 0) ? per_sm * sms : 0;
  cache[key] = r;
  return r;
}

template <typename R>
static int launch_pass_t(const PassK &k, int p, int grid, cudaStream_t s, int threads = 256) {
  STST_PROF(sizeof(R) == 8 ? "pass_f64" : "pass_f32", s);
  switch (p) {
#define CASE(PP) case PP: k_pass<R, PP><<<grid, threads, 0, s>>>(k); break;
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
    default: return STST_ERR_ARG;
  }
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}

// ------------------------------------------------------------------------------------------------
// All levels of one mat-vec in a single launch, opt-in (the c2 mat-vec's three levels otherwise pay
// three launch ramps and tails; its SMs were busy 84-92% of each launch's elapsed cycles; measured: the two
// grid barriers cost more than they save, 112.7 against 108.6 us per c2 mat-vec). Grid = the last
// level's partial-sum grid with 512 threads, every CTA resident (checked against the occupancy on the
// host); each level runs the unfused launch's element order rule (balanced contiguous ranges when a
// level holds at most two elements per thread, else grid-stride), so every output and every per-CTA
// partial is the unfused one, bitwise. Levels are separated by a grid barrier (count + generation in
// global memory); its wait is bounded: on expiry it sets bit 3 of *err and the kernel carries on (the
// results are then invalid and the caller reports the flag). Intermediate tensors are written in one
// level and read in a later one, never read before they are written, so no SM holds a stale line.
// ------------------------------------------------------------------------------------------------
#define FUSED_MAXLEV 4
struct FusedK {
  PassK lv[FUSED_MAXLEV];
  int p[FUSED_MAXLEV];
  int n;
  unsigned *bar;
  int *err;
};

__device__ __forceinline__ void grid_barrier(unsigned *bar, int *err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *vgen = bar + 1;
    const unsigned gen = *vgen;  // read before arriving: the last arrival advances it only after this
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u) + 1u;
    if (arrived == gridDim.x) {
      bar[0] = 0u;  // nobody touches the count again before the generation moves
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      for (int it = 0; *vgen == gen; ++it) {
        if (it > (1 << 22)) {
          atomicOr(err, 8);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

template <typename R>
__global__ void __launch_bounds__(512) k_pass_fused(const __grid_constant__ FusedK f) {
  if (f.lv[0].done && *f.lv[0].done) return;
  __shared__ double sh[32];
  for (int lv = 0; lv < f.n; ++lv) {
    const PassK &k = f.lv[lv];
    const long long total = k.outer * k.n_mode_out * k.inner;
    double dacc = 0.0, d2acc = 0.0;
    const long long first = k.balanced ? (blockIdx.x * total) / gridDim.x + threadIdx.x
                                       : blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long last = k.balanced ? ((blockIdx.x + 1) * total) / gridDim.x : total;
    const long long step = k.balanced ? (long long)blockDim.x : (long long)gridDim.x * blockDim.x;
    switch (f.p[lv]) {
#define CASE(PP)                                                                                        \
  case PP:                                                                                              \
    for (int idx = (int)first; idx < (int)last; idx += (int)step) pass_element<R, PP, int>(k, idx, dacc, d2acc); \
    break;
      CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
      default: break;
    }
    if (lv + 1 < f.n) {
      grid_barrier(f.bar, f.err);
    } else {
      if (k.dot_partials) {
        double s = block_sum(dacc, sh);
        if (threadIdx.x == 0) k.dot_partials[blockIdx.x] = s;
      }
      if (k.dot2_partials) {
        double s = block_sum(d2acc, sh);
        if (threadIdx.x == 0) k.dot2_partials[blockIdx.x] = s;
      }
    }
  }
}

int g_fused_matvec = 0;  // 0: one launch per level, 1: one launch for all levels where possible

// CTAs of k_pass_fused<R> that fit at once (occupancy API, cached)
template <typename R>
static int fused_resident() {
  static std::mutex mu;
  static int cache[2] = {-1, -1};
  std::lock_guard<std::mutex> lk(mu);
  int &c = cache[sizeof(R) == 8 ? 1 : 0];
  if (c >= 0) return c;
  int per_sm = 0, dev = 0, sms = 152;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pass_fused<R>, 512, 0) != cudaSuccess) per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  c = per_sm * sms;
  return c;
}

// Number of CTAs of every kernel that produces per-CTA partial sums: two per SM. Every consumer of
// the partials reduces all of them (some redundantly in each of its CTAs), so fewer, fuller CTAs
// keep that cheap; 16 warps per SM still cover the FP64 pipe latency of the mat-vec's last level.
int reduction_grid(long long total) {
  int g = grid_for(total, 256);
  if (g > 2 * 152) g = 2 * 152;
  if (g < 1) g = 1;
  return g;
}

// The kernel parameters of level ip of a plan: its contributions output-major, its inputs and outputs
// in the pool (the first level reads x); the last level's output, epilogue and partials are the
// caller's. STST_ERR_ARG when the level has more contributions than the parameters hold.
static int make_level(const Plan &plan, int ip, const void *x, int precision, const int *done, PassK &k) {
  const PassParams &pp = plan.passes[ip];
  k.n_out = pp.n_out;
  int c = 0;
  k.c_start[0] = 0;
  // contributions are stored output-major in PassParams (app == contribution)
  for (int a = 0; a < pp.n_app; ++a) {
    k.c_in[a] = pp.app_in[a];
    k.c_imag[a] = pp.app_imag[a];
    k.c_mat[a] = precision == 1 ? (const void *)pp.mat32[a] : (const void *)pp.mat[a];
  }
  for (int bo = 0; bo < pp.n_out; ++bo) {
    for (int a = 0; a < pp.n_app; ++a) {
      if (pp.coef[a][bo] != 0.0) c++;
    }
    k.c_start[bo + 1] = c;
  }
  // reorder contributions output-major
  {
    int pos = 0;
    int tin[PASS_MAXAPP], tim[PASS_MAXAPP];
    double tco[PASS_MAXAPP];
    const void *tma[PASS_MAXAPP];
    for (int bo = 0; bo < pp.n_out; ++bo)
      for (int a = 0; a < pp.n_app; ++a)
        if (pp.coef[a][bo] != 0.0) {
          if (pos >= PASS_MAXAPP) return STST_ERR_ARG;
          tin[pos] = pp.app_in[a];
          tim[pos] = pp.app_imag[a];
          tco[pos] = pp.coef[a][bo];
          tma[pos] = precision == 1 ? (const void *)pp.cmat32[a][bo] : (const void *)pp.cmat[a][bo];
          pos++;
        }
    for (int q = 0; q < pos; ++q) {
      k.c_in[q] = tin[q];
      k.c_imag[q] = tim[q];
      k.c_coef[q] = tco[q];
      k.c_mat[q] = tma[q];
    }
  }
  for (int a = 0; a < pp.n_in; ++a) k.in[a] = pp.in[a];
  for (int bo = 0; bo < pp.n_out; ++bo) k.out[bo] = pp.out[bo];
  if (ip == 0) k.in[0] = x;
  k.n_mode_out = pp.n_mode_out;
  k.n_mode_in = pp.n_mode_in;
  k.row_off = pp.row_off;
  k.inner = pp.inner;
  k.outer = pp.outer;
  k.epi = 0;
  k.b = nullptr;
  k.dotvec = nullptr;
  k.dot_partials = nullptr;
  k.dot2_partials = nullptr;
  k.done = done;
  k.balanced = 0;
  return STST_OK;
}

int run_plan(const Plan &plan, const void *x, void *y, int precision, int epi, const void *b, const void *dotvec,
             double *dot_partials, const int *done, cudaStream_t s, const void *dot2vec, double *dot2_partials) {
  (void)dot2vec;
  if (plan.geo) return run_geo(*plan.geo, x, y, precision, epi, b, dotvec, dot_partials, done, s, dot2_partials);
  const int np = (int)plan.passes.size();
  if (np == 0) return STST_ERR_STATE;  // dropped by a failed re-plan (see stst_set_potential)
  // one launch for all levels (opt-in, stst_set_fused_matvec): the handle allows it, every level's band
  // half-width has a case, and the last level's partial-sum grid of 512-thread CTAs is resident at once
  bool fused = false;
  FusedK fk;
  int fgrid = 0;
  if (plan.fuse && plan.gbar && plan.gerr && g_fused_matvec == 1 && np >= 2 && np <= FUSED_MAXLEV) {
    const PassParams &pl = plan.passes[np - 1];
    const long long tl = pl.outer * (long long)pl.n_mode_out * pl.inner;
    const int gl = reduction_grid(tl);
    bool ok = true;
    for (int ip = 0; ok && ip < np; ++ip) {
      const PassParams &q = plan.passes[ip];
      const long long t = q.outer * (long long)q.n_mode_out * q.inner;
      if (q.p < 1 || q.p > 8 || t + 152LL * 16 * 512 > 0x7fffffffLL) ok = false;
    }
    fused = ok && precision == 0 && gl <= fused_resident<double>();  // FP64 (the FP32 variant spills)
  }
  for (int ip = 0; ip < np; ++ip) {
    const PassParams &pp = plan.passes[ip];
    PassK k;
    STST_TRY(make_level(plan, ip, x, precision, done, k));
    long long total = pp.outer * (long long)pp.n_mode_out * pp.inner;
    if (total + 152LL * 16 * 512 > 0x7fffffffLL) return STST_ERR_ARG;  // k_pass indexes in 32 bits
    int grid = reduction_grid(total);
    if (ip == np - 1) {
      k.out[0] = y;
      k.epi = epi;
      k.b = b;
      k.dotvec = dotvec;
      k.dot_partials = dot_partials;
      k.dot2_partials = dot2_partials;
    } else {
      grid = grid_for(total, 256);
      if (grid > 152 * 16) grid = 152 * 16;
    }
    // the final level's grid is capped (its per-CTA partials are reduced by every consumer CTA): it runs
    // 512-thread CTAs, twice the warps per SM for the same number of partials
    const int threads = (ip == np - 1) ? 512 : 256;
    // at most two elements per resident thread: equal contiguous ranges, the inner levels in one resident wave
    // (c2: 4.87 -> 4.78 ms per solve measured with this rule; at the 3D sizes, ~14 elements per thread, the
    // grid-stride order stays faster)
    {
      const int res = precision == 1 ? pass_resident<float>(pp.p, threads) : pass_resident<double>(pp.p, threads);
      const long long slots = (long long)(ip == np - 1 ? grid : (res > 0 ? res : grid)) * threads;
      if (res > 0 && total <= 2 * slots) {
        k.balanced = 1;
        if (ip != np - 1 && grid > res) grid = res;
      }
    }
    if (fused) {
      fk.lv[ip] = k;
      fk.p[ip] = pp.p;
      if (ip == np - 1) {
        // the last level's rule decides the partials; the inner levels keep their own rule (outputs
        // do not depend on the element order)
        fgrid = grid;
        fk.n = np;
        fk.bar = plan.gbar;
        fk.err = plan.gerr;
        STST_PROF("pass_fused_f64", s);
        k_pass_fused<double><<<fgrid, 512, 0, s>>>(fk);
        STST_CUDA(cudaGetLastError());
      }
      continue;
    }
    int st = precision == 1 ? launch_pass_t<float>(k, pp.p, grid, s, threads)
                            : launch_pass_t<double>(k, pp.p, grid, s, threads);
    if (st != STST_OK) return st;
  }
  return STST_OK;
}

// ------------------------------------------------------------------------------------------------
// Mode product with a dense n x n matrix U (row-major U[i*n + j]):
//   forward (Algorithm 1 step 2): y[o, j, c] = sum_i U[i][j] x[o, i, c]   (x times U^T along the mode)
//   backward (step 4):            y[o, i, c] = sum_j U[i][j] x[o, j, c]
// A CTA owns 32 flattened columns (o, c) and all n rows; U and the x tile sit in shared memory.
// 256 threads = 8 column groups x 32 row groups; each thread keeps RPT rows x 4 columns of complex
// accumulators in registers (rows rg, rg+32, ..., columns 4 cg .. 4 cg + 3).
// ------------------------------------------------------------------------------------------------
// Mode product with U (step 2: y_j = sum_i U[i][j] x_i) or U^T (step 4), on the columns of the
// time-fastest tensor. Tile: CW = 8 CPT columns and RB = 32 RPT output rows per CTA (grid.y covers the
// rows), U's slice and the x tile staged in shared memory with cp.async; a thread holds CPT columns x
// RPT rows of accumulators. Rows past n are zero in shared memory. Every output is summed over i in
// the same order whatever the tile, so all tiles give bitwise equal results.
template <typename R, typename TI, typename TO, int RPT, int CPT>
__global__ void __launch_bounds__(256) k_modeprod(const TI *__restrict__ X, TO *__restrict__ Y, const R *__restrict__ U,
                                                  int n, long long inner, long long ncols, int backward,
                                                  const EpiDot ed, const int *done) {
  using T = typename C2<R>::T;
  constexpr int CW = 8 * CPT, RB = 32 * RPT, RBP = RB + 1;  // U rows padded: the transposed staging
                                                            // (backward) writes stride RBP, no bank conflicts
  if (done && *done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R *sU = (R *)smem_raw;                                              // n x RBP
  T *sX = (T *)(smem_raw + ((n * RBP * sizeof(R) + 15) / 16) * 16);  // n x CW
  __shared__ double sh[32];
  const long long col0 = (long long)blockIdx.x * CW;
  const int j0 = blockIdx.y * RB;
  // U slice: sU[i*RBP + jj] = coefficient of x_i in y_{j0+jj}; source reads are coalesced either way
  if (!backward) {
    for (int e = threadIdx.x; e < n * RB; e += 256) {  // (i, jj), jj fastest: source U[i][j0 + jj]
      const int i = e / RB, jj = e - i * RB;
      if (j0 + jj < n) cp_async<sizeof(R)>(&sU[i * RBP + jj], &U[(long long)i * n + j0 + jj]);
      else sU[i * RBP + jj] = (R)0;
    }
  } else {
    int e = threadIdx.x, jj = e / n, i = e - (e / n) * n;  // (jj, i), i fastest: source U[j0 + jj][i]
    const int dj = 256 / n, di = 256 - (256 / n) * n;
    for (; e < n * RB; e += 256) {
      if (j0 + jj < n) cp_async<sizeof(R)>(&sU[i * RBP + jj], &U[(long long)(j0 + jj) * n + i]);
      else sU[i * RBP + jj] = (R)0;
      i += di;
      jj += dj;
      if (i >= n) { i -= n; ++jj; }
    }
  }
  // x tile: this thread's column cc = tid % CW is fixed, its rows are tid / CW + (256 / CW) k
  {
    constexpr int RSTEP = 256 / CW;
    const int cc = threadIdx.x % CW;
    const long long col = col0 + cc;
    const bool in = col < ncols;
    const long long o = in ? col / inner : 0, c = in ? col % inner : 0;
    const TI *src = X + o * n * inner + c;
    if constexpr (sizeof(TI) == sizeof(T)) {
      for (int i = threadIdx.x / CW; i < n; i += RSTEP) {
        if (in) cp_async<sizeof(T)>(&sX[i * CW + cc], src + (long long)i * inner);
        else { T z; z.x = 0; z.y = 0; sX[i * CW + cc] = z; }
      }
    } else {
      // FP64 input converted to FP32: eight loads in flight per batch
      for (int i0 = threadIdx.x / CW; i0 < n; i0 += 8 * RSTEP) {
        TI v[8];
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          const int i = i0 + RSTEP * b;
          if (in && i < n) v[b] = src[(long long)i * inner];
          else { v[b].x = 0; v[b].y = 0; }
        }
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          const int i = i0 + RSTEP * b;
          if (i < n) {
            T t;
            t.x = (R)v[b].x;
            t.y = (R)v[b].y;
            sX[i * CW + cc] = t;
          }
        }
      }
    }
    cp_async_commit();
    cp_async_wait_all();
  }
  __syncthreads();
  double dacc[4] = {0.0, 0.0, 0.0, 0.0};
  if constexpr (CPT == 32) {
    // wide tile (n <= ~100, FP32): 32 rows x 256 columns per CTA. Warp w owns rows 8 rg .. 8 rg + 7
    // (rg = w / 2) and column group cgp = 32 (w % 2) + lane; a thread accumulates those 8 rows x the
    // columns cgp + 64 q (q < 4). A step reads 8 U values as warp broadcasts and 4 x values of
    // consecutive columns for 64 FMAs per thread (the one-row tiles read about one wavefront per FMA).
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rgw = warp >> 1, cgp = ((warp & 1) << 5) + lane;
    R ax[8][4], ay[8][4];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) { ax[r][q] = 0; ay[r][q] = 0; }
    for (int i = 0; i < n; ++i) {
      R u[8];
      T xv[4];
#pragma unroll
      for (int r = 0; r < 8; ++r) u[r] = sU[i * RBP + 8 * rgw + r];
#pragma unroll
      for (int q = 0; q < 4; ++q) xv[q] = sX[i * CW + cgp + 64 * q];
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          ax[r][q] += u[r] * xv[q].x;
          ay[r][q] += u[r] * xv[q].y;
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const long long col = col0 + cgp + 64 * q;
      if (col >= ncols) continue;
      const long long o = col / inner, cin = col % inner;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int j = j0 + 8 * rgw + r;
        if (j < n) {
          const long long idx = (o * n + j) * inner + cin;
          TO res;
          res.x = ax[r][q];
          res.y = ay[r][q];
          Y[idx] = res;
          if (ed.part) epi_dot_acc<TO>(dacc, ed, idx, (double)res.x, (double)res.y);
        }
      }
    }
  } else {
    const int cg = threadIdx.x & 7, rg = threadIdx.x >> 3;
    R ax[RPT][CPT], ay[RPT][CPT];
  #pragma unroll
    for (int r = 0; r < RPT; ++r)
  #pragma unroll
      for (int c = 0; c < CPT; ++c) { ax[r][c] = 0; ay[r][c] = 0; }
    for (int i = 0; i < n; ++i) {
      T xv[CPT];
      if constexpr (sizeof(T) == 8) {  // float2 columns: 16-byte reads
        const float4 *q = reinterpret_cast<const float4 *>(&sX[i * CW + cg * CPT]);
  #pragma unroll
        for (int h2 = 0; h2 < CPT / 2; ++h2) {
          const float4 a = q[h2];
          xv[2 * h2].x = a.x; xv[2 * h2].y = a.y; xv[2 * h2 + 1].x = a.z; xv[2 * h2 + 1].y = a.w;
        }
      } else {
  #pragma unroll
        for (int c = 0; c < CPT; ++c) xv[c] = sX[i * CW + cg * CPT + c];
      }
  #pragma unroll
      for (int r = 0; r < RPT; ++r) {
        const R u = sU[i * RBP + rg + 32 * r];
  #pragma unroll
        for (int c = 0; c < CPT; ++c) {
          ax[r][c] += u * xv[c].x;
          ay[r][c] += u * xv[c].y;
        }
      }
    }
  #pragma unroll
    for (int c = 0; c < CPT; ++c) {
      const long long col = col0 + cg * CPT + c;
      if (col >= ncols) continue;
      const long long o = col / inner, cin = col % inner;
  #pragma unroll
      for (int r = 0; r < RPT; ++r) {
        const int j = j0 + rg + 32 * r;
        if (j < n) {
          const long long idx = (o * n + j) * inner + cin;
          TO res;
          res.x = ax[r][c];
          res.y = ay[r][c];
          Y[idx] = res;
          if (ed.part) epi_dot_acc<TO>(dacc, ed, idx, (double)res.x, (double)res.y);
        }
      }
    }
  }
  if (ed.part) epi_dot_store(dacc, ed, (long long)blockIdx.y * gridDim.x + blockIdx.x, sh);
}

static size_t modeprod_smem(int n, MpCfg c, size_t rsize) {
  return ((n * (32 * c.rpt + 1) * rsize + 15) / 16) * 16 + (size_t)n * 8 * c.cpt * 2 * rsize;
}

static dim3 modeprod_grid(int n, long long ncols, MpCfg c) {
  return dim3((unsigned)grid_for(ncols, 8 * c.cpt), (unsigned)((n + 32 * c.rpt - 1) / (32 * c.rpt)));
}

template <typename R, typename TI, typename TO>
static int launch_modeprod(const TI *X, TO *Y, const R *U, int n, long long inner, long long outer, int backward,
                           const EpiDot &ed, const int *done, cudaStream_t s, MpCfg cfg) {
  const long long ncols = inner * outer;
  const dim3 grid = modeprod_grid(n, ncols, cfg);
  if (ed.part && (long long)grid.x * grid.y > STST_MAXPART) return STST_ERR_ARG;
  if (grid.x > 0x7fffffffu || grid.y > 65535u) return STST_ERR_ARG;
  STST_PROF(sizeof(R) == 8 ? "modeprod_f64" : "modeprod_f32", s);
  const size_t sm = modeprod_smem(n, cfg, sizeof(R));
  auto go = [&](auto kern) -> int {
    STST_TRY(ensure_dyn_smem((const void *)kern, sm));
    kern<<<grid, 256, sm, s>>>(X, Y, U, n, inner, ncols, backward, ed, done);
    return STST_OK;
  };
  int st = STST_ERR_ARG;
  const int key = cfg.rpt * 100 + cfg.cpt;
  switch (key) {
#define CASE(RR, CC) case RR * 100 + CC: st = go(k_modeprod<R, TI, TO, RR, CC>); break;
    CASE(1, 2) CASE(1, 4) CASE(2, 2) CASE(2, 4) CASE(3, 2) CASE(3, 4) CASE(4, 2) CASE(4, 4)
#undef CASE
    case 132:  // the wide tile, FP32 only
      if constexpr (sizeof(R) == 4) st = go(k_modeprod<R, TI, TO, 1, 32>);
      break;
    default: break;
  }
  STST_TRY(st);
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}

// ---- tile autotuner for the SIMT mode products --------------------------------------------------
// Candidates: 16 or 32 columns, 32..128 output rows per CTA. Each is timed with CUDA events (two warm
// launches, five timed) on the handle's work vectors; the fastest per (precision, n, inner, outer) is
// cached for the process. Runs outside graph capture (stst_build_fd, stst_batch_create).
MpCfg modeprod_default(int n) {
  MpCfg c;
  c.tc = 0;
  c.cpt = 4;
  c.rpt = (n + 31) / 32;
  if (c.rpt > 4) c.rpt = 4;
  if (c.rpt < 1) c.rpt = 1;
  return c;
}

int g_tune_enabled = 1;
int g_tf32_mode = 0;  // TF32 tensor-core mode products: 0 a tuner candidate, 1 off, 2 forced where they apply
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, long long, long long>, std::pair<MpCfg, float>> g_tune_cache;

template <typename R>
static int tune_one(stst_problem *h, int l, long long inner, long long outer, MpCfg *best, float *best_us) {
  using T = typename C2<R>::T;
  const int n = h->dir[l].n;
  const auto key = std::make_tuple((int)sizeof(R) + 16 * g_tf32_mode, n, inner, outer);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      *best = it->second.first;
      *best_us = it->second.second;
      return STST_OK;
    }
  }
  cudaStream_t st = h->stream;
  const R *U = sizeof(R) == 8 ? (const R *)h->U[l] : (const R *)h->U32[l];
  const T *X = (const T *)h->w_t1;
  T *Y = (T *)h->w_t2;
  cudaEvent_t e0, e1;
  STST_CUDA(cudaEventCreate(&e0));
  STST_CUDA(cudaEventCreate(&e1));
  MpCfg cand = modeprod_default(n);
  float cand_us = 1e30f;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  int status = STST_OK;
  const int maxr = (n + 31) / 32;
  // candidates: one- to four-row tiles of 16 or 32 columns, and (FP32) the wide 32 x 256 tile
  std::vector<MpCfg> cands;
  for (int rpt = 1; rpt <= 4 && rpt <= maxr; ++rpt)
    for (int cpt = 2; cpt <= 4; cpt += 2) cands.push_back(MpCfg{cpt, rpt});
  if (sizeof(R) == 4) cands.push_back(MpCfg{32, 1});
  for (const MpCfg &c : cands) {
    if (status != STST_OK) break;
    {
      if (modeprod_smem(n, c, sizeof(R)) > (size_t)optin) continue;
      for (int w = 0; w < 2 && status == STST_OK; ++w)
        status = launch_modeprod<R, T, T>(X, Y, U, n, inner, outer, 0, EpiDot(), nullptr, st, c);
      if (status != STST_OK) break;
      cudaEventRecord(e0, st);
      for (int w = 0; w < 5 && status == STST_OK; ++w)
        status = launch_modeprod<R, T, T>(X, Y, U, n, inner, outer, 0, EpiDot(), nullptr, st, c);
      cudaEventRecord(e1, st);
      const cudaError_t es = cudaEventSynchronize(e1);
      if (es != cudaSuccess) {
        stst_last_cuda = es;
        status = STST_ERR_CUDA;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      const float us = ms * 1000.f / 5.f;
      if (status == STST_OK && us < cand_us) {
        cand_us = us;
        cand = c;
      }
    }
  }
  cand.tc = 0;
  // the TF32 tensor-core kernel (FP32 only), where the shape allows it; the best SIMT tile stays the fallback
  if constexpr (sizeof(R) == 4) {
    if (status == STST_OK && g_tf32_mode != 1 && h->Utf[l] && tf32_eligible(n, inner, outer, X)) {
      int *ef = h->flags + 1;
      for (int w = 0; w < 2 && status == STST_OK; ++w)
        status = launch_modeprod_tf32<float2>((const float2 *)X, (float2 *)Y, h->Utf[l], 0, n, inner, outer, EpiDot(),
                                              nullptr, ef, st);
      if (status == STST_OK) {
        cudaEventRecord(e0, st);
        for (int w = 0; w < 5 && status == STST_OK; ++w)
          status = launch_modeprod_tf32<float2>((const float2 *)X, (float2 *)Y, h->Utf[l], 0, n, inner, outer,
                                                EpiDot(), nullptr, ef, st);
        cudaEventRecord(e1, st);
        const cudaError_t es = cudaEventSynchronize(e1);
        if (es != cudaSuccess) {
          stst_last_cuda = es;
          status = STST_ERR_CUDA;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const float us = ms * 1000.f / 5.f;
        if (status == STST_OK && (us < cand_us || g_tf32_mode == 2)) {
          cand_us = us;
          cand.tc = 1;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  STST_TRY(status);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = std::make_pair(cand, cand_us);
  }
  *best = cand;
  *best_us = cand_us;
  return STST_OK;
}

static int tune_mp_tiles(stst_problem *h) {
  if (h->prec_mode == STST_PREC_BF16 || g_tune_enabled != 1) {
    long long acc = h->n_t();
    for (int l = 1; l <= h->d; ++l) {
      const long long inner = acc, outer = h->N_dof / (acc * h->dir[l].n);
      acc *= h->dir[l].n;
      h->mp_cfg[l] = modeprod_default(h->dir[l].n);
      // a forced tile: 10 rpt + cpt, or 132 for the wide tile (FP32 preconditioner only)
      int rpt = g_tune_enabled / 10, cpt = g_tune_enabled % 10;
      if (g_tune_enabled == 132 && h->prec_mode == STST_PREC_FP32) {
        rpt = 1;
        cpt = 32;
      }
      if (rpt >= 1 && rpt <= 4 && (cpt == 2 || cpt == 4 || cpt == 32)) {
        MpCfg c;
        c.cpt = cpt;
        c.rpt = rpt;
        c.tc = 0;
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        const size_t rs = h->prec_mode == STST_PREC_FP64 ? sizeof(double) : sizeof(float);
        if (modeprod_smem(h->dir[l].n, c, rs) <= (size_t)optin) h->mp_cfg[l] = c;
      }
      // forced TF32 tensor-core products (FP32 preconditioner), used where the shape and input allow them
      if (g_tf32_mode == 2 && h->prec_mode == STST_PREC_FP32 && h->Utf[l] &&
          tf32_eligible(h->dir[l].n, inner, outer, h->w_t1))
        h->mp_cfg[l].tc = 1;
    }
    return STST_OK;
  }
  long long acc = h->n_t();
  for (int l = 1; l <= h->d; ++l) {
    const long long inner = acc, outer = h->N_dof / (acc * h->dir[l].n);
    acc *= h->dir[l].n;
    MpCfg c;
    float us = 0.f;
    if (h->prec_mode == STST_PREC_FP64) STST_TRY(tune_one<double>(h, l, inner, outer, &c, &us));
    else STST_TRY(tune_one<float>(h, l, inner, outer, &c, &us));
    h->mp_cfg[l] = c;
    h->mp_us[l] = us;
  }
  return STST_OK;
}

// ------------------------------------------------------------------------------------------------
// Time solves. Factor layout: G[(t*P + (k-1))*Ns + i] = G_i[t][t-k] (complex), D[t*Ns + i] = 1/G_i[t][t].
// Data layout: time fastest, y[i*nt + t]. A CTA of 32 threads handles 32 systems. For each chunk of
// TC time steps it stages its systems' data AND their factor rows in shared memory with coalesced
// loads (all in flight together), then runs the sequential recurrences out of shared memory. When
// the whole time axis fits (few CTAs per SM), TC = n_t and every load is issued up front.
// ------------------------------------------------------------------------------------------------
template <typename R, int P>
__global__ void __launch_bounds__(32) k_timesolve(void *__restrict__ Yv, const void *__restrict__ Gv,
                                                  const R *__restrict__ D, int nt, long long Ns, int TC,
                                                  const int *done) {
  using T = typename C2<R>::T;
  if (done && *done) return;
  extern __shared__ __align__(16) unsigned char ts_smem[];
  T *ty = (T *)ts_smem;            // [TC][33]
  T *tg = ty + TC * 33;            // [TC][P][32]
  R *td = (R *)(tg + TC * P * 32); // [TC][32]
  T *Y = (T *)Yv;
  const T *G = (const T *)Gv;
  const long long i0 = (long long)blockIdx.x * 32;
  const int s = threadIdx.x;
  const long long i = i0 + s;
  const bool act = i < Ns;
  const int nsys = (int)min((long long)32, Ns - i0);
  // stage data, factor rows and inverse diagonals of the chunk: every copy is issued before the
  // first wait, so the warp waits for the memory system once per chunk, not once per element
  auto load_chunk = [&](int t0, int tc, bool with_y) {
    if (with_y)
      for (int ss = 0; ss < nsys; ++ss)
        for (int u = s; u < tc; u += 32) cp_async<sizeof(T)>(&ty[u * 33 + ss], &Y[(i0 + ss) * nt + t0 + u]);
    if (s < nsys) {
      for (int u = 0; u < tc; ++u) {
#pragma unroll
        for (int k = 0; k < P; ++k)
          cp_async<sizeof(T)>(&tg[(u * P + k) * 32 + s], &G[((long long)(t0 + u) * P + k) * Ns + i0 + s]);
        cp_async<sizeof(R)>(&td[u * 32 + s], &D[(long long)(t0 + u) * Ns + i0 + s]);
      }
    }
    cp_async_commit();
    cp_async_wait_all();
  };
  auto store_chunk = [&](int t0, int tc) {
    for (int ss = 0; ss < nsys; ++ss)
      for (int u = s; u < tc; u += 32) Y[(i0 + ss) * nt + t0 + u] = ty[u * 33 + ss];
  };
  T zw[P];
#pragma unroll
  for (int a = 0; a < P; ++a) { zw[a].x = 0; zw[a].y = 0; }
  // forward substitution: G z = y
  for (int t0 = 0; t0 < nt; t0 += TC) {
    int tc = min(TC, nt - t0);
    load_chunk(t0, tc, true);
    __syncwarp();
    if (act) {
      for (int u = 0; u < tc; ++u) {
        T y = ty[u * 33 + s];
        R ax = y.x, ay = y.y;
#pragma unroll
        for (int k = 1; k <= P; ++k) {
          T g = tg[(u * P + (k - 1)) * 32 + s];
          T z = zw[k - 1];
          ax -= g.x * z.x - g.y * z.y;
          ay -= g.x * z.y + g.y * z.x;
        }
        R dinv = td[u * 32 + s];
        T z;
        z.x = ax * dinv;
        z.y = ay * dinv;
#pragma unroll
        for (int a = P - 1; a > 0; --a) zw[a] = zw[a - 1];
        zw[0] = z;
        ty[u * 33 + s] = z;
      }
    }
    __syncwarp();
    if (tc < nt) store_chunk(t0, tc);
    __syncwarp();
  }
  // backward substitution: G^H x = z ; x_t = (z_t - sum_k conj(G[t+k][t]) x_{t+k}) / G[t][t]
  T xw[P];
  T gw[P][P];  // gw[a][k-1] = G[t+1+a][t+1+a-k]
#pragma unroll
  for (int a = 0; a < P; ++a) {
    xw[a].x = 0;
    xw[a].y = 0;
#pragma unroll
    for (int k = 0; k < P; ++k) { gw[a][k].x = 0; gw[a][k].y = 0; }
  }
  const int nchunks = (nt + TC - 1) / TC;
  for (int ch = nchunks - 1; ch >= 0; --ch) {
    int t0 = ch * TC;
    int tc = min(TC, nt - t0);
    if (nchunks > 1) {
      load_chunk(t0, tc, true);
      __syncwarp();
    }
    if (act) {
      for (int u = tc - 1; u >= 0; --u) {
        T z = ty[u * 33 + s];
        R ax = z.x, ay = z.y;
#pragma unroll
        for (int a = 0; a < P; ++a) {
          T g = gw[a][a];  // G[t+1+a][t] (offset a+1)
          T xv = xw[a];
          ax -= g.x * xv.x + g.y * xv.y;
          ay -= g.x * xv.y - g.y * xv.x;
        }
        R dinv = td[u * 32 + s];
        T x;
        x.x = ax * dinv;
        x.y = ay * dinv;
#pragma unroll
        for (int a = P - 1; a > 0; --a) {
          xw[a] = xw[a - 1];
#pragma unroll
          for (int k = 0; k < P; ++k) gw[a][k] = gw[a - 1][k];
        }
        xw[0] = x;
#pragma unroll
        for (int k = 1; k <= P; ++k) gw[0][k - 1] = tg[(u * P + (k - 1)) * 32 + s];
        ty[u * 33 + s] = x;
      }
    }
    __syncwarp();
    store_chunk(t0, tc);
    __syncwarp();
  }
}

// ------------------------------------------------------------------------------------------------
// Parallel-in-time time solves. Each system's time axis is cut into S segments that run concurrently
// (one warp per segment, 32 systems per CTA). A banded recurrence carries a state of P values; its map
// across a segment is affine: out = (zero-start run) + T_s in. The transfer matrices T_s depend only on
// the factors and are computed once at setup (k_time_transfer). An application runs every segment from
// a zero state, carries the true states across the segments with the T_s (one lane per system, S steps),
// and reruns every segment from its true state; the same three steps solve G^H x = w backwards. The
// serial depth per solve drops from 2 n_t steps to about 4 n_t / S + 2 S.
// Layouts: T_s[((s P + r) P + c) Ns + i] (r: output state, c: input state). Forward states hold
// (w_{t-1}, ..., w_{t-P}); backward states hold (x_{t+1}, ..., x_{t+P}).
// ------------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void cmul_sub(T &acc, const T g, const T z) {  // acc -= g z
  acc.x -= g.x * z.x - g.y * z.y;
  acc.y -= g.x * z.y + g.y * z.x;
}
template <typename T>
__device__ __forceinline__ void cjmul_sub(T &acc, const T g, const T z) {  // acc -= conj(g) z
  acc.x -= g.x * z.x + g.y * z.y;
  acc.y -= g.x * z.y - g.y * z.x;
}

template <typename R, int P>
__global__ void k_time_transfer(const void *__restrict__ Gv, const R *__restrict__ D, int nt, long long Ns, int S,
                                int L, void *Tfv, void *Tbv) {
  using T = typename C2<R>::T;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= Ns * S * P) return;
  const long long i = idx % Ns, rest = idx / Ns;
  const int c = (int)(rest % P), s = (int)(rest / P);
  const T *G = (const T *)Gv;
  T *Tf = (T *)Tfv, *Tb = (T *)Tbv;
  const int a = s * L, b = min(nt, a + L);
  T st[P];
#pragma unroll
  for (int k = 0; k < P; ++k) { st[k].x = 0; st[k].y = 0; }
  st[c].x = 1;
  for (int t = a; t < b; ++t) {  // homogeneous forward recurrence
    T acc;
    acc.x = 0;
    acc.y = 0;
#pragma unroll
    for (int k = 1; k <= P; ++k) cmul_sub(acc, G[((long long)t * P + (k - 1)) * Ns + i], st[k - 1]);
    const R dinv = D[(long long)t * Ns + i];
#pragma unroll
    for (int k = P - 1; k > 0; --k) st[k] = st[k - 1];
    st[0].x = acc.x * dinv;
    st[0].y = acc.y * dinv;
  }
#pragma unroll
  for (int r = 0; r < P; ++r) Tf[((long long)(s * P + r) * P + c) * Ns + i] = st[r];
#pragma unroll
  for (int k = 0; k < P; ++k) { st[k].x = 0; st[k].y = 0; }
  st[c].x = 1;
  for (int t = b - 1; t >= a; --t) {  // homogeneous backward recurrence
    T acc;
    acc.x = 0;
    acc.y = 0;
#pragma unroll
    for (int k = 1; k <= P; ++k)
      if (t + k < nt) cjmul_sub(acc, G[((long long)(t + k) * P + (k - 1)) * Ns + i], st[k - 1]);
    const R dinv = D[(long long)t * Ns + i];
#pragma unroll
    for (int k = P - 1; k > 0; --k) st[k] = st[k - 1];
    st[0].x = acc.x * dinv;
    st[0].y = acc.y * dinv;
  }
#pragma unroll
  for (int r = 0; r < P; ++r) Tb[((long long)(s * P + r) * P + c) * Ns + i] = st[r];
}

template <typename R, int P>
__global__ void __launch_bounds__(256) k_timesolve_seg(void *__restrict__ Yv, const void *__restrict__ Gv,
                                                       const R *__restrict__ D, const void *__restrict__ Tfv,
                                                       const void *__restrict__ Tbv, int nt, long long Ns, int S,
                                                       int L, const int *done) {
  using T = typename C2<R>::T;
  if (done && *done) return;
  extern __shared__ __align__(16) unsigned char tss[];
  T *ty = (T *)tss;                              // [nt][33]: data, then w, then x
  T *tg = ty + (size_t)nt * 33;                  // [nt][P][32]: G[t][t-k]
  T *sp = tg + (size_t)nt * P * 32;              // [S][P][32]: states after a zero-start run
  T *si = sp + (size_t)S * P * 32;               // [S][P][32]: true incoming states
  T *tf = si + (size_t)S * P * 32;               // [S][P][P][32]
  T *tb = tf + (size_t)S * P * P * 32;           // [S][P][P][32]
  R *td = (R *)(tb + (size_t)S * P * P * 32);    // [nt][32]: 1 / G[t][t]
  T *Y = (T *)Yv;
  const T *G = (const T *)Gv, *Tf = (const T *)Tfv, *Tb = (const T *)Tbv;
  const int nth = blockDim.x;
  const long long i0 = (long long)blockIdx.x * 32;
  const int nsys = (int)min((long long)32, Ns - i0);
  T zero;
  zero.x = 0;
  zero.y = 0;
  for (int e = threadIdx.x; e < 32 * nt; e += nth) {  // system ss, time u: u fastest (coalesced reads)
    const int ss = e / nt, u = e - (e / nt) * nt;
    if (ss < nsys) cp_async<sizeof(T)>(&ty[u * 33 + ss], &Y[(i0 + ss) * nt + u]);
    else ty[u * 33 + ss] = zero;
  }
  for (int e = threadIdx.x; e < nt * P * 32; e += nth) {
    const int ss = e & 31;
    if (ss < nsys) cp_async<sizeof(T)>(&tg[e], &G[(long long)(e >> 5) * Ns + i0 + ss]);
    else tg[e] = zero;
  }
  for (int e = threadIdx.x; e < S * P * P * 32; e += nth) {
    const int ss = e & 31;
    if (ss < nsys) {
      cp_async<sizeof(T)>(&tf[e], &Tf[(long long)(e >> 5) * Ns + i0 + ss]);
      cp_async<sizeof(T)>(&tb[e], &Tb[(long long)(e >> 5) * Ns + i0 + ss]);
    } else {
      tf[e] = zero;
      tb[e] = zero;
    }
  }
  for (int e = threadIdx.x; e < nt * 32; e += nth) {
    const int ss = e & 31;
    if (ss < nsys) cp_async<sizeof(R)>(&td[e], &D[(long long)(e >> 5) * Ns + i0 + ss]);
    else td[e] = (R)0;
  }
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  const int lane = threadIdx.x & 31, seg = threadIdx.x >> 5;
  const int a = seg * L, b = min(nt, a + L);
  T st[P];
  auto forward = [&](bool write) {
    for (int t = a; t < b; ++t) {
      T acc = ty[t * 33 + lane];
#pragma unroll
      for (int k = 1; k <= P; ++k) cmul_sub(acc, tg[(t * P + (k - 1)) * 32 + lane], st[k - 1]);
      const R dinv = td[t * 32 + lane];
#pragma unroll
      for (int k = P - 1; k > 0; --k) st[k] = st[k - 1];
      st[0].x = acc.x * dinv;
      st[0].y = acc.y * dinv;
      if (write) ty[t * 33 + lane] = st[0];
    }
  };
  auto backward = [&](bool write) {
    for (int t = b - 1; t >= a; --t) {
      T acc = ty[t * 33 + lane];
#pragma unroll
      for (int k = 1; k <= P; ++k)
        if (t + k < nt) cjmul_sub(acc, tg[((t + k) * P + (k - 1)) * 32 + lane], st[k - 1]);
      const R dinv = td[t * 32 + lane];
#pragma unroll
      for (int k = P - 1; k > 0; --k) st[k] = st[k - 1];
      st[0].x = acc.x * dinv;
      st[0].y = acc.y * dinv;
      if (write) ty[t * 33 + lane] = st[0];
    }
  };
  // carry: one lane per system walks the segments in `dir` order; in of the first segment is zero,
  // in of the next = out of this = sp + T in
  auto carry = [&](const T *tr, int first, int step) {
    T cur[P];
#pragma unroll
    for (int k = 0; k < P; ++k) cur[k] = zero;
    for (int s2 = first, n2 = 0; n2 < S; ++n2, s2 += step) {
      T nxt[P];
#pragma unroll
      for (int r = 0; r < P; ++r) {
        si[(s2 * P + r) * 32 + lane] = cur[r];
        T o = sp[(s2 * P + r) * 32 + lane];
#pragma unroll
        for (int c = 0; c < P; ++c) {
          const T g = tr[((s2 * P + r) * P + c) * 32 + lane];
          o.x += g.x * cur[c].x - g.y * cur[c].y;
          o.y += g.x * cur[c].y + g.y * cur[c].x;
        }
        nxt[r] = o;
      }
#pragma unroll
      for (int r = 0; r < P; ++r) cur[r] = nxt[r];
    }
  };
  // G w = y
#pragma unroll
  for (int k = 0; k < P; ++k) st[k] = zero;
  forward(false);
#pragma unroll
  for (int k = 0; k < P; ++k) sp[(seg * P + k) * 32 + lane] = st[k];
  __syncthreads();
  if (seg == 0) carry(tf, 0, 1);
  __syncthreads();
#pragma unroll
  for (int k = 0; k < P; ++k) st[k] = si[(seg * P + k) * 32 + lane];
  forward(true);
  __syncthreads();
  // G^H x = w
#pragma unroll
  for (int k = 0; k < P; ++k) st[k] = zero;
  backward(false);
#pragma unroll
  for (int k = 0; k < P; ++k) sp[(seg * P + k) * 32 + lane] = st[k];
  __syncthreads();
  if (seg == 0) carry(tb, S - 1, -1);
  __syncthreads();
#pragma unroll
  for (int k = 0; k < P; ++k) st[k] = si[(seg * P + k) * 32 + lane];
  backward(true);
  __syncthreads();
  for (int e = threadIdx.x; e < nsys * nt; e += nth) {
    const int ss = e / nt, u = e - (e / nt) * nt;
    Y[(i0 + ss) * nt + u] = ty[u * 33 + ss];
  }
}

size_t ts_seg_smem(int nt, int P, int S, size_t rs) {
  const size_t cs = 2 * rs;
  return (size_t)nt * 33 * cs + (size_t)nt * P * 32 * cs + 2 * (size_t)S * P * 32 * cs +
         2 * (size_t)S * P * P * 32 * cs + (size_t)nt * 32 * rs;
}

// largest S <= 8 (segments of at least P steps) whose shared memory fits; S = 0 when none does
void ts_segments(int nt, int P, size_t rs, int *S_out, int *L_out) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  *S_out = 0;
  *L_out = nt;
  for (int S = 8; S >= 2; --S) {
    const int L = (nt + S - 1) / S;
    if (L < P || (S - 1) * L >= nt) continue;
    if (ts_seg_smem(nt, P, S, rs) > (size_t)optin) continue;
    *S_out = S;
    *L_out = L;
    return;
  }
}

template <typename R>
int launch_time_transfer(const void *G, const R *D, int nt, long long Ns, int P, int S, int L, void *Tf, void *Tb,
                         cudaStream_t s) {
  if (S < 2) return STST_OK;
  const long long n = Ns * S * P;
  STST_PROF(sizeof(R) == 8 ? "time_transfer_f64" : "time_transfer_f32", s);
  switch (P) {
#define CASE(PP) case PP: k_time_transfer<R, PP><<<grid_for(n, 128), 128, 0, s>>>(G, D, nt, Ns, S, L, Tf, Tb); break;
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
    default: return STST_ERR_ARG;
  }
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}
template int launch_time_transfer<float>(const void *, const float *, int, long long, int, int, int, void *, void *,
                                         cudaStream_t);
template int launch_time_transfer<double>(const void *, const double *, int, long long, int, int, int, void *, void *,
                                          cudaStream_t);

template <typename R>
static int launch_timesolve_seg(void *Y, const void *G, const R *D, const void *Tf, const void *Tb, int nt,
                                long long Ns, int P, int S, int L, const int *done, cudaStream_t s) {
  const size_t sm = ts_seg_smem(nt, P, S, sizeof(R));
  STST_PROF(sizeof(R) == 8 ? "timesolve_f64" : "timesolve_f32", s);
  const int grid = grid_for(Ns, 32);
  switch (P) {
#define CASE(PP)                                                                                       \
  case PP:                                                                                             \
    STST_TRY(ensure_dyn_smem((const void *)k_timesolve_seg<R, PP>, sm));                               \
    k_timesolve_seg<R, PP><<<grid, 32 * S, sm, s>>>(Y, G, D, Tf, Tb, nt, Ns, S, L, done);              \
    break;
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
    default: return STST_ERR_ARG;
  }
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}

template <typename R>
static int launch_timesolve(void *Y, const void *G, const R *D, int nt, long long Ns, int P, const int *done,
                            cudaStream_t s) {
  using T = typename C2<R>::T;
  const int grid = grid_for(Ns, 32);
  const size_t per_t = 33 * sizeof(T) + (size_t)P * 32 * sizeof(T) + 32 * sizeof(R);
  // shared memory per CTA: the whole time axis when few CTAs share an SM, else a chunk
  const int ctas_per_sm = (grid + 151) / 152;
  size_t budget = (200 * 1024) / (size_t)ctas_per_sm;
  int TC = (int)(budget / per_t);
  if (TC > nt) TC = nt;
  if (TC < 8) TC = (nt < 8) ? nt : 8;
  const size_t sm = per_t * TC;
  STST_PROF(sizeof(R) == 8 ? "timesolve_f64" : "timesolve_f32", s);
  switch (P) {
#define CASE(PP)                                                                                          \
  case PP:                                                                                                \
    STST_TRY(ensure_dyn_smem((const void *)k_timesolve<R, PP>, sm));                                          \
    k_timesolve<R, PP><<<grid, 32, sm, s>>>(Y, G, D, nt, Ns, TC, done);                                   \
    break;
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
    default: return STST_ERR_ARG;
  }
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}

// ------------------------------------------------------------------------------------------------
// Algorithm 1 steps 2-4: s = (U_s (x) I) H^{-1} (U_s^T (x) I) r.
// precision 0: FP64 throughout (scratch buffers are double2); 1: FP32 mode products and solves
// (r read as FP64, s written as FP64; intermediates float2 in the scratch buffers).
// in32 / out32: optional FP32 input / output (inner FP32 solver), replacing r / s.
// The final mode product optionally accumulates per-CTA partials of Re<r, s> into dot_partials.
// ------------------------------------------------------------------------------------------------

// ------------------------------------------------------------------------------------------------
// Fused 2D spatial transforms of Algorithm 1 (steps 2 and 4, d = 2, FP32): for one time index t the
// spatial slab X_t (n1 x n2, X_t[i1][i2] = X[t + nt (i1 + n1 i2)]) goes through both mode products in
// shared memory,
//   forward:  Y_t = U1^T X_t U2   (mode 1, then mode 2),
//   backward: Y_t = U1 X_t U2^T   (mode 2, then mode 1).
// S CTAs share a time index: the forward transform is split by rows of Y_t (a CTA needs the columns of
// U1 of its rows and all of X_t, and mode 2 stays within its rows), the backward one by columns of
// Y_t (a CTA needs the rows of U2 of its columns). Every output is accumulated over its index in
// ascending order from the FP32-rounded intermediate, as the separate mode products do, so the
// results are bitwise equal to theirs.
//
// Each contraction o(a, b) = sum_i R(i, a) C(i, b) has a real factor R (a slice of U1 or U2, staged
// so that R(i, a) = sR[i rs + a]) and a complex one C (slab or intermediate). Thread `item` = g Ra + a0
// owns the outputs a = a0 + Ra k (k < NR) and b = NC g + q (q < NC), Ra = ceil(A / NR): consecutive
// lanes read consecutive entries of R and mostly the same entries of C (broadcast), so a warp's
// shared-memory reads per step are NR + NC wavefronts against 2 NR NC FMAs.
// ------------------------------------------------------------------------------------------------
#define FD2D_NR 4
#define FD2D_NC 4
#define FD2D_MAXN 80
#define FD2D_MAXS 4

template <int NR, int NC>
__device__ __forceinline__ void fd2d_contract(const float *__restrict__ sR, int rs, int A,
                                              const float2 *__restrict__ sC, int cs_i, int cs_b, int B, int K,
                                              int a0, int Ra, int g, float ax[NR][NC], float ay[NR][NC]) {
  int ra[NR], cb[NC];
#pragma unroll
  for (int k = 0; k < NR; ++k) ra[k] = min(a0 + Ra * k, A - 1);  // clamped: results past A are not stored
#pragma unroll
  for (int q = 0; q < NC; ++q) cb[q] = min(NC * g + q, B - 1) * cs_b;
#pragma unroll
  for (int k = 0; k < NR; ++k)
#pragma unroll
    for (int q = 0; q < NC; ++q) { ax[k][q] = 0.f; ay[k][q] = 0.f; }
  for (int i = 0; i < K; ++i) {
    const float *ri = sR + (long long)i * rs;
    const float2 *ci = sC + (long long)i * cs_i;
    float u[NR];
    float2 xv[NC];
#pragma unroll
    for (int k = 0; k < NR; ++k) u[k] = ri[ra[k]];
#pragma unroll
    for (int q = 0; q < NC; ++q) xv[q] = ci[cb[q]];
#pragma unroll
    for (int k = 0; k < NR; ++k)
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        ax[k][q] += u[k] * xv[q].x;
        ay[k][q] += u[k] * xv[q].y;
      }
  }
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(512) k_fd2d(const TI *__restrict__ X, TO *__restrict__ Y, const float *__restrict__ U1,
                                              const float *__restrict__ U2, int n1, int n2, int nt, int backward,
                                              const EpiDot ed, const int *done) {
  constexpr int NR = FD2D_NR, NC = FD2D_NC;
  if (done && *done) return;
  extern __shared__ __align__(16) unsigned char fd_smem[];
  __shared__ double sh[32];
  // slab (t, i3): X_t[i1][i2] at base + nt (i1 + n1 i2), base = t + nt n1 n2 i3 (i3 = 0 for d = 2)
  const int t = blockIdx.x % nt, S = gridDim.y, part = blockIdx.y;
  const long long base = t + (long long)nt * n1 * n2 * (blockIdx.x / nt);
  const int tid = threadIdx.x, nth = blockDim.x;
  const int nsplit = backward ? n2 : n1, nother = backward ? n1 : n2;
  const int mfull = (nsplit + S - 1) / S, p0 = part * mfull, m = min(mfull, nsplit - p0);
  const int nmax = max(n1, n2);
  float2 *sX = (float2 *)fd_smem;                    // slab, X_t[i1][i2] at i1 + n1 i2
  float2 *sZ = sX + n1 * n2;                         // intermediate, mfull x nmax
  float *sRa = (float *)(sZ + mfull * nmax);         // forward: U1 columns of the part; backward: U2 rows
  float *sRb = sRa + (mfull * nmax + 3) / 4 * 4;     // forward: U2; backward: U1^T
  // staging: the factors and an FP32 slab by cp.async (all copies in flight at once), an FP64 slab
  // through registers in batches of independent loads (it is rounded to FP32 on the way)
  if (!backward) {
    for (int e = tid; e < n1 * m; e += nth) {        // sRa[i m + j] = U1[i][p0 + j]
      const int i = e / m, j = e - i * m;
      cp_async<4>(&sRa[e], &U1[i * n1 + p0 + j]);
    }
    for (int e = tid; e < n2 * n2; e += nth) cp_async<4>(&sRb[e], &U2[e]);
  } else {
    for (int e = tid; e < m * n2; e += nth) {        // sRa[c m + k] = U2[p0 + k][c]
      const int k = e / n2, c = e - k * n2;
      cp_async<4>(&sRa[c * m + k], &U2[(p0 + k) * n2 + c]);
    }
    for (int e = tid; e < n1 * n1; e += nth) {       // sRb[r n1 + j] = U1[j][r]
      const int j = e / n1, r = e - j * n1;
      cp_async<4>(&sRb[r * n1 + j], &U1[e]);
    }
  }
  if constexpr (sizeof(TI) == sizeof(float2)) {
    for (int e = tid; e < n1 * n2; e += nth) cp_async<8>(&sX[e], &X[base + (long long)nt * e]);
  } else {
    constexpr int BATCH = 8;  // independent loads in flight per thread
    const int nn = n1 * n2;
    for (int e0 = tid; e0 < nn; e0 += BATCH * nth) {
      TI v[BATCH];
#pragma unroll
      for (int u = 0; u < BATCH; ++u) {
        const int e = e0 + u * nth;
        if (e < nn) v[u] = X[base + (long long)nt * e];
      }
#pragma unroll
      for (int u = 0; u < BATCH; ++u) {
        const int e = e0 + u * nth;
        if (e < nn) sX[e] = make_float2((float)v[u].x, (float)v[u].y);
      }
    }
  }
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  float ax[NR][NC], ay[NR][NC];
  const int Ra1 = (m + NR - 1) / NR, Ra2 = (nother + NR - 1) / NR;
  if (tid < Ra1 * ((nother + NC - 1) / NC)) {
    const int a0 = tid % Ra1, g = tid / Ra1;
    if (!backward)  // Z[j][c] = sum_i U1[i][p0 + j] X[i][c], stored at sZ[j + m c]
      fd2d_contract<NR, NC>(sRa, m, m, sX, 1, n1, n2, n1, a0, Ra1, g, ax, ay);
    else            // Z[r][k] = sum_c U2[p0 + k][c] X[r][c], stored at sZ[r + n1 k]
      fd2d_contract<NR, NC>(sRa, m, m, sX, n1, 1, n1, n2, a0, Ra1, g, ax, ay);
    const int zs = backward ? n1 : 1, zb = backward ? 1 : m;  // sZ index = a zs + b zb
#pragma unroll
    for (int k = 0; k < NR; ++k)
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        const int a = a0 + Ra1 * k, b = NC * g + q;
        if (a < m && b < nother) sZ[a * zs + b * zb] = make_float2(ax[k][q], ay[k][q]);
      }
  }
  __syncthreads();
  double dacc[4] = {0.0, 0.0, 0.0, 0.0};
  if (tid < Ra2 * ((m + NC - 1) / NC)) {
    const int a0 = tid % Ra2, g = tid / Ra2;
    if (!backward)  // Y[j][k] = sum_c U2[c][k] Z[j][c]
      fd2d_contract<NR, NC>(sRb, n2, n2, sZ, m, 1, m, n2, a0, Ra2, g, ax, ay);
    else            // Y[j][k] = sum_r U1[j][r] Z[r][k]
      fd2d_contract<NR, NC>(sRb, n1, n1, sZ, 1, n1, m, n1, a0, Ra2, g, ax, ay);
#pragma unroll
    for (int k = 0; k < NR; ++k)
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        const int a = a0 + Ra2 * k, b = NC * g + q;
        if (a < nother && b < m) {
          const int i1 = backward ? a : p0 + b, i2 = backward ? p0 + b : a;
          const long long idx = base + (long long)nt * (i1 + (long long)n1 * i2);
          TO res;
          res.x = ax[k][q];
          res.y = ay[k][q];
          Y[idx] = res;
          if (ed.part) epi_dot_acc<TO>(dacc, ed, idx, (double)res.x, (double)res.y);
        }
      }
  }
  if (ed.part) epi_dot_store(dacc, ed, (long long)blockIdx.x * S + part, sh);
}

// items of the larger of the two contractions, at least 256 threads for the staging
static int fd2d_threads(int m, int nother) {
  const int i1 = ((m + FD2D_NR - 1) / FD2D_NR) * ((nother + FD2D_NC - 1) / FD2D_NC);
  const int i2 = ((nother + FD2D_NR - 1) / FD2D_NR) * ((m + FD2D_NC - 1) / FD2D_NC);
  const int nth = ((i1 > i2 ? i1 : i2) + 31) / 32 * 32;
  return nth < 256 ? 256 : nth;
}

static size_t fd2d_smem(int n1, int n2, int S) {
  const int nmax = n1 > n2 ? n1 : n2, mfull = (nmax + S - 1) / S;
  return sizeof(float2) * ((size_t)n1 * n2 + (size_t)mfull * nmax) +
         sizeof(float) * (((size_t)mfull * nmax + 3) / 4 * 4 + (size_t)nmax * nmax);
}

// S parts of a time index are usable when none of them is empty along either split dimension
static bool fd2d_split_ok(int n1, int n2, int S) {
  return (S - 1) * ((n1 + S - 1) / S) < n1 && (S - 1) * ((n2 + S - 1) / S) < n2;
}

// number of slabs (t, i3) the fused kernel runs over: n_t for d = 2, n_t n_3 for d = 3
static long long fd2d_slabs(const stst_problem *h) { return (long long)h->n_t() * (h->d == 3 ? h->dir[3].n : 1); }

bool fd2d_fits(const stst_problem *h) {
  if ((h->d != 2 && h->d != 3) || h->dir[1].n > FD2D_MAXN || h->dir[2].n > FD2D_MAXN) return false;
  if (fd2d_slabs(h) * FD2D_MAXS > STST_MAXPART || fd2d_slabs(h) > 0x7fffffffLL) return false;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return fd2d_smem(h->dir[1].n, h->dir[2].n, 1) <= (size_t)optin;
}

template <typename TI, typename TO>
static int launch_fd2d(const TI *X, TO *Y, const stst_problem *h, int backward, const EpiDot &ed, const int *done,
                       cudaStream_t s, int S) {
  const int n1 = h->dir[1].n, n2 = h->dir[2].n, nt = h->n_t();
  if (S < 1 || S > FD2D_MAXS || !fd2d_split_ok(n1, n2, S)) return STST_ERR_ARG;
  const int m = backward ? (n2 + S - 1) / S : (n1 + S - 1) / S;
  const int nth = fd2d_threads(m, backward ? n1 : n2);
  const size_t sm = fd2d_smem(n1, n2, S);
  STST_PROF("modeprod2d_f32", s);
  STST_TRY(ensure_dyn_smem((const void *)k_fd2d<TI, TO>, sm));
  k_fd2d<TI, TO><<<dim3((unsigned)fd2d_slabs(h), S), nth, sm, s>>>(X, Y, h->U32[1], h->U32[2], n1, n2, nt, backward,
                                                                   ed, done);
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}

// time solve of the preconditioner: segmented (parallel in time) or sequential, as chosen per handle
template <typename R>
static int time_solve(stst_problem *h, void *Y, const int *done, cudaStream_t st) {
  const int q = sizeof(R) == 8 ? 1 : 0;
  const void *G = q ? h->Hg : h->Hg32;
  const R *D = q ? (const R *)h->Hd : (const R *)h->Hd32;
  if (h->ts_seg[q] && h->ts_S[q] >= 2)
    return launch_timesolve_seg<R>(Y, G, D, h->Tf[q], h->Tb[q], h->n_t(), h->N_s, h->dir[0].p, h->ts_S[q],
                                   h->ts_L[q], done, st);
  return launch_timesolve<R>(Y, G, D, h->n_t(), h->N_s, h->dir[0].p, done, st);
}

// FP32 mode product of direction l: the TF32 tensor-core kernel where the tuner chose it and the shape and
// input allow it (FP32 input with aligned rows), else the SIMT tile
template <typename TI, typename TO>
static int mp32(stst_problem *h, int l, const TI *X, TO *Y, long long inner, long long outer, int backward,
                const EpiDot &ed, const int *done, cudaStream_t s) {
  const int n = h->dir[l].n;
  if constexpr (std::is_same<TI, float2>::value) {
    if (h->mp_cfg[l].tc && h->Utf[l]) {
      if (tf32_eligible(n, inner, outer, X))
        return launch_modeprod_tf32<TO>(X, Y, h->Utf[l], backward, n, inner, outer, ed, done, h->flags + 1, s);
      // the partial sums of the epilogue were counted for the tensor-core grid
      if (ed.part) return STST_ERR_ARG;
    }
  }
  return launch_modeprod<float, TI, TO>(X, Y, h->U32[l], n, inner, outer, backward, ed, done, s, h->mp_cfg[l]);
}

int fd_apply(stst_problem *h, const double *r, double *s, int precision, const EpiDot &ed, const int *done,
             void *bufA, void *bufB, float *out32, const float *in32) {
  const int d = h->d;
  cudaStream_t st = h->stream;
  const EpiDot none;
  // tensor geometry of mode l (1..d) in the time-fastest layout: inner = nt * prod_{k<l} n_k
  long long inner[STST_MAXD + 1], outer[STST_MAXD + 1];
  {
    long long acc = h->n_t();
    for (int l = 1; l <= d; ++l) {
      inner[l] = acc;
      acc *= h->dir[l].n;
    }
    long long tot = acc;
    for (int l = 1; l <= d; ++l) outer[l] = tot / (inner[l] * h->dir[l].n);
  }
  if (precision == 0) {
    // forward: r -> A -> B -> ... (alternating), solve in place, backward to s
    const double2 *src = (const double2 *)r;
    double2 *bufs[2] = {(double2 *)bufA, (double2 *)bufB};
    int cur = 0;
    for (int l = 1; l <= d; ++l) {
      double2 *dst = bufs[cur];
      STST_TRY((launch_modeprod<double, double2, double2>(src, dst, h->U[l], h->dir[l].n, inner[l], outer[l], 0, none,
                                                           done, st, h->mp_cfg[l])));
      src = dst;
      cur ^= 1;
    }
    STST_TRY(time_solve<double>(h, (void *)src, done, st));
    for (int l = d; l >= 1; --l) {
      double2 *dst = (l == 1) ? (double2 *)s : bufs[cur];
      STST_TRY((launch_modeprod<double, double2, double2>(src, dst, h->U[l], h->dir[l].n, inner[l], outer[l], 1,
                                                           l == 1 ? ed : none, done, st, h->mp_cfg[l])));
      src = dst;
      cur ^= 1;
    }
    return STST_OK;
  }
  if (precision == 2) {
    // mode products on the tensor cores (BF16 operands, FP32 accumulation), time solves in FP32
    float2 *bufs[2] = {(float2 *)bufA, (float2 *)bufB};
    int cur = 0;
    const float2 *src32 = nullptr;
    int *ef = h->flags + 1;
    // U' planes per direction: [fwd hi | bwd hi | fwd lo | bwd lo]; three-product split
    const int split = 3;
    auto Bk = [&](int l, int bwd) {
      const size_t np = pad16(h->dir[l].n);
      return (const __nv_bfloat16 *)(h->Ubf[l] + (bwd ? np * np : 0));
    };
    auto lo = [&](int l) { return 2LL * pad16(h->dir[l].n) * pad16(h->dir[l].n); };
    for (int l = 1; l <= d; ++l) {
      float2 *dst = bufs[cur];
      if (l == 1 && !in32) {
        STST_TRY((launch_modeprod_tc<double2, float2>((const double2 *)r, dst, Bk(l, 0), lo(l), split, h->dir[l].n,
                                                      inner[l], outer[l], none, done, ef, st)));
      } else {
        const float2 *in = (l == 1) ? (const float2 *)in32 : src32;
        STST_TRY((launch_modeprod_tc<float2, float2>(in, dst, Bk(l, 0), lo(l), split, h->dir[l].n, inner[l], outer[l],
                                                     none, done, ef, st)));
      }
      src32 = dst;
      cur ^= 1;
    }
    STST_TRY(time_solve<float>(h, (void *)src32, done, st));
    for (int l = d; l >= 1; --l) {
      if (l == 1) {
        if (out32) {
          STST_TRY((launch_modeprod_tc<float2, float2>(src32, (float2 *)out32, Bk(l, 1), lo(l), split, h->dir[l].n,
                                                       inner[l], outer[l], ed, done, ef, st)));
        } else {
          STST_TRY((launch_modeprod_tc<float2, double2>(src32, (double2 *)s, Bk(l, 1), lo(l), split, h->dir[l].n,
                                                        inner[l], outer[l], ed, done, ef, st)));
        }
      } else {
        float2 *dst = bufs[cur];
        STST_TRY((launch_modeprod_tc<float2, float2>(src32, dst, Bk(l, 1), lo(l), split, h->dir[l].n, inner[l],
                                                     outer[l], none, done, ef, st)));
        src32 = dst;
        cur ^= 1;
      }
    }
    return STST_OK;
  }
  // FP32
  if (h->pencil) {
    // the last direction's products and the time solves in the pencil kernel; the other directions as
    // fused 2D transforms (d = 3) or mode products
    const int CL = h->pencil;
    float2 *y32 = (float2 *)bufA, *z32 = (float2 *)bufB;
    if (d == 1) {
      if (in32 && out32) return launch_pencil<float2, float2>((const float2 *)in32, (float2 *)out32, h, CL, ed, done, st);
      if (in32) return launch_pencil<float2, double2>((const float2 *)in32, (double2 *)s, h, CL, ed, done, st);
      if (out32) return launch_pencil<double2, float2>((const double2 *)r, (float2 *)out32, h, CL, ed, done, st);
      return launch_pencil<double2, double2>((const double2 *)r, (double2 *)s, h, CL, ed, done, st);
    }
    if (d == 3 && h->fd2d) {
      const int S = h->fd2d, Sb = h->fd2d_b;
      if (in32) STST_TRY((launch_fd2d<float2, float2>((const float2 *)in32, y32, h, 0, none, done, st, S)));
      else STST_TRY((launch_fd2d<double2, float2>((const double2 *)r, y32, h, 0, none, done, st, S)));
      STST_TRY((launch_pencil<float2, float2>(y32, z32, h, CL, none, done, st)));
      if (out32) return launch_fd2d<float2, float2>(z32, (float2 *)out32, h, 1, ed, done, st, Sb);
      return launch_fd2d<float2, double2>(z32, (double2 *)s, h, 1, ed, done, st, Sb);
    }
    // mode products of directions 1 .. d-1 forward (alternating buffers), the pencil, then backward
    float2 *bufs[2] = {y32, z32};
    int cur = 0;
    const float2 *src = nullptr;
    for (int l = 1; l < d; ++l) {
      float2 *dst = bufs[cur];
      if (l == 1 && !in32)
        STST_TRY((mp32<double2, float2>(h, l, (const double2 *)r, dst, inner[l], outer[l], 0, none, done, st)));
      else
        STST_TRY((mp32<float2, float2>(h, l, l == 1 ? (const float2 *)in32 : src, dst, inner[l], outer[l], 0, none, done, st)));
      src = dst;
      cur ^= 1;
    }
    {
      float2 *dst = bufs[cur];
      STST_TRY((launch_pencil<float2, float2>(src, dst, h, CL, none, done, st)));
      src = dst;
      cur ^= 1;
    }
    for (int l = d - 1; l >= 1; --l) {
      if (l == 1) {
        if (out32)
          return mp32<float2, float2>(h, l, src, (float2 *)out32, inner[l], outer[l], 1, ed, done, st);
        return mp32<float2, double2>(h, l, src, (double2 *)s, inner[l], outer[l], 1, ed, done, st);
      }
      float2 *dst = bufs[cur];
      STST_TRY((mp32<float2, float2>(h, l, src, dst, inner[l], outer[l], 1, none,
                                                       done, st)));
      src = dst;
      cur ^= 1;
    }
    return STST_OK;
  }
  if (h->fd2d) {  // modes 1 and 2 of each transform in one kernel per (t, i3) slab; mode 3 (d = 3) separate
    float2 *y32 = (float2 *)bufA;
    const int S = h->fd2d, Sb = h->fd2d_b;
    if (in32) STST_TRY((launch_fd2d<float2, float2>((const float2 *)in32, y32, h, 0, none, done, st, S)));
    else STST_TRY((launch_fd2d<double2, float2>((const double2 *)r, y32, h, 0, none, done, st, S)));
    if (d == 3) {
      float2 *z32 = (float2 *)bufB;
      STST_TRY((mp32<float2, float2>(h, 3, y32, z32, inner[3], outer[3], 0, none,
                                                       done, st)));
      STST_TRY(time_solve<float>(h, (void *)z32, done, st));
      STST_TRY((mp32<float2, float2>(h, 3, z32, y32, inner[3], outer[3], 1, none,
                                                       done, st)));
    } else {
      STST_TRY(time_solve<float>(h, (void *)y32, done, st));
    }
    if (out32) return launch_fd2d<float2, float2>(y32, (float2 *)out32, h, 1, ed, done, st, Sb);
    return launch_fd2d<float2, double2>(y32, (double2 *)s, h, 1, ed, done, st, Sb);
  }
  float2 *bufs[2] = {(float2 *)bufA, (float2 *)bufB};
  int cur = 0;
  const float2 *src32 = nullptr;
  for (int l = 1; l <= d; ++l) {
    float2 *dst = bufs[cur];
    if (l == 1) {
      if (in32) {
        STST_TRY((mp32<float2, float2>(h, l, (const float2 *)in32, dst, inner[l], outer[l], 0, none, done, st)));
      } else {
        STST_TRY((mp32<double2, float2>(h, l, (const double2 *)r, dst, inner[l], outer[l], 0, none, done, st)));
      }
    } else {
      STST_TRY((mp32<float2, float2>(h, l, src32, dst, inner[l], outer[l], 0, none,
                                                       done, st)));
    }
    src32 = dst;
    cur ^= 1;
  }
  STST_TRY(time_solve<float>(h, (void *)src32, done, st));
  for (int l = d; l >= 1; --l) {
    if (l == 1) {
      if (out32) {
        STST_TRY((mp32<float2, float2>(h, l, src32, (float2 *)out32, inner[l], outer[l], 1, ed, done, st)));
      } else {
        STST_TRY((mp32<float2, double2>(h, l, src32, (double2 *)s, inner[l], outer[l], 1, ed, done, st)));
      }
    } else {
      float2 *dst = bufs[cur];
      STST_TRY((mp32<float2, float2>(h, l, src32, dst, inner[l], outer[l], 1, none,
                                                       done, st)));
      src32 = dst;
      cur ^= 1;
    }
  }
  return STST_OK;
}

// grid of the last backward mode product (number of partials it writes)
int fd_partials_count(stst_problem *h) {
  long long ncols = h->N_dof / h->dir[1].n;
  if (h->prec_mode == STST_PREC_BF16) return tc_partials_count(ncols);
  if (h->pencil && h->prec_mode == STST_PREC_FP32 && h->d == 1) return (int)(h->N_s / h->dir[1].n * h->pencil);
  if (h->fd2d && h->prec_mode == STST_PREC_FP32 && (!h->pencil || h->d == 3)) return (int)(fd2d_slabs(h) * h->fd2d_b);
  if (h->prec_mode == STST_PREC_FP32 && h->mp_cfg[1].tc && h->Utf[1] &&
      tf32_eligible(h->dir[1].n, h->n_t(), ncols / h->n_t(), h->w_t1))
    return tf32_partials_count(h->dir[1].n, h->n_t(), ncols / h->n_t());
  const dim3 g = modeprod_grid(h->dir[1].n, ncols, h->mp_cfg[1]);
  return (int)(g.x * g.y);
}

// ---- choice of the time-solve kernel --------------------------------------------------------------
// Measured (mode 1): both kernels timed in place on a work vector, cached per (precision, n_t, N_s, P).
// Otherwise the segmented kernel is used when the sequential one would leave SMs without a warp.
static std::map<std::tuple<int, int, long long, int>, int> g_ts_cache;
int g_ts_mode = 0;  // 0 chosen per shape, 1 sequential, 2 segmented where it fits

template <typename R>
static int tune_ts(stst_problem *h) {
  const int q = sizeof(R) == 8 ? 1 : 0;
  const int nt = h->n_t(), P = h->dir[0].p;
  const long long Ns = h->N_s;
  h->ts_seg[q] = 0;
  if (h->ts_S[q] < 2 || g_ts_mode == 1) return STST_OK;
  if (g_ts_mode == 2) {
    h->ts_seg[q] = 1;
    return STST_OK;
  }
  if (g_tune_enabled != 1) {
    h->ts_seg[q] = grid_for(Ns, 32) < 2 * 152 ? 1 : 0;
    return STST_OK;
  }
  const auto key = std::make_tuple((int)sizeof(R), nt, Ns, P);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_ts_cache.find(key);
    if (it != g_ts_cache.end()) {
      h->ts_seg[q] = it->second;
      return STST_OK;
    }
  }
  cudaStream_t st = h->stream;
  cudaEvent_t e0, e1;
  STST_CUDA(cudaEventCreate(&e0));
  STST_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int choice = 0, status = STST_OK;
  for (int v = 0; v < 2 && status == STST_OK; ++v) {
    h->ts_seg[q] = v;
    for (int w = 0; w < 2 && status == STST_OK; ++w) status = time_solve<R>(h, h->w_t1, nullptr, st);
    cudaEventRecord(e0, st);
    for (int w = 0; w < 5 && status == STST_OK; ++w) status = time_solve<R>(h, h->w_t1, nullptr, st);
    cudaEventRecord(e1, st);
    const cudaError_t es = cudaEventSynchronize(e1);
    if (es != cudaSuccess) {
      stst_last_cuda = es;
      status = STST_ERR_CUDA;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (status == STST_OK && ms < best) {
      best = ms;
      choice = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  STST_TRY(status);
  h->ts_seg[q] = choice;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_ts_cache[key] = choice;
  }
  return STST_OK;
}

// ---- choice between fused and separate 2D transforms (FP32 preconditioner, d = 2) -------------------
// h->fd2d = number S of CTAs per (t, x_3) slab of the fused kernel, 0 for the separate mode products;
// h->fd2d_b the same for the backward transform. Measured (autotune mode 1): a forward plus a backward
// transform of each variant timed on work vectors decides fused or separate; then, fused, each
// transform is timed alone per split in the form the solve runs it (forward: FP64 residual in; backward:
// FP64 out with the flexible CG's four epilogue inner products), and each keeps its fastest split.
// Cached per shape. Otherwise S is the smallest split giving two CTAs per SM, for both.
int g_fd2d_mode = 0;  // 0 chosen per shape, 1 separate kernels, 2 fused where it fits, 10 + S fused with split S
static std::map<std::tuple<int, int, int, int>, std::pair<int, int>> g_fd2d_cache;  // (n_t, n_1, n_2, n_3 or 0)

static int fd2d_default_split(const stst_problem *h) {
  int S = 1;
  while (S < FD2D_MAXS && fd2d_slabs(h) * S < 2 * 152 && fd2d_split_ok(h->dir[1].n, h->dir[2].n, S + 1)) ++S;
  return S;
}

static int tune_fd2d(stst_problem *h) {
  h->fd2d = h->fd2d_b = 0;
  if (h->prec_mode != STST_PREC_FP32 || !fd2d_fits(h) || g_fd2d_mode == 1) return STST_OK;
  if (g_fd2d_mode > 10 && fd2d_split_ok(h->dir[1].n, h->dir[2].n, g_fd2d_mode - 10)) {
    h->fd2d = h->fd2d_b = g_fd2d_mode - 10;
    return STST_OK;
  }
  if (g_fd2d_mode >= 2 || g_tune_enabled != 1) {
    h->fd2d = h->fd2d_b = fd2d_default_split(h);
    return STST_OK;
  }
  const auto key = std::make_tuple(h->n_t(), h->dir[1].n, h->dir[2].n, h->d == 3 ? h->dir[3].n : 0);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_fd2d_cache.find(key);
    if (it != g_fd2d_cache.end()) {
      h->fd2d = it->second.first;
      h->fd2d_b = it->second.second;
      return STST_OK;
    }
  }
  cudaStream_t st = h->stream;
  float2 *X = (float2 *)h->w_t1, *Y = (float2 *)h->w_t1 + h->N_dof;  // two FP32 vectors in one FP64 one
  float2 *Z = (float2 *)h->w_t2;
  STST_CUDA(cudaMemsetAsync(h->w_t1, 0, sizeof(double) * 2 * h->N_dof, st));
  long long inner[3], outer[3];
  inner[1] = h->n_t();
  outer[1] = h->N_dof / (inner[1] * h->dir[1].n);
  inner[2] = inner[1] * h->dir[1].n;
  outer[2] = h->N_dof / (inner[2] * h->dir[2].n);
  cudaEvent_t e0, e1;
  STST_CUDA(cudaEventCreate(&e0));
  STST_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int choice = 0, status = STST_OK;
  for (int S = 0; S <= FD2D_MAXS && status == STST_OK; ++S) {
    if (S > 0 && !fd2d_split_ok(h->dir[1].n, h->dir[2].n, S)) continue;
    auto run = [&]() -> int {
      if (S > 0) {
        STST_TRY((launch_fd2d<float2, float2>(X, Y, h, 0, EpiDot(), nullptr, st, S)));
        return launch_fd2d<float2, float2>(Y, X, h, 1, EpiDot(), nullptr, st, S);
      }
      STST_TRY((mp32<float2, float2>(h, 1, X, Z, inner[1], outer[1], 0, EpiDot(), nullptr, st)));
      STST_TRY((mp32<float2, float2>(h, 2, Z, Y, inner[2], outer[2], 0, EpiDot(), nullptr, st)));
      STST_TRY((mp32<float2, float2>(h, 2, Y, Z, inner[2], outer[2], 1, EpiDot(), nullptr, st)));
      return mp32<float2, float2>(h, 1, Z, X, inner[1], outer[1], 1, EpiDot(), nullptr, st);
    };
    for (int w = 0; w < 2 && status == STST_OK; ++w) status = run();
    cudaEventRecord(e0, st);
    for (int w = 0; w < 5 && status == STST_OK; ++w) status = run();
    cudaEventRecord(e1, st);
    const cudaError_t es = cudaEventSynchronize(e1);
    if (es != cudaSuccess) {
      stst_last_cuda = es;
      status = STST_ERR_CUDA;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (status == STST_OK && ms < best) {
      best = ms;
      choice = S;
    }
  }
  // fused: each transform alone per split, in the form the solve runs it (the epilogue's inner products
  // read two FP64 work vectors and write the preconditioner's partial-sum slots, which every solve
  // recomputes before reading)
  int choice_b = choice;
  if (choice > 0 && status == STST_OK) {
    double2 *D = (double2 *)h->w_t2;
    STST_CUDA(cudaMemsetAsync(h->w_t2, 0, sizeof(double2) * h->N_dof, st));
    EpiDot ed;
    ed.a = h->w_r;
    ed.b = h->w_q;
    ed.part = h->partials + PS_Z * STST_MAXPART;
    ed.cplx = 1;
    float best_f = 1e30f, best_b = 1e30f;
    for (int S = 1; S <= FD2D_MAXS && status == STST_OK; ++S) {
      if (!fd2d_split_ok(h->dir[1].n, h->dir[2].n, S) ||
          (long long)fd2d_slabs(h) * S > STST_MAXPART)
        continue;
      for (int dir = 0; dir < 2 && status == STST_OK; ++dir) {
        auto run = [&]() -> int {
          if (dir == 0) return launch_fd2d<double2, float2>(D, X, h, 0, EpiDot(), nullptr, st, S);
          return launch_fd2d<float2, double2>(X, D, h, 1, ed, nullptr, st, S);
        };
        for (int w = 0; w < 2 && status == STST_OK; ++w) status = run();
        cudaEventRecord(e0, st);
        for (int w = 0; w < 5 && status == STST_OK; ++w) status = run();
        cudaEventRecord(e1, st);
        const cudaError_t es = cudaEventSynchronize(e1);
        if (es != cudaSuccess) {
          stst_last_cuda = es;
          status = STST_ERR_CUDA;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (status != STST_OK) break;
        if (dir == 0 && ms < best_f) {
          best_f = ms;
          choice = S;
        }
        if (dir == 1 && ms < best_b) {
          best_b = ms;
          choice_b = S;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  STST_TRY(status);
  h->fd2d = choice;
  h->fd2d_b = choice_b;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_fd2d_cache[key] = std::make_pair(choice, choice_b);
  }
  return STST_OK;
}

// ---- the pencil kernel or not (FP32 preconditioner) -------------------------------------------------
// h->pencil = CTAs per pencil (1 or 2), 0 for the transforms and time solves as separate kernels.
// Measured (autotune mode 1): one whole FP32 preconditioner application of each variant, timed on work
// vectors and cached per shape. Otherwise two CTAs per pencil where that fits, else one.
int g_pencil_mode = 0;  // 0 chosen per shape, 1 off, 2 one CTA per pencil, 3 a cluster of two
static std::map<std::tuple<int, int, int, int, int>, int> g_pencil_cache;

static int tune_pencil(stst_problem *h) {
  h->pencil = 0;
  if (h->prec_mode != STST_PREC_FP32 || !h->Gp32 || g_pencil_mode == 1) return STST_OK;
  const bool f1 = pencil_fits(h, 1), f2 = pencil_fits(h, 2);
  if (g_pencil_mode == 2 || g_pencil_mode == 3) {
    const int CL = g_pencil_mode - 1;
    h->pencil = (CL == 1 ? f1 : f2) ? CL : 0;
    return STST_OK;
  }
  if (g_tune_enabled != 1) {
    h->pencil = f2 ? 2 : (f1 ? 1 : 0);
    return STST_OK;
  }
  const auto key = std::make_tuple(h->n_t(), h->dir[0].p, h->dir[1].n, h->d >= 2 ? h->dir[2].n : 0,
                                   h->d == 3 ? h->dir[3].n : 0);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_pencil_cache.find(key);
    if (it != g_pencil_cache.end()) {
      h->pencil = it->second;
      return STST_OK;
    }
  }
  cudaStream_t st = h->stream;
  STST_CUDA(cudaMemsetAsync(h->w_r, 0, sizeof(double2) * h->N_dof, st));
  cudaEvent_t e0, e1;
  STST_CUDA(cudaEventCreate(&e0));
  STST_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int choice = 0, status = STST_OK;
  for (int CL = 0; CL <= 2 && status == STST_OK; ++CL) {
    if ((CL == 1 && !f1) || (CL == 2 && !f2)) continue;
    h->pencil = CL;
    auto run = [&]() { return fd_apply(h, h->w_r, h->w_z, 1, EpiDot(), nullptr, h->w_t1, h->w_t2); };
    for (int w = 0; w < 2 && status == STST_OK; ++w) status = run();
    cudaEventRecord(e0, st);
    for (int w = 0; w < 5 && status == STST_OK; ++w) status = run();
    cudaEventRecord(e1, st);
    const cudaError_t es = cudaEventSynchronize(e1);
    if (es != cudaSuccess) {
      stst_last_cuda = es;
      status = STST_ERR_CUDA;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (status == STST_OK && ms < best) {
      best = ms;
      choice = CL;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->pencil = choice;
  STST_TRY(status);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_pencil_cache[key] = choice;
  }
  return STST_OK;
}

int tune_modeprod(stst_problem *h) {
  // the mat-vec's occupancy queries are cached here, outside any stream capture
  for (int l = 0; l <= h->d; ++l)
    for (int threads : {256, 512}) {
      pass_resident<double>(h->dir[l].p, threads);
      pass_resident<float>(h->dir[l].p, threads);
    }
  if (h->tuned) return STST_OK;
  STST_TRY(tune_mp_tiles(h));
  STST_TRY(tune_ts<float>(h));
  if (h->prec_mode == STST_PREC_FP64) STST_TRY(tune_ts<double>(h));
  STST_TRY(tune_fd2d(h));
  STST_TRY(tune_pencil(h));
  h->tuned = 1;
  return STST_OK;
}

// ------------------------------------------------------------------------------------------------
// Persistent PCG for small problems (Sec. 5.3 and Sec. 6: CG preconditioned by P-hat, x_0 = 0): the whole
// solve of one problem in one thread-block cluster, many problems in one launch (one cluster each).
// Every phase is a loop over the problem's elements by the cluster's threads, phases are separated by
// the cluster's hardware barrier, and the vectors stay in L2: they are read with ld.global.cg and written
// with st.global.cg, because an SM's L1 would otherwise keep lines of a vector another SM has rewritten.
// Per iteration: the mat-vec's levels (the handle's plan), <p, A p>, the x and r updates with ||r||^2,
// Algorithm 1 (forward mode products, the banded time solves with the FP64 factors, backward mode
// products) with <r, z>, and p = z + beta p; sums over the cluster go through per-CTA partials read back
// in rank order (deterministic). The FP64 preconditioner (plain CG) only.
// ------------------------------------------------------------------------------------------------
#include <cooperative_groups.h>
namespace cg = cooperative_groups;

#define PERSIST_MAXC 16

struct PersistResult {
  int iters, status;
  double relres;
};

struct PersistProb {
  PassK lv[FUSED_MAXLEV];
  int lv_p[FUSED_MAXLEV];
  int n_lv;
  int d, P_t;
  int n[STST_MAXD + 1];              // n[0] = n_t, n[l] = n_l
  long long inner[STST_MAXD + 1];    // inner extent of mode l (l >= 1) in the time-fastest layout
  long long N_s, N;
  const double *U[STST_MAXD + 1];
  const double2 *G;                  // FP64 time factors (the layout of k_timesolve)
  const double *D;
  const double2 *b;
  double2 *x, *r, *p, *q, *z, *t1, *t2;
  double *part;                      // 3 x PERSIST_MAXC partial sums
  double tol;
  int maxit;
  PersistResult *res;
};

__device__ __forceinline__ double2 ldcg2(const double2 *a) { return __ldcg(a); }
__device__ __forceinline__ void stcg2(double2 *a, double2 v) { __stcg(a, v); }

// one output element of a mat-vec level, as pass_element but with L2 loads and stores
template <int P>
__device__ __forceinline__ void persist_level_element(const PassK &k, long long idx) {
  const long long inner = k.inner, nmo = k.n_mode_out;
  const long long c = idx % inner, t = idx / inner;
  const int j = (int)(t % nmo);
  const long long o = t / nmo;
  const long long base = o * k.n_mode_in * inner + c;
  for (int bo = 0; bo < k.n_out; ++bo) {
    double ax = 0.0, ay = 0.0;
    for (int ci = k.c_start[bo]; ci < k.c_start[bo + 1]; ++ci) {
      const double2 *in = (const double2 *)k.in[k.c_in[ci]];
      const double *m = (const double *)k.c_mat[ci] + j * (2 * P + 1);
      const bool im = k.c_imag[ci] != 0;
#pragma unroll
      for (int qq = 0; qq <= 2 * P; ++qq) {
        const int jj = j + k.row_off - P + qq;
        if (jj >= 0 && jj < k.n_mode_in) {
          const double2 xv = ldcg2(in + base + (long long)jj * inner);
          const double mv = m[qq];
          if (im) {
            ax -= mv * xv.y;
            ay += mv * xv.x;
          } else {
            ax += mv * xv.x;
            ay += mv * xv.y;
          }
        }
      }
    }
    stcg2((double2 *)k.out[bo] + idx, make_double2(ax, ay));
  }
}

#define PERSIST_MAXT 128  // time steps a thread stages in its local memory (longer series read L2 step by step)

// The banded time solve of system i with the recurrences of k_timesolve (Algorithm 1 step 3).
template <int P>
__device__ __forceinline__ void persist_time_solve_sys(const PersistProb &pr, double2 *Y, long long i) {
  const int nt = pr.n[0];
  const long long Ns = pr.N_s;
  // the system's series in thread-local memory: its loads are all issued before the recurrence
  double2 ybuf[PERSIST_MAXT];
  const bool staged = nt <= PERSIST_MAXT;
  if (staged)
    for (int t = 0; t < nt; ++t) ybuf[t] = ldcg2(Y + i * nt + t);
  double2 w[P];
#pragma unroll
  for (int a = 0; a < P; ++a) w[a] = make_double2(0.0, 0.0);
  for (int t = 0; t < nt; ++t) {  // G z = y: z_t = (y_t - sum_k G[t][t-k] z_{t-k}) / G[t][t]
    const double2 y = staged ? ybuf[t] : ldcg2(Y + i * nt + t);
    double ax = y.x, ay = y.y;
#pragma unroll
    for (int k = 1; k <= P; ++k) {
      const double2 g = pr.G[((long long)t * P + (k - 1)) * Ns + i];
      const double2 zz = w[k - 1];
      ax -= g.x * zz.x - g.y * zz.y;
      ay -= g.x * zz.y + g.y * zz.x;
    }
    const double dinv = pr.D[(long long)t * Ns + i];
    const double2 zt = make_double2(ax * dinv, ay * dinv);
#pragma unroll
    for (int a = P - 1; a > 0; --a) w[a] = w[a - 1];
    w[0] = zt;
    if (staged) ybuf[t] = zt;
    else stcg2(Y + i * nt + t, zt);
  }
#pragma unroll
  for (int a = 0; a < P; ++a) w[a] = make_double2(0.0, 0.0);
  for (int t = nt - 1; t >= 0; --t) {  // G^H x = z: x_t = (z_t - sum_k conj(G[t+k][t]) x_{t+k}) / G[t][t]
    const double2 zt = staged ? ybuf[t] : ldcg2(Y + i * nt + t);
    double ax = zt.x, ay = zt.y;
#pragma unroll
    for (int k = 1; k <= P; ++k) {
      if (t + k < nt) {
        const double2 g = pr.G[((long long)(t + k) * P + (k - 1)) * Ns + i];
        const double2 xv = w[k - 1];
        ax -= g.x * xv.x + g.y * xv.y;  // conj(g) x
        ay -= g.x * xv.y - g.y * xv.x;
      }
    }
    const double dinv = pr.D[(long long)t * Ns + i];
    const double2 xt = make_double2(ax * dinv, ay * dinv);
#pragma unroll
    for (int a = P - 1; a > 0; --a) w[a] = w[a - 1];
    w[0] = xt;
    stcg2(Y + i * nt + t, xt);
  }
}

// mode product along direction l: forward y[o, j, c] = sum_i U[i][j] x[o, i, c], backward with U^T
__device__ __forceinline__ void persist_mode_product(const PersistProb &pr, int l, const double2 *X, double2 *Y,
                                                     int backward, long long first, long long step) {
  const int n = pr.n[l];
  const long long inner = pr.inner[l];
  const double *U = pr.U[l];
  for (long long idx = first; idx < pr.N; idx += step) {
    const long long c = idx % inner, t = idx / inner;
    const int j = (int)(t % n);
    const long long o = t / n;
    const double2 *xs = X + o * n * inner + c;
    double ax = 0.0, ay = 0.0;
    int i = 0;
    for (; i + 8 <= n; i += 8) {  // eight loads in flight per step
      double2 v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = ldcg2(xs + (long long)(i + q) * inner);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const double u = backward ? U[j * n + i + q] : U[(i + q) * n + j];
        ax += u * v[q].x;
        ay += u * v[q].y;
      }
    }
    for (; i < n; ++i) {
      const double u = backward ? U[j * n + i] : U[i * n + j];
      const double2 v = ldcg2(xs + (long long)i * inner);
      ax += u * v.x;
      ay += u * v.y;
    }
    stcg2(Y + idx, make_double2(ax, ay));
  }
}

// sum of v over the cluster (every thread gets it): block sums written per CTA, read back in rank order
__device__ __forceinline__ double cluster_sum(double v, double *slot, double *sh, cg::cluster_group &cl) {
  const double s = block_sum(v, sh);
  if (threadIdx.x == 0) __stcg(slot + cl.block_rank(), s);
  cl.sync();
  double t = 0.0;
  const int C = (int)cl.num_blocks();
  for (int a = 0; a < C; ++a) t += __ldcg(slot + a);
  return t;
}

__global__ void __launch_bounds__(256) k_persist_pcg(const PersistProb *__restrict__ probs) {
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const PersistProb &pr = probs[blockIdx.x / C];
  __shared__ double sh[32];
  const long long first = (long long)cl.block_rank() * blockDim.x + threadIdx.x;
  const long long step = (long long)C * blockDim.x;
  const long long N = pr.N;
  double *pPQ = pr.part, *pRR = pr.part + PERSIST_MAXC, *pRZ = pr.part + 2 * PERSIST_MAXC;
  // x_0 = 0, r = b, ||b||^2
  double acc = 0.0;
  for (long long e = first; e < N; e += step) {
    const double2 bv = pr.b[e];
    stcg2(pr.x + e, make_double2(0.0, 0.0));
    stcg2(pr.r + e, bv);
    acc += bv.x * bv.x + bv.y * bv.y;
  }
  const double ff = cluster_sum(acc, pRR, sh, cl);
  int status = STST_OK, it = 0;
  double rr = ff;
  // z = P-hat^{-1} r (Algorithm 1 steps 2-4); <r, z>
  auto precondition = [&](double &rz) {
    const double2 *src = pr.r;
    double2 *bufs[2] = {pr.t1, pr.t2};
    int cur = 0;
    for (int l = 1; l <= pr.d; ++l) {
      persist_mode_product(pr, l, src, bufs[cur], 0, first, step);
      cl.sync();
      src = bufs[cur];
      cur ^= 1;
    }
    double2 *y = (double2 *)src;
    for (long long i = first; i < pr.N_s; i += step) {
      switch (pr.P_t) {
#define CASE(PP) case PP: persist_time_solve_sys<PP>(pr, y, i); break;
        CASE(1) CASE(2) CASE(3) CASE(4)
#undef CASE
        default: break;
      }
    }
    cl.sync();
    for (int l = pr.d; l >= 1; --l) {
      double2 *dst = l == 1 ? pr.z : bufs[cur];
      persist_mode_product(pr, l, src, dst, 1, first, step);
      cl.sync();
      src = dst;
      cur ^= 1;
    }
    double a = 0.0;
    for (long long e = first; e < N; e += step) {
      const double2 rv = ldcg2(pr.r + e), zv = ldcg2(pr.z + e);
      a += rv.x * zv.x + rv.y * zv.y;  // Re <r, z> (real for the Hermitian P-hat)
    }
    rz = cluster_sum(a, pRZ, sh, cl);
  };
  if (ff == 0.0) {
    rr = 0.0;
  } else {
    double rho;
    precondition(rho);
    for (long long e = first; e < N; e += step) stcg2(pr.p + e, ldcg2(pr.z + e));
    cl.sync();
    while (it < pr.maxit) {
      // q = A p by the plan's levels
      for (int lv = 0; lv < pr.n_lv; ++lv) {
        const PassK &k = pr.lv[lv];
        const long long total = k.outer * k.n_mode_out * k.inner;
        for (long long e = first; e < total; e += step) {
          switch (pr.lv_p[lv]) {
#define CASE(PP) case PP: persist_level_element<PP>(k, e); break;
            CASE(1) CASE(2) CASE(3) CASE(4)
#undef CASE
            default: break;
          }
        }
        cl.sync();
      }
      double a = 0.0;
      for (long long e = first; e < N; e += step) {
        const double2 pv = ldcg2(pr.p + e), qv = ldcg2(pr.q + e);
        a += pv.x * qv.x + pv.y * qv.y;
      }
      const double pq = cluster_sum(a, pPQ, sh, cl);
      if (!(pq > 0.0) || !isfinite(pq)) {
        status = STST_BREAKDOWN;
        break;
      }
      const double alpha = rho / pq;
      a = 0.0;
      for (long long e = first; e < N; e += step) {
        const double2 pv = ldcg2(pr.p + e), qv = ldcg2(pr.q + e);
        double2 xv = ldcg2(pr.x + e), rv = ldcg2(pr.r + e);
        xv.x += alpha * pv.x;
        xv.y += alpha * pv.y;
        rv.x -= alpha * qv.x;
        rv.y -= alpha * qv.y;
        stcg2(pr.x + e, xv);
        stcg2(pr.r + e, rv);
        a += rv.x * rv.x + rv.y * rv.y;
      }
      rr = cluster_sum(a, pRR, sh, cl);
      ++it;
      if (rr <= pr.tol * pr.tol * ff) break;
      double rho_new;
      precondition(rho_new);
      const double beta = rho_new / rho;
      rho = rho_new;
      for (long long e = first; e < N; e += step) {
        const double2 zv = ldcg2(pr.z + e);
        double2 pv = ldcg2(pr.p + e);
        pv.x = zv.x + beta * pv.x;
        pv.y = zv.y + beta * pv.y;
        stcg2(pr.p + e, pv);
      }
      cl.sync();
    }
    if (status == STST_OK && rr > pr.tol * pr.tol * ff) status = STST_NOT_CONVERGED;
  }
  if (cl.block_rank() == 0 && threadIdx.x == 0) {
    pr.res->iters = it;
    pr.res->status = status;
    pr.res->relres = ff > 0.0 ? sqrt(rr / ff) : 0.0;
  }
}

extern "C" int stst_persistent_solve(int count, const stst_handle *handles, const double *const *rhs,
                                     double *const *x, double tol, int maxit, int cluster_ctas, int *iters,
                                     int *status, double *relres, void *stream) {
  if (count < 1 || !handles || !rhs || !x || !(tol >= 0.0) || maxit < 0) return STST_ERR_ARG;
  const int C = cluster_ctas == 0 ? 8 : cluster_ctas;
  if (C != 1 && C != 2 && C != 4 && C != 8 && C != 16) return STST_ERR_ARG;
  std::vector<PersistProb> probs((size_t)count);
  for (int i = 0; i < count; ++i) {
    stst_problem *h = handles[i];
    if (!h || h->magic != STST_MAGIC) return STST_ERR_HANDLE;
    if (!rhs[i] || !x[i]) return STST_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (handles[j] == h) return STST_ERR_ARG;  // the work vectors are per handle
    if (!h->fd_ready || h->prec_mode != STST_PREC_FP64 || h->geo) return STST_ERR_STATE;
    const Plan &plan = h->sys_plan;
    const int np = (int)plan.passes.size();
    if (np < 1 || np > FUSED_MAXLEV) return STST_ERR_STATE;
    PersistProb &pr = probs[i];
    for (int ip = 0; ip < np; ++ip) {
      const PassParams &pp = plan.passes[ip];
      if (pp.p < 1 || pp.p > 4) return STST_ERR_STATE;  // degrees up to 4 (the kernel's cases)
      STST_TRY(make_level(plan, ip, h->w_p, 0, nullptr, pr.lv[ip]));
      pr.lv_p[ip] = pp.p;
    }
    pr.lv[np - 1].out[0] = h->w_q;
    pr.n_lv = np;
    pr.d = h->d;
    pr.P_t = h->dir[0].p;
    if (pr.P_t < 1 || pr.P_t > 4) return STST_ERR_STATE;
    long long acc = h->n_t();
    pr.n[0] = h->n_t();
    for (int l = 1; l <= h->d; ++l) {
      pr.n[l] = h->dir[l].n;
      pr.inner[l] = acc;
      acc *= h->dir[l].n;
      pr.U[l] = h->U[l];
    }
    pr.N_s = h->N_s;
    pr.N = h->N_dof;
    pr.G = (const double2 *)h->Hg;
    pr.D = h->Hd;
    pr.b = (const double2 *)rhs[i];
    pr.x = (double2 *)x[i];
    pr.r = (double2 *)h->w_r;
    pr.p = (double2 *)h->w_p;
    pr.q = (double2 *)h->w_q;
    pr.z = (double2 *)h->w_z;
    pr.t1 = (double2 *)h->w_t1;
    pr.t2 = (double2 *)h->w_t2;
    pr.tol = tol;
    pr.maxit = maxit;
  }
  for (int i = 0; i < count; ++i) STST_CUDA(cudaStreamSynchronize(handles[i]->stream));
  cudaStream_t st = stream ? (cudaStream_t)stream : handles[0]->stream;
  // descriptors, partial sums and results: one allocation, freed before returning
  const size_t bytes_probs = sizeof(PersistProb) * count;
  const size_t bytes_part = sizeof(double) * 3 * PERSIST_MAXC * count;
  const size_t bytes_res = sizeof(PersistResult) * count;
  char *dmem = nullptr;
  STST_CUDA(cudaMalloc(&dmem, bytes_probs + bytes_part + bytes_res));
  PersistProb *dprobs = (PersistProb *)dmem;
  double *dpart = (double *)(dmem + bytes_probs);
  PersistResult *dres = (PersistResult *)(dmem + bytes_probs + bytes_part);
  for (int i = 0; i < count; ++i) {
    probs[i].part = dpart + (size_t)3 * PERSIST_MAXC * i;
    probs[i].res = dres + i;
  }
  std::vector<PersistResult> hres((size_t)count);
  int s = STST_OK;
  if (cudaMemcpyAsync(dprobs, probs.data(), bytes_probs, cudaMemcpyHostToDevice, st) != cudaSuccess) s = STST_ERR_CUDA;
  if (s == STST_OK) {
    if (C == 16) cudaFuncSetAttribute(k_persist_pcg, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(count * C));
    cfg.blockDim = dim3(256);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    STST_PROF("persist_pcg", st);
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_persist_pcg, (const PersistProb *)dprobs);
    if (e != cudaSuccess) {
      stst_last_cuda = e;
      s = STST_ERR_CUDA;
    }
  }
  if (s == STST_OK &&
      (cudaMemcpyAsync(hres.data(), dres, bytes_res, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess))
    s = STST_ERR_CUDA;
  cudaStreamSynchronize(st);
  cudaFree(dmem);
  if (s != STST_OK) return s;
  int worst = STST_OK;
  for (int i = 0; i < count; ++i) {
    if (iters) iters[i] = hres[i].iters;
    if (status) status[i] = hres[i].status;
    if (relres) relres[i] = hres[i].relres;
    if (hres[i].status > worst) worst = hres[i].status;
  }
  return worst;
}
