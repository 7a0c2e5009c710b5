// Mode-n products of Algorithm 1 (steps 2 and 4) on the tensor cores in 3xTF32, fed by TMA.
//
// For mode l the product y[o, j, c] = sum_i U'[i][j] x[o, i, c] (U' = U forward, U^T backward) is a real
// GEMM per outer index o: the complex columns c give two GEMM rows each (real and imaginary part, which are
// adjacent floats in memory), the mode index i is the contraction K and j the output N. A CTA takes tiles
// of 64 complex columns (M = 128 rows): one TMA copy (cp.async.bulk.tensor, a 3D box of 128 floats x n rows
// of one o) brings the tile into shared memory, a conversion pass splits every value v into TF32 parts
// hi + lo (tf32_split), written in the K-major core-matrix layout, and one thread issues the products
// x_hi U_hi + x_hi U_lo + x_lo U_hi (tcgen05.mma kind::tf32, FP32 accumulation in TMEM): each term of the
// contraction is good to about 2^-21 relative, near the FP32 SIMT products. U' is split the same way once
// per setup, its two parts stacked along N ([U_hi | U_lo], 2 n columns), so that one product per k-step
// gives x_hi U_hi and x_hi U_lo side by side and a second, of N = n, adds x_lo U_hi: a product costs the
// tensor core about the same time for any N up to 256, and this takes two per k-step instead of three.
// Epilogue warps read the accumulators with tcgen05.ld, add the two halves and store FP32 (or FP64)
// results.
// The CTA is persistent and warp-specialised, so that copy, split, products and epilogue of consecutive
// tiles overlap: a TMA ring of up to four stages, two A buffers and two sets of TMEM accumulators, handed
// between the roles by mbarriers (k_modeprod_tf32).
//
// TMA needs the row pitch of the tensor (inner complex values = 8 inner bytes) to be a multiple of 16 bytes,
// so the kernel serves modes with an even inner extent and FP32 input; the x coordinate of every box is a
// multiple of 128 floats (512 bytes), a box past the end of a row is filled with zeros.
//
// Every wait is bounded: when one expires the CTA sets bit 2 of *errflag, the other roles give up at their
// next wait, the copies and products still in flight are waited for (bounded), TMEM is freed and the CTA
// returns.
#include "common.cuh"
#include "async.cuh"
#include <cuda.h>
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>

// byte offset of element (r, k) of a K-major, non-swizzled 4-byte operand of `rows` rows: core matrices of
// 8 rows x 16 bytes (4 values of K); the two core matrices of one k-step (8 values of K) are adjacent
// (128 bytes apart, the leading offset), the 8-row groups of a k-step follow each other (256 bytes apart,
// the stride offset), and k-step ks starts at ks * rows * 32 bytes. Every product thus reads one contiguous
// block (rows x 32 bytes) per operand; with the 8-row groups of a row further apart (all k-steps of a row
// group together) the same products ran about four times slower.
__host__ __device__ __forceinline__ unsigned tf32_kmajor_off(int r, int k, int rows) {
  return (unsigned)((k >> 3) * (rows * 32) + (r >> 3) * 256 + ((k >> 2) & 1) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

__host__ __device__ __forceinline__ int tf32_np(int n) { return (n + 15) / 16 * 16; }
__host__ __device__ __forceinline__ int tf32_kp(int n) { return (n + 7) / 8 * 8; }

// v rounded to the nearest TF32 value (10 explicit mantissa bits; ties away from zero), by integer arithmetic
// on the bit pattern: the tensor core itself would drop the 13 low bits. Finite inputs only.
__host__ __device__ __forceinline__ unsigned tf32_round_bits(unsigned b) { return (b + 0x1000u) & 0xFFFFE000u; }

// v = hi + lo + e: hi = v rounded to TF32, lo = (v - hi) rounded to TF32 (v - hi is exact in FP32), so
// |lo| <= 2^-11 |v| and |e| <= 2^-23 |v|. Rounding (rather than the tensor core's dropping of the low bits)
// keeps the errors of the three products unbiased: a truncated split errs toward zero in every term, and
// those errors add up along the contraction instead of cancelling.
__device__ __forceinline__ void tf32_split(float v, float &hi, float &lo) {
  hi = __uint_as_float(tf32_round_bits(__float_as_uint(v)));
  lo = __uint_as_float(tf32_round_bits(__float_as_uint(v - hi)));
}

// U' planes for direction l: [forward | backward], each 2 np x kp floats in the K-major layout with rows
// j < np the TF32 high parts and rows np + j the low parts of output index j, columns = contraction index i:
// forward U'[i][j] = U[i][j], backward U[j][i].
__global__ void k_u_to_tf32_kmajor(const double *__restrict__ U, int n, int np, int kp, float *out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= np * kp) return;
  const int j = e / kp, i = e - (e / kp) * kp;
  float vf = 0.f, vb = 0.f;
  if (i < n && j < n) {
    vf = (float)U[i * n + j];
    vb = (float)U[j * n + i];
  }
  const size_t plane = (size_t)2 * np * kp;
  const unsigned oh = tf32_kmajor_off(j, i, 2 * np) / 4, ol = tf32_kmajor_off(np + j, i, 2 * np) / 4;
  float hf, lf, hb, lb;
  tf32_split(vf, hf, lf);
  tf32_split(vb, hb, lb);
  out[oh] = hf;
  out[ol] = lf;
  out[plane + oh] = hb;
  out[plane + ol] = lb;
}

int launch_u_to_tf32(const double *U, int n, float *out, cudaStream_t s) {
  const int np = tf32_np(n), kp = tf32_kp(n);
  k_u_to_tf32_kmajor<<<grid_for((long long)np * kp, 256), 256, 0, s>>>(U, n, np, kp, out);
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}

size_t tf32_planes_floats(int n) { return 4 * (size_t)tf32_np(n) * tf32_kp(n); }

__device__ __forceinline__ uint64_t tf32_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version; no swizzle, base offset 0
  return d;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, unsigned parity) {
  unsigned fin;
  asm volatile(
      "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(fin)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return fin != 0;
}

// true when the barrier's phase with the given parity has completed, polled at most `limit` times
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, int limit) {
  for (int it = 0; it < limit; ++it)
    if (mbar_try(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

// 3D tile copy of the TMA unit: box at (x, y, z) of the tensor map into shared memory, completion counted in
// bytes on the mbarrier
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::
          "r"(smem_u32(dst)),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

constexpr int TF32_WAIT = 1 << 22;  // polls of a bounded wait (a normal wait takes microseconds)
constexpr int TF32_MAXS = 6;        // TMA stages at most

// One thread's bounded wait for a barrier phase. It gives up early when another role has given up (*abort),
// and on expiry records the failure (bit 2 of *errflag) and tells the other roles. Roles off the critical
// path back off (nanosleep) between polls, so that their spinning leaves the issue slots to the warps
// that work; at most TF32_WAIT polls of at most about a microsecond each.
__device__ __forceinline__ bool role_wait(uint64_t *bar, unsigned parity, volatile int *abort, int *errflag,
                                          unsigned backoff_ns = 0) {
  for (int it = 0; it < TF32_WAIT; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255) == 255 && *abort) return false;
    if (backoff_ns) __nanosleep(backoff_ns);
  }
  *abort = 1;
  atomicOr(errflag, 4);
  return false;
}

// The same for a whole warp: lane 0 polls, the warp follows its decision, and on success every lane observes
// the completed phase itself (so that each has the barrier's acquire ordering)
__device__ __forceinline__ bool warp_wait(uint64_t *bar, unsigned parity, volatile int *abort, int *errflag,
                                          unsigned backoff_ns = 64) {
  bool ok = false;
  if ((threadIdx.x & 31) == 0) ok = role_wait(bar, parity, abort, errflag, backoff_ns);
  ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
  if (ok)
    while (!mbar_try(bar, parity)) {
    }
  return ok;
}

// Warp-specialised persistent CTA of 18 warps; the CTA's tiles are t_k = blockIdx.x + k gridDim.x, k = 0, 1, ...
// (tile t: complex columns c0 .. c0 + 63, c0 = 64 (t mod tpo), of outer index o = t / tpo).
//   warp 16 (one thread): TMA producer, S stages; waits for a stage to be released, then copies tile k into it.
//   warps 0-7: split stage k mod S into TF32 parts in A buffer k mod NB (thread: GEMM row m = tid mod 128,
//              one half of the K range), release the stage and mark the A buffer full.
//   warp 17 (one thread): waits for the A buffer and for accumulator set k mod 2 to be free, issues the
//              three products and commits them (the commit frees the A buffer and fills the accumulators).
//              The products of a tile go round-robin into nacc independent accumulators, which the tensor
//              core can work on at the same time.
//   warps 8-15: epilogue; warp w reads TMEM lanes 32 (w mod 4) .. + 31 and one half of the output
//              columns, sums the nacc accumulators, frees the set, and stores the outputs (and the
//              epilogue's inner products).
// Shared memory: S stages (n x 128 floats, 1 KB aligned) | NB x (A hi | A lo) (128 x kp each) | B (2 np x kp:
// U' high parts, then low parts).
// Barriers (phase of use j of a buffer: parity j & 1): full[s] (TMA bytes), empty[s] (256 converter
// threads), afull[b] (256), afree[b] (MMA commit), accfull[a] (MMA commit), accempty[a] (256 epilogue threads).
constexpr int TF32_THREADS = 576;

template <typename TO>
__global__ void __launch_bounds__(TF32_THREADS, 1) k_modeprod_tf32(const __grid_constant__ CUtensorMap tmap,
                                                                   TO *__restrict__ Y, const float *__restrict__ Bk,
                                                                   int n, int np, int kp,
                                                                   int tmem_cols, int nacc, long long inner, int tpo,
                                                                   long long ntiles, int S, int NB, const EpiDot ed,
                                                                   const int *done, int *errflag) {
  if (done && *done) return;
  extern __shared__ __align__(1024) unsigned char tf_smem[];
  const unsigned stage_bytes = (unsigned)n * 512u;
  const unsigned stage_pitch = (stage_bytes + 1023u) & ~1023u;
  float *sA = (float *)(tf_smem + (size_t)S * stage_pitch);  // buffer b: hi at sA + 2 b 128 kp, lo 128 kp later
  float *sB = sA + (size_t)NB * 2 * 128 * kp;
  __shared__ __align__(8) uint64_t full[TF32_MAXS], empty[TF32_MAXS], afull[2], afree[2], accfull[2], accempty[2];
  __shared__ unsigned tmem_base;
  __shared__ volatile int abort_flag;
  __shared__ double sh[32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  {
    const int chunks = 2 * np * kp * 4 / 16;
    for (int q = tid; q < chunks; q += blockDim.x) cp_async<16>((char *)sB + 16 * q, (const char *)Bk + 16 * q);
    cp_async_commit();
  }
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 256);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&afull[b], 256);
      mbar_init(&afree[b], 1);
      mbar_init(&accfull[b], 1);
      mbar_init(&accempty[b], 256);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 17) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  cp_async_wait_all();
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // B planes (generic writes) -> tensor core
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const unsigned tmem = tmem_base;
  const long long first = blockIdx.x, step = gridDim.x;
  const int ntile_cta = first < ntiles ? (int)((ntiles - 1 - first) / step + 1) : 0;
  double dacc[4] = {0.0, 0.0, 0.0, 0.0};
  if (warp == 16) {
    if (lane == 0) {
      int k = 0;
      for (; k < ntile_cta; ++k) {
        const int s = k % S, u = k / S;
        if (k >= S && !role_wait(&empty[s], (unsigned)((u - 1) & 1), &abort_flag, errflag, 64)) break;
        const long long t = first + (long long)k * step;
        const int o = (int)(t / tpo), c0 = (int)(t - (long long)o * tpo) * 64;
        mbar_expect_tx(&full[s], stage_bytes);
        tma_load_3d(tf_smem + (size_t)s * stage_pitch, &tmap, 2 * c0, 0, o, &full[s]);
      }
      // copies still in flight (after an abort): the last one issued on each stage, bounded
      for (int s = 0; s < S && s < k; ++s) {
        const int last = k - 1 - ((k - 1 - s) % S);  // the last tile issued on stage s
        mbar_wait_bounded(&full[s], (unsigned)((last / S) & 1), TF32_WAIT);
      }
    }
  } else if (warp == 17) {
    // the whole warp runs the loop (converged, the descriptors stay warp-uniform); one elected lane issues
    const unsigned LBO = 128, SBO = 256;
    // kind::tf32 instruction descriptors: D FP32 (bits 4-5 = 1), A and B TF32 (bits 7-9 and 10-12 = 2), both
    // K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28; N = 2 np (x_hi [U_hi | U_lo]) and N = np (x_lo U_hi)
    const uint32_t idesc_w =
        (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(2 * np >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    const uint32_t idesc_n =
        (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(np >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    const int nks = kp / 8;
    // descriptors of k-step 0 of each operand plane; k-step ks starts ks * rows * 32 bytes further (A: 4096
    // bytes = 256 units of the descriptor's address field; B: 2 np rows, 4 np units; its first np rows are
    // U_hi), A buffer b 1024 kp bytes after buffer 0
    const uint64_t dB = tf32_desc(smem_u32(sB), LBO, SBO);
    const uint64_t dAh0 = tf32_desc(smem_u32(sA), LBO, SBO), dAl0 = tf32_desc(smem_u32(sA + 128 * kp), LBO, SBO);
    const uint64_t dAstep = (uint64_t)(1024 * kp) >> 4;
    int k = 0;
    for (; k < ntile_cta; ++k) {
      const int b = k % NB, jb = k / NB, a = k & 1, ja = k >> 1;
      if (!warp_wait(&afull[b], (unsigned)(jb & 1), &abort_flag, errflag, 0)) break;
      if (k >= 2 && !warp_wait(&accempty[a], (unsigned)((ja - 1) & 1), &abort_flag, errflag, 0)) break;
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      unsigned elected;
      asm volatile("{\n.reg .pred e;\nelect.sync _|e, 0xffffffff;\nselp.u32 %0, 1, 0, e;\n}\n" : "=r"(elected));
      const unsigned d0 = tmem + (unsigned)(a * nacc * 2 * np);
      const uint64_t dah = dAh0 + (uint64_t)b * dAstep, dal = dAl0 + (uint64_t)b * dAstep;
      // k-step ks goes into accumulator ks mod nacc (2 np columns); its first product there overwrites it
      int c = 0;
      unsigned d = d0;
      for (int ks = 0; ks < nks; ++ks) {
        if (elected) {
          const uint64_t db = dB + (uint64_t)(4 * np) * ks;
          asm volatile(
              "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
              "l"(dah + 256 * ks), "l"(db), "r"(idesc_w), "r"(ks >= nacc ? 1 : 0));
          asm volatile(
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;\n" ::"r"(d),
              "l"(dal + 256 * ks), "l"(db), "r"(idesc_n));
        }
        if (++c == nacc) {
          c = 0;
          d = d0;
        } else {
          d += 2 * np;
        }
      }
      if (elected) {
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                         smem_u32(&afree[b]))
                     : "memory");
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                         smem_u32(&accfull[a]))
                     : "memory");
      }
      __syncwarp();
    }
    // products still in flight: the last commit covers every product issued before it
    if (lane == 0 && k > 0) mbar_wait_bounded(&accfull[(k - 1) & 1], (unsigned)(((k - 1) >> 1) & 1), TF32_WAIT);
  } else if (warp < 8) {
    // converters: GEMM row m (part m & 1 of complex column m >> 1), K chunks [k4a, k4b) of 4
    const int m = tid & 127, half = tid >> 7;
    const int nk4 = kp >> 2, k4a = half ? (nk4 + 1) / 2 : 0, k4b = half ? nk4 : (nk4 + 1) / 2;
    for (int k = 0; k < ntile_cta; ++k) {
      const int s = k % S, u = k / S, b = k % NB, jb = k / NB;
      if (!warp_wait(&full[s], (unsigned)(u & 1), &abort_flag, errflag)) break;
      if (k >= NB && !warp_wait(&afree[b], (unsigned)((jb - 1) & 1), &abort_flag, errflag)) break;
      const float *sT = (const float *)(tf_smem + (size_t)s * stage_pitch);
      float *ah = sA + (size_t)b * 2 * 128 * kp, *al = ah + 128 * kp;
#pragma unroll 2
      for (int k4 = k4a; k4 < k4b; ++k4) {
        float v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int kk = 4 * k4 + q;
          v[q] = kk < n ? sT[kk * 128 + m] : 0.f;
        }
        float4 hv, lv;
        tf32_split(v[0], hv.x, lv.x);
        tf32_split(v[1], hv.y, lv.y);
        tf32_split(v[2], hv.z, lv.z);
        tf32_split(v[3], hv.w, lv.w);
        const unsigned off = tf32_kmajor_off(m, 4 * k4, 128);
        *(float4 *)((char *)ah + off) = hv;
        *(float4 *)((char *)al + off) = lv;
      }
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // A planes -> tensor core
      mbar_arrive(&empty[s]);
      mbar_arrive(&afull[b]);
    }
  } else {
    // epilogue: TMEM lane m = GEMM row m; 16-column chunks [c16a, c16b) of the accumulators
    const int g = warp & 3, m = 32 * g + lane, part = m & 1, half = (warp - 8) >> 2;
    const int nc16 = np >> 4, c16a = half ? (nc16 + 1) / 2 : 0, c16b = half ? nc16 : (nc16 + 1) / 2;
    using R = decltype(TO().x);
    for (int k = 0; k < ntile_cta; ++k) {
      const int a = k & 1, ja = k >> 1;
      if (!warp_wait(&accfull[a], (unsigned)(ja & 1), &abort_flag, errflag)) break;
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const long long t = first + (long long)k * step;
      const int o = (int)(t / tpo);
      const long long c = (t - (long long)o * tpo) * 64 + (m >> 1);
      const bool in = c < inner;
      if (c16a == c16b) {  // no chunk for this half (np = 16): only the release
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        mbar_arrive(&accempty[a]);
      }
      // this warp's chunks of 16 columns, one at a time: both halves of the nacc accumulators read and
      // summed, then stored; the set is released right after the last chunk's loads
      for (int c16 = c16a; c16 < c16b; ++c16) {
        const int j0 = 16 * c16;
        float sm16[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) sm16[q] = 0.f;
        for (int h2 = 0; h2 < 2 * nacc; ++h2) {  // accumulator h2 / 2, half h2 % 2 (x U_hi, x_hi U_lo)
          unsigned r[16];
          const unsigned taddr =
              tmem + ((unsigned)(32 * g) << 16) + (unsigned)((a * nacc + (h2 >> 1)) * 2 * np + (h2 & 1) * np + j0);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
              : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
              : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
          for (int q = 0; q < 16; ++q) sm16[q] += __uint_as_float(r[q]);
        }
        if (c16 + 1 == c16b) {
          asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
          mbar_arrive(&accempty[a]);
        }
        if (in) {
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int j = j0 + q;
            if (j < n) {
              const long long idx = ((long long)o * n + j) * inner + c;
              const float v = sm16[q];
              if constexpr (sizeof(TO) == 16) ((double *)Y)[2 * idx + part] = (double)v;
              else ((float *)Y)[2 * idx + part] = v;
              if (ed.part) {
                // conj(a) v: the real part takes a[part] v, the imaginary part (-1)^(1-part) a[1-part] v
                const R *ea = (const R *)ed.a + 2 * idx;
                const double sgn = part ? 1.0 : -1.0;
                dacc[0] += (double)ea[part] * (double)v;
                if (ed.cplx) {
                  dacc[1] += sgn * (double)ea[1 - part] * (double)v;
                  if (ed.b) {
                    const R *eb = (const R *)ed.b + 2 * idx;
                    dacc[2] += (double)eb[part] * (double)v;
                    dacc[3] += sgn * (double)eb[1 - part] * (double)v;
                  }
                }
              }
            }
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 17) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tmem_cols));
  }
  if (ed.part) epi_dot_store(dacc, ed, blockIdx.x, sh);
}

// ---- host side ----------------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)f;
  });
  return fn;
}

// Shared-memory plan: S TMA stages (up to 4) and NB A buffers (2, else 1), the largest that fit the opt-in
// limit (less 2 KB for the static part); false when not even two stages and one A buffer fit.
struct Tf32Plan {
  int S, NB;
  size_t smem;
};

static size_t tf32_smem_of(int n, int S, int NB) {
  const size_t stage = ((size_t)n * 512 + 1023) / 1024 * 1024;
  const int np = tf32_np(n), kp = tf32_kp(n);
  return S * stage + (size_t)NB * 2 * 128 * kp * 4 + 2 * (size_t)np * kp * 4;  // B: 2 np x kp
}

// independent accumulators (2 np columns each) per tile: up to 4, two sets within the 512 TMEM columns of an SM
static int tf32_nacc(int np) {
  const int a = 512 / (4 * np);
  return a > 4 ? 4 : (a < 1 ? 1 : a);
}

static int tf32_tmem_cols(int np) {
  int cols = 32;
  while (cols < 4 * tf32_nacc(np) * np) cols *= 2;
  return cols;
}

// opt-in shared memory per CTA and SM count of the current device, queried once per device
struct Tf32Dev {
  int optin, sms;
};

static Tf32Dev tf32_dev() {
  static std::mutex mu;
  static std::map<int, Tf32Dev> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  Tf32Dev a{0, 0};
  cudaDeviceGetAttribute(&a.optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&a.sms, cudaDevAttrMultiProcessorCount, dev);
  cache[dev] = a;
  return a;
}

static bool tf32_plan(int n, Tf32Plan *pl) {
  const int optin = tf32_dev().optin;
  const size_t limit = (size_t)optin > 2048 ? (size_t)optin - 2048 : 0;
  for (int NB = 2; NB >= 1; --NB)
    for (int S = 4; S >= 2; --S)
      if (tf32_smem_of(n, S, NB) <= limit) {
        pl->S = S;
        pl->NB = NB;
        pl->smem = tf32_smem_of(n, S, NB);
        return true;
      }
  return false;
}

// The shapes the kernel serves: FP32 input with 16-byte aligned rows (even inner extent, aligned base),
// n <= 96 (one box; at most six 16-column output chunks), 32-bit coordinates, and a shared-memory plan
// within the opt-in limit (n <= 80 on this GPU).
bool tf32_eligible(int n, long long inner, long long outer, const void *X) {
  if (n < 1 || n > 96 || inner < 2 || (inner & 1) || outer < 1) return false;
  if (inner >= (1LL << 29) || outer >= (1LL << 31)) return false;
  if (((uintptr_t)X & 15) != 0) return false;
  Tf32Plan pl;
  return tf32_plan(n, &pl);
}

// persistent grid: the CTAs that fit at once (the same for both output types, so that the number of partial
// sums is known before the launch; the FP64-output variant only differs in registers), and whose TMEM
// (tmem_cols each) fits the 512 columns of an SM
static int tf32_grid(size_t smem, int tmem_cols, long long ntiles, int *grid) {
  static std::mutex mu;
  static std::map<size_t, int> resident;  // CTAs per SM for a shared-memory size
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = resident.find(smem);
    if (it != resident.end()) per_sm = it->second;
  }
  if (per_sm == 0) {
    STST_TRY(ensure_dyn_smem((const void *)k_modeprod_tf32<float2>, smem));
    STST_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_modeprod_tf32<float2>, TF32_THREADS, smem));
    if (per_sm < 1) return STST_ERR_ARG;
    std::lock_guard<std::mutex> lk(mu);
    resident[smem] = per_sm;
  }
  if (per_sm * tmem_cols > 512) per_sm = 512 / tmem_cols;
  const long long g = (long long)per_sm * tf32_dev().sms;
  *grid = (int)(ntiles < g ? ntiles : g);
  return STST_OK;
}

// y = U'-product of mode l on the tensor cores. planes: the direction's four TF32 planes (launch_u_to_tf32);
// backward selects U^T. STST_ERR_ARG where tf32_eligible does not hold.
template <typename TO>
int launch_modeprod_tf32(const float2 *X, TO *Y, const float *planes, int backward, int n, long long inner,
                         long long outer, const EpiDot &ed, const int *done, int *errflag, cudaStream_t s) {
  if (!tf32_eligible(n, inner, outer, X)) return STST_ERR_ARG;
  EncodeTiledFn enc = encode_tiled_fn();
  if (!enc) return STST_ERR_CUDA;
  const int np = tf32_np(n), kp = tf32_kp(n);
  const int tpo = (int)((inner + 63) / 64);
  const long long ntiles = outer * tpo;
  // the tensor X as floats: x = 2 inner (real and imaginary parts), y = n, z = outer; one box = 64 complex
  // columns of all n rows of one outer index. Encoded once per (address, shape) and kept (the work vectors
  // of the handles times their directions; cleared past 1024 entries).
  CUtensorMap map;
  {
    static std::mutex mu;
    static std::map<std::tuple<const void *, int, long long, long long>, CUtensorMap> maps;
    const auto key = std::make_tuple((const void *)X, n, inner, outer);
    std::lock_guard<std::mutex> lk(mu);
    auto it = maps.find(key);
    if (it != maps.end()) {
      map = it->second;
    } else {
      const cuuint64_t dims[3] = {(cuuint64_t)(2 * inner), (cuuint64_t)n, (cuuint64_t)outer};
      const cuuint64_t strides[2] = {(cuuint64_t)(8 * inner), (cuuint64_t)(8 * inner * n)};
      const cuuint32_t box[3] = {128u, (cuuint32_t)n, 1u};
      const cuuint32_t estr[3] = {1u, 1u, 1u};
      const CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)X, dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return STST_ERR_ARG;
      if (maps.size() >= 1024) maps.clear();
      maps[key] = map;
    }
  }
  Tf32Plan pl;
  if (!tf32_plan(n, &pl)) return STST_ERR_ARG;
  STST_TRY(ensure_dyn_smem((const void *)k_modeprod_tf32<TO>, pl.smem));
  // two sets of nacc accumulators of 2 np columns; no more accumulators than k-steps
  const int nks = kp / 8;
  const int nacc = tf32_nacc(np) < nks ? tf32_nacc(np) : nks, tmem_cols = tf32_tmem_cols(np);
  int grid = 0;
  STST_TRY(tf32_grid(pl.smem, tmem_cols, ntiles, &grid));
  if (ed.part && grid > STST_MAXPART) return STST_ERR_ARG;
  const float *Bk = planes + (backward ? (size_t)2 * np * kp : 0);
  STST_PROF("modeprod_tf32x3_tc", s);
  k_modeprod_tf32<TO><<<grid, TF32_THREADS, pl.smem, s>>>(map, Y, Bk, n, np, kp, tmem_cols,
                                                          nacc, inner, tpo, ntiles, pl.S, pl.NB, ed, done, errflag);
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}

// number of partial sums the epilogue writes (one per CTA)
int tf32_partials_count(int n, long long inner, long long outer) {
  Tf32Plan pl;
  int grid = 0;
  if (!tf32_plan(n, &pl) ||
      tf32_grid(pl.smem, tf32_tmem_cols(tf32_np(n)), outer * ((inner + 63) / 64), &grid) != STST_OK)
    return 0;
  return grid;
}

template int launch_modeprod_tf32<float2>(const float2 *, float2 *, const float *, int, int, long long, long long,
                                          const EpiDot &, const int *, int *, cudaStream_t);
template int launch_modeprod_tf32<double2>(const float2 *, double2 *, const float *, int, int, long long, long long,
                                           const EpiDot &, const int *, int *, cudaStream_t);
