// Mode-n products of Algorithm 1 (steps 2 and 4) on the 5th-generation tensor cores.
//
// For mode l the product y[o, j, c] = sum_i U'[i][j] x[o, i, c] (U' = U forward, U^T backward) is a
// real GEMM: the complex columns (o, c) give two GEMM rows each (real and imaginary part), the mode
// index i is the contraction K and j the output N. A CTA (4 warps) owns 64 complex columns, i.e. one
// M = 128 tile. The x tile is read from global memory (FP64 or FP32), rounded to BF16 and written
// into shared memory in the K-major core-matrix layout (8 rows x 16 bytes, no swizzle); U' is laid
// out once per setup in the same layout (stst_build_fd) and copied in with cp.async. One thread
// issues ceil(n/16) tcgen05.mma (kind::f16, BF16 x BF16 -> FP32) into a TMEM accumulator of
// 128 lanes x N_pad columns and commits them to an mbarrier; after a bounded wait the four warps read
// their 32 lanes with tcgen05.ld and store FP32 (or FP64) results. TMEM is released on every path.
#include "common.cuh"
#include "async.cuh"
#include <cstdint>

// byte offset of element (r, k) in a K-major, non-swizzled operand with K padded to kp
__host__ __device__ __forceinline__ unsigned kmajor_off(int r, int k, int kp) {
  return (unsigned)((r >> 3) * ((kp >> 3) * 128) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// U' in BF16 K-major layout, rows = output index j (N), columns = contraction index i (K), zero padded:
// forward: coefficient of x_i in y_j is U[i][j]; backward: U[j][i]. Each value v is stored as a high
// part hi = bf16(v) and a low part lo = bf16(v - hi): out = [fwd hi | bwd hi | fwd lo | bwd lo].
__global__ void k_u_to_bf16_kmajor(const double *__restrict__ U, int n, int np, int kp, __nv_bfloat16 *out) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= np * kp) return;
  int j = e / kp, i = e - (e / kp) * kp;
  float vf = 0.f, vb = 0.f;
  if (i < n && j < n) {
    vf = (float)U[i * n + j];
    vb = (float)U[j * n + i];
  }
  const unsigned off = kmajor_off(j, i, kp) / 2;
  const size_t plane = (size_t)np * kp;
  const __nv_bfloat16 hf = __float2bfloat16(vf), hb = __float2bfloat16(vb);
  out[off] = hf;
  out[plane + off] = hb;
  out[2 * plane + off] = __float2bfloat16(vf - __bfloat162float(hf));
  out[3 * plane + off] = __float2bfloat16(vb - __bfloat162float(hb));
}

int launch_u_to_bf16(const double *U, int n, __nv_bfloat16 *out, cudaStream_t s) {
  const int np = (n + 15) / 16 * 16, kp = np;
  k_u_to_bf16_kmajor<<<grid_for((long long)np * kp, 256), 256, 0, s>>>(U, n, np, kp, out);
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}

__device__ __forceinline__ uint64_t umma_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version (bits 46-48 = 0b001); no swizzle, base offset 0
  return d;
}

// SPLIT = 1: one product of BF16-rounded operands. SPLIT = 3: operands split into high and low BF16
// parts, x U ~ x_hi U_hi + x_hi U_lo + x_lo U_hi (about 16 significant bits), all three into the same
// TMEM accumulator. Bk points at the high plane of U'; its low plane is lo_stride elements further.
template <typename TI, typename TO, int SPLIT>
__global__ void __launch_bounds__(128) k_modeprod_tc(const TI *__restrict__ X, TO *__restrict__ Y,
                                                     const __nv_bfloat16 *__restrict__ Bk, long long lo_stride, int n,
                                                     int np, int kp, long long inner, long long ncols,
                                                     const EpiDot ed,
                                                     const int *done, int *errflag) {
  if (done && *done) return;
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __nv_bfloat16 *sA = (__nv_bfloat16 *)tc_smem;   // 128 x kp (high part)
  __nv_bfloat16 *sB = sA + 128 * kp;              // np x kp (high part)
  __nv_bfloat16 *sAl = sB + np * kp;              // 128 x kp (low part, SPLIT == 3)
  __nv_bfloat16 *sBl = sAl + 128 * kp;            // np x kp (low part, SPLIT == 3)
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ unsigned tmem_base;
  __shared__ double sh[32];
  const int tid = threadIdx.x;
  const long long col0 = (long long)blockIdx.x * 64;
  // B tile: contiguous np*kp BF16, 16-byte chunks
  {
    const int chunks = np * kp * 2 / 16;
    for (int q = tid; q < chunks; q += 128) cp_async<16>((char *)sB + 16 * q, (const char *)Bk + 16 * q);
    if (SPLIT == 3)
      for (int q = tid; q < chunks; q += 128)
        cp_async<16>((char *)sBl + 16 * q, (const char *)(Bk + lo_stride) + 16 * q);
    cp_async_commit();
  }
  // x tile staged as FP32 complex sX[i][cc] (i < n, cc < 64): cp.async when the input is FP32, batched
  // register loads when it is FP64 (converted on the way); every load of the CTA is in flight at once
  float2 *sX = (float2 *)(SPLIT == 3 ? sBl + np * kp : sAl);  // right after the BF16 planes in use
  {
    const int cc = tid & 63, half = tid >> 6;
    const long long col = col0 + cc;
    const bool in = col < ncols;
    const long long o = in ? col / inner : 0, c = in ? col % inner : 0;
    const TI *src = X + o * n * inner + c;
    if constexpr (sizeof(TI) == 8) {
      for (int i = half; i < n; i += 2) {
        if (in) cp_async<8>(&sX[i * 64 + cc], src + (long long)i * inner);
        else sX[i * 64 + cc] = make_float2(0.f, 0.f);
      }
      cp_async_commit();
    } else {
      for (int i0 = half; i0 < n; i0 += 16) {
        TI v[8];
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          const int i = i0 + 2 * b;
          if (in && i < n) v[b] = src[(long long)i * inner];
          else { v[b].x = 0; v[b].y = 0; }
        }
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          const int i = i0 + 2 * b;
          if (i < n) sX[i * 64 + cc] = make_float2((float)v[b].x, (float)v[b].y);
        }
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();
  // BF16 operands in the K-major core-matrix layout: one 16-byte store per (row m, 8-wide K chunk);
  // row m = 2 cc + (imag part), columns k >= n are zero
  {
    const int nk8 = kp >> 3;
    for (int e = tid; e < 128 * nk8; e += 128) {
      const int m = e & 127, k8 = e >> 7;
      const int cc = m >> 1, part = m & 1;
      __align__(16) __nv_bfloat16 hv[8], lv[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int k = k8 * 8 + q;
        float v = 0.f;
        if (k < n) {
          const float2 t = sX[k * 64 + cc];
          v = part ? t.y : t.x;
        }
        hv[q] = __float2bfloat16(v);
        lv[q] = __float2bfloat16(v - __bfloat162float(hv[q]));
      }
      const unsigned off = kmajor_off(m, k8 * 8, kp);
      *(uint4 *)((char *)sA + off) = *(const uint4 *)hv;
      if (SPLIT == 3) *(uint4 *)((char *)sAl + off) = *(const uint4 *)lv;
    }
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;\n" ::"r"(smem_u32(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // generic-proxy smem writes -> tensor core
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const unsigned tmem = tmem_base;
  const unsigned LBO = 128, SBO = (unsigned)(kp / 8) * 128;
  if (tid == 0) {
    // kind::f16 instruction descriptor: D FP32 (bit 4), A and B BF16 (bits 7, 10), both K-major,
    // N >> 3 at bits 17-22, M >> 4 at bits 24-28
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(np >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    int acc = 0;
    for (int term = 0; term < SPLIT; ++term) {
      // term 0: hi x hi, term 1: hi x lo(U), term 2: lo(x) x hi
      const __nv_bfloat16 *a = (term == 2) ? sAl : sA;
      const __nv_bfloat16 *b = (term == 1) ? sBl : sB;
      for (int ks = 0; ks < kp / 16; ++ks) {
        const uint64_t da = umma_desc(smem_u32(a) + ks * 2 * LBO, LBO, SBO);
        const uint64_t db = umma_desc(smem_u32(b) + ks * 2 * LBO, LBO, SBO);
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc));
        acc = 1;
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     smem_u32(&mbar))
                 : "memory");
  }
  // bounded wait for the MMAs (phase 0 of the barrier)
  int ok = 0;
  for (int it = 0; it < (1 << 22) && !ok; ++it) {
    unsigned fin;
    asm volatile(
        "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], 0;\nselp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(fin)
        : "r"(smem_u32(&mbar))
        : "memory");
    ok = fin;
  }
  ok = __syncthreads_and(ok);  // one decision for the whole CTA (tcgen05.ld needs whole warps)
  if (!ok && tid == 0) atomicOr(errflag, 4);
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  // this thread holds part (0 real, 1 imaginary) of each output v; conj(a) v = (a.x v.x + a.y v.y) +
  // i (a.x v.y - a.y v.x), so the real part takes a[part] v and the imaginary part (-1)^(1-part) a[1-part] v
  double dacc[4] = {0.0, 0.0, 0.0, 0.0};
  if (ok) {
    const int m = tid;  // TMEM lane = GEMM row; warp w owns lanes 32w..32w+31
    const int cc = m >> 1, part = m & 1;
    const long long col = col0 + cc;
    const bool in = col < ncols;
    const long long o = in ? col / inner : 0, c = in ? col % inner : 0;
    for (int j0 = 0; j0 < np; j0 += 16) {
      unsigned r[16];
      const unsigned taddr = tmem + ((unsigned)(32 * (tid >> 5)) << 16) + (unsigned)j0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (in) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int j = j0 + q;
          if (j < n) {
            const long long idx = (o * n + j) * inner + c;
            const float v = __uint_as_float(r[q]);
            if constexpr (sizeof(TO) == 16) ((double *)Y)[2 * idx + part] = (double)v;
            else ((float *)Y)[2 * idx + part] = v;
            if (ed.part) {
              using R = decltype(TO().x);
              const R *a = (const R *)ed.a + 2 * idx;
              const double sgn = part ? 1.0 : -1.0;
              dacc[0] += (double)a[part] * (double)v;
              if (ed.cplx) {
                dacc[1] += sgn * (double)a[1 - part] * (double)v;
                if (ed.b) {
                  const R *b = (const R *)ed.b + 2 * idx;
                  dacc[2] += (double)b[part] * (double)v;
                  dacc[3] += sgn * (double)b[1 - part] * (double)v;
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
  if (tid < 32) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;\n" ::"r"(tmem));
  }
  if (ed.part) epi_dot_store(dacc, ed, blockIdx.x, sh);
}

int tc_partials_count(long long ncols) { return grid_for(ncols, 64); }

template <typename TI, typename TO>
int launch_modeprod_tc(const TI *X, TO *Y, const __nv_bfloat16 *Bk, long long lo_stride, int split, int n,
                       long long inner, long long outer, const EpiDot &ed, const int *done, int *errflag,
                       cudaStream_t s) {
  const long long ncols = inner * outer;
  const int np = (n + 15) / 16 * 16, kp = np;
  const int grid = grid_for(ncols, 64);
  if (ed.part && grid > STST_MAXPART) return STST_ERR_ARG;
  // BF16 operands (high, and low for the split) + the FP32 staging tile of 64 complex columns
  const size_t sm = (size_t)(split == 3 ? 2 : 1) * (128 + np) * kp * sizeof(__nv_bfloat16) +
                    (size_t)n * 64 * sizeof(float2);
  STST_PROF(split == 3 ? "modeprod_bf16x3_tc" : "modeprod_bf16_tc", s);
  if (split == 3) {
    STST_TRY(ensure_dyn_smem((const void *)k_modeprod_tc<TI, TO, 3>, sm));
    k_modeprod_tc<TI, TO, 3><<<grid, 128, sm, s>>>(X, Y, Bk, lo_stride, n, np, kp, inner, ncols, ed, done,
                                                   errflag);
  } else {
    STST_TRY(ensure_dyn_smem((const void *)k_modeprod_tc<TI, TO, 1>, sm));
    k_modeprod_tc<TI, TO, 1><<<grid, 128, sm, s>>>(X, Y, Bk, lo_stride, n, np, kp, inner, ncols, ed, done,
                                                   errflag);
  }
  STST_CUDA(cudaGetLastError());
  return STST_OK;
}

template int launch_modeprod_tc<double2, float2>(const double2 *, float2 *, const __nv_bfloat16 *, long long, int, int, long long, long long, const EpiDot &, const int *, int *, cudaStream_t);
template int launch_modeprod_tc<float2, float2>(const float2 *, float2 *, const __nv_bfloat16 *, long long, int, int, long long, long long, const EpiDot &, const int *, int *, cudaStream_t);
template int launch_modeprod_tc<float2, double2>(const float2 *, double2 *, const __nv_bfloat16 *, long long, int, int, long long, long long, const EpiDot &, const int *, int *, cudaStream_t);
template int launch_modeprod_tc<double2, double2>(const double2 *, double2 *, const __nv_bfloat16 *, long long, int, int, long long, long long, const EpiDot &, const int *, int *, cudaStream_t);
