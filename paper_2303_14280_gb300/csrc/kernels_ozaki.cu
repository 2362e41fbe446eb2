// Split-product tensor-core GEMMs of the mixed form (SNK_GEMM_SPLIT) on sm_103a (tcgen05):
// F_j = X_j P (Eq. batch_local_exx) and Kt += G_j^T X_j (Eq. usym_k).
//
// Every FP64 operand is cut into bf16 slices on a fixed-point grid (an
// Ozaki-style split): for each row and each run of kOzChunk = 256 reduction
// indices, with 2^e > max |x| over the run,
//     x = sum_s q_s 2^(e - 8(s+1)),  q_0 in [-256, 256], q_s in [-128, 128],
// so every slice value is an integer times a power of two that bf16 holds
// exactly.  A product of two slices is an integer times 2^(e_a + e_b - 8(i+j+2))
// below 2^16 of that unit, and a run of 256 such products with the same i + j
// stays below 2^24 units: the tensor core's FP32 accumulation of
//     level 0: A_0 B_0,   level 1: A_0 B_1 + A_1 B_0
// is exact over a run.  The remaining products (i + j >= 2, 2^-16 smaller)
// share a third accumulator whose FP32 rounding is far below the truncation.
// After each run the epilogue warps read the accumulators from tensor memory
// and add them into double-FP32 (hi + lo float) running sums; the result is
// the sum over all runs.  Five slices (15 products) give ~2^-40 of the row and
// column maxima of a run; three slices (6 products, level 1 and 2 in one
// accumulator) give ~2^-24.
//
// The split kernel writes each operand pre-tiled: blocks of 128 rows x 32
// reduction indices, one 8 KB block per slice, slices of a block adjacent, in
// the no-swizzle K-major core-matrix layout the tcgen05 shared-memory
// descriptors read (8 rows x 16 bytes per core matrix, 128 B apart along K,
// 512 B apart along the rows).  The GEMM kernel therefore moves operands with
// plain bulk copies (cp.async.bulk) into a ring of shared-memory stages; one
// elected thread issues tcgen05.mma (M = N = 128, K = 16, bf16 in, FP32 out)
// into tensor memory; eight epilogue warps drain it.  Every wait on an
// mbarrier is bounded in time; a kernel that gives up records the error,
// releases its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "async_copy.cuh"
#include "snk_internal.h"

namespace snk {

namespace {

constexpr int kOzRows = 128;      // rows per operand block (M and N of the MMA)
constexpr int kOzKt = 32;         // reduction indices per block
constexpr int kOzChunk = 256;     // reduction indices per exact accumulation run
constexpr int kOzKtPerChunk = kOzChunk / kOzKt;
constexpr int kOzBlockBytes = kOzRows * kOzKt * 2;  // one slice of one block: 8 KB
constexpr int kOzThreads = 320;   // warp 0 copies, warp 1 issues MMAs, warps 2..9 drain
constexpr int kOzEpiWarps = 8;
constexpr unsigned long long kOzWaitNs = 2000000000ull;  // 2 s per wait, then give up

// byte offset of element (r, k) inside one 128 x 32 bf16 slice block
__host__ __device__ __forceinline__ int oz_elem_offset(int r, int k) {
  return (r & 7) * 16 + (k & 7) * 2 + (k >> 3) * 128 + (r >> 3) * 512;
}

// ---------------------------------------------------------------- split
//
// All of the slicing runs in integer and FP32 arithmetic (FP64 issues at 1/64
// of the FP32 rate on GB300): the run maximum is taken on the IEEE bit
// patterns, and each value becomes the integer N = round(x 2^(T - e)),
// T = 8 S, |N| <= 2^T, read off its significand and exponent with shifts,
// whose balanced base-256 digits are the slices.

__device__ __forceinline__ double oz_load(const OzSplitJob& j, const double* __restrict__ ws,
                                          const double* __restrict__ P, const int* __restrict__ xfunc,
                                          const int* __restrict__ sfunc, int r, int k) {
  if (r >= j.R || k >= j.K) return 0.0;
  switch (j.mode) {
    case 0: return ws[j.src_off + (int64_t)k * j.ld + r];
    case 1: return ws[j.src_off + (int64_t)(r + j.r0) * j.ld + k];
    default: return P[j.src_off + (int64_t)sfunc[j.sf_off + j.r0 + r] * j.ld + xfunc[j.xf_off + k]];
  }
}

__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// e with max < 2^e from the bit pattern of a run's largest |x| (frexp's
// exponent); 0 for runs below 2^-600, whose slices are then all zero
__device__ __forceinline__ int oz_run_exponent(unsigned long long maxbits) {
  const int ex = (int)(maxbits >> 52);
  return ex >= 1023 - 600 ? ex - 1022 : 0;
}

// N = round(x 2^(T - e)) for |x| < 2^e (zero and subnormal x give 0)
__device__ __forceinline__ long long oz_fixed(double x, int e, int T) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0) return 0;
  const long long m = (long long)((b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);  // x = +-m 2^(ex - 1075)
  const int sh = 1075 + e - T - ex;  // > 4 whenever |x| < 2^e and T <= 48
  if (sh > 60) return 0;
  const long long n = sh > 0 ? (m + (1ll << (sh - 1))) >> sh : m << (-sh);
  return (b >> 63) ? -n : n;
}

// the S slices of 8 values with the run exponent e, as bf16, stored 16 bytes
// per slice at dst (one core-matrix row of each slice block)
__device__ __forceinline__ void oz_emit8(const double* x, int e, int S, uint8_t* dst) {
  const int T = 8 * S;
  long long r[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) r[q] = oz_fixed(x[q], e, T);
  for (int s = 0; s < S; ++s) {
    const int k = T - 8 * (s + 1);
    // the slice's weight 2^(e - 8(s+1)) as a float, built from its exponent
    // bits while it is a normal number (ldexpf only below that)
    const int pw = e - 8 * (s + 1);
    const bool normal = pw >= -126 && pw <= 127;
    const float scale = normal ? __int_as_float((pw + 127) << 23) : 0.f;
    __align__(16) __nv_bfloat16 v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      long long d;
      if (k > 0) {
        d = (r[q] + (1ll << (k - 1))) >> k;  // nearest digit (ties up), |d| <= 256
        r[q] -= d * (1ll << k);
      } else {
        d = r[q];
      }
      const float fd = (float)(int)d;  // exact: |d| <= 256
      v[q] = __float2bfloat16_rn(normal ? fd * scale : ldexpf(fd, pw));  // exact: a power-of-two scaling
    }
    *reinterpret_cast<uint4*>(dst + (int64_t)s * kOzBlockBytes) = *reinterpret_cast<const uint4*>(v);
  }
}

__device__ __forceinline__ bool oz_job_fits(const OzSplitJob& j, int64_t arena_bytes, int* err) {
  const int RT = (j.R + kOzRows - 1) / kOzRows, KT = (j.K + kOzKt - 1) / kOzKt;
  if (j.dst_off < 0 || j.dst_off + (int64_t)RT * KT * j.S * kOzBlockBytes > arena_bytes || j.S > 6) {
    atomicExch(err, 2);
    return false;
  }
  return true;
}

// Column-major sources (mode 0): one CTA per (job, row block, run of 256);
// the run's row maxima first (threads along the rows, coalesced), then the
// slices of (row, 8 reduction indices) items.
__global__ void __launch_bounds__(256) oz_split_cols_kernel(const OzSplitJob* __restrict__ jobs,
                                                            const double* __restrict__ ws,
                                                            uint8_t* __restrict__ arena, int64_t arena_bytes,
                                                            int* __restrict__ err) {
  const OzSplitJob j = jobs[blockIdx.z];
  if (j.mode != 0) return;
  const int rt = blockIdx.x, c = blockIdx.y;
  const int RT = (j.R + kOzRows - 1) / kOzRows, KT = (j.K + kOzKt - 1) / kOzKt;
  if (rt >= RT || c * kOzKtPerChunk >= KT) return;
  if (!oz_job_fits(j, arena_bytes, err)) return;
  __shared__ unsigned long long part[2][kOzRows];
  __shared__ int rexp[kOzRows];
  const int t = threadIdx.x;
  const int k_begin = c * kOzChunk;
  const int r = t & (kOzRows - 1);
  const int grow = rt * kOzRows + r;
  {
    const int h = t >> 7;
    unsigned long long m = 0;
    const int k0 = k_begin + h * (kOzChunk / 2), k1 = min(k0 + kOzChunk / 2, j.K);
    if (grow < j.R)
      for (int k = k0; k < k1; ++k) {
        const unsigned long long b = abs_bits(ws[j.src_off + (int64_t)k * j.ld + grow]);
        m = b > m ? b : m;
      }
    part[h][r] = m;
  }
  __syncthreads();
  if (t < kOzRows) rexp[t] = oz_run_exponent(part[0][t] > part[1][t] ? part[0][t] : part[1][t]);
  __syncthreads();
  for (int g = t >> 7; g < kOzChunk / 8; g += 2) {  // 128 rows x 32 groups of 8 reduction indices
    const int k = k_begin + g * 8;
    if (k >= KT * kOzKt) break;
    double x[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      x[q] = (grow < j.R && k + q < j.K) ? ws[j.src_off + (int64_t)(k + q) * j.ld + grow] : 0.0;
    const int kt = k / kOzKt;
    oz_emit8(x, rexp[r], j.S,
             arena + j.dst_off + ((int64_t)rt * KT + kt) * j.S * kOzBlockBytes + oz_elem_offset(r, k % kOzKt));
  }
}

// Row-major and gathered sources (modes 1, 2): one warp per (row, run of
// 256); each lane loads 8 consecutive reduction indices, the warp reduces the
// run maximum with shuffles, and the lane writes its 8 values' slices.
__global__ void __launch_bounds__(256) oz_split_rows_kernel(const OzSplitJob* __restrict__ jobs,
                                                            const double* __restrict__ ws,
                                                            const double* __restrict__ P,
                                                            const int* __restrict__ xfunc,
                                                            const int* __restrict__ sfunc,
                                                            uint8_t* __restrict__ arena, int64_t arena_bytes,
                                                            int* __restrict__ err) {
  const OzSplitJob j = jobs[blockIdx.z];
  if (j.mode == 0) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int RT = (j.R + kOzRows - 1) / kOzRows, KT = (j.K + kOzKt - 1) / kOzKt;
  const int r = blockIdx.x * 8 + warp, c = blockIdx.y;  // row inside the padded operand
  if (r >= RT * kOzRows || c * kOzKtPerChunk >= KT) return;
  if (!oz_job_fits(j, arena_bytes, err)) return;
  const int k = c * kOzChunk + lane * 8;
  double x[8];
  unsigned long long m = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    x[q] = oz_load(j, ws, P, xfunc, sfunc, r, k + q);
    const unsigned long long b = abs_bits(x[q]);
    m = b > m ? b : m;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
    m = v > m ? v : m;
  }
  if (k >= KT * kOzKt) return;
  const int kt = k / kOzKt;
  oz_emit8(x, oz_run_exponent(m), j.S,
           arena + j.dst_off + ((int64_t)(r / kOzRows) * KT + kt) * j.S * kOzBlockBytes +
               oz_elem_offset(r % kOzRows, k % kOzKt));
}

// ---------------------------------------------------------------- PTX helpers

__device__ __forceinline__ bool oz_wait(uint64_t* bar, uint32_t parity, int* err) {
  return mbar_wait(bar, parity, err, kOzWaitNs);
}

// shared-memory matrix descriptor: no swizzle, K-major, core matrices 128 B
// apart along K (leading byte offset) and 512 B apart along M / N (stride)
__device__ __forceinline__ uint64_t oz_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)(128u >> 4) << 16;
  d |= (uint64_t)(512u >> 4) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of sm_100 and later
  return d;                // base offset 0, layout type 0 (no swizzle)
}

// instruction descriptor of kind::f16: bf16 A and B (K-major), FP32 D, M = N = 128
constexpr uint32_t kOzIdesc = (1u << 4)            // D format FP32
                              | (1u << 7)          // A format bf16
                              | (1u << 10)         // B format bf16
                              | ((128u >> 3) << 17)  // N / 8
                              | ((128u >> 4) << 24); // M / 16

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kOzIdesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 8 consecutive FP32 columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float* v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
               "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
               "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
               "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
               : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// ---------------------------------------------------------------- double-FP32 sums

// (hi, lo) += a + b + c where a + b is formed exactly (TwoSum) and c is small
__device__ __forceinline__ void ds_acc3(float& hi, float& lo, float a, float b, float c) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  // (hi, lo) + (s, e + c)
  float t = __fadd_rn(hi, s);
  float z = __fsub_rn(t, hi);
  float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, z)), __fsub_rn(s, z));
  float l = __fadd_rn(__fadd_rn(lo, err), __fadd_rn(e, c));
  hi = __fadd_rn(t, l);
  lo = __fsub_rn(l, __fsub_rn(hi, t));
}

// ---------------------------------------------------------------- GEMM

// S slices used per operand: 5 (15 products, 3 accumulators: level 0,
// level 1, the rest; one tensor-memory buffer; the running sums are
// double-FP32 with hi in the last 128 columns of tensor memory and lo in the
// epilogue's registers) or 3 (6 products, 2 accumulators: level 0, the rest;
// two buffers so that the epilogue of a run overlaps the next run's products;
// FP32 running sums in registers).
template <int S>
struct OzCfg {
  static constexpr int kAcc = S >= 5 ? 3 : 2;
  static constexpr int kBufs = S >= 5 ? 1 : 2;
  static constexpr int kStageBytes = 2 * S * kOzBlockBytes;
  static constexpr int kStages = (200 * 1024) / kStageBytes < 8 ? (200 * 1024) / kStageBytes : 8;
};

struct OzShared {
  uint64_t full[8], empty[8], tfull[2], tempty[2];
  uint32_t tmem_base;
};

template <int S>
__global__ void __launch_bounds__(kOzThreads, 1) oz_gemm_kernel(OzGemmArgs a) {
  using C = OzCfg<S>;
  extern __shared__ __align__(1024) uint8_t oz_smem[];
  uint8_t* stages = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(oz_smem) + 1023) & ~uintptr_t(1023));
  OzShared* sh = reinterpret_cast<OzShared*>(stages + C::kStages * C::kStageBytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(&sh->full[s], 1);
      mbar_init(&sh->empty[s], 1);
    }
    for (int b = 0; b < C::kBufs; ++b) {
      mbar_init(&sh->tfull[b], 1);
      mbar_init(&sh->tempty[b], kOzEpiWarps);
    }
    mbar_init_fence();
  }
  if (warp == 1) {  // the whole warp allocates all 512 columns of tensor memory
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&sh->tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh->tmem_base;
  const int ntiles = a.n_tiles;

  // tile t -> job (jobs sorted by first tile) and (mt, nt) inside it
  auto locate = [&](int t, int& jb, int& mt, int& nt) {
    int lo = 0, hi = a.n_jobs - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.jobs[mid].tile0 <= t)
        lo = mid;
      else
        hi = mid - 1;
    }
    jb = lo;
    const int u = t - a.jobs[lo].tile0;
    mt = u / a.jobs[lo].RTb;
    nt = u - mt * a.jobs[lo].RTb;
  };

  if (warp == 0) {
    // ---------------- producer: one elected lane streams the operand blocks
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      int issued[8] = {-1, -1, -1, -1, -1, -1, -1, -1};  // parity of the last phase issued per stage
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        int jb, mt, nt;
        locate(t, jb, mt, nt);
        const OzGemmJob& J = a.jobs[jb];
        const int64_t ao = J.a_off + (int64_t)mt * J.KT * J.Sa * kOzBlockBytes;
        const int64_t bo = J.b_off + (int64_t)nt * J.KT * J.Sb * kOzBlockBytes;
        // every block this tile reads must lie inside the arena (checked on the host too)
        if (ao < 0 || bo < 0 || ao + (int64_t)J.KT * J.Sa * kOzBlockBytes > a.arena_bytes ||
            bo + (int64_t)J.KT * J.Sb * kOzBlockBytes > a.arena_bytes || J.Sa < S || J.Sb < S) {
          atomicExch(a.err, 2);
          ok = false;
          break;
        }
        const uint8_t* Ab = a.arena + ao;
        const uint8_t* Bb = a.arena + bo;
        for (int kt = 0; kt < J.KT && ok; ++kt) {
          if (!oz_wait(&sh->empty[stage], phase ^ 1, a.err)) {
            ok = false;
            break;
          }
          uint8_t* st = stages + stage * C::kStageBytes;
          mbar_expect_tx(&sh->full[stage], 2 * S * kOzBlockBytes);
          bulk_copy(st, Ab + (int64_t)kt * J.Sa * kOzBlockBytes, S * kOzBlockBytes, &sh->full[stage]);
          bulk_copy(st + S * kOzBlockBytes, Bb + (int64_t)kt * J.Sb * kOzBlockBytes, S * kOzBlockBytes,
                    &sh->full[stage]);
          issued[stage] = (int)phase;
          if (++stage == C::kStages) {
            stage = 0;
            phase ^= 1;
          }
        }
      }
      if (!ok) {  // let the copies already in flight land before the CTA exits
        for (int s = 0; s < C::kStages; ++s)
          if (issued[s] >= 0) {
            const unsigned long long t0 = global_ns();
            while (!mbar_try(&sh->full[s], (uint32_t)issued[s]) && global_ns() - t0 < kOzWaitNs) {
            }
          }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: one elected lane
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int buf = 0;
      uint32_t tphase = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        int jb, mt, nt;
        locate(t, jb, mt, nt);
        const int KT = a.jobs[jb].KT;
        for (int c0 = 0; c0 < KT && ok; c0 += kOzKtPerChunk) {
          // the epilogue must have drained this buffer
          if (!oz_wait(&sh->tempty[buf], tphase ^ 1, a.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dbase = tmem + (uint32_t)(buf * C::kAcc * kOzRows);
          bool first[3] = {true, true, true};
          for (int kt = c0; kt < min(KT, c0 + kOzKtPerChunk) && ok; ++kt) {
            if (!oz_wait(&sh->full[stage], phase, a.err)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(stages + stage * C::kStageBytes);
            const uint32_t sb = sa + S * kOzBlockBytes;
#pragma unroll
            for (int i = 0; i < S; ++i)
#pragma unroll
              for (int jj = 0; jj < S; ++jj) {
                if (i + jj >= S) continue;
                const int lvl = (i + jj) < C::kAcc - 1 ? (i + jj) : C::kAcc - 1;
                const uint32_t d = dbase + (uint32_t)(lvl * kOzRows);
#pragma unroll
                for (int ks = 0; ks < kOzKt / 16; ++ks) {
                  const uint64_t ad = oz_desc(sa + i * kOzBlockBytes + ks * 256);
                  const uint64_t bd = oz_desc(sb + jj * kOzBlockBytes + ks * 256);
                  mma_bf16(d, ad, bd, first[lvl] ? 0u : 1u);
                  first[lvl] = false;
                }
              }
            mma_commit(&sh->empty[stage]);  // the stage is free once these products are done
            if (++stage == C::kStages) {
              stage = 0;
              phase ^= 1;
            }
          }
          mma_commit(&sh->tfull[buf]);  // the run's accumulators are complete
          if (++buf == C::kBufs) {
            buf = 0;
            tphase ^= 1;
          }
        }
      }
    }
  } else {
    // ---------------- epilogue: warps 2..9; lane quarter = warp % 4, column half = (warp - 2) / 4
    const int q = warp & 3, half = (warp - 2) >> 2;
    const int row = q * 32 + lane;  // tile row held by this thread
    const int col0 = half * 64;
    int buf = 0;
    uint32_t tphase = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      int jb, mt, nt;
      locate(t, jb, mt, nt);
      const OzGemmJob& J = a.jobs[jb];
      // running sums of this thread's 64 columns: FP32 (S = 3), or double-FP32 with
      // hi in tensor memory columns [384, 512) and lo here (S = 5)
      float acc[64];
#pragma unroll
      for (int c = 0; c < 64; ++c) acc[c] = 0.f;
      const uint32_t thi = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(3 * kOzRows + col0);
      bool first_run = true;
      for (int c0 = 0; c0 < J.KT && ok; c0 += kOzKtPerChunk) {
        ok = __all_sync(0xffffffffu, oz_wait(&sh->tfull[buf], tphase, a.err));
        if (!ok) break;
        tc_fence_after();
        const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * C::kAcc * kOzRows + col0);
#pragma unroll
        for (int g = 0; g < 8; ++g) {
          float v0[8], v1[8];
          tmem_ld8(tb + g * 8, v0);
          tmem_ld8(tb + kOzRows + g * 8, v1);
          if (C::kAcc == 3) {
            float v2[8], h[8];
            tmem_ld8(tb + 2 * kOzRows + g * 8, v2);
            if (first_run) {
#pragma unroll
              for (int c = 0; c < 8; ++c) h[c] = 0.f;
            } else {
              tmem_ld8(thi + g * 8, h);
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) ds_acc3(h[c], acc[g * 8 + c], v0[c], v1[c], v2[c]);
            tmem_st8(thi + g * 8, h);
          } else {
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[g * 8 + c] += v0[c] + v1[c];
          }
        }
        first_run = false;
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh->tempty[buf]);
        if (++buf == C::kBufs) {
          buf = 0;
          tphase ^= 1;
        }
      }
      if (!ok) break;
      // the tile's sums as doubles (hi + lo for S = 5)
      double res[64];
      if (C::kAcc == 3) {
#pragma unroll
        for (int g = 0; g < 8; ++g) {
          float h[8];
          if (first_run) {
#pragma unroll
            for (int c = 0; c < 8; ++c) h[c] = 0.f;
          } else {
            tmem_ld8(thi + g * 8, h);
          }
#pragma unroll
          for (int c = 0; c < 8; ++c) res[g * 8 + c] = (double)h[c] + (double)acc[g * 8 + c];
        }
      } else {
#pragma unroll
        for (int c = 0; c < 64; ++c) res[c] = (double)acc[c];
      }
      // the tile's result: rows m = mt * 128 + row of A, columns n = nt * 128 + col of B
      const int m = mt * kOzRows + row;
      if (m >= J.m_lim) continue;
      if (J.kind == 2) {
        // plain C[m][n], row-major with leading dimension ldc (test export)
#pragma unroll
        for (int c = 0; c < 64; ++c) {
          const int n = nt * kOzRows + col0 + c;
          if (n < J.n_lim) a.ws[J.out_off + (int64_t)m * J.ldc + n] = res[c];
        }
      } else if (J.kind == 3) {
        // plain C stored column-major (point fastest): the F = X P of the
        // exchange-correlation potential
        const BatchDesc& bd = a.batches[J.batch];
        double* F = a.ws + J.out_off;
#pragma unroll
        for (int c = 0; c < 64; ++c) {
          const int n = nt * kOzRows + col0 + c;
          if (n < J.n_lim) F[(int64_t)(J.c0 + n) * bd.ldq + m] = res[c];
        }
      } else if (J.kind == 0) {
        const BatchDesc& bd = a.batches[J.batch];
        // F-hat_{n m} = w_m f_n sum_k X_{m k} P_{k n}, stored column-major (point fastest)
        const double wm = m < bd.q ? a.w[bd.p0 + m] : 0.0;
        double* F = a.ws + J.out_off;
        float* F32 = a.ws32 ? a.ws32 + J.out_off32 : nullptr;
        const int* sf = a.sfunc + bd.sfunc_off;
        const double* fc = a.fcomp + bd.mf0;
#pragma unroll
        for (int c = 0; c < 64; ++c) {
          const int n = nt * kOzRows + col0 + c;
          if (n < J.n_lim) {
            const int ng = J.c0 + n;
            const double v = wm * fc[sf[ng]] * res[c];
            F[(int64_t)ng * bd.ldq + m] = v;
            if (F32) F32[(int64_t)ng * bd.ldq + m] = (float)v;
          }
        }
      } else {
        const BatchDesc& bd = a.batches[J.batch];
        // Kt_{s nu} += sum_i G-hat_{s i} X_{nu i}, scattered into the molecule's block
        const int* sf = a.sfunc + bd.sfunc_off;
        const int* xf = a.xfunc + bd.xfunc_off;
        unsigned long long* Km = a.Khat + 2 * J.out_off;
        const int64_t rowoff = (int64_t)sf[J.c0 + m] * bd.nfm;
#pragma unroll
        for (int c = 0; c < 64; ++c) {
          const int n = nt * kOzRows + col0 + c;
          if (n < J.n_lim) khat_add(&Km[2 * (rowoff + xf[n])], res[c], a.err);
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

template <int S>
size_t oz_smem_bytes() {
  return (size_t)OzCfg<S>::kStages * OzCfg<S>::kStageBytes + sizeof(OzShared) + 1024;
}

}  // namespace

int64_t oz_operand_bytes(int rows, int k, int slices) {
  const int64_t RT = (rows + kOzRows - 1) / kOzRows, KT = (k + kOzKt - 1) / kOzKt;
  return RT * KT * slices * kOzBlockBytes;
}

int oz_row_tiles(int rows) { return (rows + kOzRows - 1) / kOzRows; }

int oz_k_tiles(int k) { return (k + kOzKt - 1) / kOzKt; }

cudaError_t launch_oz_split(cudaStream_t st, const OzSplitJob* jobs, int n_jobs, int max_rows, int max_k,
                            const double* ws, const double* P, const int* xfunc, const int* sfunc, uint8_t* arena,
                            int64_t arena_bytes, int* err) {
  if (n_jobs == 0 || max_rows == 0 || max_k == 0) return cudaSuccess;
  const int row_tiles = (max_rows + kOzRows - 1) / kOzRows, runs = (max_k + kOzChunk - 1) / kOzChunk;
  // each kernel takes the jobs of its kind and returns at once for the others
  oz_split_cols_kernel<<<dim3(row_tiles, runs, n_jobs), 256, 0, st>>>(jobs, ws, arena, arena_bytes, err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  oz_split_rows_kernel<<<dim3(row_tiles * (kOzRows / 8), runs, n_jobs), 256, 0, st>>>(jobs, ws, P, xfunc, sfunc,
                                                                                        arena, arena_bytes, err);
  return cudaGetLastError();
}

template <int S>
cudaError_t launch_oz_gemm_s(cudaStream_t st, const OzGemmArgs& args, int grid) {
  const size_t smem = oz_smem_bytes<S>();
  cudaError_t e = cudaFuncSetAttribute(oz_gemm_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  oz_gemm_kernel<S><<<grid, kOzThreads, smem, st>>>(args);
  return cudaGetLastError();
}

cudaError_t launch_oz_gemm(cudaStream_t st, int slices, const OzGemmArgs& args, int num_sms) {
  if (args.n_tiles == 0) return cudaSuccess;
  const int grid = std::min(args.n_tiles, num_sms);
  switch (slices) {
    case 3: return launch_oz_gemm_s<3>(st, args, grid);
    case 4: return launch_oz_gemm_s<4>(st, args, grid);
    case 5: return launch_oz_gemm_s<5>(st, args, grid);
    case 6: return launch_oz_gemm_s<6>(st, args, grid);
    default: return cudaErrorInvalidValue;
  }
}

// The failure path of the bounded waits: an mbarrier expecting one arrival
// that never comes; the wait gives up after limit_ns and sets *err.
__global__ void wait_probe_kernel(int* err, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  mbar_init(&bar, 1);
  mbar_init_fence();
  mbar_wait(&bar, 0, err, limit_ns);
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&bar)) : "memory");
}

cudaError_t launch_wait_probe(cudaStream_t st, int* err, unsigned long long limit_ns) {
  wait_probe_kernel<<<1, 1, 0, st>>>(err, limit_ns);
  return cudaGetLastError();
}

}  // namespace snk
