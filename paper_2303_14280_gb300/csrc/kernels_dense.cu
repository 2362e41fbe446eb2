// Dense and screening kernels of libsnk (sm_103a):
//   collocation X_j (Eq. collocation), the geometry-only batch maxima of
//   Eq. (exx_fmat_approx), F-tilde = |P| Phi-tilde (Eq. exx_fmat_approx) as
//   a GEMM over batches, the sn-LinK pair screen with per-batch compaction
//   (Eq. sp_set), the integral tiles, the products F_j = X_j P (Eq.
//   batch_local_exx) and Kt += G_j^T X_j (Eq. usym_k) as FP64 or
//   double-FP32 tiles (one F / G block per density; the tensor-core split
//   products are in kernels_ozaki.cu), and the symmetrisation of Eq. (sn_k).
//
// Several molecules can share one handle: every batch knows its molecule, P
// and K are packed per molecule (row-major N_b,m^2 blocks), and column lists
// hold molecule-local function indices.
//
// FP64 on GB300 issues at 2 DFMA per SM per clock, so a 64 x 64 x 16 tile
// step is ~32k cycles of DFMA against 2k doubles of shared-memory staging:
// the FP64 GEMMs are FP64-pipe bound with plain shared-memory tiling.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "ds_arith.cuh"
#include "snk_internal.h"

namespace snk {

namespace {

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  // for non-negative doubles the IEEE bit pattern orders like the value
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// molecule of a packed-block element (the blocks are in pk_off order)
__device__ __forceinline__ int mol_of_packed(const MolDesc* mols, int n_mol, int64_t e) {
  int lo = 0, hi = n_mol - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (mols[mid].pk_off <= e)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------- FP64 GEMM tile

constexpr int TM = 64, TN = 64, TK = 16, GEMM_THREADS = 256;

// C[m][n] = sum_k A(m,k) B(k,n) for the 64 x 64 tile at (m0, n0), K = kdim.
// la(m, k), lb(k, n) return 0 outside the operands; st(m, n, c) stores.
template <class T = double, class LA, class LB, class ST>
__device__ __forceinline__ void gemm_tile(int m0, int n0, int mdim, int ndim, int kdim, LA la, LB lb,
                                          ST st, bool a_k_fast, bool b_k_fast) {
  __shared__ T As[TK][TM + 1];
  __shared__ T Bs[TK][TN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  for (int k0 = 0; k0 < kdim; k0 += TK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int e = tid + r * GEMM_THREADS;  // 0..1023
      int kk, mm;
      if (a_k_fast) {
        kk = e % TK;
        mm = e / TK;
      } else {
        mm = e % TM;
        kk = e / TM;
      }
      int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < mdim && k < kdim) ? T(la(m, k)) : T(0);
      int nn;
      if (b_k_fast) {
        kk = e % TK;
        nn = e / TK;
      } else {
        nn = e % TN;
        kk = e / TN;
      }
      int n = n0 + nn;
      k = k0 + kk;
      Bs[kk][nn] = (n < ndim && k < kdim) ? T(lb(k, n)) : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = As[kk][ty + 16 * q];
        b[q] = Bs[kk][tx + 16 * q];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int m = m0 + ty + 16 * p, n = n0 + tx + 16 * q;
      if (m < mdim && n < ndim) st(m, n, acc[p][q]);
    }
}

// ---------------------------------------------------------------- double-FP32 tile (mixed form)

// Operands as unevaluated sums hi + lo of two floats (hi = fl32(v), lo =
// fl32(v - hi): 48 significant bits).  a b = ah bh + (ah bl + al bh) + al bl:
// ah bh is split exactly into p + e (e by an FMA), the al bl term (~2^-48
// relative) is dropped, and the running sum (s, c) adds p with Knuth's
// error-free TwoSum and everything else into the compensation c.  Twelve FP32
// operations per multiply-add on the FP32 pipe (64x the FP64 issue rate on
// GB300), relative error ~k 2^-46 for a length-k sum of same-sign terms.
__device__ __forceinline__ float2 df32_split(double v) {
  const float hi = __double2float_rn(v);
  return make_float2(hi, __double2float_rn(v - (double)hi));
}

__device__ __forceinline__ void df32_mac(float2 a, float2 b, float& s, float& c) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  const float t = __fadd_rn(s, p);
  const float z = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}

// C[m][n] = sum_k A(m,k) B(k,n) for the 64 x 64 tile at (m0, n0) with float2
// (hi, lo) operands; la(m, k), lb(k, n) return (0, 0) outside the operands.
template <class LA, class LB, class ST>
__device__ __forceinline__ void df32_tile(int m0, int n0, int mdim, int ndim, int kdim, LA la, LB lb, ST st,
                                          bool a_k_fast, bool b_k_fast) {
  __shared__ float2 As[TK][TM + 1];
  __shared__ float2 Bs[TK][TN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  float s[4][4], c[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) s[a][b] = c[a][b] = 0.f;
  const float2 zero = make_float2(0.f, 0.f);
  for (int k0 = 0; k0 < kdim; k0 += TK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + r * GEMM_THREADS;
      int kk, mm;
      if (a_k_fast) {
        kk = e % TK;
        mm = e / TK;
      } else {
        mm = e % TM;
        kk = e / TM;
      }
      int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < mdim && k < kdim) ? la(m, k) : zero;
      int nn;
      if (b_k_fast) {
        kk = e % TK;
        nn = e / TK;
      } else {
        nn = e % TN;
        kk = e / TN;
      }
      const int n = n0 + nn;
      k = k0 + kk;
      Bs[kk][nn] = (n < ndim && k < kdim) ? lb(k, n) : zero;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < TK; ++kk) {
      float2 a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = As[kk][ty + 16 * q];
        b[q] = Bs[kk][tx + 16 * q];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) df32_mac(a[p], b[q], s[p][q], c[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int m = m0 + ty + 16 * p, n = n0 + tx + 16 * q;
      if (m < mdim && n < ndim) st(m, n, (double)s[p][q] + (double)c[p][q]);
    }
}

// In place: every double of buf[0, n) becomes its (hi, lo) float pair.
__global__ void split_df32_kernel(double* __restrict__ buf, int64_t n) {
  float2* out = reinterpret_cast<float2*>(buf);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = df32_split(buf[e]);
}

// dst[e] = (hi, lo) of src[e].
__global__ void split_df32_copy_kernel(const double* __restrict__ src, int64_t n, float2* __restrict__ dst) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = df32_split(src[e]);
}

// ---------------------------------------------------------------- collocation

constexpr int COL_THREADS = 128, COL_SHELLS = 8;
constexpr double kColExpCut = 60.0;  // alpha r^2 beyond which a primitive is left out of X

__global__ void __launch_bounds__(COL_THREADS) collocation_kernel(const BatchDesc* __restrict__ batches,
                                                                  const int* __restrict__ bshell,
                                                                  const int* __restrict__ bshell_col,
                                                                  const double* __restrict__ xyz,
                                                                  DeviceBasis B, double* __restrict__ ws) {
  const BatchDesc bd = batches[blockIdx.z];
  const int i = blockIdx.x * COL_THREADS + threadIdx.x;
  const int t0 = blockIdx.y * COL_SHELLS;
  if (i >= bd.ldq || t0 >= bd.nBshell) return;
  const int t1 = min(t0 + COL_SHELLS, bd.nBshell);
  const bool valid = i < bd.q;
  double x = 0.0, y = 0.0, z = 0.0;
  if (valid) {
    x = xyz[3 * (bd.p0 + i)];
    y = xyz[3 * (bd.p0 + i) + 1];
    z = xyz[3 * (bd.p0 + i) + 2];
  }
  double* X = ws + bd.xoff;
  for (int t = t0; t < t1; ++t) {
    const int sh = bshell[bd.bshell_off + t];
    const int col = bshell_col[bd.bshell_off + t];
    const int l = B.l[sh];
    double* out = X + (int64_t)col * bd.ldq + i;
    if (!valid) {
      for (int c = 0; c < (l + 1) * (l + 2) / 2; ++c) out[(int64_t)c * bd.ldq] = 0.0;
      continue;
    }
    const double dx = x - B.center[3 * sh], dy = y - B.center[3 * sh + 1], dz = z - B.center[3 * sh + 2];
    const double r2 = dx * dx + dy * dy + dz * dz;
    double rad = 0.0;
    for (int k = B.poff[sh]; k < B.poff[sh] + B.nprim[sh]; ++k) {
      // e^{-60} ~ 9e-27: primitives that far out add nothing representable next to
      // the batch's other values, and skipping the FP64 exponential is the saving
      const double x = B.exps[k] * r2;
      if (x < kColExpCut) rad += B.d[k] * exp(-x);
    }
    const double* f = B.fcomp + B.foff[sh];
    if (l == 0) {
      out[0] = rad;
    } else if (l == 1) {
      out[0] = dx * rad;
      out[bd.ldq] = dy * rad;
      out[2 * (int64_t)bd.ldq] = dz * rad;
    } else {
      const int64_t L = bd.ldq;
      out[0] = f[0] * dx * dx * rad;
      out[L] = f[1] * dx * dy * rad;
      out[2 * L] = f[2] * dx * dz * rad;
      out[3 * L] = f[3] * dy * dy * rad;
      out[4 * L] = f[4] * dy * dz * rad;
      out[5 * L] = f[5] * dz * dz * rad;
    }
  }
}

// ---------------------------------------------------------------- geometry-only screen maxima

// Phi-tilde_nu^(j) = max_i |sqrt(w_i) Phi_{nu i}|, one thread per function.
__global__ void phit_f_kernel(const BatchDesc* __restrict__ batches, const double* __restrict__ ws,
                              const double* __restrict__ w, const int* __restrict__ xfunc,
                              double* __restrict__ phit_f) {
  const BatchDesc bd = batches[blockIdx.y];
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= bd.nB) return;
  const double* X = ws + bd.xoff + (int64_t)c * bd.ldq;
  double m = 0.0;
  for (int i = 0; i < bd.q; ++i) m = fmax(m, sqrt(fabs(w[bd.p0 + i])) * fabs(X[i]));
  phit_f[bd.phf_off + xfunc[bd.xfunc_off + c]] = m;
}

// phi-tilde^(j) = max_i sqrt(w_i) sum_{mu in B_j} |Phi_{mu i}|, one block per batch.
__global__ void phit_b_kernel(const BatchDesc* __restrict__ batches, const double* __restrict__ ws,
                              const double* __restrict__ w, double* __restrict__ phit_b) {
  const BatchDesc bd = batches[blockIdx.x];
  const double* X = ws + bd.xoff;
  double m = 0.0;
  for (int i = threadIdx.x; i < bd.q; i += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < bd.nB; ++c) s += fabs(X[(int64_t)c * bd.ldq + i]);
    m = fmax(m, sqrt(fabs(w[bd.p0 + i])) * s);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r = fmax(r, red[k]);
    phit_b[blockIdx.x] = r;
  }
}

// max_nu |Phi_{nu i}| at every point i of a batch (weight of a point in the
// bound sum_i |dG_u(i)| max_nu |Phi_{nu i}| >= |dKt_{u nu}| of the learned
// screen's labels); xm is indexed by the point's position in batch order.
__global__ void xmax_kernel(const BatchDesc* __restrict__ batches, const double* __restrict__ ws,
                            double* __restrict__ xm) {
  const BatchDesc bd = batches[blockIdx.x];
  const double* X = ws + bd.xoff;
  for (int i = threadIdx.x; i < bd.q; i += blockDim.x) {
    double m = 0.0;
    for (int c = 0; c < bd.nB; ++c) m = fmax(m, fabs(X[(int64_t)c * bd.ldq + i]));
    xm[bd.p0 + i] = m;
  }
}

// Tile screen sums: one block per (tile of 128 points, batch).  The points'
// max |X| first (integer max of the IEEE bit patterns: no FP64 arithmetic),
// then per F column the warp-reduced sum over the tile of |F32| max |X|; the
// row ends with the tile's bounding sphere (centre, radius), 4 floats.
__global__ void __launch_bounds__(256) tile_sums_kernel(const BatchDesc* __restrict__ batches,
                                                        const double* __restrict__ ws, const float* __restrict__ ws32,
                                                        const double* __restrict__ xyz, int n_dens,
                                                        float* __restrict__ tsum) {
  const BatchDesc bd = batches[blockIdx.y];
  const int tile = blockIdx.x, i0 = tile * kPointTile;
  if (i0 >= bd.q) return;
  __shared__ float xt[kPointTile];
  const double* X = ws + bd.xoff;
  for (int t = threadIdx.x; t < kPointTile; t += blockDim.x) {
    unsigned long long m = 0;
    if (i0 + t < bd.q)
      for (int c = 0; c < bd.nB; ++c) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(X[(int64_t)c * bd.ldq + i0 + t]) &
                                     0x7FFFFFFFFFFFFFFFull;
        m = b > m ? b : m;
      }
    xt[t] = (float)__longlong_as_double((long long)m);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* out = tsum + bd.ssoff + (int64_t)tile * (bd.nS + 4);
  if (warp == 0) {  // bounding sphere of the tile: box centre, largest distance
    const int n = min(kPointTile, bd.q - i0);
    float mn[3] = {3e38f, 3e38f, 3e38f}, mx[3] = {-3e38f, -3e38f, -3e38f};
    for (int t = lane; t < n; t += 32)
      for (int q = 0; q < 3; ++q) {
        const float v = (float)xyz[3 * (bd.p0 + i0 + t) + q];
        mn[q] = fminf(mn[q], v);
        mx[q] = fmaxf(mx[q], v);
      }
    float cen[3];
    for (int q = 0; q < 3; ++q) {
      for (int o = 16; o > 0; o >>= 1) {
        mn[q] = fminf(mn[q], __shfl_xor_sync(0xffffffffu, mn[q], o));
        mx[q] = fmaxf(mx[q], __shfl_xor_sync(0xffffffffu, mx[q], o));
      }
      cen[q] = 0.5f * (mn[q] + mx[q]);
    }
    float r2 = 0.f;
    for (int t = lane; t < n; t += 32) {
      float d2 = 0.f;
      for (int q = 0; q < 3; ++q) {
        const float dv = (float)xyz[3 * (bd.p0 + i0 + t) + q] - cen[q];
        d2 = fmaf(dv, dv, d2);
      }
      r2 = fmaxf(r2, d2);
    }
    for (int o = 16; o > 0; o >>= 1) r2 = fmaxf(r2, __shfl_xor_sync(0xffffffffu, r2, o));
    if (lane == 0) {
      out[bd.nS] = cen[0];
      out[bd.nS + 1] = cen[1];
      out[bd.nS + 2] = cen[2];
      out[bd.nS + 3] = sqrtf(r2) * 1.0001f + 1e-6f;  // covers the float rounding of the points
    }
  }
  const int64_t dstr = (int64_t)bd.ldq * bd.nS;
  for (int c = warp; c < bd.nS; c += blockDim.x / 32) {
    float s = 0.f;
    for (int d = 0; d < n_dens; ++d) {
      const float* F = ws32 + bd.foff32 + d * dstr + (int64_t)c * bd.ldq + i0;
#pragma unroll
      for (int q = 0; q < kPointTile / 32; ++q) s += fabsf(F[lane + 32 * q]) * xt[lane + 32 * q];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[c] = s;
  }
}

// ---------------------------------------------------------------- F-tilde

// For molecule blockIdx.z: F-tilde_a^(j) = max_{mu in a} sum_nu |P_{mu nu}|
// Phi-tilde_nu^(j) over its functions mu and batches j, a GEMM (FP32 tiles,
// rounded up: an upper bound) whose store takes the shell maximum.  The molecule's batch rows are consecutive (stride N_b,m
// in Phi-tilde, N_shell,m in F-tilde).
__global__ void __launch_bounds__(GEMM_THREADS) ftilde_kernel(const MolDesc* __restrict__ mols,
                                                              const BatchDesc* __restrict__ batches,
                                                              const double* __restrict__ P,
                                                              const double* __restrict__ phit_f,
                                                              const int* __restrict__ fshell,
                                                              double* __restrict__ ft_shell) {
  const MolDesc md = mols[blockIdx.z];
  const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
  if (m0 >= md.nf || n0 >= md.nb) return;
  const double* Pm = P + md.pk_off;
  const BatchDesc b0 = batches[md.mb0];
  const double* ph = phit_f + b0.phf_off;
  double* ft = ft_shell + b0.cm_off;
  // a screening estimate: FP32 sums of non-negative terms (relative error
  // below k 2^-24 <= 3e-4 for k <= 5,000 terms), rounded up by 1e-3
  gemm_tile<float>(
      m0, n0, md.nf, md.nb, md.nf, [&](int m, int k) { return (float)fabs(Pm[(int64_t)m * md.nf + k]); },
      [&](int k, int n) { return (float)ph[(int64_t)n * md.nf + k]; },
      [&](int m, int n, float c) {
        atomic_max_nonneg(&ft[(int64_t)n * md.ns + (fshell[md.mf0 + m] - md.ms0)], (double)c * (1.0 + 1e-3));
      },
      true, true);
}

// ---------------------------------------------------------------- sn-LinK pair screen

constexpr int SCR_THREADS = 256;

// Bound of max_{r in Q_j} |A_ab(r)| for batch j: the global bound A-tilde, or,
// when the batch's bounding sphere stays clear of the segment AB that holds
// every Gaussian product centre, the smaller total-charge / distance bound.
// In FP32 (the FP64 pipe issues at 1/64 of it) with the distance rounded down
// and the charge rounded up, so the result stays an upper bound.
__device__ __forceinline__ float batch_pair_bound(const ScreenArgs& a, int j, int p, const PairHdr& h) {
  const float bnd = (float)a.bound[p] * (1.0f + 1e-6f);
  if (!a.distance) return bnd;
  const double* A = a.shell_xyz + 3 * h.sa;
  const float vx = (float)-h.ABx, vy = (float)-h.ABy, vz = (float)-h.ABz;  // B - A
  const float wx = (float)(a.bcenter[3 * j] - A[0]), wy = (float)(a.bcenter[3 * j + 1] - A[1]),
              wz = (float)(a.bcenter[3 * j + 2] - A[2]);
  const float vv = vx * vx + vy * vy + vz * vz;
  float t = vv > 0.f ? (wx * vx + wy * vy + wz * vz) / vv : 0.f;
  t = fminf(fmaxf(t, 0.f), 1.f);
  const float dx = wx - t * vx, dy = wy - t * vy, dz = wz - t * vz;
  const float d = sqrtf(dx * dx + dy * dy + dz * dz) * (1.0f - 1e-5f) - (float)a.bradius[j] - 1e-5f;
  return d > 0.f ? fminf(bnd, (float)a.qbound[p] * (1.0f + 1e-6f) / d) : bnd;
}

// sn-LinK decision for pair p in batch j, Eq. (sp_set): -1 drop, else the
// list index class + kNumClasses * precision (precision 1 = FP32 integrals,
// for pairs whose estimate max(F_a, F_b) phi A stays below fp32_bound).  The
// estimates are formed in FP32 and rounded up by 1e-5 relative, so every pair
// an exact evaluation keeps is kept, and a pair at the FP32 / FP64 border goes
// to the FP64 tier.
__device__ __forceinline__ int classify_pair(const ScreenArgs& a, const BatchDesc& bd, int j, int p, int cls,
                                             const PairHdr& h) {
  if (a.screen == SNK_SCREEN_NONE) return cls;
  const double* ft = a.ft_shell + bd.cm_off;
  const float fa = (float)ft[h.sa - bd.ms0], fb = (float)ft[h.sb - bd.ms0];
  const float bnd = batch_pair_bound(a, j, p, h) * (1.0f + 1e-5f);
  const float eK = fmaxf(fa, fb) * (float)a.phit_b[j] * bnd;
  if (!((fa * fb * bnd >= (float)a.eps_E) || (eK >= (float)a.eps_K))) return -1;
  return (a.mixed && eK < (float)a.fp32_bound) ? cls + kNumClasses : cls;
}

// Pass 1: per (batch, list) pair counts and primitive-pair counts; marks the
// shells of every kept pair (their F / G columns).  One block per batch, the
// pairs of the batch's molecule only.
__global__ void __launch_bounds__(SCR_THREADS) pair_count_kernel(ScreenArgs a, int* __restrict__ counts,
                                                                 long long* __restrict__ ppcounts,
                                                                 unsigned char* __restrict__ sflag,
                                                                 int64_t hflag_off) {
  const int j = blockIdx.x;
  const BatchDesc bd = a.batches[j];
  const MolDesc md = a.mols[bd.mol];
  signed char* codes = a.codes + a.code_off[j];    // the decision for each pair of the molecule
  unsigned char* fl = sflag + bd.cm_off;           // shells of V_j
  unsigned char* hl = sflag + hflag_off + bd.cm_off;  // shells of V_j's FP64 (high-tier) pairs
  __shared__ int s_cnt[kNumLists];
  __shared__ unsigned long long s_pp[kNumLists];
  if (threadIdx.x < kNumLists) {
    s_cnt[threadIdx.x] = 0;
    s_pp[threadIdx.x] = 0ull;
  }
  __syncthreads();
  for (int c = 0; c < kNumClasses; ++c) {
    int n[2] = {0, 0};
    unsigned long long pp[2] = {0ull, 0ull};
    for (int p = md.cr[c] + threadIdx.x; p < md.cr[c + 1]; p += SCR_THREADS) {
      const PairHdr h = a.pairs[p];
      const int li = classify_pair(a, bd, j, p, c, h);
      codes[p - md.cr[0]] = (signed char)li;
      if (li >= 0) {
        fl[h.sa - bd.ms0] = 1;
        fl[h.sb - bd.ms0] = 1;
        const int prec = li >= kNumClasses;
        if (!prec) {
          hl[h.sa - bd.ms0] = 1;
          hl[h.sb - bd.ms0] = 1;
        }
        n[prec] += 1;
        pp[prec] += (unsigned long long)(prec ? h.pp_n32 : h.pp_n);
      }
    }
    for (int prec = 0; prec < 2; ++prec) {
      if (n[prec]) {
        atomicAdd(&s_cnt[c + kNumClasses * prec], n[prec]);
        atomicAdd(&s_pp[c + kNumClasses * prec], pp[prec]);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < kNumLists) {
    counts[j * kNumLists + threadIdx.x] = s_cnt[threadIdx.x];
    ppcounts[j * kNumLists + threadIdx.x] = (long long)s_pp[threadIdx.x];
  }
}

// Pass 2: deterministic compaction (pair order kept) into the per-(batch, list)
// ranges that the host sized from pass 1, from the decisions pass 1 stored.
__global__ void __launch_bounds__(SCR_THREADS) pair_write_kernel(ScreenArgs a, const int64_t* __restrict__ list_off,
                                                                 int* __restrict__ list) {
  const int j = blockIdx.x;
  const BatchDesc bd = a.batches[j];
  const MolDesc md = a.mols[bd.mol];
  __shared__ int warp_tot[2][SCR_THREADS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const signed char* codes = a.codes + a.code_off[j];
  for (int c = 0; c < kNumClasses; ++c) {
    int64_t out[2] = {list_off[j * kNumLists + c], list_off[j * kNumLists + c + kNumClasses]};
    for (int base = md.cr[c]; base < md.cr[c + 1]; base += SCR_THREADS) {
      const int p = base + threadIdx.x;
      int li = -1;
      if (p < md.cr[c + 1]) li = codes[p - md.cr[0]];
      const unsigned bal[2] = {__ballot_sync(0xffffffffu, li >= 0 && li < kNumClasses),
                               __ballot_sync(0xffffffffu, li >= kNumClasses)};
      if (lane == 0) {
        warp_tot[0][warp] = __popc(bal[0]);
        warp_tot[1][warp] = __popc(bal[1]);
      }
      __syncthreads();
      for (int prec = 0; prec < 2; ++prec) {
        int before = 0, total = 0;
        for (int q = 0; q < SCR_THREADS / 32; ++q) {
          before += q < warp ? warp_tot[prec][q] : 0;
          total += warp_tot[prec][q];
        }
        if (li >= 0 && (li >= kNumClasses) == (prec == 1))
          list[out[prec] + before + __popc(bal[prec] & ((1u << lane) - 1u))] = p;
        out[prec] += total;
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------- F_j = X_j P, Kt += G_j^T X_j

// F-hat_{s i} = w_i f_s sum_{nu in B_j} X_{nu i} P_{nu s}: the quadrature weight
// and the Cartesian component factor of the column are folded into F.  In the
// mixed form an FP32 copy is written for the FP32 pairs.
// MODE: 0 FP64, 2 double-FP32 on (hi, lo) operands
template <int MODE>
__global__ void __launch_bounds__(GEMM_THREADS, MODE >= 2 ? 2 : 3)
    fgemm_kernel(const BatchDesc* __restrict__ batches, const double* __restrict__ P, const float2* __restrict__ P2,
                 const int* __restrict__ xfunc, const int* __restrict__ sfunc, const double* __restrict__ fcomp,
                 const double* __restrict__ w, double* __restrict__ ws, float* __restrict__ ws32, int dens) {
  const BatchDesc bd = batches[blockIdx.z];
  const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
  if (m0 >= bd.ldq || n0 >= bd.nS) return;
  const int64_t dofs = (int64_t)dens * bd.ldq * bd.nS;  // density d's F / G block
  double* F = ws + bd.foff + dofs;
  float* F32 = ws32 ? ws32 + bd.foff32 + dofs : nullptr;
  const int* xf = xfunc + bd.xfunc_off;
  const int* sf = sfunc + bd.sfunc_off;
  const double* fc = fcomp + bd.mf0;
  auto st = [&](int m, int n, double c) {
    const double wi = m < bd.q ? w[bd.p0 + m] : 0.0;
    const double v = wi * fc[sf[n]] * c;
    F[(int64_t)n * bd.ldq + m] = v;
    if (F32) F32[(int64_t)n * bd.ldq + m] = (float)v;
  };
  if (MODE == 2) {
    const float2* X2 = reinterpret_cast<const float2*>(ws + bd.xoff);
    const float2* Pm2 = P2 + bd.pk_off;
    auto la = [&](int m, int k) { return X2[(int64_t)k * bd.ldq + m]; };
    auto lb = [&](int k, int n) { return Pm2[(int64_t)xf[k] * bd.nfm + sf[n]]; };
    df32_tile(m0, n0, bd.ldq, bd.nS, bd.nB, la, lb, st, false, false);
  } else {
    const double* X = ws + bd.xoff;
    const double* Pm = P + bd.pk_off;
    auto la = [&](int m, int k) { return X[(int64_t)k * bd.ldq + m]; };
    auto lb = [&](int k, int n) { return Pm[(int64_t)xf[k] * bd.nfm + sf[n]]; };
    gemm_tile(m0, n0, bd.ldq, bd.nS, bd.nB, la, lb, st, false, false);
  }
}

// Kt_{s nu} += sum_i G-hat_{s i} X_{nu i}, scattered into the molecule's block
// of the packed accumulator (several batches add to the same entries).
template <int MODE>
__global__ void __launch_bounds__(GEMM_THREADS, MODE >= 2 ? 2 : 3)
    kgemm_kernel(const BatchDesc* __restrict__ batches, const int* __restrict__ xfunc, const int* __restrict__ sfunc,
                 const double* __restrict__ ws, unsigned long long* __restrict__ Khat, int dens, int* err) {
  const BatchDesc bd = batches[blockIdx.z];
  const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
  if (m0 >= bd.nS || n0 >= bd.nB) return;
  const int64_t dofs = (int64_t)dens * bd.ldq * bd.nS;  // density d's G block
  const int* xf = xfunc + bd.xfunc_off;
  const int* sf = sfunc + bd.sfunc_off;
  unsigned long long* Km = Khat + 2 * bd.pk_off;
  auto st = [&](int m, int n, double c) { khat_add(&Km[2 * ((int64_t)sf[m] * bd.nfm + xf[n])], c, err); };
  if (MODE == 2) {
    const float2* X2 = reinterpret_cast<const float2*>(ws + bd.xoff);
    const float2* G2 = reinterpret_cast<const float2*>(ws + bd.goff) + dofs;
    auto la = [&](int m, int k) { return G2[(int64_t)m * bd.ldq + k]; };
    auto lb = [&](int k, int n) { return X2[(int64_t)n * bd.ldq + k]; };
    df32_tile(m0, n0, bd.nS, bd.nB, bd.q, la, lb, st, true, true);
  } else {
    const double* X = ws + bd.xoff;
    const double* G = ws + bd.goff + dofs;
    auto la = [&](int m, int k) { return G[(int64_t)m * bd.ldq + k]; };
    auto lb = [&](int k, int n) { return X[(int64_t)n * bd.ldq + k]; };
    gemm_tile(m0, n0, bd.nS, bd.nB, bd.q, la, lb, st, true, true);
  }
}

// Exchange-correlation products (Sec. II.C).  F_{i n} = sum_k X_{i k} P[B_j k, B_j n]
// (Eq. fmat, no weight) into the batch's F block; V-hat_{m n} += sum_i Z_{i m}
// X_{i n} (Eq. vxc_num) scattered into the fixed-point accumulator.  MODE 0
// FP64 tiles, MODE 2 double-FP32 tiles with the operands split as they are
// staged (the FP64 X stays intact for the point kernel).
template <int MODE>
__global__ void __launch_bounds__(GEMM_THREADS, MODE >= 2 ? 2 : 3)
    xc_fgemm_kernel(const BatchDesc* __restrict__ batches, const double* __restrict__ P,
                    const int* __restrict__ xfunc, double* __restrict__ ws) {
  const BatchDesc bd = batches[blockIdx.z];
  const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
  if (m0 >= bd.ldq || n0 >= bd.nB) return;
  const double* X = ws + bd.xoff;
  double* F = ws + bd.foff;
  const int* xf = xfunc + bd.xfunc_off;
  const double* Pm = P + bd.pk_off;
  auto st = [&](int m, int n, double c) { F[(int64_t)n * bd.ldq + m] = c; };
  if (MODE == 2) {
    auto la = [&](int m, int k) { return df32_split(X[(int64_t)k * bd.ldq + m]); };
    auto lb = [&](int k, int n) { return df32_split(Pm[(int64_t)xf[k] * bd.nfm + xf[n]]); };
    df32_tile(m0, n0, bd.ldq, bd.nB, bd.nB, la, lb, st, false, false);
  } else {
    auto la = [&](int m, int k) { return X[(int64_t)k * bd.ldq + m]; };
    auto lb = [&](int k, int n) { return Pm[(int64_t)xf[k] * bd.nfm + xf[n]]; };
    gemm_tile(m0, n0, bd.ldq, bd.nB, bd.nB, la, lb, st, false, false);
  }
}

template <int MODE>
__global__ void __launch_bounds__(GEMM_THREADS, MODE >= 2 ? 2 : 3)
    xc_vgemm_kernel(const BatchDesc* __restrict__ batches, const int* __restrict__ xfunc,
                    const double* __restrict__ ws, unsigned long long* __restrict__ Vhat, int* err) {
  const BatchDesc bd = batches[blockIdx.z];
  const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
  if (m0 >= bd.nB || n0 >= bd.nB) return;
  const double* X = ws + bd.xoff;
  const double* Z = ws + bd.foff;
  const int* xf = xfunc + bd.xfunc_off;
  unsigned long long* Vm = Vhat + 2 * bd.pk_off;
  auto st = [&](int m, int n, double c) { khat_add(&Vm[2 * ((int64_t)xf[m] * bd.nfm + xf[n])], c, err); };
  if (MODE == 2) {
    auto la = [&](int m, int k) { return df32_split(Z[(int64_t)m * bd.ldq + k]); };
    auto lb = [&](int k, int n) { return df32_split(X[(int64_t)n * bd.ldq + k]); };
    df32_tile(m0, n0, bd.nB, bd.nB, bd.q, la, lb, st, true, true);
  } else {
    auto la = [&](int m, int k) { return Z[(int64_t)m * bd.ldq + k]; };
    auto lb = [&](int k, int n) { return X[(int64_t)n * bd.ldq + k]; };
    gemm_tile(m0, n0, bd.nB, bd.nB, bd.q, la, lb, st, true, true);
  }
}

// Tiles of list k of batch j (one block per (batch, list)): one per slab of
// kPointTile points, each with the whole list, so that every G entry of the
// list's launch has a single writer (its point's thread) and its additions
// come in list order.
__global__ void gen_tiles_kernel(const BatchDesc* __restrict__ batches, const int* __restrict__ counts,
                                 const int64_t* __restrict__ list_off, const int64_t* __restrict__ tstart,
                                 Tile* __restrict__ tiles) {
  const int j = blockIdx.x, k = blockIdx.y;
  const int64_t e = (int64_t)j * kNumLists + k;
  const int n = counts[e];
  if (n == 0) return;
  const int q = batches[j].q;
  const int nslab = (q + kPointTile - 1) / kPointTile;
  const int base = (int)list_off[e];
  Tile* out = tiles + tstart[e];
  for (int u = threadIdx.x; u < nslab; u += blockDim.x) {
    Tile t;
    t.batch = j;
    t.k0 = base;
    t.k1 = base + n;
    t.i0 = u * kPointTile;
    out[u] = t;
  }
}

// out[e] = sum_d |P_d[e]|: the screen's single bound for several densities.
__global__ void abs_sum_kernel(const double* __restrict__ P, int n_dens, int64_t n, double* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int d = 0; d < n_dens; ++d) v += fabs(P[d * n + e]);
    out[e] = v;
  }
}

// K_{mu nu} = (f_mu Kt_{mu nu} + f_nu Kt_{nu mu}) / 2 in every molecule block,
// Eq. (sn_k); the row factor f_mu is the Cartesian component factor that the
// integral kernel leaves out.
__global__ void finish_kernel(const MolDesc* __restrict__ mols, int n_mol, int64_t packed,
                              const unsigned long long* __restrict__ Khat, const double* __restrict__ fcomp,
                              double* __restrict__ K) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < packed; e += (int64_t)gridDim.x * blockDim.x) {
    const MolDesc md = mols[mol_of_packed(mols, n_mol, e)];
    const int64_t le = e - md.pk_off;
    const int mu = (int)(le / md.nf), nu = (int)(le % md.nf);
    const double a = __dmul_rn(fcomp[md.mf0 + mu], khat_value(Khat + 2 * e));
    const double b = __dmul_rn(fcomp[md.mf0 + nu], khat_value(Khat + 2 * (md.pk_off + (int64_t)nu * md.nf + mu)));
    // explicit rounding of both products keeps K exactly symmetric (no FMA contraction)
    K[e] = 0.5 * __dadd_rn(a, b);
  }
}

// out2[0] = max |P - P^T|, out2[1] = max |P| over every molecule block (out2
// zeroed by the caller); a non-finite entry gives +inf.
__global__ void symcheck_kernel(const MolDesc* __restrict__ mols, int n_mol, int64_t packed,
                                const double* __restrict__ P, double* __restrict__ out2) {
  double a = 0.0, b = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < packed; e += (int64_t)gridDim.x * blockDim.x) {
    const MolDesc md = mols[mol_of_packed(mols, n_mol, e)];
    const int64_t le = e - md.pk_off;
    const int mu = (int)(le / md.nf), nu = (int)(le % md.nf);
    const double v = P[e];
    a = fmax(a, fabs(v - P[md.pk_off + (int64_t)nu * md.nf + mu]));
    b = fmax(b, fabs(v));
    if (!isfinite(v)) a = INFINITY;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(&out2[0], a);
    atomic_max_nonneg(&out2[1], b);
  }
}

}  // namespace

// ---------------------------------------------------------------- launchers

cudaError_t launch_collocation(cudaStream_t st, const BatchDesc* dbatch, int nbatch, int max_ldq, int max_nBshell,
                               const int* bshell, const int* bshell_col, const double* xyz, DeviceBasis basis,
                               double* ws) {
  if (nbatch == 0 || max_ldq == 0 || max_nBshell == 0) return cudaSuccess;
  dim3 grid((max_ldq + COL_THREADS - 1) / COL_THREADS, (max_nBshell + COL_SHELLS - 1) / COL_SHELLS, nbatch);
  collocation_kernel<<<grid, COL_THREADS, 0, st>>>(dbatch, bshell, bshell_col, xyz, basis, ws);
  return cudaGetLastError();
}

cudaError_t launch_screen_geom(cudaStream_t st, const BatchDesc* dbatch, int nbatch, int max_nB, const double* ws,
                               const double* w, const int* xfunc, double* phit_f, double* phit_b) {
  if (nbatch == 0) return cudaSuccess;
  if (max_nB > 0) {
    dim3 grid((max_nB + 127) / 128, nbatch);
    phit_f_kernel<<<grid, 128, 0, st>>>(dbatch, ws, w, xfunc, phit_f);
  }
  phit_b_kernel<<<nbatch, 256, 0, st>>>(dbatch, ws, w, phit_b);
  return cudaGetLastError();
}

cudaError_t launch_tile_sums(cudaStream_t st, const BatchDesc* dbatch, int nbatch, int max_tiles, const double* ws,
                             const float* ws32, const double* xyz, int n_dens, float* tsum) {
  if (nbatch == 0 || max_tiles == 0) return cudaSuccess;
  tile_sums_kernel<<<dim3(max_tiles, nbatch), 256, 0, st>>>(dbatch, ws, ws32, xyz, n_dens, tsum);
  return cudaGetLastError();
}

cudaError_t launch_xmax(cudaStream_t st, const BatchDesc* dbatch, int nbatch, const double* ws, double* xmax) {
  if (nbatch == 0) return cudaSuccess;
  xmax_kernel<<<nbatch, 256, 0, st>>>(dbatch, ws, xmax);
  return cudaGetLastError();
}

cudaError_t launch_ftilde(cudaStream_t st, const MolDesc* mols, int n_mol, int max_nf, int max_nb,
                          const BatchDesc* batches, const double* P, const double* phit_f, const int* fshell,
                          double* ft_shell) {
  if (n_mol == 0 || max_nf == 0 || max_nb == 0) return cudaSuccess;
  dim3 grid((max_nf + TM - 1) / TM, (max_nb + TN - 1) / TN, n_mol);
  ftilde_kernel<<<grid, GEMM_THREADS, 0, st>>>(mols, batches, P, phit_f, fshell, ft_shell);
  return cudaGetLastError();
}

cudaError_t launch_pair_count(cudaStream_t st, const ScreenArgs& a, int nbatch, int* counts, long long* ppcounts,
                              unsigned char* sflag, int64_t hflag_off) {
  if (nbatch == 0) return cudaSuccess;
  pair_count_kernel<<<nbatch, SCR_THREADS, 0, st>>>(a, counts, ppcounts, sflag, hflag_off);
  return cudaGetLastError();
}

cudaError_t launch_pair_write(cudaStream_t st, const ScreenArgs& a, int nbatch, const int64_t* list_off, int* list) {
  if (nbatch == 0) return cudaSuccess;
  pair_write_kernel<<<nbatch, SCR_THREADS, 0, st>>>(a, list_off, list);
  return cudaGetLastError();
}

cudaError_t launch_fgemm(cudaStream_t st, const BatchDesc* dbatch, int nbatch, int max_ldq, int max_nS,
                         const double* P, const float2* P2, const int* xfunc, const int* sfunc, const double* fcomp,
                         const double* w, double* ws, float* ws32, int mode, int dens) {
  if (nbatch == 0 || max_ldq == 0 || max_nS == 0) return cudaSuccess;
  dim3 grid((max_ldq + TM - 1) / TM, (max_nS + TN - 1) / TN, nbatch);
  if (mode == 2)
    fgemm_kernel<2><<<grid, GEMM_THREADS, 0, st>>>(dbatch, P, P2, xfunc, sfunc, fcomp, w, ws, ws32, dens);
  else
    fgemm_kernel<0><<<grid, GEMM_THREADS, 0, st>>>(dbatch, P, P2, xfunc, sfunc, fcomp, w, ws, ws32, dens);
  return cudaGetLastError();
}

cudaError_t launch_kgemm(cudaStream_t st, const BatchDesc* dbatch, int nbatch, int max_nS, int max_nB,
                         const int* xfunc, const int* sfunc, const double* ws, unsigned long long* Khat, int mode,
                         int dens, int* err) {
  if (nbatch == 0 || max_nS == 0 || max_nB == 0) return cudaSuccess;
  dim3 grid((max_nS + TM - 1) / TM, (max_nB + TN - 1) / TN, nbatch);
  if (mode == 2)
    kgemm_kernel<2><<<grid, GEMM_THREADS, 0, st>>>(dbatch, xfunc, sfunc, ws, Khat, dens, err);
  else
    kgemm_kernel<0><<<grid, GEMM_THREADS, 0, st>>>(dbatch, xfunc, sfunc, ws, Khat, dens, err);
  return cudaGetLastError();
}

cudaError_t launch_gen_tiles(cudaStream_t st, int nbatch, const BatchDesc* batches, const int* counts,
                             const int64_t* list_off, const int64_t* tstart, Tile* tiles) {
  if (nbatch == 0) return cudaSuccess;
  gen_tiles_kernel<<<dim3(nbatch, kNumLists), 256, 0, st>>>(batches, counts, list_off, tstart, tiles);
  return cudaGetLastError();
}

cudaError_t launch_abs_sum(cudaStream_t st, const double* P, int n_dens, int64_t n, double* out) {
  if (n <= 0) return cudaSuccess;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  abs_sum_kernel<<<grid, 256, 0, st>>>(P, n_dens, n, out);
  return cudaGetLastError();
}

cudaError_t launch_split_df32(cudaStream_t st, double* buf, int64_t n) {
  if (n <= 0) return cudaSuccess;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  split_df32_kernel<<<grid, 256, 0, st>>>(buf, n);
  return cudaGetLastError();
}

cudaError_t launch_split_df32_copy(cudaStream_t st, const double* src, int64_t n, float2* dst) {
  if (n <= 0) return cudaSuccess;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  split_df32_copy_kernel<<<grid, 256, 0, st>>>(src, n, dst);
  return cudaGetLastError();
}

cudaError_t launch_finish(cudaStream_t st, const MolDesc* mols, int n_mol, int64_t packed, const unsigned long long* Khat,
                          const double* fcomp, double* K) {
  if (packed == 0) return cudaSuccess;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((packed + 255) / 256, 152 * 16));
  finish_kernel<<<blocks, 256, 0, st>>>(mols, n_mol, packed, Khat, fcomp, K);
  return cudaGetLastError();
}

cudaError_t launch_symcheck(cudaStream_t st, const MolDesc* mols, int n_mol, int64_t packed, const double* P,
                            double* out2) {
  if (packed == 0) return cudaSuccess;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((packed + 255) / 256, 152 * 8));
  symcheck_kernel<<<blocks, 256, 0, st>>>(mols, n_mol, packed, P, out2);
  return cudaGetLastError();
}

cudaError_t launch_xc_fgemm(cudaStream_t st, const BatchDesc* dbatch, int nbatch, int max_ldq, int max_nB,
                            const double* P, const int* xfunc, double* ws, int mode) {
  if (nbatch == 0 || max_ldq == 0 || max_nB == 0) return cudaSuccess;
  dim3 grid((max_ldq + TM - 1) / TM, (max_nB + TN - 1) / TN, nbatch);
  if (mode == 2)
    xc_fgemm_kernel<2><<<grid, GEMM_THREADS, 0, st>>>(dbatch, P, xfunc, ws);
  else
    xc_fgemm_kernel<0><<<grid, GEMM_THREADS, 0, st>>>(dbatch, P, xfunc, ws);
  return cudaGetLastError();
}

cudaError_t launch_xc_vgemm(cudaStream_t st, const BatchDesc* dbatch, int nbatch, int max_nB, const int* xfunc,
                            const double* ws, unsigned long long* Vhat, int mode, int* err) {
  if (nbatch == 0 || max_nB == 0) return cudaSuccess;
  dim3 grid((max_nB + TM - 1) / TM, (max_nB + TN - 1) / TN, nbatch);
  if (mode == 2)
    xc_vgemm_kernel<2><<<grid, GEMM_THREADS, 0, st>>>(dbatch, xfunc, ws, Vhat, err);
  else
    xc_vgemm_kernel<0><<<grid, GEMM_THREADS, 0, st>>>(dbatch, xfunc, ws, Vhat, err);
  return cudaGetLastError();
}

}  // namespace snk
