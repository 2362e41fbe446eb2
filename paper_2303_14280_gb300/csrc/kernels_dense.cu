// Dense and screening kernels of libsnk (sm_103a):
//   collocation X_j (Eq. collocation), the geometry-only batch maxima of
//   Eq. (exx_fmat_approx), F-tilde = |P| Phi-tilde (Eq. exx_fmat_approx) as
//   a GEMM over batches, the sn-LinK pair screen with per-batch compaction
//   (Eq. sp_set), the FP64 products F_j = X_j P (Eq. batch_local_exx) and
//   Kt += G_j^T X_j (Eq. usym_k), and the symmetrisation of Eq. (sn_k).
//
// FP64 on GB300 issues at 2 DFMA per SM per clock, so a 64 x 64 x 16 tile
// step is ~32k cycles of DFMA against 2k doubles of shared-memory staging:
// the GEMMs are FP64-pipe bound with plain shared-memory tiling.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "snk_internal.h"

namespace snk {

namespace {

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  // for non-negative doubles the IEEE bit pattern orders like the value
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// ---------------------------------------------------------------- GEMM tile

constexpr int TM = 64, TN = 64, TK = 16, GEMM_THREADS = 256;

// C[m][n] = sum_k A(m,k) B(k,n) for the 64 x 64 tile at (m0, n0), K = kdim.
// la(m, k), lb(k, n) return 0 outside the operands; st(m, n, c) stores.
template <class LA, class LB, class ST>
__device__ __forceinline__ void gemm_tile(int m0, int n0, int mdim, int ndim, int kdim, LA la, LB lb,
                                          ST st, bool a_k_fast, bool b_k_fast) {
  __shared__ double As[TK][TM + 1];
  __shared__ double Bs[TK][TN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
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
      As[kk][mm] = (m < mdim && k < kdim) ? la(m, k) : 0.0;
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
      Bs[kk][nn] = (n < ndim && k < kdim) ? lb(k, n) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double a[4], b[4];
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

// ---------------------------------------------------------------- collocation

constexpr int COL_THREADS = 128, COL_SHELLS = 8;

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
    for (int k = B.poff[sh]; k < B.poff[sh] + B.nprim[sh]; ++k) rad += B.d[k] * exp(-B.exps[k] * r2);
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
                              const double* __restrict__ w, const int* __restrict__ xfunc, int nf,
                              double* __restrict__ phit_f) {
  const BatchDesc bd = batches[blockIdx.y];
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= bd.nB) return;
  const double* X = ws + bd.xoff + (int64_t)c * bd.ldq;
  double m = 0.0;
  for (int i = 0; i < bd.q; ++i) m = fmax(m, sqrt(fabs(w[bd.p0 + i])) * fabs(X[i]));
  phit_f[(int64_t)blockIdx.y * nf + xfunc[bd.xfunc_off + c]] = m;
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

// ---------------------------------------------------------------- F-tilde

// ft_shell[j][a] = max_{mu in a} sum_nu |P_{mu nu}| Phi-tilde_nu^(j): a GEMM over
// (mu, batch) with the shell maximum folded into the store.
__global__ void __launch_bounds__(GEMM_THREADS) ftilde_kernel(const double* __restrict__ P,
                                                              const double* __restrict__ phit_f, int nf,
                                                              int nbatch, const int* __restrict__ fshell,
                                                              int ns, double* __restrict__ ft_shell) {
  const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
  gemm_tile(
      m0, n0, nf, nbatch, nf, [&](int m, int k) { return fabs(P[(int64_t)m * nf + k]); },
      [&](int k, int n) { return phit_f[(int64_t)n * nf + k]; },
      [&](int m, int n, double c) { atomic_max_nonneg(&ft_shell[(int64_t)n * ns + fshell[m]], c); }, true, true);
}

// ---------------------------------------------------------------- sn-LinK pair screen

constexpr int SCR_THREADS = 256;

// Bound of max_{r in Q_j} |A_ab(r)| for batch j: the global bound A-tilde, or,
// when the batch's bounding sphere stays clear of the segment AB that holds
// every Gaussian product centre, the smaller total-charge / distance bound.
__device__ __forceinline__ double batch_pair_bound(const ScreenArgs& a, int j, int p, const PairHdr& h) {
  const double bnd = a.bound[p];
  if (!a.distance) return bnd;
  const double* A = a.shell_xyz + 3 * h.sa;
  const double vx = -h.ABx, vy = -h.ABy, vz = -h.ABz;  // B - A
  const double wx = a.bcenter[3 * j] - A[0], wy = a.bcenter[3 * j + 1] - A[1], wz = a.bcenter[3 * j + 2] - A[2];
  const double vv = vx * vx + vy * vy + vz * vz;
  double t = vv > 0.0 ? (wx * vx + wy * vy + wz * vz) / vv : 0.0;
  t = fmin(fmax(t, 0.0), 1.0);
  const double dx = wx - t * vx, dy = wy - t * vy, dz = wz - t * vz;
  const double d = sqrt(dx * dx + dy * dy + dz * dz) - a.bradius[j];
  return d > 0.0 ? fmin(bnd, a.qbound[p] / d) : bnd;
}

// sn-LinK decision for pair p in batch j, Eq. (sp_set): -1 drop, else the
// list index class + kNumClasses * precision (precision 1 = FP32 integrals,
// for pairs whose estimate max(F_a, F_b) phi A stays below fp32_bound).
__device__ __forceinline__ int classify_pair(const ScreenArgs& a, int j, int p, int cls, const PairHdr& h) {
  if (a.screen == SNK_SCREEN_NONE) return cls;
  const double* ft = a.ft_shell + (int64_t)j * a.ns;
  const double fa = ft[h.sa], fb = ft[h.sb];
  const double bnd = batch_pair_bound(a, j, p, h);
  const double eK = fmax(fa, fb) * a.phit_b[j] * bnd;
  if (!((fa * fb * bnd >= a.eps_E) || (eK >= a.eps_K))) return -1;
  return (a.mixed && eK < a.fp32_bound) ? cls + kNumClasses : cls;
}

// Pass 1: per (batch, list) pair counts and primitive-pair counts; marks the
// shells of every kept pair (their F / G columns).  One block per batch.
__global__ void __launch_bounds__(SCR_THREADS) pair_count_kernel(ScreenArgs a, int* __restrict__ counts,
                                                                 long long* __restrict__ ppcounts,
                                                                 unsigned char* __restrict__ sflag) {
  const int j = blockIdx.x;
  unsigned char* fl = sflag + (int64_t)j * a.ns;
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
    for (int p = a.cr.b[c] + threadIdx.x; p < a.cr.b[c + 1]; p += SCR_THREADS) {
      const PairHdr h = a.pairs[p];
      const int li = classify_pair(a, j, p, c, h);
      if (li >= 0) {
        fl[h.sa] = 1;
        fl[h.sb] = 1;
        const int prec = li >= kNumClasses;
        n[prec] += 1;
        pp[prec] += (unsigned long long)h.pp_n;
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
// ranges that the host sized from pass 1.
__global__ void __launch_bounds__(SCR_THREADS) pair_write_kernel(ScreenArgs a, const int64_t* __restrict__ list_off,
                                                                 int* __restrict__ list) {
  const int j = blockIdx.x;
  __shared__ int warp_tot[2][SCR_THREADS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = 0; c < kNumClasses; ++c) {
    int64_t out[2] = {list_off[j * kNumLists + c], list_off[j * kNumLists + c + kNumClasses]};
    for (int base = a.cr.b[c]; base < a.cr.b[c + 1]; base += SCR_THREADS) {
      const int p = base + threadIdx.x;
      int li = -1;
      if (p < a.cr.b[c + 1]) li = classify_pair(a, j, p, c, a.pairs[p]);
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
// and the Cartesian component factor of the column are folded into F.
__global__ void __launch_bounds__(GEMM_THREADS) fgemm_kernel(const BatchDesc* __restrict__ batches,
                                                             const double* __restrict__ P, int nf,
                                                             const int* __restrict__ xfunc,
                                                             const int* __restrict__ sfunc,
                                                             const double* __restrict__ fcomp,
                                                             const double* __restrict__ w, double* __restrict__ ws,
                                                             float* __restrict__ ws32) {
  const BatchDesc bd = batches[blockIdx.z];
  const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
  if (m0 >= bd.ldq || n0 >= bd.nS) return;
  const double* X = ws + bd.xoff;
  double* F = ws + bd.foff;
  float* F32 = ws32 ? ws32 + bd.foff32 : nullptr;  // mixed form: FP32 copy for the FP32 pairs
  const int* xf = xfunc + bd.xfunc_off;
  const int* sf = sfunc + bd.sfunc_off;
  gemm_tile(
      m0, n0, bd.ldq, bd.nS, bd.nB, [&](int m, int k) { return X[(int64_t)k * bd.ldq + m]; },
      [&](int k, int n) { return P[(int64_t)xf[k] * nf + sf[n]]; },
      [&](int m, int n, double c) {
        const double wi = m < bd.q ? w[bd.p0 + m] : 0.0;
        const double v = wi * fcomp[sf[n]] * c;
        F[(int64_t)n * bd.ldq + m] = v;
        if (F32) F32[(int64_t)n * bd.ldq + m] = (float)v;
      },
      false, false);
}

// G += G32 over a chunk's contiguous G region (mixed form).
__global__ void merge_g32_kernel(const float* __restrict__ g32, int64_t n, double* __restrict__ g64) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    g64[e] += (double)g32[e];
}

// Kt_{s nu} += sum_i G-hat_{s i} X_{nu i}, scattered into the global N_b x N_b
// accumulator (several batches add to the same entries).
__global__ void __launch_bounds__(GEMM_THREADS) kgemm_kernel(const BatchDesc* __restrict__ batches,
                                                             const int* __restrict__ xfunc,
                                                             const int* __restrict__ sfunc, int nf,
                                                             const double* __restrict__ ws,
                                                             double* __restrict__ Khat) {
  const BatchDesc bd = batches[blockIdx.z];
  const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
  if (m0 >= bd.nS || n0 >= bd.nB) return;
  const double* X = ws + bd.xoff;
  const double* G = ws + bd.goff;
  const int* xf = xfunc + bd.xfunc_off;
  const int* sf = sfunc + bd.sfunc_off;
  gemm_tile(
      m0, n0, bd.nS, bd.nB, bd.q, [&](int m, int k) { return G[(int64_t)m * bd.ldq + k]; },
      [&](int k, int n) { return X[(int64_t)n * bd.ldq + k]; },
      [&](int m, int n, double c) { atomicAdd(&Khat[(int64_t)sf[m] * nf + xf[n]], c); }, true, true);
}

// K_{mu nu} = (f_mu Kt_{mu nu} + f_nu Kt_{nu mu}) / 2, Eq. (sn_k); the row factor
// f_mu is the Cartesian component factor that the integral kernel leaves out.
__global__ void finish_kernel(const double* __restrict__ Khat, const double* __restrict__ fcomp, int nf,
                              double* __restrict__ K) {
  const int64_t n = (int64_t)nf * nf;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int mu = (int)(e / nf), nu = (int)(e % nf);
    // explicit rounding of both products keeps K exactly symmetric (no FMA contraction)
    K[e] = 0.5 * __dadd_rn(__dmul_rn(fcomp[mu], Khat[e]), __dmul_rn(fcomp[nu], Khat[(int64_t)nu * nf + mu]));
  }
}

// out2[0] = max |P - P^T|, out2[1] = max |P| (out2 zeroed by the caller).
__global__ void symcheck_kernel(const double* __restrict__ P, int nf, double* __restrict__ out2) {
  const int64_t n = (int64_t)nf * nf;
  double a = 0.0, b = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int mu = (int)(e / nf), nu = (int)(e % nf);
    const double v = P[e];
    a = fmax(a, fabs(v - P[(int64_t)nu * nf + mu]));
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
                               const double* w, const int* xfunc, int nf, double* phit_f, double* phit_b) {
  if (nbatch == 0) return cudaSuccess;
  if (max_nB > 0) {
    dim3 grid((max_nB + 127) / 128, nbatch);
    phit_f_kernel<<<grid, 128, 0, st>>>(dbatch, ws, w, xfunc, nf, phit_f);
  }
  phit_b_kernel<<<nbatch, 256, 0, st>>>(dbatch, ws, w, phit_b);
  return cudaGetLastError();
}

cudaError_t launch_ftilde(cudaStream_t st, const double* P, const double* phit_f, int nf, int nbatch,
                          const int* fshell, int ns, double* ft_shell) {
  if (nbatch == 0) return cudaSuccess;
  dim3 grid((nf + TM - 1) / TM, (nbatch + TN - 1) / TN);
  ftilde_kernel<<<grid, GEMM_THREADS, 0, st>>>(P, phit_f, nf, nbatch, fshell, ns, ft_shell);
  return cudaGetLastError();
}

cudaError_t launch_pair_count(cudaStream_t st, const ScreenArgs& a, int nbatch, int* counts, long long* ppcounts,
                              unsigned char* sflag) {
  if (nbatch == 0) return cudaSuccess;
  pair_count_kernel<<<nbatch, SCR_THREADS, 0, st>>>(a, counts, ppcounts, sflag);
  return cudaGetLastError();
}

cudaError_t launch_pair_write(cudaStream_t st, const ScreenArgs& a, int nbatch, const int64_t* list_off, int* list) {
  if (nbatch == 0) return cudaSuccess;
  pair_write_kernel<<<nbatch, SCR_THREADS, 0, st>>>(a, list_off, list);
  return cudaGetLastError();
}

cudaError_t launch_fgemm(cudaStream_t st, const BatchDesc* dbatch, int nbatch, int max_ldq, int max_nS,
                         const double* P, int nf, const int* xfunc, const int* sfunc, const double* fcomp,
                         const double* w, double* ws, float* ws32) {
  if (nbatch == 0 || max_ldq == 0 || max_nS == 0) return cudaSuccess;
  dim3 grid((max_ldq + TM - 1) / TM, (max_nS + TN - 1) / TN, nbatch);
  fgemm_kernel<<<grid, GEMM_THREADS, 0, st>>>(dbatch, P, nf, xfunc, sfunc, fcomp, w, ws, ws32);
  return cudaGetLastError();
}

cudaError_t launch_merge_g32(cudaStream_t st, const float* g32, int64_t n, double* g64) {
  if (n == 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  merge_g32_kernel<<<blocks, 256, 0, st>>>(g32, n, g64);
  return cudaGetLastError();
}

cudaError_t launch_kgemm(cudaStream_t st, const BatchDesc* dbatch, int nbatch, int max_nS, int max_nB,
                         const int* xfunc, const int* sfunc, int nf, const double* ws, double* Khat) {
  if (nbatch == 0 || max_nS == 0 || max_nB == 0) return cudaSuccess;
  dim3 grid((max_nS + TM - 1) / TM, (max_nB + TN - 1) / TN, nbatch);
  kgemm_kernel<<<grid, GEMM_THREADS, 0, st>>>(dbatch, xfunc, sfunc, nf, ws, Khat);
  return cudaGetLastError();
}

cudaError_t launch_finish(cudaStream_t st, const double* Khat, const double* fcomp, int nf, double* K) {
  int64_t n = (int64_t)nf * nf;
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  if (blocks < 1) blocks = 1;
  finish_kernel<<<blocks, 256, 0, st>>>(Khat, fcomp, nf, K);
  return cudaGetLastError();
}

cudaError_t launch_symcheck(cudaStream_t st, const double* P, int nf, double* out2) {
  int64_t n = (int64_t)nf * nf;
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
  if (blocks < 1) blocks = 1;
  symcheck_kernel<<<blocks, 256, 0, st>>>(P, nf, out2);
  return cudaGetLastError();
}

}  // namespace snk
