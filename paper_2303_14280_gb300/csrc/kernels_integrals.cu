// Integral-contraction kernel of libsnk (sm_103a): for every shell pair (a, b)
// of a batch's pair list V_j and every grid point r_i of the batch,
//
//   Theta^n_0 = pref * F_n(zeta |P - r_i|^2)              (App. A, seed)
//   VRR over the primitive pairs, Theta^0 contracted      (App. A, Eq. vrr)
//   HRR to the target block Xi_ab                          (App. A, Eq. hrr)
//   G_{i a} += Xi_ab F_{i b},  G_{i b} += Xi_ab^T F_{i a}  (Eq. gmat, a != b)
//
// with F already scaled by w_i and the component factor of its column, so the
// 3c-CP block is never stored (the merged HRR + contraction of App. A).
//
// Parallel decomposition (Sec. II.F, batching levels (1)-(3)): one thread per
// grid point, a 128-point tile of one batch per CTA iteration, a run of pairs
// of one class per tile; persistent CTAs take tiles from an atomic ticket.  The
// Boys interpolation table of the class's L lives in shared memory.
//
// GB300 issues FP64 at 2 DFMA per SM per clock (1/64 of FP32), so the kernel
// is FP64-pipe bound by construction: table lookups, index arithmetic, F loads
// and the G atomics (L2 reductions, ~600 G/s) all hide under the DFMA stream,
// and the generated VRR/HRR minimise the FP64 instruction count.
#include <cuda_runtime.h>

#include <cstdint>

#include "os_generated.cuh"
#include "snk_internal.h"

namespace snk {

namespace {

constexpr int kIntThreads = kPointTile;
constexpr long long kBoysTMaxBits = 0x4049000000000000LL;  // bit pattern of 50.0
static_assert(kBoysTMax == 50.0, "kBoysTMaxBits encodes 50.0");

// S_n = pref * F_n(T), n = 0..L (Eq. boys).  Below T = 50: an 8-term Taylor
// expansion of F_L about the nearest table node (dF_n/dT = -F_{n+1}) and the
// downward recursion F_n = (2T F_{n+1} + e^{-T}) / (2n+1); above: F_0 =
// sqrt(pi/T)/2 and F_{n+1} = (2n+1) F_n / (2T) (e^{-T} < 2e-22 is dropped).
template <int L>
__device__ __forceinline__ void boys_seeds(double T, double pref, double pref_far, const double* tab, double* S) {
  if (__double_as_longlong(T) < kBoysTMaxBits) {
    const int k = __float2int_rn(__double2float_rn(T) * (float)(1.0 / kBoysH));
    const double* row = tab + k * kBoysCols;
    const double x = row[kBoysCols - 1] - T;  // T_k - T, |x| <= 0.05
    double f = row[7];
#pragma unroll
    for (int m = 6; m >= 0; --m) f = fma(f, x, row[m]);
    S[L] = pref * f;
    if (L > 0) {
      // e^{-T} = e^{-T_k} e^{x}, e^{x} by its 8-term Taylor polynomial
      double e = 1.0 / 5040.0;
      e = fma(e, x, 1.0 / 720.0);
      e = fma(e, x, 1.0 / 120.0);
      e = fma(e, x, 1.0 / 24.0);
      e = fma(e, x, 1.0 / 6.0);
      e = fma(e, x, 0.5);
      e = fma(e, x, 1.0);
      e = fma(e, x, 1.0);
      const double pe = (pref * row[kBoysTerms]) * e;
      const double T2 = T + T;
#pragma unroll
      for (int n = L - 1; n >= 0; --n) S[n] = fma(T2, S[n + 1], pe) * (1.0 / (2 * n + 1));
    }
  } else {
    const double r = rsqrt(T);
    S[0] = pref_far * r;
    if (L > 0) {
      const double o = 0.5 * (r * r);
#pragma unroll
      for (int n = 0; n < L; ++n) S[n + 1] = S[n] * ((2 * n + 1) * o);
    }
  }
}

// Contracted Xi_ab (no component factors) of one pair at the point (cx, cy, cz).
template <int LA, int LB>
__device__ __forceinline__ void pair_xi(const PairHdr& h, const PrimPair* __restrict__ prims, const double* tab,
                                        double cx, double cy, double cz, double* xi) {
  using C = OsClass<LA, LB>;
  double acc[C::NACC];
#pragma unroll
  for (int k = 0; k < C::NACC; ++k) acc[k] = 0.0;
  for (int q = 0; q < h.pp_n; ++q) {
    const PrimPair pp = prims[h.pp_off + q];
    const double PCx = pp.Px - cx, PCy = pp.Py - cy, PCz = pp.Pz - cz;
    const double T = pp.zeta * fma(PCx, PCx, fma(PCy, PCy, PCz * PCz));
    double S[C::L + 1];
    boys_seeds<C::L>(T, pp.pref, pp.pref_far, tab, S);
    C::vrr(S, pp.PAx, pp.PAy, pp.PAz, PCx, PCy, PCz, pp.k1, pp.k2, pp.k3, acc);
  }
  C::hrr(acc, h.ABx, h.ABy, h.ABz, xi);
}

template <int LA, int LB>
__global__ void __launch_bounds__(kIntThreads) integral_kernel(IntegralArgs a) {
  using C = OsClass<LA, LB>;
  constexpr int NA = C::NA, NB = C::NB;
  extern __shared__ double s_tab[];
  const double* gtab = a.boys + (size_t)C::L * kBoysRows * kBoysCols;
  for (int e = threadIdx.x; e < kBoysRows * kBoysCols; e += blockDim.x) s_tab[e] = gtab[e];
  __shared__ int s_tile;
  __syncthreads();
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(a.ticket, 1);
    __syncthreads();
    const int t = s_tile;
    __syncthreads();
    if (t >= a.n_tiles) break;
    const Tile tile = a.tiles[t];
    const BatchDesc bd = a.batches[tile.batch];
    const int i = tile.i0 + threadIdx.x;
    if (i >= bd.q) continue;
    const int64_t ldq = bd.ldq;
    const double cx = a.xyz[3 * (bd.p0 + i)], cy = a.xyz[3 * (bd.p0 + i) + 1], cz = a.xyz[3 * (bd.p0 + i) + 2];
    const double* F = a.ws + bd.foff + i;
    double* G = a.ws + bd.goff + i;
    const int* cmap = a.colmap + (int64_t)tile.batch * a.ns;
    double ga[NA], fa[NA];
    int cur = -1, cola = 0;
    for (int k = tile.k0; k < tile.k1; ++k) {
      const PairHdr h = a.pairs[a.pairlist[k]];
      if (h.sa != cur) {
        if (cur >= 0) {
#pragma unroll
          for (int u = 0; u < NA; ++u) atomicAdd(G + (cola + u) * ldq, ga[u]);
        }
        cur = h.sa;
        cola = cmap[cur];
#pragma unroll
        for (int u = 0; u < NA; ++u) {
          ga[u] = 0.0;
          fa[u] = F[(cola + u) * ldq];
        }
      }
      const int colb = cmap[h.sb];
      if (cola < 0 || colb < 0) continue;  // cannot happen: the screen marks both shells of a kept pair
      double fb[NB];
#pragma unroll
      for (int v = 0; v < NB; ++v) fb[v] = F[(colb + v) * ldq];
      double xi[NA * NB];
      pair_xi<LA, LB>(h, a.prims, s_tab, cx, cy, cz, xi);
#pragma unroll
      for (int u = 0; u < NA; ++u)
#pragma unroll
        for (int v = 0; v < NB; ++v) ga[u] = fma(xi[u * NB + v], fb[v], ga[u]);
      if (h.sa != h.sb) {
#pragma unroll
        for (int v = 0; v < NB; ++v) {
          double g = 0.0;
#pragma unroll
          for (int u = 0; u < NA; ++u) g = fma(xi[u * NB + v], fa[u], g);
          atomicAdd(G + (colb + v) * ldq, g);
        }
      }
    }
    if (cur >= 0) {
#pragma unroll
      for (int u = 0; u < NA; ++u) atomicAdd(G + (cola + u) * ldq, ga[u]);
    }
  }
}

template <int LA, int LB>
__global__ void debug_xi_kernel(const PairHdr* pair, const PrimPair* prims, const double* boys, int64_t n,
                                const double* xyz, double* out) {
  using C = OsClass<LA, LB>;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* tab = boys + (size_t)C::L * kBoysRows * kBoysCols;
  double xi[C::NA * C::NB];
  pair_xi<LA, LB>(*pair, prims, tab, xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], xi);
  for (int k = 0; k < C::NA * C::NB; ++k) out[i * C::NA * C::NB + k] = xi[k];
}

template <int L>
__device__ void boys_row(double T, const double* boys, double* out) {
  double S[L + 1];
  boys_seeds<L>(T, 1.0, 0.88622692545275801365, boys + (size_t)L * kBoysRows * kBoysCols, S);
  for (int n = 0; n <= L; ++n) out[n] = S[n];
}

__global__ void debug_boys_kernel(const double* boys, int64_t n, const double* T, int nmax, double* out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double* o = out + i * (nmax + 1);
  switch (nmax) {
    case 0: boys_row<0>(T[i], boys, o); break;
    case 1: boys_row<1>(T[i], boys, o); break;
    case 2: boys_row<2>(T[i], boys, o); break;
    case 3: boys_row<3>(T[i], boys, o); break;
    default: boys_row<4>(T[i], boys, o); break;
  }
}

template <int LA, int LB>
cudaError_t launch_class(cudaStream_t st, const IntegralArgs& a, int grid) {
  const size_t smem = sizeof(double) * kBoysRows * kBoysCols;
  cudaError_t e = cudaFuncSetAttribute(integral_kernel<LA, LB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  integral_kernel<LA, LB><<<grid, kIntThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <int LA, int LB>
int max_ctas(int num_sms) {
  const size_t smem = sizeof(double) * kBoysRows * kBoysCols;
  cudaFuncSetAttribute(integral_kernel<LA, LB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, integral_kernel<LA, LB>, kIntThreads, smem) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm * num_sms;
}

}  // namespace

cudaError_t launch_integrals(cudaStream_t st, int cls, const IntegralArgs& a, int grid_ctas) {
  if (a.n_tiles == 0) return cudaSuccess;
  switch (cls) {
    case 0: return launch_class<0, 0>(st, a, grid_ctas);
    case 1: return launch_class<1, 0>(st, a, grid_ctas);
    case 2: return launch_class<1, 1>(st, a, grid_ctas);
    case 3: return launch_class<2, 0>(st, a, grid_ctas);
    case 4: return launch_class<2, 1>(st, a, grid_ctas);
    case 5: return launch_class<2, 2>(st, a, grid_ctas);
  }
  return cudaErrorInvalidValue;
}

int integral_max_ctas(int cls, int num_sms) {
  switch (cls) {
    case 0: return max_ctas<0, 0>(num_sms);
    case 1: return max_ctas<1, 0>(num_sms);
    case 2: return max_ctas<1, 1>(num_sms);
    case 3: return max_ctas<2, 0>(num_sms);
    case 4: return max_ctas<2, 1>(num_sms);
    case 5: return max_ctas<2, 2>(num_sms);
  }
  return num_sms;
}

cudaError_t launch_debug_A(cudaStream_t st, int cls, const PairHdr* pair, const PrimPair* prims, const double* boys,
                           int64_t n, const double* xyz, double* xi) {
  if (n == 0) return cudaSuccess;
  const int th = 128;
  const unsigned blocks = (unsigned)((n + th - 1) / th);
  switch (cls) {
    case 0: debug_xi_kernel<0, 0><<<blocks, th, 0, st>>>(pair, prims, boys, n, xyz, xi); break;
    case 1: debug_xi_kernel<1, 0><<<blocks, th, 0, st>>>(pair, prims, boys, n, xyz, xi); break;
    case 2: debug_xi_kernel<1, 1><<<blocks, th, 0, st>>>(pair, prims, boys, n, xyz, xi); break;
    case 3: debug_xi_kernel<2, 0><<<blocks, th, 0, st>>>(pair, prims, boys, n, xyz, xi); break;
    case 4: debug_xi_kernel<2, 1><<<blocks, th, 0, st>>>(pair, prims, boys, n, xyz, xi); break;
    case 5: debug_xi_kernel<2, 2><<<blocks, th, 0, st>>>(pair, prims, boys, n, xyz, xi); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_debug_boys(cudaStream_t st, const double* boys, int64_t n, const double* T, int nmax,
                              double* out) {
  if (n == 0) return cudaSuccess;
  const int th = 128;
  debug_boys_kernel<<<(unsigned)((n + th - 1) / th), th, 0, st>>>(boys, n, T, nmax, out);
  return cudaGetLastError();
}

// Algorithmic FP64 flops per (grid point, contracted shell pair), FMA = 2:
// per primitive pair the T evaluation (8), the Boys seeds counted at the
// cheaper large-T form (1 for L = 0, else 3 + 2L; the library rsqrt is not
// counted) and the
// generated VRR; per contracted pair the generated HRR and the G_a
// contraction (2 NA NB).  The G_b half of off-diagonal pairs is not counted.
void class_flops(int cls, int nprim_pairs, double* f) {
  int vrr = 0, hrr = 0, L = 0, na = 1, nb = 1;
  switch (cls) {
#define SNK_CASE(c, A, B)          \
  case c:                          \
    vrr = OsClass<A, B>::VRR_FLOPS; \
    hrr = OsClass<A, B>::HRR_FLOPS; \
    L = OsClass<A, B>::L;           \
    na = OsClass<A, B>::NA;         \
    nb = OsClass<A, B>::NB;         \
    break;
    SNK_CASE(0, 0, 0)
    SNK_CASE(1, 1, 0)
    SNK_CASE(2, 1, 1)
    SNK_CASE(3, 2, 0)
    SNK_CASE(4, 2, 1)
    SNK_CASE(5, 2, 2)
#undef SNK_CASE
  }
  const double boys = L == 0 ? 1.0 : 3.0 + 2.0 * L;
  *f = nprim_pairs * (8.0 + boys + vrr) + hrr + 2.0 * na * nb;
}

}  // namespace snk
