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
// grid point, a 128-point tile of one batch per CTA iteration, the batch's
// whole pair list of one class per tile; persistent CTAs take tiles from an
// atomic ticket (largest batches first).  Each G entry of a launch therefore
// has a single writer, its point's thread, whose reductions land in list
// order: G, and with it K, is the same bit for bit from run to run.  The Boys
// interpolation table of the class's L lives in shared memory.
//
// GB300 issues FP64 at 2 DFMA per SM per clock (1/64 of FP32), so the kernel
// is FP64-pipe bound by construction: table lookups, index arithmetic, F loads
// and the G atomics (L2 reductions, ~600 G/s) all hide under the DFMA stream,
// and the generated VRR/HRR minimise the FP64 instruction count.  The mixed
// form adds an FP32 kernel for its low-estimate pairs and a double-FP32 one
// (ds_arith.cuh) for the rest; all three take the number of densities sharing
// each 3c-CP block as a template parameter.
#include <cuda_runtime.h>

#include <cstdint>

#include "async_copy.cuh"
#include "ds_arith.cuh"
#include "os_generated.cuh"
#include "snk_internal.h"

namespace snk {

namespace {

constexpr int kIntThreads = kPointTile;
constexpr int kMaxRun = 128;  // most pairs per staging step (the autotuner's largest candidate)
constexpr unsigned long long kCopyWaitNs = 2000000000ull;  // 2 s per wait on a bulk copy, then give up
static_assert(kMaxRun == kIntThreads, "the FP32 kernel stages a step's pairs one per thread");
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

// ND densities share every Xi block: F and G of density d sit d ldq nS
// doubles after the batch's first block.
template <int LA, int LB, int ND>
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
    const int64_t ldq = bd.ldq, dstr = (int64_t)bd.ldq * bd.nS;
    const double cx = a.xyz[3 * (bd.p0 + i)], cy = a.xyz[3 * (bd.p0 + i) + 1], cz = a.xyz[3 * (bd.p0 + i) + 2];
    const double* F = a.ws + bd.foff + i;
    double* G = a.ws + bd.goff + i;
    const int* cmap = a.colmap + bd.cm_off - bd.ms0;  // indexed by global shell id
    double ga[ND][NA], fa[ND][NA];
    int cur = -1, cola = 0;
    for (int k = tile.k0; k < tile.k1; ++k) {
      const PairHdr h = a.pairs[a.pairlist[k]];
      if (h.sa != cur) {
        if (cur >= 0) {
#pragma unroll
          for (int d = 0; d < ND; ++d)
#pragma unroll
            for (int u = 0; u < NA; ++u) atomicAdd(G + d * dstr + (cola + u) * ldq, ga[d][u]);
        }
        cur = h.sa;
        cola = cmap[cur];
#pragma unroll
        for (int d = 0; d < ND; ++d)
#pragma unroll
          for (int u = 0; u < NA; ++u) {
            ga[d][u] = 0.0;
            fa[d][u] = F[d * dstr + (cola + u) * ldq];
          }
      }
      const int colb = cmap[h.sb];
      if (cola < 0 || colb < 0) continue;  // cannot happen: the screen marks both shells of a kept pair
      double fb[ND][NB];
#pragma unroll
      for (int d = 0; d < ND; ++d)
#pragma unroll
        for (int v = 0; v < NB; ++v) fb[d][v] = F[d * dstr + (colb + v) * ldq];
      double xi[NA * NB];
      pair_xi<LA, LB>(h, a.prims, s_tab, cx, cy, cz, xi);
#pragma unroll
      for (int d = 0; d < ND; ++d)
#pragma unroll
        for (int u = 0; u < NA; ++u)
#pragma unroll
          for (int v = 0; v < NB; ++v) ga[d][u] = fma(xi[u * NB + v], fb[d][v], ga[d][u]);
      if (h.sa != h.sb) {
#pragma unroll
        for (int d = 0; d < ND; ++d)
#pragma unroll
          for (int v = 0; v < NB; ++v) {
            double g = 0.0;
#pragma unroll
            for (int u = 0; u < NA; ++u) g = fma(xi[u * NB + v], fa[d][u], g);
            atomicAdd(G + d * dstr + (colb + v) * ldq, g);
          }
      }
    }
    if (cur >= 0) {
#pragma unroll
      for (int d = 0; d < ND; ++d)
#pragma unroll
        for (int u = 0; u < NA; ++u) atomicAdd(G + d * dstr + (cola + u) * ldq, ga[d][u]);
    }
  }
}

// ---------------------------------------------------------------- FP32 pairs (mixed form)

// FP32 seeds S_n = pref F_n(T): 4-term Taylor about the nearest node of a
// 0.05-spaced float table below T = 30 (|T - T_k| <= 0.025: truncation below
// 2e-8 relative; one 16-byte row per lookup, the node fl32(k * 0.05f) formed
// in registers), the asymptotic form above (e^{-T} < 1e-13 is below FP32
// resolution).  e^{-T} of the downward recursion comes from the hardware
// exponential (__expf, ~2^-21 relative).
template <int L>
__device__ __forceinline__ void boys_seeds_f32(float T, float pref, float pref_far, const float* tab, float* S) {
  if (T < kBoysTMaxF) {
    static_assert(kBoysColsF == 4 && kBoysTermsF == 4, "an FP32 table row is one float4");
    const int k = __float2int_rn(T * (1.0f / kBoysHF));
    const float4 r = reinterpret_cast<const float4*>(tab)[k];  // F_{L+m}(T_k)/m!, m = 0..3
    const float x = (float)k * kBoysHF - T;
    float f = fmaf(r.w, x, r.z);
    f = fmaf(f, x, r.y);
    f = fmaf(f, x, r.x);
    S[L] = pref * f;
    if (L > 0) {
      const float pe = pref * __expf(-T);
      const float T2 = T + T;
#pragma unroll
      for (int n = L - 1; n >= 0; --n) S[n] = fmaf(T2, S[n + 1], pe) * (1.0f / (2 * n + 1));
    }
  } else {
    const float r = rsqrtf(T);
    S[0] = pref_far * r;
    if (L > 0) {
      const float o = 0.5f * (r * r);
#pragma unroll
      for (int n = 0; n < L; ++n) S[n + 1] = S[n] * ((2 * n + 1) * o);
    }
  }
}

// The FP32 lists of the mixed form.  Each primitive pair is a 32-byte FP32
// record {zeta, P - A, pref, pref_far, 1/(2 zeta)}; per (pair, point) the
// kernel forms A - r_i once from the (hi, lo) float splits of A and r_i, and
// P - r_i = (P - A) + (A - r_i) per primitive: accurate to FP32 relative to
// the larger of |P - A| and |A - r_i| wherever the molecule sits, which is
// what the VRR terms PA_x Theta and PC_x Theta need.  A tile is a batch's
// whole list on 128 points, taken in steps of a.run pairs: each step's pair
// headers, columns, R_a - R_b and R_a are staged in shared memory (one per
// thread, after the tile screen), and the tile's batch descriptor sits in
// shared memory too, so that nothing of the tile stays in registers across
// the pair loop.  Per pair each warp needs the pair's primitive records and
// the F columns of shell b at its 32 points:
//   - heavy classes (L >= 2): a ring of three slots per warp, filled by TMA
//     bulk copies that lane 0 issues two pairs ahead, each slot completing
//     on its own mbarrier (bounded waits);
//   - light classes: the next pair's F from global memory into registers and
//     its records into a second shared buffer while the current pair
//     computes (fewer instructions per pair than the ring, whose serial
//     issue does not pay for a pair of a few primitives).
template <int LA, int LB, int ND>
__global__ void __launch_bounds__(kIntThreads) integral_kernel_f32(IntegralArgs a) {
  using C = OsClass<LA, LB>;
  constexpr int NA = C::NA, NB = C::NB;
  constexpr int kStage = 16;               // primitive records of a pair staged (32 float4)
  constexpr bool RING = C::L >= 2;
  constexpr int kRing = 3;
  constexpr int kRecF4 = 2 * kStage;       // float4 of records per slot
  constexpr int kFbF4 = ND * NB * 32 / 4;  // float4 of F_b per ring slot
  constexpr int kW = kIntThreads / 32;
  extern __shared__ __align__(16) float s_tabf[];
  const float* gtab = a.boys_f + (size_t)C::L * kBoysRowsF * kBoysColsF;
  for (int e = threadIdx.x; e < kBoysRowsF * kBoysColsF; e += blockDim.x) s_tabf[e] = gtab[e];
  __shared__ int s_ppo[kMaxRun], s_ppn[kMaxRun], s_sa[kMaxRun], s_sb[kMaxRun], s_ca[kMaxRun], s_cb[kMaxRun];
  __shared__ float2 s_ab[kMaxRun][3];  // (hi, lo)
  __shared__ float2 s_A[kMaxRun][3];   // (hi, lo)
  __shared__ __align__(128) float4 s_ring[RING ? kW : 1][RING ? kRing : 1][RING ? kRecF4 + kFbF4 : 1];
  __shared__ __align__(8) uint64_t s_full[kW][kRing];
  __shared__ float4 s_pr[RING ? 1 : kW][2][RING ? 1 : kRecF4];
  __shared__ Tile s_t;
  __shared__ BatchDesc s_bd;
  __shared__ int s_tid, s_wcnt[kW];
  __shared__ volatile int s_abort;  // a wait ran out: the CTA stops taking work
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_abort = 0;
  if (RING && lane == 0) {
#pragma unroll
    for (int s = 0; s < kRing; ++s) mbar_init(&s_full[wid][s], 1);
    mbar_init_fence();
  }
  uint32_t prod = 0, cons = 0;  // ring: this warp's pairs issued into / taken from its slots
  for (;;) {
    __syncthreads();  // every thread is done with the previous tile's descriptors and pairs
    if (threadIdx.x == 0) {
      const int t = atomicAdd(a.ticket, 1);
      s_tid = t;
      if (t < a.n_tiles) {
        s_t = a.tiles[t];
        s_bd = a.batches[s_t.batch];
      }
    }
    __syncthreads();
    if (s_tid >= a.n_tiles || s_abort) break;
    // the tile's list in steps of a.run pairs (block-uniform loop: every
    // thread passes the same barriers)
    for (int kb = s_t.k0; kb < s_t.k1; kb += a.run) {
      // stage the step's pairs (one per thread, order kept); with the tile screen
      // only those whose bound on this tile's points reaches eps_tile
      int nrun;
      {
        const int r = threadIdx.x, n = min(a.run, s_t.k1 - kb);  // n <= kMaxRun = blockDim
        int p = 0, ca = 0, cb = 0, npp_keep = 0;
        PairHdr h{};
        bool keep = r < n;
        if (keep) {
          const int* cmap = a.colmap + s_bd.cm_off - s_bd.ms0;  // indexed by global shell id
          p = a.pairlist[kb + r];
          h = a.pairs[p];
          ca = cmap[h.sa];
          cb = cmap[h.sb];
          npp_keep = h.pp_n32;  // the leading primitive pairs the FP32 tier keeps
          if (a.eps_tile > 0.f) {
            const float* ts = a.tsum + s_bd.ssoff + (int64_t)(s_t.i0 / kPointTile) * (s_bd.nS + 4);
            float sa = 0.f, sb = 0.f;
#pragma unroll
            for (int u = 0; u < NA; ++u) sa += ts[ca + u];
#pragma unroll
            for (int v = 0; v < NB; ++v) sb += ts[cb + v];
            // |A_ab| <= min(global bound, total charge / distance) on the tile's sphere
            const double* A = a.shell_xyz + 3 * h.sa;
            const float vx = (float)-h.ABx, vy = (float)-h.ABy, vz = (float)-h.ABz;  // B - A
            const float wx = ts[s_bd.nS] - (float)A[0], wy = ts[s_bd.nS + 1] - (float)A[1],
                        wz = ts[s_bd.nS + 2] - (float)A[2];
            const float vv = vx * vx + vy * vy + vz * vz;
            float tt = vv > 0.f ? (wx * vx + wy * vy + wz * vz) / vv : 0.f;
            tt = fminf(fmaxf(tt, 0.f), 1.f);
            const float dx = wx - tt * vx, dy = wy - tt * vy, dz = wz - tt * vz;
            const float d = sqrtf(dx * dx + dy * dy + dz * dz) - ts[s_bd.nS + 3] - 1e-4f;
            const float glob = (float)a.pbound[p], smax = fmaxf(sa, sb);
            float bnd = glob;
            if (d > 0.f) bnd = fminf(bnd, (float)a.qbound[p] / d);
            keep = bnd * smax >= a.eps_tile;
            if (keep) {
              // primitive pairs come largest bound first: leave out the tail whose
              // bounds on this tile add up to less than eps_tile
              const float4* rec = a.prims_f32 + (size_t)h.pp_off * 2;
              float tail = 0.f;
              int n = h.pp_n32;
              while (n > 1) {
                const float t2 = tail + rec[2 * (n - 1) + 1].w * glob * smax;
                if (t2 >= a.eps_tile) break;
                tail = t2;
                --n;
              }
              npp_keep = n;
            }
          }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) s_wcnt[wid] = __popc(bal);
        __syncthreads();
        int before = 0;
        nrun = 0;
#pragma unroll
        for (int w = 0; w < kW; ++w) {
          before += w < wid ? s_wcnt[w] : 0;
          nrun += s_wcnt[w];
        }
        if (keep) {
          const int q = before + __popc(bal & ((1u << lane) - 1u));
          s_ppo[q] = h.pp_off;
          s_ppn[q] = npp_keep;
          s_sa[q] = h.sa;
          s_sb[q] = h.sb;
          s_ca[q] = ca;
          s_cb[q] = cb;
          const float2* ab = a.pair_ab + 4 * (size_t)p;
          const float2* pa = a.pair_a + 4 * (size_t)p;
#pragma unroll
          for (int m = 0; m < 3; ++m) {
            s_ab[q][m] = ab[m];
            s_A[q][m] = pa[m];
          }
        }
      }
      __syncthreads();
      if (threadIdx.x == 0 && nrun > 0) {  // the work this step computes, for the flop counts
        unsigned long long npp = 0;
        for (int r = 0; r < nrun; ++r) npp += (unsigned long long)s_ppn[r];
        const unsigned long long pts = (unsigned long long)min(kPointTile, s_bd.q - s_t.i0);
        atomicAdd(&a.exec[0], npp * pts);
        atomicAdd(&a.exec[1], (unsigned long long)nrun * pts);
      }
      const int i = s_t.i0 + threadIdx.x;
      const bool active = i < s_bd.q;  // inactive lanes of a partly active warp follow along
      if (nrun <= 0 || s_abort || __all_sync(0xffffffffu, !active)) continue;
      ds cx = ds_make(0.f, 0.f), cy = cx, cz = cx;
      if (active) {
        cx = ds_from(a.xyz[3 * (s_bd.p0 + i)]);
        cy = ds_from(a.xyz[3 * (s_bd.p0 + i) + 1]);
        cz = ds_from(a.xyz[3 * (s_bd.p0 + i) + 2]);
      }
      const int64_t ldq = s_bd.ldq, dstr = (int64_t)s_bd.ldq * s_bd.nS;  // density d's F / G: + d dstr
      const float* F = a.ws32 + s_bd.foff32 + i;
      double* G64 = a.ws + s_bd.goff + i;
      // the FP32 contributions are added to the FP64 G with FP64 reductions;
      // each G entry of the launch has one writer (its point's thread), so
      // they land in list order and G is the same from run to run
      auto gadd = [&](int d, int col, float v) { atomicAdd(G64 + d * dstr + col * ldq, (double)v); };
      float ga[ND][NA], fa[ND][NA];
      int cur = -1, cola = 0;
      // pair r at this thread's point, from its records (shared memory, or
      // global memory for more than kStage primitive pairs) and F_b
      auto compute = [&](int r, const float4* rec, const float (&fb)[ND][NB]) {
        const int sa = s_sa[r];
        if (sa != cur) {
          if (cur >= 0) {
#pragma unroll
            for (int d = 0; d < ND; ++d)
#pragma unroll
              for (int u = 0; u < NA; ++u) gadd(d, cola + u, ga[d][u]);
          }
          cur = sa;
          cola = s_ca[r];
#pragma unroll
          for (int d = 0; d < ND; ++d)
#pragma unroll
            for (int u = 0; u < NA; ++u) {
              ga[d][u] = 0.f;
              fa[d][u] = F[d * dstr + (cola + u) * ldq];
            }
        }
        // A - r_i, once per pair and point
        const float ACx = (s_A[r][0].x - cx.hi) + (s_A[r][0].y - cx.lo);
        const float ACy = (s_A[r][1].x - cy.hi) + (s_A[r][1].y - cy.lo);
        const float ACz = (s_A[r][2].x - cz.hi) + (s_A[r][2].y - cz.lo);
        float acc[C::NACC];
#pragma unroll
        for (int u = 0; u < C::NACC; ++u) acc[u] = 0.f;
        auto prim = [&](float4 r0, float4 r1) {
          const float PCx = r0.y + ACx, PCy = r0.z + ACy, PCz = r0.w + ACz;
          const float T = r0.x * fmaf(PCx, PCx, fmaf(PCy, PCy, PCz * PCz));
          float S[C::L + 1];
          boys_seeds_f32<C::L>(T, r1.x, r1.y, s_tabf, S);
          C::vrr(S, r0.y, r0.z, r0.w, PCx, PCy, PCz, r1.z, 2.0f * r1.z, 3.0f * r1.z, acc);
        };
        const int ppn = s_ppn[r];
        if (ppn <= kStage) {
#pragma unroll 2
          for (int q = 0; q < ppn; ++q) prim(rec[2 * q], rec[2 * q + 1]);
        } else {  // more primitive pairs than staged: global memory
          const float4* pp = a.prims_f32 + (size_t)s_ppo[r] * 2;
          for (int q = 0; q < ppn; ++q) prim(pp[2 * q], pp[2 * q + 1]);
        }
        float xi[NA * NB];
        C::hrr(acc, s_ab[r][0].x, s_ab[r][1].x, s_ab[r][2].x, xi);
#pragma unroll
        for (int d = 0; d < ND; ++d)
#pragma unroll
          for (int u = 0; u < NA; ++u)
#pragma unroll
            for (int v = 0; v < NB; ++v) ga[d][u] = fmaf(xi[u * NB + v], fb[d][v], ga[d][u]);
        if (sa != s_sb[r]) {
          const int colb = s_cb[r];
#pragma unroll
          for (int d = 0; d < ND; ++d)
#pragma unroll
            for (int v = 0; v < NB; ++v) {
              float g = 0.f;
#pragma unroll
              for (int u = 0; u < NA; ++u) g = fmaf(xi[u * NB + v], fa[d][u], g);
              gadd(d, colb + v, g);
            }
        }
      };
      if constexpr (RING) {
        // the warp's 32 points of every F column: 128 contiguous, 16-byte
        // aligned bytes (foff32, ldq and i0 are multiples of 128 floats, and
        // the columns are ldq >= i0 + 128 long)
        const float* Fw = a.ws32 + s_bd.foff32 + s_t.i0 + 32 * wid;
        // pair r into the next slot: its records (at most kStage primitive
        // pairs; longer contractions are read from global memory) and its
        // F_b columns, one bulk copy each, all on the slot's barrier.  The
        // slot was last read by this warp's lanes before the __syncwarp that
        // precedes every call.
        auto issue = [&](int r) {
          if (lane == 0) {
            const int sl = prod % kRing;
            uint64_t* bar = &s_full[wid][sl];
            const int ppn = s_ppn[r];
            const uint32_t rec_bytes = ppn <= kStage ? 32u * (uint32_t)ppn : 0u;
            fence_proxy_async_smem();
            mbar_expect_tx(bar, rec_bytes + ND * NB * 128);
            if (rec_bytes) bulk_copy(s_ring[wid][sl], a.prims_f32 + (size_t)s_ppo[r] * 2, rec_bytes, bar);
            float* fdst = reinterpret_cast<float*>(s_ring[wid][sl] + kRecF4);
            const int cb = s_cb[r];
#pragma unroll
            for (int d = 0; d < ND; ++d)
#pragma unroll
              for (int v = 0; v < NB; ++v)
                bulk_copy(fdst + (d * NB + v) * 32, Fw + d * dstr + (int64_t)(cb + v) * ldq, 128, bar);
          }
          ++prod;
        };
        for (int r = 0; r < min(nrun, kRing); ++r) issue(r);
        for (int r = 0; r < nrun; ++r) {
          const int sl = cons % kRing;
          const bool ok = __all_sync(0xffffffffu, mbar_wait(&s_full[wid][sl], (cons / kRing) & 1u, a.err,
                                                            kCopyWaitNs));
          ++cons;
          if (!ok) {
            // give up: no further work in this CTA; wait (bounded again) for
            // the copies still in flight into this warp's ring, then leave
            s_abort = 1;
            for (uint32_t q = cons - 1; q < prod; ++q)
              mbar_wait(&s_full[wid][q % kRing], (q / kRing) & 1u, nullptr, kCopyWaitNs);
            cons = prod;
            break;
          }
          if (active) {
            const float* fsl = reinterpret_cast<const float*>(s_ring[wid][sl] + kRecF4);
            float fb[ND][NB];
#pragma unroll
            for (int d = 0; d < ND; ++d)
#pragma unroll
              for (int v = 0; v < NB; ++v) fb[d][v] = fsl[(d * NB + v) * 32 + lane];
            compute(r, s_ring[wid][sl], fb);
          }
          __syncwarp();  // every lane is done with slot sl: it takes pair r + kRing
          if (r + kRing < nrun) issue(r + kRing);
        }
      } else {
        {  // the first pair's records
          const int n2 = min(s_ppn[0], kStage) * 2;
          const float4* src = a.prims_f32 + (size_t)s_ppo[0] * 2;
          if (lane < n2) s_pr[RING ? 0 : wid][0][lane] = src[lane];
          __syncwarp();
        }
        float fn[ND][NB];
#pragma unroll
        for (int d = 0; d < ND; ++d)
#pragma unroll
          for (int v = 0; v < NB; ++v) fn[d][v] = active ? F[d * dstr + (s_cb[0] + v) * ldq] : 0.f;
        for (int r = 0; r < nrun; ++r) {
          // the next pair's records and F are in flight while this pair computes
          float4 pre = make_float4(0.f, 0.f, 0.f, 0.f);
          int n2n = 0;
          if (r + 1 < nrun) {
            n2n = min(s_ppn[r + 1], kStage) * 2;
            const float4* src = a.prims_f32 + (size_t)s_ppo[r + 1] * 2;
            if (lane < n2n) pre = src[lane];
          }
          float fb[ND][NB];
#pragma unroll
          for (int d = 0; d < ND; ++d)
#pragma unroll
            for (int v = 0; v < NB; ++v) fb[d][v] = fn[d][v];
          if (active && r + 1 < nrun) {
            const int cn = s_cb[r + 1];
#pragma unroll
            for (int d = 0; d < ND; ++d)
#pragma unroll
              for (int v = 0; v < NB; ++v) fn[d][v] = F[d * dstr + (cn + v) * ldq];
          }
          if (active) compute(r, s_pr[RING ? 0 : wid][r & 1], fb);
          // every lane is past its reads of the other buffer (the previous
          // iteration's closing __syncwarp), so it can take the next records
          if (lane < n2n) s_pr[RING ? 0 : wid][(r + 1) & 1][lane] = pre;
          __syncwarp();
        }
      }
      if (active && cur >= 0) {
#pragma unroll
        for (int d = 0; d < ND; ++d)
#pragma unroll
          for (int u = 0; u < NA; ++u) gadd(d, cola + u, ga[d][u]);
      }
    }  // steps of the tile's list
  }
}

// ---------------------------------------------------------------- double-FP32 pairs (mixed form)

// Constants of the ds Boys evaluation as (hi, lo) float pairs, rounded at
// compile time: 1/m! for the e^x Taylor series, then 1/(2n+1).
struct DsConst {
  float hi, lo;
};
#define SNK_DS_C(v) {(float)(v), (float)((v) - (double)(float)(v))}
__constant__ DsConst c_ds_invfact[8] = {SNK_DS_C(1.0),         SNK_DS_C(1.0),         SNK_DS_C(1.0 / 2.0),
                                        SNK_DS_C(1.0 / 6.0),   SNK_DS_C(1.0 / 24.0),  SNK_DS_C(1.0 / 120.0),
                                        SNK_DS_C(1.0 / 720.0), SNK_DS_C(1.0 / 5040.0)};
__constant__ DsConst c_ds_inv_odd[kBoysLMax + 1] = {SNK_DS_C(1.0), SNK_DS_C(1.0 / 3.0), SNK_DS_C(1.0 / 5.0),
                                                    SNK_DS_C(1.0 / 7.0), SNK_DS_C(1.0 / 9.0)};
#undef SNK_DS_C

__device__ __forceinline__ ds ds_ld(const float2* p) {
  const float2 v = *p;
  return ds_make(v.x, v.y);
}

__device__ __forceinline__ ds ds_c(const DsConst& c) { return ds_make(c.hi, c.lo); }

// S_n = pref F_n(T), n = 0..L, in ds arithmetic: the FP64 method's 8-term
// Taylor expansion about the nearest node of the 0.1-spaced table (nodes
// rounded to ds-representable values, so T_k - T is exact to ds precision),
// the downward recursion with e^{-T} = e^{-T_k} e^{x}, and the asymptotic
// form above T = 50 with a ds reciprocal square root.
template <int L>
__device__ __forceinline__ void boys_seeds_ds(ds T, ds pref, ds pref_far, const float2* tab, ds* S) {
  if (T.hi < (float)kBoysTMax) {
    const int k = __float2int_rn(T.hi * (float)(1.0 / kBoysH));
    const float2* row = tab + k * kBoysCols;
    const ds x = ds_ld(row + kBoysCols - 1) - T;  // T_k - T, |x| <= 0.05
    ds f = ds_ld(row + 7);
#pragma unroll
    for (int m = 6; m >= 0; --m) f = fma(f, x, ds_ld(row + m));
    S[L] = pref * f;
    if (L > 0) {
      ds e = ds_c(c_ds_invfact[7]);
#pragma unroll
      for (int m = 6; m >= 0; --m) e = fma(e, x, ds_c(c_ds_invfact[m]));
      const ds pe = (pref * ds_ld(row + kBoysTerms)) * e;
      const ds T2 = ds_make(2.0f * T.hi, 2.0f * T.lo);
#pragma unroll
      for (int n = L - 1; n >= 0; --n) S[n] = fma(T2, S[n + 1], pe) * ds_c(c_ds_inv_odd[n]);
    }
  } else {
    const ds r = ds_rsqrt(T);
    S[0] = pref_far * r;
    if (L > 0) {
      const ds o = (r * r) * 0.5f;
#pragma unroll
      for (int n = 0; n < L; ++n) S[n + 1] = S[n] * (o * (float)(2 * n + 1));
    }
  }
}

// Contracted Xi_ab of one pair at the point c in ds arithmetic; the primitive
// pair data are the host-split (hi, lo) copies of PrimPair (12 pairs each).
template <int LA, int LB>
__device__ __forceinline__ void pair_xi_ds(const PairHdr& h, const float2* __restrict__ prims,
                                           const float2* __restrict__ ab, const float2* tab, ds cx, ds cy, ds cz,
                                           ds* xi) {
  using C = OsClass<LA, LB>;
  ds acc[C::NACC];
#pragma unroll
  for (int k = 0; k < C::NACC; ++k) acc[k] = ds_make(0.f, 0.f);
  for (int q = 0; q < h.pp_n; ++q) {
    const float2* pp = prims + (size_t)(h.pp_off + q) * 12;
    const ds zeta = ds_ld(pp);
    const ds PCx = ds_ld(pp + 1) - cx, PCy = ds_ld(pp + 2) - cy, PCz = ds_ld(pp + 3) - cz;
    const ds T = zeta * fma(PCx, PCx, fma(PCy, PCy, PCz * PCz));
    ds S[C::L + 1];
    boys_seeds_ds<C::L>(T, ds_ld(pp + 7), ds_ld(pp + 8), tab, S);
    C::vrr(S, ds_ld(pp + 4), ds_ld(pp + 5), ds_ld(pp + 6), PCx, PCy, PCz, ds_ld(pp + 9), ds_ld(pp + 10),
           ds_ld(pp + 11), acc);
  }
  C::hrr(acc, ds_ld(ab), ds_ld(ab + 1), ds_ld(ab + 2), xi);
}

// The FP64 lists of the mixed form in ds arithmetic: same tiles, tickets,
// contraction and FP64 G atomics as integral_kernel; F is read in FP64 and
// split, each G update is rounded to FP64 once.
template <int LA, int LB, int ND>
__global__ void __launch_bounds__(kIntThreads) integral_kernel_ds(IntegralArgs a) {
  using C = OsClass<LA, LB>;
  constexpr int NA = C::NA, NB = C::NB;
  extern __shared__ float2 s_tab2[];
  const float2* gtab = a.boys_ds + (size_t)C::L * kBoysRows * kBoysCols;
  for (int e = threadIdx.x; e < kBoysRows * kBoysCols; e += blockDim.x) s_tab2[e] = gtab[e];
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
    const int64_t ldq = bd.ldq, dstr = (int64_t)bd.ldq * bd.nS;
    const ds cx = ds_from(a.xyz[3 * (bd.p0 + i)]), cy = ds_from(a.xyz[3 * (bd.p0 + i) + 1]),
             cz = ds_from(a.xyz[3 * (bd.p0 + i) + 2]);
    const double* F = a.ws + bd.foff + i;
    double* G = a.ws + bd.goff + i;
    const int* cmap = a.colmap + bd.cm_off - bd.ms0;
    ds ga[ND][NA], fa[ND][NA];
    int cur = -1, cola = 0;
    for (int k = tile.k0; k < tile.k1; ++k) {
      const int p = a.pairlist[k];
      const PairHdr h = a.pairs[p];
      if (h.sa != cur) {
        if (cur >= 0) {
#pragma unroll
          for (int d = 0; d < ND; ++d)
#pragma unroll
            for (int u = 0; u < NA; ++u) atomicAdd(G + d * dstr + (cola + u) * ldq, ds_to(ga[d][u]));
        }
        cur = h.sa;
        cola = cmap[cur];
#pragma unroll
        for (int d = 0; d < ND; ++d)
#pragma unroll
          for (int u = 0; u < NA; ++u) {
            ga[d][u] = ds_make(0.f, 0.f);
            fa[d][u] = ds_from(F[d * dstr + (cola + u) * ldq]);
          }
      }
      const int colb = cmap[h.sb];
      if (cola < 0 || colb < 0) continue;  // cannot happen: the screen marks both shells of a kept pair
      ds fb[ND][NB];
#pragma unroll
      for (int d = 0; d < ND; ++d)
#pragma unroll
        for (int v = 0; v < NB; ++v) fb[d][v] = ds_from(F[d * dstr + (colb + v) * ldq]);
      ds xi[NA * NB];
      pair_xi_ds<LA, LB>(h, a.prims_ds, a.pair_ab + 4 * (size_t)p, s_tab2, cx, cy, cz, xi);
#pragma unroll
      for (int d = 0; d < ND; ++d)
#pragma unroll
        for (int u = 0; u < NA; ++u)
#pragma unroll
          for (int v = 0; v < NB; ++v) ga[d][u] = fma(xi[u * NB + v], fb[d][v], ga[d][u]);
      if (h.sa != h.sb) {
#pragma unroll
        for (int d = 0; d < ND; ++d)
#pragma unroll
          for (int v = 0; v < NB; ++v) {
            ds g = ds_make(0.f, 0.f);
#pragma unroll
            for (int u = 0; u < NA; ++u) g = fma(xi[u * NB + v], fa[d][u], g);
            atomicAdd(G + d * dstr + (colb + v) * ldq, ds_to(g));
          }
      }
    }
    if (cur >= 0) {
#pragma unroll
      for (int d = 0; d < ND; ++d)
#pragma unroll
        for (int u = 0; u < NA; ++u) atomicAdd(G + d * dstr + (cola + u) * ldq, ds_to(ga[d][u]));
    }
  }
}

// Training labels of the learned screen, from the plain FP64 integrals: for
// every list entry (batch j, pair ab) of the sampled batches, the sums over
// the batch's points of |dG_u(i)| max_nu |Phi_{nu i}|, dG_u the block's
// contribution to G row u of shell a (slots 0..5) or b (slots 6..11): an
// upper bound of the block's contribution to K-tilde row u.  Same tiles as
// integral_kernel.
template <int LA, int LB>
__global__ void __launch_bounds__(kIntThreads) label_kernel(IntegralArgs a, const int64_t* __restrict__ slot_base,
                                                            const int64_t* __restrict__ list_off,
                                                            const double* __restrict__ xm,
                                                            float* __restrict__ lab) {
  using C = OsClass<LA, LB>;
  constexpr int NA = C::NA, NB = C::NB;
  extern __shared__ double s_tab[];
  const double* gtab = a.boys + (size_t)C::L * kBoysRows * kBoysCols;
  for (int e = threadIdx.x; e < kBoysRows * kBoysCols; e += blockDim.x) s_tab[e] = gtab[e];
  __shared__ int s_tile;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(a.ticket, 1);
    __syncthreads();
    const int t = s_tile;
    __syncthreads();
    if (t >= a.n_tiles) break;
    const Tile tile = a.tiles[t];
    const BatchDesc bd = a.batches[tile.batch];
    const int i = tile.i0 + threadIdx.x;
    const bool active = i < bd.q;
    const int64_t ldq = bd.ldq;
    const double cx = active ? a.xyz[3 * (bd.p0 + i)] : 0.0, cy = active ? a.xyz[3 * (bd.p0 + i) + 1] : 0.0,
                 cz = active ? a.xyz[3 * (bd.p0 + i) + 2] : 0.0;
    const double* F = a.ws + bd.foff + (active ? i : 0);
    const int* cmap = a.colmap + bd.cm_off - bd.ms0;
    const int64_t s0 = slot_base[tile.batch] - list_off[(int64_t)tile.batch * kNumLists];
    for (int k = tile.k0; k < tile.k1; ++k) {
      const PairHdr h = a.pairs[a.pairlist[k]];
      const int cola = cmap[h.sa], colb = cmap[h.sb];
      float part[NA + NB];
#pragma unroll
      for (int u = 0; u < NA + NB; ++u) part[u] = 0.f;
      if (active && cola >= 0 && colb >= 0) {
        double xi[NA * NB], fa[NA], fb[NB];
#pragma unroll
        for (int u = 0; u < NA; ++u) fa[u] = F[(cola + u) * ldq];
#pragma unroll
        for (int v = 0; v < NB; ++v) fb[v] = F[(colb + v) * ldq];
        pair_xi<LA, LB>(h, a.prims, s_tab, cx, cy, cz, xi);
#pragma unroll
        for (int u = 0; u < NA; ++u) {
          double g = 0.0;
#pragma unroll
          for (int v = 0; v < NB; ++v) g = fma(xi[u * NB + v], fb[v], g);
          part[u] = (float)(fabs(g) * xm[bd.p0 + i]);
        }
        if (h.sa != h.sb) {
#pragma unroll
          for (int v = 0; v < NB; ++v) {
            double g = 0.0;
#pragma unroll
            for (int u = 0; u < NA; ++u) g = fma(xi[u * NB + v], fa[u], g);
            part[NA + v] = (float)(fabs(g) * xm[bd.p0 + i]);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < NA + NB; ++u) {
        float s = part[u];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0 && s > 0.f) atomicAdd(&lab[(s0 + k) * 12 + (u < NA ? u : 6 + (u - NA))], s);
      }
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

constexpr size_t kSmem64 = sizeof(double) * kBoysRows * kBoysCols;
constexpr size_t kSmem32 = sizeof(float) * kBoysRowsF * kBoysColsF;

// list < kNumClasses: FP64 kernel of that class; otherwise the FP32 kernel of
// class list - kNumClasses.
template <class K>
cudaError_t launch_kernel(K kernel, size_t smem, cudaStream_t st, const IntegralArgs& a, int grid) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kernel<<<grid, kIntThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <int LA, int LB, int ND>
cudaError_t launch_class_nd(cudaStream_t st, bool f32, const IntegralArgs& a, int grid) {
  if (f32) return launch_kernel(integral_kernel_f32<LA, LB, ND>, kSmem32, st, a, grid);
  if (a.hi_ds) return launch_kernel(integral_kernel_ds<LA, LB, ND>, kSmem64, st, a, grid);
  return launch_kernel(integral_kernel<LA, LB, ND>, kSmem64, st, a, grid);
}

template <int LA, int LB>
cudaError_t launch_class(cudaStream_t st, bool f32, const IntegralArgs& a, int grid) {
  return a.n_dens == 2 ? launch_class_nd<LA, LB, 2>(st, f32, a, grid) : launch_class_nd<LA, LB, 1>(st, f32, a, grid);
}

template <class K>
int ctas_for(K kernel, size_t smem, int num_sms) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kIntThreads, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  return per_sm * num_sms;
}

template <int LA, int LB, int ND>
int max_ctas_nd(bool f32, bool ds, int num_sms) {
  return f32  ? ctas_for(integral_kernel_f32<LA, LB, ND>, kSmem32, num_sms)
         : ds ? ctas_for(integral_kernel_ds<LA, LB, ND>, kSmem64, num_sms)
              : ctas_for(integral_kernel<LA, LB, ND>, kSmem64, num_sms);
}

template <int LA, int LB>
int max_ctas(bool f32, bool ds, int nd, int num_sms) {
  return nd == 2 ? max_ctas_nd<LA, LB, 2>(f32, ds, num_sms) : max_ctas_nd<LA, LB, 1>(f32, ds, num_sms);
}

}  // namespace

cudaError_t launch_integrals(cudaStream_t st, int list, const IntegralArgs& a, int grid_ctas) {
  if (a.n_tiles == 0) return cudaSuccess;
  const bool f32 = list >= kNumClasses;
  switch (list % kNumClasses) {
    case 0: return launch_class<0, 0>(st, f32, a, grid_ctas);
    case 1: return launch_class<1, 0>(st, f32, a, grid_ctas);
    case 2: return launch_class<1, 1>(st, f32, a, grid_ctas);
    case 3: return launch_class<2, 0>(st, f32, a, grid_ctas);
    case 4: return launch_class<2, 1>(st, f32, a, grid_ctas);
    case 5: return launch_class<2, 2>(st, f32, a, grid_ctas);
  }
  return cudaErrorInvalidValue;
}

int integral_max_ctas(int list, int num_sms, bool ds, int n_dens) {
  const bool f32 = list >= kNumClasses;
  switch (list % kNumClasses) {
    case 0: return max_ctas<0, 0>(f32, ds, n_dens, num_sms);
    case 1: return max_ctas<1, 0>(f32, ds, n_dens, num_sms);
    case 2: return max_ctas<1, 1>(f32, ds, n_dens, num_sms);
    case 3: return max_ctas<2, 0>(f32, ds, n_dens, num_sms);
    case 4: return max_ctas<2, 1>(f32, ds, n_dens, num_sms);
    case 5: return max_ctas<2, 2>(f32, ds, n_dens, num_sms);
  }
  return num_sms;
}

cudaError_t launch_labels(cudaStream_t st, int cls, const IntegralArgs& a, int grid, const int64_t* slot_base,
                          const int64_t* list_off, const double* xm, float* lab) {
  if (a.n_tiles == 0) return cudaSuccess;
#define SNK_LAB(A, B)                                                                                       \
  {                                                                                                         \
    cudaError_t e =                                                                                         \
        cudaFuncSetAttribute(label_kernel<A, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem64); \
    if (e != cudaSuccess) return e;                                                                         \
    label_kernel<A, B><<<grid, kIntThreads, kSmem64, st>>>(a, slot_base, list_off, xm, lab);              \
    break;                                                                                                  \
  }
  switch (cls) {
    case 0: SNK_LAB(0, 0)
    case 1: SNK_LAB(1, 0)
    case 2: SNK_LAB(1, 1)
    case 3: SNK_LAB(2, 0)
    case 4: SNK_LAB(2, 1)
    case 5: SNK_LAB(2, 2)
    default: return cudaErrorInvalidValue;
  }
#undef SNK_LAB
  return cudaGetLastError();
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
void class_flops(int cls, double* per_prim, double* per_pair) {
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
  *per_prim = 8.0 + boys + vrr;
  *per_pair = hrr + 2.0 * na * nb;
}

}  // namespace snk
