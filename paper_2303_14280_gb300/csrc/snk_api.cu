// C ABI of libsnk (include/snk.h): handle management, the density-dependent
// screen and the K build driver (Alg. 1 of the paper on one GPU: batches are
// processed in chunks whose intermediates X, F, G fit a preallocated device
// workspace; every chunk adds its contribution to one K-tilde accumulator).
//
// A handle holds one or several independent molecules.  Their batches share
// every launch: the screen, the products and the integral kernels run over
// the batches of all molecules at once, with P and K packed per molecule.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "snk_internal.h"

using namespace snk;

namespace {

// Device allocator of a handle: the caller's hook (snk_set_allocator) or, with
// alloc == nullptr, cudaMalloc / cudaFree.  Memory from the hook is handed
// back only after the handle's stream has drained, so a stream-ordered pool
// may reuse it at once.
struct Allocator {
  snk_alloc_fn alloc = nullptr;
  snk_free_fn free = nullptr;
  void* user = nullptr;
  const cudaStream_t* stream = nullptr;
};

// A device buffer that remembers how its block was allocated, so that it is
// always released the same way even after the handle's allocator changed.
template <class T>
struct DevBuf {
  using value_type = T;
  T* p = nullptr;
  size_t n = 0;
  const Allocator* al = nullptr;  // allocator for future blocks (nullptr: cudaMalloc)
  Allocator owner{};              // how p was allocated (owner.alloc == nullptr: cudaMalloc)
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) {
      if (owner.alloc) {
        if (owner.stream) cudaStreamSynchronize(*owner.stream);
        owner.free(p, owner.user);
      } else {
        cudaFree(p);
      }
    }
    p = nullptr;
    n = 0;
    owner = Allocator{};
  }
  // a new block of count elements from allocator a (or cudaMalloc), not yet owned
  static cudaError_t raw(const Allocator* a, size_t count, T** out) {
    const size_t bytes = sizeof(T) * std::max<size_t>(count, 1);
    *out = nullptr;
    if (a && a->alloc) {
      void* q = a->alloc(bytes, a->user);
      if (!q) return cudaErrorMemoryAllocation;
      if (reinterpret_cast<uintptr_t>(q) % 256 != 0) {  // the kernels rely on cudaMalloc's alignment
        a->free(q, a->user);
        return cudaErrorMisalignedAddress;
      }
      *out = static_cast<T*>(q);
      return cudaSuccess;
    }
    return cudaMalloc(out, bytes);
  }
  cudaError_t ensure(size_t count) {
    if (count <= n && p) return cudaSuccess;
    release();
    T* q = nullptr;
    cudaError_t e = raw(al, count, &q);
    if (e != cudaSuccess) return e;
    p = q;
    n = count;
    owner = (al && al->alloc) ? *al : Allocator{};
    return cudaSuccess;
  }
};

// pairs per integral tile for each class (cheap classes take longer runs);
// the autotuner replaces these per list
constexpr int kDefaultStep = 128;  // pairs staged per step of the FP32 kernel, before autotuning
constexpr int kRunCandidates[] = {2, 4, 8, 16, 32, 64, 128};
// per chunk: collocation, F operands, F high tier, F rest, integral lists, K operands, K high tier, K rest
constexpr int kPhaseEvents = 7 + kNumLists;

}  // namespace

struct snk_ctx {
  Setup s;
  snk_options opt;
  int device = 0, num_sms = 0;
  cudaStream_t stream = nullptr;
  Allocator alloc;  // device memory of every buffer below (snk_set_allocator)
  std::string err;
  int nbatch = 0;
  int64_t ws_budget = 0;
  int run[kNumLists];  // pairs per tile, per list

  // geometry (device)
  DevBuf<int> l, poff, nprim, foff, fshell, bshell, bshell_col, xfunc;
  DevBuf<double> center, exps, d, fcomp, xyz, w, boys, bound, qbound, bcenter, bradius, phit_f, phit_b;
  DevBuf<float> boys_f, boys_ds, prims_ds, pair_ab, pair_a, prims_f32;  // mixed form: FP32 and (hi, lo) copies
  DevBuf<PairHdr> pairs;
  DevBuf<PrimPair> prims;
  DevBuf<MolDesc> mols;
  int max_nf = 0, max_nb = 0;

  // learned screen
  DevBuf<float> mlp_w, shell_feat;
  DevBuf<unsigned char> keep;
  bool mlp_loaded = false;
  ScreenArgs sargs{};

  // density-dependent state
  bool have_density = false;
  int n_dens = 1;  // densities loaded (P, P2, Khat hold n_dens packed blocks)
  int ctas_nd = 0;  // density count the persistent grids (max_ctas) were sized for
  DevBuf<double> P, Pscr, ft, sym, K;  // Pscr: sum_d |P_d| for the screen of several densities
  DevBuf<unsigned long long> Khat;     // two words per entry (khat_add)
  DevBuf<float2> P2;  // (hi, lo) pairs of P for the double-FP32 GEMM
  DevBuf<int> counts, list, list2, sfunc, colmap, tickets;  // list2: rewrite target of the learned screen
  DevBuf<long long> ppcounts;
  DevBuf<unsigned char> sflag;
  DevBuf<signed char> codes;  // the screen's decision per (batch, pair)
  DevBuf<int64_t> code_off;
  DevBuf<int64_t> list_off, tstart;  // per (batch, list): first list entry, first tile
  DevBuf<BatchDesc> batch;
  DevBuf<Tile> tiles;
  DevBuf<double> ws;
  DevBuf<float> ws32;
  // tensor-core split products (SNK_GEMM_SPLIT): bf16 slice arena, split and product jobs, error flag
  DevBuf<uint8_t> arena;
  DevBuf<OzSplitJob> ozsplit;
  DevBuf<OzGemmJob> ozjobs;
  DevBuf<int> ozerr;
  // tile screen of the FP32 lists: per-tile column sums, per-list executed work
  DevBuf<float> tsum;
  DevBuf<unsigned long long> exec;
  std::vector<int> hcounts;
  std::vector<long long> hpp;
  std::vector<int64_t> hlist_off;
  std::vector<BatchDesc> hbatch;

  struct Chunk {
    int b0 = 0, b1 = 0;
    int64_t bytes = 0, xn = 0, goff = 0, gbytes = 0;
    int max_ldq = 0, max_nS = 0, max_nB = 0, max_nBshell = 0;
    int64_t tile_off[kNumLists] = {0}, tile_n[kNumLists] = {0};
    // SNK_GEMM_SPLIT: split jobs of the F and K phases, product jobs of F hi, F lo, K hi, K lo
    int ozs_off[2] = {0, 0}, ozs_n[2] = {0, 0}, ozs_rows[2] = {0, 0}, ozs_k[2] = {0, 0};
    int ozg_off[4] = {0, 0, 0, 0}, ozg_n[4] = {0, 0, 0, 0}, ozg_tiles[4] = {0, 0, 0, 0};
    int64_t arena_bytes = 0;
    int max_tiles = 0;  // 128-point tiles of the chunk's largest batch (tile screen)
  };
  std::vector<Chunk> chunks;
  int max_ctas[kNumLists] = {0};

  // exchange-correlation potential (snk_build_Vxc): its own batch descriptors
  // (X, grad X and F / Z of each batch in xcws), chunks, fixed-point V-hat and
  // E-hat, phase events
  // (with gemm = SPLIT the two products are tcgen05 split products: split and
  // product jobs of phase 0, F = X P, and phase 1, V-hat += Z^T X, per chunk)
  struct XcChunk {
    int b0 = 0, b1 = 0, max_ldq = 0, max_nB = 0, max_nBshell = 0;
    int s_off[2] = {0, 0}, s_n[2] = {0, 0}, s_rows[2] = {0, 0}, s_k[2] = {0, 0};
    int g_off[2] = {0, 0}, g_n[2] = {0, 0}, g_tiles[2] = {0, 0};
  };
  std::vector<XcChunk> xc_chunks;
  DevBuf<BatchDesc> xcbatch;
  DevBuf<double> xcws, xcE;
  DevBuf<unsigned long long> xchat;
  DevBuf<uint8_t> xcarena;
  DevBuf<OzSplitJob> xcsplit;
  DevBuf<OzGemmJob> xcjobs;
  std::vector<cudaEvent_t> xcev;
  bool xc_timed = false;
  double xc_gemm_flops = 0.0, xc_colloc_bytes = 0.0;

  // CUDA graph of the build (options.graph)
  cudaStream_t gstream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  double* gout = nullptr;
  bool graph_valid = false;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;

  // timing
  std::vector<cudaEvent_t> events;
  cudaEvent_t ev_screen0 = nullptr, ev_screen1 = nullptr;
  int64_t launches_density = 0, launches_build = 0;
  bool built = false, built_graph = false;
  snk_stats st;

  // every device buffer of the handle, for binding and moving them
  template <class F>
  void for_each_buffer(F f) {
    f(l), f(poff), f(nprim), f(foff), f(fshell), f(bshell), f(bshell_col), f(xfunc);
    f(center), f(exps), f(d), f(fcomp), f(xyz), f(w), f(boys), f(bound), f(qbound), f(bcenter), f(bradius);
    f(phit_f), f(phit_b);
    f(boys_f), f(boys_ds), f(prims_ds), f(pair_ab), f(pair_a), f(prims_f32);
    f(pairs), f(prims), f(mols), f(mlp_w), f(shell_feat), f(keep);
    f(P), f(Pscr), f(ft), f(sym), f(Khat), f(K), f(P2);
    f(counts), f(list), f(list2), f(sfunc), f(colmap), f(tickets), f(ppcounts), f(sflag), f(list_off), f(tstart);
    f(codes), f(code_off);
    f(batch), f(tiles), f(ws), f(ws32), f(arena), f(ozsplit), f(ozjobs), f(ozerr), f(tsum), f(exec);
    f(xcbatch), f(xcws), f(xcE), f(xchat), f(xcarena), f(xcsplit), f(xcjobs);
  }
  snk_ctx() {
    alloc.stream = &stream;
    for_each_buffer([this](auto& b) { b.al = &alloc; });
  }

  ~snk_ctx() {
    if (gstream) cudaStreamSynchronize(gstream);
    for (auto e : events) cudaEventDestroy(e);
    for (auto e : xcev) cudaEventDestroy(e);
    if (ev_screen0) cudaEventDestroy(ev_screen0);
    if (ev_screen1) cudaEventDestroy(ev_screen1);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (gexec) cudaGraphExecDestroy(gexec);
    if (gstream) cudaStreamDestroy(gstream);
  }
};

namespace {

int fail(snk_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(snk_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(c, e == cudaErrorMemoryAllocation ? SNK_ERR_OOM : SNK_ERR_CUDA, m);
}

#define SNK_CK(ctx, call)                                    \
  do {                                                       \
    cudaError_t _e = (call);                                 \
    if (_e != cudaSuccess) return cuda_fail(ctx, _e, #call); \
  } while (0)

template <class T>
cudaError_t upload(DevBuf<T>& b, const std::vector<T>& h, cudaStream_t st) {
  cudaError_t e = b.ensure(h.size());
  if (e != cudaSuccess || h.empty()) return e;
  return cudaMemcpyAsync(b.p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, st);
}

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

DeviceBasis dev_basis(snk_ctx* c) {
  DeviceBasis b;
  b.l = c->l.p;
  b.poff = c->poff.p;
  b.nprim = c->nprim.p;
  b.center = c->center.p;
  b.exps = c->exps.p;
  b.d = c->d.p;
  b.fcomp = c->fcomp.p;
  b.foff = c->foff.p;
  return b;
}

// geometry part of a batch descriptor (no workspace offsets)
BatchDesc geometry_desc(const Setup& s, int j) {
  BatchDesc b{};
  const Setup::Mol& m = s.mols[s.bmol[j]];
  b.p0 = s.bstart[j];
  b.q = (int)(s.bstart[j + 1] - s.bstart[j]);
  b.ldq = (int)round_up(std::max(b.q, 1), kLdqAlign);
  b.nB = s.bnf[j];
  b.xfunc_off = s.xfunc_off[j];
  b.bshell_off = s.bshell_off[j];
  b.nBshell = s.bshell_off[j + 1] - s.bshell_off[j];
  b.mol = s.bmol[j];
  b.ms0 = m.ms0;
  b.mf0 = m.mf0;
  b.nfm = m.nf;
  b.pk_off = m.pk_off;
  b.cm_off = s.cm_off[j];
  b.phf_off = s.phf_off[j];
  return b;
}

// Geometry-only screen maxima Phi-tilde and phi-tilde (Eq. exx_fmat_approx):
// collocate the batches chunk by chunk and reduce.
int geometry_screen(snk_ctx* c) {
  Setup& s = c->s;
  const int nb = c->nbatch;
  SNK_CK(c, c->phit_f.ensure((size_t)std::max<int64_t>(s.phf_total, 1)));
  SNK_CK(c, c->phit_b.ensure(std::max(nb, 1)));
  SNK_CK(c, cudaMemsetAsync(c->phit_f.p, 0, sizeof(double) * std::max<int64_t>(s.phf_total, 1), c->stream));
  SNK_CK(c, cudaMemsetAsync(c->phit_b.p, 0, sizeof(double) * std::max(nb, 1), c->stream));
  if (nb == 0) return SNK_OK;
  std::vector<BatchDesc> bd(nb);
  SNK_CK(c, c->batch.ensure(nb));
  int j = 0;
  while (j < nb) {
    int64_t off = 0;
    int j0 = j, max_ldq = 0, max_nBs = 0, max_nB = 0;
    while (j < nb) {
      BatchDesc b = geometry_desc(s, j);
      int64_t bytes = (int64_t)b.ldq * b.nB * 8;
      if (j > j0 && off * 8 + bytes > c->ws_budget) break;
      b.xoff = off;
      off += (int64_t)b.ldq * b.nB;
      bd[j] = b;
      max_ldq = std::max(max_ldq, b.ldq);
      max_nBs = std::max(max_nBs, b.nBshell);
      max_nB = std::max(max_nB, b.nB);
      ++j;
    }
    SNK_CK(c, c->ws.ensure((size_t)std::max<int64_t>(off, 1)));
    SNK_CK(c, cudaMemcpyAsync(c->batch.p + j0, bd.data() + j0, sizeof(BatchDesc) * (j - j0), cudaMemcpyHostToDevice,
                              c->stream));
    SNK_CK(c, launch_collocation(c->stream, c->batch.p + j0, j - j0, max_ldq, max_nBs, c->bshell.p, c->bshell_col.p,
                                 c->xyz.p, dev_basis(c), c->ws.p));
    SNK_CK(c, launch_screen_geom(c->stream, c->batch.p + j0, j - j0, max_nB, c->ws.p, c->w.p, c->xfunc.p,
                                 c->phit_f.p, c->phit_b.p + j0));
    SNK_CK(c, cudaStreamSynchronize(c->stream));
  }
  return SNK_OK;
}

int ensure_events(snk_ctx* c, size_t n) {
  while (c->events.size() < n) {
    cudaEvent_t e;
    SNK_CK(c, cudaEventCreate(&e));
    c->events.push_back(e);
  }
  return SNK_OK;
}

// Integral tiles (batch, run of pairs, 128-point slab) of every list of every
// chunk, written on the device: the host only computes where each (batch,
// list)'s tiles start (from the per-list counts it already holds), and
// gen_tiles writes them.  Within a (chunk, list) the batches go in
// descending order of their work -- primitive pairs x points, the cost
// measure W_j of Eq. (work_heuristic) extended by the list's pair counts --
// so that the persistent CTAs, which take tiles from a ticket in order, start
// on the largest batches and finish on the smallest (longest processing time
// first); a run's slabs stay consecutive.
int make_tiles(snk_ctx* c, cudaStream_t st) {
  const auto& bd = c->hbatch;
  const int nb = c->nbatch;
  std::vector<int64_t> tstart((size_t)std::max(nb, 1) * kNumLists, 0);
  int64_t tot = 0;
  std::vector<int> order;
  std::vector<double> cost;
  for (auto& ch : c->chunks)
    for (int k = 0; k < kNumLists; ++k) {
      ch.tile_off[k] = tot;
      const int run = c->run[k];
      if (run < 1 || run > 128)  // the FP32 kernel stages at most 128 pairs per step
        return fail(c, SNK_ERR_INVALID_ARG, "pairs per step outside 1..128");
      order.resize(ch.b1 - ch.b0);
      cost.resize(ch.b1 - ch.b0);
      for (int t = ch.b0; t < ch.b1; ++t) {
        order[t - ch.b0] = t;
        cost[t - ch.b0] = (double)c->hpp[(size_t)t * kNumLists + k] * bd[t].q;
      }
      std::stable_sort(order.begin(), order.end(),
                       [&](int x, int y) { return cost[x - ch.b0] > cost[y - ch.b0]; });
      for (int t : order) {
        const int64_t n = c->hcounts[(size_t)t * kNumLists + k];
        tstart[(size_t)t * kNumLists + k] = tot;
        tot += n > 0 ? (bd[t].q + kPointTile - 1) / kPointTile : 0;  // one tile per slab of points
      }
      ch.tile_n[k] = tot - ch.tile_off[k];
    }
  SNK_CK(c, c->tiles.ensure((size_t)std::max<int64_t>(tot, 1)));
  SNK_CK(c, upload(c->tstart, tstart, st));
  SNK_CK(c, launch_gen_tiles(st, nb, c->batch.p, c->counts.p, c->list_off.p, c->tstart.p, c->tiles.p));
  ++c->launches_density;
  return SNK_OK;
}

// Persistent-grid size of every list's integral kernel (resident CTAs per SM
// x SMs) for the kernels the options and the density count select.
void set_max_ctas(snk_ctx* c) {
  const bool ds = c->opt.precision == SNK_PREC_MIXED && c->opt.ds_integrals;
  for (int k = 0; k < kNumLists; ++k)
    c->max_ctas[k] = integral_max_ctas(k, c->num_sms, ds, c->n_dens);
  c->ctas_nd = c->n_dens;
}

int check_device_flags(snk_ctx* c);

// The tile screen runs for the FP32 lists of the mixed form when the products
// leave X and the FP32 copy of F in place (gemm FP64 or SPLIT).
bool tile_screen(const snk_ctx* c) {
  return c->opt.precision == SNK_PREC_MIXED && c->opt.eps_tile > 0.0 && c->opt.gemm != SNK_GEMM_DF32;
}

// Split and product jobs of the tensor-core GEMMs (SNK_GEMM_SPLIT) for every
// chunk: where each operand's slices go in the chunk's arena (the F phase and
// the K phase reuse the same arena), and the (batch, tier, density) products
// with their tile numbering.  Operands of a tier with no rows are left out.
int plan_tc(snk_ctx* c, double* tc_flops) {
  const auto& bd = c->hbatch;
  const int nd = c->n_dens;
  const int64_t pk = c->s.packed;
  const int S_store = std::max(c->opt.tc_slices_hi, c->opt.tc_slices_lo);
  std::vector<OzSplitJob> sj;
  std::vector<OzGemmJob> gj;
  *tc_flops = 0.0;
  for (auto& ch : c->chunks) {
    std::vector<OzGemmJob> g[4];
    for (int phase = 0; phase < 2; ++phase) {
      ch.ozs_off[phase] = (int)sj.size();
      int64_t cur = 0;
      int max_rows = 0, max_k = 0;
      auto add_split = [&](int mode, int R, int K, int ld, int r0, const BatchDesc& b, int64_t src) -> int64_t {
        OzSplitJob J{};
        J.mode = mode;
        J.R = R;
        J.K = K;
        J.S = S_store;
        J.ld = ld;
        J.r0 = r0;
        J.sf_off = b.sfunc_off;
        J.xf_off = b.xfunc_off;
        J.src_off = src;
        J.dst_off = cur;
        sj.push_back(J);
        max_rows = std::max(max_rows, R);
        max_k = std::max(max_k, K);
        const int64_t at = cur;
        cur += oz_operand_bytes(R, K, S_store);
        return at;
      };
      for (int t = ch.b0; t < ch.b1; ++t) {
        const BatchDesc& b = bd[t];
        const int hiS = b.nS_hi, loS = b.nS - b.nS_hi;
        if (b.q == 0 || b.nB == 0 || b.nS == 0) continue;
        const int64_t xs = phase == 0 ? add_split(0, b.q, b.nB, b.ldq, 0, b, b.xoff)    // X_j, rows = points
                                      : add_split(1, b.nB, b.q, b.ldq, 0, b, b.xoff);   // X_j, rows = functions
        for (int d = 0; d < nd; ++d) {
          const int64_t dofs = (int64_t)d * b.ldq * b.nS;
          for (int tier = 0; tier < 2; ++tier) {
            const int rows = tier == 0 ? hiS : loS, r0 = tier == 0 ? 0 : hiS;
            if (rows == 0) continue;
            OzGemmJob G{};
            G.batch = t;
            G.Sa = G.Sb = S_store;
            G.c0 = r0;
            if (phase == 0) {  // F[:, S_j tier] = X_j P[B_j, S_j tier]
              const int64_t ps = add_split(2, rows, b.nB, b.nfm, r0, b, b.pk_off + d * pk);
              G.a_off = xs;
              G.b_off = ps;
              G.RTa = oz_row_tiles(b.q);
              G.RTb = oz_row_tiles(rows);
              G.KT = oz_k_tiles(b.nB);
              G.kind = 0;
              G.m_lim = b.ldq;
              G.n_lim = rows;
              G.out_off = b.foff + dofs;
              G.out_off32 = b.foff32 + dofs;
            } else {  // Kt[S_j tier, B_j] += G_j[:, S_j tier]^T X_j
              const int64_t gs = add_split(1, rows, b.q, b.ldq, r0, b, b.goff + dofs);
              G.a_off = gs;
              G.b_off = xs;
              G.RTa = oz_row_tiles(rows);
              G.RTb = oz_row_tiles(b.nB);
              G.KT = oz_k_tiles(b.q);
              G.kind = 1;
              G.m_lim = rows;
              G.n_lim = b.nB;
              G.out_off = b.pk_off + d * pk;
            }
            const int sl = tier == 0 ? c->opt.tc_slices_hi : c->opt.tc_slices_lo;
            const int products = sl * (sl + 1) / 2;
            *tc_flops += 2.0 * products * 128.0 * G.RTa * 128.0 * G.RTb * 32.0 * G.KT;
            g[phase * 2 + tier].push_back(G);
          }
        }
      }
      ch.ozs_n[phase] = (int)sj.size() - ch.ozs_off[phase];
      ch.ozs_rows[phase] = max_rows;
      ch.ozs_k[phase] = max_k;
      if (cur > ch.arena_bytes)
        return fail(c, SNK_ERR_INVALID_ARG, "internal: slice arena of a chunk smaller than its operands");
    }
    for (int k = 0; k < 4; ++k) {
      ch.ozg_off[k] = (int)gj.size();
      int tiles = 0;
      for (auto& G : g[k]) {
        G.tile0 = tiles;
        tiles += G.RTa * G.RTb;
        gj.push_back(G);
      }
      ch.ozg_n[k] = (int)g[k].size();
      ch.ozg_tiles[k] = tiles;
    }
  }
  if (sj.empty()) sj.push_back(OzSplitJob{});
  if (gj.empty()) gj.push_back(OzGemmJob{});
  SNK_CK(c, upload(c->ozsplit, sj, c->stream));
  SNK_CK(c, upload(c->ozjobs, gj, c->stream));
  SNK_CK(c, c->ozerr.ensure(1));
  SNK_CK(c, cudaMemsetAsync(c->ozerr.p, 0, sizeof(int), c->stream));
  return SNK_OK;
}

// Density-dependent part of set_density once P is on the device.
int screen_and_plan(snk_ctx* c) {
  if (int rc = check_device_flags(c)) return rc;  // a failure of an earlier asynchronous build
  Setup& s = c->s;
  const int nb = c->nbatch;
  const cudaStream_t st = c->stream;
  const bool mixed = c->opt.precision == SNK_PREC_MIXED;
  c->have_density = false;
  c->graph_valid = false;
  c->launches_density = 0;
  if (c->ctas_nd != c->n_dens) set_max_ctas(c);
  SNK_CK(c, cudaEventRecord(c->ev_screen0, st));
  // symmetry check of every molecule block
  SNK_CK(c, c->sym.ensure(2 * SNK_MAX_DENSITIES));
  SNK_CK(c, cudaMemsetAsync(c->sym.p, 0, 2 * SNK_MAX_DENSITIES * sizeof(double), st));
  for (int d = 0; d < c->n_dens; ++d) {
    SNK_CK(c, launch_symcheck(st, c->mols.p, s.n_mol, s.packed, c->P.p + (size_t)d * s.packed, c->sym.p + 2 * d));
    ++c->launches_density;
  }
  double hsym[2 * SNK_MAX_DENSITIES];
  SNK_CK(c, cudaMemcpyAsync(hsym, c->sym.p, sizeof(hsym), cudaMemcpyDeviceToHost, st));
  SNK_CK(c, cudaStreamSynchronize(st));
  for (int d = 0; d < c->n_dens; ++d)
    if (!(hsym[2 * d] <= 1e-12 * hsym[2 * d + 1]))
      return fail(c, std::isfinite(hsym[2 * d]) ? SNK_ERR_NOT_SYMMETRIC : SNK_ERR_UNSUPPORTED,
                  "density matrix " + std::to_string(d) + " is not symmetric (or not finite)");
  // the screen of several densities bounds them all with sum_d |P_d|
  const double* Pscreen = c->P.p;
  if (c->n_dens > 1) {
    SNK_CK(c, c->Pscr.ensure((size_t)std::max<int64_t>(s.packed, 1)));
    SNK_CK(c, launch_abs_sum(st, c->P.p, c->n_dens, s.packed, c->Pscr.p));
    ++c->launches_density;
    Pscreen = c->Pscr.p;
  }
  const int nbx = std::max(nb, 1);
  const size_t cmn = (size_t)std::max<int64_t>(s.cm_total, 1);
  // F-tilde and the pair screen, Eqs. (exx_fmat_approx), (sp_set)
  SNK_CK(c, c->ft.ensure(cmn));
  SNK_CK(c, c->counts.ensure((size_t)nbx * kNumLists));
  SNK_CK(c, c->ppcounts.ensure((size_t)nbx * kNumLists));
  SNK_CK(c, c->sflag.ensure(2 * cmn));  // shells of V_j, then shells of its high-tier pairs
  SNK_CK(c, cudaMemsetAsync(c->ft.p, 0, sizeof(double) * cmn, st));
  SNK_CK(c, cudaMemsetAsync(c->sflag.p, 0, 2 * cmn, st));
  const int screen = c->opt.screen == SNK_SCREEN_NONE ? SNK_SCREEN_NONE : SNK_SCREEN_LINK;
  // geometry descriptors for the screen kernels
  c->hbatch.assign(nbx, BatchDesc{});
  for (int j = 0; j < nb; ++j) c->hbatch[j] = geometry_desc(s, j);
  SNK_CK(c, upload(c->batch, c->hbatch, st));
  if (screen != SNK_SCREEN_NONE) {
    SNK_CK(c, launch_ftilde(st, c->mols.p, s.n_mol, c->max_nf, c->max_nb, c->batch.p, Pscreen, c->phit_f.p,
                            c->fshell.p, c->ft.p));
    ++c->launches_density;
  }
  ScreenArgs sa;
  sa.mols = c->mols.p;
  sa.batches = c->batch.p;
  sa.pairs = c->pairs.p;
  sa.bound = c->bound.p;
  sa.qbound = c->qbound.p;
  sa.shell_xyz = c->center.p;
  sa.bcenter = c->bcenter.p;
  sa.bradius = c->bradius.p;
  sa.ft_shell = c->ft.p;
  sa.phit_b = c->phit_b.p;
  sa.screen = screen;
  sa.distance = c->opt.distance_bound ? 1 : 0;
  sa.mixed = mixed ? 1 : 0;
  sa.eps_E = c->opt.eps_E;
  sa.eps_K = c->opt.eps_K;
  sa.fp32_bound = c->opt.fp32_bound;
  {  // one decision byte per (batch, pair of the batch's molecule)
    std::vector<int64_t> coff(nbx, 0);
    int64_t tot_codes = 0;
    for (int j = 0; j < nb; ++j) {
      coff[j] = tot_codes;
      const Setup::Mol& m = s.mols[s.bmol[j]];
      tot_codes += m.cr[kNumClasses] - m.cr[0];
    }
    SNK_CK(c, c->codes.ensure((size_t)std::max<int64_t>(tot_codes, 1)));
    SNK_CK(c, upload(c->code_off, coff, st));
  }
  sa.codes = c->codes.p;
  sa.code_off = c->code_off.p;
  SNK_CK(c, launch_pair_count(st, sa, nb, c->counts.p, c->ppcounts.p, c->sflag.p, (int64_t)cmn));
  ++c->launches_density;
  c->hcounts.assign((size_t)nbx * kNumLists, 0);
  c->hpp.assign((size_t)nbx * kNumLists, 0);
  std::vector<unsigned char> hflag(2 * cmn);
  SNK_CK(c, cudaMemcpyAsync(c->hcounts.data(), c->counts.p, sizeof(int) * nbx * kNumLists, cudaMemcpyDeviceToHost, st));
  SNK_CK(c, cudaMemcpyAsync(c->hpp.data(), c->ppcounts.p, sizeof(long long) * nbx * kNumLists, cudaMemcpyDeviceToHost,
                            st));
  SNK_CK(c, cudaMemcpyAsync(hflag.data(), c->sflag.p, 2 * cmn, cudaMemcpyDeviceToHost, st));
  SNK_CK(c, cudaStreamSynchronize(st));

  // pair lists: offsets, then the deterministic compaction pass
  c->hlist_off.assign((size_t)nbx * kNumLists + 1, 0);
  int64_t tot = 0;
  for (int j = 0; j < nb; ++j)
    for (int k = 0; k < kNumLists; ++k) {
      c->hlist_off[(size_t)j * kNumLists + k] = tot;
      tot += c->hcounts[(size_t)j * kNumLists + k];
    }
  c->hlist_off[(size_t)nb * kNumLists] = tot;
  if (tot > (int64_t)0x7fffffff)
    return fail(c, SNK_ERR_UNSUPPORTED, "more than 2^31 screened (batch, pair) entries: tighten the screen");
  SNK_CK(c, c->list.ensure((size_t)std::max<int64_t>(tot, 1)));
  SNK_CK(c, upload(c->list_off, c->hlist_off, st));
  SNK_CK(c, launch_pair_write(st, sa, nb, c->list_off.p, c->list.p));
  ++c->launches_density;
  c->sargs = sa;

  // learned screen on top of the rigorous lists: the MLP skips blocks whose
  // predicted contribution is below learned_skip and, in the mixed form,
  // moves high-tier blocks predicted below learned_fp32 to the FP32 lists;
  // the lists are rewritten into the second list buffer, which becomes current
  int64_t learned_skipped = 0;
  if (c->opt.screen == SNK_SCREEN_LEARNED && c->mlp_loaded && tot > 0) {
    SNK_CK(c, c->keep.ensure((size_t)tot));
    SNK_CK(c, c->list2.ensure((size_t)tot));
    SNK_CK(c, cudaMemsetAsync(c->keep.p, 1, (size_t)tot, st));
    const float fp32_log10 = mixed ? (float)c->opt.learned_fp32 : -1e30f;
    SNK_CK(c, launch_learned_filter(st, sa, nb, c->mlp_w.p, c->list.p, c->list2.p, c->list_off.p, c->counts.p,
                                    c->ppcounts.p, c->shell_feat.p, (float)c->opt.learned_skip, fp32_log10, c->keep.p,
                                    c->sflag.p + cmn));
    c->launches_density += 2;
    std::swap(c->list.p, c->list2.p);
    std::swap(c->list.n, c->list2.n);
    SNK_CK(c, cudaMemcpyAsync(c->hcounts.data(), c->counts.p, sizeof(int) * nbx * kNumLists, cudaMemcpyDeviceToHost,
                              st));
    SNK_CK(c, cudaMemcpyAsync(c->hpp.data(), c->ppcounts.p, sizeof(long long) * nbx * kNumLists,
                              cudaMemcpyDeviceToHost, st));
    SNK_CK(c, cudaMemcpyAsync(c->hlist_off.data(), c->list_off.p, sizeof(int64_t) * nbx * kNumLists,
                              cudaMemcpyDeviceToHost, st));
    SNK_CK(c, cudaMemcpyAsync(hflag.data() + cmn, c->sflag.p + cmn, cmn, cudaMemcpyDeviceToHost, st));
    SNK_CK(c, cudaStreamSynchronize(st));
    int64_t after = 0;
    for (int64_t x = 0; x < (int64_t)nb * kNumLists; ++x) after += c->hcounts[x];
    learned_skipped = tot - after;
  }

  // shells of V_j -> F / G columns (molecule-local function indices); with
  // the split GEMMs the shells of high-tier pairs come first, [0, nS_hi)
  const bool split = mixed && c->opt.gemm == SNK_GEMM_SPLIT;
  const bool tc = split;
  std::vector<int> hcolmap(cmn, -1), hsfunc;
  auto& bd = c->hbatch;
  c->chunks.clear();
  for (int j = 0; j < nb; ++j) {
    BatchDesc& b = bd[j];
    const Setup::Mol& m = s.mols[b.mol];
    b.sfunc_off = (int)hsfunc.size();
    int col = 0;
    for (int pass = split ? 0 : 1; pass < 2; ++pass) {
      for (int a = 0; a < m.ns; ++a) {
        const bool used = hflag[(size_t)b.cm_off + a] != 0;
        const bool hi = hflag[cmn + (size_t)b.cm_off + a] != 0;
        if (!used || (pass == 0 && !hi) || (pass == 1 && split && hi)) continue;
        hcolmap[(size_t)b.cm_off + a] = col;
        const int g = m.ms0 + a;
        for (int u = 0; u < ncart(s.l[g]); ++u) hsfunc.push_back(s.foff[g] - m.mf0 + u);
        col += ncart(s.l[g]);
      }
      if (pass == 0) b.nS_hi = col;
    }
    b.nS = col;
    if (!split) b.nS_hi = col;
  }
  // counts for the statistics: integrals and algorithmic flops per list
  double per_prim[kNumClasses], per_pair[kNumClasses];
  for (int k = 0; k < kNumClasses; ++k) class_flops(k, &per_prim[k], &per_pair[k]);
  double lint[kNumLists] = {0}, lflops[kNumLists] = {0}, gflops = 0.0, gflops_hi = 0.0, xbytes = 0.0;
  int64_t kept[2] = {0, 0}, pair_points = 0;
  double listed32 = 0.0;
  for (int j = 0; j < nb; ++j) {
    gflops += 4.0 * c->n_dens * bd[j].q * (double)bd[j].nB * bd[j].nS;
    gflops_hi += 4.0 * c->n_dens * bd[j].q * (double)bd[j].nB * bd[j].nS_hi;
    xbytes += 8.0 * bd[j].ldq * (double)bd[j].nB;
    for (int k = 0; k < kNumLists; ++k) {
      const int cls = k % kNumClasses;
      const int la = cls >= 3 ? 2 : (cls >= 1 ? 1 : 0), lb = cls - la * (la + 1) / 2;
      const double n = c->hcounts[(size_t)j * kNumLists + k], npp = (double)c->hpp[(size_t)j * kNumLists + k];
      lint[k] += n * bd[j].q * ncart(la) * ncart(lb);
      lflops[k] += (npp * per_prim[cls] + n * per_pair[cls]) * bd[j].q;
      kept[k >= kNumClasses] += (int64_t)n;
      pair_points += (int64_t)n * bd[j].q;
      if (k >= kNumClasses) listed32 += n * bd[j].q;
    }
  }
  SNK_CK(c, upload(c->colmap, hcolmap, st));
  if (hsfunc.empty()) hsfunc.push_back(0);
  SNK_CK(c, upload(c->sfunc, hsfunc, st));

  // chunks under the workspace budget (Alg. 1): X, F, G in doubles, plus the
  // FP32 copies of F and G in the mixed form
  int j = 0;
  int64_t need = 1, need32 = 1, need_arena = 0, need_tsum = 1;
  const int nd = c->n_dens;
  // slice-arena bytes of one batch for the F phase (X_j and P[S_j, B_j] per
  // density, split by tier) and the K phase (X_j and G_j rows per density)
  const int S_store = std::max(c->opt.tc_slices_hi, c->opt.tc_slices_lo);
  auto oz_bytes = [&](const BatchDesc& b, int phase) -> int64_t {
    const int hiS = b.nS_hi, loS = b.nS - b.nS_hi, S5 = S_store;
    if (phase == 0)
      return oz_operand_bytes(b.q, b.nB, S5) +
             (int64_t)nd * (oz_operand_bytes(hiS, b.nB, S5) + oz_operand_bytes(loS, b.nB, S5));
    return oz_operand_bytes(b.nB, b.q, S5) +
           (int64_t)nd * (oz_operand_bytes(hiS, b.q, S5) + oz_operand_bytes(loS, b.q, S5));
  };
  while (j < nb) {
    snk_ctx::Chunk ch;
    ch.b0 = j;
    int64_t xo = 0, fo = 0, af = 0, ak = 0;
    while (j < nb) {
      // F and G of density d at foff / goff + d ldq nS
      int64_t xs = (int64_t)bd[j].ldq * bd[j].nB, fs = (int64_t)nd * bd[j].ldq * bd[j].nS;
      int64_t bytes = (xo + xs + 2 * (fo + fs)) * 8 + (mixed ? (fo + fs) * 4 : 0);
      const int64_t ozf = tc ? oz_bytes(bd[j], 0) : 0, ozk = tc ? oz_bytes(bd[j], 1) : 0;
      bytes += std::max(af + ozf, ak + ozk);
      if (j > ch.b0 && bytes > c->ws_budget) break;
      xo += xs;
      fo += fs;
      af += ozf;
      ak += ozk;
      ++j;
    }
    ch.arena_bytes = std::max(af, ak);
    need_arena = std::max(need_arena, ch.arena_bytes);
    ch.b1 = j;
    int64_t xcur = 0, fcur = xo, gcur = xo + fo, f32cur = 0, scur = 0;
    ch.xn = xo;
    ch.goff = gcur;
    ch.gbytes = fo * 8;
    for (int t = ch.b0; t < ch.b1; ++t) {
      const int64_t fs = (int64_t)nd * bd[t].ldq * bd[t].nS;
      bd[t].xoff = xcur;
      xcur += (int64_t)bd[t].ldq * bd[t].nB;
      bd[t].foff = fcur;
      bd[t].goff = gcur;
      bd[t].foff32 = f32cur;
      bd[t].ssoff = scur;
      scur += (int64_t)(bd[t].ldq / kPointTile) * (bd[t].nS + 4);
      ch.max_tiles = std::max(ch.max_tiles, bd[t].ldq / kPointTile);
      fcur += fs;
      gcur += fs;
      f32cur += fs;
      ch.max_ldq = std::max(ch.max_ldq, bd[t].ldq);
      ch.max_nS = std::max(ch.max_nS, bd[t].nS);
      ch.max_nB = std::max(ch.max_nB, bd[t].nB);
      ch.max_nBshell = std::max(ch.max_nBshell, bd[t].nBshell);
    }
    ch.bytes = (xo + 2 * fo) * 8;
    need = std::max(need, xo + 2 * fo);
    need_tsum = std::max(need_tsum, scur);
    if (mixed) need32 = std::max(need32, fo);
    c->chunks.push_back(ch);
  }
  SNK_CK(c, c->ws.ensure((size_t)need));
  if (mixed) SNK_CK(c, c->ws32.ensure((size_t)need32));
  SNK_CK(c, upload(c->batch, bd, st));
  if (tile_screen(c)) SNK_CK(c, c->tsum.ensure((size_t)need_tsum));
  SNK_CK(c, c->exec.ensure(2 * kNumLists));
  SNK_CK(c, c->ozerr.ensure(1));  // device error flag of the products and the K accumulator
  SNK_CK(c, cudaMemsetAsync(c->ozerr.p, 0, sizeof(int), st));
  double tc_flops = 0.0;
  if (tc) {
    if (int rc = plan_tc(c, &tc_flops)) return rc;
    SNK_CK(c, c->arena.ensure((size_t)std::max<int64_t>(need_arena, 16)));
  }

  if (int rc = make_tiles(c, st)) return rc;
  SNK_CK(c, c->tickets.ensure(c->chunks.size() * kNumLists + 1));
  SNK_CK(c, c->Khat.ensure((size_t)std::max<int64_t>(2 * c->n_dens * s.packed, 2)));
  if (mixed && c->opt.gemm != SNK_GEMM_FP64)
    SNK_CK(c, c->P2.ensure((size_t)std::max<int64_t>(c->n_dens * s.packed, 1)));
  SNK_CK(c, cudaEventRecord(c->ev_screen1, st));
  SNK_CK(c, cudaStreamSynchronize(st));

  snk_stats& S = c->st;
  S.n_batches = nb;
  S.pairs_learned_skipped = learned_skipped;
  S.pairs_kept = kept[0] + kept[1];
  S.pairs_kept_fp32 = kept[1];
  S.pair_points = pair_points;
  S.integrals = S.integral_flops = S.integrals_fp32 = S.flops_fp32 = 0.0;
  for (int k = 0; k < kNumClasses; ++k) {
    S.integrals_class[k] = lint[k];
    S.flops_class[k] = lflops[k];
    S.integrals += lint[k] + lint[k + kNumClasses];
    S.integral_flops += lflops[k];
    S.integrals_fp32 += lint[k + kNumClasses];
    S.flops_fp32 += lflops[k + kNumClasses];
  }
  S.gemm_flops = gflops;
  S.gemm_flops_hi = gflops_hi;
  S.colloc_bytes = xbytes;
  S.gemm_tc_flops = tc_flops;
  S.pair_points_fp32_listed = listed32;
  S.pair_points_fp32 = listed32;
  S.n_chunks = (int64_t)c->chunks.size();
  S.workspace_bytes = (int64_t)(c->ws.n * 8 + c->ws32.n * 4);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev_screen0, c->ev_screen1);
  S.ms_screen = ms;
  c->have_density = true;
  c->built = false;
  return SNK_OK;
}

// The tensor-core products record a wait that ran out (1) or an operand
// outside the slice arena (2) in a device flag; read and clear it once the
// stream has drained.
int check_device_flags(snk_ctx* c) {
  if (!c->ozerr.p) return SNK_OK;
  int h = 0;
  SNK_CK(c, cudaMemcpyAsync(&h, c->ozerr.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  SNK_CK(c, cudaStreamSynchronize(c->stream));
  if (h == 0) return SNK_OK;
  SNK_CK(c, cudaMemsetAsync(c->ozerr.p, 0, sizeof(int), c->stream));
  SNK_CK(c, cudaStreamSynchronize(c->stream));
  if (h == 1) return fail(c, SNK_ERR_TIMEOUT, "a kernel gave up waiting on its copy or product pipeline");
  if (h == kErrKhatRange)
    return fail(c, SNK_ERR_UNSUPPORTED, "a contribution to K reached 2^30 or was not finite (density or basis out of range)");
  return fail(c, SNK_ERR_CUDA, "a tensor-core product kernel found an operand outside its slice arena");
}

IntegralArgs integral_args(snk_ctx* c, size_t ci, int k) {
  const auto& ch = c->chunks[ci];
  IntegralArgs a;
  a.tiles = c->tiles.p + ch.tile_off[k];
  a.n_tiles = (int)ch.tile_n[k];
  a.ticket = c->tickets.p + ci * kNumLists + k;
  a.batches = c->batch.p;
  a.pairlist = c->list.p;
  a.pairs = c->pairs.p;
  a.prims = c->prims.p;
  a.colmap = c->colmap.p;
  a.xyz = c->xyz.p;
  a.boys = c->boys.p;
  a.ws = c->ws.p;
  a.boys_f = c->boys_f.p;
  a.ws32 = c->ws32.p;
  a.bcenter = c->bcenter.p;
  a.boys_ds = reinterpret_cast<const float2*>(c->boys_ds.p);
  a.prims_ds = reinterpret_cast<const float2*>(c->prims_ds.p);
  a.pair_ab = reinterpret_cast<const float2*>(c->pair_ab.p);
  a.prims_f32 = reinterpret_cast<const float4*>(c->prims_f32.p);
  a.pair_a = reinterpret_cast<const float2*>(c->pair_a.p);
  a.hi_ds = (c->opt.precision == SNK_PREC_MIXED && c->opt.ds_integrals) ? 1 : 0;
  a.tsum = c->tsum.p;
  a.pbound = c->bound.p;
  a.qbound = c->qbound.p;
  a.shell_xyz = c->center.p;
  a.eps_tile = (k >= kNumClasses && tile_screen(c)) ? (float)c->opt.eps_tile : 0.f;
  a.exec = c->exec.p + 2 * k;
  a.n_dens = c->n_dens;
  a.run = c->run[k];
  a.err = c->ozerr.p;
  return a;
}

// The build on stream st; timing events only when `timed` (they are left out
// of a captured graph).
int enqueue_build(snk_ctx* c, cudaStream_t st, double* dK, bool timed) {
  Setup& s = c->s;
  const bool mixed = c->opt.precision == SNK_PREC_MIXED;
  const bool tc = mixed && c->opt.gemm == SNK_GEMM_SPLIT;  // the tensor-core split products
  const bool df32 = mixed && c->opt.gemm == SNK_GEMM_DF32;
  const int gmode = df32 ? 2 : 0;
  const int nd = c->n_dens;
  const int64_t pk = s.packed;
  int ev = 0;
  c->launches_build = 0;
  auto mark = [&]() -> cudaError_t { return timed ? cudaEventRecord(c->events[ev++], st) : cudaSuccess; };
  // one tensor-core product launch over a chunk's jobs of kind k (F hi, F lo, K hi, K lo)
  auto oz_gemm = [&](const snk_ctx::Chunk& ch, int k) -> cudaError_t {
    if (ch.ozg_tiles[k] == 0) return cudaSuccess;
    OzGemmArgs g;
    g.jobs = c->ozjobs.p + ch.ozg_off[k];
    g.n_jobs = ch.ozg_n[k];
    g.n_tiles = ch.ozg_tiles[k];
    g.arena = c->arena.p;
    g.arena_bytes = (int64_t)c->arena.n;
    g.batches = c->batch.p;
    g.w = c->w.p;
    g.fcomp = c->fcomp.p;
    g.sfunc = c->sfunc.p;
    g.xfunc = c->xfunc.p;
    g.ws = c->ws.p;
    g.ws32 = c->ws32.p;
    g.Khat = c->Khat.p;
    g.err = c->ozerr.p;
    ++c->launches_build;
    return launch_oz_gemm(st, (k & 1) ? c->opt.tc_slices_lo : c->opt.tc_slices_hi, g, c->num_sms);
  };
  auto oz_split = [&](const snk_ctx::Chunk& ch, int phase) -> cudaError_t {
    if (ch.ozs_n[phase] == 0) return cudaSuccess;
    ++c->launches_build;
    return launch_oz_split(st, c->ozsplit.p + ch.ozs_off[phase], ch.ozs_n[phase], ch.ozs_rows[phase],
                           ch.ozs_k[phase], c->ws.p, c->P.p, c->xfunc.p, c->sfunc.p, c->arena.p,
                           (int64_t)c->arena.n, c->ozerr.p);
  };
  SNK_CK(c, mark());
  SNK_CK(c, cudaMemsetAsync(c->Khat.p, 0, sizeof(unsigned long long) * 2 * (size_t)std::max<int64_t>(nd * pk, 1), st));
  if (df32) {  // P2 is allocated with the density (no allocation inside a graph capture)
    SNK_CK(c, launch_split_df32_copy(st, c->P.p, nd * pk, c->P2.p));
    ++c->launches_build;
  }
  SNK_CK(c, cudaMemsetAsync(c->tickets.p, 0, sizeof(int) * c->tickets.n, st));
  SNK_CK(c, cudaMemsetAsync(c->exec.p, 0, sizeof(unsigned long long) * c->exec.n, st));
  for (size_t ci = 0; ci < c->chunks.size(); ++ci) {
    const auto& ch = c->chunks[ci];
    const int nbc = ch.b1 - ch.b0;
    const BatchDesc* db = c->batch.p + ch.b0;
    // X_j, Eq. (collocation)
    SNK_CK(c, launch_collocation(st, db, nbc, ch.max_ldq, ch.max_nBshell, c->bshell.p, c->bshell_col.p, c->xyz.p,
                                 dev_basis(c), c->ws.p));
    ++c->launches_build;
    SNK_CK(c, mark());
    // operands of F_j = X_j P_d: bf16 slices of X_j and P[S_j, B_j], or X_j as (hi, lo) float pairs
    if (tc) {
      SNK_CK(c, oz_split(ch, 0));
    } else if (df32) {
      SNK_CK(c, launch_split_df32(st, c->ws.p, ch.xn));
      ++c->launches_build;
    }
    SNK_CK(c, mark());
    // F_j = X_j P_d (w and component factors folded in), Eq. (batch_local_exx): high tier, then the rest
    if (tc) {
      SNK_CK(c, oz_gemm(ch, 0));
    } else {
      for (int d = 0; d < nd; ++d) {
        SNK_CK(c, launch_fgemm(st, db, nbc, ch.max_ldq, ch.max_nS, c->P.p + d * pk, c->P2.p + d * pk, c->xfunc.p,
                               c->sfunc.p, c->fcomp.p, c->w.p, c->ws.p, mixed ? c->ws32.p : nullptr, gmode, d));
        ++c->launches_build;
      }
    }
    SNK_CK(c, mark());
    if (tc) SNK_CK(c, oz_gemm(ch, 1));
    if (tile_screen(c)) {  // per-tile column sums of the tile screen, from X and the FP32 F
      SNK_CK(c, launch_tile_sums(st, db, nbc, ch.max_tiles, c->ws.p, c->ws32.p, c->xyz.p, nd, c->tsum.p));
      ++c->launches_build;
    }
    SNK_CK(c, cudaMemsetAsync(c->ws.p + ch.goff, 0, ch.gbytes, st));
    SNK_CK(c, mark());
    // G_j, Eq. (gmat) with the 3c-CP integrals of App. A, list by list
    for (int k = 0; k < kNumLists; ++k) {
      IntegralArgs a = integral_args(c, ci, k);
      if (a.n_tiles > 0) {
        int grid = (int)std::min<int64_t>(c->max_ctas[k], a.n_tiles);
        SNK_CK(c, launch_integrals(st, k, a, grid));
        ++c->launches_build;
      }
      SNK_CK(c, mark());
    }
    // the operands of Kt_d += G_dj^T X_j, Eq. (usym_k)
    if (tc) {
      SNK_CK(c, oz_split(ch, 1));
    } else if (df32) {
      SNK_CK(c, launch_split_df32(st, c->ws.p + ch.goff, ch.gbytes / 8));
      ++c->launches_build;
    }
    SNK_CK(c, mark());
    if (tc) {
      SNK_CK(c, oz_gemm(ch, 2));
    } else {
      for (int d = 0; d < nd; ++d) {
        SNK_CK(c, launch_kgemm(st, db, nbc, ch.max_nS, ch.max_nB, c->xfunc.p, c->sfunc.p, c->ws.p,
                               c->Khat.p + 2 * d * pk, gmode, d, c->ozerr.p));
        ++c->launches_build;
      }
    }
    SNK_CK(c, mark());
    if (tc) SNK_CK(c, oz_gemm(ch, 3));
    SNK_CK(c, mark());
  }
  // K_d = (Kt_d + Kt_d^T) / 2 in every molecule block, Eq. (sn_k)
  for (int d = 0; d < nd; ++d) {
    SNK_CK(c, launch_finish(st, c->mols.p, s.n_mol, s.packed, c->Khat.p + 2 * d * pk, c->fcomp.p, dK + d * pk));
    ++c->launches_build;
  }
  SNK_CK(c, mark());
  return SNK_OK;
}

int build(snk_ctx* c, double* dK) {
  if (!c->have_density) return fail(c, SNK_ERR_BAD_STATE, "snk_build_K called before snk_set_density");
  if (!c->opt.graph || c->n_dens > 1) {
    if (int rc = ensure_events(c, c->chunks.size() * kPhaseEvents + 2)) return rc;
    if (int rc = enqueue_build(c, c->stream, dK, true)) return rc;
    c->built = true;
    c->built_graph = false;
    return SNK_OK;
  }
  // CUDA-graph form: capture the whole build once per plan and output buffer,
  // replay it afterwards; ordered after / before the caller's stream by events
  if (int rc = ensure_events(c, 2)) return rc;
  if (!c->gstream) SNK_CK(c, cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
  if (!c->ev_in) SNK_CK(c, cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
  if (!c->ev_out) SNK_CK(c, cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
  if (!c->graph_valid || c->gout != dK) {
    if (c->gexec) {
      cudaGraphExecDestroy(c->gexec);
      c->gexec = nullptr;
    }
    cudaGraph_t g = nullptr;
    SNK_CK(c, cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_build(c, c->gstream, dK, false);
    cudaError_t e = cudaStreamEndCapture(c->gstream, &g);
    if (rc != SNK_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&c->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
    c->graph_valid = true;
    c->gout = dK;
  }
  SNK_CK(c, cudaEventRecord(c->events[0], c->stream));
  SNK_CK(c, cudaEventRecord(c->ev_in, c->stream));
  SNK_CK(c, cudaStreamWaitEvent(c->gstream, c->ev_in, 0));
  SNK_CK(c, cudaGraphLaunch(c->gexec, c->gstream));
  SNK_CK(c, cudaEventRecord(c->ev_out, c->gstream));
  SNK_CK(c, cudaStreamWaitEvent(c->stream, c->ev_out, 0));
  SNK_CK(c, cudaEventRecord(c->events[1], c->stream));
  c->built = true;
  c->built_graph = true;
  return SNK_OK;
}

void collect_times(snk_ctx* c) {
  if (!c->built) return;
  auto el = [&](int a, int b) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->events[a], c->events[b]);
    return (double)ms;
  };
  snk_stats& st = c->st;
  st.kernel_launches = c->launches_density + c->launches_build;
  if (c->built_graph) {
    if (cudaEventSynchronize(c->events[1]) != cudaSuccess) return;
    st.ms_collocation = st.ms_fgemm = st.ms_integrals = st.ms_kgemm = st.ms_integrals_fp32 = st.ms_finish = 0.0;
    for (int k = 0; k < kNumClasses; ++k) st.ms_integrals_class[k] = 0.0;
    st.ms_build = el(0, 1);
    return;
  }
  const int last = (int)c->chunks.size() * kPhaseEvents + 1;  // the event after the finish kernel
  if (cudaEventSynchronize(c->events[last]) != cudaSuccess) return;
  st.ms_collocation = st.ms_fgemm = st.ms_integrals = st.ms_kgemm = st.ms_integrals_fp32 = 0.0;
  st.ms_gemm_split = st.ms_gemm_hi = st.ms_gemm_lo = 0.0;
  for (int k = 0; k < kNumClasses; ++k) st.ms_integrals_class[k] = st.ms_integrals_class_fp32[k] = 0.0;
  int ev = 0;
  for (size_t ci = 0; ci < c->chunks.size(); ++ci) {
    const int e0 = ev;  // previous boundary
    st.ms_collocation += el(e0, e0 + 1);
    const double fs = el(e0 + 1, e0 + 2), fh = el(e0 + 2, e0 + 3), fl = el(e0 + 3, e0 + 4);
    st.ms_fgemm += fs + fh + fl;
    for (int k = 0; k < kNumLists; ++k) {
      const double t = el(e0 + 4 + k, e0 + 5 + k);
      if (k < kNumClasses) {
        st.ms_integrals_class[k] += t;
        st.ms_integrals += t;
      } else {
        st.ms_integrals_class_fp32[k - kNumClasses] += t;
        st.ms_integrals_fp32 += t;
      }
    }
    const int e1 = e0 + 4 + kNumLists;
    const double ks = el(e1, e1 + 1), kh = el(e1 + 1, e1 + 2), kl = el(e1 + 2, e1 + 3);
    st.ms_kgemm += ks + kh + kl;
    st.ms_gemm_split += fs + ks;
    st.ms_gemm_hi += fh + kh;
    st.ms_gemm_lo += fl + kl;
    ev = e1 + 3;
  }
  st.ms_finish = el(ev, ev + 1);
  st.ms_build = el(0, ev + 1);
  // the FP32 lists' work as computed (after the tile screen)
  unsigned long long hx[2 * kNumLists];
  if (c->exec.p && cudaMemcpy(hx, c->exec.p, sizeof(hx), cudaMemcpyDeviceToHost) == cudaSuccess) {
    double pp = 0.0, fl = 0.0, in = 0.0;
    for (int k = kNumClasses; k < kNumLists; ++k) {
      double per_prim, per_pair;
      const int cls = k - kNumClasses;
      class_flops(cls, &per_prim, &per_pair);
      const int la = cls >= 3 ? 2 : (cls >= 1 ? 1 : 0), lb = cls - la * (la + 1) / 2;
      fl += (double)hx[2 * k] * per_prim + (double)hx[2 * k + 1] * per_pair;
      in += (double)hx[2 * k + 1] * ncart(la) * ncart(lb);
      pp += (double)hx[2 * k + 1];
    }
    st.pair_points_fp32 = pp;
    st.flops_fp32 = fl;
    st.integrals += in - st.integrals_fp32;
    st.integrals_fp32 = in;
  }
}

// Autotuner: for every FP32 list, time the list's kernel on the last chunk's
// tiles for each candidate step of staged pairs, keep the fastest (the other
// kernels read their pairs straight from the list and have no step).
// The workspace holds that chunk's X and F after a build; the kernel's G
// output is garbage afterwards, so the caller's next build recomputes it.
int autotune(snk_ctx* c, int32_t* runs_out) {
  if (!c->have_density) return fail(c, SNK_ERR_BAD_STATE, "snk_autotune called before snk_set_density");
  if (c->chunks.empty()) {
    if (runs_out)
      for (int k = 0; k < kNumLists; ++k) runs_out[k] = c->run[k];
    return SNK_OK;
  }
  const bool graph = c->opt.graph;
  c->opt.graph = 0;
  SNK_CK(c, c->K.ensure((size_t)std::max<int64_t>(c->n_dens * c->s.packed, 1)));
  int rc = build(c, c->K.p);
  c->opt.graph = graph;
  if (rc != SNK_OK) return rc;
  SNK_CK(c, cudaStreamSynchronize(c->stream));
  const size_t ci = c->chunks.size() - 1;
  cudaEvent_t e0, e1;
  SNK_CK(c, cudaEventCreate(&e0));
  SNK_CK(c, cudaEventCreate(&e1));
  for (int k = kNumClasses; k < kNumLists; ++k) {
    if (c->chunks[ci].tile_n[k] == 0) continue;
    double best = 1e300;
    int best_run = c->run[k];
    for (int r : kRunCandidates) {
      c->run[k] = r;
      if ((rc = [&]() -> int {
             if (int e = make_tiles(c, c->stream)) return e;
             double t = 1e300;
             for (int rep = 0; rep < 2; ++rep) {
               IntegralArgs a = integral_args(c, ci, k);
               SNK_CK(c, cudaMemsetAsync(a.ticket, 0, sizeof(int), c->stream));
               SNK_CK(c, cudaEventRecord(e0, c->stream));
               SNK_CK(c, launch_integrals(c->stream, k, a, (int)std::min<int64_t>(c->max_ctas[k], a.n_tiles)));
               SNK_CK(c, cudaEventRecord(e1, c->stream));
               SNK_CK(c, cudaEventSynchronize(e1));
               float ms = 0.f;
               cudaEventElapsedTime(&ms, e0, e1);
               t = std::min(t, (double)ms);
             }
             if (t < best) {
               best = t;
               best_run = r;
             }
             return SNK_OK;
           }()) != SNK_OK)
        break;
    }
    c->run[k] = best_run;
    if (rc != SNK_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != SNK_OK) return rc;
  if ((rc = make_tiles(c, c->stream)) != SNK_OK) return rc;
  SNK_CK(c, cudaStreamSynchronize(c->stream));
  c->graph_valid = false;
  if (runs_out)
    for (int k = 0; k < kNumLists; ++k) runs_out[k] = c->run[k];
  return SNK_OK;
}

int create(int n_mol, const snk_basis* bases, const snk_grid* grids, const snk_options* opt, snk_ctx** out) {
  if (!out) return SNK_ERR_INVALID_ARG;
  *out = nullptr;
  std::unique_ptr<snk_ctx> c(new (std::nothrow) snk_ctx());
  if (!c) return SNK_ERR_OOM;
  if (opt)
    c->opt = *opt;
  else
    snk_options_default(&c->opt);
  if (c->opt.screen < 0 || c->opt.screen > 2 || c->opt.precision < 0 || c->opt.precision > 1) return SNK_ERR_INVALID_ARG;
  if (c->opt.gemm < 0 || c->opt.gemm > 2 || c->opt.ds_integrals < 0 || c->opt.ds_integrals > 1 ||
      c->opt.tc_slices_hi < 3 || c->opt.tc_slices_hi > 6 ||
      c->opt.tc_slices_lo < 3 || c->opt.tc_slices_lo > 6 || !(c->opt.eps_tile >= 0.0))
    return SNK_ERR_INVALID_ARG;
  for (int k = 0; k < kNumLists; ++k) c->run[k] = kDefaultStep;
  int rc = build_setup(n_mol, bases, grids, &c->opt, &c->s, &c->err);
  if (rc != SNK_OK) return rc;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) return SNK_ERR_CUDA;
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) return SNK_ERR_CUDA;
  if (cudaEventCreate(&c->ev_screen0) != cudaSuccess || cudaEventCreate(&c->ev_screen1) != cudaSuccess)
    return SNK_ERR_CUDA;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return SNK_ERR_CUDA;
  c->ws_budget = c->opt.workspace_bytes > 0 ? c->opt.workspace_bytes : (int64_t)(fr / 2);
  Setup& s = c->s;
  c->nbatch = (int)s.bstart.size() - 1;
  if (c->nbatch > kKhatMaxBatches) return SNK_ERR_UNSUPPORTED;  // the K accumulator's low word would overflow
  // local X columns of the B_j shells
  s.bshell_col.resize(s.bshell.size());
  for (int j = 0; j < c->nbatch; ++j) {
    int col = 0;
    for (int t = s.bshell_off[j]; t < s.bshell_off[j + 1]; ++t) {
      s.bshell_col[t] = col;
      col += ncart(s.l[s.bshell[t]]);
    }
  }
  std::vector<MolDesc> hm(s.n_mol);
  for (int m = 0; m < s.n_mol; ++m) {
    const Setup::Mol& M = s.mols[m];
    MolDesc& d = hm[m];
    d = MolDesc{};
    d.pk_off = M.pk_off;
    d.nf = M.nf;
    d.ns = M.ns;
    d.ms0 = M.ms0;
    d.mf0 = M.mf0;
    d.mb0 = M.mb0;
    d.nb = M.nb;
    for (int k = 0; k <= kNumClasses; ++k) d.cr[k] = M.cr[k];
    c->max_nf = std::max(c->max_nf, M.nf);
    c->max_nb = std::max(c->max_nb, M.nb);
  }
  // per shell features of the learned screen: l/2, log10 of the smallest and
  // largest exponent / 3
  std::vector<float> sfeat(4 * (size_t)std::max(s.ns, 1), 0.f);
  for (int a = 0; a < s.ns; ++a) {
    double mn = 1e300, mx = 0.0;
    for (int k = s.poff[a]; k < s.poff[a + 1]; ++k) {
      mn = std::min(mn, s.exps[k]);
      mx = std::max(mx, s.exps[k]);
    }
    sfeat[4 * a] = 0.5f * s.l[a];
    sfeat[4 * a + 1] = (float)(std::log10(mn) / 3.0);
    sfeat[4 * a + 2] = (float)(std::log10(mx) / 3.0);
  }
  snk_ctx* cp = c.get();
  const cudaStream_t st = cp->stream;
  if ((rc = [&]() -> int {
         SNK_CK(cp, upload(cp->shell_feat, sfeat, st));
         SNK_CK(cp, upload(cp->l, s.l, st));
         SNK_CK(cp, upload(cp->poff, s.poff, st));
         SNK_CK(cp, upload(cp->nprim, s.nprim, st));
         SNK_CK(cp, upload(cp->foff, s.foff, st));
         SNK_CK(cp, upload(cp->fshell, s.fshell, st));
         SNK_CK(cp, upload(cp->center, s.center, st));
         SNK_CK(cp, upload(cp->exps, s.exps, st));
         SNK_CK(cp, upload(cp->d, s.d, st));
         SNK_CK(cp, upload(cp->fcomp, s.fcomp, st));
         SNK_CK(cp, upload(cp->pairs, s.pairs, st));
         SNK_CK(cp, upload(cp->prims, s.prims, st));
         SNK_CK(cp, upload(cp->bound, s.bound, st));
         SNK_CK(cp, upload(cp->qbound, s.qbound, st));
         SNK_CK(cp, upload(cp->bcenter, s.bcenter, st));
         SNK_CK(cp, upload(cp->bradius, s.bradius, st));
         SNK_CK(cp, upload(cp->boys_f, s.boys_f, st));
         if (cp->opt.precision == SNK_PREC_MIXED) {
           std::vector<float> pab(s.pairs.size() * 8, 0.0f), pa(s.pairs.size() * 8, 0.0f);
           for (size_t q = 0; q < s.pairs.size(); ++q) {
             const double v[3] = {s.pairs[q].ABx, s.pairs[q].ABy, s.pairs[q].ABz};
             const double* A = &s.center[3 * (size_t)s.pairs[q].sa];
             for (int m = 0; m < 3; ++m) {
               const float hh = (float)v[m];
               pab[q * 8 + 2 * m] = hh;
               pab[q * 8 + 2 * m + 1] = (float)(v[m] - (double)hh);
               const float ah = (float)A[m];
               pa[q * 8 + 2 * m] = ah;
               pa[q * 8 + 2 * m + 1] = (float)(A[m] - (double)ah);
             }
           }
           SNK_CK(cp, upload(cp->pair_ab, pab, st));
           SNK_CK(cp, upload(cp->pair_a, pa, st));
           std::vector<float> pds(s.prims.size() * 24);
           for (size_t q = 0; q < s.prims.size(); ++q) {
             const double* v = reinterpret_cast<const double*>(&s.prims[q]);
             for (int m = 0; m < 12; ++m) {
               const float h = (float)v[m];
               pds[q * 24 + 2 * m] = h;
               pds[q * 24 + 2 * m + 1] = (float)(v[m] - (double)h);
             }
           }
           SNK_CK(cp, upload(cp->prims_ds, pds, st));
           std::vector<float> pf(s.prims.size() * 8, 0.0f);
           for (size_t q = 0; q < s.prims.size(); ++q) {
             const PrimPair& P = s.prims[q];
             float* r = &pf[q * 8];
             r[0] = (float)P.zeta;
             r[1] = (float)P.PAx;
             r[2] = (float)P.PAy;
             r[3] = (float)P.PAz;
             r[4] = (float)P.pref;
             r[5] = (float)P.pref_far;
             r[6] = (float)P.k1;
             r[7] = (float)s.prim_rel[q];
           }
           SNK_CK(cp, upload(cp->prims_f32, pf, st));
           SNK_CK(cp, upload(cp->boys_ds, s.boys_ds, st));
         }
         SNK_CK(cp, upload(cp->xyz, s.xyz, st));
         SNK_CK(cp, upload(cp->w, s.w, st));
         SNK_CK(cp, upload(cp->bshell, s.bshell, st));
         SNK_CK(cp, upload(cp->bshell_col, s.bshell_col, st));
         SNK_CK(cp, upload(cp->xfunc, s.xfunc, st));
         SNK_CK(cp, upload(cp->boys, s.boys, st));
         SNK_CK(cp, upload(cp->mols, hm, st));
         SNK_CK(cp, cudaStreamSynchronize(st));
         return SNK_OK;
       }()) != SNK_OK)
    return rc;
  if ((rc = geometry_screen(cp)) != SNK_OK) return rc;
  set_max_ctas(cp);
  std::memset(&cp->st, 0, sizeof(cp->st));
  cp->st.n_points = s.npts;
  cp->st.n_batches = cp->nbatch;
  cp->st.n_shells = s.ns;
  cp->st.n_functions = s.nf;
  cp->st.n_pairs = (int64_t)s.pairs.size();
  *out = c.release();
  return SNK_OK;
}

}  // namespace

// One tensor-core product phase of a V^xc chunk (0: F = X P, 1: V-hat += Z^T
// X): the operands' bf16 slices into the V^xc arena, then the products.  The
// row lists of both products are B_j, so xfunc serves as the product kernels'
// sfunc (the chunk's descriptors carry sfunc_off = xfunc_off).
int xc_tc_product(snk_ctx* c, const snk_ctx::XcChunk& ch, int phase, unsigned long long* Vhat) {
  const cudaStream_t st = c->stream;
  SNK_CK(c, launch_oz_split(st, c->xcsplit.p + ch.s_off[phase], ch.s_n[phase], ch.s_rows[phase], ch.s_k[phase],
                            c->xcws.p, c->P.p, c->xfunc.p, c->xfunc.p, c->xcarena.p, (int64_t)c->xcarena.n,
                            c->ozerr.p));
  OzGemmArgs g;
  g.jobs = c->xcjobs.p + ch.g_off[phase];
  g.n_jobs = ch.g_n[phase];
  g.n_tiles = ch.g_tiles[phase];
  g.arena = c->xcarena.p;
  g.arena_bytes = (int64_t)c->xcarena.n;
  g.batches = c->xcbatch.p + ch.b0;
  g.w = c->w.p;
  g.fcomp = c->fcomp.p;
  g.sfunc = c->xfunc.p;
  g.xfunc = c->xfunc.p;
  g.ws = c->xcws.p;
  g.ws32 = nullptr;
  g.Khat = Vhat;
  g.err = c->ozerr.p;
  SNK_CK(c, launch_oz_gemm(st, c->opt.tc_slices_hi, g, c->num_sms));
  return SNK_OK;
}

// V^xc of the loaded density (Sec. II.C): per chunk of batches whose X, grad X
// and F / Z fit the workspace budget, Phi and grad Phi (Eq. collocation),
// F = X P[B_j, B_j] (Eq. fmat), the density, functional and Z (Eqs. den_grid,
// exc_grid, zmat), V-hat += Z^T X (Eq. vxc_num); then V = V-hat + V-hat^T.
int build_vxc(snk_ctx* c, int fn, double* dV, double* E_host) {
  if (fn < SNK_XC_LDA_X || fn > SNK_XC_PBE) return fail(c, SNK_ERR_INVALID_ARG, "unknown functional");
  if (!dV) return fail(c, SNK_ERR_INVALID_ARG, "NULL output");
  if (!c->have_density) return fail(c, SNK_ERR_BAD_STATE, "snk_build_Vxc called before snk_set_density");
  Setup& s = c->s;
  if (c->n_dens != 1) return fail(c, SNK_ERR_BAD_STATE, "several densities are loaded: load one for snk_build_Vxc");
  const int nb = c->nbatch;
  const int64_t pk = s.packed;
  const int nm = s.n_mol;
  const bool tc = c->opt.precision == SNK_PREC_MIXED && c->opt.gemm == SNK_GEMM_SPLIT;
  const int S = c->opt.tc_slices_hi;  // slices of both tensor-core products
  if (c->xc_chunks.empty() && nb > 0) {
    // chunk budget: half of what is free now (the exchange build's buffers are
    // already held), at most half of the handle's workspace budget
    size_t fr = 0, tot = 0;
    SNK_CK(c, cudaMemGetInfo(&fr, &tot));
    const int64_t budget = std::max<int64_t>(std::min<int64_t>(c->ws_budget / 2, (int64_t)(fr / 2)), 1ll << 26);
    std::vector<BatchDesc> bd(nb);
    std::vector<OzSplitJob> sj;
    std::vector<OzGemmJob> gj;
    int64_t off = 0, most = 0, arena_most = 0;
    double flops = 0.0, bytes = 0.0;
    // slice bytes of batch b in each phase (the phases reuse one arena)
    auto arena_of = [&](const BatchDesc& b, int phase) -> int64_t {
      if (!tc || b.q == 0 || b.nB == 0) return 0;
      return phase == 0 ? oz_operand_bytes(b.q, b.nB, S) + oz_operand_bytes(b.nB, b.nB, S)
                        : 2 * oz_operand_bytes(b.nB, b.q, S);
    };
    std::vector<snk_ctx::XcChunk> chunks;
    snk_ctx::XcChunk ch;
    int64_t a0 = 0, a1 = 0;  // the chunk's slice bytes per phase
    for (int j = 0; j < nb; ++j) {
      BatchDesc b = geometry_desc(s, j);
      b.sfunc_off = b.xfunc_off;  // the products' row lists are B_j too
      const int64_t blk = (int64_t)b.ldq * b.nB;
      const int64_t need = (off + 5 * blk) * 8 + std::max(a0 + arena_of(b, 0), a1 + arena_of(b, 1));
      if (j > ch.b0 && need > budget) {
        ch.b1 = j;
        chunks.push_back(ch);
        most = std::max(most, off);
        arena_most = std::max(arena_most, std::max(a0, a1));
        ch = snk_ctx::XcChunk();
        ch.b0 = j;
        off = a0 = a1 = 0;
      }
      b.xoff = off;
      b.foff = off + 4 * blk;
      off += 5 * blk;
      a0 += arena_of(b, 0);
      a1 += arena_of(b, 1);
      bd[j] = b;
      ch.max_ldq = std::max(ch.max_ldq, b.ldq);
      ch.max_nB = std::max(ch.max_nB, b.nB);
      ch.max_nBshell = std::max(ch.max_nBshell, b.nBshell);
      flops += 2.0 * b.ldq * b.nB * (double)b.nB + 2.0 * b.q * b.nB * (double)b.nB;
      bytes += 4.0 * 8.0 * blk;
    }
    ch.b1 = nb;
    chunks.push_back(ch);
    most = std::max(most, off);
    arena_most = std::max(arena_most, std::max(a0, a1));
    if (tc) {
      for (auto& C : chunks) {
        for (int phase = 0; phase < 2; ++phase) {
          C.s_off[phase] = (int)sj.size();
          C.g_off[phase] = (int)gj.size();
          int64_t cur = 0;
          int tiles = 0;
          auto add_split = [&](int mode, int R, int K, int ld, const BatchDesc& b, int64_t src) -> int64_t {
            OzSplitJob J{};
            J.mode = mode;
            J.R = R;
            J.K = K;
            J.S = S;
            J.ld = ld;
            J.r0 = 0;
            J.sf_off = b.xfunc_off;
            J.xf_off = b.xfunc_off;
            J.src_off = src;
            J.dst_off = cur;
            sj.push_back(J);
            C.s_rows[phase] = std::max(C.s_rows[phase], R);
            C.s_k[phase] = std::max(C.s_k[phase], K);
            const int64_t at = cur;
            cur += oz_operand_bytes(R, K, S);
            return at;
          };
          for (int t = C.b0; t < C.b1; ++t) {
            const BatchDesc& b = bd[t];
            if (b.q == 0 || b.nB == 0) continue;
            OzGemmJob G{};
            G.batch = t - C.b0;  // the launch's descriptors start at the chunk's first batch
            G.Sa = G.Sb = S;
            G.c0 = 0;
            if (phase == 0) {  // F = X_j P[B_j, B_j] (P symmetric: rows of P are its columns)
              G.a_off = add_split(0, b.q, b.nB, b.ldq, b, b.xoff);
              G.b_off = add_split(2, b.nB, b.nB, b.nfm, b, b.pk_off);
              G.RTa = oz_row_tiles(b.q);
              G.RTb = oz_row_tiles(b.nB);
              G.KT = oz_k_tiles(b.nB);
              G.kind = 3;
              G.m_lim = b.ldq;
              G.n_lim = b.nB;
              G.out_off = b.foff;
            } else {  // V-hat[B_j, B_j] += Z_j^T X_j
              G.a_off = add_split(1, b.nB, b.q, b.ldq, b, b.foff);
              G.b_off = add_split(1, b.nB, b.q, b.ldq, b, b.xoff);
              G.RTa = oz_row_tiles(b.nB);
              G.RTb = oz_row_tiles(b.nB);
              G.KT = oz_k_tiles(b.q);
              G.kind = 1;
              G.m_lim = b.nB;
              G.n_lim = b.nB;
              G.out_off = b.pk_off;
            }
            G.tile0 = tiles;
            tiles += G.RTa * G.RTb;
            gj.push_back(G);
          }
          C.s_n[phase] = (int)sj.size() - C.s_off[phase];
          C.g_n[phase] = (int)gj.size() - C.g_off[phase];
          C.g_tiles[phase] = tiles;
          if (cur > arena_most) return fail(c, SNK_ERR_INVALID_ARG, "internal: V^xc slice arena too small");
        }
      }
    }
    cudaError_t e = c->xcbatch.ensure(nb);
    if (e == cudaSuccess) e = c->xcws.ensure((size_t)std::max<int64_t>(most, 1));
    if (e == cudaSuccess && tc) e = c->xcarena.ensure((size_t)std::max<int64_t>(arena_most, 1));
    if (e == cudaSuccess && tc) e = c->xcsplit.ensure(std::max<size_t>(sj.size(), 1));
    if (e == cudaSuccess && tc) e = c->xcjobs.ensure(std::max<size_t>(gj.size(), 1));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->xcbatch.p, bd.data(), sizeof(BatchDesc) * nb, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && !sj.empty())
      e = cudaMemcpyAsync(c->xcsplit.p, sj.data(), sizeof(OzSplitJob) * sj.size(), cudaMemcpyHostToDevice,
                          c->stream);
    if (e == cudaSuccess && !gj.empty())
      e = cudaMemcpyAsync(c->xcjobs.p, gj.data(), sizeof(OzGemmJob) * gj.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // the host vectors are local
    if (e != cudaSuccess) {
      const int rc = cuda_fail(c, e, "snk_build_Vxc workspace");
      return rc == SNK_OK ? SNK_ERR_CUDA : rc;
    }
    c->xc_chunks = chunks;
    c->xc_gemm_flops = flops;
    c->xc_colloc_bytes = bytes;
  }
  const bool fresh_err = !c->ozerr.p;
  SNK_CK(c, c->ozerr.ensure(1));
  if (fresh_err) SNK_CK(c, cudaMemsetAsync(c->ozerr.p, 0, sizeof(int), c->stream));
  SNK_CK(c, c->xchat.ensure((size_t)(2 * pk + 2 * nm)));
  SNK_CK(c, c->xcE.ensure((size_t)std::max(nm, 1)));
  const size_t nev = 1 + 4 * c->xc_chunks.size();
  while (c->xcev.size() < nev) {
    cudaEvent_t ev;
    SNK_CK(c, cudaEventCreate(&ev));
    c->xcev.push_back(ev);
  }
  const cudaStream_t st = c->stream;
  const int mode = c->opt.precision == SNK_PREC_MIXED ? 2 : 0;
  unsigned long long* Vhat = c->xchat.p;
  unsigned long long* Ehat = c->xchat.p + 2 * pk;
  int ev = 0;
  SNK_CK(c, cudaMemsetAsync(c->xchat.p, 0, sizeof(unsigned long long) * (2 * pk + 2 * nm), st));
  SNK_CK(c, cudaEventRecord(c->xcev[ev++], st));
  for (const auto& ch : c->xc_chunks) {
    const BatchDesc* db = c->xcbatch.p + ch.b0;
    const int n = ch.b1 - ch.b0;
    SNK_CK(c, launch_xc_colloc(st, db, n, ch.max_ldq, ch.max_nBshell, c->bshell.p, c->bshell_col.p, c->xyz.p,
                               dev_basis(c), c->xcws.p));
    SNK_CK(c, cudaEventRecord(c->xcev[ev++], st));
    if (tc) {
      if (int rc = xc_tc_product(c, ch, 0, Vhat)) return rc;
    } else {
      SNK_CK(c, launch_xc_fgemm(st, db, n, ch.max_ldq, ch.max_nB, c->P.p, c->xfunc.p, c->xcws.p, mode));
    }
    SNK_CK(c, cudaEventRecord(c->xcev[ev++], st));
    SNK_CK(c, launch_xc_point(st, db, n, ch.max_ldq, c->w.p, fn, c->xcws.p, Ehat, c->ozerr.p));
    SNK_CK(c, cudaEventRecord(c->xcev[ev++], st));
    if (tc) {
      if (int rc = xc_tc_product(c, ch, 1, Vhat)) return rc;
    } else {
      SNK_CK(c, launch_xc_vgemm(st, db, n, ch.max_nB, c->xfunc.p, c->xcws.p, Vhat, mode, c->ozerr.p));
    }
    if (&ch == &c->xc_chunks.back()) SNK_CK(c, launch_xc_finish(st, c->mols.p, nm, pk, Vhat, Ehat, dV, c->xcE.p));
    SNK_CK(c, cudaEventRecord(c->xcev[ev++], st));
  }
  if (c->xc_chunks.empty()) SNK_CK(c, launch_xc_finish(st, c->mols.p, nm, pk, Vhat, Ehat, dV, c->xcE.p));
  c->xc_timed = !c->xc_chunks.empty();
  if (!E_host) return SNK_OK;
  SNK_CK(c, cudaMemcpyAsync(E_host, c->xcE.p, sizeof(double) * nm, cudaMemcpyDeviceToHost, st));
  SNK_CK(c, cudaStreamSynchronize(st));
  return check_device_flags(c);
}

// phase times of the last snk_build_Vxc (waits for its last event)
void collect_xc_times(snk_ctx* c) {
  snk_stats& st = c->st;
  st.xc_gemm_flops = c->xc_gemm_flops;
  st.xc_colloc_bytes = c->xc_colloc_bytes;
  if (!c->xc_timed) return;
  const size_t last = 4 * c->xc_chunks.size();
  if (cudaEventSynchronize(c->xcev[last]) != cudaSuccess) return;
  double t[4] = {0.0, 0.0, 0.0, 0.0};
  for (size_t k = 0; k < last; ++k) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->xcev[k], c->xcev[k + 1]);
    t[k % 4] += ms;
  }
  st.ms_xc_collocation = t[0];
  st.ms_xc_fgemm = t[1];
  st.ms_xc_point = t[2];
  st.ms_xc_vgemm = t[3];
}

extern "C" {

void snk_options_default(snk_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->eps_basis = 1e-12;
  o->eps_E = 1e-12;
  o->eps_K = 1e-12;
  o->batch_max = 4096;
  o->precision = SNK_PREC_FP64;
  o->screen = SNK_SCREEN_LINK;
  o->fp32_bound = 1e-6;
  o->workspace_bytes = 0;
  o->distance_bound = 1;
  o->gemm = SNK_GEMM_FP64;
  o->ds_integrals = 0;
  o->learned_fp32 = -99.0;
  o->graph = 0;
  o->learned_skip = -11.0;
  o->tc_slices_hi = 5;
  o->tc_slices_lo = 4;
  o->eps_tile = 0.0;
}

const char* snk_status_string(int status) {
  switch (status) {
    case SNK_OK: return "ok";
    case SNK_ERR_INVALID_ARG: return "invalid argument";
    case SNK_ERR_UNSUPPORTED: return "unsupported input";
    case SNK_ERR_NOT_SYMMETRIC: return "density matrix not symmetric";
    case SNK_ERR_BAD_STATE: return "bad call order";
    case SNK_ERR_OOM: return "out of memory";
    case SNK_ERR_CUDA: return "CUDA error";
    case SNK_ERR_TIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

int snk_create(const snk_basis* basis, const snk_grid* grid, const snk_options* opt, snk_ctx** out) {
  if (!basis || !grid) return SNK_ERR_INVALID_ARG;
  return create(1, basis, grid, opt, out);
}

int snk_create_batch(int32_t n_mol, const snk_basis* bases, const snk_grid* grids, const snk_options* opt,
                     snk_ctx** out) {
  if (n_mol < 1 || !bases || !grids) return SNK_ERR_INVALID_ARG;
  return create(n_mol, bases, grids, opt, out);
}

int snk_set_density(snk_ctx* c, const double* P) {
  if (!c) return SNK_ERR_INVALID_ARG;
  if (!P) return fail(c, SNK_ERR_INVALID_ARG, "NULL density");
  const size_t n = (size_t)c->s.packed;
  c->have_density = false;
  c->n_dens = 1;
  SNK_CK(c, c->P.ensure(std::max<size_t>(n, 1)));
  if (n) SNK_CK(c, cudaMemcpyAsync(c->P.p, P, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
  return screen_and_plan(c);
}

int snk_set_density_multi(snk_ctx* c, int32_t n_dens, const double* const* P) {
  if (!c) return SNK_ERR_INVALID_ARG;
  if (n_dens < 1 || n_dens > SNK_MAX_DENSITIES || !P)
    return fail(c, SNK_ERR_INVALID_ARG, "need 1.." + std::to_string(SNK_MAX_DENSITIES) + " densities");
  if (c->s.n_mol != 1) return fail(c, SNK_ERR_UNSUPPORTED, "several densities need a single-molecule handle");
  for (int d = 0; d < n_dens; ++d)
    if (!P[d]) return fail(c, SNK_ERR_INVALID_ARG, "NULL density " + std::to_string(d));
  const size_t n = (size_t)c->s.packed;
  c->have_density = false;
  c->n_dens = n_dens;
  SNK_CK(c, c->P.ensure(std::max<size_t>(n * n_dens, 1)));
  for (int d = 0; d < n_dens; ++d)
    if (n) SNK_CK(c, cudaMemcpyAsync(c->P.p + d * n, P[d], sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
  return screen_and_plan(c);
}

int snk_build_K_multi(snk_ctx* c, double* const* K) {
  if (!c) return SNK_ERR_INVALID_ARG;
  if (!K) return fail(c, SNK_ERR_INVALID_ARG, "NULL output list");
  for (int d = 0; d < c->n_dens; ++d)
    if (!K[d]) return fail(c, SNK_ERR_INVALID_ARG, "NULL output " + std::to_string(d));
  const size_t n = (size_t)c->s.packed;
  SNK_CK(c, c->K.ensure(std::max<size_t>(n * c->n_dens, 1)));
  int rc = build(c, c->K.p);
  if (rc != SNK_OK) return rc;
  for (int d = 0; d < c->n_dens; ++d)
    if (n) SNK_CK(c, cudaMemcpyAsync(K[d], c->K.p + d * n, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
  SNK_CK(c, cudaStreamSynchronize(c->stream));
  return check_device_flags(c);
}

int snk_set_density_device(snk_ctx* c, const double* dP) {
  if (!c) return SNK_ERR_INVALID_ARG;
  if (!dP) return fail(c, SNK_ERR_INVALID_ARG, "NULL density");
  const size_t n = (size_t)c->s.packed;
  c->have_density = false;
  c->n_dens = 1;
  SNK_CK(c, c->P.ensure(std::max<size_t>(n, 1)));
  if (n) SNK_CK(c, cudaMemcpyAsync(c->P.p, dP, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
  return screen_and_plan(c);
}

int snk_set_density_batch(snk_ctx* c, const double* const* P) {
  if (!c) return SNK_ERR_INVALID_ARG;
  if (!P) return fail(c, SNK_ERR_INVALID_ARG, "NULL density list");
  c->have_density = false;
  c->n_dens = 1;
  SNK_CK(c, c->P.ensure(std::max<size_t>((size_t)c->s.packed, 1)));
  for (int m = 0; m < c->s.n_mol; ++m) {
    if (!P[m]) return fail(c, SNK_ERR_INVALID_ARG, "NULL density for molecule " + std::to_string(m));
    const auto& M = c->s.mols[m];
    SNK_CK(c, cudaMemcpyAsync(c->P.p + M.pk_off, P[m], sizeof(double) * M.nf * M.nf, cudaMemcpyHostToDevice,
                              c->stream));
  }
  return screen_and_plan(c);
}

// The single-output builds write one packed K: several loaded densities need
// snk_build_K_multi.
int one_density(snk_ctx* c) {
  return c->n_dens == 1 ? SNK_OK
                        : fail(c, SNK_ERR_BAD_STATE, "several densities are loaded: use snk_build_K_multi");
}

int snk_build_K_device(snk_ctx* c, double* dK) {
  if (!c) return SNK_ERR_INVALID_ARG;
  if (!dK) return fail(c, SNK_ERR_INVALID_ARG, "NULL output");
  if (int rc = one_density(c)) return rc;
  return build(c, dK);
}

int snk_build_K(snk_ctx* c, double* K) {
  if (!c) return SNK_ERR_INVALID_ARG;
  if (!K) return fail(c, SNK_ERR_INVALID_ARG, "NULL output");
  if (int rc = one_density(c)) return rc;
  const size_t n = (size_t)c->s.packed;
  SNK_CK(c, c->K.ensure(std::max<size_t>(n, 1)));
  int rc = build(c, c->K.p);
  if (rc != SNK_OK) return rc;
  if (n) SNK_CK(c, cudaMemcpyAsync(K, c->K.p, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
  SNK_CK(c, cudaStreamSynchronize(c->stream));
  return check_device_flags(c);
}

int snk_build_Vxc_device(snk_ctx* c, int32_t functional, double* dV, double* E_xc) {
  if (!c) return SNK_ERR_INVALID_ARG;
  return build_vxc(c, functional, dV, E_xc);
}

int snk_build_Vxc(snk_ctx* c, int32_t functional, double* V, double* E_xc) {
  if (!c) return SNK_ERR_INVALID_ARG;
  if (!V) return fail(c, SNK_ERR_INVALID_ARG, "NULL output");
  const size_t n = (size_t)c->s.packed;
  SNK_CK(c, c->K.ensure(std::max<size_t>(n, 1)));
  std::vector<double> e((size_t)std::max(c->s.n_mol, 1), 0.0);
  int rc = build_vxc(c, functional, c->K.p, e.data());
  if (rc != SNK_OK) return rc;
  if (n) SNK_CK(c, cudaMemcpyAsync(V, c->K.p, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
  SNK_CK(c, cudaStreamSynchronize(c->stream));
  if (E_xc)
    for (int m = 0; m < c->s.n_mol; ++m) E_xc[m] = e[m];
  return SNK_OK;
}

int snk_build_K_batch(snk_ctx* c, double* const* K) {
  if (!c) return SNK_ERR_INVALID_ARG;
  if (int rc = one_density(c)) return rc;
  if (!K) return fail(c, SNK_ERR_INVALID_ARG, "NULL output list");
  for (int m = 0; m < c->s.n_mol; ++m)
    if (!K[m]) return fail(c, SNK_ERR_INVALID_ARG, "NULL output for molecule " + std::to_string(m));
  SNK_CK(c, c->K.ensure(std::max<size_t>((size_t)c->s.packed, 1)));
  int rc = build(c, c->K.p);
  if (rc != SNK_OK) return rc;
  for (int m = 0; m < c->s.n_mol; ++m) {
    const auto& M = c->s.mols[m];
    SNK_CK(c, cudaMemcpyAsync(K[m], c->K.p + M.pk_off, sizeof(double) * M.nf * M.nf, cudaMemcpyDeviceToHost,
                              c->stream));
  }
  SNK_CK(c, cudaStreamSynchronize(c->stream));
  return check_device_flags(c);
}

int snk_autotune(snk_ctx* c, int32_t* runs) {
  if (!c) return SNK_ERR_INVALID_ARG;
  return autotune(c, runs);
}

int snk_set_stream(snk_ctx* c, void* stream) {
  if (!c) return SNK_ERR_INVALID_ARG;
  c->stream = (cudaStream_t)stream;
  return SNK_OK;
}

int snk_set_allocator(snk_ctx* c, snk_alloc_fn alloc, snk_free_fn free_fn, void* user) {
  if (!c) return SNK_ERR_INVALID_ARG;
  if ((alloc == nullptr) != (free_fn == nullptr))
    return fail(c, SNK_ERR_INVALID_ARG, "snk_set_allocator: alloc and free must both be set or both be NULL");
  SNK_CK(c, cudaStreamSynchronize(c->stream));
  if (c->gstream) SNK_CK(c, cudaStreamSynchronize(c->gstream));
  Allocator nal;
  nal.alloc = alloc;
  nal.free = alloc ? free_fn : nullptr;
  nal.user = alloc ? user : nullptr;
  nal.stream = &c->stream;
  // move every existing buffer: first all new blocks (all or none), then the copies
  std::vector<std::pair<void*, size_t>> fresh;
  cudaError_t err = cudaSuccess;
  c->for_each_buffer([&](auto& b) {
    if (err != cudaSuccess || !b.p) return;
    typename std::remove_reference<decltype(b)>::type::value_type* q = nullptr;
    err = std::remove_reference<decltype(b)>::type::raw(&nal, b.n, &q);
    if (err == cudaSuccess) fresh.emplace_back(q, sizeof(*q) * b.n);
  });
  if (err != cudaSuccess) {
    for (auto& f : fresh) {
      if (nal.alloc)
        nal.free(f.first, nal.user);
      else
        cudaFree(f.first);
    }
    return cuda_fail(c, err, "snk_set_allocator: moving the handle's buffers");
  }
  size_t k = 0;
  c->for_each_buffer([&](auto& b) {
    if (err != cudaSuccess || !b.p) return;
    auto* q = static_cast<typename std::remove_reference<decltype(b)>::type::value_type*>(fresh[k++].first);
    err = cudaMemcpyAsync(q, b.p, sizeof(*q) * b.n, cudaMemcpyDeviceToDevice, c->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
    const size_t n = b.n;
    b.release();
    b.p = q;
    b.n = n;
    b.owner = nal.alloc ? nal : Allocator{};
  });
  c->alloc = nal;
  // captured graphs and the screen arguments hold the old addresses
  if (c->gexec) {
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  c->graph_valid = false;
  c->have_density = false;
  c->built = false;
  if (err != cudaSuccess) return cuda_fail(c, err, "snk_set_allocator: copying the handle's buffers");
  return SNK_OK;
}

int snk_get_stats(const snk_ctx* c, snk_stats* out) {
  if (!c || !out) return SNK_ERR_INVALID_ARG;
  snk_ctx* m = const_cast<snk_ctx*>(c);
  collect_times(m);
  collect_xc_times(m);
  *out = m->st;
  return SNK_OK;
}

int64_t snk_n_functions(const snk_ctx* c) { return c ? c->s.nf : -1; }

int32_t snk_n_molecules(const snk_ctx* c) { return c ? c->s.n_mol : -1; }

int64_t snk_molecule_functions(const snk_ctx* c, int32_t m) {
  if (!c || m < 0 || m >= c->s.n_mol) return -1;
  return c->s.mols[m].nf;
}

const char* snk_last_error(const snk_ctx* c) { return c ? c->err.c_str() : "NULL handle"; }

void snk_destroy(snk_ctx* c) { delete c; }

int snk_debug_boys(int64_t n, const double* T, int nmax, double* out) {
  if (n < 0 || (n > 0 && (!T || !out)) || nmax < 0 || nmax > kBoysLMax) return SNK_ERR_INVALID_ARG;
  if (n == 0) return SNK_OK;
  // the same table the integral kernel uses
  Setup tab;
  build_boys_tables(&tab);
  DevBuf<double> dtab, dT, dout;
  if (dtab.ensure(tab.boys.size()) || dT.ensure(n) || dout.ensure((size_t)n * (nmax + 1))) return SNK_ERR_OOM;
  if (cudaMemcpy(dtab.p, tab.boys.data(), sizeof(double) * tab.boys.size(), cudaMemcpyHostToDevice) ||
      cudaMemcpy(dT.p, T, sizeof(double) * n, cudaMemcpyHostToDevice))
    return SNK_ERR_CUDA;
  if (launch_debug_boys(0, dtab.p, n, dT.p, nmax, dout.p) != cudaSuccess) return SNK_ERR_CUDA;
  if (cudaMemcpy(out, dout.p, sizeof(double) * n * (nmax + 1), cudaMemcpyDeviceToHost)) return SNK_ERR_CUDA;
  return SNK_OK;
}

}  // extern "C"

namespace {

// pair id of the shells sa, sb (global indices) or -1 (dropped, or different molecules)
int pair_id(const Setup& s, int sa, int sb) {
  for (const auto& M : s.mols)
    if (sa >= M.ms0 && sa < M.ms0 + M.ns) {
      if (sb < M.ms0 || sb >= M.ms0 + M.ns) return -1;
      return s.pair_index[(size_t)M.pi_off + (size_t)(sa - M.ms0) * M.ns + (sb - M.ms0)];
    }
  return -1;
}

}  // namespace

extern "C" {

int snk_debug_shell_A(snk_ctx* c, int32_t sa, int32_t sb, int64_t n, const double* xyz, double* out) {
  if (!c) return SNK_ERR_INVALID_ARG;
  Setup& s = c->s;
  if (sa < 0 || sb < 0 || sa >= s.ns || sb >= s.ns || n < 0 || (n > 0 && (!xyz || !out)))
    return fail(c, SNK_ERR_INVALID_ARG, "bad shell index or buffer");
  const int na = ncart(s.l[sa]), nb = ncart(s.l[sb]);
  const int p = pair_id(s, sa, sb);
  if (n == 0) return SNK_OK;
  if (p < 0) {
    std::fill(out, out + (size_t)n * na * nb, 0.0);
    return SNK_OK;
  }
  const PairHdr& h = s.pairs[p];
  const int ca = ncart(s.l[h.sa]), cb = ncart(s.l[h.sb]);
  DevBuf<double> dxyz, dxi;
  SNK_CK(c, dxyz.ensure(3 * n));
  SNK_CK(c, dxi.ensure((size_t)n * ca * cb));
  SNK_CK(c, cudaMemcpyAsync(dxyz.p, xyz, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, c->stream));
  SNK_CK(c, launch_debug_A(c->stream, s.pair_class[p], c->pairs.p + p, c->prims.p, c->boys.p, n, dxyz.p, dxi.p));
  std::vector<double> xi((size_t)n * ca * cb);
  SNK_CK(c, cudaMemcpyAsync(xi.data(), dxi.p, sizeof(double) * xi.size(), cudaMemcpyDeviceToHost, c->stream));
  SNK_CK(c, cudaStreamSynchronize(c->stream));
  const bool swap = h.sa != sa;
  for (int64_t i = 0; i < n; ++i)
    for (int u = 0; u < na; ++u)
      for (int v = 0; v < nb; ++v) {
        double x = swap ? xi[(size_t)i * ca * cb + v * cb + u] : xi[(size_t)i * ca * cb + u * cb + v];
        out[(size_t)i * na * nb + u * nb + v] = x * s.fcomp[s.foff[sa] + u] * s.fcomp[s.foff[sb] + v];
      }
  return SNK_OK;
}

int snk_debug_wait_timeout(snk_ctx* c, int64_t limit_ns) {
  if (!c) return SNK_ERR_INVALID_ARG;
  if (limit_ns < 1 || limit_ns > 2000000000LL) return fail(c, SNK_ERR_INVALID_ARG, "limit_ns outside 1..2e9");
  SNK_CK(c, c->ozerr.ensure(1));
  SNK_CK(c, cudaMemsetAsync(c->ozerr.p, 0, sizeof(int), c->stream));
  SNK_CK(c, launch_wait_probe(c->stream, c->ozerr.p, (unsigned long long)limit_ns));
  return check_device_flags(c);
}

int snk_debug_tc_gemm(int32_t M, int32_t N, int32_t K, const double* A, const double* B, int32_t slices,
                      double* C) {
  if (M < 0 || N < 0 || K < 0 || slices < 3 || slices > 6 || (M * (int64_t)K > 0 && !A) ||
      (N * (int64_t)K > 0 && !B) || (M * (int64_t)N > 0 && !C))
    return SNK_ERR_INVALID_ARG;
  if (M == 0 || N == 0) return SNK_OK;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SNK_ERR_CUDA;
  const int64_t a_bytes = oz_operand_bytes(M, K, slices), b_bytes = oz_operand_bytes(N, K, slices);
  DevBuf<double> src, out;
  DevBuf<uint8_t> arena;
  DevBuf<OzSplitJob> sj;
  DevBuf<OzGemmJob> gj;
  DevBuf<int> err;
  if (src.ensure((size_t)(M + N) * std::max(K, 1)) || out.ensure((size_t)M * N) ||
      arena.ensure((size_t)(a_bytes + b_bytes + 16)) || sj.ensure(2) || gj.ensure(1) || err.ensure(1))
    return SNK_ERR_OOM;
  OzSplitJob h[2] = {};
  for (int i = 0; i < 2; ++i) {
    h[i].mode = 1;
    h[i].R = i == 0 ? M : N;
    h[i].K = K;
    h[i].S = slices;
    h[i].ld = K;
    h[i].src_off = i == 0 ? 0 : (int64_t)M * K;
    h[i].dst_off = i == 0 ? 0 : a_bytes;
  }
  OzGemmJob g{};
  g.a_off = 0;
  g.b_off = a_bytes;
  g.RTa = oz_row_tiles(M);
  g.RTb = oz_row_tiles(N);
  g.KT = oz_k_tiles(K);
  g.Sa = g.Sb = slices;
  g.kind = 2;
  g.m_lim = M;
  g.n_lim = N;
  g.ldc = N;
  if (cudaMemcpy(src.p, A, sizeof(double) * M * K, cudaMemcpyHostToDevice) ||
      cudaMemcpy(src.p + (int64_t)M * K, B, sizeof(double) * N * K, cudaMemcpyHostToDevice) ||
      cudaMemcpy(sj.p, h, sizeof(h), cudaMemcpyHostToDevice) ||
      cudaMemcpy(gj.p, &g, sizeof(g), cudaMemcpyHostToDevice) || cudaMemset(err.p, 0, sizeof(int)) ||
      cudaMemset(out.p, 0, sizeof(double) * M * N))
    return SNK_ERR_CUDA;
  if (K > 0) {
    if (launch_oz_split(0, sj.p, 2, std::max(M, N), K, src.p, src.p, nullptr, nullptr, arena.p,
                        (int64_t)arena.n, err.p) != cudaSuccess)
      return SNK_ERR_CUDA;
    OzGemmArgs a{};
    a.jobs = gj.p;
    a.n_jobs = 1;
    a.n_tiles = g.RTa * g.RTb;
    a.arena = arena.p;
    a.arena_bytes = (int64_t)arena.n;
    a.ws = out.p;
    a.err = err.p;
    if (launch_oz_gemm(0, slices, a, sms) != cudaSuccess) return SNK_ERR_CUDA;
  }
  int herr = 0;
  if (cudaMemcpy(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost) ||
      cudaMemcpy(C, out.p, sizeof(double) * M * N, cudaMemcpyDeviceToHost))
    return SNK_ERR_CUDA;
  return herr == 0 ? SNK_OK : (herr == 1 ? SNK_ERR_TIMEOUT : SNK_ERR_CUDA);
}

int snk_debug_pair_bound(snk_ctx* c, int32_t sa, int32_t sb, double* bound) {
  if (!c || !bound || sa < 0 || sb < 0 || sa >= c->s.ns || sb >= c->s.ns) return SNK_ERR_INVALID_ARG;
  *bound = pair_bound(c->s, sa, sb);
  return SNK_OK;
}

int snk_debug_batches(snk_ctx* c, int64_t* n_batches, int32_t* counts, int64_t counts_cap, int64_t* perm) {
  if (!c || !n_batches) return SNK_ERR_INVALID_ARG;
  *n_batches = c->nbatch;
  if (counts) {
    if (counts_cap < c->nbatch) return fail(c, SNK_ERR_INVALID_ARG, "counts buffer too small");
    for (int j = 0; j < c->nbatch; ++j) counts[j] = (int32_t)(c->s.bstart[j + 1] - c->s.bstart[j]);
  }
  if (perm) std::copy(c->s.perm.begin(), c->s.perm.end(), perm);
  return SNK_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free variant of snk_debug_shell_A, for callers that must not
// call cudaMalloc (for example code running while a CUDA graph is being
// captured, or a host that owns all device memory through its own pool).
// The raw contracted block Xi (before component factors) goes to a fixed
// scratch array in this file instead of a per-call device allocation.
// ---------------------------------------------------------------------------

namespace {

constexpr int64_t kNoAllocMaxPoints = 4096;
constexpr int kMaxDevices = 64;

// Shared by every call on a device and never freed (it lives as long as the
// module is loaded): 4096 points x 36 doubles = 1.125 MiB per device.
static __device__ __align__(256) double g_xi_scratch[kNoAllocMaxPoints * 36];

std::mutex g_scratch_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_xi_scratch on device dev, which must be the current
// device; looked up once per device (host code cannot use the symbol's name
// as a device pointer) and kept for the life of the process's CUDA context.
cudaError_t scratch_for_device(int dev, double** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_xi_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// out[i][u][v] = f_u f_v Xi[i][u][v], or the transposed block when the stored
// pair has its shells the other way round.
__global__ void finish_shell_A_kernel(const double* __restrict__ xi, int64_t n, int ca, int cb, int swap,
                                      const double* __restrict__ fa, const double* __restrict__ fb,
                                      double* __restrict__ out) {
  const int na = swap ? cb : ca, nb = swap ? ca : cb;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * na * nb) return;
  const int64_t i = e / (na * nb);
  const int u = (int)(e % (na * nb)) / nb, v = (int)(e % nb);
  const double x = swap ? xi[i * ca * cb + v * cb + u] : xi[i * ca * cb + u * cb + v];
  out[e] = x * fa[u] * fb[v];
}

}  // namespace

extern "C" int snk_shell_A_noalloc(snk_ctx* c, int32_t sa, int32_t sb, int64_t n, const double* xyz, double* out) {
  if (!c) return SNK_ERR_INVALID_ARG;
  Setup& s = c->s;
  if (sa < 0 || sb < 0 || sa >= s.ns || sb >= s.ns || n < 0 || (n > 0 && (!xyz || !out)))
    return fail(c, SNK_ERR_INVALID_ARG, "snk_shell_A_noalloc: bad shell index or buffer");
  if (n > kNoAllocMaxPoints)
    return fail(c, SNK_ERR_INVALID_ARG,
                "snk_shell_A_noalloc: n exceeds the 4096-point scratch; split the points into calls of at most 4096");
  int cur = -1;
  SNK_CK(c, cudaGetDevice(&cur));
  if (cur != c->device)
    return fail(c, SNK_ERR_BAD_STATE,
                "snk_shell_A_noalloc: the current device is not the one the handle was created on");
  double* scratch = nullptr;
  SNK_CK(c, scratch_for_device(c->device, &scratch));
  if (n == 0) return SNK_OK;
  const int na = ncart(s.l[sa]), nb = ncart(s.l[sb]);
  const int p = pair_id(s, sa, sb);
  if (p < 0) {  // pair dropped at setup: its block is zero to below 1e-20
    SNK_CK(c, cudaMemsetAsync(out, 0, sizeof(double) * n * na * nb, c->stream));
    return SNK_OK;
  }
  const PairHdr& h = s.pairs[p];
  const int ca = ncart(s.l[h.sa]), cb = ncart(s.l[h.sb]);
  SNK_CK(c, launch_debug_A(c->stream, s.pair_class[p], c->pairs.p + p, c->prims.p, c->boys.p, n, xyz, scratch));
  const int64_t tot = n * na * nb;
  finish_shell_A_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(
      scratch, n, ca, cb, h.sa != sa ? 1 : 0, c->fcomp.p + s.foff[sa], c->fcomp.p + s.foff[sb], out);
  SNK_CK(c, cudaGetLastError());
  return SNK_OK;
}

// ---------------------------------------------------------------------------
// Learned block screen: training data from the plain method, training and
// evaluation of the MLP with the library's kernels, loading into a handle.
// ---------------------------------------------------------------------------

namespace {

// splitmix64: seeded, platform-independent random numbers for the MLP set-up
struct SplitMix {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
  }
  double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
  double normal() { return std::sqrt(-2.0 * std::log(uniform())) * std::cos(6.283185307179586 * uniform()); }
};

int learn_collect(snk_ctx* c, int stride, int64_t cap, float* feat, float* lab, int64_t* n_out) {
  if (!n_out || stride < 1 || cap < 0 || (cap > 0 && (!feat || !lab)))
    return fail(c, SNK_ERR_INVALID_ARG, "snk_learn_collect: bad arguments");
  *n_out = 0;
  if (!c->have_density) return fail(c, SNK_ERR_BAD_STATE, "snk_learn_collect called before snk_set_density");
  if (c->n_dens != 1) return fail(c, SNK_ERR_BAD_STATE, "snk_learn_collect needs one density");
  if (c->opt.screen == SNK_SCREEN_LEARNED && c->mlp_loaded)
    return fail(c, SNK_ERR_BAD_STATE, "snk_learn_collect needs the rigorous screen's lists (screen != learned)");
  const int nb = c->nbatch, nbx = std::max(nb, 1);
  const cudaStream_t st = c->stream;
  std::vector<int> sb;
  std::vector<int64_t> slot(nbx, -1), soff, entries(nbx, 0);
  int64_t tot = 0;
  for (int j = 0; j < nb; j += stride) {
    for (int L = 0; L < kNumLists; ++L) entries[j] += c->hcounts[(size_t)j * kNumLists + L];
    if (tot + entries[j] > cap) break;
    slot[j] = tot;
    sb.push_back(j);
    soff.push_back(tot);
    tot += entries[j];
  }
  if (tot == 0) return SNK_OK;
  DevBuf<float> dlab, dfeat;
  DevBuf<double> dxmax;
  DevBuf<int64_t> dslot, dsoff;
  DevBuf<int> dsb;
  DevBuf<Tile> dtile;
  SNK_CK(c, dlab.ensure((size_t)tot * 12));
  SNK_CK(c, dfeat.ensure((size_t)tot * kMlpIn));
  SNK_CK(c, dxmax.ensure((size_t)std::max<int64_t>(c->s.npts, 1)));
  SNK_CK(c, cudaMemsetAsync(dlab.p, 0, sizeof(float) * tot * 12, st));
  SNK_CK(c, cudaMemsetAsync(dxmax.p, 0, sizeof(double) * std::max<int64_t>(c->s.npts, 1), st));
  SNK_CK(c, upload(dslot, slot, st));
  SNK_CK(c, upload(dsoff, soff, st));
  SNK_CK(c, upload(dsb, sb, st));
  SNK_CK(c, launch_features(st, c->sargs, c->list.p, c->list_off.p, c->counts.p, dsb.p, dsoff.p, (int)sb.size(),
                            c->shell_feat.p, dfeat.p));
  for (size_t ci = 0; ci < c->chunks.size(); ++ci) {
    const auto& ch = c->chunks[ci];
    bool any = false;
    for (int j = ch.b0; j < ch.b1; ++j) any = any || slot[j] >= 0;
    if (!any) continue;
    const int nbc = ch.b1 - ch.b0;
    const BatchDesc* db = c->batch.p + ch.b0;
    SNK_CK(c, launch_collocation(st, db, nbc, ch.max_ldq, ch.max_nBshell, c->bshell.p, c->bshell_col.p, c->xyz.p,
                                 dev_basis(c), c->ws.p));
    SNK_CK(c, launch_fgemm(st, db, nbc, ch.max_ldq, ch.max_nS, c->P.p, nullptr, c->xfunc.p, c->sfunc.p, c->fcomp.p,
                           c->w.p, c->ws.p, nullptr, 0, 0));
    SNK_CK(c, launch_xmax(st, db, nbc, c->ws.p, dxmax.p));
    for (int k = 0; k < kNumLists; ++k) {
      std::vector<Tile> ht;
      for (int j = ch.b0; j < ch.b1; ++j) {
        if (slot[j] < 0) continue;
        const int64_t n = c->hcounts[(size_t)j * kNumLists + k], base = c->hlist_off[(size_t)j * kNumLists + k];
        for (int64_t k0 = 0; k0 < n; k0 += c->run[k])
          for (int i0 = 0; i0 < c->hbatch[j].q; i0 += kPointTile)
            ht.push_back(Tile{j, (int)(base + k0), (int)(base + std::min<int64_t>(n, k0 + c->run[k])), i0});
      }
      if (ht.empty()) continue;
      SNK_CK(c, upload(dtile, ht, st));
      SNK_CK(c, cudaMemsetAsync(c->tickets.p, 0, sizeof(int), st));
      IntegralArgs a = integral_args(c, ci, k);
      a.tiles = dtile.p;
      a.n_tiles = (int)ht.size();
      a.ticket = c->tickets.p;
      SNK_CK(c, launch_labels(st, k % kNumClasses, a, (int)std::min<int64_t>(c->max_ctas[k % kNumClasses], a.n_tiles),
                              dslot.p, c->list_off.p, dxmax.p, dlab.p));
      // the tile buffer is reused by the next list: wait for this launch
      SNK_CK(c, cudaStreamSynchronize(st));
    }
  }
  std::vector<float> hl((size_t)tot * 12);
  SNK_CK(c, cudaMemcpyAsync(hl.data(), dlab.p, sizeof(float) * hl.size(), cudaMemcpyDeviceToHost, st));
  SNK_CK(c, cudaMemcpyAsync(feat, dfeat.p, sizeof(float) * tot * kMlpIn, cudaMemcpyDeviceToHost, st));
  SNK_CK(c, cudaStreamSynchronize(st));
  for (int j : sb)
    for (int64_t e = 0; e < entries[j]; ++e) {
      const int64_t q = slot[j] + e;
      float m = 0.f;
      for (int u = 0; u < 12; ++u) m = std::max(m, hl[(size_t)q * 12 + u]);
      lab[q] = (float)(std::log10(std::max((double)m, 1e-40)) / 10.0);
    }
  *n_out = tot;
  return SNK_OK;
}

}  // namespace

extern "C" {

int snk_screen_load(snk_ctx* c, const float* weights) {
  if (!c) return SNK_ERR_INVALID_ARG;
  if (!weights) return fail(c, SNK_ERR_INVALID_ARG, "NULL weights");
  for (int e = 0; e < kMlpWeights; ++e)
    if (!std::isfinite(weights[e])) return fail(c, SNK_ERR_UNSUPPORTED, "non-finite MLP weight");
  std::vector<float> w(weights, weights + kMlpWeights);
  SNK_CK(c, upload(c->mlp_w, w, c->stream));
  SNK_CK(c, cudaStreamSynchronize(c->stream));
  c->mlp_loaded = true;
  return SNK_OK;
}

int snk_learn_collect(snk_ctx* c, int32_t stride, int64_t cap, float* features, float* labels, int64_t* n) {
  if (!c) return SNK_ERR_INVALID_ARG;
  return learn_collect(c, stride, cap, features, labels, n);
}

int snk_mlp_eval(const float* weights, const float* features, int64_t n, int32_t f16, float* out) {
  if (!weights || n < 0 || (n > 0 && (!features || !out))) return SNK_ERR_INVALID_ARG;
  if (n == 0) return SNK_OK;
  DevBuf<float> dw, dx, dy;
  if (dw.ensure(kMlpWeights) || dx.ensure((size_t)n * kMlpIn) || dy.ensure(n)) return SNK_ERR_OOM;
  if (cudaMemcpy(dw.p, weights, sizeof(float) * kMlpWeights, cudaMemcpyHostToDevice) ||
      cudaMemcpy(dx.p, features, sizeof(float) * n * kMlpIn, cudaMemcpyHostToDevice))
    return SNK_ERR_CUDA;
  if (launch_mlp_forward(0, dw.p, dx.p, n, dy.p, f16 != 0) != cudaSuccess) return SNK_ERR_CUDA;
  if (cudaMemcpy(out, dy.p, sizeof(float) * n, cudaMemcpyDeviceToHost)) return SNK_ERR_CUDA;
  return SNK_OK;
}

int snk_mlp_grad(const float* weights, const float* features, const float* labels, int64_t n, float under_weight,
                 float* grad, float* loss) {
  if (!weights || !grad || !loss || n <= 0 || !features || !labels) return SNK_ERR_INVALID_ARG;
  DevBuf<float> dw, dx, dy, dz, dd, dg, dl;
  if (dw.ensure(kMlpWeights) || dx.ensure((size_t)n * kMlpIn) || dy.ensure(n) ||
      dz.ensure((size_t)n * 3 * kMlpHidden) || dd.ensure((size_t)n * (3 * kMlpHidden + 1)) ||
      dg.ensure(kMlpWeights) || dl.ensure(1))
    return SNK_ERR_OOM;
  if (cudaMemcpy(dw.p, weights, sizeof(float) * kMlpWeights, cudaMemcpyHostToDevice) ||
      cudaMemcpy(dx.p, features, sizeof(float) * n * kMlpIn, cudaMemcpyHostToDevice) ||
      cudaMemcpy(dy.p, labels, sizeof(float) * n, cudaMemcpyHostToDevice))
    return SNK_ERR_CUDA;
  if (launch_mlp_grad(0, dw.p, dx.p, dy.p, nullptr, n, under_weight, dz.p, dd.p, dg.p, dl.p) != cudaSuccess)
    return SNK_ERR_CUDA;
  if (cudaMemcpy(grad, dg.p, sizeof(float) * kMlpWeights, cudaMemcpyDeviceToHost) ||
      cudaMemcpy(loss, dl.p, sizeof(float), cudaMemcpyDeviceToHost))
    return SNK_ERR_CUDA;
  return SNK_OK;
}

int snk_mlp_train(const float* features, const float* labels, int64_t n, int32_t epochs, int32_t batch, float lr,
                  float under_weight, uint64_t seed, int32_t init, float* weights, float* loss_history) {
  if (!features || !labels || !weights || n <= 0 || epochs < 0 || batch < 1) return SNK_ERR_INVALID_ARG;
  SplitMix rng{seed};
  std::vector<float> w(weights, weights + kMlpWeights);
  if (init) {
    // He-normal weights, zero biases; the output bias starts at the mean label
    const int nin[4] = {kMlpIn, kMlpHidden, kMlpHidden, kMlpHidden};
    const int wo[4] = {0, kMlpIn * kMlpHidden + kMlpHidden,
                       kMlpIn * kMlpHidden + kMlpHidden + kMlpHidden * kMlpHidden + kMlpHidden,
                       kMlpIn * kMlpHidden + kMlpHidden + 2 * (kMlpHidden * kMlpHidden + kMlpHidden)};
    const int nout[4] = {kMlpHidden, kMlpHidden, kMlpHidden, 1};
    std::fill(w.begin(), w.end(), 0.f);
    for (int l = 0; l < 4; ++l) {
      const double sd = std::sqrt((l == 3 ? 1.0 : 2.0) / nin[l]);
      for (int e = 0; e < nin[l] * nout[l]; ++e) w[wo[l] + e] = (float)(sd * rng.normal());
    }
    double mean = 0.0;
    for (int64_t s = 0; s < n; ++s) mean += labels[s];
    w[kMlpWeights - 1] = (float)(mean / n);
  }
  const int64_t B = std::min<int64_t>(batch, n);
  DevBuf<float> dw, dx, dy, dz, dd, dg, dm1, dm2, dl;
  DevBuf<int64_t> didx;
  const int64_t nsteps = (n + B - 1) / B;
  if (dw.ensure(kMlpWeights) || dx.ensure((size_t)n * kMlpIn) || dy.ensure(n) ||
      dz.ensure((size_t)B * 3 * kMlpHidden) || dd.ensure((size_t)B * (3 * kMlpHidden + 1)) ||
      dg.ensure(kMlpWeights) || dm1.ensure(kMlpWeights) || dm2.ensure(kMlpWeights) || dl.ensure(nsteps) ||
      didx.ensure(n))
    return SNK_ERR_OOM;
  if (cudaMemcpy(dw.p, w.data(), sizeof(float) * kMlpWeights, cudaMemcpyHostToDevice) ||
      cudaMemcpy(dx.p, features, sizeof(float) * n * kMlpIn, cudaMemcpyHostToDevice) ||
      cudaMemcpy(dy.p, labels, sizeof(float) * n, cudaMemcpyHostToDevice) ||
      cudaMemset(dm1.p, 0, sizeof(float) * kMlpWeights) || cudaMemset(dm2.p, 0, sizeof(float) * kMlpWeights))
    return SNK_ERR_CUDA;
  std::vector<int64_t> idx(n);
  for (int64_t s = 0; s < n; ++s) idx[s] = s;
  std::vector<float> hl(nsteps);
  int t = 0;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int64_t s = n - 1; s > 0; --s) std::swap(idx[s], idx[rng.next() % (uint64_t)(s + 1)]);
    if (cudaMemcpy(didx.p, idx.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice)) return SNK_ERR_CUDA;
    for (int64_t st = 0; st < nsteps; ++st) {
      const int64_t b0 = st * B, nb = std::min<int64_t>(B, n - b0);
      if (launch_mlp_grad(0, dw.p, dx.p, dy.p, didx.p + b0, nb, under_weight, dz.p, dd.p, dg.p, dl.p + st) !=
              cudaSuccess ||
          launch_adam(0, dw.p, dg.p, dm1.p, dm2.p, ++t, lr) != cudaSuccess)
        return SNK_ERR_CUDA;
    }
    if (cudaMemcpy(hl.data(), dl.p, sizeof(float) * nsteps, cudaMemcpyDeviceToHost)) return SNK_ERR_CUDA;
    double sum = 0.0, wsum = 0.0;
    for (int64_t st = 0; st < nsteps; ++st) {
      const double nb = (double)std::min<int64_t>(B, n - st * B);
      sum += hl[st] * nb;
      wsum += nb;
    }
    if (loss_history) loss_history[ep] = (float)(sum / wsum);
  }
  if (cudaMemcpy(weights, dw.p, sizeof(float) * kMlpWeights, cudaMemcpyDeviceToHost)) return SNK_ERR_CUDA;
  return SNK_OK;
}

}  // extern "C"
