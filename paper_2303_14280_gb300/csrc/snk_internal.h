// Internal declarations of libsnk (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/snk.h"

namespace snk {

constexpr int kLMax = 2;
constexpr int kNumClasses = 6;  // (0,0) (1,0) (1,1) (2,0) (2,1) (2,2)
constexpr int kNumLists = 2 * kNumClasses;  // per batch: FP64 lists, then FP32 lists
constexpr int kPointTile = 128;  // grid points per integral tile (one per thread)
constexpr int kLdqAlign = 128;   // leading-dimension padding of batch matrices

// K-hat accumulator: every entry is a pair of 64-bit integers (hi, lo) worth
// hi 2^-32 + lo 2^-76.  Integer additions are exact and
// associative, so the sum of the batches' contributions does not depend on
// the order in which they arrive (K is the same bit for bit from run to run).
// A contribution v is cut as hi = rint(v 2^32), lo = rint((v - hi 2^-32) 2^76):
// |v| < 2^30, |lo| <= 2^43 (sums of up to 2^19 batches stay below 2^62), and
// what is dropped is below 2^-77 ~ 7e-24 per contribution.
constexpr int kKhatMaxBatches = 1 << 19;
constexpr int kErrKhatRange = 3;  // device error flag: a contribution outside |v| < 2^30
#ifdef __CUDACC__
__device__ __forceinline__ void khat_add(unsigned long long* e, double v, int* err) {
  if (!(fabs(v) < 0x1p30)) {  // and NaN
    if (err) atomicExch(err, kErrKhatRange);
    return;
  }
  const long long hi = __double2ll_rn(v * 0x1p32);
  const double r = fma(-(double)hi, 0x1p-32, v);  // exact: v - hi 2^-32
  const long long lo = __double2ll_rn(r * 0x1p76);
  atomicAdd(e, (unsigned long long)hi);
  atomicAdd(e + 1, (unsigned long long)lo);
}
__device__ __forceinline__ double khat_value(const unsigned long long* e) {
  return (double)(long long)e[0] * 0x1p-32 + (double)(long long)e[1] * 0x1p-76;
}
#endif

// Boys table: rows T_k = k * kBoysH, k = 0..kBoysRows-1; for T >= kBoysTMax the
// asymptotic form is used.  One table per L = 0..4 with kBoysCols doubles per
// row: F_{L+m}(T_k)/m! for m = 0..7, exp(-T_k), T_k.
constexpr double kBoysH = 0.1;
constexpr double kBoysTMax = 50.0;
constexpr int kBoysRows = 502;
constexpr int kBoysTerms = 8;
constexpr int kBoysCols = kBoysTerms + 2;
constexpr int kBoysLMax = 2 * kLMax;

// FP32 Boys table of the mixed form: nodes T_k = fl32(k * 0.05f) up to
// kBoysTMaxF, rows of F_{L+m}(T_k)/m! for m = 0..3 (one float4).
constexpr float kBoysTMaxF = 30.0f;
constexpr float kBoysHF = 0.05f;
constexpr int kBoysRowsF = 602;
constexpr int kBoysTermsF = 4;
constexpr int kBoysColsF = kBoysTermsF;

// Learned block screen: MLP 16 -> 64 -> 64 -> 64 -> 1 (ReLU).
constexpr int kMlpIn = 16;
constexpr int kMlpHidden = 64;
constexpr int kMlpWeights = kMlpIn * kMlpHidden + kMlpHidden + 2 * (kMlpHidden * kMlpHidden + kMlpHidden) +
                            kMlpHidden + 1;

// Primitive pairs whose 3c-CP potential is below this everywhere are left out
// of a shell pair (their total effect on K is below ~1e-14 for any basis here).
constexpr double kPrimPairTol = 1e-20;
// The FP32 tier of the mixed form leaves out a pair's primitive pairs whose
// bound is below this fraction of its largest: at most 8 such terms change a
// block by < 1e-7 of its bound, the resolution of the tier's FP32 arithmetic.
constexpr double kPrimPairRelTolF32 = 1e-8;

inline int ncart(int l) { return (l + 1) * (l + 2) / 2; }
inline int class_of(int la, int lb) {  // la >= lb
  return la * (la + 1) / 2 + lb;
}

// Per primitive pair data used by the integral kernel (12 doubles).
struct PrimPair {
  double zeta;          // zeta_a + zeta_b
  double Px, Py, Pz;    // Gaussian product centre R_p
  double PAx, PAy, PAz; // R_p - R_a
  double pref;          // 2 pi / zeta * exp(-zeta_a zeta_b |AB|^2 / zeta) * d_a d_b
  double pref_far;      // pref * sqrt(pi) / 2  (large-T seed)
  double k1, k2, k3;    // 1, 2, 3 times 1 / (2 zeta)
};

// Shell pair header.  The pair's primitive pairs are stored largest bound
// first; the FP32 tier uses the first pp_n32 of them.
struct PairHdr {
  int32_t sa, sb;       // shells; l(sa) >= l(sb)
  int32_t pp_off, pp_n; // primitive pairs
  double ABx, ABy, ABz; // R_a - R_b
  int32_t pp_n32;       // primitive pairs of the FP32 tier (bound >= kPrimPairRelTolF32 x the largest)
  int32_t pad;
};

// Per grid batch, per build chunk.
struct BatchDesc {
  int64_t p0;        // first point in batch order
  int32_t q;         // number of points
  int32_t ldq;       // padded leading dimension of X, F, G
  int32_t nB;        // X columns (functions of B_j)
  int32_t nS;        // F / G columns (functions of the shells in V_j)
  int64_t xoff;      // offsets (doubles) into the chunk workspace
  int64_t foff;
  int64_t goff;
  int32_t xfunc_off; // CSR offsets into xfunc / sfunc / bshell
  int32_t sfunc_off;
  int32_t bshell_off;
  int32_t nBshell;
  int64_t foff32;    // mixed form: offset (floats) of the FP32 copy of F
  int64_t ssoff;     // tile screen: offset (floats) of the batch's per-tile column sums
  int32_t mol;       // molecule of the batch, its first shell and function, N_b,m
  int32_t ms0;
  int32_t mf0;
  int32_t nfm;
  int64_t pk_off;    // the molecule's P / K block
  int64_t cm_off;    // the batch's row of shell-local arrays (F-tilde, column maps)
  int64_t phf_off;   // the batch's row of function-local arrays (Phi-tilde)
  int32_t nS_hi;     // F / G columns [0, nS_hi) belong to shells of high-tier pairs
  int32_t pad_;
};

// Per molecule, on the device.
struct MolDesc {
  int64_t pk_off;
  int32_t nf, ns, ms0, mf0, mb0, nb;
  int32_t cr[kNumClasses + 1];
  int32_t pad;
};

// Integral-kernel tile: batch, pair-list range (the batch's whole list),
// first point.
struct Tile {
  int32_t batch, k0, k1, i0;
};

// ---------------------------------------------------------------- host setup

struct Setup {
  // molecules: shells [ms0, ms0+ns), functions [mf0, mf0+nf), batches
  // [mb0, mb0+nb), pairs of class c in [cr[c], cr[c+1]); P / K block at
  // pk_off (nf x nf, row-major); dense pair index block at pi_off (ns x ns)
  struct Mol {
    int ms0 = 0, ns = 0, mf0 = 0, nf = 0, mb0 = 0, nb = 0;
    int64_t pk_off = 0, pi_off = 0, p0 = 0, npts = 0;
    int cr[kNumClasses + 1] = {0};
  };
  int n_mol = 1;
  std::vector<Mol> mols;
  std::vector<int> bmol;                 // molecule of each batch
  std::vector<int64_t> cm_off, phf_off;  // per batch: offsets of its shell-local and function-local rows
  int64_t cm_total = 0, phf_total = 0, packed = 0;

  int ns = 0, nf = 0, nprim_total = 0;
  std::vector<int> l, nprim, poff, foff, atom;
  std::vector<double> center, exps, d, fcomp, rcut;
  std::vector<int> fshell;  // shell of each function

  // shell pairs sorted by class, then a, then b
  std::vector<PairHdr> pairs;
  std::vector<PrimPair> prims;
  std::vector<double> prim_rel;       // per primitive pair: its bound / its shell pair's bound
  std::vector<double> bound;          // rigorous max_r |A| per pair
  std::vector<double> qbound;         // rigorous total |charge| per pair: |A| <= qbound / distance
  std::vector<int> pair_class;
  int class_begin[kNumClasses + 1] = {0};
  std::vector<int> pair_index;        // dense ns x ns -> pair id or -1

  // grid, in batch order
  int64_t npts = 0;
  std::vector<double> xyz, w;
  std::vector<int64_t> perm;          // batch order -> input order
  std::vector<int64_t> bstart;        // n_batches + 1
  std::vector<double> bcenter, bradius;
  std::vector<int> bshell_off, bshell;  // B_j as shell lists (CSR)
  std::vector<int> bshell_col;          // local X column of each B_j shell
  std::vector<int> bnf;               // |B_j| in functions
  std::vector<int> xfunc_off, xfunc;  // B_j as function lists (CSR)

  std::vector<double> boys;           // (kBoysLMax+1) x kBoysRows x kBoysCols
  std::vector<float> boys_f;          // (kBoysLMax+1) x kBoysRowsF x kBoysColsF
  std::vector<float> boys_ds;         // (hi, lo) pairs: (kBoysLMax+1) x kBoysRows x kBoysCols x 2
};

// Validates and normalises the molecules' bases and grids; returns an
// snk_status and fills msg.
int build_setup(int n_mol, const snk_basis* bases, const snk_grid* grids, const snk_options* opt, Setup* s,
                std::string* msg);
void build_boys_tables(Setup* s);
double pair_bound(const Setup& s, int sa, int sb);
void prim_pair_bounds(const Setup& s, int sa, int sb, int k, int m, double* abound, double* qbound);
void host_boys(int nmax, double T, double* F);

// ---------------------------------------------------------------- kernels

struct DeviceBasis {
  const int* l;
  const int* poff;
  const int* nprim;
  const double* center;
  const double* exps;
  const double* d;
  const double* fcomp;
  const int* foff;
};

cudaError_t launch_collocation(cudaStream_t st, const BatchDesc* dbatch, int nbatch, int max_ldq,
                               int max_nBshell, const int* bshell, const int* bshell_col, const double* xyz,
                               DeviceBasis basis, double* ws);
// Phi-tilde rows at BatchDesc::phf_off of phit_f, phi-tilde at the batch index
// relative to dbatch of phit_b.
cudaError_t launch_screen_geom(cudaStream_t st, const BatchDesc* dbatch, int nbatch, int max_nB,
                               const double* ws, const double* w, const int* xfunc, double* phit_f,
                               double* phit_b);
// F-tilde of every molecule's batches (one GEMM per molecule in one launch).
cudaError_t launch_ftilde(cudaStream_t st, const MolDesc* mols, int n_mol, int max_nf, int max_nb,
                          const BatchDesc* batches, const double* P, const double* phit_f, const int* fshell,
                          double* ft_shell);
// Inputs of the sn-LinK pair screen (Eqs. sp_set, exx_fmat_approx).
struct ScreenArgs {
  const MolDesc* mols;
  const BatchDesc* batches;
  const PairHdr* pairs;
  const double* bound;      // global A-tilde per pair
  const double* qbound;     // total-charge bound per pair
  const double* shell_xyz;  // shell centres
  const double* bcenter;    // batch bounding spheres
  const double* bradius;
  const double* ft_shell;   // F-tilde per (batch, molecule-local shell), rows at BatchDesc::cm_off
  const double* phit_b;     // phi-tilde per batch
  int screen;               // snk_screen_mode
  int distance;             // 1: refine A-tilde by charge / distance per batch
  int mixed;                // 1: route low-estimate pairs to the FP32 lists
  double eps_E, eps_K, fp32_bound;
  signed char* codes;        // pass 1's decision per (batch, pair of its molecule): list index or -1
  const int64_t* code_off;   // per batch: its row of codes
};

cudaError_t launch_pair_count(cudaStream_t st, const ScreenArgs& a, int nbatch, int* counts, long long* ppcounts,
                              unsigned char* sflag, int64_t hflag_off);
cudaError_t launch_pair_write(cudaStream_t st, const ScreenArgs& a, int nbatch, const int64_t* list_off, int* list);
// P, Khat and K below are the packed molecule blocks (BatchDesc::pk_off,
// MolDesc::pk_off; Khat holds two words per entry, see khat_add); xfunc /
// sfunc hold molecule-local function indices.
// mode: 0 FP64, 2 double-FP32 (X, G and P2 then hold (hi, lo) float pairs in
// place of the doubles, see launch_split_df32).  dens: which density's F / G
// block of each batch (at foff / goff + dens ldq nS).
cudaError_t launch_fgemm(cudaStream_t st, const BatchDesc* dbatch, int nbatch, int max_ldq, int max_nS,
                         const double* P, const float2* P2, const int* xfunc, const int* sfunc,
                         const double* fcomp, const double* w, double* ws, float* ws32, int mode, int dens);
cudaError_t launch_kgemm(cudaStream_t st, const BatchDesc* dbatch, int nbatch, int max_nS, int max_nB,
                         const int* xfunc, const int* sfunc, const double* ws, unsigned long long* Khat, int mode,
                         int dens, int* err);
// In place, each double of buf[0, n) becomes the float pair (fl32(v), fl32(v - fl32(v))).
cudaError_t launch_split_df32(cudaStream_t st, double* buf, int64_t n);
cudaError_t launch_split_df32_copy(cudaStream_t st, const double* src, int64_t n, float2* dst);
// out = sum_d |P_d| over n_dens consecutive arrays of n doubles.
cudaError_t launch_abs_sum(cudaStream_t st, const double* P, int n_dens, int64_t n, double* out);
cudaError_t launch_finish(cudaStream_t st, const MolDesc* mols, int n_mol, int64_t packed,
                          const unsigned long long* Khat, const double* fcomp, double* K);
cudaError_t launch_symcheck(cudaStream_t st, const MolDesc* mols, int n_mol, int64_t packed, const double* P,
                            double* out2);

// Exchange-correlation potential (Sec. II.C).  Per batch at BatchDesc::xoff:
// X, dX/dx, dX/dy, dX/dz (ldq x nB each), then F / Z at BatchDesc::foff.
// mode: 0 FP64 tiles, 2 double-FP32 tiles.  Vhat (two words per entry of the
// molecule's block at pk_off, see khat_add) and Ehat (two words per
// molecule, at 2 BatchDesc::mol) accumulate.
cudaError_t launch_xc_colloc(cudaStream_t st, const BatchDesc* dbatch, int nbatch, int max_ldq, int max_nBshell,
                             const int* bshell, const int* bshell_col, const double* xyz, DeviceBasis basis,
                             double* ws);
cudaError_t launch_xc_fgemm(cudaStream_t st, const BatchDesc* dbatch, int nbatch, int max_ldq, int max_nB,
                            const double* P, const int* xfunc, double* ws, int mode);
cudaError_t launch_xc_point(cudaStream_t st, const BatchDesc* dbatch, int nbatch, int max_ldq, const double* w,
                            int functional, double* ws, unsigned long long* Ehat, int* err);
cudaError_t launch_xc_vgemm(cudaStream_t st, const BatchDesc* dbatch, int nbatch, int max_nB, const int* xfunc,
                            const double* ws, unsigned long long* Vhat, int mode, int* err);
// V = V-hat + V-hat^T in every molecule block of the packed matrices, and
// E[m] = E-hat of molecule m (two words per molecule).
cudaError_t launch_xc_finish(cudaStream_t st, const MolDesc* mols, int n_mol, int64_t packed,
                             const unsigned long long* Vhat, const unsigned long long* Ehat, double* V, double* E);

struct IntegralArgs {
  const Tile* tiles;
  int n_tiles;
  int* ticket;
  const BatchDesc* batches;
  const int* pairlist;
  const PairHdr* pairs;
  const PrimPair* prims;
  const int* colmap;  // per batch (rows at BatchDesc::cm_off): F/G column of each molecule shell or -1
  const double* xyz;  // batch order
  const double* boys; // device table, all L
  double* ws;
  // mixed form (FP32 lists)
  const float* boys_f;
  float* ws32;
  const double* bcenter;
  // mixed form: (hi, lo) float splits of the pair data, read by the FP32 and
  // ds kernels; hi_ds selects integral_kernel_ds for the FP64 lists
  const float2* boys_ds;   // (hi, lo) Boys table, nodes rounded to ds values
  const float2* prims_ds;  // 12 (hi, lo) pairs per primitive pair, PrimPair order
  const float2* pair_ab;   // 4 per shell pair: R_a - R_b as 3 (hi, lo) pairs, padding
  // FP32 record per primitive pair (32 bytes): {zeta, PAx, PAy, PAz}, {pref, pref_far, 1/(2 zeta),
  // its bound / the shell pair's bound}
  const float4* prims_f32;
  const float2* pair_a;    // 4 per shell pair: R_a as 3 (hi, lo) pairs, padding
  int hi_ds;
  int n_dens;      // densities: F and G of density d at foff / goff (F32: foff32) + d ldq nS
  // tile screen of the FP32 lists (eps_tile > 0): a pair is skipped on a
  // 128-point tile when bound_ab x max(sum over b's columns, sum over a's
  // columns) of tsum is below eps_tile; tsum[ssoff + tile (nS + 4) + col] =
  // sum_{i in tile} |F_col(i)| max_nu |X_nu(i)|, then the tile's centre and
  // radius; bound_ab = min(pbound, qbound / distance from the segment AB to
  // the tile's sphere)
  const float* tsum;
  const double* pbound;  // rigorous max_r |A_ab(r)| per shell pair
  const double* qbound;  // rigorous total |charge| per shell pair
  const double* shell_xyz;
  float eps_tile;
  unsigned long long* exec;  // FP32 lists: += (primitive pairs x points, pairs x points) computed
  int run;                   // FP32 lists: pairs staged (and tile-screened) per step, 1..kMaxRun
  int* err;                  // set to 1 when a bounded wait on a copy ran out
};

cudaError_t launch_integrals(cudaStream_t st, int cls, const IntegralArgs& a, int grid_ctas);
int integral_max_ctas(int cls, int num_sms, bool ds, int n_dens);
cudaError_t launch_debug_A(cudaStream_t st, int cls, const PairHdr* pair, const PrimPair* prims,
                           const double* boys, int64_t n, const double* xyz, double* xi);
cudaError_t launch_debug_boys(cudaStream_t st, const double* boys, int64_t n, const double* T,
                              int nmax, double* out);

// Algorithmic flops of the integral kernel per class and grid point: per
// primitive pair and per contracted pair (from the generator's counts).
void class_flops(int cls, double* per_prim, double* per_pair);

// Tiles of every (batch, list): ceil(count / run) runs x ceil(q / 128) slabs,
// the (batch, list)'s tiles from tiles[tstart[batch * kNumLists + list]] on.
cudaError_t launch_gen_tiles(cudaStream_t st, int nbatch, const BatchDesc* batches, const int* counts,
                             const int64_t* list_off, const int64_t* tstart, Tile* tiles);

// ---------------------------------------------------------------- split-product tensor-core GEMMs

// One operand of one batch to cut into bf16 fixed-point slices (pre-tiled
// blocks of 128 rows x 32 reduction indices, S slices per block), element
// (r, k), r < R, k < K:
//   mode 0: ws[src_off + k ld + r]                      (X_j as F = X P's left operand)
//   mode 1: ws[src_off + (r0 + r) ld + k]               (G_j rows, X_j rows: Kt = G^T X)
//   mode 2: P[src_off + sfunc[sf_off + r0 + r] ld + xfunc[xf_off + k]]  (P[S_j, B_j], P symmetric)
struct OzSplitJob {
  int32_t mode, R, K, S, ld, r0, sf_off, xf_off;
  int64_t src_off, dst_off;  // doubles into the source; bytes into the slice arena
};

// One product of one batch: C[m][n] = sum_k A[m][k] B[n][k] over the arena
// operands at a_off / b_off (RTa / RTb row blocks, KT reduction blocks, Sa /
// Sb slices stored per block); its RTa x RTb tiles are numbered from tile0.
//   kind 0: F[(c0 + n) ldq + m] = w_m f_{c0+n} C (doubles at ws + out_off, floats at ws32 + out_off32)
//   kind 1: Khat[out_off + sfunc[c0 + m] N_b,m + xfunc[n]] += C (entries of two words, khat_add)
//   kind 2: ws[out_off + m ldc + n] = C (test export)
//   kind 3: ws[out_off + (c0 + n) ldq + m] = C (column-major, no weights: F of V^xc)
struct OzGemmJob {
  int64_t a_off, b_off, out_off, out_off32;
  int32_t RTa, RTb, KT, Sa, Sb, tile0, batch, kind, m_lim, n_lim, c0, ldc;
};

struct OzGemmArgs {
  const OzGemmJob* jobs;
  int n_jobs, n_tiles;
  const uint8_t* arena;
  int64_t arena_bytes;
  const BatchDesc* batches;
  const double* w;
  const double* fcomp;
  const int* sfunc;
  const int* xfunc;
  double* ws;
  float* ws32;
  unsigned long long* Khat;
  int* err;  // set to 1 when a wait ran out, 2 when an operand lay outside the arena, kErrKhatRange
};

int64_t oz_operand_bytes(int rows, int k, int slices);
int oz_row_tiles(int rows);
int oz_k_tiles(int k);
cudaError_t launch_oz_split(cudaStream_t st, const OzSplitJob* jobs, int n_jobs, int max_rows, int max_k,
                            const double* ws, const double* P, const int* xfunc, const int* sfunc, uint8_t* arena,
                            int64_t arena_bytes, int* err);
// slices: 3..6 (products of slice pairs i + j < slices)
cudaError_t launch_oz_gemm(cudaStream_t st, int slices, const OzGemmArgs& args, int num_sms);
// one thread waits (bounded by limit_ns) on an mbarrier nothing completes: *err = 1
cudaError_t launch_wait_probe(cudaStream_t st, int* err, unsigned long long limit_ns);

// learned screen
cudaError_t launch_labels(cudaStream_t st, int cls, const IntegralArgs& a, int grid, const int64_t* slot_base,
                          const int64_t* list_off, const double* xm, float* lab);
cudaError_t launch_mlp_forward(cudaStream_t st, const float* w, const float* X, int64_t n, float* out, bool f16);
cudaError_t launch_mlp_grad(cudaStream_t st, const float* w, const float* X, const float* Y, const int64_t* idx,
                            int64_t n, float under_weight, float* Z, float* D, float* grad, float* loss);
cudaError_t launch_adam(cudaStream_t st, float* w, const float* g, float* m1, float* m2, int t, float lr);
cudaError_t launch_features(cudaStream_t st, const ScreenArgs& a, const int* pairlist, const int64_t* list_off,
                            const int* counts, const int* sample_batches, const int64_t* sample_off, int n_sample,
                            const float* shell_feat, float* feat);
// MLP over every list entry, then the lists rewritten into pairlist_out:
// entries predicted below skip_log10 dropped, high-tier entries predicted
// below fp32_log10 moved to the FP32 list of their class; list_off, counts,
// ppcounts and the high-tier shell flags (hflag, rows at cm_off) updated.
cudaError_t launch_learned_filter(cudaStream_t st, const ScreenArgs& a, int nbatch, const float* w,
                                  const int* pairlist, int* pairlist_out, int64_t* list_off, int* counts,
                                  long long* ppcounts, const float* shell_feat, float skip_log10, float fp32_log10,
                                  unsigned char* keep, unsigned char* hflag);
cudaError_t launch_xmax(cudaStream_t st, const BatchDesc* dbatch, int nbatch, const double* ws, double* xm);
// Per-tile column sums of the tile screen: for every batch, 128-point tile and
// F column, sum_i |F32_col(i)| max_nu |X_nu(i)| (summed over the densities).
cudaError_t launch_tile_sums(cudaStream_t st, const BatchDesc* dbatch, int nbatch, int max_tiles, const double* ws,
                             const float* ws32, const double* xyz, int n_dens, float* tsum);

}  // namespace snk
