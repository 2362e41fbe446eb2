/*
 * snk.h -- C ABI of libsnk: the seminumerical exact-exchange (sn-K) build of
 * hybrid Gaussian-basis Kohn-Sham DFT (arXiv 2303.14280) on one GB300 GPU.
 *
 * The library evaluates, for a basis set B, a quadrature grid Q = {(w_i, r_i)}
 * and a symmetric density matrix P,
 *
 *   Phi_{nu i}  = phi_nu(r_i)                              Sec. II.C, Eq. (collocation)
 *   F_{lam i}   = sum_nu P_{lam nu} Phi_{nu i}            Sec. II.C, Eq. (fmat)
 *   A_{mu lam}(r_i) = int phi_mu phi_lam / |r - r_i|       Sec. II.D, Eq. (3c_grid)
 *   G_{mu i}    = w_i sum_lam A_{mu lam}(r_i) F_{lam i}   Sec. II.D, Eq. (gmat)
 *   Kt_{mu nu}  = sum_i G_{mu i} Phi_{nu i}               Sec. II.D, Eq. (usym_k)
 *   K_{mu nu}   = (Kt_{mu nu} + Kt_{nu mu}) / 2           Sec. II.D, Eq. (sn_k)
 *
 * over octree grid batches Q_j (Sec. II.E) with the basis screen B_j
 * (Eq. basis_screen) and the sn-LinK pair screen V_j (Eqs. sp_set,
 * exx_fmat_approx, batch_local_exx).  A is evaluated by the Obara-Saika
 * recursions of App. A (Eqs. vrr, hrr), contracted with F on the fly.
 *
 * Forms (all through the same calls, selected by snk_options):
 *   - plain: FP64 throughout (the default);
 *   - mixed precision: blocks with a small sn-LinK estimate in FP32, the rest
 *     in FP64 or double-FP32 (hi + lo float pairs), the two products in FP64,
 *     double-FP32 or bf16 split products on the tcgen05 tensor cores; G and K
 *     accumulated in FP64;
 *   - batched: many molecules in one handle (snk_create_batch), one launch per
 *     phase, optional CUDA-graph replay and autotuned tiles;
 *   - learned screen: a small MLP, trained by the library's own kernels,
 *     skips blocks and picks the precision tier behind the rigorous screen;
 *   - several densities of one molecule in one build (snk_set_density_multi).
 *
 * Conventions
 *   - Units: bohr and hartree.  K is the bare exchange matrix: no -c_x factor
 *     and no closed-shell factor (P is used as given).
 *   - Basis functions are contracted Cartesian Gaussians, l = 0, 1, 2.  Order:
 *     shells in input order; inside a shell the Cartesian components in
 *     lexicographic order (l,0,0), (l-1,1,0), (l-1,0,1), (l-2,2,0), ...,
 *     i.e. x y z for p and xx xy xz yy yz zz for d.  Each component is
 *     normalised to unit self-overlap; the caller's contraction coefficients
 *     refer to x^l-normalised primitives.
 *   - Matrices are N_b x N_b, row-major, double precision.
 *
 * Ownership: every input is copied during the call that receives it; the
 * caller keeps ownership of all pointers it passes.  Device pointers must be
 * allocations on the device that was current at snk_create.
 *
 * Errors: every call returns SNK_OK (0) or a negative snk_status.  After an
 * error the handle stays valid for snk_last_error and snk_destroy; a build
 * that failed leaves the output untouched or partially written.  A handle is
 * not re-entrant: calls on one handle must not overlap.  No call aborts the
 * process.
 */
#ifndef SNK_H
#define SNK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SNK_OK = 0,
  SNK_ERR_INVALID_ARG = -1,   /* NULL pointer, negative size, bad index      */
  SNK_ERR_UNSUPPORTED = -2,   /* l > 2, non-finite or non-positive input     */
  SNK_ERR_NOT_SYMMETRIC = -3, /* max|P - P^T| > 1e-12 max|P|                 */
  SNK_ERR_BAD_STATE = -4,     /* build before set_density, ...               */
  SNK_ERR_OOM = -5,           /* device or host allocation failed            */
  SNK_ERR_CUDA = -6,          /* a CUDA runtime call failed                  */
  SNK_ERR_TIMEOUT = -7        /* a bounded device wait ran out               */
} snk_status;

typedef struct snk_ctx snk_ctx; /* opaque handle */

/* Contracted Cartesian basis.  All arrays are host memory, copied at create. */
typedef struct {
  int32_t n_shells;
  const int32_t *l;      /* [n_shells], 0..2, else SNK_ERR_UNSUPPORTED       */
  const int32_t *nprim;  /* [n_shells], 1..16 primitives per shell            */
  const int32_t *atom;   /* [n_shells], owning atom (informational)           */
  const double *center;  /* [3 n_shells], bohr                                */
  const double *exps;    /* [sum nprim], > 0, shell after shell               */
  const double *coefs;   /* [sum nprim], w.r.t. x^l-normalised primitives     */
} snk_basis;

/* Quadrature grid (Sec. II.C): nodes, weights (atomic quadrature x partition
 * weight) and the atom each node belongs to (used for atom-centred batching). */
typedef struct {
  int64_t n_points;      /* >= 0                                              */
  const double *xyz;     /* [3 n_points], bohr                                */
  const double *w;       /* [n_points]                                        */
  const int32_t *atom;   /* [n_points], >= 0                                  */
} snk_grid;

typedef enum { SNK_PREC_FP64 = 0, SNK_PREC_MIXED = 1 } snk_precision;
typedef enum { SNK_SCREEN_NONE = 0, SNK_SCREEN_LINK = 1, SNK_SCREEN_LEARNED = 2 } snk_screen_mode;
typedef enum { SNK_GEMM_FP64 = 0, SNK_GEMM_DF32 = 1, SNK_GEMM_SPLIT = 2 } snk_gemm_mode;

typedef struct {
  double eps_basis;        /* epsilon_B of Eq. (basis_screen); <= 0 keeps all   */
  double eps_E;            /* epsilon_E of Eq. (sp_set)                          */
  double eps_K;            /* epsilon_K of Eq. (sp_set)                          */
  int32_t batch_max;       /* largest grid batch (octree leaf), Sec. III: 4096  */
  int32_t precision;       /* snk_precision                                      */
  int32_t screen;          /* snk_screen_mode                                    */
  int32_t distance_bound;  /* 1: per batch, A-tilde = min(global bound, total
                              charge / distance to the batch) -- both rigorous;
                              0: the global bound alone, as in the paper        */
  double fp32_bound;       /* mixed form: kept pairs whose sn-LinK estimate
                              epsilon^K is below this run their integrals in FP32 */
  int64_t workspace_bytes; /* device workspace cap for batch chunks (Alg. 1); 0 = auto */
  int32_t graph;           /* 1: snk_build_K* capture the whole build in a CUDA graph
                              on first use (per density and output buffer) and
                              replay it; phase times are then not reported      */
  double learned_skip;     /* learned screen: skip a block whose predicted log10
                              contribution to K is below this (default -11)     */
  int32_t gemm;            /* mixed form: SNK_GEMM_FP64 (default); SNK_GEMM_DF32,
                              F = X P and Kt = G^T X in double-FP32 arithmetic on the
                              FP32 pipe (operands as hi + lo float pairs, error-free
                              TwoSum accumulation, ~2^-46 relative); SNK_GEMM_SPLIT,
                              both products on the tcgen05 tensor cores as sums of
                              bf16 slice products: every operand cut into slices on
                              a fixed-point grid per row and run of 256 reduction
                              indices, each run's two leading levels of products
                              accumulated exactly in FP32, the runs summed in
                              double-FP32 -- tc_slices_hi slices for the F columns
                              and G rows of shells in a batch's FP64-tier pairs,
                              tc_slices_lo for the rest                         */
  int32_t ds_integrals;    /* mixed form: 1 runs the integrals of the pairs above
                              fp32_bound in double-FP32 arithmetic (hi + lo float
                              pairs on the FP32 pipe, ~1e-14 relative) instead of
                              FP64; default 0                                   */
  double learned_fp32;     /* learned screen, mixed form: a block of the FP64 (or
                              double-FP32) tier whose predicted log10 contribution
                              is below this moves to the FP32 tier; default -99
                              (off)                                             */
  int32_t tc_slices_hi;    /* SNK_GEMM_SPLIT: bf16 slices per operand for the high-
                              tier columns / rows, 3..6 (default 5: 15 slice
                              products, ~2^-31 of the run maxima, set by the FP32
                              sum of the products below the two leading levels)  */
  int32_t tc_slices_lo;    /* SNK_GEMM_SPLIT: the same for the rest, 3..6 (default
                              4: 10 products, ~2^-30)                           */
  double eps_tile;         /* mixed form, FP32 pairs, gemm FP64 or SPLIT: a kept
                              (batch, pair) block is also screened per 128-point
                              tile of the batch (points ordered by a finer
                              octree), skipping the tile when A-tilde_ab x
                              max(sum_i |F_b(i)| max|Phi(i)|, the same with a)
                              over the tile's points -- a bound of what the
                              tile adds to any K-tilde entry, up to the
                              component factors -- is below eps_tile; on the
                              tiles kept, the pair's primitive pairs (stored
                              largest bound first) whose bounds on the tile
                              add up to less than eps_tile are left out;
                              0 = off (default)                                 */
  double reserved[3];
} snk_options;

/* Per-build counters and phase times (CUDA events on the library stream). */
typedef struct {
  int64_t n_points, n_batches, n_shells, n_functions, n_pairs;
  int64_t pairs_kept;          /* sum_j |V_j| (shell pairs)                         */
  int64_t pair_points;         /* sum_j |V_j| |Q_j|                                 */
  double integrals;            /* sum_j sum_{(a,b) in V_j} |Q_j| n_a n_b            */
  double integral_flops;       /* algorithmic FP64 flops of the integral kernel     */
  double gemm_flops;           /* flops of F = X P and Kt = G^T X                    */
  int64_t n_chunks;            /* batch chunks of the last build (Alg. 1)           */
  int64_t workspace_bytes;     /* device workspace held                              */
  int64_t kernel_launches;     /* kernels launched by the last set_density + build  */
  double ms_screen;            /* last set_density: upload, F-tilde, pair screen    */
  double ms_collocation, ms_fgemm, ms_integrals, ms_kgemm, ms_finish; /* last build  */
  double ms_build;             /* last build, first to last event                   */
  double ms_integrals_class[6];/* per class ss ps pp ds dp dd (FP64 lists)          */
  double integrals_class[6];
  double flops_class[6];
  int64_t pairs_kept_fp32;     /* mixed form: kept (batch, pair) entries run in FP32 */
  double integrals_fp32;       /* their integrals                                    */
  double flops_fp32;           /* their algorithmic FP32 flops                       */
  double ms_integrals_fp32;    /* their kernel time                                  */
  int64_t pairs_learned_skipped; /* learned screen: kept by sn-LinK, skipped by the MLP */
  double gemm_flops_hi;        /* the part of gemm_flops on high-tier columns / rows
                                  (SNK_GEMM_SPLIT; equal to gemm_flops otherwise)   */
  double ms_integrals_class_fp32[6]; /* FP32-tier kernel time per class            */
  double colloc_bytes;         /* bytes of X the collocation kernel writes per build:
                                  sum_j ldq_j |B_j| x 8 (ldq_j = |Q_j| padded to 128) */
  double ms_gemm_split;        /* last build: operand preparation of both products
                                  (slicing, splitting, the FP32-tier G merge)       */
  double ms_gemm_hi;           /* last build: both products, high-tier columns / rows */
  double ms_gemm_lo;           /* last build: both products, the remaining ones      */
  double gemm_tc_flops;        /* SNK_GEMM_SPLIT: bf16 tensor-core flops issued per build
                                  (2 M N K per slice product, padded tile sizes)     */
  double pair_points_fp32;     /* last build: FP32-tier (pair, point) evaluations made
                                  (after the tile screen; integrals_fp32 and
                                  flops_fp32 count the same work)                  */
  double pair_points_fp32_listed; /* the same before the tile screen               */
  double ms_xc_collocation;    /* last snk_build_Vxc: Phi and grad Phi               */
  double ms_xc_fgemm;          /*   F = X P                                           */
  double ms_xc_point;          /*   density, functional and Z                        */
  double ms_xc_vgemm;          /*   V-hat += Z^T X and the symmetrisation            */
  double xc_gemm_flops;        /*   flops of its two products (2 |Q_j| |B_j|^2 each) */
  double xc_colloc_bytes;      /*   bytes of Phi and grad Phi written (4 x 8 ldq_j |B_j|) */
} snk_stats;

/* Fill *opt with the defaults: eps_basis = eps_E = eps_K = 1e-12,
 * batch_max = 4096, FP64, sn-LinK screen, fp32_bound = 1e-6, workspace auto. */
void snk_options_default(snk_options *opt);

/* Geometry setup (not density dependent): normalisation, shell pairs with
 * their rigorous integral bounds, octree batches (Sec. II.E), basis screen
 * B_j (Eq. basis_screen) and the batch maxima Phi-tilde, phi-tilde of
 * Eq. (exx_fmat_approx).  opt may be NULL for the defaults. */
int snk_create(const snk_basis *basis, const snk_grid *grid, const snk_options *opt,
               snk_ctx **out);

/* Several independent molecules in one handle (the batched form): molecule m
 * has bases[m] and grids[m].  All later work runs over the batches of every
 * molecule in the same launches; each molecule keeps its own N_b,m x N_b,m
 * density and exchange block.  Shell indices of the debug calls are global
 * (molecule after molecule).  snk_create is the case n_mol = 1. */
int snk_create_batch(int32_t n_mol, const snk_basis *bases, const snk_grid *grids, const snk_options *opt,
                     snk_ctx **out);
int32_t snk_n_molecules(const snk_ctx *ctx);
int64_t snk_molecule_functions(const snk_ctx *ctx, int32_t m);

/* Load the density (symmetric to 1e-12 relative) and run the density-
 * dependent sn-LinK screen: F-tilde (Eq. exx_fmat_approx) and the pair lists
 * V_j (Eq. sp_set).  P is a host pointer to the packed blocks: molecule after
 * molecule, each N_b,m x N_b,m row-major (for one molecule simply the
 * N_b x N_b matrix). */
int snk_set_density(snk_ctx *ctx, const double *P);
/* Same with the packed P in device memory. */
int snk_set_density_device(snk_ctx *ctx, const double *dP);
/* Same from one host pointer per molecule (P[m] is N_b,m x N_b,m). */
int snk_set_density_batch(snk_ctx *ctx, const double *const *P);

/* Build K for the loaded density (Alg. 1 on one GPU).  K is host memory in the
 * packed layout of snk_set_density; the call returns when K is written.
 * Every form is reproducible bit for bit: each G entry of an integral launch
 * has a single writer whose additions come in pair-list order, and the
 * batches' contributions to K are summed as exact 64-bit fixed-point integers
 * (resolution 2^-76, |contribution| < 2^30: a larger or non-finite one gives
 * SNK_ERR_UNSUPPORTED; at most 2^19 grid batches per handle). */
int snk_build_K(snk_ctx *ctx, double *K);
/* Same, writing the packed blocks into device memory; returns once the work
 * is enqueued on the library stream (synchronise it before reading dK). */
int snk_build_K_device(snk_ctx *ctx, double *dK);
/* Same into one host buffer per molecule. */
int snk_build_K_batch(snk_ctx *ctx, double *const *K);

/* Several densities of one molecule in one build (for example the alpha and
 * beta densities of an unrestricted calculation): K_d = sn-K of P_d for each
 * d (Eqs. fmat, gmat, usym_k, sn_k with D = P_d), from one evaluation of every
 * 3c-CP block contracted with every F_d (Eq. gmat).  The screen of Eq.
 * (sp_set) runs once on sum_d |P_d|, an upper bound of each density's
 * estimates, so the kept blocks serve all densities.  n_dens in
 * 1..SNK_MAX_DENSITIES; P[d] host, N_b x N_b row-major, each symmetric
 * (SNK_ERR_NOT_SYMMETRIC otherwise).  Handles made by snk_create only
 * (SNK_ERR_UNSUPPORTED for several molecules); snk_build_K_multi writes K[d]
 * (host) for every loaded density.  snk_set_density loads one density again;
 * graph capture (options.graph) applies to one density only. */
enum { SNK_MAX_DENSITIES = 2 };
int snk_set_density_multi(snk_ctx *ctx, int32_t n_dens, const double *const *P);
int snk_build_K_multi(snk_ctx *ctx, double *const *K);

/* Exchange-correlation potential of the loaded density (Sec. II.C):
 *
 *   F_{mu i} = sum_nu P_{mu nu} Phi_{nu i}                          Eq. (fmat)
 *   rho_i = sum_mu F_{mu i} Phi_{mu i},
 *   grad rho_i = 2 sum_mu F_{mu i} grad Phi_{mu i}                  Eq. (den_grid)
 *   E^rho_i, E^gamma_i = d eps / d rho, d eps / d gamma at r_i      Eq. (exc_grid)
 *   Z_{mu i} = w_i/2 (E^rho_i Phi_{mu i} + 4 E^gamma_i grad rho . grad Phi_{mu i})   Eq. (zmat)
 *   V_{mu nu} = sum_i Phi_{mu i} Z_{nu i} + Z_{mu i} Phi_{nu i}     Eq. (vxc_num)
 *   E_xc = sum_i w_i eps(rho_i, gamma_i)
 *
 * on the handle's grid batches with the basis screen B_j (Phi, F and Z over
 * the functions of B_j only).  eps is a spin-restricted functional (energy per
 * volume, gamma = |grad rho|^2): SNK_XC_LDA_X Slater exchange, SNK_XC_PBE_X
 * PBE exchange, SNK_XC_PBE PBE exchange and correlation (PW92 uniform-gas
 * correlation); points with rho < 1e-14 add nothing.  P is the loaded
 * density as given (no closed-shell factor; one per molecule of a batch
 * handle).  The two products run as FP64 tiles (precision SNK_PREC_FP64),
 * double-FP32 tiles (SNK_PREC_MIXED) or, with gemm SNK_GEMM_SPLIT, as bf16
 * split products on the tcgen05 tensor cores (tc_slices_hi slices);
 * V is summed as exact fixed-point integers like K, so it is the same bit for
 * bit from run to run.  V_out: host (snk_build_Vxc) or device
 * (snk_build_Vxc_device, enqueued on the library stream), the packed
 * molecule blocks like K (N_b x N_b row-major for one molecule); E_xc: host,
 * one double per molecule, may be NULL (snk_build_Vxc_device then returns
 * without waiting for the stream).  SNK_ERR_BAD_STATE before snk_set_density
 * or with several densities loaded; SNK_ERR_INVALID_ARG for an unknown
 * functional or a NULL output.  The first call plans the
 * batches and sizes the V^xc workspace to at most half of the device memory
 * free at that moment (SNK_ERR_OOM if even one batch does not fit); the
 * workspace stays with the handle until snk_destroy. */
enum { SNK_XC_LDA_X = 1, SNK_XC_PBE_X = 2, SNK_XC_PBE = 3 };
int snk_build_Vxc(snk_ctx *ctx, int32_t functional, double *V_out, double *E_xc);
int snk_build_Vxc_device(snk_ctx *ctx, int32_t functional, double *dV, double *E_xc);

/* Autotuner of the integral kernels (after snk_set_density): for every FP32
 * list of the mixed form, times the kernel on the batches of the last
 * workspace chunk for 2..128 shell pairs staged (and tile-screened) per step
 * of a 128-point tile and keeps the fastest; the choice holds for later builds
 * and densities of the handle.  runs (optional, 12 entries: FP64 ss ps pp ds
 * dp dd, then FP32) receives the steps (the FP64 lists take their whole list
 * per tile and do not use theirs). */
int snk_autotune(snk_ctx *ctx, int32_t *runs);

/* Stream for all later work on this handle (a cudaStream_t; NULL = the legacy
 * default stream). */
int snk_set_stream(snk_ctx *ctx, void *stream);

/* Device memory hook (Sec. II.F, Alg. 1: the workspaces of the batches that
 * saturate device memory).  After this call every device buffer of the
 * handle -- geometry tables, density, screen lists, batch workspaces, K --
 * comes from alloc(bytes, user) and goes back through free(ptr, user), so a
 * host such as PyTorch's caching allocator owns all of the handle's memory.
 *   - alloc must return device memory of the handle's device, aligned to 256
 *     bytes, or NULL; NULL makes the call that needed the memory return
 *     SNK_ERR_OOM (the handle stays usable: set_density again, e.g. after a
 *     different allocator was set).  A block that is not 256-byte aligned is
 *     handed back and the call returns SNK_ERR_CUDA.
 *   - free is called only after the handle's stream has drained, so the block
 *     can be reused at once; it is also called from snk_destroy.
 *   - alloc = free = NULL goes back to cudaMalloc / cudaFree.  One of them NULL
 *     alone is SNK_ERR_INVALID_ARG.
 * Buffers that exist already are moved into the new allocator's memory (on
 * failure SNK_ERR_OOM and the handle keeps its old buffers); the loaded
 * density is dropped, so snk_set_density must be called again before a
 * build.  Every block is released the way it was obtained, even when the
 * allocator changes later. */
typedef void *(*snk_alloc_fn)(size_t bytes, void *user);
typedef void (*snk_free_fn)(void *ptr, void *user);
int snk_set_allocator(snk_ctx *ctx, snk_alloc_fn alloc, snk_free_fn free, void *user);

int snk_get_stats(const snk_ctx *ctx, snk_stats *stats);
int64_t snk_n_functions(const snk_ctx *ctx);
const char *snk_last_error(const snk_ctx *ctx);
const char *snk_status_string(int status);
void snk_destroy(snk_ctx *ctx);

/* ---- learned block screen ------------------------------------------------ */

/* A small MLP (16 features -> 64 -> 64 -> 64 -> 1, ReLU) predicts log10/10 of
 * the contribution of a (grid batch, shell pair) block to K.  Features (all
 * computed on the device): l_a, l_b, smallest and largest exponents of both
 * shells, distance from the batch to the pair, |AB|, F-tilde of both shells
 * (the F block norms of Eq. exx_fmat_approx), phi-tilde of the batch, the
 * rigorous batch bound A-tilde, the sn-LinK estimate epsilon^K, batch radius
 * and size.  With options.screen = SNK_SCREEN_LEARNED and weights loaded, a
 * block kept by the rigorous sn-LinK screen is skipped when the prediction is
 * below options.learned_skip (FP16 tensor-core inference, FP32 accumulation);
 * without weights the rigorous screen alone applies (the fallback).
 * Weights: SNK_MLP_WEIGHTS floats, W1[16][64] b1[64] W2[64][64] b2[64]
 * W3[64][64] b3[64] W4[64] b4. */
enum { SNK_MLP_FEATURES = 16, SNK_MLP_WEIGHTS = 9473 };

/* Copies the weights (host) into the handle; later snk_set_density calls use
 * them when options.screen is SNK_SCREEN_LEARNED. */
int snk_screen_load(snk_ctx *ctx, const float *weights);

/* Training data from the plain FP64 method itself, for the loaded density of a
 * handle with the rigorous screen: for the batches j with j % stride == 0
 * (until cap blocks), every kept block's features and label
 * log10(max_u sum_i |dG_u(i)| max_nu |Phi_{nu i}|) / 10, dG_u(i) the block's
 * contribution to G row u at point i: an upper bound of the block's
 * contribution to any K entry, from the block's actual integrals.  n receives
 * the number of blocks written (features: n x 16, labels: n). */
int snk_learn_collect(snk_ctx *ctx, int32_t stride, int64_t cap, float *features, float *labels, int64_t *n);

/* Trains the MLP on the GPU with the library's own kernels (FP32 forward,
 * backward, Adam): mini-batches of `batch` samples, `epochs` passes in a
 * seeded order, loss = mean c r^2 with r = prediction - label and c = 1 for
 * over- and under_weight for under-prediction.  init != 0 draws He-normal
 * weights from seed first; otherwise training continues from *weights.
 * loss_history (optional, epochs entries) receives the mean loss per epoch.
 * Host arrays throughout. */
int snk_mlp_train(const float *features, const float *labels, int64_t n, int32_t epochs, int32_t batch, float lr,
                  float under_weight, uint64_t seed, int32_t init, float *weights, float *loss_history);

/* Forward pass for n feature rows (host arrays): FP32 (f16 = 0) or the FP16
 * tensor-core inference path (f16 = 1). */
int snk_mlp_eval(const float *weights, const float *features, int64_t n, int32_t f16, float *out);

/* Loss and its gradient with respect to every weight (FP32 kernels), for
 * checks against an independent implementation. */
int snk_mlp_grad(const float *weights, const float *features, const float *labels, int64_t n, float under_weight,
                 float *grad, float *loss);

/* ---- test exports: expose intermediate steps for unit parity ------------- */

/* Device Boys function F_0..F_nmax (Eq. boys) at n host values T (host arrays;
 * out is n x (nmax+1)).  nmax <= 4. */
int snk_debug_boys(int64_t n, const double *T, int nmax, double *out);

/* Device 3c-CP integrals A_{mu lam}(r) (Eq. 3c_grid, normalised functions) of
 * shells sa, sb at n host points; out is n x ncart(l_sa) x ncart(l_sb). */
int snk_debug_shell_A(snk_ctx *ctx, int32_t sa, int32_t sb, int64_t n, const double *xyz,
                      double *out);

/* Host-side rigorous bound of max_r |A_{mu lam}(r)| over the shell pair
 * (sa, sb) (the A-tilde of Eq. exx_fmat_approx). */
int snk_debug_pair_bound(snk_ctx *ctx, int32_t sa, int32_t sb, double *bound);

/* The split-product tensor-core GEMM of SNK_GEMM_SPLIT on plain matrices:
 * C = A B^T with A (M x K) and B (N x K) row-major host doubles, C (M x N)
 * row-major host, each operand cut into `slices` (3..6) bf16 slices per row and
 * run of 256 columns (Sec. II.C, Eq. fmat, and Sec. II.D, Eq. usym_k, are
 * this product with the operands of a grid batch). */
int snk_debug_tc_gemm(int32_t M, int32_t N, int32_t K, const double *A, const double *B, int32_t slices,
                      double *C);

/* Failure path of the bounded device waits: one thread waits, with the wait
 * the library's copy and product pipelines use, on a shared-memory mbarrier
 * that nothing completes.  After limit_ns (1 .. 2e9 ns) it gives up and sets
 * the handle's device error flag, and the call returns what a build reports
 * in that case, SNK_ERR_TIMEOUT (SNK_ERR_INVALID_ARG for a limit out of
 * range).  The handle stays usable. */
int snk_debug_wait_timeout(snk_ctx *ctx, int64_t limit_ns);

/* Octree batches: n_batches, then for each batch the point count; the
 * permutation from batch order to input order (n_points entries). */
int snk_debug_batches(snk_ctx *ctx, int64_t *n_batches, int32_t *counts, int64_t counts_cap,
                      int64_t *perm);

/* ---- allocation-free variant -------------------------------------------- */

/* The paper has no counterpart to this entry point: it serves callers that
 * must not call cudaMalloc, such as code that runs while a CUDA graph is being
 * captured or a host that hands out all device memory from its own pool.
 *
 * Same result as snk_debug_shell_A (the 3c-CP block A_{mu lam}(r) of the
 * normalised shells sa, sb at n points, out = n x ncart(l_sa) x ncart(l_sb)),
 * but xyz (3n doubles) and out are DEVICE pointers and the call allocates
 * nothing: the intermediate block goes to a fixed scratch array inside the
 * library, 4096 points x 36 doubles (1.125 MiB), which every GPU that loads
 * the library holds until the process exits.
 *   - n > 4096 returns SNK_ERR_INVALID_ARG; split larger point sets.
 *   - The first call on a device looks the scratch address up (set-up, once
 *     per device) and keeps it for the life of the process's CUDA context;
 *     make that first call before any stream capture.
 *   - The current device must be the handle's device (SNK_ERR_BAD_STATE
 *     otherwise).
 *   - The work is enqueued on the handle's stream (snk_set_stream) and the
 *     call returns without waiting.
 *   - All calls share the one scratch array and it keeps the last call's
 *     contents; calls that overlap on the GPU (other streams, other handles)
 *     race on it.  Order them on one stream. */
int snk_shell_A_noalloc(snk_ctx *ctx, int32_t sa, int32_t sb, int64_t n, const double *xyz,
                        double *out);

#ifdef __cplusplus
}
#endif
#endif /* SNK_H */
