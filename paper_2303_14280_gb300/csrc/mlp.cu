// Learned block screen of libsnk: a small MLP (16 -> 64 -> 64 -> 64 -> 1,
// ReLU) that predicts log10 of a (grid batch, shell pair) block's
// contribution to K from cheap features of the block.
//
//   training (FP32, one thread per sample or per weight): forward with stored
//     activations, backward, gradient reduction over the mini-batch, Adam;
//   inference (FP16 operands, FP32 accumulation on the tensor cores): one
//     warp evaluates 16 blocks with mma.m16n8k16, the accumulator fragments of
//     one layer feeding the next layer's operand fragments in registers.
//
// Weights are one float array in the order W1[16][64] b1[64] W2[64][64]
// b2[64] W3[64][64] b3[64] W4[64] b4 (W[k][n] multiplies input k into unit n).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "snk_internal.h"

namespace snk {

namespace {

constexpr int NIN = kMlpIn, NH = kMlpHidden;
constexpr int OW1 = 0, OB1 = OW1 + NIN * NH, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH,
              OB3 = OW3 + NH * NH, OW4 = OB3 + NH, OB4 = OW4 + NH;
static_assert(OB4 + 1 == kMlpWeights, "weight layout");

// ---------------------------------------------------------------- FP32 forward / backward

// Forward for one sample with the weights in shared memory; stores the three
// hidden pre-activations (z1, z2, z3) if zs != nullptr.  Returns the output.
__device__ float mlp_forward_one(const float* __restrict__ w, const float* x, float* zs) {
  float a[NH], b[NH];
#pragma unroll 4
  for (int n = 0; n < NH; ++n) {
    float s = w[OB1 + n];
    for (int k = 0; k < NIN; ++k) s = fmaf(x[k], w[OW1 + k * NH + n], s);
    if (zs) zs[n] = s;
    a[n] = fmaxf(s, 0.f);
  }
#pragma unroll 4
  for (int n = 0; n < NH; ++n) {
    float s = w[OB2 + n];
    for (int k = 0; k < NH; ++k) s = fmaf(a[k], w[OW2 + k * NH + n], s);
    if (zs) zs[NH + n] = s;
    b[n] = fmaxf(s, 0.f);
  }
#pragma unroll 4
  for (int n = 0; n < NH; ++n) {
    float s = w[OB3 + n];
    for (int k = 0; k < NH; ++k) s = fmaf(b[k], w[OW3 + k * NH + n], s);
    if (zs) zs[2 * NH + n] = s;
    a[n] = fmaxf(s, 0.f);
  }
  float y = w[OB4];
  for (int k = 0; k < NH; ++k) y = fmaf(a[k], w[OW4 + k], y);
  return y;
}

__global__ void mlp_forward_kernel(const float* __restrict__ wg, const float* __restrict__ X, int64_t n,
                                   float* __restrict__ out) {
  __shared__ float w[kMlpWeights];
  for (int e = threadIdx.x; e < kMlpWeights; e += blockDim.x) w[e] = wg[e];
  __syncthreads();
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  float x[NIN];
  for (int k = 0; k < NIN; ++k) x[k] = X[s * NIN + k];
  out[s] = mlp_forward_one(w, x, nullptr);
}

// Asymmetric squared error: L = (1/n) sum_s c_s r_s^2, r = prediction - label,
// c = 1 for over-prediction and c = under_weight for under-prediction (an
// under-predicted block could be skipped wrongly).  Per sample it stores the
// pre-activations and the output gradients dL/dz of every layer.
__global__ void mlp_backward_kernel(const float* __restrict__ wg, const float* __restrict__ X,
                                    const float* __restrict__ Y, const int64_t* __restrict__ idx, int64_t n,
                                    float under_weight,
                                    float* __restrict__ Z /* n x 3NH */, float* __restrict__ D /* n x (3NH+1) */,
                                    float* __restrict__ loss) {
  __shared__ float w[kMlpWeights];
  for (int e = threadIdx.x; e < kMlpWeights; e += blockDim.x) w[e] = wg[e];
  __syncthreads();
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int64_t row = idx ? idx[s] : s;
  float x[NIN];
  for (int k = 0; k < NIN; ++k) x[k] = X[row * NIN + k];
  float* z = Z + s * 3 * NH;
  const float y = mlp_forward_one(w, x, z);
  const float r = y - Y[row];
  const float c = r < 0.f ? under_weight : 1.f;
  atomicAdd(loss, c * r * r / (float)n);
  float* d = D + s * (3 * NH + 1);
  const float dy = 2.f * c * r / (float)n;
  d[3 * NH] = dy;
  // layer 4 -> 3
  float g3[NH], g2[NH];
  for (int k = 0; k < NH; ++k) {
    g3[k] = z[2 * NH + k] > 0.f ? dy * w[OW4 + k] : 0.f;
    d[2 * NH + k] = g3[k];
  }
  for (int k = 0; k < NH; ++k) {
    float s2 = 0.f;
    for (int m = 0; m < NH; ++m) s2 = fmaf(w[OW3 + k * NH + m], g3[m], s2);
    g2[k] = z[NH + k] > 0.f ? s2 : 0.f;
    d[NH + k] = g2[k];
  }
  for (int k = 0; k < NH; ++k) {
    float s1 = 0.f;
    for (int m = 0; m < NH; ++m) s1 = fmaf(w[OW2 + k * NH + m], g2[m], s1);
    d[k] = z[k] > 0.f ? s1 : 0.f;
  }
}

// Gradient of every weight, one thread per weight, summed over the samples:
// dW_l[k][m] = sum_s a_{l-1}[s][k] d_l[s][m], db_l[m] = sum_s d_l[s][m].
__global__ void mlp_grad_reduce_kernel(const float* __restrict__ X, const int64_t* __restrict__ idx,
                                       const float* __restrict__ Z, const float* __restrict__ D, int64_t n,
                                       float* __restrict__ grad) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kMlpWeights) return;
  int layer, k = -1, m;
  if (e < OB1) {
    layer = 0;
    k = (e - OW1) / NH;
    m = (e - OW1) % NH;
  } else if (e < OW2) {
    layer = 0;
    m = e - OB1;
  } else if (e < OB2) {
    layer = 1;
    k = (e - OW2) / NH;
    m = (e - OW2) % NH;
  } else if (e < OW3) {
    layer = 1;
    m = e - OB2;
  } else if (e < OB3) {
    layer = 2;
    k = (e - OW3) / NH;
    m = (e - OW3) % NH;
  } else if (e < OW4) {
    layer = 2;
    m = e - OB3;
  } else if (e < OB4) {
    layer = 3;
    k = e - OW4;
    m = 0;
  } else {
    layer = 3;
    m = 0;
  }
  double acc = 0.0;  // FP64 sum over the samples (off the hot path)
  for (int64_t s = 0; s < n; ++s) {
    const float* d = D + s * (3 * NH + 1);
    const float dz = layer == 3 ? d[3 * NH] : d[layer * NH + m];
    float a = 1.f;
    if (k >= 0) {
      if (layer == 0)
        a = X[(idx ? idx[s] : s) * NIN + k];
      else
        a = fmaxf(Z[s * 3 * NH + (layer - 1) * NH + k], 0.f);
    }
    acc += (double)a * dz;
  }
  grad[e] = (float)acc;
}

__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m1,
                            float* __restrict__ m2, int t, float lr, float b1, float b2, float eps) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kMlpWeights) return;
  m1[e] = b1 * m1[e] + (1.f - b1) * g[e];
  m2[e] = b2 * m2[e] + (1.f - b2) * g[e] * g[e];
  const float mh = m1[e] / (1.f - powf(b1, (float)t)), vh = m2[e] / (1.f - powf(b2, (float)t));
  w[e] -= lr * mh / (sqrtf(vh) + eps);
}

// ---------------------------------------------------------------- FP16 tensor-core inference

__device__ __forceinline__ uint32_t pack_half2(float lo, float hi) {
  __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ void mma_f16(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Weights in shared memory as FP16 B fragments: for a layer with K inputs and
// N outputs, Wh[k][n] (row-major, k fastest per column pair); biases FP32.
struct MlpSmem {
  __half w1[NIN * NH];
  __half w2[NH * NH];
  __half w3[NH * NH];
  __half w4[NH * 8];  // output column 0, columns 1..7 zero
  float b1[NH], b2[NH], b3[NH], b4;
};

__device__ void load_mlp_smem(MlpSmem* sm, const float* __restrict__ wg) {
  for (int e = threadIdx.x; e < NIN * NH; e += blockDim.x) sm->w1[e] = __float2half_rn(wg[OW1 + e]);
  for (int e = threadIdx.x; e < NH * NH; e += blockDim.x) {
    sm->w2[e] = __float2half_rn(wg[OW2 + e]);
    sm->w3[e] = __float2half_rn(wg[OW3 + e]);
  }
  for (int e = threadIdx.x; e < NH * 8; e += blockDim.x)
    sm->w4[e] = (e % 8 == 0) ? __float2half_rn(wg[OW4 + e / 8]) : __float2half_rn(0.f);
  for (int e = threadIdx.x; e < NH; e += blockDim.x) {
    sm->b1[e] = wg[OB1 + e];
    sm->b2[e] = wg[OB2 + e];
    sm->b3[e] = wg[OB3 + e];
  }
  if (threadIdx.x == 0) sm->b4 = wg[OB4];
}

// B fragment of mma.m16n8k16 for columns [n0, n0+8), rows [k0, k0+16) of a
// row-major K x N half matrix W: b0 = (k0+2t, k0+2t+1; col n0+g), b1 = (+8).
__device__ __forceinline__ void load_b(const __half* W, int N, int k0, int n0, int lane, uint32_t* b) {
  const int g = lane >> 2, t = lane & 3;
  __half2 v0 = __halves2half2(W[(k0 + 2 * t) * N + n0 + g], W[(k0 + 2 * t + 1) * N + n0 + g]);
  __half2 v1 = __halves2half2(W[(k0 + 2 * t + 8) * N + n0 + g], W[(k0 + 2 * t + 9) * N + n0 + g]);
  b[0] = *reinterpret_cast<uint32_t*>(&v0);
  b[1] = *reinterpret_cast<uint32_t*>(&v1);
}

// One hidden layer on the tensor cores: in = A fragments of KT k-slices (16
// columns each) of the 16 x (16 KT) input; out = A fragments of the 16 x 64
// ReLU output (4 k-slices), built directly from the accumulator fragments.
template <int KT>
__device__ __forceinline__ void mlp_layer(const uint32_t (*in)[4], const __half* W, const float* bias, int lane,
                                          uint32_t (*out)[4]) {
  const int t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < NH / 8; ++nt) {
    float c[4] = {bias[nt * 8 + 2 * t], bias[nt * 8 + 2 * t + 1], bias[nt * 8 + 2 * t], bias[nt * 8 + 2 * t + 1]};
#pragma unroll
    for (int ks = 0; ks < KT; ++ks) {
      uint32_t b[2];
      load_b(W, NH, ks * 16, nt * 8, lane, b);
      mma_f16(c, in[ks], b);
    }
    // accumulator (row g / g+8, columns nt*8 + 2t, +1) -> operand of slice nt/2
    const int s = nt >> 1, h = nt & 1;
    out[s][2 * h] = pack_half2(fmaxf(c[0], 0.f), fmaxf(c[1], 0.f));
    out[s][2 * h + 1] = pack_half2(fmaxf(c[2], 0.f), fmaxf(c[3], 0.f));
  }
}

// 16 samples per warp: x holds the warp's 16 feature rows (row r in lanes
// 4r..4r+3 as in the A fragment).  Returns the prediction of rows g and g+8 in
// lanes with t == 0 (column 0 of the output tile).
__device__ __forceinline__ void mlp_infer16(const MlpSmem* sm, const uint32_t* a_in, int lane, float* y_g,
                                            float* y_g8) {
  uint32_t in1[1][4] = {{a_in[0], a_in[1], a_in[2], a_in[3]}};
  uint32_t h1[4][4], h2[4][4], h3[4][4];
  mlp_layer<1>(in1, sm->w1, sm->b1, lane, h1);
  mlp_layer<4>(h1, sm->w2, sm->b2, lane, h2);
  mlp_layer<4>(h2, sm->w3, sm->b3, lane, h3);
  float c[4] = {sm->b4, 0.f, sm->b4, 0.f};
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) {
    uint32_t b[2];
    load_b(sm->w4, 8, ks * 16, 0, lane, b);
    mma_f16(c, h3[ks], b);
  }
  *y_g = c[0];
  *y_g8 = c[2];
}

// Inference over n feature rows (FP16 tensor cores) for tests and tuning.
__global__ void mlp_infer_kernel(const float* __restrict__ wg, const float* __restrict__ X, int64_t n,
                                 float* __restrict__ out) {
  __shared__ MlpSmem sm;
  load_mlp_smem(&sm, wg);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t base = (blockIdx.x * (int64_t)(blockDim.x >> 5) + warp) * 16;
  if (base >= n) return;
  const int g = lane >> 2, t = lane & 3;
  auto feat = [&](int64_t r, int k) { return r < n ? X[r * NIN + k] : 0.f; };
  uint32_t a[4] = {pack_half2(feat(base + g, 2 * t), feat(base + g, 2 * t + 1)),
                   pack_half2(feat(base + g + 8, 2 * t), feat(base + g + 8, 2 * t + 1)),
                   pack_half2(feat(base + g, 2 * t + 8), feat(base + g, 2 * t + 9)),
                   pack_half2(feat(base + g + 8, 2 * t + 8), feat(base + g + 8, 2 * t + 9))};
  float y0, y1;
  mlp_infer16(&sm, a, lane, &y0, &y1);
  if (t == 0) {
    if (base + g < n) out[base + g] = y0;
    if (base + g + 8 < n) out[base + g + 8] = y1;
  }
}

}  // namespace

// ---------------------------------------------------------------- block features

// Features of block (batch j, pair p) for the learned screen (fixed affine
// scalings, no learned normalisation):
//   l_a/2, l_b/2, log10 of the smallest and largest exponents of a and b (/3),
//   distance from the batch sphere to the segment AB (/10 bohr), |AB| (/10),
//   log10 F-tilde_a, F-tilde_b, phi-tilde_j, the batch bound A-tilde_j and the
//   sn-LinK estimate epsilon^K (/10), the batch radius (/10), log10 |Q_j| (/4).
// log10(max(x, 1e-40)) of a double through its binary exponent and an FP32
// log of the mantissa: no FP64 transcendental.
__device__ __forceinline__ float log10_clamped(double x) {
  int e;
  const float m = (float)frexp(fmax(x, 1e-40), &e);  // x = m 2^e, m in [0.5, 1)
  return log10f(m) + (float)e * 0.30102999566f;
}

__device__ void block_features(const ScreenArgs& a, const BatchDesc& bd, int j, int p, const PairHdr& h,
                               const float* __restrict__ shell_feat, float* f) {
  // geometry in FP32 and logs through log10_clamped: the FP64 pipe is 1/64 of
  // the FP32 rate on this GPU, and the features feed an FP16 network
  const double* ft = a.ft_shell + bd.cm_off;
  const double fa = ft[h.sa - bd.ms0], fb = ft[h.sb - bd.ms0];
  const double* A = a.shell_xyz + 3 * h.sa;
  const float vx = (float)-h.ABx, vy = (float)-h.ABy, vz = (float)-h.ABz;
  const float wx = (float)(a.bcenter[3 * j] - A[0]), wy = (float)(a.bcenter[3 * j + 1] - A[1]),
              wz = (float)(a.bcenter[3 * j + 2] - A[2]);
  const float vv = vx * vx + vy * vy + vz * vz;
  float t = vv > 0.f ? __fdividef(wx * vx + wy * vy + wz * vz, vv) : 0.f;
  t = fminf(fmaxf(t, 0.f), 1.f);
  const float dx = wx - t * vx, dy = wy - t * vy, dz = wz - t * vz;
  const float rad = (float)a.bradius[j];
  const float d = fmaxf(sqrtf(dx * dx + dy * dy + dz * dz) - rad, 0.f);
  double bnd = a.bound[p];
  if (d > 0.f) bnd = fmin(bnd, a.qbound[p] * (double)(1.0f / d));
  const double eK = fmax(fa, fb) * a.phit_b[j] * bnd;
  f[0] = shell_feat[4 * h.sa + 0];  // l / 2
  f[1] = shell_feat[4 * h.sb + 0];
  f[2] = shell_feat[4 * h.sa + 1];  // log10 min exponent / 3
  f[3] = shell_feat[4 * h.sb + 1];
  f[4] = shell_feat[4 * h.sa + 2];  // log10 max exponent / 3
  f[5] = shell_feat[4 * h.sb + 2];
  f[6] = d / 10.f;
  f[7] = sqrtf(vv) / 10.f;
  f[8] = log10_clamped(fa) / 10.f;
  f[9] = log10_clamped(fb) / 10.f;
  f[10] = log10_clamped(a.phit_b[j]) / 10.f;
  f[11] = log10_clamped(bnd) / 10.f;
  f[12] = log10_clamped(eK) / 10.f;
  f[13] = rad / 10.f;
  f[14] = log10f((float)bd.q) / 4.f;
  f[15] = 1.f;
}

namespace {

// Features of every entry of the sampled batches' lists (collection of
// training data): entry slot = sample offset of the batch + position in its lists.
__global__ void features_kernel(ScreenArgs a, const int* __restrict__ pairlist, const int64_t* __restrict__ list_off,
                                const int* __restrict__ counts, const int* __restrict__ sample_batches,
                                const int64_t* __restrict__ sample_off, const float* __restrict__ shell_feat,
                                float* __restrict__ feat) {
  const int j = sample_batches[blockIdx.x];
  const BatchDesc bd = a.batches[j];
  const int64_t b0 = list_off[(int64_t)j * kNumLists];
  int64_t tot = 0;
  for (int L = 0; L < kNumLists; ++L) tot += counts[(int64_t)j * kNumLists + L];
  for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
    const int p = pairlist[b0 + e];
    float f[kMlpIn];
    block_features(a, bd, j, p, a.pairs[p], shell_feat, f);
    float* o = feat + (sample_off[blockIdx.x] + e) * kMlpIn;
    for (int k = 0; k < kMlpIn; ++k) o[k] = f[k];
  }
}

constexpr int kFilterSplit = 8;  // blocks per batch of the learned filter (balances the last wave)

// Learned screen: for every entry of batch j's lists, predict log10 of the
// block's contribution to K and clear its keep flag if the prediction is below
// skip_log10.  One warp evaluates 16 entries at a time on the tensor cores.
// Entries of the FP64 (high-tier) lists predicted below fp32_log10 are
// marked 2: they move to the FP32 list of their class.
__global__ void __launch_bounds__(128) learned_filter_kernel(ScreenArgs a, const float* __restrict__ wg,
                                                             const int* __restrict__ pairlist,
                                                             const int64_t* __restrict__ list_off,
                                                             const int* __restrict__ counts,
                                                             const float* __restrict__ shell_feat, float skip_log10,
                                                             float fp32_log10, unsigned char* __restrict__ keep) {
  __shared__ MlpSmem sm;
  __shared__ float fbuf[4][16][kMlpIn + 1];
  load_mlp_smem(&sm, wg);
  __syncthreads();
  const int j = blockIdx.x;
  const BatchDesc bd = a.batches[j];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int64_t b0 = list_off[(int64_t)j * kNumLists];
  int64_t tot = 0, n64 = 0;
  for (int L = 0; L < kNumLists; ++L) tot += counts[(int64_t)j * kNumLists + L];
  for (int L = 0; L < kNumClasses; ++L) n64 += counts[(int64_t)j * kNumLists + L];
  // the batch's entries are shared by gridDim.y blocks, 16 per warp step
  for (int64_t base = ((int64_t)blockIdx.y * 4 + warp) * 16; base < tot; base += (int64_t)gridDim.y * 4 * 16) {
    // lanes 0..15 compute one row of features each
    if (lane < 16) {
      const int64_t e = base + lane;
      float f[kMlpIn];
      if (e < tot) {
        const int p = pairlist[b0 + e];
        block_features(a, bd, j, p, a.pairs[p], shell_feat, f);
      } else {
        for (int k = 0; k < kMlpIn; ++k) f[k] = 0.f;
      }
      for (int k = 0; k < kMlpIn; ++k) fbuf[warp][lane][k] = f[k];
    }
    __syncwarp();
    uint32_t in[4] = {pack_half2(fbuf[warp][g][2 * t], fbuf[warp][g][2 * t + 1]),
                      pack_half2(fbuf[warp][g + 8][2 * t], fbuf[warp][g + 8][2 * t + 1]),
                      pack_half2(fbuf[warp][g][2 * t + 8], fbuf[warp][g][2 * t + 9]),
                      pack_half2(fbuf[warp][g + 8][2 * t + 8], fbuf[warp][g + 8][2 * t + 9])};
    float y0, y1;
    mlp_infer16(&sm, in, lane, &y0, &y1);
    if (t == 0) {
      // labels are trained as log10(contribution) / 10
      const int64_t e0 = base + g, e1 = base + g + 8;
      if (e0 < tot) keep[b0 + e0] = 10.f * y0 < skip_log10 ? 0 : (e0 < n64 && 10.f * y0 < fp32_log10) ? 2 : 1;
      if (e1 < tot) keep[b0 + e1] = 10.f * y1 < skip_log10 ? 0 : (e1 < n64 && 10.f * y1 < fp32_log10) ? 2 : 1;
    }
    __syncwarp();
  }
}

// Block-wide stream compaction of one list segment: appends the entries of
// src[0, n) whose code equals `want` to dst[out...]; returns the new out.
__device__ int append_coded(const int* __restrict__ src, const unsigned char* __restrict__ code, int n,
                            unsigned char want, int* __restrict__ dst, int out, const PairHdr* __restrict__ pairs,
                            bool fp32, unsigned long long* s_pp, int* warp_tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int base = 0; base < n; base += 256) {
    const int e = base + threadIdx.x;
    const bool k = e < n && code[e] == want;
    const int v = k ? src[e] : 0;
    const unsigned bal = __ballot_sync(0xffffffffu, k);
    if (lane == 0) warp_tot[warp] = __popc(bal);
    __syncthreads();
    int before = 0, total = 0;
    for (int q = 0; q < 8; ++q) {
      before += q < warp ? warp_tot[q] : 0;
      total += warp_tot[q];
    }
    if (k) {
      dst[out + before + __popc(bal & ((1u << lane) - 1u))] = v;
      atomicAdd(s_pp, (unsigned long long)(fp32 ? pairs[v].pp_n32 : pairs[v].pp_n));
    }
    out += total;
    __syncthreads();  // warp_tot is rewritten by the next chunk
  }
  return out;
}

// One block per batch: rewrites the batch's twelve lists into dst (same
// batch base, order kept): a high-tier list keeps its code-1 entries, an
// FP32 list its own code-1 entries followed by the code-2 entries of the
// high-tier list of its class.  New offsets and counts replace the old ones;
// the batch's high-tier shell flags are re-marked from the final lists.
__global__ void __launch_bounds__(256) reorder_lists_kernel(const int* __restrict__ src, int* __restrict__ dst,
                                                            int64_t* __restrict__ list_off, int* __restrict__ counts,
                                                            const unsigned char* __restrict__ keep,
                                                            const PairHdr* __restrict__ pairs,
                                                            long long* __restrict__ ppcounts,
                                                            const BatchDesc* __restrict__ batches,
                                                            const MolDesc* __restrict__ mols,
                                                            unsigned char* __restrict__ hflag) {
  __shared__ unsigned long long s_pp;
  __shared__ int warp_tot[8];
  __shared__ int64_t s_off[kNumLists];
  __shared__ int s_n[kNumLists];
  const int j = blockIdx.x;
  const int64_t seg0 = (int64_t)j * kNumLists;
  if (threadIdx.x < kNumLists) {
    s_off[threadIdx.x] = list_off[seg0 + threadIdx.x];
    s_n[threadIdx.x] = counts[seg0 + threadIdx.x];
  }
  __syncthreads();
  const int64_t b0 = s_off[0];
  int out = 0;
  int64_t new_off[kNumLists];
  int new_n[kNumLists];
  unsigned long long new_pp[kNumLists];
  for (int k = 0; k < kNumLists; ++k) {
    if (threadIdx.x == 0) s_pp = 0ull;
    __syncthreads();
    const int start = out;
    out = append_coded(src + s_off[k], keep + s_off[k], s_n[k], 1, dst + b0, out, pairs, k >= kNumClasses, &s_pp,
                       warp_tot);
    if (k >= kNumClasses) {
      const int h = k - kNumClasses;
      out = append_coded(src + s_off[h], keep + s_off[h], s_n[h], 2, dst + b0, out, pairs, true, &s_pp, warp_tot);
    }
    new_off[k] = b0 + start;
    new_n[k] = out - start;
    new_pp[k] = s_pp;
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < kNumLists; ++k) {
      list_off[seg0 + k] = new_off[k];
      counts[seg0 + k] = new_n[k];
      ppcounts[seg0 + k] = (long long)new_pp[k];
    }
  // high-tier shells of the final lists
  const BatchDesc bd = batches[j];
  const MolDesc md = mols[bd.mol];
  unsigned char* hl = hflag + bd.cm_off;
  for (int a = threadIdx.x; a < md.ns; a += blockDim.x) hl[a] = 0;
  __syncthreads();
  const int nhi = (int)(new_off[kNumClasses] - b0);
  for (int e = threadIdx.x; e < nhi; e += blockDim.x) {
    const PairHdr h = pairs[dst[b0 + e]];
    hl[h.sa - bd.ms0] = 1;
    hl[h.sb - bd.ms0] = 1;
  }
}

}  // namespace

// ---------------------------------------------------------------- launchers

cudaError_t launch_mlp_forward(cudaStream_t st, const float* w, const float* X, int64_t n, float* out, bool f16) {
  if (n == 0) return cudaSuccess;
  if (f16)
    mlp_infer_kernel<<<(unsigned)((n + 63) / 64), 128, 0, st>>>(w, X, n, out);
  else
    mlp_forward_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(w, X, n, out);
  return cudaGetLastError();
}

cudaError_t launch_mlp_grad(cudaStream_t st, const float* w, const float* X, const float* Y, const int64_t* idx,
                            int64_t n, float under_weight, float* Z, float* D, float* grad, float* loss) {
  if (n == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), st);
  if (e != cudaSuccess) return e;
  mlp_backward_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(w, X, Y, idx, n, under_weight, Z, D, loss);
  mlp_grad_reduce_kernel<<<(kMlpWeights + 127) / 128, 128, 0, st>>>(X, idx, Z, D, n, grad);
  return cudaGetLastError();
}

cudaError_t launch_adam(cudaStream_t st, float* w, const float* g, float* m1, float* m2, int t, float lr) {
  adam_kernel<<<(kMlpWeights + 127) / 128, 128, 0, st>>>(w, g, m1, m2, t, lr, 0.9f, 0.999f, 1e-8f);
  return cudaGetLastError();
}

cudaError_t launch_features(cudaStream_t st, const ScreenArgs& a, const int* pairlist, const int64_t* list_off,
                            const int* counts, const int* sample_batches, const int64_t* sample_off, int n_sample,
                            const float* shell_feat, float* feat) {
  if (n_sample == 0) return cudaSuccess;
  features_kernel<<<n_sample, 128, 0, st>>>(a, pairlist, list_off, counts, sample_batches, sample_off, shell_feat,
                                            feat);
  return cudaGetLastError();
}

cudaError_t launch_learned_filter(cudaStream_t st, const ScreenArgs& a, int nbatch, const float* w,
                                  const int* pairlist, int* pairlist_out, int64_t* list_off, int* counts,
                                  long long* ppcounts, const float* shell_feat, float skip_log10, float fp32_log10,
                                  unsigned char* keep, unsigned char* hflag) {
  if (nbatch == 0) return cudaSuccess;
  learned_filter_kernel<<<dim3(nbatch, kFilterSplit), 128, 0, st>>>(a, w, pairlist, list_off, counts, shell_feat, skip_log10, fp32_log10,
                                                keep);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  reorder_lists_kernel<<<nbatch, 256, 0, st>>>(pairlist, pairlist_out, list_off, counts, keep, a.pairs, ppcounts,
                                               a.batches, a.mols, hflag);
  return cudaGetLastError();
}

}  // namespace snk
