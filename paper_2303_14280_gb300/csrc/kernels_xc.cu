// Exchange-correlation potential of libsnk (sm_103a), Sec. II.C:
//
//   Phi_{mu i}, grad Phi_{mu i}                         Eq. (collocation)
//   F_j = X_j P[B_j, B_j]                                Eq. (fmat)       (products below)
//   rho_i = sum_mu F_{mu i} Phi_{mu i},
//   grad rho_i = 2 sum_mu F_{mu i} grad Phi_{mu i}       Eq. (den_grid)
//   eps, d eps / d rho, d eps / d gamma at each point    Eq. (exc_grid)
//   Z_{mu i} = w_i/2 (E^rho Phi + 4 E^gamma grad rho . grad Phi)   Eq. (zmat)
//   V-hat += Z_j^T X_j, V = V-hat + V-hat^T              Eq. (vxc_num)
//
// The two products are FP64 or double-FP32 tiles (kernels_dense.cu) or the
// tcgen05 split products (kernels_ozaki.cu, plain column-major epilogue for F
// and the fixed-point scatter for V-hat).
// per batch of the handle's octree, in the same column-major layout as the
// exchange build (point index fastest, leading dimension ldq): X, dX/dx,
// dX/dy, dX/dz and F (overwritten by Z) are five consecutive ldq x nB blocks.
// One thread per grid point for the collocation and the point kernel, so
// every load and store of a warp is one coalesced 256-byte row.  E_xc is
// summed per warp in a fixed order and then as an exact fixed-point integer
// (khat_add), so it is the same bit for bit from run to run, like V.
//
// Functionals (spin-restricted, energy per volume eps(rho, gamma), gamma =
// |grad rho|^2), from their published definitions:
//   SNK_XC_LDA_X  Slater exchange, C_x rho^{4/3}, C_x = -(3/4)(3/pi)^{1/3}
//   SNK_XC_PBE_X  PBE exchange: C_x rho^{4/3} (1 + kappa - kappa / (1 + mu s^2 / kappa)),
//                 s^2 = gamma / (4 (3 pi^2)^{2/3} rho^{8/3}), kappa = 0.804, mu = beta pi^2 / 3
//   SNK_XC_PBE    PBE exchange + PBE correlation rho (e_c(r_s) + H): e_c the PW92
//                 parametrisation of the uniform gas, H = g ln(1 + (beta/g) t^2
//                 (1 + A t^2) / (1 + A t^2 + A^2 t^4)), A = (beta/g) / (e^{-e_c/g} - 1),
//                 t^2 = pi gamma / (16 k_F rho^2), g = (1 - ln 2) / pi^2
// Points with rho below 1e-14 contribute nothing.
#include <cuda_runtime.h>

#include <cstdint>

#include "snk_internal.h"

namespace snk {

namespace {

constexpr int XC_THREADS = 128, XC_SHELLS = 8;
constexpr double kXcRhoMin = 1e-14;
constexpr double kXcExpCut = 60.0;  // alpha r^2 beyond which a primitive is left out of X and grad X
constexpr double kPi = 3.14159265358979323846;

__device__ __forceinline__ double pw_int(double x, int n) {  // x^n for n = 0, 1, 2 (0 for n < 0)
  return n <= 0 ? (n == 0 ? 1.0 : 0.0) : (n == 1 ? x : x * x);
}

// X and its gradient on the batch's points, shell by shell of B_j.
__global__ void __launch_bounds__(XC_THREADS)
    xc_colloc_kernel(const BatchDesc* __restrict__ batches, const int* __restrict__ bshell,
                     const int* __restrict__ bshell_col, const double* __restrict__ xyz, DeviceBasis B,
                     double* __restrict__ ws) {
  const BatchDesc bd = batches[blockIdx.z];
  const int i = blockIdx.x * XC_THREADS + threadIdx.x;
  const int t0 = blockIdx.y * XC_SHELLS;
  if (i >= bd.ldq || t0 >= bd.nBshell) return;
  const int t1 = min(t0 + XC_SHELLS, bd.nBshell);
  const bool valid = i < bd.q;
  double px = 0.0, py = 0.0, pz = 0.0;
  if (valid) {
    px = xyz[3 * (bd.p0 + i)];
    py = xyz[3 * (bd.p0 + i) + 1];
    pz = xyz[3 * (bd.p0 + i) + 2];
  }
  const int64_t blk = (int64_t)bd.nB * bd.ldq;  // X, d/dx, d/dy, d/dz blocks
  double* X = ws + bd.xoff + i;
  for (int t = t0; t < t1; ++t) {
    const int sh = bshell[bd.bshell_off + t];
    const int col = bshell_col[bd.bshell_off + t];
    const int l = B.l[sh];
    const int nc = (l + 1) * (l + 2) / 2;
    double* out = X + (int64_t)col * bd.ldq;
    if (!valid) {
      for (int c = 0; c < nc; ++c)
        for (int q = 0; q < 4; ++q) out[q * blk + (int64_t)c * bd.ldq] = 0.0;
      continue;
    }
    const double d[3] = {px - B.center[3 * sh], py - B.center[3 * sh + 1], pz - B.center[3 * sh + 2]};
    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    // radial part and its derivative over r^2 (times 2): sum d_k e^{-a_k r^2}, sum -2 a_k d_k e^{-a_k r^2}
    double R0 = 0.0, R1 = 0.0;
    for (int k = B.poff[sh]; k < B.poff[sh] + B.nprim[sh]; ++k) {
      const double x = B.exps[k] * r2;
      if (x >= kXcExpCut) continue;  // e^{-60} ~ 9e-27: nothing representable next to the rest
      const double e = B.d[k] * exp(-x);
      R0 += e;
      R1 = fma(-2.0 * B.exps[k], e, R1);
    }
    const double* fc = B.fcomp + B.foff[sh];
    // Cartesian exponents in the library's lexicographic order
    int c = 0;
    for (int ax = l; ax >= 0; --ax)
      for (int ay = l - ax; ay >= 0; --ay, ++c) {
        const int az = l - ax - ay;
        const int e[3] = {ax, ay, az};
        const double m[3] = {pw_int(d[0], ax), pw_int(d[1], ay), pw_int(d[2], az)};
        const double mono = m[0] * m[1] * m[2];
        const double f = fc[c];
        out[(int64_t)c * bd.ldq] = f * mono * R0;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          // d/dq: e_q q^{e_q - 1} (other factors) R0 + monomial q R1
          const double others = m[(q + 1) % 3] * m[(q + 2) % 3];
          const double dm = e[q] > 0 ? e[q] * pw_int(d[q], e[q] - 1) * others : 0.0;
          out[(q + 1) * blk + (int64_t)c * bd.ldq] = f * fma(dm, R0, mono * d[q] * R1);
        }
      }
  }
}

// PW92 correlation energy per electron of the unpolarised gas and d e_c / d r_s.
__device__ __forceinline__ void pw92_unpol(double rs, double& ec, double& dec) {
  constexpr double a = 0.031091, a1 = 0.21370, b1 = 7.5957, b2 = 3.5876, b3 = 1.6382, b4 = 0.49294;
  const double q = sqrt(rs);
  const double den = 2.0 * a * (q * (b1 + q * (b2 + q * (b3 + q * b4)))); // 2a (b1 rs^1/2 + b2 rs + b3 rs^3/2 + b4 rs^2)
  const double dden = 2.0 * a * (0.5 * b1 / q + b2 + 1.5 * b3 * q + 2.0 * b4 * rs);
  const double L = log1p(1.0 / den);
  const double pre = -2.0 * a * (1.0 + a1 * rs);
  ec = pre * L;
  // d/drs: -2 a a1 L + pre * d L / d den * dden, with d L / d den = -1 / (den (den + 1))
  dec = -2.0 * a * a1 * L - pre * dden / (den * (den + 1.0));
}

// eps, d eps / d rho, d eps / d gamma of functional fn at (rho, gamma), rho >= kXcRhoMin.
__device__ __forceinline__ void xc_eval(int fn, double rho, double gamma, double& e, double& vr, double& vg) {
  constexpr double kappa = 0.804, beta = 0.06672455060314922;
  const double cx = -0.75 * cbrt(3.0 / kPi);
  const double rho13 = cbrt(rho);
  const double ex_lda = cx * rho * rho13;  // C_x rho^{4/3}
  if (fn == SNK_XC_LDA_X) {
    e = ex_lda;
    vr = (4.0 / 3.0) * cx * rho13;
    vg = 0.0;
    return;
  }
  // PBE exchange in x = s^2 = c_s gamma rho^{-8/3}
  const double kf = cbrt(3.0 * kPi * kPi) * rho13;  // (3 pi^2 rho)^{1/3}
  const double inv4kf2rho2 = 1.0 / (4.0 * kf * kf * rho * rho);
  const double x = gamma * inv4kf2rho2;
  const double mu = beta * kPi * kPi / 3.0;
  const double u = 1.0 / (1.0 + (mu / kappa) * x);
  const double Fx = 1.0 + kappa * (1.0 - u);     // 1 + kappa - kappa / (1 + mu x / kappa)
  const double dFx = mu * u * u;                  // dF_x / dx
  e = ex_lda * Fx;
  // x scales as rho^{-8/3}: d x / d rho = -8x / (3 rho)
  vr = (4.0 / 3.0) * cx * rho13 * Fx - ex_lda * dFx * (8.0 / 3.0) * x / rho;
  vg = ex_lda * dFx * inv4kf2rho2;
  if (fn != SNK_XC_PBE) return;
  // PBE correlation
  const double g = (1.0 - log(2.0)) / (kPi * kPi);
  const double rs = cbrt(3.0 / (4.0 * kPi)) / rho13;
  double ec, dec_drs;
  pw92_unpol(rs, ec, dec_drs);
  const double dec_drho = -dec_drs * rs / (3.0 * rho);
  const double ct = kPi / (16.0 * kf * rho * rho);  // t^2 = ct gamma
  const double t2 = ct * gamma;
  const double ex = exp(-ec / g);
  const double A = (beta / g) / (ex - 1.0);
  const double At2 = A * t2;
  const double num = 1.0 + At2, den = 1.0 + At2 + At2 * At2;
  const double y = t2 * num / den;                 // H = g ln(1 + (beta/g) y)
  const double H = g * log1p((beta / g) * y);
  const double dH_dy = beta / (1.0 + (beta / g) * y);
  // y(t2, A) = t2 (1 + A t2) / (1 + A t2 + A^2 t2^2); with z = A t2:
  //   dy/dt2 = (1 + 2z) / den - t2 num (A + 2 A z) / den^2,  dy/dA = t2^2 / den - t2 num (t2 + 2 t2 z) / den^2
  const double dy_dt2 = (1.0 + 2.0 * At2) / den - t2 * num * A * (1.0 + 2.0 * At2) / (den * den);
  const double dy_dA = t2 * t2 / den - t2 * t2 * num * (1.0 + 2.0 * At2) / (den * den);
  const double dA_dec = A * A * ex / beta;         // A = (beta/g) / (e^{-ec/g} - 1)
  const double dt2_drho = -(7.0 / 3.0) * t2 / rho; // t^2 scales as rho^{-7/3} at fixed gamma
  e += rho * (ec + H);
  vr += ec + H + rho * (dec_drho + dH_dy * (dy_dA * dA_dec * dec_drho + dy_dt2 * dt2_drho));
  vg += rho * dH_dy * dy_dt2 * ct;
}

// Density and gradient at each point (Eq. den_grid), the functional (Eq.
// exc_grid), Z over F's block (Eq. zmat) and the point's w eps into E-hat.
__global__ void __launch_bounds__(XC_THREADS)
    xc_point_kernel(const BatchDesc* __restrict__ batches, const double* __restrict__ w, int fn,
                    double* __restrict__ ws, unsigned long long* __restrict__ Ehat, int* err) {
  const BatchDesc bd = batches[blockIdx.y];
  const int i = blockIdx.x * XC_THREADS + threadIdx.x;
  if (blockIdx.x * XC_THREADS >= bd.ldq) return;  // whole block outside the batch (block-uniform)
  const int64_t blk = (int64_t)bd.nB * bd.ldq;
  const double* X = ws + bd.xoff + i;
  double* F = ws + bd.foff + i;
  double we = 0.0;
  if (i < bd.q) {
    double rho = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int mu = 0; mu < bd.nB; ++mu) {
      const int64_t o = (int64_t)mu * bd.ldq;
      const double f = F[o];
      rho = fma(f, X[o], rho);
      gx = fma(f, X[blk + o], gx);
      gy = fma(f, X[2 * blk + o], gy);
      gz = fma(f, X[3 * blk + o], gz);
    }
    gx *= 2.0;
    gy *= 2.0;
    gz *= 2.0;
    double vr = 0.0, vg = 0.0;
    if (rho >= kXcRhoMin) {
      double e;
      xc_eval(fn, rho, gx * gx + gy * gy + gz * gz, e, vr, vg);
      we = w[bd.p0 + i] * e;
    }
    const double hw = 0.5 * w[bd.p0 + i];
    const double a = hw * vr, b = 4.0 * hw * vg;
    for (int mu = 0; mu < bd.nB; ++mu) {
      const int64_t o = (int64_t)mu * bd.ldq;
      const double gg = gx * X[blk + o] + gy * X[2 * blk + o] + gz * X[3 * blk + o];
      F[o] = fma(a, X[o], b * gg);
    }
  }
  // the warp's w eps in a fixed order, then one exact fixed-point addition
  // into the batch's molecule
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) we += __shfl_down_sync(0xffffffffu, we, s);
  if ((threadIdx.x & 31) == 0 && we != 0.0) khat_add(Ehat + 2 * bd.mol, we, err);
}

// V = V-hat + V-hat^T in every molecule block of the packed matrices, and
// each molecule's E_xc, from their fixed-point sums.
__global__ void xc_finish_kernel(const MolDesc* __restrict__ mols, int n_mol, int64_t packed,
                                 const unsigned long long* __restrict__ Vhat,
                                 const unsigned long long* __restrict__ Ehat, double* __restrict__ V,
                                 double* __restrict__ E) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < packed; e += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = n_mol - 1;  // the molecule whose block holds e (blocks in pk_off order)
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (mols[mid].pk_off <= e)
        lo = mid;
      else
        hi = mid - 1;
    }
    const int64_t off = mols[lo].pk_off, nf = mols[lo].nf;
    const int64_t r = (e - off) / nf, c = (e - off) - r * nf;
    V[e] = khat_value(Vhat + 2 * e) + khat_value(Vhat + 2 * (off + c * nf + r));
  }
  if (blockIdx.x == 0)
    for (int m = threadIdx.x; m < n_mol; m += blockDim.x) E[m] = khat_value(Ehat + 2 * m);
}

}  // namespace

cudaError_t launch_xc_colloc(cudaStream_t st, const BatchDesc* dbatch, int nbatch, int max_ldq, int max_nBshell,
                             const int* bshell, const int* bshell_col, const double* xyz, DeviceBasis basis,
                             double* ws) {
  if (nbatch == 0 || max_ldq == 0 || max_nBshell == 0) return cudaSuccess;
  dim3 grid((max_ldq + XC_THREADS - 1) / XC_THREADS, (max_nBshell + XC_SHELLS - 1) / XC_SHELLS, nbatch);
  xc_colloc_kernel<<<grid, XC_THREADS, 0, st>>>(dbatch, bshell, bshell_col, xyz, basis, ws);
  return cudaGetLastError();
}

cudaError_t launch_xc_point(cudaStream_t st, const BatchDesc* dbatch, int nbatch, int max_ldq, const double* w,
                            int functional, double* ws, unsigned long long* Ehat, int* err) {
  if (nbatch == 0 || max_ldq == 0) return cudaSuccess;
  dim3 grid((max_ldq + XC_THREADS - 1) / XC_THREADS, nbatch);
  xc_point_kernel<<<grid, XC_THREADS, 0, st>>>(dbatch, w, functional, ws, Ehat, err);
  return cudaGetLastError();
}

cudaError_t launch_xc_finish(cudaStream_t st, const MolDesc* mols, int n_mol, int64_t packed,
                             const unsigned long long* Vhat, const unsigned long long* Ehat, double* V, double* E) {
  if (n_mol == 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>(std::max<int64_t>((packed + 255) / 256, 1), 4096);
  xc_finish_kernel<<<blocks, 256, 0, st>>>(mols, n_mol, packed, Vhat, Ehat, V, E);
  return cudaGetLastError();
}

}  // namespace snk
