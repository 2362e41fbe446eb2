// Generated by gen_os.py -- do not edit.
// Straight-line Obara-Saika VRR (App. A, Eq. vrr) and HRR (Eq. hrr) for the
// 3c-CP integrals of one shell-pair class, with the FP64 operation counts.
#pragma once

namespace snk {

template <int LA, int LB> struct OsClass;

// class (0,0): 2 VRR statements, VRR 1 flops per primitive pair,
// HRR 0 flops per contracted pair
template <> struct OsClass<0, 0> {
  static constexpr int L = 0;
  static constexpr int NACC = 1;
  static constexpr int NA = 1;
  static constexpr int NB = 1;
  static constexpr int KMAX = 0;
  static constexpr int VRR_FLOPS = 1;
  static constexpr int VRR_OPS = 1;
  static constexpr int HRR_FLOPS = 0;
  static constexpr int HRR_OPS = 0;
  template <typename R>
  __device__ static __forceinline__ void vrr(const R* S, R PAx, R PAy, R PAz, R PCx, R PCy, R PCz,
                                             R k1, R k2, R k3, R* acc) {
    (void)PAx; (void)PAy; (void)PAz; (void)PCx; (void)PCy; (void)PCz; (void)k1; (void)k2; (void)k3;
    const R t000_0 = S[0];
    acc[0] += t000_0;
  }
  template <typename R>
  __device__ static __forceinline__ void hrr(const R* acc, R ABx, R ABy, R ABz, R* xi) {
    (void)ABx; (void)ABy; (void)ABz;
    const R x000_000 = acc[0];
    xi[0] = x000_000;
  }
};

// class (1,0): 8 VRR statements, VRR 12 flops per primitive pair,
// HRR 0 flops per contracted pair
template <> struct OsClass<1, 0> {
  static constexpr int L = 1;
  static constexpr int NACC = 3;
  static constexpr int NA = 3;
  static constexpr int NB = 1;
  static constexpr int KMAX = 0;
  static constexpr int VRR_FLOPS = 12;
  static constexpr int VRR_OPS = 9;
  static constexpr int HRR_FLOPS = 0;
  static constexpr int HRR_OPS = 0;
  template <typename R>
  __device__ static __forceinline__ void vrr(const R* S, R PAx, R PAy, R PAz, R PCx, R PCy, R PCz,
                                             R k1, R k2, R k3, R* acc) {
    (void)PAx; (void)PAy; (void)PAz; (void)PCx; (void)PCy; (void)PCz; (void)k1; (void)k2; (void)k3;
    const R t000_0 = S[0];
    const R t000_1 = S[1];
    const R t100_0 = fma(PAx, t000_0, -PCx * t000_1);
    const R t010_0 = fma(PAy, t000_0, -PCy * t000_1);
    const R t001_0 = fma(PAz, t000_0, -PCz * t000_1);
    acc[0] += t100_0;
    acc[1] += t010_0;
    acc[2] += t001_0;
  }
  template <typename R>
  __device__ static __forceinline__ void hrr(const R* acc, R ABx, R ABy, R ABz, R* xi) {
    (void)ABx; (void)ABy; (void)ABz;
    const R x001_000 = acc[2];
    const R x010_000 = acc[1];
    const R x100_000 = acc[0];
    xi[0] = x100_000;
    xi[1] = x010_000;
    xi[2] = x001_000;
  }
};

// class (1,1): 25 VRR statements, VRR 52 flops per primitive pair,
// HRR 18 flops per contracted pair
template <> struct OsClass<1, 1> {
  static constexpr int L = 2;
  static constexpr int NACC = 9;
  static constexpr int NA = 3;
  static constexpr int NB = 3;
  static constexpr int KMAX = 1;
  static constexpr int VRR_FLOPS = 52;
  static constexpr int VRR_OPS = 37;
  static constexpr int HRR_FLOPS = 18;
  static constexpr int HRR_OPS = 9;
  template <typename R>
  __device__ static __forceinline__ void vrr(const R* S, R PAx, R PAy, R PAz, R PCx, R PCy, R PCz,
                                             R k1, R k2, R k3, R* acc) {
    (void)PAx; (void)PAy; (void)PAz; (void)PCx; (void)PCy; (void)PCz; (void)k1; (void)k2; (void)k3;
    const R t000_0 = S[0];
    const R t000_1 = S[1];
    const R t000_2 = S[2];
    const R t100_0 = fma(PAx, t000_0, -PCx * t000_1);
    const R t100_1 = fma(PAx, t000_1, -PCx * t000_2);
    const R t010_0 = fma(PAy, t000_0, -PCy * t000_1);
    const R t010_1 = fma(PAy, t000_1, -PCy * t000_2);
    const R t001_0 = fma(PAz, t000_0, -PCz * t000_1);
    const R t001_1 = fma(PAz, t000_1, -PCz * t000_2);
    const R d000_0 = t000_0 - t000_1;
    const R t200_0 = fma(k1, d000_0, fma(PAx, t100_0, -PCx * t100_1));
    const R t110_0 = fma(PAx, t010_0, -PCx * t010_1);
    const R t101_0 = fma(PAx, t001_0, -PCx * t001_1);
    const R t020_0 = fma(k1, d000_0, fma(PAy, t010_0, -PCy * t010_1));
    const R t011_0 = fma(PAy, t001_0, -PCy * t001_1);
    const R t002_0 = fma(k1, d000_0, fma(PAz, t001_0, -PCz * t001_1));
    acc[0] += t100_0;
    acc[1] += t010_0;
    acc[2] += t001_0;
    acc[3] += t200_0;
    acc[4] += t110_0;
    acc[5] += t101_0;
    acc[6] += t020_0;
    acc[7] += t011_0;
    acc[8] += t002_0;
  }
  template <typename R>
  __device__ static __forceinline__ void hrr(const R* acc, R ABx, R ABy, R ABz, R* xi) {
    (void)ABx; (void)ABy; (void)ABz;
    const R x002_000 = acc[8];
    const R x011_000 = acc[7];
    const R x020_000 = acc[6];
    const R x101_000 = acc[5];
    const R x110_000 = acc[4];
    const R x200_000 = acc[3];
    const R x001_000 = acc[2];
    const R x010_000 = acc[1];
    const R x100_000 = acc[0];
    const R x001_001 = fma(ABz, x001_000, x002_000);
    const R x001_010 = fma(ABy, x001_000, x011_000);
    const R x001_100 = fma(ABx, x001_000, x101_000);
    const R x010_001 = fma(ABz, x010_000, x011_000);
    const R x010_010 = fma(ABy, x010_000, x020_000);
    const R x010_100 = fma(ABx, x010_000, x110_000);
    const R x100_001 = fma(ABz, x100_000, x101_000);
    const R x100_010 = fma(ABy, x100_000, x110_000);
    const R x100_100 = fma(ABx, x100_000, x200_000);
    xi[0] = x100_100;
    xi[1] = x100_010;
    xi[2] = x100_001;
    xi[3] = x010_100;
    xi[4] = x010_010;
    xi[5] = x010_001;
    xi[6] = x001_100;
    xi[7] = x001_010;
    xi[8] = x001_001;
  }
};

// class (2,0): 22 VRR statements, VRR 49 flops per primitive pair,
// HRR 0 flops per contracted pair
template <> struct OsClass<2, 0> {
  static constexpr int L = 2;
  static constexpr int NACC = 6;
  static constexpr int NA = 6;
  static constexpr int NB = 1;
  static constexpr int KMAX = 1;
  static constexpr int VRR_FLOPS = 49;
  static constexpr int VRR_OPS = 34;
  static constexpr int HRR_FLOPS = 0;
  static constexpr int HRR_OPS = 0;
  template <typename R>
  __device__ static __forceinline__ void vrr(const R* S, R PAx, R PAy, R PAz, R PCx, R PCy, R PCz,
                                             R k1, R k2, R k3, R* acc) {
    (void)PAx; (void)PAy; (void)PAz; (void)PCx; (void)PCy; (void)PCz; (void)k1; (void)k2; (void)k3;
    const R t000_0 = S[0];
    const R t000_1 = S[1];
    const R t000_2 = S[2];
    const R t100_0 = fma(PAx, t000_0, -PCx * t000_1);
    const R t100_1 = fma(PAx, t000_1, -PCx * t000_2);
    const R t010_0 = fma(PAy, t000_0, -PCy * t000_1);
    const R t010_1 = fma(PAy, t000_1, -PCy * t000_2);
    const R t001_0 = fma(PAz, t000_0, -PCz * t000_1);
    const R t001_1 = fma(PAz, t000_1, -PCz * t000_2);
    const R d000_0 = t000_0 - t000_1;
    const R t200_0 = fma(k1, d000_0, fma(PAx, t100_0, -PCx * t100_1));
    const R t110_0 = fma(PAx, t010_0, -PCx * t010_1);
    const R t101_0 = fma(PAx, t001_0, -PCx * t001_1);
    const R t020_0 = fma(k1, d000_0, fma(PAy, t010_0, -PCy * t010_1));
    const R t011_0 = fma(PAy, t001_0, -PCy * t001_1);
    const R t002_0 = fma(k1, d000_0, fma(PAz, t001_0, -PCz * t001_1));
    acc[0] += t200_0;
    acc[1] += t110_0;
    acc[2] += t101_0;
    acc[3] += t020_0;
    acc[4] += t011_0;
    acc[5] += t002_0;
  }
  template <typename R>
  __device__ static __forceinline__ void hrr(const R* acc, R ABx, R ABy, R ABz, R* xi) {
    (void)ABx; (void)ABy; (void)ABz;
    const R x002_000 = acc[5];
    const R x011_000 = acc[4];
    const R x020_000 = acc[3];
    const R x101_000 = acc[2];
    const R x110_000 = acc[1];
    const R x200_000 = acc[0];
    xi[0] = x200_000;
    xi[1] = x110_000;
    xi[2] = x101_000;
    xi[3] = x020_000;
    xi[4] = x011_000;
    xi[5] = x002_000;
  }
};

// class (2,1): 54 VRR statements, VRR 126 flops per primitive pair,
// HRR 36 flops per contracted pair
template <> struct OsClass<2, 1> {
  static constexpr int L = 3;
  static constexpr int NACC = 16;
  static constexpr int NA = 6;
  static constexpr int NB = 3;
  static constexpr int KMAX = 2;
  static constexpr int VRR_FLOPS = 126;
  static constexpr int VRR_OPS = 88;
  static constexpr int HRR_FLOPS = 36;
  static constexpr int HRR_OPS = 18;
  template <typename R>
  __device__ static __forceinline__ void vrr(const R* S, R PAx, R PAy, R PAz, R PCx, R PCy, R PCz,
                                             R k1, R k2, R k3, R* acc) {
    (void)PAx; (void)PAy; (void)PAz; (void)PCx; (void)PCy; (void)PCz; (void)k1; (void)k2; (void)k3;
    const R t000_0 = S[0];
    const R t000_1 = S[1];
    const R t000_2 = S[2];
    const R t000_3 = S[3];
    const R t100_0 = fma(PAx, t000_0, -PCx * t000_1);
    const R t100_1 = fma(PAx, t000_1, -PCx * t000_2);
    const R t100_2 = fma(PAx, t000_2, -PCx * t000_3);
    const R t010_0 = fma(PAy, t000_0, -PCy * t000_1);
    const R t010_1 = fma(PAy, t000_1, -PCy * t000_2);
    const R t010_2 = fma(PAy, t000_2, -PCy * t000_3);
    const R t001_0 = fma(PAz, t000_0, -PCz * t000_1);
    const R t001_1 = fma(PAz, t000_1, -PCz * t000_2);
    const R t001_2 = fma(PAz, t000_2, -PCz * t000_3);
    const R d000_0 = t000_0 - t000_1;
    const R t200_0 = fma(k1, d000_0, fma(PAx, t100_0, -PCx * t100_1));
    const R d000_1 = t000_1 - t000_2;
    const R t200_1 = fma(k1, d000_1, fma(PAx, t100_1, -PCx * t100_2));
    const R t110_0 = fma(PAx, t010_0, -PCx * t010_1);
    const R t101_0 = fma(PAx, t001_0, -PCx * t001_1);
    const R t020_0 = fma(k1, d000_0, fma(PAy, t010_0, -PCy * t010_1));
    const R t020_1 = fma(k1, d000_1, fma(PAy, t010_1, -PCy * t010_2));
    const R t011_0 = fma(PAy, t001_0, -PCy * t001_1);
    const R t011_1 = fma(PAy, t001_1, -PCy * t001_2);
    const R t002_0 = fma(k1, d000_0, fma(PAz, t001_0, -PCz * t001_1));
    const R t002_1 = fma(k1, d000_1, fma(PAz, t001_1, -PCz * t001_2));
    const R d100_0 = t100_0 - t100_1;
    const R t300_0 = fma(k2, d100_0, fma(PAx, t200_0, -PCx * t200_1));
    const R t210_0 = fma(PAy, t200_0, -PCy * t200_1);
    const R t201_0 = fma(PAz, t200_0, -PCz * t200_1);
    const R t120_0 = fma(PAx, t020_0, -PCx * t020_1);
    const R t111_0 = fma(PAx, t011_0, -PCx * t011_1);
    const R t102_0 = fma(PAx, t002_0, -PCx * t002_1);
    const R d010_0 = t010_0 - t010_1;
    const R t030_0 = fma(k2, d010_0, fma(PAy, t020_0, -PCy * t020_1));
    const R t021_0 = fma(PAz, t020_0, -PCz * t020_1);
    const R t012_0 = fma(PAy, t002_0, -PCy * t002_1);
    const R d001_0 = t001_0 - t001_1;
    const R t003_0 = fma(k2, d001_0, fma(PAz, t002_0, -PCz * t002_1));
    acc[0] += t200_0;
    acc[1] += t110_0;
    acc[2] += t101_0;
    acc[3] += t020_0;
    acc[4] += t011_0;
    acc[5] += t002_0;
    acc[6] += t300_0;
    acc[7] += t210_0;
    acc[8] += t201_0;
    acc[9] += t120_0;
    acc[10] += t111_0;
    acc[11] += t102_0;
    acc[12] += t030_0;
    acc[13] += t021_0;
    acc[14] += t012_0;
    acc[15] += t003_0;
  }
  template <typename R>
  __device__ static __forceinline__ void hrr(const R* acc, R ABx, R ABy, R ABz, R* xi) {
    (void)ABx; (void)ABy; (void)ABz;
    const R x003_000 = acc[15];
    const R x012_000 = acc[14];
    const R x021_000 = acc[13];
    const R x030_000 = acc[12];
    const R x102_000 = acc[11];
    const R x111_000 = acc[10];
    const R x120_000 = acc[9];
    const R x201_000 = acc[8];
    const R x210_000 = acc[7];
    const R x300_000 = acc[6];
    const R x002_000 = acc[5];
    const R x011_000 = acc[4];
    const R x020_000 = acc[3];
    const R x101_000 = acc[2];
    const R x110_000 = acc[1];
    const R x200_000 = acc[0];
    const R x002_001 = fma(ABz, x002_000, x003_000);
    const R x002_010 = fma(ABy, x002_000, x012_000);
    const R x002_100 = fma(ABx, x002_000, x102_000);
    const R x011_001 = fma(ABz, x011_000, x012_000);
    const R x011_010 = fma(ABy, x011_000, x021_000);
    const R x011_100 = fma(ABx, x011_000, x111_000);
    const R x020_001 = fma(ABz, x020_000, x021_000);
    const R x020_010 = fma(ABy, x020_000, x030_000);
    const R x020_100 = fma(ABx, x020_000, x120_000);
    const R x101_001 = fma(ABz, x101_000, x102_000);
    const R x101_010 = fma(ABy, x101_000, x111_000);
    const R x101_100 = fma(ABx, x101_000, x201_000);
    const R x110_001 = fma(ABz, x110_000, x111_000);
    const R x110_010 = fma(ABy, x110_000, x120_000);
    const R x110_100 = fma(ABx, x110_000, x210_000);
    const R x200_001 = fma(ABz, x200_000, x201_000);
    const R x200_010 = fma(ABy, x200_000, x210_000);
    const R x200_100 = fma(ABx, x200_000, x300_000);
    xi[0] = x200_100;
    xi[1] = x200_010;
    xi[2] = x200_001;
    xi[3] = x110_100;
    xi[4] = x110_010;
    xi[5] = x110_001;
    xi[6] = x101_100;
    xi[7] = x101_010;
    xi[8] = x101_001;
    xi[9] = x020_100;
    xi[10] = x020_010;
    xi[11] = x020_001;
    xi[12] = x011_100;
    xi[13] = x011_010;
    xi[14] = x011_001;
    xi[15] = x002_100;
    xi[16] = x002_010;
    xi[17] = x002_001;
  }
};

// class (2,2): 106 VRR statements, VRR 259 flops per primitive pair,
// HRR 158 flops per contracted pair
template <> struct OsClass<2, 2> {
  static constexpr int L = 4;
  static constexpr int NACC = 31;
  static constexpr int NA = 6;
  static constexpr int NB = 6;
  static constexpr int KMAX = 3;
  static constexpr int VRR_FLOPS = 259;
  static constexpr int VRR_OPS = 180;
  static constexpr int HRR_FLOPS = 158;
  static constexpr int HRR_OPS = 79;
  template <typename R>
  __device__ static __forceinline__ void vrr(const R* S, R PAx, R PAy, R PAz, R PCx, R PCy, R PCz,
                                             R k1, R k2, R k3, R* acc) {
    (void)PAx; (void)PAy; (void)PAz; (void)PCx; (void)PCy; (void)PCz; (void)k1; (void)k2; (void)k3;
    const R t000_0 = S[0];
    const R t000_1 = S[1];
    const R t000_2 = S[2];
    const R t000_3 = S[3];
    const R t000_4 = S[4];
    const R t100_0 = fma(PAx, t000_0, -PCx * t000_1);
    const R t100_1 = fma(PAx, t000_1, -PCx * t000_2);
    const R t100_2 = fma(PAx, t000_2, -PCx * t000_3);
    const R t100_3 = fma(PAx, t000_3, -PCx * t000_4);
    const R t010_0 = fma(PAy, t000_0, -PCy * t000_1);
    const R t010_1 = fma(PAy, t000_1, -PCy * t000_2);
    const R t010_2 = fma(PAy, t000_2, -PCy * t000_3);
    const R t010_3 = fma(PAy, t000_3, -PCy * t000_4);
    const R t001_0 = fma(PAz, t000_0, -PCz * t000_1);
    const R t001_1 = fma(PAz, t000_1, -PCz * t000_2);
    const R t001_2 = fma(PAz, t000_2, -PCz * t000_3);
    const R t001_3 = fma(PAz, t000_3, -PCz * t000_4);
    const R d000_0 = t000_0 - t000_1;
    const R t200_0 = fma(k1, d000_0, fma(PAx, t100_0, -PCx * t100_1));
    const R d000_1 = t000_1 - t000_2;
    const R t200_1 = fma(k1, d000_1, fma(PAx, t100_1, -PCx * t100_2));
    const R d000_2 = t000_2 - t000_3;
    const R t200_2 = fma(k1, d000_2, fma(PAx, t100_2, -PCx * t100_3));
    const R t110_0 = fma(PAx, t010_0, -PCx * t010_1);
    const R t101_0 = fma(PAx, t001_0, -PCx * t001_1);
    const R t020_0 = fma(k1, d000_0, fma(PAy, t010_0, -PCy * t010_1));
    const R t020_1 = fma(k1, d000_1, fma(PAy, t010_1, -PCy * t010_2));
    const R t020_2 = fma(k1, d000_2, fma(PAy, t010_2, -PCy * t010_3));
    const R t011_0 = fma(PAy, t001_0, -PCy * t001_1);
    const R t011_1 = fma(PAy, t001_1, -PCy * t001_2);
    const R t002_0 = fma(k1, d000_0, fma(PAz, t001_0, -PCz * t001_1));
    const R t002_1 = fma(k1, d000_1, fma(PAz, t001_1, -PCz * t001_2));
    const R t002_2 = fma(k1, d000_2, fma(PAz, t001_2, -PCz * t001_3));
    const R d100_0 = t100_0 - t100_1;
    const R t300_0 = fma(k2, d100_0, fma(PAx, t200_0, -PCx * t200_1));
    const R d100_1 = t100_1 - t100_2;
    const R t300_1 = fma(k2, d100_1, fma(PAx, t200_1, -PCx * t200_2));
    const R t210_0 = fma(PAy, t200_0, -PCy * t200_1);
    const R t201_0 = fma(PAz, t200_0, -PCz * t200_1);
    const R t201_1 = fma(PAz, t200_1, -PCz * t200_2);
    const R t120_0 = fma(PAx, t020_0, -PCx * t020_1);
    const R t120_1 = fma(PAx, t020_1, -PCx * t020_2);
    const R t111_0 = fma(PAx, t011_0, -PCx * t011_1);
    const R t102_0 = fma(PAx, t002_0, -PCx * t002_1);
    const R t102_1 = fma(PAx, t002_1, -PCx * t002_2);
    const R d010_0 = t010_0 - t010_1;
    const R t030_0 = fma(k2, d010_0, fma(PAy, t020_0, -PCy * t020_1));
    const R d010_1 = t010_1 - t010_2;
    const R t030_1 = fma(k2, d010_1, fma(PAy, t020_1, -PCy * t020_2));
    const R t021_0 = fma(PAz, t020_0, -PCz * t020_1);
    const R t021_1 = fma(PAz, t020_1, -PCz * t020_2);
    const R t012_0 = fma(PAy, t002_0, -PCy * t002_1);
    const R t012_1 = fma(PAy, t002_1, -PCy * t002_2);
    const R d001_0 = t001_0 - t001_1;
    const R t003_0 = fma(k2, d001_0, fma(PAz, t002_0, -PCz * t002_1));
    const R d001_1 = t001_1 - t001_2;
    const R t003_1 = fma(k2, d001_1, fma(PAz, t002_1, -PCz * t002_2));
    const R d200_0 = t200_0 - t200_1;
    const R t400_0 = fma(k3, d200_0, fma(PAx, t300_0, -PCx * t300_1));
    const R t310_0 = fma(PAy, t300_0, -PCy * t300_1);
    const R t301_0 = fma(PAz, t300_0, -PCz * t300_1);
    const R d020_0 = t020_0 - t020_1;
    const R t220_0 = fma(k1, d020_0, fma(PAx, t120_0, -PCx * t120_1));
    const R t211_0 = fma(PAy, t201_0, -PCy * t201_1);
    const R d002_0 = t002_0 - t002_1;
    const R t202_0 = fma(k1, d002_0, fma(PAx, t102_0, -PCx * t102_1));
    const R t130_0 = fma(PAx, t030_0, -PCx * t030_1);
    const R t121_0 = fma(PAx, t021_0, -PCx * t021_1);
    const R t112_0 = fma(PAx, t012_0, -PCx * t012_1);
    const R t103_0 = fma(PAx, t003_0, -PCx * t003_1);
    const R t040_0 = fma(k3, d020_0, fma(PAy, t030_0, -PCy * t030_1));
    const R t031_0 = fma(PAz, t030_0, -PCz * t030_1);
    const R t022_0 = fma(k1, d002_0, fma(PAy, t012_0, -PCy * t012_1));
    const R t013_0 = fma(PAy, t003_0, -PCy * t003_1);
    const R t004_0 = fma(k3, d002_0, fma(PAz, t003_0, -PCz * t003_1));
    acc[0] += t200_0;
    acc[1] += t110_0;
    acc[2] += t101_0;
    acc[3] += t020_0;
    acc[4] += t011_0;
    acc[5] += t002_0;
    acc[6] += t300_0;
    acc[7] += t210_0;
    acc[8] += t201_0;
    acc[9] += t120_0;
    acc[10] += t111_0;
    acc[11] += t102_0;
    acc[12] += t030_0;
    acc[13] += t021_0;
    acc[14] += t012_0;
    acc[15] += t003_0;
    acc[16] += t400_0;
    acc[17] += t310_0;
    acc[18] += t301_0;
    acc[19] += t220_0;
    acc[20] += t211_0;
    acc[21] += t202_0;
    acc[22] += t130_0;
    acc[23] += t121_0;
    acc[24] += t112_0;
    acc[25] += t103_0;
    acc[26] += t040_0;
    acc[27] += t031_0;
    acc[28] += t022_0;
    acc[29] += t013_0;
    acc[30] += t004_0;
  }
  template <typename R>
  __device__ static __forceinline__ void hrr(const R* acc, R ABx, R ABy, R ABz, R* xi) {
    (void)ABx; (void)ABy; (void)ABz;
    const R x004_000 = acc[30];
    const R x013_000 = acc[29];
    const R x022_000 = acc[28];
    const R x031_000 = acc[27];
    const R x040_000 = acc[26];
    const R x103_000 = acc[25];
    const R x112_000 = acc[24];
    const R x121_000 = acc[23];
    const R x130_000 = acc[22];
    const R x202_000 = acc[21];
    const R x211_000 = acc[20];
    const R x220_000 = acc[19];
    const R x301_000 = acc[18];
    const R x310_000 = acc[17];
    const R x400_000 = acc[16];
    const R x003_000 = acc[15];
    const R x012_000 = acc[14];
    const R x021_000 = acc[13];
    const R x030_000 = acc[12];
    const R x102_000 = acc[11];
    const R x111_000 = acc[10];
    const R x120_000 = acc[9];
    const R x201_000 = acc[8];
    const R x210_000 = acc[7];
    const R x300_000 = acc[6];
    const R x002_000 = acc[5];
    const R x011_000 = acc[4];
    const R x020_000 = acc[3];
    const R x101_000 = acc[2];
    const R x110_000 = acc[1];
    const R x200_000 = acc[0];
    const R x003_001 = fma(ABz, x003_000, x004_000);
    const R x012_001 = fma(ABz, x012_000, x013_000);
    const R x012_010 = fma(ABy, x012_000, x022_000);
    const R x021_001 = fma(ABz, x021_000, x022_000);
    const R x021_010 = fma(ABy, x021_000, x031_000);
    const R x030_001 = fma(ABz, x030_000, x031_000);
    const R x030_010 = fma(ABy, x030_000, x040_000);
    const R x102_001 = fma(ABz, x102_000, x103_000);
    const R x102_010 = fma(ABy, x102_000, x112_000);
    const R x102_100 = fma(ABx, x102_000, x202_000);
    const R x111_001 = fma(ABz, x111_000, x112_000);
    const R x111_010 = fma(ABy, x111_000, x121_000);
    const R x111_100 = fma(ABx, x111_000, x211_000);
    const R x120_001 = fma(ABz, x120_000, x121_000);
    const R x120_010 = fma(ABy, x120_000, x130_000);
    const R x120_100 = fma(ABx, x120_000, x220_000);
    const R x201_001 = fma(ABz, x201_000, x202_000);
    const R x201_010 = fma(ABy, x201_000, x211_000);
    const R x201_100 = fma(ABx, x201_000, x301_000);
    const R x210_001 = fma(ABz, x210_000, x211_000);
    const R x210_010 = fma(ABy, x210_000, x220_000);
    const R x210_100 = fma(ABx, x210_000, x310_000);
    const R x300_001 = fma(ABz, x300_000, x301_000);
    const R x300_010 = fma(ABy, x300_000, x310_000);
    const R x300_100 = fma(ABx, x300_000, x400_000);
    const R x002_001 = fma(ABz, x002_000, x003_000);
    const R x002_010 = fma(ABy, x002_000, x012_000);
    const R x002_100 = fma(ABx, x002_000, x102_000);
    const R x011_001 = fma(ABz, x011_000, x012_000);
    const R x011_010 = fma(ABy, x011_000, x021_000);
    const R x011_100 = fma(ABx, x011_000, x111_000);
    const R x020_001 = fma(ABz, x020_000, x021_000);
    const R x020_010 = fma(ABy, x020_000, x030_000);
    const R x020_100 = fma(ABx, x020_000, x120_000);
    const R x101_001 = fma(ABz, x101_000, x102_000);
    const R x101_010 = fma(ABy, x101_000, x111_000);
    const R x101_100 = fma(ABx, x101_000, x201_000);
    const R x110_001 = fma(ABz, x110_000, x111_000);
    const R x110_010 = fma(ABy, x110_000, x120_000);
    const R x110_100 = fma(ABx, x110_000, x210_000);
    const R x200_001 = fma(ABz, x200_000, x201_000);
    const R x200_010 = fma(ABy, x200_000, x210_000);
    const R x200_100 = fma(ABx, x200_000, x300_000);
    const R x002_002 = fma(ABz, x002_001, x003_001);
    const R x002_011 = fma(ABy, x002_001, x012_001);
    const R x002_020 = fma(ABy, x002_010, x012_010);
    const R x002_101 = fma(ABx, x002_001, x102_001);
    const R x002_110 = fma(ABx, x002_010, x102_010);
    const R x002_200 = fma(ABx, x002_100, x102_100);
    const R x011_002 = fma(ABz, x011_001, x012_001);
    const R x011_011 = fma(ABy, x011_001, x021_001);
    const R x011_020 = fma(ABy, x011_010, x021_010);
    const R x011_101 = fma(ABx, x011_001, x111_001);
    const R x011_110 = fma(ABx, x011_010, x111_010);
    const R x011_200 = fma(ABx, x011_100, x111_100);
    const R x020_002 = fma(ABz, x020_001, x021_001);
    const R x020_011 = fma(ABy, x020_001, x030_001);
    const R x020_020 = fma(ABy, x020_010, x030_010);
    const R x020_101 = fma(ABx, x020_001, x120_001);
    const R x020_110 = fma(ABx, x020_010, x120_010);
    const R x020_200 = fma(ABx, x020_100, x120_100);
    const R x101_002 = fma(ABz, x101_001, x102_001);
    const R x101_011 = fma(ABy, x101_001, x111_001);
    const R x101_020 = fma(ABy, x101_010, x111_010);
    const R x101_101 = fma(ABx, x101_001, x201_001);
    const R x101_110 = fma(ABx, x101_010, x201_010);
    const R x101_200 = fma(ABx, x101_100, x201_100);
    const R x110_002 = fma(ABz, x110_001, x111_001);
    const R x110_011 = fma(ABy, x110_001, x120_001);
    const R x110_020 = fma(ABy, x110_010, x120_010);
    const R x110_101 = fma(ABx, x110_001, x210_001);
    const R x110_110 = fma(ABx, x110_010, x210_010);
    const R x110_200 = fma(ABx, x110_100, x210_100);
    const R x200_002 = fma(ABz, x200_001, x201_001);
    const R x200_011 = fma(ABy, x200_001, x210_001);
    const R x200_020 = fma(ABy, x200_010, x210_010);
    const R x200_101 = fma(ABx, x200_001, x300_001);
    const R x200_110 = fma(ABx, x200_010, x300_010);
    const R x200_200 = fma(ABx, x200_100, x300_100);
    xi[0] = x200_200;
    xi[1] = x200_110;
    xi[2] = x200_101;
    xi[3] = x200_020;
    xi[4] = x200_011;
    xi[5] = x200_002;
    xi[6] = x110_200;
    xi[7] = x110_110;
    xi[8] = x110_101;
    xi[9] = x110_020;
    xi[10] = x110_011;
    xi[11] = x110_002;
    xi[12] = x101_200;
    xi[13] = x101_110;
    xi[14] = x101_101;
    xi[15] = x101_020;
    xi[16] = x101_011;
    xi[17] = x101_002;
    xi[18] = x020_200;
    xi[19] = x020_110;
    xi[20] = x020_101;
    xi[21] = x020_020;
    xi[22] = x020_011;
    xi[23] = x020_002;
    xi[24] = x011_200;
    xi[25] = x011_110;
    xi[26] = x011_101;
    xi[27] = x011_020;
    xi[28] = x011_011;
    xi[29] = x011_002;
    xi[30] = x002_200;
    xi[31] = x002_110;
    xi[32] = x002_101;
    xi[33] = x002_020;
    xi[34] = x002_011;
    xi[35] = x002_002;
  }
};

}  // namespace snk
