// Device arithmetic of the track model (arXiv:1811.11481 Sec. 2-4).
//
// Everything here is __host__ __device__ and single precision except the
// float64 conversion of absolute drift times (Sec. 4). The track-model
// functions take an arithmetic policy:
//   Exact - the formulas as written, one IEEE rounding per operation
//           (division and square root correctly rounded); translation units
//           that use it are compiled with -fmad=false, so that an
//           implementation of the same formulas elsewhere (the merge and the
//           compression format are defined by them) gets the same bits;
//   Fast  - fused multiply-adds and approximate reciprocal and reciprocal
//           square root (the tracklet constructor, whose discrete decisions
//           are checked against the float64 method up to near-ties).
// Both are explicit in the source, so a launch shape or register cap cannot
// change the rounding.
#pragma once

#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "tpc.h"

#define TPC_HD __host__ __device__ __forceinline__

namespace tpc {

constexpr int kNS = TPC_N_SECTORS;
constexpr int kMaxRows = TPC_MAX_ROWS;
constexpr int kSpl = TPC_SPLINE_N;

// Detector geometry as the kernels see it. The row positions are read
// through a pointer to memory of the executing side (device memory for the
// kernels): an array held in the kernel parameters would be read with one
// serialised constant-cache access per distinct row in a warp.
struct Geo {
  const float* rx;  // [n_rows] pad-row plane positions (cm)
  int32_t n_rows;
  float tan_half;
  float L;
  float bz;
  float kB;  // curvature per unit q/pT: 2.99792458e-3 * bz, rounded to float
  const float* pw;  // [n_rows] pad pitch (cm), or null
  const float* pc;  // [n_rows] pad position of y = 0, or null
  int32_t field_on;  // the final fit uses the full field below
  float field[30];   // (Bx, By, Bz) quadratic polynomials in (X, Y, Z) / 100 cm
};

// ------------------------------------------------------ arithmetic policies
struct Exact {
  static TPC_HD float fma(float a, float b, float c) { return a * b + c; }
  static TPC_HD float div(float a, float b) { return a / b; }
  static TPC_HD float rcp(float a) { return 1.0f / a; }
  static TPC_HD float sqrt(float a) { return sqrtf(a); }
  static TPC_HD float rsqrt(float a) { return 1.0f / sqrtf(a); }
};
struct Fast {
#ifdef __CUDA_ARCH__
  static __device__ __forceinline__ float fma(float a, float b, float c) {
    return __fmaf_rn(a, b, c);
  }
  static __device__ __forceinline__ float rcp(float a) { return __fdividef(1.0f, a); }
  static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
  // a > 0 wherever it is used (1 - sin^2 with |sin| < s_max, 1 + T^2, a
  // squared chord)
  static __device__ __forceinline__ float rsqrt(float a) { return rsqrtf(a); }
  static __device__ __forceinline__ float sqrt(float a) { return a * rsqrtf(a); }
#else
  static float fma(float a, float b, float c) { return std::fma(a, b, c); }
  static float rcp(float a) { return 1.0f / a; }
  static float div(float a, float b) { return a / b; }
  static float rsqrt(float a) { return 1.0f / std::sqrt(a); }
  static float sqrt(float a) { return std::sqrt(a); }
#endif
};

struct Cal {
  double vdrift, t0, tf_start;
  const float* spline;    // device [36][2][8][8][8]
  const float* spl_bound; // device [3]: max|dy coef|, max|dz coef|, active flag
  float spl_x0, spl_dx;
};

// Packed symmetric 5x5: index of (i, j), i >= j.
TPC_HD int sidx(int i, int j) { return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i; }

// --------------------------------------------------------------- arc length
// A(h) = asin(h)/h from the Maclaurin series after half-angle reductions
// asin(h) = 2 asin(h / sqrt(2 (1 + sqrt(1 - h^2)))), and B(h) = A'(h).
template <class O = Exact> TPC_HD float series_asin_over_x(float h2) {
  float p = 35.0f / 1152.0f;
  p = O::fma(h2, p, 5.0f / 112.0f);
  p = O::fma(h2, p, 3.0f / 40.0f);
  p = O::fma(h2, p, 1.0f / 6.0f);
  p = O::fma(h2, p, 1.0f);
  return p;
}
template <class O = Exact> TPC_HD float arc_factor(float h) {
  if (fabsf(h) < 0.125f) return series_asin_over_x<O>(h * h);
  if (!(fabsf(h) <= 1.0f)) return (h - h) / (h - h);  // NaN
  float hh = h, m = 1.0f;
  while (fabsf(hh) >= 0.125f) {
    float c = O::sqrt(1.0f - hh * hh);
    hh = O::div(hh, O::sqrt(2.0f * (1.0f + c)));
    m = m * 2.0f;
  }
  return O::div((m * hh) * series_asin_over_x<O>(hh * hh), h);
}
template <class O = Exact> TPC_HD float arc_factor_deriv(float h) {
  if (fabsf(h) < 0.125f) {
    float h2 = h * h;
    float c = 315.0f / 1408.0f;
    c = O::fma(h2, c, 35.0f / 144.0f);
    c = O::fma(h2, c, 15.0f / 56.0f);
    c = O::fma(h2, c, 3.0f / 10.0f);
    c = O::fma(h2, c, 1.0f / 3.0f);
    return h * c;
  }
  float e = O::rsqrt(1.0f - h * h);
  return O::div(e - arc_factor<O>(h), h);
}

// ----------------------------------------------------------- time to z
// Seeding coordinate (Sec. 4): time scaled linearly to z, reference = tf_start.
TPC_HD float seed_z(const Geo& g, const Cal& c, int mode, float z, double t, int sector) {
  if (mode == 0) return z;
  double zeta = c.vdrift * ((t - c.t0) - c.tf_start);
  // the side's sign after the rounding to float: rounding to nearest is
  // symmetric, so the bits equal those of (float)(sign * (L - zeta))
  float a = (float)((double)g.L - zeta);
  return sector < 18 ? a : -a;
}
// Absolute z once the collision time 'that' is known (Sec. 4).
TPC_HD float abs_z(const Geo& g, const Cal& c, int mode, float z, double t, int sector,
                   double that) {
  if (mode == 0) return z;
  double zeta = c.vdrift * ((t - c.t0) - that);
  float a = (float)((double)g.L - zeta);  // sign after rounding, as in seed_z
  return sector < 18 ? a : -a;
}

// -------------------------------------------------------- distortion spline
TPC_HD float clamp01(float v) { return v < 0.0f ? 0.0f : (v > 1.0f ? 1.0f : v); }
TPC_HD void spline_split(float u, int& i, float& f) {
  float t = u * (float)(kSpl - 3);
  int k = (int)t;
  if (k > kSpl - 4) k = kSpl - 4;
  if (k < 0) k = 0;
  i = k;
  f = t - (float)k;
}
TPC_HD void spline_basis(float f, float b[4]) {
  float g = 1.0f - f;
  float f2 = f * f;
  float f3 = f2 * f;
  b[0] = ((g * g) * g) / 6.0f;
  b[1] = ((3.0f * f3 - 6.0f * f2) + 4.0f) / 6.0f;
  b[2] = (((-3.0f * f3 + 3.0f * f2) + 3.0f * f) + 1.0f) / 6.0f;
  b[3] = f3 / 6.0f;
}
// (dy, dz) of sector 'sector' at (x, y, |z| = az).
TPC_HD void spline_eval(const Geo& g, const Cal& c, int sector, float x, float y, float az,
                        float out[2]) {
  float u = clamp01((x - c.spl_x0) / c.spl_dx);
  float v = clamp01((y / x + g.tan_half) / (2.0f * g.tan_half));
  float w = clamp01(az / g.L);
  int iu, iv, iw;
  float fu, fv, fw;
  spline_split(u, iu, fu);
  spline_split(v, iv, fv);
  spline_split(w, iw, fw);
  float bu[4], bv[4], bw[4];
  spline_basis(fu, bu);
  spline_basis(fv, bv);
  spline_basis(fw, bw);
#pragma unroll
  for (int comp = 0; comp < 2; ++comp) {
    const float* cf = c.spline + ((sector * 2 + comp) * kSpl) * kSpl * kSpl;
    float acc = 0.0f;
#pragma unroll
    for (int cc = 0; cc < 4; ++cc)
#pragma unroll
      for (int bb = 0; bb < 4; ++bb) {
        float wb = bw[cc] * bv[bb];
        const float* row = cf + ((iw + cc) * kSpl + (iv + bb)) * kSpl + iu;
#pragma unroll
        for (int aa = 0; aa < 4; ++aa) acc = acc + (wb * bu[aa]) * row[aa];
      }
    out[comp] = acc;
  }
}

// Calibrated position of a cluster for collision time 'that'.
TPC_HD void calibrate(const Geo& g, const Cal& c, bool spline_on, int mode, int sector, int row,
                      float y, float z, double t, double that, float& yc, float& zc) {
  float za = abs_z(g, c, mode, z, t, sector, that);
  if (spline_on) {
    float d[2];
    spline_eval(g, c, sector, g.rx[row], y, fabsf(za), d);
    yc = y + d[0];
    zc = za + d[1];
  } else {
    yc = y;
    zc = za;
  }
}

// --------------------------------------------------------- track model
// State p = (y, z, s, t, q) at local x, covariance packed (15).
struct Jac {
  float ys, yq, zs, zt, zq, sq;  // non-identity entries
};

// Exact helix transport to x2 in a uniform field with its analytic Jacobian.
// Returns false when |sin(phi)| would reach s_max.
template <class O = Exact>
TPC_HD bool transport(float kB, float s_max, float p[5], float& x, float x2, Jac& J) {
  float dx = x2 - x;
  float y = p[0], z = p[1], s = p[2], t = p[3], q = p[4];
  float kap = kB * q;
  float s2 = O::fma(-kap, dx, s);
  if (!(fabsf(s2) < s_max)) return false;
  float c1 = O::sqrt(O::fma(-s, s, 1.0f));
  float c2 = O::sqrt(O::fma(-s2, s2, 1.0f));
  float N = s + s2;
  float D = c1 + c2;
  float T = O::div(N, D);
  float dy = dx * T;
  float opt = O::fma(T, T, 1.0f);
  float d = dx * O::sqrt(opt);
  float h = (kap * d) * 0.5f;
  float A = arc_factor<O>(h);
  float l = d * A;
  float sc1 = O::div(s, c1), sc2 = O::div(s2, c2);
  float dDds = -sc1 - sc2;
  float kdx = kB * dx;
  float dDdq = kdx * sc2;
  float dTds = O::div(O::fma(-T, dDds, 2.0f), D);
  float dTdq = O::div(O::fma(-T, dDdq, -kdx), D);
  J.ys = dx * dTds;
  J.yq = dx * dTdq;
  float gg = O::div(d * T, opt);
  float dds = gg * dTds;
  float ddq = gg * dTdq;
  float E = O::rsqrt(O::fma(-h, h, 1.0f));
  float Bh = arc_factor_deriv<O>(h);
  J.zs = t * (E * dds);
  J.zq = t * O::fma(E, ddq, (kB * ((d * d) * Bh)) * 0.5f);
  J.zt = l;
  J.sq = -kdx;
  p[0] = y + dy;
  p[1] = O::fma(t, l, z);
  p[2] = s2;
  x = x2;
  return true;
}

// C' = J C J^T with index-ascending sums over the non-zero entries of J.
template <class O = Exact> TPC_HD void transport_cov(const Jac& J, float C[15]) {
  float Cf[5][5];
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j < 5; ++j) Cf[i][j] = C[sidx(i, j)];
  float T[5][5];
#pragma unroll
  for (int l = 0; l < 5; ++l) {
    T[0][l] = O::fma(J.yq, Cf[4][l], O::fma(J.ys, Cf[2][l], Cf[0][l]));
    T[1][l] = O::fma(J.zq, Cf[4][l], O::fma(J.zt, Cf[3][l], O::fma(J.zs, Cf[2][l], Cf[1][l])));
    T[2][l] = O::fma(J.sq, Cf[4][l], Cf[2][l]);
    T[3][l] = Cf[3][l];
    T[4][l] = Cf[4][l];
  }
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    C[sidx(i, 0)] = O::fma(T[i][4], J.yq, O::fma(T[i][2], J.ys, T[i][0]));
    if (i >= 1)
      C[sidx(i, 1)] =
          O::fma(T[i][4], J.zq, O::fma(T[i][3], J.zt, O::fma(T[i][2], J.zs, T[i][1])));
    if (i >= 2) C[sidx(i, 2)] = O::fma(T[i][4], J.sq, T[i][2]);
    if (i >= 3) C[sidx(i, 3)] = T[i][3];
    if (i >= 4) C[sidx(i, 4)] = T[i][4];
  }
}

template <class O = Exact>
TPC_HD bool propagate(float kB, float s_max, float p[5], float C[15], float& x, float x2) {
  Jac J;
  if (!transport<O>(kB, s_max, p, x, x2, J)) return false;
  transport_cov<O>(J, C);
  return true;
}

struct Innov {
  float r0, r1, W00, W01, W11, chi2;
};
// Innovation r = m - H p, its covariance S = H C H^T + V and W = S^-1.
template <class O = Exact>
TPC_HD Innov innovation(const float p[5], const float C[15], float my, float mz, float vy,
                        float vz) {
  Innov in;
  in.r0 = my - p[0];
  in.r1 = mz - p[1];
  float S00 = C[0] + vy;
  float S01 = C[1];
  float S11 = C[2] + vz;
  float det = O::fma(S00, S11, -(S01 * S01));
  in.W00 = O::div(S11, det);
  in.W01 = -O::div(S01, det);
  in.W11 = O::div(S00, det);
  in.chi2 = O::fma(in.r1, O::fma(in.W11, in.r1, in.W01 * in.r0),
                   in.r0 * O::fma(in.W01, in.r1, in.W00 * in.r0));
  return in;
}
// Kalman gain K = C H^T S^-1; p += K r; C -= K H C (lower triangle).
template <class O = Exact> TPC_HD void apply_update(float p[5], float C[15], const Innov& in) {
  float C0[5], C1[5];
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    C0[j] = C[sidx(j, 0)];
    C1[j] = C[sidx(j, 1)];
  }
  float K0[5], K1[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    K0[i] = O::fma(C1[i], in.W01, C0[i] * in.W00);
    K1[i] = O::fma(C1[i], in.W11, C0[i] * in.W01);
  }
#pragma unroll
  for (int i = 0; i < 5; ++i) p[i] = p[i] + O::fma(K1[i], in.r1, K0[i] * in.r0);
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j)
      C[sidx(i, j)] = C[sidx(i, j)] - O::fma(K1[i], C1[j], K0[i] * C0[j]);
}

TPC_HD void set_diag(float C[15], const float d[5]) {
#pragma unroll
  for (int i = 0; i < 15; ++i) C[i] = 0.0f;
#pragma unroll
  for (int i = 0; i < 5; ++i) C[sidx(i, i)] = d[i];
}

// Straight-line seed through two points, q/pT = 0 (tracklet seed, Sec. 2).
TPC_HD void seed_two_points(float p[5], float C[15], float& x, const float c0[5], float x0,
                            float y0, float z0, float x1, float y1, float z1) {
  float dx = x1 - x0, dy = y1 - y0, dz = z1 - z0;
  float dl = sqrtf(dx * dx + dy * dy);
  p[0] = y0;
  p[1] = z0;
  p[2] = dy / dl;
  p[3] = dz / dl;
  p[4] = 0.0f;
  x = x0;
  set_diag(C, c0);
}

// z of the closest approach of the helix to the beam line (Sec. 4).
TPC_HD float dca_z(float kB, const float p[5], float x) {
  float y = p[0], z = p[1], s = p[2], t = p[3], q = p[4];
  float kap = kB * q;
  float cs = sqrtf(1.0f - s * s);
  if (fabsf(kap) * (fabsf(x) + fabsf(y)) < 1e-4f) {
    float a = x * cs + y * s;
    return z - t * a;
  }
  float cx = x + s / kap;
  float cy = y - cs / kap;
  float rc = sqrtf(cx * cx + cy * cy);
  float rad = 1.0f / fabsf(kap);
  float f = 1.0f - rad / rc;
  float px = cx * f, py = cy * f;
  float ex = x - px, ey = y - py;
  float ch = sqrtf(ex * ex + ey * ey);
  float h = (ch * fabsf(kap)) * 0.5f;
  if (h > 1.0f) h = 1.0f;
  return z - t * (ch * arc_factor(h));
}

}  // namespace tpc
