// Device arithmetic of the track model (arXiv:1811.11481 Sec. 2-4).
//
// Everything here is __host__ __device__ and single precision except the
// float64 conversion of absolute drift times (Sec. 4). Operations are written
// one rounding at a time in a fixed order; translation units that take
// discrete decisions with these functions are compiled with -fmad=false so no
// multiply-add is contracted behind the reader's back.
#pragma once

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
TPC_HD float series_asin_over_x(float h2) {
  float p = 35.0f / 1152.0f;
  p = 5.0f / 112.0f + h2 * p;
  p = 3.0f / 40.0f + h2 * p;
  p = 1.0f / 6.0f + h2 * p;
  p = 1.0f + h2 * p;
  return p;
}
TPC_HD float arc_factor(float h) {
  if (fabsf(h) < 0.125f) return series_asin_over_x(h * h);
  if (!(fabsf(h) <= 1.0f)) return (h - h) / (h - h);  // NaN
  float hh = h, m = 1.0f;
  while (fabsf(hh) >= 0.125f) {
    float c = sqrtf(1.0f - hh * hh);
    hh = hh / sqrtf(2.0f * (1.0f + c));
    m = m * 2.0f;
  }
  return ((m * hh) * series_asin_over_x(hh * hh)) / h;
}
TPC_HD float arc_factor_deriv(float h) {
  if (fabsf(h) < 0.125f) {
    float h2 = h * h;
    float c = 315.0f / 1408.0f;
    c = 35.0f / 144.0f + h2 * c;
    c = 15.0f / 56.0f + h2 * c;
    c = 3.0f / 10.0f + h2 * c;
    c = 1.0f / 3.0f + h2 * c;
    return h * c;
  }
  float e = 1.0f / sqrtf(1.0f - h * h);
  return (e - arc_factor(h)) / h;
}

// ----------------------------------------------------------- time to z
// Seeding coordinate (Sec. 4): time scaled linearly to z, reference = tf_start.
TPC_HD float seed_z(const Geo& g, const Cal& c, int mode, float z, double t, int sector) {
  if (mode == 0) return z;
  double sg = sector < 18 ? 1.0 : -1.0;
  double zeta = c.vdrift * ((t - c.t0) - c.tf_start);
  return (float)(sg * ((double)g.L - zeta));
}
// Absolute z once the collision time 'that' is known (Sec. 4).
TPC_HD float abs_z(const Geo& g, const Cal& c, int mode, float z, double t, int sector,
                   double that) {
  if (mode == 0) return z;
  double sg = sector < 18 ? 1.0 : -1.0;
  double zeta = c.vdrift * ((t - c.t0) - that);
  return (float)(sg * ((double)g.L - zeta));
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

// 1/sqrt(1 - h^2): Maclaurin series for |h| < 1/8, else direct.
TPC_HD float inv_cos_half(float h) {
  if (fabsf(h) < 0.125f) {
    float h2 = h * h;
    float p = 35.0f / 128.0f;
    p = 5.0f / 16.0f + h2 * p;
    p = 3.0f / 8.0f + h2 * p;
    p = 0.5f + h2 * p;
    return 1.0f + h2 * p;
  }
  return 1.0f / sqrtf(1.0f - h * h);
}

// Exact helix transport to x2 in a uniform field with its analytic Jacobian.
// Returns false when |sin(phi)| would reach s_max.
TPC_HD bool transport(float kB, float s_max, float p[5], float& x, float x2, Jac& J) {
  float dx = x2 - x;
  float y = p[0], z = p[1], s = p[2], t = p[3], q = p[4];
  float kap = kB * q;
  float s2 = s - kap * dx;
  if (!(fabsf(s2) < s_max)) return false;
  float c1 = sqrtf(1.0f - s * s);
  float c2 = sqrtf(1.0f - s2 * s2);
  float ic1 = 1.0f / c1;
  float ic2 = 1.0f / c2;
  float N = s + s2;
  float D = c1 + c2;
  float iD = 1.0f / D;
  float T = N * iD;
  float dy = dx * T;
  float opt = 1.0f + T * T;
  float d = dx * sqrtf(opt);
  float h = (kap * d) * 0.5f;
  float A = arc_factor(h);
  float l = d * A;
  float dDds = -(s * ic1) - (s2 * ic2);
  float kdx = kB * dx;
  float dDdq = kdx * (s2 * ic2);
  float dTds = (2.0f - T * dDds) * iD;
  float dTdq = (-kdx - T * dDdq) * iD;
  J.ys = dx * dTds;
  J.yq = dx * dTdq;
  float gg = (d * T) / opt;
  float dds = gg * dTds;
  float ddq = gg * dTdq;
  float E = inv_cos_half(h);
  float Bh = arc_factor_deriv(h);
  J.zs = t * (E * dds);
  J.zq = t * (E * ddq + (kB * ((d * d) * Bh)) * 0.5f);
  J.zt = l;
  J.sq = -kdx;
  p[0] = y + dy;
  p[1] = z + t * l;
  p[2] = s2;
  x = x2;
  return true;
}

// C' = J C J^T with index-ascending sums over the non-zero entries of J.
TPC_HD void transport_cov(const Jac& J, float C[15]) {
  float Cf[5][5];
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j < 5; ++j) Cf[i][j] = C[sidx(i, j)];
  float T[5][5];
#pragma unroll
  for (int l = 0; l < 5; ++l) {
    T[0][l] = (Cf[0][l] + J.ys * Cf[2][l]) + J.yq * Cf[4][l];
    T[1][l] = ((Cf[1][l] + J.zs * Cf[2][l]) + J.zt * Cf[3][l]) + J.zq * Cf[4][l];
    T[2][l] = Cf[2][l] + J.sq * Cf[4][l];
    T[3][l] = Cf[3][l];
    T[4][l] = Cf[4][l];
  }
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    C[sidx(i, 0)] = (T[i][0] + T[i][2] * J.ys) + T[i][4] * J.yq;
    if (i >= 1) C[sidx(i, 1)] = ((T[i][1] + T[i][2] * J.zs) + T[i][3] * J.zt) + T[i][4] * J.zq;
    if (i >= 2) C[sidx(i, 2)] = T[i][2] + T[i][4] * J.sq;
    if (i >= 3) C[sidx(i, 3)] = T[i][3];
    if (i >= 4) C[sidx(i, 4)] = T[i][4];
  }
}

TPC_HD bool propagate(float kB, float s_max, float p[5], float C[15], float& x, float x2) {
  Jac J;
  if (!transport(kB, s_max, p, x, x2, J)) return false;
  transport_cov(J, C);
  return true;
}

struct Innov {
  float r0, r1, W00, W01, W11, chi2;
};
TPC_HD Innov innovation(const float p[5], const float C[15], float my, float mz, float vy,
                        float vz) {
  Innov in;
  in.r0 = my - p[0];
  in.r1 = mz - p[1];
  float S00 = C[0] + vy;
  float S01 = C[1];
  float S11 = C[2] + vz;
  float det = S00 * S11 - S01 * S01;
  float idet = 1.0f / det;
  in.W00 = S11 * idet;
  in.W01 = -(S01 * idet);
  in.W11 = S00 * idet;
  in.chi2 = in.r0 * (in.W00 * in.r0 + in.W01 * in.r1) + in.r1 * (in.W01 * in.r0 + in.W11 * in.r1);
  return in;
}
// Kalman gain K = C H^T S^-1; p += K r; C -= K H C (lower triangle).
TPC_HD void apply_update(float p[5], float C[15], const Innov& in) {
  float C0[5], C1[5];
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    C0[j] = C[sidx(j, 0)];
    C1[j] = C[sidx(j, 1)];
  }
  float K0[5], K1[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    K0[i] = C0[i] * in.W00 + C1[i] * in.W01;
    K1[i] = C0[i] * in.W01 + C1[i] * in.W11;
  }
#pragma unroll
  for (int i = 0; i < 5; ++i) p[i] = p[i] + (K0[i] * in.r0 + K1[i] * in.r1);
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) C[sidx(i, j)] = C[sidx(i, j)] - (K0[i] * C0[j] + K1[i] * C1[j]);
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
