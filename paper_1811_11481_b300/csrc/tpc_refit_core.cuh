// Per-track refit (arXiv:1811.11481 Sec. 3) and its adjoint, as plain
// __host__ __device__ functions; the kernels in tpc_refit.cu run one track per
// thread through them.
#pragma once

#include <cmath>

#include "tpc_math.cuh"

namespace tpc {

constexpr int kCk = 20;  // floats per checkpoint: state (5) + covariance (15)

struct TrackIn {
  const uint32_t* track_start;
  const float* yc;
  const float* zc;
  const uint32_t* meta;  // row | flags << 8 | sector << 16
};

// Where one track's per-cluster data and checkpoints live: element i at
// base + i * stride; checkpoint (pass, k, component c) at
// ck_base + ((pass - 1) * L + k) * ck_step + c * ck_comp. The contiguous
// layout has stride 1; the warp-interleaved layout has stride 32.
struct Lay {
  size_t base;
  int stride;
  size_t ck_base;
  int L;
  int ck_step;
  int ck_comp;
  TPC_HD size_t at(int i) const { return base + (size_t)i * stride; }
  TPC_HD size_t ck(int pass, int k, int c) const {
    return ck_base + ((size_t)(pass - 1) * L + k) * ck_step + (size_t)c * ck_comp;
  }
};
TPC_HD Lay contiguous_layout(uint32_t a, int n) {
  Lay l;
  l.base = a;
  l.stride = 1;
  l.ck_base = (size_t)3 * a * kCk;
  l.L = n;
  l.ck_step = kCk;
  l.ck_comp = 1;
  return l;
}

// Sector frames (Sec. 2: 18 trapezoidal sectors per side): sectors k and
// k + 18 share the frame rotated by (k + 1/2) * 20 degrees about the beam
// axis, so two frames differ by a multiple of 20 degrees.
constexpr int kFrames = 18;

struct RefitCfg {
  float kB, s_max, sigma, chi2_out, refit_inflate;
  int32_t min_acc_reject;
  float c0r[5];
  // error scale of each cluster flag bit (split, single row, single time,
  // edge, shared)
  float flag_scale[5];
  float rot_c[kFrames], rot_s[kFrames];  // cos, sin of m * 20 degrees
  float frame_c[kFrames], frame_s[kFrames];  // cos, sin of each frame's angle
  int32_t field_on;
  float field[30];  // (Bx, By, Bz) polynomials, as in Geo
};

inline void set_frame_rotations(RefitCfg& c) {
  for (int m = 0; m < kFrames; ++m) {
    double a = m * (3.14159265358979323846 / 9.0);
    c.rot_c[m] = (float)std::cos(a);
    c.rot_s[m] = (float)std::sin(a);
    double f = (m + 0.5) * (3.14159265358979323846 / 9.0);
    c.frame_c[m] = (float)std::cos(f);
    c.frame_s[m] = (float)std::sin(f);
  }
}

// ---------------------------------------------------- the full field (Sec. 3)
// (Bx, By, Bz) at global (X, Y, Z) cm: quadratic polynomials in metres.
TPC_HD void field_at(const RefitCfg& p, float X, float Y, float Z, float B[3]) {
  float x = X * 0.01f, y = Y * 0.01f, z = Z * 0.01f;
  const float m[10] = {1.0f, x, y, z, x * x, x * y, x * z, y * y, y * z, z * z};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float acc = 0.0f;
#pragma unroll
    for (int i = 0; i < 10; ++i) acc += p.field[k * 10 + i] * m[i];
    B[k] = acc;
  }
}

// Transport in the full field from x to x2 in the frame (ca, sa). The
// equations of motion of the unit direction u with x as the variable
// (dy/dx = u_y / u_x, dz/dx = u_z / u_x, du/dx = k (q/p) (u x B) / u_x, q/p
// conserved) are integrated by fourth-order Runge-Kutta in steps of at most
// 0.5 cm twice: in the full field and in the uniform field of the local Bz at
// the start. The state is the exact helix of that uniform field plus the
// difference of the two integrations (their truncation and single-precision
// rounding errors largely cancel; a uniform field gives the helix exactly);
// the covariance follows with the helix Jacobian. Fails where u_x would not
// stay positive or |sin(phi)| reaches s_max.
TPC_HD bool rk4_field(const RefitCfg& p, const float st[5], float x, float x2, float ca,
                      float sa, bool uniform, float bz, float out[5]) {
  float s = st[2], t = st[3], q = st[4];
  float cl = 1.0f / sqrtf(1.0f + t * t);
  float cf = sqrtf(1.0f - s * s);
  float v[5] = {0.0f, 0.0f, cf * cl, s * cl, t * cl};  // y, z as offsets
  float kq = 2.99792458e-3f * (q * cl);
  float dx = x2 - x;
  int ns = (int)ceilf(fabsf(dx) * 2.0f);
  if (ns < 1) ns = 1;
  float h = dx / (float)ns;
  float xx = x;
  auto deriv = [&](float xa, const float w[5], float d[5]) {
    if (!(w[2] > 0.0f)) return false;
    float b0 = 0.0f, b1 = 0.0f, b2 = bz;
    if (!uniform) {
      float B[3];
      float yy = st[0] + w[0];
      field_at(p, xa * ca - yy * sa, xa * sa + yy * ca, st[1] + w[1], B);
      b0 = B[0] * ca + B[1] * sa;
      b1 = -(B[0] * sa) + B[1] * ca;
      b2 = B[2];
    }
    float iu = 1.0f / w[2];
    float f = kq * iu;
    d[0] = w[3] * iu;
    d[1] = w[4] * iu;
    d[2] = f * (w[3] * b2 - w[4] * b1);
    d[3] = f * (w[4] * b0 - w[2] * b2);
    d[4] = f * (w[2] * b1 - w[3] * b0);
    return true;
  };
  for (int i = 0; i < ns; ++i) {
    float k1[5], k2[5], k3[5], k4[5], w[5];
    if (!deriv(xx, v, k1)) return false;
#pragma unroll
    for (int j = 0; j < 5; ++j) w[j] = v[j] + (h * 0.5f) * k1[j];
    if (!deriv(xx + h * 0.5f, w, k2)) return false;
#pragma unroll
    for (int j = 0; j < 5; ++j) w[j] = v[j] + (h * 0.5f) * k2[j];
    if (!deriv(xx + h * 0.5f, w, k3)) return false;
#pragma unroll
    for (int j = 0; j < 5; ++j) w[j] = v[j] + h * k3[j];
    if (!deriv(xx + h, w, k4)) return false;
#pragma unroll
    for (int j = 0; j < 5; ++j)
      v[j] = v[j] + (h / 6.0f) * (k1[j] + 2.0f * k2[j] + 2.0f * k3[j] + k4[j]);
    xx = (i == ns - 1) ? x2 : xx + h;
  }
  float un = sqrtf(v[2] * v[2] + v[3] * v[3] + v[4] * v[4]);
  float ux = v[2] / un, uy = v[3] / un, uz = v[4] / un;
  float rho = sqrtf(ux * ux + uy * uy);
  if (!(ux > 0.0f)) return false;
  out[0] = v[0];
  out[1] = v[1];
  out[2] = uy / rho;
  out[3] = uz / rho;
  out[4] = (q * cl) / rho;
  return true;
}

TPC_HD bool propagate_field(const RefitCfg& p, float st[5], float C[15], float& x, float x2,
                            float ca, float sa) {
  float Bs[3];
  field_at(p, x * ca - st[0] * sa, x * sa + st[0] * ca, st[1], Bs);
  float kBl = 2.99792458e-3f * Bs[2];
  float hp[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) hp[i] = st[i];
  float hx = x;
  if (!propagate(kBl, p.s_max, hp, C, hx, x2)) return false;
  float full[5], unif[5];
  if (!rk4_field(p, st, x, x2, ca, sa, false, Bs[2], full)) return false;
  if (!rk4_field(p, st, x, x2, ca, sa, true, Bs[2], unif)) return false;
  float s2 = hp[2] + (full[2] - unif[2]);
  if (!(fabsf(s2) < p.s_max)) return false;
#pragma unroll
  for (int k = 0; k < 5; ++k) st[k] = hp[k] + (full[k] - unif[k]);
  x = x2;
  return true;
}

TPC_HD int frame_of(uint32_t meta) { return (int)((meta >> 16) & 0xffu) % kFrames; }

// Rotation index from frame a to frame b (angle alpha_b - alpha_a).
TPC_HD int frame_step(int a, int b) { return b >= a ? b - a : b - a + kFrames; }

// C' = J C J^T for the rotation Jacobian: J is the identity except
// J00 = j00, J10 = j10, J20 = j20, J22 = j22.
TPC_HD void rotate_cov(float j00, float j10, float j20, float j22, float C[15]) {
  float Cf[5][5];
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j < 5; ++j) Cf[i][j] = C[sidx(i, j)];
  float M[5][5];
#pragma unroll
  for (int l = 0; l < 5; ++l) {
    M[0][l] = j00 * Cf[0][l];
    M[1][l] = Cf[1][l] + j10 * Cf[0][l];
    M[2][l] = j20 * Cf[0][l] + j22 * Cf[2][l];
    M[3][l] = Cf[3][l];
    M[4][l] = Cf[4][l];
  }
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    C[sidx(i, 0)] = M[i][0] * j00;
    if (i >= 1) C[sidx(i, 1)] = M[i][1] + j10 * M[i][0];
    if (i >= 2) C[sidx(i, 2)] = j20 * M[i][0] + j22 * M[i][2];
    if (i >= 3) C[sidx(i, 3)] = M[i][3];
    if (i >= 4) C[sidx(i, 4)] = M[i][4];
  }
}

// The same helix at the same point in a frame rotated by alpha (ca, sa =
// cos, sin): position and direction rotate and the state then refers to the
// plane x' = x ca + y sa of the new frame. The covariance follows with the
// Jacobian of the state at that plane: a shift of y at fixed x moves the
// point off the plane, and the track is followed back to it along its
// tangent. Returns false when the track would leave the new frame's forward
// half-plane or reach s_max (merged tracks, Sec. 2 second phase).
TPC_HD bool rotate_frame(float kB, float s_max, float ca, float sa, float p[5], float C[15],
                         float& x) {
  float y = p[0], s = p[2], t = p[3], q = p[4];
  float cf = sqrtf(1.0f - s * s);
  float s2 = s * ca - cf * sa;
  float c2 = cf * ca + s * sa;
  if (!(c2 > 0.0f) || !(fabsf(s2) < s_max)) return false;
  rotate_cov(cf / c2, -(sa * t) / c2, (kB * q) * sa, c2 / cf, C);
  float x2 = x * ca + y * sa;
  p[0] = -(x * sa) + y * ca;
  p[2] = s2;
  x = x2;
  return true;
}

// Position variance of a cluster: the error scaled by the factor of each
// flag bit it carries, in bit order (Sec. 3: special clusters get larger
// errors).
TPC_HD float cl_var(const RefitCfg& p, uint32_t meta) {
  uint32_t f = (meta >> 8) & 0x1fu;
  float e = p.sigma;
#pragma unroll
  for (int b = 0; b < 5; ++b)
    if (f & (1u << b)) e = e * p.flag_scale[b];
  return e * e;
}

// Seed at the outermost cluster from the circle through the innermost,
// middle and outermost clusters.
// The three points are expressed in the frame of the outermost cluster.
TPC_HD bool seed3(const Geo& g, const RefitCfg& p, const TrackIn& in, const Lay& ly, int n,
                  float st[5]) {
  if (n < 3) return false;
  int i0 = 0, im = n / 2, i2 = n - 1;
  uint32_t m0 = in.meta[ly.at(i0)], mm = in.meta[ly.at(im)], m2 = in.meta[ly.at(i2)];
  float x0 = g.rx[m0 & 0xffu], xm = g.rx[mm & 0xffu], x2 = g.rx[m2 & 0xffu];
  float y0 = in.yc[ly.at(i0)], ym = in.yc[ly.at(im)], y2 = in.yc[ly.at(i2)];
  int f2 = frame_of(m2);
  auto to_outer = [&](uint32_t m, float& xx, float& yy) {
    int d = frame_step(frame_of(m), f2);
    if (d == 0) return;
    float ca = p.rot_c[d], sa = p.rot_s[d];
    float xr = xx * ca + yy * sa;
    yy = -(xx * sa) + yy * ca;
    xx = xr;
  };
  to_outer(m0, x0, y0);
  to_outer(mm, xm, ym);
  float ax = xm - x0, ay = ym - y0, bx = x2 - x0, by = y2 - y0, ex = x2 - xm, ey = y2 - ym;
  float cross = ax * by - ay * bx;
  float la = sqrtf(ax * ax + ay * ay), lb = sqrtf(bx * bx + by * by),
        le = sqrtf(ex * ex + ey * ey);
  float kap = (-2.0f * cross) / ((la * lb) * le);
  float hs = (kap * lb) * 0.5f;
  if (!(fabsf(hs) < 1.0f)) return false;
  float s2 = (by / lb) * sqrtf(1.0f - hs * hs) - (bx / lb) * hs;
  float arc = lb * arc_factor(hs);
  st[0] = y2;
  st[1] = in.zc[ly.at(i2)];
  st[2] = s2;
  st[3] = (in.zc[ly.at(i2)] - in.zc[ly.at(i0)]) / arc;
  // without a field q/pT is not observable: it stays 0 (straight lines)
  st[4] = g.kB != 0.0f ? kap / g.kB : 0.0f;
  return true;
}

struct RefitOut {
  float st[5];
  float C[15];
  float x;
  float chi2;
  int32_t ndf;
  int32_t status;  // 0 ok, 1 propagation failed, 2 no seed
};

// Optional vertex pseudo-measurement of a track: after pass 3 the state is
// transported to the beam line (x = 0 in every sector frame) and updated
// with (y, z) = (0, zv) of variance var each, like a triggered event with a
// known vertex; it pins the absolute z scale that drift velocity and time
// offset otherwise share with every track's z0 and tan(lambda). Skipped
// when zv is NaN or the transport to x = 0 fails (|sin(phi)| would reach
// its limit). ck (may be null): 24 floats per track, the state (5) and
// covariance (15) entering the step and 1 when it was applied.
struct Vertex {
  float zv;
  float var;
  float* ck;
};
constexpr int kVtxCk = 24;

// True when the track's clusters lie in more than one sector frame.
TPC_HD bool spans_frames(const TrackIn& in, const Lay& ly, int n) {
  if (n <= 0) return false;
  int f0 = frame_of(in.meta[ly.at(0)]);
  bool multi = false;
  for (int k = 1; k < n; ++k) multi = multi || frame_of(in.meta[ly.at(k)]) != f0;
  return multi;
}

// Three passes (inward, outward, inward); rej[at(k)] receives the pass that
// rejected cluster k (0 = kept). ckpt (may be null): state before each step.
// kRot: the clusters may lie in several sector frames (the state is rotated
// into each cluster's frame before the transport to it).
// kField: transport in the full field (propagate_field) instead of the helix.
template <bool kRot, bool kField>
TPC_HD RefitOut refit_track_in(const Geo& g, const RefitCfg& p, const TrackIn& in, const Lay& ly,
                               int n, uint8_t* rej, float* seed_out, float* ckpt,
                               const Vertex vx = Vertex{NAN, 0.0f, nullptr}) {
  RefitOut o;
  for (int k = 0; k < n; ++k) rej[ly.at(k)] = 0;
  o.status = 0;
  o.chi2 = 0.0f;
  o.ndf = 0;
  float* st = o.st;
  float* C = o.C;
  if (!seed3(g, p, in, ly, n, st)) {
    o.status = 2;
    for (int i = 0; i < 5; ++i) st[i] = 0.0f;
    for (int i = 0; i < 15; ++i) C[i] = 0.0f;
    o.x = 0.0f;
    return o;
  }
  if (seed_out)
    for (int i = 0; i < 5; ++i) seed_out[i] = st[i];
  float x = g.rx[in.meta[ly.at(n - 1)] & 0xffu];
  int fr = frame_of(in.meta[ly.at(n - 1)]);  // frame of the state
  set_diag(C, p.c0r);
  float chi2 = 0.0f;
  int ndf = 0;
  for (int pass = 1; pass <= 3; ++pass) {
    if (pass > 1)
      for (int i = 0; i < 15; ++i) C[i] = C[i] * p.refit_inflate;
    chi2 = 0.0f;
    ndf = 0;
    int nacc = 0;
    // data of the current step; the next step's is loaded before the
    // current step's arithmetic so that the loads overlap it
    int i = pass == 2 ? 0 : n - 1;
    int rj = rej[ly.at(i)];
    uint32_t m = in.meta[ly.at(i)];
    float my = in.yc[ly.at(i)], mz = in.zc[ly.at(i)];
    for (int k = 0; k < n; ++k) {
      int k1 = k + 1 < n ? k + 1 : k;
      int i1 = pass == 2 ? k1 : n - 1 - k1;
      int rj1 = rej[ly.at(i1)];
      uint32_t m1 = in.meta[ly.at(i1)];
      float my1 = in.yc[ly.at(i1)], mz1 = in.zc[ly.at(i1)];
      if (!(rj != 0 && rj < pass)) {
        if (ckpt) {
          for (int j = 0; j < 5; ++j) ckpt[ly.ck(pass, k, j)] = st[j];
          for (int j = 0; j < 15; ++j) ckpt[ly.ck(pass, k, 5 + j)] = C[j];
        }
        int fi = frame_of(m);
        if (kRot && fi != fr) {
          int d = frame_step(fr, fi);
          if (!rotate_frame(p.kB, p.s_max, p.rot_c[d], p.rot_s[d], st, C, x)) {
            o.status = 1;
            o.x = x;
            return o;
          }
          fr = fi;
        }
        bool moved = kField ? propagate_field(p, st, C, x, g.rx[m & 0xffu], p.frame_c[fr],
                                              p.frame_s[fr])
                            : propagate(p.kB, p.s_max, st, C, x, g.rx[m & 0xffu]);
        if (!moved) {
          o.status = 1;
          o.x = x;
          return o;
        }
        float v = cl_var(p, m);
        Innov iv = innovation(st, C, my, mz, v, v);
        if (nacc >= p.min_acc_reject && iv.chi2 > p.chi2_out) {
          rej[ly.at(i)] = (uint8_t)pass;
        } else {
          apply_update(st, C, iv);
          chi2 = chi2 + iv.chi2;
          ndf += 2;
          ++nacc;
        }
      }
      i = i1;
      rj = rj1;
      m = m1;
      my = my1;
      mz = mz1;
    }
  }
  if (!kField && !(vx.zv != vx.zv)) {
    if (vx.ck) {
      for (int j = 0; j < 5; ++j) vx.ck[j] = st[j];
      for (int j = 0; j < 15; ++j) vx.ck[5 + j] = C[j];
      vx.ck[20] = x;
      vx.ck[21] = 0.0f;
    }
    float sv[5], Cv[15], xv = x;
    for (int j = 0; j < 5; ++j) sv[j] = st[j];
    for (int j = 0; j < 15; ++j) Cv[j] = C[j];
    if (propagate(p.kB, p.s_max, sv, Cv, xv, 0.0f)) {
      Innov iv = innovation(sv, Cv, 0.0f, vx.zv, vx.var, vx.var);
      apply_update(sv, Cv, iv);
      for (int j = 0; j < 5; ++j) st[j] = sv[j];
      for (int j = 0; j < 15; ++j) C[j] = Cv[j];
      x = xv;
      chi2 = chi2 + iv.chi2;
      ndf += 2;
      if (vx.ck) vx.ck[21] = 1.0f;
    }
  }
  o.x = x;
  o.chi2 = chi2;
  o.ndf = ndf;
  return o;
}

// multi: the track's clusters lie in more than one sector frame
// (spans_frames). kField: transport in the full field.
template <bool kField = false>
TPC_HD RefitOut refit_track(const Geo& g, const RefitCfg& p, const TrackIn& in, const Lay& ly,
                            int n, uint8_t* rej, float* seed_out, float* ckpt, bool multi,
                            const Vertex vx = Vertex{NAN, 0.0f, nullptr}) {
  return multi ? refit_track_in<true, kField>(g, p, in, ly, n, rej, seed_out, ckpt, vx)
               : refit_track_in<false, kField>(g, p, in, ly, n, rej, seed_out, ckpt, vx);
}

// ------------------------------------------------------------ dual numbers
// Forward-mode derivative in (sin phi, tan lambda, q/pT).
struct D3 {
  float v, d0, d1, d2;
};
TPC_HD D3 dc(float v) { return D3{v, 0.f, 0.f, 0.f}; }
TPC_HD D3 operator+(D3 a, D3 b) { return D3{a.v + b.v, a.d0 + b.d0, a.d1 + b.d1, a.d2 + b.d2}; }
TPC_HD D3 operator-(D3 a, D3 b) { return D3{a.v - b.v, a.d0 - b.d0, a.d1 - b.d1, a.d2 - b.d2}; }
TPC_HD D3 operator-(D3 a) { return D3{-a.v, -a.d0, -a.d1, -a.d2}; }
TPC_HD D3 operator*(D3 a, D3 b) {
  return D3{a.v * b.v, a.d0 * b.v + a.v * b.d0, a.d1 * b.v + a.v * b.d1, a.d2 * b.v + a.v * b.d2};
}
TPC_HD D3 operator*(float s, D3 b) { return D3{s * b.v, s * b.d0, s * b.d1, s * b.d2}; }
TPC_HD D3 operator/(D3 a, D3 b) {
  float q = a.v / b.v, ib = 1.0f / b.v;
  return D3{q, (a.d0 - q * b.d0) * ib, (a.d1 - q * b.d1) * ib, (a.d2 - q * b.d2) * ib};
}
TPC_HD D3 dsqrt(D3 a) {
  float s = sqrtf(a.v), h = 0.5f / s;
  return D3{s, a.d0 * h, a.d1 * h, a.d2 * h};
}
TPC_HD D3 chain(D3 a, float f, float df) { return D3{f, a.d0 * df, a.d1 * df, a.d2 * df}; }

// d/dh of B(h) = A'(h): from the series for small h, else E^3 - 2 B / h.
TPC_HD float arc_factor_deriv2(float h) {
  if (fabsf(h) < 0.125f) {
    float h2 = h * h;
    float c = 315.0f / 1408.0f;
    c = 35.0f / 144.0f + h2 * c;
    c = 15.0f / 56.0f + h2 * c;
    c = 3.0f / 10.0f + h2 * c;
    c = 1.0f / 3.0f + h2 * c;
    float dc2 = 4.0f * (315.0f / 1408.0f);
    dc2 = 3.0f * (35.0f / 144.0f) + h2 * dc2;
    dc2 = 2.0f * (15.0f / 56.0f) + h2 * dc2;
    dc2 = 3.0f / 10.0f + h2 * dc2;
    return c + 2.0f * h2 * dc2;
  }
  float e = 1.0f / sqrtf(1.0f - h * h);
  return e * e * e - 2.0f * arc_factor_deriv(h) / h;
}

// Gradient in (s, t, q) of <Jbar, J> over the state-dependent Jacobian entries.
TPC_HD void jac_vjp(float kB, float dx, float sv, float tv, float qv, float b_ys, float b_yq,
                    float b_zs, float b_zt, float b_zq, float g[3]) {
  D3 s{sv, 1.f, 0.f, 0.f}, t{tv, 0.f, 1.f, 0.f}, q{qv, 0.f, 0.f, 1.f};
  D3 kap = kB * q;
  D3 s2 = s - dx * kap;
  D3 one = dc(1.0f);
  D3 c1 = dsqrt(one - s * s);
  D3 c2 = dsqrt(one - s2 * s2);
  D3 N = s + s2;
  D3 D = c1 + c2;
  D3 T = N / D;
  D3 opt = one + T * T;
  D3 d = dx * dsqrt(opt);
  D3 h = 0.5f * (kap * d);
  D3 A = chain(h, arc_factor(h.v), arc_factor_deriv(h.v));
  D3 l = d * A;
  D3 dDds = -(s / c1) - (s2 / c2);
  float kdx = kB * dx;
  D3 dDdq = kdx * (s2 / c2);
  D3 dTds = (dc(2.0f) - T * dDds) / D;
  D3 dTdq = (dc(-kdx) - T * dDdq) / D;
  D3 Jys = dx * dTds;
  D3 Jyq = dx * dTdq;
  D3 gg = (d * T) / opt;
  D3 dds = gg * dTds;
  D3 ddq = gg * dTdq;
  D3 E = one / dsqrt(one - h * h);
  D3 Bh = chain(h, arc_factor_deriv(h.v), arc_factor_deriv2(h.v));
  D3 Jzs = t * (E * dds);
  D3 Jzq = t * (E * ddq + 0.5f * (kB * ((d * d) * Bh)));
  D3 Jzt = l;
  g[0] = b_ys * Jys.d0 + b_yq * Jyq.d0 + b_zs * Jzs.d0 + b_zt * Jzt.d0 + b_zq * Jzq.d0;
  g[1] = b_ys * Jys.d1 + b_yq * Jyq.d1 + b_zs * Jzs.d1 + b_zt * Jzt.d1 + b_zq * Jzq.d1;
  g[2] = b_ys * Jys.d2 + b_yq * Jyq.d2 + b_zs * Jzs.d2 + b_zt * Jzt.d2 + b_zq * Jzq.d2;
}

TPC_HD void unpack(const float P[15], float F[5][5]) {
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) F[i][j] = P[sidx(i, j)];
}

// Adjoint of the Kalman update at the predicted state (Pp = predicted
// covariance): on entry pb, G are the adjoints of the updated state and of
// the updated covariance (full symmetric matrix, packed); on exit those of
// the predicted ones. cbar is the adjoint of the chi2 increment; mbar
// receives the adjoint of the measurement.
TPC_HD void update_adjoint(const float Pp[15], const Innov& in, float cbar, float pb[5],
                           float G[15], float mbar[2]) {
  float P[5][5], Gf[5][5];
  unpack(Pp, P);
  unpack(G, Gf);
  float r0 = in.r0, r1 = in.r1;
  float W00 = in.W00, W01 = in.W01, W11 = in.W11;
  float u0 = W00 * r0 + W01 * r1, u1 = W01 * r0 + W11 * r1;
  float ub0 = 0.f, ub1 = 0.f;
  for (int i = 0; i < 5; ++i) {
    ub0 += P[i][0] * pb[i];
    ub1 += P[i][1] * pb[i];
  }
  float BW0[5], BW1[5];
  for (int i = 0; i < 5; ++i) {
    BW0[i] = P[i][0] * W00 + P[i][1] * W01;
    BW1[i] = P[i][0] * W01 + P[i][1] * W11;
  }
  float Bb0[5], Bb1[5], GB0[5], GB1[5];
  for (int i = 0; i < 5; ++i) {
    float a0 = 0.f, a1 = 0.f, c0 = 0.f, c1 = 0.f;
    for (int k = 0; k < 5; ++k) {
      a0 += Gf[i][k] * BW0[k];
      a1 += Gf[i][k] * BW1[k];
      c0 += Gf[i][k] * P[k][0];
      c1 += Gf[i][k] * P[k][1];
    }
    Bb0[i] = pb[i] * u0 - 2.0f * a0;
    Bb1[i] = pb[i] * u1 - 2.0f * a1;
    GB0[i] = c0;
    GB1[i] = c1;
  }
  float M00 = 0.f, M01 = 0.f, M10 = 0.f, M11 = 0.f;  // B^T G B
  for (int i = 0; i < 5; ++i) {
    M00 += P[i][0] * GB0[i];
    M01 += P[i][0] * GB1[i];
    M10 += P[i][1] * GB0[i];
    M11 += P[i][1] * GB1[i];
  }
  float Wb00 = -M00 + cbar * r0 * r0 + ub0 * r0;
  float Wb01 = -M01 + cbar * r0 * r1 + ub0 * r1;
  float Wb10 = -M10 + cbar * r1 * r0 + ub1 * r0;
  float Wb11 = -M11 + cbar * r1 * r1 + ub1 * r1;
  float rb0 = 2.0f * cbar * u0 + W00 * ub0 + W01 * ub1;
  float rb1 = 2.0f * cbar * u1 + W01 * ub0 + W11 * ub1;
  // S_bar = -W Wbar W
  float X00 = W00 * Wb00 + W01 * Wb10, X01 = W00 * Wb01 + W01 * Wb11;
  float X10 = W01 * Wb00 + W11 * Wb10, X11 = W01 * Wb01 + W11 * Wb11;
  float Sb00 = -(X00 * W00 + X01 * W01), Sb01 = -(X00 * W01 + X01 * W11);
  float Sb10 = -(X10 * W00 + X11 * W01), Sb11 = -(X10 * W01 + X11 * W11);
  float Pb[5][5];
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) Pb[i][j] = Gf[i][j];
  for (int i = 0; i < 5; ++i) {
    Pb[i][0] += Bb0[i];
    Pb[i][1] += Bb1[i];
  }
  Pb[0][0] += Sb00;
  Pb[0][1] += Sb01;
  Pb[1][0] += Sb10;
  Pb[1][1] += Sb11;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j <= i; ++j) G[sidx(i, j)] = 0.5f * (Pb[i][j] + Pb[j][i]);
  mbar[0] = rb0;
  mbar[1] = rb1;
  pb[0] -= rb0;
  pb[1] -= rb1;
}

// Adjoint of the helix transport of state and covariance. p, Cp: state and
// covariance before the step; on entry pb, G are the adjoints after it.
// J differs from the identity only in (0,2) (0,4) (1,2) (1,3) (1,4) (2,4).
TPC_HD void transport_adjoint(float kB, float dx, const float p[5], const float Cp[15],
                              const Jac& J, float pb[5], float G[15]) {
  float Cf[5][5], Gf[5][5];
  unpack(Cp, Cf);
  unpack(G, Gf);
  // M = J C (rows 3 and 4 are those of C)
  float M[5][5];
  for (int l = 0; l < 5; ++l) {
    M[0][l] = Cf[0][l] + J.ys * Cf[2][l] + J.yq * Cf[4][l];
    M[1][l] = Cf[1][l] + J.zs * Cf[2][l] + J.zt * Cf[3][l] + J.zq * Cf[4][l];
    M[2][l] = Cf[2][l] + J.sq * Cf[4][l];
    M[3][l] = Cf[3][l];
    M[4][l] = Cf[4][l];
  }
  // Jbar = 2 G J C at the state-dependent entries (rows 0 and 1)
  float Jb[2][5];
  for (int a = 0; a < 2; ++a)
    for (int b = 2; b < 5; ++b) {
      float acc = 0.f;
      for (int c = 0; c < 5; ++c) acc += Gf[a][c] * M[c][b];
      Jb[a][b] = 2.0f * acc;
    }
  float gq[3];
  jac_vjp(kB, dx, p[2], p[3], p[4], Jb[0][2], Jb[0][4], Jb[1][2], Jb[1][3], Jb[1][4], gq);
  float n2 = J.ys * pb[0] + J.zs * pb[1] + pb[2] + gq[0];
  float n3 = J.zt * pb[1] + pb[3] + gq[1];
  float n4 = J.yq * pb[0] + J.zq * pb[1] + J.sq * pb[2] + pb[4] + gq[2];
  pb[2] = n2;
  pb[3] = n3;
  pb[4] = n4;
  // X = G J (column operations), then J^T X (row operations)
  float X[5][5];
  for (int i = 0; i < 5; ++i) {
    X[i][0] = Gf[i][0];
    X[i][1] = Gf[i][1];
    X[i][2] = J.ys * Gf[i][0] + J.zs * Gf[i][1] + Gf[i][2];
    X[i][3] = J.zt * Gf[i][1] + Gf[i][3];
    X[i][4] = J.yq * Gf[i][0] + J.zq * Gf[i][1] + J.sq * Gf[i][2] + Gf[i][4];
  }
  for (int j = 0; j < 5; ++j) {
    float r0 = X[0][j], r1 = X[1][j], r2 = X[2][j], r3 = X[3][j], r4 = X[4][j];
    float c2 = J.ys * r0 + J.zs * r1 + r2;
    float c3 = J.zt * r1 + r3;
    float c4 = J.yq * r0 + J.zq * r1 + J.sq * r2 + r4;
    float col[5] = {r0, r1, c2, c3, c4};
    for (int i = j; i < 5; ++i) G[sidx(i, j)] = col[i];
  }
}

// Adjoint of the start x of a transport (the step length dx = x2 - x falls
// as x grows), for steps that start at a state-dependent x (after a frame
// rotation). p, Cp: state and covariance before the step, pe: state after
// it; pb, G: adjoints after the step (before transport_adjoint consumes
// them). The end point slides along the track (dy/dx = tan phi, dz/dx =
// tan lambda / cos phi, dsin(phi)/dx = -kappa) and the Jacobian entries
// change with dx, differentiated with a dual number in dx.
TPC_HD float transport_x_adjoint(float kB, float dx, const float p[5], const float pe[5],
                                 const float Cp[15], const Jac& J, const float pb[5],
                                 const float G[15]) {
  float kap = kB * p[4];
  float s2v = pe[2];
  float ic2 = 1.0f / sqrtf(1.0f - s2v * s2v);
  float g = pb[0] * (s2v * ic2) + pb[1] * (p[3] * ic2) - pb[2] * kap;
  D3 X{dx, 1.f, 0.f, 0.f};
  D3 s = dc(p[2]);
  float t = p[3];
  D3 one = dc(1.0f);
  D3 s2 = s - kap * X;
  D3 c1 = dsqrt(one - s * s);
  D3 c2 = dsqrt(one - s2 * s2);
  D3 N = s + s2;
  D3 D = c1 + c2;
  D3 T = N / D;
  D3 opt = one + T * T;
  D3 d = X * dsqrt(opt);
  D3 h = 0.5f * (kap * d);
  D3 A = chain(h, arc_factor(h.v), arc_factor_deriv(h.v));
  D3 l = d * A;
  D3 dDds = -(s / c1) - (s2 / c2);
  D3 kdx = kB * X;
  D3 dDdq = kdx * (s2 / c2);
  D3 dTds = (dc(2.0f) - T * dDds) / D;
  D3 dTdq = (-kdx - T * dDdq) / D;
  D3 Jys = X * dTds;
  D3 Jyq = X * dTdq;
  D3 gg = (d * T) / opt;
  D3 E = one / dsqrt(one - h * h);
  D3 Bh = chain(h, arc_factor_deriv(h.v), arc_factor_deriv2(h.v));
  D3 Jzs = t * (E * (gg * dTds));
  D3 Jzq = t * (E * (gg * dTdq) + 0.5f * (kB * ((d * d) * Bh)));
  D3 Jzt = l;
  // Jbar = 2 G J C at the entries that depend on dx: rows 0..2, columns 2..4
  float Cf[5][5], Gf[5][5];
  unpack(Cp, Cf);
  unpack(G, Gf);
  float M[5][3];
  for (int b = 0; b < 3; ++b) {
    int l2 = b + 2;
    M[0][b] = Cf[0][l2] + J.ys * Cf[2][l2] + J.yq * Cf[4][l2];
    M[1][b] = Cf[1][l2] + J.zs * Cf[2][l2] + J.zt * Cf[3][l2] + J.zq * Cf[4][l2];
    M[2][b] = Cf[2][l2] + J.sq * Cf[4][l2];
    M[3][b] = Cf[3][l2];
    M[4][b] = Cf[4][l2];
  }
  float Jb[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      float acc = 0.f;
      for (int c = 0; c < 5; ++c) acc += Gf[a][c] * M[c][b];
      Jb[a][b] = 2.0f * acc;
    }
  float gj = Jb[0][0] * Jys.d0 + Jb[0][2] * Jyq.d0 + Jb[1][0] * Jzs.d0 + Jb[1][1] * Jzt.d0 +
             Jb[1][2] * Jzq.d0 - Jb[2][2] * kB;
  return -(g + gj);
}

// Adjoint of rotate_frame at the state p (before the rotation, reference x
// fixed) with covariance Cp: on entry pb, G, xb are the adjoints of the
// rotated state, covariance and reference x; on exit pb, G are those of p
// and Cp. The rotation Jacobian depends on (sin phi, tan lambda, q/pT): its
// second-order term with a dual number in those three.
TPC_HD void rotate_adjoint(float kB, float ca, float sa, const float p[5], const float Cp[15],
                           float xb, float pb[5], float G[15]) {
  D3 s{p[2], 1.f, 0.f, 0.f}, t{p[3], 0.f, 1.f, 0.f}, q{p[4], 0.f, 0.f, 1.f};
  D3 one = dc(1.0f);
  D3 cf = dsqrt(one - s * s);
  D3 c2 = ca * cf + sa * s;
  D3 j00 = cf / c2;
  D3 j10 = -(sa * t) / c2;
  D3 j20 = (kB * sa) * q;
  D3 j22 = c2 / cf;
  float Cf[5][5], Gf[5][5];
  unpack(Cp, Cf);
  unpack(G, Gf);
  // columns 0 and 2 of J C
  float M0[5], M2[5];
  M0[0] = j00.v * Cf[0][0];
  M2[0] = j00.v * Cf[0][2];
  M0[1] = Cf[1][0] + j10.v * Cf[0][0];
  M2[1] = Cf[1][2] + j10.v * Cf[0][2];
  M0[2] = j20.v * Cf[0][0] + j22.v * Cf[2][0];
  M2[2] = j20.v * Cf[0][2] + j22.v * Cf[2][2];
  M0[3] = Cf[3][0];
  M2[3] = Cf[3][2];
  M0[4] = Cf[4][0];
  M2[4] = Cf[4][2];
  float b00 = 0.f, b10 = 0.f, b20 = 0.f, b22 = 0.f;
  for (int c = 0; c < 5; ++c) {
    b00 += Gf[0][c] * M0[c];
    b10 += Gf[1][c] * M0[c];
    b20 += Gf[2][c] * M0[c];
    b22 += Gf[2][c] * M2[c];
  }
  float gs = 2.0f * (b00 * j00.d0 + b10 * j10.d0 + b22 * j22.d0);
  float gt = 2.0f * (b10 * j10.d1);
  float gq = 2.0f * (b20 * j20.d2);
  float dsds = ca + sa * (p[2] / cf.v);
  float n0 = ca * pb[0] + sa * xb;
  float n2 = dsds * pb[2] + gs;
  pb[0] = n0;
  pb[2] = n2;
  pb[3] += gt;
  pb[4] += gq;
  // G <- J^T G J
  float X[5][5];
  for (int i = 0; i < 5; ++i) {
    X[i][0] = Gf[i][0] * j00.v + Gf[i][1] * j10.v + Gf[i][2] * j20.v;
    X[i][1] = Gf[i][1];
    X[i][2] = Gf[i][2] * j22.v;
    X[i][3] = Gf[i][3];
    X[i][4] = Gf[i][4];
  }
  for (int j = 0; j < 5; ++j) {
    float col[5] = {j00.v * X[0][j] + j10.v * X[1][j] + j20.v * X[2][j], X[1][j],
                    j22.v * X[2][j], X[3][j], X[4][j]};
    for (int i = j; i < 5; ++i) G[sidx(i, j)] = col[i];
  }
}

// ------------------------------------------- adjoint of the field transport
// Gradient of the field (T per cm) at global (X, Y, Z) cm: g[k][c] =
// dB_k / d(X, Y, Z)_c of the quadratic polynomials.
TPC_HD void field_grad(const RefitCfg& p, float X, float Y, float Z, float gB[3][3]) {
  float x = X * 0.01f, y = Y * 0.01f, z = Z * 0.01f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float* a = p.field + k * 10;
    gB[k][0] = 0.01f * (a[1] + 2.0f * a[4] * x + a[5] * y + a[6] * z);
    gB[k][1] = 0.01f * (a[2] + a[5] * x + 2.0f * a[7] * y + a[8] * z);
    gB[k][2] = 0.01f * (a[3] + a[6] * x + a[8] * y + 2.0f * a[9] * z);
  }
}

// Adjoint of one evaluation of the equations of motion d = f(xa, w) (as in
// rk4_field) given db: accumulates into wb, and into the adjoints of the
// start y, z (field position), of kq and of the uniform bz.
TPC_HD void rk4_deriv_vjp(const RefitCfg& p, const float st[5], float xa, const float w[5],
                          float ca, float sa, bool uniform, float bz, float kq,
                          const float db[5], float wb[5], float& y0b, float& z0b, float& kqb,
                          float& bzb) {
  float b0 = 0.0f, b1 = 0.0f, b2 = bz;
  float X = 0.0f, Y = 0.0f, Z = 0.0f;
  if (!uniform) {
    float B[3];
    float yy = st[0] + w[0];
    X = xa * ca - yy * sa;
    Y = xa * sa + yy * ca;
    Z = st[1] + w[1];
    field_at(p, X, Y, Z, B);
    b0 = B[0] * ca + B[1] * sa;
    b1 = -(B[0] * sa) + B[1] * ca;
    b2 = B[2];
  }
  float iu = 1.0f / w[2];
  float f = kq * iu;
  float c2 = w[3] * b2 - w[4] * b1, c3 = w[4] * b0 - w[2] * b2, c4 = w[2] * b1 - w[3] * b0;
  float iub = db[0] * w[3] + db[1] * w[4];
  wb[3] += db[0] * iu;
  wb[4] += db[1] * iu;
  float fb = db[2] * c2 + db[3] * c3 + db[4] * c4;
  float c2b = db[2] * f, c3b = db[3] * f, c4b = db[4] * f;
  wb[3] += c2b * b2 - c4b * b0;
  wb[4] += -(c2b * b1) + c3b * b0;
  wb[2] += -(c3b * b2) + c4b * b1;
  float b0b = c3b * w[4] - c4b * w[3];
  float b1b = -(c2b * w[4]) + c4b * w[2];
  float b2b = c2b * w[3] - c3b * w[2];
  kqb += fb * iu;
  iub += fb * kq;
  wb[2] += -iub * iu * iu;
  if (uniform) {
    bzb += b2b;
    return;
  }
  float gB[3][3];
  field_grad(p, X, Y, Z, gB);
  float B0b = b0b * ca - b1b * sa, B1b = b0b * sa + b1b * ca, B2b = b2b;
  float Xb = B0b * gB[0][0] + B1b * gB[1][0] + B2b * gB[2][0];
  float Yb = B0b * gB[0][1] + B1b * gB[1][1] + B2b * gB[2][1];
  float Zb = B0b * gB[0][2] + B1b * gB[1][2] + B2b * gB[2][2];
  float yyb = -(Xb * sa) + Yb * ca;
  wb[0] += yyb;
  y0b += yyb;
  wb[1] += Zb;
  z0b += Zb;
}

constexpr int kMaxSub = 64;  // stored Runge-Kutta sub-step states

// The forward pass of rk4_field with its sub-step start states kept for the
// adjoint (the first kMaxSub of them; later ones are recomputed).
struct Rk4Tape {
  float vs[kMaxSub][5];
  float v[5];  // the end state
  int ns;
};

TPC_HD void rk4_deriv(const RefitCfg& p, const float st[5], float xa, const float w[5], float ca,
                      float sa, bool uniform, float bz, float kq, float d[5]) {
  float b0 = 0.0f, b1 = 0.0f, b2 = bz;
  if (!uniform) {
    float B[3];
    float yy = st[0] + w[0];
    field_at(p, xa * ca - yy * sa, xa * sa + yy * ca, st[1] + w[1], B);
    b0 = B[0] * ca + B[1] * sa;
    b1 = -(B[0] * sa) + B[1] * ca;
    b2 = B[2];
  }
  float iu = 1.0f / w[2];
  float f = kq * iu;
  d[0] = w[3] * iu;
  d[1] = w[4] * iu;
  d[2] = f * (w[3] * b2 - w[4] * b1);
  d[3] = f * (w[4] * b0 - w[2] * b2);
  d[4] = f * (w[2] * b1 - w[3] * b0);
}

TPC_HD void rk4_substep(const RefitCfg& p, const float st[5], float xa, float h, float ca,
                        float sa, bool uniform, float bz, float kq, float v[5]) {
  float k1[5], k2[5], k3[5], k4[5], w[5];
  rk4_deriv(p, st, xa, v, ca, sa, uniform, bz, kq, k1);
  for (int j = 0; j < 5; ++j) w[j] = v[j] + (h * 0.5f) * k1[j];
  rk4_deriv(p, st, xa + h * 0.5f, w, ca, sa, uniform, bz, kq, k2);
  for (int j = 0; j < 5; ++j) w[j] = v[j] + (h * 0.5f) * k2[j];
  rk4_deriv(p, st, xa + h * 0.5f, w, ca, sa, uniform, bz, kq, k3);
  for (int j = 0; j < 5; ++j) w[j] = v[j] + h * k3[j];
  rk4_deriv(p, st, xa + h, w, ca, sa, uniform, bz, kq, k4);
  for (int j = 0; j < 5; ++j)
    v[j] = v[j] + (h / 6.0f) * (k1[j] + 2.0f * k2[j] + 2.0f * k3[j] + k4[j]);
}

// rk4_field's forward pass (same operations, without the failure checks:
// the forward refit passed them), keeping the tape; out as rk4_field's.
TPC_HD void rk4_field_fwd(const RefitCfg& p, const float st[5], float x, float x2, float ca,
                          float sa, bool uniform, float bz, Rk4Tape& tp, float out[5]) {
  float s = st[2], t = st[3], q = st[4];
  float cl = 1.0f / sqrtf(1.0f + t * t);
  float cf = sqrtf(1.0f - s * s);
  float kq = 2.99792458e-3f * (q * cl);
  float dx = x2 - x;
  int ns = (int)ceilf(fabsf(dx) * 2.0f);
  if (ns < 1) ns = 1;
  float h = dx / (float)ns;
  float v[5] = {0.0f, 0.0f, cf * cl, s * cl, t * cl};
  float xa = x;
  for (int i = 0; i < ns; ++i) {
    if (i < kMaxSub)
      for (int j = 0; j < 5; ++j) tp.vs[i][j] = v[j];
    rk4_substep(p, st, xa, h, ca, sa, uniform, bz, kq, v);
    xa = (i == ns - 1) ? x2 : xa + h;
  }
  tp.ns = ns;
  for (int j = 0; j < 5; ++j) tp.v[j] = v[j];
  float un = sqrtf(v[2] * v[2] + v[3] * v[3] + v[4] * v[4]);
  float ux = v[2] / un, uy = v[3] / un, uz = v[4] / un;
  float rho = sqrtf(ux * ux + uy * uy);
  out[0] = v[0];
  out[1] = v[1];
  out[2] = uy / rho;
  out[3] = uz / rho;
  out[4] = (q * cl) / rho;
}

// Adjoint of rk4_field from its tape: given the adjoint ob of its output, the
// adjoint sb of the start state (y, z, sin phi, tan lambda, q/pT) and of the
// uniform bz.
TPC_HD void rk4_field_rev(const RefitCfg& p, const float st[5], float x, float x2, float ca,
                          float sa, bool uniform, float bz, const Rk4Tape& tp,
                          const float ob[5], float sb[5], float& bzb) {
  float s = st[2], t = st[3], q = st[4];
  float cl = 1.0f / sqrtf(1.0f + t * t);
  float cf = sqrtf(1.0f - s * s);
  float kq = 2.99792458e-3f * (q * cl);
  int ns = tp.ns;
  float h = (x2 - x) / (float)ns;
  const float* v = tp.v;
  // output: (v0, v1, uy / rho, uz / rho, q cl / rho) with u = v / |v|
  float un = sqrtf(v[2] * v[2] + v[3] * v[3] + v[4] * v[4]);
  float ux = v[2] / un, uy = v[3] / un, uz = v[4] / un;
  float rho = sqrtf(ux * ux + uy * uy);
  float vb[5] = {ob[0], ob[1], 0.0f, 0.0f, 0.0f};
  float irho = 1.0f / rho;
  float uyb = ob[2] * irho, uzb = ob[3] * irho;
  float rhob = -(ob[2] * uy + ob[3] * uz + ob[4] * (q * cl)) * irho * irho;
  float qclb = ob[4] * irho;
  float uxb = rhob * ux * irho;
  uyb += rhob * uy * irho;
  float dotb = uxb * v[2] + uyb * v[3] + uzb * v[4];
  float iun = 1.0f / un;
  vb[2] = uxb * iun - v[2] * dotb * iun * iun * iun;
  vb[3] = uyb * iun - v[3] * dotb * iun * iun * iun;
  vb[4] = uzb * iun - v[4] * dotb * iun * iun * iun;
  float y0b = 0.0f, z0b = 0.0f, kqb = 0.0f;
  bzb = 0.0f;
  for (int i = ns - 1; i >= 0; --i) {
    float vi[5];
    if (i < kMaxSub) {
      for (int j = 0; j < 5; ++j) vi[j] = tp.vs[i][j];
    } else {
      for (int j = 0; j < 5; ++j) vi[j] = tp.vs[kMaxSub - 1][j];
      float xr = x + h * (float)(kMaxSub - 1);
      for (int r = kMaxSub - 1; r < i; ++r) {
        rk4_substep(p, st, xr, h, ca, sa, uniform, bz, kq, vi);
        xr = xr + h;
      }
    }
    float xi0 = x + h * (float)i;
    float k1[5], k2[5], k3[5], w2[5], w3[5], w4[5];
    rk4_deriv(p, st, xi0, vi, ca, sa, uniform, bz, kq, k1);
    for (int j = 0; j < 5; ++j) w2[j] = vi[j] + (h * 0.5f) * k1[j];
    rk4_deriv(p, st, xi0 + h * 0.5f, w2, ca, sa, uniform, bz, kq, k2);
    for (int j = 0; j < 5; ++j) w3[j] = vi[j] + (h * 0.5f) * k2[j];
    rk4_deriv(p, st, xi0 + h * 0.5f, w3, ca, sa, uniform, bz, kq, k3);
    for (int j = 0; j < 5; ++j) w4[j] = vi[j] + h * k3[j];
    float k1b[5], k2b[5], k3b[5], k4b[5], wb[5];
    for (int j = 0; j < 5; ++j) {
      k1b[j] = (h / 6.0f) * vb[j];
      k2b[j] = (h / 6.0f) * 2.0f * vb[j];
      k3b[j] = (h / 6.0f) * 2.0f * vb[j];
      k4b[j] = (h / 6.0f) * vb[j];
    }
    float xe = (i == ns - 1) ? x2 : xi0 + h;
    for (int j = 0; j < 5; ++j) wb[j] = 0.0f;
    rk4_deriv_vjp(p, st, xe, w4, ca, sa, uniform, bz, kq, k4b, wb, y0b, z0b, kqb, bzb);
    for (int j = 0; j < 5; ++j) {
      vb[j] += wb[j];
      k3b[j] += h * wb[j];
      wb[j] = 0.0f;
    }
    rk4_deriv_vjp(p, st, xi0 + h * 0.5f, w3, ca, sa, uniform, bz, kq, k3b, wb, y0b, z0b, kqb,
                  bzb);
    for (int j = 0; j < 5; ++j) {
      vb[j] += wb[j];
      k2b[j] += (h * 0.5f) * wb[j];
      wb[j] = 0.0f;
    }
    rk4_deriv_vjp(p, st, xi0 + h * 0.5f, w2, ca, sa, uniform, bz, kq, k2b, wb, y0b, z0b, kqb,
                  bzb);
    for (int j = 0; j < 5; ++j) {
      vb[j] += wb[j];
      k1b[j] += (h * 0.5f) * wb[j];
      wb[j] = 0.0f;
    }
    rk4_deriv_vjp(p, st, xi0, vi, ca, sa, uniform, bz, kq, k1b, wb, y0b, z0b, kqb, bzb);
    for (int j = 0; j < 5; ++j) vb[j] += wb[j];
  }
  // the start: v = (0, 0, cf cl, s cl, t cl), kq = K q cl, and q cl of the output
  float clb = vb[2] * cf + vb[3] * s + vb[4] * t + kqb * 2.99792458e-3f * q + qclb * q;
  float cfb = vb[2] * cl;
  sb[0] = y0b;
  sb[1] = z0b;
  sb[2] = vb[3] * cl - cfb * s / cf;
  sb[3] = vb[4] * cl - clb * t * cl * cl * cl;
  sb[4] = kqb * 2.99792458e-3f * cl + qclb * cl;
}

// d/dkB of the helix transport: sum of pb . d(state)/dkB and of Jbar .
// d(Jacobian entries)/dkB (Jbar = 2 G J C), with a dual number in kB.
TPC_HD float transport_kb_adjoint(float kB, float dx, const float p[5], const float Cp[15],
                                  const Jac& J, const float pb[5], const float G[15]) {
  D3 K{kB, 1.f, 0.f, 0.f};
  D3 s = dc(p[2]);
  float t = p[3], q = p[4];
  D3 one = dc(1.0f);
  D3 kap = q * K;
  D3 s2 = s - dx * kap;
  D3 c1 = dsqrt(one - s * s);
  D3 c2 = dsqrt(one - s2 * s2);
  D3 N = s + s2;
  D3 D = c1 + c2;
  D3 T = N / D;
  D3 opt = one + T * T;
  D3 d = dx * dsqrt(opt);
  D3 h = 0.5f * (kap * d);
  D3 A = chain(h, arc_factor(h.v), arc_factor_deriv(h.v));
  D3 l = d * A;
  D3 dDds = -(s / c1) - (s2 / c2);
  D3 kdx = dx * K;
  D3 dDdq = kdx * (s2 / c2);
  D3 dTds = (dc(2.0f) - T * dDds) / D;
  D3 dTdq = (-kdx - T * dDdq) / D;
  D3 Jys = dx * dTds;
  D3 Jyq = dx * dTdq;
  D3 gg = (d * T) / opt;
  D3 E = one / dsqrt(one - h * h);
  D3 Bh = chain(h, arc_factor_deriv(h.v), arc_factor_deriv2(h.v));
  D3 Jzs = t * (E * (gg * dTds));
  D3 Jzq = t * (E * (gg * dTdq) + 0.5f * (K * ((d * d) * Bh)));
  D3 Jzt = l;
  // the state: y + dx T, z + t l, s2
  float g = pb[0] * (dx * T.d0) + pb[1] * (t * l.d0) + pb[2] * s2.d0;
  // Jbar at the entries: rows 0..2, columns 2..4
  float Cf[5][5], Gf[5][5];
  unpack(Cp, Cf);
  unpack(G, Gf);
  float M[5][3];
  for (int b = 0; b < 3; ++b) {
    int l2 = b + 2;
    M[0][b] = Cf[0][l2] + J.ys * Cf[2][l2] + J.yq * Cf[4][l2];
    M[1][b] = Cf[1][l2] + J.zs * Cf[2][l2] + J.zt * Cf[3][l2] + J.zq * Cf[4][l2];
    M[2][b] = Cf[2][l2] + J.sq * Cf[4][l2];
    M[3][b] = Cf[3][l2];
    M[4][b] = Cf[4][l2];
  }
  float Jb[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      float acc = 0.f;
      for (int c = 0; c < 5; ++c) acc += Gf[a][c] * M[c][b];
      Jb[a][b] = 2.0f * acc;
    }
  float gj = Jb[0][0] * Jys.d0 + Jb[0][2] * Jyq.d0 + Jb[1][0] * Jzs.d0 + Jb[1][1] * Jzt.d0 +
             Jb[1][2] * Jzq.d0 - Jb[2][2] * dx;
  return g + gj;
}

TPC_HD bool step_active(int rj, int pass) { return !(rj != 0 && rj < pass); }

// Reverse sweep of one saved refit: writes the adjoints of the calibrated
// coordinates gyc[at(k)], gzc[at(k)] of L = gT * chi2(pass 3). kRot as for
// refit_track_in.
template <bool kRot, bool kField>
TPC_HD void refit_backward_in(const Geo& g, const RefitCfg& p, const TrackIn& in, const Lay& ly,
                              int n, const uint8_t* rej, const float* ckpt, float gT, float* gyc,
                              float* gzc, const Vertex vx = Vertex{NAN, 0.0f, nullptr}) {
  for (int k = 0; k < n; ++k) {
    gyc[ly.at(k)] = 0.0f;
    gzc[ly.at(k)] = 0.0f;
  }
  auto xof = [&](int i) { return g.rx[in.meta[ly.at(i)] & 0xffu]; };
  auto idx_of = [&](int pass, int k) { return pass == 2 ? k : n - 1 - k; };
  // x and frame of the state at the end of each pass (0: the seed's)
  float xend[4];
  int fend[4];
  xend[0] = xof(n - 1);
  fend[0] = frame_of(in.meta[ly.at(n - 1)]);
  for (int pass = 1; pass <= 3; ++pass) {
    xend[pass] = xend[pass - 1];
    fend[pass] = fend[pass - 1];
    for (int k = n - 1; k >= 0; --k) {
      int i = idx_of(pass, k);
      if (step_active(rej[ly.at(i)], pass)) {
        xend[pass] = xof(i);
        fend[pass] = frame_of(in.meta[ly.at(i)]);
        break;
      }
    }
  }
  float pb[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  float G[15];
  for (int i = 0; i < 15; ++i) G[i] = 0.0f;
  // the vertex step, when the forward applied it: its update and transport
  // reversed, which gives the adjoints of pass 3's final state
  if (!kField && !(vx.zv != vx.zv) && vx.ck && vx.ck[21] != 0.0f) {
    float pr[5], Cr[15];
    for (int j = 0; j < 5; ++j) pr[j] = vx.ck[j];
    for (int j = 0; j < 15; ++j) Cr[j] = vx.ck[5 + j];
    float xs = vx.ck[20];
    float pp[5], xx = xs;
    for (int j = 0; j < 5; ++j) pp[j] = pr[j];
    Jac J;
    transport(p.kB, 2.0f, pp, xx, 0.0f, J);
    float Cp[15];
    for (int j = 0; j < 15; ++j) Cp[j] = Cr[j];
    transport_cov(J, Cp);
    Innov iv = innovation(pp, Cp, 0.0f, vx.zv, vx.var, vx.var);
    float mb[2];
    update_adjoint(Cp, iv, gT, pb, G, mb);
    transport_adjoint(p.kB, 0.0f - xs, pr, Cr, J, pb, G);
  }
  for (int pass = 3; pass >= 1; --pass) {
    float cbar = pass == 3 ? gT : 0.0f;
    // previous active step (in processing order) at or before k, or -1
    auto prev_active = [&](int k) {
      for (; k >= 0; --k)
        if (step_active(rej[ly.at(idx_of(pass, k))], pass)) return k;
      return -1;
    };
    int kc = prev_active(n - 1);
    if (kc < 0) continue;
    // The loads of a step are issued one step ahead of its use: the
    // checkpoint of the previous active step kp, and the cluster word of the
    // step before it (kq, active in all but rare cases: when it is not, the
    // previous active step is searched for and loaded on the spot).
    float p0[5], C0[15];
    int ic = idx_of(pass, kc);
    for (int j = 0; j < 5; ++j) p0[j] = ckpt[ly.ck(pass, kc, j)];
    for (int j = 0; j < 15; ++j) C0[j] = ckpt[ly.ck(pass, kc, 5 + j)];
    uint32_t mc = in.meta[ly.at(ic)];
    float myc = in.yc[ly.at(ic)], mzc = in.zc[ly.at(ic)];
    int rjc = rej[ly.at(ic)];
    // the cluster's gradient so far (read ahead too: an add to global memory
    // would stall the step on the load); zero before pass 3
    float gyo = pass < 3 ? gyc[ly.at(ic)] : 0.0f, gzo = pass < 3 ? gzc[ly.at(ic)] : 0.0f;
    int kq = kc - 1;
    uint32_t mq = 0;
    float myq = 0.f, mzq = 0.f;
    int rjq = 0;
    if (kq >= 0) {
      int iq = idx_of(pass, kq);
      mq = in.meta[ly.at(iq)];
      myq = in.yc[ly.at(iq)];
      mzq = in.zc[ly.at(iq)];
      rjq = rej[ly.at(iq)];
    }
    while (kc >= 0) {
      // the previous active step and its cluster word
      int kp = kq;
      uint32_t mp = mq;
      float myp = myq, mzp = mzq;
      int rjp = rjq;
      if (kq >= 0 && !step_active(rjq, pass)) {
        kp = prev_active(kq - 1);
        if (kp >= 0) {
          int ip = idx_of(pass, kp);
          mp = in.meta[ly.at(ip)];
          myp = in.yc[ly.at(ip)];
          mzp = in.zc[ly.at(ip)];
          rjp = rej[ly.at(ip)];
        }
      }
      // issue the loads of the next iteration
      float p1[5], C1[15];
      float gyo1 = 0.0f, gzo1 = 0.0f;
      if (kp >= 0) {
        for (int j = 0; j < 5; ++j) p1[j] = ckpt[ly.ck(pass, kp, j)];
        for (int j = 0; j < 15; ++j) C1[j] = ckpt[ly.ck(pass, kp, 5 + j)];
        if (pass < 3) {
          size_t a1 = ly.at(idx_of(pass, kp));
          gyo1 = gyc[a1];
          gzo1 = gzc[a1];
        }
      }
      int kq2 = kp - 1;
      uint32_t mq2 = 0;
      float myq2 = 0.f, mzq2 = 0.f;
      int rjq2 = 0;
      if (kq2 >= 0) {
        int iq = idx_of(pass, kq2);
        mq2 = in.meta[ly.at(iq)];
        myq2 = in.yc[ly.at(iq)];
        mzq2 = in.zc[ly.at(iq)];
        rjq2 = rej[ly.at(iq)];
      }
      // the current step, from its checkpoint: a frame rotation when the
      // cluster lies in another sector frame, then the transport
      float xprev = kp >= 0 ? g.rx[mp & 0xffu] : xend[pass - 1];
      int fprev = kp >= 0 ? frame_of(mp) : fend[pass - 1];
      int rot = kRot ? frame_step(fprev, frame_of(mc)) : 0;
      float xi = g.rx[mc & 0xffu];
      float pr[5], Cr[15];
      for (int j = 0; j < 5; ++j) pr[j] = p0[j];
      for (int j = 0; j < 15; ++j) Cr[j] = C0[j];
      float xs = xprev;
      if (kRot && rot != 0) rotate_frame(p.kB, 2.0f, p.rot_c[rot], p.rot_s[rot], pr, Cr, xs);
      float pp[5];
      for (int j = 0; j < 5; ++j) pp[j] = pr[j];
      float xx = xs;
      Jac J;
      // the field: the helix of the local Bz plus the difference of the two
      // Runge-Kutta integrations (propagate_field)
      float kBs = p.kB, fca = 1.0f, fsa = 0.0f, Bs[3] = {0.f, 0.f, 0.f};
      int ff = 0;
      if (kField) {
        ff = frame_of(mc);
        fca = p.frame_c[ff];
        fsa = p.frame_s[ff];
        field_at(p, xs * fca - pr[0] * fsa, xs * fsa + pr[0] * fca, pr[1], Bs);
        kBs = 2.99792458e-3f * Bs[2];
      }
      transport(kBs, 2.0f, pp, xx, xi, J);
      Rk4Tape tfull, tunif;  // (used with kField only)
      if (kField) {
        float full[5], unif[5];
        rk4_field_fwd(p, pr, xs, xi, fca, fsa, false, Bs[2], tfull, full);
        rk4_field_fwd(p, pr, xs, xi, fca, fsa, true, Bs[2], tunif, unif);
        for (int k = 0; k < 5; ++k) pp[k] = pp[k] + (full[k] - unif[k]);
      }
      float Cp[15];
      for (int j = 0; j < 15; ++j) Cp[j] = Cr[j];
      transport_cov(J, Cp);
      if (rjc != pass) {
        float v = cl_var(p, mc);
        Innov iv = innovation(pp, Cp, myc, mzc, v, v);
        float mb[2];
        update_adjoint(Cp, iv, cbar, pb, G, mb);
        gyc[ly.at(ic)] = gyo + mb[0];
        gzc[ly.at(ic)] = gzo + mb[1];
      }
      float xb = 0.0f;
      if (kRot && rot != 0) xb = transport_x_adjoint(kBs, xi - xs, pr, pp, Cr, J, pb, G);
      float fb[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
      float kbb = 0.0f, bzb = 0.0f;
      if (kField) {
        // the Runge-Kutta difference and the local Bz's dependence on (y, z)
        float a_full[5], a_unif[5], bz_full = 0.0f;
        rk4_field_rev(p, pr, xs, xi, fca, fsa, false, Bs[2], tfull, pb, a_full, bz_full);
        rk4_field_rev(p, pr, xs, xi, fca, fsa, true, Bs[2], tunif, pb, a_unif, bzb);
        for (int k = 0; k < 5; ++k) fb[k] = a_full[k] - a_unif[k];
        kbb = transport_kb_adjoint(kBs, xi - xs, pr, Cr, J, pb, G);
      }
      transport_adjoint(kBs, xi - xs, pr, Cr, J, pb, G);
      if (kField) {
        float gB[3][3];
        float X = xs * fca - pr[0] * fsa, Y = xs * fsa + pr[0] * fca;
        field_grad(p, X, Y, pr[1], gB);
        float dbz_dy = -(gB[2][0] * fsa) + gB[2][1] * fca, dbz_dz = gB[2][2];
        float w = kbb * 2.99792458e-3f - bzb;  // through kB of the helix, minus the uniform run
        for (int k = 0; k < 5; ++k) pb[k] += fb[k];
        pb[0] += w * dbz_dy;
        pb[1] += w * dbz_dz;
      }
      if (kRot && rot != 0) rotate_adjoint(p.kB, p.rot_c[rot], p.rot_s[rot], p0, C0, xb, pb, G);
      kc = kp;
      if (kp >= 0) {
        ic = idx_of(pass, kp);
        for (int j = 0; j < 5; ++j) p0[j] = p1[j];
        for (int j = 0; j < 15; ++j) C0[j] = C1[j];
        mc = mp;
        myc = myp;
        mzc = mzp;
        rjc = rjp;
        gyo = gyo1;
        gzo = gzo1;
        kq = kq2;
        mq = mq2;
        myq = myq2;
        mzq = mzq2;
        rjq = rjq2;
      }
    }
    if (pass > 1)
      for (int j = 0; j < 15; ++j) G[j] = G[j] * p.refit_inflate;
  }
}

template <bool kField = false>
TPC_HD void refit_backward_track(const Geo& g, const RefitCfg& p, const TrackIn& in, const Lay& ly,
                                 int n, const uint8_t* rej, const float* ckpt, float gT,
                                 float* gyc, float* gzc, bool multi,
                                 const Vertex vx = Vertex{NAN, 0.0f, nullptr}) {
  if (multi)
    refit_backward_in<true, kField>(g, p, in, ly, n, rej, ckpt, gT, gyc, gzc, vx);
  else
    refit_backward_in<false, kField>(g, p, in, ly, n, rej, ckpt, gT, gyc, gzc, vx);
}

}  // namespace tpc
