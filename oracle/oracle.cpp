// CPU oracle for the TPC track-finding and refit hot path.
//
// TEST INFRASTRUCTURE ONLY: this file is compiled into oracle/liborc.so, which
// only the tests, the smoke check and the CPU-baseline leg of the benchmark
// load. It shares no source with the CUDA library.
//
// It is deliberately plain: brute-force loops over the clusters of a pad row,
// full 5x5 matrices, one track at a time, in the order the method states.
// Section references are to arXiv:1811.11481. Three arithmetic types
// instantiate the same templates:
//   double - the FP64 reference for continuous outputs;
//   float  - the FP32 mirror: every decision (windows, argmins, chi2 cuts) is
//            taken in single precision, one IEEE rounding per written
//            operation, so the discrete outputs of an FP32 implementation of
//            the same formulas can be compared exactly;
//   Var    - a reverse-mode tape over double that differentiates the FP64
//            refit for the gradient reference (no hand-derived adjoint here).
// In FP32 the only inverse sine (arc length of a helix chord) is evaluated
// with the half-angle identity asin(h) = 2 asin(h / sqrt(2 (1 + sqrt(1-h^2))))
// and the Maclaurin series of asin(h)/h: a fixed sequence of IEEE operations.
//
// Parity unpinned: the cellular-automaton cut values (neighbour windows, the
// pick-up cut, the miss limit) are readings of Sec. 2 and Sec. 4, which give no
// numbers; the tests pin the arithmetic and the invariants, not those values.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <omp.h>
#include <type_traits>
#include <vector>

namespace {

// ------------------------------------------------------------------ tape AD
struct Tape {
  std::vector<int> pa, pb;
  std::vector<double> da, db;
  std::vector<double> adj;
  void clear() { pa.clear(); pb.clear(); da.clear(); db.clear(); adj.clear(); }
  int push(int a, double ga, int b, double gb) {
    pa.push_back(a); da.push_back(ga); pb.push_back(b); db.push_back(gb);
    return (int)pa.size() - 1;
  }
  void backward(int root, double seed) {
    adj.assign(pa.size(), 0.0);
    if (root < 0) return;
    adj[root] = seed;
    for (int i = root; i >= 0; --i) {
      double g = adj[i];
      if (g == 0.0) continue;
      if (pa[i] >= 0) adj[pa[i]] += g * da[i];
      if (pb[i] >= 0) adj[pb[i]] += g * db[i];
    }
  }
};
// one tape per thread: tracks are differentiated independently
thread_local Tape g_tape;

struct Var {
  double v;
  int id;
  Var() : v(0.0), id(-1) {}
  Var(double x) : v(x), id(-1) {}
  static Var leaf(double x) { Var r(x); r.id = g_tape.push(-1, 0.0, -1, 0.0); return r; }
};
inline Var mk(double v, int a, double ga, int b, double gb) {
  Var r(v);
  if (a >= 0 || b >= 0) r.id = g_tape.push(a, ga, b, gb);
  return r;
}
inline Var operator+(Var a, Var b) { return mk(a.v + b.v, a.id, 1.0, b.id, 1.0); }
inline Var operator-(Var a, Var b) { return mk(a.v - b.v, a.id, 1.0, b.id, -1.0); }
inline Var operator-(Var a) { return mk(-a.v, a.id, -1.0, -1, 0.0); }
inline Var operator*(Var a, Var b) { return mk(a.v * b.v, a.id, b.v, b.id, a.v); }
inline Var operator/(Var a, Var b) {
  double q = a.v / b.v;
  return mk(q, a.id, 1.0 / b.v, b.id, -q / b.v);
}
inline bool operator<(Var a, Var b) { return a.v < b.v; }
inline bool operator>(Var a, Var b) { return a.v > b.v; }
inline bool operator<=(Var a, Var b) { return a.v <= b.v; }
inline bool operator>=(Var a, Var b) { return a.v >= b.v; }
inline bool operator==(Var a, Var b) { return a.v == b.v; }

inline double val(double x) { return x; }
inline double val(float x) { return x; }
inline double val(Var x) { return x.v; }

inline float sqrt_(float x) { return std::sqrt(x); }
inline double sqrt_(double x) { return std::sqrt(x); }
inline Var sqrt_(Var a) {
  double s = std::sqrt(a.v);
  return mk(s, a.id, 0.5 / s, -1, 0.0);
}
inline float abs_(float x) { return std::fabs(x); }
inline double abs_(double x) { return std::fabs(x); }
inline Var abs_(Var a) { return a.v < 0 ? -a : a; }
inline Var asin_(Var a) {
  return mk(std::asin(a.v), a.id, 1.0 / std::sqrt(1.0 - a.v * a.v), -1, 0.0);
}

// Wide type: float64 timestamps stay float64 in the FP32 mirror (Sec. 4).
template <class R> struct WideT { using T = double; };
template <> struct WideT<Var> { using T = Var; };
template <class R> using W = typename WideT<R>::T;
template <class R> R narrow(W<R> x);
template <> float narrow<float>(double x) { return (float)x; }
template <> double narrow<double>(double x) { return x; }
template <> Var narrow<Var>(Var x) { return x; }

// A(h) = asin(h)/h and B(h) = A'(h) = (1/sqrt(1-h^2) - A(h))/h.
inline float seriesA_f(float h2) {
  float p = 35.0f / 1152.0f;
  p = 5.0f / 112.0f + h2 * p;
  p = 3.0f / 40.0f + h2 * p;
  p = 1.0f / 6.0f + h2 * p;
  p = 1.0f + h2 * p;
  return p;
}
inline float A_of(float h) {
  if (std::fabs(h) < 0.125f) return seriesA_f(h * h);
  if (!(std::fabs(h) <= 1.0f)) return NAN;
  float hh = h, m = 1.0f;
  while (std::fabs(hh) >= 0.125f) {
    float c = std::sqrt(1.0f - hh * hh);
    hh = hh / std::sqrt(2.0f * (1.0f + c));
    m = m * 2.0f;
  }
  return ((m * hh) * seriesA_f(hh * hh)) / h;
}
inline float B_of(float h) {
  if (std::fabs(h) < 0.125f) {
    float h2 = h * h;
    float c = 315.0f / 1408.0f;
    c = 35.0f / 144.0f + h2 * c;
    c = 15.0f / 56.0f + h2 * c;
    c = 3.0f / 10.0f + h2 * c;
    c = 1.0f / 3.0f + h2 * c;
    return h * c;
  }
  float e = 1.0f / std::sqrt(1.0f - h * h);
  return (e - A_of(h)) / h;
}
// FP64: Maclaurin coefficients e_n of (1-h^2)^(-1/2) from their recurrence
// e_{n+1} = e_n (2n+1)/(2n+2); A has e_n/(2n+1), B has e_{n+1}(2n+2)/(2n+3).
template <class T> T seriesA64(T h) {
  T h2 = h * h, s = T(0.0), hp = T(1.0);
  double e = 1.0;
  for (int n = 0; n < 8; ++n) {
    s = s + (e / (2.0 * n + 1.0)) * hp;
    e = e * (2.0 * n + 1.0) / (2.0 * n + 2.0);
    hp = hp * h2;
  }
  return s;
}
template <class T> T seriesB64(T h) {
  T h2 = h * h, s = T(0.0), hp = h;
  double e = 0.5;
  for (int n = 0; n < 12; ++n) {
    s = s + (e * (2.0 * n + 2.0) / (2.0 * n + 3.0)) * hp;
    e = e * (2.0 * n + 3.0) / (2.0 * n + 4.0);
    hp = hp * h2;
  }
  return s;
}
inline double A_of(double h) {
  if (std::fabs(h) < 1e-2) return seriesA64(h);
  return std::asin(h) / h;
}
inline double B_of(double h) {
  if (std::fabs(h) < 0.05) return seriesB64(h);
  double E = 1.0 / std::sqrt(1.0 - h * h);
  return (E - std::asin(h) / h) / h;
}
inline Var A_of(Var h) {
  if (std::fabs(h.v) < 1e-2) return seriesA64(h);
  return asin_(h) / h;
}
inline Var B_of(Var h) {
  if (std::fabs(h.v) < 0.05) return seriesB64(h);
  Var E = Var(1.0) / sqrt_(Var(1.0) - h * h);
  return (E - asin_(h) / h) / h;
}


}  // namespace

// ------------------------------------------------------------ C interface
extern "C" {

struct OrcGeom {
  const float* row_x;
  int32_t n_rows;
  float tan_half;
  float drift_length;
  float bz;
  const float* pad_width;   // [n_rows] pad pitch (cm), or NULL
  const float* pad_center;  // [n_rows] pad position of y = 0, or NULL
  const float* field;       // [3][10] (Bx, By, Bz) polynomial coefficients, or NULL
};

struct OrcParams {
  float sigma;            // cluster position error (cm)
  float shared_scale;     // error scale for clusters flagged shared
  float nb_wy, nb_wz;     // neighbour windows (cm)
  float nb_teta;          // sinh(eta_max): z slope of the window
  float nb_ty;            // tan(phi_max): y slope of the window
  float nb_dmax;          // max squared straight-line deviation (cm^2)
  float chi2_pick;        // pick-up cut on the normalised distance
  int32_t max_miss;       // consecutive missed rows that end following
  int32_t max_gap;        // largest row gap inside an emitted track
  int32_t min_track_hits; // minimum hits of an emitted track
  float s_max;            // |sin(phi)| limit of the propagation
  float inward_cov_scale; // covariance scale at the start of the inward pass
  float c0t[5];           // tracklet seed covariance diagonal
  float c0r[5];           // refit covariance diagonal (start of each pass)
  float chi2_out;         // refit outlier cut
  int32_t min_acc_reject; // accepted clusters before rejection starts
  float refit_inflate;    // passes 2 and 3 start from the previous pass's
                          // final covariance times this factor
  int32_t seed_max_hits;  // chain hits used by the seed fit (Sec. 2: 4 to 10)
  float chi2_merge;       // segment-merging cut on the 5-parameter chi2
  float split_scale;      // error scales of the other special clusters
  float single_row_scale;
  float single_time_scale;
  float edge_scale;
};

struct OrcCalib {
  double vdrift;          // cm/us
  double t0;              // us
  double tf_start;        // us
  const float* spline;    // [36][2][8][8][8] or NULL
  float spl_x0, spl_dx;   // u = (x - spl_x0) / spl_dx
};

struct OrcClusters {
  int64_t n;
  int32_t mode;           // 0: z given (single events), 1: t given (time frame)
  int32_t n_events;
  const float* y;
  const float* z;
  const double* t;
  const uint8_t* row;
  const uint8_t* sector;
  const uint8_t* flags;
  const uint32_t* event;
  int32_t pads;           // 1: y holds native pad positions
};

}  // extern "C"

namespace {

constexpr double kCLight = 2.99792458e-3;
constexpr int kNS = 36;
constexpr int kSpl = 8;

struct Ctx {
  OrcGeom g;
  OrcParams p;
  OrcCalib c;
  OrcClusters cl;
  std::vector<float> rowx;
  std::vector<float> padw, padc;  // pad pitch and centre per row
  std::vector<double> field;      // [3][10] field coefficients (empty: uniform bz)
  std::vector<float> ynat;        // y (cm) of native pad positions
  std::vector<float> spline;
  bool spline_active = false;
  std::vector<float> zs32;
  std::vector<double> zs64;
  std::vector<std::vector<int64_t>> rows;  // (event, sector, row) -> clusters
  bool joseph = false;  // the refit updates its covariance in the Joseph form
  const std::vector<int64_t>& rowlist(int64_t ev, int sec, int r) const {
    return rows[((size_t)ev * kNS + sec) * g.n_rows + r];
  }
};

// Position error of a cluster in the refit (Sec. 3: special clusters get
// larger errors): sigma times the scale of each flag bit it carries, in bit
// order (split, single row, single time, edge, shared).
template <class R> R cluster_error(const Ctx& c, uint8_t flags) {
  const float sc[5] = {c.p.split_scale, c.p.single_row_scale, c.p.single_time_scale,
                       c.p.edge_scale, c.p.shared_scale};
  R e = R(c.p.sigma);
  for (int b = 0; b < 5; ++b)
    if (flags & (1u << b)) e = e * R(sc[b]);
  return e;
}

template <class R> R kB_of(const Ctx& c) { return R(kCLight) * R(c.g.bz); }
template <> float kB_of<float>(const Ctx& c) { return (float)kCLight * c.g.bz; }

// Seeding coordinate (Sec. 4): the cluster time scaled linearly to z with the
// time-frame start as reference; tracking then assumes an arbitrarily long TPC.
template <class R> R seed_z(const Ctx& c, int64_t i) {
  if (c.cl.mode == 0) return R(c.cl.z[i]);
  double sg = c.cl.sector[i] < 18 ? 1.0 : -1.0;
  double zeta = c.c.vdrift * ((c.cl.t[i] - c.c.t0) - c.c.tf_start);
  return (R)(sg * ((double)c.g.drift_length - zeta));
}

// ------------------------------------------------- distortion spline (Sec. 5.2)
// Per-sector tensor-product uniform cubic B-spline with 8 control points per
// axis (5 uniform intervals on [0,1]) for the space-point correction.
template <class R> void bspline_basis(R f, R b[4]) {
  R g = R(1) - f;
  R f2 = f * f;
  R f3 = f2 * f;
  b[0] = ((g * g) * g) / R(6);
  b[1] = ((R(3) * f3 - R(6) * f2) + R(4)) / R(6);
  b[2] = (((R(-3) * f3 + R(3) * f2) + R(3) * f) + R(1)) / R(6);
  b[3] = f3 / R(6);
}
template <class R> R clamp01(R v) { return v < R(0) ? R(0) : (v > R(1) ? R(1) : v); }
template <class R> void split_arg(R u, int& i, R& f) {
  R t = u * R(kSpl - 3);
  int k = (int)val(t);
  if (k > kSpl - 4) k = kSpl - 4;
  if (k < 0) k = 0;
  i = k;
  f = t - R((double)k);
}

// Spline coefficients become tape leaves (created on first use) when the Var
// instantiation needs their gradient.
struct CoefLeaves {
  std::map<int, Var> m;
  Var get(int idx, float v) {
    auto it = m.find(idx);
    if (it != m.end()) return it->second;
    Var l = Var::leaf(v);
    m[idx] = l;
    return l;
  }
};
template <class R> R coef_at(const Ctx& c, int idx, CoefLeaves*) { return R(c.spline[idx]); }
template <> Var coef_at<Var>(const Ctx& c, int idx, CoefLeaves* lv) {
  return lv ? lv->get(idx, c.spline[idx]) : Var(c.spline[idx]);
}

template <class R>
void spline_eval(const Ctx& c, int sector, R x, R y, R az, R out[2], CoefLeaves* lv) {
  R u = clamp01<R>((x - R(c.c.spl_x0)) / R(c.c.spl_dx));
  R v = clamp01<R>((y / x + R(c.g.tan_half)) / (R(2) * R(c.g.tan_half)));
  R w = clamp01<R>(az / R(c.g.drift_length));
  int iu, iv, iw;
  R fu, fv, fw;
  split_arg(u, iu, fu);
  split_arg(v, iv, fv);
  split_arg(w, iw, fw);
  R bu[4], bv[4], bw[4];
  bspline_basis(fu, bu);
  bspline_basis(fv, bv);
  bspline_basis(fw, bw);
  for (int comp = 0; comp < 2; ++comp) {
    R acc = R(0);
    for (int cc = 0; cc < 4; ++cc)
      for (int bb = 0; bb < 4; ++bb) {
        R wb = bw[cc] * bv[bb];
        for (int aa = 0; aa < 4; ++aa) {
          int idx = (((sector * 2 + comp) * kSpl + (iw + cc)) * kSpl + (iv + bb)) * kSpl + (iu + aa);
          acc = acc + (wb * bu[aa]) * coef_at<R>(c, idx, lv);
        }
      }
    out[comp] = acc;
  }
}

// Calibrated position of cluster i once a collision time 'that' is assigned
// (Sec. 4: conversion to absolute z, then the space-point correction).
template <class R> struct CalIn {
  W<R> vdrift, t0, t;
  R y, z;
};
template <class R> CalIn<R> cal_in(const Ctx& c, int64_t i) {
  CalIn<R> a;
  a.vdrift = W<R>(c.c.vdrift);
  a.t0 = W<R>(c.c.t0);
  a.t = W<R>(c.cl.mode == 1 ? c.cl.t[i] : 0.0);
  a.y = R(c.cl.y[i]);
  a.z = R(c.cl.mode == 0 ? c.cl.z[i] : 0.0f);
  return a;
}
template <class R>
void calibrate(const Ctx& c, int64_t i, double that, const CalIn<R>& a, R& yc, R& zc,
               CoefLeaves* lv) {
  int sec = c.cl.sector[i];
  R zabs;
  if (c.cl.mode == 0) {
    zabs = a.z;
  } else {
    W<R> sg = W<R>(sec < 18 ? 1.0 : -1.0);
    W<R> zeta = a.vdrift * ((a.t - a.t0) - W<R>(that));
    zabs = narrow<R>(sg * (W<R>((double)c.g.drift_length) - zeta));
  }
  // an all-zero spline adds exactly zero, but its coefficients still have a
  // gradient: the differentiated (Var) evaluation always includes it
  if (c.spline_active || std::is_same<R, Var>::value) {
    R d[2];
    R x = R(c.rowx[c.cl.row[i]]);
    spline_eval<R>(c, sec, x, a.y, abs_(zabs), d, lv);
    yc = a.y + d[0];
    zc = zabs + d[1];
  } else {
    yc = a.y;
    zc = zabs;
  }
}

// ---------------------------------------------------- track model (Sec. 2-3)
// State at local x: (y, z, s = sin(phi), t = tan(lambda), q = q/pT); helix in
// a uniform field Bz, kappa = kB q, d s / d x = -kappa.
template <class R> struct Trk {
  R p[5];
  R C[5][5];
  R x;
};
template <class R> void set_diag(Trk<R>& st, const float* d) {
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) st.C[i][j] = R(0);
  for (int i = 0; i < 5; ++i) st.C[i][i] = R(d[i]);
}

// C' = J C J^T, lower triangle with index-ascending sums, mirrored.
template <class R> void cov_transform(const R J[5][5], R C[5][5]) {
  R Tm[5][5];
  for (int i = 0; i < 5; ++i)
    for (int l2 = 0; l2 < 5; ++l2) {
      R acc = R(0);
      for (int k = 0; k < 5; ++k) acc = acc + J[i][k] * C[k][l2];
      Tm[i][l2] = acc;
    }
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j <= i; ++j) {
      R acc = R(0);
      for (int l2 = 0; l2 < 5; ++l2) acc = acc + Tm[i][l2] * J[j][l2];
      C[i][j] = acc;
      C[j][i] = acc;
    }
}

// Exact helix transport to the plane x2 and its analytic Jacobian.
template <class R>
bool propagate(const Ctx& c, Trk<R>& st, R x2, R* Jout = nullptr, const R* kB_local = nullptr) {
  const R kB = kB_local ? *kB_local : kB_of<R>(c);
  R dx = x2 - st.x;
  R y = st.p[0], z = st.p[1], s = st.p[2], t = st.p[3], q = st.p[4];
  R kap = kB * q;
  R s2 = s - kap * dx;
  if (!(abs_(s2) < R(c.p.s_max))) return false;
  R c1 = sqrt_(R(1) - s * s);
  R c2 = sqrt_(R(1) - s2 * s2);
  R N = s + s2;
  R D = c1 + c2;
  R T = N / D;
  R dy = dx * T;
  R opt = R(1) + T * T;
  R d = dx * sqrt_(opt);
  R h = (kap * d) * R(0.5);
  R A = A_of(h);
  R l = d * A;
  // Jacobian entries that differ from the identity
  R dDds = -(s / c1) - (s2 / c2);
  R kdx = kB * dx;
  R dDdq = kdx * (s2 / c2);
  R dTds = (R(2) - T * dDds) / D;
  R dTdq = (-kdx - T * dDdq) / D;
  R Jys = dx * dTds;
  R Jyq = dx * dTdq;
  R g = (d * T) / opt;
  R dds = g * dTds;
  R ddq = g * dTdq;
  R E = R(1) / sqrt_(R(1) - h * h);
  R Bh = B_of(h);
  R Jzs = t * (E * dds);
  R Jzq = t * (E * ddq + (kB * ((d * d) * Bh)) * R(0.5));
  R Jzt = l;
  R Jsq = -kdx;
  R J[5][5];
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) J[i][j] = R(i == j ? 1 : 0);
  J[0][2] = Jys; J[0][4] = Jyq;
  J[1][2] = Jzs; J[1][3] = Jzt; J[1][4] = Jzq;
  J[2][4] = Jsq;
  if (Jout)
    for (int i = 0; i < 5; ++i)
      for (int j = 0; j < 5; ++j) Jout[i * 5 + j] = J[i][j];
  cov_transform<R>(J, st.C);
  st.p[0] = y + dy;
  st.p[1] = z + t * l;
  st.p[2] = s2;
  st.x = x2;
  return true;
}

// ------------------------------------------------ the full field (Sec. 3)
// The final fit takes the Bx and By components of the field into account and
// a three-dimensional polynomial approximation of the field. Here the field
// is given as quadratic polynomials of (Bx, By, Bz) in the global
// coordinates in metres (monomials 1, X, Y, Z, X^2, XY, XZ, Y^2, YZ, Z^2).
template <class R> void field_at(const Ctx& c, R X, R Y, R Z, R B[3]) {
  R x = X * R(0.01), y = Y * R(0.01), z = Z * R(0.01);
  const R m[10] = {R(1), x, y, z, x * x, x * y, x * z, y * y, y * z, z * z};
  for (int k = 0; k < 3; ++k) {
    R acc = R(0);
    for (int i = 0; i < 10; ++i) acc = acc + R(c.field[k * 10 + i]) * m[i];
    B[k] = acc;
  }
}

// Transport in the full field from the state's x to x2 in the frame rotated
// by alpha. The equations of motion of the direction u (unit vector) with x
// as the variable, dy/dx = u_y / u_x, dz/dx = u_z / u_x,
// du/dx = k (q/p) (u x B) / u_x (q/p conserved, q/pT = (q/p) / |u_T|), are
// integrated by fourth-order Runge-Kutta in steps of at most 0.5 cm twice:
// in the full field and in the uniform field of the local Bz at the start
// point. The state is the exact helix of that uniform field plus the
// difference of the two integrations, so that the steps' truncation and
// rounding errors largely cancel and a uniform field gives the helix
// exactly. The covariance is transported with the helix Jacobian (a
// reading: the paper does not give the Jacobian used). Fails where u_x
// would not stay positive or |sin(phi)| reaches s_max.
template <class R>
bool rk4_field(const Ctx& c, const Trk<R>& st, R x2, double alpha, bool uniform, R bz,
               R out[5]) {
  const R ca = R(std::cos(alpha)), sa = R(std::sin(alpha));
  R s = st.p[2], t = st.p[3], q = st.p[4];
  R cl = R(1) / sqrt_(R(1) + t * t);
  R cf = sqrt_(R(1) - s * s);
  R v[5] = {R(0), R(0), cf * cl, s * cl, t * cl};  // y, z as offsets from the start
  R kq = R(kCLight) * (q * cl);
  R dx = x2 - st.x;
  int ns = (int)std::ceil(std::fabs(val(dx)) / 0.5);
  if (ns < 1) ns = 1;
  R h = dx / R((double)ns);
  R x = st.x;
  auto deriv = [&](R xx, const R w[5], R d[5]) {
    if (!(w[2] > R(0))) return false;
    R b0 = R(0), b1 = R(0), b2 = bz;
    if (!uniform) {
      R B[3];
      R yy = st.p[0] + w[0];
      field_at<R>(c, xx * ca - yy * sa, xx * sa + yy * ca, st.p[1] + w[1], B);
      b0 = B[0] * ca + B[1] * sa;
      b1 = -(B[0] * sa) + B[1] * ca;
      b2 = B[2];
    }
    R iu = R(1) / w[2];
    R f = kq * iu;
    d[0] = w[3] * iu;
    d[1] = w[4] * iu;
    d[2] = f * (w[3] * b2 - w[4] * b1);
    d[3] = f * (w[4] * b0 - w[2] * b2);
    d[4] = f * (w[2] * b1 - w[3] * b0);
    return true;
  };
  for (int i = 0; i < ns; ++i) {
    R k1[5], k2[5], k3[5], k4[5], w[5];
    if (!deriv(x, v, k1)) return false;
    for (int j = 0; j < 5; ++j) w[j] = v[j] + (h * R(0.5)) * k1[j];
    if (!deriv(x + h * R(0.5), w, k2)) return false;
    for (int j = 0; j < 5; ++j) w[j] = v[j] + (h * R(0.5)) * k2[j];
    if (!deriv(x + h * R(0.5), w, k3)) return false;
    for (int j = 0; j < 5; ++j) w[j] = v[j] + h * k3[j];
    if (!deriv(x + h, w, k4)) return false;
    for (int j = 0; j < 5; ++j)
      v[j] = v[j] + (h / R(6)) * (k1[j] + R(2) * k2[j] + R(2) * k3[j] + k4[j]);
    x = (i == ns - 1) ? x2 : x + h;
  }
  R un = sqrt_(v[2] * v[2] + v[3] * v[3] + v[4] * v[4]);
  R ux = v[2] / un, uy = v[3] / un, uz = v[4] / un;
  R rho = sqrt_(ux * ux + uy * uy);
  if (!(ux > R(0))) return false;
  out[0] = v[0];
  out[1] = v[1];
  out[2] = uy / rho;
  out[3] = uz / rho;
  out[4] = (q * cl) / rho;
  return true;
}

template <class R>
bool propagate_field(const Ctx& c, Trk<R>& st, R x2, double alpha) {
  const R ca = R(std::cos(alpha)), sa = R(std::sin(alpha));
  R Bs[3];
  field_at<R>(c, st.x * ca - st.p[0] * sa, st.x * sa + st.p[0] * ca, st.p[1], Bs);
  R kBl = R(kCLight) * Bs[2];
  Trk<R> hx = st;
  if (!propagate<R>(c, hx, x2, nullptr, &kBl)) return false;
  R full[5], unif[5];
  if (!rk4_field<R>(c, st, x2, alpha, false, Bs[2], full)) return false;
  if (!rk4_field<R>(c, st, x2, alpha, true, Bs[2], unif)) return false;
  R s2 = hx.p[2] + (full[2] - unif[2]);
  if (!(abs_(s2) < R(c.p.s_max))) return false;
  for (int k = 0; k < 5; ++k) st.p[k] = hx.p[k] + (full[k] - unif[k]);
  st.x = x2;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) st.C[i][j] = hx.C[i][j];
  return true;
}

// Kalman innovation for a (y, z) measurement with variances vy, vz.
template <class R> struct Innov {
  R r0, r1, W00, W01, W11, chi2;
};
template <class R> Innov<R> innovation(const Trk<R>& st, R my, R mz, R vy, R vz) {
  Innov<R> in;
  in.r0 = my - st.p[0];
  in.r1 = mz - st.p[1];
  R S00 = st.C[0][0] + vy;
  R S01 = st.C[1][0];
  R S11 = st.C[1][1] + vz;
  R det = S00 * S11 - S01 * S01;
  in.W00 = S11 / det;
  in.W01 = -(S01 / det);
  in.W11 = S00 / det;
  in.chi2 = in.r0 * (in.W00 * in.r0 + in.W01 * in.r1) + in.r1 * (in.W01 * in.r0 + in.W11 * in.r1);
  return in;
}
// p += K r, C -= K H C (short form), K = C H^T S^-1.
// Joseph form of the same update (Sec. 3 filter; numerically symmetric and
// positive): C = (I - K H) C (I - K H)^T + K V K^T with V = diag(vy, vz).
template <class R> void apply_update_joseph(Trk<R>& st, const Innov<R>& in, R vy, R vz) {
  R K[5][2];
  for (int i = 0; i < 5; ++i) {
    K[i][0] = st.C[i][0] * in.W00 + st.C[i][1] * in.W01;
    K[i][1] = st.C[i][0] * in.W01 + st.C[i][1] * in.W11;
  }
  for (int i = 0; i < 5; ++i) st.p[i] = st.p[i] + (K[i][0] * in.r0 + K[i][1] * in.r1);
  R A[5][5];  // I - K H
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) A[i][j] = R(i == j ? 1 : 0) - (j < 2 ? K[i][j] : R(0));
  R AC[5][5];
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) {
      R acc = R(0);
      for (int l = 0; l < 5; ++l) acc = acc + A[i][l] * st.C[l][j];
      AC[i][j] = acc;
    }
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j <= i; ++j) {
      R acc = R(0);
      for (int l = 0; l < 5; ++l) acc = acc + AC[i][l] * A[j][l];
      acc = acc + (K[i][0] * vy * K[j][0] + K[i][1] * vz * K[j][1]);
      st.C[i][j] = acc;
      st.C[j][i] = acc;
    }
}

template <class R> void apply_update(Trk<R>& st, const Innov<R>& in) {
  R K0[5], K1[5];
  for (int i = 0; i < 5; ++i) {
    K0[i] = st.C[i][0] * in.W00 + st.C[i][1] * in.W01;
    K1[i] = st.C[i][0] * in.W01 + st.C[i][1] * in.W11;
  }
  R HC0[5], HC1[5];
  for (int j = 0; j < 5; ++j) { HC0[j] = st.C[0][j]; HC1[j] = st.C[1][j]; }
  for (int i = 0; i < 5; ++i) st.p[i] = st.p[i] + (K0[i] * in.r0 + K1[i] * in.r1);
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j <= i; ++j) {
      R v = st.C[i][j] - (K0[i] * HC0[j] + K1[i] * HC1[j]);
      st.C[i][j] = v;
      st.C[j][i] = v;
    }
}

// Frame angle of a sector: sector k is rotated by ((k mod 18) + 1/2) * 20
// degrees about the beam axis (Sec. 2: 36 trapezoidal sectors).
inline double sector_alpha(int sec) { return ((sec % 18) + 0.5) * (M_PI / 9.0); }

// The same helix at the same point, expressed in a frame rotated by dalpha
// about the beam axis: the final fit of a track merged from several sectors
// (Sec. 2, second phase) runs in the frame of the sector of each cluster.
// Position and direction rotate; the state then refers to the plane
// x' = x cos + y sin of the new frame, and the covariance follows with the
// Jacobian of the state at that plane (a shift of y at fixed x moves the
// point off the plane, and the track is followed back to it along its
// tangent: dy'/dy = cos(phi)/cos(phi'), dz'/dy = -sin(dalpha) tan(lambda) /
// cos(phi'), dsin(phi')/dy = kappa sin(dalpha), dsin(phi')/dsin(phi) =
// cos(phi')/cos(phi)). Fails when the track would leave the new frame's
// forward half-plane or reach s_max.
template <class R> bool rotate(const Ctx& c, Trk<R>& st, double dalpha) {
  const R ca = R(std::cos(dalpha)), sa = R(std::sin(dalpha));
  R x = st.x, y = st.p[0], s = st.p[2], t = st.p[3], q = st.p[4];
  R cf = sqrt_(R(1) - s * s);
  R s2 = s * ca - cf * sa;
  R c2 = cf * ca + s * sa;
  if (!(c2 > R(0)) || !(abs_(s2) < R(c.p.s_max))) return false;
  R kap = kB_of<R>(c) * q;
  R J[5][5];
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) J[i][j] = R(i == j ? 1 : 0);
  J[0][0] = cf / c2;
  J[1][0] = -(sa * t) / c2;
  J[2][0] = kap * sa;
  J[2][2] = c2 / cf;
  cov_transform<R>(J, st.C);
  st.x = x * ca + y * sa;
  st.p[0] = -(x * sa) + y * ca;
  st.p[2] = s2;
  return true;
}

// Seed state through two points: straight line, q/pT = 0 (Sec. 2 seed fit).
template <class R>
void seed_two_points(const Ctx& c, Trk<R>& st, R x0, R y0, R z0, R x1, R y1, R z1) {
  R dx = x1 - x0, dy = y1 - y0, dz = z1 - z0;
  R dl = sqrt_(dx * dx + dy * dy);
  st.p[0] = y0;
  st.p[1] = z0;
  st.p[2] = dy / dl;
  st.p[3] = dz / dl;
  st.p[4] = R(0);
  st.x = x0;
  set_diag(st, c.p.c0t);
}

// z of the closest approach of the fitted helix to the beam line (Sec. 4).
template <class R> R dca_z(const Ctx& c, const Trk<R>& st) {
  const R kB = kB_of<R>(c);
  R x = st.x, y = st.p[0], z = st.p[1], s = st.p[2], t = st.p[3], q = st.p[4];
  R kap = kB * q;
  R cs = sqrt_(R(1) - s * s);
  if (abs_(kap) * (abs_(x) + abs_(y)) < R(1e-4)) {
    R a = x * cs + y * s;
    return z - t * a;
  }
  R cx = x + s / kap;
  R cy = y - cs / kap;
  R rc = sqrt_(cx * cx + cy * cy);
  R rad = R(1) / abs_(kap);
  R f = R(1) - rad / rc;
  R px = cx * f, py = cy * f;
  R ex = x - px, ey = y - py;
  R ch = sqrt_(ex * ex + ey * ey);
  R h = (ch * abs_(kap)) * R(0.5);
  if (h > R(1)) h = R(1);
  return z - t * (ch * A_of(h));
}

Ctx* build_ctx(const OrcGeom* g, const OrcParams* p, const OrcCalib* cal, const OrcClusters* cl) {
  Ctx* c = new Ctx();
  c->g = *g;
  c->p = *p;
  c->c = *cal;
  c->cl = *cl;
  c->rowx.assign(g->row_x, g->row_x + g->n_rows);
  c->g.row_x = c->rowx.data();
  if (g->field) c->field.assign(g->field, g->field + 30);
  // native pad positions (the paper's next step after Sec. 4: tracking in
  // native pad, row and time coordinates): y = (pad - centre) * pitch of the
  // cluster's row, in single precision; every step then reads that y
  if (cl->pads && g->pad_width && g->pad_center) {
    c->padw.assign(g->pad_width, g->pad_width + g->n_rows);
    c->padc.assign(g->pad_center, g->pad_center + g->n_rows);
    c->ynat.resize(cl->n);
    for (int64_t i = 0; i < cl->n; ++i) {
      int r = cl->row[i];
      float d = cl->y[i] - c->padc[r];
      c->ynat[i] = d * c->padw[r];
    }
    c->cl.y = c->ynat.data();
  } else {
    c->cl.pads = 0;
  }
  c->spline.assign((size_t)kNS * 2 * kSpl * kSpl * kSpl, 0.0f);
  if (cal->spline) {
    std::memcpy(c->spline.data(), cal->spline, c->spline.size() * sizeof(float));
    for (float v : c->spline) if (v != 0.0f) { c->spline_active = true; break; }
  }
  c->c.spline = c->spline.data();
  int ne = std::max(1, cl->n_events);
  c->rows.assign((size_t)ne * kNS * g->n_rows, {});
  for (int64_t i = 0; i < cl->n; ++i) {
    size_t k = ((size_t)cl->event[i] * kNS + cl->sector[i]) * g->n_rows + cl->row[i];
    c->rows[k].push_back(i);
  }
  c->zs32.resize(cl->n);
  c->zs64.resize(cl->n);
  for (int64_t i = 0; i < cl->n; ++i) {
    c->zs32[i] = seed_z<float>(*c, i);
    c->zs64[i] = seed_z<double>(*c, i);
  }
  return c;
}

template <class R> R zs_of(const Ctx& c, int64_t i);
template <> float zs_of<float>(const Ctx& c, int64_t i) { return c.zs32[i]; }
template <> double zs_of<double>(const Ctx& c, int64_t i) { return c.zs64[i]; }

// ------------------------------------------------------ decision margins
// How far a discrete decision (a window, a cut, the choice of the nearest
// candidate, the |sin(phi)| limit of the transport) lies from being taken the
// other way, for the parity of implementations that round differently (the
// FP64 instantiation records it). For a comparison of two quantities
// computed from cluster positions it is the distance by which those
// positions would have to move to reverse it -- the difference divided by the
// norm of its gradient with respect to the positions -- relative to the x of
// the pad row where the decision is taken; for the |sin(phi)| limit, the
// distance of |sin(phi)| from it. A hit's or a tracklet's margin is the
// smallest over its decisions.
struct Margin {
  double m = INFINITY;
  int64_t n = 0;  // decisions taken
  void take(double v) {
    if (v < m) m = v;
  }
};

// --------------------------------------------------- neighbour finder (Sec. 2)
// For hit h in row r: the pair (u in row r+1, d in row r-1), each inside a
// slope window around h -- in z the eta window of Sec. 4 (no vertex
// constraint), in y a direction window, so that legs of loopers that do not
// point to the vertex are linked too -- whose d lies closest to the straight
// line through h and u. Ties go to the lowest (u, d) index pair.
template <class R>
void neighbours_of(const Ctx& c, int64_t h, int32_t& up, int32_t& dn, Margin* mg = nullptr) {
  up = -1;
  dn = -1;
  int r = c.cl.row[h];
  if (r < 1 || r + 1 >= c.g.n_rows) return;
  if (mg) ++mg->n;
  const double xr = c.rowx[r];
  int ev = c.cl.event[h], sec = c.cl.sector[h];
  const auto& U = c.rowlist(ev, sec, r + 1);
  const auto& Dn = c.rowlist(ev, sec, r - 1);
  R xh = R(c.rowx[r]), xu = R(c.rowx[r + 1]), xd = R(c.rowx[r - 1]);
  R yh = R(c.cl.y[h]), zh = zs_of<R>(c, h);
  R dxu = xu - xh, dxd = xh - xd;
  R wy_u = dxu * R(c.p.nb_ty) + R(c.p.nb_wy);
  R wy_d = dxd * R(c.p.nb_ty) + R(c.p.nb_wy);
  R wz_u = dxu * R(c.p.nb_teta) + R(c.p.nb_wz);
  R wz_d = dxd * R(c.p.nb_teta) + R(c.p.nb_wz);
  R f = dxd / dxu;
  R dmax = R(c.p.nb_dmax);
  bool found = false;
  R best = R(0);
  // margins: a window |a - b| <= w moves by sqrt(2) per unit of position; the
  // deviation D = |e|^2 with e = p_d - p_h + (p_u - p_h) f has the gradient
  // norm 2 sqrt(D kf) with respect to the three points, kf = 1 + f^2 + (1+f)^2
  const double kf = 1.0 + (double)val(f) * (double)val(f) +
                    (1.0 + (double)val(f)) * (1.0 + (double)val(f));
  auto win = [&](R a, R w) {
    if (mg) mg->take(std::fabs(std::fabs((double)val(a)) - (double)val(w)) / (std::sqrt(2.0) * xr));
  };
  std::vector<double> passing;
  for (int64_t u : U) {
    R yu = R(c.cl.y[u]), zu = zs_of<R>(c, u);
    win(yu - yh, wy_u);
    if (!(abs_(yu - yh) <= wy_u)) continue;
    win(zu - zh, wz_u);
    if (!(abs_(zu - zh) <= wz_u)) continue;
    R py = yh - (yu - yh) * f;
    R pz = zh - (zu - zh) * f;
    for (int64_t d : Dn) {
      R yd = R(c.cl.y[d]), zd = zs_of<R>(c, d);
      win(yd - yh, wy_d);
      if (!(abs_(yd - yh) <= wy_d)) continue;
      win(zd - zh, wz_d);
      if (!(abs_(zd - zh) <= wz_d)) continue;
      R ey = yd - py, ez = zd - pz;
      R D = ey * ey + ez * ez;
      if (mg) {
        double Dv = (double)val(D);
        if (Dv > 0.0)
          mg->take(std::fabs(Dv - (double)val(dmax)) / (2.0 * std::sqrt(Dv * kf) * xr));
      }
      if (!(D <= dmax)) continue;
      if (mg) passing.push_back((double)val(D));
      // lists are in increasing index order, so strict '<' keeps the lowest pair
      if (!found || D < best) {
        found = true;
        best = D;
        up = (int32_t)u;
        dn = (int32_t)d;
      }
    }
  }
  // the nearest pair against each other pair inside the cut (gradient norm
  // of the difference bounded by the sum of the two)
  if (mg && found) {
    const double Db = (double)val(best);
    int same = 0;
    for (double Dp : passing) {
      if (Dp == Db && ++same == 1) continue;  // the chosen pair itself
      double g = 2.0 * std::sqrt(kf) * (std::sqrt(Dp) + std::sqrt(Db));
      mg->take(g > 0.0 ? std::fabs(Dp - Db) / (g * xr) : 0.0);
    }
  }
}

// -------------------------------------------------- tracklet constructor
struct TrackletOut {
  int32_t nh;
  double that;
  double state[5];
  double x;
  double margin;      // smallest decision margin (FP64 runs that ask for it)
  int64_t decisions;  // transports and pick-ups taken
};

// Nearest cluster of row r to the predicted position by the normalised
// distance d2 = ry^2 / (C_yy + sigma^2) + rz^2 / (C_zz + sigma^2) inside the
// pick-up cut, ties to the lowest input index; the clusters in calibrated
// coordinates for the collision time 'that' (Sec. 4).
template <class R>
int64_t pick(const Ctx& c, int ev, int sec, int r, const Trk<R>& st, double that,
             Margin* mg) {
  const auto& L = c.rowlist(ev, sec, r);
  R sig2 = R(c.p.sigma) * R(c.p.sigma);
  R cut = R(c.p.chi2_pick);
  R vy = st.C[0][0] + sig2;
  R vz = st.C[1][1] + sig2;
  const double xr = c.rowx[r];
  const double ivy = 1.0 / (double)val(vy), ivz = 1.0 / (double)val(vz);
  int64_t bj = -1;
  R bd = R(0), by = R(0), bz = R(0);
  struct Cand { double y, z, d2; };
  std::vector<Cand> inside;
  for (int64_t j : L) {
    R yc, zc;
    calibrate<R>(c, j, that, cal_in<R>(c, j), yc, zc, nullptr);
    R ry = yc - st.p[0];
    R rz = zc - st.p[1];
    R d2 = (ry * ry) / vy + (rz * rz) / vz;
    if (mg) {
      // gradient of d2 with respect to the predicted position
      double gy = 2.0 * (double)val(ry) * ivy, gz = 2.0 * (double)val(rz) * ivz;
      double g = std::sqrt(gy * gy + gz * gz);
      if (g > 0.0) mg->take(std::fabs((double)val(d2) - (double)val(cut)) / (g * xr));
    }
    if (!(d2 <= cut)) continue;
    if (mg) inside.push_back({(double)val(yc), (double)val(zc), (double)val(d2)});
    if (bj < 0 || d2 < bd) { bj = j; bd = d2; by = yc; bz = zc; }
  }
  if (mg) {
    ++mg->n;
    // the nearest candidate against each other candidate inside the cut
    const double yb = (double)val(by), zb = (double)val(bz), db = (double)val(bd);
    for (const Cand& q : inside) {
      double gy = 2.0 * (q.y - yb) * ivy, gz = 2.0 * (q.z - zb) * ivz;
      double g = std::sqrt(gy * gy + gz * gz);
      if (g > 0.0) mg->take(std::fabs(q.d2 - db) / (g * xr));
    }
  }
  return bj;
}

// The |sin(phi)| limit of the transport to x2 (Sec. 2 model: s2 = s - kB q dx).
template <class R> void transport_margin(const Ctx& c, const Trk<R>& st, R x2, Margin* mg) {
  if (!mg) return;
  R s2 = st.p[2] - (kB_of<R>(c) * st.p[4]) * (x2 - st.x);
  ++mg->n;
  mg->take(std::fabs(std::fabs((double)val(s2)) - (double)c.p.s_max));
}

// Sec. 2: follow the chain of links, fit it with the simplified Kalman filter,
// Sec. 4: closest approach -> collision time, calibrated coordinates, refit the
// seed, then follow outward and inward (Sec. 3: the inward pass also runs
// through the seed) picking up at most one cluster per row.
template <class R>
TrackletOut tracklet(const Ctx& c, const int32_t* upc, int64_t start, int32_t* hits,
                     Margin* mg = nullptr) {
  TrackletOut o;
  o.nh = -1;
  o.that = 0.0;
  for (int i = 0; i < 5; ++i) o.state[i] = 0.0;
  o.x = 0.0;
  o.margin = INFINITY;
  o.decisions = 0;
  for (int r = 0; r < c.g.n_rows; ++r) hits[r] = -1;
  std::vector<int64_t> H;
  int64_t cur = start;
  H.push_back(cur);
  // the seed is the first segment of at most seed_max_hits linked hits
  while (upc[cur] >= 0 && (int)H.size() < c.p.seed_max_hits) {
    cur = upc[cur];
    H.push_back(cur);
  }
  int ev = c.cl.event[start], sec = c.cl.sector[start];
  size_t n = H.size();
  const R sig2 = R(c.p.sigma) * R(c.p.sigma);
  auto X = [&](int64_t i) { return R(c.rowx[c.cl.row[i]]); };
  auto done = [&]() {
    if (mg) {
      o.margin = mg->m;
      o.decisions = mg->n;
    }
    return o;
  };
  // seed fit in seeding coordinates
  Trk<R> st;
  seed_two_points<R>(c, st, X(H[0]), R(c.cl.y[H[0]]), zs_of<R>(c, H[0]), X(H[n - 1]),
                     R(c.cl.y[H[n - 1]]), zs_of<R>(c, H[n - 1]));
  for (size_t k = 0; k < n; ++k) {
    transport_margin<R>(c, st, X(H[k]), mg);
    if (!propagate<R>(c, st, X(H[k]))) return done();
    Innov<R> in = innovation<R>(st, R(c.cl.y[H[k]]), zs_of<R>(c, H[k]), sig2, sig2);
    apply_update<R>(st, in);
  }
  double that = 0.0;
  if (c.cl.mode == 1) {
    R zd = dca_z<R>(c, st);
    double sg = sec < 18 ? 1.0 : -1.0;
    that = c.c.tf_start - (sg * (double)zd) / c.c.vdrift;
  }
  // once the collision time is known, the clusters in calibrated
  // coordinates (Sec. 4): absolute z from the drift time, then the
  // space-point correction
  auto cal = [&](int64_t i, R& y, R& z) { calibrate<R>(c, i, that, cal_in<R>(c, i), y, z, nullptr); };
  // seed fit in calibrated coordinates
  std::vector<R> yc(n), zc(n);
  for (size_t k = 0; k < n; ++k) cal(H[k], yc[k], zc[k]);
  seed_two_points<R>(c, st, X(H[0]), yc[0], zc[0], X(H[n - 1]), yc[n - 1], zc[n - 1]);
  for (size_t k = 0; k < n; ++k) {
    transport_margin<R>(c, st, X(H[k]), mg);
    if (!propagate<R>(c, st, X(H[k]))) return done();
    Innov<R> in = innovation<R>(st, yc[k], zc[k], sig2, sig2);
    apply_update<R>(st, in);
  }
  // outward
  Trk<R> best = st;
  int rlast = c.cl.row[H[n - 1]];
  int miss = 0;
  for (int r = rlast + 1; r < c.g.n_rows; ++r) {
    transport_margin<R>(c, st, R(c.rowx[r]), mg);
    if (!propagate<R>(c, st, R(c.rowx[r]))) break;
    int64_t j = pick<R>(c, ev, sec, r, st, that, mg);
    if (j >= 0) {
      R y, z;
      cal(j, y, z);
      apply_update<R>(st, innovation<R>(st, y, z, sig2, sig2));
      best = st;
      rlast = r;
      miss = 0;
    } else if (++miss >= c.p.max_miss) {
      break;
    }
  }
  // inward, through the seed
  st = best;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) st.C[i][j] = st.C[i][j] * R(c.p.inward_cov_scale);
  Trk<R> inner = st;
  int nh = 0;
  miss = 0;
  for (int r = rlast; r >= 0; --r) {
    transport_margin<R>(c, st, R(c.rowx[r]), mg);
    if (!propagate<R>(c, st, R(c.rowx[r]))) break;
    int64_t j = pick<R>(c, ev, sec, r, st, that, mg);
    if (j >= 0) {
      R y, z;
      cal(j, y, z);
      apply_update<R>(st, innovation<R>(st, y, z, sig2, sig2));
      hits[r] = (int32_t)j;
      ++nh;
      miss = 0;
      inner = st;
    } else if (++miss >= c.p.max_miss) {
      break;
    }
  }
  o.nh = nh;
  o.that = that;
  for (int i = 0; i < 5; ++i) o.state[i] = val(inner.p[i]);
  o.x = val(inner.x);
  return done();
}

// ------------------------------------------------------------- final refit
// Sec. 3: three iterations (inward, outward, inward) with outlier rejection
// on the predicted chi2; the seed of the first pass is a three-point circle.
struct RefitOut {
  double p[5];
  double C[15];
  double x;
  double chi2;
  int32_t ndf;
  int32_t status;  // 0 ok, 1 propagation failed, 2 no seed
};

template <class R>
bool seed_three_points(const Ctx& c, const std::vector<R>& x, const std::vector<R>& yc,
                       const std::vector<R>& zc, double out[5]) {
  size_t n = x.size();
  if (n < 3) return false;
  size_t i0 = 0, im = n / 2, i2 = n - 1;
  R ax = x[im] - x[i0], ay = yc[im] - yc[i0];
  R bx = x[i2] - x[i0], by = yc[i2] - yc[i0];
  R ex = x[i2] - x[im], ey = yc[i2] - yc[im];
  R cross = ax * by - ay * bx;
  R la = sqrt_(ax * ax + ay * ay), lb = sqrt_(bx * bx + by * by), le = sqrt_(ex * ex + ey * ey);
  R kap = (R(-2) * cross) / ((la * lb) * le);
  // no field: q/pT is not observable and is held at 0 (straight lines)
  R q = kB_of<R>(c) != R(0) ? kap / kB_of<R>(c) : R(0);
  R hs = (kap * lb) * R(0.5);
  if (!(abs_(hs) < R(1))) return false;
  R s2 = (by / lb) * sqrt_(R(1) - hs * hs) - (bx / lb) * hs;
  R arc = lb * A_of(hs);
  R t = (zc[i2] - zc[i0]) / arc;
  out[0] = val(yc[i2]);
  out[1] = val(zc[i2]);
  out[2] = val(s2);
  out[3] = val(t);
  out[4] = val(q);
  return true;
}

template <class R>
// priors (may be null): the state each pass starts from, per pass its x,
// the five parameters and the 15 covariance entries (lower triangle).
RefitOut refit_core(const Ctx& c, const std::vector<R>& x, const std::vector<R>& yc,
                    const std::vector<R>& zc, const std::vector<R>& var, const double seed[5],
                    uint8_t* rej, bool frozen, R* chi2_out,
                    const std::vector<double>* alpha = nullptr, double* priors = nullptr,
                    double zv = NAN, double vvar = 0.0) {
  RefitOut o;
  std::memset(&o, 0, sizeof(o));
  size_t n = x.size();
  Trk<R> st;
  for (int i = 0; i < 5; ++i) st.p[i] = R(seed[i]);
  st.x = x[n - 1];
  // frame of the state (clusters of a merged track lie in several sectors)
  double cur_alpha = alpha ? (*alpha)[n - 1] : 0.0;
  R chi2 = R(0);
  int ndf = 0;
  set_diag(st, c.p.c0r);
  for (int pass = 1; pass <= 3; ++pass) {
    if (pass > 1)
      for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) st.C[i][j] = st.C[i][j] * R(c.p.refit_inflate);
    if (priors) {
      double* pr = priors + (pass - 1) * 21;
      pr[0] = val(st.x);
      for (int i = 0; i < 5; ++i) pr[1 + i] = val(st.p[i]);
      int q = 6;
      for (int i = 0; i < 5; ++i)
        for (int j = 0; j <= i; ++j) pr[q++] = val(st.C[i][j]);
    }
    chi2 = R(0);
    ndf = 0;
    int nacc = 0;
    for (size_t k = 0; k < n; ++k) {
      size_t i = (pass == 2) ? k : n - 1 - k;
      if (rej[i] != 0 && rej[i] < pass) continue;
      if (alpha && (*alpha)[i] != cur_alpha) {
        if (!rotate<R>(c, st, (*alpha)[i] - cur_alpha)) {
          o.status = 1;
          *chi2_out = R(0);
          return o;
        }
        cur_alpha = (*alpha)[i];
      }
      bool moved = c.field.empty() ? propagate<R>(c, st, x[i])
                                   : propagate_field<R>(c, st, x[i], cur_alpha);
      if (!moved) {
        o.status = 1;
        *chi2_out = R(0);
        return o;
      }
      Innov<R> in = innovation<R>(st, yc[i], zc[i], var[i], var[i]);
      bool reject;
      if (frozen) {
        reject = rej[i] == pass;
      } else {
        reject = nacc >= c.p.min_acc_reject && in.chi2 > R(c.p.chi2_out);
        if (reject) rej[i] = (uint8_t)pass;
      }
      if (reject) continue;
      if (c.joseph) apply_update_joseph<R>(st, in, var[i], var[i]);
      else apply_update<R>(st, in);
      chi2 = chi2 + in.chi2;
      ndf += 2;
      ++nacc;
    }
  }
  // Vertex pseudo-measurement (a reading: a known vertex, as in a triggered
  // event, fixes the absolute z that drift velocity and t0 otherwise share
  // with every track's z0 and tan(lambda)): the state transported to the
  // beam line, x = 0, and updated with (y, z) = (0, zv), variance vvar each;
  // skipped when the transport fails.
  if (!(zv != zv) && c.field.empty()) {
    Trk<R> sv = st;
    if (propagate<R>(c, sv, R(0.0))) {
      Innov<R> in = innovation<R>(sv, R(0.0), R(zv), R(vvar), R(vvar));
      if (c.joseph) apply_update_joseph<R>(sv, in, R(vvar), R(vvar));
      else apply_update<R>(sv, in);
      chi2 = chi2 + in.chi2;
      ndf += 2;
      st = sv;
    }
  }
  for (int i = 0; i < 5; ++i) o.p[i] = val(st.p[i]);
  int k = 0;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j <= i; ++j) o.C[k++] = val(st.C[i][j]);
  o.x = val(st.x);
  o.chi2 = val(chi2);
  o.ndf = ndf;
  *chi2_out = chi2;
  return o;
}

// Frame angles of a track's clusters, or empty when they share one sector.
inline std::vector<double> track_alpha(const Ctx& c, const uint32_t* idx, size_t n) {
  std::vector<double> al;
  bool multi = false;
  for (size_t k = 1; k < n; ++k) multi = multi || c.cl.sector[idx[k]] != c.cl.sector[idx[0]];
  // the full field needs the frame of every step, one sector or several
  if (!multi && c.field.empty()) return al;
  al.resize(n);
  for (size_t k = 0; k < n; ++k) al[k] = sector_alpha(c.cl.sector[idx[k]]);
  return al;
}

// Three-point seed of a track whose clusters may lie in several frames: the
// points are first expressed in the frame of the outermost cluster.
template <class R>
bool seed_track(const Ctx& c, const std::vector<R>& x, const std::vector<R>& yc,
                const std::vector<R>& zc, const std::vector<double>& al, double out[5]) {
  if (al.empty()) return seed_three_points<R>(c, x, yc, zc, out);
  size_t n = x.size();
  std::vector<R> X(x), Y(yc);
  for (size_t k = 0; k < n; ++k) {
    double d = al[n - 1] - al[k];
    if (d == 0.0) continue;
    R ca = R(std::cos(d)), sa = R(std::sin(d));
    X[k] = x[k] * ca + yc[k] * sa;
    Y[k] = -(x[k] * sa) + yc[k] * ca;
  }
  return seed_three_points<R>(c, X, Y, zc, out);
}

template <class R>
void track_inputs(const Ctx& c, const uint32_t* idx, size_t n, double that, std::vector<R>& x,
                  std::vector<R>& yc, std::vector<R>& zc, std::vector<R>& var) {
  x.resize(n); yc.resize(n); zc.resize(n); var.resize(n);
  for (size_t k = 0; k < n; ++k) {
    int64_t i = idx[k];
    x[k] = R(c.rowx[c.cl.row[i]]);
    calibrate<R>(c, i, that, cal_in<R>(c, i), yc[k], zc[k], nullptr);
    R e = cluster_error<R>(c, c.cl.flags[i]);
    var[k] = e * e;
  }
}

// ----------------------------------------------------- segment merging
// Sec. 2, second phase: the track segments found in the individual sectors
// are merged before the final fit. The paper gives no procedure; the reading
// taken here:
//  - a segment is described by its refitted state at its innermost cluster
//    (in its sector's frame), its pad-row range and its collision time;
//  - segment j may continue segment i when both converged, lie in the same
//    event and on the same side (the central electrode is not crossed), j's
//    sector frame is i's or one of its two neighbours, and j starts on a pad
//    row beyond i's last one;
//  - i's state is rotated into j's frame and transported to j's innermost
//    x; in the time-frame mode j's z is first expressed with i's collision
//    time; chi2 = d^T (C_i' + C_j)^-1 d over the five parameters, by a
//    Cholesky factorisation (the pair is not compared when a pivot is not
//    positive);
//  - pairs whose tan(lambda) or q/pT differ by more than sqrt(2 chi2_merge)
//    standard deviations of the difference are not compared (these two
//    parameters are unchanged by the rotation and the transport);
//  - i -> j is a link when chi2 <= chi2_merge and j is i's best continuation
//    and i is j's best predecessor (smallest chi2, then smallest index);
//  - a merged track is a chain of links from a segment without predecessor,
//    its clusters in chain order, its collision time and start hit those of
//    that first segment; merged tracks are ordered by their first segment.
struct SegInfo {
  bool ok;
  int64_t ev;
  int side, frame, rlo, rhi;
};

template <class R>
bool merge_chi2(const Ctx& c, const R pi[5], const R Ci[15], R xi, double thi, const R pj[5],
                const R Cj[15], R xj, double thj, int fi, int fj, int side, R& chi2) {
  R cut = R(c.p.chi2_merge);
  for (int k = 3; k <= 4; ++k) {
    int d = k * (k + 1) / 2 + k;
    R dd = pi[k] - pj[k];
    if (dd * dd > (R(2) * cut) * (Ci[d] + Cj[d])) return false;
  }
  Trk<R> st;
  for (int k = 0; k < 5; ++k) st.p[k] = pi[k];
  st.x = xi;
  for (int a = 0, k = 0; a < 5; ++a)
    for (int b = 0; b <= a; ++b, ++k) {
      st.C[a][b] = Ci[k];
      st.C[b][a] = Ci[k];
    }
  if (fj != fi && !rotate<R>(c, st, sector_alpha(fj) - sector_alpha(fi))) return false;
  if (!propagate<R>(c, st, xj)) return false;
  R shift = R(0);
  if (c.cl.mode == 1) {
    double sg = side == 0 ? 1.0 : -1.0;
    shift = (R)(sg * c.c.vdrift * (thi - thj));
  }
  R d[5];
  for (int k = 0; k < 5; ++k) d[k] = st.p[k] - pj[k];
  d[1] = st.p[1] - (pj[1] + shift);
  // S = C_i' + C_j = L L^T
  R S[5][5], L[5][5];
  for (int a = 0, k = 0; a < 5; ++a)
    for (int b = 0; b <= a; ++b, ++k) S[a][b] = st.C[a][b] + Cj[k];
  for (int a = 0; a < 5; ++a)
    for (int b = 0; b <= a; ++b) {
      R acc = S[a][b];
      for (int k = 0; k < b; ++k) acc = acc - L[a][k] * L[b][k];
      if (a == b) {
        if (!(acc > R(0))) return false;
        L[a][a] = sqrt_(acc);
      } else {
        L[a][b] = acc / L[b][b];
      }
    }
  R w[5];
  for (int a = 0; a < 5; ++a) {
    R acc = d[a];
    for (int k = 0; k < a; ++k) acc = acc - L[a][k] * w[k];
    w[a] = acc / L[a][a];
  }
  R ch = R(0);
  for (int a = 0; a < 5; ++a) ch = ch + w[a] * w[a];
  chi2 = ch;
  return ch <= cut;
}

template <class R>
void merge_links(const Ctx& c, int64_t nt, const uint32_t* ts, const uint32_t* ci,
                 const double* that, const double* params, const double* cov, const double* xs,
                 const int32_t* status, int32_t* next, double* link_chi2) {
  std::vector<SegInfo> sg(nt);
  std::vector<R> P(nt * 5), Cv(nt * 15), X(nt);
  for (int64_t i = 0; i < nt; ++i) {
    SegInfo& g = sg[i];
    uint32_t a = ts[i], b = ts[i + 1];
    g.ok = status[i] == 0 && b > a;
    if (b > a) {
      uint32_t f = ci[a], l = ci[b - 1];
      g.ev = c.cl.event ? (int64_t)c.cl.event[f] : 0;
      g.side = c.cl.sector[f] < 18 ? 0 : 1;
      g.frame = c.cl.sector[f] % 18;
      g.rlo = c.cl.row[f];
      g.rhi = c.cl.row[l];
    }
    for (int k = 0; k < 5; ++k) P[i * 5 + k] = R(params[i * 5 + k]);
    for (int k = 0; k < 15; ++k) Cv[i * 15 + k] = R(cov[i * 15 + k]);
    X[i] = R(xs[i]);
  }
  // best continuation of each segment and best predecessor of each segment
  std::vector<int64_t> out(nt, -1), in(nt, -1);
  std::vector<R> out_c(nt, R(0)), in_c(nt, R(0));
  for (int64_t i = 0; i < nt; ++i) {
    if (!sg[i].ok) continue;
    for (int64_t j = 0; j < nt; ++j) {
      if (j == i || !sg[j].ok || sg[j].ev != sg[i].ev || sg[j].side != sg[i].side) continue;
      int df = (sg[j].frame - sg[i].frame + 18) % 18;
      if (!(df == 0 || df == 1 || df == 17) || !(sg[j].rlo > sg[i].rhi)) continue;
      R ch;
      if (!merge_chi2<R>(c, &P[i * 5], &Cv[i * 15], X[i], that[i], &P[j * 5], &Cv[j * 15], X[j],
                         that[j], sg[i].frame, sg[j].frame, sg[i].side, ch))
        continue;
      if (out[i] < 0 || ch < out_c[i]) { out[i] = j; out_c[i] = ch; }
      if (in[j] < 0 || ch < in_c[j] || (ch == in_c[j] && i < in[j])) { in[j] = i; in_c[j] = ch; }
    }
  }
  for (int64_t i = 0; i < nt; ++i) {
    next[i] = -1;
    link_chi2[i] = 0.0;
    if (out[i] >= 0 && in[out[i]] == i) {
      next[i] = (int32_t)out[i];
      link_chi2[i] = (double)val(out_c[i]);
    }
  }
}

// --------------------------------------- collision time after merging
// Time-frame mode (Sec. 4, the steps after merging): the vertex estimate is
// refined with the merged track's fit and the track is shifted in z to it;
// a track with clusters outside the drift volume is shifted back inside.
// Reading: the collision time moves so that the fitted helix (state p at x,
// at the innermost cluster) reaches its closest approach to the beam line at
// z = 0: every cluster's absolute z moves by -z0, i.e. the collision time by
// -sg z0 / v_drift. Then each cluster's drift time t - t0 - that must lie in
// [0, L / v_drift]; when the largest exceeds the bound the collision time
// moves up to meet it, and when the smallest is negative it moves down to it
// (this last rule wins when both apply).
template <class R>
double refine_time(const Ctx& c, const uint32_t* idx, size_t n, double that, const double p[5],
                   double x) {
  Trk<R> st;
  for (int k = 0; k < 5; ++k) st.p[k] = R(p[k]);
  st.x = R(x);
  R z0 = dca_z<R>(c, st);
  double sg = c.cl.sector[idx[0]] < 18 ? 1.0 : -1.0;
  double th = that - (sg * (double)val(z0)) / c.c.vdrift;
  double lo = c.cl.t[idx[0]] - c.c.t0, hi = lo;
  for (size_t k = 1; k < n; ++k) {
    double d = c.cl.t[idx[k]] - c.c.t0;
    lo = std::min(lo, d);
    hi = std::max(hi, d);
  }
  double T = (double)c.g.drift_length / c.c.vdrift;
  if (hi - th > T) th = th + ((hi - th) - T);
  if (lo - th < 0.0) th = th + (lo - th);
  return th;
}

// ------------------------------------------- track-model compression
// Sec. 5 (entropy reduction for the TPC data compression): only residuals
// of the clusters attached to tracks are stored, with respect to the track
// model, and the track is fitted in the distorted (uncalibrated) coordinate
// system, so that calibration effects do not enter the residuals. Reading:
// along each track (clusters in row order; the model restarts where the
// sector frame changes) the first cluster of a run is stored as quantised
// absolute (y, z); the second as the quantised difference to the first;
// from then on a Kalman filter (the tracklet filter: straight-line two-point
// seed through the first two decoded clusters, helix transport, update with
// each decoded cluster) predicts (y, z) at the next row and the residual is
// round((measured - predicted) / q). Every step uses the decoded cluster
// (prediction + residual * q), so that a decoder running the same single-
// precision arithmetic on the residuals reproduces the decoded clusters
// exactly; where the transport fails the prediction is the previous decoded
// cluster and the filter restarts there. Measured z in the time-frame mode:
// the drift time turned into z with the track's collision time and v_drift,
// without the distortion correction. Decisions in FP32.
struct CompressIO {
  const float* my;  // measured y, z per cluster of the track (encoder), or null
  const float* mz;
  int32_t* ry;      // residuals (out for the encoder, in for the decoder)
  int32_t* rz;
  float* dy;        // decoded clusters (out)
  float* dz;
};

void code_track(const Ctx& c, const uint32_t* idx, size_t n, float qy, float qz,
                bool encode, CompressIO& io) {
  const float iqy = 1.0f / qy, iqz = 1.0f / qz;
  const float sig2 = c.p.sigma * c.p.sigma;
  Trk<float> st;
  int frame = -1;
  size_t j = 0;        // position inside the current frame run
  bool model = false;  // the filter holds a state
  float px = 0.0f, pyd = 0.0f, pzd = 0.0f;  // previous decoded cluster
  for (size_t k = 0; k < n; ++k) {
    int64_t i = idx[k];
    int f = c.cl.sector[i] % 18;
    float x = c.rowx[c.cl.row[i]];
    if (f != frame) {
      frame = f;
      j = 0;
      model = false;
    }
    float prey = 0.0f, prez = 0.0f;  // prediction
    bool absolute = j == 0;
    if (j >= 2 && model && propagate<float>(c, st, x)) {
      prey = st.p[0];
      prez = st.p[1];
    } else if (!absolute) {
      prey = pyd;
      prez = pzd;
      model = false;
    }
    int32_t ry, rz;
    if (encode) {
      ry = (int32_t)std::nearbyint((io.my[k] - prey) * iqy);
      rz = (int32_t)std::nearbyint((io.mz[k] - prez) * iqz);
      io.ry[k] = ry;
      io.rz[k] = rz;
    } else {
      ry = io.ry[k];
      rz = io.rz[k];
    }
    float dy = prey + (float)ry * qy;
    float dz = prez + (float)rz * qz;
    io.dy[k] = dy;
    io.dz[k] = dz;
    if (j >= 1) {
      if (!model) {
        // (re)start: seed through the previous and this decoded cluster,
        // then the filter takes this cluster
        seed_two_points<float>(c, st, px, pyd, pzd, x, dy, dz);
        model = propagate<float>(c, st, x);
      }
      if (model) apply_update<float>(st, innovation<float>(st, dy, dz, sig2, sig2));
    }
    px = x;
    pyd = dy;
    pzd = dz;
    ++j;
  }
}

// Measured (distorted) coordinates of a track's clusters: y as given, z as
// given (event mode) or from the drift time with the track's collision time.
void distorted_coords(const Ctx& c, const uint32_t* idx, size_t n, double that,
                      std::vector<float>& y, std::vector<float>& z) {
  y.resize(n);
  z.resize(n);
  for (size_t k = 0; k < n; ++k) {
    int64_t i = idx[k];
    y[k] = c.cl.y[i];
    if (c.cl.mode == 0) {
      z[k] = c.cl.z[i];
    } else {
      double sg = c.cl.sector[i] < 18 ? 1.0 : -1.0;
      double zeta = c.c.vdrift * ((c.cl.t[i] - c.c.t0) - that);
      z[k] = (float)(sg * ((double)c.g.drift_length - zeta));
    }
  }
}

}  // namespace

// ======================================================================
// exported entry points (ctypes)
// ======================================================================
extern "C" {

void* orc_create(const OrcGeom* g, const OrcParams* p, const OrcCalib* cal,
                 const OrcClusters* cl) {
  return build_ctx(g, p, cal, cl);
}
void orc_destroy(void* ctx) { delete (Ctx*)ctx; }

void orc_seed_z(void* ctx, int prec, void* out) {
  Ctx& c = *(Ctx*)ctx;
  if (prec == 32) std::memcpy(out, c.zs32.data(), c.zs32.size() * sizeof(float));
  else std::memcpy(out, c.zs64.data(), c.zs64.size() * sizeof(double));
}

// Calibrated (yc, zc) of clusters idx[k] with collision time that[k].
void orc_calibrate(void* ctx, int prec, int64_t m, const uint32_t* idx, const double* that,
                   double* yc, double* zc) {
  Ctx& c = *(Ctx*)ctx;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < m; ++k) {
    if (prec == 32) {
      float a, b;
      calibrate<float>(c, idx[k], that[k], cal_in<float>(c, idx[k]), a, b, nullptr);
      yc[k] = a; zc[k] = b;
    } else {
      double a, b;
      calibrate<double>(c, idx[k], that[k], cal_in<double>(c, idx[k]), a, b, nullptr);
      yc[k] = a; zc[k] = b;
    }
  }
}

// Spline value at explicit points (for closed-form checks of the spline).
void orc_spline(void* ctx, int64_t m, const int32_t* sector, const double* x, const double* y,
                const double* az, double* dy, double* dz) {
  Ctx& c = *(Ctx*)ctx;
  for (int64_t k = 0; k < m; ++k) {
    double d[2];
    spline_eval<double>(c, sector[k], x[k], y[k], az[k], d, nullptr);
    dy[k] = d[0];
    dz[k] = d[1];
  }
}

// Neighbour links (original cluster indices, -1 = none) of hits[k]
// (all clusters when hits == NULL).
// margin (may be NULL; FP64 only): each hit's smallest decision margin.
void orc_neighbours(void* ctx, int prec, const int64_t* hits, int64_t nh, int32_t* up,
                    int32_t* dn, double* margin) {
  Ctx& c = *(Ctx*)ctx;
  int64_t m = hits ? nh : c.cl.n;
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t k = 0; k < m; ++k) {
    int64_t h = hits ? hits[k] : k;
    if (prec == 32) {
      neighbours_of<float>(c, h, up[k], dn[k]);
    } else {
      Margin mg;
      neighbours_of<double>(c, h, up[k], dn[k], margin ? &mg : nullptr);
      if (margin) margin[k] = mg.m;
    }
  }
}

// Link cleaner (Sec. 2 "evolution"): keep only mutual links.
void orc_clean(void* ctx, const int32_t* up, const int32_t* dn, int32_t* upc, int32_t* dnc) {
  Ctx& c = *(Ctx*)ctx;
  for (int64_t h = 0; h < c.cl.n; ++h) {
    upc[h] = (up[h] >= 0 && dn[up[h]] == h) ? up[h] : -1;
    dnc[h] = (dn[h] >= 0 && up[dn[h]] == h) ? dn[h] : -1;
  }
}

// Chain heads with at least three linked hits, increasing index order.
int64_t orc_start_hits(void* ctx, const int32_t* upc, const int32_t* dnc, int64_t* out) {
  Ctx& c = *(Ctx*)ctx;
  int64_t m = 0;
  for (int64_t h = 0; h < c.cl.n; ++h)
    if (dnc[h] < 0 && upc[h] >= 0 && upc[upc[h]] >= 0) out[m++] = h;
  return m;
}

// One tracklet per start hit; hits is [m][n_rows], state [m][5].
// margin, decisions (may be NULL; FP64 only): each tracklet's smallest
// decision margin and the number of its decisions.
void orc_tracklets(void* ctx, int prec, const int32_t* upc, int64_t m, const int64_t* starts,
                   int32_t* nh, int32_t* hits, double* that, double* state, double* xout,
                   double* margin, int64_t* decisions) {
  Ctx& c = *(Ctx*)ctx;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t k = 0; k < m; ++k) {
    Margin mg;
    TrackletOut o = prec == 32 ? tracklet<float>(c, upc, starts[k], hits + k * c.g.n_rows)
                               : tracklet<double>(c, upc, starts[k], hits + k * c.g.n_rows,
                                                  (margin || decisions) ? &mg : nullptr);
    if (margin) margin[k] = o.margin;
    if (decisions) decisions[k] = o.decisions;
    nh[k] = o.nh;
    that[k] = o.that;
    for (int i = 0; i < 5; ++i) state[k * 5 + i] = o.state[i];
    xout[k] = o.x;
  }
}

// Tracklet selector: each cluster goes to the tracklet with the most hits
// (ties: lower start index); a tracklet becomes a track when it keeps at
// least min_track_hits clusters with no row gap above max_gap.
int64_t orc_select(void* ctx, int64_t m, const int64_t* starts, const int32_t* nh,
                   const int32_t* hits, const double* that, uint32_t* track_start,
                   uint32_t* cluster_idx, double* track_that, int64_t* track_id,
                   int64_t cap_tracks, int64_t cap_clusters) {
  Ctx& c = *(Ctx*)ctx;
  int R = c.g.n_rows;
  std::vector<uint64_t> w(c.cl.n, 0);
  auto wt = [&](int64_t k) {
    return ((uint64_t)(uint32_t)nh[k] << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)starts[k]);
  };
  for (int64_t k = 0; k < m; ++k) {
    if (nh[k] < c.p.min_track_hits) continue;
    uint64_t wk = wt(k);
    for (int r = 0; r < R; ++r) {
      int32_t j = hits[k * R + r];
      if (j >= 0 && w[j] < wk) w[j] = wk;
    }
  }
  int64_t nt = 0, nc = 0;
  track_start[0] = 0;
  for (int64_t k = 0; k < m; ++k) {
    if (nh[k] < c.p.min_track_hits) continue;
    uint64_t wk = wt(k);
    int kept = 0, lastr = -1, maxgap = 0;
    for (int r = 0; r < R; ++r) {
      int32_t j = hits[k * R + r];
      if (j < 0 || w[j] != wk) continue;
      if (lastr >= 0) maxgap = std::max(maxgap, r - lastr - 1);
      lastr = r;
      ++kept;
    }
    if (kept < c.p.min_track_hits || maxgap > c.p.max_gap) continue;
    if (nt >= cap_tracks || nc + kept > cap_clusters) return -1;
    for (int r = 0; r < R; ++r) {
      int32_t j = hits[k * R + r];
      if (j >= 0 && w[j] == wk) cluster_idx[nc++] = (uint32_t)j;
    }
    track_that[nt] = that[k];
    track_id[nt] = starts[k];
    ++nt;
    track_start[nt] = (uint32_t)nc;
  }
  return nt;
}

// Refit of tracks (CSR, clusters in increasing row order). seeds: optional
// [nt][5] seed states at the outermost cluster; seeds_out receives the seeds
// used. rej: [n_assigned] rejection pass per cluster (0 kept); with
// frozen != 0 it is an input and no new decision is taken.
// zv (may be NULL): vertex z per track (NaN: none), variance vvar.
void orc_refit(void* ctx, int prec, int64_t nt, const uint32_t* track_start,
               const uint32_t* cluster_idx, const double* that, const double* seeds,
               double* seeds_out, int frozen, uint8_t* rej, double* params, double* cov,
               double* xout, double* chi2, int32_t* ndf, int32_t* status, const double* zv,
               double vvar) {
  Ctx& c = *(Ctx*)ctx;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t k = 0; k < nt; ++k) {
    size_t a = track_start[k], b = track_start[k + 1], n = b - a;
    uint8_t* rj = rej + a;
    if (!frozen) std::memset(rj, 0, n);
    RefitOut o;
    std::memset(&o, 0, sizeof(o));
    double seed[5];
    bool ok;
    std::vector<double> al = track_alpha(c, cluster_idx + a, n);
    const std::vector<double>* alp = al.empty() ? nullptr : &al;
    if (prec == 32) {
      std::vector<float> x, yc, zc, var;
      track_inputs<float>(c, cluster_idx + a, n, that[k], x, yc, zc, var);
      ok = seeds ? true : seed_track<float>(c, x, yc, zc, al, seed);
      if (seeds) for (int i = 0; i < 5; ++i) seed[i] = seeds[k * 5 + i];
      if (ok) {
        float ch;
        o = refit_core<float>(c, x, yc, zc, var, seed, rj, frozen, &ch, alp, nullptr,
                              zv ? zv[k] : NAN, vvar);
      }
    } else {
      std::vector<double> x, yc, zc, var;
      track_inputs<double>(c, cluster_idx + a, n, that[k], x, yc, zc, var);
      ok = seeds ? true : seed_track<double>(c, x, yc, zc, al, seed);
      if (seeds) for (int i = 0; i < 5; ++i) seed[i] = seeds[k * 5 + i];
      if (ok) {
        double ch;
        o = refit_core<double>(c, x, yc, zc, var, seed, rj, frozen, &ch, alp, nullptr,
                               zv ? zv[k] : NAN, vvar);
      }
    }
    if (!ok) o.status = 2;
    if (seeds_out) for (int i = 0; i < 5; ++i) seeds_out[k * 5 + i] = ok ? seed[i] : 0.0;
    for (int i = 0; i < 5; ++i) params[k * 5 + i] = o.p[i];
    for (int i = 0; i < 15; ++i) cov[k * 15 + i] = o.C[i];
    xout[k] = o.x;
    chi2[k] = o.chi2;
    ndf[k] = o.ndf;
    status[k] = o.status;
  }
}

// Gradient of L = sum_k g[k] chi2_k (pass 3) by reverse-mode differentiation
// of the FP64 refit with frozen rejections and seeds. Outputs per assigned
// cluster d/dy and d/d(t or z) of the raw measurement, and
// grad_calib = [dL/dvdrift, dL/dt0, dL/dspline[36*2*512]] (accumulated).
void orc_refit_grad(void* ctx, int64_t nt, const uint32_t* track_start,
                    const uint32_t* cluster_idx, const double* that, const double* seeds,
                    const uint8_t* rej, const double* g, double* grad_y, double* grad_zt,
                    double* grad_calib, const double* zv, double vvar) {
  Ctx& c = *(Ctx*)ctx;
  // Each track's terms (its own tape, on any thread), then summed in track
  // order, so the sums do not depend on the number of threads.
  struct Terms {
    bool ok = false;
    std::vector<double> gy, gz;
    double vd = 0.0, t0 = 0.0;
    std::vector<std::pair<int, double>> spline;
  };
  const int64_t chunk = 4096;
  std::vector<Terms> terms;
  for (int64_t k0 = 0; k0 < nt; k0 += chunk) {
    const int64_t k1 = std::min(nt, k0 + chunk);
    terms.assign((size_t)(k1 - k0), Terms());
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t k = k0; k < k1; ++k) {
      Terms& T = terms[(size_t)(k - k0)];
      size_t a = track_start[k], b = track_start[k + 1], n = b - a;
      g_tape.clear();
      CoefLeaves lv;
      Var vd = Var::leaf(c.c.vdrift);
      Var t0 = Var::leaf(c.c.t0);
      std::vector<Var> ly(n), lz(n), x(n), yc(n), zc(n), var(n);
      for (size_t q = 0; q < n; ++q) {
        int64_t i = cluster_idx[a + q];
        CalIn<Var> in;
        in.vdrift = vd;
        in.t0 = t0;
        ly[q] = Var::leaf(c.cl.y[i]);
        if (c.cl.mode == 1) {
          lz[q] = Var::leaf(c.cl.t[i]);
          in.t = lz[q];
          in.z = Var(0.0);
        } else {
          lz[q] = Var::leaf(c.cl.z[i]);
          in.z = lz[q];
          in.t = Var(0.0);
        }
        in.y = ly[q];
        x[q] = Var(c.rowx[c.cl.row[i]]);
        calibrate<Var>(c, i, that[k], in, yc[q], zc[q], &lv);
        double e = cluster_error<double>(c, c.cl.flags[i]);
        var[q] = Var(e * e);
      }
      std::vector<uint8_t> rj(rej + a, rej + b);
      std::vector<double> al = track_alpha(c, cluster_idx + a, n);
      Var chi2;
      RefitOut o = refit_core<Var>(c, x, yc, zc, var, seeds + k * 5, rj.data(), true, &chi2,
                                   al.empty() ? nullptr : &al, nullptr, zv ? zv[k] : NAN, vvar);
      if (o.status != 0) {
        g_tape.clear();
        continue;
      }
      g_tape.backward(chi2.id, g[k]);
      auto adj = [&](const Var& v) { return v.id >= 0 ? g_tape.adj[v.id] : 0.0; };
      T.ok = true;
      T.gy.resize(n);
      T.gz.resize(n);
      for (size_t q = 0; q < n; ++q) {
        // per pad for native input: dy/dpad is the row's pad pitch
        double dyp = c.cl.pads ? (double)c.padw[c.cl.row[cluster_idx[a + q]]] : 1.0;
        T.gy[q] = adj(ly[q]) * dyp;
        T.gz[q] = adj(lz[q]);
      }
      T.vd = adj(vd);
      T.t0 = adj(t0);
      for (auto& kv : lv.m) T.spline.emplace_back(kv.first, adj(kv.second));
      g_tape.clear();
    }
    for (int64_t k = k0; k < k1; ++k) {
      const Terms& T = terms[(size_t)(k - k0)];
      if (!T.ok) continue;
      size_t a = track_start[k];
      for (size_t q = 0; q < T.gy.size(); ++q) {
        grad_y[a + q] += T.gy[q];
        grad_zt[a + q] += T.gz[q];
      }
      grad_calib[0] += T.vd;
      grad_calib[1] += T.t0;
      for (auto& kv : T.spline) grad_calib[2 + kv.first] += kv.second;
    }
  }
}

// The refit's covariance update: 1 = Joseph form, 0 = the short form.
void orc_set_joseph(void* ctx, int on) { ((Ctx*)ctx)->joseph = on != 0; }

// Threads used by the parallel loops (over hits, start hits, tracks and
// clusters); n < 1 leaves the setting unchanged. Returns the count in force.
int orc_threads(int n) {
  if (n >= 1) omp_set_num_threads(n);
  return omp_get_max_threads();
}

// Segment merging (Sec. 2, second phase), decisions in precision prec.
// Inputs: the segments as a track set (CSR), their collision times and
// refitted states at the innermost cluster (params [nt][5], cov [nt][15]
// packed lower triangle, x [nt], status [nt]). Outputs: next [nt] (the
// following segment or -1) and its chi2; the merged track set (out_ts
// [nt + 1], out_ci [n_assigned], out_that and out_head [nt]). Returns the
// number of merged tracks.
int64_t orc_merge(void* ctx, int prec, int64_t nt, const uint32_t* ts, const uint32_t* ci,
                  const double* that, const double* params, const double* cov, const double* x,
                  const int32_t* status, int32_t* next, double* link_chi2, uint32_t* out_ts,
                  uint32_t* out_ci, double* out_that, int64_t* out_head) {
  Ctx& c = *(Ctx*)ctx;
  if (prec == 32)
    merge_links<float>(c, nt, ts, ci, that, params, cov, x, status, next, link_chi2);
  else
    merge_links<double>(c, nt, ts, ci, that, params, cov, x, status, next, link_chi2);
  std::vector<char> has_in(nt, 0);
  for (int64_t i = 0; i < nt; ++i)
    if (next[i] >= 0) has_in[next[i]] = 1;
  int64_t m = 0;
  uint32_t nc = 0;
  out_ts[0] = 0;
  for (int64_t i = 0; i < nt; ++i) {
    if (has_in[i]) continue;
    for (int64_t s = i; s >= 0; s = next[s])
      for (uint32_t k = ts[s]; k < ts[s + 1]; ++k) out_ci[nc++] = ci[k];
    out_that[m] = that[i];
    out_head[m] = i;
    ++m;
    out_ts[m] = nc;
  }
  return m;
}

// Track-model compression (Sec. 5): residuals (ry, rz) [n_assigned] of the
// track set's clusters and the decoded clusters (dy, dz).
void orc_compress(void* ctx, int64_t nt, const uint32_t* ts, const uint32_t* ci,
                  const double* that, float qy, float qz, int32_t* ry, int32_t* rz, float* dy,
                  float* dz) {
  Ctx& c = *(Ctx*)ctx;
  std::vector<float> my, mz;
  for (int64_t k = 0; k < nt; ++k) {
    uint32_t a = ts[k], b = ts[k + 1];
    distorted_coords(c, ci + a, b - a, that[k], my, mz);
    CompressIO io{my.data(), mz.data(), ry + a, rz + a, dy + a, dz + a};
    code_track(c, ci + a, b - a, qy, qz, true, io);
  }
}

// The decoder: clusters (dy, dz) from the residuals, the rows and sectors.
void orc_decompress(void* ctx, int64_t nt, const uint32_t* ts, const uint32_t* ci, float qy,
                    float qz, const int32_t* ry, const int32_t* rz, float* dy, float* dz) {
  Ctx& c = *(Ctx*)ctx;
  for (int64_t k = 0; k < nt; ++k) {
    uint32_t a = ts[k], b = ts[k + 1];
    CompressIO io{nullptr, nullptr, const_cast<int32_t*>(ry) + a, const_cast<int32_t*>(rz) + a,
                  dy + a, dz + a};
    code_track(c, ci + a, b - a, qy, qz, false, io);
  }
}

// Collision times of tracks refined from their fits (time-frame mode; the
// event mode and tracks whose refit failed keep theirs).
void orc_refine_time(void* ctx, int prec, int64_t nt, const uint32_t* ts, const uint32_t* ci,
                     const double* that, const double* params, const double* x,
                     const int32_t* status, double* that_out) {
  Ctx& c = *(Ctx*)ctx;
  for (int64_t k = 0; k < nt; ++k) {
    uint32_t a = ts[k], b = ts[k + 1];
    that_out[k] = that[k];
    if (c.cl.mode != 1 || status[k] != 0 || b <= a) continue;
    that_out[k] = prec == 32
        ? refine_time<float>(c, ci + a, b - a, that[k], params + 5 * k, x[k])
        : refine_time<double>(c, ci + a, b - a, that[k], params + 5 * k, x[k]);
  }
}

// Rotation of a state (and covariance, packed lower triangle) by dalpha.
int orc_rotate(void* ctx, const double* state, double x, double dalpha, const double* cov,
               double* state_out, double* x_out, double* cov_out) {
  Ctx& c = *(Ctx*)ctx;
  Trk<double> st;
  for (int i = 0; i < 5; ++i) st.p[i] = state[i];
  st.x = x;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) st.C[i][j] = cov[i * 5 + j];
  if (!rotate<double>(c, st, dalpha)) return 0;
  for (int i = 0; i < 5; ++i) state_out[i] = st.p[i];
  *x_out = st.x;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) cov_out[i * 5 + j] = st.C[i][j];
  return 1;
}

// Refit of one track given float64 points directly (for closed-form checks).
// priors (may be NULL): [3][21] the state each pass starts from (x, the
// parameters, the covariance's lower triangle); cov_out (may be NULL): [15].
int orc_refit_points(void* ctx, int64_t n, const double* x, const double* y, const double* z,
                     double var, double* params_out, double* chi2, int32_t* ndf,
                     double* priors, double* cov_out) {
  Ctx& c = *(Ctx*)ctx;
  std::vector<double> X(x, x + n), Y(y, y + n), Z(z, z + n), V(n, var);
  double seed[5];
  if (!seed_three_points<double>(c, X, Y, Z, seed)) return 2;
  std::vector<uint8_t> rj(n, 0);
  double ch;
  RefitOut o = refit_core<double>(c, X, Y, Z, V, seed, rj.data(), false, &ch, nullptr, priors);
  if (cov_out)
    for (int i = 0; i < 15; ++i) cov_out[i] = o.C[i];
  for (int i = 0; i < 5; ++i) params_out[i] = o.p[i];
  *chi2 = o.chi2;
  *ndf = o.ndf;
  return o.status;
}

// Transport in the full field (state and covariance, in the frame alpha).
int orc_propagate_field(void* ctx, const double* state_in, double x1, double x2, double alpha,
                        const double* cov_in, double* state_out, double* cov_out) {
  Ctx& c = *(Ctx*)ctx;
  if (c.field.empty()) return 0;
  Trk<double> st;
  for (int i = 0; i < 5; ++i) st.p[i] = state_in[i];
  st.x = x1;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) st.C[i][j] = cov_in[i * 5 + j];
  if (!propagate_field<double>(c, st, x2, alpha)) return 0;
  for (int i = 0; i < 5; ++i) state_out[i] = st.p[i];
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) cov_out[i * 5 + j] = st.C[i][j];
  return 1;
}

// Single-step helpers exposed for closed-form checks of the track model.
int orc_propagate(void* ctx, const double* state_in, double x1, double x2, const double* cov_in,
                  double* state_out, double* cov_out) {
  Ctx& c = *(Ctx*)ctx;
  Trk<double> st;
  for (int i = 0; i < 5; ++i) st.p[i] = state_in[i];
  st.x = x1;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) st.C[i][j] = cov_in[i * 5 + j];
  if (!propagate<double>(c, st, x2)) return 0;
  for (int i = 0; i < 5; ++i) state_out[i] = st.p[i];
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) cov_out[i * 5 + j] = st.C[i][j];
  return 1;
}

int orc_jacobian(void* ctx, const double* state_in, double x1, double x2, double* state_out,
                 double* J) {
  Ctx& c = *(Ctx*)ctx;
  Trk<double> st;
  for (int i = 0; i < 5; ++i) st.p[i] = state_in[i];
  st.x = x1;
  set_diag(st, c.p.c0r);
  if (!propagate<double>(c, st, x2, J)) return 0;
  for (int i = 0; i < 5; ++i) state_out[i] = st.p[i];
  return 1;
}

void orc_update(const double* state_in, const double* cov_in, double my, double mz, double vy,
                double vz, double* state_out, double* cov_out, double* chi2) {
  Trk<double> st;
  for (int i = 0; i < 5; ++i) st.p[i] = state_in[i];
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) st.C[i][j] = cov_in[i * 5 + j];
  st.x = 0;
  Innov<double> in = innovation<double>(st, my, mz, vy, vz);
  apply_update<double>(st, in);
  *chi2 = in.chi2;
  for (int i = 0; i < 5; ++i) state_out[i] = st.p[i];
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) cov_out[i * 5 + j] = st.C[i][j];
}

double orc_dca_z(void* ctx, const double* state, double x) {
  Ctx& c = *(Ctx*)ctx;
  Trk<double> st;
  for (int i = 0; i < 5; ++i) st.p[i] = state[i];
  st.x = x;
  return dca_z<double>(c, st);
}

double orc_arc_factor(int prec, double h) {
  return prec == 32 ? (double)A_of((float)h) : A_of(h);
}
double orc_arc_deriv(int prec, double h) {
  return prec == 32 ? (double)B_of((float)h) : B_of(h);
}

}  // extern "C"
