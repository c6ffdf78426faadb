// gv_device.cuh -- device functions of one transport step (GeantV Sec. 2.1.2
// stages PreStep .. SteppingActions), templated on the arithmetic type R of
// physics and energies: float (mixed mode: positions and boundary distances
// stay FP64) or double (FP64 everywhere).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "gv_internal.h"

namespace gv {

// ---------------------------------------------------------------- math shims
__device__ __forceinline__ float m_log(float x) { return logf(x); }
__device__ __forceinline__ double m_log(double x) { return log(x); }
__device__ __forceinline__ float m_log1p(float x) { return log1pf(x); }
__device__ __forceinline__ double m_log1p(double x) { return log1p(x); }
__device__ __forceinline__ float m_expm1(float x) { return expm1f(x); }
__device__ __forceinline__ double m_expm1(double x) { return expm1(x); }
__device__ __forceinline__ float m_exp(float x) { return expf(x); }
__device__ __forceinline__ double m_exp(double x) { return exp(x); }
__device__ __forceinline__ float m_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double m_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float m_cos(float x) { return cosf(x); }
__device__ __forceinline__ double m_cos(double x) { return cos(x); }
__device__ __forceinline__ void m_sincos(float x, float *s, float *c) { sincosf(x, s, c); }
__device__ __forceinline__ void m_sincos(double x, double *s, double *c) { sincos(x, s, c); }
__device__ __forceinline__ float m_floor(float x) { return floorf(x); }
__device__ __forceinline__ double m_floor(double x) { return floor(x); }

// Quotients of the per-step geometry and step limits.  FP32: the fast
// division (reciprocal times numerator, 2 ulp) instead of the IEEE-rounded
// one, whose correction sequence costs several instructions on every step;
// callers keep the divisor away from 0 and from the top of the range.
__device__ __forceinline__ float q_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double q_div(double a, double b) { return a / b; }
// 1/sqrt(x): the hardware reciprocal square root in FP32 (the same 2-ulp
// class as q_div), the IEEE quotient in FP64.
__device__ __forceinline__ float q_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double q_rsqrt(double x) { return 1.0 / sqrt(x); }

// log(1 + x) for |x| <= 0.16 in FP32: its Taylor series to x^8 (truncation
// error below 8e-9 there, under half an FP32 ulp of the result).
__device__ __forceinline__ float log1p_small(float x) {
  float p = -0.125f;
  p = fmaf(p, x, 0.14285714285714285f);
  p = fmaf(p, x, -0.16666666666666666f);
  p = fmaf(p, x, 0.2f);
  p = fmaf(p, x, -0.25f);
  p = fmaf(p, x, 0.3333333333333333f);
  p = fmaf(p, x, -0.5f);
  p = fmaf(p, x, 1.0f);
  return p * x;
}

template <typename R> __host__ __device__ inline R r_inf_host() {
  return static_cast<R>(1e300) * static_cast<R>(1e300);  // +inf in R
}

template <typename R> __device__ __forceinline__ R r_inf();
template <> __device__ __forceinline__ float r_inf<float>() { return __int_as_float(0x7f800000); }
template <> __device__ __forceinline__ double r_inf<double>() { return __longlong_as_double(0x7ff0000000000000ll); }

// Exact float -> double from the bits, without the FP64 pipe (on GB300 it
// also carries every conversion, at 1/64 of the FP32 rate).  Zeros and
// normal numbers; subnormals and non-finite values take the instruction.
__device__ __forceinline__ double f2d(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) {
    if ((b << 1) == 0u) return __hiloint2double(static_cast<int>(b & 0x80000000u), 0);
    return static_cast<double>(f);
  }
  const unsigned hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
  return __hiloint2double(static_cast<int>(hi), static_cast<int>(b << 29));
}
__device__ __forceinline__ double f2d(double f) { return f; }

template <typename R> struct alignas(4 * sizeof(R)) V4 { R x, y, z, w; };

// Index and state checks of the checking build (-DGV_CHECKS): a failed check
// records GV_ERR_INTERNAL in the status word it is given (if any) and the
// work goes on with clamped values; nothing traps.  The release build
// compiles them away.
#ifdef GV_CHECKS
#define GV_CHECK(status_ptr, cond)                                          \
  do {                                                                      \
    if (!(cond) && (status_ptr)) atomicCAS((status_ptr), 0, GV_ERR_INTERNAL); \
  } while (0)
#else
#define GV_CHECK(status_ptr, cond) \
  do {                             \
  } while (0)
#endif

// one bin of an alias table: acceptance q, alias index, pdf at the bin edges
template <typename R> struct AliasBin { float q; int a; R p0, p1; };

struct ModelMeta {
  double ln_Elo, inv_dl, cut;
  int nE, off;
};

struct GeoConst {
  int nsub, nsub_layer, n_layers, nx, ny;
  double hx, hy, pitch_x, pitch_y;
  double wx[2], wy[2];  // the x and y walls {-h, +h}
  float inv_pitch_x, inv_pitch_y;
  float hx_lo, hy_lo;   // the half widths rounded down to FP32
  int walls_x, walls_y; // 0: unbounded in that direction
  int field_axis;       // uniform magnetic field along x, y or z
};

struct CutConst {
  double gcut, ecut, tcut;
  unsigned mask;
};

// The cuts and the alias grids' constants in R, converted once on the host:
// on GB300 a conversion between FP64 and FP32 issues on the FP64 pipe,
// which the FP32 kernels should leave to the position arithmetic.
template <typename R> struct RConst {
  R tcut, gcut, ecut, ecut_push;  // ecut_push = max(e- cut, tracking cut)
  R ln_Elo[kNModel], inv_dl[kNModel], cut[kNModel];
  R inv_X0[GV_MAX_MAT];  // 1 / radiation length, 1/cm
  R field_k;             // 2.99792458 B: curvature (1/cm) times momentum (MeV/c); 0 without field
  R rej_min[kNModel];    // rejection sampling of model m at E >= rej_min[m]
};

// Read-only view of everything one step needs.
template <typename R> struct View {
  const V4<R> *xs;           // [(mat*3 + type)*kGridN + node], smem or global
  const float *inv_node;     // 1/E_i of the grid nodes (FP32 lookups)
  const double *zb;          // nsub+1 planes
  const unsigned char *smat; // material of each sub-slab
  const AliasBin<R> *bins;   // all models, [off + ie*kNB + j]
  const R *smax;             // integral approach bound [(mat*2 + type-1)*kGridN + node], smem or global
  int *status;               // where checks record a failure (checking build), or null
  ModelMeta meta[kNModel];
  GeoConst geo;
  CutConst cut;
  RConst<R> rc;
};

// ---------------------------------------------------------------- RNG
// Philox4x32-10: Salmon, Moraes, Dror, Shaw, SC'11 (the Random123 family).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    // one 32x32->64 multiply gives both halves of each product
    const unsigned long long p0 = static_cast<unsigned long long>(0xD2511F53u) * c.x;
    const unsigned long long p1 = static_cast<unsigned long long>(0xCD9E8D57u) * c.z;
    const uint32_t hi0 = static_cast<uint32_t>(p0 >> 32), lo0 = static_cast<uint32_t>(p0);
    const uint32_t hi1 = static_cast<uint32_t>(p1 >> 32), lo1 = static_cast<uint32_t>(p1);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// uniform in (0, 1], exact in FP32 and FP64
template <typename R> __device__ __forceinline__ R u24(uint32_t x) {
  return static_cast<R>((x >> 8) + 1u) * static_cast<R>(1.0 / 16777216.0);
}

// ---------------------------------------------------------------- tables
// Node interval i and fraction f of ln E between nodes i and i+1 (clamped).
// FP64: directly from ln E.  FP32: ln E near 10 GeV carries ~1e-6 absolute
// error, i.e. 1e-5 of a node interval, so the node comes from a coarse log2
// and the fraction from log1p(E/E_i - 1), accurate to ~1e-6 of an interval.
template <typename R> __device__ __forceinline__ void grid_pos(const View<R> &V, R E, int &i, R &f);

template <> __device__ __forceinline__ void grid_pos<double>(const View<double> &, double E, int &i, double &f) {
  const double l = (log(E) + 6.907755278982137) * (kGridPerDecade / 2.302585092994046);
  int k = static_cast<int>(floor(l));
  k = k < 0 ? 0 : (k > kGridN - 2 ? kGridN - 2 : k);
  double fr = l - static_cast<double>(k);
  fr = fr < 0.0 ? 0.0 : (fr > 1.0 ? 1.0 : fr);
  i = k;
  f = fr;
}

template <> __device__ __forceinline__ void grid_pos<float>(const View<float> &V, float E, int &i, float &f) {
  constexpr float kInvDl = static_cast<float>(kGridPerDecade / 2.302585092994046);
  const float l = (__log2f(E) + 9.965784284662087f) * 9.632959861247398f;
  int k = __float2int_rd(l);
  k = k < 0 ? 0 : (k > kGridN - 2 ? kGridN - 2 : k);
  // E/E_k - 1 lies in [-0.07, 0.16] unless E is off the grid (clamped below)
  const float x0 = fmaf(E, V.inv_node[k], -1.0f);
  float fr = (x0 >= -0.16f && x0 <= 0.16f) ? log1p_small(x0) * kInvDl : log1pf(x0) * kInvDl;
  if (fr < 0.0f && k > 0) {
    --k;
    fr = log1pf(fmaf(E, V.inv_node[k], -1.0f)) * kInvDl;
  } else if (fr >= 1.0f && k < kGridN - 2) {
    ++k;
    fr = log1pf(fmaf(E, V.inv_node[k], -1.0f)) * kInvDl;
  }
  fr = fr < 0.0f ? 0.0f : (fr > 1.0f ? 1.0f : fr);
  i = k;
  f = fr;
}

template <typename R> __device__ __forceinline__ V4<R> lerp4(const V4<R> &a, const V4<R> &b, R f) {
  V4<R> o;
  o.x = a.x + f * (b.x - a.x);
  o.y = a.y + f * (b.y - a.y);
  o.z = a.z + f * (b.z - a.z);
  o.w = a.w + f * (b.w - a.w);
  return o;
}

template <typename R>
__device__ __forceinline__ V4<R> lookup_at(const View<R> &V, int mat, int type, int i, R f) {
  GV_CHECK(V.status, i >= 0 && i <= kGridN - 2 && mat >= 0 && mat < GV_MAX_MAT && type >= 0 && type <= 2);
  const V4<R> *t = V.xs + (mat * 3 + type) * kGridN;
  return lerp4(t[i], t[i + 1], f);
}

template <typename R> __device__ __forceinline__ V4<R> lookup(const View<R> &V, int mat, int type, R E) {
  int i;
  R f;
  grid_pos(V, E, i, f);
  return lookup_at(V, mat, type, i, f);
}

// The range table holds ln R (component z for e-, w for e+), interpolated
// linearly in ln E: within an interval R is a power of E, whose slope in
// ln E, E/S(E), follows the true one to the curvature of ln R.  (R itself
// linear in ln E gives every step in an interval the interval's mean
// slope: a stopping power off by up to +-3.6 % at 32 points per decade.)
template <typename R> __device__ __forceinline__ R lnrange_at(const V4<R> &v, int type) {
  return type == 1 ? v.z : v.w;
}

// Post-step energy after a continuous-loss step s (AlongStepAction): the
// exact inverse of the interpolated range.  Rv = R(E) = exp(interpolated
// ln R), as the step limit computed it.  While R(E) - s stays in E's own
// interval, ln E' = ln E + log1p(-s/R) / p with p the interval's slope of
// ln R in ln E -- free of the cancellation R(E) - s suffers for short steps
// in FP32; otherwise the interval of ln(R - s) is found among the nodes
// below (below the first node R is linear in E).
// (i, f) is E's grid position, as grid_pos returns it.
template <typename R> __device__ R eloss_at(const View<R> &V, int mat, int type, R E, int i, R f, R s, R Rv) {
  if (s >= Rv) return R(0);
  const V4<R> *t = V.xs + (mat * 3 + type) * kGridN;
  const R Li = lnrange_at(t[i], type), Lj = lnrange_at(t[i + 1], type);
  const R dL = Lj - Li;
  const R dl = static_cast<R>(2.302585092994046 / kGridPerDecade);
  const R x = m_log1p(-q_div(s, Rv));  // ln(r / R(E)) < 0
  if (-x <= f * dL) return E * m_exp(x * q_div(dl, dL));
  const R Lr = Li + f * dL + x;  // ln r
  const R L0 = lnrange_at(t[0], type);
  if (Lr < L0) return static_cast<R>(kGridEmin) * m_exp(Lr - L0);
  int j = i;
  R Ll = Li;
  while (j > 0 && Ll > Lr) {
    --j;
    Ll = lnrange_at(t[j], type);
  }
  const R Lh = lnrange_at(t[j + 1], type);
  return m_exp(static_cast<R>(-6.907755278982137) + dl * (static_cast<R>(j) + (Lr - Ll) / (Lh - Ll)));
}

// R(E) from the interpolated table row v (as lookup_at returns it)
template <typename R> __device__ __forceinline__ R range_of(const V4<R> &v, int type) {
  return m_exp(lnrange_at(v, type));
}

template <typename R> __device__ __forceinline__ R eloss(const View<R> &V, int mat, int type, R E, R s) {
  int i;
  R f;
  grid_pos(V, E, i, f);
  return eloss_at(V, mat, type, E, i, f, s, range_of(lookup_at(V, mat, type, i, f), type));
}

// ---------------------------------------------------------------- alias sampling
template <typename R> __device__ __forceinline__ R reduced_to_physical(int m, R E, R xi, R cut) {
  switch (m) {
    case kCompton: return m_exp((R(1) - xi) * -m_log1p(R(2) * E / static_cast<R>(kME)));
    case kPair: {
      const R a = static_cast<R>(kME) / E;
      return a + xi * (R(1) - R(2) * a);
    }
    case kBrem: return cut * m_exp(xi * m_log(q_div(E, cut)));
    case kMoller: {
      const R x = q_div(cut, E);
      return x * m_exp(xi * m_log(q_div(R(0.5), x)));
    }
    case kBhabha: {
      const R x = q_div(cut, E);
      return x * m_exp(-xi * m_log(x));
    }
    default: {  // softer annihilation photon, eps_min = 1/((g+1)(1+s)), s = sqrt((g-1)/(g+1))
      const R t = E / static_cast<R>(kME);
      const R s = m_sqrt(t / (t + R(2)));
      const R lo = R(1) / ((t + R(2)) * (R(1) + s));
      return lo * m_exp(xi * m_log(R(0.5) / lo));
    }
  }
}

// ---------------------------------------------------------------- rejection
// The random stream of an interacting step: counter (id_lo, id_hi, k, block)
// under key (key0, key1).
struct RngKey {
  uint32_t idlo, idhi, k, key0, key1;
};

// Rejection samplers, the alternative to sampling tables (Sec. 3.5): the
// proposal xi ~ U(0,1] is mapped like the tables' reduced variable (linear
// for pair, 1/k for brems, 1/eps for Compton) and accepted with the DCS in
// that variable over its bound (1, 4/3 and 2).  Trial j draws proposal and
// acceptance from words 2(j%2), 2(j%2)+1 of counter block 3 + j/2; after 64
// rejections the last proposal stands.  Out of line: inlined into the step
// kernels it would cost them registers whether or not rejection is chosen.
constexpr uint32_t kRejBlock0 = 3u;
constexpr int kRejMaxTrials = 64;

template <typename R>
__device__ __noinline__ R reject_sample(const View<R> &V, int m, R E, const RngKey &g, R *xi_out, int *trials = nullptr) {
  const R cut = V.rc.cut[m];
  const R ME = static_cast<R>(kME);
  R v = R(0), xi = R(0);
  uint4 w = make_uint4(0u, 0u, 0u, 0u);
  int j = 0;
  for (; j < kRejMaxTrials; ++j) {
    if ((j & 1) == 0) w = philox4x32_10(make_uint4(g.idlo, g.idhi, g.k, kRejBlock0 + (j >> 1)), g.key0, g.key1);
    xi = u24<R>((j & 1) ? w.z : w.x);
    const R ua = u24<R>((j & 1) ? w.w : w.y);
    v = reduced_to_physical<R>(m, E, xi, cut);
    R f;
    if (m == kPair) {
      f = R(1) - R(4.0 / 3.0) * v * (R(1) - v);
    } else if (m == kBrem) {
      const R y = v / (E + ME);
      f = (R(4.0 / 3.0) - R(4.0 / 3.0) * y + y * y) * R(0.75);
    } else {  // Compton, 1 - cos theta = (1 - eps)/(kappa eps)
      const R t = (R(1) - v) / (E / ME * v), s2 = t * (R(2) - t);
      f = R(0.5) * (R(1) + v * v - v * s2);
    }
    if (ua <= f) break;
  }
  if (trials) *trials = j < kRejMaxTrials ? j + 1 : kRejMaxTrials;
  *xi_out = xi;
  return v;
}

// u: grid choice, bin + alias, in-bin position
template <typename R>
__device__ R alias_sample(const View<R> &V, int m, R E, R ug, R ub, R ui, R *xi_out = nullptr) {
  const ModelMeta &M = V.meta[m];
  const R l = (m_log(E) - V.rc.ln_Elo[m]) * V.rc.inv_dl[m];
  int ie;
  if (l <= R(0)) ie = 0;
  else if (l >= static_cast<R>(M.nE - 1)) ie = M.nE - 1;
  else {
    const int i = static_cast<int>(m_floor(l));
    ie = (ug < l - static_cast<R>(i)) ? i + 1 : i;
  }
  const R x = ub * static_cast<R>(kNB);
  int j = static_cast<int>(x);
  j = j > kNB - 1 ? kNB - 1 : (j < 0 ? 0 : j);
  const R fr = x - static_cast<R>(j);
  GV_CHECK(V.status, ie >= 0 && ie < M.nE);
  const AliasBin<R> *row = V.bins + M.off + ie * kNB;
  AliasBin<R> b = row[j];
  int bin = j;
  if (!(fr < static_cast<R>(b.q))) {
    GV_CHECK(V.status, b.a >= 0 && b.a < kNB);
    bin = b.a;
    b = row[bin];
  }
  const R p0 = b.p0, p1 = b.p1;
  const R t = q_div(ui * (p0 + p1), p0 + m_sqrt(p0 * p0 + ui * (p1 * p1 - p0 * p0)));
  const R xi = (static_cast<R>(bin) + t) * static_cast<R>(1.0 / kNB);
  if (xi_out) *xi_out = xi;
  return reduced_to_physical<R>(m, E, xi, V.rc.cut[m]);
}

// ---------------------------------------------------------------- geometry
// An FP32 upper bound of |x| from the high word of the double (exponent
// and top 20 significand bits, one unit up), in integer arithmetic: no FP64
// instruction.  Inf where the exponent does not fit FP32.
__device__ __forceinline__ float abs_upper_f(double x) {
  const unsigned hi = static_cast<unsigned>(__double2hiint(x)) & 0x7fffffffu;
  const int e = static_cast<int>(hi >> 20) - 1023 + 127;
  if (e <= 0) return 1.17549435e-38f;  // |x| below the FP32 normal range
  if (e >= 255) return __int_as_float(0x7f800000);
  return __uint_as_float((static_cast<unsigned>(e) << 23) + (((hi & 0xfffffu) + 1u) << 3));
}

// Distance to the boundary of sub-slab `sub`: FP64 coordinate differences,
// divided in R.  next = -1 when the track leaves the box.  The plane is
// chosen before the subtraction, so a warp whose lanes move both ways still
// issues one FP64 difference per axis.
template <typename R>
__device__ __forceinline__ R distance(const View<R> &V, double x, double y, double z, R u, R v, R w, int sub,
                                      int &next, int &plane) {
  GV_CHECK(V.status, sub >= 0 && sub < V.geo.nsub);
  R d = r_inf<R>();
  int nx = sub, pl = -1;
  if (w != R(0)) {
    const int up = w > R(0) ? 1 : 0;
    pl = sub + up;
    nx = up ? sub + 1 : sub - 1;
    d = q_div(static_cast<R>(V.zb[pl] - z), w);
  }
  // A wall is at least h - |x| away along any direction: when that bound,
  // from integer arithmetic, clears the plane distance with margin, the wall
  // cannot be the nearest boundary and its FP64 difference is skipped (the
  // result is the one the full test would give).
  const float dz_f = static_cast<float>(d);
  if (V.geo.walls_x && u != R(0) && !(V.geo.hx_lo - abs_upper_f(x) > 1.001f * dz_f + 1e-4f)) {
    const R dx = q_div(static_cast<R>(V.geo.wx[u > R(0) ? 1 : 0] - x), u);
    if (dx < d) { d = dx; nx = -1; pl = -2; }
  }
  if (V.geo.walls_y && v != R(0) && !(V.geo.hy_lo - abs_upper_f(y) > 1.001f * dz_f + 1e-4f)) {
    const R dy = q_div(static_cast<R>(V.geo.wy[v > R(0) ? 1 : 0] - y), v);
    if (dy < d) { d = dy; nx = -1; pl = -3; }
  }
  if (d < R(0)) d = R(0);
  if (nx >= V.geo.nsub) nx = -1;
  next = nx;
  plane = pl;
  return d;
}

__device__ __forceinline__ int locate(const double *zb, int nsub, double z, double w) {
  if (z < 0.0 || z > zb[nsub]) return -1;
  int lo = 0, hi = nsub;  // zb[lo] <= z < zb[hi]
  if (z == zb[nsub]) return w < 0.0 ? nsub - 1 : -1;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (zb[mid] <= z) lo = mid; else hi = mid;
  }
  if (z == zb[lo] && w < 0.0) return lo - 1;
  return lo;
}

// ---------------------------------------------------------------- interactions
template <typename R> struct Kids {
  int n;
  int type[3];
  R E[3];
  R d[3][3];
};

template <typename R> __device__ __forceinline__ void add_kid(Kids<R> &k, int type, R E, const R d[3]) {
  // fixed-index stores keep the arrays in registers
  if (k.n == 0) {
    k.type[0] = type; k.E[0] = E; k.d[0][0] = d[0]; k.d[0][1] = d[1]; k.d[0][2] = d[2];
  } else if (k.n == 1) {
    k.type[1] = type; k.E[1] = E; k.d[1][0] = d[0]; k.d[1][1] = d[1]; k.d[1][2] = d[2];
  } else {
    k.type[2] = type; k.E[2] = E; k.d[2][0] = d[0]; k.d[2][1] = d[1]; k.d[2][2] = d[2];
  }
  k.n += 1;
}

// Rotate unit vector d to polar angle (ct, st) and azimuth (cp, sp) about
// itself (the frame of G4ThreeVector::rotateUz).  Callers pass st from a
// cancellation-free expression so small angles survive in FP32.
template <typename R>
__device__ __forceinline__ void rotate(const R d[3], R ct, R st, R cp, R sp, R o[3]) {
  const R lx = st * cp, ly = st * sp, lz = ct;
  R up = d[0] * d[0] + d[1] * d[1];
  if (up > R(0)) {
    const R iu = q_rsqrt(up);
    up = up * iu;
    o[0] = (d[0] * d[2] * lx - d[1] * ly) * iu + d[0] * lz;
    o[1] = (d[1] * d[2] * lx + d[0] * ly) * iu + d[1] * lz;
    o[2] = -up * lx + d[2] * lz;
  } else if (d[2] < R(0)) {
    o[0] = -lx; o[1] = ly; o[2] = -lz;
  } else {
    o[0] = lx; o[1] = ly; o[2] = lz;
  }
}

// direction at polar components (along, perp) -- not normalised -- and azimuth
template <typename R>
__device__ __forceinline__ void rotate_vec(const R d[3], R along, R perp, R cp, R sp, R o[3]) {
  const R n2 = along * along + perp * perp;
  if (!(n2 > R(0))) {
    o[0] = d[0]; o[1] = d[1]; o[2] = d[2];
    return;
  }
  const R inv = q_rsqrt(n2);
  rotate(d, along * inv, perp * inv, cp, sp, o);
}

// ---------------------------------------------------------------- magnetic field
// Uniform field along a coordinate axis b (field propagation, Sec. 3.6): a
// track of charge q and momentum p turns as dd/ds = q k (d x b), k = field_k
// / p.  With d = a + c0, a = (d.b) b, g = c0 x b and th = q k s, the exact
// helix moves the track by a s + c0 s sin(th)/th + g s (1 - cos th)/th and
// turns it to a + c0 cos th + g sin th; both quotients come from sin and cos
// of th/2, free of cancellation for small th.
constexpr double kFieldSagitta = 1e-3;  // cm
constexpr double kFieldMaxTurn = 0.2;   // rad

template <typename R> __device__ __forceinline__ R field_curv(const View<R> &V, int type, R E) {
  const R p = m_sqrt(E * (E + R(2) * static_cast<R>(kME)));
  return (type == 2 ? V.rc.field_k : -V.rc.field_k) / p;
}

// Step limit: chord sagitta <= 10 um and turn <= 0.2 rad of the helix
// (curvature |k| sin of the angle to the field).
template <typename R>
__device__ __forceinline__ R field_limit(const View<R> &V, int type, R E, R u, R v, R w) {
  if (type == 0 || V.rc.field_k == R(0)) return r_inf<R>();
  // sin^2 of the angle to the field from the two other components (no
  // cancellation when the track runs nearly along the field)
  const int ax = V.geo.field_axis;
  const R sa2 = ax == 0 ? v * v + w * w : (ax == 1 ? u * u + w * w : u * u + v * v);
  const R k = field_curv(V, type, E);
  const R keff = m_sqrt(sa2) * (k < R(0) ? -k : k);
  if (!(keff > R(0))) return r_inf<R>();
  const R a = m_sqrt(static_cast<R>(8.0 * kFieldSagitta) / keff), b = static_cast<R>(kFieldMaxTurn) / keff;
  return a < b ? a : b;
}

template <typename R>
__device__ __forceinline__ void helix(const View<R> &V, int type, R E, R s, const R d[3], R dp[3], R nd[3]) {
  const int ax = V.geo.field_axis;
  const R db = d[ax];
  R a[3] = {R(0), R(0), R(0)};
  a[ax] = db;
  const R c0[3] = {d[0] - a[0], d[1] - a[1], d[2] - a[2]};
  // g = c0 x b for b the unit vector of axis ax
  R g[3];
  if (ax == 0) { g[0] = R(0); g[1] = c0[2]; g[2] = -c0[1]; }
  else if (ax == 1) { g[0] = -c0[2]; g[1] = R(0); g[2] = c0[0]; }
  else { g[0] = c0[1]; g[1] = -c0[0]; g[2] = R(0); }
  const R th = field_curv(V, type, E) * s;
  R sh, ch;
  m_sincos(R(0.5) * th, &sh, &ch);
  const R sn = R(2) * sh * ch, cs = R(1) - R(2) * sh * sh;
  const R sc = th != R(0) ? sn / th : R(1), cc = th != R(0) ? R(2) * sh * sh / th : R(0);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    dp[j] = a[j] * s + c0[j] * (s * sc) + g[j] * (s * cc);
    nd[j] = a[j] + c0[j] * cs + g[j] * sn;
  }
}

// ---------------------------------------------------------------- multiple scattering
// Gaussian multiple scattering over a charged step of length s (the MSC
// stages of Sec. 2.1.2; optional process GV_P_MSC).  Width: the Highland
// formula at the step's mean kinetic energy, with its bracket floored at 0,
//   th0 = 13.6 MeV / (beta p c) sqrt(s/X0) (1 + 0.038 ln(s / (X0 beta^2))).
// Four uniforms give four normals by Box-Muller; per transverse plane of the
// rotation frame the angle is th0 z_a and the lateral offset
// s th0 (z_b / sqrt(12) + z_a / 2), the correlated joint Gaussian of the
// small-angle theory.  The direction turns by |(theta_x, theta_y)| (at most
// pi) towards (theta_x, theta_y); the end point moves by the offset,
// shortened to 0.99 of the safety (distance to the nearest boundary of
// sub-slab `sub`, from FP64 differences) when longer.
template <typename R>
__device__ __forceinline__ void msc_step(const View<R> &V, int sub, R E_pre, R E_post, R s, R d[3], double &x,
                                         double &y, double &z, const R u[4]) {
  const R ME = static_cast<R>(kME);
  const R T = R(0.5) * (E_pre + E_post);
  const R pc = m_sqrt(T * (T + R(2) * ME));
  const R beta = pc / (T + ME);
  const R xr = s * V.rc.inv_X0[V.smat[sub]];
  const R corr = R(1) + R(0.038) * m_log(xr / (beta * beta));
  const R th0 = corr > R(0) ? R(13.6) / (beta * pc) * m_sqrt(xr) * corr : R(0);
  if (!(th0 > R(0))) return;
  const R r1 = m_sqrt(R(-2) * m_log(u[0])), r2 = m_sqrt(R(-2) * m_log(u[2]));
  R s1, c1, s2, c2;
  m_sincos(static_cast<R>(2.0 * kPi) * u[1], &s1, &c1);
  m_sincos(static_cast<R>(2.0 * kPi) * u[3], &s2, &c2);
  const R z1 = r1 * c1, z2 = r1 * s1, z3 = r2 * c2, z4 = r2 * s2;
  const R tx = th0 * z1, ty = th0 * z2;
  const R k12 = static_cast<R>(0.28867513459481287);  // 1/sqrt(12)
  const R ox = s * th0 * (z3 * k12 + z1 * R(0.5));
  const R oy = s * th0 * (z4 * k12 + z2 * R(0.5));
  // the frame of rotate(): e1, e2 perpendicular to d
  R e1[3], e2[3];
  const R up = m_sqrt(d[0] * d[0] + d[1] * d[1]);
  if (up > R(0)) {
    e1[0] = d[0] * d[2] / up; e1[1] = d[1] * d[2] / up; e1[2] = -up;
    e2[0] = -d[1] / up; e2[1] = d[0] / up; e2[2] = R(0);
  } else {
    e1[0] = d[2] < R(0) ? R(-1) : R(1); e1[1] = R(0); e1[2] = R(0);
    e2[0] = R(0); e2[1] = R(1); e2[2] = R(0);
  }
  // offset, limited by the safety of the pre-move end point
  const R len = m_sqrt(ox * ox + oy * oy);
  double sf = z - V.zb[sub];
  const double sz2 = V.zb[sub + 1] - z;
  sf = sz2 < sf ? sz2 : sf;
  if (V.geo.walls_x) {
    const double sx = V.geo.hx - fabs(x);
    sf = sx < sf ? sx : sf;
  }
  if (V.geo.walls_y) {
    const double sy = V.geo.hy - fabs(y);
    sf = sy < sf ? sy : sf;
  }
  const R safe = sf > 0.0 ? static_cast<R>(sf) : R(0);
  const R scale = (len > R(0.99) * safe) ? (len > R(0) ? R(0.99) * safe / len : R(0)) : R(1);
  x += f2d(scale * (ox * e1[0] + oy * e2[0]));
  y += f2d(scale * (ox * e1[1] + oy * e2[1]));
  z += f2d(scale * (ox * e1[2] + oy * e2[2]));
  // direction
  R th = m_sqrt(tx * tx + ty * ty);
  if (!(th > R(0))) return;
  const R cp = tx / th, sp = ty / th;
  const R PI = static_cast<R>(kPi);
  th = th > PI ? PI : th;
  R st, ct;
  m_sincos(th, &st, &ct);
  const R dn[3] = {st * (cp * e1[0] + sp * e2[0]) + ct * d[0], st * (cp * e1[1] + sp * e2[1]) + ct * d[1],
                   st * (cp * e1[2] + sp * e2[2]) + ct * d[2]};
  d[0] = dn[0];
  d[1] = dn[1];
  d[2] = dn[2];
}

template <typename R> __device__ __forceinline__ void at_rest(Kids<R> &k, R u6, R u7) {
  const R ct = R(2) * u6 - R(1);
  const R st = R(2) * m_sqrt(u6 * (R(1) - u6));
  R sp, cp;
  m_sincos(static_cast<R>(2.0 * kPi) * u7, &sp, &cp);
  const R a[3] = {st * cp, st * sp, ct};
  const R b[3] = {-a[0], -a[1], -a[2]};
  add_kid(k, 0, static_cast<R>(kME), a);
  add_kid(k, 0, static_cast<R>(kME), b);
}

// Final state (PostStepActions) of process p.  u[2..7]: grid, bin, in-bin,
// azimuth, isotropic pair.  Returns 1 survives, 0 ended, -1 not possible.
// The reduced variable of every alias-sampled model is drawn by one call
// site, so a warp whose lanes run different processes samples together and
// diverges only for the kinematics.  Angles use forms of 1 -+ cos(theta)
// without cancellation, written from the sampled xi; they are algebraically
// the textbook two-body kinematics.
template <typename R, bool REJECT = true>
__device__ int interact(const View<R> &V, int type, int p, R &E, R d[3], const R *u, const RngKey &g, Kids<R> &kids,
                        R &local, int &npair, int &nann) {
  const R ME = static_cast<R>(kME);
  const R ecut_push = V.rc.ecut_push;
  const R tcut = V.rc.tcut;
  const R ec = V.rc.ecut;
  local = R(0);
  // which model, and is it open at this energy?
  int model;
  if (type == 0) {
    if (p == 1) model = -1;  // photoelectric: nothing to sample
    else if (p == 0) model = kCompton;
    else {
      if (!(E > R(2) * ME)) return -1;
      model = kPair;
    }
  } else if (p == 0) {
    if (!(E > V.rc.gcut)) return -1;
    model = kBrem;
  } else if (p == 1) {
    if (!(E > (type == 1 ? R(2) * ec : ec))) return -1;
    model = type == 1 ? kMoller : kBhabha;
  } else {
    model = kAnnih;
  }
  R xi = R(0), v = R(0);
  if (model >= 0)
    v = (REJECT && model <= kBrem && E >= V.rc.rej_min[model]) ? reject_sample<R>(V, model, E, g, &xi)
                                                       : alias_sample<R>(V, model, E, u[2], u[3], u[4], &xi);
  R sp, cp;
  m_sincos(static_cast<R>(2.0 * kPi) * u[5], &sp, &cp);
  if (model == kCompton) {  // eps = eps0^(1-xi)
    const R k = E, kap = k * static_cast<R>(1.0 / kME);
    const R L0 = -m_log1p(R(2) * kap);
    const R a = (R(1) - xi) * L0;
    const R eps = m_exp(a);
    const R om_eps = -m_expm1(a);                   // 1 - eps
    const R ike = q_div(R(1), kap * eps);
    const R omc = om_eps * ike;                // 1 - cos(theta)
    const R opc = m_expm1(-xi * L0) * ike;     // 1 + cos(theta)
    const R st = m_sqrt(omc * opc);
    const R ct = omc < R(1) ? R(1) - omc : opc - R(1);
    R d1[3], de[3];
    rotate(d, ct, st, cp, sp, d1);
    const R k1 = eps * k, Te = k * om_eps;
    // electron momentum k d - k' d' = k [(1 - eps ct) d - eps st e_phi]
    rotate_vec(d, om_eps + eps * omc, eps * st, -cp, -sp, de);
    if (Te >= ecut_push) add_kid(kids, 1, Te, de);
    else local += Te;
    d[0] = d1[0]; d[1] = d1[1]; d[2] = d1[2];
    if (k1 < tcut) { local += k1; E = R(0); return 0; }
    E = k1;
    return 1;
  }
  if (model < 0) {  // photoelectric: the electron takes k along the photon
    if (E >= ecut_push) add_kid(kids, 1, E, d);
    else local += E;
    E = R(0);
    return 0;
  }
  if (model == kPair) {
    const R k = E;
    R Tm = v * k - ME, Tp = (R(1) - v) * k - ME;
    Tm = Tm < R(0) ? R(0) : Tm;
    Tp = Tp < R(0) ? R(0) : Tp;
    R st, ct;
    m_sincos(q_div(ME, k), &st, &ct);
    R dm[3], dp[3];
    rotate(d, ct, st, cp, sp, dm);
    rotate(d, ct, st, -cp, -sp, dp);
    npair += 1;
    if (Tm >= ecut_push) add_kid(kids, 1, Tm, dm);
    else local += Tm;
    if (Tp >= ecut_push) add_kid(kids, 2, Tp, dp);
    else {
      local += Tp;
      at_rest(kids, u[6], u[7]);
      nann += 1;
    }
    E = R(0);
    return 0;
  }
  R T = E;
  if (model == kBrem) {
    R st, ct, dg[3];
    m_sincos(q_div(ME, T + ME), &st, &ct);
    rotate(d, ct, st, cp, sp, dg);
    if (v >= tcut) add_kid(kids, 0, v, dg);
    else local += v;
    T -= v;
  } else if (model != kAnnih) {  // ionisation: Moller eps = xc (1/(2xc))^xi, Bhabha eps = xc^(1-xi)
    const R eps = v;
    const R om_eps = model == kMoller ? R(1) - eps : -m_expm1((R(1) - xi) * m_log(q_div(ec, T)));
    const R Td = eps * T;
    const R den = eps * T + R(2) * ME;
    // delta ray: cos^2 = eps (T + 2m) / (eps T + 2m), sin^2 = 2m (1 - eps) / (eps T + 2m)
    const R iden = q_div(R(1), den);
    const R ct = m_sqrt(eps * (T + R(2) * ME) * iden), st = m_sqrt(R(2) * ME * om_eps * iden);
    R dd[3], dn[3];
    rotate(d, ct, st, cp, sp, dd);
    // primary: p' = p (1 - eps) along d, sqrt(2 m T eps (1 - eps)) across
    const R P = m_sqrt(T * (T + R(2) * ME));
    rotate_vec(d, P * om_eps, m_sqrt(R(2) * ME * T * eps * om_eps), -cp, -sp, dn);
    add_kid(kids, 1, Td, dd);
    d[0] = dn[0]; d[1] = dn[1]; d[2] = dn[2];
    T = T * om_eps;
  } else {  // annihilation in flight: softer photon eps = eps_min (1/(2 eps_min))^xi
    const R t = T / ME;
    const R s = m_sqrt(t / (t + R(2)));
    const R emin = R(1) / ((t + R(2)) * (R(1) + s));
    const R Lr = m_log(R(0.5) / emin);
    const R eps = emin * m_exp(xi * Lr);
    const R D = emin * m_expm1(xi * Lr);  // eps - eps_min
    const R W = T + R(2) * ME, P = m_sqrt(T * (T + R(2) * ME)), Q = W + P;
    const R k1 = eps * W, k2 = (R(1) - eps) * W;
    // photon 1: 1 - cos = m (W (1 - 2 eps) + P) / (eps P Q), 1 + cos = D Q / (eps P)
    const R omc1 = ME * (W * (R(1) - R(2) * eps) + P) / (eps * P * Q);
    const R opc1 = D * Q / (eps * P);
    // photon 2: 1 - cos = 2 m W D / ((1 - eps) P Q), 1 + cos = (s - D) Q / ((1 - eps) P)
    const R omc2 = R(2) * ME * W * D / ((R(1) - eps) * P * Q);
    const R opc2 = (s - D) * Q / ((R(1) - eps) * P);
    R d1[3], d2[3];
    rotate(d, omc1 < R(1) ? R(1) - omc1 : opc1 - R(1), m_sqrt(omc1 * opc1), cp, sp, d1);
    rotate(d, omc2 < R(1) ? R(1) - omc2 : opc2 - R(1), m_sqrt(omc2 * opc2), -cp, -sp, d2);
    add_kid(kids, 0, k1, d1);
    add_kid(kids, 0, k2, d2);
    nann += 1;
    E = R(0);
    return 0;
  }
  if (T < tcut) {
    local += T;
    E = R(0);
    if (type == 2) {
      at_rest(kids, u[6], u[7]);
      nann += 1;
    }
    return 0;
  }
  E = T;
  return 1;
}

}  // namespace gv
