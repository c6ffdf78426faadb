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

template <typename R> __device__ __forceinline__ R r_inf();
template <> __device__ __forceinline__ float r_inf<float>() { return __int_as_float(0x7f800000); }
template <> __device__ __forceinline__ double r_inf<double>() { return __longlong_as_double(0x7ff0000000000000ll); }

template <typename R> struct alignas(4 * sizeof(R)) V4 { R x, y, z, w; };

// one bin of an alias table: acceptance q, alias index, pdf at the bin edges
template <typename R> struct AliasBin { float q; int a; R p0, p1; };

struct ModelMeta {
  double ln_Elo, inv_dl, cut;
  int nE, off;
};

struct GeoConst {
  int nsub, nsub_layer, n_layers, nx, ny;
  double hx, hy, pitch_x, pitch_y;
};

struct CutConst {
  double gcut, ecut, tcut;
  unsigned mask;
};

// Read-only view of everything one step needs.
template <typename R> struct View {
  const V4<R> *xs;           // [(mat*3 + type)*kGridN + node], smem or global
  const double *zb;          // nsub+1 planes
  const unsigned char *smat; // material of each sub-slab
  const AliasBin<R> *bins;   // all models, [off + ie*kNB + j]
  ModelMeta meta[kNModel];
  GeoConst geo;
  CutConst cut;
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
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// uniform in (0, 1], exact in FP32 and FP64
template <typename R> __device__ __forceinline__ R u24(uint32_t x) {
  return static_cast<R>((x >> 8) + 1u) * static_cast<R>(1.0 / 16777216.0);
}

// ---------------------------------------------------------------- tables
template <typename R> __device__ __forceinline__ void grid_pos(R E, int &i, R &f) {
  const R l = (m_log(E) - static_cast<R>(-6.907755278982137)) * static_cast<R>(kGridPerDecade / 2.302585092994046);
  int k = static_cast<int>(m_floor(l));
  k = k < 0 ? 0 : (k > kGridN - 2 ? kGridN - 2 : k);
  R fr = l - static_cast<R>(k);
  fr = fr < R(0) ? R(0) : (fr > R(1) ? R(1) : fr);
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

template <typename R> __device__ __forceinline__ V4<R> lookup(const View<R> &V, int mat, int type, R E) {
  int i;
  R f;
  grid_pos(E, i, f);
  const V4<R> *t = V.xs + (mat * 3 + type) * kGridN;
  return lerp4(t[i], t[i + 1], f);
}

// range is component z (e-) or w (e+)
template <typename R> __device__ __forceinline__ R range_at(const V4<R> &v, int type) {
  return type == 1 ? v.z : v.w;
}

// Post-step energy after a continuous-loss step s (AlongStepAction): the
// exact inverse of the range interpolated linearly in ln E.  While R(E) - s
// stays in E's own interval the inverse is E exp(-dl s / (R_{i+1} - R_i)),
// free of the cancellation R(E) - s suffers for short steps in FP32.
template <typename R> __device__ R eloss(const View<R> &V, int mat, int type, R E, R s) {
  const V4<R> *t = V.xs + (mat * 3 + type) * kGridN;
  int i;
  R f;
  grid_pos(E, i, f);
  const R Ri = range_at(t[i], type), Rj = range_at(t[i + 1], type);
  const R dR = Rj - Ri;
  const R Rv = Ri + f * dR;
  if (s >= Rv) return R(0);
  const R dl = static_cast<R>(2.302585092994046 / kGridPerDecade);
  if (s <= f * dR) return E * m_exp(-dl * s / dR);
  const R r = Rv - s;
  const R R0 = range_at(t[0], type);
  if (r < R0) return static_cast<R>(kGridEmin) * r / R0;
  int j = i;
  R Rl = Ri;
  while (j > 0 && Rl > r) {
    --j;
    Rl = range_at(t[j], type);
  }
  const R Rh = range_at(t[j + 1], type);
  return m_exp(static_cast<R>(-6.907755278982137) + dl * (static_cast<R>(j) + (r - Rl) / (Rh - Rl)));
}

// ---------------------------------------------------------------- alias sampling
template <typename R> __device__ __forceinline__ R reduced_to_physical(int m, R E, R xi, R cut) {
  switch (m) {
    case kCompton: return m_exp((R(1) - xi) * -m_log1p(R(2) * E / static_cast<R>(kME)));
    case kPair: {
      const R a = static_cast<R>(kME) / E;
      return a + xi * (R(1) - R(2) * a);
    }
    case kBrem: return cut * m_exp(xi * m_log(E / cut));
    case kMoller: {
      const R x = cut / E;
      return x * m_exp(xi * m_log(R(0.5) / x));
    }
    case kBhabha: {
      const R x = cut / E;
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

// u: grid choice, bin + alias, in-bin position
template <typename R>
__device__ R alias_sample(const View<R> &V, int m, R E, R ug, R ub, R ui, R *xi_out = nullptr) {
  const ModelMeta &M = V.meta[m];
  const R l = (m_log(E) - static_cast<R>(M.ln_Elo)) * static_cast<R>(M.inv_dl);
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
  const AliasBin<R> *row = V.bins + M.off + ie * kNB;
  AliasBin<R> b = row[j];
  int bin = j;
  if (!(fr < static_cast<R>(b.q))) {
    bin = b.a;
    b = row[bin];
  }
  const R p0 = b.p0, p1 = b.p1;
  const R t = ui * (p0 + p1) / (p0 + m_sqrt(p0 * p0 + ui * (p1 * p1 - p0 * p0)));
  const R xi = (static_cast<R>(bin) + t) * static_cast<R>(1.0 / kNB);
  if (xi_out) *xi_out = xi;
  return reduced_to_physical<R>(m, E, xi, static_cast<R>(M.cut));
}

// ---------------------------------------------------------------- geometry
// Distance to the boundary of sub-slab `sub`: FP64 coordinate differences,
// divided in R.  next = -1 when the track leaves the box.
template <typename R>
__device__ __forceinline__ R distance(const View<R> &V, double x, double y, double z, R u, R v, R w, int sub,
                                      int &next, int &plane) {
  R d = r_inf<R>();
  int nx = sub, pl = -1;
  if (w > R(0)) {
    d = static_cast<R>(V.zb[sub + 1] - z) / w;
    nx = sub + 1;
    pl = sub + 1;
  } else if (w < R(0)) {
    d = static_cast<R>(V.zb[sub] - z) / w;
    nx = sub - 1;
    pl = sub;
  }
  if (V.geo.hx > 0.0) {
    R dx = r_inf<R>();
    if (u > R(0)) dx = static_cast<R>(V.geo.hx - x) / u;
    else if (u < R(0)) dx = static_cast<R>(-V.geo.hx - x) / u;
    if (dx < d) { d = dx; nx = -1; pl = -2; }
  }
  if (V.geo.hy > 0.0) {
    R dy = r_inf<R>();
    if (v > R(0)) dy = static_cast<R>(V.geo.hy - y) / v;
    else if (v < R(0)) dy = static_cast<R>(-V.geo.hy - y) / v;
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

template <typename R> __device__ __forceinline__ void add_kid(Kids<R> &k, int type, R E, R a, R b, R c) {
  const int n = k.n;
  k.type[n] = type;
  k.E[n] = E;
  k.d[n][0] = a;
  k.d[n][1] = b;
  k.d[n][2] = c;
  k.n = n + 1;
}

// rotate unit vector d by polar cosine ct and azimuth phi about itself
template <typename R> __device__ __forceinline__ void rotate(const R d[3], R ct, R phi, R o[3]) {
  R st = R(1) - ct * ct;
  st = st > R(0) ? m_sqrt(st) : R(0);
  R sp, cp;
  m_sincos(phi, &sp, &cp);
  const R lx = st * cp, ly = st * sp, lz = ct;
  R up = d[0] * d[0] + d[1] * d[1];
  if (up > R(0)) {
    up = m_sqrt(up);
    o[0] = (d[0] * d[2] * lx - d[1] * ly) / up + d[0] * lz;
    o[1] = (d[1] * d[2] * lx + d[0] * ly) / up + d[1] * lz;
    o[2] = -up * lx + d[2] * lz;
  } else if (d[2] < R(0)) {
    o[0] = -lx; o[1] = ly; o[2] = -lz;
  } else {
    o[0] = lx; o[1] = ly; o[2] = lz;
  }
}

template <typename R> __device__ __forceinline__ void unit_or(R a, R b, R c, const R fb[3], R o[3]) {
  const R n2 = a * a + b * b + c * c;
  if (n2 > R(0)) {
    const R n = m_sqrt(n2);
    o[0] = a / n; o[1] = b / n; o[2] = c / n;
  } else {
    o[0] = fb[0]; o[1] = fb[1]; o[2] = fb[2];
  }
}

template <typename R> __device__ __forceinline__ void at_rest(Kids<R> &k, R u6, R u7) {
  const R ct = R(2) * u6 - R(1);
  R st = R(1) - ct * ct;
  st = st > R(0) ? m_sqrt(st) : R(0);
  R sp, cp;
  m_sincos(static_cast<R>(2.0 * kPi) * u7, &sp, &cp);
  add_kid(k, 0, static_cast<R>(kME), st * cp, st * sp, ct);
  add_kid(k, 0, static_cast<R>(kME), -(st * cp), -(st * sp), -ct);
}

// Final state (PostStepActions) of process p.  u[2..7]: grid, bin, in-bin,
// azimuth, isotropic pair.  Returns 1 survives, 0 ended, -1 not possible.
template <typename R>
__device__ int interact(const View<R> &V, int type, int p, R &E, R d[3], const R *u, Kids<R> &kids, R &local,
                        int &npair, int &nann) {
  const R ME = static_cast<R>(kME);
  const R ecut_push = static_cast<R>(V.cut.ecut > V.cut.tcut ? V.cut.ecut : V.cut.tcut);
  const R tcut = static_cast<R>(V.cut.tcut);
  const R phi = static_cast<R>(2.0 * kPi) * u[5];
  local = R(0);
  if (type == 0) {
    const R k = E;
    if (p == 0) {  // Compton
      const R eps = alias_sample<R>(V, kCompton, k, u[2], u[3], u[4]);
      R ct = R(1) - (R(1) - eps) * ME / (k * eps);
      ct = ct < R(-1) ? R(-1) : (ct > R(1) ? R(1) : ct);
      R d1[3];
      rotate(d, ct, phi, d1);
      const R k1 = eps * k, Te = k - k1;
      R de[3];
      unit_or(k * d[0] - k1 * d1[0], k * d[1] - k1 * d1[1], k * d[2] - k1 * d1[2], d, de);
      if (Te >= ecut_push) add_kid(kids, 1, Te, de[0], de[1], de[2]);
      else local += Te;
      d[0] = d1[0]; d[1] = d1[1]; d[2] = d1[2];
      if (k1 < tcut) { local += k1; E = R(0); return 0; }
      E = k1;
      return 1;
    }
    if (p == 1) {  // photoelectric
      if (k >= ecut_push) add_kid(kids, 1, k, d[0], d[1], d[2]);
      else local += k;
      E = R(0);
      return 0;
    }
    if (!(k > R(2) * ME)) return -1;  // pair
    const R x = alias_sample<R>(V, kPair, k, u[2], u[3], u[4]);
    R Tm = x * k - ME, Tp = (R(1) - x) * k - ME;
    Tm = Tm < R(0) ? R(0) : Tm;
    Tp = Tp < R(0) ? R(0) : Tp;
    const R ct = m_cos(ME / k);
    R dm[3], dp[3];
    rotate(d, ct, phi, dm);
    rotate(d, ct, phi + static_cast<R>(kPi), dp);
    npair += 1;
    if (Tm >= ecut_push) add_kid(kids, 1, Tm, dm[0], dm[1], dm[2]);
    else local += Tm;
    if (Tp >= ecut_push) add_kid(kids, 2, Tp, dp[0], dp[1], dp[2]);
    else {
      local += Tp;
      at_rest(kids, u[6], u[7]);
      nann += 1;
    }
    E = R(0);
    return 0;
  }
  R T = E;
  if (p == 0) {  // bremsstrahlung
    if (!(T > static_cast<R>(V.cut.gcut))) return -1;
    const R kg = alias_sample<R>(V, kBrem, T, u[2], u[3], u[4]);
    R dg[3];
    rotate(d, m_cos(ME / (T + ME)), phi, dg);
    if (kg >= tcut) add_kid(kids, 0, kg, dg[0], dg[1], dg[2]);
    else local += kg;
    T -= kg;
  } else if (p == 1) {  // ionisation
    const R ec = static_cast<R>(V.cut.ecut);
    if (type == 1 && !(T > R(2) * ec)) return -1;
    if (type == 2 && !(T > ec)) return -1;
    const R eps = alias_sample<R>(V, type == 1 ? kMoller : kBhabha, T, u[2], u[3], u[4]);
    const R Td = eps * T;
    R ct = m_sqrt(Td * (T + R(2) * ME) / (T * (Td + R(2) * ME)));
    ct = ct > R(1) ? R(1) : ct;
    R dd[3];
    rotate(d, ct, phi, dd);
    const R P = m_sqrt(T * (T + R(2) * ME)), Pd = m_sqrt(Td * (Td + R(2) * ME));
    R dn[3];
    unit_or(P * d[0] - Pd * dd[0], P * d[1] - Pd * dd[1], P * d[2] - Pd * dd[2], d, dn);
    add_kid(kids, 1, Td, dd[0], dd[1], dd[2]);
    d[0] = dn[0]; d[1] = dn[1]; d[2] = dn[2];
    T -= Td;
  } else {  // annihilation in flight
    const R eps = alias_sample<R>(V, kAnnih, T, u[2], u[3], u[4]);
    const R tot = T + R(2) * ME, k1 = eps * tot, k2 = tot - k1;
    const R P = m_sqrt(T * (T + R(2) * ME));
    R ct = (k1 - ME) / (eps * P);
    ct = ct < R(-1) ? R(-1) : (ct > R(1) ? R(1) : ct);
    R d1[3], d2[3];
    rotate(d, ct, phi, d1);
    unit_or(P * d[0] - k1 * d1[0], P * d[1] - k1 * d1[1], P * d[2] - k1 * d1[2], d, d2);
    add_kid(kids, 0, k1, d1[0], d1[1], d1[2]);
    add_kid(kids, 0, k2, d2[0], d2[1], d2[2]);
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
