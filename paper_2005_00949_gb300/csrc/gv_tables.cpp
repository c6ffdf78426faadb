// gv_tables.cpp -- host-side FP64 construction of the per-material tables the
// stepping loop reads: macroscopic cross sections of every discrete process,
// restricted-loss ranges, and the alias sampling tables of the final-state
// models ("sampling tables", GeantV Sec. 3.5).  The tables play the role of
// the ComputeIntLen / Spline::GetValueAt lookups of Sec. 2.1.2 and Sec. 6.3.
//
// Physics (the paper defers it to an external EM paper):
//   Compton: free-electron Klein-Nishina.
//   Photoelectric: K-shell (Sauter/Heitler) absorption x 5/4 for all shells.
//   Pair production and bremsstrahlung: complete-screening Tsai forms, with
//     the Tsai radiation length (Coulomb-corrected).
//   Ionisation: Moller (e-) / Bhabha (e+) above the cut, Berger-Seltzer
//     (ICRU 37) restricted collision loss below, density effect from the
//     plasma energy.
//   Annihilation in flight: Heitler two-photon cross section.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "gv_internal.h"

namespace gv {
namespace {

struct Medium {
  double rho = 0, I = 0;        // g/cm3, MeV
  double n_el = 0;              // electrons per cm3
  double inv_X0_cm = 0;         // 1/X0 in 1/cm
  double hw_plasma = 0;         // MeV
  int n_el_kinds = 0;
  double Z[GV_MAX_ELEM]{}, atoms[GV_MAX_ELEM]{};  // atoms per cm3
};

// Radiation logarithms of Tsai; light elements take his tabulated values.
void radiation_logs(double Z, double &L1, double &L2) {
  static const double tab[4][2] = {{5.31, 6.144}, {4.79, 5.621}, {4.74, 5.805}, {4.71, 5.924}};
  for (int k = 1; k <= 4; ++k)
    if (Z == double(k)) {
      L1 = tab[k - 1][0];
      L2 = tab[k - 1][1];
      return;
    }
  L1 = std::log(184.15 / std::cbrt(Z));
  L2 = std::log(1194.0 / std::cbrt(Z * Z));
}

double coulomb_correction(double Z) {
  const double a = kAlpha * Z, a2 = a * a;
  return a2 * (1.0 / (1.0 + a2) + 0.20206 + a2 * (-0.0369 + a2 * (0.0083 - 0.002 * a2)));
}

Medium make_medium(const gv_material &m) {
  Medium md;
  md.rho = m.rho;
  md.I = m.I_eV * 1e-6;
  md.n_el_kinds = m.n_elem;
  double inv_X0_g = 0.0;  // cm2/g
  for (int e = 0; e < m.n_elem; ++e) {
    const double Z = m.Z[e], A = m.A[e];
    md.Z[e] = Z;
    md.atoms[e] = kNA * m.rho * m.w[e] / A;
    md.n_el += Z * md.atoms[e];
    double L1, L2;
    radiation_logs(Z, L1, L2);
    inv_X0_g += m.w[e] * 4.0 * kAlpha * kRE * kRE * kNA / A *
                (Z * Z * (L1 - coulomb_correction(Z)) + Z * L2);
  }
  md.inv_X0_cm = inv_X0_g * m.rho;
  md.hw_plasma = kME / kAlpha * std::sqrt(4.0 * kPi * md.n_el * kRE * kRE * kRE);
  return md;
}

// ---- photons ---------------------------------------------------------------
// The closed form cancels to ~1e-8 relative at k ~ 1 keV in FP64, so it is
// evaluated in long double (>= 64-bit mantissa) and rounded once.
double sigma_compton_per_electron(double k) {
  using L = long double;
  const L x = static_cast<L>(k) / static_cast<L>(kME), l = std::log1p(2.0L * x), d = 1.0L + 2.0L * x;
  const L a = (1.0L + x) / (x * x) * (2.0L * (1.0L + x) / d - l / x);
  const L b = 0.5L * l / x - (1.0L + 3.0L * x) / (d * d);
  return static_cast<double>(2.0L * static_cast<L>(kPi) * static_cast<L>(kRE) * static_cast<L>(kRE) * (a + b));
}

double sigma_photo_per_atom(double Z, double k) {
  const double thomson = 8.0 * kPi / 3.0 * kRE * kRE;
  const double a2 = kAlpha * kAlpha;
  const double r = kME / k;
  return 1.25 * 4.0 * std::sqrt(2.0) * a2 * a2 * std::pow(Z, 5) * thomson * r * r * r * std::sqrt(r);
}

// integral over x of [1 - 4/3 x (1-x)], x in [m/k, 1 - m/k]
double pair_integral(double k) {
  if (k <= 2.0 * kME) return 0.0;
  auto F = [](double x) { return x - 2.0 / 3.0 * x * x + 4.0 / 9.0 * x * x * x; };
  const double lo = kME / k;
  return F(1.0 - lo) - F(lo);
}

// ---- charged -----------------------------------------------------------------
// integral over k in (kc, T] of (4/3 - 4/3 y + y^2)/k, y = k/(T+m)
double brem_integral(double T, double kc) {
  if (!(T > kc)) return 0.0;
  const double E = T + kME;
  auto G = [E](double k) { return 4.0 / 3.0 * std::log(k) - 4.0 / 3.0 * k / E + 0.5 * k * k / (E * E); };
  return G(T) - G(kc);
}

double sigma_moller_per_electron(double T, double Tc) {
  if (!(T > 2.0 * Tc)) return 0.0;
  const double g = 1.0 + T / kME, g2 = g * g, beta2 = 1.0 - 1.0 / g2;
  const double c1 = (g - 1.0) * (g - 1.0) / g2, c2 = (2.0 * g - 1.0) / g2;
  const double x = Tc / T;
  // integral over eps in [x, 1/2] of c1 + 1/e^2 - c2/e + 1/(1-e)^2 - c2/(1-e)
  const double I = c1 * (0.5 - x) + (1.0 / x - 2.0) + (2.0 - 1.0 / (1.0 - x)) -
                   c2 * (std::log(0.5 / x) + std::log(2.0 * (1.0 - x)));
  return 2.0 * kPi * kRE * kRE / (beta2 * (g - 1.0)) * I;
}

void bhabha_b(double g, double b[4]) {
  const double y = 1.0 / (g + 1.0), t = 1.0 - 2.0 * y, t2 = t * t;
  b[0] = 2.0 - y * y;
  b[1] = t * (3.0 + y * y);
  b[3] = t2 * t;
  b[2] = t2 + b[3];
}

double sigma_bhabha_per_electron(double T, double Tc) {
  if (!(T > Tc)) return 0.0;
  const double g = 1.0 + T / kME, beta2 = 1.0 - 1.0 / (g * g);
  double b[4];
  bhabha_b(g, b);
  const double x = Tc / T;
  // integral over eps in [x, 1] of 1/(beta2 e^2) - B1/e + B2 - B3 e + B4 e^2
  const double I = (1.0 / x - 1.0) / beta2 + b[0] * std::log(x) + b[1] * (1.0 - x) -
                   0.5 * b[2] * (1.0 - x * x) + b[3] * (1.0 - x * x * x) / 3.0;
  return 2.0 * kPi * kRE * kRE / (g - 1.0) * I;
}

double sigma_annih_per_electron(double T) {
  const double g = 1.0 + T / kME, s = std::sqrt((g - 1.0) * (g + 1.0));
  return kPi * kRE * kRE / (g + 1.0) *
         ((g * g + 4.0 * g + 1.0) / (s * s) * std::log(g + s) - (g + 3.0) / s);
}

// Berger-Seltzer restricted collision stopping power, MeV/cm
double dedx_collision(const Medium &md, bool positron, double T, double Tc) {
  const double tau = T / kME, g = tau + 1.0, g2 = g * g, beta2 = 1.0 - 1.0 / g2;
  double F;
  if (positron) {
    const double d = std::min(Tc, T) / kME, y = 1.0 / (g + 1.0);
    const double poly = tau + 2.0 * d - 1.5 * d * d * y - (d - d * d * d / 3.0) * y * y -
                        (0.5 * d * d - tau * d * d * d / 3.0 + 0.25 * d * d * d * d) * y * y * y;
    F = std::log(tau * d) - beta2 / tau * poly;
  } else {
    const double d = std::min(Tc, 0.5 * T) / kME;
    F = -1.0 - beta2 + std::log((tau - d) * d) + tau / (tau - d) +
        (0.5 * d * d + (2.0 * tau + 1.0) * std::log1p(-d / tau)) / g2;
  }
  const double bg2 = tau * (tau + 2.0);
  double delta = std::log(bg2) + 2.0 * std::log(md.hw_plasma / md.I) - 1.0;
  if (delta < 0.0) delta = 0.0;
  const double Im = md.I / kME;
  return 2.0 * kPi * kRE * kRE * kME * md.n_el / beta2 *
         (std::log(2.0 * (tau + 2.0) / (Im * Im)) + F - delta);
}

double dedx_radiative(const Medium &md, double T, double kc) {
  const double E = T + kME, y = std::min(kc, T) / E;
  return md.inv_X0_cm * E * y * (4.0 / 3.0 - y * (2.0 / 3.0 - y / 3.0));
}

double dedx_total(const Medium &md, bool positron, double T, const gv_cuts &c) {
  return dedx_collision(md, positron, T, c.e_cut_MeV) + dedx_radiative(md, T, c.gamma_cut_MeV);
}

// ---- quadrature: 20-point Gauss-Legendre, nodes by Newton on P_20 ---------
struct GL20 {
  double x[20], w[20];
  GL20() {
    const int n = 20;
    for (int i = 0; i < n; ++i) {
      double z = std::cos(kPi * (i + 0.75) / (n + 0.5)), dp = 1.0;
      for (int it = 0; it < 60; ++it) {
        double p0 = 1.0, p1 = z;
        for (int j = 2; j <= n; ++j) {
          const double p2 = ((2 * j - 1) * z * p1 - (j - 1) * p0) / j;
          p0 = p1;
          p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        const double step = p1 / dp;
        z -= step;
        if (std::fabs(step) < 1e-15) break;
      }
      x[i] = z;
      w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
  }
};

// integral of dT / S(T) over [a, b], in ln T, split where S has kinks
double path_length(const Medium &md, bool positron, double a, double b, const gv_cuts &c,
                   const GL20 &gl) {
  std::vector<double> br{a, b};
  const double bg = std::exp(0.5) * md.I / md.hw_plasma;  // density-effect onset
  const double kinks[3] = {positron ? c.e_cut_MeV : 2.0 * c.e_cut_MeV, c.gamma_cut_MeV,
                           kME * (std::sqrt(1.0 + bg * bg) - 1.0)};
  for (double k : kinks)
    if (k > a && k < b) br.push_back(k);
  std::sort(br.begin(), br.end());
  double sum = 0.0;
  for (size_t s = 0; s + 1 < br.size(); ++s) {
    const double u0 = std::log(br[s]), u1 = std::log(br[s + 1]);
    const double h = 0.5 * (u1 - u0), m = 0.5 * (u1 + u0);
    for (int i = 0; i < 20; ++i) {
      const double T = std::exp(m + h * gl.x[i]);
      sum += gl.w[i] * h * T / dedx_total(md, positron, T, c);
    }
  }
  return sum;
}

double grid_energy(int i) { return std::exp(std::log(kGridEmin) + i * std::log(10.0) / kGridPerDecade); }

// ---- alias tables -------------------------------------------------------------
double model_low_edge(int m, const gv_cuts &c) {
  switch (m) {
    case kCompton: return 1e-3;
    case kPair: return 1.25;
    case kBrem: return c.gamma_cut_MeV;
    case kMoller: return 2.0 * c.e_cut_MeV;
    case kBhabha: return c.e_cut_MeV;
    default: return 1e-3;
  }
}

double model_cut(int m, const gv_cuts &c) {
  if (m == kBrem) return c.gamma_cut_MeV;
  if (m == kMoller || m == kBhabha) return c.e_cut_MeV;
  return 0.0;
}

// physical variable at reduced xi (see the device twin in gv_device.cuh)
double reduced_to_physical(int m, double E, double xi, double cut) {
  switch (m) {
    case kCompton: return std::exp((1.0 - xi) * -std::log1p(2.0 * E / kME));
    case kPair: { const double a = kME / E; return a + xi * (1.0 - 2.0 * a); }
    case kBrem: return cut * std::exp(xi * std::log(E / cut));
    case kMoller: { const double x = cut / E; return x * std::exp(xi * std::log(0.5 / x)); }
    case kBhabha: { const double x = cut / E; return x * std::exp(-xi * std::log(x)); }
    default: {
      const double g = 1.0 + E / kME, lo = 0.5 * (1.0 - std::sqrt((g - 1.0) / (g + 1.0)));
      return lo * std::exp(xi * std::log(0.5 / lo));
    }
  }
}

// density of the reduced variable (differential cross section times the
// Jacobian of the map, constant factors dropped)
double reduced_density(int m, double E, double xi, double cut) {
  const double v = reduced_to_physical(m, E, xi, cut);
  switch (m) {
    case kCompton: {  // eps (1/eps + eps - sin^2 theta)
      const double t = (1.0 - v) * kME / (E * v);
      return 1.0 + v * v - v * t * (2.0 - t);
    }
    case kPair: return 1.0 - 4.0 / 3.0 * v * (1.0 - v);
    case kBrem: { const double y = v / (E + kME); return 4.0 / 3.0 - 4.0 / 3.0 * y + y * y; }
    case kMoller: {
      const double g = 1.0 + E / kME, g2 = g * g;
      const double c1 = (g - 1.0) * (g - 1.0) / g2, c2 = (2.0 * g - 1.0) / g2;
      const double w = 1.0 - v;
      return v * (c1 + (1.0 / v - c2) / v + (1.0 / w - c2) / w);
    }
    case kBhabha: {
      const double g = 1.0 + E / kME, beta2 = 1.0 - 1.0 / (g * g);
      double b[4];
      bhabha_b(g, b);
      return 1.0 / (beta2 * v) - b[0] + v * (b[1] + v * (-b[2] + v * b[3]));
    }
    default: {
      const double g = 1.0 + E / kME, A = (g + 1.0) * (g + 1.0), B = g * g + 4.0 * g + 1.0;
      auto S = [A, B](double e) { return -A + B / e - 1.0 / (e * e); };
      return v * (S(v) + S(1.0 - v));
    }
  }
}

// Vose's construction of a Walker alias table: indices go on the small/large
// stacks in ascending order and are taken from the top; residuals in FP64.
void make_alias(const double *node_pdf, float *q_out, int *alias_out) {
  double mass[kNB], total = 0.0;
  for (int j = 0; j < kNB; ++j) {
    mass[j] = 0.5 * (node_pdf[j] + node_pdf[j + 1]);
    total += mass[j];
  }
  std::vector<int> small, large;
  double prob[kNB], q[kNB];
  for (int j = 0; j < kNB; ++j) {
    prob[j] = mass[j] * kNB / total;
    q[j] = 1.0;
    alias_out[j] = j;
    (prob[j] < 1.0 ? small : large).push_back(j);
  }
  while (!small.empty() && !large.empty()) {
    const int s = small.back(), l = large.back();
    small.pop_back();
    large.pop_back();
    q[s] = prob[s];
    alias_out[s] = l;
    prob[l] = (prob[l] + prob[s]) - 1.0;
    (prob[l] < 1.0 ? small : large).push_back(l);
  }
  for (int j = 0; j < kNB; ++j) q_out[j] = static_cast<float>(q[j]);
}

}  // namespace

int build_host_tables(const gv_material *mats, int n_mats, const gv_cuts &cuts, HostTables *out,
                      std::string *err) {
  GL20 gl;
  out->n_mat = n_mats;
  out->xs.assign(static_cast<size_t>(n_mats) * 3 * kGridN * 4, 0.0);
  out->smax.assign(static_cast<size_t>(n_mats) * 2 * kGridN, 0.0);
  const unsigned pm = cuts.process_mask;
  for (int m = 0; m < n_mats; ++m) {
    const Medium md = make_medium(mats[m]);
    out->inv_X0_cm[m] = md.inv_X0_cm;
    auto at = [&](int type, int i, int q) -> double & {
      return out->xs[((static_cast<size_t>(m) * 3 + type) * kGridN + i) * 4 + q];
    };
    const double brem_scale = md.inv_X0_cm;
    for (int i = 0; i < kGridN; ++i) {
      const double E = grid_energy(i);
      if (pm & GV_P_COMPTON) at(0, i, 0) = md.n_el * sigma_compton_per_electron(E);
      if (pm & GV_P_PHOTO) {
        double s = 0.0;
        for (int e = 0; e < md.n_el_kinds; ++e) s += md.atoms[e] * sigma_photo_per_atom(md.Z[e], E);
        at(0, i, 1) = s;
      }
      if (pm & GV_P_PAIR) at(0, i, 2) = md.inv_X0_cm * pair_integral(E);
      if (pm & GV_P_BREM) {
        at(1, i, 0) = brem_scale * brem_integral(E, cuts.gamma_cut_MeV);
        at(2, i, 0) = at(1, i, 0);
      }
      if (pm & GV_P_IONI) {
        at(1, i, 1) = md.n_el * sigma_moller_per_electron(E, cuts.e_cut_MeV);
        at(2, i, 1) = md.n_el * sigma_bhabha_per_electron(E, cuts.e_cut_MeV);
      }
      if (pm & GV_P_ANNIH) at(2, i, 2) = md.n_el * sigma_annih_per_electron(E);
    }
    for (int pos = 0; pos < 2; ++pos) {
      const int type = 1 + pos, q = pos ? 3 : 2;
      double R = kGridEmin / dedx_total(md, pos, kGridEmin, cuts);
      if (!(R > 0.0) || !std::isfinite(R)) {
        if (err) *err = "non-positive stopping power at the bottom of the grid";
        return GV_ERR_BAD_ARG;
      }
      at(type, 0, q) = R;
      for (int i = 1; i < kGridN; ++i) {
        const double S = dedx_total(md, pos, grid_energy(i), cuts);
        if (!(S > 0.0)) {
          if (err) *err = "non-positive stopping power on the grid";
          return GV_ERR_BAD_ARG;
        }
        R += path_length(md, pos, grid_energy(i - 1), grid_energy(i), cuts, gl);
        at(type, i, q) = R;
      }
      double run = 0.0;  // the bound of the integral approach
      for (int i = 0; i < kGridN; ++i) {
        const double sig = at(type, i, 0) + at(type, i, 1) + (pos ? at(type, i, 2) : 0.0);
        run = std::max(run, sig);
        out->smax[(static_cast<size_t>(m) * 2 + pos) * kGridN + i] = run;
      }
    }
  }
  for (int m = 0; m < kNModel; ++m) {
    const double lo = model_low_edge(m, cuts), cut = model_cut(m, cuts);
    out->a_Elo[m] = lo;
    out->a_cut[m] = cut;
    int nE = 1;
    if (lo < kAliasEmax) nE += static_cast<int>(std::ceil(kAliasPerDecade * std::log10(kAliasEmax / lo) - 1e-6));
    out->a_nE[m] = nE;
    out->a_pdf[m].assign(static_cast<size_t>(nE) * (kNB + 1), 0.0);
    out->a_q[m].assign(static_cast<size_t>(nE) * kNB, 1.0f);
    out->a_alias[m].assign(static_cast<size_t>(nE) * kNB, 0);
    for (int ie = 0; ie < nE; ++ie) {
      const double E = lo * std::pow(10.0, static_cast<double>(ie) / kAliasPerDecade);
      double *pdf = &out->a_pdf[m][static_cast<size_t>(ie) * (kNB + 1)];
      for (int j = 0; j <= kNB; ++j) pdf[j] = reduced_density(m, E, static_cast<double>(j) / kNB, cut);
      make_alias(pdf, &out->a_q[m][static_cast<size_t>(ie) * kNB], &out->a_alias[m][static_cast<size_t>(ie) * kNB]);
    }
  }
  return GV_OK;
}

}  // namespace gv
