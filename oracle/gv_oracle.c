/*
 * gv_oracle.c -- plain FP64 CPU oracle of EM shower transport (GeantV,
 * arXiv:2005.00949).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the CPU
 * baseline leg of the benchmark.  The product library never includes, links
 * or calls it, and it shares no code with the CUDA path.
 *
 * Everything is FP64, in the order the stepping stages of Sec. 2.1.2 name
 * them.  Two transports share the stepping loop:
 *  - tabulated (default), the paper's method: cross sections interpolated
 *    linearly, and ranges as ln R, in ln E between table nodes that hold the
 *    exact quantities at the nodes of the logarithmic energy grid (the tables the
 *    paper's profiles show as Spline::GetValueAt / G4PhysicsVector, Sec.
 *    6.3); final states from sampling tables (Sec. 3.5: the alias method with
 *    a discrete intermediate variable), or by rejection where chosen;
 *  - untabulated (or_setup.exact): cross sections from their formulas at the
 *    track's own energy, the range by quadrature of 1/S from the grid node
 *    below, the post-step energy as the root of int_{E'}^{E} dE/S = s
 *    (Newton on the quadrature, bracketed), and every final state by
 *    rejection from its differential cross section.  It measures what the
 *    tables cost.
 *
 * Parity status of each function is stated beside it; "pinned" means a test
 * in tests/test_oracle_pins.py checks it against something other than itself.
 */
#include "gv_oracle.h"
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* physical constants (CODATA 2018) */
#define ME 0.51099895             /* electron mass, MeV */
#define RE 2.8179403262e-13       /* classical electron radius, cm */
#define ALPHA (1.0 / 137.035999084)
#define NAVOG 6.02214076e23
#define PI 3.14159265358979323846

/* energy grid of the cross-section / range tables: 1 keV .. 1 TeV */
#define GRID_EMIN 1e-3
#define GRID_PPD 32
#define GRID_N (9 * GRID_PPD + 1)

/* alias sampling tables */
#define ALIAS_PPD 8
#define ALIAS_NB 64
#define ALIAS_EMAX 1e6
#define ALIAS_MAXE 80

/* charged-particle step limit and continuous-loss constants */
#define STEP_ALPHA_R 0.2
#define STEP_RHO_F 0.1

#define TAG_ID 0x80000000u

/* ------------------------------------------------------------------ */
/* data                                                                */
/* ------------------------------------------------------------------ */
typedef struct {
  or_material m;
  double nel;        /* electrons / cm3 */
  double nat[OR_MAX_ELEM];
  double X0g;        /* radiation length g/cm2 */
  double I;          /* MeV */
  double plasma;     /* hbar omega_p, MeV */
} omat;

typedef struct {
  double E_lo;
  int nE;
  double pdf[ALIAS_MAXE][ALIAS_NB + 1];
  float q[ALIAS_MAXE][ALIAS_NB];
  int a[ALIAS_MAXE][ALIAS_NB];
} oalias;

struct or_ctx {
  or_setup s;
  omat mat[OR_MAX_MAT];
  int nsub;             /* total number of sub-slabs */
  double *zb;           /* nsub+1 planes */
  int *smat;            /* material of each sub-slab */
  /* tables[type][q][mat][node] */
  double tab[3][4][OR_MAX_MAT][GRID_N];
  /* integral approach: running maximum over the nodes below of the total
   * cross section of e- (0) and e+ (1) */
  double smax[2][OR_MAX_MAT][GRID_N];
  oalias alias[OR_NMODEL];
  double gl_x[16], gl_w[16];
  /* untabulated mode: the range gained across each grid interval, and the
   * energies where S(E) has a kink, per charged type (0 e-, 1 e+) */
  double dR[2][OR_MAX_MAT][GRID_N];
  double kink[2][OR_MAX_MAT][3];
  double gl6_x[6], gl6_w[6];
};

/* ------------------------------------------------------------------ */
/* Gauss-Legendre nodes by Newton iteration on P_n (textbook method)   */
/* ------------------------------------------------------------------ */
static void gauss_legendre(int n, double *x, double *w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(PI * (i + 0.75) / (n + 0.5)), pp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p1 = 1.0, p2 = 0.0;
      for (int j = 1; j <= n; ++j) {
        double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
      }
      pp = n * (z * p1 - p2) / (z * z - 1.0);
      double dz = p1 / pp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
  }
}

/* ------------------------------------------------------------------ */
/* materials: electron density, radiation length (Tsai), plasma energy */
/* ------------------------------------------------------------------ */
/* Tsai radiation logarithms: Z<=4 from Tsai's table, else the formula.
 * Pinned: PDG radiation lengths of H, C, Si, W, Pb. */
static void tsai_logs(double Z, double *Lrad, double *Lprad) {
  if (Z == 1.0) { *Lrad = 5.31; *Lprad = 6.144; }
  else if (Z == 2.0) { *Lrad = 4.79; *Lprad = 5.621; }
  else if (Z == 3.0) { *Lrad = 4.74; *Lprad = 5.805; }
  else if (Z == 4.0) { *Lrad = 4.71; *Lprad = 5.924; }
  else { *Lrad = log(184.15 * pow(Z, -1.0 / 3.0)); *Lprad = log(1194.0 * pow(Z, -2.0 / 3.0)); }
}

static double coulomb_f(double Z) {
  double a2 = (ALPHA * Z) * (ALPHA * Z);
  return a2 * (1.0 / (1.0 + a2) + 0.20206 - 0.0369 * a2 + 0.0083 * a2 * a2 - 0.002 * a2 * a2 * a2);
}

static void mat_init(omat *o, const or_material *m) {
  o->m = *m;
  o->nel = 0.0;
  double invX0 = 0.0;
  for (int i = 0; i < m->n_elem; ++i) {
    double Z = m->Z[i], A = m->A[i];
    o->nat[i] = m->rho * NAVOG * m->w[i] / A;
    o->nel += o->nat[i] * Z;
    double Lr, Lp;
    tsai_logs(Z, &Lr, &Lp);
    double inv = 4.0 * ALPHA * RE * RE * (NAVOG / A) * (Z * Z * (Lr - coulomb_f(Z)) + Z * Lp);
    invX0 += m->w[i] * inv;
  }
  o->X0g = 1.0 / invX0;
  o->I = m->I_eV * 1e-6;
  o->plasma = ME * sqrt(4.0 * PI * o->nel * RE * RE * RE) / ALPHA;
}

/* ------------------------------------------------------------------ */
/* photon cross sections                                               */
/* ------------------------------------------------------------------ */
/* Klein-Nishina total per electron.  Pinned: Thomson limit expansion,
 * high-energy limit, quadrature of the KN DCS, NIST incoherent value.
 * The closed form cancels (~1e-8 relative at 1 keV in FP64), so it is summed
 * in long double and rounded once. */
double or_klein_nishina_e(double k) {
  long double K = (long double)k / ME;
  long double l = logl(1.0L + 2.0L * K);
  long double t1 = (1.0L + K) / (K * K) * (2.0L * (1.0L + K) / (1.0L + 2.0L * K) - l / K);
  long double t2 = l / (2.0L * K);
  long double t3 = (1.0L + 3.0L * K) / ((1.0L + 2.0L * K) * (1.0L + 2.0L * K));
  return (double)(2.0L * PI * RE * RE * (t1 + t2 - t3));
}

/* Sauter-type K-shell photoabsorption x 5/4 for all shells, per atom.
 * Pinned: the Born limit of Stobbe's exact K-shell cross section (whose
 * normalisation is pinned by the hydrogen threshold value), and the size in
 * water against Hubbell & Seltzer's mu_en/rho at 10-20 keV. */
static double photo_atom(double Z, double k) {
  double sT = 8.0 * PI * RE * RE / 3.0;
  double a4 = ALPHA * ALPHA * ALPHA * ALPHA;
  return 1.25 * 4.0 * sqrt(2.0) * a4 * pow(Z, 5.0) * sT * pow(ME / k, 3.5);
}

/* complete-screening pair production: integral of 1 - 4/3 x(1-x) over the
 * kinematic range [m/k, 1-m/k].  Pinned: 7/9 high-energy limit, DCS quadrature. */
static double pair_shape_integral(double k) {
  if (k <= 2.0 * ME) return 0.0;
  double a = ME / k, b = 1.0 - a;
  return (b - a) - 2.0 / 3.0 * (b * b - a * a) + 4.0 / 9.0 * (b * b * b - a * a * a);
}

/* ------------------------------------------------------------------ */
/* charged-particle cross sections and restricted stopping powers      */
/* ------------------------------------------------------------------ */
/* discrete bremsstrahlung k in (kc, T], complete screening, per X0 unit */
static double brem_shape_integral(double T, double kc) {
  if (T <= kc) return 0.0;
  double E = T + ME;
  return 4.0 / 3.0 * log(T / kc) - 4.0 / 3.0 * (T - kc) / E + (T * T - kc * kc) / (2.0 * E * E);
}

/* Moller, per electron, delta rays in (Tc, T/2] */
static double moller_e(double T, double Tc) {
  if (T <= 2.0 * Tc) return 0.0;
  double g = T / ME + 1.0, b2 = 1.0 - 1.0 / (g * g);
  double xc = Tc / T;
  double C1 = ((g - 1.0) / g) * ((g - 1.0) / g), C2 = (2.0 * g - 1.0) / (g * g);
  double br = C1 * (0.5 - xc) + 1.0 / xc - 1.0 / (1.0 - xc) - C2 * log((1.0 - xc) / xc);
  return 2.0 * PI * RE * RE / (b2 * (g - 1.0)) * br;
}

static void bhabha_coef(double g, double *B1, double *B2, double *B3, double *B4) {
  double y = 1.0 / (1.0 + g), t = 1.0 - 2.0 * y;
  *B1 = 2.0 - y * y;
  *B2 = t * (3.0 + y * y);
  *B4 = t * t * t;
  *B3 = *B4 + t * t;
}

/* Bhabha, per electron, delta rays in (Tc, T] */
static double bhabha_e(double T, double Tc) {
  if (T <= Tc) return 0.0;
  double g = T / ME + 1.0, b2 = 1.0 - 1.0 / (g * g);
  double xc = Tc / T, B1, B2, B3, B4;
  bhabha_coef(g, &B1, &B2, &B3, &B4);
  double br = (1.0 / b2) * (1.0 / xc - 1.0) - B1 * log(1.0 / xc) + B2 * (1.0 - xc)
            - B3 * (1.0 - xc * xc) / 2.0 + B4 * (1.0 - xc * xc * xc) / 3.0;
  return 2.0 * PI * RE * RE / (g - 1.0) * br;
}

/* Heitler two-photon annihilation in flight, per electron.
 * Pinned: quadrature of the Heitler DCS over the kinematic range. */
static double annih_e(double T) {
  double g = T / ME + 1.0, q = sqrt(g * g - 1.0);
  return PI * RE * RE / (g + 1.0) * ((g * g + 4.0 * g + 1.0) / (g * g - 1.0) * log(g + q) - (g + 3.0) / q);
}

static double density_effect(const omat *o, double T) {
  double tau = T / ME, bg = sqrt(tau * (tau + 2.0));
  double d = 2.0 * log(bg) + 2.0 * log(o->plasma / o->I) - 1.0;
  return d > 0.0 ? d : 0.0;
}

/* Restricted collision stopping power (Berger-Seltzer, ICRU 37) with cut
 * Tc.  Pinned: ESTAR values for water (e-); both branches equal the
 * unrestricted ICRU 37 formulas (F+ and F-) once the cut is above the
 * largest transfer; the derivative w.r.t. the cut equals Tc x the Moller /
 * Bhabha DCS. */
static double dedx_col(const omat *o, int positron, double T, double Tc) {
  double tau = T / ME, g = tau + 1.0, b2 = 1.0 - 1.0 / (g * g);
  double Im = o->I / ME;
  double F;
  if (!positron) {
    double D = fmin(Tc, 0.5 * T) / ME;
    F = -1.0 - b2 + log((tau - D) * D) + tau / (tau - D)
      + (0.5 * D * D + (2.0 * tau + 1.0) * log(1.0 - D / tau)) / (g * g);
  } else {
    double D = fmin(Tc, T) / ME, y = 1.0 / (g + 1.0);
    double D2 = D * D, D3 = D2 * D, D4 = D3 * D;
    F = log(tau * D) - b2 / tau * (tau + 2.0 * D - 1.5 * D2 * y - (D - D3 / 3.0) * y * y
                                   - (0.5 * D2 - tau * D3 / 3.0 + 0.25 * D4) * y * y * y);
  }
  double br = log(2.0 * (tau + 2.0) / (Im * Im)) + F - density_effect(o, T);
  return 2.0 * PI * RE * RE * ME * o->nel / b2 * br;
}

/* restricted radiative loss, photons below kc (complete screening).
 * Pinned: equals E/X0 at y_c = 1 and the quadrature of k dsigma/dk. */
static double dedx_rad(const omat *o, double T, double kc) {
  double E = T + ME, yc = fmin(kc, T) / E;
  return o->m.rho / o->X0g * E * (4.0 / 3.0 * yc - 2.0 / 3.0 * yc * yc + yc * yc * yc / 3.0);
}

/* ------------------------------------------------------------------ */
/* public exact physics                                                */
/* ------------------------------------------------------------------ */
double or_material_X0(const or_ctx *c, int mat) { return c->mat[mat].X0g; }
double or_material_nel(const or_ctx *c, int mat) { return c->mat[mat].nel; }

static double xs_exact(const or_ctx *c, int type, int p, int mat, double E) {
  const omat *o = &c->mat[mat];
  const or_setup *s = &c->s;
  if (type == OR_GAMMA) {
    if (p == 0) return o->nel * or_klein_nishina_e(E);
    if (p == 1) {
      double sum = 0.0;
      for (int i = 0; i < o->m.n_elem; ++i) sum += o->nat[i] * photo_atom(o->m.Z[i], E);
      return sum;
    }
    if (p == 2) return o->m.rho / o->X0g * pair_shape_integral(E);
    return 0.0;
  }
  if (p == 0) return o->m.rho / o->X0g * brem_shape_integral(E, s->gamma_cut);
  if (type == OR_ELECTRON) {
    if (p == 1) return o->nel * moller_e(E, s->e_cut);
    return 0.0;
  }
  if (p == 1) return o->nel * bhabha_e(E, s->e_cut);
  if (p == 2) return o->nel * annih_e(E);
  return 0.0;
}

static unsigned proc_bit(int type, int p) {
  static const unsigned b[3][3] = {{OR_P_COMPTON, OR_P_PHOTO, OR_P_PAIR},
                                   {OR_P_BREM, OR_P_IONI, 0},
                                   {OR_P_BREM, OR_P_IONI, OR_P_ANNIH}};
  return b[type][p];
}

static int n_proc(int type) { return type == OR_ELECTRON ? 2 : 3; }

double or_xs(const or_ctx *c, int type, int p, int mat, double E) {
  if (p < 0 || p >= n_proc(type)) return 0.0;
  if (!(c->s.process_mask & proc_bit(type, p))) return 0.0;
  return xs_exact(c, type, p, mat, E);
}

double or_dedx_parts(const or_ctx *c, int type, int mat, double E, double cut_e, double cut_g,
                     double *col, double *rad) {
  const omat *o = &c->mat[mat];
  *col = dedx_col(o, type == OR_POSITRON, E, cut_e);
  *rad = dedx_rad(o, E, cut_g);
  return *col + *rad;
}

double or_dedx(const or_ctx *c, int type, int mat, double E) {
  double a, b;
  return or_dedx_parts(c, type, mat, E, c->s.e_cut, c->s.gamma_cut, &a, &b);
}

/* integral of dE/S over [a,b], split at the kinks of S, Gauss-Legendre in ln E */
static double inv_dedx_integral(const or_ctx *c, int type, int mat, double a, double b) {
  double cuts[8];
  int nc = 0;
  cuts[nc++] = a;
  const omat *o = &c->mat[mat];
  double kinks[3];
  kinks[0] = type == OR_POSITRON ? c->s.e_cut : 2.0 * c->s.e_cut;
  kinks[1] = c->s.gamma_cut;
  double bg = exp(0.5 - log(o->plasma / o->I));
  kinks[2] = ME * (sqrt(1.0 + bg * bg) - 1.0);
  /* sort kinks */
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j)
      if (kinks[j] < kinks[i]) { double t = kinks[i]; kinks[i] = kinks[j]; kinks[j] = t; }
  for (int i = 0; i < 3; ++i)
    if (kinks[i] > a && kinks[i] < b) cuts[nc++] = kinks[i];
  cuts[nc++] = b;
  double sum = 0.0;
  for (int k = 0; k + 1 < nc; ++k) {
    double la = log(cuts[k]), lb = log(cuts[k + 1]);
    double h = 0.5 * (lb - la), mid = 0.5 * (la + lb);
    for (int i = 0; i < 16; ++i) {
      double E = exp(mid + h * c->gl_x[i]);
      sum += h * c->gl_w[i] * E / or_dedx(c, type, mat, E);
    }
  }
  return sum;
}

double or_grid_energy(int i) { return exp(log(GRID_EMIN) + i * (log(10.0) / GRID_PPD)); }
int or_grid_size(void) { return GRID_N; }

/* Range from the bottom of the grid: R(E) = Emin/S(Emin) + int_{Emin}^{E} dE/S */
double or_range_exact(const or_ctx *c, int type, int mat, double E) {
  double R = GRID_EMIN / or_dedx(c, type, mat, GRID_EMIN);
  if (E <= GRID_EMIN) return E / GRID_EMIN * R;
  int i = 0;
  while (i + 1 < GRID_N && or_grid_energy(i + 1) <= E) {
    R += inv_dedx_integral(c, type, mat, or_grid_energy(i), or_grid_energy(i + 1));
    ++i;
  }
  if (E > or_grid_energy(i)) R += inv_dedx_integral(c, type, mat, or_grid_energy(i), E);
  return R;
}

/* ------------------------------------------------------------------ */
/* differential cross sections (shapes), used to pin alias tables       */
/* ------------------------------------------------------------------ */
/* returns dsigma/dvar up to a constant, in the physical variable:
 *  COMPTON: var = eps = k'/k            PAIR: var = x = E-_tot/k
 *  BREM:    var = k (photon energy)     MOLLER/BHABHA: var = eps = T_delta/T
 *  ANNIH:   var = eps = k1/(T+2m)       (cut: gamma cut for BREM, e cut for ioni) */
double or_dcs(int model, double E, double v, double cut) {
  (void)cut;
  switch (model) {
  case OR_M_COMPTON: {
    double K = E / ME, t = (1.0 - v) / (K * v), s2 = t * (2.0 - t);
    return 1.0 / v + v - s2;
  }
  case OR_M_PAIR: return 1.0 - 4.0 / 3.0 * v * (1.0 - v);
  case OR_M_BREM: {
    double y = v / (E + ME);
    return (4.0 / 3.0 - 4.0 / 3.0 * y + y * y) / v;
  }
  case OR_M_MOLLER: {
    double g = E / ME + 1.0;
    double C1 = ((g - 1.0) / g) * ((g - 1.0) / g), C2 = (2.0 * g - 1.0) / (g * g);
    return C1 + 1.0 / v * (1.0 / v - C2) + 1.0 / (1.0 - v) * (1.0 / (1.0 - v) - C2);
  }
  case OR_M_BHABHA: {
    double g = E / ME + 1.0, b2 = 1.0 - 1.0 / (g * g), B1, B2, B3, B4;
    bhabha_coef(g, &B1, &B2, &B3, &B4);
    return 1.0 / (b2 * v * v) - B1 / v + B2 - B3 * v + B4 * v * v;
  }
  case OR_M_ANNIH: {
    double g = E / ME + 1.0;
    double a = (g + 1.0) * (g + 1.0), b = g * g + 4.0 * g + 1.0;
    double S1 = -a + b / v - 1.0 / (v * v);
    double w = 1.0 - v;
    double S2 = -a + b / w - 1.0 / (w * w);
    return S1 + S2;
  }
  }
  return 0.0;
}

/* ------------------------------------------------------------------ */
/* alias tables: reduced variable xi in [0,1], pdf tabulated at 65 nodes */
/* ------------------------------------------------------------------ */
static double model_cut(const or_ctx *c, int model) {
  if (model == OR_M_BREM) return c->s.gamma_cut;
  if (model == OR_M_MOLLER || model == OR_M_BHABHA) return c->s.e_cut;
  return 0.0;
}

static double model_Elo(const or_ctx *c, int model) {
  switch (model) {
  case OR_M_COMPTON: return 1e-3;
  case OR_M_PAIR: return 1.25;
  case OR_M_BREM: return c->s.gamma_cut;
  case OR_M_MOLLER: return 2.0 * c->s.e_cut;
  case OR_M_BHABHA: return c->s.e_cut;
  case OR_M_ANNIH: return 1e-3;
  }
  return 1.0;
}

/* physical variable from the reduced variable at energy E */
static double xi_to_var(int model, double E, double xi, double cut) {
  switch (model) {
  case OR_M_COMPTON: {
    double e0 = 1.0 / (1.0 + 2.0 * E / ME);
    return exp((1.0 - xi) * log(e0));
  }
  case OR_M_PAIR: {
    double x0 = ME / E;
    return x0 + xi * (1.0 - 2.0 * x0);
  }
  case OR_M_BREM: return cut * exp(xi * log(E / cut));
  case OR_M_MOLLER: {
    double xc = cut / E;
    return xc * exp(xi * log(0.5 / xc));
  }
  case OR_M_BHABHA: {
    double xc = cut / E;
    return xc * exp(xi * log(1.0 / xc));
  }
  case OR_M_ANNIH: {
    double g = E / ME + 1.0, s = sqrt((g - 1.0) / (g + 1.0)), emin = 0.5 * (1.0 - s);
    return emin * exp(xi * log(0.5 / emin));
  }
  }
  return 0.0;
}

/* pdf of the reduced variable (DCS x Jacobian, constants dropped) */
static double reduced_pdf(int model, double E, double xi, double cut) {
  double v = xi_to_var(model, E, xi, cut);
  switch (model) {
  case OR_M_COMPTON: {
    double K = E / ME, t = (1.0 - v) / (K * v);
    return 1.0 + v * v - v * t * (2.0 - t);
  }
  case OR_M_PAIR: return 1.0 - 4.0 / 3.0 * v * (1.0 - v);
  case OR_M_BREM: {
    double y = v / (E + ME);
    return 4.0 / 3.0 - 4.0 / 3.0 * y + y * y;
  }
  case OR_M_MOLLER: case OR_M_BHABHA: case OR_M_ANNIH:
    return v * or_dcs(model, E, v, cut);
  }
  return 0.0;
}

/* Walker alias table by Vose's two-stack procedure (exact procedure in the
 * design notes: ascending pushes, pop from the top, FP64 residuals). */
static void build_alias_row(const double *pdf, float *q, int *a) {
  double w[ALIAS_NB], p[ALIAS_NB], W = 0.0;
  for (int j = 0; j < ALIAS_NB; ++j) { w[j] = 0.5 * (pdf[j] + pdf[j + 1]); W += w[j]; }
  int S[ALIAS_NB], L[ALIAS_NB], ns = 0, nl = 0;
  double qd[ALIAS_NB];
  for (int j = 0; j < ALIAS_NB; ++j) {
    p[j] = w[j] * ALIAS_NB / W;
    qd[j] = 1.0;
    a[j] = j;
    if (p[j] < 1.0) S[ns++] = j; else L[nl++] = j;
  }
  while (ns > 0 && nl > 0) {
    int s = S[--ns], l = L[--nl];
    qd[s] = p[s];
    a[s] = l;
    p[l] = (p[l] + p[s]) - 1.0;
    if (p[l] < 1.0) S[ns++] = l; else L[nl++] = l;
  }
  for (int j = 0; j < ALIAS_NB; ++j) q[j] = (float)qd[j];
}

static int alias_nE(double E_lo) {
  if (E_lo >= ALIAS_EMAX) return 1;
  return 1 + (int)ceil(ALIAS_PPD * log10(ALIAS_EMAX / E_lo) - 1e-6);
}

static void build_alias(or_ctx *c) {
  for (int m = 0; m < OR_NMODEL; ++m) {
    oalias *t = &c->alias[m];
    t->E_lo = model_Elo(c, m);
    t->nE = alias_nE(t->E_lo);
    if (t->nE > ALIAS_MAXE) t->nE = ALIAS_MAXE;
    double cut = model_cut(c, m);
    for (int ie = 0; ie < t->nE; ++ie) {
      double E = t->E_lo * pow(10.0, (double)ie / ALIAS_PPD);
      for (int j = 0; j <= ALIAS_NB; ++j) t->pdf[ie][j] = reduced_pdf(m, E, (double)j / ALIAS_NB, cut);
      build_alias_row(t->pdf[ie], t->q[ie], t->a[ie]);
    }
  }
}

int or_alias_info(const or_ctx *c, int model, double *E_lo, int *n_E) {
  if (model < 0 || model >= OR_NMODEL) return -1;
  *E_lo = c->alias[model].E_lo;
  *n_E = c->alias[model].nE;
  return 0;
}

int or_alias_table(const or_ctx *c, int model, int ie, double *pdf, float *q, int *alias) {
  if (model < 0 || model >= OR_NMODEL) return -1;
  const oalias *t = &c->alias[model];
  if (ie < 0 || ie >= t->nE) return -1;
  for (int j = 0; j <= ALIAS_NB; ++j) pdf[j] = t->pdf[ie][j];
  for (int j = 0; j < ALIAS_NB; ++j) { q[j] = t->q[ie][j]; alias[j] = t->a[ie][j]; }
  return 0;
}

/* ------------------------------------------------------------------ */
/* rejection samplers (the "rejection" method of Sec. 3.5)             */
/* ------------------------------------------------------------------ */
/* A proposal from a density with a closed-form inverse, accepted with the
 * ratio of the DCS to a bound of it (Sec. 3.5 compares this with sampling
 * tables and chooses per energy range).  Trial j takes its proposal and
 * acceptance uniforms from counter block REJ_BLOCK0 + j/2 of the
 * interacting step (words 2(j%2) and 2(j%2)+1); after REJ_MAX_TRIALS
 * rejections the last proposal stands.  Built for:
 *   pair       x uniform on [m/k, 1 - m/k]; accept 1 - 4/3 x(1-x)  (<= 1)
 *   brems      k = k_c (T/k_c)^xi (density 1/k); accept
 *              (4/3 - 4/3 y + y^2) / (4/3), y = k/(T+m)
 *   Compton    eps = eps0^(1-xi) (density 1/eps); accept
 *              (1 + eps^2 - eps sin^2 theta) / 2
 * The proposal's xi is the reduced variable of the sampling tables. */
/* uniform in (0, 1] from a 32-bit Philox word: 24 bits, exact in FP32 and FP64 */
static double u24(uint32_t x) { return (double)((x >> 8) + 1u) * (1.0 / 16777216.0); }

#define REJ_BLOCK0 3u
#define REJ_MAX_TRIALS 64

int or_has_rejection(int model) {
  return model == OR_M_PAIR || model == OR_M_BREM || model == OR_M_COMPTON;
}

double or_reject_sample(const or_ctx *c, int model, double E, const uint32_t rng[5], double *xi_out,
                        int *trials) {
  const double cut = model_cut(c, model);
  double v = 0.0, xi = 0.0;
  int j = 0;
  uint32_t w[4] = {0, 0, 0, 0};
  for (j = 0; j < REJ_MAX_TRIALS; ++j) {
    if ((j & 1) == 0) {
      const uint32_t ctr[4] = {rng[0], rng[1], rng[2], REJ_BLOCK0 + (uint32_t)(j >> 1)};
      const uint32_t key[2] = {rng[3], rng[4]};
      or_philox4x32_10(ctr, key, w);
    }
    xi = u24(w[2 * (j & 1)]);
    const double ua = u24(w[2 * (j & 1) + 1]);
    double f = 0.0;
    v = xi_to_var(model, E, xi, cut);
    if (model == OR_M_PAIR) {
      f = 1.0 - 4.0 / 3.0 * v * (1.0 - v);
    } else if (model == OR_M_BREM) {
      const double y = v / (E + ME);
      f = (4.0 / 3.0 - 4.0 / 3.0 * y + y * y) * 0.75;
    } else {
      const double K = E / ME, t = (1.0 - v) / (K * v), s2 = t * (2.0 - t);
      f = 0.5 * (1.0 + v * v - v * s2);
    }
    if (ua <= f) break;
  }
  if (trials) *trials = j < REJ_MAX_TRIALS ? j + 1 : REJ_MAX_TRIALS;
  if (xi_out) *xi_out = xi;
  return v;
}

/* Exact samplers of the remaining models, by rejection from their DCS with
 * the trial stream of or_reject_sample (block 3 + j/2, at most
 * EXACT_MAX_TRIALS trials):
 *   Moller   eps = T_delta/T in [x_c, 1/2], proposal density 1/eps^2,
 *            accept eps^2 dsigma/deps / (2 + C1/4): dropping the two terms
 *            with -C2 (C2 >= 0) leaves C1 eps^2 + 1 + eps^2/(1-eps)^2, at
 *            most C1/4 + 2 for eps <= 1/2
 *   Bhabha   eps in [x_c, 1], proposal 1/eps^2, accept beta^2 eps^2
 *            dsigma/deps = 1 - beta^2 eps P(eps), P = B1 - B2 eps + B3 eps^2
 *            - B4 eps^3: P' < 0 on [0, 1] (its discriminant is negative) and
 *            P(1) = 2y(1 + y + y^2) > 0, so the ratio lies in [0, 1]
 *   annih.   softer photon fraction eps in [eps_min, 1/2], proposal 1/eps,
 *            accept eps (S(eps) + S(1-eps)) / M, S(x) = -a + b/x - 1/x^2,
 *            a = (g+1)^2, b = g^2 + 4g + 1: eps S(eps) <= b - 2 sqrt(a) and
 *            eps S(1-eps) <= (2b - 4 - a)/2 for eps <= 1/2, so
 *            M = 1.5 g^2 + 5 g - 2.5 */
#define EXACT_MAX_TRIALS 4096

static double exact_other(const or_ctx *c, int model, double E, const uint32_t rng[5], double *xi_out,
                          int *trials) {
  const double cut = model_cut(c, model);
  const double g = E / ME + 1.0, b2 = 1.0 - 1.0 / (g * g);
  double v = 0.0, xi = 0.0;
  int j;
  uint32_t w[4] = {0, 0, 0, 0};
  for (j = 0; j < EXACT_MAX_TRIALS; ++j) {
    if ((j & 1) == 0) {
      const uint32_t ctr[4] = {rng[0], rng[1], rng[2], REJ_BLOCK0 + (uint32_t)(j >> 1)};
      const uint32_t key[2] = {rng[3], rng[4]};
      or_philox4x32_10(ctr, key, w);
    }
    xi = u24(w[2 * (j & 1)]);
    const double ua = u24(w[2 * (j & 1) + 1]);
    double f;
    if (model == OR_M_MOLLER) {
      const double xc = cut / E;
      v = xc / (1.0 - xi * (1.0 - 2.0 * xc));
      const double C1 = ((g - 1.0) / g) * ((g - 1.0) / g);
      f = v * v * or_dcs(model, E, v, cut) / (2.0 + 0.25 * C1);
    } else if (model == OR_M_BHABHA) {
      const double xc = cut / E;
      v = xc / (1.0 - xi * (1.0 - xc));
      f = b2 * v * v * or_dcs(model, E, v, cut);
    } else {
      v = xi_to_var(OR_M_ANNIH, E, xi, cut);
      f = v * or_dcs(model, E, v, cut) / (1.5 * g * g + 5.0 * g - 2.5);
    }
    if (ua <= f) break;
  }
  if (trials) *trials = j < EXACT_MAX_TRIALS ? j + 1 : EXACT_MAX_TRIALS;
  if (xi_out) *xi_out = xi;
  return v;
}

double or_exact_sample(const or_ctx *c, int model, double E, const uint32_t rng[5], double *xi_out,
                       int *trials) {
  if (or_has_rejection(model)) return or_reject_sample(c, model, E, rng, xi_out, trials);
  return exact_other(c, model, E, rng, xi_out, trials);
}

/* The sampler the setup chooses for (model, E): rejection where it is built
 * and E >= reject_min[model], else the sampling tables (u3: their uniforms). */
static double sample_var(const or_ctx *c, int model, double E, const double *u3, const uint32_t rng[5]) {
  if (c->s.exact) return or_exact_sample(c, model, E, rng, NULL, NULL);
  if (or_has_rejection(model) && E >= c->s.reject_min[model]) return or_reject_sample(c, model, E, rng, NULL, NULL);
  return or_alias_sample(c, model, E, u3, NULL);
}

/* Sample the physical variable at energy E with uniforms
 * u[0]: grid-energy choice, u[1]: bin + alias, u[2]: position in the bin. */
double or_alias_sample(const or_ctx *c, int model, double E, const double *u, double *xi_out) {
  const oalias *t = &c->alias[model];
  double l = log(E / t->E_lo) / (log(10.0) / ALIAS_PPD);
  int ie;
  if (l <= 0.0) ie = 0;
  else if (l >= t->nE - 1) ie = t->nE - 1;
  else {
    int i = (int)floor(l);
    ie = (u[0] < l - i) ? i + 1 : i;
  }
  double x = u[1] * ALIAS_NB;
  int j = (int)x;
  if (j > ALIAS_NB - 1) j = ALIAS_NB - 1;
  double fr = x - j;
  int b = (fr < (double)t->q[ie][j]) ? j : t->a[ie][j];
  double p0 = t->pdf[ie][b], p1 = t->pdf[ie][b + 1];
  double tt = u[2] * (p0 + p1) / (p0 + sqrt(p0 * p0 + u[2] * (p1 * p1 - p0 * p0)));
  double xi = (b + tt) / ALIAS_NB;
  if (xi_out) *xi_out = xi;
  return xi_to_var(model, E, xi, model_cut(c, model));
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).                  */
/* Pinned: Random123 known-answer vectors.                             */
/* ------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint64_t p0 = (uint64_t)0xD2511F53u * x0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ x1 ^ k0, n2 = hi0 ^ x3 ^ k1;
    x0 = n0; x1 = lo1; x2 = n2; x3 = lo0;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------ */
/* tables                                                              */
/* ------------------------------------------------------------------ */
static void build_tables(or_ctx *c) {
  memset(c->tab, 0, sizeof(c->tab));
  for (int m = 0; m < c->s.n_mat; ++m) {
    for (int i = 0; i < GRID_N; ++i) {
      double E = or_grid_energy(i);
      for (int p = 0; p < 3; ++p) c->tab[OR_GAMMA][p][m][i] = or_xs(c, OR_GAMMA, p, m, E);
      for (int p = 0; p < 2; ++p) c->tab[OR_ELECTRON][p][m][i] = or_xs(c, OR_ELECTRON, p, m, E);
      for (int p = 0; p < 3; ++p) c->tab[OR_POSITRON][p][m][i] = or_xs(c, OR_POSITRON, p, m, E);
    }
    for (int t = OR_ELECTRON; t <= OR_POSITRON; ++t) {
      int qR = t == OR_ELECTRON ? 2 : 3;
      double R = GRID_EMIN / or_dedx(c, t, m, GRID_EMIN);
      c->tab[t][qR][m][0] = R;
      for (int i = 0; i + 1 < GRID_N; ++i) {
        const double d = inv_dedx_integral(c, t, m, or_grid_energy(i), or_grid_energy(i + 1));
        c->dR[t - 1][m][i] = d;
        R += d;
        c->tab[t][qR][m][i + 1] = R;
      }
      {  /* the kinks of S(E): restricted ionisation switching to its cut, the
          * gamma cut, the onset of the density effect (sorted) */
        const omat *o = &c->mat[m];
        double *k = c->kink[t - 1][m];
        k[0] = t == OR_POSITRON ? c->s.e_cut : 2.0 * c->s.e_cut;
        k[1] = c->s.gamma_cut;
        const double bg = exp(0.5 - log(o->plasma / o->I));
        k[2] = ME * (sqrt(1.0 + bg * bg) - 1.0);
        for (int a = 0; a < 3; ++a)
          for (int b = a + 1; b < 3; ++b)
            if (k[b] < k[a]) { double x = k[a]; k[a] = k[b]; k[b] = x; }
      }
      /* the running maximum of the node values of Sigma(E) */
      double run = 0.0;
      for (int i = 0; i < GRID_N; ++i) {
        double sig = 0.0;
        for (int p = 0; p < n_proc(t); ++p) sig += c->tab[t][p][m][i];
        run = fmax(run, sig);
        c->smax[t - 1][m][i] = run;
      }
    }
  }
}


double or_table_node(const or_ctx *c, int type, int q, int mat, int i) { return c->tab[type][q][mat][i]; }

static void grid_pos(double E, int *i, double *f) {
  double l = (log(E) - log(GRID_EMIN)) / (log(10.0) / GRID_PPD);
  int k = (int)floor(l);
  if (k < 0) k = 0;
  if (k > GRID_N - 2) k = GRID_N - 2;
  double fr = l - k;
  if (fr < 0.0) fr = 0.0;
  if (fr > 1.0) fr = 1.0;
  *i = k;
  *f = fr;
}

/* Cross sections: linear in ln E between the nodes.  The range: ln R linear
 * in ln E (R a power of E within an interval).  The range's slope in ln E,
 * E/S(E), grows by ~7 % across an interval, so R linear in ln E would give
 * every step inside an interval the interval's mean slope, i.e. a stopping
 * power off by up to +-3.6 % (the untabulated transport shows it as a
 * +0.9 % deposit in the first layer of 1 GeV showers); in ln R that slope
 * error is the curvature of ln R, a few 1e-4. */
static int is_range(int type, int q) { return type != OR_GAMMA && q == (type == OR_ELECTRON ? 2 : 3); }

double or_table_lookup(const or_ctx *c, int type, int q, int mat, double E) {
  int i;
  double f;
  grid_pos(E, &i, &f);
  const double *v = c->tab[type][q][mat];
  if (is_range(type, q)) return exp(log(v[i]) + f * (log(v[i + 1]) - log(v[i])));
  return v[i] + f * (v[i + 1] - v[i]);
}

/* Integral approach (charged tracks lose energy along a step, so their
 * cross section changes): Sigma_max(E), the linear interpolation of the
 * running maximum of the node values, bounds the interpolated Sigma at every
 * energy up to E (node-wise >= with the same weights, and non-decreasing). */
double or_sigma_max(const or_ctx *c, int type, int mat, double E) {
  int i;
  double f;
  grid_pos(E, &i, &f);
  const double *v = c->smax[type - 1][mat];
  return v[i] + f * (v[i + 1] - v[i]);
}

/* Continuous loss along a step s from kinetic energy E (charged types): the
 * post-step energy is the exact inverse of the interpolated range,
 * E' = R^-1(R(E) - s), with ln R piecewise linear in ln E between nodes;
 * below the first node R is linear in E. */
double or_eloss(const or_ctx *c, int type, int mat, double E, double s) {
  int qR = type == OR_ELECTRON ? 2 : 3;
  const double *R = c->tab[type][qR][mat];
  double Rv = or_table_lookup(c, type, qR, mat, E);
  if (s >= Rv) return 0.0;
  double r = Rv - s;
  if (r < R[0]) return GRID_EMIN * r / R[0];
  int lo = 0, hi = GRID_N - 1; /* find R[lo] <= r < R[lo+1] */
  while (hi - lo > 1) {
    int mid = (lo + hi) / 2;
    if (R[mid] <= r) lo = mid; else hi = mid;
  }
  double le = log(GRID_EMIN) +
              (log(10.0) / GRID_PPD) * (lo + (log(r) - log(R[lo])) / (log(R[lo + 1]) - log(R[lo])));
  return exp(le);
}

/* ------------------------------------------------------------------ */
/* untabulated range and continuous loss                               */
/* ------------------------------------------------------------------ */
/* integral of dE/S over [a, b] (a <= b inside one grid interval), split at
 * the kinks of S, 6-point Gauss-Legendre in ln E on each piece (a grid
 * interval spans ln 10 / 32 = 0.072 in ln E, over which 6 points leave an
 * error far below 1e-12 of the integral) */
static double quad_inv_dedx(const or_ctx *c, int type, int mat, double a, double b) {
  if (!(b > a)) return 0.0;
  double edge[5];
  int ne = 0;
  edge[ne++] = a;
  const double *k = c->kink[type - 1][mat];
  for (int j = 0; j < 3; ++j)
    if (k[j] > a && k[j] < b) edge[ne++] = k[j];
  edge[ne++] = b;
  double sum = 0.0;
  for (int j = 0; j + 1 < ne; ++j) {
    const double la = log(edge[j]), lb = log(edge[j + 1]);
    const double h = 0.5 * (lb - la), mid = 0.5 * (la + lb);
    for (int i = 0; i < 6; ++i) {
      const double E = exp(mid + h * c->gl6_x[i]);
      sum += h * c->gl6_w[i] * E / or_dedx(c, type, mat, E);
    }
  }
  return sum;
}

/* grid interval i with E_i <= E < E_{i+1} (clamped to the grid) */
static int grid_interval(double E) {
  int i = (int)floor((log(E) - log(GRID_EMIN)) / (log(10.0) / GRID_PPD));
  if (i < 0) i = 0;
  if (i > GRID_N - 2) i = GRID_N - 2;
  while (i > 0 && or_grid_energy(i) > E) --i;
  while (i < GRID_N - 2 && or_grid_energy(i + 1) <= E) ++i;
  return i;
}

/* R(E) = Emin/S(Emin) + int_{Emin}^{E} dE/S: the node value (a sum of exact
 * interval quadratures) plus the quadrature from the node up to E -- no
 * interpolation */
double or_range_at(const or_ctx *c, int type, int mat, double E) {
  const int qR = type == OR_ELECTRON ? 2 : 3;
  const double R0 = c->tab[type][qR][mat][0];
  if (E <= GRID_EMIN) return E / GRID_EMIN * R0;
  const int i = grid_interval(E);
  return c->tab[type][qR][mat][i] + quad_inv_dedx(c, type, mat, or_grid_energy(i), E);
}

/* Post-step energy E' of a step s from E with range R_E = R(E): the root of
 * int_{E'}^{E} dE/S = s.  Whole grid intervals below E are subtracted from
 * s while they fit (their exact quadratures, no cancellation); inside the
 * interval that holds E' the root of int_{E'}^{top} dE/S = rem is found by
 * Newton's method on the quadrature (derivative -1/S(E')), kept inside its
 * bracket by bisection in ln E, started from the step with S(top). */
static double eloss_exact_R(const or_ctx *c, int type, int mat, double E, double R_E, double s) {
  if (!(s > 0.0)) return E;
  if (s >= R_E) return 0.0;
  const int qR = type == OR_ELECTRON ? 2 : 3;
  const double R0 = c->tab[type][qR][mat][0];
  if (E <= GRID_EMIN) return GRID_EMIN * (R_E - s) / R0;
  int i = grid_interval(E);
  double top = E, rem = s;
  double part = quad_inv_dedx(c, type, mat, or_grid_energy(i), E);
  while (part < rem) { /* E' lies below node i */
    rem -= part;
    top = or_grid_energy(i);
    if (i == 0) return GRID_EMIN * fmax(0.0, R0 - rem) / R0; /* below the grid: R linear in E */
    --i;
    part = c->dR[type - 1][mat][i];
  }
  /* root in [E_i, top]: f(x) = int_x^top dE/S - rem, decreasing, f(E_i) >= 0 > f(top) */
  double lo = or_grid_energy(i), hi = top;
  double x = top - rem * or_dedx(c, type, mat, top);
  if (!(x > lo && x < hi)) x = sqrt(lo * hi);
  for (int it = 0; it < 100; ++it) {
    const double f = quad_inv_dedx(c, type, mat, x, top) - rem;
    if (f == 0.0) return x;
    if (f > 0.0) lo = x; else hi = x;
    double xn = x + f * or_dedx(c, type, mat, x);
    if (!(xn > lo && xn < hi)) xn = sqrt(lo * hi);
    if (fabs(xn - x) <= 1e-15 * x || hi - lo <= 1e-15 * hi) return xn;
    x = xn;
  }
  return x;
}

double or_eloss_exact(const or_ctx *c, int type, int mat, double E, double s) {
  return eloss_exact_R(c, type, mat, E, or_range_at(c, type, mat, E), s);
}

/* ------------------------------------------------------------------ */
/* geometry: layered box, FP64                                         */
/* ------------------------------------------------------------------ */
int or_n_subtotal(const or_ctx *c) { return c->nsub; }
double or_plane_z(const or_ctx *c, int k) { return c->zb[k]; }

int or_locate(const or_ctx *c, double z, double w) {
  if (z < 0.0 || z > c->zb[c->nsub]) return -1;
  for (int k = 0; k < c->nsub; ++k) {
    if (z >= c->zb[k] && z < c->zb[k + 1]) {
      if (z == c->zb[k] && w < 0.0) return k - 1;
      return k;
    }
  }
  if (z == c->zb[c->nsub] && w < 0.0) return c->nsub - 1;
  return -1;
}

/* Distance to the boundary of sub-slab `sub` along dir.  next_sub = -1 for
 * leaving the calorimeter.  plane: z-plane index, or -2 (x wall), -3 (y wall).
 * Pinned: brute-force marching on small cases and the analytic plane
 * intersection on random rays. */
double or_distance(const or_ctx *c, const double pos[3], const double dir[3], int sub,
                   int *next_sub, int *plane) {
  double d = INFINITY;
  int nx = sub, pl = -1;
  if (dir[2] > 0.0) {
    d = (c->zb[sub + 1] - pos[2]) / dir[2];
    nx = sub + 1;
    pl = sub + 1;
  } else if (dir[2] < 0.0) {
    d = (c->zb[sub] - pos[2]) / dir[2];
    nx = sub - 1;
    pl = sub;
  }
  if (c->s.half_x > 0.0) {
    double dx = INFINITY;
    if (dir[0] > 0.0) dx = (c->s.half_x - pos[0]) / dir[0];
    else if (dir[0] < 0.0) dx = (-c->s.half_x - pos[0]) / dir[0];
    if (dx < d) { d = dx; nx = -1; pl = -2; }
  }
  if (c->s.half_y > 0.0) {
    double dy = INFINITY;
    if (dir[1] > 0.0) dy = (c->s.half_y - pos[1]) / dir[1];
    else if (dir[1] < 0.0) dy = (-c->s.half_y - pos[1]) / dir[1];
    if (dy < d) { d = dy; nx = -1; pl = -3; }
  }
  if (d < 0.0) d = 0.0;
  if (nx >= c->nsub) nx = -1;
  *next_sub = nx;
  *plane = pl;
  return d;
}

/* Distance from pos to the nearest boundary of sub-slab `sub` (its two
 * z-planes and the bounded x/y walls): the isotropic safety of Sec. 3.2. */
double or_safety(const or_ctx *c, const double pos[3], int sub) {
  double d = fmin(pos[2] - c->zb[sub], c->zb[sub + 1] - pos[2]);
  if (c->s.half_x > 0.0) d = fmin(d, c->s.half_x - fabs(pos[0]));
  if (c->s.half_y > 0.0) d = fmin(d, c->s.half_y - fabs(pos[1]));
  return d > 0.0 ? d : 0.0;
}

/* ------------------------------------------------------------------ */
/* uniform magnetic field (the field propagation of Sec. 3.6)          */
/* ------------------------------------------------------------------ */
/* A track of charge q and momentum p (MeV/c) in a field B (tesla) along the
 * unit vector b turns at the rate dd/ds = q k (d x b), k = c B / p with
 * c = 2.99792458 cm^-1 MeV/(c T) (the radius of curvature of 1 MeV/c in 1 T
 * is 0.33356 cm).  Splitting d = a + c0 with a = (d.b) b, and g = c0 x b,
 * the exact helix after a path s, th = q k s, is
 *   position  r0 + a s + c0 sin(th) / (q k) + g (1 - cos th) / (q k)
 *   direction a + c0 cos(th) + g sin(th).                                 */
#define FIELD_C 2.99792458
#define FIELD_SAGITTA 1e-3 /* cm */
#define FIELD_MAX_TURN 0.2 /* rad */

static double field_curvature(const or_ctx *c, int type, double E) {
  const double p = sqrt(E * (E + 2.0 * ME));
  const double q = type == OR_POSITRON ? 1.0 : -1.0;
  return q * FIELD_C * c->s.field_T / p;
}

/* Longest step with a chord sagitta <= 10 um and a turn <= 0.2 rad, taking
 * the curvature of the helix itself, |k| sin(angle between d and b). */
double or_field_step_limit(const or_ctx *c, int type, double E, const double dir[3]) {
  if (type == OR_GAMMA || c->s.field_T == 0.0) return INFINITY;
  const double db = dir[c->s.field_axis];
  const double keff = fabs(field_curvature(c, type, E)) * sqrt(fmax(0.0, 1.0 - db * db));
  if (!(keff > 0.0)) return INFINITY;
  return fmin(sqrt(8.0 * FIELD_SAGITTA / keff), FIELD_MAX_TURN / keff);
}

void or_helix(const or_ctx *c, int type, double E, double s, const double dir[3], double dpos[3],
              double ndir[3]) {
  const int ax = c->s.field_axis;
  double b[3] = {0.0, 0.0, 0.0};
  b[ax] = 1.0;
  const double db = dir[ax];
  double a[3], c0[3], g[3];
  for (int j = 0; j < 3; ++j) {
    a[j] = db * b[j];
    c0[j] = dir[j] - a[j];
  }
  g[0] = c0[1] * b[2] - c0[2] * b[1];
  g[1] = c0[2] * b[0] - c0[0] * b[2];
  g[2] = c0[0] * b[1] - c0[1] * b[0];
  const double w = (type == OR_GAMMA || c->s.field_T == 0.0) ? 0.0 : field_curvature(c, type, E);
  const double th = w * s;
  /* sin(th)/th and (1 - cos th)/th = 2 sin^2(th/2)/th, both -> their limits at 0 */
  const double sc = th != 0.0 ? sin(th) / th : 1.0;
  const double cc = th != 0.0 ? 2.0 * sin(0.5 * th) * sin(0.5 * th) / th : 0.0;
  for (int j = 0; j < 3; ++j) {
    dpos[j] = a[j] * s + c0[j] * s * sc + g[j] * s * cc;
    ndir[j] = a[j] + c0[j] * cos(th) + g[j] * sin(th);
  }
}

/* ------------------------------------------------------------------ */
/* multiple Coulomb scattering (the MSC stages of Sec. 2.1.2)          */
/* ------------------------------------------------------------------ */
/* Highland width of the projected angle for a unit-charge track of kinetic
 * energy T after a path s in material mat:
 *   theta0 = 13.6 MeV / (beta p c) sqrt(s/X0) (1 + 0.038 ln(s / (X0 beta^2)))
 * with the bracket floored at 0 (PDG, "Passage of particles through
 * matter", multiple scattering section).  Pinned: within 11 % of two widths
 * from Moliere's theory (Bethe's Gaussian approximation, and Lynch & Dahl's
 * width of the central 98 %) for 1e-3 < x/X0 < 100. */
double or_msc_theta0(const or_ctx *c, int mat, double T, double s) {
  if (!(s > 0.0) || !(T > 0.0)) return 0.0;
  const double pc = sqrt(T * (T + 2.0 * ME));
  const double beta = pc / (T + ME);
  const double X0 = c->mat[mat].X0g / c->mat[mat].m.rho;
  const double x = s / X0;
  const double corr = 1.0 + 0.038 * log(x / (beta * beta));
  return corr > 0.0 ? 13.6 / (beta * pc) * sqrt(x) * corr : 0.0;
}

/* Gaussian multiple scattering over a step of length s that took the
 * kinetic energy from E_pre to E_post, evaluated at their mean.  Four
 * uniforms give four standard normals (Box-Muller: radius from the first of
 * each pair, angle from the second); per transverse plane the angle is
 * z2 theta0 and the offset s theta0 (z1 / sqrt(12) + z2 / 2), the joint
 * Gaussian of the PDG section quoted above (correlation sqrt(3)/2).  The two
 * planes are those of the frame in which rotations act (rotate()): e1, e2
 * perpendicular to dir.  The new direction has polar angle
 * theta = |(theta_x, theta_y)| (at most pi) about dir, azimuth along
 * (theta_x, theta_y).  The offset moves the end point within the sub-slab:
 * it is shortened to 0.99 of the safety when it is longer. */
int or_msc(const or_ctx *c, int sub, double E_pre, double E_post, double s, const double dir[3],
           const double pos[3], const double u[4], double out_dir[3], double out_pos[3]) {
  const int mat = c->smat[sub];
  const double th0 = or_msc_theta0(c, mat, 0.5 * (E_pre + E_post), s);
  const double r1 = sqrt(-2.0 * log(u[0])), r2 = sqrt(-2.0 * log(u[2]));
  const double z1 = r1 * cos(2.0 * PI * u[1]), z2 = r1 * sin(2.0 * PI * u[1]);
  const double z3 = r2 * cos(2.0 * PI * u[3]), z4 = r2 * sin(2.0 * PI * u[3]);
  const double tx = th0 * z1, ty = th0 * z2;
  const double ox = s * th0 * (z3 / sqrt(12.0) + z1 / 2.0);
  const double oy = s * th0 * (z4 / sqrt(12.0) + z2 / 2.0);
  /* frame: e1, e2 perpendicular to dir, as in rotate() */
  double e1[3], e2[3];
  const double up = sqrt(dir[0] * dir[0] + dir[1] * dir[1]);
  if (up > 0.0) {
    e1[0] = dir[0] * dir[2] / up; e1[1] = dir[1] * dir[2] / up; e1[2] = -up;
    e2[0] = -dir[1] / up; e2[1] = dir[0] / up; e2[2] = 0.0;
  } else {
    e1[0] = dir[2] < 0.0 ? -1.0 : 1.0; e1[1] = 0.0; e1[2] = 0.0;
    e2[0] = 0.0; e2[1] = 1.0; e2[2] = 0.0;
  }
  double th = sqrt(tx * tx + ty * ty);
  if (th > 0.0) {
    const double cp = tx / th, sp = ty / th;
    if (th > PI) th = PI;
    const double ct = cos(th), st = sin(th);
    for (int j = 0; j < 3; ++j) out_dir[j] = st * (cp * e1[j] + sp * e2[j]) + ct * dir[j];
  } else {
    for (int j = 0; j < 3; ++j) out_dir[j] = dir[j];
  }
  double off[3];
  for (int j = 0; j < 3; ++j) off[j] = ox * e1[j] + oy * e2[j];
  const double len = sqrt(ox * ox + oy * oy);
  const double safe = or_safety(c, pos, sub);
  const double scale = (len > 0.99 * safe) ? (len > 0.0 ? 0.99 * safe / len : 0.0) : 1.0;
  for (int j = 0; j < 3; ++j) out_pos[j] = pos[j] + scale * off[j];
  return 0;
}

/* ------------------------------------------------------------------ */
/* setup                                                               */
/* ------------------------------------------------------------------ */
int or_create(const or_setup *s, or_ctx **out) {
  if (!s || !out) return -1;
  if (s->n_mat < 1 || s->n_mat > OR_MAX_MAT || s->n_sub < 1 || s->n_sub > OR_MAX_SUBSEQ ||
      s->n_layers < 1)
    return -1;
  if (s->track_cut < GRID_EMIN || s->gamma_cut < s->track_cut || s->e_cut < s->track_cut) return -1;
  /* the integral approach bounds the tabulated cross sections; the
   * untabulated transport does not take it */
  if (s->exact && (s->process_mask & OR_P_INTEGRAL)) return -1;
  or_ctx *c = (or_ctx *)calloc(1, sizeof(or_ctx));
  if (!c) return -2;
  c->s = *s;
  gauss_legendre(16, c->gl_x, c->gl_w);
  gauss_legendre(6, c->gl6_x, c->gl6_w);
  for (int m = 0; m < s->n_mat; ++m) mat_init(&c->mat[m], &s->mat[m]);
  c->nsub = s->n_layers * s->n_sub;
  c->zb = (double *)malloc(sizeof(double) * (c->nsub + 1));
  c->smat = (int *)malloc(sizeof(int) * c->nsub);
  double z = 0.0;
  c->zb[0] = 0.0;
  for (int l = 0; l < s->n_layers; ++l)
    for (int j = 0; j < s->n_sub; ++j) {
      int k = l * s->n_sub + j;
      z += s->sub_thick[j];
      c->zb[k + 1] = z;
      c->smat[k] = s->sub_mat[j];
    }
  build_tables(c);
  build_alias(c);
  *out = c;
  return 0;
}

void or_destroy(or_ctx *c) {
  if (!c) return;
  free(c->zb);
  free(c->smat);
  free(c);
}

/* ------------------------------------------------------------------ */
/* interactions (PostStepActions)                                      */
/* ------------------------------------------------------------------ */
/* rotate direction d by polar cos ct and azimuth phi about d itself */
static void rotate(const double d[3], double ct, double phi, double o[3]) {
  double st = sqrt(fmax(0.0, 1.0 - ct * ct));
  double cp = cos(phi), sp = sin(phi);
  double lx = st * cp, ly = st * sp, lz = ct;
  double up = d[0] * d[0] + d[1] * d[1];
  if (up > 0.0) {
    up = sqrt(up);
    o[0] = (d[0] * d[2] * lx - d[1] * ly) / up + d[0] * lz;
    o[1] = (d[1] * d[2] * lx + d[0] * ly) / up + d[1] * lz;
    o[2] = -up * lx + d[2] * lz;
  } else if (d[2] < 0.0) {
    o[0] = -lx; o[1] = ly; o[2] = -lz;
  } else {
    o[0] = lx; o[1] = ly; o[2] = lz;
  }
}

static void unit_or(const double p[3], const double fallback[3], double o[3]) {
  double n = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
  if (n > 0.0) { o[0] = p[0] / n; o[1] = p[1] / n; o[2] = p[2] / n; }
  else { o[0] = fallback[0]; o[1] = fallback[1]; o[2] = fallback[2]; }
}

typedef struct {
  int n;
  int type[3];
  double E[3];
  double dir[3][3];
} kids_t;

static void add_kid(kids_t *k, int type, double E, const double d[3]) {
  k->type[k->n] = type;
  k->E[k->n] = E;
  k->dir[k->n][0] = d[0]; k->dir[k->n][1] = d[1]; k->dir[k->n][2] = d[2];
  k->n++;
}

/* two back-to-back 511 keV photons, isotropic (u6, u7) */
static void annihilate_at_rest(kids_t *k, double u6, double u7) {
  double ct = 2.0 * u6 - 1.0, st = sqrt(fmax(0.0, 1.0 - ct * ct)), ph = 2.0 * PI * u7;
  double d[3] = {st * cos(ph), st * sin(ph), ct};
  double m[3] = {-d[0], -d[1], -d[2]};
  add_kid(k, OR_GAMMA, ME, d);
  add_kid(k, OR_GAMMA, ME, m);
}

/* Final state of process p of a particle of `type` with kinetic energy *E and
 * direction dir (updated in place).  u: the eight uniforms of the step
 * (u[2] grid, u[3] bin, u[4] in-bin, u[5] azimuth, u[6], u[7] isotropic).
 * Returns: 1 primary survives, 0 primary died, -1 no interaction possible.
 * *local: energy deposited at the interaction point. */
static int interact(const or_ctx *c, int type, int p, double *E, double dir[3], const double *u,
                    const uint32_t rng[5], kids_t *kids, double *local, int *n_pair, int *n_annih) {
  const or_setup *s = &c->s;
  double ecut_push = fmax(s->e_cut, s->track_cut);
  double ua[3] = {u[2], u[3], u[4]};
  double phi = 2.0 * PI * u[5];
  *local = 0.0;
  kids->n = 0;
  if (type == OR_GAMMA) {
    double k = *E;
    if (p == 0) { /* Compton */
      double eps = sample_var(c, OR_M_COMPTON, k, ua, rng);
      double K = k / ME, ct = 1.0 - (1.0 - eps) / (K * eps);
      if (ct < -1.0) ct = -1.0;
      if (ct > 1.0) ct = 1.0;
      double d1[3];
      rotate(dir, ct, phi, d1);
      double k1 = eps * k, Te = k - k1;
      double pe[3] = {k * dir[0] - k1 * d1[0], k * dir[1] - k1 * d1[1], k * dir[2] - k1 * d1[2]};
      double de[3];
      unit_or(pe, dir, de);
      if (Te >= ecut_push) add_kid(kids, OR_ELECTRON, Te, de);
      else *local += Te;
      dir[0] = d1[0]; dir[1] = d1[1]; dir[2] = d1[2];
      if (k1 < s->track_cut) { *local += k1; *E = 0.0; return 0; }
      *E = k1;
      return 1;
    }
    if (p == 1) { /* photoelectric */
      if (k >= ecut_push) add_kid(kids, OR_ELECTRON, k, dir);
      else *local += k;
      *E = 0.0;
      return 0;
    }
    /* pair */
    if (k <= 2.0 * ME) return -1;
    double x = sample_var(c, OR_M_PAIR, k, ua, rng);
    double Tm = x * k - ME, Tp = (1.0 - x) * k - ME;
    if (Tm < 0.0) Tm = 0.0;
    if (Tp < 0.0) Tp = 0.0;
    double ct = cos(ME / k), dm[3], dp[3];
    rotate(dir, ct, phi, dm);
    rotate(dir, ct, phi + PI, dp);
    *n_pair += 1;
    if (Tm >= ecut_push) add_kid(kids, OR_ELECTRON, Tm, dm);
    else *local += Tm;
    if (Tp >= ecut_push) add_kid(kids, OR_POSITRON, Tp, dp);
    else {
      *local += Tp;
      annihilate_at_rest(kids, u[6], u[7]);
      *n_annih += 1;
    }
    *E = 0.0;
    return 0;
  }
  /* charged */
  double T = *E;
  if (p == 0) { /* bremsstrahlung */
    if (T <= s->gamma_cut) return -1;
    double kg = sample_var(c, OR_M_BREM, T, ua, rng);
    double dg[3];
    rotate(dir, cos(ME / (T + ME)), phi, dg);
    if (kg >= s->track_cut) add_kid(kids, OR_GAMMA, kg, dg);
    else *local += kg;
    T -= kg;
  } else if (p == 1) { /* ionisation */
    int model = type == OR_ELECTRON ? OR_M_MOLLER : OR_M_BHABHA;
    if (type == OR_ELECTRON && T <= 2.0 * s->e_cut) return -1;
    if (type == OR_POSITRON && T <= s->e_cut) return -1;
    double eps = sample_var(c, model, T, ua, rng);
    double Td = eps * T;
    double ct = sqrt(Td * (T + 2.0 * ME) / (T * (Td + 2.0 * ME)));
    if (ct > 1.0) ct = 1.0;
    double dd[3];
    rotate(dir, ct, phi, dd);
    double P = sqrt(T * (T + 2.0 * ME)), Pd = sqrt(Td * (Td + 2.0 * ME));
    double pp[3] = {P * dir[0] - Pd * dd[0], P * dir[1] - Pd * dd[1], P * dir[2] - Pd * dd[2]};
    double dn[3];
    unit_or(pp, dir, dn);
    add_kid(kids, OR_ELECTRON, Td, dd);
    dir[0] = dn[0]; dir[1] = dn[1]; dir[2] = dn[2];
    T -= Td;
  } else { /* annihilation in flight */
    double eps = sample_var(c, OR_M_ANNIH, T, ua, rng);
    double tot = T + 2.0 * ME, k1 = eps * tot, k2 = tot - k1;
    double P = sqrt(T * (T + 2.0 * ME));
    double ct = (k1 - ME) / (eps * P);
    if (ct > 1.0) ct = 1.0;
    if (ct < -1.0) ct = -1.0;
    double d1[3];
    rotate(dir, ct, phi, d1);
    double p2[3] = {P * dir[0] - k1 * d1[0], P * dir[1] - k1 * d1[1], P * dir[2] - k1 * d1[2]};
    double d2[3];
    unit_or(p2, dir, d2);
    add_kid(kids, OR_GAMMA, k1, d1);
    add_kid(kids, OR_GAMMA, k2, d2);
    *n_annih += 1;
    *E = 0.0;
    return 0;
  }
  if (T < s->track_cut) {
    *local += T;
    *E = 0.0;
    if (type == OR_POSITRON) { annihilate_at_rest(kids, u[6], u[7]); *n_annih += 1; }
    return 0;
  }
  *E = T;
  return 1;
}

int or_interact(const or_ctx *c, int type, int proc, double E, const double dir[3],
                const double u[8], const uint32_t rng[5], double *out) {
  kids_t kids;
  double d[3] = {dir[0], dir[1], dir[2]}, local = 0.0, e = E;
  int np = 0, na = 0;
  int r = interact(c, type, proc, &e, d, u, rng, &kids, &local, &np, &na);
  for (int i = 0; i < 24; ++i) out[i] = 0.0;
  out[0] = (r == 1) ? e : (r == 0 ? -1.0 : E);
  out[1] = d[0]; out[2] = d[1]; out[3] = d[2];
  out[4] = local;
  out[5] = kids.n;
  for (int j = 0; j < kids.n; ++j) {
    out[6 + 5 * j] = kids.type[j];
    out[7 + 5 * j] = kids.E[j];
    out[8 + 5 * j] = kids.dir[j][0];
    out[9 + 5 * j] = kids.dir[j][1];
    out[10 + 5 * j] = kids.dir[j][2];
  }
  return r;
}

/* ------------------------------------------------------------------ */
/* transport (per-event loop, LIFO stack)                              */
/* ------------------------------------------------------------------ */
typedef struct {
  int type;
  double E, pos[3], dir[3], nlam;
  uint64_t id;
  uint32_t step;
  int sub;
  int primary, interacted;
} otrack;

typedef struct {
  otrack *v;
  long n, cap;
} ostack;

static void push(ostack *s, const otrack *t) {
  if (s->n == s->cap) {
    s->cap = s->cap ? 2 * s->cap : 1024;
    s->v = (otrack *)realloc(s->v, sizeof(otrack) * s->cap);
  }
  s->v[s->n++] = *t;
}

typedef struct {
  const or_ctx *c;
  const or_primary *p;
  const long *ev_first, *ev_list;
  long n_events;
  long first_event;  /* global index of row 0: the random streams use first_event + row */
  uint64_t seed;
  double *edep, *cell, *esc;
  long long *cnt;
  int tid, nthr;
} job_t;

static void score(const or_ctx *c, double *edep_ev, double *cell, int sub, const double at[3], double dE) {
  if (dE == 0.0 || sub < 0) return;
  edep_ev[sub] += dE;
  if (cell && c->s.nx > 0 && c->s.ny > 0 && c->s.half_x > 0.0 && c->s.half_y > 0.0) {
    int layer = sub / c->s.n_sub;
    int ix = (int)floor((at[0] + c->s.half_x) / (2.0 * c->s.half_x / c->s.nx));
    int iy = (int)floor((at[1] + c->s.half_y) / (2.0 * c->s.half_y / c->s.ny));
    if (ix < 0) ix = 0;
    if (ix >= c->s.nx) ix = c->s.nx - 1;
    if (iy < 0) iy = 0;
    if (iy >= c->s.ny) iy = c->s.ny - 1;
    cell[((long)layer * c->s.nx + ix) * c->s.ny + iy] += dE;
  }
}

static void run_event(const job_t *J, long ev, ostack *st) {
  const or_ctx *c = J->c;
  const or_setup *s = &c->s;
  double *edep = J->edep + ev * c->nsub;
  long long *cnt = J->cnt + ev * OR_NCOUNT;
  uint32_t key[2] = {(uint32_t)J->seed ^ (uint32_t)(ev + J->first_event), (uint32_t)(J->seed >> 32)};
  st->n = 0;
  for (long k = J->ev_first[ev + 1] - 1; k >= J->ev_first[ev]; --k) {
    long i = J->ev_list[k];
    const or_primary *p = &J->p[i];
    otrack t;
    memset(&t, 0, sizeof(t));
    t.type = p->type;
    t.E = p->E;
    t.pos[0] = p->x; t.pos[1] = p->y; t.pos[2] = p->z;
    t.dir[0] = p->u; t.dir[1] = p->v; t.dir[2] = p->w;
    t.nlam = -1.0;
    t.id = (uint64_t)p->id;
    t.step = 0;
    t.sub = or_locate(c, p->z, p->w);
    t.primary = 1;
    cnt[OR_C_TRK_G + t.type] += 1;
    push(st, &t);
  }
  while (st->n > 0) {
    otrack t = st->v[--st->n];
    if (t.sub < 0) { J->esc[ev] += t.E; if (t.type == OR_POSITRON) cnt[OR_C_EP_ESC] += 1; continue; }
    for (;;) {
      uint32_t k = t.step;
      uint32_t ctr[4] = {(uint32_t)t.id, (uint32_t)(t.id >> 32), k, 0u};
      uint32_t r0[4], r1[4];
      int have1 = 0;
      double u[8];
      or_philox4x32_10(ctr, key, r0);
      for (int j = 0; j < 4; ++j) u[j] = u24(r0[j]);
      /* PreStep: tracking cut */
      if (t.E < s->track_cut) {
        kids_t kids;
        kids.n = 0;
        score(c, edep, J->cell, t.sub, t.pos, t.E);
        if (t.type == OR_POSITRON) {
          ctr[3] = 1u;
          or_philox4x32_10(ctr, key, r1);
          annihilate_at_rest(&kids, u24(r1[2]), u24(r1[3]));
          cnt[OR_C_ANNIH] += 1;
          uint32_t idw[4];
          uint32_t ci[4] = {(uint32_t)t.id, (uint32_t)(t.id >> 32), k, TAG_ID};
          or_philox4x32_10(ci, key, idw);
          for (int j = 0; j < kids.n; ++j) {
            otrack n;
            memset(&n, 0, sizeof(n));
            n.type = OR_GAMMA; n.E = kids.E[j];
            n.pos[0] = t.pos[0]; n.pos[1] = t.pos[1]; n.pos[2] = t.pos[2];
            n.dir[0] = kids.dir[j][0]; n.dir[1] = kids.dir[j][1]; n.dir[2] = kids.dir[j][2];
            n.nlam = -1.0; n.sub = t.sub;
            n.id = (uint64_t)idw[2 * j] | ((uint64_t)idw[2 * j + 1] << 32);
            cnt[OR_C_TRK_G] += 1;
            push(st, &n);
          }
        }
        break;
      }
      int mat = c->smat[t.sub];
      int np = n_proc(t.type);
      /* ComputeIntLen */
      if (t.nlam <= 0.0) t.nlam = -log(u[0]);
      /* cross sections at the pre-step energy: interpolated in the tables,
       * or (untabulated transport) from their formulas */
      double sig[3] = {0, 0, 0}, Sig = 0.0;
      for (int p = 0; p < np; ++p) {
        sig[p] = s->exact ? or_xs(c, t.type, p, mat, t.E) : or_table_lookup(c, t.type, p, mat, t.E);
        Sig += sig[p];
      }
      int charged = t.type != OR_GAMMA;
      /* integral approach: the step is drawn with Sigma_max over the energies
       * the track can reach, the interaction accepted at the post-step point */
      const int integral = charged && (s->process_mask & OR_P_INTEGRAL);
      const double Smax = integral ? or_sigma_max(c, t.type, mat, t.E) : Sig;
      double s_phys = Smax > 0.0 ? t.nlam / Smax : INFINITY;
      double s_cont = INFINITY, R_pre = 0.0;
      if (charged) {
        double R = s->exact ? or_range_at(c, t.type, mat, t.E)
                            : or_table_lookup(c, t.type, t.type == OR_ELECTRON ? 2 : 3, mat, t.E);
        R_pre = R;
        s_cont = fmax(STEP_ALPHA_R * R, fmin(STEP_RHO_F, R));
        /* the field's step limit acts like the continuous one */
        s_cont = fmin(s_cont, or_field_step_limit(c, t.type, t.E, t.dir));
      }
      /* GeomQuery */
      int next, plane;
      double s_geom = or_distance(c, t.pos, t.dir, t.sub, &next, &plane);
      double sstep = fmin(s_phys, fmin(s_cont, s_geom));
      int lim = (s_geom == sstep) ? 0 : (s_phys == sstep ? 1 : 2); /* 0 geom 1 phys 2 cont */
      if (!(sstep < INFINITY)) { /* nothing limits the step: the track leaves */
        J->esc[ev] += t.E;
        if (t.type == OR_POSITRON) cnt[OR_C_EP_ESC] += 1;
        break;
      }
      /* Propagation: straight, or the helix of the pre-step momentum */
      double mid[3], pre_pos[3] = {t.pos[0], t.pos[1], t.pos[2]};
      const double pre_dir[3] = {t.dir[0], t.dir[1], t.dir[2]};
      if (charged && s->field_T != 0.0) {
        double dp[3], dh[3], nd[3], tmp[3];
        or_helix(c, t.type, t.E, sstep, t.dir, dp, nd);
        or_helix(c, t.type, t.E, 0.5 * sstep, t.dir, dh, tmp);
        for (int j = 0; j < 3; ++j) {
          mid[j] = pre_pos[j] + dh[j];
          t.pos[j] = pre_pos[j] + dp[j];
          t.dir[j] = nd[j];
        }
      } else {
        for (int j = 0; j < 3; ++j) {
          mid[j] = pre_pos[j] + 0.5 * sstep * t.dir[j];
          t.pos[j] = pre_pos[j] + sstep * t.dir[j];
        }
      }
      if (lim == 0) {
        if (plane >= 0) t.pos[2] = c->zb[plane];
        else if (plane == -2) t.pos[0] = pre_dir[0] > 0.0 ? s->half_x : -s->half_x;
        else if (plane == -3) t.pos[1] = pre_dir[1] > 0.0 ? s->half_y : -s->half_y;
      }
      if (Smax > 0.0) t.nlam = (lim == 1) ? 0.0 : t.nlam - sstep * Smax;
      t.step = k + 1;
      cnt[OR_C_STEPS] += 1;
      cnt[OR_C_STEPS_G + t.type] += 1;
      int pre_sub = t.sub;
      const double E_pre = t.E;
      /* AlongStepAction: continuous loss */
      if (charged) {
        double Ep = s->exact ? eloss_exact_R(c, t.type, mat, t.E, R_pre, sstep)
                             : or_eloss(c, t.type, mat, t.E, sstep);
        score(c, edep, J->cell, pre_sub, mid, t.E - Ep);
        t.E = Ep;
        if (t.E < s->track_cut) {
          score(c, edep, J->cell, pre_sub, t.pos, t.E);
          if (t.type == OR_POSITRON) {
            kids_t kids;
            kids.n = 0;
            ctr[3] = 1u;
            or_philox4x32_10(ctr, key, r1);
            annihilate_at_rest(&kids, u24(r1[2]), u24(r1[3]));
            cnt[OR_C_ANNIH] += 1;
            uint32_t idw[4];
            uint32_t ci[4] = {(uint32_t)t.id, (uint32_t)(t.id >> 32), k, TAG_ID};
            or_philox4x32_10(ci, key, idw);
            for (int j = 0; j < kids.n; ++j) {
              otrack n;
              memset(&n, 0, sizeof(n));
              n.type = OR_GAMMA; n.E = kids.E[j];
              n.pos[0] = t.pos[0]; n.pos[1] = t.pos[1]; n.pos[2] = t.pos[2];
              n.dir[0] = kids.dir[j][0]; n.dir[1] = kids.dir[j][1]; n.dir[2] = kids.dir[j][2];
              n.nlam = -1.0; n.sub = pre_sub;
              n.id = (uint64_t)idw[2 * j] | ((uint64_t)idw[2 * j + 1] << 32);
              cnt[OR_C_TRK_G] += 1;
              push(st, &n);
            }
          }
          break;
        }
      }
      /* AlongStepAction: multiple scattering of a charged track that stays in
       * the box (counter block 2 of the step) */
      if (charged && (s->process_mask & OR_P_MSC) && !(lim == 0 && next < 0)) {
        uint32_t r2[4];
        double um[4], nd[3], npos[3];
        ctr[3] = 2u;
        or_philox4x32_10(ctr, key, r2);
        for (int j = 0; j < 4; ++j) um[j] = u24(r2[j]);
        or_msc(c, pre_sub, E_pre, t.E, sstep, t.dir, t.pos, um, nd, npos);
        for (int j = 0; j < 3; ++j) { t.dir[j] = nd[j]; t.pos[j] = npos[j]; }
      }
      if (lim == 0) {
        if (next < 0) {
          J->esc[ev] += t.E;
          if (t.type == OR_POSITRON) cnt[OR_C_EP_ESC] += 1;
          if (t.primary && !t.interacted && plane == c->nsub) cnt[OR_C_UNSCAT] += 1;
          break;
        }
        t.sub = next;
        continue;
      }
      if (lim != 1) continue;
      /* PostStepActions: discrete interaction */
      double target = u[1] * Sig, cum = 0.0;
      int proc = -1;
      if (integral) { /* post-step cross sections; above their sum: no interaction */
        target = u[1] * Smax;
        for (int p = 0; p < np; ++p) {
          cum += or_table_lookup(c, t.type, p, mat, t.E);
          if (target < cum) { proc = p; break; }
        }
      } else {
        for (int p = 0; p < np; ++p) {
          cum += sig[p];
          if (target < cum) { proc = p; break; }
        }
        if (proc < 0)
          for (int p = np - 1; p >= 0; --p)
            if (sig[p] > 0.0) { proc = p; break; }
      }
      t.nlam = -1.0;
      if (proc < 0) continue;
      ctr[3] = 1u;
      or_philox4x32_10(ctr, key, r1);
      have1 = 1;
      for (int j = 0; j < 4; ++j) u[4 + j] = u24(r1[j]);
      (void)have1;
      kids_t kids;
      double local = 0.0;
      int npair = 0, nann = 0;
      const uint32_t rng[5] = {(uint32_t)t.id, (uint32_t)(t.id >> 32), k, key[0], key[1]};
      int r = interact(c, t.type, proc, &t.E, t.dir, u, rng, &kids, &local, &npair, &nann);
      if (r < 0) continue;
      t.interacted = 1;
      cnt[OR_C_PAIR] += npair;
      cnt[OR_C_ANNIH] += nann;
      score(c, edep, J->cell, t.sub, t.pos, local);
      if (kids.n > 0) {
        uint32_t idw[8];
        uint32_t ci[4] = {(uint32_t)t.id, (uint32_t)(t.id >> 32), k, TAG_ID};
        or_philox4x32_10(ci, key, idw);
        if (kids.n > 2) { ci[3] = TAG_ID + 1u; or_philox4x32_10(ci, key, idw + 4); }
        for (int j = 0; j < kids.n; ++j) {
          otrack n;
          memset(&n, 0, sizeof(n));
          n.type = kids.type[j]; n.E = kids.E[j];
          n.pos[0] = t.pos[0]; n.pos[1] = t.pos[1]; n.pos[2] = t.pos[2];
          n.dir[0] = kids.dir[j][0]; n.dir[1] = kids.dir[j][1]; n.dir[2] = kids.dir[j][2];
          n.nlam = -1.0; n.sub = t.sub;
          n.id = (uint64_t)idw[2 * j] | ((uint64_t)idw[2 * j + 1] << 32);
          cnt[OR_C_TRK_G + n.type] += 1;
          push(st, &n);
        }
      }
      if (r == 0) break;
    }
  }
}

static void *worker(void *arg) {
  job_t *J = (job_t *)arg;
  ostack st = {0, 0, 0};
  for (long ev = J->tid; ev < J->n_events; ev += J->nthr) run_event(J, ev, &st);
  free(st.v);
  return NULL;
}

int or_transport_events(const or_ctx *c, const or_primary *p, long n_prim, long first_event, long n_events,
                        uint64_t seed, double *edep, double *cell_edep, double *escape_E, long long *ev_counts,
                        int n_threads) {
  if (!c || (!p && n_prim > 0) || n_events < 0 || first_event < 0 || !edep || !escape_E || !ev_counts) return -1;
  for (long i = 0; i < n_prim; ++i)
    if ((long)p[i].event < first_event || (long)p[i].event - first_event >= n_events || p[i].type < 0 ||
        p[i].type > 2)
      return -1;
  long *first = (long *)calloc(n_events + 1, sizeof(long));
  long *list = (long *)malloc(sizeof(long) * (n_prim > 0 ? n_prim : 1));
  for (long i = 0; i < n_prim; ++i) first[p[i].event - first_event + 1]++;
  for (long e = 0; e < n_events; ++e) first[e + 1] += first[e];
  long *fill = (long *)malloc(sizeof(long) * (n_events + 1));
  memcpy(fill, first, sizeof(long) * (n_events + 1));
  for (long i = 0; i < n_prim; ++i) list[fill[p[i].event - first_event]++] = i;
  memset(edep, 0, sizeof(double) * n_events * c->nsub);
  memset(escape_E, 0, sizeof(double) * n_events);
  memset(ev_counts, 0, sizeof(long long) * n_events * OR_NCOUNT);
  long ncell = (long)c->s.n_layers * c->s.nx * c->s.ny;
  if (cell_edep && ncell > 0) memset(cell_edep, 0, sizeof(double) * ncell);
  if (n_threads < 1) n_threads = 1;
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * n_threads);
  job_t *jobs = (job_t *)calloc(n_threads, sizeof(job_t));
  for (int t = 0; t < n_threads; ++t) {
    job_t *J = &jobs[t];
    J->c = c; J->p = p; J->ev_first = first; J->ev_list = list; J->n_events = n_events;
    J->first_event = first_event;
    J->seed = seed; J->edep = edep; J->esc = escape_E; J->cnt = ev_counts;
    J->cell = (cell_edep && ncell > 0) ? (double *)calloc(ncell, sizeof(double)) : NULL;
    J->tid = t; J->nthr = n_threads;
    if (n_threads > 1) pthread_create(&th[t], NULL, worker, J);
  }
  if (n_threads == 1) worker(&jobs[0]);
  else for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
  for (int t = 0; t < n_threads; ++t) {
    if (jobs[t].cell) {
      for (long i = 0; i < ncell; ++i) cell_edep[i] += jobs[t].cell[i];
      free(jobs[t].cell);
    }
  }
  free(jobs); free(th); free(first); free(list); free(fill);
  return 0;
}

int or_transport(const or_ctx *c, const or_primary *p, long n_prim, long n_events, uint64_t seed,
                 double *edep, double *cell_edep, double *escape_E, long long *ev_counts,
                 int n_threads) {
  return or_transport_events(c, p, n_prim, 0, n_events, seed, edep, cell_edep, escape_E, ev_counts, n_threads);
}
