// gv_internal.h -- shared between the host table builder (gv_tables.cpp) and
// the CUDA translation units of libgv.  Product-internal.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/gv.h"

namespace gv {

// Cross-section / range table grid: 1 keV .. 1 TeV, 32 nodes per decade.
constexpr int kGridN = 9 * 32 + 1;
constexpr double kGridEmin = 1e-3;
constexpr int kGridPerDecade = 32;

// Alias sampling tables: 64 bins of the reduced variable, 8 energies per decade.
constexpr int kNB = 64;
constexpr int kAliasPerDecade = 8;
constexpr double kAliasEmax = 1e6;
constexpr int kNModel = 6;
enum Model { kCompton = 0, kPair = 1, kBrem = 2, kMoller = 3, kBhabha = 4, kAnnih = 5 };

constexpr double kME = 0.51099895;          // MeV
constexpr double kRE = 2.8179403262e-13;    // cm
constexpr double kAlpha = 1.0 / 137.035999084;
constexpr double kNA = 6.02214076e23;
constexpr double kPi = 3.14159265358979323846;

// Step-limit constants of the continuous processes.
constexpr double kAlphaR = 0.2;     // fraction of the range
constexpr double kRhoF = 0.1;       // cm, final range

constexpr uint32_t kTagId = 0x80000000u;

struct HostTables {
  int n_mat = 0;
  // xs[((m*3 + type)*kGridN + i)*4 + q]
  std::vector<double> xs;
  double a_Elo[kNModel];
  int a_nE[kNModel];
  double a_cut[kNModel];
  std::vector<double> a_pdf[kNModel];  // [nE][kNB+1]
  std::vector<float> a_q[kNModel];     // [nE][kNB]
  std::vector<int> a_alias[kNModel];   // [nE][kNB]
  double inv_X0_cm[GV_MAX_MAT] = {0, 0, 0, 0};  // 1 / radiation length per material, 1/cm
  // integral approach: running maximum over the nodes below of the total
  // e- (0) and e+ (1) cross section, smax[(m*2 + pos)*kGridN + i]
  std::vector<double> smax;
};

int build_host_tables(const gv_material *mats, int n_mats, const gv_cuts &cuts, HostTables *out,
                      std::string *err);

}  // namespace gv
