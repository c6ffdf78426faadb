/*
 * gv_oracle.h -- plain, slow FP64 CPU oracle of electromagnetic shower
 * transport through a layered calorimeter (GeantV, arXiv:2005.00949).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library may include,
 * link or call this code; only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark use it.  It shares no code with the CUDA
 * path: every formula below is written out a second time, independently of
 * the product's table builder.
 *
 * The paper (Sec. 3.5) defers its physics formulas to an external EM paper,
 * so the physics implemented here is the textbook set listed in the design
 * notes of this repository:
 *   Compton          free-electron Klein-Nishina
 *   photoelectric    Sauter-type K-shell formula x 5/4, photoelectron takes k
 *   pair production  complete-screening Bethe-Heitler (Tsai)
 *   bremsstrahlung   complete-screening (Tsai), discrete above the gamma cut
 *   ionisation       Moller (e-) / Bhabha (e+), discrete above the e- cut;
 *                    restricted Berger-Seltzer (ICRU 37) collision loss below
 *   annihilation     Heitler two-photon, in flight and at rest
 *   multiple scatt.  optional (OR_P_MSC): Gaussian angle of Highland width
 *                    and correlated lateral offset, within the safety
 *   magnetic field   optional uniform field along a coordinate axis: charged
 *                    tracks follow the exact helix of their pre-step momentum,
 *                    their steps limited to a 10 um sagitta and 0.2 rad;
 *                    boundaries are found along the straight line
 * Two transports: the tabulated one of the paper's method (tables
 * interpolated in ln E, sampling tables), and an untabulated one
 * (or_setup.exact) that evaluates every quantity from its definition.
 * The stepping loop follows the stage sequence of Sec. 2.1.2 (Fig. "simulation
 * stages"): PreStep, ComputeIntLen, GeomQuery, Propagation, AlongStepAction,
 * PostStepActions, SteppingActions; secondaries go to a LIFO stack (the
 * StackBuffer of Sec. 2.1.2).  Random numbers come from Philox4x32-10 (the
 * Random123 family of Sec. 3.3.2) keyed by (seed, event) and counted by
 * (track id, step, block), which is the per-track stream idea of Sec. 5.1.
 */
#ifndef GV_ORACLE_H
#define GV_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_MAX_ELEM 4
#define OR_MAX_MAT 4
#define OR_MAX_SUBSEQ 8
#define OR_NCOUNT 12

/* particle types */
enum { OR_GAMMA = 0, OR_ELECTRON = 1, OR_POSITRON = 2 };

/* process bits (process_mask) */
enum {
  OR_P_COMPTON = 1u << 0, OR_P_PHOTO = 1u << 1, OR_P_PAIR = 1u << 2,
  OR_P_BREM = 1u << 3, OR_P_IONI = 1u << 4, OR_P_ANNIH = 1u << 5,
  OR_P_MSC = 1u << 6,  /* Gaussian multiple scattering of e+- (along the step) */
  OR_P_INTEGRAL = 1u << 7  /* integral approach for the e+- cross sections along a step */
};

/* alias-sampled final-state models */
enum { OR_M_COMPTON = 0, OR_M_PAIR = 1, OR_M_BREM = 2, OR_M_MOLLER = 3,
       OR_M_BHABHA = 4, OR_M_ANNIH = 5, OR_NMODEL = 6 };

/* per-event counters written by or_transport */
enum { OR_C_STEPS = 0, OR_C_STEPS_G, OR_C_STEPS_EM, OR_C_STEPS_EP,
       OR_C_TRK_G, OR_C_TRK_EM, OR_C_TRK_EP, OR_C_PAIR, OR_C_ANNIH,
       OR_C_EP_ESC, OR_C_UNSCAT, OR_C_SPARE };

typedef struct {
  int n_elem;
  double Z[OR_MAX_ELEM], A[OR_MAX_ELEM], w[OR_MAX_ELEM]; /* w: mass fractions */
  double rho;   /* g/cm3 */
  double I_eV;  /* mean excitation energy */
} or_material;

typedef struct {
  int n_mat;
  or_material mat[OR_MAX_MAT];
  int n_layers;                     /* repeated layers along +z from z=0 */
  int n_sub;                        /* sub-slabs per layer */
  double sub_thick[OR_MAX_SUBSEQ];  /* cm */
  int sub_mat[OR_MAX_SUBSEQ];
  double half_x, half_y;            /* cm; <= 0 means unbounded */
  int nx, ny;                       /* scoring cells per layer (0: none) */
  double gamma_cut, e_cut, track_cut; /* MeV */
  unsigned process_mask;
  double field_T;                   /* uniform magnetic field, tesla (0: none) */
  int field_axis;                   /* its direction: 0 x, 1 y, 2 z */
  double reject_min[6];             /* per model: rejection sampling at E >= this (MeV);
                                       sampling tables below (and for models without one) */
  int exact;                        /* 1: untabulated transport (cross sections by formula at the
                                       track's energy, range and its inverse by quadrature and
                                       root finding, every final state by rejection from its DCS);
                                       0: the tabulated transport of the stepping tables */
} or_setup;

typedef struct {
  int type;
  double E;            /* kinetic energy, MeV */
  double x, y, z;      /* cm */
  double u, v, w;      /* unit direction */
  uint32_t event;
  uint32_t id;         /* track id of the primary within its event */
} or_primary;

typedef struct or_ctx or_ctx;

int or_create(const or_setup *s, or_ctx **out);
void or_destroy(or_ctx *c);

/* --- physics, exact (analytic or quadrature) -------------------------- */
double or_material_X0(const or_ctx *c, int mat);          /* g/cm2 */
double or_material_nel(const or_ctx *c, int mat);         /* electrons/cm3 */
double or_klein_nishina_e(double k);                      /* cm2 per electron */
double or_xs(const or_ctx *c, int type, int proc_index, int mat, double E); /* cm^-1 */
double or_dedx(const or_ctx *c, int type, int mat, double E);   /* MeV/cm */
double or_dedx_parts(const or_ctx *c, int type, int mat, double E, double cut_e, double cut_g,
                     double *col, double *rad);
double or_range_exact(const or_ctx *c, int type, int mat, double E);  /* cm */
double or_dcs(int model, double E, double var, double cut); /* shape in physical variable */

/* --- tables (nodes = exact values on the log grid) ------------------- */
int or_grid_size(void);
double or_grid_energy(int i);
double or_table_node(const or_ctx *c, int type, int q, int mat, int i);
double or_table_lookup(const or_ctx *c, int type, int q, int mat, double E);
double or_eloss(const or_ctx *c, int type, int mat, double E, double s); /* post-step energy */
double or_sigma_max(const or_ctx *c, int type, int mat, double E); /* integral approach bound */

/* --- alias sampling tables ------------------------------------------- */
int or_alias_info(const or_ctx *c, int model, double *E_lo, int *n_E);
int or_alias_table(const or_ctx *c, int model, int ie, double *pdf, float *q, int *alias);
double or_alias_sample(const or_ctx *c, int model, double E, const double *u3, double *xi);

/* --- rejection samplers (pair, brems, Compton); rng = {id_lo, id_hi, step,
 *     key0, key1} of the interacting step, trial j uses counter block 3 + j/2 */
int or_has_rejection(int model);
double or_reject_sample(const or_ctx *c, int model, double E, const uint32_t rng[5], double *xi,
                        int *trials);
/* --- exact samplers of all six models (the untabulated transport): the
 *     three above, and Moller, Bhabha and annihilation by rejection from
 *     their DCS, with the same random stream */
double or_exact_sample(const or_ctx *c, int model, double E, const uint32_t rng[5], double *xi,
                       int *trials);

/* --- untabulated range and continuous loss (charged types) ------------ */
double or_range_at(const or_ctx *c, int type, int mat, double E);  /* cm, by quadrature */
double or_eloss_exact(const or_ctx *c, int type, int mat, double E, double s); /* post-step energy */

/* --- RNG -------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* --- geometry -------------------------------------------------------- */
int or_n_subtotal(const or_ctx *c);
double or_plane_z(const or_ctx *c, int k);
int or_locate(const or_ctx *c, double z, double w);
double or_distance(const or_ctx *c, const double pos[3], const double dir[3], int sub,
                   int *next_sub, int *plane);
double or_safety(const or_ctx *c, const double pos[3], int sub);

/* --- uniform magnetic field: helix of a charged track (type 1 e-, 2 e+) */
double or_field_step_limit(const or_ctx *c, int type, double E, const double dir[3]);
void or_helix(const or_ctx *c, int type, double E, double s, const double dir[3], double dpos[3],
              double ndir[3]);

/* --- multiple scattering (Highland width, Gaussian angle and offset) -- */
double or_msc_theta0(const or_ctx *c, int mat, double T, double s);
int or_msc(const or_ctx *c, int sub, double E_pre, double E_post, double s, const double dir[3],
           const double pos[3], const double u[4], double out_dir[3], double out_pos[3]);

/* --- interactions given uniforms (unit level) ------------------------ */
int or_interact(const or_ctx *c, int type, int proc, double E, const double dir[3],
                const double u[8], const uint32_t rng[5], double *out /* 24 doubles */);

/* --- full transport --------------------------------------------------- */
int or_transport(const or_ctx *c, const or_primary *p, long n_prim, long n_events,
                 uint64_t seed, double *edep /* [n_events][n_subtotal] */,
                 double *cell_edep /* [n_layers][nx][ny] or NULL */,
                 double *escape_E /* [n_events] */,
                 long long *ev_counts /* [n_events][OR_NCOUNT] */,
                 int n_threads);
/* the events first_event .. first_event + n_events - 1 of a larger workload:
 * primaries carry global event indices, row i holds event first_event + i,
 * and the random streams are keyed by the global index */
int or_transport_events(const or_ctx *c, const or_primary *p, long n_prim, long first_event,
                        long n_events, uint64_t seed, double *edep, double *cell_edep, double *escape_E,
                        long long *ev_counts, int n_threads);

#ifdef __cplusplus
}
#endif
#endif
