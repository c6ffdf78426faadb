/*
 * gv.h -- C ABI of the GB300 (sm_103a) electromagnetic shower transport
 * library libgv.so: the per-track stepping loop of GeantV (arXiv:2005.00949,
 * Sec. 2.1.2 "Scalar and vector workflows", Fig. "simulation stages"), run for
 * thousands of events at once on one GPU.
 *
 * Conventions
 *  - Every call returns GV_OK (0) or a negative GV_ERR_* code; nothing throws
 *    across the ABI, nothing aborts the process, no kernel traps.
 *  - Energies in MeV (kinetic), lengths in cm, densities in g/cm3.
 *  - Particle types: 0 gamma, 1 electron, 2 positron.
 *  - A gv_ctx owns every device allocation it makes (tables, track queues,
 *    tallies); the caller owns primaries and result buffers.
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *    stream), e.g. torch.cuda.current_stream().cuda_stream.
 *  - Pointers documented "host or device" may be either: the library asks the
 *    CUDA driver which one it got (unified addressing).
 */
#ifndef GV_H
#define GV_H
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GV_OK 0
#define GV_ERR_BAD_ARG -1    /* an argument is out of range or inconsistent */
#define GV_ERR_NO_TABLES -2  /* gv_build_tables has not run */
#define GV_ERR_OOM -3        /* a device allocation failed */
#define GV_ERR_STACK_FULL -4 /* a track queue overflowed its capacity */
#define GV_ERR_TIMEOUT -5    /* generation budget exhausted before all tracks ended */
#define GV_ERR_NUMERIC -6    /* a track reached a non-finite energy or position */
#define GV_ERR_CUDA -7       /* a CUDA runtime call failed */
#define GV_ERR_INTERNAL -8   /* an index or state check failed (library built with GV_CHECKS) */

#define GV_MAX_ELEM 4
#define GV_MAX_MAT 4
#define GV_MAX_SUB 8
#define GV_MAX_SUBTOTAL 1024
#define GV_NCOUNT 12

/* process bits of gv_cuts.process_mask */
#define GV_P_COMPTON (1u << 0)
#define GV_P_PHOTO (1u << 1)
#define GV_P_PAIR (1u << 2)
#define GV_P_BREM (1u << 3)
#define GV_P_IONI (1u << 4)
#define GV_P_ANNIH (1u << 5)
#define GV_P_MSC (1u << 6)   /* Gaussian multiple scattering of e+- along the step (off by default) */
#define GV_P_INTEGRAL (1u << 7) /* integral approach for e+- cross sections along a step (off by default):
                                   steps drawn with the running maximum of Sigma below E, interactions
                                   accepted with the post-step cross sections */

/* arithmetic of the stepping loop */
#define GV_MIXED 0 /* FP32 physics, tables and energies; FP64 positions and boundaries */
#define GV_FP64 1  /* FP64 everywhere */

/* scheduling */
#define GV_BATCHED 0               /* all events share one population of tracks */
#define GV_ONE_EVENT_PER_LAUNCH 1  /* plain comparator: one event in flight at a time */

/* indices of gv_result.counters and of the per-event counter rows */
enum {
  GV_C_STEPS = 0, GV_C_STEPS_G, GV_C_STEPS_EM, GV_C_STEPS_EP,
  GV_C_TRK_G, GV_C_TRK_EM, GV_C_TRK_EP, GV_C_PAIR, GV_C_ANNIH,
  GV_C_EP_ESC, GV_C_UNSCAT, GV_C_GENERATIONS,
  /* gv_result.counters only: */
  GV_C_GEOM,        /* steps limited by a boundary */
  GV_C_DISCRETE,    /* steps ending in a discrete-process choice */
  GV_C_LANE_SLOTS,  /* 32 x warp iterations of the step loop (idle lanes = slots - steps) */
  GV_C_LIVE_PEAK    /* largest live-track population of a generation */
};

/* A material: n_elem elements with atomic number Z, atomic mass A (g/mol) and
 * mass fraction w; density rho (g/cm3); mean excitation energy I (eV). */
typedef struct {
  int n_elem;
  double Z[GV_MAX_ELEM], A[GV_MAX_ELEM], w[GV_MAX_ELEM];
  double rho;
  double I_eV;
} gv_material;

/* Layered box along +z from z = 0: n_layers repetitions of n_sub sub-slabs
 * (thickness sub_thick_cm[j], material sub_mat[j]).  Transverse half widths
 * half_x_cm/half_y_cm (<= 0: unbounded).  nx_cells x ny_cells scoring cells per
 * layer over the full transverse extent (0: no cell scoring).  An optional
 * uniform magnetic field of field_T tesla along the axis field_axis (0 x,
 * 1 y, 2 z; field propagation, Sec. 3.6): charged tracks follow the exact
 * helix of their pre-step momentum, with steps limited to a 10 um chord
 * sagitta and a 0.2 rad turn; boundaries are found along the straight line. */
typedef struct {
  int n_layers;
  int n_sub;
  double sub_thick_cm[GV_MAX_SUB];
  int sub_mat[GV_MAX_SUB];
  double half_x_cm, half_y_cm;
  int nx_cells, ny_cells;
  double field_T;
  int field_axis;
} gv_layers;

/* Production cuts (MeV): gamma_cut splits bremsstrahlung into continuous and
 * discrete parts, e_cut splits ionisation and decides whether Compton,
 * photo- and pair-produced leptons are tracked; track_cut (>= 1 keV) ends
 * tracks.  process_mask: GV_P_* bits of the enabled discrete processes, plus
 * GV_P_MSC for multiple scattering along charged steps.  reject_min_MeV[m]:
 * the final state of model m (GV_M_*) is sampled by rejection at energies
 * >= this, by sampling tables below (rejection is built for Compton, pair and
 * bremsstrahlung; a huge value keeps the tables everywhere).  Rejection trial
 * j draws from counter block 3 + j/2 of the interacting step. */
typedef struct {
  double gamma_cut_MeV, e_cut_MeV, track_cut_MeV;
  unsigned process_mask;
  double reject_min_MeV[6];
} gv_cuts;

/* final-state models (index of gv_cuts.reject_min_MeV and gv_unit_sample) */
#define GV_M_COMPTON 0
#define GV_M_PAIR 1
#define GV_M_BREM 2
#define GV_M_MOLLER 3
#define GV_M_BHABHA 4
#define GV_M_ANNIH 5

/* Launch and memory configuration; gv_default_config fills every field. */
typedef struct {
  int precision;              /* GV_MIXED or GV_FP64 */
  int mode;                   /* GV_BATCHED or GV_ONE_EVENT_PER_LAUNCH */
  int block_size;             /* threads per block: 64..512, multiple of 32 */
  int blocks_per_sm;          /* persistent blocks per SM */
  int steps_per_claim;        /* steps a thread takes on a claimed track per generation */
  int tail_steps_per_claim;   /* the same when fewer than tail_threshold tracks are live */
  long long tail_threshold;
  long long stack_capacity;   /* tracks per particle-type queue (each double-buffered) */
  long long refill_low_water; /* inject primaries while fewer live tracks than this */
  long long refill_batch;     /* at most this many primaries per generation */
  int generations_per_graph;  /* generations per body of the graph loop (even) */
  long long max_generations;  /* budget; exceeded -> GV_ERR_TIMEOUT */
  int per_event_counts;       /* 1: keep GV_NCOUNT counters per event (slower) */
  int process_sort;           /* 1: re-basket interacting tracks by process in each block */
  long long max_events_in_flight; /* refill only while fewer events are unfinished; 0: no cap;
                                     -1 (default): automatic. Every primary is budgeted 0.15
                                     live tracks per MeV of its energy + 64. gv_transport and
                                     gv_transport_events (GV_BATCHED) admit the next primaries
                                     while the budgets of the unfinished events fit in
                                     stack_capacity, and one at least when no track is live.
                                     gv_transport_static and GV_ONE_EVENT_PER_LAUNCH budget every
                                     event like the most energetic primary: stack_capacity /
                                     (0.15 per MeV + 64) events, at least 16 */
  int claim_chunks;           /* without process_sort: 1 (default) = every warp claims its own
                                 32-track chunks from 16 sliced counters; 0 = one claim per block */
  int along_steps;            /* with process_sort: steps an electron or positron may take without a
                                 discrete interaction before its block baskets the interactions
                                 (1..64; default 3) */
  int scoring;                /* energy tallies (1 is not available with a field):
                                 0 (default) = one FP64 atomic per deposit;
                                 1 = a lane merges consecutive deposits to the same (event,
                                 sub-slab) in a compensated sum, and after every step round its
                                 warp adds equal keys together before one FP64 atomic per key */
  int l2_persist;             /* 1: gv_transport's step kernels read the alias tables through a persisting
                                 L2 access-policy window; the context's persisting L2 set-aside is
                                 raised to the tables' size and restored by gv_destroy */
  int pipeline;               /* 0 (default): one fused step kernel per generation; 1: an
                                 along-step kernel hands the tracks due a discrete interaction to
                                 an interaction kernel that runs each warp on one (type, process)
                                 key (needs scoring = 0; stack_capacity requests per generation) */
  int local_stack;            /* 1 (default): with several rounds per claim, the basketizing kernel keeps the
                                 secondaries a block makes in a shared-memory stack and gives them to
                                 its idle lanes in the following rounds (the StackBuffer, Sec. 2.1.2)
                                 instead of leaving them to the next generation */
  int pdl;                    /* 1 (default): successive step kernels of a graph use programmatic dependent
                                 launch: a generation's blocks stage their tables while the previous
                                 generation drains, and wait for it before reading its plan */
  int device_loop;            /* 1 (default): the transport is one graph launch whose conditional WHILE
                                 node repeats generations_per_graph generations until the plan marks it
                                 done; 0: the host relaunches the generation graph and checks after
                                 1, 2, 4, ... graphs (the same kernels; ncu profiles kernels only in
                                 graphs without conditional nodes) */
  int blocking;               /* 0 (default): gv_transport returns once the transport is enqueued and
                                 gv_sync completes it; 1: gv_transport returns when it is done, with
                                 its result record filled (device_loop = 0 always behaves so) */
  int along_steps_photon;     /* the same for photons (1..64; default 5; 0: along_steps) */
} gv_config;

/* A primary track; layout shared with the seeded input generator.  Its random
 * streams are keyed by (seed, event) and counted from its track id, so an
 * event's result does not depend on the order of the array or on how events
 * are split between calls or GPUs (the per-track streams of Sec. 5.1). */
typedef struct {
  int type;
  double E_MeV;
  double x, y, z;   /* must lie inside the box (z in [0, Z_total]) */
  double u, v, w;   /* unit direction */
  unsigned event;   /* event index, < n_events */
  unsigned id;      /* track id of the primary within its event (0, 1, ...; distinct per event) */
} gv_primary;

/* Results of one gv_transport call.  Buffers are caller-owned, host or device,
 * zeroed by the library before it accumulates into them:
 *   edep         [n_events][n_layers*n_sub]  energy deposit per sub-slab (MeV)
 *   cell_edep    [n_layers][nx][ny] or NULL   summed over events (MeV)
 *   escape_E     [n_events] or NULL            kinetic energy leaving the box
 *   event_counts [n_events][GV_NCOUNT] or NULL (requires per_event_counts)
 * counters[], status and kernel_ms are filled on return. */
typedef struct {
  double *edep;
  double *cell_edep;
  double *escape_E;
  long long *event_counts;
  unsigned long long counters[16];
  int status;
  double kernel_ms;   /* device time of the step-kernel graphs (CUDA events on the work stream) */
} gv_result;

/* Fill *cfg with defaults (batched, mixed precision, autotuned launch shape). */
int gv_default_config(gv_config *cfg);

/* Create a context (the per-thread state of the paper's scheduler, Sec.
 * 2.1.1, here one per GPU and workload): validates the materials
 * (n_mats <= GV_MAX_MAT), geometry (n_layers*n_sub <= GV_MAX_SUBTOTAL) and
 * cuts, and allocates its stream and geometry arrays.  *ctx_out receives the
 * context, owned by the caller until gv_destroy.  cfg = NULL selects
 * defaults.  Uses the current CUDA device.  GV_ERR_BAD_ARG for an
 * inconsistent argument, GV_ERR_CUDA if the device cannot be set up; nothing
 * is allocated on failure. */
int gv_setup(void **ctx_out, const gv_material *mats, int n_mats, const gv_layers *geo,
             const gv_cuts *cuts, const gv_config *cfg);

/* Build the cross-section, range and alias sampling tables in FP64 on the host
 * (ComputeIntLen tables of Sec. 2.1.2, "sampling tables" of Sec. 3.5) and
 * upload them in the context's precision.  Synchronous. */
int gv_build_tables(void *ctx);

/* Transport n primaries (host or device array) of n_events events with the
 * given seed (the stepping loop of Sec. 2.1.2 stages, stack of Sec. 2.1.2,
 * scoring of Sec. 3.8.1), until every track has ended, and copy the tallies
 * into res's buffers.  The work is ordered after what the caller queued on
 * `stream` before the call, and `stream` waits for it: work the caller
 * queues on it later sees the tallies.  The call returns once the work is
 * enqueued (config blocking = 0, the default); res->counters, status and
 * kernel_ms are filled by gv_sync, which also returns the status, and the
 * tally buffers hold the results once `stream` has reached that point.  With
 * host tally buffers that are not page-locked the copies, and so the call,
 * finish before it returns.  A second transport on the same context first
 * completes the previous one (filling its result record).  The caller's
 * buffers must stay valid until then.  Transports of different contexts
 * on one GPU run one after another on the GPU (their kernels read the
 * transport's state from one constant-memory record per precision and GPU);
 * the calls themselves may come from any threads.  Returns GV_OK or an error
 * found before the work started (GV_ERR_BAD_ARG, GV_ERR_NO_TABLES,
 * GV_ERR_OOM, GV_ERR_CUDA); errors of the transport itself
 * (GV_ERR_STACK_FULL, GV_ERR_TIMEOUT, GV_ERR_NUMERIC) come from gv_sync. */
int gv_transport(void *ctx, const gv_primary *p, long long n, long long n_events,
                 unsigned long long seed, void *stream, gv_result *res);

/* gv_transport of the events first_event .. first_event + n_events - 1 (one
 * shard of a workload split by event range over several GPUs or calls):
 * primaries carry their global event index, tally row i holds event
 * first_event + i, and the random streams are keyed by the global index, so
 * the rows equal those of one transport of the whole workload.
 * gv_transport(...) is gv_transport_events(..., 0, n_events, ...). */
int gv_transport_events(void *ctx, const gv_primary *p, long long n, long long first_event,
                        long long n_events, unsigned long long seed, void *stream, gv_result *res);

/* gv_transport without any device allocation (the paper has no counterpart;
 * this entry point exists for embedding).  For callers that cannot let a
 * library call cudaMalloc/cudaFree while they run -- e.g. a host framework
 * that owns all of a GPU's memory through its own pools and budget; those
 * calls also synchronise the device and can fail under memory pressure.
 * The context must already exist (gv_setup and gv_build_tables allocate, once)
 * and use GV_MIXED.  All scratch memory -- track queues for 65,536 tracks per
 * particle type, the generation control block, and live-track counts for up
 * to 65,536 events -- sits in one file-scope device array of 25,440,256 bytes
 * that every GPU holds from the library's first use on it until the process
 * exits.  Every call asks the runtime for that array's device address on the
 * current device (a device reset gives it a new one).  Every call reuses the
 * array and clears what must start at zero.  Like gv_transport it takes the
 * GPU's constant-memory state record in turn with every other transport,
 * and holds it until it returns: calls from several threads, streams or
 * contexts run one after another and do not share the array's contents.  The call waits on the host between its launches, so it cannot
 * run on a stream that is being captured (GV_ERR_BAD_ARG) and must not run
 * while another stream of the device captures in global mode.
 *   prim      device array of n primaries;
 *   edep      device [n_events][n_layers*n_sub], zeroed, then accumulated;
 *   escape_E  device [n_events], zeroed, then accumulated;
 *   counters  host array of 16 (as gv_result.counters).
 * Runs the batched schedule on `stream` and returns when done; the events in
 * flight are capped at 65,536 / (0.15 per MeV of the most energetic primary
 * + 64), at least 16 (41 events of 10 GeV), so showers up to about 25 GeV per
 * event fit the array; beyond that GV_ERR_STACK_FULL may be returned.
 * GV_ERR_BAD_ARG: n_events > 65,536, host pointers, an FP64 context, or a
 * context with a magnetic field.  gv_sync reports the status of the last
 * transport, this one included. */
int gv_transport_static(void *ctx, const gv_primary *prim, long long n, long long n_events,
                        unsigned long long seed, void *stream, double *edep, double *escape_E,
                        unsigned long long *counters);

/* Complete the context's transport in flight, if any (the paper's
 * transport of a batch of events ends when its last track has, Sec. 2.1.1):
 * wait for it, fill its result record (counters, status, kernel_ms), then
 * wait for all work queued on `stream`.  Returns the status of the last
 * transport (GV_OK, GV_ERR_STACK_FULL, GV_ERR_TIMEOUT, GV_ERR_NUMERIC,
 * GV_ERR_INTERNAL), or GV_ERR_CUDA if a wait fails, GV_ERR_BAD_ARG for a
 * null context. */
int gv_sync(void *ctx, void *stream);

/* Release every resource of the context (what gv_setup and gv_build_tables
 * allocated, Sec. 2.1.1's per-thread state), after waiting for its work.  A
 * result record not yet collected by gv_sync stays unfilled.  ctx = NULL is
 * a no-op. */
void gv_destroy(void *ctx);

/* Static description of an error code. */
const char *gv_strerror(int code);

/* Number of kernel launches the last gv_transport issued. */
long long gv_last_launches(void *ctx);

/* ---- element-wise entry points (device pointers, asynchronous on stream) ----
 * They run the same device functions as gv_transport, in the context's
 * precision, one element per thread; inputs and outputs are FP64 arrays. */

/* Philox4x32-10 (Random123 family, Sec. 3.3.2): out[4i..4i+3] from counter
 * ctr[4i..4i+3] and key key[2i..2i+1]. */
int gv_unit_philox(const unsigned *ctr, const unsigned *key, unsigned *out, long long n,
                   void *stream);

/* Table lookup (ComputeIntLen, Spline::GetValueAt of Sec. 6.3) of particle
 * `type` in material `mat` at energies E[i]: out[4i..4i+3] = the four
 * interpolated table quantities (gamma: Compton, photo, pair, 0; e-: brems,
 * ionisation, range, 0; e+: brems, ionisation, annihilation, range). */
int gv_unit_xs_lookup(void *ctx, int type, int mat, const double *E, long long n, double *out,
                      void *stream);

/* Continuous loss (AlongStepAction): post-step kinetic energy after a step
 * s[i] from E[i]. */
int gv_unit_eloss(void *ctx, int type, int mat, const double *E, const double *s, long long n,
                  double *out, void *stream);

/* Alias-table sampling (Sec. 3.5) of model m (0 Compton, 1 pair, 2 brems,
 * 3 Moller, 4 Bhabha, 5 annihilation) at E[i] with uniforms u[3i..3i+2]
 * (grid choice, bin, in-bin): out[2i] = physical variable, out[2i+1] = xi. */
int gv_unit_alias_sample(void *ctx, int model, const double *E, const double *u, long long n,
                         double *out, void *stream);

/* Final state of process `proc` for particle `type` at E[i], direction
 * dir[3i..], uniforms u[8i..8i+7]: out[24i..] = {E' (-1 if the primary
 * ended), dir'[3], local deposit, n_children, then per child: type, E, dir[3]};
 * ret[i] = 1 survived, 0 ended, -1 no interaction possible. */
int gv_unit_interact(void *ctx, int type, int proc, const double *E, const double *dir,
                     const double *u, long long n, double *out, int *ret, void *stream);

/* Distance to the boundary of sub-slab sub[i] (GeomQuery, Box::DistanceToIn
 * of Sec. 3.2) from pos[3i..] along dir[3i..]; next[i] = sub-slab entered
 * (-1 = leaves the box), plane[i] = crossed z-plane index or -2/-3 for the
 * x/y walls. */
/* Multiple scattering over one charged step (the along-step part of GV_P_MSC,
 * independent of the context's process mask): for each i, a track of
 * kinetic energy E_pre[i] that ends the step of length s[i] cm in sub-slab
 * sub[i] with energy E_post[i], direction dir[3i..3i+2] and position
 * pos[3i..3i+2], scattered with the uniforms u[4i..4i+3] (in (0,1]).
 * Writes the new direction to out_dir[3i..] and the new position to
 * out_pos[3i..].  Device arrays; sub[i] outside the geometry gives NaN. */
int gv_unit_msc(void *ctx, const int *sub, const double *E_pre, const double *E_post, const double *s,
                const double *dir, const double *pos, const double *u, long long n, double *out_dir,
                double *out_pos, void *stream);

/* Helix of a charged track in the context's field: for each i, a track of
 * type `type` (1 e-, 2 e+) and kinetic energy E[i] moving along dir[3i..]
 * for a path s[i]; out[7i..7i+6] = displacement (3), new direction (3) and
 * the field's step limit at the start.  Device arrays. */
int gv_unit_field(void *ctx, int type, const double *E, const double *s, const double *dir, long long n,
                  double *out, void *stream);

/* The reduced-variable sampler of model `model` at energies E[i]: method 0
 * sampling tables (uniforms from counter block 0 of (i, 0, 0) under key
 * (seed, seed >> 32)), method 1 rejection (block 3 + j/2 for trial j, same
 * stream; Compton, pair and bremsstrahlung only).  out[3i..3i+2] = physical
 * variable, reduced variable, trials (1 for the tables). */
int gv_unit_sample(void *ctx, int model, int method, const double *E, long long n, unsigned long long seed,
                   double *out, void *stream);

int gv_unit_distance(void *ctx, const double *pos, const double *dir, const int *sub,
                     long long n, double *dist, int *next, int *plane, void *stream);

#ifdef __cplusplus
}
#endif
#endif
