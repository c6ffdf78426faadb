// gv_state.cuh -- device-resident state of a transport call: the
// double-buffered per-type track queues (the StackBuffer / stage baskets of
// GeantV Sec. 2.1.2, as structures of arrays), the generation control block
// and the tally pointers.
#pragma once
#include "gv_device.cuh"

namespace gv {

// Structure-of-arrays queue of one particle type.
template <typename R> struct Queue {
  double *x, *y, *z;
  R *u, *v, *w, *E, *nlam;
  unsigned long long *id;
  unsigned *ev, *step;
  int *sf;  // sub-slab | flags << 16
};

// reciprocal node energies staged in shared memory, padded to 16 bytes
constexpr unsigned kInvNodeBytes = (kGridN * sizeof(float) + 15) / 16 * 16;

constexpr int kFlagPrimary = 1;
constexpr int kFlagInteracted = 2;

template <typename R> constexpr size_t track_bytes() {
  return 3 * sizeof(double) + 5 * sizeof(R) + sizeof(unsigned long long) + 3 * sizeof(unsigned);
}

// Claim counters of the work slices, one per 128-byte line.
constexpr int kNClaim = 16;
struct alignas(128) ClaimSlot {
  unsigned n;
};

// An interaction request of the split pipeline: the along-step kernel hands
// a track that is due a discrete interaction to the interaction kernel
// (one 16-byte-aligned record per request).
template <typename R> struct alignas(16) GReq {
  double x, y, z;
  unsigned long long id;
  R E, d0, d1, d2;
  R u[6];        // u2..u7 of the step
  unsigned ev, kk;
  int sf;        // sub-slab | flags << 16
  int key;       // type * 3 + process
};
constexpr int kNReqKey = 9;

// Generation control block.  The last block of every generation writes the
// plan of the next one; kernels only read it.
struct Ctl {
  ClaimSlot claims[kNClaim];
  unsigned cnt[2][3];        // queue fill per buffer parity and type
  unsigned prim_next;        // primaries handed out so far
  unsigned prim_begin, prim_count;
  unsigned chunk_end[4];     // cumulative chunk counts in claim order: e+, e-, gamma, primaries
  unsigned claim;            // chunk claim counter
  unsigned blocks_done;
  int K;                     // steps per claimed track this generation
  unsigned chunk_B;          // tracks per block claim this generation
  int status;
  int done;
  int pad;
  unsigned ev_started, ev_done;  // events whose live-track count left / returned to zero
  unsigned max_in_flight;        // refill cap of this call (0: none)
  unsigned emax_bits;            // largest primary energy (FP32 bits), for the automatic cap
  unsigned long long gen;
  unsigned long long loop_iter;  // bodies of the device-side generation loop run so far
  unsigned long long live_peak;
  unsigned long long counters[16];
  // split pipeline: requests of this generation, per key, and the claim /
  // completion counters of the interaction kernel
  unsigned req_n;
  unsigned key_n[kNReqKey];
  unsigned claim_b, blocks_done_b;
  unsigned long long cost_started, cost_done;  // automatic cap: track budget taken by / returned from events
};

template <typename R> struct DevState {
  View<R> view;              // global-memory table pointers and constants
  Queue<R> q[2][3];
  unsigned long long capacity;
  Ctl *ctl;
  const gv_primary *prim;
  const unsigned *order;     // primary visiting order (one-event mode) or null
  unsigned n_prim, n_events;
  unsigned ev_base;          // event index of tally row 0 (the random streams use ev_base + row)
  double *edep, *cell, *escape;
  unsigned long long *evcnt;
  unsigned *evlive;          // live tracks per event (events-in-flight accounting)
  int max_in_flight;         // 0: no cap, -1: automatic from the primaries' energies
  unsigned seed_lo, seed_hi;
  int block_size, mode, K_bulk, K_tail;
  int chunk;                 // tracks per work chunk: 32 (a warp) or block_size (basketizer)
  int claim_chunks;          // chunks a warp takes per atomic claim (no basketizer)
  int along_steps;           // basketizer: steps per lane before the block basket
  int scoring;               // 0 direct atomics, 1 warp-merged (selects the kernel)
  int pipeline;              // 0 fused step kernel, 1 along-step + interaction kernels
  GReq<R> *req;              // split pipeline: request records [req_cap]
  unsigned *keyidx;          // split pipeline: request indices per key [kNReqKey][req_cap]
  unsigned long long req_cap;
  unsigned long long tail_threshold, low_water, batch, max_gen;
  int n_mat;
  unsigned xs_bytes, zb_bytes;  // staged into shared memory
  unsigned smem_req_off;        // start of the basketizer's request records
  unsigned smax_off, smax_bytes; // the integral approach's bound, staged into shared memory
  unsigned smem_lk_off;          // the block's secondary stack (local_stack)
  int local_stack;
  int grid, adaptive_chunk;  // blocks of the step kernel; spread small populations over all of them
  const unsigned long long *pcost;  // automatic cap: prefix sums of the primaries' track budgets [n_prim + 1], or null
  unsigned long long *evcost;       // automatic cap: budget held by each event in flight [n_events]
  int along_steps_g;                // basketizer: along-step budget of photons
};

}  // namespace gv
