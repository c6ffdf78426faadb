// gv_transport.cu -- the stepping loop of GeantV (Sec. 2.1.2, Fig.
// "simulation stages") as a persistent, chunk-claiming CUDA kernel driven
// generation by generation from a captured CUDA graph (a device-side while
// loop over bodies of generations), plus the C ABI.
//
// One generation: every live track of the three per-type queues (and the
// primaries injected by the refill plan) is claimed in chunks (a block's
// worth, fewer when few tracks are live; positrons, electrons, photons,
// primaries in that order), stepped K times, and written back -- survivors
// and secondaries appended to the other parity's queues with warp-aggregated
// atomics (the basketizer of scheduler v3, Sec. 2.1.1).  The last block to
// finish writes the plan of the next generation: queue chunk ranges and
// claim size, primaries to inject (the event server refill, bounded by a
// live-track budget) and the steps per claim.
//
// Host side: gv_transport enqueues one transport on the context's stream,
// ordered after the caller's stream (which then waits for it), and returns;
// gv_sync waits for it and fills the caller's result record from the
// control block copied back to pinned memory.  The step kernels read the
// transport's state record from constant memory, one copy per precision and
// GPU; transports of different contexts on one GPU take turns on it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "gv_state.cuh"

namespace gv {

// ------------------------------------------------------------------ sinks
struct BlockCnt {
  unsigned long long c[16];
};

// Scoring (SteppingActions, Sec. 3.8.1).  A lane keeps one pending
// (event, sub-slab) deposit: consecutive deposits of its track to the same sub-slab merge with a
// compensated (Kahan) sum in R; a deposit to another sub-slab flushes the
// pending one with an FP64 atomic; at the end of every round the warp groups
// its pending deposits by key (__match_any_sync), sums each group with a
// compensated shuffle reduction, and one lane per group adds it to the FP64
// tally.  pd == nullptr scores directly.
constexpr unsigned long long kNoKey = ~0ull;

template <typename R> struct Pending {
  unsigned long long key;
  R sum, comp;
};

template <typename R> __device__ __forceinline__ void kahan_add(R &sum, R &comp, R v) {
  const R y = v - comp;
  const R t = sum + y;
  comp = (t - sum) - y;
  sum = t;
}

// EXT: compiled with the cell histogram and the per-event counters; a
// kernel without them serves contexts that have neither.
template <typename R, bool EXT = true>
__device__ __forceinline__ void deposit(const View<R> &V, const DevState<R> *S, unsigned ev, int sub, double px,
                                        double py, R dE, Pending<R> *pd = nullptr) {
  if (!(dE != R(0)) || sub < 0) return;
  GV_CHECK(&S->ctl->status, ev < S->n_events && sub < V.geo.nsub);
  const unsigned long long key = static_cast<unsigned long long>(ev) * V.geo.nsub + sub;
  if (pd) {
    if (pd->key == key) {
      kahan_add(pd->sum, pd->comp, dE);
    } else {
      if (pd->key != kNoKey)
        atomicAdd(&S->edep[pd->key], f2d(pd->sum) - f2d(pd->comp));
      pd->key = key;
      pd->sum = dE;
      pd->comp = R(0);
    }
  } else {
    atomicAdd(&S->edep[key], f2d(dE));
  }
  if (EXT && S->cell) {
    const GeoConst &g = V.geo;
    const int layer = sub / g.nsub_layer;
    // the offset from the wall in FP64, the cell index in FP32 (a cell
    // edge moves by ~1e-7 of the box width; no FP64 division)
    int ix = __float2int_rd(static_cast<float>(px + g.hx) * g.inv_pitch_x);
    int iy = __float2int_rd(static_cast<float>(py + g.hy) * g.inv_pitch_y);
    ix = ix < 0 ? 0 : (ix >= g.nx ? g.nx - 1 : ix);
    iy = iy < 0 ? 0 : (iy >= g.ny ? g.ny - 1 : iy);
    atomicAdd(&S->cell[(static_cast<size_t>(layer) * g.nx + ix) * g.ny + iy], f2d(dE));
  }
}

// Warp flush of the pending deposits (all 32 lanes, converged).
template <typename R> __device__ __forceinline__ void warp_flush(const DevState<R> *S, Pending<R> &p) {
  const unsigned m = __match_any_sync(0xffffffffu, p.key);
  if (p.key != kNoKey) {
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    const R v = p.sum - p.comp;
    R acc = v, comp = R(0);
    unsigned rest = m & ~(1u << leader);
    while (rest) {  // every lane of the group runs the same iterations
      const int src = __ffs(rest) - 1;
      rest &= rest - 1u;
      const R w = __shfl_sync(m, v, src);
      if (lane == leader) kahan_add(acc, comp, w);
    }
    if (lane == leader) atomicAdd(&S->edep[p.key], f2d(acc) - f2d(comp));
  }
  p.key = kNoKey;
}

template <typename R, bool EXT = true>
__device__ __forceinline__ void count(const DevState<R> *S, BlockCnt *bc, unsigned ev, int c, unsigned long long n = 1) {
  atomicAdd(&bc->c[c], n);
  if (EXT && S->evcnt) atomicAdd(&S->evcnt[static_cast<size_t>(ev) * GV_NCOUNT + c], n);
}

template <typename R> struct Trk {
  double x, y, z;
  R u, v, w, E, nlam;
  unsigned long long id;
  unsigned ev, step;
  int sub, flags, type;
};

__device__ __forceinline__ void set_status(Ctl *ctl, int code) { atomicCAS(&ctl->status, 0, code); }

// Integral approach at the post-step point: the process whose cumulative
// post-step cross section first exceeds `target` (u Sigma_max), or -1 (no
// interaction) above their sum.  Out of line: the option would otherwise
// cost every step kernel registers.
template <typename R> __device__ __noinline__ int integral_choice(const View<R> &V, int mat, int type, R E, R target) {
  int i;
  R f;
  grid_pos(V, E, i, f);
  const V4<R> p4 = lookup_at(V, mat, type, i, f);
  R cum = p4.x;
  if (target < cum) return 0;
  cum += p4.y;
  if (target < cum) return 1;
  if (type == 2) {
    cum += p4.z;
    if (target < cum) return 2;
  }
  return -1;
}

// ------------------------------------------------------------------ one step
// PreStep .. process choice of one step.  Returns 1 if the track is still
// alive; then proc >= 0 names the discrete process due at the post-step
// point and u[] holds the step's eight uniforms for its final state.
// Secondaries made so far go to `kids`; kk is the step index whose counter
// blocks derive the children's ids.
// FIELD: compiled with the magnetic-field propagation (a field-free kernel
// keeps its registers for the rest of the step).  OPTS: compiled with the
// optional processes (multiple scattering, the integral approach); the plain
// kernel leaves their code out.
template <typename R, bool FIELD, bool OPTS, bool EXT>
__device__ int step_track(const View<R> &V, const DevState<R> *S, Trk<R> &t, Kids<R> &kids, uint32_t &kk,
                          BlockCnt *bc, int &proc_out, R *u, int &lim_out, Pending<R> *pd) {
  kids.n = 0;
  proc_out = -1;
  lim_out = -1;
  const uint32_t k = t.step;
  kk = k;
  const uint32_t key0 = S->seed_lo ^ (t.ev + S->ev_base), key1 = S->seed_hi;
  const uint32_t idlo = static_cast<uint32_t>(t.id), idhi = static_cast<uint32_t>(t.id >> 32);
  // counter block 0 is drawn only when the step needs it: a new n_lambda, or
  // a physics-limited step (process choice and alias uniforms)
  uint4 r0 = make_uint4(0u, 0u, 0u, 0u);
  bool have_r0 = false;
  const R tcut = V.rc.tcut;
  if (t.E < tcut) {  // PreStep: tracking cut
    deposit<R, EXT>(V, S, t.ev, t.sub, t.x, t.y, t.E, pd);
    if (t.type == 2) {
      const uint4 r1 = philox4x32_10(make_uint4(idlo, idhi, k, 1u), key0, key1);
      at_rest(kids, u24<R>(r1.z), u24<R>(r1.w));
      count<R, EXT>(S, bc, t.ev, GV_C_ANNIH);
    }
    return 0;
  }
  const int mat = V.smat[t.sub];
  // ComputeIntLen
  if (t.nlam <= R(0)) {
    r0 = philox4x32_10(make_uint4(idlo, idhi, k, 0u), key0, key1);
    have_r0 = true;
    t.nlam = -m_log(u24<R>(r0.x));
  }
  int gi;  // the pre-step energy's grid position serves the lookup and the loss
  R gf;
  grid_pos(V, t.E, gi, gf);
  const V4<R> s4 = lookup_at(V, mat, t.type, gi, gf);
  const R sig0 = s4.x, sig1 = s4.y, sig2 = (t.type == 1) ? R(0) : s4.z;
  const R Sig = sig0 + sig1 + sig2;
  const R INF = r_inf<R>();
  const bool charged = t.type != 0;
  // integral approach: the step is drawn with the bound Sigma_max(E) of the
  // cross sections the track can reach; the interaction is accepted at the
  // post-step point
  const bool integral = OPTS && charged && (V.cut.mask & GV_P_INTEGRAL);
  R Smax = Sig;
  if (integral) {
    const R *m = V.smax + (mat * 2 + t.type - 1) * kGridN;
    Smax = m[gi] + gf * (m[gi + 1] - m[gi]);
  }
  const R s_phys = Smax > R(0) ? q_div(t.nlam, Smax) : INF;
  R s_cont = INF, Rr = R(0);
  if (charged) {
    Rr = range_of(s4, t.type);
    const R a = static_cast<R>(kAlphaR) * Rr, b = Rr < static_cast<R>(kRhoF) ? Rr : static_cast<R>(kRhoF);
    s_cont = a > b ? a : b;
    if (FIELD && V.rc.field_k != R(0)) {  // the field's step limit acts like the continuous one
      const R sf = field_limit(V, t.type, t.E, t.u, t.v, t.w);
      s_cont = sf < s_cont ? sf : s_cont;
    }
  }
  // GeomQuery
  int next, plane;
  const R s_geom = distance(V, t.x, t.y, t.z, t.u, t.v, t.w, t.sub, next, plane);
  R s = s_cont < s_geom ? s_cont : s_geom;
  s = s_phys < s ? s_phys : s;
  const int lim = (s_geom == s) ? 0 : (s_phys == s ? 1 : 2);
  lim_out = lim;
  if (!(s < INF)) {
    atomicAdd(&S->escape[t.ev], f2d(t.E));
    if (t.type == 2) count<R, EXT>(S, bc, t.ev, GV_C_EP_ESC);
    return 0;
  }
  // Propagation: FP64 positions, advanced by displacements s d formed in R
  // (s and d are R already; an FP32 displacement is widened exactly on the
  // integer ALU, leaving the FP64 pipe one addition per coordinate; in FP64
  // mode this is one fused multiply-add)
  double mx = 0.0, my = 0.0;  // step midpoint: only cell scoring reads it
  if (FIELD && charged && V.rc.field_k != R(0)) {  // the helix of the pre-step momentum
    const R d0[3] = {t.u, t.v, t.w};
    R dp[3], nd[3];
    if (EXT && S->cell) {
      helix(V, t.type, t.E, R(0.5) * s, d0, dp, nd);
      mx = t.x + f2d(dp[0]);
      my = t.y + f2d(dp[1]);
    }
    helix(V, t.type, t.E, s, d0, dp, nd);
    t.x += f2d(dp[0]);
    t.y += f2d(dp[1]);
    t.z += f2d(dp[2]);
    if (lim == 0) {  // the crossed plane, chosen with the pre-step direction
      if (plane >= 0) t.z = V.zb[plane];
      else if (plane == -2) t.x = V.geo.wx[t.u > R(0) ? 1 : 0];
      else if (plane == -3) t.y = V.geo.wy[t.v > R(0) ? 1 : 0];
    }
    t.u = nd[0];
    t.v = nd[1];
    t.w = nd[2];
  } else {
    if (EXT && S->cell) {
      mx = t.x + f2d(R(0.5) * s * t.u);
      my = t.y + f2d(R(0.5) * s * t.v);
    }
    t.x += f2d(s * t.u);
    t.y += f2d(s * t.v);
    t.z += f2d(s * t.w);
    if (lim == 0) {
      if (plane >= 0) t.z = V.zb[plane];
      else if (plane == -2) t.x = V.geo.wx[t.u > R(0) ? 1 : 0];
      else if (plane == -3) t.y = V.geo.wy[t.v > R(0) ? 1 : 0];
    }
  }
  if (Smax > R(0)) t.nlam = (lim == 1) ? R(0) : t.nlam - s * Smax;
  t.step = k + 1;
  // the block's step counters are summed per warp by the caller; only the
  // optional per-event rows are booked here
  if (EXT && S->evcnt) {
    atomicAdd(&S->evcnt[static_cast<size_t>(t.ev) * GV_NCOUNT + GV_C_STEPS], 1ull);
    atomicAdd(&S->evcnt[static_cast<size_t>(t.ev) * GV_NCOUNT + GV_C_STEPS_G + t.type], 1ull);
  }
  const int pre_sub = t.sub;
  const R E_pre = t.E;
  // AlongStepAction
  if (charged) {
    const R Ep = eloss_at(V, mat, t.type, t.E, gi, gf, s, Rr);
    deposit<R, EXT>(V, S, t.ev, pre_sub, mx, my, t.E - Ep, pd);
    t.E = Ep;
    if (t.E < tcut) {
      deposit<R, EXT>(V, S, t.ev, pre_sub, t.x, t.y, t.E, pd);
      if (t.type == 2) {
        const uint4 r1 = philox4x32_10(make_uint4(idlo, idhi, k, 1u), key0, key1);
        at_rest(kids, u24<R>(r1.z), u24<R>(r1.w));
        count<R, EXT>(S, bc, t.ev, GV_C_ANNIH);
      }
      return 0;
    }
    // multiple scattering of a track that stays in the box (counter block 2)
    if (OPTS && (V.cut.mask & GV_P_MSC) && !(lim == 0 && next < 0)) {
      const uint4 r2 = philox4x32_10(make_uint4(idlo, idhi, k, 2u), key0, key1);
      const R um[4] = {u24<R>(r2.x), u24<R>(r2.y), u24<R>(r2.z), u24<R>(r2.w)};
      R dm[3] = {t.u, t.v, t.w};
      msc_step(V, pre_sub, E_pre, t.E, s, dm, t.x, t.y, t.z, um);
      t.u = dm[0];
      t.v = dm[1];
      t.w = dm[2];
    }
  }
  if (lim == 0) {
    if (next < 0) {
      atomicAdd(&S->escape[t.ev], f2d(t.E));
      if (t.type == 2) count<R, EXT>(S, bc, t.ev, GV_C_EP_ESC);
      if ((t.flags & kFlagPrimary) && !(t.flags & kFlagInteracted) && plane == V.geo.nsub)
        count<R, EXT>(S, bc, t.ev, GV_C_UNSCAT);
      return 0;
    }
    t.sub = next;
    return 1;
  }
  if (lim != 1) return 1;
  // PostStepActions: process choice, then the final state
  if (!have_r0) r0 = philox4x32_10(make_uint4(idlo, idhi, k, 0u), key0, key1);
  int proc = -1;
  if (integral) {  // post-step cross sections; above their sum: no interaction
    proc = integral_choice(V, mat, t.type, t.E, u24<R>(r0.y) * Smax);
  } else {
    const R target = u24<R>(r0.y) * Sig;
    R cum = sig0;
    if (target < cum) proc = 0;
    else {
      cum += sig1;
      if (target < cum) proc = 1;
      else {
        cum += sig2;
        if (target < cum) proc = 2;
      }
    }
    if (proc < 0) proc = sig2 > R(0) ? 2 : (sig1 > R(0) ? 1 : (sig0 > R(0) ? 0 : -1));
  }
  t.nlam = R(-1);
  if (proc < 0) return 1;
  const uint4 r1 = philox4x32_10(make_uint4(idlo, idhi, k, 1u), key0, key1);
  u[0] = u24<R>(r0.x); u[1] = u24<R>(r0.y); u[2] = u24<R>(r0.z); u[3] = u24<R>(r0.w);
  u[4] = u24<R>(r1.x); u[5] = u24<R>(r1.y); u[6] = u24<R>(r1.z); u[7] = u24<R>(r1.w);
  proc_out = proc;
  return 1;
}

// PostStepActions of a track whose step ended in process `proc`: the final
// state, the local deposit and the counters.  Returns 1 if the particle
// survives, 0 if it ended, -1 if the process was kinematically closed at the
// post-step energy (nothing changes).
template <typename R, bool OPTS = true, bool EXT = true>
__device__ __forceinline__ int final_state(const View<R> &V, const DevState<R> *S, BlockCnt *bc, int type, int proc,
                                           R &E, R d[3], const R *u, Kids<R> &kids, unsigned ev, int sub,
                                           double x, double y, unsigned long long id, uint32_t kk,
                                           Pending<R> *pd = nullptr) {
  R local;
  int np = 0, na = 0;
  const RngKey g = {static_cast<uint32_t>(id), static_cast<uint32_t>(id >> 32), kk, S->seed_lo ^ (ev + S->ev_base),
                    S->seed_hi};
  const int r = interact<R, OPTS>(V, type, proc, E, d, u, g, kids, local, np, na);
  if (r < 0) return -1;
  if (np) count<R, EXT>(S, bc, ev, GV_C_PAIR, np);
  if (na) count<R, EXT>(S, bc, ev, GV_C_ANNIH, na);
  deposit<R, EXT>(V, S, ev, sub, x, y, local, pd);
  return r;
}

// ------------------------------------------------------------------ queues
// Warp-aggregated append: each lane contributes c_q records of type q; one
// atomic per warp and type reserves the slots.  Must be called by all 32
// lanes of a converged warp.
__device__ __forceinline__ unsigned warp_reserve(unsigned *counter, unsigned c, unsigned &total) {
  const int lane = threadIdx.x & 31;
  unsigned incl = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  total = __shfl_sync(0xffffffffu, incl, 31);
  unsigned base = 0;
  if (lane == 31 && total) base = atomicAdd(counter, total);
  base = __shfl_sync(0xffffffffu, base, 31);
  return base + incl - c;
}

template <typename R>
__device__ __forceinline__ void store(const Queue<R> &q, unsigned slot, double x, double y, double z, R u, R v, R w,
                                      R E, R nlam, unsigned long long id, unsigned ev, unsigned step, int sf) {
  q.x[slot] = x;
  q.y[slot] = y;
  q.z[slot] = z;
  q.u[slot] = u;
  q.v[slot] = v;
  q.w[slot] = w;
  q.E[slot] = E;
  q.nlam[slot] = nlam;
  q.id[slot] = id;
  q.ev[slot] = ev;
  q.step[slot] = step;
  q.sf[slot] = sf;
}

// The parent of a step's secondaries: where they start and whose lineage
// names them.
struct Parent {
  double x, y, z;
  unsigned long long id;
  unsigned ev;
  int sub;
};

template <typename R> __device__ __forceinline__ Parent parent_of(const Trk<R> &t) {
  Parent p;
  p.x = t.x; p.y = t.y; p.z = t.z;
  p.id = t.id;
  p.ev = t.ev;
  p.sub = t.sub;
  return p;
}

// A secondary kept in the block's shared-memory stack (the StackBuffer of
// Sec. 2.1.2 for one block): its lanes take it up in a later round of the
// same claim instead of leaving it to the next generation.
template <typename R> struct LKid {
  double x, y, z;
  unsigned long long id;
  R u, v, w, E;
  unsigned ev;
  int sub, type;
};

// The block's secondary stack: `top` entries (it may run past `cap` while
// appends overflow to the global queues, and below 0 while empty lanes try
// to pop; both are only ever read through the bounds below).
template <typename R> struct LocalStack {
  LKid<R> *e;
  int *top;
  int cap;
};

// PostStepActions: append the step's secondaries to the output queues, or,
// with a local stack, to the block's stack while it has room.  Called by all
// 32 lanes of a converged warp (lanes without secondaries pass kids.n == 0).
template <typename R, bool EXT = true>
__device__ void push_kids(const DevState<R> *S, int out, const Parent &t, const Kids<R> &kids, uint32_t kk,
                          BlockCnt *bc, const LocalStack<R> *ls = nullptr) {
  const unsigned any = __ballot_sync(0xffffffffu, kids.n > 0);
  if (!any) return;
  uint32_t w[6] = {0, 0, 0, 0, 0, 0};
  if (kids.n > 0) {
    const uint32_t key0 = S->seed_lo ^ (t.ev + S->ev_base);
    const uint4 a = philox4x32_10(make_uint4(static_cast<uint32_t>(t.id), static_cast<uint32_t>(t.id >> 32), kk, kTagId),
                                  key0, S->seed_hi);
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
    if (kids.n > 2) {
      const uint4 b = philox4x32_10(
          make_uint4(static_cast<uint32_t>(t.id), static_cast<uint32_t>(t.id >> 32), kk, kTagId + 1u), key0, S->seed_hi);
      w[4] = b.x; w[5] = b.y;
    }
  }
  // the block's stack first, while it has room (the ids above keep each
  // kid's index in the list, so where it goes changes no result)
  unsigned local = 0;  // bit j: kid j went to the block's stack
  if (ls) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      if (j >= kids.n) continue;
      const int slot = atomicAdd(ls->top, 1);
      if (slot < 0 || slot >= ls->cap) continue;
      LKid<R> &e = ls->e[slot];
      e.x = t.x; e.y = t.y; e.z = t.z;
      e.id = static_cast<unsigned long long>(w[2 * j]) | (static_cast<unsigned long long>(w[2 * j + 1]) << 32);
      e.u = kids.d[j][0]; e.v = kids.d[j][1]; e.w = kids.d[j][2];
      e.E = kids.E[j];
      e.ev = t.ev;
      e.sub = t.sub;
      e.type = kids.type[j];
      atomicAdd(&bc->c[GV_C_TRK_G + kids.type[j]], 1ull);
      if (EXT && S->evcnt) atomicAdd(&S->evcnt[static_cast<size_t>(t.ev) * GV_NCOUNT + GV_C_TRK_G + kids.type[j]], 1ull);
      local |= 1u << j;
    }
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    unsigned c = 0;
#pragma unroll
    for (int j = 0; j < 3; ++j) c += (j < kids.n && kids.type[j] == q && !(local >> j & 1u)) ? 1u : 0u;
    if (!__ballot_sync(0xffffffffu, c > 0)) continue;
    unsigned total;
    unsigned slot = warp_reserve(&S->ctl->cnt[out][q], c, total);
    if ((threadIdx.x & 31) == 0 && total) atomicAdd(&bc->c[GV_C_TRK_G + q], static_cast<unsigned long long>(total));
    if (c == 0) continue;
    if (slot + c > S->capacity) {
      set_status(S->ctl, GV_ERR_STACK_FULL);
      continue;
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      if (!(j < kids.n && kids.type[j] == q) || (local >> j & 1u)) continue;
      const unsigned long long id = static_cast<unsigned long long>(w[2 * j]) |
                                    (static_cast<unsigned long long>(w[2 * j + 1]) << 32);
      store(S->q[out][q], slot, t.x, t.y, t.z, kids.d[j][0], kids.d[j][1], kids.d[j][2], kids.E[j], R(-1), id, t.ev,
            0u, t.sub);
      if (EXT && S->evcnt) atomicAdd(&S->evcnt[static_cast<size_t>(t.ev) * GV_NCOUNT + GV_C_TRK_G + q], 1ull);
      ++slot;
    }
  }
  // the event's live-track count grows before the parent's own end is booked
  if (kids.n > 0) atomicAdd(&S->evlive[t.ev], static_cast<unsigned>(kids.n));
}

// The automatic events-in-flight cap (the paper keeps a bounded number of
// events in flight, Sec. 2.1.1): a primary of energy E is budgeted 0.15
// live tracks per MeV (about 2.3 times the peak live-track count of a
// shower per MeV) plus 64, and new primaries are admitted while the budgets
// of the events in flight fit the queue capacity.  NaN or negative energies
// get the base budget.
__device__ __forceinline__ unsigned long long prim_cost(double E) {
  const double e = (E > 0.0 && E < 1e12) ? E : 0.0;
  return 64ull + static_cast<unsigned long long>(ceil(0.15 * e));
}

// An event's last track ended: the event leaves the set in flight and
// returns its budget.  Out of line: it runs once per event, and inlined at
// both of its call sites it slowed the step kernel by 0.5 %.
template <typename R> __device__ __noinline__ void event_closed(const DevState<R> *S, unsigned ev) {
  atomicAdd(&S->ctl->ev_done, 1u);
  if (S->evcost) atomicAdd(&S->ctl->cost_done, atomicExch(&S->evcost[ev], 0ull));
}

// A primary was loaded: its budget goes to its event (returned when the
// event closes), or straight back if it never entered the box.
template <typename R>
__device__ __forceinline__ void primary_cost(const DevState<R> *S, unsigned ev, double E, bool entered) {
  if (!S->evcost) return;
  if (entered) atomicAdd(&S->evcost[ev], prim_cost(E));
  else atomicAdd(&S->ctl->cost_done, prim_cost(E));
}

// A track ended: book it against its event; the last one closes the event.
template <typename R> __device__ __forceinline__ void track_ended(const DevState<R> *S, unsigned ev) {
  if (atomicSub(&S->evlive[ev], 1u) == 1u) event_closed(S, ev);
}

// An interaction request staged in shared memory by the in-block basketizer.
template <typename R> struct IReq {
  double x, y, z;
  unsigned long long id;
  R E, d0, d1, d2;
  R u[6];      // u2..u7 of the step
  unsigned ev, kk;
  int sub;
  int tp;      // in: type*3 + process; out: final_state's return code
};
constexpr int kNKey = 9;

template <typename R>
__device__ __forceinline__ void push_survivor(const DevState<R> *S, int out, const Trk<R> &t, bool alive) {
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const bool mine = alive && t.type == q;
    if (!__ballot_sync(0xffffffffu, mine)) continue;
    unsigned total;
    const unsigned slot = warp_reserve(&S->ctl->cnt[out][q], mine ? 1u : 0u, total);
    if (!mine) continue;
    if (slot >= S->capacity) {
      set_status(S->ctl, GV_ERR_STACK_FULL);
      continue;
    }
    store(S->q[out][q], slot, t.x, t.y, t.z, t.u, t.v, t.w, t.E, t.nlam, t.id, t.ev, t.step,
          t.sub | (t.flags << 16));
  }
}

// A block-stack secondary written to the output queue (e == nullptr:
// nothing).  All 32 lanes of a converged warp.
template <typename R> __device__ __forceinline__ void push_lkid(const DevState<R> *S, int out, const LKid<R> *e) {
  const int type = e ? e->type : -1;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const bool mine = type == q;
    if (!__ballot_sync(0xffffffffu, mine)) continue;
    unsigned total;
    const unsigned slot = warp_reserve(&S->ctl->cnt[out][q], mine ? 1u : 0u, total);
    if (!mine) continue;
    if (slot >= S->capacity) {
      set_status(S->ctl, GV_ERR_STACK_FULL);
      continue;
    }
    store(S->q[out][q], slot, e->x, e->y, e->z, e->u, e->v, e->w, e->E, R(-1), e->id, e->ev, 0u, e->sub);
  }
}

// ------------------------------------------------------------------ planning
// The order in which a generation's chunks are claimed: positrons, electrons,
// photons, then new primaries.  Charged-particle claims take longest (loss,
// more interactions per step), so they go first and the last claims of a
// generation, whose spread leaves blocks idle at its end, are the short
// photon ones (measured: 4 % less transport time than photons first).
__device__ __forceinline__ int claim_queue(int seg) { return seg < 3 ? 2 - seg : 3; }

template <typename R> __device__ void plan_next(const DevState<R> *S, int pn) {
  Ctl *c = S->ctl;
  const unsigned n0 = c->cnt[pn][0], n1 = c->cnt[pn][1], n2 = c->cnt[pn][2];
  const unsigned long long live = static_cast<unsigned long long>(n0) + n1 + n2;
  const unsigned rem = S->n_prim - c->prim_next;
  unsigned inj = 0;
  if (c->status == 0 && rem > 0) {
    if (S->mode == GV_ONE_EVENT_PER_LAUNCH) {
      if (live == 0) {
        const unsigned first = S->order ? S->order[c->prim_next] : c->prim_next;
        const unsigned ev = S->prim[first].event;
        while (inj < rem) {
          const unsigned i = c->prim_next + inj;
          const unsigned pi = S->order ? S->order[i] : i;
          if (S->prim[pi].event != ev) break;
          ++inj;
        }
      }
    } else if (live < S->low_water || live == 0) {
      inj = rem < S->batch ? rem : static_cast<unsigned>(S->batch);
      if (c->max_in_flight) {  // events in flight (Sec. 2.1.1): started and not yet finished
        const unsigned fl = c->ev_started - c->ev_done;
        const unsigned room = c->max_in_flight > fl ? c->max_in_flight - fl : 0u;
        inj = inj < room ? inj : room;
      }
      if (S->pcost && inj > 0) {  // automatic cap: the budgets of the events in flight fit the capacity
        if (live == 0) c->cost_done = c->cost_started;  // nothing alive: every event has closed
        const unsigned long long held = c->cost_started > c->cost_done ? c->cost_started - c->cost_done : 0ull;
        const unsigned long long room = S->capacity > held ? S->capacity - held : 0ull;
        const unsigned long long *pc = S->pcost + c->prim_next;
        const unsigned long long base = pc[0];
        if (pc[inj] - base > room) {  // the longest run of the next primaries that fits
          unsigned lo = 0, hi = inj;  // budget(lo) <= room < budget(hi)
          while (hi - lo > 1) {
            const unsigned mid = lo + (hi - lo) / 2;
            if (pc[mid] - base <= room) lo = mid;
            else hi = mid;
          }
          inj = lo;
        }
        if (inj == 0 && live == 0) inj = 1;  // one primary at least when nothing is alive
        c->cost_started += pc[inj] - base;
      }
    }
  }
  c->prim_begin = c->prim_next;
  c->prim_count = inj;
  c->prim_next += inj;
  unsigned B = static_cast<unsigned>(S->chunk);
  // With fewer live tracks than the grid has lanes (the first generations of
  // a shower and its tail), a block claims fewer tracks (a multiple of 32)
  // so that every block gets some: each block's rounds are then short, with
  // fewer warps to wait for at its barriers and its idle lanes left to the
  // secondaries of its block stack.
  if (S->adaptive_chunk) {
    const unsigned long long tot = live + inj;
    const unsigned long long per = (tot + S->grid - 1) / S->grid;
    if (per < B) B = per <= 32 ? 32u : static_cast<unsigned>((per + 31) / 32 * 32);
  }
  c->chunk_B = B;
  c->chunk_end[0] = (n2 + B - 1) / B;  // segments in claim_queue order
  c->chunk_end[1] = c->chunk_end[0] + (n1 + B - 1) / B;
  c->chunk_end[2] = c->chunk_end[1] + (n0 + B - 1) / B;
  c->chunk_end[3] = c->chunk_end[2] + (inj + B - 1) / B;
  // long claims (K_tail rounds) once every primary is injected and few
  // tracks are live: in the tail, and at the start of a batch injected at
  // once, where the block stack keeps a claim's secondaries stepping in the
  // block (one-round claims there measured slower on small batches)
  c->K = (c->prim_next == S->n_prim && live + inj < S->tail_threshold) ? S->K_tail : S->K_bulk;
  c->cnt[pn ^ 1][0] = c->cnt[pn ^ 1][1] = c->cnt[pn ^ 1][2] = 0;
  c->claim = 0;
  for (int r = 0; r < kNClaim; ++r) c->claims[r].n = 0;
  c->blocks_done = 0;
  c->req_n = 0;
  for (int k = 0; k < kNReqKey; ++k) c->key_n[k] = 0;
  c->claim_b = 0;
  c->blocks_done_b = 0;
  if (live + inj > c->live_peak) c->live_peak = live + inj;
  if (live + inj > 0) c->gen += 1;
  if (c->gen > S->max_gen && c->status == 0) c->status = GV_ERR_TIMEOUT;
  c->done = (c->status != 0) || (live == 0 && inj == 0 && c->prim_next == S->n_prim);
  if (c->done) c->chunk_end[0] = c->chunk_end[1] = c->chunk_end[2] = c->chunk_end[3] = 0;
  c->counters[GV_C_GENERATIONS] = c->gen;
}

template <typename R> __global__ void init_kernel(const DevState<R> *S) {
  Ctl *c = S->ctl;
  for (int i = 0; i < 2; ++i)
    for (int q = 0; q < 3; ++q) c->cnt[i][q] = 0;
  c->prim_next = 0;
  c->status = 0;
  c->done = 0;
  c->gen = 0;
  c->loop_iter = 0;
  c->live_peak = 0;
  c->ev_started = 0;
  c->ev_done = 0;
  c->cost_started = 0;
  c->cost_done = 0;
  if (S->max_in_flight >= 0) {
    c->max_in_flight = static_cast<unsigned>(S->max_in_flight);
  } else if (S->pcost) {  // automatic, per event: the budgets of prim_cost (plan_next)
    c->max_in_flight = 0;
  } else {  // automatic, every event budgeted like the most energetic primary:
            // ~0.065 live tracks per MeV at the peak of a shower, x2.3
    const double emax = static_cast<double>(__uint_as_float(c->emax_bits));
    const double cap = static_cast<double>(S->capacity) / (0.15 * emax + 64.0);
    c->max_in_flight = static_cast<unsigned>(cap < 16.0 ? 16.0 : (cap > 1e9 ? 1e9 : cap));
  }
  for (int i = 0; i < 16; ++i) c->counters[i] = 0;
  plan_next(S, 0);
}

// Prefix sums of the primaries' budgets for the automatic events-in-flight
// cap: pcost[i] = sum of prim_cost over primaries 0 .. i-1.  One block; each
// thread sums a contiguous run, the block scans the run totals, each thread
// writes its run's sums.
constexpr int kCostScanThreads = 1024;
template <typename R>
__global__ void __launch_bounds__(kCostScanThreads) prim_cost_kernel(const DevState<R> *S, unsigned long long *pcost) {
  __shared__ unsigned long long s_warp[kCostScanThreads / 32];
  const unsigned n = S->n_prim, tid = threadIdx.x;
  const unsigned per = (n + kCostScanThreads - 1) / kCostScanThreads;
  const unsigned lo = min(n, tid * per), hi = min(n, lo + per);
  unsigned long long sum = 0;
  for (unsigned i = lo; i < hi; ++i) sum += prim_cost(S->prim[i].E_MeV);
  const int lane = tid & 31, warp = tid >> 5;
  unsigned long long incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    unsigned long long w = s_warp[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    s_warp[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  unsigned long long run = incl - sum + (warp ? s_warp[warp - 1] : 0ull);
  if (tid == 0) pcost[0] = 0ull;
  for (unsigned i = lo; i < hi; ++i) {
    run += prim_cost(S->prim[i].E_MeV);
    pcost[i + 1] = run;
  }
}

// largest primary energy, for the automatic events-in-flight cap of the
// allocation-free entry point
template <typename R> __global__ void prim_emax_kernel(const DevState<R> *S) {
  float m = 0.0f;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < S->n_prim; i += gridDim.x * blockDim.x) {
    const float e = static_cast<float>(S->prim[i].E_MeV);
    m = e > m ? e : m;  // NaN and negative energies leave m unchanged
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(&S->ctl->emax_bits, __float_as_uint(m));
}

// ------------------------------------------------------------------ the transport's state
// The step kernels read the transport's state record (queue and tally
// pointers, seeds, switches) from a constant-memory copy, one per precision
// and GPU: its fields are then instruction operands, which costs no load and
// no register on the step path (2.7 % of the benchmark's kernel time against
// the same record read through a global pointer).  The host fills the copy
// on the transport's stream from the record in device memory; transports of
// different contexts on one GPU take turns on it (StateSlot).  The split
// pipeline's kernels read the device-memory record through their pointer:
// with them on the constant copy as well, the fused step kernel measured
// 1.1 % slower.
__constant__ DevState<float> c_state_f;
__constant__ DevState<double> c_state_d;
template <typename R> __device__ __forceinline__ const DevState<R> *tstate();
template <> __device__ __forceinline__ const DevState<float> *tstate<float>() { return &c_state_f; }
template <> __device__ __forceinline__ const DevState<double> *tstate<double>() { return &c_state_d; }

// ------------------------------------------------------------------ the kernel
// Register budget: GV_MIN_BLOCKS resident 256-thread blocks per SM in FP32
// (measured: with the along-step loop 2 blocks at up to 128 registers beat
// 3 blocks at 80 registers, which spill ~700 bytes).  FP64 runs one block
// per SM without a register cap (222 registers, no spills; 4 % faster than
// two blocks at 128 registers, which spilled).
// GV_MAX_BLOCK is the largest block the kernels are compiled for.
#ifndef GV_MIN_BLOCKS
#define GV_MIN_BLOCKS 2
#endif
#ifndef GV_MAX_BLOCK
#define GV_MAX_BLOCK 256
#endif

#ifdef GV_MAXNREG
#define GV_STEP_BOUNDS __maxnreg__(GV_MAXNREG)
#else
#define GV_STEP_BOUNDS __launch_bounds__(GV_MAX_BLOCK, sizeof(R) == 4 ? GV_MIN_BLOCKS : 1)
#endif

template <typename R, bool SORT, bool MERGE, bool FIELD, bool OPTS, bool EXT>
__global__ void GV_STEP_BOUNDS
    step_kernel(int parity) {
  const DevState<R> *__restrict__ S = tstate<R>();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ View<R> sV;
  __shared__ BlockCnt bc;
  __shared__ unsigned s_chunk, s_end[4], s_pb;
  __shared__ unsigned s_slice[kNClaim + 1];
  __shared__ int s_K, s_last;
  __shared__ unsigned s_B;
  __shared__ int s_ltop;  // the block's secondary stack (local_stack)
  __shared__ unsigned s_wcnt[SORT ? kNKey : 1][SORT ? 16 : 1];
  __shared__ unsigned s_walive[SORT ? 16 : 1];
  Ctl *ctl = S->ctl;
  const int tid = threadIdx.x;
  // Programmatic dependent launch (pdl): the next generation's blocks may
  // start as soon as this one's finish, stage their tables, and wait for
  // this grid (and its plan) to complete before reading the plan.
  asm volatile("griddepcontrol.launch_dependents;");
  if (ctl->done) return;  // a done flag seen before the wait is final: nothing planned
  // stage the cross-section tables and the geometry into shared memory
  {
    const uint4 *src = reinterpret_cast<const uint4 *>(S->view.xs);
    uint4 *dst = reinterpret_cast<uint4 *>(smem);
    for (unsigned i = tid; i < S->xs_bytes / 16; i += blockDim.x) dst[i] = src[i];
    const double *zsrc = S->view.zb;
    double *zdst = reinterpret_cast<double *>(smem + S->xs_bytes);
    const int nz = S->view.geo.nsub + 1;
    for (int i = tid; i < nz; i += blockDim.x) zdst[i] = zsrc[i];
    float *idst = reinterpret_cast<float *>(smem + S->xs_bytes + S->zb_bytes);
    for (int i = tid; i < kGridN; i += blockDim.x) idst[i] = S->view.inv_node[i];
    unsigned char *mdst = smem + S->xs_bytes + S->zb_bytes + kInvNodeBytes;
    for (int i = tid; i < S->view.geo.nsub; i += blockDim.x) mdst[i] = S->view.smat[i];
    {
      const uint4 *ssrc = reinterpret_cast<const uint4 *>(S->view.smax);
      uint4 *sdst = reinterpret_cast<uint4 *>(smem + S->smax_off);
      for (unsigned i = tid; i < S->smax_bytes / 16; i += blockDim.x) sdst[i] = ssrc[i];
    }
    if (tid == 0) {
      sV = S->view;
      sV.xs = reinterpret_cast<const V4<R> *>(smem);
      sV.zb = zdst;
      sV.inv_node = idst;
      sV.smat = mdst;
      sV.smax = reinterpret_cast<const R *>(smem + S->smax_off);
    }
    if (tid < 16) bc.c[tid] = 0;
  }
  // the previous generation, and its plan, complete before the plan is read
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (ctl->done) return;  // uniform: nothing planned for this generation
  if (tid == 0) {
    for (int i = 0; i < 4; ++i) s_end[i] = ctl->chunk_end[i];
    for (int r = 0; r <= kNClaim; ++r)
      s_slice[r] = static_cast<unsigned>((static_cast<unsigned long long>(s_end[3]) * r) / kNClaim);
    s_pb = ctl->prim_begin;
    s_K = ctl->K;
    s_B = ctl->chunk_B;
    s_ltop = 0;
  }
  __syncthreads();
  const View<R> &V = sV;
  const int in = parity, out = parity ^ 1;
  const unsigned cap = static_cast<unsigned>(S->capacity);
  const unsigned n_in[3] = {min(ctl->cnt[in][0], cap), min(ctl->cnt[in][1], cap), min(ctl->cnt[in][2], cap)};
  const unsigned n_prim_gen = ctl->prim_count;
  // With several rounds per claim, the secondaries made in a round stay in
  // the block and fill its idle lanes in the next rounds (local_stack).
  const bool use_local = SORT && S->local_stack && s_K > 1;
  LocalStack<R> lstk;
  lstk.e = reinterpret_cast<LKid<R> *>(smem + S->smem_lk_off);
  lstk.top = &s_ltop;
  lstk.cap = static_cast<int>(blockDim.x);
  int w_slice = 0;
  {
    unsigned smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    w_slice = static_cast<int>((smid * 4u + ((tid >> 5) & 3u)) % kNClaim);
  }
  Pending<R> pend;  // this lane's unflushed deposit (merged scoring)
  pend.key = kNoKey;
  pend.sum = R(0);
  pend.comp = R(0);
  Pending<R> *const pd = MERGE ? &pend : nullptr;
  const bool block_claims = SORT || S->claim_chunks == 0;
  if (block_claims) {  // the first claim; each later one is issued before the previous claim's survivors go out
    if (tid == 0) s_chunk = atomicAdd(&ctl->claim, 1u);
    __syncthreads();
  }
  for (;;) {
    // Work claiming: with the basketizer a chunk is one block (its step loop
    // syncs the block); without it every warp claims its own 32-track chunks
    // and never waits for the rest of the block.
    unsigned chunk, idx;
    if (block_claims) {
      chunk = s_chunk;
      __syncthreads();
    } else {
      // The chunk range is split into kNClaim slices, each with its own
      // counter in its own cache line: a warp draws from its SM's slice and
      // moves on when that slice is spent, so no single address takes every
      // claim of the generation.
      unsigned c0 = 0;
      if ((tid & 31) == 0) {
        c0 = 0xffffffffu;
        for (int k = 0; k < kNClaim; ++k) {
          const int r = (w_slice + k) % kNClaim;
          const unsigned lo = s_slice[r], hi = s_slice[r + 1];
          if (lo >= hi) continue;
          const unsigned c = lo + atomicAdd(&ctl->claims[r].n, 1u);
          if (c < hi) {
            c0 = c;
            w_slice = r;
            break;
          }
        }
      }
      chunk = __shfl_sync(0xffffffffu, c0, 0);
      if (chunk == 0xffffffffu) break;
    }
    if (chunk >= s_end[3]) break;
    int qsel = 0;
    while (chunk >= s_end[qsel]) ++qsel;
    {
      const bool per_block = SORT || S->claim_chunks == 0;
      const unsigned csize = per_block ? s_B : 32u;
      idx = (chunk - (qsel ? s_end[qsel - 1] : 0u)) * csize + (per_block ? tid : (tid & 31));
      if (per_block && static_cast<unsigned>(tid) >= csize) idx = 0xffffffffu;
    }
    qsel = claim_queue(qsel);
    Trk<R> t;
    bool alive = false;
    if (qsel < 3) {
      if (idx < n_in[qsel]) {
        const Queue<R> &q = S->q[in][qsel];
        t.x = q.x[idx]; t.y = q.y[idx]; t.z = q.z[idx];
        t.u = q.u[idx]; t.v = q.v[idx]; t.w = q.w[idx];
        t.E = q.E[idx]; t.nlam = q.nlam[idx];
        t.id = q.id[idx]; t.ev = q.ev[idx]; t.step = q.step[idx];
        const int sf = q.sf[idx];
        t.sub = sf & 0xffff;
        t.flags = sf >> 16;
        t.type = qsel;
        alive = true;
        GV_CHECK(&ctl->status, t.sub >= 0 && t.sub < V.geo.nsub && t.ev < S->n_events && t.E >= R(0));
      }
    } else if (idx < n_prim_gen) {
      const unsigned i = s_pb + idx;
      const unsigned pi = S->order ? S->order[i] : i;
      gv_primary p = S->prim[pi];
      const double e_in = p.E_MeV;  // the budget of the automatic cap is the caller's energy
      p.event -= S->ev_base;  // the tallies' row (events below the range wrap to a large value)
      if (p.type < 0 || p.type > 2 || p.event >= S->n_events) {  // caller's device array: check here
        set_status(ctl, GV_ERR_BAD_ARG);
        p.type = 0;
        p.event = 0;
        p.z = -1.0;
        p.E_MeV = 0.0;
      }
      t.type = p.type;
      t.E = static_cast<R>(p.E_MeV);
      t.x = p.x; t.y = p.y; t.z = p.z;
      t.u = static_cast<R>(p.u); t.v = static_cast<R>(p.v); t.w = static_cast<R>(p.w);
      t.nlam = R(-1);
      t.id = p.id;
      t.ev = p.event;
      t.step = 0;
      t.flags = kFlagPrimary;
      t.sub = locate(V.zb, V.geo.nsub, p.z, p.w);
      count<R, EXT>(S, &bc, t.ev, GV_C_TRK_G + t.type);
      if (t.sub < 0) {
        atomicAdd(&S->escape[t.ev], p.E_MeV);
        if (t.type == 2) count<R, EXT>(S, &bc, t.ev, GV_C_EP_ESC);
        primary_cost(S, t.ev, e_in, false);
      } else {
        alive = true;
        primary_cost(S, t.ev, e_in, true);
        if (atomicAdd(&S->evlive[t.ev], 1u) == 0u) atomicAdd(&ctl->ev_started, 1u);
      }
    }
    const int K = s_K;
    unsigned ended_prev = 0u;  // evlive before this lane's last track ended (1: it closed its event)
    for (int kk = 0; kk < K; ++kk) {
      // (with the basketizer the block leaves the loop together, after the
      // count barrier below shows that no lane was alive)
      if (!SORT && !__any_sync(0xffffffffu, alive)) break;
      if (use_local && kk > 0 && !alive) {  // take up a secondary of an earlier round
        const int i = atomicSub(&s_ltop, 1) - 1;
        if (i >= 0 && i < lstk.cap) {
          const LKid<R> &e = lstk.e[i];
          t.x = e.x; t.y = e.y; t.z = e.z;
          t.u = e.u; t.v = e.v; t.w = e.w;
          t.E = e.E;
          t.nlam = R(-1);
          t.id = e.id;
          t.ev = e.ev;
          t.step = 0;
          t.sub = e.sub;
          t.flags = 0;
          t.type = e.type;
          alive = true;
        }
      }
      const bool was_alive = alive;
      Kids<R> kids;
      kids.n = 0;
      uint32_t kstep = 0;
      int proc = -1, lim = -1;
      R u[8];
      // Along-step part.  With the basketizer a lane keeps stepping (boundary-
      // and continuous-limited steps need no final state) until its track is
      // due a discrete interaction, ends, or has taken along_steps steps; the
      // block then baskets the interactions.  Step tallies stay per lane and
      // are summed per warp afterwards.
      unsigned n_st = 0, n_geom = 0, n_iter = 0;
      // photons cross layers in runs of boundary-limited steps; charged tracks
      // are stopped more often by their continuous-loss limit: each type has
      // its own budget (measured best at 5 and 3 on the benchmark)
      const int inner = SORT ? (t.type == 0 ? S->along_steps_g : S->along_steps) : 1;
      for (int m = 0; m < inner && alive && proc < 0; ++m) {
        ++n_iter;
        const uint32_t before = t.step;
        alive = step_track<R, FIELD, OPTS, EXT>(V, S, t, kids, kstep, &bc, proc, u, lim, pd) != 0;
        // NaN energy, or a non-finite z (tested on its exponent bits: an FP64
        // comparison would take the FP64 pipe)
        if (!(t.E == t.E) || (__double2hiint(t.z) & 0x7ff00000) == 0x7ff00000) {
          set_status(ctl, GV_ERR_NUMERIC);
          alive = false;
          proc = -1;
        }
        if (t.step != before) {
          ++n_st;
          n_geom += lim == 0 ? 1u : 0u;
        }
      }
      if (!SORT && alive && proc >= 0) {  // final state in place (warp-divergent across processes)
        R d[3] = {t.u, t.v, t.w};
        const int r = final_state<R, OPTS, EXT>(V, S, &bc, t.type, proc, t.E, d, u, kids, t.ev, t.sub, t.x, t.y, t.id, kstep, pd);
        if (r >= 0) {
          t.u = d[0]; t.v = d[1]; t.w = d[2];
          t.flags |= kFlagInteracted;
          alive = r != 0;
        }
      }
      push_kids<R, EXT>(S, out, parent_of(t), kids, kstep, &bc);
      if (MERGE) warp_flush(S, pend);
      {  // step counters, one shared-memory atomic per warp and kind
        const unsigned wst = __reduce_add_sync(0xffffffffu, n_st);
        const unsigned wiq = __reduce_max_sync(0xffffffffu, n_iter);
        if (wst) {
          const unsigned wg = __reduce_add_sync(0xffffffffu, t.type == 0 ? n_st : 0u);
          const unsigned we = __reduce_add_sync(0xffffffffu, t.type == 1 ? n_st : 0u);
          const unsigned wx = __reduce_add_sync(0xffffffffu, (n_st && proc >= 0) ? 1u : 0u);
          const unsigned wb = __reduce_add_sync(0xffffffffu, n_geom);
          if ((tid & 31) == 0) {
            atomicAdd(&bc.c[GV_C_STEPS], static_cast<unsigned long long>(wst));
            if (wg) atomicAdd(&bc.c[GV_C_STEPS_G], static_cast<unsigned long long>(wg));
            if (we) atomicAdd(&bc.c[GV_C_STEPS_EM], static_cast<unsigned long long>(we));
            if (wst - wg - we) atomicAdd(&bc.c[GV_C_STEPS_EP], static_cast<unsigned long long>(wst - wg - we));
            if (wx) atomicAdd(&bc.c[GV_C_DISCRETE], static_cast<unsigned long long>(wx));
            if (wb) atomicAdd(&bc.c[GV_C_GEOM], static_cast<unsigned long long>(wb));
          }
        }
        if ((tid & 31) == 0 && wiq) atomicAdd(&bc.c[GV_C_LANE_SLOTS], 32ull * wiq);  // idle-lane fraction
      }
      if (SORT) {
        // Basketizer: counting sort of this step's interaction requests by
        // (type, process) -- warp ballots, a prefix sum over keys and warps,
        // one slot each -- so every warp runs a single final-state model.
        // Three block barriers per step: counts, requests, results.
        IReq<R> *req = reinterpret_cast<IReq<R> *>(smem + S->smem_req_off);
        const int key = (alive && proc >= 0) ? t.type * 3 + proc : -1;
        const int lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
        unsigned rank = 0;
#pragma unroll
        for (int k = 0; k < kNKey; ++k) {
          const unsigned m = __ballot_sync(0xffffffffu, key == k);
          if (lane == 0) s_wcnt[k][warp] = __popc(m);
          if (key == k) rank = __popc(m & ((1u << lane) - 1u));
        }
        const unsigned ma = __ballot_sync(0xffffffffu, was_alive);
        if (lane == 0) s_walive[warp] = ma;
        __syncthreads();
        if (use_local && tid == 0 && s_ltop < 0) s_ltop = 0;  // pops of an empty stack
        unsigned any = 0;
        for (int w = 0; w < nw; ++w) any |= s_walive[w];
        if (!any) break;  // uniform: no lane of the block was alive this step
        // lane k < kNKey: requests of key k in the block and in warps before this one
        unsigned ck = 0, part = 0;
        if (lane < kNKey) {
          for (int w = 0; w < nw; ++w) {
            const unsigned c = s_wcnt[lane][w];
            ck += c;
            part += (w < warp) ? c : 0u;
          }
        }
        unsigned incl = ck;
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) {
          const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        const unsigned start = incl - ck + part;  // first slot of key `lane` for this warp
        const unsigned nreq = __shfl_sync(0xffffffffu, incl, kNKey - 1);
        const unsigned mine = __shfl_sync(0xffffffffu, start, key >= 0 ? key : 0);
        const unsigned slot = key >= 0 ? mine + rank : 0u;
        if (key >= 0) {
          IReq<R> &q = req[slot];
          q.x = t.x; q.y = t.y; q.z = t.z;
          q.id = t.id;
          q.E = t.E; q.d0 = t.u; q.d1 = t.v; q.d2 = t.w;
#pragma unroll
          for (int j = 0; j < 6; ++j) q.u[j] = u[2 + j];
          q.ev = t.ev;
          q.kk = kstep;
          q.sub = t.sub;
          q.tp = key;
        }
        __syncthreads();
        Kids<R> kb;
        kb.n = 0;
        Parent par;
        uint32_t pk = 0;
        if (static_cast<unsigned>(tid) < nreq) {
          IReq<R> &q = req[tid];
          R uu[8] = {R(0), R(0), q.u[0], q.u[1], q.u[2], q.u[3], q.u[4], q.u[5]};
          R d[3] = {q.d0, q.d1, q.d2};
          R e = q.E;
          const int ty = q.tp / 3;
          const int r = final_state<R, OPTS, EXT>(V, S, &bc, ty, q.tp - 3 * ty, e, d, uu, kb, q.ev, q.sub, q.x, q.y, q.id, q.kk);
          par.x = q.x; par.y = q.y; par.z = q.z;
          par.id = q.id;
          par.ev = q.ev;
          par.sub = q.sub;
          pk = q.kk;
          q.E = e; q.d0 = d[0]; q.d1 = d[1]; q.d2 = d[2];
          q.tp = r;
        }
        push_kids<R, EXT>(S, out, par, kb, pk, &bc, use_local ? &lstk : nullptr);
        __syncthreads();
        if (key >= 0) {
          const IReq<R> &q = req[slot];
          if (q.tp >= 0) {
            t.E = q.E; t.u = q.d0; t.v = q.d1; t.w = q.d2;
            t.flags |= kFlagInteracted;
            alive = q.tp != 0;
          }
        }
      }
      if (was_alive && !alive) {
        if (kk + 1 < K) track_ended(S, t.ev);
        else ended_prev = atomicSub(&S->evlive[t.ev], 1u);  // read after the survivors are out
      }
    }
    // the next claim's atomic and the event count's are in flight while the
    // survivors are written
    unsigned next_chunk = 0u;
    if (block_claims && tid == 0) next_chunk = atomicAdd(&ctl->claim, 1u);
    if (MERGE) warp_flush(S, pend);  // nothing stays pending past a claim
    push_survivor(S, out, t, alive);
    if (ended_prev == 1u) event_closed(S, t.ev);
    if (use_local) {  // what is left on the block's stack goes to the next generation
      __syncthreads();
      const int n = max(0, min(s_ltop, lstk.cap));
      for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + tid;
        push_lkid(S, out, i < n ? &lstk.e[i] : static_cast<const LKid<R> *>(nullptr));
      }
      __syncthreads();
      if (tid == 0) s_ltop = 0;
    }
    if (block_claims) {
      if (tid == 0) s_chunk = next_chunk;
      __syncthreads();
    }
  }
  // flush block counters; the last block plans the next generation
  __syncthreads();
  if (tid < 16 && bc.c[tid]) atomicAdd(&ctl->counters[tid], bc.c[tid]);
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const unsigned t = atomicAdd(&ctl->blocks_done, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (s_last && tid == 0) {
    __threadfence();
    plan_next(S, out);
  }
}

// ------------------------------------------------------------------ split pipeline
// The same generation in two kernels.  The along-step kernel runs the lanes'
// steps until a track is due a discrete interaction, ends, or has taken its
// along-step budget, without any block barrier after the claim; a track due
// an interaction becomes a request record and its index goes to the list of
// its (type, process) key.  The interaction kernel then gives every warp 32
// requests of one key, so each warp runs one final-state model, and writes
// survivors and secondaries to the output queues; its last block plans the
// next generation.  The price is one request record written and read per
// interaction.

// Hand the tracks due an interaction to the interaction kernel.  All 32
// lanes of a converged warp.
template <typename R>
__device__ void emit_requests(const DevState<R> *S, const Trk<R> &t, bool hand, int proc, uint32_t kstep,
                              const R *u) {
  if (!__ballot_sync(0xffffffffu, hand)) return;
  Ctl *ctl = S->ctl;
  unsigned total;
  const unsigned slot = warp_reserve(&ctl->req_n, hand ? 1u : 0u, total);
  const bool ok = hand && slot < S->req_cap;
  if (hand && !ok) set_status(ctl, GV_ERR_STACK_FULL);
  const int key = t.type * 3 + proc;
  if (ok) {
    GReq<R> &q = S->req[slot];
    q.x = t.x; q.y = t.y; q.z = t.z;
    q.id = t.id;
    q.E = t.E; q.d0 = t.u; q.d1 = t.v; q.d2 = t.w;
#pragma unroll
    for (int j = 0; j < 6; ++j) q.u[j] = u[2 + j];
    q.ev = t.ev;
    q.kk = kstep;
    q.sf = t.sub | (t.flags << 16);
    q.key = key;
  }
#pragma unroll
  for (int k = 0; k < kNReqKey; ++k) {
    const bool mine = ok && key == k;
    if (!__ballot_sync(0xffffffffu, mine)) continue;
    unsigned tk;
    const unsigned pos = warp_reserve(&ctl->key_n[k], mine ? 1u : 0u, tk);
    if (mine) S->keyidx[static_cast<size_t>(k) * S->req_cap + pos] = slot;
  }
}

template <typename R>
#ifndef GV_ALONG_MIN_BLOCKS
#define GV_ALONG_MIN_BLOCKS 2
#endif
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? GV_ALONG_MIN_BLOCKS : 2) along_kernel(const DevState<R> *__restrict__ S, int parity) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ View<R> sV;
  __shared__ BlockCnt bc;
  __shared__ unsigned s_chunk, s_end[4], s_pb;
  __shared__ int s_K;
  Ctl *ctl = S->ctl;
  const int tid = threadIdx.x;
  if (ctl->done) return;
  {  // tables, planes, 1/E_i and sub-slab materials into shared memory
    const uint4 *src = reinterpret_cast<const uint4 *>(S->view.xs);
    uint4 *dst = reinterpret_cast<uint4 *>(smem);
    for (unsigned i = tid; i < S->xs_bytes / 16; i += blockDim.x) dst[i] = src[i];
    const double *zsrc = S->view.zb;
    double *zdst = reinterpret_cast<double *>(smem + S->xs_bytes);
    const int nz = S->view.geo.nsub + 1;
    for (int i = tid; i < nz; i += blockDim.x) zdst[i] = zsrc[i];
    float *idst = reinterpret_cast<float *>(smem + S->xs_bytes + S->zb_bytes);
    for (int i = tid; i < kGridN; i += blockDim.x) idst[i] = S->view.inv_node[i];
    unsigned char *mdst = smem + S->xs_bytes + S->zb_bytes + kInvNodeBytes;
    for (int i = tid; i < S->view.geo.nsub; i += blockDim.x) mdst[i] = S->view.smat[i];
    {
      const uint4 *ssrc = reinterpret_cast<const uint4 *>(S->view.smax);
      uint4 *sdst = reinterpret_cast<uint4 *>(smem + S->smax_off);
      for (unsigned i = tid; i < S->smax_bytes / 16; i += blockDim.x) sdst[i] = ssrc[i];
    }
    if (tid == 0) {
      sV = S->view;
      sV.xs = reinterpret_cast<const V4<R> *>(smem);
      sV.zb = zdst;
      sV.inv_node = idst;
      sV.smat = mdst;
      sV.smax = reinterpret_cast<const R *>(smem + S->smax_off);
      for (int i = 0; i < 4; ++i) s_end[i] = ctl->chunk_end[i];
      s_pb = ctl->prim_begin;
      s_K = ctl->K;
    }
    if (tid < 16) bc.c[tid] = 0;
  }
  __syncthreads();
  const View<R> &V = sV;
  const int in = parity, out = parity ^ 1;
  const unsigned cap = static_cast<unsigned>(S->capacity);
  const unsigned n_in[3] = {min(ctl->cnt[in][0], cap), min(ctl->cnt[in][1], cap), min(ctl->cnt[in][2], cap)};
  const unsigned n_prim_gen = ctl->prim_count;
  for (;;) {
    if (tid == 0) s_chunk = atomicAdd(&ctl->claim, 1u);
    __syncthreads();
    const unsigned chunk = s_chunk;
    __syncthreads();
    if (chunk >= s_end[3]) break;
    int qsel = 0;
    while (chunk >= s_end[qsel]) ++qsel;
    const unsigned idx = (chunk - (qsel ? s_end[qsel - 1] : 0u)) * blockDim.x + tid;
    qsel = claim_queue(qsel);
    Trk<R> t;
    bool alive = false;
    if (qsel < 3) {
      if (idx < n_in[qsel]) {
        const Queue<R> &q = S->q[in][qsel];
        t.x = q.x[idx]; t.y = q.y[idx]; t.z = q.z[idx];
        t.u = q.u[idx]; t.v = q.v[idx]; t.w = q.w[idx];
        t.E = q.E[idx]; t.nlam = q.nlam[idx];
        t.id = q.id[idx]; t.ev = q.ev[idx]; t.step = q.step[idx];
        const int sf = q.sf[idx];
        t.sub = sf & 0xffff;
        t.flags = sf >> 16;
        t.type = qsel;
        alive = true;
        GV_CHECK(&ctl->status, t.sub >= 0 && t.sub < V.geo.nsub && t.ev < S->n_events && t.E >= R(0));
      }
    } else if (idx < n_prim_gen) {
      const unsigned i = s_pb + idx;
      const unsigned pi = S->order ? S->order[i] : i;
      gv_primary p = S->prim[pi];
      const double e_in = p.E_MeV;  // the budget of the automatic cap is the caller's energy
      p.event -= S->ev_base;  // the tallies' row (events below the range wrap to a large value)
      if (p.type < 0 || p.type > 2 || p.event >= S->n_events) {  // caller's device array: check here
        set_status(ctl, GV_ERR_BAD_ARG);
        p.type = 0;
        p.event = 0;
        p.z = -1.0;
        p.E_MeV = 0.0;
      }
      t.type = p.type;
      t.E = static_cast<R>(p.E_MeV);
      t.x = p.x; t.y = p.y; t.z = p.z;
      t.u = static_cast<R>(p.u); t.v = static_cast<R>(p.v); t.w = static_cast<R>(p.w);
      t.nlam = R(-1);
      t.id = p.id;
      t.ev = p.event;
      t.step = 0;
      t.flags = kFlagPrimary;
      t.sub = locate(V.zb, V.geo.nsub, p.z, p.w);
      count(S, &bc, t.ev, GV_C_TRK_G + t.type);
      if (t.sub < 0) {
        atomicAdd(&S->escape[t.ev], p.E_MeV);
        if (t.type == 2) count(S, &bc, t.ev, GV_C_EP_ESC);
        primary_cost(S, t.ev, e_in, false);
      } else {
        alive = true;
        primary_cost(S, t.ev, e_in, true);
        if (atomicAdd(&S->evlive[t.ev], 1u) == 0u) atomicAdd(&ctl->ev_started, 1u);
      }
    }
    const int K = s_K;
    for (int kk = 0; kk < K; ++kk) {
      if (!__any_sync(0xffffffffu, alive)) break;
      const bool was_alive = alive;
      Kids<R> kids;
      kids.n = 0;
      uint32_t kstep = 0;
      int proc = -1, lim = -1;
      R u[8];
      unsigned n_st = 0, n_geom = 0, n_iter = 0;
      const int inner = t.type == 0 ? S->along_steps_g : S->along_steps;
      for (int m = 0; m < inner && alive && proc < 0; ++m) {
        ++n_iter;
        const uint32_t before = t.step;
        alive = step_track<R, true, true, true>(V, S, t, kids, kstep, &bc, proc, u, lim, static_cast<Pending<R> *>(nullptr)) != 0;
        if (!(t.E == t.E) || (__double2hiint(t.z) & 0x7ff00000) == 0x7ff00000) {
          set_status(ctl, GV_ERR_NUMERIC);
          alive = false;
          proc = -1;
        }
        if (t.step != before) {
          ++n_st;
          n_geom += lim == 0 ? 1u : 0u;
        }
      }
      push_kids(S, out, parent_of(t), kids, kstep, &bc);
      {  // step counters, one shared-memory atomic per warp and kind
        const unsigned wst = __reduce_add_sync(0xffffffffu, n_st);
        const unsigned wiq = __reduce_max_sync(0xffffffffu, n_iter);
        if (wst) {
          const unsigned wg = __reduce_add_sync(0xffffffffu, t.type == 0 ? n_st : 0u);
          const unsigned we = __reduce_add_sync(0xffffffffu, t.type == 1 ? n_st : 0u);
          const unsigned wx = __reduce_add_sync(0xffffffffu, (n_st && alive && proc >= 0) ? 1u : 0u);
          const unsigned wb = __reduce_add_sync(0xffffffffu, n_geom);
          if ((tid & 31) == 0) {
            atomicAdd(&bc.c[GV_C_STEPS], static_cast<unsigned long long>(wst));
            if (wg) atomicAdd(&bc.c[GV_C_STEPS_G], static_cast<unsigned long long>(wg));
            if (we) atomicAdd(&bc.c[GV_C_STEPS_EM], static_cast<unsigned long long>(we));
            if (wst - wg - we) atomicAdd(&bc.c[GV_C_STEPS_EP], static_cast<unsigned long long>(wst - wg - we));
            if (wx) atomicAdd(&bc.c[GV_C_DISCRETE], static_cast<unsigned long long>(wx));
            if (wb) atomicAdd(&bc.c[GV_C_GEOM], static_cast<unsigned long long>(wb));
          }
        }
        if ((tid & 31) == 0 && wiq) atomicAdd(&bc.c[GV_C_LANE_SLOTS], 32ull * wiq);
      }
      if (was_alive && !alive) track_ended(S, t.ev);
      const bool hand = alive && proc >= 0;
      emit_requests(S, t, hand, proc, kstep, u);
      alive = alive && !hand;  // the interaction kernel owns it now
    }
    push_survivor(S, out, t, alive);
  }
  __syncthreads();
  if (tid < 16 && bc.c[tid]) atomicAdd(&ctl->counters[tid], bc.c[tid]);
}

template <typename R>
__global__ void __launch_bounds__(256) interact_kernel(const DevState<R> *__restrict__ S, int parity) {
  __shared__ View<R> sV;
  __shared__ BlockCnt bc;
  __shared__ unsigned s_kend[kNReqKey], s_kn[kNReqKey];
  __shared__ int s_last;
  Ctl *ctl = S->ctl;
  const int tid = threadIdx.x, lane = tid & 31;
  if (ctl->done) return;
  if (tid == 0) {
    sV = S->view;  // tables stay in global memory: the final states read the alias bins only
    unsigned acc = 0;
    for (int k = 0; k < kNReqKey; ++k) {
      const unsigned n = min(ctl->key_n[k], static_cast<unsigned>(S->req_cap));
      s_kn[k] = n;
      acc += (n + 31u) / 32u;
      s_kend[k] = acc;
    }
  }
  if (tid < 16) bc.c[tid] = 0;
  __syncthreads();
  const View<R> &V = sV;
  const int out = parity ^ 1;
  for (;;) {
    unsigned chunk = 0;
    if (lane == 0) chunk = atomicAdd(&ctl->claim_b, 1u);
    chunk = __shfl_sync(0xffffffffu, chunk, 0);
    if (chunk >= s_kend[kNReqKey - 1]) break;
    int k = 0;
    while (chunk >= s_kend[k]) ++k;
    const unsigned pos = (chunk - (k ? s_kend[k - 1] : 0u)) * 32u + lane;
    const bool has = pos < s_kn[k];
    const int ty = k / 3, proc = k - 3 * ty;
    Trk<R> t;
    Kids<R> kids;
    kids.n = 0;
    Parent par;
    uint32_t kk = 0;
    bool alive = false;
    if (has) {
      const GReq<R> q = S->req[S->keyidx[static_cast<size_t>(k) * S->req_cap + pos]];
      R uu[8] = {R(0), R(0), q.u[0], q.u[1], q.u[2], q.u[3], q.u[4], q.u[5]};
      R d[3] = {q.d0, q.d1, q.d2};
      R e = q.E;
      t.x = q.x; t.y = q.y; t.z = q.z;
      t.id = q.id;
      t.ev = q.ev;
      t.sub = q.sf & 0xffff;
      t.flags = q.sf >> 16;
      t.type = ty;
      kk = q.kk;
      t.step = kk + 1;
      t.nlam = R(-1);
      const int r = final_state(V, S, &bc, ty, proc, e, d, uu, kids, t.ev, t.sub, t.x, t.y, q.id, q.kk);
      t.E = e;
      t.u = d[0]; t.v = d[1]; t.w = d[2];
      if (r >= 0) t.flags |= kFlagInteracted;
      alive = r != 0;
      par = parent_of(t);
    } else {
      par.x = par.y = par.z = 0.0;
      par.id = 0;
      par.ev = 0;
      par.sub = 0;
    }
    push_kids(S, out, par, kids, kk, &bc);
    if (has && !alive) track_ended(S, t.ev);
    push_survivor(S, out, t, alive);
  }
  __syncthreads();
  if (tid < 16 && bc.c[tid]) atomicAdd(&ctl->counters[tid], bc.c[tid]);
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const unsigned d = atomicAdd(&ctl->blocks_done_b, 1u);
    s_last = (d == gridDim.x - 1);
  }
  __syncthreads();
  if (s_last && tid == 0) {
    __threadfence();
    plan_next(S, out);
  }
}

}  // namespace gv

// ====================================================================== host
using namespace gv;

namespace {

struct Ctx {
  int device = 0, sm_count = 0;
  gv_config cfg;
  std::vector<gv_material> mats;
  gv_layers geo;
  gv_cuts cuts;
  int nsub = 0;
  std::vector<double> zb;
  std::vector<unsigned char> smat;
  bool tables = false;
  HostTables ht;
  // device allocations
  void *d_xs = nullptr, *d_bins = nullptr, *d_smax = nullptr;
  float *d_inv_node = nullptr;
  double *d_zb = nullptr;
  unsigned char *d_smat = nullptr;
  void *d_queues = nullptr;
  Ctl *d_ctl = nullptr;
  void *d_state = nullptr;
  double *d_edep = nullptr, *d_cell = nullptr, *d_escape = nullptr;
  unsigned long long *d_evcnt = nullptr;
  unsigned *d_evlive = nullptr;
  unsigned long long *d_evcost = nullptr;  // budget held per event (automatic in-flight cap)
  size_t ev_cap = 0;
  unsigned long long *d_pcost = nullptr;   // prefix sums of the primaries' budgets
  size_t pcost_cap = 0;
  gv_primary *d_prim = nullptr;
  unsigned *d_order = nullptr;
  size_t prim_cap = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, t0 = nullptr, t1 = nullptr;
  cudaGraphExec_t graph = nullptr;
  int loop_graph = 0;  // graph holds the device-side generation loop
  Ctl *h_ctl = nullptr;  // pinned
  long long launches = 0;
  int last_status = 0;
  // a transport whose completion gv_sync (or the next call) collects
  struct {
    bool active = false;
    gv_result *res = nullptr;
    long long launches = 0;  // launches known before the device-side loop ran
    double kernel_ms = 0.0;  // host-looped transports: measured already
    bool timed_loop = false; // kernel time = t0 .. t1 of the one graph launch
  } pend;
  ModelMeta meta[kNModel];
  size_t xs_bytes = 0, zb_bytes = 0, smem_bytes = 0, req_off = 0, bins_bytes = 0, smax_bytes = 0, smax_off = 0;
  size_t lk_off = 0;
  int grid = 0, grid_b = 0;
  // split pipeline: interaction requests and their per-key index lists
  void *d_req = nullptr;
  unsigned *d_keyidx = nullptr;
  // L2 persisting window over the alias bins (config l2_persist)
  size_t l2_window = 0, l2_old_limit = 0;
};

#define CK(x)                                  \
  do {                                         \
    cudaError_t e_ = (x);                      \
    if (e_ != cudaSuccess) return GV_ERR_CUDA; \
  } while (0)

int validate(const gv_material *mats, int n_mats, const gv_layers *geo, const gv_cuts *cuts) {
  if (!mats || !geo || !cuts || n_mats < 1 || n_mats > GV_MAX_MAT) return GV_ERR_BAD_ARG;
  for (int m = 0; m < n_mats; ++m) {
    const gv_material &x = mats[m];
    if (x.n_elem < 1 || x.n_elem > GV_MAX_ELEM || !(x.rho > 0) || !(x.I_eV > 0)) return GV_ERR_BAD_ARG;
    for (int e = 0; e < x.n_elem; ++e)
      if (!(x.Z[e] >= 1) || !(x.A[e] > 0) || !(x.w[e] > 0)) return GV_ERR_BAD_ARG;
  }
  if (geo->n_layers < 1 || geo->n_sub < 1 || geo->n_sub > GV_MAX_SUB ||
      static_cast<long long>(geo->n_layers) * geo->n_sub > GV_MAX_SUBTOTAL)
    return GV_ERR_BAD_ARG;
  for (int j = 0; j < geo->n_sub; ++j)
    if (!(geo->sub_thick_cm[j] > 0) || geo->sub_mat[j] < 0 || geo->sub_mat[j] >= n_mats) return GV_ERR_BAD_ARG;
  if (geo->nx_cells < 0 || geo->ny_cells < 0) return GV_ERR_BAD_ARG;
  if (!(std::fabs(geo->field_T) < 1e4) || geo->field_axis < 0 || geo->field_axis > 2) return GV_ERR_BAD_ARG;
  if ((geo->nx_cells > 0 || geo->ny_cells > 0) &&
      !(geo->nx_cells > 0 && geo->ny_cells > 0 && geo->half_x_cm > 0 && geo->half_y_cm > 0))
    return GV_ERR_BAD_ARG;
  if (!(cuts->track_cut_MeV >= kGridEmin) || !(cuts->gamma_cut_MeV >= cuts->track_cut_MeV) ||
      !(cuts->e_cut_MeV >= cuts->track_cut_MeV))
    return GV_ERR_BAD_ARG;
  return GV_OK;
}

int validate_cfg(const gv_config &c) {
  if (c.precision != GV_MIXED && c.precision != GV_FP64) return GV_ERR_BAD_ARG;
  if (c.mode != GV_BATCHED && c.mode != GV_ONE_EVENT_PER_LAUNCH) return GV_ERR_BAD_ARG;
  if (c.block_size < 64 || c.block_size > GV_MAX_BLOCK || c.block_size % 32) return GV_ERR_BAD_ARG;
  if (c.blocks_per_sm < 1 || c.blocks_per_sm > 32) return GV_ERR_BAD_ARG;
  if (c.steps_per_claim < 1 || c.tail_steps_per_claim < 1 || c.steps_per_claim > 4096 ||
      c.tail_steps_per_claim > 4096)
    return GV_ERR_BAD_ARG;
  if (c.stack_capacity < 1024 || c.stack_capacity > (1ll << 31)) return GV_ERR_BAD_ARG;
  if (c.refill_batch < 1 || c.refill_low_water < 0) return GV_ERR_BAD_ARG;
  if (c.generations_per_graph < 2 || c.generations_per_graph % 2 || c.generations_per_graph > 1024)
    return GV_ERR_BAD_ARG;
  if (c.max_generations < 1 || c.max_events_in_flight < -1) return GV_ERR_BAD_ARG;
  if (c.claim_chunks < 0 || c.claim_chunks > 1) return GV_ERR_BAD_ARG;
  if (c.along_steps < 1 || c.along_steps > 64) return GV_ERR_BAD_ARG;
  if (c.along_steps_photon < 0 || c.along_steps_photon > 64) return GV_ERR_BAD_ARG;
  if (c.scoring < 0 || c.scoring > 1) return GV_ERR_BAD_ARG;
  if (c.l2_persist < 0 || c.l2_persist > 1) return GV_ERR_BAD_ARG;
  if (c.local_stack < 0 || c.local_stack > 1) return GV_ERR_BAD_ARG;
  if (c.pdl < 0 || c.pdl > 1) return GV_ERR_BAD_ARG;
  if (c.device_loop < 0 || c.device_loop > 1) return GV_ERR_BAD_ARG;
  if (c.blocking < 0 || c.blocking > 1) return GV_ERR_BAD_ARG;
  if (c.pipeline < 0 || c.pipeline > 1 || (c.pipeline == 1 && c.scoring != 0)) return GV_ERR_BAD_ARG;
  return GV_OK;
}

template <typename R> size_t queue_bytes(long long cap) { return static_cast<size_t>(cap) * track_bytes<R>(); }

template <typename R> Queue<R> carve(unsigned char *&p, long long cap) {
  Queue<R> q;
  auto take = [&](size_t n) {
    unsigned char *r = p;
    p += (n + 255) / 256 * 256;
    return r;
  };
  q.x = reinterpret_cast<double *>(take(cap * sizeof(double)));
  q.y = reinterpret_cast<double *>(take(cap * sizeof(double)));
  q.z = reinterpret_cast<double *>(take(cap * sizeof(double)));
  q.u = reinterpret_cast<R *>(take(cap * sizeof(R)));
  q.v = reinterpret_cast<R *>(take(cap * sizeof(R)));
  q.w = reinterpret_cast<R *>(take(cap * sizeof(R)));
  q.E = reinterpret_cast<R *>(take(cap * sizeof(R)));
  q.nlam = reinterpret_cast<R *>(take(cap * sizeof(R)));
  q.id = reinterpret_cast<unsigned long long *>(take(cap * sizeof(unsigned long long)));
  q.ev = reinterpret_cast<unsigned *>(take(cap * sizeof(unsigned)));
  q.step = reinterpret_cast<unsigned *>(take(cap * sizeof(unsigned)));
  q.sf = reinterpret_cast<int *>(take(cap * sizeof(int)));
  return q;
}

template <typename R> size_t carve_bytes(long long cap) {
  size_t s = 0;
  const size_t sizes[12] = {8, 8, 8, sizeof(R), sizeof(R), sizeof(R), sizeof(R), sizeof(R), 8, 4, 4, 4};
  for (size_t z : sizes) s += (cap * z + 255) / 256 * 256;
  return s;
}

template <typename R> int upload_tables(Ctx *c) {
  const HostTables &h = c->ht;
  // cross sections as V4<R>
  const size_t nv = static_cast<size_t>(h.n_mat) * 3 * kGridN;
  std::vector<V4<R>> xs(nv);
  for (size_t i = 0; i < nv; ++i) {
    // the range (e- component z, e+ component w) is stored as ln R
    const int type = static_cast<int>((i / kGridN) % 3);
    xs[i].x = static_cast<R>(h.xs[4 * i + 0]);
    xs[i].y = static_cast<R>(h.xs[4 * i + 1]);
    xs[i].z = static_cast<R>(type == 1 ? std::log(h.xs[4 * i + 2]) : h.xs[4 * i + 2]);
    xs[i].w = static_cast<R>(type == 2 ? std::log(h.xs[4 * i + 3]) : h.xs[4 * i + 3]);
  }
  c->xs_bytes = nv * sizeof(V4<R>);
  CK(cudaMalloc(&c->d_xs, c->xs_bytes));
  CK(cudaMemcpy(c->d_xs, xs.data(), c->xs_bytes, cudaMemcpyHostToDevice));
  // reciprocal node energies for the FP32 interval fraction
  std::vector<float> inv(kGridN);
  for (int i = 0; i < kGridN; ++i)
    inv[i] = static_cast<float>(std::exp(-(std::log(kGridEmin) + i * std::log(10.0) / kGridPerDecade)));
  CK(cudaMalloc(&c->d_inv_node, sizeof(float) * kGridN));
  CK(cudaMemcpy(c->d_inv_node, inv.data(), sizeof(float) * kGridN, cudaMemcpyHostToDevice));
  // alias bins
  std::vector<AliasBin<R>> bins;
  for (int m = 0; m < kNModel; ++m) {
    c->meta[m].ln_Elo = std::log(h.a_Elo[m]);
    c->meta[m].inv_dl = kAliasPerDecade / std::log(10.0);
    c->meta[m].cut = h.a_cut[m];
    c->meta[m].nE = h.a_nE[m];
    c->meta[m].off = static_cast<int>(bins.size());
    for (int ie = 0; ie < h.a_nE[m]; ++ie)
      for (int j = 0; j < kNB; ++j) {
        AliasBin<R> b;
        b.q = h.a_q[m][static_cast<size_t>(ie) * kNB + j];
        b.a = h.a_alias[m][static_cast<size_t>(ie) * kNB + j];
        b.p0 = static_cast<R>(h.a_pdf[m][static_cast<size_t>(ie) * (kNB + 1) + j]);
        b.p1 = static_cast<R>(h.a_pdf[m][static_cast<size_t>(ie) * (kNB + 1) + j + 1]);
        bins.push_back(b);
      }
  }
  {  // the integral approach's bound
    std::vector<R> sm(h.smax.size());
    for (size_t i = 0; i < sm.size(); ++i) sm[i] = static_cast<R>(h.smax[i]);
    c->smax_bytes = (sm.size() * sizeof(R) + 15) / 16 * 16;
    CK(cudaMalloc(&c->d_smax, c->smax_bytes));
    CK(cudaMemcpy(c->d_smax, sm.data(), sm.size() * sizeof(R), cudaMemcpyHostToDevice));
  }
  c->bins_bytes = bins.size() * sizeof(AliasBin<R>);
  CK(cudaMalloc(&c->d_bins, c->bins_bytes));
  CK(cudaMemcpy(c->d_bins, bins.data(), c->bins_bytes, cudaMemcpyHostToDevice));
  return GV_OK;
}

// Alias bins are read at random by every interaction; a persisting L2
// window keeps them resident while the queues stream through L2.  The
// context's persisting set-aside is raised to the window (if smaller) and put
// back by gv_destroy.
int setup_l2_window(Ctx *c) {
  if (!c->cfg.l2_persist || !c->bins_bytes) return GV_OK;
  int max_persist = 0, max_window = 0;
  CK(cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, c->device));
  CK(cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, c->device));
  const size_t w = std::min(c->bins_bytes, static_cast<size_t>(std::min(max_persist, max_window)));
  if (w == 0) return GV_OK;  // no persisting L2 on this device: nothing to do
  CK(cudaDeviceGetLimit(&c->l2_old_limit, cudaLimitPersistingL2CacheSize));
  if (c->l2_old_limit < w) CK(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, w));
  c->l2_window = w;
  return GV_OK;
}

template <typename R> View<R> make_view(const Ctx *c) {
  View<R> v;
  v.xs = reinterpret_cast<const V4<R> *>(c->d_xs);
  v.inv_node = c->d_inv_node;
  v.zb = c->d_zb;
  v.smat = c->d_smat;
  v.bins = reinterpret_cast<const AliasBin<R> *>(c->d_bins);
  v.smax = reinterpret_cast<const R *>(c->d_smax);
  v.status = nullptr;  // unit kernels: no status word
  for (int m = 0; m < kNModel; ++m) v.meta[m] = c->meta[m];
  v.geo.nsub = c->nsub;
  v.geo.nsub_layer = c->geo.n_sub;
  v.geo.n_layers = c->geo.n_layers;
  v.geo.nx = c->geo.nx_cells;
  v.geo.ny = c->geo.ny_cells;
  v.geo.hx = c->geo.half_x_cm;
  v.geo.hy = c->geo.half_y_cm;
  v.geo.wx[0] = -c->geo.half_x_cm;
  v.geo.wx[1] = c->geo.half_x_cm;
  v.geo.wy[0] = -c->geo.half_y_cm;
  v.geo.wy[1] = c->geo.half_y_cm;
  {  // the half widths rounded down to FP32
    float fx = static_cast<float>(c->geo.half_x_cm), fy = static_cast<float>(c->geo.half_y_cm);
    if (static_cast<double>(fx) > c->geo.half_x_cm) fx = std::nextafter(fx, 0.0f);
    if (static_cast<double>(fy) > c->geo.half_y_cm) fy = std::nextafter(fy, 0.0f);
    v.geo.hx_lo = fx;
    v.geo.hy_lo = fy;
  }
  v.geo.walls_x = c->geo.half_x_cm > 0.0;
  v.geo.walls_y = c->geo.half_y_cm > 0.0;
  v.geo.field_axis = c->geo.field_axis;
  v.rc.field_k = static_cast<R>(2.99792458 * c->geo.field_T);
  v.geo.pitch_x = c->geo.nx_cells > 0 ? 2.0 * c->geo.half_x_cm / c->geo.nx_cells : 1.0;
  v.geo.pitch_y = c->geo.ny_cells > 0 ? 2.0 * c->geo.half_y_cm / c->geo.ny_cells : 1.0;
  v.geo.inv_pitch_x = static_cast<float>(1.0 / v.geo.pitch_x);
  v.geo.inv_pitch_y = static_cast<float>(1.0 / v.geo.pitch_y);
  v.cut.gcut = c->cuts.gamma_cut_MeV;
  v.cut.ecut = c->cuts.e_cut_MeV;
  v.cut.tcut = c->cuts.track_cut_MeV;
  v.rc.tcut = static_cast<R>(c->cuts.track_cut_MeV);
  v.rc.gcut = static_cast<R>(c->cuts.gamma_cut_MeV);
  v.rc.ecut = static_cast<R>(c->cuts.e_cut_MeV);
  v.rc.ecut_push = static_cast<R>(std::max(c->cuts.e_cut_MeV, c->cuts.track_cut_MeV));
  for (int m = 0; m < kNModel; ++m) {
    v.rc.ln_Elo[m] = static_cast<R>(c->meta[m].ln_Elo);
    v.rc.inv_dl[m] = static_cast<R>(c->meta[m].inv_dl);
    v.rc.cut[m] = static_cast<R>(c->meta[m].cut);
  }
  for (int m = 0; m < GV_MAX_MAT; ++m) v.rc.inv_X0[m] = static_cast<R>(c->ht.inv_X0_cm[m]);
  for (int m = 0; m < kNModel; ++m) {  // a threshold beyond R's range means "never"
    const double r = c->cuts.reject_min_MeV[m];
    v.rc.rej_min[m] = r < 1e30 ? static_cast<R>(r) : r_inf_host<R>();
  }
  v.cut.mask = c->cuts.process_mask;
  return v;
}

template <typename R> using StepFn = void (*)(int);

// The step kernel compiled for this configuration: basketizer or not, merged
// or direct scoring, with or without the field propagation.  The basketizing
// kernel also comes without the code of the optional processes (multiple
// scattering, the integral approach, rejection sampling), and without the
// cell histogram and per-event counters, for contexts that use none of
// them: each cut measured about 3 % on the benchmark against carrying the
// code behind run-time switches.
template <typename R> StepFn<R> pick_step_kernel(const Ctx *x) {
  const gv_config &c = x->cfg;
  const bool field = x->geo.field_T != 0.0;
  bool opts = (x->cuts.process_mask & (GV_P_MSC | GV_P_INTEGRAL)) != 0;
  for (int m = 0; m < kNModel; ++m) opts = opts || x->cuts.reject_min_MeV[m] < 1e30;
  // a transport scores cells or per-event counts only if the context has
  // cells or keeps per-event counts: otherwise both pointers stay null
  const bool ext = c.per_event_counts != 0 || static_cast<size_t>(x->geo.n_layers) * x->geo.nx_cells * x->geo.ny_cells != 0;
  if (field)
    return c.process_sort ? step_kernel<R, true, false, true, true, true> : step_kernel<R, false, false, true, true, true>;
  if (c.process_sort) {
    if (c.scoring) return step_kernel<R, true, true, false, true, true>;
    if (opts) return step_kernel<R, true, false, false, true, true>;
    return ext ? step_kernel<R, true, false, false, false, true> : step_kernel<R, true, false, false, false, false>;
  }
  return c.scoring ? step_kernel<R, false, true, false, true, true> : step_kernel<R, false, false, false, true, true>;
}

// The constant-memory state record of each precision and GPU (c_state_f,
// c_state_d) is shared by every context on that GPU.  A transport takes it
// on its stream once the previous transport of any context has released it
// (an event), fills it from its record in device memory, and releases it
// when everything it queued is on the stream.  The host lock orders the
// takes; the events order the uses on the GPU, so transports of different
// contexts on one GPU run one after another.
constexpr int kMaxDevices = 64;
std::mutex &slot_mutex() {
  static std::mutex m;
  return m;
}
cudaEvent_t g_slot_free[2][kMaxDevices];  // [FP64][device]

// Made with a context (gv_setup allocates anyway), so that the
// allocation-free entry point never creates one.
cudaError_t slot_event_create(int device, bool fp64) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(slot_mutex());
  cudaEvent_t &e = g_slot_free[fp64 ? 1 : 0][device];
  if (e) return cudaSuccess;
  return cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
}

template <typename R> class StateSlot {
 public:
  StateSlot(int device, cudaStream_t st)
      : lk_(slot_mutex()), st_(st),
        ev_(device >= 0 && device < kMaxDevices ? g_slot_free[sizeof(R) == 8 ? 1 : 0][device] : nullptr) {}
  StateSlot(const StateSlot &) = delete;
  StateSlot &operator=(const StateSlot &) = delete;
  // wait for the previous user, then copy the record into the slot
  cudaError_t take(const DevState<R> *record) {
    if (!ev_) return cudaErrorInvalidResourceHandle;
    const cudaError_t e = cudaStreamWaitEvent(st_, ev_, 0);
    if (e != cudaSuccess) return e;
    if constexpr (sizeof(R) == 8)
      return cudaMemcpyToSymbolAsync(c_state_d, record, sizeof(DevState<R>), 0, cudaMemcpyDeviceToDevice, st_);
    else
      return cudaMemcpyToSymbolAsync(c_state_f, record, sizeof(DevState<R>), 0, cudaMemcpyDeviceToDevice, st_);
  }
  ~StateSlot() {
    if (ev_) cudaEventRecord(ev_, st_);  // also after an error: what was queued is covered
  }

 private:
  std::unique_lock<std::mutex> lk_;
  cudaStream_t st_;
  cudaEvent_t ev_;
};

template <typename R> int prepare_device(Ctx *c) {
  CK(cudaSetDevice(c->device));
  CK(slot_event_create(c->device, sizeof(R) == 8));
  int rc = upload_tables<R>(c);
  if (rc) return rc;
  rc = setup_l2_window(c);
  if (rc) return rc;
  const long long cap = c->cfg.stack_capacity;
  const size_t per = carve_bytes<R>(cap);
  if (cudaMalloc(&c->d_queues, per * 6) != cudaSuccess) return GV_ERR_OOM;
  CK(cudaMalloc(&c->d_ctl, sizeof(Ctl)));
  CK(cudaMemset(c->d_ctl, 0, sizeof(Ctl)));
  CK(cudaMalloc(&c->d_state, sizeof(DevState<R>)));
  CK(cudaMallocHost(&c->h_ctl, sizeof(Ctl)));
  c->zb_bytes = ((c->nsub + 1) * sizeof(double) + 15) / 16 * 16;
  c->smax_off = c->xs_bytes + c->zb_bytes + kInvNodeBytes + (c->nsub + 15) / 16 * 16;
  c->req_off = c->smax_off + c->smax_bytes;
  if (c->cfg.pipeline) {
    const size_t rc_ = static_cast<size_t>(cap);
    if (cudaMalloc(&c->d_req, rc_ * sizeof(GReq<R>)) != cudaSuccess ||
        cudaMalloc(&c->d_keyidx, rc_ * kNReqKey * sizeof(unsigned)) != cudaSuccess)
      return GV_ERR_OOM;
    c->smem_bytes = c->req_off;
    const void *ka = reinterpret_cast<const void *>(along_kernel<R>);
    const void *kb = reinterpret_cast<const void *>(interact_kernel<R>);
    CK(cudaFuncSetAttribute(ka, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(c->smem_bytes)));
    int occ = 0, occ_b = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ka, c->cfg.block_size, c->smem_bytes));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_b, kb, 256, 0));
    if (occ < 1 || occ_b < 1) return GV_ERR_BAD_ARG;
    c->grid = c->sm_count * std::min(occ, c->cfg.blocks_per_sm);
    c->grid_b = c->sm_count * occ_b;
    return GV_OK;
  }
  c->smem_bytes = c->req_off + (c->cfg.process_sort ? sizeof(IReq<R>) * c->cfg.block_size : 0);
  c->lk_off = (c->smem_bytes + 15) / 16 * 16;
  if (c->cfg.process_sort && c->cfg.local_stack) c->smem_bytes = c->lk_off + sizeof(LKid<R>) * c->cfg.block_size;
  const void *kern = reinterpret_cast<const void *>(pick_step_kernel<R>(c));
  CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(c->smem_bytes)));
  int occ = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, c->cfg.block_size, c->smem_bytes));
  if (occ < 1) return GV_ERR_BAD_ARG;
  c->grid = c->sm_count * std::min(occ, c->cfg.blocks_per_sm);
  return GV_OK;
}

template <typename R> DevState<R> make_state(Ctx *c) {
  DevState<R> s;
  std::memset(&s, 0, sizeof(s));
  s.view = make_view<R>(c);
  unsigned char *p = static_cast<unsigned char *>(c->d_queues);
  for (int par = 0; par < 2; ++par)
    for (int q = 0; q < 3; ++q) s.q[par][q] = carve<R>(p, c->cfg.stack_capacity);
  s.capacity = static_cast<unsigned long long>(c->cfg.stack_capacity);
  s.ctl = c->d_ctl;
  s.view.status = &c->d_ctl->status;  // device address; checks of the checking build
  s.block_size = c->cfg.block_size;
  s.chunk = (c->cfg.pipeline || c->cfg.process_sort || c->cfg.claim_chunks == 0) ? c->cfg.block_size : 32;
  s.grid = c->grid;
  s.adaptive_chunk = (c->cfg.process_sort && !c->cfg.pipeline) ? 1 : 0;
  s.claim_chunks = c->cfg.claim_chunks;
  s.along_steps = c->cfg.along_steps;
  s.along_steps_g = c->cfg.along_steps_photon > 0 ? c->cfg.along_steps_photon : c->cfg.along_steps;
  s.scoring = c->cfg.scoring;
  s.pipeline = c->cfg.pipeline;
  s.req = reinterpret_cast<GReq<R> *>(c->d_req);
  s.keyidx = c->d_keyidx;
  s.req_cap = c->d_req ? static_cast<unsigned long long>(c->cfg.stack_capacity) : 0ull;
  s.mode = c->cfg.mode;
  s.K_bulk = c->cfg.steps_per_claim;
  s.K_tail = c->cfg.tail_steps_per_claim;
  s.tail_threshold = static_cast<unsigned long long>(c->cfg.tail_threshold);
  s.low_water = static_cast<unsigned long long>(c->cfg.mode == GV_ONE_EVENT_PER_LAUNCH ? 1 : c->cfg.refill_low_water);
  s.batch = static_cast<unsigned long long>(c->cfg.refill_batch);
  s.max_gen = static_cast<unsigned long long>(c->cfg.max_generations);
  s.n_mat = static_cast<int>(c->mats.size());
  s.xs_bytes = static_cast<unsigned>(c->xs_bytes);
  s.zb_bytes = static_cast<unsigned>(c->zb_bytes);
  s.smem_req_off = static_cast<unsigned>(c->req_off);
  s.smax_off = static_cast<unsigned>(c->smax_off);
  s.smem_lk_off = static_cast<unsigned>(c->lk_off);
  s.local_stack = c->cfg.local_stack;
  s.smax_bytes = static_cast<unsigned>(c->smax_bytes);
  return s;
}

// The gate at the end of every body of the device-side generation loop: it
// keeps the loop running while the transport is not done.  The loop cannot
// outrun its budget: after max_iter bodies the gate records GV_ERR_TIMEOUT,
// marks the transport done and ends the loop (the generation budget itself
// ends it earlier through plan_next).
__global__ void loop_gate_kernel(Ctl *ctl, cudaGraphConditionalHandle h, unsigned long long max_iter) {
  const unsigned long long it = ++ctl->loop_iter;
  int stop = ctl->done;
  if (!stop && it >= max_iter) {
    if (ctl->status == 0) ctl->status = GV_ERR_TIMEOUT;
    ctl->done = 1;
    stop = 1;
  }
  cudaGraphSetConditional(h, stop ? 0u : 1u);
}

// Puts the persisting-L2 window on every kernel node of g.
cudaError_t set_l2_window(const Ctx *c, cudaGraph_t g) {
  size_t nn = 0;
  cudaError_t e = cudaGraphGetNodes(g, nullptr, &nn);
  std::vector<cudaGraphNode_t> nodes(nn);
  if (e == cudaSuccess && nn) e = cudaGraphGetNodes(g, nodes.data(), &nn);
  cudaKernelNodeAttrValue v{};
  v.accessPolicyWindow.base_ptr = c->d_bins;
  v.accessPolicyWindow.num_bytes = c->l2_window;
  v.accessPolicyWindow.hitRatio = 1.0f;
  v.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
  v.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
  for (size_t i = 0; e == cudaSuccess && i < nn; ++i) {
    cudaGraphNodeType ty;
    e = cudaGraphNodeGetType(nodes[i], &ty);
    if (e == cudaSuccess && ty == cudaGraphNodeTypeKernel)
      e = cudaGraphKernelNodeSetAttribute(nodes[i], cudaKernelNodeAttributeAccessPolicyWindow, &v);
  }
  return e;
}

// The generations of one graph body, recorded on the (capturing) stream.
template <typename R> cudaError_t record_generations(Ctx *c) {
  const DevState<R> *S = reinterpret_cast<const DevState<R> *>(c->d_state);
  if (c->cfg.pipeline) {
    for (int i = 0; i < c->cfg.generations_per_graph; ++i) {
      along_kernel<R><<<c->grid, c->cfg.block_size, c->smem_bytes, c->stream>>>(S, i & 1);
      interact_kernel<R><<<c->grid_b, 256, 0, c->stream>>>(S, i & 1);
    }
    return cudaGetLastError();
  }
  const StepFn<R> step = pick_step_kernel<R>(c);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  for (int i = 0; i < c->cfg.generations_per_graph; ++i) {
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(c->grid);
    lc.blockDim = dim3(c->cfg.block_size);
    lc.dynamicSmemBytes = c->smem_bytes;
    lc.stream = c->stream;
    lc.attrs = attr;
    lc.numAttrs = (c->cfg.pdl && i > 0) ? 1 : 0;  // overlap with the previous generation's tail
    const int parity = i & 1;
    const cudaError_t e = cudaLaunchKernelEx(&lc, step, parity);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// The transport as one graph: a device-side while loop whose body runs
// generations_per_graph generations and then the gate, so the host launches
// once and waits once, and no body starts after the plan that ends the
// transport (the rest of its own body returns at once).
template <typename R> int capture_loop_graph(Ctx *c) {
  cudaGraph_t outer = nullptr;
  if (cudaGraphCreate(&outer, 0) != cudaSuccess) return GV_ERR_CUDA;
  cudaGraphConditionalHandle h;
  cudaGraphNodeParams np = {};
  cudaGraphNode_t node;
  if (cudaGraphConditionalHandleCreate(&h, outer, 1u, cudaGraphCondAssignDefault) != cudaSuccess) {
    cudaGraphDestroy(outer);
    return GV_ERR_CUDA;
  }
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  if (cudaGraphAddNode(&node, outer, nullptr, nullptr, 0, &np) != cudaSuccess) {
    cudaGraphDestroy(outer);
    return GV_ERR_CUDA;
  }
  cudaGraph_t body = np.conditional.phGraph_out[0];
  if (cudaStreamBeginCaptureToGraph(c->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
      cudaSuccess) {
    cudaGraphDestroy(outer);
    return GV_ERR_CUDA;
  }
  cudaError_t e = record_generations<R>(c);
  const unsigned long long max_iter =
      static_cast<unsigned long long>(c->cfg.max_generations) / c->cfg.generations_per_graph + 2;
  if (e == cudaSuccess) {
    loop_gate_kernel<<<1, 1, 0, c->stream>>>(c->d_ctl, h, max_iter);
    e = cudaGetLastError();
  }
  cudaGraph_t captured = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(c->stream, &captured);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess && c->l2_window) e = set_l2_window(c, body);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph, outer, 0);
  cudaGraphDestroy(outer);
  if (e != cudaSuccess) {
    c->graph = nullptr;
    return GV_ERR_CUDA;
  }
  c->loop_graph = 1;
  return GV_OK;
}

template <typename R> int capture_graph(Ctx *c) {
  if (c->graph) return GV_OK;
  c->loop_graph = 0;
  if (c->cfg.device_loop && capture_loop_graph<R>(c) == GV_OK) return GV_OK;
  cudaGetLastError();  // no conditional nodes in this runtime: generations looped by the host
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = record_generations<R>(c);
  const cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess && c->l2_window) e = set_l2_window(c, g);  // the window rides on every step launch
  if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) c->graph = nullptr;
  return e == cudaSuccess ? GV_OK : GV_ERR_CUDA;
}

bool is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Completes the transport in flight (if any): waits for its last copy, then
// fills the caller's result record from the pinned control block.
int finish_pending(Ctx *c) {
  if (!c->pend.active) return c->last_status;
  c->pend.active = false;
  CK(cudaEventSynchronize(c->ev_out));
  const Ctl &h = *c->h_ctl;
  double kernel_ms = c->pend.kernel_ms;
  long long launches = c->pend.launches;
  if (c->pend.timed_loop) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c->t0, c->t1));
    kernel_ms = ms;
    launches += static_cast<long long>(h.loop_iter) * (c->cfg.generations_per_graph * (c->cfg.pipeline ? 2 : 1) + 1);
  }
  c->launches = launches;
  const int status = h.status;
  gv_result *res = c->pend.res;
  if (res) {
    for (int i = 0; i < 16; ++i) res->counters[i] = h.counters[i];
    res->counters[GV_C_GENERATIONS] = h.gen;
    res->counters[15] = h.live_peak;
    res->status = status;
    res->kernel_ms = kernel_ms;
  }
  c->last_status = status;
  return status;
}

template <typename R>
int run_transport(Ctx *c, const gv_primary *p, long long n, long long first_event, long long n_events,
                  unsigned long long seed, cudaStream_t user, gv_result *res) {
  CK(cudaSetDevice(c->device));
  const int nsub = c->nsub;
  const size_t ncell = static_cast<size_t>(c->geo.n_layers) * c->geo.nx_cells * c->geo.ny_cells;
  if (static_cast<size_t>(n_events) > c->ev_cap) {
    cudaFree(c->d_edep);
    cudaFree(c->d_escape);
    cudaFree(c->d_evcnt);
    cudaFree(c->d_evlive);
    cudaFree(c->d_evcost);
    c->d_edep = nullptr;
    c->d_escape = nullptr;
    c->d_evcnt = nullptr;
    c->d_evlive = nullptr;
    c->d_evcost = nullptr;
    c->ev_cap = 0;
    if (cudaMalloc(&c->d_edep, sizeof(double) * n_events * nsub) != cudaSuccess ||
        cudaMalloc(&c->d_escape, sizeof(double) * n_events) != cudaSuccess ||
        cudaMalloc(&c->d_evcnt, sizeof(unsigned long long) * n_events * GV_NCOUNT) != cudaSuccess ||
        cudaMalloc(&c->d_evlive, sizeof(unsigned) * n_events) != cudaSuccess ||
        cudaMalloc(&c->d_evcost, sizeof(unsigned long long) * n_events) != cudaSuccess)
      return GV_ERR_OOM;
    c->ev_cap = n_events;
  }
  // the automatic events-in-flight cap of a batched transport budgets every
  // event by its own primaries (prim_cost_kernel, plan_next)
  const bool cost_cap = c->cfg.max_events_in_flight < 0 && c->cfg.mode == GV_BATCHED && n > 0;
  if (cost_cap && static_cast<size_t>(n) + 1 > c->pcost_cap) {
    cudaFree(c->d_pcost);
    c->d_pcost = nullptr;
    c->pcost_cap = 0;
    if (cudaMalloc(&c->d_pcost, sizeof(unsigned long long) * (n + 1)) != cudaSuccess) return GV_ERR_OOM;
    c->pcost_cap = static_cast<size_t>(n) + 1;
  }
  if (ncell && !c->d_cell) {
    if (cudaMalloc(&c->d_cell, sizeof(double) * ncell) != cudaSuccess) return GV_ERR_OOM;
  }
  const bool dev_prim = is_device_ptr(p);
  std::vector<unsigned> order;
  if (c->cfg.mode == GV_ONE_EVENT_PER_LAUNCH || !dev_prim) {
    if (static_cast<size_t>(n) > c->prim_cap) {
      cudaFree(c->d_prim);
      cudaFree(c->d_order);
      c->d_prim = nullptr;
      c->d_order = nullptr;
      if (cudaMalloc(&c->d_prim, sizeof(gv_primary) * n) != cudaSuccess ||
          cudaMalloc(&c->d_order, sizeof(unsigned) * n) != cudaSuccess)
        return GV_ERR_OOM;
      c->prim_cap = n;
    }
  }
  // the work stream waits for whatever the caller queued before
  CK(cudaEventRecord(c->ev_in, user));
  CK(cudaStreamWaitEvent(c->stream, c->ev_in, 0));
  const gv_primary *dp = p;
  std::vector<gv_primary> hp;
  if (!dev_prim) {
    CK(cudaMemcpyAsync(c->d_prim, p, sizeof(gv_primary) * n, cudaMemcpyHostToDevice, c->stream));
    dp = c->d_prim;
  }
  if (c->cfg.mode == GV_ONE_EVENT_PER_LAUNCH) {
    if (dev_prim) {
      hp.resize(n);
      CK(cudaMemcpyAsync(hp.data(), p, sizeof(gv_primary) * n, cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
    }
    const gv_primary *src = dev_prim ? hp.data() : p;
    order.resize(n);
    for (long long i = 0; i < n; ++i) order[i] = static_cast<unsigned>(i);
    std::stable_sort(order.begin(), order.end(), [src](unsigned a, unsigned b) { return src[a].event < src[b].event; });
    CK(cudaMemcpyAsync(c->d_order, order.data(), sizeof(unsigned) * n, cudaMemcpyHostToDevice, c->stream));
  }
  CK(cudaMemsetAsync(c->d_edep, 0, sizeof(double) * n_events * nsub, c->stream));
  CK(cudaMemsetAsync(c->d_escape, 0, sizeof(double) * n_events, c->stream));
  if (ncell) CK(cudaMemsetAsync(c->d_cell, 0, sizeof(double) * ncell, c->stream));
  const bool evc = c->cfg.per_event_counts != 0 && res && res->event_counts;
  if (evc) CK(cudaMemsetAsync(c->d_evcnt, 0, sizeof(unsigned long long) * n_events * GV_NCOUNT, c->stream));
  CK(cudaMemsetAsync(c->d_evlive, 0, sizeof(unsigned) * n_events, c->stream));
  if (cost_cap) CK(cudaMemsetAsync(c->d_evcost, 0, sizeof(unsigned long long) * n_events, c->stream));
  DevState<R> s = make_state<R>(c);
  s.prim = dp;
  s.order = c->cfg.mode == GV_ONE_EVENT_PER_LAUNCH ? c->d_order : nullptr;
  s.n_prim = static_cast<unsigned>(n);
  s.n_events = static_cast<unsigned>(n_events);
  s.ev_base = static_cast<unsigned>(first_event);
  s.edep = c->d_edep;
  s.cell = (ncell && res && res->cell_edep) ? c->d_cell : nullptr;
  s.escape = c->d_escape;
  s.evcnt = evc ? c->d_evcnt : nullptr;
  s.evlive = c->d_evlive;
  s.max_in_flight = static_cast<int>(std::min<long long>(c->cfg.max_events_in_flight, 0x7fffffffll));
  s.pcost = cost_cap ? c->d_pcost : nullptr;
  s.evcost = cost_cap ? c->d_evcost : nullptr;
  s.seed_lo = static_cast<unsigned>(seed);
  s.seed_hi = static_cast<unsigned>(seed >> 32);
  static thread_local DevState<R> staged;  // pinned copy not needed: synchronous below
  staged = s;
  CK(cudaMemcpyAsync(c->d_state, &staged, sizeof(s), cudaMemcpyHostToDevice, c->stream));
  const DevState<R> *S = reinterpret_cast<const DevState<R> *>(c->d_state);
  StateSlot<R> slot(c->device, c->stream);  // held until every launch below is queued
  CK(slot.take(S));
  if (cost_cap) {
    prim_cost_kernel<R><<<1, kCostScanThreads, 0, c->stream>>>(S, c->d_pcost);
  } else if (s.max_in_flight < 0) {
    CK(cudaMemsetAsync(&c->d_ctl->emax_bits, 0, sizeof(unsigned), c->stream));
    if (n > 0) prim_emax_kernel<R><<<static_cast<int>(std::min<long long>((n + 255) / 256, 4 * c->sm_count)), 256, 0,
                                     c->stream>>>(S);
  }
  init_kernel<R><<<1, 1, 0, c->stream>>>(S);
  CK(cudaGetLastError());
  int rc = capture_graph<R>(c);
  if (rc) return rc;
  long long launches = (s.max_in_flight < 0 && n > 0) ? 2 : 1;
  double kernel_ms = 0.0;
  if (c->loop_graph) {  // one launch: the device-side loop runs until the transport is done
    CK(cudaEventRecord(c->t0, c->stream));
    CK(cudaGraphLaunch(c->graph, c->stream));
    CK(cudaEventRecord(c->t1, c->stream));
  } else {  // the host relaunches the generation graph until the plan says done
    int between = 1;
    for (;;) {
      CK(cudaEventRecord(c->t0, c->stream));
      for (int i = 0; i < between; ++i) CK(cudaGraphLaunch(c->graph, c->stream));
      CK(cudaEventRecord(c->t1, c->stream));
      launches += static_cast<long long>(between) * c->cfg.generations_per_graph * (c->cfg.pipeline ? 2 : 1);
      CK(cudaMemcpyAsync(c->h_ctl, c->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, c->t0, c->t1));
      kernel_ms += ms;
      if (c->h_ctl->done) break;
      between = std::min(between * 2, 64);
    }
  }
  // the control block and the tallies follow on the work stream; the
  // caller's stream waits for them
  CK(cudaMemcpyAsync(c->h_ctl, c->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
  if (res->edep)
    CK(cudaMemcpyAsync(res->edep, c->d_edep, sizeof(double) * n_events * nsub, cudaMemcpyDefault, c->stream));
  if (res->escape_E)
    CK(cudaMemcpyAsync(res->escape_E, c->d_escape, sizeof(double) * n_events, cudaMemcpyDefault, c->stream));
  if (res->cell_edep && ncell)
    CK(cudaMemcpyAsync(res->cell_edep, c->d_cell, sizeof(double) * ncell, cudaMemcpyDefault, c->stream));
  if (evc)
    CK(cudaMemcpyAsync(res->event_counts, c->d_evcnt, sizeof(long long) * n_events * GV_NCOUNT, cudaMemcpyDefault,
                       c->stream));
  CK(cudaEventRecord(c->ev_out, c->stream));
  CK(cudaStreamWaitEvent(user, c->ev_out, 0));
  c->pend.active = true;
  c->pend.res = res;
  c->pend.launches = launches;
  c->pend.kernel_ms = kernel_ms;
  c->pend.timed_loop = c->loop_graph != 0;
  if (c->cfg.blocking || !c->loop_graph) return finish_pending(c);
  return GV_OK;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

int gv_default_config(gv_config *cfg) {
  if (!cfg) return GV_ERR_BAD_ARG;
  cfg->precision = GV_MIXED;
  cfg->mode = GV_BATCHED;
  // measured on 2000 x 10 GeV e- in Pb/polystyrene (GB300): the basketizing
  // kernel with block claims, 2 blocks of 256 per SM, up to 3 along-steps per
  // basket round for electrons and positrons and 5 for photons, one round
  // per claim
  cfg->block_size = 256;
  cfg->blocks_per_sm = 2;
  cfg->steps_per_claim = 1;
  cfg->tail_steps_per_claim = 4;
  cfg->tail_threshold = 1ll << 15;
  cfg->stack_capacity = 1ll << 23;
  cfg->refill_low_water = 1ll << 21;
  cfg->refill_batch = 1ll << 14;
  cfg->generations_per_graph = 16;
  cfg->max_generations = 1ll << 20;
  cfg->per_event_counts = 0;
  cfg->process_sort = 1;
  cfg->max_events_in_flight = -1;
  cfg->claim_chunks = 0;
  cfg->along_steps = 3;
  cfg->along_steps_photon = 5;
  cfg->scoring = 0;
  cfg->l2_persist = 0;
  cfg->pipeline = 0;
  cfg->local_stack = 1;
  cfg->pdl = 1;
  cfg->device_loop = 1;
  cfg->blocking = 0;
  return GV_OK;
}

int gv_setup(void **ctx_out, const gv_material *mats, int n_mats, const gv_layers *geo, const gv_cuts *cuts,
             const gv_config *cfg) {
  if (!ctx_out) return GV_ERR_BAD_ARG;
  *ctx_out = nullptr;
  int rc = validate(mats, n_mats, geo, cuts);
  if (rc) return rc;
  gv_config c;
  gv_default_config(&c);
  if (cfg) c = *cfg;
  rc = validate_cfg(c);
  if (rc) return rc;
  if (geo->field_T != 0.0 && c.scoring != 0) return GV_ERR_BAD_ARG;  // no merged-scoring field kernel
  Ctx *x = new Ctx();
  x->cfg = c;
  x->mats.assign(mats, mats + n_mats);
  x->geo = *geo;
  x->cuts = *cuts;
  x->nsub = geo->n_layers * geo->n_sub;
  x->zb.resize(x->nsub + 1);
  x->smat.resize(x->nsub);
  double z = 0.0;
  x->zb[0] = 0.0;
  for (int l = 0; l < geo->n_layers; ++l)
    for (int j = 0; j < geo->n_sub; ++j) {
      const int k = l * geo->n_sub + j;
      z += geo->sub_thick_cm[j];
      x->zb[k + 1] = z;
      x->smat[k] = static_cast<unsigned char>(geo->sub_mat[j]);
    }
  if (cudaGetDevice(&x->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&x->sm_count, cudaDevAttrMultiProcessorCount, x->device) != cudaSuccess) {
    delete x;
    return GV_ERR_CUDA;
  }
  if (cudaMalloc(&x->d_zb, sizeof(double) * (x->nsub + 1)) != cudaSuccess ||
      cudaMalloc(&x->d_smat, x->nsub) != cudaSuccess ||
      cudaMemcpy(x->d_zb, x->zb.data(), sizeof(double) * (x->nsub + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(x->d_smat, x->smat.data(), x->nsub, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaStreamCreateWithFlags(&x->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&x->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&x->ev_out, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreate(&x->t0) != cudaSuccess || cudaEventCreate(&x->t1) != cudaSuccess) {
    gv_destroy(x);
    return GV_ERR_CUDA;
  }
  *ctx_out = x;
  return GV_OK;
}

int gv_build_tables(void *ctx) {
  Ctx *c = static_cast<Ctx *>(ctx);
  if (!c) return GV_ERR_BAD_ARG;
  if (c->tables) return GV_OK;
  std::string err;
  int rc = build_host_tables(c->mats.data(), static_cast<int>(c->mats.size()), c->cuts, &c->ht, &err);
  if (rc) return rc;
  rc = c->cfg.precision == GV_FP64 ? prepare_device<double>(c) : prepare_device<float>(c);
  if (rc) return rc;
  c->tables = true;
  return GV_OK;
}

int gv_transport_events(void *ctx, const gv_primary *p, long long n, long long first_event, long long n_events,
                        unsigned long long seed, void *stream, gv_result *res) {
  Ctx *c = static_cast<Ctx *>(ctx);
  if (!c || (!p && n > 0) || n < 0 || n_events < 1 || n > 0xffffffffll || first_event < 0 ||
      first_event + n_events > 0xffffffffll)
    return GV_ERR_BAD_ARG;
  if (!c->tables) return GV_ERR_NO_TABLES;
  if (!res || !res->edep) return GV_ERR_BAD_ARG;
  if (res->event_counts && !c->cfg.per_event_counts) return GV_ERR_BAD_ARG;
  if (!is_device_ptr(p)) {
    for (long long i = 0; i < n; ++i)
      if (p[i].type < 0 || p[i].type > 2 || p[i].event < static_cast<unsigned long long>(first_event) ||
          p[i].event - static_cast<unsigned long long>(first_event) >= static_cast<unsigned long long>(n_events) ||
          !(p[i].E_MeV >= 0))
        return GV_ERR_BAD_ARG;
  }
  finish_pending(c);  // the previous transport of this context completes first
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return c->cfg.precision == GV_FP64 ? run_transport<double>(c, p, n, first_event, n_events, seed, s, res)
                                     : run_transport<float>(c, p, n, first_event, n_events, seed, s, res);
}

int gv_transport(void *ctx, const gv_primary *p, long long n, long long n_events, unsigned long long seed,
                 void *stream, gv_result *res) {
  return gv_transport_events(ctx, p, n, 0, n_events, seed, stream, res);
}

int gv_sync(void *ctx, void *stream) {
  Ctx *c = static_cast<Ctx *>(ctx);
  if (!c) return GV_ERR_BAD_ARG;
  const int rc = finish_pending(c);
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return GV_ERR_CUDA;
  return rc;
}

long long gv_last_launches(void *ctx) {
  Ctx *c = static_cast<Ctx *>(ctx);
  return c ? c->launches : -1;
}

void gv_destroy(void *ctx) {
  Ctx *c = static_cast<Ctx *>(ctx);
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  c->pend.active = false;  // a result not collected by gv_sync stays unfilled
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->l2_window) {  // release the persisting lines and the set-aside taken at setup
    cudaCtxResetPersistingL2Cache();
    cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, c->l2_old_limit);
  }
  cudaFree(c->d_xs);
  cudaFree(c->d_inv_node);
  cudaFree(c->d_bins);
  cudaFree(c->d_smax);
  cudaFree(c->d_zb);
  cudaFree(c->d_smat);
  cudaFree(c->d_queues);
  cudaFree(c->d_ctl);
  cudaFree(c->d_state);
  cudaFree(c->d_edep);
  cudaFree(c->d_cell);
  cudaFree(c->d_escape);
  cudaFree(c->d_evcnt);
  cudaFree(c->d_evlive);
  cudaFree(c->d_evcost);
  cudaFree(c->d_pcost);
  cudaFree(c->d_prim);
  cudaFree(c->d_order);
  cudaFree(c->d_req);
  cudaFree(c->d_keyidx);
  if (c->h_ctl) cudaFreeHost(c->h_ctl);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->t0) cudaEventDestroy(c->t0);
  if (c->t1) cudaEventDestroy(c->t1);
  if (c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

const char *gv_strerror(int code) {
  switch (code) {
    case GV_OK: return "ok";
    case GV_ERR_BAD_ARG: return "bad argument";
    case GV_ERR_NO_TABLES: return "tables not built";
    case GV_ERR_OOM: return "device allocation failed";
    case GV_ERR_STACK_FULL: return "track queue overflow";
    case GV_ERR_TIMEOUT: return "generation budget exhausted";
    case GV_ERR_NUMERIC: return "non-finite track state";
    case GV_ERR_CUDA: return "CUDA runtime error";
    case GV_ERR_INTERNAL: return "internal check failed";
    default: return "unknown error";
  }
}

}  // extern "C"

// exported for the element-wise entry points (gv_unit.cu)
namespace gv {
int ctx_views(void *ctx, int *precision, View<float> *vf, View<double> *vd) {
  Ctx *c = static_cast<Ctx *>(ctx);
  if (!c) return GV_ERR_BAD_ARG;
  if (!c->tables) return GV_ERR_NO_TABLES;
  *precision = c->cfg.precision;
  if (c->cfg.precision == GV_FP64) *vd = make_view<double>(c);
  else *vf = make_view<float>(c);
  return GV_OK;
}
int ctx_nmat(void *ctx) { return static_cast<int>(static_cast<Ctx *>(ctx)->mats.size()); }
}  // namespace gv

// ====================================================================== transport without allocation
// Some callers must not have this library allocate device memory while they
// run: a host framework that hands out all of a GPU's memory from its own
// pools under a fixed budget (as large event-processing frameworks do) cannot
// let a library call cudaMalloc behind its back, and cudaMalloc/cudaFree also
// synchronise the whole device and may fail or stall under memory pressure.
// gv_transport_static runs the same step kernel as gv_transport, but keeps
// every piece of scratch memory it needs -- the double-buffered track queues,
// the generation control block, the kernel's state record and the per-event
// live-track counts -- in the file-scope array below, sized once for a modest
// maximum.  The array is part of the module image: every GPU that loads
// libgv holds it until the process exits.
namespace {
constexpr long long kStaticCap = 1 << 16;         // tracks per particle type and buffer
constexpr long long kStaticMaxEvents = 1 << 16;   // events per call
constexpr size_t kStaticCtlOff = 0;
constexpr size_t kStaticStateOff = 4096;
constexpr size_t kStaticEvliveOff = 12288;
constexpr size_t kStaticQueueOff = kStaticEvliveOff + sizeof(unsigned) * kStaticMaxEvents;
constexpr size_t kStaticQueueBytes = 6 * static_cast<size_t>(kStaticCap) * track_bytes<float>();
constexpr size_t kStaticBytes = kStaticQueueOff + kStaticQueueBytes;  // 25,440,256 bytes
static_assert(sizeof(Ctl) <= kStaticStateOff - kStaticCtlOff, "control block does not fit");
static_assert(sizeof(DevState<float>) <= kStaticEvliveOff - kStaticStateOff, "state does not fit");
static_assert(kStaticCap % 64 == 0, "queue arrays must stay 256-byte aligned");
}  // namespace

static __device__ __align__(256) unsigned char g_gv_static_scratch[kStaticBytes];

namespace {

// Device address of the scratch array on the current device.  Host code only
// sees a host-side stand-in under the array's name, so the address is asked
// of the runtime, with the device current, on every call: a cached address
// would outlive a device reset or a new primary context.
int static_scratch(unsigned char **base) {
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_gv_static_scratch) != cudaSuccess || !p) {
    cudaGetLastError();
    return GV_ERR_CUDA;
  }
  *base = static_cast<unsigned char *>(p);
  return GV_OK;
}

// carve the queues of the scratch array exactly as carve() does for the
// context's own allocation (every array a multiple of 256 bytes long)
Queue<float> carve_static(unsigned char *&p) {
  Queue<float> q;
  auto take = [&](size_t n) {
    unsigned char *r = p;
    p += n;
    return r;
  };
  const size_t C = static_cast<size_t>(kStaticCap);
  q.x = reinterpret_cast<double *>(take(C * 8));
  q.y = reinterpret_cast<double *>(take(C * 8));
  q.z = reinterpret_cast<double *>(take(C * 8));
  q.u = reinterpret_cast<float *>(take(C * 4));
  q.v = reinterpret_cast<float *>(take(C * 4));
  q.w = reinterpret_cast<float *>(take(C * 4));
  q.E = reinterpret_cast<float *>(take(C * 4));
  q.nlam = reinterpret_cast<float *>(take(C * 4));
  q.id = reinterpret_cast<unsigned long long *>(take(C * 8));
  q.ev = reinterpret_cast<unsigned *>(take(C * 4));
  q.step = reinterpret_cast<unsigned *>(take(C * 4));
  q.sf = reinterpret_cast<int *>(take(C * 4));
  return q;
}

// the state record travels as a kernel argument, so no staging copy is needed
__global__ void static_state_kernel(DevState<float> s, DevState<float> *dst) {
  *dst = s;
  s.ctl->emax_bits = 0u;
}

}  // namespace

extern "C" int gv_transport_static(void *ctx, const gv_primary *prim, long long n, long long n_events,
                                   unsigned long long seed, void *stream, double *edep, double *escape_E,
                                   unsigned long long *counters) {
  Ctx *c = static_cast<Ctx *>(ctx);
  if (!c || n < 0 || (n > 0 && !prim) || n_events < 1 || !edep || !escape_E || !counters) return GV_ERR_BAD_ARG;
  if (!c->tables) return GV_ERR_NO_TABLES;
  if (c->cfg.precision != GV_MIXED) return GV_ERR_BAD_ARG;  // the array is sized for the mixed layout
  if (c->geo.field_T != 0.0) return GV_ERR_BAD_ARG;          // its kernel is the field-free one
  if (n_events > kStaticMaxEvents || n > 0xffffffffll) return GV_ERR_BAD_ARG;
  if (cudaSetDevice(c->device) != cudaSuccess) return GV_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  {  // the call waits on the host between launches: a capturing stream cannot take it
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
      cudaGetLastError();
      return GV_ERR_CUDA;
    }
    if (cs != cudaStreamCaptureStatusNone) return GV_ERR_BAD_ARG;
  }
  if ((n > 0 && !is_device_ptr(prim)) || !is_device_ptr(edep) || !is_device_ptr(escape_E)) return GV_ERR_BAD_ARG;
  finish_pending(c);  // a gv_transport of this context still in flight completes first
  unsigned char *base = nullptr;
  int rc = static_scratch(&base);
  if (rc) return rc;
  const size_t smem = c->req_off;  // tables and geometry; the non-basketizing kernel
  if (cudaFuncSetAttribute(step_kernel<float, false, false, false, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem)) != cudaSuccess)
    return GV_ERR_CUDA;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, step_kernel<float, false, false, false, true, true>, c->cfg.block_size, smem) !=
          cudaSuccess ||
      occ < 1)
    return GV_ERR_CUDA;
  const int grid = c->sm_count * std::min(occ, c->cfg.blocks_per_sm);
  // the tallies and the event counts start from zero on every call
  if (cudaMemsetAsync(edep, 0, sizeof(double) * n_events * c->nsub, st) != cudaSuccess ||
      cudaMemsetAsync(escape_E, 0, sizeof(double) * n_events, st) != cudaSuccess ||
      cudaMemsetAsync(base + kStaticEvliveOff, 0, sizeof(unsigned) * n_events, st) != cudaSuccess)
    return GV_ERR_CUDA;
  DevState<float> s = make_state<float>(c);
  unsigned char *qp = base + kStaticQueueOff;
  for (int par = 0; par < 2; ++par)
    for (int q = 0; q < 3; ++q) s.q[par][q] = carve_static(qp);
  s.capacity = static_cast<unsigned long long>(kStaticCap);
  s.ctl = reinterpret_cast<Ctl *>(base + kStaticCtlOff);
  s.view.status = &s.ctl->status;
  s.mode = GV_BATCHED;
  s.chunk = c->cfg.block_size;  // the non-basketizing kernel, one claim per block
  s.adaptive_chunk = 0;
  s.claim_chunks = 0;
  s.low_water = static_cast<unsigned long long>(kStaticCap / 4);
  s.batch = std::min<unsigned long long>(s.batch, 64);
  s.max_in_flight = -1;  // automatic: capacity / (0.15 per MeV of the most energetic primary + 64)
  s.prim = prim;
  s.order = nullptr;
  s.n_prim = static_cast<unsigned>(n);
  s.n_events = static_cast<unsigned>(n_events);
  s.edep = edep;
  s.cell = nullptr;
  s.escape = escape_E;
  s.evcnt = nullptr;
  s.evlive = reinterpret_cast<unsigned *>(base + kStaticEvliveOff);
  s.ev_base = 0;
  s.seed_lo = static_cast<unsigned>(seed);
  s.seed_hi = static_cast<unsigned>(seed >> 32);
  DevState<float> *S = reinterpret_cast<DevState<float> *>(base + kStaticStateOff);
  StateSlot<float> slot(c->device, st);  // held until the last generation is queued
  static_state_kernel<<<1, 1, 0, st>>>(s, S);
  if (slot.take(S) != cudaSuccess) return GV_ERR_CUDA;
  if (n > 0)
    prim_emax_kernel<float><<<static_cast<int>(std::min<long long>((n + 255) / 256, 4 * c->sm_count)), 256, 0, st>>>(S);
  init_kernel<float><<<1, 1, 0, st>>>(S);
  if (cudaGetLastError() != cudaSuccess) return GV_ERR_CUDA;
  int between = 1;
  for (;;) {
    for (int i = 0; i < 2 * between; ++i)
      step_kernel<float, false, false, false, true, true><<<grid, c->cfg.block_size, smem, st>>>(i & 1);
    if (cudaGetLastError() != cudaSuccess) return GV_ERR_CUDA;
    if (cudaMemcpyAsync(c->h_ctl, s.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return GV_ERR_CUDA;
    if (c->h_ctl->done) break;
    between = std::min(between * 2, 32);
  }
  for (int i = 0; i < 16; ++i) counters[i] = c->h_ctl->counters[i];
  counters[GV_C_GENERATIONS] = c->h_ctl->gen;
  counters[15] = c->h_ctl->live_peak;
  c->last_status = c->h_ctl->status;  // what a later gv_sync on this context reports
  return c->last_status;
}
