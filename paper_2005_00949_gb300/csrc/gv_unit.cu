// gv_unit.cu -- element-wise entry points over the device functions of one
// transport step: Philox, table lookup, continuous loss, alias sampling,
// final states and the slab navigator.  Each runs one element per thread in
// the context's precision, reading the tables from global memory.
#include <cuda_runtime.h>

#include "gv_device.cuh"

namespace gv {
int ctx_views(void *ctx, int *precision, View<float> *vf, View<double> *vd);
int ctx_nmat(void *ctx);

namespace {

constexpr int kThreads = 256;

inline int blocks_for(long long n) { return static_cast<int>((n + kThreads - 1) / kThreads); }

__global__ void k_philox(const unsigned *ctr, const unsigned *key, unsigned *out, long long n) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
  const uint4 r = philox4x32_10(c, key[2 * i], key[2 * i + 1]);
  out[4 * i] = r.x;
  out[4 * i + 1] = r.y;
  out[4 * i + 2] = r.z;
  out[4 * i + 3] = r.w;
}

template <typename R>
__global__ void k_lookup(View<R> V, int type, int mat, const double *E, long long n, double *out) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const V4<R> v = lookup(V, mat, type, static_cast<R>(E[i]));
  out[4 * i] = v.x;
  out[4 * i + 1] = v.y;
  out[4 * i + 2] = type == 1 ? range_of(v, type) : v.z;  // the range, from its interpolated logarithm
  out[4 * i + 3] = type == 2 ? range_of(v, type) : v.w;
}

template <typename R>
__global__ void k_eloss(View<R> V, int type, int mat, const double *E, const double *s, long long n, double *out) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  out[i] = eloss(V, mat, type, static_cast<R>(E[i]), static_cast<R>(s[i]));
}

template <typename R>
__global__ void k_alias(View<R> V, int model, const double *E, const double *u, long long n, double *out) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  R xi;
  const R v = alias_sample<R>(V, model, static_cast<R>(E[i]), static_cast<R>(u[3 * i]), static_cast<R>(u[3 * i + 1]),
                              static_cast<R>(u[3 * i + 2]), &xi);
  out[2 * i] = v;
  out[2 * i + 1] = xi;
}

template <typename R>
__global__ void k_interact(View<R> V, int type, int proc, const double *E, const double *dir, const double *u,
                           long long n, double *out, int *ret) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  R e = static_cast<R>(E[i]);
  R d[3] = {static_cast<R>(dir[3 * i]), static_cast<R>(dir[3 * i + 1]), static_cast<R>(dir[3 * i + 2])};
  R uu[8];
  for (int j = 0; j < 8; ++j) uu[j] = static_cast<R>(u[8 * i + j]);
  Kids<R> kids;
  kids.n = 0;
  R local = R(0);
  int np = 0, na = 0;
  // a rejection sampler, where configured, draws from the stream (i, 0, 0) under key (0, 0)
  const RngKey g = {static_cast<uint32_t>(i), static_cast<uint32_t>(i >> 32), 0u, 0u, 0u};
  const int r = interact(V, type, proc, e, d, uu, g, kids, local, np, na);
  double *o = out + 24 * i;
  for (int j = 0; j < 24; ++j) o[j] = 0.0;
  o[0] = r == 1 ? static_cast<double>(e) : (r == 0 ? -1.0 : E[i]);
  o[1] = d[0];
  o[2] = d[1];
  o[3] = d[2];
  o[4] = local;
  o[5] = kids.n;
  for (int j = 0; j < kids.n; ++j) {
    o[6 + 5 * j] = kids.type[j];
    o[7 + 5 * j] = kids.E[j];
    o[8 + 5 * j] = kids.d[j][0];
    o[9 + 5 * j] = kids.d[j][1];
    o[10 + 5 * j] = kids.d[j][2];
  }
  ret[i] = r;
}

template <typename R>
__global__ void k_distance(View<R> V, const double *pos, const double *dir, const int *sub, long long n, double *dist,
                           int *next, int *plane) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  int nx, pl;
  if (sub[i] < 0 || sub[i] >= V.geo.nsub) {  // not a sub-slab: report, touch no table
    dist[i] = -1.0;
    next[i] = -1;
    plane[i] = -1;
    return;
  }
  const R d = distance(V, pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], static_cast<R>(dir[3 * i]),
                       static_cast<R>(dir[3 * i + 1]), static_cast<R>(dir[3 * i + 2]), sub[i], nx, pl);
  dist[i] = d;
  next[i] = nx;
  plane[i] = pl;
}

template <typename R>
__global__ void k_msc(View<R> V, const int *sub, const double *Ea, const double *Eb, const double *sv,
                      const double *dir, const double *pos, const double *u, long long n, double *od, double *op) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  if (sub[i] < 0 || sub[i] >= V.geo.nsub) {  // not a sub-slab: report, touch no table
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    for (int j = 0; j < 3; ++j) od[3 * i + j] = op[3 * i + j] = nan;
    return;
  }
  R d[3] = {static_cast<R>(dir[3 * i]), static_cast<R>(dir[3 * i + 1]), static_cast<R>(dir[3 * i + 2])};
  const R uu[4] = {static_cast<R>(u[4 * i]), static_cast<R>(u[4 * i + 1]), static_cast<R>(u[4 * i + 2]),
                   static_cast<R>(u[4 * i + 3])};
  double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
  msc_step(V, sub[i], static_cast<R>(Ea[i]), static_cast<R>(Eb[i]), static_cast<R>(sv[i]), d, x, y, z, uu);
  od[3 * i] = d[0];
  od[3 * i + 1] = d[1];
  od[3 * i + 2] = d[2];
  op[3 * i] = x;
  op[3 * i + 1] = y;
  op[3 * i + 2] = z;
}

template <typename R>
__global__ void k_field(View<R> V, int type, const double *E, const double *sv, const double *dir, long long n,
                        double *out) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const R d[3] = {static_cast<R>(dir[3 * i]), static_cast<R>(dir[3 * i + 1]), static_cast<R>(dir[3 * i + 2])};
  R dp[3], nd[3];
  const R e = static_cast<R>(E[i]);
  helix(V, type, e, static_cast<R>(sv[i]), d, dp, nd);
  for (int j = 0; j < 3; ++j) {
    out[7 * i + j] = dp[j];
    out[7 * i + 3 + j] = nd[j];
  }
  out[7 * i + 6] = field_limit(V, type, e, d[0], d[1], d[2]);
}

template <typename R>
__global__ void k_sample(View<R> V, int model, int method, const double *E, long long n, uint32_t k0, uint32_t k1,
                         double *out) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const RngKey g = {static_cast<uint32_t>(i), static_cast<uint32_t>(i >> 32), 0u, k0, k1};
  const R e = static_cast<R>(E[i]);
  R xi, v;
  int tr = 1;
  if (method == 1) {
    v = reject_sample<R>(V, model, e, g, &xi, &tr);
  } else {
    const uint4 w = philox4x32_10(make_uint4(g.idlo, g.idhi, 0u, 0u), k0, k1);
    v = alias_sample<R>(V, model, e, u24<R>(w.x), u24<R>(w.y), u24<R>(w.z), &xi);
  }
  out[3 * i] = v;
  out[3 * i + 1] = xi;
  out[3 * i + 2] = tr;
}

int launch_status() { return cudaGetLastError() == cudaSuccess ? GV_OK : GV_ERR_CUDA; }

}  // namespace
}  // namespace gv

using namespace gv;

extern "C" {

int gv_unit_philox(const unsigned *ctr, const unsigned *key, unsigned *out, long long n, void *stream) {
  if (n < 0 || (n > 0 && (!ctr || !key || !out))) return GV_ERR_BAD_ARG;
  if (n == 0) return GV_OK;
  k_philox<<<blocks_for(n), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(ctr, key, out, n);
  return launch_status();
}

#define GV_UNIT_DISPATCH(launch_f, launch_d)        \
  int prec;                                         \
  View<float> vf;                                   \
  View<double> vd;                                  \
  int rc = ctx_views(ctx, &prec, &vf, &vd);         \
  if (rc) return rc;                                \
  cudaStream_t s = static_cast<cudaStream_t>(stream); \
  if (prec == GV_FP64) { launch_d; } else { launch_f; } \
  return launch_status();

int gv_unit_xs_lookup(void *ctx, int type, int mat, const double *E, long long n, double *out, void *stream) {
  if (!ctx || type < 0 || type > 2 || n < 0 || (n > 0 && (!E || !out))) return GV_ERR_BAD_ARG;
  if (mat < 0 || mat >= ctx_nmat(ctx)) return GV_ERR_BAD_ARG;
  if (n == 0) return GV_OK;
  GV_UNIT_DISPATCH((k_lookup<float><<<blocks_for(n), kThreads, 0, s>>>(vf, type, mat, E, n, out)),
                   (k_lookup<double><<<blocks_for(n), kThreads, 0, s>>>(vd, type, mat, E, n, out)))
}

int gv_unit_eloss(void *ctx, int type, int mat, const double *E, const double *sv, long long n, double *out,
                  void *stream) {
  if (!ctx || type < 1 || type > 2 || n < 0 || (n > 0 && (!E || !sv || !out))) return GV_ERR_BAD_ARG;
  if (mat < 0 || mat >= ctx_nmat(ctx)) return GV_ERR_BAD_ARG;
  if (n == 0) return GV_OK;
  GV_UNIT_DISPATCH((k_eloss<float><<<blocks_for(n), kThreads, 0, s>>>(vf, type, mat, E, sv, n, out)),
                   (k_eloss<double><<<blocks_for(n), kThreads, 0, s>>>(vd, type, mat, E, sv, n, out)))
}

int gv_unit_alias_sample(void *ctx, int model, const double *E, const double *u, long long n, double *out,
                         void *stream) {
  if (!ctx || model < 0 || model >= kNModel || n < 0 || (n > 0 && (!E || !u || !out))) return GV_ERR_BAD_ARG;
  if (n == 0) return GV_OK;
  GV_UNIT_DISPATCH((k_alias<float><<<blocks_for(n), kThreads, 0, s>>>(vf, model, E, u, n, out)),
                   (k_alias<double><<<blocks_for(n), kThreads, 0, s>>>(vd, model, E, u, n, out)))
}

int gv_unit_interact(void *ctx, int type, int proc, const double *E, const double *dir, const double *u, long long n,
                     double *out, int *ret, void *stream) {
  if (!ctx || type < 0 || type > 2 || proc < 0 || proc > (type == 1 ? 1 : 2) || n < 0 ||
      (n > 0 && (!E || !dir || !u || !out || !ret)))
    return GV_ERR_BAD_ARG;
  if (n == 0) return GV_OK;
  GV_UNIT_DISPATCH((k_interact<float><<<blocks_for(n), kThreads, 0, s>>>(vf, type, proc, E, dir, u, n, out, ret)),
                   (k_interact<double><<<blocks_for(n), kThreads, 0, s>>>(vd, type, proc, E, dir, u, n, out, ret)))
}

int gv_unit_distance(void *ctx, const double *pos, const double *dir, const int *sub, long long n, double *dist,
                     int *next, int *plane, void *stream) {
  if (!ctx || n < 0 || (n > 0 && (!pos || !dir || !sub || !dist || !next || !plane))) return GV_ERR_BAD_ARG;
  if (n == 0) return GV_OK;
  GV_UNIT_DISPATCH((k_distance<float><<<blocks_for(n), kThreads, 0, s>>>(vf, pos, dir, sub, n, dist, next, plane)),
                   (k_distance<double><<<blocks_for(n), kThreads, 0, s>>>(vd, pos, dir, sub, n, dist, next, plane)))
}

int gv_unit_msc(void *ctx, const int *sub, const double *E_pre, const double *E_post, const double *sv,
                const double *dir, const double *pos, const double *u, long long n, double *out_dir,
                double *out_pos, void *stream) {
  if (!ctx || n < 0 || (n > 0 && (!sub || !E_pre || !E_post || !sv || !dir || !pos || !u || !out_dir || !out_pos)))
    return GV_ERR_BAD_ARG;
  if (n == 0) return GV_OK;
  GV_UNIT_DISPATCH(
      (k_msc<float><<<blocks_for(n), kThreads, 0, s>>>(vf, sub, E_pre, E_post, sv, dir, pos, u, n, out_dir, out_pos)),
      (k_msc<double><<<blocks_for(n), kThreads, 0, s>>>(vd, sub, E_pre, E_post, sv, dir, pos, u, n, out_dir, out_pos)))
}

int gv_unit_field(void *ctx, int type, const double *E, const double *sv, const double *dir, long long n,
                  double *out, void *stream) {
  if (!ctx || type < 1 || type > 2 || n < 0 || (n > 0 && (!E || !sv || !dir || !out))) return GV_ERR_BAD_ARG;
  if (n == 0) return GV_OK;
  GV_UNIT_DISPATCH((k_field<float><<<blocks_for(n), kThreads, 0, s>>>(vf, type, E, sv, dir, n, out)),
                   (k_field<double><<<blocks_for(n), kThreads, 0, s>>>(vd, type, E, sv, dir, n, out)))
}

int gv_unit_sample(void *ctx, int model, int method, const double *E, long long n, unsigned long long seed,
                   double *out, void *stream) {
  if (!ctx || model < 0 || model >= kNModel || method < 0 || method > 1 || n < 0 || (n > 0 && (!E || !out)))
    return GV_ERR_BAD_ARG;
  if (method == 1 && model > kBrem) return GV_ERR_BAD_ARG;  // rejection is built for Compton, pair, brems
  if (n == 0) return GV_OK;
  const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
  GV_UNIT_DISPATCH((k_sample<float><<<blocks_for(n), kThreads, 0, s>>>(vf, model, method, E, n, k0, k1, out)),
                   (k_sample<double><<<blocks_for(n), kThreads, 0, s>>>(vd, model, method, E, n, k0, k1, out)))
}

}  // extern "C"
