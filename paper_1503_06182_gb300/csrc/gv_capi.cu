// gv_capi.cu -- host engine behind include/vegas.h.
//
// A context owns the device state of one VEGAS integration (grid pack,
// iteration state, accumulators) and, unless the caller hands it one, the
// workspace (tile partials, per-iteration records).  A stage of itmx
// iterations (Section 2.1; the two-stage runs of Section 3.2) is enqueued as
//   itmx x [fill -> reduce (with the per-axis grid refinement)]
// (with a histogram, its kernel after each reduce; with VEGAS+, the
// segment, statistics, allocation and layout kernels after each reduce),
// and, by default, captured once into a CUDA graph that is replayed by later
// calls with the same shape; the iteration counter, the derived integrand
// constants and the grid are read from device memory, so a replay needs no
// re-capture.  The constants are re-derived (one small kernel, outside the
// graph) only when the integrand or its parameters change.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/vegas.h"
#include "gv_fill.cuh"

namespace gv {
cudaError_t launch_fill_gauss(int fp32, int ept, const GvFillArgs& a, int n_tiles, size_t smem,
                              cudaStream_t s, bool pdl);
cudaError_t launch_fill_dy(int fp32, int ept, const GvFillArgs& a, int n_tiles, size_t smem,
                           cudaStream_t s, bool pdl);
cudaError_t launch_fill_ee3j(int fp32, int ept, const GvFillArgs& a, int n_tiles, size_t smem,
                             cudaStream_t s, bool pdl);
cudaError_t launch_fill_dynlo(int fp32, int ept, const GvFillArgs& a, int n_tiles, size_t smem,
                             cudaStream_t s, bool pdl);
cudaError_t launch_fill_gauss_eval(int fp32, const GvFillArgs& a, uint32_t it, const long long* ev,
                                   long long n, double* w, int* bins, cudaStream_t s);
cudaError_t launch_fill_dy_eval(int fp32, const GvFillArgs& a, uint32_t it, const long long* ev,
                                long long n, double* w, int* bins, cudaStream_t s);
cudaError_t launch_fill_ee3j_eval(int fp32, const GvFillArgs& a, uint32_t it, const long long* ev,
                                  long long n, double* w, int* bins, cudaStream_t s);
cudaError_t launch_fill_dynlo_eval(int fp32, const GvFillArgs& a, uint32_t it, const long long* ev,
                                  long long n, double* w, int* bins, cudaStream_t s);
// The last CUDA error behind a VEGAS_ECUDA status, per host thread.
cudaError_t& last_cuda_error() {
  static thread_local cudaError_t e = cudaSuccess;
  return e;
}
}  // namespace gv

namespace {

#define GV_TRY(expr)                   \
  do {                                 \
    cudaError_t _e = (expr);           \
    if (_e != cudaSuccess) {           \
      gv_last_cuda_error() = _e;       \
      return VEGAS_ECUDA;              \
    }                                  \
  } while (0)

cudaError_t& gv_last_cuda_error() { return gv::last_cuda_error(); }

cudaError_t launch_fill_any(int ig, int fp32, int ept, const GvFillArgs& a, int n_tiles,
                            size_t smem, cudaStream_t s, bool pdl) {
  switch (ig) {
    case GV_GAUSS: return gv::launch_fill_gauss(fp32, ept, a, n_tiles, smem, s, pdl);
    case GV_DY: return gv::launch_fill_dy(fp32, ept, a, n_tiles, smem, s, pdl);
    case GV_EE3J: return gv::launch_fill_ee3j(fp32, ept, a, n_tiles, smem, s, pdl);
    case GV_DYNLO: return gv::launch_fill_dynlo(fp32, ept, a, n_tiles, smem, s, pdl);
  }
  return cudaErrorInvalidValue;
}

// Parameter validation: counts and physical ranges.
int check_params(int ig, int ndim, const double* p, int np) {
  if (!p && np > 0) return VEGAS_EINVAL;
  for (int i = 0; i < np; ++i)
    if (!std::isfinite(p[i])) return VEGAS_EINVAL;
  switch (ig) {
    case VEGAS_GAUSS:
      if ((np != 1 && np != 2) || ndim < 1 || !(p[0] > 0.0)) return VEGAS_EINVAL;
      return VEGAS_OK;
    case VEGAS_DY:
      if (np != 10 || ndim < 4) return VEGAS_EINVAL;
      if (!(p[0] > 0 && p[1] > 0 && p[2] > 0 && p[3] > 0 && p[3] < 1 && p[4] > 0 && p[5] > 0 &&
            p[6] > p[5] && p[6] < p[0] && p[9] > 0))
        return VEGAS_EINVAL;
      return VEGAS_OK;
    case VEGAS_EE3J:
      if ((np != 1 && np != 2) || ndim < 5 || !(p[0] > 0.0 && p[0] < 1.0)) return VEGAS_EINVAL;
      if (np == 2 && !(p[1] > 0.0)) return VEGAS_EINVAL;
      return VEGAS_OK;
    case VEGAS_DY_NLO:
      if (np != 11 || check_params(VEGAS_DY, ndim, p, 10) || !(std::fabs(p[10]) <= 50.0))
        return VEGAS_EINVAL;
      return VEGAS_OK;
  }
  return VEGAS_EINVAL;
}

int maxd_class(int d) { return d <= 4 ? 4 : (d <= 8 ? 8 : 16); }

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

constexpr int kHostRecMax = 64;  // iterations whose records fit the mapped result block
constexpr size_t kHostRecOff = 256;  // byte offset of the records in it
static_assert(sizeof(GvState) <= kHostRecOff, "state fits before the records");

// Autotuner cache: best events-per-thread per (integrand, precision, mode,
// d class, nbins, log2 tiles).  Results are identical for every choice.
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;

std::string tune_key(int dev, int ig, int fp32, int mode, int d, int N, int n_tiles) {
  char buf[160];
  int lg = 0;
  while ((1 << (lg + 1)) <= n_tiles && lg < 30) ++lg;
  snprintf(buf, sizeof buf, "dev%d:ig%d:fp%d:m%d:d%d:N%d:t%d", dev, ig, fp32, mode, maxd_class(d),
           N, lg);
  return buf;
}

}  // namespace

struct GraphEntry {
  std::string key;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaEvent_t> events;  // 3 per iteration when timed
};

struct vegas_ctx {
  int ndim = 0, nbins = 0;
  uint64_t seed = 0;
  uint32_t batch = 0;
  double alpha = 1.5;
  int fp32 = 0, adapt = 1, ept_opt = 0, nonfinite_policy = 0, use_graph = 1, timing = 0;
  int pdl = 1;
  int device = 0, sm_count = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // fixed device memory
  void* fixed = nullptr;
  double* grid = nullptr;
  GvState* st = nullptr;
  double* params = nullptr;
  double* kconst = nullptr;
  double* sums = nullptr;
  int* tickets = nullptr;  // reduce tickets (zero between iterations)
  int nacc_max = 0;
  // histogram of the observable (hist_nh = 0: none); hist_valid: the last
  // stage filled it
  int hist_nh = 0;
  double hist_lo = 0.0, hist_hi = 0.0;
  double* hist_acc = nullptr;  // [4][GV_HIST_MAX + 2]
  double* hist_out = nullptr;  // [2][GV_HIST_MAX + 2]
  bool hist_valid = false;
  // VEGAS+ (strat = 1): the allocation persists across stages with the same
  // ncall (plus_C); plus_valid: it exists on the device
  int strat = 0, beta_j = 3;
  void* plus_mem = nullptr;
  long long plus_nh = 0, plus_C = 0;
  int plus_s = 0, plus_tiles = 0;
  bool plus_valid = false;
  long long plus_tab_C = 0;  // the C of the ab table on the device (0: none)
  GvPlusArgs pa;  // device arrays of the allocation (pointers only)
  GvPlusFill* plus_fill = nullptr;  // the stratified fill's data (device)
  // VEGAS+: the hypercube statistics, allocation and layout of an iteration
  // run on this stream beside the reduce (forked after the fill, joined
  // before the next fill)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // autotuning: a copy of the grid pack and the state to return to after
  // trial iterations, and whether trials are running (no results to host)
  void* tune_backup = nullptr;
  bool tuning = false;
  // workspace
  void* ws = nullptr;
  size_t ws_bytes = 0;
  bool ws_external = false;
  // pinned host staging for results
  void* pinned = nullptr;
  size_t pinned_bytes = 0;
  // mapped pinned memory the finalising thread writes a plain forward stage's
  // results into (state, then up to kHostRecMax iteration records), so that
  // fetching them is a synchronisation, not two copies
  void* hres = nullptr;
  void* hres_dev = nullptr;
  bool last_zero_copy = false;
  // derived constants currently on the device
  int consts_ig = -1;
  double consts_params[GV_MAXPARAMS] = {0};
  // last launch
  int last_itmx = 0, last_mode = 0, last_ept = 0;
  double* last_per_iter = nullptr;
  bool pending = false;
  std::vector<cudaEvent_t> pending_events;
  double t_ms[3] = {0, 0, 0};       // fill, reduce, refine
  int64_t n_launch[3] = {0, 0, 0};
  std::vector<GraphEntry> graphs;
};

namespace {

void clear_graphs(vegas_ctx* c) {
  for (auto& g : c->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    for (auto e : g.events) cudaEventDestroy(e);
  }
  c->graphs.clear();
  c->pending_events.clear();
}

size_t grid_doubles(int d, int N) { return GvGridLayout{d, N}.doubles(); }

// events: the fill's capacity (ncall, or ncall + 2 nh with VEGAS+); plus_f:
// room for the per-event J g of VEGAS+
// chained iterations per autotuning trial (iteration records are sized for them)
constexpr int kTuneIter = 8;

size_t workspace_bytes(int d, int N, int64_t ncall, int itmx, int mode, int nhist,
                       bool plus_f = false) {
  const int64_t n_tiles = (ncall + GV_TILE - 1) / GV_TILE;
  const int nch = mode ? GV_MAXCH : 1;
  const int nacc = mode ? 2 * GV_MAXCH : 2 + d * N + 2 * nhist;
  int tpc = 0, gx = 0, gy = 0;
  gv::reduce_grid((int)std::min<int64_t>(n_tiles, 0x7fffffff), nacc, &tpc, &gx, &gy);
  size_t b = align256((size_t)n_tiles * nacc * 16);
  b += align256((size_t)n_tiles * nch * 4);
  b += align256((size_t)std::max(itmx, kTuneIter) * (2 + 2 * GV_NGRAD) * 8);
  b += align256((size_t)gy * gx * 32 * sizeof(GvSlot));
  // VEGAS+: segment sums (16 B) per range and per hypercube (nh <= ncall / 4)
  if (plus_f) b += align256((size_t)(ncall / GV_PLUS_SEG + 1) * 16) + align256((size_t)(ncall / 4 + 1) * 16);
  return b;
}

// VEGAS+ strata per axis: the largest s >= 1 with 4 s^d <= C and
// s^d <= 2^22 (at least four events per hypercube on average).
int plus_nstrat(int d, int64_t C) {
  int64_t s = 1;
  for (;;) {
    const int64_t t = s + 1;
    int64_t p = 1;
    for (int a = 0; a < d; ++a) {
      p *= t;
      if (p > ((int64_t)1 << 22) || 4 * p > C) return (int)s;
    }
    s = t;
  }
}

int64_t ipow(int64_t b, int e) {
  int64_t r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

int ensure_workspace(vegas_ctx* c, size_t need) {
  if (c->ws_bytes >= need && c->ws) return VEGAS_OK;
  if (c->ws_external) return VEGAS_ENOMEM;
  if (c->ws) {
    cudaStreamSynchronize(c->stream);
    cudaFree(c->ws);
    c->ws = nullptr;
    c->ws_bytes = 0;
    clear_graphs(c);
  }
  size_t bytes = std::max(need, (size_t)1 << 20);
  if (cudaMalloc(&c->ws, bytes) != cudaSuccess) {
    cudaGetLastError();
    c->ws = nullptr;
    return VEGAS_ENOMEM;
  }
  c->ws_bytes = bytes;
  return VEGAS_OK;
}

int ensure_pinned(vegas_ctx* c, size_t need) {
  if (c->pinned_bytes >= need) return VEGAS_OK;
  if (c->pinned) cudaFreeHost(c->pinned);
  c->pinned = nullptr;
  c->pinned_bytes = 0;
  if (cudaHostAlloc(&c->pinned, need, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return VEGAS_ENOMEM;
  }
  c->pinned_bytes = need;
  return VEGAS_OK;
}

struct Plan {
  int ig, fp32, mode, itmx, n_tiles, nacc, nch, ept, reduce_ctas, tiles_per_cta;
  int nhist;  // histogram bins with underflow and overflow (0: none)
  int slot_major;  // slot-major partials and the single-level reduce (forward stages)
  int hoist;       // the fill makes its Philox words before it waits (gv_fill_hoistable)
  int plus, s;     // VEGAS+: strata per axis
  long long nh;    // hypercubes
  long long cap;   // events the fill's grid can hold
  double2* seg_h;  // each hypercube's first segment sums (VEGAS+)
  double2* seg_r;  // each range's continuing segment sums (VEGAS+)
  int64_t ncall;
  size_t smem;
  ulonglong2* part;
  int* tileE;
  double* per_iter;
  GvSlot* cpart;
};

GvFillArgs fill_args(const vegas_ctx* c, const Plan& p, int k = 0) {
  GvFillArgs a;
  a.kst = k;
  a.ndim = c->ndim;
  a.nbins = c->nbins;
  a.nch = p.nch;
  a.nacc = p.nacc;
  a.ncall = p.ncall;
  a.seed = c->seed;
  a.batch = c->batch;
  a.kconst = c->kconst;
  a.grid = c->grid;
  a.st = c->st;
  a.part = p.part;
  a.tileE = p.tileE;
  a.slot_major = p.slot_major;
  a.hoist = p.hoist;
  a.n_tiles = p.n_tiles;
  a.nhist = p.nhist;
  if (p.nhist) {
    const double invw = (double)c->hist_nh / (c->hist_hi - c->hist_lo);
    a.h_lo = c->hist_lo;
    a.h_invw = invw;
    a.h_lo_f = (float)c->hist_lo;
    a.h_invw_f = (float)invw;
  }
  if (p.plus) a.plus = c->plus_fill;
  return a;
}

// VEGAS+ kernels' arguments for iteration k of a plan (k < 0: set-up).
GvPlusArgs plus_args(const vegas_ctx* c, const Plan& p, int k) {
  GvPlusArgs a = c->pa;
  a.ncall = p.ncall;
  a.beta_j = c->beta_j;
  a.n_tiles = p.n_tiles;
  a.k = k < 0 ? 0 : k;
  a.last = k == p.itmx - 1;
  a.inv_m1 = k > 0 ? 1.0 / (double)k : 0.0;
  a.seg_h = p.seg_h;
  a.seg_r = p.seg_r;
  a.cap = p.cap;
  a.per_iter = p.per_iter;
  a.st = c->st;
  return a;
}

// Device memory of a VEGAS+ allocation of nh hypercubes and n_tiles tiles
// (zeroed; the allocation itself is made by the caller).
int ensure_plus(vegas_ctx* c, long long nh, int n_tiles) {
  if (c->plus_mem && c->plus_nh == nh && c->plus_tiles >= n_tiles) return VEGAS_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->plus_mem) cudaFree(c->plus_mem);
  c->plus_mem = nullptr;
  c->plus_valid = false;
  clear_graphs(c);
  const long long nb = (nh + 255) / 256;
  size_t off = 0;
  const size_t o_off = off;
  off = align256(off + (size_t)(nh + 1) * 8);
  const size_t o_n = off;
  off = align256(off + (size_t)nh * 4);
  const size_t o_ab = off;
  off = align256(off + (size_t)nh * 16);
  const size_t o_ab32 = off;
  off = align256(off + (size_t)nh * 8);
  const size_t o_t = off;
  off = align256(off + (size_t)n_tiles * 4);
  const size_t o_var = off;
  off = align256(off + (size_t)nh * 8);
  const size_t o_dw = off;
  off = align256(off + (size_t)nh * 8);
  const size_t o_tp = off;  // the fill's per-tile sums, then the finishing kernel's per-CTA sums
  off = align256(off + (size_t)(n_tiles + 16) * 16);
  const size_t o_np = off;
  off = align256(off + (size_t)nb * 8);
  const long long ng = (nb + 31) / 32;
  const size_t o_gs = off;
  off = align256(off + (size_t)ng * 8);
  const size_t o_gc = off;
  off = align256(off + (size_t)ng * 4);
  const size_t o_sc = off;
  off = align256(off + 64);
  const size_t o_pf = off;
  off = align256(off + sizeof(GvPlusFill));
  const size_t o_tab = off;
  off = align256(off + (size_t)GV_PLUS_NTAB * 8 * 3);
  if (cudaMalloc(&c->plus_mem, off) != cudaSuccess) {
    cudaGetLastError();
    c->plus_mem = nullptr;
    return VEGAS_ENOMEM;
  }
  char* b = (char*)c->plus_mem;
  GvPlusArgs& a = c->pa;
  a.nh = nh;
  a.inv_nh2 = 1.0 / ((double)nh * (double)nh);
  a.off = (long long*)(b + o_off);
  a.n = (int*)(b + o_n);
  a.ab = (double2*)(b + o_ab);
  a.ab32 = (float2*)(b + o_ab32);
  a.tile_h0 = (int*)(b + o_t);
  a.var = (double*)(b + o_var);
  a.dw = (double*)(b + o_dw);
  a.tpart = (double2*)(b + o_tp);
  a.fpart = a.tpart + n_tiles;
  a.npart = (long long*)(b + o_np);
  a.gsum = (long long*)(b + o_gs);
  a.gctr = (int*)(b + o_gc);
  // 64 bytes: the event count, three scalars, the fill's used tiles, the
  // finishing kernel's counter
  a.ncall_dev = (long long*)(b + o_sc);
  a.scal = (double*)(b + o_sc + 8);
  a.tiles_used = (int*)(b + o_sc + 32);
  a.fctr = (int*)(b + o_sc + 36);
  c->plus_fill = (GvPlusFill*)(b + o_pf);
  a.inv = (const double*)(b + o_tab);
  a.abtab = (const double2*)(b + o_tab + (size_t)GV_PLUS_NTAB * 8);
  GV_TRY(cudaMemsetAsync(c->plus_mem, 0, off, c->stream));
  std::vector<double> inv(GV_PLUS_NTAB, 0.0);
  for (int n = 1; n < GV_PLUS_NTAB; ++n) inv[n] = 1.0 / (double)n;
  // a pageable copy is staged before cudaMemcpyAsync returns
  GV_TRY(cudaMemcpyAsync((void*)a.inv, inv.data(), inv.size() * 8, cudaMemcpyHostToDevice,
                         c->stream));
  c->plus_nh = nh;
  c->plus_tab_C = 0;
  c->plus_tiles = n_tiles;
  return VEGAS_OK;
}

GvHistArgs hist_args(const vegas_ctx* c, const Plan& p, int k) {
  GvHistArgs h;
  h.sums = c->sums + 2 + (size_t)c->ndim * c->nbins;
  h.per_iter = p.per_iter;
  h.nhist = p.nhist;
  h.k = k;
  h.last = k == p.itmx - 1;
  h.inv_c = 1.0 / (double)p.ncall;
  h.inv_cm1 = 1.0 / (double)(p.ncall - 1);
  h.acc = c->hist_acc;
  h.out = c->hist_out;
  return h;
}

// A plain forward stage of at most kHostRecMax iterations hands its results
// over through the mapped block (VEGAS+ finishes its iterations in another
// kernel, and the adjoint has more channels).
bool zero_copy(const vegas_ctx* c, const Plan& p) {
  return c->hres_dev && !c->tuning && p.mode == 0 && !p.plus && p.itmx <= kHostRecMax;
}

GvReduceArgs reduce_args(const vegas_ctx* c, const Plan& p, int k) {
  GvReduceArgs r;
  r.ndim = c->ndim;
  r.nbins = c->nbins;
  r.nch = p.nch;
  r.nacc = p.nacc;
  r.has_bins = p.mode == 0;
  r.nhist = p.nhist;
  r.plus = p.plus;
  if (zero_copy(c, p)) {
    r.host_st = (GvState*)c->hres_dev;
    r.host_rec = (double*)((char*)c->hres_dev + kHostRecOff);
  }
  if (p.plus) r.tiles_used = c->pa.tiles_used;
  r.k = k;
  r.last = k == p.itmx - 1;
  r.refine_follows = (p.mode == 0 && c->adapt) ? 1 : 0;
  r.mode = p.mode;
  r.ncall = p.ncall;
  r.inv_c = 1.0 / (double)p.ncall;
  r.inv_cm1 = 1.0 / (double)(p.ncall - 1);
  r.inv_m1 = k > 0 ? 1.0 / (double)k : 0.0;
  r.n_tiles = p.n_tiles;
  r.tiles_per_cta = p.tiles_per_cta;
  r.part = p.part;
  r.tileE = p.tileE;
  r.st = c->st;
  r.cpart = p.cpart;
  r.sums = c->sums;
  r.per_iter = p.per_iter;
  r.tickets = c->tickets;
  r.alpha = c->alpha;
  r.inv_nbins = 1.0 / (double)c->nbins;
  r.grid = c->grid;
  return r;
}

// Upload the parameters and re-derive the integrand constants if the
// integrand or a parameter changed since the last derivation.
int ensure_consts(vegas_ctx* c, int ig, const double* params, int np) {
  double hp[GV_MAXPARAMS] = {0};
  for (int i = 0; i < np && i < GV_MAXPARAMS - 1; ++i) hp[i] = params[i];
  hp[GV_MAXPARAMS - 1] = (double)np;
  if (c->consts_ig == ig && memcmp(hp, c->consts_params, sizeof hp) == 0) return VEGAS_OK;
  // a pageable copy is staged before cudaMemcpyAsync returns
  GV_TRY(cudaMemcpyAsync(c->params, hp, sizeof hp, cudaMemcpyHostToDevice, c->stream));
  GV_TRY(gv::launch_consts(ig, c->params, c->kconst, c->stream));
  c->consts_ig = ig;
  memcpy(c->consts_params, hp, sizeof hp);
  return VEGAS_OK;
}

cudaError_t launch_fill_plan(const vegas_ctx* c, const Plan& p, int ept, bool pdl = false,
                             int k = 0) {
  const GvFillArgs a = fill_args(c, p, k);
  if (p.mode) return gv::launch_fill_adjoint(p.fp32, ept, a, p.n_tiles, p.smem, c->stream, pdl);
  if (p.nhist) return gv::launch_fill_hist(p.ig, p.fp32, a, p.n_tiles, p.smem, c->stream, pdl);
  if (p.plus) return gv::launch_fill_plus(p.ig, p.fp32, a, p.n_tiles, p.smem, c->stream, pdl);
  return launch_fill_any(p.ig, p.fp32, ept, a, p.n_tiles, p.smem, c->stream, pdl);
}

// Pick events per thread by timing one fill launch per candidate.  Runs
// between two setup kernels, so the trial launches leave no trace.
int enqueue_body(vegas_ctx* c, const Plan& p, std::vector<cudaEvent_t>* ev, bool capture);

// Events per thread for a plain forward stage, by timing what a stage runs:
// kTuneIter chained iterations (fills and reduces with the refinement, by
// programmatic launch) per candidate, best of kTuneRep, from the same grid
// and state each time (saved before, restored after; no result goes to the
// host).  In a stage, the fills of iterations k > 0 make their Philox words
// while the previous refinement runs, and a shape whose CTAs are all
// resident at once does that for every tile: single fill launches, timed
// alone, miss it.  4 is kept unless another candidate is more than 0.5%
// faster.
constexpr int kTuneRep = 5;
int autotune_chained(vegas_ctx* c, Plan& p, const std::string& key) {
  const size_t gbytes = grid_doubles(c->ndim, c->nbins) * sizeof(double);
  if (!c->tune_backup) {
    if (cudaMalloc(&c->tune_backup, gbytes + sizeof(GvState)) != cudaSuccess) {
      cudaGetLastError();
      c->tune_backup = nullptr;
      return VEGAS_ENOMEM;
    }
  }
  char* bk = (char*)c->tune_backup;
  GV_TRY(cudaMemcpyAsync(bk, c->grid, gbytes, cudaMemcpyDeviceToDevice, c->stream));
  GV_TRY(cudaMemcpyAsync(bk + gbytes, c->st, sizeof(GvState), cudaMemcpyDeviceToDevice, c->stream));
  cudaEvent_t e0, e1;
  GV_TRY(cudaEventCreate(&e0));
  GV_TRY(cudaEventCreate(&e1));
  Plan t = p;
  t.itmx = kTuneIter;
  c->tuning = true;
  int st = VEGAS_OK;
  float best = 1e30f, t4 = 1e30f;
  int best_ept = 4;
  for (const int ept : {1, 2, 4, 8}) {
    if (c->ndim > 8 && ept == 8) continue;
    // a shape the device cannot launch (registers, shared memory) is skipped
    if (launch_fill_plan(c, t, ept) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    t.ept = ept;
    float best_i = 1e30f;
    for (int rep = 0; rep <= kTuneRep && !st; ++rep) {  // rep 0 warms up
      cudaEventRecord(e0, c->stream);
      st = enqueue_body(c, t, nullptr, false);
      cudaEventRecord(e1, c->stream);
      if (!st && cudaEventSynchronize(e1) != cudaSuccess) st = VEGAS_ECUDA;
      float ms = 0;
      if (!st && rep > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) best_i = std::min(best_i, ms);
      cudaMemcpyAsync(c->grid, bk, gbytes, cudaMemcpyDeviceToDevice, c->stream);
      cudaMemcpyAsync(c->st, bk + gbytes, sizeof(GvState), cudaMemcpyDeviceToDevice, c->stream);
    }
    if (st) break;
    if (ept == 4) t4 = best_i;
    if (best_i < best) {
      best = best_i;
      best_ept = ept;
    }
  }
  c->tuning = false;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) {
    cudaStreamSynchronize(c->stream);
    cudaGetLastError();
    return st;
  }
  GV_TRY(cudaGetLastError());
  if (best_ept != 4 && t4 < 1e30f && best > 0.995f * t4) best_ept = 4;
  p.ept = best_ept;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = best_ept;
  return VEGAS_OK;
}

int autotune(vegas_ctx* c, Plan& p) {
  const std::string key = tune_key(c->device, p.ig, p.fp32, p.mode, c->ndim, c->nbins, p.n_tiles);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      p.ept = it->second;
      return VEGAS_OK;
    }
  }
  if (p.mode == 0 && !p.plus && !p.nhist) return autotune_chained(c, p, key);
  const int cands_fwd[] = {1, 2, 4, 8};
  const int cands_adj[] = {1, 2, 4};
  const int* cands = p.mode ? cands_adj : cands_fwd;
  const int nc = p.mode ? 3 : 4;
  cudaEvent_t e0, e1;
  GV_TRY(cudaEventCreate(&e0));
  GV_TRY(cudaEventCreate(&e1));
  // the fastest candidate, but 4 events per thread (the best for every forward
  // fill measured) unless another is more than 2% faster: a few trial launches
  // are noisy enough to flip a 10% difference now and then
  float best = 1e30f, t4 = 1e30f;
  int best_ept = 4;
  for (int i = 0; i < nc; ++i) {
    const int ept = cands[i];
    if (c->ndim > 8 && ept == 8) continue;
    cudaError_t err = launch_fill_plan(c, p, ept);  // warm-up
    if (err != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    float best_i = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, c->stream);
      launch_fill_plan(c, p, ept);
      cudaEventRecord(e1, c->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) break;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      best_i = std::min(best_i, ms);
    }
    if (ept == 4) t4 = best_i;
    if (best_i < best) {
      best = best_i;
      best_ept = ept;
    }
  }
  if (best_ept != 4 && t4 < 1e30f && best > 0.98f * t4) best_ept = 4;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  GV_TRY(cudaGetLastError());
  // the trial launches touched the iteration invariants: restore them
  GV_TRY(gv::launch_reset(c->st, c->stream));
  p.ept = best_ept;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = best_ept;
  return VEGAS_OK;
}

int make_plan(vegas_ctx* c, int64_t ncall, int itmx, int ig, int mode, Plan& p) {
  p.ig = ig;
  p.fp32 = c->fp32;
  p.mode = mode;
  p.itmx = itmx;
  p.ncall = ncall;
  // VEGAS+: strata, and room for up to ncall + 2 nh events (each hypercube's
  // share is floored, then raised to at least 2)
  p.plus = (mode == 0 && c->strat) ? 1 : 0;
  p.s = 0;
  p.nh = 0;
  p.seg_h = nullptr;
  p.seg_r = nullptr;
  int64_t cap = ncall;
  if (p.plus) {
    if (c->hist_nh > 0 || ncall < 8 || ncall > ((int64_t)1 << 30)) return VEGAS_EINVAL;
    p.s = plus_nstrat(c->ndim, ncall);
    p.nh = ipow(p.s, c->ndim);
    cap = ncall + 2 * p.nh;
  }
  p.cap = cap;
  const int64_t nt = (cap + GV_TILE - 1) / GV_TILE;
  if (nt > 0x7fffffff) return VEGAS_EINVAL;
  p.n_tiles = (int)nt;
  p.nch = mode ? GV_MAXCH : 1;
  p.slot_major = mode == 0 ? 1 : 0;
  p.nhist = (mode == 0 && c->hist_nh > 0) ? c->hist_nh + 2 : 0;
  p.nacc = mode ? 2 * GV_MAXCH : 2 + c->ndim * c->nbins + 2 * p.nhist;
  {
    const GvFillSmem plain(c->ndim, c->nbins, c->fp32 ? 4 : 8, mode == 0, c->ndim > 4, p.nhist,
                           p.plus != 0, false);
    const GvFillSmem words(c->ndim, c->nbins, c->fp32 ? 4 : 8, mode == 0, c->ndim > 4, p.nhist,
                           p.plus != 0, true);
    p.hoist = gv_fill_hoistable(mode == 0, p.plus != 0, c->ndim) &&
                      words.total <= GV_WORDS_SMEM_MAX
                  ? 1
                  : 0;
    p.smem = (p.hoist ? words : plain).total;
  }
  int gx = 0, gy = 0;
  gv::reduce_grid(p.n_tiles, p.nacc, &p.tiles_per_cta, &gx, &gy);
  p.reduce_ctas = gx * gy;
  const size_t need = workspace_bytes(c->ndim, c->nbins, cap, itmx, mode, p.nhist, p.plus != 0);
  int st = ensure_workspace(c, need);
  if (st) return st;
  char* w = (char*)c->ws;
  p.part = (ulonglong2*)w;
  w += align256((size_t)p.n_tiles * p.nacc * 16);
  p.tileE = (int*)w;
  w += align256((size_t)p.n_tiles * p.nch * 4);
  p.per_iter = (double*)w;
  w += align256((size_t)std::max(itmx, kTuneIter) * (2 + 2 * GV_NGRAD) * 8);
  p.cpart = (GvSlot*)w;
  if (p.plus) {
    w += align256((size_t)gy * gx * 32 * sizeof(GvSlot));
    p.seg_r = (double2*)w;
    w += align256((size_t)(cap / GV_PLUS_SEG + 1) * 16);
    p.seg_h = (double2*)w;
  }
  p.ept = c->ept_opt;
  return VEGAS_OK;
}

// VEGAS+: the table of (C/(nh n), sqrt(1/(nh n))) for n < GV_PLUS_NTAB, in
// the same FP64 operations as for any other n.
int upload_abtab(vegas_ctx* c, long long C, long long nh) {
  if (c->plus_tab_C == C) return VEGAS_OK;
  std::vector<double> t(2 * (size_t)GV_PLUS_NTAB, 0.0);
  for (int n = 1; n < GV_PLUS_NTAB; ++n) {
    const double nhd = (double)nh * (double)n;
    t[2 * (size_t)n] = (double)C / nhd;
    t[2 * (size_t)n + 1] = std::sqrt(1.0 / nhd);
  }
  // a pageable copy is staged before cudaMemcpyAsync returns
  GV_TRY(cudaMemcpyAsync((void*)c->pa.abtab, t.data(), t.size() * 8, cudaMemcpyHostToDevice,
                         c->stream));
  c->plus_tab_C = C;
  return VEGAS_OK;
}

// VEGAS+: make sure the allocation for ncall exists (uniform if it is new).
int ensure_allocation(vegas_ctx* c, const Plan& p) {
  int st = ensure_plus(c, p.nh, p.n_tiles);
  if (st) return st;
  st = upload_abtab(c, p.ncall, p.nh);
  if (st) return st;
  c->plus_s = p.s;
  // the fill's view of the allocation (the workspace may have moved)
  GvPlusFill f;
  f.s = p.s;
  f.inv_s = 1.0f / (float)p.s;
  f.nh = p.nh;
  f.magic = ~0ull / (unsigned long long)p.s;
  f.off = c->pa.off;
  f.ab = c->pa.ab;
  f.ab32 = c->pa.ab32;
  f.tile_h0 = c->pa.tile_h0;
  f.ncall = c->pa.ncall_dev;
  f.seg_h = p.seg_h;
  f.seg_r = p.seg_r;
  f.tiles_used = c->pa.tiles_used;
  f.var = c->pa.var;
  f.dw = c->pa.dw;
  f.tpart = c->pa.tpart;
  f.inv = c->pa.inv;
  f.beta_j = c->beta_j;
  // a pageable copy is staged before cudaMemcpyAsync returns
  GV_TRY(cudaMemcpyAsync(c->plus_fill, &f, sizeof f, cudaMemcpyHostToDevice, c->stream));
  if (c->plus_valid && c->plus_C == p.ncall) return VEGAS_OK;
  GvPlusArgs a = plus_args(c, p, -1);
  a.uniform = 1;
  GV_TRY(gv::launch_plus_alloc(a, c->stream, false));
  GV_TRY(gv::launch_plus_layout(a, c->stream, false));
  c->plus_valid = true;
  c->plus_C = p.ncall;
  return VEGAS_OK;
}

// The side stream and its fork/join events (made once per context).
int ensure_side(vegas_ctx* c) {
  if (c->side) return VEGAS_OK;
  int least = 0, greatest = 0;
  GV_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
  c->pa.prio = greatest;
  GV_TRY(cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, greatest));
  GV_TRY(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
  GV_TRY(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  return VEGAS_OK;
}

int enqueue_body(vegas_ctx* c, const Plan& p, std::vector<cudaEvent_t>* ev, bool capture) {
  const unsigned flags = capture ? cudaEventRecordExternal : 0u;
  const size_t rsmem = gv::reduce_smem_bytes(c->nbins);
  // programmatic launches chain the kernels of consecutive iterations; the
  // first fill follows ordinary work and timed runs keep plain launches
  const bool pdl = c->pdl && !ev;
  for (int k = 0; k < p.itmx; ++k) {
    if (ev) GV_TRY(cudaEventRecordWithFlags((*ev)[3 * k], c->stream, flags));
    GV_TRY(launch_fill_plan(c, p, p.ept, pdl && k > 0, k));
    if (p.plus) {
      // fork: the statistics' completion needs the fill's results only
      GV_TRY(cudaEventRecord(c->ev_fork, c->stream));
      GV_TRY(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    }
    if (ev) GV_TRY(cudaEventRecordWithFlags((*ev)[3 * k + 1], c->stream, flags));
    // the previous iteration's histogram estimates, beside this fill, have
    // read the bin sums this reduce overwrites
    if (p.nhist && k > 0) GV_TRY(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    // (VEGAS+: a plain launch, so that its CTAs do not hold the SMs while
    // they wait for the fill; the more urgent kernels beside it go first)
    if (p.slot_major)
      GV_TRY(gv::launch_reduce_slots(reduce_args(c, p, k), rsmem, c->stream, pdl && !p.plus));
    else
      GV_TRY(gv::launch_reduce(reduce_args(c, p, k), rsmem, c->stream, pdl));
    if (p.nhist) {
      // the histogram's estimates on the side stream: the next fill reads
      // nothing they touch, so it follows the reduce alone
      GV_TRY(cudaEventRecord(c->ev_fork, c->stream));
      GV_TRY(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
      GV_TRY(gv::launch_hist(hist_args(c, p, k), c->side, false));
      GV_TRY(cudaEventRecord(c->ev_join, c->side));
      if (k == p.itmx - 1) GV_TRY(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    }
    if (p.plus) {
      // beside the reduce: the statistics' completion from the fill's tile
      // sums and crossing hypercubes (sigma_k; the stage's combination with
      // the reduce's I_k), then the next iteration's allocation and its
      // layout; joined after the reduce, before the next fill (which comes in
      // by programmatic launch after the reduce and makes its Philox words
      // while the reduce finishes).
      const GvPlusArgs a = plus_args(c, p, k);
      GV_TRY(gv::launch_plus_finish(a, c->side, false));
      if (c->adapt) {
        GV_TRY(gv::launch_plus_alloc(a, c->side, pdl));
        GV_TRY(gv::launch_plus_layout(a, c->side, pdl));
      }
      GV_TRY(cudaEventRecord(c->ev_join, c->side));
      GV_TRY(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    }
    if (ev) GV_TRY(cudaEventRecordWithFlags((*ev)[3 * k + 2], c->stream, flags));
  }
  return VEGAS_OK;
}

GraphEntry* find_entry(vegas_ctx* c, const std::string& key) {
  for (auto& g : c->graphs)
    if (g.key == key) return &g;
  return nullptr;
}

int new_events(std::vector<cudaEvent_t>& ev, size_t n) {
  ev.resize(n);
  for (auto& e : ev) GV_TRY(cudaEventCreate(&e));
  return VEGAS_OK;
}

void drop_oldest_entry(vegas_ctx* c) {
  cudaStreamSynchronize(c->stream);
  GraphEntry& old = c->graphs.front();
  if (old.exec) cudaGraphExecDestroy(old.exec);
  for (auto e : old.events) cudaEventDestroy(e);
  c->graphs.erase(c->graphs.begin());
}

int enqueue_stage(vegas_ctx* c, int64_t ncall, int itmx, int ig, const double* params, int np,
                  int mode) {
  if (c->pending) {
    // the results of an unfetched launch are superseded (work stays in stream
    // order, so nothing overlaps); its timing events are dropped
    c->pending = false;
    c->pending_events.clear();
  }
  if (ncall < 2 || ncall > ((int64_t)1 << 40) || itmx < 1 || itmx > 100000) return VEGAS_EINVAL;
  int st = check_params(ig, c->ndim, params, np);
  if (st) return st;
  if (mode && (ig != VEGAS_DY || c->strat)) return VEGAS_EINVAL;
  Plan p;
  st = make_plan(c, ncall, itmx, ig, mode, p);
  if (st) return st;
  st = ensure_consts(c, ig, params, np);
  if (st) return st;
  if (p.plus) {
    st = ensure_allocation(c, p);
    if (st) return st;
  }
  if (p.plus || p.nhist) {
    st = ensure_side(c);
    if (st) return st;
  }
  if (p.nhist || p.plus) {
    p.ept = 4;  // the histogram and the stratified fills have one shape
  } else if (p.ept == 0) {
    st = autotune(c, p);
    if (st) return st;
  }
  c->hist_valid = p.nhist > 0;
  c->last_itmx = itmx;
  c->last_mode = mode;
  c->last_ept = p.ept;
  c->last_per_iter = p.per_iter;
  c->last_zero_copy = zero_copy(c, p);
  c->pending_events.clear();
  const bool graph_ok = c->use_graph && c->stream != nullptr;
  if (!graph_ok) {
    std::vector<cudaEvent_t>* evp = nullptr;
    if (c->timing) {
      const std::string key = "plain-events:" + std::to_string(itmx);
      GraphEntry* ge = find_entry(c, key);
      if (!ge) {
        if (c->graphs.size() >= 16) drop_oldest_entry(c);
        GraphEntry g;
        g.key = key;
        st = new_events(g.events, 3 * (size_t)itmx);
        if (st) return st;
        c->graphs.push_back(g);
        ge = &c->graphs.back();
      }
      evp = &ge->events;
    }
    st = enqueue_body(c, p, evp, false);
    if (st) return st;
    if (evp) c->pending_events = *evp;
    c->pending = true;
    return VEGAS_OK;
  }
  char kb[400];
  snprintf(kb, sizeof kb, "graph:%d:%d:%d:%lld:%d:%d:%d:%a:%d%d:%llu:%u:%p:%p:h%d:%a:%a:p%d:%d:%p",
           ig, p.fp32, mode, (long long)ncall, itmx, p.ept, c->adapt, c->alpha, c->timing, c->pdl,
           (unsigned long long)c->seed, c->batch, c->ws, (void*)c->stream, p.nhist, c->hist_lo,
           c->hist_hi, p.plus, c->beta_j, c->plus_mem);
  const std::string key(kb);
  GraphEntry* ge = find_entry(c, key);
  if (!ge) {
    if (c->graphs.size() >= 16) drop_oldest_entry(c);
    GraphEntry g;
    g.key = key;
    if (c->timing) {
      st = new_events(g.events, 3 * (size_t)itmx);
      if (st) return st;
    }
    cudaGraph_t graph;
    GV_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    st = enqueue_body(c, p, c->timing ? &g.events : nullptr, true);
    const cudaError_t ce = cudaStreamEndCapture(c->stream, &graph);
    if (st) {
      if (ce == cudaSuccess) cudaGraphDestroy(graph);
      for (auto e : g.events) cudaEventDestroy(e);
      return st;
    }
    GV_TRY(ce);
    const cudaError_t ie = cudaGraphInstantiate(&g.exec, graph, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(graph);
    GV_TRY(ie);
    c->graphs.push_back(g);
    ge = &c->graphs.back();
  }
  GV_TRY(cudaGraphLaunch(ge->exec, c->stream));
  c->pending_events = ge->events;
  c->pending = true;
  return VEGAS_OK;
}

// Wait for the pending stage; copy the state and the per-iteration records.
int fetch_stage(vegas_ctx* c, GvState* hs, std::vector<double>* per_iter) {
  if (!c->pending) return VEGAS_EINVAL;
  const int stride = c->last_mode ? 2 + 2 * GV_NGRAD : 2;
  const size_t nrec = (size_t)c->last_itmx * stride;
  if (c->last_zero_copy) {
    // the finalising thread wrote the state and the records into the mapped
    // block; they are visible once the stream is done
    GV_TRY(cudaStreamSynchronize(c->stream));
    const volatile GvState* hv = (const volatile GvState*)c->hres;
    memset(hs, 0, sizeof *hs);
    hs->it = hv->it;
    hs->nonfinite = hv->nonfinite;
    hs->status = hv->status;
    hs->integral = hv->integral;
    hs->error = hv->error;
    hs->chi2 = hv->chi2;
    if (per_iter) {
      const volatile double* rv = (const volatile double*)((char*)c->hres + kHostRecOff);
      per_iter->resize(nrec);
      for (size_t i = 0; i < nrec; ++i) (*per_iter)[i] = rv[i];
    }
  } else {
    const size_t need = sizeof(GvState) + nrec * sizeof(double) + 64;
    int st = ensure_pinned(c, need);
    if (st) return st;
    char* pin = (char*)c->pinned;
    GV_TRY(cudaMemcpyAsync(pin, c->st, sizeof(GvState), cudaMemcpyDeviceToHost, c->stream));
    double* pin_rec = (double*)(pin + ((sizeof(GvState) + 63) & ~(size_t)63));
    GV_TRY(cudaMemcpyAsync(pin_rec, c->last_per_iter, nrec * sizeof(double),
                           cudaMemcpyDeviceToHost, c->stream));
    GV_TRY(cudaStreamSynchronize(c->stream));
    memcpy(hs, pin, sizeof(GvState));
    if (per_iter) per_iter->assign(pin_rec, pin_rec + nrec);
  }
  if (!c->pending_events.empty()) {
    for (size_t k = 0; k + 2 < c->pending_events.size(); k += 3) {
      float t[2] = {0.f, 0.f};
      for (int q = 0; q < 2; ++q)
        if (cudaEventElapsedTime(&t[q], c->pending_events[k + q], c->pending_events[k + q + 1]) ==
            cudaSuccess) {
          c->t_ms[q] += t[q];
          c->n_launch[q] += 1;
        }
    }
    cudaGetLastError();
    c->pending_events.clear();
  }
  c->pending = false;
  if (hs->status) return VEGAS_EDEVICE;
  if (hs->nonfinite && c->nonfinite_policy == 0) return VEGAS_ENONFINITE;
  return VEGAS_OK;
}

int valid_grid(const double* e, int d, int N) {
  for (int a = 0; a < d; ++a) {
    const double* r = e + (size_t)a * (N + 1);
    if (r[0] != 0.0 || r[N] != 1.0) return 0;
    for (int i = 0; i < N; ++i)
      if (!(r[i + 1] > r[i])) return 0;
  }
  return 1;
}

int upload_grid(vegas_ctx* c, const double* edges) {
  const size_t n = (size_t)c->ndim * (c->nbins + 1);
  GV_TRY(cudaMemcpyAsync(c->grid, edges, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  GV_TRY(gv::launch_grid_pack(c->ndim, c->nbins, c->grid, c->stream));
  GV_TRY(cudaStreamSynchronize(c->stream));
  return VEGAS_OK;
}

struct StateBlob {
  uint32_t magic, version;
  int32_t ndim, nbins;
  uint64_t seed, it;
  uint32_t batch;
  int32_t fp32, adapt, nonfinite_policy;
  double alpha;
};
const uint32_t kStateMagic = 0x47564547u;  // "GVEG"

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

const char* vegas_strerror(int status) {
  switch (status) {
    case VEGAS_OK: return "ok";
    case VEGAS_EINVAL: return "invalid argument";
    case VEGAS_ENOMEM: return "out of memory";
    case VEGAS_ECUDA: return "CUDA runtime error";
    case VEGAS_EGRID: return "invalid grid (edges must be 0 = e_0 < ... < e_N = 1)";
    case VEGAS_ENONFINITE: return "non-finite weights were seen (counted as 0)";
    case VEGAS_EDEVICE: return "device-side check failed";
    case VEGAS_ESTATE: return "checkpoint does not match this context";
  }
  return "unknown status";
}

int vegas_init(int ndim, int nbins, uint64_t seed, vegas_ctx** out) {
  if (!out) return VEGAS_EINVAL;
  *out = nullptr;
  if (ndim < 1 || ndim > VEGAS_MAX_DIM || nbins < VEGAS_MIN_BINS || nbins > VEGAS_MAX_BINS ||
      ndim * nbins > VEGAS_MAX_DIM_BINS)
    return VEGAS_EINVAL;
  vegas_ctx* c = new vegas_ctx();
  c->ndim = ndim;
  c->nbins = nbins;
  c->seed = seed;
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device) !=
          cudaSuccess ||
      cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
    gv_last_cuda_error() = cudaGetLastError();
    delete c;
    return VEGAS_ECUDA;
  }
  c->own_stream = true;
  // the mapped result block (without it, results are copied)
  if (cudaHostAlloc(&c->hres, kHostRecOff + kHostRecMax * 2 * sizeof(double),
                    cudaHostAllocMapped) == cudaSuccess) {
    if (cudaHostGetDevicePointer(&c->hres_dev, c->hres, 0) != cudaSuccess) {
      cudaGetLastError();
      cudaFreeHost(c->hres);
      c->hres = nullptr;
      c->hres_dev = nullptr;
    }
  } else {
    cudaGetLastError();
    c->hres = nullptr;
  }
  // slots: channel sums, bin sums, the largest histogram's sums
  c->nacc_max = std::max(2 * GV_MAXCH, 2 + ndim * nbins + 2 * (GV_HIST_MAX + 2));
  const size_t gd = grid_doubles(ndim, nbins);
  size_t off = 0;
  const size_t o_grid = off;
  off = align256(off + gd * 8);
  const size_t o_st = off;
  off = align256(off + sizeof(GvState));
  const size_t o_par = off;
  off = align256(off + GV_MAXPARAMS * 8);
  const size_t o_k = off;
  off = align256(off + GV_NCONST * 8);
  const size_t o_sums = off;
  off = align256(off + (size_t)c->nacc_max * 8);
  const size_t o_tick = off;
  off = align256(off + gv_tickets_ints(c->nacc_max) * 4);
  const size_t o_hist = off;
  off = align256(off + (size_t)6 * (GV_HIST_MAX + 2) * 8);
  if (cudaMalloc(&c->fixed, off) != cudaSuccess) {
    cudaGetLastError();
    cudaStreamDestroy(c->stream);
    delete c;
    return VEGAS_ENOMEM;
  }
  char* b = (char*)c->fixed;
  c->grid = (double*)(b + o_grid);
  c->st = (GvState*)(b + o_st);
  c->params = (double*)(b + o_par);
  c->kconst = (double*)(b + o_k);
  c->sums = (double*)(b + o_sums);
  c->tickets = (int*)(b + o_tick);
  c->hist_acc = (double*)(b + o_hist);
  c->hist_out = c->hist_acc + 4 * (GV_HIST_MAX + 2);
  int st = VEGAS_OK;
  if (cudaMemsetAsync(c->fixed, 0, off, c->stream) != cudaSuccess ||
      gv::launch_reset(c->st, c->stream) != cudaSuccess)
    st = VEGAS_ECUDA;
  if (!st) {
    std::vector<double> e((size_t)ndim * (nbins + 1));
    for (int a = 0; a < ndim; ++a)
      for (int i = 0; i <= nbins; ++i) e[(size_t)a * (nbins + 1) + i] = (double)i / nbins;
    st = upload_grid(c, e.data());
  }
  if (st) {
    vegas_free(c);
    return st;
  }
  *out = c;
  return VEGAS_OK;
}

void vegas_free(vegas_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  clear_graphs(c);
  if (c->ws && !c->ws_external) cudaFree(c->ws);
  if (c->fixed) cudaFree(c->fixed);
  if (c->plus_mem) cudaFree(c->plus_mem);
  if (c->pinned) cudaFreeHost(c->pinned);
  if (c->hres) cudaFreeHost(c->hres);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->tune_backup) cudaFree(c->tune_backup);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  delete c;
}

int vegas_set_option(vegas_ctx* c, int key, double v) {
  if (!c || !std::isfinite(v)) return VEGAS_EINVAL;
  switch (key) {
    case VEGAS_OPT_ALPHA:
      if (v < 0.0) return VEGAS_EINVAL;
      c->alpha = v;
      return VEGAS_OK;
    case VEGAS_OPT_PRECISION:
      if (v != 0.0 && v != 1.0) return VEGAS_EINVAL;
      c->fp32 = (int)v;
      return VEGAS_OK;
    case VEGAS_OPT_ADAPT:
      if (v != 0.0 && v != 1.0) return VEGAS_EINVAL;
      c->adapt = (int)v;
      return VEGAS_OK;
    case VEGAS_OPT_EPT:
      if (v != 0.0 && v != 1.0 && v != 2.0 && v != 4.0 && v != 8.0) return VEGAS_EINVAL;
      if (v == 8.0 && c->ndim > 8) return VEGAS_EINVAL;
      c->ept_opt = (int)v;
      return VEGAS_OK;
    case VEGAS_OPT_NONFINITE:
      if (v != 0.0 && v != 1.0) return VEGAS_EINVAL;
      c->nonfinite_policy = (int)v;
      return VEGAS_OK;
    case VEGAS_OPT_GRAPH:
      if (v != 0.0 && v != 1.0) return VEGAS_EINVAL;
      c->use_graph = (int)v;
      return VEGAS_OK;
    case VEGAS_OPT_TIMING:
      if (v != 0.0 && v != 1.0) return VEGAS_EINVAL;
      c->timing = (int)v;
      return VEGAS_OK;
    case VEGAS_OPT_PDL:
      if (v != 0.0 && v != 1.0) return VEGAS_EINVAL;
      c->pdl = (int)v;
      clear_graphs(c);
      return VEGAS_OK;
    case VEGAS_OPT_STRAT:
      if (v != 0.0 && v != 1.0) return VEGAS_EINVAL;
      if (c->stream) cudaStreamSynchronize(c->stream);
      c->strat = (int)v;
      clear_graphs(c);
      return VEGAS_OK;
    case VEGAS_OPT_BETA: {
      const double j = 4.0 * v;
      if (!(j >= 0.0 && j <= 4.0) || j != std::floor(j)) return VEGAS_EINVAL;
      if (c->stream) cudaStreamSynchronize(c->stream);
      c->beta_j = (int)j;
      clear_graphs(c);
      return VEGAS_OK;
    }
    case VEGAS_OPT_BATCH_ID:
      if (v < 0.0 || v >= 16777216.0 || v != std::floor(v)) return VEGAS_EINVAL;
      c->batch = (uint32_t)v;
      return VEGAS_OK;
  }
  return VEGAS_EINVAL;
}

int vegas_set_stream(vegas_ctx* c, void* stream) {
  if (!c) return VEGAS_EINVAL;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  c->own_stream = false;
  c->stream = (cudaStream_t)stream;
  clear_graphs(c);
  return VEGAS_OK;
}

int vegas_workspace_size(const vegas_ctx* c, int64_t ncall, int itmx, size_t* bytes) {
  if (!c || !bytes || ncall < 2 || itmx < 1) return VEGAS_EINVAL;
  const int nhist = c->hist_nh > 0 ? c->hist_nh + 2 : 0;
  *bytes = std::max(workspace_bytes(c->ndim, c->nbins, ncall, itmx, 0, nhist),
                    workspace_bytes(c->ndim, c->nbins, ncall, itmx, 1, 0));
  return VEGAS_OK;
}

int vegas_strat_get(vegas_ctx* c, int* nstrat, int64_t* ncubes, int32_t* counts, double* var) {
  if (!c || !c->plus_valid) return VEGAS_EINVAL;
  GV_TRY(cudaStreamSynchronize(c->stream));
  if (nstrat) *nstrat = c->plus_s;
  if (ncubes) *ncubes = c->plus_nh;
  if (counts)
    GV_TRY(cudaMemcpy(counts, c->pa.n, (size_t)c->plus_nh * 4, cudaMemcpyDeviceToHost));
  if (var) GV_TRY(cudaMemcpy(var, c->pa.var, (size_t)c->plus_nh * 8, cudaMemcpyDeviceToHost));
  return VEGAS_OK;
}

int vegas_strat_set(vegas_ctx* c, int64_t ncall, const int32_t* counts) {
  if (!c || !counts || ncall < 8 || ncall > ((int64_t)1 << 30)) return VEGAS_EINVAL;
  const int s = plus_nstrat(c->ndim, ncall);
  const int64_t nh = ipow(s, c->ndim);
  int64_t total = 0;
  for (int64_t h = 0; h < nh; ++h) {
    if (counts[h] < 2) return VEGAS_EINVAL;
    total += counts[h];
  }
  if (total > ncall + 2 * nh) return VEGAS_EINVAL;
  const int n_tiles = (int)((ncall + 2 * nh + GV_TILE - 1) / GV_TILE);
  int st = ensure_plus(c, nh, n_tiles);
  if (st) return st;
  st = upload_abtab(c, ncall, nh);
  if (st) return st;
  // the counts, their sums per CTA of 256 hypercubes and per group of 32
  // CTAs, and the total; then the layout
  const int64_t nb = (nh + 255) / 256, ng = (nb + 31) / 32;
  std::vector<long long> agg((size_t)nb, 0), gsum((size_t)ng, 0);
  long long run = 0;
  for (int64_t b = 0; b < nb; ++b) {
    for (int64_t h = b * 256; h < std::min(nh, (b + 1) * 256); ++h) agg[(size_t)b] += counts[h];
    gsum[(size_t)(b / 32)] += agg[(size_t)b];
    run += agg[(size_t)b];
  }
  GV_TRY(cudaMemcpyAsync(c->pa.n, counts, (size_t)nh * 4, cudaMemcpyHostToDevice, c->stream));
  GV_TRY(cudaMemcpyAsync(c->pa.npart, agg.data(), (size_t)nb * 8, cudaMemcpyHostToDevice,
                         c->stream));
  GV_TRY(cudaMemcpyAsync(c->pa.gsum, gsum.data(), (size_t)ng * 8, cudaMemcpyHostToDevice,
                         c->stream));
  GV_TRY(cudaMemcpyAsync(c->pa.ncall_dev, &run, 8, cudaMemcpyHostToDevice, c->stream));
  GvPlusArgs a = c->pa;
  a.ncall = ncall;
  a.n_tiles = n_tiles;
  GV_TRY(gv::launch_plus_layout(a, c->stream, false));
  GV_TRY(cudaStreamSynchronize(c->stream));  // the host vectors go out of scope
  c->plus_s = s;
  c->plus_C = ncall;
  c->plus_valid = true;
  return VEGAS_OK;
}

int vegas_hist_set(vegas_ctx* c, int nbins, double lo, double hi) {
  if (!c || nbins < 0 || nbins > VEGAS_HIST_MAX_BINS) return VEGAS_EINVAL;
  if (nbins > 0 && !(std::isfinite(lo) && std::isfinite(hi) && hi > lo &&
                     std::isfinite((double)nbins / (hi - lo))))
    return VEGAS_EINVAL;
  if (c->stream) cudaStreamSynchronize(c->stream);
  clear_graphs(c);
  c->hist_nh = nbins;
  c->hist_lo = nbins > 0 ? lo : 0.0;
  c->hist_hi = nbins > 0 ? hi : 0.0;
  c->hist_valid = false;
  return VEGAS_OK;
}

int vegas_hist_get(vegas_ctx* c, double* value, double* error, double* last_sums) {
  if (!c || c->hist_nh <= 0 || !c->hist_valid) return VEGAS_EINVAL;
  const size_t hb = (size_t)c->hist_nh + 2;
  GV_TRY(cudaStreamSynchronize(c->stream));
  if (value) GV_TRY(cudaMemcpy(value, c->hist_out, hb * sizeof(double), cudaMemcpyDeviceToHost));
  if (error)
    GV_TRY(cudaMemcpy(error, c->hist_out + hb, hb * sizeof(double), cudaMemcpyDeviceToHost));
  if (last_sums) {
    // device order: sum w^2 per bin, then sum w; returned as sum w, then sum w^2
    const double* d = c->sums + 2 + (size_t)c->ndim * c->nbins;
    GV_TRY(cudaMemcpy(last_sums, d + hb, hb * sizeof(double), cudaMemcpyDeviceToHost));
    GV_TRY(cudaMemcpy(last_sums + hb, d, hb * sizeof(double), cudaMemcpyDeviceToHost));
  }
  return VEGAS_OK;
}

int vegas_set_workspace(vegas_ctx* c, void* ptr, size_t bytes) {
  if (!c) return VEGAS_EINVAL;
  if (ptr && ((uintptr_t)ptr % 256 != 0)) return VEGAS_EINVAL;
  if (c->stream) cudaStreamSynchronize(c->stream);
  clear_graphs(c);
  if (c->ws && !c->ws_external) cudaFree(c->ws);
  c->ws = ptr;
  c->ws_bytes = ptr ? bytes : 0;
  c->ws_external = ptr != nullptr;
  return VEGAS_OK;
}

int vegas_launch(vegas_ctx* c, int64_t ncall, int itmx, int id, const double* params, int np) {
  if (!c) return VEGAS_EINVAL;
  return enqueue_stage(c, ncall, itmx, id, params, np, 0);
}

int vegas_fetch(vegas_ctx* c, double* integral, double* error, double* chi2, double* per_iter,
                int64_t* nonfinite) {
  if (!c || c->last_mode != 0) return VEGAS_EINVAL;
  GvState hs;
  std::vector<double> rec;
  const int st = fetch_stage(c, &hs, per_iter ? &rec : nullptr);
  if (st && st != VEGAS_ENONFINITE) return st;
  if (integral) *integral = hs.integral;
  if (error) *error = hs.error;
  if (chi2) *chi2 = hs.chi2;
  if (nonfinite) *nonfinite = (int64_t)hs.nonfinite;
  if (per_iter) memcpy(per_iter, rec.data(), rec.size() * sizeof(double));
  return st;
}

int vegas_iterate(vegas_ctx* c, int64_t ncall, int itmx, int id, const double* params, int np,
                  double* integral, double* error, double* chi2, double* per_iter) {
  if (!c) return VEGAS_EINVAL;
  int st = enqueue_stage(c, ncall, itmx, id, params, np, 0);
  if (st) return st;
  return vegas_fetch(c, integral, error, chi2, per_iter, nullptr);
}

int vegas_adjoint(vegas_ctx* c, int64_t ncall, int itmx, int id, const double* params, int np,
                  double* grad, double* grad_err, double* integral, double* error,
                  double* per_iter_grad) {
  if (!c || !grad || !grad_err) return VEGAS_EINVAL;
  int st = enqueue_stage(c, ncall, itmx, id, params, np, 1);
  if (st) return st;
  GvState hs;
  std::vector<double> rec;
  st = fetch_stage(c, &hs, per_iter_grad ? &rec : nullptr);
  if (st && st != VEGAS_ENONFINITE) return st;
  for (int q = 0; q < GV_NGRAD; ++q) {
    grad[q] = hs.grad[q];
    grad_err[q] = hs.grad_err[q];
  }
  if (integral) *integral = hs.integral;
  if (error) *error = hs.error;
  if (per_iter_grad) {
    const int stride = 2 + 2 * GV_NGRAD;
    for (int k = 0; k < itmx; ++k)
      for (int q = 0; q < GV_NGRAD; ++q) {
        per_iter_grad[(k * GV_NGRAD + q) * 2] = rec[(size_t)k * stride + 2 + 2 * q];
        per_iter_grad[(k * GV_NGRAD + q) * 2 + 1] = rec[(size_t)k * stride + 3 + 2 * q];
      }
  }
  return st;
}

int vegas_grid_get(const vegas_ctx* c, double* edges) {
  if (!c || !edges) return VEGAS_EINVAL;
  const size_t n = (size_t)c->ndim * (c->nbins + 1);
  GV_TRY(cudaStreamSynchronize(c->stream));
  GV_TRY(cudaMemcpy(edges, c->grid, n * sizeof(double), cudaMemcpyDeviceToHost));
  return VEGAS_OK;
}

int vegas_grid_set(vegas_ctx* c, const double* edges) {
  if (!c || !edges) return VEGAS_EINVAL;
  if (!valid_grid(edges, c->ndim, c->nbins)) return VEGAS_EGRID;
  GV_TRY(cudaStreamSynchronize(c->stream));
  return upload_grid(c, edges);
}

int vegas_state_size(const vegas_ctx* c, size_t* bytes) {
  if (!c || !bytes) return VEGAS_EINVAL;
  *bytes = sizeof(StateBlob) + (size_t)c->ndim * (c->nbins + 1) * sizeof(double);
  return VEGAS_OK;
}

int vegas_state_get(const vegas_ctx* c, void* buf, size_t bytes) {
  size_t need = 0;
  if (!c || !buf || vegas_state_size(c, &need) || bytes < need) return VEGAS_EINVAL;
  StateBlob h;
  memset(&h, 0, sizeof h);
  h.magic = kStateMagic;
  h.version = 1;
  h.ndim = c->ndim;
  h.nbins = c->nbins;
  h.seed = c->seed;
  GvState hs;
  GV_TRY(cudaStreamSynchronize(c->stream));
  GV_TRY(cudaMemcpy(&hs, c->st, sizeof hs, cudaMemcpyDeviceToHost));
  h.it = hs.it;
  h.batch = c->batch;
  h.fp32 = c->fp32;
  h.adapt = c->adapt;
  h.nonfinite_policy = c->nonfinite_policy;
  h.alpha = c->alpha;
  memcpy(buf, &h, sizeof h);
  return vegas_grid_get(c, (double*)((char*)buf + sizeof h));
}

int vegas_state_set(vegas_ctx* c, const void* buf, size_t bytes) {
  size_t need = 0;
  if (!c || !buf || vegas_state_size(c, &need)) return VEGAS_EINVAL;
  if (bytes < need) return VEGAS_ESTATE;
  StateBlob h;
  memcpy(&h, buf, sizeof h);
  if (h.magic != kStateMagic || h.version != 1 || h.ndim != c->ndim || h.nbins != c->nbins)
    return VEGAS_ESTATE;
  std::vector<double> e((size_t)c->ndim * (c->nbins + 1));
  memcpy(e.data(), (const char*)buf + sizeof h, e.size() * sizeof(double));
  if (!valid_grid(e.data(), c->ndim, c->nbins)) return VEGAS_EGRID;
  GV_TRY(cudaStreamSynchronize(c->stream));
  c->seed = h.seed;
  c->batch = h.batch;
  c->fp32 = h.fp32;
  c->adapt = h.adapt;
  c->nonfinite_policy = h.nonfinite_policy;
  c->alpha = h.alpha;
  GvState hs;
  GV_TRY(cudaMemcpy(&hs, c->st, sizeof hs, cudaMemcpyDeviceToHost));
  hs.it = h.it;
  hs.it0 = h.it;
  GV_TRY(cudaMemcpy(c->st, &hs, sizeof hs, cudaMemcpyHostToDevice));
  clear_graphs(c);
  c->plus_valid = false;  // a VEGAS+ allocation is not part of a checkpoint
  return upload_grid(c, e.data());
}

int vegas_eval_events(vegas_ctx* c, int id, const double* params, int np, uint32_t iteration,
                      const int64_t* events, int64_t n, double* w, int32_t* bins) {
  if (!c || n < 0 || (n > 0 && (!events || !w || !bins))) return VEGAS_EINVAL;
  int st = check_params(id, c->ndim, params, np);
  if (st) return st;
  if (n == 0) return VEGAS_OK;
  GV_TRY(cudaStreamSynchronize(c->stream));
  void* dmem = nullptr;
  const size_t bytes = (size_t)n * (8 + 8 + 4 * c->ndim) + 64;
  if (cudaMalloc(&dmem, bytes) != cudaSuccess) {
    cudaGetLastError();
    return VEGAS_ENOMEM;
  }
  long long* dev = (long long*)dmem;
  double* dw = (double*)(dev + n);
  int* db = (int*)(dw + n);
  st = ensure_consts(c, id, params, np);
  if (st) {
    cudaFree(dmem);
    return st;
  }
  cudaError_t e = cudaMemcpyAsync(dev, events, (size_t)n * 8, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) {
    GvFillArgs a;
    memset(&a, 0, sizeof a);
    a.ndim = c->ndim;
    a.nbins = c->nbins;
    a.seed = c->seed;
    a.batch = c->batch;
    a.kconst = c->kconst;
    a.grid = c->grid;
    a.st = c->st;
    switch (id) {
      case GV_GAUSS: e = gv::launch_fill_gauss_eval(c->fp32, a, iteration, dev, n, dw, db, c->stream); break;
      case GV_DY: e = gv::launch_fill_dy_eval(c->fp32, a, iteration, dev, n, dw, db, c->stream); break;
      case GV_EE3J: e = gv::launch_fill_ee3j_eval(c->fp32, a, iteration, dev, n, dw, db, c->stream); break;
      default: e = gv::launch_fill_dynlo_eval(c->fp32, a, iteration, dev, n, dw, db, c->stream); break;
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(w, dw, (size_t)n * 8, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(bins, db, (size_t)n * 4 * c->ndim, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(dmem);
  if (e != cudaSuccess) {
    gv_last_cuda_error() = e;
    return VEGAS_ECUDA;
  }
  return VEGAS_OK;
}

int vegas_rng_words(uint64_t seed, uint32_t iteration, uint32_t batch, int64_t first, int64_t n,
                    int ndim, uint32_t* out) {
  if (n < 0 || first < 0 || ndim < 1 || ndim > VEGAS_MAX_DIM || (n > 0 && !out))
    return VEGAS_EINVAL;
  if (n == 0) return VEGAS_OK;
  uint32_t* d = nullptr;
  const size_t bytes = (size_t)n * ndim * 4;
  if (cudaMalloc(&d, bytes) != cudaSuccess) {
    cudaGetLastError();
    return VEGAS_ENOMEM;
  }
  cudaError_t e = gv::launch_rng_words(seed, iteration, batch, (unsigned long long)first, n, ndim,
                                       d, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(out, d, bytes, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) {
    gv_last_cuda_error() = e;
    return VEGAS_ECUDA;
  }
  return VEGAS_OK;
}

int vegas_last_sums(const vegas_ctx* c, double* sums) {
  if (!c || !sums) return VEGAS_EINVAL;
  GV_TRY(cudaStreamSynchronize(c->stream));
  GV_TRY(cudaMemcpy(sums, c->sums, (size_t)(2 + c->ndim * c->nbins) * sizeof(double),
                    cudaMemcpyDeviceToHost));
  return VEGAS_OK;
}

int vegas_kernel_time(vegas_ctx* c, int kernel, double* total_ms, int64_t* launches, int reset) {
  if (!c || kernel < VEGAS_KERNEL_FILL || kernel > VEGAS_KERNEL_REFINE) return VEGAS_EINVAL;
  if (total_ms) *total_ms = c->t_ms[kernel];
  if (launches) *launches = c->n_launch[kernel];
  if (reset) {
    c->t_ms[kernel] = 0.0;
    c->n_launch[kernel] = 0;
  }
  return VEGAS_OK;
}

int vegas_get_ept(const vegas_ctx* c, int* ept) {
  if (!c || !ept) return VEGAS_EINVAL;
  *ept = c->last_ept;
  return VEGAS_OK;
}

}  // extern "C"
