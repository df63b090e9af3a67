// gv_batch.cu -- many independent VEGAS integrations per launch.
//
// The paper contrasts one run whose events all feed one grid with many
// independent runs (Section 2.1); here many *different* integrations (uneven
// dimension, call count and integrand) share the GPU.  Each iteration is
//   one persistent fill launch per dimension class (at most 4, 8, 16 axes)
//   over a work list of (integration, tile) items,
//   one reduce launch whose CTAs serve all integrations (task table) and
//   refine each integration's axes as they complete,
// and the itmx iterations are captured in one CUDA graph.  The work list
// orders the integrations by decreasing expected cost (largest first) and
// CTAs take items from an integer counter; since every tile is summed
// exactly, the schedule cannot change any result.  Integration b uses Philox
// batch word b, so its results are bit-identical to those of a single
// context with VEGAS_OPT_BATCH_ID = b.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/vegas.h"
#include "gv_fill_batch.cuh"

namespace {

#define GB_TRY(expr)                 \
  do {                               \
    if ((expr) != cudaSuccess) {     \
      cudaGetLastError();            \
      return VEGAS_ECUDA;            \
    }                                \
  } while (0)

size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

int batch_check_params(int ig, int ndim, const double* p, int np) {
  for (int i = 0; i < np; ++i)
    if (!std::isfinite(p[i])) return VEGAS_EINVAL;
  switch (ig) {
    case VEGAS_GAUSS: return (np == 1 && ndim >= 1 && p[0] > 0.0) ? VEGAS_OK : VEGAS_EINVAL;
    case VEGAS_DY:
      return (np == 10 && ndim >= 4 && p[0] > 0 && p[1] > 0 && p[2] > 0 && p[3] > 0 && p[3] < 1 &&
              p[4] > 0 && p[5] > 0 && p[6] > p[5] && p[6] < p[0] && p[9] > 0)
                 ? VEGAS_OK
                 : VEGAS_EINVAL;
    case VEGAS_EE3J:
      return ((np == 1 || np == 2) && ndim >= 5 && p[0] > 0.0 && p[0] < 1.0 &&
              (np == 1 || p[1] > 0.0))
                 ? VEGAS_OK
                 : VEGAS_EINVAL;
  }
  return VEGAS_EINVAL;
}

// Rough relative cost of one tile, for the largest-first order only.
double tile_cost(int ig, int d) {
  switch (ig) {
    case VEGAS_GAUSS: return 1.0 + 0.25 * d;
    case VEGAS_DY: return 3.0 + 0.25 * d;
    default: return 2.5 + 0.25 * d;
  }
}

struct Member {
  int ig, d, np, n_tiles, nacc, gx, gy;
  int64_t ncall;
  double params[GV_MAXPARAMS];
  double* grid;
  GvState* st;
  double* par;
  double* kconst;
  GvSlot* cpart;
  double* sums;
  ulonglong2* part;
  int* tileE;
  int* tickets;
};

}  // namespace

struct vegas_batch {
  int n = 0, N = 0;
  uint64_t seed = 0;
  int fp32 = 1, adapt = 1, ept_opt = 0, nonfinite_policy = 0, use_graph = 1;
  int grid_opt = 0;  // eighths of the resident CTAs per list (0: tuned)
  double alpha = 1.5;
  int device = 0, sm_count = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<Member> m;
  void* dmem = nullptr;
  // per-iteration records [n][cap][2]
  double* per_iter = nullptr;
  int per_iter_cap = 0;
  // launch tables
  GvFillArgs* d_fill = nullptr;
  GvReduceArgs* d_red = nullptr;
  int4* d_red_tasks = nullptr;
  int n_red_tasks = 0;
  // one work list per dimension class (members of at most 4, 8, 16 axes) and
  // integrand
  struct FillClass {
    int maxd = 0, ig = 0, n = 0, ctas = 0;
    long long total = 0;
    size_t smem = 0;
    int* d_order = nullptr;
    long long* d_start = nullptr;
    unsigned long long* d_counter = nullptr;
  };
  std::vector<FillClass> cls;
  // the lists' fill launches of one iteration run side by side: list
  // launch_order[0] on the main stream, the others on side streams forked from
  // it and joined before the reduce, so that a list's CTAs take the SMs the
  // previous lists' last CTAs leave idle
  std::vector<int> launch_order;  // largest estimated cost first
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  size_t reduce_smem = 0;
  int ept = 0;
  int cta_eighths = 8;  // each list's persistent grid: this many eighths of its resident CTAs
  // graph cache
  std::string graph_key;
  cudaGraphExec_t graph = nullptr;
  // pinned results
  void* pinned = nullptr;
  size_t pinned_bytes = 0;
};

namespace {

// Dimension class of a member (the same classes as the single-context fill).
int dim_class(int ig, int d) { return (d <= 4 && ig != VEGAS_EE3J) ? 4 : d <= 8 ? 8 : 16; }

// The list's fill launch (its counter reset first) and its occupancy.
cudaError_t fill_class(vegas_batch* B, const vegas_batch::FillClass& c, int ept, int ctas,
                       cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(c.d_counter, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  auto f = c.maxd == 4 ? (B->fp32 ? gv::fill_batch_f4 : gv::fill_batch_d4)
           : c.maxd == 8 ? (B->fp32 ? gv::fill_batch_f8 : gv::fill_batch_d8)
                         : (B->fp32 ? gv::fill_batch_f16 : gv::fill_batch_d16);
  return f(c.ig, ept, ctas, c.smem, s, B->d_fill, c.d_order, c.d_start, c.n, c.total,
           c.d_counter);
}

int class_occupancy(vegas_batch* B, const vegas_batch::FillClass& c, int ept) {
  auto f = c.maxd == 4 ? (B->fp32 ? gv::fill_batch_occ_f4 : gv::fill_batch_occ_d4)
           : c.maxd == 8 ? (B->fp32 ? gv::fill_batch_occ_f8 : gv::fill_batch_occ_d8)
                         : (B->fp32 ? gv::fill_batch_occ_f16 : gv::fill_batch_occ_d16);
  return std::max(1, f(c.ig, ept, c.smem));
}

// A list's persistent grid: eighths/8 of its resident CTAs on every SM.
int class_ctas(vegas_batch* B, const vegas_batch::FillClass& c, int ept, int eighths) {
  return std::max(1, class_occupancy(B, c, ept) * B->sm_count * eighths / 8);
}

// All lists' fill launches of one iteration, side by side (as in a stage):
// list launch_order[0] on the main stream, the others on side streams forked
// from it and joined back.
cudaError_t fill_lists(vegas_batch* B, int ept, const std::vector<int>& ctas) {
  const int nl = (int)B->launch_order.size();
  cudaError_t e = cudaSuccess;
  if (nl > 1) e = cudaEventRecord(B->fork, B->stream);
  for (int i = 0; i < nl && e == cudaSuccess; ++i) {
    const int li = B->launch_order[i];
    const auto& c = B->cls[li];
    if (i == 0) {
      e = fill_class(B, c, ept, ctas[li], B->stream);
    } else {
      cudaStream_t s = B->side[i - 1];
      e = cudaStreamWaitEvent(s, B->fork, 0);
      if (e == cudaSuccess) e = fill_class(B, c, ept, ctas[li], s);
      if (e == cudaSuccess) e = cudaEventRecord(B->join[i - 1], s);
    }
  }
  for (int i = 1; i < nl && e == cudaSuccess; ++i)
    e = cudaStreamWaitEvent(B->stream, B->join[i - 1], 0);
  return e;
}

int reset_all(vegas_batch* B) {
  for (const Member& x : B->m)
    GB_TRY(gv::launch_reset(x.st, B->stream));
  return VEGAS_OK;
}

// (Re)build the device argument tables; per_iter must be allocated.
int upload_tables(vegas_batch* B) {
  const int n = B->n;
  std::vector<GvFillArgs> fa(n);
  std::vector<GvReduceArgs> ra(n);
  std::vector<int4> rt;
  for (int b = 0; b < n; ++b) {
    const Member& x = B->m[b];
    GvFillArgs& a = fa[b];
    memset(&a, 0, sizeof a);
    a.ndim = x.d;
    a.nbins = B->N;
    a.nch = 1;
    a.nacc = x.nacc;
    a.ncall = x.ncall;
    a.seed = B->seed;
    a.batch = (unsigned)b;
    a.kconst = x.kconst;
    a.grid = x.grid;
    a.st = x.st;
    a.part = x.part;
    a.tileE = x.tileE;
    GvReduceArgs& r = ra[b];
    memset(&r, 0, sizeof r);
    r.ndim = x.d;
    r.nbins = B->N;
    r.nch = 1;
    r.nacc = x.nacc;
    r.has_bins = 1;
    r.refine_follows = B->adapt;
    r.mode = 0;
    r.ncall = x.ncall;
    r.inv_c = 1.0 / (double)x.ncall;
    r.inv_cm1 = 1.0 / (double)(x.ncall - 1);
    r.n_tiles = x.n_tiles;
    int gx = 0, gy = 0;
    gv::reduce_grid(x.n_tiles, x.nacc, &r.tiles_per_cta, &gx, &gy);
    r.part = x.part;
    r.tileE = x.tileE;
    r.st = x.st;
    r.cpart = x.cpart;
    r.sums = x.sums;
    r.per_iter = B->per_iter + (size_t)b * B->per_iter_cap * 2;
    r.tickets = x.tickets;
    r.alpha = B->alpha;
    r.inv_nbins = 1.0 / (double)B->N;
    r.grid = x.grid;
    for (int yy = 0; yy < gy; ++yy)
      for (int xx = 0; xx < gx; ++xx) rt.push_back(make_int4(b, xx, yy, gx * gy));
  }
  // tables live in one allocation, reallocated when the task counts change
  cudaFree(B->d_fill);
  B->d_fill = nullptr;
  const size_t bytes = a256(sizeof(GvFillArgs) * n) + a256(sizeof(GvReduceArgs) * n) +
                       a256(sizeof(int4) * rt.size());
  void* t = nullptr;
  GB_TRY(cudaMalloc(&t, bytes));
  char* c = (char*)t;
  B->d_fill = (GvFillArgs*)c;
  c += a256(sizeof(GvFillArgs) * n);
  B->d_red = (GvReduceArgs*)c;
  c += a256(sizeof(GvReduceArgs) * n);
  B->d_red_tasks = (int4*)c;
  B->n_red_tasks = (int)rt.size();
  GB_TRY(cudaMemcpy(B->d_fill, fa.data(), sizeof(GvFillArgs) * n, cudaMemcpyHostToDevice));
  GB_TRY(cudaMemcpy(B->d_red, ra.data(), sizeof(GvReduceArgs) * n, cudaMemcpyHostToDevice));
  GB_TRY(cudaMemcpy(B->d_red_tasks, rt.data(), sizeof(int4) * rt.size(), cudaMemcpyHostToDevice));
  return VEGAS_OK;
}

int ensure_per_iter(vegas_batch* B, int itmx) {
  if (itmx <= B->per_iter_cap) return VEGAS_OK;
  if (B->graph) {
    cudaGraphExecDestroy(B->graph);
    B->graph = nullptr;
    B->graph_key.clear();
  }
  cudaFree(B->per_iter);
  B->per_iter = nullptr;
  const int cap = std::max(itmx, 16);
  if (cudaMalloc(&B->per_iter, sizeof(double) * 2 * cap * B->n) != cudaSuccess) {
    cudaGetLastError();
    B->per_iter_cap = 0;
    return VEGAS_ENOMEM;
  }
  B->per_iter_cap = cap;
  return upload_tables(B);
}

int enqueue_iterations(vegas_batch* B, int itmx) {
  std::vector<int> ctas;
  for (const auto& c : B->cls) ctas.push_back(c.ctas);
  for (int k = 0; k < itmx; ++k) {
    GB_TRY(fill_lists(B, B->ept, ctas));
    GB_TRY(gv::launch_reduce_batch(B->d_red, B->d_red_tasks, B->n_red_tasks, k, k == itmx - 1,
                                   k > 0 ? 1.0 / (double)k : 0.0, B->reduce_smem, B->stream));
  }
  return VEGAS_OK;
}

// Choose the launch shape by timing one iteration's fills, side by side as
// in a stage (fastest of three, between resets): events per thread 4 or 8
// (256- or 128-thread CTAs) and each list's persistent grid, all, 3/4 or 1/2
// of its resident CTAs (fewer CTAs per list leave room for the lists that
// run beside it).  4 events per thread and full grids are kept unless
// another shape is more than 2% faster (the trials are noisy).  Results do
// not depend on the choice.
int autotune_batch(vegas_batch* B) {
  const int fixed_ept = B->ept_opt;
  cudaEvent_t e0, e1;
  GB_TRY(cudaEventCreate(&e0));
  GB_TRY(cudaEventCreate(&e1));
  const int def_ept = fixed_ept ? fixed_ept : 4;
  const int def_eighths = B->grid_opt ? B->grid_opt : 8;
  float best = 1e30f, t_def = 1e30f;
  int best_ept = def_ept, best_eighths = def_eighths;
  for (int ept : {4, 8}) {
    if (fixed_ept && ept != fixed_ept) continue;
    for (int eighths : {8, 6, 4}) {
      if (B->grid_opt) eighths = B->grid_opt;
      std::vector<int> ctas;
      for (const auto& c : B->cls) ctas.push_back(class_ctas(B, c, ept, eighths));
      float t = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {
        GB_TRY(cudaEventRecord(e0, B->stream));
        GB_TRY(fill_lists(B, ept, ctas));
        GB_TRY(cudaEventRecord(e1, B->stream));
        GB_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        t = std::min(t, ms);
      }
      if (ept == def_ept && eighths == def_eighths) t_def = t;
      if (t < best) {
        best = t;
        best_ept = ept;
        best_eighths = eighths;
      }
      if (B->grid_opt) break;
    }
  }
  if ((best_ept != def_ept || best_eighths != def_eighths) && best > 0.98f * t_def) {
    best_ept = def_ept;
    best_eighths = def_eighths;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  B->ept = best_ept;
  B->cta_eighths = best_eighths;
  int st = reset_all(B);
  if (st) return st;
  for (auto& c : B->cls) c.ctas = class_ctas(B, c, B->ept, B->cta_eighths);
  return VEGAS_OK;
}

}  // namespace

extern "C" {

int vegas_batch_create(int n, const int* ndim, const int64_t* ncall, const int* integrand_id,
                       const double* params, const int* nparams, int nbins, uint64_t seed,
                       int precision, vegas_batch** out) {
  if (!out) return VEGAS_EINVAL;
  *out = nullptr;
  if (n < 1 || n > (1 << 20) || !ndim || !ncall || !integrand_id || !params || !nparams ||
      nbins < VEGAS_MIN_BINS || nbins > VEGAS_MAX_BINS || (precision != 0 && precision != 1))
    return VEGAS_EINVAL;
  for (int b = 0; b < n; ++b) {
    if (ndim[b] < 1 || ndim[b] > VEGAS_MAX_DIM || ndim[b] * nbins > VEGAS_MAX_DIM_BINS ||
        ncall[b] < 2 || ncall[b] > ((int64_t)1 << 40) || nparams[b] < 0 ||
        nparams[b] > VEGAS_MAX_PARAMS - 1)
      return VEGAS_EINVAL;
    if (batch_check_params(integrand_id[b], ndim[b], params + (size_t)b * VEGAS_MAX_PARAMS,
                           nparams[b]))
      return VEGAS_EINVAL;
  }
  vegas_batch* B = new vegas_batch();
  B->n = n;
  B->N = nbins;
  B->seed = seed;
  B->fp32 = precision;
  if (cudaGetDevice(&B->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&B->sm_count, cudaDevAttrMultiProcessorCount, B->device) !=
          cudaSuccess ||
      cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete B;
    return VEGAS_ECUDA;
  }
  B->own_stream = true;
  B->m.resize(n);
  // one allocation for every member's state, grid, accumulators and partials
  size_t off = 0;
  std::vector<size_t> o(n * 10);  // 10 sub-allocations per member
  for (int b = 0; b < n; ++b) {
    Member& x = B->m[b];
    x.ig = integrand_id[b];
    x.d = ndim[b];
    x.ncall = ncall[b];
    x.np = nparams[b];
    for (int i = 0; i < GV_MAXPARAMS; ++i)
      x.params[i] = i < x.np ? params[(size_t)b * VEGAS_MAX_PARAMS + i] : 0.0;
    x.params[GV_MAXPARAMS - 1] = (double)x.np;
    x.n_tiles = (int)((x.ncall + GV_TILE - 1) / GV_TILE);
    x.nacc = 2 + x.d * nbins;
    int tpc = 0;
    gv::reduce_grid(x.n_tiles, x.nacc, &tpc, &x.gx, &x.gy);
    size_t* q = &o[b * 10];
    q[0] = off;
    off = a256(off + GvGridLayout{x.d, nbins}.doubles() * 8);
    q[1] = off;
    off = a256(off + sizeof(GvState));
    q[2] = off;
    off = a256(off + GV_MAXPARAMS * 8);
    q[3] = off;
    off = a256(off + GV_NCONST * 8);
    q[4] = off;  // cpart
    off = a256(off + (size_t)x.gy * x.gx * 32 * sizeof(GvSlot));
    q[5] = off;
    off = a256(off + (size_t)x.nacc * 8);
    q[7] = off;
    off = a256(off + (size_t)x.n_tiles * x.nacc * 16);
    q[8] = off;
    off = a256(off + (size_t)x.n_tiles * 4);
    q[6] = off;  // tickets
    off = a256(off + gv_tickets_ints(x.nacc) * 4);
  }
  const size_t o_order = off;
  off = a256(off + (size_t)n * 4);
  const size_t o_start = off;
  off = a256(off + (size_t)(n + 9) * 8);
  const size_t o_ccount = off;  // up to nine list counters, one per 128-byte line
  off = a256(off + 9 * 128);
  if (cudaMalloc(&B->dmem, off) != cudaSuccess) {
    cudaGetLastError();
    vegas_batch_free(B);
    return VEGAS_ENOMEM;
  }
  char* base = (char*)B->dmem;
  for (int b = 0; b < n; ++b) {
    Member& x = B->m[b];
    const size_t* q = &o[b * 10];
    x.grid = (double*)(base + q[0]);
    x.st = (GvState*)(base + q[1]);
    x.par = (double*)(base + q[2]);
    x.kconst = (double*)(base + q[3]);
    x.cpart = (GvSlot*)(base + q[4]);
    x.sums = (double*)(base + q[5]);
    x.part = (ulonglong2*)(base + q[7]);
    x.tileE = (int*)(base + q[8]);
    x.tickets = (int*)(base + q[6]);
  }
  int st = VEGAS_OK;
  if (cudaMemsetAsync(B->dmem, 0, off, B->stream) != cudaSuccess) st = VEGAS_ECUDA;
  // uniform grids, constants, reset state
  for (int b = 0; b < n && !st; ++b) {
    Member& x = B->m[b];
    std::vector<double> e((size_t)x.d * (nbins + 1));
    for (int a = 0; a < x.d; ++a)
      for (int i = 0; i <= nbins; ++i) e[(size_t)a * (nbins + 1) + i] = (double)i / nbins;
    if (cudaMemcpy(x.grid, e.data(), e.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(x.par, x.params, sizeof x.params, cudaMemcpyHostToDevice) != cudaSuccess ||
        gv::launch_grid_pack(x.d, nbins, x.grid, B->stream) != cudaSuccess ||
        gv::launch_consts(x.ig, x.par, x.kconst, B->stream) != cudaSuccess ||
        gv::launch_reset(x.st, B->stream) != cudaSuccess)
      st = VEGAS_ECUDA;
  }
  // work lists, one per dimension class and integrand: largest expected cost first
  if (!st) {
    std::vector<int> order;
    std::vector<long long> start;
    int pos = 0, slot = 0;
    for (int maxd : {4, 8, 16}) {
      for (int ig : {VEGAS_GAUSS, VEGAS_DY, VEGAS_EE3J}) {
        std::vector<int> mem;
        for (int b = 0; b < n; ++b)
          if (B->m[b].ig == ig && dim_class(B->m[b].ig, B->m[b].d) == maxd) mem.push_back(b);
        if (mem.empty()) continue;
        std::stable_sort(mem.begin(), mem.end(), [&](int p, int q) {
          return B->m[p].n_tiles * tile_cost(B->m[p].ig, B->m[p].d) >
                 B->m[q].n_tiles * tile_cost(B->m[q].ig, B->m[q].d);
        });
        vegas_batch::FillClass c;
        c.maxd = maxd;
        c.ig = ig;
        c.n = (int)mem.size();
        c.d_order = (int*)(base + o_order) + pos;
        c.d_start = (long long*)(base + o_start) + pos + slot;
        c.d_counter = (unsigned long long*)(base + o_ccount + 128 * slot);
        long long acc = 0;
        start.push_back(0);
        for (int b : mem) {
          order.push_back(b);
          acc += B->m[b].n_tiles;
          start.push_back(acc);
          c.smem = std::max(c.smem,
                            GvFillSmem(B->m[b].d, nbins, B->fp32 ? 4 : 8, true, maxd > 4).total);
        }
        c.total = acc;
        B->cls.push_back(c);
        pos += c.n;
        ++slot;
      }
    }
    if (cudaMemcpy(base + o_order, order.data(), order.size() * 4, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(base + o_start, start.data(), start.size() * 8, cudaMemcpyHostToDevice) !=
            cudaSuccess)
      st = VEGAS_ECUDA;
  }
  // launch order of the lists (largest estimated cost first), side streams
  // and the events that fork and join them
  if (!st) {
    std::vector<double> cost(B->cls.size(), 0.0);
    for (size_t i = 0; i < B->cls.size(); ++i)
      for (int b = 0; b < n; ++b)
        if (B->m[b].ig == B->cls[i].ig && dim_class(B->m[b].ig, B->m[b].d) == B->cls[i].maxd)
          cost[i] += (double)B->m[b].n_tiles * tile_cost(B->m[b].ig, B->m[b].d);
    for (size_t i = 0; i < B->cls.size(); ++i) B->launch_order.push_back((int)i);
    std::stable_sort(B->launch_order.begin(), B->launch_order.end(),
                     [&](int p, int q) { return cost[p] > cost[q]; });
    if (B->cls.size() > 1 &&
        cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) != cudaSuccess)
      st = VEGAS_ECUDA;
    for (size_t i = 1; i < B->cls.size() && !st; ++i) {
      cudaStream_t sd = nullptr;
      cudaEvent_t ev = nullptr;
      if (cudaStreamCreateWithFlags(&sd, cudaStreamNonBlocking) != cudaSuccess) {
        st = VEGAS_ECUDA;
        break;
      }
      B->side.push_back(sd);
      if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        st = VEGAS_ECUDA;
        break;
      }
      B->join.push_back(ev);
    }
    if (st) cudaGetLastError();
  }
  if (!st) {
    B->reduce_smem = gv::reduce_smem_bytes(nbins);
    st = ensure_per_iter(B, 16);
  }
  if (!st && cudaStreamSynchronize(B->stream) != cudaSuccess) st = VEGAS_ECUDA;
  if (st) {
    vegas_batch_free(B);
    return st;
  }
  *out = B;
  return VEGAS_OK;
}

void vegas_batch_free(vegas_batch* B) {
  if (!B) return;
  if (B->stream) cudaStreamSynchronize(B->stream);
  if (B->graph) cudaGraphExecDestroy(B->graph);
  cudaFree(B->d_fill);
  cudaFree(B->per_iter);
  cudaFree(B->dmem);
  if (B->pinned) cudaFreeHost(B->pinned);
  for (cudaStream_t sd : B->side) cudaStreamDestroy(sd);
  for (cudaEvent_t ev : B->join) cudaEventDestroy(ev);
  if (B->fork) cudaEventDestroy(B->fork);
  if (B->own_stream && B->stream) cudaStreamDestroy(B->stream);
  delete B;
}

int vegas_batch_set_option(vegas_batch* B, int key, double v) {
  if (!B || !std::isfinite(v)) return VEGAS_EINVAL;
  switch (key) {
    case VEGAS_OPT_ALPHA:
      if (v < 0.0) return VEGAS_EINVAL;
      B->alpha = v;
      break;
    case VEGAS_OPT_PRECISION:
      return VEGAS_EINVAL;  // fixed at creation (it sizes shared memory)
    case VEGAS_OPT_ADAPT:
      if (v != 0.0 && v != 1.0) return VEGAS_EINVAL;
      B->adapt = (int)v;
      break;
    case VEGAS_OPT_EPT:
      if (v != 0.0 && v != 4.0 && v != 8.0) return VEGAS_EINVAL;
      B->ept_opt = (int)v;
      B->ept = 0;
      break;
    case VEGAS_OPT_BATCH_GRID:
      if (!(v >= 0.0 && v <= 8.0) || v != std::floor(v)) return VEGAS_EINVAL;
      B->grid_opt = (int)v;
      B->ept = 0;
      break;
    case VEGAS_OPT_NONFINITE:
      if (v != 0.0 && v != 1.0) return VEGAS_EINVAL;
      B->nonfinite_policy = (int)v;
      return VEGAS_OK;
    case VEGAS_OPT_GRAPH:
      if (v != 0.0 && v != 1.0) return VEGAS_EINVAL;
      B->use_graph = (int)v;
      break;
    default:
      return VEGAS_EINVAL;
  }
  if (B->graph) {
    cudaStreamSynchronize(B->stream);
    cudaGraphExecDestroy(B->graph);
    B->graph = nullptr;
    B->graph_key.clear();
  }
  return upload_tables(B);
}

int vegas_batch_set_stream(vegas_batch* B, void* stream) {
  if (!B) return VEGAS_EINVAL;
  if (B->stream) cudaStreamSynchronize(B->stream);
  if (B->own_stream && B->stream) cudaStreamDestroy(B->stream);
  B->own_stream = false;
  B->stream = (cudaStream_t)stream;
  if (B->graph) {
    cudaGraphExecDestroy(B->graph);
    B->graph = nullptr;
    B->graph_key.clear();
  }
  return VEGAS_OK;
}

int vegas_batch_iterate(vegas_batch* B, int itmx, double* integral, double* error,
                        double* chi2_dof, double* per_iter) {
  if (!B || itmx < 1 || itmx > 100000 || !integral || !error || !chi2_dof) return VEGAS_EINVAL;
  int st = ensure_per_iter(B, itmx);
  if (st) return st;
  if (!B->ept) {
    st = autotune_batch(B);
    if (st) return st;
  }
  const bool graph_ok = B->use_graph && B->stream != nullptr;
  if (graph_ok) {
    const std::string key = std::to_string(itmx) + ":" + std::to_string(B->ept) + ":" +
                            std::to_string(B->cta_eighths) + ":" + std::to_string(B->adapt);
    if (!B->graph || B->graph_key != key) {
      if (B->graph) {
        cudaGraphExecDestroy(B->graph);
        B->graph = nullptr;
      }
      cudaGraph_t g;
      GB_TRY(cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal));
      st = enqueue_iterations(B, itmx);
      const cudaError_t ce = cudaStreamEndCapture(B->stream, &g);
      if (st) {
        if (ce == cudaSuccess) cudaGraphDestroy(g);
        return st;
      }
      GB_TRY(ce);
      const cudaError_t ie = cudaGraphInstantiate(&B->graph, g, 0);
      cudaGraphDestroy(g);
      GB_TRY(ie);
      B->graph_key = key;
    }
    GB_TRY(cudaGraphLaunch(B->graph, B->stream));
  } else {
    st = enqueue_iterations(B, itmx);
    if (st) return st;
  }
  // results: every member's state and per-iteration records
  const size_t need = sizeof(GvState) * B->n + sizeof(double) * 2 * B->per_iter_cap * B->n + 64;
  if (B->pinned_bytes < need) {
    if (B->pinned) cudaFreeHost(B->pinned);
    B->pinned = nullptr;
    B->pinned_bytes = 0;
    if (cudaHostAlloc(&B->pinned, need, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return VEGAS_ENOMEM;
    }
    B->pinned_bytes = need;
  }
  GvState* hs = (GvState*)B->pinned;
  double* hp = (double*)((char*)B->pinned + ((sizeof(GvState) * B->n + 63) & ~(size_t)63));
  for (int b = 0; b < B->n; ++b)
    GB_TRY(cudaMemcpyAsync(hs + b, B->m[b].st, sizeof(GvState), cudaMemcpyDeviceToHost,
                           B->stream));
  GB_TRY(cudaMemcpyAsync(hp, B->per_iter, sizeof(double) * 2 * B->per_iter_cap * B->n,
                         cudaMemcpyDeviceToHost, B->stream));
  GB_TRY(cudaStreamSynchronize(B->stream));
  unsigned long long bad = 0;
  for (int b = 0; b < B->n; ++b) {
    integral[b] = hs[b].integral;
    error[b] = hs[b].error;
    chi2_dof[b] = hs[b].chi2;
    bad += hs[b].nonfinite;
    if (per_iter)
      memcpy(per_iter + (size_t)b * itmx * 2, hp + (size_t)b * B->per_iter_cap * 2,
             sizeof(double) * 2 * itmx);
  }
  if (bad && B->nonfinite_policy == 0) return VEGAS_ENONFINITE;
  return VEGAS_OK;
}

int vegas_batch_grid_get(const vegas_batch* B, int index, double* edges) {
  if (!B || !edges || index < 0 || index >= B->n) return VEGAS_EINVAL;
  const Member& x = B->m[index];
  GB_TRY(cudaStreamSynchronize(B->stream));
  GB_TRY(cudaMemcpy(edges, x.grid, sizeof(double) * x.d * (B->N + 1), cudaMemcpyDeviceToHost));
  return VEGAS_OK;
}

}  // extern "C"
