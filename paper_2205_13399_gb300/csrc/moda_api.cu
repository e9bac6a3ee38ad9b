// Host side of the C ABI declared in include/moda.h: validation, instance
// upload, the cooling schedule with its integer acceptance thresholds, the
// -ln(u) table, run buffers, launch, wait and result read-back.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "moda.h"
#include "moda_check.h"
#include "moda_host.h"
#include "moda_internal.h"

namespace {

thread_local std::string g_error;

moda_status fail(moda_status st, const std::string &msg) {
  g_error = msg;
  return st;
}

moda_status cuda_fail(cudaError_t e, const char *what) {
  return fail(MODA_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define MODA_CUDA(call)                                 \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

// Per-device constant data: the -ln(u) table and schedules.
struct DeviceData {
  double *table = nullptr;
  float *tablef = nullptr;  // the same entries rounded to float (warp engine)
  double tmin = 0, tmax = 0;
  struct Sched {
    double *delta = nullptr;
    int64_t *lo = nullptr, *hi = nullptr;
    int32_t count = 0;
    bool frozen = false;  // the last entry holds for every later iteration
  };
  std::map<std::tuple<double, double, double>, Sched> schedules;
};

std::mutex g_dev_mutex;
std::map<int, DeviceData> g_dev;

std::vector<double> neglog_table_host() {
  std::vector<double> T(moda::kTableSize);
  for (int idx = 0; idx < moda::kTableSize; ++idx)
    T[idx] = -std::log((static_cast<double>(idx) + 0.5) / 65536.0);
  return T;
}

// Returns the device table (built once per device); caller holds the lock.
moda_status device_table(int dev, DeviceData **out) {
  DeviceData &dd = g_dev[dev];
  if (!dd.table) {
    std::vector<double> T = neglog_table_host();
    double *d = nullptr;
    MODA_CUDA(cudaMalloc(&d, sizeof(double) * T.size()));
    cudaError_t e = cudaMemcpy(d, T.data(), sizeof(double) * T.size(),
                               cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(d);
      return cuda_fail(e, "upload -ln(u) table");
    }
    std::vector<float> Tf(T.size());
    for (size_t i = 0; i < T.size(); ++i) Tf[i] = static_cast<float>(T[i]);
    float *f = nullptr;
    e = cudaMalloc(&f, sizeof(float) * Tf.size());
    if (e == cudaSuccess)
      e = cudaMemcpy(f, Tf.data(), sizeof(float) * Tf.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(d);
      if (f) cudaFree(f);
      return cuda_fail(e, "upload -ln(u) table");
    }
    dd.table = d;
    dd.tablef = f;
    dd.tmax = T.front();
    dd.tmin = T.back();
  }
  *out = &dd;
  return MODA_OK;
}

// Alg. 3: before each iteration, "if delta > delta_f: delta <- delta (1 -
// xi)".  The entries stop changing at the first delta <= delta_f; later
// iterations reuse the last entry.  Thresholds: a <= floor(delta T_min)
// accepts for every draw, a > floor(delta T_max) rejects for every draw,
// because delta * T is monotone in T under IEEE rounding.
moda_status device_schedule(DeviceData &dd, double d0, double df, double xi,
                            int64_t I_max, DeviceData::Sched *out) {
  auto key = std::make_tuple(d0, df, xi);
  auto it = dd.schedules.find(key);
  if (it != dd.schedules.end() &&
      (it->second.frozen || it->second.count >= I_max)) {
    *out = it->second;
    return MODA_OK;
  }
  std::vector<double> delta;
  std::vector<int64_t> lo, hi;
  double d = d0;
  const double factor = 1.0 - xi;
  bool frozen = false;
  for (int64_t t = 1; t <= std::max<int64_t>(I_max, 1); ++t) {
    if (d > df) d = d * factor;
    delta.push_back(d);
    lo.push_back(static_cast<int64_t>(std::floor(d * dd.tmin)));
    hi.push_back(static_cast<int64_t>(std::floor(d * dd.tmax)));
    if (!(d > df)) {
      frozen = true;
      break;
    }
  }
  DeviceData::Sched s;
  s.count = static_cast<int32_t>(delta.size());
  s.frozen = frozen;
  MODA_CUDA(cudaMalloc(&s.delta, sizeof(double) * delta.size()));
  MODA_CUDA(cudaMalloc(&s.lo, sizeof(int64_t) * lo.size()));
  MODA_CUDA(cudaMalloc(&s.hi, sizeof(int64_t) * hi.size()));
  MODA_CUDA(cudaMemcpy(s.delta, delta.data(), sizeof(double) * delta.size(),
                       cudaMemcpyHostToDevice));
  MODA_CUDA(cudaMemcpy(s.lo, lo.data(), sizeof(int64_t) * lo.size(),
                       cudaMemcpyHostToDevice));
  MODA_CUDA(cudaMemcpy(s.hi, hi.data(), sizeof(int64_t) * hi.size(),
                       cudaMemcpyHostToDevice));
  // A shorter schedule for the same key may still be read by a run in
  // flight, so it is kept, not freed.
  dd.schedules[key] = s;
  *out = s;
  return MODA_OK;
}

}  // namespace

namespace moda {
void set_last_error(const char *msg) { g_error = msg; }

moda_status schedule_view(int device, double delta0, double deltaf, double xi,
                          int64_t I_max, ScheduleView *out) {
  std::lock_guard<std::mutex> lock(g_dev_mutex);
  DeviceData *dd = nullptr;
  moda_status st = device_table(device, &dd);
  if (st != MODA_OK) return st;
  DeviceData::Sched sch;
  st = device_schedule(*dd, delta0, deltaf, xi, I_max, &sch);
  if (st != MODA_OK) return st;
  *out = ScheduleView{sch.delta, sch.lo, sch.hi, sch.count, dd->table, dd->tmin, dd->tmax};
  return MODA_OK;
}
}  // namespace moda

struct moda_instance_s;
namespace {
moda_status finish_instance(moda_instance inst, const moda_penalty *pen, moda_instance *out);
}  // namespace

struct moda_instance_s {
  int32_t n = 0, m = 0, W = 0;
  int device = 0;
  int64_t w1 = 0, w2 = 0;
  int64_t b1 = 0, b2 = 0;  // bounds of the local fields
  int64_t c1max = 0, c2max = 0;  // largest cost-QUBO coefficients
  std::vector<int32_t> Fs1, Fs2, D;  // host copies
  int32_t *dFs1 = nullptr, *dFs2 = nullptr, *dD = nullptr;
};

// Device bytes a server has admitted and not yet seen freed.
struct ServerAccount {
  std::atomic<size_t> in_use{0};
};

struct moda_run_s {
  moda_instance inst = nullptr;
  moda_params prm{};
  int32_t R = 0, s = 0, threads = 0, bpt = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t start = nullptr, stop = nullptr;
  int64_t *arch_E = nullptr;
  uint32_t *arch_bits = nullptr;
  int32_t *arch_count = nullptr;
  uint32_t *x_final = nullptr;
  int64_t *E_final = nullptr;
  int64_t *stats = nullptr;
  int64_t *trace = nullptr;
  int32_t *error = nullptr;
  unsigned char *fcache = nullptr;
  bool checked = false;
  size_t bytes = 0;  // device memory held by the run's buffers
  std::shared_ptr<ServerAccount> acct;  // serving: released on destroy
  int32_t nsnap = 0;  // archive snapshots: I_max / snapshot_every
  int32_t *snap_count = nullptr;
  int64_t *snap_E = nullptr;
  uint32_t *snap_bits = nullptr;
  bool warp = false;  // run by the warp annealer
  // the warp-annealer launch's shared device buffers (work list, field
  // caches), freed with the last run of that launch
  std::shared_ptr<struct WarpScratch> wscratch;
};

namespace {

// Device memory of runs comes from the stream-ordered allocator: it is
// allocated on the stream that uses it and given back with cudaFreeAsync,
// which (unlike cudaFree) does not wait for every kernel on the device, so
// retiring one run never stalls the others.  The default pool of each
// device keeps freed memory for reuse.
std::mutex g_pool_mutex;
std::map<int, cudaStream_t> g_free_streams;

// Per device: a library stream for frees of finished runs, and the pool
// set to keep its memory.
cudaStream_t free_stream(int dev) {
  std::lock_guard<std::mutex> lock(g_pool_mutex);
  auto it = g_free_streams.find(dev);
  if (it != g_free_streams.end()) return it->second;
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  g_free_streams[dev] = st;
  return st;
}

// Free device memory including what the pool holds unused.
cudaError_t free_memory(int dev, size_t *free_b) {
  size_t f = 0, total = 0;
  cudaError_t e = cudaMemGetInfo(&f, &total);
  if (e != cudaSuccess) return e;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t reserved = 0, used = 0;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) ==
            cudaSuccess &&
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess &&
        reserved > used)
      f += (size_t)(reserved - used);
  }
  *free_b = f;
  return cudaSuccess;
}

// `done`: the run's work has finished (or never started), so the memory
// may go back on the library's stream; otherwise it is freed in the order
// of the run's own stream.
void free_run_buffers(moda_run r, bool done = false) {
  void *ptrs[] = {r->arch_E, r->arch_bits, r->arch_count, r->x_final,
                  r->E_final, r->stats, r->trace, r->error, r->fcache,
                  r->snap_count, r->snap_E, r->snap_bits};
  cudaStream_t fs = done ? free_stream(r->inst->device) : r->stream;
  for (void *p : ptrs)
    if (p) cudaFreeAsync(p, fs);
  if (r->start) cudaEventDestroy(r->start);
  if (r->stop) cudaEventDestroy(r->stop);
  r->wscratch.reset();
}

bool run_done(moda_run r) { return cudaEventQuery(r->stop) == cudaSuccess; }

// A prepared launch: kernel arguments and launch shape.
struct Prepared {
  moda::AnnealArgs args;
  int workers, rounds;
  bool narrow;
  size_t smem;
  moda::WarpRun wrun;  // the warp annealer's view of the run (r->warp)
};

// The device buffers one warp-annealer launch shares among its runs.
}  // namespace
struct WarpScratch {
  int device = 0;
  void *list = nullptr;   // run descriptors, work items, item counter
  void *cache = nullptr;  // field caches of the resident warps
  ~WarpScratch() {
    cudaStream_t fs = free_stream(device);
    if (list) cudaFreeAsync(list, fs);
    if (cache) cudaFreeAsync(cache, fs);
  }
};
namespace {

// Options the warp annealer runs: the archive escape, without
// normalisation, snapshots or fast-forward.
bool warp_options(const moda_params *p) {
  return p->escape == MODA_ESC_ARCHIVE && p->normalize == 0 && p->snapshot_every == 0 &&
         p->fast_forward == 0;
}

// Whether prepare_run gives a request to the warp annealer.
bool uses_warp(const moda_params *p) {
  return p->engine == 2 || (p->engine == 0 && warp_options(p) && p->block_threads == 0);
}

// The engine of a plain anneal with the automatic choice: the same rule as
// batches and the server (the warp engine whenever the options allow it).
moda_params resolve_plain(moda_instance, const moda_params *p) { return *p; }

// Archive slots with field-cache records per resident team by default.
// A jump to a slot without records rebuilds its fields (O(n^3) by the
// team), which costs as much as hundreds of jumps: on the n = 75 workload
// (archives of up to 528 members) 512 slots took 695 ms and 256 slots
// 7.3 s against 353 ms with 1,024, so the default covers the archives that
// runs reach rather than a byte budget.
constexpr int kWarpCacheSlots = 1024;

// Field-cache slots per team of a warp-engine run before the launch's
// memory budget is applied: all s (field_cache = 1), none (2), min(s,
// cache_slots) when given, else min(s, kWarpCacheSlots).
int warp_slots(moda_instance inst, const moda_params &p) {
  const int s = p.archive_size > 0 ? p.archive_size : inst->m;
  if (p.field_cache == 2) return 0;
  if (p.field_cache == 1) return s;
  if (p.cache_slots > 0) return std::min(s, p.cache_slots);
  return std::min(s, kWarpCacheSlots);
}
// Archive energies kept in shared memory per warp, at most.
constexpr int kWarpSmemEnergies = 512;

}  // namespace

extern "C" {

const char *moda_last_error(void) { return g_error.c_str(); }

moda_status moda_create_instance(int32_t n, const int16_t *F1,
                                 const int16_t *F2, const int16_t *D,
                                 const moda_penalty *pen, moda_instance *out) {
  if (!out) return fail(MODA_EINVAL, "out is NULL");
  *out = nullptr;
  if (!F1 || !F2 || !D) return fail(MODA_EINVAL, "NULL matrix");
  if (n < 2 || n > moda::kMaxN)
    return fail(MODA_EINVAL, "n must be in [2, 128]");
  if (pen && pen->kind != 0 && pen->kind != 1)
    return fail(MODA_EINVAL, "penalty kind must be 0 or 1");
  if (pen && pen->kind == 1 && (pen->w1 < 0 || pen->w2 < 0))
    return fail(MODA_EINVAL, "explicit penalty weights must be >= 0");
  const int nn = n * n;
  for (int e = 0; e < nn; ++e)
    if (F1[e] < 0 || F2[e] < 0 || D[e] < 0)
      return fail(MODA_EINVAL, "flows and distances must be non-negative");
  for (int a = 0; a < n; ++a) {
    if (D[a * n + a] != 0)
      return fail(MODA_EINVAL, "distance matrix needs a zero diagonal");
    for (int b = 0; b < a; ++b)
      if (D[a * n + b] != D[b * n + a])
        return fail(MODA_EINVAL, "distance matrix must be symmetric");
  }
  moda_instance inst = new (std::nothrow) moda_instance_s;
  if (!inst) return fail(MODA_ENOMEM, "host allocation");
  inst->n = n;
  inst->m = nn;
  inst->W = (nn + 31) / 32;
  inst->Fs1.resize(nn);
  inst->Fs2.resize(nn);
  inst->D.resize(nn);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      inst->Fs1[i * n + j] = (int32_t)F1[i * n + j] + (int32_t)F1[j * n + i];
      inst->Fs2[i * n + j] = (int32_t)F2[i * n + j] + (int32_t)F2[j * n + i];
      inst->D[i * n + j] = D[i * n + j];
    }
  return finish_instance(inst, pen, out);
}

}  // extern "C"

namespace {

// Bounds, penalty weights and device upload of an instance whose host
// Fs1, Fs2 and D are filled; takes ownership of `inst`.
moda_status finish_instance(moda_instance inst, const moda_penalty *pen, moda_instance *out) {
  const int n = inst->n, nn = inst->m;
  // Bound of every local field and of w_k: (max row sum of Fs) x (max row
  // sum of D).
  int64_t dmax = 0, f1max = 0, f2max = 0;
  for (int i = 0; i < n; ++i) {
    int64_t sd = 0, s1 = 0, s2 = 0;
    for (int j = 0; j < n; ++j) {
      sd += inst->D[i * n + j];
      s1 += inst->Fs1[i * n + j];
      s2 += inst->Fs2[i * n + j];
    }
    dmax = std::max(dmax, sd);
    f1max = std::max(f1max, s1);
    f2max = std::max(f2max, s2);
  }
  const int64_t b1 = f1max * dmax, b2 = f2max * dmax;  // every entry is >= 0
  {
    int64_t e1 = 0, e2 = 0, ed = 0;
    for (int e = 0; e < nn; ++e) {
      e1 = std::max<int64_t>(e1, inst->Fs1[e]);
      e2 = std::max<int64_t>(e2, inst->Fs2[e]);
      ed = std::max<int64_t>(ed, inst->D[e]);
    }
    inst->c1max = e1 * ed;
    inst->c2max = e2 * ed;
  }
  if (b1 >= (int64_t(1) << 31) || b2 >= (int64_t(1) << 31)) {
    delete inst;
    return fail(MODA_EOVERFLOW, "local fields may exceed int32");
  }
  if (pen && pen->kind == 1) {
    inst->w1 = pen->w1;
    inst->w2 = pen->w2;
  } else {
    inst->w1 = b1;
    inst->w2 = b2;
  }
  inst->b1 = b1;
  inst->b2 = b2;
  cudaGetDevice(&inst->device);
  // One stream-ordered allocation on the library's own stream, and the
  // uploads on it too: neither waits for work in flight elsewhere on the
  // device (a server creates an instance per request while others run).
  const size_t bytes = sizeof(int32_t) * nn;
  cudaStream_t fs = free_stream(inst->device);
  void *base = nullptr;
  cudaError_t e = cudaMallocAsync(&base, 3 * bytes, fs);
  if (e == cudaSuccess) {
    inst->dFs1 = static_cast<int32_t *>(base);
    inst->dFs2 = inst->dFs1 + nn;
    inst->dD = inst->dFs2 + nn;
    e = cudaMemcpyAsync(inst->dFs1, inst->Fs1.data(), bytes, cudaMemcpyHostToDevice, fs);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(inst->dFs2, inst->Fs2.data(), bytes, cudaMemcpyHostToDevice, fs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(inst->dD, inst->D.data(), bytes, cudaMemcpyHostToDevice, fs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(fs);
  if (e != cudaSuccess) {
    moda_destroy_instance(inst);
    return cuda_fail(e, "instance upload");
  }
  *out = inst;
  return MODA_OK;
}

}  // namespace

extern "C" {

moda_status moda_scalarize(moda_instance src, int32_t gamma_num, int32_t gamma_den,
                           moda_instance *out) {
  if (!out) return fail(MODA_EINVAL, "out is NULL");
  *out = nullptr;
  if (!src) return fail(MODA_EINVAL, "NULL instance");
  if (gamma_den < 1 || gamma_num < 0 || gamma_num > gamma_den)
    return fail(MODA_EINVAL, "need 0 <= gamma_num <= gamma_den, gamma_den >= 1");
  moda_instance inst = new (std::nothrow) moda_instance_s;
  if (!inst) return fail(MODA_ENOMEM, "host allocation");
  const int nn = src->m;
  inst->n = src->n;
  inst->m = nn;
  inst->W = src->W;
  inst->Fs1.resize(nn);
  inst->Fs2.assign(nn, 0);
  inst->D = src->D;
  for (int e = 0; e < nn; ++e) {
    const int64_t v = (int64_t)gamma_num * src->Fs1[e] +
                      (int64_t)(gamma_den - gamma_num) * src->Fs2[e];
    if (v >= (int64_t(1) << 31)) {
      delete inst;
      return fail(MODA_EOVERFLOW, "scalarised flows exceed int32");
    }
    inst->Fs1[e] = (int32_t)v;
  }
  cudaSetDevice(src->device);
  return finish_instance(inst, nullptr, out);
}

void moda_destroy_instance(moda_instance inst) {
  if (!inst) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(inst->device);
  // stream-ordered, without synchronising the device; every run of the
  // instance has been destroyed (and so has finished) by now
  if (inst->dFs1) cudaFreeAsync(inst->dFs1, free_stream(inst->device));
  cudaSetDevice(prev);
  delete inst;
}

moda_status moda_instance_info(moda_instance inst, int32_t *n, int64_t *w1,
                               int64_t *w2) {
  if (!inst) return fail(MODA_EINVAL, "NULL instance");
  if (n) *n = inst->n;
  if (w1) *w1 = inst->w1;
  if (w2) *w2 = inst->w2;
  return MODA_OK;
}

}  // extern "C"

namespace {

// The warp annealer's part of prepare_run: validated params, the run's
// buffers, and its WarpRun descriptor (field-cache slots, on-chip archive
// energies and the work list are settled when the launch is planned).
moda_status prepare_warp_run(moda_instance inst, const moda_params *p, cudaStream_t stream,
                             moda_run *out, Prepared *pl) {
  const int m = inst->m;
  if (p->field_cache < 0 || p->field_cache > 2)
    return fail(MODA_EINVAL, "field_cache must be 0 (auto), 1 (on) or 2 (off)");
  if (p->prefetch < 0 || p->prefetch > moda::kWarpMaxLA + 1)
    return fail(MODA_EINVAL, "prefetch must be in [0, 15] for the warp engine");
  if (p->cache_slots < 0) return fail(MODA_EINVAL, "cache_slots must be >= 0");
  if (p->block_threads < 0 || p->block_threads % 32 || p->block_threads > 256)
    return fail(MODA_EINVAL, "warp engine: block_threads must be 32 G, G in 1..8 (0: auto)");
  cudaSetDevice(inst->device);
  moda_run r = new (std::nothrow) moda_run_s;
  if (!r) return fail(MODA_ENOMEM, "host allocation");
  r->inst = inst;
  r->prm = *p;
  r->R = p->replicas;
  r->s = p->archive_size > 0 ? p->archive_size : m;
  r->stream = stream;
  r->warp = true;
  const size_t R = r->R, s = r->s, W = inst->W;
  moda_status st = MODA_OK;
  size_t bytes = 0;
  auto alloc = [&](void **ptr, size_t nb) {
    if (st != MODA_OK) return;
    bytes += nb;
    cudaError_t e = cudaMallocAsync(ptr, nb, stream);
    if (e != cudaSuccess)
      st = fail(MODA_ENOMEM, std::string("device allocation: ") + cudaGetErrorString(e));
  };
  alloc((void **)&r->arch_E, R * s * 2 * sizeof(int64_t));
  alloc((void **)&r->arch_bits, R * s * W * sizeof(uint32_t) + 32);
  alloc((void **)&r->arch_count, R * sizeof(int32_t));
  alloc((void **)&r->x_final, R * W * sizeof(uint32_t));
  alloc((void **)&r->E_final, R * 2 * sizeof(int64_t));
  alloc((void **)&r->stats, R * moda::kStats * sizeof(int64_t));
  alloc((void **)&r->error, sizeof(int32_t));
  if (p->trace && p->I_max > 0)
    alloc((void **)&r->trace, R * (size_t)p->I_max * 3 * sizeof(int64_t));
  DeviceData *dd = nullptr;
  DeviceData::Sched sch;
  if (st == MODA_OK) {
    std::lock_guard<std::mutex> lock(g_dev_mutex);
    st = device_table(inst->device, &dd);
    if (st == MODA_OK) st = device_schedule(*dd, p->delta0, p->deltaf, p->xi, p->I_max, &sch);
  }
  if (st == MODA_OK) {
    cudaError_t e = cudaEventCreate(&r->start);
    if (e == cudaSuccess) e = cudaEventCreate(&r->stop);
    if (e != cudaSuccess) st = cuda_fail(e, "event");
  }
  if (st != MODA_OK) {
    free_run_buffers(r);
    delete r;
    return st;
  }
  moda::WarpRun w{};
  w.n = inst->n;
  w.m = m;
  w.W = inst->W;
  w.s = r->s;
  w.narrow = moda::narrow_ok(inst->n, inst->b1, inst->b2, inst->w1, inst->w2) ? 1 : 0;
  w.accept = p->accept;
  w.archive = p->archive;
  w.nsched = sch.count;
  w.replicas = p->replicas;
  w.replica_base = (uint32_t)p->replica_base;
  w.seed_lo = (uint32_t)(p->seed & 0xFFFFFFFFull);
  w.seed_hi = (uint32_t)(p->seed >> 32);
  w.magic = (uint32_t)(0xFFFFFFFFu / (uint32_t)inst->n) + 1u;
  w.I_max = p->I_max;
  w.w1 = inst->w1;
  w.w2 = inst->w2;
  w.sch_delta = sch.delta;
  w.sch_lo = sch.lo;
  w.sch_hi = sch.hi;
  w.table = dd->table;
  w.tablef = dd->tablef;
  w.Fs1 = inst->dFs1;
  w.Fs2 = inst->dFs2;
  w.D = inst->dD;
  w.arch_E = r->arch_E;
  w.arch_bits = r->arch_bits;
  w.arch_count = r->arch_count;
  w.x_final = r->x_final;
  w.E_final = r->E_final;
  w.stats = r->stats;
  w.trace = r->trace;
  w.error = r->error;
  pl->wrun = w;
  pl->narrow = w.narrow != 0;
  r->bytes = bytes;
  *out = r;
  return MODA_OK;
}

// Validates a request, chooses the block shape and shared-memory placement,
// allocates the run's buffers and fills the kernel arguments; nothing is
// enqueued.  On failure nothing is left allocated.  `budgeted`: the caller
// has already budgeted device memory for the field cache, so an automatic
// field cache is used without the free-memory check.
moda_status prepare_run(moda_instance inst, const moda_params *p,
                        cudaStream_t stream, moda_run *out, Prepared *pl,
                        bool budgeted = false) {
  *out = nullptr;
  if (!inst || !p) return fail(MODA_EINVAL, "NULL instance or params");
  const int m = inst->m;
  if (p->replicas < 1) return fail(MODA_EINVAL, "replicas must be >= 1");
  if (p->I_max < 0 || p->I_max > 0xFFFFFFFFll)
    return fail(MODA_EINVAL, "I_max must be in [0, 2^32)");
  if (!(p->delta0 > 0) || !(p->deltaf > 0) || !(p->xi > 0) || !(p->xi < 1))
    return fail(MODA_EINVAL, "need delta0 > 0, deltaf > 0, 0 < xi < 1");
  if (p->beta < 0) return fail(MODA_EINVAL, "beta must be >= 0");
  if (p->archive_size < 0 || p->archive_size > m)
    return fail(MODA_EINVAL, "archive_size must be in [0, m]");
  if (p->accept != MODA_STRICT && p->accept != MODA_LENIENT)
    return fail(MODA_EINVAL, "accept must be MODA_STRICT or MODA_LENIENT");
  if (p->archive != MODA_EXPLORE && p->archive != MODA_EXPLOIT)
    return fail(MODA_EINVAL, "archive must be MODA_EXPLORE or MODA_EXPLOIT");
  if (p->escape != MODA_ESC_ARCHIVE && p->escape != MODA_ESC_OFFSET)
    return fail(MODA_EINVAL, "escape must be MODA_ESC_ARCHIVE or MODA_ESC_OFFSET");
  if ((uint64_t)p->replica_base + (uint64_t)p->replicas > 0x100000000ull)
    return fail(MODA_EINVAL, "replica indices must fit 32 bits");
  if (p->engine < 0 || p->engine > 2)
    return fail(MODA_EINVAL, "engine must be 0 (auto), 1 (block) or 2 (warp)");
  if (p->engine == 2 && !warp_options(p))
    return fail(MODA_EUNSUPPORTED,
                "the warp engine needs the archive escape without normalize, "
                "snapshot_every or fast_forward");
  if (uses_warp(p)) return prepare_warp_run(inst, p, stream, out, pl);

  // Block shape: B rounds of T threads own the bits, B * T >= m.
  static const int kRounds[] = {1, 2, 3, 4, 6, 8};
  int T = 0, B = 0;
  if (p->block_threads > 0) {
    if (p->block_threads % 32 || p->block_threads > moda::kMaxWorkers)
      return fail(MODA_EINVAL, "block_threads must be a multiple of 32, <= 960");
    T = p->block_threads;
    for (int b : kRounds)
      if ((int64_t)b * T >= m) {
        B = b;
        break;
      }
    if (!B) return fail(MODA_EUNSUPPORTED, "block_threads too small for n");
  } else {
    for (int b : kRounds)
      if ((int64_t)b * moda::kMaxWorkers >= m) {
        B = b;
        break;
      }
    if (!B) return fail(MODA_EUNSUPPORTED, "n too large for this build");
    T = ((m + B - 1) / B + 31) / 32 * 32;
  }
  const int s_cap = p->archive_size > 0 ? p->archive_size : m;
  int dev_smem = 0;
  cudaSetDevice(inst->device);
  MODA_CUDA(cudaDeviceGetAttribute(&dev_smem,
                                   cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                   inst->device));
  if (p->field_cache < 0 || p->field_cache > 2)
    return fail(MODA_EINVAL, "field_cache must be 0 (auto), 1 (on) or 2 (off)");
  if (p->prefetch < 0 || p->prefetch > moda::kMaxLookahead + 1)
    return fail(MODA_EINVAL, "prefetch must be in [0, 4]");
  if (p->normalize != 0 && p->normalize != 1)
    return fail(MODA_EINVAL, "normalize must be 0 or 1");
  if (p->snapshot_every < 0) return fail(MODA_EINVAL, "snapshot_every must be >= 0");
  if (p->snapshot_every > 0 && p->I_max / p->snapshot_every > 1000000)
    return fail(MODA_EINVAL, "more than 10^6 snapshots");
  if (p->fast_forward != 0 && p->fast_forward != 1)
    return fail(MODA_EINVAL, "fast_forward must be 0 or 1");
  if (p->fast_forward &&
      (p->escape != MODA_ESC_ARCHIVE || p->normalize || p->snapshot_every))
    return fail(MODA_EINVAL,
                "fast_forward needs the archive escape, normalize = 0 and snapshot_every = 0");
  const bool ff = p->fast_forward == 1;
  const bool narrow = moda::narrow_ok(inst->n, inst->b1, inst->b2, inst->w1, inst->w2);
  // Field cache: one record of the fields per archive slot, so a jump to
  // the archive reloads the member's fields instead of rebuilding them.
  // Used when the escape jumps to the archive and the records fit in (by
  // default) 60 % of the free device memory.
  const size_t cache_bytes =
      (size_t)p->replicas * s_cap * moda::slot_layout(m, narrow).bytes;
  bool want_cache = p->escape == MODA_ESC_ARCHIVE && p->field_cache != 2;
  if (want_cache && p->field_cache == 0 && !budgeted) {
    size_t free_b = 0;
    MODA_CUDA(free_memory(inst->device, &free_b));
    want_cache = cache_bytes <= free_b / 10 * 6;
  }
  // Shared-memory placement, best first: the field cache (if wanted), the
  // prefetch distance (1, then 0 iterations, then reading the cache in
  // place, unless prescribed), the archive energies and states on chip
  // (then energies only, then neither), Delta E published in shared
  // memory.
  moda::Placement place{};
  bool placed = false;
  moda::SmemLayout lay{};
  const int la_hi = p->prefetch > 0 ? p->prefetch - 1 : 1;
  // (prefetch distance -1: the cache is read in place, no buffers)
  const int la_lo = p->prefetch > 0 ? p->prefetch - 1 : -1;
  for (int c = want_cache ? 1 : 0; c >= 0 && !placed; --c)
    for (int la = c ? la_hi : 0; la >= (c ? la_lo : 0) && !placed; --la)
      for (int opt = 0; opt < 3 && !placed; ++opt)
        for (int de = 1; de >= 0 && !placed; --de) {
          const moda::Placement pl{opt <= 1, opt == 0, c == 1, la, de == 1, narrow, ff};
          const moda::SmemLayout l =
              moda::smem_layout(inst->n, m, inst->W, s_cap, T, B, pl);
          if ((int64_t)l.total <= dev_smem) {
            lay = l;
            place = pl;
            placed = true;
          }
        }
  if (!placed)
    return fail(MODA_EUNSUPPORTED, "shared memory need exceeds the device limit");
  if (p->field_cache == 1 && !place.field_cache)
    return fail(MODA_EUNSUPPORTED, "field cache does not fit");
  const bool use_cache = place.field_cache;

  moda_run r = new (std::nothrow) moda_run_s;
  if (!r) return fail(MODA_ENOMEM, "host allocation");
  r->inst = inst;
  r->prm = *p;
  r->R = p->replicas;
  r->s = p->archive_size > 0 ? p->archive_size : m;
  r->threads = T;
  r->bpt = B;
  r->stream = stream;

  const size_t R = r->R, s = r->s, W = inst->W;
  moda_status st = MODA_OK;
  size_t bytes = 0;
  auto alloc = [&](void **ptr, size_t nb) {
    if (st != MODA_OK) return;
    bytes += nb;
    cudaError_t e = cudaMallocAsync(ptr, nb, stream);
    if (e != cudaSuccess) st = fail(MODA_ENOMEM, std::string("device allocation: ") +
                                                     cudaGetErrorString(e));
  };
  alloc((void **)&r->arch_E, R * s * 2 * sizeof(int64_t));
  // 32 spare bytes: a bulk copy reads whole 16-byte blocks around a state
  alloc((void **)&r->arch_bits, R * s * W * sizeof(uint32_t) + 32);
  if (use_cache) alloc((void **)&r->fcache, cache_bytes);
  alloc((void **)&r->arch_count, R * sizeof(int32_t));
  alloc((void **)&r->x_final, R * W * sizeof(uint32_t));
  alloc((void **)&r->E_final, R * 2 * sizeof(int64_t));
  alloc((void **)&r->stats, R * moda::kStats * sizeof(int64_t));
  alloc((void **)&r->error, sizeof(int32_t));
  if (p->trace && p->I_max > 0)
    alloc((void **)&r->trace, R * (size_t)p->I_max * 3 * sizeof(int64_t));
  if (p->snapshot_every > 0 && p->I_max / p->snapshot_every > 0) {
    r->nsnap = (int32_t)(p->I_max / p->snapshot_every);
    const size_t ns = (size_t)r->nsnap;
    alloc((void **)&r->snap_count, R * ns * sizeof(int32_t));
    alloc((void **)&r->snap_E, R * ns * s * 2 * sizeof(int64_t));
    alloc((void **)&r->snap_bits, R * ns * s * W * sizeof(uint32_t));
  }
  if (st != MODA_OK) {
    free_run_buffers(r);
    delete r;
    return st;
  }

  DeviceData *dd = nullptr;
  DeviceData::Sched sch;
  {
    std::lock_guard<std::mutex> lock(g_dev_mutex);
    st = device_table(inst->device, &dd);
    if (st == MODA_OK)
      st = device_schedule(*dd, p->delta0, p->deltaf, p->xi, p->I_max, &sch);
  }
  if (st != MODA_OK) {
    free_run_buffers(r);
    delete r;
    return st;
  }

  moda::AnnealArgs a{};
  a.n = inst->n;
  a.m = m;
  a.W = inst->W;
  a.s = r->s;
  a.I_max = p->I_max;
  a.replica_base = (uint32_t)p->replica_base;
  a.seed_lo = (uint32_t)(p->seed & 0xFFFFFFFFull);
  a.seed_hi = (uint32_t)(p->seed >> 32);
  a.w1 = inst->w1;
  a.w2 = inst->w2;
  a.beta = p->beta;
  a.accept = p->accept;
  a.archive = p->archive;
  a.escape = p->escape;
  a.magic = (uint32_t)(0xFFFFFFFFu / (uint32_t)inst->n) + 1u;
  a.energies_in_smem = place.energies_in_smem;
  a.bits_in_smem = place.bits_in_smem;
  a.lookahead = place.lookahead;
  a.de_in_smem = place.de_in_smem;
  a.normalize = p->normalize;
  a.s1 = p->normalize ? moda::norm_scale(inst->c1max) : 1.0;
  a.s2 = p->normalize ? moda::norm_scale(inst->c2max) : 1.0;
  a.tmin = dd->tmin;
  a.tmax = dd->tmax;
  a.snap_every = r->nsnap > 0 ? p->snapshot_every : 0;
  a.nsnap = r->nsnap;
  a.snap_count = r->snap_count;
  a.snap_E = r->snap_E;
  a.snap_bits = r->snap_bits;
  a.nsched = sch.count;
  a.sch_delta = sch.delta;
  a.sch_lo = sch.lo;
  a.sch_hi = sch.hi;
  a.table = dd->table;
  a.tablef = dd->tablef;
  a.Fs1 = inst->dFs1;
  a.Fs2 = inst->dFs2;
  a.D = inst->dD;
  a.fcache = r->fcache;
  a.arch_E = r->arch_E;
  a.arch_bits = r->arch_bits;
  a.arch_count = r->arch_count;
  a.x_final = r->x_final;
  a.E_final = r->E_final;
  a.stats = r->stats;
  a.trace = r->trace;
  a.error = r->error;
  a.fast_forward = p->fast_forward;

  cudaError_t e = cudaEventCreate(&r->start);
  if (e == cudaSuccess) e = cudaEventCreate(&r->stop);
  if (e != cudaSuccess) {
    free_run_buffers(r);
    delete r;
    return cuda_fail(e, "event");
  }
  pl->args = a;
  pl->workers = T;
  pl->rounds = B;
  pl->narrow = place.narrow;
  pl->smem = lay.total;
  r->bytes = bytes;
  *out = r;
  return MODA_OK;
}

// Device bytes a run of `p` on `inst` allocates, with or without the field
// cache (the same buffers as prepare_run).
size_t run_bytes(moda_instance inst, const moda_params &p, bool cache) {
  const size_t R = (size_t)p.replicas, m = (size_t)inst->m, W = (size_t)inst->W;
  const size_t s = p.archive_size > 0 ? (size_t)p.archive_size : m;
  const bool narrow = moda::narrow_ok(inst->n, inst->b1, inst->b2, inst->w1, inst->w2);
  size_t b = R * s * 2 * sizeof(int64_t) + R * s * W * sizeof(uint32_t) + 32 +
             R * sizeof(int32_t) + R * W * sizeof(uint32_t) + R * 2 * sizeof(int64_t) +
             R * moda::kStats * sizeof(int64_t) + sizeof(int32_t);
  if (cache && uses_warp(&p)) {
    // the field caches of up to R resident teams
    b += R * moda::align_up(moda::warp_cache_bytes(inst->n, (int)m, warp_slots(inst, p)), 256);
  } else if (cache && p.escape == MODA_ESC_ARCHIVE && p.field_cache != 2) {
    b += R * s * moda::slot_layout((int)m, narrow).bytes;
  }
  if (p.trace && p.I_max > 0) b += R * (size_t)p.I_max * 3 * sizeof(int64_t);
  if (p.snapshot_every > 0) {
    const size_t ns = (size_t)(p.I_max / p.snapshot_every);
    b += R * ns * (sizeof(int32_t) + s * 2 * sizeof(int64_t) + s * W * sizeof(uint32_t));
  }
  return b;
}

// A planned launch of the warp annealer.
struct WarpGroup {
  std::vector<int> idx;  // its runs
  moda::WarpLaunch L{};
  bool narrow = true;
  int grid = 0, warps = 0;
  std::shared_ptr<WarpScratch> scratch;
};

// Plans one launch of the warp annealer over runs[G.idx[k]] (all of one
// variant, narrow or not): the block shape, the field-cache slots and
// on-chip archive energies of each run within `cache_budget` bytes; then
// allocates and uploads, on `stream`, the work list (replicas of the
// largest runs first), clears the item counter and each run's status word.
// The runs share the launch's buffers until the last of them is destroyed.
moda_status plan_warp_group(std::vector<moda_run> &runs, std::vector<Prepared> &pls,
                            WarpGroup &G, cudaStream_t stream, size_t cache_budget) {
  const std::vector<int> &idx = G.idx;
  const moda_run r0 = runs[idx[0]];
  const int dev = r0->inst->device;
  const bool narrow = pls[idx[0]].narrow;
  int n_max = 2, m_max = 4, s_max = 1, la = 2;
  int64_t items_total = 0;
  {
    const int pf = r0->prm.prefetch;
    la = pf > 0 ? pf - 1 : moda::kWarpMaxLA;
  }
  for (int k : idx) {
    const moda_run r = runs[k];
    n_max = std::max(n_max, r->inst->n);
    m_max = std::max(m_max, r->inst->m);
    s_max = std::max(s_max, r->s);
    items_total += r->R;
  }
  int sms = 1, optin = 0;
  MODA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  MODA_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  // Team shape (one team of G warps per block): the largest G (at most one
  // warp per 128-bit chunk) and prefetch distance whose resident teams hold
  // every replica at once, so that few replicas run with short
  // iterations; when even single warps cannot hold them all, single warps
  // (the most replicas in flight).  The on-chip archive energies shrink if
  // nothing fits.
  // The launch shape depends only on these; the server and batches plan
  // the same shapes again and again, so the occupancy queries run once per
  // shape and device (a plan is a pure function of the key).
  const int la_max = la;
  // params.block_threads = 32 G prescribes the team size
  const int forced = r0->prm.block_threads / 32;
  int best_w = 0, best_blocks = 0, se_max = std::min(s_max, kWarpSmemEnergies);
  moda::WarpSmem sm{};
  int kw = 1;
  bool sfields = false;
  int nbf = 0, laf = 0, kwf = 1;
  struct Shape {
    int best_w, best_blocks, la, kw, se_max, nbf, laf, kwf;
    bool sfields;
    moda::WarpSmem sm;
  };
  static std::mutex shape_mu;
  static std::map<std::array<int64_t, 8>, Shape> shapes;
  const std::array<int64_t, 8> key = {dev, narrow ? 1 : 0, n_max, m_max, s_max, items_total,
                                      la_max, forced};
  bool known = false;
  {
    std::lock_guard<std::mutex> lk(shape_mu);
    auto it = shapes.find(key);
    if (it != shapes.end()) {
      const Shape &sh = it->second;
      best_w = sh.best_w;
      best_blocks = sh.best_blocks;
      la = sh.la;
      kw = sh.kw;
      se_max = sh.se_max;
      nbf = sh.nbf;
      laf = sh.laf;
      kwf = sh.kwf;
      sfields = sh.sfields;
      sm = sh.sm;
      known = true;
    }
  }
  if (!known) {
    const int nc_max = (m_max + 127) / 128;
    // (lookahead, window) pairs, preferred first; la + window + 1 buffers
    static const int kOpts[][2] = {{14, 15}, {10, 11}, {8, 9}, {6, 7}, {5, 6}, {4, 5},
                                   {3, 4}, {2, 3}, {1, 2}, {2, 1}, {1, 1}, {0, 1}};
    auto resident = [&](int G, int la_try, int kw_try, int se_try, int *blocks,
                        moda::WarpSmem *out) {
      const moda::WarpSmem L =
          moda::warp_smem(n_max, m_max, se_try, la_try + kw_try + 1, G, false, kw_try);
      *blocks = 0;
      if ((int64_t)L.total > optin) return false;
      if (moda::warp_occupancy(narrow, false, G, L.total, blocks) != cudaSuccess || *blocks < 1)
        return false;
      *out = L;
      return true;
    };
    // (a shorter on-chip archive-energy list is traded for buffers)
    const int se_opts[2] = {se_max, std::min(se_max, 128)};
    for (int gsz = forced > 0 ? forced : std::min(8, nc_max); gsz >= 1 && best_w == 0; --gsz)
      for (const auto &o : kOpts)
        for (int se_try : se_opts) {
          if (o[0] > la_max || best_w != 0) continue;
          int blocks = 0;
          moda::WarpSmem L{};
          if (resident(gsz, o[0], o[1], se_try, &blocks, &L) &&
              ((int64_t)blocks * sms >= items_total || forced > 0)) {
            best_w = gsz;
            best_blocks = blocks;
            la = o[0];
            kw = o[1];
            sm = L;
            se_max = se_try;
          }
        }
    for (int attempt = 0; attempt < 2 && best_w == 0; ++attempt) {
      // throughput: single warps, the most resident (then the larger window)
      for (const auto &o : kOpts) {
        if (o[0] > la_max) continue;
        int blocks = 0;
        moda::WarpSmem L{};
        if (resident(1, o[0], o[1], se_max, &blocks, &L) && blocks > best_blocks) {
          best_w = 1;
          best_blocks = blocks;
          la = o[0];
          kw = o[1];
          sm = L;
        }
      }
      if (best_w == 0) se_max = std::min(se_max, 64);
    }
    if (best_w == 0) return fail(MODA_EUNSUPPORTED, "warp engine: shared memory need exceeds the device");
    // The fields of a flip's state on chip too, where that keeps the
    // residency (as many teams, or still every replica, per launch).
    {
      const moda::WarpSmem L = moda::warp_smem(n_max, m_max, se_max, la + kw + 1, best_w, true, kw);
      int blocks = 0;
      if ((int64_t)L.total <= optin &&
          moda::warp_occupancy(narrow, false, best_w, L.total, &blocks) == cudaSuccess &&
          (blocks >= best_blocks || (int64_t)blocks * sms >= items_total)) {
        sfields = true;
        best_blocks = blocks;
        sm = L;
      }
    }
    // The frozen layout (once the schedule no longer changes a jump brings
    // only the record's header): the longest window whose header buffers
    // keep the residency, in the same shared memory, when it is longer than
    // the window of full records.  (A window position with a candidate bit
    // then reads that chunk's penalties from the record in global memory; on
    // P25, whose full-record windows already reach 15, that cost 13 ms.)
    for (const auto &o : kOpts) {
      if (o[0] > la_max || o[1] <= kw) continue;
      const int nb = o[0] + o[1] + 1;
      const moda::WarpSmem L =
          moda::warp_smem(n_max, m_max, se_max, la + kw + 1, best_w, sfields, kw, nb, o[1]);
      int blocks = 0;
      if ((int64_t)L.total <= optin &&
          moda::warp_occupancy(narrow, true, best_w, L.total, &blocks) == cudaSuccess &&
          blocks >= best_blocks) {
        nbf = nb;
        laf = o[0];
        kwf = o[1];
        sm = L;
        break;
      }
    }
    std::lock_guard<std::mutex> lk(shape_mu);
    shapes[key] = Shape{best_w, best_blocks, la, kw, se_max, nbf, laf, kwf, sfields, sm};
  }
  const int64_t resident_teams = (int64_t)best_blocks * sms;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(resident_teams, items_total));
  const size_t warps = (size_t)grid;  // teams, one per block
  // Field-cache slots per run (warp_slots), fewer where field_cache = 0 and
  // the launch's caches would exceed the budget.
  std::vector<int> cs(idx.size());
  auto stride_of = [&]() {
    size_t st = 0;
    for (size_t k = 0; k < idx.size(); ++k) {
      const moda_run r = runs[idx[k]];
      st = std::max(st, moda::warp_cache_bytes(r->inst->n, r->inst->m, cs[k]));
    }
    return moda::align_up(st, 256);
  };
  for (size_t k = 0; k < idx.size(); ++k) {
    const moda_run r = runs[idx[k]];
    cs[k] = warp_slots(r->inst, r->prm);
  }
  size_t stride = stride_of();
  while (warps * stride > cache_budget) {
    bool shrunk = false;
    for (size_t k = 0; k < idx.size(); ++k)
      if (runs[idx[k]]->prm.field_cache == 0 && cs[k] > 16) {
        cs[k] = cs[k] * 3 / 4;
        shrunk = true;
      }
    if (!shrunk) return fail(MODA_ENOMEM, "warp engine: field caches exceed the memory budget");
    stride = stride_of();
  }
  // Run descriptors and the work list.
  std::vector<moda::WarpRun> descs(idx.size());
  std::vector<std::pair<int, int>> order;  // (m, k) largest first
  for (size_t k = 0; k < idx.size(); ++k) {
    moda::WarpRun w = pls[idx[k]].wrun;
    w.cslots = cs[k];
    w.se = std::min(runs[idx[k]]->s, se_max);
    descs[k] = w;
    order.emplace_back(-runs[idx[k]]->inst->m, (int)k);
  }
  std::stable_sort(order.begin(), order.end());
  std::vector<int2> items;
  items.reserve((size_t)items_total);
  for (const auto &o : order)
    for (int q = 0; q < runs[idx[o.second]]->R; ++q) items.push_back(make_int2(o.second, q));
  auto scratch = std::make_shared<WarpScratch>();
  scratch->device = dev;
  // on failure after this point, work already enqueued may still use the
  // scratch: wait for the stream before it is freed
  struct SyncOnFail {
    cudaStream_t s;
    bool armed;
    ~SyncOnFail() {
      if (armed) cudaStreamSynchronize(s);
    }
  } guard{stream, true};
  const size_t d_bytes = moda::align_up(sizeof(moda::WarpRun) * descs.size(), 256);
  const size_t i_bytes = moda::align_up(sizeof(int2) * items.size(), 256);
  MODA_CUDA(cudaMallocAsync(&scratch->list, d_bytes + i_bytes + 256, stream));
  if (warps * stride > 0) {
    cudaError_t e = cudaMallocAsync(&scratch->cache, warps * stride, stream);
    if (e != cudaSuccess)
      return fail(MODA_ENOMEM, std::string("warp engine field caches: ") + cudaGetErrorString(e));
  }
  unsigned char *base = static_cast<unsigned char *>(scratch->list);
  MODA_CUDA(cudaMemcpyAsync(base, descs.data(), sizeof(moda::WarpRun) * descs.size(),
                            cudaMemcpyHostToDevice, stream));
  MODA_CUDA(cudaMemcpyAsync(base + d_bytes, items.data(), sizeof(int2) * items.size(),
                            cudaMemcpyHostToDevice, stream));
  MODA_CUDA(cudaMemsetAsync(base + d_bytes + i_bytes, 0, sizeof(int32_t), stream));
  moda::WarpLaunch L{};
  L.runs = reinterpret_cast<const moda::WarpRun *>(base);
  L.items = reinterpret_cast<const int2 *>(base + d_bytes);
  L.nitems = (int32_t)items.size();
  L.lookahead = la;
  L.stage = moda::warp_stage(m_max, best_w) ? 1 : 0;
  L.sfields = sfields ? 1 : 0;
  L.window = kw;
  L.nbuf = la + kw + 1;
  L.nbuf_f = nbf;
  L.lookahead_f = laf;
  L.window_f = kwf;
  L.team = best_w;
  L.counter = reinterpret_cast<int32_t *>(base + d_bytes + i_bytes);
  L.cache = static_cast<unsigned char *>(scratch->cache);
  L.cache_stride = stride;
  L.sm = sm;
  for (int k : idx) {
    moda_run r = runs[k];
    MODA_CUDA(cudaMemsetAsync(r->error, 0, sizeof(int32_t), stream));
    r->wscratch = scratch;
    r->threads = best_w;  // warps per replica
    r->bpt = grid;
  }
  G.L = L;
  G.narrow = narrow;
  G.grid = grid;
  G.warps = 1;  // teams per block
  G.scratch = scratch;
  guard.armed = false;
  return MODA_OK;
}

// Launches a planned group on `stream` between its runs' start and stop
// events.
moda_status launch_warp_group(std::vector<moda_run> &runs, const WarpGroup &G,
                              cudaStream_t stream) {
  for (int k : G.idx) MODA_CUDA(cudaEventRecord(runs[k]->start, stream));
  MODA_CUDA(moda::launch_warp(G.L, G.narrow, G.grid, G.warps, stream));
  for (int k : G.idx) MODA_CUDA(cudaEventRecord(runs[k]->stop, stream));
  return MODA_OK;
}

// Enqueues a prepared run on its stream: clear the status word, start
// event, kernel, stop event.
moda_status enqueue_run(moda_run r, const Prepared &pl) {
  cudaError_t e = cudaMemsetAsync(r->error, 0, sizeof(int32_t), r->stream);
  if (e == cudaSuccess) e = cudaEventRecord(r->start, r->stream);
  if (e == cudaSuccess)
    e = moda::launch_anneal(pl.args, r->R, pl.workers, pl.rounds, pl.narrow, pl.smem, r->stream);
  if (e == cudaSuccess) e = cudaEventRecord(r->stop, r->stream);
  if (e != cudaSuccess) return cuda_fail(e, "launch");
  return MODA_OK;
}

}  // namespace

extern "C" {

moda_status moda_anneal(moda_instance inst, const moda_params *p,
                        void *cuda_stream, moda_run *out) {
  if (!out) return fail(MODA_EINVAL, "out is NULL");
  *out = nullptr;
  Prepared pl{};
  moda_run r = nullptr;
  if (!inst || !p) return fail(MODA_EINVAL, "NULL instance or params");
  const moda_params q = resolve_plain(inst, p);
  moda_status st = prepare_run(inst, &q, static_cast<cudaStream_t>(cuda_stream), &r, &pl);
  if (st != MODA_OK) return st;
  if (r->warp) {
    size_t free_b = 0;
    MODA_CUDA(free_memory(inst->device, &free_b));
    std::vector<moda_run> rs{r};
    std::vector<Prepared> ps{pl};
    WarpGroup G;
    G.idx = {0};
    st = plan_warp_group(rs, ps, G, r->stream, free_b / 10 * 6);
    if (st == MODA_OK) st = launch_warp_group(rs, G, r->stream);
  } else {
    st = enqueue_run(r, pl);
  }
  if (st != MODA_OK) {
    const std::string msg = g_error;
    cudaStreamSynchronize(r->stream);
    free_run_buffers(r, true);
    delete r;
    return fail(st, msg);
  }
  *out = r;
  return MODA_OK;
}

moda_status moda_wait(moda_run r, int64_t timeout_ms) {
  if (!r) return fail(MODA_EINVAL, "NULL run");
  cudaSetDevice(r->inst->device);
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaEventQuery(r->stop);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) return cuda_fail(e, "run");
    if (timeout_ms >= 0) {
      const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(
                          std::chrono::steady_clock::now() - t0)
                          .count();
      if (ms >= timeout_ms) return fail(MODA_ETIMEOUT, "run still executing");
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  if (!r->checked) {
    int32_t err = 0;
    MODA_CUDA(cudaMemcpy(&err, r->error, sizeof(err), cudaMemcpyDeviceToHost));
    if (err != 0)
      return fail(MODA_ECUDA,
                  "device-side check failed: code " + std::to_string(err) +
                      (err == moda::kErrCopyTimeout ? " (a bounded wait for a field-cache copy gave up)"
                       : err == moda::kErrVariant   ? " (kernel variant launched for a run it does not fit)"
                                                    : ""));
    r->checked = true;
  }
  return MODA_OK;
}

moda_status moda_read_replica(moda_run r, int32_t rep, int32_t *count,
                              int64_t *E, uint32_t *bits, uint32_t *x,
                              int64_t *E_final, int64_t *stats) {
  if (!r) return fail(MODA_EINVAL, "NULL run");
  if (rep < -1 || rep >= r->R) return fail(MODA_EINVAL, "replica out of range");
  cudaSetDevice(r->inst->device);
  if (!run_done(r)) return fail(MODA_EBUSY, "run still executing");
  const size_t first = rep < 0 ? 0 : (size_t)rep;
  const size_t cnt = rep < 0 ? (size_t)r->R : 1;
  const size_t s = r->s, W = r->inst->W;
  auto d2h = cudaMemcpyDeviceToHost;
  if (count)
    MODA_CUDA(cudaMemcpy(count, r->arch_count + first, cnt * sizeof(int32_t), d2h));
  if (E)
    MODA_CUDA(cudaMemcpy(E, r->arch_E + first * s * 2, cnt * s * 2 * sizeof(int64_t), d2h));
  if (bits)
    MODA_CUDA(cudaMemcpy(bits, r->arch_bits + first * s * W,
                         cnt * s * W * sizeof(uint32_t), d2h));
  if (x)
    MODA_CUDA(cudaMemcpy(x, r->x_final + first * W, cnt * W * sizeof(uint32_t), d2h));
  if (E_final)
    MODA_CUDA(cudaMemcpy(E_final, r->E_final + first * 2, cnt * 2 * sizeof(int64_t), d2h));
  if (stats)
    MODA_CUDA(cudaMemcpy(stats, r->stats + first * moda::kStats,
                         cnt * moda::kStats * sizeof(int64_t), d2h));
  return MODA_OK;
}

moda_status moda_read_trace(moda_run r, int32_t rep, int64_t *trace) {
  if (!r || !trace) return fail(MODA_EINVAL, "NULL argument");
  if (!r->trace) return fail(MODA_EINVAL, "run was not traced");
  if (rep < 0 || rep >= r->R) return fail(MODA_EINVAL, "replica out of range");
  cudaSetDevice(r->inst->device);
  if (!run_done(r)) return fail(MODA_EBUSY, "run still executing");
  const size_t len = (size_t)r->prm.I_max * 3;
  MODA_CUDA(cudaMemcpy(trace, r->trace + (size_t)rep * len, len * sizeof(int64_t),
                       cudaMemcpyDeviceToHost));
  return MODA_OK;
}

}  // extern "C"

namespace {

// The non-dominated members of replica `rep` (or all, rep == -1) of an
// archive held on the device as counts[q * ns + j], energies at
// E + (q * ns + j) * s * 2 and states at bits + (q * ns + j) * s * W: the
// final archives (ns = 1, j = 0) or snapshot j of ns.
moda_status archive_front(moda_run r, int32_t rep, moda_point *pts, int32_t cap,
                          int32_t *count, uint8_t *perms, const int32_t *dcnt,
                          const int64_t *dE, const uint32_t *dbits, size_t ns, size_t j) {
  const int n = r->inst->n, W = r->inst->W;
  const size_t s = r->s;
  const int first = rep < 0 ? 0 : rep, last = rep < 0 ? r->R : rep + 1;
  struct Cand {
    int64_t e1, e2;
    int32_t rep, slot;
  };
  std::vector<Cand> c;
  std::vector<int64_t> E(s * 2);
  for (int q = first; q < last; ++q) {
    int32_t cnt = 0;
    const size_t row = (size_t)q * ns + j;
    MODA_CUDA(cudaMemcpy(&cnt, dcnt + row, sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (cnt <= 0) continue;
    MODA_CUDA(cudaMemcpy(E.data(), dE + row * s * 2, sizeof(int64_t) * 2 * (size_t)cnt,
                         cudaMemcpyDeviceToHost));
    for (int32_t k = 0; k < cnt; ++k) c.push_back({E[2 * k], E[2 * k + 1], q, k});
  }
  std::sort(c.begin(), c.end(), [](const Cand &a, const Cand &b) {
    if (a.e1 != b.e1) return a.e1 < b.e1;
    if (a.e2 != b.e2) return a.e2 < b.e2;
    if (a.rep != b.rep) return a.rep < b.rep;
    return a.slot < b.slot;
  });
  // Sweep in E1 order: a point survives iff its E2 is below every E2 seen
  // so far (points with equal E1 and larger E2 are dominated; equal vectors
  // keep the first, i.e. the lowest (replica, slot)).
  std::vector<Cand> keep;
  bool any = false;
  int64_t best2 = 0;
  for (const Cand &q : c) {
    if (!any || q.e2 < best2) {
      keep.push_back(q);
      best2 = q.e2;
      any = true;
    }
  }
  *count = (int32_t)keep.size();
  const int wr = std::min<int32_t>(cap, (int32_t)keep.size());
  std::vector<uint32_t> word(W);
  for (int k = 0; k < wr; ++k) {
    const Cand &q = keep[k];
    MODA_CUDA(cudaMemcpy(word.data(), dbits + (((size_t)q.rep * ns + j) * s + q.slot) * W,
                         W * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    std::vector<int> rows(n, 0), cols(n, 0), loc(n, -1);
    for (int p = 0; p < n * n; ++p)
      if ((word[p >> 5] >> (p & 31)) & 1u) {
        rows[p / n]++;
        cols[p % n]++;
        loc[p / n] = p % n;
      }
    int64_t g = 0;
    for (int i = 0; i < n; ++i)
      g += (int64_t)(1 - rows[i]) * (1 - rows[i]) + (int64_t)(1 - cols[i]) * (1 - cols[i]);
    moda_point &o = pts[k];
    o.E1 = q.e1;
    o.E2 = q.e2;
    o.g = g;
    o.c1 = q.e1 - r->inst->w1 * (g / 2);
    o.c2 = q.e2 - r->inst->w2 * (g / 2);
    o.feasible = g == 0;
    o.replica = q.rep;
    o.slot = q.slot;
    o.pad = 0;
    if (perms)
      for (int i = 0; i < n; ++i)
        perms[(size_t)k * n + i] = g == 0 ? (uint8_t)loc[i] : (uint8_t)0xFF;
  }
  return MODA_OK;
}

}  // namespace

extern "C" {

moda_status moda_read_archive(moda_run r, int32_t rep, moda_point *pts,
                              int32_t cap, int32_t *count, uint8_t *perms) {
  if (!r || !count) return fail(MODA_EINVAL, "NULL argument");
  if (rep < -1 || rep >= r->R) return fail(MODA_EINVAL, "replica out of range");
  if (cap < 0 || (cap > 0 && !pts)) return fail(MODA_EINVAL, "bad output buffer");
  cudaSetDevice(r->inst->device);
  if (!run_done(r)) return fail(MODA_EBUSY, "run still executing");
  return archive_front(r, rep, pts, cap, count, perms, r->arch_count, r->arch_E,
                       r->arch_bits, 1, 0);
}

moda_status moda_read_snapshot(moda_run r, int32_t snap, int32_t rep, moda_point *pts,
                               int32_t cap, int32_t *count, uint8_t *perms) {
  if (!r || !count) return fail(MODA_EINVAL, "NULL argument");
  if (r->nsnap == 0) return fail(MODA_EINVAL, "the run took no snapshots");
  if (snap < 0 || snap >= r->nsnap) return fail(MODA_EINVAL, "snapshot out of range");
  if (rep < -1 || rep >= r->R) return fail(MODA_EINVAL, "replica out of range");
  if (cap < 0 || (cap > 0 && !pts)) return fail(MODA_EINVAL, "bad output buffer");
  cudaSetDevice(r->inst->device);
  if (!run_done(r)) return fail(MODA_EBUSY, "run still executing");
  return archive_front(r, rep, pts, cap, count, perms, r->snap_count, r->snap_E,
                       r->snap_bits, (size_t)r->nsnap, (size_t)snap);
}

moda_status moda_run_elapsed_ms(moda_run r, float *ms) {
  if (!r || !ms) return fail(MODA_EINVAL, "NULL argument");
  cudaSetDevice(r->inst->device);
  if (!run_done(r)) return fail(MODA_EBUSY, "run still executing");
  MODA_CUDA(cudaEventElapsedTime(ms, r->start, r->stop));
  return MODA_OK;
}

void moda_destroy_run(moda_run r) {
  if (!r) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(r->inst->device);
  if (r->stop) cudaEventSynchronize(r->stop);
  free_run_buffers(r, true);
  if (r->acct) r->acct->in_use -= r->bytes;
  cudaSetDevice(prev);
  delete r;
}


// ---- many instances in one graph launch ---------------------------------

moda_status moda_anneal_batch(const moda_instance *insts, const moda_params *params,
                              int32_t count, void *cuda_stream, moda_run *outs) {
  if (!insts || !params || !outs || count < 1)
    return fail(MODA_EINVAL, "need instances, params, outs and count >= 1");
  for (int32_t i = 0; i < count; ++i) outs[i] = nullptr;
  for (int32_t i = 0; i < count; ++i)
    if (!insts[i] || insts[i]->device != insts[0]->device)
      return fail(MODA_EINVAL, "every instance must exist and live on one device");
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  // Device memory for the whole batch: every run's own buffers first; then
  // the field caches of block-engine runs (automatic ones) in order of
  // size, smallest first, while they fit in 60 % of the free memory; what
  // is left goes to the warp-engine launches.
  std::vector<moda_params> prm(params, params + count);
  size_t warp_budget = 0;
  {
    cudaSetDevice(insts[0]->device);
    size_t free_b = 0;
    MODA_CUDA(free_memory(insts[0]->device, &free_b));
    size_t lean = 0;
    for (int32_t i = 0; i < count; ++i) lean += run_bytes(insts[i], prm[i], false);
    if (lean > free_b / 10 * 9)
      return fail(MODA_ENOMEM, "the batch needs " + std::to_string(lean) +
                                   " bytes of run buffers; " + std::to_string(free_b) + " free");
    size_t budget = free_b / 10 * 6 > lean ? free_b / 10 * 6 - lean : 0;
    std::vector<std::pair<size_t, int32_t>> want;
    for (int32_t i = 0; i < count; ++i)
      if (!uses_warp(&prm[i]) && prm[i].field_cache == 0 && prm[i].escape == MODA_ESC_ARCHIVE)
        want.emplace_back(run_bytes(insts[i], prm[i], true) - run_bytes(insts[i], prm[i], false),
                          i);
    std::sort(want.begin(), want.end());
    for (const auto &w : want) {
      if (w.first <= budget)
        budget -= w.first;
      else
        prm[w.second].field_cache = 2;
    }
    warp_budget = budget;
  }
  std::vector<moda_run> runs(count, nullptr);
  std::vector<Prepared> pls(count);
  auto release = [&]() {
    for (moda_run r : runs)
      if (r) {
        free_run_buffers(r);
        delete r;
      }
  };
  for (int32_t i = 0; i < count; ++i) {
    moda_status st = prepare_run(insts[i], &prm[i], stream, &runs[i], &pls[i], true);
    if (st != MODA_OK) {
      const std::string msg = "request " + std::to_string(i) + ": " + g_error;
      release();
      return fail(st, msg);
    }
  }
  // Warp-engine runs: one launch per (variant, size class, prefetch
  // distance), a class spanning at most a factor of two in 128-bit chunks
  // so that no warp's shared memory is sized far beyond its run.
  std::map<std::tuple<int, int, int>, std::vector<int>> classes;
  for (int32_t i = 0; i < count; ++i) {
    if (!runs[i]->warp) continue;
    const int nc = (runs[i]->inst->m + 127) / 128;
    int cls = 0;
    while ((2 << cls) <= nc) ++cls;
    classes[std::make_tuple(pls[i].narrow ? 1 : 0, -cls, runs[i]->prm.prefetch)].push_back(i);
  }
  std::vector<WarpGroup> groups;
  for (auto &kv : classes) {
    WarpGroup G;
    G.idx = kv.second;
    groups.push_back(std::move(G));
  }
  for (WarpGroup &G : groups) {
    moda_status st = plan_warp_group(runs, pls, G, stream, warp_budget / groups.size());
    if (st != MODA_OK) {
      const std::string msg = g_error;
      cudaStreamSynchronize(stream);
      release();
      return fail(st, msg);
    }
  }
  // One CUDA graph: per block-engine run a chain (start event, status word
  // cleared, kernel, stop event); per warp-engine launch its runs' start
  // events, the persistent kernel, their stop events.  The chains share no
  // edge, so the GPU runs them side by side.
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  for (int32_t i = 0; i < count && e == cudaSuccess; ++i) {
    moda_run r = runs[i];
    if (r->warp) continue;
    const Prepared &pl = pls[i];
    cudaGraphNode_t n0, n1, n2, n3;
    const void *func = nullptr;
    e = moda::anneal_function(pl.rounds, pl.narrow, moda::kernel_mode(pl.args, pl.rounds), pl.smem,
                              &func);
    if (e == cudaSuccess) e = cudaGraphAddEventRecordNode(&n0, g, nullptr, 0, r->start);
    if (e == cudaSuccess) {
      cudaMemsetParams mp{};
      mp.dst = r->error;
      mp.value = 0;
      mp.elementSize = sizeof(int32_t);
      mp.width = 1;
      mp.height = 1;
      e = cudaGraphAddMemsetNode(&n1, g, &n0, 1, &mp);
    }
    if (e == cudaSuccess) {
      void *kargs[1] = {const_cast<moda::AnnealArgs *>(&pl.args)};
      cudaKernelNodeParams kp{};
      kp.func = const_cast<void *>(func);
      kp.gridDim = dim3((unsigned)r->R);
      kp.blockDim = dim3((unsigned)(pl.workers + 64));
      kp.sharedMemBytes = (unsigned)pl.smem;
      kp.kernelParams = kargs;
      kp.extra = nullptr;
      e = cudaGraphAddKernelNode(&n2, g, &n1, 1, &kp);
    }
    if (e == cudaSuccess) e = cudaGraphAddEventRecordNode(&n3, g, &n2, 1, r->stop);
  }
  for (const WarpGroup &G : groups) {
    if (e != cudaSuccess) break;
    std::vector<cudaGraphNode_t> starts;
    for (int k : G.idx) {
      cudaGraphNode_t nd;
      e = cudaGraphAddEventRecordNode(&nd, g, nullptr, 0, runs[k]->start);
      if (e != cudaSuccess) break;
      starts.push_back(nd);
    }
    const void *func = nullptr;
    const size_t smem = (size_t)G.warps * G.L.sm.total;
    if (e == cudaSuccess) e = moda::warp_function(G.narrow, G.L.nbuf_f > 0, G.L.team, smem, &func);
    cudaGraphNode_t kn;
    if (e == cudaSuccess) {
      void *kargs[1] = {const_cast<moda::WarpLaunch *>(&G.L)};
      cudaKernelNodeParams kp{};
      kp.func = const_cast<void *>(func);
      kp.gridDim = dim3((unsigned)G.grid);
      kp.blockDim = dim3((unsigned)(32 * G.warps * G.L.team));
      kp.sharedMemBytes = (unsigned)smem;
      kp.kernelParams = kargs;
      kp.extra = nullptr;
      e = cudaGraphAddKernelNode(&kn, g, starts.data(), starts.size(), &kp);
    }
    for (int k : G.idx) {
      if (e != cudaSuccess) break;
      cudaGraphNode_t nd;
      e = cudaGraphAddEventRecordNode(&nd, g, &kn, 1, runs[k]->stop);
    }
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(ex, stream);
  // both may go while the launch runs: an executable graph in flight is
  // freed when it completes
  if (ex) cudaGraphExecDestroy(ex);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaStreamSynchronize(stream);
    release();
    return cuda_fail(e, "batch graph");
  }
  for (int32_t i = 0; i < count; ++i) outs[i] = runs[i];
  return MODA_OK;
}

}  // extern "C"

// ---- serving ------------------------------------------------------------

namespace {

struct Request {
  int64_t ticket = 0;
  moda_instance inst = nullptr;
  moda_params prm{};
  enum State { kPending, kRunning, kDone, kFailed } state = kPending;
  moda_run run = nullptr;
  size_t bytes = 0;
  moda_status err = MODA_OK;
  std::string msg;
};

}  // namespace

struct moda_server_s {
  int device = 0;
  size_t budget = 0;
  // bytes of admitted runs until they are destroyed (by the caller after a
  // poll, or by the server)
  std::shared_ptr<ServerAccount> acct = std::make_shared<ServerAccount>();
  cudaStream_t user_stream = nullptr;
  std::vector<cudaStream_t> streams;
  size_t next_stream = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::shared_ptr<Request>> pending;
  std::vector<std::shared_ptr<Request>> running;
  std::map<int64_t, std::shared_ptr<Request>> tickets;
  std::thread worker;
  bool stopping = false;
  int64_t next_ticket = 1;
  int64_t admitted = 0, completed = 0;
};

namespace {

constexpr int kServerStreams = 32;

// The server's thread: retires finished runs (their bytes return to the
// budget) and admits waiting requests in arrival order while their buffers
// fit the budget, each on a stream of its own, so a request starts as soon
// as memory allows, beside those already running.
void server_loop(moda_server_s *S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lock(S->mu);
  for (;;) {
    for (size_t i = 0; i < S->running.size();) {
      auto &q = S->running[i];
      const cudaError_t e = cudaEventQuery(q->run->stop);
      if (e == cudaErrorNotReady) {
        ++i;
        continue;
      }
      if (e != cudaSuccess) {
        q->state = Request::kFailed;
        q->err = MODA_ECUDA;
        q->msg = std::string("run: ") + cudaGetErrorString(e);
      } else {
        q->state = Request::kDone;
      }
      ++S->completed;
      S->running.erase(S->running.begin() + (long)i);
    }
    while (!S->pending.empty()) {
      std::shared_ptr<Request> q = S->pending.front();
      if (S->stopping) {  // not started: cancelled
        q->state = Request::kFailed;
        q->err = MODA_EINVAL;
        q->msg = "server destroyed before the request started";
        S->pending.pop_front();
        continue;
      }
      moda_params prm = q->prm;
      const size_t full = run_bytes(q->inst, prm, true);
      const size_t lean = run_bytes(q->inst, prm, false);
      const size_t in_use = S->acct->in_use.load();
      if (in_use + full > S->budget) {
        if (!S->running.empty()) break;  // wait for memory
        if (in_use + lean > S->budget) {
          if (in_use > 0) break;  // wait for the caller's runs to be destroyed
          q->state = Request::kFailed;
          q->err = MODA_ENOMEM;
          q->msg = "request needs " + std::to_string(lean) + " bytes, budget " +
                   std::to_string(S->budget);
          S->pending.pop_front();
          continue;
        }
        prm.field_cache = 2;  // alone on the GPU and without the cache it fits
      }
      S->pending.pop_front();
      cudaStream_t st = S->user_stream;
      if (!st) {
        st = S->streams[S->next_stream];
        S->next_stream = (S->next_stream + 1) % S->streams.size();
      }
      Prepared pl{};
      moda_run r = nullptr;
      // the cache was budgeted above (prm.field_cache == 2 when it does not fit)
      moda_status rs = prepare_run(q->inst, &prm, st, &r, &pl, true);
      if (rs == MODA_OK) {
        if (r->warp) {
          std::vector<moda_run> rs1{r};
          std::vector<Prepared> ps1{pl};
          WarpGroup G;
          G.idx = {0};
          const size_t cache_b = run_bytes(q->inst, prm, true) - run_bytes(q->inst, prm, false);
          rs = plan_warp_group(rs1, ps1, G, st, cache_b);
          if (rs == MODA_OK) rs = launch_warp_group(rs1, G, st);
        } else {
          rs = enqueue_run(r, pl);
        }
        if (rs != MODA_OK) {
          cudaStreamSynchronize(st);
          free_run_buffers(r, true);
          delete r;
          r = nullptr;
        }
      }
      if (rs == MODA_ENOMEM && (!S->running.empty() || S->acct->in_use.load() > 0)) {
        S->pending.push_front(q);  // memory held elsewhere: retry when it frees
        break;
      }
      if (rs != MODA_OK) {
        q->state = Request::kFailed;
        q->err = rs;
        q->msg = g_error;
        continue;
      }
      q->run = r;
      q->bytes = r->bytes;
      q->state = Request::kRunning;
      r->acct = S->acct;
      S->acct->in_use += r->bytes;
      ++S->admitted;
      S->running.push_back(q);
    }
    if (S->stopping && S->pending.empty() && S->running.empty()) break;
    S->cv.wait_for(lock, std::chrono::microseconds(S->running.empty() ? 2000 : 100));
  }
}

}  // namespace

extern "C" {

moda_status moda_server_create(size_t hbm_budget, void *cuda_stream, moda_server *out) {
  if (!out) return fail(MODA_EINVAL, "out is NULL");
  *out = nullptr;
  auto *S = new (std::nothrow) moda_server_s;
  if (!S) return fail(MODA_ENOMEM, "host allocation");
  cudaGetDevice(&S->device);
  S->budget = hbm_budget;
  if (S->budget == 0) {  // free memory less a reserve of 1/8 (at least 1 GiB)
    size_t free_b = 0;
    cudaError_t e = free_memory(S->device, &free_b);
    if (e != cudaSuccess) {
      delete S;
      return cuda_fail(e, "cudaMemGetInfo");
    }
    const size_t reserve = std::max<size_t>(free_b / 8, size_t(1) << 30);
    S->budget = free_b > reserve ? free_b - reserve : 0;
  }
  S->user_stream = static_cast<cudaStream_t>(cuda_stream);
  if (!S->user_stream) {
    for (int i = 0; i < kServerStreams; ++i) {
      cudaStream_t st = nullptr;
      cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
      if (e != cudaSuccess) {
        for (cudaStream_t x : S->streams) cudaStreamDestroy(x);
        delete S;
        return cuda_fail(e, "stream");
      }
      S->streams.push_back(st);
    }
  }
  try {
    S->worker = std::thread(server_loop, S);
  } catch (...) {
    for (cudaStream_t x : S->streams) cudaStreamDestroy(x);
    delete S;
    return fail(MODA_ENOMEM, "server thread");
  }
  *out = S;
  return MODA_OK;
}

moda_status moda_server_submit(moda_server S, moda_instance inst, const moda_params *p,
                               int64_t *ticket) {
  if (!S || !inst || !p || !ticket) return fail(MODA_EINVAL, "NULL argument");
  if (inst->device != S->device) return fail(MODA_EINVAL, "instance on another device");
  auto q = std::make_shared<Request>();
  q->inst = inst;
  q->prm = *p;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->stopping) return fail(MODA_EINVAL, "server is shutting down");
    q->ticket = S->next_ticket++;
    S->pending.push_back(q);
    S->tickets[q->ticket] = q;
    *ticket = q->ticket;
  }
  S->cv.notify_one();
  return MODA_OK;
}

moda_status moda_server_poll(moda_server S, int64_t ticket, moda_run *done) {
  if (!S || !done) return fail(MODA_EINVAL, "NULL argument");
  *done = nullptr;
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->tickets.find(ticket);
  if (it == S->tickets.end()) return fail(MODA_EINVAL, "unknown ticket");
  std::shared_ptr<Request> q = it->second;
  if (q->state == Request::kDone) {
    *done = q->run;
    S->tickets.erase(it);
    return MODA_OK;
  }
  if (q->state == Request::kFailed) {
    S->tickets.erase(it);
    return fail(q->err, q->msg);
  }
  return MODA_OK;
}

moda_status moda_server_info(moda_server S, int64_t *pending, int64_t *running,
                             size_t *bytes_in_use, size_t *budget) {
  if (!S) return fail(MODA_EINVAL, "NULL server");
  std::lock_guard<std::mutex> lock(S->mu);
  if (pending) *pending = (int64_t)S->pending.size();
  if (running) *running = (int64_t)S->running.size();
  if (bytes_in_use) *bytes_in_use = S->acct->in_use.load();
  if (budget) *budget = S->budget;
  return MODA_OK;
}

void moda_server_destroy(moda_server S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stopping = true;
  }
  S->cv.notify_one();
  if (S->worker.joinable()) S->worker.join();
  for (auto &kv : S->tickets)
    if (kv.second->state == Request::kDone && kv.second->run) moda_destroy_run(kv.second->run);
  for (cudaStream_t x : S->streams) cudaStreamDestroy(x);
  delete S;
}


// ---- SB-DA front (Alg. 2) ------------------------------------------------

moda_status moda_sbda_front(moda_instance src, const moda_run *runs, int32_t count,
                            moda_point *pts, int32_t cap, int32_t *total, uint8_t *perms) {
  if (!src || !runs || count < 1 || !total || (cap > 0 && !pts))
    return fail(MODA_EINVAL, "need the instance, runs, count >= 1 and outputs");
  const int n = src->n, m = src->m, W = src->W;
  struct Cand {
    int64_t c1, c2;
    int32_t run, rep;
    std::vector<uint8_t> perm;
  };
  std::vector<Cand> cand;
  for (int32_t i = 0; i < count; ++i) {
    moda_run r = runs[i];
    if (!r || r->inst->n != n) return fail(MODA_EINVAL, "run of another size");
    if (!run_done(r)) return fail(MODA_EBUSY, "run still executing");
    const int R = r->R, s = r->s;
    std::vector<int32_t> cnt(R);
    std::vector<uint32_t> bits((size_t)R * s * W), x((size_t)R * W);
    moda_status st = moda_read_replica(r, -1, cnt.data(), nullptr, bits.data(), x.data(),
                                       nullptr, nullptr);
    if (st != MODA_OK) return st;
    for (int q = 0; q < R; ++q) {
      // the run's best state: its one archive member, else the initial state
      const uint32_t *w = cnt[q] > 0 ? bits.data() + (size_t)q * s * W : x.data() + (size_t)q * W;
      std::vector<uint8_t> perm(n, 0xFF);
      std::vector<int> colc(n, 0);
      bool ok = true;
      for (int f = 0; f < n && ok; ++f) {
        int ones = 0;
        for (int u = 0; u < n; ++u) {
          const int p = f * n + u;
          if ((w[p >> 5] >> (p & 31)) & 1u) {
            ++ones;
            perm[f] = (uint8_t)u;
            ++colc[u];
          }
        }
        ok = ones == 1;
      }
      for (int u = 0; u < n && ok; ++u) ok = colc[u] == 1;
      if (!ok) continue;  // infeasible: not a solution of the QAP
      // c_k = sum_ij F^k_ij d_{pi(i) pi(j)} = (1/2) sum_ij Fs^k_ij d_{pi(i) pi(j)}
      int64_t c1 = 0, c2 = 0;
      for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
          const int64_t d = src->D[perm[a] * n + perm[b]];
          c1 += (int64_t)src->Fs1[a * n + b] * d;
          c2 += (int64_t)src->Fs2[a * n + b] * d;
        }
      cand.push_back(Cand{c1 / 2, c2 / 2, i, q, std::move(perm)});
    }
  }
  // non-dominated by (c1, c2); among equal vectors the lowest (run, replica)
  std::vector<size_t> order(cand.size());
  for (size_t k = 0; k < order.size(); ++k) order[k] = k;
  std::sort(order.begin(), order.end(), [&](size_t a, size_t b) {
    return std::tie(cand[a].c1, cand[a].c2, cand[a].run, cand[a].rep) <
           std::tie(cand[b].c1, cand[b].c2, cand[b].run, cand[b].rep);
  });
  std::vector<size_t> keep;
  int64_t best2 = INT64_MAX;
  for (size_t k : order) {  // ascending c1: kept iff c2 beats every earlier one
    if (cand[k].c2 < best2) {
      keep.push_back(k);
      best2 = cand[k].c2;
    }
  }
  *total = (int32_t)keep.size();
  const int32_t nw = std::min<int32_t>(cap, (int32_t)keep.size());
  for (int32_t k = 0; k < nw; ++k) {
    const Cand &c = cand[keep[k]];
    moda_point p{};
    p.E1 = c.c1;
    p.E2 = c.c2;
    p.c1 = c.c1;
    p.c2 = c.c2;
    p.g = 0;
    p.feasible = 1;
    p.replica = c.rep;
    p.slot = c.run;
    pts[k] = p;
    if (perms) memcpy(perms + (size_t)k * n, c.perm.data(), (size_t)n);
  }
  return MODA_OK;
}


// ---- autotuning ------------------------------------------------------------

moda_status moda_check_accept(const int64_t *a, const double *delta, const uint32_t *idx,
                              int32_t count, void *cuda_stream, uint8_t *accept, int8_t *path) {
  if (count < 0) return fail(MODA_EINVAL, "count must be >= 0");
  if (count > 0 && (!a || !delta || !idx || !accept || !path))
    return fail(MODA_EINVAL, "NULL array");
  for (int32_t k = 0; k < count; ++k) {
    if (a[k] < 0) return fail(MODA_EINVAL, "penalties must be >= 0");
    if (!(delta[k] > 0.0) || !std::isfinite(delta[k]))
      return fail(MODA_EINVAL, "delta must be positive and finite");
    if (idx[k] >= (uint32_t)moda::kTableSize) return fail(MODA_EINVAL, "idx must be < 65536");
  }
  if (count == 0) return MODA_OK;
  int dev = 0;
  MODA_CUDA(cudaGetDevice(&dev));
  DeviceData *dd = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_dev_mutex);
    moda_status st = device_table(dev, &dd);
    if (st != MODA_OK) return st;
  }
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  const size_t n = (size_t)count;
  const size_t bytes = n * (8 + 8 + 4 + 1 + 1) + 64;
  unsigned char *d = nullptr;
  MODA_CUDA(cudaMalloc(&d, bytes));
  int64_t *da = reinterpret_cast<int64_t *>(d);
  double *dd_ = reinterpret_cast<double *>(d + 8 * n);
  uint32_t *di = reinterpret_cast<uint32_t *>(d + 16 * n);
  uint8_t *dacc = d + 20 * n;
  int8_t *dpath = reinterpret_cast<int8_t *>(d + 21 * n);
  cudaError_t e = cudaMemcpyAsync(da, a, 8 * n, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dd_, delta, 8 * n, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(di, idx, 4 * n, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess)
    e = moda::launch_check_accept(da, dd_, di, count, dd->table, dd->tablef, dacc, dpath, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(accept, dacc, n, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(path, dpath, n, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "moda_check_accept");
  return MODA_OK;
}

moda_status moda_autotune(moda_instance inst, const moda_params *params, int32_t trial_iters,
                          void *cuda_stream, moda_params *best, float *best_ms) {
  if (!inst || !params || !best) return fail(MODA_EINVAL, "NULL argument");
  if (trial_iters < 1) return fail(MODA_EINVAL, "trial_iters must be >= 1");
  const int m = inst->m;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  const moda_params resolved = resolve_plain(inst, params);
  params = &resolved;
  if (uses_warp(params)) {
    // Warp engine: prefetch distances 0, 2, 4 and 6, each timed on the
    // request's own replicas at the cold end of the schedule.
    moda_params trial = *params;
    trial.I_max = trial_iters;
    trial.delta0 = params->deltaf;
    trial.trace = 0;
    bool found = false;
    float fastest = 0.f;
    moda_params winner = *params;
    for (int32_t pf : {1, 3, 7, 11, 15}) {
      trial.prefetch = pf;
      moda_run r = nullptr;
      if (moda_anneal(inst, &trial, stream, &r) != MODA_OK) continue;
      float ms = 0.f;
      const bool ok = moda_wait(r, -1) == MODA_OK && moda_run_elapsed_ms(r, &ms) == MODA_OK;
      moda_destroy_run(r);
      if (ok && (!found || ms < fastest)) {
        found = true;
        fastest = ms;
        winner.prefetch = pf;
      }
    }
    if (!found) return fail(MODA_EUNSUPPORTED, "no prefetch distance runs this instance");
    *best = winner;
    if (best_ms) *best_ms = fastest;
    return MODA_OK;
  }
  // Candidates: every block shape the kernel has (B bits per thread, the
  // fewest threads that hold m bits) and, when the escape jumps to the
  // archive, prefetch distances 1 and 2 besides the automatic choice.
  std::vector<int32_t> shapes;
  for (int b : {1, 2, 3, 4, 6, 8}) {
    const int64_t T = ((m + b - 1) / b + 31) / 32 * 32;
    if (T >= 32 && T <= moda::kMaxWorkers &&
        std::find(shapes.begin(), shapes.end(), (int32_t)T) == shapes.end())
      shapes.push_back((int32_t)T);
  }
  std::vector<int32_t> prefetches = {0};
  if (params->escape == MODA_ESC_ARCHIVE && params->field_cache != 2) {
    prefetches.push_back(2);
    prefetches.push_back(3);
  }
  // Trials run the cold end of the schedule (delta0 = deltaf, where a run
  // spends most of its iterations) on at most one replica per SM.
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, inst->device);
  moda_params trial = *params;
  trial.replicas = std::min(params->replicas, sms);
  trial.I_max = trial_iters;
  trial.delta0 = params->deltaf;
  trial.trace = 0;
  trial.snapshot_every = 0;
  trial.fast_forward = 0;  // every trial iteration runs
  bool found = false;
  float fastest = 0.f;
  moda_params winner = *params;
  for (int32_t T : shapes)
    for (int32_t pf : prefetches) {
      trial.block_threads = T;
      trial.prefetch = pf;
      moda_run r = nullptr;
      if (moda_anneal(inst, &trial, stream, &r) != MODA_OK) continue;  // does not fit
      float ms = 0.f;
      const bool ok = moda_wait(r, -1) == MODA_OK && moda_run_elapsed_ms(r, &ms) == MODA_OK;
      moda_destroy_run(r);
      if (ok && (!found || ms < fastest)) {
        found = true;
        fastest = ms;
        winner.block_threads = T;
        winner.prefetch = pf;
      }
    }
  if (!found) return fail(MODA_EUNSUPPORTED, "no candidate shape runs this instance");
  *best = winner;
  if (best_ms) *best_ms = fastest;
  return MODA_OK;
}

}  // extern "C"
