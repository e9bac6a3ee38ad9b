// moda_anneal_noalloc: the annealing launch for callers that must not
// allocate device memory.  Some programs cannot call cudaMalloc at the
// point where they anneal: a serving process that hands all of its device
// memory to its own fixed pool (a driver allocation there would fail or
// stall every request), or code whose device memory is owned by a host
// framework that forbids allocations outside its allocator.  This entry
// point takes the instance from host arrays and writes into device output
// buffers the caller owns; everything else the kernel needs -- its field
// cache (scratch), the cooling schedule, the -ln(u) table and the
// instance's matrices -- lives in file-scope device arrays of fixed size,
// which every GPU that loads this library holds until the process exits.
//
// Limits: n <= 128; with the archive escape, replicas * s * r * ceil8(m)
// <= kScratchBytes (64 MiB), r = 8 bytes per bit when every |Delta E_k|
// stays below 2^31 and 16 otherwise (the field-cache record of one archive
// slot); at most kSchedMax schedule entries before the temperature reaches
// delta_f.  No call may be made while its stream is being captured.
//
// The arrays are shared by every call: two calls whose device work
// overlaps (different streams, or different host threads) race on them and
// give wrong results.  Nothing in them has to start at zero: every field
// cache record is written before it is read, and the matrices, table and
// schedule are copied in by each call (the table at set-up).
//
// Set-up: the first call on a device, with that device current, looks up
// the device address of each array (cudaGetSymbolAddress) and uploads the
// -ln(u) table.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "moda.h"
#include "moda_internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;  // field cache
constexpr int kSchedMax = 1 << 16;                   // schedule entries
constexpr int kNN = moda::kMaxN * moda::kMaxN;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];
static __device__ __align__(256) double g_table[moda::kTableSize];
static __device__ __align__(256) float g_tablef[moda::kTableSize];
static __device__ __align__(256) double g_sched_delta[kSchedMax];
static __device__ __align__(256) int64_t g_sched_lo[kSchedMax];
static __device__ __align__(256) int64_t g_sched_hi[kSchedMax];
static __device__ __align__(256) int32_t g_fs1[kNN];
static __device__ __align__(256) int32_t g_fs2[kNN];
static __device__ __align__(256) int32_t g_d[kNN];

struct DeviceSymbols {
  bool ready = false;
  unsigned char *scratch = nullptr;
  double *table = nullptr, *delta = nullptr;
  float *tablef = nullptr;
  int64_t *lo = nullptr, *hi = nullptr;
  int32_t *fs1 = nullptr, *fs2 = nullptr, *d = nullptr;
  double tmin = 0, tmax = 0;
};

// Host staging for the uploads (static, so a call allocates nothing on the
// host either); calls are serialised by g_mutex while they use it.
std::mutex g_mutex;
DeviceSymbols g_symbols[64];
double h_table[moda::kTableSize];
float h_tablef[moda::kTableSize];
double h_delta[kSchedMax];
int64_t h_lo[kSchedMax], h_hi[kSchedMax];
int32_t h_fs1[kNN], h_fs2[kNN], h_d[kNN];

moda_status nofail(moda_status st, const std::string &msg) {
  moda::set_last_error(msg);
  return st;
}

template <typename T>
cudaError_t symbol(T **out, const void *sym) {
  return cudaGetSymbolAddress(reinterpret_cast<void **>(out), sym);
}

// Once per device, with that device current.
moda_status setup(int dev, DeviceSymbols **out) {
  if (dev < 0 || dev >= 64) return nofail(MODA_EUNSUPPORTED, "device index >= 64");
  DeviceSymbols &S = g_symbols[dev];
  if (!S.ready) {
    cudaError_t e = symbol(&S.scratch, g_scratch);
    if (e == cudaSuccess) e = symbol(&S.table, g_table);
    if (e == cudaSuccess) e = symbol(&S.tablef, g_tablef);
    if (e == cudaSuccess) e = symbol(&S.delta, g_sched_delta);
    if (e == cudaSuccess) e = symbol(&S.lo, g_sched_lo);
    if (e == cudaSuccess) e = symbol(&S.hi, g_sched_hi);
    if (e == cudaSuccess) e = symbol(&S.fs1, g_fs1);
    if (e == cudaSuccess) e = symbol(&S.fs2, g_fs2);
    if (e == cudaSuccess) e = symbol(&S.d, g_d);
    if (e != cudaSuccess)
      return nofail(MODA_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    for (int idx = 0; idx < moda::kTableSize; ++idx)
      h_table[idx] = -std::log((static_cast<double>(idx) + 0.5) / 65536.0);
    for (int idx = 0; idx < moda::kTableSize; ++idx) h_tablef[idx] = static_cast<float>(h_table[idx]);
    e = cudaMemcpy(S.table, h_table, sizeof(h_table), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(S.tablef, h_tablef, sizeof(h_tablef), cudaMemcpyHostToDevice);
    if (e != cudaSuccess)
      return nofail(MODA_ECUDA, std::string("table upload: ") + cudaGetErrorString(e));
    S.tmax = h_table[0];
    S.tmin = h_table[moda::kTableSize - 1];
    S.ready = true;
  }
  *out = &S;
  return MODA_OK;
}

}  // namespace

extern "C" moda_status moda_anneal_noalloc(int32_t n, const int16_t *F1,
                                           const int16_t *F2, const int16_t *D,
                                           const moda_penalty *pen,
                                           const moda_params *p,
                                           const moda_device_outputs *out,
                                           void *cuda_stream) {
  if (!F1 || !F2 || !D || !p || !out)
    return nofail(MODA_EINVAL, "NULL argument");
  if (!out->arch_E || !out->arch_bits || !out->arch_count || !out->x_final ||
      !out->E_final || !out->stats || !out->error)
    return nofail(MODA_EINVAL, "NULL output buffer");
  if (n < 2 || n > moda::kMaxN) return nofail(MODA_EINVAL, "n must be in [2, 128]");
  const int m = n * n, W = (m + 31) / 32;
  if (p->replicas < 1) return nofail(MODA_EINVAL, "replicas must be >= 1");
  if (p->I_max < 0 || p->I_max > 0xFFFFFFFFll)
    return nofail(MODA_EINVAL, "I_max must be in [0, 2^32)");
  if (!(p->delta0 > 0) || !(p->deltaf > 0) || !(p->xi > 0) || !(p->xi < 1))
    return nofail(MODA_EINVAL, "need delta0 > 0, deltaf > 0, 0 < xi < 1");
  if (p->beta < 0) return nofail(MODA_EINVAL, "beta must be >= 0");
  if (p->archive_size < 0 || p->archive_size > m)
    return nofail(MODA_EINVAL, "archive_size must be in [0, m]");
  if ((p->accept != MODA_STRICT && p->accept != MODA_LENIENT) ||
      (p->archive != MODA_EXPLORE && p->archive != MODA_EXPLOIT) ||
      (p->escape != MODA_ESC_ARCHIVE && p->escape != MODA_ESC_OFFSET))
    return nofail(MODA_EINVAL, "bad accept / archive / escape mode");
  if ((uint64_t)p->replica_base + (uint64_t)p->replicas > 0x100000000ull)
    return nofail(MODA_EINVAL, "replica indices must fit 32 bits");
  if (p->trace) return nofail(MODA_EUNSUPPORTED, "trace needs an allocation");
  if (pen && (pen->kind < 0 || pen->kind > 1 || (pen->kind == 1 && (pen->w1 < 0 || pen->w2 < 0))))
    return nofail(MODA_EINVAL, "bad penalty");
  const int s = p->archive_size > 0 ? p->archive_size : m;

  std::lock_guard<std::mutex> lock(g_mutex);
  // Instance: the same checks and symmetrised flows as moda_create_instance.
  int32_t *fs1 = h_fs1, *fs2 = h_fs2, *dd = h_d;
  int64_t dmax = 0, f1max = 0, f2max = 0;
  for (int i = 0; i < n; ++i) {
    if (D[i * n + i] != 0) return nofail(MODA_EINVAL, "distance matrix needs a zero diagonal");
    int64_t sd = 0, s1 = 0, s2 = 0;
    for (int j = 0; j < n; ++j) {
      if (F1[i * n + j] < 0 || F2[i * n + j] < 0 || D[i * n + j] < 0)
        return nofail(MODA_EINVAL, "flows and distances must be non-negative");
      if (D[i * n + j] != D[j * n + i])
        return nofail(MODA_EINVAL, "distance matrix must be symmetric");
      fs1[i * n + j] = (int32_t)F1[i * n + j] + F1[j * n + i];
      fs2[i * n + j] = (int32_t)F2[i * n + j] + F2[j * n + i];
      dd[i * n + j] = D[i * n + j];
      sd += dd[i * n + j];
      s1 += fs1[i * n + j];
      s2 += fs2[i * n + j];
    }
    dmax = std::max(dmax, sd);
    f1max = std::max(f1max, s1);
    f2max = std::max(f2max, s2);
  }
  if (f1max * dmax >= (int64_t(1) << 31) || f2max * dmax >= (int64_t(1) << 31))
    return nofail(MODA_EOVERFLOW, "local fields may exceed int32");
  if (p->normalize != 0 && p->normalize != 1)
    return nofail(MODA_EINVAL, "normalize must be 0 or 1");
  if (p->snapshot_every != 0)
    return nofail(MODA_EUNSUPPORTED, "archive snapshots need allocated buffers");
  if (p->fast_forward != 0 && p->fast_forward != 1)
    return nofail(MODA_EINVAL, "fast_forward must be 0 or 1");
  if (p->fast_forward && (p->escape != MODA_ESC_ARCHIVE || p->normalize))
    return nofail(MODA_EINVAL, "fast_forward needs the archive escape and normalize = 0");
  int64_t e1max = 0, e2max = 0, edmax = 0;  // largest entries (normalisation)
  for (int e = 0; e < n * n; ++e) {
    e1max = std::max<int64_t>(e1max, fs1[e]);
    e2max = std::max<int64_t>(e2max, fs2[e]);
    edmax = std::max<int64_t>(edmax, dd[e]);
  }
  const int64_t w1 = pen && pen->kind == 1 ? pen->w1 : f1max * dmax;
  const int64_t w2 = pen && pen->kind == 1 ? pen->w2 : f2max * dmax;

  // Block shape: B rounds of T threads own the bits (as moda_anneal).
  static const int kRounds[] = {1, 2, 3, 4, 6, 8};
  int T = 0, B = 0;
  for (int b : kRounds)
    if ((int64_t)b * (p->block_threads > 0 ? p->block_threads : moda::kMaxWorkers) >= m) {
      B = b;
      break;
    }
  if (!B) return nofail(MODA_EUNSUPPORTED, "n too large for the block size");
  if (p->block_threads > 0) {
    if (p->block_threads % 32 || p->block_threads > moda::kMaxWorkers)
      return nofail(MODA_EINVAL, "block_threads must be a multiple of 32, <= 960");
    T = p->block_threads;
  } else {
    T = ((m + B - 1) / B + 31) / 32 * 32;
  }

  int dev = 0;
  cudaGetDevice(&dev);
  DeviceSymbols *S = nullptr;
  {
    moda_status st = setup(dev, &S);
    if (st != MODA_OK) return st;
  }
  int dev_smem = 0;
  if (cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
      cudaSuccess)
    return nofail(MODA_ECUDA, "device attribute query failed");
  const bool narrow = moda::narrow_ok(n, f1max * dmax, f2max * dmax, w1, w2);
  const size_t rec = moda::slot_layout(m, narrow).bytes;
  // The field cache (the only user of the scratch array) serves jumps to
  // the archive; runs with the offset escape never touch the scratch.
  const bool cache = p->escape == MODA_ESC_ARCHIVE;
  if (cache && (size_t)p->replicas * (size_t)s * rec > kScratchBytes)
    return nofail(MODA_EUNSUPPORTED,
                  "replicas * archive slots * field record exceed the 64 MiB scratch array");
  // Shared-memory placement with the field cache on (escape by jumps) or off.
  moda::Placement place{};
  moda::SmemLayout lay{};
  bool placed = false;
  for (int la = cache ? 1 : 0; la >= (cache ? -1 : 0) && !placed; --la)
    for (int opt = 0; opt < 3 && !placed; ++opt)
      for (int de = 1; de >= 0 && !placed; --de) {
        const moda::Placement pl{opt <= 1, opt == 0, cache, la, de == 1, narrow,
                                 p->fast_forward == 1};
        const moda::SmemLayout l = moda::smem_layout(n, m, W, s, T, B, pl);
        if ((int64_t)l.total <= dev_smem) {
          place = pl;
          lay = l;
          placed = true;
        }
      }
  if (!placed) return nofail(MODA_EUNSUPPORTED, "shared memory need exceeds the device limit");

  // Schedule (Alg. 3: cool before each iteration while delta > delta_f).
  int nsched = 0;
  {
    double d = p->delta0;
    const double factor = 1.0 - p->xi;
    for (int64_t t = 1; t <= std::max<int64_t>(p->I_max, 1); ++t) {
      if (nsched == kSchedMax)
        return nofail(MODA_EUNSUPPORTED, "cooling schedule longer than 65536 entries");
      if (d > p->deltaf) d = d * factor;
      h_delta[nsched] = d;
      h_lo[nsched] = static_cast<int64_t>(std::floor(d * S->tmin));
      h_hi[nsched] = static_cast<int64_t>(std::floor(d * S->tmax));
      ++nsched;
      if (!(d > p->deltaf)) break;
    }
  }
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  {
    // The uploads below read the static host staging arrays, which the
    // next call overwrites: a captured call would replay another call's
    // instance and schedule, so no call may be captured.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess)
      return nofail(MODA_ECUDA, "cudaStreamIsCapturing failed");
    if (cs != cudaStreamCaptureStatusNone)
      return nofail(MODA_EUNSUPPORTED, "moda_anneal_noalloc cannot be captured into a graph");
  }
  const size_t nn4 = sizeof(int32_t) * (size_t)m;
  cudaError_t e = cudaMemcpyAsync(S->fs1, fs1, nn4, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S->fs2, fs2, nn4, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S->d, dd, nn4, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(S->delta, h_delta, sizeof(double) * nsched, cudaMemcpyHostToDevice,
                        stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(S->lo, h_lo, sizeof(int64_t) * nsched, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(S->hi, h_hi, sizeof(int64_t) * nsched, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(out->error, 0, sizeof(int32_t), stream);
  if (e != cudaSuccess)
    return nofail(MODA_ECUDA, std::string("upload: ") + cudaGetErrorString(e));
  // The host staging arrays are pageable: each copy has read them before
  // cudaMemcpyAsync returns, so the next call may reuse them.

  moda::AnnealArgs a{};
  a.n = n;
  a.m = m;
  a.W = W;
  a.s = s;
  a.I_max = p->I_max;
  a.replica_base = (uint32_t)p->replica_base;
  a.seed_lo = (uint32_t)(p->seed & 0xFFFFFFFFull);
  a.seed_hi = (uint32_t)(p->seed >> 32);
  a.magic = (uint32_t)(0xFFFFFFFFu / (uint32_t)n) + 1u;
  a.w1 = w1;
  a.w2 = w2;
  a.beta = p->beta;
  a.accept = p->accept;
  a.archive = p->archive;
  a.escape = p->escape;
  a.nsched = nsched;
  a.energies_in_smem = place.energies_in_smem;
  a.bits_in_smem = place.bits_in_smem;
  a.lookahead = place.lookahead;
  a.de_in_smem = place.de_in_smem;
  a.normalize = p->normalize;
  a.s1 = p->normalize ? moda::norm_scale(e1max * edmax) : 1.0;
  a.s2 = p->normalize ? moda::norm_scale(e2max * edmax) : 1.0;
  a.tmin = S->tmin;
  a.tmax = S->tmax;
  a.sch_delta = S->delta;
  a.sch_lo = S->lo;
  a.sch_hi = S->hi;
  a.table = S->table;
  a.tablef = S->tablef;
  a.Fs1 = S->fs1;
  a.Fs2 = S->fs2;
  a.D = S->d;
  a.fcache = cache ? S->scratch : nullptr;
  a.arch_E = out->arch_E;
  a.arch_bits = out->arch_bits;
  a.arch_count = out->arch_count;
  a.x_final = out->x_final;
  a.E_final = out->E_final;
  a.stats = out->stats;
  a.trace = nullptr;
  a.error = out->error;
  a.fast_forward = p->fast_forward;
  e = moda::launch_anneal(a, p->replicas, T, B, place.narrow, lay.total, stream);
  if (e != cudaSuccess) return nofail(MODA_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  return MODA_OK;
}
