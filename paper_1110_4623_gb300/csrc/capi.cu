// Object sizing and initialisation, co-residency queries and error reporting of the C ABI.
// Algorithm 1 ("CreateSpinLock") allocates one word on the GPU and zeroes it from the CPU;
// here the caller owns the memory and gsync_*_init writes each object's initial state with
// one small kernel on the caller's stream.
#include <cuda.h>
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>

#include "common.cuh"

namespace gsync_impl {
thread_local int g_last_cuda_error = 0;
}
using namespace gsync_impl;

namespace {

// Driver calls for kernels owned by the caller: a kernel handle (CUfunction, which the
// caller gets from cudaGetFuncBySymbol) is valid in any runtime instance of the process,
// while a host-stub pointer is only known to the runtime that registered it.
struct DriverCalls {
  CUresult (*occ_blocks)(int*, CUfunction, int, size_t);
  CUresult (*occ_clusters)(int*, CUfunction, const CUlaunchConfig*);
  CUresult (*launch)(const CUlaunchConfig*, CUfunction, void**, void**);
};

int driver_calls(const DriverCalls** out) {
  static DriverCalls calls;
  static int status = -1;
  static std::mutex mu;
  std::lock_guard<std::mutex> g(mu);
  if (status < 0) {
    void *a = nullptr, *b = nullptr, *c = nullptr;
    cudaDriverEntryPointQueryResult qa, qb, qc;
    const bool ok =
        cudaGetDriverEntryPointByVersion("cuOccupancyMaxActiveBlocksPerMultiprocessor", &a, 12000, cudaEnableDefault,
                                         &qa) == cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuOccupancyMaxActiveClusters", &b, 12000, cudaEnableDefault, &qb) ==
            cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuLaunchKernelEx", &c, 12000, cudaEnableDefault, &qc) == cudaSuccess &&
        qa == cudaDriverEntryPointSuccess && qb == cudaDriverEntryPointSuccess && qc == cudaDriverEntryPointSuccess;
    if (ok) {
      calls.occ_blocks = (CUresult(*)(int*, CUfunction, int, size_t))a;
      calls.occ_clusters = (CUresult(*)(int*, CUfunction, const CUlaunchConfig*))b;
      calls.launch = (CUresult(*)(const CUlaunchConfig*, CUfunction, void**, void**))c;
    }
    (void)cudaGetLastError();
    status = ok ? 1 : 0;
  }
  if (!status) return GSYNC_ECUDA;
  *out = &calls;
  return GSYNC_OK;
}

// cuStreamWriteValue32 (32-bit stream memory operations; a driver that lacks them returns
// CUDA_ERROR_NOT_SUPPORTED from the call, and the caller falls back).
using StreamWrite32 = CUresult (*)(CUstream, CUdeviceptr, cuuint32_t, unsigned int);
StreamWrite32 stream_write32() {
  static StreamWrite32 fn = nullptr;
  static bool looked = false;
  static std::mutex mu;
  std::lock_guard<std::mutex> g(mu);
  if (!looked) {
    looked = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuStreamWriteValue32", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (StreamWrite32)p;
    (void)cudaGetLastError();
  }
  return fn;
}

constexpr uint32_t kLine = 128;
constexpr uint32_t kMagic = 0x6B5C0000u;
enum : uint32_t { kPrimMutex = 1, kPrimBarrier = 2, kPrimSem = 3, kPrimCond = 4 };

constexpr size_t kCohortBytes = 32 * 1024;  // room for a 4 KB page homed on each die
constexpr size_t kPage = 4096;              // granularity of the dies' address interleave

struct InitSpec {
  uint32_t header[16];
  uint32_t nwords;
  uint32_t queue_slots;  // SLEEP_QUEUE: flag lines start at line 3
  uint32_t ring_slots;   // RING: entry lines start at line 3, all empty
  uint32_t spin_sem_s;   // spin semaphores: initial S (line 1), else 0
  uint32_t die_table;    // COHORT: write die[] at kDieTableWord
  uint32_t die[gsync::kMaxSmIds / 4];  // packed bytes
};

__global__ void init_state_kernel(uint32_t* s, InitSpec spec) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < spec.nwords; i += gridDim.x * blockDim.x) {
    uint32_t v = 0;
    if (i < 16) v = spec.header[i];
    if (spec.die_table && i >= gsync::kDieTableWord && i < gsync::kDieTableWord + gsync::kMaxSmIds / 4)
      v = spec.die[i - gsync::kDieTableWord];
    const uint32_t line = i / 32, word = i % 32;
    if (spec.queue_slots && word == 0 && line >= 3 && line < 3 + spec.queue_slots) {
      // Slot k first serves ticket k; before that it holds k - Q, the ticket of the previous
      // lap, which no waiter can be waiting for.  Slot 0 holds ticket 0: the lock is free.
      const uint32_t k = line - 3;
      v = k == 0 ? 0u : k - spec.queue_slots;
    }
    if (spec.ring_slots && word == 0 && line >= 3 && line < 3 + spec.ring_slots) v = gsync::kRingEmpty;
    if (spec.spin_sem_s && line == 1 && word == 0) v = spec.spin_sem_s;
    s[i] = v;
  }
}

int launch_init(void* state, size_t bytes, const InitSpec& spec, cudaStream_t st) {
  if (!state || !aligned(state, kLine)) return GSYNC_EINVAL;
  if ((size_t)spec.nwords * 4 > bytes) return GSYNC_EINVAL;
  const uint32_t threads = 256;
  uint32_t blocks = (spec.nwords + threads - 1) / threads;
  if (blocks > 1024) blocks = 1024;
  init_state_kernel<<<blocks, threads, 0, st>>>((uint32_t*)state, spec);
  GSYNC_CUDA(cudaGetLastError());
  return GSYNC_OK;
}

void fill_header(InitSpec& spec, uint32_t prim, uint32_t kind, uint32_t n, uint32_t param,
                 const gsync_backoff* bo, uint64_t timeout_ns, uint32_t mode) {
  memset(&spec, 0, sizeof spec);
  spec.header[gsync::kHdrMagic] = kMagic | (prim << 8) | kind;
  spec.header[gsync::kHdrN] = n;
  spec.header[gsync::kHdrParam] = param;
  if (bo) {
    spec.header[gsync::kHdrPolicy] = bo->policy;
    spec.header[gsync::kHdrMinNs] = bo->min_ns;
    spec.header[gsync::kHdrMaxNs] = bo->max_ns;
    if (bo->policy == GSYNC_BACKOFF_SPIN_THEN_SLEEP) spec.header[gsync::kHdrSpin] = bo->spin ? bo->spin : 32u;
  }
  spec.header[gsync::kHdrTimeoutLo] = (uint32_t)timeout_ns;
  spec.header[gsync::kHdrTimeoutHi] = (uint32_t)(timeout_ns >> 32);
  spec.header[gsync::kHdrMode] = mode;
}

uint32_t pow2_at_least(uint32_t n) {
  uint32_t q = 1;
  while (q < n) q <<= 1;
  return q;
}

uint32_t tree_nodes(uint32_t n, uint32_t fan) {
  uint32_t total = 0, width = n;
  for (;;) {
    const uint32_t nodes = (width + fan - 1) / fan;
    total += nodes;
    if (nodes == 1) break;
    width = nodes;
  }
  return total;
}

uint32_t barrier_lines(int kind, uint32_t n, uint32_t param) {
  switch (kind) {
    case GSYNC_BAR_ATOMIC:
    case GSYNC_BAR_CLUSTER:
      return 4;
    case GSYNC_BAR_FLAG: {
      const uint32_t fl = (n + 31) / 32;
      return 1 + fl + (param ? 1 : fl);
    }
    case GSYNC_BAR_TREE:
      return 2 + tree_nodes(n, param & 0xFFFFu);
    case GSYNC_BAR_SHARDED:
      return 1 + param + (n + 31) / 32;
    case GSYNC_BAR_DIE:
      return (uint32_t)(kCohortBytes / kLine);
    case GSYNC_BAR_SPLIT:
      return 1 + (param >> 8) + 2 * (param & 0xFFu) + 2;
    case GSYNC_BAR_COUNT: {
      const uint32_t S = (param >> 16) & 0x7Fu;
      return 2 + (S > 1 ? S : 0);
    }
    case GSYNC_BAR_EXCHANGE:
      return 2 + (2 * n * 16 + kLine - 1) / kLine;  // counter, then 2 x n 16-byte records
  }
  return 0;
}

}  // namespace

extern "C" {

int gsync_last_cuda_error(void) { return g_last_cuda_error; }

size_t gsync_mutex_bytes(int kind, int max_waiters) {
  if (kind < GSYNC_MUTEX_CAS_SPIN || kind > GSYNC_MUTEX_CLUSTER_MCS || max_waiters < 1) return 0;
  if (max_waiters > (1 << 24)) return 0;
  if (kind == GSYNC_MUTEX_COHORT) return kCohortBytes;
  const bool queued = kind == GSYNC_MUTEX_SLEEP_QUEUE || kind == GSYNC_MUTEX_RING;
  const uint32_t q = queued ? pow2_at_least((uint32_t)max_waiters) : 0;
  return (size_t)(3 + q) * kLine;
}

}  // extern "C"

namespace {

// Two-die objects (COHORT mutex, DIE barrier): measures the SM-to-die map and the home die
// of the state's 4 KB pages, puts each die's per-die lines on a page homed on that die, and
// fills the header offsets and the die table of `spec`.
int place_on_dies(void* state, InitSpec& spec, cudaStream_t st) {
  uint8_t die[gsync::kMaxSmIds];
  int ndies = 1, sms = 0;
  if (int rc = device_topology(st, die, &ndies, &sms)) return rc;
  // Candidate pages for the per-die lines (at most five per die): every 4 KB boundary past
  // the shared lines and the die table (lines 0-4) with five lines of room before the end.
  constexpr uintptr_t kDieLines = 5;
  const uintptr_t lo = (uintptr_t)state, hi = lo + kCohortBytes;
  const uintptr_t first = (lo + 5 * kLine + kPage - 1) & ~(uintptr_t)(kPage - 1);
  const int npages =
      first + kDieLines * kLine <= hi ? (int)((hi - kDieLines * kLine - first) / kPage) + 1 : 0;
  if (npages < 2) return GSYNC_EINVAL;
  uint8_t home[gsync::kMaxSmIds] = {};
  if (ndies == 2)
    if (int rc = line_homes((const void*)first, npages, kPage, die, sms, st, home)) return rc;
  // Die d's lines go on the first page homed on d; a die with no such page (or a one-die
  // GPU) takes the next unused page, which only costs locality.
  int page[2] = {-1, -1};
  for (int d = 0; d < 2; ++d)
    for (int i = 0; i < npages && page[d] < 0; ++i)
      if (home[i] == d && i != page[0]) page[d] = i;
  for (int d = 0; d < 2; ++d)
    for (int i = 0; i < npages && page[d] < 0; ++i)
      if (i != page[0] && i != page[1]) page[d] = i;
  for (int d = 0; d < 2; ++d)
    spec.header[d ? gsync::kHdrDieOff1 : gsync::kHdrDieOff0] = (uint32_t)((first + (size_t)page[d] * kPage - lo) / 4);
  spec.nwords = (uint32_t)(kCohortBytes / 4);
  spec.die_table = 1;
  memset(spec.die, 0, sizeof spec.die);
  for (int i = 0; i < sms; ++i) ((uint8_t*)spec.die)[i] = ndies == 2 ? die[i] : 0;
  return GSYNC_OK;
}

// CLUSTER and CLUSTER_MCS: the header and the global ticket lock (3 lines).
int init_cluster_kind(uint32_t kind, void* state, size_t bytes, int budget, const gsync_backoff* backoff,
                      uint64_t timeout_ns, void* stream) {
  if (!state || !aligned(state, kLine) || bytes < 3 * kLine || budget < 1 || budget > 32767) return GSYNC_EINVAL;
  if (backoff && backoff->policy > GSYNC_BACKOFF_SPIN_THEN_SLEEP) return GSYNC_EINVAL;
  InitSpec spec;
  fill_header(spec, kPrimMutex, kind, 0, (uint32_t)budget, backoff, timeout_ns, 0);
  spec.nwords = 3 * kLine / 4;
  return launch_init(state, bytes, spec, (cudaStream_t)stream);
}

}  // namespace

extern "C" {

int gsync_mutex_init_cohort(void* state, size_t bytes, int budget, const gsync_backoff* backoff, uint64_t timeout_ns,
                            void* stream) {
  if (!state || !aligned(state, kLine) || bytes < kCohortBytes || budget < 1 || budget > 32767) return GSYNC_EINVAL;
  if (backoff && backoff->policy > GSYNC_BACKOFF_SPIN_THEN_SLEEP) return GSYNC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  InitSpec spec;
  fill_header(spec, kPrimMutex, GSYNC_MUTEX_COHORT, 0, (uint32_t)budget, backoff, timeout_ns, 0);
  if (int rc = place_on_dies(state, spec, st)) return rc;
  return launch_init(state, bytes, spec, st);
}

int gsync_mutex_init_cluster(void* state, size_t bytes, int budget, const gsync_backoff* backoff, uint64_t timeout_ns,
                             void* stream) {
  return init_cluster_kind(GSYNC_MUTEX_CLUSTER, state, bytes, budget, backoff, timeout_ns, stream);
}

int gsync_mutex_init_cluster_mcs(void* state, size_t bytes, int budget, const gsync_backoff* backoff,
                                 uint64_t timeout_ns, void* stream) {
  return init_cluster_kind(GSYNC_MUTEX_CLUSTER_MCS, state, bytes, budget, backoff, timeout_ns, stream);
}

int gsync_mutex_init(void* state, size_t bytes, int kind, int max_waiters, const gsync_backoff* backoff,
                     uint64_t timeout_ns, void* stream) {
  const size_t need = gsync_mutex_bytes(kind, max_waiters);
  if (need == 0 || bytes < need) return GSYNC_EINVAL;
  if (backoff && backoff->policy > GSYNC_BACKOFF_SPIN_THEN_SLEEP) return GSYNC_EINVAL;
  if (kind == GSYNC_MUTEX_COHORT)
    return gsync_mutex_init_cohort(state, bytes, GSYNC_COHORT_DEFAULT_BUDGET, backoff, timeout_ns, stream);
  if (kind == GSYNC_MUTEX_CLUSTER)
    return gsync_mutex_init_cluster(state, bytes, GSYNC_COHORT_DEFAULT_BUDGET, backoff, timeout_ns, stream);
  if (kind == GSYNC_MUTEX_CLUSTER_MCS)
    return gsync_mutex_init_cluster_mcs(state, bytes, GSYNC_COHORT_DEFAULT_BUDGET, backoff, timeout_ns, stream);
  const bool queued = kind == GSYNC_MUTEX_SLEEP_QUEUE || kind == GSYNC_MUTEX_RING;
  const uint32_t q = queued ? pow2_at_least((uint32_t)max_waiters) : 0;
  InitSpec spec;
  fill_header(spec, kPrimMutex, (uint32_t)kind, (uint32_t)max_waiters, q, backoff, timeout_ns, 0);
  spec.nwords = (uint32_t)(need / 4);
  spec.queue_slots = kind == GSYNC_MUTEX_SLEEP_QUEUE ? q : 0u;
  spec.ring_slots = kind == GSYNC_MUTEX_RING ? q : 0u;
  return launch_init(state, bytes, spec, (cudaStream_t)stream);
}

size_t gsync_barrier_bytes(int kind, int nblocks, int param) {
  if (nblocks < 1 || nblocks > (1 << 20)) return 0;
  switch (kind) {
    case GSYNC_BAR_ATOMIC: break;
    case GSYNC_BAR_FLAG: if ((param != 0 && param != 1) || nblocks > 8192) return 0; break;
    case GSYNC_BAR_TREE: {
      const int fan = param & 0xFFFF, form = param >> 16;
      if (param < 0 || fan < 2 || fan > 1024 || form > 1) return 0;
      break;
    }
    case GSYNC_BAR_CLUSTER: {
      const int c = param & 0xF, form = (param >> 4) & 0xF, sleep16 = param >> 8;
      if (param < 0 || c < 1 || c > 8 || nblocks % c || form > 2 || sleep16 > 1023) return 0;
      break;
    }
    case GSYNC_BAR_SHARDED: if (param < 1 || param > 32 || param > nblocks) return 0; break;
    case GSYNC_BAR_DIE: if (param != 0 && param != 1) return 0; break;
    case GSYNC_BAR_COUNT: {
      const int sleep16 = param & 0xFFFF, S = param >> 16;
      if (param < 0 || sleep16 > 1023 || S > 64) return 0;
      break;
    }
    case GSYNC_BAR_EXCHANGE: if (param < 0 || param > 1023) return 0; break;
    case GSYNC_BAR_SPLIT: {
      const int S = param & 0xFF, R = param >> 8;
      if (param < 0 || S < 1 || S > 64 || R < 1 || R > 64) return 0;
      break;
    }
    default: return 0;
  }
  return (size_t)barrier_lines(kind, (uint32_t)nblocks, (uint32_t)param) * kLine;
}

int gsync_barrier_init(void* state, size_t bytes, int kind, int nblocks, int param, uint64_t timeout_ns,
                       void* stream) {
  const size_t need = gsync_barrier_bytes(kind, nblocks, param);
  if (need == 0 || bytes < need) return GSYNC_EINVAL;
  InitSpec spec;
  const uint32_t mode = kind == GSYNC_BAR_FLAG ? (uint32_t)param : 0u;
  fill_header(spec, kPrimBarrier, (uint32_t)kind, (uint32_t)nblocks, (uint32_t)param, nullptr, timeout_ns, mode);
  if (kind == GSYNC_BAR_DIE)
    if (int rc = place_on_dies(state, spec, (cudaStream_t)stream)) return rc;
  spec.nwords = (uint32_t)(need / 4);
  return launch_init(state, bytes, spec, (cudaStream_t)stream);
}

size_t gsync_sem_bytes(int kind) {
  if (kind < GSYNC_SEM_TICKET || kind > GSYNC_SEM_WINDOW) return 0;
  return 4 * kLine;
}

int gsync_sem_init(void* state, size_t bytes, int kind, int initial_count, const gsync_backoff* backoff,
                   uint64_t timeout_ns, void* stream) {
  const size_t need = gsync_sem_bytes(kind);
  if (need == 0 || bytes < need || initial_count < 1 || initial_count > (1 << 30)) return GSYNC_EINVAL;
  if (backoff && backoff->policy > GSYNC_BACKOFF_SPIN_THEN_SLEEP) return GSYNC_EINVAL;
  InitSpec spec;
  fill_header(spec, kPrimSem, (uint32_t)kind, (uint32_t)initial_count, 0, backoff, timeout_ns, 0);
  spec.nwords = (uint32_t)(need / 4);
  const bool spin = kind == GSYNC_SEM_SPIN || kind == GSYNC_SEM_SPIN_BACKOFF;
  spec.spin_sem_s = spin ? (uint32_t)initial_count + 1u : 0u;
  return launch_init(state, bytes, spec, (cudaStream_t)stream);
}

size_t gsync_cond_bytes(void) { return 3 * kLine; }

int gsync_cond_init(void* state, size_t bytes, const gsync_backoff* backoff, uint64_t timeout_ns, void* stream) {
  if (bytes < gsync_cond_bytes()) return GSYNC_EINVAL;
  if (backoff && backoff->policy > GSYNC_BACKOFF_SPIN_THEN_SLEEP) return GSYNC_EINVAL;
  InitSpec spec;
  fill_header(spec, kPrimCond, 0, 0, 0, backoff, timeout_ns, 0);
  spec.nwords = (uint32_t)(gsync_cond_bytes() / 4);
  return launch_init(state, bytes, spec, (cudaStream_t)stream);
}

int gsync_object_abort_flag(const void* state, uint32_t* flag_out, void* stream) {
  if (!state || !flag_out || !aligned(state, kLine)) return GSYNC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  GSYNC_CUDA(cudaMemcpyAsync(flag_out, (const uint32_t*)state + gsync::kHdrAbort, 4, cudaMemcpyDeviceToHost, st));
  GSYNC_CUDA(cudaStreamSynchronize(st));
  return GSYNC_OK;
}

int gsync_object_abort(void* state, void* stream) {
  if (!state || !aligned(state, kLine)) return GSYNC_EINVAL;
  constexpr uint32_t kHostAbort = 2u;  // bit 0 is set by a device wait that timed out
  uint32_t* word = (uint32_t*)state + gsync::kHdrAbort;
  // A stream write is carried out by the GPU's front end: no SM (a memset kernel could wait
  // behind the very grid it is meant to stop, which may hold every SM) and no staging of
  // host memory (a copy from pageable memory waits for the legacy default stream, where the
  // stuck kernel may be running).
  if (const StreamWrite32 write = stream_write32())
    if (write((CUstream)stream, (CUdeviceptr)word, kHostAbort, 0u) == CUDA_SUCCESS) return GSYNC_OK;
  // Without stream memory operations: a copy from host memory (lands only if the stuck kernel
  // is not on the legacy default stream).
  static const uint32_t kValue = kHostAbort;
  GSYNC_CUDA(cudaMemcpyAsync(word, &kValue, 4, cudaMemcpyHostToDevice, (cudaStream_t)stream));
  return GSYNC_OK;
}

int gsync_check_coresident(const void* kernel, int grid, int block_threads, size_t smem_bytes, int cluster,
                           int* max_blocks_out) {
  if (!kernel || !max_blocks_out || grid < 1 || block_threads < 1 || block_threads > 1024 || cluster < 1 ||
      cluster > 16)
    return GSYNC_EINVAL;
  const DriverCalls* d = nullptr;
  if (int rc = driver_calls(&d)) return rc;
  CUfunction f = (CUfunction)kernel;
  int maxb = 0;
  if (cluster > 1) {
    CUlaunchAttribute attr[1];
    attr[0].id = CU_LAUNCH_ATTRIBUTE_CLUSTER_DIMENSION;
    attr[0].value.clusterDim.x = (unsigned)cluster;
    attr[0].value.clusterDim.y = 1;
    attr[0].value.clusterDim.z = 1;
    CUlaunchConfig cfg = {};
    cfg.gridDimX = (unsigned)cluster;
    cfg.gridDimY = cfg.gridDimZ = 1;
    cfg.blockDimX = (unsigned)block_threads;
    cfg.blockDimY = cfg.blockDimZ = 1;
    cfg.sharedMemBytes = (unsigned)smem_bytes;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (d->occ_clusters(&clusters, f, &cfg) != CUDA_SUCCESS) return GSYNC_EINVAL;
    maxb = clusters * cluster;
  } else {
    int per_sm = 0, sms = 0;
    if (d->occ_blocks(&per_sm, f, block_threads, smem_bytes) != CUDA_SUCCESS) return GSYNC_EINVAL;
    if (int rc = device_sms(&sms)) return rc;
    maxb = per_sm * sms;
  }
  *max_blocks_out = maxb;
  return grid <= maxb ? GSYNC_OK : GSYNC_ENOTRESIDENT;
}

int gsync_launch_coresident(const void* kernel, int grid, int block_threads, size_t smem_bytes, int cluster,
                            void** args, void* stream) {
  int maxb = 0;
  if (int rc = gsync_check_coresident(kernel, grid, block_threads, smem_bytes, cluster, &maxb)) return rc;
  if (cluster > 1 && grid % cluster) return GSYNC_EINVAL;
  const DriverCalls* d = nullptr;
  if (int rc = driver_calls(&d)) return rc;
  CUlaunchAttribute attr[1];
  if (cluster > 1) {
    attr[0].id = CU_LAUNCH_ATTRIBUTE_CLUSTER_DIMENSION;
    attr[0].value.clusterDim.x = (unsigned)cluster;
    attr[0].value.clusterDim.y = 1;
    attr[0].value.clusterDim.z = 1;
  } else {
    attr[0].id = CU_LAUNCH_ATTRIBUTE_COOPERATIVE;
    attr[0].value.cooperative = 1;
  }
  CUlaunchConfig cfg = {};
  cfg.gridDimX = (unsigned)grid;
  cfg.gridDimY = cfg.gridDimZ = 1;
  cfg.blockDimX = (unsigned)block_threads;
  cfg.blockDimY = cfg.blockDimZ = 1;
  cfg.sharedMemBytes = (unsigned)smem_bytes;
  cfg.hStream = (CUstream)stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const CUresult r = d->launch(&cfg, (CUfunction)kernel, args, nullptr);
  if (r == CUDA_ERROR_COOPERATIVE_LAUNCH_TOO_LARGE) return GSYNC_ENOTRESIDENT;
  if (r != CUDA_SUCCESS) {
    g_last_cuda_error = (int)r;
    return GSYNC_ECUDA;
  }
  return GSYNC_OK;
}

int gsync_device_sm_count(int* sms_out) {
  if (!sms_out) return GSYNC_EINVAL;
  return device_sms(sms_out);
}

int gsync_max_coresident_blocks(int workload, int kind, int block_threads, int cluster, int* max_blocks_out) {
  if (!max_blocks_out || block_threads < 32 || block_threads > 256 || block_threads % 32) return GSYNC_EINVAL;
  switch (workload) {
    case 0: return max_blocks_barrier(kind, block_threads, cluster, max_blocks_out);
    case 1: return max_blocks_mutex(kind, block_threads, max_blocks_out);
    case 2: return max_blocks_sem(kind, block_threads, max_blocks_out);
  }
  return GSYNC_EINVAL;
}

}  // extern "C"
