// Mutex workload (Section 6, "Results": each block runs a loop of lock/unlock pairs).
//
// Block b makes `acq` acquisitions (id = b * acq + a).  Before each lock its master thread
// waits delay[id] SM cycles; inside the critical section thread 0 reads `total` (the grant's
// position) and increments it with a plain load and store, and the block's threads add
// addend[id] ^ (i * 0x9E3779B1) to data[i] for i < cs_words with plain loads and stores.
// After the unlock thread 0 writes id into the grant log at that position.  Broken exclusion
// loses updates to total/data or repeats a position in the log; the fair kinds also record
// their ticket so the host can check grants follow ticket order (the cohort lock: each die's
// grants follow that die's tickets).
#include "common.cuh"

using namespace gsync_impl;

namespace {

constexpr int kMaxThreads = 256;
constexpr int kNoLock = -1;     // no mutex at all: the critical-section probe (T_cs)
constexpr int kFrameOnly = -2;  // the probe's frame (acquire load, barriers, release) around an empty body
constexpr uint32_t kGolden = 0x9E3779B1u;

// The critical section's data update: data[i] += v ^ (i * kGolden) for i < cs_words, word i on
// thread i mod blockDim.  cs_load issues a thread's first loads -- one word, or up to
// kCsInFlight of them for a section wider than the block (WIDE) -- before thread 0's own
// bookkeeping (the read and write of total), so that thread 0 waits for one L2 round trip, not two;
// cs_store finishes them, and a WIDE section's further passes keep kCsInFlight loads per thread
// in flight.  Narrow sections run in a kernel of their own.
constexpr int kCsInFlight = 4;
template <bool WIDE>
__device__ __forceinline__ void cs_load(const uint32_t* data, uint32_t cs_words, uint32_t (&x)[kCsInFlight]) {
#pragma unroll
  for (int k = 0; k < (WIDE ? kCsInFlight : 1); ++k) {
    const uint32_t j = threadIdx.x + k * blockDim.x;
    x[k] = j < cs_words ? data[j] : 0u;
  }
}
template <bool WIDE>
__device__ __forceinline__ void cs_store(uint32_t* data, uint32_t cs_words, uint32_t v, uint32_t (&x)[kCsInFlight]) {
#pragma unroll
  for (int k = 0; k < (WIDE ? kCsInFlight : 1); ++k) {
    const uint32_t j = threadIdx.x + k * blockDim.x;
    if (j < cs_words) data[j] = x[k] + (v ^ (j * kGolden));
  }
  if (!WIDE) return;
  const uint32_t step = blockDim.x * kCsInFlight;
  for (uint32_t base = threadIdx.x + step; base < cs_words; base += step) {
    uint32_t y[kCsInFlight];
#pragma unroll
    for (int k = 0; k < kCsInFlight; ++k) {
      const uint32_t j = base + k * blockDim.x;
      y[k] = j < cs_words ? data[j] : 0u;
    }
#pragma unroll
    for (int k = 0; k < kCsInFlight; ++k) {
      const uint32_t j = base + k * blockDim.x;
      if (j < cs_words) data[j] = y[k] + (v ^ (j * kGolden));
    }
  }
}

template <int KIND, bool WIDE>
__global__ void __launch_bounds__(kMaxThreads, 8)
    mutex_workload_kernel(uint32_t* state, int acq, int cs_words, const uint32_t* __restrict__ delay,
                          const uint32_t* __restrict__ addend, uint32_t* data, uint32_t* total, uint32_t* grant_log,
                          uint32_t* ticket_out, uint32_t* count, uint32_t* status) {
  const uint32_t b = blockIdx.x, tid = threadIdx.x;
  const uint32_t n = gridDim.x * (uint32_t)acq;
  gsync::MutexRef m;
  if (KIND == GSYNC_MUTEX_CLUSTER) {
    __shared__ gsync::ClusterLocal cluster_lock;
    m = gsync::mutex_attach_cluster(state, &cluster_lock);
  } else if (KIND == GSYNC_MUTEX_CLUSTER_MCS) {
    __shared__ gsync::McsNode node;
    m = gsync::mutex_attach_cluster_mcs(state, &node);
  } else if (KIND >= 0) {
    m = gsync::mutex_attach(state);
  }
  if (KIND >= 0) {
    const bool bad_queue =
        (KIND == GSYNC_MUTEX_SLEEP_QUEUE || KIND == GSYNC_MUTEX_RING) && gridDim.x > m.qmask + 1u;
    if (m.kind != (uint32_t)KIND || bad_queue) {
      if (tid == 0) gsync::ptx::atom_or_relaxed(status, GSYNC_STATUS_CONFIG);
      return;
    }
  }
  uint32_t done = 0;
  for (int a = 0; a < acq; ++a) {
    const uint32_t id = b * (uint32_t)acq + (uint32_t)a;
    const uint32_t v = addend[id];
    if (tid == 0 && delay) spin_cycles(delay[id]);
    gsync::Token t{GSYNC_OK, 0xFFFFFFFFu};
    if (KIND >= 0) {
      t = gsync::mutex_lock<KIND>(m);
      if (t.status != GSYNC_OK) {
        if (tid == 0) record_status(status, t.status);
        break;
      }
    } else {
      // What a lock adds around the body even uncontended: one acquire load, one block barrier.
      if (tid == 0) (void)gsync::ptx::ld_acquire(status + 32);
      __syncthreads();
    }
    // ---- critical section ----
    uint32_t x[kCsInFlight];
    if (KIND != kFrameOnly) cs_load<WIDE>(data, (uint32_t)cs_words, x);  // data and total never overlap
    uint32_t seq = 0;
    if (KIND != kFrameOnly && tid == 0) {
      seq = *total;
      *total = seq + 1u;
    }
    if (KIND != kFrameOnly) cs_store<WIDE>(data, (uint32_t)cs_words, v, x);
    // ---- end of critical section ----
    if (KIND >= 0) {
      gsync::mutex_unlock<KIND>(m, t);
    } else {
      __syncthreads();
      if (tid == 0) gsync::ptx::st_release(status + 32, id);  // the release store of an unlock
    }
    // The grant log and the ticket record are this acquisition's own slots, which only the
    // host reads after the launch: written after the release, their stores' acknowledgements
    // stay off the hand-off path (the release waits only for the section's own stores).
    if (KIND != kFrameOnly && tid == 0) {
      if (seq < n) {
        grant_log[seq] = id;
      } else {
        gsync::ptx::atom_or_relaxed(status, GSYNC_STATUS_VIOLATION);
      }
      // COHORT: tickets are per die; bit 31 records the die so the host can check each
      // die's grants in ticket order.  CLUSTER_MCS has no cluster-wide ticket (its queue order
      // is the order of the tail swaps): it records none.
      ticket_out[id] = KIND == GSYNC_MUTEX_COHORT        ? (m.die << 31) | (t.ticket & 0x7FFFFFFFu)
                       : KIND == GSYNC_MUTEX_CLUSTER     ? ((b / gsync::ptx::cluster_nctarank()) << 20) | (t.ticket & 0xFFFFFu)
                       : KIND == GSYNC_MUTEX_CLUSTER_MCS ? 0xFFFFFFFFu
                                                         : t.ticket;
    }
    ++done;
  }
  if (tid == 0) count[b] = done;
  // the cluster's shared memory (block 0's lock, or every block's node) outlives every user
  if (KIND == GSYNC_MUTEX_CLUSTER || KIND == GSYNC_MUTEX_CLUSTER_MCS) gsync::mutex_cluster_end();
}

using KernelFn = void (*)(uint32_t*, int, int, const uint32_t*, const uint32_t*, uint32_t*, uint32_t*, uint32_t*,
                          uint32_t*, uint32_t*, uint32_t*);

template <bool WIDE>
KernelFn pick_width(int kind) {
  switch (kind) {
    case GSYNC_MUTEX_CAS_SPIN: return mutex_workload_kernel<GSYNC_MUTEX_CAS_SPIN, WIDE>;
    case GSYNC_MUTEX_CAS_BACKOFF: return mutex_workload_kernel<GSYNC_MUTEX_CAS_BACKOFF, WIDE>;
    case GSYNC_MUTEX_TICKET: return mutex_workload_kernel<GSYNC_MUTEX_TICKET, WIDE>;
    case GSYNC_MUTEX_SLEEP_QUEUE: return mutex_workload_kernel<GSYNC_MUTEX_SLEEP_QUEUE, WIDE>;
    case GSYNC_MUTEX_COHORT: return mutex_workload_kernel<GSYNC_MUTEX_COHORT, WIDE>;
    case GSYNC_MUTEX_RING: return mutex_workload_kernel<GSYNC_MUTEX_RING, WIDE>;
    case GSYNC_MUTEX_CLUSTER: return mutex_workload_kernel<GSYNC_MUTEX_CLUSTER, WIDE>;
    case GSYNC_MUTEX_CLUSTER_MCS: return mutex_workload_kernel<GSYNC_MUTEX_CLUSTER_MCS, WIDE>;
  }
  return nullptr;
}

// A critical section wider than the block runs in the kernel that batches its loads.
KernelFn pick(int kind, bool wide) { return wide ? pick_width<true>(kind) : pick_width<false>(kind); }

int check_work(const gsync_mutex_work* w) {
  if (!w || w->nblocks < 1 || w->acq < 0 || w->cs_words < 0 || w->block_threads < 32 ||
      w->block_threads > kMaxThreads || w->block_threads % 32)
    return GSYNC_EINVAL;
  if ((uint64_t)w->nblocks * (uint64_t)w->acq >= (1ull << 31)) return GSYNC_EINVAL;
  if (w->kind == GSYNC_MUTEX_CLUSTER || w->kind == GSYNC_MUTEX_CLUSTER_MCS) {
    // cluster ids and tickets must fit the recorded (cluster << 20) | ticket
    if (w->cluster < 2 || w->cluster > 8 || w->nblocks % w->cluster || w->nblocks / w->cluster > 4096 ||
        (uint64_t)w->cluster * (uint64_t)w->acq >= (1ull << 20))
      return GSYNC_EINVAL;
  } else if (w->cluster > 1) {
    return GSYNC_EINVAL;
  }
  return GSYNC_OK;
}

int launch_cluster(const gsync_mutex_work* w) {
  return w->kind == GSYNC_MUTEX_CLUSTER || w->kind == GSYNC_MUTEX_CLUSTER_MCS ? w->cluster : 1;
}

size_t round_up(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

namespace gsync_impl {
int max_blocks_mutex(int kind, int block_threads, int* out) {
  // both widths must fit: the grid limit is the smaller of the two
  KernelFn kn = pick(kind, false), kw = pick(kind, true);
  if (!kn || !kw) return GSYNC_EINVAL;
  int n_narrow = 0, n_wide = 0;
  if (int rc = max_coresident(kn, block_threads, 1, 0, &n_narrow)) return rc;
  if (int rc = max_coresident(kw, block_threads, 1, 0, &n_wide)) return rc;
  *out = n_narrow < n_wide ? n_narrow : n_wide;
  return GSYNC_OK;
}
}  // namespace gsync_impl

extern "C" int gsync_bench_mutex(void* state, const gsync_mutex_work* w, void* stream) {
  if (int rc = check_work(w)) return rc;
  if (!state || !aligned(state, 128)) return GSYNC_EINVAL;
  if (!w->addend || !w->total || !w->grant_log || !w->ticket || !w->count || !w->status ||
      (w->cs_words > 0 && !w->data))
    return GSYNC_EINVAL;
  KernelFn k = pick(w->kind, w->cs_words > w->block_threads);
  if (!k) return GSYNC_EINVAL;
  return launch_coresident(k, w->nblocks, w->block_threads, launch_cluster(w), 0, (cudaStream_t)stream,
                           (uint32_t*)state, w->acq,
                           w->cs_words, w->delay, w->addend, w->data, w->total, w->grant_log, w->ticket, w->count,
                           w->status);
}

extern "C" size_t gsync_bench_mutex_workspace_bytes(int kind, int nblocks, int acq, int cs_words) {
  const size_t sb = gsync_mutex_bytes(kind, nblocks);
  if (sb == 0 || nblocks < 1 || acq < 0 || cs_words < 0) return 0;
  const size_t n = (size_t)nblocks * (size_t)acq;
  return round_up(sb) + 4 * round_up(4 * n) + round_up(4 * (size_t)cs_words) + round_up(4 * (size_t)nblocks) +
         2 * round_up(4);
}

extern "C" int gsync_bench_mutex_host(const gsync_mutex_work* w, const gsync_backoff* backoff, void* workspace,
                                      size_t workspace_bytes, void* stream) {
  if (int rc = check_work(w)) return rc;
  const size_t need = gsync_bench_mutex_workspace_bytes(w->kind, w->nblocks, w->acq, w->cs_words);
  if (need == 0 || !workspace || workspace_bytes < need || !aligned(workspace, 256)) return GSYNC_EINVAL;
  if (!w->addend || !w->total || !w->grant_log || !w->ticket || !w->count || !w->status ||
      (w->cs_words > 0 && !w->data))
    return GSYNC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = (size_t)w->nblocks * (size_t)w->acq;
  char* p = (char*)workspace;
  const size_t sb = gsync_mutex_bytes(w->kind, w->nblocks);
  void* state = p;                 p += round_up(sb);
  uint32_t* d_delay = (uint32_t*)p;  p += round_up(4 * n);
  uint32_t* d_add = (uint32_t*)p;    p += round_up(4 * n);
  uint32_t* d_log = (uint32_t*)p;    p += round_up(4 * n);
  uint32_t* d_tick = (uint32_t*)p;   p += round_up(4 * n);
  uint32_t* d_data = (uint32_t*)p;   p += round_up(4 * (size_t)w->cs_words);
  uint32_t* d_count = (uint32_t*)p;  p += round_up(4 * (size_t)w->nblocks);
  uint32_t* d_total = (uint32_t*)p;  p += round_up(4);
  uint32_t* d_status = (uint32_t*)p; p += round_up(4);

  if (w->delay) GSYNC_CUDA(cudaMemcpyAsync(d_delay, w->delay, 4 * n, cudaMemcpyHostToDevice, st));
  GSYNC_CUDA(cudaMemcpyAsync(d_add, w->addend, 4 * n, cudaMemcpyHostToDevice, st));
  if (w->cs_words) GSYNC_CUDA(cudaMemsetAsync(d_data, 0, 4 * (size_t)w->cs_words, st));
  GSYNC_CUDA(cudaMemsetAsync(d_total, 0, 4, st));
  GSYNC_CUDA(cudaMemsetAsync(d_status, 0, 4, st));
  if (int rc = gsync_mutex_init(state, sb, w->kind, w->nblocks, backoff, 0, stream)) return rc;
  gsync_mutex_work dw = *w;
  dw.delay = w->delay ? d_delay : nullptr;
  dw.addend = d_add;
  dw.data = d_data;
  dw.total = d_total;
  dw.grant_log = d_log;
  dw.ticket = d_tick;
  dw.count = d_count;
  dw.status = d_status;
  if (int rc = gsync_bench_mutex(state, &dw, stream)) return rc;
  if (w->cs_words) GSYNC_CUDA(cudaMemcpyAsync(w->data, d_data, 4 * (size_t)w->cs_words, cudaMemcpyDeviceToHost, st));
  GSYNC_CUDA(cudaMemcpyAsync(w->total, d_total, 4, cudaMemcpyDeviceToHost, st));
  GSYNC_CUDA(cudaMemcpyAsync(w->grant_log, d_log, 4 * n, cudaMemcpyDeviceToHost, st));
  GSYNC_CUDA(cudaMemcpyAsync(w->ticket, d_tick, 4 * n, cudaMemcpyDeviceToHost, st));
  GSYNC_CUDA(cudaMemcpyAsync(w->count, d_count, 4 * (size_t)w->nblocks, cudaMemcpyDeviceToHost, st));
  GSYNC_CUDA(cudaMemcpyAsync(w->status, d_status, 4, cudaMemcpyDeviceToHost, st));
  GSYNC_CUDA(cudaStreamSynchronize(st));
  return GSYNC_OK;
}

// T_cs probe: one block runs the critical-section body, framed like a lock hand-off (an
// acquire load and a barrier before it, a barrier and the release store after it), `iters`
// times with no lock and no delays.  scratch: [0, 128) status and the
// release word (status + 32), then total, data, count, grant log.
extern "C" int gsync_probe_cs(int cs_words, int block_threads, int iters, void* scratch, uint64_t* out,
                              void* stream) {
  if (!scratch || !out || cs_words < -1 || iters < 1 || block_threads < 32 || block_threads > kMaxThreads ||
      block_threads % 32 || !aligned(scratch, 256))
    return GSYNC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  char* p = (char*)scratch;
  uint32_t* status = (uint32_t*)p;   p += 256;
  uint32_t* total = (uint32_t*)p;    p += 256;
  uint32_t* count = (uint32_t*)p;    p += 256;
  uint32_t* data = (uint32_t*)p;     p += round_up(4 * (size_t)(cs_words > 0 ? cs_words : 0));
  uint32_t* log = (uint32_t*)p;      p += round_up(4 * (size_t)iters);
  uint32_t* tick = (uint32_t*)p;     p += round_up(4 * (size_t)iters);
  uint32_t* add = (uint32_t*)p;      p += round_up(4 * (size_t)iters);
  const size_t bytes = (size_t)(p - (char*)scratch);
  GSYNC_CUDA(cudaMemsetAsync(scratch, 0, bytes, st));
  cudaEvent_t e0, e1;
  GSYNC_CUDA(cudaEventCreate(&e0));
  GSYNC_CUDA(cudaEventCreate(&e1));
  GSYNC_CUDA(cudaEventRecord(e0, st));
  if (cs_words < 0) {  // frame only: the acquire load, barriers and release store, no body
    mutex_workload_kernel<kFrameOnly, false><<<1, block_threads, 0, st>>>(nullptr, iters, 0, nullptr, add, data, total, log,
                                                                  tick, count, status);
  } else if (cs_words > block_threads) {  // the same body, and the same width, as the workload's
    mutex_workload_kernel<kNoLock, true><<<1, block_threads, 0, st>>>(nullptr, iters, cs_words, nullptr, add, data,
                                                                     total, log, tick, count, status);
  } else {
    mutex_workload_kernel<kNoLock, false><<<1, block_threads, 0, st>>>(nullptr, iters, cs_words, nullptr, add, data,
                                                                      total, log, tick, count, status);
  }
  GSYNC_CUDA(cudaGetLastError());
  GSYNC_CUDA(cudaEventRecord(e1, st));
  GSYNC_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  GSYNC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  out[0] = (uint64_t)(ms * 1e6);
  return GSYNC_OK;
}

// Size of the scratch buffer gsync_probe_cs needs.
extern "C" size_t gsync_probe_cs_scratch_bytes(int cs_words, int iters) {
  if (cs_words < -1 || iters < 1) return 0;
  return 3 * 256 + round_up(4 * (size_t)(cs_words > 0 ? cs_words : 0)) + 3 * round_up(4 * (size_t)iters);
}
