// Condition-variable workload: a bounded producer/consumer queue of item ids under one
// mutex (TICKET, COHORT or CLUSTER) and two condition variables (condition variables are named as future work in
// Section 7; the design is in gsync_device.cuh).  Each item id is put once and must be taken
// exactly once: seen[] counts takes, and the consumers' int64 sums must add up to the sum of
// the items' values.
#include "common.cuh"

using namespace gsync_impl;
namespace ptx = gsync::ptx;

namespace {

constexpr int kMaxThreads = 256;

// The queue's bookkeeping, guarded by the mutex (plain accesses by the holder's thread 0, the
// whole struct in one 16-byte load and one 16-byte store: one L2 round trip per look).
struct __align__(16) Queue {
  uint32_t count, head, tail, capacity;
};

template <int MKIND>
__global__ void __launch_bounds__(kMaxThreads)
    condvar_workload_kernel(uint32_t* mutex_state, uint32_t* nf_state, uint32_t* ne_state, Queue* q, uint32_t* buf,
                            int producers, int items_per_producer, int items_per_consumer,
                            const uint32_t* __restrict__ value, uint32_t* seen, int64_t* sum, uint32_t* count,
                            uint32_t* status, uint32_t* acquisitions) {
  gsync::MutexRef m;
  if (MKIND == GSYNC_MUTEX_CLUSTER) {
    __shared__ gsync::ClusterLocal cluster_lock;
    m = gsync::mutex_attach_cluster(mutex_state, &cluster_lock);
  } else if (MKIND == GSYNC_MUTEX_CLUSTER_MCS) {
    __shared__ gsync::McsNode node;
    m = gsync::mutex_attach_cluster_mcs(mutex_state, &node);
  } else {
    m = gsync::mutex_attach(mutex_state);
  }
  const gsync::CondRef not_full = gsync::cond_attach(nf_state), not_empty = gsync::cond_attach(ne_state);
  const bool producer = (int)blockIdx.x < producers;
  const int ops = producer ? items_per_producer : items_per_consumer;
  const bool t0 = threadIdx.x == 0;
  __shared__ int s_ok;
  __shared__ uint32_t s_id;
  Queue qv = {0u, 0u, 0u, 1u};  // thread 0's copy of *q while it holds the mutex
  // ... and of the counters of the condition variable it signals (taken in the same round trip)
  const gsync::CondRef& to_signal = producer ? not_empty : not_full;
  gsync::CondSnap snap = {0u, 0u};
  int64_t my_sum = 0;
  uint32_t taken = 0;
  for (int i = 0; i < ops; ++i) {
    gsync::Token tok = gsync::mutex_lock<MKIND>(m);
    if (tok.status != GSYNC_OK) {
      if (t0) record_status(status, tok.status);
      break;
    }
    // Acquisitions of the mutex in this round (the lock, and one per wait that takes it again),
    // counted after the unlock so that the release does not wait for the count's store.
    uint32_t acq_round = 1u;
    // wait while the buffer is full (producer) or empty (consumer); re-test after each wake
    int rc = GSYNC_OK;
    for (;;) {
      if (t0) {
        snap = gsync::cond_snapshot_thread(to_signal);
        qv = *q;
        s_ok = producer ? qv.count < qv.capacity : qv.count > 0u;
      }
      __syncthreads();
      if (s_ok) break;
      rc = gsync::cond_wait<MKIND>(producer ? not_full : not_empty, m, tok);
      if (rc != GSYNC_OK) break;
      ++acq_round;  // the wait took the mutex again
    }
    if (rc != GSYNC_OK) {
      if (t0) {
        record_status(status, rc);
        if (acquisitions) ptx::red_add_relaxed(acquisitions, acq_round);
      }
      break;  // the mutex is not held after a failed wait
    }
    if (t0) {
      if (producer) {
        const uint32_t id = blockIdx.x * (uint32_t)items_per_producer + (uint32_t)i;
        buf[qv.tail % qv.capacity] = id;
        *q = Queue{qv.count + 1u, qv.head, qv.tail + 1u, qv.capacity};
        gsync::cond_signal_thread(not_empty, snap);
      } else {
        s_id = buf[qv.head % qv.capacity];
        *q = Queue{qv.count - 1u, qv.head + 1u, qv.tail, qv.capacity};
        gsync::cond_signal_thread(not_full, snap);
      }
    }
    gsync::mutex_unlock<MKIND>(m, tok);
    if (t0 && acquisitions) ptx::red_add_relaxed(acquisitions, acq_round);
    if (!producer && t0) {
      const uint32_t id = s_id;
      if (id < (uint32_t)(producers * items_per_producer)) {
        atomicAdd(seen + id, 1u);
        my_sum += (int64_t)(int32_t)value[id];
        ++taken;
      } else {
        ptx::atom_or_relaxed(status, GSYNC_STATUS_VIOLATION);
      }
    }
  }
  if (!producer && t0) {
    const uint32_t c = blockIdx.x - (uint32_t)producers;
    sum[c] = my_sum;
    count[c] = taken;
  }
  // the cluster's shared memory (block 0's lock, or every block's node) outlives every user
  if (MKIND == GSYNC_MUTEX_CLUSTER || MKIND == GSYNC_MUTEX_CLUSTER_MCS) gsync::mutex_cluster_end();
}

size_t round_up(size_t n) { return (n + 255) & ~(size_t)255; }

// Critical-section probe of the queue (the roofline's T_cs for the condition-variable
// workload): one block alternates a put and a take, each the workload's critical section --
// the test of the queue under block barriers, the slot and the queue's state, the signal --
// framed like a hand-off (an acquire load and a barrier before, a barrier and a release store
// after), with no mutex and no waits.  frame_only runs the frame around an empty body.
__global__ void __launch_bounds__(kMaxThreads)
    condvar_cs_probe_kernel(uint32_t* nf_state, uint32_t* ne_state, Queue* q, uint32_t* buf, int iters, int frame_only,
                            uint32_t* word) {
  const gsync::CondRef not_full = gsync::cond_attach(nf_state), not_empty = gsync::cond_attach(ne_state);
  const bool t0 = threadIdx.x == 0;
  __shared__ int s_ok;
  __shared__ uint32_t s_id;
  Queue qv = {0u, 0u, 0u, 1u};
  uint32_t acc = 0;
  if (t0) s_id = 0;
  for (int i = 0; i < iters; ++i) {
    if (t0) (void)ptx::ld_acquire(word);
    __syncthreads();
    const bool put = (i & 1) == 0;
    if (!frame_only) {
      gsync::CondSnap snap = {0u, 0u};
      if (t0) {
        snap = gsync::cond_snapshot_thread(put ? not_empty : not_full);
        qv = *q;
        s_ok = put ? qv.count < qv.capacity : qv.count > 0u;
      }
      __syncthreads();
      if (t0 && s_ok) {
        if (put) {
          buf[qv.tail % qv.capacity] = (uint32_t)i;
          *q = Queue{qv.count + 1u, qv.head, qv.tail + 1u, qv.capacity};
          gsync::cond_signal_thread(not_empty, snap);
        } else {
          s_id = buf[qv.head % qv.capacity];
          *q = Queue{qv.count - 1u, qv.head + 1u, qv.tail, qv.capacity};
          gsync::cond_signal_thread(not_full, snap);
        }
      }
    }
    __syncthreads();
    if (t0) {
      acc += s_id;
      ptx::st_release(word, (uint32_t)i);
    }
  }
  if (t0 && acc == 0xFFFFFFFFu) word[1] = acc;  // keeps the taken ids live
}

}  // namespace

// The mutex sits first in the workspace and takes the largest of the kinds' sizes.
size_t mutex_region() {
  size_t n = 0;
  for (int kind : {GSYNC_MUTEX_TICKET, GSYNC_MUTEX_COHORT, GSYNC_MUTEX_CLUSTER, GSYNC_MUTEX_CLUSTER_MCS}) {
    const size_t k = gsync_mutex_bytes(kind, 1);
    n = k > n ? k : n;
  }
  return round_up(n);
}

extern "C" size_t gsync_bench_condvar_workspace_bytes(int capacity) {
  if (capacity < 1 || capacity > (1 << 24)) return 0;
  return mutex_region() + 2 * round_up(gsync_cond_bytes()) + round_up(sizeof(Queue)) +
         round_up(4 * (size_t)capacity);
}

extern "C" int gsync_bench_condvar(const gsync_condvar_work* w, const gsync_backoff* backoff, void* workspace,
                                   size_t workspace_bytes, void* stream) {
  if (!w || w->producers < 1 || w->consumers < 1 || w->items_per_producer < 0 || w->capacity < 1 ||
      w->block_threads < 32 || w->block_threads > kMaxThreads || w->block_threads % 32)
    return GSYNC_EINVAL;
  const int64_t items = (int64_t)w->producers * w->items_per_producer;
  if (items > (1ll << 30) || items % w->consumers) return GSYNC_EINVAL;
  if (!w->value || !w->seen || !w->sum || !w->count || !w->status) return GSYNC_EINVAL;
  const bool clustered = w->mutex_kind == GSYNC_MUTEX_CLUSTER || w->mutex_kind == GSYNC_MUTEX_CLUSTER_MCS;
  if (w->mutex_kind != GSYNC_MUTEX_TICKET && w->mutex_kind != GSYNC_MUTEX_COHORT && !clustered) return GSYNC_EINVAL;
  const int cluster = !clustered ? 1 : w->cluster ? w->cluster : 4;
  if ((clustered && (cluster < 2 || cluster > 8)) || (w->producers + w->consumers) % cluster) return GSYNC_EINVAL;
  const size_t need = gsync_bench_condvar_workspace_bytes(w->capacity);
  if (need == 0 || !workspace || workspace_bytes < need || !aligned(workspace, 256)) return GSYNC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  char* p = (char*)workspace;
  uint32_t* mstate = (uint32_t*)p;  p += mutex_region();
  uint32_t* nf = (uint32_t*)p;      p += round_up(gsync_cond_bytes());
  uint32_t* ne = (uint32_t*)p;      p += round_up(gsync_cond_bytes());
  Queue* q = (Queue*)p;             p += round_up(sizeof(Queue));
  uint32_t* buf = (uint32_t*)p;
  const uint64_t timeout_ns = 10000000000ull;
  if (int rc = gsync_mutex_init(mstate, gsync_mutex_bytes(w->mutex_kind, 1), w->mutex_kind, 1, backoff, timeout_ns,
                                stream))
    return rc;
  if (int rc = gsync_cond_init(nf, gsync_cond_bytes(), backoff, timeout_ns, stream)) return rc;
  if (int rc = gsync_cond_init(ne, gsync_cond_bytes(), backoff, timeout_ns, stream)) return rc;
  const Queue q0 = {0u, 0u, 0u, (uint32_t)w->capacity};
  GSYNC_CUDA(cudaMemcpyAsync(q, &q0, sizeof q0, cudaMemcpyHostToDevice, st));
  GSYNC_CUDA(cudaStreamSynchronize(st));  // q0 lives on this stack frame
  const int items_per_consumer = (int)(items / w->consumers);
  auto kernel = w->mutex_kind == GSYNC_MUTEX_COHORT        ? condvar_workload_kernel<GSYNC_MUTEX_COHORT>
                : w->mutex_kind == GSYNC_MUTEX_CLUSTER     ? condvar_workload_kernel<GSYNC_MUTEX_CLUSTER>
                : w->mutex_kind == GSYNC_MUTEX_CLUSTER_MCS ? condvar_workload_kernel<GSYNC_MUTEX_CLUSTER_MCS>
                                                           : condvar_workload_kernel<GSYNC_MUTEX_TICKET>;
  return launch_coresident(kernel, w->producers + w->consumers, w->block_threads, cluster, 0, st, mstate, nf, ne, q, buf,
                           w->producers, w->items_per_producer, items_per_consumer, w->value, w->seen, w->sum,
                           w->count, w->status, w->acquisitions);
}

// T_cs probe of the condition-variable queue: see condvar_cs_probe_kernel.  workspace as for
// gsync_bench_condvar (capacity 16 is enough); out[0] (host) = elapsed ns for `iters` critical
// sections.  Synchronizes `stream`.
extern "C" int gsync_probe_condvar_cs(int block_threads, int iters, int frame_only, void* workspace,
                                      size_t workspace_bytes, uint64_t* out, void* stream) {
  if (!out || iters < 1 || block_threads < 32 || block_threads > kMaxThreads || block_threads % 32) return GSYNC_EINVAL;
  const size_t need = gsync_bench_condvar_workspace_bytes(16);
  if (!workspace || workspace_bytes < need || !aligned(workspace, 256)) return GSYNC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  char* p = (char*)workspace;
  uint32_t* word = (uint32_t*)p;    p += mutex_region();  // the frame's acquire/release word
  uint32_t* nf = (uint32_t*)p;      p += round_up(gsync_cond_bytes());
  uint32_t* ne = (uint32_t*)p;      p += round_up(gsync_cond_bytes());
  Queue* q = (Queue*)p;             p += round_up(sizeof(Queue));
  uint32_t* buf = (uint32_t*)p;
  if (int rc = gsync_cond_init(nf, gsync_cond_bytes(), nullptr, 1000000000ull, stream)) return rc;
  if (int rc = gsync_cond_init(ne, gsync_cond_bytes(), nullptr, 1000000000ull, stream)) return rc;
  const Queue q0 = {0u, 0u, 0u, 16u};
  GSYNC_CUDA(cudaMemcpyAsync(q, &q0, sizeof q0, cudaMemcpyHostToDevice, st));
  GSYNC_CUDA(cudaMemsetAsync(word, 0, 256, st));
  cudaEvent_t e0, e1;
  GSYNC_CUDA(cudaEventCreate(&e0));
  GSYNC_CUDA(cudaEventCreate(&e1));
  GSYNC_CUDA(cudaEventRecord(e0, st));
  condvar_cs_probe_kernel<<<1, block_threads, 0, st>>>(nf, ne, q, buf, iters, frame_only, word);
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
