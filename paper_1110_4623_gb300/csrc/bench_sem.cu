// Counting-semaphore workload (Section 6, "Results": each block runs a loop of wait/post
// pairs; Section 5: at most n blocks inside the critical section at once).
//
// Block b makes `pairs` wait/post pairs (id = b * pairs + p).  Inside, for hold[id] SM cycles
// from entry, thread 0 counts itself into `occupancy` with an atomic add, raises
// `max_occupancy` to its count (the capacity invariant, checked on the host), increments
// `total` with a plain load/store when n == 1 (exclusion makes it exact) and adds addend[id]
// to `tally` atomically; at the end of the hold it counts itself out of `occupancy`, then
// posts.
#include "common.cuh"

using namespace gsync_impl;

namespace {

constexpr int kMaxThreads = 256;

constexpr int kNoSem = -1;     // no semaphore at all: the critical-section probe
constexpr int kSemFrame = -2;  // the probe's frame around an empty critical section
// Cycles into the hold after which thread 0 does the section's bookkeeping: ~0.5 us at the
// 2.07 GHz clock, longer than an L2 round trip to a line on either die (0.2-0.4 us), so the
// values it needs have returned (a hold shorter than this does it at the hold's end).
constexpr uint32_t kBookkeepCycles = 1024;

// Spin until `cycles` SM cycles have passed since h0 (clock64 at the hold's start).
__device__ __forceinline__ void spin_until(long long h0, uint32_t cycles) {
  while (clock64() - h0 < (long long)cycles) {
  }
}

template <int KIND>
__global__ void __launch_bounds__(kMaxThreads, 8)
    sem_workload_kernel(uint32_t* state, int pairs, const uint32_t* __restrict__ hold,
                        const uint32_t* __restrict__ addend, uint32_t* occupancy, uint32_t* max_occupancy,
                        uint32_t* total, uint32_t* tally, uint32_t* count, uint32_t* status) {
  const uint32_t b = blockIdx.x, tid = threadIdx.x;
  gsync::SemRef s;
  if (KIND >= 0) {
    s = gsync::sem_attach(state);
    if (s.kind != (uint32_t)KIND) {
      if (tid == 0) gsync::ptx::atom_or_relaxed(status, GSYNC_STATUS_CONFIG);
      return;
    }
  } else {
    s.n = 1;
  }
  uint32_t done = 0;
  for (int p = 0; p < pairs; ++p) {
    const uint32_t id = b * (uint32_t)pairs + (uint32_t)p;
    // This pair's inputs are the block's own: read them before the wait, so that their loads
    // overlap it instead of lengthening the critical section.
    uint32_t hold_cycles = 0, add = 0;
    if (KIND != kSemFrame && tid == 0) {
      hold_cycles = hold ? hold[id] : 0u;
      add = addend[id];
    }
    int rc = GSYNC_OK;
    if (KIND >= 0) {
      rc = gsync::sem_wait<KIND>(s);
    } else {
      if (tid == 0) (void)gsync::ptx::ld_acquire(status + 32);
      __syncthreads();
    }
    if (rc != GSYNC_OK) {
      if (tid == 0) record_status(status, rc);
      break;
    }
    if (KIND != kSemFrame && tid == 0) {
      // The hold (hold[id] cycles from entry) starts at once.  n = 1: the plain read of total
      // goes out with the occupancy atomic, and their round trip overlaps the hold's first
      // kBookkeepCycles; then the running maximum, total's store and the tally go out
      // mid-hold, so that at the post only the occupancy decrement is still in flight.
      const long long h0 = clock64();
      const uint32_t t = s.n == 1u ? *total : 0u;
      const uint32_t o = gsync::ptx::atom_add_relaxed(occupancy, 1u) + 1u;
      spin_until(h0, min(hold_cycles, kBookkeepCycles));
      gsync::ptx::atom_max_relaxed(max_occupancy, o);
      if (s.n == 1u) *total = t + 1u;
      gsync::ptx::red_add_relaxed(tally, add);
      spin_until(h0, hold_cycles);
      gsync::ptx::atom_add_relaxed(occupancy, 0xFFFFFFFFu);
    }
    int rc2 = GSYNC_OK;
    if (KIND >= 0) {
      rc2 = gsync::sem_post<KIND>(s);
    } else {
      __syncthreads();
      if (tid == 0) {
        gsync::ptx::fence_acq_rel();
        gsync::ptx::st_relaxed(status + 32, id);
      }
    }
    if (rc2 != GSYNC_OK) {
      if (tid == 0) record_status(status, rc2);
      break;
    }
    ++done;
  }
  if (tid == 0) count[b] = done;
}

using KernelFn = void (*)(uint32_t*, int, const uint32_t*, const uint32_t*, uint32_t*, uint32_t*, uint32_t*,
                          uint32_t*, uint32_t*, uint32_t*);

KernelFn pick(int kind) {
  switch (kind) {
    case GSYNC_SEM_TICKET: return sem_workload_kernel<GSYNC_SEM_TICKET>;
    case GSYNC_SEM_SPIN: return sem_workload_kernel<GSYNC_SEM_SPIN>;
    case GSYNC_SEM_SPIN_BACKOFF: return sem_workload_kernel<GSYNC_SEM_SPIN_BACKOFF>;
    case GSYNC_SEM_WINDOW: return sem_workload_kernel<GSYNC_SEM_WINDOW>;
  }
  return nullptr;
}

}  // namespace

namespace gsync_impl {
int max_blocks_sem(int kind, int block_threads, int* out) {
  KernelFn k = pick(kind);
  if (!k) return GSYNC_EINVAL;
  return max_coresident(k, block_threads, 1, 0, out);
}
}  // namespace gsync_impl

extern "C" int gsync_bench_sem(void* state, const gsync_sem_work* w, void* stream) {
  if (!state || !w || !aligned(state, 128)) return GSYNC_EINVAL;
  if (w->nblocks < 1 || w->pairs < 0 || w->block_threads < 32 || w->block_threads > kMaxThreads ||
      w->block_threads % 32 || w->initial_count < 1)
    return GSYNC_EINVAL;
  if (!w->addend || !w->occupancy || !w->max_occupancy || !w->total || !w->tally || !w->count || !w->status)
    return GSYNC_EINVAL;
  KernelFn k = pick(w->kind);
  if (!k) return GSYNC_EINVAL;
  return launch_coresident(k, w->nblocks, w->block_threads, 1, 0, (cudaStream_t)stream, (uint32_t*)state, w->pairs,
                           w->hold, w->addend, w->occupancy, w->max_occupancy, w->total, w->tally, w->count,
                           w->status);
}

// Semaphore critical-section probe: one block runs the workload's wait/post frame without a
// semaphore (an acquire load and a barrier before, a barrier and a release after) around the
// critical section -- occupancy bookkeeping, hold[p] cycles, the tally -- for p < iters.
// out[0] = elapsed ns (CUDA events; synchronizes `stream`).  scratch: 1024 bytes.
extern "C" int gsync_probe_sem_cs(int block_threads, int iters, const uint32_t* hold, const uint32_t* addend,
                                  void* scratch, uint64_t* out, void* stream) {
  if (!scratch || !out || (!addend && hold) || iters < 1 || block_threads < 32 || block_threads > kMaxThreads ||
      block_threads % 32 || !aligned(scratch, 256))
    return GSYNC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t* w = (uint32_t*)scratch;
  GSYNC_CUDA(cudaMemsetAsync(scratch, 0, 1024, st));
  cudaEvent_t e0, e1;
  GSYNC_CUDA(cudaEventCreate(&e0));
  GSYNC_CUDA(cudaEventCreate(&e1));
  GSYNC_CUDA(cudaEventRecord(e0, st));
  if (hold == nullptr && addend == nullptr) {  // frame only
    sem_workload_kernel<kSemFrame><<<1, block_threads, 0, st>>>(nullptr, iters, nullptr, nullptr, w, w + 32, w + 64,
                                                                w + 96, w + 128, w + 160);
  } else {
    sem_workload_kernel<kNoSem><<<1, block_threads, 0, st>>>(nullptr, iters, hold, addend, w, w + 32, w + 64, w + 96,
                                                             w + 128, w + 160);
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
