// Barrier workload (Section 6, "Results": one kernel, a loop of global barriers per block).
//
// Round r: block b writes slot[(r & 1) * B + b] = r * B + b, crosses the barrier, then reads
// slots of the same half.  Double-buffering by round parity makes one barrier per round
// enough: a block can only overwrite half (r & 1) again in round r + 2, after crossing
// barrier r + 1, which every block reaches only after finishing its round-r reads.
//   full    : every slot is read by the block's threads; the block records the XOR of the
//             slots (chk), folds the sum of their lowbias32 hashes into mix, and counts slots
//             that do not hold this round's value (bad).
//   sampled : thread 0 reads partner p = (b + r + 1) mod B only, folds lowbias32(slot_p) into
//             mix and counts a stale read in bad.  This keeps the per-round work O(1) so the
//             kernel time measures the barrier itself at large grids.
// EXCHANGE carries each block's slot value in its arrival instead: the block publishes r * B + b
// with barrier_exchange and reads the others' values with barrier_exchange_read (the slot
// buffers are not used); the results are the same.
#include "common.cuh"

using namespace gsync_impl;

namespace {

constexpr int kMaxThreads = 256;

// Register budget: the full-fold variant reduces three values per round (64 registers); the
// sampled variant's flag gather keeps two 16-byte vectors in flight (42 registers).  Both
// still fit 8 blocks of 128 threads per SM, the shape of the 1184-block workloads.
template <int KIND, bool FULL, bool TRACE = false>
__global__ void __launch_bounds__(kMaxThreads, FULL ? 4 : 6)
    barrier_workload_kernel(uint32_t* state, int rounds, uint32_t* slots, uint32_t* chk, uint32_t* mix_out,
                            uint32_t* bad_out, uint32_t* status, uint64_t* trace = nullptr) {
  gsync::BarrierRef bar = gsync::barrier_attach(state);
  const uint32_t B = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  if (bar.kind != (uint32_t)KIND || bar.n != B ||
      (KIND == GSYNC_BAR_CLUSTER && gsync::ptx::cluster_nctarank() != (bar.param & 0xFu))) {
    if (tid == 0) gsync::ptx::atom_or_relaxed(status, GSYNC_STATUS_CONFIG);
    return;  // uniform: every block sees the same header
  }
  __shared__ uint32_t red_x[kMaxThreads / 32], red_s[kMaxThreads / 32], red_b[kMaxThreads / 32];
  uint32_t mix = 0, bad = 0;
  constexpr bool kExchange = KIND == GSYNC_BAR_EXCHANGE;
  // The value of slot j this round: the slot buffer, or block j's exchange record.
  auto slot = [&](const uint32_t* buf, uint32_t j, uint32_t& nb) -> uint32_t {
    if constexpr (kExchange) {
      uint64_t v = 0;
      if (gsync::barrier_exchange_read(bar, j, v) != GSYNC_OK) {
        ++nb;
        return 0xFFFFFFFFu;
      }
      return (uint32_t)v;
    } else {
      return buf[j];
    }
  };
  // Sampled fold with slot buffers: the partner read of round r is folded in round r + 1,
  // after that round's slot store has been issued, so the read's round trip and the store's
  // acknowledgement (which the next arrival's release waits for) overlap instead of following
  // one another.  The read is still ordered before the next arrival by that release, so no
  // block can overwrite the slot before it is read.
  constexpr bool kDeferFold = !FULL && !kExchange;
  uint32_t pend_v = 0, pend_want = 0;
  bool pend = false;
  for (int r = 0; r < rounds; ++r) {
    uint32_t* buf = slots + (uint32_t)(r & 1) * B;
    const uint32_t rb = (uint32_t)r * B;
    if (!kExchange && tid == 0) buf[b] = rb + b;
    if (kDeferFold && tid == 0 && pend) {
      mix = rotl32(mix, 5) ^ lowbias32(pend_v);
      bad += pend_v != pend_want;
      pend = false;
    }
    if (TRACE && tid == 0) trace[2u * ((uint64_t)b * (uint32_t)rounds + (uint32_t)r)] = gsync::ptx::globaltimer();
    int rc;
    if constexpr (kExchange) {
      rc = gsync::barrier_exchange(bar, rb + b);
    } else {
      rc = gsync::barrier_wait<KIND>(bar);
    }
    if (TRACE && tid == 0) trace[2u * ((uint64_t)b * (uint32_t)rounds + (uint32_t)r) + 1u] = gsync::ptx::globaltimer();
    if (rc != GSYNC_OK) {
      if (tid == 0) record_status(status, rc);
      // The hardware cluster barrier has no timeout: every block of a cluster must keep
      // crossing for all rounds, or a peer would wait forever.  After a failure the object's
      // abort word makes each later crossing return within a few polls.
      if (KIND != GSYNC_BAR_CLUSTER) break;
      continue;
    }
    if (FULL) {
      uint32_t x = 0, s = 0, nb = 0;
      for (uint32_t j = tid; j < B; j += blockDim.x) {
        const uint32_t v = slot(buf, j, nb);
        x ^= v;
        s += lowbias32(v);
        nb += v != rb + j;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        x ^= __shfl_xor_sync(0xFFFFFFFFu, x, o);
        s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
        nb += __shfl_xor_sync(0xFFFFFFFFu, nb, o);
      }
      if ((tid & 31) == 0) {
        red_x[tid >> 5] = x;
        red_s[tid >> 5] = s;
        red_b[tid >> 5] = nb;
      }
      __syncthreads();
      if (tid == 0) {
        const uint32_t nw = (blockDim.x + 31) / 32;
        uint32_t X = 0, S = 0, NB = 0;
        for (uint32_t w = 0; w < nw; ++w) {
          X ^= red_x[w];
          S += red_s[w];
          NB += red_b[w];
        }
        chk[rb + b] = X;
        mix = rotl32(mix, 5) ^ S;
        bad += NB;
      }
    } else if (tid == 0) {
      const uint32_t p = (b + (uint32_t)r + 1u) % B;
      const uint32_t v = slot(buf, p, bad);
      if constexpr (kDeferFold) {
        pend_v = v;
        pend_want = rb + p;
        pend = true;
      } else {
        mix = rotl32(mix, 5) ^ lowbias32(v);
        bad += v != rb + p;
      }
    }
  }
  if (kDeferFold && tid == 0 && pend) {
    mix = rotl32(mix, 5) ^ lowbias32(pend_v);
    bad += pend_v != pend_want;
  }
  if (tid == 0) {
    mix_out[b] = mix;
    bad_out[b] = bad;
  }
}

using KernelFn = void (*)(uint32_t*, int, uint32_t*, uint32_t*, uint32_t*, uint32_t*, uint32_t*, uint64_t*);

KernelFn pick(int kind, int full) {
  switch (kind) {
    case GSYNC_BAR_ATOMIC: return full ? barrier_workload_kernel<GSYNC_BAR_ATOMIC, true> : barrier_workload_kernel<GSYNC_BAR_ATOMIC, false>;
    case GSYNC_BAR_FLAG: return full ? barrier_workload_kernel<GSYNC_BAR_FLAG, true> : barrier_workload_kernel<GSYNC_BAR_FLAG, false>;
    case GSYNC_BAR_TREE: return full ? barrier_workload_kernel<GSYNC_BAR_TREE, true> : barrier_workload_kernel<GSYNC_BAR_TREE, false>;
    case GSYNC_BAR_CLUSTER: return full ? barrier_workload_kernel<GSYNC_BAR_CLUSTER, true> : barrier_workload_kernel<GSYNC_BAR_CLUSTER, false>;
    case GSYNC_BAR_SHARDED: return full ? barrier_workload_kernel<GSYNC_BAR_SHARDED, true> : barrier_workload_kernel<GSYNC_BAR_SHARDED, false>;
    case GSYNC_BAR_DIE: return full ? barrier_workload_kernel<GSYNC_BAR_DIE, true> : barrier_workload_kernel<GSYNC_BAR_DIE, false>;
    case GSYNC_BAR_SPLIT: return full ? barrier_workload_kernel<GSYNC_BAR_SPLIT, true> : barrier_workload_kernel<GSYNC_BAR_SPLIT, false>;
    case GSYNC_BAR_COUNT: return full ? barrier_workload_kernel<GSYNC_BAR_COUNT, true> : barrier_workload_kernel<GSYNC_BAR_COUNT, false>;
    case GSYNC_BAR_EXCHANGE: return full ? barrier_workload_kernel<GSYNC_BAR_EXCHANGE, true> : barrier_workload_kernel<GSYNC_BAR_EXCHANGE, false>;
  }
  return nullptr;
}

KernelFn pick_trace(int kind) {
  switch (kind) {
    case GSYNC_BAR_ATOMIC: return barrier_workload_kernel<GSYNC_BAR_ATOMIC, false, true>;
    case GSYNC_BAR_FLAG: return barrier_workload_kernel<GSYNC_BAR_FLAG, false, true>;
    case GSYNC_BAR_TREE: return barrier_workload_kernel<GSYNC_BAR_TREE, false, true>;
    case GSYNC_BAR_CLUSTER: return barrier_workload_kernel<GSYNC_BAR_CLUSTER, false, true>;
    case GSYNC_BAR_SHARDED: return barrier_workload_kernel<GSYNC_BAR_SHARDED, false, true>;
    case GSYNC_BAR_DIE: return barrier_workload_kernel<GSYNC_BAR_DIE, false, true>;
    case GSYNC_BAR_SPLIT: return barrier_workload_kernel<GSYNC_BAR_SPLIT, false, true>;
    case GSYNC_BAR_COUNT: return barrier_workload_kernel<GSYNC_BAR_COUNT, false, true>;
    case GSYNC_BAR_EXCHANGE: return barrier_workload_kernel<GSYNC_BAR_EXCHANGE, false, true>;
  }
  return nullptr;
}

}  // namespace

// Phase trace of the sampled barrier workload: trace[2 * (b * rounds + r)] and [+ 1] receive
// block b's %globaltimer just before and just after its round-r barrier_wait.
extern "C" int gsync_probe_barrier_trace(void* state, const gsync_barrier_work* w, uint64_t* trace, void* stream) {
  if (!state || !w || !trace || !aligned(state, 128) || w->full) return GSYNC_EINVAL;
  if (w->nblocks < 1 || w->rounds < 0 || w->block_threads < 32 || w->block_threads > kMaxThreads ||
      w->block_threads % 32 || !w->slots || !w->mix || !w->bad || !w->status)
    return GSYNC_EINVAL;
  KernelFn k = pick_trace(w->kind);
  if (!k) return GSYNC_EINVAL;
  int cluster = 1;
  if (w->kind == GSYNC_BAR_CLUSTER) {
    cluster = w->cluster;
    if (cluster < 1 || cluster > 8 || w->nblocks % cluster) return GSYNC_EINVAL;
  }
  return launch_coresident(k, w->nblocks, w->block_threads, cluster, 0, (cudaStream_t)stream, (uint32_t*)state,
                           w->rounds, w->slots, w->chk, w->mix, w->bad, w->status, trace);
}

namespace gsync_impl {
int max_blocks_barrier(int kind, int block_threads, int cluster, int* out) {
  KernelFn k = pick(kind, 0);
  if (!k) return GSYNC_EINVAL;
  return max_coresident(k, block_threads, kind == GSYNC_BAR_CLUSTER ? cluster : 1, 0, out);
}
}  // namespace gsync_impl

extern "C" int gsync_bench_barrier(void* state, const gsync_barrier_work* w, void* stream) {
  if (!state || !w || !aligned(state, 128)) return GSYNC_EINVAL;
  if (w->nblocks < 1 || w->rounds < 0 || w->block_threads < 32 || w->block_threads > kMaxThreads ||
      w->block_threads % 32)
    return GSYNC_EINVAL;
  if (!w->slots || !w->mix || !w->bad || !w->status || (w->full && !w->chk)) return GSYNC_EINVAL;
  KernelFn k = pick(w->kind, w->full);
  if (!k) return GSYNC_EINVAL;
  int cluster = 1;
  if (w->kind == GSYNC_BAR_CLUSTER) {
    cluster = w->cluster;
    if (cluster < 1 || cluster > 8 || w->nblocks % cluster) return GSYNC_EINVAL;
  }
  return launch_coresident(k, w->nblocks, w->block_threads, cluster, 0, (cudaStream_t)stream, (uint32_t*)state,
                           w->rounds, w->slots, w->chk, w->mix, w->bad, w->status, (uint64_t*)nullptr);
}

// ---------------------------------------------------------------------------------------
// Barrier workload without allocation.  Some callers cannot call cudaMalloc: code that runs
// where a device allocation is not allowed or would stall (a host callback, a loop that
// must not take the implicit device synchronization of cudaMalloc/cudaFree, or a plugin
// whose host framework owns all device memory).  This entry point keeps the barrier object
// and the slot buffers in one file-scope device array instead of caller memory.  The array
// is part of the loaded module, so every GPU that loads the library holds it until exit.
// ---------------------------------------------------------------------------------------
namespace {

constexpr size_t kStaticScratchBytes = 128 * 1024;
constexpr size_t kStaticSlotBytes = 2 * (size_t)GSYNC_STATIC_MAX_BLOCKS * 4;  // 32 KiB
constexpr size_t kStaticStateBytes = kStaticScratchBytes - kStaticSlotBytes;  // 96 KiB
static_assert(kStaticStateBytes % 256 == 0, "slot buffers start on a 256-byte boundary");

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// In host code the name g_static_scratch is only a stand-in; the kernel needs the array's
// device address, looked up here with the caller's device current.  The lookup is repeated
// on every call rather than cached: after a cudaDeviceReset the library's module is loaded
// again and the array may move, so an address kept from before would be stale.  The lookup
// allocates nothing; the first one on a device (and the first after a reset) loads the
// module there.
int static_scratch_address(void** out) {
  void* p = nullptr;
  GSYNC_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
  *out = p;
  return GSYNC_OK;
}

}  // namespace

extern "C" int gsync_bench_barrier_static(const gsync_barrier_work* w, int param, uint64_t timeout_ns,
                                          void* stream) {
  if (!w || w->nblocks < 1 || w->nblocks > GSYNC_STATIC_MAX_BLOCKS) return GSYNC_EINVAL;
  if (!w->mix || !w->bad || !w->status || (w->full && !w->chk)) return GSYNC_EINVAL;
  // The two-die barrier's init measures the die map and synchronizes the stream, which the
  // callers of this entry point cannot afford: it is refused here.
  if (w->kind == GSYNC_BAR_DIE) return GSYNC_EINVAL;
  const int p = w->kind == GSYNC_BAR_CLUSTER ? (param & ~0xF) | w->cluster : param;
  const size_t state_bytes = gsync_barrier_bytes(w->kind, w->nblocks, p);
  if (state_bytes == 0 || state_bytes > kStaticStateBytes) return GSYNC_EINVAL;
  void* base = nullptr;
  if (int rc = static_scratch_address(&base)) return rc;
  void* state = base;
  uint32_t* slots = (uint32_t*)((unsigned char*)base + kStaticStateBytes);
  cudaStream_t st = (cudaStream_t)stream;
  // The array keeps the previous call's contents: rewrite the whole object and clear the slots.
  if (int rc = gsync_barrier_init(state, state_bytes, w->kind, w->nblocks, p, timeout_ns, stream)) return rc;
  GSYNC_CUDA(cudaMemsetAsync(slots, 0, 2 * (size_t)w->nblocks * 4, st));
  gsync_barrier_work dw = *w;
  dw.slots = slots;
  return gsync_bench_barrier(state, &dw, stream);
}
