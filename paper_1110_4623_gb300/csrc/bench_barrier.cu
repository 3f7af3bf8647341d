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
#include "common.cuh"

using namespace gsync_impl;

namespace {

constexpr int kMaxThreads = 256;

// The full-fold variant reduces three values per round and needs more than 32 registers;
// at 128 threads per block it still fits 8 blocks per SM.
template <int KIND, bool FULL>
__global__ void __launch_bounds__(kMaxThreads, FULL ? 4 : 8)
    barrier_workload_kernel(uint32_t* state, int rounds, uint32_t* slots, uint32_t* chk, uint32_t* mix_out,
                            uint32_t* bad_out, uint32_t* status) {
  gsync::BarrierRef bar = gsync::barrier_attach(state);
  const uint32_t B = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  if (bar.kind != (uint32_t)KIND || bar.n != B ||
      (KIND == GSYNC_BAR_CLUSTER && gsync::ptx::cluster_nctarank() != bar.param)) {
    if (tid == 0) gsync::ptx::atom_or_relaxed(status, GSYNC_STATUS_CONFIG);
    return;  // uniform: every block sees the same header
  }
  __shared__ uint32_t red_x[kMaxThreads / 32], red_s[kMaxThreads / 32], red_b[kMaxThreads / 32];
  uint32_t mix = 0, bad = 0;
  for (int r = 0; r < rounds; ++r) {
    uint32_t* buf = slots + (uint32_t)(r & 1) * B;
    const uint32_t rb = (uint32_t)r * B;
    if (tid == 0) buf[b] = rb + b;
    const int rc = gsync::barrier_wait<KIND>(bar);
    if (rc != GSYNC_OK) {
      if (tid == 0) record_status(status, rc);
      break;
    }
    if (FULL) {
      uint32_t x = 0, s = 0, nb = 0;
      for (uint32_t j = tid; j < B; j += blockDim.x) {
        const uint32_t v = buf[j];
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
      const uint32_t v = buf[p];
      mix = rotl32(mix, 5) ^ lowbias32(v);
      bad += v != rb + p;
    }
  }
  if (tid == 0) {
    mix_out[b] = mix;
    bad_out[b] = bad;
  }
}

using KernelFn = void (*)(uint32_t*, int, uint32_t*, uint32_t*, uint32_t*, uint32_t*, uint32_t*);

KernelFn pick(int kind, int full) {
  switch (kind) {
    case GSYNC_BAR_ATOMIC: return full ? barrier_workload_kernel<GSYNC_BAR_ATOMIC, true> : barrier_workload_kernel<GSYNC_BAR_ATOMIC, false>;
    case GSYNC_BAR_FLAG: return full ? barrier_workload_kernel<GSYNC_BAR_FLAG, true> : barrier_workload_kernel<GSYNC_BAR_FLAG, false>;
    case GSYNC_BAR_TREE: return full ? barrier_workload_kernel<GSYNC_BAR_TREE, true> : barrier_workload_kernel<GSYNC_BAR_TREE, false>;
    case GSYNC_BAR_CLUSTER: return full ? barrier_workload_kernel<GSYNC_BAR_CLUSTER, true> : barrier_workload_kernel<GSYNC_BAR_CLUSTER, false>;
  }
  return nullptr;
}

}  // namespace

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
                           w->rounds, w->slots, w->chk, w->mix, w->bad, w->status);
}
