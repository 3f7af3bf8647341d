// Hand-off probes: how fast one block can tell another "you may go" on GB300 (Section 4's
// machine abstraction extended to the signalling forms a Blackwell design can choose from).
//
// gsync_probe_handoff   ping-pong between two SMs through global memory, with a choice of
//                       release form (signal) and observation form (wait).
// gsync_probe_cluster   inside one thread-block cluster: the hardware cluster barrier, a
//                       distributed-shared-memory flag ping-pong, and a remote mbarrier
//                       arrive ping-pong.
// gsync_probe_fence     cost of a gpu-scope fence with and without stores in flight.
// Every wait is bounded by a 1 s globaltimer deadline; on expiry the probe records status 1.
#include "common.cuh"

using namespace gsync_impl;
namespace ptx = gsync::ptx;

namespace {

constexpr uint64_t kDeadlineNs = 1000000000ull;

__device__ __forceinline__ void signal(int mode, uint32_t* f, uint32_t v) {
  switch (mode) {
    case GSYNC_SIGNAL_ST_RELEASE: ptx::st_release(f, v); break;
    case GSYNC_SIGNAL_FENCE_ST_RELAXED: ptx::fence_acq_rel(); ptx::st_relaxed(f, v); break;
    case GSYNC_SIGNAL_ST_RELAXED: ptx::st_relaxed(f, v); break;
    case GSYNC_SIGNAL_RED_RELEASE: ptx::red_add_release(f, 1u); break;
    default: ptx::atom_exch_release(f, v); break;
  }
}

// Returns false on timeout.
__device__ __forceinline__ bool wait_for(int mode, const uint32_t* f, uint32_t v, uint64_t deadline) {
  uint32_t polls = 0;
  for (;;) {
    uint32_t x;
    if (mode == GSYNC_WAIT_LD_ACQUIRE) {
      x = ptx::ld_acquire(f);
    } else if (mode == GSYNC_WAIT_LD_VOLATILE_FENCE) {
      x = ptx::ld_volatile(f);
    } else if (mode == GSYNC_WAIT_LD_RELAXED_X2) {
      // two polls in flight, the second issued ~40 ns after the first
      const uint32_t a = ptx::ld_relaxed(f);
      __nanosleep(0);
      const uint32_t b = ptx::ld_relaxed(f);
      x = a == v ? a : b;
    } else {
      x = ptx::ld_relaxed(f);
    }
    if (x == v) break;
    if ((++polls & 63u) == 0 && ptx::globaltimer() > deadline) return false;
  }
  if (mode == GSYNC_WAIT_LD_RELAXED_FENCE || mode == GSYNC_WAIT_LD_VOLATILE_FENCE || mode == GSYNC_WAIT_LD_RELAXED_X2)
    ptx::fence_acq_rel();
  if (mode == GSYNC_WAIT_LD_RELAXED_THEN_ACQUIRE) (void)ptx::ld_acquire(f);
  return true;
}

__global__ void probe_handoff_kernel(uint32_t* scratch, int signal_mode, int wait_mode, int sm_a, int sm_b, int iters,
                                     uint64_t* out) {
  extern __shared__ uint32_t big_smem[];
  if (threadIdx.x != 0) return;
  const int sm = (int)ptx::smid();
  const bool is_a = sm == sm_a, is_b = sm == sm_b && sm_b != sm_a;
  if (!is_a && !is_b) return;
  big_smem[0] = 0;
  uint32_t* fa = scratch;
  uint32_t* fb = scratch + 32;
  uint32_t* stop = scratch + 64;
  const uint64_t deadline = ptx::globaltimer() + kDeadlineNs;
  const int warm = 64;
  uint64_t t0 = 0;
  for (int i = 1; i <= iters + warm; ++i) {
    if (is_a) {
      if (i == warm + 1) t0 = ptx::globaltimer();
      signal(signal_mode, fa, (uint32_t)i);
      if (!wait_for(wait_mode, fb, (uint32_t)i, deadline)) {
        ptx::st_relaxed(stop, 1u);
        out[3] = 1;
        return;
      }
    } else {
      if (!wait_for(wait_mode, fa, (uint32_t)i, deadline)) {
        ptx::st_relaxed(stop, 1u);
        return;
      }
      signal(signal_mode, fb, (uint32_t)i);
    }
  }
  if (is_a) {
    out[0] = ptx::globaltimer() - t0;
    out[1] = (uint64_t)sm_a;
    out[3] = 0;
  } else {
    out[2] = (uint64_t)sm_b;
  }
}

// ---- inside one cluster ---------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t map_rank(uint32_t local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}

__device__ __forceinline__ void st_cluster_release(uint32_t addr, uint32_t v) {
  asm volatile("st.release.cluster.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_cluster_acquire(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.acquire.cluster.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}

// One 16-byte record in a cluster block's shared memory, read and written as one relaxed
// 128-bit access (the record of a lock whose hand-off carries its data).
__device__ __forceinline__ void st_cluster_relaxed_b128(uint32_t addr, uint64_t lo, uint64_t hi) {
  asm volatile("{\n\t.reg .b128 t;\n\tmov.b128 t, {%1, %2};\n\tst.relaxed.cluster.shared::cluster.b128 [%0], t;\n\t}"
               ::"r"(addr), "l"(lo), "l"(hi) : "memory");
}

__device__ __forceinline__ uint64_t ld_cluster_relaxed_b128_lo(uint32_t addr) {
  uint64_t lo, hi;
  asm volatile("{\n\t.reg .b128 t;\n\tld.relaxed.cluster.shared::cluster.b128 t, [%2];\n\tmov.b128 {%0, %1}, t;\n\t}"
               : "=l"(lo), "=l"(hi) : "r"(addr) : "memory");
  (void)hi;
  return lo;
}

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_remote_arrive(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait_parity(uint32_t addr, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}

// op 0: every thread of every block runs `iters` hardware cluster barriers.
// op 1: ranks 0 and c-1 ping-pong a flag in each other's shared memory (release/acquire).
// op 2: ranks 0 and c-1 ping-pong remote mbarrier arrivals (hardware wait).
// op 3: as op 1 with a 16-byte record in each other's shared memory, written and polled with
//       relaxed 128-bit accesses (no fence on either side): the writer pushes into the
//       poller's shared memory, and the poller polls its own.
// op 4: as op 3, pulled: each rank writes the record in its own shared memory and polls the
//       peer's (the form of a lock whose record lives in one block that every waiter polls).
// out[0] = elapsed ns of the loop on rank 0 (per op: out[0] / iters; per hand-off for
// ops 1-4: out[0] / (2 * iters)); out[3] = status.
__global__ void probe_cluster_kernel(int op, int iters, uint64_t* out) {
  __shared__ __align__(8) uint64_t mbar;
  __shared__ __align__(16) uint64_t rec[2];
  __shared__ uint32_t flag;
  const uint32_t rank = ptx::cluster_ctarank(), n = ptx::cluster_nctarank();
  const uint32_t peer = rank == 0 ? n - 1 : 0;
  if (threadIdx.x == 0) {
    flag = 0;
    rec[0] = rec[1] = 0;
    mbar_init(smem_addr(&mbar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  ptx::cluster_sync();
  const bool player = n > 1 && (rank == 0 || rank == n - 1) && blockIdx.x < n;  // first cluster only
  uint64_t t0 = ptx::globaltimer();
  int status = 0;
  if (op == 0) {
    for (int i = 0; i < iters; ++i) ptx::cluster_sync();
  } else if (player && threadIdx.x == 0) {
    const uint64_t deadline = t0 + kDeadlineNs;
    const uint32_t my_flag = smem_addr(&flag), peer_flag = map_rank(my_flag, peer);
    const uint32_t my_mbar = smem_addr(&mbar), peer_mbar = map_rank(my_mbar, peer);
    const uint32_t my_rec = smem_addr(rec), peer_rec = map_rank(my_rec, peer);
    for (int i = 1; i <= iters && status == 0; ++i) {
      const bool serve = rank == 0;
      if (serve) {
        if (op == 1) st_cluster_release(peer_flag, (uint32_t)i);
        else if (op == 3) st_cluster_relaxed_b128(peer_rec, (uint64_t)i, (uint64_t)i);
        else if (op == 4) st_cluster_relaxed_b128(my_rec, (uint64_t)i, (uint64_t)i);
        else mbar_remote_arrive(peer_mbar);
      }
      uint32_t polls = 0;
      if (op == 1) {
        while (ld_cluster_acquire(my_flag) != (uint32_t)i)
          if ((++polls & 63u) == 0 && ptx::globaltimer() > deadline) { status = 1; break; }
      } else if (op == 3 || op == 4) {
        const uint32_t poll_rec = op == 3 ? my_rec : peer_rec;
        while (ld_cluster_relaxed_b128_lo(poll_rec) != (uint64_t)i)
          if ((++polls & 63u) == 0 && ptx::globaltimer() > deadline) { status = 1; break; }
      } else {
        while (!mbar_try_wait_parity(my_mbar, (uint32_t)((i - 1) & 1)))
          if ((++polls & 63u) == 0 && ptx::globaltimer() > deadline) { status = 1; break; }
      }
      if (!serve && status == 0) {
        if (op == 1) st_cluster_release(peer_flag, (uint32_t)i);
        else if (op == 3) st_cluster_relaxed_b128(peer_rec, (uint64_t)i, (uint64_t)i);
        else if (op == 4) st_cluster_relaxed_b128(my_rec, (uint64_t)i, (uint64_t)i);
        else mbar_remote_arrive(peer_mbar);
      }
    }
  }
  const uint64_t t1 = ptx::globaltimer();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    out[0] = t1 - t0;
    out[3] = (uint64_t)status;
  }
  __syncwarp();
  ptx::cluster_sync();  // no block leaves while a peer may still touch its shared memory
}

// op 0: fence.acq_rel.gpu alone; op 1: a relaxed store then the fence; op 2: a 4-word
// coalesced store by the thread then the fence; op 3: fence.acq_rel.cluster.
__global__ void probe_fence_kernel(uint32_t* scratch, int op, int iters, uint64_t* out) {
  const long long c0 = clock64();
  const uint64_t t0 = ptx::globaltimer();
  for (int i = 0; i < iters; ++i) {
    if (op == 1) ptx::st_relaxed(scratch + 32 * (i & 7), (uint32_t)i);
    if (op == 2) {
      for (int k = 0; k < 4; ++k) scratch[64 * k + (i & 31)] = (uint32_t)i;
    }
    if (op == 3) {
      asm volatile("fence.acq_rel.cluster;" ::: "memory");
    } else {
      ptx::fence_acq_rel();
    }
  }
  const uint64_t t1 = ptx::globaltimer();
  const long long c1 = clock64();
  out[0] = t1 - t0;
  out[1] = (uint64_t)(c1 - c0);
}

constexpr size_t kHandoffSmem = 160 * 1024;

}  // namespace

extern "C" int gsync_probe_handoff(int signal_mode, int wait_mode, int sm_a, int sm_b, int iters, void* scratch,
                                   uint64_t* out, void* stream) {
  int sms = 0;
  if (int rc = device_sms(&sms)) return rc;
  if (signal_mode < 0 || signal_mode > GSYNC_SIGNAL_EXCH_RELEASE || wait_mode < 0 ||
      wait_mode > GSYNC_WAIT_LD_RELAXED_X2 || sm_a < 0 || sm_b < 0 || sm_a >= sms || sm_b >= sms || sm_a == sm_b ||
      iters < 1 || !scratch || !out || !aligned(scratch, 128))
    return GSYNC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  GSYNC_CUDA(cudaFuncSetAttribute(probe_handoff_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kHandoffSmem));
  GSYNC_CUDA(cudaMemsetAsync(scratch, 0, 512, st));
  GSYNC_CUDA(cudaMemsetAsync(out, 0, 4 * sizeof(uint64_t), st));
  return launch_coresident(probe_handoff_kernel, sms, 32, 1, kHandoffSmem, st, (uint32_t*)scratch, signal_mode,
                           wait_mode, sm_a, sm_b, iters, out);
}

extern "C" int gsync_probe_cluster(int op, int cluster, int iters, uint64_t* out, void* stream) {
  if (op < 0 || op > 4 || cluster < 1 || cluster > 8 || iters < 1 || !out || (op > 0 && cluster < 2))
    return GSYNC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  GSYNC_CUDA(cudaMemsetAsync(out, 0, 4 * sizeof(uint64_t), st));
  return launch_coresident(probe_cluster_kernel, cluster, 128, cluster, 0, st, op, iters, out);
}

extern "C" int gsync_probe_fence(int op, int iters, void* scratch, uint64_t* out, void* stream) {
  if (op < 0 || op > 3 || iters < 1 || !scratch || !out || !aligned(scratch, 256)) return GSYNC_EINVAL;
  probe_fence_kernel<<<1, 1, 0, (cudaStream_t)stream>>>((uint32_t*)scratch, op, iters, out);
  GSYNC_CUDA(cudaGetLastError());
  return GSYNC_OK;
}
