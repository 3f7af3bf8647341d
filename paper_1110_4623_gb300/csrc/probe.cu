// Memory-system probes (Section 3, "Benchmarks"; Section 4, "Machine Abstraction").
//
// The paper classifies a GPU by timing one master thread per block issuing 1000 accesses of
// one kind -- {volatile, atomic} x {contentious (every block on one 4-byte word),
// noncontentious (own word, 256 bytes apart)} x {read, write}, plus the volatile tests
// preceded by a single atomic -- on a saturated GPU.  The same kernels run here with the
// PTX-scoped operations a GB300 design actually uses (acquire/relaxed loads, release stores,
// red, 64-bit and acq_rel atomics), and three latency probes feed the roofline of the
// primitives: a dependent atomic chain (round trip to L2), a ping-pong between two SMs
// (release-store to acquire-load hand-off), and __nanosleep's real sleep time.
#include "common.cuh"

using namespace gsync_impl;
namespace ptx = gsync::ptx;

namespace {

template <int OP>
__global__ void probe_tput_kernel(uint32_t* scratch, int contentious, int pre_atomic, int iters, uint64_t* times) {
  if (threadIdx.x != 0) return;  // only the master thread of each block accesses memory
  uint32_t* p = contentious ? scratch : scratch + blockIdx.x * 64u;  // 64 words = 256 bytes
  if (pre_atomic) atomicAdd(p, 0u);
  uint32_t acc = 0;
  const uint64_t t0 = ptx::globaltimer();
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
    if (OP == GSYNC_PROBE_VOLATILE_LOAD) acc += ptx::ld_volatile(p);
    if (OP == GSYNC_PROBE_VOLATILE_STORE) ptx::st_volatile(p, (uint32_t)i);
    if (OP == GSYNC_PROBE_ATOMIC_READ) acc += atomicAdd(p, 0u);
    if (OP == GSYNC_PROBE_ATOMIC_WRITE) acc += atomicExch(p, 0u);
    if (OP == GSYNC_PROBE_LOAD_ACQUIRE) acc += ptx::ld_acquire(p);
    if (OP == GSYNC_PROBE_LOAD_RELAXED) acc += ptx::ld_relaxed(p);
    if (OP == GSYNC_PROBE_STORE_RELEASE) ptx::st_release(p, (uint32_t)i);
    if (OP == GSYNC_PROBE_RED_ADD) ptx::red_add_relaxed(p, 1u);
    if (OP == GSYNC_PROBE_ATOMIC_ADD64) acc += (uint32_t)atomicAdd((unsigned long long*)p, 1ull);
    if (OP == GSYNC_PROBE_ATOMIC_ACQREL) acc += ptx::atom_add_acq_rel(p, 1u);
  }
  const uint64_t t1 = ptx::globaltimer();
  times[2 * blockIdx.x] = t0;
  times[2 * blockIdx.x + 1] = t1;
  if (acc == 0x7FFFFFFFu) p[1] = acc;  // keeps the loaded values live
}

using TputFn = void (*)(uint32_t*, int, int, int, uint64_t*);

TputFn pick_tput(int op) {
  switch (op) {
    case GSYNC_PROBE_VOLATILE_LOAD: return probe_tput_kernel<GSYNC_PROBE_VOLATILE_LOAD>;
    case GSYNC_PROBE_VOLATILE_STORE: return probe_tput_kernel<GSYNC_PROBE_VOLATILE_STORE>;
    case GSYNC_PROBE_ATOMIC_READ: return probe_tput_kernel<GSYNC_PROBE_ATOMIC_READ>;
    case GSYNC_PROBE_ATOMIC_WRITE: return probe_tput_kernel<GSYNC_PROBE_ATOMIC_WRITE>;
    case GSYNC_PROBE_LOAD_ACQUIRE: return probe_tput_kernel<GSYNC_PROBE_LOAD_ACQUIRE>;
    case GSYNC_PROBE_LOAD_RELAXED: return probe_tput_kernel<GSYNC_PROBE_LOAD_RELAXED>;
    case GSYNC_PROBE_STORE_RELEASE: return probe_tput_kernel<GSYNC_PROBE_STORE_RELEASE>;
    case GSYNC_PROBE_RED_ADD: return probe_tput_kernel<GSYNC_PROBE_RED_ADD>;
    case GSYNC_PROBE_ATOMIC_ADD64: return probe_tput_kernel<GSYNC_PROBE_ATOMIC_ADD64>;
    case GSYNC_PROBE_ATOMIC_ACQREL: return probe_tput_kernel<GSYNC_PROBE_ATOMIC_ACQREL>;
  }
  return nullptr;
}

// One thread, `iters` dependent accesses: the next address depends on the loaded value
// (the word holds 0, so the address never changes, but the compiler cannot know that).
template <int OP>
__global__ void probe_latency_kernel(uint32_t* scratch, int iters, uint64_t* out) {
  ptx::st_relaxed(scratch, 0u);
  ptx::fence_acq_rel();
  uint32_t v = 0;
  const uint64_t t0 = ptx::globaltimer();
  const long long c0 = clock64();
  for (int i = 0; i < iters; ++i) {
    uint32_t* q = scratch + ((v >> 31) << 1);  // stays 8-byte aligned for the 64-bit atomic
    if (OP == GSYNC_PROBE_ATOMIC_READ) v = ptx::atom_add_relaxed(q, 0u);
    if (OP == GSYNC_PROBE_LOAD_RELAXED) v = ptx::ld_relaxed(q);
    if (OP == GSYNC_PROBE_VOLATILE_LOAD) v = ptx::ld_volatile(q);
    if (OP == GSYNC_PROBE_LOAD_ACQUIRE) v = ptx::ld_acquire(q);
    if (OP == GSYNC_PROBE_ATOMIC_WRITE) v = atomicExch(q, 0u);
    if (OP == GSYNC_PROBE_ATOMIC_ADD64) v = (uint32_t)atomicAdd((unsigned long long*)q, 0ull);
    if (OP == GSYNC_PROBE_ATOMIC_ACQREL) v = ptx::atom_add_acq_rel(q, 0u);
  }
  const long long c1 = clock64();
  const uint64_t t1 = ptx::globaltimer();
  out[0] = t1 - t0;
  out[1] = (uint64_t)(c1 - c0);
  if (v == 0x7FFFFFFFu) scratch[1] = v;
}

// Ping-pong between the blocks that land on SMs sm_a and sm_b (one block per SM: the launch
// asks for more than half an SM's shared memory).  Side A stores i to line 0 and waits for
// i on line 1; side B waits for i on line 0 and answers on line 1.  Every wait is bounded
// by a 1 s globaltimer deadline; on expiry the side records status 1 and stops.
__global__ void probe_pingpong_kernel(uint32_t* scratch, int sm_a, int sm_b, int iters, uint64_t* out) {
  extern __shared__ uint32_t big_smem[];
  if (threadIdx.x != 0) return;
  const int sm = (int)ptx::smid();
  const bool is_a = sm == sm_a, is_b = sm == sm_b && sm_b != sm_a;
  if (!is_a && !is_b) return;
  big_smem[0] = 0;
  uint32_t* fa = scratch;
  uint32_t* fb = scratch + 32;
  uint32_t* stop = scratch + 64;
  const uint64_t deadline = ptx::globaltimer() + 1000000000ull;
  const int warm = 64;
  uint64_t t0 = 0;
  for (int i = 1; i <= iters + warm; ++i) {
    if (is_a) {
      if (i == warm + 1) t0 = ptx::globaltimer();
      ptx::st_release(fa, (uint32_t)i);
    }
    uint32_t* wait_on = is_a ? fb : fa;
    uint32_t polls = 0;
    while (ptx::ld_acquire(wait_on) != (uint32_t)i) {
      if ((++polls & 63u) == 0 && (ptx::globaltimer() > deadline || ptx::ld_relaxed(stop) != 0)) {
        ptx::st_relaxed(stop, 1u);
        if (is_a) out[3] = 1;
        return;
      }
    }
    if (is_b) ptx::st_release(fb, (uint32_t)i);
  }
  if (is_a) {
    out[0] = ptx::globaltimer() - t0;
    out[1] = (uint64_t)sm_a;
    out[3] = 0;
  } else {
    out[2] = (uint64_t)sm_b;
  }
}

__global__ void probe_nanosleep_kernel(const uint32_t* req, int n, int iters, uint64_t* out) {
  for (int i = 0; i < n; ++i) {
    const uint32_t ns = req[i];
    const uint64_t t0 = ptx::globaltimer();
    for (int k = 0; k < iters; ++k) __nanosleep(ns);
    out[i] = (ptx::globaltimer() - t0) / (uint64_t)iters;
  }
}

constexpr size_t kPingPongSmem = 160 * 1024;

}  // namespace

extern "C" int gsync_probe_throughput(int op, int contentious, int pre_atomic, int nblocks, int block_threads,
                                      int iters, void* scratch, uint64_t* times, void* stream) {
  TputFn k = pick_tput(op);
  if (!k || nblocks < 1 || iters < 0 || block_threads < 1 || block_threads > 1024 || !scratch || !times ||
      !aligned(scratch, 256))
    return GSYNC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  GSYNC_CUDA(cudaMemsetAsync(scratch, 0, (size_t)256 * (size_t)nblocks, st));
  return launch_coresident(k, nblocks, block_threads, 1, 0, st, (uint32_t*)scratch, contentious, pre_atomic, iters,
                           times);
}

extern "C" int gsync_probe_latency(int op, int iters, void* scratch, uint64_t* out, void* stream) {
  if (iters < 1 || !scratch || !out || !aligned(scratch, 128)) return GSYNC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  void (*k)(uint32_t*, int, uint64_t*) = nullptr;
  switch (op) {
    case GSYNC_PROBE_VOLATILE_LOAD: k = probe_latency_kernel<GSYNC_PROBE_VOLATILE_LOAD>; break;
    case GSYNC_PROBE_ATOMIC_READ: k = probe_latency_kernel<GSYNC_PROBE_ATOMIC_READ>; break;
    case GSYNC_PROBE_ATOMIC_WRITE: k = probe_latency_kernel<GSYNC_PROBE_ATOMIC_WRITE>; break;
    case GSYNC_PROBE_LOAD_ACQUIRE: k = probe_latency_kernel<GSYNC_PROBE_LOAD_ACQUIRE>; break;
    case GSYNC_PROBE_LOAD_RELAXED: k = probe_latency_kernel<GSYNC_PROBE_LOAD_RELAXED>; break;
    case GSYNC_PROBE_ATOMIC_ADD64: k = probe_latency_kernel<GSYNC_PROBE_ATOMIC_ADD64>; break;
    case GSYNC_PROBE_ATOMIC_ACQREL: k = probe_latency_kernel<GSYNC_PROBE_ATOMIC_ACQREL>; break;
    default: return GSYNC_EINVAL;  // stores and red return nothing to chain on
  }
  k<<<1, 32, 0, st>>>((uint32_t*)scratch, iters, out);
  GSYNC_CUDA(cudaGetLastError());
  return GSYNC_OK;
}

extern "C" int gsync_probe_pingpong(int sm_a, int sm_b, int iters, void* scratch, uint64_t* out, void* stream) {
  int sms = 0;
  if (int rc = device_sms(&sms)) return rc;
  if (sm_a < 0 || sm_b < 0 || sm_a >= sms || sm_b >= sms || sm_a == sm_b || iters < 1 || !scratch || !out ||
      !aligned(scratch, 128))
    return GSYNC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  GSYNC_CUDA(cudaFuncSetAttribute(probe_pingpong_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kPingPongSmem));
  GSYNC_CUDA(cudaMemsetAsync(scratch, 0, 512, st));
  GSYNC_CUDA(cudaMemsetAsync(out, 0, 4 * sizeof(uint64_t), st));
  return launch_coresident(probe_pingpong_kernel, sms, 32, 1, kPingPongSmem, st, (uint32_t*)scratch, sm_a, sm_b,
                           iters, out);
}

extern "C" int gsync_probe_nanosleep(const uint32_t* req_ns, int n, int iters, uint64_t* out_ns, void* stream) {
  if (!req_ns || !out_ns || n < 1 || iters < 1) return GSYNC_EINVAL;
  probe_nanosleep_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(req_ns, n, iters, out_ns);
  GSYNC_CUDA(cudaGetLastError());
  return GSYNC_OK;
}
