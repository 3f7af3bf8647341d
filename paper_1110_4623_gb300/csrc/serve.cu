// Persistent serving loop with continuous batching, built on the library's own ticket lock and
// ticket-window semaphore (the paper motivates its primitives with task queues, Section 1, and
// names hardware enqueue/dequeue as a wish, Section 7).
//
// The host publishes requests into a ring of 16-byte entries (each entry carries its sequence
// number twice, one copy in each of its two 8-byte halves, each half written with one store).
// The ring is caller memory: pinned host memory, which the admitters poll across the host
// link, or managed memory placed in device memory, which the host writes in place and the
// admitters poll through L2.  Inside one co-resident
// launch:
//   * admitter blocks wait on the admission semaphore (n = number of in-flight slots), take
//     the next request index under the ring's ticket lock, wait for that entry to appear,
//     claim a free slot and publish the request in it (generation-tagged chunk counter,
//     release store of the slot state);
//   * every other block claims chunks of any active slot (compare-and-swap on the slot's
//     generation:chunk counter), sums the chunk's int32 values in int64, adds the partial to
//     the slot's accumulator; the block that finishes a request's last chunk writes the result
//     and a completion flag into pinned host memory, frees the slot and posts the semaphore.
// Requests that arrive while others run are admitted as slots free up and their chunks run
// side by side with older requests' chunks.  Every wait is bounded (the object timeouts, or
// the loop's own deadline) and the host's shutdown word ends the loop.
//
// The per-request-launch baseline runs the same chunked segmented sum as one kernel launch
// per request and completes it the same way (result and flag in pinned host memory).
#include <pthread.h>
#include <stddef.h>
#include <sched.h>
#include <string.h>
#include <unistd.h>

#include <atomic>
#include <chrono>
#include <thread>
#include <vector>

#include "common.cuh"

using namespace gsync_impl;
namespace ptx = gsync::ptx;

namespace {

constexpr int kThreads = 256;
// Ring entries sit one per 128-byte line, so the host writing entry q never touches a line
// that an admitter polls for another entry.
constexpr size_t kRingStride = 128;
static_assert(sizeof(gsync_serve_req) == 16 && offsetof(gsync_serve_req, seq) == 0 &&
                  offsetof(gsync_serve_req, len) == 4 && offsetof(gsync_serve_req, off) == 8 &&
                  offsetof(gsync_serve_req, seq_check) == 12,
              "the producer writes an entry as two 8-byte halves {seq, len} and {off, seq_check}");
static_assert(__BYTE_ORDER__ == __ORDER_LITTLE_ENDIAN__, "the entry halves are packed little-endian");
// The active mask is kept in kMaskCopies copies on separate lines (set and cleared in all,
// read from one per worker) to spread the workers' polling.
constexpr uint32_t kMaskCopies = 4;

struct Slot {  // one 128-byte line; the first 16 bytes are everything a chunk claim reads
  uint32_t state;       // 0 free, 1 claimed by an admitter, 2 active
  uint32_t gen;         // bumped every time the slot takes a request
  uint32_t next_chunk;  // (gen & 0xFFFF) << 16 | next chunk to hand out
  uint32_t nchunks;
  uint32_t done_chunks;
  uint32_t id;
  int64_t off;
  int64_t len;
  unsigned long long acc;
  uint32_t pad[20];
};
static_assert(sizeof(Slot) == 128, "one line per slot");

struct Args {
  const gsync_serve_req* ring;  // device view of the host ring
  uint32_t ring_mask;
  const uint32_t* shutdown;  // device view (host writes)
  uint32_t* dev_shutdown;    // device copy of the shutdown word, set by an admitter (own line)
  int64_t* res;              // device view of host results
  uint32_t* done;            // device view of host completion flags
  const int32_t* pool;
  uint32_t* ring_lock;       // gsync mutex (TICKET)
  uint32_t* admit_sem;       // gsync semaphore (WINDOW), n = nslots
  Slot* slots;
  uint32_t* active_mask;     // one bit per slot (nslots <= 64)
  uint32_t* stats;           // [0] admitted, [32] chunks, [64] completed (own lines)
  uint32_t* status;
  unsigned long long* trace;  // optional per-request timestamps (4 per request)
  uint32_t nslots, admitters, chunk_elems;
  uint64_t timeout_ns;
};

__device__ __forceinline__ uint32_t ld_acquire_sys(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint4 ld_acquire_sys_v4(const void* p) {
  uint4 v;
  asm volatile("ld.acquire.sys.global.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p)
               : "memory");
  return v;
}
__device__ __forceinline__ void st_release_sys(uint32_t* p, uint32_t v) {
  asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_sys_s64(int64_t* p, int64_t v) {
  asm volatile("st.relaxed.sys.global.s64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Block-wide int64 sum of pool[a, b): 16-byte streaming loads over the aligned middle, eight
// of them in flight per thread (issued before any is added; the last, partial pass -- every
// request's last chunk -- too, with the loads past the end predicated off), scalars at the
// ends.
__device__ __forceinline__ long long block_sum(const int32_t* pool, int64_t a, int64_t b) {
  constexpr int kInFlight = 8;
  long long s = 0;
  int64_t a4 = (a + 3) & ~(int64_t)3;
  if (a4 > b) a4 = b;
  const int64_t b4 = a4 + ((b - a4) & ~(int64_t)3);
  for (int64_t i = a + threadIdx.x; i < a4; i += blockDim.x) s += pool[i];
  const int4* v = reinterpret_cast<const int4*>(pool + a4);
  const int64_t nv = (b4 - a4) >> 2;
  const int64_t step = (int64_t)blockDim.x * kInFlight;
  int64_t i = threadIdx.x;
  for (; i + (kInFlight - 1) * (int64_t)blockDim.x < nv; i += step) {
    int4 x[kInFlight];
#pragma unroll
    for (int k = 0; k < kInFlight; ++k) x[k] = __ldcs(v + i + k * (int64_t)blockDim.x);
#pragma unroll
    for (int k = 0; k < kInFlight; ++k) s += (long long)x[k].x + x[k].y + x[k].z + x[k].w;
  }
  if (i < nv) {  // fewer than kInFlight left for this thread: issue them all before adding
    int4 x[kInFlight];
#pragma unroll
    for (int k = 0; k < kInFlight; ++k) {
      const int64_t j = i + k * (int64_t)blockDim.x;
      x[k] = j < nv ? __ldcs(v + j) : make_int4(0, 0, 0, 0);
    }
#pragma unroll
    for (int k = 0; k < kInFlight; ++k) s += (long long)x[k].x + x[k].y + x[k].z + x[k].w;
  }
  for (int64_t i = b4 + threadIdx.x; i < b; i += blockDim.x) s += pool[i];
  __shared__ long long red[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  long long t = 0;
  if (threadIdx.x == 0)
    for (uint32_t w = 0; w < (blockDim.x + 31) / 32; ++w) t += red[w];
  __syncthreads();
  return t;  // valid in thread 0
}

__device__ __forceinline__ bool gen_after(uint32_t a, uint32_t b) { return (int16_t)(uint16_t)(a - b) > 0; }

// Thread 0: claims one chunk of slot s, or returns false.  The claim is one fetch-and-add on
// the slot's (generation:16 | chunk:16) counter, so racing workers each get a distinct chunk
// in one round trip.  A result past the generation's chunk count is an over-claim and is
// dropped (a request has at most 32767 chunks, so over-claims never reach the generation
// bits).  A claim that lands after the slot moved to a newer request is a real chunk of that
// request: the worker waits (bounded) for the newer generation to be published and serves
// it.  A claim of an older generation than the one now published is dropped.
__device__ bool claim_chunk(Slot* slot, uint32_t& chunk, uint32_t& gen, bool& last, uint64_t timeout_ns) {
  const uint32_t v = gsync::ptx::atom_add_relaxed(&slot->next_chunk, 1u);
  const uint32_t g = v >> 16, c = v & 0xFFFFu;
  uint64_t deadline = 0;
  for (;;) {
    const uint4 h = gsync::ptx::ld_acquire_v4(&slot->state);
    const uint32_t hg = h.y & 0xFFFFu;
    if (h.x == 2u && hg == g) {
      if (c >= h.w) return false;
      chunk = c;
      gen = h.y;
      last = c + 1u == h.w;
      return true;
    }
    if (gen_after(hg, g) || (hg == g && h.x != 2u && h.x != 1u)) return false;  // stale claim
    // generation g is being set up (or not yet published): wait for it, bounded
    const uint64_t now = ptx::globaltimer();
    if (deadline == 0) deadline = now + timeout_ns;
    if (now > deadline) return false;
  }
}

__global__ void __launch_bounds__(kThreads) serve_kernel(Args a) {
  const uint32_t tid = threadIdx.x;
  const gsync::MutexRef lock = gsync::mutex_attach(a.ring_lock);
  const gsync::SemRef sem = gsync::sem_attach(a.admit_sem);
  __shared__ int s_cmd;       // 0 continue, 1 exit
  __shared__ uint32_t s_slot;
  __shared__ int64_t s_lo, s_hi;
  const bool admitter = blockIdx.x < a.admitters;
  uint32_t idle = 0, scan = blockIdx.x % a.nslots;
  uint64_t idle_since = 0;

  if (admitter) {
    // Admitters: semaphore -> ring index (ticket lock) -> wait for that entry -> slot.  The
    // permit and the index are taken before the request exists, so its arrival only waits
    // for one read of host memory.  Thread 0 does everything; the block only idles.
    if (tid == 0) {
      for (;;) {
        if (ptx::ld_relaxed(a.dev_shutdown)) break;
        int rc = gsync::sem_wait_thread<GSYNC_SEM_WINDOW>(sem);
        if (rc != GSYNC_OK) { record_status(a.status, rc); break; }
        if (ptx::ld_relaxed(a.dev_shutdown)) {  // pass the permit on so blocked admitters exit too
          gsync::sem_post_thread<GSYNC_SEM_WINDOW>(sem);
          break;
        }
        // The ring's head index is the ticket of the ring lock: tickets are handed out in
        // order from 0, one per acquisition, so the holder needs no head word and releases
        // the lock at once.
        const gsync::Token t = gsync::mutex_lock_thread<GSYNC_MUTEX_TICKET>(lock);
        if (t.status != GSYNC_OK) { record_status(a.status, t.status); break; }
        const uint32_t h = t.ticket;
        gsync::mutex_unlock_thread<GSYNC_MUTEX_TICKET>(lock, t.ticket);
        // wait for entry h (seq == seq_check == h + 1) or shutdown
        const gsync_serve_req* e =
            (const gsync_serve_req*)((const char*)a.ring + (size_t)(h & a.ring_mask) * kRingStride);
        uint4 v;
        uint32_t polls = 0;
        bool stop = false;
        const uint64_t t0 = ptx::globaltimer();
        for (;;) {
          v = ld_acquire_sys_v4(e);
          if (v.x == h + 1u && v.w == h + 1u) break;
          if ((++polls & 15u) == 0) {
            if (ld_acquire_sys(a.shutdown)) {
              ptx::st_release(a.dev_shutdown, 1u);
              stop = true;
              break;
            }
            if (ptx::globaltimer() - t0 > a.timeout_ns * 16) { record_status(a.status, GSYNC_ETIMEDOUT); stop = true; break; }
          }
        }
        if (stop) {  // the permit goes back so that admitters blocked on it can see shutdown
          gsync::sem_post_thread<GSYNC_SEM_WINDOW>(sem);
          break;
        }
        const uint32_t req_len = v.y, req_off = v.z, req_id = h;
        if (a.trace) a.trace[4ull * req_id] = ptx::globaltimer();
        // claim a free slot (the permit guarantees one)
        uint32_t s = h % a.nslots;
        bool got = false;
        for (uint32_t k = 0; k < 4u * a.nslots; ++k) {
          if (ptx::atom_cas_acquire(&a.slots[s].state, 0u, 1u) == 0u) { got = true; break; }
          if (++s == a.nslots) s = 0;
        }
        if (!got) { record_status(a.status, GSYNC_ETIMEDOUT); break; }
        Slot* sl = &a.slots[s];
        // gen, nchunks and the chunk counter are read (and the counter added to) by workers
        // at any time, so they are written with strong (relaxed) stores; the rest is read
        // only after the release of state = 2.
        const uint32_t gen = ptx::ld_relaxed(&sl->gen) + 1u;
        const uint32_t nch = (req_len + a.chunk_elems - 1u) / a.chunk_elems;
        ptx::st_relaxed(&sl->gen, gen);
        sl->id = req_id;
        sl->off = (int64_t)req_off;
        sl->len = (int64_t)req_len;
        ptx::st_relaxed(&sl->nchunks, nch == 0 ? 1u : nch);
        sl->acc = 0ull;
        sl->done_chunks = 0u;
        ptx::st_relaxed(&sl->next_chunk, (gen & 0xFFFFu) << 16);
        ptx::st_release(&sl->state, 2u);
        for (uint32_t m = 0; m < kMaskCopies; ++m) atomicOr(&a.active_mask[32u * m + (s >> 5)], 1u << (s & 31));
        ptx::red_add_relaxed(a.stats, 1u);
        if (a.trace) a.trace[4ull * req_id + 1] = ptx::globaltimer();
      }
    }
    return;
  }

  // Workers: claim chunks of active slots until shutdown.
  for (;;) {
    if (tid == 0) {
      s_cmd = 2;  // nothing yet
      const uint32_t* my_mask = a.active_mask + 32u * (blockIdx.x % kMaskCopies);
      uint64_t mask;  // both mask words in one load (the copy starts a line)
      asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(mask) : "l"(my_mask) : "memory");
      // Visit only the set bits, in the order scan, scan + 1, ..., nslots - 1, 0, ..., scan - 1
      // (bits at or above `scan` first): a walk over all slots with a division per step costs a
      // single thread ~10 us, which every idle worker would pay whenever any slot is active.
      const uint64_t upper = mask & (~0ull << scan), lower = mask & ~(~0ull << scan);
      bool got = false;
      for (int pass = 0; pass < 2 && !got; ++pass) {
        for (uint64_t m = pass ? lower : upper; m && !got; m &= m - 1u) {
          const uint32_t s = (uint32_t)__ffsll((long long)m) - 1u;
          uint32_t c, g;
          bool last;
          if (!claim_chunk(&a.slots[s], c, g, last, a.timeout_ns)) continue;
          // The last chunk is handed out: the slot has no more work to find, so it leaves the
          // active mask now (it cannot be reused before this chunk completes).
          if (last)
            for (uint32_t k = 0; k < kMaskCopies; ++k) atomicAnd(&a.active_mask[32u * k + (s >> 5)], ~(1u << (s & 31)));
          Slot* sl = &a.slots[s];
          const int64_t lo = sl->off + (int64_t)c * a.chunk_elems;
          int64_t hi = lo + a.chunk_elems;
          if (hi > sl->off + sl->len) hi = sl->off + sl->len;
          s_slot = s; s_lo = lo; s_hi = hi;
          if (a.trace && c == 0) a.trace[4ull * sl->id + 2] = ptx::globaltimer();
          s_cmd = 0;
          scan = s;
          got = true;
        }
      }
      if (s_cmd == 2) {
        if ((idle & 15u) == 15u && ptx::ld_relaxed(a.dev_shutdown)) s_cmd = 1;
        if ((++idle & 255u) == 0) {
          if (ld_acquire_sys(a.shutdown)) s_cmd = 1;
          const uint64_t now = ptx::globaltimer();
          if (idle_since == 0) idle_since = now;
          else if (now - idle_since > a.timeout_ns * 16) { record_status(a.status, GSYNC_ETIMEDOUT); s_cmd = 1; }
        }
        if (s_cmd == 2) __nanosleep(32);
      } else {
        idle = 0;
        idle_since = 0;
      }
    }
    __syncthreads();
    const int cmd = s_cmd;
    if (cmd == 1) break;
    if (cmd == 2) { __syncthreads(); continue; }
    const long long part = block_sum(a.pool, s_lo, s_hi);
    if (tid == 0) {
      Slot* sl = &a.slots[s_slot];
      atomicAdd(&sl->acc, (unsigned long long)part);
      ptx::red_add_relaxed(a.stats + 32, 1u);
      const uint32_t d = ptx::atom_add_acq_rel(&sl->done_chunks, 1u) + 1u;
      if (d == sl->nchunks) {
        const long long total = (long long)atomicAdd(&sl->acc, 0ull);
        const uint32_t id = sl->id;
        if (a.trace) a.trace[4ull * id + 3] = ptx::globaltimer();
        st_relaxed_sys_s64(a.res + id, total);
        st_release_sys(a.done + id, 1u);
        ptx::st_release(&sl->state, 0u);
        gsync::sem_post_thread<GSYNC_SEM_WINDOW>(sem);
        ptx::red_add_relaxed(a.stats + 64, 1u);
      }
    }
    __syncthreads();
  }
}

// Baseline: one launch per request; block j sums chunk j; the last block completes it.
__global__ void __launch_bounds__(kThreads) segsum_kernel(const int32_t* pool, int64_t off, int64_t len,
                                                          uint32_t chunk_elems, unsigned long long* acc,
                                                          uint32_t* counter, uint32_t id, int64_t* res,
                                                          uint32_t* done) {
  const int64_t lo = off + (int64_t)blockIdx.x * chunk_elems;
  int64_t hi = lo + chunk_elems;
  if (hi > off + len) hi = off + len;
  const long long part = block_sum(pool, lo, hi);
  if (threadIdx.x == 0) {
    atomicAdd(acc, (unsigned long long)part);
    const uint32_t d = ptx::atom_add_acq_rel(counter, 1u) + 1u;
    if (d == gridDim.x) {
      const long long total = (long long)atomicAdd(acc, 0ull);
      st_relaxed_sys_s64(res + id, total);
      st_release_sys(done + id, 1u);
    }
  }
}

int host_dev_ptr(void* host, void** dev) {
  GSYNC_CUDA(cudaHostGetDevicePointer(dev, host, 0));
  return GSYNC_OK;
}

// The ring's device view.  Pinned host memory is mapped (host_dev_ptr).  A ring in managed
// memory has one address on both sides; on a GPU whose host reaches managed memory in place
// over a coherent link (cudaDevAttrDirectManagedMemAccessFromHost), it is advised to live in
// device memory and to stay mapped for the host, and is moved there before the host clears it:
// the producer's stores then cross the link into device memory, and the admitters poll it
// through the GPU's L2 instead of across the link.
int ring_device_ptr(void* ring, size_t bytes, cudaStream_t st, void** dev) {
  cudaPointerAttributes attr;
  GSYNC_CUDA(cudaPointerGetAttributes(&attr, ring));
  if (attr.type != cudaMemoryTypeManaged) return host_dev_ptr(ring, dev);
  int devid = 0, direct = 0;
  GSYNC_CUDA(cudaGetDevice(&devid));
  GSYNC_CUDA(cudaDeviceGetAttribute(&direct, cudaDevAttrDirectManagedMemAccessFromHost, devid));
  if (direct) {
    cudaMemLocation gpu = {};
    gpu.type = cudaMemLocationTypeDevice;
    gpu.id = devid;
    cudaMemLocation cpu = {};
    cpu.type = cudaMemLocationTypeHost;
    GSYNC_CUDA(cudaMemAdvise(ring, bytes, cudaMemAdviseSetPreferredLocation, gpu));
    GSYNC_CUDA(cudaMemAdvise(ring, bytes, cudaMemAdviseSetAccessedBy, cpu));
    GSYNC_CUDA(cudaMemPrefetchAsync(ring, bytes, gpu, 0, st));
    GSYNC_CUDA(cudaStreamSynchronize(st));
  }
  *dev = ring;
  return GSYNC_OK;
}

using Clock = std::chrono::steady_clock;

// Pins a host thread to one core (counted from the last core down) so that the producer and
// the collector are not descheduled behind each other.  Best effort: ignored on failure.
void pin_to_core_from_end(std::thread& t, int k) {
  const long n = sysconf(_SC_NPROCESSORS_ONLN);
  if (n < 4) return;
  cpu_set_t set;
  CPU_ZERO(&set);
  CPU_SET((int)(n - 1 - k), &set);
  (void)pthread_setaffinity_np(t.native_handle(), sizeof(set), &set);
}

int64_t now_ns(Clock::time_point t0) {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - t0).count();
}

void spin_until(Clock::time_point t) {
  while (Clock::now() < t) {
  }
}

// Counters shared by the host threads of a run, one per cache line: the collector updates
// `completed` while the producer (or launcher) reads it and writes `published`, and a line
// shared between writers on different cores would bounce on every update.
struct alignas(128) HostCounter {
  std::atomic<int> v{0};
};
struct alignas(128) HostFlag {
  std::atomic<bool> v{false};
};

// Polls completion flags in order of arrival; records the host time each flag is first seen.
// A pass scans from the oldest incomplete request to the last one published (or launched), at
// most 4096 of them: only requests in flight can complete, so a pass stays as short as the
// work in flight instead of walking a fixed window of flags.
void collect(const gsync_serve_cfg* cfg, volatile uint32_t* done, Clock::time_point t0, const int64_t* sched,
             int64_t* lat, std::atomic<int>* completed, std::atomic<bool>* abort_flag,
             const std::atomic<int>* published) {
  const int n = cfg->nreq;
  std::vector<char> seen(n, 0);
  int low = 0, count = 0, reported = 0;
  while (count < n && !abort_flag->load(std::memory_order_relaxed)) {
    const int hi = std::min(std::min(n, low + 4096), published->load(std::memory_order_acquire));
    for (int q = low; q < hi; ++q) {
      if (seen[q]) continue;
      if (done[q]) {
        std::atomic_thread_fence(std::memory_order_acquire);
        lat[q] = now_ns(t0) - sched[q];
        seen[q] = 1;
        ++count;
      }
    }
    while (low < n && seen[low]) ++low;
    if (count != reported) {  // stored only when it moves, so readers keep the line cached
      completed->store(count, std::memory_order_release);
      reported = count;
    }
  }
}

// Every request must lie inside the pool and fit the chunk counter.
int check_requests(const gsync_serve_cfg* cfg, const gsync_serve_buffers* buf) {
  for (int q = 0; q < cfg->nreq; ++q) {
    const int64_t o = buf->offset[q], n = buf->length[q];
    if (o < 0 || n < 1 || o > buf->pool_elems - n) return GSYNC_EINVAL;
    if ((n + cfg->chunk_elems - 1) / cfg->chunk_elems > 32767) return GSYNC_EINVAL;
    if (q > 0 && buf->sched_ns[q] < buf->sched_ns[q - 1]) return GSYNC_EINVAL;
  }
  return GSYNC_OK;
}

}  // namespace

extern "C" size_t gsync_serve_workspace_bytes(int nslots) {
  if (nslots < 1 || nslots > 64) return 0;
  return 3 * 128 /* ring lock */ + 4 * 128 /* semaphore */ + (size_t)nslots * 128 +
         128 * kMaskCopies /* active mask */ + 3 * 128 /* stats */ + 128 /* status */ + 128 /* device shutdown */;
}

extern "C" int gsync_serve_run(const gsync_serve_cfg* cfg, gsync_serve_buffers* buf, void* workspace,
                               size_t workspace_bytes, void* stream) {
  if (!cfg || !buf || !workspace || cfg->nreq < 1 || cfg->nslots < 1 || cfg->nslots > 64 || cfg->nblocks < 2 ||
      cfg->admitters < 1 || cfg->admitters >= cfg->nblocks || cfg->chunk_elems < 1024 || cfg->ring_slots < 2 ||
      (cfg->ring_slots & (cfg->ring_slots - 1)) || !aligned(workspace, 256))
    return GSYNC_EINVAL;
  if (workspace_bytes < gsync_serve_workspace_bytes(cfg->nslots)) return GSYNC_EINVAL;
  if (!buf->pool || !buf->offset || !buf->length || !buf->sched_ns || !buf->ring || !buf->ctrl || !buf->res ||
      !buf->done || !buf->latency_ns)
    return GSYNC_EINVAL;
  if (int rc = check_requests(cfg, buf)) return rc;
  if (buf->pool_elems > (int64_t)0xFFFFFFFFll) return GSYNC_EINVAL;  // 32-bit offsets in the ring
  cudaStream_t st = (cudaStream_t)stream;
  char* p = (char*)workspace;
  uint32_t* ring_lock = (uint32_t*)p; p += 3 * 128;
  uint32_t* sem = (uint32_t*)p;       p += 4 * 128;
  Slot* slots = (Slot*)p;             p += (size_t)cfg->nslots * 128;
  uint32_t* mask = (uint32_t*)p;      p += 128 * kMaskCopies;
  uint32_t* stats = (uint32_t*)p;     p += 3 * 128;
  uint32_t* status = (uint32_t*)p;    p += 128;
  uint32_t* dev_shutdown = (uint32_t*)p;
  GSYNC_CUDA(cudaMemsetAsync(workspace, 0, gsync_serve_workspace_bytes(cfg->nslots), st));
  // Admitters may legitimately wait for a permit or an index while arrivals are sparse: the
  // lock and the semaphore get 16x the per-wait bound.
  const uint64_t wait_ns = (cfg->timeout_ns ? cfg->timeout_ns : 2000000000ull) * 16;
  if (int rc = gsync_mutex_init(ring_lock, 3 * 128, GSYNC_MUTEX_TICKET, 1, nullptr, wait_ns, stream)) return rc;
  gsync_backoff sbo = {GSYNC_BACKOFF_EXPONENTIAL, 64, 2000, 0};
  if (int rc = gsync_sem_init(sem, 4 * 128, GSYNC_SEM_WINDOW, cfg->nslots, &sbo, wait_ns, stream)) return rc;

  // The host threads write these arrays on the latency path: touch every page first.
  for (int q = 0; q < cfg->nreq; ++q) buf->latency_ns[q] = 0;
  if (buf->publish_ns)
    for (int q = 0; q < cfg->nreq; ++q) buf->publish_ns[q] = 0;
  // Host control word ctrl[32] = shutdown; the ring starts empty (no entry has a valid seq).
  void* d_ring = nullptr;
  if (int rc = ring_device_ptr(buf->ring, kRingStride * (size_t)cfg->ring_slots, st, &d_ring)) return rc;
  volatile uint32_t* ctrl = buf->ctrl;
  ctrl[32] = 0;
  memset(buf->ring, 0, kRingStride * (size_t)cfg->ring_slots);
  for (int q = 0; q < cfg->nreq; ++q) buf->done[q] = 0;
  std::atomic_thread_fence(std::memory_order_seq_cst);

  Args a;
  void *d_ctrl, *d_res, *d_done;
  if (int rc = host_dev_ptr((void*)buf->ctrl, &d_ctrl)) return rc;
  if (int rc = host_dev_ptr(buf->res, &d_res)) return rc;
  if (int rc = host_dev_ptr((void*)buf->done, &d_done)) return rc;
  a.ring = (const gsync_serve_req*)d_ring;
  a.ring_mask = (uint32_t)cfg->ring_slots - 1u;
  a.shutdown = (const uint32_t*)d_ctrl + 32;
  a.dev_shutdown = dev_shutdown;
  a.res = (int64_t*)d_res;
  a.done = (uint32_t*)d_done;
  a.pool = buf->pool;
  a.ring_lock = ring_lock;
  a.admit_sem = sem;
  a.slots = slots;
  a.active_mask = mask;
  a.stats = stats;
  a.status = status;
  a.trace = (unsigned long long*)buf->trace;
  a.nslots = (uint32_t)cfg->nslots;
  a.admitters = (uint32_t)cfg->admitters;
  a.chunk_elems = (uint32_t)cfg->chunk_elems;
  a.timeout_ns = cfg->timeout_ns ? cfg->timeout_ns : 2000000000ull;
  if (int rc = launch_coresident(serve_kernel, cfg->nblocks, kThreads, 1, 0, st, a)) return rc;

  // The loop is running (or about to): publish requests on their schedule, collect completions.
  std::this_thread::sleep_for(std::chrono::microseconds(cfg->start_delay_us));
  const Clock::time_point t0 = Clock::now();
  HostCounter completed_c, published_c;
  HostFlag abort_f;
  std::atomic<int>& completed = completed_c.v;
  std::atomic<int>& published = published_c.v;
  std::atomic<bool>& abort_flag = abort_f.v;
  std::thread collector(collect, cfg, buf->done, t0, buf->sched_ns, buf->latency_ns, &completed, &abort_flag,
                        &published);
  pin_to_core_from_end(collector, 1);
  const auto deadline = Clock::now() + std::chrono::nanoseconds(buf->sched_ns[cfg->nreq - 1]) +
                        std::chrono::seconds(cfg->drain_timeout_s);
  // The producer runs on its own pinned core too; this thread only waits.
  std::atomic<int> prod_rc{GSYNC_OK};
  std::thread producer([&]() {
    // Publishes every request whose time has come in one batch.  Each entry is written with
    // two aligned 8-byte stores, {seq, len} and {off, seq_check}, and no fence: each store is
    // single-copy atomic, so an entry whose seq and seq_check both read q + 1 holds request
    // q's len and off whatever order the two stores became visible in (a reader that sees
    // one half of an older lap's entry finds that half's sequence number stale).  One
    // write per half, with nothing to wait for between them, keeps the producer on schedule
    // where its stores cross the host link into device memory.
    int q = 0;
    while (q < cfg->nreq) {
      spin_until(t0 + std::chrono::nanoseconds(buf->sched_ns[q]));
      const int64_t now = now_ns(t0);
      int qe = q + 1;
      while (qe < cfg->nreq && buf->sched_ns[qe] <= now && qe - q < 64) ++qe;
      // The ring entry of request i is reused only after request i - ring_slots completed.
      while (qe - 1 - completed.load(std::memory_order_acquire) >= cfg->ring_slots) {
        if (Clock::now() > deadline || abort_flag.load(std::memory_order_relaxed)) {
          prod_rc.store(GSYNC_ETIMEDOUT);
          return;
        }
      }
      for (int i = q; i < qe; ++i) {
        uint64_t* e = (uint64_t*)((char*)buf->ring + (size_t)(i & (cfg->ring_slots - 1)) * kRingStride);
        const uint64_t seq = (uint32_t)(i + 1);
        // little-endian layout of gsync_serve_req: seq | len << 32, then off | seq_check << 32
        __atomic_store_n(e, seq | ((uint64_t)(uint32_t)buf->length[i] << 32), __ATOMIC_RELAXED);
        __atomic_store_n(e + 1, (uint64_t)(uint32_t)buf->offset[i] | (seq << 32), __ATOMIC_RELAXED);
      }
      published.store(qe, std::memory_order_release);
      if (buf->publish_ns) {
        const int64_t t = now_ns(t0);
        for (int i = q; i < qe; ++i) buf->publish_ns[i] = t;
      }
      q = qe;
    }
  });
  pin_to_core_from_end(producer, 0);
  int rc = GSYNC_OK;
  while (completed.load(std::memory_order_acquire) < cfg->nreq) {
    if (Clock::now() > deadline || prod_rc.load() != GSYNC_OK) {
      rc = GSYNC_ETIMEDOUT;
      break;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  abort_flag.store(true);
  producer.join();
  if (rc == GSYNC_OK) rc = prod_rc.load();
  collector.join();
  __atomic_store_n(&buf->ctrl[32], 1u, __ATOMIC_RELEASE);
  GSYNC_CUDA(cudaStreamSynchronize(st));
  uint32_t hstat[4] = {0, 0, 0, 0};
  GSYNC_CUDA(cudaMemcpy(&hstat[0], stats, 4, cudaMemcpyDeviceToHost));
  GSYNC_CUDA(cudaMemcpy(&hstat[1], stats + 32, 4, cudaMemcpyDeviceToHost));
  GSYNC_CUDA(cudaMemcpy(&hstat[2], stats + 64, 4, cudaMemcpyDeviceToHost));
  GSYNC_CUDA(cudaMemcpy(&hstat[3], status, 4, cudaMemcpyDeviceToHost));
  buf->stats[0] = hstat[0];
  buf->stats[1] = hstat[1];
  buf->stats[2] = hstat[2];
  buf->stats[3] = hstat[3];
  if (rc == GSYNC_OK && hstat[3]) rc = GSYNC_ETIMEDOUT;
  return rc;
}

extern "C" size_t gsync_serve_baseline_workspace_bytes(int nreq) {
  if (nreq < 1) return 0;
  return (size_t)nreq * 16;
}

extern "C" int gsync_serve_baseline(const gsync_serve_cfg* cfg, gsync_serve_buffers* buf, void* workspace,
                                    size_t workspace_bytes, void* const* streams, int nstreams) {
  if (!cfg || !buf || !workspace || cfg->nreq < 1 || cfg->chunk_elems < 1024 || !streams || nstreams < 1 ||
      workspace_bytes < gsync_serve_baseline_workspace_bytes(cfg->nreq) || !aligned(workspace, 16))
    return GSYNC_EINVAL;
  if (!buf->pool || !buf->offset || !buf->length || !buf->sched_ns || !buf->res || !buf->done || !buf->latency_ns)
    return GSYNC_EINVAL;
  if (int rc = check_requests(cfg, buf)) return rc;
  unsigned long long* acc = (unsigned long long*)workspace;
  uint32_t* counter = (uint32_t*)(acc + cfg->nreq);
  GSYNC_CUDA(cudaMemsetAsync(workspace, 0, gsync_serve_baseline_workspace_bytes(cfg->nreq), (cudaStream_t)streams[0]));
  GSYNC_CUDA(cudaStreamSynchronize((cudaStream_t)streams[0]));
  for (int q = 0; q < cfg->nreq; ++q) buf->done[q] = 0;
  for (int q = 0; q < cfg->nreq; ++q) buf->latency_ns[q] = 0;
  if (buf->publish_ns)
    for (int q = 0; q < cfg->nreq; ++q) buf->publish_ns[q] = 0;
  std::atomic_thread_fence(std::memory_order_seq_cst);
  void *d_res, *d_done;
  if (int rc = host_dev_ptr(buf->res, &d_res)) return rc;
  if (int rc = host_dev_ptr((void*)buf->done, &d_done)) return rc;
  const Clock::time_point t0 = Clock::now();
  HostCounter completed_c, published_c;
  HostFlag abort_f;
  std::atomic<int>& completed = completed_c.v;
  std::atomic<int>& published = published_c.v;
  std::atomic<bool>& abort_flag = abort_f.v;
  std::thread collector(collect, cfg, buf->done, t0, buf->sched_ns, buf->latency_ns, &completed, &abort_flag,
                        &published);
  pin_to_core_from_end(collector, 1);
  int dev = 0;
  GSYNC_CUDA(cudaGetDevice(&dev));
  std::atomic<int> launch_rc{GSYNC_OK};
  // The launching loop runs on its own pinned core, like the persistent loop's producer.
  std::thread launcher([&]() {
    if (cudaSetDevice(dev) != cudaSuccess) {
      launch_rc.store(GSYNC_ECUDA);
      return;
    }
    for (int q = 0; q < cfg->nreq; ++q) {
      spin_until(t0 + std::chrono::nanoseconds(buf->sched_ns[q]));
      const int64_t len = buf->length[q];
      const unsigned nb = (unsigned)((len + cfg->chunk_elems - 1) / cfg->chunk_elems);
      segsum_kernel<<<nb, kThreads, 0, (cudaStream_t)streams[q % nstreams]>>>(
          buf->pool, buf->offset[q], len, (uint32_t)cfg->chunk_elems, acc + q, counter + 2 * q, (uint32_t)q,
          (int64_t*)d_res, (uint32_t*)d_done);
      // The collector's scan bound, 16 launches ahead, moved once every 16 launches: a store
      // per launch would bounce the line between this core and the collector's, and this
      // loop is what limits the arm at high rates.
      if ((q & 15) == 0) published.store(std::min(cfg->nreq, q + 16), std::memory_order_release);
      if (buf->publish_ns) buf->publish_ns[q] = now_ns(t0);
      if (cudaGetLastError() != cudaSuccess) {
        launch_rc.store(GSYNC_ECUDA);
        return;
      }
    }
  });
  pin_to_core_from_end(launcher, 0);
  launcher.join();
  int rc = launch_rc.load();
  const auto deadline = Clock::now() + std::chrono::seconds(cfg->drain_timeout_s);
  while (rc == GSYNC_OK && completed.load(std::memory_order_acquire) < cfg->nreq) {
    if (Clock::now() > deadline) rc = GSYNC_ETIMEDOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  abort_flag.store(true);
  collector.join();
  for (int s = 0; s < nstreams; ++s) GSYNC_CUDA(cudaStreamSynchronize((cudaStream_t)streams[s]));
  return rc;
}

namespace {

__global__ void host_pingpong_kernel(uint32_t* words, int iters, uint32_t* status) {
  // words[0]: device -> host, words[32]: host -> device (separate lines).
  const uint64_t deadline = ptx::globaltimer() + 2000000000ull;
  for (int i = 1; i <= iters; ++i) {
    st_release_sys(words, (uint32_t)i);
    uint32_t polls = 0;
    while (ld_acquire_sys(words + 32) != (uint32_t)i) {
      if ((++polls & 63u) == 0 && ptx::globaltimer() > deadline) {
        *status = 1;
        st_release_sys(words, 0xFFFFFFFFu);  // tells the host thread to stop
        return;
      }
    }
  }
}

}  // namespace

extern "C" int gsync_probe_host_pingpong(uint32_t* words, int iters, uint64_t* out_ns, void* stream) {
  if (!words || !out_ns || iters < 1) return GSYNC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  void* dwords = nullptr;
  if (int rc = host_dev_ptr(words, &dwords)) return rc;
  volatile uint32_t* w = words;
  w[0] = 0;
  w[32] = 0;
  w[48] = 0;  // device-side status word
  std::atomic_thread_fence(std::memory_order_seq_cst);
  host_pingpong_kernel<<<1, 1, 0, st>>>((uint32_t*)dwords, iters, (uint32_t*)dwords + 48);
  GSYNC_CUDA(cudaGetLastError());
  const auto deadline = Clock::now() + std::chrono::seconds(5);
  Clock::time_point t0 = Clock::now();
  bool ok = true;
  for (int i = 1; i <= iters && ok; ++i) {
    uint32_t v;
    while ((v = __atomic_load_n(&words[0], __ATOMIC_ACQUIRE)) != (uint32_t)i) {
      if (v == 0xFFFFFFFFu || Clock::now() > deadline) { ok = false; break; }
    }
    if (i == 1) t0 = Clock::now();
    __atomic_store_n(&words[32], (uint32_t)i, __ATOMIC_RELEASE);
  }
  const auto t1 = Clock::now();
  GSYNC_CUDA(cudaStreamSynchronize(st));
  if (!ok || w[48]) return GSYNC_ETIMEDOUT;
  out_ns[0] = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(t1 - t0).count();
  return GSYNC_OK;
}
