// gsync_device.cuh -- device-side inter-block synchronization primitives for sm_103a.
//
// Stuart & Owens, "Efficient Synchronization Primitives for GPUs": barriers, mutexes and
// counting semaphores with *block semantics* (Section 3: one request per block, made by a
// master thread, with __syncthreads arbitrating inside the block).  The API follows the
// paper's listing (Section 5, "API"): Barrier(), Mutex Lock()/Unlock(), Semaphore
// Wait()/Post(), with no non-blocking variants.
//
// Every object lives in caller-owned device memory, laid out by gsync_*_init() (gsync.h):
// line 0 is a read-only header, and every word that blocks contend on sits on its own
// 128-byte line.  A kernel attaches once (gsync::*_attach reads the header into registers)
// and then calls the block-level functions, which all threads of the block must reach.
//
// Memory model (PTX ISA): the paper's "volatile" polls become ld.acquire.gpu, its plain
// release stores become st.release.gpu, and its atomics become atom.{relaxed,acquire,
// acq_rel}.gpu, which make the critical-section data of a block (plain loads and stores by
// any of its threads) visible to the next holder: __syncthreads orders the block's accesses
// before the master's gpu-scope release, and the acquiring master's __syncthreads orders
// them before its threads' accesses.
//
// Every wait is bounded: a wait that sees no progress for the object's timeout (globaltimer
// nanoseconds) sets the object's abort word and returns GSYNC_ETIMEDOUT; waits that see the
// abort word set return GSYNC_EABORTED.  Nothing traps, asserts or spins forever.
#pragma once
#include <stdint.h>

#include "gsync.h"

namespace gsync {

// ---------------------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------------------
namespace ptx {
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.volatile.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint4 ld_relaxed_v4(const uint32_t* p) {
  uint4 v;
  asm volatile("ld.relaxed.gpu.global.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p)
               : "memory");
  return v;
}
__device__ __forceinline__ uint4 ld_acquire_v4(const uint32_t* p) {
  uint4 v;
  asm volatile("ld.acquire.gpu.global.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p)
               : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_v4(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.v4.u32 [%0], {%1, %1, %1, %1};" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t atom_add_acq_rel_u64(uint64_t* p, uint64_t v) {
  uint64_t r;
  asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;" : "=l"(r) : "l"(p), "l"(v) : "memory");
  return r;
}
__device__ __forceinline__ uint64_t atom_add_relaxed_u64(uint64_t* p, uint64_t v) {
  uint64_t r;
  asm volatile("atom.relaxed.gpu.global.add.u64 %0, [%1], %2;" : "=l"(r) : "l"(p), "l"(v) : "memory");
  return r;
}
__device__ __forceinline__ void red_add_release_u64(uint64_t* p, uint64_t v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_volatile(uint32_t* p, uint32_t v) {
  asm volatile("st.volatile.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t atom_add_relaxed(uint32_t* p, uint32_t v) {
  uint32_t r;
  asm volatile("atom.relaxed.gpu.global.add.u32 %0, [%1], %2;" : "=r"(r) : "l"(p), "r"(v) : "memory");
  return r;
}
__device__ __forceinline__ uint32_t atom_add_acquire(uint32_t* p, uint32_t v) {
  uint32_t r;
  asm volatile("atom.acquire.gpu.global.add.u32 %0, [%1], %2;" : "=r"(r) : "l"(p), "r"(v) : "memory");
  return r;
}
__device__ __forceinline__ uint32_t atom_add_release(uint32_t* p, uint32_t v) {
  uint32_t r;
  asm volatile("atom.release.gpu.global.add.u32 %0, [%1], %2;" : "=r"(r) : "l"(p), "r"(v) : "memory");
  return r;
}
__device__ __forceinline__ uint32_t atom_add_acq_rel(uint32_t* p, uint32_t v) {
  uint32_t r;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(r) : "l"(p), "r"(v) : "memory");
  return r;
}
__device__ __forceinline__ void red_add_relaxed(uint32_t* p, uint32_t v) {
  asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_add_release(uint32_t* p, uint32_t v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t atom_cas_acquire(uint32_t* p, uint32_t cmp, uint32_t v) {
  uint32_t r;
  asm volatile("atom.acquire.gpu.global.cas.b32 %0, [%1], %2, %3;" : "=r"(r) : "l"(p), "r"(cmp), "r"(v) : "memory");
  return r;
}
__device__ __forceinline__ uint32_t atom_exch_acquire(uint32_t* p, uint32_t v) {
  uint32_t r;
  asm volatile("atom.acquire.gpu.global.exch.b32 %0, [%1], %2;" : "=r"(r) : "l"(p), "r"(v) : "memory");
  return r;
}
__device__ __forceinline__ uint32_t atom_exch_release(uint32_t* p, uint32_t v) {
  uint32_t r;
  asm volatile("atom.release.gpu.global.exch.b32 %0, [%1], %2;" : "=r"(r) : "l"(p), "r"(v) : "memory");
  return r;
}
__device__ __forceinline__ uint32_t atom_exch_relaxed(uint32_t* p, uint32_t v) {
  uint32_t r;
  asm volatile("atom.relaxed.gpu.global.exch.b32 %0, [%1], %2;" : "=r"(r) : "l"(p), "r"(v) : "memory");
  return r;
}
__device__ __forceinline__ void atom_or_relaxed(uint32_t* p, uint32_t v) {
  asm volatile("red.relaxed.gpu.global.or.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void atom_max_relaxed(uint32_t* p, uint32_t v) {
  asm volatile("red.relaxed.gpu.global.max.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// 128-bit acquire load and release store of one 16-byte-aligned record (two u64 halves, the
// low half at the lower address).  A .b128 access is one memory operation, not two 64-bit
// halves, so a reader that sees one half of a release sees the other.
__device__ __forceinline__ void ld_acquire_b128(const void* p, uint64_t& lo, uint64_t& hi) {
  asm volatile("{\n\t.reg .b128 t;\n\tld.acquire.gpu.global.b128 t, [%2];\n\tmov.b128 {%0, %1}, t;\n\t}"
               : "=l"(lo), "=l"(hi)
               : "l"(p)
               : "memory");
}
__device__ __forceinline__ void st_release_b128(void* p, uint64_t lo, uint64_t hi) {
  asm volatile("{\n\t.reg .b128 t;\n\tmov.b128 t, {%0, %1};\n\tst.release.gpu.global.b128 [%2], t;\n\t}"
               ::"l"(lo), "l"(hi), "l"(p)
               : "memory");
}
// Relaxed forms: the same single 16-byte access, with no ordering of other accesses.
__device__ __forceinline__ void ld_relaxed_b128(const void* p, uint64_t& lo, uint64_t& hi) {
  asm volatile("{\n\t.reg .b128 t;\n\tld.relaxed.gpu.global.b128 t, [%2];\n\tmov.b128 {%0, %1}, t;\n\t}"
               : "=l"(lo), "=l"(hi)
               : "l"(p)
               : "memory");
}
__device__ __forceinline__ void st_relaxed_b128(void* p, uint64_t lo, uint64_t hi) {
  asm volatile("{\n\t.reg .b128 t;\n\tmov.b128 t, {%0, %1};\n\tst.relaxed.gpu.global.b128 [%2], t;\n\t}"
               ::"l"(lo), "l"(hi), "l"(p)
               : "memory");
}
__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint32_t smid() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_nctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
// Generic address of the same shared-memory variable in cluster block `rank` (mapa).
template <typename T>
__device__ __forceinline__ T* map_cluster_rank(T* p, uint32_t rank) {
  uint64_t r;
  asm volatile("mapa.u64 %0, %1, %2;" : "=l"(r) : "l"((uint64_t)p), "r"(rank));
  return (T*)r;
}
// Cluster-scope accesses through generic addresses (shared memory of any block of the
// cluster, reached with mapa).
__device__ __forceinline__ uint32_t atom_add_relaxed_cluster(uint32_t* p, uint32_t v) {
  uint32_t r;
  asm volatile("atom.relaxed.cluster.add.u32 %0, [%1], %2;" : "=r"(r) : "l"(p), "r"(v) : "memory");
  return r;
}
__device__ __forceinline__ uint32_t ld_relaxed_cluster(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.cluster.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t ld_acquire_cluster_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.acquire.cluster.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_cluster_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.release.cluster.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t atom_exch_relaxed_cluster(uint32_t* p, uint32_t v) {
  uint32_t r;
  asm volatile("atom.relaxed.cluster.exch.b32 %0, [%1], %2;" : "=r"(r) : "l"(p), "r"(v) : "memory");
  return r;
}
__device__ __forceinline__ uint32_t atom_cas_relaxed_cluster(uint32_t* p, uint32_t cmp, uint32_t v) {
  uint32_t r;
  asm volatile("atom.relaxed.cluster.cas.b32 %0, [%1], %2, %3;" : "=r"(r) : "l"(p), "r"(cmp), "r"(v) : "memory");
  return r;
}
__device__ __forceinline__ uint64_t ld_relaxed_cluster_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.cluster.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_cluster_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.cluster.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// One 16-byte record in the shared memory of a cluster block, read or written as one relaxed
// 128-bit access at cluster scope (generic address from mapa).
__device__ __forceinline__ void ld_relaxed_cluster_b128(const void* p, uint64_t& lo, uint64_t& hi) {
  asm volatile("{\n\t.reg .b128 t;\n\tld.relaxed.cluster.b128 t, [%2];\n\tmov.b128 {%0, %1}, t;\n\t}"
               : "=l"(lo), "=l"(hi)
               : "l"(p)
               : "memory");
}
__device__ __forceinline__ void st_relaxed_cluster_b128(void* p, uint64_t lo, uint64_t hi) {
  asm volatile("{\n\t.reg .b128 t;\n\tmov.b128 t, {%0, %1};\n\tst.relaxed.cluster.b128 [%2], t;\n\t}"
               ::"l"(lo), "l"(hi), "l"(p)
               : "memory");
}
// Hardware barrier over every thread of every block of the cluster.  The non-.aligned
// forms let threads of a warp arrive from divergent paths.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
}  // namespace ptx

// Wrap-safe "a is after b" for uint32 tickets and epochs (fewer than 2^31 outstanding).
__device__ __forceinline__ bool after(uint32_t a, uint32_t b) { return (int32_t)(a - b) > 0; }

// ---------------------------------------------------------------------------------------
// State layout (words; a line is 32 words = 128 bytes)
// ---------------------------------------------------------------------------------------
enum : uint32_t { kLineWords = 32 };
enum HeaderWord : uint32_t {
  kHdrMagic = 0, kHdrN = 1, kHdrParam = 2, kHdrPolicy = 3, kHdrMinNs = 4, kHdrMaxNs = 5,
  kHdrTimeoutLo = 6, kHdrTimeoutHi = 7, kHdrAbort = 8, kHdrMode = 9,
  kHdrDieOff0 = 10, kHdrDieOff1 = 11,  // COHORT: word offset of each die's local lock
  kHdrSpin = 12,                       // SPIN_THEN_SLEEP backoff: failed attempts before sleeping
};
// COHORT: lines 3-4 hold the die of every SM (one byte per SM id, 256 entries).
enum : uint32_t { kDieTableWord = 3 * kLineWords, kMaxSmIds = 256 };

// Bounded polling: every 32 polls it checks the deadline (set lazily at the first check,
// so an uncontended call never reads the timer) and the object's abort word.
struct Waiter {
  uint64_t deadline = 0;
  uint32_t polls = 0;
  __device__ __forceinline__ int tick(uint64_t timeout_ns, uint32_t* abort_word) {
    if ((++polls & 31u) != 0) return GSYNC_OK;
    const uint64_t now = ptx::globaltimer();
    if (deadline == 0) deadline = now + timeout_ns;
    if (ptx::ld_relaxed(abort_word) != 0) return GSYNC_EABORTED;
    if (now > deadline) {
      ptx::atom_or_relaxed(abort_word, 1u);
      return GSYNC_ETIMEDOUT;
    }
    return GSYNC_OK;
  }
};

struct Backoff {
  uint32_t policy, min_ns, max_ns, spin;
  // Next sleep after `cur`: doubling up to max_ns (exponential), or the paper's cyclic
  // policy that adds min_ns after each failure and wraps back to min_ns past max_ns.
  __device__ __forceinline__ uint32_t next(uint32_t cur) const {
    if (policy == GSYNC_BACKOFF_LINEAR_CYCLIC) {
      const uint32_t n = cur + min_ns;
      return n > max_ns ? min_ns : n;
    }
    const uint32_t n = cur * 2u;
    return n > max_ns ? max_ns : n;
  }
};

__device__ __forceinline__ uint64_t header_timeout(const uint32_t* s) {
  uint64_t t = ((uint64_t)s[kHdrTimeoutHi] << 32) | s[kHdrTimeoutLo];
  return t ? t : 2000000000ull;
}

// ---------------------------------------------------------------------------------------
// Mutex (Section 5 "Mutex"; Appendix: spin-lock mutex, FA mutex)
// ---------------------------------------------------------------------------------------
// line 1: lock word (CAS kinds) or ticket counter (TICKET, SLEEP_QUEUE, COHORT global lock,
//         RING tail)
// line 2: turn (TICKET, COHORT global lock) or head pointer (RING)
// lines 3 .. 3+Q-1: one flag per queue slot (SLEEP_QUEUE) or ring entry (RING), Q = power of
//         two >= waiters
// COHORT: lines 3-4 the SM-to-die table; for each die d, at word offset kHdrDieOff<d> (on a
//   4 KB page homed on die d), a local ticket counter line and a local turn line whose first
//   8 bytes hold {served ticket (low 32), cohort word (high 32)}.
// CLUSTER: the same protocol with the thread-block cluster as the group: lines 1-2 hold the
//   global ticket lock and each cluster's local lock is a ClusterLocal in the shared memory
//   of the cluster's block 0 (see mutex_attach_cluster).
// CLUSTER_MCS: lines 1-2 the global ticket lock; the cluster's local lock is an MCS queue of
//   McsNode, one in each block's shared memory (see mutex_attach_cluster_mcs).
// The local lock of a CLUSTER mutex, declared __shared__ by the kernel.
struct ClusterLocal {
  uint32_t next;
  uint32_t pad;
  uint64_t turn;  // {served ticket (low 32), cohort word (high 32)}
};
// CLUSTER_MCS: each block's node of the cluster's MCS queue, declared __shared__ by the kernel
// (see mutex_attach_cluster_mcs).  Block 0's `tail` names the last block to queue; every
// block's `link` is written by its successor and `rec` by its predecessor, and `seq` counts
// the block's own queueings (only its thread 0 touches it).
struct McsNode {
  uint32_t tail;  // block 0 only: (rank + 1) | seq << 4 of the last block to queue, 0 = free
  uint32_t seq;
  uint64_t link;  // successor's rank | successor's seq << 4 | this block's seq << 32
  uint64_t rec;   // the grant: seq (bits 0-15) | owned (16) | passes (17-31) | global ticket (32-47)
  uint64_t pad;
};

struct MutexRef {
  uint32_t* s;
  uint32_t kind, qmask;
  Backoff bo;
  uint64_t timeout_ns;
  uint32_t* local;  // COHORT: this block's die's local lock (counter line, then turn line)
  uint32_t die;     // COHORT: the die of this block's SM (0 or 1)
  ClusterLocal* cl; // CLUSTER: the cluster's local lock (in block 0's shared memory)
  McsNode* mcs;     // CLUSTER_MCS: this block's own node
  uint32_t* mcs_tail;  // CLUSTER_MCS: the cluster's tail (in block 0's shared memory)
  __device__ __forceinline__ uint32_t* lockw() const { return s + 1 * kLineWords; }
  __device__ __forceinline__ uint32_t* turn() const { return s + 2 * kLineWords; }
  __device__ __forceinline__ uint32_t* flag(uint32_t t) const { return s + (3 + (t & qmask)) * kLineWords; }
  __device__ __forceinline__ uint32_t* abort_word() const { return s + kHdrAbort; }
  __device__ __forceinline__ uint32_t* local_next() const { return local; }
  __device__ __forceinline__ uint64_t* local_turn() const { return (uint64_t*)(local + kLineWords); }
  __device__ __forceinline__ uint32_t budget() const { return qmask + 1u; }
};

__device__ __forceinline__ MutexRef mutex_attach(void* state) {
  MutexRef m;
  m.s = (uint32_t*)state;
  m.kind = m.s[kHdrMagic] & 0xFFu;
  m.qmask = m.s[kHdrParam] ? m.s[kHdrParam] - 1u : 0u;
  m.bo.policy = m.s[kHdrPolicy];
  m.bo.min_ns = m.s[kHdrMinNs];
  m.bo.max_ns = m.s[kHdrMaxNs];
  m.bo.spin = m.s[kHdrSpin];
  m.timeout_ns = header_timeout(m.s);
  m.local = nullptr;
  m.cl = nullptr;
  m.mcs = nullptr;
  m.mcs_tail = nullptr;
  m.die = 0;
  if (m.kind == GSYNC_MUTEX_COHORT) {
    const uint32_t sm = ptx::smid();
    const uint8_t* table = (const uint8_t*)(m.s + kDieTableWord);
    m.die = (sm < kMaxSmIds && table[sm]) ? 1u : 0u;
    m.local = m.s + m.s[m.die ? kHdrDieOff1 : kHdrDieOff0];
  }
  return m;
}

// CLUSTER mutex: every thread of every block of the (cluster-launched) grid calls this at the
// kernel's start with the same __shared__ ClusterLocal; it initialises block 0's copy and
// crosses the hardware cluster barrier, so the local lock is ready before anyone uses it.
// The kernel must call mutex_cluster_end() before any of its blocks exits: block 0's shared
// memory has to outlive the other blocks' last access to it.
__device__ __forceinline__ MutexRef mutex_attach_cluster(void* state, ClusterLocal* local) {
  MutexRef m = mutex_attach(state);
  if (ptx::cluster_ctarank() == 0 && threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) {
    local->next = 0;
    local->turn = 0;
  }
  m.cl = ptx::map_cluster_rank(local, 0u);
  ptx::cluster_sync();
  return m;
}
__device__ __forceinline__ void mutex_cluster_end() { ptx::cluster_sync(); }

// CLUSTER_MCS mutex: every thread of every block of the (cluster-launched) grid calls this at
// the kernel's start with the same __shared__ McsNode; each block clears its own node, and the
// hardware cluster barrier makes the nodes ready before anyone queues.  The kernel must call
// mutex_cluster_end() before any of its blocks exits (its node is written by its neighbours).
__device__ __forceinline__ MutexRef mutex_attach_cluster_mcs(void* state, McsNode* node) {
  MutexRef m = mutex_attach(state);
  if (threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) {
    node->tail = 0u;
    node->seq = 0u;
    node->link = 0ull;
    node->rec = 0ull;
  }
  m.mcs = node;
  m.mcs_tail = &ptx::map_cluster_rank(node, 0u)->tail;
  ptx::cluster_sync();
  return m;
}

// Result of a lock: the status, the ticket the holder needs to unlock, and (COHORT) the
// cohort word -- passes within the die so far (bits 30..16) and the global ticket (15..0) --
// and the die's ticket counter as read right after the lock was taken.
struct Token {
  int status;
  uint32_t ticket;
  uint32_t cohort;
  uint32_t next_seen;
};

// RING: the value of an empty ring entry (block ids are below it).
enum : uint32_t { kRingEmpty = 0xFFFFFFFFu };

// COHORT local turn word: bit 31 of the high half says the cohort already holds the global
// lock (the next local holder inherits it instead of queueing for it).
enum : uint32_t { kCohortOwned = 0x80000000u };
// CLUSTER_MCS record: bit 16 says the cluster already holds the global lock.
constexpr uint64_t kMcsOwned = 1ull << 16;

// Master-thread lock.  Returns the ticket (ticket kinds) in tok.ticket.
template <int KIND>
__device__ __forceinline__ Token mutex_lock_thread(const MutexRef& m) {
  Waiter w;
  if (KIND == GSYNC_MUTEX_CAS_SPIN || KIND == GSYNC_MUTEX_CAS_BACKOFF) {
    // Algorithm 1 / spin-lock mutex: swap 1 in until the old value was 0 (atomicCAS form).
    // SPIN_THEN_SLEEP (Section 5's stand-in for a futex) spins `spin` failed attempts first.
    uint32_t sleep_ns = m.bo.min_ns;
    uint32_t spins = m.bo.policy == GSYNC_BACKOFF_SPIN_THEN_SLEEP ? m.bo.spin : 0u;
    while (ptx::atom_cas_acquire(m.lockw(), 0u, 1u) != 0u) {
      if (int rc = w.tick(m.timeout_ns, m.abort_word())) return {rc, 0u};
      if (KIND == GSYNC_MUTEX_CAS_BACKOFF) {
        if (spins) {
          --spins;
          continue;
        }
        __nanosleep(sleep_ns);
        sleep_ns = m.bo.next(sleep_ns);
      }
    }
    return {GSYNC_OK, 0xFFFFFFFFu};
  } else if (KIND == GSYNC_MUTEX_TICKET) {
    // FA mutex: take a ticket, poll the turn; sleep in proportion to the queue ahead.
    const uint32_t t = ptx::atom_add_relaxed(m.lockw(), 1u);
    uint32_t cur;
    while ((cur = ptx::ld_acquire(m.turn())) != t) {
      if (int rc = w.tick(m.timeout_ns, m.abort_word())) return {rc, t};
      const uint32_t ahead = t - cur;
      if (m.bo.min_ns && ahead > 1u && ahead < 0x80000000u) {
        const uint32_t ns = (ahead - 1u) * m.bo.min_ns;
        __nanosleep(ns < m.bo.max_ns ? ns : m.bo.max_ns);
      }
    }
    return {GSYNC_OK, t};
  } else if (KIND == GSYNC_MUTEX_COHORT) {
    // Lock cohorting (Dice, Marathe and Shavit, PPoPP 2012) over GB300's two dies: a ticket
    // lock per die, on a line homed on that die, and a global ticket lock between the dies.
    // A holder passes the lock to the next waiter of its own die -- a hand-off that never
    // leaves the die -- up to `budget` times in a row, with the global lock passed along.
    const uint32_t t = ptx::atom_add_relaxed(m.local_next(), 1u);
    uint64_t v;
    while ((uint32_t)(v = ptx::ld_acquire_u64(m.local_turn())) != t) {
      if (int rc = w.tick(m.timeout_ns, m.abort_word())) return {rc, t, 0u};
      const uint32_t ahead = t - (uint32_t)v;
      if (m.bo.min_ns && ahead > 1u && ahead < 0x80000000u) {
        const uint32_t ns = (ahead - 1u) * m.bo.min_ns;
        __nanosleep(ns < m.bo.max_ns ? ns : m.bo.max_ns);
      }
    }
    // The read of the die's ticket counter (is anyone queued behind?) is issued now and only
    // consumed at unlock, so its round trip overlaps the critical section.
    const uint32_t word = (uint32_t)(v >> 32);
    if (word & kCohortOwned) return {GSYNC_OK, t, word & ~kCohortOwned, ptx::ld_relaxed(m.local_next())};
    // First of a cohort: queue for the global lock (at most one waiter per die).
    const uint32_t g = ptx::atom_add_relaxed(m.lockw(), 1u) & 0xFFFFu;
    while ((ptx::ld_acquire(m.turn()) & 0xFFFFu) != g) {
      if (int rc = w.tick(m.timeout_ns, m.abort_word())) return {rc, t, 0u};
      if (m.bo.min_ns) __nanosleep(m.bo.min_ns);
    }
    return {GSYNC_OK, t, g, ptx::ld_relaxed(m.local_next())};
  } else if (KIND == GSYNC_MUTEX_CLUSTER) {
    // The cohort protocol with the cluster as the group: the local ticket lock lives in the
    // shared memory of the cluster's block 0 and is passed with cluster-scope release and
    // acquire (distributed shared memory); the global ticket lock is passed between clusters.
    const uint32_t t = ptx::atom_add_relaxed_cluster(&m.cl->next, 1u);
    uint64_t v;
    while ((uint32_t)(v = ptx::ld_acquire_cluster_u64(&m.cl->turn)) != t) {
      if (int rc = w.tick(m.timeout_ns, m.abort_word())) return {rc, t, 0u};
      const uint32_t ahead = t - (uint32_t)v;
      if (m.bo.min_ns && ahead > 1u && ahead < 0x80000000u) {
        const uint32_t ns = (ahead - 1u) * m.bo.min_ns;
        __nanosleep(ns < m.bo.max_ns ? ns : m.bo.max_ns);
      }
    }
    const uint32_t word = (uint32_t)(v >> 32);
    if (word & kCohortOwned) return {GSYNC_OK, t, word & ~kCohortOwned, ptx::ld_relaxed_cluster(&m.cl->next)};
    const uint32_t g = ptx::atom_add_relaxed(m.lockw(), 1u) & 0xFFFFu;
    while ((ptx::ld_acquire(m.turn()) & 0xFFFFu) != g) {
      if (int rc = w.tick(m.timeout_ns, m.abort_word())) return {rc, t, 0u};
      if (m.bo.min_ns) __nanosleep(m.bo.min_ns);
    }
    return {GSYNC_OK, t, g, ptx::ld_relaxed_cluster(&m.cl->next)};
  } else if (KIND == GSYNC_MUTEX_CLUSTER_MCS) {
    // The cohort protocol with an MCS queue (Mellor-Crummey and Scott, 1991) as the cluster's
    // local lock: swap this block into the cluster's tail, link into the predecessor's node,
    // and spin on a record in this block's own shared memory, which the predecessor pushes
    // with a cluster-scope release.  Nothing is reset between rounds: the node's link and
    // record carry sequence numbers (this block's count of queueings) and are checked
    // against them.  A grant that is not owned (or a free queue) sends the block on to the
    // global ticket lock, as in CLUSTER.
    const uint32_t me = ptx::cluster_ctarank();
    const uint32_t seq = ++m.mcs->seq;
    const uint32_t prev = ptx::atom_exch_relaxed_cluster(m.mcs_tail, (me + 1u) | (seq << 4));
    if (prev != 0u) {
      McsNode* pn = ptx::map_cluster_rank(m.mcs, (prev & 0xFu) - 1u);
      ptx::st_relaxed_cluster_u64(&pn->link, (uint64_t)me | ((uint64_t)seq << 4) | ((uint64_t)(prev >> 4) << 32));
      uint64_t r;
      while ((((uint32_t)(r = ptx::ld_acquire_cluster_u64(&m.mcs->rec))) ^ seq) & 0xFFFFu) {
        if (int rc = w.tick(m.timeout_ns, m.abort_word())) return {rc, seq, 0u};
      }
      if (r & kMcsOwned) return {GSYNC_OK, seq, (uint32_t)(r >> 32) | (((uint32_t)(r >> 17) & 0x7FFFu) << 16), 0u};
    }
    const uint32_t g = ptx::atom_add_relaxed(m.lockw(), 1u) & 0xFFFFu;
    while ((ptx::ld_acquire(m.turn()) & 0xFFFFu) != g) {
      if (int rc = w.tick(m.timeout_ns, m.abort_word())) return {rc, seq, 0u};
      if (m.bo.min_ns) __nanosleep(m.bo.min_ns);
    }
    return {GSYNC_OK, seq, g, 0u};
  } else if (KIND == GSYNC_MUTEX_RING) {
    // Ring-buffer sleeping mutex (Section 5, design alternative): claim the ring's end with a
    // fetch-and-add on the tail, write this block's id there, then poll the head pointer and
    // the entry it names until that entry is this block.  Two reads per poll, as Section 5
    // counts against it.
    const uint32_t t = ptx::atom_add_relaxed(m.lockw(), 1u);
    const uint32_t me = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    ptx::st_relaxed(m.flag(t), me);
    for (;;) {
      const uint32_t h = ptx::ld_acquire(m.turn());
      if (ptx::ld_acquire(m.flag(h)) == me) break;
      if (int rc = w.tick(m.timeout_ns, m.abort_word())) return {rc, t};
      if (m.bo.min_ns) __nanosleep(m.bo.min_ns);
    }
    return {GSYNC_OK, t};
  } else {
    // Queue lock: take a slot, poll the slot's own flag until it holds this ticket.
    const uint32_t t = ptx::atom_add_relaxed(m.lockw(), 1u);
    uint32_t* f = m.flag(t);
    while (ptx::ld_acquire(f) != t) {
      if (int rc = w.tick(m.timeout_ns, m.abort_word())) return {rc, t};
      if (m.bo.min_ns) __nanosleep(m.bo.min_ns);
    }
    return {GSYNC_OK, t};
  }
}

// COHORT / CLUSTER: `pass_local` = false releases the global lock even when a waiter of the
// same group is queued (a condition-variable wait uses it: see cond_wait_thread).
template <int KIND>
__device__ __forceinline__ void mutex_unlock_thread(const MutexRef& m, const Token& tok, bool pass_local = true) {
  const uint32_t ticket = tok.ticket;
  if (KIND == GSYNC_MUTEX_CAS_SPIN || KIND == GSYNC_MUTEX_CAS_BACKOFF) {
    ptx::st_release(m.lockw(), 0u);
  } else if (KIND == GSYNC_MUTEX_TICKET) {
    ptx::st_release(m.turn(), ticket + 1u);  // only the holder writes turn: no atomic
  } else if (KIND == GSYNC_MUTEX_COHORT) {
    // A waiter of this die holds ticket + 1 iff the local counter moved past it: known from
    // the read made at lock time, else read again now.  One that arrives after the read
    // finds the global lock released and queues for it: safe.
    const uint32_t passes = (tok.cohort >> 16) & 0x7FFFu, g = tok.cohort & 0xFFFFu;
    const bool may_pass = pass_local && passes + 1u < m.budget();
    const bool local_waiter =
        may_pass && (tok.next_seen != ticket + 1u || ptx::ld_relaxed(m.local_next()) != ticket + 1u);
    if (local_waiter) {
      const uint32_t word = kCohortOwned | ((passes + 1u) << 16) | g;
      ptx::st_release_u64(m.local_turn(), ((uint64_t)word << 32) | (ticket + 1u));
    } else {
      ptx::st_release(m.turn(), (g + 1u) & 0xFFFFu);
      ptx::st_release_u64(m.local_turn(), (uint64_t)(ticket + 1u));
    }
  } else if (KIND == GSYNC_MUTEX_CLUSTER) {
    const uint32_t passes = (tok.cohort >> 16) & 0x7FFFu, g = tok.cohort & 0xFFFFu;
    const bool may_pass = pass_local && passes + 1u < m.budget();
    const bool local_waiter =
        may_pass && (tok.next_seen != ticket + 1u || ptx::ld_relaxed_cluster(&m.cl->next) != ticket + 1u);
    if (local_waiter) {
      const uint32_t word = kCohortOwned | ((passes + 1u) << 16) | g;
      ptx::st_release_cluster_u64(&m.cl->turn, ((uint64_t)word << 32) | (ticket + 1u));
    } else {
      ptx::st_release(m.turn(), (g + 1u) & 0xFFFFu);
      ptx::st_release_cluster_u64(&m.cl->turn, (uint64_t)(ticket + 1u));
    }
  } else if (KIND == GSYNC_MUTEX_CLUSTER_MCS) {
    // Pass to the linked successor (owned: the global lock stays with the cluster) while the
    // budget allows; else release the global lock, then free the cluster's queue: push a
    // record that is not owned to the successor, or swap the tail back to empty if it still
    // names this block, or else wait (bounded) for the successor that swapped in to link.
    const uint32_t passes = (tok.cohort >> 16) & 0x7FFFu, g = tok.cohort & 0xFFFFu, seq = ticket;
    uint64_t link = ptx::ld_relaxed_cluster_u64(&m.mcs->link);
    bool linked = (uint32_t)(link >> 32) == seq;
    if (linked && pass_local && passes + 1u < m.budget()) {
      McsNode* sn = ptx::map_cluster_rank(m.mcs, (uint32_t)link & 0xFu);
      ptx::st_release_cluster_u64(&sn->rec, (uint64_t)(((uint32_t)link >> 4) & 0xFFFFu) | kMcsOwned |
                                                ((uint64_t)(passes + 1u) << 17) | ((uint64_t)g << 32));
      return;
    }
    ptx::st_release(m.turn(), (g + 1u) & 0xFFFFu);
    if (!linked) {
      const uint32_t mine = (ptx::cluster_ctarank() + 1u) | (seq << 4);
      if (ptx::atom_cas_relaxed_cluster(m.mcs_tail, mine, 0u) == mine) return;
      Waiter w;
      while ((uint32_t)((link = ptx::ld_relaxed_cluster_u64(&m.mcs->link)) >> 32) != seq)
        if (w.tick(m.timeout_ns, m.abort_word())) return;  // the successor times out in turn
    }
    McsNode* sn = ptx::map_cluster_rank(m.mcs, (uint32_t)link & 0xFu);
    ptx::st_relaxed_cluster_u64(&sn->rec, (uint64_t)(((uint32_t)link >> 4) & 0xFFFFu));
  } else if (KIND == GSYNC_MUTEX_RING) {
    // Clear this block's entry before moving the head past it, so that no block can match
    // its own id left over from an earlier lap of the ring.
    ptx::st_relaxed(m.flag(ticket), kRingEmpty);
    ptx::st_release(m.turn(), ticket + 1u);
  } else {
    ptx::st_release(m.flag(ticket + 1u), ticket + 1u);
  }
}

// Ticket-only form for the kinds whose unlock needs nothing but the ticket.
template <int KIND>
__device__ __forceinline__ void mutex_unlock_thread(const MutexRef& m, uint32_t ticket) {
  static_assert(KIND != GSYNC_MUTEX_COHORT && KIND != GSYNC_MUTEX_CLUSTER && KIND != GSYNC_MUTEX_CLUSTER_MCS,
                "a cohort unlock needs the whole Token");
  mutex_unlock_thread<KIND>(m, Token{GSYNC_OK, ticket, 0u, 0u});
}

// Block-level lock (all threads): thread 0 acquires, the block then proceeds together.
// Only the status is shared; the rest of the token stays in thread 0's registers, the thread
// that unlocks (so a read it issued while locking can still be in flight).
template <int KIND>
__device__ __forceinline__ Token mutex_lock(const MutexRef& m) {
  __shared__ int s_status;
  Token t{GSYNC_OK, 0u, 0u, 0u};
  if (threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) {
    t = mutex_lock_thread<KIND>(m);
    s_status = t.status;
  }
  __syncthreads();
  t.status = s_status;
  return t;
}

// Block-level lock with a wait bound for this call (ns), instead of the object's own: on
// expiry the call returns GSYNC_ETIMEDOUT and, as any timed-out wait does, marks the object
// aborted (an abandoned ticket leaves the lock unusable).
template <int KIND>
__device__ __forceinline__ Token mutex_lock(const MutexRef& m, uint64_t timeout_ns) {
  MutexRef bounded = m;
  bounded.timeout_ns = timeout_ns;
  return mutex_lock<KIND>(bounded);
}

// Block-level unlock: the block's critical-section accesses complete before the release.
template <int KIND>
__device__ __forceinline__ void mutex_unlock(const MutexRef& m, Token t) {
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) mutex_unlock_thread<KIND>(m, t);
}

// ---------------------------------------------------------------------------------------
// Condition variable (named as future work in Section 7; the paper gives no algorithm)
// ---------------------------------------------------------------------------------------
// line 1: tickets (waiters so far), line 2: signals (waiters released so far).  A waiter
// takes its ticket while it still holds the mutex, so a signal made under the mutex after
// the waiter's release cannot be lost; signal and broadcast must be called with the mutex
// held, which also makes them plain (non-atomic) updates.  Waiters are released in ticket
// order; a signal with no waiter does nothing.
struct CondRef {
  uint32_t* s;
  Backoff bo;
  uint64_t timeout_ns;
  __device__ __forceinline__ uint32_t* tickets() const { return s + 1 * kLineWords; }
  __device__ __forceinline__ uint32_t* signals() const { return s + 2 * kLineWords; }
  __device__ __forceinline__ uint32_t* abort_word() const { return s + kHdrAbort; }
};

__device__ __forceinline__ CondRef cond_attach(void* state) {
  CondRef c;
  c.s = (uint32_t*)state;
  c.bo.policy = c.s[kHdrPolicy];
  c.bo.min_ns = c.s[kHdrMinNs];
  c.bo.max_ns = c.s[kHdrMaxNs];
  c.bo.spin = 0;
  c.timeout_ns = header_timeout(c.s);
  return c;
}

// Thread 0, holding mutex m with token tok: waits on cv and returns holding m again (tok is
// the new token).  Releases m, polls the signals counter past its ticket, takes m again.
template <int MKIND>
__device__ __forceinline__ int cond_wait_thread(const CondRef& cv, const MutexRef& m, Token& tok) {
  const uint32_t t = ptx::ld_relaxed(cv.tickets());
  ptx::st_relaxed(cv.tickets(), t + 1u);  // under the mutex: no other writer
  // The cluster cohort lock releases its global lock here rather than passing within the
  // cluster: the waiter waits for a block that changes the condition, and a cluster's few
  // neighbouring blocks often share one role (all producers, say), so they would each take
  // the lock only to wait in turn, keeping it from the blocks that could signal.  A die holds
  // half the grid, of mixed roles, and the two-die cohort lock keeps passing within the die
  // (measured faster on the producer/consumer workload; the cluster lock gains ~25 % here).
  mutex_unlock_thread<MKIND>(m, tok, MKIND != GSYNC_MUTEX_CLUSTER && MKIND != GSYNC_MUTEX_CLUSTER_MCS);
  Waiter w;
  uint32_t sleep_ns = cv.bo.min_ns;
  while (!after(ptx::ld_acquire(cv.signals()), t)) {
    if (int rc = w.tick(cv.timeout_ns, cv.abort_word())) return rc;
    if (sleep_ns) {
      __nanosleep(sleep_ns);
      sleep_ns = cv.bo.next(sleep_ns);
    }
  }
  tok = mutex_lock_thread<MKIND>(m);
  return tok.status;
}

// Thread 0, holding the mutex: release the oldest waiter, if any.
__device__ __forceinline__ void cond_signal_thread(const CondRef& cv) {
  const uint32_t sg = ptx::ld_relaxed(cv.signals()), tk = ptx::ld_relaxed(cv.tickets());
  if (sg != tk) ptx::st_relaxed(cv.signals(), sg + 1u);
}

// The two counters a signal reads.  Only holders of the mutex write them, so a snapshot that
// thread 0 takes while it holds the mutex stays exact until it releases the mutex (waiting on
// any condition variable releases it too).  Taking the snapshot together with the critical
// section's own first loads puts the signal's round trip in their shadow.
struct CondSnap {
  uint32_t signals, tickets;
};
__device__ __forceinline__ CondSnap cond_snapshot_thread(const CondRef& cv) {
  return CondSnap{ptx::ld_relaxed(cv.signals()), ptx::ld_relaxed(cv.tickets())};
}
// Thread 0, holding the mutex without a break since it took `snap` of cv: as cond_signal_thread.
__device__ __forceinline__ void cond_signal_thread(const CondRef& cv, CondSnap snap) {
  if (snap.signals != snap.tickets) ptx::st_relaxed(cv.signals(), snap.signals + 1u);
}

// Thread 0, holding the mutex: release every waiter.
__device__ __forceinline__ void cond_broadcast_thread(const CondRef& cv) {
  ptx::st_relaxed(cv.signals(), ptx::ld_relaxed(cv.tickets()));
}

// Block-level wait: all threads call it while the block holds m (the block's accesses before
// the call are released with the mutex); returns holding m, with t the new token in thread 0.
template <int MKIND>
__device__ __forceinline__ int cond_wait(const CondRef& cv, const MutexRef& m, Token& t) {
  __shared__ int s_rc;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) s_rc = cond_wait_thread<MKIND>(cv, m, t);
  __syncthreads();
  const int rc = s_rc;
  return rc;
}

// ---------------------------------------------------------------------------------------
// Counting semaphore (Section 5 "Semaphore"; Appendix: spin-lock and sleeping semaphores)
// ---------------------------------------------------------------------------------------
// TICKET (sleeping): line 1 count, line 2 ticket, line 3 turn; header N = max count.
// SPIN / SPIN_BACKOFF: line 1 S (initially N + 1; 0 while a block updates it).
// WINDOW: line 1 ticket, line 2 turn (the number of posts); the holders are the tickets in
//   [turn, turn + N).  Not in the paper: its FA semaphore's post must learn from the count
//   whether anyone waits (a round trip to L2) before it may advance the turn; here the post
//   only advances the turn, and the wait pays for it with a load of the turn issued beside
//   its ticket fetch-and-add.
struct SemRef {
  uint32_t* s;
  uint32_t kind, n;
  Backoff bo;
  uint64_t timeout_ns;
  __device__ __forceinline__ uint32_t* word(int line) const { return s + line * kLineWords; }
  __device__ __forceinline__ uint32_t* abort_word() const { return s + kHdrAbort; }
};

__device__ __forceinline__ SemRef sem_attach(void* state) {
  SemRef r;
  r.s = (uint32_t*)state;
  r.kind = r.s[kHdrMagic] & 0xFFu;
  r.n = r.s[kHdrN];
  r.bo.policy = r.s[kHdrPolicy];
  r.bo.min_ns = r.s[kHdrMinNs];
  r.bo.max_ns = r.s[kHdrMaxNs];
  r.bo.spin = r.s[kHdrSpin];
  r.timeout_ns = header_timeout(r.s);
  return r;
}

template <int KIND>
__device__ __forceinline__ int sem_wait_thread(const SemRef& s) {
  Waiter w;
  if (KIND == GSYNC_SEM_TICKET) {
    // One atomic when under capacity; otherwise take a wait ticket and poll the turn.
    const uint32_t old = ptx::atom_add_acquire(s.word(1), 1u);
    if ((int32_t)old < (int32_t)s.n) return GSYNC_OK;
    const uint32_t wi = ptx::atom_add_relaxed(s.word(2), 1u);
    uint32_t turn;
    while (!after(turn = ptx::ld_acquire(s.word(3)), wi)) {
      if (int rc = w.tick(s.timeout_ns, s.abort_word())) return rc;
      // Sleep in proportion to the waiters ahead (wi - turn of them), capped at max_ns.
      const uint32_t ahead = wi - turn;
      if (s.bo.min_ns && ahead < 0x80000000u) {
        const uint32_t ns = ahead * s.bo.min_ns;
        __nanosleep(ns < s.bo.max_ns ? ns : s.bo.max_ns);
      }
    }
    return GSYNC_OK;
  } else if (KIND == GSYNC_SEM_WINDOW) {
    // The load of the turn does not wait for the ticket's return (the fetch-and-add is
    // relaxed; the acquire is the load's).  A turn read early is smaller, so it can only
    // delay the entry, never allow one too many.
    const uint32_t t = ptx::atom_add_relaxed(s.word(1), 1u);
    uint32_t turn = ptx::ld_acquire(s.word(2));
    while (!after(turn + s.n, t)) {
      if (int rc = w.tick(s.timeout_ns, s.abort_word())) return rc;
      // Sleep in proportion to the holders that must leave before this ticket's turn.
      const uint32_t ahead = t - (turn + s.n) + 1u;
      if (s.bo.min_ns && ahead < 0x80000000u) {
        const uint32_t ns = ahead * s.bo.min_ns;
        __nanosleep(ns < s.bo.max_ns ? ns : s.bo.max_ns);
      }
      turn = ptx::ld_acquire(s.word(2));
    }
    return GSYNC_OK;
  } else {
    uint32_t sleep_ns = s.bo.min_ns;
    for (;;) {
      const uint32_t v = ptx::atom_exch_acquire(s.word(1), 0u);
      if (v > 1u) {
        ptx::atom_exch_relaxed(s.word(1), v - 1u);
        return GSYNC_OK;
      }
      if (v == 1u) ptx::atom_exch_relaxed(s.word(1), 1u);
      if (int rc = w.tick(s.timeout_ns, s.abort_word())) return rc;
      if (KIND == GSYNC_SEM_SPIN_BACKOFF) {
        __nanosleep(sleep_ns);
        sleep_ns = s.bo.next(sleep_ns);
      }
    }
  }
}

template <int KIND>
__device__ __forceinline__ int sem_post_thread(const SemRef& s) {
  if (KIND == GSYNC_SEM_TICKET) {
    // One release fence covers both writes: each strong write after it is a release.
    ptx::fence_acq_rel();
    const uint32_t old = ptx::atom_add_relaxed(s.word(1), 0xFFFFFFFFu);
    if ((int32_t)old > (int32_t)s.n) ptx::red_add_relaxed(s.word(3), 1u);
    return GSYNC_OK;
  } else if (KIND == GSYNC_SEM_WINDOW) {
    ptx::red_add_release(s.word(2), 1u);  // no return trip: the poster goes on at once
    return GSYNC_OK;
  } else {
    Waiter w;
    for (;;) {
      const uint32_t v = ptx::atom_exch_acquire(s.word(1), 0u);
      if (v > 0u) {
        ptx::atom_exch_release(s.word(1), v + 1u);
        return GSYNC_OK;
      }
      if (int rc = w.tick(s.timeout_ns, s.abort_word())) return rc;
    }
  }
}

template <int KIND>
__device__ __forceinline__ int sem_wait(const SemRef& s) {
  __shared__ int s_rc;
  if (threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) s_rc = sem_wait_thread<KIND>(s);
  __syncthreads();
  const int rc = s_rc;
  return rc;
}

// Block-level wait with a wait bound for this call (ns): GSYNC_ETIMEDOUT on expiry, and the
// object is marked aborted (a ticket taken and abandoned holds a permit forever).
template <int KIND>
__device__ __forceinline__ int sem_wait(const SemRef& s, uint64_t timeout_ns) {
  SemRef bounded = s;
  bounded.timeout_ns = timeout_ns;
  return sem_wait<KIND>(bounded);
}

template <int KIND>
__device__ __forceinline__ int sem_post(const SemRef& s) {
  __shared__ int s_rc;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) s_rc = sem_post_thread<KIND>(s);
  __syncthreads();
  const int rc = s_rc;
  return rc;
}

// ---------------------------------------------------------------------------------------
// Grid barrier (Section 5 "Barrier"): every block of the grid participates.
// ---------------------------------------------------------------------------------------
// ATOMIC : lines 1 and 3 arrival counters (odd and even epochs), line 2 release epoch.
// FLAG   : lines 1.. arrival flags (one word per block, packed), then release flags (one
//          word per block, packed; mode 1: a single release word on its own line).  At most
//          8192 blocks; the master block's threads gather the flags.
// TREE   : param = fan | form << 16.  Lines 2.. one counter line per tree node, level by
//          level, the root last.  Form 0: line 1 the release epoch; the last arriver at a node
//          resets it and counts in at the parent, and the root's last arriver advances the
//          epoch, which every block polls.  Form 1 (counting): 64-bit node counters that only
//          grow; the arrival that brings a node to a multiple of its size is its last one and
//          counts in at the parent, and the root's last add is the release: every other block
//          polls the root until base + e x (root's size).
// SHARDED: lines 1..S: S = param arrival counters (block b counts into counter b mod S with a
//          fire-and-forget red.release; counters only grow, so after crossing e counter s
//          holds e x (blocks of shard s)); then release flags (one word per block, packed).
//          Warp 0 of block 0 watches the S counters and writes the release flags.
// CLUSTER: param = c | form << 4 | sleep << 8, c the cluster size (1..8).  Its first stage is
//          the hardware cluster barrier, which cannot time out: every block of a cluster must
//          make the same number of barrier_wait calls, also after one returned an error (the
//          object's abort word makes those calls return quickly).  Then, by form:
//          0: ATOMIC over the cluster leaders (lines 1 and 3 arrival counters, line 2 the
//             release epoch), which every block polls;
//          1: counting over the leaders: line 1 a 64-bit counter that only grows; each leader
//             adds 1 per crossing, and every block polls it until base + e x (n / c), so the
//             last leader's add is the release (as COUNT); a leader sleeps `sleep` ns per 16
//             leader arrivals still missing before its first poll;
//          2: as 1, but only the leader polls; the other blocks of its cluster wait at a
//             second hardware cluster barrier, which the leader reaches once it has seen the
//             crossing complete (and they take its result from its shared memory).
// DIE    : line 1 a flat arrival counter (registration crossings), line 2 {members of die
//          0, members of die 1, blocks of die 0, blocks of die 1, dies with blocks}, lines
//          3-4 the SM-to-die table; for each die d, at word offset kHdrDieOff<d> (on a 4 KB
//          page homed on die d): line 0 the arrival counter of odd epochs, line 1 the
//          release epoch, line 3 the arrival counter of even epochs; die 0's lines 2 and 4
//          are the top counters of odd and even epochs.  A block's first crossing of a launch
//          registers it (flat count, membership per die); later crossings count in per die,
//          and the second die to finish releases both.  param 1: every crossing counts all
//          blocks on die 0's arrival counters, and the last arriver writes both release words.
// SPLIT  : param = S | R << 8 (1..64 each).  Lines 1..R the release copies, then 2S arrival
//          counters (S of odd epochs, then S of even epochs), then the top counters of odd and
//          even epochs.  Block b counts in on counter b mod S and polls copy b mod R; the last
//          arriver at a counter counts in at the top (when S > 1), and the last there writes
//          every copy.  The blocks that used a counter reset it (the releaser after the
//          release), as in counter_arrive_wait.
// COUNT  : line 1 a 64-bit arrival counter that only grows.  Each block adds 1 per crossing
//          and polls it until it reaches base + e x n for its e-th crossing since attach: the
//          last arrival's increment is the release itself (no epoch word, no release store).
//          param bits 0-9: ns of sleep before the first poll per 16 arrivals still missing
//          (0: none); bits 16-22: S.  S > 1 counts in two levels: block b adds to sub-counter
//          b mod S (lines 2 .. S+1), the arrival that completes a sub-counter's crossing adds 1
//          to the line-1 counter with a fire-and-forget release, and every block polls line 1
//          until it reaches base + e x G (G = min(S, n) sub-counters in use).
// Epochs increase by one per crossing and are compared for equality, so no phase resets.
struct BarrierRef {
  uint32_t* s;
  uint32_t kind, n, param, mode;
  uint32_t epoch;  // epoch of the last crossing, kept by each block
  uint64_t timeout_ns;
  uint32_t die, n_mine, active;  // DIE: this block's die, its die's blocks (0 = unregistered), dies
  uint64_t base, sub_base;       // COUNT: counters' values at attach (multiples of their parties)
  uint64_t epoch_base;           // EXCHANGE: the global epoch at attach (base / n)
  uint32_t root, root_size;      // TREE counting form: the root's node index and its arrivals
  __device__ __forceinline__ uint32_t* die_line(uint32_t d, uint32_t i) const {
    return s + s[d ? kHdrDieOff1 : kHdrDieOff0] + i * kLineWords;
  }
  __device__ __forceinline__ uint32_t* line(uint32_t i) const { return s + i * kLineWords; }
  __device__ __forceinline__ uint32_t* abort_word() const { return s + kHdrAbort; }
  __device__ __forceinline__ uint32_t flag_lines() const { return (n + kLineWords - 1) / kLineWords; }
  __device__ __forceinline__ uint32_t* arrive_flags() const { return line(1); }
  __device__ __forceinline__ uint32_t* release_flags() const {
    return kind == GSYNC_BAR_SHARDED ? line(1 + param) : line(1 + flag_lines());
  }
};

// Reads the header and the current epoch.  All blocks must attach between the same two
// crossings (normally at kernel start).
__device__ __forceinline__ BarrierRef barrier_attach(void* state) {
  BarrierRef b;
  b.s = (uint32_t*)state;
  b.kind = b.s[kHdrMagic] & 0xFFu;
  b.n = b.s[kHdrN];
  b.param = b.s[kHdrParam];
  b.mode = b.s[kHdrMode];
  b.timeout_ns = header_timeout(b.s);
  b.die = 0;
  if (b.kind == GSYNC_BAR_FLAG || b.kind == GSYNC_BAR_SHARDED) {
    // A block's own release flag always holds the epoch of the last crossing.
    b.epoch = b.mode ? ptx::ld_relaxed(b.release_flags()) : ptx::ld_relaxed(b.release_flags() + blockIdx.x);
  } else if (b.kind == GSYNC_BAR_TREE) {
    b.epoch = ptx::ld_relaxed(b.line(1));
    if ((b.param >> 16) != 0u) {
      // Counting form: locate the root; its counter read here lies in [k S, k S + S - 1] (no
      // crossing completes before this block arrives), so rounding down gives every block the
      // same base.
      const uint32_t fan = max(b.param & 0xFFFFu, 2u);
      uint32_t width = b.n, total = 0;
      for (;;) {
        const uint32_t nodes = (width + fan - 1u) / fan;
        total += nodes;
        if (nodes <= 1u) break;
        width = nodes;
      }
      b.root = total - 1u;
      b.root_size = width;
      const uint64_t v = ptx::ld_relaxed_u64((const uint64_t*)b.line(2u + b.root));
      b.base = width ? v - v % width : v;
      b.epoch = 0;
    }
  } else if (b.kind == GSYNC_BAR_SPLIT) {
    b.epoch = ptx::ld_relaxed(b.line(1u + blockIdx.x % (b.param >> 8)));
  } else if (b.kind == GSYNC_BAR_COUNT || b.kind == GSYNC_BAR_EXCHANGE) {
    // No crossing can complete before every block has attached and arrived, so the counter
    // read here lies in [k P, k P + P - 1] for its P parties per crossing: rounding down
    // gives every block the same base (and every block of a sub-counter the same sub-base).
    const uint32_t S = (b.param >> 16) & 0x7Fu;
    const uint64_t P = S > 1u ? (uint64_t)min(S, b.n) : (uint64_t)b.n;
    const uint64_t c = ptx::ld_relaxed_u64((const uint64_t*)b.line(1));
    b.base = c - c % P;
    b.epoch_base = b.base / P;
    b.sub_base = 0;
    if (S > 1u) {
      const uint32_t g = blockIdx.x % S;
      const uint64_t members = (b.n - g + S - 1u) / S;
      const uint64_t v = ptx::ld_relaxed_u64((const uint64_t*)b.line(2u + g));
      b.sub_base = v - v % members;
    }
    b.epoch = 0;
  } else if (b.kind == GSYNC_BAR_CLUSTER && ((b.param >> 4) & 0xFu) != 0u) {
    // Counting form: rounded down to a multiple of the leaders, as for COUNT.
    const uint32_t c = b.param & 0xFu;
    const uint64_t P = (uint64_t)(b.n / (c ? c : 1u));
    const uint64_t v = ptx::ld_relaxed_u64((const uint64_t*)b.line(1));
    b.base = P ? v - v % P : v;
    b.epoch = 0;
  } else if (b.kind == GSYNC_BAR_DIE) {
    const uint32_t sm = ptx::smid();
    const uint8_t* table = (const uint8_t*)(b.s + kDieTableWord);
    b.die = (sm < kMaxSmIds && table[sm]) ? 1u : 0u;
    b.epoch = ptx::ld_relaxed(b.die_line(b.die, 1));  // both dies' release words move together
  } else {
    b.epoch = ptx::ld_relaxed(b.line(2));
  }
  b.n_mine = 0;
  b.active = 0;
  return b;
}

// Bounded poll of a release word until it holds e1 (acquire).
__device__ __forceinline__ int wait_epoch(const BarrierRef& b, const uint32_t* rel, uint32_t e1) {
  Waiter w;
  while (ptx::ld_acquire(rel) != e1)
    if (int rc = w.tick(b.timeout_ns, b.abort_word())) return rc;
  return GSYNC_OK;
}

// Master thread of a SPLIT barrier (see the layout above).
__device__ __forceinline__ int split_arrive_wait(const BarrierRef& b, uint32_t e1) {
  const uint32_t S = b.param & 0xFFu, R = b.param >> 8;
  const uint32_t groups = min(S, b.n), c = blockIdx.x % S;
  const uint32_t members = (b.n - c + S - 1u) / S;
  const bool odd = (e1 & 1u) != 0u;
  uint32_t* cnt = b.line(1u + R + (odd ? 0u : S) + c);
  uint32_t* top = b.line(1u + R + 2u * S + (odd ? 0u : 1u));
  uint32_t* rel = b.line(1u + blockIdx.x % R);
  if (ptx::atom_add_acq_rel(cnt, 1u) != members - 1u) return wait_epoch(b, rel, e1);
  if (groups > 1u && ptx::atom_add_acq_rel(top, 1u) != groups - 1u) {
    ptx::st_relaxed(cnt, 0u);
    return wait_epoch(b, rel, e1);
  }
  ptx::fence_acq_rel();  // release: everything acquired above precedes every copy
  for (uint32_t r = 0; r < R; ++r) ptx::st_relaxed(b.line(1u + r), e1);
  ptx::st_relaxed(cnt, 0u);
  if (groups > 1u) ptx::st_relaxed(top, 0u);
  return GSYNC_OK;
}

// Master thread of a DIE barrier (see the layout above).
__device__ __forceinline__ int die_arrive_wait(BarrierRef& b, uint32_t e1) {
  uint32_t* rel = b.die_line(b.die, 1);
  if (b.param == 1u) {
    // Flat arrivals on one counter pair (die 0's page), release words on both dies: the
    // split protocol with one counter and one release copy per die, each block polling the
    // copy homed on its own die.
    uint32_t* cnt = b.die_line(0, (e1 & 1u) ? 0u : 3u);
    if (ptx::atom_add_acq_rel(cnt, 1u) != b.n - 1u) return wait_epoch(b, rel, e1);
    ptx::fence_acq_rel();
    ptx::st_relaxed(b.die_line(0, 1), e1);
    ptx::st_relaxed(b.die_line(1, 1), e1);
    ptx::st_relaxed(cnt, 0u);
    return GSYNC_OK;
  }
  uint32_t* info = b.line(2);
  if (b.n_mine == 0) {
    // Registration crossing: count in on the flat counter, and into this die's membership.
    ptx::red_add_relaxed(info + b.die, 1u);
    const uint32_t old = ptx::atom_add_acq_rel(b.line(1), 1u);  // release: orders the red above
    int rc = GSYNC_OK;
    if (old == b.n - 1u) {
      ptx::st_relaxed(b.line(1), 0u);
      const uint32_t m0 = ptx::ld_relaxed(info), m1 = ptx::ld_relaxed(info + 1);
      ptx::st_relaxed(info, 0u);
      ptx::st_relaxed(info + 1, 0u);
      ptx::st_relaxed(info + 2, m0);
      ptx::st_relaxed(info + 3, m1);
      ptx::st_relaxed(info + 4, (m0 ? 1u : 0u) + (m1 ? 1u : 0u));
      ptx::fence_acq_rel();  // release: everything above precedes both release words
      ptx::st_relaxed(b.die_line(0, 1), e1);
      ptx::st_relaxed(b.die_line(1, 1), e1);
    } else {
      rc = wait_epoch(b, rel, e1);
    }
    if (rc == GSYNC_OK) {
      b.n_mine = ptx::ld_relaxed(info + 2 + b.die);
      b.active = ptx::ld_relaxed(info + 4);
    }
    return rc;
  }
  // Counters alternate by epoch parity (as in counter_arrive_wait): the releasing block
  // resets the ones it used after the release.
  const bool odd = (e1 & 1u) != 0u;
  uint32_t* cnt = b.die_line(b.die, odd ? 0u : 3u);
  const uint32_t old = ptx::atom_add_acq_rel(cnt, 1u);
  if (old != b.n_mine - 1u) return wait_epoch(b, rel, e1);
  // Last of this die; the second die to get here releases both dies.
  uint32_t* top = b.die_line(0, odd ? 2u : 4u);
  if (b.active == 2u && ptx::atom_add_acq_rel(top, 1u) != 1u) {
    ptx::st_relaxed(cnt, 0u);
    return wait_epoch(b, rel, e1);
  }
  ptx::fence_acq_rel();
  ptx::st_relaxed(b.die_line(0, 1), e1);
  ptx::st_relaxed(b.die_line(1, 1), e1);
  ptx::st_relaxed(cnt, 0u);
  if (b.active == 2u) ptx::st_relaxed(top, 0u);
  return GSYNC_OK;
}

// Master-thread arrival on a two-stage atomic counter of `parties` participants.  Crossings
// alternate between two counters (lines 1 and 3, by epoch parity), so the last arriver
// releases first and resets its counter after, off the release path: the counter is next
// used two crossings later, which no block can reach before the last arriver has arrived at
// the crossing in between.
__device__ __forceinline__ int counter_arrive_wait(const BarrierRef& b, uint32_t parties, uint32_t e1) {
  uint32_t* cnt = b.line((e1 & 1u) ? 1u : 3u);
  const uint32_t old = ptx::atom_add_acq_rel(cnt, 1u);
  if (old == parties - 1u) {
    ptx::st_release(b.line(2), e1);
    ptx::st_relaxed(cnt, 0u);
    return GSYNC_OK;
  }
  Waiter w;
  while (ptx::ld_acquire(b.line(2)) != e1)
    if (int rc = w.tick(b.timeout_ns, b.abort_word())) return rc;
  return GSYNC_OK;
}

template <int KIND>
__device__ __forceinline__ int barrier_wait(BarrierRef& b) {
  static_assert(KIND != GSYNC_BAR_EXCHANGE, "the exchange barrier crosses with barrier_exchange");
  __shared__ int s_rc;
  const bool master = threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0;
  const uint32_t e1 = b.epoch + 1u;
  if (KIND == GSYNC_BAR_CLUSTER) {
    ptx::cluster_sync();  // every block of the cluster has arrived (release/acquire, cluster)
  } else {
    __syncthreads();
  }
  if (KIND == GSYNC_BAR_ATOMIC) {
    if (master) s_rc = counter_arrive_wait(b, b.n, e1);
  } else if (KIND == GSYNC_BAR_DIE) {
    if (master) s_rc = die_arrive_wait(b, e1);
  } else if (KIND == GSYNC_BAR_SPLIT) {
    if (master) s_rc = split_arrive_wait(b, e1);
  } else if (KIND == GSYNC_BAR_COUNT) {
    if (master) {
      const uint32_t S = (b.param >> 16) & 0x7Fu, sleep16 = b.param & 0x3FFu;
      uint64_t* top = (uint64_t*)b.line(1);
      int rc = GSYNC_OK;
      uint64_t target, missing;
      if (S > 1u) {
        const uint32_t g = blockIdx.x % S;
        const uint64_t members = (b.n - g + S - 1u) / S;
        const uint64_t sub_target = b.sub_base + (uint64_t)e1 * members;
        const uint64_t now = ptx::atom_add_acq_rel_u64((uint64_t*)b.line(2u + g), 1ull) + 1ull;
        if (now == sub_target) ptx::red_add_release_u64(top, 1ull);  // this sub-counter is complete
        target = b.base + (uint64_t)e1 * min(S, b.n);
        missing = sub_target - now;
      } else {
        target = b.base + (uint64_t)e1 * b.n;
        const uint64_t now = ptx::atom_add_acq_rel_u64(top, 1ull) + 1ull;
        missing = target - now;
      }
      if (missing) {
        // Sleep in proportion to the arrivals still missing, to keep the early arrivers' polls
        // off the counter while the atomic unit works through the rest of the arrivals.
        if (sleep16 && missing < (1ull << 24)) {
          const uint64_t ns = missing * sleep16 / 16u;
          __nanosleep((uint32_t)(ns < 4000u ? ns : 4000u));
        }
      }
      if (S > 1u || missing) {
        Waiter w;
        while (ptx::ld_acquire_u64(top) < target)
          if ((rc = w.tick(b.timeout_ns, b.abort_word())) != GSYNC_OK) break;
      }
      s_rc = rc;
    }
  } else if (KIND == GSYNC_BAR_CLUSTER) {
    const uint32_t form = (b.param >> 4) & 0xFu, c = b.param & 0xFu;
    const bool leader = ptx::cluster_ctarank() == 0;
    if (form == 0u) {
      if (master) {
        int rc = GSYNC_OK;
        if (leader) {
          rc = counter_arrive_wait(b, b.n / (c ? c : 1u), e1);
        } else {
          Waiter w;
          while (ptx::ld_acquire(b.line(2)) != e1)
            if ((rc = w.tick(b.timeout_ns, b.abort_word())) != GSYNC_OK) break;
        }
        s_rc = rc;
      }
    } else {
      if (master && (leader || form == 1u)) {
        uint64_t* cnt = (uint64_t*)b.line(1);
        const uint64_t target = b.base + (uint64_t)e1 * (b.n / (c ? c : 1u));
        uint64_t missing = 1;
        if (leader) {
          // release: orders the cluster's writes (acquired through the cluster barrier) first
          missing = target - (ptx::atom_add_acq_rel_u64(cnt, 1ull) + 1ull);
          const uint32_t sleep16 = (b.param >> 8) & 0x3FFu;
          if (missing && sleep16 && missing < (1ull << 24)) {
            const uint64_t ns = missing * sleep16 / 16u;
            __nanosleep((uint32_t)(ns < 4000u ? ns : 4000u));
          }
        }
        int rc = GSYNC_OK;
        if (missing) {
          Waiter w;
          while (ptx::ld_acquire_u64(cnt) < target)
            if ((rc = w.tick(b.timeout_ns, b.abort_word())) != GSYNC_OK) break;
        }
        s_rc = rc;
      }
      if (form == 2u) {
        ptx::cluster_sync();  // the leader has seen the crossing complete, or given up
        if (master && !leader) s_rc = (int)ptx::ld_relaxed_cluster((const uint32_t*)ptx::map_cluster_rank(&s_rc, 0u));
      }
    }
  } else if (KIND == GSYNC_BAR_TREE && (b.param >> 16) != 0u) {
    if (master) {
      // Counting combining tree: count in at the leaf; the arrival that completes a node's
      // crossing counts in at the parent; the root's completing add is the release.
      const uint32_t fan = max(b.param & 0xFFFFu, 2u);
      uint32_t width = b.n, node = blockIdx.x / fan, off = 0;
      bool released = false;
      for (;;) {
        const uint32_t nodes = (width + fan - 1u) / fan;
        const uint32_t size = min(fan, width - node * fan);
        const uint64_t now = ptx::atom_add_acq_rel_u64((uint64_t*)b.line(2u + off + node), 1ull) + 1ull;
        if (now % size != 0u) break;  // not this node's last arrival
        if (nodes == 1u) {
          released = true;  // the root's last arrival: the crossing is complete
          break;
        }
        off += nodes;
        width = nodes;
        node /= fan;
      }
      int rc = GSYNC_OK;
      if (!released) {
        const uint64_t target = b.base + (uint64_t)e1 * b.root_size;
        const uint64_t* root = (const uint64_t*)b.line(2u + b.root);
        Waiter w;
        while (ptx::ld_acquire_u64(root) < target)
          if ((rc = w.tick(b.timeout_ns, b.abort_word())) != GSYNC_OK) break;
      }
      s_rc = rc;
    }
  } else if (KIND == GSYNC_BAR_TREE) {
    if (master) {
      // Combining tree: count in at the leaf; the last arriver at a node resets it and
      // counts in at the parent; the last arriver at the root advances the epoch.
      const uint32_t fan = max(b.param & 0xFFFFu, 2u);
      uint32_t width = b.n, node = blockIdx.x / fan, off = 0;
      int rc = GSYNC_OK;
      for (;;) {
        const uint32_t nodes = (width + fan - 1) / fan;
        const uint32_t size = min(fan, width - node * fan);
        uint32_t* c = b.line(2 + off + node);
        const uint32_t old = ptx::atom_add_acq_rel(c, 1u);
        if (old + 1u < size) {
          Waiter w;
          while (ptx::ld_acquire(b.line(1)) != e1)
            if ((rc = w.tick(b.timeout_ns, b.abort_word())) != GSYNC_OK) break;
          break;
        }
        ptx::st_relaxed(c, 0u);
        if (nodes == 1u) {
          ptx::st_release(b.line(1), e1);
          break;
        }
        off += nodes;
        width = nodes;
        node /= fan;
      }
      s_rc = rc;
    }
  } else if (KIND == GSYNC_BAR_SHARDED) {
    const uint32_t S = b.param;
    if (blockIdx.x == 0) {
      if (threadIdx.x < 32 && threadIdx.y == 0 && threadIdx.z == 0) {
        // Lane s < S watches counter s until it reaches e1 x (blocks of shard s, master
        // excluded for shard 0), in wrapping uint32 arithmetic.
        const uint32_t lane = threadIdx.x;
        int rc = GSYNC_OK;
        if (lane < S) {
          const uint32_t members = (b.n - lane + S - 1u) / S - (lane == 0u ? 1u : 0u);
          const uint32_t target = e1 * members;
          Waiter w;
          while (ptx::ld_relaxed(b.line(1 + lane)) != target)
            if ((rc = w.tick(b.timeout_ns, b.abort_word())) != GSYNC_OK) break;
        }
        ptx::fence_acq_rel();  // acquire: the arrivals this lane counted
        const int worst = __reduce_max_sync(0xFFFFFFFFu, rc);
        __syncwarp();
        if (worst == GSYNC_OK) {
          ptx::fence_acq_rel();  // release: every lane's acquisitions precede the release flags
          const uint32_t nvec = (b.n + 3u) >> 2;
          for (uint32_t v = lane; v < nvec; v += 32u) ptx::st_relaxed_v4(b.release_flags() + 4u * v, e1);
        }
        if (lane == 0) s_rc = worst;
      }
    } else if (master) {
      ptx::red_add_release(b.line(1 + blockIdx.x % S), 1u);
      Waiter w;
      int rc = GSYNC_OK;
      while (ptx::ld_acquire(b.release_flags() + blockIdx.x) != e1)
        if ((rc = w.tick(b.timeout_ns, b.abort_word())) != GSYNC_OK) break;
      s_rc = rc;
    }
  } else {  // GSYNC_BAR_FLAG: decentralized XF barrier, block 0 is the master block
    if (blockIdx.x == 0) {
      // Every thread of the master block watches its share of the arrival flags as 16-byte
      // vectors (thread t: vectors t, t + nthr, ...).  Each pass issues a thread's pending
      // loads back to back (2 in flight, neither waiting on the other) before it checks them,
      // so a pass costs about one L2 round trip.  The flag arrays span whole lines, so a
      // vector never leaves them; word 0 (the master's own flag) and words past n are
      // ignored.  Each thread then fences to acquire what it saw, the block agrees that all
      // arrived, and each thread fences again before writing its share of the release flags.
      const uint32_t tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
      const uint32_t nthr = blockDim.x * blockDim.y * blockDim.z;
      const uint32_t nvec = (b.n + 3u) >> 2;
      Waiter w;
      int rc = GSYNC_OK;
      for (uint32_t v0 = tid; v0 < nvec && rc == GSYNC_OK; v0 += 2u * nthr) {
        uint32_t pending = 0;
        for (uint32_t k = 0; k < 2u; ++k)
          if (v0 + k * nthr < nvec) pending |= 1u << k;
        while (pending) {
          uint4 x[2];
#pragma unroll
          for (uint32_t k = 0; k < 2u; ++k)
            if ((pending >> k) & 1u) x[k] = ptx::ld_relaxed_v4(b.arrive_flags() + 4u * (v0 + k * nthr));
          uint32_t still = 0;
#pragma unroll
          for (uint32_t k = 0; k < 2u; ++k) {
            if (!((pending >> k) & 1u)) continue;
            const uint32_t base = 4u * (v0 + k * nthr);
            const bool ok = (base == 0u || base >= b.n || x[k].x == e1) && (base + 1u >= b.n || x[k].y == e1) &&
                            (base + 2u >= b.n || x[k].z == e1) && (base + 3u >= b.n || x[k].w == e1);
            if (!ok) still |= 1u << k;
          }
          pending = still;
          if (pending && (rc = w.tick(b.timeout_ns, b.abort_word())) != GSYNC_OK) break;
        }
      }
      ptx::fence_acq_rel();  // acquire: what this thread's relaxed loads observed
      const int any_bad = __syncthreads_or(rc != GSYNC_OK);
      if (!any_bad) {
        ptx::fence_acq_rel();  // release: every thread's acquisitions precede the release flags
        if (b.mode) {
          if (master) ptx::st_relaxed(b.release_flags(), e1);
        } else {
          for (uint32_t v = tid; v < nvec; v += nthr) ptx::st_relaxed_v4(b.release_flags() + 4u * v, e1);
        }
      }
      if (master) s_rc = !any_bad ? GSYNC_OK : (rc != GSYNC_OK ? rc : GSYNC_EABORTED);
    } else if (master) {
      ptx::st_release(b.arrive_flags() + blockIdx.x, e1);
      uint32_t* rel = b.mode ? b.release_flags() : b.release_flags() + blockIdx.x;
      Waiter w;
      int rc = GSYNC_OK;
      while (ptx::ld_acquire(rel) != e1)
        if ((rc = w.tick(b.timeout_ns, b.abort_word())) != GSYNC_OK) break;
      s_rc = rc;
    }
  }
  __syncthreads();
  const int rc = s_rc;
  b.epoch = e1;
  return rc;
}

// EXCHANGE: the counting barrier whose arrivals carry one 64-bit value per block -- a barrier
// and an all-gather in one (a GB300 design; the paper's barriers publish data through memory
// written before a fenced arrival).  Line 1 is the growing counter; from line 2, one 16-byte
// record {global epoch, value} per block and epoch parity.  A block's arrival writes its
// record with one relaxed 128-bit store and counts in with a relaxed fetch-and-add: no fence,
// so the device may make the two visible in either order.  After the crossing, a reader polls
// a block's record until it shows the crossing's epoch; a 128-bit access is one access, so the
// value it then holds is the one published for that crossing.  Records alternate by epoch
// parity: a block rewrites its record of parity e mod 2 for crossing e + 2 only after passing
// e + 1, which every reader of crossing e reaches only after its reads.  The global epoch
// (epoch_base + crossings since attach) keeps growing across launches, so a record left by an
// earlier launch never matches.  The crossing orders the exchanged values only: writes a
// block made to other memory before it are not published -- GSYNC_BAR_COUNT does that.
__device__ __forceinline__ uint64_t* exchange_record(const BarrierRef& b, uint64_t epoch, uint32_t blk) {
  return (uint64_t*)b.line(2) + 2u * ((uint32_t)(epoch & 1u) * b.n + blk);
}

// All threads of the block: publish `value` (thread 0's) for this crossing and cross.  An
// object of another kind returns GSYNC_EINVAL without crossing.
__device__ __forceinline__ int barrier_exchange(BarrierRef& b, uint64_t value) {
  if (b.kind != GSYNC_BAR_EXCHANGE) return GSYNC_EINVAL;  // uniform: every thread reads the same header
  __shared__ int s_rc;
  const bool master = threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0;
  const uint32_t e1 = b.epoch + 1u;
  __syncthreads();
  if (master) {
    const uint64_t ge = b.epoch_base + e1;
    uint64_t* counter = (uint64_t*)b.line(1);
    ptx::st_relaxed_b128(exchange_record(b, ge, blockIdx.x), ge, value);
    const uint64_t target = b.base + (uint64_t)e1 * b.n;
    const uint64_t missing = target - (ptx::atom_add_relaxed_u64(counter, 1ull) + 1ull);
    const uint32_t sleep16 = b.param & 0x3FFu;
    int rc = GSYNC_OK;
    if (missing) {
      if (sleep16 && missing < (1ull << 24)) {
        const uint64_t ns = missing * sleep16 / 16u;
        __nanosleep((uint32_t)(ns < 4000u ? ns : 4000u));
      }
      Waiter w;
      while (ptx::ld_relaxed_u64(counter) < target)
        if ((rc = w.tick(b.timeout_ns, b.abort_word())) != GSYNC_OK) break;
    }
    s_rc = rc;
  }
  __syncthreads();
  const int rc = s_rc;
  b.epoch = e1;
  return rc;
}

// Any thread, after barrier_exchange returned GSYNC_OK: the value block `blk` published for
// that crossing (polls its record, bounded).  Must complete before the block's next crossing.
__device__ __forceinline__ int barrier_exchange_read(const BarrierRef& b, uint32_t blk, uint64_t& value) {
  if (b.kind != GSYNC_BAR_EXCHANGE || blk >= b.n) return GSYNC_EINVAL;
  const uint64_t ge = b.epoch_base + b.epoch;
  const uint64_t* rec = exchange_record(b, ge, blk);
  Waiter w;
  uint64_t lo, hi;
  for (;;) {
    ptx::ld_relaxed_b128(rec, lo, hi);
    if (lo == ge) break;
    if (int rc = w.tick(b.timeout_ns, b.abort_word())) return rc;
  }
  value = hi;
  return GSYNC_OK;
}

// barrier_wait with a wait bound for this call (ns) instead of the object's own; on expiry
// GSYNC_ETIMEDOUT, and the object is marked aborted (the crossing cannot complete for the
// others either).
template <int KIND>
__device__ __forceinline__ int barrier_wait(BarrierRef& b, uint64_t timeout_ns) {
  const uint64_t own = b.timeout_ns;
  b.timeout_ns = timeout_ns;
  const int rc = barrier_wait<KIND>(b);
  b.timeout_ns = own;
  return rc;
}

}  // namespace gsync
