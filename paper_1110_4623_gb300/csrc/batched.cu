// Batched persistent kernel: many independent mutexes of uneven contention and many barrier
// groups driven by one co-resident launch.
//
// Section 6 measures one primitive instance at a time; a real persistent kernel serves
// thousands of instances at once, with contention set by key popularity.  Here acquisition i
// (key keys[i], addend adds[i]) belongs to block i mod G and runs in order on that block's
// thread 0: lock mutex[key] with the policy of the key's contention class, add the int64
// addend to sum[key] and increment count[key] with plain loads and stores, unlock.  Blocks
// that belong to a barrier group also cross `rounds` group barriers spread evenly over their
// acquisitions, with the sampled slot check of the barrier workload (partner
// p = (j + r + 1) mod size inside the group).  The autotuner chooses, per contention class,
// the mutex kind (spin / spin + backoff / ticket, the carrying ticket or two-die cohort lock,
// or -- in a cluster launch -- the cluster cohort lock for keys below kLocalKeys), the backoff
// constants (0 = pure spinning, otherwise __nanosleep) and the cluster size of the group
// barriers.
#include "common.cuh"

using namespace gsync_impl;
namespace ptx = gsync::ptx;

namespace {

constexpr int kMaxThreads = 256;
// Per-object memory: a mutex is a header line and two lines (lock word, turn); a group
// barrier a header line, two arrival counters (by epoch parity) and the release epoch.
constexpr uint32_t kMutexObjWords = 3 * gsync::kLineWords;
constexpr uint32_t kBarObjWords = 4 * gsync::kLineWords;
// Keys below this may use the cluster locks (the cluster cohort lock and the carrying locks
// over clusters): their local locks live in a table in each block's shared memory (32 bytes a
// key).
constexpr uint32_t kLocalKeys = 256;

// A key's slot in a cluster launch.  The cluster cohort lock uses block 0's {ticket, turn};
// the carrying lock over clusters block 0's ticket and a 16-byte record {served, cohort word,
// sum}; the three-level carrying lock the tail in block 0's ticket word, and in every block
// its own MCS node: the link (in `turn`), the pushed record, and its count of queueings (in
// `pad`).
struct __align__(16) LocalSlot {
  gsync::ClusterLocal cl;
  uint64_t rec[2];
};

struct Args {
  uint32_t* mutex_state;
  const uint8_t* key_class;
  const uint32_t* policy;
  const int32_t* keys;
  const int64_t* adds;
  int64_t* sum;
  uint32_t* count;
  const int32_t* group_start;
  const int32_t* group_size;
  const int32_t* group_of_block;
  uint32_t* group_state;
  uint32_t* slots;
  uint32_t* mix;
  uint32_t* bad;
  uint32_t* status;
  uint32_t* cohort_state;
  uint64_t timeout_ns;
  int32_t nkeys, nacq, rounds, nclasses, ngroups, ncohort, clustered;
};

// Per-key two-die cohort objects (gsync_mutex_init_cohort's layout and placement).
constexpr uint32_t kCohortObjWords = 32u * 1024u / 4u;

__device__ __forceinline__ gsync::Token lock_by_policy(const gsync::MutexRef& m) {
  switch (m.kind) {
    case GSYNC_MUTEX_CAS_SPIN: return gsync::mutex_lock_thread<GSYNC_MUTEX_CAS_SPIN>(m);
    case GSYNC_MUTEX_CAS_BACKOFF: return gsync::mutex_lock_thread<GSYNC_MUTEX_CAS_BACKOFF>(m);
    case GSYNC_MUTEX_CLUSTER: return gsync::mutex_lock_thread<GSYNC_MUTEX_CLUSTER>(m);
    default: return gsync::mutex_lock_thread<GSYNC_MUTEX_TICKET>(m);
  }
}

__device__ __forceinline__ void unlock_by_policy(const gsync::MutexRef& m, const gsync::Token& t) {
  if (m.kind == GSYNC_MUTEX_TICKET) gsync::mutex_unlock_thread<GSYNC_MUTEX_TICKET>(m, t.ticket);
  else if (m.kind == GSYNC_MUTEX_CLUSTER) gsync::mutex_unlock_thread<GSYNC_MUTEX_CLUSTER>(m, t);
  else gsync::mutex_unlock_thread<GSYNC_MUTEX_CAS_SPIN>(m, t.ticket);
}

// GSYNC_BATCHED_TICKET_CARRY: the ticket lock (take a ticket, wait for the turn, sleeping in
// proportion to the waiters ahead) whose turn line also holds what it guards.  Line 2 of the
// key's object is one 16-byte record {turn, count, sum}: the waiter's load of the turn brings
// the count and sum with it, and the holder's store of the next turn writes the new count and
// sum in the same store.  A hand-off therefore carries the data: the critical section makes
// no L2 round trip of its own.  Both accesses are relaxed.  Everything the lock guards is in
// that one 16-byte location, and a .b128 access is a single access to it, so the value a
// holder reads is exactly the record its predecessor wrote, and the value it writes depends
// on what it read: coherence on the one location orders the hand-offs, and no fence (no wait
// for earlier stores, no acquire) is needed on the hand-off path.  The key's count and sum
// stay in the record until batched_collect_kernel copies them out after the launch.
__device__ __forceinline__ int carry_add(uint32_t* obj, const uint32_t* pol, int64_t add, uint64_t timeout_ns) {
  uint32_t* ticket = obj + 1 * gsync::kLineWords;
  uint32_t* rec = obj + 2 * gsync::kLineWords;
  const uint32_t t = ptx::atom_add_relaxed(ticket, 1u);
  gsync::Waiter w;
  uint64_t lo, hi;
  for (;;) {
    ptx::ld_relaxed_b128(rec, lo, hi);
    const uint32_t ahead = t - (uint32_t)lo;
    if (ahead == 0u) break;
    if (int rc = w.tick(timeout_ns, obj + gsync::kHdrAbort)) return rc;
    if (pol[1] && ahead > 1u && ahead < 0x80000000u) {
      const uint32_t ns = (ahead - 1u) * pol[1];
      __nanosleep(ns < pol[2] ? ns : pol[2]);
    }
  }
  // critical section: count + 1 and sum + add, published with the next turn
  const uint64_t next = (uint64_t)(t + 1u) | ((uint64_t)((uint32_t)(lo >> 32) + 1u) << 32);
  ptx::st_relaxed_b128(rec, next, (uint64_t)((int64_t)hi + add));
  return GSYNC_OK;
}

// Word offset of die d's local lock in a cohort object, or 0 when the object was not set up
// by gsync_mutex_init_cohort (then the key is refused instead of using stray lines).
__device__ __forceinline__ uint32_t cohort_local_offset(const uint32_t* obj, uint32_t d) {
  const uint32_t off = __ldg(obj + (d ? gsync::kHdrDieOff1 : gsync::kHdrDieOff0));
  const bool ok = (__ldg(obj + gsync::kHdrMagic) & 0xFFu) == (uint32_t)GSYNC_MUTEX_COHORT &&
                  off >= 5u * gsync::kLineWords && off + 2u * gsync::kLineWords <= kCohortObjWords;
  return ok ? off : 0u;
}

// GSYNC_BATCHED_COHORT_CARRY: the two-die cohort lock (a ticket lock per die, on a 4 KB page
// homed on that die, under a global ticket lock) with carrying records.  Each die's turn line
// holds one 16-byte record {served ticket, cohort word, sum}, the global turn line one record
// {turn, -, sum}.  The holder takes the sum from the record that granted it the lock: its
// die's record when the cohort word says the die already holds the global lock, else the
// global record once the global turn reaches its global ticket.  It passes sum + add on in the
// record it releases: its die's record, with the global lock kept by the die, while a waiter of
// its die is queued and fewer than `budget` passes were made in a row; else the global record
// and then its die's record without the cohort bit.  A pass inside a die never leaves the die.
// Each record is read and written as one relaxed 128-bit access and a holder's sum comes only
// from the record that granted it the lock, so, as in carry_add, coherence on that one location
// orders each hand-off and no fence is needed.  The die's ticket counter is read beside each
// poll that may see the grant (the first, and those after one that found a single holder
// ahead): the counter only grows, so a waiter seen in any read is still queued at the
// release, and one not seen finds the global lock released and queues for it.  The last
// acquisition has no waiter behind it and so releases the global lock: after the launch the
// global record holds the key's sum, and the dies' ticket counters add up to its count.
__device__ __forceinline__ int cohort_carry_add(uint32_t* obj, uint32_t die, const uint32_t* pol, int64_t add,
                                                uint64_t timeout_ns) {
  const uint32_t off = cohort_local_offset(obj, die);
  if (off == 0u) return GSYNC_EINVAL;
  uint32_t* local = obj + off;
  uint32_t* lnext = local;
  uint32_t* lrec = local + gsync::kLineWords;
  uint32_t* gnext = obj + 1 * gsync::kLineWords;
  uint32_t* grec = obj + 2 * gsync::kLineWords;
  const uint32_t budget = pol[3] ? min(pol[3], 32767u) : (uint32_t)GSYNC_COHORT_DEFAULT_BUDGET;
  const uint32_t t = ptx::atom_add_relaxed(lnext, 1u);
  gsync::Waiter w;
  uint64_t lo, hi;
  uint32_t seen = t + 1u, prev_ahead = 1u;  // t + 1: no waiter known behind this ticket
  for (;;) {
    // Only a poll that may see the grant reads the counter beside it.
    if (prev_ahead <= 1u) seen = ptx::ld_relaxed(lnext);
    ptx::ld_relaxed_b128(lrec, lo, hi);
    const uint32_t ahead = t - (uint32_t)lo;
    if (ahead == 0u) break;
    prev_ahead = ahead;
    if (int rc = w.tick(timeout_ns, obj + gsync::kHdrAbort)) return rc;
    if (pol[1] && ahead > 1u && ahead < 0x80000000u) {
      const uint32_t ns = (ahead - 1u) * pol[1];
      __nanosleep(ns < pol[2] ? ns : pol[2]);
    }
  }
  uint32_t word = (uint32_t)(lo >> 32);
  int64_t sum = (int64_t)hi;
  if (word & gsync::kCohortOwned) {
    word &= ~gsync::kCohortOwned;
  } else {
    // First of a cohort: queue for the global lock (at most one waiter per die).
    const uint32_t g = ptx::atom_add_relaxed(gnext, 1u) & 0xFFFFu;
    for (;;) {
      seen = ptx::ld_relaxed(lnext);
      ptx::ld_relaxed_b128(grec, lo, hi);
      if (((uint32_t)lo & 0xFFFFu) == g) break;
      if (int rc = w.tick(timeout_ns, obj + gsync::kHdrAbort)) return rc;
      if (pol[1]) __nanosleep(pol[1]);
    }
    word = g;
    sum = (int64_t)hi;
  }
  // critical section: sum + add, published with the hand-off
  sum += add;
  const uint32_t passes = (word >> 16) & 0x7FFFu, g = word & 0xFFFFu;
  if (passes + 1u < budget && seen != t + 1u) {
    const uint32_t w2 = gsync::kCohortOwned | ((passes + 1u) << 16) | g;
    ptx::st_relaxed_b128(lrec, (uint64_t)(t + 1u) | ((uint64_t)w2 << 32), (uint64_t)sum);
  } else {
    ptx::st_relaxed_b128(grec, (uint64_t)((g + 1u) & 0xFFFFu), (uint64_t)sum);
    ptx::st_relaxed_b128(lrec, (uint64_t)(t + 1u), (uint64_t)sum);
  }
  return GSYNC_OK;
}

__device__ __forceinline__ bool uses_cohort_carry(const Args& a, const uint32_t* pol, uint32_t key) {
  return pol[0] == GSYNC_BATCHED_COHORT_CARRY && key < (uint32_t)a.ncohort;
}

// GSYNC_BATCHED_CLUSTER_CARRY: the cohort protocol of cohort_carry_add with the thread-block
// cluster as the group.  The group's ticket counter and record are the key's LocalSlot in the
// shared memory of the cluster's block 0, reached through distributed shared memory with
// relaxed cluster-scope accesses (a 128-bit record access is one access there too); the global
// ticket and record are lines 1 and 2 of the key's object, as in cohort_carry_add.  A pass
// inside the cluster never touches L2.  The local counters die with the launch, so the
// kernel's end adds each cluster's count of the key's acquisitions to count[].
__device__ __forceinline__ int cluster_carry_add(LocalSlot* slot, uint32_t* obj, const uint32_t* pol, int64_t add,
                                                 uint64_t timeout_ns) {
  uint32_t* lnext = &slot->cl.next;
  uint64_t* lrec = slot->rec;
  uint32_t* gnext = obj + 1 * gsync::kLineWords;
  uint32_t* grec = obj + 2 * gsync::kLineWords;
  const uint32_t budget = pol[3] ? min(pol[3], 32767u) : (uint32_t)GSYNC_COHORT_DEFAULT_BUDGET;
  const uint32_t t = ptx::atom_add_relaxed_cluster(lnext, 1u);
  gsync::Waiter w;
  uint64_t lo, hi;
  uint32_t seen = t + 1u, prev_ahead = 1u;  // t + 1: no waiter known behind this ticket
  for (;;) {
    if (prev_ahead <= 1u) seen = ptx::ld_relaxed_cluster(lnext);
    ptx::ld_relaxed_cluster_b128(lrec, lo, hi);
    const uint32_t ahead = t - (uint32_t)lo;
    if (ahead == 0u) break;
    prev_ahead = ahead;
    if (int rc = w.tick(timeout_ns, obj + gsync::kHdrAbort)) return rc;
    if (pol[1] && ahead > 1u && ahead < 0x80000000u) {
      const uint32_t ns = (ahead - 1u) * pol[1];
      __nanosleep(ns < pol[2] ? ns : pol[2]);
    }
  }
  uint32_t word = (uint32_t)(lo >> 32);
  int64_t sum = (int64_t)hi;
  if (word & gsync::kCohortOwned) {
    word &= ~gsync::kCohortOwned;
  } else {
    // First of a cohort: queue for the global lock (at most one waiter per cluster).
    const uint32_t g = ptx::atom_add_relaxed(gnext, 1u) & 0xFFFFu;
    for (;;) {
      seen = ptx::ld_relaxed_cluster(lnext);
      ptx::ld_relaxed_b128(grec, lo, hi);
      if (((uint32_t)lo & 0xFFFFu) == g) break;
      if (int rc = w.tick(timeout_ns, obj + gsync::kHdrAbort)) return rc;
      if (pol[1]) __nanosleep(pol[1]);
    }
    word = g;
    sum = (int64_t)hi;
  }
  // critical section: sum + add, published with the hand-off
  sum += add;
  const uint32_t passes = (word >> 16) & 0x7FFFu, g = word & 0xFFFFu;
  if (passes + 1u < budget && seen != t + 1u) {
    const uint32_t w2 = gsync::kCohortOwned | ((passes + 1u) << 16) | g;
    ptx::st_relaxed_cluster_b128(lrec, (uint64_t)(t + 1u) | ((uint64_t)w2 << 32), (uint64_t)sum);
  } else {
    ptx::st_relaxed_b128(grec, (uint64_t)((g + 1u) & 0xFFFFu), (uint64_t)sum);
    ptx::st_relaxed_cluster_b128(lrec, (uint64_t)(t + 1u), (uint64_t)sum);
  }
  return GSYNC_OK;
}

// Whether a key runs the cluster carrying lock in this launch (cluster launch, key below
// kLocalKeys); such a key's other launches' kinds and the collect pass must agree on it.
__device__ __forceinline__ bool uses_cluster_carry(const Args& a, const uint32_t* pol, uint32_t key) {
  return pol[0] == GSYNC_BATCHED_CLUSTER_CARRY && a.clustered && key < kLocalKeys;
}

// GSYNC_BATCHED_CLUSTER_DIE_CARRY: the carrying cohort protocol over three levels -- the
// cluster, the die (ticket and record on the cohort object's page homed on this block's die)
// and the global lock (lines 1-2 of the cohort object).  The cluster level is an MCS queue
// (Mellor-Crummey and Scott, 1991) in distributed shared memory: a block swaps itself into
// the tail in block 0's slot, links itself into its predecessor's node, and polls a record in
// its own shared memory, which its predecessor writes when it passes the lock (a push: one
// remote store, no remote poll).  A holder takes the sum from the record that granted it the
// lock and releases, in order of preference: to its linked successor in the cluster (the
// record owned: the die and global locks stay with the cluster); to the next waiting cluster
// of its die (the die record owned: the global lock stays with the die), then frees its
// cluster; or it releases the global lock, then its die, then its cluster.  Nothing is reset
// between rounds: a block's node carries its own sequence number of queueings on the key, and
// every link and pushed record is checked against it.  An owned cluster record carries what
// its cohort's last holder needs: lo = seq:16 | owned:1 | cluster passes:7 | die passes:8 |
// die ticket:16 | global ticket:16, hi = sum.  The die record is {served, owned:1 | die
// passes:15 | global ticket:16, sum} and the global record {turn, -, sum}; served tickets and
// the global turn are compared in 16 bits (fewer than 2^15 waiters at either level).  Every
// access to a record is one relaxed 128-bit access, so, as in cohort_carry_add, no fence is
// needed.
constexpr uint64_t kClusterOwned = 1ull << 16;

__device__ __forceinline__ bool uses_hier_carry(const Args& a, const uint32_t* pol, uint32_t key) {
  return pol[0] == GSYNC_BATCHED_CLUSTER_DIE_CARRY && a.clustered && key < kLocalKeys && key < (uint32_t)a.ncohort;
}

__device__ __forceinline__ int hier_carry_add(LocalSlot* slot, uint32_t* obj, uint32_t die, const uint32_t* pol,
                                              int64_t add, uint64_t timeout_ns) {
  const uint32_t off = cohort_local_offset(obj, die);
  if (off == 0u) return GSYNC_EINVAL;
  uint32_t* dnext = obj + off;
  uint32_t* drec = dnext + gsync::kLineWords;
  uint32_t* gnext = obj + 1 * gsync::kLineWords;
  uint32_t* grec = obj + 2 * gsync::kLineWords;
  const uint32_t b = pol[3] ? pol[3] : (uint32_t)GSYNC_COHORT_DEFAULT_BUDGET;
  const uint32_t cbudget = min(b, 127u), dbudget = min(b, 255u);
  // The cluster level: an MCS queue.  The tail (block 0's slot) names the last block to queue
  // as (rank + 1) | seq << 4; each block's own slot holds its node: the link its successor
  // writes, (rank, seq << 4, the holder's seq << 32), and the record its predecessor pushes.
  const uint32_t me = ptx::cluster_ctarank();
  uint32_t* tailp = &ptx::map_cluster_rank(slot, 0u)->cl.next;
  uint64_t* mylink = &slot->cl.turn;
  const uint32_t seq = ++slot->cl.pad;  // this block's queueings on the key (plain: only this thread)
  const uint32_t mine = (me + 1u) | (seq << 4);
  const uint32_t prev = ptx::atom_exch_relaxed_cluster(tailp, mine);
  gsync::Waiter w;
  uint64_t lo = 0, hi = 0;
  uint32_t seen_d = 0u;
  bool asked_d = false, owned = false;
  if (prev != 0u) {
    LocalSlot* ps = ptx::map_cluster_rank(slot, (prev & 0xFu) - 1u);
    ptx::st_relaxed_cluster_u64(&ps->cl.turn, (uint64_t)me | ((uint64_t)seq << 4) | ((uint64_t)(prev >> 4) << 32));
    seen_d = ptx::ld_relaxed(dnext);  // consumed only at the release, and only if past the die ticket
    asked_d = true;
    for (uint32_t polls = 1;; ++polls) {
      ptx::ld_relaxed_cluster_b128(slot->rec, lo, hi);  // this block's own shared memory
      if ((((uint32_t)lo ^ seq) & 0xFFFFu) == 0u) break;
      if ((polls & 31u) == 0u)
        if (int rc = w.tick(timeout_ns, obj + gsync::kHdrAbort)) return rc;
    }
    owned = (lo & kClusterOwned) != 0u;
  }
  uint32_t cp, dp, td, g;
  int64_t sum;
  if (owned) {
    cp = (uint32_t)(lo >> 17) & 0x7Fu;
    dp = (uint32_t)(lo >> 24) & 0xFFu;
    td = (uint32_t)(lo >> 32) & 0xFFFFu;
    g = (uint32_t)(lo >> 48) & 0xFFFFu;
    sum = (int64_t)hi;
  } else {
    // First of a cluster cohort: queue at the die level (at most one waiter per cluster).
    cp = 0u;
    td = ptx::atom_add_relaxed(dnext, 1u);
    uint32_t prev_d = 1u;
    for (;;) {
      if (prev_d <= 1u) seen_d = ptx::ld_relaxed(dnext);
      ptx::ld_relaxed_b128(drec, lo, hi);
      const uint32_t ahead = (td - (uint32_t)lo) & 0xFFFFu;
      if (ahead == 0u) break;
      prev_d = ahead;
      if (int rc = w.tick(timeout_ns, obj + gsync::kHdrAbort)) return rc;
    }
    asked_d = true;
    const uint32_t dword = (uint32_t)(lo >> 32);
    if (dword & gsync::kCohortOwned) {
      dp = (dword >> 16) & 0x7FFFu;
      g = dword & 0xFFFFu;
      sum = (int64_t)hi;
    } else {
      // First of a die cohort: queue for the global lock (at most one waiter per die).
      dp = 0u;
      g = ptx::atom_add_relaxed(gnext, 1u) & 0xFFFFu;
      for (;;) {
        seen_d = ptx::ld_relaxed(dnext);
        ptx::ld_relaxed_b128(grec, lo, hi);
        if (((uint32_t)lo & 0xFFFFu) == g) break;
        if (int rc = w.tick(timeout_ns, obj + gsync::kHdrAbort)) return rc;
      }
      sum = (int64_t)hi;
    }
    td &= 0xFFFFu;
  }
  // critical section: sum + add, published with the hand-off
  sum += add;
  const uint64_t s = (uint64_t)sum;
  uint64_t link = ptx::ld_relaxed_cluster_u64(mylink);
  bool linked = (uint32_t)(link >> 32) == seq;
  if (linked && cp + 1u < cbudget) {
    LocalSlot* ss = ptx::map_cluster_rank(slot, (uint32_t)link & 0xFu);
    const uint64_t rec = (uint64_t)(((uint32_t)link >> 4) & 0xFFFFu) | kClusterOwned | ((uint64_t)(cp + 1u) << 17) |
                         ((uint64_t)dp << 24) | ((uint64_t)td << 32) | ((uint64_t)g << 48);
    ptx::st_relaxed_cluster_b128(ss->rec, rec, s);
    return GSYNC_OK;
  }
  // Another cluster of this die waits iff the die counter is past td + 1 (a read made before
  // this cohort's die ticket was taken is behind it and says nothing: read again).
  uint32_t behind = (seen_d - (td + 1u)) & 0xFFFFu;
  if (!asked_d || behind >= 0x8000u) behind = (ptx::ld_relaxed(dnext) - (td + 1u)) & 0xFFFFu;
  if (dp + 1u < dbudget && behind != 0u && behind < 0x8000u) {
    const uint32_t dw = gsync::kCohortOwned | ((dp + 1u) << 16) | g;
    ptx::st_relaxed_b128(drec, (uint64_t)((td + 1u) & 0xFFFFu) | ((uint64_t)dw << 32), s);
  } else {
    ptx::st_relaxed_b128(grec, (uint64_t)((g + 1u) & 0xFFFFu), s);
    ptx::st_relaxed_b128(drec, (uint64_t)((td + 1u) & 0xFFFFu), s);
  }
  // Free the cluster level: push a record that is not owned to the successor, or swap the
  // tail back to empty; a block that swapped in meanwhile links itself shortly: wait for it.
  if (!linked) {
    link = ptx::ld_relaxed_cluster_u64(mylink);
    linked = (uint32_t)(link >> 32) == seq;
  }
  if (!linked) {
    if (ptx::atom_cas_relaxed_cluster(tailp, mine, 0u) == mine) return GSYNC_OK;
    for (;;) {
      link = ptx::ld_relaxed_cluster_u64(mylink);
      if ((uint32_t)(link >> 32) == seq) break;
      if (int rc = w.tick(timeout_ns, obj + gsync::kHdrAbort)) return rc;
    }
  }
  LocalSlot* ss = ptx::map_cluster_rank(slot, (uint32_t)link & 0xFu);
  ptx::st_relaxed_cluster_b128(ss->rec, (uint64_t)(((uint32_t)link >> 4) & 0xFFFFu), s);
  return GSYNC_OK;
}

// After the batched kernel: each carrying key's count and sum move from its record to count[]
// and sum[], and the record's count and sum return to zero (its turn stays, matching the
// ticket counter), so the next launch starts from zero like the other kinds' outputs.  A
// cohort-carrying key's count is the sum of its dies' ticket counters and its sum is in the
// global record; its counters, turns and records all return to zero.
__global__ void batched_collect_kernel(Args a) {
  const uint32_t key = blockIdx.x * blockDim.x + threadIdx.x;
  if (key >= (uint32_t)a.nkeys) return;
  const uint32_t cls = a.key_class[key];
  const uint32_t* pol = a.policy + 4u * (cls < (uint32_t)a.nclasses ? cls : 0u);
  if (uses_cohort_carry(a, pol, key)) {
    uint32_t* obj = a.cohort_state + (size_t)key * kCohortObjWords;
    const uint32_t off[2] = {cohort_local_offset(obj, 0u), cohort_local_offset(obj, 1u)};
    if (off[0] == 0u || off[1] == 0u) return;  // refused by the batched kernel already
    uint32_t n = 0;
    for (uint32_t d = 0; d < 2u; ++d) {
      uint32_t* local = obj + off[d];
      n += local[0];
      local[0] = 0u;
      uint64_t* lrec = (uint64_t*)(local + gsync::kLineWords);
      lrec[0] = 0;
      lrec[1] = 0;
    }
    uint64_t* grec = (uint64_t*)(obj + 2 * gsync::kLineWords);
    a.count[key] = n;
    a.sum[key] = (int64_t)grec[1];
    obj[1 * gsync::kLineWords] = 0u;
    grec[0] = 0;
    grec[1] = 0;
    return;
  }
  if (uses_hier_carry(a, pol, key)) {
    // count[] already holds the clusters' counts; the cohort object's global record holds the
    // sum; its global and die counters and records return to zero
    uint32_t* obj = a.cohort_state + (size_t)key * kCohortObjWords;
    const uint32_t off[2] = {cohort_local_offset(obj, 0u), cohort_local_offset(obj, 1u)};
    if (off[0] == 0u || off[1] == 0u) return;  // refused by the batched kernel already
    for (uint32_t d = 0; d < 2u; ++d) {
      uint32_t* local = obj + off[d];
      local[0] = 0u;
      uint64_t* drec = (uint64_t*)(local + gsync::kLineWords);
      drec[0] = 0;
      drec[1] = 0;
    }
    uint64_t* grec = (uint64_t*)(obj + 2 * gsync::kLineWords);
    a.sum[key] = (int64_t)grec[1];
    obj[1 * gsync::kLineWords] = 0u;
    grec[0] = 0;
    grec[1] = 0;
    return;
  }
  if (uses_cluster_carry(a, pol, key)) {
    // count[] already holds the clusters' counts; the global record holds the sum
    uint32_t* obj = a.mutex_state + key * kMutexObjWords;
    uint64_t* grec = (uint64_t*)(obj + 2 * gsync::kLineWords);
    a.sum[key] = (int64_t)grec[1];
    obj[1 * gsync::kLineWords] = 0u;
    grec[0] = 0;
    grec[1] = 0;
    return;
  }
  if (pol[0] != GSYNC_BATCHED_TICKET_CARRY && pol[0] != GSYNC_BATCHED_COHORT_CARRY &&
      pol[0] != GSYNC_BATCHED_CLUSTER_CARRY && pol[0] != GSYNC_BATCHED_CLUSTER_DIE_CARRY)
    return;
  uint64_t* rec = (uint64_t*)(a.mutex_state + key * kMutexObjWords + 2 * gsync::kLineWords);
  const uint64_t lo = rec[0];
  a.count[key] = (uint32_t)(lo >> 32);
  a.sum[key] = (int64_t)rec[1];
  rec[0] = lo & 0xFFFFFFFFull;
  rec[1] = 0;
}

// One crossing of the group barrier with the sampled slot check.
template <int BKIND>
__device__ __forceinline__ int group_cross(gsync::BarrierRef& bar, uint32_t* gslots, uint32_t gsize, uint32_t grank,
                                           uint32_t r, uint32_t& mix, uint32_t& bad) {
  uint32_t* buf = gslots + (r & 1u) * gsize;
  if (threadIdx.x == 0) buf[grank] = r * gsize + grank;
  const int rc = gsync::barrier_wait<BKIND>(bar);
  if (rc == GSYNC_OK && threadIdx.x == 0) {
    const uint32_t p = (grank + r + 1u) % gsize;
    const uint32_t v = buf[p];
    mix = rotl32(mix, 5) ^ lowbias32(v);
    bad += v != r * gsize + p;
  }
  return rc;
}

// MAXT: the largest block the instantiation runs.  Eight blocks per SM leave 32 registers a
// thread at 256 threads and 64 at 128; the 128-thread instantiation keeps thread 0's lock
// paths out of local memory (no spills).
template <int BKIND, int MAXT>
__global__ void __launch_bounds__(MAXT, 8) batched_kernel(Args a) {
  const uint32_t G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  __shared__ int s_fail;
  if (tid == 0) s_fail = 0;
  // The cluster cohort lock's local locks (one per key below kLocalKeys; block 0 of each
  // cluster holds the ones in use).  Initialised before any block of the cluster can use them,
  // and kept alive by the cluster barrier at the end of the kernel.
  __shared__ LocalSlot local_locks[BKIND == GSYNC_BAR_CLUSTER ? kLocalKeys : 1];
  if (BKIND == GSYNC_BAR_CLUSTER) {
    for (uint32_t i = tid; i < kLocalKeys; i += blockDim.x) {
      local_locks[i].cl.next = 0u;
      local_locks[i].cl.pad = 0u;
      local_locks[i].cl.turn = 0ull;
      local_locks[i].rec[0] = 0ull;
      local_locks[i].rec[1] = 0ull;
    }
    ptx::cluster_sync();
  }
  // The die of this block's SM, from the die table every cohort object carries.
  uint32_t die = 0;
  if (a.ncohort > 0 && tid == 0) {
    const uint32_t sm = ptx::smid();
    die = sm < gsync::kMaxSmIds && ((const uint8_t*)(a.cohort_state + gsync::kDieTableWord))[sm] ? 1u : 0u;
  }
  int g = a.group_of_block[b];
  if (g >= a.ngroups) g = -1;
  gsync::BarrierRef bar;
  uint32_t gsize = 0, grank = 0;
  uint32_t* gslots = nullptr;
  if (g >= 0) {
    gsize = (uint32_t)a.group_size[g];
    grank = b - (uint32_t)a.group_start[g];
    bool ok = grank < gsize && gsize >= 1u && (uint32_t)a.group_start[g] + gsize <= G;
    if (BKIND == GSYNC_BAR_CLUSTER) {
      // The hardware cluster barrier cannot time out, so every block of this block's cluster
      // must be in the same group; every block of the cluster reads the same entries and so
      // reaches the same verdict before any cluster barrier runs.
      const uint32_t c = ptx::cluster_nctarank(), c0 = b - ptx::cluster_ctarank();
      ok = ok && ((uint32_t)a.group_start[g] % c == 0u) && (gsize % c == 0u);
      for (uint32_t k = 0; k < c; ++k) ok = ok && a.group_of_block[c0 + k] == g;
    }
    if (!ok) {
      if (tid == 0) ptx::atom_or_relaxed(a.status, GSYNC_STATUS_CONFIG);
      g = -1;
    }
  }
  if (g >= 0) {
    gslots = a.slots + 2u * (uint32_t)a.group_start[g];
    bar.s = a.group_state + (uint32_t)g * kBarObjWords;
    bar.kind = BKIND;
    bar.n = gsize;
    bar.param = BKIND == GSYNC_BAR_CLUSTER ? ptx::cluster_nctarank() : 0u;
    bar.mode = 0;
    bar.timeout_ns = a.timeout_ns;
    bar.epoch = ptx::ld_relaxed(bar.line(2));
  }
  const uint32_t nacq = (uint32_t)a.nacq;
  const uint32_t nmine = b < nacq ? (nacq - 1u - b) / G + 1u : 0u;
  const uint32_t rounds = g >= 0 ? (uint32_t)a.rounds : 0u;
  uint32_t crossed = 0, mix = 0, bad = 0;
  int bar_rc = GSYNC_OK;
  __syncthreads();
  for (uint32_t j = 0; j < nmine; ++j) {
    if (tid == 0 && !s_fail) {
      const uint32_t i = b + j * G;
      const uint32_t key = (uint32_t)a.keys[i];
      // The addend is this block's own input: read it before the lock, so that its load (from
      // DRAM on a launch's first touch) overlaps the wait instead of lengthening the section.
      const int64_t add = a.adds[i];
      if (key >= (uint32_t)a.nkeys) {
        ptx::atom_or_relaxed(a.status, GSYNC_STATUS_VIOLATION);
        s_fail = 1;
      } else {
        const uint32_t cls = a.key_class[key];
        const uint32_t* pol = a.policy + 4u * (cls < (uint32_t)a.nclasses ? cls : 0u);
        if (pol[0] == GSYNC_BATCHED_TICKET_CARRY || pol[0] == GSYNC_BATCHED_COHORT_CARRY ||
            pol[0] == GSYNC_BATCHED_CLUSTER_CARRY || pol[0] == GSYNC_BATCHED_CLUSTER_DIE_CARRY) {
          int rc;
          if (BKIND == GSYNC_BAR_CLUSTER && uses_hier_carry(a, pol, key))
            rc = hier_carry_add(&local_locks[key], a.cohort_state + (size_t)key * kCohortObjWords, die, pol, add,
                                a.timeout_ns);
          else if (BKIND == GSYNC_BAR_CLUSTER && uses_cluster_carry(a, pol, key))
            rc = cluster_carry_add(ptx::map_cluster_rank(&local_locks[key], 0u), a.mutex_state + key * kMutexObjWords,
                                   pol, add, a.timeout_ns);
          else if (uses_cohort_carry(a, pol, key))
            rc = cohort_carry_add(a.cohort_state + (size_t)key * kCohortObjWords, die, pol, add, a.timeout_ns);
          else
            rc = carry_add(a.mutex_state + key * kMutexObjWords, pol, add, a.timeout_ns);
          if (rc != GSYNC_OK) {
            record_status(a.status, rc);
            s_fail = 1;
          }
        } else {
        gsync::MutexRef m;
        m.s = a.mutex_state + key * kMutexObjWords;
        const bool cohort = BKIND == GSYNC_BAR_CLUSTER && pol[0] == (uint32_t)GSYNC_MUTEX_CLUSTER && key < kLocalKeys;
        m.kind = cohort ? (uint32_t)GSYNC_MUTEX_CLUSTER
                        : pol[0] <= (uint32_t)GSYNC_MUTEX_TICKET ? pol[0] : (uint32_t)GSYNC_MUTEX_TICKET;
        // cohort budget (fourth policy word, 0 = the default), kept as budget - 1
        m.qmask = cohort ? (pol[3] ? min(pol[3], 32767u) : (uint32_t)GSYNC_COHORT_DEFAULT_BUDGET) - 1u : 0u;
        m.cl = cohort ? ptx::map_cluster_rank(&local_locks[key].cl, 0u) : nullptr;
        m.local = nullptr;
        m.die = 0;
        m.bo.policy = GSYNC_BACKOFF_EXPONENTIAL;
        m.bo.min_ns = pol[1];
        m.bo.max_ns = pol[2];
        m.bo.spin = 0;
        m.timeout_ns = a.timeout_ns;
        const gsync::Token t = lock_by_policy(m);
        if (t.status != GSYNC_OK) {
          record_status(a.status, t.status);
          s_fail = 1;
        } else {
          a.sum[key] += add;
          a.count[key] += 1u;
          unlock_by_policy(m, t);
        }
        }
      }
    }
    if (rounds) {
      const uint32_t target = (uint32_t)(((uint64_t)(j + 1u) * rounds) / nmine);
      while (crossed < target) {
        const int rc = group_cross<BKIND>(bar, gslots, gsize, grank, crossed++, mix, bad);
        if (bar_rc == GSYNC_OK) bar_rc = rc;
      }
    }
  }
  // Every member crosses all rounds, also after an error (see the CLUSTER barrier's note).
  while (crossed < rounds) {
    const int rc = group_cross<BKIND>(bar, gslots, gsize, grank, crossed++, mix, bad);
    if (bar_rc == GSYNC_OK) bar_rc = rc;
  }
  if (tid == 0) {
    if (bar_rc != GSYNC_OK) record_status(a.status, bar_rc);
    a.mix[b] = mix;
    a.bad[b] = bad;
  }
  if (BKIND == GSYNC_BAR_CLUSTER) {
    ptx::cluster_sync();  // block 0's local locks outlive every user
    // The cluster carrying locks' acquisitions of each key: counted by the cluster's ticket
    // (block 0's slot), or by each block's own queueings on the MCS level.
    const bool rank0 = ptx::cluster_ctarank() == 0;
    for (uint32_t key = tid; key < kLocalKeys && key < (uint32_t)a.nkeys; key += blockDim.x) {
      const uint32_t cls = a.key_class[key];
      const uint32_t* pol = a.policy + 4u * (cls < (uint32_t)a.nclasses ? cls : 0u);
      const uint32_t n = uses_hier_carry(a, pol, key) ? local_locks[key].cl.pad
                         : rank0 && uses_cluster_carry(a, pol, key) ? local_locks[key].cl.next : 0u;
      if (n) ptx::red_add_relaxed(a.count + key, n);
    }
  }
}

template <int MAXT>
int launch_batched(const gsync_batched_work* w, int cluster, const Args& a, cudaStream_t st) {
  if (cluster > 1)
    return launch_coresident(batched_kernel<GSYNC_BAR_CLUSTER, MAXT>, w->nblocks, w->block_threads, cluster, 0, st, a);
  if (w->plain_launch) {
    // For stream capture: an ordinary launch after the same co-residency check.  All blocks
    // are resident as long as no other kernel occupies the GPU when the graph runs.
    int maxb = 0;
    if (int rc = max_coresident(batched_kernel<GSYNC_BAR_ATOMIC, MAXT>, w->block_threads, 1, 0, &maxb)) return rc;
    if (w->nblocks > maxb) return GSYNC_ENOTRESIDENT;
    batched_kernel<GSYNC_BAR_ATOMIC, MAXT><<<w->nblocks, w->block_threads, 0, st>>>(a);
    GSYNC_CUDA(cudaGetLastError());
    return GSYNC_OK;
  }
  return launch_coresident(batched_kernel<GSYNC_BAR_ATOMIC, MAXT>, w->nblocks, w->block_threads, 1, 0, st, a);
}

}  // namespace

extern "C" int gsync_bench_batched(const gsync_batched_work* w, void* stream) {
  if (!w || w->nkeys < 1 || w->nacq < 0 || w->nblocks < 1 || w->ngroups < 0 || w->rounds < 0 || w->nclasses < 1 ||
      w->block_threads < 32 || w->block_threads > kMaxThreads || w->block_threads % 32)
    return GSYNC_EINVAL;
  if (!w->mutex_state || !w->key_class || !w->policy || !w->keys || !w->adds || !w->sum || !w->count ||
      !w->group_of_block || !w->mix || !w->bad || !w->status || !aligned(w->mutex_state, 128))
    return GSYNC_EINVAL;
  if (w->ngroups > 0 && (!w->group_start || !w->group_size || !w->group_state || !w->slots ||
                         !aligned(w->group_state, 128)))
    return GSYNC_EINVAL;
  if (w->ncohort < 0 || (w->ncohort > 0 && (!w->cohort_state || !aligned(w->cohort_state, 128))))
    return GSYNC_EINVAL;
  const int cluster = w->cluster < 1 ? 1 : w->cluster;
  if (cluster > 8 || w->nblocks % cluster) return GSYNC_EINVAL;
  Args a;
  a.mutex_state = (uint32_t*)w->mutex_state;
  a.key_class = w->key_class;
  a.policy = w->policy;
  a.keys = w->keys;
  a.adds = w->adds;
  a.sum = w->sum;
  a.count = w->count;
  a.group_start = w->group_start;
  a.group_size = w->group_size;
  a.group_of_block = w->group_of_block;
  a.group_state = (uint32_t*)w->group_state;
  a.slots = w->slots;
  a.mix = w->mix;
  a.bad = w->bad;
  a.status = w->status;
  a.cohort_state = (uint32_t*)w->cohort_state;
  a.ncohort = w->ncohort < w->nkeys ? w->ncohort : w->nkeys;
  a.clustered = w->cluster > 1 ? 1 : 0;
  a.timeout_ns = w->timeout_ns ? w->timeout_ns : 2000000000ull;
  a.nkeys = w->nkeys;
  a.nacq = w->nacq;
  a.rounds = w->rounds;
  a.nclasses = w->nclasses;
  a.ngroups = w->ngroups;
  cudaStream_t st = (cudaStream_t)stream;
  const int rc = w->block_threads <= 128 ? launch_batched<128>(w, cluster, a, st)
                                          : launch_batched<kMaxThreads>(w, cluster, a, st);
  if (rc != GSYNC_OK) return rc;
  batched_collect_kernel<<<(w->nkeys + 255) / 256, 256, 0, st>>>(a);
  GSYNC_CUDA(cudaGetLastError());
  return GSYNC_OK;
}
