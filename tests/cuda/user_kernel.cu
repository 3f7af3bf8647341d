// A program written the way a user of the library writes one: its own kernels call the
// device primitives of gsync_device.cuh, the objects are created through the C ABI, and the
// grids are launched through the library's co-residency gate.
//   user_kernel: the counting barrier and the two-die cohort mutex, a plain launch.
//   user_kernel_cluster: the GB300 defaults -- the counting barrier, the cluster cohort mutex
//     (its local lock, or each block's MCS node, in the kernel's shared memory) and the
//     ticket-window semaphore -- in launches with clusters of 4 and 8.
//   user_kernel_exchange: the exchange barrier as an all-gather, over two launches.
//   bounded_waits_kernel: the per-call wait bounds of sem_wait, mutex_lock and barrier_wait.
// Checked exactly: every round of the barrier sees every block's value of that round, a
// counter updated with plain loads and stores under the mutex ends at blocks x rounds, and
// the semaphore never admits more than its count.  Prints "OK" and exits 0 on success.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "gsync.h"
#include "gsync_device.cuh"

__global__ void user_kernel(void* bar_state, void* mutex_state, uint32_t* slots, uint32_t* counter,
                            uint32_t* bad, int rounds) {
  gsync::BarrierRef bar = gsync::barrier_attach(bar_state);
  const gsync::MutexRef m = gsync::mutex_attach(mutex_state);
  const uint32_t b = blockIdx.x, B = gridDim.x;
  for (int r = 0; r < rounds; ++r) {
    uint32_t* buf = slots + (r & 1) * B;  // double-buffered by round parity
    if (threadIdx.x == 0) buf[b] = (uint32_t)r * B + b;
    if (gsync::barrier_wait<GSYNC_BAR_COUNT>(bar) != GSYNC_OK) {
      if (threadIdx.x == 0) atomicAdd(bad, 1u);
      return;
    }
    if (threadIdx.x == 0) {
      const uint32_t p = (b + (uint32_t)r + 1u) % B;
      if (buf[p] != (uint32_t)r * B + p) atomicAdd(bad, 1u);
    }
    gsync::Token t = gsync::mutex_lock<GSYNC_MUTEX_COHORT>(m);
    if (t.status != GSYNC_OK) {
      if (threadIdx.x == 0) atomicAdd(bad, 1u);
      return;
    }
    if (threadIdx.x == 0) *counter = *counter + 1u;  // plain read-modify-write under the mutex
    gsync::mutex_unlock<GSYNC_MUTEX_COHORT>(m, t);
  }
}

// MKIND: the cluster cohort lock in its ticket form (GSYNC_MUTEX_CLUSTER) or its MCS form
// (GSYNC_MUTEX_CLUSTER_MCS, the GB300 default), each attached its own way.
template <int MKIND>
__global__ void user_kernel_cluster(void* bar_state, void* mutex_state, void* sem_state, uint32_t* slots,
                                    uint32_t* counter, uint32_t* bad, uint32_t* occ, int rounds) {
  __shared__ gsync::ClusterLocal cluster_lock;
  __shared__ gsync::McsNode node;
  gsync::BarrierRef bar = gsync::barrier_attach(bar_state);
  const gsync::MutexRef m = MKIND == GSYNC_MUTEX_CLUSTER_MCS ? gsync::mutex_attach_cluster_mcs(mutex_state, &node)
                                                             : gsync::mutex_attach_cluster(mutex_state, &cluster_lock);
  const gsync::SemRef s = gsync::sem_attach(sem_state);
  const uint32_t b = blockIdx.x, B = gridDim.x;
  bool ok = true;
  for (int r = 0; r < rounds && ok; ++r) {
    uint32_t* buf = slots + (r & 1) * B;
    if (threadIdx.x == 0) buf[b] = (uint32_t)r * B + b;
    if (gsync::barrier_wait<GSYNC_BAR_COUNT>(bar) != GSYNC_OK) {
      ok = false;
      break;
    }
    if (threadIdx.x == 0) {
      const uint32_t p = (b + (uint32_t)r + 1u) % B;
      if (buf[p] != (uint32_t)r * B + p) atomicAdd(bad, 1u);
    }
    gsync::Token t = gsync::mutex_lock<MKIND>(m);
    if (t.status != GSYNC_OK) {
      ok = false;
      break;
    }
    if (threadIdx.x == 0) *counter = *counter + 1u;  // plain read-modify-write under the mutex
    gsync::mutex_unlock<MKIND>(m, t);
    if (gsync::sem_wait<GSYNC_SEM_WINDOW>(s) != GSYNC_OK) {
      ok = false;
      break;
    }
    if (threadIdx.x == 0) {
      const uint32_t o = atomicAdd(occ, 1u) + 1u;  // holders inside, and the most seen
      atomicMax(occ + 1, o);
      atomicSub(occ, 1u);
    }
    gsync::sem_post<GSYNC_SEM_WINDOW>(s);
  }
  if (!ok && threadIdx.x == 0) atomicAdd(bad, 1u);
  gsync::mutex_cluster_end();  // the cluster's shared memory outlives every user in it
}

// The exchange barrier as an all-gather: each round every block publishes one value and reads
// two others' (its right neighbour's and block 0's) after the crossing.
__global__ void user_kernel_exchange(void* bar_state, uint32_t* bad, int rounds) {
  gsync::BarrierRef bar = gsync::barrier_attach(bar_state);
  const uint32_t b = blockIdx.x, B = gridDim.x;
  for (int r = 0; r < rounds; ++r) {
    const uint64_t mine = ((uint64_t)r << 32) | (b * 7u + 1u);
    if (gsync::barrier_exchange(bar, mine) != GSYNC_OK) {
      if (threadIdx.x == 0) atomicAdd(bad, 1u);
      return;
    }
    if (threadIdx.x < 2) {
      const uint32_t q = threadIdx.x == 0 ? (b + 1u) % B : 0u;
      uint64_t v = 0;
      const int rc = gsync::barrier_exchange_read(bar, q, v);
      if (rc != GSYNC_OK || v != (((uint64_t)r << 32) | (q * 7u + 1u))) atomicAdd(bad, 1u);
    }
  }
}

// The per-call wait bounds: block 0 takes the semaphore's only permit and then waits for a
// second one, takes the mutex and then asks for it again, and waits at a barrier that block 1
// never reaches -- each second wait bounded at 1 ms, so each must return GSYNC_ETIMEDOUT after
// about that long (rc[i], elapsed ns in ns_out[i]).
__global__ void bounded_waits_kernel(void* sem_state, void* mutex_state, void* bar_state, int* rc, uint64_t* ns_out) {
  if (blockIdx.x != 0) return;  // block 1 never arrives at the barrier
  const gsync::SemRef s = gsync::sem_attach(sem_state);
  const gsync::MutexRef m = gsync::mutex_attach(mutex_state);
  gsync::BarrierRef bar = gsync::barrier_attach(bar_state);
  const uint64_t bound = 1000000ull;
  uint64_t t0;
  int r = gsync::sem_wait<GSYNC_SEM_WINDOW>(s);
  t0 = gsync::ptx::globaltimer();
  if (r == GSYNC_OK) r = gsync::sem_wait<GSYNC_SEM_WINDOW>(s, bound);
  if (threadIdx.x == 0) { rc[0] = r; ns_out[0] = gsync::ptx::globaltimer() - t0; }
  gsync::Token t = gsync::mutex_lock<GSYNC_MUTEX_TICKET>(m);
  t0 = gsync::ptx::globaltimer();
  r = t.status == GSYNC_OK ? gsync::mutex_lock<GSYNC_MUTEX_TICKET>(m, bound).status : t.status;
  if (threadIdx.x == 0) { rc[1] = r; ns_out[1] = gsync::ptx::globaltimer() - t0; }
  t0 = gsync::ptx::globaltimer();
  r = gsync::barrier_wait<GSYNC_BAR_COUNT>(bar, bound);
  if (threadIdx.x == 0) { rc[2] = r; ns_out[2] = gsync::ptx::globaltimer() - t0; }
}

// The cluster barrier's counting forms (1: every block polls the leaders' counter; 2: the
// other blocks of a cluster wait at a second cluster barrier for their leader): the second
// cluster of the grid never arrives, so the leaders' count stays short and the bounded wait
// (1 ms) of both blocks of the first cluster must end with an error: GSYNC_ETIMEDOUT for the
// block whose wait ran out first, GSYNC_EABORTED or GSYNC_ETIMEDOUT for the other (the first
// marks the object aborted) -- in form 2 the leader's result reaches its cluster through the
// leader's shared memory, so both report the leader's.
__global__ void bounded_cluster_wait_kernel(void* bar_state, int* rc, uint64_t* ns_out) {
  if (blockIdx.x >= 2) return;  // the second cluster (blocks 2 and 3) never arrives
  gsync::BarrierRef bar = gsync::barrier_attach(bar_state);
  const uint64_t t0 = gsync::ptx::globaltimer();
  const int r = gsync::barrier_wait<GSYNC_BAR_CLUSTER>(bar, 1000000ull);
  if (threadIdx.x == 0) { rc[blockIdx.x] = r; ns_out[blockIdx.x] = gsync::ptx::globaltimer() - t0; }
}

#define CHECK(x)                                                              \
  do {                                                                        \
    int rc_ = (int)(x);                                                       \
    if (rc_) {                                                                \
      printf("FAIL %s = %d (cuda %d) line %d\n", #x, rc_, gsync_last_cuda_error(), __LINE__); \
      return 1;                                                               \
    }                                                                         \
  } while (0)

int main() {
  const int threads = 128, rounds = 500;
  cudaFunction_t f;
  CHECK(cudaGetFuncBySymbol(&f, (const void*)user_kernel));
  int maxb = 0;
  CHECK(gsync_check_coresident((const void*)f, 1, threads, 0, 1, &maxb));
  // A grid one block larger than fits must be refused before anything runs.
  if (gsync_check_coresident((const void*)f, maxb + 1, threads, 0, 1, &maxb) != GSYNC_ENOTRESIDENT) {
    printf("FAIL oversized grid not refused\n");
    return 1;
  }
  const int B = maxb < 1184 ? maxb : 1184;
  void *bar = nullptr, *mtx = nullptr;
  uint32_t *slots = nullptr, *counter = nullptr, *bad = nullptr;
  const size_t bar_bytes = gsync_barrier_bytes(GSYNC_BAR_COUNT, B, 8);
  const size_t mtx_bytes = gsync_mutex_bytes(GSYNC_MUTEX_COHORT, B);
  CHECK(cudaMalloc(&bar, bar_bytes));
  CHECK(cudaMalloc(&mtx, mtx_bytes));
  CHECK(cudaMalloc(&slots, 2 * B * sizeof(uint32_t)));
  CHECK(cudaMalloc(&counter, 2 * sizeof(uint32_t)));
  bad = counter + 1;
  CHECK(cudaMemset(counter, 0, 2 * sizeof(uint32_t)));
  CHECK(gsync_barrier_init(bar, bar_bytes, GSYNC_BAR_COUNT, B, 8, 0, nullptr));
  gsync_backoff bo = {GSYNC_BACKOFF_EXPONENTIAL, 128, 4000, 0};
  CHECK(gsync_mutex_init(mtx, mtx_bytes, GSYNC_MUTEX_COHORT, B, &bo, 0, nullptr));
  int r = rounds;
  void* args[] = {&bar, &mtx, &slots, &counter, &bad, &r};
  CHECK(gsync_launch_coresident((const void*)f, B, threads, 0, 1, args, nullptr));
  CHECK(cudaDeviceSynchronize());
  uint32_t h[2];
  CHECK(cudaMemcpy(h, counter, sizeof h, cudaMemcpyDeviceToHost));
  if (h[1] != 0 || h[0] != (uint32_t)B * rounds) {
    printf("FAIL counter %u (want %u), bad %u\n", h[0], (uint32_t)B * rounds, h[1]);
    return 1;
  }

  // The exchange barrier on the same grid.
  {
    cudaFunction_t fx;
    CHECK(cudaGetFuncBySymbol(&fx, (const void*)user_kernel_exchange));
    int maxx = 0;
    CHECK(gsync_check_coresident((const void*)fx, 1, threads, 0, 1, &maxx));
    const int BX = maxx < 1184 ? maxx : 1184;
    void* xbar = nullptr;
    const size_t xbytes = gsync_barrier_bytes(GSYNC_BAR_EXCHANGE, BX, 8);
    CHECK(cudaMalloc(&xbar, xbytes));
    CHECK(gsync_barrier_init(xbar, xbytes, GSYNC_BAR_EXCHANGE, BX, 8, 0, nullptr));
    CHECK(cudaMemset(bad, 0, sizeof(uint32_t)));
    void* xargs[] = {&xbar, &bad, &r};
    for (int launch = 0; launch < 2; ++launch) {  // the second launch continues the epochs
      CHECK(gsync_launch_coresident((const void*)fx, BX, threads, 0, 1, xargs, nullptr));
      CHECK(cudaDeviceSynchronize());
    }
    uint32_t hb = 0;
    CHECK(cudaMemcpy(&hb, bad, sizeof hb, cudaMemcpyDeviceToHost));
    if (hb != 0) {
      printf("FAIL exchange kernel: %u bad reads\n", hb);
      return 1;
    }
    CHECK(cudaFree(xbar));
  }

  // The GB300 defaults in a cluster launch: the counting barrier, the ticket-window semaphore,
  // and the cluster cohort lock in its ticket form (clusters of 4) and its MCS form (clusters
  // of 8, the default).
  int cl_blocks[2] = {0, 0};
  uint32_t cl_max[2] = {0u, 0u};
  for (int form = 0; form < 2; ++form) {
    const int mkind = form ? GSYNC_MUTEX_CLUSTER_MCS : GSYNC_MUTEX_CLUSTER;
    cudaFunction_t fc;
    CHECK(cudaGetFuncBySymbol(&fc, form ? (const void*)user_kernel_cluster<GSYNC_MUTEX_CLUSTER_MCS>
                                        : (const void*)user_kernel_cluster<GSYNC_MUTEX_CLUSTER>));
    const int C = form ? 8 : 4, n = 4;
    int maxc = 0;
    CHECK(gsync_check_coresident((const void*)fc, C, threads, 0, C, &maxc));
    const int BC = (maxc < 1184 ? maxc : 1184) / C * C;
    void *bar2 = nullptr, *mtx2 = nullptr, *sem = nullptr;
    uint32_t* w = nullptr;  // counter, bad, occupancy, max occupancy
    uint32_t* slots2 = nullptr;
    const size_t bar2_bytes = gsync_barrier_bytes(GSYNC_BAR_COUNT, BC, 8);
    const size_t mtx2_bytes = gsync_mutex_bytes(mkind, BC);
    const size_t sem_bytes = gsync_sem_bytes(GSYNC_SEM_WINDOW);
    CHECK(cudaMalloc(&bar2, bar2_bytes));
    CHECK(cudaMalloc(&mtx2, mtx2_bytes));
    CHECK(cudaMalloc(&sem, sem_bytes));
    CHECK(cudaMalloc(&w, 4 * sizeof(uint32_t)));
    CHECK(cudaMalloc(&slots2, 2 * BC * sizeof(uint32_t)));
    CHECK(cudaMemset(w, 0, 4 * sizeof(uint32_t)));
    CHECK(gsync_barrier_init(bar2, bar2_bytes, GSYNC_BAR_COUNT, BC, 8, 0, nullptr));
    CHECK(gsync_mutex_init(mtx2, mtx2_bytes, mkind, BC, &bo, 0, nullptr));
    gsync_backoff sbo = {GSYNC_BACKOFF_EXPONENTIAL, 16, 2000, 0};
    CHECK(gsync_sem_init(sem, sem_bytes, GSYNC_SEM_WINDOW, n, &sbo, 0, nullptr));
    uint32_t *cnt2 = w, *bad2 = w + 1, *occ = w + 2;
    void* args2[] = {&bar2, &mtx2, &sem, &slots2, &cnt2, &bad2, &occ, &r};
    CHECK(gsync_launch_coresident((const void*)fc, BC, threads, 0, C, args2, nullptr));
    CHECK(cudaDeviceSynchronize());
    uint32_t h2[4];
    CHECK(cudaMemcpy(h2, w, sizeof h2, cudaMemcpyDeviceToHost));
    if (h2[1] != 0 || h2[0] != (uint32_t)BC * rounds || h2[2] != 0 || h2[3] < 1 || h2[3] > (uint32_t)n) {
      printf("FAIL cluster kernel (mutex kind %d): counter %u (want %u), bad %u, occupancy %u, max %u (n %d)\n",
             mkind, h2[0], (uint32_t)BC * rounds, h2[1], h2[2], h2[3], n);
      return 1;
    }
    cl_blocks[form] = BC;
    cl_max[form] = h2[3];
  }

  // Per-call wait bounds: each second wait must end with GSYNC_ETIMEDOUT after ~1 ms (the
  // objects' own timeouts are 10 s).
  cudaFunction_t fb;
  CHECK(cudaGetFuncBySymbol(&fb, (const void*)bounded_waits_kernel));
  void *sem3 = nullptr, *mtx3 = nullptr, *bar3 = nullptr;
  int* rc3 = nullptr;
  uint64_t* ns3 = nullptr;
  const size_t bar3_bytes = gsync_barrier_bytes(GSYNC_BAR_COUNT, 2, 0);
  CHECK(cudaMalloc(&sem3, gsync_sem_bytes(GSYNC_SEM_WINDOW)));
  CHECK(cudaMalloc(&mtx3, gsync_mutex_bytes(GSYNC_MUTEX_TICKET, 2)));
  CHECK(cudaMalloc(&bar3, bar3_bytes));
  CHECK(cudaMalloc(&rc3, 3 * sizeof(int)));
  CHECK(cudaMalloc(&ns3, 3 * sizeof(uint64_t)));
  const uint64_t own = 10000000000ull;
  CHECK(gsync_sem_init(sem3, gsync_sem_bytes(GSYNC_SEM_WINDOW), GSYNC_SEM_WINDOW, 1, nullptr, own, nullptr));
  CHECK(gsync_mutex_init(mtx3, gsync_mutex_bytes(GSYNC_MUTEX_TICKET, 2), GSYNC_MUTEX_TICKET, 2, nullptr, own, nullptr));
  CHECK(gsync_barrier_init(bar3, bar3_bytes, GSYNC_BAR_COUNT, 2, 0, own, nullptr));
  void* args3[] = {&sem3, &mtx3, &bar3, &rc3, &ns3};
  CHECK(gsync_launch_coresident((const void*)fb, 2, threads, 0, 1, args3, nullptr));
  CHECK(cudaDeviceSynchronize());
  int hrc[3];
  uint64_t hns[3];
  CHECK(cudaMemcpy(hrc, rc3, sizeof hrc, cudaMemcpyDeviceToHost));
  CHECK(cudaMemcpy(hns, ns3, sizeof hns, cudaMemcpyDeviceToHost));
  for (int i = 0; i < 3; ++i)
    if (hrc[i] != GSYNC_ETIMEDOUT || hns[i] < 1000000ull || hns[i] > 200000000ull) {
      printf("FAIL bounded wait %d: rc %d after %llu ns\n", i, hrc[i], (unsigned long long)hns[i]);
      return 1;
    }
  // The same bound in the cluster barrier's counting forms, in a launch with clusters of 2.
  cudaFunction_t fcb;
  CHECK(cudaGetFuncBySymbol(&fcb, (const void*)bounded_cluster_wait_kernel));
  for (int form = 1; form <= 2; ++form) {
    const int param = 2 | form << 4;
    const size_t bytes = gsync_barrier_bytes(GSYNC_BAR_CLUSTER, 4, param);
    void* bar4 = nullptr;
    CHECK(cudaMalloc(&bar4, bytes));
    CHECK(gsync_barrier_init(bar4, bytes, GSYNC_BAR_CLUSTER, 4, param, own, nullptr));
    CHECK(cudaMemset(rc3, 0, 2 * sizeof(int)));
    void* args4[] = {&bar4, &rc3, &ns3};
    CHECK(gsync_launch_coresident((const void*)fcb, 4, threads, 0, 2, args4, nullptr));
    CHECK(cudaDeviceSynchronize());
    CHECK(cudaMemcpy(hrc, rc3, 2 * sizeof(int), cudaMemcpyDeviceToHost));
    CHECK(cudaMemcpy(hns, ns3, 2 * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    bool timed_out = false;
    for (int i = 0; i < 2; ++i) {
      timed_out = timed_out || hrc[i] == GSYNC_ETIMEDOUT;
      if ((hrc[i] != GSYNC_ETIMEDOUT && hrc[i] != GSYNC_EABORTED) || hns[i] < 1000000ull || hns[i] > 200000000ull) {
        printf("FAIL cluster barrier form %d, block %d: rc %d after %llu ns\n", form, i, hrc[i],
               (unsigned long long)hns[i]);
        return 1;
      }
    }
    if (!timed_out || (form == 2 && hrc[0] != hrc[1])) {
      printf("FAIL cluster barrier form %d: rc %d / %d\n", form, hrc[0], hrc[1]);
      return 1;
    }
    CHECK(cudaFree(bar4));
  }
  printf("OK %d blocks x %d rounds; in clusters (ticket form, MCS form): %d / %d blocks, at most %u / %u of 4 "
         "inside; bounded waits ended after %.2f / %.2f / %.2f ms\n", B, rounds, cl_blocks[0], cl_blocks[1],
         cl_max[0], cl_max[1], hns[0] / 1e6, hns[1] / 1e6, hns[2] / 1e6);
  return 0;
}
