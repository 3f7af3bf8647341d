// A program written the way a user of the library writes one: its own kernel calls the
// device primitives of gsync_device.cuh (the counting barrier and the cohort mutex), the
// objects are created through the C ABI, and the grid is launched through the library's
// co-residency gate.  Checked exactly: every round of the barrier sees every block's value of
// that round, and a counter updated with plain loads and stores under the mutex ends at
// blocks x rounds.  Prints "OK" and exits 0 on success.
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
  printf("OK %d blocks x %d rounds\n", B, rounds);
  return 0;
}
