// Internal helpers shared by the library's translation units: CUDA error capture, argument
// checks and the co-resident launch (Section 5: a grid barrier is only safe when every block
// of the grid is resident at once -- the "persistent threads" requirement).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "gsync.h"
#include "gsync_device.cuh"

namespace gsync_impl {

// Last CUDA error seen on this host thread (read with gsync_last_cuda_error()).
extern thread_local int g_last_cuda_error;

inline int cuda_fail(cudaError_t e) {
  g_last_cuda_error = (int)e;
  (void)cudaGetLastError();  // clear a sticky-free launch error so later calls are clean
  return GSYNC_ECUDA;
}

#define GSYNC_CUDA(call)                                         \
  do {                                                           \
    cudaError_t e_ = (call);                                     \
    if (e_ != cudaSuccess) return ::gsync_impl::cuda_fail(e_);   \
  } while (0)

inline bool aligned(const void* p, uintptr_t a) { return ((uintptr_t)p & (a - 1)) == 0; }

inline int device_sms(int* sms) {
  int dev = 0;
  GSYNC_CUDA(cudaGetDevice(&dev));
  GSYNC_CUDA(cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev));
  return GSYNC_OK;
}

// Largest co-resident grid of `kernel` with `block` threads (and clusters of `cluster`).
template <typename... Params>
int max_coresident(void (*kernel)(Params...), int block, int cluster, size_t smem, int* out) {
  if (cluster > 1) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)cluster);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    GSYNC_CUDA(cudaOccupancyMaxActiveClusters(&clusters, (const void*)kernel, &cfg));
    *out = clusters * cluster;
    return GSYNC_OK;
  }
  int per_sm = 0, sms = 0;
  GSYNC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem));
  if (int rc = device_sms(&sms)) return rc;
  *out = per_sm * sms;
  return GSYNC_OK;
}

// Launches `kernel` so that all `grid` blocks are resident together, or refuses with
// GSYNC_ENOTRESIDENT before anything runs: a cooperative launch without clusters, and an
// occupancy-checked launch with cluster dimensions otherwise.
template <typename... Params, typename... Args>
int launch_coresident(void (*kernel)(Params...), int grid, int block, int cluster, size_t smem,
                      cudaStream_t stream, Args... args) {
  int maxb = 0;
  if (int rc = max_coresident(kernel, block, cluster, smem, &maxb)) return rc;
  if (grid > maxb) return GSYNC_ENOTRESIDENT;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  if (cluster > 1) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
  } else {
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
  }
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, args...);
  if (e == cudaErrorCooperativeLaunchTooLarge) return GSYNC_ENOTRESIDENT;
  if (e != cudaSuccess) return cuda_fail(e);
  return GSYNC_OK;
}

// SM-to-die map of the current device (0/1 per SM id; measured on first use, then cached),
// and the home die of `nlines` lines base + i * stride (<= 256 lines; synchronizes `st`).
int device_topology(cudaStream_t st, uint8_t* die_of_sm, int* ndies, int* sms);
int line_homes(const void* base, int nlines, size_t stride, const uint8_t* die_of_sm, int sms, cudaStream_t st,
               uint8_t* die_out);

// Maps a device-side wait result onto the caller's status bits.
__device__ __forceinline__ void record_status(uint32_t* status, int rc) {
  if (rc == GSYNC_OK || status == nullptr) return;
  const uint32_t bit = rc == GSYNC_ETIMEDOUT ? GSYNC_STATUS_TIMEOUT
                       : rc == GSYNC_EABORTED ? GSYNC_STATUS_ABORTED
                                               : GSYNC_STATUS_CONFIG;
  gsync::ptx::atom_or_relaxed(status, bit);
}

__device__ __forceinline__ uint32_t lowbias32(uint32_t x) {
  // C. Wellons' "lowbias32" integer hash (hash-prospector, 2018).
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

__device__ __forceinline__ uint32_t rotl32(uint32_t x, int k) { return (x << k) | (x >> (32 - k)); }

__device__ __forceinline__ void spin_cycles(uint32_t cycles) {
  if (cycles == 0) return;
  const long long t0 = clock64();
  while (clock64() - t0 < (long long)cycles) {
  }
}

// Per-workload kernel lookup for gsync_max_coresident_blocks (defined by each workload unit).
int max_blocks_barrier(int kind, int block_threads, int cluster, int* out);
int max_blocks_mutex(int kind, int block_threads, int* out);
int max_blocks_sem(int kind, int block_threads, int* out);

}  // namespace gsync_impl
