// Topology probes: which SMs share a die, and which die a global-memory line is homed on.
//
// GB300 is two dies, each with its own L2 and HBM stacks; an atomic or a poll on a line homed
// on the other die crosses the die-to-die link.  Section 4's machine abstraction distinguishes
// contentious from noncontentious accesses; on a two-die part the distance to a line's home
// is a third axis, and these probes measure it: the round-trip time of a chain of dependent
// atomics from one SM to one line.
//
// gsync_probe_rtt_by_sm    one line, every SM in turn (one block per SM, taking turns so the
//                          line is never contended).
// gsync_probe_rtt_by_line  one SM, every line of a strided range in turn.
// Every wait is bounded by a 1 s globaltimer deadline; on expiry the probe sets status bit 0.
#include <string.h>

#include <mutex>

#include "common.cuh"

using namespace gsync_impl;
namespace ptx = gsync::ptx;

namespace {

constexpr uint64_t kDeadlineNs = 1000000000ull;
constexpr size_t kOnePerSmSmem = 160 * 1024;  // > half an SM's shared memory: one block per SM
constexpr int kWarm = 4;

// `iters` dependent exchanges on `line` (each returns the value the next one writes), then a
// fence so that the last round trip has completed before the clock is read.  Returns ns.
__device__ __forceinline__ uint64_t time_chain(uint32_t* line, int iters) {
  uint32_t v = 0;
  for (int i = 0; i < kWarm; ++i) v = ptx::atom_exch_relaxed(line, v);
  ptx::fence_acq_rel();
  const uint64_t t0 = ptx::globaltimer();
  for (int i = 0; i < iters; ++i) v = ptx::atom_exch_relaxed(line, v);
  ptx::fence_acq_rel();
  return ptx::globaltimer() - t0;
}

__global__ void rtt_by_sm_kernel(uint32_t* line, uint32_t* turn, int iters, uint64_t* out_ns, uint32_t* status) {
  extern __shared__ uint32_t one_per_sm[];
  if (threadIdx.x != 0) return;
  one_per_sm[0] = 0;
  const uint64_t deadline = ptx::globaltimer() + kDeadlineNs;
  uint32_t polls = 0;
  while (ptx::ld_acquire(turn) != blockIdx.x) {
    if ((++polls & 63u) == 0 && ptx::globaltimer() > deadline) {
      atomicOr(status, 1u);
      return;  // the turn never comes: later blocks time out the same way
    }
  }
  out_ns[ptx::smid()] = time_chain(line, iters);
  ptx::st_release(turn, blockIdx.x + 1u);
}

__global__ void rtt_by_line_kernel(int sm, uint32_t* base, int nlines, int stride_words, int iters,
                                   uint64_t* out_ns) {
  extern __shared__ uint32_t one_per_sm[];
  if (threadIdx.x != 0 || (int)ptx::smid() != sm) return;
  one_per_sm[0] = 0;
  for (int i = 0; i < nlines; ++i) out_ns[i] = time_chain(base + (size_t)i * stride_words, iters);
}

}  // namespace

extern "C" int gsync_probe_rtt_by_sm(void* line, int iters, void* scratch, uint64_t* out_ns, uint32_t* status,
                                     void* stream) {
  int sms = 0;
  if (int rc = device_sms(&sms)) return rc;
  if (!line || !scratch || !out_ns || !status || iters < 1 || iters > (1 << 20) || !aligned(line, 4) ||
      !aligned(scratch, 128))
    return GSYNC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  GSYNC_CUDA(cudaFuncSetAttribute(rtt_by_sm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOnePerSmSmem));
  GSYNC_CUDA(cudaMemsetAsync(scratch, 0, 128, st));
  GSYNC_CUDA(cudaMemsetAsync(out_ns, 0, (size_t)sms * sizeof(uint64_t), st));
  GSYNC_CUDA(cudaMemsetAsync(status, 0, sizeof(uint32_t), st));
  return launch_coresident(rtt_by_sm_kernel, sms, 32, 1, kOnePerSmSmem, st, (uint32_t*)line, (uint32_t*)scratch,
                           iters, out_ns, status);
}

extern "C" int gsync_probe_rtt_by_line(int sm, void* base, int nlines, int stride_bytes, int iters, uint64_t* out_ns,
                                       void* stream) {
  int sms = 0;
  if (int rc = device_sms(&sms)) return rc;
  if (sm < 0 || sm >= sms || !base || !out_ns || nlines < 1 || nlines > (1 << 16) || stride_bytes < 4 ||
      stride_bytes % 4 || iters < 1 || iters > (1 << 16) || !aligned(base, 4))
    return GSYNC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  GSYNC_CUDA(cudaFuncSetAttribute(rtt_by_line_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kOnePerSmSmem));
  GSYNC_CUDA(cudaMemsetAsync(out_ns, 0, (size_t)nlines * sizeof(uint64_t), st));
  return launch_coresident(rtt_by_line_kernel, sms, 32, 1, kOnePerSmSmem, st, sm, (uint32_t*)base, nlines,
                           stride_bytes / 4, iters, out_ns);
}

// ---- the device's SM-to-die map, measured once per device and process ----------------------

namespace {

// Static scratch for the measurement, so that it needs no allocation: line 0 is the probed
// line, line 1 the turn word.
__device__ __align__(128) uint32_t g_topo_lines[64];
__device__ uint64_t g_topo_ns[gsync::kMaxSmIds];
__device__ uint32_t g_topo_status;

constexpr int kTopoIters = 64;
constexpr double kMinGapNs = 60.0;  // a near/far split smaller than this is one die

struct Topology {
  bool valid = false;
  int sms = 0, ndies = 1;
  uint8_t die[gsync::kMaxSmIds] = {};
};
std::mutex g_topo_mu;
Topology g_topo[64];

// Splits values at the midpoint of their range; returns false when the range is too narrow
// to be two populations.
bool split(const double* v, int n, uint8_t* far_out) {
  double lo = v[0], hi = v[0];
  for (int i = 1; i < n; ++i) {
    lo = v[i] < lo ? v[i] : lo;
    hi = v[i] > hi ? v[i] : hi;
  }
  const bool two = hi - lo >= kMinGapNs;
  const double mid = 0.5 * (lo + hi);
  for (int i = 0; i < n; ++i) far_out[i] = two && v[i] > mid ? 1 : 0;
  return two;
}

int measure(cudaStream_t st, Topology* t) {
  int sms = 0;
  if (int rc = device_sms(&sms)) return rc;
  if (sms > (int)gsync::kMaxSmIds) return GSYNC_EINVAL;
  void *lines = nullptr, *ns = nullptr, *status = nullptr;
  GSYNC_CUDA(cudaGetSymbolAddress(&lines, g_topo_lines));
  GSYNC_CUDA(cudaGetSymbolAddress(&ns, g_topo_ns));
  GSYNC_CUDA(cudaGetSymbolAddress(&status, g_topo_status));
  if (int rc = gsync_probe_rtt_by_sm(lines, kTopoIters, (uint32_t*)lines + 32, (uint64_t*)ns, (uint32_t*)status, st))
    return rc;
  uint64_t h_ns[gsync::kMaxSmIds];
  uint32_t h_status = 0;
  GSYNC_CUDA(cudaMemcpyAsync(h_ns, ns, sizeof(uint64_t) * sms, cudaMemcpyDeviceToHost, st));
  GSYNC_CUDA(cudaMemcpyAsync(&h_status, status, 4, cudaMemcpyDeviceToHost, st));
  GSYNC_CUDA(cudaStreamSynchronize(st));
  if (h_status) return GSYNC_ETIMEDOUT;
  double v[gsync::kMaxSmIds];
  for (int i = 0; i < sms; ++i) v[i] = (double)h_ns[i] / kTopoIters;
  t->sms = sms;
  t->ndies = split(v, sms, t->die) ? 2 : 1;
  t->valid = true;
  return GSYNC_OK;
}

}  // namespace

namespace gsync_impl {

int device_topology(cudaStream_t st, uint8_t* die_of_sm, int* ndies, int* sms) {
  int dev = 0;
  GSYNC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return GSYNC_EINVAL;
  std::lock_guard<std::mutex> g(g_topo_mu);
  Topology& t = g_topo[dev];
  if (!t.valid)
    if (int rc = measure(st, &t)) return rc;
  memcpy(die_of_sm, t.die, gsync::kMaxSmIds);
  *ndies = t.ndies;
  *sms = t.sms;
  return GSYNC_OK;
}

int line_homes(const void* base, int nlines, size_t stride, const uint8_t* die_of_sm, int sms, cudaStream_t st,
               uint8_t* die_out) {
  int sm0 = -1;
  for (int s = 0; s < sms && sm0 < 0; ++s)
    if (die_of_sm[s] == 0) sm0 = s;
  if (sm0 < 0 || nlines < 1 || nlines > (int)gsync::kMaxSmIds) return GSYNC_EINVAL;
  std::lock_guard<std::mutex> g(g_topo_mu);  // the static scratch is shared with the SM probe
  void* ns = nullptr;
  GSYNC_CUDA(cudaGetSymbolAddress(&ns, g_topo_ns));
  if (int rc = gsync_probe_rtt_by_line(sm0, (void*)base, nlines, (int)stride, kTopoIters / 4, (uint64_t*)ns, st))
    return rc;
  uint64_t h_ns[gsync::kMaxSmIds];
  GSYNC_CUDA(cudaMemcpyAsync(h_ns, ns, sizeof(uint64_t) * nlines, cudaMemcpyDeviceToHost, st));
  GSYNC_CUDA(cudaStreamSynchronize(st));
  double v[gsync::kMaxSmIds];
  for (int i = 0; i < nlines; ++i) v[i] = (double)h_ns[i] / (kTopoIters / 4);
  // Near to an SM of die 0 means homed on die 0.
  if (nlines == 1) die_out[0] = 0;
  else split(v, nlines, die_out);
  return GSYNC_OK;
}

}  // namespace gsync_impl

extern "C" int gsync_device_topology(uint8_t* die_of_sm, int* ndies_out, void* stream) {
  if (!die_of_sm || !ndies_out) return GSYNC_EINVAL;
  uint8_t die[gsync::kMaxSmIds];
  int nd = 0, sms = 0;
  if (int rc = device_topology((cudaStream_t)stream, die, &nd, &sms)) return rc;
  memcpy(die_of_sm, die, (size_t)sms);
  *ndies_out = nd;
  return GSYNC_OK;
}
