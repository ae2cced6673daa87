// Host-side helpers shared by the decoder translation units: constellation
// constants, the device's SM count and the library's stream-ordered pool.
#pragma once

#include <math.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

namespace grand {

// Fixed-point scale of each square constellation, shared by demodulation and
// the likelihood (Def. III.1; d of Eq. 2 with E_b = 1).
struct QamConst {
  float q[7];      // 256/d rounded to float, index m = log2(M)/2 (M = 4 .. 4096)
  float inv_d[7];  // 1/d rounded to float
};

// m = log2(M) / 2 for the supported square constellations, else 0.
inline int m_of(int M) {
  switch (M) {
    case 4: return 1;
    case 16: return 2;
    case 64: return 3;
    case 256: return 4;
    case 1024: return 5;
    case 4096: return 6;
    default: return 0;
  }
}

inline QamConst make_qam_const() {
  QamConst c{};
  for (int m = 1; m <= 6; ++m) {
    const int M = 1 << (2 * m);
    const double d = sqrt(3.0 * m / (double)(M - 1));
    c.q[m] = (float)(256.0 / d);
    c.inv_d[m] = (float)(1.0 / d);
  }
  return c;
}

constexpr int kMaxDevices = 64;

// Stream-ordered scratch comes from a memory pool owned by the library, one
// per device, created at the first allocation on that device and kept for the
// life of the process. Its release threshold is raised so that scratch stays
// cached between calls (a pool otherwise returns its memory to the system at
// every synchronisation and the next call maps it again); the device's
// default pool, which other code in the process may use, keeps its settings.
inline cudaMemPool_t lib_pool(int dev) {
  static std::mutex mu;
  static cudaMemPool_t pools[kMaxDevices] = {};
  if (dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    // Never reuse a block whose free is still pending on another stream by
    // making the allocating stream wait for that stream: concurrent decodes
    // (the serving loop's streams, a long frame's continuation) would then
    // serialise behind one another. The pool grows instead, and keeps it.
    int no = 0;
    cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
    pools[dev] = pool;
  }
  return pools[dev];
}

// Stream-ordered allocation from the library's pool of the current device
// (freed with cudaFreeAsync). Inside a stream capture it becomes a graph
// memory node like cudaMallocAsync.
inline cudaError_t scratch_alloc(void** ptr, size_t bytes, cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaMemPool_t pool = lib_pool(dev);
  if (!pool) return cudaErrorMemoryAllocation;
  return cudaMallocFromPoolAsync(ptr, bytes, pool, st);
}

// SM count of the current device, cached per device index (threads may race
// to fill an entry; they store the same value).
inline int sm_count() {
  static std::atomic<int> cached[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
  if (dev >= 0 && dev < kMaxDevices) {
    const int n = cached[dev].load(std::memory_order_relaxed);
    if (n > 0) return n;
  }
  int n = 0;
  if (dev < 0 || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
  if (dev >= 0 && dev < kMaxDevices && n > 1) cached[dev].store(n, std::memory_order_relaxed);
  return n;
}

// NVTX range over a host scope (enqueue of one stage), for profilers that
// group launches by range (ncu --nvtx, Nsight Systems). Costs nothing when no
// profiler is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace grand
