// Host-side helpers shared by the decoder translation units: constellation
// constants, the device's SM count and the stream-ordered pool setting.
#pragma once

#include <math.h>
#include <stdint.h>

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

// Keep the scratch of repeated calls cached: the default stream-ordered pool
// of the device otherwise returns its memory to the system at every
// synchronisation and the next call maps it again. Once per device.
inline void keep_pool_cached() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  done[dev] = true;
}

inline int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
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
