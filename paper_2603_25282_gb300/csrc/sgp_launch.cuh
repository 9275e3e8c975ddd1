// sgp_launch.cuh -- host-side launchers for the pass kernels, dispatched on
// the line length N (a compile-time parameter of every kernel).
#pragma once
#include <cuda_runtime.h>

#include "sgp_kernels.cuh"

namespace sgp {

// Elements per thread: 8 (FP32) / 4 (FP64) for powers of two, 6 for 3*2^k.
template <typename R, int N>
constexpr int elems_per_thread() {
  return (N % 3 == 0) ? 6 : (sizeof(R) == 4 ? 8 : 4);
}

// Line lengths with compiled kernels.
#define SGP_FOR_EACH_N(X) \
  X(16) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768) X(1024)

inline bool supported_n(int n) {
  switch (n) {
#define SGP_CASE(N) case N:
    SGP_FOR_EACH_N(SGP_CASE)
#undef SGP_CASE
    return true;
    default:
      return false;
  }
}

// Launch geometry of one pass (for accounting and the observables scratch).
struct PassGeom {
  int threads;
  int rows_or_tile;   // rows per CTA (x-pass) or columns per CTA (line pass)
  size_t smem;
};

template <typename R> PassGeom xpass_geom(int N);
template <typename R> PassGeom linepass_geom(int N);

// Set the kernels' shared-memory attributes for line length N on the
// current device (done before any stream capture).
template <typename R> cudaError_t prepare_xpass(int N);
template <typename R> cudaError_t prepare_linepass(int N);

template <typename R>
cudaError_t launch_xpass(int N, const XPassArgs<R>& a, int members, cudaStream_t s);
template <typename R>
cudaError_t launch_linepass(int N, const LPassArgs<R>& a, int planes, int members,
                            cudaStream_t s);
template <typename R>
cudaError_t launch_obs_x(int N, const ObsXArgs<R>& a, int members, cudaStream_t s);
template <typename R>
cudaError_t launch_obs_line(int N, const ObsLArgs<R>& a, int planes, int members,
                            cudaStream_t s);

}  // namespace sgp
