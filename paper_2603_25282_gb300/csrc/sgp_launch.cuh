// sgp_launch.cuh -- host-side launchers for the pass kernels, dispatched on
// the line length N (a compile-time parameter of every kernel) and on the
// kernel variant V chosen by the autotuner.
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
#define SGP_FOR_EACH_N_POW2(X) X(16) X(32) X(64) X(128) X(256) X(512) X(1024)

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

// Kernel variants of a pass (the tile and radix schedules the autotuner
// chooses from):
//   0  default geometry (x-pass: about 256 threads per CTA; line pass: up
//      to 512 threads, TILE >= 4 FP32 / 2 FP64 columns) and radix plan
//   1  CTAs of about half the threads (line pass: TILE down to 1)
//   2  CTAs of about a quarter of the threads
//   3  FP32 only.  N a power of two: radix-4 plan (4 elements per thread
//      instead of 8: more stages, half the registers per line element).
//      N = 3*2^k: 12 elements per thread, radix 6 then 4s (96 = 6*4*4 in
//      three stages instead of 6*2*2*2*2 in five), in CTAs of 128 threads
//      (x-pass geometry 1, line-pass geometry 2: a thread holds 120
//      registers of field data)
//   4  FP32 only.  Line pass: geometry 1 with the tile loaded by tensor
//      copies (TMA) into shared memory; x-pass: the same as variant 1
//   5  FP32, x-pass of 3D grids with NX = NY = 64 or 128 only: the steps'
//      x-passes become xy-plane passes (k_xyplane: one thread-block cluster
//      per z plane, the y transforms done there), so a step drops its
//      y-line passes; x-passes outside the steps are those of variant 1
//   6  x-pass: the rows of geometry 2 with the nonlinear flow shared by the
//      256 threads of the CTA (k_xpass_wide; for small grids, whose CTAs
//      are few); line pass: the same as variant 2
constexpr int kVariants = 7;

template <typename R, int N, int V>
constexpr int variant_elems() {
  return V == 3 ? (N % 3 == 0 ? 12 : 4) : elems_per_thread<R, N>();
}
// geometry of variant V for the x-pass (PART 0) and the line pass (PART 1)
template <int N, int V, int PART>
constexpr int variant_geom() {
  return V == 3 ? (N % 3 == 0 ? 1 + PART : 0) : (V == 4 || V == 5) ? 1 : V == 6 ? 2 : V;
}

// Does variant V exist for line length N (prec_bytes 4 or 8)?
inline bool variant_exists(int prec_bytes, int N, int V) {
  if (!supported_n(N) || V < 0 || V >= kVariants) return false;
  if (V == 3 || V == 4) return prec_bytes == 4;
  return V != 5;       // variant 5 depends on the whole grid (plane_ok in the host runtime)
}
// Elements per thread of variant V (the twiddle table layout depends on it).
inline int variant_elems_rt(int prec_bytes, int N, int V) {
  if (V == 3) return N % 3 == 0 ? 12 : 4;
  return (N % 3 == 0) ? 6 : (prec_bytes == 4 ? 8 : 4);
}

// Launch geometry of one pass (for accounting and the observables scratch).
struct PassGeom {
  int threads;
  int rows_or_tile;   // rows per CTA (x-pass) or columns per CTA (line pass)
  size_t smem;
};

// Per-variant entry points (explicitly instantiated in sgp_inst.cu).
template <typename R, int V> PassGeom xpass_geom_v(int N);
template <typename R, int V> PassGeom linepass_geom_v(int N);
template <typename R, int V> cudaError_t prepare_xpass_v(int N);
template <typename R, int V> cudaError_t prepare_linepass_v(int N);
template <typename R, int V>
cudaError_t launch_xpass_v(int N, const XPassArgs<R>& a, int members, cudaStream_t s);
template <typename R, int V>
cudaError_t launch_linepass_v(int N, const LPassArgs<R>& a, int planes, int members,
                              cudaStream_t s);
// Variant 4 of the line pass (tile loads by tensor copies over `map`).
cudaError_t launch_linepass_tma(int N, const LPassArgs<float>& a, const CUtensorMap& map, int planes,
                                int members, cudaStream_t s);
cudaError_t prepare_linepass_tma(int N);
PassGeom linepass_geom_tma(int N);
// Variant 5 of the x-pass: the xy-plane pass over `planes` z planes of
// `members` members (N = NX = NY; twy: the y twiddles; err: the word a
// bounded wait for a hand-over sets when it gives up).
cudaError_t launch_xyplane(int N, const XPassArgs<float>& a, const TwE<float>* twy, int* err, int planes,
                           int members, cudaStream_t s);
cudaError_t prepare_xyplane(int N);
// Variant 6 of the x-pass (k_xpass_wide).
template <typename R>
cudaError_t launch_xpass_wide(int N, const XPassArgs<R>& a, int members, cudaStream_t s);
template <typename R>
cudaError_t prepare_xpass_wide(int N);

// x-pass variants 4 and 5 are variant 1 (variant 5's plane pass has its own
// entry point) and variant 6 has the geometry of variant 2 (its own kernel,
// dispatched first); the line pass has its own variant 4 and takes variant
// 2 for 6
#define SGP_VARIANT_SWITCH_X(V, CALL, FAIL)                  \
  switch (V) {                                               \
    case 0: return CALL(0);                                  \
    case 1: return CALL(1);                                  \
    case 2: return CALL(2);                                  \
    case 3:                                                  \
      if constexpr (sizeof(R) == 4) return CALL(3);          \
      return FAIL;                                           \
    case 4:                                                  \
    case 5:                                                  \
      if constexpr (sizeof(R) == 4) return CALL(1);          \
      return FAIL;                                           \
    case 6: return CALL(2);                                  \
    default: return FAIL;                                    \
  }
#define SGP_VARIANT_SWITCH(V, CALL, FAIL)                    \
  switch (V) {                                               \
    case 0: return CALL(0);                                  \
    case 1: return CALL(1);                                  \
    case 2: return CALL(2);                                  \
    case 3:                                                  \
      if constexpr (sizeof(R) == 4) return CALL(3);          \
      return FAIL;                                           \
    case 6: return CALL(2);                                  \
    default: return FAIL;                                    \
  }

template <typename R>
inline PassGeom xpass_geom(int N, int V = 0) {
#define SGP_C(v) xpass_geom_v<R, v>(N)
  SGP_VARIANT_SWITCH_X(V, SGP_C, (PassGeom{0, 0, 0}))
#undef SGP_C
}
template <typename R>
inline PassGeom linepass_geom(int N, int V = 0) {
  if constexpr (sizeof(R) == 4)
    if (V == 4) return linepass_geom_tma(N);
#define SGP_C(v) linepass_geom_v<R, v>(N)
  SGP_VARIANT_SWITCH(V, SGP_C, (PassGeom{0, 0, 0}))
#undef SGP_C
}
// Set the kernels' shared-memory attributes for line length N on the
// current device (done before any stream capture).
template <typename R>
inline cudaError_t prepare_xpass(int N, int V = 0) {
  if (V == 6) {
    const cudaError_t e = prepare_xpass_wide<R>(N);
    if (e != cudaSuccess) return e;
  }
#define SGP_C(v) prepare_xpass_v<R, v>(N)
  SGP_VARIANT_SWITCH_X(V, SGP_C, cudaErrorInvalidValue)
#undef SGP_C
}
template <typename R>
inline cudaError_t prepare_linepass(int N, int V = 0) {
  if constexpr (sizeof(R) == 4)
    if (V == 4) return prepare_linepass_tma(N);
#define SGP_C(v) prepare_linepass_v<R, v>(N)
  SGP_VARIANT_SWITCH(V, SGP_C, cudaErrorInvalidValue)
#undef SGP_C
}
template <typename R>
inline cudaError_t launch_xpass(int N, int V, const XPassArgs<R>& a, int members, cudaStream_t s) {
  if (V == 6) return launch_xpass_wide<R>(N, a, members, s);
#define SGP_C(v) launch_xpass_v<R, v>(N, a, members, s)
  SGP_VARIANT_SWITCH_X(V, SGP_C, cudaErrorInvalidValue)
#undef SGP_C
}
// Variants 0-3 of the line pass (variant 4 goes through launch_linepass_tma).
template <typename R>
inline cudaError_t launch_linepass(int N, int V, const LPassArgs<R>& a, int planes, int members,
                                   cudaStream_t s) {
#define SGP_C(v) launch_linepass_v<R, v>(N, a, planes, members, s)
  SGP_VARIANT_SWITCH(V, SGP_C, cudaErrorInvalidValue)
#undef SGP_C
}
#undef SGP_VARIANT_SWITCH
#undef SGP_VARIANT_SWITCH_X

// Observables kernels (default geometry only).
template <typename R>
cudaError_t launch_obs_x(int N, const ObsXArgs<R>& a, int members, cudaStream_t s);
template <typename R>
cudaError_t launch_obs_line(int N, const ObsLArgs<R>& a, int planes, int members,
                            cudaStream_t s);

}  // namespace sgp
