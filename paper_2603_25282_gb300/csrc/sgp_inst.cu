// sgp_inst.cu -- explicit instantiation of the pass kernels and their
// launchers for one precision (SGP_REAL), one kernel family (SGP_PART:
// 0 = x-lines, 1 = strided lines) and one kernel variant (SGP_VAR, see
// sgp_launch.cuh).  Built once per combination so that the instantiations
// compile in parallel; the observables kernels come with variant 0.
#include "sgp_launch.cuh"

#ifndef SGP_REAL
#error "define SGP_REAL (float or double)"
#endif
#ifndef SGP_PART
#error "define SGP_PART (0 or 1)"
#endif
#ifndef SGP_VAR
#define SGP_VAR 0
#endif

#define SGP_FOR_EACH_VN SGP_FOR_EACH_N

namespace sgp {

namespace {
// Opt in to more than 48 KB of dynamic shared memory once per device.
template <typename K>
cudaError_t prepare(K kern, size_t smem, int* done_dev) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (*done_dev == dev) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) *done_dev = dev;
  return e;
}
}  // namespace

typedef SGP_REAL Real;
constexpr int V = SGP_VAR;

#if SGP_PART == 0

template <>
PassGeom xpass_geom_v<Real, V>(int N) {
  switch (N) {
#define SGP_CASE(NN)                                                        \
  case NN: {                                                                \
    typedef XCfg<Real, NN, variant_elems<Real, NN, V>(), variant_geom<NN, V, SGP_PART>()> Cfg;            \
    return PassGeom{Cfg::THREADS, Cfg::ROWS, Cfg::SMEM};                    \
  }
    SGP_FOR_EACH_VN(SGP_CASE)
#undef SGP_CASE
    default:
      return PassGeom{0, 0, 0};
  }
}

template <int N>
static cudaError_t xpass_prepare_n() {
  constexpr int E = variant_elems<Real, N, V>();
  constexpr int G = variant_geom<N, V, SGP_PART>();
  static int done = -1;
  cudaError_t e = prepare(k_xpass<Real, N, E, G>, XCfg<Real, N, E, G>::SMEM, &done);
#if SGP_VAR == 0
  if (e != cudaSuccess) return e;
  static int done_o = -1;
  e = prepare(k_obs_x<Real, N, E>, XCfg<Real, N, E>::SMEM, &done_o);
#endif
  return e;
}

template <int N>
static cudaError_t xpass_n(const XPassArgs<Real>& a, int members, cudaStream_t s) {
  constexpr int E = variant_elems<Real, N, V>();
  constexpr int G = variant_geom<N, V, SGP_PART>();
  typedef XCfg<Real, N, E, G> Cfg;
  cudaError_t e = xpass_prepare_n<N>();
  if (e != cudaSuccess) return e;
  dim3 grid((a.rows + Cfg::ROWS - 1) / Cfg::ROWS, members);
  k_xpass<Real, N, E, G><<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <>
cudaError_t prepare_xpass_v<Real, V>(int N) {
  switch (N) {
#define SGP_CASE(NN) \
  case NN:           \
    return xpass_prepare_n<NN>();
    SGP_FOR_EACH_VN(SGP_CASE)
#undef SGP_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t launch_xpass_v<Real, V>(int N, const XPassArgs<Real>& a, int members, cudaStream_t s) {
  switch (N) {
#define SGP_CASE(NN) \
  case NN:           \
    return xpass_n<NN>(a, members, s);
    SGP_FOR_EACH_VN(SGP_CASE)
#undef SGP_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

#if SGP_XY_PLANE
// x-pass variant 5 (FP32): the xy-plane pass of 3D grids with NX = NY = N;
// compiled with variant 1, whose x-pass serves the variant's other x-passes
static_assert(sizeof(Real) == 4, "the xy-plane pass is FP32 only");

template <int N>
static cudaError_t xyplane_prepare_n() {
  typedef PlCfg<Real, N, elems_per_thread<Real, N>()> Cfg;
  static int done = -1;
  return prepare(k_xyplane<Real, N, elems_per_thread<Real, N>()>, Cfg::SMEM, &done);
}

template <int N>
static cudaError_t xyplane_n(const XPassArgs<Real>& a, const TwE<Real>* twy, int* err, int planes, int members,
                             cudaStream_t s) {
  constexpr int E = elems_per_thread<Real, N>();
  typedef PlCfg<Real, N, E> Cfg;
  cudaError_t e = xyplane_prepare_n<N>();
  if (e != cudaSuccess) return e;
  dim3 grid(Cfg::CS, planes, members);      // the kernel's cluster is (CS, 1, 1)
  k_xyplane<Real, N, E><<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(a, twy, err);
  return cudaGetLastError();
}

cudaError_t prepare_xyplane(int N) {
  switch (N) {
    case 64: return xyplane_prepare_n<64>();
    case 128: return xyplane_prepare_n<128>();
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_xyplane(int N, const XPassArgs<Real>& a, const TwE<Real>* twy, int* err, int planes,
                           int members, cudaStream_t s) {
  switch (N) {
    case 64: return xyplane_n<64>(a, twy, err, planes, members, s);
    case 128: return xyplane_n<128>(a, twy, err, planes, members, s);
    default: return cudaErrorInvalidValue;
  }
}
#endif

#if SGP_VAR == 2
// x-pass variant 6 (k_xpass_wide): geometry 2, compiled with variant 2
template <int N>
static cudaError_t xpass_wide_prepare_n() {
  constexpr int E = elems_per_thread<Real, N>();
  static int done = -1;
  return prepare(k_xpass_wide<Real, N, E>, XCfg<Real, N, E, 2>::SMEM, &done);
}

template <>
cudaError_t prepare_xpass_wide<Real>(int N) {
  switch (N) {
#define SGP_CASE(NN) \
  case NN:           \
    return xpass_wide_prepare_n<NN>();
    SGP_FOR_EACH_N(SGP_CASE)
#undef SGP_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <int N>
static cudaError_t xpass_wide_n(const XPassArgs<Real>& a, int members, cudaStream_t s) {
  constexpr int E = elems_per_thread<Real, N>();
  typedef XCfg<Real, N, E, 2> Cfg;
  cudaError_t e = xpass_wide_prepare_n<N>();
  if (e != cudaSuccess) return e;
  dim3 grid((a.rows + Cfg::ROWS - 1) / Cfg::ROWS, members);
  k_xpass_wide<Real, N, E><<<grid, kXWideThreads, Cfg::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <>
cudaError_t launch_xpass_wide<Real>(int N, const XPassArgs<Real>& a, int members, cudaStream_t s) {
  switch (N) {
#define SGP_CASE(NN) \
  case NN:           \
    return xpass_wide_n<NN>(a, members, s);
    SGP_FOR_EACH_N(SGP_CASE)
#undef SGP_CASE
    default:
      return cudaErrorInvalidValue;
  }
}
#endif

#if SGP_VAR == 0
template <int N>
static cudaError_t obs_x_n(const ObsXArgs<Real>& a, int members, cudaStream_t s) {
  constexpr int E = elems_per_thread<Real, N>();
  typedef XCfg<Real, N, E> Cfg;
  cudaError_t e = xpass_prepare_n<N>();
  if (e != cudaSuccess) return e;
  dim3 grid((a.rows + Cfg::ROWS - 1) / Cfg::ROWS, members);
  k_obs_x<Real, N, E><<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <>
cudaError_t launch_obs_x<Real>(int N, const ObsXArgs<Real>& a, int members, cudaStream_t s) {
  switch (N) {
#define SGP_CASE(NN) \
  case NN:           \
    return obs_x_n<NN>(a, members, s);
    SGP_FOR_EACH_N(SGP_CASE)
#undef SGP_CASE
    default:
      return cudaErrorInvalidValue;
  }
}
#endif

#else  // SGP_PART == 1

template <>
PassGeom linepass_geom_v<Real, V>(int N) {
  switch (N) {
#define SGP_CASE(NN)                                                        \
  case NN: {                                                                \
    typedef LCfg<Real, NN, variant_elems<Real, NN, V>(), variant_geom<NN, V, SGP_PART>()> Cfg;            \
    return PassGeom{Cfg::THREADS, Cfg::TILE, Cfg::SMEM};                    \
  }
    SGP_FOR_EACH_VN(SGP_CASE)
#undef SGP_CASE
    default:
      return PassGeom{0, 0, 0};
  }
}

template <int N>
static cudaError_t linepass_prepare_n() {
  constexpr int E = variant_elems<Real, N, V>();
  constexpr int G = variant_geom<N, V, SGP_PART>();
  static int done = -1;
  cudaError_t e = prepare(k_linepass<Real, N, E, G>,
                          LCfg<Real, N, E, G>::SMEM + LCfg<Real, N, E, G>::TAB, &done);
#if SGP_VAR == 0
  if (e != cudaSuccess) return e;
  static int done_o = -1;
  e = prepare(k_obs_line<Real, N, E>, LCfg<Real, N, E>::SMEM, &done_o);
#endif
  return e;
}

template <int N>
static cudaError_t linepass_n(const LPassArgs<Real>& a, int planes, int members,
                              cudaStream_t s) {
  constexpr int E = variant_elems<Real, N, V>();
  constexpr int G = variant_geom<N, V, SGP_PART>();
  typedef LCfg<Real, N, E, G> Cfg;
  cudaError_t e = linepass_prepare_n<N>();
  if (e != cudaSuccess) return e;
  dim3 grid((a.nx + Cfg::TILE - 1) / Cfg::TILE, planes, members);
  // the mode-table entries in shared memory when the pass mixes
  const size_t smem = Cfg::SMEM + line_table_bytes<Cfg>(a.mode, a.axis);
  k_linepass<Real, N, E, G><<<grid, Cfg::THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

template <>
cudaError_t prepare_linepass_v<Real, V>(int N) {
  switch (N) {
#define SGP_CASE(NN) \
  case NN:           \
    return linepass_prepare_n<NN>();
    SGP_FOR_EACH_VN(SGP_CASE)
#undef SGP_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t launch_linepass_v<Real, V>(int N, const LPassArgs<Real>& a, int planes, int members,
                                       cudaStream_t s) {
  switch (N) {
#define SGP_CASE(NN) \
  case NN:           \
    return linepass_n<NN>(a, planes, members, s);
    SGP_FOR_EACH_VN(SGP_CASE)
#undef SGP_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

#if SGP_LINE_TMA
// line-pass variant 4 (FP32): geometry 1 with the tile loaded by tensor
// copies; compiled with variant 1, whose geometry it shares
static_assert(sizeof(Real) == 4, "tensor-copy tile loads are FP32 only");

template <int N>
static cudaError_t linepass_tma_prepare_n() {
  constexpr int E = elems_per_thread<Real, N>();
  static int done = -1;
  return prepare(k_linepass_tma<Real, N, E, 1>, LCfg<Real, N, E, 1>::TSMEM + LCfg<Real, N, E, 1>::TAB, &done);
}

template <int N>
static cudaError_t linepass_tma_n(const LPassArgs<Real>& a, const CUtensorMap& map, int planes, int members,
                                  cudaStream_t s) {
  constexpr int E = elems_per_thread<Real, N>();
  typedef LCfg<Real, N, E, 1> Cfg;
  cudaError_t e = linepass_tma_prepare_n<N>();
  if (e != cudaSuccess) return e;
  dim3 grid((a.nx + Cfg::TILE - 1) / Cfg::TILE, planes, members);
  const size_t smem = Cfg::TSMEM + line_table_bytes<Cfg>(a.mode, a.axis);
  k_linepass_tma<Real, N, E, 1><<<grid, Cfg::THREADS, smem, s>>>(a, map);
  return cudaGetLastError();
}

PassGeom linepass_geom_tma(int N) { return linepass_geom_v<Real, 1>(N); }

cudaError_t prepare_linepass_tma(int N) {
  switch (N) {
#define SGP_CASE(NN) \
  case NN:           \
    return linepass_tma_prepare_n<NN>();
    SGP_FOR_EACH_N(SGP_CASE)
#undef SGP_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_linepass_tma(int N, const LPassArgs<Real>& a, const CUtensorMap& map, int planes,
                                int members, cudaStream_t s) {
  switch (N) {
#define SGP_CASE(NN) \
  case NN:           \
    return linepass_tma_n<NN>(a, map, planes, members, s);
    SGP_FOR_EACH_N(SGP_CASE)
#undef SGP_CASE
    default:
      return cudaErrorInvalidValue;
  }
}
#endif

#if SGP_VAR == 0
template <int N>
static cudaError_t obs_line_n(const ObsLArgs<Real>& a, int planes, int members,
                              cudaStream_t s) {
  constexpr int E = elems_per_thread<Real, N>();
  typedef LCfg<Real, N, E> Cfg;
  cudaError_t e = linepass_prepare_n<N>();
  if (e != cudaSuccess) return e;
  dim3 grid((a.nx + Cfg::TILE - 1) / Cfg::TILE, planes, members);
  k_obs_line<Real, N, E><<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <>
cudaError_t launch_obs_line<Real>(int N, const ObsLArgs<Real>& a, int planes, int members,
                                  cudaStream_t s) {
  switch (N) {
#define SGP_CASE(NN) \
  case NN:           \
    return obs_line_n<NN>(a, planes, members, s);
    SGP_FOR_EACH_N(SGP_CASE)
#undef SGP_CASE
    default:
      return cudaErrorInvalidValue;
  }
}
#endif

#endif

}  // namespace sgp
