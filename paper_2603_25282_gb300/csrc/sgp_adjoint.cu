// sgp_adjoint.cu -- the passes of a gradient for one precision (SGP_REAL):
// the adjoint x-pass that carries g back through a nonlinear substep (with
// the inverse and forward x-transforms of the neighbouring linear substeps
// fused in), the line pass with the hooks (the sweep adds the per-mode
// parameter terms of a linear substep after its forward transform; the
// state VJP of the linear flow is the linear flow over -d, so the rest is
// the forward line pass), and the x-pass of the recomputation that keeps a
// copy of every nonlinear substep's output.  Formulas: sgp_adjoint.cuh.
#include "sgp_adjoint.cuh"
#include "sgp_launch.cuh"

#ifndef SGP_REAL
#error "define SGP_REAL (float or double)"
#endif

namespace sgp {
namespace {

typedef SGP_REAL Real;

// The adjoint x-pass for block (bx, member): the CTA's rows are bx * ROWS ..
// bx * ROWS + ROWS - 1 of x-pass geometry 2 (rows of about 64 threads side
// by side).  The nonlinear adjoint is the long part (several hundred
// instructions per point, FP64 coordinates) and the grids of a gradient run
// are small, so the CTA has kXAdjThreads threads: the first FT = ROWS * T
// transform the rows (synchronised by a named barrier of their own), then
// all of them share the rows' points, staged in the exchange buffers;
// Phi_out comes from global memory point by point.
constexpr int kXAdjThreads = 256;
constexpr int kXAdjGeom = 2;          // x-pass geometry of the rows

template <typename R, int N, int E>
__global__ void __launch_bounds__(kXAdjThreads, 2) k_xadj(XAdjArgs<R> a) {
  typedef cplx<R> C;
  typedef XCfg<R, N, E, kXAdjGeom> Cfg;
  constexpr int T = Cfg::T, FT = Cfg::THREADS, ROWS = Cfg::ROWS;
  static_assert(kXAdjThreads % FT == 0 && FT % 32 == 0, "adjoint x-pass geometry");
  constexpr int GT = FT == kXAdjThreads ? 0 : FT;       // the transforms' barrier
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TwE<R>* tw = reinterpret_cast<TwE<R>*>(smem_raw);
  C* xb = reinterpret_cast<C*>(tw + N);
  __shared__ double s_rot[3];
  __shared__ double red[kXAdjThreads / 32 * NLA_NT];
  const int member = blockIdx.y;
  const int tid = threadIdx.x;
  const int g = tid / T;
  const int i = tid - g * T;
  for (int k = tid; k < N; k += kXAdjThreads) tw[k] = a.tw[k];
  if (tid == 0) {
    const double t = *a.t_base + a.t_off;
    sincos(a.mp[member].omega * t, &s_rot[1], &s_rot[0]);
    s_rot[2] = t;
  }
  const int bstride = ROWS * Cfg::LP;
  const size_t mo = (size_t)member * 5 * a.ntot;
  const int row = blockIdx.x * ROWS + g;
  const bool valid = tid < FT && row < a.rows;
  C* base = a.g + mo + (size_t)(valid ? row : 0) * N + i;
  C* b0 = xb + g * Cfg::LP;
  C v[5][E];
  if (tid < FT) {
#pragma unroll
    for (int c = 0; c < 5; ++c)
#pragma unroll
      for (int e = 0; e < E; ++e) v[c][e] = valid ? base[(size_t)c * a.ntot + T * e] : mkc((R)0, (R)0);
  }
  __syncthreads();                    // twiddles and s_rot
  if (tid < FT) {
    if (a.mode & XP_INV) fft_lines<R, N, E, +1, 5, Cfg::NB, GT>(v, i, tw, b0, bstride, 1);
    group_sync<GT>(1);                // the exchanges' reads of the buffers are done
#pragma unroll
    for (int c = 0; c < 5; ++c)
#pragma unroll
      for (int e = 0; e < E; ++e) b0[c * bstride + i + T * e] = v[c][e];
  }
  __syncthreads();                    // the rows are staged
  double acc[NLA_NT] = {0.0, 0.0, 0.0, 0.0};
  {
    const MemberPrm& P = a.mp[member];
    NLAdjPrm<R> q;
    q.d = (R)a.delta;
    q.c0p = (R)(P.c0 + P.c2 / 5.0);
    q.c1 = (R)P.c1;
    q.c2 = (R)P.c2;
    q.tdgg = (R)(s_rot[2] * 2.0 * (P.gx2h - P.gy2h));
    const R co = (R)s_rot[0], si = (R)s_rot[1];
    const R gx2h = (R)P.gx2h, gy2h = (R)P.gy2h, gz2h = (R)P.gz2h;
#pragma unroll 1
    for (int p = tid; p < ROWS * N; p += kXAdjThreads) {
      const int r = p / N, j = p - r * N;
      const int rw = blockIdx.x * ROWS + r;
      if (rw >= a.rows) break;          // p only grows
      const int iy = rw % a.ny, iz = rw / a.ny;
      const R x = a.x0 + (R)j * a.hx, y = a.y0 + (R)iy * a.hy, z = a.z0 + (R)iz * a.hz;
      const R xr = co * x + si * y, yr = co * y - si * x;
      const R V = gx2h * xr * xr + gy2h * yr * yr + gz2h * z * z;
      const C* pr = a.phi + mo + (size_t)rw * N + j;
      C* sp = xb + r * Cfg::LP + j;
      C psi[5], gp[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        psi[c] = pr[(size_t)c * a.ntot];
        gp[c] = sp[c * bstride];
      }
      nl_adjoint_point<R>(psi, gp, V, xr * yr, q, acc);
#pragma unroll
      for (int c = 0; c < 5; ++c) sp[c * bstride] = gp[c];
    }
  }
  __syncthreads();                    // every point is done
  if (tid < FT) {
#pragma unroll
    for (int c = 0; c < 5; ++c)
#pragma unroll
      for (int e = 0; e < E; ++e) v[c][e] = b0[c * bstride + i + T * e];
    if (a.mode & XP_FWD) fft_lines<R, N, E, -1, 5, Cfg::NB, GT>(v, i, tw, b0, bstride, 1);
    if (valid) {
#pragma unroll
      for (int c = 0; c < 5; ++c)
#pragma unroll
        for (int e = 0; e < E; ++e) base[(size_t)c * a.ntot + T * e] = v[c][e];
    }
  }
  double out[NLA_NT];
  block_sums<NLA_NT>(acc, out, red);
  if (tid < NLA_NT) {
    const int slot[NLA_NT] = {GP_OMEGA, GP_C0, GP_C1, GP_C2};
    a.partials[((size_t)member * a.prows + blockIdx.x) * GP_N + slot[tid]] += out[tid];
  }
}

// the x-pass of the recomputation: geometry 2, with the copy after the flow
constexpr int kTapGeom = 2;

template <typename R, int N, int E>
__global__ void __launch_bounds__(XCfg<R, N, E, kTapGeom>::THREADS, XCfg<R, N, E, kTapGeom>::MINB)
k_xpass_tap(XPassArgs<R> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  xpass_body<R, N, E, kTapGeom, false, true>(a, blockIdx.x, blockIdx.y, smem_raw);
}

// the line pass of a gradient: geometry 2 of the line pass (more, smaller CTAs)
constexpr int kAdjLineGeom = 2;

template <typename R, int N, int E, int G>
__global__ void __launch_bounds__(LCfg<R, N, E, G>::THREADS, LCfg<R, N, E, G>::MINB)
k_linepass_adj(LPassArgs<R> a, AdjHook<R> h) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  linepass_body<R, N, E, G, false, false, AdjHook<R>>(a, blockIdx.x, blockIdx.y, blockIdx.z, smem_raw, nullptr, h);
}

// Opt in to more than 48 KB of dynamic shared memory once per device.
template <typename K>
cudaError_t opt_in(K kern, size_t smem, int* done_dev) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (*done_dev == dev) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) *done_dev = dev;
  return e;
}

template <int N>
cudaError_t xadj_n(const XAdjArgs<Real>& a, int members, cudaStream_t s) {
  constexpr int E = elems_per_thread<Real, N>();
  typedef XCfg<Real, N, E, kXAdjGeom> Cfg;
  static int done = -1;
  const cudaError_t e = opt_in(k_xadj<Real, N, E>, Cfg::SMEM, &done);
  if (e != cudaSuccess) return e;
  dim3 grid((a.rows + Cfg::ROWS - 1) / Cfg::ROWS, members);
  k_xadj<Real, N, E><<<grid, kXAdjThreads, Cfg::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <int N>
cudaError_t xpass_tap_n(const XPassArgs<Real>& a, int members, cudaStream_t s) {
  constexpr int E = elems_per_thread<Real, N>();
  typedef XCfg<Real, N, E, kTapGeom> Cfg;
  static int done = -1;
  const cudaError_t e = opt_in(k_xpass_tap<Real, N, E>, Cfg::SMEM, &done);
  if (e != cudaSuccess) return e;
  dim3 grid((a.rows + Cfg::ROWS - 1) / Cfg::ROWS, members);
  k_xpass_tap<Real, N, E><<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <int N>
cudaError_t linepass_adj_n(const LPassArgs<Real>& a, const AdjHook<Real>& h, int planes, int members,
                           cudaStream_t s) {
  constexpr int E = elems_per_thread<Real, N>();
  constexpr int G = kAdjLineGeom;
  typedef LCfg<Real, N, E, G> Cfg;
  // the hook's staging sits behind the largest mode-table region
  constexpr size_t HB = AdjHook<Real>::smem_bytes<Real, N, Cfg::TILE>();
  static_assert(Cfg::SMEM + Cfg::TAB + HB <= 227 * 1024, "line pass of a gradient: shared memory");
  static int done = -1;
  const cudaError_t e = opt_in(k_linepass_adj<Real, N, E, G>, Cfg::SMEM + Cfg::TAB + HB, &done);
  if (e != cudaSuccess) return e;
  dim3 grid((a.nx + Cfg::TILE - 1) / Cfg::TILE, planes, members);
  const size_t smem = Cfg::SMEM + Cfg::TAB + (h.spec ? HB : 0);
  k_linepass_adj<Real, N, E, G><<<grid, Cfg::THREADS, smem, s>>>(a, h);
  return cudaGetLastError();
}

}  // namespace

template <>
cudaError_t launch_xadj<Real>(int N, const XAdjArgs<Real>& a, int members, cudaStream_t s) {
  switch (N) {
#define SGP_CASE(NN) \
  case NN:           \
    return xadj_n<NN>(a, members, s);
    SGP_FOR_EACH_N(SGP_CASE)
#undef SGP_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t launch_xpass_tap<Real>(int N, const XPassArgs<Real>& a, int members, cudaStream_t s) {
  switch (N) {
#define SGP_CASE(NN) \
  case NN:           \
    return xpass_tap_n<NN>(a, members, s);
    SGP_FOR_EACH_N(SGP_CASE)
#undef SGP_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t launch_linepass_adj<Real>(int N, const LPassArgs<Real>& a, const AdjHook<Real>& h, int planes,
                                      int members, cudaStream_t s) {
  switch (N) {
#define SGP_CASE(NN) \
  case NN:           \
    return linepass_adj_n<NN>(a, h, planes, members, s);
    SGP_FOR_EACH_N(SGP_CASE)
#undef SGP_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <>
int xadj_ctas<Real>(int N, int rows) {
  switch (N) {
#define SGP_CASE(NN)                                               \
  case NN: {                                                       \
    typedef XCfg<Real, NN, elems_per_thread<Real, NN>(), kXAdjGeom> Cfg;  \
    return (rows + Cfg::ROWS - 1) / Cfg::ROWS;                     \
  }
    SGP_FOR_EACH_N(SGP_CASE)
#undef SGP_CASE
    default:
      return 0;
  }
}

template <>
int linepass_adj_tiles<Real>(int N, int nx) {
  switch (N) {
#define SGP_CASE(NN)                                                          \
  case NN: {                                                                  \
    typedef LCfg<Real, NN, elems_per_thread<Real, NN>(), kAdjLineGeom> Cfg;   \
    return (nx + Cfg::TILE - 1) / Cfg::TILE;                                  \
  }
    SGP_FOR_EACH_N(SGP_CASE)
#undef SGP_CASE
    default:
      return 0;
  }
}

#if SGP_REDUCE_PARAMS
namespace {
__global__ void k_reduce_params(const double* part, int nrows, int members, double* dp) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= members * GP_N) return;
  const int m = id / GP_N, k = id - m * GP_N;
  const double* p = part + (size_t)m * nrows * GP_N + k;
  double s = 0.0;
  for (int b = 0; b < nrows; ++b) s += p[(size_t)b * GP_N];
  dp[id] = s;
}
}  // namespace

cudaError_t launch_reduce_params(const double* part, int nrows, int members, double* dp, cudaStream_t s) {
  const int n = members * GP_N;
  k_reduce_params<<<(n + 127) / 128, 128, 0, s>>>(part, nrows, members, dp);
  return cudaGetLastError();
}
#endif

}  // namespace sgp
