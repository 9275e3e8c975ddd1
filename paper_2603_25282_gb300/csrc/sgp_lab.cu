// sgp_lab.cu -- lab-frame output: psi_l(x, t) = exp(i l Omega t) phi_l(R(t)^T x, t),
// the inverse of the mapping (mapping) evaluated on the grid as in Eq.
// (RSDA2).  The rotation by theta = Omega t is split into exact quarter
// turns (index permutations of a square periodic grid, since -x_j =
// x_{(N-j) mod N}) and a remainder |theta_r| <= pi/4 done by three shears
// exp(a y d_x) exp(b x d_y) exp(a y d_x), a = -tan(theta_r/2), b =
// sin(theta_r).  A shear translates every line by a distance proportional
// to the other coordinate: a forward line FFT, the phase exp(i nu_p c) per
// mode (angle in FP64), the inverse FFT.
#include "sgp_lab.cuh"

namespace sgp {
namespace {

// exp(i nu c) / N for the mode at FFT index p of a length-N line, with
// nu = kfac * p_signed (kfac = pi / L) and the shift c; FP64 angle
template <typename R>
__device__ __forceinline__ cplx<R> shear_phase(int p, int N, double kfac, double c) {
  const int ps = p < N / 2 ? p : p - N;
  double s, co;
  sincos(kfac * (double)ps * c, &s, &co);
  const double inv = 1.0 / (double)N;
  return mkc((R)(co * inv), (R)(s * inv));
}

// x-lines (rows of all five components), rows side by side as the x-pass
template <typename R, int N, int E>
__global__ void __launch_bounds__(XCfg<R, N, E>::THREADS)
k_shear_rows(ShearArgs<R> a) {
  typedef cplx<R> C;
  typedef XCfg<R, N, E> Cfg;
  constexpr int T = Cfg::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TwE<R>* tw = reinterpret_cast<TwE<R>*>(smem_raw);
  C* xb = reinterpret_cast<C*>(tw + N);
  const int g = threadIdx.x / T;
  const int i = threadIdx.x - g * T;
  for (int k = threadIdx.x; k < N; k += Cfg::THREADS) tw[k] = a.tw[k];
  const int row = blockIdx.x * Cfg::ROWS + g;
  const bool valid = row < a.rows;
  C* base = a.field + (size_t)(valid ? row : 0) * N + i;
  C v[5][E];
#pragma unroll
  for (int c = 0; c < 5; ++c)
#pragma unroll
    for (int e = 0; e < E; ++e)
      v[c][e] = valid ? base[(size_t)c * a.ntot + T * e] : mkc((R)0, (R)0);
  C* b0 = xb + g * Cfg::LP;
  const int bstride = Cfg::ROWS * Cfg::LP;
  fft_lines<R, N, E, -1, 5, Cfg::NB>(v, i, tw, b0, bstride);
  const double other = a.o0 + (double)((valid ? row : 0) % a.ny) * a.h0;
  const double shift = a.coef * other;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const C ph = shear_phase<R>(i + T * e, N, a.kfac, shift);
#pragma unroll
    for (int c = 0; c < 5; ++c) v[c][e] = cmul(v[c][e], ph);
  }
  fft_lines<R, N, E, +1, 5, Cfg::NB>(v, i, tw, b0, bstride);
  if (a.lab_phase) {
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      double s, co;
      sincos((double)(2 - c) * a.theta, &s, &co);
      const C ph = mkc((R)co, (R)s);
#pragma unroll
      for (int e = 0; e < E; ++e) v[c][e] = cmul(v[c][e], ph);
    }
  }
  if (valid) {
#pragma unroll
    for (int c = 0; c < 5; ++c)
#pragma unroll
      for (int e = 0; e < E; ++e) base[(size_t)c * a.ntot + T * e] = v[c][e];
  }
}

// y-lines over a tile of consecutive x columns, as the line pass
template <typename R, int N, int E>
__global__ void __launch_bounds__(LCfg<R, N, E>::THREADS)
k_shear_cols(ShearArgs<R> a) {
  typedef cplx<R> C;
  typedef LCfg<R, N, E> Cfg;
  constexpr int T = Cfg::T;
  constexpr int TILE = Cfg::TILE;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TwE<R>* tw = reinterpret_cast<TwE<R>*>(smem_raw);
  C* xb = reinterpret_cast<C*>(tw + N);
  const int col = threadIdx.x % TILE;
  const int i = threadIdx.x / TILE;
  for (int k = threadIdx.x; k < N; k += Cfg::THREADS) tw[k] = a.tw[k];
  const int xcol = blockIdx.x * TILE + col;
  const bool valid = xcol < a.rows;
  C* base = a.field + (size_t)blockIdx.y * a.plane_stride + (valid ? xcol : 0) +
            (size_t)i * a.line_stride;
  const size_t step = (size_t)T * a.line_stride;
  C v[5][E];
#pragma unroll
  for (int c = 0; c < 5; ++c)
#pragma unroll
    for (int e = 0; e < E; ++e)
      v[c][e] = valid ? base[(size_t)c * a.ntot + e * step] : mkc((R)0, (R)0);
  C* b0 = xb + col * Cfg::LP;
  const int bstride = TILE * Cfg::LP;
  fft_lines<R, N, E, -1, 5, Cfg::NB>(v, i, tw, b0, bstride);
  const double shift = a.coef * (a.o0 + (double)(valid ? xcol : 0) * a.h0);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const C ph = shear_phase<R>(i + T * e, N, a.kfac, shift);
#pragma unroll
    for (int c = 0; c < 5; ++c) v[c][e] = cmul(v[c][e], ph);
  }
  fft_lines<R, N, E, +1, 5, Cfg::NB>(v, i, tw, b0, bstride);
  if (valid) {
#pragma unroll
    for (int c = 0; c < 5; ++c)
#pragma unroll
      for (int e = 0; e < E; ++e) base[(size_t)c * a.ntot + e * step] = v[c][e];
  }
}

// out(x) = in(R_{k pi/2} x) on an n x n grid (per z plane, five components):
// k = 1: out[iy][ix] = in[ix][(n - iy) % n]; k = 2: in[(n - iy) % n][(n - ix) % n];
// k = 3: in[(n - ix) % n][iy]
template <typename R>
__global__ void k_quarter(const cplx<R>* in, cplx<R>* out, int n, long long ntot, int k) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= ntot) return;
  const long long nn = (long long)n * n;
  const long long z = id / nn;
  const int r = (int)(id - z * nn);
  const int iy = r / n, ix = r - iy * n;
  int sy, sx;
  if (k == 1) {
    sy = ix;
    sx = (n - iy) % n;
  } else if (k == 2) {
    sy = (n - iy) % n;
    sx = (n - ix) % n;
  } else {
    sy = (n - ix) % n;
    sx = iy;
  }
  const long long src = z * nn + (long long)sy * n + sx;
#pragma unroll
  for (int c = 0; c < 5; ++c) out[(size_t)c * ntot + id] = in[(size_t)c * ntot + src];
}

template <typename K>
cudaError_t prepare(K kern, size_t smem) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename R, int N>
cudaError_t rows_n(const ShearArgs<R>& a, cudaStream_t s) {
  constexpr int E = elems_per_thread<R, N>();
  typedef XCfg<R, N, E> Cfg;
  cudaError_t e = prepare(k_shear_rows<R, N, E>, Cfg::SMEM);
  if (e != cudaSuccess) return e;
  k_shear_rows<R, N, E><<<(a.rows + Cfg::ROWS - 1) / Cfg::ROWS, Cfg::THREADS, Cfg::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <typename R, int N>
cudaError_t cols_n(const ShearArgs<R>& a, int planes, cudaStream_t s) {
  constexpr int E = elems_per_thread<R, N>();
  typedef LCfg<R, N, E> Cfg;
  cudaError_t e = prepare(k_shear_cols<R, N, E>, Cfg::SMEM);
  if (e != cudaSuccess) return e;
  dim3 grid((a.rows + Cfg::TILE - 1) / Cfg::TILE, planes);
  k_shear_cols<R, N, E><<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

template <typename R>
cudaError_t launch_shear_rows(int N, const ShearArgs<R>& a, cudaStream_t s) {
  switch (N) {
#define SGP_CASE(NN) \
  case NN:           \
    return rows_n<R, NN>(a, s);
    SGP_FOR_EACH_N(SGP_CASE)
#undef SGP_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <typename R>
cudaError_t launch_shear_cols(int N, const ShearArgs<R>& a, int planes, cudaStream_t s) {
  switch (N) {
#define SGP_CASE(NN) \
  case NN:           \
    return cols_n<R, NN>(a, planes, s);
    SGP_FOR_EACH_N(SGP_CASE)
#undef SGP_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <typename R>
cudaError_t launch_quarter(const cplx<R>* in, cplx<R>* out, int n, long long ntot, int k,
                           cudaStream_t s) {
  k_quarter<R><<<(unsigned)((ntot + 255) / 256), 256, 0, s>>>(in, out, n, ntot, k);
  return cudaGetLastError();
}

template cudaError_t launch_shear_rows<float>(int, const ShearArgs<float>&, cudaStream_t);
template cudaError_t launch_shear_rows<double>(int, const ShearArgs<double>&, cudaStream_t);
template cudaError_t launch_shear_cols<float>(int, const ShearArgs<float>&, int, cudaStream_t);
template cudaError_t launch_shear_cols<double>(int, const ShearArgs<double>&, int, cudaStream_t);
template cudaError_t launch_quarter<float>(const cplx<float>*, cplx<float>*, int, long long, int,
                                           cudaStream_t);
template cudaError_t launch_quarter<double>(const cplx<double>*, cplx<double>*, int, long long, int,
                                            cudaStream_t);

}  // namespace sgp
