// sgp_fft.cuh -- complex helpers and the in-CTA line FFT used by every pass.
//
// The discrete transforms are those of Sec. 3.1 (forward with the kernel
// exp(-2 pi i p j / N), inverse with exp(+2 pi i p j / N)); normalisation is
// not applied here (the 1/N factors are folded into the per-mode tables).
//
// Line FFT scheme: a line of N complex values is owned by T = N/E threads;
// thread i holds elements i + T*c (c = 0..E-1) in registers ("layout A").
// Each Stockham radix stage (radix RD, span NS = product of earlier radices)
// reads its butterfly inputs straight from layout A (butterfly b = i + T*k
// takes elements b + r*N/RD = i + T*(k + r*E/RD)), applies the twiddles
// exp(-+2 pi i (b mod NS) r / (NS*RD)), does the RD-point DFT and scatters to
// (b div NS)*NS*RD + (b mod NS) + r*NS; a shared-memory exchange brings the
// data back to layout A.  The last stage's scatter is layout A itself, so a
// transform of S stages needs S-1 exchanges and leaves the result in natural
// order in the same layout as its input.
//
// All five components of a point live in the same thread, which lets the
// pointwise nonlinear flow and the per-mode 5x5 mix run on registers between
// two transforms.  The stage twiddles are formed once per stage and reused
// for the five components; exchanges alternate between two buffers so that
// one __syncthreads per component and stage suffices.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sgp {

// ----------------------------------------------------------------------------
// complex helpers (float2 / double2)
// ----------------------------------------------------------------------------
template <typename R> struct cplx_t;
template <> struct cplx_t<float> { typedef float2 type; };
template <> struct cplx_t<double> { typedef double2 type; };
template <typename R> using cplx = typename cplx_t<R>::type;

__device__ __forceinline__ float2 mkc(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mkc(double a, double b) { return make_double2(a, b); }

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mkc(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mkc(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cconj(C a) { return mkc(a.x, -a.y); }
template <typename C> __device__ __forceinline__ C cneg(C a) { return mkc(-a.x, -a.y); }
// a * b
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return mkc(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
  return mkc(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
// conj(a) * b
template <typename C> __device__ __forceinline__ C cconjmul(C a, C b) {
  return mkc(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}
template <typename C, typename R> __device__ __forceinline__ C cscale(C a, R s) { return mkc(a.x * s, a.y * s); }
// i * a and -i * a
template <typename C> __device__ __forceinline__ C cmuli(C a) { return mkc(-a.y, a.x); }
template <typename C> __device__ __forceinline__ C cmulmi(C a) { return mkc(a.y, -a.x); }
// acc + a * s (s real)
template <typename C, typename R> __device__ __forceinline__ C caxpy(C acc, C a, R s) {
  return mkc(fma(a.x, s, acc.x), fma(a.y, s, acc.y));
}
template <typename C> __device__ __forceinline__ auto cabs2(C a) -> decltype(a.x) {
  return fma(a.x, a.x, a.y * a.y);
}

// FP32: the lane-wise operations as packed two-lane instructions (one issue
// slot for both parts).  Each lane rounds exactly like the scalar form:
// a - b is the fused b*(-1) + a, exact before its single rounding.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }
__device__ __forceinline__ float2 caxpy(float2 acc, float2 a, float s) {
  return __ffma2_rn(a, make_float2(s, s), acc);
}

// ----------------------------------------------------------------------------
// radix plans
// ----------------------------------------------------------------------------
// Radix of stage s for a length-N line with E elements per thread: greedy over
// {8, 6, 4, 3, 2}, each radix dividing both E and what is left of N.  Returns
// 0 past the last stage.
__host__ __device__ constexpr int radix_at(int N, int E, int s) {
  int rem = N;
  for (int k = 0; k <= s; ++k) {
    if (rem == 1) return 0;
    int r = 0;
    if (E % 8 == 0 && rem % 8 == 0) r = 8;
    else if (E % 6 == 0 && rem % 6 == 0) r = 6;
    else if (E % 4 == 0 && rem % 4 == 0) r = 4;
    else if (E % 3 == 0 && rem % 3 == 0) r = 3;
    else if (E % 2 == 0 && rem % 2 == 0) r = 2;
    else return -1;  // no plan: rejected at compile time below
    if (k == s) return r;
    rem /= r;
  }
  return 0;
}

__host__ __device__ constexpr bool plan_ok(int N, int E) {
  if (N % E) return false;
  int s = 0, prod = 1;
  while (true) {
    int r = radix_at(N, E, s);
    if (r < 0) return false;
    if (r == 0) break;
    prod *= r;
    ++s;
  }
  return prod == N;
}

__host__ __device__ constexpr int num_stages(int N, int E) {
  int s = 0;
  while (radix_at(N, E, s) > 0) ++s;
  return s;
}

// Twiddle table layout: stage by stage (stages s >= 1, the first has none),
// inside a stage r-major: entry (s, r, j) = W_{NS*RD}^{j r} = exp(-2 pi i j r
// / (NS RD)) at tw_offset(N, E, s) + (r - 1) * NS + j, j < NS, 1 <= r < RD.
// Butterflies of one warp read consecutive j for a fixed r, so the lookups
// do not collide in the shared-memory banks.  The table has N - RD_0 < N
// entries (sum over stages of NS (RD - 1) telescopes to N - RD_0).
__host__ __device__ constexpr int tw_offset(int N, int E, int s) {
  int off = 0, ns = 1;
  for (int k = 0; k < s; ++k) {
    const int rd = radix_at(N, E, k);
    if (k >= 1) off += (rd - 1) * ns;
    ns *= rd;
  }
  return off;
}

// Shared-memory padding: one element every 128 bytes breaks the power-of-two
// strides of the early stages across banks.
template <typename R> struct PadShift;
template <> struct PadShift<float> { static constexpr int value = 4; };
template <> struct PadShift<double> { static constexpr int value = 3; };
template <typename R> __device__ __forceinline__ int padx(int idx) {
  return idx + (idx >> PadShift<R>::value);
}
// Padded line length (+1 so that consecutive lines start in different banks).
template <typename R> __host__ __device__ constexpr int line_pad(int N) {
  return N + (N >> PadShift<R>::value) + 1;
}
// Padded line length for TILE lines exchanged side by side (the line pass):
// a warp holds 32/TILE positions of TILE lines, so the line-to-line offset
// decides the banks.  The extra words below give the fewest shared-memory
// wavefronts over all exchanges of the Stockham stages, found by counting
// them for every (N, E, TILE) the line-pass variants use; e.g. FP32
// N = 512, TILE = 8: +2 gives 1024 wavefronts per CTA instead of 1792 with
// +1, and N = 48, TILE = 32: +0 gives 576 instead of 2304.
template <typename R> __host__ __device__ constexpr int line_pad_extra(int N, int TILE) {
  if (sizeof(R) == 4) {
    if (TILE >= 16) return (N == 16 || N == 48) ? 0 : 1;
    if (TILE == 8) return N == 96 ? 0 : 2;
    if (TILE == 4) return N == 192 ? 0 : 4;
    if (TILE == 2) return N == 384 ? 0 : 8;
    return 0;
  }
  if (TILE == 4) return 2;
  if (TILE == 2) return N % 3 == 0 ? 4 : 0;
  return TILE == 1 ? 0 : 1;
}
template <typename R> __host__ __device__ constexpr int line_pad_tile(int N, int TILE) {
  return N + (N >> PadShift<R>::value) + line_pad_extra<R>(N, TILE);
}

// ----------------------------------------------------------------------------
// small DFTs, DIR = -1 forward, +1 inverse
// ----------------------------------------------------------------------------
template <int DIR, typename C> __device__ __forceinline__ C rot_mi(C a) {
  // multiply by -i (forward) or +i (inverse)
  return DIR < 0 ? cmulmi(a) : cmuli(a);
}

// x * k for the butterfly constants sqrt(1/2) and sqrt(3)/2.  In FP32 the
// constant is the unevaluated sum hi + lo and the product is formed as
// fma(x, hi, x*lo): one rounding of x*(hi + lo).  A plain rounded constant
// (or fma(x, lo, x*hi), whose small term is lost against the rounded large
// product) biases every forward/inverse pair the same way: with k^2 = 1/2
// rounded, each radix-8 butterfly would shrink the norm by ~1e-8 and a
// long run would lose mass steadily.
__device__ __forceinline__ float mul_rt_half(float x) {
  return fmaf(x, 0.7071067690849304f, x * 1.21016175e-08f);
}
__device__ __forceinline__ double mul_rt_half(double x) { return x * 0.70710678118654752440; }
__device__ __forceinline__ float mul_rt3_half(float x) {
  return fmaf(x, 0.8660253882408142f, x * 1.5543625e-08f);
}
__device__ __forceinline__ double mul_rt3_half(double x) { return x * 0.86602540378443864676; }

// Twiddle table entries.  FP32: W = hi + lo (both float2), applied with
// tw_mul as one rounding of the product with the unevaluated sum, so the
// table's rounding does not shrink or grow every forward/inverse pair; FP64:
// the rounded value alone.
template <typename R> struct TwE;
template <> struct TwE<float> { float2 hi, lo; };
template <> struct TwE<double> { double2 hi; };

__device__ __forceinline__ TwE<float> tw_conj(TwE<float> t) {
  return TwE<float>{make_float2(t.hi.x, -t.hi.y), make_float2(t.lo.x, -t.lo.y)};
}
__device__ __forceinline__ TwE<double> tw_conj(TwE<double> t) {
  return TwE<double>{make_double2(t.hi.x, -t.hi.y)};
}
__device__ __forceinline__ float2 tw_mul(float2 x, TwE<float> w) {
  const float sr = fmaf(x.x, w.lo.x, -x.y * w.lo.y);
  const float si = fmaf(x.x, w.lo.y, x.y * w.lo.x);
  return make_float2(fmaf(x.x, w.hi.x, fmaf(-x.y, w.hi.y, sr)),
                     fmaf(x.x, w.hi.y, fmaf(x.y, w.hi.x, si)));
}
__device__ __forceinline__ double2 tw_mul(double2 x, TwE<double> w) {
  return make_double2(fma(x.x, w.hi.x, -x.y * w.hi.y), fma(x.x, w.hi.y, x.y * w.hi.x));
}
// The same product with each of the four partial products rounded once with
// its own correction, then combined.  Needed when a twiddle component is
// exact in FP32 (+-1/2, as at multiples of 30 degrees in the plans with a
// factor 3): in tw_mul the lo term of the other component is then added to
// an exactly representable partial product, stays below half an ulp and is
// rounded away every time, and since the hi part of sqrt(3)/2 is rounded
// down the product is always slightly too small (a steady mass loss of a few
// 1e-9 per transform).  Here no correction meets an exact value alone.
__device__ __forceinline__ float2 tw_mul_split(float2 x, TwE<float> w) {
  const float p = fmaf(x.x, w.hi.x, x.x * w.lo.x);
  const float q = fmaf(x.y, w.hi.y, x.y * w.lo.y);
  const float r = fmaf(x.x, w.hi.y, x.x * w.lo.y);
  const float s = fmaf(x.y, w.hi.x, x.y * w.lo.x);
  return make_float2(p - q, r + s);
}
__device__ __forceinline__ double2 tw_mul_split(double2 x, TwE<double> w) { return tw_mul(x, w); }
// twiddle product of a length-N plan
template <int N, typename C, typename W>
__device__ __forceinline__ C tw_apply(C x, W w) {
  if constexpr (N % 3 == 0)
    return tw_mul_split(x, w);
  else
    return tw_mul(x, w);
}

template <int RD, int DIR, typename C> struct Dft;

template <int DIR, typename C> struct Dft<2, DIR, C> {
  __device__ __forceinline__ static void run(C (&x)[2]) {
    C a = x[0], b = x[1];
    x[0] = cadd(a, b);
    x[1] = csub(a, b);
  }
};

template <int DIR, typename C> struct Dft<4, DIR, C> {
  __device__ __forceinline__ static void run(C (&x)[4]) {
    C t0 = cadd(x[0], x[2]), t1 = csub(x[0], x[2]);
    C t2 = cadd(x[1], x[3]), t3 = rot_mi<DIR>(csub(x[1], x[3]));
    x[0] = cadd(t0, t2);
    x[2] = csub(t0, t2);
    x[1] = cadd(t1, t3);
    x[3] = csub(t1, t3);
  }
};

template <int DIR, typename C> struct Dft<8, DIR, C> {
  __device__ __forceinline__ static void run(C (&x)[8]) {
    C e[4] = {x[0], x[2], x[4], x[6]};
    C o[4] = {x[1], x[3], x[5], x[7]};
    Dft<4, DIR, C>::run(e);
    Dft<4, DIR, C>::run(o);
    // twiddles W8^k, k = 1..3 (forward: (1-i)/sqrt2, -i, (-1-i)/sqrt2)
    C o1 = o[1], o2 = o[2], o3 = o[3];
    if (DIR < 0) {
      o1 = mkc(mul_rt_half(o1.x + o1.y), mul_rt_half(o1.y - o1.x));
      o2 = cmulmi(o2);
      o3 = mkc(mul_rt_half(o3.y - o3.x), -mul_rt_half(o3.x + o3.y));
    } else {
      o1 = mkc(mul_rt_half(o1.x - o1.y), mul_rt_half(o1.y + o1.x));
      o2 = cmuli(o2);
      o3 = mkc(-mul_rt_half(o3.x + o3.y), mul_rt_half(o3.x - o3.y));
    }
    x[0] = cadd(e[0], o[0]);
    x[4] = csub(e[0], o[0]);
    x[1] = cadd(e[1], o1);
    x[5] = csub(e[1], o1);
    x[2] = cadd(e[2], o2);
    x[6] = csub(e[2], o2);
    x[3] = cadd(e[3], o3);
    x[7] = csub(e[3], o3);
  }
};

template <int DIR, typename C> struct Dft<3, DIR, C> {
  __device__ __forceinline__ static void run(C (&x)[3]) {
    typedef decltype(x[0].x) R;
    C t = cadd(x[1], x[2]);
    C u = csub(x[1], x[2]);
    C m = mkc(fma(t.x, (R)-0.5, x[0].x), fma(t.y, (R)-0.5, x[0].y));
    // forward: X1 = m - i s3 u, X2 = m + i s3 u
    const R su_x = mul_rt3_half(u.x), su_y = mul_rt3_half(u.y);
    C iu = DIR < 0 ? mkc(su_y, -su_x) : mkc(-su_y, su_x);
    x[0] = cadd(x[0], t);
    x[1] = cadd(m, iu);
    x[2] = csub(m, iu);
  }
};

template <int DIR, typename C> struct Dft<6, DIR, C> {
  __device__ __forceinline__ static void run(C (&x)[6]) {
    typedef decltype(x[0].x) R;
    C e[3] = {x[0], x[2], x[4]};
    C o[3] = {x[1], x[3], x[5]};
    Dft<3, DIR, C>::run(e);
    Dft<3, DIR, C>::run(o);
    // W6^1 = 1/2 -+ i s3, W6^2 = -1/2 -+ i s3 (s3 = sqrt(3)/2):
    // o * (+-1/2 + i sg s3) = (+-o.x/2 - sg s3 o.y, +-o.y/2 + sg s3 o.x)
    const R sg = DIR < 0 ? (R)-1 : (R)1;
    const R a1x = mul_rt3_half(o[1].x), a1y = mul_rt3_half(o[1].y);
    const R a2x = mul_rt3_half(o[2].x), a2y = mul_rt3_half(o[2].y);
    C o1 = mkc((R)0.5 * o[1].x - sg * a1y, (R)0.5 * o[1].y + sg * a1x);
    C o2 = mkc((R)-0.5 * o[2].x - sg * a2y, (R)-0.5 * o[2].y + sg * a2x);
    x[0] = cadd(e[0], o[0]);
    x[3] = csub(e[0], o[0]);
    x[1] = cadd(e[1], o1);
    x[4] = csub(e[1], o1);
    x[2] = cadd(e[2], o2);
    x[5] = csub(e[2], o2);
  }
};

// ----------------------------------------------------------------------------
// barrier of the threads that share a set of exchange buffers
// ----------------------------------------------------------------------------
// GT = 0: the whole CTA; GT = 32: one warp; otherwise the GT threads (a
// multiple of 32) that use named barrier `id` (1..15; 0 is the CTA's).
template <int GT>
__device__ __forceinline__ void group_sync(int id) {
  if constexpr (GT == 0) {
    __syncthreads();
  } else if constexpr (GT == 32) {
    __syncwarp();
  } else {
    static_assert(GT % 32 == 0, "named barriers count whole warps");
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "n"(GT) : "memory");
  }
}

// ----------------------------------------------------------------------------
// Stockham stages over NC components held in registers
// ----------------------------------------------------------------------------
// v[c][e]: element i + T*e of component c's line.  tw: the stage twiddle
// table (TwE entries), in shared memory.  Exchange buffers: buffer b of this
// thread group's line is buf0 + b * bstride (padded, LP elements).  With
// NB = 2 components alternate between two buffers and every component's
// exchange has its own barrier; with NB = NC each component has its own
// buffer, so a stage writes all components, passes one barrier and reads
// them all (one more barrier before the next stage writes): the five
// butterflies of a stage are independent work for the scheduler.  DIR = -1
// forward, +1 inverse.  Every thread of the CTA must call this (barriers).
template <typename R, int N, int E, int DIR, int NC, int NB, int S, int NS, int GT>
struct FftStages {
  typedef cplx<R> C;
  __device__ __forceinline__ static void run(C (&v)[NC][E], int i, const TwE<R>* tw,
                                             C* buf0, int bstride, int bid) {
    constexpr int RD = radix_at(N, E, S);
    if constexpr (RD > 0) {
      constexpr int T = N / E;
      constexpr int B = E / RD;
      constexpr bool LAST = (NS * RD == N);
      constexpr int TOFF = tw_offset(N, E, S);
      TwE<R> w[B][RD];
#pragma unroll
      for (int k = 0; k < B; ++k) {
        if constexpr (NS > 1) {
          const int j = (i + T * k) % NS;
#pragma unroll
          for (int r = 1; r < RD; ++r) {
            const TwE<R> t = tw[TOFF + (r - 1) * NS + j];
            w[k][r] = DIR < 0 ? t : tw_conj(t);
          }
        }
      }
      // NB = NC: the previous stage's reads of the buffers must be done
      if constexpr (!LAST && NB != 2 && S > 0) group_sync<GT>(bid);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        C* buf = buf0 + (NB == 2 ? ((S * NC + c) & 1) : c) * bstride;
#pragma unroll
        for (int k = 0; k < B; ++k) {
          C x[RD];
#pragma unroll
          for (int r = 0; r < RD; ++r) {
            x[r] = v[c][k + r * B];
            if constexpr (NS > 1) {
              if (r > 0) x[r] = tw_apply<N>(x[r], w[k][r]);
            }
          }
          Dft<RD, DIR, C>::run(x);
          if constexpr (LAST) {
#pragma unroll
            for (int r = 0; r < RD; ++r) v[c][k + r * B] = x[r];
          } else {
            const int b = i + T * k;
            const int idxD = (b / NS) * NS * RD + (b % NS);
#pragma unroll
            for (int r = 0; r < RD; ++r) buf[padx<R>(idxD + r * NS)] = x[r];
          }
        }
        if constexpr (!LAST && NB == 2) {
          group_sync<GT>(bid);
#pragma unroll
          for (int e = 0; e < E; ++e) v[c][e] = buf[padx<R>(i + T * e)];
        }
      }
      if constexpr (!LAST && NB != 2) {
        group_sync<GT>(bid);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const C* buf = buf0 + c * bstride;
#pragma unroll
          for (int e = 0; e < E; ++e) v[c][e] = buf[padx<R>(i + T * e)];
        }
      }
      FftStages<R, N, E, DIR, NC, NB, S + 1, NS * RD, GT>::run(v, i, tw, buf0, bstride, bid);
    }
  }
};

// Exact adjoint of FftStages<..., -1, ...>: the stages in reverse order, each
// gathering its butterfly inputs from the forward stage's scatter positions,
// applying the inverse RD-point DFT and then the conjugated twiddles, and
// leaving its outputs at the forward stage's input positions (layout A).
// With the same rounded twiddle table, forward followed by this adjoint
// equals N times the identity up to |W|^2 - 1 and butterfly rounding: the
// twiddle phase errors cancel instead of accumulating over many steps.
template <typename R, int N, int E, int NC, int NB, int S, int NS, int GT>
struct FftStagesAdj {
  typedef cplx<R> C;
  __device__ __forceinline__ static void run(C (&v)[NC][E], int i, const TwE<R>* tw,
                                             C* buf0, int bstride, int bid) {
    constexpr int RD = radix_at(N, E, S);
    if constexpr (RD > 0) {
      // later forward stages come first in the adjoint
      FftStagesAdj<R, N, E, NC, NB, S + 1, NS * RD, GT>::run(v, i, tw, buf0, bstride, bid);
      constexpr int T = N / E;
      constexpr int B = E / RD;
      constexpr bool LAST = (NS * RD == N);
      // the first buffer-using stage of the adjoint is the one before LAST
      constexpr bool FIRSTBUF = (NS * RD * radix_at(N, E, S + 1) == N);
      constexpr int TOFF = tw_offset(N, E, S);
      TwE<R> w[B][RD];
#pragma unroll
      for (int k = 0; k < B; ++k) {
        if constexpr (NS > 1) {
          const int j = (i + T * k) % NS;
#pragma unroll
          for (int r = 1; r < RD; ++r) w[k][r] = tw_conj(tw[TOFF + (r - 1) * NS + j]);
        }
      }
      if constexpr (!LAST && NB != 2) {
        if constexpr (!FIRSTBUF) group_sync<GT>(bid);     // earlier reads of the buffers done
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          C* buf = buf0 + c * bstride;
#pragma unroll
          for (int e = 0; e < E; ++e) buf[padx<R>(i + T * e)] = v[c][e];
        }
        group_sync<GT>(bid);
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        C* buf = buf0 + (NB == 2 ? ((S * NC + c) & 1) : c) * bstride;
        if constexpr (!LAST && NB == 2) {
#pragma unroll
          for (int e = 0; e < E; ++e) buf[padx<R>(i + T * e)] = v[c][e];
          group_sync<GT>(bid);
        }
#pragma unroll
        for (int k = 0; k < B; ++k) {
          C x[RD];
          if constexpr (LAST) {
#pragma unroll
            for (int r = 0; r < RD; ++r) x[r] = v[c][k + r * B];
          } else {
            const int b = i + T * k;
            const int idxD = (b / NS) * NS * RD + (b % NS);
#pragma unroll
            for (int r = 0; r < RD; ++r) x[r] = buf[padx<R>(idxD + r * NS)];
          }
          Dft<RD, +1, C>::run(x);
#pragma unroll
          for (int r = 0; r < RD; ++r) {
            if constexpr (NS > 1) {
              if (r > 0) x[r] = tw_apply<N>(x[r], w[k][r]);
            }
            v[c][k + r * B] = x[r];
          }
        }
      }
    }
  }
};

// Line transforms of NC components (forward DIR = -1, inverse +1); NB
// exchange buffers of bstride elements from buf0 (see FftStages).
template <typename R, int N, int E, int DIR, int NC, int NB, int GT = 0>
__device__ __forceinline__ void fft_lines(cplx<R> (&v)[NC][E], int i, const TwE<R>* tw,
                                          cplx<R>* buf0, int bstride, int bid = 0) {
  static_assert(plan_ok(N, E), "no radix plan for this (N, E)");
  static_assert(NB == 2 || NB == NC, "two alternating buffers or one per component");
  // the previous user of the exchange buffers may still be reading
  group_sync<GT>(bid);
  if constexpr (DIR < 0)
    FftStages<R, N, E, -1, NC, NB, 0, 1, GT>::run(v, i, tw, buf0, bstride, bid);
  else
    FftStagesAdj<R, N, E, NC, NB, 0, 1, GT>::run(v, i, tw, buf0, bstride, bid);
}

}  // namespace sgp
