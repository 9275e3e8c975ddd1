// sgp_kernels.cuh -- pass kernels of the compact splitting propagator.
//
// Two kinds of passes stream the field once each (read + write):
//   x-pass   : contiguous x-lines of all five components of one grid row;
//              optional inverse x-FFT, the exact nonlinear flow (Eq.
//              (solution2)) at every point, optional forward x-FFT.
//   line pass: strided lines (y, or z in 3D) over a tile of consecutive x
//              positions; optional forward FFT, the per-mode linear flow
//              exp(-i|nu|^2 d/2) exp(i d Q) (Eq. (sl1)), optional inverse FFT.
// Between passes the field stays in a mixed representation (transformed
// along the axes already done), so a TS2 step in 2D is one x-pass and one
// line pass.
//
// The per-mode 5x5 matrix exp(i d Q) is never stored: Q = lambda n.f with
// lambda = sqrt(Omega^2 + gamma^2 |nu_perp|^2) (Sec. 3.1; the eigenvalues of Q
// are lambda*{-2..2}), so exp(i d Q) is the spin-2 image of the SU(2) matrix
// U = exp(i d lambda n.sigma/2).  Writing U11 = cp*ahat, U12 = sp*bhat (cp, sp
// real, ahat, bhat unit), the spin-2 image factors as
// diag(w^m) d(cp, sp) diag(z^m), w = ahat*bhat, z = ahat*conj(bhat),
// m = 2..-2, with d the real spin-2 rotation matrix below.  The same
// factorisation gives exp(-i c1 d F.f) of Eq. (solution2).
#pragma once
#include <cuda.h>   // CUtensorMap (the TMA tile loads of line-pass variant 4)

#include "sgp_fft.cuh"

namespace sgp {

// x-pass mode bits
enum { XP_INV = 1, XP_NL = 2, XP_FWD = 4 };

// Physical parameters of one batch member (Sec. 1, Eq. (CGPEs) and the
// harmonic trap), kept in FP64 on the device and read by every CTA of the
// member.
struct MemberPrm {
  double omega, gamma, c0, c1, c2;
  double gx2h, gy2h, gz2h;   // gx^2/2, gy^2/2, gz^2/2 (gz2h = 0 in 2D)
};
// line-pass mode bits
enum { LP_FWD = 1, LP_MIX = 2, LP_INV = 4 };

template <typename R>
struct XPassArgs {
  cplx<R>* field;        // [batch][5][ntot]
  const TwE<R>* tw;      // W_Nx^k, k < Nx
  long long ntot;        // nx*ny*nz
  int rows;              // ny*nz rows per member
  int ny;
  int mode;
  R x0, hx, y0, hy, z0, hz;      // coordinates x_j = x0 + j*hx
  // nonlinear flow over delta at time t = *t_base + t_off
  R delta;
  const MemberPrm* mp;           // [batch]
  const double* t_base;
  double t_off;
  // the copy of the rows right after the nonlinear flow (physical space,
  // same layout as the field) that the x-pass's TAP form writes
  cplx<R>* tap;
};

template <typename R>
struct LPassArgs {
  cplx<R>* field;
  const TwE<R>* tw;           // W_N^k along the line axis
  long long ntot;
  int nx;                     // number of x positions (tile axis)
  long long line_stride;      // element stride along the line
  long long plane_stride;     // element stride between planes (blockIdx.y)
  int mode;
  int axis;                   // 1: lines along y (2D); 2: lines along z (3D)
  int NX, NY;                 // grid sizes along x and y (mode indices)
  // per-mode table over (|p|, |q|), MT_STRIDE values per entry (see MT_*);
  // member m uses mt + m * mt_member (mt_member = 0 when all members share
  // Omega and gamma)
  const R* mt;
  long long mt_member;
  const cplx<R>* kz;          // exp(-i nu_z^2 d/2) - 1 (3D only)
  R inv_hi, inv_lo;           // 1/(NX NY [NZ]) as an unevaluated sum hi + lo
  // TMA tile loads (line-pass variant 4): the first member's index in the
  // batch (tensor coordinate of component c of member m: (mc0 + m) * 5 + c)
  // and the word a bounded wait that gave up sets
  int mc0;
  int* err;
};

// Entry layout of the per-mode table of the linear flow over delta, indexed
// by (|p|, |q|) (everything below depends on nu_x^2 and nu_y^2 only):
//   khat  = exp(-i (nu_x^2 + nu_y^2) delta/2) - 1
//   am1   = ahat - 1, cm1 = cp - 1, sp: U11 = cp*ahat (|ahat| = 1) and
//           U12 = sp*bhat of U = exp(i delta lambda n.sigma/2),
//           lambda^2 = Omega^2 + gamma^2 |nu_perp|^2
//   (bx, by) = (|nu_x|, |nu_y|)/|nu_perp|; the mode direction is
//           bhat = (sign(p) bx, -sign(q) by) = (nu_x - i nu_y)/|nu_perp|.
// The small quantities khat, am1, cm1, sp are formed in FP64 without
// cancellation, so the flow is applied as v + (increment) with the increment
// accurate to its own rounding (see apply_flow_increment).
enum { MT_KHR = 0, MT_KHI, MT_AM1R, MT_AM1I, MT_CM1, MT_SP, MT_BX, MT_BY, MT_STRIDE };

// ----------------------------------------------------------------------------
// spin-2 image of an SU(2) element, applied as an increment
// ----------------------------------------------------------------------------
// e = (D - I) v for D = diag(w^m) d(cp, sp) diag(z^m), w = ahat*bhat,
// z = ahat*conj(bhat) (|ahat| = |bhat| = 1), given am1 = ahat - 1,
// cm1 = cp - 1 and sp (cp^2 + sp^2 = 1).  Written as
//   D - I = diag(w^m) (d - I) diag(z^m) + diag(ahat^(2m) - 1),
// where every entry of d - I and every ahat^(2m) - 1 is built from the small
// inputs without cancellation, so e carries an error relative to its own
// size: the rounding of the (fixed) factors does not accumulate over steps.
template <typename R>
__device__ __forceinline__ void spin2_increment(const cplx<R> (&v)[5], cplx<R> am1,
                                                cplx<R> bhat, R cm1, R sp,
                                                cplx<R> (&e)[5]) {
  typedef cplx<R> C;
  const R r6 = (R)2.44948974278317809820;
  const C ahat = mkc((R)1 + am1.x, am1.y);
  // ahat^2 - 1 = am1 (2 + am1), ahat^4 - 1 = g2 (2 + g2)
  const C g2 = cmul(am1, mkc((R)2 + am1.x, am1.y));
  const C g4 = cmul(g2, mkc((R)2 + g2.x, g2.y));
  const C w = cmul(ahat, bhat);
  const C z = cmulc(ahat, bhat);
  const C z2 = cmul(z, z);
  const C u0 = cmul(z2, v[0]);
  const C u1 = cmul(z, v[1]);
  const C u2 = v[2];
  const C u3 = cmulc(v[3], z);
  const C u4 = cmulc(v[4], z2);
  // d(c, s) - I with c = 1 + cm1, s = sp
  const R c = (R)1 + cm1, s = sp;
  const R c2m1 = cm1 * ((R)2 + cm1);            // c^2 - 1
  const R c2 = (R)1 + c2m1, s2 = s * s, cs = c * s;
  const R Am1 = c2m1 * (c2 + (R)1);             // c^4 - 1
  const R B = s2 * s2;
  const R P = (R)2 * c2 * cs;                   // 2 c^3 s
  const R Qv = (R)2 * cs * s2;                  // 2 c s^3
  const R Rv = r6 * c2 * s2;                    // sqrt6 c^2 s^2
  const R Sv = r6 * cs * (c2 - s2);             // sqrt6 c s (c^2 - s^2)
  const R T1m1 = Am1 - (R)3 * c2 * s2;          // c^2 (c^2 - 3 s^2) - 1
  const R T2 = s2 * ((R)3 * c2 - s2);
  const R M0m1 = Am1 + B - (R)4 * c2 * s2;      // c^4 + s^4 - 4 c^2 s^2 - 1
  C o0 = cscale(u0, Am1);
  o0 = caxpy(o0, u1, P);
  o0 = caxpy(o0, u2, Rv);
  o0 = caxpy(o0, u3, Qv);
  o0 = caxpy(o0, u4, B);
  C o1 = cscale(u0, -P);
  o1 = caxpy(o1, u1, T1m1);
  o1 = caxpy(o1, u2, Sv);
  o1 = caxpy(o1, u3, T2);
  o1 = caxpy(o1, u4, Qv);
  C o2 = cscale(u0, Rv);
  o2 = caxpy(o2, u1, -Sv);
  o2 = caxpy(o2, u2, M0m1);
  o2 = caxpy(o2, u3, Sv);
  o2 = caxpy(o2, u4, Rv);
  C o3 = cscale(u0, -Qv);
  o3 = caxpy(o3, u1, T2);
  o3 = caxpy(o3, u2, -Sv);
  o3 = caxpy(o3, u3, T1m1);
  o3 = caxpy(o3, u4, P);
  C o4 = cscale(u0, B);
  o4 = caxpy(o4, u1, -Qv);
  o4 = caxpy(o4, u2, Rv);
  o4 = caxpy(o4, u3, -P);
  o4 = caxpy(o4, u4, Am1);
  const C w2 = cmul(w, w);
  e[0] = cadd(cmul(w2, o0), cmul(g4, v[0]));
  e[1] = cadd(cmul(w, o1), cmul(g2, v[1]));
  e[2] = o2;
  e[3] = cadd(cmulc(o3, w), cmulc(v[3], g2));     // conj(w) o3 + (conj(ahat^2) - 1) v3
  e[4] = cadd(cmulc(o4, w2), cmulc(v[4], g4));
}

// x * c for a constant given as the unevaluated sum hi + lo (FP32), so the
// product carries only its own rounding; plain product in FP64.
__device__ __forceinline__ float mulc2(float x, float hi, float lo) { return fmaf(x, hi, x * lo); }
__device__ __forceinline__ double mulc2(double x, double hi, double lo) { return x * hi; }

// sin and cos of a small angle.  For |a| < 0.6 the Taylor series to degree
// 9 (sin) and 10 (cos) is used: the remainders are below |a|^11/11! and
// |a|^12/12! (< 1e-10 relative at |a| = 0.6), far below FP32 rounding, and
// sin keeps full relative accuracy for tiny a, which the increment forms
// need.  Larger angles go to the library sincosf.
__device__ __forceinline__ void sincos_small(float a, float* s, float* c) {
  if (fabsf(a) < 0.6f) {
    const float a2 = a * a;
    float ps = fmaf(a2, 2.7557319e-6f, -1.9841270e-4f);   // 1/9!, -1/7!
    ps = fmaf(a2, ps, 8.3333333e-3f);                      // 1/5!
    ps = fmaf(a2, ps, -1.6666667e-1f);                     // -1/3!
    *s = fmaf(a * a2, ps, a);
    float pc = fmaf(a2, -2.7557319e-7f, 2.4801587e-5f);    // -1/10!, 1/8!
    pc = fmaf(a2, pc, -1.3888889e-3f);                     // -1/6!
    pc = fmaf(a2, pc, 4.1666667e-2f);                      // 1/4!
    pc = fmaf(a2, pc, -0.5f);                              // -1/2!
    *c = fmaf(a2, pc, 1.0f);
  } else {
    sincosf(a, s, c);
  }
}
__device__ __forceinline__ void sincos_small(double a, double* s, double* c) { sincos(a, s, c); }
// 1/a: IEEE division in FP64
// 1/a (FP32): the hardware estimate refined by one Newton-Raphson step,
// r + r (1 - a r), within about an ulp (the arguments here lie in (0, 2]).
__device__ __forceinline__ float rcp_r(float a) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return fmaf(r, fmaf(-a, r, 1.0f), r);
}
__device__ __forceinline__ double rcp_r(double a) { return 1.0 / a; }

__device__ __forceinline__ void sincos_r(float a, float* s, float* c) { sincosf(a, s, c); }
__device__ __forceinline__ void sincos_r(double a, double* s, double* c) { sincos(a, s, c); }
// 1/sqrt(a): the hardware estimate plus one Newton step (about 0.5 ulp and
// without the estimate's bias, which would otherwise make the spin-2
// rotation below systematically non-unitary in FP32).
__device__ __forceinline__ float rsqrt_r(float a) {
  const float r = rsqrtf(a);
  const float e = fmaf(-a * r, r, 1.0f);
  return fmaf(0.5f * r, e, r);
}
__device__ __forceinline__ double rsqrt_r(double a) { return rsqrt(a); }

// unit complex in the direction of u (1 if u == 0) and |u|
template <typename C, typename R>
__device__ __forceinline__ C unit_dir(C u, R& mag) {
  const R m2 = cabs2(u);
  if (m2 > (R)0) {
    const R ri = rsqrt_r(m2);
    mag = m2 * ri;
    return mkc(u.x * ri, u.y * ri);
  }
  mag = (R)0;
  return mkc((R)1, (R)0);
}

// SU(2) parameters of the spin rotation exp(-i c1 d F.f) of Eq. (solution2):
// U = cos(k/2) - i sin(k/2) Fhat.sigma, k = c1 d |F|, so U11 = cos(k/2) - i q Fz
// and U12 = -i q conj(F+), q = sin(k/2)/|F|.  ahat - 1 and cp - 1 are formed
// without cancellation:
//   cp - 1 = -q^2 |F+|^2 / (1 + cp),  ahat - 1 = (cos - cp - i q Fz)/cp,
//   cos - cp = -q^2 Fz^2 / (cos + cp).
// Also returns sin and cos of k/2 and 1/|F|.  False (U = I) when F = 0.
template <typename R>
struct SpinRot {
  cplx<R> am1, bhat;
  R cpm1, sp;
  R sh, ch, rFn, Fn;
};

template <typename R>
__device__ __forceinline__ bool spin_rotation(R Fz, cplx<R> Fp, R c1, R delta, SpinRot<R>& o) {
  const R Fp2 = cabs2(Fp);
  const R F2 = Fp2 + Fz * Fz;
  if (!(F2 > (R)0)) return false;
  const R rFn = rsqrt_r(F2);
  const R Fn = F2 * rFn;
  R sh, ch;
  sincos_small((R)0.5 * c1 * delta * Fn, &sh, &ch);
  const R q = sh * rFn;
  const R qFz = q * Fz;
  const R cp2 = ch * ch + qFz * qFz;
  const R icp = rsqrt_r(cp2);
  const R cp = cp2 * icp;
  o.cpm1 = -(q * q * Fp2) * rcp_r((R)1 + cp);
  const R cmc = ch > (R)0 ? -(qFz * qFz) * rcp_r(ch + cp) : ch - cp;   // cos - cp
  o.am1 = mkc(cmc * icp, -qFz * icp);
  R mag;
  o.bhat = unit_dir(mkc(-Fp.y, -Fp.x), mag);   // direction of -i conj(F+)
  o.sp = q * mag;
  o.sh = sh;
  o.ch = ch;
  o.rFn = rFn;
  o.Fn = Fn;
  return true;
}

// ----------------------------------------------------------------------------
// exact nonlinear flow at one point (Sec. 3.2, Eq. (solution2))
// ----------------------------------------------------------------------------
// (F.f) u with the spin-2 matrices of Sec. 1: tridiagonal, diagonal
// (2, 1, 0, -1, -2) Fz, F- = conj(F+) above and F+ below the diagonal,
// times sqrt(6)/2 next to the middle row.  Fz and Fp may carry a common
// real factor.
template <typename R>
__device__ __forceinline__ void spin_dot(R Fz, cplx<R> Fp, const cplx<R> (&u)[5], cplx<R> (&o)[5]) {
  typedef cplx<R> C;
  const C sFp = cscale(Fp, (R)1.22474487139158904910);
  const R Fz2 = (R)2 * Fz;
  o[0] = cadd(cscale(u[0], Fz2), cconjmul(Fp, u[1]));
  o[1] = cadd(cadd(cmul(Fp, u[0]), cscale(u[1], Fz)), cconjmul(sFp, u[2]));
  o[2] = cadd(cmul(sFp, u[1]), cconjmul(sFp, u[3]));
  o[3] = cadd(csub(cmul(sFp, u[2]), cscale(u[3], Fz)), cconjmul(Fp, u[4]));
  o[4] = csub(cmul(Fp, u[3]), cscale(u[4], Fz2));
}

// Two functions of x = a^2 by their Taylor series (for x < 0.25, i.e.
// |a| < 0.5, the remainders are below 3e-11 relative, far below FP32
// rounding, and both keep full relative accuracy for small a, which the
// increment forms need): sinc_sq(x) = sin(a)/a, cosm1_sq(x) = cos(a) - 1.
__device__ __forceinline__ float sinc_sq(float x) {
  float p = fmaf(x, 2.7557319e-6f, -1.9841270e-4f);   // 1/9!, -1/7!
  p = fmaf(x, p, 8.3333333e-3f);                       // 1/5!
  p = fmaf(x, p, -1.6666667e-1f);                      // -1/3!
  return fmaf(x, p, 1.0f);
}
__device__ __forceinline__ float cosm1_sq(float x) {
  float p = fmaf(x, -2.7557319e-7f, 2.4801587e-5f);   // -1/10!, 1/8!
  p = fmaf(x, p, -1.3888889e-3f);                      // -1/6!
  p = fmaf(x, p, 4.1666667e-2f);                       // 1/4!
  p = fmaf(x, p, -0.5f);                               // -1/2!
  return x * p;
}

template <typename R>
__device__ __forceinline__ void nonlinear_point(cplx<R> (&v)[5], R V, R delta,
                                                R c0p, R c1, R c2) {
  typedef cplx<R> C;
  constexpr bool F32 = sizeof(R) == 4;
  const R r6 = (R)2.44948974278317809820;
  const R rs5 = (R)0.44721359549995793928;   // 1/sqrt(5)
  const R a0 = cabs2(v[0]), a1 = cabs2(v[1]), a2 = cabs2(v[2]);
  const R a3 = cabs2(v[3]), a4 = cabs2(v[4]);
  const R rho = a0 + a1 + a2 + a3 + a4;
  const R Fz = (R)2 * (a0 - a4) + a1 - a3;
  // F_+ = 2(conj(p2) p1 + conj(m1) m2) + sqrt6 (conj(p1) p0 + conj(p0) m1)
  C Fp = cscale(cadd(cconjmul(v[0], v[1]), cconjmul(v[3], v[4])), (R)2);
  Fp = cadd(Fp, cscale(cadd(cconjmul(v[1], v[2]), cconjmul(v[2], v[3])), r6));
  // A00 = (2 p2 m2 - 2 p1 m1 + p0^2)/sqrt5
  C A00 = csub(cmul(v[0], v[4]), cmul(v[1], v[3]));
  A00 = cscale(cadd(cscale(A00, (R)2), cmul(v[2], v[2])), rs5);
  // (1) singlet-pair rotation, as the increment of
  //     b = cos(th) Psi + i sin(th)/S (rho/5 Psi - A00 A conj(Psi)),
  //     th = c2 S d, S^2 = rho^2/25 - |A00|^2/5
  const R S2 = rho * rho * (R)0.04 - cabs2(A00) * (R)0.2;
  R cm1, sinc;       // cos(th) - 1 and sin(th)/S
  const R th2 = c2 * delta * c2 * delta * (S2 > (R)0 ? S2 : (R)0);
  if (F32 && th2 < (R)0.25) {
    // half-angle series in u = (th/2)^2, no square root: sh = sin(th/2) =
    // (th/2) q, ch = cos(th/2); cm1 = -2 sh^2, sin(th)/S = 2 sh ch / S =
    // c2 d q ch.  As in the form below, (1 + cm1)^2 + (sinc S)^2 - 1 =
    // -4 sh^2 (1 - sh^2 - ch^2): the rounding of the series enters the norm
    // only times sh^2.
    const float u = 0.25f * (float)th2;
    const R q = (R)sinc_sq(u), ch = (R)1 + (R)cosm1_sq(u);
    cm1 = (R)-2 * (R)u * q * q;
    sinc = c2 * delta * q * ch;
  } else {
    R S = (R)0, rS = (R)0;
    if (S2 > (R)0) {
      rS = rsqrt_r(S2);
      S = S2 * rS;
    }
    R sh1, ch1;
    sincos_small((R)0.5 * c2 * S * delta, &sh1, &ch1);
    cm1 = (R)-2 * sh1 * sh1;
    sinc = S > (R)0 ? (R)2 * sh1 * ch1 * rS : c2 * delta;
  }
  // increment = (cm1 + i sinc rho/5) Psi - (i sinc A00/sqrt5) (sqrt5 A conj(Psi)),
  // sqrt5 A conj(Psi) = (conj m2, -conj m1, conj p0, -conj p1, conj p2)
  const C al = mkc(cm1, sinc * rho * (R)0.2);
  const C be = cmuli(cscale(A00, sinc * rs5));
  C inc[5], b[5];
  {
    const C ac[5] = {cconj(v[4]), cneg(cconj(v[3])), cconj(v[2]),
                     cneg(cconj(v[1])), cconj(v[0])};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      inc[k] = csub(cmul(al, v[k]), cmul(be, ac[k]));
      b[k] = cadd(v[k], inc[k]);
    }
  }
  // (2) spin rotation exp(-iK) b, K = c1 d F.f, applied as an increment.
  //     FP32, when every point of the warp has |K| = 2 |c1 d| |F| <= 3.5e-3:
  //     the degree-2 Taylor polynomial, e = -iK (b - (i/2) K b); its
  //     remainder |K|^3/6 < 7.2e-9 relative is a quarter of an FP32
  //     rounding and it changes |b|^2 by |K|^4/4 < 4e-11.  Otherwise the
  //     spin-2 image of the SU(2) element (spin_rotation), exact for any K.
  bool taylor = false;
  if constexpr (F32) {
    const R k1 = c1 * delta;
    const R K2 = (R)4 * k1 * k1 * (cabs2(Fp) + Fz * Fz);
    taylor = __all_sync(0xffffffffu, K2 <= (R)(3.5e-3 * 3.5e-3));
    if (taylor) {
      C Kb[5], cb[5], e[5];
      spin_dot<R>(k1 * Fz, cscale(Fp, k1), b, Kb);
#pragma unroll
      for (int k = 0; k < 5; ++k) cb[k] = caxpy(b[k], cmulmi(Kb[k]), (R)0.5);
      spin_dot<R>(k1 * Fz, cscale(Fp, k1), cb, e);
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        e[k] = cmulmi(e[k]);
        inc[k] = cadd(inc[k], e[k]);
        b[k] = cadd(b[k], e[k]);
      }
    }
  }
  SpinRot<R> sr;
  if (!taylor && spin_rotation<R>(Fz, Fp, c1, delta, sr)) {
    const C am1 = sr.am1, bhat = sr.bhat;
    const R cpm1 = sr.cpm1, sp = sr.sp;
    C e[5];
    spin2_increment<R>(b, am1, bhat, cpm1, sp, e);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      inc[k] = cadd(inc[k], e[k]);
      b[k] = cadd(b[k], e[k]);
    }
  }
  // (3) scalar phase exp(-i ph) - 1 = (-2 sin^2(ph/2), -sin ph), ph = d (V + (c0 + c2/5) rho),
  //     from the half angle so that |1 + pm1|^2 - 1 = -4 sh^2 (1 - sh^2 - ch^2)
  R sh3, ch3;
  sincos_small((R)-0.5 * delta * (V + c0p * rho), &sh3, &ch3);
  const C pm1 = mkc((R)-2 * sh3 * sh3, (R)2 * sh3 * ch3);
#pragma unroll
  for (int k = 0; k < 5; ++k) v[k] = cadd(v[k], cadd(inc[k], cmul(pm1, b[k])));
}

// ----------------------------------------------------------------------------
// x-pass kernel
// ----------------------------------------------------------------------------
// Geometry variant G: about 256 >> G threads per CTA (rows of the x-pass
// side by side); G > 0 gives more, smaller CTAs for small grids.
template <typename R, int N, int E, int G = 0>
struct XCfg {
  static constexpr int T = N / E;
  static constexpr int CT = 256 >> G;
  static constexpr int ROWS = (CT / T) > 0 ? (CT / T) : 1;
  static constexpr int THREADS = ROWS * T;
  static constexpr int LP = line_pad<R>(N);
  static constexpr int NB = 5;                  // one exchange buffer per component, which
                                                // also stages the rows for the nonlinear flow
  static constexpr int XCH = NB * ROWS * LP;    // exchange buffers (complex)
  static constexpr int BUF = XCH;
  // rows wider than a warp synchronise their exchanges with a named barrier
  // of their own (GT threads) instead of the CTA's
  static constexpr int GT = (ROWS > 1 && ROWS < 16 && T % 32 == 0) ? T : 0;
  static constexpr size_t SMEM = sizeof(TwE<R>) * (size_t)N + sizeof(cplx<R>) * (size_t)BUF;
  // two CTAs per SM when they fit in shared memory; four for the FP32
  // 128-thread geometry (at most 128 registers, a few spilled: 7% faster
  // than the natural ~160 registers at N = 128, 2% slower at N = 512,
  // where the autotuner prefers the 256-thread geometry anyway)
  static constexpr int MINB = (sizeof(R) == 4 && G == 1 && E <= 8 && 4 * SMEM <= 220 * 1024) ? 4
                              : (2 * SMEM <= 220 * 1024 && THREADS <= 128 * (E <= 8 ? 2 : 1)) ? 2 : 1;
};

// x-pass: rows of all five components.  The nonlinear flow runs on the rows
// staged in shared memory between the two transforms, as a plain loop over
// points: one copy of its code (the unrolled form did not fit the
// instruction cache) and registers only for the point being processed.
// Each row's staging area is its own exchange buffers and each thread
// stages, processes and reads back only the points it holds, so the rows
// of a CTA synchronise independently (Cfg::GT) and the nonlinear flow needs
// one barrier.
// Field loads of a pass: plain (may be served by L1), or L2-only when the
// data was written by other CTAs of the same launch (the persistent
// ensemble kernel), whose stores the SM's L1 does not see.
template <bool CG, typename C>
__device__ __forceinline__ C ld_field(const C* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

// The nonlinear flow at the points i + T e of one row that the calling thread
// holds, staged in the row's exchange buffers b0 + c * bstride: the thread
// processes exactly the points it staged, so no barrier is needed.  prm: the
// member's rotation and parameters (cos, sin of Omega t, c0 + c2/5, c1, c2,
// gx^2/2, gy^2/2, gz^2/2); yz: the row's y and z.
template <typename R, int N, int E>
__device__ __forceinline__ void row_flow(cplx<R> (&v)[5][E], const XPassArgs<R>& a, cplx<R>* b0,
                                         int bstride, int i, const R* prm, const R* yz) {
  typedef cplx<R> C;
  constexpr int T = N / E;
#pragma unroll
  for (int c = 0; c < 5; ++c)
#pragma unroll
    for (int e = 0; e < E; ++e) b0[c * bstride + i + T * e] = v[c][e];
  const R co = prm[0], si = prm[1];
  const R c0p = prm[2], c1 = prm[3], c2 = prm[4];
  const R gx2h = prm[5], gy2h = prm[6], gz2h = prm[7];
#pragma unroll 1
  for (int j = i; j < N; j += T) {
    const R y = yz[0];
    const R zz = gz2h * yz[1] * yz[1];
    const R x = a.x0 + (R)j * a.hx;
    const R xr = co * x + si * y;
    const R yr = co * y - si * x;
    const R V = gx2h * xr * xr + gy2h * yr * yr + zz;
    C* pp = b0 + j;
    C p[5] = {pp[0], pp[bstride], pp[2 * bstride], pp[3 * bstride], pp[4 * bstride]};
    nonlinear_point<R>(p, V, a.delta, c0p, c1, c2);
#pragma unroll
    for (int c = 0; c < 5; ++c) pp[c * bstride] = p[c];
  }
#pragma unroll
  for (int c = 0; c < 5; ++c)
#pragma unroll
    for (int e = 0; e < E; ++e) v[c][e] = b0[c * bstride + i + T * e];
}

// Body of the x-pass for block (bx, member): the CTA's rows are
// bx * ROWS .. bx * ROWS + ROWS - 1 of member `member`.  Called by k_xpass
// with the block's own coordinates and by the persistent ensemble kernel
// for each work item it takes.
template <typename R, int N, int E, int G, bool CG = false, bool TAP = false>
__device__ __forceinline__ void xpass_body(const XPassArgs<R>& a, int bx, int member,
                                           unsigned char* smem_raw) {
  typedef cplx<R> C;
  typedef XCfg<R, N, E, G> Cfg;
  constexpr int T = Cfg::T;
  TwE<R>* tw = reinterpret_cast<TwE<R>*>(smem_raw);
  C* xb = reinterpret_cast<C*>(tw + N);
  // rotation cos/sin and the member's parameters in R, formed once per CTA
  // (FP64 work runs at a small fraction of the FP32 rate on this part)
  __shared__ R s_prm[8];
  __shared__ R s_yz[Cfg::ROWS][2];    // y and z of the CTA's rows
  const int g = threadIdx.x / T;
  const int i = threadIdx.x - g * T;
  for (int k = threadIdx.x; k < N; k += Cfg::THREADS) tw[k] = a.tw[k];
  if ((a.mode & XP_NL) && threadIdx.x == 0) {
    const MemberPrm& P = a.mp[member];
    const double t = *a.t_base + a.t_off;
    double sn, cs;
    sincos(P.omega * t, &sn, &cs);
    s_prm[0] = (R)cs;
    s_prm[1] = (R)sn;
    s_prm[2] = (R)(P.c0 + P.c2 / 5.0);
    s_prm[3] = (R)P.c1;
    s_prm[4] = (R)P.c2;
    s_prm[5] = (R)P.gx2h;
    s_prm[6] = (R)P.gy2h;
    s_prm[7] = (R)P.gz2h;
  }
  if ((a.mode & XP_NL) && threadIdx.x < Cfg::ROWS) {
    const int rr = bx * Cfg::ROWS + threadIdx.x;
    s_yz[threadIdx.x][0] = a.y0 + (R)(rr % a.ny) * a.hy;
    s_yz[threadIdx.x][1] = a.z0 + (R)(rr / a.ny) * a.hz;
  }
  const int row = bx * Cfg::ROWS + g;
  const bool valid = row < a.rows;
  C* base = a.field + (size_t)member * 5 * a.ntot + (size_t)(valid ? row : 0) * N + i;
  C v[5][E];
#pragma unroll
  for (int c = 0; c < 5; ++c)
#pragma unroll
    for (int e = 0; e < E; ++e)
      v[c][e] = valid ? ld_field<CG>(base + (size_t)c * a.ntot + T * e) : mkc((R)0, (R)0);
  // twiddles, s_prm and s_yz come from other rows' threads
  __syncthreads();
  constexpr int GT = Cfg::GT;
  const int bid = 1 + g;              // the row's named barrier when GT > 0
  C* b0 = xb + g * Cfg::LP;           // the row's buffer of component c: b0 + c * bstride
  const int bstride = Cfg::ROWS * Cfg::LP;
  if (a.mode & XP_INV) fft_lines<R, N, E, +1, 5, Cfg::NB, GT>(v, i, tw, b0, bstride, bid);
  if (a.mode & XP_NL) {
    group_sync<GT>(bid);              // the row's exchange reads are done
    row_flow<R, N, E>(v, a, b0, bstride, i, s_prm, s_yz[g]);
    if constexpr (TAP) {
      if (valid) {
        C* tp = a.tap + (base - a.field);
#pragma unroll
        for (int c = 0; c < 5; ++c)
#pragma unroll
          for (int e = 0; e < E; ++e) tp[(size_t)c * a.ntot + T * e] = v[c][e];
      }
    }
  }
  if (a.mode & XP_FWD) fft_lines<R, N, E, -1, 5, Cfg::NB, GT>(v, i, tw, b0, bstride, bid);
  if (valid) {
#pragma unroll
    for (int c = 0; c < 5; ++c)
#pragma unroll
      for (int e = 0; e < E; ++e) base[(size_t)c * a.ntot + T * e] = v[c][e];
  }
}

template <typename R, int N, int E, int G>
__global__ void __launch_bounds__(XCfg<R, N, E, G>::THREADS, XCfg<R, N, E, G>::MINB)
k_xpass(XPassArgs<R> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  xpass_body<R, N, E, G>(a, blockIdx.x, blockIdx.y, smem_raw);
}

// x-pass variant 6 (small grids): the rows of x-pass geometry 2 (about 64
// threads side by side) transformed by their FT threads, and the nonlinear
// flow at the rows' points shared by all kXWideThreads threads of the CTA.
// A small grid fills few SMs, and a thread of the other variants takes its
// E points through the flow one after the other; here each takes
// ROWS * N / kXWideThreads.  The transforms synchronise with a named
// barrier of the FT threads; the arithmetic per line and per point is that
// of the other variants with the same elements per thread.
constexpr int kXWideThreads = 256;

template <typename R, int N, int E>
__global__ void __launch_bounds__(kXWideThreads, 2) k_xpass_wide(XPassArgs<R> a) {
  typedef cplx<R> C;
  typedef XCfg<R, N, E, 2> Cfg;
  constexpr int T = Cfg::T, FT = Cfg::THREADS, ROWS = Cfg::ROWS;
  static_assert(kXWideThreads % FT == 0 && FT % 32 == 0, "x-pass variant 6 geometry");
  constexpr int GT = FT == kXWideThreads ? 0 : FT;      // the transforms' barrier
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TwE<R>* tw = reinterpret_cast<TwE<R>*>(smem_raw);
  C* xb = reinterpret_cast<C*>(tw + N);
  __shared__ R s_prm[8];
  __shared__ R s_yz[ROWS][2];
  const int member = blockIdx.y;
  const int tid = threadIdx.x;
  const int g = tid / T;
  const int i = tid - g * T;
  for (int k = tid; k < N; k += kXWideThreads) tw[k] = a.tw[k];
  if ((a.mode & XP_NL) && tid == 0) {
    const MemberPrm& P = a.mp[member];
    const double t = *a.t_base + a.t_off;
    double sn, cs;
    sincos(P.omega * t, &sn, &cs);
    s_prm[0] = (R)cs;
    s_prm[1] = (R)sn;
    s_prm[2] = (R)(P.c0 + P.c2 / 5.0);
    s_prm[3] = (R)P.c1;
    s_prm[4] = (R)P.c2;
    s_prm[5] = (R)P.gx2h;
    s_prm[6] = (R)P.gy2h;
    s_prm[7] = (R)P.gz2h;
  }
  if ((a.mode & XP_NL) && tid < ROWS) {
    const int rr = blockIdx.x * ROWS + tid;
    s_yz[tid][0] = a.y0 + (R)(rr % a.ny) * a.hy;
    s_yz[tid][1] = a.z0 + (R)(rr / a.ny) * a.hz;
  }
  const int bstride = ROWS * Cfg::LP;
  const int row = blockIdx.x * ROWS + g;
  const bool valid = tid < FT && row < a.rows;
  C* base = a.field + (size_t)member * 5 * a.ntot + (size_t)(valid ? row : 0) * N + i;
  C* b0 = xb + g * Cfg::LP;
  C v[5][E];
  if (tid < FT) {
#pragma unroll
    for (int c = 0; c < 5; ++c)
#pragma unroll
      for (int e = 0; e < E; ++e) v[c][e] = valid ? base[(size_t)c * a.ntot + T * e] : mkc((R)0, (R)0);
  }
  __syncthreads();                    // twiddles, s_prm, s_yz
  if (tid < FT && (a.mode & XP_INV)) fft_lines<R, N, E, +1, 5, Cfg::NB, GT>(v, i, tw, b0, bstride, 1);
  if (a.mode & XP_NL) {
    if (tid < FT) {
      group_sync<GT>(1);              // the exchanges' reads of the buffers are done
#pragma unroll
      for (int c = 0; c < 5; ++c)
#pragma unroll
        for (int e = 0; e < E; ++e) b0[c * bstride + i + T * e] = v[c][e];
    }
    __syncthreads();                  // the rows are staged
    const R co = s_prm[0], si = s_prm[1];
    const R c0p = s_prm[2], c1 = s_prm[3], c2 = s_prm[4];
    const R gx2h = s_prm[5], gy2h = s_prm[6], gz2h = s_prm[7];
#pragma unroll 1
    for (int p = tid; p < ROWS * N; p += kXWideThreads) {
      const int r = p / N, j = p - r * N;
      if (blockIdx.x * ROWS + r >= a.rows) break;     // p only grows
      const R y = s_yz[r][0];
      const R zz = gz2h * s_yz[r][1] * s_yz[r][1];
      const R x = a.x0 + (R)j * a.hx;
      const R xr = co * x + si * y;
      const R yr = co * y - si * x;
      const R V = gx2h * xr * xr + gy2h * yr * yr + zz;
      C* pp = xb + r * Cfg::LP + j;
      C q[5] = {pp[0], pp[bstride], pp[2 * bstride], pp[3 * bstride], pp[4 * bstride]};
      nonlinear_point<R>(q, V, a.delta, c0p, c1, c2);
#pragma unroll
      for (int c = 0; c < 5; ++c) pp[c * bstride] = q[c];
    }
    __syncthreads();                  // every point is done
    if (tid < FT) {
#pragma unroll
      for (int c = 0; c < 5; ++c)
#pragma unroll
        for (int e = 0; e < E; ++e) v[c][e] = b0[c * bstride + i + T * e];
    }
  }
  if (tid < FT) {
    if (a.mode & XP_FWD) fft_lines<R, N, E, -1, 5, Cfg::NB, GT>(v, i, tw, b0, bstride, 1);
    if (valid) {
#pragma unroll
      for (int c = 0; c < 5; ++c)
#pragma unroll
        for (int e = 0; e < E; ++e) base[(size_t)c * a.ntot + T * e] = v[c][e];
    }
  }
}

// ----------------------------------------------------------------------------
// line-pass kernel (strided lines, tile of TILE consecutive x positions)
// ----------------------------------------------------------------------------
// Line pass geometry: up to 512 threads per CTA; 8 FP32 (4 FP64) columns
// per tile at N = 512, i.e. 64 B contiguous per line element (a 256-thread,
// 4-column variant measured slower: 32 B segments split HBM bursts between
// CTAs).
// Geometry variant G = 0: up to 512 threads per CTA, TILE clamped to
// [TMIN, TMAX]; G > 0: about 512 >> G threads, TILE down to 1 column (more,
// smaller CTAs for small grids, at the cost of shorter contiguous segments).
template <typename R, int N, int E, int G = 0>
struct LCfg {
  static constexpr int T = N / E;
  static constexpr int TMAX = sizeof(R) == 4 ? 32 : 16;
  static constexpr int TMIN = G == 0 ? (sizeof(R) == 4 ? 4 : 2) : 1;
  static constexpr int TT = 512 >> G;
  static constexpr int TILE = (TT / T) > TMAX ? TMAX : ((TT / T) < TMIN ? TMIN : (TT / T));
  static constexpr int THREADS = TILE * T;
  static constexpr int LP = line_pad_tile<R>(N, TILE);
  // two alternating exchange buffers (one per component measured 3% slower
  // here: the larger buffers cost more than the barriers they save)
  static constexpr int NB = 2;
  static constexpr size_t SMEM = sizeof(TwE<R>) * (size_t)N + sizeof(cplx<R>) * (size_t)(NB * TILE * LP);
  static constexpr int MINB = (THREADS <= (E <= 8 ? 256 : 128) && 2 * SMEM <= 220 * 1024) ? 2 : 1;
  // lines along y in 2D: the tile's slice of the per-mode table (TILE
  // columns x (N/2 + 1) entries), copied to shared memory asynchronously
  // at the start so that the mix does not wait on L2 for every mode
  static constexpr size_t TAB = (size_t)TILE * (N / 2 + 1) * MT_STRIDE * sizeof(R);
  // 3D z-lines: TILE entries and the N z factors
  static constexpr size_t TABZ = (size_t)TILE * MT_STRIDE * sizeof(R) + (size_t)N * sizeof(cplx<R>);
  static_assert(SMEM + TAB <= 227 * 1024 && TABZ <= TAB, "line pass shared memory");
  // variant 4 (tile loads by tensor copies): TSTG components in flight, as
  // many (at most 4) as keep two CTAs on an SM; the staging buffers share
  // the exchange buffers' region, enlarged to TREG elements if needed
  static constexpr int XB = NB * TILE * LP;
  static constexpr size_t treg(int k) { return (size_t)(k * TILE * N > XB ? k * TILE * N : XB); }
  static constexpr bool tfits(int k) {
    return 2 * (sizeof(TwE<R>) * (size_t)N + sizeof(cplx<R>) * treg(k) + TAB + 1024) <= 226 * 1024;
  }
  static constexpr int TSTG = tfits(4) ? 4 : tfits(3) ? 3 : 2;
  static constexpr size_t TREG = treg(TSTG);
  static constexpr size_t TSMEM = sizeof(TwE<R>) * (size_t)N + sizeof(cplx<R>) * TREG;
};

// dynamic shared memory added to a line pass for its table copies
template <typename Cfg>
inline size_t line_table_bytes(int mode, int axis) {
  if (!(mode & LP_MIX)) return 0;
  return axis == 1 ? Cfg::TAB : axis == 2 ? Cfg::TABZ : 0;
}

template <typename R> struct ModeEntry { R khr, khi, am1r, am1i, cm1, sp, bx, by; };

// a mode-table entry from the shared-memory copy of the table
__device__ __forceinline__ ModeEntry<float> load_mode_shared(const float* t, int idx) {
  const float4 a = reinterpret_cast<const float4*>(t)[2 * idx];
  const float4 b = reinterpret_cast<const float4*>(t)[2 * idx + 1];
  return ModeEntry<float>{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
}
__device__ __forceinline__ ModeEntry<double> load_mode_shared(const double* t, int idx) {
  const double2* q = reinterpret_cast<const double2*>(t) + 4 * idx;
  const double2 a = q[0], b = q[1], c = q[2], d = q[3];
  return ModeEntry<double>{a.x, a.y, b.x, b.y, c.x, c.y, d.x, d.y};
}

// 16-byte asynchronous copy global -> shared (completes at cp_async_wait)
__device__ __forceinline__ void cp_async16(void* dst_shared, const void* src_global) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_shared);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src_global) : "memory");
}
// 8-byte asynchronous copy global -> shared (through L1)
__device__ __forceinline__ void cp_async8(void* dst_shared, const void* src_global) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_shared);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src_global) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// the 3D kinetic factor from the (x, y) one and the z one: (1 + kh)(1 + kz) - 1
template <typename C>
__device__ __forceinline__ C kinetic_z(C kh, C kz) {
  return cadd(cadd(kh, kz), cmul(kh, kz));
}

// linear flow of one Fourier mode (signed indices ps, qs) with its table
// entry m and kinetic factor kh = exp(-i |nu|^2 delta/2) - 1, including the
// 1/(NX NY [NZ]) of the forward transforms:
//   v <- (1 + khat) D v / N = (v + f) / N,  f = e + khat (v + e),  e = (D - I) v.
template <typename R>
__device__ __forceinline__ void mix_entry(cplx<R> (&v)[5], const LPassArgs<R>& a,
                                          const ModeEntry<R>& m, int ps, int qs, cplx<R> kh) {
  typedef cplx<R> C;
  const C bhat = mkc(ps < 0 ? -m.bx : m.bx, qs < 0 ? m.by : -m.by);
  C e[5];
  spin2_increment<R>(v, mkc(m.am1r, m.am1i), bhat, m.cm1, m.sp, e);
  C t[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const C x = cadd(v[k], e[k]);
    t[k] = cadd(v[k], cadd(e[k], cmul(kh, x)));
  }
  if (a.inv_lo == (R)0) {
    // 1/N exact (N a power of two): one packed scaling
#pragma unroll
    for (int k = 0; k < 5; ++k) v[k] = cscale(t[k], a.inv_hi);
  } else {
#pragma unroll
    for (int k = 0; k < 5; ++k)
      v[k] = mkc(mulc2(t[k].x, a.inv_hi, a.inv_lo), mulc2(t[k].y, a.inv_hi, a.inv_lo));
  }
}

// ----------------------------------------------------------------------------
// TMA tile loads of the line pass (variant 4)
// ----------------------------------------------------------------------------
// The tile of a line pass is TILE columns x N line elements of each
// component: at a 512^2 grid, 32 bytes of each of 512 rows 4 KB apart.  In
// variant 4 one thread moves it into shared memory with tensor copies
// (cp.async.bulk.tensor over a 4D map of the field, [comp*member][z][y][x],
// 8-byte elements), two components in flight in the two exchange buffers,
// and the threads read their elements from there; the completion is
// tracked by an mbarrier (transaction bytes) per buffer.  A box holds at
// most 256 elements along each dimension, so a line of N > 256 elements is
// tma_rows<N>() rows per box, N / tma_rows<N>() boxes.
template <int N>
__host__ __device__ constexpr int tma_rows() {
  int d = 1;
  while (N % d != 0 || N / d > 256) ++d;
  return N / d;
}

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of the given parity, at most max_cycles of clock64;
// false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity, long long max_cycles) {
  const long long t0 = clock64();
  while (!mbar_try_wait(b, parity))
    if (clock64() - t0 > max_cycles) return false;
  return true;
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, unsigned long long* bar,
                                            int c0, int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, const void* src, int c0, int c1, int c2,
                                             int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];\n" ::"l"(
          reinterpret_cast<unsigned long long>(map)),
      "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(src))
      : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
// the bulk groups committed before the last `n` have finished reading shared memory
template <int n>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;\n" ::"n"(n) : "memory");
}
// every committed bulk group is complete (its writes performed)
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
// shared-memory writes of this thread visible to the tensor copies that follow
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// limit of a tile-load wait: about a second at the GPU's clock
constexpr long long kTmaWaitCycles = 2000000000LL;

// ----------------------------------------------------------------------------
// xy-plane pass (3D, FP32, NX = NY = N): one thread-block cluster per z plane
// ----------------------------------------------------------------------------
// The x-pass and the two y-line passes of a 3D step fused: a cluster of
// CS = N / L CTAs holds one z plane of one member, CTA r owning the rows
// y = r L .. r L + L - 1 (row phase) and the columns x = r L .. r L + L - 1
// (column phase).  With XP_INV the plane comes in by columns, takes the
// inverse y transform and is handed to the row owners; the rows take the
// inverse x transform, the nonlinear flow and the forward x transform; with
// XP_FWD they are handed back to the column owners for the forward y
// transform and leave by columns.  A hand-over is a set of asynchronous
// stores into the other CTAs' shared memory (distributed shared memory),
// each counting its bytes on an mbarrier of the receiving CTA, which waits
// for all of them (a bounded wait: past the limit the error word is set);
// a cluster barrier before it makes sure every CTA is done with the buffers
// the stores land in.
// The field is then y- and x-spectral between passes, so a step needs only
// this pass and the z-line pass.  Every line takes exactly the arithmetic of
// the x-pass and the y-line pass with the same elements per thread, so the
// results equal those of the unfused passes bit for bit.
template <typename R, int N, int E>
struct PlCfg {
  static constexpr int T = N / E;             // threads per line
  static constexpr int L = 16;                // lines per CTA in either phase
  static constexpr int CS = N / L;            // CTAs per cluster
  static constexpr int THREADS = L * T;
  static constexpr int MINB = 512 / THREADS;  // 16 warps per SM
  static constexpr int LP = line_pad<R>(N);   // row exchange buffers (x-pass layout)
  static constexpr int RSTR = L * LP;         // row phase: component stride
  static constexpr int CP = line_pad_tile<R>(N, L);   // column exchange buffers (line-pass layout)
  static constexpr int CSTR = L * CP;         // column phase: buffer stride (two buffers)
  static constexpr int SL = 5 * N * L;        // column-layout slice [c][y][x - r L]
  static constexpr int REG = (5 * RSTR > SL ? 5 * RSTR : SL) > 2 * CSTR ? (5 * RSTR > SL ? 5 * RSTR : SL)
                                                                        : 2 * CSTR;
  static constexpr size_t SMEM = 2 * sizeof(TwE<R>) * (size_t)N + sizeof(cplx<R>) * (size_t)REG;
  static_assert(N % L == 0 && L % T == 0 && CS >= 2 && CS <= 8, "xy-plane pass geometry");
  static_assert(MINB * SMEM <= 227 * 1024, "xy-plane pass shared memory");
};

// thread-block clusters: the two halves of a barrier over the cluster
// (release / acquire: this CTA's shared-memory accesses before the arrive
// are performed before the other CTAs pass their wait), the address of a
// shared-memory location in another CTA of the cluster, an asynchronous
// store there that counts its bytes on an mbarrier of that CTA, and a
// bounded wait on a local mbarrier that such stores complete (acquire at
// cluster scope: the stored data are visible after it)
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
__device__ __forceinline__ unsigned cluster_map(const void* p, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(smem_addr(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_async(unsigned addr, float2 v, unsigned bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];\n" ::"r"(addr),
               "f"(v.x), "f"(v.y), "r"(bar)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cluster(unsigned long long* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_cluster(unsigned long long* b, unsigned parity, long long max_cycles) {
  const long long t0 = clock64();
  while (!mbar_try_wait_cluster(b, parity))
    if (clock64() - t0 > max_cycles) return false;
  return true;
}

template <typename R, int N, int E>
__global__ void __cluster_dims__(PlCfg<R, N, E>::CS, 1, 1)
    __launch_bounds__(PlCfg<R, N, E>::THREADS, PlCfg<R, N, E>::MINB)
k_xyplane(XPassArgs<R> a, const TwE<R>* __restrict__ twy_g, int* err) {
  typedef cplx<R> C;
  typedef PlCfg<R, N, E> Cfg;
  constexpr int T = Cfg::T, L = Cfg::L;
  // bytes a CTA receives in one hand-over: L lines of N elements, five components
  constexpr unsigned XBYTES = 5u * L * N * sizeof(C);
  static_assert(sizeof(R) == 4, "xy-plane pass: FP32");
  extern __shared__ __align__(16) unsigned char smem_pl[];
  TwE<R>* twx = reinterpret_cast<TwE<R>*>(smem_pl);
  TwE<R>* twy = twx + N;
  C* X = reinterpret_cast<C*>(twy + N);
  __shared__ R s_prm[8];
  __shared__ R s_yz[L][2];
  // completion of the two hand-overs into this CTA (rows, then columns)
  __shared__ __align__(8) unsigned long long s_bar[2];
  const int r = blockIdx.x;                  // rank in the cluster (gridDim.x = CS)
  const int plane = blockIdx.y;
  const int member = blockIdx.z;
  const bool inv = a.mode & XP_INV, fwd = a.mode & XP_FWD;
  if (threadIdx.x == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    mbar_fence_init();
    if (inv) mbar_expect_tx(&s_bar[0], XBYTES);
    if (fwd) mbar_expect_tx(&s_bar[1], XBYTES);
  }
  for (int k = threadIdx.x; k < N; k += Cfg::THREADS) {
    twx[k] = a.tw[k];
    twy[k] = twy_g[k];
  }
  if ((a.mode & XP_NL) && threadIdx.x == 0) {
    const MemberPrm& P = a.mp[member];
    const double t = *a.t_base + a.t_off;
    double sn, cs;
    sincos(P.omega * t, &sn, &cs);
    s_prm[0] = (R)cs;
    s_prm[1] = (R)sn;
    s_prm[2] = (R)(P.c0 + P.c2 / 5.0);
    s_prm[3] = (R)P.c1;
    s_prm[4] = (R)P.c2;
    s_prm[5] = (R)P.gx2h;
    s_prm[6] = (R)P.gy2h;
    s_prm[7] = (R)P.gz2h;
  }
  if ((a.mode & XP_NL) && threadIdx.x < L) {
    s_yz[threadIdx.x][0] = a.y0 + (R)(r * L + threadIdx.x) * a.hy;
    s_yz[threadIdx.x][1] = a.z0 + (R)plane * a.hz;
  }
  C* fm = a.field + (size_t)member * 5 * a.ntot + (size_t)plane * N * N;
  // row phase: row g (y = r L + g), thread i of the row holds x = i + T e
  const int g = threadIdx.x / T;
  const int i = threadIdx.x - g * T;
  C* rb0 = X + g * Cfg::LP;
  // column phase: column cl (x = r L + cl), thread ic of the column holds y = ic + T e
  const int cl = threadIdx.x % L;
  const int ic = threadIdx.x / L;
  C* cb0 = X + cl * Cfg::CP;
  C v[5][E];
  if (inv) {
    const C* src = fm + (size_t)ic * N + r * L + cl;
#pragma unroll
    for (int c = 0; c < 5; ++c)
#pragma unroll
      for (int e = 0; e < E; ++e) v[c][e] = src[(size_t)c * a.ntot + (size_t)T * e * N];
    __syncthreads();                         // tables, s_prm, s_yz, mbarriers
    fft_lines<R, N, E, +1, 5, 2>(v, ic, twy, cb0, Cfg::CSTR);
    // every CTA is done with its exchange buffers, and every CTA's mbarriers
    // are initialised
    cluster_arrive();
    cluster_wait();
    // y = ic + T e goes to row (ic + T e) % L of CTA (ic + T e) / L = T e / L
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int y = ic + T * e;
      const unsigned rank = (unsigned)(T * e / L);
      const unsigned dst = cluster_map(X, rank) + (unsigned)(((y % L) * Cfg::LP + r * L + cl) * sizeof(C));
      const unsigned bar = cluster_map(&s_bar[0], rank);
#pragma unroll
      for (int c = 0; c < 5; ++c) st_async(dst + (unsigned)(c * Cfg::RSTR * sizeof(C)), v[c][e], bar);
    }
    if (!mbar_wait_cluster(&s_bar[0], 0, kTmaWaitCycles) && err) atomicExch(err, 1);
#pragma unroll
    for (int c = 0; c < 5; ++c)
#pragma unroll
      for (int e = 0; e < E; ++e) v[c][e] = rb0[c * Cfg::RSTR + i + T * e];
    fft_lines<R, N, E, +1, 5, 5>(v, i, twx, rb0, Cfg::RSTR);
  } else {
    const C* src = fm + (size_t)(r * L + g) * N + i;
#pragma unroll
    for (int c = 0; c < 5; ++c)
#pragma unroll
      for (int e = 0; e < E; ++e) v[c][e] = src[(size_t)c * a.ntot + T * e];
    __syncthreads();                         // tables, s_prm, s_yz, mbarriers
  }
  if (a.mode & XP_NL) {
    __syncthreads();                         // the rows' exchange reads are done
    row_flow<R, N, E>(v, a, rb0, Cfg::RSTR, i, s_prm, s_yz[g]);
  }
  if (fwd) {
    // the forward x transform reads and writes the row buffers; the other
    // CTAs may store into them once every CTA has arrived after it
    fft_lines<R, N, E, -1, 5, 5>(v, i, twx, rb0, Cfg::RSTR);
    cluster_arrive();
    cluster_wait();
    // x = i + T e goes to column x % L of CTA x / L = T e / L (column layout)
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int x = i + T * e;
      const unsigned rank = (unsigned)(T * e / L);
      const unsigned dst = cluster_map(X, rank) + (unsigned)(((r * L + g) * L + x % L) * sizeof(C));
      const unsigned bar = cluster_map(&s_bar[1], rank);
#pragma unroll
      for (int c = 0; c < 5; ++c) st_async(dst + (unsigned)(c * N * L * sizeof(C)), v[c][e], bar);
    }
    if (!mbar_wait_cluster(&s_bar[1], 0, kTmaWaitCycles) && err) atomicExch(err, 1);
#pragma unroll
    for (int c = 0; c < 5; ++c)
#pragma unroll
      for (int e = 0; e < E; ++e) v[c][e] = X[c * N * L + (ic + T * e) * L + cl];
    fft_lines<R, N, E, -1, 5, 2>(v, ic, twy, cb0, Cfg::CSTR);
    C* dst = fm + (size_t)ic * N + r * L + cl;
#pragma unroll
    for (int c = 0; c < 5; ++c)
#pragma unroll
      for (int e = 0; e < E; ++e) dst[(size_t)c * a.ntot + (size_t)T * e * N] = v[c][e];
  } else {
    C* dst = fm + (size_t)(r * L + g) * N + i;
#pragma unroll
    for (int c = 0; c < 5; ++c)
#pragma unroll
      for (int e = 0; e < E; ++e) dst[(size_t)c * a.ntot + T * e] = v[c][e];
  }
}

// Body of the line pass for block (bx, plane, member): the CTA's columns
// are bx * TILE .. bx * TILE + TILE - 1 of plane `plane` (the z slice for
// y-lines, the y row for z-lines) of member `member`.  Called by k_linepass
// with the block's own coordinates and by the persistent ensemble kernel.
// A line pass's hooks after its forward transform and after its mix: the
// adjoint sweep's line pass adds the per-mode parameter terms of the linear
// flow after the forward transform (the tile then holds the full transform
// of g), and the recomputation keeps a copy of the tile after the mix.  The
// forward passes take NoHook.
// A hook may also stage data of its own in shared memory behind the mode
// table's region (hsm), with copies it starts before the field loads.
struct NoHook {
  template <typename R, int N, int E, int TILE, int THREADS>
  __device__ __forceinline__ void prefetch(unsigned char*, const LPassArgs<R>&, int, int, int) const {}
  template <typename R, int N, int E, int THREADS>
  __device__ __forceinline__ void after_fwd(const cplx<R> (&)[5][E], const LPassArgs<R>&, int, int, bool, int, int,
                                            int, size_t, const unsigned char*) const {}
  template <typename R, int N, int E>
  __device__ __forceinline__ void after_mix(const cplx<R> (&)[5][E], const LPassArgs<R>&, bool, size_t) const {}
};

template <typename R, int N, int E, int G, bool CG = false, bool TMA = false, class Hook = NoHook>
__device__ __forceinline__ void linepass_body(const LPassArgs<R>& a, int bx, int plane, int member,
                                              unsigned char* smem_raw,
                                              const CUtensorMap* tmap = nullptr, const Hook& hook = Hook()) {
  typedef cplx<R> C;
  typedef LCfg<R, N, E, G> Cfg;
  constexpr int T = Cfg::T;
  constexpr int TILE = Cfg::TILE;
  TwE<R>* tw = reinterpret_cast<TwE<R>*>(smem_raw);
  C* xb = reinterpret_cast<C*>(tw + N);
  const int col = threadIdx.x % TILE;
  const int i = threadIdx.x / TILE;
  for (int k = threadIdx.x; k < N; k += Cfg::THREADS) tw[k] = a.tw[k];
  const int xcol = bx * TILE + col;
  const bool valid = xcol < a.nx;
  // With the mix, the mode-table entries the tile uses go to shared memory
  // behind the exchange buffers by asynchronous copies issued here, which
  // complete while the field loads and the forward transform run (the
  // launch adds the bytes of line_table_bytes for exactly these cases):
  //   2D y-lines: the rows |p| of the tile's columns (idle columns of a
  //     ragged tile use p = 0), TILE x (N/2 + 1) entries;
  //   3D z-lines: the tile's TILE entries at (|p|, |q|), q = plane,
  //     then the z factors kz[0..N).
  constexpr int HN = N / 2 + 1;
  constexpr int GR = MT_STRIDE * (int)sizeof(R) / 16;          // 16-byte pieces per entry
  R* smt = reinterpret_cast<R*>(xb + (TMA ? Cfg::TREG : (size_t)Cfg::XB));
  const bool stab = (a.mode & LP_MIX) && a.axis == 1;
  const bool stabz = (a.mode & LP_MIX) && a.axis == 2;
  if (stabz) {
    const R* mtm = a.mt + (size_t)member * a.mt_member;
    const int qq = plane;
    int aqs = qq < a.NY / 2 ? qq : qq - a.NY;
    aqs = aqs < 0 ? -aqs : aqs;
    constexpr int KZ = N * (int)sizeof(C) / 16;
    for (int k = threadIdx.x; k < TILE * GR + KZ; k += Cfg::THREADS) {
      if (k < TILE * GR) {
        const int cc = k / GR, g = k - cc * GR;
        int p = bx * TILE + cc;
        p = p < a.nx ? p : 0;
        int ps = p < a.NX / 2 ? p : p - a.NX;
        ps = ps < 0 ? -ps : ps;
        cp_async16(reinterpret_cast<char*>(smt) + (size_t)k * 16,
                   reinterpret_cast<const char*>(mtm) +
                       ((size_t)(ps * (a.NY / 2 + 1) + aqs) * GR + g) * 16);
      } else {
        const int kk = k - TILE * GR;
        cp_async16(reinterpret_cast<char*>(smt) + (size_t)k * 16,
                   reinterpret_cast<const char*>(a.kz) + (size_t)kk * 16);
      }
    }
    cp_async_commit();
  }
  if (stab) {
    const R* mtm = a.mt + (size_t)member * a.mt_member;
    for (int k = threadIdx.x; k < TILE * HN * GR; k += Cfg::THREADS) {
      const int cc = k / (HN * GR);
      const int rem = k - cc * HN * GR;
      int p = bx * TILE + cc;
      p = p < a.nx ? p : 0;
      int ps = p < a.NX / 2 ? p : p - a.NX;
      ps = ps < 0 ? -ps : ps;
      cp_async16(reinterpret_cast<char*>(smt) + ((size_t)cc * HN * GR + rem) * 16,
                 reinterpret_cast<const char*>(mtm) + ((size_t)ps * HN * GR + rem) * 16);
    }
    cp_async_commit();
  }
  unsigned char* hsm = reinterpret_cast<unsigned char*>(smt) + Cfg::TAB;
  hook.template prefetch<R, N, E, TILE, Cfg::THREADS>(hsm, a, bx, plane, member);
  C* base = a.field + (size_t)member * 5 * a.ntot + (size_t)plane * a.plane_stride +
            (valid ? xcol : 0) + (size_t)i * a.line_stride;
  const size_t step = (size_t)T * a.line_stride;
  C v[5][E];
  if constexpr (TMA) {
    // the five components through Cfg::TSTG staging buffers in the exchange
    // buffers' region (each [line element][TILE]); columns past the grid's
    // edge come in as zeros
    static_assert(sizeof(R) == 4 && TILE % 2 == 0, "tile loads: FP32, an even number of columns");
    constexpr int NSTG = Cfg::TSTG;
    __shared__ __align__(8) unsigned long long s_bar[NSTG];
    constexpr int RB = tma_rows<N>();
    constexpr unsigned BYTES = (unsigned)(TILE * N * sizeof(C));
    const int x0 = bx * TILE;
    const int mc = (a.mc0 + member) * 5;
    auto issue = [&](int c) {
      C* st = xb + (c % NSTG) * TILE * N;
      mbar_expect_tx(&s_bar[c % NSTG], BYTES);
#pragma unroll
      for (int b = 0; b < N / RB; ++b) {
        if (a.axis == 1) tma_load_4d(st + b * RB * TILE, tmap, &s_bar[c % NSTG], x0, b * RB, plane, mc + c);
        else tma_load_4d(st + b * RB * TILE, tmap, &s_bar[c % NSTG], x0, plane, b * RB, mc + c);
      }
    };
    if (threadIdx.x == 0) {
      for (int k = 0; k < NSTG; ++k) mbar_init(&s_bar[k], 1);
      mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int k = 0; k < NSTG; ++k) issue(k);
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      if (!mbar_wait(&s_bar[c % NSTG], (unsigned)((c / NSTG) & 1), kTmaWaitCycles) && a.err) atomicExch(a.err, 1);
      const C* st = xb + (c % NSTG) * TILE * N;
#pragma unroll
      for (int e = 0; e < E; ++e) v[c][e] = st[(i + T * e) * TILE + col];
      if (c + NSTG < 5) {
        __syncthreads();                // every thread has read the buffer
        if (threadIdx.x == 0) issue(c + NSTG);
      }
    }
  } else {
#pragma unroll
    for (int c = 0; c < 5; ++c)
#pragma unroll
      for (int e = 0; e < E; ++e)
        v[c][e] = valid ? ld_field<CG>(base + (size_t)c * a.ntot + e * step) : mkc((R)0, (R)0);
  }
  C* b0 = xb + col * Cfg::LP;
  const int bstride = TILE * Cfg::LP;
  if (a.mode & LP_FWD) fft_lines<R, N, E, -1, 5, Cfg::NB>(v, i, tw, b0, bstride);
  // thread i of column xcol holds line elements i + T e; the tile's
  // element offset of (c, e) is base - field + c ntot + e step
  hook.template after_fwd<R, N, E, Cfg::THREADS>(v, a, i, xcol, valid, plane, member, bx,
                                                  (size_t)(base - a.field), hsm);
  if (a.mode & LP_MIX) {
    const int pm = valid ? xcol : 0;   // idle threads of a ragged tile read mode 0
    if (stab) {
      cp_async_wait();
      __syncthreads();
      const int ps = pm < a.NX / 2 ? pm : pm - a.NX;
      const R* tcol = smt + (size_t)col * HN * MT_STRIDE;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int pos = i + T * e;
        const int qs = pos < N / 2 ? pos : pos - N;
        C p5[5] = {v[0][e], v[1][e], v[2][e], v[3][e], v[4][e]};
        const ModeEntry<R> m = load_mode_shared(tcol, qs < 0 ? -qs : qs);
        mix_entry<R>(p5, a, m, ps, qs, mkc(m.khr, m.khi));
#pragma unroll
        for (int c = 0; c < 5; ++c) v[c][e] = p5[c];
      }
    } else if (stabz) {
      cp_async_wait();
      __syncthreads();
      const int ps = pm < a.NX / 2 ? pm : pm - a.NX;
      const int qq = plane;
      const int qs = qq < a.NY / 2 ? qq : qq - a.NY;
      const ModeEntry<R> m = load_mode_shared(smt, col);
      const C kh = mkc(m.khr, m.khi);
      const C* skz = reinterpret_cast<const C*>(smt + TILE * MT_STRIDE);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int pos = i + T * e;
        C p5[5] = {v[0][e], v[1][e], v[2][e], v[3][e], v[4][e]};
        mix_entry<R>(p5, a, m, ps, qs, kinetic_z(kh, skz[pos]));
#pragma unroll
        for (int c = 0; c < 5; ++c) v[c][e] = p5[c];
      }
    }
  }
  hook.template after_mix<R, N, E>(v, a, valid, (size_t)(base - a.field));
  if (a.mode & LP_INV) fft_lines<R, N, E, +1, 5, Cfg::NB>(v, i, tw, b0, bstride);
  if constexpr (TMA) {
    // the five components out through the two exchange buffers: each is
    // written there, then stored by tensor copies (columns past the grid's
    // edge are not written); a buffer is written again once the copy that
    // read it is done
    constexpr int RB = tma_rows<N>();
    const int x0 = bx * TILE;
    const int mc = (a.mc0 + member) * 5;
    __syncthreads();                    // the exchanges' reads of the buffers are done
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      C* st = xb + (c & 1) * TILE * N;
      if (c >= 2) {
        if (threadIdx.x == 0) bulk_wait_read<1>();     // the copy of component c - 2 read the buffer
        __syncthreads();
      }
#pragma unroll
      for (int e = 0; e < E; ++e) st[(i + T * e) * TILE + col] = v[c][e];
      fence_proxy_async();
      __syncthreads();
      if (threadIdx.x == 0) {
#pragma unroll
        for (int b = 0; b < N / RB; ++b) {
          if (a.axis == 1) tma_store_4d(tmap, st + b * RB * TILE, x0, b * RB, plane, mc + c);
          else tma_store_4d(tmap, st + b * RB * TILE, x0, plane, b * RB, mc + c);
        }
        bulk_commit();
      }
    }
    if (threadIdx.x == 0) bulk_wait_all();
  } else if (valid) {
#pragma unroll
    for (int c = 0; c < 5; ++c)
#pragma unroll
      for (int e = 0; e < E; ++e) base[(size_t)c * a.ntot + e * step] = v[c][e];
  }
}

template <typename R, int N, int E, int G>
__global__ void __launch_bounds__(LCfg<R, N, E, G>::THREADS, LCfg<R, N, E, G>::MINB)
k_linepass(LPassArgs<R> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  linepass_body<R, N, E, G>(a, blockIdx.x, blockIdx.y, blockIdx.z, smem_raw);
}

// variant 4: the same pass with the tile loaded by tensor copies
template <typename R, int N, int E, int G>
__global__ void __launch_bounds__(LCfg<R, N, E, G>::THREADS, LCfg<R, N, E, G>::MINB)
k_linepass_tma(LPassArgs<R> a, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(128) unsigned char smem_tma[];    // tensor copies land 128-byte aligned
  linepass_body<R, N, E, G, false, true>(a, blockIdx.x, blockIdx.y, blockIdx.z, smem_tma, &tmap);
}

// ----------------------------------------------------------------------------
// observables (Sec. 2), FP64 sums
// ----------------------------------------------------------------------------
// term indices of the per-member sums
enum {
  OB_M0 = 0,     // 0..4 component masses
  OB_WX = 5, OB_WY = 6, OB_WZ = 7,
  OB_POT = 8, OB_INT = 9,
  OB_KX = 10, OB_LZX = 11, OB_SOCX = 12,
  OB_KY = 13, OB_LZY = 14, OB_SOCY = 15,
  OB_KZ = 16,
  OB_NT = 19      // (the z-line kernel also writes two unused slots after OB_KZ)
};

struct ObsArgsBase {
  long long ntot;
  int rows, ny;
  double x0, hx, y0, hy, z0, hz;
  double t;
  const MemberPrm* mp;   // [batch]
  double* partials;      // [member][nblocks][terms of the kernel]
  int nblocks;           // blocks per member
};

constexpr int OBX_NT = 13;   // terms written by k_obs_x  (OB_M0 .. OB_SOCX)
constexpr int OBL_NT = 3;    // terms written by k_obs_line (kin, lz, soc)

template <typename R>
struct ObsXArgs : ObsArgsBase {
  const cplx<R>* field;
  const TwE<R>* tw;
  R dnu;                 // pi/Lx / Nx (derivative factor with the 1/N of the forward transform)
  int NX;
};

template <typename R>
struct ObsLArgs : ObsArgsBase {
  const cplx<R>* field;
  const TwE<R>* tw;
  int nx;
  long long line_stride, plane_stride;
  int axis;              // 1: y lines, 2: z lines
  R dnu;                 // pi/L / N along the line axis
  int NL;                // line length
};

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Block reduction of NTERM sums; thread 0 writes them to out[0..NTERM-1].
template <int NTERM>
__device__ __forceinline__ void block_sums(double (&acc)[NTERM], double* out, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NTERM; ++k) {
    const double s = warp_sum(acc[k]);
    if (lane == 0) red[warp * NTERM + k] = s;
  }
  __syncthreads();
  if (threadIdx.x < NTERM) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w * NTERM + threadIdx.x];
    out[threadIdx.x] = s;
  }
}

// x-lines: pointwise terms and the x-derivative terms.
template <typename R, int N, int E>
__global__ void __launch_bounds__(XCfg<R, N, E>::THREADS)
k_obs_x(ObsXArgs<R> a) {
  typedef cplx<R> C;
  typedef XCfg<R, N, E> Cfg;
  constexpr int T = Cfg::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TwE<R>* tw = reinterpret_cast<TwE<R>*>(smem_raw);
  C* xb = reinterpret_cast<C*>(tw + N);
  __shared__ double red[32 * 10];
  const int g = threadIdx.x / T;
  const int i = threadIdx.x - g * T;
  for (int k = threadIdx.x; k < N; k += Cfg::THREADS) tw[k] = a.tw[k];
  const int row = blockIdx.x * Cfg::ROWS + g;
  const bool valid = row < a.rows;
  const C* base = a.field + (size_t)blockIdx.y * 5 * a.ntot + (size_t)(valid ? row : 0) * N + i;
  C v[5][E];
#pragma unroll
  for (int c = 0; c < 5; ++c)
#pragma unroll
    for (int e = 0; e < E; ++e)
      v[c][e] = valid ? base[(size_t)c * a.ntot + T * e] : mkc((R)0, (R)0);
  C* b0 = xb + g * Cfg::LP;
  const int bstride = Cfg::ROWS * Cfg::LP;
  fft_lines<R, N, E, -1, 5, Cfg::NB>(v, i, tw, b0, bstride);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int p = i + T * e;
    const int ps = p < N / 2 ? p : p - N;
    const R f = (R)ps * a.dnu;
#pragma unroll
    for (int c = 0; c < 5; ++c) v[c][e] = cscale(cmuli(v[c][e]), f);
  }
  fft_lines<R, N, E, +1, 5, Cfg::NB>(v, i, tw, b0, bstride);
  double acc[13];
#pragma unroll
  for (int k = 0; k < 13; ++k) acc[k] = 0.0;
  if (valid) {
    const MemberPrm& P = a.mp[blockIdx.y];
    const double co = cos(P.omega * a.t), si = sin(P.omega * a.t);
    const int ky = row % a.ny, kz = row / a.ny;
    const double y = a.y0 + ky * a.hy, z = a.z0 + kz * a.hz;
    const double s6h = 1.22474487139158904910, s6 = 2.44948974278317809820;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const double x = a.x0 + (i + T * e) * a.hx;
      double re[5], im[5], dr[5], di[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        const C u = base[(size_t)c * a.ntot + T * e];
        re[c] = (double)u.x; im[c] = (double)u.y;
        dr[c] = (double)v[c][e].x; di[c] = (double)v[c][e].y;
      }
      double m[5], rho = 0.0, kin = 0.0, lzi = 0.0;
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        m[c] = re[c] * re[c] + im[c] * im[c];
        rho += m[c];
        kin += dr[c] * dr[c] + di[c] * di[c];
        lzi += re[c] * di[c] - im[c] * dr[c];       // Im(conj(phi) dphi)
        acc[c] += m[c];
      }
      const double xr = co * x + si * y, yr = co * y - si * x;
      acc[OB_WX] += xr * xr * rho;
      acc[OB_WY] += yr * yr * rho;
      acc[OB_WZ] += z * z * rho;
      acc[OB_POT] += (P.gx2h * xr * xr + P.gy2h * yr * yr + P.gz2h * z * z) * rho;
      const double Fz = 2.0 * (m[0] - m[4]) + m[1] - m[3];
      // F_+ = 2(conj(p2)p1 + conj(m1)m2) + sqrt6 (conj(p1)p0 + conj(p0)m1)
      const double fpr = 2.0 * (re[0] * re[1] + im[0] * im[1] + re[3] * re[4] + im[3] * im[4]) +
                         s6 * (re[1] * re[2] + im[1] * im[2] + re[2] * re[3] + im[2] * im[3]);
      const double fpi = 2.0 * (re[0] * im[1] - im[0] * re[1] + re[3] * im[4] - im[3] * re[4]) +
                         s6 * (re[1] * im[2] - im[1] * re[2] + re[2] * im[3] - im[2] * re[3]);
      const double aR = 2.0 * (re[0] * re[4] - im[0] * im[4]) - 2.0 * (re[1] * re[3] - im[1] * im[3]) +
                        re[2] * re[2] - im[2] * im[2];
      const double aI = 2.0 * (re[0] * im[4] + im[0] * re[4]) - 2.0 * (re[1] * im[3] + im[1] * re[3]) +
                        2.0 * re[2] * im[2];
      acc[OB_INT] += 0.5 * P.c0 * rho * rho + 0.5 * P.c1 * (fpr * fpr + fpi * fpi + Fz * Fz) +
                     0.5 * P.c2 * (aR * aR + aI * aI) * 0.2;
      acc[OB_KX] += 0.5 * kin;
      acc[OB_LZX] += -y * lzi;
      // SOC, x part: sum_i coef_i Re[-conj(phi_i) d phi_{i+1} + conj(phi_{i+1}) d phi_i]
      const double coef[4] = {1.0, s6h, s6h, 1.0};
      double soc = 0.0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const double t1 = re[k] * dr[k + 1] + im[k] * di[k + 1];
        const double t2 = re[k + 1] * dr[k] + im[k + 1] * di[k];
        soc += coef[k] * (t2 - t1);
      }
      acc[OB_SOCX] += soc;
    }
  }
  double* out = a.partials + ((size_t)blockIdx.y * a.nblocks + blockIdx.x) * OBX_NT;
  block_sums<OBX_NT>(acc, out, red);
}

// strided lines: derivative terms along y (or z).
template <typename R, int N, int E>
__global__ void __launch_bounds__(LCfg<R, N, E>::THREADS)
k_obs_line(ObsLArgs<R> a) {
  typedef cplx<R> C;
  typedef LCfg<R, N, E> Cfg;
  constexpr int T = Cfg::T;
  constexpr int TILE = Cfg::TILE;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TwE<R>* tw = reinterpret_cast<TwE<R>*>(smem_raw);
  C* xb = reinterpret_cast<C*>(tw + N);
  __shared__ double red[32 * 3];
  const int col = threadIdx.x % TILE;
  const int i = threadIdx.x / TILE;
  for (int k = threadIdx.x; k < N; k += Cfg::THREADS) tw[k] = a.tw[k];
  const int xcol = blockIdx.x * TILE + col;
  const bool valid = xcol < a.nx;
  const C* base = a.field + (size_t)blockIdx.z * 5 * a.ntot + (size_t)blockIdx.y * a.plane_stride +
                  (valid ? xcol : 0) + (size_t)i * a.line_stride;
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
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int p = i + T * e;
    const int ps = p < N / 2 ? p : p - N;
    const R f = (R)ps * a.dnu;
#pragma unroll
    for (int c = 0; c < 5; ++c) v[c][e] = cscale(cmuli(v[c][e]), f);
  }
  fft_lines<R, N, E, +1, 5, Cfg::NB>(v, i, tw, b0, bstride);
  double acc[3] = {0.0, 0.0, 0.0};
  if (valid) {
    const double x = a.x0 + xcol * a.hx;
    const double s6h = 1.22474487139158904910;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      double re[5], im[5], dr[5], di[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        const C u = base[(size_t)c * a.ntot + e * step];
        re[c] = (double)u.x; im[c] = (double)u.y;
        dr[c] = (double)v[c][e].x; di[c] = (double)v[c][e].y;
      }
      double kin = 0.0, lzi = 0.0;
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        kin += dr[c] * dr[c] + di[c] * di[c];
        lzi += re[c] * di[c] - im[c] * dr[c];
      }
      acc[0] += 0.5 * kin;
      if (a.axis == 1) {
        acc[1] += x * lzi;
        // SOC, y part: sum_i coef_i Re[i conj(phi_i) d phi_{i+1} + i conj(phi_{i+1}) d phi_i]
        const double coef[4] = {1.0, s6h, s6h, 1.0};
        double soc = 0.0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          // Re(i conj(a) b) = -(Im(conj(a) b)) = -(ar*bi - ai*br)
          const double t1 = re[k] * di[k + 1] - im[k] * dr[k + 1];
          const double t2 = re[k + 1] * di[k] - im[k + 1] * dr[k];
          soc -= coef[k] * (t1 + t2);
        }
        acc[2] += soc;
      }
    }
  }
  double* out = a.partials +
                ((size_t)blockIdx.z * a.nblocks + (size_t)blockIdx.y * gridDim.x + blockIdx.x) * OBL_NT;
  block_sums<OBL_NT>(acc, out, red);
}

// Fixed-order sum of per-block partials: out[m*ostride + ooff + k] =
// sum_b part[(m*nblocks + b)*nterm + k].  One thread per (member, term).
static __global__ void k_reduce_partials(const double* part, int nblocks, int nterm, int members,
                                  double* out, int ostride, int ooff) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= members * nterm) return;
  const int m = id / nterm, k = id - m * nterm;
  const double* p = part + (size_t)m * nblocks * nterm + k;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += p[(size_t)b * nterm];
  out[(size_t)m * ostride + ooff + k] = s;
}

}  // namespace sgp
