// sgp_adjoint.cuh -- argument blocks and launchers of the adjoint kernels.
//
// Objective gradients are propagated backwards through the substeps of the
// composition (Sec. 3.3).  Both flows are exact Hamiltonian flows that are
// reversed by negating their step (the linear flow is unitary; the
// nonlinear flow of Eq. (solution2) conserves rho, F and |A00|), which gives
// the vector-Jacobian products used here.  With g = dJ/dRe + i dJ/dIm at a
// substep's output Phi_out:
//   linear flow L(d):     g_in = L(-d) g
//   nonlinear flow N(d):  g_in = -i DN_{-d}(Phi_out)[i g]
// (the flow is symplectic for the form Im<u, v>, so the transpose of its
// Jacobian is -i DN^{-1} i).  Parameter derivatives:
//   N(d): the four parts of the local Hamiltonian (c0 rho^2/2, c1 |F|^2/2,
//         c2 |A00|^2/2 and the trap) commute, so dN/dp = d X_p(Phi_out) with
//         X_c0 = -i rho psi, X_c1 = -i (F.f) psi, X_c2 = -i A00 A conj(psi),
//         X_Omega = -i t (gx^2 - gy^2) x_r y_r psi (V depends on Omega t);
//   L(d): per mode exp(i a.f), a = d (-gamma nu_y, gamma nu_x, -Omega), so
//         dL/dp Phi = inverse[i (w.f) (L Phi)^] with the left-trivialised
//         derivative w = a^(a^.da) + (sin|a|/|a|)(da - a^(a^.da))
//                        - ((1 - cos|a|)/|a|)(a^ x da).
#pragma once
#include <cuda_runtime.h>

#include "sgp_kernels.cuh"

namespace sgp {

// slots of the per-member parameter gradient (dJ/dOmega, dgamma, dc0, dc1, dc2)
enum { GP_OMEGA = 0, GP_GAMMA = 1, GP_C0 = 2, GP_C1 = 3, GP_C2 = 4, GP_N = 5 };
// terms of the nonlinear and linear adjoint partial sums
enum { NLA_OMEGA = 0, NLA_C0, NLA_C1, NLA_C2, NLA_NT };
enum { LPA_OMEGA = 0, LPA_GAMMA, LPA_NT };

// ----------------------------------------------------------------------------
// pointwise and per-mode pieces
// ----------------------------------------------------------------------------
// <a, b> = sum conj(a_k) b_k over the five components
template <typename C>
__device__ __forceinline__ C inner5(const C (&a)[5], const C (&b)[5]) {
  C s = cconjmul(a[0], b[0]);
#pragma unroll
  for (int k = 1; k < 5; ++k) s = cadd(s, cconjmul(a[k], b[k]));
  return s;
}

// (w.f) v for a real vector w (spin-2 matrices, components l = 2..-2):
// rows 2 wz v0 + w- v1, w+ v0 + wz v1 + (r6/2) w- v2, (r6/2)(w+ v1 + w- v3),
// (r6/2) w+ v2 - wz v3 + w- v4, w+ v3 - 2 wz v4  with w+- = wx +- i wy.
template <typename R>
__device__ __forceinline__ void spin_dot5(R wx, R wy, R wz, const cplx<R> (&v)[5],
                                          cplx<R> (&o)[5]) {
  typedef cplx<R> C;
  const R r6h = (R)1.22474487139158904910;
  const C wp = mkc(wx, wy), wm = mkc(wx, -wy);
  o[0] = cadd(cscale(v[0], (R)2 * wz), cmul(wm, v[1]));
  o[1] = cadd(cadd(cmul(wp, v[0]), cscale(v[1], wz)), cscale(cmul(wm, v[2]), r6h));
  o[2] = cscale(cadd(cmul(wp, v[1]), cmul(wm, v[3])), r6h);
  o[3] = csub(cadd(cscale(cmul(wp, v[2]), r6h), cmul(wm, v[4])), cscale(v[3], wz));
  o[4] = csub(cmul(wp, v[3]), cscale(v[4], (R)2 * wz));
}

// sqrt5 A conj(v) = (conj v_-2, -conj v_-1, conj v_0, -conj v_1, conj v_2)
template <typename C>
__device__ __forceinline__ void acon5(const C (&v)[5], C (&o)[5]) {
  o[0] = cconj(v[4]);
  o[1] = cneg(cconj(v[3]));
  o[2] = cconj(v[2]);
  o[3] = cneg(cconj(v[1]));
  o[4] = cconj(v[0]);
}

// (x cos x - sin x) / x^3: the series -1/3 + x^2/30 - x^4/840 + x^6/45360
// - x^8/3991680 below |x| = 1/2 (remainder < 1e-12 relative), else direct.
template <typename R>
__device__ __forceinline__ R sinc_slope(R x, R sx, R cx) {
  const R x2 = x * x;
  if (x2 < (R)0.25) {
    R p = (R)(-1.0 / 3991680.0);
    p = fma(p, x2, (R)(1.0 / 45360.0));
    p = fma(p, x2, (R)(-1.0 / 840.0));
    p = fma(p, x2, (R)(1.0 / 30.0));
    return fma(p, x2, (R)(-1.0 / 3.0));
  }
  return (x * cx - sx) / (x2 * x);
}

template <typename R>
__device__ __forceinline__ void apply_spin(const cplx<R> (&v)[5], const SpinRot<R>& sr, bool rot,
                                           cplx<R> (&o)[5]) {
  if (rot) {
    cplx<R> e[5];
    spin2_increment<R>(v, sr.am1, sr.bhat, sr.cpm1, sr.sp, e);
#pragma unroll
    for (int k = 0; k < 5; ++k) o[k] = cadd(v[k], e[k]);
  } else {
#pragma unroll
    for (int k = 0; k < 5; ++k) o[k] = v[k];
  }
}

// Member constants of the nonlinear adjoint in the field precision: the
// substep size d, c0 + c2/5, c1, c2, and t (gx^2 - gy^2) at the substep's
// time t (the factor of the Omega term).
template <typename R>
struct NLAdjPrm {
  R d, c0p, c1, c2, tdgg;
};

// Nonlinear flow at one point: g <- -i DN_{-d}(Phi_out)[i g] with psi =
// Phi_out there, and the parameter terms d Re<g, X_p(Phi_out)> added to acc
// (slots NLA_*; each term formed in the field precision, the sums kept in
// FP64).  N = (phase) o (spin rotation) o (singlet rotation) as in
// Eq. (solution2); the tangent is carried through the same three factors of
// N_{-d} at Phi_out.  rho, F and |A00| are the same at every stage
// (conserved), so their tangents are formed once from the input tangent.
// V: the trap at the mapped point; xy = xr yr, the mapped coordinates'
// product.
template <typename R>
__device__ __forceinline__ void nl_adjoint_point(const cplx<R> (&psi)[5], cplx<R> (&g)[5], R V, R xy,
                                                 const NLAdjPrm<R>& q, double (&acc)[NLA_NT]) {
  typedef cplx<R> C;
  const R r6 = (R)2.44948974278317809820;
  const R rs5 = (R)0.44721359549995793928;
  const R d = q.d;
  const R dl = -d;                          // the inverse flow's step
  const R c0p = q.c0p, c1 = q.c1, c2 = q.c2;
  // local densities of Phi_out (Sec. 1)
  const R n0 = cabs2(psi[0]), n1 = cabs2(psi[1]), n2 = cabs2(psi[2]);
  const R n3 = cabs2(psi[3]), n4 = cabs2(psi[4]);
  const R rho = n0 + n1 + n2 + n3 + n4;
  const R Fz = (R)2 * (n0 - n4) + n1 - n3;
  C Fp = cscale(cadd(cconjmul(psi[0], psi[1]), cconjmul(psi[3], psi[4])), (R)2);
  Fp = cadd(Fp, cscale(cadd(cconjmul(psi[1], psi[2]), cconjmul(psi[2], psi[3])), r6));
  C A00 = csub(cmul(psi[0], psi[4]), cmul(psi[1], psi[3]));
  A00 = cscale(cadd(cscale(A00, (R)2), cmul(psi[2], psi[2])), rs5);
  C ac[5];
  acon5(psi, ac);
  // parameter terms d Re<g, X_p(Phi_out)> = d Im<g, i X_p>
  {
    C Fpsi[5];
    spin_dot5<R>(Fp.x, Fp.y, Fz, psi, Fpsi);
    const C ip = inner5(g, psi);
    const C ia = inner5(g, ac);
    acc[NLA_C0] += (double)(d * rho * ip.y);
    acc[NLA_C1] += (double)(d * inner5(g, Fpsi).y);
    acc[NLA_C2] += (double)(d * cmul(A00, ia).y * rs5);
    acc[NLA_OMEGA] += (double)(d * q.tdgg * xy * ip.y);
  }
  // tangent v = i g at Phi_out
  C v[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) v[k] = cmuli(g[k]);
  const R drho = (R)2 * inner5(psi, v).x;
  R dFz = (R)0;
  {
    const R mz[5] = {(R)2, (R)1, (R)0, (R)-1, (R)-2};
#pragma unroll
    for (int k = 0; k < 5; ++k) dFz += mz[k] * cconjmul(psi[k], v[k]).x;
    dFz *= (R)2;
  }
  // dF+ = <v, f+ psi> + <psi, f+ v>;  f+ u = (2 u1, r6 u2, r6 u3, 2 u4, 0)
  C dFp = cadd(cconjmul(v[0], cscale(psi[1], (R)2)), cconjmul(psi[0], cscale(v[1], (R)2)));
  dFp = cadd(dFp, cscale(cadd(cconjmul(v[1], psi[2]), cconjmul(psi[1], v[2])), r6));
  dFp = cadd(dFp, cscale(cadd(cconjmul(v[2], psi[3]), cconjmul(psi[2], v[3])), r6));
  dFp = cadd(dFp, cscale(cadd(cconjmul(v[3], psi[4]), cconjmul(psi[3], v[4])), (R)2));
  // dA00 = (2/sqrt5)(v0 m2 + p2 v4 - v1 m1 - p1 v3 + p0 v2) in component order
  C dA = cadd(cmul(v[0], psi[4]), cmul(psi[0], v[4]));
  dA = csub(dA, cadd(cmul(v[1], psi[3]), cmul(psi[1], v[3])));
  dA = cscale(cadd(dA, cmul(psi[2], v[2])), (R)2 * rs5);
  // (1) singlet rotation over dl
  const R kap = c2 * dl;
  const R S2 = rho * rho * (R)0.04 - cabs2(A00) * (R)0.2;
  const R S = S2 > (R)0 ? sqrt(S2) : (R)0;
  const R xs = kap * S;
  R sx, cx;
  sincos_r(xs, &sx, &cx);
  const R sinc = S > (R)0 ? sx / S : kap;
  const R gsl = sinc_slope<R>(xs, sx, cx);
  const R SdS = rho * drho * (R)0.04 - cconjmul(A00, dA).x * (R)0.2;
  const R dC = -kap * sinc * SdS;
  const R dsinc = kap * kap * kap * gsl * SdS;
  C av[5];
  acon5(v, av);
  C b[5], db[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const C W = csub(cscale(psi[k], rho * (R)0.2), cscale(cmul(A00, ac[k]), rs5));
    C dW = cadd(cscale(psi[k], drho * (R)0.2), cscale(v[k], rho * (R)0.2));
    dW = csub(dW, cscale(cadd(cmul(dA, ac[k]), cmul(A00, av[k])), rs5));
    b[k] = cadd(cscale(psi[k], cx), cmuli(cscale(W, sinc)));
    db[k] = cadd(cadd(cscale(psi[k], dC), cscale(v[k], cx)),
                 cmuli(cadd(cscale(W, dsinc), cscale(dW, sinc))));
  }
  // (2) spin rotation over dl: U = exp(i a.f), a = -c1 dl F; dU = U i (w.f),
  //     w = Fh(Fh.da) + (sin k/k)(da - Fh(Fh.da)) - ((1 - cos k)/k)(Fh x da),
  //     k = c1 dl |F|, da = -c1 dl dF
  SpinRot<R> sr;
  const bool rot = spin_rotation<R>(Fz, Fp, c1, dl, sr);
  const R dax = -c1 * dl * dFp.x, day = -c1 * dl * dFp.y, daz = -c1 * dl * dFz;
  R wx = dax, wy = day, wz = daz;
  if (rot) {
    const R fx = Fp.x * sr.rFn, fy = Fp.y * sr.rFn, fz = Fz * sr.rFn;
    const R hk = (R)0.5 * c1 * dl * sr.Fn;
    const R ratio = hk != (R)0 ? sr.sh / hk : (R)1;
    const R sk = ratio * sr.ch;          // sin k / k
    const R ck = sr.sh * ratio;          // (1 - cos k) / k
    const R fd = fx * dax + fy * day + fz * daz;
    const R px = fx * fd, py = fy * fd, pz = fz * fd;
    wx = px + sk * (dax - px) - ck * (fy * daz - fz * day);
    wy = py + sk * (day - py) - ck * (fz * dax - fx * daz);
    wz = pz + sk * (daz - pz) - ck * (fx * day - fy * dax);
  }
  C wb[5], w[5];
  spin_dot5<R>(wx, wy, wz, b, wb);
#pragma unroll
  for (int k = 0; k < 5; ++k) w[k] = cadd(db[k], cmuli(wb[k]));
  C cst[5], dc[5];
  apply_spin<R>(b, sr, rot, cst);
  apply_spin<R>(w, sr, rot, dc);
  // (3) scalar phase exp(-i th), th = dl (V + c0' rho); g_in = -i v3
  R sth, cth;
  sincos_r(dl * (V + c0p * rho), &sth, &cth);
  const C ph = mkc(cth, -sth);
  const R qq = dl * c0p * drho;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const C v3 = cmul(ph, csub(dc[k], cmuli(cscale(cst[k], qq))));
    g[k] = cmulmi(v3);
  }
}

// Linear flow at one mode (signed indices ps, qs of the x and y wavenumbers
// nu = (pxl ps, pyl qs), pxl = pi/Lx, pyl = pi/Ly): the derivatives in
// Omega and gamma, -Re<g^, i (w.f) S^>, added to acc[LPA_*] (each formed in
// the field precision, the sums kept in FP64; the caller scales the sums).
// gv, sv: the mode of the transforms of g and of Phi_out.
template <typename R>
__device__ __forceinline__ void lin_param_mode(const cplx<R> (&gv)[5], const cplx<R> (&sv)[5], int ps, int qs,
                                               R gamma, R omega, R dR, R pxl, R pyl, double (&acc)[LPA_NT]) {
  typedef cplx<R> C;
  const R r6R = (R)2.44948974278317809820;
  // P+ = <g, f+ s>, P- = <g, f- s>, Pz = <g, fz s> in the field precision
  const C Pp = cadd(cscale(cadd(cconjmul(gv[0], sv[1]), cconjmul(gv[3], sv[4])), (R)2),
                    cscale(cadd(cconjmul(gv[1], sv[2]), cconjmul(gv[2], sv[3])), r6R));
  const C Pm = cadd(cscale(cadd(cconjmul(gv[1], sv[0]), cconjmul(gv[4], sv[3])), (R)2),
                    cscale(cadd(cconjmul(gv[2], sv[1]), cconjmul(gv[3], sv[2])), r6R));
  const C Pz = cadd(cscale(csub(cconjmul(gv[0], sv[0]), cconjmul(gv[4], sv[4])), (R)2),
                    csub(cconjmul(gv[1], sv[1]), cconjmul(gv[3], sv[3])));
  // Im<g, (w.f) s> = wx Im(P+ + P-)/2 - wy Re(P+ - P-)/2 + wz Im Pz
  const R kx = (R)0.5 * (Pp.y + Pm.y);
  const R ky = (R)-0.5 * (Pp.x - Pm.x);
  const R kz = Pz.y;
  const R nxR = pxl * (R)ps, nyR = pyl * (R)qs;
  const R ax = dR * (-gamma * nyR), ay = dR * (gamma * nxR), az = dR * (-omega);
  const R th2 = ax * ax + ay * ay + az * az;
  const R das[2][3] = {{(R)0, (R)0, -dR}, {-dR * nyR, dR * nxR, (R)0}};
  R sk = (R)1, ck = (R)0, hx = (R)0, hy = (R)0, hz = (R)0;
  if (th2 > (R)0) {
    const R ith = rsqrt_r(th2);
    const R th = th2 * ith;
    hx = ax * ith;
    hy = ay * ith;
    hz = az * ith;
    R sh, ch;
    sincos_small((R)0.5 * th, &sh, &ch);   // series below 0.6 rad (FP32)
    sk = (R)2 * sh * ch * ith;             // sin th / th
    ck = (R)2 * sh * sh * ith;             // (1 - cos th) / th
  }
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const R dx = das[p][0], dy = das[p][1], dz = das[p][2];
    const R fd = hx * dx + hy * dy + hz * dz;
    const R px = hx * fd, py = hy * fd, pz = hz * fd;
    const R wx = px + sk * (dx - px) - ck * (hy * dz - hz * dy);
    const R wy = py + sk * (dy - py) - ck * (hz * dx - hx * dz);
    const R wz = pz + sk * (dz - pz) - ck * (hx * dy - hy * dx);
    acc[p] -= (double)(wx * kx + wy * ky + wz * kz);
  }
}

// ----------------------------------------------------------------------------
// the passes of the recomputation and of the adjoint sweep
// ----------------------------------------------------------------------------
// x-pass of the adjoint sweep (k_xadj): rows of g, optional inverse
// x-transform (XP_INV), the nonlinear adjoint at every point with Phi_out
// (phi, physical space), optional forward x-transform (XP_FWD).  Each CTA
// adds its parameter terms to its own row of the partials.
template <typename R>
struct XAdjArgs {
  cplx<R>* g;               // [member][5][ntot]
  const cplx<R>* phi;       // [member][5][ntot]: the substep's output state
  const TwE<R>* tw;         // x twiddles (default radix plan)
  long long ntot;
  int rows, ny;
  int mode;                 // XP_INV | XP_FWD
  R x0, hx, y0, hy, z0, hz;  // coordinates x_j = x0 + j hx as in the x-pass
  double delta;             // forward substep size
  const double* t_base;     // the substep's time is *t_base + t_off
  double t_off;
  const MemberPrm* mp;
  double* partials;         // [member][prows][GP_N]; the x-pass CTAs own rows 0..
  int prows;
};

// Hooks of the line passes of a gradient.  In the sweep (spec set) the
// Omega and gamma terms of every mode of the tile, taken after the forward
// transform, go to the CTA's row prow0 + plane * tiles + tile of the
// partials; spec is the transform of Phi_out at the same element offsets
// as the field, scale the factor that makes the product of the two
// transforms a sum over the grid.  In the recomputation (tap set) the tile
// is copied to tap after the mix: the transform of the linear substep's
// output divided by the transform length.
template <typename R>
struct AdjHook {
  const cplx<R>* spec;
  cplx<R>* tap;
  const MemberPrm* mp;
  double* partials;
  int prows, prow0, tiles;
  double Lx, Ly, delta, scale;
  // bytes of shared memory the hook stages: the tile of spec
  template <typename RR, int N, int TILE>
  static constexpr size_t smem_bytes() { return (size_t)5 * N * TILE * sizeof(cplx<RR>); }
  // the tile of spec ([component][line element][column]) to shared memory
  // by asynchronous copies, issued before the field loads
  template <typename RR, int N, int E, int TILE, int THREADS>
  __device__ __forceinline__ void prefetch(unsigned char* hsm, const LPassArgs<RR>& a, int bx, int plane,
                                           int member) const {
    typedef cplx<RR> C;
    if (!spec) return;
    const C* src = spec + (size_t)member * 5 * a.ntot + (size_t)plane * a.plane_stride + (size_t)bx * TILE;
    C* dst = reinterpret_cast<C*>(hsm);
    for (int k = threadIdx.x; k < 5 * N * TILE; k += THREADS) {
      const int cl = k % TILE, ln = (k / TILE) % N, c = k / (TILE * N);
      if (bx * TILE + cl >= a.nx) continue;
      const C* from = src + (size_t)c * a.ntot + (size_t)ln * a.line_stride + cl;
      if constexpr (sizeof(C) == 16) cp_async16(dst + k, from);
      else cp_async8(dst + k, from);
    }
    cp_async_commit();
  }
  template <typename RR, int N, int E, int THREADS>
  __device__ __forceinline__ void after_fwd(const cplx<RR> (&v)[5][E], const LPassArgs<RR>& a, int i, int xcol,
                                            bool valid, int plane, int member, int bx, size_t,
                                            const unsigned char* hsm) const {
    typedef cplx<RR> C;
    constexpr int T = N / E;
    constexpr int TILE = THREADS / T;
    constexpr double kPi = 3.14159265358979323846;
    if (!spec) return;                 // the same for every thread of the launch
    __shared__ double red[(THREADS + 31) / 32 * LPA_NT];
    cp_async_wait();
    __syncthreads();                   // the tile of spec is in shared memory
    const MemberPrm& P = mp[member];
    double acc[LPA_NT] = {0.0, 0.0};
    if (valid) {
      const RR pxl = (RR)(kPi / Lx), pyl = (RR)(kPi / Ly);
      const RR gam = (RR)P.gamma, om = (RR)P.omega, dR = (RR)delta;
      const int ps = xcol < a.NX / 2 ? xcol : xcol - a.NX;
      const C* sp = reinterpret_cast<const C*>(hsm) + (xcol - bx * TILE);
#pragma unroll 1
      for (int e = 0; e < E; ++e) {
        // the mode's y index: the line element (y lines) or the plane (z lines)
        const int ln = i + T * e;
        const int q = a.axis == 1 ? ln : plane;
        const int qs = q < a.NY / 2 ? q : q - a.NY;
        C gv[5], sv[5];
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          gv[c] = v[c][e];
          sv[c] = sp[((size_t)c * N + ln) * TILE];
        }
        lin_param_mode<RR>(gv, sv, ps, qs, gam, om, dR, pxl, pyl, acc);
      }
      acc[0] *= scale;
      acc[1] *= scale;
    }
    double out[LPA_NT];
    block_sums<LPA_NT>(acc, out, red);
    if (threadIdx.x < LPA_NT) {
      double* row = partials + ((size_t)member * prows + prow0 + (size_t)plane * tiles + bx) * GP_N;
      row[threadIdx.x == 0 ? GP_OMEGA : GP_GAMMA] += out[threadIdx.x];
    }
  }
  template <typename RR, int N, int E>
  __device__ __forceinline__ void after_mix(const cplx<RR> (&v)[5][E], const LPassArgs<RR>& a, bool valid,
                                            size_t off) const {
    constexpr int T = N / E;
    if (!tap || !valid) return;
    cplx<RR>* tp = reinterpret_cast<cplx<RR>*>(tap) + off;
    const size_t step = (size_t)T * a.line_stride;
#pragma unroll
    for (int c = 0; c < 5; ++c)
#pragma unroll
      for (int e = 0; e < E; ++e) tp[(size_t)c * a.ntot + e * step] = v[c][e];
  }
};

// Launchers (sgp_adjoint.cu, one unit per precision), all at fixed
// geometries: the adjoint x-pass; the x-pass that also copies the rows
// after the nonlinear flow to a.tap (x-pass geometry 2); the line pass
// with the hooks (line-pass geometry 2); the CTA counts that size the
// partials.
template <typename R>
cudaError_t launch_xadj(int N, const XAdjArgs<R>& a, int members, cudaStream_t s);
template <typename R>
cudaError_t launch_xpass_tap(int N, const XPassArgs<R>& a, int members, cudaStream_t s);
template <typename R>
cudaError_t launch_linepass_adj(int N, const LPassArgs<R>& a, const AdjHook<R>& h, int planes, int members,
                                cudaStream_t s);
template <typename R>
int xadj_ctas(int N, int rows);                 // CTAs per member of launch_xadj
template <typename R>
int linepass_adj_tiles(int N, int nx);          // tiles per plane of launch_linepass_adj
// dp[m][k] = sum over rows of part[m][row][k], k < GP_N (fixed order)
cudaError_t launch_reduce_params(const double* part, int nrows, int members, double* dp,
                                 cudaStream_t s);

}  // namespace sgp
