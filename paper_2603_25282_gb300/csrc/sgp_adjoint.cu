// sgp_adjoint.cu -- adjoint kernels of the compact splitting propagator:
// the pointwise vector-Jacobian product of the exact nonlinear flow with its
// parameter derivatives, and the per-mode parameter derivatives of the
// linear flow.  The state VJP of the linear flow is the linear flow over -d
// (the forward pass kernels).  Formulas: sgp_adjoint.cuh.
#include "sgp_adjoint.cuh"

namespace sgp {
namespace {

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

// Block sums of acc[0..nterm) added to row[slot[k]] (the block's own row of
// the partials, so no two blocks write the same word and the order of the
// additions is fixed).
__device__ __forceinline__ void block_accumulate(double (&acc)[NLA_NT], int nterm, const int4 slot,
                                                 double* row) {
  __shared__ double red[kAdjThreads / 32][NLA_NT];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = 0; k < nterm; ++k) {
    const double s = warp_sum(acc[k]);
    if (lane == 0) red[wid][k] = s;
  }
  __syncthreads();
  if (threadIdx.x < nterm) {
    double s = 0.0;
    for (int w = 0; w < kAdjThreads / 32; ++w) s += red[w][threadIdx.x];
    const int k = threadIdx.x;
    const int sl = k == 0 ? slot.x : (k == 1 ? slot.y : (k == 2 ? slot.z : slot.w));
    row[sl] += s;
  }
}

// ----------------------------------------------------------------------------
// nonlinear flow: g <- -i DN_{-d}(Phi_out)[i g], plus the parameter terms
// ----------------------------------------------------------------------------
// N = (phase) o (spin rotation) o (singlet rotation) as in Eq. (solution2);
// the tangent is carried through the same three factors of N_{-d} at
// Phi_out.  rho, F and |A00| are the same at every stage (conserved), so
// their tangents are formed once from the input tangent.
template <typename R>
__global__ void __launch_bounds__(kAdjThreads) k_nl_adjoint(NLAdjArgs<R> a) {
  typedef cplx<R> C;
  const int m = blockIdx.y;
  const MemberPrm& P = a.mp[m];
  __shared__ double s_rot[3];
  if (threadIdx.x == 0) {
    const double t = *a.t_base + a.t_off;
    sincos(P.omega * t, &s_rot[1], &s_rot[0]);
    s_rot[2] = t;
  }
  __syncthreads();
  const double co = s_rot[0], si = s_rot[1], tsub = s_rot[2];
  const R r6 = (R)2.44948974278317809820;
  const R rs5 = (R)0.44721359549995793928;
  const R d = (R)a.delta;
  const R dl = -d;                          // the inverse flow's step
  const R c0p = (R)(P.c0 + P.c2 / 5.0), c1 = (R)P.c1, c2 = (R)P.c2;
  const double dgg = 2.0 * (P.gx2h - P.gy2h);
  double acc[NLA_NT] = {0.0, 0.0, 0.0, 0.0};
  C* gbase = a.g + (size_t)m * 5 * a.ntot;
  const C* pbase = a.phi + (size_t)m * 5 * a.ntot;
  const long long nxy = (long long)a.nx * a.ny;
  for (long long id = (long long)blockIdx.x * kAdjThreads + threadIdx.x; id < a.ntot;
       id += (long long)a.nblocks * kAdjThreads) {
    const long long iz = id / nxy;
    const long long rem = id - iz * nxy;
    const int iy = (int)(rem / a.nx), ix = (int)(rem - (long long)iy * a.nx);
    const double x = a.x0 + ix * a.hx, y = a.y0 + iy * a.hy, z = a.z0 + iz * a.hz;
    const double xr = co * x + si * y, yr = co * y - si * x;
    const R V = (R)(P.gx2h * xr * xr + P.gy2h * yr * yr + P.gz2h * z * z);
    C psi[5], g[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      psi[k] = pbase[(size_t)k * a.ntot + id];
      g[k] = gbase[(size_t)k * a.ntot + id];
    }
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
      const double ipi = (double)ip.y;
      acc[NLA_C0] += (double)d * (double)rho * ipi;
      acc[NLA_C1] += (double)d * (double)inner5(g, Fpsi).y;
      acc[NLA_C2] += (double)d * (double)cmul(A00, ia).y * (double)rs5;
      acc[NLA_OMEGA] += (double)d * tsub * dgg * xr * yr * ipi;
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
    const R q = dl * c0p * drho;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const C v3 = cmul(ph, csub(dc[k], cmuli(cscale(cst[k], q))));
      gbase[(size_t)k * a.ntot + id] = cmulmi(v3);
    }
  }
  block_accumulate(acc, NLA_NT, make_int4(GP_OMEGA, GP_C0, GP_C1, GP_C2),
                   a.partials + ((size_t)m * a.nblocks + blockIdx.x) * GP_N);
}

// ----------------------------------------------------------------------------
// linear flow: per-mode derivative in Omega and gamma
// ----------------------------------------------------------------------------
// Re<g^, i (w.f) S^> summed over the modes of the unnormalised transforms,
// times 1/(NX NY [NZ]) (Parseval with the forward 1/N of Sec. 3.1).
template <typename R>
__global__ void __launch_bounds__(kAdjThreads) k_lin_param(LinParArgs<R> a) {
  typedef cplx<R> C;
  const int m = blockIdx.y;
  const MemberPrm& P = a.mp[m];
  const double r6 = 2.44948974278317809820;
  const double kPi = 3.14159265358979323846;
  double acc[NLA_NT] = {0.0, 0.0, 0.0, 0.0};
  const C* gb = a.g + (size_t)m * 5 * a.ntot;
  const C* sb = a.s + (size_t)m * 5 * a.ntot;
  for (long long id = (long long)blockIdx.x * kAdjThreads + threadIdx.x; id < a.ntot;
       id += (long long)a.nblocks * kAdjThreads) {
    const int ix = (int)(id % a.NX);
    const int iy = (int)((id / a.NX) % a.NY);
    const int ps = ix < a.NX / 2 ? ix : ix - a.NX;
    const int qs = iy < a.NY / 2 ? iy : iy - a.NY;
    C gv[5], sv[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      gv[k] = gb[(size_t)k * a.ntot + id];
      sv[k] = sb[(size_t)k * a.ntot + id];
    }
    // P+ = <g, f+ s>, P- = <g, f- s>, Pz = <g, fz s> in the field precision
    const R r6R = (R)r6;
    const C Pp = cadd(cscale(cadd(cconjmul(gv[0], sv[1]), cconjmul(gv[3], sv[4])), (R)2),
                      cscale(cadd(cconjmul(gv[1], sv[2]), cconjmul(gv[2], sv[3])), r6R));
    const C Pm = cadd(cscale(cadd(cconjmul(gv[1], sv[0]), cconjmul(gv[4], sv[3])), (R)2),
                      cscale(cadd(cconjmul(gv[2], sv[1]), cconjmul(gv[3], sv[2])), r6R));
    const C Pz = cadd(cscale(csub(cconjmul(gv[0], sv[0]), cconjmul(gv[4], sv[4])), (R)2),
                      csub(cconjmul(gv[1], sv[1]), cconjmul(gv[3], sv[3])));
    // Im<g, (w.f) s> = wx Im(P+ + P-)/2 - wy Re(P+ - P-)/2 + wz Im Pz
    const double kx = 0.5 * ((double)Pp.y + (double)Pm.y);
    const double ky = -0.5 * ((double)Pp.x - (double)Pm.x);
    const double kz = (double)Pz.y;
    // w in the field precision (its rounding enters the sum once)
    const R dR = (R)a.delta, nxR = (R)(kPi / a.Lx) * (R)ps, nyR = (R)(kPi / a.Ly) * (R)qs;
    const R ax = dR * (-(R)P.gamma * nyR), ay = dR * ((R)P.gamma * nxR), az = dR * (-(R)P.omega);
    const R th2 = ax * ax + ay * ay + az * az;
    const R das[2][3] = {{(R)0, (R)0, -dR}, {-dR * nyR, dR * nxR, (R)0}};
    R sk = (R)1, ck = (R)0, hx = (R)0, hy = (R)0, hz = (R)0;
    if (th2 > (R)0) {
      const R th = sqrt(th2);
      const R ith = (R)1 / th;
      hx = ax * ith;
      hy = ay * ith;
      hz = az * ith;
      R sh, ch;
      sincos_r((R)0.5 * th, &sh, &ch);
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
      acc[p] -= a.scale * ((double)wx * kx + (double)wy * ky + (double)wz * kz);
    }
  }
  block_accumulate(acc, LPA_NT, make_int4(GP_OMEGA, GP_GAMMA, 0, 0),
                   a.partials + ((size_t)m * a.nblocks + blockIdx.x) * GP_N);
}

__global__ void k_reduce_params(const double* part, int nblocks, int members, double* dp) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= members * GP_N) return;
  const int m = id / GP_N, k = id - m * GP_N;
  const double* p = part + (size_t)m * nblocks * GP_N + k;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += p[(size_t)b * GP_N];
  dp[id] = s;
}

}  // namespace

template <typename R>
cudaError_t launch_nl_adjoint(const NLAdjArgs<R>& a, int members, cudaStream_t s) {
  dim3 grid(a.nblocks, members);
  k_nl_adjoint<R><<<grid, kAdjThreads, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_lin_param(const LinParArgs<R>& a, int members, cudaStream_t s) {
  dim3 grid(a.nblocks, members);
  k_lin_param<R><<<grid, kAdjThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_reduce_params(const double* part, int nblocks, int members, double* dp,
                                 cudaStream_t s) {
  const int n = members * GP_N;
  k_reduce_params<<<(n + 127) / 128, 128, 0, s>>>(part, nblocks, members, dp);
  return cudaGetLastError();
}

template cudaError_t launch_nl_adjoint<float>(const NLAdjArgs<float>&, int, cudaStream_t);
template cudaError_t launch_nl_adjoint<double>(const NLAdjArgs<double>&, int, cudaStream_t);
template cudaError_t launch_lin_param<float>(const LinParArgs<float>&, int, cudaStream_t);
template cudaError_t launch_lin_param<double>(const LinParArgs<double>&, int, cudaStream_t);

}  // namespace sgp
