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

__device__ __forceinline__ void block_sums(double (&acc)[NLA_NT], int nterm, double* out) {
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
    out[threadIdx.x] = s;
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
  __shared__ double s_rot[2];
  if (threadIdx.x == 0) sincos(P.omega * a.t, &s_rot[1], &s_rot[0]);
  __syncthreads();
  const double co = s_rot[0], si = s_rot[1];
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
      acc[NLA_OMEGA] += (double)d * a.t * dgg * xr * yr * ipi;
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
  block_sums(acc, NLA_NT, a.partials + ((size_t)m * a.nblocks + blockIdx.x) * NLA_NT);
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
    const double nux = kPi * ps / a.Lx, nuy = kPi * qs / a.Ly;
    double gr[5][2], sr[5][2];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const C gv = gb[(size_t)k * a.ntot + id], sv = sb[(size_t)k * a.ntot + id];
      gr[k][0] = gv.x; gr[k][1] = gv.y;
      sr[k][0] = sv.x; sr[k][1] = sv.y;
    }
    // <g, u> for complex pairs in FP64
    auto cdot = [&](int i, int j, double* re, double* im) {
      *re += gr[i][0] * sr[j][0] + gr[i][1] * sr[j][1];
      *im += gr[i][0] * sr[j][1] - gr[i][1] * sr[j][0];
    };
    double ppr = 0, ppi = 0, pmr = 0, pmi = 0, pzr = 0, pzi = 0;
    {
      double r, i;
      r = i = 0; cdot(0, 1, &r, &i); ppr += 2 * r; ppi += 2 * i;
      r = i = 0; cdot(1, 2, &r, &i); ppr += r6 * r; ppi += r6 * i;
      r = i = 0; cdot(2, 3, &r, &i); ppr += r6 * r; ppi += r6 * i;
      r = i = 0; cdot(3, 4, &r, &i); ppr += 2 * r; ppi += 2 * i;
      r = i = 0; cdot(1, 0, &r, &i); pmr += 2 * r; pmi += 2 * i;
      r = i = 0; cdot(2, 1, &r, &i); pmr += r6 * r; pmi += r6 * i;
      r = i = 0; cdot(3, 2, &r, &i); pmr += r6 * r; pmi += r6 * i;
      r = i = 0; cdot(4, 3, &r, &i); pmr += 2 * r; pmi += 2 * i;
      const double mz[5] = {2, 1, 0, -1, -2};
      for (int k = 0; k < 5; ++k) {
        r = i = 0; cdot(k, k, &r, &i); pzr += mz[k] * r; pzi += mz[k] * i;
      }
    }
    (void)pzr;
    // Im<g, (w.f) s> = wx Im(P+ + P-)/2 - wy Re(P+ - P-)/2 + wz Im Pz
    const double kx = 0.5 * (ppi + pmi), ky = -0.5 * (ppr - pmr), kz = pzi;
    const double ax = a.delta * (-P.gamma * nuy), ay = a.delta * (P.gamma * nux),
                 az = a.delta * (-P.omega);
    const double th = sqrt(ax * ax + ay * ay + az * az);
    double das[2][3] = {{0.0, 0.0, -a.delta}, {-a.delta * nuy, a.delta * nux, 0.0}};
    for (int p = 0; p < 2; ++p) {
      const double dx = das[p][0], dy = das[p][1], dz = das[p][2];
      double wx = dx, wy = dy, wz = dz;
      if (th > 0.0) {
        const double hx = ax / th, hy = ay / th, hz = az / th;
        double sn, cs;
        sincos(th, &sn, &cs);
        const double sk = sn / th;
        const double ck = 2.0 * sin(0.5 * th) * sin(0.5 * th) / th;
        const double fd = hx * dx + hy * dy + hz * dz;
        const double px = hx * fd, py = hy * fd, pz = hz * fd;
        wx = px + sk * (dx - px) - ck * (hy * dz - hz * dy);
        wy = py + sk * (dy - py) - ck * (hz * dx - hx * dz);
        wz = pz + sk * (dz - pz) - ck * (hx * dy - hy * dx);
      }
      acc[p] -= a.scale * (wx * kx + wy * ky + wz * kz);
    }
  }
  block_sums(acc, LPA_NT, a.partials + ((size_t)m * a.nblocks + blockIdx.x) * LPA_NT);
}

__global__ void k_accum_params(const double* part, int nblocks, int nterm, int members,
                               int4 slots, double* dp) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= members * nterm) return;
  const int m = id / nterm, k = id - m * nterm;
  const double* p = part + (size_t)m * nblocks * nterm + k;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += p[(size_t)b * nterm];
  const int slot = k == 0 ? slots.x : (k == 1 ? slots.y : (k == 2 ? slots.z : slots.w));
  dp[(size_t)m * GP_N + slot] += s;
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

cudaError_t launch_accum_params(const double* part, int nblocks, int nterm, int members,
                                const int* slots, double* dp, cudaStream_t s) {
  const int4 sl = make_int4(slots[0], nterm > 1 ? slots[1] : 0, nterm > 2 ? slots[2] : 0,
                            nterm > 3 ? slots[3] : 0);
  const int n = members * nterm;
  k_accum_params<<<(n + 127) / 128, 128, 0, s>>>(part, nblocks, nterm, members, sl, dp);
  return cudaGetLastError();
}

template cudaError_t launch_nl_adjoint<float>(const NLAdjArgs<float>&, int, cudaStream_t);
template cudaError_t launch_nl_adjoint<double>(const NLAdjArgs<double>&, int, cudaStream_t);
template cudaError_t launch_lin_param<float>(const LinParArgs<float>&, int, cudaStream_t);
template cudaError_t launch_lin_param<double>(const LinParArgs<double>&, int, cudaStream_t);

}  // namespace sgp
