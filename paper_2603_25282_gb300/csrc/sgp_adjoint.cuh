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

template <typename R>
struct NLAdjArgs {
  cplx<R>* g;               // [member][5][ntot]: in g at the substep output, out g at its input
  const cplx<R>* phi;       // [member][5][ntot]: the substep's output state (physical space)
  long long ntot;
  int nx, ny;
  double x0, hx, y0, hy, z0, hz;
  double delta;             // forward substep size
  const double* t_base;     // the substep's time is *t_base + t_off (FP64, on the device)
  double t_off;
  const MemberPrm* mp;
  double* partials;         // [member][nblocks][GP_N], each block adds to its own row
  int nblocks;
};

template <typename R>
struct LinParArgs {
  const cplx<R>* g;         // unnormalised full transforms of g and of Phi_out
  const cplx<R>* s;
  long long ntot;
  int NX, NY;
  double Lx, Ly;
  double delta;
  double scale;             // 1/(NX NY [NZ])
  const MemberPrm* mp;
  double* partials;         // [member][nblocks][GP_N], as NLAdjArgs
  int nblocks;
};

constexpr int kAdjThreads = 256;

// blocks per member of the adjoint kernels (fixed, so the sums are deterministic)
inline int adjoint_blocks(long long ntot) {
  const long long b = (ntot + kAdjThreads - 1) / kAdjThreads;
  return (int)(b < 1024 ? b : 1024);
}

template <typename R>
cudaError_t launch_nl_adjoint(const NLAdjArgs<R>& a, int members, cudaStream_t s);
template <typename R>
cudaError_t launch_lin_param(const LinParArgs<R>& a, int members, cudaStream_t s);
// dp[m][k] = sum over blocks of part[m][b][k], k < GP_N (fixed order)
cudaError_t launch_reduce_params(const double* part, int nblocks, int members, double* dp,
                                 cudaStream_t s);

}  // namespace sgp
