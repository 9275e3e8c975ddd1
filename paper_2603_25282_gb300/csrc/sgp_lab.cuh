// sgp_lab.cuh -- launchers of the lab-frame output kernels (sgp_lab.cu).
#pragma once
#include <cuda_runtime.h>

#include "sgp_launch.cuh"

namespace sgp {

// One shear of one member's field: every line along the transform axis is
// translated by coef * (o0 + j * h0), j the line's index along the other
// axis, via a forward FFT, the phase exp(i nu c) per mode and the inverse
// FFT (1/N applied).  Rows (x-lines): rows = ny * nz lines, j = row mod ny.
// Columns (y-lines): rows = nx columns, j = the column's x index, planes =
// nz z-planes at plane_stride.
template <typename R>
struct ShearArgs {
  cplx<R>* field;            // [5][ntot], one member
  const TwE<R>* tw;          // twiddles of the line axis (default radix plan)
  long long ntot;
  int rows;                  // lines (rows) or columns
  int ny;                    // rows: y extent (j = row mod ny)
  long long line_stride;     // columns: element stride along y (nx)
  long long plane_stride;    // columns: element stride between z planes (nx ny)
  double coef;               // shear coefficient
  double o0, h0;             // coordinate of the other axis: o0 + j h0
  double kfac;               // pi / L along the line axis (nu_p = kfac p)
  double theta;              // rows: exp(i l theta) applied after the shear if lab_phase
  int lab_phase;
};

template <typename R>
cudaError_t launch_shear_rows(int N, const ShearArgs<R>& a, cudaStream_t s);
template <typename R>
cudaError_t launch_shear_cols(int N, const ShearArgs<R>& a, int planes, cudaStream_t s);
template <typename R>
cudaError_t launch_quarter(const cplx<R>* in, cplx<R>* out, int n, long long ntot, int k,
                           cudaStream_t s);

}  // namespace sgp
