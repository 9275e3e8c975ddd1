// sgp_api.cu -- the C ABI declared in include/sgp.h: context management,
// per-substep tables, pass orchestration of TS2/TS4 and the observables.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sgp.h"
#include "sgp_launch.cuh"

using namespace sgp;

namespace {

constexpr double kPi = 3.14159265358979323846;

// TS4 coefficients of Sec. 3.3 (c = 2^(1/3)).
const double kCbrt2 = std::cbrt(2.0);
const double kA1 = 1.0 / (2.0 * (2.0 - kCbrt2));
const double kA2 = (1.0 - kCbrt2) / (2.0 * (2.0 - kCbrt2));
const double kB1 = 1.0 / (2.0 - kCbrt2);
const double kB2 = -kCbrt2 / (2.0 - kCbrt2);

// ----------------------------------------------------------------------------
// table kernels (FP64 arithmetic, stored in the context precision)
// ----------------------------------------------------------------------------
// Rounding of an FP64 complex target to the working precision.  For FP32
// the 5x5 neighbourhood (+-2 ulp per coordinate) of the rounded pair is
// searched for the smallest ||z| - |target|| + wz |z - target| (relative).
// Twiddles use wz = 0.02: the inverse transform applies conj(W) on the same
// path as the forward W, so only |W| enters the round trip and a modulus
// error would otherwise accumulate over the steps.
__device__ inline void store_pair_w(double tx, double ty, double wz, float* ox, float* oy) {
  const double m = sqrt(tx * tx + ty * ty);
  float xs[5], ys[5];
  xs[2] = (float)tx;
  ys[2] = (float)ty;
  xs[1] = nextafterf(xs[2], -INFINITY); xs[0] = nextafterf(xs[1], -INFINITY);
  xs[3] = nextafterf(xs[2], INFINITY);  xs[4] = nextafterf(xs[3], INFINITY);
  ys[1] = nextafterf(ys[2], -INFINITY); ys[0] = nextafterf(ys[1], -INFINITY);
  ys[3] = nextafterf(ys[2], INFINITY);  ys[4] = nextafterf(ys[3], INFINITY);
  double best = 1e300;
  for (int a = 0; a < 5; ++a)
    for (int b = 0; b < 5; ++b) {
      const double x = xs[a], y = ys[b];
      const double dz = sqrt((x - tx) * (x - tx) + (y - ty) * (y - ty));
      const double dm = fabs(sqrt(x * x + y * y) - m);
      const double sc = dm + wz * dz;
      if (sc < best) {
        best = sc;
        *ox = xs[a];
        *oy = ys[b];
      }
    }
}
__device__ inline void store_pair_w(double tx, double ty, double, double* ox, double* oy) {
  *ox = tx;
  *oy = ty;
}

// Stage-ordered twiddle table of a length-N line with E elements per thread
// (layout of tw_offset in sgp_fft.cuh): entry (s, r, j) = W_{NS*RD}^{j r},
// evaluated in FP64; FP32 entries are stored as hi + lo (see TwE).
__device__ inline void tw_angle(int N, int E, int k, double* s_out, double* c_out, bool* used) {
  int off = 0, ns = radix_at(N, E, 0), st = 1;
  *used = false;
  while (true) {
    const int rd = radix_at(N, E, st);
    if (rd <= 0) return;
    const int cnt = (rd - 1) * ns;
    if (k < off + cnt) {
      const int local = k - off;
      const int r = local / ns + 1, j = local - (r - 1) * ns;
      sincospi(-2.0 * (double)(j * r) / (double)(ns * rd), s_out, c_out);
      *used = true;
      return;
    }
    off += cnt;
    ns *= rd;
    ++st;
  }
}
__global__ void k_twiddles_f32(int N, int E, TwE<float>* out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  double s = 0.0, c = 1.0;
  bool used;
  tw_angle(N, E, k, &s, &c, &used);
  const float hx = (float)c, hy = (float)s;
  out[k] = TwE<float>{make_float2(hx, hy), make_float2((float)(c - hx), (float)(s - hy))};
}
__global__ void k_twiddles_f64(int N, int E, TwE<double>* out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  double s = 0.0, c = 1.0;
  bool used;
  tw_angle(N, E, k, &s, &c, &used);
  out[k] = TwE<double>{make_double2(c, s)};
}

// Elements per thread of the line kernels (elems_per_thread<R, N>).
inline int elems_for(int N, int prec) {
  return (N % 3 == 0) ? 6 : (prec == SGP_F32 ? 8 : 4);
}

// Per-mode table of the linear flow over delta (Sec. 3.1, Eq. (sl1)), one
// entry per (|p|, |q|) in the layout MT_* of sgp_kernels.cuh.  The angles are
// formed and the exponentials evaluated in FP64, and the small quantities
// exp(-i chi) - 1, ahat - 1, cp - 1 are written without cancellation:
//   exp(-i chi) - 1 = (-2 sin^2(chi/2), -sin chi),
//   U11 = c - i s Omega/lambda (c, s = cos, sin of delta lambda/2),
//   cp - 1 = -s^2 gamma^2 |nu_perp|^2 / lambda^2 / (1 + cp),
//   ahat - 1 = (c - cp - i s Omega/lambda)/cp,  c - cp = -s^2 Omega^2/lambda^2/(c + cp).
// kz[r] = exp(-i nu_z^2 delta/2) - 1.
template <typename R>
__global__ void k_linear_tables(double delta, double omega, double gamma, int NX, int NY,
                                int NZ, double Lx, double Ly, double Lz, R* mt, cplx<R>* kz) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  const int hq = NY / 2 + 1;
  const int nent = (NX / 2 + 1) * hq;
  if (id < nent) {
    const int ap = id / hq, aq = id - ap * hq;
    const double nup = kPi * ap / Lx, nuq = kPi * aq / Ly;
    const double nperp = sqrt(nup * nup + nuq * nuq);
    const double lamb = sqrt(omega * omega + gamma * gamma * nperp * nperp);
    double am1r = 0.0, am1i = 0.0, cm1 = 0.0, sp = 0.0;
    if (lamb > 0.0) {
      double sn, cs;
      sincos(0.5 * delta * lamb, &sn, &cs);
      const double so = sn * omega / lamb;          // s Omega / lambda
      const double sg = sn * gamma * nperp / lamb;  // s gamma |nu_perp| / lambda
      const double cp = sqrt(cs * cs + so * so);
      cm1 = -(sg * sg) / (1.0 + cp);
      const double cmc = cs > 0.0 ? -(so * so) / (cs + cp) : cs - cp;
      if (cp > 0.0) {
        am1r = cmc / cp;
        am1i = -so / cp;
      }
      sp = sg;
    }
    const double chi = 0.5 * (nup * nup + nuq * nuq) * delta;
    double sh, ch;
    sincos(0.5 * chi, &sh, &ch);
    R* e = mt + (size_t)MT_STRIDE * id;
    e[MT_KHR] = (R)(-2.0 * sh * sh);
    e[MT_KHI] = (R)(-2.0 * sh * ch);
    e[MT_AM1R] = (R)am1r;
    e[MT_AM1I] = (R)am1i;
    e[MT_CM1] = (R)cm1;
    e[MT_SP] = (R)sp;
    if (nperp > 0.0)
      store_pair_w(nup / nperp, nuq / nperp, 0.02, &e[MT_BX], &e[MT_BY]);
    else {
      e[MT_BX] = (R)1;
      e[MT_BY] = (R)0;
    }
  }
  if (id < NZ) {
    const int ks_ = id < NZ / 2 ? id : id - NZ;
    const double nu = kPi * ks_ / Lz;
    double sh, ch;
    sincos(0.25 * nu * nu * delta, &sh, &ch);
    kz[id] = mkc((R)(-2.0 * sh * sh), (R)(-2.0 * sh * ch));
  }
}

__global__ void k_set_time(double* t, double v) { *t = v; }

// ----------------------------------------------------------------------------
// context
// ----------------------------------------------------------------------------
struct LinTables {
  double delta = 0.0;
  void* mt = nullptr;    // per-mode table, MT_STRIDE values per (|p|, |q|)
  void* kz = nullptr;    // z kinetic factors (NZ entries)
};

}  // namespace

struct sgp_ctx {
  int dim = 2;
  int n[3] = {1, 1, 1};
  double L[3] = {1, 1, 1};
  double h[3] = {1, 1, 1};
  int batch = 1;
  int prec = SGP_F32;
  int device = 0;
  cudaStream_t stream = nullptr;
  long long ntot = 0;
  size_t elem = 8;
  void* field = nullptr;
  void* tw[3] = {nullptr, nullptr, nullptr};
  double* t_dev = nullptr;
  double t = 0.0;
  sgp_params prm{};
  bool have_params = false;
  bool have_state = false;
  std::vector<LinTables> tables;    // cache keyed by delta (params fixed)
  double* partials = nullptr;       // observables scratch
  size_t partials_len = 0;
  double* obs_dev = nullptr;        // [batch][OB_NT]
  long long launches = 0;
  // profiling: event pairs per launch kind (enabled by sgp_set_profiling)
  bool profiling = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof;
  std::vector<cudaEvent_t> event_pool;
  std::string err;
};

namespace {

std::string g_create_err;

sgp_status fail(sgp_ctx* c, sgp_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c)
    c->err = buf;
  else
    g_create_err = buf;
  return s;
}

#define SGP_CUDA(ctx, call)                                                              \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail((ctx), SGP_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),     \
                  __FILE__, __LINE__);                                                   \
  } while (0)

enum { PK_X = 0, PK_Y = 1, PK_Z = 2, PK_TAB = 3, PK_OBS = 4, PK_OTHER = 5, PK_N = 6 };

cudaEvent_t take_event(sgp_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Records an event pair around one launch when profiling is on.
struct ProfScope {
  sgp_ctx* c;
  int kind;
  cudaEvent_t a = nullptr, b = nullptr;
  ProfScope(sgp_ctx* ctx, int k) : c(ctx), kind(k) {
    if (c->profiling) {
      a = take_event(c);
      b = take_event(c);
      cudaEventRecord(a, c->stream);
    }
  }
  ~ProfScope() {
    if (a) {
      cudaEventRecord(b, c->stream);
      c->prof.push_back({kind, {a, b}});
    }
  }
};

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

bool finite_params(const sgp_params* p) {
  const double v[8] = {p->omega, p->gamma, p->c0, p->c1, p->c2, p->gx, p->gy, p->gz};
  for (double x : v)
    if (!std::isfinite(x)) return false;
  return true;
}

void free_tables(sgp_ctx* c) {
  for (auto& t : c->tables) {
    cudaFree(t.mt);
    cudaFree(t.kz);
  }
  c->tables.clear();
}

template <typename R>
sgp_status get_tables(sgp_ctx* c, double delta, const LinTables** out) {
  for (auto& t : c->tables)
    if (t.delta == delta) {
      *out = &t;
      return SGP_OK;
    }
  if (c->tables.size() >= 8) free_tables(c);
  LinTables t;
  t.delta = delta;
  const int NX = c->n[0], NY = c->n[1], NZ = c->n[2];
  const size_t nent = (size_t)(NX / 2 + 1) * (NY / 2 + 1);
  SGP_CUDA(c, cudaMalloc(&t.mt, nent * MT_STRIDE * sizeof(R)));
  SGP_CUDA(c, cudaMalloc(&t.kz, (size_t)NZ * sizeof(cplx<R>)));
  const int work = (int)std::max<size_t>(nent, (size_t)NZ);
  ProfScope ps(c, PK_TAB);
  k_linear_tables<R><<<(work + 255) / 256, 256, 0, c->stream>>>(
      delta, c->prm.omega, c->prm.gamma, NX, NY, NZ, c->L[0], c->L[1], c->L[2], (R*)t.mt,
      (cplx<R>*)t.kz);
  c->launches++;
  SGP_CUDA(c, cudaGetLastError());
  c->tables.push_back(t);
  *out = &c->tables.back();
  return SGP_OK;
}

// ----------------------------------------------------------------------------
// passes
// ----------------------------------------------------------------------------
template <typename R>
sgp_status x_pass(sgp_ctx* c, int mode, double delta, double t_off) {
  XPassArgs<R> a{};
  a.field = (cplx<R>*)c->field;
  a.tw = (const TwE<R>*)c->tw[0];
  a.ntot = c->ntot;
  a.rows = c->n[1] * c->n[2];
  a.ny = c->n[1];
  a.mode = mode;
  a.x0 = (R)-c->L[0];
  a.hx = (R)c->h[0];
  a.y0 = (R)-c->L[1];
  a.hy = (R)c->h[1];
  a.z0 = c->dim == 3 ? (R)-c->L[2] : (R)0;
  a.hz = c->dim == 3 ? (R)c->h[2] : (R)0;
  a.delta = (R)delta;
  a.c0p = (R)(c->prm.c0 + c->prm.c2 / 5.0);
  a.c1 = (R)c->prm.c1;
  a.c2 = (R)c->prm.c2;
  a.gx2h = (R)(0.5 * c->prm.gx * c->prm.gx);
  a.gy2h = (R)(0.5 * c->prm.gy * c->prm.gy);
  a.gz2h = c->dim == 3 ? (R)(0.5 * c->prm.gz * c->prm.gz) : (R)0;
  a.omega = c->prm.omega;
  a.t_base = c->t_dev;
  a.t_off = t_off;
  c->launches++;
  ProfScope ps(c, PK_X);
  SGP_CUDA(c, launch_xpass<R>(c->n[0], a, c->batch, c->stream));
  return SGP_OK;
}

// axis 1: lines along y (planes = z slices); axis 2: lines along z (planes = y rows)
template <typename R>
sgp_status line_pass(sgp_ctx* c, int axis, int mode, const LinTables* t) {
  LPassArgs<R> a{};
  a.field = (cplx<R>*)c->field;
  a.tw = (const TwE<R>*)c->tw[axis];
  a.ntot = c->ntot;
  a.nx = c->n[0];
  const long long nxy = (long long)c->n[0] * c->n[1];
  int planes;
  if (axis == 1) {
    a.line_stride = c->n[0];
    a.plane_stride = nxy;
    planes = c->n[2];
  } else {
    a.line_stride = nxy;
    a.plane_stride = c->n[0];
    planes = c->n[1];
  }
  a.mode = mode;
  a.axis = axis;
  a.NX = c->n[0];
  a.NY = c->n[1];
  if (t) {
    a.mt = (const R*)t->mt;
    a.kz = (const cplx<R>*)t->kz;
  }
  {
    const double inv = 1.0 / ((double)c->n[0] * c->n[1] * (c->dim == 3 ? c->n[2] : 1));
    a.inv_hi = (R)inv;
    a.inv_lo = (R)(inv - (double)a.inv_hi);
  }
  c->launches++;
  ProfScope ps(c, axis == 1 ? PK_Y : PK_Z);
  SGP_CUDA(c, launch_linepass<R>(c->n[axis], a, planes, c->batch, c->stream));
  return SGP_OK;
}

#define SGP_TRY(x)                   \
  do {                               \
    sgp_status s_ = (x);             \
    if (s_ != SGP_OK) return s_;     \
  } while (0)

// Linear flow over delta between x-passes.  Entry: x-spectral (the x-pass
// has done its forward transform).  Exit: x-spectral.
template <typename R>
sgp_status linear_middle(sgp_ctx* c, double delta) {
  const LinTables* t = nullptr;
  SGP_TRY(get_tables<R>(c, delta, &t));
  if (c->dim == 2) {
    SGP_TRY(line_pass<R>(c, 1, LP_FWD | LP_MIX | LP_INV, t));
  } else {
    SGP_TRY(line_pass<R>(c, 1, LP_FWD, nullptr));
    SGP_TRY(line_pass<R>(c, 2, LP_FWD | LP_MIX | LP_INV, t));
    SGP_TRY(line_pass<R>(c, 1, LP_INV, nullptr));
  }
  return SGP_OK;
}

// Run nsteps of the composition.  Adjacent nonlinear substeps at the same
// time are merged (exact flow property), so the pass sequence is
//   N  L  N  L ... L  N   (N as x-passes, L as the line passes).
template <typename R>
sgp_status run_steps(sgp_ctx* c, long long nsteps, double dt, int scheme) {
  // substep pattern of one step, Sec. 3.3
  std::vector<std::pair<char, double>> seq;
  if (scheme == SGP_TS2) {
    seq = {{'N', 0.5}, {'L', 1.0}, {'N', 0.5}};
  } else {
    seq = {{'N', kA1}, {'L', kB1}, {'N', kA2}, {'L', kB2},
           {'N', kA2}, {'L', kB1}, {'N', kA1}};
  }
  const double t0 = c->t;
  c->launches++;
  {
    ProfScope ps(c, PK_OTHER);
    k_set_time<<<1, 1, 0, c->stream>>>(c->t_dev, t0);
  }
  SGP_CUDA(c, cudaGetLastError());
  // first nonlinear substep (physical in, x-spectral out)
  SGP_TRY(x_pass<R>(c, XP_NL | XP_FWD, seq[0].second * dt, 0.0));
  const int inner = (int)seq.size();
  for (long long s = 0; s < nsteps; ++s) {
    double toff = (double)s * dt;      // offset of this step's start from t0
    double sub = 0.0;                  // time advanced within the step
    for (int k = 1; k < inner; ++k) {
      if (seq[k].first == 'L') {
        const double d = seq[k].second * dt;
        SGP_TRY(linear_middle<R>(c, d));
        sub += seq[k].second;
      } else {
        double coef = seq[k].second;
        const bool last_in_step = (k == inner - 1);
        const bool last = last_in_step && (s == nsteps - 1);
        if (last_in_step && !last) coef += seq[0].second;   // merge with next step's first N
        const double tn = last_in_step ? (double)(s + 1) * dt : toff + sub * dt;
        const int mode = last ? (XP_INV | XP_NL) : (XP_INV | XP_NL | XP_FWD);
        SGP_TRY(x_pass<R>(c, mode, coef * dt, tn));
      }
    }
  }
  c->t = t0 + (double)nsteps * dt;
  return SGP_OK;
}

template <typename R>
sgp_status substep(sgp_ctx* c, int kind, double delta) {
  c->launches++;
  k_set_time<<<1, 1, 0, c->stream>>>(c->t_dev, c->t);
  SGP_CUDA(c, cudaGetLastError());
  if (kind == SGP_SUB_NONLINEAR) {
    SGP_TRY(x_pass<R>(c, XP_NL, delta, 0.0));
  } else {
    SGP_TRY(x_pass<R>(c, XP_FWD, 0.0, 0.0));
    SGP_TRY(linear_middle<R>(c, delta));
    SGP_TRY(x_pass<R>(c, XP_INV, 0.0, 0.0));
    c->t += delta;
  }
  return SGP_OK;
}

// ----------------------------------------------------------------------------
// observables
// ----------------------------------------------------------------------------
template <typename R>
sgp_status observables(sgp_ctx* c, sgp_obs* out) {
  const int NX = c->n[0];
  const PassGeom gx = xpass_geom<R>(NX);
  const int rows = c->n[1] * c->n[2];
  const int nbx = (rows + gx.rows_or_tile - 1) / gx.rows_or_tile;
  ObsXArgs<R> ax{};
  ax.ntot = c->ntot;
  ax.rows = rows;
  ax.ny = c->n[1];
  ax.x0 = -c->L[0];
  ax.hx = c->h[0];
  ax.y0 = -c->L[1];
  ax.hy = c->h[1];
  ax.z0 = c->dim == 3 ? -c->L[2] : 0.0;
  ax.hz = c->dim == 3 ? c->h[2] : 0.0;
  ax.omega = c->prm.omega;
  ax.t = c->t;
  ax.c0 = c->prm.c0;
  ax.c1 = c->prm.c1;
  ax.c2 = c->prm.c2;
  ax.gx2h = 0.5 * c->prm.gx * c->prm.gx;
  ax.gy2h = 0.5 * c->prm.gy * c->prm.gy;
  ax.gz2h = c->dim == 3 ? 0.5 * c->prm.gz * c->prm.gz : 0.0;
  ax.partials = c->partials;
  ax.nblocks = nbx;
  ax.field = (const cplx<R>*)c->field;
  ax.tw = (const TwE<R>*)c->tw[0];
  ax.dnu = (R)(kPi / c->L[0] / NX);
  ax.NX = NX;
  c->launches++;
  {
    ProfScope ps(c, PK_OBS);
    SGP_CUDA(c, launch_obs_x<R>(NX, ax, c->batch, c->stream));
  }
  c->launches++;
  k_reduce_partials<<<(c->batch * OBX_NT + 127) / 128, 128, 0, c->stream>>>(
      c->partials, nbx, OBX_NT, c->batch, c->obs_dev, OB_NT, 0);
  SGP_CUDA(c, cudaGetLastError());
  for (int axis = 1; axis < c->dim; ++axis) {
    const int NL = c->n[axis];
    const PassGeom gl = linepass_geom<R>(NL);
    ObsLArgs<R> al{};
    static_cast<ObsArgsBase&>(al) = static_cast<const ObsArgsBase&>(ax);
    al.field = (const cplx<R>*)c->field;
    al.tw = (const TwE<R>*)c->tw[axis];
    al.nx = NX;
    const long long nxy = (long long)c->n[0] * c->n[1];
    int planes;
    if (axis == 1) {
      al.line_stride = NX;
      al.plane_stride = nxy;
      planes = c->n[2];
    } else {
      al.line_stride = nxy;
      al.plane_stride = NX;
      planes = c->n[1];
    }
    al.axis = axis;
    al.dnu = (R)(kPi / c->L[axis] / NL);
    al.NL = NL;
    const int tiles = (NX + gl.rows_or_tile - 1) / gl.rows_or_tile;
    al.nblocks = tiles * planes;
    c->launches++;
    {
      ProfScope ps(c, PK_OBS);
      SGP_CUDA(c, launch_obs_line<R>(NL, al, planes, c->batch, c->stream));
    }
    c->launches++;
    k_reduce_partials<<<(c->batch * OBL_NT + 127) / 128, 128, 0, c->stream>>>(
        c->partials, al.nblocks, OBL_NT, c->batch, c->obs_dev, OB_NT,
        axis == 1 ? OB_KY : OB_KZ);
    SGP_CUDA(c, cudaGetLastError());
  }
  std::vector<double> h((size_t)c->batch * OB_NT, 0.0);
  SGP_CUDA(c, cudaMemcpyAsync(h.data(), c->obs_dev, h.size() * sizeof(double),
                              cudaMemcpyDeviceToHost, c->stream));
  SGP_CUDA(c, cudaStreamSynchronize(c->stream));
  const double cell = c->h[0] * c->h[1] * (c->dim == 3 ? c->h[2] : 1.0);
  bool finite = true;
  for (int m = 0; m < c->batch; ++m) {
    const double* s = &h[(size_t)m * OB_NT];
    if (c->dim == 2) {
      // OB_KZ slot is not written in 2D (the z-line pass does not run)
    }
    sgp_obs o{};
    o.t = c->t;
    o.mass = 0.0;
    o.magnetization = 0.0;
    for (int k = 0; k < 5; ++k) {
      o.comp_mass[k] = cell * s[OB_M0 + k];
      o.mass += o.comp_mass[k];
      o.magnetization += (2 - k) * o.comp_mass[k];
    }
    o.width2[0] = cell * s[OB_WX];
    o.width2[1] = cell * s[OB_WY];
    o.width2[2] = cell * s[OB_WZ];
    const double kz = c->dim == 3 ? s[OB_KZ] : 0.0;
    o.e_kin = cell * (s[OB_KX] + s[OB_KY] + kz);
    o.e_pot = cell * s[OB_POT];
    o.lz = cell * (s[OB_LZX] + s[OB_LZY]);
    o.e_rot = -c->prm.omega * o.lz;
    o.e_int = cell * s[OB_INT];
    o.e_soc = -c->prm.gamma * cell * (s[OB_SOCX] + s[OB_SOCY]);
    o.energy = o.e_kin + o.e_pot + o.e_rot + o.e_int + o.e_soc;
    const double chk[6] = {o.mass, o.energy, o.magnetization, o.lz, o.width2[0], o.width2[1]};
    for (double v : chk)
      if (!std::isfinite(v)) finite = false;
    out[m] = o;
  }
  if (!finite) return fail(c, SGP_ENONFINITE, "non-finite observable");
  return SGP_OK;
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

int sgp_version(void) { return 100; }

const char* sgp_status_string(sgp_status s) {
  switch (s) {
    case SGP_OK: return "SGP_OK";
    case SGP_EINVAL: return "SGP_EINVAL";
    case SGP_ENOMEM: return "SGP_ENOMEM";
    case SGP_ECUDA: return "SGP_ECUDA";
    case SGP_ETIMEOUT: return "SGP_ETIMEOUT";
    case SGP_ENONFINITE: return "SGP_ENONFINITE";
    case SGP_ESTATE: return "SGP_ESTATE";
    case SGP_EUNSUPPORTED: return "SGP_EUNSUPPORTED";
  }
  return "unknown";
}

const char* sgp_last_error(const sgp_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

sgp_status sgp_create_grid(int dim, const int* n, const double* L, int batch, int prec,
                           int device, void* stream, sgp_ctx** out) {
  g_create_err.clear();
  if (!out || !n || !L) return fail(nullptr, SGP_EINVAL, "NULL argument");
  *out = nullptr;
  if (dim != 2 && dim != 3) return fail(nullptr, SGP_EINVAL, "dim must be 2 or 3 (got %d)", dim);
  if (prec != SGP_F32 && prec != SGP_F64)
    return fail(nullptr, SGP_EINVAL, "prec must be SGP_F32 or SGP_F64");
  if (batch < 1 || batch > 65535)
    return fail(nullptr, SGP_EINVAL, "batch must be in [1, 65535] (got %d)", batch);
  for (int a = 0; a < dim; ++a) {
    if (!supported_n(n[a]))
      return fail(nullptr, SGP_EINVAL,
                  "n[%d] = %d not supported (2^a 3^b in {16..1024}, b <= 1)", a, n[a]);
    if (!(L[a] > 0.0) || !std::isfinite(L[a]))
      return fail(nullptr, SGP_EINVAL, "L[%d] must be positive and finite", a);
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return fail(nullptr, SGP_EINVAL, "CUDA device %d not available", device);
  DeviceGuard guard(device);
  sgp_ctx* c = new sgp_ctx();
  c->dim = dim;
  for (int a = 0; a < 3; ++a) {
    c->n[a] = a < dim ? n[a] : 1;
    c->L[a] = a < dim ? L[a] : 1.0;
    c->h[a] = 2.0 * c->L[a] / c->n[a];
  }
  c->batch = batch;
  c->prec = prec;
  c->device = device;
  c->stream = (cudaStream_t)stream;
  c->ntot = (long long)c->n[0] * c->n[1] * c->n[2];
  c->elem = prec == SGP_F32 ? 8 : 16;
  c->prm.gx = c->prm.gy = c->prm.gz = 1.0;
  auto bail = [&](sgp_status s, const char* what, cudaError_t e) {
    fail(nullptr, s, "%s: %s", what, cudaGetErrorString(e));
    sgp_destroy(c);
    return s;
  };
  cudaError_t e;
  const size_t fbytes = (size_t)batch * 5 * c->ntot * c->elem;
  if ((e = cudaMalloc(&c->field, fbytes)) != cudaSuccess)
    return bail(SGP_ENOMEM, "field allocation", e);
  if ((e = cudaMemsetAsync(c->field, 0, fbytes, c->stream)) != cudaSuccess)
    return bail(SGP_ECUDA, "field clear", e);
  for (int a = 0; a < dim; ++a) {
    if ((e = cudaMalloc(&c->tw[a], (size_t)c->n[a] * 16)) != cudaSuccess)
      return bail(SGP_ENOMEM, "twiddle allocation", e);
    const int E = elems_for(c->n[a], prec);
    if (prec == SGP_F32)
      k_twiddles_f32<<<(c->n[a] + 255) / 256, 256, 0, c->stream>>>(c->n[a], E, (TwE<float>*)c->tw[a]);
    else
      k_twiddles_f64<<<(c->n[a] + 255) / 256, 256, 0, c->stream>>>(c->n[a], E, (TwE<double>*)c->tw[a]);
    c->launches++;
  }
  if ((e = cudaMalloc(&c->t_dev, sizeof(double))) != cudaSuccess)
    return bail(SGP_ENOMEM, "time allocation", e);
  // observables scratch: the largest per-kernel partial array
  const PassGeom gx = prec == SGP_F32 ? xpass_geom<float>(c->n[0]) : xpass_geom<double>(c->n[0]);
  size_t need = (size_t)((c->n[1] * c->n[2] + gx.rows_or_tile - 1) / gx.rows_or_tile) * OBX_NT;
  for (int a = 1; a < dim; ++a) {
    const PassGeom gl = prec == SGP_F32 ? linepass_geom<float>(c->n[a]) : linepass_geom<double>(c->n[a]);
    const size_t tiles = (size_t)(c->n[0] + gl.rows_or_tile - 1) / gl.rows_or_tile;
    const size_t planes = a == 1 ? c->n[2] : c->n[1];
    need = std::max(need, tiles * planes * OBL_NT);
  }
  c->partials_len = need * batch;
  if ((e = cudaMalloc(&c->partials, c->partials_len * sizeof(double))) != cudaSuccess)
    return bail(SGP_ENOMEM, "observables scratch", e);
  if ((e = cudaMalloc(&c->obs_dev, (size_t)batch * OB_NT * sizeof(double))) != cudaSuccess)
    return bail(SGP_ENOMEM, "observables output", e);
  if ((e = cudaMemsetAsync(c->obs_dev, 0, (size_t)batch * OB_NT * sizeof(double), c->stream)) !=
      cudaSuccess)
    return bail(SGP_ECUDA, "observables clear", e);
  if ((e = cudaGetLastError()) != cudaSuccess) return bail(SGP_ECUDA, "table launch", e);
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return bail(SGP_ECUDA, "create sync", e);
  *out = c;
  return SGP_OK;
}

sgp_status sgp_set_params(sgp_ctx* c, const sgp_params* p) {
  if (!c) return SGP_EINVAL;
  if (!p) return fail(c, SGP_EINVAL, "NULL params");
  if (!finite_params(p)) return fail(c, SGP_EINVAL, "non-finite parameter");
  DeviceGuard guard(c->device);
  // tables depend on (Omega, gamma); they may still be in use by queued work
  cudaStreamSynchronize(c->stream);
  free_tables(c);
  c->prm = *p;
  c->have_params = true;
  return SGP_OK;
}

sgp_status sgp_set_state(sgp_ctx* c, const void* src, int src_on_device, double t0) {
  if (!c) return SGP_EINVAL;
  if (!src) return fail(c, SGP_EINVAL, "NULL src");
  if (!std::isfinite(t0)) return fail(c, SGP_EINVAL, "non-finite t0");
  DeviceGuard guard(c->device);
  const size_t bytes = (size_t)c->batch * 5 * c->ntot * c->elem;
  SGP_CUDA(c, cudaMemcpyAsync(c->field, src, bytes,
                              src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              c->stream));
  if (!src_on_device) SGP_CUDA(c, cudaStreamSynchronize(c->stream));
  c->t = t0;
  c->have_state = true;
  return SGP_OK;
}

sgp_status sgp_get_state(sgp_ctx* c, void* dst, int dst_on_device) {
  if (!c) return SGP_EINVAL;
  if (!dst) return fail(c, SGP_EINVAL, "NULL dst");
  DeviceGuard guard(c->device);
  const size_t bytes = (size_t)c->batch * 5 * c->ntot * c->elem;
  SGP_CUDA(c, cudaMemcpyAsync(dst, c->field, bytes,
                              dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                              c->stream));
  if (!dst_on_device) SGP_CUDA(c, cudaStreamSynchronize(c->stream));
  return SGP_OK;
}

sgp_status sgp_get_time(const sgp_ctx* c, double* t) {
  if (!c || !t) return SGP_EINVAL;
  *t = c->t;
  return SGP_OK;
}

sgp_status sgp_step(sgp_ctx* c, long long nsteps, double dt, int scheme) {
  if (!c) return SGP_EINVAL;
  if (nsteps < 0) return fail(c, SGP_EINVAL, "nsteps < 0");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, SGP_EINVAL, "dt must be positive and finite");
  if (scheme != SGP_TS2 && scheme != SGP_TS4) return fail(c, SGP_EINVAL, "unknown scheme %d", scheme);
  if (!c->have_state) return fail(c, SGP_ESTATE, "sgp_step before sgp_set_state");
  if (nsteps == 0) return SGP_OK;
  DeviceGuard guard(c->device);
  return c->prec == SGP_F32 ? run_steps<float>(c, nsteps, dt, scheme)
                            : run_steps<double>(c, nsteps, dt, scheme);
}

sgp_status sgp_substep(sgp_ctx* c, int kind, double delta) {
  if (!c) return SGP_EINVAL;
  if (kind != SGP_SUB_NONLINEAR && kind != SGP_SUB_LINEAR)
    return fail(c, SGP_EINVAL, "unknown substep kind %d", kind);
  if (!std::isfinite(delta)) return fail(c, SGP_EINVAL, "non-finite delta");
  if (!c->have_state) return fail(c, SGP_ESTATE, "sgp_substep before sgp_set_state");
  DeviceGuard guard(c->device);
  return c->prec == SGP_F32 ? substep<float>(c, kind, delta) : substep<double>(c, kind, delta);
}

sgp_status sgp_observables(sgp_ctx* c, sgp_obs* out) {
  if (!c) return SGP_EINVAL;
  if (!out) return fail(c, SGP_EINVAL, "NULL out");
  if (!c->have_state) return fail(c, SGP_ESTATE, "sgp_observables before sgp_set_state");
  DeviceGuard guard(c->device);
  return c->prec == SGP_F32 ? observables<float>(c, out) : observables<double>(c, out);
}

sgp_status sgp_synchronize(sgp_ctx* c) {
  if (!c) return SGP_EINVAL;
  DeviceGuard guard(c->device);
  SGP_CUDA(c, cudaStreamSynchronize(c->stream));
  return SGP_OK;
}

long long sgp_launch_count(const sgp_ctx* c) { return c ? c->launches : 0; }

static void recycle_events(sgp_ctx* c) {
  for (auto& p : c->prof) {
    c->event_pool.push_back(p.second.first);
    c->event_pool.push_back(p.second.second);
  }
  c->prof.clear();
}

sgp_status sgp_set_profiling(sgp_ctx* c, int enable) {
  if (!c) return SGP_EINVAL;
  DeviceGuard guard(c->device);
  SGP_CUDA(c, cudaStreamSynchronize(c->stream));
  recycle_events(c);
  c->profiling = enable != 0;
  return SGP_OK;
}

sgp_status sgp_get_profile(sgp_ctx* c, long long* launches, double* ms) {
  if (!c || !launches || !ms) return SGP_EINVAL;
  DeviceGuard guard(c->device);
  SGP_CUDA(c, cudaStreamSynchronize(c->stream));
  for (int k = 0; k < PK_N; ++k) {
    launches[k] = 0;
    ms[k] = 0.0;
  }
  for (auto& p : c->prof) {
    float t = 0.f;
    SGP_CUDA(c, cudaEventElapsedTime(&t, p.second.first, p.second.second));
    launches[p.first] += 1;
    ms[p.first] += t;
  }
  recycle_events(c);
  return SGP_OK;
}

sgp_status sgp_destroy(sgp_ctx* c) {
  if (!c) return SGP_OK;
  DeviceGuard guard(c->device);
  cudaStreamSynchronize(c->stream);
  free_tables(c);
  cudaFree(c->field);
  for (void* t : c->tw) cudaFree(t);
  cudaFree(c->t_dev);
  cudaFree(c->partials);
  cudaFree(c->obs_dev);
  recycle_events(c);
  for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
  delete c;
  return SGP_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------
// allocation-free observables (sgp_observables_static)
// ----------------------------------------------------------------------------
// Fixed-size scratch in file-scope device arrays.  Host code must not use
// these names as addresses: it looks the device addresses up with
// cudaGetSymbolAddress (once per device) and passes them to the kernels.
namespace {
constexpr int kStaticMaxBatch = 64;
constexpr size_t kStaticMaxPartials = (size_t)1 << 19;     // doubles
constexpr int kStaticMaxN = 1024;

static __device__ __align__(256) double g_static_partials[kStaticMaxPartials];
static __device__ __align__(256) double g_static_sums[kStaticMaxBatch * OB_NT];
static __device__ __align__(256) double2 g_static_tw[3 * kStaticMaxN];   // TwE: 16 B each

struct StaticScratch {
  double* partials = nullptr;
  double* sums = nullptr;
  void* tw = nullptr;
};
constexpr int kMaxDevices = 64;
StaticScratch g_scratch[kMaxDevices];
bool g_scratch_ready[kMaxDevices] = {false};
std::string g_static_err;

sgp_status static_fail(sgp_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_static_err = buf;
  g_create_err = buf;
  return s;
}

// Device addresses of the scratch arrays for the current device (set-up on
// the first call per device).
sgp_status static_scratch(int device, StaticScratch** out) {
  if (device < 0 || device >= kMaxDevices) return static_fail(SGP_EINVAL, "device %d out of range", device);
  if (!g_scratch_ready[device]) {
    StaticScratch sc;
    cudaError_t e;
    if ((e = cudaGetSymbolAddress((void**)&sc.partials, g_static_partials)) != cudaSuccess ||
        (e = cudaGetSymbolAddress((void**)&sc.sums, g_static_sums)) != cudaSuccess ||
        (e = cudaGetSymbolAddress(&sc.tw, g_static_tw)) != cudaSuccess)
      return static_fail(SGP_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_scratch[device] = sc;
    g_scratch_ready[device] = true;
  }
  *out = &g_scratch[device];
  return SGP_OK;
}

template <typename R>
sgp_status observables_static_impl(int dim, const int* nn, const double* LL, int batch,
                                   const sgp_params* prm, double t, const void* field,
                                   cudaStream_t stream, StaticScratch* sc, sgp_obs* out) {
  int n[3] = {1, 1, 1};
  double L[3] = {1, 1, 1}, h[3] = {1, 1, 1};
  for (int a = 0; a < dim; ++a) {
    n[a] = nn[a];
    L[a] = LL[a];
    h[a] = 2.0 * L[a] / n[a];
  }
  const long long ntot = (long long)n[0] * n[1] * n[2];
  const PassGeom gx = xpass_geom<R>(n[0]);
  const int rows = n[1] * n[2];
  const int nbx = (rows + gx.rows_or_tile - 1) / gx.rows_or_tile;
  if ((size_t)nbx * OBX_NT * batch > kStaticMaxPartials)
    return static_fail(SGP_EINVAL, "grid/batch needs %zu partial sums (limit %zu)",
                       (size_t)nbx * OBX_NT * batch, kStaticMaxPartials);
  for (int a = 1; a < dim; ++a) {
    const PassGeom gl = linepass_geom<R>(n[a]);
    const size_t tiles = (size_t)(n[0] + gl.rows_or_tile - 1) / gl.rows_or_tile;
    const size_t planes = a == 1 ? n[2] : n[1];
    if (tiles * planes * OBL_NT * batch > kStaticMaxPartials)
      return static_fail(SGP_EINVAL, "grid/batch needs %zu partial sums (limit %zu)",
                         tiles * planes * OBL_NT * batch, kStaticMaxPartials);
  }
  cudaError_t e;
  // twiddles of every axis into the static table (TwE entries of 16 bytes)
  TwE<R>* tw[3];
  for (int a = 0; a < dim; ++a) {
    tw[a] = reinterpret_cast<TwE<R>*>(reinterpret_cast<char*>(sc->tw) + (size_t)a * kStaticMaxN * 16);
    const int E = elems_for(n[a], sizeof(R) == 4 ? SGP_F32 : SGP_F64);
    if (sizeof(R) == 4)
      k_twiddles_f32<<<(n[a] + 255) / 256, 256, 0, stream>>>(n[a], E, (TwE<float>*)tw[a]);
    else
      k_twiddles_f64<<<(n[a] + 255) / 256, 256, 0, stream>>>(n[a], E, (TwE<double>*)tw[a]);
  }
  // the reduction writes only the slots of the passes that run: start at zero
  if ((e = cudaMemsetAsync(sc->sums, 0, sizeof(double) * (size_t)batch * OB_NT, stream)) != cudaSuccess)
    return static_fail(SGP_ECUDA, "clear sums: %s", cudaGetErrorString(e));
  ObsXArgs<R> ax{};
  ax.ntot = ntot;
  ax.rows = rows;
  ax.ny = n[1];
  ax.x0 = -L[0];
  ax.hx = h[0];
  ax.y0 = -L[1];
  ax.hy = h[1];
  ax.z0 = dim == 3 ? -L[2] : 0.0;
  ax.hz = dim == 3 ? h[2] : 0.0;
  ax.omega = prm->omega;
  ax.t = t;
  ax.c0 = prm->c0;
  ax.c1 = prm->c1;
  ax.c2 = prm->c2;
  ax.gx2h = 0.5 * prm->gx * prm->gx;
  ax.gy2h = 0.5 * prm->gy * prm->gy;
  ax.gz2h = dim == 3 ? 0.5 * prm->gz * prm->gz : 0.0;
  ax.partials = sc->partials;
  ax.nblocks = nbx;
  ax.field = (const cplx<R>*)field;
  ax.tw = tw[0];
  ax.dnu = (R)(kPi / L[0] / n[0]);
  ax.NX = n[0];
  if ((e = launch_obs_x<R>(n[0], ax, batch, stream)) != cudaSuccess)
    return static_fail(SGP_ECUDA, "obs_x: %s", cudaGetErrorString(e));
  k_reduce_partials<<<(batch * OBX_NT + 127) / 128, 128, 0, stream>>>(
      sc->partials, nbx, OBX_NT, batch, sc->sums, OB_NT, 0);
  for (int axis = 1; axis < dim; ++axis) {
    const int NL = n[axis];
    const PassGeom gl = linepass_geom<R>(NL);
    ObsLArgs<R> al{};
    static_cast<ObsArgsBase&>(al) = static_cast<const ObsArgsBase&>(ax);
    al.field = (const cplx<R>*)field;
    al.tw = tw[axis];
    al.nx = n[0];
    const long long nxy = (long long)n[0] * n[1];
    int planes;
    if (axis == 1) {
      al.line_stride = n[0];
      al.plane_stride = nxy;
      planes = n[2];
    } else {
      al.line_stride = nxy;
      al.plane_stride = n[0];
      planes = n[1];
    }
    al.axis = axis;
    al.dnu = (R)(kPi / L[axis] / NL);
    al.NL = NL;
    al.nblocks = ((n[0] + gl.rows_or_tile - 1) / gl.rows_or_tile) * planes;
    if ((e = launch_obs_line<R>(NL, al, planes, batch, stream)) != cudaSuccess)
      return static_fail(SGP_ECUDA, "obs_line: %s", cudaGetErrorString(e));
    k_reduce_partials<<<(batch * OBL_NT + 127) / 128, 128, 0, stream>>>(
        sc->partials, al.nblocks, OBL_NT, batch, sc->sums, OB_NT, axis == 1 ? OB_KY : OB_KZ);
  }
  if ((e = cudaGetLastError()) != cudaSuccess)
    return static_fail(SGP_ECUDA, "launch: %s", cudaGetErrorString(e));
  double hsum[kStaticMaxBatch * OB_NT];   // host staging on the stack, no heap
  if ((e = cudaMemcpyAsync(hsum, sc->sums, sizeof(double) * (size_t)batch * OB_NT,
                           cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(stream)) != cudaSuccess)
    return static_fail(SGP_ECUDA, "read sums: %s", cudaGetErrorString(e));
  const double cell = h[0] * h[1] * (dim == 3 ? h[2] : 1.0);
  bool finite = true;
  for (int m = 0; m < batch; ++m) {
    const double* s = &hsum[(size_t)m * OB_NT];
    sgp_obs o{};
    o.t = t;
    for (int k = 0; k < 5; ++k) {
      o.comp_mass[k] = cell * s[OB_M0 + k];
      o.mass += o.comp_mass[k];
      o.magnetization += (2 - k) * o.comp_mass[k];
    }
    o.width2[0] = cell * s[OB_WX];
    o.width2[1] = cell * s[OB_WY];
    o.width2[2] = cell * s[OB_WZ];
    o.e_kin = cell * (s[OB_KX] + s[OB_KY] + (dim == 3 ? s[OB_KZ] : 0.0));
    o.e_pot = cell * s[OB_POT];
    o.lz = cell * (s[OB_LZX] + s[OB_LZY]);
    o.e_rot = -prm->omega * o.lz;
    o.e_int = cell * s[OB_INT];
    o.e_soc = -prm->gamma * cell * (s[OB_SOCX] + s[OB_SOCY]);
    o.energy = o.e_kin + o.e_pot + o.e_rot + o.e_int + o.e_soc;
    if (!std::isfinite(o.mass) || !std::isfinite(o.energy)) finite = false;
    out[m] = o;
  }
  if (!finite) return static_fail(SGP_ENONFINITE, "non-finite observable");
  return SGP_OK;
}
}  // namespace

extern "C" {

sgp_status sgp_observables_static(int dim, const int* n, const double* L, int batch, int prec,
                                  const sgp_params* p, double t, const void* field_dev,
                                  int device, void* stream, sgp_obs* out) {
  g_create_err.clear();
  if (!n || !L || !p || !field_dev || !out) return static_fail(SGP_EINVAL, "NULL argument");
  if (dim != 2 && dim != 3) return static_fail(SGP_EINVAL, "dim must be 2 or 3 (got %d)", dim);
  if (prec != SGP_F32 && prec != SGP_F64) return static_fail(SGP_EINVAL, "prec must be SGP_F32 or SGP_F64");
  if (batch < 1 || batch > kStaticMaxBatch)
    return static_fail(SGP_EINVAL, "batch must be in [1, %d] (got %d)", kStaticMaxBatch, batch);
  for (int a = 0; a < dim; ++a) {
    if (!supported_n(n[a]) || n[a] > kStaticMaxN)
      return static_fail(SGP_EINVAL, "n[%d] = %d not supported", a, n[a]);
    if (!(L[a] > 0.0) || !std::isfinite(L[a]))
      return static_fail(SGP_EINVAL, "L[%d] must be positive and finite", a);
  }
  if (!finite_params(p) || !std::isfinite(t)) return static_fail(SGP_EINVAL, "non-finite parameter or time");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return static_fail(SGP_EINVAL, "CUDA device %d not available", device);
  DeviceGuard guard(device);
  StaticScratch* sc = nullptr;
  sgp_status st = static_scratch(device, &sc);
  if (st != SGP_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  return prec == SGP_F32 ? observables_static_impl<float>(dim, n, L, batch, p, t, field_dev, s, sc, out)
                         : observables_static_impl<double>(dim, n, L, batch, p, t, field_dev, s, sc, out);
}

}  // extern "C"
