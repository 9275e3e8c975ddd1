// sgp_api.cu -- the C ABI declared in include/sgp.h: contexts and ensembles,
// per-substep tables, pass orchestration of TS2/TS4 (with CUDA-graph replay
// of step chunks) and the observables.
#include <cuda.h>
#include <cudaTypedefs.h>   // the driver's tensor-map encoder, fetched through the runtime
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/sgp.h"
#include "sgp_adjoint.cuh"
#include "sgp_lab.cuh"
#include "sgp_launch.cuh"
#include "sgp_persist.cuh"

using namespace sgp;

namespace {

constexpr double kPi = 3.14159265358979323846;

// TS4 coefficients of Sec. 3.3 (c = 2^(1/3)).
const double kCbrt2 = std::cbrt(2.0);
const double kA1 = 1.0 / (2.0 * (2.0 - kCbrt2));
const double kA2 = (1.0 - kCbrt2) / (2.0 * (2.0 - kCbrt2));
const double kB1 = 1.0 / (2.0 - kCbrt2);
const double kB2 = -kCbrt2 / (2.0 - kCbrt2);

// Steps per captured CUDA graph (sgp_step replays it and runs the rest).
constexpr long long kGraphChunk = 64;

// ----------------------------------------------------------------------------
// table kernels (FP64 arithmetic, stored in the context precision)
// ----------------------------------------------------------------------------
// Rounding of an FP64 unit-direction pair to FP32: the 5x5 neighbourhood
// (+-2 ulp per coordinate) of the rounded pair is searched for the smallest
// ||z| - |target|| + wz |z - target|, so the stored direction is of unit
// modulus to well below an ulp.
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
__device__ inline void tw_angle(int N, int E, int k, double* s_out, double* c_out) {
  int off = 0, ns = radix_at(N, E, 0), st = 1;
  while (true) {
    const int rd = radix_at(N, E, st);
    if (rd <= 0) return;
    const int cnt = (rd - 1) * ns;
    if (k < off + cnt) {
      const int local = k - off;
      const int r = local / ns + 1, j = local - (r - 1) * ns;
      sincospi(-2.0 * (double)(j * r) / (double)(ns * rd), s_out, c_out);
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
  tw_angle(N, E, k, &s, &c);
  const float hx = (float)c, hy = (float)s;
  out[k] = TwE<float>{make_float2(hx, hy), make_float2((float)(c - hx), (float)(s - hy))};
}
__global__ void k_twiddles_f64(int N, int E, TwE<double>* out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  double s = 0.0, c = 1.0;
  tw_angle(N, E, k, &s, &c);
  out[k] = TwE<double>{make_double2(c, s)};
}

// Elements per thread of the line kernels (elems_per_thread<R, N>).
inline int elems_for(int N, int prec) {
  return (N % 3 == 0) ? 6 : (prec == SGP_F32 ? 8 : 4);
}

// Per-mode table of the linear flow over delta (Sec. 3.1, Eq. (sl1)), one
// entry per (|p|, |q|) in the layout MT_* of sgp_kernels.cuh, one table per
// member (blockIdx.y) with that member's Omega and gamma.  The angles are
// formed and the exponentials evaluated in FP64, and the small quantities
// exp(-i chi) - 1, ahat - 1, cp - 1 are written without cancellation:
//   exp(-i chi) - 1 = (-2 sin^2(chi/2), -sin chi),
//   U11 = c - i s Omega/lambda (c, s = cos, sin of delta lambda/2),
//   cp - 1 = -s^2 gamma^2 |nu_perp|^2 / lambda^2 / (1 + cp),
//   ahat - 1 = (c - cp - i s Omega/lambda)/cp,  c - cp = -s^2 Omega^2/lambda^2/(c + cp).
// kz[r] = exp(-i nu_z^2 delta/2) - 1 (shared by all members).
template <typename R>
__global__ void k_linear_tables(double delta, const MemberPrm* mp, int NX, int NY, int NZ,
                                double Lx, double Ly, double Lz, R* mt, long long mt_member,
                                cplx<R>* kz) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  const double omega = mp[m].omega, gamma = mp[m].gamma;
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
    R* e = mt + (size_t)m * mt_member + (size_t)MT_STRIDE * id;
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
  if (m == 0 && id < NZ) {
    const int ks_ = id < NZ / 2 ? id : id - NZ;
    const double nu = kPi * ks_ / Lz;
    double sh, ch;
    sincos(0.25 * nu * nu * delta, &sh, &ch);
    kz[id] = mkc((R)(-2.0 * sh * sh), (R)(-2.0 * sh * ch));
  }
}

// Device FP64 time: set before a run of steps, advanced inside it (so a
// replayed graph advances it too).
__global__ void k_set_time(double* t, double v) { *t = v; }
__global__ void k_add_time(double* t, double v) { *t += v; }

// Copies of many separate buffers in one launch: the ensemble's member
// states between the caller's page-locked host buffers (read and written by
// the GPU through their device mapping) and the member fields.  Entry m
// moves n16 16-byte units from src to dst; its blocks start at block
// `first` (kXferChunk units per block, the last one partial).
struct MemberXfer {
  const uint4* src;
  uint4* dst;
  long long n16;
  long long first;
};
constexpr int kXferThreads = 256;
constexpr int kXferUnroll = 16;
constexpr int kXferChunk = kXferThreads * kXferUnroll;

__global__ void __launch_bounds__(kXferThreads) k_copy_members(const MemberXfer* __restrict__ x, int count) {
  __shared__ int s_m;
  if (threadIdx.x == 0) {
    int lo = 0, hi = count - 1;                 // the last entry whose first block <= blockIdx.x
    const long long b = blockIdx.x;
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (x[mid].first <= b) lo = mid;
      else hi = mid - 1;
    }
    s_m = lo;
  }
  __syncthreads();
  const MemberXfer m = x[s_m];
  const long long base = (blockIdx.x - m.first) * (long long)kXferChunk + threadIdx.x;
  uint4 v[kXferUnroll];
#pragma unroll
  for (int k = 0; k < kXferUnroll; ++k) {
    const long long j = base + (long long)k * kXferThreads;
    if (j < m.n16) v[k] = m.src[j];
  }
#pragma unroll
  for (int k = 0; k < kXferUnroll; ++k) {
    const long long j = base + (long long)k * kXferThreads;
    if (j < m.n16) m.dst[j] = v[k];
  }
}

struct LinTables {
  double delta = 0.0;
  void* mt = nullptr;    // per-mode tables, MT_STRIDE values per (|p|, |q|), per member
  void* kz = nullptr;    // z kinetic factors (NZ entries)
};

struct GraphEntry {
  long long steps;
  double dt;
  int scheme;
  cudaGraphExec_t exec;
};

MemberPrm member_prm(const sgp_params& p, int dim) {
  MemberPrm m;
  m.omega = p.omega;
  m.gamma = p.gamma;
  m.c0 = p.c0;
  m.c1 = p.c1;
  m.c2 = p.c2;
  m.gx2h = 0.5 * p.gx * p.gx;
  m.gy2h = 0.5 * p.gy * p.gy;
  m.gz2h = dim == 3 ? 0.5 * p.gz * p.gz : 0.0;
  return m;
}

// Recorded trajectory for the adjoint: the state every `interval` steps
// (sqrt(nsteps) by default) and the device buffers of the backward sweep.
struct AdjRec {
  bool valid = false;
  long long nsteps = 0, interval = 0, nck = 0;
  double dt = 0.0, t0 = 0.0;
  int scheme = 0;
  void* ckpt = nullptr;            // nck states
  size_t ckpt_cap = 0;
  void* seg = nullptr;             // the states of one recomputed segment
  size_t seg_cap = 0;
  void* g = nullptr;               // adjoint state
  size_t g_cap = 0;
  void* spec = nullptr;            // transform of a substep output
  size_t spec_cap = 0;
  double* dp = nullptr;            // [batch][GP_N]
  size_t dp_cap = 0;
  void* lab = nullptr;             // one member's field, lab-frame output
  size_t lab_cap = 0;
  double* part = nullptr;          // per-block partial sums [batch][blocks][GP_N]
  size_t part_cap = 0;
  // captured full-length segment and what it was captured for
  cudaGraphExec_t graph = nullptr;
  long long graph_len = 0, graph_launches = 0;
  double graph_dt = 0.0;
  int graph_scheme = -1;
  const void* graph_key[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  // pipelined sweep: a second segment buffer, and captured recomputations
  // [0][b] and adjoint sweeps [1][b] of a full segment in buffer b
  void* seg2 = nullptr;
  size_t seg2_cap = 0;
  cudaGraphExec_t pgraph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  long long pgraph_launches[2][2] = {{0, 0}, {0, 0}};
  const void* pgraph_key[2][2][6] = {};
  long long pgraph_len = 0;
  double pgraph_dt = 0.0;
  int pgraph_scheme = -1;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};   // start, recomputed[2], swept[2]
};

void free_adj_pgraphs(AdjRec& r) {
  for (auto& row : r.pgraph)
    for (auto& g : row) {
      if (g) cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

// Device allocator of a context: the caller's (sgp_set_allocator) or
// cudaMalloc/cudaFree when none was set.
struct Allocator {
  sgp_alloc_fn alloc = nullptr;
  sgp_free_fn free = nullptr;
  void* user = nullptr;
};
Allocator g_allocator;     // for contexts created from now on

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
  bool own_stream = false;
  long long ntot = 0;
  size_t elem = 8;
  void* field = nullptr;
  void* tw[3] = {nullptr, nullptr, nullptr};     // twiddles of the default radix plan per axis
  void* tw4[3] = {nullptr, nullptr, nullptr};    // FP32 plan of variant 3 (4 or 12 elements), on demand
  // line-pass variant 4: tensor maps of the field per line axis (made on
  // first use) and the word a tile-load wait that gave up sets
  alignas(64) CUtensorMap tmap[3];
  const void* tmap_field[3] = {nullptr, nullptr, nullptr};   // the field a map was made for
  int* err_dev = nullptr;
  int var[3] = {0, 0, 0};                        // kernel variant per axis (x-pass, y, z lines)
  double* t_dev = nullptr;
  double t = 0.0;
  std::vector<sgp_params> prm;      // per member
  MemberPrm* mp_dev = nullptr;      // per member, on the device
  bool shared_lin = true;           // all members share Omega and gamma
  bool have_state = false;
  std::vector<LinTables> tables;    // cache keyed by delta
  long long tables_gen = 0;         // bumped whenever cached tables are freed
  void* rec = nullptr;              // std::vector<PersistPass<R>>*: passes are recorded, not launched
  std::vector<GraphEntry> graphs;   // captured step chunks
  bool use_graphs = true;
  double* partials = nullptr;       // observables scratch
  size_t partials_len = 0;
  double* obs_dev = nullptr;        // [batch][OB_NT]
  long long launches = 0;
  // profiling: event pairs per launch kind (enabled by sgp_set_profiling)
  bool profiling = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof;
  std::vector<cudaEvent_t> event_pool;
  AdjRec adj;
  // health check of sgp_step
  long long health_every = 0;
  double health_tol = 0.0;
  bool health_ref = false;          // m0 holds the mass at the last set_state
  std::vector<double> m0;
  double* mass_dev = nullptr;       // [batch] + partials
  // member window of the passes: members [win0, win0 + wcnt) (wcnt = 0:
  // the whole batch); set only inside sgp_step_host
  int win0 = 0, wcnt = 0;
  cudaStream_t cs_in = nullptr, cs_out = nullptr;   // copy streams of sgp_step_host
  cudaStream_t cs_alt = nullptr;                    // its second compute stream
  double* t_dev_alt = nullptr;                      // and that stream's device time
  std::vector<cudaEvent_t> pipe_ev;                 // its ordering events
  Allocator alloc;                  // taken from g_allocator at creation
  std::string err;
};

namespace {

std::string g_create_err;

cudaError_t dev_alloc(sgp_ctx* c, void** p, size_t bytes) {
  if (c->alloc.alloc) {
    *p = c->alloc.alloc(bytes, c->device, (void*)c->stream, c->alloc.user);
    if (!*p) return cudaErrorMemoryAllocation;
    if (reinterpret_cast<uintptr_t>(*p) % 16 != 0) {   // kernels copy 16-byte pieces
      c->alloc.free(*p, c->device, (void*)c->stream, c->alloc.user);
      *p = nullptr;
      return cudaErrorMisalignedAddress;
    }
    return cudaSuccess;
  }
  return cudaMalloc(p, bytes);
}

// Frees a buffer of the context.  With the caller's allocator the context
// stream is synchronised first (a pooled block may be handed out again at
// once); cudaFree synchronises by itself.
void dev_free(sgp_ctx* c, void* p) {
  if (!p) return;
  if (c->alloc.free) {
    cudaStreamSynchronize(c->stream);
    c->alloc.free(p, c->device, (void*)c->stream, c->alloc.user);
  } else {
    cudaFree(p);
  }
}

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

#define SGP_TRY(x)                   \
  do {                               \
    sgp_status s_ = (x);             \
    if (s_ != SGP_OK) return s_;     \
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

void free_graphs(sgp_ctx* c) {
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
}

void free_tables(sgp_ctx* c) {
  free_adj_pgraphs(c->adj);
  if (c->adj.graph) {            // the captured adjoint segment points at the tables
    cudaGraphExecDestroy(c->adj.graph);
    c->adj.graph = nullptr;
  }
  for (auto& t : c->tables) {
    dev_free(c, t.mt);
    dev_free(c, t.kz);
  }
  c->tables.clear();
  c->tables_gen++;
}

// Copies the per-member parameters to the device (synchronous) and drops the
// tables and graphs that depend on them.
sgp_status upload_params(sgp_ctx* c) {
  SGP_CUDA(c, cudaStreamSynchronize(c->stream));
  free_graphs(c);
  free_tables(c);
  std::vector<MemberPrm> h(c->batch);
  c->shared_lin = true;
  for (int m = 0; m < c->batch; ++m) {
    h[m] = member_prm(c->prm[m], c->dim);
    if (c->prm[m].omega != c->prm[0].omega || c->prm[m].gamma != c->prm[0].gamma)
      c->shared_lin = false;
  }
  SGP_CUDA(c, cudaMemcpy(c->mp_dev, h.data(), sizeof(MemberPrm) * h.size(), cudaMemcpyHostToDevice));
  return SGP_OK;
}

template <typename R>
sgp_status get_tables(sgp_ctx* c, double delta, const LinTables** out) {
  for (auto& t : c->tables)
    if (t.delta == delta) {
      *out = &t;
      return SGP_OK;
    }
  if (c->tables.size() >= 8) {
    free_graphs(c);      // captured graphs point at the tables
    free_tables(c);
  }
  LinTables t;
  t.delta = delta;
  const int NX = c->n[0], NY = c->n[1], NZ = c->n[2];
  const size_t nent = (size_t)(NX / 2 + 1) * (NY / 2 + 1);
  const int ntab = c->shared_lin ? 1 : c->batch;
  SGP_CUDA(c, dev_alloc(c, &t.mt, nent * MT_STRIDE * sizeof(R) * ntab));
  SGP_CUDA(c, dev_alloc(c, &t.kz, (size_t)NZ * sizeof(cplx<R>)));
  const int work = (int)std::max<size_t>(nent, (size_t)NZ);
  {
    ProfScope ps(c, PK_TAB);
    dim3 grid((work + 255) / 256, ntab);
    k_linear_tables<R><<<grid, 256, 0, c->stream>>>(delta, c->mp_dev, NX, NY, NZ, c->L[0],
                                                    c->L[1], c->L[2], (R*)t.mt,
                                                    (long long)(nent * MT_STRIDE), (cplx<R>*)t.kz);
  }
  c->launches++;
  SGP_CUDA(c, cudaGetLastError());
  c->tables.push_back(t);
  *out = &c->tables.back();
  return SGP_OK;
}

// ----------------------------------------------------------------------------
// passes
// ----------------------------------------------------------------------------
// members the passes work on and the field of the first of them
int window_members(const sgp_ctx* c) { return c->wcnt ? c->wcnt : c->batch; }
void* window_field(sgp_ctx* c) {
  return (char*)c->field + (size_t)c->win0 * 5 * c->ntot * c->elem;
}

// The driver's cuTensorMapEncodeTiled, through the runtime (no link to the
// driver library); null when the driver does not provide it.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  }
  return fn;
}

// Tensor map of the FP32 field for the line pass along `axis` (variant 4):
// 4D, [5 * batch][nz][ny][nx] of 8-byte elements, x innermost; the box is
// TILE columns by tma_rows(N) line elements (y for axis 1, z for axis 2).
// The map holds the address of the batch it covers (base): the context's
// field, the autotuner's scratch copy, or a buffer of the adjoint sweep; it
// is made again whenever a pass works on another one (a map travels by
// value into the kernel's parameters, also into captured graphs).
sgp_status ensure_tmap(sgp_ctx* c, int axis, void* base) {
  if (c->tmap_field[axis] == base) return SGP_OK;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return fail(c, SGP_EUNSUPPORTED, "the driver has no tensor-map encoder (variant 4)");
  const int N = c->n[axis];
  const cuuint32_t tile = (cuuint32_t)linepass_geom<float>(N, 4).rows_or_tile;
  int rows = 1;
  for (int d = 1; d <= N; ++d)
    if (N % d == 0 && N / d <= 256) {
      rows = N / d;
      break;
    }
  const cuuint64_t nx = (cuuint64_t)c->n[0], ny = (cuuint64_t)c->n[1], nz = (cuuint64_t)c->n[2];
  const cuuint64_t dims[4] = {nx, ny, nz, (cuuint64_t)5 * c->batch};
  const cuuint64_t strides[3] = {nx * 8, nx * ny * 8, nx * ny * nz * 8};
  const cuuint32_t box[4] = {tile, axis == 1 ? (cuuint32_t)rows : 1u, axis == 2 ? (cuuint32_t)rows : 1u, 1u};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = enc(&c->tmap[axis], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, base, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(c, SGP_ECUDA, "tensor map for axis %d: driver error %d", axis, (int)r);
  c->tmap_field[axis] = base;
  return SGP_OK;
}

// Is x-pass variant 5 usable here (3D FP32 grid with NX = NY = 64 or 128)?
bool plane_ok(const sgp_ctx* c) {
  return c->prec == SGP_F32 && c->dim == 3 && c->n[0] == c->n[1] && (c->n[0] == 64 || c->n[0] == 128);
}
// The steps' x-passes are xy-plane passes (x-pass variant 5): they also do
// the y transforms, and the linear flow between them is the z-line pass
// alone.  Not while passes are recorded for the persistent ensemble kernel,
// which has no plane pass.
bool plane_pass(const sgp_ctx* c) { return c->var[0] == 5 && !c->rec; }

template <typename R>
XPassArgs<R> x_args(const sgp_ctx* c, void* field, int mode, double delta, double t_off) {
  XPassArgs<R> a{};
  a.field = (cplx<R>*)field;
  a.tw = (const TwE<R>*)(c->var[0] == 3 ? c->tw4[0] : c->tw[0]);
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
  a.mp = c->mp_dev + c->win0;
  a.t_base = c->t_dev;
  a.t_off = t_off;
  return a;
}

template <typename R>
sgp_status x_pass_on(sgp_ctx* c, void* field, int mode, double delta, double t_off) {
  XPassArgs<R> a = x_args<R>(c, field, mode, delta, t_off);
  if (c->rec) {
    // recorded for the persistent ensemble kernel (default radix plan)
    PersistPass<R> p{};
    a.tw = (const TwE<R>*)c->tw[0];
    p.kind = PK_XPASS;
    p.N = c->n[0];
    const int rows = persist_xrows<R>(c->n[0]);
    p.tiles = (a.rows + rows - 1) / rows;
    p.members = window_members(c);
    p.x = a;
    static_cast<std::vector<PersistPass<R>>*>(c->rec)->push_back(p);
    return SGP_OK;
  }
  c->launches++;
  ProfScope ps(c, PK_X);
  SGP_CUDA(c, launch_xpass<R>(c->n[0], c->var[0], a, window_members(c), c->stream));
  return SGP_OK;
}

// xy-plane pass (x-pass variant 5, FP32): the x-pass with the y transforms,
// one cluster per z plane of each member
template <typename R>
sgp_status xy_pass_on(sgp_ctx* c, void* field, int mode, double delta, double t_off) {
  if constexpr (sizeof(R) != 4) {
    return fail(c, SGP_EINVAL, "the xy-plane pass is FP32 only");
  } else {
    const XPassArgs<R> a = x_args<R>(c, field, mode, delta, t_off);
    c->launches++;
    ProfScope ps(c, PK_X);
    SGP_CUDA(c, launch_xyplane(c->n[0], a, (const TwE<R>*)c->tw[1], c->err_dev, c->n[2],
                                window_members(c), c->stream));
    return SGP_OK;
  }
}

// the x-passes of the steps and substeps (xy-plane passes under variant 5)
template <typename R>
sgp_status x_pass(sgp_ctx* c, int mode, double delta, double t_off) {
  if (plane_pass(c)) return xy_pass_on<R>(c, window_field(c), mode, delta, t_off);
  return x_pass_on<R>(c, window_field(c), mode, delta, t_off);
}

// axis 1: lines along y (planes = z slices); axis 2: lines along z (planes = y rows)
template <typename R>
sgp_status line_pass_on(sgp_ctx* c, void* field, int axis, int mode, const LinTables* t) {
  LPassArgs<R> a{};
  a.field = (cplx<R>*)field;
  a.tw = (const TwE<R>*)(c->var[axis] == 3 ? c->tw4[axis] : c->tw[axis]);
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
    a.mt_member = c->shared_lin ? 0 : (long long)(c->n[0] / 2 + 1) * (c->n[1] / 2 + 1) * MT_STRIDE;
    a.mt = (const R*)t->mt + (size_t)c->win0 * a.mt_member;
    a.kz = (const cplx<R>*)t->kz;
  }
  {
    const double inv = 1.0 / ((double)c->n[0] * c->n[1] * (c->dim == 3 ? c->n[2] : 1));
    a.inv_hi = (R)inv;
    a.inv_lo = (R)(inv - (double)a.inv_hi);
  }
  a.mc0 = c->win0;
  a.err = c->err_dev;
  if (c->rec) {
    // recorded for the persistent ensemble kernel (2D: lines along y)
    PersistPass<R> p{};
    a.tw = (const TwE<R>*)c->tw[axis];
    p.kind = PK_LINE;
    p.N = c->n[axis];
    const int tile = persist_ltile<R>(c->n[axis]);
    p.tiles = ((a.nx + tile - 1) / tile) * planes;
    p.members = window_members(c);
    p.l = a;
    static_cast<std::vector<PersistPass<R>>*>(c->rec)->push_back(p);
    return SGP_OK;
  }
  if constexpr (sizeof(R) == 4) {
    if (c->var[axis] == 4) {
      // the batch the window's field belongs to (member coordinates mc0 + m)
      char* batch_base = (char*)field - (size_t)c->win0 * 5 * c->ntot * c->elem;
      SGP_TRY(ensure_tmap(c, axis, batch_base));
      c->launches++;
      ProfScope ps(c, axis == 1 ? PK_Y : PK_Z);
      SGP_CUDA(c, launch_linepass_tma(c->n[axis], a, c->tmap[axis], planes, window_members(c), c->stream));
      return SGP_OK;
    }
  }
  c->launches++;
  ProfScope ps(c, axis == 1 ? PK_Y : PK_Z);
  SGP_CUDA(c, launch_linepass<R>(c->n[axis], c->var[axis], a, planes, window_members(c), c->stream));
  return SGP_OK;
}

template <typename R>
sgp_status line_pass(sgp_ctx* c, int axis, int mode, const LinTables* t) {
  return line_pass_on<R>(c, window_field(c), axis, mode, t);
}

// Linear flow over delta between x-passes.  Entry: x-spectral (the x-pass
// has done its forward transform; with xy, x- and y-spectral: the x-passes
// are xy-plane passes).  Exit: the same.
template <typename R>
sgp_status linear_middle_on(sgp_ctx* c, void* f, double delta, bool xy = false) {
  const LinTables* t = nullptr;
  SGP_TRY(get_tables<R>(c, delta, &t));
  if (c->dim == 2) {
    SGP_TRY(line_pass_on<R>(c, f, 1, LP_FWD | LP_MIX | LP_INV, t));
  } else if (xy) {
    SGP_TRY(line_pass_on<R>(c, f, 2, LP_FWD | LP_MIX | LP_INV, t));
  } else {
    SGP_TRY(line_pass_on<R>(c, f, 1, LP_FWD, nullptr));
    SGP_TRY(line_pass_on<R>(c, f, 2, LP_FWD | LP_MIX | LP_INV, t));
    SGP_TRY(line_pass_on<R>(c, f, 1, LP_INV, nullptr));
  }
  return SGP_OK;
}

template <typename R>
sgp_status linear_middle(sgp_ctx* c, double delta) {
  return linear_middle_on<R>(c, window_field(c), delta, plane_pass(c));
}

// substep pattern of one step, Sec. 3.3
std::vector<std::pair<char, double>> scheme_seq(int scheme) {
  switch (scheme) {
    case SGP_TS2: return {{'N', 0.5}, {'L', 1.0}, {'N', 0.5}};
    case SGP_TS2_LNL: return {{'L', 0.5}, {'N', 1.0}, {'L', 0.5}};
    case SGP_TS4_LOUTER:
      return {{'L', kA1}, {'N', kB1}, {'L', kA2}, {'N', kB2}, {'L', kA2}, {'N', kB1}, {'L', kA1}};
    default:
      return {{'N', kA1}, {'L', kB1}, {'N', kA2}, {'L', kB2}, {'N', kA2}, {'L', kB1}, {'N', kA1}};
  }
}

bool valid_scheme(int scheme) {
  return scheme == SGP_TS2 || scheme == SGP_TS4 || scheme == SGP_TS2_LNL || scheme == SGP_TS4_LOUTER;
}

struct SubRec {
  char kind;
  double delta;
  double toff;     // time of the substep relative to the start of the run
};

// Substeps of n steps of the scheme, with the substeps of the same kind that
// meet at a step boundary merged: nonlinear flows at the same time (the flow
// of Eq. (solution2) over a then b is the flow over a + b) and linear flows
// (time-independent in the rotating frame, so L(a) L(b) = L(a + b)).  Time
// advances in the linear substeps; a nonlinear substep at the end of step s
// is at (s + 1) dt, a linear one carries its start time.
std::vector<SubRec> merged_substeps(int scheme, long long n, double dt) {
  const auto seq = scheme_seq(scheme);
  std::vector<SubRec> subs;
  for (long long s = 0; s < n; ++s) {
    double sub = 0.0;
    for (size_t k = 0; k < seq.size(); ++k) {
      const double delta = seq[k].second * dt;
      const char kind = seq[k].first;
      // a nonlinear flow acts at the current time (the end of step s exactly
      // (s + 1) dt); a linear flow is stamped with its start time
      const double toff = (kind == 'N' && k == seq.size() - 1) ? (double)(s + 1) * dt
                                                                 : (double)s * dt + sub * dt;
      if (kind == 'L') sub += seq[k].second;
      if (k == 0 && !subs.empty() && subs.back().kind == kind)
        subs.back().delta += delta;        // meets the previous step's last substep
      else
        subs.push_back({kind, delta, toff});
    }
  }
  return subs;
}

// Issue nsteps of the composition from the device time *t_dev and advance
// it by nsteps*dt, physical space in and out.  The merged substeps become
// passes: a nonlinear flow is an x-pass (inverse x-FFT if the field is
// x-spectral, the flow, forward x-FFT if a linear flow follows); a linear
// flow is the line passes on the x-spectral field (a forward x-pass first if
// the field is physical).  With the nonlinear flow outside (TS2, TS4) a step
// is N L N L ... with one x-pass per N; with the linear flow outside the
// run starts with a forward x-pass and ends with an inverse one.
template <typename R>
sgp_status emit_steps(sgp_ctx* c, long long nsteps, double dt, int scheme) {
  const std::vector<SubRec> subs = merged_substeps(scheme, nsteps, dt);
  bool xspec = false;
  for (size_t j = 0; j < subs.size(); ++j) {
    if (subs[j].kind == 'N') {
      int mode = XP_NL | (xspec ? XP_INV : 0);
      xspec = (j + 1 < subs.size());
      if (xspec) mode |= XP_FWD;
      SGP_TRY(x_pass<R>(c, mode, subs[j].delta, subs[j].toff));
    } else {
      if (!xspec) SGP_TRY(x_pass<R>(c, XP_FWD, 0.0, 0.0));
      xspec = true;
      SGP_TRY(linear_middle<R>(c, subs[j].delta));
    }
  }
  if (xspec) SGP_TRY(x_pass<R>(c, XP_INV, 0.0, 0.0));
  if (c->rec) return SGP_OK;           // recording passes only; the caller advances the time
  c->launches++;
  {
    ProfScope ps(c, PK_OTHER);
    k_add_time<<<1, 1, 0, c->stream>>>(c->t_dev, (double)nsteps * dt);
  }
  SGP_CUDA(c, cudaGetLastError());
  return SGP_OK;
}

// Tables for every linear substep size a run of the scheme uses, merged ones
// included (before a capture).
template <typename R>
sgp_status ensure_tables(sgp_ctx* c, double dt, int scheme) {
  // two passes: a full cache is emptied when a new table is made, which can
  // drop a table the first pass made; the second makes it again (a scheme
  // needs at most three sizes, so it evicts nothing)
  for (int pass = 0; pass < 2; ++pass)
    for (auto& st : merged_substeps(scheme, 3, dt))
      if (st.kind == 'L') {
        const LinTables* t = nullptr;
        SGP_TRY(get_tables<R>(c, st.delta, &t));
      }
  return SGP_OK;
}

// Captured chunk of `steps` steps on the context stream (cached).
template <typename R>
sgp_status get_graph(sgp_ctx* c, long long steps, double dt, int scheme, cudaGraphExec_t* out) {
  for (auto& g : c->graphs)
    if (g.steps == steps && g.dt == dt && g.scheme == scheme) {
      *out = g.exec;
      return SGP_OK;
    }
  if (c->graphs.size() >= 8) free_graphs(c);
  SGP_TRY(ensure_tables<R>(c, dt, scheme));
  const long long launches0 = c->launches;
  SGP_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  sgp_status st = emit_steps<R>(c, steps, dt, scheme);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
  c->launches = launches0;      // counted when replayed
  if (st != SGP_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return fail(c, SGP_ECUDA, "stream capture: %s", cudaGetErrorString(e));
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(c, SGP_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  c->graphs.push_back({steps, dt, scheme, exec});
  *out = exec;
  return SGP_OK;
}

// Launches issued by one chunk of `steps` steps (for the launch counter):
// the pass count of emit_steps plus the time update.
long long chunk_launches(const sgp_ctx* c, long long steps, int scheme) {
  const long long per_l = (c->dim == 2 || plane_pass(c)) ? 1 : 3;
  long long n = 1;
  bool xspec = false;
  const std::vector<SubRec> subs = merged_substeps(scheme, steps, 1.0);
  for (size_t j = 0; j < subs.size(); ++j) {
    if (subs[j].kind == 'N') {
      n += 1;
      xspec = (j + 1 < subs.size());
    } else {
      n += (xspec ? 0 : 1) + per_l;
      xspec = true;
    }
  }
  return n + (xspec ? 1 : 0);
}

template <typename R>
sgp_status run_steps(sgp_ctx* c, long long nsteps, double dt, int scheme) {
  c->launches++;
  {
    ProfScope ps(c, PK_OTHER);
    k_set_time<<<1, 1, 0, c->stream>>>(c->t_dev, c->t);
  }
  SGP_CUDA(c, cudaGetLastError());
  long long done = 0;
  if (c->use_graphs && !c->profiling && c->wcnt == 0 && nsteps >= 2 * kGraphChunk) {
    cudaGraphExec_t exec = nullptr;
    SGP_TRY(get_graph<R>(c, kGraphChunk, dt, scheme, &exec));
    const long long reps = nsteps / kGraphChunk;
    for (long long r = 0; r < reps; ++r) SGP_CUDA(c, cudaGraphLaunch(exec, c->stream));
    c->launches += reps * chunk_launches(c, kGraphChunk, scheme);
    done = reps * kGraphChunk;
  }
  if (done < nsteps) SGP_TRY(emit_steps<R>(c, nsteps - done, dt, scheme));
  c->t += (double)nsteps * dt;
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
// host-to-host propagation with the copies overlapped (sgp_step_host)
// ----------------------------------------------------------------------------
// The batch is split into `chunks` member groups.  All copies to the device
// are issued on cs_in; each group's steps run after its copy has landed
// (the passes restricted to the group by the member window), alternately
// on the context stream and on cs_alt with its own device time, so that
// the last passes of one group overlap the first of the next; each group's
// copy back runs on cs_out after its steps.  The copy engines move group
// k+1 in and group k-1 out while group k is propagated.
template <typename R>
sgp_status step_host_impl(sgp_ctx* c, const void* hin, double t0, void* hout, long long nsteps,
                          double dt, int scheme, int chunks) {
  if (!c->cs_in) SGP_CUDA(c, cudaStreamCreateWithFlags(&c->cs_in, cudaStreamNonBlocking));
  if (!c->cs_out) SGP_CUDA(c, cudaStreamCreateWithFlags(&c->cs_out, cudaStreamNonBlocking));
  if (!c->cs_alt) SGP_CUDA(c, cudaStreamCreateWithFlags(&c->cs_alt, cudaStreamNonBlocking));
  if (!c->t_dev_alt) SGP_CUDA(c, dev_alloc(c, (void**)&c->t_dev_alt, sizeof(double)));
  // the linear-flow tables of the run exist before the streams fork
  if (nsteps > 0) SGP_TRY(ensure_tables<R>(c, dt, scheme));
  const size_t nev = 2 * (size_t)chunks + 2;
  while (c->pipe_ev.size() < nev) {
    cudaEvent_t e = nullptr;
    SGP_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    c->pipe_ev.push_back(e);
  }
  cudaEvent_t* ev = c->pipe_ev.data();   // [0] start, [1] end, then in[k], done[k]
  const size_t mb = (size_t)5 * c->ntot * c->elem;
  std::vector<int> m0(chunks + 1);
  for (int k = 0; k <= chunks; ++k) m0[k] = (int)((long long)c->batch * k / chunks);
  // earlier work of the context stream on the field comes first
  SGP_CUDA(c, cudaEventRecord(ev[0], c->stream));
  SGP_CUDA(c, cudaStreamWaitEvent(c->cs_in, ev[0], 0));
  SGP_CUDA(c, cudaStreamWaitEvent(c->cs_out, ev[0], 0));
  SGP_CUDA(c, cudaStreamWaitEvent(c->cs_alt, ev[0], 0));
  for (int k = 0; k < chunks; ++k) {
    const size_t off = (size_t)m0[k] * mb, bytes = (size_t)(m0[k + 1] - m0[k]) * mb;
    SGP_CUDA(c, cudaMemcpyAsync((char*)c->field + off, (const char*)hin + off, bytes,
                                cudaMemcpyHostToDevice, c->cs_in));
    SGP_CUDA(c, cudaEventRecord(ev[2 + k], c->cs_in));
  }
  c->adj.valid = false;
  c->health_ref = false;
  c->have_state = true;
  sgp_status st = SGP_OK;
  for (int k = 0; k < chunks && st == SGP_OK; ++k) {
    const size_t off = (size_t)m0[k] * mb, bytes = (size_t)(m0[k + 1] - m0[k]) * mb;
    // odd groups on the second compute stream with its own device time
    const bool alt = (k & 1) != 0;
    if (alt) {
      std::swap(c->stream, c->cs_alt);
      std::swap(c->t_dev, c->t_dev_alt);
    }
    cudaError_t e = cudaStreamWaitEvent(c->stream, ev[2 + k], 0);
    c->win0 = m0[k];
    c->wcnt = m0[k + 1] - m0[k];
    c->t = t0;
    if (e != cudaSuccess)
      st = fail(c, SGP_ECUDA, "stream wait: %s", cudaGetErrorString(e));
    else if (nsteps > 0)
      st = run_steps<R>(c, nsteps, dt, scheme);
    c->win0 = 0;
    c->wcnt = 0;
    if (st == SGP_OK) e = cudaEventRecord(ev[2 + chunks + k], c->stream);
    if (alt) {
      std::swap(c->stream, c->cs_alt);
      std::swap(c->t_dev, c->t_dev_alt);
    }
    if (st != SGP_OK) break;
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->cs_out, ev[2 + chunks + k], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync((char*)hout + off, (const char*)c->field + off, bytes,
                          cudaMemcpyDeviceToHost, c->cs_out);
    if (e != cudaSuccess) st = fail(c, SGP_ECUDA, "copy back: %s", cudaGetErrorString(e));
  }
  c->t = t0 + (double)nsteps * dt;
  // later work of the context stream comes after the copies back; the host
  // buffers are done with when this returns, also after an error
  cudaError_t e = cudaEventRecord(ev[1], c->cs_out);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, ev[1], 0);
  const cudaError_t e1 = cudaStreamSynchronize(c->cs_in);
  const cudaError_t e2 = cudaStreamSynchronize(c->cs_out);
  const cudaError_t e3 = cudaStreamSynchronize(c->stream);
  const cudaError_t e4 = cudaStreamSynchronize(c->cs_alt);
  if (st != SGP_OK) return st;
  for (cudaError_t x : {e, e1, e2, e3, e4})
    if (x != cudaSuccess) return fail(c, SGP_ECUDA, "sgp_step_host: %s", cudaGetErrorString(x));
  return SGP_OK;
}

// ----------------------------------------------------------------------------
// adjoint: checkpointed record and backward sweep
// ----------------------------------------------------------------------------
size_t state_bytes(const sgp_ctx* c) { return (size_t)c->batch * 5 * c->ntot * c->elem; }

sgp_status ensure_buf(sgp_ctx* c, void** p, size_t* cap, size_t bytes) {
  if (*cap >= bytes && *p) return SGP_OK;
  SGP_CUDA(c, cudaStreamSynchronize(c->stream));
  dev_free(c, *p);
  *p = nullptr;
  *cap = 0;
  SGP_CUDA(c, dev_alloc(c, p, bytes));
  *cap = bytes;
  return SGP_OK;
}

void free_adj(sgp_ctx* c) {
  AdjRec& r = c->adj;
  if (r.graph) cudaGraphExecDestroy(r.graph);
  free_adj_pgraphs(r);
  for (cudaEvent_t e : r.ev)
    if (e) cudaEventDestroy(e);
  dev_free(c, r.ckpt);
  dev_free(c, r.seg);
  dev_free(c, r.seg2);
  dev_free(c, r.g);
  dev_free(c, r.spec);
  dev_free(c, r.dp);
  dev_free(c, r.part);
  dev_free(c, r.lab);
  r = AdjRec();
}

// Forward run of nsteps that stores the state at the start of every chunk
// of `interval` steps.  The chunks run on the ordinary step path.
template <typename R>
sgp_status record_steps(sgp_ctx* c, long long nsteps, double dt, int scheme, long long interval) {
  AdjRec& r = c->adj;
  r.valid = false;
  if (interval <= 0) interval = (long long)std::ceil(std::sqrt((double)nsteps));
  if (interval > nsteps) interval = nsteps;
  const long long nck = (nsteps + interval - 1) / interval;
  const size_t sb = state_bytes(c);
  SGP_TRY(ensure_buf(c, &r.ckpt, &r.ckpt_cap, sb * (size_t)nck));
  r.t0 = c->t;
  for (long long k = 0; k < nck; ++k) {
    SGP_CUDA(c, cudaMemcpyAsync((char*)r.ckpt + sb * (size_t)k, c->field, sb,
                                cudaMemcpyDeviceToDevice, c->stream));
    const long long n = std::min(interval, nsteps - k * interval);
    SGP_TRY(run_steps<R>(c, n, dt, scheme));
  }
  r.nsteps = nsteps;
  r.interval = interval;
  r.nck = nck;
  r.dt = dt;
  r.scheme = scheme;
  r.valid = true;
  return SGP_OK;
}

// Rows of the parameter partials per member: one per CTA of the adjoint
// x-pass, then one per CTA of the line pass that holds the full transform
// (y lines in 2D, z lines in 3D).
template <typename R>
int adjoint_prows(const sgp_ctx* c) {
  const int axis = c->dim == 2 ? 1 : 2;
  const int planes = c->dim == 2 ? c->n[2] : c->n[1];
  return xadj_ctas<R>(c->n[0], c->n[1] * c->n[2]) + linepass_adj_tiles<R>(c->n[axis], c->n[0]) * planes;
}

// g <- (D N_d(Phi_in))^T g at Phi_out = phi (physical space), plus the
// parameter terms; with XP_INV g comes in x-spectral (the inverse
// x-transform first), with XP_FWD it leaves x-spectral
template <typename R>
sgp_status adjoint_nonlinear(sgp_ctx* c, const void* phi, double delta, double t_off, int mode) {
  XAdjArgs<R> a{};
  a.g = (cplx<R>*)c->adj.g;
  a.phi = (const cplx<R>*)phi;
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
  a.delta = delta;
  a.t_base = c->t_dev;
  a.t_off = t_off;
  a.mp = c->mp_dev;
  a.partials = c->adj.part;
  a.prows = adjoint_prows<R>(c);
  c->launches++;
  ProfScope ps(c, PK_X);
  SGP_CUDA(c, launch_xadj<R>(c->n[0], a, c->batch, c->stream));
  return SGP_OK;
}

// The linear flow over delta on the x-spectral field f through the line
// pass of a gradient (in 3D between the y-line transforms), the field left
// x-spectral.  h: its hooks (the parameter terms of the sweep or the copy
// of the recomputation).
template <typename R>
sgp_status linear_hooked(sgp_ctx* c, void* f, double delta, const AdjHook<R>& h) {
  const LinTables* t = nullptr;
  SGP_TRY(get_tables<R>(c, delta, &t));
  const int axis = c->dim == 2 ? 1 : 2;
  if (c->dim == 3) SGP_TRY(line_pass_on<R>(c, f, 1, LP_FWD, nullptr));
  LPassArgs<R> a{};
  a.field = (cplx<R>*)f;
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
  a.mode = LP_FWD | LP_MIX | LP_INV;
  a.axis = axis;
  a.NX = c->n[0];
  a.NY = c->n[1];
  a.mt_member = c->shared_lin ? 0 : (long long)(c->n[0] / 2 + 1) * (c->n[1] / 2 + 1) * MT_STRIDE;
  a.mt = (const R*)t->mt;
  a.kz = (const cplx<R>*)t->kz;
  {
    const double inv = 1.0 / ((double)c->n[0] * c->n[1] * (c->dim == 3 ? c->n[2] : 1));
    a.inv_hi = (R)inv;
    a.inv_lo = (R)(inv - (double)a.inv_hi);
  }
  a.err = c->err_dev;
  c->launches++;
  {
    ProfScope ps(c, axis == 1 ? PK_Y : PK_Z);
    SGP_CUDA(c, launch_linepass_adj<R>(c->n[axis], a, h, planes, c->batch, c->stream));
  }
  if (c->dim == 3) SGP_TRY(line_pass_on<R>(c, f, 1, LP_INV, nullptr));
  return SGP_OK;
}

// g <- L(-d) g on the x-spectral g, with the Omega and gamma terms of every
// mode; phi_tap: the recomputation's copy of the substep's output after the
// mix (its full transform divided by the number of grid points, so the
// products of the two transforms sum over the grid with scale 1)
template <typename R>
sgp_status adjoint_linear(sgp_ctx* c, double delta, const void* phi_tap) {
  AdjHook<R> h{};
  h.spec = (const cplx<R>*)phi_tap;
  h.mp = c->mp_dev;
  h.partials = c->adj.part;
  h.prows = adjoint_prows<R>(c);
  h.prow0 = xadj_ctas<R>(c->n[0], c->n[1] * c->n[2]);
  const int axis = c->dim == 2 ? 1 : 2;
  h.tiles = linepass_adj_tiles<R>(c->n[axis], c->n[0]);
  h.Lx = c->L[0];
  h.Ly = c->L[1];
  h.delta = delta;
  h.scale = 1.0;
  return linear_hooked<R>(c, c->adj.g, -delta, h);
}

// Substeps of a recomputed segment of n steps (times relative to its start).
std::vector<SubRec> segment_substeps(int scheme, long long n, double dt) {
  return merged_substeps(scheme, n, dt);
}

// The states of a segment recomputed from seg[0] (the segment's start) with
// the passes of the forward steps, working in place on seg[0]: the output
// of nonlinear substep j is copied to seg[j + 1] (physical space) by the
// x-pass after its flow, and the output of the k-th linear substep, after
// the mix, to spec[k] (its transform over the number of grid points) by
// the line pass.  Times relative to the segment start on the device clock.
template <typename R>
sgp_status emit_recompute(sgp_ctx* c, const std::vector<SubRec>& subs, char* seg, char* spec) {
  const size_t sb = state_bytes(c);
  size_t nl = 0;
  bool xspec = false;
  for (size_t j = 0; j < subs.size(); ++j) {
    if (subs[j].kind == 'N') {
      int mode = XP_NL | (xspec ? XP_INV : 0);
      xspec = (j + 1 < subs.size());
      if (xspec) mode |= XP_FWD;
      XPassArgs<R> a = x_args<R>(c, seg, mode, subs[j].delta, subs[j].toff);
      a.tw = (const TwE<R>*)c->tw[0];
      a.tap = (cplx<R>*)(seg + sb * (j + 1));
      c->launches++;
      ProfScope ps(c, PK_X);
      SGP_CUDA(c, launch_xpass_tap<R>(c->n[0], a, c->batch, c->stream));
    } else {
      if (!xspec) SGP_TRY(x_pass_on<R>(c, seg, XP_FWD, 0.0, 0.0));
      xspec = true;
      AdjHook<R> h{};
      h.tap = (cplx<R>*)(spec + sb * nl++);
      SGP_TRY(linear_hooked<R>(c, seg, subs[j].delta, h));
    }
  }
  return SGP_OK;
}

// g carried back through a recomputed segment's substeps in reverse order.
// g stays x-spectral between a linear substep and the nonlinear one before
// it, as the field does between the forward passes: a nonlinear substep is
// one adjoint x-pass (the inverse x-transform of the linear substep after
// it and the forward x-transform of the one before it fused in), a linear
// substep one line pass of a gradient (2D; in 3D with the two y-line
// passes).  g is physical at the segment's ends.
template <typename R>
sgp_status emit_adjoint(sgp_ctx* c, const std::vector<SubRec>& subs, const char* seg, const char* spec) {
  AdjRec& r = c->adj;
  const size_t sb = state_bytes(c);
  size_t nl = 0;
  for (const SubRec& q : subs) nl += q.kind == 'L';
  bool xspec = false;
  for (size_t j = subs.size(); j-- > 0;) {
    if (subs[j].kind == 'N') {
      int mode = xspec ? XP_INV : 0;
      if (j > 0 && subs[j - 1].kind == 'L') mode |= XP_FWD;
      SGP_TRY(adjoint_nonlinear<R>(c, seg + sb * (j + 1), subs[j].delta, subs[j].toff, mode));
      xspec = (mode & XP_FWD) != 0;
    } else {
      if (!xspec) SGP_TRY(x_pass_on<R>(c, r.g, XP_FWD, 0.0, 0.0));
      SGP_TRY(adjoint_linear<R>(c, subs[j].delta, spec + sb * --nl));
      xspec = true;
    }
  }
  if (xspec) SGP_TRY(x_pass_on<R>(c, r.g, XP_INV, 0.0, 0.0));
  return SGP_OK;
}

// One segment: the recomputation, then the adjoint sweep through it (the
// linear substeps' copies spec_off bytes into the segment buffer).
template <typename R>
sgp_status emit_segment(sgp_ctx* c, const std::vector<SubRec>& subs, size_t spec_off) {
  char* seg = (char*)c->adj.seg;
  SGP_TRY(emit_recompute<R>(c, subs, seg, seg + spec_off));
  return emit_adjoint<R>(c, subs, seg, seg + spec_off);
}

void free_adj_graph(sgp_ctx* c) {
  if (c->adj.graph) cudaGraphExecDestroy(c->adj.graph);
  c->adj.graph = nullptr;
}

// Captured full-length segment (cached; rebuilt when the run, the buffers or
// the tables change).
template <typename R>
sgp_status segment_graph(sgp_ctx* c, const std::vector<SubRec>& subs, size_t spec_off, cudaGraphExec_t* out) {
  AdjRec& r = c->adj;
  const void* key[5] = {r.seg, r.g, r.spec, r.part, c->t_dev};
  if (r.graph && r.graph_len == r.interval && r.graph_dt == r.dt &&
      r.graph_scheme == r.scheme && std::memcmp(key, r.graph_key, sizeof key) == 0) {
    *out = r.graph;
    return SGP_OK;
  }
  free_adj_graph(c);
  const long long launches0 = c->launches;
  SGP_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  sgp_status st = emit_segment<R>(c, subs, spec_off);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
  r.graph_launches = c->launches - launches0;
  c->launches = launches0;
  if (st != SGP_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return fail(c, SGP_ECUDA, "stream capture: %s", cudaGetErrorString(e));
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(c, SGP_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  r.graph = exec;
  r.graph_len = r.interval;
  r.graph_dt = r.dt;
  r.graph_scheme = r.scheme;
  std::memcpy(r.graph_key, key, sizeof key);
  *out = exec;
  return SGP_OK;
}

// Captured recomputation (kind 0) or adjoint sweep (kind 1) of a full
// segment in buffer b, issued on the current c->stream with the current
// c->t_dev (cached per kind and buffer; rebuilt when the run, the buffers
// or the tables change).
template <typename R>
sgp_status pipe_graph(sgp_ctx* c, int kind, int b, const std::vector<SubRec>& subs, char* seg, char* spec,
                      cudaGraphExec_t* out) {
  AdjRec& r = c->adj;
  const void* key[6] = {seg, r.g, r.spec, r.part, c->t_dev, c->stream};
  if (r.pgraph_len != r.interval || r.pgraph_dt != r.dt || r.pgraph_scheme != r.scheme) {
    free_adj_pgraphs(r);
    r.pgraph_len = r.interval;
    r.pgraph_dt = r.dt;
    r.pgraph_scheme = r.scheme;
  }
  cudaGraphExec_t& g = r.pgraph[kind][b];
  if (g && std::memcmp(key, r.pgraph_key[kind][b], sizeof key) == 0) {
    *out = g;
    return SGP_OK;
  }
  if (g) cudaGraphExecDestroy(g);
  g = nullptr;
  const long long launches0 = c->launches;
  SGP_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  sgp_status st = kind == 0 ? emit_recompute<R>(c, subs, seg, spec) : emit_adjoint<R>(c, subs, seg, spec);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
  r.pgraph_launches[kind][b] = c->launches - launches0;
  c->launches = launches0;
  if (st != SGP_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return fail(c, SGP_ECUDA, "stream capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&g, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    g = nullptr;
    return fail(c, SGP_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  std::memcpy(r.pgraph_key[kind][b], key, sizeof key);
  *out = g;
  return SGP_OK;
}

// Backward sweep with the recomputation of segment k - 1 running on a
// second stream (cs_alt, with its own device time) while g is carried back
// through segment k on the context stream.  The two use alternate segment
// buffers: segment k's recomputation waits until the sweep through segment
// k + 2 (the buffer's previous user) is done, and segment k's sweep waits
// for its recomputation.  The kernels of a small grid fill a fraction of
// the GPU, so the two streams overlap.  The operations and their order on
// each buffer are those of the serial sweep, so is the result.
template <typename R>
sgp_status backward_sweep_pipelined(sgp_ctx* c, const std::vector<SubRec>& full, size_t spec_off) {
  AdjRec& r = c->adj;
  const size_t sb = state_bytes(c);
  if (!c->cs_alt) SGP_CUDA(c, cudaStreamCreateWithFlags(&c->cs_alt, cudaStreamNonBlocking));
  if (!c->t_dev_alt) SGP_CUDA(c, dev_alloc(c, (void**)&c->t_dev_alt, sizeof(double)));
  for (cudaEvent_t& e : r.ev)
    if (!e) SGP_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  char* segs[2] = {(char*)r.seg, (char*)r.seg2};
  char* specs[2] = {segs[0] + spec_off, segs[1] + spec_off};   // the linear substeps' copies
  const bool graphs = c->use_graphs && !c->profiling;
  // the recomputations start after the work already on the context stream
  SGP_CUDA(c, cudaEventRecord(r.ev[0], c->stream));
  SGP_CUDA(c, cudaStreamWaitEvent(c->cs_alt, r.ev[0], 0));
  for (long long k = r.nck - 1; k >= 0; --k) {
    const int b = (int)(k & 1);
    const long long n = std::min(r.interval, r.nsteps - k * r.interval);
    const double tk = r.t0 + (double)(k * r.interval) * r.dt;
    const std::vector<SubRec> part = n == r.interval ? std::vector<SubRec>() : segment_substeps(r.scheme, n, r.dt);
    const std::vector<SubRec>& subs = n == r.interval ? full : part;
    // recomputation of segment k on the second stream
    if (k + 2 < r.nck) SGP_CUDA(c, cudaStreamWaitEvent(c->cs_alt, r.ev[3 + b], 0));
    std::swap(c->stream, c->cs_alt);
    std::swap(c->t_dev, c->t_dev_alt);
    sgp_status st = SGP_OK;
    c->launches++;
    k_set_time<<<1, 1, 0, c->stream>>>(c->t_dev, tk);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(segs[b], (const char*)r.ckpt + sb * (size_t)k, sb, cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) {
      st = fail(c, SGP_ECUDA, "segment start: %s", cudaGetErrorString(e));
    } else if (n == r.interval && graphs) {
      cudaGraphExec_t exec = nullptr;
      st = pipe_graph<R>(c, 0, b, subs, segs[b], specs[b], &exec);
      if (st == SGP_OK && (e = cudaGraphLaunch(exec, c->stream)) != cudaSuccess)
        st = fail(c, SGP_ECUDA, "graph launch: %s", cudaGetErrorString(e));
      c->launches += r.pgraph_launches[0][b];
    } else {
      st = emit_recompute<R>(c, subs, segs[b], specs[b]);
    }
    if (st == SGP_OK && (e = cudaEventRecord(r.ev[1 + b], c->stream)) != cudaSuccess)
      st = fail(c, SGP_ECUDA, "event: %s", cudaGetErrorString(e));
    std::swap(c->stream, c->cs_alt);
    std::swap(c->t_dev, c->t_dev_alt);
    if (st != SGP_OK) return st;
    // adjoint sweep through segment k on the context stream
    SGP_CUDA(c, cudaStreamWaitEvent(c->stream, r.ev[1 + b], 0));
    c->launches++;
    k_set_time<<<1, 1, 0, c->stream>>>(c->t_dev, tk);
    SGP_CUDA(c, cudaGetLastError());
    if (n == r.interval && graphs) {
      cudaGraphExec_t exec = nullptr;
      SGP_TRY(pipe_graph<R>(c, 1, b, subs, segs[b], specs[b], &exec));
      SGP_CUDA(c, cudaGraphLaunch(exec, c->stream));
      c->launches += r.pgraph_launches[1][b];
    } else {
      SGP_TRY(emit_adjoint<R>(c, subs, segs[b], specs[b]));
    }
    SGP_CUDA(c, cudaEventRecord(r.ev[3 + b], c->stream));
  }
  // the second stream's last work is done before anything that follows
  SGP_CUDA(c, cudaEventRecord(r.ev[1], c->cs_alt));
  SGP_CUDA(c, cudaStreamWaitEvent(c->stream, r.ev[1], 0));
  return SGP_OK;
}

// Backward sweep over the recorded trajectory: each segment is recomputed
// from its checkpoint, then g is carried back through its substeps in
// reverse order.  Pipelined over two streams when a second segment buffer
// fits (backward_sweep_pipelined); otherwise serial, full-length segments
// replaying one captured graph.
template <typename R>
sgp_status backward_sweep(sgp_ctx* c) {
  AdjRec& r = c->adj;
  const size_t sb = state_bytes(c);
  const auto seq = scheme_seq(r.scheme);
  // a segment buffer: the start state (the recomputation's working state),
  // one slot per substep (the nonlinear substeps' outputs), then the copies
  // of the linear substeps' outputs after the mix
  const size_t per_seg = (size_t)r.interval * seq.size() + 1;
  size_t nlin = 0;
  for (const auto& q : seq) nlin += q.first == 'L';
  const size_t seg_bytes = sb * (per_seg + (size_t)r.interval * nlin);
  SGP_TRY(ensure_buf(c, &r.seg, &r.seg_cap, seg_bytes));
  const int nblocks = adjoint_prows<R>(c);
  const size_t part_bytes = (size_t)c->batch * nblocks * GP_N * sizeof(double);
  SGP_TRY(ensure_buf(c, (void**)&r.part, &r.part_cap, part_bytes));
  SGP_CUDA(c, cudaMemsetAsync(r.part, 0, part_bytes, c->stream));
  for (const auto& st : merged_substeps(r.scheme, std::min<long long>(r.interval, 3), r.dt))
    if (st.kind == 'L') {       // tables of the forward and the reversed linear substeps
      const LinTables* t = nullptr;
      SGP_TRY(get_tables<R>(c, st.delta, &t));
      SGP_TRY(get_tables<R>(c, -st.delta, &t));
    }
  const std::vector<SubRec> full = segment_substeps(r.scheme, r.interval, r.dt);
  // the pipelined sweep: two segment buffers, if the memory is there
  const size_t pipe_bytes = seg_bytes;
  bool pipe = r.nck > 1;
  for (int k = 0; k < 2 && pipe; ++k) {
    void** p = k ? &r.seg2 : &r.seg;
    size_t* cap = k ? &r.seg2_cap : &r.seg_cap;
    if (*cap >= pipe_bytes) continue;
    SGP_CUDA(c, cudaStreamSynchronize(c->stream));
    dev_free(c, *p);
    *p = nullptr;
    *cap = 0;
    if (dev_alloc(c, p, pipe_bytes) == cudaSuccess) {
      *cap = pipe_bytes;
    } else {
      cudaGetLastError();
      *p = nullptr;
      pipe = false;
    }
  }
  if (!pipe) SGP_TRY(ensure_buf(c, &r.seg, &r.seg_cap, seg_bytes));
  if (pipe) {
    SGP_TRY(backward_sweep_pipelined<R>(c, full, sb * per_seg));
    c->launches++;
    SGP_CUDA(c, launch_reduce_params(r.part, nblocks, c->batch, r.dp, c->stream));
    return SGP_OK;
  }
  const bool graphs = c->use_graphs && !c->profiling;
  for (long long k = r.nck - 1; k >= 0; --k) {
    const long long n = std::min(r.interval, r.nsteps - k * r.interval);
    const double tk = r.t0 + (double)(k * r.interval) * r.dt;
    c->launches++;
    k_set_time<<<1, 1, 0, c->stream>>>(c->t_dev, tk);
    SGP_CUDA(c, cudaGetLastError());
    SGP_CUDA(c, cudaMemcpyAsync(r.seg, (const char*)r.ckpt + sb * (size_t)k, sb,
                                cudaMemcpyDeviceToDevice, c->stream));
    if (n == r.interval && graphs && r.nck > 1) {
      cudaGraphExec_t exec = nullptr;
      SGP_TRY(segment_graph<R>(c, full, sb * per_seg, &exec));
      SGP_CUDA(c, cudaGraphLaunch(exec, c->stream));
      c->launches += r.graph_launches;
    } else {
      SGP_TRY(emit_segment<R>(c, n == r.interval ? full : segment_substeps(r.scheme, n, r.dt), sb * per_seg));
    }
  }
  c->launches++;
  SGP_CUDA(c, launch_reduce_params(r.part, nblocks, c->batch, r.dp, c->stream));
  return SGP_OK;
}

// ----------------------------------------------------------------------------
// lab-frame output (Eq. (RSDA2)): quarter turns + three shears + exp(i l Omega t)
// ----------------------------------------------------------------------------
template <typename R>
sgp_status state_lab(sgp_ctx* c, void* dst, int on_device) {
  AdjRec& r = c->adj;
  const size_t sbm = (size_t)5 * c->ntot * c->elem;
  SGP_TRY(ensure_buf(c, &r.lab, &r.lab_cap, sbm));
  const double q = 0.5 * kPi;
  for (int m = 0; m < c->batch; ++m) {
    const double th = c->prm[m].omega * c->t;
    const long long k = (long long)std::llround(th / q);
    const double thr = th - (double)k * q;
    const int kk = (int)(((k % 4) + 4) % 4);
    if (kk && (c->n[0] != c->n[1] || c->L[0] != c->L[1]))
      return fail(c, SGP_EINVAL,
                  "rotation by %.3f rad needs quarter turns: the x-y grid must be square", th);
    const char* src = (const char*)c->field + sbm * m;
    cplx<R>* A = (cplx<R>*)r.lab;
    if (kk) {
      c->launches++;
      SGP_CUDA(c, launch_quarter<R>((const cplx<R>*)src, A, c->n[0], c->ntot, kk, c->stream));
    } else {
      SGP_CUDA(c, cudaMemcpyAsync(A, src, sbm, cudaMemcpyDeviceToDevice, c->stream));
    }
    ShearArgs<R> rows{};
    rows.field = A;
    rows.tw = (const TwE<R>*)c->tw[0];
    rows.ntot = c->ntot;
    rows.rows = c->n[1] * c->n[2];
    rows.ny = c->n[1];
    rows.coef = -std::tan(0.5 * thr);
    rows.o0 = -c->L[1];
    rows.h0 = c->h[1];
    rows.kfac = kPi / c->L[0];
    ShearArgs<R> cols{};
    cols.field = A;
    cols.tw = (const TwE<R>*)c->tw[1];
    cols.ntot = c->ntot;
    cols.rows = c->n[0];
    cols.line_stride = c->n[0];
    cols.plane_stride = (long long)c->n[0] * c->n[1];
    cols.coef = std::sin(thr);
    cols.o0 = -c->L[0];
    cols.h0 = c->h[0];
    cols.kfac = kPi / c->L[1];
    c->launches += 3;
    SGP_CUDA(c, launch_shear_rows<R>(c->n[0], rows, c->stream));
    SGP_CUDA(c, launch_shear_cols<R>(c->n[1], cols, c->n[2], c->stream));
    rows.lab_phase = 1;
    rows.theta = th;
    SGP_CUDA(c, launch_shear_rows<R>(c->n[0], rows, c->stream));
    SGP_CUDA(c, cudaMemcpyAsync((char*)dst + sbm * m, A, sbm,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                c->stream));
  }
  SGP_CUDA(c, cudaStreamSynchronize(c->stream));
  return SGP_OK;
}

// ----------------------------------------------------------------------------
// health check: per-member mass in FP64 (Sec. 2)
// ----------------------------------------------------------------------------
constexpr int kMassBlocks = 64;

template <typename R>
__global__ void k_mass(const cplx<R>* f, long long n, double* part) {
  const int m = blockIdx.y;
  const cplx<R>* b = f + (size_t)m * n;
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const cplx<R> v = b[i];
    s += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
  }
  __shared__ double red[8];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    part[(size_t)m * kMassBlocks + blockIdx.x] = t;
  }
}

// masses of all members into out[batch] (synchronises)
template <typename R>
sgp_status member_mass(sgp_ctx* c, std::vector<double>& out) {
  if (!c->mass_dev)
    SGP_CUDA(c, dev_alloc(c, (void**)&c->mass_dev, sizeof(double) * c->batch * (kMassBlocks + 1)));
  double* part = c->mass_dev + c->batch;
  c->launches += 2;
  k_mass<R><<<dim3(kMassBlocks, c->batch), 256, 0, c->stream>>>((const cplx<R>*)c->field,
                                                                 5 * c->ntot, part);
  k_reduce_partials<<<(c->batch + 127) / 128, 128, 0, c->stream>>>(part, kMassBlocks, 1, c->batch,
                                                                   c->mass_dev, 1, 0);
  SGP_CUDA(c, cudaGetLastError());
  out.resize(c->batch);
  SGP_CUDA(c, cudaMemcpyAsync(out.data(), c->mass_dev, sizeof(double) * c->batch,
                              cudaMemcpyDeviceToHost, c->stream));
  SGP_CUDA(c, cudaStreamSynchronize(c->stream));
  const double cell = c->h[0] * c->h[1] * (c->dim == 3 ? c->h[2] : 1.0);
  for (double& v : out) v *= cell;
  return SGP_OK;
}

// sgp_step with the health check: chunks of health_every steps, each
// followed by the mass comparison
template <typename R>
sgp_status checked_steps(sgp_ctx* c, long long nsteps, double dt, int scheme) {
  if (!c->health_ref) {
    SGP_TRY(member_mass<R>(c, c->m0));
    c->health_ref = true;
  }
  std::vector<double> m;
  long long done = 0;
  while (done < nsteps) {
    const long long n = std::min(c->health_every, nsteps - done);
    SGP_TRY(run_steps<R>(c, n, dt, scheme));
    done += n;
    SGP_TRY(member_mass<R>(c, m));
    for (int k = 0; k < c->batch; ++k) {
      if (!std::isfinite(m[k]))
        return fail(c, SGP_ENONFINITE, "member %d: mass %g after %lld of %lld steps", k, m[k],
                    done, nsteps);
      const double drift = std::fabs(m[k] / c->m0[k] - 1.0);
      if (!(drift <= c->health_tol))
        return fail(c, SGP_EDRIFT, "member %d: mass %.17g drifted %.3e from %.17g after %lld of %lld steps",
                    k, m[k], drift, c->m0[k], done, nsteps);
    }
  }
  return SGP_OK;
}

// ----------------------------------------------------------------------------
// kernel variants: plan and autotuner
// ----------------------------------------------------------------------------
void drop_graphs(sgp_ctx* c) {
  free_graphs(c);
  free_adj_pgraphs(c->adj);
  if (c->adj.graph) {
    cudaGraphExecDestroy(c->adj.graph);
    c->adj.graph = nullptr;
  }
}

// Does variant v exist for axis a of this context's grid?  Variants 0-4
// depend on the line length alone; variant 5 is the x-pass variant of 3D
// FP32 grids with NX = NY = 64 or 128.
bool axis_variant_ok(const sgp_ctx* c, int a, int v) {
  if (v == 5) return a == 0 && plane_ok(c);
  return variant_exists(c->prec == SGP_F32 ? 4 : 8, c->n[a], v);
}

// Switch axis `a` to variant v: twiddles of its radix plan, kernel
// attributes; captured graphs are dropped (they embed the old kernels).
sgp_status use_variant(sgp_ctx* c, int a, int v) {
  if (!axis_variant_ok(c, a, v))
    return fail(c, SGP_EINVAL, "variant %d does not exist for N = %d on axis %d", v, c->n[a], a);
  if (v == 4 && !tensor_map_encoder())      // fetched now, not inside a later stream capture
    return fail(c, SGP_EUNSUPPORTED, "the driver has no tensor-map encoder (variant 4)");
  if (v == 5) {
    const cudaError_t e = prepare_xyplane(c->n[0]);
    if (e != cudaSuccess) return fail(c, SGP_ECUDA, "kernel attributes: %s", cudaGetErrorString(e));
  }
  if (v == 3 && !c->tw4[a]) {
    SGP_CUDA(c, cudaStreamSynchronize(c->stream));
    SGP_CUDA(c, dev_alloc(c, &c->tw4[a], (size_t)c->n[a] * sizeof(TwE<float>)));
    k_twiddles_f32<<<(c->n[a] + 255) / 256, 256, 0, c->stream>>>(c->n[a], variant_elems_rt(4, c->n[a], 3),
                                                                (TwE<float>*)c->tw4[a]);
    c->launches++;
    SGP_CUDA(c, cudaGetLastError());
  }
  cudaError_t e = c->prec == SGP_F32
                      ? (a == 0 ? prepare_xpass<float>(c->n[a], v) : prepare_linepass<float>(c->n[a], v))
                      : (a == 0 ? prepare_xpass<double>(c->n[a], v) : prepare_linepass<double>(c->n[a], v));
  if (e != cudaSuccess) return fail(c, SGP_ECUDA, "kernel attributes: %s", cudaGetErrorString(e));
  if (c->var[a] != v) {
    SGP_CUDA(c, cudaStreamSynchronize(c->stream));
    drop_graphs(c);
    c->var[a] = v;
  }
  return SGP_OK;
}

// process-wide results of the autotuner, keyed by device, precision, grid
// and batch
std::map<std::string, std::vector<int>>& tune_cache() {
  static std::map<std::string, std::vector<int>> m;
  return m;
}

std::string tune_key(const sgp_ctx* c) {
  char b[160];
  snprintf(b, sizeof b, "%d:%d:%d:%d:%d:%d:%d", c->device, c->prec, c->dim, c->n[0], c->n[1],
           c->n[2], c->batch);
  return b;
}

// Times the variants axis by axis (coordinate descent: axis a's variants
// with the other axes at their current choice) by running `reps` TS2 steps
// of dt = 1e-3 on a scratch copy of the field with CUDA events after one
// warm-up step: the data stay a physical state, so the nonlinear flow takes
// its usual branches, and the pass interplay of a real step is included.  A
// variant replaces an earlier (lower-numbered) one only when it is at least
// 1.5% faster, so near-ties resolve the same way run to run.  ms_out[3][7]:
// ms per step with that variant (-1 where a variant does not exist or the
// axis is absent).
template <typename R>
sgp_status autotune_impl(sgp_ctx* c, int reps, double* ms_out) {
  const size_t sb = state_bytes(c);
  void* scratch = nullptr;
  SGP_CUDA(c, cudaStreamSynchronize(c->stream));
  SGP_CUDA(c, dev_alloc(c, &scratch, sb));
  SGP_CUDA(c, cudaMemcpyAsync(scratch, c->field, sb, cudaMemcpyDeviceToDevice, c->stream));
  std::swap(c->field, scratch);            // the steps below advance the copy
  const double dt = 1e-3;
  sgp_status st = ensure_tables<R>(c, dt, SGP_TS2);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int best[3] = {c->var[0], c->var[1], c->var[2]};
  if (ms_out)
    for (int k = 0; k < 3 * kVariants; ++k) ms_out[k] = -1.0;
  for (int a = 0; a < c->dim && st == SGP_OK; ++a) {
    double best_ms = -1.0;
    for (int v = 0; v < kVariants && st == SGP_OK; ++v) {
      if (!axis_variant_ok(c, a, v)) continue;
      if (a == 0 && v == 4) continue;     // the x-pass of variant 4 is variant 1
      if (a != 0 && v == 6) continue;     // the line pass of variant 6 is variant 2
      if (v == 4 && !tensor_map_encoder()) continue;
      st = use_variant(c, a, v);
      if (st != SGP_OK) break;
      c->launches++;
      k_set_time<<<1, 1, 0, c->stream>>>(c->t_dev, c->t);
      st = emit_steps<R>(c, 1, dt, SGP_TS2);
      if (st != SGP_OK) break;
      cudaEventRecord(e0, c->stream);
      st = emit_steps<R>(c, reps, dt, SGP_TS2);
      cudaEventRecord(e1, c->stream);
      if (st != SGP_OK) break;
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        st = fail(c, SGP_ECUDA, "autotune timing: %s", cudaGetErrorString(cudaGetLastError()));
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      const double avg = ms / reps;
      if (ms_out) ms_out[a * kVariants + v] = avg;
      if (best_ms < 0.0 || avg < 0.985 * best_ms) {
        best_ms = avg;
        best[a] = v;
      }
    }
    if (st == SGP_OK) st = use_variant(c, a, best[a]);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(c->stream);
  std::swap(c->field, scratch);
  dev_free(c, scratch);
  if (st == SGP_OK) tune_cache()[tune_key(c)] = std::vector<int>(best, best + 3);
  return st;
}

// ----------------------------------------------------------------------------
// observables
// ----------------------------------------------------------------------------
void assemble_obs(const double* s, int dim, double cell, double t, const sgp_params& p,
                  sgp_obs* o) {
  *o = sgp_obs{};
  o->t = t;
  for (int k = 0; k < 5; ++k) {
    o->comp_mass[k] = cell * s[OB_M0 + k];
    o->mass += o->comp_mass[k];
    o->magnetization += (2 - k) * o->comp_mass[k];
  }
  o->width2[0] = cell * s[OB_WX];
  o->width2[1] = cell * s[OB_WY];
  o->width2[2] = cell * s[OB_WZ];
  o->e_kin = cell * (s[OB_KX] + s[OB_KY] + (dim == 3 ? s[OB_KZ] : 0.0));
  o->e_pot = cell * s[OB_POT];
  o->lz = cell * (s[OB_LZX] + s[OB_LZY]);
  o->e_rot = -p.omega * o->lz;
  o->e_int = cell * s[OB_INT];
  o->e_soc = -p.gamma * cell * (s[OB_SOCX] + s[OB_SOCY]);
  o->energy = o->e_kin + o->e_pot + o->e_rot + o->e_int + o->e_soc;
}

bool obs_finite(const sgp_obs& o) {
  const double chk[6] = {o.mass, o.energy, o.magnetization, o.lz, o.width2[0], o.width2[1]};
  for (double v : chk)
    if (!std::isfinite(v)) return false;
  return true;
}

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
  ax.t = c->t;
  ax.mp = c->mp_dev;
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
    assemble_obs(&h[(size_t)m * OB_NT], c->dim, cell, c->t, c->prm[m], &out[m]);
    finite = finite && obs_finite(out[m]);
  }
  if (!finite) return fail(c, SGP_ENONFINITE, "non-finite observable");
  return SGP_OK;
}

sgp_status validate_grid(int dim, const int* n, const double* L, int batch, int prec) {
  if (!n || !L) return fail(nullptr, SGP_EINVAL, "NULL argument");
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
  return SGP_OK;
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

int sgp_version(void) { return 200; }

sgp_status sgp_set_allocator(sgp_alloc_fn alloc, sgp_free_fn free_fn, void* user) {
  if ((alloc == nullptr) != (free_fn == nullptr)) {
    g_create_err = "allocator and free function must be given together";
    return SGP_EINVAL;
  }
  g_allocator.alloc = alloc;
  g_allocator.free = free_fn;
  g_allocator.user = user;
  return SGP_OK;
}

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
    case SGP_EDRIFT: return "SGP_EDRIFT";
  }
  return "unknown";
}

const char* sgp_last_error(const sgp_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

sgp_status sgp_destroy(sgp_ctx* c);

sgp_status sgp_create_grid(int dim, const int* n, const double* L, int batch, int prec,
                           int device, void* stream, sgp_ctx** out) {
  g_create_err.clear();
  if (!out) return fail(nullptr, SGP_EINVAL, "NULL argument");
  *out = nullptr;
  SGP_TRY(validate_grid(dim, n, L, batch, prec));
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return fail(nullptr, SGP_EINVAL, "CUDA device %d not available", device);
  DeviceGuard guard(device);
  sgp_ctx* c = new sgp_ctx();
  c->alloc = g_allocator;
  c->dim = dim;
  for (int a = 0; a < 3; ++a) {
    c->n[a] = a < dim ? n[a] : 1;
    c->L[a] = a < dim ? L[a] : 1.0;
    c->h[a] = 2.0 * c->L[a] / c->n[a];
  }
  c->batch = batch;
  c->prec = prec;
  c->device = device;
  c->ntot = (long long)c->n[0] * c->n[1] * c->n[2];
  c->elem = prec == SGP_F32 ? 8 : 16;
  sgp_params defaults{};
  defaults.gx = defaults.gy = defaults.gz = 1.0;
  c->prm.assign(batch, defaults);
  auto bail = [&](sgp_status s, const char* what, cudaError_t e) {
    fail(nullptr, s, "%s: %s", what, cudaGetErrorString(e));
    sgp_destroy(c);
    return s;
  };
  cudaError_t e;
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    if ((e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking)) != cudaSuccess)
      return bail(SGP_ECUDA, "stream", e);
    c->own_stream = true;
  }
  // kernel attributes now, so that no later capture has to set them
  for (int a = 0; a < dim; ++a) {
    e = prec == SGP_F32 ? (a == 0 ? prepare_xpass<float>(c->n[a]) : prepare_linepass<float>(c->n[a]))
                        : (a == 0 ? prepare_xpass<double>(c->n[a]) : prepare_linepass<double>(c->n[a]));
    if (e != cudaSuccess) return bail(SGP_ECUDA, "kernel attributes", e);
  }
  const size_t fbytes = (size_t)batch * 5 * c->ntot * c->elem;
  if ((e = dev_alloc(c, &c->field, fbytes)) != cudaSuccess)
    return bail(SGP_ENOMEM, "field allocation", e);
  if ((e = cudaMemsetAsync(c->field, 0, fbytes, c->stream)) != cudaSuccess)
    return bail(SGP_ECUDA, "field clear", e);
  for (int a = 0; a < dim; ++a) {
    if ((e = dev_alloc(c, &c->tw[a], (size_t)c->n[a] * 16)) != cudaSuccess)
      return bail(SGP_ENOMEM, "twiddle allocation", e);
    const int E = elems_for(c->n[a], prec);
    if (prec == SGP_F32)
      k_twiddles_f32<<<(c->n[a] + 255) / 256, 256, 0, c->stream>>>(c->n[a], E, (TwE<float>*)c->tw[a]);
    else
      k_twiddles_f64<<<(c->n[a] + 255) / 256, 256, 0, c->stream>>>(c->n[a], E, (TwE<double>*)c->tw[a]);
    c->launches++;
  }
  if ((e = dev_alloc(c, (void**)&c->t_dev, sizeof(double))) != cudaSuccess)
    return bail(SGP_ENOMEM, "time allocation", e);
  if ((e = dev_alloc(c, (void**)&c->err_dev, sizeof(int))) != cudaSuccess)
    return bail(SGP_ENOMEM, "error word allocation", e);
  if ((e = cudaMemsetAsync(c->err_dev, 0, sizeof(int), c->stream)) != cudaSuccess)
    return bail(SGP_ECUDA, "error word clear", e);
  if ((e = dev_alloc(c, (void**)&c->mp_dev, sizeof(MemberPrm) * batch)) != cudaSuccess)
    return bail(SGP_ENOMEM, "parameter allocation", e);
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
  if ((e = dev_alloc(c, (void**)&c->partials, c->partials_len * sizeof(double))) != cudaSuccess)
    return bail(SGP_ENOMEM, "observables scratch", e);
  if ((e = dev_alloc(c, (void**)&c->obs_dev, (size_t)batch * OB_NT * sizeof(double))) != cudaSuccess)
    return bail(SGP_ENOMEM, "observables output", e);
  if ((e = cudaMemsetAsync(c->obs_dev, 0, (size_t)batch * OB_NT * sizeof(double), c->stream)) !=
      cudaSuccess)
    return bail(SGP_ECUDA, "observables clear", e);
  if ((e = cudaGetLastError()) != cudaSuccess) return bail(SGP_ECUDA, "table launch", e);
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return bail(SGP_ECUDA, "create sync", e);
  if (upload_params(c) != SGP_OK) {
    fail(nullptr, SGP_ECUDA, "%s", c->err.c_str());
    sgp_destroy(c);
    return SGP_ECUDA;
  }
  *out = c;
  return SGP_OK;
}

sgp_status sgp_set_params(sgp_ctx* c, const sgp_params* p) {
  if (!c) return SGP_EINVAL;
  if (!p) return fail(c, SGP_EINVAL, "NULL params");
  if (!finite_params(p)) return fail(c, SGP_EINVAL, "non-finite parameter");
  DeviceGuard guard(c->device);
  c->adj.valid = false;
  c->prm.assign(c->batch, *p);
  return upload_params(c);
}

sgp_status sgp_set_params_batch(sgp_ctx* c, const sgp_params* p, int count) {
  if (!c) return SGP_EINVAL;
  if (!p) return fail(c, SGP_EINVAL, "NULL params");
  if (count != c->batch) return fail(c, SGP_EINVAL, "count %d != batch %d", count, c->batch);
  for (int m = 0; m < count; ++m)
    if (!finite_params(&p[m])) return fail(c, SGP_EINVAL, "non-finite parameter (member %d)", m);
  DeviceGuard guard(c->device);
  c->adj.valid = false;
  c->prm.assign(p, p + count);
  return upload_params(c);
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
  c->adj.valid = false;
  c->health_ref = false;
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

sgp_status sgp_get_state_lab(sgp_ctx* c, void* dst, int dst_on_device) {
  if (!c) return SGP_EINVAL;
  if (!dst) return fail(c, SGP_EINVAL, "NULL dst");
  if (c->dim < 2) return fail(c, SGP_EINVAL, "lab frame needs dim 2 or 3");
  DeviceGuard guard(c->device);
  return c->prec == SGP_F32 ? state_lab<float>(c, dst, dst_on_device)
                            : state_lab<double>(c, dst, dst_on_device);
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
  if (!valid_scheme(scheme)) return fail(c, SGP_EINVAL, "unknown scheme %d", scheme);
  if (!c->have_state) return fail(c, SGP_ESTATE, "sgp_step before sgp_set_state");
  if (nsteps == 0) return SGP_OK;
  DeviceGuard guard(c->device);
  c->adj.valid = false;
  if (c->health_every > 0)
    return c->prec == SGP_F32 ? checked_steps<float>(c, nsteps, dt, scheme)
                              : checked_steps<double>(c, nsteps, dt, scheme);
  return c->prec == SGP_F32 ? run_steps<float>(c, nsteps, dt, scheme)
                            : run_steps<double>(c, nsteps, dt, scheme);
}

sgp_status sgp_substep_plan(int scheme, long long nsteps, double dt, long long cap, char* kinds,
                            double* deltas, double* toffs, long long* count) {
  if (!count) return SGP_EINVAL;
  *count = 0;
  if (!valid_scheme(scheme) || nsteps < 0 || !(dt > 0.0) || !std::isfinite(dt)) return SGP_EINVAL;
  if (cap > 0 && (!kinds || !deltas || !toffs)) return SGP_EINVAL;
  const std::vector<SubRec> subs = merged_substeps(scheme, nsteps, dt);
  *count = (long long)subs.size();
  for (long long k = 0; k < cap && k < *count; ++k) {
    kinds[k] = subs[(size_t)k].kind;
    deltas[k] = subs[(size_t)k].delta;
    toffs[k] = subs[(size_t)k].toff;
  }
  return SGP_OK;
}

sgp_status sgp_step_host(sgp_ctx* c, const void* host_in, double t0, void* host_out,
                         long long nsteps, double dt, int scheme, int chunks) {
  if (!c) return SGP_EINVAL;
  if (!host_in || !host_out) return fail(c, SGP_EINVAL, "NULL host buffer");
  if (chunks < 1 || chunks > c->batch)
    return fail(c, SGP_EINVAL, "chunks %d not in [1, batch = %d]", chunks, c->batch);
  if (nsteps < 0) return fail(c, SGP_EINVAL, "nsteps < 0");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, SGP_EINVAL, "dt must be positive and finite");
  if (!std::isfinite(t0)) return fail(c, SGP_EINVAL, "non-finite t0");
  if (!valid_scheme(scheme)) return fail(c, SGP_EINVAL, "unknown scheme %d", scheme);
  DeviceGuard guard(c->device);
  return c->prec == SGP_F32 ? step_host_impl<float>(c, host_in, t0, host_out, nsteps, dt, scheme, chunks)
                            : step_host_impl<double>(c, host_in, t0, host_out, nsteps, dt, scheme, chunks);
}

sgp_status sgp_set_health_check(sgp_ctx* c, long long every, double drift_tol) {
  if (!c) return SGP_EINVAL;
  if (every < 0) return fail(c, SGP_EINVAL, "every < 0");
  if (!(drift_tol >= 0.0) || !std::isfinite(drift_tol))
    return fail(c, SGP_EINVAL, "drift_tol must be finite and >= 0");
  c->health_every = every;
  c->health_tol = drift_tol;
  return SGP_OK;
}

sgp_status sgp_record(sgp_ctx* c, long long nsteps, double dt, int scheme, long long interval) {
  if (!c) return SGP_EINVAL;
  if (nsteps <= 0) return fail(c, SGP_EINVAL, "nsteps must be positive");
  if (interval < 0) return fail(c, SGP_EINVAL, "interval < 0");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, SGP_EINVAL, "dt must be positive and finite");
  if (!valid_scheme(scheme)) return fail(c, SGP_EINVAL, "unknown scheme %d", scheme);
  if (!c->have_state) return fail(c, SGP_ESTATE, "sgp_record before sgp_set_state");
  DeviceGuard guard(c->device);
  return c->prec == SGP_F32 ? record_steps<float>(c, nsteps, dt, scheme, interval)
                            : record_steps<double>(c, nsteps, dt, scheme, interval);
}

sgp_status sgp_backward(sgp_ctx* c, const void* g_T, int g_T_on_device, void* g_0,
                        int g_0_on_device, double* dparams) {
  if (!c) return SGP_EINVAL;
  if (!g_T || !g_0) return fail(c, SGP_EINVAL, "NULL gradient buffer");
  if (!c->adj.valid) return fail(c, SGP_ESTATE, "sgp_backward without a valid sgp_record");
  DeviceGuard guard(c->device);
  AdjRec& r = c->adj;
  const size_t sb = state_bytes(c);
  SGP_TRY(ensure_buf(c, &r.g, &r.g_cap, sb));
  SGP_TRY(ensure_buf(c, (void**)&r.dp, &r.dp_cap, sizeof(double) * GP_N * c->batch));
  SGP_CUDA(c, cudaMemcpyAsync(r.g, g_T, sb, g_T_on_device ? cudaMemcpyDeviceToDevice
                                                         : cudaMemcpyHostToDevice, c->stream));
  SGP_CUDA(c, cudaMemsetAsync(r.dp, 0, sizeof(double) * GP_N * c->batch, c->stream));
  SGP_TRY(c->prec == SGP_F32 ? backward_sweep<float>(c) : backward_sweep<double>(c));
  SGP_CUDA(c, cudaMemcpyAsync(g_0, r.g, sb, g_0_on_device ? cudaMemcpyDeviceToDevice
                                                         : cudaMemcpyDeviceToHost, c->stream));
  if (dparams)
    SGP_CUDA(c, cudaMemcpyAsync(dparams, r.dp, sizeof(double) * GP_N * c->batch,
                                cudaMemcpyDeviceToHost, c->stream));
  SGP_CUDA(c, cudaStreamSynchronize(c->stream));
  return SGP_OK;
}

sgp_status sgp_set_graphs(sgp_ctx* c, int enable) {
  if (!c) return SGP_EINVAL;
  c->use_graphs = enable != 0;
  return SGP_OK;
}

int sgp_variant_exists(int prec, int n, int variant) {
  if (prec != SGP_F32 && prec != SGP_F64) return 0;
  return variant_exists(prec == SGP_F32 ? 4 : 8, n, variant) ? 1 : 0;
}

sgp_status sgp_set_plan(sgp_ctx* c, const int* variants) {
  if (!c) return SGP_EINVAL;
  if (!variants) return fail(c, SGP_EINVAL, "NULL variants");
  for (int a = 0; a < c->dim; ++a)
    if (!axis_variant_ok(c, a, variants[a]))
      return fail(c, SGP_EINVAL, "variant %d does not exist for N = %d on axis %d", variants[a],
                  c->n[a], a);
  DeviceGuard guard(c->device);
  for (int a = 0; a < c->dim; ++a) SGP_TRY(use_variant(c, a, variants[a]));
  return SGP_OK;
}

sgp_status sgp_get_plan(const sgp_ctx* c, int* variants) {
  if (!c || !variants) return SGP_EINVAL;
  for (int a = 0; a < 3; ++a) variants[a] = a < c->dim ? c->var[a] : 0;
  return SGP_OK;
}

sgp_status sgp_autotune(sgp_ctx* c, int reps, int flags, double* ms_out) {
  if (!c) return SGP_EINVAL;
  if (reps < 1 || reps > 1000) return fail(c, SGP_EINVAL, "reps must be in [1, 1000]");
  DeviceGuard guard(c->device);
  if (!(flags & SGP_TUNE_FORCE) && !ms_out) {
    auto it = tune_cache().find(tune_key(c));
    if (it != tune_cache().end()) {
      for (int a = 0; a < c->dim; ++a) SGP_TRY(use_variant(c, a, it->second[a]));
      return SGP_OK;
    }
  }
  return c->prec == SGP_F32 ? autotune_impl<float>(c, reps, ms_out)
                            : autotune_impl<double>(c, reps, ms_out);
}

sgp_status sgp_substep(sgp_ctx* c, int kind, double delta) {
  if (!c) return SGP_EINVAL;
  if (kind != SGP_SUB_NONLINEAR && kind != SGP_SUB_LINEAR)
    return fail(c, SGP_EINVAL, "unknown substep kind %d", kind);
  if (!std::isfinite(delta)) return fail(c, SGP_EINVAL, "non-finite delta");
  if (!c->have_state) return fail(c, SGP_ESTATE, "sgp_substep before sgp_set_state");
  DeviceGuard guard(c->device);
  c->adj.valid = false;
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
  if (c->err_dev) {
    int err = 0;
    SGP_CUDA(c, cudaMemcpy(&err, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
      SGP_CUDA(c, cudaMemset(c->err_dev, 0, sizeof(int)));
      c->have_state = false;
      return fail(c, SGP_ETIMEOUT, "a tile-load wait of line-pass variant 4 gave up; the state is undefined "
                                   "until it is set again");
    }
  }
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
  if (c->stream || c->own_stream) cudaStreamSynchronize(c->stream);
  free_graphs(c);
  free_tables(c);
  free_adj(c);
  dev_free(c, c->field);
  for (void* t : c->tw) dev_free(c, t);
  for (void* t : c->tw4) dev_free(c, t);
  dev_free(c, c->t_dev);
  dev_free(c, c->err_dev);
  dev_free(c, c->mp_dev);
  dev_free(c, c->partials);
  dev_free(c, c->obs_dev);
  dev_free(c, c->mass_dev);
  recycle_events(c);
  for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
  for (cudaEvent_t e : c->pipe_ev) cudaEventDestroy(e);
  if (c->cs_in) cudaStreamDestroy(c->cs_in);
  if (c->cs_out) cudaStreamDestroy(c->cs_out);
  if (c->cs_alt) cudaStreamDestroy(c->cs_alt);
  dev_free(c, c->t_dev_alt);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
  return SGP_OK;
}

}  // extern "C"

// ============================================================================
// ensembles of independent runs with different grids (one graph per chunk)
// ============================================================================
struct sgp_ens {
  int dim = 2;
  int count = 0;
  int prec = SGP_F32;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<sgp_ctx*> groups;            // one context per distinct grid
  std::vector<cudaStream_t> gstreams;      // capture branches
  std::vector<cudaEvent_t> join;           // one per group
  cudaEvent_t fork = nullptr;
  std::vector<int> member_group, member_index;
  std::vector<GraphEntry> graphs;
  double t = 0.0;
  bool have_state = false;
  long long launches = 0;
  std::string err;
  // the persistent work-queue kernel (2D, line lengths of persist_supported)
  bool persist_ok = false;          // every group can run in it
  bool use_persist = true;
  int persist_grid = 0;             // CTAs: the number that fit on the GPU at once
  double wait_seconds = 1.0;        // limit of every device-side wait
  long long wait_cycles = 0;
  int* done_dev = nullptr;          // finished tiles of each member
  PersistCtl* ctl_dev = nullptr;
  std::vector<int> gbase;           // the first member (counter) of each group
  struct PProg {
    long long steps;
    double dt;
    int scheme;
    std::vector<long long> gens;    // the groups' table generations it points at
    void* dev;                      // PersistPass<R>[passes * groups]
    PersistLayout lay;
    long long nitems;
    cudaGraphExec_t graph;          // captured launch (nullptr: launched directly)
  };
  std::vector<PProg> progs;
  int stall_member = -1;            // test hook: withhold one completion signal
  // sgp_ensemble_step_host with page-locked buffers: the copy lists of
  // k_copy_members (in, then out) on the device
  MemberXfer* xfer_dev = nullptr;
};

namespace {

sgp_status efail(sgp_ens* e, sgp_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (e)
    e->err = buf;
  else
    g_create_err = buf;
  return s;
}

void ens_free_graphs(sgp_ens* e) {
  for (auto& g : e->graphs) cudaGraphExecDestroy(g.exec);
  e->graphs.clear();
}

// Issue `steps` steps of every group: group g on stream s(g).
template <typename R>
sgp_status ens_emit(sgp_ens* e, long long steps, double dt, int scheme, bool branches) {
  for (size_t g = 0; g < e->groups.size(); ++g) {
    sgp_ctx* c = e->groups[g];
    const cudaStream_t saved = c->stream;
    c->stream = branches ? e->gstreams[g] : e->stream;
    sgp_status st = emit_steps<R>(c, steps, dt, scheme);
    c->stream = saved;
    if (st != SGP_OK) return efail(e, st, "group %zu: %s", g, c->err.c_str());
  }
  return SGP_OK;
}

template <typename R>
sgp_status ens_graph(sgp_ens* e, long long steps, double dt, int scheme, cudaGraphExec_t* out) {
  for (auto& g : e->graphs)
    if (g.steps == steps && g.dt == dt && g.scheme == scheme) {
      *out = g.exec;
      return SGP_OK;
    }
  if (e->graphs.size() >= 8) ens_free_graphs(e);
  for (sgp_ctx* c : e->groups) {
    const cudaStream_t saved = c->stream;
    c->stream = e->stream;
    sgp_status st = ensure_tables<R>(c, dt, scheme);
    c->stream = saved;
    if (st != SGP_OK) return efail(e, st, "%s", c->err.c_str());
  }
  std::vector<long long> l0;
  for (sgp_ctx* c : e->groups) l0.push_back(c->launches);
  cudaError_t ce = cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal);
  if (ce != cudaSuccess) return efail(e, SGP_ECUDA, "begin capture: %s", cudaGetErrorString(ce));
  cudaEventRecord(e->fork, e->stream);
  for (size_t g = 0; g < e->groups.size(); ++g) cudaStreamWaitEvent(e->gstreams[g], e->fork, 0);
  sgp_status st = ens_emit<R>(e, steps, dt, scheme, true);
  for (size_t g = 0; g < e->groups.size(); ++g) {
    cudaEventRecord(e->join[g], e->gstreams[g]);
    cudaStreamWaitEvent(e->stream, e->join[g], 0);
  }
  cudaGraph_t graph = nullptr;
  ce = cudaStreamEndCapture(e->stream, &graph);
  for (size_t g = 0; g < e->groups.size(); ++g) e->groups[g]->launches = l0[g];
  if (st != SGP_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (ce != cudaSuccess) return efail(e, SGP_ECUDA, "end capture: %s", cudaGetErrorString(ce));
  cudaGraphExec_t exec = nullptr;
  ce = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) return efail(e, SGP_ECUDA, "graph instantiate: %s", cudaGetErrorString(ce));
  e->graphs.push_back({steps, dt, scheme, exec});
  *out = exec;
  return SGP_OK;
}

void ens_free_progs(sgp_ens* e) {
  for (auto& p : e->progs) {
    if (p.graph) cudaGraphExecDestroy(p.graph);
    dev_free(e->groups[0], p.dev);
  }
  e->progs.clear();
}

std::vector<long long> ens_table_gens(const sgp_ens* e) {
  std::vector<long long> g;
  for (const sgp_ctx* c : e->groups) g.push_back(c->tables_gen);
  return g;
}

// The queue program of `steps` steps: every group's passes recorded from
// emit_steps, interleaved pass by pass (all groups' items of pass 0, then of
// pass 1, ...), and the layout the kernel decodes work items with.  Cached
// per (steps, dt, scheme) while the tables it points at stay.
template <typename R>
sgp_status ens_persist_program(sgp_ens* e, long long steps, double dt, int scheme,
                               sgp_ens::PProg** out) {
  const std::vector<long long> gens = ens_table_gens(e);
  for (auto& p : e->progs)
    if (p.steps == steps && p.dt == dt && p.scheme == scheme && p.gens == gens) {
      *out = &p;
      return SGP_OK;
    }
  if (e->progs.size() >= 4) ens_free_progs(e);
  const size_t G = e->groups.size();
  std::vector<std::vector<PersistPass<R>>> per(G);
  for (size_t g = 0; g < G; ++g) {
    sgp_ctx* c = e->groups[g];
    const cudaStream_t saved = c->stream;
    c->stream = e->stream;
    sgp_status st = ensure_tables<R>(c, dt, scheme);
    c->rec = &per[g];
    if (st == SGP_OK) st = emit_steps<R>(c, steps, dt, scheme);
    c->rec = nullptr;
    c->stream = saved;
    if (st != SGP_OK) return efail(e, st, "group %zu: %s", g, c->err.c_str());
  }
  const size_t P = per[0].size();
  for (size_t g = 1; g < G; ++g)
    if (per[g].size() != P) return efail(e, SGP_EINVAL, "groups issue different pass sequences");
  // passes alternate x-pass, line pass, ..., x-pass; the layout describes
  // the items of one pass of each kind
  sgp_ens::PProg pp{};
  PersistLayout& lay = pp.lay;
  lay.groups = (int)G;
  lay.xoff[0] = lay.loff[0] = 0;
  for (size_t p = 0; p < P; ++p)
    for (size_t g = 0; g < G; ++g) {
      const PersistPass<R>& q = per[g][p];
      if (q.kind != (p % 2 ? PK_LINE : PK_XPASS) || P % 2 == 0)
        return efail(e, SGP_EINVAL, "unexpected pass sequence for the persistent kernel");
      int& t = q.kind == PK_XPASS ? lay.xt[g] : lay.lt[g];
      if (p < 2) t = q.tiles;
      else if (t != q.tiles) return efail(e, SGP_EINVAL, "passes of one kind differ in tiles");
    }
  for (size_t g = 0; g < G; ++g) {
    lay.xi[g] = (lay.xt[g] + kTilesPerItem - 1) / kTilesPerItem;
    lay.li[g] = (lay.lt[g] + kTilesPerItem - 1) / kTilesPerItem;
    lay.xoff[g + 1] = lay.xoff[g] + per[g][0].members * lay.xi[g];
    lay.loff[g + 1] = lay.loff[g] + per[g][0].members * (P > 1 ? lay.li[g] : 0);
    lay.base[g] = e->gbase[g];
  }
  lay.IX = lay.xoff[G];
  lay.IL = lay.loff[G];
  std::vector<PersistPass<R>> prog;
  prog.reserve(P * G);
  for (size_t p = 0; p < P; ++p)
    for (size_t g = 0; g < G; ++g) prog.push_back(per[g][p]);
  const long long item = (long long)(P / 2) * (lay.IX + lay.IL) + lay.IX;
  if (item >= (1LL << 31)) return efail(e, SGP_EUNSUPPORTED, "too many work items for one launch");
  const size_t bytes = prog.size() * sizeof(PersistPass<R>);
  cudaError_t ce = dev_alloc(e->groups[0], &pp.dev, bytes);
  if (ce != cudaSuccess) return efail(e, SGP_ENOMEM, "persistent program: %s", cudaGetErrorString(ce));
  ce = cudaMemcpy(pp.dev, prog.data(), bytes, cudaMemcpyHostToDevice);
  if (ce != cudaSuccess) {
    dev_free(e->groups[0], pp.dev);
    return efail(e, SGP_ECUDA, "persistent program: %s", cudaGetErrorString(ce));
  }
  pp.steps = steps;
  pp.dt = dt;
  pp.scheme = scheme;
  pp.gens = ens_table_gens(e);       // after ensure_tables: the tables recorded above
  pp.nitems = item;
  pp.graph = nullptr;
  e->progs.push_back(pp);
  *out = &e->progs.back();
  return SGP_OK;
}

// One launch of a program on the ensemble stream: the queue head and the
// completion counters cleared, the persistent kernel, every group's time
// advanced.
template <typename R>
sgp_status ens_persist_issue(sgp_ens* e, const sgp_ens::PProg& p) {
  cudaError_t ce = cudaMemsetAsync(&e->ctl_dev->head, 0, sizeof(unsigned long long), e->stream);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(e->done_dev, 0, sizeof(int) * (size_t)e->count, e->stream);
  if (ce == cudaSuccess)
    ce = launch_persistent<R>((const PersistPass<R>*)p.dev, p.lay, (int)p.nitems, e->done_dev, e->ctl_dev,
                              e->wait_cycles, e->persist_grid, e->stream);
  for (sgp_ctx* c : e->groups)
    if (ce == cudaSuccess) {
      k_add_time<<<1, 1, 0, e->stream>>>(c->t_dev, (double)p.steps * p.dt);
      ce = cudaGetLastError();
    }
  if (ce != cudaSuccess) return efail(e, SGP_ECUDA, "persistent launch: %s", cudaGetErrorString(ce));
  return SGP_OK;
}

// nsteps steps through the persistent kernel: one captured launch per chunk
// of kGraphChunk steps, the rest launched directly; then the control word:
// SGP_ETIMEOUT if a wait gave up (the call synchronises for this).
template <typename R>
sgp_status ens_run_persistent(sgp_ens* e, long long nsteps, double dt, int scheme) {
  // control word: no failure, no withheld signal (all bytes 0xff = -1)
  cudaError_t ce = cudaMemsetAsync(&e->ctl_dev->err, 0, 16, e->stream);   // err, pad, err_item
  if (ce == cudaSuccess) ce = cudaMemsetAsync(&e->ctl_dev->withhold, 0xff, sizeof(long long), e->stream);
  long long done = 0;
  while (ce == cudaSuccess && done < nsteps) {
    const long long steps = nsteps - done >= kGraphChunk ? kGraphChunk : nsteps - done;
    sgp_ens::PProg* p = nullptr;
    SGP_TRY(ens_persist_program<R>(e, steps, dt, scheme, &p));
    const bool stall = done == 0 && e->stall_member >= 0;
    if (stall) {
      // the member's first work item (pass 0) will not signal its completion
      const int g = e->member_group[e->stall_member];
      const long long withhold = p->lay.xoff[g] + (long long)e->member_index[e->stall_member] * p->lay.xi[g];
      ce = cudaMemcpyAsync(&e->ctl_dev->withhold, &withhold, sizeof(long long), cudaMemcpyHostToDevice,
                           e->stream);      // pageable source: staged before the call returns
      if (ce != cudaSuccess) break;
    }
    if (steps == kGraphChunk && !p->graph) {
      ce = cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal);
      if (ce != cudaSuccess) break;
      sgp_status st = ens_persist_issue<R>(e, *p);
      cudaGraph_t graph = nullptr;
      ce = cudaStreamEndCapture(e->stream, &graph);
      if (st != SGP_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
      }
      if (ce != cudaSuccess) break;
      ce = cudaGraphInstantiate(&p->graph, graph, 0);
      cudaGraphDestroy(graph);
      if (ce != cudaSuccess) break;
    }
    if (p->graph) {
      ce = cudaGraphLaunch(p->graph, e->stream);
    } else {
      SGP_TRY(ens_persist_issue<R>(e, *p));
    }
    if (ce == cudaSuccess && stall)
      ce = cudaMemsetAsync(&e->ctl_dev->withhold, 0xff, sizeof(long long), e->stream);
    e->launches += 1 + (long long)e->groups.size();
    done += steps;
  }
  PersistCtl ctl{};
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(&ctl, e->ctl_dev, sizeof ctl, cudaMemcpyDeviceToHost, e->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(e->stream);
  e->stall_member = -1;
  e->t += (double)nsteps * dt;
  for (sgp_ctx* c : e->groups) c->t = e->t;
  if (ce != cudaSuccess) return efail(e, SGP_ECUDA, "persistent run: %s", cudaGetErrorString(ce));
  if (ctl.err) {
    e->have_state = false;
    return efail(e, SGP_ETIMEOUT,
                 "a device-side wait gave up after %.3g s (work item %lld); the members' states are "
                 "undefined until they are set again",
                 e->wait_seconds, ctl.err_item);
  }
  return SGP_OK;
}

template <typename R>
sgp_status ens_run(sgp_ens* e, long long nsteps, double dt, int scheme) {
  if (e->persist_ok && e->use_persist) {
    for (sgp_ctx* c : e->groups) {
      k_set_time<<<1, 1, 0, e->stream>>>(c->t_dev, e->t);
      e->launches++;
    }
    return ens_run_persistent<R>(e, nsteps, dt, scheme);
  }
  for (sgp_ctx* c : e->groups) {
    k_set_time<<<1, 1, 0, e->stream>>>(c->t_dev, e->t);
    e->launches++;
  }
  cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) return efail(e, SGP_ECUDA, "set time: %s", cudaGetErrorString(ce));
  long long done = 0;
  if (nsteps >= kGraphChunk) {
    cudaGraphExec_t exec = nullptr;
    SGP_TRY(ens_graph<R>(e, kGraphChunk, dt, scheme, &exec));
    const long long reps = nsteps / kGraphChunk;
    for (long long r = 0; r < reps; ++r) {
      ce = cudaGraphLaunch(exec, e->stream);
      if (ce != cudaSuccess) return efail(e, SGP_ECUDA, "graph launch: %s", cudaGetErrorString(ce));
    }
    for (sgp_ctx* c : e->groups) e->launches += reps * chunk_launches(c, kGraphChunk, scheme);
    done = reps * kGraphChunk;
  }
  if (done < nsteps) {
    long long l0 = 0;
    for (sgp_ctx* c : e->groups) l0 += c->launches;
    SGP_TRY(ens_emit<R>(e, nsteps - done, dt, scheme, false));
    long long l1 = 0;
    for (sgp_ctx* c : e->groups) l1 += c->launches;
    e->launches += l1 - l0;
  }
  e->t += (double)nsteps * dt;
  for (sgp_ctx* c : e->groups) c->t = e->t;
  return SGP_OK;
}

}  // namespace

extern "C" {

sgp_status sgp_ensemble_destroy(sgp_ens* e);

sgp_status sgp_ensemble_create(int dim, int count, const int* n, const double* L, int prec,
                               int device, void* stream, sgp_ens** out) {
  g_create_err.clear();
  if (!out || !n || !L) return efail(nullptr, SGP_EINVAL, "NULL argument");
  *out = nullptr;
  if (count < 1) return efail(nullptr, SGP_EINVAL, "count must be >= 1");
  for (int m = 0; m < count; ++m) {
    sgp_status st = validate_grid(dim, n + (size_t)m * dim, L + (size_t)m * dim, 1, prec);
    if (st != SGP_OK) return efail(nullptr, st, "member %d: %s", m, g_create_err.c_str());
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return efail(nullptr, SGP_EINVAL, "CUDA device %d not available", device);
  DeviceGuard guard(device);
  sgp_ens* e = new sgp_ens();
  e->dim = dim;
  e->count = count;
  e->prec = prec;
  e->device = device;
  cudaError_t ce;
  if (stream) {
    e->stream = (cudaStream_t)stream;
  } else {
    if ((ce = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking)) != cudaSuccess) {
      sgp_ensemble_destroy(e);
      return efail(nullptr, SGP_ECUDA, "stream: %s", cudaGetErrorString(ce));
    }
    e->own_stream = true;
  }
  // group members by grid (sizes and half-widths)
  std::map<std::vector<double>, int> key2g;
  std::vector<std::vector<int>> members;
  e->member_group.resize(count);
  e->member_index.resize(count);
  for (int m = 0; m < count; ++m) {
    std::vector<double> key;
    for (int a = 0; a < dim; ++a) key.push_back(n[(size_t)m * dim + a]);
    for (int a = 0; a < dim; ++a) key.push_back(L[(size_t)m * dim + a]);
    auto it = key2g.find(key);
    int g;
    if (it == key2g.end()) {
      g = (int)members.size();
      key2g[key] = g;
      members.push_back({});
    } else {
      g = it->second;
    }
    e->member_group[m] = g;
    e->member_index[m] = (int)members[g].size();
    members[g].push_back(m);
  }
  for (size_t g = 0; g < members.size(); ++g) {
    const int m0 = members[g][0];
    cudaStream_t gs = nullptr;
    if ((ce = cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking)) != cudaSuccess) {
      sgp_ensemble_destroy(e);
      return efail(nullptr, SGP_ECUDA, "stream: %s", cudaGetErrorString(ce));
    }
    e->gstreams.push_back(gs);
    cudaEvent_t ev = nullptr;
    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    e->join.push_back(ev);
    sgp_ctx* c = nullptr;
    sgp_status st = sgp_create_grid(dim, n + (size_t)m0 * dim, L + (size_t)m0 * dim,
                                    (int)members[g].size(), prec, device, e->stream, &c);
    if (st != SGP_OK) {
      std::string msg = g_create_err;
      sgp_ensemble_destroy(e);
      return efail(nullptr, st, "group %zu: %s", g, msg.c_str());
    }
    e->groups.push_back(c);
  }
  cudaEventCreateWithFlags(&e->fork, cudaEventDisableTiming);
  // the persistent work-queue kernel: 2D ensembles whose every line length
  // it is compiled for
  int base = 0;
  for (sgp_ctx* c : e->groups) {
    e->gbase.push_back(base);
    base += c->batch;
  }
  bool ok = dim == 2 && (int)e->groups.size() <= kPersistMaxGroups;
  for (sgp_ctx* c : e->groups) ok = ok && persist_supported(c->n[0]) && persist_supported(c->n[1]);
  if (ok) {
    int bps = 0, sms = 0, khz = 0;
    ce = prec == SGP_F32 ? persist_prepare<float>(&bps) : persist_prepare<double>(&bps);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, device);
    if (ce == cudaSuccess && bps > 0) ce = dev_alloc(e->groups[0], (void**)&e->done_dev, sizeof(int) * count);
    if (ce == cudaSuccess && bps > 0) ce = dev_alloc(e->groups[0], (void**)&e->ctl_dev, sizeof(PersistCtl));
    if (ce != cudaSuccess) {
      sgp_ensemble_destroy(e);
      return efail(nullptr, SGP_ECUDA, "persistent kernel set-up: %s", cudaGetErrorString(ce));
    }
    e->persist_ok = bps > 0;
    e->persist_grid = bps * sms;
    if (khz <= 0) khz = 2000000;        // the limit is approximate: assume 2 GHz if unknown
    e->wait_cycles = (long long)(e->wait_seconds * khz * 1e3);
  }
  *out = e;
  return SGP_OK;
}

int sgp_ensemble_groups(const sgp_ens* e) { return e ? (int)e->groups.size() : 0; }

sgp_status sgp_ensemble_set_persistent(sgp_ens* e, int enable) {
  if (!e) return SGP_EINVAL;
  if (enable && !e->persist_ok)
    return efail(e, SGP_EUNSUPPORTED, "the persistent kernel needs a 2D ensemble of at most 32 grids "
                                      "with line lengths in {64, 96, 128, 192, 256, 384, 512}");
  e->use_persist = enable != 0;
  return SGP_OK;
}

int sgp_ensemble_persistent(const sgp_ens* e) { return e && e->persist_ok && e->use_persist ? 1 : 0; }

sgp_status sgp_ensemble_set_wait_limit(sgp_ens* e, double seconds) {
  if (!e) return SGP_EINVAL;
  if (!(seconds > 0.0) || !std::isfinite(seconds) || seconds > 3600.0)
    return efail(e, SGP_EINVAL, "wait limit must be in (0, 3600] seconds");
  int khz = 0;
  cudaError_t ce = cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, e->device);
  if (ce != cudaSuccess) return efail(e, SGP_ECUDA, "%s", cudaGetErrorString(ce));
  if (khz <= 0) khz = 2000000;
  e->wait_seconds = seconds;
  e->wait_cycles = (long long)(seconds * khz * 1e3);
  return SGP_OK;
}

sgp_status sgp_ensemble_inject_stall(sgp_ens* e, int member) {
  if (!e) return SGP_EINVAL;
  if (member < 0 || member >= e->count) return efail(e, SGP_EINVAL, "member %d out of range", member);
  if (!(e->persist_ok && e->use_persist)) return efail(e, SGP_EUNSUPPORTED, "the persistent kernel is not in use");
  e->stall_member = member;
  return SGP_OK;
}

sgp_status sgp_ensemble_set_params(sgp_ens* e, const sgp_params* p) {
  if (!e) return SGP_EINVAL;
  if (!p) return efail(e, SGP_EINVAL, "NULL params");
  DeviceGuard guard(e->device);
  ens_free_graphs(e);
  ens_free_progs(e);
  for (size_t g = 0; g < e->groups.size(); ++g) {
    sgp_ctx* c = e->groups[g];
    std::vector<sgp_params> sub(c->batch);
    for (int m = 0; m < e->count; ++m)
      if (e->member_group[m] == (int)g) sub[e->member_index[m]] = p[m];
    sgp_status st = sgp_set_params_batch(c, sub.data(), c->batch);
    if (st != SGP_OK) return efail(e, st, "%s", c->err.c_str());
  }
  return SGP_OK;
}

sgp_status sgp_ensemble_set_member_state(sgp_ens* e, int member, const void* src,
                                         int src_on_device, double t0) {
  if (!e) return SGP_EINVAL;
  if (member < 0 || member >= e->count) return efail(e, SGP_EINVAL, "member %d out of range", member);
  if (!src) return efail(e, SGP_EINVAL, "NULL src");
  if (!std::isfinite(t0)) return efail(e, SGP_EINVAL, "non-finite t0");
  if (e->have_state && t0 != e->t) return efail(e, SGP_EINVAL, "all members share the time");
  DeviceGuard guard(e->device);
  sgp_ctx* c = e->groups[e->member_group[member]];
  const size_t bytes = 5 * (size_t)c->ntot * c->elem;
  char* dst = (char*)c->field + (size_t)e->member_index[member] * bytes;
  cudaError_t ce = cudaMemcpyAsync(dst, src, bytes,
                                   src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                   e->stream);
  if (ce == cudaSuccess && !src_on_device) ce = cudaStreamSynchronize(e->stream);
  if (ce != cudaSuccess) return efail(e, SGP_ECUDA, "copy: %s", cudaGetErrorString(ce));
  e->t = t0;
  for (sgp_ctx* g : e->groups) {
    g->t = t0;
    g->have_state = true;
  }
  e->have_state = true;
  return SGP_OK;
}

sgp_status sgp_ensemble_get_member_state(sgp_ens* e, int member, void* dst, int dst_on_device) {
  if (!e) return SGP_EINVAL;
  if (member < 0 || member >= e->count) return efail(e, SGP_EINVAL, "member %d out of range", member);
  if (!dst) return efail(e, SGP_EINVAL, "NULL dst");
  DeviceGuard guard(e->device);
  sgp_ctx* c = e->groups[e->member_group[member]];
  const size_t bytes = 5 * (size_t)c->ntot * c->elem;
  const char* src = (const char*)c->field + (size_t)e->member_index[member] * bytes;
  cudaError_t ce = cudaMemcpyAsync(dst, src, bytes,
                                   dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                   e->stream);
  if (ce == cudaSuccess && !dst_on_device) ce = cudaStreamSynchronize(e->stream);
  if (ce != cudaSuccess) return efail(e, SGP_ECUDA, "copy: %s", cudaGetErrorString(ce));
  return SGP_OK;
}

sgp_status sgp_ensemble_step_host(sgp_ens* e, const void* const* host_in, double t0,
                                  void* const* host_out, long long nsteps, double dt, int scheme) {
  if (!e) return SGP_EINVAL;
  if (!host_in || !host_out) return efail(e, SGP_EINVAL, "NULL pointer array");
  for (int m = 0; m < e->count; ++m)
    if (!host_in[m] || !host_out[m]) return efail(e, SGP_EINVAL, "NULL host buffer (member %d)", m);
  if (!std::isfinite(t0)) return efail(e, SGP_EINVAL, "non-finite t0");
  if (nsteps < 0) return efail(e, SGP_EINVAL, "nsteps < 0");
  if (!(dt > 0.0) || !std::isfinite(dt)) return efail(e, SGP_EINVAL, "dt must be positive and finite");
  if (!valid_scheme(scheme)) return efail(e, SGP_EINVAL, "unknown scheme %d", scheme);
  DeviceGuard guard(e->device);
  // every copy in, the steps and every copy out in the order of the
  // ensemble stream, one synchronisation at the end.  When every buffer is
  // page-locked and mapped into the device (cudaHostAlloc, or registered),
  // each direction is one k_copy_members launch; otherwise one copy per
  // member and direction.
  std::vector<MemberXfer> xl;
  long long blocks[2] = {0, 0};
  for (int dir = 0; dir < 2; ++dir)
    for (int m = 0; m < e->count; ++m) {
      sgp_ctx* c = e->groups[e->member_group[m]];
      const size_t bytes = 5 * (size_t)c->ntot * c->elem;
      const void* h = dir == 0 ? host_in[m] : host_out[m];
      cudaPointerAttributes pa{};
      if (bytes % 16 != 0 || cudaPointerGetAttributes(&pa, h) != cudaSuccess ||
          pa.type != cudaMemoryTypeHost || !pa.devicePointer ||
          reinterpret_cast<uintptr_t>(pa.devicePointer) % 16 != 0) {
        cudaGetLastError();          // an unregistered pointer may leave an error behind
        xl.clear();
        dir = 2;
        break;
      }
      char* f = (char*)c->field + (size_t)e->member_index[m] * bytes;
      MemberXfer x;
      x.src = (const uint4*)(dir == 0 ? pa.devicePointer : (void*)f);
      x.dst = (uint4*)(dir == 0 ? (void*)f : pa.devicePointer);
      x.n16 = (long long)(bytes / 16);
      x.first = blocks[dir];
      blocks[dir] += (x.n16 + kXferChunk - 1) / kXferChunk;
      xl.push_back(x);
    }
  const bool kcopy = !xl.empty() && blocks[0] < (1LL << 31) && blocks[1] < (1LL << 31);
  cudaError_t ce = cudaSuccess;
  if (kcopy) {
    if (!e->xfer_dev)
      ce = dev_alloc(e->groups[0], (void**)&e->xfer_dev, 2 * sizeof(MemberXfer) * (size_t)e->count);
    // pageable source: staged before the call returns, in stream order
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(e->xfer_dev, xl.data(), xl.size() * sizeof(MemberXfer), cudaMemcpyHostToDevice,
                           e->stream);
    if (ce == cudaSuccess) {
      k_copy_members<<<(unsigned)blocks[0], kXferThreads, 0, e->stream>>>(e->xfer_dev, e->count);
      ce = cudaGetLastError();
      e->launches++;
    }
  } else {
    for (int m = 0; m < e->count && ce == cudaSuccess; ++m) {
      sgp_ctx* c = e->groups[e->member_group[m]];
      const size_t bytes = 5 * (size_t)c->ntot * c->elem;
      ce = cudaMemcpyAsync((char*)c->field + (size_t)e->member_index[m] * bytes, host_in[m], bytes,
                           cudaMemcpyHostToDevice, e->stream);
    }
  }
  if (ce != cudaSuccess) {
    cudaStreamSynchronize(e->stream);
    return efail(e, SGP_ECUDA, "copy in: %s", cudaGetErrorString(ce));
  }
  e->t = t0;
  for (sgp_ctx* g : e->groups) {
    g->t = t0;
    g->have_state = true;
  }
  e->have_state = true;
  sgp_status st = SGP_OK;
  if (nsteps > 0)
    st = e->prec == SGP_F32 ? ens_run<float>(e, nsteps, dt, scheme)
                            : ens_run<double>(e, nsteps, dt, scheme);
  if (kcopy) {
    if (st == SGP_OK) {
      k_copy_members<<<(unsigned)blocks[1], kXferThreads, 0, e->stream>>>(e->xfer_dev + e->count, e->count);
      ce = cudaGetLastError();
      e->launches++;
    }
  } else {
    for (int m = 0; m < e->count && st == SGP_OK && ce == cudaSuccess; ++m) {
      sgp_ctx* c = e->groups[e->member_group[m]];
      const size_t bytes = 5 * (size_t)c->ntot * c->elem;
      ce = cudaMemcpyAsync(host_out[m], (const char*)c->field + (size_t)e->member_index[m] * bytes,
                           bytes, cudaMemcpyDeviceToHost, e->stream);
    }
  }
  const cudaError_t cs = cudaStreamSynchronize(e->stream);   // host buffers free after this
  if (st != SGP_OK) return st;
  if (ce == cudaSuccess) ce = cs;
  if (ce != cudaSuccess) return efail(e, SGP_ECUDA, "copy out: %s", cudaGetErrorString(ce));
  return SGP_OK;
}

sgp_status sgp_ensemble_step(sgp_ens* e, long long nsteps, double dt, int scheme) {
  if (!e) return SGP_EINVAL;
  if (nsteps < 0) return efail(e, SGP_EINVAL, "nsteps < 0");
  if (!(dt > 0.0) || !std::isfinite(dt)) return efail(e, SGP_EINVAL, "dt must be positive and finite");
  if (!valid_scheme(scheme)) return efail(e, SGP_EINVAL, "unknown scheme %d", scheme);
  if (!e->have_state) return efail(e, SGP_ESTATE, "sgp_ensemble_step before any member state");
  if (nsteps == 0) return SGP_OK;
  DeviceGuard guard(e->device);
  return e->prec == SGP_F32 ? ens_run<float>(e, nsteps, dt, scheme)
                            : ens_run<double>(e, nsteps, dt, scheme);
}

sgp_status sgp_ensemble_observables(sgp_ens* e, sgp_obs* out) {
  if (!e) return SGP_EINVAL;
  if (!out) return efail(e, SGP_EINVAL, "NULL out");
  if (!e->have_state) return efail(e, SGP_ESTATE, "no state");
  DeviceGuard guard(e->device);
  int first_bad = -1;
  for (size_t g = 0; g < e->groups.size(); ++g) {
    sgp_ctx* c = e->groups[g];
    std::vector<sgp_obs> tmp(c->batch);
    sgp_status st = sgp_observables(c, tmp.data());
    if (st != SGP_OK && st != SGP_ENONFINITE) return efail(e, st, "%s", c->err.c_str());
    for (int m = 0; m < e->count; ++m)
      if (e->member_group[m] == (int)g) {
        out[m] = tmp[e->member_index[m]];
        if (!std::isfinite(out[m].mass) || !std::isfinite(out[m].energy) ||
            !std::isfinite(out[m].magnetization) || !std::isfinite(out[m].lz))
          if (first_bad < 0 || m < first_bad) first_bad = m;
      }
  }
  // every member is written; a non-finite one is reported like sgp_observables
  if (first_bad >= 0) return efail(e, SGP_ENONFINITE, "member %d: non-finite observables", first_bad);
  return SGP_OK;
}

sgp_status sgp_ensemble_autotune(sgp_ens* e, int reps, int flags) {
  if (!e) return SGP_EINVAL;
  DeviceGuard guard(e->device);
  for (sgp_ctx* g : e->groups) {
    sgp_status st = sgp_autotune(g, reps, flags, nullptr);
    if (st != SGP_OK) return efail(e, st, "%s", g->err.c_str());
  }
  ens_free_graphs(e);
  return SGP_OK;
}

sgp_status sgp_ensemble_synchronize(sgp_ens* e) {
  if (!e) return SGP_EINVAL;
  DeviceGuard guard(e->device);
  cudaError_t ce = cudaStreamSynchronize(e->stream);
  if (ce != cudaSuccess) return efail(e, SGP_ECUDA, "%s", cudaGetErrorString(ce));
  return SGP_OK;
}

long long sgp_ensemble_launch_count(const sgp_ens* e) { return e ? e->launches : 0; }

const char* sgp_ensemble_last_error(const sgp_ens* e) { return e ? e->err.c_str() : g_create_err.c_str(); }

sgp_status sgp_ensemble_destroy(sgp_ens* e) {
  if (!e) return SGP_OK;
  DeviceGuard guard(e->device);
  if (e->stream) cudaStreamSynchronize(e->stream);
  ens_free_graphs(e);
  if (!e->groups.empty()) {
    ens_free_progs(e);
    dev_free(e->groups[0], e->done_dev);
    dev_free(e->groups[0], e->ctl_dev);
    dev_free(e->groups[0], e->xfer_dev);
  }
  for (sgp_ctx* c : e->groups) sgp_destroy(c);
  for (cudaStream_t s : e->gstreams) cudaStreamDestroy(s);
  for (cudaEvent_t ev : e->join) cudaEventDestroy(ev);
  if (e->fork) cudaEventDestroy(e->fork);
  if (e->own_stream) cudaStreamDestroy(e->stream);
  delete e;
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
static __device__ __align__(256) MemberPrm g_static_prm[kStaticMaxBatch];

struct StaticScratch {
  double* partials = nullptr;
  double* sums = nullptr;
  void* tw = nullptr;
  MemberPrm* prm = nullptr;
};
constexpr int kMaxDevices = 64;
StaticScratch g_scratch[kMaxDevices];
bool g_scratch_ready[kMaxDevices] = {false};

sgp_status static_fail(sgp_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_create_err = buf;
  return s;
}

// Load every kernel sgp_observables_static can launch (all line lengths,
// both precisions) on the current device.  CUDA loads kernels lazily, at
// their first use, and loading places their code in device memory; doing it
// here, in the set-up, leaves nothing to load (or allocate) in later calls.
// cudaFuncSetAttribute (inside the prepare_* calls) and cudaFuncGetAttributes
// load the function they are given.
cudaError_t static_preload_kernels() {
  cudaError_t e = cudaSuccess;
#define SGP_PRELOAD(N)                                                         \
  if (e == cudaSuccess) e = prepare_xpass<float>(N);                           \
  if (e == cudaSuccess) e = prepare_linepass<float>(N);                        \
  if (e == cudaSuccess) e = prepare_xpass<double>(N);                          \
  if (e == cudaSuccess) e = prepare_linepass<double>(N);
  SGP_FOR_EACH_N(SGP_PRELOAD)
#undef SGP_PRELOAD
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_reduce_partials);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_twiddles_f32);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_twiddles_f64);
  return e;
}

// Device addresses of the scratch arrays for the current device, and every
// kernel loaded (set-up on the first call per device).
sgp_status static_scratch(int device, StaticScratch** out) {
  if (device < 0 || device >= kMaxDevices) return static_fail(SGP_EINVAL, "device %d out of range", device);
  if (!g_scratch_ready[device]) {
    StaticScratch sc;
    cudaError_t e;
    if ((e = cudaGetSymbolAddress((void**)&sc.partials, g_static_partials)) != cudaSuccess ||
        (e = cudaGetSymbolAddress((void**)&sc.sums, g_static_sums)) != cudaSuccess ||
        (e = cudaGetSymbolAddress(&sc.tw, g_static_tw)) != cudaSuccess ||
        (e = cudaGetSymbolAddress((void**)&sc.prm, g_static_prm)) != cudaSuccess)
      return static_fail(SGP_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    if ((e = static_preload_kernels()) != cudaSuccess)
      return static_fail(SGP_ECUDA, "loading the observables kernels: %s", cudaGetErrorString(e));
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
  for (int a = 0; a < dim; ++a) {
    e = sizeof(R) == 4 ? (a == 0 ? prepare_xpass<float>(n[a]) : prepare_linepass<float>(n[a]))
                       : (a == 0 ? prepare_xpass<double>(n[a]) : prepare_linepass<double>(n[a]));
    if (e != cudaSuccess) return static_fail(SGP_ECUDA, "kernel attributes: %s", cudaGetErrorString(e));
  }
  // parameters: one entry for every member, staged from the stack
  MemberPrm hp[kStaticMaxBatch];
  for (int m = 0; m < batch; ++m) hp[m] = member_prm(*prm, dim);
  if ((e = cudaMemcpyAsync(sc->prm, hp, sizeof(MemberPrm) * batch, cudaMemcpyHostToDevice, stream)) !=
      cudaSuccess)
    return static_fail(SGP_ECUDA, "parameters: %s", cudaGetErrorString(e));
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
  ax.t = t;
  ax.mp = sc->prm;
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
    assemble_obs(&hsum[(size_t)m * OB_NT], dim, cell, t, *prm, &out[m]);
    finite = finite && obs_finite(out[m]);
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
