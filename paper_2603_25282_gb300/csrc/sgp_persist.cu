// sgp_persist.cu -- the persistent work-queue kernel of 2D ensembles for one
// precision (SGP_REAL); see sgp_persist.cuh.
#include "sgp_persist.cuh"

#ifndef SGP_REAL
#error "define SGP_REAL (float or double)"
#endif

#define SGP_PERSIST_N(X) X(64) X(96) X(128) X(192) X(256) X(384) X(512)

namespace sgp {

namespace {

constexpr int kPersistThreads = 256;

template <typename R, int N>
struct PCfg {
  static constexpr int E = elems_per_thread<R, N>();
  typedef XCfg<R, N, E, 0> X;        // x-pass: ~256 threads per CTA
  typedef LCfg<R, N, E, 1> Lc;       // line pass: ~256 threads per CTA
  static_assert(X::THREADS == kPersistThreads && Lc::THREADS == kPersistThreads,
                "the persistent kernel runs every pass with 256 threads");
  static constexpr size_t SMEM = X::SMEM > Lc::SMEM + Lc::TAB ? X::SMEM : Lc::SMEM + Lc::TAB;
};

template <typename R>
constexpr size_t persist_smem() {
  size_t m = 0;
#define SGP_MAXS(NN) m = PCfg<R, NN>::SMEM > m ? PCfg<R, NN>::SMEM : m;
  SGP_PERSIST_N(SGP_MAXS)
#undef SGP_MAXS
  return m;
}

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <typename R>
__device__ __forceinline__ void run_item(const PersistPass<R>& p, int tile, int member,
                                         unsigned char* smem) {
  if (p.kind == PK_XPASS) {
    switch (p.N) {
#define SGP_XCASE(NN)                                                             \
  case NN:                                                                        \
    xpass_body<R, NN, PCfg<R, NN>::E, 0, true>(p.x, tile, member, smem);          \
    break;
      SGP_PERSIST_N(SGP_XCASE)
#undef SGP_XCASE
      default:
        break;
    }
  } else {
    switch (p.N) {
#define SGP_LCASE(NN)                                                             \
  case NN:                                                                        \
    linepass_body<R, NN, PCfg<R, NN>::E, 1, true>(p.l, tile, 0, member, smem);    \
    break;
      SGP_PERSIST_N(SGP_LCASE)
#undef SGP_LCASE
      default:
        break;
    }
  }
}

// Work items in queue order; see sgp_persist.cuh.  Thread 0 takes the
// items: the index of the next one is fetched (atomicAdd) while the current
// one is processed.  The item's pass p, group, member and tiles follow from
// the program's layout by 32-bit arithmetic; for a pass after the member's
// first, thread 0 waits until the member's counter of finished items
// reaches the items of its earlier passes, (p + 1)/2 x-passes and p/2 line
// passes (bounded by wait_cycles of clock64).  The field is read with
// L2-only loads (other CTAs wrote it); after a CTA barrier, thread 0 fences
// at gpu scope (the fence is cumulative: it orders the stores the barrier
// made visible to it) and signals the item done.
template <typename R>
__global__ void __launch_bounds__(kPersistThreads, 2)
k_ens_persistent(const PersistPass<R>* __restrict__ prog, const __grid_constant__ PersistLayout lay,
                 int nitems, int* done, PersistCtl* ctl, long long wait_cycles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) PersistPass<R> s_pass;
  __shared__ int s_stop, s_ent, s_tile0, s_tile1, s_member, s_slot, s_item;
  const int pair = lay.IX + lay.IL;
  int next = 0;
  if (threadIdx.x == 0) next = (int)atomicAdd(&ctl->head, 1ull);
  while (true) {
    if (threadIdx.x == 0) {
      const int it = next;
      int stop = 0, ent = 0, tile0 = 0, tile1 = 0, ml = 0, slot = 0;
      if (it >= nitems || *(volatile int*)&ctl->err != 0) {
        stop = 1;
      } else {
        next = (int)atomicAdd(&ctl->head, 1ull);      // the following item, fetched early
        // pass p: x-passes and line passes alternate
        const int q = it / pair;
        int r = it - q * pair;
        const bool line = r >= lay.IX;
        if (line) r -= lay.IX;
        const int p = 2 * q + (line ? 1 : 0);
        const int* off = line ? lay.loff : lay.xoff;
        int g = 0;
        while (g + 1 < lay.groups && off[g + 1] <= r) ++g;
        const int items = line ? lay.li[g] : lay.xi[g];
        const int tiles = line ? lay.lt[g] : lay.xt[g];
        const int rl = r - off[g];
        ml = rl / items;
        tile0 = (rl - ml * items) * kTilesPerItem;
        tile1 = tile0 + kTilesPerItem < tiles ? tile0 + kTilesPerItem : tiles;
        ent = p * lay.groups + g;
        slot = lay.base[g] + ml;
        const int need = ((p + 1) / 2) * lay.xi[g] + (p / 2) * lay.li[g];
        if (need > 0) {
          const long long t0 = clock64();
          while (ld_acquire(done + slot) < need) {
            if (*(volatile int*)&ctl->err != 0) {
              stop = 1;
              break;
            }
            if (clock64() - t0 > wait_cycles) {
              if (atomicCAS(&ctl->err, 0, 1) == 0) ctl->err_item = it;
              stop = 1;
              break;
            }
            __nanosleep(64);
          }
        }
      }
      s_item = it;
      s_stop = stop;
      s_ent = ent;
      s_tile0 = tile0;
      s_tile1 = tile1;
      s_member = ml;
      s_slot = slot;
    }
    // the item's descriptor to shared memory by warp 0 (the decision above
    // is warp 0's own), then one barrier for the whole CTA
    if (threadIdx.x < 32) {
      __syncwarp();
      if (!s_stop) {
        const int* src = reinterpret_cast<const int*>(prog + s_ent);
        int* dst = reinterpret_cast<int*>(&s_pass);
        for (int k = threadIdx.x; k < (int)(sizeof(PersistPass<R>) / sizeof(int)); k += 32)
          dst[k] = __ldg(src + k);
      }
    }
    __syncthreads();
    if (s_stop) break;
    for (int t = s_tile0; t < s_tile1; ++t) {
      if (t > s_tile0) __syncthreads();     // the previous tile's shared-memory reads are done
      run_item<R>(s_pass, t, s_member, smem_raw);
    }
    // every thread's stores of the item, then one gpu-scope fence (cumulative
    // over the barrier) before the completion signal
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      if (s_item != ctl->withhold) atomicAdd(done + s_slot, 1);
    }
  }
}

}  // namespace

typedef SGP_REAL Real;
static_assert(sizeof(PersistPass<Real>) % sizeof(int) == 0, "descriptor copied as ints");

template <>
int persist_xrows<Real>(int N) {
  switch (N) {
#define SGP_C(NN) case NN: return PCfg<Real, NN>::X::ROWS;
    SGP_PERSIST_N(SGP_C)
#undef SGP_C
    default: return 0;
  }
}

template <>
int persist_ltile<Real>(int N) {
  switch (N) {
#define SGP_C(NN) case NN: return PCfg<Real, NN>::Lc::TILE;
    SGP_PERSIST_N(SGP_C)
#undef SGP_C
    default: return 0;
  }
}

template <>
cudaError_t persist_prepare<Real>(int* blocks_per_sm) {
  constexpr size_t smem = persist_smem<Real>();
  cudaError_t e = cudaFuncSetAttribute(k_ens_persistent<Real>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_ens_persistent<Real>,
                                                       kPersistThreads, smem);
}

template <>
cudaError_t launch_persistent<Real>(const PersistPass<Real>* prog, const PersistLayout& lay,
                                    int nitems, int* done, PersistCtl* ctl,
                                    long long wait_cycles, int grid, cudaStream_t s) {
  k_ens_persistent<Real><<<grid, kPersistThreads, persist_smem<Real>(), s>>>(prog, lay, nitems, done,
                                                                             ctl, wait_cycles);
  return cudaGetLastError();
}

#if SGP_PERSIST_DEFINE_SUPPORTED
bool persist_supported(int N) {
  switch (N) {
#define SGP_C(NN) case NN:
    SGP_PERSIST_N(SGP_C)
#undef SGP_C
    return true;
    default:
      return false;
  }
}
#endif

}  // namespace sgp
