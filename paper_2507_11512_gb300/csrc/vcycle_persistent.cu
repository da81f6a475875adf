// The whole V-cycle (Fig. 1 applied recursively, Sec. 3.2.1 multicolour
// symmetric Gauss-Seidel, Sec. 3.2.4 fused residual-restriction, eq. (3)
// prolongation) as one persistent cooperative kernel.
//
// The multi-launch V-cycle costs one dependent kernel per colour phase
// (~110 per cycle); below the finest level each of those is latency-bound.
// Here one grid of one 1024-thread CTA per SM walks a host-built schedule of
// phases and synchronises between phases with a bounded grid barrier:
//   * finest/large levels: all CTAs; each CTA owns a contiguous, 32-row
//     aligned slice of the phase's rows, and before arriving at the barrier
//     it issues TMA bulk L2 prefetches of its slice of the *next* phase's
//     ELL slots, so the matrix stream continues through the barrier;
//   * small levels (<= kSmallRows rows): the first kSmallCtas CTAs only,
//     with their own barrier; the other CTAs go straight to the next
//     all-CTA barrier.
// Phases, their order and their arithmetic are exactly those of the
// multi-launch V-cycle (bitwise-equal results), except that the first forward
// sweep from z = 0 does not even load the ELL slots whose neighbours are
// known to be zero (colours not yet visited).
//
// Vectors are read through L2 (ld.global.cg): values written by another SM in
// an earlier phase must not be served from a stale L1 line.  Every spin-wait
// is bounded; on timeout the kernel raises a device status word that the
// solve reports (HPG_ERR_TIMEOUT) and all CTAs leave.

#include <string.h>

#include "hpg_internal.cuh"

namespace hpg {

constexpr int kPvcThreads = 1024;
constexpr int kMaxPhases = 448;
constexpr long long kSmallRows = 65536;   // levels with at most this many rows
constexpr int kSmallCtas = 16;            // ... run on this many CTAs
constexpr unsigned long long kSpinLimit = 1ULL << 22;   // ~0.2 s of polling

enum PhaseKind { PH_GS = 0, PH_RESTRICT = 1, PH_PROLONG = 2, PH_ZERO = 3 };

struct PvcLevel {
  Geom g;
  const int* cols;
  const void* vals;   // float* or double*, by the kernel's precision
};

struct PvcPhase {
  unsigned char kind, level, colour, from_zero;
  int ncta;           // CTAs that work on this phase
  const void* r;      // GS: rhs; RESTRICT: fine rhs
  void* z;            // GS: solution; RESTRICT: fine solution; PROLONG/ZERO: fine solution
  void* aux;          // RESTRICT: coarse rhs (out); PROLONG: coarse correction (in)
};

struct PvcParams {
  int nphases;
  int nsmall;         // CTAs of the small barrier
  unsigned* bar;      // [0] count, [32] generation of the all-CTA barrier; [64], [96]: small
  int* status;
  PvcLevel lev[kMaxLevels];
  PvcPhase ph[kMaxPhases];
};

// --------------------------------------------------------------- barrier
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile(const int* p) {
  return *reinterpret_cast<const volatile int*>(p);
}

// Generation barrier among `n` CTAs.  Thread 0 reads the generation, makes
// the CTA's writes visible (fence), arrives; the last arrival resets the
// count and publishes the next generation; the others poll it (bounded).
// Returns false (in every thread) if any CTA gave up.
__device__ bool pvc_barrier(unsigned* bar, unsigned n, int* status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned* count = bar;
    unsigned* gen = bar + 32;
    const unsigned g = ld_acquire_gpu(gen);
    __threadfence();
    int ok = 1;
    if (atomicAdd(count, 1u) + 1u == n) {
      atomicExch(count, 0u);
      __threadfence();
      st_release_gpu(gen, g + 1u);
    } else {
      unsigned long long spins = 0;
      while (ld_acquire_gpu(gen) == g) {
        if (ld_volatile(status) != 0) {
          ok = 0;
          break;
        }
        if (++spins > kSpinLimit) {
          atomicExch(status, HPG_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    s_ok = ok && ld_volatile(status) == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

// ------------------------------------------------------------- phase work
// Colour of the neighbour at slot s of a row of colour c: an odd offset along
// an axis flips that axis's parity bit.
__device__ __forceinline__ int neighbour_colour(int c, int s) {
  const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = s / 9 - 1;
  return c ^ ((dx & 1) | ((dy & 1) << 1) | ((dz & 1) << 2));
}

// Slice [beg, end) of `count` rows starting at row0 owned by CTA b of n:
// contiguous, split on 32-row boundaries.
__device__ __forceinline__ void cta_slice(long long row0, long long count, int b, int n,
                                          long long& beg, long long& end) {
  const long long chunks = (count + 31) / 32;
  beg = row0 + (chunks * b / n) * 32;
  end = row0 + (chunks * (b + 1) / n) * 32;
  if (end > row0 + count) end = row0 + count;
  if (beg > end) beg = end;
}

template <typename T>
__device__ void phase_gs(const PvcParams& P, const PvcPhase& ph) {
  const PvcLevel& L = P.lev[ph.level];
  const T* __restrict__ vals = static_cast<const T*>(L.vals);
  const int* __restrict__ cols = L.cols;
  const T* r = static_cast<const T*>(ph.r);
  T* x = static_cast<T*>(ph.z);
  const long long ns = L.g.n_store;
  const int c = ph.colour;
  const long long row0 = L.g.off[c];
  const long long valid_end = ph.from_zero ? row0 : ns;
  long long beg, end;
  cta_slice(row0, L.g.off[c + 1] - row0, blockIdx.x, ph.ncta, beg, end);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (long long q = beg + 32LL * warp; q < end; q += 32LL * (kPvcThreads / 32)) {
    const long long row = q + lane;
    if (row >= end) break;
    T acc = __ldcg(r + row);
#pragma unroll
    for (int s = 0; s < kSlots; ++s) {
      if (s == kCentre) continue;
      if (ph.from_zero && neighbour_colour(c, s) >= c) continue;   // neighbour still zero
      const T a = ld_stream(vals + s * ns + row);
      const int col = ld_stream(cols + s * ns + row);
      const T xv = (col < valid_end) ? __ldcg(x + col) : T(0);
      acc = fma(-a, xv, acc);
    }
    const T diag = ld_stream(vals + kCentre * ns + row);
    x[row] = acc / diag;
  }
}

template <typename T>
__device__ void phase_restrict(const PvcParams& P, const PvcPhase& ph) {
  const PvcLevel& F = P.lev[ph.level];
  const PvcLevel& C = P.lev[ph.level + 1];
  const T* __restrict__ vals = static_cast<const T*>(F.vals);
  const int* __restrict__ cols = F.cols;
  const T* r = static_cast<const T*>(ph.r);
  const T* z = static_cast<const T*>(ph.z);
  T* rc = static_cast<T*>(ph.aux);
  const long long ns = F.g.n_store;
  const int cx = F.g.cdx[kCoarseColour], cy = F.g.cdy[kCoarseColour];
  const long long cnt = (long long)cx * cy * F.g.cdz[kCoarseColour];
  const long long row0 = F.g.off[kCoarseColour];
  long long beg, end;
  cta_slice(row0, cnt, blockIdx.x, ph.ncta, beg, end);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (long long q = beg + 32LL * warp; q < end; q += 32LL * (kPvcThreads / 32)) {
    const long long row = q + lane;
    if (row >= end) break;
    T acc = __ldcg(r + row);
#pragma unroll
    for (int s = 0; s < kSlots; ++s) {
      const T a = ld_stream(vals + s * ns + row);
      const int col = ld_stream(cols + s * ns + row);
      acc = fma(-a, __ldcg(z + col), acc);
    }
    const long long p = row - row0;
    const int I = (int)(p % cx);
    const int J = (int)((p / cx) % cy);
    const int K = (int)(p / ((long long)cx * cy));
    rc[store_index(C.g, I, J, K)] = acc;
  }
}

template <typename T>
__device__ void phase_prolong(const PvcParams& P, const PvcPhase& ph) {
  const PvcLevel& F = P.lev[ph.level];
  const PvcLevel& C = P.lev[ph.level + 1];
  T* z = static_cast<T*>(ph.z);
  const T* zc = static_cast<const T*>(ph.aux);
  const int cx = F.g.cdx[kCoarseColour], cy = F.g.cdy[kCoarseColour];
  const long long cnt = (long long)cx * cy * F.g.cdz[kCoarseColour];
  const long long row0 = F.g.off[kCoarseColour];
  long long beg, end;
  cta_slice(row0, cnt, blockIdx.x, ph.ncta, beg, end);
  for (long long row = beg + threadIdx.x; row < end; row += kPvcThreads) {
    const long long p = row - row0;
    const int I = (int)(p % cx);
    const int J = (int)((p / cx) % cy);
    const int K = (int)(p / ((long long)cx * cy));
    z[row] = __ldcg(z + row) + __ldcg(zc + store_index(C.g, I, J, K));
  }
}

template <typename T>
__device__ void phase_zero(const PvcParams& P, const PvcPhase& ph) {
  const PvcLevel& L = P.lev[ph.level];
  T* z = static_cast<T*>(ph.z);
  long long beg, end;
  cta_slice(0, L.g.n_store, blockIdx.x, ph.ncta, beg, end);
  for (long long row = beg + threadIdx.x; row < end; row += kPvcThreads) z[row] = T(0);
}

// Bulk L2 prefetch of this CTA's slice of a GS / restriction phase's slots.
template <typename T>
__device__ void prefetch_phase(const PvcParams& P, const PvcPhase& ph) {
  if (ph.kind != PH_GS && ph.kind != PH_RESTRICT) return;
  const PvcLevel& L = P.lev[ph.level];
  const long long ns = L.g.n_store;
  long long row0, count;
  if (ph.kind == PH_GS) {
    row0 = L.g.off[ph.colour];
    count = L.g.off[ph.colour + 1] - row0;
  } else {
    row0 = L.g.off[kCoarseColour];
    count = L.g.off[kCoarseColour + 1] - row0;   // whole 32-row aligned block
  }
  long long beg, end;
  cta_slice(row0, count, blockIdx.x, ph.ncta, beg, end);
  // slices start on 32-row boundaries; round the length up to 32 rows (still
  // inside the padded colour block) so every range is a multiple of 16 bytes
  long long len = (end - beg + 31) / 32 * 32;
  if (beg + len > row0 + ((count + 31) / 32) * 32) len = row0 + ((count + 31) / 32) * 32 - beg;
  if (len <= 0) return;
  const int t = threadIdx.x;
  if (t < 2 * kSlots) {
    const int s = t % kSlots;
    if (ph.kind == PH_GS && ph.from_zero && s != kCentre &&
        neighbour_colour(ph.colour, s) >= ph.colour)
      return;
    if (t < kSlots)
      prefetch_l2_bulk(static_cast<const T*>(L.vals) + s * ns + beg, (unsigned)(len * sizeof(T)));
    else if (s != kCentre || ph.kind == PH_RESTRICT)
      prefetch_l2_bulk(L.cols + s * ns + beg, (unsigned)(len * sizeof(int)));
  }
}

template <typename T>
__global__ void __launch_bounds__(kPvcThreads, 1) vcycle_persistent_kernel(
    const __grid_constant__ PvcParams P) {
  if (ld_volatile(P.status) != 0) return;
  const unsigned nall = gridDim.x;
  for (int ip = 0; ip < P.nphases; ++ip) {
    const PvcPhase& ph = P.ph[ip];
    if (ip == P.nphases - 1) pdl_trigger();
    if ((int)blockIdx.x < ph.ncta) {
      switch (ph.kind) {
        case PH_GS: phase_gs<T>(P, ph); break;
        case PH_RESTRICT: phase_restrict<T>(P, ph); break;
        case PH_PROLONG: phase_prolong<T>(P, ph); break;
        default: phase_zero<T>(P, ph); break;
      }
    }
    if (ip + 1 == P.nphases) break;
    const PvcPhase& nx = P.ph[ip + 1];
    const int nbar = ph.ncta > nx.ncta ? ph.ncta : nx.ncta;
    if ((int)blockIdx.x >= nbar) continue;
    if ((int)blockIdx.x < nx.ncta && nx.ncta == (int)nall) prefetch_phase<T>(P, nx);
    const bool all = nbar == (int)nall;
    if (!pvc_barrier(P.bar + (all ? 0 : 64), all ? nall : (unsigned)P.nsmall, P.status)) return;
  }
}

// --------------------------------------------------------------- host side
template <typename T> struct PvcPrec;
template <> struct PvcPrec<float> {
  static constexpr int idx = 1;
  static const void* vals(const Level& L) { return L.v32; }
};
template <> struct PvcPrec<double> {
  static constexpr int idx = 0;
  static const void* vals(const Level& L) { return L.v64; }
};

struct Schedule {
  PvcParams* P;
  int n = 0;
  bool ok = true;
  int last[kMaxLevels];
  int nfull = 0;
  int nsmall = 0;
  double bytes = 0.0;
  size_t sv = 4, sx = 4;
};

static int level_ctas(const hpg_problem* h, const Schedule& S, int l) {
  return h->lev[l].g.n_store > kSmallRows ? S.nfull : S.nsmall;
}

static void push(Schedule& S, PvcPhase ph) {
  if (S.n >= kMaxPhases) {
    S.ok = false;
    return;
  }
  S.P->ph[S.n++] = ph;
}

static int needed_slots(int c, bool from_zero) {
  int k = 0;
  for (int s = 0; s < kSlots; ++s) {
    if (s == kCentre) continue;
    const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = s / 9 - 1;
    const int nc = c ^ ((dx & 1) | ((dy & 1) << 1) | ((dz & 1) << 2));
    if (!from_zero || nc < c) ++k;
  }
  return k;
}

static void sched_gs(hpg_problem* h, Schedule& S, int l, const void* r, void* z, int c,
                     bool from_zero) {
  if (S.last[l] == c) return;   // same colour again: identical result, skipped
  S.last[l] = c;
  PvcPhase ph;
  memset(&ph, 0, sizeof(ph));
  ph.kind = PH_GS;
  ph.level = (unsigned char)l;
  ph.colour = (unsigned char)c;
  ph.from_zero = from_zero ? 1 : 0;
  ph.ncta = level_ctas(h, S, l);
  ph.r = r;
  ph.z = z;
  push(S, ph);
  const int k = needed_slots(c, from_zero);
  S.bytes += (double)h->lev[l].cnt[c] * ((k + 1) * S.sv + k * 4.0 + (2 + k / 26.0) * S.sx);
}

static void sched_symgs(hpg_problem* h, Schedule& S, int l, const void* r, void* z,
                        bool from_zero) {
  for (int c = 0; c < kColours; ++c) sched_gs(h, S, l, r, z, c, from_zero);
  for (int c = kColours - 1; c >= 0; --c) sched_gs(h, S, l, r, z, c, false);
}

static void sched_vcycle(hpg_problem* h, Schedule& S, int l, const void* r, void* z, int pi) {
  S.last[l] = -1;
  if (l == h->nlev - 1) {
    sched_symgs(h, S, l, r, z, true);
    return;
  }
  if (h->pre == 0) {
    PvcPhase ph;
    memset(&ph, 0, sizeof(ph));
    ph.kind = PH_ZERO;
    ph.level = (unsigned char)l;
    ph.ncta = level_ctas(h, S, l);
    ph.z = z;
    push(S, ph);
  }
  for (int it = 0; it < h->pre; ++it) sched_symgs(h, S, l, r, z, it == 0);
  const Level& L = h->lev[l];
  const Level& C = h->lev[l + 1];
  const long long cnt = C.n;
  PvcPhase ph;
  memset(&ph, 0, sizeof(ph));
  ph.kind = PH_RESTRICT;
  ph.level = (unsigned char)l;
  ph.ncta = level_ctas(h, S, l);
  ph.r = r;
  ph.z = z;
  ph.aux = C.rhs[pi];
  push(S, ph);
  S.bytes += (double)cnt * (27.0 * (S.sv + 4.0) + 3.0 * S.sx);
  sched_vcycle(h, S, l + 1, C.rhs[pi], C.sol[pi], pi);
  memset(&ph, 0, sizeof(ph));
  ph.kind = PH_PROLONG;
  ph.level = (unsigned char)l;
  ph.ncta = level_ctas(h, S, l);
  ph.z = z;
  ph.aux = C.sol[pi];
  push(S, ph);
  S.bytes += (double)cnt * 3.0 * S.sx;
  S.last[l] = -1;
  for (int it = 0; it < h->post; ++it) sched_symgs(h, S, l, r, z, false);
  (void)L;
}

// Grid of the persistent kernel: one 1024-thread CTA per SM, if the device
// can keep them all resident for a cooperative launch.
static int pvc_grid(hpg_problem* h) {
  if (h->pvc_ctas != 0) return h->pvc_ctas;
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device);
  int per_sm_f = 0, per_sm_d = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_f, vcycle_persistent_kernel<float>,
                                                kPvcThreads, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_d, vcycle_persistent_kernel<double>,
                                                kPvcThreads, 0);
  cudaGetLastError();
  h->pvc_ctas = (coop && per_sm_f >= 1 && per_sm_d >= 1) ? h->num_sms : -1;
  return h->pvc_ctas;
}

template <typename T>
static int launch_pvc_t(hpg_problem* h, int level, const T* r, T* z, cudaStream_t s) {
  const int grid = pvc_grid(h);
  if (grid <= 0 || !h->pvc_bar || !h->dev_status) return HPG_ERR_UNSUPPORTED;
  static thread_local PvcParams P;   // 15 KB: kept off the stack
  memset(&P, 0, sizeof(P));
  Schedule S;
  S.P = &P;
  S.nfull = grid;
  S.nsmall = grid < kSmallCtas ? grid : kSmallCtas;
  S.sv = sizeof(T);
  S.sx = sizeof(T);
  for (int l = 0; l < kMaxLevels; ++l) S.last[l] = -1;
  const int pi = PvcPrec<T>::idx;
  for (int l = 0; l < h->nlev; ++l) {
    P.lev[l].g = h->lev[l].g;
    P.lev[l].cols = h->lev[l].cols;
    P.lev[l].vals = PvcPrec<T>::vals(h->lev[l]);
  }
  sched_vcycle(h, S, level, r, z, pi);
  if (!S.ok) return HPG_ERR_UNSUPPORTED;
  P.nphases = S.n;
  P.nsmall = S.nsmall;
  P.bar = h->pvc_bar;
  P.status = h->dev_status;
  h->pdl_next = false;   // cooperative grid: full serialisation with the predecessor
  return launch(h, K_VCYCLE, level, PvcPrec<T>::idx == 0 ? HPG_FP64 : HPG_FP32, S.bytes, s,
                "vcycle_persistent_kernel", [&] {
                  cudaLaunchConfig_t cfg = {};
                  cfg.gridDim = dim3((unsigned)grid);
                  cfg.blockDim = dim3(kPvcThreads);
                  cfg.stream = s;
                  cudaLaunchAttribute attr[1];
                  attr[0].id = cudaLaunchAttributeCooperative;
                  attr[0].val.cooperative = 1;
                  cfg.attrs = attr;
                  cfg.numAttrs = 1;
                  return cudaLaunchKernelEx(&cfg, vcycle_persistent_kernel<T>, P);
                });
}

int launch_pvc(hpg_problem* h, int level, hpg_prec prec, const void* r, void* z,
               cudaStream_t s) {
  if (prec == HPG_FP64) return launch_pvc_t<double>(h, level, (const double*)r, (double*)z, s);
  return launch_pvc_t<float>(h, level, (const float*)r, (float*)z, s);
}

}  // namespace hpg
