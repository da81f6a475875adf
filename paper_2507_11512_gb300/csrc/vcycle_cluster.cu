// The coarse part of the V-cycle in one thread-block cluster.
//
// Below the finest level every colour phase (Sec. 3.2.1) touches few rows
// and the data sit in L2, so a launch per phase is latency-bound (~2.5-5 us
// each, ~80 of them per cycle at 128^3).  Here one cluster of up to 16 CTAs
// of 1024 threads runs the whole V-cycle from a coarse level down to the
// coarsest and back (Fig. 1 applied recursively: symmetric multicolour
// Gauss-Seidel, the fused residual-restriction of Sec. 3.2.4, the injection
// prolongation of eq. (3)) from a host-built schedule of phases, separated by
// the hardware cluster barrier (barrier.cluster arrive.release / wait.acquire).
// Phases and arithmetic are those of the one-launch-per-phase V-cycle, so the
// results are equal; the first forward sweep from z = 0 also skips loading
// the ELL slots whose neighbours are known to be zero.
//
// Vectors are read through L2 (ld.global.cg) because other SMs of the
// cluster wrote them in earlier phases.

#include <cooperative_groups.h>
#include <string.h>

#include "hpg_internal.cuh"

namespace cg = cooperative_groups;

namespace hpg {

constexpr int kVcThreads = 1024;
constexpr int kMaxPhases = 448;
constexpr long long kClusterRows = 300000;   // levels with at most this many rows

enum PhaseKind { PH_GS = 0, PH_RESTRICT = 1, PH_PROLONG = 2, PH_ZERO = 3 };

struct VcLevel {
  Geom g;
  const int* cols;
  const void* vals;   // float* or double*, by the kernel's precision
};

struct VcPhase {
  unsigned char kind, level, colour, from_zero;
  const void* r;      // GS: rhs; RESTRICT: fine rhs
  void* z;            // GS: solution; RESTRICT: fine solution; PROLONG/ZERO: fine solution
  void* aux;          // RESTRICT: coarse rhs (out); PROLONG: coarse correction (in)
};

struct VcParams {
  int nphases;
  VcLevel lev[kMaxLevels];
  VcPhase ph[kMaxPhases];
};

// Colour of the neighbour at slot s of a row of colour c: an odd offset along
// an axis flips that axis's parity bit.
__device__ __forceinline__ int neighbour_colour(int c, int s) {
  const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = s / 9 - 1;
  return c ^ ((dx & 1) | ((dy & 1) << 1) | ((dz & 1) << 2));
}

// Rows handled by this thread: 32-row chunks dealt round-robin first over the
// cluster's CTAs, then over their warps, so a phase of a few hundred rows
// still spreads over every SM of the cluster and each warp reads 32
// consecutive rows per slot.  Levels run here have fewer than 2^31 / 27 slots,
// so 32-bit offsets suffice.
struct ClusterRows {
  int first, step;
  __device__ ClusterRows(unsigned rank, unsigned nctas) {
    const int gw = (threadIdx.x >> 5) * (int)nctas + (int)rank;
    first = gw * 32 + (threadIdx.x & 31);
    step = (int)nctas * kVcThreads;
  }
};

// One row's sum over slots [S0, S0 + NS): the indices and values of the
// group are loaded together, then the gathers, then the FMAs, so a warp pays
// two L2 round trips per group instead of two per slot (coarse phases have a
// warp or two per SM, nothing else hides the latency).  Slots whose
// neighbour is known to be zero are masked, not loaded.
template <typename T, int S0, int NS>
__device__ __forceinline__ T row_group(const T* __restrict__ vals, const int* __restrict__ cols,
                                       const T* x, int ns, int row, int c, bool from_zero,
                                       int valid_end, T acc) {
  int col[NS];
  T a[NS];
  bool use[NS];
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    const int s = S0 + i;
    use[i] = !(from_zero && neighbour_colour(c, s) >= c);
    col[i] = use[i] ? __ldg(cols + s * ns + row) : 0;
    a[i] = use[i] ? __ldg(vals + s * ns + row) : T(0);
  }
  T xv[NS];
#pragma unroll
  for (int i = 0; i < NS; ++i) xv[i] = (use[i] && col[i] < valid_end) ? __ldcg(x + col[i]) : T(0);
#pragma unroll
  for (int i = 0; i < NS; ++i)
    if (use[i]) acc = fma(-a[i], xv[i], acc);
  return acc;
}

template <typename T>
__device__ void phase_gs(const VcParams& P, const VcPhase& ph, const ClusterRows& cr) {
  const VcLevel& L = P.lev[ph.level];
  const T* __restrict__ vals = static_cast<const T*>(L.vals);
  const int* __restrict__ cols = L.cols;
  const T* r = static_cast<const T*>(ph.r);
  T* x = static_cast<T*>(ph.z);
  const int ns = (int)L.g.n_store;
  const int c = ph.colour;
  const bool from_zero = ph.from_zero != 0;
  const int row0 = (int)L.g.off[c], row1 = (int)L.g.off[c + 1];
  const int valid_end = from_zero ? row0 : ns;
  for (int row = row0 + cr.first; row < row1; row += cr.step) {
    const T diag = __ldg(vals + kCentre * ns + row);
    T acc = __ldcg(r + row);
    acc = row_group<T, 0, 13>(vals, cols, x, ns, row, c, from_zero, valid_end, acc);
    acc = row_group<T, 14, 13>(vals, cols, x, ns, row, c, from_zero, valid_end, acc);
    x[row] = acc / diag;
  }
}

template <typename T>
__device__ void phase_restrict(const VcParams& P, const VcPhase& ph, const ClusterRows& cr) {
  const VcLevel& F = P.lev[ph.level];
  const VcLevel& C = P.lev[ph.level + 1];
  const T* __restrict__ vals = static_cast<const T*>(F.vals);
  const int* __restrict__ cols = F.cols;
  const T* r = static_cast<const T*>(ph.r);
  const T* z = static_cast<const T*>(ph.z);
  T* rc = static_cast<T*>(ph.aux);
  const int ns = (int)F.g.n_store;
  const int cx = F.g.cdx[kCoarseColour], cy = F.g.cdy[kCoarseColour];
  const int cnt = cx * cy * F.g.cdz[kCoarseColour];
  const int row0 = (int)F.g.off[kCoarseColour];
  for (int p = cr.first; p < cnt; p += cr.step) {
    const int row = row0 + p;
    T acc = __ldcg(r + row);
    // same slot order as the one-launch-per-phase restriction: 0..26
    acc = row_group<T, 0, 14>(vals, cols, z, ns, row, 0, false, ns, acc);
    acc = row_group<T, 14, 13>(vals, cols, z, ns, row, 0, false, ns, acc);
    const int I = p % cx;
    const int J = (p / cx) % cy;
    const int K = p / (cx * cy);
    rc[store_index(C.g, I, J, K)] = acc;
  }
}

template <typename T>
__device__ void phase_prolong(const VcParams& P, const VcPhase& ph, const ClusterRows& cr) {
  const VcLevel& F = P.lev[ph.level];
  const VcLevel& C = P.lev[ph.level + 1];
  T* z = static_cast<T*>(ph.z);
  const T* zc = static_cast<const T*>(ph.aux);
  const int cx = F.g.cdx[kCoarseColour], cy = F.g.cdy[kCoarseColour];
  const int cnt = cx * cy * F.g.cdz[kCoarseColour];
  const int row0 = (int)F.g.off[kCoarseColour];
  for (int p = cr.first; p < cnt; p += cr.step) {
    const int I = p % cx;
    const int J = (p / cx) % cy;
    const int K = p / (cx * cy);
    z[row0 + p] = __ldcg(z + row0 + p) + __ldcg(zc + store_index(C.g, I, J, K));
  }
}

template <typename T>
__device__ void phase_zero(const VcParams& P, const VcPhase& ph, const ClusterRows& cr) {
  T* z = static_cast<T*>(ph.z);
  const int ns = (int)P.lev[ph.level].g.n_store;
  for (int row = cr.first; row < ns; row += cr.step) z[row] = T(0);
}

template <typename T>
__global__ void __launch_bounds__(kVcThreads, 1)
vcycle_cluster_kernel(const __grid_constant__ VcParams P) {
  pdl_wait();   // the fine level's restriction wrote the coarse rhs
  cg::cluster_group cluster = cg::this_cluster();
  const ClusterRows cr(cluster.block_rank(), cluster.num_blocks());
  for (int ip = 0; ip < P.nphases; ++ip) {
    const VcPhase& ph = P.ph[ip];
    switch (ph.kind) {
      case PH_GS: phase_gs<T>(P, ph, cr); break;
      case PH_RESTRICT: phase_restrict<T>(P, ph, cr); break;
      case PH_PROLONG: phase_prolong<T>(P, ph, cr); break;
      default: phase_zero<T>(P, ph, cr); break;
    }
    if (ip + 1 < P.nphases) cluster.sync();
  }
  pdl_trigger();
}

// --------------------------------------------------------------- host side
template <typename T> struct VcPrec;
template <> struct VcPrec<float> {
  static constexpr int idx = 1;
  static const void* vals(const Level& L) { return L.v32; }
};
template <> struct VcPrec<double> {
  static constexpr int idx = 0;
  static const void* vals(const Level& L) { return L.v64; }
};

struct Schedule {
  VcParams* P;
  int n = 0;
  bool ok = true;
  int last[kMaxLevels];
  double bytes = 0.0;
  double sv = 4, sx = 4;
};

static void push(Schedule& S, const VcPhase& ph) {
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

static VcPhase make_phase(int kind, int level) {
  VcPhase ph;
  memset(&ph, 0, sizeof(ph));
  ph.kind = (unsigned char)kind;
  ph.level = (unsigned char)level;
  return ph;
}

static void sched_gs(hpg_problem* h, Schedule& S, int l, const void* r, void* z, int c,
                     bool from_zero) {
  if (S.last[l] == c) return;   // same colour again: identical result, skipped
  S.last[l] = c;
  VcPhase ph = make_phase(PH_GS, l);
  ph.colour = (unsigned char)c;
  ph.from_zero = from_zero ? 1 : 0;
  ph.r = r;
  ph.z = z;
  push(S, ph);
  const int k = needed_slots(c, from_zero);
  S.bytes += (double)h->lev[l].cnt[c] * ((k + 1) * S.sv + k * 4.0 + (2.0 + k / 26.0) * S.sx);
}

static void sched_symgs(hpg_problem* h, Schedule& S, int l, const void* r, void* z,
                        bool from_zero) {
  for (int c = 0; c < kColours; ++c) sched_gs(h, S, l, r, z, c, from_zero);
  for (int c = kColours - 1; c >= 0; --c) sched_gs(h, S, l, r, z, c, false);
}

// Mirrors the one-launch-per-phase V-cycle exactly (same phases, same order).
static void sched_vcycle(hpg_problem* h, Schedule& S, int l, const void* r, void* z, int pi) {
  S.last[l] = -1;
  if (l == h->nlev - 1) {
    sched_symgs(h, S, l, r, z, true);
    return;
  }
  if (h->pre == 0) {
    VcPhase ph = make_phase(PH_ZERO, l);
    ph.z = z;
    push(S, ph);
  }
  for (int it = 0; it < h->pre; ++it) sched_symgs(h, S, l, r, z, it == 0);
  const Level& C = h->lev[l + 1];
  VcPhase ph = make_phase(PH_RESTRICT, l);
  ph.r = r;
  ph.z = z;
  ph.aux = C.rhs[pi];
  push(S, ph);
  S.bytes += (double)C.n * (27.0 * (S.sv + 4.0) + 3.0 * S.sx);
  sched_vcycle(h, S, l + 1, C.rhs[pi], C.sol[pi], pi);
  ph = make_phase(PH_PROLONG, l);
  ph.z = z;
  ph.aux = C.sol[pi];
  push(S, ph);
  S.bytes += (double)C.n * 3.0 * S.sx;
  S.last[l] = -1;
  for (int it = 0; it < h->post; ++it) sched_symgs(h, S, l, r, z, false);
}

// CTAs of the cluster: 16 (non-portable size) when the device can place such
// a cluster of 1024-thread CTAs, else 8; 0 if neither.
template <typename T>
static int cluster_size_for(hpg_problem* h) {
  int& cached = h->vc_cluster[VcPrec<T>::idx];
  if (cached != 0) return cached;
  cached = -1;
  cudaFuncSetAttribute(vcycle_cluster_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed,
                       1);
  for (int cs : {16, 8}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cs);
    cfg.blockDim = dim3(kVcThreads);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, vcycle_cluster_kernel<T>, &cfg) ==
            cudaSuccess &&
        nclusters >= 1) {
      cached = cs;
      break;
    }
  }
  cudaGetLastError();
  return cached;
}

template <typename T>
static int launch_vc_t(hpg_problem* h, int level, const T* r, T* z, cudaStream_t s) {
  const int cs = cluster_size_for<T>(h);
  if (cs <= 0) return HPG_ERR_UNSUPPORTED;
  static thread_local VcParams P;   // 14 KB: kept off the stack; copied at launch
  memset(&P, 0, sizeof(P));
  Schedule S;
  S.P = &P;
  S.sv = sizeof(T);
  S.sx = sizeof(T);
  for (int l = 0; l < kMaxLevels; ++l) S.last[l] = -1;
  for (int l = 0; l < h->nlev; ++l) {
    P.lev[l].g = h->lev[l].g;
    P.lev[l].cols = h->lev[l].cols;
    P.lev[l].vals = VcPrec<T>::vals(h->lev[l]);
  }
  sched_vcycle(h, S, level, r, z, VcPrec<T>::idx);
  if (!S.ok) return HPG_ERR_UNSUPPORTED;
  P.nphases = S.n;
  return launch(h, K_VCYCLE, level, VcPrec<T>::idx == 0 ? HPG_FP64 : HPG_FP32, S.bytes, s,
                "vcycle_cluster_kernel", [&] {
                  cudaLaunchConfig_t cfg = {};
                  cfg.gridDim = dim3((unsigned)cs);
                  cfg.blockDim = dim3(kVcThreads);
                  cfg.stream = s;
                  cudaLaunchAttribute attr[2];
                  attr[0].id = cudaLaunchAttributeClusterDimension;
                  attr[0].val.clusterDim.x = (unsigned)cs;
                  attr[0].val.clusterDim.y = 1;
                  attr[0].val.clusterDim.z = 1;
                  cfg.attrs = attr;
                  cfg.numAttrs = 1;
                  if (h->pdl_enabled && h->pdl_next && !h->profiling) {
                    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
                    attr[1].val.programmaticStreamSerializationAllowed = 1;
                    cfg.numAttrs = 2;
                  }
                  return cudaLaunchKernelEx(&cfg, vcycle_cluster_kernel<T>, P);
                });
}

int launch_vcycle_cluster(hpg_problem* h, int level, hpg_prec prec, const void* r, void* z,
                          cudaStream_t s) {
  if (!h->coarse_cluster || h->lev[level].g.n_store > kClusterRows) return HPG_ERR_UNSUPPORTED;
  if (prec == HPG_FP64)
    return launch_vc_t<double>(h, level, (const double*)r, (double*)z, s);
  return launch_vc_t<float>(h, level, (const float*)r, (float*)z, s);
}

}  // namespace hpg
