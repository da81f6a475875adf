// Internal definitions of the HPG-MxP GB300 library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "hpgmxp.h"

namespace hpg {

constexpr int kSlots = 27;        // 27-point stencil (Sec. 2)
constexpr int kCentre = 13;       // slot of offset (0,0,0)
constexpr int kColours = 8;       // independent sets of the 27-point stencil
constexpr int kCoarseColour = 7;  // colour of the coarse-coincident points
constexpr int kMaxLevels = 8;
constexpr int kMaxRestart = 64;
constexpr int kRowAlign = 32;     // colour blocks start on 32-row boundaries
constexpr double kDiag = 26.0;    // diagonal of the stencil, times theta_i (Sec. 3)

// ------------------------------------------------------------ error handling
void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define HPG_CK(call)                                                     \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) return ::hpg::cuda_fail(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define HPG_CK_LAUNCH(what)                                              \
  do {                                                                   \
    cudaError_t e_ = cudaGetLastError();                                 \
    if (e_ != cudaSuccess) return ::hpg::cuda_fail(e_, what, __FILE__, __LINE__); \
  } while (0)

// ------------------------------------------------------------------ geometry
// Level geometry passed by value (as __grid_constant__) to every kernel that
// maps between grid coordinates and colour-blocked storage rows.
struct Geom {
  int nx, ny, nz;
  int cdx[kColours], cdy[kColours], cdz[kColours];  // colour-block extents
  long long off[kColours + 1];                      // colour-block starts
  long long n_store;
};

// Parity of i (resp. j, k) of the points in colour c: colour bit 0 is
// (i+1)&1, so bit set <=> i even.
__host__ __device__ inline int colour_parity_x(int c) { return 1 - (c & 1); }
__host__ __device__ inline int colour_parity_y(int c) { return 1 - ((c >> 1) & 1); }
__host__ __device__ inline int colour_parity_z(int c) { return 1 - ((c >> 2) & 1); }

__host__ __device__ inline int colour_of(int i, int j, int k) {
  return ((i + 1) & 1) | (((j + 1) & 1) << 1) | (((k + 1) & 1) << 2);
}

__host__ __device__ inline long long store_index(const Geom& g, int i, int j, int k) {
  const int c = colour_of(i, j, k);
  return g.off[c] + (long long)(i >> 1) +
         (long long)g.cdx[c] * ((long long)(j >> 1) + (long long)g.cdy[c] * (k >> 1));
}

// Colour of storage row `row` (blocks are ordered by colour).
__device__ inline int colour_of_row(const Geom& g, long long row) {
  int c = 0;
#pragma unroll
  for (int q = 1; q < kColours; ++q) c += (row >= g.off[q]) ? 1 : 0;
  return c;
}

// ------------------------------------------------------------- cached loads
// Matrix entries are read once per sweep: stream them past L1 and mark them
// evict-first in L2 so that the vectors stay resident.
__device__ __forceinline__ float ld_stream(const float* p) { return __ldcs(p); }
__device__ __forceinline__ double ld_stream(const double* p) { return __ldcs(p); }
__device__ __forceinline__ int ld_stream(const int* p) { return __ldcs(p); }

// Matrix load of the bandwidth-variant kernels: streamed (evict-first), or
// cached normally where the slice is read again soon (a streamed level's
// kept colour phases, levels below the streaming size).
template <bool STREAM, typename V>
__device__ __forceinline__ V ld_matrix(const V* p) {
  if (STREAM) return __ldcs(p);
  return __ldg(p);
}

// Load marked evict-last in L2 (an L2 cache policy made by createpolicy).
__device__ __forceinline__ unsigned long long l2_evict_last_policy() {
  unsigned long long pol;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ float ld_evict_last(const float* p) {
  float v;
  asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;"
      : "=f"(v) : "l"(p), "l"(l2_evict_last_policy()));
  return v;
}
__device__ __forceinline__ double ld_evict_last(const double* p) {
  double v;
  asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;"
      : "=d"(v) : "l"(p), "l"(l2_evict_last_policy()));
  return v;
}
__device__ __forceinline__ int ld_evict_last(const int* p) {
  int v;
  asm("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;"
      : "=r"(v) : "l"(p), "l"(l2_evict_last_policy()));
  return v;
}

// How a kernel reads a level's matrix: streamed evict-first (levels larger
// than L2), cached normally, or marked evict-last (the small coarse levels,
// read by every V-cycle: without the mark the finest level's traffic pushes
// them out of L2 between V-cycles).
enum MatLoad { kMatStream = 0, kMatCached = 1, kMatResident = 2 };
template <int MODE, typename V>
__device__ __forceinline__ V ld_mat(const V* p) {
  if constexpr (MODE == kMatStream) return __ldcs(p);
  else if constexpr (MODE == kMatResident) return ld_evict_last(p);
  else return __ldg(p);
}

// Levels whose FP32 ELL slots exceed this many bytes stream their matrix
// (evict-first); smaller (coarse) levels keep theirs in the 126 MB L2.
constexpr long long kStreamMatrixBytes = 96LL << 20;
// Levels whose FP32 ELL slots take at most this many bytes are read
// evict-last.  Measured on GB300 at 128^3: marking the 57 MB level 1 as well
// made its sweeps 2.5x slower, even alone.
constexpr long long kResidentMatrixBytes = 16LL << 20;

// ---------------------------------------------- programmatic dependent launch
// Kernels of the solve chain are launched with programmatic stream
// serialization: the next kernel may start while its predecessor drains.
// Every kernel calls pdl_trigger() on entry, may touch data that no earlier
// kernel of the chain writes (the matrix) before pdl_wait(), and reads or
// writes everything else only after pdl_wait(), which returns once all
// prerequisite grids have completed and their writes are visible.  Without a
// programmatic launch both are no-ops.
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Load of a vector that an earlier kernel of the chain wrote.  A kernel
// launched programmatically is alive while its predecessor still writes, so
// the read-only path (ld.global.nc: __ldg, or a const __restrict__ pointer
// the compiler lowers to it) is not valid for such data: it is only for data
// that no kernel writes while the reader runs (the matrix, or the input of a
// kernel that is never launched programmatically).  Measured on
// GB300: a multi-RHS Gauss-Seidel phase whose neighbour gathers took the
// read-only path, with its matrix slots loaded before pdl_wait(), returned
// values from before the previous kernel's writes on every run; with these
// coherent L1-cached loads (ld.global.ca) it is bitwise exact (the 128^3
// solve measured 0.13 % slower than with the read-only gathers).  The load is
// volatile inline assembly, so it stays after pdl_wait() in program order.
template <typename V>
__device__ __forceinline__ V ld_dep(const V* p) {
  return __ldca(p);
}

// Bulk prefetch of [p, p + bytes) into L2 by the TMA engine (no registers,
// no completion to wait for).  p must be 16-byte aligned, bytes a multiple
// of 16.
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// ------------------------------------------------- TMA bulk copies, mbarriers
// 1-D bulk copies global -> shared by the TMA engine, completion counted in
// bytes on a shared-memory mbarrier.  Addresses must be 16-byte aligned and
// sizes multiples of 16 bytes.
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}
// Bounded wait for the given phase parity; false if the limit ran out (each
// try_wait suspends for at most a short hardware-defined time, so the limit
// is well under a few seconds).
constexpr unsigned kMbarWaitLimit = 1u << 20;
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned phase) {
  for (unsigned it = 0; it < kMbarWaitLimit; ++it)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}

// Slots (bit s) a Gauss-Seidel phase of colour c reads.  Normally every slot;
// in the first forward sweep from z = 0 only the diagonal and the slots whose
// neighbour colour is below c: colours not yet visited are still zero, so
// their entries need not even be loaded.  An odd offset along an axis flips
// that axis's parity bit of the colour.
__host__ __device__ constexpr unsigned gs_slot_mask(int c, bool from_zero) {
  if (!from_zero) return (1u << 27) - 1u;
  unsigned m = 1u << 13;
  for (int s = 0; s < 27; ++s) {
    const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = s / 9 - 1;
    const int nc = c ^ ((dx & 1) | ((dy & 1) << 1) | ((dz & 1) << 2));
    if (nc < c) m |= 1u << s;
  }
  return m;
}

// One thread of the block prefetches the block's slice [row, row + rows) of
// the 27 value and index slots of a slot-major ELL matrix.  row and rows are
// multiples of 4 (colour blocks start on 32-row boundaries), so every range
// starts on a 16-byte boundary and has a multiple-of-16 size.
template <typename TV>
__device__ __forceinline__ void prefetch_ell_rows(const TV* vals, const int* cols, long long ns,
                                                  long long row, int rows) {
  if (threadIdx.x != 0 || rows <= 0) return;
  for (int s = 0; s < 27; ++s) {
    prefetch_l2_bulk(vals + s * ns + row, (unsigned)(rows * sizeof(TV)));
    prefetch_l2_bulk(cols + s * ns + row, (unsigned)(rows * sizeof(int)));
  }
}

// ------------------------------------------------------------ host objects
struct Level {
  Geom g;
  long long n = 0;        // grid points
  long long nnz = 0;      // structural non-zeros
  long long cnt[kColours] = {0};
  int* cols = nullptr;    // [27][n_store]
  float* v32 = nullptr;   // [27][n_store]
  double* v64 = nullptr;  // [27][n_store]
  double* theta = nullptr;  // natural order, or null
  // V-cycle work vectors of this level (coarse levels: restricted residual and
  // correction; every level: scratch), per precision: [0] FP64, [1] FP32.
  void* rhs[2] = {nullptr, nullptr};
  void* sol[2] = {nullptr, nullptr};
  // pipelined symmetric sweep (streamed levels): per-tile completion flags
  // [kMaxPipePhases][pipe_tiles] and the sweep's control words
  // (kPipeQueue, kPipeFinish, kPipeEpoch, kPipeAbort)
  int* pipe_flags = nullptr;
  unsigned* pipe_sync = nullptr;
  int pipe_tiles = 0;
};

constexpr int kPipeTileRows = 256;   // rows of one tile (= threads of its CTA)
constexpr int kMaxPipePhases = 16;   // colour phases of one symmetric sweep (15 used)
enum PipeWord { kPipeQueue = 0, kPipeFinish = 1, kPipeEpoch = 2, kPipeAbort = 3, kPipeWords = 4 };

struct Workspace;   // GMRES buffers (krylov.cu)
struct BatchSpace;  // multi-right-hand-side buffers and tuned launch shapes (batch.cu)
struct Profiler;    // per-kernel-class CUDA-event timing (profile.cu)

// Kernel classes reported by the profiler.
enum KernelClass {
  K_GEN = 0, K_PERMUTE, K_SPMV, K_RESIDUAL, K_GS, K_RESTRICT, K_PROLONG, K_CGS2_GEMVT,
  K_CGS2_REORTH, K_CGS2_FINAL, K_ARNOLDI_SCALE, K_TRSM, K_COMBINE, K_UPDATE_X,
  K_CYCLE_START, K_NORM, K_VCYCLE, K_GRADIENT, K_NUM_CLASSES
};
const char* kernel_class_name(int cls);

}  // namespace hpg

struct hpg_problem {
  int device = 0;
  int num_sms = 0;
  double beta = 0.0;
  int nlev = 1;
  int pre = 1, post = 1;
  bool hierarchy = false;
  hpg::Level lev[hpg::kMaxLevels];
  hpg::Workspace* ws = nullptr;
  hpg::BatchSpace* batch = nullptr;
  hpg::Profiler* prof = nullptr;
  long long launches = 0;   // kernel launches enqueued (diagnostics)
  bool profiling = false;   // event-bracketed launches, no PDL
  bool eager = false;       // host-driven solve instead of the solve graph
  bool pdl_enabled = true;  // programmatic dependent launch on the chain
  bool pdl_next = false;    // the previous stream operation was a kernel
  bool coarse_cluster = false;    // coarse levels of a V-cycle in one cluster kernel
  bool gs_halo = false;           // streamed GS phases stage z's neighbourhood in shared memory
  bool coarse_cta = false;        // coarsest level's sweep in one CTA when it fits
  long long pdl_rows = 16384;     // latency-variant GS phases launched programmatically up
                                  // to this many rows
  int gs_pipeline = 1;            // pipelined sweep kernel: 0 never; on streamed levels
                                  // 1 FP64 sweeps only (measured faster there), 2 always;
                                  // 3 every level
  unsigned* pipe_err = nullptr;   // device word: a pipelined sweep's wait ran out
  int vc_cluster[2] = {0, 0};     // its cluster size per precision (0: not probed, <0: none)
};

namespace hpg {

// Profiling: when enabled, every launch is bracketed by two CUDA events on
// its stream; prof_begin returns a slot (or -1 when disabled).
int prof_begin(hpg_problem* h, cudaStream_t s);
void prof_end(hpg_problem* h, int slot, int cls, int level, int prec, double bytes,
              cudaStream_t s);
void destroy_profiler(hpg_problem* h);

// Enqueues kernel<<<grid, block, 0, s>>>(args...), with the programmatic
// serialization attribute when the previous operation on s was a kernel of
// the chain (and not while profiling).
template <typename... KArgs, typename... Args>
cudaError_t kl(hpg_problem* h, void (*kern)(KArgs...), int grid, int block, cudaStream_t s,
               Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  if (h->pdl_enabled && h->pdl_next && !h->profiling) {
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// Launches `f` (a lambda that enqueues one kernel with kl), counts it,
// profiles it with its algorithmic DRAM bytes, and checks the launch.
template <typename F>
int launch(hpg_problem* h, int cls, int level, int prec, double bytes, cudaStream_t s,
           const char* what, F&& f) {
  const int slot = prof_begin(h, s);
  if (slot >= 0) h->pdl_next = false;
  const cudaError_t e0 = f();
  const cudaError_t e = e0 != cudaSuccess ? e0 : cudaGetLastError();
  prof_end(h, slot, cls, level, prec, bytes, s);
  h->launches++;
  h->pdl_next = true;
  if (e != cudaSuccess) return cuda_fail(e, what, __FILE__, __LINE__);
  return HPG_OK;
}

// Allocation helpers (cudaMalloc; zero-filled).
int dev_alloc(void** p, size_t bytes);
void dev_free(void* p);

// Launchers shared between translation units.  Every one returns HPG_OK or
// an error code and counts its launches in h->launches.
int launch_spmv(hpg_problem* h, int level, hpg_prec prec, const void* x, void* y,
                cudaStream_t s);
int launch_residual64(hpg_problem* h, const double* b, const double* x, double* r,
                      cudaStream_t s);
// c0_done: z already holds the first sweep's colour-0 phase, z_i = r_i / a_ii
// on colour block 0 (written by the kernel that produced r).
int run_vcycle(hpg_problem* h, int level, hpg_prec prec, const void* r, void* z,
               cudaStream_t s, bool c0_done = false);
// V-cycle from `level` down in one thread-block cluster; HPG_ERR_UNSUPPORTED
// when the level is too large or no cluster fits (the caller then launches
// one kernel per phase).
int launch_vcycle_cluster(hpg_problem* h, int level, hpg_prec prec, const void* r, void* z,
                          cudaStream_t s);
int launch_permute(hpg_problem* h, int level, int direction, hpg_prec in_prec,
                   const void* in, hpg_prec out_prec, void* out, cudaStream_t s);
void destroy_workspace(hpg_problem* h);
void destroy_batch(hpg_problem* h);
// Multi-system batches (hpg_batch_t) whose graph uses h's batch buffers.
int batch_owners(const hpg_problem* h);
// Drops h's captured multi-right-hand-side solve graph (recaptured on use).
void drop_batch_graph(hpg_problem* h);

inline size_t prec_size(hpg_prec p) {
  switch (p) {
    case HPG_FP64: return 8;
    case HPG_FP32: return 4;
    case HPG_BF16: return 2;
    case HPG_FP16: return 2;
  }
  return 0;
}

inline int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace hpg
