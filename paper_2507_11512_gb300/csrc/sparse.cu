// Stencil-matrix kernels: ELLPACK SpMV, the FP64 outer residual, one colour
// phase of multicolour Gauss-Seidel, the fused residual-restriction and the
// injection prolongation, plus the V-cycle that strings them together.
//
// Kernels read the slot-major ELL arrays by level size: streaming
// (evict-first) where the matrix is larger than L2, normally cached on
// mid-size levels, and marked evict-last on the small coarse levels (read by
// every V-cycle; measured on GB300 at 128^3, this cut a V-cycle from 570 to
// 494 us).  x is gathered through the read-only path; rows of one colour block
// are contiguous, so a warp reads each slot of 32 consecutive rows as one
// 128-byte (FP32) or 256-byte (FP64) transaction.

#include <limits.h>
#include <string.h>

#include <algorithm>

#include "hpg_internal.cuh"

namespace hpg {

template <typename T> struct Prec;
template <> struct Prec<float> {
  static constexpr int idx = 1;
  static const float* vals(const Level& L) { return L.v32; }
};
template <> struct Prec<double> {
  static constexpr int idx = 0;
  static const double* vals(const Level& L) { return L.v64; }
};

// ------------------------------------------------------------------ kernels
// y = A x over all storage rows (Sec. 3.2.2; Algorithm 3 SpMV).
template <typename T>
__global__ void __launch_bounds__(256)
spmv_kernel(const T* __restrict__ vals, const int* __restrict__ cols, long long ns,
            const T* __restrict__ x, T* __restrict__ y) {
  pdl_trigger();
  const long long row0 = blockIdx.x * (long long)blockDim.x;
  prefetch_ell_rows(vals, cols, ns, row0, (int)min((long long)blockDim.x, ns - row0));
  pdl_wait();
  const long long row = row0 + threadIdx.x;
  if (row >= ns) return;
  T acc = T(0);
#pragma unroll
  for (int s = 0; s < kSlots; ++s) {
    const T a = ld_stream(vals + s * ns + row);
    const int c = ld_stream(cols + s * ns + row);
    acc = fma(a, ld_dep(x + c), acc);
  }
  y[row] = acc;
}

// r = b - A x in FP64 (Algorithm 3, outer residual).
__global__ void __launch_bounds__(256)
residual64_kernel(const double* __restrict__ vals, const int* __restrict__ cols, long long ns,
                  const double* __restrict__ b, const double* __restrict__ x,
                  double* __restrict__ r) {
  pdl_trigger();
  const long long row0 = blockIdx.x * (long long)blockDim.x;
  prefetch_ell_rows(vals, cols, ns, row0, (int)min((long long)blockDim.x, ns - row0));
  pdl_wait();
  const long long row = row0 + threadIdx.x;
  if (row >= ns) return;
  double acc = ld_dep(b + row);
#pragma unroll
  for (int s = 0; s < kSlots; ++s) {
    const double a = ld_stream(vals + s * ns + row);
    const int c = ld_stream(cols + s * ns + row);
    acc = fma(-a, ld_dep(x + c), acc);
  }
  r[row] = acc;
}

// Rows a thread of a bandwidth-variant Gauss-Seidel phase takes, and the
// 16-byte vector types that load one slot of them at once.
template <typename T> struct PhaseRows;
template <> struct PhaseRows<float> {
  static constexpr int R = 4;
  using V = float4;
  using I = int4;
};
template <> struct PhaseRows<double> {
  static constexpr int R = 2;
  using V = double2;
  using I = int2;
};
__device__ __forceinline__ void split_rows(const float4& v, float (&o)[4]) {
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void split_rows(const double2& v, double (&o)[2]) {
  o[0] = v.x; o[1] = v.y;
}
__device__ __forceinline__ float4 join_rows(const float (&o)[4]) {
  return make_float4(o[0], o[1], o[2], o[3]);
}
__device__ __forceinline__ double2 join_rows(const double (&o)[2]) {
  return make_double2(o[0], o[1]);
}
__device__ __forceinline__ void split_rows(const int4& v, int (&o)[4]) {
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void split_rows(const int2& v, int (&o)[2]) {
  o[0] = v.x; o[1] = v.y;
}

// One Gauss-Seidel colour phase (Sec. 3.2.1, relaxation form of eq. (1)):
// for every row i of the colour block [row0, row0 + nrows),
//   x_i <- (r_i - sum_{j != i} a_ij x_j) / a_ii.
// The block is an independent set, so no row reads a value written by this
// launch.  Entries x_j with j >= valid_end read as zero: the first forward
// sweep from z = 0 passes valid_end = start of the current colour block, so
// that colours not yet visited count as zero without a memset.
//
// Bandwidth variant, for levels whose matrix streams from HBM: a thread takes
// PhaseRows<T>::R consecutive rows and loads each slot's values and indices
// for them as one 16-byte vector (the colour blocks start and end on 32-row
// boundaries, so the rows divide evenly and the loads are aligned), and r
// and x likewise: the launcher sends vectors off a 16-byte boundary (caller
// pointers) to the one-row-per-thread latency kernel instead, whose per-row
// arithmetic is the same (a branch on the alignment inside this kernel cost
// 1 %).  Each row's
// arithmetic is the one-row-per-thread kernel's, in the same order.  Two
// 256-thread CTAs per SM with 128 registers, so a thread has its rows' loads
// in flight at once (a 128^3 FP32 phase is 256 CTAs, one wave).  Measured on
// GB300 against one row per thread in 32 registers (8 CTAs per SM): level-0
// phase 10.72 -> 9.35 us, 128^3 solve 102.8 -> 97.4 ms, 320^3 3534 ->
// 3401 ms; 2 rows per thread in 64 registers 99.7 ms, 4 rows in 64 or 80
// registers 103.0 / 101.9 ms, 4 rows in 128-thread CTAs 97.7 ms.  The
// matrix is read evict-first.  No early trigger and no load before the
// programmatic wait: measured on GB300, letting the next phase's CTAs start
// early (or prefetching its slots into L2) slows this bandwidth-bound chain
// down; launched with the programmatic attribute but triggering only as its
// blocks exit, the next launch is prepared while a phase drains (faster).
//
// MC = -1 reads every slot.  MC = c (0..7) is the phase of colour c in the
// first forward sweep from z = 0: only the slots whose neighbour colour is
// below c are loaded (the others multiply zeros), and the set is fixed at
// compile time, so the loads of a row issue as one straight-line batch.  A
// run-time slot mask made these phases no faster than full ones on GB300
// (colour 0, which loads only the diagonal, took 70 % of a full phase).
template <typename T, bool STREAM, int MC>
__global__ void __launch_bounds__(256, 2)
gs_phase_kernel(const T* __restrict__ vals, const int* __restrict__ cols, long long ns,
                const T* __restrict__ r, T* x, long long row0, long long nrows,
                long long valid_end) {
  constexpr unsigned kMask = MC < 0 ? (1u << kSlots) - 1u : gs_slot_mask(MC, true);
  constexpr int NR = PhaseRows<T>::R;
  using V = typename PhaseRows<T>::V;
  using I = typename PhaseRows<T>::I;
  pdl_wait();
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (NR * t >= nrows) return;
  const long long row = row0 + NR * t;
  T acc[NR];
  split_rows(ld_dep(reinterpret_cast<const V*>(r + row)), acc);
#pragma unroll
  for (int s = 0; s < kSlots; ++s) {
    if (s == kCentre || !((kMask >> s) & 1u)) continue;
    T a[NR];
    int c[NR];
    split_rows(ld_matrix<STREAM>(reinterpret_cast<const V*>(vals + s * ns + row)), a);
    split_rows(ld_matrix<STREAM>(reinterpret_cast<const I*>(cols + s * ns + row)), c);
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      const T xv = (c[q] < valid_end) ? ld_dep(x + c[q]) : T(0);
      acc[q] = fma(-a[q], xv, acc[q]);
    }
  }
  T diag[NR];
  split_rows(ld_matrix<STREAM>(reinterpret_cast<const V*>(vals + kCentre * ns + row)), diag);
#pragma unroll
  for (int q = 0; q < NR; ++q) acc[q] = acc[q] / diag[q];
  *reinterpret_cast<V*>(x + row) = join_rows(acc);
}

// The bandwidth-variant instantiation of a phase of colour c.
template <typename T, bool STREAM>
using GsPhaseFn = void (*)(const T*, const int*, long long, const T*, T*, long long, long long,
                           long long);
template <typename T, bool STREAM>
static GsPhaseFn<T, STREAM> gs_phase_fn(int c, bool from_zero) {
  if (!from_zero) return gs_phase_kernel<T, STREAM, -1>;
  switch (c) {
    case 0: return gs_phase_kernel<T, STREAM, 0>;
    case 1: return gs_phase_kernel<T, STREAM, 1>;
    case 2: return gs_phase_kernel<T, STREAM, 2>;
    case 3: return gs_phase_kernel<T, STREAM, 3>;
    case 4: return gs_phase_kernel<T, STREAM, 4>;
    case 5: return gs_phase_kernel<T, STREAM, 5>;
    case 6: return gs_phase_kernel<T, STREAM, 6>;
    default: return gs_phase_kernel<T, STREAM, 7>;
  }
}

// A colour block's rows (a multiple of kRowAlign) split evenly into the
// bandwidth-variant phase's rows per thread.
static_assert(kRowAlign % PhaseRows<float>::R == 0 && kRowAlign % PhaseRows<double>::R == 0,
              "colour blocks must split evenly into a thread's rows");

// TMA-tiled variant of the streamed phase (option HPG_OPT_GS_HALO): a CTA
// takes whole x-lines of its colour block -- lines J0 .. J0+L-1 of plane K --
// and moves everything its rows read into shared memory with 1-D bulk
// asynchronous copies (TMA) completing on one mbarrier: the 27 value and 26
// index slices of its rows, their r, and the z values the rows can touch.  A
// neighbour of a point of colour c in colour c' lies in plane K or K-1 / K+1
// of block c' (which one follows from c's z parity, when c and c' differ in
// z), and in lines J0-1 .. J0+L-1 or J0 .. J0+L of it (likewise in y), whole
// lines in x: at most 11 contiguous runs of block storage per tile.  Then
// every thread computes its row from shared memory alone; a gather reads
// index col + delta[slot], delta being the shared-memory offset of the run
// holding that slot's neighbours minus the run's start in the vector.  Same
// slots, order and arithmetic as gs_phase_kernel: results equal bit for bit.
// STREAM marks the matrix copies evict-first in L2.  The copy wait is
// bounded: if it runs out the CTA sets `err` (the solve then reports
// HPG_ERR_TIMEOUT), waits (bounded) once more for its copies and skips its
// rows.
constexpr int kHaloMaxThreads = 256;
constexpr int kHaloRuns = 24;   // (colour, plane offset) pairs: 8 x 3

template <typename T>
__host__ __device__ constexpr int halo_align() { return 16 / (int)sizeof(T); }

// Lines per CTA for a colour block with x extent cdx (whole lines, at most
// kHaloMaxThreads rows); 0 if a line alone is longer.
__host__ __device__ inline int halo_lines(int cdx) {
  return cdx > kHaloMaxThreads || cdx < 1 ? 0 : kHaloMaxThreads / cdx;
}
// Elements of one staged row slice (the tile's rows, aligned out on both ends).
__host__ __device__ inline int halo_rpad(int rows, int align) {
  return (rows + 2 * align + align - 1) / align * align;
}

__device__ __forceinline__ void bulk_g2s_evict_first(void* dst, const void* src, unsigned bytes,
                                                     unsigned long long* bar,
                                                     unsigned long long pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1], %2, [%3], %4;"
      ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
      : "memory");
}

template <typename T, bool STREAM>
__global__ void __launch_bounds__(kHaloMaxThreads)
gs_phase_halo_kernel(const T* __restrict__ vals, const int* __restrict__ cols, long long ns,
                     const T* __restrict__ r, T* x, const __grid_constant__ Geom g, int c,
                     int L, unsigned* err) {
  extern __shared__ __align__(16) unsigned char halo_smem[];
  __shared__ unsigned long long bar;
  __shared__ long long run_delta[kHaloRuns];
  __shared__ int sdelta[kSlots];
  __shared__ unsigned s_total;
  constexpr int A = halo_align<T>();
  const int cdx = g.cdx[c], cdy = g.cdy[c];
  const int njt = (cdy + L - 1) / L;
  const int K = blockIdx.x / njt;
  const int J0 = (blockIdx.x % njt) * L;
  const int Lr = min(L, cdy - J0);
  const int nrows = Lr * cdx;
  const int rpad = halo_rpad(L * cdx, A);
  const long long row0 = g.off[c] + (long long)cdx * (J0 + (long long)cdy * K);
  const long long row_al = row0 & ~(long long)(A - 1);
  const int shift = (int)(row0 - row_al);
  const unsigned slice = (unsigned)((shift + nrows + A - 1) / A * A);   // elements
  T* sv = reinterpret_cast<T*>(halo_smem);                 // [27][rpad]
  int* sc = reinterpret_cast<int*>(sv + kSlots * rpad);     // [27][rpad]
  T* sr = reinterpret_cast<T*>(sc + kSlots * rpad);         // [rpad]
  T* sx = sr + rpad;                                        // staged z runs
  if (threadIdx.x < 32) {
    // lane i plans z run i = (colour c2 = i / 3, plane offset dk = i % 3 - 1)
    const int lane = threadIdx.x;
    const int pz = colour_parity_z(c), py = colour_parity_y(c);
    long long gs_al = 0;
    unsigned elems = 0;
    if (lane < kHaloRuns) {
      const int c2 = lane / 3, dk = lane % 3 - 1;
      const int diff = c ^ c2;
      bool use = c2 != c;
      if (dk != 0) use = use && (diff & 4) && (dk == -1 ? pz == 0 : pz == 1);
      int jlo = J0, jhi = J0 + Lr - 1;
      if (diff & 2) {
        if (py == 0) jlo -= 1;
        else jhi += 1;
      }
      jlo = max(jlo, 0);
      jhi = min(jhi, g.cdy[c2] - 1);
      const int kp = K + dk;
      use = use && kp >= 0 && kp < g.cdz[c2] && jlo <= jhi;
      if (use) {
        const long long gs0 =
            g.off[c2] + (long long)g.cdx[c2] * (jlo + (long long)g.cdy[c2] * kp);
        const long long ge0 = gs0 + (long long)g.cdx[c2] * (jhi - jlo + 1);
        gs_al = gs0 & ~(long long)(A - 1);
        const long long ge_al = (ge0 + A - 1) & ~(long long)(A - 1);
        elems = (unsigned)(ge_al - gs_al);
      }
    }
    // exclusive prefix sum of the run sizes: shared-memory offsets
    unsigned incl = elems;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    const unsigned soff = incl - elems;
    const unsigned zt = __shfl_sync(0xffffffffu, incl, 31);
    if (lane < kHaloRuns)
      run_delta[lane] = elems ? (long long)soff - gs_al : (long long)(-(1LL << 40));
    if (lane == 0) {
      mbar_init(&bar, 1);
      fence_mbar_init();
      // 27 value slices, 26 index slices (not the centre's), r, the z runs
      mbar_expect_tx(&bar, (unsigned)sizeof(T) * (kSlots * slice + slice + zt) +
                               4u * (kSlots - 1) * slice);
      s_total = zt;
    }
    __syncwarp();
    unsigned long long pol = 0;
    if (STREAM)
      asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    if (elems) bulk_g2s(sx + soff, x + gs_al, elems * (unsigned)sizeof(T), &bar);
    if (lane < kSlots) {
      const T* vsrc = vals + lane * ns + row_al;
      if (STREAM)
        bulk_g2s_evict_first(sv + lane * rpad, vsrc, slice * (unsigned)sizeof(T), &bar, pol);
      else
        bulk_g2s(sv + lane * rpad, vsrc, slice * (unsigned)sizeof(T), &bar);
      if (lane != kCentre) {
        const int* csrc = cols + lane * ns + row_al;
        if (STREAM)
          bulk_g2s_evict_first(sc + lane * rpad, csrc, slice * 4u, &bar, pol);
        else
          bulk_g2s(sc + lane * rpad, csrc, slice * 4u, &bar);
      }
    }
    if (lane == kSlots) bulk_g2s(sr, r + row_al, slice * (unsigned)sizeof(T), &bar);
    __syncwarp();
    if (lane < kSlots && lane != kCentre) {
      const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
      const int c2 = c ^ ((dx & 1) | ((dy & 1) << 1) | ((dz & 1) << 2));
      const int dk = (pz + dz) >> 1;   // floor: -1, 0 or +1
      const long long d = run_delta[c2 * 3 + dk + 1];
      sdelta[lane] = (d < -(1LL << 31) || d > (1LL << 31)) ? INT_MIN / 2 : (int)d;
    }
  }
  __syncthreads();
  if (!mbar_wait(&bar, 0)) {
    if (threadIdx.x == 0 && err) atomicExch(err, 2u);
    mbar_wait(&bar, 0);   // bounded: the copies target this CTA's shared memory
    return;
  }
  const int t = threadIdx.x;
  if (t >= nrows) return;
  const unsigned nsm = s_total;
  const int e = shift + t;
  T acc = sr[e];
#pragma unroll
  for (int q = 0; q < kSlots; ++q) {
    if (q == kCentre) continue;
    const unsigned idx = (unsigned)(sc[q * rpad + e] + sdelta[q]);
    const T xv = idx < nsm ? sx[idx] : T(0);
    acc = fma(-sv[q * rpad + e], xv, acc);
  }
  x[row0 + t] = acc / sv[kCentre * rpad + e];
}

// Threads per CTA of the latency variant; measured on GB300 at 128^3, the
// FP32 solve took 106.6 / 106.1 / 106.0 / 105.0 / 109.0 ms with 32 / 64 / 128
// / 256 / 512, while the FP64 solve was 3 % slower with 256 than with 64.
template <typename T>
__host__ __device__ constexpr int small_threads() {
  return sizeof(T) == 4 ? 256 : 64;
}

// Latency variant, for coarse levels (matrix resident in L2, at most a few
// tens of thousands of rows per phase): one row per thread, small_threads<T>()
// per CTA, and each thread loads its row's 27 indices and values *before* the
// programmatic wait -- the matrix does not depend on earlier kernels -- so that
// latency overlaps the previous phase; after the wait it issues all the
// gathers of x at once.  Same slot order and arithmetic as gs_phase_kernel.
// early != 0: the next kernel may launch as soon as this one starts (the
// small phases of levels 2-3; without it the 128^3 solve took 145.8 instead
// of 102.9 ms); 0: only as this one's blocks exit (the 32768-row level-1
// phases: 102.9 -> 102.3 ms, while an early trigger there made it 105.6 ms).
// MODE (MatLoad): kMatCached, or kMatResident for the small levels whose
// matrix is kept in L2 evict-last.  MC as in gs_phase_kernel: -1 all slots,
// c the first forward sweep's colour c (slots with a later neighbour colour
// are neither loaded nor gathered).
template <typename T, int MODE, int MC>
__global__ void __launch_bounds__(small_threads<T>())
gs_phase_small_kernel(const T* __restrict__ vals, const int* __restrict__ cols, long long ns,
                      const T* __restrict__ r, T* x, long long row0, long long nrows,
                      long long valid_end, int early) {
  constexpr unsigned kMask = MC < 0 ? (1u << kSlots) - 1u : gs_slot_mask(MC, true);
  if (early) pdl_trigger();
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const bool live = t < nrows;
  const long long row = row0 + (live ? t : 0);
  int col[kSlots];
  T a[kSlots];
#pragma unroll
  for (int s = 0; s < kSlots; ++s) {
    const bool use = live && ((kMask >> s) & 1u);
    col[s] = use ? ld_mat<MODE>(cols + s * ns + row) : 0;
    a[s] = use ? ld_mat<MODE>(vals + s * ns + row) : T(1);
  }
  pdl_wait();
  if (!live) return;
  T xv[kSlots];
#pragma unroll
  for (int s = 0; s < kSlots; ++s)
    xv[s] = (s != kCentre && ((kMask >> s) & 1u) && col[s] < valid_end) ? ld_dep(x + col[s])
                                                                        : T(0);
  T acc = ld_dep(r + row);
#pragma unroll
  for (int s = 0; s < kSlots; ++s)
    if (s != kCentre && ((kMask >> s) & 1u)) acc = fma(-a[s], xv[s], acc);
  x[row] = acc / a[kCentre];
}

// The latency-variant instantiation of a phase of colour c.
template <typename T>
using GsSmallFn = void (*)(const T*, const int*, long long, const T*, T*, long long, long long,
                           long long, int);
template <typename T, int MODE>
static GsSmallFn<T> gs_small_fn_mode(int c, bool from_zero) {
  if (!from_zero) return gs_phase_small_kernel<T, MODE, -1>;
  switch (c) {
    case 0: return gs_phase_small_kernel<T, MODE, 0>;
    case 1: return gs_phase_small_kernel<T, MODE, 1>;
    case 2: return gs_phase_small_kernel<T, MODE, 2>;
    case 3: return gs_phase_small_kernel<T, MODE, 3>;
    case 4: return gs_phase_small_kernel<T, MODE, 4>;
    case 5: return gs_phase_small_kernel<T, MODE, 5>;
    case 6: return gs_phase_small_kernel<T, MODE, 6>;
    default: return gs_phase_small_kernel<T, MODE, 7>;
  }
}
template <typename T>
static GsSmallFn<T> gs_small_fn(int mode, int c, bool from_zero) {
  return mode == kMatResident ? gs_small_fn_mode<T, kMatResident>(c, from_zero)
                              : gs_small_fn_mode<T, kMatCached>(c, from_zero);
}

// ---------------------------------------------- pipelined symmetric sweep
// One kernel runs all colour phases of a symmetric sweep (Sec. 3.2.1) on a
// level whose matrix streams from memory.  The phases' rows are cut into
// tiles of kPipeTileRows rows, handed out in phase order by an atomic queue.
// A tile of phase p may start once the tiles of phase p-1 that cover the grid
// planes K-1 .. K+1 of its own rows (k = 2K + parity: every neighbour of a
// point of plane K lies in planes K-1..K+1 of any colour block) have
// finished.  That covers the values it reads and the readers of the values it
// overwrites, in phase p-1 directly and, because each of those tiles waited
// for its own window, in every earlier phase.  Waits are bounded: a wait that
// runs out sets the error and abort words, and every tile still queued is
// then skipped (the sweep's values are garbage; the solve reports a timeout).
// The queue is deterministic in what each row computes: every row sees the
// same neighbour values as in the phase-by-phase sweep, so results are equal
// bit for bit.  Gathers go through L2 (other CTAs of this kernel write z).
struct PipePhase {
  long long row0;        // first storage row of the colour block
  long long nrows;       // rows of the block (padded)
  long long valid_end;   // gathers at or above this row read zero (from-zero sweep)
  long long cnt;         // grid points of the block (planes of cdx*cdy points)
  long long plane;       // cdx * cdy of this block
  unsigned mask;         // slots read (masked first sweep)
  int masked;            // 1: first forward sweep from z = 0
  int tile0;             // first queue index of the phase
};
struct PipePlan {
  int nphases;
  int total_tiles;
  int tile_stride;       // flag row length (tiles of the largest block)
  PipePhase ph[kMaxPipePhases];
};

constexpr unsigned kPipeWaitPolls = 1u << 21;   // about 0.2-0.4 s of 100 ns naps

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// One row of a colour phase, arithmetic as gs_phase_kernel; gathers via L2.
template <typename T, bool STREAM, bool MASKED>
__device__ __forceinline__ void pipe_row(const T* __restrict__ vals, const int* __restrict__ cols,
                                         long long ns, const T* __restrict__ r, T* z,
                                         long long row, long long valid_end, unsigned mask) {
  T acc = ld_dep(r + row);
#pragma unroll
  for (int s = 0; s < kSlots; ++s) {
    if (s == kCentre) continue;
    if (MASKED) {
      const bool use = (mask >> s) & 1u;
      T a = T(0);
      int c = 0;
      if (use) {
        a = ld_matrix<STREAM>(vals + s * ns + row);
        c = ld_matrix<STREAM>(cols + s * ns + row);
      }
      const T xv = (use && c < valid_end) ? __ldcg(z + c) : T(0);
      acc = fma(-a, xv, acc);
    } else {
      const T a = ld_matrix<STREAM>(vals + s * ns + row);
      const int c = ld_matrix<STREAM>(cols + s * ns + row);
      const T xv = (c < valid_end) ? __ldcg(z + c) : T(0);
      acc = fma(-a, xv, acc);
    }
  }
  const T diag = ld_matrix<STREAM>(vals + kCentre * ns + row);
  z[row] = acc / diag;
}

template <typename T, bool STREAM>
__global__ void __launch_bounds__(kPipeTileRows, 6)
gs_pipeline_kernel(const T* __restrict__ vals, const int* __restrict__ cols, long long ns,
                   const T* __restrict__ r, T* z, const __grid_constant__ PipePlan plan,
                   int* flags, unsigned* sync, unsigned* err) {
  __shared__ int s_tile;
  __shared__ int s_abort;
  pdl_trigger();
  pdl_wait();
  const int done_mark = (int)*(volatile unsigned*)(sync + kPipeEpoch) + 1;
  for (;;) {
    if (threadIdx.x == 0) {
      s_tile = (int)atomicAdd(sync + kPipeQueue, 1u);
      s_abort = (int)*(volatile unsigned*)(sync + kPipeAbort);
    }
    __syncthreads();
    const int tile = s_tile;
    if (tile >= plan.total_tiles || s_abort) break;
    int p = 0;
    while (p + 1 < plan.nphases && tile >= plan.ph[p + 1].tile0) ++p;
    const PipePhase& ph = plan.ph[p];
    const int t = tile - ph.tile0;
    const long long r0 = (long long)t * kPipeTileRows;
    if (p > 0 && threadIdx.x < 32) {
      // window of phase p-1: planes K0-1 .. K1+1 of its block
      const PipePhase& pp = plan.ph[p - 1];
      const long long P1 = min(ph.cnt, r0 + kPipeTileRows);
      if (r0 < P1) {
        const long long K0 = r0 / ph.plane, K1 = (P1 - 1) / ph.plane;
        const long long lo = max(0LL, (K0 - 1) * pp.plane);
        const long long hi = min(pp.nrows, (K1 + 2) * pp.plane);
        const int tlo = (int)(lo / kPipeTileRows);
        const int thi = (int)((hi + kPipeTileRows - 1) / kPipeTileRows);
        const int* f = flags + (long long)(p - 1) * plan.tile_stride;
        bool ok = false;
        for (unsigned it = 0; it < kPipeWaitPolls; ++it) {
          bool mine = true;
          for (int q = tlo + (int)threadIdx.x; q < thi; q += 32)
            mine = mine && ld_acquire(f + q) == done_mark;
          if (__all_sync(0xffffffffu, mine)) {
            ok = true;
            break;
          }
          if (*(volatile unsigned*)(sync + kPipeAbort)) break;
          __nanosleep(100);
        }
        if (!ok && threadIdx.x == 0) {
          if (!*(volatile unsigned*)(sync + kPipeAbort)) atomicExch(err, 1u);
          atomicExch(sync + kPipeAbort, 1u);
          s_abort = 1;
        }
        __threadfence();
      }
    }
    __syncthreads();
    if (s_abort) break;
    const long long lr = r0 + threadIdx.x;
    if (lr < ph.nrows) {
      if (ph.masked)
        pipe_row<T, STREAM, true>(vals, cols, ns, r, z, ph.row0 + lr, ph.valid_end, ph.mask);
      else
        pipe_row<T, STREAM, false>(vals, cols, ns, r, z, ph.row0 + lr, ph.valid_end, ph.mask);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      st_release(flags + (long long)p * plan.tile_stride + t, done_mark);
    }
  }
  // the last CTA out resets the queue and moves to the next epoch
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(sync + kPipeFinish, 1u) == gridDim.x - 1) {
      sync[kPipeQueue] = 0u;
      sync[kPipeFinish] = 0u;
      sync[kPipeAbort] = 0u;
      atomicAdd(sync + kPipeEpoch, 1u);
      __threadfence();
    }
  }
}

// Fused residual + injection restriction (Sec. 3.2.4, last equation):
// rc_I = r_{f_c(I)} - sum_j A_{f_c(I) j} z_j for every coarse point I.  The
// coarse-coincident fine points are exactly fine colour block 7, stored in the
// same lexicographic order as the coarse grid, so threads walk that block
// contiguously and scatter into the coarse colour blocks.
//
// zc0 (optional): the coarse level's first forward sweep from zero starts
// with colour 0, whose rows have no neighbour of a lower colour, so that
// phase is z_I = rc_I / a_II; with zc0 set it is done here, for the coarse
// points of colour 0, and the sweep skips the phase (same values).
// 32 registers (8 CTAs per SM, a 128^3 level-0 restriction is one wave):
// measured 0.15 % faster 128^3 solves than the 34-register build.
template <typename T, int MODE>
__global__ void __launch_bounds__(256, 8)
restrict_kernel(const __grid_constant__ Geom gf, const __grid_constant__ Geom gc,
                const T* __restrict__ vals, const int* __restrict__ cols,
                const T* __restrict__ r, const T* __restrict__ z, T* __restrict__ rc,
                T* __restrict__ zc0, const T* __restrict__ cdiag) {
  pdl_trigger();
  const int cx = gf.cdx[kCoarseColour], cy = gf.cdy[kCoarseColour];
  const long long cnt = (long long)cx * cy * gf.cdz[kCoarseColour];
  const long long ns = gf.n_store;
  const long long p0 = blockIdx.x * (long long)blockDim.x;
  pdl_wait();
  const long long p = p0 + threadIdx.x;
  if (p >= cnt) return;
  const long long row = gf.off[kCoarseColour] + p;
  T acc = ld_dep(r + row);
#pragma unroll
  for (int s = 0; s < kSlots; ++s) {
    const T a = ld_mat<MODE>(vals + s * ns + row);
    const int c = ld_mat<MODE>(cols + s * ns + row);
    acc = fma(-a, ld_dep(z + c), acc);
  }
  const int I = (int)(p % cx);
  const int J = (int)((p / cx) % cy);
  const int K = (int)(p / ((long long)cx * cy));
  const long long R = store_index(gc, I, J, K);
  rc[R] = acc;
  if (zc0 && colour_of(I, J, K) == 0) zc0[R] = acc / cdiag[R];
}

// Prolongation P = R^T and correction (Fig. 1, eq. (3) transposed):
// z_{f_c(I)} += zc_I.
template <typename T>
__global__ void __launch_bounds__(256)
prolong_kernel(const __grid_constant__ Geom gf, const __grid_constant__ Geom gc,
               const T* __restrict__ zc, T* __restrict__ z) {
  pdl_trigger();
  pdl_wait();
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int cx = gf.cdx[kCoarseColour], cy = gf.cdy[kCoarseColour];
  const long long cnt = (long long)cx * cy * gf.cdz[kCoarseColour];
  if (p >= cnt) return;
  const int I = (int)(p % cx);
  const int J = (int)((p / cx) % cy);
  const int K = (int)(p / ((long long)cx * cy));
  const long long row = gf.off[kCoarseColour] + p;
  z[row] += ld_dep(zc + store_index(gc, I, J, K));
}

// ----------------------------------------------------------------- launchers
constexpr int kThreads = 256;

// Largest colour slice (values + indices) a streamed level's phase leaves in
// L2 for a later phase (symgs).
constexpr long long kKeepSliceBytes = 96LL << 20;

// MatLoad of a level (by its FP32 ELL slot bytes).
static int mat_mode(const Level& L) {
  const long long b = L.g.n_store * 27LL * 8;
  return b > kStreamMatrixBytes ? kMatStream : b > kResidentMatrixBytes ? kMatCached
                                                                        : kMatResident;
}

template <typename T>
static auto restrict_fn(const Level& L) -> decltype(&restrict_kernel<T, kMatStream>) {
  switch (mat_mode(L)) {
    case kMatStream: return restrict_kernel<T, kMatStream>;
    case kMatCached: return restrict_kernel<T, kMatCached>;
    default: return restrict_kernel<T, kMatResident>;
  }
}

// Algorithmic DRAM bytes per row (ELL with 27 padded slots, int32 indices;
// every vector entry read or written once).  sv / sx: value / vector bytes.
static double bytes_spmv_row(double sv, double sx) { return 27.0 * (sv + 4.0) + 2.0 * sx; }
// GS phase, per row reading k off-diagonal slots: k + 1 values, k indices
// (the diagonal's is implied), r_i, the new x_i, and x gathered once (in
// proportion to the slots read).
static double bytes_restrict_row(double sv, double sx) { return 27.0 * (sv + 4.0) + 3.0 * sx; }

template <typename T>
static int spmv_t(hpg_problem* h, int level, const T* x, T* y, cudaStream_t s) {
  const Level& L = h->lev[level];
  const long long ns = L.g.n_store;
  const T* vals = Prec<T>::vals(L);
  return launch(h, K_SPMV, level, Prec<T>::idx == 0 ? HPG_FP64 : HPG_FP32,
                L.n * bytes_spmv_row(sizeof(T), sizeof(T)), s, "spmv_kernel", [&] {
                  return kl(h, spmv_kernel<T>, grid_for(ns, kThreads), kThreads, s, vals, L.cols,
                            ns, x, y);
                });
}

int launch_spmv(hpg_problem* h, int level, hpg_prec prec, const void* x, void* y,
                cudaStream_t s) {
  if (prec == HPG_FP64) return spmv_t<double>(h, level, (const double*)x, (double*)y, s);
  return spmv_t<float>(h, level, (const float*)x, (float*)y, s);
}

int launch_residual64(hpg_problem* h, const double* b, const double* x, double* r,
                      cudaStream_t s) {
  const Level& L = h->lev[0];
  const long long ns = L.g.n_store;
  return launch(h, K_RESIDUAL, 0, HPG_FP64, L.n * (27.0 * 12.0 + 3.0 * 8.0), s,
                "residual64_kernel", [&] {
                  return kl(h, residual64_kernel, grid_for(ns, kThreads), kThreads, s, L.v64,
                            L.cols, ns, b, x, r);
                });
}

// State of the sweeps on one level: the colour of the most recent phase when
// nothing else has touched the level's solution since.  A phase repeating
// that colour would recompute identical values from identical inputs, so it
// is skipped (it happens at the forward/backward turn and between sweeps).
struct SweepState {
  int last = -1;
};

// Dynamic shared memory of a TMA-tiled phase of colour c with L lines per
// CTA: the row slices (27 values, 27 index slots, r) and every z run the tile
// may copy, each rounded out to 16-byte boundaries.
template <typename T>
static size_t halo_smem_bytes(const Geom& g, int c, int L) {
  const size_t rpad = (size_t)halo_rpad(L * g.cdx[c], halo_align<T>());
  size_t bytes = rpad * (kSlots * sizeof(T) + kSlots * 4 + sizeof(T));
  size_t elems = 0;
  for (int c2 = 0; c2 < kColours; ++c2) {
    if (c2 == c) continue;
    const int diff = c ^ c2;
    const int planes = (diff & 4) ? 2 : 1;
    const int lines = L + ((diff & 2) ? 1 : 0);
    elems += (size_t)planes * ((size_t)lines * g.cdx[c2] + 2 * halo_align<T>());
  }
  return bytes + elems * sizeof(T);
}

// Launches the TMA-tiled phase when it applies (option set, FP32, whole lines
// fit a CTA, r and z 16-byte aligned); returns false to use gs_phase_kernel.
template <typename T, bool STREAM>
static bool launch_gs_halo(hpg_problem* h, const Level& L, const T* r, T* z, int c,
                           cudaStream_t s, cudaError_t* e) {
  if constexpr (sizeof(T) != 4) {
    return false;
  } else {
  if (!h->gs_halo || (((uintptr_t)z | (uintptr_t)r) & 15u) != 0) return false;
  const int lines = halo_lines(L.g.cdx[c]);
  if (lines < 1 || L.cnt[c] == 0) return false;
  const size_t smem = halo_smem_bytes<T>(L.g, c, lines);
  if (smem > (160u << 10)) return false;
  if (smem > (48u << 10) &&
      cudaFuncSetAttribute(gs_phase_halo_kernel<T, STREAM>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, 160 << 10) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const int threads = (lines * L.g.cdx[c] + 31) / 32 * 32;
  const int grid = L.g.cdz[c] * ((L.g.cdy[c] + lines - 1) / lines);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  *e = cudaLaunchKernelEx(&cfg, gs_phase_halo_kernel<T, STREAM>, Prec<T>::vals(L),
                          (const int*)L.cols, L.g.n_store, r, z, L.g, c, lines, h->pipe_err);
  return true;
  }
}

template <typename T>
static int gs_phase(hpg_problem* h, int level, const T* r, T* z, int c, bool from_zero,
                    SweepState& st, cudaStream_t s, bool keep = false) {
  if (st.last == c) return HPG_OK;
  const Level& L = h->lev[level];
  const long long row0 = L.g.off[c];
  const long long nrows = L.g.off[c + 1] - row0;
  st.last = c;
  if (nrows == 0) return HPG_OK;
  const long long valid_end = from_zero ? row0 : L.g.n_store;
  const T* vals = Prec<T>::vals(L);
  const int nslots = __builtin_popcount(gs_slot_mask(c, from_zero)) - 1;   // off-diagonal
  const double row_bytes =
      (nslots + 1.0) * sizeof(T) + nslots * 4.0 + (2.0 + nslots / 26.0) * sizeof(T);
  return launch(h, K_GS, level, Prec<T>::idx == 0 ? HPG_FP64 : HPG_FP32, L.cnt[c] * row_bytes, s,
                "gs_phase_kernel", [&] {
                  if (L.g.n_store * 27LL * 8 > kStreamMatrixBytes) {
                    // launched programmatically after a kernel of the chain, but the
                    // phase never triggers early and waits before its first load
                    // (see gs_phase_kernel): the next phase's launch is set up while
                    // this one drains; measured 103.6 -> 102.9 ms at 128^3
                    if (((uintptr_t)r | (uintptr_t)z) & 15u)   // see gs_phase_kernel
                      return kl(h, gs_small_fn<T>(kMatCached, c, from_zero),
                                grid_for(nrows, small_threads<T>()), small_threads<T>(), s,
                                vals, L.cols, L.g.n_store, r, z, row0, nrows, valid_end, 0);
                    cudaError_t he = cudaSuccess;
                    if (!from_zero &&
                        (keep ? launch_gs_halo<T, false>(h, L, r, z, c, s, &he)
                              : launch_gs_halo<T, true>(h, L, r, z, c, s, &he)))
                      return he;
                    if (keep)   // slice read again soon after: leave it in L2
                      return kl(h, gs_phase_fn<T, false>(c, from_zero),
                                grid_for(nrows / PhaseRows<T>::R, kThreads), kThreads, s,
                                vals, L.cols, L.g.n_store, r, z, row0, nrows, valid_end);
                    return kl(h, gs_phase_fn<T, true>(c, from_zero),
                              grid_for(nrows / PhaseRows<T>::R, kThreads), kThreads, s, vals,
                              L.cols, L.g.n_store, r, z, row0, nrows, valid_end);
                  }
                  // measured on GB300: programmatic overlap helps the smallest
                  // phases and slows phases of tens of thousands of rows (with
                  // the 32768-row level-1 phases overlapped too, the 128^3
                  // solve took 110.3 ms instead of 107.4)
                  const int early = nrows > h->pdl_rows ? 0 : 1;
                  return kl(h, gs_small_fn<T>(mat_mode(L), c, from_zero),
                            grid_for(nrows, small_threads<T>()), small_threads<T>(), s, vals,
                            L.cols, L.g.n_store, r, z, row0, nrows, valid_end, early);
                });
}


// Resident CTAs of the pipelined sweep kernel (queried once per precision).
template <typename T>
static int pipeline_grid(hpg_problem* h) {
  static int per_sm = 0;
  if (per_sm == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gs_pipeline_kernel<T, true>,
                                                      kPipeTileRows, 0) != cudaSuccess ||
        per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
  }
  return per_sm * h->num_sms;
}

// One symmetric sweep as one pipelined kernel (levels with completion
// flags): the phases the phase-by-phase sweep would launch, in its order and
// with its skipping of a repeated colour.
template <typename T>
static int symgs_pipelined(hpg_problem* h, int level, const T* r, T* z, bool from_zero,
                           SweepState& st, cudaStream_t s) {
  const Level& L = h->lev[level];
  PipePlan plan;
  memset(&plan, 0, sizeof(plan));
  plan.tile_stride = L.pipe_tiles;
  double bytes = 0.0;
  int tiles = 0;
  auto add = [&](int c, bool fz) {
    if (st.last == c) return;
    st.last = c;
    const long long nrows = L.g.off[c + 1] - L.g.off[c];
    if (nrows == 0) return;
    PipePhase& ph = plan.ph[plan.nphases++];
    ph.row0 = L.g.off[c];
    ph.nrows = nrows;
    ph.valid_end = fz ? ph.row0 : L.g.n_store;
    ph.plane = (long long)L.g.cdx[c] * L.g.cdy[c];
    ph.cnt = ph.plane * L.g.cdz[c];
    ph.mask = gs_slot_mask(c, fz);
    ph.masked = fz ? 1 : 0;
    ph.tile0 = tiles;
    tiles += (int)((nrows + kPipeTileRows - 1) / kPipeTileRows);
    const int nslots = __builtin_popcount(ph.mask) - 1;
    bytes += L.cnt[c] * ((nslots + 1.0) * sizeof(T) + nslots * 4.0 +
                         (2.0 + nslots / 26.0) * sizeof(T));
  };
  for (int c = 0; c < kColours; ++c) add(c, from_zero);
  for (int c = kColours - 1; c >= 0; --c) add(c, false);
  plan.total_tiles = tiles;
  if (tiles == 0) return HPG_OK;
  const int grid = std::min(pipeline_grid<T>(h), tiles);
  return launch(h, K_GS, level, Prec<T>::idx == 0 ? HPG_FP64 : HPG_FP32, bytes, s,
                "gs_pipeline_kernel", [&] {
                  h->pdl_next = false;
                  const bool stream = L.g.n_store * 27LL * 8 > kStreamMatrixBytes;
                  return kl(h, stream ? gs_pipeline_kernel<T, true> : gs_pipeline_kernel<T, false>,
                            grid, kPipeTileRows, s, Prec<T>::vals(L), L.cols, L.g.n_store, r, z,
                            plan, L.pipe_flags, L.pipe_sync, h->pipe_err);
                });
}

// One symmetric Gauss-Seidel sweep (eqs. (1)-(2)): colours 0..7 then 7..0.
template <typename T>
static int symgs(hpg_problem* h, int level, const T* r, T* z, bool from_zero, SweepState& st,
                 cudaStream_t s) {
  const bool streamed_level = h->lev[level].g.n_store * 27LL * 8 > kStreamMatrixBytes;
  const bool pipe = h->gs_pipeline == 3 ||
                    (streamed_level && (h->gs_pipeline == 2 ||
                                        (h->gs_pipeline == 1 && sizeof(T) == 8)));
  if (pipe && h->lev[level].pipe_flags && h->pipe_err)
    return symgs_pipelined<T>(h, level, r, z, from_zero, st, s);
  int rc;
  // Where a colour's slice of the matrix fits in L2 with room to spare:
  // the slice of colour kColours - 2 is read again right after the turning
  // colour, so its forward phase leaves it in L2 (the others stream
  // evict-first); measured 1.2 % faster solves at 128^3 FP32.  The last phase
  // (colour 0) leaves its slice in L2 too: after the post-smoothing, the
  // Krylov SpMV reads the matrix from the colour-0 block on; 0.3 % faster.
  const Level& L = h->lev[level];
  const auto fits = [&](int c) {
    return (double)(L.g.off[c + 1] - L.g.off[c]) * kSlots * (sizeof(T) + 4.0) <=
           (double)kKeepSliceBytes;
  };
  for (int c = 0; c < kColours; ++c)
    if ((rc = gs_phase<T>(h, level, r, z, c, from_zero, st, s, c == kColours - 2 && fits(c))))
      return rc;
  for (int c = kColours - 1; c >= 0; --c)
    if ((rc = gs_phase<T>(h, level, r, z, c, false, st, s, c == 0 && fits(c)))) return rc;
  return HPG_OK;
}

// ------------------------------------------- coarsest level in one CTA
// The coarsest level's symmetric sweep from z = 0 (Fig. 1: one sweep there)
// in a single CTA, when every colour block has at most kCtaSweepRows rows:
// z lives in shared memory, a __syncthreads() separates the colour phases
// (instead of a kernel boundary, ~1.3 us each when launched), and each
// thread loads the next phase's matrix row and r_i into registers while the
// current phase computes, so the L2 latency of the matrix is off the chain.
// Phases, slot sets, summation order and division are those of the launched
// phases (gs_phase_small_kernel), so z is equal bit for bit.
constexpr int kCtaSweepRows = 512;
struct CtaSweepPhase {
  int row0, nrows, valid_end;
  unsigned mask;
};
struct CtaSweepPlan {
  int nphases;
  int c0_rows;   // rows [0, c0_rows) of z already hold colour 0's first phase
  CtaSweepPhase ph[kMaxPipePhases];
};

template <typename T, int MODE>
__global__ void __launch_bounds__(kCtaSweepRows, 1)
coarse_sweep_cta_kernel(const T* __restrict__ vals, const int* __restrict__ cols, int ns,
                        const T* __restrict__ r, T* __restrict__ z,
                        const __grid_constant__ CtaSweepPlan plan) {
  extern __shared__ __align__(16) unsigned char cta_smem[];
  T* sz = reinterpret_cast<T*>(cta_smem);
  const int t = threadIdx.x;
  pdl_trigger();
  int col[kSlots];
  T a[kSlots];
  T rr = T(0);
  // phase p's row of this thread: matrix and r (no earlier kernel writes
  // the matrix, so phase 0's loads go out before the programmatic wait)
  auto load = [&](int p, bool rhs) {
    const CtaSweepPhase& ph = plan.ph[p];
    const bool live = t < ph.nrows;
    const int row = ph.row0 + (live ? t : 0);
#pragma unroll
    for (int q = 0; q < kSlots; ++q) {
      const bool use = live && ((ph.mask >> q) & 1u);
      col[q] = use ? ld_mat<MODE>(cols + (long long)q * ns + row) : 0;
      a[q] = use ? ld_mat<MODE>(vals + (long long)q * ns + row) : T(1);
    }
    if (rhs) rr = live ? ld_dep(r + row) : T(0);
  };
  load(0, false);
  pdl_wait();
  if (t < plan.ph[0].nrows) rr = ld_dep(r + plan.ph[0].row0 + t);
  for (int i = t; i < ns; i += blockDim.x) sz[i] = i < plan.c0_rows ? ld_dep(z + i) : T(0);
  __syncthreads();
  for (int p = 0; p < plan.nphases; ++p) {
    const CtaSweepPhase& ph = plan.ph[p];
    T acc = rr;
    T diag = a[kCentre];
    const bool live = t < ph.nrows;
    T xv[kSlots];
#pragma unroll
    for (int q = 0; q < kSlots; ++q)
      xv[q] = (q != kCentre && ((ph.mask >> q) & 1u) && col[q] < ph.valid_end) ? sz[col[q]]
                                                                                : T(0);
#pragma unroll
    for (int q = 0; q < kSlots; ++q)
      if (q != kCentre && ((ph.mask >> q) & 1u)) acc = fma(-a[q], xv[q], acc);
    if (p + 1 < plan.nphases) load(p + 1, true);
    if (live) sz[ph.row0 + t] = acc / diag;
    __syncthreads();
  }
  for (int i = t; i < ns; i += blockDim.x) z[i] = sz[i];
}

// Runs the coarsest level's sweep from zero in one CTA if it fits; returns
// HPG_ERR_UNSUPPORTED otherwise (the caller launches the phases).
template <typename T>
static int coarsest_sweep_cta(hpg_problem* h, int level, const T* r, T* z, bool c0_done,
                              cudaStream_t s) {
  const Level& L = h->lev[level];
  if (!h->coarse_cta || h->gs_pipeline == 3 ||
      L.g.n_store * (long long)sizeof(T) > (64LL << 10))
    return HPG_ERR_UNSUPPORTED;
  for (int c = 0; c < kColours; ++c)
    if (L.g.off[c + 1] - L.g.off[c] > kCtaSweepRows) return HPG_ERR_UNSUPPORTED;
  CtaSweepPlan plan;
  memset(&plan, 0, sizeof(plan));
  plan.c0_rows = c0_done ? (int)L.g.off[1] : 0;
  int last = c0_done ? 0 : -1;
  double bytes = 0.0;
  auto add = [&](int c, bool fz) {
    if (last == c) return;
    last = c;
    const int nrows = (int)(L.g.off[c + 1] - L.g.off[c]);
    if (nrows == 0) return;
    CtaSweepPhase& ph = plan.ph[plan.nphases++];
    ph.row0 = (int)L.g.off[c];
    ph.nrows = nrows;
    ph.valid_end = fz ? (int)L.g.off[c] : (int)L.g.n_store;
    ph.mask = gs_slot_mask(c, fz);
    const int nslots = __builtin_popcount(ph.mask) - 1;
    bytes += L.cnt[c] * ((nslots + 1.0) * sizeof(T) + nslots * 4.0 +
                         (2.0 + nslots / 26.0) * sizeof(T));
  };
  for (int c = 0; c < kColours; ++c) add(c, true);
  for (int c = kColours - 1; c >= 0; --c) add(c, false);
  if (plan.nphases == 0) return HPG_ERR_UNSUPPORTED;
  const size_t smem = sizeof(T) * (size_t)L.g.n_store;
  const int mode = mat_mode(L);
  auto kern = mode == kMatResident ? coarse_sweep_cta_kernel<T, kMatResident>
                                   : coarse_sweep_cta_kernel<T, kMatCached>;
  if (smem > (48u << 10) &&
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 << 10) !=
          cudaSuccess) {
    cudaGetLastError();
    return HPG_ERR_UNSUPPORTED;
  }
  return launch(h, K_GS, level, Prec<T>::idx == 0 ? HPG_FP64 : HPG_FP32, bytes, s,
                "coarse_sweep_cta_kernel", [&] {
                  cudaLaunchConfig_t cfg = {};
                  cfg.gridDim = dim3(1u);
                  cfg.blockDim = dim3((unsigned)kCtaSweepRows);
                  cfg.dynamicSmemBytes = smem;
                  cfg.stream = s;
                  cudaLaunchAttribute attr[1];
                  if (h->pdl_enabled && h->pdl_next && !h->profiling) {
                    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
                    attr[0].val.programmaticStreamSerializationAllowed = 1;
                    cfg.attrs = attr;
                    cfg.numAttrs = 1;
                  }
                  return cudaLaunchKernelEx(&cfg, kern, Prec<T>::vals(L), (const int*)L.cols,
                                            (int)L.g.n_store, r, z, plan);
                });
}

// The coarsest level of a V-cycle: one symmetric sweep from z = 0.
template <typename T>
static int coarsest_sweep(hpg_problem* h, int l, const T* r, T* z, bool c0_done,
                          cudaStream_t s) {
  int rc = coarsest_sweep_cta<T>(h, l, r, z, c0_done, s);
  if (rc != HPG_ERR_UNSUPPORTED) return rc;
  SweepState st;
  if (c0_done) st.last = 0;
  return symgs<T>(h, l, r, z, true, st, s);
}

// Whether the restriction from level l also runs the first phase (colour 0)
// of level l+1's first sweep from zero: true when that sweep goes through the
// launched phases (not the cluster kernel) and starts from zero (the
// coarsest level, or a pre-smoother).
static bool fuse_first_phase(const hpg_problem* h, int l) {
  return !h->coarse_cluster && (l + 1 == h->nlev - 1 || h->pre >= 1);
}

template <typename T>
static int vcycle_t(hpg_problem* h, int l, const T* r, T* z, cudaStream_t s,
                    bool c0_done = false) {
  const Level& L = h->lev[l];
  SweepState st;
  if (c0_done) st.last = 0;   // colour 0 of the first sweep came with the restriction
  int rc = launch_vcycle_cluster(h, l, Prec<T>::idx == 0 ? HPG_FP64 : HPG_FP32, r, z, s);
  if (rc != HPG_ERR_UNSUPPORTED) return rc;   // small level: the rest runs in one cluster
  if (l == h->nlev - 1) return coarsest_sweep<T>(h, l, r, z, c0_done, s);
  if (h->pre == 0) {
    HPG_CK(cudaMemsetAsync(z, 0, sizeof(T) * L.g.n_store, s));
    h->pdl_next = false;
  }
  for (int it = 0; it < h->pre; ++it)
    if ((rc = symgs<T>(h, l, r, z, it == 0, st, s))) return rc;
  const Level& C = h->lev[l + 1];
  T* rc_vec = (T*)C.rhs[Prec<T>::idx];
  T* zc_vec = (T*)C.sol[Prec<T>::idx];
  const bool fuse = fuse_first_phase(h, l);
  const long long cnt = (long long)L.g.cdx[kCoarseColour] * L.g.cdy[kCoarseColour] *
                        L.g.cdz[kCoarseColour];
  const int prec = Prec<T>::idx == 0 ? HPG_FP64 : HPG_FP32;
  const T* vals = Prec<T>::vals(L);
  rc = launch(h, K_RESTRICT, l, prec, cnt * bytes_restrict_row(sizeof(T), sizeof(T)), s,
              "restrict_kernel", [&] {
                return kl(h, restrict_fn<T>(L), grid_for(cnt, kThreads), kThreads, s, L.g,
                          C.g, vals, L.cols, r, z, rc_vec, fuse ? zc_vec : (T*)nullptr,
                          Prec<T>::vals(C) + kCentre * C.g.n_store);
              });
  if (rc) return rc;
  if ((rc = vcycle_t<T>(h, l + 1, rc_vec, zc_vec, s, fuse))) return rc;
  rc = launch(h, K_PROLONG, l, prec, cnt * 3.0 * sizeof(T), s, "prolong_kernel", [&] {
    return kl(h, prolong_kernel<T>, grid_for(cnt, kThreads), kThreads, s, L.g, C.g,
              (const T*)zc_vec, z);
  });
  if (rc) return rc;
  st.last = -1;
  for (int it = 0; it < h->post; ++it)
    if ((rc = symgs<T>(h, l, r, z, false, st, s))) return rc;
  return HPG_OK;
}

// `sweeps` symmetric sweeps on one level; from_zero: z enters as 0 (its
// contents are never read).
template <typename T>
static int smooth_t(hpg_problem* h, int level, const T* r, T* z, int sweeps, bool from_zero,
                    cudaStream_t s) {
  const Level& L = h->lev[level];
  if (sweeps == 0) {
    if (from_zero) {
      HPG_CK(cudaMemsetAsync(z, 0, sizeof(T) * L.g.n_store, s));
      h->pdl_next = false;
    }
    return HPG_OK;
  }
  SweepState st;
  int rc;
  for (int it = 0; it < sweeps; ++it)
    if ((rc = symgs<T>(h, level, r, z, from_zero && it == 0, st, s))) return rc;
  return HPG_OK;
}

int run_vcycle(hpg_problem* h, int level, hpg_prec prec, const void* r, void* z,
               cudaStream_t s, bool c0_done) {
  if (prec == HPG_FP64)
    return vcycle_t<double>(h, level, (const double*)r, (double*)z, s, c0_done);
  return vcycle_t<float>(h, level, (const float*)r, (float*)z, s, c0_done);
}

}  // namespace hpg

using namespace hpg;

extern "C" {

HPG_API int hpg_spmv(hpg_problem_t* h, int level, hpg_prec prec, const void* x, void* y,
                     void* stream) {
  if (!h || !x || !y || level < 0 || level >= h->nlev ||
      (prec != HPG_FP64 && prec != HPG_FP32) || x == y) {
    set_error("hpg_spmv: invalid argument (handle, level %d, prec %d, pointers)", level,
              (int)prec);
    return HPG_ERR_INVALID;
  }
  h->pdl_next = false;
  return launch_spmv(h, level, prec, x, y, (cudaStream_t)stream);
}

HPG_API int hpg_mg_vcycle(hpg_problem_t* h, int level, hpg_prec prec, const void* r, void* z,
                          void* stream) {
  if (!h || !r || !z || level < 0 || level >= h->nlev ||
      (prec != HPG_FP64 && prec != HPG_FP32) || r == z) {
    set_error("hpg_mg_vcycle: invalid argument (handle, level %d, prec %d, pointers)", level,
              (int)prec);
    return HPG_ERR_INVALID;
  }
  if (!h->hierarchy) {
    set_error("hpg_mg_vcycle: call hpg_build_mg_hierarchy first");
    return HPG_ERR_STATE;
  }
  h->pdl_next = false;
  return run_vcycle(h, level, prec, r, z, (cudaStream_t)stream);
}

HPG_API int hpg_mg_smooth(hpg_problem_t* h, int level, hpg_prec prec, const void* r, void* z,
                          int sweeps, int z_is_zero, void* stream) {
  if (!h || !r || !z || level < 0 || level >= h->nlev ||
      (prec != HPG_FP64 && prec != HPG_FP32) || r == z || sweeps < 0) {
    set_error("hpg_mg_smooth: invalid argument (handle, level %d, prec %d, sweeps %d, pointers)",
              level, (int)prec, sweeps);
    return HPG_ERR_INVALID;
  }
  if (!h->hierarchy) {
    set_error("hpg_mg_smooth: call hpg_build_mg_hierarchy first");
    return HPG_ERR_STATE;
  }
  h->pdl_next = false;
  const cudaStream_t s = (cudaStream_t)stream;
  if (prec == HPG_FP64)
    return smooth_t<double>(h, level, (const double*)r, (double*)z, sweeps, z_is_zero != 0, s);
  return smooth_t<float>(h, level, (const float*)r, (float*)z, sweeps, z_is_zero != 0, s);
}

}  // extern "C"

// ------------------------------------------------------ allocation-free V-cycle
// hpg_mg_vcycle_noalloc: the same V-cycle as hpg_mg_vcycle, but the coarse
// levels' work vectors (restricted residuals and corrections) live in one
// file-scope device array instead of buffers the handle allocated.  It is for
// callers that must not allocate device memory at the time of the call.
#include <mutex>

namespace hpg {

constexpr size_t kStaticScratchBytes = (size_t)HPG_NOALLOC_SCRATCH_BYTES;

// Shared by every call on a device; every GPU that loads this library holds
// it until the process exits.
static __device__ __align__(256) unsigned char g_vcycle_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
static void* g_scratch_addr[kMaxDevices];
static std::mutex g_scratch_mutex;

// Device address of g_vcycle_scratch on the current device.  In host code the
// array's name is only a stand-in, so the address is looked up once per device
// (with that device current) and cached.
static int scratch_address(void** out) {
  int dev = 0;
  HPG_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("hpg_mg_vcycle_noalloc: device %d out of range", dev);
    return HPG_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_vcycle_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return HPG_OK;
}

// Same schedule as vcycle_t; coarse vectors come from crhs / csol.
template <typename T>
static int vcycle_noalloc_t(hpg_problem* h, int l, const T* r, T* z, T* const* crhs,
                            T* const* csol, cudaStream_t s, bool c0_done = false) {
  const Level& L = h->lev[l];
  SweepState st;
  if (c0_done) st.last = 0;   // colour 0 of the first sweep came with the restriction
  int rc;
  if (l == h->nlev - 1) return coarsest_sweep<T>(h, l, r, z, c0_done, s);
  if (h->pre == 0) {
    HPG_CK(cudaMemsetAsync(z, 0, sizeof(T) * L.g.n_store, s));
    h->pdl_next = false;
  }
  for (int it = 0; it < h->pre; ++it)
    if ((rc = symgs<T>(h, l, r, z, it == 0, st, s))) return rc;
  const Level& C = h->lev[l + 1];
  T* rc_vec = crhs[l + 1];
  T* zc_vec = csol[l + 1];
  const bool fuse = l + 1 == h->nlev - 1 || h->pre >= 1;
  const long long cnt = (long long)L.g.cdx[kCoarseColour] * L.g.cdy[kCoarseColour] *
                        L.g.cdz[kCoarseColour];
  const int prec = Prec<T>::idx == 0 ? HPG_FP64 : HPG_FP32;
  const T* vals = Prec<T>::vals(L);
  rc = launch(h, K_RESTRICT, l, prec, cnt * bytes_restrict_row(sizeof(T), sizeof(T)), s,
              "restrict_kernel", [&] {
                return kl(h, restrict_fn<T>(L), grid_for(cnt, kThreads), kThreads, s, L.g,
                          C.g, vals, L.cols, r, z, rc_vec, fuse ? zc_vec : (T*)nullptr,
                          Prec<T>::vals(C) + kCentre * C.g.n_store);
              });
  if (rc) return rc;
  if ((rc = vcycle_noalloc_t<T>(h, l + 1, rc_vec, zc_vec, crhs, csol, s, fuse))) return rc;
  rc = launch(h, K_PROLONG, l, prec, cnt * 3.0 * sizeof(T), s, "prolong_kernel", [&] {
    return kl(h, prolong_kernel<T>, grid_for(cnt, kThreads), kThreads, s, L.g, C.g,
              (const T*)zc_vec, z);
  });
  if (rc) return rc;
  st.last = -1;
  for (int it = 0; it < h->post; ++it)
    if ((rc = symgs<T>(h, l, r, z, false, st, s))) return rc;
  return HPG_OK;
}

template <typename T>
static int vcycle_noalloc_entry(hpg_problem* h, int level, const T* r, T* z, cudaStream_t s) {
  // carve the coarse vectors of levels level+1 .. nlev-1 out of the array
  size_t need = 0;
  for (int l = level + 1; l < h->nlev; ++l) need += 2 * sizeof(T) * (size_t)h->lev[l].g.n_store;
  if (need > kStaticScratchBytes) {
    set_error("hpg_mg_vcycle_noalloc: the coarse levels need %zu bytes of work space, more "
              "than the %zu-byte static array (use hpg_mg_vcycle)",
              need, kStaticScratchBytes);
    return HPG_ERR_INVALID;
  }
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  T* crhs[kMaxLevels] = {nullptr};
  T* csol[kMaxLevels] = {nullptr};
  size_t off = 0;
  for (int l = level + 1; l < h->nlev; ++l) {
    crhs[l] = reinterpret_cast<T*>(static_cast<unsigned char*>(base) + off);
    off += sizeof(T) * (size_t)h->lev[l].g.n_store;
    csol[l] = reinterpret_cast<T*>(static_cast<unsigned char*>(base) + off);
    off += sizeof(T) * (size_t)h->lev[l].g.n_store;
  }
  // the array keeps the previous call's contents: zero the part this call
  // uses (padding entries of the coarse vectors must read as zero)
  if (need > 0) {
    HPG_CK(cudaMemsetAsync(base, 0, need, s));
  }
  h->pdl_next = false;
  return vcycle_noalloc_t<T>(h, level, r, z, crhs, csol, s);
}

}  // namespace hpg

extern "C" {

HPG_API int hpg_mg_vcycle_noalloc(hpg_problem_t* h, int level, hpg_prec prec, const void* r,
                                  void* z, void* stream) {
  if (!h || !r || !z || level < 0 || level >= h->nlev ||
      (prec != HPG_FP64 && prec != HPG_FP32) || r == z) {
    set_error("hpg_mg_vcycle_noalloc: invalid argument (handle, level %d, prec %d, pointers)",
              level, (int)prec);
    return HPG_ERR_INVALID;
  }
  if (!h->hierarchy) {
    set_error("hpg_mg_vcycle_noalloc: call hpg_build_mg_hierarchy first");
    return HPG_ERR_STATE;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == HPG_FP64)
    return vcycle_noalloc_entry<double>(h, level, (const double*)r, (double*)z, s);
  return vcycle_noalloc_entry<float>(h, level, (const float*)r, (float*)z, s);
}

}  // extern "C"
