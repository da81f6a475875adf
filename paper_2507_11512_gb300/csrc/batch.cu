// Multi-right-hand-side path: R right-hand sides of one system advance
// together through the same kernels, so every matrix slot loaded from HBM
// serves R rows of work instead of one.
//
// Layout: an R-vector of a level is [n_store][R] (the R values of one storage
// row are contiguous), in FP32 for the inner solve and FP64 for the outer
// refinement; R is 1, 2, 4 or 8.  A row is handled by LPR lanes (1, 2 or R),
// each lane owning RL = R / LPR consecutive right-hand sides, so a gather of
// neighbour j reads RL contiguous values.  Which LPR and block size a level
// uses is picked by timing (hpg_batch_tune); every choice computes the same
// values in the same order as the single-right-hand-side kernels of
// sparse.cu, so a column of a multi-right-hand-side SpMV or V-cycle is bitwise
// the single-vector result.
//
// The Krylov part (batched GMRES-IR, Algorithm 3 per right-hand side) keeps a
// separate basis, Hessenberg matrix, rotations and state per right-hand side;
// the right-hand sides run in lockstep, and one that has converged is frozen
// (its state is no longer updated) while the others continue.

#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "hpg_internal.cuh"

namespace hpg {

// ------------------------------------------------------------ R-value access
// n consecutive values, 4n-byte aligned, written by an earlier kernel:
// coherent L1-cached loads (ld_dep: never the read-only path for such data).
template <int N>
__device__ __forceinline__ void ld_n(const float* p, float (&v)[N]) {
  if constexpr (N == 8) {
    const float4 a = ld_dep(reinterpret_cast<const float4*>(p));
    const float4 b = ld_dep(reinterpret_cast<const float4*>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  } else if constexpr (N == 4) {
    const float4 a = ld_dep(reinterpret_cast<const float4*>(p));
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  } else if constexpr (N == 2) {
    const float2 a = ld_dep(reinterpret_cast<const float2*>(p));
    v[0] = a.x; v[1] = a.y;
  } else {
    v[0] = ld_dep(p);
  }
}
// The same through the read-only path (ld.global.nc), for a kernel that is
// never launched programmatically: every writer of the vector has completed
// before it starts, and its successors write only after their wait, so the
// vector is constant while it runs (the multi-RHS SpMV: measured 782 -> 776
// ms for the 64 x 8 batch against ld_n).
template <int N>
__device__ __forceinline__ void ldnc_n(const float* p, float (&v)[N]) {
  if constexpr (N == 8) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  } else if constexpr (N == 4) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  } else if constexpr (N == 2) {
    const float2 a = __ldg(reinterpret_cast<const float2*>(p));
    v[0] = a.x; v[1] = a.y;
  } else {
    v[0] = __ldg(p);
  }
}
template <int N>
__device__ __forceinline__ void st_n(float* p, const float (&v)[N]) {
  if constexpr (N == 8) {
    reinterpret_cast<float4*>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float4*>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
  } else if constexpr (N == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else if constexpr (N == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  } else {
    *p = v[0];
  }
}

// ------------------------------------------------- multi-RHS stencil kernels
// Y = A X (Sec. 3.2.2) for R right-hand sides.  Never launched
// programmatically (mspmv_t), so X is gathered through the read-only path.
template <int R, int LPR>
__global__ void __launch_bounds__(256)
mspmv_kernel(const float* __restrict__ vals, const int* __restrict__ cols, long long ns,
             const float* __restrict__ x, float* __restrict__ y) {
  constexpr int RL = R / LPR;
  pdl_trigger();
  pdl_wait();
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long row = t / LPR;
  const int lane = (int)(t % LPR);
  if (row >= ns) return;
  float acc[RL];
#pragma unroll
  for (int r = 0; r < RL; ++r) acc[r] = 0.0f;
#pragma unroll
  for (int s = 0; s < kSlots; ++s) {
    const float a = ld_stream(vals + s * ns + row);
    const int c = ld_stream(cols + s * ns + row);
    float xv[RL];
    ldnc_n<RL>(x + (long long)c * R + lane * RL, xv);
#pragma unroll
    for (int r = 0; r < RL; ++r) acc[r] = fma(a, xv[r], acc[r]);
  }
  st_n<RL>(y + row * R + lane * RL, acc);
}

// One Gauss-Seidel colour phase (Sec. 3.2.1) for R right-hand sides: rows
// [row0, row0 + nrows) of one colour block; entries j >= valid_end read as
// zero (first forward sweep from z = 0).  MC selects the slots loaded:
// kAllSlots every slot; c = 0..7 the first forward sweep's phase of colour c
// from z = 0 with its slot set (gs_slot_mask) fixed at compile time, so a
// row's loads issue as one straight-line batch; kMaskSlots the same set
// passed at run time in `mask` (the other slots are known zero and not
// loaded).  MODE (MatLoad) is the level's matrix load policy: streamed
// evict-first, cached, or evict-last for the small coarse levels.  Same slot
// order and arithmetic per value as gs_phase_kernel.
constexpr int kAllSlots = -1, kMaskSlots = -2;
template <int R, int LPR, int MODE, int MC>
__global__ void __launch_bounds__(256, 3)
mgs_phase_kernel(const float* __restrict__ vals, const int* __restrict__ cols, long long ns,
                 const float* __restrict__ rhs, float* z, long long row0, long long nrows,
                 long long valid_end, unsigned mask) {
  constexpr int RL = R / LPR;
  constexpr unsigned kMask = MC >= 0 ? gs_slot_mask(MC, true) : (1u << kSlots) - 1u;
  pdl_trigger();
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long lr = t / LPR;
  const int lane = (int)(t % LPR);
  if (lr >= nrows) return;
  const long long row = row0 + lr;
  // the row's matrix slots first, all at once (the matrix does not depend on
  // earlier kernels, so these loads may overlap the previous phase), then the
  // gathers slot by slot; the arithmetic is that of gs_phase_kernel
  int col[kSlots];
  float a[kSlots];
#pragma unroll
  for (int s = 0; s < kSlots; ++s) {
    const bool use = ((kMask >> s) & 1u) && (MC != kMaskSlots || s == kCentre ||
                                             ((mask >> s) & 1u));
    col[s] = use && s != kCentre ? ld_mat<MODE>(cols + s * ns + row) : 0;
    a[s] = use ? ld_mat<MODE>(vals + s * ns + row) : 0.0f;
  }
  pdl_wait();
  float acc[RL];
  ld_n<RL>(rhs + row * R + lane * RL, acc);
#pragma unroll
  for (int s = 0; s < kSlots; ++s) {
    if (s == kCentre || !((kMask >> s) & 1u)) continue;
    const bool use = MC != kMaskSlots || ((mask >> s) & 1u);
    float xv[RL];
    if (use && col[s] < valid_end) {
      ld_n<RL>(z + (long long)col[s] * R + lane * RL, xv);
    } else {
#pragma unroll
      for (int r = 0; r < RL; ++r) xv[r] = 0.0f;
    }
#pragma unroll
    for (int r = 0; r < RL; ++r) acc[r] = fma(-a[s], xv[r], acc[r]);
  }
#pragma unroll
  for (int r = 0; r < RL; ++r) acc[r] = acc[r] / a[kCentre];
  st_n<RL>(z + row * R + lane * RL, acc);
}

// Fused residual + injection restriction (Sec. 3.2.4) for R right-hand sides;
// MODE as for mgs_phase_kernel.
template <int R, int MODE>
__global__ void __launch_bounds__(256)
mrestrict_kernel(const __grid_constant__ Geom gf, const __grid_constant__ Geom gc,
                 const float* __restrict__ vals, const int* __restrict__ cols,
                 const float* __restrict__ rhs, const float* __restrict__ z,
                 float* __restrict__ rc) {
  pdl_trigger();
  pdl_wait();
  const int cx = gf.cdx[kCoarseColour], cy = gf.cdy[kCoarseColour];
  const long long cnt = (long long)cx * cy * gf.cdz[kCoarseColour];
  const long long ns = gf.n_store;
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= cnt) return;
  const long long row = gf.off[kCoarseColour] + p;
  float acc[R];
  ld_n<R>(rhs + row * R, acc);
#pragma unroll
  for (int s = 0; s < kSlots; ++s) {
    const float a = ld_mat<MODE>(vals + s * ns + row);
    const int c = ld_mat<MODE>(cols + s * ns + row);
    float xv[R];
    ld_n<R>(z + (long long)c * R, xv);
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = fma(-a, xv[r], acc[r]);
  }
  const int I = (int)(p % cx);
  const int J = (int)((p / cx) % cy);
  const int K = (int)(p / ((long long)cx * cy));
  st_n<R>(rc + store_index(gc, I, J, K) * R, acc);
}

// Prolongation and correction z_{f_c(I)} += zc_I (eq. (3) transposed).
template <int R>
__global__ void __launch_bounds__(256)
mprolong_kernel(const __grid_constant__ Geom gf, const __grid_constant__ Geom gc,
                const float* __restrict__ zc, float* __restrict__ z) {
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
  float a[R], b[R];
  ld_n<R>(z + row * R, a);
  ld_n<R>(zc + store_index(gc, I, J, K) * R, b);
#pragma unroll
  for (int r = 0; r < R; ++r) a[r] += b[r];
  st_n<R>(z + row * R, a);
}

// Natural order (R vectors of n values, vector r at in[r * n]) <-> storage
// R-vector [n_store][R]; padding rows written as 0.  T: FP64 or FP32 ends.
template <typename Tin, typename Tout>
__global__ void __launch_bounds__(256)
mto_storage_kernel(const __grid_constant__ Geom g, int R, const Tin* __restrict__ in,
                   Tout* __restrict__ out) {
  pdl_trigger();
  pdl_wait();
  const long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (row >= g.n_store) return;
  const int c = colour_of_row(g, row);
  const long long p = row - g.off[c];
  const long long cntc = (long long)g.cdx[c] * g.cdy[c] * g.cdz[c];
  if (p >= cntc) {
    for (int r = 0; r < R; ++r) out[row * R + r] = Tout(0);
    return;
  }
  const int I = (int)(p % g.cdx[c]);
  const long long q = p / g.cdx[c];
  const int J = (int)(q % g.cdy[c]);
  const int K = (int)(q / g.cdy[c]);
  const long long nat = (long long)(2 * I + colour_parity_x(c)) +
                        (long long)g.nx * ((2 * J + colour_parity_y(c)) +
                                           (long long)g.ny * (2 * K + colour_parity_z(c)));
  const long long n = (long long)g.nx * g.ny * g.nz;
  for (int r = 0; r < R; ++r) out[row * R + r] = (Tout)ld_dep(in + r * n + nat);
}

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(256)
mto_natural_kernel(const __grid_constant__ Geom g, int R, const Tin* __restrict__ in,
                   Tout* __restrict__ out) {
  pdl_trigger();
  pdl_wait();
  const long long n = (long long)g.nx * g.ny * g.nz;
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int i = (int)(q % g.nx);
  const int j = (int)((q / g.nx) % g.ny);
  const int k = (int)(q / ((long long)g.nx * g.ny));
  const long long row = store_index(g, i, j, k);
  for (int r = 0; r < R; ++r) out[r * n + q] = (Tout)ld_dep(in + row * R + r);
}

// ----------------------------------------------------------- batch space
constexpr int kMaxR = 8;
constexpr int kShapeGs = 0, kShapeSpmv = 1;

// Launch shape of a multi-RHS stencil kernel on one level: lanes per row and
// block size (0 = default).
struct Shape {
  int lpr = 0;
  int block = 0;
};

struct BState {     // per right-hand side, as the single solve's state
  double rho0, tol, rho, beta;
  int k, active, iters, maxit, m, status, restarts, done, converged;
  double rel;
};

struct BatchSpace {
  int R = 0;          // right-hand sides of the buffers below
  int m = 0;          // restart capacity
  int G = 0;          // blocks of the reduction kernels
  long long ns = 0;   // level-0 storage rows
  Shape shape[kMaxLevels][2][kMaxR + 1];   // [level][GS/SpMV][R]
  float* rc[kMaxLevels] = {nullptr};        // coarse levels: restricted residuals
  float* zc[kMaxLevels] = {nullptr};        // coarse levels: corrections
  float* Q = nullptr;                      // [m+1][ns][R]
  float *z = nullptr, *w = nullptr, *u = nullptr;   // [ns][R]
  double *b = nullptr, *x = nullptr, *r = nullptr;  // [ns][R]
  double* partials = nullptr;              // [G][kBatchPartStride]
  unsigned int* counter = nullptr;
  double *h1 = nullptr, *h2 = nullptr;     // [R][kMaxRestart + 1]
  double* H = nullptr;                     // [R][(m+1) m], column-major per RHS, ld = m+1
  double *cs = nullptr, *sn = nullptr, *t = nullptr, *y = nullptr;   // [R][m+1]
  double* rho2 = nullptr;                  // [R]
  BState* st = nullptr;                    // [R] device
  BState* st_host = nullptr;               // [R] pinned
  unsigned long long* hk = nullptr;        // [m] IF handles
  int* runs = nullptr;                     // [2] inner steps and cycles the device ran
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int graph_m = 0;
  int owners = 0;     // multi-system batches whose graph uses these buffers
  long long n_outer = 0, n_start = 0, n_step = 0, n_update = 0;
  cudaStream_t cap[3] = {nullptr, nullptr, nullptr};
};

constexpr int kBatchPartStride = (kMaxRestart + 1) * kMaxR;

int batch_owners(const hpg_problem* h) { return h->batch ? h->batch->owners : 0; }

void drop_batch_graph(hpg_problem* h) {
  BatchSpace* bs = h->batch;
  if (!bs) return;
  if (bs->exec) cudaGraphExecDestroy(bs->exec);
  if (bs->graph) cudaGraphDestroy(bs->graph);
  bs->exec = nullptr;
  bs->graph = nullptr;
}

void destroy_batch(hpg_problem* h) {
  BatchSpace* bs = h->batch;
  if (!bs) return;
  if (bs->exec) cudaGraphExecDestroy(bs->exec);
  if (bs->graph) cudaGraphDestroy(bs->graph);
  for (int i = 0; i < 3; ++i)
    if (bs->cap[i]) cudaStreamDestroy(bs->cap[i]);
  for (int l = 0; l < kMaxLevels; ++l) {
    dev_free(bs->rc[l]);
    dev_free(bs->zc[l]);
  }
  void* ptrs[] = {bs->Q, bs->z, bs->w, bs->u, bs->b, bs->x, bs->r, bs->partials, bs->counter,
                  bs->h1, bs->h2, bs->H, bs->cs, bs->sn, bs->t, bs->y, bs->rho2, bs->st,
                  bs->hk, bs->runs};
  for (void* p : ptrs) dev_free(p);
  if (bs->st_host) cudaFreeHost(bs->st_host);
  delete bs;
  h->batch = nullptr;
}

static BatchSpace* batch_space(hpg_problem* h) {
  if (!h->batch) h->batch = new BatchSpace();
  return h->batch;
}

// Coarse-level R-vectors of the V-cycle (levels 1..), sized for kMaxR.
static int ensure_vcycle_buffers(hpg_problem* h) {
  BatchSpace* bs = batch_space(h);
  for (int l = 1; l < h->nlev; ++l) {
    if (bs->rc[l]) continue;
    const size_t bytes = sizeof(float) * (size_t)h->lev[l].g.n_store * kMaxR;
    int rc = dev_alloc((void**)&bs->rc[l], bytes);
    if (rc == HPG_OK) rc = dev_alloc((void**)&bs->zc[l], bytes);
    if (rc) return rc;
  }
  return HPG_OK;
}

// ------------------------------------------------------- stencil launchers
static bool streamed(const Level& L) { return L.g.n_store * 27LL * 8 > kStreamMatrixBytes; }

static Shape shape_of(hpg_problem* h, int level, int kind, int R) {
  Shape sh = h->batch ? h->batch->shape[level][kind][R] : Shape();
  if (sh.lpr == 0) sh.lpr = 1;
  if (sh.block == 0) sh.block = streamed(h->lev[level]) ? 256 : 64;
  return sh;
}

// Load policy of a level's matrix (as in sparse.cu): streamed evict-first
// where the FP32 ELL arrays exceed the streaming size, evict-last where they
// are small (coarse levels read by every V-cycle), cached otherwise.
static int mmat_mode(const Level& L) {
  const long long b = L.g.n_store * 27LL * 8;
  return b > kStreamMatrixBytes ? kMatStream : b > kResidentMatrixBytes ? kMatCached
                                                                        : kMatResident;
}

template <int R, int LPR, int MODE, int MC>
static cudaError_t mgs_kl(hpg_problem* h, int grid, int block, cudaStream_t s, const float* vals,
                          const int* cols, long long ns, const float* rhs, float* z,
                          long long row0, long long nrows, long long valid_end, unsigned mask) {
  return kl(h, mgs_phase_kernel<R, LPR, MODE, MC>, grid, block, s, vals, cols, ns, rhs, z, row0,
            nrows, valid_end, mask);
}

// Colour c of the first sweep from zero with its compile-time slot set.
template <int R, int MODE>
static cudaError_t mgs_colour(hpg_problem* h, int c, int grid, int block, cudaStream_t s,
                              const float* vals, const int* cols, long long ns,
                              const float* rhs, float* z, long long row0, long long nrows,
                              long long valid_end, unsigned mask) {
  switch (c) {
#define HPG_MGS_CASE(C)                                                                   \
  case C:                                                                                 \
    return mgs_kl<R, 1, MODE, C>(h, grid, block, s, vals, cols, ns, rhs, z, row0, nrows, \
                                 valid_end, mask);
    HPG_MGS_CASE(0) HPG_MGS_CASE(1) HPG_MGS_CASE(2) HPG_MGS_CASE(3)
    HPG_MGS_CASE(4) HPG_MGS_CASE(5) HPG_MGS_CASE(6) HPG_MGS_CASE(7)
#undef HPG_MGS_CASE
  }
  return cudaErrorInvalidValue;
}

template <int R, int LPR, int MODE>
static cudaError_t mgs_launch(hpg_problem* h, int c, bool masked, int grid, int block,
                              cudaStream_t s, const float* vals, const int* cols, long long ns,
                              const float* rhs, float* z, long long row0, long long nrows,
                              long long valid_end, unsigned mask) {
  if (!masked)
    return mgs_kl<R, LPR, MODE, kAllSlots>(h, grid, block, s, vals, cols, ns, rhs, z, row0,
                                           nrows, valid_end, mask);
  if constexpr (LPR == 1)
    return mgs_colour<R, MODE>(h, c, grid, block, s, vals, cols, ns, rhs, z, row0, nrows,
                               valid_end, mask);
  return mgs_kl<R, LPR, MODE, kMaskSlots>(h, grid, block, s, vals, cols, ns, rhs, z, row0, nrows,
                                          valid_end, mask);
}

template <int R, int LPR>
static cudaError_t mgs_mode(hpg_problem* h, int mode, int c, bool masked, int grid, int block,
                            cudaStream_t s, const float* vals, const int* cols, long long ns,
                            const float* rhs, float* z, long long row0, long long nrows,
                            long long valid_end, unsigned mask) {
  if (mode == kMatStream)
    return mgs_launch<R, LPR, kMatStream>(h, c, masked, grid, block, s, vals, cols, ns, rhs, z,
                                          row0, nrows, valid_end, mask);
  if (mode == kMatResident)
    return mgs_launch<R, LPR, kMatResident>(h, c, masked, grid, block, s, vals, cols, ns, rhs,
                                            z, row0, nrows, valid_end, mask);
  return mgs_launch<R, LPR, kMatCached>(h, c, masked, grid, block, s, vals, cols, ns, rhs, z,
                                        row0, nrows, valid_end, mask);
}

template <int R>
static cudaError_t mgs_dispatch(hpg_problem* h, int lpr, int mode, int c, bool masked,
                                long long nrows, int block, cudaStream_t s, const float* vals,
                                const int* cols, long long ns, const float* rhs, float* z,
                                long long row0, long long valid_end, unsigned mask) {
  constexpr int L2 = R >= 2 ? 2 : 1;
  const int grid = grid_for(nrows * lpr, block);
  if (lpr == 1)
    return mgs_mode<R, 1>(h, mode, c, masked, grid, block, s, vals, cols, ns, rhs, z, row0,
                          nrows, valid_end, mask);
  if (lpr == 2)
    return mgs_mode<R, L2>(h, mode, c, masked, grid, block, s, vals, cols, ns, rhs, z, row0,
                           nrows, valid_end, mask);
  return mgs_mode<R, R>(h, mode, c, masked, grid, block, s, vals, cols, ns, rhs, z, row0, nrows,
                        valid_end, mask);
}

struct BSweep {
  int last = -1;   // colour of the latest phase on unchanged data (skipped if repeated)
};

template <int R>
static int mgs_phase(hpg_problem* h, int level, const float* rhs, float* z, int c,
                     bool from_zero, BSweep& sw, cudaStream_t s) {
  if (sw.last == c) return HPG_OK;
  const Level& L = h->lev[level];
  const long long row0 = L.g.off[c];
  const long long nrows = L.g.off[c + 1] - row0;
  sw.last = c;
  if (nrows == 0) return HPG_OK;
  const long long valid_end = from_zero ? row0 : L.g.n_store;
  const unsigned mask = gs_slot_mask(c, from_zero);
  const int nslots = __builtin_popcount(mask) - 1;
  const double row_bytes = (nslots + 1.0) * 4 + nslots * 4.0 + R * (2.0 + nslots / 26.0) * 4;
  const Shape sh = shape_of(h, level, kShapeGs, R);
  return launch(h, K_GS, level, HPG_FP32, L.cnt[c] * row_bytes, s, "mgs_phase_kernel", [&] {
    // phases of up to HPG_OPT_PDL_ROWS rows (none of a streamed level by
    // default) are launched programmatically; measured on GB300, launching
    // the 110,592-row phases of a 96^3 system so as well (triggering at
    // block exit) made its 8-RHS solve 72.6 instead of 70.9 ms
    if (nrows > h->pdl_rows) h->pdl_next = false;
    return mgs_dispatch<R>(h, sh.lpr, mmat_mode(L), c, from_zero, nrows, sh.block, s, L.v32,
                           L.cols, L.g.n_store, rhs, z, row0, valid_end, mask);
  });
}

template <int R>
static int msymgs(hpg_problem* h, int level, const float* rhs, float* z, bool from_zero,
                  BSweep& sw, cudaStream_t s) {
  int rc;
  for (int c = 0; c < kColours; ++c)
    if ((rc = mgs_phase<R>(h, level, rhs, z, c, from_zero, sw, s))) return rc;
  for (int c = kColours - 1; c >= 0; --c)
    if ((rc = mgs_phase<R>(h, level, rhs, z, c, false, sw, s))) return rc;
  return HPG_OK;
}

template <int R, int LPR>
static cudaError_t mspmv_launch(hpg_problem* h, const Level& L, int block, cudaStream_t s,
                                const float* x, float* y) {
  return kl(h, mspmv_kernel<R, LPR>, grid_for(L.g.n_store * LPR, block), block, s, L.v32, L.cols,
            L.g.n_store, x, y);
}

template <int R>
static int mspmv_t(hpg_problem* h, int level, const float* x, float* y, cudaStream_t s) {
  const Level& L = h->lev[level];
  const Shape sh = shape_of(h, level, kShapeSpmv, R);
  constexpr int L2 = R >= 2 ? 2 : 1;
  return launch(h, K_SPMV, level, HPG_FP32, L.g.n_store * (27.0 * 8 + 2.0 * 4 * R), s,
                "mspmv_kernel", [&] {
                  h->pdl_next = false;   // required by the read-only gathers of X
                  if (sh.lpr == 1) return mspmv_launch<R, 1>(h, L, sh.block, s, x, y);
                  if (sh.lpr == 2) return mspmv_launch<R, L2>(h, L, sh.block, s, x, y);
                  return mspmv_launch<R, R>(h, L, sh.block, s, x, y);
                });
}

// z = M^{-1} r for R right-hand sides: the V-cycle of sparse.cu, phase for
// phase, on R-vectors.
template <int R>
static int mvcycle_t(hpg_problem* h, int l, const float* rhs, float* z, cudaStream_t s) {
  const Level& L = h->lev[l];
  BatchSpace* bs = h->batch;
  BSweep sw;
  int rc;
  if (l == h->nlev - 1) return msymgs<R>(h, l, rhs, z, true, sw, s);
  if (h->pre == 0) {
    HPG_CK(cudaMemsetAsync(z, 0, sizeof(float) * L.g.n_store * R, s));
    h->pdl_next = false;
  }
  for (int it = 0; it < h->pre; ++it)
    if ((rc = msymgs<R>(h, l, rhs, z, it == 0, sw, s))) return rc;
  const Level& C = h->lev[l + 1];
  float* rcv = bs->rc[l + 1];
  float* zcv = bs->zc[l + 1];
  const long long cnt = (long long)L.g.cdx[kCoarseColour] * L.g.cdy[kCoarseColour] *
                        L.g.cdz[kCoarseColour];
  rc = launch(h, K_RESTRICT, l, HPG_FP32, cnt * (27.0 * 8 + 3.0 * 4 * R), s, "mrestrict_kernel",
              [&] {
                const int mode = mmat_mode(L);
                auto kern = mode == kMatStream     ? mrestrict_kernel<R, kMatStream>
                            : mode == kMatResident ? mrestrict_kernel<R, kMatResident>
                                                   : mrestrict_kernel<R, kMatCached>;
                return kl(h, kern, grid_for(cnt, 256), 256, s, L.g, C.g, L.v32, L.cols, rhs, z,
                          rcv);
              });
  if (rc) return rc;
  if ((rc = mvcycle_t<R>(h, l + 1, rcv, zcv, s))) return rc;
  rc = launch(h, K_PROLONG, l, HPG_FP32, cnt * 3.0 * 4 * R, s, "mprolong_kernel", [&] {
    return kl(h, mprolong_kernel<R>, grid_for(cnt, 256), 256, s, L.g, C.g, (const float*)zcv, z);
  });
  if (rc) return rc;
  sw.last = -1;
  for (int it = 0; it < h->post; ++it)
    if ((rc = msymgs<R>(h, l, rhs, z, false, sw, s))) return rc;
  return HPG_OK;
}

static int run_mvcycle(hpg_problem* h, int R, int level, const float* rhs, float* z,
                       cudaStream_t s) {
  switch (R) {
    case 1: return mvcycle_t<1>(h, level, rhs, z, s);
    case 2: return mvcycle_t<2>(h, level, rhs, z, s);
    case 4: return mvcycle_t<4>(h, level, rhs, z, s);
    default: return mvcycle_t<8>(h, level, rhs, z, s);
  }
}

static int run_mspmv(hpg_problem* h, int R, int level, const float* x, float* y,
                     cudaStream_t s) {
  switch (R) {
    case 1: return mspmv_t<1>(h, level, x, y, s);
    case 2: return mspmv_t<2>(h, level, x, y, s);
    case 4: return mspmv_t<4>(h, level, x, y, s);
    default: return mspmv_t<8>(h, level, x, y, s);
  }
}

static bool valid_r(int R) { return R == 1 || R == 2 || R == 4 || R == 8; }

// ------------------------------------------------------- batched Krylov
// Threads of the element-wise Krylov kernels walk the R-vector [ns][R] as a
// flat array with a grid stride that is a multiple of R, so a thread always
// meets the same right-hand side, r = threadIdx.x % R.
constexpr int kBThreads = 256;
constexpr int kBWarps = kBThreads / 32;
constexpr int kGroupBlocks = 16;   // blocks per first-level reduction group

// Sum over the lanes of a warp that hold the same right-hand side; lanes
// 0..R-1 end with the sums of right-hand sides 0..R-1.
template <int R, typename A>
__device__ __forceinline__ A warp_sum_r(A v) {
#pragma unroll
  for (int o = 16; o >= R; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic grid sum of nred = ncol * R entries (entry j * R + r):
// warps, then the block, store one partial per block; the last block of each
// group of kGroupBlocks blocks (ticket) adds its group's partials in block
// order, and the last group to finish adds the group sums in group order into
// sums[] (shared).  Returns true in that final block.
template <int R, int KMAX, typename A>
__device__ bool mblock_partials_last(const A (&acc)[KMAX], int ncol, double* partials,
                                     double* gpart, unsigned int* counter, double* sums) {
  __shared__ A red[kBWarps][KMAX * R];   // warp sums (exact in A)
  __shared__ int role;   // 0: done, 1: group closer, 2: final closer
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nred = ncol * R;
#pragma unroll
  for (int j = 0; j < KMAX; ++j) {
    if (j < ncol) {
      const A v = warp_sum_r<R>(acc[j]);
      if (lane < R) red[warp][j * R + lane] = v;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nred; i += kBThreads) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kBWarps; ++q) s += (double)red[q][i];
    partials[(long long)blockIdx.x * kBatchPartStride + i] = s;
  }
  __threadfence();
  __syncthreads();
  const int g = blockIdx.x / kGroupBlocks;
  const int ngroups = (gridDim.x + kGroupBlocks - 1) / kGroupBlocks;
  const int gb0 = g * kGroupBlocks;
  const int gb1 = min((int)gridDim.x, gb0 + kGroupBlocks);
  if (threadIdx.x == 0) role = (atomicAdd(counter + 1 + g, 1u) == (unsigned)(gb1 - gb0 - 1));
  __syncthreads();
  if (!role) return false;
  __threadfence();
  for (int i = threadIdx.x; i < nred; i += kBThreads) {
    double s = 0.0;
    for (int b = gb0; b < gb1; ++b) s += __ldcg(partials + (long long)b * kBatchPartStride + i);
    gpart[(long long)g * kBatchPartStride + i] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    counter[1 + g] = 0u;
    role = (atomicAdd(counter, 1u) == (unsigned)(ngroups - 1)) ? 2 : 0;
  }
  __syncthreads();
  if (role != 2) return false;
  __threadfence();
  for (int i = threadIdx.x; i < nred; i += kBThreads) {
    double s = 0.0;
    for (int q = 0; q < ngroups; ++q) s += __ldcg(gpart + (long long)q * kBatchPartStride + i);
    sums[i] = s;
  }
  if (threadIdx.x == 0) counter[0] = 0u;
  __syncthreads();
  return true;
}

// Arnoldi column and Givens update (Algorithm 3) of one right-hand side, one
// warp, in two parts as in the single solve: brotate_warp applies the old
// rotations 0..k-1 to column k = h1 + h2 (rows 0..k; it needs no beta) while
// the final pass streams, and leaves the rotated column in H; bgivens_warp,
// once beta is known, forms rotation k from H[k,k] and beta, updates t and rho
// and returns whether this right-hand side's cycle continues.  Same
// operations in the same order as doing it all at the end.
__device__ void brotate_warp(int k, const double* __restrict__ h1,
                             const double* __restrict__ h2, double* __restrict__ hcol,
                             const double* __restrict__ cs, const double* __restrict__ sn,
                             double* hs, double* css, double* sns) {
  const int lane = threadIdx.x & 31;
  for (int j = lane; j <= k; j += 32) {
    hs[j] = ld_dep(h1 + j) + ld_dep(h2 + j);
    if (j < k) {
      css[j] = ld_dep(cs + j);
      sns[j] = ld_dep(sn + j);
    }
  }
  __syncwarp();
  if (lane == 0) {
    for (int j = 0; j < k; ++j) {
      const double a = hs[j], b = hs[j + 1];
      hs[j] = css[j] * a + sns[j] * b;
      hs[j + 1] = -sns[j] * a + css[j] * b;
    }
  }
  __syncwarp();
  for (int j = lane; j <= k; j += 32) hcol[j] = hs[j];
}

__device__ bool bgivens_warp(double beta, int k, double* __restrict__ hcol,
                             double* __restrict__ cs, double* __restrict__ sn,
                             double* __restrict__ t, BState* st) {
  const int lane = threadIdx.x & 31;
  bool go = false;
  if (lane == 0) {
    st->beta = beta;
    if (!isfinite(beta)) {
      st->status = HPG_ERR_NAN;
      st->active = 0;
      hcol[k + 1] = beta;
    } else {
      const double a = __ldcg(hcol + k);   // H[k,k] after the old rotations
      const double mu = hypot(a, beta);
      if (!(mu > 0.0) || !isfinite(mu)) {
        st->status = isfinite(mu) ? HPG_ERR_BREAKDOWN : HPG_ERR_NAN;
        st->active = 0;
        hcol[k + 1] = beta;
      } else {
        const double c = a / mu, sv = beta / mu;
        cs[k] = c;
        sn[k] = sv;
        hcol[k] = mu;
        hcol[k + 1] = 0.0;
        const double tk = t[k];
        t[k + 1] = -sv * tk;
        t[k] = c * tk;
        const double rho = fabs(-sv * tk);
        st->rho = rho;
        st->k = k + 1;
        st->iters += 1;
        go = !(rho / st->rho0 < st->tol || st->iters >= st->maxit || k + 1 >= st->m);
        st->active = go ? 1 : 0;
      }
    }
  }
  return __shfl_sync(0xffffffffu, go, 0);
}

enum BPassKind { kBGemvT = 0, kBReorth = 1, kBFinal = 2 };

// Rows per thread per iteration of the multi-right-hand-side CGS2 passes: the
// KMAX x V basis values of an iteration take at most 64 registers.
template <int KMAX>
__host__ __device__ constexpr int mpass_vec() {
  return KMAX <= 16 ? 4 : KMAX <= 32 ? 2 : 1;
}
constexpr int kHStride = kMaxRestart + 1;   // per-RHS stride of h1, h2, cs, sn, t, y

// One CGS2 pass (Algorithm 3, CGS2 procedure) for R right-hand sides, each
// against its own basis q_0..q_{ncol-1}: GEMVT h1 = Q^T w; reorth
// w' = w - Q h1 (stored over w), h2 = Q^T w'; final w'' = w' - Q h2 into the
// basis column ncol, ||w''||^2, then (last block, one warp per right-hand
// side still active) the Arnoldi column and the Givens update.  Per-thread
// sums in FP32, grid sums in FP64, as the single solve.
template <int R, int KMAX, int KIND>
__global__ void __launch_bounds__(kBThreads, (KMAX <= 32 ? 2 : 1))
mcgs2_pass_kernel(const float* __restrict__ Q, long long len, int ncol, float* w,
                  const double* __restrict__ h1, const double* __restrict__ h2, float* wout,
                  double* partials, double* gpart, unsigned int* counter,
                  double* __restrict__ out, double* __restrict__ H, int ldh,
                  double* __restrict__ cs, double* __restrict__ sn, double* __restrict__ t,
                  BState* st, int* runs, unsigned long long next) {
  // one row of coefficients per right-hand side; rows padded by one so that
  // the R rows a warp reads at once (r = lane % R) fall into distinct banks
  __shared__ float shc[R][KMAX + 1];
  __shared__ double sums[KMAX * R];
  __shared__ double hs[R][kMaxRestart + 2], css[R][kMaxRestart], sns[R][kMaxRestart];
  pdl_trigger();
  pdl_wait();
  const int r = threadIdx.x % R;
  if (KIND != kBGemvT) {
    const double* hc = KIND == kBReorth ? h1 : h2;
    for (int i = threadIdx.x; i < ncol * R; i += kBThreads)
      shc[i % R][i / R] = (float)ld_dep(hc + (i % R) * kHStride + i / R);
    __syncthreads();
  }
  // the old rotations of each active right-hand side's Arnoldi column, one
  // warp per right-hand side of block 0, while the other blocks stream; block
  // 0 takes its ticket (and the final block reads H) only afterwards
  if (KIND == kBFinal && blockIdx.x == 0) {
    for (int rr = threadIdx.x >> 5; rr < R; rr += kBWarps)
      if (st[rr].active)
        brotate_warp(ncol - 1, h1 + rr * kHStride, h2 + rr * kHStride,
                     H + (long long)rr * ldh * (ldh - 1) + (long long)(ncol - 1) * ldh,
                     cs + rr * kHStride, sn + rr * kHStride, hs[rr], css[rr], sns[rr]);
  }
  float acc[KMAX];
#pragma unroll
  for (int j = 0; j < KMAX; ++j) acc[j] = 0.0f;
  // A thread keeps one right-hand side r (the block size and the grid stride
  // are multiples of R) and takes V consecutive storage rows of it per
  // iteration, issuing all their basis and w loads before any arithmetic, so
  // that KMAX x V loads are in flight (in the in-place passes the store to
  // wout could otherwise hold back the next row's loads).  Row group g holds
  // rows g*V .. g*V+V-1; their elements sit R apart, and the R lanes of a row
  // together read R contiguous values.
  constexpr int V = mpass_vec<KMAX>();
  // this thread's coefficients in registers where they fit beside the basis
  // values and the sums (the final pass keeps one sum, up to 16 columns all)
  constexpr bool kRegCoef = KIND == kBFinal || KMAX <= 16;
  float coef[kRegCoef ? KMAX : 1];
  if constexpr (kRegCoef) {
#pragma unroll
    for (int j = 0; j < KMAX; ++j) coef[j] = (KIND != kBGemvT && j < ncol) ? shc[r][j] : 0.0f;
  }
  const long long rows = len / R;
  const long long ng = rows / V;
  const long long slot0 = (blockIdx.x * (long long)kBThreads + threadIdx.x) / R;
  const long long nslots = (long long)gridDim.x * (kBThreads / R);
  for (long long g = slot0; g < ng; g += nslots) {
    const long long e0 = g * V * R + r;
    float wr[V];
    float q[KMAX][V];
#pragma unroll
    for (int v = 0; v < V; ++v) wr[v] = __ldcs(w + e0 + v * R);
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
      if (j < ncol) {
#pragma unroll
        for (int v = 0; v < V; ++v) q[j][v] = __ldcs(Q + j * len + e0 + v * R);
      }
    if (KIND == kBGemvT) {
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int j = 0; j < KMAX; ++j)
          if (j < ncol) acc[j] = fma(q[j][v], wr[v], acc[j]);
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        float sc = 0.0f;
#pragma unroll
        for (int j = 0; j < KMAX; ++j)
          if (j < ncol) sc = fma(q[j][v], kRegCoef ? coef[j] : shc[r][j], sc);
        wr[v] = wr[v] - sc;
      }
#pragma unroll
      for (int v = 0; v < V; ++v) wout[e0 + v * R] = wr[v];
#pragma unroll
      for (int v = 0; v < V; ++v) {
        if (KIND == kBReorth) {
#pragma unroll
          for (int j = 0; j < KMAX; ++j)
            if (j < ncol) acc[j] = fma(q[j][v], wr[v], acc[j]);
        } else {
          acc[0] = fma(wr[v], wr[v], acc[0]);
        }
      }
    }
  }
  const int nc = KIND == kBFinal ? 1 : ncol;
  if (!mblock_partials_last<R, KMAX>(acc, nc, partials, gpart, counter, sums)) return;
  if (KIND != kBFinal) {
    for (int i = threadIdx.x; i < nc * R; i += kBThreads)
      out[(i % R) * kHStride + i / R] = sums[i];
    return;
  }
  const int warp = threadIdx.x >> 5;
  __shared__ int any_go;
  if (threadIdx.x == 0) any_go = 0;
  __syncthreads();
  for (int rr = warp; rr < R; rr += kBWarps) {
    if (!st[rr].active) continue;
    const bool go = bgivens_warp(
        sqrt(sums[rr]), ncol - 1,
        H + (long long)rr * ldh * (ldh - 1) + (long long)(ncol - 1) * ldh,
        cs + rr * kHStride, sn + rr * kHStride, t + rr * kHStride, st + rr);
    if (go && (threadIdx.x & 31) == 0) any_go = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    runs[0] += 1;
    if (next) cudaGraphSetConditional(next, any_go ? 1u : 0u);
  }
}

// q_{k+1} = w'' / beta for every right-hand side whose step completed (its
// state advanced to k + 1 with a finite, positive beta).
template <int R>
__global__ void __launch_bounds__(kBThreads)
mscale_kernel(float* __restrict__ qnew, long long len, int k1, const BState* st) {
  pdl_trigger();
  pdl_wait();
  __shared__ float inv[R];
  __shared__ bool ok[R];
  if (threadIdx.x < R) {
    const BState& s = st[threadIdx.x];
    ok[threadIdx.x] = s.k == k1 && isfinite(s.beta) && s.beta > 0.0;
    inv[threadIdx.x] = ok[threadIdx.x] ? (float)(1.0 / s.beta) : 0.0f;
  }
  __syncthreads();
  const int r = threadIdx.x % R;
  if (!ok[r]) return;
  const long long stride = (long long)gridDim.x * kBThreads;
  for (long long e = blockIdx.x * (long long)kBThreads + threadIdx.x; e < len; e += stride)
    qnew[e] = qnew[e] * inv[r];
}

// y_r = H_r[:k_r, :k_r]^{-1} t_r, one warp per right-hand side.
template <int R>
__global__ void mtrsm_kernel(const double* __restrict__ H, int ldh, const double* __restrict__ t,
                             double* __restrict__ y, const BState* st) {
  pdl_trigger();
  pdl_wait();
  __shared__ double tt[R][kMaxRestart + 1];
  __shared__ double yi_s[R];
  const int rr = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (rr >= R) return;
  const int k = st[rr].k;
  const double* Hr = H + (long long)rr * ldh * (ldh - 1);
  for (int j = lane; j < k; j += 32) tt[rr][j] = ld_dep(t + rr * kHStride + j);
  __syncwarp();
  for (int i = k - 1; i >= 0; --i) {
    if (lane == 0) {
      yi_s[rr] = tt[rr][i] / ld_dep(Hr + (long long)i * ldh + i);
      y[rr * kHStride + i] = yi_s[rr];
    }
    __syncwarp();
    const double yi = yi_s[rr];
    for (int j = lane; j < i; j += 32) tt[rr][j] -= ld_dep(Hr + (long long)i * ldh + j) * yi;
    __syncwarp();
  }
}

// u = Q y per right-hand side (its own k_r columns).
template <int R>
__global__ void __launch_bounds__(kBThreads)
mcombine_kernel(const float* __restrict__ Q, long long len, const double* __restrict__ y,
                const BState* st, int kmax, float* __restrict__ u) {
  pdl_trigger();
  pdl_wait();
  __shared__ float ys[R][kMaxRestart + 1];
  __shared__ int ks[R];
  for (int i = threadIdx.x; i < R * kmax; i += kBThreads)
    ys[i / kmax][i % kmax] = (float)ld_dep(y + (i / kmax) * kHStride + i % kmax);
  if (threadIdx.x < R) ks[threadIdx.x] = st[threadIdx.x].k;
  __syncthreads();
  const int r = threadIdx.x % R;
  const int k = ks[r];
  const long long stride = (long long)gridDim.x * kBThreads;
  for (long long e = blockIdx.x * (long long)kBThreads + threadIdx.x; e < len; e += stride) {
    float acc = 0.0f;
    for (int j = 0; j < k; ++j) acc = fma(__ldcs(Q + j * len + e), ys[r][j], acc);
    u[e] = acc;
  }
}

// x += d (FP64 accumulation of the FP32 correction).
__global__ void __launch_bounds__(kBThreads)
mupdate_x_kernel(double* __restrict__ x, const float* __restrict__ d, long long len) {
  pdl_trigger();
  pdl_wait();
  const long long e = blockIdx.x * (long long)kBThreads + threadIdx.x;
  if (e < len) x[e] += (double)ld_dep(d + e);
}

// r = b - A x (FP64, Algorithm 3 outer residual) and ||r_r||^2 per
// right-hand side, one thread per storage row.
template <int R>
__global__ void __launch_bounds__(kBThreads)
mresidual_kernel(const double* __restrict__ vals, const int* __restrict__ cols, long long ns,
                 const double* __restrict__ b, const double* __restrict__ x,
                 double* __restrict__ res, double* partials, double* gpart,
                 unsigned int* counter, double* __restrict__ out) {
  pdl_trigger();
  pdl_wait();
  double acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = 0.0;
  const long long stride = (long long)gridDim.x * kBThreads;
  for (long long row = blockIdx.x * (long long)kBThreads + threadIdx.x; row < ns;
       row += stride) {
    double v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = ld_dep(b + row * R + r);
#pragma unroll
    for (int s = 0; s < kSlots; ++s) {
      const double a = ld_stream(vals + s * ns + row);
      const int c = ld_stream(cols + s * ns + row);
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = fma(-a, ld_dep(x + (long long)c * R + r), v[r]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      res[row * R + r] = v[r];
      acc[r] = fma(v[r], v[r], acc[r]);
    }
  }
  __shared__ double sums[R];
  if (mblock_partials_last<1, R>(acc, R, partials, gpart, counter, sums) && threadIdx.x < R)
    out[threadIdx.x] = sums[threadIdx.x];
}

// ||v_r||^2 of an FP64 R-vector.
template <int R>
__global__ void __launch_bounds__(kBThreads)
mnorm2_kernel(const double* __restrict__ v, long long ns, double* partials, double* gpart,
              unsigned int* counter, double* __restrict__ out) {
  pdl_trigger();
  pdl_wait();
  double acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = 0.0;
  const long long stride = (long long)gridDim.x * kBThreads;
  for (long long row = blockIdx.x * (long long)kBThreads + threadIdx.x; row < ns;
       row += stride)
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const double vr = ld_dep(v + row * R + r);
      acc[r] = fma(vr, vr, acc[r]);
    }
  __shared__ double sums[R];
  if (mblock_partials_last<1, R>(acc, R, partials, gpart, counter, sums) && threadIdx.x < R)
    out[threadIdx.x] = sums[threadIdx.x];
}

// Outer test per right-hand side (as the single solve's); a right-hand side
// already done stays done.  In graph mode it keeps the WHILE node open while
// any right-hand side is not done.
template <int R>
__global__ void mouter_check_kernel(const double* __restrict__ rho2, BState* st,
                                    unsigned long long loop) {
  pdl_trigger();
  pdl_wait();
  __shared__ int open;
  if (threadIdx.x == 0) open = 0;
  __syncthreads();
  if (threadIdx.x < R) {
    BState& s = st[threadIdx.x];
    if (!s.done) {
      const double rho = sqrt(ld_dep(rho2 + threadIdx.x));
      const double rel = rho / s.rho0;
      s.rho = rho;
      s.rel = rel;
      bool done = true;
      if (!isfinite(rel)) {
        s.status = HPG_ERR_NAN;
      } else if (rel < s.tol) {
        s.converged = 1;
      } else if (s.status != HPG_OK) {
      } else if (s.iters >= s.maxit) {
        s.status = HPG_ERR_NOT_CONVERGED;
      } else {
        done = false;
      }
      s.done = done ? 1 : 0;
      if (!done) atomicOr(&open, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && loop) cudaGraphSetConditional(loop, open ? 1u : 0u);
}

// Start of a restart cycle for every right-hand side not done: q_0 = r / rho,
// t = rho e_1, k = 0; done ones are frozen (k = 0, inactive).  In graph mode
// opens step 0's IF node if any right-hand side is active.
template <int R>
__global__ void __launch_bounds__(kBThreads)
mcycle_start_kernel(const double* __restrict__ res, long long len, float* __restrict__ q0,
                    double* __restrict__ t, BState* st, int m, int* runs,
                    const unsigned long long* __restrict__ handles, int nhandles) {
  pdl_trigger();
  pdl_wait();
  __shared__ double inv[R];
  __shared__ int act[R];
  if (threadIdx.x < R) {
    const BState& s = st[threadIdx.x];
    act[threadIdx.x] = !s.done;
    inv[threadIdx.x] = act[threadIdx.x] ? 1.0 / s.rho : 0.0;
  }
  __syncthreads();
  const long long e = blockIdx.x * (long long)kBThreads + threadIdx.x;
  const int r = threadIdx.x % R;
  if (e < len) q0[e] = act[r] ? (float)(ld_dep(res + e) * inv[r]) : 0.0f;
  if (blockIdx.x != 0) return;
  if (threadIdx.x < R) {
    BState& s = st[threadIdx.x];
    double* tr = t + threadIdx.x * kHStride;
    tr[0] = act[threadIdx.x] ? s.rho : 0.0;
    for (int j = 1; j <= m; ++j) tr[j] = 0.0;
    s.k = 0;
    s.active = act[threadIdx.x];
    if (act[threadIdx.x]) s.restarts += 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int any = 0;
    for (int q = 0; q < R; ++q) any |= act[q];
    runs[1] += any;
    for (int j = 0; j < nhandles; ++j)
      cudaGraphSetConditional(handles[j], (j == 0 && any) ? 1u : 0u);
  }
}

// ---------------------------------------------------------- host: buffers
static int ensure_bworkspace(hpg_problem* h, int R, int m) {
  int rc = ensure_vcycle_buffers(h);
  if (rc) return rc;
  BatchSpace* bs = h->batch;
  if (bs->Q && bs->R == R && bs->m >= m) return HPG_OK;
  if (bs->owners > 0) {
    set_error("batch buffers of this problem belong to a multi-system batch (%d right-hand "
              "sides, restart %d); destroy the batch first", bs->R, bs->m);
    return HPG_ERR_STATE;
  }
  // (re)allocate the Krylov buffers; graph and shapes survive only the shapes
  if (bs->exec) cudaGraphExecDestroy(bs->exec);
  if (bs->graph) cudaGraphDestroy(bs->graph);
  bs->exec = nullptr;
  bs->graph = nullptr;
  void** ptrs[] = {(void**)&bs->Q, (void**)&bs->z, (void**)&bs->w, (void**)&bs->u,
                   (void**)&bs->b, (void**)&bs->x, (void**)&bs->r, (void**)&bs->partials,
                   (void**)&bs->counter, (void**)&bs->h1, (void**)&bs->h2, (void**)&bs->H,
                   (void**)&bs->cs, (void**)&bs->sn, (void**)&bs->t, (void**)&bs->y,
                   (void**)&bs->rho2, (void**)&bs->st, (void**)&bs->hk, (void**)&bs->runs};
  for (void** p : ptrs) {
    dev_free(*p);
    *p = nullptr;
  }
  if (bs->st_host) cudaFreeHost(bs->st_host);
  bs->st_host = nullptr;
  const long long ns = h->lev[0].g.n_store;
  bs->R = R;
  bs->m = m;
  bs->ns = ns;
  long long g = (ns * R + kBThreads - 1) / kBThreads;
  if (g > 4LL * h->num_sms) g = 4LL * h->num_sms;
  bs->G = (int)(g < 1 ? 1 : g);
  const size_t nr = (size_t)ns * R;
  rc = dev_alloc((void**)&bs->Q, sizeof(float) * nr * (m + 1));
  rc = rc ? rc : dev_alloc((void**)&bs->z, sizeof(float) * nr);
  rc = rc ? rc : dev_alloc((void**)&bs->w, sizeof(float) * nr);
  rc = rc ? rc : dev_alloc((void**)&bs->u, sizeof(float) * nr);
  rc = rc ? rc : dev_alloc((void**)&bs->b, sizeof(double) * nr);
  rc = rc ? rc : dev_alloc((void**)&bs->x, sizeof(double) * nr);
  rc = rc ? rc : dev_alloc((void**)&bs->r, sizeof(double) * nr);
  // block partials, then one row per reduction group
  rc = rc ? rc : dev_alloc((void**)&bs->partials,
                           sizeof(double) * kBatchPartStride * (bs->G + bs->G / kGroupBlocks + 1));
  rc = rc ? rc : dev_alloc((void**)&bs->counter, sizeof(unsigned) * (2 + bs->G / kGroupBlocks + 1));
  rc = rc ? rc : dev_alloc((void**)&bs->h1, sizeof(double) * kHStride * R);
  rc = rc ? rc : dev_alloc((void**)&bs->h2, sizeof(double) * kHStride * R);
  rc = rc ? rc : dev_alloc((void**)&bs->H, sizeof(double) * (size_t)(m + 1) * m * R);
  rc = rc ? rc : dev_alloc((void**)&bs->cs, sizeof(double) * kHStride * R);
  rc = rc ? rc : dev_alloc((void**)&bs->sn, sizeof(double) * kHStride * R);
  rc = rc ? rc : dev_alloc((void**)&bs->t, sizeof(double) * kHStride * R);
  rc = rc ? rc : dev_alloc((void**)&bs->y, sizeof(double) * kHStride * R);
  rc = rc ? rc : dev_alloc((void**)&bs->rho2, sizeof(double) * kMaxR);
  rc = rc ? rc : dev_alloc((void**)&bs->st, sizeof(BState) * R);
  rc = rc ? rc : dev_alloc((void**)&bs->hk, sizeof(unsigned long long) * (m + 1));
  rc = rc ? rc : dev_alloc((void**)&bs->runs, sizeof(int) * 2);
  for (int i = 0; i < 3 && rc == HPG_OK; ++i) {
    if (bs->cap[i]) continue;
    cudaError_t e = cudaStreamCreateWithFlags(&bs->cap[i], cudaStreamNonBlocking);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaStreamCreate", __FILE__, __LINE__);
  }
  if (rc == HPG_OK) {
    cudaError_t e = cudaMallocHost((void**)&bs->st_host, sizeof(BState) * R);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMallocHost", __FILE__, __LINE__);
  }
  if (rc) destroy_batch(h);
  return rc;
}

static double* gpart_of(BatchSpace* bs) { return bs->partials + (size_t)kBatchPartStride * bs->G; }

// ------------------------------------------------------ host: solve pieces
// Grid of a multi-right-hand-side CGS2 pass: one wave of the instantiation's
// resident blocks, at most the G blocks the partials are sized for.
template <int R, int KMAX, int KIND>
static int mpass_grid(hpg_problem* h) {
  static int per_sm = 0;
  if (per_sm == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mcgs2_pass_kernel<R, KMAX, KIND>,
                                                      kBThreads, 0) != cudaSuccess ||
        per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
  }
  const int g = per_sm * h->num_sms;
  return g < h->batch->G ? g : h->batch->G;
}

template <int R, int KMAX, int KIND>
static cudaError_t enqueue_mpass(hpg_problem* h, int ncol, float* wout, double* out,
                                 unsigned long long next, cudaStream_t s) {
  BatchSpace* bs = h->batch;
  const long long len = bs->ns * R;
  return kl(h, mcgs2_pass_kernel<R, KMAX, KIND>, mpass_grid<R, KMAX, KIND>(h), kBThreads, s,
            (const float*)bs->Q, len,
            ncol, bs->w, (const double*)bs->h1, (const double*)bs->h2, wout, bs->partials,
            gpart_of(bs), bs->counter, out, bs->H, bs->m + 1, bs->cs, bs->sn, bs->t, bs->st,
            bs->runs, next);
}

template <int R, int KIND>
static int launch_mpass(hpg_problem* h, int ncol, float* wout, double* out,
                        unsigned long long next, cudaStream_t s) {
  static const int cls[3] = {K_CGS2_GEMVT, K_CGS2_REORTH, K_CGS2_FINAL};
  const double bytes = (double)h->lev[0].n * R * 4.0 * (ncol + (KIND == kBGemvT ? 1 : 2));
  return launch(h, cls[KIND], 0, HPG_FP32, bytes, s, "mcgs2_pass_kernel", [&] {
    if (ncol <= 8) return enqueue_mpass<R, 8, KIND>(h, ncol, wout, out, next, s);
    if (ncol <= 16) return enqueue_mpass<R, 16, KIND>(h, ncol, wout, out, next, s);
    if (ncol <= 32) return enqueue_mpass<R, 32, KIND>(h, ncol, wout, out, next, s);
    return enqueue_mpass<R, 64, KIND>(h, ncol, wout, out, next, s);
  });
}

template <int R>
static int enqueue_mstep(hpg_problem* h, int k, unsigned long long next, cudaStream_t s) {
  BatchSpace* bs = h->batch;
  const long long len = bs->ns * R;
  int rc;
  if ((rc = mvcycle_t<R>(h, 0, bs->Q + k * len, bs->z, s))) return rc;
  if ((rc = mspmv_t<R>(h, 0, bs->z, bs->w, s))) return rc;
  const int ncol = k + 1;
  float* qnew = bs->Q + (k + 1) * len;
  if ((rc = launch_mpass<R, kBGemvT>(h, ncol, nullptr, bs->h1, 0ULL, s))) return rc;
  if ((rc = launch_mpass<R, kBReorth>(h, ncol, bs->w, bs->h2, 0ULL, s))) return rc;
  if ((rc = launch_mpass<R, kBFinal>(h, ncol, qnew, nullptr, next, s))) return rc;
  return launch(h, K_ARNOLDI_SCALE, 0, HPG_FP32, 8.0 * len, s, "mscale_kernel", [&] {
    return kl(h, mscale_kernel<R>, bs->G, kBThreads, s, qnew, len, k + 1,
              (const BState*)bs->st);
  });
}

template <int R>
static int enqueue_mupdate(hpg_problem* h, int k_model, cudaStream_t s) {
  BatchSpace* bs = h->batch;
  const long long len = bs->ns * R;
  int rc = launch(h, K_TRSM, 0, HPG_FP64, 0.0, s, "mtrsm_kernel", [&] {
    return kl(h, mtrsm_kernel<R>, 1, 32 * R, s, (const double*)bs->H, bs->m + 1,
              (const double*)bs->t, bs->y, (const BState*)bs->st);
  });
  if (rc) return rc;
  rc = launch(h, K_COMBINE, 0, HPG_FP32, 4.0 * len * (k_model + 1), s, "mcombine_kernel", [&] {
    return kl(h, mcombine_kernel<R>, bs->G, kBThreads, s, (const float*)bs->Q, len,
              (const double*)bs->y, (const BState*)bs->st, bs->m, bs->u);
  });
  if (rc) return rc;
  if ((rc = mvcycle_t<R>(h, 0, bs->u, bs->z, s))) return rc;
  return launch(h, K_UPDATE_X, 0, HPG_FP64, 20.0 * len, s, "mupdate_x_kernel", [&] {
    return kl(h, mupdate_x_kernel, grid_for(len, kBThreads), kBThreads, s, bs->x,
              (const float*)bs->z, len);
  });
}

template <int R>
static int enqueue_mouter(hpg_problem* h, unsigned long long loop, cudaStream_t s) {
  BatchSpace* bs = h->batch;
  const Level& L = h->lev[0];
  int rc = launch(h, K_RESIDUAL, 0, HPG_FP64, L.n * (27.0 * 12.0 + 3.0 * 8.0 * R), s,
                  "mresidual_kernel", [&] {
                    return kl(h, mresidual_kernel<R>, bs->G, kBThreads, s, (const double*)L.v64,
                              (const int*)L.cols, bs->ns, (const double*)bs->b,
                              (const double*)bs->x, bs->r, bs->partials, gpart_of(bs),
                              bs->counter, bs->rho2);
                  });
  if (rc) return rc;
  return launch(h, K_NORM, 0, HPG_FP64, 0.0, s, "mouter_check_kernel", [&] {
    return kl(h, mouter_check_kernel<R>, 1, 32, s, (const double*)bs->rho2, bs->st, loop);
  });
}

template <int R>
static int enqueue_mcycle_start(hpg_problem* h, const unsigned long long* handles, int nh,
                                cudaStream_t s) {
  BatchSpace* bs = h->batch;
  const long long len = bs->ns * R;
  return launch(h, K_CYCLE_START, 0, HPG_FP32, 12.0 * len, s, "mcycle_start_kernel", [&] {
    return kl(h, mcycle_start_kernel<R>, grid_for(len, kBThreads), kBThreads, s,
              (const double*)bs->r, len, bs->Q, bs->t, bs->st, bs->m, bs->runs, handles, nh);
  });
}

// ---------------------------------------------------------- host: capture
static int bappend_conditional(hpg_problem* h, cudaStream_t s, cudaGraphConditionalHandle handle,
                               cudaGraphConditionalNodeType type, cudaGraph_t* body) {
  cudaStreamCaptureStatus cst;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edges = nullptr;
  size_t nd = 0;
  HPG_CK(cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, &deps, &edges, &nd));
  if (cst != cudaStreamCaptureStatusActive) {
    set_error("batch capture: stream is not capturing");
    return HPG_ERR_CUDA;
  }
  cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
  p.conditional.handle = handle;
  p.conditional.type = type;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  HPG_CK(cudaGraphAddNode(&node, g, deps, edges, nd, &p));
  *body = p.conditional.phGraph_out[0];
  HPG_CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1,
                                             cudaStreamSetCaptureDependencies));
  h->pdl_next = false;
  return HPG_OK;
}

// Adds the whole batched solve of handle h (everything after b, x and the
// states are in place) to graph G as an independent branch:
//   outer test -> WHILE(any right-hand side not done) { cycle start ->
//   IF(h_0){step 0} -> ... -> IF(h_{m-1}){step m-1} -> update -> outer test }
template <int R>
static int capture_msolve(hpg_problem* h, int m, cudaGraph_t G, unsigned long long* hk_dev) {
  BatchSpace* bs = h->batch;
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
  cudaStream_t s0 = bs->cap[0], s1 = bs->cap[1], s2 = bs->cap[2];
  cudaGraphConditionalHandle loop;
  HPG_CK(cudaGraphConditionalHandleCreate(&loop, G, 0, 0));
  const long long launches_before = h->launches;
  HPG_CK(cudaStreamBeginCaptureToGraph(s0, G, nullptr, nullptr, 0, mode));
  h->pdl_next = false;
  long long mark = h->launches;
  int rc = enqueue_mouter<R>(h, (unsigned long long)loop, s0);
  bs->n_outer = h->launches - mark;
  cudaGraph_t body = nullptr;
  if (rc == HPG_OK) rc = bappend_conditional(h, s0, loop, cudaGraphCondTypeWhile, &body);
  cudaGraph_t g_end = nullptr;
  cudaError_t e = cudaStreamEndCapture(s0, &g_end);
  if (rc || e != cudaSuccess) {
    h->launches = launches_before;
    return rc ? rc : cuda_fail(e, "cudaStreamEndCapture(batch main)", __FILE__, __LINE__);
  }
  std::vector<cudaGraphConditionalHandle> hk(m);
  for (int k = 0; k < m; ++k) HPG_CK(cudaGraphConditionalHandleCreate(&hk[k], body, 0, 0));
  HPG_CK(cudaMemcpy(hk_dev, hk.data(), sizeof(unsigned long long) * m, cudaMemcpyHostToDevice));
  HPG_CK(cudaStreamBeginCaptureToGraph(s1, body, nullptr, nullptr, 0, mode));
  h->pdl_next = false;
  mark = h->launches;
  rc = enqueue_mcycle_start<R>(h, hk_dev, m, s1);
  bs->n_start = h->launches - mark;
  for (int k = 0; k < m && rc == HPG_OK; ++k) {
    cudaGraph_t sb = nullptr;
    rc = bappend_conditional(h, s1, hk[k], cudaGraphCondTypeIf, &sb);
    if (rc) break;
    e = cudaStreamBeginCaptureToGraph(s2, sb, nullptr, nullptr, 0, mode);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "cudaStreamBeginCaptureToGraph(batch step)", __FILE__, __LINE__);
      break;
    }
    h->pdl_next = false;
    mark = h->launches;
    rc = enqueue_mstep<R>(h, k, k + 1 < m ? (unsigned long long)hk[k + 1] : 0ULL, s2);
    bs->n_step = h->launches - mark;
    cudaGraph_t sb_end = nullptr;
    e = cudaStreamEndCapture(s2, &sb_end);
    if (rc == HPG_OK && e != cudaSuccess)
      rc = cuda_fail(e, "cudaStreamEndCapture(batch step)", __FILE__, __LINE__);
  }
  mark = h->launches;
  if (rc == HPG_OK) rc = enqueue_mupdate<R>(h, m / 2, s1);
  bs->n_update = h->launches - mark;
  if (rc == HPG_OK) rc = enqueue_mouter<R>(h, (unsigned long long)loop, s1);
  h->launches = launches_before;   // capture enqueues nothing that runs
  cudaGraph_t body_end = nullptr;
  e = cudaStreamEndCapture(s1, &body_end);
  if (rc) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture(batch body)", __FILE__, __LINE__);
  h->pdl_next = false;
  return HPG_OK;
}

static int capture_msolve_r(hpg_problem* h, int R, int m, cudaGraph_t G,
                            unsigned long long* hk_dev) {
  switch (R) {
    case 1: return capture_msolve<1>(h, m, G, hk_dev);
    case 2: return capture_msolve<2>(h, m, G, hk_dev);
    case 4: return capture_msolve<4>(h, m, G, hk_dev);
    default: return capture_msolve<8>(h, m, G, hk_dev);
  }
}

// -------------------------------------------------- host: inputs / outputs
// b, x (natural order, R vectors of n) into the storage R-vectors, ||b_r||,
// and the initial states; a right-hand side with b_r = 0 is done at once with
// x_r = 0.  Synchronises s (the states need ||b_r|| on the host).
template <int R>
static int mprepare(hpg_problem* h, const double* B, const double* X, double tol, int m,
                    int maxit, cudaStream_t s) {
  BatchSpace* bs = h->batch;
  const Level& L = h->lev[0];
  const int gs = grid_for(L.g.n_store, 256);
  int rc = launch(h, K_PERMUTE, 0, HPG_FP64, 0.0, s, "mto_storage_kernel", [&] {
    return kl(h, mto_storage_kernel<double, double>, gs, 256, s, L.g, R, B, bs->b);
  });
  if (rc) return rc;
  rc = launch(h, K_PERMUTE, 0, HPG_FP64, 0.0, s, "mto_storage_kernel", [&] {
    return kl(h, mto_storage_kernel<double, double>, gs, 256, s, L.g, R, X, bs->x);
  });
  if (rc) return rc;
  rc = launch(h, K_NORM, 0, HPG_FP64, 8.0 * L.n * R, s, "mnorm2_kernel", [&] {
    return kl(h, mnorm2_kernel<R>, bs->G, kBThreads, s, (const double*)bs->b, bs->ns,
              bs->partials, gpart_of(bs), bs->counter, bs->rho2);
  });
  if (rc) return rc;
  double rho0_sq[kMaxR];
  HPG_CK(cudaMemcpyAsync(rho0_sq, bs->rho2, sizeof(double) * R, cudaMemcpyDeviceToHost, s));
  HPG_CK(cudaStreamSynchronize(s));
  h->pdl_next = false;
  for (int r = 0; r < R; ++r) {
    BState& st = bs->st_host[r];
    memset(&st, 0, sizeof(st));
    st.rho0 = sqrt(rho0_sq[r]);
    st.tol = tol;
    st.maxit = maxit;
    st.m = m;
    st.status = HPG_OK;
    if (!(st.rho0 == st.rho0) || isinf(st.rho0)) {
      st.status = HPG_ERR_NAN;
      st.done = 1;
    } else if (st.rho0 == 0.0) {
      st.done = 1;
      st.converged = 1;
      HPG_CK(cudaMemset2DAsync(bs->x + r, sizeof(double) * R, 0, sizeof(double), bs->ns, s));
    }
  }
  HPG_CK(cudaMemcpyAsync(bs->st, bs->st_host, sizeof(BState) * R, cudaMemcpyHostToDevice, s));
  HPG_CK(cudaMemsetAsync(bs->runs, 0, sizeof(int) * 2, s));
  return HPG_OK;
}

// x back to natural order, states to the host, the per-RHS infos.
template <int R>
static int mfinish(hpg_problem* h, double* X, hpg_solve_info* infos, long long launches0,
                   bool graph, cudaStream_t s) {
  BatchSpace* bs = h->batch;
  const Level& L = h->lev[0];
  h->pdl_next = false;
  int rc = launch(h, K_PERMUTE, 0, HPG_FP64, 0.0, s, "mto_natural_kernel", [&] {
    return kl(h, mto_natural_kernel<double, double>, grid_for(L.n, 256), 256, s, L.g, R,
              (const double*)bs->x, X);
  });
  if (rc) return rc;
  int runs[2];
  HPG_CK(cudaMemcpyAsync(bs->st_host, bs->st, sizeof(BState) * R, cudaMemcpyDeviceToHost, s));
  HPG_CK(cudaMemcpyAsync(runs, bs->runs, sizeof(runs), cudaMemcpyDeviceToHost, s));
  HPG_CK(cudaStreamSynchronize(s));
  h->pdl_next = false;
  long long kl_count = h->launches - launches0;
  if (graph) {
    // outer test once per cycle plus the first, start and update per cycle,
    // one step body per inner step the device ran
    kl_count += (long long)(runs[1] + 1) * bs->n_outer +
                (long long)runs[1] * (bs->n_start + bs->n_update) + (long long)runs[0] * bs->n_step;
  }
  int status = HPG_OK;
  for (int r = 0; r < R; ++r) {
    const BState& st = bs->st_host[r];
    const bool conv = st.converged != 0;
    int sr = conv ? HPG_OK : (st.status != HPG_OK ? st.status : HPG_ERR_NOT_CONVERGED);
    if (infos) {
      hpg_solve_info& inf = infos[r];
      memset(&inf, 0, sizeof(inf));
      inf.iterations = st.iters;
      inf.restarts = st.restarts;
      inf.converged = conv ? 1 : 0;
      inf.status = sr;
      inf.rel_residual = conv && st.rho0 == 0.0 ? 0.0 : st.rel;
      inf.rho0 = st.rho0;
      inf.kernel_launches = (int)kl_count;
      inf.graph_launches = graph ? 1 : 0;
    }
    if (sr != HPG_OK && (status == HPG_OK || status == HPG_ERR_NOT_CONVERGED)) status = sr;
  }
  return status;
}

template <int R>
static int msolve_t(hpg_problem* h, const double* B, double* X, double tol, int m, int maxit,
                    hpg_solve_info* infos, cudaStream_t s) {
  int rc;
  if ((rc = ensure_bworkspace(h, R, m))) return rc;
  BatchSpace* bs = h->batch;
  const long long launches0 = h->launches;
  h->pdl_next = false;
  if ((rc = mprepare<R>(h, B, X, tol, m, maxit, s))) return rc;
  const bool graph = !h->profiling && !h->eager;
  if (graph) {
    if (!bs->exec || bs->graph_m != m) {
      if (bs->exec) cudaGraphExecDestroy(bs->exec);
      if (bs->graph) cudaGraphDestroy(bs->graph);
      bs->exec = nullptr;
      bs->graph = nullptr;
      cudaGraph_t G;
      HPG_CK(cudaGraphCreate(&G, 0));
      rc = capture_msolve<R>(h, m, G, bs->hk);
      if (rc) return rc;   // a failed capture's graph is abandoned, not destroyed
      cudaError_t e = cudaGraphInstantiate(&bs->exec, G, 0);
      if (e != cudaSuccess) {
        bs->exec = nullptr;
        return cuda_fail(e, "cudaGraphInstantiate(batch)", __FILE__, __LINE__);
      }
      bs->graph = G;
      bs->graph_m = m;
    }
    HPG_CK(cudaGraphLaunch(bs->exec, s));
  } else {
    auto read_states = [&]() -> int {
      HPG_CK(cudaMemcpyAsync(bs->st_host, bs->st, sizeof(BState) * R, cudaMemcpyDeviceToHost,
                             s));
      HPG_CK(cudaStreamSynchronize(s));
      h->pdl_next = false;
      return HPG_OK;
    };
    auto any = [&](bool active) {
      for (int r = 0; r < R; ++r)
        if (active ? bs->st_host[r].active != 0 : bs->st_host[r].done == 0) return true;
      return false;
    };
    if ((rc = enqueue_mouter<R>(h, 0ULL, s))) return rc;
    if ((rc = read_states())) return rc;
    while (any(false)) {
      if ((rc = enqueue_mcycle_start<R>(h, nullptr, 0, s))) return rc;
      if ((rc = read_states())) return rc;
      int kmax = 0;
      for (int k = 0; k < m && any(true); ++k) {
        if ((rc = enqueue_mstep<R>(h, k, 0ULL, s))) return rc;
        if ((rc = read_states())) return rc;
        kmax = k + 1;
      }
      if ((rc = enqueue_mupdate<R>(h, kmax, s))) return rc;
      if ((rc = enqueue_mouter<R>(h, 0ULL, s))) return rc;
      if ((rc = read_states())) return rc;
    }
  }
  return mfinish<R>(h, X, infos, launches0, graph, s);
}

// --------------------------------------------------- host: launch tuning
// Times every launch shape of the multi-RHS Gauss-Seidel sweep on each level
// and of the level-0 SpMV, on zero data (the work does not depend on the
// values), and keeps the fastest.  Shapes: lanes per row 1, 2 or R, blocks of
// 64, 128 or 256 threads.
template <int R>
static int tune_t(hpg_problem* h, int reps, cudaStream_t s) {
  int rc = ensure_vcycle_buffers(h);
  if (rc) return rc;
  BatchSpace* bs = h->batch;
  float *x0 = nullptr, *y0 = nullptr;
  const size_t bytes0 = sizeof(float) * (size_t)h->lev[0].g.n_store * R;
  rc = dev_alloc((void**)&x0, bytes0);
  rc = rc ? rc : dev_alloc((void**)&y0, bytes0);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (rc == HPG_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    rc = cuda_fail(cudaGetLastError(), "cudaEventCreate", __FILE__, __LINE__);
  std::vector<int> lprs = {1};
  if (R >= 2) lprs.push_back(2);
  if (R > 2) lprs.push_back(R);
  const int blocks[3] = {64, 128, 256};
  for (int l = 0; l < h->nlev && rc == HPG_OK; ++l) {
    for (int kind = 0; kind < 2 && rc == HPG_OK; ++kind) {
      if (kind == kShapeSpmv && l > 0) continue;
      float* a = l == 0 ? x0 : bs->rc[l];
      float* b = l == 0 ? y0 : bs->zc[l];
      float best = 1e30f;
      Shape best_shape;
      for (int lpr : lprs)
        for (int blk : blocks) {
          bs->shape[l][kind][R].lpr = lpr;
          bs->shape[l][kind][R].block = blk;
          float ms = 0.0f;
          for (int it = 0; it <= reps && rc == HPG_OK; ++it) {
            if (it == 1 && cudaEventRecord(e0, s) != cudaSuccess) rc = HPG_ERR_CUDA;
            h->pdl_next = false;
            BSweep sw;
            rc = kind == kShapeGs ? msymgs<R>(h, l, a, b, false, sw, s)
                                  : mspmv_t<R>(h, l, a, b, s);
          }
          if (rc) break;
          if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
              cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "tuning events", __FILE__, __LINE__);
            break;
          }
          if (ms < best) {
            best = ms;
            best_shape = bs->shape[l][kind][R];
          }
        }
      bs->shape[l][kind][R] = best_shape;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  dev_free(x0);
  dev_free(y0);
  h->pdl_next = false;
  if (bs->exec) {   // captured launches carry the old shapes
    cudaGraphExecDestroy(bs->exec);
    bs->exec = nullptr;
    if (bs->graph) cudaGraphDestroy(bs->graph);
    bs->graph = nullptr;
  }
  return rc;
}

}  // namespace hpg

// ------------------------------------------------------- multi-system batch
// Several problems (grids of any size) with nrhs right-hand sides each,
// solved by one launch of one CUDA graph that holds every problem's batched
// solve as an independent branch.
struct hpg_batch {
  std::vector<hpg_problem*> hs;
  int nrhs = 0;
  int restart = 0;
  std::vector<unsigned long long*> hk;   // IF handles of each branch
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

using namespace hpg;

static void free_batch(hpg_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (unsigned long long* p : b->hk) dev_free(p);
  for (hpg_problem* h : b->hs)
    if (h->batch && h->batch->owners > 0) h->batch->owners -= 1;
  delete b;
}

// (Re)captures the batch graph with the problems' current launch shapes.
static int capture_batch_graph(hpg_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  cudaGraph_t G = nullptr;
  HPG_CK(cudaGraphCreate(&G, 0));
  int rc = HPG_OK;
  for (size_t i = 0; i < b->hs.size() && rc == HPG_OK; ++i)
    rc = capture_msolve_r(b->hs[i], b->nrhs, b->restart, G, b->hk[i]);
  if (rc) return rc;   // a failed capture's graph is abandoned, not destroyed
  cudaError_t e = cudaGraphInstantiate(&b->exec, G, 0);
  if (e != cudaSuccess) {
    b->exec = nullptr;
    return cuda_fail(e, "cudaGraphInstantiate(batch)", __FILE__, __LINE__);
  }
  b->graph = G;
  return HPG_OK;
}

template <int R>
static int batch_prepare(hpg_problem* h, const double* B, const double* X, double tol, int m,
                         int maxit, cudaStream_t s) {
  return mprepare<R>(h, B, X, tol, m, maxit, s);
}

extern "C" {

HPG_API int hpg_batch_tune(hpg_problem_t* h, int nrhs, void* stream) {
  if (!h || !valid_r(nrhs)) {
    set_error("hpg_batch_tune: invalid argument (nrhs %d)", nrhs);
    return HPG_ERR_INVALID;
  }
  if (!h->hierarchy) {
    set_error("hpg_batch_tune: call hpg_build_mg_hierarchy first");
    return HPG_ERR_STATE;
  }
  cudaStream_t s = (cudaStream_t)stream;
  switch (nrhs) {
    case 1: return tune_t<1>(h, 3, s);
    case 2: return tune_t<2>(h, 3, s);
    case 4: return tune_t<4>(h, 3, s);
    default: return tune_t<8>(h, 3, s);
  }
}

HPG_API int hpg_batch_create(hpg_problem_t* const* hs, int nsys, int nrhs, int restart,
                             hpg_batch_t** out) {
  if (out) *out = nullptr;
  if (!hs || nsys < 1 || !out || !valid_r(nrhs) || restart < 1 || restart > kMaxRestart) {
    set_error("hpg_batch_create: invalid argument (nsys %d, nrhs %d, restart %d)", nsys, nrhs,
              restart);
    return HPG_ERR_INVALID;
  }
  for (int i = 0; i < nsys; ++i) {
    if (!hs[i] || !hs[i]->hierarchy) {
      set_error("hpg_batch_create: problem %d is missing or has no hierarchy", i);
      return HPG_ERR_INVALID;
    }
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) {
        set_error("hpg_batch_create: problem %d appears twice", i);
        return HPG_ERR_INVALID;
      }
  }
  hpg_batch* b = new hpg_batch();
  b->nrhs = nrhs;
  b->restart = restart;
  int rc = HPG_OK;
  for (int i = 0; i < nsys && rc == HPG_OK; ++i) {
    rc = ensure_bworkspace(hs[i], nrhs, restart);
    if (rc == HPG_OK) {
      b->hs.push_back(hs[i]);
      hs[i]->batch->owners += 1;
      unsigned long long* hk = nullptr;
      rc = dev_alloc((void**)&hk, sizeof(unsigned long long) * (restart + 1));
      if (rc == HPG_OK) b->hk.push_back(hk);
    }
  }
  if (rc == HPG_OK) rc = capture_batch_graph(b);
  if (rc) {
    free_batch(b);
    return rc;
  }
  *out = b;
  return HPG_OK;
}

HPG_API int hpg_batch_solve(hpg_batch_t* b, const double* const* B, double* const* X, double tol,
                            int maxit, hpg_solve_info* infos, void* stream) {
  if (!b || !B || !X || !(tol > 0.0) || maxit < 0) {
    set_error("hpg_batch_solve: invalid argument (tol %g, maxit %d)", tol, maxit);
    return HPG_ERR_INVALID;
  }
  const int nsys = (int)b->hs.size();
  for (int i = 0; i < nsys; ++i)
    if (!B[i] || !X[i]) {
      set_error("hpg_batch_solve: system %d has no b or x", i);
      return HPG_ERR_INVALID;
    }
  cudaStream_t s = (cudaStream_t)stream;
  const int R = b->nrhs;
  std::vector<long long> launches0(nsys);
  int rc = HPG_OK;
  for (int i = 0; i < nsys && rc == HPG_OK; ++i) {
    hpg_problem* h = b->hs[i];
    launches0[i] = h->launches;
    h->pdl_next = false;
    switch (R) {
      case 1: rc = batch_prepare<1>(h, B[i], X[i], tol, b->restart, maxit, s); break;
      case 2: rc = batch_prepare<2>(h, B[i], X[i], tol, b->restart, maxit, s); break;
      case 4: rc = batch_prepare<4>(h, B[i], X[i], tol, b->restart, maxit, s); break;
      default: rc = batch_prepare<8>(h, B[i], X[i], tol, b->restart, maxit, s); break;
    }
  }
  if (rc) return rc;
  HPG_CK(cudaGraphLaunch(b->exec, s));
  int status = HPG_OK;
  for (int i = 0; i < nsys; ++i) {
    hpg_problem* h = b->hs[i];
    hpg_solve_info* inf = infos ? infos + (size_t)i * R : nullptr;
    int si;
    switch (R) {
      case 1: si = mfinish<1>(h, X[i], inf, launches0[i], true, s); break;
      case 2: si = mfinish<2>(h, X[i], inf, launches0[i], true, s); break;
      case 4: si = mfinish<4>(h, X[i], inf, launches0[i], true, s); break;
      default: si = mfinish<8>(h, X[i], inf, launches0[i], true, s); break;
    }
    if (si != HPG_OK && (status == HPG_OK || status == HPG_ERR_NOT_CONVERGED)) status = si;
  }
  return status;
}

HPG_API int hpg_batch_tune_solve(hpg_batch_t* b, const double* const* B, double* const* X,
                                 double tol, int maxit, float* times_ms, void* stream) {
  if (!b || !B || !X || !(tol > 0.0) || maxit < 0) {
    set_error("hpg_batch_tune_solve: invalid argument");
    return HPG_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int R = b->nrhs;
  std::vector<int> lprs = {1};
  if (R >= 2) lprs.push_back(2);
  if (R > 2) lprs.push_back(R);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  HPG_CK(cudaEventCreate(&e0));
  HPG_CK(cudaEventCreate(&e1));
  auto set_all = [&](int lpr) {
    for (hpg_problem* h : b->hs) {
      BatchSpace* bs = h->batch;
      for (int l = 0; l < h->nlev; ++l)
        for (int kind = 0; kind < 2; ++kind) bs->shape[l][kind][R] = Shape{lpr, 0};
    }
  };
  int rc = HPG_OK;
  float best = 1e30f;
  int best_lpr = 1;
  // one untimed solve first (lazy module loading, first-touch of buffers)
  for (int pass = 0; pass <= (int)lprs.size() && rc == HPG_OK; ++pass) {
    const int lpr = lprs[pass == 0 ? 0 : pass - 1];
    set_all(lpr);
    rc = capture_batch_graph(b);
    if (rc) break;
    for (size_t i = 0; i < b->hs.size() && rc == HPG_OK; ++i) {   // every solve from x0 = 0
      const Level& L0 = b->hs[i]->lev[0];
      if (cudaMemsetAsync(X[i], 0, sizeof(double) * L0.n * R, s) != cudaSuccess)
        rc = cuda_fail(cudaGetLastError(), "cudaMemsetAsync(batch tuning x0)", __FILE__, __LINE__);
    }
    if (rc) break;
    if (cudaEventRecord(e0, s) != cudaSuccess) {
      rc = HPG_ERR_CUDA;
      break;
    }
    const int st = hpg_batch_solve(b, B, X, tol, maxit, nullptr, stream);
    if (st != HPG_OK && st != HPG_ERR_NOT_CONVERGED) {
      rc = st;
      break;
    }
    float ms = 0.0f;
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = cuda_fail(cudaGetLastError(), "batch tuning events", __FILE__, __LINE__);
      break;
    }
    if (pass > 0 && times_ms) times_ms[pass - 1] = ms;
    if (pass > 0 && ms < best) {
      best = ms;
      best_lpr = lpr;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  set_all(best_lpr);
  return capture_batch_graph(b);
}

HPG_API int hpg_batch_destroy(hpg_batch_t* b) {
  free_batch(b);
  return HPG_OK;
}

}  // extern "C"

namespace hpg {
}  // namespace hpg

using namespace hpg;

extern "C" {

HPG_API int hpg_gmres_ir_solve_batch(hpg_problem_t* h, int nrhs, const double* B, double* X,
                                     double tol, int restart, int maxit,
                                     hpg_solve_info* infos, void* stream) {
  if (infos)
    for (int r = 0; r < (nrhs > 0 && nrhs <= kMaxR ? nrhs : 0); ++r) memset(&infos[r], 0, sizeof(hpg_solve_info));
  if (!h || !B || !X || !valid_r(nrhs) || !(tol > 0.0) || restart < 1 ||
      restart > kMaxRestart || maxit < 0) {
    set_error("hpg_gmres_ir_solve_batch: invalid argument (nrhs %d, tol %g, restart %d, "
              "maxit %d)", nrhs, tol, restart, maxit);
    return HPG_ERR_INVALID;
  }
  if (!h->hierarchy) {
    set_error("hpg_gmres_ir_solve_batch: call hpg_build_mg_hierarchy first");
    return HPG_ERR_STATE;
  }
  cudaStream_t s = (cudaStream_t)stream;
  switch (nrhs) {
    case 1: return msolve_t<1>(h, B, X, tol, restart, maxit, infos, s);
    case 2: return msolve_t<2>(h, B, X, tol, restart, maxit, infos, s);
    case 4: return msolve_t<4>(h, B, X, tol, restart, maxit, infos, s);
    default: return msolve_t<8>(h, B, X, tol, restart, maxit, infos, s);
  }
}

HPG_API int hpg_spmv_batch(hpg_problem_t* h, int level, int nrhs, const float* X, float* Y,
                           void* stream) {
  if (!h || !X || !Y || X == Y || level < 0 || level >= h->nlev || !valid_r(nrhs)) {
    set_error("hpg_spmv_batch: invalid argument (level %d, nrhs %d, pointers)", level, nrhs);
    return HPG_ERR_INVALID;
  }
  h->pdl_next = false;
  return run_mspmv(h, nrhs, level, X, Y, (cudaStream_t)stream);
}

HPG_API int hpg_mg_vcycle_batch(hpg_problem_t* h, int level, int nrhs, const float* R,
                                float* Z, void* stream) {
  if (!h || !R || !Z || R == Z || level < 0 || level >= h->nlev || !valid_r(nrhs)) {
    set_error("hpg_mg_vcycle_batch: invalid argument (level %d, nrhs %d, pointers)", level,
              nrhs);
    return HPG_ERR_INVALID;
  }
  if (!h->hierarchy) {
    set_error("hpg_mg_vcycle_batch: call hpg_build_mg_hierarchy first");
    return HPG_ERR_STATE;
  }
  int rc = ensure_vcycle_buffers(h);
  if (rc) return rc;
  h->pdl_next = false;
  return run_mvcycle(h, nrhs, level, R, Z, (cudaStream_t)stream);
}

HPG_API int hpg_permute_batch(hpg_problem_t* h, int level, int direction, int nrhs,
                              const float* in, float* out, void* stream) {
  if (!h || !in || !out || level < 0 || level >= h->nlev || !valid_r(nrhs) ||
      (direction != 0 && direction != 1)) {
    set_error("hpg_permute_batch: invalid argument (level %d, direction %d, nrhs %d)", level,
              direction, nrhs);
    return HPG_ERR_INVALID;
  }
  const Level& L = h->lev[level];
  cudaStream_t s = (cudaStream_t)stream;
  h->pdl_next = false;
  return launch(h, K_PERMUTE, level, HPG_FP32, 0.0, s, "mpermute", [&] {
    if (direction == 0)
      return kl(h, mto_storage_kernel<float, float>, grid_for(L.g.n_store, 256), 256, s, L.g,
                nrhs, in, out);
    return kl(h, mto_natural_kernel<float, float>, grid_for(L.n, 256), 256, s, L.g, nrhs, in,
              out);
  });
}

HPG_API int hpg_batch_set_shape(hpg_problem_t* h, int level, int kind, int nrhs, int lpr,
                                int block) {
  if (!h || level < 0 || level >= h->nlev || (kind != 0 && kind != 1) || !valid_r(nrhs) ||
      (lpr != 0 && lpr != 1 && lpr != 2 && lpr != nrhs) || (lpr == 2 && nrhs < 2) ||
      (block != 0 && block != 64 && block != 128 && block != 256)) {
    set_error("hpg_batch_set_shape: invalid argument (level %d, kind %d, nrhs %d, lpr %d, "
              "block %d)", level, kind, nrhs, lpr, block);
    return HPG_ERR_INVALID;
  }
  BatchSpace* bs = batch_space(h);
  bs->shape[level][kind][nrhs].lpr = lpr;
  bs->shape[level][kind][nrhs].block = block;
  if (bs->exec) {   // captured launches carry the old shape
    cudaGraphExecDestroy(bs->exec);
    bs->exec = nullptr;
    if (bs->graph) cudaGraphDestroy(bs->graph);
    bs->graph = nullptr;
  }
  return HPG_OK;
}

HPG_API int hpg_batch_get_shape(const hpg_problem_t* h, int level, int kind, int nrhs, int* lpr,
                                int* block) {
  if (!h || !lpr || !block || level < 0 || level >= h->nlev || (kind != 0 && kind != 1) ||
      !valid_r(nrhs)) {
    set_error("hpg_batch_get_shape: invalid argument");
    return HPG_ERR_INVALID;
  }
  const Shape sh = shape_of(const_cast<hpg_problem_t*>(h), level, kind, nrhs);
  *lpr = sh.lpr;
  *block = sh.block;
  return HPG_OK;
}

}  // extern "C"
