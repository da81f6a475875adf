// GMRES-IR (Algorithm 3): CGS2 orthogonalisation as tall-skinny GEMV passes
// with deterministic two-stage reductions, the Arnoldi normalisation fused
// with the Givens update of the Hessenberg QR, the dense triangular solve, the
// solution update and the FP64 outer residual, driven by a host loop.
//
// Precision (Algorithm 3: blue steps may be low precision): the basis Q, the
// preconditioned vector z and w = A z are in the inner precision T with
// per-thread accumulation in T; block and global sums, H, the rotations, t, y,
// the outer residual, its norm and x are FP64.

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "hpg_internal.cuh"


namespace hpg {

constexpr int kRedThreads = 256;   // threads of every reduction kernel
constexpr int kWarps = kRedThreads / 32;
constexpr int kPartStride = 64;    // partials row stride (>= max columns)

struct SolveState {
  double rho0;    // ||b||_2
  double tol;
  double rho;     // latest residual norm (outer: true, inner: Givens estimate)
  double beta;    // latest Arnoldi norm
  int k;          // inner steps completed in the current cycle
  int active;     // 1 while the inner loop continues
  int iters;      // inner steps over all cycles
  int maxit;
  int m;          // restart length
  int status;     // HPG_OK, HPG_ERR_BREAKDOWN, HPG_ERR_NAN, HPG_ERR_NOT_CONVERGED
  int restarts;   // restart cycles started
  int done;       // outer loop finished
  int converged;  // ||b - A x|| / ||b|| < tol
  double rel;     // latest true relative residual (FP64)
  double wmax;    // max |w''| of the latest Arnoldi vector (scaled bases)
};

struct Workspace {
  int m = 0;              // restart capacity
  hpg_prec prec = HPG_FP32;   // inner precision T
  hpg_prec basis = HPG_FP32;  // basis storage B
  int G = 0;              // blocks of the reduction kernels
  void* Q = nullptr;      // [m+1][ns] basis (B)
  float* qscale = nullptr;  // [m+1] per-vector scales of a 2-byte basis
  float* qf = nullptr;    // [ns] current basis vector, dequantised (2-byte basis)
  void* z = nullptr;      // [ns] M^{-1} q_k, then M^{-1} (Q y)
  void* w = nullptr;      // [ns] A z
  void* u = nullptr;      // [ns] Q y
  double* b = nullptr;    // [ns] storage-order b
  double* x = nullptr;    // [ns] storage-order x
  double* r = nullptr;    // [ns] outer residual
  double* stage = nullptr;  // [2][n] natural-order staging for host b, x
  double* partials = nullptr;  // [G][kPartStride]
  unsigned int* counter = nullptr;
  double* h1 = nullptr;   // [kPartStride]
  double* h2 = nullptr;
  double* H = nullptr;    // [(m+1) x m] column-major, ld = m+1
  double* cs = nullptr;   // [m+1]
  double* sn = nullptr;
  double* t = nullptr;
  double* y = nullptr;
  double* rho2 = nullptr;  // ||r||^2 and max |r| of the outer residual
  SolveState* st = nullptr;      // device
  SolveState* st_host = nullptr; // pinned mirror
  unsigned long long* hk = nullptr;  // [m] IF-node handles of the captured cycle
  // whole-solve CUDA graph (captured lazily per restart length / precision)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int graph_m = 0;
  hpg_prec graph_prec = HPG_FP32;
  hpg_prec graph_basis = HPG_FP32;
  int graph_nodes = 0;
  // kernels per segment of the captured graph (for the launch count)
  long long n_outer = 0, n_start = 0, n_step = 0, n_update = 0;
  cudaStream_t cap[3] = {nullptr, nullptr, nullptr};
};

void destroy_workspace(hpg_problem* h) {
  Workspace* ws = h->ws;
  if (!ws) return;
  if (ws->exec) cudaGraphExecDestroy(ws->exec);
  if (ws->graph) cudaGraphDestroy(ws->graph);
  for (int i = 0; i < 3; ++i)
    if (ws->cap[i]) cudaStreamDestroy(ws->cap[i]);
  void* ptrs[] = {ws->Q,  ws->z,  ws->w,  ws->u,  ws->b,  ws->x,    ws->r,
                  ws->stage, ws->partials, ws->counter, ws->h1, ws->h2, ws->H, ws->cs,
                  ws->sn, ws->t,  ws->y,  ws->rho2, ws->st, ws->hk,
                  ws->qscale, ws->qf};
  for (void* p : ptrs) dev_free(p);
  if (ws->st_host) cudaFreeHost(ws->st_host);
  delete ws;
  h->ws = nullptr;
}

static int ensure_workspace(hpg_problem* h, int m, hpg_prec prec, hpg_prec basis) {
  if (h->ws && h->ws->m >= m && h->ws->prec == prec && h->ws->basis == basis) return HPG_OK;
  destroy_workspace(h);
  Workspace* ws = new Workspace();
  h->ws = ws;
  const Level& L = h->lev[0];
  const long long ns = L.g.n_store;
  const size_t es = prec_size(prec);
  ws->m = m;
  ws->prec = prec;
  ws->basis = basis;
  // reduction grids: up to 8 blocks per SM (the CGS2 passes use one wave of
  // resident blocks, at most G)
  long long g = (ns + kRedThreads - 1) / kRedThreads;
  const long long gmax = 8LL * h->num_sms;
  if (g > gmax) g = gmax;
  ws->G = (int)(g < 1 ? 1 : g);
  int rc = HPG_OK;
  rc = rc ? rc : dev_alloc(&ws->Q, prec_size(basis) * ns * (m + 1));
  rc = rc ? rc : dev_alloc((void**)&ws->qscale, sizeof(float) * (m + 1));
  if (basis != prec) rc = rc ? rc : dev_alloc((void**)&ws->qf, sizeof(float) * ns);
  rc = rc ? rc : dev_alloc(&ws->z, es * ns);
  rc = rc ? rc : dev_alloc(&ws->w, es * ns);
  rc = rc ? rc : dev_alloc(&ws->u, es * ns);
  rc = rc ? rc : dev_alloc((void**)&ws->b, 8 * ns);
  rc = rc ? rc : dev_alloc((void**)&ws->x, 8 * ns);
  rc = rc ? rc : dev_alloc((void**)&ws->r, 8 * ns);
  rc = rc ? rc : dev_alloc((void**)&ws->stage, 8 * 2 * L.n);
  rc = rc ? rc : dev_alloc((void**)&ws->partials, 8 * (size_t)ws->G * kPartStride);
  rc = rc ? rc : dev_alloc((void**)&ws->counter, 16);
  rc = rc ? rc : dev_alloc((void**)&ws->h1, 8 * kPartStride);
  rc = rc ? rc : dev_alloc((void**)&ws->h2, 8 * kPartStride);
  rc = rc ? rc : dev_alloc((void**)&ws->H, 8 * (size_t)(m + 1) * m);
  rc = rc ? rc : dev_alloc((void**)&ws->cs, 8 * (m + 1));
  rc = rc ? rc : dev_alloc((void**)&ws->sn, 8 * (m + 1));
  rc = rc ? rc : dev_alloc((void**)&ws->t, 8 * (m + 1));
  rc = rc ? rc : dev_alloc((void**)&ws->y, 8 * (m + 1));
  rc = rc ? rc : dev_alloc((void**)&ws->st, sizeof(SolveState));
  rc = rc ? rc : dev_alloc((void**)&ws->rho2, 16);
  rc = rc ? rc : dev_alloc((void**)&ws->hk, sizeof(unsigned long long) * (m + 1));
  for (int i = 0; i < 3 && rc == HPG_OK; ++i) {
    cudaError_t e = cudaStreamCreateWithFlags(&ws->cap[i], cudaStreamNonBlocking);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaStreamCreate", __FILE__, __LINE__);
  }
  if (rc == HPG_OK) {
    cudaError_t e = cudaMallocHost((void**)&ws->st_host, sizeof(SolveState));
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMallocHost", __FILE__, __LINE__);
  }
  if (rc != HPG_OK) destroy_workspace(h);
  return rc;
}

// -------------------------------------------------------------- reductions
template <typename A>
__device__ __forceinline__ A warp_sum(A v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename A>
__device__ __forceinline__ A warp_max(A v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ------------------------------------------------------------ vector access
// Four consecutive rows of a vector (16-byte aligned: storage rows come in
// multiples of 32).  Streaming variants for data read once, L2 variants for
// data read twice in one pass.
template <typename T> struct Vec4;
template <> struct Vec4<float> {
  static __device__ __forceinline__ void ld_cs(const float* p, float (&v)[4]) {
    const float4 t = __ldcs(reinterpret_cast<const float4*>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  }
  static __device__ __forceinline__ void ld_cg(const float* p, float (&v)[4]) {
    const float4 t = __ldcg(reinterpret_cast<const float4*>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  }
  static __device__ __forceinline__ void st(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <> struct Vec4<double> {
  static __device__ __forceinline__ void ld_cs(const double* p, double (&v)[4]) {
    const double2 a = __ldcs(reinterpret_cast<const double2*>(p));
    const double2 b = __ldcs(reinterpret_cast<const double2*>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
  static __device__ __forceinline__ void ld_cg(const double* p, double (&v)[4]) {
    const double2 a = __ldcg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldcg(reinterpret_cast<const double2*>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
  static __device__ __forceinline__ void st(double* p, const double (&v)[4]) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
};

// ----------------------------------------------------------------- CGS2
// Pass kinds of the three-pass CGS2 (Algorithm 3, CGS2 procedure):
//   kGemvT:   h1 = Q^T w                                     (GEMVT)
//   kReorth:  w' = w - Q h1 (stored), h2 = Q^T w'            (GEMV + reorth GEMVT)
//   kFinal:   q_new = w' - Q h2, ||q_new||^2                 (reorth GEMV + norm)
//             then (last block) the Arnoldi column and the Givens update
//
// Each pass streams w and the k+1 basis columns once.  A thread takes a row
// group of V consecutive rows per grid-stride iteration and issues one
// 16/8/4-byte load per column for it before using any of them (KMAX x V
// values in registers), so a resident warp keeps k+2 coalesced loads in
// flight; it keeps only the k+1 accumulators across iterations.  Per-thread
// sums are in T; warp, block and grid sums in FP64.  The grid sum is
// deterministic: every block stores its partial sums, and the last block to
// finish (atomic ticket) adds them in block order.
enum PassKind { kGemvT = 0, kReorth = 1, kFinal = 2 };

// ------------------------------------------------------------ basis storage
// The Krylov basis is stored in the inner precision T, or -- FP32 inner solve
// only -- in BF16 or FP16 with one FP32 scale per vector: q_j = sigma_j u_j
// with u_j = q_j / max_i |q_ij| in [-1, 1], so FP16 can neither overflow nor
// flush a whole vector to zero.  Arithmetic on the basis is in T.
template <typename B>
__host__ __device__ constexpr bool basis_scaled() {
  return sizeof(B) == 2;
}
__device__ __forceinline__ float basis_to(float v) { return v; }
__device__ __forceinline__ double basis_to(double v) { return v; }
__device__ __forceinline__ float basis_to(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float basis_to(__half v) { return __half2float(v); }
template <typename B> __device__ __forceinline__ B basis_from(float v);
template <> __device__ __forceinline__ __nv_bfloat16 basis_from<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ __half basis_from<__half>(float v) {
  return __float2half_rn(v);
}

// Rows per thread per iteration: the basis values of a row group (KMAX x V
// elements of B) take at most 64 registers up to KMAX = 32 (FP64: 16), and
// one row group of a column is one 16-, 8-, 4- or 2-byte load.
template <typename B, int KMAX>
__host__ __device__ constexpr int pass_vec() {
  return sizeof(B) == 8   ? (KMAX <= 8 ? 2 : 1)
         : sizeof(B) == 4 ? (KMAX <= 16 ? 4 : KMAX <= 32 ? 2 : 1)
                          : (KMAX <= 16 ? 8 : KMAX <= 32 ? 4 : 2);
}
// Resident blocks per SM the register budget is sized for.
template <typename T, int KMAX>
__host__ __device__ constexpr int pass_min_blocks() {
  return (sizeof(T) == 4 ? KMAX <= 32 : KMAX <= 16) ? 2 : 1;
}

// V consecutive elements (V * sizeof(E) bytes, aligned to that size up to 16:
// storage rows come in multiples of 32), streaming loads / plain stores.
// FP32 and FP64 elements move as float/double vector types (moving them
// through integer vectors measured up to 2x slower for FP64 passes); 2-byte
// elements move as packed integers.
// Load policy: KEEP leaves the lines in L2 (a later pass reads them again),
// otherwise they stream (evict-first).
template <bool KEEP, typename P>
__device__ __forceinline__ P ld_policy(const P* p) {
  if constexpr (KEEP) return __ldcg(p);
  else return __ldcs(p);
}

template <typename E, int V, bool KEEP = false>
__device__ __forceinline__ void ld_group(const E* p, E (&v)[V]) {
  if constexpr (sizeof(E) == 8 && V == 1) {
    v[0] = ld_policy<KEEP>(p);
  } else if constexpr (sizeof(E) == 8) {
    static_assert(V % 2 == 0, "FP64 row groups of 1 or 2k elements");
#pragma unroll
    for (int i = 0; i < V / 2; ++i) {
      const double2 t = ld_policy<KEEP>(reinterpret_cast<const double2*>(p) + i);
      v[2 * i] = t.x;
      v[2 * i + 1] = t.y;
    }
  } else if constexpr (sizeof(E) == 4 && V % 4 == 0) {
#pragma unroll
    for (int i = 0; i < V / 4; ++i) {
      const float4 t = ld_policy<KEEP>(reinterpret_cast<const float4*>(p) + i);
      v[4 * i] = t.x;
      v[4 * i + 1] = t.y;
      v[4 * i + 2] = t.z;
      v[4 * i + 3] = t.w;
    }
  } else if constexpr (sizeof(E) == 4 && V == 2) {
    const float2 t = ld_policy<KEEP>(reinterpret_cast<const float2*>(p));
    v[0] = t.x;
    v[1] = t.y;
  } else if constexpr (sizeof(E) == 4) {
    static_assert(V == 1, "FP32 row groups of 1, 2 or 4k elements");
    v[0] = ld_policy<KEEP>(p);
  } else {
    static_assert(sizeof(E) == 2, "2-, 4- or 8-byte elements");
    constexpr int bytes = 2 * V;
    if constexpr (bytes % 16 == 0) {
#pragma unroll
      for (int i = 0; i < bytes / 16; ++i) {
        const uint4 t = ld_policy<KEEP>(reinterpret_cast<const uint4*>(p) + i);
        memcpy(reinterpret_cast<char*>(v) + 16 * i, &t, 16);
      }
    } else if constexpr (bytes == 8) {
      const uint2 t = ld_policy<KEEP>(reinterpret_cast<const uint2*>(p));
      memcpy(v, &t, 8);
    } else if constexpr (bytes == 4) {
      const unsigned t = ld_policy<KEEP>(reinterpret_cast<const unsigned*>(p));
      memcpy(v, &t, 4);
    } else {
      static_assert(bytes == 2, "2-byte row groups of 1, 2, 4 or 8k elements");
      const unsigned short t = ld_policy<KEEP>(reinterpret_cast<const unsigned short*>(p));
      memcpy(v, &t, 2);
    }
  }
}
template <typename E, int V>
__device__ __forceinline__ void st_group(E* p, const E (&v)[V]) {
  if constexpr (sizeof(E) == 8 && V == 1) {
    *p = v[0];
  } else if constexpr (sizeof(E) == 8) {
#pragma unroll
    for (int i = 0; i < V / 2; ++i)
      reinterpret_cast<double2*>(p)[i] = make_double2(v[2 * i], v[2 * i + 1]);
  } else if constexpr (sizeof(E) == 4 && V % 4 == 0) {
#pragma unroll
    for (int i = 0; i < V / 4; ++i)
      reinterpret_cast<float4*>(p)[i] =
          make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
  } else if constexpr (sizeof(E) == 4 && V == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  } else if constexpr (sizeof(E) == 4) {
    *p = v[0];
  } else {
    constexpr int bytes = 2 * V;
    if constexpr (bytes % 16 == 0) {
#pragma unroll
      for (int i = 0; i < bytes / 16; ++i) {
        uint4 t;
        memcpy(&t, reinterpret_cast<const char*>(v) + 16 * i, 16);
        reinterpret_cast<uint4*>(p)[i] = t;
      }
    } else if constexpr (bytes == 8) {
      uint2 t;
      memcpy(&t, v, 8);
      *reinterpret_cast<uint2*>(p) = t;
    } else if constexpr (bytes == 4) {
      unsigned t;
      memcpy(&t, v, 4);
      *reinterpret_cast<unsigned*>(p) = t;
    } else {
      unsigned short t;
      memcpy(&t, v, 2);
      *reinterpret_cast<unsigned short*>(p) = t;
    }
  }
}

// Block sums of acc[0..nred) (FP64), stored as this block's partials; the last
// block to arrive adds all blocks' partials in block order into sums[] (shared)
// and returns true.  With MAXLAST the last entry is a maximum instead of a
// sum (combined with max at every stage).  Every thread of the block must
// call it.
template <typename A, int KMAX, bool MAXLAST = false>
__device__ bool block_partials_last(const A (&acc)[KMAX], int nred, double* __restrict__ partials,
                                    unsigned int* counter, double* sums) {
  __shared__ double red[kWarps][KMAX];
  __shared__ double red2[kRedThreads];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < KMAX; ++j) {
    if (j < nred) {
      const bool mx = MAXLAST && j == nred - 1;
      const A v = mx ? warp_max(acc[j]) : warp_sum(acc[j]);
      if (lane == 0) red[warp][j] = (double)v;
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nred; j += kRedThreads) {
    const bool mx = MAXLAST && j == nred - 1;
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kWarps; ++q) s = mx ? fmax(s, red[q][j]) : s + red[q][j];
    partials[(long long)blockIdx.x * kPartStride + j] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return false;
  __threadfence();
  constexpr int groups = kRedThreads / KMAX;
  const int j = threadIdx.x % KMAX, grp = threadIdx.x / KMAX;
  const bool mx = MAXLAST && j == nred - 1;
  double s = 0.0;
  if (j < nred) {
    // blocks grp, grp + groups, ... in ascending order; 16 loads in flight
    // per thread, so the serial tail is a few L2 round trips
    constexpr int kBatch = 16;
    const int G = (int)gridDim.x;
    for (int b0 = grp; b0 < G; b0 += kBatch * groups) {
      double v[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int b = b0 + u * groups;
        v[u] = b < G ? __ldcg(partials + (long long)b * kPartStride + j) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < kBatch; ++u)
        if (b0 + u * groups < G) s = mx ? fmax(s, v[u]) : s + v[u];
    }
  }
  red2[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x < nred) {
    const bool mxj = MAXLAST && (int)threadIdx.x == nred - 1;
    double tsum = 0.0;
    for (int q = 0; q < groups; ++q) {
      const double v = red2[q * KMAX + threadIdx.x];
      tsum = mxj ? fmax(tsum, v) : tsum + v;
    }
    sums[threadIdx.x] = tsum;
  }
  if (threadIdx.x == 0) *counter = 0u;
  __syncthreads();
  return true;
}

// Arnoldi column and Givens update of Algorithm 3 for inner step k, in two
// parts.  The column is H[:,k] = h1 + h2 with H[k+1,k] = beta.  Applying the
// old rotations 0..k-1 to it touches rows 0..k only, so it needs h1 and h2
// but not beta: one warp of the final CGS2 pass does it while the pass
// streams (arnoldi_rotate_warp) and leaves the rotated column in H[0..k, k].
// Once beta = ||w''|| is known, the last block forms rotation k that zeroes
// H[k+1,k], updates t and rho = |t[k+1]| (arnoldi_givens_warp).  Same
// operations in the same order as applying everything at the end.  In graph
// mode the next step's IF node (handle `next`) is opened while the cycle
// stays active.
template <int KMAX>
__device__ void arnoldi_rotate_warp(int k, const double* __restrict__ h1,
                                    const double* __restrict__ h2, double* __restrict__ H,
                                    int ldh, const double* __restrict__ cs,
                                    const double* __restrict__ sn) {
  __shared__ double hs[KMAX + 1], css[KMAX], sns[KMAX];
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
  double* hc = H + (long long)k * ldh;
  for (int j = lane; j <= k; j += 32) hc[j] = hs[j];
}

__device__ void arnoldi_givens_warp(double beta, int k, double* __restrict__ H, int ldh,
                                    double* __restrict__ cs, double* __restrict__ sn,
                                    double* __restrict__ t, SolveState* st,
                                    unsigned long long next) {
  if ((threadIdx.x & 31) != 0) return;
  double* hc = H + (long long)k * ldh;
  st->beta = beta;
  bool go = false;
  if (!isfinite(beta)) {
    st->status = HPG_ERR_NAN;
    st->active = 0;
    hc[k + 1] = beta;
  } else {
    const double a = __ldcg(hc + k);   // H[k,k] after the old rotations
    const double mu = hypot(a, beta);
    if (!(mu > 0.0) || !isfinite(mu)) {
      st->status = isfinite(mu) ? HPG_ERR_BREAKDOWN : HPG_ERR_NAN;
      st->active = 0;
      hc[k + 1] = beta;
    } else {
      const double c = a / mu, sv = beta / mu;
      cs[k] = c;
      sn[k] = sv;
      hc[k] = mu;
      hc[k + 1] = 0.0;
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
  if (next) cudaGraphSetConditional(next, go ? 1u : 0u);
}

// One CGS2 pass (kind KIND) over the basis columns q_0..q_{ncol-1} stored as
// B (scaled by qscale[j] when B is a 2-byte format: the scales are folded into
// the coefficients and the results, so the inner loop only converts).
//   kGemvT:  h1 = Q^T w
//   kReorth: w' = w - Q h1, written over w in place (wout == w), h2 = Q^T w'
//   kFinal:  w'' = w' - Q h2 written to `wout` in T (a basis column when
//            B == T; w itself, in place, for a scaled basis, whose
//            quantisation needs max |w''| first), ||w''||^2 (and max |w''|),
//            then (last block) the Arnoldi column and the Givens update.
// Storing w' costs one vector write and saves the final pass a second GEMV
// (FP64 passes are close to the FP64 FMA rate of this GPU); the values are
// those of recomputing it (same operands, same order).
template <typename T, typename B, int KMAX, int KIND>
__global__ void __launch_bounds__(kRedThreads, (pass_min_blocks<T, KMAX>()))
cgs2_pass_kernel(const B* __restrict__ Q, long long ns, int ncol, const T* w,
                 const float* __restrict__ qscale, const double* __restrict__ h1,
                 const double* __restrict__ h2, T* wout, double* __restrict__ partials,
                 unsigned int* counter, double* __restrict__ out, double* __restrict__ H,
                 int ldh, double* __restrict__ cs, double* __restrict__ sn,
                 double* __restrict__ t, SolveState* st, unsigned long long next,
                 int zigzag) {
  constexpr int V = pass_vec<B, KMAX>();
  constexpr bool S = basis_scaled<B>();
  constexpr bool MAXLAST = S && KIND == kFinal;
  __shared__ T shc[KMAX];   // h1 (reorth) or h2 (final), scaled for a 2-byte basis
  __shared__ double sums[KMAX];
  pdl_trigger();
  pdl_wait();   // w, Q and h come from earlier kernels
  if (KIND != kGemvT) {
    const double* hc = KIND == kReorth ? h1 : h2;
    for (int j = threadIdx.x; j < ncol; j += kRedThreads)
      shc[j] = (T)(S ? ld_dep(hc + j) * (double)ld_dep(qscale + j) : ld_dep(hc + j));
    __syncthreads();
  }
  // the rotations that do not need beta, by one warp while the pass streams;
  // block 0 takes its ticket (and the last block reads H) only afterwards
  if (KIND == kFinal && blockIdx.x == 0 && threadIdx.x < 32)
    arnoldi_rotate_warp<KMAX>(ncol - 1, h1, h2, H, ldh, cs, sn);
  T acc[KMAX];
#pragma unroll
  for (int j = 0; j < KMAX; ++j) acc[j] = T(0);
  // Zig-zag over the passes (zigzag != 0, basis vectors much smaller than
  // L2): the reorth pass walks the rows backwards, so it starts on the rows
  // the GEMVT pass read last (still in L2), and the final pass forwards again;
  // the first two passes keep their lines in L2.  Measured on GB300: 0.8 %
  // faster 128^3 GMRES(30) solves; with 131 MB vectors (320^3) the backward
  // pass streamed at half the rate of a forward one.
  const bool rev = zigzag && KIND == kReorth;
  const bool keep = zigzag && KIND != kFinal;
  const long long ng = ns / V;
  const long long stride = (long long)gridDim.x * kRedThreads;
  auto load = [&](long long g, T (&wr)[V], B (&q)[KMAX][V]) {
    if (keep) {
      ld_group<T, V, true>(w + g * V, wr);
#pragma unroll
      for (int j = 0; j < KMAX; ++j)
        if (j < ncol) ld_group<B, V, true>(Q + j * ns + g * V, q[j]);
    } else {
      ld_group<T, V, false>(w + g * V, wr);
#pragma unroll
      for (int j = 0; j < KMAX; ++j)
        if (j < ncol) ld_group<B, V, false>(Q + j * ns + g * V, q[j]);
    }
  };
  for (long long gi = blockIdx.x * (long long)kRedThreads + threadIdx.x; gi < ng; gi += stride) {
    const long long g = rev ? ng - 1 - gi : gi;
    T wr[V];
    B q[KMAX][V];
    load(g, wr, q);
    const long long r0 = g * V;
    if (KIND == kGemvT) {
#pragma unroll
      for (int j = 0; j < KMAX; ++j)
        if (j < ncol) {
#pragma unroll
          for (int v = 0; v < V; ++v) acc[j] = fma((T)basis_to(q[j][v]), wr[v], acc[j]);
        }
    } else {
      // s = (Q c)_row, c = h1 or h2.  Rows always sum over j in ascending
      // order; for a 2-byte basis (8 rows per thread) the column-outer order
      // reads each coefficient from shared memory once per row group
      // (measured faster there, slower for FP32/FP64 rows).
      T sc[V];
#pragma unroll
      for (int v = 0; v < V; ++v) sc[v] = T(0);
      if constexpr (S) {
#pragma unroll
        for (int j = 0; j < KMAX; ++j)
          if (j < ncol) {
            const T c = shc[j];
#pragma unroll
            for (int v = 0; v < V; ++v) sc[v] = fma((T)basis_to(q[j][v]), c, sc[v]);
          }
      } else {
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
          for (int j = 0; j < KMAX; ++j)
            if (j < ncol) sc[v] = fma((T)basis_to(q[j][v]), shc[j], sc[v]);
      }
#pragma unroll
      for (int v = 0; v < V; ++v) wr[v] = wr[v] - sc[v];   // w' = w - Q h1 / w'' = w' - Q h2
      st_group<T, V>(wout + r0, wr);
      if (KIND == kReorth) {
#pragma unroll
        for (int j = 0; j < KMAX; ++j)
          if (j < ncol) {
#pragma unroll
            for (int v = 0; v < V; ++v) acc[j] = fma((T)basis_to(q[j][v]), wr[v], acc[j]);
          }
      } else {
#pragma unroll
        for (int v = 0; v < V; ++v) {
          acc[0] = fma(wr[v], wr[v], acc[0]);
          if (MAXLAST) acc[1] = fmax(acc[1], fabs(wr[v]));
        }
      }
    }
  }
  const int nred = KIND == kFinal ? (MAXLAST ? 2 : 1) : ncol;
  if (!block_partials_last<T, KMAX, MAXLAST>(acc, nred, partials, counter, sums)) return;
  if (KIND != kFinal) {
    for (int j = threadIdx.x; j < nred; j += kRedThreads)
      out[j] = S ? sums[j] * (double)ld_dep(qscale + j) : sums[j];
  } else if (threadIdx.x < 32) {
    if (MAXLAST && threadIdx.x == 0) st->wmax = sums[1];
    arnoldi_givens_warp(sqrt(sums[0]), ncol - 1, H, ldh, cs, sn, t, st, next);
  }
}

// The next V-cycle's first phase, done by the kernel that writes its input r:
// the first forward sweep from zero starts with colour 0, whose rows have no
// neighbour of a lower colour, so z_i = r_i / a_ii on the colour-0 block
// [0, c0_rows) (c0_rows = 0: not done).  Same division as the phase.
template <typename T>
__device__ __forceinline__ void first_phase4(long long i0, const T (&v)[4], T* __restrict__ z0,
                                             const T* __restrict__ diag, long long c0_rows) {
  if (i0 >= c0_rows) return;
  T d[4], zv[4];
  Vec4<T>::ld_cs(diag + i0, d);
#pragma unroll
  for (int r = 0; r < 4; ++r) zv[r] = v[r] / d[r];
  Vec4<T>::st(z0 + i0, zv);
}

// q_new /= beta (the Arnoldi normalisation), beta from the solve state.
template <typename T>
__global__ void __launch_bounds__(256)
arnoldi_scale_kernel(T* __restrict__ qnew, long long ns, const SolveState* st,
                     T* __restrict__ z0, const T* __restrict__ diag, long long c0_rows) {
  pdl_trigger();
  pdl_wait();
  // one FP64 division per block (FP64 throughput is low on this GPU)
  __shared__ T s_inv;
  __shared__ bool s_ok;
  if (threadIdx.x == 0) {
    const double beta = st->beta;
    s_ok = isfinite(beta) && beta > 0.0;
    s_inv = s_ok ? (T)(1.0 / beta) : T(0);
  }
  __syncthreads();
  if (!s_ok) return;
  const T inv = s_inv;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < (ns >> 2);
       g += stride) {
    T v[4];
    Vec4<T>::ld_cs(qnew + (g << 2), v);
#pragma unroll
    for (int r = 0; r < 4; ++r) v[r] = v[r] * inv;
    Vec4<T>::st(qnew + (g << 2), v);
    first_phase4<T>(g << 2, v, z0, diag, c0_rows);
  }
}

// Scaled basis: q_new = w'' / beta stored as u = w'' / max|w''| in B with
// sigma = max|w''| / beta, and the dequantised sigma * u in FP32 (the next
// V-cycle's input, so that it preconditions the vector the basis holds).
template <typename B>
__global__ void __launch_bounds__(256)
arnoldi_quantize_kernel(const float* __restrict__ wpp, long long ns, B* __restrict__ qnew,
                        float* __restrict__ qf, float* __restrict__ sigma_out,
                        const SolveState* st, float* __restrict__ z0,
                        const float* __restrict__ diag, long long c0_rows) {
  pdl_trigger();
  pdl_wait();
  __shared__ float s_inv_m, s_sigma;
  __shared__ bool s_ok;
  if (threadIdx.x == 0) {
    const double beta = st->beta, m = st->wmax;
    s_ok = isfinite(beta) && beta > 0.0 && m > 0.0;
    s_inv_m = s_ok ? (float)(1.0 / m) : 0.0f;
    s_sigma = s_ok ? (float)(m / beta) : 0.0f;
  }
  __syncthreads();
  if (!s_ok) return;
  const float inv_m = s_inv_m, sigma = s_sigma;
  if (blockIdx.x == 0 && threadIdx.x == 0) *sigma_out = sigma;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < (ns >> 2);
       g += stride) {
    float v[4];
    ld_group<float, 4>(wpp + (g << 2), v);
    B u[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      u[r] = basis_from<B>(v[r] * inv_m);
      v[r] = sigma * basis_to(u[r]);
    }
    st_group<B, 4>(qnew + (g << 2), u);
    st_group<float, 4>(qf + (g << 2), v);
    first_phase4<float>(g << 2, v, z0, diag, c0_rows);
  }
}

// y = H[:k,:k]^{-1} t[:k] (the dense TRSM of Algorithm 3), one warp,
// column-oriented back substitution.
__global__ void trsm_kernel(const double* __restrict__ H, int ldh, const double* __restrict__ t,
                            double* __restrict__ y, const SolveState* st) {
  pdl_trigger();
  pdl_wait();
  __shared__ double tt[kMaxRestart + 1];
  __shared__ double yi_s;
  const int k = st->k;
  for (int j = threadIdx.x; j < k; j += 32) tt[j] = ld_dep(t + j);
  __syncwarp();
  for (int i = k - 1; i >= 0; --i) {
    if (threadIdx.x == 0) {
      yi_s = tt[i] / ld_dep(H + (long long)i * ldh + i);
      y[i] = yi_s;
    }
    __syncwarp();
    const double yi = yi_s;
    for (int j = threadIdx.x; j < i; j += 32) tt[j] -= ld_dep(H + (long long)i * ldh + j) * yi;
    __syncwarp();
  }
}

// u = Q[:, :k] y (Algorithm 3, r <- Q t), k read from the solve state; a
// scaled basis folds sigma_j into y_j.
template <typename T, typename B>
__global__ void __launch_bounds__(256)
basis_combine_kernel(const B* __restrict__ Q, long long ns, const double* __restrict__ y,
                     const float* __restrict__ qscale, const SolveState* st,
                     T* __restrict__ u) {
  pdl_trigger();
  pdl_wait();
  __shared__ T ys[kMaxRestart + 1];
  const int k = st->k;
  for (int j = threadIdx.x; j < k; j += blockDim.x)
    ys[j] = (T)(basis_scaled<B>() ? ld_dep(y + j) * (double)ld_dep(qscale + j) : ld_dep(y + j));
  __syncthreads();
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= (ns >> 2)) return;
  T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll 4
  for (int j = 0; j < k; ++j) {
    B q[4];
    ld_group<B, 4>(Q + j * ns + (g << 2), q);
#pragma unroll
    for (int r = 0; r < 4; ++r) acc[r] = fma((T)basis_to(q[r]), ys[j], acc[r]);
  }
  st_group<T, 4>(u + (g << 2), acc);
}

// x += d (Algorithm 3, mixed-precision update: FP64 accumulation).
template <typename T>
__global__ void __launch_bounds__(256)
update_x_kernel(double* __restrict__ x, const T* __restrict__ d, long long ns) {
  pdl_trigger();
  pdl_wait();
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < ns) x[i] += (double)ld_dep(d + i);
}

// r = b - A x, ||r||^2 and max |r| (FP64; the maximum scales q_0 of a
// 2-byte basis).
__global__ void __launch_bounds__(kRedThreads)
residual_norm_kernel(const double* __restrict__ vals, const int* __restrict__ cols, long long ns,
                     const double* __restrict__ b, const double* __restrict__ x,
                     double* __restrict__ r, double* __restrict__ partials,
                     unsigned int* counter, double* __restrict__ out) {
  pdl_trigger();
  pdl_wait();
  double acc[2] = {0.0, 0.0};
  const long long stride = (long long)gridDim.x * kRedThreads;
  for (long long row = blockIdx.x * (long long)kRedThreads + threadIdx.x; row < ns;
       row += stride) {
    double v = ld_dep(b + row);
#pragma unroll
    for (int s = 0; s < kSlots; ++s) {
      const double a = ld_stream(vals + s * ns + row);
      const int c = ld_stream(cols + s * ns + row);
      v = fma(-a, ld_dep(x + c), v);
    }
    r[row] = v;
    acc[0] = fma(v, v, acc[0]);
    acc[1] = fmax(acc[1], fabs(v));
  }
  __shared__ double sums[2];
  if (block_partials_last<double, 2, true>(acc, 2, partials, counter, sums) && threadIdx.x < 2)
    out[threadIdx.x] = sums[threadIdx.x];
}

// ||v||^2 of an FP64 vector.
__global__ void __launch_bounds__(kRedThreads)
norm2_kernel(const double* __restrict__ v, long long ns, double* __restrict__ partials,
             unsigned int* counter, double* __restrict__ out) {
  pdl_trigger();
  pdl_wait();
  double acc[1] = {0.0};
  const long long stride = (long long)gridDim.x * kRedThreads;
  for (long long i = blockIdx.x * (long long)kRedThreads + threadIdx.x; i < ns; i += stride) {
    const double vi = ld_dep(v + i);
    acc[0] = fma(vi, vi, acc[0]);
  }
  __shared__ double sums[1];
  if (block_partials_last<double, 1>(acc, 1, partials, counter, sums) && threadIdx.x == 0)
    out[0] = sums[0];
}

// Outer convergence test of Algorithm 3 on the FP64 residual norm:
// ||r|| / ||b|| < tol ends the solve; so do a recorded breakdown / NaN and
// maxit.  In graph mode it sets the WHILE node's condition.
__global__ void outer_check_kernel(const double* __restrict__ rho2, SolveState* st,
                                   const unsigned* __restrict__ pipe_err, unsigned long long loop) {
  pdl_trigger();
  pdl_wait();
  if (threadIdx.x != 0) return;
  const double rho = sqrt(ld_dep(rho2));
  const double rel = rho / st->rho0;
  st->rho = rho;
  st->rel = rel;
  bool done = true;
  if (pipe_err && ld_dep(pipe_err) != 0) {
    st->status = HPG_ERR_TIMEOUT;   // a kernel's bounded wait gave up
  } else if (!isfinite(rel)) {
    st->status = HPG_ERR_NAN;
  } else if (rel < st->tol) {
    st->converged = 1;
  } else if (st->status != HPG_OK) {
  } else if (st->iters >= st->maxit) {
    st->status = HPG_ERR_NOT_CONVERGED;
  } else {
    done = false;
  }
  st->done = done ? 1 : 0;
  if (loop) cudaGraphSetConditional(loop, done ? 0u : 1u);
}

// Start of a restart cycle: q_0 = r / rho, t = rho e_1, k = 0; in graph mode
// opens step 0's IF node and closes the others.  A scaled basis stores
// u_0 = r / max|r| with sigma_0 = max|r| / rho and the dequantised q_0 in
// FP32 for the first V-cycle.
template <typename T, typename B>
__global__ void __launch_bounds__(256)
cycle_start_kernel(const double* __restrict__ r, long long ns, B* __restrict__ q0,
                   float* __restrict__ qf, float* __restrict__ qscale,
                   const double* __restrict__ rho2, double* __restrict__ t, SolveState* st,
                   const unsigned long long* __restrict__ handles, int nhandles,
                   T* __restrict__ z0, const T* __restrict__ diag, long long c0_rows) {
  pdl_trigger();
  pdl_wait();
  // the scalars once per block (one FP64 division each)
  __shared__ double s_inv;
  __shared__ float s_sigma;
  const double rho = st->rho;
  if (threadIdx.x == 0) {
    if constexpr (basis_scaled<B>()) {
      const double m = ld_dep(rho2 + 1);
      s_inv = m > 0.0 ? 1.0 / m : 0.0;
      s_sigma = (float)(m / rho);
    } else {
      s_inv = 1.0 / rho;
    }
  }
  __syncthreads();
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if constexpr (basis_scaled<B>()) {
    const double inv = s_inv;
    const float sigma = s_sigma;
    if (i < ns) {
      const B u = basis_from<B>((float)(ld_dep(r + i) * inv));
      q0[i] = u;
      const float v = sigma * basis_to(u);
      qf[i] = v;
      if (i < c0_rows) z0[i] = v / diag[i];   // the first V-cycle's first phase
    }
    if (i == 0) qscale[0] = sigma;
  } else {
    const double inv = s_inv;
    if (i < ns) {
      const T v = (T)(ld_dep(r + i) * inv);
      q0[i] = v;
      if (i < c0_rows) z0[i] = v / diag[i];   // the first V-cycle's first phase
    }
  }
  if (i == 0) {
    t[0] = rho;
    for (int j = 1; j <= st->m; ++j) t[j] = 0.0;
    st->k = 0;
    st->active = 1;
    st->restarts += 1;
    for (int j = 0; j < nhandles; ++j) cudaGraphSetConditional(handles[j], j == 0 ? 1u : 0u);
  }
}

// Busy-wait of a fixed number of clock cycles (bounded; no flag is waited
// on).  Profiled solves put one at the start of every inner step so that the
// host enqueues the step's launches before the device reaches them, and each
// event pair then brackets only its kernel.
__global__ void delay_kernel(long long cycles) {
  const long long t0 = clock64();
  long long spins = 0;
  while (clock64() - t0 < cycles && spins < (1LL << 40)) ++spins;
}

// ----------------------------------------------------------------- launchers
template <typename T> constexpr int prec_of() { return sizeof(T) == 8 ? HPG_FP64 : HPG_FP32; }

// Basis vectors up to this size take the zig-zag pass order (cgs2_pass_kernel).
constexpr long long kZigZagVectorBytes = 32LL << 20;

// Grid of a CGS2 pass: every resident block of the instantiation (one wave
// of grid-stride blocks), at most the G blocks the partials are sized for.
template <typename T, typename B, int KMAX, int KIND>
static int pass_grid(hpg_problem* h) {
  static int per_sm = 0;
  if (per_sm == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, cgs2_pass_kernel<T, B, KMAX, KIND>, kRedThreads, 0) != cudaSuccess ||
        per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
  }
  const int g = per_sm * h->num_sms;
  return g < h->ws->G ? g : h->ws->G;
}

template <typename T, typename B, int KMAX, int KIND>
static cudaError_t enqueue_pass(hpg_problem* h, const B* Q, long long ns, int ncol, const T* w,
                                T* wout, double* out, unsigned long long next, cudaStream_t s) {
  Workspace* ws = h->ws;
  return kl(h, cgs2_pass_kernel<T, B, KMAX, KIND>, pass_grid<T, B, KMAX, KIND>(h), kRedThreads,
            s, Q, ns, ncol, w, (const float*)ws->qscale, (const double*)ws->h1,
            (const double*)ws->h2, wout, ws->partials, ws->counter, out, ws->H, ws->m + 1,
            ws->cs, ws->sn, ws->t, ws->st, next,
            ns * (long long)sizeof(B) <= kZigZagVectorBytes ? 1 : 0);
}

// One CGS2 pass over q_0..q_{ncol-1} (k = ncol - 1); the final pass also
// forms the Arnoldi column and the Givens update and opens `next`.
template <typename T, typename B, int KIND>
static int launch_pass(hpg_problem* h, const B* Q, long long ns, int ncol, const T* w, T* wout,
                       double* out, unsigned long long next, cudaStream_t s) {
  static const int cls[3] = {K_CGS2_GEMVT, K_CGS2_REORTH, K_CGS2_FINAL};
  // Q columns + w (+ the w' / w'' write)
  const double bytes = (double)h->lev[0].n *
                       (ncol * (double)sizeof(B) + (KIND == kGemvT ? 1.0 : 2.0) * sizeof(T));
  return launch(h, cls[KIND], 0, prec_of<T>(), bytes, s, "cgs2_pass_kernel", [&] {
    if (ncol <= 8) return enqueue_pass<T, B, 8, KIND>(h, Q, ns, ncol, w, wout, out, next, s);
    if (ncol <= 16)
      return enqueue_pass<T, B, 16, KIND>(h, Q, ns, ncol, w, wout, out, next, s);
    if (ncol <= 32)
      return enqueue_pass<T, B, 32, KIND>(h, Q, ns, ncol, w, wout, out, next, s);
    return enqueue_pass<T, B, 64, KIND>(h, Q, ns, ncol, w, wout, out, next, s);
  });
}

// Rows [0, first_phase_rows) of level 0 (its colour-0 block) whose first
// V-cycle phase the kernel producing the V-cycle's input writes along with
// it; 0 when the V-cycle does not start with a sweep from zero there.
static long long first_phase_rows(const hpg_problem* h) {
  return (h->pre >= 1 || h->nlev == 1) ? h->lev[0].g.off[1] : 0;
}
template <typename T> static const T* level0_diag(const hpg_problem* h);
template <> const float* level0_diag<float>(const hpg_problem* h) {
  return h->lev[0].v32 + kCentre * h->lev[0].g.n_store;
}
template <> const double* level0_diag<double>(const hpg_problem* h) {
  return h->lev[0].v64 + kCentre * h->lev[0].g.n_store;
}

// One inner step k (0-based): z = M^{-1} q_k, w = A z, CGS2 against
// q_0..q_k, q_{k+1} = w / ||w||, Givens update; `next` opens step k+1.
// A scaled basis preconditions the dequantised q_k (qf) and quantises
// q_{k+1} after the norm and max of w'' are known.
template <typename T, typename B>
static int enqueue_step(hpg_problem* h, int k, hpg_prec prec, unsigned long long next,
                        cudaStream_t s) {
  Workspace* ws = h->ws;
  const long long ns = h->lev[0].g.n_store;
  B* Q = (B*)ws->Q;
  T* z = (T*)ws->z;
  T* w = (T*)ws->w;
  constexpr bool S = basis_scaled<B>();
  const void* r_in;
  if constexpr (S) r_in = ws->qf;
  else r_in = Q + (long long)k * ns;
  int rc;
  // colour 0 of the V-cycle's first sweep came with r_in (first_phase_rows)
  if ((rc = run_vcycle(h, 0, prec, r_in, z, s, first_phase_rows(h) > 0))) return rc;
  if ((rc = launch_spmv(h, 0, prec, z, w, s))) return rc;
  const int ncol = k + 1;
  B* qnew = Q + (long long)(k + 1) * ns;
  T* wout;
  if constexpr (S) wout = w;   // w'' in place, quantised below
  else wout = qnew;
  if ((rc = launch_pass<T, B, kGemvT>(h, Q, ns, ncol, w, nullptr, ws->h1, 0ULL, s))) return rc;
  if ((rc = launch_pass<T, B, kReorth>(h, Q, ns, ncol, w, w, ws->h2, 0ULL, s))) return rc;
  if ((rc = launch_pass<T, B, kFinal>(h, Q, ns, ncol, w, wout, nullptr, next, s))) return rc;
  if constexpr (S) {
    return launch(h, K_ARNOLDI_SCALE, 0, prec_of<T>(),
                  h->lev[0].n * (2.0 * sizeof(T) + sizeof(B)), s, "arnoldi_quantize_kernel",
                  [&] {
                    return kl(h, arnoldi_quantize_kernel<B>, grid_for(ns / 4, 256), 256, s,
                              (const float*)w, ns, qnew, ws->qf, ws->qscale + k + 1,
                              (const SolveState*)ws->st, (float*)z, level0_diag<float>(h),
                              first_phase_rows(h));
                  });
  } else {
    return launch(h, K_ARNOLDI_SCALE, 0, prec_of<T>(), 2.0 * h->lev[0].n * sizeof(T), s,
                  "arnoldi_scale_kernel", [&] {
                    return kl(h, arnoldi_scale_kernel<T>, grid_for(ns / 4, 256), 256, s, qnew,
                              ns, (const SolveState*)ws->st, z, level0_diag<T>(h),
                              first_phase_rows(h));
                  });
  }
}

// End of a cycle: y = H^{-1} t, u = Q y, d = M^{-1} u, x += d.
template <typename T, typename B>
static int enqueue_cycle_update(hpg_problem* h, hpg_prec prec, int k_model, cudaStream_t s) {
  Workspace* ws = h->ws;
  const long long ns = h->lev[0].g.n_store;
  const double n = (double)h->lev[0].n;
  int rc;
  rc = launch(h, K_TRSM, 0, HPG_FP64, 0.0, s, "trsm_kernel", [&] {
    return kl(h, trsm_kernel, 1, 32, s, (const double*)ws->H, ws->m + 1, (const double*)ws->t,
              ws->y, (const SolveState*)ws->st);
  });
  if (rc) return rc;
  rc = launch(h, K_COMBINE, 0, prec_of<T>(), n * (k_model * (double)sizeof(B) + sizeof(T)), s,
              "basis_combine_kernel", [&] {
                return kl(h, basis_combine_kernel<T, B>, grid_for(ns / 4, 256), 256, s,
                          (const B*)ws->Q, ns, (const double*)ws->y,
                          (const float*)ws->qscale, (const SolveState*)ws->st, (T*)ws->u);
              });
  if (rc) return rc;
  if ((rc = run_vcycle(h, 0, prec, ws->u, ws->z, s))) return rc;
  return launch(h, K_UPDATE_X, 0, HPG_FP64, n * (16.0 + sizeof(T)), s, "update_x_kernel", [&] {
    return kl(h, update_x_kernel<T>, grid_for(ns, 256), 256, s, ws->x, (const T*)ws->z, ns);
  });
}

// r = b - A x, ||r||, outer test (sets `loop` in graph mode).
static int enqueue_outer(hpg_problem* h, unsigned long long loop, cudaStream_t s) {
  Workspace* ws = h->ws;
  const Level& L = h->lev[0];
  const long long ns = L.g.n_store;
  int rc = launch(h, K_RESIDUAL, 0, HPG_FP64, L.n * (27.0 * 12.0 + 3.0 * 8.0), s,
                  "residual_norm_kernel", [&] {
                    return kl(h, residual_norm_kernel, ws->G, kRedThreads, s,
                              (const double*)L.v64, (const int*)L.cols, ns,
                              (const double*)ws->b, (const double*)ws->x, ws->r, ws->partials,
                              ws->counter, ws->rho2);
                  });
  if (rc) return rc;
  return launch(h, K_NORM, 0, HPG_FP64, 0.0, s, "outer_check_kernel", [&] {
    return kl(h, outer_check_kernel, 1, 32, s, (const double*)ws->rho2, ws->st,
              (const unsigned*)h->pipe_err, loop);
  });
}

template <typename T, typename B>
static int enqueue_cycle_start(hpg_problem* h, const unsigned long long* handles, int nh,
                               cudaStream_t s) {
  Workspace* ws = h->ws;
  const long long ns = h->lev[0].g.n_store;
  const double row_bytes = 8.0 + sizeof(B) + (basis_scaled<B>() ? sizeof(float) : 0.0);
  return launch(h, K_CYCLE_START, 0, prec_of<T>(), h->lev[0].n * row_bytes, s,
                "cycle_start_kernel", [&] {
                  return kl(h, cycle_start_kernel<T, B>, grid_for(ns, 256), 256, s,
                            (const double*)ws->r, ns, (B*)ws->Q, ws->qf, ws->qscale,
                            (const double*)ws->rho2, ws->t, ws->st, handles, nh, (T*)ws->z,
                            level0_diag<T>(h), first_phase_rows(h));
                });
}

static int read_state(hpg_problem* h, cudaStream_t s) {
  Workspace* ws = h->ws;
  HPG_CK(cudaMemcpyAsync(ws->st_host, ws->st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
  HPG_CK(cudaStreamSynchronize(s));
  h->pdl_next = false;
  return HPG_OK;
}

// ------------------------------------------------------------- graph capture
// Appends a conditional node (IF or WHILE on `handle`) to the graph being
// captured on stream s and returns its body graph; later captured work on s
// depends on the conditional node.
static int append_conditional(hpg_problem* h, cudaStream_t s, cudaGraphConditionalHandle handle,
                              cudaGraphConditionalNodeType type, cudaGraph_t* body) {
  cudaStreamCaptureStatus cst;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edges = nullptr;
  size_t nd = 0;
  HPG_CK(cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, &deps, &edges, &nd));
  if (cst != cudaStreamCaptureStatusActive) {
    set_error("append_conditional: stream is not capturing");
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

// Captures the whole GMRES-IR solve (everything after b, x and rho0 are in
// place) as one graph:
//   outer residual + test -> WHILE(not done) {
//     cycle start -> IF(h_0){step 0} -> ... -> IF(h_{m-1}){step m-1}
//     -> TRSM, Q y, V-cycle, x += d -> outer residual + test }
// Each step's Givens kernel opens the next step's IF node while the cycle
// continues, so converged cycles skip the remaining steps on the device.
template <typename T, typename B>
static int capture_solve_graph(hpg_problem* h, int m, hpg_prec prec) {
  Workspace* ws = h->ws;
  if (ws->exec && ws->graph_m == m && ws->graph_prec == prec && ws->graph_basis == ws->basis)
    return HPG_OK;
  if (ws->exec) cudaGraphExecDestroy(ws->exec);
  if (ws->graph) cudaGraphDestroy(ws->graph);
  ws->exec = nullptr;
  ws->graph = nullptr;
  cudaGraph_t g;
  HPG_CK(cudaGraphCreate(&g, 0));
  ws->graph = g;
  cudaGraphConditionalHandle loop;
  HPG_CK(cudaGraphConditionalHandleCreate(&loop, g, 0, 0));
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
  int rc = HPG_OK;
  cudaStream_t s0 = ws->cap[0], s1 = ws->cap[1], s2 = ws->cap[2];
  cudaGraph_t body = nullptr;
  const long long launches_before = h->launches;
  HPG_CK(cudaStreamBeginCaptureToGraph(s0, g, nullptr, nullptr, 0, mode));
  h->pdl_next = false;
  long long mark = h->launches;
  rc = enqueue_outer(h, (unsigned long long)loop, s0);
  ws->n_outer = h->launches - mark;
  if (rc == HPG_OK) rc = append_conditional(h, s0, loop, cudaGraphCondTypeWhile, &body);
  cudaGraph_t g_end = nullptr;
  cudaError_t e = cudaStreamEndCapture(s0, &g_end);
  if (rc || e != cudaSuccess) {
    ws->graph = nullptr;   // a failed capture's graph is abandoned, not destroyed
    return rc ? rc : cuda_fail(e, "cudaStreamEndCapture(main)", __FILE__, __LINE__);
  }
  // WHILE body
  std::vector<cudaGraphConditionalHandle> hk(m);
  for (int k = 0; k < m; ++k) HPG_CK(cudaGraphConditionalHandleCreate(&hk[k], body, 0, 0));
  HPG_CK(cudaMemcpy(ws->hk, hk.data(), sizeof(unsigned long long) * m, cudaMemcpyHostToDevice));
  HPG_CK(cudaStreamBeginCaptureToGraph(s1, body, nullptr, nullptr, 0, mode));
  h->pdl_next = false;
  mark = h->launches;
  rc = enqueue_cycle_start<T, B>(h, ws->hk, m, s1);
  ws->n_start = h->launches - mark;
  for (int k = 0; k < m && rc == HPG_OK; ++k) {
    cudaGraph_t sb = nullptr;
    rc = append_conditional(h, s1, hk[k], cudaGraphCondTypeIf, &sb);
    if (rc) break;
    e = cudaStreamBeginCaptureToGraph(s2, sb, nullptr, nullptr, 0, mode);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "cudaStreamBeginCaptureToGraph(step)", __FILE__, __LINE__);
      break;
    }
    h->pdl_next = false;
    mark = h->launches;
    rc = enqueue_step<T, B>(h, k, prec, k + 1 < m ? (unsigned long long)hk[k + 1] : 0ULL, s2);
    ws->n_step = h->launches - mark;
    cudaGraph_t sb_end = nullptr;
    e = cudaStreamEndCapture(s2, &sb_end);
    if (rc == HPG_OK && e != cudaSuccess)
      rc = cuda_fail(e, "cudaStreamEndCapture(step)", __FILE__, __LINE__);
  }
  mark = h->launches;
  if (rc == HPG_OK) rc = enqueue_cycle_update<T, B>(h, prec, m / 2, s1);
  ws->n_update = h->launches - mark;
  if (rc == HPG_OK) rc = enqueue_outer(h, (unsigned long long)loop, s1);
  h->launches = launches_before;   // capture enqueues nothing that runs
  cudaGraph_t body_end = nullptr;
  e = cudaStreamEndCapture(s1, &body_end);
  if (rc || e != cudaSuccess) {
    ws->graph = nullptr;   // a failed capture's graph is abandoned, not destroyed
    return rc ? rc : cuda_fail(e, "cudaStreamEndCapture(body)", __FILE__, __LINE__);
  }
  e = cudaGraphInstantiate(&ws->exec, g, 0);
  if (e != cudaSuccess) {
    ws->exec = nullptr;
    return cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
  }
  size_t nn = 0;
  cudaGraphGetNodes(g, nullptr, &nn);
  ws->graph_nodes = (int)nn;
  ws->graph_m = m;
  ws->graph_prec = prec;
  ws->graph_basis = ws->basis;
  h->pdl_next = false;
  return HPG_OK;
}

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T, typename B>
static int solve_t(hpg_problem* h, const double* b, double* x, double tol, int m, int maxit,
                   hpg_prec prec, hpg_prec basis, hpg_solve_info* info, cudaStream_t s) {
  int rc;
  if ((rc = ensure_workspace(h, m, prec, basis))) return rc;
  Workspace* ws = h->ws;
  const Level& L = h->lev[0];
  const long long ns = L.g.n_store, n = L.n;
  const long long launches0 = h->launches;
  h->pdl_next = false;
  // inputs to storage order (host buffers staged through device memory)
  const double* b_dev = b;
  const double* x_dev = x;
  const bool b_host = !is_device_ptr(b), x_host = !is_device_ptr(x);
  if (b_host) {
    HPG_CK(cudaMemcpyAsync(ws->stage, b, 8 * n, cudaMemcpyHostToDevice, s));
    b_dev = ws->stage;
  }
  if (x_host) {
    HPG_CK(cudaMemcpyAsync(ws->stage + n, x, 8 * n, cudaMemcpyHostToDevice, s));
    x_dev = ws->stage + n;
  }
  h->pdl_next = false;
  if ((rc = launch_permute(h, 0, 0, HPG_FP64, b_dev, HPG_FP64, ws->b, s))) return rc;
  if ((rc = launch_permute(h, 0, 0, HPG_FP64, x_dev, HPG_FP64, ws->x, s))) return rc;
  rc = launch(h, K_NORM, 0, HPG_FP64, 8.0 * n, s, "norm2_kernel", [&] {
    return kl(h, norm2_kernel, ws->G, kRedThreads, s, (const double*)ws->b, ns, ws->partials,
              ws->counter, ws->h1);
  });
  if (rc) return rc;
  double rho0_sq = 0.0;
  HPG_CK(cudaMemcpyAsync(&rho0_sq, ws->h1, 8, cudaMemcpyDeviceToHost, s));
  HPG_CK(cudaStreamSynchronize(s));
  h->pdl_next = false;
  const double rho0 = sqrt(rho0_sq);
  SolveState init;
  memset(&init, 0, sizeof(init));
  init.tol = tol;
  init.maxit = maxit;
  init.m = m;
  init.status = HPG_OK;
  init.rho0 = rho0;
  int status = HPG_OK;
  bool converged = false;
  int graph_launches = 0;
  const bool use_graph = !h->profiling && !h->eager;
  if (!(rho0 == rho0) || isinf(rho0)) {
    status = HPG_ERR_NAN;
    *ws->st_host = init;
  } else if (rho0 == 0.0) {
    // b = 0: the solution is x = 0
    HPG_CK(cudaMemsetAsync(ws->x, 0, 8 * ns, s));
    converged = true;
    *ws->st_host = init;
  } else {
    *ws->st_host = init;
    HPG_CK(cudaMemcpyAsync(ws->st, ws->st_host, sizeof(SolveState), cudaMemcpyHostToDevice, s));
    h->pdl_next = false;
    if (use_graph) {
      if ((rc = capture_solve_graph<T, B>(h, m, prec))) return rc;
      HPG_CK(cudaGraphLaunch(ws->exec, s));
      graph_launches = 1;
      h->pdl_next = false;
      if ((rc = read_state(h, s))) return rc;
    } else {
      // eager mode (profiling): the same sequence driven from the host
      if ((rc = enqueue_outer(h, 0ULL, s))) return rc;
      if ((rc = read_state(h, s))) return rc;
      while (!ws->st_host->done) {
        if ((rc = enqueue_cycle_start<T, B>(h, nullptr, 0, s))) return rc;
        for (int k = 0; k < m; ++k) {
          if (h->profiling) {
            // instrumentation only: not counted with the solve's kernels
            HPG_CK(kl(h, delay_kernel, 1, 32, s, 4000000LL));
            h->pdl_next = false;
          }
          if ((rc = enqueue_step<T, B>(h, k, prec, 0ULL, s))) return rc;
          if ((rc = read_state(h, s))) return rc;
          if (!ws->st_host->active) break;
        }
        if ((rc = enqueue_cycle_update<T, B>(h, prec, ws->st_host->k, s))) return rc;
        if ((rc = enqueue_outer(h, 0ULL, s))) return rc;
        if ((rc = read_state(h, s))) return rc;
      }
    }
    converged = ws->st_host->converged != 0;
    status = converged ? HPG_OK : ws->st_host->status;
    if (!converged && status == HPG_OK) status = HPG_ERR_NOT_CONVERGED;
  }
  // solution back to natural order (and to the host buffer if needed)
  double* x_out = x_host ? ws->stage + n : x;
  h->pdl_next = false;
  if ((rc = launch_permute(h, 0, 1, HPG_FP64, ws->x, HPG_FP64, x_out, s))) return rc;
  if (x_host) HPG_CK(cudaMemcpyAsync(x, x_out, 8 * n, cudaMemcpyDeviceToHost, s));
  HPG_CK(cudaStreamSynchronize(s));
  h->pdl_next = false;
  const SolveState& fs = *ws->st_host;
  if (fs.status == HPG_ERR_TIMEOUT) {
    if (h->pipe_err) HPG_CK(cudaMemset(h->pipe_err, 0, sizeof(unsigned) * 4));
    status = HPG_ERR_TIMEOUT;
    converged = false;
  }
  if (info) {
    info->iterations = fs.iters;
    info->restarts = fs.restarts;
    info->converged = converged ? 1 : 0;
    info->status = status;
    info->rel_residual = converged && rho0 == 0.0 ? 0.0 : fs.rel;
    info->rho0 = rho0;
    long long kl_count = h->launches - launches0;
    if (graph_launches) {
      // kernels the device ran inside the graph: the outer test once more
      // than the cycles, cycle start and update per cycle, one step body per
      // inner iteration (skipped IF bodies launch nothing)
      kl_count += (long long)(fs.restarts + 1) * ws->n_outer +
                  (long long)fs.restarts * (ws->n_start + ws->n_update) +
                  (long long)fs.iters * ws->n_step;
    }
    info->kernel_launches = (int)kl_count;
    info->graph_launches = graph_launches;
  }
  if (status != HPG_OK) set_error("hpg_gmres_ir_solve: %s after %d iterations (rel %g)",
                                  hpg_status_string(status), fs.iters, fs.rel);
  return status;
}

}  // namespace hpg

using namespace hpg;

extern "C" {

HPG_API int hpg_set_execution(hpg_problem_t* h, int mode) {
  if (!h || (mode != HPG_EXEC_GRAPH && mode != HPG_EXEC_EAGER)) {
    set_error("hpg_set_execution: invalid handle or mode %d", mode);
    return HPG_ERR_INVALID;
  }
  h->eager = mode == HPG_EXEC_EAGER;
  return HPG_OK;
}

HPG_API int hpg_gmres_ir_solve(hpg_problem_t* h, const double* b, double* x, double tol,
                               int restart, int maxit, hpg_prec inner, hpg_prec basis,
                               hpg_solve_info* info, void* stream) {
  if (info) memset(info, 0, sizeof(*info));
  if (!h || !b || !x || !(tol > 0.0) || restart < 1 || restart > kMaxRestart || maxit < 0) {
    set_error("hpg_gmres_ir_solve: invalid argument (tol %g, restart %d, maxit %d)", tol,
              restart, maxit);
    if (info) info->status = HPG_ERR_INVALID;
    return HPG_ERR_INVALID;
  }
  if (!h->hierarchy) {
    set_error("hpg_gmres_ir_solve: call hpg_build_mg_hierarchy first");
    if (info) info->status = HPG_ERR_STATE;
    return HPG_ERR_STATE;
  }
  const bool ok = (inner == HPG_FP64 && basis == HPG_FP64) ||
                  (inner == HPG_FP32 &&
                   (basis == HPG_FP32 || basis == HPG_BF16 || basis == HPG_FP16));
  if (!ok) {
    set_error("hpg_gmres_ir_solve: inner %d / basis %d not supported (FP64/FP64, or FP32 inner "
              "with an FP32, BF16 or FP16 basis)",
              (int)inner, (int)basis);
    if (info) info->status = HPG_ERR_UNSUPPORTED;
    return HPG_ERR_UNSUPPORTED;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (inner == HPG_FP64)
    return solve_t<double, double>(h, b, x, tol, restart, maxit, inner, basis, info, s);
  if (basis == HPG_BF16)
    return solve_t<float, __nv_bfloat16>(h, b, x, tol, restart, maxit, inner, basis, info, s);
  if (basis == HPG_FP16)
    return solve_t<float, __half>(h, b, x, tol, restart, maxit, inner, basis, info, s);
  return solve_t<float, float>(h, b, x, tol, restart, maxit, inner, basis, info, s);
}

}  // extern "C"
