// GMRES-IR (Algorithm 3): CGS2 orthogonalisation as tall-skinny GEMV passes
// with deterministic two-stage reductions, the Arnoldi normalisation fused
// with the Givens update of the Hessenberg QR, the dense triangular solve, the
// solution update and the FP64 outer residual, driven by a host loop.
//
// Precision (Algorithm 3: blue steps may be low precision): the basis Q, the
// preconditioned vector z and w = A z are in the inner precision T with
// per-thread accumulation in T; block and global sums, H, the rotations, t, y,
// the outer residual, its norm and x are FP64.

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
  int status;     // HPG_OK, HPG_ERR_BREAKDOWN or HPG_ERR_NAN
};

struct Workspace {
  int m = 0;              // restart capacity
  hpg_prec prec = HPG_FP32;
  int G = 0;              // blocks of the reduction kernels
  void* Q = nullptr;      // [m+1][ns] basis
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
  SolveState* st = nullptr;      // device
  SolveState* st_host = nullptr; // pinned mirror
};

void destroy_workspace(hpg_problem* h) {
  Workspace* ws = h->ws;
  if (!ws) return;
  void* ptrs[] = {ws->Q, ws->z, ws->w, ws->u, ws->b, ws->x, ws->r, ws->stage, ws->partials,
                  ws->counter, ws->h1, ws->h2, ws->H, ws->cs, ws->sn, ws->t, ws->y, ws->st};
  for (void* p : ptrs) dev_free(p);
  if (ws->st_host) cudaFreeHost(ws->st_host);
  delete ws;
  h->ws = nullptr;
}

static int ensure_workspace(hpg_problem* h, int m, hpg_prec prec) {
  if (h->ws && h->ws->m >= m && h->ws->prec == prec) return HPG_OK;
  destroy_workspace(h);
  Workspace* ws = new Workspace();
  h->ws = ws;
  const Level& L = h->lev[0];
  const long long ns = L.g.n_store;
  const size_t es = prec_size(prec);
  ws->m = m;
  ws->prec = prec;
  long long g = (ns + kRedThreads - 1) / kRedThreads;
  ws->G = (int)(g < 2LL * h->num_sms ? g : 2LL * h->num_sms);
  if (ws->G < 1) ws->G = 1;
  int rc = HPG_OK;
  rc = rc ? rc : dev_alloc(&ws->Q, es * ns * (m + 1));
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

// Reduces acc[0..nred) over the block into partials[blockIdx.x][.] and, when
// `out` is given, lets the last block to finish sum the partials of all blocks
// in a fixed order into out[0..nred).  Deterministic for a fixed grid.
template <typename A, int KMAX>
__device__ void block_reduce(const A (&acc)[KMAX], int nred, double* __restrict__ partials,
                             unsigned int* counter, double* __restrict__ out) {
  __shared__ double red[kWarps][KMAX];
  __shared__ double red2[kRedThreads];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < KMAX; ++j) {
    if (j < nred) {
      const A v = warp_sum(acc[j]);
      if (lane == 0) red[warp][j] = (double)v;
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nred; j += kRedThreads) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kWarps; ++q) s += red[q][j];
    partials[(long long)blockIdx.x * kPartStride + j] = s;
  }
  if (!out) return;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  constexpr int groups = kRedThreads / KMAX;
  const int j = threadIdx.x % KMAX, grp = threadIdx.x / KMAX;
  double s = 0.0;
  if (j < nred)
    for (int b = grp; b < (int)gridDim.x; b += groups)
      s += __ldcg(partials + (long long)b * kPartStride + j);
  red2[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x < nred) {
    double tsum = 0.0;
    for (int q = 0; q < groups; ++q) tsum += red2[q * KMAX + threadIdx.x];
    out[threadIdx.x] = tsum;
  }
  if (threadIdx.x == 0) *counter = 0u;
}

// ----------------------------------------------------------------- CGS2
// Pass kinds of the three-pass CGS2 (Algorithm 3, CGS2 procedure):
//   kGemvT:   h1 = Q^T w                                    (GEMVT)
//   kReorth:  h2 = Q^T (w - Q h1)                           (GEMV + reorth GEMVT)
//   kFinal:   q_new = (w - Q h1) - Q h2, partial ||q_new||^2 (reorth GEMV + norm)
// The GEMV w - Q h1 is recomputed row-locally in the last pass (same code, same
// rounding) instead of being stored.
enum PassKind { kGemvT = 0, kReorth = 1, kFinal = 2 };

template <typename T, int KMAX, int KIND>
__global__ void __launch_bounds__(kRedThreads)
cgs2_pass_kernel(const T* __restrict__ Q, long long ns, int ncol, const T* __restrict__ w,
                 const double* __restrict__ h1, const double* __restrict__ h2,
                 T* __restrict__ qnew, double* __restrict__ partials, unsigned int* counter,
                 double* __restrict__ out) {
  __shared__ T sh1[KMAX], sh2[KMAX];
  if (KIND != kGemvT) {
    for (int j = threadIdx.x; j < ncol; j += kRedThreads) {
      sh1[j] = (T)h1[j];
      if (KIND == kFinal) sh2[j] = (T)h2[j];
    }
    __syncthreads();
  }
  T acc[KMAX];
#pragma unroll
  for (int j = 0; j < KMAX; ++j) acc[j] = T(0);
  const long long stride = (long long)gridDim.x * kRedThreads;
  for (long long i = blockIdx.x * (long long)kRedThreads + threadIdx.x; i < ns; i += stride) {
    T wi = w[i];
    if (KIND == kGemvT) {
#pragma unroll
      for (int j = 0; j < KMAX; ++j)
        if (j < ncol) acc[j] = fma(__ldcs(Q + j * ns + i), wi, acc[j]);
    } else {
      T q[KMAX];
      T s = T(0);
#pragma unroll
      for (int j = 0; j < KMAX; ++j)
        if (j < ncol) {
          q[j] = __ldcs(Q + j * ns + i);
          s = fma(q[j], sh1[j], s);
        }
      wi = wi - s;  // w - Q h1
      if (KIND == kReorth) {
#pragma unroll
        for (int j = 0; j < KMAX; ++j)
          if (j < ncol) acc[j] = fma(q[j], wi, acc[j]);
      } else {
        T s2 = T(0);
#pragma unroll
        for (int j = 0; j < KMAX; ++j)
          if (j < ncol) s2 = fma(q[j], sh2[j], s2);
        wi = wi - s2;  // (w - Q h1) - Q h2
        qnew[i] = wi;
        acc[0] = fma(wi, wi, acc[0]);
      }
    }
  }
  block_reduce<T, KMAX>(acc, KIND == kFinal ? 1 : ncol, partials, counter, out);
}

// beta = ||q_new||, q_new /= beta over all rows, and (block 0) the Arnoldi
// column H[:,k] = h1 + h2, H[k+1,k] = beta followed by the Givens update of
// Algorithm 3: rotations 0..k-1 applied to column k, rotation k formed to
// zero H[k+1,k], t updated, rho = |t[k+1]|.
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
arnoldi_finish_kernel(T* __restrict__ qnew, long long ns, const double* __restrict__ partials,
                      int nparts, int k, const double* __restrict__ h1,
                      const double* __restrict__ h2, double* __restrict__ H, int ldh,
                      double* __restrict__ cs, double* __restrict__ sn, double* __restrict__ t,
                      SolveState* st) {
  __shared__ double red[kRedThreads];
  double s = 0.0;
  for (int b = threadIdx.x; b < nparts; b += kRedThreads) s += partials[(long long)b * kPartStride];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = kRedThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double beta = sqrt(red[0]);
  const bool finite = isfinite(beta);
  if (finite && beta > 0.0) {
    const T inv = (T)(1.0 / beta);
    const long long stride = (long long)gridDim.x * kRedThreads;
    for (long long i = blockIdx.x * (long long)kRedThreads + threadIdx.x; i < ns; i += stride)
      qnew[i] = qnew[i] * inv;
  }
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double* hc = H + (long long)k * ldh;
  for (int j = 0; j <= k; ++j) hc[j] = h1[j] + h2[j];
  hc[k + 1] = beta;
  st->beta = beta;
  if (!finite) {
    st->status = HPG_ERR_NAN;
    st->active = 0;
    return;
  }
  for (int j = 0; j < k; ++j) {
    const double a = hc[j], b = hc[j + 1];
    hc[j] = cs[j] * a + sn[j] * b;
    hc[j + 1] = -sn[j] * a + cs[j] * b;
  }
  const double mu = hypot(hc[k], hc[k + 1]);
  if (!(mu > 0.0) || !isfinite(mu)) {
    st->status = isfinite(mu) ? HPG_ERR_BREAKDOWN : HPG_ERR_NAN;
    st->active = 0;
    return;
  }
  cs[k] = hc[k] / mu;
  sn[k] = hc[k + 1] / mu;
  hc[k] = mu;
  hc[k + 1] = 0.0;
  t[k + 1] = -sn[k] * t[k];
  t[k] = cs[k] * t[k];
  const double rho = fabs(t[k + 1]);
  st->rho = rho;
  st->k = k + 1;
  st->iters += 1;
  if (rho / st->rho0 < st->tol || st->iters >= st->maxit || k + 1 >= st->m) st->active = 0;
}

// y = H[:k,:k]^{-1} t[:k] (the dense TRSM of Algorithm 3), one warp,
// column-oriented back substitution.
__global__ void trsm_kernel(const double* __restrict__ H, int ldh, const double* __restrict__ t,
                            double* __restrict__ y, const SolveState* st) {
  __shared__ double tt[kMaxRestart + 1];
  __shared__ double yi_s;
  const int k = st->k;
  for (int j = threadIdx.x; j < k; j += 32) tt[j] = t[j];
  __syncwarp();
  for (int i = k - 1; i >= 0; --i) {
    if (threadIdx.x == 0) {
      yi_s = tt[i] / H[(long long)i * ldh + i];
      y[i] = yi_s;
    }
    __syncwarp();
    const double yi = yi_s;
    for (int j = threadIdx.x; j < i; j += 32) tt[j] -= H[(long long)i * ldh + j] * yi;
    __syncwarp();
  }
}

// u = Q[:, :k] y (Algorithm 3, r <- Q t), k read from the solve state.
template <typename T>
__global__ void __launch_bounds__(256)
basis_combine_kernel(const T* __restrict__ Q, long long ns, const double* __restrict__ y,
                     const SolveState* st, T* __restrict__ u) {
  __shared__ T ys[kMaxRestart + 1];
  const int k = st->k;
  for (int j = threadIdx.x; j < k; j += blockDim.x) ys[j] = (T)y[j];
  __syncthreads();
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= ns) return;
  T acc = T(0);
  for (int j = 0; j < k; ++j) acc = fma(__ldcs(Q + j * ns + i), ys[j], acc);
  u[i] = acc;
}

// x += d (Algorithm 3, mixed-precision update: FP64 accumulation).
template <typename T>
__global__ void __launch_bounds__(256)
update_x_kernel(double* __restrict__ x, const T* __restrict__ d, long long ns) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < ns) x[i] += (double)d[i];
}

// r = b - A x and ||r||^2 partials (FP64), last block stores rho = ||r||.
__global__ void __launch_bounds__(kRedThreads)
residual_norm_kernel(const double* __restrict__ vals, const int* __restrict__ cols, long long ns,
                     const double* __restrict__ b, const double* __restrict__ x,
                     double* __restrict__ r, double* __restrict__ partials,
                     unsigned int* counter, double* __restrict__ out) {
  double acc[1] = {0.0};
  const long long stride = (long long)gridDim.x * kRedThreads;
  for (long long row = blockIdx.x * (long long)kRedThreads + threadIdx.x; row < ns;
       row += stride) {
    double v = b[row];
#pragma unroll
    for (int s = 0; s < kSlots; ++s) {
      const double a = ld_stream(vals + s * ns + row);
      const int c = ld_stream(cols + s * ns + row);
      v = fma(-a, __ldg(x + c), v);
    }
    r[row] = v;
    acc[0] = fma(v, v, acc[0]);
  }
  block_reduce<double, 1>(acc, 1, partials, counter, out);
}

// ||v||^2 of an FP64 vector.
__global__ void __launch_bounds__(kRedThreads)
norm2_kernel(const double* __restrict__ v, long long ns, double* __restrict__ partials,
             unsigned int* counter, double* __restrict__ out) {
  double acc[1] = {0.0};
  const long long stride = (long long)gridDim.x * kRedThreads;
  for (long long i = blockIdx.x * (long long)kRedThreads + threadIdx.x; i < ns; i += stride)
    acc[0] = fma(v[i], v[i], acc[0]);
  block_reduce<double, 1>(acc, 1, partials, counter, out);
}

// Start of a restart cycle: rho = sqrt(out2), q_0 = r / rho, t = rho e_1.
template <typename T>
__global__ void __launch_bounds__(256)
cycle_start_kernel(const double* __restrict__ r, long long ns, const double* __restrict__ rho2,
                   T* __restrict__ q0, double* __restrict__ t, SolveState* st) {
  const double rho = sqrt(*rho2);
  const double inv = 1.0 / rho;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < ns) q0[i] = (T)(r[i] * inv);
  if (i == 0) {
    t[0] = rho;
    for (int j = 1; j <= st->m; ++j) t[j] = 0.0;
    st->rho = rho;
    st->k = 0;
    st->active = 1;
  }
}

// ----------------------------------------------------------------- launchers
template <typename T> constexpr int prec_of() { return sizeof(T) == 8 ? HPG_FP64 : HPG_FP32; }

template <typename T, int KMAX, int KIND>
static void enqueue_pass(hpg_problem* h, const T* Q, long long ns, int ncol, const T* w,
                         T* qnew, double* out, cudaStream_t s) {
  Workspace* ws = h->ws;
  cgs2_pass_kernel<T, KMAX, KIND><<<ws->G, kRedThreads, 0, s>>>(
      Q, ns, ncol, w, ws->h1, ws->h2, qnew, ws->partials, ws->counter, out);
}

template <typename T, int KIND>
static int launch_pass(hpg_problem* h, const T* Q, long long ns, int ncol, const T* w, T* qnew,
                       double* out, cudaStream_t s) {
  static const int cls[3] = {K_CGS2_GEMVT, K_CGS2_REORTH, K_CGS2_FINAL};
  const double vecs = ncol + (KIND == kFinal ? 2 : 1);   // Q columns + w (+ q_new)
  const double bytes = (double)h->lev[0].n * vecs * sizeof(T);
  return launch(h, cls[KIND], 0, prec_of<T>(), bytes, s, "cgs2_pass_kernel", [&] {
    if (ncol <= 8)
      enqueue_pass<T, 8, KIND>(h, Q, ns, ncol, w, qnew, out, s);
    else if (ncol <= 16)
      enqueue_pass<T, 16, KIND>(h, Q, ns, ncol, w, qnew, out, s);
    else if (ncol <= 32)
      enqueue_pass<T, 32, KIND>(h, Q, ns, ncol, w, qnew, out, s);
    else
      enqueue_pass<T, 64, KIND>(h, Q, ns, ncol, w, qnew, out, s);
  });
}

// One inner step k (0-based): z = M^{-1} q_k, w = A z, CGS2 against
// q_0..q_k, q_{k+1} = w / ||w||, Givens update.
template <typename T>
static int inner_step(hpg_problem* h, int k, hpg_prec prec, cudaStream_t s) {
  Workspace* ws = h->ws;
  const long long ns = h->lev[0].g.n_store;
  T* Q = (T*)ws->Q;
  T* z = (T*)ws->z;
  T* w = (T*)ws->w;
  int rc;
  if ((rc = run_vcycle(h, 0, prec, Q + (long long)k * ns, z, s))) return rc;
  if ((rc = launch_spmv(h, 0, prec, z, w, s))) return rc;
  const int ncol = k + 1;
  T* qnew = Q + (long long)(k + 1) * ns;
  if ((rc = launch_pass<T, kGemvT>(h, Q, ns, ncol, w, nullptr, ws->h1, s))) return rc;
  if ((rc = launch_pass<T, kReorth>(h, Q, ns, ncol, w, nullptr, ws->h2, s))) return rc;
  if ((rc = launch_pass<T, kFinal>(h, Q, ns, ncol, w, qnew, nullptr, s))) return rc;
  return launch(h, K_ARNOLDI_FINISH, 0, prec_of<T>(), 2.0 * h->lev[0].n * sizeof(T), s,
                "arnoldi_finish_kernel", [&] {
                  arnoldi_finish_kernel<T><<<ws->G, kRedThreads, 0, s>>>(
                      qnew, ns, ws->partials, ws->G, k, ws->h1, ws->h2, ws->H, ws->m + 1,
                      ws->cs, ws->sn, ws->t, ws->st);
                });
}

// End of a cycle: y = H^{-1} t, u = Q y, d = M^{-1} u, x += d.
template <typename T>
static int cycle_update(hpg_problem* h, hpg_prec prec, int k_host, cudaStream_t s) {
  Workspace* ws = h->ws;
  const long long ns = h->lev[0].g.n_store;
  const double n = (double)h->lev[0].n;
  int rc;
  rc = launch(h, K_TRSM, 0, HPG_FP64, 0.0, s, "trsm_kernel", [&] {
    trsm_kernel<<<1, 32, 0, s>>>(ws->H, ws->m + 1, ws->t, ws->y, ws->st);
  });
  if (rc) return rc;
  rc = launch(h, K_COMBINE, 0, prec_of<T>(), n * (k_host + 1) * sizeof(T), s,
              "basis_combine_kernel", [&] {
                basis_combine_kernel<T><<<grid_for(ns, 256), 256, 0, s>>>(
                    (const T*)ws->Q, ns, ws->y, ws->st, (T*)ws->u);
              });
  if (rc) return rc;
  if ((rc = run_vcycle(h, 0, prec, ws->u, ws->z, s))) return rc;
  return launch(h, K_UPDATE_X, 0, HPG_FP64, n * (16.0 + sizeof(T)), s, "update_x_kernel", [&] {
    update_x_kernel<T><<<grid_for(ns, 256), 256, 0, s>>>(ws->x, (const T*)ws->z, ns);
  });
}

static int read_state(hpg_problem* h, cudaStream_t s) {
  Workspace* ws = h->ws;
  HPG_CK(cudaMemcpyAsync(ws->st_host, ws->st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
  HPG_CK(cudaStreamSynchronize(s));
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

template <typename T>
static int solve_t(hpg_problem* h, const double* b, double* x, double tol, int m, int maxit,
                   hpg_prec prec, hpg_solve_info* info, cudaStream_t s) {
  int rc;
  if ((rc = ensure_workspace(h, m, prec))) return rc;
  Workspace* ws = h->ws;
  const Level& L = h->lev[0];
  const long long ns = L.g.n_store, n = L.n;
  const long long launches0 = h->launches;
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
  if ((rc = launch_permute(h, 0, 0, HPG_FP64, b_dev, HPG_FP64, ws->b, s))) return rc;
  if ((rc = launch_permute(h, 0, 0, HPG_FP64, x_dev, HPG_FP64, ws->x, s))) return rc;
  SolveState init;
  memset(&init, 0, sizeof(init));
  init.tol = tol;
  init.maxit = maxit;
  init.m = m;
  init.status = HPG_OK;
  *ws->st_host = init;
  HPG_CK(cudaMemcpyAsync(ws->st, ws->st_host, sizeof(SolveState), cudaMemcpyHostToDevice, s));
  rc = launch(h, K_NORM, 0, HPG_FP64, 8.0 * n, s, "norm2_kernel", [&] {
    norm2_kernel<<<ws->G, kRedThreads, 0, s>>>(ws->b, ns, ws->partials, ws->counter, ws->h1);
  });
  if (rc) return rc;
  double rho0_sq = 0.0;
  HPG_CK(cudaMemcpyAsync(&rho0_sq, ws->h1, 8, cudaMemcpyDeviceToHost, s));
  HPG_CK(cudaStreamSynchronize(s));
  const double rho0 = sqrt(rho0_sq);
  int status = HPG_OK;
  int iters = 0, restarts = 0;
  double rel = 0.0;
  bool converged = false;
  if (!(rho0 == rho0) || isinf(rho0)) {
    status = HPG_ERR_NAN;
  } else if (rho0 == 0.0) {
    // b = 0: the solution is x = 0
    HPG_CK(cudaMemsetAsync(ws->x, 0, 8 * ns, s));
    converged = true;
  } else {
    init.rho0 = rho0;
    *ws->st_host = init;
    HPG_CK(cudaMemcpyAsync(ws->st, ws->st_host, sizeof(SolveState), cudaMemcpyHostToDevice, s));
    while (true) {
      rc = launch(h, K_RESIDUAL, 0, HPG_FP64, n * (27.0 * 12.0 + 3.0 * 8.0), s,
                  "residual_norm_kernel", [&] {
                    residual_norm_kernel<<<ws->G, kRedThreads, 0, s>>>(
                        L.v64, L.cols, ns, ws->b, ws->x, ws->r, ws->partials, ws->counter,
                        ws->h2);
                  });
      if (rc) return rc;
      double rho_sq = 0.0;
      HPG_CK(cudaMemcpyAsync(&rho_sq, ws->h2, 8, cudaMemcpyDeviceToHost, s));
      if ((rc = read_state(h, s))) return rc;
      const double rho = sqrt(rho_sq);
      rel = rho / rho0;
      iters = ws->st_host->iters;
      if (!(rho == rho) || isinf(rho)) {
        status = HPG_ERR_NAN;
        break;
      }
      if (rel < tol) {
        converged = true;
        break;
      }
      if (ws->st_host->status != HPG_OK) {
        status = ws->st_host->status;
        break;
      }
      if (iters >= maxit) {
        status = HPG_ERR_NOT_CONVERGED;
        break;
      }
      rc = launch(h, K_CYCLE_START, 0, prec_of<T>(), n * (8.0 + sizeof(T)), s,
                  "cycle_start_kernel", [&] {
                    cycle_start_kernel<T><<<grid_for(ns, 256), 256, 0, s>>>(
                        ws->r, ns, ws->h2, (T*)ws->Q, ws->t, ws->st);
                  });
      if (rc) return rc;
      for (int k = 0; k < m; ++k) {
        if ((rc = inner_step<T>(h, k, prec, s))) return rc;
        if ((rc = read_state(h, s))) return rc;
        if (!ws->st_host->active) break;
      }
      if (ws->st_host->k > 0) {
        if ((rc = cycle_update<T>(h, prec, ws->st_host->k, s))) return rc;
      }
      restarts++;
      if (ws->st_host->status != HPG_OK && ws->st_host->k == 0) {
        status = ws->st_host->status;
        break;
      }
    }
  }
  // solution back to natural order (and to the host buffer if needed)
  double* x_out = x_host ? ws->stage + n : x;
  if ((rc = launch_permute(h, 0, 1, HPG_FP64, ws->x, HPG_FP64, x_out, s))) return rc;
  if (x_host) HPG_CK(cudaMemcpyAsync(x, x_out, 8 * n, cudaMemcpyDeviceToHost, s));
  HPG_CK(cudaStreamSynchronize(s));
  if (converged) status = HPG_OK;
  if (info) {
    info->iterations = iters;
    info->restarts = restarts;
    info->converged = converged ? 1 : 0;
    info->status = status;
    info->rel_residual = rel;
    info->rho0 = rho0;
    info->kernel_launches = (int)(h->launches - launches0);
    info->graph_launches = 0;
  }
  if (status != HPG_OK) set_error("hpg_gmres_ir_solve: %s after %d iterations (rel %g)",
                                  hpg_status_string(status), iters, rel);
  return status;
}

}  // namespace hpg

using namespace hpg;

extern "C" {

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
  if ((inner != HPG_FP64 && inner != HPG_FP32) || basis != inner) {
    set_error("hpg_gmres_ir_solve: inner %d / basis %d not supported (basis must equal inner)",
              (int)inner, (int)basis);
    if (info) info->status = HPG_ERR_UNSUPPORTED;
    return HPG_ERR_UNSUPPORTED;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (inner == HPG_FP64) return solve_t<double>(h, b, x, tol, restart, maxit, inner, info, s);
  return solve_t<float>(h, b, x, tol, restart, maxit, inner, info, s);
}

}  // extern "C"
