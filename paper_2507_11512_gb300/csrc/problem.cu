// Problem set-up: the 27-point ELLPACK matrix generated on the device in
// colour-blocked storage order, the multigrid hierarchy, vector reordering,
// and the error / status plumbing of the C ABI.
//
// Matrix (Sec. 2-3): row i couples grid point i to every point within one
// step along each axis; diagonal 26 (times theta_i when given), off-diagonal
// -1 + beta*(dx+dy+dz)/3 at neighbour offset d; neighbours outside the grid
// are dropped (boundary rows have fewer non-zeros).  Storage (Sec. 3.2.2):
// ELLPACK with 27 slots per row, slot-major ("column-major" ELL: slot s of all
// rows is contiguous), int32 column indices shared by an FP64 and an FP32
// value array.  Rows are ordered by colour (Sec. 3.2.1: the matrix and the
// vectors are reordered symmetrically by independent sets).

#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>

#include "hpg_internal.cuh"

namespace hpg {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  set_error("%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  return e == cudaErrorMemoryAllocation ? HPG_ERR_ALLOC : HPG_ERR_CUDA;
}

int dev_alloc(void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
  }
  e = cudaMemset(*p, 0, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemset", __FILE__, __LINE__);
  return HPG_OK;
}

void dev_free(void* p) {
  if (p) cudaFree(p);
}

// ----------------------------------------------------------------- geometry
static Geom make_geom(int nx, int ny, int nz, long long cnt[kColours]) {
  Geom g;
  memset(&g, 0, sizeof(g));
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  long long off = 0;
  for (int c = 0; c < kColours; ++c) {
    const int px = colour_parity_x(c), py = colour_parity_y(c), pz = colour_parity_z(c);
    g.cdx[c] = (nx - px + 1) / 2;
    g.cdy[c] = (ny - py + 1) / 2;
    g.cdz[c] = (nz - pz + 1) / 2;
    if (g.cdx[c] < 0) g.cdx[c] = 0;
    if (g.cdy[c] < 0) g.cdy[c] = 0;
    if (g.cdz[c] < 0) g.cdz[c] = 0;
    cnt[c] = (long long)g.cdx[c] * g.cdy[c] * g.cdz[c];
    g.off[c] = off;
    off += (cnt[c] + kRowAlign - 1) / kRowAlign * kRowAlign;
  }
  g.off[kColours] = off;
  g.n_store = off;
  return g;
}

static long long axis_pairs(int n) { return n >= 1 ? 3LL * n - 2 : 0; }

// ------------------------------------------------------------------ kernels
// One thread per storage row writes the row's 27 ELL slots.
__global__ void gen_ell_kernel(const __grid_constant__ Geom g, double beta,
                               const double* __restrict__ theta, int* __restrict__ cols,
                               double* __restrict__ v64, float* __restrict__ v32) {
  pdl_trigger();
  pdl_wait();
  const long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (row >= g.n_store) return;
  const long long ns = g.n_store;
  const int c = colour_of_row(g, row);
  const long long p = row - g.off[c];
  const long long cntc = (long long)g.cdx[c] * g.cdy[c] * g.cdz[c];
  if (p >= cntc) {
    // padding row: identity (diagonal 1), so sweeps and products keep its
    // (zero) vector entries at zero
    for (int s = 0; s < kSlots; ++s) {
      cols[s * ns + row] = (int)row;
      v64[s * ns + row] = (s == kCentre) ? 1.0 : 0.0;
      v32[s * ns + row] = (s == kCentre) ? 1.0f : 0.0f;
    }
    return;
  }
  const int I = (int)(p % g.cdx[c]);
  const long long q = p / g.cdx[c];
  const int J = (int)(q % g.cdy[c]);
  const int K = (int)(q / g.cdy[c]);
  const int i = 2 * I + colour_parity_x(c);
  const int j = 2 * J + colour_parity_y(c);
  const int k = 2 * K + colour_parity_z(c);
  const double th =
      theta ? ld_dep(theta + (long long)i + (long long)g.nx * (j + (long long)g.ny * k)) : 1.0;
  for (int s = 0; s < kSlots; ++s) {
    const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = s / 9 - 1;
    const int ni = i + dx, nj = j + dy, nk = k + dz;
    const bool inside = ni >= 0 && ni < g.nx && nj >= 0 && nj < g.ny && nk >= 0 && nk < g.nz;
    long long col = row;
    double val = 0.0;
    if (inside) {
      col = store_index(g, ni, nj, nk);
      val = (s == kCentre) ? kDiag * th : -1.0 + beta * (double)(dx + dy + dz) / 3.0;
    }
    cols[s * ns + row] = (int)col;
    v64[s * ns + row] = val;
    v32[s * ns + row] = (float)val;
  }
}

// theta of the coarse grid by injection: theta_c(I,J,K) = theta_f(2I,2J,2K).
__global__ void inject_theta_kernel(int fnx, int fny, int cnx, int cny, int cnz,
                                    const double* __restrict__ tf, double* __restrict__ tc) {
  pdl_trigger();
  pdl_wait();
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n = (long long)cnx * cny * cnz;
  if (q >= n) return;
  const int I = (int)(q % cnx);
  const int J = (int)((q / cnx) % cny);
  const int K = (int)(q / ((long long)cnx * cny));
  tc[q] = ld_dep(tf + 2LL * I + (long long)fnx * (2LL * J + (long long)fny * 2 * K));
}

// Gradient of a loss with respect to the per-cell diagonal scales: only
// a_ii = 26 theta_i depends on theta_i, so with x = A^{-1} b and the adjoint
// lambda = A^{-T} dL/dx, dL/dtheta_i = -lambda_i (d a_ii / d theta_i) x_i
// = (-26 lambda_i) x_i (natural order, FP64).
__global__ void __launch_bounds__(256)
diag_scale_gradient_kernel(long long n, const double* __restrict__ lam,
                           const double* __restrict__ x, double* __restrict__ grad) {
  pdl_trigger();
  pdl_wait();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride)
    grad[i] = (-kDiag * ld_dep(lam + i)) * ld_dep(x + i);
}

template <typename Tin, typename Tout>
__global__ void to_storage_kernel(const __grid_constant__ Geom g, const Tin* __restrict__ in,
                                  Tout* __restrict__ out) {
  pdl_trigger();
  pdl_wait();
  const long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (row >= g.n_store) return;
  const int c = colour_of_row(g, row);
  const long long p = row - g.off[c];
  const long long cntc = (long long)g.cdx[c] * g.cdy[c] * g.cdz[c];
  if (p >= cntc) {
    out[row] = Tout(0);
    return;
  }
  const int I = (int)(p % g.cdx[c]);
  const long long q = p / g.cdx[c];
  const int J = (int)(q % g.cdy[c]);
  const int K = (int)(q / g.cdy[c]);
  const int i = 2 * I + colour_parity_x(c);
  const int j = 2 * J + colour_parity_y(c);
  const int k = 2 * K + colour_parity_z(c);
  out[row] = (Tout)ld_dep(in + (long long)i + (long long)g.nx * (j + (long long)g.ny * k));
}

template <typename Tin, typename Tout>
__global__ void to_natural_kernel(const __grid_constant__ Geom g, const Tin* __restrict__ in,
                                  Tout* __restrict__ out) {
  pdl_trigger();
  pdl_wait();
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n = (long long)g.nx * g.ny * g.nz;
  if (q >= n) return;
  const int i = (int)(q % g.nx);
  const int j = (int)((q / g.nx) % g.ny);
  const int k = (int)(q / ((long long)g.nx * g.ny));
  out[q] = (Tout)ld_dep(in + store_index(g, i, j, k));
}

// ----------------------------------------------------------------- launchers
static int build_level_matrix(hpg_problem* h, int l) {
  Level& L = h->lev[l];
  const long long ns = L.g.n_store;
  int rc;
  if ((rc = dev_alloc((void**)&L.cols, sizeof(int) * kSlots * ns))) return rc;
  if ((rc = dev_alloc((void**)&L.v64, sizeof(double) * kSlots * ns))) return rc;
  if ((rc = dev_alloc((void**)&L.v32, sizeof(float) * kSlots * ns))) return rc;
  return launch(h, K_GEN, l, HPG_FP64, ns * kSlots * (4.0 + 8.0 + 4.0), 0, "gen_ell_kernel",
                [&] {
                  return kl(h, gen_ell_kernel, grid_for(ns, 256), 256, (cudaStream_t)0, L.g,
                            h->beta, (const double*)L.theta, L.cols, L.v64, L.v32);
                });
}

static void free_level(Level& L, bool keep_matrix) {
  for (int p = 0; p < 2; ++p) {
    dev_free(L.rhs[p]);
    dev_free(L.sol[p]);
    L.rhs[p] = L.sol[p] = nullptr;
  }
  dev_free(L.pipe_flags);
  dev_free(L.pipe_sync);
  L.pipe_flags = nullptr;
  L.pipe_sync = nullptr;
  L.pipe_tiles = 0;
  if (!keep_matrix) {
    dev_free(L.cols);
    dev_free(L.v32);
    dev_free(L.v64);
    dev_free(L.theta);
    L.cols = nullptr;
    L.v32 = nullptr;
    L.v64 = nullptr;
    L.theta = nullptr;
  }
}

static void init_level_geom(Level& L, int nx, int ny, int nz) {
  L.g = make_geom(nx, ny, nz, L.cnt);
  L.n = (long long)nx * ny * nz;
  L.nnz = axis_pairs(nx) * axis_pairs(ny) * axis_pairs(nz);
}

int launch_permute(hpg_problem* h, int level, int direction, hpg_prec in_prec,
                   const void* in, hpg_prec out_prec, void* out, cudaStream_t s) {
  const Level& L = h->lev[level];
  const int T = 256;
  const double bytes = (double)L.n * (prec_size(in_prec) + prec_size(out_prec));
  return launch(h, K_PERMUTE, level, out_prec, bytes, s, "permute kernel", [&] {
    if (direction == 0) {
      const int G = grid_for(L.g.n_store, T);
      if (in_prec == HPG_FP64 && out_prec == HPG_FP64)
        return kl(h, to_storage_kernel<double, double>, G, T, s, L.g, (const double*)in,
                  (double*)out);
      if (in_prec == HPG_FP64 && out_prec == HPG_FP32)
        return kl(h, to_storage_kernel<double, float>, G, T, s, L.g, (const double*)in,
                  (float*)out);
      if (in_prec == HPG_FP32 && out_prec == HPG_FP64)
        return kl(h, to_storage_kernel<float, double>, G, T, s, L.g, (const float*)in,
                  (double*)out);
      return kl(h, to_storage_kernel<float, float>, G, T, s, L.g, (const float*)in,
                (float*)out);
    }
    const int G = grid_for(L.n, T);
    if (in_prec == HPG_FP64 && out_prec == HPG_FP64)
      return kl(h, to_natural_kernel<double, double>, G, T, s, L.g, (const double*)in,
                (double*)out);
    if (in_prec == HPG_FP64 && out_prec == HPG_FP32)
      return kl(h, to_natural_kernel<double, float>, G, T, s, L.g, (const double*)in,
                (float*)out);
    if (in_prec == HPG_FP32 && out_prec == HPG_FP64)
      return kl(h, to_natural_kernel<float, double>, G, T, s, L.g, (const float*)in,
                (double*)out);
    return kl(h, to_natural_kernel<float, float>, G, T, s, L.g, (const float*)in,
              (float*)out);
  });
}

}  // namespace hpg

using namespace hpg;

// ------------------------------------------------------------------- C ABI
extern "C" {

HPG_API const char* hpg_status_string(int status) {
  switch (status) {
    case HPG_OK: return "HPG_OK";
    case HPG_ERR_INVALID: return "HPG_ERR_INVALID";
    case HPG_ERR_CUDA: return "HPG_ERR_CUDA";
    case HPG_ERR_NOT_CONVERGED: return "HPG_ERR_NOT_CONVERGED";
    case HPG_ERR_BREAKDOWN: return "HPG_ERR_BREAKDOWN";
    case HPG_ERR_NAN: return "HPG_ERR_NAN";
    case HPG_ERR_ALLOC: return "HPG_ERR_ALLOC";
    case HPG_ERR_STATE: return "HPG_ERR_STATE";
    case HPG_ERR_UNSUPPORTED: return "HPG_ERR_UNSUPPORTED";
    case HPG_ERR_TIMEOUT: return "HPG_ERR_TIMEOUT";
  }
  return "HPG_ERR_UNKNOWN";
}

HPG_API const char* hpg_last_error(void) { return g_last_error.c_str(); }

HPG_API int hpg_setup_problem(int nx, int ny, int nz, const hpg_stencil_params* p,
                              hpg_problem_t** out) {
  g_last_error.clear();
  if (!out) {
    set_error("hpg_setup_problem: out is NULL");
    return HPG_ERR_INVALID;
  }
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1) {
    set_error("hpg_setup_problem: grid %d x %d x %d has an edge < 1", nx, ny, nz);
    return HPG_ERR_INVALID;
  }
  const long long n = (long long)nx * ny * nz;
  // storage rows (with colour-block padding) times 27 slots must fit int32
  // column indices and int32 slot offsets
  if ((n + 8LL * kRowAlign) * kSlots >= (1LL << 31)) {
    set_error("hpg_setup_problem: grid %d x %d x %d is too large (n*27 >= 2^31)", nx, ny,
              nz);
    return HPG_ERR_INVALID;
  }
  const double beta = p ? p->beta : 0.0;
  if (!(beta == beta) || beta > 1.0 || beta < -1.0) {
    set_error("hpg_setup_problem: beta = %g outside [-1, 1]", beta);
    return HPG_ERR_INVALID;
  }
  hpg_problem* h = new hpg_problem();
  int rc = HPG_OK;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e != cudaSuccess) {
    rc = cuda_fail(e, "cudaGetDevice", __FILE__, __LINE__);
    delete h;
    return rc;
  }
  h->beta = beta;
  h->nlev = 1;
  h->pdl_next = false;
  Level& L0 = h->lev[0];
  init_level_geom(L0, nx, ny, nz);
  if (p && p->theta) {
    rc = dev_alloc((void**)&L0.theta, sizeof(double) * n);
    if (rc == HPG_OK) {
      e = cudaMemcpy(L0.theta, p->theta, sizeof(double) * n, cudaMemcpyDefault);
      if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpy(theta)", __FILE__, __LINE__);
    }
  }
  if (rc == HPG_OK) rc = build_level_matrix(h, 0);
  if (rc == HPG_OK) {
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) rc = cuda_fail(e, "problem generation", __FILE__, __LINE__);
  }
  if (rc != HPG_OK) {
    hpg_destroy(h);
    return rc;
  }
  *out = h;
  return HPG_OK;
}

HPG_API int hpg_build_mg_hierarchy(hpg_problem_t* h, int levels, int pre_sweeps,
                                   int post_sweeps) {
  g_last_error.clear();
  if (!h) {
    set_error("hpg_build_mg_hierarchy: NULL handle");
    return HPG_ERR_INVALID;
  }
  if (levels < 1 || levels > kMaxLevels || pre_sweeps < 0 || post_sweeps < 0 ||
      pre_sweeps > 16 || post_sweeps > 16) {
    set_error("hpg_build_mg_hierarchy: levels %d (1..%d), sweeps %d/%d (0..16)", levels,
              kMaxLevels, pre_sweeps, post_sweeps);
    return HPG_ERR_INVALID;
  }
  if (batch_owners(h) > 0) {
    set_error("hpg_build_mg_hierarchy: %d multi-system batch(es) still use this problem; "
              "destroy them first", batch_owners(h));
    return HPG_ERR_STATE;
  }
  h->pdl_next = false;
  // drop a previous hierarchy (keep level 0's matrix) and everything sized by it
  destroy_workspace(h);
  destroy_batch(h);
  for (int l = 0; l < h->nlev; ++l) free_level(h->lev[l], l == 0);
  h->nlev = 1;
  h->hierarchy = false;
  int nx = h->lev[0].g.nx, ny = h->lev[0].g.ny, nz = h->lev[0].g.nz;
  int nl = 1;
  while (nl < levels && nx % 2 == 0 && ny % 2 == 0 && nz % 2 == 0) {
    nx /= 2;
    ny /= 2;
    nz /= 2;
    nl++;
  }
  int rc = HPG_OK;
  for (int l = 1; l < nl && rc == HPG_OK; ++l) {
    const Level& F = h->lev[l - 1];
    Level& C = h->lev[l];
    init_level_geom(C, F.g.nx / 2, F.g.ny / 2, F.g.nz / 2);
    h->nlev = l + 1;
    if (F.theta) {
      rc = dev_alloc((void**)&C.theta, sizeof(double) * C.n);
      if (rc) break;
      rc = launch(h, K_GEN, l, HPG_FP64, 16.0 * C.n, 0, "inject_theta_kernel", [&] {
        return kl(h, inject_theta_kernel, grid_for(C.n, 256), 256, (cudaStream_t)0, F.g.nx,
                  F.g.ny, C.g.nx, C.g.ny, C.g.nz, (const double*)F.theta, C.theta);
      });
      if (rc) break;
    }
    rc = build_level_matrix(h, l);
  }
  for (int l = 1; l < h->nlev && rc == HPG_OK; ++l) {
    Level& L = h->lev[l];
    for (int pi = 0; pi < 2 && rc == HPG_OK; ++pi) {
      const size_t es = pi == 0 ? 8 : 4;
      rc = dev_alloc(&L.rhs[pi], es * L.g.n_store);
      if (rc == HPG_OK) rc = dev_alloc(&L.sol[pi], es * L.g.n_store);
    }
  }
  // completion flags of the pipelined sweep on levels whose matrix streams
  if (rc == HPG_OK && !h->pipe_err) rc = dev_alloc((void**)&h->pipe_err, sizeof(unsigned) * 4);
  for (int l = 0; l < h->nlev && rc == HPG_OK; ++l) {
    Level& L = h->lev[l];
    long long maxrows = 0;
    for (int c = 0; c < kColours; ++c) maxrows = std::max(maxrows, L.g.off[c + 1] - L.g.off[c]);
    L.pipe_tiles = (int)((maxrows + kPipeTileRows - 1) / kPipeTileRows);
    rc = dev_alloc((void**)&L.pipe_flags, sizeof(int) * (size_t)kMaxPipePhases * L.pipe_tiles);
    if (rc == HPG_OK) rc = dev_alloc((void**)&L.pipe_sync, sizeof(unsigned) * kPipeWords);
  }
  if (rc == HPG_OK) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) rc = cuda_fail(e, "hierarchy build", __FILE__, __LINE__);
  }
  if (rc != HPG_OK) return rc;
  h->pre = pre_sweeps;
  h->post = post_sweeps;
  h->hierarchy = true;
  return HPG_OK;
}

HPG_API int hpg_num_levels(const hpg_problem_t* h, int* levels) {
  if (!h || !levels) {
    set_error("hpg_num_levels: NULL argument");
    return HPG_ERR_INVALID;
  }
  *levels = h->nlev;
  return HPG_OK;
}

HPG_API int hpg_level_info(const hpg_problem_t* h, int level, hpg_level_desc* out) {
  if (!h || !out || level < 0 || level >= h->nlev) {
    set_error("hpg_level_info: bad handle, output or level %d", level);
    return HPG_ERR_INVALID;
  }
  const Level& L = h->lev[level];
  out->nx = L.g.nx;
  out->ny = L.g.ny;
  out->nz = L.g.nz;
  out->n = L.n;
  out->n_store = L.g.n_store;
  out->nnz = L.nnz;
  for (int c = 0; c <= kColours; ++c) out->colour_offset[c] = L.g.off[c];
  for (int c = 0; c < kColours; ++c) out->colour_count[c] = L.cnt[c];
  return HPG_OK;
}

HPG_API int hpg_permute(hpg_problem_t* h, int level, int direction, hpg_prec in_prec,
                        const void* in, hpg_prec out_prec, void* out, void* stream) {
  g_last_error.clear();
  if (!h || !in || !out || level < 0 || level >= h->nlev || (direction != 0 && direction != 1) ||
      (in_prec != HPG_FP64 && in_prec != HPG_FP32) ||
      (out_prec != HPG_FP64 && out_prec != HPG_FP32)) {
    set_error("hpg_permute: invalid argument");
    return HPG_ERR_INVALID;
  }
  h->pdl_next = false;
  return launch_permute(h, level, direction, in_prec, in, out_prec, out, (cudaStream_t)stream);
}

HPG_API int hpg_set_option(hpg_problem_t* h, int option, int value) {
  if (!h) {
    set_error("hpg_set_option: NULL handle");
    return HPG_ERR_INVALID;
  }
  if (batch_owners(h) > 0) {
    // a batch's captured graph embeds the current choices
    set_error("hpg_set_option: %d multi-system batch(es) use this problem; destroy them "
              "first", batch_owners(h));
    return HPG_ERR_STATE;
  }
  switch (option) {
    case HPG_OPT_COARSE_CLUSTER: h->coarse_cluster = value != 0; break;
    case HPG_OPT_PDL: h->pdl_enabled = value != 0; break;
    case HPG_OPT_GS_HALO: h->gs_halo = value != 0; break;
    case HPG_OPT_COARSE_CTA: h->coarse_cta = value != 0; break;
    case HPG_OPT_PDL_ROWS:
      if (value < 0) {
        set_error("hpg_set_option: HPG_OPT_PDL_ROWS takes a row count >= 0, not %d", value);
        return HPG_ERR_INVALID;
      }
      h->pdl_rows = value;
      break;
    case HPG_OPT_GS_PIPELINE:
      if (value < 0 || value > 3) {
        set_error("hpg_set_option: HPG_OPT_GS_PIPELINE takes 0..3, not %d", value);
        return HPG_ERR_INVALID;
      }
      h->gs_pipeline = value;
      break;
    default:
      set_error("hpg_set_option: unknown option %d", option);
      return HPG_ERR_INVALID;
  }
  if (h->ws) destroy_workspace(h);   // captured graphs embed the old choice
  drop_batch_graph(h);
  return HPG_OK;
}

HPG_API int hpg_diag_scale_gradient(hpg_problem_t* h, const double* lambda, const double* x,
                                    double* grad, void* stream) {
  g_last_error.clear();
  if (!h || !lambda || !x || !grad) {
    set_error("hpg_diag_scale_gradient: invalid argument (handle or pointers)");
    return HPG_ERR_INVALID;
  }
  const long long n = h->lev[0].n;
  h->pdl_next = false;
  const cudaStream_t s = (cudaStream_t)stream;
  return launch(h, K_GRADIENT, 0, HPG_FP64, 24.0 * n, s, "diag_scale_gradient_kernel", [&] {
    return kl(h, diag_scale_gradient_kernel, (int)std::min<long long>(grid_for(n, 256),
                                                                      8LL * h->num_sms),
              256, s, n, lambda, x, grad);
  });
}

HPG_API int hpg_inject_stall(hpg_problem_t* h, int level, int tiles) {
  if (!h || level < 0 || level >= h->nlev || tiles < 0 || !h->lev[level].pipe_sync) {
    set_error("hpg_inject_stall: invalid argument (level %d, tiles %d)", level, tiles);
    return HPG_ERR_INVALID;
  }
  const unsigned v = (unsigned)tiles;
  HPG_CK(cudaMemcpy(h->lev[level].pipe_sync + kPipeQueue, &v, sizeof(v), cudaMemcpyHostToDevice));
  return HPG_OK;
}

HPG_API int hpg_destroy(hpg_problem_t* h) {
  if (!h) return HPG_OK;
  if (batch_owners(h) > 0) {
    // the batch's graph points at this problem's buffers
    set_error("hpg_destroy: %d multi-system batch(es) still use this problem; call "
              "hpg_batch_destroy first", batch_owners(h));
    return HPG_ERR_STATE;
  }
  destroy_workspace(h);
  destroy_batch(h);
  destroy_profiler(h);
  for (int l = 0; l < kMaxLevels; ++l) free_level(h->lev[l], false);
  dev_free(h->pipe_err);
  delete h;
  return HPG_OK;
}

}  // extern "C"
