/* A plain C caller of the HPG-MxP library: only include/hpgmxp.h and
 * libhpgmxp.so, no Python, no CUDA headers.  Used by tests/test_c_abi.py.
 *
 *   abi_check host   argument validation and status strings (no GPU needed)
 *   abi_check solve  16^3 MxP GMRES(30)-IR of b = 1 with host buffers (the
 *                    library stages them through device memory), printing
 *                    iterations, restarts and the FP64 relative residual
 */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "hpgmxp.h"

static int expect(int got, int want, const char* what) {
  if (got != want) {
    fprintf(stderr, "%s: status %d (%s), expected %d; last error: %s\n", what, got,
            hpg_status_string(got), want, hpg_last_error());
    return 1;
  }
  return 0;
}

static int host_checks(void) {
  int bad = 0;
  hpg_problem_t* h = NULL;
  hpg_stencil_params p = {2.0, NULL};   /* |beta| > 1: rejected */
  bad |= expect(hpg_setup_problem(0, 4, 4, NULL, &h), HPG_ERR_INVALID, "edge 0");
  bad |= h != NULL;
  bad |= expect(hpg_setup_problem(4, 4, 4, &p, &h), HPG_ERR_INVALID, "beta 2");
  bad |= expect(hpg_setup_problem(4, 4, 4, NULL, NULL), HPG_ERR_INVALID, "out NULL");
  bad |= expect(hpg_spmv(NULL, 0, HPG_FP32, NULL, NULL, NULL), HPG_ERR_INVALID, "spmv");
  bad |= expect(hpg_mg_vcycle(NULL, 0, HPG_FP32, NULL, NULL, NULL), HPG_ERR_INVALID, "vcycle");
  bad |= expect(hpg_gmres_ir_solve(NULL, NULL, NULL, 1e-9, 30, 100, HPG_FP32, HPG_FP32, NULL,
                                   NULL), HPG_ERR_INVALID, "solve");
  bad |= expect(hpg_destroy(NULL), HPG_OK, "destroy NULL");
  bad |= strcmp(hpg_status_string(HPG_OK), "") == 0;
  printf("host checks %s\n", bad ? "FAILED" : "ok");
  return bad;
}

static int solve(void) {
  const int nx = 16, ny = 16, nz = 16, n = nx * ny * nz;
  hpg_stencil_params p = {0.5, NULL};
  hpg_problem_t* h = NULL;
  int rc = hpg_setup_problem(nx, ny, nz, &p, &h);
  if (rc) return expect(rc, HPG_OK, "setup");
  rc = hpg_build_mg_hierarchy(h, 4, 1, 1);
  if (rc) return expect(rc, HPG_OK, "hierarchy");
  double* b = (double*)malloc(sizeof(double) * n);
  double* x = (double*)calloc(n, sizeof(double));
  for (int i = 0; i < n; ++i) b[i] = 1.0;
  hpg_solve_info info;
  memset(&info, 0, sizeof(info));
  rc = hpg_gmres_ir_solve(h, b, x, 1e-9, 30, 10000, HPG_FP32, HPG_FP32, &info, NULL);
  printf("status %d iterations %d restarts %d converged %d rel_residual %.3e\n", rc,
         info.iterations, info.restarts, info.converged, info.rel_residual);
  int bad = expect(rc, HPG_OK, "solve") || !info.converged || !(info.rel_residual < 1e-9);
  bad |= expect(hpg_destroy(h), HPG_OK, "destroy");
  free(b);
  free(x);
  return bad;
}

int main(int argc, char** argv) {
  if (argc > 1 && strcmp(argv[1], "solve") == 0) return solve();
  return host_checks();
}
