/* The C ABI used from plain C (no torch, no GPU needed): host-only handles, table
 * queries and the documented error codes.  Built and run by tests/test_c_abi.py. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "delimit.h"

#define CHECK(cond)                                                   \
  do {                                                                \
    if (!(cond)) {                                                    \
      fprintf(stderr, "check failed at line %d: %s\n", __LINE__, #cond); \
      return 1;                                                       \
    }                                                                 \
  } while (0)

int main(void) {
  /* 30 directions on the z >= 0 hemisphere (a golden-angle spiral), one shell */
  enum { M = 30 };
  double dirs[M * 3], bvals[M];
  for (int i = 0; i < M; ++i) {
    const double z = 1.0 - (i + 0.5) / M, r = sqrt(1.0 - z * z), ph = 2.399963229728653 * i;
    dirs[3 * i] = r * cos(ph);
    dirs[3 * i + 1] = r * sin(ph);
    dirs[3 * i + 2] = z;
    bvals[i] = 1000.0;
  }
  CHECK(delimit_version() >= 100);

  delimit_sh_basis* b = NULL;
  CHECK(delimit_sh_basis_create(dirs, bvals, M, 4, 0.006, DELIMIT_HOST_ONLY, &b) == DELIMIT_OK && b);
  int n_shells = 0, n_coef = 0, n_dirs = 0;
  CHECK(delimit_sh_basis_info(b, &n_shells, &n_coef, &n_dirs) == DELIMIT_OK);
  CHECK(n_shells == 1 && n_coef == 15 && n_dirs == M);

  /* order must be even: INVALID_ARG, and a message */
  delimit_sh_basis* bad = NULL;
  CHECK(delimit_sh_basis_create(dirs, bvals, M, 3, 0.006, DELIMIT_HOST_ONLY, &bad) == DELIMIT_ERR_INVALID_ARG);
  CHECK(bad == NULL && strlen(delimit_last_error()) > 0);
  /* lambda = 0 with fewer directions than coefficients: RANK_DEFICIENT */
  CHECK(delimit_sh_basis_create(dirs, bvals, 10, 4, 0.0, DELIMIT_HOST_ONLY, &bad) == DELIMIT_ERR_RANK_DEFICIENT);

  /* a host-only handle refuses compute calls */
  CHECK(delimit_signal2sh(b, NULL, NULL, 1, 1, 1, 1, DELIMIT_F32, DELIMIT_F32, NULL) == DELIMIT_ERR_INVALID_ARG);

  /* LSC geometry: order 4 in, one shell, radius 0.4 rad, 2 rings x 6 sectors (K = 13) */
  delimit_lsc_geometry* g = NULL;
  CHECK(delimit_lsc_geometry_create(b, 4, 1, 0.4, 2, 6, DELIMIT_WINDOW_SAME, DELIMIT_HOST_ONLY, &g) == DELIMIT_OK);
  int K = 0, ni = 0, no = 0, si = 0, so = 0;
  int64_t nn = 0;
  CHECK(delimit_lsc_geometry_info(g, &K, &ni, &no, &si, &so, &nn) == DELIMIT_OK);
  CHECK(K == 13 && ni == 15 && no == 15 && si == 1 && so == 1 && nn >= M);
  /* the resampled geometry has no neighbour-bin table */
  CHECK(delimit_lsc_neighbour_table(g, 0, 0, NULL, NULL, NULL) == DELIMIT_ERR_INVALID_ARG);

  /* the resampling-free form: every direction is its own neighbour, binned to the origin */
  delimit_lsc_geometry* gn = NULL;
  CHECK(delimit_lsc_geometry_create(b, 4, 1, 0.4, 2, 6, DELIMIT_WINDOW_SAME, DELIMIT_HOST_ONLY | DELIMIT_LSC_NEIGHBOURS,
                                    &gn) == DELIMIT_OK);
  int64_t indptr[M + 1];
  CHECK(delimit_lsc_neighbour_table(gn, 0, 0, indptr, NULL, NULL) == DELIMIT_OK);
  CHECK(indptr[0] == 0 && indptr[M] >= M);
  int64_t idx[4096];
  int32_t bins[4096];
  CHECK(indptr[M] <= 4096);
  CHECK(delimit_lsc_neighbour_table(gn, 0, 0, indptr, idx, bins) == DELIMIT_OK);
  for (int i = 0; i < M; ++i) {
    int self = 0;
    for (int64_t e = indptr[i]; e < indptr[i + 1]; ++e) {
      CHECK(bins[e] >= 0 && bins[e] < K);
      if (idx[e] == i) {
        self = 1;
        CHECK(bins[e] == 0);
      }
    }
    CHECK(self);
  }
  /* unknown flags */
  delimit_lsc_geometry* gx = NULL;
  CHECK(delimit_lsc_geometry_create(b, 4, 1, 0.4, 2, 6, DELIMIT_WINDOW_SAME, 0x100u, &gx) == DELIMIT_ERR_INVALID_ARG);

  CHECK(strcmp(delimit_status_string(DELIMIT_ERR_WORKSPACE), "workspace too small") == 0);
  CHECK(delimit_lsc_geometry_destroy(gn) == DELIMIT_OK);
  CHECK(delimit_lsc_geometry_destroy(g) == DELIMIT_OK);
  CHECK(delimit_sh_basis_destroy(b) == DELIMIT_OK);
  printf("c abi ok\n");
  return 0;
}
