/* A plain C99 client of libhsvd (include/hsvd.h).
 *
 * factor_on_device() is a complete use of the library on a device matrix:
 * plan, run, status, factors copied to host buffers, destroy.  It needs a
 * GPU and is only compiled and linked here.  main() calls the entry points
 * that need no device (the schedule helpers, the error strings, argument
 * validation, which rejects bad plans before any device work) and prints
 * "ok" when they behave as the header documents. */
#include <stdio.h>
#include <string.h>

#include "hsvd.h"

int factor_on_device(const float* dA, int64_t m, int64_t n, float* U, float* S, float* V, int32_t* rank,
                     void* stream) {
  hsvd_plan_t plan = NULL;
  const int64_t ms[1] = {m}, ns[1] = {n}, lda[1] = {n};
  const void* inputs[1] = {dA};
  hsvd_report rep;
  hsvd_status st = hsvd_plan(&plan, 1, ms, ns, 512, 512, HSVD_TRUNC_FIXED_K, 64.0, 64, HSVD_TREE_COL_THEN_ROW,
                             HSVD_PREC_BF16_MIXED, HSVD_DTYPE_F32, NULL);
  if (st != HSVD_OK) return (int)st;
  st = hsvd_run(plan, inputs, lda, stream);
  if (st == HSVD_OK) st = hsvd_status_query(plan, 1, &rep);
  if (st == HSVD_OK && (rep.nonfinite || rep.tensor_timeouts)) st = HSVD_ECUDA;
  /* column-major U (m x rank) and V (n x rank), descending S */
  if (st == HSVD_OK) st = hsvd_factors(plan, 0, rank, U, m, S, V, n, HSVD_WHERE_HOST, stream);
  if (st != HSVD_OK) fprintf(stderr, "hsvd: %s %s\n", hsvd_error_string(st), hsvd_last_error(plan));
  hsvd_destroy(plan);
  return (int)st;
}

static int check_jacobi_rounds(int32_t n) {
  /* every pair of the n columns appears once over the n - 1 rounds */
  static int seen[64][64];
  int32_t r, s, p, q;
  memset(seen, 0, sizeof(seen));
  for (r = 0; r < n - 1; ++r)
    for (s = 0; s < n / 2; ++s) {
      if (hsvd_jacobi_pair(n, r, s, &p, &q) != HSVD_OK) return 0;
      if (p < 0 || q < 0 || p >= n || q >= n || p == q) return 0;
      seen[p < q ? p : q][p < q ? q : p] += 1;
    }
  for (p = 0; p < n; ++p)
    for (q = p + 1; q < n; ++q)
      if (seen[p][q] != 1) return 0;
  return hsvd_jacobi_pair(n, n - 1, 0, &p, &q) == HSVD_EINVAL;
}

int main(void) {
  const int64_t m[1] = {64}, n[1] = {64};
  hsvd_plan_t plan = NULL;
  hsvd_status st;
  if (hsvd_tree_levels(1) != 0 || hsvd_tree_levels(2) != 1 || hsvd_tree_levels(3) != 2 ||
      hsvd_tree_levels(7) != 3 || hsvd_tree_levels(64) != 6 || hsvd_tree_levels(0) != -1) {
    printf("tree levels\n");
    return 1;
  }
  if (!check_jacobi_rounds(8) || !check_jacobi_rounds(64)) {
    printf("jacobi pairs\n");
    return 2;
  }
  if (strcmp(hsvd_error_string(HSVD_OK), "") == 0 || strcmp(hsvd_error_string(HSVD_EINVAL), "") == 0) {
    printf("error strings\n");
    return 3;
  }
  /* gamma must lie in (0, 1): rejected before any allocation, plan stays NULL */
  st = hsvd_plan(&plan, 1, m, n, 32, 32, HSVD_TRUNC_GAMMA, 1.5, 8, HSVD_TREE_COL_THEN_ROW, HSVD_PREC_F32,
                 HSVD_DTYPE_F32, NULL);
  if (st != HSVD_EINVAL || plan != NULL) {
    printf("plan validation\n");
    return 4;
  }
  hsvd_destroy(NULL);
  if (hsvd_workspace_bytes(NULL) != 0 || hsvd_launches_per_run(NULL) != -1) {
    printf("null plan queries\n");
    return 5;
  }
  printf("ok\n");
  return 0;
}
