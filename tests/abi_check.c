/* A plain C99 caller of libsubmat.so: the header compiles as C and the host-side entry
 * points (defaults, status strings, row sharding, argument validation) run without a GPU.
 * Built and run by tests/test_abi_cpu.py. */
#include <stdio.h>
#include <string.h>

#include "submat.h"

static int failures = 0;
#define CHECK(cond)                                               \
  do {                                                            \
    if (!(cond)) {                                                \
      fprintf(stderr, "check failed at line %d: %s\n", __LINE__, #cond); \
      ++failures;                                                 \
    }                                                             \
  } while (0)

int main(void) {
  submat_opts o;
  submat_default_opts(&o);
  CHECK(o.k_max == 40 && o.root_sign == -1 && o.use_graph == 1);
  CHECK(strcmp(submat_status_string(SUBMAT_OK), "ok") == 0);
  CHECK(strlen(submat_status_string(SUBMAT_ETIMEOUT)) > 0);

  /* tridiag(1,2,1) of order 6: rows of 2, 3, 3, 3, 3, 2 entries */
  int32_t rowptr[7] = {0, 2, 5, 8, 11, 14, 16};
  int32_t colind[16] = {0, 1, 0, 1, 2, 1, 2, 3, 2, 3, 4, 3, 4, 5, 4, 5};
  int32_t b0, e0, b1, e1;
  CHECK(submat_shard_rows(6, rowptr, 2, 0, &b0, &e0) == SUBMAT_OK);
  CHECK(submat_shard_rows(6, rowptr, 2, 1, &b1, &e1) == SUBMAT_OK);
  CHECK(b0 == 0 && e0 == b1 && e1 == 6 && b1 > 0 && b1 < 6);
  CHECK(submat_shard_rows(6, rowptr, 2, 2, &b0, &e0) == SUBMAT_EINVAL);

  /* rejected on the host before any CUDA call */
  submat_csr csr = {6, 16, rowptr, colind, 0};
  submat_plan_t plan = NULL;
  CHECK(submat_plan(&csr, 0, NULL, &plan) == SUBMAT_EINVAL && plan == NULL);
  CHECK(strlen(submat_last_error()) > 0);
  int32_t bad_rowptr[7] = {0, 2, 5, 8, 11, 14, 15};    /* rowptr[n] != nnz */
  submat_csr bad = {6, 16, bad_rowptr, colind, 0};
  CHECK(submat_plan(&bad, 2, NULL, &plan) == SUBMAT_EINVAL && plan == NULL);
  CHECK(submat_invroot(NULL, NULL, NULL, NULL, 0) == SUBMAT_EINVAL);
  CHECK(submat_invroot_backward(NULL, NULL, NULL, NULL) == SUBMAT_EINVAL);
  submat_plan_destroy(NULL);

  if (failures) return 1;
  printf("abi_check ok\n");
  return 0;
}
