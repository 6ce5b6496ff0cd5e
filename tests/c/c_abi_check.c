/* Plain C99 client of the library's C ABI (no C++, no torch): includes the public header,
 * links against libcs_gb300.so and calls the host-only entry points, so the header and the
 * exported symbols are checked from C.  With a GPU it also creates an operator and applies it. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "cs_gb300.h"

int main(int argc, char** argv) {
  const int64_t N = 4096, M = 1024;
  int32_t* omega = (int32_t*)malloc(sizeof(int32_t) * (size_t)M);
  int8_t* d = (int8_t*)malloc((size_t)N);
  int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
  if (!omega || !d || !perm) return 2;
  if (cs_operator_draws(N, M, 0x0C5001u, omega, d) != CS_OK) {
    fprintf(stderr, "draws: %s\n", cs_last_error());
    return 1;
  }
  for (int64_t i = 1; i < M; ++i)
    if (omega[i] <= omega[i - 1]) return 1;   /* sorted, distinct */
  for (int64_t n = 0; n < N; ++n)
    if (d[n] != 1 && d[n] != -1) return 1;
  if (cs_operator_perm(N, 7u, perm) != CS_OK) return 1;
  /* an unsupported size is refused with a message */
  if (cs_operator_draws(4097, 8, 1u, omega, NULL) != CS_ERR_UNSUPPORTED_N || strlen(cs_last_error()) == 0) return 1;
  /* the batched selection checks its arguments on the host; an empty batch is a no-op */
  if (cs_select_topk_batched(1, 16, 17, (const float*)16, NULL, (int32_t*)16, NULL) != CS_ERR_INVALID_ARG) return 1;
  if (cs_select_topk_batched(0, 16, 4, NULL, NULL, NULL, NULL) != CS_OK) return 1;
  if (cs_launch_count() < 0) return 1;
  printf("omega[0]=%d omega[M-1]=%d d[0]=%d perm[0]=%d launches=%lld\n", (int)omega[0], (int)omega[M - 1], (int)d[0],
         (int)perm[0], (long long)cs_launch_count());
  if (argc > 1 && strcmp(argv[1], "--gpu") == 0) {
    cs_op_t op = cs_op_create(N, M, 0x0C5001u);
    if (!op) {
      fprintf(stderr, "create: %s\n", cs_last_error());
      return 1;
    }
    cs_op_destroy(op);
  }
  free(omega);
  free(d);
  free(perm);
  return 0;
}
