/* A plain C99 consumer of the library: include/tenergy.h needs no C++ and
 * no CUDA header, and the exported symbols link and run.  Without a GPU
 * te_create reports TE_ECUDA; with one it creates and frees a handle and
 * rejects a descriptor with nocc = 0 before any launch. */
#include <stdio.h>
#include <string.h>

#include "tenergy.h"

int main(void) {
  te_handle h = NULL;
  te_status st = te_create(&h, 0, NULL);
  if (st != TE_OK) {
    printf("create %d %s\n", (int)st, te_last_error());
    return st == TE_ECUDA ? 0 : 1;
  }
  te_cluster c;
  memset(&c, 0, sizeof c);
  size_t bytes = 0;
  te_status ws = te_workspace_bytes(h, &c, TE_FP64, &bytes);
  printf("create 0; workspace of an empty descriptor %d %s\n", (int)ws, te_last_error());
  te_destroy(h);
  return ws == TE_EINVAL ? 0 : 1;
}
