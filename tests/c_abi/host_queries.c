/* A plain C99 caller of the library: the host-side entry points of include/lattice_ms.h used without
 * Python, torch or CUDA headers.  Reads d and the d x d entries of M (row-major) from the command line
 * and prints what the plan reports, one item per line:
 *   rc <status>                   (and "err <message>" when the status is not LAT_OK)
 *   info <m> <d_M> <e_1> .. <e_d>
 *   layout <nax> <split> <ax_len...>
 *   ws <bytes for 2 load cases, binary64> <the same with the conjugate-gradient vectors>
 *   point <p_1> .. <p_d>          (m lines, plan order)
 *   freq <h_1> .. <h_d>           (m lines, spectral order)
 */
#include <stdio.h>
#include <stdlib.h>

#include "lattice_ms.h"

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  const int d = atoi(argv[1]);
  if (d < 1 || d > 3 || argc != 2 + d * d) return 2;
  int64_t M[9];
  for (int i = 0; i < d * d; ++i) M[i] = (int64_t)atoll(argv[2 + i]);
  lat_plan* plan = NULL;
  const int rc = lattice_plan(M, d, &plan);
  printf("rc %d\n", rc);
  if (rc != LAT_OK) {
    printf("err %s\n", lattice_last_error());
    return plan == NULL ? 0 : 3;   /* a failed call leaves no plan */
  }
  int64_t m = 0, e[3] = {0, 0, 0};
  int d_M = 0;
  if (lattice_plan_info(plan, &m, &d_M, e) != LAT_OK) return 4;
  printf("info %lld %d", (long long)m, d_M);
  for (int j = 0; j < d; ++j) printf(" %lld", (long long)e[j]);
  printf("\n");
  int nax = 0, ng = 0, split = 0, ax[6], grp[6];
  if (lattice_plan_layout(plan, &nax, ax, &ng, grp, &split) != LAT_OK) return 5;
  printf("layout %d %d", nax, split);
  for (int j = 0; j < nax; ++j) printf(" %d", ax[j]);
  printf("\n");
  printf("ws %zu %zu\n", lattice_workspace_bytes(plan, 2, LAT_FP64),
         lattice_workspace_bytes(plan, 2, LAT_FP64 | LAT_WS_CG));
  int64_t* p = (int64_t*)malloc((size_t)m * d * sizeof(int64_t));
  int64_t* h = (int64_t*)malloc((size_t)m * d * sizeof(int64_t));
  if (!p || !h) return 6;
  if (lattice_points(plan, p) != LAT_OK || lattice_freqs(plan, h) != LAT_OK) return 7;
  for (int64_t i = 0; i < m; ++i) {
    printf("point");
    for (int j = 0; j < d; ++j) printf(" %lld", (long long)p[i * d + j]);
    printf("\nfreq");
    for (int j = 0; j < d; ++j) printf(" %lld", (long long)h[i * d + j]);
    printf("\n");
  }
  free(p);
  free(h);
  lattice_plan_destroy(plan);
  lattice_plan_destroy(NULL);   /* NULL is ignored */
  return 0;
}
