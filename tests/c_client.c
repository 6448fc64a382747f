/* A plain C client of libstrom: builds the running example (Example 1, the
 * 1-D toy system, N = 3) from polynomial data through the C ABI only,
 * relaxes it, exports and re-imports the SDP, and exercises the host-only
 * calls (neighbour selection, moment rank test). It prints one line per
 * result for the test that compiles and runs it; solver calls need a GPU and
 * are only checked for a clean status. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "strom.h"

#define NV 3 /* clique variables (x_{k-1}, u_{k-1}, x_k) */

/* a polynomial with at most 8 terms in NV variables */
typedef struct {
  int n;
  double c[8];
  uint8_t e[8 * NV];
} poly;

static void term(poly* p, double c, int a, int b, int d) {
  p->c[p->n] = c;
  p->e[p->n * NV + 0] = (uint8_t)a;
  p->e[p->n * NV + 1] = (uint8_t)b;
  p->e[p->n * NV + 2] = (uint8_t)d;
  p->n++;
}

static strom_poly view(const poly* p) {
  strom_poly s;
  s.nterms = p->n;
  s.coef = p->c;
  s.expo = p->e;
  return s;
}

int main(void) {
  const int N = 3;
  const double dt = 0.1, Pf = 1.0, x_init = 2.0;
  poly f[3], g[3], h[3][2];
  strom_poly gv[3], hv[3][2];
  strom_clique cl[3];
  memset(f, 0, sizeof f);
  memset(g, 0, sizeof g);
  memset(h, 0, sizeof h);
  for (int k = 0; k < N; ++k) {
    term(&f[k], 1.0, 0, 2, 0); /* u^2 */
    term(&f[k], 1.0, 2, 0, 0); /* x_{k-1}^2 */
    if (k == N - 1) term(&f[k], Pf, 0, 0, 2);
    term(&g[k], 1.0, 0, 0, 0); /* 1 - u^2 */
    term(&g[k], -1.0, 0, 2, 0);
    term(&h[k][0], 1.0, 0, 0, 1); /* x_k + (dt - 1) x_{k-1} + dt u x_{k-1} */
    term(&h[k][0], dt - 1.0, 1, 0, 0);
    term(&h[k][0], dt, 1, 1, 0);
    gv[k] = view(&g[k]);
    hv[k][0] = view(&h[k][0]);
    int nh = 1;
    if (k == 0) { /* x_0 - x_init */
      term(&h[k][1], 1.0, 1, 0, 0);
      term(&h[k][1], -x_init, 0, 0, 0);
      hv[k][1] = view(&h[k][1]);
      nh = 2;
    }
    cl[k].f = view(&f[k]);
    cl[k].ng = 1;
    cl[k].g = &gv[k];
    cl[k].nh = nh;
    cl[k].h = hv[k];
  }
  strom_problem_desc d = {N, 1, 1, 2, x_init, cl};
  strom_problem* prob = NULL;
  int st = strom_problem_create(&d, &prob);
  printf("problem_create %d\n", st);
  if (st != STROM_OK) return 1;
  strom_sdp* sdp = NULL;
  st = strom_relax(prob, &sdp);
  printf("relax %d\n", st);
  if (st != STROM_OK) return 1;
  strom_sdp_info info;
  strom_sdp_info_get(sdp, &info);
  printf("info nblocks %d nsvec %lld m %lld nnz %lld kinds %lld %lld %lld %lld %lld\n", info.nblocks,
         (long long)info.nsvec, (long long)info.m, (long long)info.nnz, (long long)info.rows_by_kind[0],
         (long long)info.rows_by_kind[1], (long long)info.rows_by_kind[2], (long long)info.rows_by_kind[3],
         (long long)info.rows_by_kind[4]);

  /* export, then import the same arrays */
  int32_t* bn = malloc(sizeof(int32_t) * info.nblocks);
  int8_t* bk = malloc(info.nblocks);
  int32_t* bc = malloc(sizeof(int32_t) * info.nblocks);
  double* C = malloc(sizeof(double) * info.nsvec);
  int64_t* rp = malloc(sizeof(int64_t) * (info.m + 1));
  int32_t* col = malloc(sizeof(int32_t) * info.nnz);
  double* val = malloc(sizeof(double) * info.nnz);
  double* b = malloc(sizeof(double) * info.m);
  int8_t* rk = malloc(info.m);
  int32_t* rc = malloc(sizeof(int32_t) * info.m);
  st = strom_sdp_export(sdp, bn, NULL, bk, bc, C, rp, col, val, b, rk, rc);
  strom_sdp_desc in = {N, 1, 1, info.nblocks, bn, bk, bc, NULL, C, info.m, rp, col, val, b, rk, rc};
  strom_sdp* again = NULL;
  int st2 = strom_sdp_import(&in, &again);
  strom_sdp_info info2;
  if (st2 == STROM_OK) strom_sdp_info_get(again, &info2);
  printf("export %d import %d same %d\n", st, st2,
         st2 == STROM_OK && info2.nsvec == info.nsvec && info2.m == info.m && info2.nnz == info.nnz);
  /* a malformed import: a consensus row in the last clique */
  rk[info.m - 1] = STROM_ROW_CONS;
  strom_sdp* bad = NULL;
  printf("bad_import %d\n", strom_sdp_import(&in, &bad));

  /* neighbour selection on a unit square of keys */
  const double keys[8] = {0, 0, 1, 0, 0, 1, 1, 1};
  const double q[2] = {0.2, 0.3};
  int32_t idx[3];
  double wt[3];
  int32_t k = 0;
  st = strom_warm_select(keys, 4, 2, q, idx, wt, &k);
  printf("warm_select %d k %d idx %d %d %d wt %.6f %.6f %.6f\n", st, k, idx[0], idx[1], idx[2], wt[0], wt[1],
         wt[2]);

  /* rank test of the rank-1 lifting of z = (0.5, -0.25, 0.75): basis
   * 1, z1, z2, z3, z1^2, z1 z2, z1 z3, z2^2, z2 z3, z3^2 */
  const double z[3] = {0.5, -0.25, 0.75};
  double v[10] = {1, z[0], z[1], z[2], z[0] * z[0], z[0] * z[1], z[0] * z[2], z[1] * z[1], z[1] * z[2], z[2] * z[2]};
  double M[100];
  for (int i = 0; i < 10; ++i)
    for (int j = 0; j < 10; ++j) M[j * 10 + i] = v[i] * v[j];
  strom_rank_test rt;
  double zb[3];
  st = strom_moment_rank_test(M, 3, NULL, 1e-8, &rt, zb);
  printf("rank_test %d rank %d flat %d zbar %.6f %.6f %.6f\n", st, rt.rank, rt.flat, zb[0], zb[1], zb[2]);

  /* the solver needs a GPU: a clean status either way */
  strom_options opt;
  strom_options_default(&opt);
  strom_solver* sv = NULL;
  const strom_sdp* list[1] = {sdp};
  st = strom_solver_create(list, 1, &opt, &sv);
  printf("solver_create %s\n", st == STROM_OK ? "ok" : (st == STROM_ERR_CUDA ? "cuda-unavailable" : "error"));
  if (sv) strom_solver_destroy(sv);

  strom_sdp_destroy(again);
  strom_sdp_destroy(sdp);
  strom_problem_destroy(prob);
  free(bn); free(bk); free(bc); free(C); free(rp); free(col); free(val); free(b); free(rk); free(rc);
  return 0;
}
