/* A plain C99 caller of libmf.so's host-side entry points (no GPU needed):
 * generate a rotor-stator mesh, read its sizes and arrays, write and read back
 * a checkpoint, and hit the argument checks.  Prints one line per check;
 * exits non-zero on the first failure.  Used by tests/test_library_c_abi.py. */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include "mf.h"

#define CHECK(c, msg) do { if (!(c)) { printf("FAIL %s\n", msg); return 1; } } while (0)

int main(int argc, char** argv) {
  const char* ckpt = argc > 1 ? argv[1] : "demo.ckpt";
  mf_mesh_params p;
  mf_mesh_params_defaults(&p);
  p.d = 3; p.k = 2; p.m = 4; p.n_r = 2; p.n_s = 2; p.n_z = 2; p.blades = 2;
  mf_mesh* m = NULL;
  CHECK(mf_mesh_rotor_stator(&p, &m) == MF_OK && m, "generate");
  int d = 0, k = 0, n_R = 0, n_z = 0;
  int64_t nn = 0, nc = 0;
  CHECK(mf_mesh_sizes(m, &d, &k, &nn, &nc, &n_R, &n_z) == MF_OK, "sizes");
  printf("sizes %d %d %lld %lld %d %d\n", d, k, (long long)nn, (long long)nc, n_R, n_z);

  uint8_t* wall = (uint8_t*)malloc((size_t)nn);
  int32_t* cells = (int32_t*)malloc((size_t)nc * 27 * sizeof(int32_t));
  CHECK(wall && cells && mf_mesh_read(m, NULL, NULL, wall, cells, NULL, NULL, NULL) == MF_OK, "read");
  long long moving = 0;
  for (int64_t i = 0; i < nn; ++i) moving += wall[i] == 2;
  printf("moving_wall_nodes %lld first_cell_node %d\n", moving, cells[0]);

  const int64_t nv = nn * (d + 1);
  double* un = (double*)malloc((size_t)nv * sizeof(double));
  double* um = (double*)malloc((size_t)nv * sizeof(double));
  double* a = (double*)malloc((size_t)nv * sizeof(double));
  double* b = (double*)malloc((size_t)nv * sizeof(double));
  for (int64_t i = 0; i < nv; ++i) { un[i] = 0.001 * (double)i - 3.0; um[i] = 1.0 / (1.0 + (double)i); }
  mf_checkpoint_info info = {2, 7, 0.014, 0.3, 0.002, 1e-3, 1.0}, got;
  CHECK(mf_checkpoint_write(ckpt, m, &info, un, um) == MF_OK, "checkpoint write");
  CHECK(mf_checkpoint_read(ckpt, m, &got, a, b) == MF_OK, "checkpoint read");
  CHECK(memcmp(a, un, (size_t)nv * sizeof(double)) == 0 && memcmp(b, um, (size_t)nv * sizeof(double)) == 0,
        "checkpoint arrays");
  CHECK(got.bdf == 2 && got.step == 7 && got.t == 0.014 && got.theta == 0.3, "checkpoint info");
  printf("checkpoint ok\n");

  mf_mesh_params bad = p;
  bad.k = 9;
  mf_mesh* m2 = NULL;
  CHECK(mf_mesh_rotor_stator(&bad, &m2) == MF_ERR_ARG && m2 == NULL, "bad k rejected");
  mf_mesh_params cp;
  CHECK(mf_mesh_coarsen_map(&p, &cp, NULL, NULL) == MF_OK && cp.m == 2 && cp.n_z == 1, "coarsen");
  printf("args ok\n");
  mf_mesh_free(m);
  free(wall); free(cells); free(un); free(um); free(a); free(b);
  return 0;
}
