/* A plain C99 client of libmbf (include/mbf.h), compiled and run by
 * tests/test_c_abi_cpu.py: the host side of the boundary without Python.
 *   1. build the factors of a 2-D DFT problem with a caller-written entry function
 *      (Case (ii) of §1.1: the kernel is given by its entries), checkpointed to a file;
 *   2. build again with the same file (loaded, not rebuilt) and compare the two sets;
 *   3. create an operator: MBF_OK on a machine with a GPU, MBF_ERR_CUDA without one
 *      (there is no CPU apply);
 *   4. error handling: NULL arguments and a missing file return codes and messages.
 * Prints one line per check; exits non-zero if any check fails. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "mbf.h"

static int fails = 0;
#define CHECK(cond, what)                                                   \
  do {                                                                      \
    if (cond) {                                                             \
      printf("ok   %s\n", what);                                            \
    } else {                                                                \
      printf("FAIL %s (%s)\n", what, mbf_last_error());                     \
      ++fails;                                                              \
    }                                                                       \
  } while (0)

/* exp(-2 pi i x.xi), the kernel of the discrete Fourier transform (§1.1) */
static void dft_entries(const double* x, int64_t m, const double* xi, int64_t n, int32_t dim, double* out,
                        void* ctx) {
  const double two_pi = 6.283185307179586;
  int64_t a, b;
  int k;
  (void)ctx;
  for (b = 0; b < n; ++b)
    for (a = 0; a < m; ++a) {
      double ph = 0.0;
      for (k = 0; k < dim; ++k) ph += x[a * dim + k] * xi[b * dim + k];
      out[2 * (a + m * b)] = cos(two_pi * ph);
      out[2 * (a + m * b) + 1] = -sin(two_pi * ph);
    }
}

static int same_factors(const mbf_factors_t* p, const mbf_factors_t* q) {
  const int64_t c = (int64_t)1 << p->dim;
  int64_t nL = 1, ul, vl, l;
  int i;
  if (p->dim != q->dim || p->L != q->L || p->n_out != q->n_out || p->n_in != q->n_in || p->n_w != q->n_w ||
      p->max_leaf_x != q->max_leaf_x || p->max_leaf_w != q->max_leaf_w || p->nnz != q->nnz)
    return 0;
  for (i = 0; i < p->L; ++i) nL *= c;
  if (memcmp(p->RU, q->RU, sizeof(int32_t) * (size_t)(p->L + 1)) ||
      memcmp(p->RV, q->RV, sizeof(int32_t) * (size_t)(p->L + 1)))
    return 0;
  if (memcmp(p->x_perm, q->x_perm, sizeof(int64_t) * (size_t)p->n_out) ||
      memcmp(p->w_off, q->w_off, sizeof(int64_t) * (size_t)(nL + 1)))
    return 0;
  ul = nL * p->max_leaf_x * p->RU[p->L];
  vl = nL * p->max_leaf_w * p->RV[p->L];
  if (memcmp(p->UL, q->UL, 16 * (size_t)ul) || memcmp(p->VL, q->VL, 16 * (size_t)vl)) return 0;
  for (l = p->L / 2; l < p->L; ++l) {
    const int64_t g = nL * c * (int64_t)p->RU[l + 1] * p->RU[l];
    if (memcmp(p->G[l - p->L / 2], q->G[l - p->L / 2], 16 * (size_t)g)) return 0;
  }
  return 1;
}

int main(int argc, char** argv) {
  mbf_problem_t prob;
  mbf_build_opts_t opts;
  mbf_factors_h f1 = NULL, f2 = NULL, f3 = NULL;
  mbf_factors_t v1, v2;
  mbf_op_t op = NULL;
  int s;
  if (argc < 2) {
    fprintf(stderr, "usage: %s <factor file path>\n", argv[0]);
    return 2;
  }
  printf("%s\n", mbf_version());
  memset(&prob, 0, sizeof prob);
  prob.dim = 2;
  prob.n = 16;
  prob.L = 2;
  prob.r = 8;
  prob.tree = MBF_TREE_UNIFORM;
  memset(&opts, 0, sizeof opts);
  opts.seed = 5;
  opts.factor_file = argv[1];

  CHECK(mbf_build_factors(&prob, dft_entries, NULL, &opts, &f1) == MBF_OK, "build with a C entry function");
  CHECK(f1 && mbf_factors_view(f1, &v1) == MBF_OK && v1.n_out == 256 && v1.nnz > 0, "factor view");
  CHECK(mbf_build_factors(&prob, dft_entries, NULL, &opts, &f2) == MBF_OK, "second build loads the checkpoint");
  CHECK(f2 && mbf_factors_view(f2, &v2) == MBF_OK && same_factors(&v1, &v2), "checkpoint is bit-identical");
  CHECK(mbf_factors_load(argv[1], &f3) == MBF_OK, "load the factor file");
  if (f3) mbf_factors_destroy(f3);
  f3 = NULL;

  s = mbf_op_create(&v1, &op);
  CHECK(s == MBF_OK || s == MBF_ERR_CUDA, "operator creation: MBF_OK with a GPU, MBF_ERR_CUDA without");
  printf("op_create status %d\n", s);
  if (s == MBF_OK) CHECK(mbf_op_destroy(op) == MBF_OK, "destroy");

  CHECK(mbf_build_factors(NULL, dft_entries, NULL, &opts, &f3) == MBF_ERR_INVALID, "NULL problem");
  CHECK(strlen(mbf_last_error()) > 0, "error message");
  CHECK(mbf_factors_load("/nonexistent/dir/f.mbf", &f3) == MBF_ERR_IO, "missing factor file");
  CHECK(mbf_factors_save(&v1, "/nonexistent/dir/f.mbf") == MBF_ERR_IO, "unwritable path");

  mbf_factors_destroy(f1);
  mbf_factors_destroy(f2);
  printf("%d failed\n", fails);
  return fails ? 1 : 0;
}
