/*
 * mbf.h -- C ABI of the GB300 butterfly-factorization apply library (libmbf.so).
 *
 * The library applies a multidimensional butterfly factorization (BF)
 *     K ~ U^L G^{L-1} ... G^h M^h (H^h)^* ... (H^{L-1})^* (V^L)^*,   h = L/2,
 * of a complementary low-rank kernel matrix K = (K(x, xi))_{x in X, xi in Omega}
 * (Li, Yang & Ying, "Multidimensional Butterfly Factorization", §1.1 eq. (GBF),
 * §2.3 eq. (gbf)) to vectors on one GPU, and its adjoint K^*.  Factors are built
 * once on the host in FP64 (§2.3 middle level by SVD via random sampling, §2.1;
 * §2.4 recursive factorization), packed into a per-level tile layout and kept
 * resident in device memory.
 *
 * Conventions shared by every call:
 *   - Points.  X = {(n_1/n, .., n_d/n)}, Omega = {(n_1, .., n_d) : -n/2 <= n_k < n/2}
 *     (§1.1, eqs. X, Omega).  Natural index of x: sum_k n_k n^(d-1-k); of xi:
 *     sum_k (xi_k + n/2) n^(d-1-k) (row-major).
 *   - Vectors.  Complex single precision, interleaved (re, im) float pairs, laid out
 *     [nrhs][N] in natural order.  Device pointers unless a call says "host".
 *   - Ownership.  Callers own every buffer they pass; the library never frees them.
 *     Handles returned by *_create / *_build own their memory until *_destroy.
 *   - Errors.  Every call returns an mbf_status (MBF_OK = 0).  No exception crosses
 *     the ABI.  mbf_last_error() returns a thread-local message for the last failure.
 *   - Streams.  `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Applies are asynchronous with respect to the host.
 */
#ifndef MBF_H
#define MBF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum mbf_status {
  MBF_OK = 0,
  MBF_ERR_INVALID = 1,   /* bad argument, unsupported size or layout            */
  MBF_ERR_OOM = 2,       /* host or device allocation failed                    */
  MBF_ERR_CUDA = 3,      /* a CUDA runtime call failed                          */
  MBF_ERR_BUSY = 4,      /* server has no free slot or memory budget right now  */
  MBF_ERR_TIMEOUT = 5,   /* a device-side wait ran past its limit; see status   */
  MBF_ERR_IO = 6,        /* factor file could not be read or written            */
  MBF_ERR_NOT_FOUND = 7  /* unknown ticket                                      */
} mbf_status;

typedef enum mbf_tree_kind {
  MBF_TREE_UNIFORM = 0,  /* Omega tree over the uniform grid (§2.2)                     */
  MBF_TREE_POLAR = 1,    /* Omega tree over the polar image p(xi) in [0,1]^2 (§3.1-3.2)  */
  MBF_TREE_SQUARE = 2,   /* Omega tree over a square holding an explicit point subset,   */
                         /* e.g. one corona Omega_t of the multiscale split (§4.2)        */
  MBF_TREE_POINTS = 3    /* explicit non-uniform point sets on both sides (§2.6): the X  */
                         /* tree over x_pts in [0,1)^dim, the Omega tree over w_pts in   */
                         /* the square [w_lo, w_lo + w_side)^dim; empty nodes kept as     */
                         /* zero-point nodes; natural order = the order of the arrays     */
} mbf_tree_kind;

typedef enum mbf_precision {
  MBF_PREC_AUTO = 0,     /* FP32 SIMT for nrhs < 8 (or the tuner's crossover), split-  */
                         /* BF16x3 tensor path otherwise; an operator whose leaf groups */
                         /* exceed the SIMT kernel's limits takes the tensor path for  */
                         /* any nrhs                                                    */
  MBF_PREC_FP32_SIMT = 1,/* complex64 factors, FP32 FMA, FP32 accumulate; returns      */
                         /* MBF_ERR_INVALID on such an operator                         */
  MBF_PREC_TF32 = 2,     /* tensor cores, TF32-rounded operands, FP32 accumulate       */
                         /* (forward only; about 1e-3 relative error; never AUTO)      */
  MBF_PREC_BF16X3 = 3    /* tensor cores, split-BF16 (hi*hi + hi*lo + lo*hi), FP32 acc  */
} mbf_precision;

/* Problem description for the builder (§1.1 and §2.2). */
typedef struct mbf_problem {
  int32_t dim;          /* d = 2 or 3                                                   */
  int32_t n;            /* grid points per axis, a power of two                          */
  int32_t L;            /* tree depth: even, 2 <= L <= log2(n) for the X tree            */
  int32_t r;            /* maximum rank r of every low-rank block                        */
  int32_t tree;         /* mbf_tree_kind for the Omega side; the X tree is uniform        */
  int32_t reserved0;
  /* MBF_TREE_SQUARE only: the Omega points kept (natural indices, host, n_w entries)
   * and the square [w_lo, w_lo + w_side)^d, in frequency units, that roots the tree. */
  int64_t n_w;
  const int64_t* w_index;
  double w_lo;
  double w_side;
  /* MBF_TREE_POINTS only: the point sets themselves (host, row-major [count][dim]):
   * X points in [0,1)^dim, Omega points (frequencies) in [w_lo, w_lo + w_side)^dim.
   * n is not used for them; the operator maps vectors of n_w_pts to vectors of n_x_pts. */
  int64_t n_x_pts;
  const double* x_pts;
  int64_t n_w_pts;
  const double* w_pts;
} mbf_problem_t;

/* Kernel entry evaluation, Case (ii) of §1.1: fill the m x n block
 *   out[2*(a + m*b) + 0/1] = Re/Im K(x_a, xi_b),  a < m, b < n  (column-major)
 * x: host [m][dim] doubles in [0,1)^d; xi: host [n][dim] doubles (integer-valued).
 * Called from several host threads at once; must be thread safe. */
typedef void (*mbf_entry_fn)(const double* x, int64_t m, const double* xi, int64_t n,
                             int32_t dim, double* out, void* ctx);

/* Built-in kernels (ctx unused):
 *  mbf_kernel_dft       exp(-2 pi i x.xi)                               (§1.1)
 *  mbf_kernel_fio_iso   exp(2 pi i (x.xi + c(x)|xi|)),
 *                       c(x) = (2 + sin 2pi x_1 sin 2pi x_2)/16           (§3.3, c_1 = c_2)
 *  mbf_kernel_fio_ellip exp(2 pi i (x.xi + sqrt(c_1^2 xi_1^2 + c_2^2 xi_2^2))), eq. example1phi */
void mbf_kernel_dft(const double* x, int64_t m, const double* xi, int64_t n, int32_t dim,
                    double* out, void* ctx);
void mbf_kernel_fio_iso(const double* x, int64_t m, const double* xi, int64_t n, int32_t dim,
                        double* out, void* ctx);
void mbf_kernel_fio_ellip(const double* x, int64_t m, const double* xi, int64_t n, int32_t dim,
                          double* out, void* ctx);

typedef struct mbf_build_opts {
  uint64_t seed;        /* per-block generators are seeded from (seed, side, i, j)        */
  int32_t sample_factor;/* sample sets of size sample_factor * r (default 3)              */
  int32_t max_rounds;   /* representative-set iterations of §2.1 (default 3)              */
  double tol;           /* drop singular values below tol * sigma_1 (default 1e-14)       */
  int32_t threads;      /* host threads (0 = all cores)                                   */
  int32_t reserved;
  /* Optional checkpoint (NULL: none).  If a factor file exists at this path it is loaded
   * instead of building (its dim, L, sizes, Omega point set and ranks <= r are checked
   * against the problem, and 16 kernel entries recorded in `path`.kernel against the
   * entry function: MBF_ERR_INVALID on a mismatch or a missing record); otherwise the
   * factors are built and written there with their kernel record.  The seed and the
   * options are not recorded: name one file per (seed, options).  mbf_build_msbf uses
   * `path`.t<k> for corona k. */
  const char* factor_file;
} mbf_build_opts_t;

/* Padded FP64 factor set: the interchange layout shared by the builder, the packer
 * and factor import.  c = 2^dim, h = L/2.  Complex arrays are interleaved doubles.
 * Blocks of one level share a padded rank R; entries beyond a block's true rank,
 * or beyond a leaf's true point count, are zero.  Host memory throughout.
 *   x_perm[n_out]  tree order -> natural index of X; x_off[c^L + 1] leaf offsets
 *   w_perm[n_w]    tree order -> natural index into the input vector; w_off[c^L + 1]
 *   RU[L+1], RV[L+1]  padded ranks of levels h..L on the X / Omega side (RU[h] == RV[h])
 *   UL  [c^L][max_leaf_x][RU[L]]   rows of U^L_i (eq. expression-U at level L)
 *   VL  [c^L][max_leaf_w][RV[L]]   rows of V^L_j
 *   G[l-h]  [c^l][c^(L-l-1)][c][RU[l+1]][c][RU[l]]  : G[..][i][jp][t][k2][tp][k] is entry
 *           (k2, k) of column block tp of G^l_{c i + t, jp} (eq. RSh2), l = h..L-1
 *   H[l-h]  same shape with RV: blocks H^l_{c j + t, ip} of eq. (VF)
 *   S   [c^h][c^h][RU[h]] real: diagonal of S^h_{i,j} (eq. Kij, form of eq. lowrank1) */
typedef struct mbf_factors {
  int32_t dim, L;
  int64_t n_out, n_in, n_w;
  const int64_t* x_perm;
  const int64_t* x_off;
  const int64_t* w_perm;
  const int64_t* w_off;
  const int32_t* RU;
  const int32_t* RV;
  int32_t max_leaf_x, max_leaf_w;
  const double* UL;
  const double* VL;
  const double* const* G;
  const double* const* H;
  const double* S;
  int64_t nnz;          /* algorithmic nonzeros (true ranks, no padding); 0 if unknown */
} mbf_factors_t;

typedef struct mbf_factors_s* mbf_factors_h;  /* host FP64 factors owned by the library */
typedef struct mbf_op_s* mbf_op_t;            /* device-resident packed operator        */
typedef struct mbf_server_s* mbf_server_t;    /* serving loop                           */
typedef struct mbf_msbf_s* mbf_msbf_t;        /* multiscale factorization (§4)          */

/* Products with the operator, Case (i) of §1.1: out = K in (adjoint = 0) or out = K^* in
 * (adjoint = 1) for nrhs vectors; host, complex FP64 interleaved, laid out [nrhs][len]
 * in natural order (in: n_in, out: n_out for K; the reverse for K^*).  Called from one
 * host thread at a time. */
typedef void (*mbf_apply_fn)(const double* in, double* out, int64_t nrhs, int32_t adjoint, void* ctx);

/* Build the FP64 factors of an operator known only through products with K and K^*
 * (Case (i) of §1.1; PBF-m / MBF-m of §3.3, §4.3): the middle level by the SVD via
 * random matrix-vector multiplication (§2.1) of every block K^h_{i,j}, from K applied
 * to the zero-padded Gaussian matrices C^P_j (r + 8 columns per Omega node j) and K^*
 * to R^P_i (§2.3); the recursion as for mbf_build_factors.  prob as for
 * mbf_build_factors (uniform or polar Omega tree, or explicit point sets); opts.seed
 * seeds the Gaussian matrices; the factor_file option is not used.  2 c^h (r + 8)
 * products in all, in calls of at most 256 vectors. */
mbf_status mbf_build_from_applies(const mbf_problem_t* prob, mbf_apply_fn fn, void* ctx,
                                  const mbf_build_opts_t* opts, mbf_factors_h* out);

/* Build the FP64 factors on the host (§2.3-2.4, Case (ii)); threads per opts.
 * The builder keeps O(N log N) memory by recomputing each middle-level block for the
 * V side instead of storing U^h, V^h (§2.5, interleaved construction). */
mbf_status mbf_build_factors(const mbf_problem_t* prob, mbf_entry_fn fn, void* ctx,
                             const mbf_build_opts_t* opts, mbf_factors_h* out);
/* Read-only view of built factors (pointers valid until mbf_factors_destroy). */
mbf_status mbf_factors_view(mbf_factors_h f, mbf_factors_t* view);
mbf_status mbf_factors_destroy(mbf_factors_h f);

/* Factor files: the checkpoint of the host construction, so that the FP64 build runs
 * once and later processes load its result.  mbf_factors_save writes a factor set
 * (validated first, MBF_ERR_INVALID if inconsistent) to `path`: a 64-byte header
 * (magic, version, byte-order tag, dim, L, sizes, nnz), the arrays of mbf_factors_t in
 * their order above, and a checksum; it writes `path`.tmp and renames it, so `path` never
 * holds a partial file.  mbf_factors_load reads such a file into library-owned host
 * factors (free with mbf_factors_destroy).  A missing, truncated, foreign or corrupt
 * file, or a failed write, returns MBF_ERR_IO.  Host only; no device is needed. */
mbf_status mbf_factors_save(const mbf_factors_t* f, const char* path);
mbf_status mbf_factors_load(const char* path, mbf_factors_h* out);

/* Pack a factor set (built here or supplied by the caller) into the device tile
 * layout on the current CUDA device and return a resident operator.  The factor
 * arrays are only read during the call. */
mbf_status mbf_op_create(const mbf_factors_t* f, mbf_op_t* out);
/* The device bytes the packed factors of f will take, without a device: *simt_bytes the
 * FP32 SIMT arena and its item table, *tensor_bytes the split-BF16 tiles (0 when the
 * tensor path cannot take the operator).  The tensor adjoint adds tensor_bytes again on
 * its first use, TF32 applies likewise; workspaces come on top.  Packs on the host to
 * count (host memory and time of the packing itself).  Either pointer may be NULL. */
mbf_status mbf_factors_device_bytes(const mbf_factors_t* f, int64_t* simt_bytes, int64_t* tensor_bytes);
/* mbf_build_factors + mbf_op_create + mbf_factors_destroy, then the error estimate
 * below on 256 sampled outputs (needs the device; kept for mbf_op_info). */
mbf_status mbf_build_from_entries(const mbf_problem_t* prob, mbf_entry_fn fn, void* ctx,
                                  const mbf_build_opts_t* opts, mbf_op_t* out);
mbf_status mbf_op_destroy(mbf_op_t op);

typedef struct mbf_op_info {
  int32_t dim, L, c, n_stages;
  int64_t n_out, n_in;
  int32_t RU[32], RV[32];
  int64_t nnz_algorithmic;      /* nonzeros of the unpadded factors (the §2.5 apply cost):
                                   mbf_factors_t.nnz, or when that is 0 the nonzero
                                   entries the packer stored                             */
  int64_t bytes_algorithmic;    /* 8 * nnz_algorithmic (complex64)                        */
  int64_t bytes_packed;         /* device bytes of the packed tiles incl. padding         */
  int64_t bytes_stage[32];      /* packed bytes streamed by each forward stage            */
  int32_t grid, threads, smem;  /* persistent launch shape of the SIMT apply              */
  int64_t nnz_stage[32];        /* nonzero factor entries applied by each forward stage    */
  int64_t nnz_leaf_u;           /* of which U^L (part of the last stage)                  */
  int32_t tensor_ok;            /* 1 if the tensor-core path is available                 */
  int32_t tensor_stages;        /* G / H levels applied by the tensor-core kernel         */
  int64_t bytes_tensor;         /* device bytes of its split-bf16 tiles                   */
  int32_t tensor_smem, tensor_slots;  /* its shared memory per CTA and A-ring depth      */
  char tensor_unavailable[128]; /* why not, if tensor_ok == 0                             */
  double eps;                   /* error estimate against the direct sum (§3.3), -1 if none */
  int32_t eps_samples;          /* sampled outputs it was taken on                          */
  int32_t reserved_eps;
} mbf_op_info_t;
mbf_status mbf_op_info(mbf_op_t op, mbf_op_info_t* info);

/* Error estimate of the numerical sections (§3.3, §4.3): the relative L2 error
 *     e = sqrt( sum_{x in S} |u_f(x) - u(x)|^2 / sum_{x in S} |u(x)|^2 )
 * of the operator's result u_f = K_f g against the direct sum u = K g (§1.1, eq. kernel)
 * on n_samples distinct output points S.  g has iid complex standard normal entries on
 * the Omega points the operator covers (zero elsewhere); g and S are drawn from `seed`
 * by a counter-based generator (splitmix64).  u_f is one FP32 apply on the current
 * device on `stream` (synchronized; a device wait that gave up returns MBF_ERR_TIMEOUT);
 * u(x) is summed in FP64 on the host from entries of fn (as for the builder; called from
 * several threads).  The operator must be built on the grids X, Omega of eqs. (X),
 * (Omega) with n^d points.  Allocates two vectors on the device for the call.  The result
 * is written to *eps (if not NULL) and kept for mbf_op_info.  Grid problems only (the
 * operator keeps no point coordinates): mbf_build_from_entries skips it for
 * MBF_TREE_POINTS. */
mbf_status mbf_op_estimate_error(mbf_op_t op, mbf_entry_fn fn, void* ctx, int32_t n_samples,
                                 uint64_t seed, void* stream, double* eps);

/* u = K_f g (forward) for nrhs vectors.  g: device [nrhs][n_in] complex64, u: device
 * [nrhs][n_out] complex64 (fully overwritten).  Asynchronous on `stream`.  Calls on
 * one operator must not overlap on the device (they share its workspace); use the
 * server, or several operators, for concurrent applies.  A device wait that runs
 * out of time sets the operator's status word; mbf_op_check() reports it. */
mbf_status mbf_apply(mbf_op_t op, const void* g, void* u, int64_t nrhs, int32_t precision,
                     void* stream);
/* g = K_f^* u (adjoint): the same factors conjugate-transposed in reverse order.  On
 * the tensor cores (MBF_PREC_BF16X3, or AUTO from the tensor crossover) the tiles are
 * conjugate-transposed on the device on the first such call and kept (as much device
 * memory again as the forward tiles); MBF_PREC_TF32 is rejected for the adjoint. */
mbf_status mbf_apply_adjoint(mbf_op_t op, const void* u, void* g, int64_t nrhs,
                             int32_t precision, void* stream);
/* Same as mbf_apply but g and u are HOST buffers; synchronizes `stream` before
 * returning.  Page-locked buffers the device can address (cudaHostAlloc,
 * cudaHostRegister) are read and written by the tensor path's kernels across the host
 * link directly; other buffers are copied in and out through device staging buffers
 * (allocated on first use, kept by the operator). */
mbf_status mbf_apply_host(mbf_op_t op, const void* g_host, void* u_host, int64_t nrhs,
                          int32_t precision, void* stream);
/* u_b = K_f g_b for nbatch independent panels of nrhs vectors each, host buffers:
 * g_host [nbatch][nrhs][n_in] and u_host [nbatch][nrhs][n_out] complex64 (every panel
 * of u fully overwritten).  The panels are pipelined through two device staging pairs:
 * the copy engines bring panel b+1 in and take panel b-1 out while panel b is applied
 * on `stream`, so with page-locked buffers (cudaHostAlloc, cudaHostRegister) the
 * transfers overlap the apply (pageable buffers give the same result, serialised).
 * The staging pairs and the two copy streams are allocated on first use and kept by
 * the operator.  Synchronizes before returning, also after an error.  nbatch = 0 or
 * nrhs = 0 does nothing; MBF_ERR_INVALID for NULL buffers or negative counts.  Calls
 * on one operator must not overlap (they share its workspace and staging). */
mbf_status mbf_apply_host_batch(mbf_op_t op, const void* g_host, void* u_host, int64_t nbatch, int64_t nrhs,
                                int32_t precision, void* stream);
/* Allocation-free forward apply (FP32 SIMT kernel; MBF_ERR_INVALID on an operator it
 * cannot apply, see MBF_PREC_FP32_SIMT).  The paper has no counterpart: this is a service
 * for callers that may not allocate device memory when they apply an operator --
 * e.g. processes whose device memory is wholly owned by another allocator or held
 * to a fixed budget, or latency-critical loops where an allocation (which may
 * synchronize the device) is not allowed.  Same arguments and result as
 * mbf_apply with precision MBF_PREC_FP32_SIMT; the coefficient workspace and the
 * grid-barrier counter live in one fixed 4 MiB device array that the library
 * reserves on every device that loads it, until the process exits.
 *   - Needs 256 + 4 * (stages * c^(L-1)) (rounded up to 256) + stages * 8 * (c^L * max
 *     rank) * (RHS per pass: 1, 2 or 4) bytes, stages = 2 (L - L/2) + 1; more returns
 *     MBF_ERR_INVALID and launches nothing.
 *   - The first call on each device looks up the array's device address on that
 *     device (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - All calls share the array, which keeps the last call's contents; the barrier
 *     counter is cleared at the start of every call.  Calls that overlap on the GPU
 *     race on the array: serialize them.  Device waits that run out of time are
 *     reported by mbf_op_check on `op`, as for mbf_apply. */
mbf_status mbf_apply_static(mbf_op_t op, const void* g, void* u, int64_t nrhs, void* stream);
/* Synchronize `stream` and return MBF_ERR_TIMEOUT if a device wait of a previous
 * apply on this operator ran out of time (and clear the flag), else MBF_OK. */
mbf_status mbf_op_check(mbf_op_t op, void* stream);
/* Failure-detection test hook (no counterpart in the paper; off by default).  With
 * stage >= 0, later FP32 SIMT applies on this operator make the dependency wait of
 * group 0 of that stage (execution order, 1 .. n_stages - 1) wait for one producer more
 * than the plan has, so that the wait can only end by running out of time; wait_ns > 0
 * shortens every wait of those applies on a dependency counter, the pass barrier or a
 * chunk copy from 2 s to wait_ns.  The apply then stops early, its output undefined,
 * and mbf_op_check reports MBF_ERR_TIMEOUT, as for a real stall.  stage = -1 and
 * wait_ns = 0 restore normal applies.  MBF_ERR_INVALID for a stage beyond the plan or a
 * negative limit. */
mbf_status mbf_op_debug_stall(mbf_op_t op, int32_t stage, int64_t wait_ns);
/* Allocation-failure test hook (no counterpart in the paper; off by default).  With
 * after >= 0, the library's operator allocations (mbf_op_create and the workspaces an
 * apply allocates on first use) succeed `after` more times, then one fails as if the
 * device were out of memory -- the call reports MBF_ERR_OOM and frees what it had
 * taken -- and the hook turns itself off.  after = -1 turns it off.  Process-wide. */
mbf_status mbf_debug_fail_alloc(int64_t after);

/* Kernel timing, a measurement aid (no counterpart in the paper; off by default).
 * While enabled, every kernel an apply on this operator launches is bracketed by two
 * CUDA events recorded on the apply's stream.  mbf_op_profile() waits for those events
 * and returns, per kernel kind, the launches and their total device time since
 * profiling was last enabled, then clears them.  Enabling adds two event records per
 * launch to the stream; it does not change what the kernels compute. */
#define MBF_PROFILE_KINDS 8
typedef struct mbf_profile {
  int32_t n_kinds;
  char name[MBF_PROFILE_KINDS][32];
  int64_t launches[MBF_PROFILE_KINDS];
  double ms[MBF_PROFILE_KINDS];
} mbf_profile_t;
mbf_status mbf_op_set_profiling(mbf_op_t op, int32_t enable);
mbf_status mbf_op_profile(mbf_op_t op, mbf_profile_t* out);

/* ------------------------------------------------------------------ multiscale (§4)
 * The multiscale butterfly factorization of a 2-D kernel with a singularity at xi = 0:
 *     K ~ K_C R_C + sum_t BF_t R_t                                          (eq. f1)
 * over the coronas Omega_t = {n/2^(t+2) < max_k |xi_k| <= n/2^(t+1)} (eq.
 * domaindecomp) for the t with n/2^(t+2) >= n_center/2, and the centre Omega_C (the
 * rest, with n_center = 16: the paper's 16 x 16 centre, 17 x 17 points by the
 * inequalities).  BF_t is a butterfly factorization on quadtrees of depth
 * L_t = 2 floor((log2 n - t) / 2) over X and over the square [-n/2^(t+1), n/2^(t+1))^2
 * (upper faces closed) that holds Omega_t; K_C is kept dense in HBM (complex64).
 *   mbf_build_msbf     builds every part on the host (FP64, as mbf_build_factors; prob
 *                      gives dim = 2, n and r; its L and tree are ignored) and K_C through
 *                      the entry callback, then uploads them.
 *   mbf_msbf_create    assembles one from resident operators (same n_out / n_in; their
 *                      Omega trees must hold disjoint point sets) and the centre kernel
 *                      center_kernel [n_c][n_out] (complex FP64 interleaved, centre-point
 *                      major) on the natural Omega indices center_index [n_c].  With
 *                      take_ownership the parts are destroyed with it.
 *   mbf_msbf_apply     u = K_C g_C + sum_t BF_t g, device [nrhs][n] buffers, stream-ordered:
 *                      the centre product writes u, each part adds into it.
 *   mbf_msbf_apply_adjoint  g = K^* u (FP32 SIMT or split-BF16x3 tensor-core parts;
 *                           MBF_PREC_TF32 is rejected). */
typedef struct mbf_msbf_info {
  int32_t n_parts;
  int32_t part_t[16], part_L[16];
  int64_t part_points[16], part_nnz[16];
  int64_t n_out, n_in, n_center_points;
  int64_t nnz_algorithmic;      /* sum of the parts' nonzeros + n_out * n_center_points  */
  int64_t bytes_algorithmic;
} mbf_msbf_info_t;
mbf_status mbf_build_msbf(const mbf_problem_t* prob, mbf_entry_fn fn, void* ctx,
                          const mbf_build_opts_t* opts, int32_t n_center, mbf_msbf_t* out);
mbf_status mbf_msbf_create(const mbf_op_t* parts, int32_t n_parts, const double* center_kernel,
                           const int64_t* center_index, int64_t n_center_points,
                           int32_t take_ownership, mbf_msbf_t* out);
mbf_status mbf_msbf_apply(mbf_msbf_t m, const void* g, void* u, int64_t nrhs, int32_t precision,
                          void* stream);
mbf_status mbf_msbf_apply_adjoint(mbf_msbf_t m, const void* u, void* g, int64_t nrhs,
                                  int32_t precision, void* stream);
mbf_status mbf_msbf_info(mbf_msbf_t m, mbf_msbf_info_t* info);
/* The i-th part (borrowed handle, e.g. for mbf_op_info or mbf_op_tune). */
mbf_status mbf_msbf_part(mbf_msbf_t m, int32_t i, mbf_op_t* op);
mbf_status mbf_msbf_destroy(mbf_msbf_t m);

/* ------------------------------------------------------------------ autotuner
 * The paper has no counterpart (its applies are single-threaded CPU loops).  Measures,
 * on `stream` with device buffers it allocates and frees itself, (a) the FP32 SIMT apply
 * for 1, 2, 4, 8, 16, 32 and 64 RHS, (b) the tensor-core apply of one 64-RHS panel for
 * two or three panel buffers, each with the even A-tile ring depths 2 .. 16 that fit
 * shared memory beside them (8 configurations at most), then keeps the fastest and
 * sets the RHS count from which MBF_PREC_AUTO takes the tensor cores to the smallest
 * measured count at which one panel is faster than the SIMT apply.  Blocking; the
 * operator must be idle.  The choices stay with the operator until it is destroyed. */
typedef struct mbf_tune_result {
  int32_t n_simt;
  int32_t simt_rhs[8];
  double simt_ms[8];            /* device time of one SIMT apply of simt_rhs[i] RHS  */
  int32_t n_slots;
  int32_t slots[8];
  double tc_ms[8];              /* one 64-RHS panel with slots[i] A-ring slots and
                                   panel_buffers[i] panel buffers                    */
  int32_t tc_slots_chosen;      /* 0 if the tensor path is unavailable               */
  int32_t tc_min_rhs;           /* AUTO uses the tensor cores from this many RHS     */
  int32_t panel_buffers[8];     /* panel buffers of configuration i (2 or 3)          */
  int32_t tc_buffers_chosen;    /* panel buffers kept                                 */
  int32_t reserved_tune;
} mbf_tune_result_t;
mbf_status mbf_op_tune(mbf_op_t op, void* stream, mbf_tune_result_t* out);

/* ------------------------------------------------------------------ serving
 * The paper has no counterpart.  A server owns a worker thread, a few CUDA streams
 * (slots) and a staging budget on one device; operators stay resident and are shared.
 *   mbf_submit   queues u = K_f g for device buffers g [nrhs][n_in], u [nrhs][n_out]
 *                (complex64; caller-owned, live until the ticket is DONE or ERROR).  It
 *                never blocks: a request that does not fit the staging budget
 *                (2 nrhs max(n_in, n_out) 8 bytes reserved until it completes) or the
 *                queue returns MBF_ERR_BUSY.
 *   worker       continuous batching: whenever a slot is free it forms a batch: the
 *                oldest queued request with the queued requests on the same operator
 *                (FIFO, up to max_batch_rhs RHS, applied at once: in place through a
 *                table of the requests' rows up to 64 RHS, beyond that through a staging
 *                panel) is its first group.  When requests back up (more queued than
 *                max_inflight * max_batch_ops) and more operators are queued than slots
 *                are free, the oldest requests on other operators add groups the same
 *                way, spreading the queued operators over the free slots, at most
 *                max_batch_ops per batch, each group's factor traffic at most
 *                mix_work_pct percent of the first group's.  The batch is launched on
 *                the slot's stream, its groups in parallel branches -- as one captured
 *                CUDA graph (one graph launch for requests of several operators and RHS
 *                counts) when use_graphs is set.  A group borrows a workspace of its
 *                operator for the batch (the operator's own one when free, else one of a
 *                pool the operator keeps, allocated on first need), so batches overlap on
 *                the device, of one operator or of several.  While others are running or
 *                waiting, a batch's persistent kernels share 1 / max_inflight of the SMs,
 *                split among its groups in proportion to their factor traffic.
 *                The precision is MBF_PREC_AUTO for each group's RHS count.
 *   mbf_poll     state and timestamps of a ticket; a ticket is forgotten after the poll
 *                that reports DONE or ERROR (later polls: MBF_ERR_NOT_FOUND).
 * An operator used by a server must not be applied by the caller at the same time. */
typedef struct mbf_server_opts {
  int64_t staging_budget_bytes; /* device bytes for staging (0: 1 GiB)                 */
  int32_t max_inflight;         /* slots = batches on the device at once (0: 4, <= 16)  */
  int32_t max_batch_rhs;        /* RHS coalesced into one apply (0: 64)                */
  int32_t max_queue;            /* queued requests (0: 4096)                           */
  int32_t use_graphs;           /* 1: each batch is one CUDA graph launch              */
  int32_t max_batch_ops;        /* operators (groups) per batch (0: 4, <= 8)           */
  int32_t mix_work_pct;         /* a further operator joins a batch only if its group's
                                   factor traffic is <= this percent of the first
                                   group's (0: 25)                                     */
} mbf_server_opts_t;
typedef int64_t mbf_ticket_t;
enum { MBF_REQ_QUEUED = 0, MBF_REQ_RUNNING = 1, MBF_REQ_DONE = 2, MBF_REQ_ERROR = 3 };
typedef struct mbf_request_status {
  int32_t state;                /* MBF_REQ_*                                            */
  int32_t error;                /* mbf_status of a failed request                       */
  int32_t batch_requests;       /* requests in the batch that carried this one         */
  int32_t batch_rhs;            /* RHS of that batch                                   */
  double t_submit, t_start, t_done;   /* seconds since the server was created          */
} mbf_request_status_t;
typedef struct mbf_server_stats {
  int64_t submitted, completed, failed, rejected_busy;
  int64_t batches, coalesced_requests, graph_launches, graph_instantiations;
  int32_t max_batch_requests, max_concurrent_batches;
  int64_t mixed_batches;        /* batches that held requests of more than one operator */
  int32_t max_batch_ops;        /* most operators in one batch                          */
  int32_t reserved_stats;
} mbf_server_stats_t;
mbf_status mbf_server_create(const mbf_server_opts_t* opts, mbf_server_t* out);
/* The worker's batch rule as a pure host function (for tests of the policy): for n
 * queued requests, oldest first, on operators ops[i] in [0, n_ops) with nrhs[i] RHS,
 * a group's factor traffic taken as op_work[op] * its RHS count, and free_slots free
 * slots, writes the group of the next batch each request joins (-1: stays queued) to
 * group_of[i].  opts as for mbf_server_create (NULL: defaults).  Needs no device. */
mbf_status mbf_debug_form_batch(const int32_t* ops, const int64_t* nrhs, int64_t n, const double* op_work,
                                int32_t n_ops, int32_t free_slots, const mbf_server_opts_t* opts,
                                int32_t* group_of);
/* The worker's split of a batch's SMs among its n groups, as a pure host function: share
 * SMs in proportion to work[k] (each > 0 and finite), at least one per group, the rounding
 * remainder to the group of most work (the first of equal ones); written to sms_out[k].
 * The shares sum to share when share >= n.  Needs no device. */
mbf_status mbf_debug_split_sms(const double* work, int32_t n, int32_t share, int32_t* sms_out);
/* Host interpreter of the packed device layouts (for tests of the packers without a
 * device): packs the factor set on the host exactly as mbf_op_create does before it
 * uploads, then applies the packed data in FP64 as the layout defines it.  path 0: the
 * FP32 SIMT arena (items of complex64 entries); path 1: the tensor path, the split-BF16
 * tiles of the G / H levels (each entry hi + lo) with the leaf items of the SIMT arena, the
 * adjoint through the adjoint tile plan with the tiles read conjugate-transposed.  Forward
 * (adjoint = 0, eq. gbf) or adjoint (1).  in / out: host
 * complex128 (interleaved doubles), [nrhs][n_in] -> [nrhs][n_out] (adjoint: n_out ->
 * n_in), out fully overwritten.  MBF_ERR_INVALID for an invalid factor set, a tensor
 * path (or adjoint) the tiles do not fit (the reason in mbf_last_error), or a packed layout that
 * breaks its own definition (an entry outside the arena, a nonzero in the tiles' rank
 * padding, a leaf point outside its group). */
mbf_status mbf_debug_layout_apply(const mbf_factors_t* f, int32_t path, int32_t adjoint, const void* in,
                                  void* out, int64_t nrhs);
mbf_status mbf_submit(mbf_server_t s, mbf_op_t op, const void* g, void* u, int64_t nrhs,
                      mbf_ticket_t* ticket);
mbf_status mbf_poll(mbf_server_t s, mbf_ticket_t ticket, mbf_request_status_t* status);
/* Wait until nothing is queued or running (at most timeout_s; MBF_ERR_TIMEOUT after). */
mbf_status mbf_server_drain(mbf_server_t s, double timeout_s);
mbf_status mbf_server_stats(mbf_server_t s, mbf_server_stats_t* out);
/* Finishes queued and running requests, then frees the server. */
mbf_status mbf_server_destroy(mbf_server_t s);

/* Thread-local text of the last error ("" if none). */
const char* mbf_last_error(void);
/* Library version string. */
const char* mbf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MBF_H */
