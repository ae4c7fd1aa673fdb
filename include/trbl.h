/*
 * trbl.h -- C ABI of the GB300 thick-restart block Lanczos library for
 * M-scheme shell-model Hamiltonians (Shimizu, Mizusaki, Utsuno, Tsunoda,
 * "Thick-restart block Lanczos method for large-scale shell-model
 * calculations", arXiv 1902.02064).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Return value: TRBL_OK (0) or a TRBL_ERR_* status.  No C++ exception
 *   crosses this boundary.  trbl_last_error() returns a message for the last
 *   failing call on the calling thread (thread-local, owned by the library,
 *   valid until the next failing call on that thread).
 * - "Host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *   global memory of the current device.  The caller owns every buffer it
 *   passes; the library owns the objects it creates (trbl_basis,
 *   trbl_hamiltonian) and frees them in the matching *_destroy call.
 * - Streams are passed as `void*` holding a cudaStream_t (NULL = legacy
 *   default stream).  Work is enqueued asynchronously on that stream unless
 *   an entry point says it synchronises.
 * - A model space of one species lists its single-particle m-states in a
 *   fixed order; bit i of a determinant's bit string is m-state i
 *   (Sec. II Eq. (mbasis); App. A Table I).  At most 32 m-states per species.
 * - Species determinants are ordered by ascending 2M and, within equal 2M,
 *   by the unsigned value of the bit string.  The product basis (App. A
 *   Eq. (part)) is a sequence of blocks, one per 2M_A (ascending) for which
 *   both species have determinants with 2M_A + 2M_B = 2M; inside a block the
 *   state (iA, iB) has index offset + iA * N_B + iB.
 * - A block of vectors is row-major: row i (basis state i) holds q values,
 *   rows ld elements apart (ld >= q).
 * - One CUDA device per process: kernel attributes and the SM count are set
 *   up once, on the device current at the first call that launches work.
 */
#ifndef TRBL_H
#define TRBL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TRBL_OK 0
#define TRBL_ERR_ARG 1       /* invalid argument (null pointer, size, layout) */
#define TRBL_ERR_CUDA 2      /* a CUDA runtime or library call failed */
#define TRBL_ERR_OOM 3       /* device or host allocation failed */
#define TRBL_ERR_BREAKDOWN 4 /* block QR found a rank-deficient block it could not repair, or the block
                                or T holds NaN or Inf (for example from a caller's block) */
#define TRBL_ERR_NOCONV 5    /* iteration limit reached; partial results returned */

#define TRBL_F32 0 /* IEEE binary32 vectors */
#define TRBL_F64 1 /* IEEE binary64 vectors */

/* One species' single-particle space: n_states m-states with their 2j, 2m and
 * shell index, occupied by n_particles particles.  Arrays are host memory of
 * length n_states, read during the call only. */
typedef struct trbl_space {
  int n_states;
  const int* twoj;
  const int* twom;
  const int* orbit;
  int n_particles;
} trbl_space;

typedef struct trbl_basis trbl_basis;
typedef struct trbl_hamiltonian trbl_hamiltonian;

/* Sizes of a basis, filled by trbl_basis_info. */
typedef struct trbl_basis_sizes {
  int64_t dim;          /* M-scheme dimension D */
  int32_t n_det[2];     /* determinants of species A, B (all 2M) */
  int32_t n_blocks;     /* product blocks */
  int64_t n_jumps[2];   /* one-body jump entries of A, B, diagonal a=c included */
  int32_t n_delta;      /* number of 2m-transfer classes, 2*span/2+1 */
} trbl_basis_sizes;

/* Builds the two-species M-scheme basis of total 2M = twoM: determinant
 * enumeration (Sec. II Eq. (mbasis)), the product blocks of App. A
 * Eq. (part), and the one-body jump lists of App. B.2 (every
 * a+_a a_c |S> with its target, source and sign; the paper stores them per
 * partition, here per target determinant and 2m transfer).  Host-only work:
 * it needs no GPU.  *out is owned by the library.
 * Errors: TRBL_ERR_ARG for null pointers, more than 32 m-states, particle
 * numbers outside [0, n_states], or an empty basis. */
int trbl_basis_create(const trbl_space* A, const trbl_space* B, int twoM, trbl_basis** out);

/* Frees a basis.  The caller must destroy every Hamiltonian built on it first. */
void trbl_basis_destroy(trbl_basis* b);

/* Fills *sizes.  Host-only. */
int trbl_basis_info(const trbl_basis* b, trbl_basis_sizes* sizes);

/* Copies the basis description into caller-owned host arrays (any may be
 * NULL to skip it): bitsA/twoMA [n_det[0]], bitsB/twoMB [n_det[1]], and
 * blocks [n_blocks * 7] as rows (2M_A, 2M_B, offset, N_A, N_B, first A
 * determinant, first B determinant).  Host-only. */
int trbl_basis_export(const trbl_basis* b, uint32_t* bitsA, int32_t* twoMA, uint32_t* bitsB,
                      int32_t* twoMB, int64_t* blocks);

/* Copies the one-body jump list of one species (0 = A, 1 = B) into
 * caller-owned host arrays of length n_jumps[species]: jump e maps source
 * determinant src[e] to target tgt[e] by a+_{a[e]} a_{c[e]} with fermion sign
 * sign[e] (+1/-1), global determinant indices (App. B.2, the "one-body
 * jumps").  Diagonal entries a = c (number operators) are included.
 * Entries are ordered by target, then 2m transfer, then source.  Host-only. */
int trbl_basis_export_jumps(const trbl_basis* b, int species, int32_t* tgt, int32_t* src,
                            int32_t* a, int32_t* c, int8_t* sign);

/* Builds the device tables of H = H1 + H2 (Sec. II) on the current CUDA
 * device: like-particle target lists with their summed coefficients
 * (App. B.1) and the cross-species coefficient table used with the jump
 * lists (App. B.2 Eq. (pntwobodybit)).  Inputs are host FP64 arrays, read
 * during the call only:
 *   h1A[nA*nA]  h(1)_ac of a+_a a_c for species A (row a, column c);
 *   h1B[nB*nB]  the same for species B;
 *   VAA[nA^4]   h(2)_abcd of a+_a a+_b a_d a_c, index ((a*nA+b)*nA+c)*nA+d,
 *               read only for a<b, c<d;
 *   VBB[nB^4]   the same for species B;
 *   VAB[nA*nB*nA*nB] coefficient of a+_a b+_b b_d a_c, index
 *               ((a*nB+b)*nA+c)*nB+d.
 * Coefficients that do not conserve 2m are ignored, but every entry must be
 * finite.  The caller keeps b alive while *out exists.  Errors:
 * TRBL_ERR_ARG (null argument, or a NaN or Inf entry in any array),
 * TRBL_ERR_OOM, TRBL_ERR_CUDA. */
int trbl_hamiltonian_create(const trbl_basis* b, const double* h1A, const double* h1B,
                            const double* VAA, const double* VBB, const double* VAB,
                            trbl_hamiltonian** out);

/* Frees the Hamiltonian's device tables (synchronises the device first). */
void trbl_hamiltonian_destroy(trbl_hamiltonian* h);

/* W = H V for a block of q vectors (Alg. 3/4 line "W := H V_k"), matrix
 * elements generated on the fly from the jump lists (App. B).  V and W are
 * device arrays of D rows, leading dimensions ldv, ldw >= q, element type
 * dtype (TRBL_F32 or TRBL_F64, accumulation in that type).  W is
 * overwritten; V and W must not overlap.  1 <= q <= 64.  Asynchronous on
 * stream.  Errors: TRBL_ERR_ARG, TRBL_ERR_CUDA (launch failure). */
int trbl_apply_block(const trbl_hamiltonian* h, const void* V, int64_t ldv, void* W, int64_t ldw,
                     int q, int dtype, void* stream);

/* C = B^T W: the m x q projection coefficients of a block W (D x q) on m
 * stored vectors B (D x m), the product "alpha_k := V_k^T W" of Alg. 3/4 and
 * the coefficients of the reorthogonalisation against the Krylov basis
 * (Sec. III C/D).  B and W are device arrays of element type dtype
 * (TRBL_F32 or TRBL_F64), row-major with leading dimensions ldb >= m,
 * ldw >= q; C is a device FP64 array, row-major m x q (leading dimension
 * q), overwritten.  Products are summed in dtype inside fixed row chunks and
 * the chunk sums are added in FP64 in a fixed order (bit-reproducible for
 * given sizes).  1 <= q <= 64, m >= 1.  A Gram matrix of FP32 data (B ==
 * W, ldb == ldw, m == q with q = 8, 16, 32 or 64: the "W^T W" of the block
 * Cholesky QR) goes to a kernel that reads the block once, with products
 * summed in FP32 over runs of at most 32 rows and the runs in FP64.  The
 * partial-sum scratch (chunks x m x q doubles) is taken with
 * cudaMallocAsync and released with cudaFreeAsync on the stream.
 * Asynchronous on stream.  Errors: TRBL_ERR_ARG, TRBL_ERR_OOM,
 * TRBL_ERR_CUDA. */
int trbl_block_dot(const void* B, int64_t ldb, int m, const void* W, int64_t ldw, int q, int64_t D,
                   int dtype, double* C, void* stream);

/* Number of independent parameters of H on these spaces, in the canonical
 * order used by trbl_grad: one-body A (a <= c with equal 2m, a-major), one-body
 * B, two-body AA (pairs I = (i<j) lexicographic, J >= I with equal pair 2m),
 * BB, then AB (pairs (a, b) a-major, J >= I with equal pair 2m).  A
 * parameter at slot (I, J) with I != J sets both V_IJ and V_JI. */
int trbl_param_count(const trbl_basis* b, int64_t* n);

/* Hellmann-Feynman gradient (Sec. II: H is linear in its parameters, so
 * dE_k/dtheta = <x_k| dH/dtheta |x_k> for a normalised eigenvector x_k):
 * dtheta[p] = sum over the nvec given vectors of <x| dH/dtheta_p |x>, for
 * every parameter in trbl_param_count's order.  For a cluster of
 * (near-)degenerate levels pass the whole cluster: the sum is the derivative
 * of the cluster's eigenvalue sum, Tr(P_C dH/dtheta).  X: device, D x nvec
 * row-major (ld ldx), dtype TRBL_F32 or TRBL_F64, 1 <= nvec <= 32;
 * dtheta: host FP64 [nparams].  The elements visited are those of the block
 * product (App. B); bins are summed with FP64 atomics.  The first call
 * builds device tables kept with the Hamiltonian.  Synchronises the stream.
 * Errors: TRBL_ERR_ARG (including nparams != trbl_param_count),
 * TRBL_ERR_OOM, TRBL_ERR_CUDA. */
int trbl_grad(const trbl_hamiltonian* h, const void* X, int64_t ldx, int nvec, int dtype, double* dtheta,
              int64_t nparams, void* stream);

/* trbl_grad for several level clusters in one pass: the nvec columns of X
 * are split into ncl clusters of consecutive columns, cluster c holding
 * columns first[c] .. first[c+1] - 1 (host array, first[0] = 0, first[ncl]
 * = nvec, increasing); dtheta[c * nparams + p] (host) receives the
 * derivative of cluster c's eigenvalue sum, Tr(P_c dH/dtheta_p).  Same
 * traversal of the product's elements as trbl_grad, each element's products
 * summed per cluster; FP64 bins of ncl x (bins of trbl_grad) are kept with
 * the Hamiltonian (grown as needed).  Synchronises the stream.  Errors:
 * TRBL_ERR_ARG, TRBL_ERR_OOM, TRBL_ERR_CUDA. */
int trbl_grad_clusters(const trbl_hamiltonian* h, const void* X, int64_t ldx, int nvec, int dtype,
                       const int* first, int ncl, double* dtheta, int64_t nparams, void* stream);

/* trbl_block_dot on the tensor cores (TRBL_PROJ_TENSOR arithmetic) for
 * FP32 data: same arguments, layout and errors, with dtype TRBL_F32 only,
 * q <= 32, B and W 16-byte aligned and ldb, ldw multiples of 4
 * (TRBL_ERR_ARG otherwise). */
int trbl_block_dot_tc(const void* B, int64_t ldb, int m, const void* W, int64_t ldw, int q, int64_t D, double* C,
                      void* stream);

/* Block update Out[:, 0:n] = alpha * In[:, 0:K] U + beta * Out over D rows:
 * the "W := W - V_k alpha_k" and reorthogonalisation updates of Alg. 3/4
 * (Sec. III C/D) and W R^-1 of the block QR.  In, Out: device, row-major,
 * leading dimensions ldi >= K and ldo >= n, dtype TRBL_F32 or TRBL_F64, must
 * not overlap; U: device FP64 K x n row-major (ld ldu >= n).  algo:
 * TRBL_PROJ_TENSOR or TRBL_PROJ_CUDA_CORE (FP32 data; FP64 data ignore it);
 * the tensor-core form needs In 16-byte aligned with ldi a multiple of 4
 * and falls back to the CUDA cores otherwise.  For n > 32 it is the wide
 * form the solver uses for the thick restart v_i := sum_j v_j U_ji and the
 * Ritz vectors (Sec. III D): 128 x 128 output tiles, split TF32 operands, a
 * fresh tensor-memory accumulator every 32 values of K, summed in FP32
 * registers with round-to-nearest adds.  Allocates stream-ordered scratch
 * (cudaMallocAsync) for the tensor-core form.  Asynchronous on
 * stream.  Errors: TRBL_ERR_ARG, TRBL_ERR_OOM, TRBL_ERR_CUDA. */
int trbl_block_update(const void* In, int64_t ldi, int K, const double* U, int64_t ldu, int n, void* Out,
                      int64_t ldo, int64_t D, double alpha, double beta, int dtype, int algo, void* stream);

/* Allocation-free form of trbl_block_dot, for callers that must not
 * allocate device memory during the call: code running where the CUDA
 * allocator may not be entered (inside host callbacks, or while another
 * component owns and budgets all device memory) and latency-critical loops
 * that cannot afford an allocation's implicit synchronisation.  The paper
 * has no counterpart; it is a service of this library.
 *
 * Same arguments, layouts, arithmetic and errors as trbl_block_dot, except
 * that the partial-sum scratch is a fixed array compiled into the library
 * (TRBL_NOALLOC_SCRATCH_BYTES per device, held by every device that loads
 * the library until the process exits).  It calls no cudaMalloc, cudaFree
 * or allocating library routine.  m * q * 8 must not exceed
 * TRBL_NOALLOC_SCRATCH_BYTES (TRBL_ERR_ARG otherwise); larger products use
 * fewer row chunks, never more scratch.
 *
 * The first call on a device looks up the scratch array's device address
 * (with that device current) and loads every kernel this entry point can
 * launch, for both element types and every q, so that CUDA's lazy module
 * loading takes no device memory during a later call; make that first call
 * before any stream capture.  All calls on a device share the one array: calls whose
 * executions overlap on the GPU (different streams, or different host
 * threads) race and give wrong results.  Every call overwrites the part of
 * the scratch it reads, so no clearing is needed between calls. */
#define TRBL_NOALLOC_SCRATCH_BYTES (8u << 20)
int trbl_block_dot_noalloc(const void* B, int64_t ldb, int m, const void* W, int64_t ldw, int q, int64_t D,
                           int dtype, double* C, void* stream);

/* Arithmetic of the FP32 block projections C = B^T W and updates
 * Out = alpha In U + beta Out (mixed precision).  TRBL_PROJ_TENSOR: tcgen05
 * tensor-core MMAs on split TF32 operands (x = hi + lo with TF32 hi and lo,
 * |x - hi - lo| <= 2^-22 |x|; a b formed as a_hi b_hi + a_hi b_lo + a_lo b_hi
 * in FP32 tensor memory; projections drain every 128 rows into compensated
 * FP32 sums, FP64 per row chunk, which keeps the tensor cores' round-toward-
 * zero accumulation from biasing the sums), for q or n <= 32
 * and 16-byte aligned row-major operands, other shapes falling back to the
 * CUDA cores.  The solver sends updates with K < 256 to the CUDA cores,
 * which are faster there.  TRBL_PROJ_CUDA_CORE: FP32 FMAs on the CUDA cores with FP64
 * combination of row chunks.  FP64 data always use FP64 FMAs. */
#define TRBL_PROJ_TENSOR 0
#define TRBL_PROJ_CUDA_CORE 1

#define TRBL_PREC_F64 1   /* FP64 vectors, apply and projections */
#define TRBL_PREC_MIXED 2 /* FP32 vectors and apply; FP64 CGS2 coefficients, CholQR2, Ritz */

/* Solver parameters (Alg. 4).  Zero fields take the documented defaults. */
typedef struct trbl_params {
  int nev;             /* wanted lowest eigenpairs */
  int q;               /* block size p of the paper, 1..64 */
  int max_basis;       /* l_m: Lanczos vectors kept before a thick restart */
  int keep;            /* l_s: Ritz vectors kept at a restart; 0 = nev + (max_basis-nev)/4,
                          clipped to max_basis - 2q */
  double tol;          /* converged when ||beta_k U_{last q rows,i}|| <= tol * ||H|| for i < nev */
  int precision;       /* TRBL_PREC_F64 or TRBL_PREC_MIXED */
  int max_iter;        /* block iterations cap; 0 = 100000 */
  int check_every;     /* Rayleigh-Ritz convergence test every this many block steps (restarts always
                          test); 0 = adaptive: a test once the block steps since the previous test
                          have taken twelve times as long as that test did (tests then take at most
                          a thirteenth of the time) */
  uint64_t seed;       /* start block: uniform(-1,1) from splitmix64(seed<<32 + i*q + j) */
  double normH;        /* ||H|| used by tol; 0 = estimated by the solver (largest |Ritz value|) */
  int projections;     /* TRBL_PROJ_TENSOR (0, default) or TRBL_PROJ_CUDA_CORE: how the FP32
                          projections and updates of mixed precision are computed */
  int reorth;          /* TRBL_REORTH_SELECTIVE (0, default) or TRBL_REORTH_TWICE (below) */
  int refine;          /* trbl_solve in TRBL_PREC_MIXED: 1 = when the true residuals (FP64 apply)
                          of the converged pairs exceed tol * ||H||, lower the estimate's target
                          (below tol by the measured gap) and iterate on, at most three rounds,
                          until they meet tol or the FP32 floor alone reaches 0.9 tol; 0 = stop
                          at the estimate (default).  Ignored by the stepwise and batched
                          solvers. */
} trbl_params;

/* Reorthogonalisation of a block step (Sec. III C/D: the block is made
 * orthogonal to every stored Lanczos vector).
 * TRBL_REORTH_SELECTIVE: classical Gram-Schmidt against the last two blocks
 *   (the three-term part of the recurrence, which carries W = H V_k's large
 *   components), one full pass against every stored vector, and a second
 *   full pass only in the steps where a column of the block lost more than
 *   half its squared norm in the first (the Daniel-Gragg-Kaufman-Stewart
 *   test).  One full pass removes what the first leaves when the block was
 *   already orthogonal to the basis up to rounding.
 * TRBL_REORTH_TWICE: two full passes every step (classical Gram-Schmidt
 *   applied twice). */
#define TRBL_REORTH_SELECTIVE 0
#define TRBL_REORTH_TWICE 1

/* Per-solve statistics (per-phase times mirror the paper's Fig. 5(c)). */
typedef struct trbl_stats {
  int iterations;      /* block Lanczos steps (applications of H to a block) */
  int restarts;        /* thick restarts */
  int converged;       /* eigenpairs meeting the tolerance */
  int status;          /* return value of trbl_solve */
  double normH;        /* ||H|| used by the tolerance */
  double ms_total, ms_apply, ms_orth, ms_qr, ms_ritz, ms_restart;
  int basis_size;      /* Lanczos vectors in the basis now (stepwise solver; the last step's for trbl_solve) */
  int second_passes;   /* block steps that ran a second full reorthogonalisation pass */
  double ms_copy_in, ms_copy_out;  /* trbl_solver_step_host: device time of the block copies from / to
                                      host memory (CUDA events on the solver's stream), summed */
} trbl_stats;

/* Lowest nev eigenpairs of H by the thick-restart block Lanczos method
 * (Sec. III D, Alg. 4, restart of Eq. (trb-tmat)), with full
 * reorthogonalisation against every stored Lanczos vector (p->reorth:
 * selective, or classical Gram-Schmidt applied twice) and Cholesky-QR
 * applied twice as the block QR.
 * Outputs: evals[nev] (host, ascending), resid[nev] (host, true residual
 * norms ||H x - theta x|| recomputed with a fresh FP64 apply, may be NULL),
 * evecs (device, D x nev row-major FP64 in TRBL_PREC_F64 and FP32 in mixed
 * mode, may be NULL), *stats (host, may be NULL).  Allocates its own device
 * workspace (basis of D x max_basis) and synchronises the stream before it
 * returns.  Errors: TRBL_ERR_ARG, TRBL_ERR_OOM, TRBL_ERR_CUDA,
 * TRBL_ERR_BREAKDOWN, TRBL_ERR_NOCONV (outputs then hold the best current
 * approximations). */
int trbl_solve(const trbl_hamiltonian* h, const trbl_params* p, double* evals, double* resid,
               void* evecs, trbl_stats* stats, void* stream);

/* Batched form of trbl_solve for nset Hamiltonians (for example many
 * parameter sets of one model space, or sectors of uneven dimension), all
 * with the same parameters p (max_basis at most the smallest dimension).  One persistent launch of the block product serves every
 * set, and each other operation of a block step is one launch over all
 * sets; the step is captured into a CUDA graph per basis size and replayed
 * on a private stream.  Rayleigh-Ritz tests and restarts run
 * between replays on host worker threads (each set on its own stream), all
 * sets testing at the same steps.  stats: iterations = block steps, ms_total
 * = wall time of the whole call, ms_apply = wall time of the batched block
 * steps (product, orthogonalisation, QR of every set), ms_ritz = wall time
 * of the tests and restarts between them, second_passes = set-steps that
 * ran a second full reorthogonalisation pass (the selective schedule takes
 * its DGKS decision per set on the device, inside the captured step: the
 * second pass's launches return at once for the sets that skip it).  The
 * Hamiltonians may live on one
 * basis (parameter sets) or on bases of different dimension (sectors of
 * other 2M or particle numbers): each set keeps its own tables, work list
 * and dimension D_s, and each batched launch covers all sets.  Outputs are
 * set-major: evals and resid [nset * nev] (host), evecs (device, may be
 * NULL) the sets' D_s x nev blocks one after another, status [nset] (host, per-set
 * return code, may be NULL); stats summarises the batch.  Needs
 * q * element size = 16 * 2^i bytes.  A rank-deficient block stops its set
 * with TRBL_ERR_BREAKDOWN (the column-wise repair of trbl_solve is not
 * available in batched steps).  Synchronises the stream.  Returns the first
 * failing set's code, TRBL_OK when all sets finished. */
int trbl_solve_batch(const trbl_hamiltonian* const* hs, int nset, const trbl_params* p, double* evals,
                     double* resid, void* evecs, int* status, trbl_stats* stats, void* stream);

/* Kernels of the block product (App. B; same elements, same arithmetic):
 * TRBL_APPLY_GROUPED serves every q and both precisions; TRBL_APPLY_FAST is
 * the FP32 kernel for q = 8, 16, 32 (16-byte aligned rows, D * ld < 2^31,
 * at most 31 two-m transfer classes), with fewer instructions per generated
 * element.  A product the chosen kernel cannot take runs on the grouped
 * kernel. */
#define TRBL_APPLY_GROUPED 0
#define TRBL_APPLY_FAST 1
/* The grouped kernel with half the lanes per generated element, each lane
 * moving two 16-byte chunks of the V row (rows of 32, 64 or 128 bytes;
 * other rows as TRBL_APPLY_GROUPED). */
#define TRBL_APPLY_GROUPED_X2 2
/* Split product for FP32 and q a multiple of 16 (16-byte aligned rows,
 * D * ld < 2^31): the like-particle terms (App. B.1) by the grouped kernel,
 * then the factorised proton-neutron term (App. B.2, Eq. (pntwobodybit)) by
 * a source-stationary kernel.  That kernel owns a 16-column slice of one
 * target slab (a proton determinant's neutron rows) in shared memory; each
 * source row V[p, n, :] it gathers is multiplied into every outgoing neutron
 * jump of n at once, so a row is read once per transfer class instead of
 * once per generated element.  Its sums are formed with shared-memory
 * atomic adds, so the FP32 rounding of W can differ from run to run (within
 * the same error bound); the other kernels are deterministic.  Other
 * products run as TRBL_APPLY_GROUPED.  Blocks per SM of the cross-term
 * kernel: 2 (384 threads, 8 outgoing jumps per register batch, two row
 * gathers in flight per lane group) or 1 (512 threads, 8 jumps, four
 * gathers in flight). */
#define TRBL_APPLY_SPLIT 3
/* The split product with 4 outgoing jumps per register batch and four row
 * gathers in flight per lane group, 2 blocks of 512 threads per SM. */
#define TRBL_APPLY_SPLIT_X4 4
/* The split product whose cross-term kernel stages the source rows in
 * shared memory by TMA (chunks of consecutive source rows, one 16-column x
 * 32-row box per proton jump, two chunks in flight) and runs one source
 * row per warp, its 8 lane groups on 8 outgoing jumps; 1 block per SM. */
#define TRBL_APPLY_SPLIT_TMA 5
/* Launch shapes trbl_apply_autotune times, in this order (kernel, neutron
 * rows per work item, resident blocks per SM): grouped 16/32/64/128; fast
 * 16/32/64 at 8 blocks per SM (32 registers a thread); fast 16/32/64 at 6
 * blocks per SM (40 registers); grouped with two chunks per lane 16/32/64;
 * split at 64 rows (rows per work item of its like-particle launch) at 2
 * blocks per SM and split with four jumps per batch at 64 rows.
 * Lanes per element and chunks per lane follow from the kernel and the row
 * width (one lane group reads one whole V row). */
#define TRBL_TUNE_CANDIDATES 15

/* Times the block product of h at block size q and dtype for each launch
 * shape above that applies and keeps the fastest; ms [TRBL_TUNE_CANDIDATES]
 * (host, may be NULL) receives the average time per candidate (NaN for a
 * shape that does not apply to q and dtype) and *best_rows the chosen rows
 * per work item (trbl_apply_get_shape gives the whole shape).  Allocates two
 * D x q scratch blocks for the timing.  Synchronises the stream. */
int trbl_apply_autotune(trbl_hamiltonian* h, int q, int dtype, float* ms, int* best_rows, void* stream);

/* Sets the block product's rows per work item (1..4096), keeping its
 * kernel; the product's results do not depend on it.  Host only; not while
 * a product of h is running.  Errors: TRBL_ERR_ARG. */
int trbl_apply_set_rows(trbl_hamiltonian* h, int rows_per_item);

/* Sets the whole launch shape: kernel (TRBL_APPLY_GROUPED, TRBL_APPLY_FAST,
 * TRBL_APPLY_GROUPED_X2, TRBL_APPLY_SPLIT, TRBL_APPLY_SPLIT_X4 or
 * TRBL_APPLY_SPLIT_TMA), rows per work item (1..4096) and resident blocks
 * per SM: 6 or 8 for the fast kernel; 1 or 2 for TRBL_APPLY_SPLIT, 2 for
 * TRBL_APPLY_SPLIT_X4, 1 for TRBL_APPLY_SPLIT_TMA; any of 1, 2, 6, 8 for
 * the grouped kernels, which ignore it.  Same rules as
 * trbl_apply_set_rows.  Errors: TRBL_ERR_ARG. */
int trbl_apply_set_shape(trbl_hamiltonian* h, int kernel, int rows_per_item, int blocks_per_sm);

/* The current launch shape (any output may be NULL).  Host only. */
int trbl_apply_get_shape(const trbl_hamiltonian* h, int* kernel, int* rows_per_item, int* blocks_per_sm);

/* Summation of the FP32 fast kernel's rows.  0 (default): one FP32 sum per
 * column in the grouped kernel's order.  1: short FP32 partial sums (one
 * cross-term task, or up to 8 like-particle sources) added into a two-word
 * row sum by Knuth's TwoSum, so the rounding of a row does not grow with
 * its length; the product's error is then set by the FP32 inputs.  Host
 * only; not while a product of h is running.  Errors: TRBL_ERR_ARG. */
int trbl_apply_set_compensated(trbl_hamiltonian* h, int on);

/* Stepwise form of trbl_solve for callers that drive the iteration
 * themselves.  A solver owns its device workspace (basis of D x max_basis
 * vectors plus O(D q) blocks) and runs every call on the stream given here;
 * calls synchronise that stream before they return.
 *
 * trbl_solver_create: validates p (copied), allocates, and builds the
 *   orthonormal start block (Alg. 4, first line).  Errors as trbl_solve.
 * trbl_solver_step: one block step of Alg. 4 -- W := H V_k, alpha_k,
 *   full reorthogonalisation, V_{k+1} beta_k := QR(W), Rayleigh-Ritz when due
 *   (every check_every steps and before every restart) -- followed by a thick
 *   restart (Eq. (trb-tmat)) when the basis is full.  *converged (may be
 *   NULL) receives the number of converged pairs when a Rayleigh-Ritz test
 *   ran in this step, else -1.  After convergence further steps do nothing.
 * trbl_solver_step_host: the same step with the current block V_k read from
 *   host memory block_in (D x q, row-major, element type of the precision:
 *   FP64 or FP32; NULL keeps the device copy) before the step and the next
 *   block written to host memory block_out (same layout; NULL skips) after
 *   it.  Pinned host memory (trbl_host_alloc) makes the copies
 *   asynchronous.
 * trbl_solver_block: device address and byte size of the current block V_k
 *   (D x q row-major), valid until the next step.
 * trbl_solver_stats: statistics so far (ms_total counts from creation).
 * trbl_solver_finish: Ritz values (ascending), true residuals and Ritz
 *   vectors of the current basis, as trbl_solve returns them; TRBL_ERR_NOCONV
 *   when not all nev pairs met the tolerance (outputs still filled).
 * trbl_solver_destroy: synchronises the stream and frees the solver. */
/* Row sharding of the block product over several GPUs (the paper's
 * distributed matrix-vector product, App. C, with every GPU holding the
 * tables): rows of W are split into contiguous ranges of whole target slabs
 * (the rows (pA', nB') of one proton determinant pA'); a shard's product
 * reads the slabs of its targets' source proton determinants, which the
 * shard receives from the others before the product (an all-gather of V
 * slices, or only the listed ranges), and the projections are sharded by the
 * same rows with the m x q coefficients summed across shards.  All host
 * only; they need no GPU.
 *
 * trbl_shard_plan: bounds[nranks + 1] (host) receives slab-aligned row
 *   boundaries, bounds[0] = 0 and bounds[nranks] = D, balanced by the
 *   elements the product generates per row (the cross term's proton x
 *   neutron jump pairs, plus one for a row's like-particle and diagonal
 *   work); work[nranks] (host, may be NULL) the estimate per shard.
 * trbl_shard_sources: the V rows the product of rows [row_begin, row_end)
 *   reads, as *nranges merged [begin, end) pairs in ranges[2 * cap] (host;
 *   NULL with cap 0 only counts).  The rows must be slab boundaries. */
int trbl_shard_plan(const trbl_basis* b, int nranks, int64_t* bounds, int64_t* work);
int trbl_shard_sources(const trbl_basis* b, int64_t row_begin, int64_t row_end, int64_t* ranges, int64_t cap,
                       int64_t* nranges);

/* Restricts the product of h (trbl_apply_block) to rows [row_begin,
 * row_end) of W, slab boundaries of the basis (0 and D restore the whole
 * product); the other rows of W are not written.  Needs the grouped or fast
 * kernel (16-byte aligned rows of q * element size = 16 * 2^i bytes), and
 * the solvers need the whole product.  Host only; not while a product of h
 * is running.  Errors: TRBL_ERR_ARG. */
int trbl_hamiltonian_set_rows(trbl_hamiltonian* h, int64_t row_begin, int64_t row_end);

typedef struct trbl_solver trbl_solver;

/* Page-locked host memory (cudaHostAlloc, portable) for the blocks of
 * trbl_solver_step_host, so that their copies run asynchronously at the
 * link's rate.  The pages are placed on the host memory node nearest
 * `device` (cudaDevAttrHostNumaId) by binding the calling thread's NUMA
 * policy to it during the allocation (the thread's policy is restored
 * after; default placement where the system refuses or the device reports
 * no node).  *numa_node (may be NULL) receives the node that holds the
 * buffer's first page (the nearest node if that cannot be queried; -1 if
 * neither is known).  The caller owns the buffer and frees it with
 * trbl_host_free.  Errors: TRBL_ERR_ARG, TRBL_ERR_OOM, TRBL_ERR_CUDA. */
int trbl_host_alloc(size_t bytes, int device, void** out, int* numa_node);
int trbl_host_free(void* p);

int trbl_solver_create(const trbl_hamiltonian* h, const trbl_params* p, void* stream, trbl_solver** out);
int trbl_solver_step(trbl_solver* s, int* converged);
int trbl_solver_step_host(trbl_solver* s, const void* block_in, void* block_out, int* converged);
int trbl_solver_block(trbl_solver* s, void** block, int64_t* bytes);
int trbl_solver_stats(trbl_solver* s, trbl_stats* stats);
int trbl_solver_finish(trbl_solver* s, double* evals, double* resid, void* evecs, trbl_stats* stats);
void trbl_solver_destroy(trbl_solver* s);

/* Checkpoint and resume of a stepwise solver.  The state between block
 * steps of Alg. 4 is the Lanczos basis V_1 .. V_k (after a thick restart:
 * the kept Ritz vectors and the new block, Eq. (trb-tmat)), the current
 * block V_{k+1}, the projected matrix T and a few counters; it is written
 * to and read from caller-owned host memory in a library-defined format
 * (a header, then T as max_basis x max_basis FP64, V_{k+1} as D x q and the
 * basis as D x (stored vectors), row-major, in the precision's element
 * type).  Checkpoints are meant for host memory or files of the same
 * build; the paper stores its Lanczos vectors on disk only for want of
 * memory (App. C), not to resume.
 *
 * trbl_solver_state_bytes: *bytes = size of the state now (it grows with
 *   the basis; smallest right after a restart).
 * trbl_solver_save: writes the state to host (at least state_bytes bytes;
 *   pinned memory is faster).  Synchronises the solver's stream.  Errors:
 *   TRBL_ERR_ARG (null, too small, or the solver has already converged:
 *   finish it instead), TRBL_ERR_CUDA.
 * trbl_solver_load: replaces the state of s, created with the same
 *   Hamiltonian dimension, q, max_basis, keep and precision, by a saved
 *   one; the next steps continue the saved iteration (with a fixed
 *   check_every the results equal an uninterrupted run's).  Statistics
 *   resume from the saved counts.  Errors: TRBL_ERR_ARG (not a state of
 *   this library, or saved with other sizes), TRBL_ERR_CUDA. */
int trbl_solver_state_bytes(trbl_solver* s, int64_t* bytes);
int trbl_solver_save(trbl_solver* s, void* host, int64_t bytes);
int trbl_solver_load(trbl_solver* s, const void* host, int64_t bytes);

/* Number of kernels this library has launched in the process so far
 * (every entry point counts its own launches; library calls such as the
 * cuSOLVER eigensolver are not counted). */
long long trbl_kernel_launches(void);

/* Message of the last failing call on this thread ("" if none). */
const char* trbl_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TRBL_H */
