// Tall-skinny dense kernels used by the solver (blas.cu).
#pragma once

#include "internal.h"

namespace trbl {

// Device scratch of the dense kernels (owned by the caller).
struct Workspace {
  double* partial = nullptr;  // block_dot partial sums
  size_t partial_bytes = 0;
  int sm_count = 152;
  float* ut = nullptr;        // rowgemm_tc: split transpose of U
  size_t ut_bytes = 0;
  bool tensor = false;        // FP32 projections on the tensor cores when shapes allow
  int tc_min_k = 1;           // rowgemm_ws: smallest K sent to the tensor cores
};

// Bytes of Workspace::partial needed by block_dot with these m, q.
size_t block_dot_workspace_bytes(int m, int q, int sm_count);

// C[m x q] (FP64, row-major, ld q) = B[:, 0:m]^T W[:, 0:q] over D rows.
template <typename T>
int block_dot(const T* B, int64_t ldb, int m, const T* W, int64_t ldw, int q, int64_t D, double* C,
              Workspace& ws, cudaStream_t s);

// block_dot with a caller-given partial-sum buffer of partial_bytes: the
// number of row chunks is capped so that chunks * m * q doubles fit.
// TRBL_ERR_ARG when even one chunk does not fit.
template <typename T>
int block_dot_capped(const T* B, int64_t ldb, int m, const T* W, int64_t ldw, int q, int64_t D, double* C,
                     double* partial, size_t partial_bytes, int sm_count, cudaStream_t s);

// Loads (under lazy module loading) every kernel block_dot_capped can launch.
int block_dot_capped_load_kernels();

// Out[:, 0:n] = alpha * In[:, 0:K] U[K x n] + beta * Out (U FP64 row-major, ld ldu).
// In and Out must not overlap.
template <typename T>
int rowgemm(const T* In, int64_t ldi, int K, const double* U, int64_t ldu, int n, T* Out,
            int64_t ldo, int64_t D, double alpha, double beta, cudaStream_t s);

// FP32 Out = alpha * In U + beta * Out (n <= 32) with In streamed by TMA
// (rowgemm_tma.cu); -1 when the shapes or alignment do not allow it.
int rowgemm_tma(const float* In, int64_t ldi, int K, const double* U, int64_t ldu, int n, float* Out, int64_t ldo,
                int64_t D, double alpha, double beta, cudaStream_t s);
// Enqueues a copy of the TMA-wait timeout word (0 = none) to host memory.
int tma_error_to_host(int* host, cudaStream_t s);
// FP32 C = B^T W (q <= 32) with TMA-streamed operands (dot_tma.cu); -1 when
// the shapes or alignment do not allow it.
int block_dot_tma(const float* B, int64_t ldb, int m, const float* W, int64_t ldw, int q, int64_t D, double* C,
                  double* partial, size_t partial_bytes, int sm_count, cudaStream_t s);
int dot_error_to_host(int* host, cudaStream_t s);

// rowgemm through the workspace: FP32 data with ws.tensor set go to the
// tensor-core kernel when the shapes allow, else as rowgemm.
template <typename T>
int rowgemm_ws(const T* In, int64_t ldi, int K, const double* U, int64_t ldu, int n, T* Out, int64_t ldo, int64_t D,
               double alpha, double beta, Workspace& ws, cudaStream_t s);

// G = W^T W (q x q, FP64) for a D x q block: a CUDA-core Gram kernel for
// FP32 data with q = 8, 16, 32 or 64, block_dot otherwise; deterministic.
template <typename T>
int gram(const T* W, int64_t ldw, int q, int64_t D, double* G, Workspace& ws, cudaStream_t s);

// out[c] = sum_r W[r][c]^2 for a D x q block (q <= 256), deterministic.
template <typename T>
int col_sumsq(const T* W, int64_t ldw, int q, int64_t D, double* out, Workspace& ws, cudaStream_t s);

// Tensor-core (tcgen05, split TF32) forms for FP32 data, n / q <= 32
// (proj_tc.cu); -1 when the shapes, alignment or workspace do not allow them.
int block_dot_tc(const float* B, int64_t ldb, int m, const float* W, int64_t ldw, int q, int64_t D, double* C,
                 double* partial, size_t partial_bytes, int sm_count, cudaStream_t s);
size_t rowgemm_tc_workspace_bytes(int K);
int rowgemm_tc(const float* In, int64_t ldi, int K, const double* U, int64_t ldu, int n, float* Out, int64_t ldo,
               int64_t D, double alpha, double beta, float* ut, size_t ut_bytes, cudaStream_t s);
// Enqueues a copy of the tensor-core kernels' wait-timeout word to host memory.
int tc_error_to_host(int* host, cudaStream_t s);

// Wide FP32 GEMM on the tensor cores (gemm_wide_tc.cu): Out[:, 0:n] =
// alpha In[:, 0:K] U + beta Out, U FP64 K x n row-major, any n.  The split
// of U into the workspace (gemm_wide_tc_workspace_bytes) can be done once
// and reused by several runs over row panels.  -1 when shapes, alignment or
// workspace do not allow it.
size_t gemm_wide_tc_workspace_bytes(int K, int n);
int gemm_wide_tc_split(const double* U, int64_t ldu, int K, int n, float* ut, size_t ut_bytes, cudaStream_t s);
int gemm_wide_tc_run(const float* In, int64_t ldi, int K, int n, const float* ut, float* Out, int64_t ldo, int64_t D,
                     double alpha, double beta, int sm_count, cudaStream_t s);
int gemm_wide_tc(const float* In, int64_t ldi, int K, const double* U, int64_t ldu, int n, float* Out, int64_t ldo,
                 int64_t D, double alpha, double beta, float* ut, size_t ut_bytes, int sm_count, cudaStream_t s);
// Enqueues a copy of the wide GEMM's wait-timeout word to host memory.
int wide_error_to_host(int* host, cudaStream_t s);

// Batched forms for nset problems of equal column shapes, one launch each
// (plus the reduction): problem s reads and writes through the s-th entry of
// device arrays of pointers and has Ds[s] rows (device array; D = the
// largest, which sizes the grid).  block_dot_batched uses about 1,024 rows
// per thread block so that many small problems fill the GPU together.
// skip (device array, or null): problem s does nothing when skip[s] != 0
// (its outputs keep their contents).
template <typename T>
int block_dot_batched(const T* const* B, int64_t ldb, int m, const T* const* W, int64_t ldw, int q,
                      const int64_t* Ds, int64_t D, double* const* C, double* const* partial, size_t partial_bytes,
                      int nset, cudaStream_t s, const int* skip = nullptr);
template <typename T>
int rowgemm_batched(const T* const* In, int64_t ldi, int K, const double* const* U, int64_t ldu, int n,
                    T* const* Out, int64_t ldo, const int64_t* Ds, int64_t D, double alpha, double beta, int nset,
                    cudaStream_t s, const int* skip = nullptr);
// out[s][c] = sum_r W[s][r][c]^2 over the Ds[s] rows of problem s (q <= 256),
// deterministic; partial[s] needs (4 x SMs) x q doubles.
template <typename T>
int col_sumsq_batched(const T* const* W, int64_t ldw, int q, const int64_t* Ds, int64_t D, double* const* out,
                      double* const* partial, size_t partial_bytes, int sm_count, int nset, cudaStream_t s);

// dst[:, 0:ncol] = src[:, 0:ncol] (with type conversion).
template <typename S, typename T>
int copy_cols(const S* src, int64_t lds, T* dst, int64_t ldd, int64_t D, int ncol, cudaStream_t s);

// X[:, 0] *= a (one column, leading dimension ldx).
template <typename T>
int scale_col(T* X, int64_t ldx, int64_t D, double a, cudaStream_t s);

// Seeded uniform(-1, 1) block: entry (r, col0 + c) uses counter
// (seed << 32) + r * ncol_total + col0 + c through splitmix64.
template <typename T>
int random_block(T* X, int64_t ldx, int64_t D, int ncol, int ncol_total, int col0, uint64_t seed,
                 cudaStream_t s);

}  // namespace trbl
