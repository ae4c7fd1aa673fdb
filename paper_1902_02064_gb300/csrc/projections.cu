// Public projection entry points: C = B^T W (Sec. III C/D, "alpha_k := V_k^T W"
// and the reorthogonalisation coefficients) on the CUDA cores
// (trbl_block_dot) or the tensor cores (trbl_block_dot_tc), and the block
// update Out = alpha In U + beta Out (trbl_block_update), with
// stream-ordered scratch.
#include "blas.cuh"

using namespace trbl;

namespace {

int check_dev(const void* p, const char* name) {
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(TRBL_ERR_ARG, "%s: not a CUDA pointer (%s)", name, cudaGetErrorString(e));
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
    return fail(TRBL_ERR_ARG, "%s must be device memory", name);
  return TRBL_OK;
}

}  // namespace

extern "C" int trbl_block_dot(const void* B, int64_t ldb, int m, const void* W, int64_t ldw, int q, int64_t D,
                              int dtype, double* C, void* stream) {
  clear_error();
  if (!B || !W || !C) return fail(TRBL_ERR_ARG, "null argument");
  if (m < 1 || q < 1 || q > 64 || D < 1) return fail(TRBL_ERR_ARG, "bad sizes m=%d q=%d D=%lld", m, q, (long long)D);
  if (ldb < m || ldw < q) return fail(TRBL_ERR_ARG, "leading dimension smaller than the column count");
  if (dtype != TRBL_F32 && dtype != TRBL_F64) return fail(TRBL_ERR_ARG, "bad dtype %d", dtype);
  int rc = check_dev(B, "B");
  if (!rc) rc = check_dev(W, "W");
  if (!rc) rc = check_dev(C, "C");
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  TRBL_CUDA(cudaGetDevice(&dev));
  TRBL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const size_t bytes = block_dot_workspace_bytes(m, q, sms);
  void* part = nullptr;
  TRBL_CUDA(cudaMallocAsync(&part, bytes, s));
  if (dtype == TRBL_F32 && B == W && ldb == ldw && m == q && (q == 8 || q == 16 || q == 32 || q == 64)) {
    // a Gram matrix: the dedicated kernel reads the block once
    Workspace ws;
    ws.partial = static_cast<double*>(part);
    ws.partial_bytes = bytes;
    ws.sm_count = sms;
    rc = gram<float>(static_cast<const float*>(W), ldw, q, D, C, ws, s);
  } else if (dtype == TRBL_F64)
    rc = block_dot_capped<double>(static_cast<const double*>(B), ldb, m, static_cast<const double*>(W), ldw, q, D, C,
                                  static_cast<double*>(part), bytes, sms, s);
  else
    rc = block_dot_capped<float>(static_cast<const float*>(B), ldb, m, static_cast<const float*>(W), ldw, q, D, C,
                                 static_cast<double*>(part), bytes, sms, s);
  cudaError_t e = cudaFreeAsync(part, s);
  if (rc) return rc;
  TRBL_CUDA(e);
  return TRBL_OK;
}

extern "C" int trbl_block_dot_tc(const void* B, int64_t ldb, int m, const void* W, int64_t ldw, int q, int64_t D,
                                 double* C, void* stream) {
  clear_error();
  if (!B || !W || !C) return fail(TRBL_ERR_ARG, "null argument");
  if (m < 1 || q < 1 || q > 32 || D < 1) return fail(TRBL_ERR_ARG, "bad sizes m=%d q=%d D=%lld", m, q, (long long)D);
  if (ldb < m || ldw < q) return fail(TRBL_ERR_ARG, "leading dimension smaller than the column count");
  if ((reinterpret_cast<uintptr_t>(B) | reinterpret_cast<uintptr_t>(W)) & 15 || ldb % 4 || ldw % 4)
    return fail(TRBL_ERR_ARG, "B and W must be 16-byte aligned with leading dimensions a multiple of 4");
  int rc = check_dev(B, "B");
  if (!rc) rc = check_dev(W, "W");
  if (!rc) rc = check_dev(C, "C");
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  TRBL_CUDA(cudaGetDevice(&dev));
  TRBL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const size_t bytes = block_dot_workspace_bytes(m, q, sms);
  void* part = nullptr;
  TRBL_CUDA(cudaMallocAsync(&part, bytes, s));
  rc = block_dot_tc(static_cast<const float*>(B), ldb, m, static_cast<const float*>(W), ldw, q, D, C,
                    static_cast<double*>(part), bytes, sms, s);
  if (rc == -1) rc = fail(TRBL_ERR_ARG, "shapes not supported by the tensor-core projection");
  cudaError_t e = cudaFreeAsync(part, s);
  if (rc) return rc;
  TRBL_CUDA(e);
  return TRBL_OK;
}

extern "C" int trbl_block_update(const void* In, int64_t ldi, int K, const double* U, int64_t ldu, int n, void* Out,
                                 int64_t ldo, int64_t D, double alpha, double beta, int dtype, int algo,
                                 void* stream) {
  clear_error();
  if (!In || !U || !Out) return fail(TRBL_ERR_ARG, "null argument");
  if (K < 1 || n < 1 || D < 1) return fail(TRBL_ERR_ARG, "bad sizes K=%d n=%d D=%lld", K, n, (long long)D);
  if (ldi < K || ldo < n || ldu < n) return fail(TRBL_ERR_ARG, "leading dimension smaller than the column count");
  if (dtype != TRBL_F32 && dtype != TRBL_F64) return fail(TRBL_ERR_ARG, "bad dtype %d", dtype);
  if (algo != TRBL_PROJ_TENSOR && algo != TRBL_PROJ_CUDA_CORE) return fail(TRBL_ERR_ARG, "bad algo %d", algo);
  int rc = check_dev(In, "In");
  if (!rc) rc = check_dev(U, "U");
  if (!rc) rc = check_dev(Out, "Out");
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (dtype == TRBL_F64)
    return rowgemm<double>(static_cast<const double*>(In), ldi, K, U, ldu, n, static_cast<double*>(Out), ldo, D,
                           alpha, beta, s);
  if (algo == TRBL_PROJ_CUDA_CORE)
    return rowgemm<float>(static_cast<const float*>(In), ldi, K, U, ldu, n, static_cast<float*>(Out), ldo, D, alpha,
                          beta, s);
  if (n > 32) {
    // wide update on the tensor cores (gemm_wide_tc), CUDA cores where its shapes do not apply
    const size_t ub = gemm_wide_tc_workspace_bytes(K, n);
    void* ut = nullptr;
    TRBL_CUDA(cudaMallocAsync(&ut, ub, s));
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    rc = gemm_wide_tc(static_cast<const float*>(In), ldi, K, U, ldu, n, static_cast<float*>(Out), ldo, D, alpha, beta,
                      static_cast<float*>(ut), ub, sms, s);
    if (rc == -1)
      rc = rowgemm<float>(static_cast<const float*>(In), ldi, K, U, ldu, n, static_cast<float*>(Out), ldo, D, alpha,
                          beta, s);
    cudaError_t e = cudaFreeAsync(ut, s);
    if (rc) return rc;
    TRBL_CUDA(e);
    return TRBL_OK;
  }
  Workspace ws;
  ws.tensor = true;
  ws.ut_bytes = rowgemm_tc_workspace_bytes(K);
  void* ut = nullptr;
  TRBL_CUDA(cudaMallocAsync(&ut, ws.ut_bytes, s));
  ws.ut = static_cast<float*>(ut);
  rc = rowgemm_ws<float>(static_cast<const float*>(In), ldi, K, U, ldu, n, static_cast<float*>(Out), ldo, D, alpha,
                         beta, ws, s);
  cudaError_t e = cudaFreeAsync(ut, s);
  if (rc) return rc;
  TRBL_CUDA(e);
  return TRBL_OK;
}
