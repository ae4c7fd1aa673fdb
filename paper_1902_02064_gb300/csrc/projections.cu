// Public projection entry point: C = B^T W (Sec. III C/D, "alpha_k := V_k^T W"
// and the reorthogonalisation coefficients), on the block_dot kernels of
// blas.cu with stream-ordered partial-sum scratch.
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
  if (dtype == TRBL_F64)
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
