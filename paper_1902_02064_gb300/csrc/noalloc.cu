// trbl_block_dot_noalloc: C = B^T W with no device allocation.
//
// The partial-sum scratch of the projection kernels lives in a file-scope
// device array of TRBL_NOALLOC_SCRATCH_BYTES.  Host code cannot use the
// array's name as a device address, so the first call on each device looks
// the address up with cudaGetSymbolAddress (that device current) and caches
// it; later calls on that device reuse it.  The same first call loads every
// kernel the entry point can launch (both element types, every block-width
// bucket, the reduction), so that lazy module loading never loads one, and
// takes device memory for it, during a later call.  Calls that overlap on
// one device share the array and race.
#include <mutex>

#include "blas.cuh"

using namespace trbl;

namespace {

static __device__ __align__(256) double g_scratch[TRBL_NOALLOC_SCRATCH_BYTES / sizeof(double)];

constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {};
int g_sm_count[kMaxDevices] = {};
std::mutex g_mutex;

// Device address of g_scratch and the SM count of the current device.
int scratch_on(int dev, double** addr, int* sms) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    const int rc = block_dot_capped_load_kernels();
    if (rc) return rc;
    g_sm_count[dev] = n > 0 ? n : 1;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *addr = g_scratch_addr[dev];
  *sms = g_sm_count[dev];
  return TRBL_OK;
}

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

extern "C" int trbl_block_dot_noalloc(const void* B, int64_t ldb, int m, const void* W, int64_t ldw, int q,
                                      int64_t D, int dtype, double* C, void* stream) {
  clear_error();
  if (!B || !W || !C) return fail(TRBL_ERR_ARG, "null argument");
  if (m < 1 || q < 1 || q > 64 || D < 1) return fail(TRBL_ERR_ARG, "bad sizes m=%d q=%d D=%lld", m, q, (long long)D);
  if (ldb < m || ldw < q) return fail(TRBL_ERR_ARG, "leading dimension smaller than the column count");
  if (dtype != TRBL_F32 && dtype != TRBL_F64) return fail(TRBL_ERR_ARG, "bad dtype %d", dtype);
  if (size_t(m) * q * sizeof(double) > TRBL_NOALLOC_SCRATCH_BYTES)
    return fail(TRBL_ERR_ARG, "m*q = %lld coefficients exceed the %u-byte no-alloc scratch", (long long)m * q,
                TRBL_NOALLOC_SCRATCH_BYTES);
  int rc = check_dev(B, "B");
  if (!rc) rc = check_dev(W, "W");
  if (!rc) rc = check_dev(C, "C");
  if (rc) return rc;
  int dev = 0;
  TRBL_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(TRBL_ERR_ARG, "device %d beyond the supported %d", dev, kMaxDevices);
  double* scratch = nullptr;
  int sms = 0;
  rc = scratch_on(dev, &scratch, &sms);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (dtype == TRBL_F64)
    return block_dot_capped<double>(static_cast<const double*>(B), ldb, m, static_cast<const double*>(W), ldw, q, D,
                                    C, scratch, TRBL_NOALLOC_SCRATCH_BYTES, sms, s);
  return block_dot_capped<float>(static_cast<const float*>(B), ldb, m, static_cast<const float*>(W), ldw, q, D, C,
                                 scratch, TRBL_NOALLOC_SCRATCH_BYTES, sms, s);
}
