// Autotuner of the grouped block product: the number of neutron rows per
// work item sets the grid size, the share of staging work per thread block
// and how many target determinants are in flight (L2 reuse).  Each candidate
// is timed with CUDA events on the caller's stream and the fastest is kept.
#include <algorithm>

#include "internal.h"

using namespace trbl;

extern "C" int trbl_apply_autotune(trbl_hamiltonian* h, int q, int dtype, float* ms, int* best_rows, void* stream) {
  clear_error();
  static const int kCand[4] = {16, 32, 64, 128};
  if (!h) return fail(TRBL_ERR_ARG, "null Hamiltonian");
  if (q < 1 || q > 64 || (dtype != TRBL_F32 && dtype != TRBL_F64)) return fail(TRBL_ERR_ARG, "bad q or dtype");
  if (!h->garena) return fail(TRBL_ERR_ARG, "the grouped product is not available for this basis");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bytes = size_t(h->b->D) * q * (dtype == TRBL_F64 ? 8 : 4);
  void* buf = nullptr;
  TRBL_CUDA(cudaMalloc(&buf, 2 * bytes));
  TRBL_CUDA(cudaMemsetAsync(buf, 0, bytes, s));
  void* V = buf;
  void* W = static_cast<char*>(buf) + bytes;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int bestr = h->rows_per_item;
  int rc = TRBL_OK;
  for (int c = 0; c < 4 && !rc; ++c) {
    rc = set_work_items(h, kCand[c]);
    if (rc) break;
    rc = launch_apply(h, V, q, W, q, q, dtype, s);  // warm-up
    if (rc) break;
    cudaEventRecord(e0, s);
    for (int r = 0; r < 3 && !rc; ++r) rc = launch_apply(h, V, q, W, q, q, dtype, s);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    t /= 3.f;
    if (ms) ms[c] = t;
    if (t < best) {
      best = t;
      bestr = kCand[c];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (rc) return rc;
  if (best_rows) *best_rows = bestr;
  return set_work_items(h, bestr);
}

extern "C" int trbl_apply_set_rows(trbl_hamiltonian* h, int rows_per_item) {
  clear_error();
  if (!h) return fail(TRBL_ERR_ARG, "null Hamiltonian");
  if (rows_per_item < 1 || rows_per_item > 4096) return fail(TRBL_ERR_ARG, "rows per work item must be in [1, 4096]");
  if (!h->garena) return fail(TRBL_ERR_ARG, "the grouped product is not available for this basis");
  return set_work_items(h, rows_per_item);
}
