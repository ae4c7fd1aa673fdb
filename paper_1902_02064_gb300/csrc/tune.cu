// Autotuner of the block product's launch shape.  Three knobs:
// * the kernel: the grouped kernel (any q, FP32 or FP64), the same with
//   two 16-byte chunks per lane (half the lanes per element), the FP32
//   fast kernel (rows of 32, 64 or 128 bytes), or the split product (FP32,
//   q a multiple of 16: like-particle terms by the grouped kernel, the
//   cross-species term by the source-stationary kernel);
// * neutron rows per work item: the grid size, the share of staging work per
//   thread block and how many target determinants are in flight (L2 reuse);
// * resident thread blocks per SM the fast kernel is compiled for (8 blocks
//   at 32 registers a thread, or 6 at 40): warps in flight against
//   registers per warp.
// Lanes per element and chunks per lane follow from the kernel, q and the
// element size (one lane group reads one whole row of V).  Each candidate is
// timed with CUDA events on the caller's stream and the fastest is kept;
// the product's results do not depend on the choice.
#include <algorithm>
#include <cmath>

#include "internal.h"

using namespace trbl;

namespace {

struct Shape {
  int kernel, rows, bps;
};

// Candidate order, as reported in trbl_apply_autotune's ms[].
constexpr Shape kCand[TRBL_TUNE_CANDIDATES] = {
    {TRBL_APPLY_GROUPED, 16, 8}, {TRBL_APPLY_GROUPED, 32, 8}, {TRBL_APPLY_GROUPED, 64, 8},
    {TRBL_APPLY_GROUPED, 128, 8}, {TRBL_APPLY_FAST, 16, 8},   {TRBL_APPLY_FAST, 32, 8},
    {TRBL_APPLY_FAST, 64, 8},     {TRBL_APPLY_FAST, 16, 6},   {TRBL_APPLY_FAST, 32, 6},
    {TRBL_APPLY_FAST, 64, 6},     {TRBL_APPLY_GROUPED_X2, 16, 8}, {TRBL_APPLY_GROUPED_X2, 32, 8},
    {TRBL_APPLY_GROUPED_X2, 64, 8}, {TRBL_APPLY_SPLIT, 64, 2},   {TRBL_APPLY_SPLIT_X4, 64, 2}};

int set_shape(trbl_hamiltonian* h, const Shape& c) {
  h->apply_kernel = c.kernel;
  h->blocks_per_sm = c.bps;
  return h->rows_per_item == c.rows ? TRBL_OK : set_work_items(h, c.rows);
}

}  // namespace

extern "C" int trbl_apply_autotune(trbl_hamiltonian* h, int q, int dtype, float* ms, int* best_rows, void* stream) {
  clear_error();
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
  const bool fast = dtype == TRBL_F32 && (q == 8 || q == 16 || q == 32) && h->g32.likeB && h->b->ND <= 31 &&
                    h->b->D * q < (int64_t(1) << 31);
  const int row_bytes = q * (dtype == TRBL_F64 ? 8 : 4);
  const bool x2 = row_bytes == 32 || row_bytes == 64 || row_bytes == 128;
  const bool split = dtype == TRBL_F32 && (q == 16 || q == 32 || q == 64) && h->pn.oseg && h->b->D * q < (int64_t(1) << 31);
  float best = 1e30f;
  Shape keep{h->apply_kernel, h->rows_per_item, h->blocks_per_sm};
  int rc = TRBL_OK;
  for (int c = 0; c < TRBL_TUNE_CANDIDATES && !rc; ++c) {
    if (ms) ms[c] = NAN;
    if (kCand[c].kernel == TRBL_APPLY_FAST && !fast) continue;
    if (kCand[c].kernel == TRBL_APPLY_GROUPED_X2 && !x2) continue;
    if ((kCand[c].kernel == TRBL_APPLY_SPLIT || kCand[c].kernel == TRBL_APPLY_SPLIT_X4) && !split) continue;
    rc = set_shape(h, kCand[c]);
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
      keep = kCand[c];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (rc) return rc;
  if (best_rows) *best_rows = keep.rows;
  return set_shape(h, keep);
}

extern "C" int trbl_apply_set_rows(trbl_hamiltonian* h, int rows_per_item) {
  clear_error();
  if (!h) return fail(TRBL_ERR_ARG, "null Hamiltonian");
  if (rows_per_item < 1 || rows_per_item > 4096) return fail(TRBL_ERR_ARG, "rows per work item must be in [1, 4096]");
  if (!h->garena) return fail(TRBL_ERR_ARG, "the grouped product is not available for this basis");
  return set_work_items(h, rows_per_item);
}

extern "C" int trbl_apply_set_shape(trbl_hamiltonian* h, int kernel, int rows_per_item, int blocks_per_sm) {
  clear_error();
  if (!h) return fail(TRBL_ERR_ARG, "null Hamiltonian");
  if (kernel != TRBL_APPLY_GROUPED && kernel != TRBL_APPLY_FAST && kernel != TRBL_APPLY_GROUPED_X2 &&
      kernel != TRBL_APPLY_SPLIT && kernel != TRBL_APPLY_SPLIT_X4 && kernel != TRBL_APPLY_SPLIT_TMA)
    return fail(TRBL_ERR_ARG, "unknown kernel %d", kernel);
  if (rows_per_item < 1 || rows_per_item > 4096) return fail(TRBL_ERR_ARG, "rows per work item must be in [1, 4096]");
  if (kernel == TRBL_APPLY_FAST && blocks_per_sm != 6 && blocks_per_sm != 8)
    return fail(TRBL_ERR_ARG, "blocks per SM of the fast kernel must be 6 or 8");
  if (kernel == TRBL_APPLY_SPLIT && blocks_per_sm != 1 && blocks_per_sm != 2)
    return fail(TRBL_ERR_ARG, "blocks per SM of the split product must be 1 or 2");
  if (kernel == TRBL_APPLY_SPLIT_X4 && blocks_per_sm != 2)
    return fail(TRBL_ERR_ARG, "blocks per SM of TRBL_APPLY_SPLIT_X4 must be 2");
  if (kernel == TRBL_APPLY_SPLIT_TMA && blocks_per_sm != 1)
    return fail(TRBL_ERR_ARG, "blocks per SM of TRBL_APPLY_SPLIT_TMA must be 1");
  if (blocks_per_sm != 1 && blocks_per_sm != 2 && blocks_per_sm != 6 && blocks_per_sm != 8)
    return fail(TRBL_ERR_ARG, "blocks per SM must be 1, 2, 6 or 8");
  if (!h->garena) return fail(TRBL_ERR_ARG, "the grouped product is not available for this basis");
  return set_shape(h, Shape{kernel, rows_per_item, blocks_per_sm});
}

extern "C" int trbl_apply_get_shape(const trbl_hamiltonian* h, int* kernel, int* rows_per_item, int* blocks_per_sm) {
  clear_error();
  if (!h) return fail(TRBL_ERR_ARG, "null Hamiltonian");
  if (kernel) *kernel = h->apply_kernel;
  if (rows_per_item) *rows_per_item = h->rows_per_item;
  if (blocks_per_sm) *blocks_per_sm = h->blocks_per_sm;
  return TRBL_OK;
}

extern "C" int trbl_apply_set_compensated(trbl_hamiltonian* h, int on) {
  clear_error();
  if (!h) return fail(TRBL_ERR_ARG, "null Hamiltonian");
  if (on != 0 && on != 1) return fail(TRBL_ERR_ARG, "compensated must be 0 or 1");
  h->apply_compensated = on;
  return TRBL_OK;
}
