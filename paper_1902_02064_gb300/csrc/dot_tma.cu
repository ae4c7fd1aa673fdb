// Block projection C = B^T W (FP32 data, FP64 result) with TMA-streamed
// operands: the coefficients "alpha_k := V_k^T W" and those of the
// reorthogonalisation (Sec. III C/D), and the Gram matrix of the block QR.
//
// A thread block owns a 128-column tile of B (4 TMA boxes of 32 columns)
// and a range of rows, which it streams in 64-row stages together with the
// matching rows of W (one box) through a 2-stage shared-memory ring
// (128-byte swizzle, mbarrier completion).  Threads keep 4 x 4 register
// tiles (4 columns of B x 4 columns of W): FP32 products summed per stage,
// stage sums added into a second FP32 level, and the block's partial sums
// written in FP64 for the fixed-order reduction of blas.cu.
#include <cuda.h>

#include <algorithm>

#include "blas.cuh"
#include "tma.cuh"

namespace trbl {

int make_tmap_2d_f32(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows, uint64_t ld,
                     uint32_t box_cols, uint32_t box_rows);
void reduce_partials(const double* partial, int nchunk, int mq, double* C, cudaStream_t s);

namespace {

constexpr int kRS = 64;       // rows per stage
constexpr int kBox = kRS * 32;  // floats per 64 x 32 box (8 KB)
constexpr int kStages = 2;

__device__ int g_dot_err = 0;

__device__ __forceinline__ void lds4v(const float* p, float (&x)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  x[0] = v.x;
  x[1] = v.y;
  x[2] = v.z;
  x[3] = v.w;
}

// Row rr, 16-byte chunk c of a 64 x 32 box stored with 128-byte swizzle.
__device__ __forceinline__ const float* chunk(const float* box, int rr, int c) {
  return box + rr * 32 + ((c ^ (rr & 7)) << 2);
}

__global__ void __launch_bounds__(256, 2) block_dot_tma_kernel(const __grid_constant__ CUtensorMap tb,
                                                               const __grid_constant__ CUtensorMap tw, int m, int q,
                                                               int64_t D, int64_t rows_per_chunk, int nbox,
                                                               double* __restrict__ partial) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float* bufs = reinterpret_cast<float*>(smem_raw);  // [kStages][5 boxes]
  uint64_t* bars = reinterpret_cast<uint64_t*>(bufs + size_t(kStages) * 5 * kBox);
  int& s_abort = *reinterpret_cast<int*>(bars + kStages);
  const int tid = threadIdx.x;
  const int tm = tid & 31, tq = tid >> 5;
  const int m0 = blockIdx.x * 128;
  const int64_t r_begin = int64_t(blockIdx.y) * rows_per_chunk;
  const int64_t r_end = std::min(D, r_begin + rows_per_chunk);
  const int64_t njobs = r_end > r_begin ? (r_end - r_begin + kRS - 1) / kRS : 0;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 1);
    fence_barrier_init();
    s_abort = 0;
  }
  __syncthreads();
  const uint32_t stage_bytes = uint32_t(nbox + 1) * kBox * 4;
  auto issue = [&](int64_t j) {
    const int s = int(j % kStages);
    float* st = bufs + size_t(s) * 5 * kBox;
    const int y = int(r_begin + j * kRS);
    mbar_expect_tx(&bars[s], stage_bytes);
    for (int b = 0; b < nbox; ++b) tma_load_2d(st + b * kBox, &tb, m0 + 32 * b, y, &bars[s]);
    tma_load_2d(st + 4 * kBox, &tw, 0, y, &bars[s]);
  };
  int64_t issued = 0;
  if (tid == 0)
    for (; issued < std::min<int64_t>(kStages, njobs); ++issued) issue(issued);
  float acc[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  const int bb = tm >> 3, bc = tm & 7;  // box and chunk of this thread's 4 B columns
  int64_t j = 0;
  for (; j < njobs; ++j) {
    const int s = int(j % kStages);
    if (!mbar_wait(&bars[s], uint32_t((j / kStages) & 1), &g_dot_err)) s_abort = 1;
    const float* st = bufs + size_t(s) * 5 * kBox;
    const float* Bb = st + bb * kBox;
    const float* Wb = st + 4 * kBox;
    // rows past the chunk end are either zero (past D) or belong to the next
    // chunk: mask them out
    const int valid = int(std::min<int64_t>(kRS, r_end - (r_begin + j * kRS)));
    float t[4][4];
    for (int i = 0; i < 4; ++i)
      for (int jj = 0; jj < 4; ++jj) t[i][jj] = 0.f;
#pragma unroll 4
    for (int rr = 0; rr < valid; ++rr) {
      float b[4], w[4];
      lds4v(chunk(Bb, rr, bc), b);
      lds4v(chunk(Wb, rr, tq), w);
      for (int i = 0; i < 4; ++i)
        for (int jj = 0; jj < 4; ++jj) t[i][jj] = fmaf(b[i], w[jj], t[i][jj]);
    }
    for (int i = 0; i < 4; ++i)
      for (int jj = 0; jj < 4; ++jj) acc[i][jj] += t[i][jj];
    __syncthreads();
    if (s_abort) break;
    if (tid == 0 && issued < njobs) issue(issued++);
  }
  if (s_abort && tid == 0)
    for (int64_t jj = j + 1; jj < issued; ++jj) mbar_wait(&bars[jj % kStages], uint32_t((jj / kStages) & 1), nullptr);
  double* P = partial + int64_t(blockIdx.y) * m * q;
  for (int i = 0; i < 4; ++i) {
    const int bi = m0 + 4 * tm + i;
    if (bi >= m) continue;
    for (int jj = 0; jj < 4; ++jj) {
      const int wj = 4 * tq + jj;
      if (wj < q) P[int64_t(bi) * q + wj] = double(acc[i][jj]);
    }
  }
}

}  // namespace

// -1 when shapes or alignment do not allow the TMA path.
int block_dot_tma(const float* B, int64_t ldb, int m, const float* W, int64_t ldw, int q, int64_t D, double* C,
                  double* partial, size_t partial_bytes, int sm_count, cudaStream_t s) {
  if (m <= 0 || q <= 0 || q > 32 || D <= 0) return -1;
  if ((reinterpret_cast<uintptr_t>(B) | reinterpret_cast<uintptr_t>(W)) & 15) return -1;
  if ((ldb * 4) % 16 || (ldw * 4) % 16) return -1;
  if (D > (int64_t(1) << 31) - kRS) return -1;
  const int mtiles = (m + 127) / 128;
  const size_t per_chunk = size_t(m) * q * sizeof(double);
  const int64_t fit = int64_t(partial_bytes / per_chunk);
  if (fit < 1) return -1;
  int64_t nchunk = (4 * sm_count + mtiles - 1) / mtiles;
  nchunk = std::max<int64_t>(1, std::min(std::min(nchunk, (D + kRS - 1) / kRS), fit));
  int64_t rows = (D + nchunk - 1) / nchunk;
  rows = (rows + kRS - 1) / kRS * kRS;
  nchunk = (D + rows - 1) / rows;
  CUtensorMap tb, tw;
  int rc = make_tmap_2d_f32(&tb, B, uint64_t(m), uint64_t(D), uint64_t(ldb), 32, kRS);
  if (!rc) rc = make_tmap_2d_f32(&tw, W, uint64_t(q), uint64_t(D), uint64_t(ldw), 32, kRS);
  if (rc) return rc;
  const size_t smem = size_t(kStages) * 5 * kBox * 4 + 8 * kStages + 16;
  static const cudaError_t cfg =
      cudaFuncSetAttribute(block_dot_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  TRBL_CUDA(cfg);
  const int nbox = std::min(4, (m + 31) / 32);
  dim3 grid(mtiles, unsigned(nchunk));
  block_dot_tma_kernel<<<grid, 256, smem, s>>>(tb, tw, m, q, D, rows, nbox, partial); note_launch();
  TRBL_CUDA(cudaGetLastError());
  reduce_partials(partial, int(nchunk), m * q, C, s);
  TRBL_CUDA(cudaGetLastError());
  return TRBL_OK;
}

int dot_error_to_host(int* host, cudaStream_t s) {
  TRBL_CUDA(cudaMemcpyFromSymbolAsync(host, g_dot_err, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
  return TRBL_OK;
}

}  // namespace trbl
