// Block projections on the tensor cores (tcgen05, TF32 with split operands),
// FP32 data: C = B^T W (the coefficients "alpha_k := V_k^T W" and those of
// the reorthogonalisation of Sec. III C/D, and the Gram matrices of the
// block QR) and Out = alpha In U + beta Out (the update "W -= V C" and
// W R^-1).
//
// Precision: every FP32 operand value x is split into TF32 parts
// x = hi + lo (|x - hi - lo| <= 2^-22 |x|), and a product a b is formed as
// a_hi b_hi + a_hi b_lo + a_lo b_hi (three MMAs into one FP32 accumulator
// in tensor memory); the dropped a_lo b_lo is below 2^-22 |a b|.  The
// projection drains its accumulator into FP64 registers every 64 stages
// (2,048 rows), so FP32 sums never run over more than 2,048 rows; row
// chunks are then combined in FP64 in a fixed order.
//
// Pipeline of one thread block (256 threads): thread 0 streams 32-row
// stages of the operands by TMA (128-byte swizzle) into a ring of four raw
// stages; all threads convert a raw stage into split K-major operand tiles
// (a transpose for the projection, whose operands are row-major in K) in one
// of two conversion buffers; thread 0 then issues the stage's MMAs and
// commits them to an mbarrier that frees the conversion buffer.  Waits are
// bounded (tma.cuh): a timeout sets an error word the solver reads at its
// next synchronisation, and the block waits (bounded) for its copies and
// MMAs in flight before it frees its tensor memory.  Shared memory (over
// 160 KB) admits one such block per SM, so the 32 tensor-memory columns a
// block allocates are always available.
#include <cuda.h>

#include <algorithm>

#include "blas.cuh"
#include "tc.cuh"

namespace trbl {

int make_tmap_2d_f32(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows, uint64_t ld,
                     uint32_t box_cols, uint32_t box_rows);
void reduce_partials(const double* partial, int nchunk, int mq, double* C, cudaStream_t s);

namespace {

constexpr int kThreadsTC = 256;
constexpr int kRawStages = 4;
constexpr int kDrain = 64;          // projection stages between FP64 drains
constexpr int kTile = 128;          // MMA M: columns of B (projection) or rows of In (update)
constexpr int kN = 32;              // MMA N
constexpr uint32_t kIdesc = idesc_tf32(kTile, kN);
constexpr int kBox = 32 * 32 * 4;   // 32 x 32 FP32 box, 4 KB
constexpr int kTileBytes = kTile * 128;  // 128 rows of 128 bytes, 16 KB

__device__ int g_tc_err = 0;

__device__ __forceinline__ float4 ld4(const unsigned char* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(unsigned char* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}

// Transpose-and-split of one 4 x 4 micro-block of a raw 32-row x 32-column
// box (row = K index r, column = MMA row i; 128-byte swizzle) into the
// K-major hi and lo tiles (row i, K chunk rb): rows r = 4 rb + j, columns
// i = 4 cb + e.  Rows r >= valid read as zero.  The (rb, cb) assignment of
// the caller keeps the eight threads of each 16-byte access phase on
// distinct chunk positions for both the loads and the stores.
__device__ __forceinline__ void transpose_split(const unsigned char* box, unsigned char* hi, unsigned char* lo, int rb,
                                                int cb, int valid) {
  float v[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int r = 4 * rb + j;
    float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r < valid) x = ld4(box + r * 128 + ((cb ^ (r & 7)) << 4));
    v[j][0] = x.x;
    v[j][1] = x.y;
    v[j][2] = x.z;
    v[j][3] = x.w;
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int i = 4 * cb + e;
    const int off = i * 128 + ((rb ^ (i & 7)) << 4);
    float h[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) tf32_split(v[j][e], h[j], l[j]);
    st4(hi + off, h[0], h[1], h[2], h[3]);
    st4(lo + off, l[0], l[1], l[2], l[3]);
  }
}

// Issues the three split MMAs of each of the four K steps of a stage.
__device__ __forceinline__ void issue_split_mmas(uint32_t tmem, const unsigned char* ahi, const unsigned char* alo,
                                                 const unsigned char* bhi, const unsigned char* blo, bool first) {
  const uint64_t dah = sdesc_k128(ahi), dal = sdesc_k128(alo), dbh = sdesc_k128(bhi), dbl = sdesc_k128(blo);
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    const uint64_t o = uint64_t(2 * kk);  // +32 bytes in the start-address field
    mma_tf32(tmem, dah + o, dbh + o, kIdesc, (first && kk == 0) ? 0u : 1u);
    mma_tf32(tmem, dah + o, dbl + o, kIdesc, 1u);
    mma_tf32(tmem, dal + o, dbh + o, kIdesc, 1u);
  }
}

struct TcShared {
  uint64_t full[kRawStages];  // raw stage landed (TMA)
  uint64_t mdone[2];          // conversion buffer's MMAs completed
  uint32_t tmem;              // tensor-memory base address
  int abort;
};

__device__ __forceinline__ unsigned char* align1024(unsigned char* p) {
  return reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

__device__ __forceinline__ void tc_setup(TcShared& sh, int warp) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < kRawStages; ++s) mbar_init(&sh.full[s], 1);
    for (int b = 0; b < 2; ++b) mbar_init(&sh.mdone[b], 1);
    fence_barrier_init();
    sh.abort = 0;
  }
  __syncwarp();
  if (warp == 0) {
    tmem_alloc(&sh.tmem, 32);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

__device__ __forceinline__ void tc_teardown(TcShared& sh, int warp) {
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(sh.tmem, 32);
  }
}

}  // namespace

namespace {

constexpr int kConvBytes = 2 * kTileBytes + 2 * kBox;  // A hi, A lo, B hi, B lo

// Waits (bounded) for the copies still in flight and the last committed
// MMAs of a block that gives up, so that it can free its tensor memory and
// exit safely.
__device__ void tc_drain_after_abort(TcShared& sh, int64_t j, int64_t issued, int64_t committed) {
  for (int64_t jj = j; jj < issued; ++jj)
    mbar_wait(&sh.full[jj % kRawStages], uint32_t((jj / kRawStages) & 1), nullptr);
  if (committed >= 0) mbar_wait(&sh.mdone[committed & 1], uint32_t((committed >> 1) & 1), nullptr);
}

// FP64 partial sums of C = B^T W: blockIdx.x = 128-column tile of B,
// blockIdx.y = row chunk (rows_per_chunk rows, a multiple of 32).  The MMA's
// rows are B's columns (M = 128), its columns W's (N = 32), K runs over the
// chunk's rows.  Raw stage: 4 boxes of B (32 rows x 32 columns) and one of
// W; conversion transposes them into K-major split tiles.
__global__ void __launch_bounds__(kThreadsTC, 1)
    block_dot_tc_kernel(const __grid_constant__ CUtensorMap tb, const __grid_constant__ CUtensorMap tw, int m, int q,
                        int64_t D, int64_t rows_per_chunk, double* __restrict__ partial) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = align1024(smem_raw);
  unsigned char* raw = base;                              // [kRawStages][5 boxes]
  unsigned char* conv = base + kRawStages * 5 * kBox;     // [2][kConvBytes]
  TcShared& sh = *reinterpret_cast<TcShared*>(conv + 2 * kConvBytes);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kTile;
  const int nbox = std::min(4, (m - m0 + 31) / 32);
  const int64_t r_begin = int64_t(blockIdx.y) * rows_per_chunk;
  const int64_t r_end = std::min(D, r_begin + rows_per_chunk);
  const int64_t njobs = r_end > r_begin ? (r_end - r_begin + 31) / 32 : 0;
  tc_setup(sh, warp);
  const uint32_t tmem = sh.tmem;
  const uint32_t stage_bytes = uint32_t(nbox + 1) * kBox;
  auto issue = [&](int64_t j) {
    const int s = int(j % kRawStages);
    unsigned char* st = raw + s * 5 * kBox;
    const int y = int(r_begin + j * 32);
    mbar_expect_tx(&sh.full[s], stage_bytes);
    for (int b = 0; b < nbox; ++b) tma_load_2d(st + b * kBox, &tb, m0 + 32 * b, y, &sh.full[s]);
    tma_load_2d(st + 4 * kBox, &tw, 0, y, &sh.full[s]);
  };
  int64_t issued = 0, committed = -1;
  if (tid == 0)
    for (; issued < std::min<int64_t>(kRawStages, njobs); ++issued) issue(issued);
  // conversion role: box mybox, micro-block (rb, cb) of it (see transpose_split)
  const int P = tid >> 3, a = tid & 7;
  const int rb = a, cb = ((P & 1) << 2) + (((a >> 1) + ((P >> 1) & 3)) & 3);
  const int mybox = P >> 3;
  double acc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = 0.0;
  bool first = true;
  int64_t j = 0;
  for (; j < njobs; ++j) {
    const int s = int(j % kRawStages), c = int(j & 1);
    bool ok = mbar_wait(&sh.full[s], uint32_t((j / kRawStages) & 1), &g_tc_err);
    if (j >= 2) ok = mbar_wait(&sh.mdone[c], uint32_t(((j - 2) >> 1) & 1), &g_tc_err) && ok;
    if (!ok) sh.abort = 1;
    const unsigned char* st = raw + s * 5 * kBox;
    unsigned char* cv = conv + c * kConvBytes;
    const int valid = int(std::min<int64_t>(32, r_end - (r_begin + j * 32)));
    if (ok) {
      if (mybox < nbox)
        transpose_split(st + mybox * kBox, cv + mybox * kBox, cv + kTileBytes + mybox * kBox, rb, cb, valid);
      if (tid < 64) transpose_split(st + 4 * kBox, cv + 2 * kTileBytes, cv + 2 * kTileBytes + kBox, rb, cb, valid);
    }
    fence_async_smem();
    __syncthreads();
    if (sh.abort) break;
    if (tid == 0) {
      if (issued < njobs) issue(issued++);
      tc_fence_after();
      issue_split_mmas(tmem, cv, cv + kTileBytes, cv + 2 * kTileBytes, cv + 2 * kTileBytes + kBox, first);
      mma_commit(&sh.mdone[c]);
      first = false;
    }
    committed = j;
    if ((j + 1) % kDrain == 0 || j == njobs - 1) {
      // move the FP32 accumulator into FP64 registers and restart it
      if (!mbar_wait(&sh.mdone[c], uint32_t((j >> 1) & 1), &g_tc_err)) sh.abort = 1;
      tc_fence_after();
      float v[16];
      tmem_ld16(tmem + (uint32_t(32 * (warp & 3)) << 16) + uint32_t(16 * (warp >> 2)), v);
#pragma unroll
      for (int i = 0; i < 16; ++i) acc[i] += double(v[i]);
      tc_fence_before();
      __syncthreads();
      if (sh.abort) break;
      first = true;
    }
  }
  if (sh.abort) {
    if (tid == 0) tc_drain_after_abort(sh, j, issued, committed);
    tc_teardown(sh, warp);
    return;
  }
  double* Pp = partial + int64_t(blockIdx.y) * m * q;
  const int i = m0 + 32 * (warp & 3) + lane;
  const int c0 = 16 * (warp >> 2);
  if (i < m) {
#pragma unroll
    for (int k = 0; k < 16; ++k)
      if (c0 + k < q) Pp[int64_t(i) * q + c0 + k] = acc[k];
  }
  tc_teardown(sh, warp);
}

// U (K x n, FP64, row-major) as TF32 parts of its transpose for the update's
// B operand: ut[j][k] = hi(U[k][j]), ut[32 + j][k] = lo, rows of Kp values
// (zero past K and n).
__global__ void ut_split_kernel(const double* __restrict__ U, int64_t ldu, int K, int n, int Kp,
                                float* __restrict__ ut) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 32 * Kp) return;
  const int j = e / Kp, k = e - j * Kp;
  const double u = (k < K && j < n) ? U[int64_t(k) * ldu + j] : 0.0;
  const float hi = tf32_round(float(u));
  const float lo = tf32_round(float(u - double(hi)));
  ut[int64_t(j) * Kp + k] = hi;
  ut[int64_t(32 + j) * Kp + k] = lo;
}

// Out = alpha In U + beta Out for persistent blocks striding over 128-row
// tiles of In; the MMA's rows are In's rows (M = 128), its columns U's
// (N = 32), K runs over In's columns in stages of 32.  Raw stage: one In box
// (32 columns x 128 rows, already K-major) and one box of U's split
// transpose (32 columns x 64 rows: hi, then lo); conversion splits In into
// hi and lo tiles of the same layout and copies U's parts.
__global__ void __launch_bounds__(kThreadsTC, 1)
    rowgemm_tc_kernel(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tu, int K, int n,
                      float* __restrict__ Out, int64_t ldo, int64_t D, float alpha, float beta) {
  constexpr int kRawBytes = kTileBytes + 2 * kBox;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = align1024(smem_raw);
  unsigned char* raw = base;                                // [kRawStages][kRawBytes]
  unsigned char* conv = base + kRawStages * kRawBytes;      // [2][kConvBytes]
  TcShared& sh = *reinterpret_cast<TcShared*>(conv + 2 * kConvBytes);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ntiles = (D + kTile - 1) / kTile;
  const int nk = (K + 31) / 32;
  const int64_t my_tiles = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t njobs = my_tiles * nk;
  tc_setup(sh, warp);
  const uint32_t tmem = sh.tmem;
  auto issue = [&](int64_t j) {
    const int s = int(j % kRawStages);
    unsigned char* st = raw + s * kRawBytes;
    const int64_t ti = blockIdx.x + (j / nk) * gridDim.x;
    const int kc = int(j % nk);
    mbar_expect_tx(&sh.full[s], uint32_t(kRawBytes));
    tma_load_2d(st, &tin, kc * 32, int(ti * kTile), &sh.full[s]);
    tma_load_2d(st + kTileBytes, &tu, kc * 32, 0, &sh.full[s]);
  };
  int64_t issued = 0, committed = -1;
  if (tid == 0)
    for (; issued < std::min<int64_t>(kRawStages, njobs); ++issued) issue(issued);
  int64_t j = 0;
  for (; j < njobs; ++j) {
    const int s = int(j % kRawStages), c = int(j & 1);
    const int kc = int(j % nk);
    bool ok = mbar_wait(&sh.full[s], uint32_t((j / kRawStages) & 1), &g_tc_err);
    if (j >= 2) ok = mbar_wait(&sh.mdone[c], uint32_t(((j - 2) >> 1) & 1), &g_tc_err) && ok;
    if (!ok) sh.abort = 1;
    const unsigned char* st = raw + s * kRawBytes;
    unsigned char* cv = conv + c * kConvBytes;
    if (ok) {
      // In: same layout in and out, 16 bytes per access (conflict-free)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int off = (tid + u * kThreadsTC) * 16;
        const float4 x = ld4(st + off);
        float h[4], l[4];
        tf32_split(x.x, h[0], l[0]);
        tf32_split(x.y, h[1], l[1]);
        tf32_split(x.z, h[2], l[2]);
        tf32_split(x.w, h[3], l[3]);
        st4(cv + off, h[0], h[1], h[2], h[3]);
        st4(cv + kTileBytes + off, l[0], l[1], l[2], l[3]);
      }
      // U's hi and lo parts (8 KB)
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int off = (tid + u * kThreadsTC) * 16;
        *reinterpret_cast<float4*>(cv + 2 * kTileBytes + off) = ld4(st + kTileBytes + off);
      }
    }
    fence_async_smem();
    __syncthreads();
    if (sh.abort) break;
    if (tid == 0) {
      if (issued < njobs) issue(issued++);
      tc_fence_after();
      issue_split_mmas(tmem, cv, cv + kTileBytes, cv + 2 * kTileBytes, cv + 2 * kTileBytes + kBox, kc == 0);
      mma_commit(&sh.mdone[c]);
    }
    committed = j;
    if (kc == nk - 1) {
      // epilogue of the tile: this thread's row, 16 of the 32 columns
      if (!mbar_wait(&sh.mdone[c], uint32_t((j >> 1) & 1), &g_tc_err)) sh.abort = 1;
      tc_fence_after();
      float v[16];
      tmem_ld16(tmem + (uint32_t(32 * (warp & 3)) << 16) + uint32_t(16 * (warp >> 2)), v);
      const int64_t r = (blockIdx.x + (j / nk) * gridDim.x) * kTile + 32 * (warp & 3) + lane;
      const int c0 = 16 * (warp >> 2);
      if (!sh.abort && r < D) {
        float* o = Out + r * ldo + c0;
#pragma unroll
        for (int k = 0; k < 16; ++k)
          if (c0 + k < n) o[k] = (beta == 0.f) ? alpha * v[k] : fmaf(beta, o[k], alpha * v[k]);
      }
      tc_fence_before();
      __syncthreads();
      if (sh.abort) break;
    }
  }
  if (sh.abort && tid == 0) tc_drain_after_abort(sh, j, issued, committed);
  tc_teardown(sh, warp);
}

int sm_count_now() {
  static const int sms = [] {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 148;
  }();
  return sms;
}

}  // namespace

int block_dot_tc(const float* B, int64_t ldb, int m, const float* W, int64_t ldw, int q, int64_t D, double* C,
                 double* partial, size_t partial_bytes, int sm_count, cudaStream_t s) {
  if (m <= 0 || q <= 0 || q > kN || D <= 0) return -1;
  if ((reinterpret_cast<uintptr_t>(B) | reinterpret_cast<uintptr_t>(W)) & 15) return -1;
  if ((ldb * 4) % 16 || (ldw * 4) % 16) return -1;
  if (D > (int64_t(1) << 31) - 64) return -1;
  const int mtiles = (m + kTile - 1) / kTile;
  const size_t per_chunk = size_t(m) * q * sizeof(double);
  const int64_t fit = int64_t(partial_bytes / per_chunk);
  if (fit < 1) return -1;
  // one block per SM
  int64_t nchunk = std::max(1, sm_count / mtiles);
  nchunk = std::max<int64_t>(1, std::min(std::min(nchunk, (D + 31) / 32), fit));
  int64_t rows = (D + nchunk - 1) / nchunk;
  rows = (rows + 31) / 32 * 32;
  nchunk = (D + rows - 1) / rows;
  CUtensorMap tb, tw;
  int rc = make_tmap_2d_f32(&tb, B, uint64_t(m), uint64_t(D), uint64_t(ldb), 32, 32);
  if (!rc) rc = make_tmap_2d_f32(&tw, W, uint64_t(q), uint64_t(D), uint64_t(ldw), 32, 32);
  if (rc) return rc;
  const size_t smem = size_t(kRawStages) * 5 * kBox + 2 * size_t(kConvBytes) + sizeof(TcShared) + 1024;
  static const cudaError_t cfg =
      cudaFuncSetAttribute(block_dot_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  TRBL_CUDA(cfg);
  const dim3 grid{unsigned(mtiles), unsigned(nchunk), 1u};
  block_dot_tc_kernel<<<grid, kThreadsTC, smem, s>>>(tb, tw, m, q, D, rows, partial); note_launch();
  TRBL_CUDA(cudaGetLastError());
  reduce_partials(partial, int(nchunk), m * q, C, s);
  TRBL_CUDA(cudaGetLastError());
  return TRBL_OK;
}

size_t rowgemm_tc_workspace_bytes(int K) { return size_t(64) * ((K + 31) / 32 * 32) * sizeof(float); }

int rowgemm_tc(const float* In, int64_t ldi, int K, const double* U, int64_t ldu, int n, float* Out, int64_t ldo,
               int64_t D, double alpha, double beta, float* ut, size_t ut_bytes, cudaStream_t s) {
  if (K <= 0 || n <= 0 || n > kN || D <= 0) return -1;
  if ((reinterpret_cast<uintptr_t>(In) & 15) || (ldi * 4) % 16) return -1;
  if (D > (int64_t(1) << 31) - 2 * kTile) return -1;
  const int Kp = (K + 31) / 32 * 32;
  if (!ut || ut_bytes < rowgemm_tc_workspace_bytes(K) || (reinterpret_cast<uintptr_t>(ut) & 15)) return -1;
  ut_split_kernel<<<(32 * Kp + 255) / 256, 256, 0, s>>>(U, ldu, K, n, Kp, ut); note_launch();
  TRBL_CUDA(cudaGetLastError());
  CUtensorMap tin, tu;
  int rc = make_tmap_2d_f32(&tin, In, uint64_t(K), uint64_t(D), uint64_t(ldi), 32, kTile);
  if (!rc) rc = make_tmap_2d_f32(&tu, ut, uint64_t(Kp), 64, uint64_t(Kp), 32, 64);
  if (rc) return rc;
  const size_t smem = size_t(kRawStages) * (kTileBytes + 2 * kBox) + 2 * size_t(kConvBytes) + sizeof(TcShared) + 1024;
  static const cudaError_t cfg =
      cudaFuncSetAttribute(rowgemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  TRBL_CUDA(cfg);
  const int64_t ntiles = (D + kTile - 1) / kTile;
  const int grid = int(std::min<int64_t>(ntiles, sm_count_now()));
  rowgemm_tc_kernel<<<grid, kThreadsTC, smem, s>>>(tin, tu, K, n, Out, ldo, D, float(alpha), float(beta));
  note_launch();
  TRBL_CUDA(cudaGetLastError());
  return TRBL_OK;
}

int tc_error_to_host(int* host, cudaStream_t s) {
  TRBL_CUDA(cudaMemcpyFromSymbolAsync(host, g_tc_err, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
  return TRBL_OK;
}

}  // namespace trbl
