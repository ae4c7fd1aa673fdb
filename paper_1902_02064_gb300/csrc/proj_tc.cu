// Block projections on the tensor cores (tcgen05, TF32 with split operands),
// FP32 data: C = B^T W (the coefficients "alpha_k := V_k^T W" and those of
// the reorthogonalisation of Sec. III C/D, and the Gram matrices of the
// block QR) and Out = alpha In U + beta Out (the update "W -= V C" and
// W R^-1).
//
// Precision: every FP32 operand value x is split into TF32 parts
// x = hi + lo (|x - hi - lo| <= 2^-22 |x|), and a product a b is formed as
// a_hi b_hi + a_hi b_lo + a_lo b_hi (MMAs into FP32 accumulators in tensor
// memory, summed when read out); the dropped a_lo b_lo is below 2^-22 |a b|.
// The large a_hi b_hi products have an accumulator of their own, the two
// small cross terms share a second one.
//
// The tensor cores' FP32 accumulation rounds toward zero, so every MMA into
// a growing sum loses a fraction of an ulp in one direction: summed over
// 2,048 rows (256 MMAs of K = 8, plus 256 of the cross terms into the same
// accumulator) a Gram matrix came out about 1.6e-5 low on its diagonal,
// leaving the block QR's vectors that much longer than unit length.  The
// projection therefore drains its accumulators every kDrain = 4 stages (128
// rows, 16 MMAs) into compensated FP32 sums (TwoSum, error-free for the
// large part), which become FP64 per row chunk; row chunks are then
// combined in FP64 in a fixed order.
//
// Warp-specialised pipeline of one thread block (320 threads), chained by
// mbarriers only:
// * warp 0 (one lane) streams 32-row stages of the operands by TMA
//   (128-byte swizzle) into a ring of four raw stages;
// * warps 2-9 (256 threads) convert a raw stage into split K-major operand
//   tiles (a transpose for the projection, whose operands are row-major in
//   K) in one of two conversion buffers, then release the raw stage, and
//   read a finished accumulator out one stage later, when its MMAs have
//   had a stage's time to complete;
// * warp 1 (one lane) issues the stage's MMAs and commits them to an
//   mbarrier that frees the conversion buffer;
// * two accumulators in tensor memory alternate between segments (the
//   projection's 4-stage drains) or output tiles (the update), so the
//   converter warps read one out while the MMAs fill the other.
// Waits are bounded (tma.cuh): a timeout sets an error word the solver
// reads at its next synchronisation, and the block waits (bounded) for its
// copies and MMAs in flight before it frees its tensor memory.  Shared
// memory (over 200 KB) admits one such block per SM, so the 128
// tensor-memory columns a block allocates are always available.
#include <cuda.h>

#include <algorithm>

#include "blas.cuh"
#include "tc.cuh"

namespace trbl {

int make_tmap_2d_f32(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows, uint64_t ld,
                     uint32_t box_cols, uint32_t box_rows);
void reduce_partials(const double* partial, int nchunk, int mq, double* C, cudaStream_t s);

namespace {

constexpr int kConvWarps = 8;
constexpr int kThreadsTC = 64 + 32 * kConvWarps;  // producer warp, MMA warp, converter warps
constexpr int kRawStages = 4;
constexpr int kDrain = 4;           // projection stages per accumulator segment
constexpr int kTile = 128;          // MMA M: columns of B (projection) or rows of In (update)
constexpr int kN = 32;              // MMA N (one accumulator = 32 tensor-memory columns)
constexpr int kConvBufs = 2;
constexpr uint32_t kTmemCols = 128;  // two accumulators of 64 columns (hi*hi + lo*hi | hi*lo)
constexpr uint32_t kIdesc = idesc_tf32(kTile, kN);
constexpr uint32_t kIdesc2 = idesc_tf32(kTile, 2 * kN);
constexpr int kBox = 32 * 32 * 4;   // 32 x 32 FP32 box, 4 KB
constexpr int kTileBytes = kTile * 128;  // 128 rows of 128 bytes, 16 KB
constexpr int kConvBytes = 2 * kTileBytes + 2 * kBox;  // A hi, A lo, B hi, B lo

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

// Issues the split MMAs of the four K steps of a stage.  B's hi and lo
// tiles are adjacent (rows 0-31 hi, 32-63 lo), so one N = 64 MMA forms
// a_hi b_hi (accumulator columns 0-31) and a_hi b_lo (columns 32-63) with
// one read of a_hi; a second, N = 32, adds a_lo b_hi into columns 32-63,
// beside the other small cross term.
__device__ __forceinline__ void issue_split_mmas(uint32_t acc, const unsigned char* cv, bool first) {
  const uint64_t dah = sdesc_k128(cv), dal = sdesc_k128(cv + kTileBytes);
  const uint64_t db = sdesc_k128(cv + 2 * kTileBytes);
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    const uint64_t o = uint64_t(2 * kk);  // +32 bytes in the start-address field
    mma_tf32(acc, dah + o, db + o, kIdesc2, (first && kk == 0) ? 0u : 1u);
    mma_tf32(acc + uint32_t(kN), dal + o, db + o, kIdesc, 1u);
  }
}

struct TcShared {
  uint64_t full[kRawStages];   // raw stage landed (TMA bytes)
  uint64_t empty[kRawStages];  // raw stage converted (one arrival per converter warp)
  uint64_t cfull[kConvBufs];   // conversion buffer written (per converter warp)
  uint64_t mdone[kConvBufs];   // conversion buffer's MMAs completed (commit)
  uint64_t accfull[2];         // accumulator's MMAs completed (commit)
  uint64_t accfree[2];         // accumulator read out (per converter warp)
  uint32_t tmem;               // tensor-memory base address
  int abort;
};

__device__ __forceinline__ unsigned char* align1024(unsigned char* p) {
  return reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

__device__ __forceinline__ bool aborted(const TcShared& sh) { return *reinterpret_cast<const volatile int*>(&sh.abort); }
__device__ __forceinline__ void set_abort(TcShared& sh) { *reinterpret_cast<volatile int*>(&sh.abort) = 1; }

// Bounded wait; a timeout stops the whole block.
__device__ __forceinline__ bool wait_or_abort(TcShared& sh, uint64_t* bar, uint32_t parity) {
  if (mbar_wait(bar, parity, &g_tc_err)) return true;
  set_abort(sh);
  return false;
}

__device__ __forceinline__ void tc_setup(TcShared& sh, int warp) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < kRawStages; ++s) {
      mbar_init(&sh.full[s], 1);
      mbar_init(&sh.empty[s], kConvWarps);
    }
    for (int b = 0; b < kConvBufs; ++b) {
      mbar_init(&sh.cfull[b], kConvWarps);
      mbar_init(&sh.mdone[b], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sh.accfull[b], 1);
      mbar_init(&sh.accfree[b], kConvWarps);
    }
    fence_barrier_init();
    sh.abort = 0;
  }
  __syncwarp();
  if (warp == 0) {
    tmem_alloc(&sh.tmem, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

// Whole block, after every role has left its loop.  After a timeout, the
// producer lane waits (bounded) for the copies that may still be in flight
// (only the last kRawStages issued: an earlier slot was refilled, so its
// copy had been consumed) and the MMA lane for its last commit, before the
// tensor memory is freed.
__device__ __forceinline__ void tc_finish(TcShared& sh, int warp, int lane, int64_t issued, int64_t committed) {
  __syncthreads();
  if (aborted(sh)) {
    if (warp == 0 && lane == 0)
      for (int64_t jj = std::max<int64_t>(0, issued - kRawStages); jj < issued; ++jj)
        mbar_wait(&sh.full[jj % kRawStages], uint32_t((jj / kRawStages) & 1), nullptr);
    if (warp == 1 && lane == 0 && committed >= 0)
      mbar_wait(&sh.mdone[committed % kConvBufs], uint32_t((committed / kConvBufs) & 1), nullptr);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(sh.tmem, kTmemCols);
  }
}

// Converter warps: signal that this warp's part of a buffer is written
// (stores made visible to the tensor core first).
__device__ __forceinline__ void warp_arrive_async(uint64_t* bar, int lane) {
  fence_async_smem();
  __syncwarp();
  if (lane == 0) mbar_arrive(bar);
}

// This converter thread's 16 accumulator values (its lane's row, its warp's
// column half) of accumulator a: the a_hi b_hi columns in v, the columns of
// the two cross terms in w.  The warp index mod 4 selects the 32
// tensor-memory lanes a warp may read.
__device__ __forceinline__ void acc_load2(uint32_t tmem, int warp, int a, float (&v)[16], float (&w)[16]) {
  const uint32_t base = tmem + (uint32_t(32 * (warp & 3)) << 16) + uint32_t(a * 2 * kN + 16 * ((warp - 2) >> 2));
  uint32_t rv[16], rw[16];
  tmem_ld16_nowait(base, rv);
  tmem_ld16_nowait(base + kN, rw);
  tmem_wait_ld();
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(rv[i]), w[i] = __uint_as_float(rw[i]);
}

// The same, summed.
__device__ __forceinline__ void acc_load(uint32_t tmem, int warp, int a, float (&v)[16]) {
  float w[16];
  acc_load2(tmem, warp, a, v, w);
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] += w[i];
}

// s + e := hi + x exactly (Knuth's TwoSum, round-to-nearest adds that the
// compiler may not contract or reorder).
__device__ __forceinline__ void two_sum(float& hi, float x, float& e) {
  const float s = __fadd_rn(hi, x);
  const float xb = __fsub_rn(s, hi);
  const float hb = __fsub_rn(s, xb);
  e = __fadd_rn(__fsub_rn(hi, hb), __fsub_rn(x, xb));
  hi = s;
}

}  // namespace

namespace {

// FP64 partial sums of C = B^T W: blockIdx.x = 128-column tile of B,
// blockIdx.y = row chunk (rows_per_chunk rows, a multiple of 32).  The MMA's
// rows are B's columns (M = 128), its columns W's (N = 32), K runs over the
// chunk's rows.  Raw stage j: 4 boxes of B (32 rows x 32 columns) and one of
// W; conversion transposes them into K-major split tiles in buffer j mod 3.
// Accumulator segment g (stages kDrain g .. kDrain g + kDrain - 1) uses
// accumulator g & 1; the converters read segment g out after converting
// the first stage of segment g + 1 (the last segment after the loop).
__global__ void __launch_bounds__(kThreadsTC, 1)
    block_dot_tc_kernel(const __grid_constant__ CUtensorMap tb, const __grid_constant__ CUtensorMap tw, int m, int q,
                        int64_t D, int64_t rows_per_chunk, double* __restrict__ partial) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = align1024(smem_raw);
  unsigned char* raw = base;                              // [kRawStages][5 boxes]
  unsigned char* conv = base + kRawStages * 5 * kBox;     // [kConvBufs][kConvBytes]
  TcShared& sh = *reinterpret_cast<TcShared*>(conv + kConvBufs * kConvBytes);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kTile;
  const int nbox = std::min(4, (m - m0 + 31) / 32);
  const int64_t r_begin = int64_t(blockIdx.y) * rows_per_chunk;
  const int64_t r_end = std::min(D, r_begin + rows_per_chunk);
  const int64_t njobs = r_end > r_begin ? (r_end - r_begin + 31) / 32 : 0;
  tc_setup(sh, warp);
  const uint32_t tmem = sh.tmem;
  int64_t issued = 0, committed = -1;
  float sum_hi[16], sum_lo[16];  // compensated sum of the drained segments
#pragma unroll
  for (int i = 0; i < 16; ++i) sum_hi[i] = sum_lo[i] = 0.f;

  if (warp == 0) {
    // ---- TMA producer ----
    if (lane == 0) {
      const uint32_t stage_bytes = uint32_t(nbox + 1) * kBox;
      for (int64_t j = 0; j < njobs; ++j) {
        const int s = int(j % kRawStages);
        if (j >= kRawStages && !wait_or_abort(sh, &sh.empty[s], uint32_t((j / kRawStages - 1) & 1))) break;
        if (aborted(sh)) break;
        unsigned char* st = raw + s * 5 * kBox;
        const int y = int(r_begin + j * 32);
        mbar_expect_tx(&sh.full[s], stage_bytes);
        for (int b = 0; b < nbox; ++b) tma_load_2d(st + b * kBox, &tb, m0 + 32 * b, y, &sh.full[s]);
        tma_load_2d(st + 4 * kBox, &tw, 0, y, &sh.full[s]);
        issued = j + 1;
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      for (int64_t j = 0; j < njobs; ++j) {
        const int c = int(j % kConvBufs);
        const int64_t g = j / kDrain;
        const int a = int(g & 1);
        const bool seg_first = j % kDrain == 0;
        if (seg_first && g >= 2 && !wait_or_abort(sh, &sh.accfree[a], uint32_t(((g - 2) >> 1) & 1))) break;
        if (!wait_or_abort(sh, &sh.cfull[c], uint32_t((j / kConvBufs) & 1))) break;
        if (aborted(sh)) break;
        tc_fence_after();
        issue_split_mmas(tmem + uint32_t(a * 2 * kN), conv + c * kConvBytes, seg_first);
        mma_commit(&sh.mdone[c]);
        if (j % kDrain == kDrain - 1 || j == njobs - 1) mma_commit(&sh.accfull[a]);
        committed = j;
      }
    }
  } else {
    // ---- converters ----
    const int ct = tid - 64;
    const int P = ct >> 3, a8 = ct & 7;
    const int rb = a8, cb = ((P & 1) << 2) + (((a8 >> 1) + ((P >> 1) & 3)) & 3);
    const int mybox = P >> 3;
    // segment g's accumulator into the compensated sums
    auto drain = [&](int64_t g) -> bool {
      const int a = int(g & 1);
      if (!wait_or_abort(sh, &sh.accfull[a], uint32_t((g >> 1) & 1))) return false;
      tc_fence_after();
      float v[16], w[16];
      acc_load2(tmem, warp, a, v, w);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.accfree[a]);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        float e;
        two_sum(sum_hi[i], v[i], e);
        sum_lo[i] = __fadd_rn(sum_lo[i], __fadd_rn(e, w[i]));
      }
      return true;
    };
    bool live = true;
    for (int64_t j = 0; j < njobs; ++j) {
      const int s = int(j % kRawStages), c = int(j % kConvBufs);
      live = false;
      if (!wait_or_abort(sh, &sh.full[s], uint32_t((j / kRawStages) & 1))) break;
      if (j >= kConvBufs && !wait_or_abort(sh, &sh.mdone[c], uint32_t((j / kConvBufs - 1) & 1))) break;
      if (aborted(sh)) break;
      const unsigned char* st = raw + s * 5 * kBox;
      unsigned char* cv = conv + c * kConvBytes;
      const int valid = int(std::min<int64_t>(32, r_end - (r_begin + j * 32)));
      if (mybox < nbox)
        transpose_split(st + mybox * kBox, cv + mybox * kBox, cv + kTileBytes + mybox * kBox, rb, cb, valid);
      if (ct < 64) transpose_split(st + 4 * kBox, cv + 2 * kTileBytes, cv + 2 * kTileBytes + kBox, rb, cb, valid);
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.empty[s]);
      warp_arrive_async(&sh.cfull[c], lane);
      if (j % kDrain == 0 && j > 0 && !drain(j / kDrain - 1)) break;
      live = true;
    }
    if (live && njobs > 0 && !aborted(sh)) drain((njobs - 1) / kDrain);
  }
  const bool ok = !aborted(sh);
  tc_finish(sh, warp, lane, issued, committed);
  if (warp >= 2 && ok && !aborted(sh)) {
    double* Pp = partial + int64_t(blockIdx.y) * m * q;
    const int i = m0 + 32 * (warp & 3) + lane;
    const int c0 = 16 * ((warp - 2) >> 2);
    if (i < m) {
#pragma unroll
      for (int k = 0; k < 16; ++k)
        if (c0 + k < q) Pp[int64_t(i) * q + c0 + k] = double(sum_hi[k]) + double(sum_lo[k]);
    }
  }
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

// Epilogue of one 128-row output tile held in accumulator a: this converter
// thread's row, 16 of the 32 columns.
__device__ __forceinline__ void update_epilogue(TcShared& sh, uint32_t tmem, int warp, int lane, int a, int64_t t,
                                                int64_t tile, float* __restrict__ Out, int64_t ldo, int64_t D, int n,
                                                float alpha, float beta) {
  if (!wait_or_abort(sh, &sh.accfull[a], uint32_t((t >> 1) & 1))) return;
  tc_fence_after();
  float v[16];
  acc_load(tmem, warp, a, v);
  tc_fence_before();
  __syncwarp();
  if (lane == 0) mbar_arrive(&sh.accfree[a]);
  const int64_t r = tile * kTile + 32 * (warp & 3) + lane;
  const int c0 = 16 * ((warp - 2) >> 2);
  if (r < D && c0 < n) {
    float* o = Out + r * ldo + c0;
    const int nc = std::min(16, n - c0);
    if (nc == 16 && (reinterpret_cast<uintptr_t>(o) & 15) == 0) {
      // 16-byte loads and stores
      float4* o4 = reinterpret_cast<float4*>(o);
      float4 old4[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) old4[k] = beta != 0.f ? o4[k] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int k = 0; k < 4; ++k)
        o4[k] = make_float4(fmaf(beta, old4[k].x, alpha * v[4 * k]), fmaf(beta, old4[k].y, alpha * v[4 * k + 1]),
                            fmaf(beta, old4[k].z, alpha * v[4 * k + 2]), fmaf(beta, old4[k].w, alpha * v[4 * k + 3]));
      return;
    }
    float old[16];
    // all loads of the row first: one memory latency per tile, not one per column
#pragma unroll
    for (int k = 0; k < 16; ++k) old[k] = (beta != 0.f && k < nc) ? o[k] : 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k)
      if (k < nc) o[k] = fmaf(beta, old[k], alpha * v[k]);
  }
}

// Out = alpha In U + beta Out for persistent blocks striding over 128-row
// tiles of In; the MMA's rows are In's rows (M = 128), its columns U's
// (N = 32), K runs over In's columns in stages of 32.  Raw stage: one In box
// (32 columns x 128 rows, already K-major) and one box of U's split
// transpose (32 columns x 64 rows: hi, then lo); conversion splits In into
// hi and lo tiles of the same layout and copies U's parts.  The block's
// t-th tile uses accumulator t & 1; its epilogue runs after the converters
// have converted the next stage, so it overlaps the tile's last MMAs.
__global__ void __launch_bounds__(kThreadsTC, 1)
    rowgemm_tc_kernel(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tu, int K, int n,
                      float* __restrict__ Out, int64_t ldo, int64_t D, float alpha, float beta) {
  constexpr int kRawBytes = kTileBytes + 2 * kBox;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = align1024(smem_raw);
  unsigned char* raw = base;                                // [kRawStages][kRawBytes]
  unsigned char* conv = base + kRawStages * kRawBytes;      // [kConvBufs][kConvBytes]
  TcShared& sh = *reinterpret_cast<TcShared*>(conv + kConvBufs * kConvBytes);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ntiles = (D + kTile - 1) / kTile;
  const int nk = (K + 31) / 32;
  const int64_t my_tiles = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t njobs = my_tiles * nk;
  tc_setup(sh, warp);
  const uint32_t tmem = sh.tmem;
  int64_t issued = 0, committed = -1;

  if (warp == 0) {
    // ---- TMA producer ----
    if (lane == 0) {
      for (int64_t j = 0; j < njobs; ++j) {
        const int s = int(j % kRawStages);
        if (j >= kRawStages && !wait_or_abort(sh, &sh.empty[s], uint32_t((j / kRawStages - 1) & 1))) break;
        if (aborted(sh)) break;
        unsigned char* st = raw + s * kRawBytes;
        const int64_t tile = blockIdx.x + (j / nk) * gridDim.x;
        const int kc = int(j % nk);
        mbar_expect_tx(&sh.full[s], uint32_t(kRawBytes));
        tma_load_2d(st, &tin, kc * 32, int(tile * kTile), &sh.full[s]);
        tma_load_2d(st + kTileBytes, &tu, kc * 32, 0, &sh.full[s]);
        issued = j + 1;
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      for (int64_t j = 0; j < njobs; ++j) {
        const int c = int(j % kConvBufs);
        const int64_t t = j / nk;
        const int kc = int(j % nk);
        const int a = int(t & 1);
        if (kc == 0 && t >= 2 && !wait_or_abort(sh, &sh.accfree[a], uint32_t(((t - 2) >> 1) & 1))) break;
        if (!wait_or_abort(sh, &sh.cfull[c], uint32_t((j / kConvBufs) & 1))) break;
        if (aborted(sh)) break;
        tc_fence_after();
        issue_split_mmas(tmem + uint32_t(a * 2 * kN), conv + c * kConvBytes, kc == 0);
        mma_commit(&sh.mdone[c]);
        if (kc == nk - 1) mma_commit(&sh.accfull[a]);
        committed = j;
      }
    }
  } else {
    // ---- converters (and epilogues) ----
    const int ct = tid - 64;
    int64_t pending = -1;  // local tile index whose epilogue is due
    for (int64_t j = 0; j < njobs; ++j) {
      const int s = int(j % kRawStages), c = int(j % kConvBufs);
      if (!wait_or_abort(sh, &sh.full[s], uint32_t((j / kRawStages) & 1))) break;
      if (j >= kConvBufs && !wait_or_abort(sh, &sh.mdone[c], uint32_t((j / kConvBufs - 1) & 1))) break;
      if (aborted(sh)) break;
      const unsigned char* st = raw + s * kRawBytes;
      unsigned char* cv = conv + c * kConvBytes;
      // In: same layout in and out, 16 bytes per access (conflict-free)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int off = (ct + u * 256) * 16;
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
        const int off = (ct + u * 256) * 16;
        *reinterpret_cast<float4*>(cv + 2 * kTileBytes + off) = ld4(st + kTileBytes + off);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.empty[s]);
      warp_arrive_async(&sh.cfull[c], lane);
      if (pending >= 0) {
        update_epilogue(sh, tmem, warp, lane, int(pending & 1), pending, blockIdx.x + pending * gridDim.x, Out, ldo,
                        D, n, alpha, beta);
        pending = -1;
      }
      if (j % nk == nk - 1) pending = j / nk;
    }
    if (pending >= 0 && !aborted(sh))
      update_epilogue(sh, tmem, warp, lane, int(pending & 1), pending, blockIdx.x + pending * gridDim.x, Out, ldo, D,
                      n, alpha, beta);
  }
  tc_finish(sh, warp, lane, issued, committed);
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
  const size_t smem = size_t(kRawStages) * 5 * kBox + kConvBufs * size_t(kConvBytes) + sizeof(TcShared) + 1024;
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
  const size_t smem = size_t(kRawStages) * (kTileBytes + 2 * kBox) + kConvBufs * size_t(kConvBytes) + sizeof(TcShared) + 1024;
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
