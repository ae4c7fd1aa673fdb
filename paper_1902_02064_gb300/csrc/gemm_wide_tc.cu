// Wide tall-skinny GEMM on the tensor cores (tcgen05, TF32 with split
// operands): Out[:, 0:n] = alpha In[:, 0:K] U + beta Out for FP32 In and Out
// and FP64 U, with n up to a few thousand columns.  This is the thick
// restart's v_i := sum_j v_j U_ji (Sec. III D, the restart formulas under
// Eq. (trb-tmat)) and the Ritz vectors x_i = V y_i of the final Rayleigh-
// Ritz step: K = the basis size (<= 1024), n = the kept vectors (several
// hundred), D rows.
//
// Precision: In and U are split into TF32 parts x = hi + lo (|x - hi - lo|
// <= 2^-22 |x|); a product is a_hi b_hi + a_hi b_lo + a_lo b_hi.  U's parts
// are stacked per 128-column tile as 256 K-major rows (hi, then lo), so one
// N = 256 MMA forms a_hi b_hi (accumulator columns 0-127) and a_hi b_lo
// (128-255), and one N = 128 MMA adds a_lo b_hi into columns 128-255.  The
// tensor cores' FP32 accumulation rounds toward zero, which biases long
// sums; every 32-wide K chunk therefore starts a fresh accumulator (4 MMA
// steps), and the converter warps add each chunk's result into FP32
// register sums with round-to-nearest adds.
//
// Thread block (320 threads), chained by mbarriers only:
// * warp 0 (one lane): TMA loads of a 128-row x 32-column box of In and the
//   256-row x 32-column box of U's split transpose into a ring of 3 stages;
// * warp 1 (one lane): issues the chunk's 8 MMAs into one of two
//   accumulators (2 x 256 tensor-memory columns) and commits them;
// * warps 2-9: split the stage's In box into hi and lo tiles (one of two
//   conversion buffers), then drain the previous chunk's accumulator into
//   their register sums (warp w reads tensor-memory lanes 32 (w mod 4) ..
//   +31 = tile rows, and 64 of the 128 output columns); after a tile's last
//   chunk they write the 128 x 128 output tile.
// Persistent blocks take row tiles t = blockIdx.x + i gridDim.x and, for
// each, all column tiles in turn (the row tile of In is re-read from L2).
// Waits are bounded (tma.cuh); a timeout sets this file's error word, which
// the solver reads at its next synchronisation.  About 210 KB of shared memory
// admit one block per SM, so the 512 tensor-memory columns are free.
#include <cuda.h>

#include <algorithm>

#include "blas.cuh"
#include "tc.cuh"

namespace trbl {

int make_tmap_2d_f32(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows, uint64_t ld,
                     uint32_t box_cols, uint32_t box_rows);

namespace {

__device__ int g_wide_err = 0;

constexpr int kConv = 8;                   // converter warps
constexpr int kThreadsW = 64 + 32 * kConv;  // producer, MMA, converters
constexpr int kStages = 3;
constexpr int kBufs = 2;
constexpr int kM = 128;    // rows per tile (MMA M)
constexpr int kNT = 128;   // output columns per tile
constexpr int kABytes = kM * 128;        // 128 rows x 32 FP32 (16 KB)
constexpr int kBBytes = 2 * kNT * 128;   // 256 rows x 32 FP32 (32 KB)
constexpr int kStageBytes = kABytes + kBBytes;
constexpr int kConvBytes = 2 * kABytes;  // A hi, A lo
constexpr uint32_t kTmemCols = 512;      // two accumulators of 256 columns
constexpr uint32_t kIdescHiLo = idesc_tf32(kM, 2 * kNT);
constexpr uint32_t kIdescHi = idesc_tf32(kM, kNT);

struct WShared {
  uint64_t full[kStages];   // stage landed (TMA bytes)
  uint64_t empty[kStages];  // stage consumed: converter warps (A) + MMA commit (B)
  uint64_t cfull[kBufs];    // conversion buffer written
  uint64_t mdone[kBufs];    // conversion buffer's MMAs completed
  uint64_t accfull[2];      // accumulator's MMAs completed
  uint64_t accfree[2];      // accumulator drained
  uint32_t tmem;
  int abort;
};

__device__ __forceinline__ bool w_aborted(const WShared& sh) { return *reinterpret_cast<const volatile int*>(&sh.abort); }
__device__ __forceinline__ bool w_wait(WShared& sh, uint64_t* bar, uint32_t parity) {
  if (mbar_wait(bar, parity, &g_wide_err)) return true;
  *reinterpret_cast<volatile int*>(&sh.abort) = 1;
  return false;
}

__global__ void __launch_bounds__(kThreadsW, 1)
    gemm_wide_tc_kernel(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tu, int K, int n,
                        float* __restrict__ Out, int64_t ldo, int64_t D, float alpha, float beta) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* stages = base;                           // [kStages][A | B]
  unsigned char* conv = base + kStages * kStageBytes;     // [kBufs][A hi | A lo]
  WShared& sh = *reinterpret_cast<WShared*>(conv + kBufs * kConvBytes);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t nrt = (D + kM - 1) / kM;
  const int nct = (n + kNT - 1) / kNT;
  const int nk = (K + 31) / 32;
  const int64_t my_rt = nrt > blockIdx.x ? (nrt - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t nchunks = my_rt * nct * nk;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&sh.full[s], 1);
      mbar_init(&sh.empty[s], kConv + 1);
    }
    for (int b = 0; b < kBufs; ++b) {
      mbar_init(&sh.cfull[b], kConv);
      mbar_init(&sh.mdone[b], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&sh.accfull[a], 1);
      mbar_init(&sh.accfree[a], kConv);
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
  const uint32_t tmem = sh.tmem;
  int64_t issued = 0, committed = -1;

  if (warp == 0) {
    // ---- TMA producer ----
    if (lane == 0) {
      for (int64_t j = 0; j < nchunks; ++j) {
        const int s = int(j % kStages);
        if (j >= kStages && !w_wait(sh, &sh.empty[s], uint32_t((j / kStages - 1) & 1))) break;
        if (w_aborted(sh)) break;
        const int kc = int(j % nk);
        const int64_t job = j / nk;  // (row tile, column tile) of this block
        const int ct = int(job % nct);
        const int64_t rt = blockIdx.x + (job / nct) * gridDim.x;
        unsigned char* st = stages + s * kStageBytes;
        mbar_expect_tx(&sh.full[s], uint32_t(kStageBytes));
        tma_load_2d(st, &tin, kc * 32, int(rt * kM), &sh.full[s]);
        tma_load_2d(st + kABytes, &tu, kc * 32, ct * 2 * kNT, &sh.full[s]);
        issued = j + 1;
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      for (int64_t j = 0; j < nchunks; ++j) {
        const int s = int(j % kStages), c = int(j % kBufs), a = int(j & 1);
        if (j >= 2 && !w_wait(sh, &sh.accfree[a], uint32_t((j / 2 - 1) & 1))) break;
        if (!w_wait(sh, &sh.cfull[c], uint32_t((j / kBufs) & 1))) break;
        if (w_aborted(sh)) break;
        tc_fence_after();
        const unsigned char* cv = conv + c * kConvBytes;
        const uint64_t dah = sdesc_k128(cv), dal = sdesc_k128(cv + kABytes);
        const uint64_t db = sdesc_k128(stages + s * kStageBytes + kABytes);
        const uint32_t acc = tmem + uint32_t(a * 2 * kNT);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t o = uint64_t(2 * kk);  // +32 bytes in the start-address field
          mma_tf32(acc, dah + o, db + o, kIdescHiLo, kk == 0 ? 0u : 1u);
          mma_tf32(acc + uint32_t(kNT), dal + o, db + o, kIdescHi, 1u);
        }
        mma_commit(&sh.mdone[c]);
        mma_commit(&sh.empty[s]);
        mma_commit(&sh.accfull[a]);
        committed = j;
      }
    }
  } else {
    // ---- converters, drains and epilogues ----
    const int ct_ = tid - 64;
    const int quad = warp & 3, half = (warp - 2) >> 2;
    float sum[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) sum[i] = 0.f;
    // chunk j's accumulator into the sums; after the job's last chunk, the
    // output tile (this thread: row 32 quad + lane, columns 64 half .. +63)
    auto drain = [&](int64_t j) -> bool {
      const int a = int(j & 1);
      if (!w_wait(sh, &sh.accfull[a], uint32_t((j >> 1) & 1))) return false;
      tc_fence_after();
      const uint32_t ta = tmem + (uint32_t(32 * quad) << 16) + uint32_t(a * 2 * kNT + 64 * half);
      // two rounds of four loads in flight, one wait each
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {
        uint32_t v0[16], w0[16], v1[16], w1[16];
        tmem_ld16_nowait(ta + uint32_t(32 * h2), v0);
        tmem_ld16_nowait(ta + uint32_t(kNT + 32 * h2), w0);
        tmem_ld16_nowait(ta + uint32_t(32 * h2 + 16), v1);
        tmem_ld16_nowait(ta + uint32_t(kNT + 32 * h2 + 16), w1);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          float& s0 = sum[32 * h2 + i];
          float& s1 = sum[32 * h2 + 16 + i];
          s0 = __fadd_rn(s0, __fadd_rn(__uint_as_float(v0[i]), __uint_as_float(w0[i])));
          s1 = __fadd_rn(s1, __fadd_rn(__uint_as_float(v1[i]), __uint_as_float(w1[i])));
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.accfree[a]);
      if (j % nk == nk - 1) {
        const int64_t job = j / nk;
        const int c0 = int(job % nct) * kNT + 64 * half;
        const int64_t r = (blockIdx.x + (job / nct) * gridDim.x) * kM + 32 * quad + lane;
        if (r < D && c0 < n) {
          float* o = Out + r * ldo + c0;
          const int nc = std::min(64, n - c0);
          if (nc == 64 && beta == 0.f && (reinterpret_cast<uintptr_t>(o) & 15) == 0) {
            // 16-byte stores: a quarter of the store instructions
#pragma unroll
            for (int i = 0; i < 64; i += 4)
              *reinterpret_cast<float4*>(o + i) =
                  make_float4(alpha * sum[i], alpha * sum[i + 1], alpha * sum[i + 2], alpha * sum[i + 3]);
          } else {
#pragma unroll
            for (int i = 0; i < 64; ++i)
              if (i < nc) o[i] = beta != 0.f ? fmaf(beta, o[i], alpha * sum[i]) : alpha * sum[i];
          }
        }
#pragma unroll
        for (int i = 0; i < 64; ++i) sum[i] = 0.f;
      }
      return true;
    };
    bool live = true;
    for (int64_t j = 0; j < nchunks; ++j) {
      const int s = int(j % kStages), c = int(j % kBufs);
      live = false;
      if (!w_wait(sh, &sh.full[s], uint32_t((j / kStages) & 1))) break;
      if (j >= kBufs && !w_wait(sh, &sh.mdone[c], uint32_t((j / kBufs - 1) & 1))) break;
      if (w_aborted(sh)) break;
      const unsigned char* st = stages + s * kStageBytes;
      unsigned char* cv = conv + c * kConvBytes;
      // In: identical layout in and out, 16 bytes per access (conflict-free)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int off = (ct_ + u * 256) * 16;
        const float4 x = *reinterpret_cast<const float4*>(st + off);
        float h[4], l[4];
        tf32_split(x.x, h[0], l[0]);
        tf32_split(x.y, h[1], l[1]);
        tf32_split(x.z, h[2], l[2]);
        tf32_split(x.w, h[3], l[3]);
        *reinterpret_cast<float4*>(cv + off) = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4*>(cv + kABytes + off) = make_float4(l[0], l[1], l[2], l[3]);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.empty[s]);
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.cfull[c]);
      if (j > 0 && !drain(j - 1)) break;
      live = true;
    }
    if (live && nchunks > 0 && !w_aborted(sh)) drain(nchunks - 1);
  }

  // ---- teardown: after a timeout, wait (bounded) for copies and MMAs in flight ----
  __syncthreads();
  if (w_aborted(sh)) {
    if (warp == 0 && lane == 0)
      for (int64_t jj = std::max<int64_t>(0, issued - kStages); jj < issued; ++jj)
        mbar_wait(&sh.full[jj % kStages], uint32_t((jj / kStages) & 1), nullptr);
    if (warp == 1 && lane == 0 && committed >= 0)
      mbar_wait(&sh.accfull[committed & 1], uint32_t((committed >> 1) & 1), nullptr);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// U (K x n FP64, row-major, ld ldu) as TF32 parts of its transpose, stacked
// per 128-column tile: ut[(256 ct + j) Kp + k] = hi(U[k][128 ct + j]),
// ut[(256 ct + 128 + j) Kp + k] = lo(...), zero past K and n.
__global__ void ut_wide_split_kernel(const double* __restrict__ U, int64_t ldu, int K, int n, int Kp, int nct,
                                     float* __restrict__ ut) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= int64_t(nct) * kNT * Kp) return;
  const int64_t col = e / Kp;  // global output column 128 ct + j
  const int k = int(e - col * Kp);
  const int ct = int(col / kNT), j = int(col - int64_t(ct) * kNT);
  const double u = (k < K && col < n) ? U[int64_t(k) * ldu + col] : 0.0;
  const float hi = tf32_round(float(u));
  const float lo = tf32_round(float(u - double(hi)));
  ut[(int64_t(2 * ct) * kNT + j) * Kp + k] = hi;
  ut[(int64_t(2 * ct + 1) * kNT + j) * Kp + k] = lo;
}

}  // namespace

size_t gemm_wide_tc_workspace_bytes(int K, int n) {
  const int Kp = (K + 31) / 32 * 32;
  const int nct = (n + kNT - 1) / kNT;
  return size_t(nct) * 2 * kNT * Kp * sizeof(float);
}

int gemm_wide_tc_split(const double* U, int64_t ldu, int K, int n, float* ut, size_t ut_bytes, cudaStream_t s) {
  if (K <= 0 || n <= 0) return -1;
  if (!ut || ut_bytes < gemm_wide_tc_workspace_bytes(K, n) || (reinterpret_cast<uintptr_t>(ut) & 15)) return -1;
  const int Kp = (K + 31) / 32 * 32;
  const int nct = (n + kNT - 1) / kNT;
  const int64_t nel = int64_t(nct) * kNT * Kp;
  ut_wide_split_kernel<<<unsigned((nel + 255) / 256), 256, 0, s>>>(U, ldu, K, n, Kp, nct, ut);
  note_launch();
  TRBL_CUDA(cudaGetLastError());
  return TRBL_OK;
}

int gemm_wide_tc_run(const float* In, int64_t ldi, int K, int n, const float* ut, float* Out, int64_t ldo, int64_t D,
                     double alpha, double beta, int sm_count, cudaStream_t s) {
  if (K <= 0 || n <= 0 || D <= 0) return -1;
  if ((reinterpret_cast<uintptr_t>(In) & 15) || (ldi * 4) % 16 || ldi < K || ldo < n) return -1;
  if (D > (int64_t(1) << 31) - kM) return -1;
  const int Kp = (K + 31) / 32 * 32;
  const int nct = (n + kNT - 1) / kNT;
  CUtensorMap tin, tu;
  int rc = make_tmap_2d_f32(&tin, In, uint64_t(K), uint64_t(D), uint64_t(ldi), 32, kM);
  if (!rc) rc = make_tmap_2d_f32(&tu, ut, uint64_t(Kp), uint64_t(nct) * 2 * kNT, uint64_t(Kp), 32, 2 * kNT);
  if (rc) return rc;
  const size_t smem = size_t(kStages) * kStageBytes + size_t(kBufs) * kConvBytes + sizeof(WShared) + 1024;
  static const cudaError_t cfg =
      cudaFuncSetAttribute(gemm_wide_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  TRBL_CUDA(cfg);
  const int64_t nrt = (D + kM - 1) / kM;
  const int grid = int(std::min<int64_t>(nrt, sm_count > 0 ? sm_count : 148));
  gemm_wide_tc_kernel<<<grid, kThreadsW, smem, s>>>(tin, tu, K, n, Out, ldo, D, float(alpha), float(beta));
  note_launch();
  TRBL_CUDA(cudaGetLastError());
  return TRBL_OK;
}

int gemm_wide_tc(const float* In, int64_t ldi, int K, const double* U, int64_t ldu, int n, float* Out, int64_t ldo,
                 int64_t D, double alpha, double beta, float* ut, size_t ut_bytes, int sm_count, cudaStream_t s) {
  if ((reinterpret_cast<uintptr_t>(In) & 15) || (ldi * 4) % 16 || ldi < K || ldo < n || D <= 0 ||
      D > (int64_t(1) << 31) - kM)
    return -1;
  const int rc = gemm_wide_tc_split(U, ldu, K, n, ut, ut_bytes, s);
  if (rc) return rc;
  return gemm_wide_tc_run(In, ldi, K, n, ut, Out, ldo, D, alpha, beta, sm_count, s);
}

int wide_error_to_host(int* host, cudaStream_t s) {
  TRBL_CUDA(cudaMemcpyFromSymbolAsync(host, g_wide_err, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
  return TRBL_OK;
}

}  // namespace trbl
