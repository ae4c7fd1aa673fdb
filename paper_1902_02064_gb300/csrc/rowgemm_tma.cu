// Tall-skinny update Out[:, 0:n] = alpha * In[:, 0:K] U + beta * Out with
// In FP32 (the Krylov basis, D x K row-major) and n <= 32: the
// "W -= V C" step of the reorthogonalisation (Sec. III C/D) and W R^{-1} of
// the block QR.
//
// In is streamed by TMA (cp.async.bulk.tensor.2d) in 256-row x 32-column
// boxes with 128-byte swizzle into a ring of shared-memory stages; each
// stage's arrival is tracked by an mbarrier with expected bytes.  U is
// converted from FP64 once per thread block into shared memory.  Warps own
// 32-row x 16-column patches of the output tile; a lane holds 4 rows
// (8 apart) x 4 columns, so the 8 distinct rows a warp reads per k fall in
// distinct banks under the swizzle.  Persistent blocks stride over row
// tiles.  Waits are bounded (tma.cuh): a timeout sets an error word the
// solver reads at its next synchronisation.
#include <cuda.h>

#include <algorithm>

#include "blas.cuh"
#include "tma.cuh"

namespace trbl {
namespace {

constexpr int kRT = 256;  // rows per tile (TMA box rows)
constexpr int kKC = 32;   // K per stage (TMA box columns: 128 bytes)

__device__ int g_tma_err = 0;

__device__ __forceinline__ void lds4f(const float* p, float (&x)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  x[0] = v.x;
  x[1] = v.y;
  x[2] = v.z;
  x[3] = v.w;
}

template <int NP>
__global__ void __launch_bounds__(NP * 16) rowgemm_tma_kernel(const __grid_constant__ CUtensorMap tmap, int K,
                                                              const double* __restrict__ U, int64_t ldu, int n,
                                                              float* __restrict__ Out, int64_t ldo, int64_t D,
                                                              float alpha, float beta, int nstage) {
  constexpr int NT = NP * 16;  // (kRT / 32 row blocks) x (NP / 16 column halves) warps
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float* stages = reinterpret_cast<float*>(smem_raw);
  const int Kp = (K + kKC - 1) / kKC * kKC;
  float* Us = stages + size_t(nstage) * kRT * kKC;
  uint64_t* bars = reinterpret_cast<uint64_t*>(Us + size_t(Kp) * NP);
  int& s_abort = *reinterpret_cast<int*>(bars + nstage);  // kept in the dynamic region: the swizzled
                                                          // stages need a 1024-byte aligned start
  const int tid = threadIdx.x;
  for (int i = tid; i < Kp * NP; i += NT) {
    const int k = i / NP, c = i - k * NP;
    Us[i] = (k < K && c < n) ? float(U[int64_t(k) * ldu + c]) : 0.f;
  }
  if (tid == 0) {
    for (int s = 0; s < nstage; ++s) mbar_init(&bars[s], 1);
    fence_barrier_init();
    s_abort = 0;
  }
  __syncthreads();
  const int64_t ntiles = (D + kRT - 1) / kRT;
  const int nk = Kp / kKC;
  const int64_t my_tiles = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t njobs = my_tiles * nk;
  auto issue = [&](int64_t j) {
    const int s = int(j % nstage);
    const int64_t ti = blockIdx.x + (j / nk) * gridDim.x;
    const int kc = int(j % nk);
    mbar_expect_tx(&bars[s], kRT * kKC * 4);
    tma_load_2d(stages + size_t(s) * kRT * kKC, &tmap, kc * kKC, int(ti * kRT), &bars[s]);
  };
  int64_t issued = 0;
  if (tid == 0) {
    for (; issued < std::min<int64_t>(nstage, njobs); ++issued) issue(issued);
  }
  const int warp = tid >> 5, lane = tid & 31;
  const int rb = warp % (kRT / 32), ch = warp / (kRT / 32);
  const int row8 = lane >> 2, cq = lane & 3;
  const int rbase = rb * 32 + row8;  // rows rbase + 8 i
  const int cbase = ch * 16 + cq * 4;
  // acc sums one 32-wide K chunk; tot sums the chunks (round-to-nearest
  // adds), so a long K does not run through one FP32 accumulator
  float acc[4][4], tot[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) acc[i][j] = tot[i][j] = 0.f;
  int64_t j = 0;
  for (; j < njobs; ++j) {
    const int s = int(j % nstage);
    const uint32_t par = uint32_t((j / nstage) & 1);
    const int kc = int(j % nk);
    if (!mbar_wait(&bars[s], par, &g_tma_err)) s_abort = 1;
    const float* Bs = stages + size_t(s) * kRT * kKC;
    const float* U0 = Us + size_t(kc) * kKC * NP + cbase;
#pragma unroll 8
    for (int kk = 0; kk < kKC; ++kk) {
      const int col = (((kk >> 2) ^ row8) << 2) | (kk & 3);
      float b[4], u[4];
      for (int i = 0; i < 4; ++i) b[i] = Bs[(rbase + 8 * i) * kKC + col];
      lds4f(U0 + kk * NP, u);
      for (int i = 0; i < 4; ++i)
        for (int jj = 0; jj < 4; ++jj) acc[i][jj] = fmaf(b[i], u[jj], acc[i][jj]);
    }
    for (int i = 0; i < 4; ++i)
      for (int jj = 0; jj < 4; ++jj) {
        tot[i][jj] = __fadd_rn(tot[i][jj], acc[i][jj]);
        acc[i][jj] = 0.f;
      }
    if (kc == nk - 1) {
      const int64_t ti = blockIdx.x + (j / nk) * gridDim.x;
      for (int i = 0; i < 4; ++i) {
        const int64_t r = ti * kRT + rbase + 8 * i;
        if (r < D) {
          for (int jj = 0; jj < 4; ++jj) {
            const int c = cbase + jj;
            if (c < n) {
              float* o = Out + r * ldo + c;
              const float v = alpha * tot[i][jj];
              *o = (beta == 0.f) ? v : fmaf(beta, *o, v);
            }
          }
        }
        for (int jj = 0; jj < 4; ++jj) tot[i][jj] = 0.f;
      }
    }
    __syncthreads();  // stage s fully read
    if (s_abort) break;
    if (tid == 0 && issued < njobs) issue(issued++);
  }
  if (s_abort && tid == 0) {
    // let copies still in flight land before the block exits (bounded)
    for (int64_t jj = j + 1; jj < issued; ++jj)
      mbar_wait(&bars[jj % nstage], uint32_t((jj / nstage) & 1), nullptr);
  }
}

template <int NP>
int launch_np(const CUtensorMap& map, int K, const double* U, int64_t ldu, int n, float* Out, int64_t ldo, int64_t D,
              double alpha, double beta, cudaStream_t s) {
  static const int sms = [] {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 148;
  }();
  const int Kp = (K + kKC - 1) / kKC * kKC;
  const size_t ubytes = size_t(Kp) * NP * 4;
  const size_t stage = size_t(kRT) * kKC * 4;
  const size_t limit = 225 * 1024;
  int nstage = 3;
  while (nstage > 2 && size_t(nstage) * stage + ubytes + 64 > limit) --nstage;
  const size_t smem = size_t(nstage) * stage + ubytes + 8 * size_t(nstage) + 16;
  if (smem > limit) return -1;
  static const cudaError_t cfg =
      cudaFuncSetAttribute(rowgemm_tma_kernel<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(limit));
  TRBL_CUDA(cfg);
  const int64_t ntiles = (D + kRT - 1) / kRT;
  const int per_sm = smem * 2 <= limit ? 2 : 1;
  const int grid = int(std::min<int64_t>(ntiles, int64_t(sms) * per_sm));
  rowgemm_tma_kernel<NP><<<grid, NP * 16, smem, s>>>(map, K, U, ldu, n, Out, ldo, D, float(alpha), float(beta),
                                                     nstage); note_launch();
  TRBL_CUDA(cudaGetLastError());
  return TRBL_OK;
}

}  // namespace

namespace {
int encode_tmap_2d_f32(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows, uint64_t ld,
                       uint32_t box_cols, uint32_t box_rows, CUtensorMapSwizzle swizzle) {
  using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static const EncodeFn encode = []() -> EncodeFn {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<EncodeFn>(fn);
  }();
  if (!encode) return fail(TRBL_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {ld * 4};
  const cuuint32_t box[2] = {box_cols, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(TRBL_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", int(r));
  return TRBL_OK;
}
}  // namespace

int make_tmap_2d_f32(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows, uint64_t ld,
                     uint32_t box_cols, uint32_t box_rows) {
  return encode_tmap_2d_f32(map, base, cols, rows, ld, box_cols, box_rows, CU_TENSOR_MAP_SWIZZLE_128B);
}

int make_tmap_2d_f32_rows(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows, uint64_t ld,
                          uint32_t box_cols, uint32_t box_rows) {
  return encode_tmap_2d_f32(map, base, cols, rows, ld, box_cols, box_rows, CU_TENSOR_MAP_SWIZZLE_NONE);
}

int rowgemm_tma(const float* In, int64_t ldi, int K, const double* U, int64_t ldu, int n, float* Out, int64_t ldo,
                int64_t D, double alpha, double beta, cudaStream_t s) {
  if (K <= 0 || n <= 0 || n > 32 || D <= 0) return -1;
  if ((reinterpret_cast<uintptr_t>(In) & 15) || (ldi * 4) % 16) return -1;
  if (D > (int64_t(1) << 31) - kRT) return -1;
  CUtensorMap map;
  int rc = make_tmap_2d_f32(&map, In, uint64_t(K), uint64_t(D), uint64_t(ldi), kKC, kRT);
  if (rc) return rc;
  if (n <= 16) return launch_np<16>(map, K, U, ldu, n, Out, ldo, D, alpha, beta, s);
  return launch_np<32>(map, K, U, ldu, n, Out, ldo, D, alpha, beta, s);
}

int tma_error_to_host(int* host, cudaStream_t s) {
  TRBL_CUDA(cudaMemcpyFromSymbolAsync(host, g_tma_err, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
  return TRBL_OK;
}

}  // namespace trbl
