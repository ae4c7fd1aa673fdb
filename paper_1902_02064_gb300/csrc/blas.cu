// Tall-skinny dense kernels of the block Lanczos step (Sec. III C/D):
//   * block_dot:  C = B^T W  (m x q coefficients of W against m stored
//     vectors; Alg. 3/4 "alpha_k := V_k^T W" and the reorthogonalisation),
//   * rowgemm:    Out = alpha * In U + beta * Out  (W -= B C in the
//     reorthogonalisation, W R^{-1} in the block QR, and the restart
//     compression v_k := sum_j v_j U_jk of Sec. III D),
//   * column copies, casts and the seeded start block.
// Vectors are row-major D x ld.  Small matrices (C, U, R) are FP64.
// In FP32 storage the products are FP32 FMAs summed in two FP32 levels per
// thread block, and the per-block partial sums are reduced across blocks in
// FP64 in a fixed order (deterministic).
#include <algorithm>
#include <type_traits>

#include "blas.cuh"

namespace trbl {

namespace {

constexpr int MT = 128;  // stored vectors per block_dot tile

// Four consecutive values from shared memory as 16-byte vector loads
// (address 16-byte aligned).
__device__ __forceinline__ void lds4(const float* p, float (&x)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  x[0] = v.x;
  x[1] = v.y;
  x[2] = v.z;
  x[3] = v.w;
}
__device__ __forceinline__ void lds4(const double* p, double (&x)[4]) {
  const double2 v0 = *reinterpret_cast<const double2*>(p);
  const double2 v1 = *reinterpret_cast<const double2*>(p + 2);
  x[0] = v0.x;
  x[1] = v0.y;
  x[2] = v1.x;
  x[3] = v1.y;
}

template <typename T>
struct DotCfg;
template <>
struct DotCfg<float> {
  static constexpr int RS = 32;  // rows per shared-memory stage
};
template <>
struct DotCfg<double> {
  static constexpr int RS = 16;
};

// partial[chunk][i][j] = sum over the chunk's rows r of B[r, m0+i] W[r, j]
// grid = (m tiles, row chunks); threads = 32 x (QP/4); thread (tm, tq)
// owns b-columns 4tm..4tm+3 and w-columns 4tq..4tq+3.
template <typename T, int QP>
__global__ void __launch_bounds__(32 * (QP / 4)) block_dot_kernel(
    const T* __restrict__ B, int64_t ldb, int m, const T* __restrict__ W, int64_t ldw, int q,
    int64_t D, int64_t rows_per_chunk, double* __restrict__ partial) {
  constexpr int RS = DotCfg<T>::RS;
  constexpr int NT = 32 * (QP / 4);
  __shared__ __align__(16) T Bs[RS][MT];
  __shared__ __align__(16) T Ws[RS][QP];
  const int tid = threadIdx.x;
  const int tm = tid & 31, tq = tid >> 5;
  const int m0 = blockIdx.x * MT;
  const int64_t r_begin = int64_t(blockIdx.y) * rows_per_chunk;
  const int64_t r_end = min(D, r_begin + rows_per_chunk);
  T acc[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int64_t r0 = r_begin; r0 < r_end; r0 += RS) {
    for (int idx = tid; idx < RS * MT; idx += NT) {
      const int rr = idx / MT, cc = idx - rr * MT;
      const int64_t r = r0 + rr;
      Bs[rr][cc] = (r < r_end && m0 + cc < m) ? B[r * ldb + m0 + cc] : T(0);
    }
    for (int idx = tid; idx < RS * QP; idx += NT) {
      const int rr = idx / QP, cc = idx - rr * QP;
      const int64_t r = r0 + rr;
      Ws[rr][cc] = (r < r_end && cc < q) ? W[r * ldw + cc] : T(0);
    }
    __syncthreads();
    T t[4][4];
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) t[i][j] = T(0);
#pragma unroll 4
    for (int rr = 0; rr < RS; ++rr) {
      T b[4], w[4];
      lds4(&Bs[rr][4 * tm], b);
      lds4(&Ws[rr][4 * tq], w);
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) t[i][j] = fma(b[i], w[j], t[i][j]);
    }
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) acc[i][j] += t[i][j];
    __syncthreads();
  }
  double* P = partial + int64_t(blockIdx.y) * m * q;
  for (int i = 0; i < 4; ++i) {
    const int bi = m0 + 4 * tm + i;
    if (bi >= m) continue;
    for (int j = 0; j < 4; ++j) {
      const int wj = 4 * tq + j;
      if (wj < q) P[int64_t(bi) * q + wj] = double(acc[i][j]);
    }
  }
}


// block_dot_kernel for several problems of equal shapes: grid z = problem;
// problem z reads B[z], W[z] and writes partial[z].
template <typename T, int QP>
__global__ void __launch_bounds__(32 * (QP / 4)) block_dot_batched_kernel(
    const T* const* __restrict__ Bs_, int64_t ldb, int m, const T* const* __restrict__ Ws_, int64_t ldw, int q,
    const int64_t* __restrict__ Ds, int64_t rows_per_chunk, double* const* __restrict__ partials,
    const int* __restrict__ skip) {
  if (skip && skip[blockIdx.z]) return;
  const int64_t D = Ds[blockIdx.z];
  const T* __restrict__ B = Bs_[blockIdx.z];
  const T* __restrict__ W = Ws_[blockIdx.z];
  double* __restrict__ partial = partials[blockIdx.z];
  constexpr int RS = DotCfg<T>::RS;
  constexpr int NT = 32 * (QP / 4);
  __shared__ __align__(16) T Bs[RS][MT];
  __shared__ __align__(16) T Ws[RS][QP];
  const int tid = threadIdx.x;
  const int tm = tid & 31, tq = tid >> 5;
  const int m0 = blockIdx.x * MT;
  const int64_t r_begin = int64_t(blockIdx.y) * rows_per_chunk;
  const int64_t r_end = min(D, r_begin + rows_per_chunk);
  T acc[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int64_t r0 = r_begin; r0 < r_end; r0 += RS) {
    for (int idx = tid; idx < RS * MT; idx += NT) {
      const int rr = idx / MT, cc = idx - rr * MT;
      const int64_t r = r0 + rr;
      Bs[rr][cc] = (r < r_end && m0 + cc < m) ? B[r * ldb + m0 + cc] : T(0);
    }
    for (int idx = tid; idx < RS * QP; idx += NT) {
      const int rr = idx / QP, cc = idx - rr * QP;
      const int64_t r = r0 + rr;
      Ws[rr][cc] = (r < r_end && cc < q) ? W[r * ldw + cc] : T(0);
    }
    __syncthreads();
    T t[4][4];
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) t[i][j] = T(0);
#pragma unroll 4
    for (int rr = 0; rr < RS; ++rr) {
      T b[4], w[4];
      lds4(&Bs[rr][4 * tm], b);
      lds4(&Ws[rr][4 * tq], w);
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) t[i][j] = fma(b[i], w[j], t[i][j]);
    }
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) acc[i][j] += t[i][j];
    __syncthreads();
  }
  double* P = partial + int64_t(blockIdx.y) * m * q;
  for (int i = 0; i < 4; ++i) {
    const int bi = m0 + 4 * tm + i;
    if (bi >= m) continue;
    for (int j = 0; j < 4; ++j) {
      const int wj = 4 * tq + j;
      if (wj < q) P[int64_t(bi) * q + wj] = double(acc[i][j]);
    }
  }
}


__global__ void reduce_partials_kernel(const double* __restrict__ partial, int nchunk, int mq,
                                       double* __restrict__ C) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= mq) return;
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += partial[int64_t(c) * mq + i];
  C[i] = s;
}

__global__ void reduce_partials_batched_kernel(double* const* __restrict__ partial, int nchunk, int mq,
                                               double* const* __restrict__ C, const int* __restrict__ skip) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= mq || (skip && skip[blockIdx.y])) return;
  const double* P = partial[blockIdx.y];
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += P[int64_t(c) * mq + i];
  C[blockIdx.y][i] = s;
}

// Out[r, c] = alpha * sum_k In[r, k] U[k, c] + beta * Out[r, c]
// Tile RT rows x CT columns, k staged KC at a time; thread owns 4 x 4.
template <typename T, int RT, int CT>
__global__ void __launch_bounds__(RT * CT / 16) rowgemm_kernel(
    const T* __restrict__ In, int64_t ldi, int K, const double* __restrict__ U, int64_t ldu, int n,
    T* __restrict__ Out, int64_t ldo, int64_t D, double alpha, double beta) {
  constexpr int KC = 32;
  constexpr int NT = RT * CT / 16;
  constexpr int TR = RT / 4;
  __shared__ __align__(16) T Bs[KC][RT + 4];
  __shared__ __align__(16) T Us[KC][CT];
  const int tid = threadIdx.x;
  const int tr = tid % TR, tc = tid / TR;
  const int64_t r0 = int64_t(blockIdx.x) * RT;
  const int c0 = blockIdx.y * CT;
  T acc[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int k0 = 0; k0 < K; k0 += KC) {
    for (int idx = tid; idx < RT * KC; idx += NT) {
      const int rr = idx / KC, kk = idx - rr * KC;
      const int64_t r = r0 + rr;
      Bs[kk][rr] = (r < D && k0 + kk < K) ? In[r * ldi + k0 + kk] : T(0);
    }
    for (int idx = tid; idx < KC * CT; idx += NT) {
      const int kk = idx / CT, cc = idx - kk * CT;
      Us[kk][cc] = (k0 + kk < K && c0 + cc < n) ? T(U[int64_t(k0 + kk) * ldu + c0 + cc]) : T(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < KC; ++kk) {
      T b[4], u[4];
      lds4(&Bs[kk][4 * tr], b);
      lds4(&Us[kk][4 * tc], u);
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(b[i], u[j], acc[i][j]);
    }
    __syncthreads();
  }
  for (int i = 0; i < 4; ++i) {
    const int64_t r = r0 + 4 * tr + i;
    if (r >= D) continue;
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + 4 * tc + j;
      if (c >= n) continue;
      T* o = Out + r * ldo + c;
      const T v = T(alpha) * acc[i][j];
      *o = (beta == 0.0) ? v : fma(T(beta), *o, v);
    }
  }
}


// rowgemm_kernel for several problems of equal shapes: grid z = problem;
// problem z reads In[z], U[z] and updates Out[z].
template <typename T, int RT, int CT>
__global__ void __launch_bounds__(RT * CT / 16) rowgemm_batched_kernel(
    const T* const* __restrict__ Ins, int64_t ldi, int K, const double* const* __restrict__ Us_, int64_t ldu, int n,
    T* const* __restrict__ Outs, int64_t ldo, const int64_t* __restrict__ Ds, double alpha, double beta,
    const int* __restrict__ skip) {
  if (skip && skip[blockIdx.z]) return;
  const int64_t D = Ds[blockIdx.z];
  if (int64_t(blockIdx.x) * RT >= D) return;
  const T* __restrict__ In = Ins[blockIdx.z];
  const double* __restrict__ U = Us_[blockIdx.z];
  T* __restrict__ Out = Outs[blockIdx.z];
  constexpr int KC = 32;
  constexpr int NT = RT * CT / 16;
  constexpr int TR = RT / 4;
  __shared__ __align__(16) T Bs[KC][RT + 4];
  __shared__ __align__(16) T Us[KC][CT];
  const int tid = threadIdx.x;
  const int tr = tid % TR, tc = tid / TR;
  const int64_t r0 = int64_t(blockIdx.x) * RT;
  const int c0 = blockIdx.y * CT;
  T acc[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int k0 = 0; k0 < K; k0 += KC) {
    for (int idx = tid; idx < RT * KC; idx += NT) {
      const int rr = idx / KC, kk = idx - rr * KC;
      const int64_t r = r0 + rr;
      Bs[kk][rr] = (r < D && k0 + kk < K) ? In[r * ldi + k0 + kk] : T(0);
    }
    for (int idx = tid; idx < KC * CT; idx += NT) {
      const int kk = idx / CT, cc = idx - kk * CT;
      Us[kk][cc] = (k0 + kk < K && c0 + cc < n) ? T(U[int64_t(k0 + kk) * ldu + c0 + cc]) : T(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < KC; ++kk) {
      T b[4], u[4];
      lds4(&Bs[kk][4 * tr], b);
      lds4(&Us[kk][4 * tc], u);
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(b[i], u[j], acc[i][j]);
    }
    __syncthreads();
  }
  for (int i = 0; i < 4; ++i) {
    const int64_t r = r0 + 4 * tr + i;
    if (r >= D) continue;
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + 4 * tc + j;
      if (c >= n) continue;
      T* o = Out + r * ldo + c;
      const T v = T(alpha) * acc[i][j];
      *o = (beta == 0.0) ? v : fma(T(beta), *o, v);
    }
  }
}


// Tall-skinny Out[:, 0:n] = alpha * In[:, 0:K] U + beta * Out with n <= NP <= 64:
// U (K x n, FP64) is converted once per thread block into shared memory;
// persistent blocks stride over row tiles of RT rows; the In tile of the
// next K-chunk is fetched into registers while the current one is used.
template <typename T, int NP>
__global__ void __launch_bounds__(512) rowgemm_tall_kernel(const T* __restrict__ In, int64_t ldi, int K,
                                                           const double* __restrict__ U, int64_t ldu, int n,
                                                           T* __restrict__ Out, int64_t ldo, int64_t D,
                                                           double alpha, double beta) {
  constexpr int NT = 512, KC = 32;
  constexpr int TC = NP / 4, TR = NT / TC, RT = 4 * TR;
  constexpr int LD = RT + 4;
  constexpr int PER = RT * KC / NT;  // In elements each thread fetches per chunk
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Us = reinterpret_cast<T*>(smem_raw);  // [Kp * NP], Kp = K rounded up to KC
  const int Kp = (K + KC - 1) / KC * KC;
  T* Bs = Us + size_t(Kp) * NP;            // [2][KC][LD]
  const int tid = threadIdx.x;
  for (int i = tid; i < Kp * NP; i += NT) {
    const int k = i / NP, c = i - k * NP;
    Us[i] = (k < K && c < n) ? T(U[int64_t(k) * ldu + c]) : T(0);
  }
  const int tr = tid % TR, tc = tid / TR;
  const int64_t ntiles = (D + RT - 1) / RT;
  const T al = T(alpha), be = T(beta);
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * RT;
    T acc[4][4];
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    T pre[PER];
    auto fetch = [&](int k0) {
#pragma unroll
      for (int e = 0; e < PER; ++e) {
        const int idx = tid + e * NT;
        const int rr = idx / KC, kk = idx - rr * KC;
        const int64_t r = r0 + rr;
        pre[e] = (r < D && k0 + kk < K) ? In[r * ldi + k0 + kk] : T(0);
      }
    };
    auto stash = [&](int buf) {
#pragma unroll
      for (int e = 0; e < PER; ++e) {
        const int idx = tid + e * NT;
        const int rr = idx / KC, kk = idx - rr * KC;
        Bs[(buf * KC + kk) * LD + rr] = pre[e];
      }
    };
    fetch(0);
    __syncthreads();  // Us ready; previous tile's readers of Bs are done
    stash(0);
    __syncthreads();
    int buf = 0;
    for (int k0 = 0; k0 < K; k0 += KC) {
      const bool more = k0 + KC < K;
      if (more) fetch(k0 + KC);
      const T* B0 = Bs + buf * KC * LD + 4 * tr;
      const T* U0 = Us + size_t(k0) * NP + 4 * tc;
#pragma unroll 8
      for (int kk = 0; kk < KC; ++kk) {
        T b[4], u[4];
        lds4(B0 + kk * LD, b);
        lds4(U0 + kk * NP, u);
        for (int i = 0; i < 4; ++i)
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(b[i], u[j], acc[i][j]);
      }
      if (more) {
        stash(buf ^ 1);
        __syncthreads();
        buf ^= 1;
      }
    }
    for (int i = 0; i < 4; ++i) {
      const int64_t r = r0 + 4 * tr + i;
      if (r >= D) continue;
      for (int j = 0; j < 4; ++j) {
        const int c = 4 * tc + j;
        if (c >= n) continue;
        T* o = Out + r * ldo + c;
        const T v = al * acc[i][j];
        *o = (beta == 0.0) ? v : fma(be, *o, v);
      }
    }
  }
}

// Narrow forms for q (resp. n) <= NQ <= 4 columns: the one-vector Lanczos
// (q = 1) and the column-wise QR.  The wide kernels above compute 4 x 4
// register tiles, so up to 15 of 16 products would be padding; in FP64,
// whose FMA rate is a small fraction of FP32's, that padding dominated.
//
// partial[chunk][i][j] = sum over the chunk's rows r of B[r, i] W[r, j]:
// thread = one column i of B (256 consecutive columns per block, coalesced
// row reads), W's row broadcast to all threads.  FP32 data sum 32-row
// segments before adding them to the running sum.
template <typename T, int NQ>
__global__ void __launch_bounds__(256) dot_narrow_kernel(const T* __restrict__ B, int64_t ldb, int m,
                                                        const T* __restrict__ W, int64_t ldw, int q, int64_t D,
                                                        int64_t rows_per_chunk, double* __restrict__ partial) {
  const int i = blockIdx.x * 256 + threadIdx.x;
  const int64_t r0 = int64_t(blockIdx.y) * rows_per_chunk;
  const int64_t r1 = min(D, r0 + rows_per_chunk);
  T acc[NQ];
#pragma unroll
  for (int j = 0; j < NQ; ++j) acc[j] = T(0);
  if (i < m) {
    for (int64_t r = r0; r < r1; r += 32) {
      const int64_t re = min(r1, r + 32);
      T t[NQ];
#pragma unroll
      for (int j = 0; j < NQ; ++j) t[j] = T(0);
      for (int64_t rr = r; rr < re; ++rr) {
        const T b = B[rr * ldb + i];
#pragma unroll
        for (int j = 0; j < NQ; ++j)
          if (j < q) t[j] = fma(b, __ldg(W + rr * ldw + j), t[j]);
      }
#pragma unroll
      for (int j = 0; j < NQ; ++j) acc[j] += t[j];
    }
    double* P = partial + int64_t(blockIdx.y) * m * q + int64_t(i) * q;
#pragma unroll
    for (int j = 0; j < NQ; ++j)
      if (j < q) P[j] = double(acc[j]);
  }
}

// Out[r, 0:n] = alpha In[r, 0:K] U + beta Out[r, 0:n], n <= NQ: a warp per
// row (lanes stride over K, coalesced), U staged in shared memory, the
// lanes' partial sums combined by shuffles; persistent blocks of 8 warps.
template <typename T, int NQ>
__global__ void __launch_bounds__(256) rowgemm_narrow_kernel(const T* __restrict__ In, int64_t ldi, int K,
                                                            const double* __restrict__ U, int64_t ldu, int n,
                                                            T* __restrict__ Out, int64_t ldo, int64_t D, double alpha,
                                                            double beta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Us = reinterpret_cast<T*>(smem_raw);  // [K][NQ]
  for (int e = threadIdx.x; e < K * NQ; e += 256) {
    const int k = e / NQ, c = e - k * NQ;
    Us[e] = c < n ? T(U[int64_t(k) * ldu + c]) : T(0);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = int64_t(gridDim.x) * 8;
  for (int64_t r = int64_t(blockIdx.x) * 8 + (threadIdx.x >> 5); r < D; r += warps) {
    const T* row = In + r * ldi;
    T acc[NQ];
#pragma unroll
    for (int c = 0; c < NQ; ++c) acc[c] = T(0);
    for (int k = lane; k < K; k += 32) {
      const T x = row[k];
#pragma unroll
      for (int c = 0; c < NQ; ++c) acc[c] = fma(x, Us[k * NQ + c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < NQ; ++c)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
    if (lane < n) {
      T v = acc[0];
#pragma unroll
      for (int c = 1; c < NQ; ++c)
        if (lane == c) v = acc[c];
      T* o = Out + r * ldo + lane;
      const T a = T(alpha) * v;
      *o = (beta == 0.0) ? a : fma(T(beta), *o, a);
    }
  }
}

template <typename T>
__global__ void scale_col_kernel(T* __restrict__ X, int64_t ldx, int64_t D, double a) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r < D) X[r * ldx] = T(a * double(X[r * ldx]));
}

template <typename S, typename T>
__global__ void copy_cols_kernel(const S* __restrict__ src, int64_t lds, T* __restrict__ dst,
                                 int64_t ldd, int64_t D, int ncol) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t r = i / ncol;
  const int c = int(i - r * ncol);
  if (r >= D) return;
  dst[r * ldd + c] = T(src[r * lds + c]);
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// X[r, c] = 2u - 1 with u = top 53 bits of splitmix64((seed<<32) + r*ncol_total + col0 + c)
template <typename T>
__global__ void random_block_kernel(T* __restrict__ X, int64_t ldx, int64_t D, int ncol,
                                    int ncol_total, int col0, uint64_t seed) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t r = i / ncol;
  const int c = int(i - r * ncol);
  if (r >= D) return;
  const uint64_t ctr = ((seed & 0xffffffffull) << 32) + uint64_t(r) * ncol_total + col0 + c;
  const double u = double(splitmix64(ctr) >> 11) * (1.0 / 9007199254740992.0);
  X[r * ldx + c] = T(2.0 * u - 1.0);
}

template <typename T, int QP>
int dot_launch(const T* B, int64_t ldb, int m, const T* W, int64_t ldw, int q, int64_t D,
               double* C, Workspace& ws, cudaStream_t s) {
  constexpr int RS = DotCfg<T>::RS;
  const int mtiles = (m + MT - 1) / MT;
  const int target = 4 * ws.sm_count;
  int64_t nchunk = (target + mtiles - 1) / mtiles;
  const int64_t max_chunks = (D + RS - 1) / RS;
  if (nchunk > max_chunks) nchunk = max_chunks;
  if (nchunk < 1) nchunk = 1;
  int64_t rows = (D + nchunk - 1) / nchunk;
  rows = (rows + RS - 1) / RS * RS;
  nchunk = (D + rows - 1) / rows;
  const size_t need = size_t(nchunk) * m * q * sizeof(double);
  if (need > ws.partial_bytes) return fail(TRBL_ERR_ARG, "block_dot workspace too small");
  dim3 grid(mtiles, unsigned(nchunk));
  block_dot_kernel<T, QP><<<grid, 32 * (QP / 4), 0, s>>>(B, ldb, m, W, ldw, q, D, rows, ws.partial); note_launch();
  TRBL_CUDA(cudaGetLastError());
  const int mq = m * q;
  reduce_partials_kernel<<<(mq + 255) / 256, 256, 0, s>>>(ws.partial, int(nchunk), mq, C); note_launch();
  TRBL_CUDA(cudaGetLastError());
  return TRBL_OK;
}

template <typename T, int QP>
int dot_launch_capped(const T* B, int64_t ldb, int m, const T* W, int64_t ldw, int q, int64_t D, double* C,
                      double* partial, size_t partial_bytes, int sm_count, cudaStream_t s) {
  constexpr int RS = DotCfg<T>::RS;
  const int mtiles = (m + MT - 1) / MT;
  const size_t per_chunk = size_t(m) * q * sizeof(double);
  const int64_t fit = int64_t(partial_bytes / per_chunk);
  if (fit < 1) return fail(TRBL_ERR_ARG, "block_dot: m*q = %lld exceeds the partial-sum buffer", (long long)m * q);
  int64_t nchunk = (4 * sm_count + mtiles - 1) / mtiles;
  const int64_t max_chunks = (D + RS - 1) / RS;
  nchunk = std::max<int64_t>(1, std::min(std::min(nchunk, max_chunks), fit));
  int64_t rows = (D + nchunk - 1) / nchunk;
  rows = (rows + RS - 1) / RS * RS;
  nchunk = (D + rows - 1) / rows;
  dim3 grid(mtiles, unsigned(nchunk));
  block_dot_kernel<T, QP><<<grid, 32 * (QP / 4), 0, s>>>(B, ldb, m, W, ldw, q, D, rows, partial); note_launch();
  TRBL_CUDA(cudaGetLastError());
  const int mq = m * q;
  reduce_partials_kernel<<<(mq + 255) / 256, 256, 0, s>>>(partial, int(nchunk), mq, C); note_launch();
  TRBL_CUDA(cudaGetLastError());
  return TRBL_OK;
}

// block_dot for q <= 4 through dot_narrow_kernel; the chunk count fits the
// workspace that block_dot_workspace_bytes sizes for the same m and q.
template <typename T>
int dot_narrow(const T* B, int64_t ldb, int m, const T* W, int64_t ldw, int q, int64_t D, double* C, Workspace& ws,
               cudaStream_t s) {
  const int mt = (m + 255) / 256;
  const int64_t fit = int64_t(ws.partial_bytes / (size_t(m) * q * sizeof(double)));
  if (fit < 1) return fail(TRBL_ERR_ARG, "block_dot workspace too small");
  int64_t nchunk = std::max<int64_t>(1, std::min<int64_t>((4 * ws.sm_count + mt - 1) / mt, fit));
  nchunk = std::min<int64_t>(nchunk, (D + 31) / 32);
  int64_t rows = (D + nchunk - 1) / nchunk;
  rows = (rows + 31) / 32 * 32;
  nchunk = (D + rows - 1) / rows;
  const dim3 grid{unsigned(mt), unsigned(nchunk), 1u};
  if (q == 1)
    dot_narrow_kernel<T, 1><<<grid, 256, 0, s>>>(B, ldb, m, W, ldw, q, D, rows, ws.partial);
  else if (q == 2)
    dot_narrow_kernel<T, 2><<<grid, 256, 0, s>>>(B, ldb, m, W, ldw, q, D, rows, ws.partial);
  else
    dot_narrow_kernel<T, 4><<<grid, 256, 0, s>>>(B, ldb, m, W, ldw, q, D, rows, ws.partial);
  note_launch();
  TRBL_CUDA(cudaGetLastError());
  const int mq = m * q;
  reduce_partials_kernel<<<(mq + 255) / 256, 256, 0, s>>>(ws.partial, int(nchunk), mq, C);
  note_launch();
  TRBL_CUDA(cudaGetLastError());
  return TRBL_OK;
}

template <typename T, int NQ>
int narrow_launch(const T* In, int64_t ldi, int K, const double* U, int64_t ldu, int n, T* Out, int64_t ldo,
                  int64_t D, double alpha, double beta, cudaStream_t s) {
  static const cudaError_t cfg = cudaFuncSetAttribute(rowgemm_narrow_kernel<T, NQ>,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  TRBL_CUDA(cfg);
  static const int sms = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 148;
  }();
  const size_t smem = size_t(K) * NQ * sizeof(T);
  const int64_t blocks = std::min<int64_t>((D + 7) / 8, int64_t(sms) * 4);
  rowgemm_narrow_kernel<T, NQ><<<unsigned(blocks), 256, smem, s>>>(In, ldi, K, U, ldu, n, Out, ldo, D, alpha, beta);
  note_launch();
  TRBL_CUDA(cudaGetLastError());
  return TRBL_OK;
}

}  // namespace

void reduce_partials(const double* partial, int nchunk, int mq, double* C, cudaStream_t s) {
  reduce_partials_kernel<<<(mq + 255) / 256, 256, 0, s>>>(partial, nchunk, mq, C); note_launch();
}

template <typename T>
int block_dot_batched(const T* const* B, int64_t ldb, int m, const T* const* W, int64_t ldw, int q,
                      const int64_t* Ds, int64_t D, double* const* C, double* const* partial, size_t partial_bytes,
                      int nset, cudaStream_t s, const int* skip) {
  if (m <= 0 || nset <= 0 || D <= 0) return TRBL_OK;
  constexpr int RS = DotCfg<T>::RS;
  const int mtiles = (m + MT - 1) / MT;
  const int64_t fit = int64_t(partial_bytes / (size_t(m) * q * sizeof(double)));
  if (fit < 1) return fail(TRBL_ERR_ARG, "batched block_dot: workspace too small");
  // about 1,024 rows per block: the problems together fill the GPU
  int64_t nchunk = std::min<int64_t>(std::min<int64_t>((D + 1023) / 1024, fit), 65535);
  nchunk = std::max<int64_t>(nchunk, 1);
  int64_t rows = (D + nchunk - 1) / nchunk;
  rows = (rows + RS - 1) / RS * RS;
  nchunk = (D + rows - 1) / rows;
  const dim3 grid{unsigned(mtiles), unsigned(nchunk), unsigned(nset)};
#define TRBL_BDOT(QP) \
  block_dot_batched_kernel<T, QP><<<grid, 32 * (QP / 4), 0, s>>>(B, ldb, m, W, ldw, q, Ds, rows, partial, skip)
  if (q <= 4) TRBL_BDOT(4);
  else if (q <= 8) TRBL_BDOT(8);
  else if (q <= 16) TRBL_BDOT(16);
  else if (q <= 32) TRBL_BDOT(32);
  else if (q <= 64) TRBL_BDOT(64);
  else return fail(TRBL_ERR_ARG, "batched block_dot: q=%d > 64", q);
#undef TRBL_BDOT
  note_launch();
  TRBL_CUDA(cudaGetLastError());
  const int mq = m * q;
  const dim3 rgrid{unsigned((mq + 255) / 256), unsigned(nset), 1u};
  reduce_partials_batched_kernel<<<rgrid, 256, 0, s>>>(partial, int(nchunk), mq, C, skip); note_launch();
  TRBL_CUDA(cudaGetLastError());
  return TRBL_OK;
}

template <typename T>
int rowgemm_batched(const T* const* In, int64_t ldi, int K, const double* const* U, int64_t ldu, int n,
                    T* const* Out, int64_t ldo, const int64_t* Ds, int64_t D, double alpha, double beta, int nset,
                    cudaStream_t s, const int* skip) {
  if (n <= 0 || D <= 0 || K <= 0 || nset <= 0) return TRBL_OK;
  if (n <= 16) {
    constexpr int RT = 128, CT = 16;
    const dim3 grid{unsigned((D + RT - 1) / RT), unsigned((n + CT - 1) / CT), unsigned(nset)};
    rowgemm_batched_kernel<T, RT, CT><<<grid, RT * CT / 16, 0, s>>>(In, ldi, K, U, ldu, n, Out, ldo, Ds, alpha, beta,
                                                                                 skip);
  } else if (n <= 32) {
    constexpr int RT = 128, CT = 32;
    const dim3 grid{unsigned((D + RT - 1) / RT), unsigned((n + CT - 1) / CT), unsigned(nset)};
    rowgemm_batched_kernel<T, RT, CT><<<grid, RT * CT / 16, 0, s>>>(In, ldi, K, U, ldu, n, Out, ldo, Ds, alpha, beta,
                                                                                 skip);
  } else {
    constexpr int RT = 64, CT = 64;
    const dim3 grid{unsigned((D + RT - 1) / RT), unsigned((n + CT - 1) / CT), unsigned(nset)};
    rowgemm_batched_kernel<T, RT, CT><<<grid, RT * CT / 16, 0, s>>>(In, ldi, K, U, ldu, n, Out, ldo, Ds, alpha, beta,
                                                                                 skip);
  }
  note_launch();
  TRBL_CUDA(cudaGetLastError());
  return TRBL_OK;
}

template int block_dot_batched<float>(const float* const*, int64_t, int, const float* const*, int64_t, int,
                                      const int64_t*, int64_t, double* const*, double* const*, size_t, int,
                                      cudaStream_t, const int*);
template int block_dot_batched<double>(const double* const*, int64_t, int, const double* const*, int64_t, int,
                                       const int64_t*, int64_t, double* const*, double* const*, size_t, int,
                                       cudaStream_t, const int*);
template int rowgemm_batched<float>(const float* const*, int64_t, int, const double* const*, int64_t, int,
                                    float* const*, int64_t, const int64_t*, int64_t, double, double, int,
                                    cudaStream_t, const int*);
template int rowgemm_batched<double>(const double* const*, int64_t, int, const double* const*, int64_t, int,
                                     double* const*, int64_t, const int64_t*, int64_t, double, double, int,
                                     cudaStream_t, const int*);

template <typename T>
int block_dot_capped(const T* B, int64_t ldb, int m, const T* W, int64_t ldw, int q, int64_t D, double* C,
                     double* partial, size_t partial_bytes, int sm_count, cudaStream_t s) {
  if (m <= 0 || D <= 0) return fail(TRBL_ERR_ARG, "block_dot: empty operand");
  if (q <= 4) return dot_launch_capped<T, 4>(B, ldb, m, W, ldw, q, D, C, partial, partial_bytes, sm_count, s);
  if (q <= 8) return dot_launch_capped<T, 8>(B, ldb, m, W, ldw, q, D, C, partial, partial_bytes, sm_count, s);
  if (q <= 16) return dot_launch_capped<T, 16>(B, ldb, m, W, ldw, q, D, C, partial, partial_bytes, sm_count, s);
  if (q <= 32) return dot_launch_capped<T, 32>(B, ldb, m, W, ldw, q, D, C, partial, partial_bytes, sm_count, s);
  if (q <= 64) return dot_launch_capped<T, 64>(B, ldb, m, W, ldw, q, D, C, partial, partial_bytes, sm_count, s);
  return fail(TRBL_ERR_ARG, "block_dot: q=%d > 64", q);
}

int block_dot_capped_load_kernels() {
  // cudaFuncGetAttributes loads a kernel that lazy module loading has not
  // loaded yet, so no later block_dot_capped call loads (and allocates) one.
  cudaFuncAttributes a;
  const void* fns[] = {
      reinterpret_cast<const void*>(block_dot_kernel<float, 4>),   reinterpret_cast<const void*>(block_dot_kernel<float, 8>),
      reinterpret_cast<const void*>(block_dot_kernel<float, 16>),  reinterpret_cast<const void*>(block_dot_kernel<float, 32>),
      reinterpret_cast<const void*>(block_dot_kernel<float, 64>),  reinterpret_cast<const void*>(block_dot_kernel<double, 4>),
      reinterpret_cast<const void*>(block_dot_kernel<double, 8>),  reinterpret_cast<const void*>(block_dot_kernel<double, 16>),
      reinterpret_cast<const void*>(block_dot_kernel<double, 32>), reinterpret_cast<const void*>(block_dot_kernel<double, 64>),
      reinterpret_cast<const void*>(reduce_partials_kernel)};
  for (const void* f : fns) TRBL_CUDA(cudaFuncGetAttributes(&a, f));
  return TRBL_OK;
}

template int block_dot_capped<float>(const float*, int64_t, int, const float*, int64_t, int, int64_t, double*,
                                     double*, size_t, int, cudaStream_t);
template int block_dot_capped<double>(const double*, int64_t, int, const double*, int64_t, int, int64_t, double*,
                                      double*, size_t, int, cudaStream_t);

size_t block_dot_workspace_bytes(int m, int q, int sm_count) {
  const int mtiles = (m + MT - 1) / MT;
  const int64_t nchunk = (4 * sm_count + mtiles - 1) / mtiles + 1;
  return size_t(nchunk) * m * q * sizeof(double);
}

template <typename T>
int block_dot(const T* B, int64_t ldb, int m, const T* W, int64_t ldw, int q, int64_t D, double* C,
              Workspace& ws, cudaStream_t s) {
  if (m <= 0) return TRBL_OK;
  if constexpr (std::is_same<T, float>::value) {
    if (ws.tensor) {
      const int rc = block_dot_tc(B, ldb, m, W, ldw, q, D, C, ws.partial, ws.partial_bytes, ws.sm_count, s);
      if (rc != -1) return rc;
    }
    const int rc = block_dot_tma(B, ldb, m, W, ldw, q, D, C, ws.partial, ws.partial_bytes, ws.sm_count, s);
    if (rc != -1) return rc;
  }
  if (std::is_same<T, double>::value && q <= 4) return dot_narrow<T>(B, ldb, m, W, ldw, q, D, C, ws, s);
  if (q <= 4) return dot_launch<T, 4>(B, ldb, m, W, ldw, q, D, C, ws, s);
  if (q <= 8) return dot_launch<T, 8>(B, ldb, m, W, ldw, q, D, C, ws, s);
  if (q <= 16) return dot_launch<T, 16>(B, ldb, m, W, ldw, q, D, C, ws, s);
  if (q <= 32) return dot_launch<T, 32>(B, ldb, m, W, ldw, q, D, C, ws, s);
  if (q <= 64) return dot_launch<T, 64>(B, ldb, m, W, ldw, q, D, C, ws, s);
  return fail(TRBL_ERR_ARG, "block_dot: q=%d > 64", q);
}

template <typename T, int NP>
int tall_launch(const T* In, int64_t ldi, int K, const double* U, int64_t ldu, int n, T* Out, int64_t ldo,
                int64_t D, double alpha, double beta, cudaStream_t s, size_t smem, int sms) {
  static const cudaError_t cfg = cudaFuncSetAttribute(rowgemm_tall_kernel<T, NP>,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  TRBL_CUDA(cfg);
  constexpr int RT = 4 * (512 / (NP / 4));
  const int64_t ntiles = (D + RT - 1) / RT;
  const int grid = int(std::min<int64_t>(ntiles, sms));
  rowgemm_tall_kernel<T, NP><<<grid, 512, smem, s>>>(In, ldi, K, U, ldu, n, Out, ldo, D, alpha, beta); note_launch();
  TRBL_CUDA(cudaGetLastError());
  return TRBL_OK;
}

template <typename T>
int rowgemm(const T* In, int64_t ldi, int K, const double* U, int64_t ldu, int n, T* Out,
            int64_t ldo, int64_t D, double alpha, double beta, cudaStream_t s) {
  if (n <= 0 || D <= 0) return TRBL_OK;
  if (K <= 0) {
    // Out = beta * Out
    if (beta == 1.0) return TRBL_OK;
  }
  if constexpr (std::is_same<T, float>::value) {
    if (K > 0 && n <= 32) {
      const int rc = rowgemm_tma(In, ldi, K, U, ldu, n, Out, ldo, D, alpha, beta, s);
      if (rc != -1) return rc;
    }
  }
  if (std::is_same<T, double>::value && K > 0 && n <= 4 && size_t(K) * 4 * sizeof(T) <= 200 * 1024) {
    if (n == 1) return narrow_launch<T, 1>(In, ldi, K, U, ldu, n, Out, ldo, D, alpha, beta, s);
    if (n == 2) return narrow_launch<T, 2>(In, ldi, K, U, ldu, n, Out, ldo, D, alpha, beta, s);
    return narrow_launch<T, 4>(In, ldi, K, U, ldu, n, Out, ldo, D, alpha, beta, s);
  }
  if (K > 0 && n <= 64) {
    const int NP = n <= 16 ? 16 : (n <= 32 ? 32 : 64);
    const int RT = 4 * (512 / (NP / 4));
    const int Kp = (K + 31) / 32 * 32;
    const size_t smem = (size_t(Kp) * NP + size_t(2) * 32 * (RT + 4)) * sizeof(T);
    if (smem <= 200 * 1024) {
      static const int sms = [] {
        int dev = 0, n = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        return n > 0 ? n : 148;
      }();
      if (NP == 16) return tall_launch<T, 16>(In, ldi, K, U, ldu, n, Out, ldo, D, alpha, beta, s, smem, sms);
      if (NP == 32) return tall_launch<T, 32>(In, ldi, K, U, ldu, n, Out, ldo, D, alpha, beta, s, smem, sms);
      return tall_launch<T, 64>(In, ldi, K, U, ldu, n, Out, ldo, D, alpha, beta, s, smem, sms);
    }
  }
  if (n <= 16) {
    constexpr int RT = 128, CT = 16;
    dim3 grid(unsigned((D + RT - 1) / RT), unsigned((n + CT - 1) / CT));
    rowgemm_kernel<T, RT, CT><<<grid, RT * CT / 16, 0, s>>>(In, ldi, K, U, ldu, n, Out, ldo, D, alpha, beta); note_launch();
  } else if (n <= 32) {
    constexpr int RT = 128, CT = 32;
    dim3 grid(unsigned((D + RT - 1) / RT), unsigned((n + CT - 1) / CT));
    rowgemm_kernel<T, RT, CT><<<grid, RT * CT / 16, 0, s>>>(In, ldi, K, U, ldu, n, Out, ldo, D, alpha, beta); note_launch();
  } else {
    constexpr int RT = 64, CT = 64;
    dim3 grid(unsigned((D + RT - 1) / RT), unsigned((n + CT - 1) / CT));
    rowgemm_kernel<T, RT, CT><<<grid, RT * CT / 16, 0, s>>>(In, ldi, K, U, ldu, n, Out, ldo, D, alpha, beta); note_launch();
  }
  TRBL_CUDA(cudaGetLastError());
  return TRBL_OK;
}

template <typename T>
int rowgemm_ws(const T* In, int64_t ldi, int K, const double* U, int64_t ldu, int n, T* Out, int64_t ldo, int64_t D,
               double alpha, double beta, Workspace& ws, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (ws.tensor && n > 0 && D > 0 && K > 0 && K >= ws.tc_min_k) {
      const int rc = rowgemm_tc(In, ldi, K, U, ldu, n, Out, ldo, D, alpha, beta, ws.ut, ws.ut_bytes, s);
      if (rc != -1) return rc;
    }
  }
  return rowgemm<T>(In, ldi, K, U, ldu, n, Out, ldo, D, alpha, beta, s);
}

// Squared column norms of a D x q block (row-major, ld ldw): one block per
// row range, thread t on column t mod q; FP32 data is squared and summed in
// FP32 over runs of 32 rows, the runs in FP64; the block's columns are
// reduced in a fixed order into partial[block][c].
template <typename T>
__global__ void col_sumsq_kernel(const T* __restrict__ W, int64_t ldw, int q, int64_t D, int64_t rows_per_block,
                                 double* __restrict__ partial) {
  __shared__ double red[256];
  const int t = threadIdx.x;
  const int per = blockDim.x / q;  // rows per sweep
  const int c = t % q, rl = t / q;
  double acc = 0.0;
  if (rl < per) {
    const int64_t r0 = int64_t(blockIdx.x) * rows_per_block;
    const int64_t r1 = r0 + rows_per_block < D ? r0 + rows_per_block : D;
    if constexpr (std::is_same<T, float>::value) {
      float run = 0.f;
      int cnt = 0;
      for (int64_t r = r0 + rl; r < r1; r += per) {
        const float x = W[r * ldw + c];
        run = fmaf(x, x, run);
        if (++cnt == 32) {
          acc += double(run);
          run = 0.f;
          cnt = 0;
        }
      }
      acc += double(run);
    } else {
      for (int64_t r = r0 + rl; r < r1; r += per) {
        const double x = W[r * ldw + c];
        acc = fma(x, x, acc);
      }
    }
  }
  red[t] = acc;
  __syncthreads();
  if (t < q) {
    double v = 0.0;
    for (int k = 0; k < per; ++k) v += red[k * q + t];
    partial[int64_t(blockIdx.x) * q + t] = v;
  }
}

// The same for a contiguous FP32 block (ldw = q, q a multiple of 4 dividing
// 128, 16-byte aligned) read as float4s: float4 i of the block covers
// columns 4 i mod q .. + 3, so thread t of a block whose range starts on a
// row boundary keeps columns 4 t mod q .. + 3 while striding by 256
// float4s.  Four loads in flight per thread; FP32 runs of 32 float4s, FP64
// beyond; threads with the same columns are summed in a fixed order.
__global__ void __launch_bounds__(256) col_sumsq_vec_kernel(const float* __restrict__ W, int q, int64_t D,
                                                            int64_t rows_per_block, double* __restrict__ partial) {
  __shared__ double red[256][4];
  const int t = threadIdx.x;
  const int64_t r0 = int64_t(blockIdx.x) * rows_per_block;
  const int64_t r1 = r0 + rows_per_block < D ? r0 + rows_per_block : D;
  const float4* p = reinterpret_cast<const float4*>(W) + r0 * (q / 4);
  const int64_t n4 = r1 > r0 ? (r1 - r0) * (q / 4) : 0;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  float run[4] = {0.f, 0.f, 0.f, 0.f};
  int cnt = 0;
  int64_t i = t;
  for (; i + 3 * 256 < n4; i += 4 * 256) {
    float4 x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) x[u] = __ldg(p + i + 256 * u);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      run[0] = fmaf(x[u].x, x[u].x, run[0]);
      run[1] = fmaf(x[u].y, x[u].y, run[1]);
      run[2] = fmaf(x[u].z, x[u].z, run[2]);
      run[3] = fmaf(x[u].w, x[u].w, run[3]);
    }
    if (++cnt == 8) {
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[k] += double(run[k]), run[k] = 0.f;
      cnt = 0;
    }
  }
  for (; i < n4; i += 256) {
    const float4 x = __ldg(p + i);
    run[0] = fmaf(x.x, x.x, run[0]);
    run[1] = fmaf(x.y, x.y, run[1]);
    run[2] = fmaf(x.z, x.z, run[2]);
    run[3] = fmaf(x.w, x.w, run[3]);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) red[t][k] = acc[k] + double(run[k]);
  __syncthreads();
  if (t < q) {
    const int q4 = q / 4;
    double v = 0.0;
    for (int j = t / 4; j < 256; j += q4) v += red[j][t % 4];
    partial[int64_t(blockIdx.x) * q + t] = v;
  }
}

// Gram matrix G = W^T W of a D x Q block of FP32 data (Q = 8, 16, 32 or
// 64), FP64 result.  A block stages 16 KB of rows (4096 / Q) at a time in
// shared memory, the next chunk's loads in flight (in registers) while the
// current one is used; (Q/4)^2 threads each own a 4 x 4 tile of G and
// 256 / (Q/4)^2 row groups split the staged rows; products are summed in
// FP32 over runs of at most 32 rows of a thread, the runs into a two-word
// FP32 sum by TwoSum (error-free; GB300's FP64 adds are too slow to take
// every run) and that sum into FP64 at the end.  The
// row groups' sums are reduced in a fixed order into partial[block] (the
// staging buffer's shared memory reused), the blocks' by
// reduce_partials_kernel: the result does not depend on timing.
template <int Q>
__global__ void __launch_bounds__(256, 2) gram_f32_kernel(const float* __restrict__ W, int64_t ldw, int64_t D,
                                                          int64_t rows_per_block, double* __restrict__ partial) {
  constexpr int kRows = 4096 / Q;
  constexpr int TQ = Q / 4;                 // tiles per side
  constexpr int kGroups = 256 / (TQ * TQ);  // row groups
  constexpr int kBytes = kRows * Q * 4 > Q * Q * 8 ? kRows * Q * 4 : Q * Q * 8;
  __shared__ __align__(16) unsigned char sm[kBytes];
  float* xs = reinterpret_cast<float*>(sm);
  double* red = reinterpret_cast<double*>(sm);
  const int t = threadIdx.x;
  const int tile = t % (TQ * TQ), grp = t / (TQ * TQ);
  const int ti = tile / TQ, tj = tile % TQ;
  const int64_t r0 = int64_t(blockIdx.x) * rows_per_block;
  const int64_t r1 = r0 + rows_per_block < D ? r0 + rows_per_block : D;
  const bool vec = (ldw % 4) == 0 && (reinterpret_cast<uintptr_t>(W) & 15) == 0;
  float hi[4][4], lo[4][4], run[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) hi[a][b] = lo[a][b] = run[a][b] = 0.f;
  // hi + lo += run exactly (Knuth's TwoSum; round-to-nearest adds the
  // compiler may not contract or reorder), then run = 0
  auto flush = [&]() {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const float x = run[a][b], h = hi[a][b];
        const float sum = __fadd_rn(h, x);
        const float xb = __fsub_rn(sum, h);
        const float hb = __fsub_rn(sum, xb);
        lo[a][b] = __fadd_rn(lo[a][b], __fadd_rn(__fsub_rn(h, hb), __fsub_rn(x, xb)));
        hi[a][b] = sum;
        run[a][b] = 0.f;
      }
  };
  // chunk loads: float4 e = t + 256 u (u < 4) is row e / (Q/4), columns 4 (e mod Q/4) ..
  float4 pre[4];
  auto load = [&](int64_t c0) {
    const int nr = int(r1 - c0 < kRows ? r1 - c0 : kRows);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = t + 256 * u, rr = e / (Q / 4), cc = e % (Q / 4);
      pre[u] = rr < nr ? __ldg(reinterpret_cast<const float4*>(W + (c0 + rr) * ldw + 4 * cc))
                       : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  if (vec && r0 < r1) load(r0);
  int cnt = 0;
  for (int64_t c0 = r0; c0 < r1; c0 += kRows) {
    const int nr = int(r1 - c0 < kRows ? r1 - c0 : kRows);
    __syncthreads();
    if (vec) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = t + 256 * u;
        *reinterpret_cast<float4*>(xs + 4 * e) = pre[u];
      }
    } else {
      for (int e = t; e < kRows * Q; e += 256) {
        const int rr = e / Q, cc = e % Q;
        xs[e] = rr < nr ? W[(c0 + rr) * ldw + cc] : 0.f;
      }
    }
    __syncthreads();
    if (vec && c0 + kRows < r1) load(c0 + kRows);
    for (int rr = grp; rr < nr; rr += kGroups) {
      const float4 x = *reinterpret_cast<const float4*>(xs + rr * Q + 4 * ti);
      const float4 y = *reinterpret_cast<const float4*>(xs + rr * Q + 4 * tj);
      const float xa[4] = {x.x, x.y, x.z, x.w}, ya[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) run[a][b] = fmaf(xa[a], ya[b], run[a][b]);
      if (++cnt == 32) {
        flush();
        cnt = 0;
      }
    }
  }
  flush();
  // row groups in order 0, 1, ... into red (the first barrier also ends
  // every thread's reads of the staged rows)
  for (int g = 0; g < kGroups; ++g) {
    __syncthreads();
    if (grp == g) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const double v = double(hi[a][b]) + double(lo[a][b]);
          double& d = red[(4 * ti + a) * Q + 4 * tj + b];
          d = g == 0 ? v : d + v;
        }
    }
  }
  __syncthreads();
  for (int e = t; e < Q * Q; e += 256) partial[int64_t(blockIdx.x) * Q * Q + e] = red[e];
}

template <int Q>
int gram_f32_launch(const float* W, int64_t ldw, int64_t D, double* G, Workspace& ws, cudaStream_t s) {
  int64_t nblk = std::min<int64_t>(int64_t(4) * ws.sm_count, (D + 4096 / Q - 1) / (4096 / Q));
  nblk = std::max<int64_t>(1, std::min<int64_t>(nblk, int64_t(ws.partial_bytes / (sizeof(double) * Q * Q))));
  const int64_t rows = (D + nblk - 1) / nblk;
  nblk = (D + rows - 1) / rows;
  gram_f32_kernel<Q><<<unsigned(nblk), 256, 0, s>>>(W, ldw, D, rows, ws.partial); note_launch();
  TRBL_CUDA(cudaGetLastError());
  reduce_partials_kernel<<<(Q * Q + 255) / 256, 256, 0, s>>>(ws.partial, int(nblk), Q * Q, G); note_launch();
  TRBL_CUDA(cudaGetLastError());
  return TRBL_OK;
}

// col_sumsq_kernel over several problems: grid y = problem; a block whose
// row range lies past its problem's rows writes zeros.
template <typename T>
__global__ void col_sumsq_batched_kernel(const T* const* __restrict__ Ws, int64_t ldw, int q,
                                         const int64_t* __restrict__ Ds, int64_t rows_per_block,
                                         double* const* __restrict__ partials) {
  __shared__ double red[256];
  const T* __restrict__ W = Ws[blockIdx.y];
  const int64_t D = Ds[blockIdx.y];
  const int t = threadIdx.x;
  const int per = blockDim.x / q;
  const int c = t % q, rl = t / q;
  double acc = 0.0;
  if (rl < per) {
    const int64_t r0 = int64_t(blockIdx.x) * rows_per_block;
    const int64_t r1 = r0 + rows_per_block < D ? r0 + rows_per_block : D;
    for (int64_t r = r0 + rl; r < r1; r += per) {
      const double x = double(W[r * ldw + c]);
      acc = fma(x, x, acc);
    }
  }
  red[t] = acc;
  __syncthreads();
  if (t < q) {
    double v = 0.0;
    for (int k = 0; k < per; ++k) v += red[k * q + t];
    partials[blockIdx.y][int64_t(blockIdx.x) * q + t] = v;
  }
}

template <typename T>
int col_sumsq_batched(const T* const* W, int64_t ldw, int q, const int64_t* Ds, int64_t D, double* const* out,
                      double* const* partial, size_t partial_bytes, int sm_count, int nset, cudaStream_t s) {
  if (q <= 0 || q > 256 || D <= 0 || nset <= 0) return fail(TRBL_ERR_ARG, "col_sumsq_batched: q=%d", q);
  int64_t nblk = std::min<int64_t>(std::max(1, (4 * sm_count + nset - 1) / nset), (D + 255) / 256);
  nblk = std::max<int64_t>(1, std::min<int64_t>(nblk, int64_t(partial_bytes / (sizeof(double) * q))));
  const int64_t rows = (D + nblk - 1) / nblk;
  nblk = (D + rows - 1) / rows;
  const dim3 grid{unsigned(nblk), unsigned(nset), 1u};
  col_sumsq_batched_kernel<T><<<grid, 256, 0, s>>>(W, ldw, q, Ds, rows, partial); note_launch();
  TRBL_CUDA(cudaGetLastError());
  const dim3 rgrid{unsigned((q + 255) / 256), unsigned(nset), 1u};
  reduce_partials_batched_kernel<<<rgrid, 256, 0, s>>>(partial, int(nblk), q, out, nullptr); note_launch();
  TRBL_CUDA(cudaGetLastError());
  return TRBL_OK;
}

template <typename T>
int col_sumsq(const T* W, int64_t ldw, int q, int64_t D, double* out, Workspace& ws, cudaStream_t s) {
  if (q <= 0 || q > 256 || D <= 0) return fail(TRBL_ERR_ARG, "col_sumsq: q=%d D=%lld", q, (long long)D);
  int64_t nblk = std::min<int64_t>(int64_t(4) * ws.sm_count, (D + 255) / 256);
  nblk = std::max<int64_t>(1, std::min<int64_t>(nblk, int64_t(ws.partial_bytes / (sizeof(double) * q))));
  const int64_t rows = (D + nblk - 1) / nblk;
  nblk = (D + rows - 1) / rows;
  bool vec = false;
  if constexpr (std::is_same<T, float>::value)
    vec = ldw == q && q % 4 == 0 && 128 % q == 0 && (reinterpret_cast<uintptr_t>(W) & 15) == 0;
  if (vec)
    col_sumsq_vec_kernel<<<unsigned(nblk), 256, 0, s>>>(reinterpret_cast<const float*>(W), q, D, rows, ws.partial);
  else
    col_sumsq_kernel<T><<<unsigned(nblk), 256, 0, s>>>(W, ldw, q, D, rows, ws.partial);
  note_launch();
  TRBL_CUDA(cudaGetLastError());
  reduce_partials_kernel<<<(q + 255) / 256, 256, 0, s>>>(ws.partial, int(nblk), q, out); note_launch();
  TRBL_CUDA(cudaGetLastError());
  return TRBL_OK;
}

template <typename T>
int gram(const T* W, int64_t ldw, int q, int64_t D, double* G, Workspace& ws, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (D > 0 && ldw >= q) {
      if (q == 8) return gram_f32_launch<8>(W, ldw, D, G, ws, s);
      if (q == 16) return gram_f32_launch<16>(W, ldw, D, G, ws, s);
      if (q == 32) return gram_f32_launch<32>(W, ldw, D, G, ws, s);
      if (q == 64) return gram_f32_launch<64>(W, ldw, D, G, ws, s);
    }
  }
  return block_dot<T>(W, ldw, q, W, ldw, q, D, G, ws, s);
}

template <typename S, typename T>
int copy_cols(const S* src, int64_t lds, T* dst, int64_t ldd, int64_t D, int ncol, cudaStream_t s) {
  if (ncol <= 0 || D <= 0) return TRBL_OK;
  const int64_t n = D * ncol;
  copy_cols_kernel<S, T><<<unsigned((n + 255) / 256), 256, 0, s>>>(src, lds, dst, ldd, D, ncol); note_launch();
  TRBL_CUDA(cudaGetLastError());
  return TRBL_OK;
}

template <typename T>
int scale_col(T* X, int64_t ldx, int64_t D, double a, cudaStream_t s) {
  scale_col_kernel<T><<<unsigned((D + 255) / 256), 256, 0, s>>>(X, ldx, D, a); note_launch();
  TRBL_CUDA(cudaGetLastError());
  return TRBL_OK;
}

template <typename T>
int random_block(T* X, int64_t ldx, int64_t D, int ncol, int ncol_total, int col0, uint64_t seed,
                 cudaStream_t s) {
  const int64_t n = D * ncol;
  random_block_kernel<T><<<unsigned((n + 255) / 256), 256, 0, s>>>(X, ldx, D, ncol, ncol_total, col0, seed); note_launch();
  TRBL_CUDA(cudaGetLastError());
  return TRBL_OK;
}

template int block_dot<float>(const float*, int64_t, int, const float*, int64_t, int, int64_t, double*, Workspace&, cudaStream_t);
template int block_dot<double>(const double*, int64_t, int, const double*, int64_t, int, int64_t, double*, Workspace&, cudaStream_t);
template int rowgemm<float>(const float*, int64_t, int, const double*, int64_t, int, float*, int64_t, int64_t, double, double, cudaStream_t);
template int rowgemm<double>(const double*, int64_t, int, const double*, int64_t, int, double*, int64_t, int64_t, double, double, cudaStream_t);
template int rowgemm_ws<float>(const float*, int64_t, int, const double*, int64_t, int, float*, int64_t, int64_t, double, double, Workspace&, cudaStream_t);
template int col_sumsq<float>(const float*, int64_t, int, int64_t, double*, Workspace&, cudaStream_t);
template int gram<float>(const float*, int64_t, int, int64_t, double*, Workspace&, cudaStream_t);
template int col_sumsq_batched<float>(const float* const*, int64_t, int, const int64_t*, int64_t, double* const*,
                                      double* const*, size_t, int, int, cudaStream_t);
template int col_sumsq_batched<double>(const double* const*, int64_t, int, const int64_t*, int64_t, double* const*,
                                       double* const*, size_t, int, int, cudaStream_t);
template int gram<double>(const double*, int64_t, int, int64_t, double*, Workspace&, cudaStream_t);
template int col_sumsq<double>(const double*, int64_t, int, int64_t, double*, Workspace&, cudaStream_t);
template int rowgemm_ws<double>(const double*, int64_t, int, const double*, int64_t, int, double*, int64_t, int64_t, double, double, Workspace&, cudaStream_t);
template int copy_cols<float, float>(const float*, int64_t, float*, int64_t, int64_t, int, cudaStream_t);
template int copy_cols<double, double>(const double*, int64_t, double*, int64_t, int64_t, int, cudaStream_t);
template int copy_cols<float, double>(const float*, int64_t, double*, int64_t, int64_t, int, cudaStream_t);
template int copy_cols<double, float>(const double*, int64_t, float*, int64_t, int64_t, int, cudaStream_t);
template int random_block<float>(float*, int64_t, int64_t, int, int, int, uint64_t, cudaStream_t);
template int scale_col<float>(float*, int64_t, int64_t, double, cudaStream_t);
template int scale_col<double>(double*, int64_t, int64_t, double, cudaStream_t);
template int random_block<double>(double*, int64_t, int64_t, int, int, int, uint64_t, cudaStream_t);

}  // namespace trbl
