// FP32 block product W = H V for rows of 32, 64 or 128 bytes (q = 8, 16,
// 32): the default product of the mixed-precision solver.
//
// Same arithmetic and work decomposition as the grouped kernel
// (apply_grouped.cu): like-particle rows of App. B.1 and the factorised
// proton-neutron term of App. B.2, Eq. (pntwobodybit); one thread block per
// (target proton determinant pA', chunk of neutron rows); a warp per output
// row; groups of LPE lanes, each lane one 16-byte chunk, so a group reads a
// whole V row per generated element.  What differs is the instruction count
// per generated element, which bounded the grouped kernel (about 6.8 warp
// instructions per element, most of them integer address and index work):
//
// * element offsets are 32-bit (the caller's D * ld < 2^31 is checked on the
//   host), so a source address is one wide multiply-add on a per-row base;
// * the like-particle sources come as packed (offset, coefficient) pairs, one
//   8-byte load per element: species A's are staged in shared memory per
//   target, species B's are a table of (source row, coefficient) pairs;
// * the cross term's coefficient row is walked with a pointer increment and
//   its source offsets are 32-bit shared-memory words;
// * the q / 4 products of an element run as paired FP32 FMAs (fma.rn.f32x2),
//   two lanes' worth of columns per instruction;
// * the per-target staging runs on all warps: warp 0 forms the 2m-transfer
//   ranges of the staged proton jumps with a warp scan, the other warps
//   stage the like-particle sources meanwhile.
//
// Summation: by default every product of a row goes into one FP32 sum per
// column, in the grouped kernel's order (the two kernels agree bit for
// bit).  With compensated sums (trbl_apply_set_compensated) a lane adds the
// products of one cross-term task, or of at most 8 like-particle sources,
// into a short FP32 partial sum, and the partial sums into a two-word
// (hi + lo) row sum by Knuth's TwoSum: the rounding error of a row no longer
// grows with its ~900 terms, so the FP32 product's error drops toward the
// rounding of its inputs (the FP32 vector and coefficients).
//
// Partial sums of the lane groups are combined with warp shuffles and one
// group stores the row: no atomics, a fixed summation order.
#include <algorithm>

#include "internal.h"

namespace trbl {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxSmem = 227 * 1024;

typedef unsigned long long u64;

__device__ __forceinline__ u64 pack2(float a, float b) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void unpack2(u64 v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
// 16 bytes of V through the read-only path as two 64-bit halves.
__device__ __forceinline__ void ldg16(const float* p, u64& lo, u64& hi) {
  asm volatile("ld.global.nc.v2.b64 {%0, %1}, [%2];" : "=l"(lo), "=l"(hi) : "l"(p));
}
// acc (two FP32 lanes) += c * x, both lanes in one instruction.
__device__ __forceinline__ void fma2(u64& acc, u64 cc, u64 x) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(cc), "l"(x));
}
__device__ __forceinline__ void axpy4(u64 (&acc)[2], float c, u64 x0, u64 x1) {
  const u64 cc = pack2(c, c);
  fma2(acc[0], cc, x0);
  fma2(acc[1], cc, x1);
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
  u64 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b) {
  u64 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
// Row accumulator of a lane's four columns: with COMP the running sum is
// kept as hi + lo, each partial sum t entering by Knuth's TwoSum (exact:
// hi + lo + t = hi' + lo' up to the rounding of lo), so the rounding of a
// long sum no longer grows with its length; without COMP a plain sum.
template <bool COMP>
struct RowAcc {
  u64 hi[2] = {0ull, 0ull};
  u64 lo[2] = {0ull, 0ull};
  __device__ __forceinline__ void add(const u64 (&t)[2]) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      if (COMP) {
        const u64 sum = add2(hi[i], t[i]);
        const u64 tb = sub2(sum, hi[i]);
        const u64 hb = sub2(sum, tb);
        lo[i] = add2(lo[i], add2(sub2(hi[i], hb), sub2(t[i], tb)));
        hi[i] = sum;
      } else {
        hi[i] = add2(hi[i], t[i]);
      }
    }
  }
  __device__ __forceinline__ void result(float (&r)[4]) const {
    u64 s0 = hi[0], s1 = hi[1];
    if (COMP) {
      s0 = add2(s0, lo[0]);
      s1 = add2(s1, lo[1]);
    }
    unpack2(s0, r[0], r[1]);
    unpack2(s1, r[2], r[3]);
  }
};

template <int LPE, bool COMP>
__device__ __forceinline__ void fast_body(const DevH<float>& h, const DevG<float>& g, int item_index,
                                          const float* __restrict__ V, int ld, float* __restrict__ W, int64_t ldw) {
  constexpr int G = 32 / LPE;  // element groups per warp
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ND = h.ND;
  const int maxP = g.maxP, maxQ = g.maxQ, maxK = g.maxK;
  int2* pp = reinterpret_cast<int2*>(smem_raw);            // [maxQ] (offset of (pA, nB = 0), coefficient bits)
  int* pj = reinterpret_cast<int*>(pp + maxQ);             // [maxP + 1] offset of (source pA, nB = 0)
  float* scoef = reinterpret_cast<float*>(pj + maxP + 1);  // [(maxP + 1) * maxK], proton sign folded in
  int* pstart = reinterpret_cast<int*>(scoef + size_t(maxP + 1) * maxK);  // [32] staged jumps by transfer
  int* nq = pstart + 32;                                                  // [1]

  const int4 item = g.work[item_index];
  const int pA = item.x, blk = item.y, r0 = item.z, nrows = item.w;
  const int off = int(h.boff[blk]);
  const int nb = h.bnb[blk];
  const int iA = pA - h.bgA[blk];
  const int gB0 = h.bgB[blk];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // ---- stage the proton side of pA' ----
  if (warp == 0) {
    int c = 0;
    if (lane < ND && h.srcblk[blk * ND + lane] >= 0)
      c = h.jsegA[int64_t(pA) * ND + lane + 1] - h.jsegA[int64_t(pA) * ND + lane];
    int s = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += t;
    }
    pstart[lane] = s - c;  // lanes >= ND carry the total (their count is 0)
    if (lane == 0) nq[0] = h.hoffA[pA + 1] - h.hoffA[pA];
  } else {
    const int q0 = h.hoffA[pA], Q = h.hoffA[pA + 1] - q0;
    for (int i = tid - 32; i < Q; i += kThreads - 32)
      pp[i] = make_int2((off + h.hsrcA[q0 + i] * nb) * ld, __float_as_int(h.hcoefA[q0 + i]));
  }
  __syncthreads();
  // staged proton jumps: warp w fills the transfer classes w, w + 8, ...
  for (int di = warp; di < ND; di += kWarps) {
    const int ps = pstart[di], cnt = pstart[di + 1] - ps;
    if (cnt == 0) continue;
    const int sb = h.srcblk[blk * ND + di];
    const int soff = int(h.boff[sb]);
    const int snb = h.bnb[sb];
    const int e0 = h.jsegA[int64_t(pA) * ND + di];
    for (int i = lane; i < cnt; i += 32) pj[ps + i] = (soff + h.jA[e0 + i].x * snb) * ld;
    for (int i = lane; i < cnt * maxK; i += 32) {
      const int pi = i / maxK, k = i - pi * maxK;
      const int op = h.jA[e0 + pi].y;
      const float c = g.ccoef[size_t(op >> 1) * maxK + k];
      scoef[size_t(ps + pi) * maxK + k] = __int_as_float(__float_as_int(c) ^ ((op & 1) << 31));
    }
  }
  __syncthreads();

  // ---- rows ----
  const int grp = lane / LPE, sub = lane - grp * LPE;
  const float* Vl = V + sub * 4;
  const int Q = nq[0];
  const int rowA = off + iA * nb;
  const float* Vnn = Vl + rowA * ld;  // row (pA', nB = 0)
  for (int rr = warp; rr < nrows; rr += kWarps) {
    const int iB = r0 + rr;
    const int pB = gB0 + iB;
    // With COMP, partial sums of at most 8 like-particle elements (or of
    // one task of the cross term) enter a compensated row accumulator one at a
    // time; without it every product goes straight into one FP32 sum, in the
    // grouped kernel's order.
    RowAcc<COMP> racc;
    u64 acc[2] = {0ull, 0ull};
    constexpr int kStep = COMP ? 8 * G : (1 << 28);  // one pass without COMP
    // like-particle rows of species B: sources (pA', nB) in the target's own slab
    {
      const int e0 = h.hoffB[pB], e1 = h.hoffB[pB + 1];
      for (int c0 = e0 + grp; c0 < e1; c0 += kStep) {
        const int ce = COMP ? min(e1, c0 + kStep) : e1;
#pragma unroll 2
        for (int e = c0; e < ce; e += G) {
          const int2 u = g.likeB[e];
          u64 x0, x1;
          ldg16(Vnn + u.x * ld, x0, x1);
          axpy4(acc, __int_as_float(u.y), x0, x1);
        }
        if (COMP) {
          racc.add(acc);
          acc[0] = acc[1] = 0ull;
        }
      }
    }
    // like-particle rows of species A: sources (pA, nB')
    {
      const float* Vpp = Vl + iB * ld;
      for (int c0 = grp; c0 < Q; c0 += kStep) {
        const int ce = COMP ? min(Q, c0 + kStep) : Q;
#pragma unroll 2
        for (int i = c0; i < ce; i += G) {
          const int2 u = pp[i];
          u64 x0, x1;
          ldg16(Vpp + u.x, x0, x1);
          axpy4(acc, __int_as_float(u.y), x0, x1);
        }
        if (COMP) {
          racc.add(acc);
          acc[0] = acc[1] = 0ull;
        }
      }
    }
    // proton jump x neutron jump of opposite 2m transfer: one task per
    // incoming neutron jump, looping over the staged proton jumps of the
    // opposite transfer; the neutron sign flips the staged coefficient
    {
      const int e1 = h.jsegB[int64_t(pB + 1) * ND];
      for (int e = h.jsegB[int64_t(pB) * ND] + grp; e < e1; e += G) {
        const int2 jb = g.jB2[e];
        const int di = ND - 1 - ((jb.y >> 1) & 255);
        const int ps = pstart[di], pe = pstart[di + 1];
        const int neg = (jb.y & 1) << 31;
        const float* cp = scoef + size_t(ps) * maxK + (jb.y >> 9);
        const float* nsrc = Vl + jb.x * ld;
        int p = ps;
        for (; p + 1 < pe; p += 2) {
          const float c0 = __int_as_float(__float_as_int(cp[0]) ^ neg);
          const float c1 = __int_as_float(__float_as_int(cp[maxK]) ^ neg);
          cp += 2 * maxK;
          u64 a0, a1, b0, b1;
          ldg16(nsrc + pj[p], a0, a1);
          ldg16(nsrc + pj[p + 1], b0, b1);
          axpy4(acc, c0, a0, a1);
          axpy4(acc, c1, b0, b1);
        }
        if (p < pe) {
          const float c0 = __int_as_float(__float_as_int(cp[0]) ^ neg);
          u64 a0, a1;
          ldg16(nsrc + pj[p], a0, a1);
          axpy4(acc, c0, a0, a1);
        }
        if (COMP) {
          racc.add(acc);
          acc[0] = acc[1] = 0ull;
        }
      }
    }
    if (!COMP) racc.add(acc);
    float r[4];
    racc.result(r);
#pragma unroll
    for (int o = LPE; o < 32; o <<= 1)
#pragma unroll
      for (int j = 0; j < 4; ++j) r[j] += __shfl_xor_sync(0xffffffffu, r[j], o);
    if (grp == 0)
      *reinterpret_cast<float4*>(W + int64_t(rowA + iB) * ldw + sub * 4) = make_float4(r[0], r[1], r[2], r[3]);
  }
}

template <int LPE, int MINB, bool COMP>
__global__ void __launch_bounds__(kThreads, MINB)
    apply_fast_kernel(DevH<float> h, DevG<float> g, const float* __restrict__ V, int ld, float* __restrict__ W,
                      int64_t ldw) {
  fast_body<LPE, COMP>(h, g, blockIdx.x, V, ld, W, ldw);
}

// Several Hamiltonians, on one basis or on bases of different dimension:
// blockIdx.y selects the set, which reads Vs[set] and writes Ws[set]; a set
// with fewer work items than the grid leaves the rest idle.
template <int LPE, int MINB, bool COMP>
__global__ void __launch_bounds__(kThreads, MINB)
    apply_fast_batch_kernel(const DevH<float>* __restrict__ hs, const DevG<float>* __restrict__ gs,
                            const float* const* __restrict__ Vs, int ld, float* const* __restrict__ Ws, int64_t ldw) {
  if (int(blockIdx.x) >= gs[blockIdx.y].nwork) return;
  const DevH<float> h = hs[blockIdx.y];
  const DevG<float> g = gs[blockIdx.y];
  fast_body<LPE, COMP>(h, g, blockIdx.x, Vs[blockIdx.y], ld, Ws[blockIdx.y], ldw);
}

size_t fast_smem(const DevG<float>& g) {
  return size_t(g.maxQ) * 8 + size_t(g.maxP + 1) * 4 + size_t(g.maxP + 1) * g.maxK * 4 + 33 * 4;
}

template <int LPE, int MINB, bool COMP>
int launch_lpe(const DevH<float>& h, const DevG<float>& g, const float* V, int ld, float* W, int64_t ldw,
               cudaStream_t s) {
  static const cudaError_t cfg = cudaFuncSetAttribute(apply_fast_kernel<LPE, MINB, COMP>,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
  TRBL_CUDA(cfg);
  const size_t sm = fast_smem(g);
  if (sm > size_t(kMaxSmem)) return fail(TRBL_ERR_ARG, "product needs %zu bytes of shared memory", sm);
  apply_fast_kernel<LPE, MINB, COMP><<<g.nwork, kThreads, sm, s>>>(h, g, V, ld, W, ldw);
  note_launch();
  TRBL_CUDA(cudaGetLastError());
  return TRBL_OK;
}

template <int LPE, int MINB, bool COMP>
int launch_batch_lpe(const DevH<float>* hs, const DevG<float>* gs, int nset, int nwork, size_t sm,
                     const float* const* V, int ld, float* const* W, int64_t ldw, cudaStream_t s) {
  static const cudaError_t cfg = cudaFuncSetAttribute(apply_fast_batch_kernel<LPE, MINB, COMP>,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
  TRBL_CUDA(cfg);
  if (sm > size_t(kMaxSmem)) return fail(TRBL_ERR_ARG, "product needs %zu bytes of shared memory", sm);
  const dim3 grid{static_cast<unsigned>(nwork), static_cast<unsigned>(nset), 1u};
  apply_fast_batch_kernel<LPE, MINB, COMP><<<grid, kThreads, sm, s>>>(hs, gs, V, ld, W, ldw);
  note_launch();
  TRBL_CUDA(cudaGetLastError());
  return TRBL_OK;
}

// Whether the fast kernel takes this call: FP32 rows of 32, 64 or 128 bytes,
// 16-byte aligned, at most 31 transfer classes, 32-bit element offsets.
bool fast_ok(const trbl_hamiltonian* h, const void* V, int64_t ldv, const void* W, int64_t ldw, int q) {
  if (!fast_tables_ok(h, ldv, q)) return false;
  if ((reinterpret_cast<uintptr_t>(V) | reinterpret_cast<uintptr_t>(W)) & 15) return false;
  if (ldw % 4 || ldw < q) return false;
  return true;
}

template <int LPE>
int launch_q(const trbl_hamiltonian* h, const float* v, int ld, float* w, int64_t ldw, cudaStream_t s) {
  const bool b6 = h->blocks_per_sm == 6;
  if (h->apply_compensated)
    return b6 ? launch_lpe<LPE, 6, true>(h->d32, h->g32, v, ld, w, ldw, s)
              : launch_lpe<LPE, 8, true>(h->d32, h->g32, v, ld, w, ldw, s);
  return b6 ? launch_lpe<LPE, 6, false>(h->d32, h->g32, v, ld, w, ldw, s)
            : launch_lpe<LPE, 8, false>(h->d32, h->g32, v, ld, w, ldw, s);
}

template <int LPE>
int launch_batch_q(const trbl_hamiltonian* h0, const DevH<float>* hs, const DevG<float>* gs, int nset, int nwork,
                   size_t smem, const float* const* v, int ld, float* const* w, int64_t ldw, cudaStream_t s) {
  const bool b6 = h0->blocks_per_sm == 6;
  if (h0->apply_compensated)
    return b6 ? launch_batch_lpe<LPE, 6, true>(hs, gs, nset, nwork, smem, v, ld, w, ldw, s)
              : launch_batch_lpe<LPE, 8, true>(hs, gs, nset, nwork, smem, v, ld, w, ldw, s);
  return b6 ? launch_batch_lpe<LPE, 6, false>(hs, gs, nset, nwork, smem, v, ld, w, ldw, s)
            : launch_batch_lpe<LPE, 8, false>(hs, gs, nset, nwork, smem, v, ld, w, ldw, s);
}

}  // namespace

int launch_fast(const trbl_hamiltonian* h, const void* V, int64_t ldv, void* W, int64_t ldw, int q, int dtype,
                cudaStream_t s) {
  if (dtype != TRBL_F32 || h->apply_kernel != TRBL_APPLY_FAST || !fast_ok(h, V, ldv, W, ldw, q)) return -1;
  const float* v = static_cast<const float*>(V);
  float* w = static_cast<float*>(W);
  const int ld = int(ldv);
  switch (q) {
    case 8: return launch_q<2>(h, v, ld, w, ldw, s);
    case 16: return launch_q<4>(h, v, ld, w, ldw, s);
    default: return launch_q<8>(h, v, ld, w, ldw, s);
  }
}

size_t fast_smem_bytes(const trbl_hamiltonian* h) { return fast_smem(h->g32); }

bool fast_tables_ok(const trbl_hamiltonian* h, int64_t ld, int q) {
  if (!h->g32.likeB || h->g32.nwork == 0 || h->b->ND > 31) return false;
  if (q != 8 && q != 16 && q != 32) return false;
  if (ld % 4 || ld < q) return false;
  return h->b->D * ld < (int64_t(1) << 31);
}

int launch_fast_batch(const trbl_hamiltonian* h0, bool all, const void* hs_dev, const void* gs_dev, int nset,
                      int nwork, size_t smem, const void* Vs, int64_t ldv, const void* Ws, int64_t ldw, int q,
                      cudaStream_t s) {
  if (!all || h0->apply_kernel != TRBL_APPLY_FAST || !fast_tables_ok(h0, ldv, q) || ldw % 4 || ldw < q) return -1;
  const auto* hs = static_cast<const DevH<float>*>(hs_dev);
  const auto* gs = static_cast<const DevG<float>*>(gs_dev);
  const auto* v = static_cast<const float* const*>(Vs);
  auto* w = static_cast<float* const*>(const_cast<void*>(Ws));
  const int ld = int(ldv);
  switch (q) {
    case 8: return launch_batch_q<2>(h0, hs, gs, nset, nwork, smem, v, ld, w, ldw, s);
    case 16: return launch_batch_q<4>(h0, hs, gs, nset, nwork, smem, v, ld, w, ldw, s);
    default: return launch_batch_q<8>(h0, hs, gs, nset, nwork, smem, v, ld, w, ldw, s);
  }
}

}  // namespace trbl
