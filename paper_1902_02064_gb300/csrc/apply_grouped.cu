// Grouped block product W = H V: the fast path of trbl_apply_block.
//
// Same arithmetic as the row kernel in apply.cu (like-particle rows of
// App. B.1 plus the factorised proton-neutron term of App. B.2,
// Eq. (pntwobodybit)), organised for GB300:
//
// * One thread block per (target proton determinant pA', chunk of up to 128
//   neutron rows of its product block).  The proton side of every generated
//   element -- the incoming one-body jumps of pA' with their source slab
//   offsets, the interaction rows they select, and the like-particle
//   sources of pA' -- is staged once in shared memory and shared by all
//   rows of the chunk.
// * A warp owns one output row (pA', nB') at a time.  Its lanes form G
//   groups of LPE lanes, each lane moving CPL 16-byte chunks, so a group
//   reads one whole V row (q values; a 128-byte cache line at q = 32 FP32,
//   read by 8 lanes x 1 chunk, which measured 9 % faster than 4 x 2) per
//   generated element, and the G groups work on G different elements of
//   the same row.  The integer work of an element (jump entry, sign,
//   coefficient lookup, address) is done once per group, not per column.
// * The groups' partial sums are combined with warp shuffles and one group
//   stores the row: no atomics, deterministic summation order.
// * The cross-species coefficient V^AB_{ab,cd} is read from a compressed
//   table: for a proton jump (a, c) only neutron pairs (b, d) with the
//   opposite 2m transfer can contribute, so each (a, c) row keeps just that
//   class (k indexes the class), and each neutron jump stores its k and
//   its transfer class.
// * The cross-species part runs task by task: each incoming neutron jump of
//   the row is one task of a lane group, looping over the staged proton
//   jumps of the opposite transfer.
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"

namespace trbl {
namespace {

constexpr int kRowsPerItem = 128;
constexpr int kThreads = 256;
constexpr int kMaxSmem = 227 * 1024;  // dynamic shared memory limit of a block on sm_103a

// Thread blocks per SM the compiler must fit (so registers per thread): 8
// (32 registers) for FP32 rows of up to two 16-byte chunks per lane lifts
// the kernel from 6 to 8 resident blocks and was 15 % faster on the
// 18.6M-dim product (the gathers are latency-bound: more warps keep more
// rows in flight).  Wider rows and FP64 keep the compiler's choice (32
// registers would spill their accumulators).
template <typename T, int CPL>
struct MinBlocks {
  static constexpr int value = (sizeof(T) == 4 && CPL <= 2) ? 8 : 1;
};

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using V = float4;
  static constexpr int N = 4;
};
template <>
struct Vec16<double> {
  using V = double2;
  static constexpr int N = 2;
};

__device__ __forceinline__ void load16(const float* p, float (&x)[4]) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  x[0] = v.x;
  x[1] = v.y;
  x[2] = v.z;
  x[3] = v.w;
}
__device__ __forceinline__ void load16(const double* p, double (&x)[2]) {
  const double2 v = __ldg(reinterpret_cast<const double2*>(p));
  x[0] = v.x;
  x[1] = v.y;
}
__device__ __forceinline__ void store16(float* p, const float (&x)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
}
__device__ __forceinline__ void store16(double* p, const double (&x)[2]) {
  *reinterpret_cast<double2*>(p) = make_double2(x[0], x[1]);
}

__device__ __forceinline__ float flip(float c, int neg) { return __int_as_float(__float_as_int(c) ^ (neg << 31)); }
__device__ __forceinline__ double flip(double c, int neg) {
  return __longlong_as_double(__double_as_longlong(c) ^ ((long long)neg << 63));
}

template <typename T, int LPE, int CPL>
__device__ __forceinline__ void grouped_body(const DevH<T>& h, const DevG<T>& g, int item_index,
                                             const T* __restrict__ V, int64_t ldv, T* __restrict__ W, int64_t ldw,
                                             int skip_pn) {
  constexpr int VPL = Vec16<T>::N;  // values per 16-byte chunk
  constexpr int G = 32 / LPE;       // element groups per warp
  constexpr int CW = VPL * LPE;     // values covered by one chunk across the group
  constexpr int NW = kThreads / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ND = h.ND;
  const int maxP = g.maxP, maxQ = g.maxQ, maxK = g.maxK;
  int64_t* pj_off = reinterpret_cast<int64_t*>(smem_raw);   // [maxP + 1] first row of the source slab * ldv
  int64_t* pp_off = pj_off + maxP + 1;                        // [maxQ] source row (at nB = 0) * ldv
  T* scoef = reinterpret_cast<T*>(pp_off + maxQ);            // [(maxP + 1) * maxK]
  T* pp_coef = scoef + size_t(maxP + 1) * maxK;               // [maxQ]
  int* pj_op = reinterpret_cast<int*>(pp_coef + maxQ);       // [maxP + 1] negative-sign bit
  int* pstart = pj_op + maxP + 1;                             // [ND + 1]
  int* nq = pstart + ND + 1;                                  // [1] like-particle source count

  const int4 item = g.work[item_index];
  const int pA = item.x, blk = item.y, r0 = item.z, nrows = item.w;
  const int64_t off = h.boff[blk];
  const int nb = h.bnb[blk];
  const int iA = pA - h.bgA[blk];
  const int gB0 = h.bgB[blk];
  const int tid = threadIdx.x;

  // ---- stage the proton side of pA' ----
  if (tid == 0) {
    int acc = 0;
    for (int di = 0; di < ND; ++di) {
      pstart[di] = acc;
      if (h.srcblk[blk * ND + di] >= 0)
        acc += h.jsegA[int64_t(pA) * ND + di + 1] - h.jsegA[int64_t(pA) * ND + di];
    }
    pstart[ND] = acc;
    nq[0] = h.hoffA[pA + 1] - h.hoffA[pA];
  }
  __syncthreads();
  for (int di = 0; di < ND && !skip_pn; ++di) {
    const int cnt = pstart[di + 1] - pstart[di];
    if (cnt == 0) continue;
    const int sb = h.srcblk[blk * ND + di];
    const int64_t soff = h.boff[sb];
    const int snb = h.bnb[sb];
    const int e0 = h.jsegA[int64_t(pA) * ND + di];
    for (int i = tid; i < cnt; i += kThreads) {
      const int2 ja = h.jA[e0 + i];
      const int p = pstart[di] + i;
      pj_off[p] = (soff + int64_t(ja.x) * snb) * ldv;
      pj_op[p] = ja.y & 1;
    }
    for (int i = tid; i < cnt * maxK; i += kThreads) {
      const int pi = i / maxK, k = i - pi * maxK;
      const int2 ja = h.jA[e0 + pi];
      scoef[size_t(pstart[di] + pi) * maxK + k] = flip(g.ccoef[size_t(ja.y >> 1) * maxK + k], ja.y & 1);
    }
  }
  {
    const int q0 = h.hoffA[pA];
    for (int i = tid; i < nq[0]; i += kThreads) {
      pp_off[i] = (off + int64_t(h.hsrcA[q0 + i]) * nb) * ldv;
      pp_coef[i] = h.hcoefA[q0 + i];
    }
  }
  __syncthreads();

  // ---- rows ----
  const int warp = tid >> 5, lane = tid & 31;
  const int grp = lane / LPE, sub = lane - grp * LPE;
  const T* Vl = V + sub * VPL;
  const int Q = nq[0];
  const int ld = int(ldv);  // row offsets inside one 2M group fit in 32 bits (checked on the host)
  const int64_t rowA = off + int64_t(iA) * nb;
  const T* Vnn = Vl + rowA * ldv;  // row (pA', nB = 0)
  for (int rr = warp; rr < nrows; rr += NW) {
    const int iB = r0 + rr;
    const int pB = gB0 + iB;
    T acc[CPL][VPL];
    for (int cc = 0; cc < CPL; ++cc)
      for (int j = 0; j < VPL; ++j) acc[cc][j] = T(0);
    T x[CPL][VPL];
    // like-particle rows of species B: sources (pA', nB)
#pragma unroll 2
    for (int e = h.hoffB[pB] + grp, ee = h.hoffB[pB + 1]; e < ee; e += G) {
      const T c = h.hcoefB[e];
      const T* src = Vnn + h.hsrcB[e] * ld;
      for (int cc = 0; cc < CPL; ++cc) load16(src + cc * CW, x[cc]);
      for (int cc = 0; cc < CPL; ++cc)
        for (int j = 0; j < VPL; ++j) acc[cc][j] = fma(c, x[cc][j], acc[cc][j]);
    }
    // like-particle rows of species A: sources (pA, nB')
    const T* Vpp = Vl + iB * ld;
#pragma unroll 2
    for (int e = grp; e < Q; e += G) {
      const T c = pp_coef[e];
      const T* src = Vpp + pp_off[e];
      for (int cc = 0; cc < CPL; ++cc) load16(src + cc * CW, x[cc]);
      for (int cc = 0; cc < CPL; ++cc)
        for (int j = 0; j < VPL; ++j) acc[cc][j] = fma(c, x[cc][j], acc[cc][j]);
    }
    // proton jump x neutron jump with opposite 2m transfer.  Every incoming
    // neutron jump of the row is one task; a task runs over the proton jumps
    // of the opposite transfer class.  The staged coefficients carry the
    // proton sign, the neutron sign is the low bit of the jump's op.
    // Skipped when the source-stationary kernel (apply_pn.cu) adds this term.
    if (!skip_pn) {
      const int e1 = h.jsegB[int64_t(pB + 1) * ND];
      for (int e = h.jsegB[int64_t(pB) * ND] + grp; e < e1; e += G) {
        const int2 jb = g.jB2[e];
        const int di = ND - 1 - ((jb.y >> 1) & 255);
        const int ps = pstart[di], pe = pstart[di + 1];
        const int neg = jb.y & 1;
        const T* crow = scoef + (jb.y >> 9);
        const T* nsrc = Vl + jb.x * ld;
        int p = ps;
        for (; p + 1 < pe; p += 2) {
          const T c0 = flip(crow[p * maxK], neg), c1 = flip(crow[(p + 1) * maxK], neg);
          const T* s0 = nsrc + pj_off[p];
          const T* s1 = nsrc + pj_off[p + 1];
          T x0[CPL][VPL], x1[CPL][VPL];
          for (int cc = 0; cc < CPL; ++cc) load16(s0 + cc * CW, x0[cc]);
          for (int cc = 0; cc < CPL; ++cc) load16(s1 + cc * CW, x1[cc]);
          for (int cc = 0; cc < CPL; ++cc)
            for (int j = 0; j < VPL; ++j) acc[cc][j] = fma(c0, x0[cc][j], acc[cc][j]);
          for (int cc = 0; cc < CPL; ++cc)
            for (int j = 0; j < VPL; ++j) acc[cc][j] = fma(c1, x1[cc][j], acc[cc][j]);
        }
        if (p < pe) {
          const T c0 = flip(crow[p * maxK], neg);
          const T* s0 = nsrc + pj_off[p];
          for (int cc = 0; cc < CPL; ++cc) load16(s0 + cc * CW, x[cc]);
          for (int cc = 0; cc < CPL; ++cc)
            for (int j = 0; j < VPL; ++j) acc[cc][j] = fma(c0, x[cc][j], acc[cc][j]);
        }
      }
    }
    for (int o = LPE; o < 32; o <<= 1)
      for (int cc = 0; cc < CPL; ++cc)
        for (int j = 0; j < VPL; ++j) acc[cc][j] += __shfl_xor_sync(0xffffffffu, acc[cc][j], o);
    if (grp == 0) {
      T* dst = W + (rowA + iB) * ldw + sub * VPL;
      for (int cc = 0; cc < CPL; ++cc) store16(dst + cc * CW, acc[cc]);
    }
  }
}

template <typename T, int LPE, int CPL>
__global__ void __launch_bounds__(kThreads, MinBlocks<T, CPL>::value) apply_grouped_kernel(DevH<T> h, DevG<T> g, const T* __restrict__ V,
                                                                 int64_t ldv, T* __restrict__ W, int64_t ldw,
                                                                 int skip_pn) {
  grouped_body<T, LPE, CPL>(h, g, blockIdx.x, V, ldv, W, ldw, skip_pn);
}

// Several Hamiltonians, on one basis or on bases of different dimension:
// blockIdx.y selects the set, which reads Vs[set] and writes Ws[set];
// blockIdx.x runs over the largest work list and a set with fewer work
// items leaves the rest idle.
template <typename T, int LPE, int CPL>
__global__ void __launch_bounds__(kThreads, MinBlocks<T, CPL>::value)
    apply_grouped_batch_kernel(const DevH<T>* __restrict__ hs, const DevG<T>* __restrict__ gs,
                               const T* const* __restrict__ Vs, int64_t ldv, T* const* __restrict__ Ws, int64_t ldw) {
  if (int(blockIdx.x) >= gs[blockIdx.y].nwork) return;
  const DevH<T> h = hs[blockIdx.y];
  const DevG<T> g = gs[blockIdx.y];
  grouped_body<T, LPE, CPL>(h, g, blockIdx.x, Vs[blockIdx.y], ldv, Ws[blockIdx.y], ldw, 0);
}

size_t smem_bytes(int maxP, int maxQ, int maxK, int ND, size_t tsize) {
  return size_t(maxP + 1) * 8 + size_t(maxQ) * 8 + (size_t(maxP + 1) * maxK + maxQ) * tsize +
         size_t(maxP + 1) * 4 + size_t(ND + 2) * 4;
}

template <typename T, int LPE, int CPL>
int launch_lpe(const DevH<T>& h, const DevG<T>& g, const T* V, int64_t ldv, T* W, int64_t ldw, cudaStream_t s,
               int skip_pn) {
  const size_t sm = smem_bytes(g.maxP, g.maxQ, g.maxK, h.ND, sizeof(T));
  // opt in once to the largest dynamic shared memory a block may use (thread-safe initialisation)
  static const cudaError_t cfg = cudaFuncSetAttribute(apply_grouped_kernel<T, LPE, CPL>,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
  TRBL_CUDA(cfg);
  if (sm > size_t(kMaxSmem)) return fail(TRBL_ERR_ARG, "product needs %zu bytes of shared memory", sm);
  apply_grouped_kernel<T, LPE, CPL><<<g.nwork, kThreads, sm, s>>>(h, g, V, ldv, W, ldw, skip_pn); note_launch();
  TRBL_CUDA(cudaGetLastError());
  return TRBL_OK;
}

// Row of q values = 16 * 2^i bytes: groups of LPE = min(4, chunks) lanes,
// CPL 16-byte chunks per lane.
template <typename T>
int launch_typed(const trbl_hamiltonian* hm, const DevH<T>& h, const DevG<T>& g, const T* V, int64_t ldv, T* W,
                 int64_t ldw, int q, cudaStream_t s, int skip_pn = 0) {
  const int bytes = q * int(sizeof(T));
  if (bytes % 16) return -1;
  if ((reinterpret_cast<uintptr_t>(V) | reinterpret_cast<uintptr_t>(W)) & 15) return -1;
  if ((ldv * int64_t(sizeof(T))) % 16 || (ldw * int64_t(sizeof(T))) % 16) return -1;
  if (int64_t(hm->b->max_group) * ldv >= (int64_t(1) << 31)) return -1;
  // TRBL_APPLY_GROUPED_X2: half the lanes per element, two 16-byte chunks
  // each (twice the elements in flight per warp instruction, half the
  // loads per lane group)
  const bool x2 = hm->apply_kernel == TRBL_APPLY_GROUPED_X2 && !skip_pn;
  switch (bytes / 16) {
    case 1: return launch_lpe<T, 1, 1>(h, g, V, ldv, W, ldw, s, skip_pn);
    case 2: return x2 ? launch_lpe<T, 1, 2>(h, g, V, ldv, W, ldw, s, skip_pn) : launch_lpe<T, 2, 1>(h, g, V, ldv, W, ldw, s, skip_pn);
    case 4: return x2 ? launch_lpe<T, 2, 2>(h, g, V, ldv, W, ldw, s, skip_pn) : launch_lpe<T, 4, 1>(h, g, V, ldv, W, ldw, s, skip_pn);
    case 8: return x2 ? launch_lpe<T, 4, 2>(h, g, V, ldv, W, ldw, s, skip_pn) : launch_lpe<T, 8, 1>(h, g, V, ldv, W, ldw, s, skip_pn);
    case 16: return launch_lpe<T, 4, 4>(h, g, V, ldv, W, ldw, s, skip_pn);
    case 32: return launch_lpe<T, 4, 8>(h, g, V, ldv, W, ldw, s, skip_pn);
    default: return -1;
  }
}

template <typename T, int LPE, int CPL>
int launch_batch_lpe(const DevH<T>* hs, const DevG<T>* gs, int nset, int nwork, size_t sm, const T* const* V,
                     int64_t ldv, T* const* W, int64_t ldw, cudaStream_t s) {
  static const cudaError_t cfg = cudaFuncSetAttribute(apply_grouped_batch_kernel<T, LPE, CPL>,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
  TRBL_CUDA(cfg);
  if (sm > size_t(kMaxSmem)) return fail(TRBL_ERR_ARG, "product needs %zu bytes of shared memory", sm);
  const dim3 grid{static_cast<unsigned>(nwork), static_cast<unsigned>(nset), 1u};
  apply_grouped_batch_kernel<T, LPE, CPL><<<grid, kThreads, sm, s>>>(hs, gs, V, ldv, W, ldw); note_launch();
  TRBL_CUDA(cudaGetLastError());
  return TRBL_OK;
}

template <typename T>
int batch_typed(const DevH<T>* hs, const DevG<T>* gs, int nset, int nwork, size_t sm, const T* const* V, int64_t ldv,
                T* const* W, int64_t ldw, int q, cudaStream_t s) {
  switch (q * int(sizeof(T)) / 16) {
    case 1: return launch_batch_lpe<T, 1, 1>(hs, gs, nset, nwork, sm, V, ldv, W, ldw, s);
    case 2: return launch_batch_lpe<T, 2, 1>(hs, gs, nset, nwork, sm, V, ldv, W, ldw, s);
    case 4: return launch_batch_lpe<T, 4, 1>(hs, gs, nset, nwork, sm, V, ldv, W, ldw, s);
    case 8: return launch_batch_lpe<T, 8, 1>(hs, gs, nset, nwork, sm, V, ldv, W, ldw, s);
    case 16: return launch_batch_lpe<T, 4, 4>(hs, gs, nset, nwork, sm, V, ldv, W, ldw, s);
    case 32: return launch_batch_lpe<T, 4, 8>(hs, gs, nset, nwork, sm, V, ldv, W, ldw, s);
    default: return fail(TRBL_ERR_ARG, "batched product: q * element size must be 16 * 2^i bytes (<= 512)");
  }
}

}  // namespace

size_t grouped_smem_bytes(const trbl_hamiltonian* h, int dtype) {
  const auto& g = h->g32;
  return smem_bytes(g.maxP, g.maxQ, g.maxK, h->b->ND, dtype == TRBL_F64 ? 8 : 4);
}

int launch_grouped_batch(const void* hs_dev, const void* gs_dev, int nset, int nwork, size_t smem, const void* Vs,
                         int64_t ldv, const void* Ws, int64_t ldw, int q, int dtype, cudaStream_t s) {
  if (dtype == TRBL_F64)
    return batch_typed<double>(static_cast<const DevH<double>*>(hs_dev), static_cast<const DevG<double>*>(gs_dev),
                               nset, nwork, smem, static_cast<const double* const*>(Vs), ldv,
                               static_cast<double* const*>(const_cast<void*>(Ws)), ldw, q, s);
  return batch_typed<float>(static_cast<const DevH<float>*>(hs_dev), static_cast<const DevG<float>*>(gs_dev), nset,
                            nwork, smem, static_cast<const float* const*>(Vs), ldv,
                            static_cast<float* const*>(const_cast<void*>(Ws)), ldw, q, s);
}

int launch_grouped_like(const trbl_hamiltonian* h, const float* V, int64_t ldv, float* W, int64_t ldw, int q,
                        cudaStream_t s) {
  if (!h->garena || h->g32.nwork == 0) return -1;
  return launch_typed<float>(h, h->d32, h->g32, V, ldv, W, ldw, q, s, 1);
}

int launch_grouped(const trbl_hamiltonian* h, const void* V, int64_t ldv, void* W, int64_t ldw, int q, int dtype,
                   cudaStream_t s) {
  if (!h->garena || h->g32.nwork == 0) return -1;
  const int sp = launch_split(h, V, ldv, W, ldw, q, dtype, s);
  if (sp != -1) return sp;
  const int f = launch_fast(h, V, ldv, W, ldw, q, dtype, s);
  if (f != -1) return f;
  if (dtype == TRBL_F64)
    return launch_typed<double>(h, h->d64, h->g64, static_cast<const double*>(V), ldv, static_cast<double*>(W), ldw,
                                q, s);
  return launch_typed<float>(h, h->d32, h->g32, static_cast<const float*>(V), ldv, static_cast<float*>(W), ldw, q, s);
}

int upload_grouped(trbl_hamiltonian* h) {
  const trbl_basis* b = h->b;
  const Species& A = b->sp[0];
  const Species& B = b->sp[1];
  const int nA = A.n, nB = B.n, ND = b->ND, span = b->dspan;
  // 2m-transfer classes of neutron pairs (b, d): k = index of (b, d) in its class
  std::vector<int> kidx(size_t(nB) * nB, -1), ncls(ND, 0);
  for (int bb = 0; bb < nB; ++bb)
    for (int d = 0; d < nB; ++d) {
      const int dn = B.twom[bb] - B.twom[d] + span;
      if (dn < 0 || dn >= ND) continue;
      kidx[size_t(bb) * nB + d] = ncls[dn]++;
    }
  int maxK = 1;
  for (int c : ncls) maxK = std::max(maxK, c);
  if (ND > 256 || maxK >= (1 << 22)) return TRBL_OK;  // op packing limits: row kernel serves
  // compressed coefficient rows: row (a, c) uses the class of transfer m_c - m_a
  std::vector<double> cc(size_t(nA) * nA * maxK, 0.0);
  for (int a = 0; a < nA; ++a)
    for (int c = 0; c < nA; ++c) {
      const int dn = A.twom[c] - A.twom[a] + span;
      if (dn < 0 || dn >= ND) continue;
      for (int bb = 0; bb < nB; ++bb)
        for (int d = 0; d < nB; ++d) {
          if (B.twom[bb] - B.twom[d] + span != dn) continue;
          cc[(size_t(a) * nA + c) * maxK + kidx[size_t(bb) * nB + d]] =
              h->vab[(size_t(a) * nA + c) * nB * nB + size_t(bb) * nB + d];
        }
    }
  std::vector<float> cc32(cc.begin(), cc.end());
  // neutron jumps with compressed ops
  std::vector<int2> jB2(B.jsrc.size());
  for (size_t e = 0; e < jB2.size(); ++e) {
    const int src = B.jsrc[e];
    const int loc = src - B.gfirst[B.group[src]];
    const int k = kidx[size_t(B.ja[e]) * nB + B.jc[e]];
    const int dn = B.twom[B.ja[e]] - B.twom[B.jc[e]] + span;
    jB2[e] = make_int2(loc, (k << 9) | (dn << 1) | (B.jsign[e] < 0 ? 1 : 0));
  }
  int maxP = 1, maxQ = 1;
  const int nblk = int(b->blocks.size());
  for (int k = 0; k < nblk; ++k) {
    const Block& bl = b->blocks[k];
    const int a0 = A.gfirst[bl.gA];
    for (int ia = 0; ia < bl.na; ++ia) {
      const int pA = a0 + ia;
      int P = 0;
      for (int di = 0; di < ND; ++di)
        if (b->srcblk[size_t(k) * ND + di] >= 0) P += A.jseg[size_t(pA) * ND + di + 1] - A.jseg[size_t(pA) * ND + di];
      const int Q = h->hoff[0][pA + 1] - h->hoff[0][pA];
      maxP = std::max(maxP, P);
      maxQ = std::max(maxQ, Q);
    }
  }
  const size_t sm64 = smem_bytes(maxP, maxQ, maxK, ND, 8);
  if (sm64 > 200 * 1024) {
    // tables too large for the grouped kernel: leave it disabled (row kernel serves)
    return TRBL_OK;
  }

  // species-B like-particle rows packed as (source local index, FP32 coefficient bits)
  std::vector<int2> likeB(h->hsrc[1].size());
  for (size_t e = 0; e < likeB.size(); ++e) {
    const float c = float(h->hcoef[1][e]);
    int bits;
    std::memcpy(&bits, &c, 4);
    likeB[e] = make_int2(h->hsrc[1][e], bits);
  }
  size_t o_jB2 = 0;
  size_t o_c64 = (o_jB2 + jB2.size() * sizeof(int2) + 255) & ~size_t(255);
  size_t o_c32 = (o_c64 + cc.size() * 8 + 255) & ~size_t(255);
  size_t o_lB = (o_c32 + cc32.size() * 4 + 255) & ~size_t(255);
  size_t total = o_lB + likeB.size() * sizeof(int2) + 256;
  void* arena = nullptr;
  TRBL_CUDA(cudaMalloc(&arena, total));
  h->garena = arena;
  char* base = static_cast<char*>(arena);
  TRBL_CUDA(cudaMemcpy(base + o_jB2, jB2.data(), jB2.size() * sizeof(int2), cudaMemcpyHostToDevice));
  TRBL_CUDA(cudaMemcpy(base + o_c64, cc.data(), cc.size() * 8, cudaMemcpyHostToDevice));
  TRBL_CUDA(cudaMemcpy(base + o_c32, cc32.data(), cc32.size() * 4, cudaMemcpyHostToDevice));
  if (!likeB.empty())
    TRBL_CUDA(cudaMemcpy(base + o_lB, likeB.data(), likeB.size() * sizeof(int2), cudaMemcpyHostToDevice));
  auto fill = [&](auto& g, size_t o_c) {
    using TT = typename std::remove_const<typename std::remove_pointer<decltype(g.ccoef)>::type>::type;
    g.maxP = maxP;
    g.maxQ = maxQ;
    g.maxK = maxK;
    g.jB2 = reinterpret_cast<const int2*>(base + o_jB2);
    g.ccoef = reinterpret_cast<const TT*>(base + o_c);
  };
  fill(h->g64, o_c64);
  fill(h->g32, o_c32);
  h->g64.likeB = nullptr;
  h->g32.likeB = reinterpret_cast<const int2*>(base + o_lB);
  const int rc = upload_pn(h, kidx, ncls, maxK);
  if (rc) return rc;
  return set_work_items(h, kRowsPerItem);
}

// Work items (target proton determinant, block, first neutron row, rows) in
// basis order, rows_per_item neutron rows each; replaces the current list.
int set_work_items(trbl_hamiltonian* h, int rows_per_item) {
  if (rows_per_item < 1) return fail(TRBL_ERR_ARG, "rows per work item must be positive");
  const trbl_basis* b = h->b;
  const Species& A = b->sp[0];
  std::vector<int4> work;
  const int64_t rb = h->row_begin, re = h->row_end < 0 ? b->D : h->row_end;
  for (size_t k = 0; k < b->blocks.size(); ++k) {
    const Block& bl = b->blocks[k];
    const int a0 = A.gfirst[bl.gA];
    for (int ia = 0; ia < bl.na; ++ia) {
      const int64_t slab = bl.off + int64_t(ia) * bl.nb;
      if (slab < rb || slab >= re) continue;
      for (int r0 = 0; r0 < bl.nb; r0 += rows_per_item)
        work.push_back(make_int4(a0 + ia, int(k), r0, std::min(rows_per_item, bl.nb - r0)));
    }
  }
  if (work.size() > size_t(0x7fffffff)) return fail(TRBL_ERR_ARG, "too many work items");
  if (work.empty())  // a shard without rows: one item of zero rows
    work.push_back(make_int4(A.gfirst[b->blocks[0].gA], 0, 0, 0));
  void* p = nullptr;
  TRBL_CUDA(cudaMalloc(&p, work.size() * sizeof(int4)));
  cudaError_t e = cudaMemcpy(p, work.data(), work.size() * sizeof(int4), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(p);
    return cuda_fail(e, "cudaMemcpy(work items)");
  }
  if (h->gwork) {
    cudaDeviceSynchronize();
    cudaFree(h->gwork);
  }
  h->gwork = p;
  h->rows_per_item = rows_per_item;
  h->g64.work = h->g32.work = static_cast<const int4*>(p);
  h->g64.nwork = h->g32.nwork = int(work.size());
  return set_pn_slabs(h);
}

}  // namespace trbl
