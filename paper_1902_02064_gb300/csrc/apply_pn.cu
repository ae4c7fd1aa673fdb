// Source-stationary cross-species product: the proton-neutron part of
// W = H V (App. B.2, Eq. (pntwobodybit)) for FP32 blocks, q a multiple of 16.
//
// The p-n term links a source row (pA, nB) to a target row (pA', nB') through
// a proton jump pA -> pA' (a+_a a_c, sign s_p) and a neutron jump nB -> nB'
// (b+_b b_d, sign s_n) of opposite 2m transfer, with coefficient
// s_p s_n V^AB_{ab,cd}.  Generated target by target (the grouped kernel),
// every element gathers its own source row: one row per element.  Here the
// loop order is turned around.  For a target proton determinant pA' and one
// transfer class, all proton jumps into pA' of that class read the same
// neutron source rows nB of their source slabs, and a source row nB feeds
// every outgoing neutron jump of nB of the opposite class.  A lane group
// therefore takes a source row, gathers V[pA, nB, :] once per proton jump,
// and multiplies it into one register accumulator per outgoing neutron jump
// (z_j += s_p V^AB_{a b_j, c d_j} V[pA, nB, :]); the accumulators are then
// added into their target rows nB'_j (times s_n).  A row of V is read once
// per (proton jump, source row) instead of once per generated element:
// 79 instead of 740 row reads per target row on the 18.6M-dim 5+5 space.
//
// * One thread block per (target slab pA', 16-column slice of W).  The slab
//   slice lives in shared memory (at most 1,651 rows x 64 bytes there),
//   initialised from W, which already holds the like-particle terms (the
//   grouped kernel ran first), and written back at the end.
// * Classes run one after another: the proton jumps of the class (source
//   slab offsets, and their coefficient rows with the proton sign applied)
//   are staged in shared memory, then lane groups of 4 lanes (16 bytes each,
//   one 64-byte row slice) walk the source rows of the class.
// * Targets are added with shared-memory atomic adds.  A row's 16 columns
//   are stored with their 4-column chunks permuted by the row index
//   ((row >> 1) & 3 exchanges floats inside a chunk) so that lane groups
//   adding to different rows in the same instruction spread over the banks.
//   The order of the adds is not fixed, so the FP32 rounding can differ from
//   run to run.
#include <cuda.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "tma.cuh"

namespace trbl {
namespace {

constexpr int kSlice = 16;  // columns of W per thread block
constexpr int kPnMaxSmem = 227 * 1024;

__device__ __forceinline__ float flipf(float c, int neg) { return __int_as_float(__float_as_int(c) ^ (neg << 31)); }

// Shared-memory position of column c (0..15) of slab row r.
__device__ __forceinline__ int acc_pos(int r, int c) { return r * kSlice + (c ^ ((r >> 1) & 3)); }

// Variants (registers per thread bound the accumulators and the gathers in
// flight): kJB outgoing neutron jumps per register batch, IU source rows
// gathered together (their coefficients read as one IU-wide vector), NT
// threads per block, MINB resident blocks per SM (shared memory allows two
// at the largest slab; 2 x 512 threads leave 64 registers a thread, 2 x 384
// leave 80).
template <int kJB, int IU, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    apply_pn_kernel(DevH<float> h, DevG<float> g, DevPN t, const float* __restrict__ V, int64_t ldv,
                    float* __restrict__ W, int64_t ldw) {
  static_assert(kJB % 4 == 0 && (IU == 2 || IU == 4), "batch of 4k jumps, 2 or 4 rows per gather");
  constexpr int kPnThreads = NT;
  constexpr int kGroups = NT / 4;
  extern __shared__ __align__(16) float pn_smem[];
  const int2 slab = t.slabs[blockIdx.x];
  const int pA = slab.x, blk = slab.y;
  const int col0 = blockIdx.y * kSlice;
  const int ND = h.ND, maxK = g.maxK;
  const int nb = h.bnb[blk];
  const int64_t rowA = h.boff[blk] + int64_t(pA - h.bgA[blk]) * nb;
  const int maxPp = (t.maxPc + 3) & ~3;
  float* acc = pn_smem;                                                  // [nbmax * 16]
  int* poff = reinterpret_cast<int*>(acc + size_t(t.nbmax) * kSlice);   // [maxPp]
  float* pcoef = reinterpret_cast<float*>(poff + maxPp);                // [maxK * maxPp], k-major
  const int tid = threadIdx.x;

  // the slab slice of W (like-particle terms) into the accumulator
  for (int i = tid; i < nb * 4; i += kPnThreads) {
    const int r = i >> 2, c = (i & 3) * 4;
    const float4 w = *reinterpret_cast<const float4*>(W + (rowA + r) * ldw + col0 + c);
    acc[acc_pos(r, c)] = w.x;
    acc[acc_pos(r, c + 1)] = w.y;
    acc[acc_pos(r, c + 2)] = w.z;
    acc[acc_pos(r, c + 3)] = w.w;
  }

  const int lane = tid & 31;
  const int grp = tid >> 2, sub = tid & 3;
  const unsigned gmask = 0xFu << (lane & ~3);  // the 4 lanes of this lane group
  const int ld = int(ldv);  // V offsets inside one block fit in 32 bits (D * ldv < 2^31, checked on the host)
  for (int di = 0; di < ND; ++di) {
    const int sb = h.srcblk[blk * ND + di];
    if (sb < 0) continue;
    const int e0 = h.jsegA[int64_t(pA) * ND + di];
    const int P = h.jsegA[int64_t(pA) * ND + di + 1] - e0;
    if (P == 0) continue;
    const int tn = ND - 1 - di;  // neutron transfer class opposite to the proton class
    const int Kc = t.ncls[tn];
    const int Pp = (P + IU - 1) / IU * IU;  // coefficient row stride (IU-aligned vectors)
    const int snb = h.bnb[sb];
    __syncthreads();  // the previous class is done with the staging buffers
    for (int i = tid; i < Pp; i += kPnThreads) poff[i] = i < P ? h.jA[e0 + i].x * snb * ld : 0;
    for (int x = tid; x < Pp * Kc; x += kPnThreads) {
      const int k = x / Pp, i = x - k * Pp;
      float c = 0.f;
      if (i < P) {
        const int2 ja = h.jA[e0 + i];
        c = flipf(g.ccoef[size_t(ja.y >> 1) * maxK + k], ja.y & 1);
      }
      pcoef[x] = c;  // pcoef[k * Pp + i]
    }
    __syncthreads();
    const float* Vs = V + h.boff[sb] * ldv + col0 + sub * 4;
    const int64_t n0 = int64_t(h.bgB[sb]) * ND + tn;
    for (int n = grp; n < snb; n += kGroups) {
      // segment of n's outgoing jumps of class tn: lanes 0 and 1 load its ends
      const int se = __ldg(&t.oseg[n0 + int64_t(n) * ND + (sub & 1)]);
      const int s0 = __shfl_sync(gmask, se, 0, 4), s1 = __shfl_sync(gmask, se, 1, 4);
      const float* vrow = Vs + n * ld;
      for (int jb = s0; jb < s1; jb += kJB) {
        // the batch's packed jump entries, one or two per lane, shared by shuffles
        int ent[kJB / 4];
#pragma unroll
        for (int r = 0; r < kJB / 4; ++r) {
          const int e = jb + sub + 4 * r;
          ent[r] = e < s1 ? __ldg(&t.jout[e]) : 0;
        }
        // coefficient row offsets k_j * Pp (< 2^16), two per register
        unsigned kpk[kJB / 2];
#pragma unroll
        for (int j = 0; j < kJB; j += 2) {
          const unsigned k0 = ((__shfl_sync(gmask, ent[j >> 2], j & 3, 4) >> 1) & 127) * Pp;
          const unsigned k1 = ((__shfl_sync(gmask, ent[j >> 2], (j + 1) & 3, 4) >> 1) & 127) * Pp;
          kpk[j >> 1] = k0 | (k1 << 16);
        }
        float4 z[kJB];
#pragma unroll
        for (int j = 0; j < kJB; ++j) z[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        int i = 0;
        for (; i + IU <= P; i += IU) {
          float4 v[IU];
#pragma unroll
          for (int u = 0; u < IU; ++u) v[u] = __ldg(reinterpret_cast<const float4*>(vrow + poff[i + u]));
#pragma unroll
          for (int j = 0; j < kJB; ++j) {
            const float* cp = pcoef + ((kpk[j >> 1] >> (16 * (j & 1))) & 0xFFFFu) + i;
            float c[IU];
            if constexpr (IU == 4) {
              const float4 c4 = *reinterpret_cast<const float4*>(cp);
              c[0] = c4.x, c[1] = c4.y, c[2] = c4.z, c[3] = c4.w;
            } else {
              const float2 c2 = *reinterpret_cast<const float2*>(cp);
              c[0] = c2.x, c[1] = c2.y;
            }
#pragma unroll
            for (int u = 0; u < IU; ++u) {
              z[j].x = fmaf(c[u], v[u].x, z[j].x);
              z[j].y = fmaf(c[u], v[u].y, z[j].y);
              z[j].z = fmaf(c[u], v[u].z, z[j].z);
              z[j].w = fmaf(c[u], v[u].w, z[j].w);
            }
          }
        }
        for (; i < P; ++i) {
          const float4 v = __ldg(reinterpret_cast<const float4*>(vrow + poff[i]));
#pragma unroll
          for (int j = 0; j < kJB; ++j) {
            const float c = pcoef[((kpk[j >> 1] >> (16 * (j & 1))) & 0xFFFFu) + i];
            z[j].x = fmaf(c, v.x, z[j].x);
            z[j].y = fmaf(c, v.y, z[j].y);
            z[j].z = fmaf(c, v.z, z[j].z);
            z[j].w = fmaf(c, v.w, z[j].w);
          }
        }
        const int J = min(kJB, s1 - jb);
        // the entries again (L1 hits), so that they need no registers during the products
#pragma unroll
        for (int r = 0; r < kJB / 4; ++r) {
          const int e = jb + sub + 4 * r;
          ent[r] = e < s1 ? __ldg(&t.jout[e]) : 0;
        }
#pragma unroll
        for (int j = 0; j < kJB; ++j) {
          const int e = __shfl_sync(gmask, ent[j >> 2], j & 3, 4);
          if (j < J) {
            const int r = e >> 8, neg = e & 1;
            float* dst = acc + r * kSlice;
            const int x = (r >> 1) & 3;
            const int c = sub * 4;
            atomicAdd(dst + ((c + 0) ^ x), flipf(z[j].x, neg));
            atomicAdd(dst + ((c + 1) ^ x), flipf(z[j].y, neg));
            atomicAdd(dst + ((c + 2) ^ x), flipf(z[j].z, neg));
            atomicAdd(dst + ((c + 3) ^ x), flipf(z[j].w, neg));
          }
        }
      }
    }
  }
  __syncthreads();
  for (int i = tid; i < nb * 4; i += kPnThreads) {
    const int r = i >> 2, c = (i & 3) * 4;
    *reinterpret_cast<float4*>(W + (rowA + r) * ldw + col0 + c) =
        make_float4(acc[acc_pos(r, c)], acc[acc_pos(r, c + 1)], acc[acc_pos(r, c + 2)], acc[acc_pos(r, c + 3)]);
  }
}

// ---------------------------------------------------------------------------
// Staged form (TRBL_APPLY_SPLIT_TMA).  The source rows of a class are read
// in chunks of C consecutive source determinants nB: for each proton jump of
// the class, 2-D TMA boxes of 16 columns x 32 rows land the C rows of that
// jump's source slab in shared memory, two chunks in flight (a producer warp
// and full/empty mbarriers).  A consumer warp takes one source row at a time;
// its 8 lane groups take 8 of the row's outgoing neutron jumps, all reading
// the same staged 64-byte row (a shared-memory broadcast), so control flow
// is uniform across the warp and V is read from shared memory only.  The
// row's jump entries still come from global memory, one dependent load per
// source row, and their latency is what bounds this form.
// The chunk length is chosen per class so that a chunk fills the stage
// buffer (C * P * 64 bytes, P proton jumps; C a multiple of the 32-row box,
// at most 256).  Every mbarrier wait is bounded:
// a timeout records an error word (read by the solver) and the warp stops;
// the producer waits (bounded) for its copies in flight before the block
// ends.

constexpr int kTmaWarps = 16;                  // consumer warps
constexpr int kTmaThreads = (kTmaWarps + 1) * 32;  // and one producer warp
constexpr int kBoxRows = 32;                   // rows of one TMA box (16 columns x 32 rows, 2 KB)
constexpr int kTmaMaxSmem = 226 * 1024;        // dynamic shared memory opt-in (the static word takes the rest)

__device__ int g_pn_err = 0;

__global__ void __launch_bounds__(kTmaThreads, 1)
    apply_pn_tma_kernel(const __grid_constant__ CUtensorMap vmap, DevH<float> h, DevG<float> g, DevPN t,
                        float* __restrict__ W, int64_t ldw, int stage_floats) {
  extern __shared__ __align__(128) unsigned char pn_raw[];
  float* stage0 = reinterpret_cast<float*>(pn_raw);            // [2][stage_floats]
  float* acc = stage0 + 2 * size_t(stage_floats);               // [nbmax * 16]
  float* coef = acc + size_t(t.nbmax) * kSlice;                  // [maxCoef] all classes' coefficients, i-major
  const int ND = h.ND, maxK = g.maxK;
  int* rowbase = reinterpret_cast<int*>(coef + t.maxCoef);     // [maxP] first row of each proton jump's source slab
  int* ctab = rowbase + g.maxP;                                 // [ND][10] class table
  uint64_t* bars = reinterpret_cast<uint64_t*>(ctab + ND * 10 + 2);  // full[2], empty[2] (8-byte aligned below)
  bars = reinterpret_cast<uint64_t*>((reinterpret_cast<uintptr_t>(bars) + 7) & ~uintptr_t(7));
  __shared__ int s_ncls;

  const int2 slab = t.slabs[blockIdx.x];
  const int pA = slab.x, blk = slab.y;
  const int col0 = blockIdx.y * kSlice;
  const int nb = h.bnb[blk];
  const int64_t rowA = h.boff[blk] + int64_t(pA - h.bgA[blk]) * nb;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  for (int i = tid; i < nb * 4; i += kTmaThreads) {
    const int r = i >> 2, c = (i & 3) * 4;
    const float4 w = *reinterpret_cast<const float4*>(W + (rowA + r) * ldw + col0 + c);
    acc[acc_pos(r, c)] = w.x;
    acc[acc_pos(r, c + 1)] = w.y;
    acc[acc_pos(r, c + 2)] = w.z;
    acc[acc_pos(r, c + 3)] = w.w;
  }
  // class table: (P, Kc, source rows, chunk rows C, coefficient offset, oseg base, proton-jump list
  // start, source block, first-row offset)
  if (tid == 0) {
    int nc = 0, coff = 0, roff = 0;
    for (int di = 0; di < ND; ++di) {
      const int sb = h.srcblk[blk * ND + di];
      if (sb < 0) continue;
      const int e0 = h.jsegA[int64_t(pA) * ND + di];
      const int P = h.jsegA[int64_t(pA) * ND + di + 1] - e0;
      if (P == 0) continue;
      const int tn = ND - 1 - di;
      const int C = min(256, stage_floats / (P * kSlice)) & ~(kBoxRows - 1);
      int* e = ctab + nc * 10;
      e[0] = P;
      e[1] = t.ncls[tn];
      e[2] = h.bnb[sb];
      e[3] = C;
      e[4] = coff;
      e[5] = h.bgB[sb] * ND + tn;
      e[6] = e0;
      e[7] = sb;
      e[8] = roff;
      coff += P * e[1];
      roff += P;
      ++nc;
    }
    s_ncls = nc;
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init(&bars[2], kTmaWarps);
    mbar_init(&bars[3], kTmaWarps);
    fence_barrier_init();
  }
  __syncthreads();
  const int ncls = s_ncls;
  for (int ci = 0; ci < ncls; ++ci) {
    const int* e = ctab + ci * 10;
    const int P = e[0], Kc = e[1], snb = e[2], e0 = e[6];
    const int64_t sbase = h.boff[e[7]];
    for (int i = tid; i < P; i += kTmaThreads) rowbase[e[8] + i] = int(sbase + int64_t(h.jA[e0 + i].x) * snb);
    for (int x = tid; x < P * Kc; x += kTmaThreads) {
      const int i = x / Kc, k = x - i * Kc;
      const int2 ja = h.jA[e0 + i];
      coef[e[4] + x] = flipf(g.ccoef[size_t(ja.y >> 1) * maxK + k], ja.y & 1);
    }
  }
  __syncthreads();

  if (warp == kTmaWarps) {
    // producer: one lane issues the boxes of every chunk, two chunks ahead
    if (lane == 0) {
      int tch = 0;
      bool ok = true;
      for (int ci = 0; ci < ncls && ok; ++ci) {
        const int* e = ctab + ci * 10;
        const int P = e[0], snb = e[2], C = e[3];
        const int* rb = rowbase + e[8];
        for (int n0 = 0; n0 < snb && ok; n0 += C, ++tch) {
          const int st = tch & 1;
          if (tch >= 2 && !mbar_wait(&bars[2 + st], uint32_t(((tch >> 1) - 1) & 1), &g_pn_err)) {
            ok = false;
            break;
          }
          float* dst = stage0 + size_t(st) * stage_floats;
          mbar_expect_tx(&bars[st], uint32_t(P * C * kSlice * 4));
          for (int i = 0; i < P; ++i)
            for (int b = 0; b < C; b += kBoxRows)
              tma_load_2d(dst + size_t(i * C + b) * kSlice, &vmap, col0, rb[i] + n0 + b, &bars[st]);
        }
      }
      // no copy may be in flight when the block ends: the last two chunks' boxes have landed
      for (int k = max(0, tch - 2); k < tch; ++k) mbar_wait(&bars[k & 1], uint32_t((k >> 1) & 1), &g_pn_err);
    }
  } else {
    const int grp = lane >> 2, sub = lane & 3;
    int tch = 0;
    bool ok = true;
    for (int ci = 0; ci < ncls && ok; ++ci) {
      const int* e = ctab + ci * 10;
      const int P = e[0], Kc = e[1], snb = e[2], C = e[3];
      const float* cbase = coef + e[4];
      const int obase = e[5];
      for (int n0 = 0; n0 < snb; n0 += C, ++tch) {
        const int st = tch & 1;
        if (!mbar_wait(&bars[st], uint32_t((tch >> 1) & 1), &g_pn_err)) {
          ok = false;
          break;
        }
        const float* xs = stage0 + size_t(st) * stage_floats + sub * 4;
        const int cn = min(C, snb - n0);
        for (int u = warp; u < cn; u += kTmaWarps) {
          const int n = n0 + u;
          const int s0 = __ldg(&t.oseg[obase + n * ND]);
          const int s1 = __ldg(&t.oseg[obase + n * ND + 1]);
          for (int jb = s0; jb < s1; jb += 8) {
            const int j = jb + grp;
            const int ent = j < s1 ? __ldg(&t.jout[j]) : 0;
            const float* cr = cbase + ((ent >> 1) & 127);
            const float* xr = xs + u * kSlice;
            float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
            for (int i = 0; i < P; ++i) {
              const float4 x = *reinterpret_cast<const float4*>(xr + size_t(i) * C * kSlice);
              const float c = cr[i * Kc];
              z.x = fmaf(c, x.x, z.x);
              z.y = fmaf(c, x.y, z.y);
              z.z = fmaf(c, x.z, z.z);
              z.w = fmaf(c, x.w, z.w);
            }
            if (j < s1) {
              const int r = ent >> 8, neg = ent & 1;
              float* dst = acc + r * kSlice;
              const int xm = (r >> 1) & 3;
              const int c = sub * 4;
              atomicAdd(dst + ((c + 0) ^ xm), flipf(z.x, neg));
              atomicAdd(dst + ((c + 1) ^ xm), flipf(z.y, neg));
              atomicAdd(dst + ((c + 2) ^ xm), flipf(z.z, neg));
              atomicAdd(dst + ((c + 3) ^ xm), flipf(z.w, neg));
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars[2 + st]);
      }
    }
  }
  __syncthreads();
  for (int i = tid; i < nb * 4; i += kTmaThreads) {
    const int r = i >> 2, c = (i & 3) * 4;
    *reinterpret_cast<float4*>(W + (rowA + r) * ldw + col0 + c) =
        make_float4(acc[acc_pos(r, c)], acc[acc_pos(r, c + 1)], acc[acc_pos(r, c + 2)], acc[acc_pos(r, c + 3)]);
  }
}

// Shared memory of the staged kernel: two stages, the accumulator, every
// class's coefficients and first source rows, the class table, barriers.
size_t pn_tma_fixed_bytes(const trbl_hamiltonian* h) {
  const int ND = h->b->ND;
  return size_t(h->pn.nbmax) * kSlice * 4 + size_t(h->pn.maxCoef) * 4 + size_t(h->g32.maxP) * 4 +
         size_t(ND) * 10 * 4 + 16 + 4 * 8;
}

size_t pn_smem_bytes(int nbmax, int maxPc, int maxK) {
  const size_t maxPp = size_t(maxPc + 3) & ~size_t(3);
  return size_t(nbmax) * kSlice * 4 + maxPp * 4 + maxPp * maxK * 4;
}

template <int kJB, int IU, int NT, int MINB>
int launch_pn(const trbl_hamiltonian* h, dim3 grid, size_t sm, const float* V, int64_t ldv, float* W, int64_t ldw,
              cudaStream_t s) {
  // opt in once to the largest dynamic shared memory a block may use (thread-safe initialisation)
  static const cudaError_t cfg = cudaFuncSetAttribute(apply_pn_kernel<kJB, IU, NT, MINB>,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize, kPnMaxSmem);
  TRBL_CUDA(cfg);
  apply_pn_kernel<kJB, IU, NT, MINB><<<grid, NT, sm, s>>>(h->d32, h->g32, h->pn, V, ldv, W, ldw);
  note_launch();
  TRBL_CUDA(cudaGetLastError());
  return TRBL_OK;
}

}  // namespace

int upload_pn(trbl_hamiltonian* h, const std::vector<int>& kidx, const std::vector<int>& ncls, int maxK) {
  const trbl_basis* b = h->b;
  const Species& A = b->sp[0];
  const Species& B = b->sp[1];
  const int ND = b->ND, span = b->dspan, nB = B.n;
  const int ndetB = int(B.bits.size());
  int nbmax = 1, maxPc = 1, maxCoef = 1;
  for (size_t k = 0; k < b->blocks.size(); ++k) {
    const Block& bl = b->blocks[k];
    nbmax = std::max(nbmax, bl.nb);
    const int a0 = A.gfirst[bl.gA];
    for (int ia = 0; ia < bl.na; ++ia) {
      int nco = 0;
      for (int di = 0; di < ND; ++di)
        if (b->srcblk[k * ND + di] >= 0) {
          const int P = A.jseg[size_t(a0 + ia) * ND + di + 1] - A.jseg[size_t(a0 + ia) * ND + di];
          maxPc = std::max(maxPc, P);
          nco += P * ncls[ND - 1 - di];
        }
      maxCoef = std::max(maxCoef, nco);
    }
  }
  if (pn_smem_bytes(nbmax, maxPc, maxK) > size_t(kPnMaxSmem)) return TRBL_OK;  // slab too large: not available
  // packing of the jump entries (k < 128, target < 2^23) and of the coefficient row offsets (< 2^16)
  if (maxK > 128 || nbmax >= (1 << 23) || size_t(maxPc + 3) / 4 * 4 * maxK >= (1u << 16)) return TRBL_OK;
  // outgoing neutron jumps by (source, transfer class), targets ascending
  std::vector<int32_t> oseg(size_t(ndetB) * ND + 1, 0);
  for (size_t e = 0; e < B.jsrc.size(); ++e) {
    const int tn = B.twom[B.ja[e]] - B.twom[B.jc[e]] + span;
    oseg[size_t(B.jsrc[e]) * ND + tn + 1]++;
  }
  for (size_t i = 1; i < oseg.size(); ++i) oseg[i] += oseg[i - 1];
  std::vector<int32_t> fillp(oseg.begin(), oseg.end() - 1);
  std::vector<int32_t> jout(B.jsrc.size());
  for (int tB = 0; tB < ndetB; ++tB) {
    const int tloc = tB - B.gfirst[B.group[tB]];
    for (int e = B.jseg[size_t(tB) * ND]; e < B.jseg[size_t(tB + 1) * ND]; ++e) {
      const int tn = B.twom[B.ja[e]] - B.twom[B.jc[e]] + span;
      const int k = kidx[size_t(B.ja[e]) * nB + B.jc[e]];
      jout[fillp[size_t(B.jsrc[e]) * ND + tn]++] = (tloc << 8) | (k << 1) | (B.jsign[e] < 0 ? 1 : 0);
    }
  }
  const size_t o_oseg = 0;
  const size_t o_jout = (o_oseg + oseg.size() * 4 + 255) & ~size_t(255);
  const size_t o_ncls = (o_jout + jout.size() * 4 + 255) & ~size_t(255);
  const size_t total = o_ncls + size_t(ND) * 4 + 256;
  void* arena = nullptr;
  TRBL_CUDA(cudaMalloc(&arena, total));
  h->pnarena = arena;
  char* base = static_cast<char*>(arena);
  TRBL_CUDA(cudaMemcpy(base + o_oseg, oseg.data(), oseg.size() * 4, cudaMemcpyHostToDevice));
  if (!jout.empty()) TRBL_CUDA(cudaMemcpy(base + o_jout, jout.data(), jout.size() * 4, cudaMemcpyHostToDevice));
  TRBL_CUDA(cudaMemcpy(base + o_ncls, ncls.data(), size_t(ND) * 4, cudaMemcpyHostToDevice));
  h->pn.oseg = reinterpret_cast<const int32_t*>(base + o_oseg);
  h->pn.jout = reinterpret_cast<const int32_t*>(base + o_jout);
  h->pn.ncls = reinterpret_cast<const int32_t*>(base + o_ncls);
  h->pn.nbmax = nbmax;
  h->pn.maxPc = maxPc;
  h->pn.maxCoef = maxCoef;
  return TRBL_OK;
}

// Target slabs inside the row range, largest first (equal sizes in basis order).
int set_pn_slabs(trbl_hamiltonian* h) {
  if (!h->pn.oseg) return TRBL_OK;
  const trbl_basis* b = h->b;
  const Species& A = b->sp[0];
  const int64_t rb = h->row_begin, re = h->row_end < 0 ? b->D : h->row_end;
  std::vector<int2> slabs;
  std::vector<int> size;
  for (size_t k = 0; k < b->blocks.size(); ++k) {
    const Block& bl = b->blocks[k];
    const int a0 = A.gfirst[bl.gA];
    for (int ia = 0; ia < bl.na; ++ia) {
      const int64_t slab = bl.off + int64_t(ia) * bl.nb;
      if (slab < rb || slab >= re || bl.nb == 0) continue;
      slabs.push_back(make_int2(a0 + ia, int(k)));
      size.push_back(bl.nb);
    }
  }
  std::vector<size_t> order(slabs.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return size[x] > size[y]; });
  std::vector<int2> sorted(slabs.size());
  for (size_t i = 0; i < order.size(); ++i) sorted[i] = slabs[order[i]];
  void* p = nullptr;
  if (!sorted.empty()) {
    TRBL_CUDA(cudaMalloc(&p, sorted.size() * sizeof(int2)));
    cudaError_t e = cudaMemcpy(p, sorted.data(), sorted.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(p);
      return cuda_fail(e, "cudaMemcpy(target slabs)");
    }
  }
  if (h->pnslabs) {
    cudaDeviceSynchronize();
    cudaFree(h->pnslabs);
  }
  h->pnslabs = p;
  h->pn.slabs = static_cast<const int2*>(p);
  h->pn.nslab = int(sorted.size());
  return TRBL_OK;
}

// Stage size of the staged kernel (floats per stage; 0: it does not fit).
int pn_tma_stage_floats(const trbl_hamiltonian* h) {
  const size_t fixed = pn_tma_fixed_bytes(h);
  if (fixed + 2048 >= size_t(kTmaMaxSmem)) return 0;
  size_t st = (size_t(kTmaMaxSmem) - fixed - 2048) / 2 / 4;  // slack for the alignment of the stages
  st = std::min<size_t>(st, 40 * 1024 / 4) & ~size_t(255);  // 40 KB stages are enough to hide the copies
  if (st < size_t(h->pn.maxPc) * kBoxRows * kSlice) return 0;  // at least one box per proton jump
  return int(st);
}

int pn_tma_error_to_host(int* host, cudaStream_t s) {
  TRBL_CUDA(cudaMemcpyFromSymbolAsync(host, g_pn_err, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
  return TRBL_OK;
}

int launch_split(const trbl_hamiltonian* h, const void* V, int64_t ldv, void* W, int64_t ldw, int q, int dtype,
                 cudaStream_t s) {
  if ((h->apply_kernel != TRBL_APPLY_SPLIT && h->apply_kernel != TRBL_APPLY_SPLIT_X4 &&
       h->apply_kernel != TRBL_APPLY_SPLIT_TMA) ||
      dtype != TRBL_F32 || !h->pn.oseg)
    return -1;
  if (q != 16 && q != 32 && q != 64) return -1;
  if ((reinterpret_cast<uintptr_t>(V) | reinterpret_cast<uintptr_t>(W)) & 15) return -1;
  if (ldv % 4 || ldw % 4) return -1;
  if (h->b->D * ldv >= (int64_t(1) << 31)) return -1;
  const float* Vf = static_cast<const float*>(V);
  float* Wf = static_cast<float*>(W);
  const int rc = launch_grouped_like(h, Vf, ldv, Wf, ldw, q, s);
  if (rc) return rc == -1 ? fail(TRBL_ERR_ARG, "split product: the like-particle launch does not apply") : rc;
  if (h->pn.nslab == 0) return TRBL_OK;
  const dim3 grid{static_cast<unsigned>(h->pn.nslab), static_cast<unsigned>(q / kSlice), 1u};
  if (h->apply_kernel == TRBL_APPLY_SPLIT_TMA) {
    const int stage = pn_tma_stage_floats(h);
    if (!stage) return fail(TRBL_ERR_ARG, "split product: the staged cross-term kernel does not fit in shared memory");
    CUtensorMap map;
    const int r = make_tmap_2d_f32_rows(&map, Vf, uint64_t(q), uint64_t(h->b->D), uint64_t(ldv), kSlice, kBoxRows);
    if (r) return r;
    const size_t sm = pn_tma_fixed_bytes(h) + size_t(2) * stage * 4 + 128;
    static const cudaError_t cfg =
        cudaFuncSetAttribute(apply_pn_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTmaMaxSmem);
    TRBL_CUDA(cfg);
    apply_pn_tma_kernel<<<grid, kTmaThreads, sm, s>>>(map, h->d32, h->g32, h->pn, Wf, ldw, stage);
    note_launch();
    TRBL_CUDA(cudaGetLastError());
    return TRBL_OK;
  }
  const size_t sm = pn_smem_bytes(h->pn.nbmax, h->pn.maxPc, h->g32.maxK);
  if (h->apply_kernel == TRBL_APPLY_SPLIT_X4) return launch_pn<4, 4, 512, 2>(h, grid, sm, Vf, ldv, Wf, ldw, s);
  if (h->blocks_per_sm == 1) return launch_pn<8, 4, 512, 1>(h, grid, sm, Vf, ldv, Wf, ldw, s);
  return launch_pn<8, 2, 384, 2>(h, grid, sm, Vf, ldv, Wf, ldw, s);
}

}  // namespace trbl
