// Block Hamiltonian product W = H V on the two-species M-scheme basis with
// matrix elements generated on the fly (App. B), and the upload of the tables
// it reads.
//
// H = H_A (x) 1 + 1 (x) H_B + H_AB.  For an output row (pA', nB'):
//   * like-particle rows (App. B.1): sum over pA of H_A[pA', pA] V[pA, nB']
//     and over nB of H_B[nB', nB] V[pA', nB];
//   * cross-species part (App. B.2 Eq. (pntwobodybit)): the term
//     a+_a b+_b b_d a_c factorises into a one-body jump of species A
//     (pA -> pA', sign sA) times one of species B (nB -> nB', sign sB) with
//     opposite 2m transfers, so the row sums sA sB V^AB_{ab,cd} V[pA, nB]
//     over incoming A jumps x incoming B jumps of matching transfer.
//     Diagonal jumps (a = c, b = d) carry the number-operator parts.
// Every generated element is used for all q columns of the block, which is
// the point of the block method (Sec. IV B).
#include <cstdio>
#include <cstring>
#include <vector>

#include "internal.h"

namespace trbl {

namespace {

struct ArenaPlan {
  size_t bytes = 0;
  size_t take(size_t n) {
    size_t o = (bytes + 255) & ~size_t(255);
    bytes = o + n;
    return o;
  }
};

template <typename T>
__device__ __forceinline__ int find_block(const DevH<T>& h, int64_t r) {
  int lo = 0, hi = h.nblk - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(h.boff + mid) <= r)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// One thread per (row, column): gathers every source of its output element.
template <typename T>
__global__ void __launch_bounds__(256) apply_rows_kernel(DevH<T> h, const T* __restrict__ V,
                                                         int64_t ldv, T* __restrict__ W,
                                                         int64_t ldw, int q, int64_t D) {
  const int64_t gt = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t r = gt / q;
  const int col = int(gt - r * q);
  if (r >= D) return;
  const int blk = find_block(h, r);
  const int64_t off = __ldg(h.boff + blk);
  const int nb = __ldg(h.bnb + blk);
  const int64_t loc = r - off;
  const int iA = int(loc / nb);
  const int iB = int(loc - int64_t(iA) * nb);
  const int pA = __ldg(h.bgA + blk) + iA;
  const int pB = __ldg(h.bgB + blk) + iB;
  const T* Vc = V + col;
  T acc = T(0);
  // like-particle rows of species A: same neutron determinant
  for (int e = __ldg(h.hoffA + pA), ee = __ldg(h.hoffA + pA + 1); e < ee; ++e)
    acc += __ldg(h.hcoefA + e) * Vc[(off + int64_t(__ldg(h.hsrcA + e)) * nb + iB) * ldv];
  // like-particle rows of species B: same proton determinant
  const int64_t rowA = off + int64_t(iA) * nb;
  for (int e = __ldg(h.hoffB + pB), ee = __ldg(h.hoffB + pB + 1); e < ee; ++e)
    acc += __ldg(h.hcoefB + e) * Vc[(rowA + __ldg(h.hsrcB + e)) * ldv];
  // cross-species part: A jump with transfer index di x B jump with the opposite transfer
  const int ND = h.ND;
  const int nB2 = h.nB * h.nB;
  for (int di = 0; di < ND; ++di) {
    const int sb = __ldg(h.srcblk + blk * ND + di);
    if (sb < 0) continue;
    const int pb = __ldg(h.jsegA + int64_t(pA) * ND + di);
    const int pe = __ldg(h.jsegA + int64_t(pA) * ND + di + 1);
    const int dn = ND - 1 - di;
    const int nbg = __ldg(h.jsegB + int64_t(pB) * ND + dn);
    const int ne = __ldg(h.jsegB + int64_t(pB) * ND + dn + 1);
    if (pb == pe || nbg == ne) continue;
    const int64_t soff = __ldg(h.boff + sb);
    const int snb = __ldg(h.bnb + sb);
    for (int ep = pb; ep < pe; ++ep) {
      const int2 ja = __ldg(h.jA + ep);
      const T* vrow = Vc + (soff + int64_t(ja.x) * snb) * ldv;
      const T* coef = h.vab + int64_t(ja.y >> 1) * nB2;
      const int negA = ja.y & 1;
      T part = T(0);
      for (int en = nbg; en < ne; ++en) {
        const int2 jb = __ldg(h.jB + en);
        T c = __ldg(coef + (jb.y >> 1));
        if ((jb.y ^ negA) & 1) c = -c;
        part += c * vrow[int64_t(jb.x) * ldv];
      }
      acc += part;
    }
  }
  W[r * ldw + col] = acc;
}

template <typename T>
int launch_typed(const DevH<T>& h, int64_t D, const T* V, int64_t ldv, T* W, int64_t ldw, int q,
                 cudaStream_t s) {
  const int64_t threads = D * q;
  const int bs = 256;
  const int64_t grid = (threads + bs - 1) / bs;
  if (grid > 0x7fffffffLL) return fail(TRBL_ERR_ARG, "block too large for one launch");
  apply_rows_kernel<T><<<unsigned(grid), bs, 0, s>>>(h, V, ldv, W, ldw, q, D); note_launch();
  TRBL_CUDA(cudaGetLastError());
  return TRBL_OK;
}

}  // namespace

int upload_tables(trbl_hamiltonian* h) {
  const trbl_basis* b = h->b;
  const Species& A = b->sp[0];
  const Species& B = b->sp[1];
  const int nblk = int(b->blocks.size());
  std::vector<int64_t> boff(nblk);
  std::vector<int32_t> bnb(nblk), bgA(nblk), bgB(nblk);
  for (int k = 0; k < nblk; ++k) {
    boff[k] = b->blocks[k].off;
    bnb[k] = b->blocks[k].nb;
    bgA[k] = A.gfirst[b->blocks[k].gA];
    bgB[k] = B.gfirst[b->blocks[k].gB];
  }
  auto pack = [](const Species& S) {
    std::vector<int2> v(S.jsrc.size());
    for (size_t e = 0; e < v.size(); ++e) {
      int src = S.jsrc[e];
      int loc = src - S.gfirst[S.group[src]];
      int op = ((S.ja[e] * S.n + S.jc[e]) << 1) | (S.jsign[e] < 0 ? 1 : 0);
      v[e] = make_int2(loc, op);
    }
    return v;
  };
  std::vector<int2> jA = pack(A), jB = pack(B);
  std::vector<float> hcA32(h->hcoef[0].begin(), h->hcoef[0].end());
  std::vector<float> hcB32(h->hcoef[1].begin(), h->hcoef[1].end());
  std::vector<float> vab32(h->vab.begin(), h->vab.end());

  struct Item {
    const void* src;
    size_t bytes;
    size_t off;
  };
  std::vector<Item> items;
  ArenaPlan plan;
  auto add = [&](const void* p, size_t n) {
    size_t o = plan.take(n > 0 ? n : 1);
    items.push_back({p, n, o});
    return o;
  };
  size_t o_boff = add(boff.data(), boff.size() * 8);
  size_t o_bnb = add(bnb.data(), bnb.size() * 4);
  size_t o_bgA = add(bgA.data(), bgA.size() * 4);
  size_t o_bgB = add(bgB.data(), bgB.size() * 4);
  size_t o_srcblk = add(b->srcblk.data(), b->srcblk.size() * 4);
  size_t o_jsegA = add(A.jseg.data(), A.jseg.size() * 4);
  size_t o_jA = add(jA.data(), jA.size() * 8);
  size_t o_jsegB = add(B.jseg.data(), B.jseg.size() * 4);
  size_t o_jB = add(jB.data(), jB.size() * 8);
  size_t o_hoffA = add(h->hoff[0].data(), h->hoff[0].size() * 4);
  size_t o_hsrcA = add(h->hsrc[0].data(), h->hsrc[0].size() * 4);
  size_t o_hcA64 = add(h->hcoef[0].data(), h->hcoef[0].size() * 8);
  size_t o_hcA32 = add(hcA32.data(), hcA32.size() * 4);
  size_t o_hoffB = add(h->hoff[1].data(), h->hoff[1].size() * 4);
  size_t o_hsrcB = add(h->hsrc[1].data(), h->hsrc[1].size() * 4);
  size_t o_hcB64 = add(h->hcoef[1].data(), h->hcoef[1].size() * 8);
  size_t o_hcB32 = add(hcB32.data(), hcB32.size() * 4);
  size_t o_vab64 = add(h->vab.data(), h->vab.size() * 8);
  size_t o_vab32 = add(vab32.data(), vab32.size() * 4);

  TRBL_CUDA(cudaGetDevice(&h->device));
  void* arena = nullptr;
  TRBL_CUDA(cudaMalloc(&arena, plan.bytes));
  h->arena = arena;
  h->arena_bytes = plan.bytes;
  char* base = static_cast<char*>(arena);
  for (const Item& it : items)
    if (it.bytes) TRBL_CUDA(cudaMemcpy(base + it.off, it.src, it.bytes, cudaMemcpyHostToDevice));

  auto fill = [&](auto& d, size_t o_hcA, size_t o_hcB, size_t o_vab) {
    using TT = typename std::remove_pointer<typename std::remove_const<
        typename std::remove_pointer<decltype(d.vab)>::type>::type>::type;
    d.nblk = nblk;
    d.ND = b->ND;
    d.nA = A.n;
    d.nB = B.n;
    d.boff = reinterpret_cast<const int64_t*>(base + o_boff);
    d.bnb = reinterpret_cast<const int32_t*>(base + o_bnb);
    d.bgA = reinterpret_cast<const int32_t*>(base + o_bgA);
    d.bgB = reinterpret_cast<const int32_t*>(base + o_bgB);
    d.srcblk = reinterpret_cast<const int32_t*>(base + o_srcblk);
    d.jsegA = reinterpret_cast<const int32_t*>(base + o_jsegA);
    d.jA = reinterpret_cast<const int2*>(base + o_jA);
    d.jsegB = reinterpret_cast<const int32_t*>(base + o_jsegB);
    d.jB = reinterpret_cast<const int2*>(base + o_jB);
    d.hoffA = reinterpret_cast<const int32_t*>(base + o_hoffA);
    d.hsrcA = reinterpret_cast<const int32_t*>(base + o_hsrcA);
    d.hcoefA = reinterpret_cast<const TT*>(base + o_hcA);
    d.hoffB = reinterpret_cast<const int32_t*>(base + o_hoffB);
    d.hsrcB = reinterpret_cast<const int32_t*>(base + o_hsrcB);
    d.hcoefB = reinterpret_cast<const TT*>(base + o_hcB);
    d.vab = reinterpret_cast<const TT*>(base + o_vab);
  };
  fill(h->d64, o_hcA64, o_hcB64, o_vab64);
  fill(h->d32, o_hcA32, o_hcB32, o_vab32);
  return upload_grouped(h);
}

int launch_apply(const trbl_hamiltonian* h, const void* V, int64_t ldv, void* W, int64_t ldw,
                 int q, int dtype, cudaStream_t s) {
  const int g = launch_grouped(h, V, ldv, W, ldw, q, dtype, s);
  if (g != -1) return g;
  if (h->row_end >= 0 && (h->row_begin != 0 || h->row_end != h->b->D))
    return fail(TRBL_ERR_ARG, "a row-restricted product needs 16-byte aligned rows of q * element size = 16 * 2^i "
                              "bytes (the grouped and fast kernels)");
  const int64_t D = h->b->D;
  if (dtype == TRBL_F64)
    return launch_typed<double>(h->d64, D, static_cast<const double*>(V), ldv,
                                static_cast<double*>(W), ldw, q, s);
  return launch_typed<float>(h->d32, D, static_cast<const float*>(V), ldv, static_cast<float*>(W),
                             ldw, q, s);
}

}  // namespace trbl

using namespace trbl;

static int check_device_ptr(const void* p, const char* name) {
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(TRBL_ERR_ARG, "%s: not a CUDA pointer (%s)", name, cudaGetErrorString(e));
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
    return fail(TRBL_ERR_ARG, "%s must be device memory", name);
  return TRBL_OK;
}

extern "C" int trbl_apply_block(const trbl_hamiltonian* h, const void* V, int64_t ldv, void* W,
                                int64_t ldw, int q, int dtype, void* stream) {
  clear_error();
  if (!h || !V || !W) return fail(TRBL_ERR_ARG, "null argument");
  if (q < 1 || q > 64) return fail(TRBL_ERR_ARG, "q=%d outside [1, 64]", q);
  if (ldv < q || ldw < q) return fail(TRBL_ERR_ARG, "leading dimension smaller than q");
  if (dtype != TRBL_F32 && dtype != TRBL_F64) return fail(TRBL_ERR_ARG, "bad dtype %d", dtype);
  int rc = check_device_ptr(V, "V");
  if (rc) return rc;
  rc = check_device_ptr(W, "W");
  if (rc) return rc;
  if (V == W) return fail(TRBL_ERR_ARG, "V and W must not overlap");
  return launch_apply(h, V, ldv, W, ldw, q, dtype, static_cast<cudaStream_t>(stream));
}
