// Hellmann-Feynman gradient: sum over given vectors x_k of <x_k| dH/dtheta |x_k>
// for every parameter theta of H (Sec. II: H is linear in h(1)_ac and in the
// two-body matrix elements, so dH/dtheta is the operator term theta
// multiplies).
//
// The adjoint traversal visits the same elements as the block product
// (App. B): for an output row i and a generated element (i <- j, operator
// term T, fermion sign s) it adds s * sum_k x_k[i] x_k[j] to the bin of T.
// Cross-species elements come from proton jump x neutron jump pairs
// (App. B.2); like-particle pairs of determinants are split into their
// individual one-body and two-body terms (with spectators) from the bit
// strings, because the product kernels only keep their summed coefficient.
// Bins are FP64, filled with atomic adds (summation order not fixed); the
// host folds term bins into the canonical parameter order: a parameter at
// slot (I, J), I != J, multiplies both the term (I, J) and its conjugate
// (J, I).
#include <algorithm>
#include <vector>

#include "internal.h"

namespace trbl {
namespace {

struct GradTables {
  const uint32_t* bitsA;
  const uint32_t* bitsB;
  const int32_t* pA_off;  // structural like-particle pairs of species A by target: source local index
  const int32_t* pA_src;
  const int32_t* pB_off;
  const int32_t* pB_src;
  double* b1A;  // [nA*nA]
  double* b1B;  // [nB*nB]
  double* b2A;  // [nA^4], index ((a*nA+b)*nA+c)*nA+d, a<b, c<d
  double* b2B;
  double* bAB;  // [(a*nA+c)*nB*nB + b*nB+d]
};

__device__ __forceinline__ int sign_before(uint32_t s, int x) { return (__popc(s & ((1u << x) - 1u)) & 1) ? -1 : 1; }

// sign of x+_a x+_b x_d x_c acting on s (x_c first)
__device__ int two_body_sign_dev(uint32_t s, int a, int b, int c, int d) {
  int sg = sign_before(s, c);
  s ^= 1u << c;
  sg *= sign_before(s, d);
  s ^= 1u << d;
  sg *= sign_before(s, b);
  s |= 1u << b;
  sg *= sign_before(s, a);
  return sg;
}

__device__ __forceinline__ int bit_index(uint32_t x) { return __ffs(x) - 1; }

// Adds dot to the bins of every like-particle term linking source s to target t.
// The diagonal terms (s = t: n_a and n_a n_b) go to the thread block's
// shared bins d1[a], d2[a n + b], which every row of the block hits, or to
// b1, b2 when d1, d2 are null.
__device__ void add_like_terms(uint32_t t, uint32_t s, int n, double dot, double* b1, double* b2, double* d1,
                               double* d2) {
  const uint32_t diff = t ^ s;
  const int moved = __popc(diff) >> 1;
  if (moved == 0) {
    for (uint32_t r = s; r; r &= r - 1) {
      const int a = bit_index(r);
      if (d1)
        atomicAdd(d1 + a, dot);
      else
        atomicAdd(b1 + a * n + a, dot);
      for (uint32_t r2 = r & (r - 1); r2; r2 &= r2 - 1) {
        const int b = bit_index(r2);
        if (d2)
          atomicAdd(d2 + a * n + b, dot);  // n_a n_b, sign +1
        else
          atomicAdd(b2 + ((size_t(a) * n + b) * n + a) * n + b, dot);
      }
    }
  } else if (moved == 1) {
    const int a = bit_index(t & diff), c = bit_index(s & diff);
    // one-body a+_a a_c
    const int sg1 = sign_before(s, c) * sign_before(s ^ (1u << c), a);
    atomicAdd(b1 + a * n + c, sg1 * dot);
    // two-body with a spectator x occupied in both
    for (uint32_t r = s & t; r; r &= r - 1) {
      const int x = bit_index(r);
      const int a1 = min(a, x), b1_ = max(a, x), c1 = min(c, x), d1 = max(c, x);
      const int sg = two_body_sign_dev(s, a1, b1_, c1, d1);
      atomicAdd(b2 + ((size_t(a1) * n + b1_) * n + c1) * n + d1, sg * dot);
    }
  } else {
    const uint32_t cr = t & diff, an = s & diff;
    const int a = bit_index(cr), b = bit_index(cr & (cr - 1));
    const int c = bit_index(an), d = bit_index(an & (an - 1));
    const int sg = two_body_sign_dev(s, a, b, c, d);
    atomicAdd(b2 + ((size_t(a) * n + b) * n + c) * n + d, sg * dot);
  }
}

template <typename T>
__device__ __forceinline__ double warp_dot(T x, T y) {
  double v = double(x) * double(y);
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One warp per output row; lane k holds x_k[row] (nvec <= 32).
template <typename T>
__device__ void grad_row(const DevH<T>& h, const GradTables& g, const T* __restrict__ X, int64_t ldx, int nvec,
                         int64_t r, int lane, double* sAB, double* s1A, double* s2A, double* s1B, double* s2B) {
  int lo = 0, hi = h.nblk - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (h.boff[mid] <= r)
      lo = mid;
    else
      hi = mid - 1;
  }
  const int blk = lo;
  const int64_t off = h.boff[blk];
  const int nb = h.bnb[blk];
  const int iA = int((r - off) / nb), iB = int((r - off) - int64_t(iA) * nb);
  const int gA0 = h.bgA[blk], gB0 = h.bgB[blk];
  const int pA = gA0 + iA, pB = gB0 + iB;
  const T xr = lane < nvec ? X[r * ldx + lane] : T(0);
  const int nA = h.nA, nB = h.nB, nB2 = nB * nB, ND = h.ND;
  // cross-species elements
  for (int di = 0; di < ND; ++di) {
    const int sb = h.srcblk[blk * ND + di];
    if (sb < 0) continue;
    const int pb = h.jsegA[int64_t(pA) * ND + di], pe = h.jsegA[int64_t(pA) * ND + di + 1];
    const int dn = ND - 1 - di;
    const int nbg = h.jsegB[int64_t(pB) * ND + dn], ne = h.jsegB[int64_t(pB) * ND + dn + 1];
    if (pb == pe || nbg == ne) continue;
    const int64_t soff = h.boff[sb];
    const int snb = h.bnb[sb];
    for (int ep = pb; ep < pe; ++ep) {
      const int2 ja = h.jA[ep];
      const int64_t rowA = soff + int64_t(ja.x) * snb;
      for (int en = nbg; en < ne; ++en) {
        const int2 jb = h.jB[en];
        const int64_t src = rowA + jb.x;
        const T xs = lane < nvec ? X[src * ldx + lane] : T(0);
        const double d = warp_dot(xr, xs);
        if (lane == 0) {
          const double v = ((ja.y ^ jb.y) & 1) ? -d : d;
          const int ia = ja.y >> 1, ib = jb.y >> 1;
          if (ia % (nA + 1) == 0 && ib % (nB + 1) == 0)
            atomicAdd(sAB + (ia / (nA + 1)) * nB + ib / (nB + 1), v);  // n_a n_b: every row hits it
          else
            atomicAdd(g.bAB + int64_t(ia) * nB2 + ib, v);
        }
      }
    }
  }
  (void)nA;
  // like-particle pairs of species A (neutron unchanged)
  const uint32_t tA = g.bitsA[pA];
  for (int e = g.pA_off[pA]; e < g.pA_off[pA + 1]; ++e) {
    const int sA = g.pA_src[e];
    const int64_t src = off + int64_t(sA) * nb + iB;
    const T xs = lane < nvec ? X[src * ldx + lane] : T(0);
    const double d = warp_dot(xr, xs);
    if (lane == 0) add_like_terms(tA, g.bitsA[gA0 + sA], h.nA, d, g.b1A, g.b2A, s1A, s2A);
  }
  // like-particle pairs of species B (proton unchanged)
  const uint32_t tB = g.bitsB[pB];
  for (int e = g.pB_off[pB]; e < g.pB_off[pB + 1]; ++e) {
    const int sB = g.pB_src[e];
    const int64_t src = off + int64_t(iA) * nb + sB;
    const T xs = lane < nvec ? X[src * ldx + lane] : T(0);
    const double d = warp_dot(xr, xs);
    if (lane == 0) add_like_terms(tB, g.bitsB[gB0 + sB], h.nB, d, g.b1B, g.b2B, s1B, s2B);
  }
}

// Persistent blocks of 8 warps, a warp per row at a time.  The diagonal
// bins (n_a n_b across species, n_a and n_a n_b within one), which every
// row adds to, are summed in shared memory and added to the global bins
// once per block; the other bins take global atomic adds.
template <typename T>
__global__ void __launch_bounds__(256) grad_kernel(DevH<T> h, GradTables g, const T* __restrict__ X, int64_t ldx,
                                                   int nvec, int64_t D) {
  __shared__ double sAB[32 * 32], s2A[32 * 32], s2B[32 * 32], s1A[32], s1B[32];
  const int tid = threadIdx.x, lane = tid & 31;
  for (int i = tid; i < 32 * 32; i += blockDim.x) sAB[i] = s2A[i] = s2B[i] = 0.0;
  if (tid < 32) s1A[tid] = s1B[tid] = 0.0;
  __syncthreads();
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t r = int64_t(blockIdx.x) * wpb + (tid >> 5); r < D; r += int64_t(gridDim.x) * wpb)
    grad_row<T>(h, g, X, ldx, nvec, r, lane, sAB, s1A, s2A, s1B, s2B);
  __syncthreads();
  const int nA = h.nA, nB = h.nB;
  for (int i = tid; i < nA * nB; i += blockDim.x) {
    const int a = i / nB, b = i - a * nB;
    const double v = sAB[a * nB + b];
    if (v != 0.0) atomicAdd(g.bAB + int64_t(a * nA + a) * nB * nB + b * nB + b, v);
  }
  for (int i = tid; i < nA * nA; i += blockDim.x) {
    const int a = i / nA, b = i - a * nA;
    const double v = s2A[i];
    if (v != 0.0) atomicAdd(g.b2A + ((size_t(a) * nA + b) * nA + a) * nA + b, v);
  }
  for (int i = tid; i < nB * nB; i += blockDim.x) {
    const int a = i / nB, b = i - a * nB;
    const double v = s2B[i];
    if (v != 0.0) atomicAdd(g.b2B + ((size_t(a) * nB + b) * nB + a) * nB + b, v);
  }
  if (tid < nA && s1A[tid] != 0.0) atomicAdd(g.b1A + tid * nA + tid, s1A[tid]);
  if (tid < nB && s1B[tid] != 0.0) atomicAdd(g.b1B + tid * nB + tid, s1B[tid]);
}

// Structural like-particle pairs (same 2M group, at most two particles moved)
// of one species, by target, as local source indices.
// Inclusive sum of v over the lanes of this lane's cluster (a contiguous
// lane range starting at s0) up to this lane.
__device__ __forceinline__ double seg_scan(double v, int lane, int s0) {
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane - o >= s0) v += t;
  }
  return v;
}

// grad_row for several level clusters at once: the lanes (vectors) of a
// cluster are summed per element, and the cluster's last lane adds the sum
// to the cluster's own bins (offset boff from g's bins).
template <typename T>
__device__ void grad_row_cl(const DevH<T>& h, const GradTables& g, const T* __restrict__ X, int64_t ldx, int nvec,
                            int64_t r, int lane, int s0, bool tail, size_t boff) {
  int lo = 0, hi = h.nblk - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (h.boff[mid] <= r)
      lo = mid;
    else
      hi = mid - 1;
  }
  const int blk = lo;
  const int64_t off = h.boff[blk];
  const int nb = h.bnb[blk];
  const int iA = int((r - off) / nb), iB = int((r - off) - int64_t(iA) * nb);
  const int gA0 = h.bgA[blk], gB0 = h.bgB[blk];
  const int pA = gA0 + iA, pB = gB0 + iB;
  const double xr = lane < nvec ? double(X[r * ldx + lane]) : 0.0;
  const int nB = h.nB, nB2 = nB * nB, ND = h.ND;
  for (int di = 0; di < ND; ++di) {
    const int sb = h.srcblk[blk * ND + di];
    if (sb < 0) continue;
    const int pb = h.jsegA[int64_t(pA) * ND + di], pe = h.jsegA[int64_t(pA) * ND + di + 1];
    const int dn = ND - 1 - di;
    const int nbg = h.jsegB[int64_t(pB) * ND + dn], ne = h.jsegB[int64_t(pB) * ND + dn + 1];
    if (pb == pe || nbg == ne) continue;
    const int64_t soff = h.boff[sb];
    const int snb = h.bnb[sb];
    for (int ep = pb; ep < pe; ++ep) {
      const int2 ja = h.jA[ep];
      const int64_t rowA = soff + int64_t(ja.x) * snb;
      for (int en = nbg; en < ne; ++en) {
        const int2 jb = h.jB[en];
        const int64_t src = rowA + jb.x;
        const double xs = lane < nvec ? double(X[src * ldx + lane]) : 0.0;
        const double d = seg_scan(xr * xs, lane, s0);
        if (tail) atomicAdd(g.bAB + boff + int64_t(ja.y >> 1) * nB2 + (jb.y >> 1), ((ja.y ^ jb.y) & 1) ? -d : d);
      }
    }
  }
  const uint32_t tA = g.bitsA[pA];
  for (int e = g.pA_off[pA]; e < g.pA_off[pA + 1]; ++e) {
    const int sA = g.pA_src[e];
    const int64_t src = off + int64_t(sA) * nb + iB;
    const double xs = lane < nvec ? double(X[src * ldx + lane]) : 0.0;
    const double d = seg_scan(xr * xs, lane, s0);
    if (tail) add_like_terms(tA, g.bitsA[gA0 + sA], h.nA, d, g.b1A + boff, g.b2A + boff, nullptr, nullptr);
  }
  const uint32_t tB = g.bitsB[pB];
  for (int e = g.pB_off[pB]; e < g.pB_off[pB + 1]; ++e) {
    const int sB = g.pB_src[e];
    const int64_t src = off + int64_t(iA) * nb + sB;
    const double xs = lane < nvec ? double(X[src * ldx + lane]) : 0.0;
    const double d = seg_scan(xr * xs, lane, s0);
    if (tail) add_like_terms(tB, g.bitsB[gB0 + sB], h.nB, d, g.b1B + boff, g.b2B + boff, nullptr, nullptr);
  }
}

// Lane ranges of the level clusters: cluster c holds lanes first[c] ..
// first[c + 1] - 1.
struct ClusterMap {
  int first[33];
  int ncl;
};

// Persistent blocks of 8 warps, a warp per row at a time; each cluster's
// bins are nbins doubles after the previous cluster's.
template <typename T>
__global__ void __launch_bounds__(256) grad_cluster_kernel(DevH<T> h, GradTables g, const T* __restrict__ X,
                                                           int64_t ldx, int nvec, int64_t D, ClusterMap cm,
                                                           int64_t nbins) {
  const int tid = threadIdx.x, lane = tid & 31;
  int cid = 0;
  while (cid + 1 < cm.ncl && cm.first[cid + 1] <= lane) ++cid;
  const bool valid = lane < nvec;
  const int s0 = valid ? cm.first[cid] : lane;
  const bool tail = valid && lane == cm.first[cid + 1] - 1;
  const size_t boff = size_t(cid) * size_t(nbins);
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t r = int64_t(blockIdx.x) * wpb + (tid >> 5); r < D; r += int64_t(gridDim.x) * wpb)
    grad_row_cl<T>(h, g, X, ldx, nvec, r, lane, s0, tail, boff);
}

void like_pairs(const Species& S, std::vector<int32_t>* off, std::vector<int32_t>* src) {
  const size_t N = S.bits.size();
  off->assign(N + 1, 0);
  src->clear();
  for (size_t t = 0; t < N; ++t) {
    (*off)[t] = int32_t(src->size());
    const int g = S.group[t];
    const int f = S.gfirst[g], c = S.gcount[g];
    for (int i = 0; i < c; ++i)
      if (__builtin_popcount(S.bits[t] ^ S.bits[f + i]) <= 4) src->push_back(i);
  }
  (*off)[N] = int32_t(src->size());
}

struct GradState {
  void* arena = nullptr;
  GradTables g{};
  size_t nbins = 0;
  double* cbins = nullptr;  // per-cluster bins of trbl_grad_clusters
  size_t cbins_cap = 0;     // doubles
  ~GradState() {
    if (arena) cudaFree(arena);
    if (cbins) cudaFree(cbins);
  }
};

// Canonical parameter list of one like species (one-body a <= c with equal
// 2m; two-body pairs I = (i<j) lexicographic, J >= I with equal pair 2m) and
// of the cross species ((a, b) a-major): same order as the input generator
// and the oracle.
template <typename F1, typename F2>
void for_like_params(const std::vector<int>& m, F1 one, F2 two) {
  const int n = int(m.size());
  for (int a = 0; a < n; ++a)
    for (int c = a; c < n; ++c)
      if (m[a] == m[c]) one(a, c);
  std::vector<std::pair<int, int>> pairs;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) pairs.push_back({i, j});
  const size_t P = pairs.size();
  for (size_t I = 0; I < P; ++I)
    for (size_t J = I; J < P; ++J)
      if (m[pairs[I].first] + m[pairs[I].second] == m[pairs[J].first] + m[pairs[J].second])
        two(pairs[I].first, pairs[I].second, pairs[J].first, pairs[J].second);
}

}  // namespace
}  // namespace trbl

using namespace trbl;

namespace {

int64_t count_params(const trbl_basis* b) {
  int64_t n = 0;
  for (int s = 0; s < 2; ++s) for_like_params(b->sp[s].twom, [&](int, int) { ++n; }, [&](int, int, int, int) { ++n; });
  const auto& mA = b->sp[0].twom;
  const auto& mB = b->sp[1].twom;
  const int nA = int(mA.size()), nB = int(mB.size());
  const int P = nA * nB;
  for (int I = 0; I < P; ++I)
    for (int J = I; J < P; ++J)
      if (mA[I / nB] + mB[I % nB] == mA[J / nB] + mB[J % nB]) ++n;
  return n;
}

}  // namespace

namespace {

// Term bins (one-body a c, two-body (a b)(c d), cross (a c)(b d)) folded into
// the canonical parameter order: a parameter at slot (I, J), I != J,
// multiplies both the term (I, J) and its conjugate (J, I).
void fold_bins(const trbl_basis* b, const double* bins, double* dtheta) {
  const Species& A = b->sp[0];
  const Species& B = b->sp[1];
  const int nA = A.n, nB = B.n;
  const size_t n1A = size_t(nA) * nA, n1B = size_t(nB) * nB;
  const double* b1A = bins;
  const double* b1B = b1A + n1A;
  const double* b2A = b1B + n1B;
  const double* b2B = b2A + n1A * n1A;
  const double* bAB = b2B + n1B * n1B;
  int64_t p = 0;
  // one-body A, one-body B, then AA, BB, AB (the generator's order)
  for_like_params(A.twom, [&](int a, int c) { dtheta[p++] = b1A[a * nA + c] + (a != c ? b1A[c * nA + a] : 0.0); },
                  [&](int, int, int, int) {});
  for_like_params(B.twom, [&](int a, int c) { dtheta[p++] = b1B[a * nB + c] + (a != c ? b1B[c * nB + a] : 0.0); },
                  [&](int, int, int, int) {});
  auto two_like = [&](const double* b2, int n) {
    return [&, b2, n](int i, int j, int k, int l) {
      const double v = b2[((size_t(i) * n + j) * n + k) * n + l];
      const bool same = (i == k && j == l);
      dtheta[p++] = v + (same ? 0.0 : b2[((size_t(k) * n + l) * n + i) * n + j]);
    };
  };
  for_like_params(A.twom, [&](int, int) {}, two_like(b2A, nA));
  for_like_params(B.twom, [&](int, int) {}, two_like(b2B, nB));
  const int P = nA * nB, nB2 = nB * nB;
  for (int I = 0; I < P; ++I)
    for (int J = I; J < P; ++J) {
      const int a = I / nB, bb = I % nB, c = J / nB, d = J % nB;
      if (A.twom[a] + B.twom[bb] != A.twom[c] + B.twom[d]) continue;
      const double v = bAB[size_t(a * nA + c) * nB2 + bb * nB + d];
      dtheta[p++] = v + (I == J ? 0.0 : bAB[size_t(c * nA + a) * nB2 + d * nB + bb]);
    }
}

// One-time device tables of the gradient kernels, kept with the Hamiltonian:
// bit strings, structural like-particle pairs, and one set of FP64 bins.
int ensure_grad_state(trbl_hamiltonian* h) {
  if (h->grad) return TRBL_OK;
  const trbl_basis* b = h->b;
  const Species& A = b->sp[0];
  const Species& B = b->sp[1];
  const int nA = A.n, nB = B.n;
    // one-time tables: bit strings and structural like-particle pairs
    auto* st = new (std::nothrow) GradState();
    if (!st) return fail(TRBL_ERR_OOM, "host allocation failed");
    std::vector<int32_t> oA, sA, oB, sB;
    like_pairs(A, &oA, &sA);
    like_pairs(B, &oB, &sB);
    const size_t n1A = size_t(nA) * nA, n1B = size_t(nB) * nB;
    const size_t n2A = n1A * n1A, n2B = n1B * n1B, nAB = n1A * n1B;
    st->nbins = n1A + n1B + n2A + n2B + nAB;
    size_t bytes = 0;
    auto take = [&](size_t nb) {
      size_t o = (bytes + 255) & ~size_t(255);
      bytes = o + nb;
      return o;
    };
    const size_t o_bins = take(st->nbins * 8), o_bA = take(A.bits.size() * 4), o_bB = take(B.bits.size() * 4);
    const size_t o_oA = take(oA.size() * 4), o_sA = take(std::max<size_t>(sA.size(), 1) * 4);
    const size_t o_oB = take(oB.size() * 4), o_sB = take(std::max<size_t>(sB.size(), 1) * 4);
    cudaError_t e = cudaMalloc(&st->arena, bytes);
    if (e != cudaSuccess) {
      delete st;
      return cuda_fail(e, "cudaMalloc(gradient tables)");
    }
    char* base = static_cast<char*>(st->arena);
    auto put = [&](size_t o, const void* p, size_t n) { return cudaMemcpy(base + o, p, n, cudaMemcpyHostToDevice); };
    if (put(o_bA, A.bits.data(), A.bits.size() * 4) || put(o_bB, B.bits.data(), B.bits.size() * 4) ||
        put(o_oA, oA.data(), oA.size() * 4) || (sA.size() && put(o_sA, sA.data(), sA.size() * 4)) ||
        put(o_oB, oB.data(), oB.size() * 4) || (sB.size() && put(o_sB, sB.data(), sB.size() * 4))) {
      delete st;
      return fail(TRBL_ERR_CUDA, "upload of gradient tables failed");
    }
    double* bins = reinterpret_cast<double*>(base + o_bins);
    st->g.bitsA = reinterpret_cast<const uint32_t*>(base + o_bA);
    st->g.bitsB = reinterpret_cast<const uint32_t*>(base + o_bB);
    st->g.pA_off = reinterpret_cast<const int32_t*>(base + o_oA);
    st->g.pA_src = reinterpret_cast<const int32_t*>(base + o_sA);
    st->g.pB_off = reinterpret_cast<const int32_t*>(base + o_oB);
    st->g.pB_src = reinterpret_cast<const int32_t*>(base + o_sB);
    st->g.b1A = bins;
    st->g.b1B = st->g.b1A + n1A;
    st->g.b2A = st->g.b1B + n1B;
    st->g.b2B = st->g.b2A + n2A;
    st->g.bAB = st->g.b2B + n2B;
    h->grad = st;
  return TRBL_OK;
}

}  // namespace

extern "C" int trbl_param_count(const trbl_basis* b, int64_t* n) {
  clear_error();
  if (!b || !n) return fail(TRBL_ERR_ARG, "null argument");
  *n = count_params(b);
  return TRBL_OK;
}

extern "C" int trbl_grad(const trbl_hamiltonian* hc, const void* X, int64_t ldx, int nvec, int dtype,
                         double* dtheta, int64_t nparams, void* stream) {
  clear_error();
  if (!hc || !X || !dtheta) return fail(TRBL_ERR_ARG, "null argument");
  if (nvec < 1 || nvec > 32 || ldx < nvec) return fail(TRBL_ERR_ARG, "need 1 <= nvec <= 32 and ldx >= nvec");
  if (dtype != TRBL_F32 && dtype != TRBL_F64) return fail(TRBL_ERR_ARG, "bad dtype %d", dtype);
  trbl_hamiltonian* h = const_cast<trbl_hamiltonian*>(hc);
  const trbl_basis* b = h->b;
  const int64_t np = count_params(b);
  if (nparams != np) return fail(TRBL_ERR_ARG, "nparams=%lld, the spaces have %lld", (long long)nparams, (long long)np);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  {
    const int rc = ensure_grad_state(h);
    if (rc) return rc;
  }
  GradState* st = static_cast<GradState*>(h->grad);
  TRBL_CUDA(cudaMemsetAsync(st->g.b1A, 0, st->nbins * 8, s));
  const int64_t D = b->D;
  static const int sms = [] {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 148;
  }();
  const unsigned grid = unsigned(std::max<int64_t>(1, std::min<int64_t>((D + 7) / 8, int64_t(4) * sms)));
  if (dtype == TRBL_F64)
    grad_kernel<double><<<grid, 256, 0, s>>>(h->d64, st->g, static_cast<const double*>(X), ldx, nvec, D);
  else
    grad_kernel<float><<<grid, 256, 0, s>>>(h->d32, st->g, static_cast<const float*>(X), ldx, nvec, D);
  note_launch();
  TRBL_CUDA(cudaGetLastError());
  std::vector<double> bins(st->nbins);
  TRBL_CUDA(cudaMemcpyAsync(bins.data(), st->g.b1A, st->nbins * 8, cudaMemcpyDeviceToHost, s));
  TRBL_CUDA(cudaStreamSynchronize(s));
  fold_bins(b, bins.data(), dtheta);
  return TRBL_OK;
}

extern "C" int trbl_grad_clusters(const trbl_hamiltonian* hc, const void* X, int64_t ldx, int nvec, int dtype,
                                  const int* first, int ncl, double* dtheta, int64_t nparams, void* stream) {
  clear_error();
  if (!hc || !X || !dtheta || !first) return fail(TRBL_ERR_ARG, "null argument");
  if (nvec < 1 || nvec > 32 || ldx < nvec) return fail(TRBL_ERR_ARG, "need 1 <= nvec <= 32 and ldx >= nvec");
  if (dtype != TRBL_F32 && dtype != TRBL_F64) return fail(TRBL_ERR_ARG, "bad dtype %d", dtype);
  if (ncl < 1 || ncl > nvec) return fail(TRBL_ERR_ARG, "need 1 <= ncl <= nvec");
  if (first[0] != 0 || first[ncl] != nvec) return fail(TRBL_ERR_ARG, "first[0] must be 0 and first[ncl] nvec");
  ClusterMap cm{};
  cm.ncl = ncl;
  for (int c = 0; c <= ncl; ++c) {
    if (c > 0 && first[c] <= first[c - 1]) return fail(TRBL_ERR_ARG, "cluster boundaries must increase");
    cm.first[c] = first[c];
  }
  trbl_hamiltonian* h = const_cast<trbl_hamiltonian*>(hc);
  const trbl_basis* b = h->b;
  const int64_t np = count_params(b);
  if (nparams != np) return fail(TRBL_ERR_ARG, "nparams=%lld, the spaces have %lld", (long long)nparams, (long long)np);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  {
    const int rc = ensure_grad_state(h);
    if (rc) return rc;
  }
  GradState* st = static_cast<GradState*>(h->grad);
  const size_t need = st->nbins * size_t(ncl);
  if (need > st->cbins_cap) {
    if (st->cbins) {
      TRBL_CUDA(cudaStreamSynchronize(s));
      cudaFree(st->cbins);
      st->cbins = nullptr;
      st->cbins_cap = 0;
    }
    cudaError_t e = cudaMalloc(&st->cbins, need * 8);
    if (e != cudaSuccess) {
      cudaGetLastError();
      st->cbins = nullptr;
      return fail(TRBL_ERR_OOM, "cluster gradient bins of %.1f MB: %s", need * 8 / 1e6, cudaGetErrorString(e));
    }
    st->cbins_cap = need;
  }
  TRBL_CUDA(cudaMemsetAsync(st->cbins, 0, need * 8, s));
  GradTables gc = st->g;  // same tables, bins of cluster 0 at cbins
  gc.b1A = st->cbins;
  gc.b1B = st->cbins + (st->g.b1B - st->g.b1A);
  gc.b2A = st->cbins + (st->g.b2A - st->g.b1A);
  gc.b2B = st->cbins + (st->g.b2B - st->g.b1A);
  gc.bAB = st->cbins + (st->g.bAB - st->g.b1A);
  const int64_t D = b->D;
  static const int sms = [] {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 148;
  }();
  const unsigned grid = unsigned(std::max<int64_t>(1, std::min<int64_t>((D + 7) / 8, int64_t(4) * sms)));
  if (dtype == TRBL_F64)
    grad_cluster_kernel<double><<<grid, 256, 0, s>>>(h->d64, gc, static_cast<const double*>(X), ldx, nvec, D, cm,
                                                     int64_t(st->nbins));
  else
    grad_cluster_kernel<float><<<grid, 256, 0, s>>>(h->d32, gc, static_cast<const float*>(X), ldx, nvec, D, cm,
                                                    int64_t(st->nbins));
  note_launch();
  TRBL_CUDA(cudaGetLastError());
  std::vector<double> bins(need);
  TRBL_CUDA(cudaMemcpyAsync(bins.data(), st->cbins, need * 8, cudaMemcpyDeviceToHost, s));
  TRBL_CUDA(cudaStreamSynchronize(s));
  for (int c = 0; c < ncl; ++c) fold_bins(b, bins.data() + size_t(c) * st->nbins, dtheta + size_t(c) * nparams);
  return TRBL_OK;
}

void trbl_grad_state_free(void* g) { delete static_cast<GradState*>(g); }
