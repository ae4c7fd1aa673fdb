// Row sharding of the block product over several GPUs: the single-node
// form of the paper's distributed matrix-vector product (App. C, the 2-D
// distribution with shifts and reductions), recast for GPUs that each hold
// a copy of the tables.
//
// * Rows of W are split into contiguous ranges of whole target slabs (all
//   rows (pA', nB') of one proton determinant pA'), balanced by the number
//   of elements the product generates for them.  The estimate counts, for
//   every row, the cross-term elements exactly (incoming proton jumps of
//   each 2m transfer times incoming neutron jumps of the opposite one, App.
//   B.2) plus one for the row's like-particle and diagonal work.
// * A shard's targets read the slabs of their source proton determinants:
//   the target itself (species-B like-particle rows, diagonal), its
//   one-body-jump sources (the cross term) and its like-particle sources
//   (at most two protons moved, same 2M_A).  trbl_shard_sources lists those
//   slabs as merged row ranges: the V rows a shard must receive before its
//   product (an all-gather of V slices, or only these ranges).
// * trbl_hamiltonian_set_rows restricts a Hamiltonian's product to one
//   shard's rows; the projections are sharded by the same rows and summed
//   across shards (an all-reduce of the m x q coefficients).
#include <algorithm>
#include <vector>

#include "internal.h"

using namespace trbl;

namespace {

// Cross-term elements plus one, summed over the rows of target slab
// (block k, local proton index ia).
int64_t slab_work(const trbl_basis* b, int k, int ia) {
  const Species& A = b->sp[0];
  const Species& B = b->sp[1];
  const Block& bl = b->blocks[k];
  const int ND = b->ND;
  const int pA = A.gfirst[bl.gA] + ia;
  std::vector<int> jA(ND, 0);
  for (int di = 0; di < ND; ++di)
    if (b->srcblk[size_t(k) * ND + di] >= 0)
      jA[di] = A.jseg[size_t(pA) * ND + di + 1] - A.jseg[size_t(pA) * ND + di];
  int64_t w = 0;
  const int b0 = B.gfirst[bl.gB];
  for (int ib = 0; ib < bl.nb; ++ib) {
    const int pB = b0 + ib;
    int64_t e = 1;
    for (int dn = 0; dn < ND; ++dn) {
      const int cnt = B.jseg[size_t(pB) * ND + dn + 1] - B.jseg[size_t(pB) * ND + dn];
      if (cnt) e += int64_t(cnt) * jA[ND - 1 - dn];
    }
    w += e;
  }
  return w;
}

// Block and local proton index of the slab that starts at row r, or false.
bool slab_at(const trbl_basis* b, int64_t r, int* k_out, int* ia_out) {
  for (size_t k = 0; k < b->blocks.size(); ++k) {
    const Block& bl = b->blocks[k];
    if (r < bl.off || r >= bl.off + int64_t(bl.na) * bl.nb) continue;
    const int64_t rel = r - bl.off;
    if (rel % bl.nb) return false;
    *k_out = int(k);
    *ia_out = int(rel / bl.nb);
    return true;
  }
  return false;
}

}  // namespace

namespace trbl {
// Whether row r is a slab boundary (r == D counts).
bool is_slab_boundary(const trbl_basis* b, int64_t r) {
  if (r == 0 || r == b->D) return true;
  int k, ia;
  return slab_at(b, r, &k, &ia);
}
}  // namespace trbl

extern "C" int trbl_shard_plan(const trbl_basis* b, int nranks, int64_t* bounds, int64_t* work) {
  clear_error();
  if (!b || !bounds) return fail(TRBL_ERR_ARG, "null argument");
  if (nranks < 1) return fail(TRBL_ERR_ARG, "nranks must be positive");
  // slabs in basis order with their work
  std::vector<int64_t> start, w;
  for (size_t k = 0; k < b->blocks.size(); ++k) {
    const Block& bl = b->blocks[k];
    if (bl.nb == 0) continue;
    for (int ia = 0; ia < bl.na; ++ia) {
      start.push_back(bl.off + int64_t(ia) * bl.nb);
      w.push_back(slab_work(b, int(k), ia));
    }
  }
  const size_t ns = start.size();
  int64_t total = 0;
  for (int64_t x : w) total += x;
  // cut after the slab where the running work first reaches r / nranks of the total
  bounds[0] = 0;
  size_t s = 0;
  int64_t acc = 0;
  for (int r = 1; r < nranks; ++r) {
    const double goal = double(total) * r / nranks;
    while (s < ns && double(acc) + 0.5 * double(w[s]) < goal) acc += w[s++];
    bounds[r] = s < ns ? start[s] : b->D;
  }
  bounds[nranks] = b->D;
  if (work) {
    for (int r = 0; r < nranks; ++r) work[r] = 0;
    int r = 0;
    for (size_t i = 0; i < ns; ++i) {
      while (r + 1 < nranks && start[i] >= bounds[r + 1]) ++r;
      work[r] += w[i];
    }
  }
  return TRBL_OK;
}

extern "C" int trbl_shard_sources(const trbl_basis* b, int64_t row_begin, int64_t row_end, int64_t* ranges,
                                  int64_t cap, int64_t* nranges) {
  clear_error();
  if (!b || !nranges) return fail(TRBL_ERR_ARG, "null argument");
  if (row_begin < 0 || row_end > b->D || row_begin > row_end || !is_slab_boundary(b, row_begin) ||
      !is_slab_boundary(b, row_end))
    return fail(TRBL_ERR_ARG, "rows [%lld, %lld) are not slab boundaries of the basis", (long long)row_begin,
                (long long)row_end);
  const Species& A = b->sp[0];
  const int ND = b->ND;
  std::vector<std::pair<int64_t, int64_t>> slabs;  // [begin, end) rows of source slabs
  auto add_slab = [&](int pA) {
    const int g = A.group[pA];
    for (const Block& bl : b->blocks)
      if (bl.gA == g) {
        const int64_t r0 = bl.off + int64_t(pA - A.gfirst[g]) * bl.nb;
        if (bl.nb) slabs.push_back({r0, r0 + bl.nb});
        return;
      }
  };
  for (size_t k = 0; k < b->blocks.size(); ++k) {
    const Block& bl = b->blocks[k];
    if (bl.nb == 0) continue;
    for (int ia = 0; ia < bl.na; ++ia) {
      const int64_t r0 = bl.off + int64_t(ia) * bl.nb;
      if (r0 < row_begin || r0 >= row_end) continue;
      const int pA = A.gfirst[bl.gA] + ia;
      add_slab(pA);  // species-B like-particle rows and the diagonal
      for (int di = 0; di < ND; ++di) {
        if (b->srcblk[k * ND + di] < 0) continue;
        for (int e = A.jseg[size_t(pA) * ND + di]; e < A.jseg[size_t(pA) * ND + di + 1]; ++e) add_slab(A.jsrc[e]);
      }
      // like-particle sources: same 2M_A, at most two protons moved
      const uint32_t t = A.bits[pA];
      const int g0 = A.gfirst[bl.gA];
      for (int s = g0; s < g0 + A.gcount[bl.gA]; ++s)
        if (__builtin_popcount(A.bits[s] ^ t) <= 4) add_slab(s);
    }
  }
  std::sort(slabs.begin(), slabs.end());
  std::vector<std::pair<int64_t, int64_t>> merged;
  for (const auto& x : slabs) {
    if (!merged.empty() && x.first <= merged.back().second)
      merged.back().second = std::max(merged.back().second, x.second);
    else
      merged.push_back(x);
  }
  *nranges = int64_t(merged.size());
  if (ranges) {
    if (cap < int64_t(merged.size())) return fail(TRBL_ERR_ARG, "%zu ranges do not fit in %lld", merged.size(),
                                                  (long long)cap);
    for (size_t i = 0; i < merged.size(); ++i) {
      ranges[2 * i] = merged[i].first;
      ranges[2 * i + 1] = merged[i].second;
    }
  }
  return TRBL_OK;
}

extern "C" int trbl_hamiltonian_set_rows(trbl_hamiltonian* h, int64_t row_begin, int64_t row_end) {
  clear_error();
  if (!h) return fail(TRBL_ERR_ARG, "null Hamiltonian");
  const trbl_basis* b = h->b;
  if (row_begin < 0 || row_end > b->D || row_begin > row_end || !is_slab_boundary(b, row_begin) ||
      !is_slab_boundary(b, row_end))
    return fail(TRBL_ERR_ARG, "rows [%lld, %lld) are not slab boundaries of the basis", (long long)row_begin,
                (long long)row_end);
  if (!h->garena) return fail(TRBL_ERR_ARG, "the grouped product is not available for this basis");
  h->row_begin = row_begin;
  h->row_end = row_end;
  return set_work_items(h, h->rows_per_item > 0 ? h->rows_per_item : 16);
}
