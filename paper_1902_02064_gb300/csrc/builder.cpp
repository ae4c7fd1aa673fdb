// Host-side builder: determinant enumeration, product blocks, one-body jump
// lists and like-particle Hamiltonian rows.
//
// - Determinants are bit strings (Sec. II Eq. (mbasis), App. A Table I).
// - The basis is the proton x neutron factorisation of App. A Eq. (part),
//   blocked by 2M_A.
// - One-body jumps a+_a a_c |S> (App. B.2) are stored gathered by target
//   determinant and 2m transfer, so the apply kernels read, for one output
//   row, every source that feeds it without atomics.
// - Like-particle rows (App. B.1) sum every one- and two-body term that links
//   two determinants of the same species into one coefficient; the paper
//   locates the target by binary search (App. B.1), which is what `find`
//   does here, once, at build time.
#include <algorithm>
#include <cmath>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>

#include "internal.h"

namespace trbl {

static thread_local std::string g_err;
static std::atomic<long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

void clear_error() { g_err.clear(); }

int cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? TRBL_ERR_OOM : TRBL_ERR_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

int Species::group_of_M(int M) const {
  auto it = std::lower_bound(gM.begin(), gM.end(), M);
  if (it == gM.end() || *it != M) return -1;
  return int(it - gM.begin());
}

int Species::find(uint32_t b, int M) const {
  int g = group_of_M(M);
  if (g < 0) return -1;
  auto first = bits.begin() + gfirst[g];
  auto last = first + gcount[g];
  auto it = std::lower_bound(first, last, b);
  if (it == last || *it != b) return -1;
  return int(it - bits.begin());
}

// Sign of a+_a a_c acting on s (a_c first); 0 when the result vanishes.
static int one_body_sign(uint32_t s, int a, int c, uint32_t* out) {
  uint64_t t = s;
  int sg = 1;
  if (!(t >> c & 1)) return 0;
  if (__builtin_popcountll(t & ((1ull << c) - 1)) & 1) sg = -sg;
  t ^= 1ull << c;
  if (t >> a & 1) return 0;
  if (__builtin_popcountll(t & ((1ull << a) - 1)) & 1) sg = -sg;
  t |= 1ull << a;
  *out = uint32_t(t);
  return sg;
}

// Sign of x+_a x+_b x_d x_c acting on s (x_c first); 0 when it vanishes.
static int two_body_sign(uint32_t s, int a, int b, int c, int d, uint32_t* out) {
  uint64_t t = s;
  int sg = 1;
  const int ops[4] = {c, d, b, a};
  for (int i = 0; i < 4; ++i) {
    int x = ops[i];
    bool create = i >= 2;
    bool occ = t >> x & 1;
    if (create == occ) return 0;
    if (__builtin_popcountll(t & ((1ull << x) - 1)) & 1) sg = -sg;
    t ^= 1ull << x;
  }
  *out = uint32_t(t);
  return sg;
}

static int build_species(const trbl_space* s, Species* sp) {
  if (!s || !s->twom) return fail(TRBL_ERR_ARG, "null species description");
  if (s->n_states < 1 || s->n_states > 32)
    return fail(TRBL_ERR_ARG, "n_states=%d outside [1, 32]", s->n_states);
  if (s->n_particles < 0 || s->n_particles > s->n_states)
    return fail(TRBL_ERR_ARG, "n_particles=%d outside [0, %d]", s->n_particles, s->n_states);
  sp->n = s->n_states;
  sp->k = s->n_particles;
  sp->twom.assign(s->twom, s->twom + s->n_states);
  // Enumerate k-subsets in increasing bit-string value (Gosper's hack).
  std::vector<std::pair<int, uint32_t>> dets;
  const int n = sp->n, k = sp->k;
  if (k == 0) {
    dets.push_back({0, 0u});
  } else {
    uint64_t x = (1ull << k) - 1, lim = 1ull << n;
    while (x < lim) {
      int M = 0;
      for (int i = 0; i < n; ++i)
        if (x >> i & 1) M += sp->twom[i];
      dets.push_back({M, uint32_t(x)});
      uint64_t c = x & (~x + 1), r = x + c;
      x = (((r ^ x) >> 2) / c) | r;
      if (dets.size() > (size_t(1) << 30)) return fail(TRBL_ERR_ARG, "species space too large");
    }
  }
  std::stable_sort(dets.begin(), dets.end(),
                   [](const std::pair<int, uint32_t>& p, const std::pair<int, uint32_t>& q) {
                     return p.first < q.first;
                   });
  const size_t N = dets.size();
  sp->bits.resize(N);
  sp->dM.resize(N);
  sp->group.resize(N);
  for (size_t i = 0; i < N; ++i) {
    sp->bits[i] = dets[i].second;
    sp->dM[i] = dets[i].first;
    if (i == 0 || dets[i].first != dets[i - 1].first) {
      sp->gM.push_back(dets[i].first);
      sp->gfirst.push_back(int32_t(i));
      sp->gcount.push_back(0);
    }
    sp->gcount.back()++;
    sp->group[i] = int32_t(sp->gM.size() - 1);
  }
  return TRBL_OK;
}

// Incoming one-body jumps of every target determinant, ordered by
// (2m transfer, source, a).
static void build_jumps(Species* sp, int dspan, int ND) {
  const int n = sp->n;
  const size_t N = sp->bits.size();
  sp->jseg.assign(N * ND + 1, 0);
  sp->jsrc.clear();
  sp->ja.clear();
  sp->jc.clear();
  sp->jsign.clear();
  struct E {
    int di, src, a, c, sg;
  };
  std::vector<E> es;
  for (size_t t = 0; t < N; ++t) {
    es.clear();
    uint32_t tb = sp->bits[t];
    for (int a = 0; a < n; ++a) {
      if (!(tb >> a & 1)) continue;
      for (int c = 0; c < n; ++c) {
        if (c != a && (tb >> c & 1)) continue;
        uint32_t sb = (tb & ~(1u << a)) | (1u << c);
        int Ms = sp->dM[t] - sp->twom[a] + sp->twom[c];
        int src = sp->find(sb, Ms);
        uint32_t chk = 0;
        int sg = one_body_sign(sb, a, c, &chk);
        // src always exists: every k-subset is a determinant.
        es.push_back({sp->twom[a] - sp->twom[c] + dspan, src, a, c, sg});
        (void)chk;
      }
    }
    std::sort(es.begin(), es.end(), [](const E& x, const E& y) {
      if (x.di != y.di) return x.di < y.di;
      if (x.src != y.src) return x.src < y.src;
      return x.a < y.a;
    });
    size_t base = sp->jsrc.size();
    size_t e = 0;
    for (int di = 0; di < ND; ++di) {
      sp->jseg[t * ND + di] = int32_t(base + e);
      while (e < es.size() && es[e].di == di) {
        sp->jsrc.push_back(es[e].src);
        sp->ja.push_back(es[e].a);
        sp->jc.push_back(es[e].c);
        sp->jsign.push_back(int8_t(es[e].sg));
        ++e;
      }
    }
  }
  sp->jseg[N * ND] = int32_t(sp->jsrc.size());
}

}  // namespace trbl

using namespace trbl;

extern "C" const char* trbl_last_error(void) { return g_err.c_str(); }

extern "C" long long trbl_kernel_launches(void) { return g_launches.load(); }

extern "C" int trbl_basis_create(const trbl_space* A, const trbl_space* B, int twoM,
                                 trbl_basis** out) {
  clear_error();
  if (!out) return fail(TRBL_ERR_ARG, "out is null");
  *out = nullptr;
  trbl_basis* b = new (std::nothrow) trbl_basis();
  if (!b) return fail(TRBL_ERR_OOM, "host allocation failed");
  int rc = build_species(A, &b->sp[0]);
  if (rc == TRBL_OK) rc = build_species(B, &b->sp[1]);
  if (rc != TRBL_OK) {
    delete b;
    return rc;
  }
  b->twoM = twoM;
  int span = 0;
  for (int s = 0; s < 2; ++s) {
    const auto& tm = b->sp[s].twom;
    int lo = *std::min_element(tm.begin(), tm.end()), hi = *std::max_element(tm.begin(), tm.end());
    span = std::max(span, hi - lo);
  }
  b->dspan = span;
  b->ND = 2 * span + 1;
  const Species& SA = b->sp[0];
  const Species& SB = b->sp[1];
  int64_t off = 0;
  for (size_t g = 0; g < SA.gM.size(); ++g) {
    int mB = twoM - SA.gM[g];
    int gb = SB.group_of_M(mB);
    if (gb < 0) continue;
    Block bl{SA.gM[g], mB, off, SA.gcount[g], SB.gcount[gb], int(g), gb};
    b->blocks.push_back(bl);
    off += int64_t(bl.na) * bl.nb;
  }
  b->D = off;
  if (b->D == 0) {
    delete b;
    return fail(TRBL_ERR_ARG, "empty basis for 2M=%d", twoM);
  }
  if (b->D > (int64_t(1) << 40)) {
    delete b;
    return fail(TRBL_ERR_ARG, "dimension too large");
  }
  const int nblk = int(b->blocks.size());
  b->srcblk.assign(size_t(nblk) * b->ND, -1);
  for (int k = 0; k < nblk; ++k)
    for (int di = 0; di < b->ND; ++di) {
      int mA = b->blocks[k].mA - (di - span);
      for (int j = 0; j < nblk; ++j)
        if (b->blocks[j].mA == mA) b->srcblk[size_t(k) * b->ND + di] = j;
    }
  for (int s = 0; s < 2; ++s)
    for (int c : b->sp[s].gcount) b->max_group = std::max(b->max_group, c);
  build_jumps(&b->sp[0], span, b->ND);
  build_jumps(&b->sp[1], span, b->ND);
  *out = b;
  return TRBL_OK;
}

extern "C" void trbl_basis_destroy(trbl_basis* b) { delete b; }

extern "C" int trbl_basis_info(const trbl_basis* b, trbl_basis_sizes* s) {
  clear_error();
  if (!b || !s) return fail(TRBL_ERR_ARG, "null argument");
  s->dim = b->D;
  s->n_det[0] = int32_t(b->sp[0].bits.size());
  s->n_det[1] = int32_t(b->sp[1].bits.size());
  s->n_blocks = int32_t(b->blocks.size());
  s->n_jumps[0] = int64_t(b->sp[0].jsrc.size());
  s->n_jumps[1] = int64_t(b->sp[1].jsrc.size());
  s->n_delta = b->ND;
  return TRBL_OK;
}

extern "C" int trbl_basis_export(const trbl_basis* b, uint32_t* bitsA, int32_t* twoMA,
                                 uint32_t* bitsB, int32_t* twoMB, int64_t* blocks) {
  clear_error();
  if (!b) return fail(TRBL_ERR_ARG, "null basis");
  const Species& A = b->sp[0];
  const Species& B = b->sp[1];
  if (bitsA) std::copy(A.bits.begin(), A.bits.end(), bitsA);
  if (twoMA) std::copy(A.dM.begin(), A.dM.end(), twoMA);
  if (bitsB) std::copy(B.bits.begin(), B.bits.end(), bitsB);
  if (twoMB) std::copy(B.dM.begin(), B.dM.end(), twoMB);
  if (blocks) {
    for (size_t k = 0; k < b->blocks.size(); ++k) {
      const Block& bl = b->blocks[k];
      int64_t* r = blocks + 7 * k;
      r[0] = bl.mA;
      r[1] = bl.mB;
      r[2] = bl.off;
      r[3] = bl.na;
      r[4] = bl.nb;
      r[5] = A.gfirst[bl.gA];
      r[6] = B.gfirst[bl.gB];
    }
  }
  return TRBL_OK;
}

extern "C" int trbl_basis_export_jumps(const trbl_basis* b, int species, int32_t* tgt,
                                       int32_t* src, int32_t* a, int32_t* c, int8_t* sign) {
  clear_error();
  if (!b || species < 0 || species > 1) return fail(TRBL_ERR_ARG, "bad basis or species");
  const Species& S = b->sp[species];
  const size_t N = S.bits.size();
  for (size_t t = 0; t < N; ++t)
    for (int32_t e = S.jseg[t * b->ND]; e < S.jseg[(t + 1) * b->ND]; ++e) {
      if (tgt) tgt[e] = int32_t(t);
      if (src) src[e] = S.jsrc[e];
      if (a) a[e] = S.ja[e];
      if (c) c[e] = S.jc[e];
      if (sign) sign[e] = S.jsign[e];
    }
  return TRBL_OK;
}

// Like-particle rows of one species: every one-body term h1[a][c] and
// two-body term V[a][b][c][d] (a<b, c<d) applied to every determinant,
// accumulated per (target, source) and ordered by target.
static void like_rows(const Species& S, const double* h1, const double* V, std::vector<int32_t>* off,
                      std::vector<int32_t>* src, std::vector<double>* coef) {
  const int n = S.n;
  const size_t N = S.bits.size();
  std::vector<std::map<int32_t, double>> rows(N);  // rows[target][source]
  for (size_t s = 0; s < N; ++s) {
    const uint32_t sb = S.bits[s];
    const int Ms = S.dM[s];
    for (int c = 0; c < n; ++c) {
      if (!(sb >> c & 1)) continue;
      for (int a = 0; a < n; ++a) {
        double h = h1[a * n + c];
        if (h == 0.0 || S.twom[a] != S.twom[c]) continue;
        uint32_t tb;
        int sg = one_body_sign(sb, a, c, &tb);
        if (!sg) continue;
        int t = S.find(tb, Ms);
        rows[t][int32_t(s)] += sg * h;
      }
    }
    for (int c = 0; c < n; ++c) {
      if (!(sb >> c & 1)) continue;
      for (int d = c + 1; d < n; ++d) {
        if (!(sb >> d & 1)) continue;
        const int mcd = S.twom[c] + S.twom[d];
        for (int a = 0; a < n; ++a)
          for (int bb = a + 1; bb < n; ++bb) {
            if (S.twom[a] + S.twom[bb] != mcd) continue;
            double v = V[((size_t(a) * n + bb) * n + c) * n + d];
            if (v == 0.0) continue;
            uint32_t tb;
            int sg = two_body_sign(sb, a, bb, c, d, &tb);
            if (!sg) continue;
            int t = S.find(tb, Ms);
            rows[t][int32_t(s)] += sg * v;
          }
      }
    }
  }
  off->assign(N + 1, 0);
  src->clear();
  coef->clear();
  for (size_t t = 0; t < N; ++t) {
    (*off)[t] = int32_t(src->size());
    const int32_t g0 = S.gfirst[S.group[t]];
    for (auto& kv : rows[t]) {
      src->push_back(kv.first - g0);  // local index inside the (shared) 2M group
      coef->push_back(kv.second);
    }
  }
  (*off)[N] = int32_t(src->size());
}

extern "C" int trbl_hamiltonian_create(const trbl_basis* b, const double* h1A, const double* h1B,
                                       const double* VAA, const double* VBB, const double* VAB,
                                       trbl_hamiltonian** out) {
  clear_error();
  if (!out) return fail(TRBL_ERR_ARG, "out is null");
  *out = nullptr;
  if (!b || !h1A || !h1B || !VAA || !VBB || !VAB) return fail(TRBL_ERR_ARG, "null argument");
  {
    const size_t nA = size_t(b->sp[0].n), nB = size_t(b->sp[1].n);
    const struct {
      const double* x;
      size_t n;
      const char* name;
    } arrays[] = {{h1A, nA * nA, "h1A"}, {h1B, nB * nB, "h1B"}, {VAA, nA * nA * nA * nA, "VAA"},
                  {VBB, nB * nB * nB * nB, "VBB"}, {VAB, nA * nB * nA * nB, "VAB"}};
    for (const auto& a : arrays)
      for (size_t i = 0; i < a.n; ++i)
        if (!std::isfinite(a.x[i])) return fail(TRBL_ERR_ARG, "%s[%zu] is not finite", a.name, i);
  }
  trbl_hamiltonian* h = new (std::nothrow) trbl_hamiltonian();
  if (!h) return fail(TRBL_ERR_OOM, "host allocation failed");
  h->b = b;
  like_rows(b->sp[0], h1A, VAA, &h->hoff[0], &h->hsrc[0], &h->hcoef[0]);
  like_rows(b->sp[1], h1B, VBB, &h->hoff[1], &h->hsrc[1], &h->hcoef[1]);
  const int nA = b->sp[0].n, nB = b->sp[1].n;
  const auto& mA = b->sp[0].twom;
  const auto& mB = b->sp[1].twom;
  h->vab.assign(size_t(nA) * nA * nB * nB, 0.0);
  for (int a = 0; a < nA; ++a)
    for (int c = 0; c < nA; ++c)
      for (int bb = 0; bb < nB; ++bb)
        for (int d = 0; d < nB; ++d) {
          if (mA[a] + mB[bb] != mA[c] + mB[d]) continue;
          h->vab[(size_t(a) * nA + c) * nB * nB + size_t(bb) * nB + d] =
              VAB[((size_t(a) * nB + bb) * nA + c) * nB + d];
        }
  int rc = upload_tables(h);
  if (rc != TRBL_OK) {
    delete h;
    return rc;
  }
  *out = h;
  return TRBL_OK;
}

extern "C" void trbl_hamiltonian_destroy(trbl_hamiltonian* h) {
  if (!h) return;
  if (h->arena || h->garena || h->grad || h->gwork || h->pnarena || h->pnslabs) cudaDeviceSynchronize();
  if (h->gwork) cudaFree(h->gwork);
  if (h->pnslabs) cudaFree(h->pnslabs);
  if (h->pnarena) cudaFree(h->pnarena);
  if (h->grad) trbl_grad_state_free(h->grad);
  if (h->arena) cudaFree(h->arena);
  if (h->garena) cudaFree(h->garena);
  delete h;
}
