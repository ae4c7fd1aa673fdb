// Thick-restart block Lanczos solver (Sec. III D, Alg. 4) on one GPU.
//
// Per block step k (Alg. 4 inner loop):
//   W := H V_k                          on-the-fly block product (apply.cu)
//   alpha_k := V_k^T W                  first Gram-Schmidt pass coefficients
//   orthogonalise W against every stored Lanczos vector: classical
//     Gram-Schmidt applied twice (the full reorthogonalisation of Sec. III)
//   V_{k+1} beta_k := QR(W)             Cholesky QR applied twice, FP64 Gram
//   T gets alpha_k on its block diagonal and beta_k below/above it
//     (Eq. (tmat-blan); after a restart the arrow form of Eq. (trb-tmat))
//   Rayleigh-Ritz: eigenpairs (theta_i, U_i) of T; the residual of Ritz
//     pair i is ||beta_k U_{last q rows, i}||
// When the basis would exceed max_basis (l_m) vectors, restart: keep the
// l_s lowest Ritz vectors v_i := sum_j v_j U_ji, put V_{k_m+1} after them,
// and rebuild T as diag(theta_1..l_s) bordered by r = beta_{k_m} U_{last
// q rows, 1:l_s} (Eq. (trb-tmat) and the restart formulas below it).
//
// The paper leaves the QR method open; this uses Cholesky QR twice with
// the Gram matrix in FP64.  A column whose Cholesky pivot falls below a
// threshold (an exhausted Krylov direction) is replaced by a fresh seeded
// random vector, the block is re-orthogonalised, and beta_k = V_{k+1}^T W.
// The small symmetric eigenproblem uses cuSOLVER's syevd (FP64).
#include <cusolverDn.h>

#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <type_traits>
#include <climits>
#include <cmath>
#include <map>
#include <atomic>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "blas.cuh"

namespace trbl {
namespace {

#define TRBL_SOLVER(call)                                                         \
  do {                                                                            \
    cusolverStatus_t s_ = (call);                                                 \
    if (s_ != CUSOLVER_STATUS_SUCCESS)                                            \
      return fail(TRBL_ERR_CUDA, "%s: cusolver status %d", #call, int(s_));       \
  } while (0)

#define TRY(...)                \
  do {                          \
    int rc_ = (__VA_ARGS__);    \
    if (rc_) return rc_;        \
  } while (0)

// Cholesky G = R^T R (R upper) of a q x q FP64 Gram matrix, R^{-1}, and
// per-column deficiency flags: column j is marked when its pivot is at most
// thresh_abs, or thresh_rel times its own norm, or thresh_max times the
// largest column norm of the block.
// One block of 64 threads; flags[0] counts deficient columns, flags[1+j] marks them.
__global__ void chol_kernel(const double* __restrict__ G, int q, double thresh_abs, double thresh_rel,
                            double thresh_max, double* __restrict__ R, double* __restrict__ Rinv,
                            int* __restrict__ flags) {
  __shared__ double Rs[64][65];
  __shared__ double diag0[64];
  __shared__ double dmax;
  const int t = threadIdx.x;
  for (int i = t; i < q * q; i += blockDim.x) {
    const int r = i / q, c = i - r * q;
    Rs[r][c] = (c >= r) ? G[i] : 0.0;
  }
  if (t < q) diag0[t] = G[t * q + t];
  if (t == 0) flags[0] = 0;
  if (t < q) flags[1 + t] = 0;
  __syncthreads();
  if (t == 0) {
    double m = 0.0;
    for (int j = 0; j < q; ++j) m = fmax(m, diag0[j]);
    dmax = m;
  }
  __syncthreads();
  for (int j = 0; j < q; ++j) {
    if (t == 0) {
      double d = Rs[j][j];
      for (int k = 0; k < j; ++k) d -= Rs[k][j] * Rs[k][j];
      const double lim = fmax(fmax(thresh_abs * thresh_abs, thresh_rel * thresh_rel * fmax(diag0[j], 0.0)),
                              thresh_max * thresh_max * dmax);
      if (!(d > lim)) {
        flags[0] += 1;
        flags[1 + j] = 1;
        d = fmax(fabs(diag0[j]), 1e-300);
      }
      Rs[j][j] = sqrt(d);
    }
    __syncthreads();
    if (t > j && t < q) {
      double s = Rs[j][t];
      for (int k = 0; k < j; ++k) s -= Rs[k][j] * Rs[k][t];
      Rs[j][t] = s / Rs[j][j];
    }
    __syncthreads();
  }
  for (int i = t; i < q * q; i += blockDim.x) {
    const int r = i / q, c = i - r * q;
    R[i] = (c >= r) ? Rs[r][c] : 0.0;
  }
  // column t of R^{-1} by back substitution
  if (t < q) {
    double x[64];
    for (int j = t + 1; j < q; ++j) x[j] = 0.0;
    for (int j = t; j >= 0; --j) {
      double s = (j == t) ? 1.0 : 0.0;
      for (int k = j + 1; k <= t; ++k) s -= Rs[j][k] * x[k];
      x[j] = s / Rs[j][j];
    }
    for (int j = 0; j < q; ++j) Rinv[j * q + t] = (j <= t) ? x[j] : 0.0;
  }
}


// beta = R2 R1 (both upper triangular, q x q row-major)
__global__ void upper_mul_kernel(const double* __restrict__ R2, const double* __restrict__ R1, int q,
                                 double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= q * q) return;
  const int r = i / q, c = i - r * q;
  double s = 0.0;
  for (int k = r; k <= c; ++k) s += R2[r * q + k] * R1[k * q + c];
  out[i] = (c >= r) ? s : 0.0;
}

// T[b0+i][b0+j] = (C[(b0+i)*q + j] + C[(b0+j)*q + i]) / 2
__global__ void set_alpha_kernel(double* __restrict__ T, int ldt, const double* __restrict__ C, int b0, int q) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= q * q) return;
  const int r = i / q, c = i - r * q;
  T[int64_t(b0 + r) * ldt + b0 + c] = 0.5 * (C[(b0 + r) * q + c] + C[(b0 + c) * q + r]);
}

// C1[(b0 + i) q + j] = Cl[(q + i) q + j] + C[(b0 + i) q + j] (+ C2[...]): the
// projection of H V_k onto V_k summed over the local and full passes
__global__ void sum_alpha_kernel(double* __restrict__ C1, const double* __restrict__ Cl,
                                 const double* __restrict__ C, const double* __restrict__ C2, int b0, int ql,
                                 int q) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= q * q) return;
  const int r = i / q, c = i - r * q;
  double v = Cl[(ql - q + r) * q + c] + C[(b0 + r) * q + c];
  if (C2) v += C2[(b0 + r) * q + c];
  C1[(b0 + r) * q + c] = v;
}

// T[r0+i][c0+j] = beta[i][j], T[c0+j][r0+i] = beta[i][j]
__global__ void set_beta_kernel(double* __restrict__ T, int ldt, const double* __restrict__ beta, int r0,
                                int c0, int q) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= q * q) return;
  const int r = i / q, c = i - r * q;
  const double v = beta[i];
  T[int64_t(r0 + r) * ldt + c0 + c] = v;
  T[int64_t(c0 + c) * ldt + r0 + r] = v;
}

// res[i] = || beta U[nb-q : nb, i] ||  for i < n (U column-major, ld ldu)
__global__ void ritz_resid_kernel(const double* __restrict__ beta, int q, const double* __restrict__ U,
                                  int ldu, int nb, int n, double* __restrict__ res) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* u = U + int64_t(i) * ldu + (nb - q);
  double s2 = 0.0;
  for (int a = 0; a < q; ++a) {
    double s = 0.0;
    for (int b = 0; b < q; ++b) s += beta[a * q + b] * u[b];
    s2 += s * s;
  }
  res[i] = sqrt(s2);
}

// Ut[k][c] = U(k, c) for k < nb, c < n: column-major (ld ldu) -> row-major (ld n)
__global__ void transpose_kernel(const double* __restrict__ U, int ldu, int nb, int n, double* __restrict__ Ut) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb * n) return;
  const int k = i / n, c = i - k * n;
  Ut[i] = U[int64_t(c) * ldu + k];
}

// Thick-restart T (Eq. (trb-tmat)): diag(theta[0:ls]) bordered by
// r[a][i] = sum_b beta[a][b] U[nb-q+b][i] in rows/cols ls..ls+q-1.
__global__ void restart_t_kernel(double* __restrict__ T, int ldt, const double* __restrict__ theta,
                                 const double* __restrict__ beta, int q, const double* __restrict__ U,
                                 int ldu, int nb, int ls) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ls) T[int64_t(i) * ldt + i] = theta[i];
  if (i >= ls * q) return;
  const int a = i / ls, c = i - a * ls;
  const double* u = U + int64_t(c) * ldu + (nb - q);
  double s = 0.0;
  for (int b = 0; b < q; ++b) s += beta[a * q + b] * u[b];
  T[int64_t(ls + a) * ldt + c] = s;
  T[int64_t(c) * ldt + ls + a] = s;
}

// Per-column partial sums of ||HX - theta X||^2 over a row chunk.
__global__ void resid_partial_kernel(const double* __restrict__ HX, const double* __restrict__ X, int n,
                                     const double* __restrict__ theta, int64_t D, int64_t rows,
                                     double* __restrict__ part) {
  const int c = threadIdx.x;
  if (c >= n) return;
  const int64_t r0 = int64_t(blockIdx.x) * rows, r1 = min(D, r0 + rows);
  const double th = theta[c];
  double s = 0.0;
  for (int64_t r = r0; r < r1; ++r) {
    const double d = HX[r * n + c] - th * X[r * n + c];
    s += d * d;
  }
  part[int64_t(blockIdx.x) * n + c] = s;
}

__global__ void resid_final_kernel(const double* __restrict__ part, int nchunk, int n, double* __restrict__ out) {
  const int c = threadIdx.x;
  if (c >= n) return;
  double s = 0.0;
  for (int k = 0; k < nchunk; ++k) s += part[int64_t(k) * n + c];
  out[c] = sqrt(s);
}

// Layout of the small int buffer shared by device and pinned host memory.
constexpr int kF1 = 0;     // pass-1 Cholesky: count, then one flag per column
constexpr int kF2 = 80;    // pass-2 Cholesky
constexpr int kInfo = 160; // syevd info
constexpr int kTmaErr = 170;  // TMA wait timeout word
constexpr int kFlagInts = 192;
constexpr double kCheckRatio = 12.0;  // adaptive Rayleigh-Ritz cadence (see Solver::step)

// ---- batched forms of a block step's small kernels ----
// Per-set device pointers of the batched solver's step (entry s = set s).
template <typename T>
struct SetPtrs {
  T* basis;
  T* Vk;
  double* C;
  double* G;
  double* R1;
  double* R1i;
  double* R2;
  double* R2i;
  double* beta;
  double* Tm;
  int* flags;
  double thr1;  // absolute pivot threshold of the pass-1 Cholesky (tau ||H||)
  int64_t D;    // the set's dimension
};

// block s = set s: the pass-1 (pass = 1) or pass-2 Cholesky of its Gram
// matrix (chol_kernel's arithmetic on the set's buffers)
template <typename T>
__global__ void chol_batched_kernel(const SetPtrs<T>* __restrict__ sp, int q, int pass, double thresh_rel,
                                    double thresh_max) {
  const SetPtrs<T> p = sp[blockIdx.x];
  const double* __restrict__ G = p.G;
  double* __restrict__ R = pass == 1 ? p.R1 : p.R2;
  double* __restrict__ Rinv = pass == 1 ? p.R1i : p.R2i;
  int* __restrict__ flags = p.flags + (pass == 1 ? kF1 : kF2);
  const double thresh_abs = pass == 1 ? p.thr1 : 0.0;

  __shared__ double Rs[64][65];
  __shared__ double diag0[64];
  __shared__ double dmax;
  const int t = threadIdx.x;
  for (int i = t; i < q * q; i += blockDim.x) {
    const int r = i / q, c = i - r * q;
    Rs[r][c] = (c >= r) ? G[i] : 0.0;
  }
  if (t < q) diag0[t] = G[t * q + t];
  if (t == 0) flags[0] = 0;
  if (t < q) flags[1 + t] = 0;
  __syncthreads();
  if (t == 0) {
    double m = 0.0;
    for (int j = 0; j < q; ++j) m = fmax(m, diag0[j]);
    dmax = m;
  }
  __syncthreads();
  for (int j = 0; j < q; ++j) {
    if (t == 0) {
      double d = Rs[j][j];
      for (int k = 0; k < j; ++k) d -= Rs[k][j] * Rs[k][j];
      const double lim = fmax(fmax(thresh_abs * thresh_abs, thresh_rel * thresh_rel * fmax(diag0[j], 0.0)),
                              thresh_max * thresh_max * dmax);
      if (!(d > lim)) {
        flags[0] += 1;
        flags[1 + j] = 1;
        d = fmax(fabs(diag0[j]), 1e-300);
      }
      Rs[j][j] = sqrt(d);
    }
    __syncthreads();
    if (t > j && t < q) {
      double s = Rs[j][t];
      for (int k = 0; k < j; ++k) s -= Rs[k][j] * Rs[k][t];
      Rs[j][t] = s / Rs[j][j];
    }
    __syncthreads();
  }
  for (int i = t; i < q * q; i += blockDim.x) {
    const int r = i / q, c = i - r * q;
    R[i] = (c >= r) ? Rs[r][c] : 0.0;
  }
  // column t of R^{-1} by back substitution
  if (t < q) {
    double x[64];
    for (int j = t + 1; j < q; ++j) x[j] = 0.0;
    for (int j = t; j >= 0; --j) {
      double s = (j == t) ? 1.0 : 0.0;
      for (int k = j + 1; k <= t; ++k) s -= Rs[j][k] * x[k];
      x[j] = s / Rs[j][j];
    }
    for (int j = 0; j < q; ++j) Rinv[j * q + t] = (j <= t) ? x[j] : 0.0;
  }
}



// grid (., sets): T_s[b0 + i][b0 + j] = (C_s[(b0+i) q + j] + C_s[(b0+j) q + i]) / 2
template <typename T>
__global__ void set_alpha_batched_kernel(const SetPtrs<T>* __restrict__ sp, int ldt, int b0, int q) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= q * q) return;
  const SetPtrs<T> p = sp[blockIdx.y];
  const int r = i / q, c = i - r * q;
  p.Tm[int64_t(b0 + r) * ldt + b0 + c] = 0.5 * (p.C[(b0 + r) * q + c] + p.C[(b0 + c) * q + r]);
}

// Selective reorthogonalisation of a batch: dst[s] = src[s] + off (the
// local window's first column in every set's basis)
template <typename T>
__global__ void offset_ptrs_kernel(T* const* __restrict__ src, int64_t off, T** __restrict__ dst, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i] + off;
}

// The DGKS test per set: skip[s] = 0 (run the second full pass) when a
// column of W kept at most half its squared norm through the first (G's
// diagonal after, nb before; NaN runs it too), else 1.
__global__ void dgks_flags_kernel(const double* const* __restrict__ G, const double* const* __restrict__ nb, int q,
                                  int* __restrict__ skip, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int again = 0;
  for (int j = 0; j < q; ++j)
    if (!(G[i][j * q + j] > 0.5 * nb[i][j])) again = 1;
  skip[i] = again ? 0 : 1;
}

// alpha of the selective pass: the projection on V_k summed over the local
// pass (Cl rows ql - q ..), the full pass (C) and, where it ran, the second
// (C + ldt q); symmetrised into T_s as set_alpha_batched_kernel does
template <typename T>
__global__ void set_alpha_sel_batched_kernel(const SetPtrs<T>* __restrict__ sp, double* const* __restrict__ Cl,
                                             const int* __restrict__ skip, int ldt, int b0, int ql, int q) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= q * q) return;
  const SetPtrs<T> p = sp[blockIdx.y];
  const double* cl = Cl[blockIdx.y];
  const bool two = skip[blockIdx.y] == 0;
  const int r = i / q, c = i - r * q;
  auto a = [&](int x, int y) {
    double v = cl[(ql - q + x) * q + y] + p.C[(b0 + x) * q + y];
    if (two) v += p.C[size_t(ldt) * q + (b0 + x) * q + y];
    return v;
  };
  p.Tm[int64_t(b0 + r) * ldt + b0 + c] = 0.5 * (a(r, c) + a(c, r));
}

// grid (., sets): beta_s = R2_s R1_s, then its two copies in T_s
template <typename T>
__global__ void beta_batched_kernel(const SetPtrs<T>* __restrict__ sp, int ldt, int r0, int c0, int q, int set_t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= q * q) return;
  const SetPtrs<T> p = sp[blockIdx.y];
  const int r = i / q, c = i - r * q;
  double s = 0.0;
  for (int k = r; k <= c; ++k) s += p.R2[r * q + k] * p.R1[k * q + c];
  const double v = (c >= r) ? s : 0.0;
  p.beta[i] = v;
  if (set_t) {
    p.Tm[int64_t(r0 + r) * ldt + c0 + c] = v;
    p.Tm[int64_t(c0 + c) * ldt + r0 + r] = v;
  }
}

// grid (., sets): basis_s[:, col0 : col0 + q] = Vk_s over the set's D rows
template <typename T>
__global__ void append_batched_kernel(const SetPtrs<T>* __restrict__ sp, int q, int ldb, int col0) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const SetPtrs<T> p = sp[blockIdx.y];
  if (i >= p.D * q) return;
  const int64_t r = i / q;
  const int c = int(i - r * q);
  p.basis[r * ldb + col0 + c] = p.Vk[i];
}

// out[2 s], out[2 s + 1] = the deficient-column counts of set s's two Cholesky passes
template <typename T>
__global__ void gather_counts_kernel(const SetPtrs<T>* __restrict__ sp, int nset, int* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nset) return;
  out[2 * i] = sp[i].flags[kF1];
  out[2 * i + 1] = sp[i].flags[kF2];
}

// Host-side progress trace, on when the environment sets TRBL_TRACE=1.
static bool trace_on() {
  static const bool on = [] {
    const char* e = getenv("TRBL_TRACE");
    return e && e[0] == '1';
  }();
  return on;
}
static void trace(const char* fmt, ...) {
  if (!trace_on()) return;
  va_list ap;
  va_start(ap, fmt);
  fprintf(stderr, "[trbl] ");
  vfprintf(stderr, fmt, ap);
  fprintf(stderr, "\n");
  fflush(stderr);
  va_end(ap);
}

struct Timer {
  cudaEvent_t ev[8];
  bool on = false;
  int init(bool want) {
    on = want;
    if (!on) return TRBL_OK;
    for (auto& e : ev) TRBL_CUDA(cudaEventCreate(&e));
    return TRBL_OK;
  }
  void rec(int i, cudaStream_t s) {
    if (on) cudaEventRecord(ev[i], s);
  }
  double ms(int a, int b) {
    if (!on) return 0.0;
    float x = 0.f;
    cudaEventElapsedTime(&x, ev[a], ev[b]);
    return x;
  }
  ~Timer() {
    if (on)
      for (auto& e : ev) cudaEventDestroy(e);
  }
};

struct Arena {
  void* base = nullptr;
  size_t off = 0, cap = 0;
  template <typename X>
  X* take(size_t n) {
    size_t o = (off + 255) & ~size_t(255);
    off = o + n * sizeof(X);
    return reinterpret_cast<X*>(static_cast<char*>(base) + o);
  }
  ~Arena() {
    if (base) cudaFree(base);
  }
};

template <typename T>
struct Solver {
  const trbl_hamiltonian* h;
  const trbl_params* p;
  cudaStream_t s;
  int64_t D;
  int q, nev, mb, ls, dtype;
  double tau;      // pass-1 deficiency threshold relative to ||H||
  double tau_max;  // pass-1 deficiency threshold relative to the block's largest column
  Workspace ws;
  Arena ar;
  T *basis, *Vk, *W, *W2, *Wsave, *panel;
  int64_t panel_rows;
  double *C, *G, *R1, *R1i, *R2, *R2i, *beta, *Tm, *Aw, *theta, *Ut, *res, *syev_work, *Xd, *HXd, *rpart, *rtrue;
  double *Cl, *Gn;  // local-pass coefficients (up to (2q + 3) x q), squared column norms before the full pass
  bool gram_ready = false;  // G holds W^T W of the current W (set by the selective pass)
  int second_passes = 0;
  int *flags, *devinfo;
  int lwork;
  int64_t nchunk_res;
  cusolverDnHandle_t sol = nullptr;
  float* utw = nullptr;      // split TF32 transpose of a restart / Ritz coefficient matrix (gemm_wide_tc)
  size_t utw_bytes = 0;
  double *hbuf;  // pinned: theta[mb], res[mb], flags as doubles
  int* hflags;
  uint64_t reseed = 0;
  double normH = 0.0;
  bool skip_warmup = false;  // batch members after the first share the warmed eigensolver

  ~Solver() {
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (sol) cusolverDnDestroy(sol);
    if (hbuf) cudaFreeHost(hbuf);
    if (syev_work) cudaFree(syev_work);
  }

  int apply(const T* V, T* Wout) { return launch_apply(h, V, q, Wout, q, q, dtype, s); }

  // W -= B[:, 0:nb] (B^T W), twice
  int cgs2(T* Wb, int nb, double* Cout_first) {
    if (nb == 0) return TRBL_OK;
    TRY(block_dot<T>(basis, mb, nb, Wb, q, q, D, C, ws, s));
    if (Cout_first && Cout_first != C)
      TRBL_CUDA(cudaMemcpyAsync(Cout_first, C, sizeof(double) * nb * q, cudaMemcpyDeviceToDevice, s));
    TRY(rowgemm_ws<T>(basis, mb, nb, C, q, q, Wb, q, D, -1.0, 1.0, ws, s));
    TRY(block_dot<T>(basis, mb, nb, Wb, q, q, D, C + size_t(mb) * q, ws, s));
    TRY(rowgemm_ws<T>(basis, mb, nb, C + size_t(mb) * q, q, q, Wb, q, D, -1.0, 1.0, ws, s));
    return TRBL_OK;
  }

  // Selective reorthogonalisation (TRBL_REORTH_SELECTIVE): classical
  // Gram-Schmidt against the last two blocks (the three-term part of the
  // recurrence), one full pass against all nb stored vectors, and a second
  // full pass only when a column of W lost more than half its squared norm
  // in the first (Daniel-Gragg-Kaufman-Stewart).  C1's rows nb-q .. nb
  // receive the projection of W onto V_k summed over the passes.
  int cgs_selective(T* Wb, int nb, double* C1) {
    // The local window ends at column nb and starts on a 16-byte boundary
    // (after a thick restart nb = l_s + q is odd in general; a window at an
    // unaligned column would leave the TMA and tensor-core kernels for the
    // generic ones), so it may hold up to 3 columns more than 2q.
    constexpr int kAlign = int(16 / sizeof(T));
    const int c0 = std::max(0, nb - 2 * q) / kAlign * kAlign;
    const int ql = nb - c0;
    const T* Bl = basis + c0;
    TRY(block_dot<T>(Bl, mb, ql, Wb, q, q, D, Cl, ws, s));
    TRY(rowgemm_ws<T>(Bl, mb, ql, Cl, q, q, Wb, q, D, -1.0, 1.0, ws, s));
    // squared column norms before the full pass, and after it the block's
    // Gram matrix, whose diagonal holds them after (the DGKS test) and which
    // the block QR reuses when no second pass follows
    TRY(col_sumsq<T>(Wb, q, q, D, Gn, ws, s));
    TRY(block_dot<T>(basis, mb, nb, Wb, q, q, D, C, ws, s));
    TRY(rowgemm_ws<T>(basis, mb, nb, C, q, q, Wb, q, D, -1.0, 1.0, ws, s));
    TRY(gram<T>(Wb, q, q, D, G, ws, s));
    TRBL_CUDA(cudaMemcpyAsync(hbuf + 2 * mb, Gn, sizeof(double) * q, cudaMemcpyDeviceToHost, s));
    TRBL_CUDA(cudaMemcpyAsync(hbuf + 2 * mb + q, G, sizeof(double) * q * q, cudaMemcpyDeviceToHost, s));
    TRBL_CUDA(cudaStreamSynchronize(s));
    bool again = false;
    for (int j = 0; j < q; ++j) {
      const double before = hbuf[2 * mb + j], after = hbuf[2 * mb + q + j * q + j];
      if (!(after > 0.5 * before)) again = true;  // also catches NaN and a vanished column
    }
    gram_ready = !again && Wb == W;
    double* C2 = nullptr;
    if (again) {
      C2 = C + size_t(mb) * q;
      TRY(block_dot<T>(basis, mb, nb, Wb, q, q, D, C2, ws, s));
      TRY(rowgemm_ws<T>(basis, mb, nb, C2, q, q, Wb, q, D, -1.0, 1.0, ws, s));
      ++second_passes;
    }
    sum_alpha_kernel<<<(q * q + 127) / 128, 128, 0, s>>>(C1, Cl, C, C2, nb - q, ql, q); note_launch();
    TRBL_CUDA(cudaGetLastError());
    return TRBL_OK;
  }

  // Cholesky QR twice: Vk = W R^{-1}, beta = R2 R1.  Returns the number of
  // deficient columns found in pass 1 (their flags stay in hflags).
  int cholqr2(T* Win, double thresh_abs, double thresh_rel, double thresh_max, int* ndef) {
    TRY(cholqr2_async(Win, thresh_abs, thresh_rel, thresh_max));
    TRBL_CUDA(cudaStreamSynchronize(s));
    TRY(wait_errors());
    *ndef = hflags[kF1] + hflags[kF2];
    return TRBL_OK;
  }

  // Cholesky QR twice, enqueued only: the deficiency counts are copied to
  // pinned host memory (hflags) for the caller to read after synchronising.
  int cholqr2_async(T* Win, double thresh_abs, double thresh_rel, double thresh_max) {
    if (!(gram_ready && Win == W)) TRY(gram<T>(Win, q, q, D, G, ws, s));
    gram_ready = false;
    chol_kernel<<<1, 64, 0, s>>>(G, q, thresh_abs, thresh_rel, thresh_max, R1, R1i, flags + kF1); note_launch();
    TRBL_CUDA(cudaGetLastError());
    TRBL_CUDA(cudaMemcpyAsync(hflags + kF1, flags + kF1, sizeof(int) * (q + 1), cudaMemcpyDeviceToHost, s));
    TRY(rowgemm_ws<T>(Win, q, q, R1i, q, q, W2, q, D, 1.0, 0.0, ws, s));
    TRY(gram<T>(W2, q, q, D, G, ws, s));
    chol_kernel<<<1, 64, 0, s>>>(G, q, 0.0, 1e-3, 0.0, R2, R2i, flags + kF2); note_launch();
    TRBL_CUDA(cudaGetLastError());
    TRBL_CUDA(cudaMemcpyAsync(hflags + kF2, flags + kF2, sizeof(int), cudaMemcpyDeviceToHost, s));
    TRY(rowgemm_ws<T>(W2, q, q, R2i, q, q, Vk, q, D, 1.0, 0.0, ws, s));
    upper_mul_kernel<<<(q * q + 127) / 128, 128, 0, s>>>(R2, R1, q, beta); note_launch();
    TRBL_CUDA(cudaGetLastError());
    // wait-timeout words of the TMA and tensor-core kernels, read by wait_errors()
    TRY(tma_error_to_host(hflags + kTmaErr, s));
    TRY(dot_error_to_host(hflags + kTmaErr + 1, s));
    TRY(tc_error_to_host(hflags + kTmaErr + 2, s));
    TRY(wide_error_to_host(hflags + kTmaErr + 3, s));
    TRY(pn_tma_error_to_host(hflags + kTmaErr + 4, s));
    return TRBL_OK;
  }

  // After the stream synchronised past cholqr2_async.
  int wait_errors() {
    if (hflags[kTmaErr] || hflags[kTmaErr + 1] || hflags[kTmaErr + 2] || hflags[kTmaErr + 3])
      return fail(TRBL_ERR_CUDA, "a bounded wait in a projection kernel timed out");
    if (hflags[kTmaErr + 4]) return fail(TRBL_ERR_CUDA, "a bounded wait in the staged cross-term kernel timed out");
    return TRBL_OK;
  }

  // QR of W (already orthogonal to the basis).  Cholesky QR twice when the
  // block is well conditioned; otherwise the column-wise path below.
  int block_qr(int nb) {
    int ndef = 0;
    TRY(cholqr2(W, tau * normH, 0.0, tau_max, &ndef));
    if (ndef == 0) return TRBL_OK;
    return column_qr(nb);
  }

  // Stable column-by-column QR of W: classical Gram-Schmidt twice against
  // the basis and the earlier columns.  A column whose residual is at most
  // tau * ||H|| (an exhausted Krylov direction) is replaced by a seeded
  // random vector orthogonalised the same way.  beta_k = V_{k+1}^T W holds
  // exactly because every dropped residual is negligible.
  int column_qr(int nb) {
    trace("column QR at nb %d", nb);
    TRBL_CUDA(cudaMemcpyAsync(Wsave, W, sizeof(T) * D * q, cudaMemcpyDeviceToDevice, s));
    TRY(block_dot<T>(W, q, q, W, q, q, D, G, ws, s));
    TRBL_CUDA(cudaMemcpyAsync(hbuf, G, sizeof(double) * q * q, cudaMemcpyDeviceToHost, s));
    TRBL_CUDA(cudaStreamSynchronize(s));
    double cmax = 0.0;
    for (int j = 0; j < q; ++j) {
      if (!std::isfinite(hbuf[j * q + j]))
        return fail(TRBL_ERR_BREAKDOWN, "non-finite values in the Lanczos block (NaN or Inf in H or the vectors)");
      cmax = std::max(cmax, std::sqrt(std::max(hbuf[j * q + j], 0.0)));
    }
    const double thr = std::max(tau * normH, (dtype == TRBL_F64 ? 1e-13 : 1e-6) * cmax);
    for (int j = 0; j < q; ++j) {
      T* wj = W + j;
      for (int attempt = 0; attempt < 2; ++attempt) {
        for (int pass = 0; pass < 2; ++pass) {
          if (nb > 0) {
            TRY(block_dot<T>(basis, mb, nb, wj, q, 1, D, C, ws, s));
            TRY(rowgemm<T>(basis, mb, nb, C, 1, 1, wj, q, D, -1.0, 1.0, s));
          }
          if (j > 0) {
            TRY(block_dot<T>(W, q, j, wj, q, 1, D, C, ws, s));
            TRY(rowgemm<T>(W, q, j, C, 1, 1, wj, q, D, -1.0, 1.0, s));
          }
        }
        TRY(block_dot<T>(wj, q, 1, wj, q, 1, D, G, ws, s));
        TRBL_CUDA(cudaMemcpyAsync(hbuf, G, sizeof(double), cudaMemcpyDeviceToHost, s));
        TRBL_CUDA(cudaStreamSynchronize(s));
        const double nrm = std::sqrt(std::max(hbuf[0], 0.0));
        if (nrm > thr || (attempt == 1 && nrm > 0.0)) {
          TRY(scale_col<T>(wj, q, D, 1.0 / nrm, s));
          break;
        }
        if (attempt == 1) return fail(TRBL_ERR_BREAKDOWN, "block QR: no new direction left (basis spans the space?)");
        TRY(random_block<T>(wj, q, D, 1, q, j, p->seed + 0x9e37ull * (++reseed), s));
      }
    }
    TRBL_CUDA(cudaMemcpyAsync(Vk, W, sizeof(T) * D * q, cudaMemcpyDeviceToDevice, s));
    TRY(block_dot<T>(Vk, q, q, Wsave, q, q, D, beta, ws, s));
    return TRBL_OK;
  }

  // Eigenpairs of T[0:nb, 0:nb]; copies theta[0:nev], theta[nb-1] and the
  // residual estimates res[0:nev] to the host.
  int ritz(int nb) {
    const auto w0 = std::chrono::steady_clock::now();
    TRBL_CUDA(cudaMemcpy2DAsync(Aw, sizeof(double) * mb, Tm, sizeof(double) * mb, sizeof(double) * nb, nb,
                                cudaMemcpyDeviceToDevice, s));
    TRBL_SOLVER(cusolverDnDsyevd(sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, nb, Aw, mb, theta,
                                 syev_work, lwork, devinfo));
    if (trace_on()) {
      cudaStreamSynchronize(s);
      trace("ritz nb %d: syevd wall %.2f ms", nb,
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0).count());
    }
    const int n = std::min(nev, nb);
    ritz_resid_kernel<<<(n + 127) / 128, 128, 0, s>>>(beta, q, Aw, mb, nb, n, res); note_launch();
    TRBL_CUDA(cudaGetLastError());
    TRBL_CUDA(cudaMemcpyAsync(hbuf, theta, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
    TRBL_CUDA(cudaMemcpyAsync(hbuf + mb, res, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    TRBL_CUDA(cudaMemcpyAsync(hflags + kInfo, devinfo, sizeof(int), cudaMemcpyDeviceToHost, s));
    TRBL_CUDA(cudaStreamSynchronize(s));
    if (hflags[kInfo] != 0) return fail(TRBL_ERR_CUDA, "syevd info=%d", hflags[kInfo]);
    for (int i = 0; i < nb; ++i)
      if (!std::isfinite(hbuf[i])) return fail(TRBL_ERR_BREAKDOWN, "non-finite Ritz values (NaN or Inf in T)");
    const double est = std::max(std::fabs(hbuf[0]), std::fabs(hbuf[nb - 1]));
    if (p->normH <= 0.0) normH = std::max(normH, est);
    return TRBL_OK;
  }

  // Out[rows x n] (row-major, ld ldo) = In[rows x K] (row-major, ld ldi) U,
  // U FP64 K x n row-major (ld n): the dense GEMMs of the restart and of the
  // Ritz vectors.  FP32 data with n > 32 run on the tensor cores
  // (gemm_wide_tc: split TF32, fresh accumulators every 32 K values summed
  // in FP32 registers); FP64 data and narrow products use rowgemm.  With
  // presplit set, utw already holds U's split (gemm_wide_tc_split).
  int gemm_rm(const T* In, int64_t ldi, int K, const double* U, int n, T* Out, int64_t ldo, int64_t rows,
              bool presplit = false) {
    if (rows <= 0 || n <= 0 || K <= 0) return TRBL_OK;
    if constexpr (std::is_same<T, float>::value) {
      if (n > 32) {
        int rc = presplit ? TRBL_OK : gemm_wide_tc_split(U, n, K, n, utw, utw_bytes, s);
        if (rc == TRBL_OK) rc = gemm_wide_tc_run(In, ldi, K, n, utw, Out, ldo, rows, 1.0, 0.0, ws.sm_count, s);
        if (rc != -1) return rc;
      }
    }
    return rowgemm<T>(In, ldi, K, U, n, n, Out, ldo, rows, 1.0, 0.0, s);
  }

  // basis[:, 0:n_out] <- basis[:, 0:nb] U[:, 0:n_out] in row panels
  int compress(int nb, int n_out) {
    transpose_kernel<<<(nb * n_out + 255) / 256, 256, 0, s>>>(Aw, mb, nb, n_out, Ut); note_launch();
    TRBL_CUDA(cudaGetLastError());
    bool presplit = false;
    if constexpr (std::is_same<T, float>::value) {
      if (n_out > 32) presplit = gemm_wide_tc_split(Ut, n_out, nb, n_out, utw, utw_bytes, s) == TRBL_OK;
    }
    for (int64_t r0 = 0; r0 < D; r0 += panel_rows) {
      const int64_t nr = std::min(panel_rows, D - r0);
      // panel rows padded to a multiple of 8 columns (16-byte aligned rows)
      const int ldp = (n_out + 7) / 8 * 8;
      TRY(gemm_rm(basis + r0 * mb, mb, nb, Ut, n_out, panel, ldp, nr, presplit));
      TRY(copy_cols<T, T>(panel, ldp, basis + r0 * mb, mb, nr, n_out, s));
    }
    return TRBL_OK;
  }

  // target of the residual estimate as a fraction of tol (trbl_solve's
  // refinement lowers it when the true residuals of mixed precision miss tol)
  double est_scale = 1.0;

  // ---- stepping state ----
  Timer tm;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  double ms_apply = 0, ms_orth = 0, ms_qr = 0, ms_ritz = 0, ms_restart = 0;
  double since_check_ms = 0, last_check_ms = 0;  // adaptive Rayleigh-Ritz cadence
  int nb = 0, iter = 0, restarts = 0, conv = 0;
  bool done = false, have_ritz = false, finished = false;
  // T[0:nb, 0:nb] is complete (no block appended since its last Rayleigh-
  // Ritz step) but its eigenpairs are not on the device: set by load() for a
  // state saved in that condition, cleared by the next step.
  bool t_complete = false;

  // Start block: seeded random D x q, orthonormalised (Alg. 4, first line).
  int init() {
    TRY(tm.init(true));
    TRBL_CUDA(cudaEventCreate(&t0));
    TRBL_CUDA(cudaEventCreate(&t1));
    TRBL_CUDA(cudaEventRecord(t0, s));
    trace("init: D=%lld q=%d nev=%d max_basis=%d keep=%d", (long long)D, q, nev, mb, ls);
    TRY(random_block<T>(W, q, D, q, q, 0, p->seed, s));
    int ndef = 0;
    TRY(cholqr2(W, 0.0, 1e-8, tau_max, &ndef));
    if (ndef) TRY(column_qr(0));
    TRY(copy_cols<T, T>(Vk, q, basis, mb, D, q, s));
    nb = q;
    return TRBL_OK;
  }

  // One block step of Alg. 4 (plus a thick restart when the basis is full).
  int step(int* conv_out) {
    if (conv_out) *conv_out = -1;
    if (done) {
      if (conv_out) *conv_out = conv;
      return TRBL_OK;
    }
    const int max_iter = p->max_iter > 0 ? p->max_iter : 100000;
    t_complete = false;
    trace("iter %d nb %d", iter, nb);
    tm.rec(0, s);
    TRY(apply(Vk, W));
    tm.rec(1, s);
    double* C1 = C + size_t(2) * mb * q;
    if (p->reorth == TRBL_REORTH_TWICE)
      TRY(cgs2(W, nb, C1));
    else
      TRY(cgs_selective(W, nb, C1));
    set_alpha_kernel<<<(q * q + 127) / 128, 128, 0, s>>>(Tm, mb, C1, nb - q, q); note_launch();
    TRBL_CUDA(cudaGetLastError());
    tm.rec(2, s);
    TRY(block_qr(nb));
    tm.rec(3, s);
    ++iter;
    const bool need_restart = nb + q > mb;
    // Rayleigh-Ritz cadence: every check_every steps, or (check_every = 0)
    // once the block steps since the previous test took kCheckRatio times as
    // long as that test (tests then cost at most 1 / (1 + kCheckRatio) of the time)
    const bool due = p->check_every > 0 ? iter % p->check_every == 0 : since_check_ms >= kCheckRatio * last_check_ms;
    const bool check = need_restart || due || iter >= max_iter;
    have_ritz = false;
    if (check) {
      TRY(ritz(nb));
      have_ritz = true;
      const double lim = p->tol * normH * est_scale;
      conv = 0;
      for (int i = 0; i < std::min(nev, nb); ++i)
        if (hbuf[mb + i] <= lim) ++conv;
      if (nb >= nev && conv == nev) done = true;
      if (conv_out) *conv_out = conv;
      trace("ritz: theta0 %.12g normH %.6g converged %d", hbuf[0], normH, conv);
    }
    tm.rec(4, s);
    if (!done && iter < max_iter) {
      if (need_restart) {
        trace("restart nb %d -> %d", nb, ls + q);
        TRY(compress(nb, ls));
        TRBL_CUDA(cudaMemsetAsync(Tm, 0, sizeof(double) * mb * mb, s));
        restart_t_kernel<<<(ls * q + 127) / 128, 128, 0, s>>>(Tm, mb, theta, beta, q, Aw, mb, nb, ls); note_launch();
        TRBL_CUDA(cudaGetLastError());
        TRY(copy_cols<T, T>(Vk, q, basis + ls, mb, D, q, s));
        nb = ls + q;
        have_ritz = false;
        ++restarts;
      } else {
        set_beta_kernel<<<(q * q + 127) / 128, 128, 0, s>>>(Tm, mb, beta, nb, nb - q, q); note_launch();
        TRBL_CUDA(cudaGetLastError());
        TRY(copy_cols<T, T>(Vk, q, basis + nb, mb, D, q, s));
        nb += q;
        have_ritz = false;
      }
    }
    tm.rec(5, s);
    TRBL_CUDA(cudaEventSynchronize(tm.ev[5]));
    ms_apply += tm.ms(0, 1);
    ms_orth += tm.ms(1, 2);
    ms_qr += tm.ms(2, 3);
    ms_ritz += tm.ms(3, 4);
    ms_restart += tm.ms(4, 5);
    if (check) {
      last_check_ms = tm.ms(3, 4);
      since_check_ms = 0;
    } else {
      since_check_ms += tm.ms(0, 3) + tm.ms(4, 5);
    }
    trace("step %d phases ms: apply %.2f orth %.2f qr %.2f ritz %.2f restart %.2f", iter, tm.ms(0, 1), tm.ms(1, 2),
          tm.ms(2, 3), tm.ms(3, 4), tm.ms(4, 5));
    return TRBL_OK;
  }

  // ---- pieces of a block step for the batched driver ----
  // Everything after W = H V_k with no host synchronisation: CGS2, alpha,
  // Cholesky QR twice, and (unless the basis is full) beta and the append of
  // V_{k+1}.  Safe to capture in a CUDA graph for a fixed nb.
  int step_device(bool append) {
    double* C1 = C + size_t(2) * mb * q;
    TRY(cgs2(W, nb, C1));
    set_alpha_kernel<<<(q * q + 127) / 128, 128, 0, s>>>(Tm, mb, C1, nb - q, q); note_launch();
    TRBL_CUDA(cudaGetLastError());
    TRY(cholqr2_async(W, tau * normH, 0.0, tau_max));
    if (append) {
      set_beta_kernel<<<(q * q + 127) / 128, 128, 0, s>>>(Tm, mb, beta, nb, nb - q, q); note_launch();
      TRBL_CUDA(cudaGetLastError());
      TRY(copy_cols<T, T>(Vk, q, basis + nb, mb, D, q, s));
    }
    return TRBL_OK;
  }

  // After step_device ran (stream synchronised): deficiency check, Rayleigh-
  // Ritz when due, and the thick restart when the basis was full.
  int step_after(bool appended, bool check_due, int max_iter) {
    TRY(wait_errors());
    if (hflags[kF1] + hflags[kF2] > 0)
      return fail(TRBL_ERR_BREAKDOWN, "batched step: rank-deficient block (the batched driver has no repair path)");
    ++iter;
    const int nb_old = nb;
    const bool check = !appended || check_due || iter >= max_iter;
    if (check && !done) {
      TRY(ritz(nb_old));
      const double lim = p->tol * normH * est_scale;
      conv = 0;
      for (int i = 0; i < std::min(nev, nb_old); ++i)
        if (hbuf[mb + i] <= lim) ++conv;
      if (nb_old >= nev && conv == nev) done = true;
    }
    if (appended) {
      nb += q;
      have_ritz = false;
    } else {
      // all sets of a batch share one basis schedule, so a set that has
      // converged restarts with the others (its kept Ritz pairs survive)
      if (!check || done) TRY(ritz(nb_old));
      TRY(compress(nb_old, ls));
      TRBL_CUDA(cudaMemsetAsync(Tm, 0, sizeof(double) * mb * mb, s));
      restart_t_kernel<<<(ls * q + 127) / 128, 128, 0, s>>>(Tm, mb, theta, beta, q, Aw, mb, nb_old, ls); note_launch();
      TRBL_CUDA(cudaGetLastError());
      TRY(copy_cols<T, T>(Vk, q, basis + ls, mb, D, q, s));
      nb = ls + q;
      have_ritz = false;
      ++restarts;
    }
    return TRBL_OK;
  }

  void fill_stats(trbl_stats* st, int status) {
    st->iterations = iter;
    st->restarts = restarts;
    st->converged = conv;
    st->status = status;
    st->normH = normH;
    st->ms_apply = ms_apply;
    st->ms_orth = ms_orth;
    st->ms_qr = ms_qr;
    st->ms_ritz = ms_ritz;
    st->ms_restart = ms_restart;
    st->basis_size = nb;
    st->second_passes = second_passes;
  }

  // ---- checkpoint: the state between block steps ----
  // Header, then T (mb x mb FP64), beta (q x q FP64, for the residual
  // estimates of a finish right after a load), V_k (D x q) and the basis
  // (D x nb, packed), all in host memory.  `complete` is 1 when T[0:nb,
  // 0:nb] had its Rayleigh-Ritz step without a block appended after it (a
  // step that stopped at max_iter): a finish then uses all nb rows, as the
  // uninterrupted solver does.
  struct State {
    uint64_t magic;
    int32_t version, dtype, q, mb, ls, nb, iter, restarts, conv, complete;
    int64_t D;
    uint64_t reseed;
    double normH, since_check_ms, last_check_ms, ms[5];
  };
  static constexpr uint64_t kStateMagic = 0x5441545342525454ull;
  size_t state_bytes_for(int n) const {
    return sizeof(State) + sizeof(double) * (size_t(mb) * mb + size_t(q) * q) + sizeof(T) * size_t(D) * (q + n);
  }
  size_t state_bytes() const { return state_bytes_for(nb); }

  int save(void* host, int64_t bytes) {
    if (done) return fail(TRBL_ERR_ARG, "the solver has converged: finish it instead of saving its state");
    const size_t need = state_bytes();
    if (!host || bytes < 0 || size_t(bytes) < need) return fail(TRBL_ERR_ARG, "the state needs %zu bytes", need);
    State st{};
    st.magic = kStateMagic;
    st.version = 1;
    st.dtype = dtype;
    st.q = q;
    st.mb = mb;
    st.ls = ls;
    st.nb = nb;
    st.iter = iter;
    st.restarts = restarts;
    st.conv = conv;
    st.complete = (have_ritz || t_complete) ? 1 : 0;
    st.D = D;
    st.reseed = reseed;
    st.normH = normH;
    st.since_check_ms = since_check_ms;
    st.last_check_ms = last_check_ms;
    const double ms[5] = {ms_apply, ms_orth, ms_qr, ms_ritz, ms_restart};
    std::memcpy(st.ms, ms, sizeof(ms));
    unsigned char* o = static_cast<unsigned char*>(host);
    std::memcpy(o, &st, sizeof(st));
    o += sizeof(st);
    TRBL_CUDA(cudaMemcpyAsync(o, Tm, sizeof(double) * mb * mb, cudaMemcpyDeviceToHost, s));
    o += sizeof(double) * mb * mb;
    TRBL_CUDA(cudaMemcpyAsync(o, beta, sizeof(double) * q * q, cudaMemcpyDeviceToHost, s));
    o += sizeof(double) * q * q;
    TRBL_CUDA(cudaMemcpyAsync(o, Vk, sizeof(T) * D * q, cudaMemcpyDeviceToHost, s));
    o += sizeof(T) * D * q;
    TRBL_CUDA(cudaMemcpy2DAsync(o, sizeof(T) * nb, basis, sizeof(T) * mb, sizeof(T) * nb, size_t(D),
                                cudaMemcpyDeviceToHost, s));
    TRBL_CUDA(cudaStreamSynchronize(s));
    return TRBL_OK;
  }

  int load(const void* host, int64_t bytes) {
    if (!host || bytes < int64_t(sizeof(State))) return fail(TRBL_ERR_ARG, "not a solver state");
    State st;
    std::memcpy(&st, host, sizeof(st));
    if (st.magic != kStateMagic || st.version != 1) return fail(TRBL_ERR_ARG, "not a solver state of this library");
    if (st.dtype != dtype || st.q != q || st.mb != mb || st.ls != ls || st.D != D)
      return fail(TRBL_ERR_ARG, "state saved with other sizes (D %lld, q %d, max_basis %d, keep %d, precision)",
                  (long long)st.D, st.q, st.mb, st.ls);
    if (st.nb < q || st.nb > mb) return fail(TRBL_ERR_ARG, "corrupt state (basis size %d)", st.nb);
    if (st.complete != 0 && st.complete != 1) return fail(TRBL_ERR_ARG, "corrupt state (flag %d)", st.complete);
    if (size_t(bytes) < state_bytes_for(st.nb)) return fail(TRBL_ERR_ARG, "truncated state");
    const unsigned char* i = static_cast<const unsigned char*>(host) + sizeof(st);
    TRBL_CUDA(cudaMemcpyAsync(Tm, i, sizeof(double) * mb * mb, cudaMemcpyHostToDevice, s));
    i += sizeof(double) * mb * mb;
    TRBL_CUDA(cudaMemcpyAsync(beta, i, sizeof(double) * q * q, cudaMemcpyHostToDevice, s));
    i += sizeof(double) * q * q;
    TRBL_CUDA(cudaMemcpyAsync(Vk, i, sizeof(T) * D * q, cudaMemcpyHostToDevice, s));
    i += sizeof(T) * D * q;
    TRBL_CUDA(cudaMemcpy2DAsync(basis, sizeof(T) * mb, i, sizeof(T) * st.nb, sizeof(T) * st.nb, size_t(D),
                                cudaMemcpyHostToDevice, s));
    TRBL_CUDA(cudaStreamSynchronize(s));
    nb = st.nb;
    iter = st.iter;
    restarts = st.restarts;
    conv = st.conv;
    reseed = st.reseed;
    normH = st.normH;
    since_check_ms = st.since_check_ms;
    last_check_ms = st.last_check_ms;
    ms_apply = st.ms[0];
    ms_orth = st.ms[1];
    ms_qr = st.ms[2];
    ms_ritz = st.ms[3];
    ms_restart = st.ms[4];
    done = have_ritz = finished = false;
    t_complete = st.complete == 1;
    return TRBL_OK;
  }

  // Ritz values, vectors and true residuals of the current basis.
  int finish(double* evals, double* resid, void* evecs, trbl_stats* st) {
    const int status = done ? TRBL_OK : TRBL_ERR_NOCONV;
    trace("finish: status %d", status);
    // After an append or a restart the basis holds one more block than T's
    // last Rayleigh-Ritz step saw; the Ritz pairs below use the block
    // diagonal part of T that is complete (rows 0 .. nb - q).
    int nr = (have_ritz || t_complete) ? nb : nb - q;
    if (!have_ritz) TRY(ritz(nr));
    const int n = std::min(nev, nr);
    for (int i = 0; i < n; ++i) evals[i] = hbuf[i];
    for (int i = n; i < nev; ++i) evals[i] = NAN;
    transpose_kernel<<<(nr * n + 255) / 256, 256, 0, s>>>(Aw, mb, nr, n, Ut); note_launch();
    TRBL_CUDA(cudaGetLastError());
    if (evecs) TRY(gemm_rm(basis, mb, nr, Ut, n, static_cast<T*>(evecs), nev, D));
    if (resid) {
      // true residuals ||H x - theta x|| with an FP64 apply, q columns at a time
      const int64_t nchunk = nchunk_res;
      const int64_t rows = (D + nchunk - 1) / nchunk;
      for (int c0 = 0; c0 < n; c0 += q) {
        const int nc = std::min(q, n - c0);
        if constexpr (std::is_same<T, double>::value) {
          TRY(rowgemm<double>(basis, mb, nr, Ut + c0, n, nc, Xd, nc, D, 1.0, 0.0, s));
        } else {
          TRY(rowgemm<T>(basis, mb, nr, Ut + c0, n, nc, W, nc, D, 1.0, 0.0, s));
          TRY(copy_cols<T, double>(W, nc, Xd, nc, D, nc, s));
        }
        TRY(launch_apply(h, Xd, nc, HXd, nc, nc, TRBL_F64, s));
        resid_partial_kernel<<<unsigned(nchunk), 64, 0, s>>>(HXd, Xd, nc, theta + c0, D, rows, rpart); note_launch();
        TRBL_CUDA(cudaGetLastError());
        resid_final_kernel<<<1, 64, 0, s>>>(rpart, int(nchunk), nc, rtrue + c0); note_launch();
        TRBL_CUDA(cudaGetLastError());
      }
      TRBL_CUDA(cudaMemcpyAsync(resid, rtrue, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    }
    TRBL_CUDA(cudaEventRecord(t1, s));
    TRBL_CUDA(cudaStreamSynchronize(s));
    if (resid)
      for (int i = n; i < nev; ++i) resid[i] = NAN;
    if (st) {
      fill_stats(st, status);
      float tot = 0.f;
      cudaEventElapsedTime(&tot, t0, t1);
      st->ms_total = tot;
    }
    finished = true;
    if (status == TRBL_ERR_NOCONV)
      return fail(TRBL_ERR_NOCONV, "not converged after %d block iterations (%d of %d pairs)", iter, conv, nev);
    return TRBL_OK;
  }

  int setup() {
    const trbl_basis* b = h->b;
    D = b->D;
    q = p->q;
    nev = p->nev;
    mb = p->max_basis;
    dtype = std::is_same<T, double>::value ? TRBL_F64 : TRBL_F32;
    tau = dtype == TRBL_F64 ? 1e-10 : 1e-4;
    tau_max = dtype == TRBL_F64 ? 1e-6 : 1e-3;
    if (q < 1 || q > 64) return fail(TRBL_ERR_ARG, "q=%d outside [1, 64]", q);
    if (h->row_end >= 0 && (h->row_begin != 0 || h->row_end != D))
      return fail(TRBL_ERR_ARG, "the solver needs the product over all rows (trbl_hamiltonian_set_rows(h, 0, D))");
    if (nev < 1) return fail(TRBL_ERR_ARG, "nev must be positive");
    if (p->reorth != TRBL_REORTH_SELECTIVE && p->reorth != TRBL_REORTH_TWICE)
      return fail(TRBL_ERR_ARG, "reorth must be TRBL_REORTH_SELECTIVE or TRBL_REORTH_TWICE");
    if (mb > D) return fail(TRBL_ERR_ARG, "max_basis=%d exceeds the dimension %lld", mb, (long long)D);
    if (mb < nev + 2 * q) return fail(TRBL_ERR_ARG, "max_basis must be at least nev + 2q");
    if (!(p->tol > 0.0)) return fail(TRBL_ERR_ARG, "tol must be positive");
    ls = p->keep;
    if (ls <= 0) ls = nev + (mb - nev) / 4;
    ls = std::min(ls, mb - 2 * q);
    if (ls < nev) return fail(TRBL_ERR_ARG, "keep=%d smaller than nev=%d", ls, nev);
    normH = p->normH > 0.0 ? p->normH : 0.0;
    int dev = 0;
    TRBL_CUDA(cudaGetDevice(&dev));
    TRBL_CUDA(cudaDeviceGetAttribute(&ws.sm_count, cudaDevAttrMultiProcessorCount, dev));
    panel_rows = std::max<int64_t>(4096, (int64_t(1) << 30) / (int64_t(ls) * sizeof(T)));
    panel_rows = std::min(panel_rows, D);
    const size_t dq = size_t(D) * q;
    ws.partial_bytes = block_dot_workspace_bytes(q, q, ws.sm_count);
    for (int m = 1; m <= mb; ++m)
      ws.partial_bytes = std::max(ws.partial_bytes, block_dot_workspace_bytes(m, q, ws.sm_count));
    nchunk_res = std::min<int64_t>(4 * ws.sm_count, (D + 1023) / 1024);
    // Two passes over the same sequence of takes: size, then carve.
    for (int pass = 0; pass < 2; ++pass) {
      ar.off = 0;
      basis = ar.take<T>(size_t(D) * mb);
      Vk = ar.take<T>(dq);
      W = ar.take<T>(dq);
      W2 = ar.take<T>(dq);
      Wsave = ar.take<T>(dq);
      panel = ar.take<T>(size_t(panel_rows) * ((ls + 7) / 8 * 8));
      C = ar.take<double>(size_t(3) * mb * q);
      Cl = ar.take<double>(size_t(2 * q + 4) * q);
      Gn = ar.take<double>(q);
      G = ar.take<double>(q * q);
      R1 = ar.take<double>(q * q);
      R1i = ar.take<double>(q * q);
      R2 = ar.take<double>(q * q);
      R2i = ar.take<double>(q * q);
      beta = ar.take<double>(q * q);
      Tm = ar.take<double>(size_t(mb) * mb);
      Aw = ar.take<double>(size_t(mb) * mb);
      Ut = ar.take<double>(size_t(mb) * mb);
      utw_bytes = std::is_same<T, float>::value ? gemm_wide_tc_workspace_bytes(mb, mb) : 0;
      utw = ar.take<float>(utw_bytes / sizeof(float) + 4);
      theta = ar.take<double>(mb);
      res = ar.take<double>(mb);
      Xd = ar.take<double>(dq);
      HXd = ar.take<double>(dq);
      rpart = ar.take<double>(size_t(nchunk_res) * q);
      rtrue = ar.take<double>(mb);
      ws.ut = ar.take<float>(rowgemm_tc_workspace_bytes(mb) / sizeof(float));
      ws.partial = ar.take<double>(ws.partial_bytes / sizeof(double));
      flags = ar.take<int>(kFlagInts);
      if (pass == 0) {
        const size_t bytes = ar.off;
        cudaError_t e = cudaMalloc(&ar.base, bytes);
        if (e != cudaSuccess) {
          cudaGetLastError();
          ar.base = nullptr;
          return fail(TRBL_ERR_OOM, "solver workspace of %.2f GB: %s", bytes / 1e9, cudaGetErrorString(e));
        }
        ar.cap = bytes;
      }
    }
    devinfo = flags + kInfo;
    ws.ut_bytes = rowgemm_tc_workspace_bytes(mb);
    ws.tensor = p->projections == TRBL_PROJ_TENSOR;
    // With 32 columns the tensor-core update (16-byte epilogue stores) is the
    // faster one at every K (D = 18.6M: 2.0 against 3.2 ms at K = 32, 2.9
    // against 4.0 ms at K = 64); with 16 columns or fewer the CUDA-core kernel
    // stays faster below K = 256 (D = 2M, n = 16: 0.20 against 0.17 ms at
    // K = 32, 0.78 against 0.59 ms at K = 256).  The projection is faster on
    // the tensor cores at every m.
    ws.tc_min_k = q >= 32 ? 1 : 256;
    trace("workspace %.3f GB at %p", ar.cap / 1e9, ar.base);
    if (cusolverDnCreate(&sol) != CUSOLVER_STATUS_SUCCESS) return fail(TRBL_ERR_CUDA, "cusolverDnCreate failed");
    TRBL_SOLVER(cusolverDnSetStream(sol, s));
    TRBL_SOLVER(cusolverDnDsyevd_bufferSize(sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, mb, Aw, mb,
                                            theta, &lwork));
    trace("syevd lwork %d", lwork);
    {
      cudaError_t e = cudaMalloc(&syev_work, sizeof(double) * size_t(std::max(lwork, 1)));
      if (e != cudaSuccess) {
        cudaGetLastError();
        syev_work = nullptr;
        return fail(TRBL_ERR_OOM, "syevd workspace: %s", cudaGetErrorString(e));
      }
    }
    TRBL_CUDA(cudaMemsetAsync(Tm, 0, sizeof(double) * mb * mb, s));
    const size_t nh = size_t(2) * mb + size_t(2) * q * q;  // Ritz values, residuals / two q x q Gram matrices
    TRBL_CUDA(cudaMallocHost(&hbuf, sizeof(double) * nh + sizeof(int) * kFlagInts));
    hflags = reinterpret_cast<int*>(hbuf + nh);
    // The eigensolver loads size-dependent kernel variants on first use,
    // which can take seconds; run it once per size class here so that the
    // iteration does not pay it.
    for (int n = q; !skip_warmup && n <= mb; n = (n < mb && 2 * n > mb) ? mb : 2 * n) {
      TRBL_CUDA(cudaMemsetAsync(Aw, 0, sizeof(double) * size_t(mb) * n, s));
      TRBL_SOLVER(cusolverDnDsyevd(sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, Aw, mb, theta,
                                   syev_work, lwork, devinfo));
      if (n == mb) break;
    }
    TRBL_CUDA(cudaStreamSynchronize(s));
    return TRBL_OK;
  }
};


// Type-erased solver behind the C ABI.
struct SolverBase {
  virtual ~SolverBase() {}
  virtual int init() = 0;
  virtual int step(int* conv) = 0;
  virtual int finish(double* evals, double* resid, void* evecs, trbl_stats* st) = 0;
  virtual void stats(trbl_stats* st) = 0;
  virtual void* block() = 0;
  virtual size_t block_bytes() = 0;
  virtual bool is_done() = 0;
  virtual int iterations() = 0;
  virtual size_t state_bytes() = 0;
  virtual int save(void* host, int64_t bytes) = 0;
  virtual int load(const void* host, int64_t bytes) = 0;
  // Lower the estimate's target to scale * tol and let the solver step on.
  virtual void retarget(double scale) = 0;
  virtual double norm_h() = 0;
};

template <typename T>
struct SolverImpl : SolverBase {
  Solver<T> S{};
  int init() override { return S.init(); }
  int step(int* c) override { return S.step(c); }
  int finish(double* e, double* r, void* v, trbl_stats* st) override { return S.finish(e, r, v, st); }
  void stats(trbl_stats* st) override {
    S.fill_stats(st, TRBL_OK);
    float tot = 0.f;
    cudaEventRecord(S.t1, S.s);
    cudaEventSynchronize(S.t1);
    cudaEventElapsedTime(&tot, S.t0, S.t1);
    st->ms_total = tot;
  }
  void* block() override { return S.Vk; }
  size_t block_bytes() override { return sizeof(T) * size_t(S.D) * S.q; }
  bool is_done() override { return S.done; }
  void retarget(double scale) override {
    S.est_scale = scale;
    S.done = false;
    S.finished = false;
  }
  double norm_h() override { return S.normH; }
  int iterations() override { return S.iter; }
  size_t state_bytes() override { return S.state_bytes(); }
  int save(void* host, int64_t bytes) override { return S.save(host, bytes); }
  int load(const void* host, int64_t bytes) override { return S.load(host, bytes); }
};

}  // namespace
}  // namespace trbl

namespace trbl {
namespace {

// Several Hamiltonians on one basis solved together.  One persistent launch
// applies all of them (the grouped kernel over work items x sets), and every
// other operation of a block step (CGS2, alpha, Cholesky QR twice, beta, the
// append) is one launch over all sets, reading the sets' pointers from
// device arrays; the step is captured once per basis size into a CUDA graph
// and replayed.  Rayleigh-Ritz tests and restarts run between replays on
// host worker threads, each set on its own stream, so the small eigensolver
// calls of different sets overlap on the GPU.
template <typename T>
struct BatchDriver {
  using clock = std::chrono::steady_clock;
  std::vector<Solver<T>*> sets;
  trbl_params prm{};
  cudaStream_t s = nullptr;         // the batch's own stream (capture origin)
  std::vector<cudaStream_t> ss;     // one stream per set
  std::vector<cudaEvent_t> ev_done;  // end of a set's host-driven work
  int nset = 0, nwork = 0, dtype = 0, device = 0, nthreads = 1;
  size_t smem = 0, smem_fast = 0;
  const trbl_hamiltonian* h0 = nullptr;  // the first set's Hamiltonian: launch shape of the batch's product
  bool all_fast = false;                 // the FP32 fast product applies to every set
  int64_t D = 0;                         // the largest set dimension (grid sizes)
  std::vector<int64_t> Ds;               // each set's dimension
  std::vector<size_t> voff;              // each set's V_k (and W) offset in the shared buffer, in elements
  size_t vtotal = 0;                     // elements of all sets' V_k together
  int64_t* P_D = nullptr;                // device copy of Ds
  int q = 0, mb = 0;
  void* shared = nullptr;  // V_k and W of all sets, set-major
  void* tables = nullptr;  // DevH<T>[nset], DevG<T>[nset]
  // batched step: device arrays of per-set pointers, per-set records, counts
  void* bptr = nullptr;
  T** P_basis = nullptr;
  T** P_W = nullptr;
  T** P_W2 = nullptr;
  T** P_Vk = nullptr;
  double** P_C1 = nullptr;
  double** P_C2 = nullptr;
  double** P_G = nullptr;
  double** P_R1i = nullptr;
  double** P_R2i = nullptr;
  double** P_part = nullptr;
  T** P_Bl = nullptr;      // selective pass: the local window of each basis (written in the step)
  double** P_Cl = nullptr;  // selective pass: local coefficients
  double** P_Gn = nullptr;  // selective pass: squared column norms before the full pass
  int* dskip = nullptr;     // selective pass: 1 where a set skips the second full pass
  int64_t second_passes = 0;
  SetPtrs<T>* dsp = nullptr;
  int* dcounts = nullptr;
  SetPtrs<T>* hsp = nullptr;  // pinned: the records, thresholds refreshed before each step
  int* hcounts = nullptr;     // pinned: 2 counts per set, then the four wait-timeout words
  size_t part_bytes = 0;
  std::map<int, cudaGraphExec_t> graphs;
  std::vector<int> rc;
  std::vector<std::string> msg;
  clock::time_point t_start;
  double ms_steps = 0, ms_between = 0;

  ~BatchDriver() {
    if (s) cudaStreamSynchronize(s);
    for (cudaStream_t x : ss)
      if (x) cudaStreamSynchronize(x);
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    for (auto* S : sets) delete S;
    for (cudaEvent_t e : ev_done)
      if (e) cudaEventDestroy(e);
    for (cudaStream_t x : ss)
      if (x) cudaStreamDestroy(x);
    if (shared) cudaFree(shared);
    if (tables) cudaFree(tables);
    if (bptr) cudaFree(bptr);
    if (hsp) cudaFreeHost(hsp);
    if (hcounts) cudaFreeHost(hcounts);
  }

  static double ms_since(clock::time_point t) {
    return std::chrono::duration<double, std::milli>(clock::now() - t).count();
  }

  // f(i) for every set i in [i0, nset) still without error, on up to
  // nthreads host threads (the caller's among them).  Each thread binds the
  // caller's device; a failure is kept in rc[i] with its message in msg[i]
  // (error messages are per thread).
  template <typename F>
  void for_sets(int i0, F f) {
    std::atomic<int> next{i0};
    auto work = [&] {
      cudaSetDevice(device);
      for (int i; (i = next.fetch_add(1)) < nset;) {
        if (rc[i] != TRBL_OK) continue;
        rc[i] = f(i);
        if (rc[i] != TRBL_OK) msg[i] = trbl_last_error();
      }
    };
    std::vector<std::thread> th;
    const int nt = std::min(nthreads, nset - i0);
    for (int t = 1; t < nt; ++t) {
      try {
        th.emplace_back(work);
      } catch (...) {
        break;  // fewer threads: the others take the work
      }
    }
    work();
    for (auto& t : th) t.join();
  }

  // Set i's setup and start block on its own stream.
  int setup_set(const trbl_hamiltonian* h, int i) {
    Solver<T>* S = sets[i];
    T* V0 = static_cast<T*>(shared);
    S->h = h;
    S->p = &prm;
    S->s = ss[i];
    S->skip_warmup = i > 0;
    TRY(S->setup());
    S->Vk = V0 + voff[i];
    S->W = V0 + vtotal + voff[i];
    TRY(S->init());
    TRBL_CUDA(cudaEventRecord(ev_done[i], ss[i]));
    return TRBL_OK;
  }

  int setup(const trbl_hamiltonian* const* hs) {
    t_start = clock::now();
    q = prm.q;
    mb = prm.max_basis;
    dtype = std::is_same<T, double>::value ? TRBL_F64 : TRBL_F32;
    const int bytes = q * int(sizeof(T));
    if (bytes % 16 || (bytes & (bytes - 1)) || bytes > 512)
      return fail(TRBL_ERR_ARG, "batched solve needs q * element size = 16 * 2^i bytes (<= 512)");
    // sets may live on different bases (sectors of other 2M or particle
    // numbers): each keeps its own dimension, tables and work list
    all_fast = dtype == TRBL_F32;
    Ds.assign(nset, 0);
    voff.assign(nset, 0);
    vtotal = 0;
    nwork = 0;
    for (int i = 0; i < nset; ++i) {
      if (!hs[i]) return fail(TRBL_ERR_ARG, "null Hamiltonian in the batch (set %d)", i);
      if (!hs[i]->garena) return fail(TRBL_ERR_ARG, "the grouped product is not available for the basis of set %d", i);
      if (hs[i]->row_end >= 0 && (hs[i]->row_begin != 0 || hs[i]->row_end != hs[i]->b->D))
        return fail(TRBL_ERR_ARG, "set %d: the solver needs the product over all rows", i);
      if (hs[i]->rows_per_item != hs[0]->rows_per_item)
        TRY(set_work_items(const_cast<trbl_hamiltonian*>(hs[i]), hs[0]->rows_per_item));
      smem = std::max(smem, grouped_smem_bytes(hs[i], dtype));
      if (dtype == TRBL_F32) {
        smem_fast = std::max(smem_fast, fast_smem_bytes(hs[i]));
        all_fast = all_fast && fast_tables_ok(hs[i], q, q);
      }
      Ds[i] = hs[i]->b->D;
      voff[i] = vtotal;
      vtotal += size_t(Ds[i]) * q;
      D = std::max(D, Ds[i]);
      nwork = std::max(nwork, hs[i]->g32.nwork);
    }
    h0 = hs[0];
    TRBL_CUDA(cudaGetDevice(&device));
    nthreads = int(std::max(1u, std::min(16u, std::thread::hardware_concurrency())));
    rc.assign(nset, TRBL_OK);
    msg.assign(nset, std::string());
    ss.assign(nset, nullptr);
    ev_done.assign(nset, nullptr);
    for (int i = 0; i < nset; ++i) {
      TRBL_CUDA(cudaStreamCreateWithFlags(&ss[i], cudaStreamNonBlocking));
      TRBL_CUDA(cudaEventCreateWithFlags(&ev_done[i], cudaEventDisableTiming));
    }
    TRBL_CUDA(cudaMalloc(&shared, sizeof(T) * vtotal * 2));
    TRBL_CUDA(cudaMalloc(&tables, (sizeof(DevH<T>) + sizeof(DevG<T>)) * nset));
    std::vector<DevH<T>> hv(nset);
    std::vector<DevG<T>> gv(nset);
    for (int i = 0; i < nset; ++i) {
      if constexpr (std::is_same<T, double>::value) {
        hv[i] = hs[i]->d64;
        gv[i] = hs[i]->g64;
      } else {
        hv[i] = hs[i]->d32;
        gv[i] = hs[i]->g32;
      }
    }
    TRBL_CUDA(cudaMemcpy(tables, hv.data(), sizeof(DevH<T>) * nset, cudaMemcpyHostToDevice));
    TRBL_CUDA(cudaMemcpy(static_cast<char*>(tables) + sizeof(DevH<T>) * nset, gv.data(), sizeof(DevG<T>) * nset,
                         cudaMemcpyHostToDevice));
    for (int i = 0; i < nset; ++i) {
      auto* S = new (std::nothrow) Solver<T>{};
      if (!S) return fail(TRBL_ERR_OOM, "host allocation failed");
      sets.push_back(S);
    }
    // set 0 first: it loads the eigensolver's kernel variants for all sets
    rc[0] = setup_set(hs[0], 0);
    if (rc[0] != TRBL_OK) return rc[0];
    for_sets(1, [&](int i) { return setup_set(hs[i], i); });
    for (int i = 0; i < nset; ++i)
      if (rc[i] != TRBL_OK) return fail(rc[i], "batched solve, set %d: %s", i, msg[i].c_str());
    TRY(setup_pointers());
    trace("batch setup: %d sets, %.1f ms", nset, ms_since(t_start));
    return TRBL_OK;
  }

  // Device arrays of the sets' pointers for the batched step.
  int setup_pointers() {
    const size_t np = size_t(nset);
    const size_t bytes = np * (5 * sizeof(T*) + 8 * sizeof(double*)) + np * sizeof(SetPtrs<T>) + 3 * np * sizeof(int) +
                         np * sizeof(int64_t) + 512;
    TRBL_CUDA(cudaMalloc(&bptr, bytes));
    TRBL_CUDA(cudaMallocHost(&hsp, np * sizeof(SetPtrs<T>)));
    TRBL_CUDA(cudaMallocHost(&hcounts, (3 * np + 4) * sizeof(int)));
    std::vector<char> host(bytes);
    size_t off = 0;
    auto place = [&](auto** dev, auto f) {
      using P = std::remove_reference_t<decltype(**dev)>;
      *dev = reinterpret_cast<P*>(static_cast<char*>(bptr) + off);
      P* h = reinterpret_cast<P*>(host.data() + off);
      for (int i = 0; i < nset; ++i) h[i] = f(*sets[i]);
      off += np * sizeof(P);
    };
    place(&P_basis, [](Solver<T>& S) { return S.basis; });
    place(&P_W, [](Solver<T>& S) { return S.W; });
    place(&P_W2, [](Solver<T>& S) { return S.W2; });
    place(&P_Vk, [](Solver<T>& S) { return S.Vk; });
    place(&P_C1, [](Solver<T>& S) { return S.C; });
    place(&P_C2, [&](Solver<T>& S) { return S.C + size_t(mb) * q; });
    place(&P_G, [](Solver<T>& S) { return S.G; });
    place(&P_R1i, [](Solver<T>& S) { return S.R1i; });
    place(&P_R2i, [](Solver<T>& S) { return S.R2i; });
    place(&P_part, [](Solver<T>& S) { return S.ws.partial; });
    place(&P_Bl, [](Solver<T>& S) { return S.basis; });
    place(&P_Cl, [](Solver<T>& S) { return S.Cl; });
    place(&P_Gn, [](Solver<T>& S) { return S.Gn; });
    off = (off + 15) & ~size_t(15);
    dsp = reinterpret_cast<SetPtrs<T>*>(static_cast<char*>(bptr) + off);
    for (int i = 0; i < nset; ++i) {
      Solver<T>& S = *sets[i];
      hsp[i] = SetPtrs<T>{S.basis, S.Vk, S.C, S.G, S.R1, S.R1i, S.R2, S.R2i, S.beta, S.Tm, S.flags, 0.0, Ds[i]};
    }
    off += np * sizeof(SetPtrs<T>);
    off = (off + 15) & ~size_t(15);
    P_D = reinterpret_cast<int64_t*>(static_cast<char*>(bptr) + off);
    std::memcpy(host.data() + off, Ds.data(), np * sizeof(int64_t));
    off += np * sizeof(int64_t);
    dcounts = reinterpret_cast<int*>(static_cast<char*>(bptr) + off);
    off += 2 * np * sizeof(int);
    dskip = reinterpret_cast<int*>(static_cast<char*>(bptr) + off);
    std::memset(host.data() + off, 0, np * sizeof(int));
    part_bytes = sets[0]->ws.partial_bytes;
    TRBL_CUDA(cudaMemcpy(bptr, host.data(), bytes, cudaMemcpyHostToDevice));
    return TRBL_OK;
  }

  // One block step of every set (Alg. 4 after the product): the selective
  // reorthogonalisation (or CGS2 with TRBL_REORTH_TWICE) against each basis, alpha into T, Cholesky QR twice, beta and the append of
  // V_{k+1}, each a single launch over all sets; then the deficiency counts
  // and wait-timeout words to pinned host memory.
  int enqueue(bool append) {
    const void* gtab = static_cast<char*>(tables) + sizeof(DevH<T>) * nset;
    int rf = -1;
    if (dtype == TRBL_F32)
      rf = launch_fast_batch(h0, all_fast, tables, gtab, nset, nwork, smem_fast, P_Vk, q, P_W, q, q, s);
    if (rf == -1)
      TRY(launch_grouped_batch(tables, gtab, nset, nwork, smem, P_Vk, q, P_W, q, q, dtype, s));
    else if (rf != TRBL_OK)
      return rf;
    const int nb = sets[0]->nb;
    const T* const* cB = P_basis;
    const T* const* cW = P_W;
    const T* const* cW2 = P_W2;
    const dim3 gq{unsigned((q * q + 127) / 128), unsigned(nset), 1u};
    if (prm.reorth == TRBL_REORTH_TWICE) {
      TRY(block_dot_batched<T>(cB, mb, nb, cW, q, q, P_D, D, P_C1, P_part, part_bytes, nset, s));
      TRY(rowgemm_batched<T>(cB, mb, nb, P_C1, q, q, P_W, q, P_D, D, -1.0, 1.0, nset, s));
      TRY(block_dot_batched<T>(cB, mb, nb, cW, q, q, P_D, D, P_C2, P_part, part_bytes, nset, s));
      TRY(rowgemm_batched<T>(cB, mb, nb, P_C2, q, q, P_W, q, P_D, D, -1.0, 1.0, nset, s));
      set_alpha_batched_kernel<T><<<gq, 128, 0, s>>>(dsp, mb, nb - q, q); note_launch();
      TRY(block_dot_batched<T>(cW, q, q, cW, q, q, P_D, D, P_G, P_part, part_bytes, nset, s));
    } else {
      // the single solver's selective pass, with the DGKS decision taken on
      // the device: the second full pass (and the Gram matrix after it) runs
      // for the sets whose flag asks for it, the others return at once
      constexpr int kAlign = int(16 / sizeof(T));
      const int c0 = std::max(0, nb - 2 * q) / kAlign * kAlign;
      const int ql = nb - c0;
      offset_ptrs_kernel<T><<<(nset + 127) / 128, 128, 0, s>>>(P_basis, c0, P_Bl, nset); note_launch();
      const T* const* cBl = P_Bl;
      TRY(block_dot_batched<T>(cBl, mb, ql, cW, q, q, P_D, D, P_Cl, P_part, part_bytes, nset, s));
      TRY(rowgemm_batched<T>(cBl, mb, ql, P_Cl, q, q, P_W, q, P_D, D, -1.0, 1.0, nset, s));
      TRY(col_sumsq_batched<T>(cW, q, q, P_D, D, P_Gn, P_part, part_bytes, sets[0]->ws.sm_count, nset, s));
      TRY(block_dot_batched<T>(cB, mb, nb, cW, q, q, P_D, D, P_C1, P_part, part_bytes, nset, s));
      TRY(rowgemm_batched<T>(cB, mb, nb, P_C1, q, q, P_W, q, P_D, D, -1.0, 1.0, nset, s));
      TRY(block_dot_batched<T>(cW, q, q, cW, q, q, P_D, D, P_G, P_part, part_bytes, nset, s));
      dgks_flags_kernel<<<(nset + 127) / 128, 128, 0, s>>>(P_G, P_Gn, q, dskip, nset); note_launch();
      TRY(block_dot_batched<T>(cB, mb, nb, cW, q, q, P_D, D, P_C2, P_part, part_bytes, nset, s, dskip));
      TRY(rowgemm_batched<T>(cB, mb, nb, P_C2, q, q, P_W, q, P_D, D, -1.0, 1.0, nset, s, dskip));
      TRY(block_dot_batched<T>(cW, q, q, cW, q, q, P_D, D, P_G, P_part, part_bytes, nset, s, dskip));
      set_alpha_sel_batched_kernel<T><<<gq, 128, 0, s>>>(dsp, P_Cl, dskip, mb, nb - q, ql, q); note_launch();
    }
    chol_batched_kernel<T><<<nset, 64, 0, s>>>(dsp, q, 1, 0.0, sets[0]->tau_max); note_launch();
    TRY(rowgemm_batched<T>(cW, q, q, P_R1i, q, q, P_W2, q, P_D, D, 1.0, 0.0, nset, s));
    TRY(block_dot_batched<T>(cW2, q, q, cW2, q, q, P_D, D, P_G, P_part, part_bytes, nset, s));
    chol_batched_kernel<T><<<nset, 64, 0, s>>>(dsp, q, 2, 1e-3, 0.0); note_launch();
    TRY(rowgemm_batched<T>(cW2, q, q, P_R2i, q, q, P_Vk, q, P_D, D, 1.0, 0.0, nset, s));
    beta_batched_kernel<T><<<gq, 128, 0, s>>>(dsp, mb, nb, nb - q, q, append ? 1 : 0); note_launch();
    if (append) {
      const dim3 ga{unsigned((D * q + 255) / 256), unsigned(nset), 1u};
      append_batched_kernel<T><<<ga, 256, 0, s>>>(dsp, q, mb, nb); note_launch();
    }
    gather_counts_kernel<T><<<(nset + 127) / 128, 128, 0, s>>>(dsp, nset, dcounts); note_launch();
    TRBL_CUDA(cudaGetLastError());
    TRBL_CUDA(cudaMemcpyAsync(hcounts, dcounts, sizeof(int) * 2 * nset, cudaMemcpyDeviceToHost, s));
    TRBL_CUDA(cudaMemcpyAsync(hcounts + 2 * nset + 4, dskip, sizeof(int) * nset, cudaMemcpyDeviceToHost, s));
    TRY(tma_error_to_host(hcounts + 2 * nset, s));
    TRY(dot_error_to_host(hcounts + 2 * nset + 1, s));
    TRY(tc_error_to_host(hcounts + 2 * nset + 2, s));
    TRY(wide_error_to_host(hcounts + 2 * nset + 3, s));
    return TRBL_OK;
  }

  // Pivot thresholds of the sets' pass-1 Cholesky (tau ||H||, ||H|| being
  // each set's current estimate) to the device records, before a step.
  int refresh_thresholds() {
    for (int i = 0; i < nset; ++i) hsp[i].thr1 = sets[i]->tau * sets[i]->normH;
    TRBL_CUDA(cudaMemcpyAsync(dsp, hsp, sizeof(SetPtrs<T>) * nset, cudaMemcpyHostToDevice, s));
    return TRBL_OK;
  }

  int graph_for(int nb, bool append, cudaGraphExec_t* out) {
    auto it = graphs.find(nb);
    if (it != graphs.end()) {
      *out = it->second;
      return TRBL_OK;
    }
    cudaGraph_t g = nullptr;
    TRBL_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const int r = enqueue(append);
    const cudaError_t e = cudaStreamEndCapture(s, &g);
    if (r) {
      if (g) cudaGraphDestroy(g);
      return r;
    }
    TRBL_CUDA(e);
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    TRBL_CUDA(ei);
    graphs[nb] = ex;
    *out = ex;
    return TRBL_OK;
  }

  int run(double* evals, double* resid, void* evecs, int* status, trbl_stats* st) {
    const int nev = prm.nev;
    const int max_iter = prm.max_iter > 0 ? prm.max_iter : 100000;
    double since_check = 0, last_check = 0;
    int it = 0;
    for (; it < max_iter; ++it) {
      bool all = true;
      for (int i = 0; i < nset; ++i) all = all && (sets[i]->done || rc[i] != TRBL_OK);
      if (all) break;
      const int nb = sets[0]->nb;
      const bool append = nb + q <= mb;
      const auto t0 = clock::now();
      for (int i = 0; i < nset; ++i) TRBL_CUDA(cudaStreamWaitEvent(s, ev_done[i], 0));
      TRY(refresh_thresholds());
      if (it == 0) {
        TRY(enqueue(append));  // eager first step: lazily configured kernels set up outside capture
      } else {
        cudaGraphExec_t ex;
        TRY(graph_for(nb, append, &ex));
        TRBL_CUDA(cudaGraphLaunch(ex, s));
      }
      TRBL_CUDA(cudaStreamSynchronize(s));
      for (int i = 0; i < nset; ++i) {
        int* hf = sets[i]->hflags;
        hf[kF1] = hcounts[2 * i];
        hf[kF2] = hcounts[2 * i + 1];
        for (int k = 0; k < 4; ++k) hf[kTmaErr + k] = hcounts[2 * nset + k];
        if (prm.reorth != TRBL_REORTH_TWICE && hcounts[2 * nset + 4 + i] == 0) ++second_passes;
      }
      const double t_step = ms_since(t0);
      ms_steps += t_step;
      since_check += t_step;
      // all sets test at the same steps: every check_every steps, or (adaptive)
      // once the steps since the last test took kCheckRatio times as long as it
      const bool due = prm.check_every > 0 ? (it + 1) % prm.check_every == 0 : since_check >= kCheckRatio * last_check;
      const bool check = due || !append;
      const auto t1 = clock::now();
      for_sets(0, [&](int i) {
        TRY(sets[i]->step_after(append, check, max_iter));
        TRBL_CUDA(cudaEventRecord(ev_done[i], ss[i]));
        return TRBL_OK;
      });
      const double t_between = ms_since(t1);
      ms_between += t_between;
      if (check) {
        last_check = t_between;
        since_check = 0;
      }
      trace("batch step %d nb %d: steps %.2f ms, between %.2f ms%s", it, nb, t_step, t_between, check ? " (test)" : "");
    }
    std::vector<char> failed(nset);
    for (int i = 0; i < nset; ++i) failed[i] = rc[i] != TRBL_OK;
    for_sets(0, [&](int i) {
      const int r = sets[i]->finish(evals + size_t(i) * nev, resid ? resid + size_t(i) * nev : nullptr,
                                    evecs ? static_cast<T*>(evecs) + voff[i] / q * nev : nullptr, nullptr);
      const cudaError_t e = cudaStreamSynchronize(ss[i]);
      if (r == TRBL_OK && e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize (batched finish)");
      return r;
    });
    int worst = TRBL_OK, first = -1, nbad = 0, conv = 0;
    for (int i = 0; i < nset; ++i) {
      if (failed[i])
        for (int k = 0; k < nev; ++k) evals[size_t(i) * nev + k] = NAN;
      if (status) status[i] = rc[i];
      if (rc[i] != TRBL_OK) {
        ++nbad;
        if (first < 0) {
          first = i;
          worst = rc[i];
        }
      }
      conv += sets[i]->conv;
    }
    if (st) {
      *st = trbl_stats{};
      st->iterations = it;
      st->restarts = sets[0]->restarts;
      st->converged = conv;
      st->status = worst;
      st->normH = sets[0]->normH;
      st->ms_total = ms_since(t_start);
      st->ms_apply = ms_steps;
      st->ms_ritz = ms_between;
      st->second_passes = int(std::min<int64_t>(second_passes, 0x7fffffff));
    }
    trace("batch: %d steps, steps %.1f ms, between %.1f ms, total %.1f ms", it, ms_steps, ms_between,
          ms_since(t_start));
    if (worst != TRBL_OK)
      return fail(worst, "batched solve: %d of %d sets did not finish cleanly; set %d: %s", nbad, nset, first,
                  msg[first].c_str());
    return TRBL_OK;
  }
};

}  // namespace
}  // namespace trbl

struct trbl_solver {
  trbl_params params;
  cudaStream_t stream = nullptr;
  trbl::SolverBase* impl = nullptr;
  cudaEvent_t cev[4] = {nullptr, nullptr, nullptr, nullptr};  // host-buffer copies: in begin/end, out begin/end
  double ms_copy_in = 0, ms_copy_out = 0;
  ~trbl_solver() {
    delete impl;
    for (cudaEvent_t e : cev)
      if (e) cudaEventDestroy(e);
  }
};

using namespace trbl;

extern "C" int trbl_solver_create(const trbl_hamiltonian* h, const trbl_params* p, void* stream,
                                  trbl_solver** out) {
  clear_error();
  if (!out) return fail(TRBL_ERR_ARG, "out is null");
  *out = nullptr;
  if (!h || !p) return fail(TRBL_ERR_ARG, "null argument");
  trbl_solver* sv = new (std::nothrow) trbl_solver();
  if (!sv) return fail(TRBL_ERR_OOM, "host allocation failed");
  sv->params = *p;
  sv->stream = static_cast<cudaStream_t>(stream);
  int rc = TRBL_OK;
  auto make = [&](auto* impl) {
    if (!impl) {
      rc = fail(TRBL_ERR_OOM, "host allocation failed");
      return;
    }
    impl->S.h = h;
    impl->S.p = &sv->params;
    impl->S.s = sv->stream;
    sv->impl = impl;
    rc = impl->S.setup();
    if (rc == TRBL_OK) rc = impl->init();
  };
  if (p->precision == TRBL_PREC_F64)
    make(new (std::nothrow) SolverImpl<double>());
  else if (p->precision == TRBL_PREC_MIXED)
    make(new (std::nothrow) SolverImpl<float>());
  else
    rc = fail(TRBL_ERR_ARG, "precision must be TRBL_PREC_F64 or TRBL_PREC_MIXED");
  if (rc != TRBL_OK) {
    delete sv;
    return rc;
  }
  *out = sv;
  return TRBL_OK;
}

extern "C" int trbl_solver_step(trbl_solver* sv, int* converged) {
  clear_error();
  if (!sv || !sv->impl) return fail(TRBL_ERR_ARG, "null solver");
  return sv->impl->step(converged);
}

extern "C" int trbl_solver_step_host(trbl_solver* sv, const void* block_in, void* block_out, int* converged) {
  clear_error();
  if (!sv || !sv->impl) return fail(TRBL_ERR_ARG, "null solver");
  const size_t bytes = sv->impl->block_bytes();
  // the two copies are timed with events on the solver's stream
  if (!sv->cev[0])
    for (auto& e : sv->cev) TRBL_CUDA(cudaEventCreate(&e));
  cudaEvent_t* ev = sv->cev;
  TRBL_CUDA(cudaEventRecord(ev[0], sv->stream));
  if (block_in)
    TRBL_CUDA(cudaMemcpyAsync(sv->impl->block(), block_in, bytes, cudaMemcpyHostToDevice, sv->stream));
  TRBL_CUDA(cudaEventRecord(ev[1], sv->stream));
  int rc = sv->impl->step(converged);
  if (rc) return rc;
  float in_ms = 0.f, out_ms = 0.f;
  if (block_out) {
    TRBL_CUDA(cudaEventRecord(ev[2], sv->stream));
    TRBL_CUDA(cudaMemcpyAsync(block_out, sv->impl->block(), bytes, cudaMemcpyDeviceToHost, sv->stream));
    TRBL_CUDA(cudaEventRecord(ev[3], sv->stream));
    TRBL_CUDA(cudaStreamSynchronize(sv->stream));
    TRBL_CUDA(cudaEventElapsedTime(&out_ms, ev[2], ev[3]));
  }
  TRBL_CUDA(cudaEventSynchronize(ev[1]));
  TRBL_CUDA(cudaEventElapsedTime(&in_ms, ev[0], ev[1]));
  if (block_in) sv->ms_copy_in += in_ms;
  sv->ms_copy_out += out_ms;
  trace("step_host: copy in %.2f ms, copy out %.2f ms (%zu bytes each)", in_ms, out_ms, bytes);
  return TRBL_OK;
}

extern "C" int trbl_solver_state_bytes(trbl_solver* sv, int64_t* bytes) {
  clear_error();
  if (!sv || !sv->impl || !bytes) return fail(TRBL_ERR_ARG, "null argument");
  *bytes = int64_t(sv->impl->state_bytes());
  return TRBL_OK;
}

extern "C" int trbl_solver_save(trbl_solver* sv, void* host, int64_t bytes) {
  clear_error();
  if (!sv || !sv->impl) return fail(TRBL_ERR_ARG, "null solver");
  return sv->impl->save(host, bytes);
}

extern "C" int trbl_solver_load(trbl_solver* sv, const void* host, int64_t bytes) {
  clear_error();
  if (!sv || !sv->impl) return fail(TRBL_ERR_ARG, "null solver");
  return sv->impl->load(host, bytes);
}

extern "C" int trbl_solver_block(trbl_solver* sv, void** block, int64_t* bytes) {
  clear_error();
  if (!sv || !sv->impl) return fail(TRBL_ERR_ARG, "null solver");
  if (block) *block = sv->impl->block();
  if (bytes) *bytes = int64_t(sv->impl->block_bytes());
  return TRBL_OK;
}

extern "C" int trbl_solver_stats(trbl_solver* sv, trbl_stats* st) {
  clear_error();
  if (!sv || !sv->impl || !st) return fail(TRBL_ERR_ARG, "null argument");
  *st = trbl_stats{};
  sv->impl->stats(st);
  st->ms_copy_in = sv->ms_copy_in;
  st->ms_copy_out = sv->ms_copy_out;
  return TRBL_OK;
}

extern "C" int trbl_solver_finish(trbl_solver* sv, double* evals, double* resid, void* evecs,
                                  trbl_stats* stats) {
  clear_error();
  if (!sv || !sv->impl || !evals) return fail(TRBL_ERR_ARG, "null argument");
  if (stats) *stats = trbl_stats{};
  int rc = sv->impl->finish(evals, resid, evecs, stats);
  if (stats) stats->status = rc;
  return rc;
}

extern "C" void trbl_solver_destroy(trbl_solver* sv) {
  if (!sv) return;
  if (sv->stream) cudaStreamSynchronize(sv->stream);
  delete sv;
}

extern "C" int trbl_solve(const trbl_hamiltonian* h, const trbl_params* p, double* evals, double* resid,
                          void* evecs, trbl_stats* stats, void* stream) {
  clear_error();
  if (!h || !p || !evals) return fail(TRBL_ERR_ARG, "null argument");
  if (stats) *stats = trbl_stats{};
  trbl_solver* sv = nullptr;
  int rc = trbl_solver_create(h, p, stream, &sv);
  if (rc != TRBL_OK) {
    if (stats) stats->status = rc;
    return rc;
  }
  const int max_iter = p->max_iter > 0 ? p->max_iter : 100000;
  while (rc == TRBL_OK && !sv->impl->is_done() && sv->impl->iterations() < max_iter) rc = sv->impl->step(nullptr);
  const bool refine = p->refine && p->precision == TRBL_PREC_MIXED;
  std::vector<double> rloc;
  double* rr = resid;
  if (refine && !rr) {
    rloc.assign(size_t(p->nev), 0.0);
    rr = rloc.data();
  }
  if (rc == TRBL_OK) rc = trbl_solver_finish(sv, evals, rr, evecs, stats);
  // Refinement: the estimate bounds the residual of the FP32 Lanczos
  // recurrence; the FP32 vectors and product add a floor of their own, so a
  // true residual may exceed tol when the estimate meets it.  Taking the
  // floor as the measured gap (true^2 - estimate^2), lower the estimate's
  // target so that both together stay below 0.9 tol, and step on; stop when
  // the true residuals meet tol, the floor alone reaches 0.9 tol, or after
  // three rounds.
  double scale = 1.0;
  for (int round = 0; refine && rc == TRBL_OK && round < 3; ++round) {
    const double lim = p->tol * sv->impl->norm_h();
    double worst = 0.0;
    for (int i = 0; i < p->nev; ++i)
      if (std::isfinite(rr[i])) worst = std::max(worst, rr[i]);
    if (worst <= lim || sv->impl->iterations() >= max_iter) break;
    const double est = lim * scale, target = 0.9 * lim;
    const double floor2 = std::max(0.0, worst * worst - est * est);
    if (floor2 >= target * target) break;
    double next = std::sqrt(target * target - floor2) / lim;
    if (!(next < scale)) next = 0.8 * scale;
    scale = next;
    trace("refine round %d: worst true residual %.3g of tol %.3g, estimate target %.3f tol", round, worst / lim * p->tol,
          p->tol, scale);
    sv->impl->retarget(scale);
    while (rc == TRBL_OK && !sv->impl->is_done() && sv->impl->iterations() < max_iter) rc = sv->impl->step(nullptr);
    if (rc == TRBL_OK) rc = trbl_solver_finish(sv, evals, rr, evecs, stats);
  }
  std::string keep = trbl_last_error();
  trbl_solver_destroy(sv);
  if (rc != TRBL_OK) fail(rc, "%s", keep.c_str());
  if (stats) stats->status = rc;
  return rc;
}

extern "C" int trbl_solve_batch(const trbl_hamiltonian* const* hs, int nset, const trbl_params* p, double* evals,
                                double* resid, void* evecs, int* status, trbl_stats* stats, void* stream) {
  clear_error();
  if (!hs || nset < 1 || !p || !evals) return fail(TRBL_ERR_ARG, "null argument or empty batch");
  // CUDA graphs cannot be captured on the legacy default stream: run on a
  // private stream ordered after the caller's.
  cudaStream_t caller = static_cast<cudaStream_t>(stream);
  cudaStream_t s = nullptr;
  cudaEvent_t ready = nullptr;
  TRBL_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  TRBL_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
  TRBL_CUDA(cudaEventRecord(ready, caller));
  TRBL_CUDA(cudaStreamWaitEvent(s, ready, 0));
  int rc;
  if (p->precision == TRBL_PREC_F64) {
    BatchDriver<double> B;
    B.prm = *p;
    B.s = s;
    B.nset = nset;
    rc = B.setup(hs);
    if (!rc) rc = B.run(evals, resid, evecs, status, stats);
  } else if (p->precision == TRBL_PREC_MIXED) {
    BatchDriver<float> B;
    B.prm = *p;
    B.s = s;
    B.nset = nset;
    rc = B.setup(hs);
    if (!rc) rc = B.run(evals, resid, evecs, status, stats);
  } else {
    rc = fail(TRBL_ERR_ARG, "precision must be TRBL_PREC_F64 or TRBL_PREC_MIXED");
  }
  cudaStreamSynchronize(s);
  cudaEventDestroy(ready);
  cudaStreamDestroy(s);
  return rc;
}
