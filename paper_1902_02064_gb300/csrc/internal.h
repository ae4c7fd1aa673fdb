// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/trbl.h"

namespace trbl {

// Records a message for trbl_last_error() and returns `code`.
int fail(int code, const char* fmt, ...);
// Clears the thread's error message (start of every entry point).
void clear_error();
// Counts one launch of a library kernel (trbl_kernel_launches).
void note_launch();
// TRBL_ERR_CUDA with the call site and CUDA's message when e != cudaSuccess.
int cuda_fail(cudaError_t e, const char* what);

#define TRBL_CUDA(call)                                                  \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) return ::trbl::cuda_fail(e_, #call);          \
  } while (0)

// One species of the two-species basis.
struct Species {
  int n = 0, k = 0;
  std::vector<int> twom;
  std::vector<uint32_t> bits;   // determinants, sorted by (2M, value)
  std::vector<int32_t> dM;      // 2M of each determinant
  std::vector<int32_t> group;   // determinant -> group index
  std::vector<int32_t> gM, gfirst, gcount;  // groups of equal 2M, ascending
  // One-body jumps gathered by target: entries of target t with 2m transfer
  // index di are [jseg[t*ND+di], jseg[t*ND+di+1]).
  std::vector<int32_t> jseg;
  std::vector<int32_t> jsrc;    // global source determinant
  std::vector<int32_t> ja, jc;  // a+_a a_c
  std::vector<int8_t> jsign;
  int find(uint32_t b, int M) const;  // global index or -1
  int group_of_M(int M) const;        // group index or -1
};

struct Block {
  int mA, mB;
  int64_t off;
  int na, nb;
  int gA, gB;  // group indices in species A and B
};

}  // namespace trbl

struct trbl_basis {
  trbl::Species sp[2];
  int twoM = 0;
  int dspan = 0;  // 2m transfers lie in [-dspan, dspan]
  int ND = 1;     // 2*dspan + 1
  std::vector<trbl::Block> blocks;
  std::vector<int32_t> srcblk;  // [blk*ND + di]: block holding M_A - delta, or -1
  int64_t D = 0;
  int max_group = 0;  // largest 2M group of either species
};

namespace trbl {

// Device-side tables of one Hamiltonian (all pointers are device memory).
template <typename T>
struct DevH {
  int nblk, ND, nA, nB;
  const int64_t* boff;
  const int32_t* bnb;
  const int32_t* bgA;   // first A determinant of the block's A group
  const int32_t* bgB;
  const int32_t* srcblk;
  // one-body jumps by target: (source local index, op = (a*n+c)<<1 | negative)
  const int32_t* jsegA;
  const int2* jA;
  const int32_t* jsegB;
  const int2* jB;
  // like-particle H rows by target determinant: source local index, coefficient
  const int32_t* hoffA;
  const int32_t* hsrcA;
  const T* hcoefA;
  const int32_t* hoffB;
  const int32_t* hsrcB;
  const T* hcoefB;
  // cross-species table vab[(a*nA+c)*nB*nB + b*nB+d] = V^AB_{ab,cd}
  const T* vab;
};

// Extra tables of the grouped block-product kernel (apply_grouped.cu).
template <typename T>
struct DevG {
  const int4* work;     // (target A determinant, block, first neutron row, row count)
  int nwork;
  int maxP, maxQ, maxK; // per-target proton jumps, like-particle A sources, coefficient row length
  const int2* jB2;      // neutron jumps: (source local index, (k << 9) | (transfer << 1) | negative), k = pair index in its 2m-transfer class
  const T* ccoef;       // ccoef[(a*nA + c) * maxK + k] = V^AB_{a b_k, c d_k} for the class of transfer m_c - m_a
  const int2* likeB;    // FP32 tables only: species-B like-particle rows as (source local index, FP32 coefficient bits)
};

// Tables of the source-stationary cross-species kernel (apply_pn.cu).
struct DevPN {
  const int32_t* oseg;  // outgoing neutron jumps of source determinant n (global) with transfer index tn:
                        // entries [oseg[n*ND+tn], oseg[n*ND+tn+1])
  const int32_t* jout;  // (target local index in its 2M group << 8) | (k << 1) | negative, k = pair index in its class
  const int32_t* ncls;  // [ND] neutron pairs (b, d) per transfer class
  const int2* slabs;    // target slabs (A determinant, block), largest first
  int nslab;
  int maxPc;            // largest number of proton jumps into one determinant from one transfer class
  int nbmax;            // largest neutron group of a block
  int maxCoef;          // largest sum over classes of (proton jumps x pairs of the class) of one determinant
};

}  // namespace trbl

struct trbl_hamiltonian {
  const trbl_basis* b = nullptr;
  int device = 0;
  // host copies of the like-particle rows (by target, global determinant index)
  std::vector<int32_t> hoff[2], hsrc[2];
  std::vector<double> hcoef[2];
  std::vector<double> vab;  // (a*nA+c)*nB*nB + b*nB+d
  // device allocations (one arena)
  void* arena = nullptr;
  trbl::DevH<double> d64;
  trbl::DevH<float> d32;
  trbl::DevG<double> g64;
  trbl::DevG<float> g32;
  void* garena = nullptr;
  void* gwork = nullptr;   // work items of the grouped kernel
  trbl::DevPN pn{};        // source-stationary cross-species kernel (pn.oseg null: not available)
  void* pnarena = nullptr;
  void* pnslabs = nullptr;
  int rows_per_item = 0;   // neutron rows per work item (autotuned)
  int apply_kernel = TRBL_APPLY_FAST;  // FP32 product: TRBL_APPLY_FAST where it applies, else the grouped kernel
  int blocks_per_sm = 8;   // resident thread blocks per SM the FP32 fast kernel is compiled for (8 or 6)
  int apply_compensated = 0;  // FP32 fast kernel: compensated (TwoSum) row sums
  int64_t row_begin = 0, row_end = -1;  // rows of W the product computes (slab-aligned; -1: all)
  void* grad = nullptr;  // gradient tables, built on the first trbl_grad call
  size_t arena_bytes = 0;
};

// Frees the gradient tables of a Hamiltonian (grad.cu).
void trbl_grad_state_free(void* g);

namespace trbl {
// Uploads the tables of h to the current device (apply.cu).
int upload_tables(trbl_hamiltonian* h);
// Builds and uploads the grouped-kernel tables (apply_grouped.cu).
int upload_grouped(trbl_hamiltonian* h);
// Builds and uploads the source-stationary cross-species tables
// (apply_pn.cu); kidx[b*nB+d] = index of the neutron pair (b, d) in its
// transfer class, ncls = pairs per class.  Leaves the kernel unavailable
// (h->pn.oseg null) when its shared memory would not fit.
int upload_pn(trbl_hamiltonian* h, const std::vector<int>& kidx, const std::vector<int>& ncls, int maxK);
// Replaces the source-stationary kernel's list of target slabs (those inside
// the Hamiltonian's row range).
int set_pn_slabs(trbl_hamiltonian* h);
// The split product (like-particle terms by the grouped kernel, then the
// cross-species term by the source-stationary kernel) when h->apply_kernel
// is TRBL_APPLY_SPLIT and it applies; -1 (nothing launched) otherwise.
int launch_split(const trbl_hamiltonian* h, const void* V, int64_t ldv, void* W, int64_t ldw, int q, int dtype,
                 cudaStream_t s);
// Floats per stage of the staged cross-term kernel for h; 0 when its shared
// memory does not fit.
int pn_tma_stage_floats(const trbl_hamiltonian* h);
// Wait-timeout word of the staged cross-term kernel (stream-ordered copy to
// host memory).
int pn_tma_error_to_host(int* host, cudaStream_t s);
// The grouped kernel without the cross-species term (FP32); -1 when it does
// not apply.
int launch_grouped_like(const trbl_hamiltonian* h, const float* V, int64_t ldv, float* W, int64_t ldw, int q,
                        cudaStream_t s);
// Replaces the grouped kernel's work items (rows_per_item rows each), for
// the target slabs inside the Hamiltonian's row range.
int set_work_items(trbl_hamiltonian* h, int rows_per_item);
// Whether row r starts a target slab of the basis (0 and D count).
bool is_slab_boundary(const trbl_basis* b, int64_t r);
// Dynamic shared memory of the grouped kernel for one Hamiltonian.
size_t grouped_smem_bytes(const trbl_hamiltonian* h, int dtype);
// One launch of the grouped kernel over nset Hamiltonians (device arrays of
// DevH<T> / DevG<T>, possibly on bases of different dimension), set s
// reading the device pointer Vs[s] and writing Ws[s]; nwork = the largest
// work list.
int launch_grouped_batch(const void* hs_dev, const void* gs_dev, int nset, int nwork, size_t smem, const void* Vs,
                         int64_t ldv, const void* Ws, int64_t ldw, int q, int dtype, cudaStream_t s);
// Enqueues W = H V with the grouped kernel when q and the alignment allow it;
// returns -1 (nothing launched) otherwise.
int launch_grouped(const trbl_hamiltonian* h, const void* V, int64_t ldv, void* W, int64_t ldw, int q,
                   int dtype, cudaStream_t s);
// FP32 fast product (apply_fast.cu): enqueues W = H V and returns TRBL_OK or
// an error, or returns -1 (nothing launched) when it does not apply (dtype,
// q, alignment, sizes, or h->apply_kernel).
int launch_fast(const trbl_hamiltonian* h, const void* V, int64_t ldv, void* W, int64_t ldw, int q, int dtype,
                cudaStream_t s);
size_t fast_smem_bytes(const trbl_hamiltonian* h);
// The fast product over nset Hamiltonians (device arrays of DevH<float> /
// DevG<float> and of per-set V and W pointers); shape from h0; all = the
// fast kernel applies to every set; -1 when it does not apply.
int launch_fast_batch(const trbl_hamiltonian* h0, bool all, const void* hs_dev, const void* gs_dev, int nset,
                      int nwork, size_t smem, const void* Vs, int64_t ldv, const void* Ws, int64_t ldw, int q,
                      cudaStream_t s);
// Whether the fast kernel can take products of h with row strides ld.
bool fast_tables_ok(const trbl_hamiltonian* h, int64_t ld, int q);
// Enqueues W = H V (apply.cu).
int launch_apply(const trbl_hamiltonian* h, const void* V, int64_t ldv, void* W, int64_t ldw,
                 int q, int dtype, cudaStream_t s);
}  // namespace trbl
