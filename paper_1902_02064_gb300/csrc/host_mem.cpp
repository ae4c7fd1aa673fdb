// Pinned host buffers for the host-buffer solver steps
// (trbl_solver_step_host): cudaHostAlloc (portable, page-locked) memory
// placed on the host memory node nearest the GPU.
//
// Placement.  A page-locked page is allocated when cudaHostAlloc runs, by
// the calling thread, so the thread's NUMA memory policy decides its node.
// trbl_host_alloc binds the calling thread's policy to the GPU's nearest node
// (cudaDevAttrHostNumaId) for the duration of the call and restores it after
// (set_mempolicy / get_mempolicy system calls; where they are refused or the
// device reports no node, the default policy applies).  The node that holds
// the buffer's first page is reported back (move_pages query), so a caller
// sees where it landed.
//
// An earlier form bound an anonymous mapping with mbind, touched it and
// registered it with cudaHostRegister: its isolated copy rates matched, but
// inside the solver's step loop its host-to-device copies took seconds.
#include <sys/syscall.h>
#include <unistd.h>

#include <cstring>
#include <map>
#include <mutex>

#include "internal.h"

using namespace trbl;

namespace {

std::mutex g_mu;
std::map<void*, size_t> g_bufs;  // live buffers and their sizes

constexpr int kMpolDefault = 0;     // MPOL_DEFAULT
constexpr int kMpolBind = 2;        // MPOL_BIND
constexpr unsigned long kMaxNode = 1024;
constexpr int kWords = int(kMaxNode / (8 * sizeof(unsigned long)));

// The calling thread's policy, to restore after the allocation.
struct Policy {
  int mode = kMpolDefault;
  unsigned long mask[kWords] = {};
  bool saved = false;
};

bool get_policy(Policy* p) {
#if defined(SYS_get_mempolicy)
  p->saved = syscall(SYS_get_mempolicy, &p->mode, p->mask, kMaxNode, nullptr, 0UL) == 0;
#endif
  return p->saved;
}

bool bind_to(int node) {
#if defined(SYS_set_mempolicy)
  if (node < 0 || node >= int(kMaxNode)) return false;
  unsigned long mask[kWords] = {};
  mask[node / (8 * sizeof(unsigned long))] = 1UL << (node % (8 * sizeof(unsigned long)));
  return syscall(SYS_set_mempolicy, kMpolBind, mask, kMaxNode) == 0;
#else
  (void)node;
  return false;
#endif
}

void restore(const Policy& p) {
#if defined(SYS_set_mempolicy)
  if (p.saved)
    syscall(SYS_set_mempolicy, p.mode, p.mode == kMpolDefault ? nullptr : p.mask,
            p.mode == kMpolDefault ? 0UL : kMaxNode);
  else
    syscall(SYS_set_mempolicy, kMpolDefault, nullptr, 0UL);
#else
  (void)p;
#endif
}

// Node of the page at p (-1 if the query is not available).
int page_node(void* p) {
#if defined(SYS_move_pages)
  void* pages[1] = {p};
  int status[1] = {-1};
  if (syscall(SYS_move_pages, 0, 1UL, pages, nullptr, status, 0) == 0 && status[0] >= 0) return status[0];
#else
  (void)p;
#endif
  return -1;
}

}  // namespace

extern "C" int trbl_host_alloc(size_t bytes, int device, void** out, int* numa_node) {
  clear_error();
  if (!out || bytes == 0) return fail(TRBL_ERR_ARG, "null output or zero size");
  *out = nullptr;
  int node = -1;
  if (cudaDeviceGetAttribute(&node, cudaDevAttrHostNumaId, device) != cudaSuccess) {
    cudaGetLastError();
    node = -1;
  }
  Policy old;
  const bool bound = node >= 0 && get_policy(&old) && bind_to(node);
  void* p = nullptr;
  const cudaError_t e = cudaHostAlloc(&p, bytes, cudaHostAllocPortable);
  if (bound) restore(old);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? TRBL_ERR_OOM : TRBL_ERR_CUDA, "cudaHostAlloc of %zu bytes: %s",
                bytes, cudaGetErrorString(e));
  }
  if (numa_node) {
    const int at = page_node(p);
    *numa_node = at >= 0 ? at : node;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  g_bufs[p] = bytes;
  *out = p;
  return TRBL_OK;
}

extern "C" int trbl_host_free(void* p) {
  clear_error();
  if (!p) return TRBL_OK;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_bufs.find(p);
    if (it == g_bufs.end()) return fail(TRBL_ERR_ARG, "not a buffer of trbl_host_alloc");
    g_bufs.erase(it);
  }
  TRBL_CUDA(cudaFreeHost(p));
  return TRBL_OK;
}
