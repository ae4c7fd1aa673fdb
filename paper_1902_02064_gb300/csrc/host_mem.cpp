// Pinned host buffers on the host memory node closest to a GPU, for the
// host-buffer solver steps (trbl_solver_step_host): a block copied between
// the host and the GPU every step moves at the speed of the link between the
// GPU and the memory node the pages sit on, so pages first touched by a
// thread on another node cross the inter-socket link as well.
//
// The buffer is an anonymous mapping bound to the node with the mbind system
// call, touched page by page on this thread (placing every page there), then
// page-locked with cudaHostRegister.  Where the device reports no host node
// or the binding is refused, it is plain cudaMallocHost memory.
#include <sys/mman.h>
#include <sys/syscall.h>
#include <unistd.h>

#include <cstring>
#include <map>
#include <mutex>

#include "internal.h"

using namespace trbl;

namespace {

constexpr int kMpolBind = 2;  // MPOL_BIND of the Linux memory-policy interface

struct HostBuf {
  size_t bytes;
  bool mapped;  // mmap + cudaHostRegister (else cudaMallocHost)
};
std::mutex g_mu;
std::map<void*, HostBuf> g_bufs;

// Binds [p, p + bytes) to NUMA node `node`; false when the kernel refuses.
bool bind_to_node(void* p, size_t bytes, int node) {
  if (node < 0 || node >= 1024) return false;
  unsigned long mask[1024 / (8 * sizeof(unsigned long))] = {};
  mask[node / (8 * sizeof(unsigned long))] = 1ul << (node % (8 * sizeof(unsigned long)));
  const long r = syscall(SYS_mbind, p, bytes, kMpolBind, mask, 1024ul, 0u);
  return r == 0;
}

}  // namespace

extern "C" int trbl_host_alloc(size_t bytes, int device, void** out, int* numa_node) {
  clear_error();
  if (!out || bytes == 0) return fail(TRBL_ERR_ARG, "null output or zero size");
  *out = nullptr;
  if (numa_node) *numa_node = -1;
  int node = -1;
  if (cudaDeviceGetAttribute(&node, cudaDevAttrHostNumaId, device) != cudaSuccess) {
    cudaGetLastError();
    node = -1;
  }
  const size_t page = size_t(sysconf(_SC_PAGESIZE));
  const size_t len = (bytes + page - 1) / page * page;
  if (node >= 0) {
    void* p = mmap(nullptr, len, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
    if (p != MAP_FAILED) {
      if (bind_to_node(p, len, node)) {
        std::memset(p, 0, len);  // first touch: every page on the bound node
        if (cudaHostRegister(p, len, cudaHostRegisterDefault) == cudaSuccess) {
          std::lock_guard<std::mutex> lk(g_mu);
          g_bufs[p] = HostBuf{len, true};
          *out = p;
          if (numa_node) *numa_node = node;
          return TRBL_OK;
        }
        cudaGetLastError();
      }
      munmap(p, len);
    }
  }
  void* p = nullptr;
  TRBL_CUDA(cudaMallocHost(&p, bytes));
  std::lock_guard<std::mutex> lk(g_mu);
  g_bufs[p] = HostBuf{bytes, false};
  *out = p;
  return TRBL_OK;
}

extern "C" int trbl_host_free(void* p) {
  clear_error();
  if (!p) return TRBL_OK;
  HostBuf b;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_bufs.find(p);
    if (it == g_bufs.end()) return fail(TRBL_ERR_ARG, "not a buffer of trbl_host_alloc");
    b = it->second;
    g_bufs.erase(it);
  }
  if (b.mapped) {
    const cudaError_t e = cudaHostUnregister(p);
    munmap(p, b.bytes);
    TRBL_CUDA(e);
    return TRBL_OK;
  }
  TRBL_CUDA(cudaFreeHost(p));
  return TRBL_OK;
}
