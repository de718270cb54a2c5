// ttn_rdm_noalloc: reduced density matrix of a TTN whose node tensors already
// sit in device memory, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or any allocating routine at all: code
// running inside another framework's memory pool or arena, embedded runtimes
// that forbid allocation after start-up, or hosts that pre-plan every device
// byte. ttn_rdm needs a handle whose workspace the caller allocated; this entry
// point instead takes the caller's node tensors and output buffer and keeps its
// only scratch -- one contraction vector per node -- in a fixed array compiled
// into the library. Every GPU that loads the library holds that array (1 MiB)
// until the process exits.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ttn_heom.h"
#include "kernels.cuh"
#include "plan.hpp"

namespace {

// Scratch of ttn_rdm_noalloc: the per-node vectors v_u (length = rank of the
// bond to the parent). Shared by every call on a device.
constexpr int64_t kRdmScratchComplex = 65536;  // 1 MiB of double2
static __device__ __align__(256) double2 g_rdm_scratch[kRdmScratchComplex];

// Device address of g_rdm_scratch, looked up once per device and kept for the
// life of the process: after cudaDeviceReset (which unloads the module) the
// cached address is stale, so a process that resets a device must not call
// ttn_rdm_noalloc on it again.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double2* g_scratch_ptr[kMaxDevices] = {nullptr};

void set_err(char* buf, size_t len, const std::string& m) {
  if (buf && len > 0) {
    std::strncpy(buf, m.c_str(), len - 1);
    buf[len - 1] = '\0';
  }
}

}  // namespace

extern "C" ttn_status ttn_rdm_noalloc(const ttn_tree* tree, const int32_t* leg_dims, const int32_t* ranks,
                                      const void* const* node_dev, void* rho_dev, void* stream, char* err,
                                      size_t err_len) {
  using namespace ttn;
  if (!tree || !leg_dims || !ranks || !node_dev || !rho_dev) {
    set_err(err, err_len, "null argument");
    return TTN_EINVAL;
  }
  Plan p;
  std::string e = p.build(tree->n_nodes, tree->parent, tree->n_legs, tree->leg_node, leg_dims, ranks);
  if (!e.empty()) {
    set_err(err, err_len, e);
    return e.rfind("UNSUPPORTED", 0) == 0 ? TTN_EUNSUPPORTED : TTN_EINVAL;
  }
  // scratch layout: node u's vector at offset off[u], length dims[u][0]
  std::vector<int64_t> off(p.tree.n_nodes, 0);
  int64_t need = 0;
  for (int u = 0; u < p.tree.n_nodes; ++u) {
    off[u] = need;
    if (u != 0) need += p.dims[u][0];
  }
  if (need > kRdmScratchComplex) {
    set_err(err, err_len,
            "ttn_rdm_noalloc: the tree needs " + std::to_string(need) +
                " complex scratch entries (sum of bond ranks); the fixed limit is " +
                std::to_string(kRdmScratchComplex));
    return TTN_EINVAL;
  }
  for (int u = 0; u < p.tree.n_nodes; ++u)
    if (!node_dev[u]) {
      set_err(err, err_len, "null node pointer");
      return TTN_EINVAL;
    }
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) {
    set_err(err, err_len, std::string("cudaGetDevice: ") + cudaGetErrorString(ce));
    return TTN_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_err(err, err_len, "ttn_rdm_noalloc: device ordinal " + std::to_string(dev) + " is beyond the " +
                              std::to_string(kMaxDevices) + " devices it keeps a scratch address for");
    return TTN_EINVAL;
  }
  double2* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
      void* ptr = nullptr;
      ce = cudaGetSymbolAddress(&ptr, g_rdm_scratch);
      if (ce != cudaSuccess || !ptr) {
        set_err(err, err_len, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(ce));
        return TTN_ECUDA;
      }
      g_scratch_ptr[dev] = (double2*)ptr;
    }
    scratch = g_scratch_ptr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  // Every scratch entry this call reads is written earlier in the same call
  // (children before parents, postorder), so nothing needs clearing.
  for (int u : p.tree.postorder) {
    const auto& d = p.dims[u];
    const double2* w[3] = {nullptr, nullptr, nullptr};
    for (int li = (u == 0 ? 2 : 1); li < 3; ++li) {
      const Leg& L = p.tree.legs[u][li];
      if (L.kind == 'n') w[li] = scratch + off[L.v];
    }
    launch_rdm_node((const double2*)node_dev[u], d[0], d[1], d[2], u == 0, w[1], w[2],
                    u == 0 ? (double2*)rho_dev : scratch + off[u], s);
  }
  ce = cudaGetLastError();
  if (ce != cudaSuccess) {
    set_err(err, err_len, std::string("launch: ") + cudaGetErrorString(ce));
    return TTN_ECUDA;
  }
  return TTN_OK;
}
