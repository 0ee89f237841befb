// sp_jvp_static: the tangent step for one direction without any allocation.
//
// sp_jvp keeps its intermediate fields (the six curl/velocity fields on the
// Gauss-Lobatto planes and the three product fields) in workspaces that
// sp_create allocates with cudaMalloc. This variant keeps them instead in one
// file-scope __device__ array of fixed size, so the call itself never
// allocates. It is meant for callers that cannot allocate device memory at
// the time they need a Jacobian action: a process whose GPU memory is already
// committed to its own pool allocator (a further cudaMalloc may fail or
// fragment that reservation), or code on a latency-critical path where
// cudaMalloc/cudaFree would stall other streams with an implicit device
// synchronisation.
#include <mutex>

#include "sp_internal.h"

namespace {

// 8 MiB: enough for 48 x 65 x 48 in FP64 (4.6 MB) and for every grid up to
// 64 x 65 x 64 in mixed precision. Every GPU that loads the library holds it
// until the process exits.
constexpr size_t kStaticScratchBytes = (size_t)8 << 20;
__device__ __align__(256) unsigned char g_jvp_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of the static array on the current device. The symbol's
// host-side name is only a stand-in; its device address has to be looked up
// once per device, with that device current.
cudaError_t scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_jvp_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" sp_status sp_jvp_static(sp_ctx* c, const double* du, double* Jdu, void* stream) {
  if (!c || !du || !Jdu || du == Jdu) return sp_fail(c, SP_EINVAL, "sp_jvp_static: bad arguments");
  if (!c->has_base) return sp_fail(c, SP_EINVAL, "sp_jvp_static: call sp_set_base first");
  if (c->geom != 0) return sp_fail(c, SP_EINVAL, "sp_jvp_static: plane Couette contexts only");
  const bool f32 = c->cfg.prec == SP_MIXED;
  const size_t esz = f32 ? 8 : 16;  // one complex value of the transforms
  const size_t b6 = ((size_t)6 * c->NY * c->Mm * esz + 255) / 256 * 256;
  const size_t b3 = (size_t)3 * c->NY * c->Mm * esz;
  if (b6 + b3 > kStaticScratchBytes)
    return sp_fail(c, SP_EINVAL, "sp_jvp_static: the grid needs " + std::to_string(b6 + b3) +
                                     " bytes of scratch; the static buffer holds " +
                                     std::to_string(kStaticScratchBytes));
  int dev = 0;
  sp_status s = sp_cuda(c, cudaGetDevice(&dev), "sp_jvp_static: device");
  if (s != SP_OK) return s;
  if (dev != c->dev)
    return sp_fail(c, SP_EINVAL, "sp_jvp_static: the context's device must be the current device");
  void* base = nullptr;
  if ((s = sp_cuda(c, scratch_address(dev, &base), "sp_jvp_static: scratch address")) != SP_OK) return s;
  unsigned char* p = static_cast<unsigned char*>(base);
  void* ws6 = p;
  void* ws3 = p + b6;
  cudaStream_t st = (cudaStream_t)stream;
  // every entry of both intermediates is written before it is read, so the
  // contents left by an earlier call need no clearing
  if ((s = sp_cuda(c, launch_yinv(c, f32, du, ws6, 1, st), "yinv")) != SP_OK) return s;
  if ((s = sp_cuda(c, launch_xz(c, f32, XZ_TANGENT, ws6, ws3, 1, st), "xz tangent")) != SP_OK) return s;
  // the second part runs to the end of the array: the chains' scratch may use all of it
  return sp_tangent_solve(c, f32, ws3, kStaticScratchBytes - b6, du, Jdu, ws6, 1, st);
}
