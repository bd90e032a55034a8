// read_vm_static: a variant of read_vm (host output) that allocates nothing.
//
// read_vm copies V to a host buffer through a device staging buffer that the
// context allocates with cudaMalloc on its first host read.  This variant
// stages through a fixed array in the library's own device image instead, so
// a caller whose device memory is fully reserved by another allocator, or who
// cannot accept the device-wide synchronisation that cudaMalloc/cudaFree may
// imply, can still read results.
//
// The staging array is a file-scope __device__ array of kStageFloats floats
// (8 MiB): every GPU that loads this library holds it until the process
// exits.  In host code its name is only a host-side stand-in, so the device
// address is obtained once per device with cudaGetSymbolAddress and passed to
// the kernel.  All calls share the array and it keeps the last call's
// contents; nothing in it needs to start at zero because each call overwrites
// every element it copies out.  Calls that overlap on the GPU (for example two
// contexts reading on different streams at the same time) race on the array.
//
// With CUDA's lazy module loading (the default), the device memory of this
// file's module, the 8 MiB array included, is reserved when the module is
// first used.  fibers_create therefore looks the address up on its device
// (prepare_static_stage), so the reservation happens there, where allocating
// is expected, and not inside the first read_vm_static call.  If that
// look-up failed at creation, the first read_vm_static call on the device
// tries again, and then it may reserve the array itself.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "fibers.h"
#include "fibers_internal.h"

namespace {

constexpr size_t kStageFloats = size_t(1) << 21;  // 2,097,152 nodes = 8 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_vm_stage[kStageFloats];

std::mutex g_setup_mu;
float* g_stage_addr[kMaxDevices] = {};

// Same gather as read_vm: V = u + Vrest of every real node, ragged order.
__global__ void gather_stage_kernel(const fib::FiberDesc* fibers, int32_t n_fibers, const float* u, float* stage,
                                    float add) {
  for (int32_t f = blockIdx.x; f < n_fibers; f += gridDim.x) {
    const fib::FiberDesc fd = fibers[f];
    for (int i = threadIdx.x; i < fd.n; i += blockDim.x) stage[fd.coff + i] = u[fd.slot + i] + add;
  }
}

// Device address of the staging array on `device` (which must be current).
cudaError_t stage_address(int device, float** out) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_stage_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_vm_stage);
    if (e != cudaSuccess) return e;
    g_stage_addr[device] = static_cast<float*>(p);
  }
  *out = g_stage_addr[device];
  return cudaSuccess;
}

// Restores the calling thread's current device when the call returns.
struct DeviceGuard {
  int saved = -1;
  DeviceGuard() {
    if (cudaGetDevice(&saved) != cudaSuccess) saved = -1;
  }
  ~DeviceGuard() {
    if (saved >= 0) cudaSetDevice(saved);
  }
};

}  // namespace

int fib::prepare_static_stage(int device) {
  if (device < 0 || device >= kMaxDevices) return (int)cudaErrorInvalidDevice;
  float* p = nullptr;
  return (int)stage_address(device, &p);
}

extern "C" fib_status read_vm_static(fib_ctx* ctx, float* host_out, size_t capacity) {
  fib::CtxView v;
  fib_status st = fib::ctx_view(ctx, &v);
  if (st != FIB_OK) return st;
  if (v.total > (int64_t)kStageFloats)
    return fib::ctx_fail(ctx, FIB_EINVAL,
                         "read_vm_static stages at most 2097152 nodes (8 MiB per GPU); this context has more, "
                         "use read_vm");
  if (capacity < (size_t)v.total) return fib::ctx_fail(ctx, FIB_EINVAL, "capacity is smaller than the node count");
  if (v.total > 0 && !host_out) return fib::ctx_fail(ctx, FIB_EINVAL, "host_out is NULL");
  if (v.device < 0 || v.device >= kMaxDevices) return fib::ctx_fail(ctx, FIB_ENOTSUP, "device index out of range");
  const DeviceGuard keep_device;
  cudaError_t e = cudaSetDevice(v.device);
  if (e != cudaSuccess) return fib::ctx_fail(ctx, FIB_ECUDA, cudaGetErrorString(e));
  float* stage = nullptr;
  e = stage_address(v.device, &stage);
  if (e != cudaSuccess) return fib::ctx_fail(ctx, FIB_ECUDA, cudaGetErrorString(e));
  if (v.total > 0) {
    const int grid = v.n_fibers < 65535 ? (v.n_fibers > 0 ? v.n_fibers : 1) : 65535;
    gather_stage_kernel<<<grid, 256, 0, v.stream>>>(v.fibers, v.n_fibers, v.u, stage, v.vrest);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fib::ctx_fail(ctx, FIB_ECUDA, cudaGetErrorString(e));
    ++*v.launches;
    e = cudaMemcpyAsync(host_out, stage, sizeof(float) * (size_t)v.total, cudaMemcpyDeviceToHost, v.stream);
    if (e != cudaSuccess) return fib::ctx_fail(ctx, FIB_ECUDA, cudaGetErrorString(e));
  }
  e = cudaStreamSynchronize(v.stream);
  if (e != cudaSuccess) return fib::ctx_fail(ctx, FIB_ECUDA, cudaGetErrorString(e));
  int32_t flag = 0;
  e = cudaMemcpy(&flag, v.flag, sizeof(flag), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fib::ctx_fail(ctx, FIB_ECUDA, cudaGetErrorString(e));
  if (flag & 1) return fib::ctx_fail(ctx, FIB_ENONFINITE, "state became non-finite (NaN/Inf)");
  return FIB_OK;
}
