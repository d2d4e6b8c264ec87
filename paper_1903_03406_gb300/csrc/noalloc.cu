// Predicate batch evaluation that allocates no device memory.
//
// cdr_eval_predicates stages its host inputs and outputs in device buffers that
// it takes with cudaMalloc and gives back with cudaFree on every call. Two kinds
// of caller cannot work that way:
//  * a caller that keeps kernels running on other streams while it checks
//    geometry: cudaFree waits for the whole device, so every call would stall
//    that work until it drains;
//  * a process whose device memory is held by a caching allocator (PyTorch's,
//    for one): the memory sits reserved in the cache, so a plain cudaMalloc can
//    fail although the process has memory to spare.
// cdr_eval_predicates_noalloc stages the same data in one array that lives in
// this file's device image (g_eval_scratch below). The array exists on every GPU
// that loads the library, from module load until the process exits. Its size
// limits one call to CDR_EVAL_NOALLOC_MAX_ITEMS items.
//
// Host code never uses the name g_eval_scratch as a pointer. On the host that
// name stands for a host-side shadow, not device memory: a kernel handed it
// would fault, or silently touch the wrong memory where the GPU can reach host
// memory. The device address comes from cudaGetSymbolAddress, looked up once per
// device with that device current, on the first call made there.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/cdr.h"

// This file takes its own copy of the device geometry, with internal linkage,
// so that its out-of-line exact predicates do not clash with the kernels'.
namespace {
#include "predicates.cuh"
}  // namespace

namespace {
using namespace cdr;

constexpr int kMaxItems = CDR_EVAL_NOALLOC_MAX_ITEMS;
// Layout of the scratch array: every part starts on a 256-byte boundary.
constexpr size_t kOffItems = 0;                                      // n * 16 doubles
constexpr size_t kOffPoints = kOffItems + (size_t)kMaxItems * 128;   // n * 3 doubles
constexpr size_t kOffSigns = kOffPoints + (size_t)kMaxItems * 24;    // n ints
constexpr size_t kScratchBytes = kOffSigns + (size_t)kMaxItems * 4;  // 2.44 MiB
static_assert(kOffPoints % 256 == 0 && kOffSigns % 256 == 0, "scratch parts must stay aligned");

static __device__ __align__(256) unsigned char g_eval_scratch[kScratchBytes];

// The batch kernel of cdr_eval_predicates, reading its items from and writing
// its results to the scratch array. Every slot i < n is written, so what an
// earlier call left in the array is never read.
__global__ void k_eval_pred_noalloc(int kind, const double* in, int n, int* sign, double* outp) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double* q = in + 16 * (size_t)i;
    D3 a{q[0], q[1], q[2]}, b{q[3], q[4], q[5]}, c{q[6], q[7], q[8]}, d{q[9], q[10], q[11]},
        e{q[12], q[13], q[14]};
    int sg = 0;
    D3 o{0, 0, 0};
    switch (kind) {
      case 0: sg = orient3d(a, b, c, d); break;
      case 1: sg = insphere(a, b, c, d, e); break;
      case 2: sg = diametral(a, b, c); break;
      case 3: sg = equatorial(a, b, c, d); break;
      case 4: {
        D3 off;
        sg = tet_circumcenter_fixed(a, b, c, d, o, off) ? 1 : 0;
        break;
      }
      case 5: sg = tri_circumcenter_fixed(a, b, c, o) ? 1 : 0; break;
      case 6: o = midpoint_fixed(a, b); sg = 1; break;
      case 7: sg = tet_bad_fixed(a, b, c, d, q[12]) ? 1 : 0; break;
      case 8: sg = orient3d_exact(a, b, c, d); break;
      case 9: sg = insphere_exact(a, b, c, d, e); break;
      case 10: sg = equatorial_exact(a, b, c, d); break;
      case 11: sg = diametral_exact(a, b, c); break;
    }
    sign[i] = sg;
    outp[3 * (size_t)i] = o.x;
    outp[3 * (size_t)i + 1] = o.y;
    outp[3 * (size_t)i + 2] = o.z;
  }
}

// Device addresses of this file's scratch array and of its copy of the
// exact-arithmetic overflow flag, per device (null until first use there).
constexpr int kMaxDevices = 64;
struct DevScratch {
  unsigned char* base = nullptr;
  int* overflow = nullptr;
};
std::mutex g_setup_mutex;
DevScratch g_dev[kMaxDevices];

int scratch_for_current_device(DevScratch* out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return CDR_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return CDR_ERR_INVALID_INPUT;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DevScratch& d = g_dev[dev];
  if (!d.base) {
    unsigned char* base = nullptr;
    int* flag = nullptr;
    if (cudaGetSymbolAddress((void**)&base, g_eval_scratch) != cudaSuccess ||
        cudaGetSymbolAddress((void**)&flag, g_exact_overflow) != cudaSuccess || !base || !flag) {
      cudaGetLastError();
      return CDR_ERR_CUDA;
    }
    d.overflow = flag;
    d.base = base;
  }
  *out = d;
  return CDR_OK;
}

}  // namespace

extern "C" int cdr_eval_predicates_noalloc(int32_t kind, const double* in, int32_t n,
                                           int32_t* sign, double* out, void* stream) {
  if (kind < 0 || kind > 11 || n < 0 || !in || !sign) return CDR_ERR_INVALID_INPUT;
  if (n > kMaxItems) return CDR_ERR_TOO_LARGE;
  if (n == 0) return CDR_OK;
  DevScratch d;
  int st = scratch_for_current_device(&d);
  if (st != CDR_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  double* din = (double*)(d.base + kOffItems);
  double* dout = (double*)(d.base + kOffPoints);
  int* dsg = (int*)(d.base + kOffSigns);
  // the overflow flag is the one part that must start at zero: the exact
  // routines only ever set it
  cudaMemsetAsync(d.overflow, 0, sizeof(int), s);
  cudaMemcpyAsync(din, in, (size_t)n * 128, cudaMemcpyHostToDevice, s);
  k_eval_pred_noalloc<<<(n + 127) / 128, 128, 0, s>>>(kind, din, n, dsg, dout);
  cudaMemcpyAsync(sign, dsg, (size_t)n * 4, cudaMemcpyDeviceToHost, s);
  if (out) cudaMemcpyAsync(out, dout, (size_t)n * 24, cudaMemcpyDeviceToHost, s);
  int ov = 0;
  cudaMemcpyAsync(&ov, d.overflow, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return CDR_ERR_CUDA;
  return ov ? CDR_ERR_INTERNAL : CDR_OK;
}
