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
// memory. The device address comes from cudaGetSymbolAddress, looked up on every
// call with the call's device current. Nothing is cached, so a call made after
// the caller reset the device (cudaDeviceReset, which reloads this module and
// may move the array) still gets the array's current address.
#include <cuda_runtime.h>

#include <cstdint>

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
// its results to the scratch array; both run each item through eval_item.
// Every slot i < n is written, so what an earlier call left in the array is
// never read.
__global__ void k_eval_pred_noalloc(int kind, const double* in, int n, int* sign, double* outp) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int sg;
    D3 o;
    eval_item(kind, in + 16 * (size_t)i, &sg, &o);
    sign[i] = sg;
    outp[3 * (size_t)i] = o.x;
    outp[3 * (size_t)i + 1] = o.y;
    outp[3 * (size_t)i + 2] = o.z;
  }
}

// Device addresses of this file's scratch array and of its copy of the
// exact-arithmetic overflow flag on the current device, looked up afresh.
struct DevScratch {
  unsigned char* base = nullptr;
  int* overflow = nullptr;
};

int scratch_for_current_device(DevScratch* out) {
  unsigned char* base = nullptr;
  int* flag = nullptr;
  if (cudaGetSymbolAddress((void**)&base, g_eval_scratch) != cudaSuccess ||
      cudaGetSymbolAddress((void**)&flag, g_exact_overflow) != cudaSuccess || !base || !flag) {
    cudaGetLastError();
    return CDR_ERR_CUDA;
  }
  out->base = base;
  out->overflow = flag;
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
