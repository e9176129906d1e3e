// hmat_noalloc.cu -- truncation entry point that allocates no memory.
//
// Some callers cannot let a library allocate device memory: real-time or
// embedded hosts that reserve all device memory up front (an allocation in
// the middle of a run could fail or stall), and applications whose own memory
// pool owns the whole GPU (memory taken behind the pool's back breaks its
// accounting).  trunc_lowrank_noalloc serves them: it does the same
// truncation as trunc_lowrank, but its scratch memory is a fixed array
// compiled into the library instead of a cudaMalloc'ed buffer.  The call
// reads the new rank back and synchronises the context stream before it
// returns.
//
// The array is a file-scope __device__ variable of HM_NOALLOC_DOUBLES doubles
// (16 MiB).  Every GPU that loads the library holds it until the process
// exits, whether or not the entry point is used.  Host code cannot use the
// array's name as a device address, so the first call on each device asks the
// runtime for the address (cudaGetSymbolAddress, with that device current)
// and caches it; that first call should come before any stream capture
// begins on that device.
// All calls share the one array: calls that overlap on the GPU (two streams,
// or two host threads) race on it and must be serialised by the caller.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "hmat.h"
#include "hmat_device.cuh"

namespace hm_internal {
int ctx_device(const hmat_ctx* c);
cudaStream_t ctx_stream(const hmat_ctx* c);
void set_last_error(const char* msg);
}  // namespace hm_internal

namespace {

// 2 Mi doubles = 16 MiB; the first 32 doubles hold the status word and the
// new rank, the scratch of the truncation starts at double 32 (256 bytes).
const int64_t HM_NOALLOC_DOUBLES = (int64_t)1 << 21;
const int64_t HM_NOALLOC_HEADER = 32;
const int HM_NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) double g_noalloc_scratch[HM_NOALLOC_DOUBLES];

double* g_noalloc_ptr[HM_NOALLOC_MAX_DEVICES] = {nullptr};
std::mutex g_noalloc_mutex;

// One CTA truncates U V^T in place; the problem comes by value, the scratch
// and the result words live in the static array.
__global__ void __launch_bounds__(HM_THREADS) trunc_noalloc_kernel(int m, int n, int l, double* U, int ldu,
                                                                  double* V, int ldv, double eps,
                                                                  double* scratch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  hm::Smem& s = *reinterpret_cast<hm::Smem*>(smem_raw);
  int* status = reinterpret_cast<int*>(scratch);
  int64_t* k_new = reinterpret_cast<int64_t*>(scratch + 1);
  double* SA = scratch + HM_NOALLOC_HEADER;
  double* SB = SA + (int64_t)m * l;
  double* W = SB + (int64_t)n * l;
  double* Jg = W + (int64_t)m * l;
  for (int idx = threadIdx.x; idx < m * l; idx += HM_THREADS) SA[idx] = U[(int64_t)(idx / m) * ldu + idx % m];
  for (int idx = threadIdx.x; idx < n * l; idx += HM_THREADS) SB[idx] = V[(int64_t)(idx / n) * ldv + idx % n];
  __syncthreads();
  hm::TruncIn in;
  in.nb = 1;
  in.m = m;
  in.n[0] = n;
  in.k[0] = l;
  in.SA[0] = SA;
  in.SB[0] = SB;
  in.W = W;
  in.Jg = Jg;
  int cap = l < m ? l : m;
  if (n < cap) cap = n;
  int k = hm::trunc_core(in, eps, cap, U, ldu, V, ldv, status, s);
  if (threadIdx.x == 0) *k_new = k;
}

// Address of the static array on the current device (set up once per device).
cudaError_t noalloc_scratch(int device, double** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (device < 0 || device >= HM_NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(trunc_noalloc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(hm::Smem));
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[device] = (double*)p;
  }
  *out = g_noalloc_ptr[device];
  return cudaSuccess;
}

hmat_status fail(hmat_status code, const std::string& msg) {
  hm_internal::set_last_error(msg.c_str());
  return code;
}

}  // namespace

extern "C" hmat_status trunc_lowrank_noalloc(hmat_ctx* ctx, int64_t m, int64_t n, int64_t k, double* U, int64_t ldu,
                                             double* V, int64_t ldv, double eps, int64_t* k_new) {
  if (!ctx || !U || !V || !k_new || m < 0 || n < 0 || k < 0 || ldu < std::max<int64_t>(m, 1) ||
      ldv < std::max<int64_t>(n, 1) || !(eps >= 0.0))
    return fail(HMAT_ERR_ARG, "trunc_lowrank_noalloc: bad arguments");
  // the kernel indexes with 32-bit sizes and leading dimensions
  if (ldu > INT32_MAX || ldv > INT32_MAX)
    return fail(HMAT_ERR_ARG, "trunc_lowrank_noalloc: ldu and ldv must be at most 2^31 - 1");
  if (k > HM_LMAX) return fail(HMAT_ERR_ARG, "trunc_lowrank_noalloc: k must be <= 256");
  int64_t need = HM_NOALLOC_HEADER + (2 * m + n) * k + 2 * k * k;
  if (need > HM_NOALLOC_DOUBLES)
    return fail(HMAT_ERR_ARG, "trunc_lowrank_noalloc: (2m + n) k + 2 k^2 = " + std::to_string(need - HM_NOALLOC_HEADER) +
                                  " doubles exceeds the fixed scratch of " +
                                  std::to_string(HM_NOALLOC_DOUBLES - HM_NOALLOC_HEADER) + " doubles");
  int device = hm_internal::ctx_device(ctx);
  cudaStream_t st = hm_internal::ctx_stream(ctx);
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return fail(HMAT_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  double* scratch = nullptr;
  e = noalloc_scratch(device, &scratch);
  if (e != cudaSuccess) return fail(HMAT_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  if (k == 0 || m == 0 || n == 0) {
    *k_new = 0;
    return HMAT_OK;
  }
  // the status word must start at zero; the rest is written before it is read
  e = cudaMemsetAsync(scratch, 0, HM_NOALLOC_HEADER * sizeof(double), st);
  if (e != cudaSuccess) return fail(HMAT_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  trunc_noalloc_kernel<<<1, HM_THREADS, sizeof(hm::Smem), st>>>((int)m, (int)n, (int)k, U, (int)ldu, V, (int)ldv, eps,
                                                                scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(HMAT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  int64_t header[2] = {0, 0};
  e = cudaMemcpyAsync(header, scratch, sizeof(header), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(HMAT_ERR_CUDA, std::string("result copy: ") + cudaGetErrorString(e));
  int status = (int)(header[0] & 0xffffffff);
  if (status != 0) return fail((hmat_status)status, "trunc_lowrank_noalloc: device status");
  *k_new = header[1];
  return HMAT_OK;
}
