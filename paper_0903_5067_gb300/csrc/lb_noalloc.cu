// lb_fluid_sums_noalloc: fluid mass and momentum of a population field, computed without
// allocating device memory.
//
// Some callers cannot allocate device memory at the point where they need these sums: a host
// application whose device memory is all reserved by another allocator (a framework's caching
// allocator, a memory pool sized to the whole GPU), where a cudaMalloc of its own would fail
// or fragment that pool; and time-critical loops, where cudaFree's implicit device-wide
// synchronisation and the allocation's latency are not acceptable.  This entry point serves
// them: its per-block partial sums go to a fixed scratch array declared below at file scope,
// which every GPU that loads the library holds until the process exits.
#include <cuda_runtime.h>
#include <mutex>

#include "../../include/lb.h"
#include "lb_engine.h"

namespace {

constexpr int kThreads = 256;
// one partial (sum n, sum Jx, sum Jy, sum Jz) per block of 256 nodes: 65536 blocks cover
// boxes up to 256^3 nodes; 2 MiB of device memory
constexpr int kMaxBlocks = 65536;
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_noalloc_partials[kMaxBlocks * 4];
__device__ __align__(256) double g_noalloc_result[4];

// D3Q19 velocity components in the library's ABI order
__constant__ int c_ex[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
__constant__ int c_ey[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
__constant__ int c_ez[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

__global__ void __launch_bounds__(kThreads) k_partials(const double* __restrict__ pop, long long nnodes,
                                                       double* __restrict__ part) {
  const long long t = blockIdx.x * (long long)kThreads + threadIdx.x;
  double v[4] = {0, 0, 0, 0};
  if (t < nnodes) {
    for (int i = 0; i < 19; ++i) {
      const double n = pop[(long long)i * nnodes + t];
      v[0] += n;
      v[1] += c_ex[i] * n;
      v[2] += c_ey[i] * n;
      v[3] += c_ez[i] * n;
    }
  }
  __shared__ double sh[4][kThreads / 32];
  for (int q = 0; q < 4; ++q) {
    double a = v[q];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) sh[q][threadIdx.x >> 5] = a;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double a = 0;
    for (int w = 0; w < kThreads / 32; ++w) a += sh[threadIdx.x][w];
    part[4ll * blockIdx.x + threadIdx.x] = a;  // every slot in use is overwritten each call
  }
}

// fixed-order reduction of the partials; writes mass and momentum in physical units
__global__ void __launch_bounds__(kThreads) k_finish(const double* __restrict__ part, int nblocks, double a3,
                                                     double mom_scale, double* __restrict__ out) {
  double v[4] = {0, 0, 0, 0};
  for (int b = threadIdx.x; b < nblocks; b += kThreads)
    for (int q = 0; q < 4; ++q) v[q] += part[4ll * b + q];
  __shared__ double sh[4][kThreads / 32];
  for (int q = 0; q < 4; ++q) {
    double a = v[q];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) sh[q][threadIdx.x >> 5] = a;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double a = 0;
    for (int w = 0; w < kThreads / 32; ++w) a += sh[threadIdx.x][w];
    out[threadIdx.x] = threadIdx.x == 0 ? a * a3 : a * mom_scale;
  }
}

std::mutex g_setup_mutex;
bool g_ready[kMaxDevices] = {};
double* g_partials_addr[kMaxDevices] = {};
double* g_result_addr[kMaxDevices] = {};

// Device addresses of the file-scope arrays.  In host code the arrays' names are host-side
// stand-ins, not device addresses, so each device's addresses are looked up once, with that
// device current, and cached.
int device_addresses(int dev, double** partials, double** result) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_ready[dev]) {
    void* p = nullptr;
    void* r = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess) return LB_ERR_CUDA;
    if (cudaGetSymbolAddress(&r, g_noalloc_result) != cudaSuccess) return LB_ERR_CUDA;
    g_partials_addr[dev] = static_cast<double*>(p);
    g_result_addr[dev] = static_cast<double*>(r);
    g_ready[dev] = true;
  }
  *partials = g_partials_addr[dev];
  *result = g_result_addr[dev];
  return LB_OK;
}

}  // namespace

extern "C" int lb_fluid_sums_noalloc(const double* pop_dev, int L, double a, double h, double* out_host,
                                     void* stream) {
  using gblb::api_fail;
  if (!pop_dev || !out_host) return api_fail(LB_ERR_ARG, "lb_fluid_sums_noalloc: null population or output pointer");
  if (!(a > 0) || !(h > 0)) return api_fail(LB_ERR_ARG, "lb_fluid_sums_noalloc: a and h must be > 0");
  if (L < 1 || L > LB_NOALLOC_MAX_L)
    return api_fail(LB_ERR_ARG, "lb_fluid_sums_noalloc: L outside [1, LB_NOALLOC_MAX_L] (the fixed scratch holds "
                                "the partial sums of at most 256^3 nodes)");
  const long long nnodes = (long long)L * L * L;
  int nblocks = (int)((nnodes + kThreads - 1) / kThreads);
  if (nblocks > kMaxBlocks) return api_fail(LB_ERR_ARG, "lb_fluid_sums_noalloc: box beyond the scratch capacity");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return api_fail(LB_ERR_CUDA, "lb_fluid_sums_noalloc: no usable current device");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (s) {  // the scratch address below belongs to the current device: the stream must too
    int sdev = -1;
    if (cudaStreamGetDevice(s, &sdev) != cudaSuccess)
      return api_fail(LB_ERR_ARG, "lb_fluid_sums_noalloc: the stream is not a valid CUDA stream");
    if (sdev != dev)
      return api_fail(LB_ERR_ARG, "lb_fluid_sums_noalloc: the stream belongs to another device than the current one");
  }
  double* partials = nullptr;
  double* result = nullptr;
  if (device_addresses(dev, &partials, &result) != LB_OK)
    return api_fail(LB_ERR_CUDA, "lb_fluid_sums_noalloc: cudaGetSymbolAddress of the scratch array failed");
  // launches checked by their own return codes: an error left pending by the caller's
  // earlier work is neither taken nor reported here
  {
    void* args[] = {(void*)&pop_dev, (void*)&nnodes, (void*)&partials};
    if (cudaLaunchKernel((const void*)k_partials, dim3((unsigned)nblocks), dim3(kThreads), args, 0, s) != cudaSuccess)
      return api_fail(LB_ERR_CUDA, "lb_fluid_sums_noalloc: partial-sum kernel launch failed");
  }
  {
    const double a3 = a * a * a, ms = a * a * a * a / h;
    void* args[] = {(void*)&partials, (void*)&nblocks, (void*)&a3, (void*)&ms, (void*)&result};
    if (cudaLaunchKernel((const void*)k_finish, dim3(1), dim3(kThreads), args, 0, s) != cudaSuccess)
      return api_fail(LB_ERR_CUDA, "lb_fluid_sums_noalloc: final-sum kernel launch failed");
  }
  if (cudaMemcpyAsync(out_host, result, 4 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return api_fail(LB_ERR_CUDA, "lb_fluid_sums_noalloc: copy of the sums to the host failed");
  const cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return api_fail(LB_ERR_CUDA, cudaGetErrorString(e));
  return LB_OK;
}
