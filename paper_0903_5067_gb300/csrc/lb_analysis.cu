// Chain observables of Sec. III A/B computed on the GPU from a device trajectory of unwrapped
// bead positions traj[t][n][3] (FP64): g1, g2, g3 (monomer, monomer-in-CM and centre-of-mass
// mean-square displacements), Rouse modes X_p and their time correlation, static and dynamic
// structure factors S(k), S(k, t) (isotropic: exp(i k.r) averaged over the directions of k is
// sin(kr)/(kr)).
//
// Every output element is one thread block's fixed-order sum: threads stride over the
// summation domain in a fixed pattern and combine in a fixed shared-memory tree, so results
// are reproducible bit for bit.  No kernel allocates memory; outputs are caller-owned device
// arrays.  All arithmetic is FP64.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/lb.h"

namespace {

constexpr int kThreads = 256;

// fixed-order block reduction of NV values per thread (result valid in thread 0)
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double (*sh)[kThreads]) {
  const int t = threadIdx.x;
#pragma unroll
  for (int q = 0; q < NV; ++q) sh[q][t] = v[q];
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (t < s) {
#pragma unroll
      for (int q = 0; q < NV; ++q) sh[q][t] += sh[q][t + s];
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = sh[q][0];
}

__device__ __forceinline__ void centre(const double* __restrict__ f, int N, double c[3]) {
  double s0 = 0, s1 = 0, s2 = 0;
  for (int n = 0; n < N; ++n) {
    s0 += f[3 * n];
    s1 += f[3 * n + 1];
    s2 += f[3 * n + 2];
  }
  c[0] = s0 / N;
  c[1] = s1 / N;
  c[2] = s2 / N;
}

// one block per lag: origins t0 strided over the threads
__global__ void __launch_bounds__(kThreads) k_msd(const double* __restrict__ traj, int T, int N, int i0, int i1,
                                                  double* __restrict__ out, int nlag) {
  __shared__ double sh[3][kThreads];
  const int lag = blockIdx.x;
  const int norig = T - lag;
  double v[3] = {0, 0, 0};
  for (int t0 = threadIdx.x; t0 < norig; t0 += kThreads) {
    const double* fa = traj + (size_t)t0 * N * 3;
    const double* fb = traj + (size_t)(t0 + lag) * N * 3;
    double ca[3], cb[3];
    centre(fa, N, ca);
    centre(fb, N, cb);
    double dcm[3], s3 = 0;
    for (int q = 0; q < 3; ++q) {
      dcm[q] = cb[q] - ca[q];
      s3 += dcm[q] * dcm[q];
    }
    v[2] += s3;
    for (int w = 0; w < 2; ++w) {
      const int i = w ? i1 : i0;
      double s1 = 0, s2 = 0;
      for (int q = 0; q < 3; ++q) {
        const double d = fb[3 * i + q] - fa[3 * i + q];
        s1 += d * d;
        const double dr = d - dcm[q];
        s2 += dr * dr;
      }
      v[0] += s1;
      v[1] += s2;
    }
  }
  block_sum<3>(v, sh);
  if (threadIdx.x == 0) {
    const bool any = norig > 0;
    out[lag] = any ? v[0] / (2.0 * norig) : 0.0;
    out[nlag + lag] = any ? v[1] / (2.0 * norig) : 0.0;
    out[2 * nlag + lag] = any ? v[2] / norig : 0.0;
  }
}

// one block per frame; threads over (p, component); the sum over n in bead order
__global__ void __launch_bounds__(kThreads) k_rouse_modes(const double* __restrict__ traj, int N, int P,
                                                          double* __restrict__ X) {
  const int t = blockIdx.x;
  const double* f = traj + (size_t)t * N * 3;
  for (int e = threadIdx.x; e < 3 * P; e += kThreads) {
    const int p = 1 + e / 3, q = e % 3;
    double s = 0;
    for (int n = 1; n <= N; ++n) s += f[3 * (n - 1) + q] * cospi((double)p * ((double)n - 0.5) / (double)N);
    X[(size_t)t * P * 3 + e] = s / N;
  }
}

// one block per (p, lag)
__global__ void __launch_bounds__(kThreads) k_rouse_corr(const double* __restrict__ X, int T, int P,
                                                         double* __restrict__ c, int nlag) {
  __shared__ double sh[1][kThreads];
  const int p = blockIdx.x, lag = blockIdx.y;
  const int norig = T - lag;
  double v[1] = {0};
  for (int t0 = threadIdx.x; t0 < norig; t0 += kThreads) {
    const double* a = X + ((size_t)t0 * P + p) * 3;
    const double* b = X + ((size_t)(t0 + lag) * P + p) * 3;
    v[0] += b[0] * a[0] + b[1] * a[1] + b[2] * a[2];
  }
  block_sum<1>(v, sh);
  if (threadIdx.x == 0) c[(size_t)p * nlag + lag] = norig > 0 ? v[0] / norig : 0.0;
}

__device__ __forceinline__ double sinc_kr(double k, double r2) {
  const double x = k * sqrt(r2);
  return x == 0.0 ? 1.0 : sin(x) / x;
}

// one block per k: pairs i < j of every frame (the sum is symmetric; the N diagonal terms
// are 1 each); the threads walk all ordered pairs and skip i >= j
__global__ void __launch_bounds__(kThreads) k_static_sk(const double* __restrict__ traj, int T, int N,
                                                        const double* __restrict__ ks, double* __restrict__ S) {
  __shared__ double sh[1][kThreads];
  const double k = ks[blockIdx.x];
  const long long nn = (long long)N * N;
  const long long total = nn * T;
  double v[1] = {0};
  for (long long u = threadIdx.x; u < total; u += kThreads) {
    const int t = (int)(u / nn);
    const int r = (int)(u - (long long)t * nn);
    const int i = r / N, j = r - (r / N) * N;
    if (i >= j) continue;
    const double* f = traj + (size_t)t * N * 3;
    const double dx = f[3 * i] - f[3 * j], dy = f[3 * i + 1] - f[3 * j + 1], dz = f[3 * i + 2] - f[3 * j + 2];
    v[0] += sinc_kr(k, dx * dx + dy * dy + dz * dz);
  }
  block_sum<1>(v, sh);
  if (threadIdx.x == 0) S[blockIdx.x] = ((double)N * T + 2.0 * v[0]) / ((double)N * T);
}

// one block per (k, lag): all ordered pairs (i, j) at the origins t0 = 0, s, 2s, ...
__global__ void __launch_bounds__(kThreads) k_dynamic_sk(const double* __restrict__ traj, int T, int N,
                                                         const double* __restrict__ ks, int stride,
                                                         double* __restrict__ S, int nlag) {
  __shared__ double sh[1][kThreads];
  const double k = ks[blockIdx.x];
  const int lag = blockIdx.y;
  const int norig = T - lag > 0 ? (T - lag + stride - 1) / stride : 0;
  const long long nn = (long long)N * N;
  const long long total = nn * norig;
  double v[1] = {0};
  for (long long u = threadIdx.x; u < total; u += kThreads) {
    const int o = (int)(u / nn);
    const int r = (int)(u - (long long)o * nn);
    const int i = r / N, j = r - (r / N) * N;
    const int t0 = o * stride;
    const double* fa = traj + (size_t)t0 * N * 3;
    const double* fb = traj + (size_t)(t0 + lag) * N * 3;
    const double dx = fb[3 * i] - fa[3 * j], dy = fb[3 * i + 1] - fa[3 * j + 1], dz = fb[3 * i + 2] - fa[3 * j + 2];
    v[0] += sinc_kr(k, dx * dx + dy * dy + dz * dz);
  }
  block_sum<1>(v, sh);
  if (threadIdx.x == 0) S[(size_t)blockIdx.x * nlag + lag] = norig > 0 ? v[0] / ((double)N * norig) : 0.0;
}

// one block: 1/r_ij over the pairs i < j of every frame
__global__ void __launch_bounds__(kThreads) k_inverse_radius(const double* __restrict__ traj, int T, int N,
                                                             double* __restrict__ out) {
  __shared__ double sh[1][kThreads];
  const long long nn = (long long)N * N;
  const long long total = nn * T;
  double v[1] = {0};
  for (long long u = threadIdx.x; u < total; u += kThreads) {
    const int t = (int)(u / nn);
    const int r = (int)(u - (long long)t * nn);
    const int i = r / N, j = r - (r / N) * N;
    if (i >= j) continue;
    const double* f = traj + (size_t)t * N * 3;
    const double dx = f[3 * i] - f[3 * j], dy = f[3 * i + 1] - f[3 * j + 1], dz = f[3 * i + 2] - f[3 * j + 2];
    v[0] += 1.0 / sqrt(dx * dx + dy * dy + dz * dz);
  }
  block_sum<1>(v, sh);
  if (threadIdx.x == 0) out[0] = 2.0 * v[0] / ((double)N * N * T);
}

int launch_status() {
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return LB_OK;
  return e == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA;
}

}  // namespace

extern "C" {

int lb_analysis_msd(const double* traj, int T, int N, int max_lag, int i0, int i1, double* out, void* stream) {
  if (!traj || !out || T < 1 || N < 1 || max_lag < 0 || i0 < 0 || i1 < 0 || i0 >= N || i1 >= N) return LB_ERR_ARG;
  k_msd<<<max_lag + 1, kThreads, 0, (cudaStream_t)stream>>>(traj, T, N, i0, i1, out, max_lag + 1);
  return launch_status();
}

int lb_analysis_rouse_modes(const double* traj, int T, int N, int P, double* X, void* stream) {
  if (!traj || !X || T < 1 || N < 2 || P < 1 || P > N - 1) return LB_ERR_ARG;
  k_rouse_modes<<<T, kThreads, 0, (cudaStream_t)stream>>>(traj, N, P, X);
  return launch_status();
}

int lb_analysis_rouse_correlation(const double* X, int T, int P, int max_lag, double* c, void* stream) {
  if (!X || !c || T < 1 || P < 1 || max_lag < 0 || max_lag > 65535) return LB_ERR_ARG;
  k_rouse_corr<<<dim3(P, max_lag + 1), kThreads, 0, (cudaStream_t)stream>>>(X, T, P, c, max_lag + 1);
  return launch_status();
}

int lb_analysis_static_sk(const double* traj, int T, int N, const double* k, int nk, double* S, void* stream) {
  if (!traj || !k || !S || T < 1 || N < 1 || nk < 1) return LB_ERR_ARG;
  k_static_sk<<<nk, kThreads, 0, (cudaStream_t)stream>>>(traj, T, N, k, S);
  return launch_status();
}

int lb_analysis_inverse_radius(const double* traj, int T, int N, double* out, void* stream) {
  if (!traj || !out || T < 1 || N < 2) return LB_ERR_ARG;
  k_inverse_radius<<<1, kThreads, 0, (cudaStream_t)stream>>>(traj, T, N, out);
  return launch_status();
}

int lb_analysis_dynamic_sk(const double* traj, int T, int N, const double* k, int nk, int max_lag,
                           int origin_stride, double* S, void* stream) {
  if (!traj || !k || !S || T < 1 || N < 1 || nk < 1 || max_lag < 0 || max_lag > 65535 || origin_stride < 1)
    return LB_ERR_ARG;
  k_dynamic_sk<<<dim3(nk, max_lag + 1), kThreads, 0, (cudaStream_t)stream>>>(traj, T, N, k, origin_stride, S,
                                                                               max_lag + 1);
  return launch_status();
}

}  // extern "C"
