// Brownian dynamics of bead-spring chains with hydrodynamic interaction (Sec. II C): the
// Ito-Euler update r += (D/kT) F dt + sqrt(2 dt) B.W, D/kT = zeta^-1 on the diagonal blocks and
// the regularised Rotne-Prager-Yamakawa mobility off the diagonal, B.W from Fixman's truncated
// Chebyshev expansion of sqrt(D) applied to the noise vector.  The chain model is that of the
// LB runs (FENE bonds, WCA between all pairs, Sec. II A), in an infinite medium.
//
// One thread block per chain (replica) runs many steps per launch with the chain in shared
// memory: positions, forces, the 3N x 3N mobility matrix (symmetric: mat-vecs read it by
// columns, so that consecutive threads read consecutive words) and the Chebyshev vectors.
// Per step: forces, the matrix, the noise, power iterations for the spectral bounds of D, the
// Chebyshev recurrence, the update.  Positions are kept in FP64 in global memory; the
// arithmetic type R is FP32 or FP64.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <memory>
#include <vector>

#include "../../include/lb.h"
#include "d3q19.cuh"
#include "lb_engine.h"
#include "philox.cuh"

namespace gblb {
namespace {

constexpr int kBDThreads = 256;
constexpr int kBDMaxDegree = 64;
constexpr uint32_t kTagBD = 3;

template <class R>
struct BDK {
  int N;
  R kT, zeta, eta, radius, dt, kfene, R0sq, eps, sig2, rc2;
  int hi, degree, piters;
  uint32_t k0;
  double* x;  // [replica][3N], unwrapped positions
  unsigned* status;
};

template <class R>
__device__ __forceinline__ R rcp(R v) {
  return R(1) / v;
}

// block-wide sum of one value per thread (fixed order); every thread gets the result
template <class R>
__device__ R block_sum(R v, R* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  R s = R(0);
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  __syncthreads();
  return s;
}

// out = a * (M v) + b * v + c * u (M symmetric, n x n, leading dimension n; u may be null),
// and, with y, also y += cy * out.  Two neighbouring threads per output row, each over half
// the columns with two partial sums (M read by columns: consecutive rows are consecutive
// words), combined by a shuffle; the pair's even thread writes.
template <class R>
__device__ __forceinline__ void matvec(const R* __restrict__ M, int n, const R* __restrict__ v, R a, R b, R c,
                                       const R* __restrict__ u, R* __restrict__ out, R* __restrict__ y = nullptr,
                                       R cy = R(0)) {
  const int half = threadIdx.x & 1, h0 = half ? n / 2 : 0, h1 = half ? n : n / 2;
  for (int row = threadIdx.x >> 1; row < n; row += blockDim.x >> 1) {
    R s0 = R(0), s1 = R(0);
    int col = h0;
    for (; col + 1 < h1; col += 2) {
      s0 += M[col * n + row] * v[col];
      s1 += M[(col + 1) * n + row] * v[col + 1];
    }
    if (col < h1) s0 += M[col * n + row] * v[col];
    R sum = s0 + s1;
    sum += __shfl_xor_sync(__activemask(), sum, 1);  // the pair (2k, 2k+1) is active together
    if (!half) {
      R o = a * sum + b * v[row];
      if (u) o += c * u[row];
      out[row] = o;
      if (y) y[row] += cy * o;
    }
  }
}

template <class R>
__global__ void __launch_bounds__(kBDThreads) k_bd_steps(const BDK<R> P, uint32_t step0, int nsteps) {
  extern __shared__ __align__(16) unsigned char bsm[];
  const int N = P.N, n = 3 * N, tid = threadIdx.x, nt = blockDim.x;
  R* M = reinterpret_cast<R*>(bsm);  // n x n
  R* x = M + n * n;                  // positions (arithmetic copy)
  R* F = x + n;                      // forces
  R* W = F + n;                      // noise
  R* y = W + n;                      // B.W
  R* t0 = y + n;                     // Chebyshev / power-iteration vectors
  R* t1 = t0 + n;
  R* t2 = t1 + n;
  R* red = t2 + n;                   // 32 partial sums
  R* coef = red + 32;                // Chebyshev coefficients
  R* scal = coef + kBDMaxDegree + 1; // [0] lam_min, [1] lam_max
  double* gx = P.x + (size_t)blockIdx.x * n;
  const uint32_t k1 = kTagBD | ((uint32_t)blockIdx.x << 8);
  for (int t = tid; t < n; t += nt) x[t] = (R)gx[t];
  __syncthreads();
  for (int it = 0; it < nsteps; ++it) {
    const uint32_t step = step0 + (uint32_t)it;
    // forces: FENE on bonds, WCA on all pairs (fixed summation order per bead)
    for (int i = tid; i < N; i += nt) {
      R f[3] = {R(0), R(0), R(0)};
      for (int j = 0; j < N; ++j) {
        if (j == i) continue;
        const R d0 = x[3 * i] - x[3 * j], d1 = x[3 * i + 1] - x[3 * j + 1], d2 = x[3 * i + 2] - x[3 * j + 2];
        const R r2 = d0 * d0 + d1 * d1 + d2 * d2;
        R coefv = R(0);
        if (r2 < P.rc2) {
          const R s2 = P.sig2 / r2, s6 = s2 * s2 * s2;
          coefv += R(24) * P.eps / r2 * (R(2) * s6 * s6 - s6);
        }
        if (j == i - 1 || j == i + 1) {
          if (r2 >= P.R0sq)
            atomicOr(P.status, 1u);
          else
            coefv -= P.kfene / (R(1) - r2 / P.R0sq);
        }
        f[0] += coefv * d0;
        f[1] += coefv * d1;
        f[2] += coefv * d2;
      }
      F[3 * i] = f[0];
      F[3 * i + 1] = f[1];
      F[3 * i + 2] = f[2];
    }
    // mobility D/kT: zeta^-1 on the diagonal blocks, regularised RPY elsewhere
    const R self = rcp(P.zeta);
    for (int pr = tid; pr < N * N; pr += nt) {  // consecutive threads: consecutive i (store stride 3)
      const int j = pr / N, i = pr - (pr / N) * N;
      R blk[3][3];
      if (i == j || !P.hi) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) blk[a][b] = (i == j && a == b) ? self : R(0);
      } else {
        const R d[3] = {x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1], x[3 * i + 2] - x[3 * j + 2]};
        const R r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        const R r = sqrt(r2);
        R ci, cr;
        if (r >= R(2) * P.radius) {
          const R a2 = P.radius * P.radius / r2;
          const R pre = rcp(R(8) * R(M_PI) * P.eta * r);
          ci = pre * (R(1) + R(2) * a2 / R(3));
          cr = pre * (R(1) - R(2) * a2);
        } else {
          const R q = r / P.radius;
          const R pre = rcp(R(6) * R(M_PI) * P.eta * P.radius);
          ci = pre * (R(1) - R(9) * q / R(32));
          cr = pre * (R(3) * q / R(32));
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) blk[a][b] = (a == b ? ci : R(0)) + cr * d[a] * d[b] / r2;
      }
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) M[(3 * j + b) * n + 3 * i + a] = blk[a][b];
    }
    // noise: 3 standard normals per bead from one Philox call, counter (step, bead, 0, 0)
    for (int i = tid; i < N; i += nt) {
      R g[4];
      gauss4<R>(step, (uint32_t)i, 0u, P.k0, k1, g);
      W[3 * i] = g[0];
      W[3 * i + 1] = g[1];
      W[3 * i + 2] = g[2];
    }
    __syncthreads();
    if (P.hi) {
      // spectral bounds of D = kT M by power iterations (lam_max: on D; lam_min: on lam_max I - D)
      const R inv = rcp(sqrt(R(n)));
      for (int t = tid; t < n; t += nt) t0[t] = inv;
      __syncthreads();
      // the iterate is normalised every fourth iteration and after the last (the direction,
      // and so the Rayleigh quotient below, does not depend on it; four unnormalised
      // iterations change the norm by at most lam_max^4)
      R* pa = t0;  // the iterate
      R* pb = t1;
      for (int k = 0; k < P.piters; ++k) {
        matvec<R>(M, n, pa, P.kT, R(0), R(0), nullptr, pb);
        __syncthreads();
        if ((k & 3) == 3 || k == P.piters - 1) {
          R part = R(0);
          for (int t = tid; t < n; t += nt) part += pb[t] * pb[t];
          const R nrm = rcp(sqrt(block_sum<R>(part, red)));
          for (int t = tid; t < n; t += nt) pb[t] *= nrm;
          __syncthreads();
        }
        R* sw = pa;
        pa = pb;
        pb = sw;
      }
      if (pa != t0) {  // the iterate back into t0
        for (int t = tid; t < n; t += nt) t0[t] = pa[t];
        __syncthreads();
      }
      matvec<R>(M, n, t0, P.kT, R(0), R(0), nullptr, t1);
      __syncthreads();
      R part = R(0);
      for (int t = tid; t < n; t += nt) part += t0[t] * t1[t];
      const R lam_max = R(1.05) * block_sum<R>(part, red);
      for (int t = tid; t < n; t += nt) t0[t] = inv;
      __syncthreads();
      pa = t0;
      pb = t1;
      for (int k = 0; k < P.piters; ++k) {
        matvec<R>(M, n, pa, -P.kT, lam_max, R(0), nullptr, pb);  // (lam_max I - D) v
        __syncthreads();
        if ((k & 3) == 3 || k == P.piters - 1) {
          R pp = R(0);
          for (int t = tid; t < n; t += nt) pp += pb[t] * pb[t];
          const R nrm = rcp(sqrt(block_sum<R>(pp, red)));
          for (int t = tid; t < n; t += nt) pb[t] *= nrm;
          __syncthreads();
        }
        R* sw = pa;
        pa = pb;
        pb = sw;
      }
      if (pa != t0) {
        for (int t = tid; t < n; t += nt) t0[t] = pa[t];
        __syncthreads();
      }
      matvec<R>(M, n, t0, -P.kT, lam_max, R(0), nullptr, t1);
      __syncthreads();
      R pq = R(0);
      for (int t = tid; t < n; t += nt) pq += t0[t] * t1[t];
      const R mu = block_sum<R>(pq, red);
      R lam_min = R(0.5) * (lam_max - mu);
      if (lam_min < lam_max / R(1000)) lam_min = lam_max / R(1000);
      // Chebyshev coefficients of sqrt on [lam_min, lam_max] from the degree+1 nodes
      const int K = P.degree + 1;
      for (int k = tid; k < K; k += nt) {
        R s = R(0);
        for (int j = 0; j < K; ++j) {
          const R th = R(M_PI) * (R(j) + R(0.5)) / R(K);
          const R xj = R(0.5) * (lam_max + lam_min) + R(0.5) * (lam_max - lam_min) * cos(th);
          s += sqrt(xj) * cos(R(k) * th);
        }
        coef[k] = (k == 0 ? R(1) : R(2)) / R(K) * s;
      }
      __syncthreads();
      // recurrence: y = sum_k c_k T_k(Dt) W, Dt = s D - t I
      const R sc = R(2) / (lam_max - lam_min), tc = (lam_max + lam_min) / (lam_max - lam_min);
      matvec<R>(M, n, W, sc * P.kT, -tc, R(0), nullptr, t1);  // T_1 W
      __syncthreads();
      for (int t = tid; t < n; t += nt) y[t] = coef[0] * W[t] + coef[1] * t1[t];
      __syncthreads();  // y and t1 are next touched by other threads (the mat-vecs' rows)
      R* tp = W;   // T_{k-1}
      R* tcur = t1;  // T_k
      R* tn = t2;
      for (int k = 2; k < K; ++k) {
        // 2 Dt T_k - T_{k-1}, added to y times c_k by the thread that forms each row
        matvec<R>(M, n, tcur, R(2) * sc * P.kT, R(-2) * tc, R(-1), tp, tn, y, coef[k]);
        __syncthreads();
        R* sw = tp;
        tp = tcur;
        tcur = tn;
        tn = (sw == W) ? t0 : sw;  // never overwrite W before the recurrence is done
      }
    } else {
      const R amp = sqrt(P.kT / P.zeta);
      for (int t = tid; t < n; t += nt) y[t] = amp * W[t];
      __syncthreads();
    }
    // update: r += M F dt + sqrt(2 dt) B W (drift through the same mobility)
    matvec<R>(M, n, F, P.dt, R(0), R(0), nullptr, t1);
    __syncthreads();
    const R nz = sqrt(R(2) * P.dt);
    for (int t = tid; t < n; t += nt) {
      const double nx = gx[t] + (double)(t1[t] + nz * y[t]);
      gx[t] = nx;
      x[t] = (R)nx;
    }
    __syncthreads();
  }
}

class BDBase {
 public:
  virtual ~BDBase() {}
  virtual void step(int64_t n, uint32_t k0, cudaStream_t s) = 0;
  virtual void get(double* x, cudaStream_t s) = 0;
  virtual unsigned status(cudaStream_t s) = 0;
};

template <class R>
class BDT final : public BDBase {
 public:
  BDT(int reps, const BDK<R>& P, const double* x0) : reps_(reps), P_(P) {
    const size_t n = 3 * (size_t)P.N;
    cuda_check(cudaMalloc(&P_.x, reps * n * sizeof(double)), "BD positions");
    cuda_check(cudaMalloc(&P_.status, sizeof(unsigned)), "BD status");
    cuda_check(cudaMemcpy(P_.x, x0, reps * n * sizeof(double), cudaMemcpyHostToDevice), "upload BD positions");
    cuda_check(cudaMemset(P_.status, 0, sizeof(unsigned)), "BD status");
    smem_ = (n * n + 8 * n + 32 + kBDMaxDegree + 1 + 2) * sizeof(R);
    if (smem_ > 48 * 1024)
      cuda_check(cudaFuncSetAttribute(k_bd_steps<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_),
                 "BD shared memory");
  }
  ~BDT() override {
    cudaFree(P_.x);
    cudaFree(P_.status);
  }
  void step(int64_t n, uint32_t k0, cudaStream_t s) override {
    const int chunk = 4096;  // steps per launch
    for (int64_t done = 0; done < n;) {
      const int m = (int)(n - done < chunk ? n - done : chunk);
      k_bd_steps<R><<<reps_, kBDThreads, smem_, s>>>(P_, k0 + (uint32_t)done, m);
      cuda_check(cudaGetLastError(), "BD kernel");
      done += m;
    }
  }
  void get(double* x, cudaStream_t s) override {
    cuda_check(cudaMemcpyAsync(x, P_.x, reps_ * 3 * (size_t)P_.N * sizeof(double), cudaMemcpyDeviceToHost, s),
               "download BD positions");
    cuda_check(cudaStreamSynchronize(s), "sync BD");
  }
  unsigned status(cudaStream_t s) override {
    unsigned st = 0;
    cuda_check(cudaMemcpyAsync(&st, P_.status, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "BD status");
    cuda_check(cudaStreamSynchronize(s), "sync BD status");
    return st;
  }

 private:
  int reps_;
  BDK<R> P_;
  size_t smem_ = 0;
};

int bd_fail(int code) { return code; }

}  // namespace
}  // namespace gblb

using namespace gblb;

struct lb_bd {
  std::unique_ptr<BDBase> b;
  int reps = 0, N = 0;
  int64_t step = 0;
  cudaStream_t stream = nullptr;
};

namespace {

template <class F>
int bd_guard(F&& f) {
  try {
    return f();
  } catch (const LbError& e) {
    return bd_fail(e.code);
  } catch (...) {
    return LB_ERR_CUDA;
  }
}

template <class R>
BDK<R> bd_params(int N, double kT, double zeta, double eta_s, double dt, double k_fene, double R0, double eps,
                 double sigma, int hi, int degree, int piters, uint64_t seed) {
  BDK<R> P;
  memset(&P, 0, sizeof(P));
  P.N = N;
  P.kT = (R)kT;
  P.zeta = (R)zeta;
  P.eta = (R)eta_s;
  P.radius = (R)(zeta / (6.0 * M_PI * eta_s));
  P.dt = (R)dt;
  P.kfene = (R)k_fene;
  P.R0sq = (R)(R0 * R0);
  P.eps = (R)eps;
  P.sig2 = (R)(sigma * sigma);
  P.rc2 = (R)(pow(2.0, 1.0 / 3.0) * sigma * sigma);
  P.hi = hi ? 1 : 0;
  P.degree = degree;
  P.piters = piters;
  P.k0 = (uint32_t)(seed & 0xffffffffu);
  return P;
}

}  // namespace

extern "C" {

int lb_bd_create(lb_bd** out, int replicas, int N, double kT, double zeta, double eta_s, double dt, double k_fene,
                 double R0, double eps, double sigma, int hi, int degree, int power_iters, uint64_t seed,
                 const double* x0, int precision) {
  if (!out || !x0 || replicas < 1 || replicas > 65535 || N < 1 || !(kT > 0) || !(zeta > 0) || !(eta_s > 0) ||
      !(dt > 0) || !(k_fene >= 0) || !(R0 > 0) || !(sigma > 0) || degree < 1 || degree > kBDMaxDegree ||
      power_iters < 1 || (precision != LB_FP64 && precision != LB_FP32))
    return LB_ERR_ARG;
  const int max_n = precision == LB_FP64 ? 52 : 74;  // the 3N x 3N matrix lives in shared memory
  if (N > max_n) return LB_ERR_ARG;
  return bd_guard([&] {
    std::unique_ptr<lb_bd> b(new lb_bd);
    b->reps = replicas;
    b->N = N;
    if (precision == LB_FP64)
      b->b.reset(new BDT<double>(replicas, bd_params<double>(N, kT, zeta, eta_s, dt, k_fene, R0, eps, sigma, hi,
                                                             degree, power_iters, seed),
                                 x0));
    else
      b->b.reset(new BDT<float>(replicas, bd_params<float>(N, kT, zeta, eta_s, dt, k_fene, R0, eps, sigma, hi,
                                                           degree, power_iters, seed),
                                x0));
    *out = b.release();
    return (int)LB_OK;
  });
}

int lb_bd_set_stream(lb_bd* b, void* stream) {
  if (!b) return LB_ERR_ARG;
  b->stream = (cudaStream_t)stream;
  return LB_OK;
}

int lb_bd_step(lb_bd* b, int64_t n) {
  if (!b || n < 0) return LB_ERR_ARG;
  return bd_guard([&] {
    b->b->step(n, (uint32_t)b->step, b->stream);
    b->step += n;
    return (int)LB_OK;
  });
}

int lb_bd_sync(lb_bd* b) {
  if (!b) return LB_ERR_ARG;
  return bd_guard([&] { return b->b->status(b->stream) ? (int)LB_ERR_FENE : (int)LB_OK; });
}

int lb_bd_get_beads(lb_bd* b, double* x, size_t cap) {
  if (!b || !x) return LB_ERR_ARG;
  if (cap < (size_t)b->reps * 3 * b->N) return LB_ERR_ARG;
  return bd_guard([&] {
    b->b->get(x, b->stream);
    return b->b->status(b->stream) ? (int)LB_ERR_FENE : (int)LB_OK;
  });
}

int64_t lb_bd_get_step(lb_bd* b) { return b ? b->step : -1; }

void lb_bd_destroy(lb_bd* b) { delete b; }

}  // extern "C"
