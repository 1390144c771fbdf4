// Batched replicas: R independent boxes of possibly different L (and chains of different N)
// advanced together, one launch per kernel stage for all replicas.
//
// The paper's explicit-solvent runs form an ensemble of independent boxes (box sizes
// L = 10..35 for the finite-size extrapolation, Sec. II E and Sec. III B; the CPU-cost study
// sums three box sizes per chain length, Sec. III C).  Each replica owns an ordinary engine
// (its memory, noise keys and chain); the batch drives them in lockstep:
//   - k_batch_bead: one thread block per replica's chain (side stream, concurrent),
//   - k_batch_lb: a tile table over all replicas' nodes, persistent thread blocks walking it,
//   - k_batch_apply: the force corrections of every replica.
// Step indices come from a device counter so that a captured CUDA graph of G steps (G even)
// can be replayed; the tile size and the number of persistent blocks are chosen by a
// measuring autotuner.
#include <math.h>
#include <string.h>

#include <memory>
#include <vector>

#include "../../include/lb.h"
#include "lb_engine_impl.cuh"

namespace gblb {

template <class S, class R>
struct ReplicaK {
  S* pop[2];
  FluidK<R> P;
  ChainK<R> C;
  unsigned long long nnodes;
  unsigned long long tile0;  // first global tile of this replica
  float invL;
  int has_chain;
};

__global__ void k_set_step(uint32_t* d_step, uint32_t v) { *d_step = v; }
__global__ void k_add_step(uint32_t* d_step, uint32_t v) { *d_step += v; }

// Decompose node = x + L (y + L z), node < 2^24 (boxes up to 256^3), with a float
// reciprocal and an exact integer correction.
__device__ __forceinline__ unsigned div_small(unsigned n, unsigned L, float invL, unsigned& rem) {
  int q = __float2int_rz(__uint2float_rn(n) * invL);
  int r = (int)n - q * (int)L;
  if (r < 0) {
    --q;
    r += (int)L;
  } else if (r >= (int)L) {
    ++q;
    r -= (int)L;
  }
  rem = (unsigned)r;
  return (unsigned)q;
}

// Per-replica fields of the batched LB kernel; the shared fluid parameters and up to
// kBatchGroup replicas travel in the kernel's parameter block (constant bank), so the
// collision's coefficients stay instruction operands as in the single-box kernel.
constexpr int kBatchGroup = 64;

template <class S>
struct BatchRep {
  S* pop[2];
  unsigned long long nnodes, tile0, plane;
  unsigned long long* nonpos;
  unsigned L;
  float invL;
};

template <class S, class R>
struct BatchLB {
  FluidK<R> P;
  int nrep;
  unsigned long long total_tiles;
  BatchRep<S> rep[kBatchGroup];
  RoundKeys rk[kBatchGroup];
};

template <class S, class R, bool DEV, bool NOISE>
__global__ void __launch_bounds__(512) k_batch_lb(const __grid_constant__ BatchLB<S, R> B, int parity,
                                                   const uint32_t* __restrict__ d_step, uint32_t j) {
  const uint32_t step = *d_step + j;
  const unsigned T = blockDim.x;
  // contiguous chunk of tiles per block: consecutive tiles mostly share a replica
  const unsigned long long per = (B.total_tiles + gridDim.x - 1) / gridDim.x;
  const unsigned long long t_begin = blockIdx.x * per;
  const unsigned long long t_end = t_begin + per < B.total_tiles ? t_begin + per : B.total_tiles;
  int r = 0;
  for (unsigned long long tile = t_begin; tile < t_end; ++tile) {
    while (r + 1 < B.nrep && B.rep[r + 1].tile0 <= tile) ++r;  // uniform
    const BatchRep<S>& rp = B.rep[r];
    const unsigned long long node = (tile - rp.tile0) * T + threadIdx.x;
    if (node < rp.nnodes) {
      const unsigned L = rp.L;
      unsigned x, y;
      const unsigned t = div_small((unsigned)node, L, rp.invL, x);
      const unsigned z = div_small(t, L, rp.invL, y);
      lb_node_update<S, R, DEV, NOISE>(rp.pop[parity], rp.pop[parity ^ 1], B.P, L, rp.plane, B.rk[r], rp.nonpos,
                                       step, x, y, z);
    }
  }
}

template <class S, class R, bool DEV>
__global__ void __launch_bounds__(512) k_batch_bead(const ReplicaK<S, R>* __restrict__ reps, int parity,
                                                     const uint32_t* __restrict__ d_step, uint32_t j) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ FluidK<R> sP;
  __shared__ ChainK<R> sC;
  const ReplicaK<S, R>& rp = reps[blockIdx.x];
  if (!rp.has_chain) return;
  {
    const unsigned* a = reinterpret_cast<const unsigned*>(&rp.P);
    unsigned* b = reinterpret_cast<unsigned*>(&sP);
    for (unsigned w = threadIdx.x; w < sizeof(FluidK<R>) / 4; w += blockDim.x) b[w] = a[w];
    const unsigned* c = reinterpret_cast<const unsigned*>(&rp.C);
    unsigned* d = reinterpret_cast<unsigned*>(&sC);
    for (unsigned w = threadIdx.x; w < sizeof(ChainK<R>) / 4; w += blockDim.x) d[w] = c[w];
  }
  __syncthreads();
  bead_step_block<S, R, DEV>(rp.pop[parity], sP, sC, pend_complete(sC), *d_step + j, smem);
}

template <class S, class R>
__global__ void __launch_bounds__(256) k_batch_apply(const ReplicaK<S, R>* __restrict__ reps, int parity) {
  const ReplicaK<S, R>& rp = reps[blockIdx.z];
  if (!rp.has_chain) return;
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= *rp.C.p_count) return;
  const int i = blockIdx.y;
  S* p = rp.pop[parity ^ 1] + (unsigned long long)i * rp.P.plane + (unsigned)rp.C.p_pos[u].x;
  st<S, R>(p, ld<S, R>(p) + rp.C.p_dn[i * rp.C.cap + u]);
}

class Batch {
 public:
  virtual ~Batch() {}
  virtual size_t workspace_bytes() const = 0;
  virtual void bind(void* base) = 0;
  virtual void initialise(cudaStream_t s) = 0;
  virtual void step(int64_t n, uint32_t k0, cudaStream_t s) = 0;
  virtual Engine& replica(int r) = 0;
  virtual void autotune(cudaStream_t s, int* threads, int* blocks_per_sm) = 0;
  virtual void set_shape(int threads, int blocks_per_sm) = 0;
};

template <class S, class R, bool DEV>
class BatchT final : public Batch {
 public:
  BatchT(const std::vector<Config>& cfgs, const std::vector<std::vector<double>>& x0) : x0_(x0) {
    for (const Config& c : cfgs) eng_.emplace_back(new EngineT<S, R, DEV>(c));
    size_t off = 0;
    for (auto& e : eng_) {
      off = align_up(off, 256);
      offs_.push_back(off);
      off += e->workspace_bytes();
    }
    off = align_up(off, 256);
    table_off_ = off;
    off += cfgs.size() * sizeof(ReplicaK<S, R>);
    off = align_up(off, 256);
    step_off_ = off;
    off += 256;
    bytes_ = align_up(off, 256);
  }
  ~BatchT() override {
    if (graph_exec_) cudaGraphExecDestroy(graph_exec_);
    if (side_) cudaStreamDestroy(side_);
    if (cap_) cudaStreamDestroy(cap_);
    if (ev_ready_) cudaEventDestroy(ev_ready_);
    if (ev_bead_) cudaEventDestroy(ev_bead_);
  }

  size_t workspace_bytes() const override { return bytes_; }

  void bind(void* base) override {
    base_ = static_cast<unsigned char*>(base);
    for (size_t r = 0; r < eng_.size(); ++r) eng_[r]->bind(base_ + offs_[r]);
    d_reps_ = reinterpret_cast<ReplicaK<S, R>*>(base_ + table_off_);
    d_step_ = reinterpret_cast<uint32_t*>(base_ + step_off_);
  }

  void initialise(cudaStream_t s) override {
    for (size_t r = 0; r < eng_.size(); ++r)
      eng_[r]->initialise(x0_[r].empty() ? nullptr : x0_[r].data(), nullptr, s);
    smem_ = 0;
    for (auto& e : eng_)
      if (e->chain_length() > 0 && e->bead_smem_bytes() > smem_) smem_ = e->bead_smem_bytes();
    if (smem_ > 48 * 1024)
      cuda_check(cudaFuncSetAttribute(k_batch_bead<S, R, DEV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem_),
                 "batch bead shared memory");
    cap_max_ = 8;
    for (auto& e : eng_) cap_max_ = e->pending_capacity() > cap_max_ ? e->pending_capacity() : cap_max_;
    upload_table(s);
    drop_graph();
  }

  Engine& replica(int r) override { return *eng_[r]; }

  void set_shape(int threads, int blocks_per_sm) override {
    threads_ = threads;
    bps_ = blocks_per_sm;
    drop_graph();
  }

  // Lockstep steps k0 .. k0 + n - 1: CUDA graphs of kGraph steps where possible.
  void step(int64_t n, uint32_t k0, cudaStream_t s) override {
    if (n <= 0) return;
    ensure_streams();
    if (table_threads_ != threads_) upload_table(s);
    k_set_step<<<1, 1, 0, s>>>(d_step_, k0);
    cuda_check(cudaGetLastError(), "set step");
    int64_t done = 0;
    if (n >= kGraph && eng_[0]->parity() == 0) {
      if (!graph_exec_) build_graph(s);
      for (; done + kGraph <= n; done += kGraph) cuda_check(cudaGraphLaunch(graph_exec_, s), "graph launch");
    }
    for (int64_t j = done; j < n; ++j) launch_step(s, (uint32_t)(j - done), /*advance=*/false);
    if (done < n) {
      k_add_step<<<1, 1, 0, s>>>(d_step_, (uint32_t)(n - done));
      cuda_check(cudaGetLastError(), "advance step");
    }
  }

  void autotune(cudaStream_t s, int* best_threads, int* best_bps) override {
    ensure_streams();
    int dev = 0, sms = 0;
    cuda_check(cudaGetDevice(&dev), "device");
    cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    const int cand_t[3] = {128, 256, 512};
    const int cand_b[4] = {0, 2, 4, 8};
    cudaEvent_t e0, e1;
    cuda_check(cudaEventCreate(&e0), "event");
    cuda_check(cudaEventCreate(&e1), "event");
    float best = 1e30f;
    int bt = threads_, bb = bps_;
    for (int t : cand_t)
      for (int b : cand_b) {
        if (b > 0 && b * t > 2048) continue;
        set_shape(t, b);
        upload_table(s);
        k_set_step<<<1, 1, 0, s>>>(d_step_, 0);
        for (int w = 0; w < 2; ++w) launch_step(s, 0, true);
        cuda_check(cudaEventRecord(e0, s), "event");
        for (int w = 0; w < 6; ++w) launch_step(s, 0, true);
        cuda_check(cudaEventRecord(e1, s), "event");
        cuda_check(cudaEventSynchronize(e1), "event sync");
        float ms = 0;
        cuda_check(cudaEventElapsedTime(&ms, e0, e1), "event time");
        if (ms < best) {
          best = ms;
          bt = t;
          bb = b;
        }
      }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    set_shape(bt, bb);
    // the trial steps changed the state: start again from the initial configuration
    initialise(s);
    *best_threads = bt;
    *best_bps = bb;
    (void)sms;
  }

 private:
  static constexpr int kGraph = 16;

  void ensure_streams() {
    if (side_) return;
    int least = 0, greatest = 0;
    cuda_check(cudaDeviceGetStreamPriorityRange(&least, &greatest), "stream priorities");
    cuda_check(cudaStreamCreateWithPriority(&side_, cudaStreamNonBlocking, greatest), "side stream");
    cuda_check(cudaStreamCreateWithFlags(&cap_, cudaStreamNonBlocking), "capture stream");
    cuda_check(cudaEventCreateWithFlags(&ev_ready_, cudaEventDisableTiming), "event");
    cuda_check(cudaEventCreateWithFlags(&ev_bead_, cudaEventDisableTiming), "event");
  }

  void drop_graph() {
    if (graph_exec_) cudaGraphExecDestroy(graph_exec_);
    graph_exec_ = nullptr;
  }

  void upload_table(cudaStream_t s) {
    std::vector<ReplicaK<S, R>> tab(eng_.size());
    unsigned long long t = 0;
    for (size_t r = 0; r < eng_.size(); ++r) {
      ReplicaK<S, R>& q = tab[r];
      memset(&q, 0, sizeof(q));
      q.pop[0] = eng_[r]->buffer(0);
      q.pop[1] = eng_[r]->buffer(1);
      q.P = eng_[r]->fluid_params();
      q.C = eng_[r]->chain_params();
      q.nnodes = eng_[r]->nodes();
      q.tile0 = t;
      q.invL = 1.0f / (float)q.P.L;
      q.has_chain = eng_[r]->chain_length() > 0;
      noise_ = q.P.ncalls > 0;
      t += (q.nnodes + threads_ - 1) / threads_;
    }
    total_tiles_ = t;
    groups_.clear();
    for (size_t g0 = 0; g0 < eng_.size(); g0 += kBatchGroup) {
      BatchLB<S, R> G;
      memset(&G, 0, sizeof(G));
      G.P = tab[g0].P;
      unsigned long long tt = 0;
      const size_t g1 = g0 + kBatchGroup < eng_.size() ? g0 + kBatchGroup : eng_.size();
      G.nrep = (int)(g1 - g0);
      for (size_t r = g0; r < g1; ++r) {
        BatchRep<S>& q = G.rep[r - g0];
        q.pop[0] = tab[r].pop[0];
        q.pop[1] = tab[r].pop[1];
        q.nnodes = tab[r].nnodes;
        q.tile0 = tt;
        q.plane = tab[r].P.plane;
        q.nonpos = tab[r].P.nonpos;
        q.L = tab[r].P.L;
        q.invL = tab[r].invL;
        G.rk[r - g0] = tab[r].P.rk;
        tt += (q.nnodes + threads_ - 1) / threads_;
      }
      G.total_tiles = tt;
      groups_.push_back(G);
    }
    cuda_check(cudaMemcpyAsync(d_reps_, tab.data(), tab.size() * sizeof(ReplicaK<S, R>), cudaMemcpyHostToDevice, s),
               "upload replica table");
    cuda_check(cudaStreamSynchronize(s), "sync table");
    table_threads_ = threads_;
  }

  // one lockstep step; kernels read step = *d_step + j (advance: bump the counter after)
  void launch_step(cudaStream_t s, uint32_t j, bool advance) {
    const int par = eng_[0]->parity();
    const int R_ = (int)eng_.size();
    cuda_check(cudaEventRecord(ev_ready_, s), "record ready");
    cuda_check(cudaStreamWaitEvent(side_, ev_ready_, 0), "wait ready");
    k_batch_bead<S, R, DEV><<<R_, 512, smem_, side_>>>(d_reps_, par, d_step_, j);
    cuda_check(cudaGetLastError(), "batch bead");
    cuda_check(cudaEventRecord(ev_bead_, side_), "record bead");
    int dev = 0, sms = 0;
    cuda_check(cudaGetDevice(&dev), "device");
    cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    for (const BatchLB<S, R>& G : groups_) {
      unsigned grid = (unsigned)G.total_tiles;
      if (bps_ > 0 && (unsigned long long)sms * bps_ < G.total_tiles) grid = (unsigned)(sms * bps_);
      if (noise_)
        k_batch_lb<S, R, DEV, true><<<grid, threads_, 0, s>>>(G, par, d_step_, j);
      else
        k_batch_lb<S, R, DEV, false><<<grid, threads_, 0, s>>>(G, par, d_step_, j);
      cuda_check(cudaGetLastError(), "batch LB");
    }
    cuda_check(cudaStreamWaitEvent(s, ev_bead_, 0), "wait bead");
    k_batch_apply<S, R><<<dim3((cap_max_ + 255) / 256, Q, R_), 256, 0, s>>>(d_reps_, par);
    cuda_check(cudaGetLastError(), "batch apply");
    if (advance) k_add_step<<<1, 1, 0, s>>>(d_step_, 1);
    for (auto& e : eng_) e->flip();
  }

  // Captured on an internal stream (the legacy default stream cannot be captured) and
  // replayed on the caller's stream.
  void build_graph(cudaStream_t s) {
    drop_graph();
    cudaGraph_t g = nullptr;
    cuda_check(cudaStreamBeginCapture(cap_, cudaStreamCaptureModeThreadLocal), "begin capture");
    for (int j = 0; j < kGraph; ++j) launch_step(cap_, (uint32_t)j, false);
    k_add_step<<<1, 1, 0, cap_>>>(d_step_, kGraph);
    cuda_check(cudaStreamEndCapture(cap_, &g), "end capture");
    cuda_check(cudaGraphInstantiate(&graph_exec_, g, 0), "instantiate graph");
    cudaGraphDestroy(g);
    // capture only recorded the launches: kGraph (even) flips left the parity unchanged
  }

  std::vector<std::unique_ptr<EngineT<S, R, DEV>>> eng_;
  std::vector<BatchLB<S, R>> groups_;
  std::vector<std::vector<double>> x0_;
  std::vector<size_t> offs_;
  size_t table_off_ = 0, step_off_ = 0, bytes_ = 0, smem_ = 0;
  unsigned char* base_ = nullptr;
  ReplicaK<S, R>* d_reps_ = nullptr;
  uint32_t* d_step_ = nullptr;
  unsigned long long total_tiles_ = 0;
  int threads_ = 256, bps_ = 0, table_threads_ = -1, cap_max_ = 8;
  bool noise_ = true;
  cudaStream_t side_ = nullptr, cap_ = nullptr;
  cudaEvent_t ev_ready_ = nullptr, ev_bead_ = nullptr;
  cudaGraphExec_t graph_exec_ = nullptr;
};

}  // namespace gblb

using namespace gblb;

struct lb_batch {
  std::unique_ptr<Batch> b;
  std::vector<Config> cfgs;
  cudaStream_t stream = nullptr;
  void* ws = nullptr;
  bool ws_owned = false;
  bool live = false;
  int64_t step = 0;
};

namespace {

int bfail(int code) { return code; }

template <class F>
int bguard(F&& f) {
  try {
    return f();
  } catch (const LbError& e) {
    return bfail(e.code);
  } catch (...) {
    return LB_ERR_CUDA;
  }
}

void bmaterialise(lb_batch* bt) {
  if (bt->live) return;
  if (!bt->ws) {
    void* p = nullptr;
    cuda_check(cudaMalloc(&p, bt->b->workspace_bytes()), "batch workspace");
    bt->ws = p;
    bt->ws_owned = true;
  }
  bt->b->bind(bt->ws);
  bt->b->initialise(bt->stream);
  bt->live = true;
}

}  // namespace

extern "C" {

int lb_batch_create(lb_batch** out, int R, const int* L, const int* N, const uint64_t* seeds, double rho, double eta,
                    double eta_b, double kT, double h, double a, double m, double zeta, double k_fene, double R0,
                    double eps, double sigma, const double* x0, int precision, int md_substeps) {
  if (!out || R < 1 || R > 4096 || !L || !seeds) return LB_ERR_ARG;
  if (md_substeps < 1 || md_substeps > 16) return LB_ERR_ARG;
  *out = nullptr;
  if (precision != LB_FP32 && precision != LB_FP64) return LB_ERR_ARG;
  if (!(rho > 0) || !(eta > 0) || !(eta_b > 0) || !(h > 0) || !(a > 0) || !(kT >= 0)) return LB_ERR_ARG;
  if (!(m > 0) || !(zeta >= 0) || !(k_fene >= 0) || !(R0 > 0) || !(eps >= 0) || !(sigma > 0)) return LB_ERR_ARG;
  return bguard([&] {
    std::vector<Config> cfgs(R);
    std::vector<std::vector<double>> xs(R);
    size_t off = 0;
    for (int r = 0; r < R; ++r) {
      Config& c = cfgs[r];
      if (L[r] < 4 || L[r] > 256) return (int)LB_ERR_ARG;
      const int Nr = N ? N[r] : 0;
      if (Nr < 0 || Nr > 1024 || (Nr > 0 && !x0) || 8ll * Nr * md_substeps > 16384) return (int)LB_ERR_ARG;
      c.L = L[r];
      c.rho = rho;
      c.eta = eta;
      c.eta_b = eta_b;
      c.kT = kT;
      c.h = h;
      c.a = a;
      c.seed = seeds[r];
      c.precision = precision;
      c.replica = r & 0xffffff;
      c.N = Nr;
      c.m = m;
      c.zeta = zeta;
      c.kfene = k_fene;
      c.R0 = R0;
      c.eps = eps;
      c.sigma = sigma;
      c.substeps = md_substeps;
      if (Nr > 0) {
        xs[r].assign(x0 + off, x0 + off + 3 * (size_t)Nr);
        off += 3 * (size_t)Nr;
        const double box = c.L * a;
        for (int i = 0; i + 1 < Nr; ++i) {
          double r2 = 0;
          for (int q = 0; q < 3; ++q) {
            double d = xs[r][3 * i + q] - xs[r][3 * (i + 1) + q];
            d -= box * nearbyint(d / box);
            r2 += d * d;
          }
          if (r2 >= R0 * R0) return (int)LB_ERR_FENE;
        }
      }
    }
    auto* bt = new lb_batch();
    bt->cfgs = cfgs;
    if (precision == LB_FP32)
      bt->b.reset(new BatchT<float, float, true>(cfgs, xs));
    else
      bt->b.reset(new BatchT<double, double, false>(cfgs, xs));
    *out = bt;
    return (int)LB_OK;
  });
}

int lb_batch_set_stream(lb_batch* bt, void* stream) {
  if (!bt) return LB_ERR_ARG;
  bt->stream = static_cast<cudaStream_t>(stream);
  return LB_OK;
}

int lb_batch_workspace_size(lb_batch* bt, size_t* bytes) {
  if (!bt || !bytes) return LB_ERR_ARG;
  *bytes = bt->b->workspace_bytes();
  return LB_OK;
}

int lb_batch_bind_workspace(lb_batch* bt, void* device_ptr, size_t bytes) {
  if (!bt || !device_ptr) return LB_ERR_ARG;
  if (bt->live) return LB_ERR_STATE;
  if (reinterpret_cast<uintptr_t>(device_ptr) % 256 != 0 || bytes < bt->b->workspace_bytes()) return LB_ERR_ARG;
  bt->ws = device_ptr;
  bt->ws_owned = false;
  return LB_OK;
}

int lb_batch_autotune(lb_batch* bt, int* threads, int* blocks_per_sm) {
  if (!bt || !threads || !blocks_per_sm) return LB_ERR_ARG;
  if (bt->live && bt->step > 0) return LB_ERR_STATE;
  return bguard([&] {
    bmaterialise(bt);
    bt->b->autotune(bt->stream, threads, blocks_per_sm);
    return (int)LB_OK;
  });
}

int lb_batch_set_shape(lb_batch* bt, int threads, int blocks_per_sm) {
  if (!bt || (threads != 128 && threads != 256 && threads != 512) || blocks_per_sm < 0 || blocks_per_sm > 16)
    return LB_ERR_ARG;
  bt->b->set_shape(threads, blocks_per_sm);
  return LB_OK;
}

int lb_batch_step(lb_batch* bt, int64_t n) {
  if (!bt || n < 0) return LB_ERR_ARG;
  return bguard([&] {
    bmaterialise(bt);
    bt->b->step(n, (uint32_t)bt->step, bt->stream);
    bt->step += n;
    return (int)LB_OK;
  });
}

int lb_batch_sync(lb_batch* bt) {
  if (!bt) return LB_ERR_ARG;
  return bguard([&] {
    if (!bt->live) return (int)LB_OK;
    cuda_check(cudaStreamSynchronize(bt->stream), "sync");
    for (size_t r = 0; r < bt->cfgs.size(); ++r) {
      const unsigned st = bt->b->replica((int)r).read_status(bt->stream);
      if (st & ST_FENE) return (int)LB_ERR_FENE;
      if (st & ST_NONFINITE) return (int)LB_ERR_NONFINITE;
    }
    return (int)LB_OK;
  });
}

int lb_batch_get_populations(lb_batch* bt, int r, double* out, size_t cap) {
  if (!bt || !out || r < 0 || r >= (int)bt->cfgs.size()) return LB_ERR_ARG;
  const size_t L = bt->cfgs[r].L;
  if (cap < 19 * L * L * L) return LB_ERR_ARG;
  return bguard([&] {
    bmaterialise(bt);
    bt->b->replica(r).get_populations(out, bt->stream);
    return (int)LB_OK;
  });
}

int lb_batch_get_beads(lb_batch* bt, int r, double* x, double* v, size_t cap) {
  if (!bt || r < 0 || r >= (int)bt->cfgs.size()) return LB_ERR_ARG;
  if (cap < 3 * (size_t)bt->cfgs[r].N) return LB_ERR_ARG;
  return bguard([&] {
    bmaterialise(bt);
    bt->b->replica(r).get_beads(x, v, bt->stream);
    return (int)LB_OK;
  });
}

int lb_batch_get_observables(lb_batch* bt, int r, double* out, size_t cap) {
  if (!bt || !out || r < 0 || r >= (int)bt->cfgs.size() || cap < LB_NOBS) return LB_ERR_ARG;
  return bguard([&] {
    bmaterialise(bt);
    bt->b->replica(r).observables(out, bt->step, 0, bt->stream);
    return (int)LB_OK;
  });
}

int lb_batch_accumulate(lb_batch* bt) {
  if (!bt) return LB_ERR_ARG;
  return bguard([&] {
    bmaterialise(bt);
    for (size_t r = 0; r < bt->cfgs.size(); ++r)
      if (bt->cfgs[r].N > 0) bt->b->replica((int)r).observables(nullptr, bt->step, 1, bt->stream);
    return (int)LB_OK;
  });
}

int64_t lb_batch_nodes(lb_batch* bt) {
  if (!bt) return -1;
  int64_t n = 0;
  for (auto& c : bt->cfgs) n += (int64_t)c.L * c.L * c.L;
  return n;
}

void lb_batch_destroy(lb_batch* bt) {
  if (!bt) return;
  bt->b.reset();
  if (bt->ws_owned && bt->ws) cudaFree(bt->ws);
  delete bt;
}

}  // extern "C"
