// Batched replicas: R independent boxes of possibly different L (and chains of different N)
// advanced together, one launch per kernel stage for all replicas.
//
// The paper's explicit-solvent runs form an ensemble of independent boxes (box sizes
// L = 10..35 for the finite-size extrapolation, Sec. II E and Sec. III B; the CPU-cost study
// sums three box sizes per chain length, Sec. III C).  Each replica owns an ordinary engine
// (its memory, noise keys and chain); the batch drives them in lockstep:
//   - k_batch_bead: one thread block per replica's chain; it releases the LB kernel of the
//     same step at its start (programmatic dependent launch, one stream),
//   - k_batch_lb: a tile table over all replicas' nodes, persistent thread blocks walking it;
//     nodes marked by the previous step's bead kernel add its force corrections to what they
//     pull, the bead kernel adds them to its gathers,
//   - k_batch_apply: the last step's force corrections, once at the end of each call.
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
  PendK<R> pd[2];  // pending corrections of a step of parity j: writes slot j, reads slot j ^ 1
  unsigned long long nnodes;
  unsigned long long tile0;  // first global tile of this replica
  int has_chain;
};

__global__ void k_set_step(uint32_t* d_step, uint32_t v) { *d_step = v; }
__global__ void k_add_step(uint32_t* d_step, uint32_t v) { *d_step += v; }

// n / d for n < 2^24 and 2 <= d <= 256 by one multiply-high with m = ceil(2^32 / d): with
// e = m d - 2^32 < d, n m / 2^32 = n / d + n e / (d 2^32) and n e < 2^32 keeps the error below
// the distance of n / d to the next integer (checked exhaustively for every d and n in range).
__host__ __device__ __forceinline__ unsigned magic_of(unsigned d) {
  return (unsigned)((0x100000000ull + d - 1) / d);
}
__device__ __forceinline__ unsigned div_magic(unsigned n, unsigned m) { return __umulhi(n, m); }

// Per-replica fields of the batched LB kernel; the shared fluid parameters and up to
// kBatchGroup replicas travel in the kernel's parameter block (constant bank), so the
// collision's coefficients stay instruction operands as in the single-box kernel.
constexpr int kBatchGroup = 64;

// A replica's nodes are enumerated as thread slots: with two nodes per thread (even L) slot
// s is the pair (x0 = 2 (s mod L/2), row = s div L/2), otherwise the node (s mod L, s div L);
// row = y + L z.  Tiles of T consecutive slots; tile0 is the replica's first tile.
template <class S, class R>
struct BatchRep {
  S* pop[2];
  unsigned long long tile0, plane;
  unsigned nslots;   // L^3 / 2 (pairs) or L^3
  unsigned rowlen;   // slots per row: L / 2 or L
  unsigned mag_row;  // magic_of(rowlen)
  unsigned mag_L;    // magic_of(L)
  unsigned seg0;     // first mask word of the replica
  unsigned long long* nonpos;
  const R* p_dense[2];  // dense correction fields by slot
  unsigned L;
  int pair;
};

template <class S, class R>
struct BatchLB {
  FluidK<R> P;
  int nrep;
  unsigned long long total_tiles;
  const unsigned* mask[2];       // marks of the nodes that pull from pending nodes, by slot
  unsigned long long* counter;   // this group's two tile counters (by step parity)
  BatchRep<S, R> rep[kBatchGroup];
  RoundKeys rk[kBatchGroup];
};

// One tile (T = blockDim.x consecutive thread slots of replica r): pull-stream + collide
// (Sec. II B), one or two nodes per thread.  A node marked by the previous step adds that
// step's corrections to what it pulls (replicas without a chain have no correction field and
// are never marked); the pull is issued before the mark is known, and one copy of the
// collision follows, as in lb_tile.  Coordinates come from the slot by two multiply-highs.
template <class S, class R, bool DEV, bool NOISE>
__device__ __forceinline__ void batch_tile(const BatchLB<S, R>& B, const int r, const unsigned long long tile,
                                           const int parity, const uint32_t step, unsigned char* dsm) {
  const unsigned T = blockDim.x;
  const int pslot = parity ^ 1;  // the previous step's corrections
  const BatchRep<S, R>& rp = B.rep[r];
  const unsigned sl = (unsigned)(tile - rp.tile0) * T + threadIdx.x;
  if (sl >= rp.nslots) return;
  const unsigned L = rp.L;
  const unsigned row = div_magic(sl, rp.mag_row);
  const unsigned xs = sl - row * rp.rowlen;
  const unsigned z = div_magic(row, rp.mag_L);
  const unsigned y = row - z * L;
  const unsigned pl = (unsigned)rp.plane;
  const bool corr = rp.p_dense[pslot] != nullptr;
  R* col = reinterpret_cast<R*>(dsm);
  if (sizeof(R) == 4 && rp.pair) {
    const unsigned x0 = 2 * xs;
    const unsigned node = x0 + L * row;
    const unsigned mw = corr ? B.mask[pslot][rp.seg0 + (node >> kSegShift)] >> (node & 31u) : 0u;
    R n0[Q], n1[Q];
    lb_pull2<S, R, unsigned>(rp.pop[parity], L, pl, x0, y, z, n0, n1);
    if (mw & 3u) {  // marked nodes stage their corrections one after the other
#pragma unroll 1
      for (unsigned j = 0; j < 2; ++j) {
        if (!((mw >> j) & 1u)) continue;
        stage_corrections<R>(rp.p_dense[pslot], rp.plane, L, x0 + j, y, z, col + threadIdx.x, T);
        if (j == 0) {
#pragma unroll
          for (int i = 0; i < Q; ++i) n0[i] += col[threadIdx.x + i * T];
        } else {
#pragma unroll
          for (int i = 0; i < Q; ++i) n1[i] += col[threadIdx.x + i * T];
        }
      }
    }
    lb_collide2_store<S, R, DEV, NOISE, unsigned>(n0, n1, rp.pop[parity ^ 1], B.P, pl, B.rk[r], rp.nonpos, step,
                                                  node);
  } else {
    const unsigned node = xs + L * row;
    const unsigned mw = corr ? B.mask[pslot][rp.seg0 + (node >> kSegShift)] : 0u;
    R n[Q];
    lb_pull<S, R, unsigned>(rp.pop[parity], L, pl, xs, y, z, n);
    if ((mw >> (node & 31u)) & 1u) {
      stage_corrections<R>(rp.p_dense[pslot], rp.plane, L, xs, y, z, col + threadIdx.x, T);
#pragma unroll
      for (int i = 0; i < Q; ++i) n[i] += col[threadIdx.x + i * T];
    }
    lb_collide_store<S, R, DEV, NOISE, unsigned>(n, rp.pop[parity ^ 1], B.P, pl, B.rk[r], rp.nonpos, step, node);
  }
}

// tiles a persistent block takes from the counter at a time
constexpr unsigned kChunk = 2;

// PERSIST: persistent blocks take tiles from a per-group counter in chunks of kChunk (blocks
// that start late, e.g. beside a bead block, simply take fewer); each block's tiles increase,
// so the replica search only moves forward.  The counter of this step's parity was zeroed by
// the previous step's bead kernel.  Otherwise one block per tile: the tile is the block
// index and the replica a binary search over the table, both uniform across the block, so the
// replica's fields (its Philox round keys among them) stay in the constant bank and uniform
// registers; the hardware block scheduler balances the load.
// FP32: at most 64 registers (two 512-thread or four 256-thread blocks per SM), as the
// single-box kernel with two nodes per thread.
template <class S, class R, bool DEV, bool NOISE, bool PERSIST>
__global__ void __launch_bounds__(512, sizeof(R) == 4 ? 2 : 1) k_batch_lb(const __grid_constant__ BatchLB<S, R> B, int parity,
                                                   const uint32_t* __restrict__ d_step, uint32_t j) {
  extern __shared__ __align__(16) unsigned char dsm[];  // staged corrections, 19 x T
  const uint32_t step = *d_step + j;
  if (!PERSIST) {
    const unsigned long long tile = blockIdx.x;
    int lo = 0, hi = B.nrep - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (B.rep[mid].tile0 <= tile) lo = mid;
      else hi = mid - 1;
    }
    batch_tile<S, R, DEV, NOISE>(B, lo, tile, parity, step, dsm);
    return;
  }
  __shared__ unsigned long long s_next;
  unsigned long long* ctr = B.counter + parity;
  if (threadIdx.x == 0) s_next = atomicAdd(ctr, (unsigned long long)kChunk);
  __syncthreads();
  unsigned long long cur = s_next;
  int r = 0;
  while (cur < B.total_tiles) {
    __syncthreads();  // every thread has read s_next
    if (threadIdx.x == 0) s_next = atomicAdd(ctr, (unsigned long long)kChunk);  // next chunk, early
    const unsigned long long t_end = cur + kChunk < B.total_tiles ? cur + kChunk : B.total_tiles;
    for (unsigned long long tile = cur; tile < t_end; ++tile) {
      while (r + 1 < B.nrep && B.rep[r + 1].tile0 <= tile) ++r;  // uniform
      batch_tile<S, R, DEV, NOISE>(B, r, tile, parity, step, dsm);
    }
    __syncthreads();
    cur = s_next;
  }
}

// One 256-thread block per replica's chain: in FP32 at most 80 registers per thread, which
// leaves room on its SM for four 256-thread LB blocks.  Block 0 also zeroes the tile
// counters the next step's LB launches will use.
template <class S, class R, bool DEV>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 3 : 1) k_batch_bead(const ReplicaK<S, R>* __restrict__ reps, int parity,
                                                     const uint32_t* __restrict__ d_step, uint32_t j,
                                                     unsigned long long* __restrict__ counters, int ngroups) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ FluidK<R> sP;
  __shared__ ChainK<R> sC;
  allow_dependent_launch();
  if (blockIdx.x == 0)
    for (int g = threadIdx.x; g < ngroups; g += blockDim.x) counters[2 * g + (parity ^ 1)] = 0ull;
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
  const uint32_t step = *d_step + j;
  PendK<R> Pd = rp.pd[parity];
  Pd.have_prev = 1;  // an empty list after a flush
  bead_step_block<S, R, DEV>(rp.pop[parity], sP, sC, Pd, step, smem);
}

// zero the counts of one pending slot of every replica (after the flush applied it)
template <class S, class R>
__global__ void k_batch_clear(const ReplicaK<S, R>* __restrict__ reps, int nrep, int slot) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrep; r += gridDim.x * blockDim.x)
    if (reps[r].has_chain) *reps[r].pd[slot].cur_count = 0;
}

// B[i][node] += dn_i for the pending list of `slot` of every replica, into buffer `buf`, and
// those entries of the dense correction field back to zero
template <class S, class R>
__global__ void __launch_bounds__(256) k_batch_apply(const ReplicaK<S, R>* __restrict__ reps, int buf, int slot) {
  const ReplicaK<S, R>& rp = reps[blockIdx.z];
  if (!rp.has_chain) return;
  const PendK<R>& pd = rp.pd[slot];
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= *pd.cur_count) return;
  const int i = blockIdx.y;
  const int4 q = pd.cur_pos[u];
  const unsigned long long off = (unsigned long long)i * rp.P.plane + (unsigned)q.x;
  S* p = rp.pop[buf] + off;
  st<S, R>(p, ld<S, R>(p) + pd.cur_dn[i * pd.cap + u]);
  pd.cur_dense[off] = R(0);
  if (i == 0) clear_marks(pd.cur_mask, pd.seg0, (int)rp.P.L, q.y, q.z, q.w);
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
  virtual void set_options(int noise_fluid, int noise_beads, int stress_only) = 0;
};

template <class S, class R, bool DEV>
class BatchT final : public Batch {
 public:
  // noise switches of every replica (before initialise: the kernels' tables take them then)
  void set_options(int noise_fluid, int noise_beads, int stress_only) override {
    for (auto& e : eng_) {
      Config c = e->config();
      c.noise_fluid = noise_fluid ? 1 : 0;
      c.noise_beads = noise_beads ? 1 : 0;
      c.stress_only = stress_only ? 1 : 0;
      e->set_config(c);
    }
  }

  BatchT(const std::vector<Config>& cfgs, const std::vector<std::vector<double>>& x0) : x0_(x0) {
    for (const Config& c : cfgs) eng_.emplace_back(new EngineT<S, R, DEV>(c));
    size_t off = 0;
    for (auto& e : eng_) {
      off = align_up(off, 256);
      offs_.push_back(off);
      off += e->workspace_bytes();
    }
    // marks: one 32-bit word per 32 nodes of every replica, two slots
    max_segs_ = 0;
    for (auto& e : eng_) max_segs_ += (e->nodes() + 31) >> kSegShift;
    off = align_up(off, 256);
    flags_off_ = off;
    off += 2 * max_segs_ * sizeof(unsigned);
    off = align_up(off, 256);
    counters_off_ = off;
    off += 2 * (cfgs.size() / kBatchGroup + 1) * sizeof(unsigned long long);
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
    if (cap_) cudaStreamDestroy(cap_);
  }

  size_t workspace_bytes() const override { return bytes_; }

  void bind(void* base) override {
    base_ = static_cast<unsigned char*>(base);
    for (size_t r = 0; r < eng_.size(); ++r) eng_[r]->bind(base_ + offs_[r]);
    d_reps_ = reinterpret_cast<ReplicaK<S, R>*>(base_ + table_off_);
    flags_[0] = reinterpret_cast<unsigned*>(base_ + flags_off_);
    flags_[1] = flags_[0] + max_segs_;
    counters_ = reinterpret_cast<unsigned long long*>(base_ + counters_off_);
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
    // the engines zeroed their pending counts; no node is marked
    cuda_check(cudaMemsetAsync(flags_[0], 0, 2 * max_segs_ * sizeof(unsigned), s), "memset marks");
    const size_t lbsm = (size_t)Q * 512 * sizeof(R);
    if (lbsm > 48 * 1024) {  // FP64: staged corrections of a 512-thread tile
      for (int v = 0; v < 4; ++v)
        cuda_check(cudaFuncSetAttribute(lb_kernel(v & 1, v >> 1), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)lbsm),
                   "batch LB shared memory");
    }
    cuda_check(cudaMemsetAsync(counters_, 0, 2 * (eng_.size() / kBatchGroup + 1) * sizeof(unsigned long long), s),
               "memset tile counters");
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
    flush(s);
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
        flush(s);
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
    if (cap_) return;
    cuda_check(cudaStreamCreateWithFlags(&cap_, cudaStreamNonBlocking), "capture stream");
  }

  // apply the last step's corrections (slot = parity of that step) to the current buffer and
  // empty that slot, so the next call's first step finds nothing pending
  void flush(cudaStream_t s) {
    const int par = eng_[0]->parity();
    const int slot = par ^ 1;
    const int R_ = (int)eng_.size();
    k_batch_apply<S, R><<<dim3((cap_max_ + 255) / 256, Q, R_), 256, 0, s>>>(d_reps_, par, slot);
    cuda_check(cudaGetLastError(), "batch apply");
    k_batch_clear<S, R><<<1, 256, 0, s>>>(d_reps_, R_, slot);
    cuda_check(cudaGetLastError(), "batch clear");
  }

  // two nodes per thread slot for even boxes in single-precision arithmetic (as the single-box
  // kernel)
  static bool pair_slots(unsigned L) { return (L & 1u) == 0 && sizeof(R) == 4; }

  // the batched LB kernel for noise on/off, persistent blocks or one block per tile
  using BatchLbKernel = void (*)(const BatchLB<S, R>, int, const uint32_t*, uint32_t);
  static BatchLbKernel lb_kernel(bool noise, bool persist) {
    if (noise) return persist ? k_batch_lb<S, R, DEV, true, true> : k_batch_lb<S, R, DEV, true, false>;
    return persist ? k_batch_lb<S, R, DEV, false, true> : k_batch_lb<S, R, DEV, false, false>;
  }

  void drop_graph() {
    if (graph_exec_) cudaGraphExecDestroy(graph_exec_);
    graph_exec_ = nullptr;
  }

  void upload_table(cudaStream_t s) {
    std::vector<ReplicaK<S, R>> tab(eng_.size());
    unsigned long long t = 0, segs = 0;
    for (size_t r = 0; r < eng_.size(); ++r) {
      ReplicaK<S, R>& q = tab[r];
      memset(&q, 0, sizeof(q));
      q.pop[0] = eng_[r]->buffer(0);
      q.pop[1] = eng_[r]->buffer(1);
      q.P = eng_[r]->fluid_params();
      q.C = eng_[r]->chain_params();
      q.nnodes = eng_[r]->nodes();
      q.tile0 = t;
      q.has_chain = eng_[r]->chain_length() > 0;
      for (int jj = 0; jj < 2; ++jj) {
        PendK<R>& pd = q.pd[jj];
        pd.prev_mask = flags_[jj ^ 1];
        pd.prev_dense = eng_[r]->pending_dense(jj ^ 1);
        pd.cur_dense = eng_[r]->pending_dense(jj);
        pd.plane = eng_[r]->plane();
        pd.cur_pos = eng_[r]->pending_pos(jj);
        pd.cur_dn = eng_[r]->pending_dn(jj);
        pd.cur_count = eng_[r]->pending_count(jj);
        pd.cur_mask = flags_[jj];
        pd.mark = 1;
        pd.cap = eng_[r]->pending_capacity();
        pd.seg0 = (unsigned)segs;
      }
      segs += (q.nnodes + 31) >> kSegShift;
      noise_ = q.P.ncalls > 0;
      t += (q.nnodes / (pair_slots(q.P.L) ? 2 : 1) + threads_ - 1) / threads_;
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
      G.mask[0] = flags_[0];
      G.mask[1] = flags_[1];
      G.counter = counters_ + 2 * groups_.size();
      for (size_t r = g0; r < g1; ++r) {
        BatchRep<S, R>& q = G.rep[r - g0];
        q.pop[0] = tab[r].pop[0];
        q.pop[1] = tab[r].pop[1];
        q.tile0 = tt;
        q.plane = tab[r].P.plane;
        q.nonpos = tab[r].P.nonpos;
        q.L = tab[r].P.L;
        q.pair = pair_slots(q.L);
        q.rowlen = q.pair ? q.L / 2 : q.L;
        q.nslots = (unsigned)(tab[r].nnodes / (q.pair ? 2 : 1));
        q.mag_row = magic_of(q.rowlen);
        q.mag_L = magic_of(q.L);
        q.seg0 = tab[r].pd[0].seg0;
        for (int jj = 0; jj < 2; ++jj) q.p_dense[jj] = eng_[r]->pending_dense(jj);
        G.rk[r - g0] = tab[r].P.rk;
        tt += (q.nslots + threads_ - 1) / threads_;
      }
      G.total_tiles = tt;
      groups_.push_back(G);
    }
    cuda_check(cudaMemcpyAsync(d_reps_, tab.data(), tab.size() * sizeof(ReplicaK<S, R>), cudaMemcpyHostToDevice, s),
               "upload replica table");
    cuda_check(cudaStreamSynchronize(s), "sync table");
    table_threads_ = threads_;
  }

  // one lockstep step; kernels read step = *d_step + j (advance: bump the counter after).
  // The bead kernel releases the first LB launch at its start; the next step's bead kernel,
  // an ordinary launch, waits for both.  The force corrections stay pending (see k_batch_lb).
  void launch_step(cudaStream_t s, uint32_t j, bool advance) {
    const int par = eng_[0]->parity();
    const int R_ = (int)eng_.size();
    k_batch_bead<S, R, DEV><<<R_, 256, smem_, s>>>(d_reps_, par, d_step_, j, counters_, (int)groups_.size());
    cuda_check(cudaGetLastError(), "batch bead");
    int dev = 0, sms = 0;
    cuda_check(cudaGetDevice(&dev), "device");
    cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    bool first = true;
    for (const BatchLB<S, R>& G : groups_) {
      unsigned grid = (unsigned)G.total_tiles;
      if (bps_ > 0 && (unsigned long long)sms * bps_ < G.total_tiles) grid = (unsigned)(sms * bps_);
      cudaLaunchConfig_t lc;
      memset(&lc, 0, sizeof(lc));
      lc.gridDim = dim3(grid);
      lc.blockDim = dim3(threads_);
      lc.dynamicSmemBytes = (size_t)Q * threads_ * sizeof(R);
      lc.stream = s;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      at[0].val.programmaticStreamSerializationAllowed = 1;
      lc.attrs = at;
      lc.numAttrs = first ? 1 : 0;
      cuda_check(cudaLaunchKernelEx(&lc, lb_kernel(noise_, bps_ > 0), G, par, (const uint32_t*)d_step_, j),
                 "batch LB");
      first = false;
    }
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
  size_t table_off_ = 0, step_off_ = 0, flags_off_ = 0, counters_off_ = 0, bytes_ = 0, smem_ = 0;
  unsigned long long* counters_ = nullptr;
  size_t max_segs_ = 0;
  unsigned* flags_[2] = {nullptr, nullptr};  // node marks by slot
  unsigned char* base_ = nullptr;
  ReplicaK<S, R>* d_reps_ = nullptr;
  uint32_t* d_step_ = nullptr;
  unsigned long long total_tiles_ = 0;
  int threads_ = 256, bps_ = 0, table_threads_ = -1, cap_max_ = 8;
  bool noise_ = true;
  cudaStream_t cap_ = nullptr;
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

int lb_batch_set_options(lb_batch* bt, int noise_fluid, int noise_beads, int stress_only) {
  if (!bt) return LB_ERR_ARG;
  if (bt->live) return LB_ERR_STATE;
  for (Config& c : bt->cfgs) {
    c.noise_fluid = noise_fluid ? 1 : 0;
    c.noise_beads = noise_beads ? 1 : 0;
    c.stress_only = stress_only ? 1 : 0;
  }
  bt->b->set_options(noise_fluid, noise_beads, stress_only);
  return LB_OK;
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
