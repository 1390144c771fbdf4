// Engine implementation, templated on the population storage type S, the arithmetic type
// R and whether populations are stored as deviations from w_i rho0 (DEV).
#pragma once
#include <math.h>
#include <string.h>

#include <vector>

#include "lb_adjoint.cuh"
#include "lb_device.cuh"
#include "lb_engine.h"

namespace gblb {

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

template <class S, class R, bool DEV>
class EngineT final : public Engine {
 public:
  explicit EngineT(const Config& c) : cfg_(c) {
    L_ = c.L;
    nnodes_ = (unsigned long long)L_ * L_ * L_;
    plane_ = align_up(nnodes_, 64);
    N_ = c.N;
    nsub_ = c.substeps > 0 ? c.substeps : 1;
    cap_ = 8 * (N_ > 0 ? N_ : 1) * nsub_;
    nparts_ = (int)((nnodes_ + 255) / 256);
    layout(nullptr);
  }

  size_t workspace_bytes() const override { return bytes_; }

  void bind(void* base) override { layout(static_cast<unsigned char*>(base)); }

  void set_config(const Config& c) override { cfg_ = c; }

  void initialise(const double* x0, const double* v0, cudaStream_t s) override {
    snap_valid_ = false;
    {
      dim3 blk, grd;
      lb_launch_shape(blk, grd, pair_nodes());
      const size_t sb = lb_stage_bytes(blk);
      if (sb > 48 * 1024)  // FP64: staged corrections of a 256-thread tile
        for (int v = 0; v < 8; ++v)
          cuda_check(cudaFuncSetAttribute(lb_kernel(v & 1, (v >> 1) & 1, v >> 2, pair_nodes()),
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb),
                     "LB kernel shared memory");
    }
    if (bead_smem() > 48 * 1024)
      cuda_check(cudaFuncSetAttribute(k_bead_step<S, R, DEV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)bead_smem()),
                 "bead kernel shared memory");
    const unsigned long long nb = (nnodes_ + 255) / 256;
    k_init_rest<S, R, DEV><<<(unsigned)nb, 256, 0, s>>>(pop_[0], nnodes_, plane_, (R)cfg_.rho);
    cuda_check(cudaGetLastError(), "init populations");
    cur_ = 0;
    cuda_check(cudaMemsetAsync(status_, 0, sizeof(unsigned), s), "memset status");
    cuda_check(cudaMemsetAsync(nonpos_, 0, sizeof(unsigned long long), s), "memset counter");
    cuda_check(cudaMemsetAsync(acc_, 0, 4 * sizeof(double), s), "memset accumulators");
    if (N_ > 0) {
      const double box = cfg_.L * cfg_.a;
      std::vector<R> xw(3 * N_), xlo(3 * N_), vv(3 * N_);
      std::vector<int> im(3 * N_);
      for (int t = 0; t < 3 * N_; ++t) {
        const double xu = x0[t];
        double k = floor(xu / box);
        double xr = xu - k * box;
        R xs = (R)xr;
        if (xs >= (R)box) {
          xs = (R)0;
          xr -= box;
          k += 1;
        }
        xw[t] = xs;
        xlo[t] = (R)(xr - (double)xs);
        im[t] = (int)k;
        vv[t] = v0 ? (R)v0[t] : (R)0;
      }
      cuda_check(cudaMemcpyAsync(x_, xw.data(), 3 * N_ * sizeof(R), cudaMemcpyHostToDevice, s), "upload x");
      cuda_check(cudaMemcpyAsync(xl_, xlo.data(), 3 * N_ * sizeof(R), cudaMemcpyHostToDevice, s), "upload xl");
      cuda_check(cudaMemcpyAsync(img_, im.data(), 3 * N_ * sizeof(int), cudaMemcpyHostToDevice, s), "upload img");
      cuda_check(cudaMemcpyAsync(v_, vv.data(), 3 * N_ * sizeof(R), cudaMemcpyHostToDevice, s), "upload v");
      cuda_check(cudaMemcpyAsync(xref_, x0, 3 * N_ * sizeof(double), cudaMemcpyHostToDevice, s), "upload xref");
      cuda_check(cudaStreamSynchronize(s), "sync upload");
      const ChainK<R> C = chain();
      k_chain_init_forces<R><<<1, 512, 6 * N_ * sizeof(R), s>>>(C);
      cuda_check(cudaGetLastError(), "init forces");
    }
    for (int j = 0; j < 2; ++j) {
      cuda_check(cudaMemsetAsync(p_count_[j], 0, sizeof(int), s), "memset pending");
      if (corr_[j]) cuda_check(cudaMemsetAsync(corr_[j], 0, (size_t)Q * plane_ * sizeof(R), s), "memset corrections");
    }
    for (int j = 0; j < 2; ++j)
      cuda_check(cudaMemsetAsync(masks_[j], 0, nsegs() * sizeof(unsigned), s), "memset marks");
  }

  // One coupled step, complete on return: the bead kernel, then the LB kernel, released as
  // soon as the bead kernel is resident (both read only buffer A), then the force correction
  // adds the bead reaction to buffer B.  One stream.
  void step(uint32_t k, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1) override {
    flush(s);
    const FluidK<R> P = fluid();
    const S* A = pop_[cur_];
    S* Bo = pop_[cur_ ^ 1];
    const PendK<R> Pd = pend(false);
    if (N_ > 0) {
      launch_bead(A, P, Pd, k, s, ev0 == nullptr);
      snap_valid_ = true;
      snap_k_ = k;
    }
    launch_lb(A, Bo, P, Pd, k, s, ev0, ev1);
    if (N_ > 0) apply(Bo, P, pslot_, s);
    cur_ ^= 1;
  }

  // One coupled step whose force correction stays pending: the next deferred step adds it
  // where it reads the populations (the LB kernel at the nodes this step marks, the bead
  // kernel in its gather), and flush() applies it.  Stream order gives every dependency: the bead
  // kernel of step k starts after the LB and bead kernels of step k-1 have completed, and
  // the LB kernel of step k, released early, touches nothing the bead kernel of step k
  // reads or writes.
  void step_deferred(uint32_t k, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1) override {
    if (N_ == 0) {
      step(k, s, ev0, ev1);
      return;
    }
    const FluidK<R> P = fluid();
    const S* A = pop_[cur_];
    S* Bo = pop_[cur_ ^ 1];
    if (open_) pslot_ ^= 1;
    const PendK<R> Pd = pend(true);
    launch_bead(A, P, Pd, k, s, ev0 == nullptr);
    snap_valid_ = true;
    snap_k_ = k;
    launch_lb(A, Bo, P, Pd, k, s, ev0, ev1);
    open_ = true;
    cur_ ^= 1;
  }

  // One complete step with the bead kernel's state arrays given (the adjoint's recomputation:
  // read a saved state, write the next one); the context's own bead arrays are not touched.
  void step_with_chain(uint32_t k, cudaStream_t s, const ChainK<R>& C, const FluidK<R>& P) {
    flush(s);
    const S* A = pop_[cur_];
    S* Bo = pop_[cur_ ^ 1];
    const PendK<R> Pd = pend(false);
    launch_bead(A, P, Pd, k, s, true, &C);
    launch_lb(A, Bo, P, Pd, k, s, nullptr, nullptr);
    apply(Bo, P, pslot_, s);
    cur_ ^= 1;
  }

  // apply the pending force correction of the last deferred step
  void flush(cudaStream_t s) override {
    if (!open_) return;
    apply(pop_[cur_], fluid(), pslot_, s);
    open_ = false;
  }

  void adjoint_displacement(int64_t T, int K, uint32_t k0, double* O, double* gx, double* gz,
                            cudaStream_t s) override {
    flush(s);
    snap_valid_ = false;
    if (N_ == 0) throw LbError(S_STATE, "adjoint needs a chain");
    if (nsub_ != 1) throw LbError(S_STATE, "adjoint needs one MD step per LB step");
    const FluidK<R> P = fluid();
    if (P.body_on) throw LbError(S_STATE, "adjoint does not support the fluid body force");
    if (T < 1 || K < 1) throw LbError(S_ARG, "T and K must be >= 1");
    const size_t popb = (size_t)Q * plane_ * sizeof(S);
    const size_t n3 = 3 * (size_t)N_;
    // layout() places the six bead arrays x_, xl_, img_, v_, F_, Fc_ one after the other, so
    // a saved state is the population field plus one copy of that span
    unsigned char* const bead0 = reinterpret_cast<unsigned char*>(x_);
    const size_t beadb = (size_t)(reinterpret_cast<unsigned char*>(Fc_ + n3) - bead0);
    {
      const unsigned char* arr[6] = {bead0, reinterpret_cast<unsigned char*>(xl_),
                                     reinterpret_cast<unsigned char*>(img_), reinterpret_cast<unsigned char*>(v_),
                                     reinterpret_cast<unsigned char*>(F_), reinterpret_cast<unsigned char*>(Fc_)};
      for (int i = 1; i < 6; ++i)
        if (arr[i] <= arr[i - 1]) throw LbError(S_STATE, "bead arrays are not laid out in order");
    }
    const int nck = (int)((T + K - 1) / K);
    const size_t stb = align_up(popb + beadb, 256);  // one saved state, 256-byte aligned
    const size_t lamb = (size_t)Q * plane_ * sizeof(R);
    // scratch layout
    size_t off = 0;
    auto take = [&](size_t b) {
      off = align_up(off, 256);
      const size_t o = off;
      off += b;
      return o;
    };
    const size_t o_ck = take((size_t)nck * stb);
    // two pools of the states t0 .. t0 + K of a segment (slot 0 a copy of its checkpoint): the
    // recomputation of one segment fills one pool while the reverse sweep of the segment after
    // it reads the other
    const size_t o_pool = take(2 * (size_t)(K + 1) * stb);
    const size_t o_fin = take(stb);
    const size_t o_lam0 = take(lamb), o_lam1 = take(lamb);
    const size_t o_bar = take(3 * n3 * sizeof(R));
    // bead adjoint scratch with its own corner entries (the recomputation running beside it
    // uses the context's): in the kernel's shared memory when it fits, else here
    AdjK<R> A;
    memset(&A, 0, sizeof(A));
    const size_t adj_scratch = carve_adj_scratch<R>(A, nullptr, N_, cap_);
    const size_t ne = 8 * (size_t)N_;
    size_t M = 1;
    while (M < ne) M <<= 1;
    const size_t smem_base = align_up(align_up(6 * n3 / 3 * sizeof(R) + 32, 16) + M * 8 + ne * 4 + 64, 16);
    const bool scratch_in_smem = smem_base + adj_scratch <= 200 * 1024;
    const size_t o_adj = take(scratch_in_smem ? 16 : adj_scratch);
    const size_t o_z = take(sizeof(double));
    const size_t o_ctr = take(2 * sizeof(uint32_t));  // step counters of the segment graphs
    unsigned char* base = nullptr;
    cuda_check(cudaMalloc(&base, off), "adjoint scratch");
    S* const own_pop[2] = {pop_[0], pop_[1]};
    struct Restore {  // the context's own population buffers, the scratch, the second stream
      EngineT* e;     // and the events, also on an error
      S* p0;
      S* p1;
      unsigned char* p;
      cudaStream_t s2, cs;
      std::vector<cudaEvent_t> ev;
      cudaGraphExec_t g[6];  // recomputation by pool, reverse sweep by pool and lambda parity
      ~Restore() {
        e->pop_[0] = p0;
        e->pop_[1] = p1;
        for (cudaStream_t x : {s2, cs})
          if (x) {
            cudaStreamSynchronize(x);
            cudaStreamDestroy(x);
          }
        for (cudaGraphExec_t x : g)
          if (x) cudaGraphExecDestroy(x);
        for (cudaEvent_t x : ev) cudaEventDestroy(x);
        cudaFree(p);
      }
    } guard{this, own_pop[0], own_pop[1], base, nullptr, nullptr, {}, {}};
    auto new_event = [&]() {
      cudaEvent_t x = nullptr;
      cuda_check(cudaEventCreateWithFlags(&x, cudaEventDisableTiming), "adjoint event");
      guard.ev.push_back(x);
      return x;
    };
    auto save_state = [&](unsigned char* dst) {
      cuda_check(cudaMemcpyAsync(dst, pop_[cur_], popb, cudaMemcpyDeviceToDevice, s), "save pops");
      cuda_check(cudaMemcpyAsync(dst + popb, bead0, beadb, cudaMemcpyDeviceToDevice, s), "save beads");
    };
    auto ck = [&](int i) { return base + o_ck + (size_t)i * stb; };
    auto pool = [&](int pid, int i) { return base + o_pool + ((size_t)pid * (K + 1) + i) * stb; };
    // a state's bead arrays, at their offsets within the saved span
    auto at = [&](unsigned char* st, const void* arr) {
      return st + popb + (size_t)(reinterpret_cast<const unsigned char*>(arr) - bead0);
    };
    // 1. forward pass with checkpoints every K steps (deferred force corrections between
    //    checkpoints, the same arithmetic as complete steps when the storage type is the
    //    arithmetic type; complete steps otherwise)
    std::vector<double> x0h(n3), xTh(n3);
    get_beads(x0h.data(), nullptr, s);
    const bool deferred = sizeof(S) == sizeof(R);
    for (int64_t t = 0; t < T; ++t) {
      if (t % K == 0) {
        flush(s);
        save_state(ck((int)(t / K)));
      }
      if (deferred)
        step_deferred((uint32_t)(k0 + t), s, nullptr, nullptr);
      else
        step((uint32_t)(k0 + t), s, nullptr, nullptr);
    }
    flush(s);
    save_state(base + o_fin);
    get_beads(xTh.data(), nullptr, s);
    double obj = 0.0;
    std::vector<R> xb0(n3);
    for (size_t t = 0; t < n3; ++t) {
      const double d = xTh[t] - x0h[t];
      obj += d * d;
      xb0[t] = (R)(2.0 * d);
    }
    // 2. adjoint state at T
    R* lam[2] = {reinterpret_cast<R*>(base + o_lam0), reinterpret_cast<R*>(base + o_lam1)};
    cuda_check(cudaMemsetAsync(lam[0], 0, lamb, s), "lambda");
    cuda_check(cudaMemsetAsync(lam[1], 0, lamb, s), "lambda");
    R* bars = reinterpret_cast<R*>(base + o_bar);
    A.xbar = bars;
    A.vbar = bars + n3;
    A.fbar = bars + 2 * n3;
    cuda_check(cudaMemsetAsync(bars, 0, 3 * n3 * sizeof(R), s), "bars");
    cuda_check(cudaMemcpyAsync(A.xbar, xb0.data(), n3 * sizeof(R), cudaMemcpyHostToDevice, s), "xbar");
    if (scratch_in_smem) {
      A.smem_scratch = 1;
      A.smem_off = (unsigned)smem_base;
    } else {
      carve_adj_scratch<R>(A, base + o_adj, N_, cap_);
    }
    A.zbar = reinterpret_cast<double*>(base + o_z);
    cuda_check(cudaMemsetAsync(A.zbar, 0, sizeof(double), s), "zbar");
    const ChainK<R> C = chain();
    const size_t smem = scratch_in_smem ? smem_base + adj_scratch : smem_base;
    if (smem > 48 * 1024)
      cuda_check(cudaFuncSetAttribute(k_adj_bead<S, R, DEV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                 "adjoint smem");
    dim3 blk, grd;
    lb_launch_shape(blk, grd, false);  // the adjoint LB kernel: one node per thread
    int cur_lam = 0;
    // 3. reverse sweep over the segments.  The states t0 .. t1 - 1 of a segment sit in the
    //    slots of a pool: slot 0 a copy of its checkpoint, slots 1 .. written by the
    //    recomputation, whose steps read the populations and bead state of slot i and write
    //    those of slot i + 1 (the context's population buffers pointed at the slots).  The
    //    reverse steps read a slot's state in place.  The recomputation of segment k - 1 needs
    //    only its checkpoint, so it runs on a second stream beside the reverse sweep of segment
    //    k, in the other pool.  A full segment's recomputation or reverse sweep is the same
    //    sequence of launches at other step numbers: each is captured once as a CUDA graph whose
    //    kernels add their step argument to a device counter, and replayed.
    uint32_t* d_ctr = reinterpret_cast<uint32_t*>(base + o_ctr);
    FluidK<R> Prec = P, Prev = P;
    Prec.d_step = d_ctr;
    Prev.d_step = d_ctr + 1;
    auto recompute_ops = [&](int64_t t0, int64_t t1, int pid, cudaStream_t st, const FluidK<R>& Pk, bool rel) {
      for (int64_t t = t0; t < t1; ++t) {
        const int i = (int)(t - t0);
        unsigned char* a = pool(pid, i);
        unsigned char* b = pool(pid, i + 1);
        pop_[cur_] = reinterpret_cast<S*>(a);
        pop_[cur_ ^ 1] = reinterpret_cast<S*>(b);
        ChainK<R> Cs = C;  // read the bead state of slot i, write the next state into slot i + 1
        Cs.x_in = reinterpret_cast<const R*>(at(a, x_));
        Cs.xl_in = reinterpret_cast<const R*>(at(a, xl_));
        Cs.img_in = reinterpret_cast<const int*>(at(a, img_));
        Cs.v_in = reinterpret_cast<const R*>(at(a, v_));
        Cs.F_in = reinterpret_cast<const R*>(at(a, F_));
        Cs.x = reinterpret_cast<R*>(at(b, x_));
        Cs.xl = reinterpret_cast<R*>(at(b, xl_));
        Cs.img = reinterpret_cast<int*>(at(b, img_));
        Cs.v = reinterpret_cast<R*>(at(b, v_));
        Cs.F = reinterpret_cast<R*>(at(b, F_));
        Cs.Fc = reinterpret_cast<R*>(at(b, Fc_));
        Cs.snap = nullptr;
        step_with_chain(rel ? (uint32_t)(t - t0) : (uint32_t)(k0 + t), st, Cs, Pk);
      }
    };
    auto reverse_ops = [&](int64_t t0, int64_t t1, int pid, cudaStream_t st, const FluidK<R>& Pk, bool rel) {
      for (int64_t t = t1 - 1; t >= t0; --t) {
        unsigned char* stt = pool(pid, (int)(t - t0));
        const S* pops = reinterpret_cast<const S*>(stt);
        ChainK<R> Ct = C;
        Ct.x = reinterpret_cast<R*>(at(stt, x_));
        Ct.xl = reinterpret_cast<R*>(at(stt, xl_));
        Ct.img = reinterpret_cast<int*>(at(stt, img_));
        Ct.v = reinterpret_cast<R*>(at(stt, v_));
        Ct.F = reinterpret_cast<R*>(at(stt, F_));
        Ct.Fc = reinterpret_cast<R*>(at(stt, Fc_));
        const uint32_t kt = rel ? (uint32_t)(t - t0) : (uint32_t)(k0 + t);
        // the adjoint LB kernel (all nodes) and, beside it, the bead adjoint (one block), which
        // adds its forced-node terms to lambda once the LB kernel has written it
        cudaLaunchAttribute at1[1];
        at1[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at1[0].val.programmaticStreamSerializationAllowed = 1;
        cudaLaunchConfig_t la;
        memset(&la, 0, sizeof(la));
        la.gridDim = grd;
        la.blockDim = blk;
        la.stream = st;
        la.attrs = at1;
        la.numAttrs = 1;
        const R* lin = lam[cur_lam];
        R* lout = lam[cur_lam ^ 1];
        if (Pk.ncalls > 0)
          cuda_check(cudaLaunchKernelEx(&la, k_adj_lb<S, R, DEV, true>, pops, lin, lout, Pk, kt), "adjoint LB");
        else
          cuda_check(cudaLaunchKernelEx(&la, k_adj_lb<S, R, DEV, false>, pops, lin, lout, Pk, kt), "adjoint LB");
        cudaLaunchConfig_t lbd = la;
        lbd.gridDim = dim3(1);
        lbd.blockDim = dim3(512);
        lbd.dynamicSmemBytes = smem;
        cuda_check(cudaLaunchKernelEx(&lbd, k_adj_bead<S, R, DEV>, pops, lin, lout, Pk, Ct, A, kt), "adjoint bead");
        cur_lam ^= 1;
      }
    };
    // Run a segment's launches on stream st: directly for a partial segment, else as the graph
    // g (captured on the first use; ctr is the graph's step counter, set to the segment's first
    // step).  ops(stream, relative) enqueues the launches; book() does on the host what they do
    // to its state, for a replay.
    auto run_segment = [&](int64_t t0, int64_t t1, cudaStream_t st, cudaGraphExec_t& g, uint32_t* ctr, auto&& ops,
                           auto&& book) {
      if (t1 - t0 < K) {
        ops(st, false);
        return;
      }
      k_store_value<uint32_t><<<1, 1, 0, st>>>(ctr, (uint32_t)(k0 + t0));
      cuda_check(cudaGetLastError(), "step counter");
      if (!g) {
        if (!guard.cs) cuda_check(cudaStreamCreateWithFlags(&guard.cs, cudaStreamNonBlocking), "capture stream");
        cudaGraph_t gr = nullptr;
        cuda_check(cudaStreamBeginCapture(guard.cs, cudaStreamCaptureModeThreadLocal), "begin capture");
        ops(guard.cs, true);
        cuda_check(cudaStreamEndCapture(guard.cs, &gr), "end capture");
        const cudaError_t ie = cudaGraphInstantiate(&g, gr, 0);
        cudaGraphDestroy(gr);
        cuda_check(ie, "instantiate segment graph");
      } else {
        book();
      }
      cuda_check(cudaGraphLaunch(g, st), "segment graph");
    };
    auto recompute = [&](int sgi, int pid) {
      const int64_t t0 = (int64_t)sgi * K, t1 = t0 + K < T ? t0 + K : T;
      cuda_check(cudaMemcpyAsync(pool(pid, 0), ck(sgi), stb, cudaMemcpyDeviceToDevice, guard.s2), "checkpoint");
      run_segment(
          t0, t1, guard.s2, guard.g[pid], d_ctr,
          [&](cudaStream_t st, bool rel) { recompute_ops(t0, t1, pid, st, rel ? Prec : P, rel); }, [] {});
    };
    auto reverse = [&](int sgi, int pid) {
      const int64_t t0 = (int64_t)sgi * K, t1 = t0 + K < T ? t0 + K : T;
      run_segment(
          t0, t1, s, guard.g[2 + 2 * pid + cur_lam], d_ctr + 1,
          [&](cudaStream_t st, bool rel) { reverse_ops(t0, t1, pid, st, rel ? Prev : P, rel); },
          [&] { cur_lam ^= (int)((t1 - t0) & 1); });  // the captured sequence's effect on the parity
    };
    cuda_check(cudaStreamCreateWithFlags(&guard.s2, cudaStreamNonBlocking), "adjoint stream");
    {
      cudaEvent_t fwd = new_event();  // the forward pass and its checkpoints are complete
      cuda_check(cudaEventRecord(fwd, s), "event");
      cuda_check(cudaStreamWaitEvent(guard.s2, fwd, 0), "wait");
    }
    std::vector<cudaEvent_t> rec_done(nck), rev_done(nck);
    recompute(nck - 1, 0);
    rec_done[nck - 1] = new_event();
    cuda_check(cudaEventRecord(rec_done[nck - 1], guard.s2), "event");
    for (int sgi = nck - 1; sgi >= 0; --sgi) {
      const int pid = (nck - 1 - sgi) & 1;
      if (sgi >= 1) {  // the next segment's recomputation, into the pool the last reverse sweep read
        if (sgi + 1 <= nck - 1) cuda_check(cudaStreamWaitEvent(guard.s2, rev_done[sgi + 1], 0), "wait");
        recompute(sgi - 1, pid ^ 1);
        rec_done[sgi - 1] = new_event();
        cuda_check(cudaEventRecord(rec_done[sgi - 1], guard.s2), "event");
      }
      cuda_check(cudaStreamWaitEvent(s, rec_done[sgi], 0), "wait");
      reverse(sgi, pid);
      rev_done[sgi] = new_event();
      cuda_check(cudaEventRecord(rev_done[sgi], s), "event");
    }
    pop_[0] = own_pop[0];
    pop_[1] = own_pop[1];
    auto load_state = [&](const unsigned char* src) {
      cuda_check(cudaMemcpyAsync(pop_[cur_], src, popb, cudaMemcpyDeviceToDevice, s), "load pops");
      cuda_check(cudaMemcpyAsync(bead0, src + popb, beadb, cudaMemcpyDeviceToDevice, s), "load beads");
    };
    // 4. the initial force F_0 = F_cons(x_0): xbar += H(x_0) fbar
    {
      ChainK<R> C0 = C;
      C0.x = reinterpret_cast<R*>(at(ck(0), x_));
      C0.xl = reinterpret_cast<R*>(at(ck(0), xl_));
      C0.img = reinterpret_cast<int*>(at(ck(0), img_));
      k_chain_force_vjp<R><<<1, 512, 6 * n3 / 3 * sizeof(R), s>>>(C0, A.fbar, A.xbar);
    }
    cuda_check(cudaGetLastError(), "initial force adjoint");
    std::vector<R> xbh(n3);
    double zb = 0.0;
    cuda_check(cudaMemcpyAsync(xbh.data(), A.xbar, n3 * sizeof(R), cudaMemcpyDeviceToHost, s), "dl xbar");
    cuda_check(cudaMemcpyAsync(&zb, A.zbar, sizeof(double), cudaMemcpyDeviceToHost, s), "dl zbar");
    // 5. leave the context at the end of the forward run
    load_state(base + o_fin);
    cuda_check(cudaStreamSynchronize(s), "adjoint sync");
    *O = obj;
    for (size_t t = 0; t < n3; ++t) gx[t] = (double)xbh[t] - 2.0 * (xTh[t] - x0h[t]);
    *gz = zb;
  }

  // --- access for the batched driver (one engine per replica, stepped in lockstep) ---
  FluidK<R> fluid_params() const { return fluid(); }
  ChainK<R> chain_params() const { return chain(); }
  S* buffer(int i) const { return pop_[i]; }
  int parity() const { return cur_; }
  void flip() { cur_ ^= 1; }
  unsigned long long nodes() const { return nnodes_; }
  int pending_capacity() const { return cap_; }
  // pending-correction lists of slot j (the batched driver keeps its own slot order)
  int4* pending_pos(int j) const { return p_pos_[j]; }
  R* pending_dn(int j) const { return p_dn_[j]; }
  int* pending_count(int j) const { return p_count_[j]; }
  R* pending_dense(int j) const { return corr_[j]; }
  unsigned long long plane() const { return plane_; }
  size_t bead_smem_bytes() const { return bead_smem(); }
  int chain_length() const { return N_; }
  const Config& config() const { return cfg_; }

  // The full FP64 populations to or from the caller's host array.  Page-locked host memory that
  // the device addresses directly (pinned or registered, the whole array inside one
  // allocation) is written or read by one conversion kernel over all 19 planes, with no
  // staging copy; other host memory goes through the second population buffer in chunks of
  // as many FP64 planes as it holds, one conversion kernel and one copy per chunk.
  void get_populations(double* out, cudaStream_t s) override {
    flush(s);
    double* direct = static_cast<double*>(device_view(out, (size_t)Q * nnodes_ * sizeof(double)));
    if (direct) {
      k_planes_to_f64<S, R, DEV><<<conv_grid(Q), 256, 0, s>>>(direct, pop_[cur_], nnodes_, plane_, 0, cfg_.rho);
      cuda_check(cudaGetLastError(), "planes to f64");
    } else {
      double* stage = reinterpret_cast<double*>(pop_[cur_ ^ 1]);
      const int chunk = stage_planes();
      for (int p0 = 0; p0 < Q; p0 += chunk) {
        const int np = p0 + chunk <= Q ? chunk : Q - p0;
        k_planes_to_f64<S, R, DEV><<<conv_grid(np), 256, 0, s>>>(stage, pop_[cur_], nnodes_, plane_, p0, cfg_.rho);
        cuda_check(cudaGetLastError(), "planes to f64");
        cuda_check(cudaMemcpyAsync(out + (size_t)p0 * nnodes_, stage, (size_t)np * nnodes_ * sizeof(double),
                                   cudaMemcpyDeviceToHost, s),
                   "download planes");
      }
    }
    cuda_check(cudaStreamSynchronize(s), "sync download");
  }

  void set_populations(const double* in, cudaStream_t s) override {
    flush(s);
    const double* direct =
        static_cast<const double*>(device_view(in, (size_t)Q * nnodes_ * sizeof(double)));
    if (direct) {
      k_planes_from_f64<S, R, DEV><<<conv_grid(Q), 256, 0, s>>>(pop_[cur_], direct, nnodes_, plane_, 0, cfg_.rho);
      cuda_check(cudaGetLastError(), "planes from f64");
    } else {
      double* stage = reinterpret_cast<double*>(pop_[cur_ ^ 1]);
      const int chunk = stage_planes();
      for (int p0 = 0; p0 < Q; p0 += chunk) {
        const int np = p0 + chunk <= Q ? chunk : Q - p0;
        cuda_check(cudaMemcpyAsync(stage, in + (size_t)p0 * nnodes_, (size_t)np * nnodes_ * sizeof(double),
                                   cudaMemcpyHostToDevice, s),
                   "upload planes");
        k_planes_from_f64<S, R, DEV><<<conv_grid(np), 256, 0, s>>>(pop_[cur_], stage, nnodes_, plane_, p0, cfg_.rho);
        cuda_check(cudaGetLastError(), "planes from f64");
      }
    }
    cuda_check(cudaStreamSynchronize(s), "sync upload");
  }

  // bead arrays are final once the bead kernel of the last step has run (pending fluid
  // corrections do not touch them): no flush.  One kernel forms the FP64 unwrapped positions
  // and velocities in a device staging area, then one copy per output array.
  void get_beads(double* x, double* v, cudaStream_t s) override {
    if (N_ == 0) return;
    enqueue_beads(x, v, s);
    cuda_check(cudaStreamSynchronize(s), "sync beads");
  }

  void enqueue_beads(double* x, double* v, cudaStream_t s) override {
    if (N_ == 0) return;
    const int n3 = 3 * N_;
    k_bead_readback<R><<<(n3 + 255) / 256, 256, 0, s>>>(x_, xl_, img_, v_, n3, cfg_.L * cfg_.a, rb_);
    cuda_check(cudaGetLastError(), "bead read-back");
    if (x) cuda_check(cudaMemcpyAsync(x, rb_, n3 * sizeof(double), cudaMemcpyDeviceToHost, s), "dl x");
    if (v) cuda_check(cudaMemcpyAsync(v, rb_ + n3, n3 * sizeof(double), cudaMemcpyDeviceToHost, s), "dl v");
  }

  void enqueue_status(unsigned* host, cudaStream_t s) override {
    cuda_check(cudaMemcpyAsync(host, status_, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "status");
  }

  // Asynchronous read-back.  While the last step's snapshot holds the bead state, the copies
  // run on the engine's own stream after an event on s, so that s goes on with the next steps
  // (the bead kernel that next rewrites the slot waits for them); otherwise the read-back
  // kernel and the copies are queued on s itself.  Either way `done` is recorded on the
  // engine's stream, so read-backs complete in the order they were asked for.
  void enqueue_beads_async(double* x, double* v, unsigned* status_host, cudaEvent_t done,
                           cudaStream_t s) override {
    if (!side_) {
      cuda_check(cudaStreamCreateWithFlags(&side_, cudaStreamNonBlocking), "read-back stream");
      cuda_check(cudaEventCreateWithFlags(&step_ev_, cudaEventDisableTiming), "event");
      for (int j = 0; j < 2; ++j) cuda_check(cudaEventCreateWithFlags(&copy_ev_[j], cudaEventDisableTiming), "event");
    }
    if (N_ == 0 || !snap_valid_) {
      enqueue_beads(x, v, s);
      enqueue_status(status_host, s);
      cuda_check(cudaEventRecord(step_ev_, s), "record read-back");
      cuda_check(cudaStreamWaitEvent(side_, step_ev_, 0), "wait read-back");
      cuda_check(cudaEventRecord(done, side_), "record read-back");
      return;
    }
    const int p = (int)(snap_k_ & 1u);
    const size_t n3 = 3 * (size_t)N_;
    const double* sn = snap_ + (size_t)p * 2 * n3;
    cuda_check(cudaEventRecord(step_ev_, s), "record step");
    cuda_check(cudaStreamWaitEvent(side_, step_ev_, 0), "wait step");
    if (x) cuda_check(cudaMemcpyAsync(x, sn, n3 * sizeof(double), cudaMemcpyDeviceToHost, side_), "dl x");
    if (v) cuda_check(cudaMemcpyAsync(v, sn + n3, n3 * sizeof(double), cudaMemcpyDeviceToHost, side_), "dl v");
    enqueue_status(status_host, side_);
    cuda_check(cudaEventRecord(copy_ev_[p], side_), "record copy");
    snap_pending_[p] = true;
    cuda_check(cudaEventRecord(done, side_), "record read-back");
  }

  void drain() override {
    if (side_) cuda_check(cudaStreamSynchronize(side_), "drain read-backs");
  }

  ~EngineT() override {
    if (side_) {
      cudaStreamSynchronize(side_);
      cudaStreamDestroy(side_);
      cudaEventDestroy(step_ev_);
      cudaEventDestroy(copy_ev_[0]);
      cudaEventDestroy(copy_ev_[1]);
    }
  }

  void observables(double* out, int64_t step, int accumulate, cudaStream_t s) override {
    flush(s);
    ObsK<R> O = obs(step, accumulate);
    if (!accumulate) {
      k_fluid_partials<S, R, DEV><<<nparts_, 256, 0, s>>>(pop_[cur_], nnodes_, plane_, parts_);
      cuda_check(cudaGetLastError(), "fluid partials");
      O.nparts = nparts_;
    }
    k_observables<R><<<1, 256, 0, s>>>(O);
    cuda_check(cudaGetLastError(), "observables");
    if (out) {
      cuda_check(cudaMemcpyAsync(out, obs_, kNObs * sizeof(double), cudaMemcpyDeviceToHost, s), "dl obs");
      cuda_check(cudaStreamSynchronize(s), "sync obs");
    }
  }

  void reset_reference(cudaStream_t s) override {
    if (N_ == 0) return;
    std::vector<double> xu(3 * N_);
    get_beads(xu.data(), nullptr, s);
    cuda_check(cudaMemcpyAsync(xref_, xu.data(), 3 * N_ * sizeof(double), cudaMemcpyHostToDevice, s), "xref");
    cuda_check(cudaMemsetAsync(acc_, 0, 4 * sizeof(double), s), "acc");
    cuda_check(cudaStreamSynchronize(s), "sync ref");
  }

  // bead arrays are final once the bead kernel of the last step has run (pending fluid
  // corrections do not touch them), so no flush
  void record_frame(double* dst, cudaStream_t s) override {
    if (N_ == 0) return;
    const int n3 = 3 * N_;
    k_record_frame<R><<<(n3 + 255) / 256, 256, 0, s>>>(x_, xl_, img_, n3, cfg_.L * cfg_.a, dst);
    cuda_check(cudaGetLastError(), "record frame");
  }

  void debug_coupling_cells(int* nodes, double* x_stored, cudaStream_t s) override {
    if (N_ == 0) throw LbError(S_STATE, "no chain");
    if (nodes) cuda_check(cudaMemcpyAsync(nodes, e_node_, (size_t)cap_ * sizeof(int), cudaMemcpyDeviceToHost, s),
                          "corner nodes");
    std::vector<R> xs(3 * (size_t)N_);
    cuda_check(cudaMemcpyAsync(xs.data(), x_, xs.size() * sizeof(R), cudaMemcpyDeviceToHost, s), "stored x");
    cuda_check(cudaStreamSynchronize(s), "sync debug");
    if (x_stored)
      for (size_t t = 0; t < xs.size(); ++t) x_stored[t] = (double)xs[t];
  }

  unsigned read_status(cudaStream_t s) override {
    unsigned st = 0;
    cuda_check(cudaMemcpyAsync(&st, status_, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "status");
    cuda_check(cudaStreamSynchronize(s), "sync status");
    return st;
  }

  // checkpoint: populations (storage type, L^3 per plane), bead arrays, xref, acc, counter
  size_t state_bytes() const override {
    return 19 * nnodes_ * sizeof(S) + (size_t)N_ * 3 * (5 * sizeof(R) + sizeof(int) + sizeof(double)) +
           4 * sizeof(double) + sizeof(unsigned long long);
  }
  void save_state(void* host, cudaStream_t s) override {
    flush(s);
    unsigned char* p = static_cast<unsigned char*>(host);
    for (int i = 0; i < Q; ++i) {
      cuda_check(cudaMemcpyAsync(p, pop_[cur_] + (size_t)i * plane_, nnodes_ * sizeof(S), cudaMemcpyDeviceToHost, s),
                 "save pop");
      p += nnodes_ * sizeof(S);
    }
    p = copy_beads(p, true, s);
    cuda_check(cudaStreamSynchronize(s), "sync save");
  }
  void load_state(const void* host, cudaStream_t s) override {
    flush(s);
    snap_valid_ = false;
    unsigned char* p = const_cast<unsigned char*>(static_cast<const unsigned char*>(host));
    for (int i = 0; i < Q; ++i) {
      cuda_check(cudaMemcpyAsync(pop_[cur_] + (size_t)i * plane_, p, nnodes_ * sizeof(S), cudaMemcpyHostToDevice, s),
                 "load pop");
      p += nnodes_ * sizeof(S);
    }
    p = copy_beads(p, false, s);
    cuda_check(cudaStreamSynchronize(s), "sync load");
  }

 private:
  unsigned char* copy_beads(unsigned char* p, bool save, cudaStream_t s) {
    auto mv = [&](void* dev, size_t bytes) {
      if (bytes == 0) return;
      if (save)
        cuda_check(cudaMemcpyAsync(p, dev, bytes, cudaMemcpyDeviceToHost, s), "save state");
      else
        cuda_check(cudaMemcpyAsync(dev, p, bytes, cudaMemcpyHostToDevice, s), "load state");
      p += bytes;
    };
    const size_t n3 = 3 * (size_t)N_;
    mv(x_, n3 * sizeof(R));
    mv(xl_, n3 * sizeof(R));
    mv(img_, n3 * sizeof(int));
    mv(v_, n3 * sizeof(R));
    mv(F_, n3 * sizeof(R));
    mv(Fc_, n3 * sizeof(R));
    mv(xref_, n3 * sizeof(double));
    mv(acc_, 4 * sizeof(double));
    mv(nonpos_, sizeof(unsigned long long));
    return p;
  }

  // Bead kernel of step k: one cluster of bead_cluster() blocks; with `chained`, launched with
  // programmatic stream serialization (it waits for the previous grid before reading, so only
  // its launch overlaps).
  void launch_bead(const S* A, const FluidK<R>& P, const PendK<R>& Pd, uint32_t k, cudaStream_t s, bool chained,
                   const ChainK<R>* Cover = nullptr) {
    if (snap_pending_[k & 1u]) {  // this kernel rewrites the snapshot slot being read back
      cuda_check(cudaStreamWaitEvent(s, copy_ev_[k & 1u], 0), "wait read-back");
      snap_pending_[k & 1u] = false;
    }
    const int G = bead_cluster();
    cudaLaunchConfig_t lc;
    memset(&lc, 0, sizeof(lc));
    lc.gridDim = dim3((unsigned)G);
    lc.blockDim = dim3(512);
    lc.dynamicSmemBytes = bead_smem();
    lc.stream = s;
    cudaLaunchAttribute at[2];
    int na = 0;
    at[na].id = cudaLaunchAttributeClusterDimension;
    at[na].val.clusterDim.x = (unsigned)G;
    at[na].val.clusterDim.y = 1;
    at[na].val.clusterDim.z = 1;
    ++na;
    if (chained) {
      at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      at[na].val.programmaticStreamSerializationAllowed = 1;
      ++na;
    }
    lc.attrs = at;
    lc.numAttrs = (unsigned)na;
    cuda_check(cudaLaunchKernelEx(&lc, k_bead_step<S, R, DEV>, A, P, Cover ? *Cover : chain(), Pd, k), "bead kernel");
    cuda_check(cudaGetLastError(), "bead kernel");
  }

  // LB kernel, launched with programmatic stream serialization.  After the bead kernel of the
  // same step it may start once the bead kernel has signalled (at its start; the LB kernel
  // reads nothing the bead kernel writes) and waits for it before completing.  Without a
  // chain it follows the previous LB kernel and waits for that grid before reading.  Timing
  // events, when given, bracket it, and then every launch is an ordinary one.
  void launch_lb(const S* A, S* Bo, const FluidK<R>& P0, const PendK<R>& Pd, uint32_t k, cudaStream_t s,
                 cudaEvent_t ev0, cudaEvent_t ev1) {
    FluidK<R> P = P0;
    const bool chained = ev0 == nullptr;
    P.pdl = chained ? (N_ > 0 ? 2 : 1) : 0;
    P.angle_tab = sizeof(R) == 8 ? 1 : 0;
    dim3 blk, grd;
    lb_launch_shape(blk, grd, pair_nodes());
    cudaLaunchConfig_t lc;
    memset(&lc, 0, sizeof(lc));
    if (P.pdl & 2) grd.z += 1;  // the plane of waiting blocks
    lc.gridDim = grd;
    lc.blockDim = blk;
    lc.dynamicSmemBytes = Pd.have_prev ? lb_stage_bytes(blk) : 0;  // staged corrections
    lc.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = at;
    lc.numAttrs = chained ? 1 : 0;
    if (ev0) cudaEventRecord(ev0, s);
    cuda_check(cudaLaunchKernelEx(&lc, lb_kernel(P.ncalls > 0, narrow_offsets(), N_ > 0, pair_nodes()), A, Bo, P, Pd, k),
               "LB kernel");
    if (ev1) cudaEventRecord(ev1, s);
    cuda_check(cudaGetLastError(), "LB kernel");
  }

  void apply(S* buf, const FluidK<R>& P, int slot, cudaStream_t s) {
    k_apply_pending<S, R><<<dim3((cap_ + 255) / 256, Q), 256, 0, s>>>(buf, P, p_pos_[slot], p_dn_[slot],
                                                                     p_count_[slot], cap_, corr_[slot],
                                                                     masks_[slot], 0u);
    cuda_check(cudaGetLastError(), "apply kernel");
  }

  // pending-correction block: deferred steps read slot pslot_^1 (when open) and write
  // pslot_ with node marks; complete steps write slot pslot_ only, without marks
  PendK<R> pend(bool deferred) const {
    PendK<R> Pd;
    memset(&Pd, 0, sizeof(Pd));
    const int c = pslot_, p = pslot_ ^ 1;
    Pd.have_prev = (deferred && open_) ? 1 : 0;
    Pd.prev_mask = masks_[p];
    Pd.prev_dense = corr_[p];
    Pd.cur_dense = corr_[c];
    Pd.plane = plane_;
    Pd.cur_pos = p_pos_[c];
    Pd.cur_dn = p_dn_[c];
    Pd.cur_count = p_count_[c];
    Pd.cur_mask = masks_[c];
    Pd.mark = deferred ? 1 : 0;
    Pd.cap = cap_;
    Pd.seg0 = 0;
    return Pd;
  }

  size_t nsegs() const { return (size_t)((nnodes_ + 31) >> kSegShift); }

  // FP64 planes the second population buffer holds as a staging area (at least one: a plane
  // of L^3 doubles fits in 19 planes of any storage type)
  int stage_planes() const {
    const size_t fit = (size_t)Q * plane_ * sizeof(S) / ((size_t)nnodes_ * sizeof(double));
    return fit < 1 ? 1 : (fit > (size_t)Q ? Q : (int)fit);
  }
  // conversion grid: np planes, blocks of 256 threads striding over a plane
  dim3 conv_grid(int np) const {
    unsigned long long bx = (nnodes_ + 255) / 256;
    if (bx > 1024) bx = 1024;
    return dim3((unsigned)bx, (unsigned)np);
  }
  // the device's address of a host range [p, p + bytes) in one page-locked allocation it can
  // address, or null (pageable memory, or a range not inside one such allocation)
  static void* device_view(const void* p, size_t bytes) {
    cudaPointerAttributes a0, a1;
    const unsigned char* last = static_cast<const unsigned char*>(p) + bytes - 1;
    if (cudaPointerGetAttributes(&a0, p) != cudaSuccess || cudaPointerGetAttributes(&a1, last) != cudaSuccess) {
      cudaGetLastError();  // an unregistered pointer is not an error of the caller's stream
      return nullptr;
    }
    if (a0.type != cudaMemoryTypeHost || a1.type != cudaMemoryTypeHost || !a0.devicePointer || !a1.devicePointer)
      return nullptr;
    if (static_cast<unsigned char*>(a1.devicePointer) != static_cast<unsigned char*>(a0.devicePointer) + (bytes - 1))
      return nullptr;
    return a0.devicePointer;
  }

  // the LB kernel for noise on/off, 32-bit (all 19 planes below 2^32 elements) or 64-bit
  // element offsets, with or without the deferred force corrections (a chain), and with two
  // nodes per thread along x (even L) or one
  using LbKernel = void (*)(const S*, S*, const FluidK<R>, const PendK<R>, const uint32_t);
  template <bool NOISE, class I, bool CORR>
  static LbKernel lb_kernel_p(bool pair) {
    return pair ? k_lb_step<S, R, DEV, NOISE, I, CORR, true> : k_lb_step<S, R, DEV, NOISE, I, CORR, false>;
  }
  static LbKernel lb_kernel(bool noise, bool narrow, bool corr, bool pair) {
    using U = unsigned;
    using W = unsigned long long;
    if (corr) {
      if (noise) return narrow ? lb_kernel_p<true, U, true>(pair) : lb_kernel_p<true, W, true>(pair);
      return narrow ? lb_kernel_p<false, U, true>(pair) : lb_kernel_p<false, W, true>(pair);
    }
    if (noise) return narrow ? lb_kernel_p<true, U, false>(pair) : lb_kernel_p<true, W, false>(pair);
    return narrow ? lb_kernel_p<false, U, false>(pair) : lb_kernel_p<false, W, false>(pair);
  }
  bool narrow_offsets() const { return (unsigned long long)Q * plane_ <= 0xFFFFFFFFull; }
  // two nodes per thread along x: every row starts at an even element offset (even L); in
  // single-precision arithmetic only (the FP64 kernel is bound by FP64 arithmetic, which two
  // nodes per thread do not reduce)
  bool pair_nodes() const { return (L_ & 1) == 0 && sizeof(R) == 4; }

  // threads along x cover a row of L nodes (L/2 threads with two nodes each), up to 256 per
  // block; the rest of the 256 threads take further rows
  void lb_launch_shape(dim3& blk, dim3& grd, bool pair) const {
    const unsigned row = pair ? (unsigned)L_ / 2 : (unsigned)L_;
    unsigned bx = (row + 31) / 32 * 32;
    if (bx > 256) bx = 256;
    const unsigned by = 256 / bx;
    blk = dim3(bx, by, 1);
    grd = dim3((row + bx - 1) / bx, ((unsigned)L_ + by - 1) / by, (unsigned)L_);
  }
  // staged corrections of marked nodes: 19 values per thread of a tile
  size_t lb_stage_bytes(const dim3& blk) const { return (size_t)Q * blk.x * blk.y * sizeof(R); }

  size_t bead_smem() const {
    // phase 5: up to kGroupHashMax entries a node table (4 x H ints, H >= 2 x entries), entry
    // slots and lists and scan scratch; beyond, sort keys, leader slots and chunk counts
    const size_t ne = 8 * (size_t)N_ * nsub_;
    size_t groupb;
    if (ne <= (size_t)kGroupHashMax) {
      size_t H = 64;
      while (H < 2 * ne) H <<= 1;
      groupb = (4 * H + 2 * ne + 65) * sizeof(int);
    } else {
      size_t M = 32;
      while (M < ne) M <<= 1;
      groupb = M * 8 + ne * 4 + ((ne + 31) / 32) * 4;
    }
    // positions (hi, lo); in a cluster also half-step velocities and image counters
    const size_t posb = bead_cluster() > 1 ? 9 * (size_t)N_ * sizeof(R) + 3 * (size_t)N_ * sizeof(int)
                                           : 6 * (size_t)N_ * sizeof(R);
    return groupb > posb ? groupb : posb;
  }

  // Blocks of the bead kernel's cluster: one per 16 beads, at most 8 (the portable cluster
  // size); one block when the entries need the sorted grouping
  int bead_cluster() const {
    if (8 * (size_t)N_ * nsub_ > (size_t)kGroupHashMax) return 1;
    const int g = N_ / 16;
    return g < 1 ? 1 : (g > 8 ? 8 : g);
  }

  FluidK<R> fluid() const {
    FluidK<R> P;
    memset(&P, 0, sizeof(P));
    const Config& c = cfg_;
    P.L = (unsigned)L_;
    P.plane = plane_;
    P.rho0 = (R)c.rho;
    const double nu = c.eta * c.h / (c.rho * c.a * c.a);
    const double nub = c.eta_b * c.h / (c.rho * c.a * c.a);
    const double gs = 1.0 - 2.0 / (6.0 * nu + 1.0);
    const double gb = 1.0 - 2.0 / (9.0 * nub + 1.0);
    P.gs = (R)gs;
    P.gb = (R)gb;
    const bool noise = c.noise_fluid && c.kT > 0.0;
    P.ncalls = noise ? (c.stress_only ? 1 : 2) : 0;
    const double mu = 3.0 * c.kT * c.h * c.h / pow(c.a, 5);
    for (int k = 0; k < Q; ++k) {
      double g = 0.0;
      if (k == 4) g = gb;
      if (k >= 5 && k <= 9) g = gs;
      const double bk = norm36(k) / 36.0;
      const bool on = noise && k >= 4 && (k <= 9 || !c.stress_only);
      const double cn = on ? sqrt(mu * bk * (1.0 - g * g)) : 0.0;
      P.cnoise[k] = (R)cn;
      P.am[k] = (R)(g / bk);
      P.ae[k] = (R)((1.0 - g) / bk);
      P.ag[k] = (R)(cn / bk);
      P.wam[k] = (R)(g / bk / 36.0);
      P.wae[k] = (R)((1.0 - g) / bk / 36.0);
      P.wag[k] = (R)(cn / bk / 36.0);
    }
    P.k0 = (uint32_t)(c.seed & 0xffffffffu);
    P.k1 = (uint32_t)(0u | ((uint32_t)c.replica << 8));
    P.rk = make_round_keys(P.k0, P.k1);
    double body[3] = {0, 0, 0};
    if (c.counter_force && c.N > 0) {
      const double vol = pow(c.L * c.a, 3);
      for (int q = 0; q < 3; ++q) body[q] = -c.N * c.ext[q] / vol;
    }
    P.body_on = (body[0] != 0 || body[1] != 0 || body[2] != 0) ? 1 : 0;
    for (int q = 0; q < 3; ++q) P.body_dJ[q] = (R)(body[q] * c.h * c.h / c.a);
    P.nonpos = nonpos_;
    return P;
  }

  ChainK<R> chain() const {
    ChainK<R> C;
    memset(&C, 0, sizeof(C));
    const Config& c = cfg_;
    C.N = N_;
    C.m = (R)c.m;
    C.zeta = (R)c.zeta;
    C.kfene = (R)c.kfene;
    C.R0sq = (R)(c.R0 * c.R0);
    C.eps = (R)c.eps;
    C.sig2 = (R)(c.sigma * c.sigma);
    C.rc2 = (R)(pow(2.0, 1.0 / 3.0) * c.sigma * c.sigma);
    C.h = (R)(c.h / nsub_);  // the MD step
    C.a = (R)c.a;
    C.box = (R)(c.L * c.a);
    C.half_box = (R)(0.5 * c.L * c.a);
    const bool noise = c.noise_beads && c.kT > 0.0;
    C.amp = noise ? (R)sqrt(2.0 * c.kT * c.zeta / (c.h / nsub_)) : (R)0;
    C.k0 = (uint32_t)(c.seed & 0xffffffffu);
    C.k1 = (uint32_t)(1u | ((uint32_t)c.replica << 8));
    for (int q = 0; q < 3; ++q) C.ext[q] = (R)c.ext[q];
    C.u_scale = (R)(c.a / c.h);
    C.inv_a3 = (R)(1.0 / (c.a * c.a * c.a));
    C.dJ_scale = (R)(c.h * c.h / c.a);
    C.nsub = nsub_;
    C.spread = (R)(1.0 / nsub_);
    C.fc_hist = fch_;
    C.x = x_;
    C.xl = xl_;
    C.img = img_;
    C.v = v_;
    C.F = F_;
    C.Fc = Fc_;
    C.x_in = x_;
    C.xl_in = xl_;
    C.img_in = img_;
    C.v_in = v_;
    C.F_in = F_;
    C.vh = vh_;
    C.fcons = fcons_;
    C.e_node = e_node_;
    C.e_w = e_w_;
    C.e_mom = e_mom_;
    C.p_pos = p_pos_[0];
    C.p_dn = p_dn_[0];
    C.p_count = p_count_[0];
    C.cap = cap_;
    C.status = status_;
    C.snap = N_ > 0 ? snap_ : nullptr;
    C.snap_box = cfg_.L * cfg_.a;
    return C;
  }

  ObsK<R> obs(int64_t step, int accumulate) const {
    ObsK<R> O;
    memset(&O, 0, sizeof(O));
    const Config& c = cfg_;
    O.part = parts_;
    O.nparts = 0;
    O.mass_rest = DEV ? c.rho * (double)nnodes_ : 0.0;
    O.a3 = c.a * c.a * c.a;
    O.u_scale = c.a / c.h;
    O.N = N_;
    O.x = x_;
    O.xl = xl_;
    O.img = img_;
    O.v = v_;
    O.Fc = Fc_;
    O.box = c.L * c.a;
    O.m = c.m;
    O.h = c.h / nsub_;
    O.xref = xref_;
    O.acc = acc_;
    O.nonpos = nonpos_;
    O.out = obs_;
    O.step = step;
    O.accumulate = accumulate;
    return O;
  }

  // carve the workspace; with base == nullptr only computes the size
  void layout(unsigned char* base) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> unsigned char* {
      off = align_up(off, 256);
      unsigned char* p = base ? base + off : nullptr;
      off += bytes;
      return p;
    };
    const size_t popb = Q * plane_ * sizeof(S);
    pop_[0] = reinterpret_cast<S*>(take(popb));
    pop_[1] = reinterpret_cast<S*>(take(popb));
    const size_t n3 = 3 * (size_t)(N_ > 0 ? N_ : 1);
    x_ = reinterpret_cast<R*>(take(n3 * sizeof(R)));
    xl_ = reinterpret_cast<R*>(take(n3 * sizeof(R)));
    img_ = reinterpret_cast<int*>(take(n3 * sizeof(int)));
    v_ = reinterpret_cast<R*>(take(n3 * sizeof(R)));
    F_ = reinterpret_cast<R*>(take(n3 * sizeof(R)));
    Fc_ = reinterpret_cast<R*>(take(n3 * sizeof(R)));
    vh_ = reinterpret_cast<R*>(take(n3 * sizeof(R)));
    fcons_ = reinterpret_cast<R*>(take(n3 * sizeof(R)));
    fch_ = reinterpret_cast<R*>(take(n3 * nsub_ * sizeof(R)));
    xref_ = reinterpret_cast<double*>(take(n3 * sizeof(double)));
    rb_ = reinterpret_cast<double*>(take(2 * n3 * sizeof(double)));
    snap_ = reinterpret_cast<double*>(take(4 * n3 * sizeof(double)));
    e_node_ = reinterpret_cast<int*>(take(cap_ * sizeof(int)));
    e_w_ = reinterpret_cast<R*>(take(cap_ * sizeof(R)));
    e_mom_ = reinterpret_cast<R*>(take(4 * cap_ * sizeof(R)));
    for (int j = 0; j < 2; ++j) {
      p_pos_[j] = reinterpret_cast<int4*>(take(cap_ * sizeof(int4)));
      p_dn_[j] = reinterpret_cast<R*>(take((size_t)Q * cap_ * sizeof(R)));
      p_count_[j] = reinterpret_cast<int*>(take(sizeof(int)));
      masks_[j] = reinterpret_cast<unsigned*>(take(nsegs() * sizeof(unsigned)));
      corr_[j] = N_ > 0 ? reinterpret_cast<R*>(take((size_t)Q * plane_ * sizeof(R))) : nullptr;
    }
    status_ = reinterpret_cast<unsigned*>(take(sizeof(unsigned)));
    nonpos_ = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long)));
    acc_ = reinterpret_cast<double*>(take(4 * sizeof(double)));
    obs_ = reinterpret_cast<double*>(take(kNObs * sizeof(double)));
    parts_ = reinterpret_cast<double*>(take(4 * (size_t)nparts_ * sizeof(double)));
    bytes_ = align_up(off, 256);
  }

  Config cfg_;
  int L_ = 0, N_ = 0, cap_ = 8, nparts_ = 0, nsub_ = 1;
  unsigned long long nnodes_ = 0, plane_ = 0;
  size_t bytes_ = 0;
  int cur_ = 0;
  S* pop_[2] = {nullptr, nullptr};
  R *fch_ = nullptr;
  R *x_ = nullptr, *xl_ = nullptr, *v_ = nullptr, *F_ = nullptr, *Fc_ = nullptr, *vh_ = nullptr, *fcons_ = nullptr;
  int* img_ = nullptr;
  double* xref_ = nullptr;
  double* rb_ = nullptr;  // bead read-back staging: 3N positions, 3N velocities (FP64)
  double* snap_ = nullptr;  // two slots of the same, written by the bead kernel every step
  // the snapshot of step snap_k_ holds the bead state (no state change since that step)
  bool snap_valid_ = false;
  uint32_t snap_k_ = 0;
  // read-backs of snapshot slots on the engine's own stream, not yet known to be complete
  bool snap_pending_[2] = {false, false};
  cudaStream_t side_ = nullptr;
  cudaEvent_t step_ev_ = nullptr, copy_ev_[2] = {nullptr, nullptr};
  int* e_node_ = nullptr;
  R *e_w_ = nullptr, *e_mom_ = nullptr;
  int4* p_pos_[2] = {nullptr, nullptr};
  R* p_dn_[2] = {nullptr, nullptr};
  int* p_count_[2] = {nullptr, nullptr};
  unsigned* masks_[2] = {nullptr, nullptr};  // marks of the nodes that pull from pending nodes, by slot
  R* corr_[2] = {nullptr, nullptr};     // dense correction fields [i][plane], zero but at pending nodes
  int pslot_ = 0;
  bool open_ = false;  // a deferred step's correction is pending
  unsigned* status_ = nullptr;
  unsigned long long* nonpos_ = nullptr;
  double *acc_ = nullptr, *obs_ = nullptr, *parts_ = nullptr;
};

}  // namespace gblb
