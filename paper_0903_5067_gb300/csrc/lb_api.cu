// C ABI of libgblb (declared in include/lb.h): context management, validation, workspace,
// checkpoints and the test hooks.  The numerical work lives in the engines (lb_f64.cu,
// lb_f32.cu, lb_h16.cu) and in lb_device.cuh.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "../../include/lb.h"
#include "lb_device.cuh"
#include "lb_engine.h"
#include "philox.cuh"

using namespace gblb;

namespace gblb {
// test hooks
__global__ void k_philox(const uint32_t* __restrict__ ctr, long long n, uint32_t k0, uint32_t k1,
                         uint32_t* __restrict__ out) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const U4 r = philox4x32_10(U4{ctr[4 * t], ctr[4 * t + 1], ctr[4 * t + 2], ctr[4 * t + 3]}, k0, k1);
  out[4 * t] = r.x;
  out[4 * t + 1] = r.y;
  out[4 * t + 2] = r.z;
  out[4 * t + 3] = r.w;
}

__global__ void k_cell_index_f32(const float* __restrict__ x, long long n, float a, int L, int* __restrict__ out) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  float fr;
  out[t] = cell_of<float>(x[t], a, L, fr);
}

}  // namespace gblb

struct lb_ctx {
  Config cfg;
  std::vector<double> x0, v0;
  int obs_stride = 0;
  // trajectory recording: caller-owned device ring of traj_cap frames of 3N doubles
  double* traj = nullptr;
  int traj_cap = 0, traj_stride = 0;
  int64_t traj_frames = 0, traj_origin = 0;
  cudaStream_t stream = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  bool ws_owned = false;
  bool live = false;  // device state initialised
  int64_t step = 0;
  std::unique_ptr<Engine> eng;
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> evs;
  // asynchronous bead read-backs: a ring of events and pinned status words by ticket
  static constexpr int kTickets = 8;
  cudaEvent_t tev[kTickets] = {};
  unsigned* tstatus = nullptr;
  int64_t tickets = 0;
  double timed_ms = 0.0;
  int64_t timed_launches = 0;
};

namespace {

int fail(int code, const char* msg);
void record_frame(lb_ctx* ctx);

// the message of this thread's last failing call, until lb_last_error takes it
thread_local std::string t_last_error;

int fail(int code, const char* msg) {
  t_last_error = msg ? msg : "";
  if (getenv("GBLB_VERBOSE")) fprintf(stderr, "libgblb: %s\n", msg);
  return code;
}

}  // namespace

namespace gblb {
// failure with a message for this thread's lb_last_error, for entry points outside this file
int api_fail(int code, const char* msg) { return fail(code, msg); }
}  // namespace gblb

namespace {

template <class F>
int guarded(F&& f) {
  try {
    return f();
  } catch (const LbError& e) {
    return fail(e.code, e.what());
  } catch (const std::bad_alloc&) {
    return fail(LB_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(LB_ERR_CUDA, e.what());
  }
}

Engine* make_engine(const Config& c) {
  switch (c.precision) {
    case LB_FP64: return make_engine_f64(c);
    case LB_FP32: return make_engine_f32(c);
    case LB_BF16: return make_engine_bf16(c);
    case LB_FP16: return make_engine_f16(c);
  }
  throw LbError(LB_ERR_ARG, "unknown precision");
}

double min_image(double d, double box) { return d - box * nearbyint(d / box); }

// Host-side chain generator: walk of fixed step `bond` from the box centre, unit directions
// uniform on the sphere (Marsaglia 1972) from the Philox stream tag 2, optional rejection
// of trial beads closer than sigma to an earlier non-adjacent bead.
bool generate_chain(const Config& c, double bond, int saw, std::vector<double>& X) {
  const int N = c.N;
  const double box = c.L * c.a;
  X.assign(3 * (size_t)N, 0.0);
  for (int q = 0; q < 3; ++q) X[q] = 0.5 * box;
  const uint32_t k0 = (uint32_t)(c.seed & 0xffffffffu), k1 = 2u | ((uint32_t)c.replica << 8);
  for (int i = 1; i < N; ++i) {
    bool placed = false;
    for (uint32_t tr = 0; tr < 1000 && !placed; ++tr) {
      double d[3];
      for (uint32_t call = 0;; ++call) {
        const U4 r = philox4x32_10(U4{(uint32_t)i, tr, call, 0u}, k0, k1);
        const double v1 = 2.0 * uniform_f64(r.x) - 1.0, v2 = 2.0 * uniform_f64(r.y) - 1.0;
        const double s = v1 * v1 + v2 * v2;
        if (s < 1.0) {
          const double f = 2.0 * sqrt(1.0 - s);
          d[0] = v1 * f;
          d[1] = v2 * f;
          d[2] = 1.0 - 2.0 * s;
          break;
        }
        if (call > 64) return false;
      }
      double t[3];
      for (int q = 0; q < 3; ++q) t[q] = X[3 * (i - 1) + q] + bond * d[q];
      bool ok = true;
      if (saw) {
        for (int j = 0; j < i - 1 && ok; ++j) {
          double r2 = 0;
          for (int q = 0; q < 3; ++q) {
            const double dd = min_image(t[q] - X[3 * j + q], box);
            r2 += dd * dd;
          }
          if (r2 < c.sigma * c.sigma) ok = false;
        }
      }
      if (ok) {
        for (int q = 0; q < 3; ++q) X[3 * i + q] = t[q];
        placed = true;
      }
    }
    if (!placed) return false;
  }
  return true;
}

void record_frame(lb_ctx* ctx) {
  double* dst = ctx->traj + (size_t)(ctx->traj_frames % ctx->traj_cap) * 3 * (size_t)ctx->cfg.N;
  ctx->eng->record_frame(dst, ctx->stream);
  ctx->traj_frames += 1;
}

void materialise(lb_ctx* ctx) {
  if (ctx->live) return;
  if (!ctx->eng) ctx->eng.reset(make_engine(ctx->cfg));
  if (!ctx->ws) {
    const size_t b = ctx->eng->workspace_bytes();
    void* p = nullptr;
    cuda_check(cudaMalloc(&p, b), "workspace allocation");
    ctx->ws = p;
    ctx->ws_bytes = b;
    ctx->ws_owned = true;
  }
  ctx->eng->bind(ctx->ws);
  ctx->eng->initialise(ctx->x0.empty() ? nullptr : ctx->x0.data(), ctx->v0.empty() ? nullptr : ctx->v0.data(),
                       ctx->stream);
  ctx->live = true;
}

int status_from_device(unsigned st) {
  if (st & ST_FENE) return fail(LB_ERR_FENE, "a FENE bond reached R0");
  if (st & ST_NONFINITE) return fail(LB_ERR_NONFINITE, "a non-finite value appeared in the state");
  if (st & ST_TIMEOUT) return fail(LB_ERR_TIMEOUT, "a device wait ran out of iterations");
  return LB_OK;
}

void drain_timing(lb_ctx* ctx) {
  if (ctx->evs.empty()) return;
  cuda_check(cudaStreamSynchronize(ctx->stream), "sync timing");
  for (auto& e : ctx->evs) {
    float ms = 0.f;
    cuda_check(cudaEventElapsedTime(&ms, e.first, e.second), "event time");
    ctx->timed_ms += ms;
    ctx->timed_launches += 1;
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  ctx->evs.clear();
}

const uint64_t kMagic = 0x47424c4243484b31ull;  // "GBLBCHK1"

}  // namespace

extern "C" {

int lb_create(lb_ctx** out, int L, double rho, double eta, double eta_b, double kT, double h, double a,
              uint64_t seed, int precision) {
  if (!out) return fail(LB_ERR_ARG, "invalid argument: !out");
  *out = nullptr;
  if (L < 4 || L > 1290) return fail(LB_ERR_ARG, "L out of range [4, 1290]");
  if (!(rho > 0) || !(eta > 0) || !(eta_b > 0) || !(h > 0) || !(a > 0) || !(kT >= 0))
    return fail(LB_ERR_ARG, "rho, eta, eta_b, h, a must be > 0 and kT >= 0");
  if (precision < LB_FP64 || precision > LB_FP16) return fail(LB_ERR_ARG, "unknown precision");
  return guarded([&] {
    auto* c = new lb_ctx();
    c->cfg.L = L;
    c->cfg.rho = rho;
    c->cfg.eta = eta;
    c->cfg.eta_b = eta_b;
    c->cfg.kT = kT;
    c->cfg.h = h;
    c->cfg.a = a;
    c->cfg.seed = seed;
    c->cfg.precision = precision;
    *out = c;
    return (int)LB_OK;
  });
}

int lb_add_chain(lb_ctx* ctx, int N, double m, double zeta, double k_fene, double R0, double eps, double sigma,
                 const double* x0, const double* v0, double bond, int saw) {
  if (!ctx) return fail(LB_ERR_ARG, "invalid argument: !ctx");
  if (ctx->live || ctx->cfg.N > 0) return fail(LB_ERR_STATE, "chain must be added once, before the first step");
  if (N < 1 || N > 1024) return fail(LB_ERR_ARG, "N out of range [1, 1024]");
  if (8ll * N * ctx->cfg.substeps > 16384) return fail(LB_ERR_ARG, "8 N substeps exceeds 16384");
  if (!(m > 0) || !(zeta >= 0) || !(k_fene >= 0) || !(R0 > 0) || !(eps >= 0) || !(sigma > 0))
    return fail(LB_ERR_ARG, "invalid chain parameters");
  return guarded([&] {
    Config& c = ctx->cfg;
    c.N = N;
    c.m = m;
    c.zeta = zeta;
    c.kfene = k_fene;
    c.R0 = R0;
    c.eps = eps;
    c.sigma = sigma;
    if (x0) {
      ctx->x0.assign(x0, x0 + 3 * (size_t)N);
    } else {
      if (!(bond > 0) || bond >= R0) {
        c.N = 0;
        return fail(LB_ERR_ARG, "generated chain needs 0 < bond < R0");
      }
      if (!generate_chain(c, bond, saw, ctx->x0)) {
        c.N = 0;
        return fail(LB_ERR_ARG, "chain generator could not place every bead");
      }
    }
    for (double v : ctx->x0)
      if (!std::isfinite(v)) {
        c.N = 0;
        return fail(LB_ERR_ARG, "non-finite bead position");
      }
    const double box = c.L * c.a;
    for (int i = 0; i + 1 < N; ++i) {
      double r2 = 0;
      for (int q = 0; q < 3; ++q) {
        const double d = min_image(ctx->x0[3 * i + q] - ctx->x0[3 * (i + 1) + q], box);
        r2 += d * d;
      }
      if (r2 >= R0 * R0) {
        c.N = 0;
        ctx->x0.clear();
        return fail(LB_ERR_FENE, "initial bond stretched beyond R0");
      }
    }
    if (v0)
      ctx->v0.assign(v0, v0 + 3 * (size_t)N);
    else
      ctx->v0.clear();
    ctx->eng.reset();
    return (int)LB_OK;
  });
}

int lb_set_options(lb_ctx* ctx, int noise_fluid, int noise_beads, int stress_only, const double ext_bead_force[3],
                   int counter_force_fluid) {
  if (!ctx) return fail(LB_ERR_ARG, "invalid argument: !ctx");
  Config& c = ctx->cfg;
  c.noise_fluid = noise_fluid ? 1 : 0;
  c.noise_beads = noise_beads ? 1 : 0;
  c.stress_only = stress_only ? 1 : 0;
  for (int q = 0; q < 3; ++q) c.ext[q] = ext_bead_force ? ext_bead_force[q] : 0.0;
  c.counter_force = counter_force_fluid ? 1 : 0;
  if (ctx->eng) ctx->eng->set_config(c);
  return LB_OK;
}

int lb_set_md_substeps(lb_ctx* ctx, int n) {
  if (!ctx || n < 1 || n > 16) return fail(LB_ERR_ARG, "invalid argument: !ctx || n < 1 || n > 16");
  if (ctx->live) return fail(LB_ERR_STATE, "substeps must be set before the first device call");
  if (8ll * ctx->cfg.N * n > 16384) return fail(LB_ERR_ARG, "8 N substeps exceeds 16384");
  ctx->cfg.substeps = n;
  ctx->eng.reset();
  return LB_OK;
}

int lb_set_stream(lb_ctx* ctx, void* stream) {
  if (!ctx) return fail(LB_ERR_ARG, "invalid argument: !ctx");
  ctx->stream = static_cast<cudaStream_t>(stream);
  return LB_OK;
}

int lb_workspace_size(lb_ctx* ctx, size_t* bytes) {
  if (!ctx || !bytes) return fail(LB_ERR_ARG, "invalid argument: !ctx || !bytes");
  return guarded([&] {
    if (!ctx->eng) ctx->eng.reset(make_engine(ctx->cfg));
    *bytes = ctx->eng->workspace_bytes();
    return (int)LB_OK;
  });
}

int lb_bind_workspace(lb_ctx* ctx, void* device_ptr, size_t bytes) {
  if (!ctx || !device_ptr) return fail(LB_ERR_ARG, "invalid argument: !ctx || !device_ptr");
  if (ctx->live) return fail(LB_ERR_STATE, "workspace must be bound before the first device call");
  if (reinterpret_cast<uintptr_t>(device_ptr) % 256 != 0) return fail(LB_ERR_ARG, "workspace not 256-byte aligned");
  return guarded([&] {
    if (!ctx->eng) ctx->eng.reset(make_engine(ctx->cfg));
    if (bytes < ctx->eng->workspace_bytes()) return fail(LB_ERR_ARG, "workspace too small");
    if (ctx->ws_owned) cudaFree(ctx->ws);
    ctx->ws = device_ptr;
    ctx->ws_bytes = bytes;
    ctx->ws_owned = false;
    return (int)LB_OK;
  });
}

int lb_step(lb_ctx* ctx, int64_t n) {
  if (!ctx || n < 0) return fail(LB_ERR_ARG, "invalid argument: !ctx || n < 0");
  return guarded([&] {
    materialise(ctx);
    for (int64_t t = 0; t < n; ++t) {
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      if (ctx->timing) {
        cuda_check(cudaEventCreate(&e0), "event");
        cuda_check(cudaEventCreate(&e1), "event");
        ctx->evs.emplace_back(e0, e1);
      }
      ctx->eng->step_deferred((uint32_t)ctx->step, ctx->stream, e0, e1);
      ctx->step += 1;
      if (ctx->obs_stride > 0 && ctx->cfg.N > 0 && ctx->step % ctx->obs_stride == 0)
        ctx->eng->observables(nullptr, ctx->step, 1, ctx->stream);
      if (ctx->traj && (ctx->step - ctx->traj_origin) % ctx->traj_stride == 0) record_frame(ctx);
    }
    // the last step's force correction stays pending: every call that reads or replaces the
    // fluid state applies it first
    return (int)LB_OK;
  });
}

int lb_sync(lb_ctx* ctx) {
  if (!ctx) return fail(LB_ERR_ARG, "invalid argument: !ctx");
  return guarded([&] {
    if (!ctx->live) return (int)LB_OK;
    cuda_check(cudaStreamSynchronize(ctx->stream), "stream sync");
    return status_from_device(ctx->eng->read_status(ctx->stream));
  });
}

int lb_get_populations(lb_ctx* ctx, double* out, size_t cap) {
  if (!ctx || !out) return fail(LB_ERR_ARG, "invalid argument: !ctx || !out");
  const size_t need = 19 * (size_t)ctx->cfg.L * ctx->cfg.L * ctx->cfg.L;
  if (cap < need) return fail(LB_ERR_ARG, "population buffer too small");
  return guarded([&] {
    materialise(ctx);
    ctx->eng->get_populations(out, ctx->stream);
    return status_from_device(ctx->eng->read_status(ctx->stream));
  });
}

int lb_set_populations(lb_ctx* ctx, const double* in, size_t count) {
  if (!ctx || !in) return fail(LB_ERR_ARG, "invalid argument: !ctx || !in");
  const size_t need = 19 * (size_t)ctx->cfg.L * ctx->cfg.L * ctx->cfg.L;
  if (count != need) return fail(LB_ERR_ARG, "population count must be 19 L^3");
  return guarded([&] {
    materialise(ctx);
    ctx->eng->set_populations(in, ctx->stream);
    return (int)LB_OK;
  });
}

int lb_get_beads(lb_ctx* ctx, double* x, double* v, size_t cap) {
  if (!ctx) return fail(LB_ERR_ARG, "invalid argument: !ctx");
  if (cap < 3 * (size_t)ctx->cfg.N) return fail(LB_ERR_ARG, "bead buffer too small");
  if (!ctx->live) {
    // before the first device call the chain is the host-staged initial state
    const size_t n3 = 3 * (size_t)ctx->cfg.N;
    for (size_t t = 0; t < n3; ++t) {
      if (x) x[t] = ctx->x0[t];
      if (v) v[t] = ctx->v0.empty() ? 0.0 : ctx->v0[t];
    }
    return (int)LB_OK;
  }
  return guarded([&] {
    materialise(ctx);
    ctx->eng->get_beads(x, v, ctx->stream);
    return status_from_device(ctx->eng->read_status(ctx->stream));
  });
}

int lb_get_beads_async(lb_ctx* ctx, double* x, double* v, size_t cap, int64_t* ticket) {
  if (!ctx || !ticket) return fail(LB_ERR_ARG, "invalid argument: !ctx || !ticket");
  if (cap < 3 * (size_t)ctx->cfg.N) return fail(LB_ERR_ARG, "bead buffer too small");
  return guarded([&] {
    materialise(ctx);
    if (!ctx->tstatus) {
      cuda_check(cudaMallocHost(&ctx->tstatus, lb_ctx::kTickets * sizeof(unsigned)), "pinned status");
      for (int j = 0; j < lb_ctx::kTickets; ++j)
        cuda_check(cudaEventCreateWithFlags(&ctx->tev[j], cudaEventDisableTiming), "event");
    }
    const int slot = (int)(ctx->tickets % lb_ctx::kTickets);
    ctx->eng->enqueue_beads_async(x, v, ctx->tstatus + slot, ctx->tev[slot], ctx->stream);
    *ticket = ctx->tickets++;
    return (int)LB_OK;
  });
}

int lb_wait(lb_ctx* ctx, int64_t ticket) {
  if (!ctx || ticket < 0 || ticket >= ctx->tickets) return fail(LB_ERR_ARG, "invalid argument: !ctx || ticket < 0 || ticket >= ctx->tickets");
  return guarded([&] {
    const int slot = (int)(ticket % lb_ctx::kTickets);
    // a later read-back in the same slot completes after this one: waiting on it suffices
    cuda_check(cudaEventSynchronize(ctx->tev[slot]), "wait read-back");
    return status_from_device(ctx->tstatus[slot]);
  });
}

int lb_get_observables(lb_ctx* ctx, double* out, size_t cap) {
  if (!ctx || !out) return fail(LB_ERR_ARG, "invalid argument: !ctx || !out");
  if (cap < LB_NOBS) return fail(LB_ERR_ARG, "observable buffer too small");
  return guarded([&] {
    materialise(ctx);
    ctx->eng->observables(out, ctx->step, 0, ctx->stream);
    return status_from_device(ctx->eng->read_status(ctx->stream));
  });
}

int lb_record_trajectory(lb_ctx* ctx, double* traj_dev, int capacity, int stride) {
  if (!ctx) return fail(LB_ERR_ARG, "invalid argument: !ctx");
  if (!traj_dev || capacity <= 0 || stride <= 0) {
    ctx->traj = nullptr;
    ctx->traj_cap = ctx->traj_stride = 0;
    return LB_OK;
  }
  if (ctx->cfg.N <= 0) return fail(LB_ERR_STATE, "trajectory recording needs a chain");
  return guarded([&] {
    materialise(ctx);
    ctx->traj = traj_dev;
    ctx->traj_cap = capacity;
    ctx->traj_stride = stride;
    ctx->traj_frames = 0;
    ctx->traj_origin = ctx->step;
    record_frame(ctx);
    return (int)LB_OK;
  });
}

int lb_trajectory_frames(lb_ctx* ctx, int64_t* frames) {
  if (!ctx || !frames) return fail(LB_ERR_ARG, "invalid argument: !ctx || !frames");
  *frames = ctx->traj ? ctx->traj_frames : 0;
  return LB_OK;
}

int lb_set_obs_stride(lb_ctx* ctx, int stride) {
  if (!ctx || stride < 0) return fail(LB_ERR_ARG, "invalid argument: !ctx || stride < 0");
  ctx->obs_stride = stride;
  return LB_OK;
}

int lb_reset_reference(lb_ctx* ctx) {
  if (!ctx) return fail(LB_ERR_ARG, "invalid argument: !ctx");
  return guarded([&] {
    materialise(ctx);
    ctx->eng->reset_reference(ctx->stream);
    return (int)LB_OK;
  });
}

int lb_save(lb_ctx* ctx, const char* path) {
  if (!ctx || !path) return fail(LB_ERR_ARG, "invalid argument: !ctx || !path");
  return guarded([&] {
    materialise(ctx);
    std::vector<unsigned char> buf(ctx->eng->state_bytes());
    ctx->eng->save_state(buf.data(), ctx->stream);
    FILE* f = fopen(path, "wb");
    if (!f) return fail(LB_ERR_ARG, "cannot open checkpoint for writing");
    const uint64_t sz = buf.size();
    bool ok = fwrite(&kMagic, 8, 1, f) == 1 && fwrite(&ctx->cfg, sizeof(Config), 1, f) == 1 &&
              fwrite(&ctx->step, sizeof(int64_t), 1, f) == 1 && fwrite(&sz, 8, 1, f) == 1 &&
              fwrite(buf.data(), 1, buf.size(), f) == buf.size();
    ok = (fclose(f) == 0) && ok;
    return ok ? (int)LB_OK : fail(LB_ERR_ARG, "checkpoint write failed");
  });
}

int lb_load(lb_ctx* ctx, const char* path) {
  if (!ctx || !path) return fail(LB_ERR_ARG, "invalid argument: !ctx || !path");
  return guarded([&] {
    FILE* f = fopen(path, "rb");
    if (!f) return fail(LB_ERR_ARG, "cannot open checkpoint");
    uint64_t magic = 0, sz = 0;
    Config c;
    int64_t step = 0;
    bool ok = fread(&magic, 8, 1, f) == 1 && magic == kMagic && fread(&c, sizeof(Config), 1, f) == 1 &&
              fread(&step, sizeof(int64_t), 1, f) == 1 && fread(&sz, 8, 1, f) == 1;
    if (!ok || c.L != ctx->cfg.L || c.precision != ctx->cfg.precision || c.N != ctx->cfg.N) {
      fclose(f);
      return fail(LB_ERR_STATE, "checkpoint does not match the context (L, precision, N)");
    }
    std::vector<unsigned char> buf(sz);
    ok = fread(buf.data(), 1, sz, f) == sz;
    fclose(f);
    if (!ok) return fail(LB_ERR_ARG, "truncated checkpoint");
    ctx->cfg = c;
    materialise(ctx);
    ctx->eng->set_config(c);
    if (sz != ctx->eng->state_bytes()) return fail(LB_ERR_STATE, "checkpoint size mismatch");
    ctx->eng->load_state(buf.data(), ctx->stream);
    ctx->step = step;
    return (int)LB_OK;
  });
}

int lb_adjoint_displacement(lb_ctx* ctx, int64_t T, int K, double* objective, double* grad_x0, size_t cap,
                            double* grad_zeta) {
  if (!ctx || !objective || !grad_x0 || !grad_zeta || T < 1 || K < 1) return fail(LB_ERR_ARG, "invalid argument: !ctx || !objective || !grad_x0 || !grad_zeta || T < 1 || K < 1");
  if (ctx->cfg.N == 0) return fail(LB_ERR_STATE, "adjoint needs a chain");
  if (cap < 3 * (size_t)ctx->cfg.N) return fail(LB_ERR_ARG, "gradient buffer too small");
  if (ctx->step != 0) return fail(LB_ERR_STATE, "adjoint must start from the initial state");
  return guarded([&] {
    materialise(ctx);
    ctx->eng->adjoint_displacement(T, K, (uint32_t)ctx->step, objective, grad_x0, grad_zeta, ctx->stream);
    ctx->step += T;
    return status_from_device(ctx->eng->read_status(ctx->stream));
  });
}

int64_t lb_get_step(lb_ctx* ctx) { return ctx ? ctx->step : -1; }

int lb_set_timing(lb_ctx* ctx, int enable) {
  if (!ctx) return fail(LB_ERR_ARG, "invalid argument: !ctx");
  return guarded([&] {
    drain_timing(ctx);
    ctx->timing = enable != 0;
    ctx->timed_ms = 0.0;
    ctx->timed_launches = 0;
    return (int)LB_OK;
  });
}

int lb_get_timing(lb_ctx* ctx, double* total_ms, int64_t* launches) {
  if (!ctx) return fail(LB_ERR_ARG, "invalid argument: !ctx");
  return guarded([&] {
    drain_timing(ctx);
    if (total_ms) *total_ms = ctx->timed_ms;
    if (launches) *launches = ctx->timed_launches;
    return (int)LB_OK;
  });
}

void lb_destroy(lb_ctx* ctx) {
  if (!ctx) return;
  try {
    drain_timing(ctx);
  } catch (...) {
  }
  if (ctx->tstatus) {  // asynchronous read-backs may still be in flight
    if (ctx->live) {
      cudaStreamSynchronize(ctx->stream);
      try {
        ctx->eng->drain();
      } catch (...) {
      }
    }
    for (int j = 0; j < lb_ctx::kTickets; ++j)
      if (ctx->tev[j]) cudaEventDestroy(ctx->tev[j]);
    cudaFreeHost(ctx->tstatus);
  }
  if (ctx->ws_owned && ctx->ws) cudaFree(ctx->ws);
  delete ctx;
}

size_t lb_last_error(char* buf, size_t cap) {
  const size_t n = t_last_error.size();
  if (buf && cap > 0) {
    const size_t m = n < cap - 1 ? n : cap - 1;
    memcpy(buf, t_last_error.data(), m);
    buf[m] = '\0';
  }
  t_last_error.clear();
  return n;
}

const char* lb_strerror(int status) {
  switch (status) {
    case LB_OK: return "ok";
    case LB_ERR_ARG: return "invalid argument";
    case LB_ERR_CUDA: return "CUDA runtime error";
    case LB_ERR_OOM: return "device out of memory";
    case LB_ERR_FENE: return "FENE bond stretched to r >= R0";
    case LB_ERR_NONFINITE: return "non-finite state";
    case LB_ERR_TIMEOUT: return "device wait timed out";
    case LB_ERR_STATE: return "call not valid in the current state";
  }
  return "unknown status";
}

int lb_philox4x32_10(const uint32_t* ctr_dev, int64_t n, uint32_t k0, uint32_t k1, uint32_t* out_dev,
                     void* stream) {
  if (n < 0 || (n > 0 && (!ctr_dev || !out_dev))) return fail(LB_ERR_ARG, "invalid argument: n < 0 || (n > 0 && (!ctr_dev || !out_dev))");
  if (n == 0) return LB_OK;
  k_philox<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(ctr_dev, n, k0, k1, out_dev);
  return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ERR_CUDA;
}

int lb_debug_coupling_cells(lb_ctx* ctx, int32_t* nodes, double* x_stored, size_t cap) {
  if (!ctx) return fail(LB_ERR_ARG, "invalid argument: !ctx");
  if (ctx->cfg.N == 0) return fail(LB_ERR_STATE, "no chain");
  if (!ctx->live) return fail(LB_ERR_STATE, "the context has not stepped");
  if ((nodes && cap < 8 * (size_t)ctx->cfg.N * ctx->cfg.substeps) || (x_stored && cap < 3 * (size_t)ctx->cfg.N))
    return fail(LB_ERR_ARG, "buffer too small");
  return guarded([&] {
    ctx->eng->debug_coupling_cells(nodes, x_stored, ctx->stream);
    return (int)LB_OK;
  });
}

int lb_cell_index_f32(const float* x_dev, int64_t n, float a, int L, int32_t* out_dev, void* stream) {
  if (n < 0 || L < 1 || !(a > 0) || (n > 0 && (!x_dev || !out_dev))) return fail(LB_ERR_ARG, "invalid argument: n < 0 || L < 1 || !(a > 0) || (n > 0 && (!x_dev || !out_dev))");
  if (n == 0) return LB_OK;
  k_cell_index_f32<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(x_dev, n, a, L,
                                                                                               out_dev);
  return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ERR_CUDA;
}

}  // extern "C"
