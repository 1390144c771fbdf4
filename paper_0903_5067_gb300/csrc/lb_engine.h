// Host-side engine interface: one implementation per storage precision, each in its own
// translation unit.  The C ABI (lb_api.cu) owns the context and calls through this.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <stdexcept>
#include <string>

namespace gblb {

struct Config {
  int L = 0;
  double rho = 1, eta = 1, eta_b = 1, kT = 0, h = 1, a = 1;
  uint64_t seed = 0;
  int precision = 1;
  int replica = 0;
  // chain
  int N = 0;
  double m = 1, zeta = 0, kfene = 0, R0 = 1, eps = 0, sigma = 1;
  // options
  int noise_fluid = 1, noise_beads = 1, stress_only = 0, counter_force = 0;
  int substeps = 1;  // MD steps per LB step
  double ext[3] = {0, 0, 0};
};

// status codes (mirrors lb.h)
enum { S_OK = 0, S_ARG = 1, S_CUDA = 2, S_OOM = 3, S_FENE = 4, S_NONFINITE = 5, S_TIMEOUT = 6, S_STATE = 7 };

struct LbError : std::runtime_error {
  int code;
  LbError(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

// records msg as the calling thread's last error (returned by lb_last_error) and returns code
int api_fail(int code, const char* msg);

inline void cuda_check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    if (e == cudaErrorMemoryAllocation) throw LbError(S_OOM, std::string(what) + ": " + cudaGetErrorString(e));
    throw LbError(S_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  }
}

constexpr int kNObs = 20;

class Engine {
 public:
  virtual ~Engine() {}
  virtual size_t workspace_bytes() const = 0;
  virtual void bind(void* base) = 0;
  // fluid at rest, chain from x0/v0 (3N doubles each, v0 may be null), forces F0
  virtual void initialise(const double* x0, const double* v0, cudaStream_t s) = 0;
  virtual void set_config(const Config& c) = 0;  // options changed (same sizes)
  // one step, complete on return (ev0/ev1, when given, bracket the LB kernel)
  virtual void step(uint32_t k, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1) = 0;
  // one step whose bead force correction stays pending until the next deferred step reads
  // it or flush() applies it; every other method flushes first
  virtual void step_deferred(uint32_t k, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1) = 0;
  virtual void flush(cudaStream_t s) = 0;
  virtual void get_populations(double* out, cudaStream_t s) = 0;
  virtual void set_populations(const double* in, cudaStream_t s) = 0;
  virtual void get_beads(double* x, double* v, cudaStream_t s) = 0;
  // the same read-back enqueued on s without waiting (x, v: host memory that stays valid
  // until the stream reaches the copies; pinned memory makes them asynchronous)
  virtual void enqueue_beads(double* x, double* v, cudaStream_t s) = 0;
  // enqueue a copy of the device status word to host memory
  virtual void enqueue_status(unsigned* host, cudaStream_t s) = 0;
  // bead read-back and status copy after the work queued on s so far, completing `done`;
  // off the stream s where the last step's snapshot holds the state (see EngineT)
  virtual void enqueue_beads_async(double* x, double* v, unsigned* status_host, cudaEvent_t done,
                                   cudaStream_t s) = 0;
  // wait for read-backs in flight on the engine's own stream
  virtual void drain() = 0;
  virtual void observables(double* out, int64_t step, int accumulate, cudaStream_t s) = 0;
  virtual void reset_reference(cudaStream_t s) = 0;
  // write the current unwrapped bead positions (3N doubles) to device memory
  virtual void record_frame(double* dst, cudaStream_t s) = 0;
  virtual unsigned read_status(cudaStream_t s) = 0;
  // the last step's corner nodes (8 N s) and stored bead coordinates (3 N, high part), to host
  virtual void debug_coupling_cells(int* nodes, double* x_stored, cudaStream_t s) = 0;
  // adjoint: objective O = sum_b |x_b(T) - x_b(0)|^2 over T steps from the current state,
  // its gradient with respect to the current bead positions (3N) and zeta, noise fixed,
  // forward checkpoints every K steps; leaves the state at step k0 + T
  virtual void adjoint_displacement(int64_t T, int K, uint32_t k0, double* O, double* gx, double* gz,
                                    cudaStream_t s) = 0;
  // raw state for checkpoints
  virtual size_t state_bytes() const = 0;
  virtual void save_state(void* host, cudaStream_t s) = 0;
  virtual void load_state(const void* host, cudaStream_t s) = 0;
};

Engine* make_engine_f64(const Config& c);
Engine* make_engine_f32(const Config& c);
Engine* make_engine_bf16(const Config& c);
Engine* make_engine_f16(const Config& c);

}  // namespace gblb
