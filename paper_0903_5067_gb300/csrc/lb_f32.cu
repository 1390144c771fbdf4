// FP32 engine: populations stored as FP32 deviations n_i - w_i rho0, FP32 arithmetic.
#include "lb_engine_impl.cuh"
namespace gblb {
Engine* make_engine_f32(const Config& c) { return new EngineT<float, float, true>(c); }
}  // namespace gblb
