// 16-bit storage engines: deviations stored as BF16 or FP16, FP32 arithmetic.
#include "lb_engine_impl.cuh"
namespace gblb {
Engine* make_engine_bf16(const Config& c) { return new EngineT<__nv_bfloat16, float, true>(c); }
Engine* make_engine_f16(const Config& c) { return new EngineT<__half, float, true>(c); }
}  // namespace gblb
