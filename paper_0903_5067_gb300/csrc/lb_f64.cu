// FP64 engine: full populations in FP64, FP64 arithmetic (the plain path).
#include "lb_engine_impl.cuh"
namespace gblb {
Engine* make_engine_f64(const Config& c) { return new EngineT<double, double, false>(c); }
}  // namespace gblb
