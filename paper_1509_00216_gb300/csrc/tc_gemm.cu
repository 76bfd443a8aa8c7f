// Tensor-core (tcgen05) sigma path.
#include "engine.hpp"

namespace mpslcc {

void tc_prepare(Ctx& c, SigmaPlan& P, int prec) {
  throw Error(ST_ARG, "tensor-core sigma path not built yet");
}
void tc_sigma(Ctx& c, SigmaPlan& P, const double* x, double* y) {
  throw Error(ST_ARG, "tensor-core sigma path not built yet");
}

}  // namespace mpslcc
