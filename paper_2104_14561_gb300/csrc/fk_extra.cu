// Adjoint: not built yet.
#include "fk_internal.h"

extern "C" {

fk_status fk_adjoint(fk_plan* plan, const void* u_terminal, const double* cotangent_u0,
                     double* dtheta, void* du_terminal, int checkpoint_every,
                     cudaStream_t stream) {
  (void)plan; (void)u_terminal; (void)cotangent_u0; (void)dtheta; (void)du_terminal;
  (void)checkpoint_every; (void)stream;
  return FK_ERR_UNSUPPORTED;
}

}  // extern "C"
