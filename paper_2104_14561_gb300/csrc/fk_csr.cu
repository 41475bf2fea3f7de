// Assembled-CSR path (Eq. (e36) with Q Psi stored once): not built yet.
#include "fk_internal.h"

fk_status fk_csr_assemble(fk_plan* p, cudaStream_t s) {
  (void)p;
  (void)s;
  return FK_ERR_UNSUPPORTED;
}

fk_status fk_csr_step(fk_plan* p, const void* u_in, void* u_out, void* snap, cudaStream_t s) {
  (void)p; (void)u_in; (void)u_out; (void)snap; (void)s;
  return FK_ERR_UNSUPPORTED;
}
