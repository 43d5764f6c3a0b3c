// Consistent DSA (App. B) -- placeholder until the solver lands.
#include "common.cuh"

namespace rte {
struct DsaState {};
void dsa_state_free(DsaState* s) { delete s; }
int dsa_setup(rte_batch_t, cudaStream_t) { return RTE_OK; }
int dsa_apply(rte_batch_t, const double*, double*, double, int, const uint8_t*, int*, cudaStream_t) {
  return fail(RTE_ESTATE, "DSA not available");
}
}  // namespace rte
