// Asynchronous Parareal persistent kernel (Eq. (12), Algorithm 2).
#include "common.cuh"

namespace pr {

int run_async(pr_ctx* c, const pr_async_opts*, double*, pr_stats*, pr_event*, size_t, size_t*) {
  return fail(c, PR_ESTATE, "asynchronous path not built");
}

}  // namespace pr
