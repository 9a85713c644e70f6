// Split-precision path of H.psi (placeholder until the tcgen05 kernels land).
#include <string>

#include "su2_device.h"

namespace su2 {
int split_prepare(su2_env*, int, std::string& err) {
  err = "split-precision path not available in this build";
  return SU2_EINVAL;
}
int split_apply(su2_env*, const double*, double*, std::string& err) {
  err = "split-precision path not prepared (build the environment with prepare_split=1)";
  return SU2_EINVAL;
}
void split_free(su2_env*) {}
}  // namespace su2
