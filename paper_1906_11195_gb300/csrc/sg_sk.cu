// sg_sk.cu -- Sherrington-Kirkpatrick model, host side.
#include "../../include/sg.h"
#include "sg_model.h"

namespace sg {

Model* make_sk_model(int n, const int8_t* J, int n_replicas, const double* temps, uint64_t seed,
                     int kernel, int block, const std::vector<int64_t>& tw,
                     const std::vector<int64_t>& tm) {
    (void)n; (void)J; (void)n_replicas; (void)temps; (void)seed; (void)kernel; (void)block;
    (void)tw; (void)tm;
    fail(SG_EINVAL, "SK model not available in this build");
}

}  // namespace sg
