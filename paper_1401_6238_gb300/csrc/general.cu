// general.cu -- general path (placeholder until its kernels land).
#include "general.h"

namespace hk {

struct GeneralPlan {
    int unused;
};

hankel_status general_create(GeneralPlan** out, const std::vector<hankel_desc>&, hankel_dtype, uint32_t, int64_t*,
                             int64_t*, int64_t*, int64_t*, int64_t*, std::string& err) {
    *out = nullptr;
    err = "this plan needs the general path (complex data, distinct vectors or BHHB), not built yet";
    return HANKEL_EUNSUPPORTED;
}
hankel_status general_forward(GeneralPlan*, const void*, const void*, void*, void*, cudaStream_t, std::string& err) {
    err = "general path not built";
    return HANKEL_EUNSUPPORTED;
}
hankel_status general_backward(GeneralPlan*, const void*, const void*, const void*, void*, void*, cudaStream_t,
                               std::string& err) {
    err = "general path not built";
    return HANKEL_EUNSUPPORTED;
}
void general_info(GeneralPlan*, int64_t* jobs, int64_t* launches, int64_t* lengths, int64_t* ws) {
    *jobs = *launches = *lengths = *ws = 0;
}
void general_destroy(GeneralPlan* g) { delete g; }

}  // namespace hk
