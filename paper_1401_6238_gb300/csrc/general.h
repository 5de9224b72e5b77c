// general.h -- the general path: complex data, distinct mode vectors, alpha
// with its own x_1, and block Hankel tensors of any level (BHHB is level 2).
// Spectra of every distinct operand are computed once into plan workspace,
// then each product is one k-dimensional transform.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "hankel.h"

namespace hk {

struct GeneralPlan;

hankel_status general_create(GeneralPlan** out, const std::vector<hankel_mdesc>& descs, hankel_dtype dtype,
                             uint32_t flags, int64_t* h_elems, int64_t* x_elems, int64_t* y_elems, int64_t* sum_L,
                             int64_t* max_L, std::string& err);
hankel_status general_forward(GeneralPlan* g, const void* h, const void* x, void* y, void* alpha, cudaStream_t st,
                              std::string& err);
hankel_status general_backward(GeneralPlan* g, const void* gy, const void* h, const void* x, void* gh, void* gx,
                               cudaStream_t st, std::string& err);
void general_info(GeneralPlan* g, int64_t* jobs, int64_t* launches, int64_t* lengths, int64_t* ws_bytes);
void general_destroy(GeneralPlan* g);

}  // namespace hk
