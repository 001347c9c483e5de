// Internal helpers of api.cu used by other translation units.
#pragma once

#include "../../include/mirage.h"
#include "kernels.cuh"
#include "table.h"

namespace mirage {
const KernelTable& kernel_table();
int geometry_ok(const mirage_geom_t& g);
template <typename T>
Prob<T> problem_layout(const mirage_problem_t& p);
}  // namespace mirage
