// Library-internal entry points of the column model (not part of the C ABI).
#pragma once
#include <cuda_runtime_api.h>

namespace kktgb {

// Objective partial sums: part[b * stride] for b < nblocks (one per CTA of a
// fixed grid of nblocks CTAs of 256 threads); the caller sums them in a fixed
// order.  Returns false on bad parameters.
bool tray_objective_partials(const double* params, const double* d_w, double* d_part, int stride,
                             int nblocks, cudaStream_t stream);

}  // namespace kktgb
