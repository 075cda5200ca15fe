// Library-internal entry points of the column model (not part of the C ABI).
#pragma once
#include <cuda_runtime_api.h>

#include "kkt.h"

namespace kktgb {

// Objective partial sums: part[b * stride] for b < nblocks (one per CTA of a
// fixed grid of nblocks CTAs of 256 threads); the caller sums them in a fixed
// order.  Returns false on bad parameters.
bool tray_objective_partials(const double* params, const double* d_w, double* d_part, int stride,
                             int nblocks, cudaStream_t stream);

// kkt_tray_eval with an optional per-tray initial state d_x0[k] (device;
// NULL: x0bar of the parameters on every tray) in the stage-0 rows.
kkt_status tray_eval(const double* params, const double* d_x0, const double* d_w, const double* d_lam,
                     double obj_weight, double* d_f, double* d_grad, double* d_c, double* d_Jval,
                     double* d_Wval, cudaStream_t stream);

}  // namespace kktgb
