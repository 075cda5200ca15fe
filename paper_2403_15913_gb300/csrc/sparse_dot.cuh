// Row-times-vector gathers of the sparse products (W v, J x, J^T y).  Each
// entry needs two dependent loads (its index, then the values), so a loop
// that finishes one entry before loading the next pays that latency once per
// entry.  These helpers issue the index loads of four entries, then their
// value loads, then the four FMAs in the original order: the same rounded
// result, one latency per four entries.
#pragma once
#include <cuda_runtime.h>

namespace kktgb {

constexpr int kGatherBatch = 4;

// s + sum_{q in [q0, q1)} A[idx[q]] * v[col[q]]
__device__ __forceinline__ double gather_dot(int q0, int q1, const int* __restrict__ idx,
                                             const int* __restrict__ col, const double* __restrict__ A,
                                             const double* __restrict__ v, double s) {
    for (int q = q0; q < q1; q += kGatherBatch) {
        int ia[kGatherBatch], ic[kGatherBatch];
#pragma unroll
        for (int u = 0; u < kGatherBatch; ++u) {
            const bool ok = q + u < q1;
            ia[u] = ok ? idx[q + u] : 0;
            ic[u] = ok ? col[q + u] : 0;
        }
        double a[kGatherBatch], b[kGatherBatch];
#pragma unroll
        for (int u = 0; u < kGatherBatch; ++u) {
            const bool ok = q + u < q1;
            a[u] = ok ? A[ia[u]] : 0.0;
            b[u] = ok ? v[ic[u]] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kGatherBatch; ++u)
            if (q + u < q1) s = fma(a[u], b[u], s);
    }
    return s;
}

// s + sum_{q in [q0, q1)} A[q] * v[col[q]]   (values stored in entry order)
__device__ __forceinline__ double gather_dot_direct(int q0, int q1, const int* __restrict__ col,
                                                    const double* __restrict__ A,
                                                    const double* __restrict__ v, double s) {
    for (int q = q0; q < q1; q += kGatherBatch) {
        int ic[kGatherBatch];
        double a[kGatherBatch];
#pragma unroll
        for (int u = 0; u < kGatherBatch; ++u) {
            const bool ok = q + u < q1;
            ic[u] = ok ? col[q + u] : 0;
            a[u] = ok ? A[q + u] : 0.0;
        }
        double b[kGatherBatch];
#pragma unroll
        for (int u = 0; u < kGatherBatch; ++u) b[u] = q + u < q1 ? v[ic[u]] : 0.0;
#pragma unroll
        for (int u = 0; u < kGatherBatch; ++u)
            if (q + u < q1) s = fma(a[u], b[u], s);
    }
    return s;
}

}  // namespace kktgb
