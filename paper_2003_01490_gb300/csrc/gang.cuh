// gang.cuh -- one launch of a kernel over many independent instances (the
// boxes of a batch): the launch's blocks are the instances' own grids laid end
// to end, off[i] .. off[i + 1] - 1 for instance i (off: n + 1 prefix sums of
// the block counts), and each block copies its instance's parameter block
// from the table into shared memory and runs the kernel's body with its block
// index within that instance's grid. The bodies are the single-instance
// kernels' code, so an instance computes in a gang launch what it computes
// alone.
#pragma once

#include <cuda_runtime.h>

namespace lbmdem {

// instance of launch block b: the largest i with off[i] <= b
__device__ __forceinline__ int gang_instance(const int* __restrict__ off, int n, int b) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// the parameter block of instance i into shared memory (all threads of the
// block take part; ends with a barrier)
template <typename P>
__device__ __forceinline__ void gang_load(const P* __restrict__ table, int i, P& sp) {
    static_assert(sizeof(P) % 4 == 0, "parameter blocks are copied in words");
    const int* src = reinterpret_cast<const int*>(table + i);
    int* dst = reinterpret_cast<int*>(&sp);
    const int nthreads = (int)(blockDim.x * blockDim.y * blockDim.z);
    const int t = (int)(threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z));
    for (int w = t; w < (int)(sizeof(P) / 4); w += nthreads) dst[w] = src[w];
    __syncthreads();
}

}  // namespace lbmdem
