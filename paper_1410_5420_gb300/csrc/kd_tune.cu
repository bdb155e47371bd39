// kd_tune.cu -- synthetic clouds for the autotuner.
//
// kd_autotune (kd_api.cu) times candidate build parameters on a cloud of the
// requested size, k and dtype.  This kernel fills that cloud on the device
// from a counter-based generator: value i is the splitmix64 output
// (Steele, Lea and Flood, OOPSLA 2014) of seed + (i + 1) * golden gamma,
// mapped to float32 uniform in [0, 1) (24-bit draws), int32 uniform in
// [0, 2^24) or int64 uniform in [0, 2^40).  It holds none of the tree
// build's arithmetic: the timings only need a cloud of the right shape.
#include <cstdint>

#include <cuda_runtime.h>

namespace kd {

__device__ __forceinline__ uint64_t tune_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void __launch_bounds__(256) k_tune_cloud(int dtype, void* __restrict__ out, int64_t count, uint64_t seed) {
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < count; i += (int64_t)gridDim.x * 256) {
        const uint64_t r = tune_mix(seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull);
        if (dtype == 0)
            static_cast<int32_t*>(out)[i] = (int32_t)(r >> 40);
        else if (dtype == 1)
            static_cast<int64_t*>(out)[i] = (int64_t)(r >> 24);
        else
            static_cast<float*>(out)[i] = (float)(r >> 40) * (1.0f / 16777216.0f);
    }
}

cudaError_t launch_tune_cloud(int dtype, void* coords, int64_t count, uint64_t seed, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    int64_t g = (count + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    k_tune_cloud<<<(unsigned)g, 256, 0, s>>>(dtype, coords, count, seed);
    return cudaGetLastError();
}

}  // namespace kd
