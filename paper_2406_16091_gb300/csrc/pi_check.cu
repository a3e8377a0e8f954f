// pi_check.cu -- FP64 totals of per-particle outputs, for the invariant
// checks (every within-cutoff pair is seen from both sides, so the vector
// sums V_i over all particles of a system total zero up to rounding).
//
// The only FP64 arithmetic on the GPU: two launches with a fixed reduction
// order (no atomics), so the result is the same on every run.
#include "pi_internal.cuh"

namespace pi {

namespace {

constexpr int TOTAL_THREADS = 256;

// Block (s, g) sums the g-th of TOTAL_PARTS interleaved slices of system s.
__global__ void __launch_bounds__(TOTAL_THREADS) k_total_partial(const float* __restrict__ v,
                                                                 Systems sy,
                                                                 double* __restrict__ partial)
{
    __shared__ double red[TOTAL_THREADS];
    const int s = blockIdx.x, g = blockIdx.y;
    const uint32_t p0 = sy.pbase[s], p1 = sy.pbase[s + 1];
    double acc = 0.0;
    for (uint32_t i = p0 + (uint32_t)g * TOTAL_THREADS + threadIdx.x; i < p1;
         i += (uint32_t)gridDim.y * TOTAL_THREADS)
        acc += (double)v[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = TOTAL_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[(size_t)s * gridDim.y + g] = red[0];
}

__global__ void k_total_final(const double* __restrict__ partial, int parts, int S,
                              double* __restrict__ out)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int g = 0; g < parts; ++g) acc += partial[(size_t)s * parts + g];
        out[s] = acc;
    }
}

}  // namespace

cudaError_t launch_total_f64(const float* v, const Systems& sy, double* partial, int parts,
                             double* out, cudaStream_t s)
{
    k_total_partial<<<dim3((unsigned)sy.S, (unsigned)parts), TOTAL_THREADS, 0, s>>>(v, sy, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_total_final<<<(sy.S + 127) / 128, 128, 0, s>>>(partial, parts, sy.S, out);
    return cudaGetLastError();
}

}  // namespace pi
