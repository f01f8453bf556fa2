// FP64 instantiations of the Roe-AM kernels.
#include "roeam_kernels.cuh"

namespace roeam {
extern template struct AblationLaunchers<double>;   // in roeam_k64_abl.cu
template struct Launchers<double>;

// Fixed-order reduction of nblocks rows of `width` partials (first half sums, second half
// maxima when width == 8; all sums when width == 4) into out[width]. One warp per column.
__global__ void reduce_partials_kernel(const double *partials, int nblocks, int width, double *out)
{
    const int k = blockIdx.x;
    const bool is_max = width == 8 && k >= 4;
    double v = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 32) {
        const double x = partials[(size_t)b * width + k];
        v = is_max ? fmax(v, x) : v + x;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double x = __shfl_xor_sync(0xffffffffu, v, o);
        v = is_max ? fmax(v, x) : v + x;
    }
    if (threadIdx.x == 0) out[k] = v;
}

// The library's reciprocal, reciprocal square root and square root on n values, in FP64 and
// in FP32 (of the values rounded to float): out holds n rows of 6.
__global__ void math_check_kernel(int n, const double *x, double *out)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const double v = x[k];
        const float f = (float)v;
        out[6 * k + 0] = rcp(v);
        out[6 * k + 1] = rsq(v);
        out[6 * k + 2] = sqrt0(v);
        out[6 * k + 3] = (double)rcp(f);
        out[6 * k + 4] = (double)rsq(f);
        out[6 * k + 5] = (double)sqrt0(f);
    }
}

cudaError_t launch_math_check(int n, const double *x, double *out, cudaStream_t s)
{
    math_check_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, x, out);
    return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const double *partials, int nblocks, int width, double *out, cudaStream_t s)
{
    reduce_partials_kernel<<<width, 32, 0, s>>>(partials, nblocks, width, out);
    return cudaGetLastError();
}
}  // namespace roeam
