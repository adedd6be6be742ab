// Streaming vector kernels of the Krylov solver: conversions, axpy, Jacobi scaling, and the FP64
// reductions of the Arnoldi process (batched dot products and the fused update + norm of classical
// Gram-Schmidt).  All reductions are two-stage and deterministic: per-block partial sums in a caller
// scratch array, then one pass that sums the partials in a fixed order.
#include "hb_internal.cuh"

namespace hb {

namespace {

constexpr int kVB = 256;             // threads per block
constexpr int kChunk = kVB * 8;      // vector elements per block-chunk in the batched dot
constexpr int kMaxK = 256;           // largest number of simultaneous dot products

inline int nblk(int64_t n, int b) { return int((n + b - 1) / b); }

int g_sm_count = 0;
int sm_count() {
    if (g_sm_count == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (g_sm_count <= 0) g_sm_count = 148;
    }
    return g_sm_count;
}

template <typename A, typename B>
__global__ void convert_kernel(const A *__restrict__ x, B *__restrict__ y, int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        y[i] = B(x[i]);
}

__global__ void axpy_kernel(double a, const double *__restrict__ x, double *__restrict__ y, int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        y[i] += a * x[i];
}

__global__ void scale_copy_kernel(double a, const double *__restrict__ x, double *__restrict__ y, int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        y[i] = a * x[i];
}

template <typename T>
__global__ void precond_kernel(const double *__restrict__ x, const double *__restrict__ d, T *__restrict__ z,
                               int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        z[i] = T(x[i] / d[i]);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// partials[b * (k+1) + j] = sum over this block's chunks of V_j . w (j < k) and w . w (j = k)
__global__ void __launch_bounds__(kVB) multidot_kernel(const double *__restrict__ V, int64_t ld, int k,
                                                       const double *__restrict__ w, int64_t n,
                                                       double *__restrict__ partials) {
    __shared__ double sw[kChunk];
    __shared__ double sp[kVB / 32][kMaxK + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int j = tid; j < (kVB / 32) * (kMaxK + 1); j += kVB) (&sp[0][0])[j] = 0.0;
    __syncthreads();
    for (int64_t c0 = int64_t(blockIdx.x) * kChunk; c0 < n; c0 += int64_t(gridDim.x) * kChunk) {
        const int m = int(n - c0 < kChunk ? n - c0 : kChunk);
        for (int t = tid; t < kChunk; t += kVB) sw[t] = t < m ? w[c0 + t] : 0.0;
        __syncthreads();
        for (int j = 0; j <= k; ++j) {
            double s = 0.0;
            if (j < k) {
                const double *v = V + int64_t(j) * ld + c0;
#pragma unroll
                for (int t = 0; t < kChunk / kVB; ++t) {
                    const int idx = tid + t * kVB;
                    if (idx < m) s += v[idx] * sw[idx];
                }
            } else {
#pragma unroll
                for (int t = 0; t < kChunk / kVB; ++t) {
                    const int idx = tid + t * kVB;
                    s += sw[idx] * sw[idx];
                }
            }
            s = warp_sum(s);
            if (lane == 0) sp[warp][j] += s;
        }
        __syncthreads();
    }
    for (int j = tid; j <= k; j += kVB) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < kVB / 32; ++q) s += sp[q][j];
        partials[int64_t(blockIdx.x) * (k + 1) + j] = s;
    }
}

// result[j] = sum_b partials[b * stride + j] for j < cnt
__global__ void finish_kernel(const double *__restrict__ partials, int nb, int stride, int cnt,
                              double *__restrict__ result) {
    const int j = blockIdx.x;
    if (j >= cnt) return;
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += partials[int64_t(b) * stride + j];
    __shared__ double red[32];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0) result[j] = t;
    }
}

// w -= sum_j h[j] V_j, then partials[b] = this block's share of ||w||^2
__global__ void __launch_bounds__(kVB) multiaxpy_norm_kernel(const double *__restrict__ V, int64_t ld, int k,
                                                             const double *__restrict__ h, double *__restrict__ w,
                                                             int64_t n, double *__restrict__ partials) {
    __shared__ double sh[kMaxK];
    __shared__ double red[kVB / 32];
    for (int j = threadIdx.x; j < k; j += kVB) sh[j] = h[j];
    __syncthreads();
    double s = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * kVB + threadIdx.x; i < n; i += int64_t(gridDim.x) * kVB) {
        double x = w[i];
        for (int j = 0; j < k; ++j) x -= sh[j] * V[int64_t(j) * ld + i];
        w[i] = x;
        s += x * x;
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < kVB / 32; ++q) t += red[q];
        partials[blockIdx.x] = t;
    }
}

__global__ void combine_kernel(const double *__restrict__ V, int64_t ld, int k, const double *__restrict__ c,
                               double *__restrict__ y, int64_t n) {
    __shared__ double sc[kMaxK];
    for (int j = threadIdx.x; j < k; j += blockDim.x) sc[j] = c[j];
    __syncthreads();
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        double x = 0.0;
        for (int j = 0; j < k; ++j) x += sc[j] * V[int64_t(j) * ld + i];
        y[i] = x;
    }
}

__global__ void __launch_bounds__(kVB) dot_kernel(const double *__restrict__ x, const double *__restrict__ y,
                                                  int64_t n, double *__restrict__ partials) {
    __shared__ double red[kVB / 32];
    double s = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * kVB + threadIdx.x; i < n; i += int64_t(gridDim.x) * kVB) s += x[i] * y[i];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < kVB / 32; ++q) t += red[q];
        partials[blockIdx.x] = t;
    }
}

int stream_grid(int64_t n) {
    const int cap = sm_count() * 8;
    const int need = nblk(n, kVB);
    return need < cap ? (need > 0 ? need : 1) : cap;
}

}  // namespace

int multidot_blocks(int64_t n) {
    const int cap = sm_count() * 2;
    const int need = nblk(n, kChunk);
    return need < cap ? (need > 0 ? need : 1) : cap;
}

template <typename A, typename B>
void launch_convert(const A *x, B *y, int64_t n, cudaStream_t s) {
    if (n > 0) convert_kernel<A, B><<<stream_grid(n), kVB, 0, s>>>(x, y, n);
}

void launch_axpy(double a, const double *x, double *y, int64_t n, cudaStream_t s) {
    if (n > 0) axpy_kernel<<<stream_grid(n), kVB, 0, s>>>(a, x, y, n);
}

void launch_scale_copy(double a, const double *x, double *y, int64_t n, cudaStream_t s) {
    if (n > 0) scale_copy_kernel<<<stream_grid(n), kVB, 0, s>>>(a, x, y, n);
}

template <typename T>
void launch_precond(const double *x, const double *d, T *z, int64_t n, cudaStream_t s) {
    if (n > 0) precond_kernel<T><<<stream_grid(n), kVB, 0, s>>>(x, d, z, n);
}

void launch_multidot(const double *V, int64_t ld, int k, const double *w, int64_t n, double *partials,
                     double *result, cudaStream_t s) {
    const int nb = multidot_blocks(n);
    multidot_kernel<<<nb, kVB, 0, s>>>(V, ld, k, w, n, partials);
    finish_kernel<<<k + 1, 256, 0, s>>>(partials, nb, k + 1, k + 1, result);
}

void launch_multiaxpy_norm(const double *V, int64_t ld, int k, const double *h, double *w, int64_t n,
                           double *partials, double *result, cudaStream_t s) {
    const int nb = stream_grid(n);
    multiaxpy_norm_kernel<<<nb, kVB, 0, s>>>(V, ld, k, h, w, n, partials);
    finish_kernel<<<1, 256, 0, s>>>(partials, nb, 1, 1, result);
}

void launch_combine(const double *V, int64_t ld, int k, const double *c, double *y, int64_t n,
                    cudaStream_t s) {
    if (n > 0) combine_kernel<<<stream_grid(n), kVB, 0, s>>>(V, ld, k, c, y, n);
}

void launch_dot(const double *x, const double *y, int64_t n, double *partials, double *result,
                cudaStream_t s) {
    const int nb = stream_grid(n);
    dot_kernel<<<nb, kVB, 0, s>>>(x, y, n, partials);
    finish_kernel<<<1, 256, 0, s>>>(partials, nb, 1, 1, result);
}

template void launch_convert<double, float>(const double *, float *, int64_t, cudaStream_t);
template void launch_convert<float, double>(const float *, double *, int64_t, cudaStream_t);
template void launch_precond<float>(const double *, const double *, float *, int64_t, cudaStream_t);
template void launch_precond<double>(const double *, const double *, double *, int64_t, cudaStream_t);

}  // namespace hb
