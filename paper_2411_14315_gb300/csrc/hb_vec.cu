// Streaming vector kernels of the Krylov solver: conversions, axpy, Jacobi scaling, and the FP64
// reductions of the Arnoldi process (batched dot products and the fused update + norm of classical
// Gram-Schmidt).  All reductions are two-stage and deterministic: per-block partial sums in a caller
// scratch array, then one pass that sums the partials in a fixed order.
#include "hb_internal.cuh"

#include <algorithm>
#include <utility>

namespace hb {

namespace {

constexpr int kVB = 256;             // threads per block
constexpr int kMaxK = 256;           // largest number of simultaneous dot products

inline int nblk(int64_t n, int b) { return int((n + b - 1) / b); }

int sm_count() { return device_sms(); }

template <typename A, typename B>
__global__ void convert_kernel(const A *__restrict__ x, B *__restrict__ y, int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        y[i] = B(x[i]);
}

// FP32 copy of an FP64 state [node][4][N] with p_off subtracted from the pressure field
__global__ void convert_state_kernel(const double *__restrict__ y, float *__restrict__ y32, int64_t n, int N,
                                     double p_off) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const int f = int((i / N) & 3);
        y32[i] = float(f == 3 ? y[i] - p_off : y[i]);
    }
}

__global__ void axpy_kernel(double a, const double *__restrict__ x, double *__restrict__ y, int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        y[i] += a * x[i];
}

__global__ void scale_copy_kernel(double a, const double *__restrict__ x, double *__restrict__ y, int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        y[i] = a * x[i];
}

// z = x * dinv (right Jacobi preconditioning with the stored inverse diagonal), in z's precision
template <typename T>
__global__ void precond_kernel(const double *__restrict__ x, const double *__restrict__ dinv, T *__restrict__ z,
                               int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        z[i] = T(x[i] * dinv[i]);
}

__global__ void reciprocal_kernel(const double *d, double *dinv, int64_t n) {   // may run in place
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        dinv[i] = 1.0 / d[i];
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// partials[b * pstride + col0 + j] = this block's share of V_j . w (j < K) and partials[b * pstride + wcol]
// its share of w . w.  Each thread keeps one FP64 accumulator per basis vector in registers over its whole
// grid-stride range (K, the number of vectors, is a compile-time constant), so every element of w is read
// once and all K + 1 loads of an element are in flight together; the cross-thread sums happen once per
// block at the end.
template <int K>
__global__ void __launch_bounds__(kVB) multidot_kernel(const double *__restrict__ V, int64_t ld,
                                                       const double *__restrict__ w, int64_t n,
                                                       double *__restrict__ partials, int pstride, int col0,
                                                       int wcol, const int *gate) {
    if (gate && *gate == 0) return;
    __shared__ double sp[kVB / 32][K + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double acc[K + 1];
#pragma unroll
    for (int j = 0; j <= K; ++j) acc[j] = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * kVB + tid; i < n; i += int64_t(gridDim.x) * kVB) {
        const double wi = w[i];
#pragma unroll
        for (int j = 0; j < K; ++j) acc[j] = fma(V[int64_t(j) * ld + i], wi, acc[j]);
        acc[K] = fma(wi, wi, acc[K]);
    }
#pragma unroll
    for (int j = 0; j <= K; ++j) {
        const double t = warp_sum(acc[j]);
        if (lane == 0) sp[warp][j] = t;
    }
    __syncthreads();
    for (int j = tid; j <= K; j += kVB) {
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < kVB / 32; ++q) t += sp[q][j];
        partials[int64_t(blockIdx.x) * pstride + (j < K ? col0 + j : wcol)] = t;
    }
}

// result[j] = sum_b partials[b * stride + j] for j < cnt.  With a gate that is 0: zero_if_closed writes
// zeros, otherwise the result is left unchanged.
__global__ void finish_kernel(const double *__restrict__ partials, int nb, int stride, int cnt,
                              double *__restrict__ result, const int *gate = nullptr, int zero_if_closed = 0) {
    const int j = blockIdx.x;
    if (j >= cnt) return;
    if (gate && *gate == 0) {
        if (zero_if_closed && threadIdx.x == 0) result[j] = 0.0;
        return;
    }
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

// w -= sum_j h[j] V_j, then partials[b] = this block's share of ||w||^2 (two elements per thread step,
// so twice the loads are in flight)
__global__ void __launch_bounds__(kVB) multiaxpy_norm_kernel(const double *__restrict__ V, int64_t ld, int k,
                                                             const double *__restrict__ h, double *__restrict__ w,
                                                             int64_t n, double *__restrict__ partials,
                                                             const int *gate) {
    if (gate && *gate == 0) return;
    __shared__ double sh[kMaxK];
    __shared__ double red[kVB / 32];
    for (int j = threadIdx.x; j < k; j += kVB) sh[j] = h[j];
    __syncthreads();
    double s = 0.0;
    const int64_t stride = int64_t(gridDim.x) * kVB;
    for (int64_t i = int64_t(blockIdx.x) * kVB + threadIdx.x; i < n; i += 2 * stride) {
        const int64_t i2 = i + stride;
        const bool two = i2 < n;
        double x = w[i], x2 = two ? w[i2] : 0.0;
        for (int j = 0; j < k; ++j) {
            const double *vj = V + int64_t(j) * ld;
            x = fma(-sh[j], vj[i], x);
            if (two) x2 = fma(-sh[j], vj[i2], x2);
        }
        w[i] = x;
        s = fma(x, x, s);
        if (two) {
            w[i2] = x2;
            s = fma(x2, x2, s);
        }
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

// ---------------------------------------------------------------------------------------------------
// time-domain marching (generalized-alpha, one time level per node row of 4 values)

// out[r] = c0 + sum_k (c_{2k-1} cos k omega t + c_{2k} sin k omega t) for rows of real series
// [rows][2 n_h + 1]; the phase is reduced exactly through the period fraction frac = t / T mod 1
__global__ void series_at_kernel(const double *__restrict__ coef, int64_t rows, int n_h, double frac,
                                 double *__restrict__ out) {
    const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const double *c = coef + r * (2 * n_h + 1);
    double v = c[0];
    for (int k = 1; k <= n_h; ++k) {
        double f = double(k) * frac;
        f -= floor(f);
        double sn, cs;
        sincospi(2.0 * f, &sn, &cs);
        v += c[2 * k - 1] * cs + c[2 * k] * sn;
    }
    out[r] = v;
}

// predictor: u1 = un, du1 = (gamma - 1) / gamma dun (velocity; pressure rate unused)
__global__ void galpha_predict_kernel(const double *__restrict__ un, const double *__restrict__ dun,
                                      double *__restrict__ u1, double *__restrict__ du1, int64_t n, double cg) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    u1[i] = un[i];
    du1[i] = (i & 3) == 3 ? 0.0 : cg * dun[i];
}

// prescribed velocities at t_{n+1}: u1 = g, du1 = (g - un) / (gamma dt) + (gamma - 1) / gamma dun
__global__ void galpha_dirichlet_kernel(const int *__restrict__ nodes, int n_dir, const double *__restrict__ g,
                                        const double *__restrict__ un, const double *__restrict__ dun,
                                        double *__restrict__ u1, double *__restrict__ du1, double inv_gdt,
                                        double cg) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= 3 * n_dir) return;
    const int d = r / 3, i = r - 3 * d;
    const int64_t k = int64_t(nodes[d]) * 4 + i;
    u1[k] = g[r];
    du1[k] = (g[r] - un[k]) * inv_gdt + cg * dun[k];
}

// stage values: ya = un + af (u1 - un), dya = dun + am (du1 - dun)
__global__ void galpha_stage_kernel(const double *__restrict__ un, const double *__restrict__ u1,
                                    const double *__restrict__ dun, const double *__restrict__ du1,
                                    double *__restrict__ ya, double *__restrict__ dya, int64_t n, double af,
                                    double am) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    ya[i] = un[i] + af * (u1[i] - un[i]);
    dya[i] = dun[i] + am * (du1[i] - dun[i]);
}

// corrector: u1 += d, du1 += d / (gamma dt) on the velocity
__global__ void galpha_correct_kernel(double *__restrict__ u1, double *__restrict__ du1,
                                      const double *__restrict__ d, int64_t n, double inv_gdt) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    u1[i] += d[i];
    if ((i & 3) != 3) du1[i] += d[i] * inv_gdt;
}

// dst[node][f][k] = src[node][f] for one instance column k of an [n][4][N] array
__global__ void put_instance_kernel(const double *__restrict__ src, double *__restrict__ dst, int64_t n4, int k,
                                    int N) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n4) dst[i * N + k] = src[i];
}

// partials[b] = this block's share of sum over velocity entries (i mod 4 != 3) of x_i^2
__global__ void __launch_bounds__(kVB) vel_norm2_kernel(const double *__restrict__ x, int64_t n,
                                                        double *__restrict__ partials) {
    __shared__ double red[kVB / 32];
    double s = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * kVB + threadIdx.x; i < n; i += int64_t(gridDim.x) * kVB)
        if ((i & 3) != 3) s = fma(x[i], x[i], s);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < kVB / 32; ++q) t += red[q];
        partials[blockIdx.x] = t;
    }
}

// gate = 1 when classical Gram-Schmidt lost more than half of ||w||^2 (a second pass is needed)
__global__ void reorth_gate_kernel(const double *before2, const double *after2, int *gate) {
    *gate = (*after2 < 0.5 * *before2) ? 1 : 0;
}

// One Arnoldi column: h = h1 + h2 and ||w|| give column j of the Hessenberg matrix; apply the previous
// Givens rotations, form rotation j, update the rotated right-hand side g, record |g[j+1]| (the GMRES
// residual estimate) and 1 / ||w|| for the normalisation of the next basis vector.
__global__ void arnoldi_update_kernel(int j, int m, const double *__restrict__ h1, const double *__restrict__ h2,
                                      const double *__restrict__ nrm2, double *__restrict__ R,
                                      double *__restrict__ cs, double *__restrict__ sn, double *__restrict__ g,
                                      double *__restrict__ resid, double *__restrict__ invnorm) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double col[kMaxK + 1];
    for (int i = 0; i <= j; ++i) col[i] = h1[i] + h2[i];
    const double hn = sqrt(fmax(*nrm2, 0.0));
    col[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
        const double a0 = col[i], a1 = col[i + 1];
        col[i] = cs[i] * a0 + sn[i] * a1;
        col[i + 1] = -sn[i] * a0 + cs[i] * a1;
    }
    const double den = hypot(col[j], col[j + 1]);
    cs[j] = den > 0 ? col[j] / den : 1.0;
    sn[j] = den > 0 ? col[j + 1] / den : 0.0;
    col[j] = den;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    for (int i = 0; i <= j; ++i) R[i * m + j] = col[i];
    resid[j] = fabs(g[j + 1]);
    *invnorm = hn > 0 ? 1.0 / hn : 0.0;
}

// start of a restart cycle: beta = sqrt(beta2), g = (beta, 0, ...), invbeta = 1 / beta
__global__ void cycle_init_kernel(const double *beta2, int m, double *g, double *invbeta) {
    const int i = threadIdx.x;
    const double beta = sqrt(fmax(*beta2, 0.0));
    for (int k = i; k <= m; k += blockDim.x) g[k] = (k == 0) ? beta : 0.0;
    if (i == 0) *invbeta = beta > 0 ? 1.0 / beta : 0.0;
}

__global__ void scale_dev_kernel(const double *__restrict__ x, const double *__restrict__ sp, double *__restrict__ y,
                                 int64_t n) {
    const double a = *sp;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        y[i] = a * x[i];
}

int stream_grid(int64_t n) {
    const int cap = sm_count() * 8;
    const int need = nblk(n, kVB);
    return need < cap ? (need > 0 ? need : 1) : cap;
}

}  // namespace

// One full wave of multidot_kernel<K> (the grid-stride loop gives every block the same share, so a
// partial second wave would double the time), at most one block per 2048 elements.
template <int K>
int multidot_blocks(int64_t n) {
    static LaunchCache cache;
    const int cap = sm_count() * cached_blocks_per_sm(cache, multidot_kernel<K>, kVB, 0);
    const int need = nblk(n, kVB * 8);
    return need < cap ? (need > 0 ? need : 1) : cap;
}

// Partials of one tile of K vectors; returns the block count used.
template <int K>
int multidot_tile(const double *V, int64_t ld, const double *w, int64_t n, double *partials, int pstride,
                  int col0, int wcol, int nb, cudaStream_t s, const int *gate) {
    if (nb == 0) nb = multidot_blocks<K>(n);
    multidot_kernel<K><<<nb, kVB, 0, s>>>(V, ld, w, n, partials, pstride, col0, wcol, gate);
    return nb;
}

template <int... Ks>
int multidot_dispatch(std::integer_sequence<int, Ks...>, int k, const double *V, int64_t ld, const double *w,
                      int64_t n, double *partials, int pstride, int col0, int wcol, int nb, cudaStream_t s,
                      const int *gate) {
    int used = 0;
    ((k == Ks + 1 ? (used = multidot_tile<Ks + 1>(V, ld, w, n, partials, pstride, col0, wcol, nb, s, gate), 0)
                  : 0),
     ...);
    return used;
}

template <typename A, typename B>
void launch_convert(const A *x, B *y, int64_t n, cudaStream_t s) {
    if (n > 0) convert_kernel<A, B><<<stream_grid(n), kVB, 0, s>>>(x, y, n);
}

void launch_convert_state(const double *y, float *y32, int64_t n, int N, double p_off, cudaStream_t s) {
    if (n > 0) convert_state_kernel<<<stream_grid(n), kVB, 0, s>>>(y, y32, n, N, p_off);
}

void launch_axpy(double a, const double *x, double *y, int64_t n, cudaStream_t s) {
    if (n > 0) axpy_kernel<<<stream_grid(n), kVB, 0, s>>>(a, x, y, n);
}

void launch_scale_copy(double a, const double *x, double *y, int64_t n, cudaStream_t s) {
    if (n > 0) scale_copy_kernel<<<stream_grid(n), kVB, 0, s>>>(a, x, y, n);
}

template <typename T>
void launch_precond(const double *x, const double *dinv, T *z, int64_t n, cudaStream_t s) {
    if (n > 0) precond_kernel<T><<<stream_grid(n), kVB, 0, s>>>(x, dinv, z, n);
}

void launch_reciprocal(const double *d, double *dinv, int64_t n, cudaStream_t s) {
    if (n > 0) reciprocal_kernel<<<stream_grid(n), kVB, 0, s>>>(d, dinv, n);
}

void launch_multidot(const double *V, int64_t ld, int k, const double *w, int64_t n, double *partials,
                     double *result, cudaStream_t s, const int *gate) {
    // tiles of up to 32 vectors (w is read once per tile), all with the first tile's block count; every
    // tile also writes the same w . w column, computed identically
    int nb = 0;
    for (int j0 = 0; j0 < k; j0 += 32) {
        const int kt = k - j0 < 32 ? k - j0 : 32;
        nb = multidot_dispatch(std::make_integer_sequence<int, 32>{}, kt, V + int64_t(j0) * ld, ld, w, n, partials,
                               k + 1, j0, k, nb, s, gate);
    }
    finish_kernel<<<k + 1, 256, 0, s>>>(partials, nb, k + 1, k + 1, result, gate, 1);
}

void launch_multiaxpy_norm(const double *V, int64_t ld, int k, const double *h, double *w, int64_t n,
                           double *partials, double *result, cudaStream_t s, const int *gate) {
    static LaunchCache cache;                   // one full wave (equal shares per block)
    const int nb = std::min(stream_grid(n), sm_count() * cached_blocks_per_sm(cache, multiaxpy_norm_kernel, kVB, 0));
    multiaxpy_norm_kernel<<<nb, kVB, 0, s>>>(V, ld, k, h, w, n, partials, gate);
    finish_kernel<<<1, 256, 0, s>>>(partials, nb, 1, 1, result, gate, 0);
}

void launch_reorth_gate(const double *before2, const double *after2, int *gate, cudaStream_t s) {
    reorth_gate_kernel<<<1, 1, 0, s>>>(before2, after2, gate);
}

void launch_arnoldi_update(int j, int m, const double *h1, const double *h2, const double *nrm2, double *R,
                           double *cs, double *sn, double *g, double *resid, double *invnorm, cudaStream_t s) {
    arnoldi_update_kernel<<<1, 32, 0, s>>>(j, m, h1, h2, nrm2, R, cs, sn, g, resid, invnorm);
}

void launch_cycle_init(const double *beta2, int m, double *g, double *invbeta, cudaStream_t s) {
    cycle_init_kernel<<<1, 256, 0, s>>>(beta2, m, g, invbeta);
}

void launch_scale_dev(const double *x, const double *sp, double *y, int64_t n, cudaStream_t s) {
    if (n > 0) scale_dev_kernel<<<stream_grid(n), kVB, 0, s>>>(x, sp, y, n);
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

void launch_series_at(const double *coef, int64_t rows, int n_h, double frac, double *out, cudaStream_t s) {
    if (rows > 0) series_at_kernel<<<nblk(rows, 128), 128, 0, s>>>(coef, rows, n_h, frac, out);
}

void launch_galpha_predict(const double *un, const double *dun, double *u1, double *du1, int64_t n, double cg,
                           const int *dir_nodes, int n_dir, const double *g, double inv_gdt, cudaStream_t s) {
    if (n > 0) galpha_predict_kernel<<<nblk(n, kVB), kVB, 0, s>>>(un, dun, u1, du1, n, cg);
    if (n_dir > 0)
        galpha_dirichlet_kernel<<<nblk(int64_t(3) * n_dir, kVB), kVB, 0, s>>>(dir_nodes, n_dir, g, un, dun, u1, du1,
                                                                              inv_gdt, cg);
}

void launch_galpha_stage(const double *un, const double *u1, const double *dun, const double *du1, double *ya,
                         double *dya, int64_t n, double af, double am, cudaStream_t s) {
    if (n > 0) galpha_stage_kernel<<<nblk(n, kVB), kVB, 0, s>>>(un, u1, dun, du1, ya, dya, n, af, am);
}

void launch_galpha_correct(double *u1, double *du1, const double *d, int64_t n, double inv_gdt, cudaStream_t s) {
    if (n > 0) galpha_correct_kernel<<<nblk(n, kVB), kVB, 0, s>>>(u1, du1, d, n, inv_gdt);
}

void launch_put_instance(const double *src, double *dst, int64_t n4, int k, int N, cudaStream_t s) {
    if (n4 > 0) put_instance_kernel<<<nblk(n4, kVB), kVB, 0, s>>>(src, dst, n4, k, N);
}

void launch_vel_norm2(const double *x, int64_t n, double *partials, double *result, cudaStream_t s) {
    const int nb = stream_grid(n);
    vel_norm2_kernel<<<nb, kVB, 0, s>>>(x, n, partials);
    finish_kernel<<<1, 256, 0, s>>>(partials, nb, 1, 1, result);
}

template void launch_convert<double, float>(const double *, float *, int64_t, cudaStream_t);
template void launch_convert<float, double>(const float *, double *, int64_t, cudaStream_t);
template void launch_convert<double, double>(const double *, double *, int64_t, cudaStream_t);
template void launch_convert<float, float>(const float *, float *, int64_t, cudaStream_t);
template void launch_precond<float>(const double *, const double *, float *, int64_t, cudaStream_t);
template void launch_precond<double>(const double *, const double *, double *, int64_t, cudaStream_t);

}  // namespace hb
