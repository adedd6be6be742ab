// Boundary and time-series kernels of libhbgls: Neumann faces (traction and backflow stabilisation,
// Sec. 2.3), resistance-outlet flow rates, sampling of boundary waveforms at the
// instances (Eqs. upgh_def, upghharm) and the real discrete Fourier transforms of the state
// (Eq. upghdft; reconstruction of Sec. 3.2).
#include "hb_internal.cuh"

namespace hb {

namespace {

// ---------------------------------------------------------------------------------------------------
// Neumann faces: -int N_A h n_i and backflow -int N_A (rho/2) beta |u.n|_- u_i (3 edge midpoints)

// Outlet flow rates Q[o][n] += sum over the outlet's faces of (S/3) sum_b x_b . n (Q cleared by the
// caller).  Grid: (face chunks of 256) x (instances); one face per thread, outlets in groups of 8,
// warp-shuffle and shared-memory reduction, one global atomic per block, outlet and instance.
template <typename T, int MODE>
__global__ void outlet_flux_kernel(FaceArgs<T> a, int n_out) {
    constexpr int G = 8;
    __shared__ T acc[G];
    const int n = blockIdx.y, N4 = 4 * a.N, lane = threadIdx.x & 31;
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    const T *x = (MODE == MODE_RES) ? a.y : a.v;
    int o = -1;
    T s = 0;
    if (f < a.n_faces) {
        o = a.foutlet[f];
        if (o >= 0) {
            const T nx = a.fgeo[4 * f], ny = a.fgeo[4 * f + 1], nz = a.fgeo[4 * f + 2], S = a.fgeo[4 * f + 3];
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const int nd = a.fnodes[3 * f + b];
                if (MODE != MODE_RES && (a.flag[nd] & 1)) continue;
                const T *r = x + size_t(nd) * N4 + n;
                s += r[0] * nx + r[a.N] * ny + r[2 * a.N] * nz;
            }
            s *= S / T(3);
        }
    }
    for (int o0 = 0; o0 < n_out; o0 += G) {
        if (threadIdx.x < G) acc[threadIdx.x] = T(0);
        __syncthreads();
#pragma unroll
        for (int g = 0; g < G; ++g) {
            T v = (o == o0 + g) ? s : T(0);
            for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
            if (lane == 0 && v != T(0)) atomicAdd(acc + g, v);
        }
        __syncthreads();
        if (threadIdx.x < G && o0 + threadIdx.x < n_out && acc[threadIdx.x] != T(0))
            atomicAdd(a.Q + (o0 + threadIdx.x) * a.N + n, acc[threadIdx.x]);
        __syncthreads();
    }
}

// Deterministic flow rates: one block of kFluxThreads per (outlet, instance); thread j sums the outlet's
// faces j, j + kFluxThreads, ... in list order and a fixed tree combines the threads; Q is written, not
// accumulated.
constexpr int kFluxThreads = 256;
template <typename T, int MODE>
__global__ void __launch_bounds__(kFluxThreads) outlet_flux_det_kernel(FaceArgs<T> a) {
    __shared__ T red[kFluxThreads];
    const int o = blockIdx.x, n = blockIdx.y, lane = threadIdx.x, N4 = 4 * a.N;
    const T *x = (MODE == MODE_RES) ? a.y : a.v;
    T s = 0;
    for (int j = a.optr[o] + lane; j < a.optr[o + 1]; j += kFluxThreads) {
        const int f = a.oface[j];
        const T nx = a.fgeo[4 * f], ny = a.fgeo[4 * f + 1], nz = a.fgeo[4 * f + 2], S = a.fgeo[4 * f + 3];
        T sf = 0;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int nd = a.fnodes[3 * f + b];
            if (MODE != MODE_RES && (a.flag[nd] & 1)) continue;
            const T *r = x + size_t(nd) * N4 + n;
            sf += r[0] * nx + r[a.N] * ny + r[2 * a.N] * nz;
        }
        s += sf * (S / T(3));
    }
    red[lane] = s;
    __syncthreads();
    for (int w = kFluxThreads / 2; w > 0; w >>= 1) {
        if (lane < w) red[lane] += red[lane + w];
        __syncthreads();
    }
    if (lane == 0) a.Q[o * a.N + n] = red[0];
}

template <typename T, int MODE>
__global__ void face_kernel(FaceArgs<T> a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_faces * a.N) return;
    const int N = a.N, N4 = 4 * N;
    const int f = i / N, n = i - f * N;
    const T nrm[3] = {a.fgeo[4 * f], a.fgeo[4 * f + 1], a.fgeo[4 * f + 2]};
    const T S3 = a.fgeo[4 * f + 3] / T(3);
    int nd[3];
    T u[3][3], v[3][3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        nd[b] = a.fnodes[3 * f + b];
        const T *r = a.y + size_t(nd[b]) * N4 + n;
#pragma unroll
        for (int k = 0; k < 3; ++k) u[b][k] = r[k * N];
        if (MODE != MODE_RES) {
            const bool dir = a.flag[nd[b]] & 1;
            const T *rv = a.v + size_t(nd[b]) * N4 + n;
#pragma unroll
            for (int k = 0; k < 3; ++k) v[b][k] = dir ? T(0) : rv[k * N];
        }
    }
    const int o = a.foutlet[f];
    T h = 0;
    if (o >= 0) {
        if (MODE == MODE_RES) h = a.hbase[o * N + n] - a.R[o] * a.Q[o * N + n];
        else h = -a.R[o] * a.Q[o * N + n];
    }
    T c[3][3];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int k = 0; k < 3; ++k) c[b][k] = -S3 * h * nrm[k];
    const T cb = -S3 * T(0.5) * (T(0.5) * a.rho * a.beta);
    const int e0[3] = {0, 1, 0}, e1[3] = {1, 2, 2};
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        T um[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) um[k] = T(0.5) * (u[e0[m]][k] + u[e1[m]][k]);
        const T s = um[0] * nrm[0] + um[1] * nrm[1] + um[2] * nrm[2];
        const T sm = s < T(0) ? s : T(0);
        T term[3];
        if (MODE == MODE_RES) {
#pragma unroll
            for (int k = 0; k < 3; ++k) term[k] = sm * um[k];
        } else {
            T vm[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) vm[k] = T(0.5) * (v[e0[m]][k] + v[e1[m]][k]);
            const T vn = (MODE == MODE_JVE && s < T(0)) ? vm[0] * nrm[0] + vm[1] * nrm[1] + vm[2] * nrm[2] : T(0);
#pragma unroll
            for (int k = 0; k < 3; ++k) term[k] = sm * vm[k] + vn * um[k];
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            c[e0[m]][k] += cb * term[k];
            c[e1[m]][k] += cb * term[k];
        }
    }
    if (a.fbuf) {                              // deterministic scatter: the face's own slots
        T *fs = a.fbuf + size_t(f) * 9 * N + n;
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int k = 0; k < 3; ++k) fs[(3 * b + k) * N] = c[b][k];
        return;
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        if (a.flag[nd[b]] & 1) continue;       // prescribed velocity rows are set by the element pass
#pragma unroll
        for (int k = 0; k < 3; ++k) atomicAdd(a.out + size_t(nd[b]) * N4 + k * N + n, c[b][k]);
    }
}

// Deterministic gather of the element and face slots, one thread per (node, field, instance): fields
// 0-3 go to out (prescribed velocity rows: a.presc), fields 4-6 (F = 7) sum T into tbuf; F = 3 adds the
// face slots alone to the velocity rows of out.
template <typename T>
__global__ void det_gather_kernel(DetGatherArgs<T> a) {
    const int N = a.N, F = a.F;
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= a.n_nodes * F * N) return;
    const int64_t A = t / (int64_t(F) * N);
    const int r = int(t - A * F * N), f = r / N, n = r - f * N;
    if (F == 3) {                  // faces only, added to a product written before (assembled operator)
        if (a.flag[A] & 1) return;
        T s = 0;
        for (int k = a.fptr[A]; k < a.fptr[A + 1]; ++k) s += a.fbuf[(size_t(a.fslot[k]) * 3 + f) * N + n];
        a.out[A * 4 * N + r] += s;
        return;
    }
    const bool presc = (a.flag[A] & 1) && (f < 3 || f >= 4);
    T s = 0;
    if (presc) {
        if (f < 3) s = a.presc == 2 ? a.v[A * 4 * N + r] : T(a.presc == 1 ? 1 : 0);
    } else {
        // eight slot indices, then eight slot values in flight at a time; the additions keep the list order
        constexpr int U = 8;
        const int k0 = a.eptr[A], k1 = a.eptr[A + 1];
        for (int k = k0; k < k1; k += U) {
            int e[U];
#pragma unroll
            for (int j = 0; j < U; ++j) e[j] = k + j < k1 ? __ldg(a.eslot + k + j) : -1;
            T x[U];
#pragma unroll
            for (int j = 0; j < U; ++j) x[j] = e[j] >= 0 ? __ldg(a.cbuf + (size_t(e[j]) * F + f) * N + n) : T(0);
#pragma unroll
            for (int j = 0; j < U; ++j)
                if (k + j < k1) s += x[j];
        }
        if (a.fptr && f < 3)
            for (int k = a.fptr[A]; k < a.fptr[A + 1]; ++k) s += a.fbuf[(size_t(a.fslot[k]) * 3 + f) * N + n];
    }
    if (f < 4) a.out[A * 4 * N + r] = s;
    else a.tbuf[(A * 3 + (f - 4)) * N + n] = s;
}

// out[A][i][n] += sum_k H[n][k] tbuf[A][i][k] on free velocity rows (F = 7)
template <typename T>
__global__ void det_apply_h_kernel(DetGatherArgs<T> a) {
    const int N = a.N;
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= a.n_nodes * 3 * N) return;
    const int64_t A = t / (3 * N);
    if (a.flag[A] & 1) return;
    const int r = int(t - A * 3 * N), i = r / N, n = r - i * N;
    const T *h = a.H + size_t(n) * N, *x = a.tbuf + (A * 3 + i) * N;
    T s = 0;
    for (int k = 0; k < N; ++k) s += h[k] * x[k];
    a.out[A * 4 * N + i * N + n] += s;
}

// ---------------------------------------------------------------------------------------------------
// boundary-condition sampling and harmonic transforms (Eqs. upgh_def, upghdft)

// angle 2 pi k n / N reduced exactly to [0, 2 pi) through (k n mod N)
__device__ __forceinline__ void cos_sin_kn(int k, int n, int N, double &c, double &s) {
    const int r = int((long long)k * n % N);
    sincospi(2.0 * double(r) / double(N), &s, &c);
}

__global__ void sample_waveforms_kernel(const double *__restrict__ coef, int n_wave, int n_h, int N,
                                        double *__restrict__ W) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_wave * N) return;
    const int w = i / N, n = i - w * N;
    const double *c = coef + size_t(w) * (2 * n_h + 1);
    double q = c[0];
    for (int k = 1; k <= n_h; ++k) {
        double cs, sn;
        cos_sin_kn(k, n, N, cs, sn);
        q += c[2 * k - 1] * cs + c[2 * k] * sn;
    }
    W[i] = q;
}

__global__ void apply_dirichlet_kernel(const int *__restrict__ dir_nodes, int n_dir,
                                       const double *__restrict__ g, double *__restrict__ y, int N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_dir * 3 * N) return;
    const int d = i / (3 * N), r = i - d * 3 * N;
    y[size_t(dir_nodes[d]) * 4 * N + r] = g[i];
}

// inverse = 0: coef[row][m] from y[row][n] (a0, a_k = 2/N sum y cos, b_k = 2/N sum y sin)
// inverse = 1: y[row][n] from coef[row][m]
__global__ void harmonics_kernel(const double *__restrict__ in, double *__restrict__ out, int64_t rows,
                                 int N, int n_h) {
    const int M = 2 * n_h + 1;
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= rows * M) return;
    const int64_t row = i / M;
    const int m = int(i - row * M);
    const double *y = in + row * N;
    double acc = 0.0;
    if (m == 0) {
        for (int n = 0; n < N; ++n) acc += y[n];
        acc /= double(N);
    } else {
        const int k = (m + 1) / 2;
        const bool is_sin = (m % 2) == 0;
        for (int n = 0; n < N; ++n) {
            double cs, sn;
            cos_sin_kn(k, n, N, cs, sn);
            acc += y[n] * (is_sin ? sn : cs);
        }
        acc *= 2.0 / double(N);
    }
    out[i] = acc;
}

__global__ void synthesis_kernel(const double *__restrict__ coef, double *__restrict__ y, int64_t rows,
                                 int N, int n_h) {
    const int M = 2 * n_h + 1;
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= rows * N) return;
    const int64_t row = i / N;
    const int n = int(i - row * N);
    const double *c = coef + row * M;
    double acc = c[0];
    for (int k = 1; k <= n_h; ++k) {
        double cs, sn;
        cos_sin_kn(k, n, N, cs, sn);
        acc += c[2 * k - 1] * cs + c[2 * k] * sn;
    }
    y[i] = acc;
}

inline int nblk(int64_t n, int b) { return int((n + b - 1) / b); }

}  // namespace

template <typename T>
void launch_faces(int mode, const FaceArgs<T> &a, bool has_resistance, int n_out, cudaStream_t s) {
    const int64_t n = int64_t(a.n_faces) * a.N;
    if (n == 0 || mode == MODE_DIAG) return;
    const int g = nblk(n, 128);
    if (a.fbuf) {                                  // deterministic scatter
        const dim3 fg(unsigned(n_out), unsigned(a.N));
        if (mode == MODE_RES || mode == MODE_TRES) {
            if (has_resistance && n_out > 0) outlet_flux_det_kernel<T, MODE_RES><<<fg, kFluxThreads, 0, s>>>(a);
            face_kernel<T, MODE_RES><<<g, 128, 0, s>>>(a);
        } else if (mode == MODE_JVP) {
            if (has_resistance && n_out > 0) outlet_flux_det_kernel<T, MODE_JVP><<<fg, kFluxThreads, 0, s>>>(a);
            face_kernel<T, MODE_JVP><<<g, 128, 0, s>>>(a);
        } else {
            if (has_resistance && n_out > 0) outlet_flux_det_kernel<T, MODE_JVE><<<fg, kFluxThreads, 0, s>>>(a);
            face_kernel<T, MODE_JVE><<<g, 128, 0, s>>>(a);
        }
        return;
    }
    if (mode == MODE_RES || mode == MODE_TRES) {   // a time level's residual has the same boundary terms
        if (has_resistance) outlet_flux_kernel<T, MODE_RES><<<dim3(nblk(a.n_faces, 256), a.N), 256, 0, s>>>(a, n_out);
        face_kernel<T, MODE_RES><<<g, 128, 0, s>>>(a);
    } else if (mode == MODE_JVP) {
        if (has_resistance) outlet_flux_kernel<T, MODE_JVP><<<dim3(nblk(a.n_faces, 256), a.N), 256, 0, s>>>(a, n_out);
        face_kernel<T, MODE_JVP><<<g, 128, 0, s>>>(a);
    } else {
        if (has_resistance) outlet_flux_kernel<T, MODE_JVE><<<dim3(nblk(a.n_faces, 256), a.N), 256, 0, s>>>(a, n_out);
        face_kernel<T, MODE_JVE><<<g, 128, 0, s>>>(a);
    }
}

void launch_sample_waveforms(const double *coef, int n_wave, int n_h, int N, double T, double *W,
                             cudaStream_t s) {
    (void)T;
    if (n_wave > 0) sample_waveforms_kernel<<<nblk(int64_t(n_wave) * N, 128), 128, 0, s>>>(coef, n_wave, n_h, N, W);
}

void launch_apply_dirichlet(const int *dir_nodes, int n_dir, const double *g, double *y, int N,
                            cudaStream_t s) {
    if (n_dir > 0)
        apply_dirichlet_kernel<<<nblk(int64_t(n_dir) * 3 * N, 256), 256, 0, s>>>(dir_nodes, n_dir, g, y, N);
}

void launch_harmonics(const double *in, double *out, int64_t rows, int N, int n_h, int inverse, double T,
                      cudaStream_t s) {
    (void)T;
    if (rows == 0) return;
    if (!inverse)
        harmonics_kernel<<<nblk(rows * (2 * n_h + 1), 256), 256, 0, s>>>(in, out, rows, N, n_h);
    else
        synthesis_kernel<<<nblk(rows * N, 256), 256, 0, s>>>(in, out, rows, N, n_h);
}

template <typename T>
void launch_det_gather(const DetGatherArgs<T> &a, cudaStream_t s) {
    if (a.n_nodes <= 0) return;
    det_gather_kernel<T><<<nblk(a.n_nodes * a.F * a.N, 256), 256, 0, s>>>(a);
    if (a.F == 7) det_apply_h_kernel<T><<<nblk(a.n_nodes * 3 * a.N, 256), 256, 0, s>>>(a);
}

template void launch_det_gather<float>(const DetGatherArgs<float> &, cudaStream_t);
template void launch_det_gather<double>(const DetGatherArgs<double> &, cudaStream_t);
template void launch_faces<float>(int, const FaceArgs<float> &, bool, int, cudaStream_t);
template void launch_faces<double>(int, const FaceArgs<double> &, bool, int, cudaStream_t);

}  // namespace hb
