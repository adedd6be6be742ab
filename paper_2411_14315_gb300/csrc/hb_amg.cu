// Aggregation multigrid preconditioner for the assembled paper tangent (an extension; Sec. 2.3 uses Jacobi).
//
// Level 0 is the assembled operator of Eqs. (K_mat), (ctangent), (F_mat) per node pair and instance
// (hb_assembled.cu); level l + 1 aggregates the nodes of level l.  With piecewise-constant prolongation P
// (velocity only onto nodes whose velocity is free, pressure onto every node) the Galerkin coarse operator
// P^T A P is the sum of the fine pair blocks over the pairs of two aggregates: the fine K, G, D, L blocks
// already vanish on prescribed-velocity rows / columns, and the pair mass (which carries the pseudo-time
// shift and the time coupling rho M (H v), H acting on the instance index only) is summed over pairs of
// two free nodes.  A V-cycle smooths with damped 4 x 4 node-block Jacobi (per node and instance, inverted
// through the pressure Schur complement), computes level residuals with the level's sparse product (the
// same kernel as the fine operator, with W = shift x + rho H x per node), restricts and prolongs by
// gathers (no atomics), and smooths more on the coarsest level.  Every sweep count and weight is fixed, so
// the preconditioner is a fixed linear operator and plain right-preconditioned GMRES applies.
#include "hb_internal.cuh"

namespace hb {

namespace {

inline int nblk(int64_t n, int b) { return int((n + b - 1) / b); }

// b_c[I][f][n] = sum over the fine nodes i of aggregate I of r_f[i][f][n] (velocity only from free nodes)
template <typename T>
__global__ void amg_restrict_kernel(const int *__restrict__ aptr, const int *__restrict__ aidx,
                                    const uint8_t *__restrict__ flag_f, const T *__restrict__ r_f, T *__restrict__ b_c,
                                    int64_t n_c, int N) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int N4 = 4 * N;
    if (t >= n_c * N4) return;
    const int64_t I = t / N4;
    const int fn = int(t - I * N4), f = fn / N;
    T s = 0;
    for (int k = aptr[I]; k < aptr[I + 1]; ++k) {
        const int i = aidx[k];
        if (f < 3 && (flag_f[i] & 1)) continue;
        s += r_f[int64_t(i) * N4 + fn];
    }
    b_c[t] = s;
}

// x_f[i][f][n] += x_c[agg[i]][f][n] (velocity only onto free nodes)
template <typename T>
__global__ void amg_prolong_kernel(const int *__restrict__ agg, const uint8_t *__restrict__ flag_f,
                                   const T *__restrict__ x_c, T *__restrict__ x_f, int64_t n_f, int N) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int N4 = 4 * N;
    if (t >= n_f * N4) return;
    const int64_t i = t / N4;
    const int fn = int(t - i * N4);
    if (fn < 3 * N && (flag_f[i] & 1)) return;
    x_f[t] += x_c[int64_t(agg[i]) * N4 + fn];
}

// coarse pair blocks: coef_c[cp][k][n] = sum of coef_f over the fine pairs listed for cp; mass over the
// listed pairs whose two nodes are free (mmask)
template <typename T>
__global__ void amg_coarse_coef_kernel(const int *__restrict__ cptr, const int *__restrict__ cidx,
                                       const T *__restrict__ coef_f, T *__restrict__ coef_c, int64_t nnz_c, int N) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int N8 = 8 * N;
    if (t >= nnz_c * N8) return;
    const int64_t cp = t / N8;
    const int kn = int(t - cp * N8);
    T s = 0;
    for (int k = cptr[cp]; k < cptr[cp + 1]; ++k) s += coef_f[int64_t(cidx[k]) * N8 + kn];
    coef_c[t] = s;
}

template <typename T>
__global__ void amg_coarse_mass_kernel(const int *__restrict__ cptr, const int *__restrict__ cidx,
                                       const uint8_t *__restrict__ mmask, const T *__restrict__ mass_f,
                                       T *__restrict__ mass_c, int64_t nnz_c) {
    const int64_t cp = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (cp >= nnz_c) return;
    T s = 0;
    for (int k = cptr[cp]; k < cptr[cp + 1]; ++k)
        if (mmask[cidx[k]]) s += mass_f[cidx[k]];
    mass_c[cp] = s;
}

// x = omega D^-1 r (accumulate = 0) or x += omega D^-1 r, D the node-block diagonal (+ shift M_AA);
// prescribed-velocity rows are the identity
template <typename T>
__global__ void amg_smooth_kernel(const T *__restrict__ coef, const T *__restrict__ mass, const int *__restrict__ dpos,
                                  const uint8_t *__restrict__ flag, const T *__restrict__ r, T *__restrict__ x,
                                  int64_t n_nodes, int N, double omega, double shift, const double *__restrict__ shift_dev,
                                  int accumulate) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n_nodes * N) return;
    const int64_t A = i / N;
    const int n = int(i - A * N);
    const double sh = shift_dev ? *shift_dev : shift;
    const int64_t base = A * 4 * N + n;
    const double r0 = r[base], r1 = r[base + N], r2 = r[base + 2 * N], rp = r[base + 3 * N];
    const T *c = coef + int64_t(dpos[A]) * 8 * N + n;
    const double l = double(c[7 * N]);
    double z0, z1, z2, zp;
    if (flag[A] & 1) {
        z0 = r0;
        z1 = r1;
        z2 = r2;
        zp = l != 0.0 ? rp / l : rp;
    } else {
        const double ks = double(c[0]) + sh * double(mass[dpos[A]]);
        const double g0 = c[N], g1 = c[2 * N], g2 = c[3 * N], d0 = c[4 * N], d1 = c[5 * N], d2 = c[6 * N];
        const double ik = 1.0 / ks;
        const double S = l - (d0 * g0 + d1 * g1 + d2 * g2) * ik;
        zp = (rp - (d0 * r0 + d1 * r1 + d2 * r2) * ik) / S;
        z0 = (r0 - g0 * zp) * ik;
        z1 = (r1 - g1 * zp) * ik;
        z2 = (r2 - g2 * zp) * ik;
    }
    if (accumulate) {
        x[base] += T(omega * z0);
        x[base + N] += T(omega * z1);
        x[base + 2 * N] += T(omega * z2);
        x[base + 3 * N] += T(omega * zp);
    } else {
        x[base] = T(omega * z0);
        x[base + N] = T(omega * z1);
        x[base + 2 * N] = T(omega * z2);
        x[base + 3 * N] = T(omega * zp);
    }
}

template <typename T>
__global__ void amg_sub_kernel(const T *__restrict__ b, const T *__restrict__ ax, T *__restrict__ r, int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        r[i] = b[i] - ax[i];
}

}  // namespace

template <typename T>
void launch_amg_restrict(const int *aptr, const int *aidx, const uint8_t *flag_f, const T *r_f, T *b_c, int64_t n_c,
                         int N, cudaStream_t s) {
    if (n_c > 0) amg_restrict_kernel<T><<<nblk(n_c * 4 * N, 256), 256, 0, s>>>(aptr, aidx, flag_f, r_f, b_c, n_c, N);
}
template <typename T>
void launch_amg_prolong(const int *agg, const uint8_t *flag_f, const T *x_c, T *x_f, int64_t n_f, int N,
                        cudaStream_t s) {
    if (n_f > 0) amg_prolong_kernel<T><<<nblk(n_f * 4 * N, 256), 256, 0, s>>>(agg, flag_f, x_c, x_f, n_f, N);
}
template <typename T>
void launch_amg_coarse(const int *cptr, const int *cidx, const uint8_t *mmask, const T *coef_f, const T *mass_f,
                       T *coef_c, T *mass_c, int64_t nnz_c, int N, bool with_mass, cudaStream_t s) {
    if (nnz_c <= 0) return;
    amg_coarse_coef_kernel<T><<<nblk(nnz_c * 8 * N, 256), 256, 0, s>>>(cptr, cidx, coef_f, coef_c, nnz_c, N);
    if (with_mass) amg_coarse_mass_kernel<T><<<nblk(nnz_c, 256), 256, 0, s>>>(cptr, cidx, mmask, mass_f, mass_c, nnz_c);
}
template <typename T>
void launch_amg_smooth(const T *coef, const T *mass, const int *dpos, const uint8_t *flag, const T *r, T *x,
                       int64_t n_nodes, int N, double omega, double shift, const double *shift_dev, int accumulate,
                       cudaStream_t s) {
    if (n_nodes > 0)
        amg_smooth_kernel<T><<<nblk(n_nodes * N, 256), 256, 0, s>>>(coef, mass, dpos, flag, r, x, n_nodes, N, omega,
                                                                    shift, shift_dev, accumulate);
}
template <typename T>
void launch_amg_sub(const T *b, const T *ax, T *r, int64_t n, cudaStream_t s) {
    if (n > 0) amg_sub_kernel<T><<<std::min(nblk(n, 256), 4096), 256, 0, s>>>(b, ax, r, n);
}

#define HB_AMG_INST(T)                                                                                             \
    template void launch_amg_restrict<T>(const int *, const int *, const uint8_t *, const T *, T *, int64_t, int,   \
                                         cudaStream_t);                                                            \
    template void launch_amg_prolong<T>(const int *, const uint8_t *, const T *, T *, int64_t, int, cudaStream_t); \
    template void launch_amg_coarse<T>(const int *, const int *, const uint8_t *, const T *, const T *, T *, T *,  \
                                       int64_t, int, bool, cudaStream_t);                                          \
    template void launch_amg_smooth<T>(const T *, const T *, const int *, const uint8_t *, const T *, T *, int64_t, \
                                       int, double, double, const double *, int, cudaStream_t);                    \
    template void launch_amg_sub<T>(const T *, const T *, T *, int64_t, cudaStream_t);
HB_AMG_INST(float)
HB_AMG_INST(double)
#undef HB_AMG_INST

}  // namespace hb
