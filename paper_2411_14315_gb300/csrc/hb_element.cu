// Fused element kernels of the HB-GLS residual and its Jacobian-vector products (arXiv 2411.14315,
// Sec. 2.2-2.3), plus the per-element geometry precompute.
//
// One CTA processes one element patch at a time: it stages the patch's node rows (all N instances of
// every field) in shared memory, applies the time-coupling H = E^-1 Omega E (Eq. NS-harm) to them
// there, runs one thread per (element, instance) over the patch, accumulates element contributions
// per local node with shared-memory atomics, and flushes each local node once to global memory.  The
// H terms of the residual, -H N_A (least-squares) and rho N_A H u (Galerkin), are applied to the
// patch-assembled T = rho M u - int N_A tau L at flush time: H is linear and acts on the instance
// index only, so applying it per patch and summing equals applying it after global assembly.
#include "hb_internal.cuh"

namespace hb {

namespace {

struct Layout {
    size_t H, geom, Y, V, HY, HV, T, node, conn, total;
};

__host__ __device__ inline size_t pad16(size_t b) { return (b + 15) & ~size_t(15); }

__host__ __device__ inline Layout make_layout(int mode, int N, int nl, int ep, size_t ts) {
    Layout L;
    size_t o = 0;
    const size_t row4 = size_t(nl) * 4 * N * ts, row3 = size_t(nl) * 3 * N * ts;
    L.H = o;    o += pad16(size_t(N) * N * ts);
    L.geom = o; o += pad16(size_t(ep) * kGeomStride * ts);
    L.Y = o;    o += pad16(row4);
    L.V = o;    if (mode == MODE_JVP || mode == MODE_JVE) o += pad16(row4);
    L.HY = o;   if (mode == MODE_RES || mode == MODE_JVE) o += pad16(row3);
    L.HV = o;   if (mode == MODE_JVE || mode == MODE_JVP) o += pad16(row3);
    L.T = o;    if (mode == MODE_RES || mode == MODE_JVE) o += pad16(row3);
    L.node = o; o += pad16(size_t(nl) * 4);
    L.conn = o; o += pad16(size_t(ep) * 4);
    L.total = o;
    return L;
}

// ---------------------------------------------------------------------------------------------------
// per (element, instance) arithmetic

template <typename T>
__device__ __forceinline__ T rsqrt_t(T x);
template <>
__device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt(x); }

__device__ __forceinline__ void load_geom(const float *g, float gN[4][3], float &V, float &g2) {
    const float4 *g4 = reinterpret_cast<const float4 *>(g);
    const float4 a0 = g4[0], a1 = g4[1], a2 = g4[2], a3 = g4[3];
    gN[0][0] = a0.x; gN[0][1] = a0.y; gN[0][2] = a0.z;
    gN[1][0] = a0.w; gN[1][1] = a1.x; gN[1][2] = a1.y;
    gN[2][0] = a1.z; gN[2][1] = a1.w; gN[2][2] = a2.x;
    gN[3][0] = a2.y; gN[3][1] = a2.z; gN[3][2] = a2.w;
    V = a3.x;
    g2 = a3.y;
}

__device__ __forceinline__ void load_geom(const double *g, double gN[4][3], double &V, double &g2) {
    const double2 *g2v = reinterpret_cast<const double2 *>(g);
    double v[14];
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        const double2 t = g2v[k];
        v[2 * k] = t.x;
        v[2 * k + 1] = t.y;
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int j = 0; j < 3; ++j) gN[a][j] = v[3 * a + j];
    V = v[12];
    g2 = v[13];
}

// NT > 0: the number of instances is the compile-time constant NT; NT = 0: runtime N
template <typename T, int MODE, int NT>
__device__ __forceinline__ void element_instance(int e, int n, int Nrt, T rho, T mu, T shift,
                                                 const T *__restrict__ sGeom,
                                                 const uint32_t *__restrict__ sConn,
                                                 const T *__restrict__ sY, const T *__restrict__ sV,
                                                 const T *__restrict__ sHY, const T *__restrict__ sHV,
                                                 const int *__restrict__ sNode, T *__restrict__ gout,
                                                 T *sT) {
    const int N = NT > 0 ? NT : Nrt;
    const int N4 = 4 * N, N3 = 3 * N;
    const uint32_t c = sConn[e];
    const int lo[4] = {int(c & 255u), int((c >> 8) & 255u), int((c >> 16) & 255u), int(c >> 24)};
    // global rows of the 4 nodes at this instance: contributions without instance coupling are added
    // there directly (native global reductions)
    T *go[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) go[a] = gout + size_t(sNode[lo[a]]) * N4 + n;
    T gN[4][3], V, g2;
    load_geom(sGeom + e * kGeomStride, gN, V, g2);
    const T w = V * T(0.25);
    const T qb = T(kQB), qd = T(kQA - kQB);
    const T m20 = V * T(0.05);   // int N_a N_b = V (1 + delta_ab) / 20

    // frozen / current velocity at the 4 nodes
    T u[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) u[a][i] = sY[lo[a] * N4 + i * N + n];
    T usum[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) usum[i] = u[0][i] + u[1][i] + u[2][i] + u[3][i];

    if constexpr (MODE == MODE_DIAG) {
        T dvel[4] = {0, 0, 0, 0}, udNs[4] = {0, 0, 0, 0};
        T taus = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            T uq[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) uq[i] = qb * usum[i] + qd * u[q][i];
            T udN[4];
#pragma unroll
            for (int a = 1; a < 4; ++a) udN[a] = uq[0] * gN[a][0] + uq[1] * gN[a][1] + uq[2] * gN[a][2];
            udN[0] = -(udN[1] + udN[2] + udN[3]);
            const T tau = rsqrt_t<T>(udN[1] * udN[1] + udN[2] * udN[2] + udN[3] * udN[3] + g2);
            taus += tau;
            dvel[q] += w * rho * qd * udN[q];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                udNs[a] += udN[a];
                dvel[a] += w * rho * tau * udN[a] * udN[a];
            }
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const T gg = gN[a][0] * gN[a][0] + gN[a][1] * gN[a][1] + gN[a][2] * gN[a][2];
            const T dv = dvel[a] + w * rho * qb * udNs[a] + mu * V * gg + shift * V * T(0.1);
            const T dp = (w / rho) * taus * gg;
            atomicAdd(go[a], dv);
            atomicAdd(go[a] + N, dv);
            atomicAdd(go[a] + 2 * N, dv);
            atomicAdd(go[a] + 3 * N, dp);
        }
        return;
    } else if constexpr (MODE == MODE_RES) {
        T p[4], hu[4][3];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            p[a] = sY[lo[a] * N4 + 3 * N + n];
#pragma unroll
            for (int i = 0; i < 3; ++i) hu[a][i] = sHY[lo[a] * N3 + i * N + n];
        }
        T gU[3][3], gP[3], husum[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            husum[i] = hu[0][i] + hu[1][i] + hu[2][i] + hu[3][i];
#pragma unroll
            for (int j = 0; j < 3; ++j)
                gU[i][j] = u[0][i] * gN[0][j] + u[1][i] * gN[1][j] + u[2][i] * gN[2][j] + u[3][i] * gN[3][j];
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) gP[j] = p[0] * gN[0][j] + p[1] * gN[1][j] + p[2] * gN[2][j] + p[3] * gN[3][j];
        T qm[4][3], tt[4][3];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int i = 0; i < 3; ++i) qm[a][i] = tt[a][i] = T(0);
        T S[3] = {0, 0, 0}, convs[3] = {0, 0, 0};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            T uq[3], huq[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                uq[i] = qb * usum[i] + qd * u[q][i];
                huq[i] = qb * husum[i] + qd * hu[q][i];
            }
            T udN[4];
#pragma unroll
            for (int a = 1; a < 4; ++a) udN[a] = uq[0] * gN[a][0] + uq[1] * gN[a][1] + uq[2] * gN[a][2];
            udN[0] = -(udN[1] + udN[2] + udN[3]);
            const T tau = rsqrt_t<T>(udN[1] * udN[1] + udN[2] * udN[2] + udN[3] * udN[3] + g2);
            T tL[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const T conv = uq[0] * gU[i][0] + uq[1] * gU[i][1] + uq[2] * gU[i][2];
                tL[i] = tau * (rho * (huq[i] + conv) + gP[i]);
                convs[i] += conv;
                S[i] += tL[i];
                qm[q][i] += w * rho * qd * conv;
                tt[q][i] -= w * qd * tL[i];
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int i = 0; i < 3; ++i) qm[a][i] += w * udN[a] * tL[i];
        }
        const T pbar = T(0.25) * (p[0] + p[1] + p[2] + p[3]);
        const T div = gU[0][0] + gU[1][1] + gU[2][2];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const T visc = gN[a][0] * gU[i][0] + gN[a][1] * gU[i][1] + gN[a][2] * gU[i][2];
                const T vq = qm[a][i] + w * rho * qb * convs[i] + mu * V * visc - V * gN[a][i] * pbar;
                const T vt = tt[a][i] + rho * m20 * (usum[i] + u[a][i]) - w * qb * S[i];
                atomicAdd(go[a] + i * N, vq);
                atomicAdd(sT + lo[a] * N3 + i * N + n, vt);
            }
            const T qc = w * div + (w / rho) * (gN[a][0] * S[0] + gN[a][1] * S[1] + gN[a][2] * S[2]);
            atomicAdd(go[a] + 3 * N, qc);
        }
        return;
    } else if constexpr (MODE == MODE_JVP) {
        T dv[4][3], dvp[4], hdv[4][3];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            dvp[a] = sV[lo[a] * N4 + 3 * N + n];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                dv[a][i] = sV[lo[a] * N4 + i * N + n];
                hdv[a][i] = sHV[lo[a] * N3 + i * N + n];
            }
        }
        T gV[3][3], gVp[3], dvsum[3], hdvsum[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            dvsum[i] = dv[0][i] + dv[1][i] + dv[2][i] + dv[3][i];
            hdvsum[i] = hdv[0][i] + hdv[1][i] + hdv[2][i] + hdv[3][i];
#pragma unroll
            for (int j = 0; j < 3; ++j)
                gV[i][j] = dv[0][i] * gN[0][j] + dv[1][i] * gN[1][j] + dv[2][i] * gN[2][j] + dv[3][i] * gN[3][j];
        }
#pragma unroll
        for (int j = 0; j < 3; ++j)
            gVp[j] = dvp[0] * gN[0][j] + dvp[1] * gN[1][j] + dvp[2] * gN[2][j] + dvp[3] * gN[3][j];
        T qm[4][3];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int i = 0; i < 3; ++i) qm[a][i] = T(0);
        T S[3] = {0, 0, 0}, ugvs[3] = {0, 0, 0};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            T uq[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) uq[i] = qb * usum[i] + qd * u[q][i];
            T udN[4];
#pragma unroll
            for (int a = 1; a < 4; ++a) udN[a] = uq[0] * gN[a][0] + uq[1] * gN[a][1] + uq[2] * gN[a][2];
            udN[0] = -(udN[1] + udN[2] + udN[3]);
            const T tau = rsqrt_t<T>(udN[1] * udN[1] + udN[2] * udN[2] + udN[3] * udN[3] + g2);
            T X[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const T ugv = uq[0] * gV[i][0] + uq[1] * gV[i][1] + uq[2] * gV[i][2];
                X[i] = tau * (rho * ugv + gVp[i]);
                ugvs[i] += ugv;
                S[i] += X[i];
                qm[q][i] += w * rho * qd * ugv;
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int i = 0; i < 3; ++i) qm[a][i] += w * udN[a] * X[i];
        }
        const T pbar = T(0.25) * (dvp[0] + dvp[1] + dvp[2] + dvp[3]);
        const T div = gV[0][0] + gV[1][1] + gV[2][2];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const T visc = gN[a][0] * gV[i][0] + gN[a][1] * gV[i][1] + gN[a][2] * gV[i][2];
                const T mv = m20 * (dvsum[i] + dv[a][i]);
                const T mhv = m20 * (hdvsum[i] + hdv[a][i]);     // F block: H (rho M v) = rho M (H v)
                const T vq = qm[a][i] + w * rho * qb * ugvs[i] + mu * V * visc - V * gN[a][i] * pbar
                           + shift * mv + rho * mhv;
                atomicAdd(go[a] + i * N, vq);
            }
            const T qc = w * div + (w / rho) * (gN[a][0] * S[0] + gN[a][1] * S[1] + gN[a][2] * S[2]);
            atomicAdd(go[a] + 3 * N, qc);
        }
        return;
    } else {  // MODE_JVE
        T p[4], hu[4][3], dv[4][3], dvp[4], hdv[4][3];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            p[a] = sY[lo[a] * N4 + 3 * N + n];
            dvp[a] = sV[lo[a] * N4 + 3 * N + n];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                hu[a][i] = sHY[lo[a] * N3 + i * N + n];
                dv[a][i] = sV[lo[a] * N4 + i * N + n];
                hdv[a][i] = sHV[lo[a] * N3 + i * N + n];
            }
        }
        T gU[3][3], gP[3], gV[3][3], gVp[3], husum[3], dvsum[3], hdvsum[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            husum[i] = hu[0][i] + hu[1][i] + hu[2][i] + hu[3][i];
            dvsum[i] = dv[0][i] + dv[1][i] + dv[2][i] + dv[3][i];
            hdvsum[i] = hdv[0][i] + hdv[1][i] + hdv[2][i] + hdv[3][i];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                gU[i][j] = u[0][i] * gN[0][j] + u[1][i] * gN[1][j] + u[2][i] * gN[2][j] + u[3][i] * gN[3][j];
                gV[i][j] = dv[0][i] * gN[0][j] + dv[1][i] * gN[1][j] + dv[2][i] * gN[2][j] + dv[3][i] * gN[3][j];
            }
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            gP[j] = p[0] * gN[0][j] + p[1] * gN[1][j] + p[2] * gN[2][j] + p[3] * gN[3][j];
            gVp[j] = dvp[0] * gN[0][j] + dvp[1] * gN[1][j] + dvp[2] * gN[2][j] + dvp[3] * gN[3][j];
        }
        T qm[4][3], tt[4][3];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int i = 0; i < 3; ++i) qm[a][i] = tt[a][i] = T(0);
        T S[3] = {0, 0, 0}, dconvs[3] = {0, 0, 0};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            T uq[3], huq[3], duq[3], hduq[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                uq[i] = qb * usum[i] + qd * u[q][i];
                huq[i] = qb * husum[i] + qd * hu[q][i];
                duq[i] = qb * dvsum[i] + qd * dv[q][i];
                hduq[i] = qb * hdvsum[i] + qd * hdv[q][i];
            }
            T udN[4], dudN[4];
#pragma unroll
            for (int a = 1; a < 4; ++a) {
                udN[a] = uq[0] * gN[a][0] + uq[1] * gN[a][1] + uq[2] * gN[a][2];
                dudN[a] = duq[0] * gN[a][0] + duq[1] * gN[a][1] + duq[2] * gN[a][2];
            }
            udN[0] = -(udN[1] + udN[2] + udN[3]);
            dudN[0] = -(dudN[1] + dudN[2] + dudN[3]);
            const T tau = rsqrt_t<T>(udN[1] * udN[1] + udN[2] * udN[2] + udN[3] * udN[3] + g2);
            const T dtau = -tau * tau * tau * (udN[1] * dudN[1] + udN[2] * dudN[2] + udN[3] * dudN[3]);
            T tL[3], dtL[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const T conv = uq[0] * gU[i][0] + uq[1] * gU[i][1] + uq[2] * gU[i][2];
                const T dconv = duq[0] * gU[i][0] + duq[1] * gU[i][1] + duq[2] * gU[i][2]
                              + uq[0] * gV[i][0] + uq[1] * gV[i][1] + uq[2] * gV[i][2];
                const T L = rho * (huq[i] + conv) + gP[i];
                const T dL = rho * (hduq[i] + dconv) + gVp[i];
                tL[i] = tau * L;
                dtL[i] = dtau * L + tau * dL;
                dconvs[i] += dconv;
                S[i] += dtL[i];
                qm[q][i] += w * rho * qd * dconv;
                tt[q][i] -= w * qd * dtL[i];
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int i = 0; i < 3; ++i) qm[a][i] += w * (dudN[a] * tL[i] + udN[a] * dtL[i]);
        }
        const T pbar = T(0.25) * (dvp[0] + dvp[1] + dvp[2] + dvp[3]);
        const T div = gV[0][0] + gV[1][1] + gV[2][2];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const T visc = gN[a][0] * gV[i][0] + gN[a][1] * gV[i][1] + gN[a][2] * gV[i][2];
                const T mv = m20 * (dvsum[i] + dv[a][i]);
                const T vq = qm[a][i] + w * rho * qb * dconvs[i] + mu * V * visc - V * gN[a][i] * pbar + shift * mv;
                const T vt = tt[a][i] + rho * mv - w * qb * S[i];
                atomicAdd(go[a] + i * N, vq);
                atomicAdd(sT + lo[a] * N3 + i * N + n, vt);
            }
            const T qc = w * div + (w / rho) * (gN[a][0] * S[0] + gN[a][1] * S[1] + gN[a][2] * S[2]);
            atomicAdd(go[a] + 3 * N, qc);
        }
        return;
    }
}

// ---------------------------------------------------------------------------------------------------
// the patch kernel

// 16-byte global -> shared copy that does not block the issuing thread (completion: cp_async_wait_all)
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// H is circulant: H[j][k] = h[(j - k) mod N] with h its first column (h[0] = 0).  For a fixed N one row
// of N values is multiplied with the kernel held in registers; x_in may equal x_out (read fully first).
template <typename T, int NT>
__device__ __forceinline__ void circulant_row(const T *__restrict__ hcol, const T *x_in, T *x_out) {
    T x[NT], h[NT];
#pragma unroll
    for (int k = 0; k < NT; ++k) x[k] = x_in[k];
#pragma unroll
    for (int d = 0; d < NT; ++d) h[d] = hcol[d];
#pragma unroll
    for (int m = 0; m < NT; ++m) {
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < NT; ++k)
            if (k != m) acc += h[(m - k + NT) % NT] * x[k];
        x_out[m] = acc;
    }
}

// Shared-memory pointers of one patch pass.
template <typename T>
struct PatchSmem {
    T *H, *geom, *Y, *V, *HY, *HV, *T_;
    int *node;
    uint32_t *conn;
};

template <typename T, int MODE>
__device__ __forceinline__ PatchSmem<T> patch_smem(unsigned char *smem, int N, int nl_max, int ep_max) {
    const Layout L = make_layout(MODE, N, nl_max, ep_max, sizeof(T));
    PatchSmem<T> m;
    m.H = reinterpret_cast<T *>(smem + L.H);
    m.geom = reinterpret_cast<T *>(smem + L.geom);
    m.Y = reinterpret_cast<T *>(smem + L.Y);
    m.V = reinterpret_cast<T *>(smem + L.V);
    m.HY = reinterpret_cast<T *>(smem + L.HY);
    m.HV = reinterpret_cast<T *>(smem + L.HV);
    m.T_ = reinterpret_cast<T *>(smem + L.T);
    m.node = reinterpret_cast<int *>(smem + L.node);
    m.conn = reinterpret_cast<uint32_t *>(smem + L.conn);
    return m;
}

// Stage H (fixed N: its first column; runtime N: the full matrix).
template <typename T, int NT>
__device__ __forceinline__ void stage_H(const ElemArgs<T> &a, T *sH, int N) {
    if constexpr (NT > 0) {
        for (int i = threadIdx.x; i < N; i += blockDim.x) sH[i] = a.H[i * N];
    } else {
        for (int i = threadIdx.x; i < N * N; i += blockDim.x) sH[i] = a.H[i];
    }
}

// One patch: gather, Dirichlet masking, in-patch H products, element-instance work, H T flush.
// Ends with a block barrier, so shared memory can be reused by the next patch.
template <typename T, int MODE, int NT>
__device__ __forceinline__ void patch_pass(const ElemArgs<T> &a, int p, const PatchSmem<T> &sm, T shift) {
    const int N = NT > 0 ? NT : a.N, N4 = 4 * N, N3 = 3 * N;
    T *sH = sm.H, *sGeom = sm.geom, *sY = sm.Y, *sV = sm.V, *sHY = sm.HY, *sHV = sm.HV, *sT = sm.T_;
    int *sNode = sm.node;
    uint32_t *sConn = sm.conn;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int e0 = a.pv.eptr[p], ne = a.pv.eptr[p + 1] - e0;
    const int q0 = a.pv.nptr[p], nl = a.pv.nptr[p + 1] - q0;
    for (int i = tid; i < nl; i += nt) sNode[i] = a.pv.nodes[q0 + i];
    for (int i = tid; i < ne; i += nt) sConn[i] = a.pv.lconn[e0 + i];
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.pv.geom + size_t(e0) * kGeomStride);
        uint4 *dst = reinterpret_cast<uint4 *>(sGeom);
        const int nvec = int(ne * kGeomStride * sizeof(T) / 16);
        for (int i = tid; i < nvec; i += nt) dst[i] = src[i];
    }
    if constexpr (MODE == MODE_RES || MODE == MODE_JVE)
        for (int i = tid; i < nl * N3; i += nt) sT[i] = T(0);
    __syncthreads();

    // gather the patch's node rows (4 N values per node) with asynchronous 16-byte copies, so every
    // thread keeps all of its loads in flight
    const int cpr = int(N4 * sizeof(T) / 16);
    for (int i = tid; i < nl * cpr; i += nt) {
        const int l = i / cpr, c = i - l * cpr;
        const size_t gidx = size_t(sNode[l]) * cpr + c;
        cp_async16(reinterpret_cast<uint4 *>(sY) + i, reinterpret_cast<const uint4 *>(a.y) + gidx);
        if constexpr (MODE == MODE_JVP || MODE == MODE_JVE)
            cp_async16(reinterpret_cast<uint4 *>(sV) + i, reinterpret_cast<const uint4 *>(a.v) + gidx);
    }
    cp_async_wait_all();
    __syncthreads();
    if constexpr (MODE == MODE_JVP || MODE == MODE_JVE) {
        // Dirichlet velocity entries of the direction are not unknowns: treat them as 0 (only the
        // patches touching a Dirichlet boundary have any)
        const int d0 = a.pv.dptr[p], nd = a.pv.dptr[p + 1] - d0;
        if (nd > 0) {
            for (int i = tid; i < nd * N3; i += nt) {
                const int k = i / N3, r = i - k * N3;
                sV[int(a.pv.dloc[d0 + k]) * N4 + r] = T(0);
            }
            __syncthreads();
        }
    }
    if constexpr (MODE != MODE_DIAG) {
        // time coupling of the staged velocities: (H x)[l][i][n] = sum_k H[n][k] x[l][i][k] for
        // x = u (RES, JVE) and x = v (JVP, JVE)
        constexpr bool hy = (MODE == MODE_RES || MODE == MODE_JVE);
        constexpr bool hv = (MODE == MODE_JVP || MODE == MODE_JVE);
        constexpr int nsrc = (hy ? 1 : 0) + (hv ? 1 : 0);
        if constexpr (NT > 0) {
            const int rows = nl * 3;
            for (int r = tid; r < nsrc * rows; r += nt) {
                const int which = hy ? (r >= rows) : 1, rr = r - (r >= rows) * rows, l = rr / 3, f = rr - 3 * l;
                const T *src = (which ? sV : sY) + l * N4 + f * N;
                T *dst = (which ? sHV : sHY) + l * N3 + f * N;
                circulant_row<T, NT>(sH, src, dst);
            }
        } else {
            for (int i = tid; i < nl * N3; i += nt) {
                const int l = i / N3, r = i - l * N3, f = r / N, n = r - f * N;
                const T *h = sH + n * N;
                if constexpr (hy) {
                    const T *x = sY + l * N4 + f * N;
                    T acc = 0;
                    for (int k = 0; k < N; ++k) acc += h[k] * x[k];
                    sHY[i] = acc;
                }
                if constexpr (hv) {
                    const T *xv = sV + l * N4 + f * N;
                    T acc2 = 0;
                    for (int k = 0; k < N; ++k) acc2 += h[k] * xv[k];
                    sHV[i] = acc2;
                }
            }
        }
        __syncthreads();
    }

    for (int i = tid; i < ne * N; i += nt) {
        const int e = i / N, n = i - e * N;
        element_instance<T, MODE, NT>(e, n, N, a.rho, a.mu, shift, sGeom, sConn, sY, sV, sHY, sHV, sNode,
                                      a.out, sT);
    }
    __syncthreads();

    // H T on the patch-assembled T rows (fixed N: in place, one row per thread)
    if constexpr ((MODE == MODE_RES || MODE == MODE_JVE) && NT > 0) {
        for (int r = tid; r < nl * 3; r += nt) {
            T *row = sT + (r / 3) * N3 + (r % 3) * N;
            circulant_row<T, NT>(sH, row, row);
        }
        __syncthreads();
    }

    // flush: out += H T on the velocity rows, once per local node
    if constexpr (MODE == MODE_RES || MODE == MODE_JVE) {
        for (int i = tid; i < nl * N3; i += nt) {
            const int l = i / N3, r = i - l * N3;
            T val;
            if constexpr (NT > 0) {
                val = sT[i];
            } else {
                const int f = r / N, n = r - f * N;
                const T *h = sH + n * N;
                const T *t = sT + l * N3 + f * N;
                val = T(0);
                for (int k = 0; k < N; ++k) val += h[k] * t[k];
            }
            atomicAdd(a.out + size_t(sNode[l]) * N4 + r, val);
        }
    }
    __syncthreads();
}

template <typename T, int MODE, int NT>
__global__ void __launch_bounds__(kBlock, (sizeof(T) == 4 ? 2 : 1)) elem_kernel(ElemArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = NT > 0 ? NT : a.N;
    const PatchSmem<T> sm = patch_smem<T, MODE>(smem, N, a.pv.nl_max, a.pv.ep_max);
    const T shift = a.shift_dev ? T(*a.shift_dev) : a.shift;
    stage_H<T, NT>(a, sm.H, N);
    for (int p = blockIdx.x; p < a.pv.n_patches; p += gridDim.x) patch_pass<T, MODE, NT>(a, p, sm, shift);
}

// Persistent kernel over the patches of many problems: work items (problem, patch) are taken from a
// global counter, so problems of uneven size share the SMs; each item runs the fixed-N pass of its
// problem's instance count (9, 13, 21) or the generic one.
template <typename T, int MODE>
__global__ void __launch_bounds__(kBlock, (sizeof(T) == 4 ? 2 : 1)) batch_elem_kernel(const ElemArgs<T> *__restrict__ args,
                                                               const int *__restrict__ first_item, int n_prob,
                                                               int n_items, int *counter) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    int last = -1;
    while (true) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= n_items) break;
        int lo = 0, hi = n_prob - 1;               // problem owning this item: first_item[q] <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (first_item[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        const ElemArgs<T> &a = args[lo];
        const int patch = item - first_item[lo];
        const T shift = a.shift_dev ? T(*a.shift_dev) : a.shift;
        switch (a.N) {
            case 9: {
                const PatchSmem<T> sm = patch_smem<T, MODE>(smem, 9, a.pv.nl_max, a.pv.ep_max);
                if (lo != last) { stage_H<T, 9>(a, sm.H, 9); __syncthreads(); }
                patch_pass<T, MODE, 9>(a, patch, sm, shift);
                break;
            }
            case 13: {
                const PatchSmem<T> sm = patch_smem<T, MODE>(smem, 13, a.pv.nl_max, a.pv.ep_max);
                if (lo != last) { stage_H<T, 13>(a, sm.H, 13); __syncthreads(); }
                patch_pass<T, MODE, 13>(a, patch, sm, shift);
                break;
            }
            case 21: {
                const PatchSmem<T> sm = patch_smem<T, MODE>(smem, 21, a.pv.nl_max, a.pv.ep_max);
                if (lo != last) { stage_H<T, 21>(a, sm.H, 21); __syncthreads(); }
                patch_pass<T, MODE, 21>(a, patch, sm, shift);
                break;
            }
            default: {
                const PatchSmem<T> sm = patch_smem<T, MODE>(smem, a.N, a.pv.nl_max, a.pv.ep_max);
                if (lo != last) { stage_H<T, 0>(a, sm.H, a.N); __syncthreads(); }
                patch_pass<T, MODE, 0>(a, patch, sm, shift);
                break;
            }
        }
        last = lo;
    }
}

// ---------------------------------------------------------------------------------------------------
// geometry precompute: grad N_a, V, C_I nu^2 G:G with G = J^-T J^-1 (metric of the parent map)

template <typename T>
__global__ void geom_kernel(const double *__restrict__ xyz, const int *__restrict__ tets, int n_tets,
                            double nu, T *__restrict__ geom) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_tets) return;
    double x[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int nd = tets[4 * e + a];
#pragma unroll
        for (int i = 0; i < 3; ++i) x[a][i] = xyz[3 * nd + i];
    }
    double J[3][3];   // J[i][k] = (x_{k+1} - x_0)_i
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) J[i][k] = x[k + 1][i] - x[0][i];
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    const double id = 1.0 / det;
    double Ji[3][3];  // inverse: Ji[k][i] = d xi_k / d x_i
    Ji[0][0] = c00 * id;
    Ji[1][0] = c01 * id;
    Ji[2][0] = c02 * id;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
    T *g = geom + size_t(e) * kGeomStride;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        g[i] = T(-(Ji[0][i] + Ji[1][i] + Ji[2][i]));
#pragma unroll
        for (int k = 0; k < 3; ++k) g[3 * (k + 1) + i] = T(Ji[k][i]);
    }
    double GG = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const double Gij = Ji[0][i] * Ji[0][j] + Ji[1][i] * Ji[1][j] + Ji[2][i] * Ji[2][j];
            GG += Gij * Gij;
        }
    g[12] = T(fabs(det) / 6.0);
    g[13] = T(kCI * nu * nu * GG);
    g[14] = T(0);
    g[15] = T(0);
}

inline int nblk(int64_t n, int b) { return int((n + b - 1) / b); }

}  // namespace

size_t elem_smem_bytes(int mode, int N, int nl_max, int ep_max, size_t tsize) {
    return make_layout(mode, N, nl_max, ep_max, tsize).total;
}

template <typename T, int MODE, int NT>
static void launch_elem_n(const ElemArgs<T> &a, int grid, cudaStream_t s) {
    const size_t smem = elem_smem_bytes(MODE, a.N, a.pv.nl_max, a.pv.ep_max, sizeof(T));
    static size_t configured = 0;
    if (smem > 48 * 1024 && smem > configured) {
        cudaFuncSetAttribute(elem_kernel<T, MODE, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        configured = smem;
    }
    elem_kernel<T, MODE, NT><<<grid, kBlock, smem, s>>>(a);
}

// fixed-N instantiations for the instance counts of the workloads; any other N runs the generic kernel
template <typename T, int MODE>
static void launch_elem_mode(const ElemArgs<T> &a, int grid, cudaStream_t s) {
    switch (a.N) {
        case 9: launch_elem_n<T, MODE, 9>(a, grid, s); break;
        case 13: launch_elem_n<T, MODE, 13>(a, grid, s); break;
        case 21: launch_elem_n<T, MODE, 21>(a, grid, s); break;
        default: launch_elem_n<T, MODE, 0>(a, grid, s); break;
    }
}

template <typename T>
void launch_elem(int mode, const ElemArgs<T> &a, int grid, cudaStream_t s) {
    switch (mode) {
        case MODE_RES: launch_elem_mode<T, MODE_RES>(a, grid, s); break;
        case MODE_JVP: launch_elem_mode<T, MODE_JVP>(a, grid, s); break;
        case MODE_JVE: launch_elem_mode<T, MODE_JVE>(a, grid, s); break;
        default: launch_elem_mode<T, MODE_DIAG>(a, grid, s); break;
    }
}

template <typename T>
void launch_batch_elem(int mode, const ElemArgs<T> *args, const int *first_item, int n_prob, int n_items,
                       int *counter, size_t smem, int grid, cudaStream_t s) {
    auto go = [&](auto kern) {
        if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        kern<<<grid, kBlock, smem, s>>>(args, first_item, n_prob, n_items, counter);
    };
    switch (mode) {
        case MODE_RES: go(batch_elem_kernel<T, MODE_RES>); break;
        case MODE_JVP: go(batch_elem_kernel<T, MODE_JVP>); break;
        case MODE_JVE: go(batch_elem_kernel<T, MODE_JVE>); break;
        default: go(batch_elem_kernel<T, MODE_DIAG>); break;
    }
}

template <typename T>
void launch_geom(const double *xyz, const int *tets, int n_tets, double nu, T *geom, cudaStream_t s) {
    if (n_tets > 0) geom_kernel<T><<<nblk(n_tets, 128), 128, 0, s>>>(xyz, tets, n_tets, nu, geom);
}

template void launch_elem<float>(int, const ElemArgs<float> &, int, cudaStream_t);
template void launch_elem<double>(int, const ElemArgs<double> &, int, cudaStream_t);
template void launch_batch_elem<float>(int, const ElemArgs<float> *, const int *, int, int, int *, size_t, int,
                                       cudaStream_t);
template void launch_batch_elem<double>(int, const ElemArgs<double> *, const int *, int, int, int *, size_t, int,
                                        cudaStream_t);
template void launch_geom<float>(const double *, const int *, int, double, float *, cudaStream_t);
template void launch_geom<double>(const double *, const int *, int, double, double *, cudaStream_t);

}  // namespace hb
