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

#include <algorithm>

namespace hb {

namespace {

struct Layout {
    size_t H, geom, Y, V, HY, HV, T, node, conn, total;
};

__host__ __device__ inline size_t pad16(size_t b) { return (b + 15) & ~size_t(15); }

// The two slot buffers come first, sized for slot_cap ints each (0: the patch set's own slot size), so
// a batch of problems with different node caps can stage the next problem's slot while the current one
// computes.
__host__ __device__ inline Layout make_layout(int mode, int N, int nl, int ep, size_t ts, int slot_cap = 0) {
    Layout L;
    size_t o = 0;
    const size_t row4 = size_t(nl) * 4 * N * ts, row3 = size_t(nl) * 3 * N * ts;
    L.node = o; o += pad16(size_t(2) * size_t(slot_cap > 0 ? slot_cap : slot_ints(nl)) * 4);
    L.H = o;    o += pad16(size_t(N) * N * ts);
    L.geom = o; o += pad16(size_t(ep) * kGeomStride * ts);
    L.Y = o;    o += pad16(row4);
    L.V = o;    if (mode == MODE_JVP || mode == MODE_JVE || mode == MODE_TRES) o += pad16(row4);
    L.HY = o;   if (mode == MODE_RES || mode == MODE_JVE) o += pad16(row3);
    L.HV = o;
    if (mode == MODE_JVE) o += pad16(row3);
    if (mode == MODE_JVP) o += pad16(size_t(nl) * w_stride(N, int(ts)) * ts);   // W rows, padded
    L.T = o;    if (mode == MODE_RES || mode == MODE_JVE) o += pad16(row3);
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

// ---------------------------------------------------------------------------------------------------
// Lanes of the paper-tangent pass: FP64 runs one instance per thread (lane = double); FP32 runs two
// instances per thread (lane = float2) on Blackwell's paired FP32 instructions, which halves the
// issue slots of the arithmetic.

template <typename T>
struct LaneOf;
template <>
struct LaneOf<double> { using type = double; };
template <>
struct LaneOf<float> { using type = float2; };

// Launch variants of the paper-tangent pass (the other passes always run variant 0):
//   0: 256 threads per block; FP32 runs two instances per thread on paired instructions
//   1: 384 threads per block, one instance per thread (fewer registers, more resident warps; default)
//   2: 512 threads per block, one instance per thread
//   3: 192 threads per block, one instance per thread, four resident blocks per SM (with patches small
//      enough for four blocks' shared memory, the gather and barrier phases of one block overlap the
//      element work of the others)
// minb: resident blocks per SM the register allocation is bounded for
template <typename T, int VAR>
struct ElemCfg;
template <typename T>
struct ElemCfg<T, 0> { static constexpr int block = 256, minb = sizeof(T) == 4 ? 2 : 1; using lane = typename LaneOf<T>::type; };
template <typename T>
struct ElemCfg<T, 1> { static constexpr int block = 384, minb = sizeof(T) == 4 ? 2 : 1; using lane = T; };
template <typename T>
struct ElemCfg<T, 2> { static constexpr int block = 512, minb = sizeof(T) == 4 ? 2 : 1; using lane = T; };
template <typename T>
struct ElemCfg<T, 3> { static constexpr int block = 192, minb = sizeof(T) == 4 ? 4 : 1; using lane = T; };

__device__ __forceinline__ unsigned long long f2_bits(float2 a) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 bits_f2(unsigned long long r) {
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
__device__ __forceinline__ double lfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float2 lfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double lmul(double a, double b) { return a * b; }
__device__ __forceinline__ float2 lmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ double ladd(double a, double b) { return a + b; }
__device__ __forceinline__ float2 ladd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ double lsub(double a, double b) { return a - b; }
__device__ __forceinline__ float2 lsub(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return bits_f2(r);
}
__device__ __forceinline__ float lfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float lmul(float a, float b) { return a * b; }
__device__ __forceinline__ float ladd(float a, float b) { return a + b; }
__device__ __forceinline__ float lsub(float a, float b) { return a - b; }
template <typename L, typename T>
__device__ __forceinline__ L lsplat(T s) {
    if constexpr (sizeof(L) == 2 * sizeof(T)) return make_float2(s, s);
    else return s;
}
__device__ __forceinline__ double lrsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float lrsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ float2 lrsqrt(float2 x) { return make_float2(rsqrtf(x.x), rsqrtf(x.y)); }
// the lane's instances of a staged row: p[0] (and p[d1] for the second instance of a pair)
template <typename L, typename T>
__device__ __forceinline__ L lload(const T *p, int d1) {
    if constexpr (sizeof(L) == 2 * sizeof(T)) return make_float2(p[0], p[d1]);
    else return p[0];
}
// global accumulation; d1 = 0 marks a pair whose second instance does not exist
__device__ __forceinline__ void lred(double *p, double v, int) { atomicAdd(p, v); }
__device__ __forceinline__ void lred(float *p, float v, int) { atomicAdd(p, v); }
__device__ __forceinline__ void lred(float *p, float2 v, int d1) {
    atomicAdd(p, v.x);
    if (d1) atomicAdd(p + d1, v.y);
}
template <typename L>
__device__ __forceinline__ L ldot3(const L *a, const L *b, L c) {
    return lfma(a[0], b[0], lfma(a[1], b[1], lfma(a[2], b[2], c)));
}
template <typename L>
__device__ __forceinline__ L ldot3(const L *a, const L *b) {
    return lfma(a[0], b[0], lfma(a[1], b[1], lmul(a[2], b[2])));
}

// Paper-tangent Jv (P + C) v of one element at the lane's instances n0 (and n0 + d1), Eqs. (ptangent),
// (K_mat), (ctangent), (F_mat), with U and tau frozen at the state y.  sW holds W = shift v + rho H v
// per patch node: the F block rho M (H v) and the pseudo-time mass shift M v share the mass matrix.
//
// The element sums are regrouped so that no per-node accumulator is carried through the quadrature
// loop (exact algebra; only the rounding order differs from the term-by-term form):
//   sum_q udN_q[a] X_q[i]            = grad N_a . Mx[:, i],  Mx[j][i] = sum_q u_q[j] X_q[i]
//   sum_q (u_q . grad v_i)           = (sum_a u_a) . grad v_i  (the 4 points average to the centroid)
//   visc, pressure and Mx terms      = grad N_a . Z[:, i],   Z = w rho Mx + mu V (grad v)^T - V pbar I
// with X_q = tau_q (u_q . grad v + grad q / rho) the strong residual of the direction over rho.
//
// PIPE (the pipelined pass, FP32): the packed local connectivity sits in slot 14 of the element's geometry
// record instead of sConn, and the staged direction rows are the caller's unmodified values, so the
// velocity of nodes with prescribed velocity is masked to 0 here, at load time.
//
// DET (deterministic scatter): instead of reductions into gout, the element stores its 16 contributions
// (node a, field f) at cslot[(4 a + f) N + n]; a node-level gather sums them in a fixed order.
template <typename L, typename T>
__device__ __forceinline__ void lstore(T *p, L v, int d1) {
    if constexpr (sizeof(L) == 2 * sizeof(T)) {
        p[0] = v.x;
        if (d1) p[d1] = v.y;
    } else {
        p[0] = v;
    }
}

template <typename T, typename L, int NT, bool PIPE = false, bool DET = false>
__device__ __forceinline__ void jvp_lanes(int e, int n0, int d1, int Nrt, T rho, T mu, T omega2, T cs,
                                          const T *__restrict__ sGeom, const uint32_t *__restrict__ sConn,
                                          const T *__restrict__ sY, const T *__restrict__ sV,
                                          const T *__restrict__ sW, const int *__restrict__ sNode,
                                          T *__restrict__ gout, T *__restrict__ cslot = nullptr) {
    const int N = NT > 0 ? NT : Nrt, N4 = 4 * N, WS = w_stride(N, int(sizeof(T)));
    uint32_t c;
    if constexpr (PIPE) c = __float_as_uint(float(sGeom[e * kGeomStride + 14]));
    else c = sConn[e];
    const int lo[4] = {int(c & 255u), int((c >> 8) & 255u), int((c >> 16) & 255u), int(c >> 24)};
    int rY[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) rY[a] = lo[a] * N4 + n0;
    // velocity of the direction at the 4 nodes: 0 where the velocity is prescribed (PIPE only; the
    // other passes zero those entries in shared memory after staging)
    bool vfree[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) vfree[a] = !PIPE || sNode[lo[a]] >= 0;
    T gs[4][3], V, g2s;
    load_geom(sGeom + e * kGeomStride, gs, V, g2s);
    L gN[3][3];   // grad N_a of the vertices a = 1, 2, 3 (grad N_0 = -(sum of these))
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int j = 0; j < 3; ++j) gN[a][j] = lsplat<L>(gs[a + 1][j]);

    // gradients of the direction: grad v_i = sum_{a >= 1} (v_a - v_0)_i grad N_a, same for q
    L gV[3][3], gVp[3], pbar;
    // time domain (NT = 1): the direction's velocity at the quadrature points, for the least-squares
    // acceleration term cs v_q inside L (cs = shift / rho, 0 when unused)
    constexpr int NVQ = NT == 1 ? 4 : 1;
    L vn[NVQ][3];
    {
        L dv0[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) dv0[i] = vfree[0] ? lload<L>(sV + rY[0] + i * N, d1) : lsplat<L>(T(0));
        if constexpr (NT == 1) {
#pragma unroll
            for (int i = 0; i < 3; ++i) vn[0][i] = dv0[i];
        }
        const L dp0 = lload<L>(sV + rY[0] + 3 * N, d1);
        pbar = dp0;
#pragma unroll
        for (int a = 1; a < 4; ++a) {
            const L dp = lload<L>(sV + rY[a] + 3 * N, d1);
            pbar = ladd(pbar, dp);
            const L ddp = lsub(dp, dp0);
#pragma unroll
            for (int j = 0; j < 3; ++j) gVp[j] = a == 1 ? lmul(ddp, gN[0][j]) : lfma(ddp, gN[a - 1][j], gVp[j]);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const L va = vfree[a] ? lload<L>(sV + rY[a] + i * N, d1) : lsplat<L>(T(0));
                if constexpr (NT == 1) vn[a][i] = va;
                const L dd = lsub(va, dv0[i]);
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    gV[i][j] = a == 1 ? lmul(dd, gN[0][j]) : lfma(dd, gN[a - 1][j], gV[i][j]);
            }
        }
        pbar = lmul(pbar, lsplat<L>(T(0.25) * V));          // V times the element mean of q
        const L ir = lsplat<L>(T(1) / rho);
#pragma unroll
        for (int j = 0; j < 3; ++j) gVp[j] = lmul(gVp[j], ir);
    }

    // frozen velocity at the 4 nodes, turned into its values at the 4 quadrature points
    L uq[4][3], usum[3], Ug[3];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) uq[a][i] = lload<L>(sY + rY[a] + i * N, d1);
#pragma unroll
    for (int i = 0; i < 3; ++i) usum[i] = ladd(ladd(uq[0][i], uq[1][i]), ladd(uq[2][i], uq[3][i]));
#pragma unroll
    for (int i = 0; i < 3; ++i) Ug[i] = ldot3(usum, gV[i]);
    {
        const L qb = lsplat<L>(T(kQB)), qd = lsplat<L>(T(kQA - kQB));
#pragma unroll
        for (int i = 0; i < 3; ++i) usum[i] = lmul(usum[i], qb);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int i = 0; i < 3; ++i) uq[a][i] = lfma(qd, uq[a][i], usum[i]);
    }

    // quadrature loop: tau_q, X_q and the two element sums Mx and S
    L Mx[3][3], S[3];
    const L g2 = lsplat<L>(g2s + omega2);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        L udN[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) udN[a] = ldot3(uq[q], gN[a]);
        const L tau = lrsqrt(lfma(udN[0], udN[0], lfma(udN[1], udN[1], lfma(udN[2], udN[2], g2))));
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            L Lv = ldot3(uq[q], gV[i], gVp[i]);
            if constexpr (NT == 1) {
                // + cs v_q: v at quadrature point q is qb sum_a v_a + qd v_q (barycentric weights)
                const L vq = lfma(lsplat<L>(T(kQA - kQB)), vn[q][i],
                                  lmul(lsplat<L>(T(kQB)), ladd(ladd(vn[0][i], vn[1][i]), ladd(vn[2][i], vn[3][i]))));
                Lv = lfma(lsplat<L>(cs), vq, Lv);
            }
            const L X = lmul(tau, Lv);
            S[i] = q == 0 ? X : ladd(S[i], X);
#pragma unroll
            for (int j = 0; j < 3; ++j) Mx[j][i] = q == 0 ? lmul(uq[q][j], X) : lfma(uq[q][j], X, Mx[j][i]);
        }
    }

    const T w = V * T(0.25);
    T *go[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) go[a] = gout + size_t(uint32_t(sNode[lo[a]]) & ~kDirBit) * N4 + n0;
    // continuity rows: w div v + (w / rho) grad N_a . sum_q X_q (Eq. K_mat, G and D blocks)
    {
        const L wdiv = lmul(lsplat<L>(w), ladd(gV[0][0], ladd(gV[1][1], gV[2][2])));
        L Sw[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) Sw[i] = lmul(lsplat<L>(w), S[i]);
        L gS[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) gS[a] = ldot3(gN[a], Sw);
        if constexpr (DET) {
            lstore(cslot + 3 * N + n0, lsub(wdiv, ladd(gS[0], ladd(gS[1], gS[2]))), d1);
#pragma unroll
            for (int a = 0; a < 3; ++a) lstore(cslot + (4 * (a + 1) + 3) * N + n0, ladd(wdiv, gS[a]), d1);
        } else {
            lred(go[0] + 3 * N, lsub(wdiv, ladd(gS[0], ladd(gS[1], gS[2]))), d1);
#pragma unroll
            for (int a = 0; a < 3; ++a) lred(go[a + 1] + 3 * N, ladd(wdiv, gS[a]), d1);
        }
    }
    // Z[j][i] = w rho Mx[j][i] + mu V d_j v_i - V pbar delta_ij
    {
        const L wr = lsplat<L>(w * rho), muV = lsplat<L>(mu * V);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) Mx[j][i] = lfma(wr, Mx[j][i], lmul(muV, gV[i][j]));
#pragma unroll
        for (int i = 0; i < 3; ++i) Mx[i][i] = lsub(Mx[i][i], pbar);
    }
    // momentum rows
    const L m20 = lsplat<L>(V * T(0.05));                  // int N_a N_b = V (1 + delta_ab) / 20
    const L kb = lsplat<L>(w * rho * T(kQB)), kd = lsplat<L>(w * rho * T(kQA - kQB));
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        L Wa[4];
        const int rW0 = i * N + n0;
#pragma unroll
        for (int a = 0; a < 4; ++a) Wa[a] = lload<L>(sW + lo[a] * WS + rW0, d1);
        const L Wsum = ladd(ladd(Wa[0], Wa[1]), ladd(Wa[2], Wa[3]));
        const L cW = lfma(kb, Ug[i], lmul(m20, Wsum));
        const L Zi[3] = {Mx[0][i], Mx[1][i], Mx[2][i]};
        L gz[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) gz[a] = ldot3(gN[a], Zi);
        const L gz0 = ladd(gz[0], ladd(gz[1], gz[2]));
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            L val = a == 0 ? lsub(cW, gz0) : ladd(cW, gz[a - 1]);
            val = lfma(kd, ldot3(uq[a], gV[i]), val);
            val = lfma(m20, Wa[a], val);
            // prescribed velocity rows are set apart (the deterministic gather skips them)
            if constexpr (DET) lstore(cslot + (4 * a + i) * N + n0, val, d1);
            else if (PIPE ? vfree[a] : sNode[lo[a]] >= 0) lred(go[a] + i * N, val, d1);
        }
    }
}

// NT > 0: the number of instances is the compile-time constant NT; NT = 0: runtime N
// rbvms (RES, JVE): full RBVMS (Sec. 2.2, remark 2 after Eq. tau): with u' = -tau L / rho added to the
// advecting velocity the momentum rows gain the cross stress - int N_a (tau L . grad) u_i and the Reynolds
// stress - int (1 / rho) (tau L . grad N_a) (tau L)_i (and their derivatives in JVE).
template <typename T, int MODE, int NT, bool DET = false>
__device__ __forceinline__ void element_instance(int e, int n, int Nrt, T rho, T mu, T shift, T omega2, int rbvms,
                                                 const T *__restrict__ sGeom,
                                                 const uint32_t *__restrict__ sConn,
                                                 const T *__restrict__ sY, const T *__restrict__ sV,
                                                 const T *__restrict__ sHY, const T *__restrict__ sHV,
                                                 const int *__restrict__ sNode, T *__restrict__ gout,
                                                 T *sT, T *__restrict__ cslot = nullptr) {
    const int N = NT > 0 ? NT : Nrt;
    const int N4 = 4 * N, N3 = 3 * N;
    const uint32_t c = sConn[e];
    const int lo[4] = {int(c & 255u), int((c >> 8) & 255u), int((c >> 16) & 255u), int(c >> 24)};
    // global rows of the 4 nodes at this instance: contributions without instance coupling are added
    // there directly (native global reductions)
    T *go[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) go[a] = gout + size_t(uint32_t(sNode[lo[a]]) & ~kDirBit) * N4 + n;
    T gN[4][3], V, g2;
    load_geom(sGeom + e * kGeomStride, gN, V, g2);
    g2 += omega2;                 // tau_hat (Eq. tauhat) of the time-domain passes; 0 for HB
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
            if constexpr (DET) {
                T *cs = cslot + 4 * a * N + n;
                cs[0] = cs[N] = cs[2 * N] = dv;
                cs[3 * N] = dp;
                continue;
            }
            if (sNode[lo[a]] >= 0) {            // prescribed velocity rows are set apart
                atomicAdd(go[a], dv);
                atomicAdd(go[a] + N, dv);
                atomicAdd(go[a] + 2 * N, dv);
            }
            atomicAdd(go[a] + 3 * N, dp);
        }
        return;
    } else if constexpr (MODE == MODE_RES || MODE == MODE_TRES) {
        // HB: hu = (H u) at the nodes, T = rho M u - int N tau L goes through H at the flush.
        // Time domain (TRES): hu = du/dt, and the Galerkin term rho M du/dt is added directly.
        constexpr bool TM = MODE == MODE_TRES;
        T p[4], hu[4][3];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            p[a] = sY[lo[a] * N4 + 3 * N + n];
#pragma unroll
            for (int i = 0; i < 3; ++i) hu[a][i] = TM ? sV[lo[a] * N4 + i * N + n] : sHY[lo[a] * N3 + i * N + n];
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
            if (!TM && rbvms) {
                T ctL[3], tdN[4];
#pragma unroll
                for (int i = 0; i < 3; ++i) ctL[i] = tL[0] * gU[i][0] + tL[1] * gU[i][1] + tL[2] * gU[i][2];
#pragma unroll
                for (int a = 0; a < 4; ++a) tdN[a] = tL[0] * gN[a][0] + tL[1] * gN[a][1] + tL[2] * gN[a][2];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int i = 0; i < 3; ++i)
                        qm[a][i] -= w * ((a == q ? qb + qd : qb) * ctL[i] + tdN[a] * tL[i] / rho);
            }
        }
        const T pbar = T(0.25) * (p[0] + p[1] + p[2] + p[3]);
        const T div = gU[0][0] + gU[1][1] + gU[2][2];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const T visc = gN[a][0] * gU[i][0] + gN[a][1] * gU[i][1] + gN[a][2] * gU[i][2];
                T vq = qm[a][i] + w * rho * qb * convs[i] + mu * V * visc - V * gN[a][i] * pbar;
                if constexpr (DET) {
                    if constexpr (TM) {
                        cslot[(4 * a + i) * N + n] = vq + rho * m20 * (husum[i] + hu[a][i]);
                    } else {
                        cslot[(7 * a + i) * N + n] = vq;
                        cslot[(7 * a + 4 + i) * N + n] = tt[a][i] + rho * m20 * (usum[i] + u[a][i]) - w * qb * S[i];
                    }
                    continue;
                }
                if (sNode[lo[a]] >= 0) {        // prescribed velocity rows are set apart
                    if constexpr (TM) {
                        vq += rho * m20 * (husum[i] + hu[a][i]);
                        atomicAdd(go[a] + i * N, vq);
                    } else {
                        const T vt = tt[a][i] + rho * m20 * (usum[i] + u[a][i]) - w * qb * S[i];
                        atomicAdd(go[a] + i * N, vq);
                        atomicAdd(sT + lo[a] * N3 + i * N + n, vt);
                    }
                }
            }
            const T qc = w * div + (w / rho) * (gN[a][0] * S[0] + gN[a][1] * S[1] + gN[a][2] * S[2]);
            if constexpr (DET) cslot[((TM ? 4 : 7) * a + 3) * N + n] = qc;
            else atomicAdd(go[a] + 3 * N, qc);
        }
        return;
    } else {  // MODE_JVE (MODE_JVP runs jvp_lanes)
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
            if (rbvms) {
                T dc[3], tdN[4], dtdN[4];
#pragma unroll
                for (int i = 0; i < 3; ++i)
                    dc[i] = dtL[0] * gU[i][0] + dtL[1] * gU[i][1] + dtL[2] * gU[i][2]
                          + tL[0] * gV[i][0] + tL[1] * gV[i][1] + tL[2] * gV[i][2];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    tdN[a] = tL[0] * gN[a][0] + tL[1] * gN[a][1] + tL[2] * gN[a][2];
                    dtdN[a] = dtL[0] * gN[a][0] + dtL[1] * gN[a][1] + dtL[2] * gN[a][2];
                }
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int i = 0; i < 3; ++i)
                        qm[a][i] -= w * ((a == q ? qb + qd : qb) * dc[i] + (dtdN[a] * tL[i] + tdN[a] * dtL[i]) / rho);
            }
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
                if constexpr (DET) {
                    cslot[(7 * a + i) * N + n] = vq;
                    cslot[(7 * a + 4 + i) * N + n] = vt;
                    continue;
                }
                if (sNode[lo[a]] >= 0) {        // prescribed velocity rows are set apart
                    atomicAdd(go[a] + i * N, vq);
                    atomicAdd(sT + lo[a] * N3 + i * N + n, vt);
                }
            }
            const T qc = w * div + (w / rho) * (gN[a][0] * S[0] + gN[a][1] * S[1] + gN[a][2] * S[2]);
            if constexpr (DET) cslot[(7 * a + 3) * N + n] = qc;
            else atomicAdd(go[a] + 3 * N, qc);
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
__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gmem_src) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Copy patch p's slot into shared memory (issued by one thread; completion: that thread's
// cp_async_wait_all, then a block barrier).
__device__ __forceinline__ void stage_slot(const int *slots, int stride, int p, int *dst) {
    const int4 *src = reinterpret_cast<const int4 *>(slots + size_t(p) * stride);
    for (int i = 0; i < stride / 4; ++i) cp_async16(dst + 4 * i, src + i);
}

// Prefetch of the next patch's slot, run by patch_pass on every thread (thread 0 issues the copies).
struct SlotPrefetch {
    const int *slots;
    int stride, next, n_patches;
    int *dst;
    __device__ __forceinline__ void operator()() const {
        if (threadIdx.x == 0 && next < n_patches) stage_slot(slots, stride, next, dst);
    }
};

// H is circulant: H[j][k] = h[(j - k) mod N] with h its first column (h[0] = 0).  For a fixed N one row
// of N values is multiplied with the kernel held in registers; x_in may equal x_out (read fully first).
// With SCALED, x_out = alpha (H x) + beta x.
template <typename T, int NT, bool SCALED = false>
__device__ __forceinline__ void circulant_row(const T *__restrict__ hcol, const T *x_in, T *x_out,
                                              T alpha = T(1), T beta = T(0)) {
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
        x_out[m] = SCALED ? alpha * acc + beta * x[m] : acc;
    }
}

// Shared-memory pointers of one patch pass.
template <typename T>
struct PatchSmem {
    T *H, *geom, *Y, *V, *HY, *HV, *T_;
    int *slot0;                    // slot buffer b at slot0 + b * slot_cap
    int slot_cap;
    uint32_t *conn;
    __device__ __forceinline__ int *slot(int b) const { return slot0 + b * slot_cap; }
};

template <typename T, int MODE>
__device__ __forceinline__ PatchSmem<T> patch_smem(unsigned char *smem, int N, int nl_max, int ep_max,
                                                   int slot_cap = 0) {
    const Layout L = make_layout(MODE, N, nl_max, ep_max, sizeof(T), slot_cap);
    PatchSmem<T> m;
    m.H = reinterpret_cast<T *>(smem + L.H);
    m.geom = reinterpret_cast<T *>(smem + L.geom);
    m.Y = reinterpret_cast<T *>(smem + L.Y);
    m.V = reinterpret_cast<T *>(smem + L.V);
    m.HY = reinterpret_cast<T *>(smem + L.HY);
    m.HV = reinterpret_cast<T *>(smem + L.HV);
    m.T_ = reinterpret_cast<T *>(smem + L.T);
    m.slot0 = reinterpret_cast<int *>(smem + L.node);
    m.slot_cap = slot_cap > 0 ? slot_cap : slot_ints(nl_max);
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

// One patch whose slot is staged in sSlot: gather, Dirichlet masking, in-patch H products,
// element-instance work, H T flush.  `prefetch` runs on every thread once the staged rows are no longer
// being written (the caller uses it to stage the next patch's slot).  Ends with a block barrier, so
// shared memory can be reused by the next patch.
template <typename T, int MODE, int NT, typename L, typename Prefetch, bool DET = false>
__device__ __forceinline__ void patch_pass(const ElemArgs<T> &a, const PatchSmem<T> &sm, const int *sSlot, T shift,
                                           Prefetch prefetch) {
    const int N = NT > 0 ? NT : a.N, N4 = 4 * N, N3 = 3 * N;
    T *sH = sm.H, *sGeom = sm.geom, *sY = sm.Y, *sV = sm.V, *sHY = sm.HY, *sHV = sm.HV, *sT = sm.T_;
    uint32_t *sConn = sm.conn;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int e0 = sSlot[0], ne = sSlot[1], nl = sSlot[2], nd = sSlot[3];
    const int *sNode = sSlot + 4;           // global node ids, kDirBit on prescribed velocities
    if constexpr ((MODE == MODE_RES || MODE == MODE_JVE) && !DET)
        for (int i = tid; i < nl * N3; i += nt) sT[i] = T(0);

    // asynchronous copies of the patch's element data and node rows (4 N values per node), so every
    // thread keeps all of its loads in flight
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.pv.geom + size_t(e0) * kGeomStride);
        uint4 *dst = reinterpret_cast<uint4 *>(sGeom);
        const int nvec = int(ne * kGeomStride * sizeof(T) / 16);
        for (int i = tid; i < nvec; i += nt) cp_async16(dst + i, src + i);
        for (int i = tid; i < ne; i += nt) cp_async4(sConn + i, a.pv.lconn + e0 + i);
    }
    constexpr int VPC = int(16 / sizeof(T));       // values per 16-byte chunk
    const int cpr = N4 / VPC;
    for (int i = tid; i < nl * cpr; i += nt) {
        const int l = i / cpr, c = i - l * cpr;
        const size_t gidx = size_t(uint32_t(sNode[l]) & ~kDirBit) * cpr + c;
        cp_async16(reinterpret_cast<uint4 *>(sY) + i, reinterpret_cast<const uint4 *>(a.y) + gidx);
        if constexpr (MODE == MODE_JVP || MODE == MODE_JVE || MODE == MODE_TRES)
            cp_async16(reinterpret_cast<uint4 *>(sV) + i, reinterpret_cast<const uint4 *>(a.v) + gidx);
    }
    if constexpr (MODE == MODE_JVP) {
        if (a.W) {              // W = shift v + rho H v from the global spectral pass
            const int wpr = w_stride(N, int(sizeof(T))) * int(sizeof(T)) / 16;
            for (int i = tid; i < nl * wpr; i += nt) {
                const int l = i / wpr, c = i - l * wpr;
                const size_t gidx = size_t(uint32_t(sNode[l]) & ~kDirBit) * wpr + c;
                cp_async16(reinterpret_cast<uint4 *>(sHV) + i, reinterpret_cast<const uint4 *>(a.W) + gidx);
            }
        }
    }
    cp_async_wait_all();
    if constexpr (MODE == MODE_JVP || MODE == MODE_JVE) {
        // prescribed velocity entries of the direction are not unknowns: each thread zeroes them in the
        // chunks it copied itself (complete after its own wait)
        if (nd > 0) {
            for (int i = tid; i < nl * cpr; i += nt) {
                const int l = i / cpr;
                if (sNode[l] >= 0) continue;
                const int c = i - l * cpr;
#pragma unroll
                for (int j = 0; j < VPC; ++j)
                    if (c * VPC + j < N3) sV[l * N4 + c * VPC + j] = T(0);
            }
        }
    }
    __syncthreads();
    if (MODE != MODE_DIAG && MODE != MODE_TRES && !(MODE == MODE_JVP && a.W)) {
        // time coupling of the staged velocities: (H x)[l][i][n] = sum_k H[n][k] x[l][i][k] for
        // x = u (RES, JVE) and x = v (JVP, JVE)
        constexpr bool hy = (MODE == MODE_RES || MODE == MODE_JVE);
        constexpr bool hv = (MODE == MODE_JVP || MODE == MODE_JVE);
        constexpr int nsrc = (hy ? 1 : 0) + (hv ? 1 : 0);
        if constexpr (NT > 0 && MODE == MODE_JVP) {
            // JVP stages W = shift v + rho H v (the mass-matrix terms of the tangent)
            const int WS = w_stride(N, int(sizeof(T)));
            for (int r = tid; r < nl * 3; r += nt) {
                const int l = r / 3, f = r - 3 * l;
                circulant_row<T, NT, true>(sH, sV + l * N4 + f * N, sHV + l * WS + f * N, a.rho, shift);
            }
        } else if constexpr (NT > 0) {
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
                    if constexpr (MODE == MODE_JVP) sHV[l * w_stride(N, int(sizeof(T))) + r] = a.rho * acc2 + shift * xv[n];
                    else sHV[i] = acc2;
                }
            }
        }
        __syncthreads();
    }

    prefetch();
    // prescribed velocity rows of the output (no element or face term reaches them): 0 for the
    // residual (left from the clearing), 1 for the Jacobi diagonal, v (identity) for Jacobian products;
    // patches sharing a node store the same values
    if constexpr (MODE != MODE_RES && MODE != MODE_TRES && !DET) {
        if (nd > 0) {
            for (int i = tid; i < nl * N3; i += nt) {
                const int l = i / N3;
                if (sNode[l] >= 0) continue;
                const size_t g = size_t(uint32_t(sNode[l]) & ~kDirBit) * N4 + (i - l * N3);
                a.out[g] = MODE == MODE_DIAG ? T(1) : a.v[g];
            }
        }
    }
    if constexpr (MODE == MODE_JVP) {
        // a thread takes instances k and k + NP of one element (FP32 pairs; FP64: NP = N, one instance)
        constexpr int LW = int(sizeof(L) / sizeof(T));
        const int NP = (N + LW - 1) / LW;
        for (int i = tid; i < ne * NP; i += nt) {
            const int e = i / NP, k = i - e * NP;
            const int d1 = (LW == 2 && k + NP < N) ? NP : 0;
            jvp_lanes<T, L, NT, false, DET>(e, k, d1, N, a.rho, a.mu, a.omega2, a.ls_mass ? shift / a.rho : T(0), sGeom,
                                            sConn, sY, sV, sHV, sNode, a.out,
                                            DET ? a.cbuf + (size_t(e0) + size_t(e)) * 16 * size_t(N) : nullptr);
        }
    } else {
        for (int i = tid; i < ne * N; i += nt) {
            const int e = i / N, n = i - e * N;
            element_instance<T, MODE, NT, DET>(e, n, N, a.rho, a.mu, shift, a.omega2, a.rbvms, sGeom, sConn, sY, sV,
                                               sHY, sHV, sNode, a.out, sT,
                                               DET ? a.cbuf + (size_t(e0) + size_t(e)) * size_t(det_slot_values(MODE)) * N
                                                   : nullptr);
        }
    }
    __syncthreads();

    // H T on the patch-assembled T rows (fixed N: in place, one row per thread)
    if constexpr ((MODE == MODE_RES || MODE == MODE_JVE) && NT > 0 && !DET) {
        for (int r = tid; r < nl * 3; r += nt) {
            T *row = sT + (r / 3) * N3 + (r % 3) * N;
            circulant_row<T, NT>(sH, row, row);
        }
        __syncthreads();
    }

    // flush: out += H T on the velocity rows, once per local node
    if constexpr ((MODE == MODE_RES || MODE == MODE_JVE) && !DET) {
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
            if (sNode[l] >= 0) atomicAdd(a.out + size_t(sNode[l]) * N4 + r, val);
        }
    }
    __syncthreads();
}

// Persistent element pass: block b takes patches b, b + G, b + 2G, ... (G = gridDim.x) and stages each
// next patch's slot while the current one computes.
template <typename T, int MODE, int NT, int VAR, bool DET = false>
__global__ void __launch_bounds__(ElemCfg<T, VAR>::block, ElemCfg<T, VAR>::minb) elem_kernel(ElemArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = NT > 0 ? NT : a.N;
    const PatchSmem<T> sm = patch_smem<T, MODE>(smem, N, a.pv.nl_max, a.pv.ep_max);
    const T shift = a.shift_dev ? T(*a.shift_dev) : a.shift;
    int p = blockIdx.x;
    const int P = a.pv.n_patches;
    if (p >= P) return;
    stage_H<T, NT>(a, sm.H, N);
    if (threadIdx.x == 0) stage_slot(a.pv.slots, a.pv.slot_stride, p, sm.slot(0));
    cp_async_wait_all();
    __syncthreads();
    for (int cur = 0; p < P; p += gridDim.x, cur ^= 1) {
        const SlotPrefetch pf{a.pv.slots, a.pv.slot_stride, p + int(gridDim.x), P, sm.slot(cur ^ 1)};
        patch_pass<T, MODE, NT, typename ElemCfg<T, VAR>::lane, SlotPrefetch, DET>(a, sm, sm.slot(cur), shift, pf);
        cp_async_wait_all();
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------------------
// Pipelined paper-tangent pass (FP32, fixed N, W given): one producer warp and C consumer warps per block,
// one block per SM, two patch stages in shared memory.  The producer copies a patch's slot, element
// geometry (with the packed local connectivity in slot 14) and node rows of y, v and W into a free stage
// with 1-D bulk asynchronous copies (cp.async.bulk) that complete on the stage's "full" mbarrier; the
// consumers wait on it, compute the patch's element-instances and release the stage on its "empty"
// mbarrier.  No block-wide barrier sits in the patch loop: while the consumers work on one stage the
// other is being filled, and consumer warps that finish a patch early go on to the next stage.
//
// Every wait is bounded (kPipeSpinLimit polls); a wait that gives up sets *err (1: a consumer's wait for
// data, 2: the producer's wait for a free stage) and the block leaves the loop; before the producer
// exits it waits, again bounded, until every copy it issued has landed.

constexpr long long kPipeSpinLimit = 1ll << 26;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the phase of the given parity; false if it gave up
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    for (long long i = 0; i < kPipeSpinLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16) completing on bar
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// One stage of the pipelined pass: slot, geometry, y rows, v rows, W rows (each 16-byte aligned).
struct PipeLayout {
    size_t slot, geom, Y, V, W, stage;
};
__host__ __device__ inline PipeLayout pipe_layout(int N, int nl, int ep) {
    PipeLayout L;
    size_t o = 0;
    L.slot = o; o += pad16(size_t(slot_ints(nl)) * 4);
    L.geom = o; o += pad16(size_t(ep) * kGeomStride * 4);
    L.Y = o;    o += pad16(size_t(nl) * 4 * N * 4);
    L.V = o;    o += pad16(size_t(nl) * 4 * N * 4);
    L.W = o;    o += pad16(size_t(nl) * w_stride(N, 4) * 4);
    L.stage = o;
    return L;
}

// PW producer warps: 1 = one warp issuing 1-D bulk copies (cp.async.bulk, completion counted in bytes);
// PW > 1 = PW warps issuing 16-byte cp.async copies spread over all their lanes, each lane signalling the
// stage's barrier once its own copies have landed (cp.async.mbarrier.arrive.noinc).  The bulk form moves a
// patch with ~3 copies per node, which the bulk-copy engine serves at a lower rate than the LSU serves many
// 16-byte copies from 128 lanes.
template <typename L, int NT, int C, int PW>
__global__ void __launch_bounds__((C + PW) * 32, 1) jvp_pipe_kernel(ElemArgs<float> a, int *err) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[2], empty[2];
    constexpr int N = NT, N4 = 4 * N, N3 = 3 * N, WS = w_stride(NT, 4);
    constexpr int LW = int(sizeof(L) / sizeof(float));
    constexpr int NP = (N + LW - 1) / LW;
    const PipeLayout PL = pipe_layout(N, a.pv.nl_max, a.pv.ep_max);
    const int P = a.pv.n_patches, stride = a.pv.slot_stride;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        mbar_init(&full[0], PW == 1 ? 1 : PW * 32);
        mbar_init(&full[1], PW == 1 ? 1 : PW * 32);
        mbar_init(&empty[0], C);
        mbar_init(&empty[1], C);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    __syncthreads();
    if (PW > 1 && warp >= C) {
        // ---- producer warps (16-byte copies)
        const int pt = int(threadIdx.x) - C * 32;
        constexpr int NPT = PW * 32, CPR = N4 / 4, WPR = WS / 4, RPN = 2 * CPR + WPR;
        int issued = -1, k = 0;
        for (int p = int(blockIdx.x); p < P; ++k, p += int(gridDim.x)) {
            const int s = k & 1;
            if (k >= 2 && !mbar_wait_bounded(&empty[s], uint32_t(((k >> 1) - 1) & 1))) {
                if (pt == 0) atomicExch(err, 2);
                break;
            }
            unsigned char *st = smem + size_t(s) * PL.stage;
            const int *gslot = a.pv.slots + size_t(p) * stride;
            const int e0 = gslot[0], ne = gslot[1], nl = gslot[2];
            for (int i = pt; i < stride / 4; i += NPT) cp_async16(st + PL.slot + 16 * size_t(i), gslot + 4 * i);
            const float *gg = a.pv.geom + size_t(e0) * kGeomStride;
            for (int i = pt; i < ne * (kGeomStride / 4); i += NPT) cp_async16(st + PL.geom + 16 * size_t(i), gg + 4 * i);
            for (int i = pt; i < nl * RPN; i += NPT) {
                const int l = i / RPN, c = i - l * RPN;
                const size_t node = size_t(uint32_t(__ldg(gslot + 4 + l)) & ~kDirBit);
                if (c < CPR) cp_async16(st + PL.Y + (size_t(l) * CPR + c) * 16, a.y + node * N4 + 4 * c);
                else if (c < 2 * CPR)
                    cp_async16(st + PL.V + (size_t(l) * CPR + c - CPR) * 16, a.v + node * N4 + 4 * (c - CPR));
                else cp_async16(st + PL.W + (size_t(l) * WPR + c - 2 * CPR) * 16, a.W + node * WS + 4 * (c - 2 * CPR));
            }
            asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(smem_u32(&full[s])) : "memory");
            issued = k;
        }
        cp_async_wait_all();                        // no copy of this thread is in flight at exit
        (void)issued;
        return;
    }
    if (PW == 1 && warp == C) {
        // ---- producer warp.  The next patch's header and node ids are loaded into registers before the
        // wait for a free stage, so their global-load latency overlaps the consumers' work.
        constexpr int IDS = 8;                      // node ids per lane: patches of up to 256 nodes
        int k = 0, issued = -1;
        int p = int(blockIdx.x);
        int e0 = 0, ne = 0, nl = 0, ids[IDS];
        auto load_patch = [&](int q) {
            const int *gs = a.pv.slots + size_t(q) * stride;
            e0 = gs[0];
            ne = gs[1];
            nl = gs[2];
#pragma unroll
            for (int j = 0; j < IDS; ++j) {
                const int l = lane + 32 * j;
                ids[j] = l < a.pv.nl_max ? gs[4 + l] : 0;
            }
        };
        if (p < P) load_patch(p);
        for (; p < P; ++k, p += int(gridDim.x)) {
            const int s = k & 1;
            if (k >= 2 && !mbar_wait_bounded(&empty[s], uint32_t(((k >> 1) - 1) & 1))) {
                if (lane == 0) atomicExch(err, 2);
                break;
            }
            unsigned char *st = smem + size_t(s) * PL.stage;
            const int *gslot = a.pv.slots + size_t(p) * stride;
            const uint32_t bytes = uint32_t(stride) * 4 + uint32_t(ne) * kGeomStride * 4 +
                                   uint32_t(nl) * uint32_t(2 * N4 + WS) * 4;
            if (lane == 0) {
                mbar_arrive_expect_tx(&full[s], bytes);
                bulk_g2s(st + PL.slot, gslot, uint32_t(stride) * 4, &full[s]);
                bulk_g2s(st + PL.geom, a.pv.geom + size_t(e0) * kGeomStride, uint32_t(ne) * kGeomStride * 4, &full[s]);
            }
            __syncwarp();
#pragma unroll
            for (int j = 0; j < IDS; ++j) {
                const int l = lane + 32 * j;
                if (l < nl) {
                    const size_t node = size_t(uint32_t(ids[j]) & ~kDirBit);
                    bulk_g2s(st + PL.Y + size_t(l) * N4 * 4, a.y + node * N4, N4 * 4, &full[s]);
                    bulk_g2s(st + PL.V + size_t(l) * N4 * 4, a.v + node * N4, N4 * 4, &full[s]);
                    bulk_g2s(st + PL.W + size_t(l) * WS * 4, a.W + node * WS, WS * 4, &full[s]);
                }
            }
            issued = k;
            if (p + int(gridDim.x) < P) load_patch(p + int(gridDim.x));
        }
        // every copy this warp issued has landed before the block may exit
        for (int j = (issued >= 1 ? issued - 1 : 0); j <= issued; ++j)
            if (!mbar_wait_bounded(&full[j & 1], uint32_t((j >> 1) & 1)) && lane == 0) atomicExch(err, 3);
        return;
    }
    // ---- consumer warps
    const int ct = threadIdx.x, nct = C * 32;
    for (int k = 0;; ++k) {
        const int p = int(blockIdx.x) + k * int(gridDim.x);
        if (p >= P) break;
        const int s = k & 1;
        if (!mbar_wait_bounded(&full[s], uint32_t((k >> 1) & 1))) {
            if (lane == 0) atomicExch(err, 1);
            return;
        }
        const unsigned char *st = smem + size_t(s) * PL.stage;
        const int *sSlot = reinterpret_cast<const int *>(st + PL.slot);
        const float *sGeom = reinterpret_cast<const float *>(st + PL.geom);
        const float *sY = reinterpret_cast<const float *>(st + PL.Y);
        const float *sV = reinterpret_cast<const float *>(st + PL.V);
        const float *sW = reinterpret_cast<const float *>(st + PL.W);
        const int ne = sSlot[1], nl = sSlot[2], nd = sSlot[3];
        const int *sNode = sSlot + 4;
        // prescribed velocity rows of the output: v (identity rows); patches sharing a node store the
        // same values
        if (nd > 0) {
            for (int i = ct; i < nl * N3; i += nct) {
                const int l = i / N3;
                if (sNode[l] >= 0) continue;
                const int r = i - l * N3;
                a.out[size_t(uint32_t(sNode[l]) & ~kDirBit) * N4 + r] = sV[l * N4 + r];
            }
        }
        for (int i = ct; i < ne * NP; i += nct) {
            const int e = i / NP, kk = i - e * NP;
            const int d1 = (LW == 2 && kk + NP < N) ? NP : 0;
            jvp_lanes<float, L, NT, true>(e, kk, d1, N, a.rho, a.mu, a.omega2, 0.f, sGeom, nullptr, sY, sV, sW,
                                          sNode, a.out);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
}

// Persistent kernel over the patches of several problems with the same instance count.  Work items
// [item_begin, item_end) are taken from a global counter, so problems of uneven size share the SMs; the
// batch slot of item i (bslot_stride ints at bslots + i * bslot_stride) holds the owning problem's index
// in its first int and the patch's own slot from int 4 on.  The next item is claimed, and its slot
// staged, while the current one computes.
struct BatchPrefetch {
    const int *bslots;
    int bslot_stride, item_begin, item_end;
    int *counter, *s_next, *dst;
    __device__ __forceinline__ void operator()() const {
        if (threadIdx.x != 0) return;
        const int item = item_begin + atomicAdd(counter, 1);
        *s_next = item;
        if (item < item_end) stage_slot(bslots, bslot_stride, item, dst);
    }
};

// NT = -1: one launch for members of any instance count; each problem switch dispatches to the pass
// specialised for its N (9, 13, 21) or the generic one.
template <typename T, int MODE, int NT, typename L, typename Prefetch>
__device__ __forceinline__ void batch_patch(const ElemArgs<T> &a, const PatchSmem<T> &sm, const int *slot, T shift,
                                            Prefetch pf) {
    if constexpr (NT >= 0) {
        patch_pass<T, MODE, NT, L>(a, sm, slot, shift, pf);
    } else {
        switch (a.N) {
            case 9: patch_pass<T, MODE, 9, L>(a, sm, slot, shift, pf); break;
            case 13: patch_pass<T, MODE, 13, L>(a, sm, slot, shift, pf); break;
            case 21: patch_pass<T, MODE, 21, L>(a, sm, slot, shift, pf); break;
            default: patch_pass<T, MODE, 0, L>(a, sm, slot, shift, pf); break;
        }
    }
}

template <typename T, int MODE, int NT, int VAR>
__global__ void __launch_bounds__(ElemCfg<T, VAR>::block, ElemCfg<T, VAR>::minb)
    batch_elem_kernel(const ElemArgs<T> *__restrict__ args, const int *__restrict__ bslots, int bslot_stride,
                      int item_begin, int item_end, int *counter) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item[2];
    __shared__ ElemArgs<T> s_args;                 // the current problem's arguments
    // the batch slot buffers sit at the start of every member problem's layout (slot_cap = bslot_stride)
    int *const slot0 = reinterpret_cast<int *>(smem);
    BatchPrefetch{bslots, bslot_stride, item_begin, item_end, counter, &s_item[0], slot0}();
    cp_async_wait_all();
    __syncthreads();
    int last = -1;
    for (int cur = 0;; cur ^= 1) {
        if (s_item[cur] >= item_end) break;
        const int *bslot = slot0 + cur * bslot_stride;
        const int q = bslot[0];
        if (q != last) {
            if (threadIdx.x == 0) s_args = args[q];
            __syncthreads();
        }
        const ElemArgs<T> &a = s_args;
        const int N = NT > 0 ? NT : a.N;
        const PatchSmem<T> sm = patch_smem<T, MODE>(smem, N, a.pv.nl_max, a.pv.ep_max, bslot_stride);
        if (q != last) {
            // fixed N (also inside the all-N launch): the first column of the circulant H; generic: all of H
            const bool fixedN = NT > 0 || (NT < 0 && (N == 9 || N == 13 || N == 21));
            if (fixedN) stage_H<T, 1>(a, sm.H, N);
            else stage_H<T, 0>(a, sm.H, N);
            __syncthreads();
        }
        const T shift = a.shift_dev ? T(*a.shift_dev) : a.shift;
        const BatchPrefetch pf{bslots, bslot_stride, item_begin, item_end, counter, &s_item[cur ^ 1],
                               slot0 + (cur ^ 1) * bslot_stride};
        batch_patch<T, MODE, NT, typename ElemCfg<T, VAR>::lane>(a, sm, bslot + 4, shift, pf);
        cp_async_wait_all();
        __syncthreads();
        last = q;
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

__global__ void pack_conn_kernel(const uint32_t *__restrict__ lconn, float *__restrict__ geom, int n_tets) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n_tets) geom[size_t(e) * kGeomStride + 14] = __uint_as_float(lconn[e]);
}

inline int nblk(int64_t n, int b) { return int((n + b - 1) / b); }

}  // namespace

size_t elem_smem_bytes(int mode, int N, int nl_max, int ep_max, size_t tsize, int slot_cap) {
    return make_layout(mode, N, nl_max, ep_max, tsize, slot_cap).total;
}

// grid: upper bound on the blocks (the patch count); the persistent kernel runs at most one wave
template <typename T, int MODE, int NT, int VAR, bool DET = false>
static void launch_elem_v(const ElemArgs<T> &a, int grid, cudaStream_t s) {
    const size_t smem = elem_smem_bytes(MODE, a.N, a.pv.nl_max, a.pv.ep_max, sizeof(T));
    static LaunchCache cache;
    auto kern = elem_kernel<T, MODE, NT, VAR, DET>;
    grid = std::min(grid, cached_blocks_per_sm(cache, kern, ElemCfg<T, VAR>::block, smem) * device_sms());
    if (grid > 0) kern<<<grid, ElemCfg<T, VAR>::block, smem, s>>>(a);
}

// Pipelined paper-tangent pass (variants 4 and 5): one block per SM; false if it cannot run (no W rows,
// no status word, or two stages do not fit the opt-in shared memory), so the caller falls back.
template <typename L, int NT, int C, int PW>
static bool launch_pipe(const ElemArgs<float> &a, cudaStream_t s) {
    if (!a.W || !a.err || a.pv.n_patches <= 0 || a.pv.nl_max > 256) return false;   // producer holds 256 ids
    const size_t smem = 2 * pipe_layout(NT, a.pv.nl_max, a.pv.ep_max).stage;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (smem + 64 > size_t(optin)) return false;
    static LaunchCache cache;
    auto kern = jvp_pipe_kernel<L, NT, C, PW>;
    const int per = cached_blocks_per_sm(cache, kern, (C + PW) * 32, smem);
    const int grid = std::min(a.pv.n_patches, per * device_sms());
    kern<<<grid, (C + PW) * 32, smem, s>>>(a, a.err);
    return true;
}

template <typename T, int MODE, int NT>
static void launch_elem_n(const ElemArgs<T> &a, int grid, cudaStream_t s) {
    if (a.cbuf) {          // deterministic scatter: FP32 paper tangent one instance per thread (variant 1)
        launch_elem_v<T, MODE, NT, (MODE == MODE_JVP && sizeof(T) == 4) ? 1 : 0, true>(a, grid, s);
        return;
    }
    if constexpr (MODE == MODE_JVP && sizeof(T) == 4 && (NT == 9 || NT == 13 || NT == 21)) {
        // 4: one instance per thread, 20 consumer warps and 4 producer warps (16-byte copies); 5: instance
        // pairs on paired FP32 instructions, 12 consumer warps; 6: as 4 with one producer warp issuing bulk
        // copies.  Without the W rows (or if the stages do not fit) they run variant 1.
        if (a.variant == 4 && launch_pipe<float, NT, 20, 4>(a, s)) return;
        if (a.variant == 5 && launch_pipe<float2, NT, 12, 4>(a, s)) return;
        if (a.variant == 6 && launch_pipe<float, NT, 20, 1>(a, s)) return;
    }
    if constexpr (MODE == MODE_JVP && sizeof(T) == 4) {
        if (a.variant == 1 || a.variant >= 4) {
            launch_elem_v<T, MODE, NT, 1>(a, grid, s);
            return;
        }
        if (a.variant == 2) {
            launch_elem_v<T, MODE, NT, 2>(a, grid, s);
            return;
        }
        if (a.variant == 3) {
            launch_elem_v<T, MODE, NT, 3>(a, grid, s);
            return;
        }
    }
    launch_elem_v<T, MODE, NT, 0>(a, grid, s);
}

// fixed-N instantiations for the instance counts of the workloads; any other N runs the generic kernel
template <typename T, int MODE>
static void launch_elem_mode(const ElemArgs<T> &a, int grid, cudaStream_t s) {
    switch (a.N) {
        case 1: launch_elem_n<T, MODE, 1>(a, grid, s); break;
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
        case MODE_TRES: launch_elem_n<T, MODE_TRES, 1>(a, grid, s); break;   // one time level
        default: launch_elem_mode<T, MODE_DIAG>(a, grid, s); break;
    }
}

template <typename T, int MODE, int VAR>
static void launch_batch_var(const BatchGroup<T> &g, size_t smem, int grid, cudaStream_t s) {
    auto go = [&](auto kern) {
        static LaunchCache cache;
        grid = std::min(grid, cached_blocks_per_sm(cache, kern, ElemCfg<T, VAR>::block, smem) * device_sms());
        kern<<<grid, ElemCfg<T, VAR>::block, smem, s>>>(g.args, g.bslots, g.bslot_stride, g.item_begin, g.item_end,
                                                         g.counter);
    };
    switch (g.N) {
        case -1: go(batch_elem_kernel<T, MODE, -1, VAR>); break;     // every member in one launch
        case 9: go(batch_elem_kernel<T, MODE, 9, VAR>); break;
        case 13: go(batch_elem_kernel<T, MODE, 13, VAR>); break;
        case 21: go(batch_elem_kernel<T, MODE, 21, VAR>); break;
        default: go(batch_elem_kernel<T, MODE, 0, VAR>); break;
    }
}

// the paper-tangent pass in FP32 follows the batch's launch variant; every other pass runs variant 0
template <typename T, int MODE>
static void launch_batch_mode(const BatchGroup<T> &g, size_t smem, int grid, cudaStream_t s) {
    if constexpr (MODE == MODE_JVP && sizeof(T) == 4) {
        if (g.variant == 1 || g.variant >= 4) return launch_batch_var<T, MODE, 1>(g, smem, grid, s);
        if (g.variant == 2) return launch_batch_var<T, MODE, 2>(g, smem, grid, s);
        if (g.variant == 3) return launch_batch_var<T, MODE, 3>(g, smem, grid, s);
    }
    launch_batch_var<T, MODE, 0>(g, smem, grid, s);
}

template <typename T>
void launch_batch_elem(int mode, const BatchGroup<T> &g, size_t smem, int grid, cudaStream_t s) {
    switch (mode) {
        case MODE_RES: launch_batch_mode<T, MODE_RES>(g, smem, grid, s); break;
        case MODE_JVP: launch_batch_mode<T, MODE_JVP>(g, smem, grid, s); break;
        case MODE_JVE: launch_batch_mode<T, MODE_JVE>(g, smem, grid, s); break;
        default: launch_batch_mode<T, MODE_DIAG>(g, smem, grid, s); break;
    }
}

template <typename T>
void launch_geom(const double *xyz, const int *tets, int n_tets, double nu, T *geom, cudaStream_t s) {
    if (n_tets > 0) geom_kernel<T><<<nblk(n_tets, 128), 128, 0, s>>>(xyz, tets, n_tets, nu, geom);
}

void launch_pack_conn(const uint32_t *lconn, float *geom, int n_tets, cudaStream_t s) {
    if (n_tets > 0) pack_conn_kernel<<<nblk(n_tets, 256), 256, 0, s>>>(lconn, geom, n_tets);
}

size_t pipe_smem_bytes(int N, int nl_max, int ep_max) {
    if (N != 9 && N != 13 && N != 21) return 0;
    return 2 * pipe_layout(N, nl_max, ep_max).stage;
}

template void launch_elem<float>(int, const ElemArgs<float> &, int, cudaStream_t);
template void launch_elem<double>(int, const ElemArgs<double> &, int, cudaStream_t);
template void launch_batch_elem<float>(int, const BatchGroup<float> &, size_t, int, cudaStream_t);
template void launch_batch_elem<double>(int, const BatchGroup<double> &, size_t, int, cudaStream_t);
template void launch_geom<float>(const double *, const int *, int, double, float *, cudaStream_t);
template void launch_geom<double>(const double *, const int *, int, double, double *, cudaStream_t);

}  // namespace hb
