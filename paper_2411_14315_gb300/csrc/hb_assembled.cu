// Assembled ("condensed") paper tangent of the HB-GLS method (arXiv 2411.14315, Sec. 2.3 and Sec. 4):
// the blocks K, G, D, L of Eqs. (K_mat), (ctangent) stored per node pair and instance, so that a
// Jacobian-vector product becomes a row-wise sparse product that streams the stored coefficients.
//
// Per node pair (A, B) and instance n eight values, [pair][8][N]:
//   0    K_AB   = int rho N_A u.grad N_B + mu grad N_A . grad N_B + rho tau (u.grad N_A)(u.grad N_B)
//   1-3  G_AB,i = - int dN_A/dx_i N_B + int (u.grad N_A) tau dN_B/dx_i
//   4-6  D_AB,j =   int N_A dN_B/dx_j + int dN_A/dx_j tau (u.grad N_B)
//   7    L_AB   = (1 / rho) int tau grad N_A . grad N_B
// with U and tau frozen at the state of the assembly (the paper's tangent), and per pair the consistent
// mass M_AB, instance independent.  The F block rho M (H v) and the pseudo-time mass shift M v enter as
// M_AB W_B with W = shift v + rho H v per node (M and H commute).  Prescribed velocities are built in at
// assembly: their rows carry no K, G, M terms (the product writes v there) and their columns no K, D
// terms (v's prescribed entries count as zero).
#include "hb_internal.cuh"

#include <algorithm>

namespace hb {

namespace {

inline int nblk(int64_t n, int b) { return int((n + b - 1) / b); }

template <typename T>
__device__ __forceinline__ T rsqrt_a(T x);
template <>
__device__ __forceinline__ float rsqrt_a<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double rsqrt_a<double>(double x) { return rsqrt(x); }

// One element at one instance: node ids, prescribed flags, shape gradients and the quadrature values
// u_q . grad N_b and tau_q of the frozen state.
template <typename T>
struct AsmElem {
    bool dir[4];
    T gN[4][3], V, w;
    T udN[4][4], tau[4];           // udN[q][b] = u_q . grad N_b
};

template <typename T>
__device__ __forceinline__ void asm_elem_load(const AsmArgs<T> &a, int64_t e, int n, AsmElem<T> &s) {
    const int N = a.N, N4 = 4 * N;
    int nd[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        nd[k] = a.tets[4 * e + k];
        s.dir[k] = a.flag[nd[k]] & 1;
    }
    const T *g = a.geom + e * kGeomStride;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) s.gN[k][j] = g[3 * k + j];
    s.V = g[12];
    s.w = s.V * T(0.25);
    const T g2 = g[13] + a.omega2;
    T u[4][3];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) u[k][j] = a.y[int64_t(nd[k]) * N4 + j * N + n];
    const T qa = T(kQA), qb = T(kQB);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        T uq[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) uq[j] = qb * (u[0][j] + u[1][j] + u[2][j] + u[3][j]) + (qa - qb) * u[q][j];
#pragma unroll
        for (int b = 0; b < 4; ++b) s.udN[q][b] = uq[0] * s.gN[b][0] + uq[1] * s.gN[b][1] + uq[2] * s.gN[b][2];
        s.tau[q] = rsqrt_a<T>(s.udN[q][1] * s.udN[q][1] + s.udN[q][2] * s.udN[q][2] + s.udN[q][3] * s.udN[q][3] + g2);
    }
}

// The (ra, cb) block of one element at one instance added into the pair slot c (stride N between the
// 8 values): global reductions, or plain read-modify-write where the calling thread owns the row.
template <typename T, bool OWN>
__device__ __forceinline__ void asm_pair(const AsmElem<T> &s, int ra, int cb, T rho, T mu, T *c, int N) {
    const T qa = T(kQA), qb = T(kQB), w = s.w;
    T kgal = 0, ksupg = 0, gs = 0, ds = 0, lt = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const T Na = (q == ra) ? qa : qb;
        kgal += Na * s.udN[q][cb];
        ksupg += s.tau[q] * s.udN[q][ra] * s.udN[q][cb];
        gs += s.tau[q] * s.udN[q][ra];             // times dN_B/dx_i
        ds += s.tau[q] * s.udN[q][cb];             // times dN_A/dx_j
        lt += s.tau[q];
    }
    const T gg = s.gN[ra][0] * s.gN[cb][0] + s.gN[ra][1] * s.gN[cb][1] + s.gN[ra][2] * s.gN[cb][2];
    auto add = [&](T *p, T v) {
        if constexpr (OWN) *p += v;
        else atomicAdd(p, v);
    };
    if (!s.dir[ra]) {
        if (!s.dir[cb]) add(c, w * rho * kgal + mu * s.V * gg + w * rho * ksupg);
#pragma unroll
        for (int j = 0; j < 3; ++j) add(c + (1 + j) * N, -w * s.gN[ra][j] + w * gs * s.gN[cb][j]);
    }
    if (!s.dir[cb]) {
#pragma unroll
        for (int j = 0; j < 3; ++j) add(c + (4 + j) * N, w * s.gN[cb][j] + w * ds * s.gN[ra][j]);
    }
    add(c + 7 * N, (w / rho) * lt * gg);
}

// One thread per (element, instance): the element's 16 (a, b) blocks at instance n, reduced into the
// pair slots epos[e][4 a + b] (coalesced over n).
template <typename T>
__global__ void assemble_kernel(AsmArgs<T> a) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int N = a.N;
    if (i >= a.n_tets * int64_t(N)) return;
    const int64_t e = i / N;
    const int n = int(i - e * N);
    AsmElem<T> s;
    asm_elem_load(a, e, n, s);
    const int *pos = a.epos + e * 16;
#pragma unroll
    for (int ra = 0; ra < 4; ++ra)
#pragma unroll
        for (int cb = 0; cb < 4; ++cb)
            asm_pair<T, false>(s, ra, cb, a.rho, a.mu, a.coef + int64_t(pos[4 * ra + cb]) * 8 * N + n, N);
}

// Deterministic assembly: one thread per (row node A, instance) owns row A at that instance and adds the
// row-A blocks of A's elements in the fixed order of the list rslot[rptr[A] .. rptr[A + 1]) (entries
// element x 4 + local index of A); no two threads write one value.
template <typename T>
__global__ void assemble_rows_kernel(AsmArgs<T> a) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int N = a.N;
    if (i >= a.n_nodes * int64_t(N)) return;
    const int64_t A = i / N;
    const int n = int(i - A * N);
    for (int k = a.rptr[A]; k < a.rptr[A + 1]; ++k) {
        const int64_t e = a.rslot[k] >> 2;
        const int ra = a.rslot[k] & 3;
        AsmElem<T> s;
        asm_elem_load(a, e, n, s);
        const int *pos = a.epos + e * 16 + 4 * ra;
#pragma unroll
        for (int cb = 0; cb < 4; ++cb)
            asm_pair<T, true>(s, ra, cb, a.rho, a.mu, a.coef + int64_t(pos[cb]) * 8 * N + n, N);
    }
}

// Consistent mass per pair, int N_A N_B = V (1 + delta_ab) / 20, rows of prescribed velocity left out.
template <typename T>
__global__ void assemble_mass_kernel(AsmArgs<T> a) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= a.n_tets) return;
    const T V = a.geom[e * kGeomStride + 12];
    for (int ra = 0; ra < 4; ++ra) {
        if (a.flag[a.tets[4 * e + ra]] & 1) continue;
        for (int cb = 0; cb < 4; ++cb) atomicAdd(a.mass + a.epos[e * 16 + 4 * ra + cb], V * T(ra == cb ? 0.1 : 0.05));
    }
}

// The same by rows in list order (deterministic)
template <typename T>
__global__ void assemble_mass_rows_kernel(AsmArgs<T> a) {
    const int64_t A = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (A >= a.n_nodes || (a.flag[A] & 1)) return;
    for (int k = a.rptr[A]; k < a.rptr[A + 1]; ++k) {
        const int64_t e = a.rslot[k] >> 2;
        const int ra = a.rslot[k] & 3;
        const T V = a.geom[e * kGeomStride + 12];
        for (int cb = 0; cb < 4; ++cb) a.mass[a.epos[e * 16 + 4 * ra + cb]] += V * T(ra == cb ? 0.1 : 0.05);
    }
}

// W = shift v + rho H v on the velocity rows of every node (the F block rho M (H v) of Eq. F_mat and the
// pseudo-time mass of Sec. 2.3 enter the tangent as M W), 0 on prescribed velocities and in the row
// padding.  A block stages NB nodes of v in shared memory with 16-byte loads (a node's 4N values are a
// multiple of 16 bytes), one thread per (node, field) row forms its N outputs, and the block writes the
// padded W rows back contiguously.  H is circulant, so for fixed N its first column H[d][0] is the whole
// operator, held in registers.
template <typename T, int NT>
struct SpecTile {
    static constexpr int NB = (sizeof(T) == 4 ? 64 : 32) / (NT == 0 ? 2 : 1);   // nodes per block
    static constexpr int NM = NT > 0 ? NT : kMaxN;
    static constexpr int PER = 16 / int(sizeof(T));                              // values per 16 bytes
    static constexpr int WP = w_stride(NM, int(sizeof(T))) + PER;                // shared row pitch (16 B
                                                                                  // aligned, skewed banks)
    static constexpr int MINB = sizeof(T) == 4 ? 8 : 1;  // FP32: 8 resident blocks; FP64: no register cap
};

template <typename T, int NT>
__global__ void __launch_bounds__(3 * SpecTile<T, NT>::NB, SpecTile<T, NT>::MINB)
    spectral_w_kernel(const T *__restrict__ v, const T *__restrict__ H, const uint8_t *__restrict__ flag,
                      T *__restrict__ W, int ws, int64_t n_nodes, int Nrt, T rho, T shift,
                      const double *__restrict__ shift_dev) {
    using S = SpecTile<T, NT>;
    // for fixed N each thread holds its row in registers, so the W tile overwrites the staged v tile
    // (half the shared memory, twice the resident blocks); the generic N path keeps two tiles
    constexpr bool inplace = NT > 0;
    constexpr int XS = S::NB * 4 * S::NM, WSZ = S::NB * S::WP;
    __shared__ __align__(16) T sbuf[inplace ? (XS > WSZ ? XS : WSZ) : XS + WSZ];
    T *sx = sbuf, *sw = inplace ? sbuf : sbuf + XS;
    const int N = NT > 0 ? NT : Nrt, N4 = 4 * N, wp = ws + S::PER;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t node0 = int64_t(blockIdx.x) * S::NB;
    const int nn = int(n_nodes - node0 < S::NB ? n_nodes - node0 : S::NB);
    {
        const int chunks = nn * N4 * int(sizeof(T)) / 16;
        const uint4 *src = reinterpret_cast<const uint4 *>(v + node0 * N4);
        uint4 *dst = reinterpret_cast<uint4 *>(sx);
        for (int i = tid; i < chunks; i += nt) dst[i] = src[i];
    }
    const T sh = shift_dev ? T(*shift_dev) : shift;
    __syncthreads();
    const int l = tid / 3, f = tid - 3 * l;
    const bool live = l < nn && !(flag[node0 + l] & 1);
    T *o = sw + l * wp + f * N;
    if constexpr (NT > 0) {
        T xv[NT], h[NT];
        if (live) {
            const T *x = sx + l * N4 + f * N;
#pragma unroll
            for (int k = 0; k < NT; ++k) xv[k] = x[k];
        }
        __syncthreads();                       // every row is in registers before the tile is overwritten
        if (live) {
#pragma unroll
            for (int d = 0; d < NT; ++d) h[d] = H[d * NT];
#pragma unroll
            for (int m = 0; m < NT; ++m) {
                T acc = T(0);
#pragma unroll
                for (int k = 0; k < NT; ++k)
                    if (k != m) acc += h[(m - k + NT) % NT] * xv[k];
                o[m] = rho * acc + sh * xv[m];
            }
        }
    } else if (live) {
        const T *x = sx + l * N4 + f * N;
        for (int m = 0; m < N; ++m) {
            T acc = T(0);
            for (int k = 0; k < N; ++k) acc += H[m * N + k] * x[k];
            o[m] = rho * acc + sh * x[m];
        }
    }
    if (l < nn) {
        if (!live)
            for (int m = 0; m < N; ++m) o[m] = T(0);
        if (f == 2)
            for (int c = 3 * N; c < ws; ++c) sw[l * wp + c] = T(0);
    }
    __syncthreads();
    // rows of ws values are whole 16-byte chunks; wq is a compile-time constant for fixed N
    const int wq = NT > 0 ? w_stride(NT, int(sizeof(T))) / S::PER : ws / S::PER, pq = wq + 1;
    uint4 *dst = reinterpret_cast<uint4 *>(W + node0 * ws);
    const uint4 *src = reinterpret_cast<const uint4 *>(sw);
    for (int i = tid; i < nn * wq; i += nt) {
        const int r = i / wq;
        dst[i] = src[r * pq + (i - r * wq)];
    }
}

// Tensor-core form of the same pass for FP32 and N = 9, 13, 21.  A block's velocity rows (node, field)
// form X [rows][N], and W = X B with B[k][m] = rho H[m][k] + shift delta_km.  TF32 products on the tensor
// cores (mma.sync m16n8k8, FP32 accumulation) with every operand split into a TF32 head and a TF32 tail,
// x = hi + lo: W = Xlo Bhi + Xhi Blo + Xhi Bhi keeps FP32 accuracy (the dropped Xlo Blo is ~2^-22
// relative).  One warp per 16-row tile; K and the output columns are padded to multiples of 8.
__device__ __forceinline__ uint32_t tf32_bits(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                 "{%8, %9}, {%0, %1, %2, %3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void cpa16(void *smem_dst, const void *gmem_src) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cpa_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cpa_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Persistent over tiles of 64 nodes with two tile buffers: the copies of the block's next tile are in
// flight while the current one is multiplied and written back.
template <int NT>
struct SpecTc {
    static constexpr int NB = 64, ROWS = 3 * NB, TILES = ROWS / 16, TPW = (TILES + 5) / 6;
    static constexpr int N4 = 4 * NT, KP = (NT + 7) / 8 * 8, NS = KP / 8;
    static constexpr int WS = w_stride(NT, 4), WP = WS + 4, WQ = WS / 4, PQ = WP / 4;
    static constexpr int XS = NB * N4 > NB * WP ? NB * N4 : NB * WP;
};

template <int NT>
__global__ void __launch_bounds__(192) spectral_w_tc_kernel(const float *__restrict__ v, const float *__restrict__ H,
                                                            const uint8_t *__restrict__ flag, float *__restrict__ W,
                                                            int64_t n_nodes, float rho, float shift,
                                                            const double *__restrict__ shift_dev) {
    using S = SpecTc<NT>;
    constexpr int NB = S::NB, N4 = S::N4, KP = S::KP, NS = S::NS, TPW = S::TPW;
    constexpr int WS = S::WS, WP = S::WP, WQ = S::WQ, PQ = S::PQ;
    __shared__ __align__(16) float sx[2][S::XS];                  // v tiles; W rows written in place
    __shared__ uint32_t sBh[KP * KP], sBl[KP * KP];               // B as TF32 head and tail, [k][m]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n_tiles = (n_nodes + NB - 1) / NB;
    int64_t t = blockIdx.x;
    if (t >= n_tiles) return;
    const float sh = shift_dev ? float(*shift_dev) : shift;
    for (int i = tid; i < KP * KP; i += 192) {
        const int k = i / KP, m = i - k * KP;
        const float b = (k < NT && m < NT) ? rho * H[m * NT + k] + (k == m ? sh : 0.f) : 0.f;
        const uint32_t hi = tf32_bits(b);
        sBh[i] = hi;
        sBl[i] = tf32_bits(b - __uint_as_float(hi));
    }
    auto load = [&](int64_t tile, int buf) {
        const int64_t n0 = tile * NB;
        const int nn = int(n_nodes - n0 < NB ? n_nodes - n0 : NB);
        const uint4 *src = reinterpret_cast<const uint4 *>(v + n0 * N4);
        uint4 *dst = reinterpret_cast<uint4 *>(sx[buf]);
        for (int i = tid; i < nn * N4 / 4; i += 192) cpa16(dst + i, src + i);
        cpa_commit();
    };
    load(t, 0);
    const int g = lane >> 2, q = lane & 3;
    for (int b = 0; t < n_tiles; t += gridDim.x, b ^= 1) {
        if (t + gridDim.x < n_tiles) load(t + gridDim.x, b ^ 1);
        else cpa_commit();                                         // empty group: uniform counting
        cpa_wait1();                                               // this thread's copies of tile t
        __syncthreads();                                           // everyone's (and B)
        const int64_t node0 = t * NB;
        const int nn = int(n_nodes - node0 < NB ? n_nodes - node0 : NB);
        float *x = sx[b];
        float acc[TPW][NS][4];
#pragma unroll
        for (int u = 0; u < TPW; ++u) {
            const int tile = warp + 6 * u;
#pragma unroll
            for (int j = 0; j < NS; ++j) acc[u][j][0] = acc[u][j][1] = acc[u][j][2] = acc[u][j][3] = 0.f;
            if (tile >= S::TILES) continue;
            // rows past the last node hold stale values; their outputs are never written
            const int r0 = tile * 16 + g, r1 = r0 + 8;
            const float *x0 = x + (r0 / 3) * N4 + (r0 % 3) * NT;
            const float *x1 = x + (r1 / 3) * N4 + (r1 % 3) * NT;
#pragma unroll
            for (int ks = 0; ks < NS; ++ks) {
                const int k0 = ks * 8 + q, k1 = k0 + 4;
                const float av[4] = {k0 < NT ? x0[k0] : 0.f, k0 < NT ? x1[k0] : 0.f, k1 < NT ? x0[k1] : 0.f,
                                     k1 < NT ? x1[k1] : 0.f};
                uint32_t ah[4], al[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    ah[i] = tf32_bits(av[i]);
                    al[i] = tf32_bits(av[i] - __uint_as_float(ah[i]));
                }
#pragma unroll
                for (int j = 0; j < NS; ++j) {
                    const int c = j * 8 + g;
                    const uint32_t bh0 = sBh[k0 * KP + c], bh1 = sBh[k1 * KP + c];
                    const uint32_t bl0 = sBl[k0 * KP + c], bl1 = sBl[k1 * KP + c];
                    mma_tf32(acc[u][j], al, bh0, bh1);
                    mma_tf32(acc[u][j], ah, bl0, bl1);
                    mma_tf32(acc[u][j], ah, bh0, bh1);
                }
            }
        }
        __syncthreads();                                           // every v row read: W overwrites it
#pragma unroll
        for (int u = 0; u < TPW; ++u) {
            const int tile = warp + 6 * u;
            if (tile >= S::TILES) continue;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = tile * 16 + g + 8 * h, l = r / 3, f = r - 3 * l;
                if (l >= nn) continue;
                const bool dir = flag[node0 + l] & 1;
                float *o = x + l * WP + f * NT;
#pragma unroll
                for (int j = 0; j < NS; ++j) {
                    const int m = j * 8 + 2 * q;
                    if (m < NT) o[m] = dir ? 0.f : acc[u][j][2 * h];
                    if (m + 1 < NT) o[m + 1] = dir ? 0.f : acc[u][j][2 * h + 1];
                }
            }
        }
        for (int i = tid; i < nn * (WS - 3 * NT); i += 192) {
            const int l = i / (WS - 3 * NT);
            x[l * WP + 3 * NT + (i - l * (WS - 3 * NT))] = 0.f;    // row padding
        }
        __syncthreads();
        uint4 *dst = reinterpret_cast<uint4 *>(W + node0 * WS);
        const uint4 *src = reinterpret_cast<const uint4 *>(x);
        for (int i = tid; i < nn * WQ; i += 192) {
            const int r = i / WQ;
            dst[i] = src[r * PQ + (i - r * WQ)];
        }
        __syncthreads();                                           // buffer b free for tile t + 2 G
    }
    cpa_wait0();
}

template <int NT>
void launch_spectral_tc(const float *v, const float *H, const uint8_t *flag, float *W, int64_t n_nodes, float rho,
                        float shift, const double *shift_dev, cudaStream_t s) {
    static LaunchCache cache;
    const int grid_cap = device_sms() * cached_blocks_per_sm(cache, spectral_w_tc_kernel<NT>, 192, 0);
    const int64_t tiles = (n_nodes + SpecTc<NT>::NB - 1) / SpecTc<NT>::NB;
    const int grid = int(std::min<int64_t>(tiles, grid_cap));
    spectral_w_tc_kernel<NT><<<grid, 192, 0, s>>>(v, H, flag, W, n_nodes, rho, shift, shift_dev);
}

// out = (assembled tangent) v: one thread per (row, instance), rows_per_block rows of a block; each
// thread sums its row's pairs in registers and stores once (no atomics).  Prescribed velocity rows
// return v.
template <typename T>
__global__ void __launch_bounds__(256) spmv_kernel(SpmvArgs<T> a, int rows_per_block) {
    const int N = a.N, N4 = 4 * N;
    const int r = threadIdx.x / N, n = threadIdx.x - r * N;
    if (r >= rows_per_block) return;
    const int64_t A = int64_t(blockIdx.x) * rows_per_block + r;
    if (A >= a.n_nodes) return;
    T s0 = 0, s1 = 0, s2 = 0, sp = 0;
    const int j1 = a.rowptr[A + 1];
#pragma unroll 4
    for (int j = a.rowptr[A]; j < j1; ++j) {
        const int64_t B = a.col[j];
        const T *c = a.coef + int64_t(j) * 8 * N + n;
        const T *vb = a.v + B * N4 + n;
        const T *wb = a.W + B * a.w_stride + n;
        const T m = a.mass[j];
        const T v0 = vb[0], v1 = vb[N], v2 = vb[2 * N], q = vb[3 * N];
        const T K = c[0];
        s0 += K * v0 + c[N] * q + m * wb[0];
        s1 += K * v1 + c[2 * N] * q + m * wb[N];
        s2 += K * v2 + c[3 * N] * q + m * wb[2 * N];
        sp += c[4 * N] * v0 + c[5 * N] * v1 + c[6 * N] * v2 + c[7 * N] * q;
    }
    T *o = a.out + A * N4 + n;
    if (a.flag[A] & 1) {
        const T *va = a.v + A * N4 + n;
        o[0] = va[0];
        o[N] = va[N];
        o[2 * N] = va[2 * N];
    } else {
        o[0] = s0;
        o[N] = s1;
        o[2 * N] = s2;
    }
    o[3 * N] = sp;
}

// Node-block Jacobi preconditioner from the assembled tangent: per node and instance the 4 x 4 diagonal
// block [[(k + s) I, g], [d^T, l]] (k = K_AA, g = G_AA, d = D_AA, l = L_AA, s = shift M_AA; the F block's
// diagonal is rho M_AA H_nn = 0) is inverted through its pressure Schur complement
// l - d . g / (k + s).  z = block^-1 x; prescribed velocities keep z_u = x_u (their rows are the identity).
template <typename T, typename Z>
__global__ void block_jacobi_kernel(const T *__restrict__ coef, const T *__restrict__ mass,
                                    const int *__restrict__ dpos, const uint8_t *__restrict__ flag,
                                    const double *__restrict__ x, Z *__restrict__ z, int64_t n_nodes, int N,
                                    double shift, const double *__restrict__ shift_dev) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n_nodes * N) return;
    const int64_t A = i / N;
    const int n = int(i - A * N);
    const double sh = shift_dev ? *shift_dev : shift;
    const int64_t base = A * 4 * N + n;
    const double r0 = x[base], r1 = x[base + N], r2 = x[base + 2 * N], rp = x[base + 3 * N];
    const T *c = coef + int64_t(dpos[A]) * 8 * N + n;
    const double l = double(c[7 * N]);
    if (flag[A] & 1) {
        z[base] = Z(r0);
        z[base + N] = Z(r1);
        z[base + 2 * N] = Z(r2);
        z[base + 3 * N] = Z(l != 0.0 ? rp / l : rp);
        return;
    }
    const double ks = double(c[0]) + sh * double(mass[dpos[A]]);
    const double g0 = c[N], g1 = c[2 * N], g2 = c[3 * N], d0 = c[4 * N], d1 = c[5 * N], d2 = c[6 * N];
    const double ik = 1.0 / ks;
    const double S = l - (d0 * g0 + d1 * g1 + d2 * g2) * ik;
    const double zp = (rp - (d0 * r0 + d1 * r1 + d2 * r2) * ik) / S;
    z[base] = Z((r0 - g0 * zp) * ik);
    z[base + N] = Z((r1 - g1 * zp) * ik);
    z[base + 2 * N] = Z((r2 - g2 * zp) * ik);
    z[base + 3 * N] = Z(zp);
}

}  // namespace

template <typename T, typename Z>
void launch_block_jacobi(const T *coef, const T *mass, const int *dpos, const uint8_t *flag, const double *x, Z *z,
                         int64_t n_nodes, int N, double shift, const double *shift_dev, cudaStream_t s) {
    const int64_t n = n_nodes * N;
    if (n > 0)
        block_jacobi_kernel<T, Z><<<nblk(n, 256), 256, 0, s>>>(coef, mass, dpos, flag, x, z, n_nodes, N, shift, shift_dev);
}

template <typename T>
void launch_assemble(const AsmArgs<T> &a, cudaStream_t s) {
    if (a.rptr) {
        const int64_t n = a.n_nodes * int64_t(a.N);
        if (n > 0) assemble_rows_kernel<T><<<nblk(n, 128), 128, 0, s>>>(a);
        return;
    }
    const int64_t n = a.n_tets * int64_t(a.N);
    if (n > 0) assemble_kernel<T><<<nblk(n, 128), 128, 0, s>>>(a);
}

template <typename T>
void launch_assemble_mass(const AsmArgs<T> &a, cudaStream_t s) {
    if (a.rptr) {
        if (a.n_nodes > 0) assemble_mass_rows_kernel<T><<<nblk(a.n_nodes, 128), 128, 0, s>>>(a);
        return;
    }
    if (a.n_tets > 0) assemble_mass_kernel<T><<<nblk(a.n_tets, 128), 128, 0, s>>>(a);
}

template <typename T>
void launch_spectral_w(const T *v, const T *H, const uint8_t *flag, T *W, int ws, int64_t n_nodes, int N, T rho,
                       T shift, const double *shift_dev, cudaStream_t s, int path, int *err) {
    if (n_nodes == 0) return;
    if constexpr (sizeof(T) == 4) {
        // FP32 at the compile-time instance counts: the tensor-core forms
        if (path == 0 && launch_spectral_w_tc5(v, H, flag, W, n_nodes, N, rho, shift, shift_dev, err, s)) return;
        if (path <= 1) switch (N) {
            case 9: launch_spectral_tc<9>(v, H, flag, W, n_nodes, rho, shift, shift_dev, s); return;
            case 13: launch_spectral_tc<13>(v, H, flag, W, n_nodes, rho, shift, shift_dev, s); return;
            case 21: launch_spectral_tc<21>(v, H, flag, W, n_nodes, rho, shift, shift_dev, s); return;
            default: break;
        }
    }
#define HB_SPEC(NTV)                                                                                              \
    spectral_w_kernel<T, NTV><<<nblk(n_nodes, SpecTile<T, NTV>::NB), 3 * SpecTile<T, NTV>::NB, 0, s>>>(        \
        v, H, flag, W, ws, n_nodes, N, rho, shift, shift_dev)
    switch (N) {
        case 1: HB_SPEC(1); break;
        case 9: HB_SPEC(9); break;
        case 13: HB_SPEC(13); break;
        case 21: HB_SPEC(21); break;
        default: HB_SPEC(0); break;
    }
#undef HB_SPEC
}

template <typename T>
void launch_spmv(const SpmvArgs<T> &a, cudaStream_t s) {
    const int rpb = a.N <= 256 ? 256 / a.N : 1;
    if (a.n_nodes > 0) spmv_kernel<T><<<nblk(a.n_nodes, rpb), rpb * a.N, 0, s>>>(a, rpb);
}

template void launch_assemble<float>(const AsmArgs<float> &, cudaStream_t);
template void launch_assemble<double>(const AsmArgs<double> &, cudaStream_t);
template void launch_assemble_mass<float>(const AsmArgs<float> &, cudaStream_t);
template void launch_assemble_mass<double>(const AsmArgs<double> &, cudaStream_t);
template void launch_spectral_w<float>(const float *, const float *, const uint8_t *, float *, int, int64_t, int, float,
                                       float, const double *, cudaStream_t, int, int *);
template void launch_spectral_w<double>(const double *, const double *, const uint8_t *, double *, int, int64_t, int,
                                        double, double, const double *, cudaStream_t, int, int *);
template void launch_spmv<float>(const SpmvArgs<float> &, cudaStream_t);
template void launch_block_jacobi<float, float>(const float *, const float *, const int *, const uint8_t *,
                                                const double *, float *, int64_t, int, double, const double *,
                                                cudaStream_t);
template void launch_block_jacobi<float, double>(const float *, const float *, const int *, const uint8_t *,
                                                 const double *, double *, int64_t, int, double, const double *,
                                                 cudaStream_t);
template void launch_block_jacobi<double, double>(const double *, const double *, const int *, const uint8_t *,
                                                  const double *, double *, int64_t, int, double, const double *,
                                                  cudaStream_t);
template void launch_spmv<double>(const SpmvArgs<double> &, cudaStream_t);

}  // namespace hb
