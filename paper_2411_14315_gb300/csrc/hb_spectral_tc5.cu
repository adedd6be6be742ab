// Node-level spectral pass W = shift v + rho H v of the paper's tangent (F block, Eq. F_mat, applied as
// rho M (H v); the pseudo-time shift uses the same mass matrix, Sec. 2.3) on Blackwell's fifth-generation
// tensor cores: tcgen05.mma with the accumulator in tensor memory (TMEM).
//
// The velocity rows of the nodes, (node, field) with N instances each, form X [3 n][N]; W = X B with
// B[k][m] = rho H[m][k] + shift delta_km (H = E^-1 Omega E of Eq. NS-harm, circulant).  A block takes
// tiles of 128 rows: the rows are loaded with coalesced global loads, split into a TF32 head and tail
// (x = hi + lo) and written in the canonical no-swizzle K-major layout of the MMA operands (core matrices
// of 8 rows x 16 bytes); one elected thread issues the products Xlo Bhi + Xhi Blo + Xhi Bhi (the dropped
// Xlo Blo is ~2^-22 relative, so the result keeps FP32 accuracy) into a 128 x NC FP32 accumulator in TMEM
// and commits them to an mbarrier; the four warps then read their 32 TMEM lanes (rows) back with
// tcgen05.ld and store W, zero on nodes whose velocity is prescribed.  K = N is padded with zero columns
// to a multiple of 8 (the K of one kind::tf32 instruction) and the output columns to NC = 16 or 32.
//
// Every wait is bounded: a wait that gives up stores a nonzero code in *err, the block still frees its
// TMEM and returns.
#include "hb_internal.cuh"

namespace hb {

namespace {

constexpr long long kTc5SpinLimit = 1ll << 26;
constexpr int kTc5Rows = 128;                 // M of one MMA (cta_group::1)

template <int NT>
struct Tc5 {
    static constexpr int K = (NT + 7) / 8 * 8;            // padded reduction length (16 or 24)
    static constexpr int NC = NT <= 16 ? 16 : 32;        // padded output columns of the MMA
    static constexpr int TCOLS = 32;                      // TMEM columns allocated: a power of 2, >= 32
    static constexpr int KC = K / 4;                      // core matrices along K (4 TF32 = 16 bytes)
    static constexpr int LBO = 128;                       // bytes between core matrices along K
    static constexpr int SBO = KC * 128;                  // bytes between 8-row groups
    static constexpr int A_BYTES = kTc5Rows / 8 * SBO;    // one part (head or tail) of the X tile
    static constexpr int B_BYTES = NC / 8 * SBO;          // one part of B^T [NC][K]
    static constexpr int N4 = 4 * NT, WS = w_stride(NT, 4);
    static constexpr int NPT = kTc5Rows / 3;              // whole nodes per tile (3 velocity rows each)
    static constexpr int SMEM = 2 * A_BYTES + 2 * B_BYTES + NPT * WS * 4;
};

// byte offset of element (row, k) in the canonical no-swizzle K-major layout
template <int NT>
__device__ __forceinline__ int canon(int row, int k) {
    return (row >> 3) * Tc5<NT>::SBO + (k >> 2) * Tc5<NT>::LBO + (row & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ uint32_t s_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// shared-memory matrix descriptor: start address, leading (K) and stride (M/N) byte offsets, the fixed
// version field (0b001 at bits 46-48), no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = uint64_t((saddr >> 4) & 0x3FFFu);
    d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
    d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
    d |= uint64_t(1) << 46;
    return d;
}

// instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major, N and M
template <int NC>
__host__ __device__ constexpr uint32_t idesc_tf32() {
    return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(NC >> 3) << 17) | (uint32_t(kTc5Rows >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32_ss(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ bool mbar_wait_parity(uint64_t *bar, uint32_t parity) {
    for (long long i = 0; i < kTc5SpinLimit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(s_addr(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// 32 lanes x NC columns of the accumulator for this warp (row = its TMEM lane quarter + lane)
template <int NC>
__device__ __forceinline__ void tmem_load_row(uint32_t taddr, float (&r)[NC]);

template <>
__device__ __forceinline__ void tmem_load_row<16>(uint32_t taddr, float (&r)[16]) {
    uint32_t u[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
          "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) r[j] = __uint_as_float(u[j]);
}

template <>
__device__ __forceinline__ void tmem_load_row<32>(uint32_t taddr, float (&r)[32]) {
    uint32_t u[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
          "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15]),
          "=r"(u[16]), "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23]),
          "=r"(u[24]), "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) r[j] = __uint_as_float(u[j]);
}

template <int NT>
__global__ void __launch_bounds__(128) spectral_tc5_kernel(const float *__restrict__ v, const float *__restrict__ H,
                                                           const uint8_t *__restrict__ flag, float *__restrict__ W,
                                                           int64_t n_nodes, float rho, float shift,
                                                           const double *__restrict__ shift_dev, int *err) {
    using S = Tc5<NT>;
    constexpr int K = S::K, NC = S::NC, N4 = S::N4, WS = S::WS, NPT = S::NPT;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    unsigned char *sAh = smem, *sAl = smem + S::A_BYTES, *sBh = smem + 2 * S::A_BYTES,
                  *sBl = smem + 2 * S::A_BYTES + S::B_BYTES;
    float *sOut = reinterpret_cast<float *>(smem + 2 * S::A_BYTES + 2 * S::B_BYTES);   // [NPT][WS]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t n_tiles = (n_nodes + NPT - 1) / NPT;
    if (int64_t(blockIdx.x) >= n_tiles) return;                     // uniform per block, before any TMEM use
    const float sh = shift_dev ? float(*shift_dev) : shift;
    // B^T [NC][K]: Bt[m][k] = rho H[m][k] + shift delta_mk (zero outside N x N), head and tail
    for (int i = tid; i < NC * K; i += 128) {
        const int m = i / K, k = i - m * K;
        const float b = (m < NT && k < NT) ? rho * H[m * NT + k] + (m == k ? sh : 0.f) : 0.f;
        const uint32_t hi = tf32_rna(b);
        *reinterpret_cast<uint32_t *>(sBh + canon<NT>(m, k)) = hi;
        *reinterpret_cast<uint32_t *>(sBl + canon<NT>(m, k)) = tf32_rna(b - __uint_as_float(hi));
    }
    // X rows past the tile's 3 NPT rows and the zero columns k in [4 ceil(NT / 4), K) never change
    for (int i = tid; i < kTc5Rows * K; i += 128) {
        const int m = i / K, k = i - m * K;
        if (m >= 3 * NPT || k >= 4 * ((NT + 3) / 4)) {
            *reinterpret_cast<uint32_t *>(sAh + canon<NT>(m, k)) = 0u;
            *reinterpret_cast<uint32_t *>(sAl + canon<NT>(m, k)) = 0u;
        }
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(s_addr(&tmem_slot)),
                     "r"(uint32_t(S::TCOLS))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(s_addr(&mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_slot;
    constexpr uint32_t idesc = idesc_tf32<NC>();
    uint32_t phase = 0;
    // work item (velocity row m of the tile, K chunk c of 4 instances): row m is (node m / 3, field m % 3);
    // CH chunks per row carry real instances (the rest of K is zero padding written once above); LPT
    // items per thread, loaded one tile ahead into registers
    constexpr int CH = (NT + 3) / 4, ITEMS = 3 * NPT * CH, LPT = (ITEMS + 127) / 128;
    float pre[LPT][4];
    auto fetch = [&](int64_t tile) {
        const int64_t b0 = tile * NPT;
        const int nb = int(n_nodes - b0 < NPT ? n_nodes - b0 : NPT);
#pragma unroll
        for (int u = 0; u < LPT; ++u) {
            const int i = tid + 128 * u, m = i / CH, c = i - m * CH, l = m / 3;
            const float *row = v + (b0 + l) * N4 + (m - 3 * l) * NT + 4 * c;
#pragma unroll
            for (int q = 0; q < 4; ++q) pre[u][q] = (i < ITEMS && l < nb && 4 * c + q < NT) ? row[q] : 0.f;
        }
    };
    fetch(blockIdx.x);
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int64_t n0 = t * NPT;
        const int nn = int(n_nodes - n0 < NPT ? n_nodes - n0 : NPT);
        // X tile from the prefetched rows: TF32 head and tail, one 16-byte store each per chunk (a chunk is
        // one row of a core matrix in the canonical layout)
#pragma unroll
        for (int u = 0; u < LPT; ++u) {
            const int i = tid + 128 * u;
            if (i >= ITEMS) continue;
            const int m = i / CH, c = i - m * CH;
            uint4 hv, lv;
            uint32_t *h = &hv.x, *lo = &lv.x;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                h[q] = tf32_rna(pre[u][q]);
                lo[q] = tf32_rna(pre[u][q] - __uint_as_float(h[q]));
            }
            *reinterpret_cast<uint4 *>(sAh + canon<NT>(m, 4 * c)) = hv;
            *reinterpret_cast<uint4 *>(sAl + canon<NT>(m, 4 * c)) = lv;
        }
        // the next tile's rows are in flight while this one is multiplied and written back
        if (t + gridDim.x < n_tiles) fetch(t + gridDim.x);
        // generic-proxy writes of the operands -> visible to the tensor core (async proxy)
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (tid == 0) {
            const uint32_t ah = s_addr(sAh), al = s_addr(sAl), bh = s_addr(sBh), bl = s_addr(sBl);
#pragma unroll
            for (int ks = 0; ks < K / 8; ++ks) {
                const uint32_t off = uint32_t(ks) * 2 * S::LBO;       // 8 TF32 = two core matrices along K
                const uint64_t dah = smem_desc(ah + off, S::LBO, S::SBO), dal = smem_desc(al + off, S::LBO, S::SBO);
                const uint64_t dbh = smem_desc(bh + off, S::LBO, S::SBO), dbl = smem_desc(bl + off, S::LBO, S::SBO);
                mma_tf32_ss(tmem, dal, dbh, idesc, ks > 0 ? 1u : 0u);
                mma_tf32_ss(tmem, dah, dbl, idesc, 1u);
                mma_tf32_ss(tmem, dah, dbh, idesc, 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             s_addr(&mbar))
                         : "memory");
        }
        if (!mbar_wait_parity(&mbar, phase)) {
            if (lane == 0) atomicExch(err, 4);
            break;                                     // uniform: every thread polls the same barrier
        }
        phase ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        // accumulator row m = 32 warp + lane -> staged W row (node m / 3, field m % 3), then whole node rows
        // of WS values go out with 16-byte stores (zero on prescribed velocities and in the row padding)
        {
            float acc[NC];
            tmem_load_row<NC>(tmem + (uint32_t(32 * warp) << 16), acc);
            const int m = 32 * warp + lane;
            if (m < 3 * NPT) {
                const int l = m / 3, f = m - 3 * l;
#pragma unroll
                for (int j = 0; j < NT; ++j) sOut[l * WS + f * NT + j] = acc[j];
                if (f == 2)
#pragma unroll
                    for (int j = 3 * NT; j < WS; ++j) sOut[l * WS + j] = 0.f;
            }
        }
        __syncthreads();
        float4 *dst = reinterpret_cast<float4 *>(W + n0 * WS);
        const float4 *so = reinterpret_cast<const float4 *>(sOut);
        for (int i = tid; i < nn * WS / 4; i += 128) {
            const int l = (4 * i) / WS;
            dst[i] = (flag[n0 + l] & 1) ? make_float4(0.f, 0.f, 0.f, 0.f) : so[i];
        }
        // every lane's TMEM reads and every operand and staging read are done before the next tile
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    }
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(uint32_t(S::TCOLS))
                     : "memory");
}

template <int NT>
void launch_tc5(const float *v, const float *H, const uint8_t *flag, float *W, int64_t n_nodes, float rho, float shift,
                const double *shift_dev, int *err, cudaStream_t s) {
    auto kern = spectral_tc5_kernel<NT>;
    const size_t smem = Tc5<NT>::SMEM;
    // 4 blocks per SM (4 x ~42 KB of shared memory; 4 x 32 = 128 of the 512 TMEM columns, so an allocation
    // never waits); the loop is persistent over the tiles
    const int per = 4;
    const int64_t tiles = (n_nodes + Tc5<NT>::NPT - 1) / Tc5<NT>::NPT;
    const int grid = int(std::min<int64_t>(tiles, int64_t(per) * device_sms()));
    kern<<<grid, 128, smem, s>>>(v, H, flag, W, n_nodes, rho, shift, shift_dev, err);
}

}  // namespace

bool launch_spectral_w_tc5(const float *v, const float *H, const uint8_t *flag, float *W, int64_t n_nodes, int N,
                           float rho, float shift, const double *shift_dev, int *err, cudaStream_t s) {
    if (n_nodes <= 0 || !err) return false;
    switch (N) {
        case 9: launch_tc5<9>(v, H, flag, W, n_nodes, rho, shift, shift_dev, err, s); return true;
        case 13: launch_tc5<13>(v, H, flag, W, n_nodes, rho, shift, shift_dev, err, s); return true;
        case 21: launch_tc5<21>(v, H, flag, W, n_nodes, rho, shift, shift_dev, err, s); return true;
        default: return false;
    }
}

}  // namespace hb
