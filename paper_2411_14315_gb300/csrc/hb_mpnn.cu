// Learned warm start: a small message-passing network over the mesh graph that predicts the harmonic
// coefficients of the solution from the geometry and boundary data (arXiv 2411.14315 only suggests, in
// Sec. 4, that harmonic balance solutions could serve as machine-learning datasets; the network is not
// part of the method).  Weights are stored in BF16; all arithmetic and accumulation is FP32.
//
// Every MLP is mlp(X) = relu(X W1 + b1) W2 + b2 with W1 (k x H) followed by b1 and W2 (H x o) followed
// by b2 in one contiguous parameter block, so [X, 1] times the augmented (k+1) x H matrix is X W1 + b1.
// Forward: h = enc(x); per layer m_e = msg([h_src, h_dst, e_e]), a = sum_e->i m_e, h += upd([h, a]);
// out = dec(h).  Loss: mean squared error against normalised target harmonics.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <unordered_map>
#include <vector>

#include "hb_internal.cuh"
#include "hbgls.h"

namespace hb {

// provided by hb_api.cu
hb_status learned_inputs(hb_problem *p, LearnedInputs &out);
uint64_t problem_uid(const hb_problem *p);
hb_status learned_set_initial(hb_problem *p, const double *harmonics_host);
hb_status set_error(hb_status st, const std::string &msg);

namespace {

constexpr int kWarps = 8;                 // rows in flight per block (one warp per row)
constexpr int kMaxOutPerLane = 3;         // output width <= 96
constexpr int kWChunk = 32;               // rows per weight-gradient chunk
constexpr int kWQ = 40;                   // weight-gradient outputs per thread (<= 256 x 40)

struct Seg {
    const float *base;                    // row r reads base[(idx ? idx[r] : r) * ld + k]
    const int *idx;
    int width, ld;
};
struct Segs {
    Seg s[3];
    int n, total;
};
struct DSeg {
    float *base;                          // null: gradient not needed
    const int *idx;
    int width, ld;
};
struct DSegs {
    DSeg s[3];
    int n;
};

__device__ __forceinline__ float seg_value(const Segs &in, int r, int k) {
    int off = 0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        if (q < in.n) {
            const Seg &sg = in.s[q];
            if (k < off + sg.width) {
                const int row = sg.idx ? sg.idx[r] : r;
                return sg.base[size_t(row) * sg.ld + (k - off)];
            }
            off += sg.width;
        }
    }
    return 0.f;
}

// ymode 0: Y[r] = y; 1: Y[r] += y (residual); 2: Y[ydst[r]] += y (atomic scatter)
__global__ void mlp_fwd_kernel(Segs in, const __nv_bfloat16 *__restrict__ w, int hid, int kout, int rows,
                               float *__restrict__ A_save, float *__restrict__ Y, int ymode,
                               const int *__restrict__ ydst) {
    extern __shared__ float sm[];
    const int kin = in.total;
    float *sW1 = sm;                                  // (kin + 1) x hid
    float *sW2 = sW1 + (kin + 1) * hid;               // (hid + 1) x kout
    float *sx = sW2 + (hid + 1) * kout;               // kWarps x (kin + 1)
    float *sa = sx + kWarps * (kin + 1);              // kWarps x (hid + 1)
    const int n1 = (kin + 1) * hid, n2 = (hid + 1) * kout;
    for (int i = threadIdx.x; i < n1 + n2; i += blockDim.x) sm[i] = __bfloat162float(w[i]);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *x = sx + warp * (kin + 1);
    float *a = sa + warp * (hid + 1);
    for (int r = blockIdx.x * kWarps + warp; r < rows; r += gridDim.x * kWarps) {
        for (int k = lane; k < kin; k += 32) x[k] = seg_value(in, r, k);
        if (lane == 0) {
            x[kin] = 1.f;
            a[hid] = 1.f;
        }
        __syncwarp();
        for (int j = lane; j < hid; j += 32) {
            float z = 0.f;
            for (int k = 0; k <= kin; ++k) z += x[k] * sW1[k * hid + j];
            z = fmaxf(z, 0.f);
            a[j] = z;
            if (A_save) A_save[size_t(r) * hid + j] = z;
        }
        __syncwarp();
        for (int t = 0; t < kMaxOutPerLane; ++t) {
            const int o = lane + 32 * t;
            if (o >= kout) break;
            float y = 0.f;
            for (int j = 0; j <= hid; ++j) y += a[j] * sW2[j * kout + o];
            if (ymode == 0) Y[size_t(r) * kout + o] = y;
            else if (ymode == 1) Y[size_t(r) * kout + o] += y;
            else atomicAdd(Y + size_t(ydst[r]) * kout + o, y);
        }
        __syncwarp();
    }
}

// Row-wise backward: dY (gathered through dYidx when the forward scattered), dZ = (dY W2^T) * [A > 0]
// saved for the weight gradients, dX = dZ W1^T added into the gradients of the input segments.
__global__ void mlp_bwd_kernel(Segs in, const __nv_bfloat16 *__restrict__ w, int hid, int kout, int rows,
                               const float *__restrict__ A_save, const float *__restrict__ dY,
                               const int *__restrict__ dYidx, float *__restrict__ dZ_save, DSegs dx) {
    extern __shared__ float sm[];
    const int kin = in.total;
    float *sW1T = sm;                                 // hid x kin   (W1 transposed, no bias row)
    float *sW2T = sW1T + hid * kin;                   // kout x hid  (W2 transposed, no bias row)
    float *sdy = sW2T + kout * hid;                   // kWarps x kout
    float *sdz = sdy + kWarps * kout;                 // kWarps x hid
    for (int i = threadIdx.x; i < kin * hid; i += blockDim.x) {
        const int k = i / hid, j = i - k * hid;
        sW1T[j * kin + k] = __bfloat162float(w[i]);
    }
    const __nv_bfloat16 *w2 = w + (kin + 1) * hid;
    for (int i = threadIdx.x; i < hid * kout; i += blockDim.x) {
        const int j = i / kout, o = i - j * kout;
        sW2T[o * hid + j] = __bfloat162float(w2[i]);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *dy = sdy + warp * kout;
    float *dz = sdz + warp * hid;
    for (int r = blockIdx.x * kWarps + warp; r < rows; r += gridDim.x * kWarps) {
        const int yr = dYidx ? dYidx[r] : r;
        for (int o = lane; o < kout; o += 32) dy[o] = dY[size_t(yr) * kout + o];
        __syncwarp();
        for (int j = lane; j < hid; j += 32) {
            float s = 0.f;
            for (int o = 0; o < kout; ++o) s += sW2T[o * hid + j] * dy[o];
            const float g = A_save[size_t(r) * hid + j] > 0.f ? s : 0.f;
            dz[j] = g;
            dZ_save[size_t(r) * hid + j] = g;
        }
        __syncwarp();
        int off = 0;
        for (int q = 0; q < dx.n; ++q) {
            const DSeg &sg = dx.s[q];
            if (sg.base) {
                const int row = sg.idx ? sg.idx[r] : r;
                for (int k = lane; k < sg.width; k += 32) {
                    float s = 0.f;
                    for (int j = 0; j < hid; ++j) s += sW1T[j * kin + off + k] * dz[j];
                    atomicAdd(sg.base + size_t(row) * sg.ld + k, s);
                }
            }
            off += sg.width;
        }
        __syncwarp();
    }
}

// G[k][j] += sum_r U[r][k] V[r][j] with U augmented by a column of ones (k = ku gives the bias
// gradient, which follows the weight matrix in the parameter layout).
__global__ void __launch_bounds__(256) wgrad_kernel(Segs U, int rows, const float *__restrict__ V,
                                                    const int *__restrict__ vidx, int nv, float *__restrict__ G) {
    __shared__ float sU[kWChunk][200];
    __shared__ float sV[kWChunk][96];
    const int ku = U.total, nout = (ku + 1) * nv;
    float acc[kWQ];
#pragma unroll
    for (int q = 0; q < kWQ; ++q) acc[q] = 0.f;
    for (int c0 = blockIdx.x * kWChunk; c0 < rows; c0 += gridDim.x * kWChunk) {
        const int R = min(kWChunk, rows - c0);
        for (int i = threadIdx.x; i < kWChunk * (ku + 1); i += blockDim.x) {
            const int r = i / (ku + 1), k = i - r * (ku + 1);
            sU[r][k] = (r < R) ? (k == ku ? 1.f : seg_value(U, c0 + r, k)) : 0.f;
        }
        for (int i = threadIdx.x; i < kWChunk * nv; i += blockDim.x) {
            const int r = i / nv, j = i - r * nv;
            float v = 0.f;
            if (r < R) {
                const int vr = vidx ? vidx[c0 + r] : c0 + r;
                v = V[size_t(vr) * nv + j];
            }
            sV[r][j] = v;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kWQ; ++q) {
            const int o = threadIdx.x + 256 * q;
            if (o < nout) {
                const int k = o / nv, j = o - k * nv;
                float s = 0.f;
                for (int r = 0; r < kWChunk; ++r) s += sU[r][k] * sV[r][j];
                acc[q] += s;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < kWQ; ++q) {
        const int o = threadIdx.x + 256 * q;
        if (o < nout && acc[q] != 0.f) atomicAdd(G + o, acc[q]);
    }
}

// Tensor-core form of mlp_fwd_kernel: a warp takes 16 rows; both layers are mma.sync m16n8k8 TF32 products
// with FP32 accumulation.  The BF16 weights are exact in TF32; the FP32 activations are split into a TF32
// head and tail (x = hi + lo), so X W = Xhi W + Xlo W keeps FP32 accuracy (the tail's own TF32 rounding is
// ~2^-22 relative).  Shared memory: W1 as [KP1][HS] (bias row kin, zero rows up to KP1), W2 as [KP2][OS]
// (bias row hid), and per warp the 16 input rows [16][XS] and hidden rows [16][AS] (a column of ones at
// kin / hid).  Strides are padded so that the fragment loads of a warp hit 32 distinct banks.
constexpr int kTcWarps = 8;

__device__ __forceinline__ uint32_t tf32_of(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_m16n8k8_tf32(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                 "{%8, %9}, {%0, %1, %2, %3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

struct TcDims {
    int kin, hid, kout, KP1, KP2, HS, OS, XS, AS;
};
__host__ __device__ inline TcDims tc_dims(int kin, int hid, int kout) {
    TcDims d;
    d.kin = kin;
    d.hid = hid;
    d.kout = kout;
    d.KP1 = (kin + 1 + 7) / 8 * 8;            // K of layer 1 (inputs + bias), padded to the MMA's K
    d.KP2 = (hid + 1 + 7) / 8 * 8;
    d.HS = (hid + 31) / 32 * 32 + 8;          // row stride of W1 (words): 8 mod 32 spreads k rows over banks
    d.OS = (kout + 31) / 32 * 32 + 8;         // row stride of W2, same
    d.XS = d.KP1 + 4;                         // row stride of the staged inputs: 4 mod 8 words
    d.AS = d.KP2 + 4;
    return d;
}
__host__ __device__ inline size_t tc_smem_floats(const TcDims &d) {
    return size_t(d.KP1) * d.HS + size_t(d.KP2) * d.OS + size_t(kTcWarps) * 16 * (d.XS + d.AS);
}

template <int NT1>
__global__ void __launch_bounds__(32 * kTcWarps) mlp_fwd_tc_kernel(Segs in, const __nv_bfloat16 *__restrict__ w,
                                                                   int hid, int kout, int rows,
                                                                   float *__restrict__ A_save, float *__restrict__ Y,
                                                                   int ymode, const int *__restrict__ ydst) {
    extern __shared__ float sm[];
    const TcDims d = tc_dims(in.total, hid, kout);
    const int kin = d.kin;
    float *sW1 = sm, *sW2 = sW1 + size_t(d.KP1) * d.HS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    float *sX = sW2 + size_t(d.KP2) * d.OS + size_t(warp) * 16 * (d.XS + d.AS);
    float *sA = sX + 16 * d.XS;
    // weights (the parameter block: W1 [kin][hid], b1 [hid], W2 [hid][kout], b2 [kout])
    for (int i = threadIdx.x; i < d.KP1 * hid; i += blockDim.x) {
        const int k = i / hid, j = i - k * hid;
        sW1[k * d.HS + j] = k <= kin ? __bfloat162float(w[k * hid + j]) : 0.f;
    }
    const __nv_bfloat16 *w2 = w + (kin + 1) * hid;
    const int kop = (kout + 7) / 8 * 8;
    for (int i = threadIdx.x; i < d.KP2 * kop; i += blockDim.x) {
        const int k = i / kop, o = i - k * kop;
        sW2[k * d.OS + o] = (k <= hid && o < kout) ? __bfloat162float(w2[k * kout + o]) : 0.f;
    }
    __syncthreads();
    for (int r0 = (blockIdx.x * kTcWarps + warp) * 16; r0 < rows; r0 += gridDim.x * kTcWarps * 16) {
        // stage the 16 input rows (segments gathered; bias column of ones; zero padding)
        for (int i = lane; i < 16 * d.KP1; i += 32) {
            const int rr = i / d.KP1, k = i - rr * d.KP1, r = r0 + rr;
            float x = 0.f;
            if (r < rows) x = k < kin ? seg_value(in, r, k) : (k == kin ? 1.f : 0.f);
            sX[rr * d.XS + k] = x;
        }
        __syncwarp();
        // layer 1: Z = [X, 1] [W1; b1], NT1 tiles of 8 hidden units
        float acc[NT1][4];
#pragma unroll
        for (int t = 0; t < NT1; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;
        for (int k0 = 0; k0 < d.KP1; k0 += 8) {
            const float av[4] = {sX[g * d.XS + k0 + q], sX[(g + 8) * d.XS + k0 + q], sX[g * d.XS + k0 + q + 4],
                                 sX[(g + 8) * d.XS + k0 + q + 4]};
            uint32_t ah[4], al[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                ah[i] = tf32_of(av[i]);
                al[i] = tf32_of(av[i] - __uint_as_float(ah[i]));
            }
#pragma unroll
            for (int t = 0; t < NT1; ++t) {
                const uint32_t b0 = __float_as_uint(sW1[(k0 + q) * d.HS + 8 * t + g]);
                const uint32_t b1 = __float_as_uint(sW1[(k0 + q + 4) * d.HS + 8 * t + g]);
                mma_m16n8k8_tf32(acc[t], al, b0, b1);
                mma_m16n8k8_tf32(acc[t], ah, b0, b1);
            }
        }
        // relu, save, stage [A, 1]
#pragma unroll
        for (int t = 0; t < NT1; ++t)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int rr = g + 8 * h, r = r0 + rr;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int j = 8 * t + 2 * q + c;
                    const float z = fmaxf(acc[t][2 * h + c], 0.f);
                    sA[rr * d.AS + j] = z;
                    if (A_save && r < rows && j < hid) A_save[size_t(r) * hid + j] = z;
                }
            }
        for (int i = lane; i < 16 * (d.KP2 - hid); i += 32) {
            const int rr = i / (d.KP2 - hid), k = hid + (i - rr * (d.KP2 - hid));
            sA[rr * d.AS + k] = k == hid ? 1.f : 0.f;
        }
        __syncwarp();
        // layer 2: Y = [A, 1] [W2; b2], NT2 tiles of 8 outputs
        constexpr int NT2 = 12;                   // outputs <= 96
        float out[NT2][4];
#pragma unroll
        for (int t = 0; t < NT2; ++t) out[t][0] = out[t][1] = out[t][2] = out[t][3] = 0.f;
        for (int k0 = 0; k0 < d.KP2; k0 += 8) {
            const float av[4] = {sA[g * d.AS + k0 + q], sA[(g + 8) * d.AS + k0 + q], sA[g * d.AS + k0 + q + 4],
                                 sA[(g + 8) * d.AS + k0 + q + 4]};
            uint32_t ah[4], al[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                ah[i] = tf32_of(av[i]);
                al[i] = tf32_of(av[i] - __uint_as_float(ah[i]));
            }
#pragma unroll
            for (int t = 0; t < NT2; ++t) {
                if (8 * t >= kout) break;
                const uint32_t b0 = __float_as_uint(sW2[(k0 + q) * d.OS + 8 * t + g]);
                const uint32_t b1 = __float_as_uint(sW2[(k0 + q + 4) * d.OS + 8 * t + g]);
                mma_m16n8k8_tf32(out[t], al, b0, b1);
                mma_m16n8k8_tf32(out[t], ah, b0, b1);
            }
        }
#pragma unroll
        for (int t = 0; t < NT2; ++t)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = r0 + g + 8 * h;
                if (r >= rows) continue;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int o = 8 * t + 2 * q + c;
                    if (o >= kout) continue;
                    const float y = out[t][2 * h + c];
                    if (ymode == 0) Y[size_t(r) * kout + o] = y;
                    else if (ymode == 1) Y[size_t(r) * kout + o] += y;
                    else atomicAdd(Y + size_t(ydst[r]) * kout + o, y);
                }
            }
        __syncwarp();
    }
}

// loss += sum (out - target)^2 / count; dout = 2 (out - target) / count
__global__ void mse_kernel(const float *__restrict__ out, const float *__restrict__ tgt, int64_t count,
                           float *__restrict__ dout, float *__restrict__ loss) {
    __shared__ float red[8];
    float s = 0.f;
    const float inv = 1.f / float(count);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x) {
        const float d = out[i] - tgt[i];
        s += d * d;
        dout[i] = 2.f * d * inv;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int q = 0; q < int(blockDim.x >> 5); ++q) t += red[q];
        atomicAdd(loss, t * inv);
    }
}

__global__ void adam_kernel(float *__restrict__ p, __nv_bfloat16 *__restrict__ p16, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v, int64_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        p16[i] = __float2bfloat16(pi);
    }
}

__global__ void to_bf16_kernel(const float *__restrict__ p, __nv_bfloat16 *__restrict__ q, int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        q[i] = __float2bfloat16(p[i]);
}

inline int grid_for(int64_t rows, int per_block, int cap = 1184) {
    const int64_t g = (rows + per_block - 1) / per_block;
    return int(std::max<int64_t>(1, std::min<int64_t>(g, cap)));
}

}  // namespace
}  // namespace hb

using namespace hb;

// ------------------------------------------------------------------------------------------------------
// host side

namespace {

template <typename T>
struct Buf {
    T *p = nullptr;
    size_t n = 0;
    ~Buf() {
        if (p) cudaFree(p);
    }
    cudaError_t ensure(size_t m) {
        if (m <= n && p) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        cudaError_t e = cudaMalloc(&p, std::max<size_t>(m, 1) * sizeof(T));
        if (e == cudaSuccess) n = std::max<size_t>(m, 1);
        return e;
    }
};

struct Graph {
    int n = 0, ne = 0;
    Buf<float> x, e;                  // [n][f_in], [ne][f_e]
    Buf<int> src, dst;
    std::vector<Buf<float>> h;        // layers + 1 node states [n][H]
    std::vector<Buf<float>> agg;      // per layer [n][H]
    std::vector<Buf<float>> Am, Au;   // per layer saved activations [ne][H], [n][H]
    Buf<float> Aenc, Adec, out, tgt, dout, dZ, dH0, dH1, dAgg;
    double u_ref = 1, p_ref = 0, rho = 1;
};

}  // namespace

struct hb_mpnn {
    int device = 0;
    int hidden = 64, layers = 3, n_h = 10, f_in = 0, f_e = 4, f_out = 0;
    double p_scale = 1.0;
    std::vector<int> kin, kout, off;  // per MLP: input width, output width, parameter offset
    int64_t n_params = 0;
    Buf<float> P, G, M, V, loss;
    Buf<__nv_bfloat16> P16;
    int64_t step = 0;
    cudaStream_t stream = nullptr;
    std::unordered_map<uint64_t, Graph> graphs;   // keyed by the problem's unique id
    bool tensor_cores = true;                     // forward MLPs on mma.sync TF32 (hidden 32 or 64)
};

namespace {

#define MP_CUDA(expr)                                                                                   \
    do {                                                                                                \
        cudaError_t _e = (expr);                                                                        \
        if (_e != cudaSuccess)                                                                          \
            return set_error(_e == cudaErrorMemoryAllocation ? HB_ERR_OOM : HB_ERR_CUDA,                \
                             std::string(#expr) + ": " + cudaGetErrorString(_e));                       \
    } while (0)
#define MP_TRY(expr)                                                                                    \
    do {                                                                                                \
        hb_status _s = (expr);                                                                          \
        if (_s != HB_OK) return _s;                                                                     \
    } while (0)

size_t fwd_smem(int kin, int hid, int kout) {
    return size_t((kin + 1) * hid + (hid + 1) * kout + kWarps * (kin + 1) + kWarps * (hid + 1)) * sizeof(float);
}
size_t bwd_smem(int kin, int hid, int kout) {
    return size_t(hid * kin + kout * hid + kWarps * kout + kWarps * hid) * sizeof(float);
}

Segs segs(std::initializer_list<Seg> l) {
    Segs s{};
    s.n = 0;
    s.total = 0;
    for (const Seg &x : l) {
        s.s[s.n++] = x;
        s.total += x.width;
    }
    return s;
}
DSegs dsegs(std::initializer_list<DSeg> l) {
    DSegs s{};
    s.n = 0;
    for (const DSeg &x : l) s.s[s.n++] = x;
    return s;
}

hb_status run_fwd(hb_mpnn *net, int which, const Segs &in, int rows, float *A_save, float *Y, int ymode,
                  const int *ydst) {
    const int kin = net->kin[size_t(which)], kout = net->kout[size_t(which)], H = net->hidden;
    if (net->tensor_cores && (H == 32 || H == 64) && kout <= 96 && rows > 0) {
        const size_t sm = tc_smem_floats(tc_dims(kin, H, kout)) * sizeof(float);
        const int grid = grid_for(rows, kTcWarps * 16, 2 * 152);
        if (H == 64) {
            MP_CUDA(cudaFuncSetAttribute(mlp_fwd_tc_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)));
            mlp_fwd_tc_kernel<8><<<grid, 32 * kTcWarps, sm, net->stream>>>(
                in, net->P16.p + net->off[size_t(which)], H, kout, rows, A_save, Y, ymode, ydst);
        } else {
            MP_CUDA(cudaFuncSetAttribute(mlp_fwd_tc_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)));
            mlp_fwd_tc_kernel<4><<<grid, 32 * kTcWarps, sm, net->stream>>>(
                in, net->P16.p + net->off[size_t(which)], H, kout, rows, A_save, Y, ymode, ydst);
        }
        MP_CUDA(cudaGetLastError());
        return HB_OK;
    }
    const size_t sm = fwd_smem(kin, H, kout);
    MP_CUDA(cudaFuncSetAttribute(mlp_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)));
    mlp_fwd_kernel<<<grid_for(rows, kWarps), 32 * kWarps, sm, net->stream>>>(
        in, net->P16.p + net->off[size_t(which)], H, kout, rows, A_save, Y, ymode, ydst);
    MP_CUDA(cudaGetLastError());
    return HB_OK;
}

hb_status run_bwd(hb_mpnn *net, int which, const Segs &in, int rows, const float *A_save, const float *dY,
                  const int *dYidx, float *dZ, const DSegs &dx) {
    const int kin = net->kin[size_t(which)], kout = net->kout[size_t(which)], H = net->hidden;
    const size_t sm = bwd_smem(kin, H, kout);
    MP_CUDA(cudaFuncSetAttribute(mlp_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)));
    mlp_bwd_kernel<<<grid_for(rows, kWarps), 32 * kWarps, sm, net->stream>>>(
        in, net->P16.p + net->off[size_t(which)], H, kout, rows, A_save, dY, dYidx, dZ, dx);
    MP_CUDA(cudaGetLastError());
    // weight gradients: [X, 1]^T dZ into (W1, b1); [A, 1]^T dY into (W2, b2)
    float *G = net->G.p + net->off[size_t(which)];
    wgrad_kernel<<<grid_for(rows, kWChunk, 304), 256, 0, net->stream>>>(in, rows, dZ, nullptr, H, G);
    Segs a = segs({Seg{A_save, nullptr, H, H}});
    wgrad_kernel<<<grid_for(rows, kWChunk, 304), 256, 0, net->stream>>>(a, rows, dY, dYidx, kout,
                                                                         G + (kin + 1) * H);
    MP_CUDA(cudaGetLastError());
    return HB_OK;
}

hb_status build_graph(hb_mpnn *net, hb_problem *p, Graph &g) {
    LearnedInputs in;
    MP_TRY(learned_inputs(p, in));
    if (in.n_h != net->n_h) return set_error(HB_ERR_INVALID_ARG, "network n_h differs from the problem's");
    const int n = int(in.n_nodes);
    // undirected edges of the tetrahedra, both directions
    std::vector<uint64_t> keys;
    keys.reserve(size_t(6 * in.n_tets));
    static const int pr[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
    for (int64_t t = 0; t < in.n_tets; ++t)
        for (auto &q : pr) {
            uint64_t a = uint64_t(in.tets[size_t(4 * t + q[0])]), b = uint64_t(in.tets[size_t(4 * t + q[1])]);
            if (a > b) std::swap(a, b);
            keys.push_back((a << 32) | b);
        }
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    std::vector<int> src, dst;
    src.reserve(2 * keys.size());
    dst.reserve(2 * keys.size());
    for (uint64_t k : keys) {
        const int a = int(k >> 32), b = int(k & 0xffffffffu);
        src.push_back(a);
        dst.push_back(b);
        src.push_back(b);
        dst.push_back(a);
    }
    // node and edge features
    double c[3] = {0, 0, 0}, lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d) {
            c[d] += in.xyz[size_t(3 * i + d)] / n;
            lo[d] = std::min(lo[d], in.xyz[size_t(3 * i + d)]);
            hi[d] = std::max(hi[d], in.xyz[size_t(3 * i + d)]);
        }
    double L = 0;
    for (int d = 0; d < 3; ++d) L = std::max(L, 0.5 * (hi[d] - lo[d]));
    if (L <= 0) L = 1;
    double pmax = 0;
    for (int i = 0; i < n; ++i) {
        double s = 0;
        for (int d = 0; d < 3; ++d) s += in.profile[size_t(3 * i + d)] * in.profile[size_t(3 * i + d)];
        pmax = std::max(pmax, std::sqrt(s));
    }
    if (pmax <= 0) pmax = 1;
    const int M = 2 * in.n_h + 1;
    const double a0 = std::fabs(in.wave[0]) > 0 ? std::fabs(in.wave[0]) : 1.0;
    std::vector<float> x(size_t(n) * net->f_in, 0.f);
    for (int i = 0; i < n; ++i) {
        float *r = &x[size_t(i) * net->f_in];
        for (int d = 0; d < 3; ++d) r[d] = float((in.xyz[size_t(3 * i + d)] - c[d]) / L);
        r[3] = float(in.flags[size_t(i)] & 1);
        r[4] = float((in.flags[size_t(i)] >> 1) & 1);
        r[5] = float((in.flags[size_t(i)] >> 2) & 1);
        for (int d = 0; d < 3; ++d) r[6 + d] = float(in.profile[size_t(3 * i + d)] / pmax);
        for (int m = 0; m < M && 9 + m < net->f_in; ++m) r[9 + m] = float(in.wave[size_t(m)] / a0);
    }
    std::vector<float> e(src.size() * size_t(net->f_e));
    for (size_t k = 0; k < src.size(); ++k) {
        double dv[3], len = 0;
        for (int d = 0; d < 3; ++d) {
            dv[d] = (in.xyz[size_t(3 * dst[k] + d)] - in.xyz[size_t(3 * src[k] + d)]) / L;
            len += dv[d] * dv[d];
        }
        for (int d = 0; d < 3; ++d) e[k * size_t(net->f_e) + size_t(d)] = float(dv[d]);
        e[k * size_t(net->f_e) + 3] = float(std::sqrt(len));
    }
    g.n = n;
    g.ne = int(src.size());
    g.u_ref = in.u_ref > 0 ? in.u_ref : 1.0;
    g.p_ref = in.p_ref;
    g.rho = in.rho;
    const int H = net->hidden;
    MP_CUDA(g.x.ensure(x.size()));
    MP_CUDA(g.e.ensure(e.size()));
    MP_CUDA(g.src.ensure(src.size()));
    MP_CUDA(g.dst.ensure(dst.size()));
    MP_CUDA(cudaMemcpy(g.x.p, x.data(), x.size() * sizeof(float), cudaMemcpyHostToDevice));
    MP_CUDA(cudaMemcpy(g.e.p, e.data(), e.size() * sizeof(float), cudaMemcpyHostToDevice));
    MP_CUDA(cudaMemcpy(g.src.p, src.data(), src.size() * sizeof(int), cudaMemcpyHostToDevice));
    MP_CUDA(cudaMemcpy(g.dst.p, dst.data(), dst.size() * sizeof(int), cudaMemcpyHostToDevice));
    g.h.resize(size_t(net->layers + 1));
    g.agg.resize(size_t(net->layers));
    g.Am.resize(size_t(net->layers));
    g.Au.resize(size_t(net->layers));
    for (auto &b : g.h) MP_CUDA(b.ensure(size_t(n) * H));
    for (auto &b : g.agg) MP_CUDA(b.ensure(size_t(n) * H));
    for (auto &b : g.Am) MP_CUDA(b.ensure(size_t(g.ne) * H));
    for (auto &b : g.Au) MP_CUDA(b.ensure(size_t(n) * H));
    MP_CUDA(g.Aenc.ensure(size_t(n) * H));
    MP_CUDA(g.Adec.ensure(size_t(n) * H));
    MP_CUDA(g.out.ensure(size_t(n) * net->f_out));
    MP_CUDA(g.tgt.ensure(size_t(n) * net->f_out));
    MP_CUDA(g.dout.ensure(size_t(n) * net->f_out));
    MP_CUDA(g.dZ.ensure(size_t(std::max(n, g.ne)) * H));
    MP_CUDA(g.dH0.ensure(size_t(n) * H));
    MP_CUDA(g.dH1.ensure(size_t(n) * H));
    MP_CUDA(g.dAgg.ensure(size_t(n) * H));
    return HB_OK;
}

hb_status graph_for(hb_mpnn *net, hb_problem *p, Graph *&g) {
    const uint64_t key = problem_uid(p);
    auto it = net->graphs.find(key);
    if (it == net->graphs.end()) {
        Graph &ng = net->graphs[key];
        hb_status st = build_graph(net, p, ng);
        if (st != HB_OK) {
            net->graphs.erase(key);
            return st;
        }
        g = &ng;
    } else {
        g = &it->second;
    }
    return HB_OK;
}

hb_status forward(hb_mpnn *net, Graph &g) {
    const int H = net->hidden, n = g.n, ne = g.ne;
    MP_TRY(run_fwd(net, 0, segs({Seg{g.x.p, nullptr, net->f_in, net->f_in}}), n, g.Aenc.p, g.h[0].p, 0, nullptr));
    for (int l = 0; l < net->layers; ++l) {
        const float *h = g.h[size_t(l)].p;
        MP_CUDA(cudaMemsetAsync(g.agg[size_t(l)].p, 0, size_t(n) * H * sizeof(float), net->stream));
        MP_TRY(run_fwd(net, 1 + 2 * l,
                       segs({Seg{h, g.src.p, H, H}, Seg{h, g.dst.p, H, H}, Seg{g.e.p, nullptr, net->f_e, net->f_e}}),
                       ne, g.Am[size_t(l)].p, g.agg[size_t(l)].p, 2, g.dst.p));
        MP_CUDA(cudaMemcpyAsync(g.h[size_t(l + 1)].p, h, size_t(n) * H * sizeof(float), cudaMemcpyDeviceToDevice,
                                net->stream));
        MP_TRY(run_fwd(net, 2 + 2 * l, segs({Seg{h, nullptr, H, H}, Seg{g.agg[size_t(l)].p, nullptr, H, H}}), n,
                       g.Au[size_t(l)].p, g.h[size_t(l + 1)].p, 1, nullptr));
    }
    MP_TRY(run_fwd(net, 1 + 2 * net->layers, segs({Seg{g.h[size_t(net->layers)].p, nullptr, H, H}}), n, g.Adec.p,
                   g.out.p, 0, nullptr));
    return HB_OK;
}

hb_status backward(hb_mpnn *net, Graph &g) {
    const int H = net->hidden, n = g.n, ne = g.ne, Ld = net->layers;
    MP_CUDA(cudaMemsetAsync(net->G.p, 0, size_t(net->n_params) * sizeof(float), net->stream));
    float *dA = g.dH0.p, *dB = g.dH1.p;   // dA: gradient wrt the current h, dB: scratch for the next
    MP_CUDA(cudaMemsetAsync(dA, 0, size_t(n) * H * sizeof(float), net->stream));
    MP_TRY(run_bwd(net, 1 + 2 * Ld, segs({Seg{g.h[size_t(Ld)].p, nullptr, H, H}}), n, g.Adec.p, g.dout.p, nullptr,
                   g.dZ.p, dsegs({DSeg{dA, nullptr, H, H}})));
    for (int l = Ld - 1; l >= 0; --l) {
        const float *h = g.h[size_t(l)].p;
        // dh_l = dh_{l+1} + upd's input gradient (h part); da = upd's input gradient (agg part)
        MP_CUDA(cudaMemcpyAsync(dB, dA, size_t(n) * H * sizeof(float), cudaMemcpyDeviceToDevice, net->stream));
        MP_CUDA(cudaMemsetAsync(g.dAgg.p, 0, size_t(n) * H * sizeof(float), net->stream));
        MP_TRY(run_bwd(net, 2 + 2 * l, segs({Seg{h, nullptr, H, H}, Seg{g.agg[size_t(l)].p, nullptr, H, H}}), n,
                       g.Au[size_t(l)].p, dA, nullptr, g.dZ.p,
                       dsegs({DSeg{dB, nullptr, H, H}, DSeg{g.dAgg.p, nullptr, H, H}})));
        // messages: dm_e = da[dst_e]; their input gradients go to h[src_e] and h[dst_e]
        MP_TRY(run_bwd(net, 1 + 2 * l,
                       segs({Seg{h, g.src.p, H, H}, Seg{h, g.dst.p, H, H}, Seg{g.e.p, nullptr, net->f_e, net->f_e}}),
                       ne, g.Am[size_t(l)].p, g.dAgg.p, g.dst.p, g.dZ.p,
                       dsegs({DSeg{dB, g.src.p, H, H}, DSeg{dB, g.dst.p, H, H}, DSeg{nullptr, nullptr, net->f_e, 0}})));
        std::swap(dA, dB);
    }
    MP_TRY(run_bwd(net, 0, segs({Seg{g.x.p, nullptr, net->f_in, net->f_in}}), n, g.Aenc.p, dA, nullptr, g.dZ.p,
                   dsegs({DSeg{nullptr, nullptr, net->f_in, 0}})));
    return HB_OK;
}

// normalised targets: u / u_ref; p: (p - p_ref) / (p_scale rho u_ref^2) on the mean, without the shift
// otherwise
void normalise(const Graph &g, int M, double p_scale, const double *harm, std::vector<float> &out) {
    out.resize(size_t(g.n) * 4 * M);
    const double su = 1.0 / g.u_ref, sp = 1.0 / (p_scale * g.rho * g.u_ref * g.u_ref);
    for (int i = 0; i < g.n; ++i)
        for (int f = 0; f < 4; ++f)
            for (int m = 0; m < M; ++m) {
                const size_t k = (size_t(i) * 4 + f) * M + m;
                double v = harm[k];
                if (f < 3) v *= su;
                else v = (m == 0 ? v - g.p_ref : v) * sp;
                out[k] = float(v);
            }
}

hb_status loss_grad(hb_mpnn *net, hb_problem *p, const double *target, float *loss_out) {
    Graph *g = nullptr;
    MP_TRY(graph_for(net, p, g));
    const int M = 2 * net->n_h + 1;
    std::vector<float> t;
    normalise(*g, M, net->p_scale, target, t);
    MP_CUDA(cudaMemcpyAsync(g->tgt.p, t.data(), t.size() * sizeof(float), cudaMemcpyHostToDevice, net->stream));
    MP_TRY(forward(net, *g));
    MP_CUDA(cudaMemsetAsync(net->loss.p, 0, sizeof(float), net->stream));
    const int64_t cnt = int64_t(g->n) * net->f_out;
    mse_kernel<<<grid_for(cnt, 256, 1184), 256, 0, net->stream>>>(g->out.p, g->tgt.p, cnt, g->dout.p, net->loss.p);
    MP_CUDA(cudaGetLastError());
    MP_TRY(backward(net, *g));
    float l = 0;
    MP_CUDA(cudaMemcpyAsync(&l, net->loss.p, sizeof(float), cudaMemcpyDeviceToHost, net->stream));
    MP_CUDA(cudaStreamSynchronize(net->stream));   // t (host) consumed, loss read
    if (loss_out) *loss_out = l;
    return HB_OK;
}

}  // namespace

extern "C" {

hb_status hb_mpnn_create(const hb_mpnn_config *cfg, int device, hb_mpnn **out) {
    if (!cfg || !out) return set_error(HB_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (cfg->hidden < 32 || cfg->hidden > 64 || cfg->layers < 1 || cfg->layers > 8 || cfg->n_h < 0 ||
        cfg->n_h > 11)
        return set_error(HB_ERR_INVALID_ARG, "hidden in [32,64], layers in [1,8], n_h in [0,11]");
    MP_CUDA(cudaSetDevice(device));
    hb_mpnn *net = new hb_mpnn();
    net->device = device;
    net->hidden = cfg->hidden;
    net->layers = cfg->layers;
    net->n_h = cfg->n_h;
    net->p_scale = cfg->p_scale > 0 ? cfg->p_scale : 1.0;
    net->f_in = kLearnedFeatures;
    net->f_out = 4 * (2 * cfg->n_h + 1);
    const int H = net->hidden;
    auto add = [&](int kin, int kout) {
        net->kin.push_back(kin);
        net->kout.push_back(kout);
        net->off.push_back(int(net->n_params));
        net->n_params += int64_t(kin + 1) * H + int64_t(H + 1) * kout;
    };
    add(net->f_in, H);
    for (int l = 0; l < net->layers; ++l) {
        add(2 * H + net->f_e, H);
        add(2 * H, H);
    }
    add(H, net->f_out);
    if (cudaStreamCreateWithFlags(&net->stream, cudaStreamNonBlocking) != cudaSuccess ||
        net->P.ensure(size_t(net->n_params)) != cudaSuccess || net->G.ensure(size_t(net->n_params)) != cudaSuccess ||
        net->M.ensure(size_t(net->n_params)) != cudaSuccess || net->V.ensure(size_t(net->n_params)) != cudaSuccess ||
        net->P16.ensure(size_t(net->n_params)) != cudaSuccess || net->loss.ensure(1) != cudaSuccess) {
        delete net;
        return set_error(HB_ERR_OOM, "network allocation failed");
    }
    // He-style initialisation, zero biases; the output layers of the message and update MLPs start
    // small (x 0.1) so that summed messages (about 14 per node on tetrahedral meshes) and the residual
    // updates leave the node states at their encoder scale at the start of training
    std::vector<float> p(size_t(net->n_params), 0.f);
    std::mt19937_64 rng(uint64_t(cfg->seed));
    std::normal_distribution<double> nd(0.0, 1.0);
    for (size_t k = 0; k < net->kin.size(); ++k) {
        const int kin = net->kin[k], kout = net->kout[k];
        const bool inner = k > 0 && k + 1 < net->kin.size();
        float *w = &p[size_t(net->off[k])];
        for (int i = 0; i < kin * H; ++i) w[i] = float(nd(rng) * std::sqrt(2.0 / kin));
        float *w2 = w + (kin + 1) * H;
        const double s2 = std::sqrt(1.0 / H) * (inner ? 0.1 : 1.0);
        for (int i = 0; i < H * kout; ++i) w2[i] = float(nd(rng) * s2);
    }
    *out = net;
    return hb_mpnn_set_params(net, p.data());
}

hb_status hb_mpnn_set_tensor_cores(hb_mpnn *net, int enable) {
    if (!net) return set_error(HB_ERR_INVALID_ARG, "null network");
    net->tensor_cores = enable != 0;
    return HB_OK;
}

hb_status hb_mpnn_destroy(hb_mpnn *net) {
    if (!net) return HB_OK;
    cudaSetDevice(net->device);
    cudaStreamSynchronize(net->stream);
    cudaStream_t s = net->stream;
    delete net;
    cudaStreamDestroy(s);
    return HB_OK;
}

int64_t hb_mpnn_num_params(const hb_mpnn *net) { return net ? net->n_params : 0; }

hb_status hb_mpnn_get_params(hb_mpnn *net, float *host) {
    if (!net || !host) return set_error(HB_ERR_INVALID_ARG, "null argument");
    MP_CUDA(cudaMemcpy(host, net->P.p, size_t(net->n_params) * sizeof(float), cudaMemcpyDeviceToHost));
    return HB_OK;
}

hb_status hb_mpnn_set_params(hb_mpnn *net, const float *host) {
    if (!net || !host) return set_error(HB_ERR_INVALID_ARG, "null argument");
    MP_CUDA(cudaSetDevice(net->device));
    MP_CUDA(cudaMemcpy(net->P.p, host, size_t(net->n_params) * sizeof(float), cudaMemcpyHostToDevice));
    to_bf16_kernel<<<grid_for(net->n_params, 256, 1184), 256, 0, net->stream>>>(net->P.p, net->P16.p, net->n_params);
    MP_CUDA(cudaGetLastError());
    MP_CUDA(cudaMemsetAsync(net->M.p, 0, size_t(net->n_params) * sizeof(float), net->stream));
    MP_CUDA(cudaMemsetAsync(net->V.p, 0, size_t(net->n_params) * sizeof(float), net->stream));
    MP_CUDA(cudaStreamSynchronize(net->stream));
    net->step = 0;
    return HB_OK;
}

hb_status hb_mpnn_loss_grad(hb_mpnn *net, hb_problem *p, const double *target, float *loss, float *grad) {
    if (!net || !p || !target) return set_error(HB_ERR_INVALID_ARG, "null argument");
    MP_CUDA(cudaSetDevice(net->device));
    MP_TRY(loss_grad(net, p, target, loss));
    if (grad) MP_CUDA(cudaMemcpy(grad, net->G.p, size_t(net->n_params) * sizeof(float), cudaMemcpyDeviceToHost));
    return HB_OK;
}

hb_status hb_mpnn_train_step(hb_mpnn *net, hb_problem *p, const double *target, float lr, float *loss) {
    if (!net || !p || !target) return set_error(HB_ERR_INVALID_ARG, "null argument");
    if (!(lr > 0)) return set_error(HB_ERR_INVALID_ARG, "learning rate must be > 0");
    MP_CUDA(cudaSetDevice(net->device));
    MP_TRY(loss_grad(net, p, target, loss));
    ++net->step;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, float(net->step)), c2 = 1.f - std::pow(b2, float(net->step));
    adam_kernel<<<grid_for(net->n_params, 256, 1184), 256, 0, net->stream>>>(
        net->P.p, net->P16.p, net->G.p, net->M.p, net->V.p, net->n_params, lr, b1, b2, 1e-8f, c1, c2);
    MP_CUDA(cudaGetLastError());
    MP_CUDA(cudaStreamSynchronize(net->stream));
    return HB_OK;
}

hb_status hb_mpnn_predict(hb_mpnn *net, hb_problem *p, double *harmonics) {
    if (!net || !p || !harmonics) return set_error(HB_ERR_INVALID_ARG, "null argument");
    MP_CUDA(cudaSetDevice(net->device));
    Graph *g = nullptr;
    MP_TRY(graph_for(net, p, g));
    MP_TRY(forward(net, *g));
    const int M = 2 * net->n_h + 1;
    std::vector<float> o(size_t(g->n) * 4 * M);
    MP_CUDA(cudaMemcpyAsync(o.data(), g->out.p, o.size() * sizeof(float), cudaMemcpyDeviceToHost, net->stream));
    MP_CUDA(cudaStreamSynchronize(net->stream));
    const double su = g->u_ref, sp = net->p_scale * g->rho * g->u_ref * g->u_ref;
    for (int i = 0; i < g->n; ++i)
        for (int f = 0; f < 4; ++f)
            for (int m = 0; m < M; ++m) {
                const size_t k = (size_t(i) * 4 + f) * M + m;
                double v = o[k];
                if (f < 3) v *= su;
                else v = v * sp + (m == 0 ? g->p_ref : 0.0);
                harmonics[k] = v;
            }
    return HB_OK;
}

hb_status hb_mpnn_graph(hb_mpnn *net, hb_problem *p, float *x, int32_t *src, int32_t *dst, float *e,
                        int64_t *n_edges) {
    if (!net || !p || !n_edges) return set_error(HB_ERR_INVALID_ARG, "null argument");
    MP_CUDA(cudaSetDevice(net->device));
    Graph *g = nullptr;
    MP_TRY(graph_for(net, p, g));
    *n_edges = g->ne;
    if (x) MP_CUDA(cudaMemcpy(x, g->x.p, size_t(g->n) * net->f_in * sizeof(float), cudaMemcpyDeviceToHost));
    if (src) MP_CUDA(cudaMemcpy(src, g->src.p, size_t(g->ne) * sizeof(int), cudaMemcpyDeviceToHost));
    if (dst) MP_CUDA(cudaMemcpy(dst, g->dst.p, size_t(g->ne) * sizeof(int), cudaMemcpyDeviceToHost));
    if (e) MP_CUDA(cudaMemcpy(e, g->e.p, size_t(g->ne) * net->f_e * sizeof(float), cudaMemcpyDeviceToHost));
    return HB_OK;
}

hb_status hb_mpnn_warm_start(hb_mpnn *net, hb_problem *p) {
    if (!net || !p) return set_error(HB_ERR_INVALID_ARG, "null argument");
    LearnedInputs in;
    MP_TRY(learned_inputs(p, in));
    std::vector<double> h(size_t(in.n_nodes) * 4 * (2 * in.n_h + 1));
    MP_TRY(hb_mpnn_predict(net, p, h.data()));
    return learned_set_initial(p, h.data());
}

}  // extern "C"
