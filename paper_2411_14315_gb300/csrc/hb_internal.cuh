// Internal declarations shared by the CUDA translation units of libhbgls (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstddef>
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <vector>

namespace hb {

// SM count of the current device (cached per device; problems may live on several devices).
inline int device_sms() {
    static std::atomic<int> cache[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    int n = cache[dev].load(std::memory_order_relaxed);
    if (n <= 0) {
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        n = std::max(1, n);
        cache[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

// Launch setup of kernels, per kernel and device: the dynamic shared memory a kernel was opted into and
// its resident blocks per SM for a given dynamic shared-memory size.  The kernels are shared by every
// problem, on any device and host thread, so the cache is keyed by kernel and device and guarded.
struct LaunchCache {
    std::mutex m;
    std::map<std::pair<const void *, int>, size_t> opted;              // (kernel, device) -> opted smem
    std::map<std::tuple<const void *, int, size_t>, int> per_sm;       // (kernel, device, smem) -> blocks/SM
};

template <typename K>
int cached_blocks_per_sm(LaunchCache &c, K kern, int block, size_t smem) {
    int dev = 0;
    cudaGetDevice(&dev);
    const void *kf = reinterpret_cast<const void *>(kern);
    std::lock_guard<std::mutex> lock(c.m);
    if (smem > 48 * 1024) {
        size_t &o = c.opted[std::make_pair(kf, dev)];
        if (smem > o) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
            o = smem;
        }
    }
    const auto key = std::make_tuple(kf, dev, smem);
    const auto it = c.per_sm.find(key);
    if (it != c.per_sm.end()) return it->second;
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, block, smem);
    per = std::max(1, per);
    c.per_sm[key] = per;
    return per;
}

// Kernel variants of the fused element pass.
enum Mode : int {
    MODE_RES = 0,    // residual, Eq. (Rmc)
    MODE_JVP = 1,    // paper tangent (P + C) v, Eqs. (ptangent), (K_mat), (ctangent), (F_mat)
    MODE_JVE = 2,    // exact Jacobian-vector product
    MODE_DIAG = 3,   // Jacobi diagonal of P (+ pseudo mass), Sec. 2.3
    MODE_TRES = 4,   // time-domain GLS residual of one time level (Sec. 3, Eq. tauhat): the argument
                     // slot of the direction holds du/dt; Galerkin rho M du/dt, no H terms
    MODE_JVA = 5     // paper tangent through the assembled operator (host-side dispatch only)
};

constexpr int kGeomStride = 16;       // per element: grad N_a (4 x 3), V, C_I nu^2 G:G, 2 pad
constexpr int kMaxN = 31;             // largest number of time instances supported
constexpr int kJvpVariants = 7;       // launch variants of the FP32 paper-tangent element pass
constexpr double kCI = 3.0;           // Eq. (tau)
// 4-point degree-2 Gauss rule on a tetrahedron (barycentric coordinates of the points)
constexpr double kQA = 0.5854101966249685;
constexpr double kQB = 0.1381966011250105;

// Fields per local node staged in shared memory, by mode.
// JVP stages y, v and W = shift v + rho H v (the F block is applied as rho M (H v): M and H commute;
// the pseudo-time shift uses the same mass matrix); RES stages y and
// H u; JVE stages y, H u, v, H v.  Element contributions that need no instance coupling go straight to
// global memory; RES and JVE accumulate T (3 fields) per patch node in shared memory for H T.
__host__ __device__ constexpr int in_fields(int mode) {
    return mode == MODE_RES ? 7 : mode == MODE_JVP ? 11 : mode == MODE_JVE ? 14 : mode == MODE_TRES ? 8 : 4;
}
// Row stride of the staged / gathered W = shift v + rho H v rows (3 N values): padded to 16 bytes, so a
// node's W row can be copied with 16-byte asynchronous copies.
__host__ __device__ constexpr int w_stride(int N, int tsize) { return (3 * N * tsize + 15) / 16 * 16 / tsize; }
__host__ __device__ constexpr int out_fields(int mode) {
    return (mode == MODE_RES || mode == MODE_JVE) ? 3 : 0;
}

// Element patches: elements renumbered so each patch's elements are contiguous; each patch lists its
// distinct nodes; each element stores its 4 nodes as local indices (uint8) into that list.
// Per patch one slot of slot_ints(nl_max) ints (a multiple of 16 bytes): [0] first element, [1] element
// count, [2] node count, [3] count of nodes with prescribed velocity, [4 + l] global id of local node l,
// bit 31 set when its velocity is prescribed (Dirichlet).
__host__ __device__ constexpr int slot_ints(int nl_max) { return 4 + ((nl_max + 3) & ~3); }
constexpr uint32_t kDirBit = 0x80000000u;

template <typename T>
struct PatchView {
    int n_patches;
    int nl_max;                    // largest node count of a patch
    int ep_max;                    // largest element count of a patch
    int slot_stride;               // ints per slot, slot_ints(nl_max)
    const int *slots;              // [P][slot_stride]
    const uint32_t *lconn;         // [E]
    const T *geom;                 // [E][kGeomStride]
};

template <typename T>
struct ElemArgs {
    PatchView<T> pv;
    const T *y;                    // state, instance layout [n][4][N]
    const T *v;                    // direction (JVP, JVE); du/dt (TRES)
    T *out;                        // accumulated output, instance layout (zeroed by the caller)
    const T *H;                    // [N][N]
    const uint8_t *flag;           // per node, bit 0: Dirichlet velocity
    int N;
    T rho, mu, shift;
    const T *W = nullptr;          // JVP: W = shift v + rho H v per node, rows of w_stride(N) (a global
                                   // spectral pass), gathered instead of formed per patch; nullptr: per patch
    T omega2 = 0;                  // acceleration term of tau_hat (Eq. tauhat); 0 for the HB passes
    int ls_mass = 0;               // time domain (one instance): the shift also enters the least-squares L
                                   // of the tangent (d(du/dt) = shift / rho d u); not its Jacobi diagonal
    const double *shift_dev = nullptr;   // if set, the shift is read from device memory instead
    int variant = 0;               // launch variant of the FP32 paper-tangent pass, [0, kJvpVariants)
    int *err = nullptr;            // device status word of the pipelined pass: a bounded wait that gave up
                                   // stores a nonzero code (left untouched otherwise)
    int rbvms = 0;                 // residual and exact Jacobian: add the full-RBVMS cross- and
                                   // Reynolds-stress terms of u' = -tau L / rho (Sec. 2.2, remark 2)
    T *cbuf = nullptr;             // JVP, deterministic scatter: per-element contribution slots
                                   // [E (patch order)][4 nodes][4 fields][N], gathered per node afterwards
};

// Deterministic scatter (no floating-point atomics): the element pass stores each element's contributions
// in its own slot of cbuf, [element in patch order][4 nodes][F fields][N], F = 7 for the residual and the
// exact Jacobian (4 direct rows, then the 3 rows of T that go through H) and 4 otherwise; Neumann faces
// store theirs in fbuf, [face][3 nodes][3 fields][N].  The gather sums, per node, field and instance, its
// element slots (eslot = element x 4 + local node) and face slots (fslot = face x 3 + local node) in the
// fixed order of the lists, and then out += H T on the velocity rows; prescribed velocity rows get
// presc (0: 0, 1: 1, 2: v).
__host__ __device__ constexpr int det_slot_values(int mode) { return (mode == MODE_RES || mode == MODE_JVE) ? 28 : 16; }

template <typename T>
struct DetGatherArgs {
    int64_t n_nodes;
    int N, F, presc;
    const int *eptr, *eslot;       // node -> element slots, CSR over nodes
    const T *cbuf;
    const int *fptr, *fslot;       // node -> face slots (null: no faces)
    const T *fbuf;
    const uint8_t *flag;
    const T *v;                    // presc 2
    const T *H;                    // F = 7: the N x N operator H
    T *tbuf;                       // F = 7: [n_nodes][3][N] scratch (sum of T)
    T *out;
};
template <typename T>
void launch_det_gather(const DetGatherArgs<T> &a, cudaStream_t s);

// Boundary (Neumann) faces.
template <typename T>
struct FaceArgs {
    int n_faces;                   // Neumann faces
    const int *fnodes;             // [F][3]
    const T *fgeo;                 // [F][4]: outward unit normal, area
    const int *foutlet;            // [F] outlet index or -1 (traction free)
    const T *hbase;                // [n_out][N]: -P_d(t_n)
    const T *R;                    // [n_out] resistance (0 for pressure outlets)
    T *Q;                          // [n_out][N] outlet flux scratch (zeroed by caller)
    const uint8_t *flag;
    const T *y;
    const T *v;
    T *out;
    int N;
    T rho, beta;
    T *fbuf = nullptr;             // deterministic scatter: per-face slots [F][3 nodes][3 fields][N]
    const int *optr = nullptr;     // and the outlet flow rates summed in a fixed order: faces of outlet o
    const int *oface = nullptr;    // are oface[optr[o] .. optr[o + 1])
};

// shared memory of one element-pass block; slot_cap = 0: the patch set's own slot size
size_t elem_smem_bytes(int mode, int N, int nl_max, int ep_max, size_t tsize, int slot_cap = 0);

template <typename T>
void launch_elem(int mode, const ElemArgs<T> &a, int grid, cudaStream_t s);
template <typename T>
void launch_geom(const double *xyz, const int *tets_patch_order, int n_tets, double nu, T *geom,
                 cudaStream_t s);
// FP32 geometry records carry the packed local connectivity of their patch in slot 14 (read by the
// pipelined paper-tangent pass, which copies the geometry and nothing else per element)
void launch_pack_conn(const uint32_t *lconn, float *geom, int n_tets, cudaStream_t s);
// dynamic shared memory of the pipelined pass (two stages), 0 if it has no kernel for N
size_t pipe_smem_bytes(int N, int nl_max, int ep_max);
// persistent element pass over the patches of several problems that share one instance count N: args on
// the device; batch slot i (bslot_stride ints at bslots + i * bslot_stride) = [problem index, 0, 0, 0,
// that problem's slot of the patch]; the group's items are [item_begin, item_end); *counter must be 0 at
// launch; the layout's slot buffers take bslot_stride ints each
template <typename T>
struct BatchGroup {
    const ElemArgs<T> *args;
    const int *bslots;
    int bslot_stride, N, item_begin, item_end;
    int variant;                   // launch variant of the FP32 paper-tangent pass
    int *counter;
};
template <typename T>
void launch_batch_elem(int mode, const BatchGroup<T> &g, size_t smem, int grid, cudaStream_t s);
// outlet flow rates (resistance outlets only; Q must be cleared before) then face terms
template <typename T>
void launch_faces(int mode, const FaceArgs<T> &a, bool has_resistance, int n_out, cudaStream_t s);

// sampling of boundary waveforms (Eq. upgh_def at the instances of Eq. upghharm)
void launch_sample_waveforms(const double *coef, int n_wave, int n_h, int N, double T, double *W,
                             cudaStream_t s);
void launch_apply_dirichlet(const int *dir_nodes, int n_dir, const double *g, double *y, int N,
                            cudaStream_t s);
void launch_harmonics(const double *y, double *coef, int64_t rows, int N, int n_h, int inverse,
                      double T, cudaStream_t s);

// vector kernels
template <typename A, typename B>
void launch_convert(const A *x, B *y, int64_t n, cudaStream_t s);
void launch_axpy(double a, const double *x, double *y, int64_t n, cudaStream_t s);
// FP32 copy of a state [n / (4 N)][4][N] with p_off subtracted from its pressure: the frozen state of the
// mixed-precision operators, which use the pressure only through its gradient (exact Jacobian), so an
// outlet pressure level far above the dynamic pressure does not cost FP32 digits
void launch_convert_state(const double *y, float *y32, int64_t n, int N, double p_off, cudaStream_t s);
void launch_scale_copy(double a, const double *x, double *y, int64_t n, cudaStream_t s);
// z = x * dinv in z's precision (right Jacobi preconditioning); dinv = 1 / d
template <typename T>
void launch_precond(const double *x, const double *dinv, T *z, int64_t n, cudaStream_t s);
void launch_reciprocal(const double *d, double *dinv, int64_t n, cudaStream_t s);   // d == dinv allowed
// partials[nb * (k + 1)]; result[k + 1] = (V_j . w for j < k, w . w)
// With a non-null gate that holds 0 at run time, launch_multidot writes zeros and launch_multiaxpy_norm
// leaves w and result unchanged (the second, conditional pass of classical Gram-Schmidt).
void launch_multidot(const double *V, int64_t ld, int k, const double *w, int64_t n, double *partials,
                     double *result, cudaStream_t s, const int *gate = nullptr);
// w -= sum_j h[j] V_j; result[0] = ||w||^2 after the update (partials scratch as above)
void launch_multiaxpy_norm(const double *V, int64_t ld, int k, const double *h, double *w, int64_t n,
                           double *partials, double *result, cudaStream_t s, const int *gate = nullptr);
void launch_reorth_gate(const double *before2, const double *after2, int *gate, cudaStream_t s);
// device-side GMRES bookkeeping (Hessenberg column, Givens rotations, residual estimate)
void launch_arnoldi_update(int j, int m, const double *h1, const double *h2, const double *nrm2, double *R,
                           double *cs, double *sn, double *g, double *resid, double *invnorm, cudaStream_t s);
void launch_cycle_init(const double *beta2, int m, double *g, double *invbeta, cudaStream_t s);
void launch_scale_dev(const double *x, const double *sp, double *y, int64_t n, cudaStream_t s);
// y = sum_j c[j] V_j (c on device)
void launch_combine(const double *V, int64_t ld, int k, const double *c, double *y, int64_t n,
                    cudaStream_t s);
void launch_dot(const double *x, const double *y, int64_t n, double *partials, double *result,
                cudaStream_t s);

// time-domain marching (generalized-alpha; node rows of 4 values, [n][4])
// out[r] = series r at the period fraction frac (real series [rows][2 n_h + 1]: a0, a1, b1, ...)
void launch_series_at(const double *coef, int64_t rows, int n_h, double frac, double *out, cudaStream_t s);
// u1 = un, du1 = cg dun (cg = (gamma - 1) / gamma); prescribed velocities u1 = g (rows [n_dir][3]) with
// du1 = (g - un) inv_gdt + cg dun
void launch_galpha_predict(const double *un, const double *dun, double *u1, double *du1, int64_t n, double cg,
                           const int *dir_nodes, int n_dir, const double *g, double inv_gdt, cudaStream_t s);
void launch_galpha_stage(const double *un, const double *u1, const double *dun, const double *du1, double *ya,
                         double *dya, int64_t n, double af, double am, cudaStream_t s);
void launch_galpha_correct(double *u1, double *du1, const double *d, int64_t n, double inv_gdt, cudaStream_t s);
void launch_put_instance(const double *src, double *dst, int64_t n4, int k, int N, cudaStream_t s);
void launch_vel_norm2(const double *x, int64_t n, double *partials, double *result, cudaStream_t s);

// Assembled paper tangent (hb_assembled.cu): per node pair and instance [pair][8][N] = K, G_1..3, D_1..3,
// L, and per pair the consistent mass.
template <typename T>
struct AsmArgs {
    int64_t n_tets;
    int N;
    const int *tets;               // [E][4] global node ids (the assembly's element order)
    const T *geom;                 // [E][kGeomStride] in the same order
    const int *epos;               // [E][16] pair slot of (local a, local b) = 4 a + b
    const uint8_t *flag;           // per node, bit 0: prescribed velocity
    const T *y;                    // frozen state [n][4][N]
    T *coef;                       // [nnz][8][N], cleared before the assembly
    T *mass;                       // [nnz], cleared before the assembly
    T rho, mu;
    T omega2 = 0;                  // constant added under the root of tau (time-discretisation term)
    // deterministic assembly (set: one thread per row and instance adds the row's element blocks in
    // list order): node A's (element x 4 + local index) entries are rslot[rptr[A] .. rptr[A + 1])
    int64_t n_nodes = 0;
    const int *rptr = nullptr, *rslot = nullptr;
};
template <typename T>
struct SpmvArgs {
    int64_t n_nodes;
    int N, w_stride;               // W rows of w_stride values
    const int *rowptr, *col;       // CSR of the node pairs (rows = nodes, the diagonal included)
    const T *coef, *mass;
    const T *v;                    // direction [n][4][N]
    const T *W;                    // shift v + rho H v, rows [n][w_stride], 0 on prescribed velocities
    T *out;                        // [n][4][N], every entry written
    const uint8_t *flag;
};
template <typename T>
void launch_assemble(const AsmArgs<T> &a, cudaStream_t s);
template <typename T>
void launch_assemble_mass(const AsmArgs<T> &a, cudaStream_t s);
// W = shift v + rho H v (velocity rows; H [N][N]; shift from shift_dev if set), rows of ws values.
// FP32 at N = 9, 13, 21: path 0 = tcgen05 tensor cores with a TMEM accumulator (needs err, the status word
// of its bounded waits), 1 = warp-level mma.sync, 2 = FP32 FMAs; FP64 and other N always take the FMAs.
template <typename T>
void launch_spectral_w(const T *v, const T *H, const uint8_t *flag, T *W, int ws, int64_t n_nodes, int N, T rho,
                       T shift, const double *shift_dev, cudaStream_t s, int path = 1, int *err = nullptr);
// the tcgen05 form (hb_spectral_tc5.cu); false if it has no kernel for N
bool launch_spectral_w_tc5(const float *v, const float *H, const uint8_t *flag, float *W, int64_t n_nodes, int N,
                           float rho, float shift, const double *shift_dev, int *err, cudaStream_t s);
template <typename T>
void launch_spmv(const SpmvArgs<T> &a, cudaStream_t s);
// z = (node-block diagonal of the assembled tangent + shift M_AA)^-1 x per node and instance; dpos[A] is
// the slot of the pair (A, A)
template <typename T, typename Z>
void launch_block_jacobi(const T *coef, const T *mass, const int *dpos, const uint8_t *flag, const double *x, Z *z,
                         int64_t n_nodes, int N, double shift, const double *shift_dev, cudaStream_t s);

// Aggregation multigrid on the assembled tangent (hb_amg.cu)
template <typename T>
void launch_amg_restrict(const int *aptr, const int *aidx, const uint8_t *flag_f, const T *r_f, T *b_c, int64_t n_c,
                         int N, cudaStream_t s);
template <typename T>
void launch_amg_prolong(const int *agg, const uint8_t *flag_f, const T *x_c, T *x_f, int64_t n_f, int N,
                        cudaStream_t s);
template <typename T>
void launch_amg_coarse(const int *cptr, const int *cidx, const uint8_t *mmask, const T *coef_f, const T *mass_f,
                       T *coef_c, T *mass_c, int64_t nnz_c, int N, bool with_mass, cudaStream_t s);
template <typename T>
void launch_amg_smooth(const T *coef, const T *mass, const int *dpos, const uint8_t *flag, const T *r, T *x,
                       int64_t n_nodes, int N, double omega, double shift, const double *shift_dev, int accumulate,
                       cudaStream_t s);
template <typename T>
void launch_amg_sub(const T *b, const T *ax, T *r, int64_t n, cudaStream_t s);

// Inputs of the learned warm start taken from a problem (host copies).
constexpr int kLearnedFeatures = 32;  // per-node input features of the network
struct LearnedInputs {
    int64_t n_nodes = 0, n_tets = 0;
    int n_h = 0;
    std::vector<double> xyz;          // [n][3]
    std::vector<int32_t> tets;        // [E][4]
    std::vector<uint8_t> flags;       // bit 0 wall, bit 1 inflow, bit 2 outlet / traction cap
    std::vector<double> profile;      // [n][3] inflow profile (0 off the inflow caps)
    std::vector<double> wave;         // real series of the first inflow waveform [2 n_h + 1]
    double u_ref = 1, p_ref = 0, rho = 1;
};

}  // namespace hb
