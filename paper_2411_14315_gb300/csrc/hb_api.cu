// Host runtime and C ABI of libhbgls: problem set-up (face orientation, Morton-ordered element patches,
// geometry), boundary data, operator dispatch and the pseudo-time Newton-GMRES solve
// (arXiv 2411.14315, Sec. 2.3: Eq. NR, Eq. splitK, pseudo time stepping, Jacobi + GMRES).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "hb_internal.cuh"
#include "hbgls.h"

using namespace hb;

namespace {

thread_local std::string g_err;

hb_status fail(hb_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

#define HB_CUDA(expr)                                                                                   \
    do {                                                                                                \
        cudaError_t _e = (expr);                                                                        \
        if (_e != cudaSuccess)                                                                          \
            return fail(_e == cudaErrorMemoryAllocation ? HB_ERR_OOM : HB_ERR_CUDA,                     \
                        std::string(#expr) + ": " + cudaGetErrorString(_e));                            \
    } while (0)

#define HB_TRY(expr)                                                                                    \
    do {                                                                                                \
        hb_status _s = (expr);                                                                          \
        if (_s != HB_OK) return _s;                                                                     \
    } while (0)

#define HB_LAUNCHED(p, k)                                                                               \
    do {                                                                                                \
        (p)->launches += (k);                                                                           \
        cudaError_t _e = cudaGetLastError();                                                            \
        if (_e != cudaSuccess) return fail(HB_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(_e)); \
    } while (0)

constexpr double kC1 = 1.5;   // generalized-alpha with rho_inf = 0 (Sec. 2.3)

template <typename T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept : p(o.p), n(o.n) {
        o.p = nullptr;
        o.n = 0;
    }
    DBuf &operator=(DBuf &&o) noexcept {
        if (this != &o) {
            release();
            p = o.p;
            n = o.n;
            o.p = nullptr;
            o.n = 0;
        }
        return *this;
    }
    ~DBuf() { release(); }
    void swap(DBuf &o) {
        std::swap(p, o.p);
        std::swap(n, o.n);
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
};

template <typename T>
struct PatchSetDev {
    int P = 0, nl_max = 0, ep_max = 0;
    DBuf<int> slots;                    // [P][slot_ints(nl_max)], see PatchView
    DBuf<uint32_t> lconn;
    DBuf<T> geom;
    std::vector<int> h_eptr, h_nptr, h_nodes;   // host copies, to rebuild the slots' Dirichlet bits
    DBuf<int> det_ptr, det_slot;        // deterministic scatter: node -> (element in patch order x 4 + a)
    PatchView<T> view() const {
        return PatchView<T>{P, nl_max, ep_max, slot_ints(nl_max), slots.p, lconn.p, geom.p};
    }
};

struct Inflow {
    int tag;
    std::vector<double> profile;   // [n_nodes][3] or empty = parabolic (separable data)
    std::vector<double> coef;      // real series (a0, a1, b1, ...) of the waveform (separable data)
    std::vector<double> harm;      // [n_nodes][3][2 n_h + 1] per-point harmonics (general data) or empty
};

struct Outlet {
    int tag;
    double R;                      // 0 for a pressure outlet
    std::vector<double> coef;
};

}  // namespace

struct hb_problem {
    uint64_t uid = 0;                // unique per problem in this process
    std::vector<int32_t> tets_morton; // elements in Morton order of their centroids (patch input)
    hb_mpnn *learned = nullptr;      // attached warm-start network (not owned)
    std::vector<double> h_prof;      // per-node Dirichlet profile (after prepare_bc)
    std::vector<int> h_wave;         // per-node: -2 free, -1 wall, >= 0 inflow index
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int64_t n_nodes = 0, n_tets = 0, n_faces = 0;
    int n_h = 0, N = 1;
    double rho = 1, mu = 1, T = 1, omega = 1, beta = 0.2;
    std::vector<double> xyz;
    std::vector<int32_t> tets, faces, face_tag;
    std::vector<double> fnormal, farea;
    double vol_mean = 0, vol_min = 0;
    PatchSetDev<float> ps32;         // FP32 passes except the exact Jacobian's
    PatchSetDev<float> ps32e;        // FP32 exact-Jacobian pass (smaller patches: more staged fields)
    PatchSetDev<double> ps64;
    DBuf<double> d_xyz;
    DBuf<int> d_tets_ord;
    DBuf<double> H64;
    DBuf<float> H32;
    // boundary data
    std::vector<Inflow> inflows;
    std::vector<Outlet> outlets;
    bool bc_dirty = true;
    int n_dir = 0, n_nf = 0, n_out = 0;
    bool has_res = false;
    double u_c = 0;
    std::vector<double> level;       // mean outlet pressure per instance
    DBuf<int> d_dir_nodes, d_nf_nodes, d_nf_out;
    DBuf<uint8_t> d_flag;
    DBuf<double> d_dir_prof, d_g, d_W, d_coef;
    DBuf<double> d_nf_geo64, d_hbase64, d_R64, d_Q64;
    DBuf<float> d_nf_geo32, d_hbase32, d_R32, d_Q32;
    // state and work
    DBuf<double> y;
    bool y_set = false;
    DBuf<double> w64a, w64b;
    DBuf<float> w32a, w32b, w32c;
    DBuf<double> scratch, small;
    int64_t launches = 0;
    int64_t dev_bytes = 0;
    int sm_count = 148;
    // Krylov storage (lazily sized)
    int km = 0;
    DBuf<double> kV, kz64, kdx, kdiag, kres, ktmp, kh;   // kdiag: inverse Jacobi diagonal during a solve
    DBuf<float> kz32, kw32, ky32, kdiag32;
    // graph-captured GMRES restart cycles, one per operator (paper tangent / exact)
    struct CycleGraph {
        cudaGraphExec_t exec = nullptr;
        int m = 0, precision = -1, precond = -1;
        double shift = 0;
        int64_t launches = 0;
        uint64_t gen = 0;              // the problem's settings generation it was captured at
    } cycle[3];                        // paper tangent, exact Jacobian, assembled paper tangent
    // settings generation: bumped by every change that captured launches depend on (kernel arguments
    // taken by value, buffers that can be reallocated): boundary data, patches, backflow, stabilisation,
    // summation mode, spectral path, launch variant.  Captured graphs are replayed only at their own.
    uint64_t gen = 0;
    DBuf<double> gm;
    DBuf<int> gate;
    DBuf<double> shift_dev;
    double shift_host = 0;
    // element-kernel timing
    bool prof_on = false;
    DBuf<double> ylearn, kd;              // learned prediction and the direction towards it (use_learned 2)
    DBuf<double> yprev;                   // state before a Newton step (line search)
    // assembled paper tangent (Sec. 4's condensed storage): CSR of node pairs, element -> pair slots
    struct Assembled {
        int64_t nnz = 0;
        DBuf<int> rowptr, col, epos, tets, dpos;   // dpos[A]: slot of the pair (A, A)
        DBuf<float> geom32, coef32, mass32, W32;
        DBuf<double> geom64, coef64, mass64, W64;
        bool ready32 = false, ready64 = false;   // coefficients assembled (at the last state given)
        bool mass32_done = false, mass64_done = false;
        std::vector<int> h_rowptr, h_col;         // host copy of the pair structure (multigrid set-up)
        DBuf<int> det_ptr, det_slot;              // deterministic assembly: row node -> (element x 4 + a)
    } as;
    // aggregation multigrid on the assembled tangent (precond = 2): level 0 is `as`; levels 1.. are built
    struct AmgLevel {
        int64_t n = 0, nnz = 0;
        DBuf<int> rowptr, col, dpos;              // levels >= 1
        DBuf<uint8_t> flag;                       // levels >= 1 (bit 0: velocity prescribed)
        DBuf<int> agg, aptr, aidx;                // to the next level: node -> aggregate, aggregate -> nodes
        DBuf<int> cptr, cidx;                     // next level's pairs -> this level's pairs
        DBuf<uint8_t> mmask;                      // this level's pairs whose two nodes are free
        DBuf<float> coef32, mass32, x32, b32, r32, ax32, W32;
        DBuf<double> coef64, mass64, x64, b64, r64, ax64, W64;
    };
    std::vector<AmgLevel> amg;
    bool amg_mass32 = false, amg_mass64 = false;
    double omega2 = 0;                    // acceleration term of tau_hat in the element passes (time domain)
    int ls_mass = 0;                      // time domain: the shift enters the tangent's least-squares L too
    hb_problem *tm = nullptr;             // internal one-instance copy that runs the time-domain march
    DBuf<double> tm_un, tm_dun, tm_u1, tm_du1, tm_dya, tm_prev, d_march;
    bool march_done = false;
    bool learned_dir = false;
    int jvp_variant = 1;                  // launch variant of the FP32 paper-tangent pass
    DBuf<int> d_err;                      // status word of the pipelined element pass (0: no wait gave up)
    int stab = 0;                         // 0: GLS as printed; 1: full RBVMS (hb_set_stabilization)
    int spectral_path = 1;                // FP32 W pass: 0 tcgen05, 1 mma.sync, 2 FMAs (hb_set_spectral_path)
    int scatter = 1;                      // 0: deterministic (slots + fixed-order gather), 1: atomic (hb_set_scatter)
    DBuf<int> det_fptr, det_fslot;        // node -> Neumann-face slots (face x 3 + b)
    DBuf<int> det_optr, det_oface;        // resistance outlet o -> its Neumann faces, in face order
    DBuf<float> det_c32, det_t32, det_f32;     // element slots, T sums, face slots (FP32)
    DBuf<double> det_c64, det_t64, det_f64;    // (FP64)
    double ct_dt = 0;                     // coefficient of (1 / dt)^2 under the root of tau, dt = T / N
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev;
    size_t prof_used = 0;
};

namespace {

template <typename T>
hb_status dalloc(hb_problem *p, DBuf<T> &b, size_t n) {
    if (b.n >= n && b.p) return HB_OK;
    if (b.p) {
        p->dev_bytes -= int64_t(b.n * sizeof(T));
        b.release();
    }
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc(&b.p, n * sizeof(T));
    if (e != cudaSuccess) {
        b.p = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? HB_ERR_OOM : HB_ERR_CUDA,
                    std::string("cudaMalloc(") + std::to_string(n * sizeof(T)) + "): " + cudaGetErrorString(e));
    }
    b.n = n;
    p->dev_bytes += int64_t(n * sizeof(T));
    return HB_OK;
}

// set-up copies are synchronous: the host vectors are usually temporaries
template <typename T>
hb_status upload(hb_problem *p, DBuf<T> &b, const std::vector<T> &h) {
    HB_TRY(dalloc(p, b, h.size()));
    if (!h.empty()) {
        HB_CUDA(cudaMemcpyAsync(b.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, p->stream));
        HB_CUDA(cudaStreamSynchronize(p->stream));
    }
    return HB_OK;
}

// ct_dt (1 / dt)^2 with dt = 2 pi / (N w) = T / N, added under the root of Eq. (tau) (Sec. 2.2, remark 4)
double tau_dt_term(const hb_problem *p) {
    const double dt = p->T / double(p->N);
    return p->ct_dt / (dt * dt);
}

// mean outlet pressure level over outlets and instances (0 without outlets)
double p_level(const hb_problem *p) {
    double pr = 0;
    for (double v : p->level) pr += v / double(p->level.size());
    return pr;
}

inline uint64_t spread3(uint64_t x) {  // 21 bits -> every third bit
    x &= 0x1fffff;
    x = (x | x << 32) & 0x1f00000000ffffULL;
    x = (x | x << 16) & 0x1f0000ff0000ffULL;
    x = (x | x << 8) & 0x100f00f00f00f00fULL;
    x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
    x = (x | x << 2) & 0x1249249249249249ULL;
    return x;
}

// Greedy patches along the Morton order: close a patch when it would exceed NL nodes or EP elements.
// Inside a patch the elements are then re-sequenced so that an element shares no node with the `window`
// elements before it where possible: threads of one warp that handle the same instance of elements a
// short distance apart then add into different shared-memory addresses.
struct HostPatches {
    std::vector<int> eptr, nptr, nodes;
    std::vector<uint32_t> lconn;
    std::vector<int> perm;          // element k of the patch order is element perm[k] of the input order
    int nl_max = 0, ep_max = 0;
};

HostPatches build_patches(const std::vector<int32_t> &tets_ord, int64_t n_tets, int64_t n_nodes, int NL, int EP,
                          int window) {
    HostPatches hp;
    std::vector<int> stamp(size_t(n_nodes), -1), local(size_t(n_nodes), 0);
    std::vector<uint32_t> lc(static_cast<size_t>(n_tets));
    hp.eptr.push_back(0);
    hp.nptr.push_back(0);
    int pid = 0, cur_nodes = 0, cur_elems = 0;
    for (int64_t e = 0; e < n_tets; ++e) {
        const int32_t *t = &tets_ord[size_t(4 * e)];
        int fresh = 0;
        for (int a = 0; a < 4; ++a) {
            bool dup = false;
            for (int b = 0; b < a; ++b) dup |= (t[b] == t[a]);
            if (!dup && stamp[t[a]] != pid) ++fresh;
        }
        if (cur_elems > 0 && (cur_nodes + fresh > NL || cur_elems + 1 > EP)) {
            hp.eptr.push_back(int(e));
            hp.nptr.push_back(int(hp.nodes.size()));
            hp.nl_max = std::max(hp.nl_max, cur_nodes);
            hp.ep_max = std::max(hp.ep_max, cur_elems);
            ++pid;
            cur_nodes = 0;
            cur_elems = 0;
        }
        uint32_t packed = 0;
        for (int a = 0; a < 4; ++a) {
            if (stamp[t[a]] != pid) {
                stamp[t[a]] = pid;
                local[t[a]] = cur_nodes++;
                hp.nodes.push_back(t[a]);
            }
            packed |= uint32_t(local[t[a]]) << (8 * a);
        }
        lc[size_t(e)] = packed;
        ++cur_elems;
    }
    hp.eptr.push_back(int(n_tets));
    hp.nptr.push_back(int(hp.nodes.size()));
    hp.nl_max = std::max(hp.nl_max, cur_nodes);
    hp.ep_max = std::max(hp.ep_max, cur_elems);
    // re-sequence inside each patch
    hp.perm.resize(size_t(n_tets));
    hp.lconn.resize(size_t(n_tets));
    std::vector<int> cnt(256, 0), rem, placed;
    const int P = int(hp.eptr.size()) - 1;
    for (int q = 0; q < P; ++q) {
        const int e0 = hp.eptr[size_t(q)], e1 = hp.eptr[size_t(q + 1)];
        rem.clear();
        placed.clear();
        for (int e = e0; e < e1; ++e) rem.push_back(e);
        std::fill(cnt.begin(), cnt.end(), 0);
        for (int k = e0; k < e1; ++k) {
            size_t pick = 0;
            for (size_t j = 0; j < rem.size(); ++j) {
                const uint32_t c = lc[size_t(rem[j])];
                bool clash = false;
                for (int a = 0; a < 4; ++a) clash |= cnt[(c >> (8 * a)) & 255u] > 0;
                if (!clash) {
                    pick = j;
                    break;
                }
            }
            const int e = rem[pick];
            rem.erase(rem.begin() + long(pick));
            hp.perm[size_t(k)] = e;
            hp.lconn[size_t(k)] = lc[size_t(e)];
            placed.push_back(e);
            for (int a = 0; a < 4; ++a) ++cnt[(lc[size_t(e)] >> (8 * a)) & 255u];
            if (int(placed.size()) > window) {
                const uint32_t old = lc[size_t(placed[placed.size() - 1 - size_t(window)])];
                for (int a = 0; a < 4; ++a) --cnt[(old >> (8 * a)) & 255u];
            }
        }
    }
    return hp;
}

// Largest patch node cap whose shared-memory layout for `mode` fits `budget` bytes (3 elements per
// node), and whose layout for every mode fits the per-block hardware limit.
int choose_nl(int N, size_t ts, size_t budget, int mode) {
    const size_t hw = 227 * 1024;
    int nl = 8;
    for (int c = 8; c <= 160; ++c) {
        if (elem_smem_bytes(mode, N, c, 3 * c, ts) > budget) break;
        bool ok = true;
        for (int m = 0; m < 4; ++m) ok &= elem_smem_bytes(m, N, c, 3 * c, ts) <= hw;
        if (!ok) break;
        nl = c;
    }
    return nl;
}

// Per-patch slots: first element, element count, node count, Dirichlet node count, then the patch's
// node ids with bit 31 set on nodes whose velocity is prescribed (flag bit 0).
template <typename T>
hb_status upload_slots(hb_problem *p, PatchSetDev<T> &ps, const std::vector<uint8_t> *flag) {
    const int S = slot_ints(ps.nl_max);
    std::vector<int> sl(size_t(std::max(1, ps.P)) * size_t(S), 0);
    for (int q = 0; q < ps.P; ++q) {
        int *o = sl.data() + size_t(q) * size_t(S);
        const int k0 = ps.h_nptr[size_t(q)], k1 = ps.h_nptr[size_t(q + 1)];
        o[0] = ps.h_eptr[size_t(q)];
        o[1] = ps.h_eptr[size_t(q + 1)] - o[0];
        o[2] = k1 - k0;
        int nd = 0;
        for (int k = k0; k < k1; ++k) {
            const int node = ps.h_nodes[size_t(k)];
            const bool dir = flag && ((*flag)[size_t(node)] & 1);
            nd += dir ? 1 : 0;
            o[4 + (k - k0)] = dir ? int(uint32_t(node) | 0x80000000u) : node;
        }
        o[3] = nd;
    }
    return upload(p, ps.slots, sl);
}

// Lists of the deterministic scatter: node -> the slots whose node is it, in increasing slot order
// (counting sort of node_of_slot; entries < 0 are skipped).
void node_slot_lists(const std::vector<int> &node_of_slot, int64_t n_nodes, std::vector<int> &ptr,
                     std::vector<int> &list) {
    ptr.assign(size_t(n_nodes) + 1, 0);
    for (int nd : node_of_slot)
        if (nd >= 0) ++ptr[size_t(nd) + 1];
    for (int64_t i = 0; i < n_nodes; ++i) ptr[size_t(i) + 1] += ptr[size_t(i)];
    list.assign(size_t(ptr[size_t(n_nodes)]), 0);
    std::vector<int> fill(ptr.begin(), ptr.end() - 1);
    for (size_t k = 0; k < node_of_slot.size(); ++k)
        if (node_of_slot[k] >= 0) list[size_t(fill[size_t(node_of_slot[k])]++)] = int(k);
}

// Patches sized so that `size_mode`'s shared-memory layout fits `budget` (two blocks per SM for FP32,
// one for FP64), unless nl_override gives the node cap.
template <typename T>
hb_status make_patchset(hb_problem *p, PatchSetDev<T> &ps, const std::vector<int32_t> &tets_ord, size_t budget,
                        int nl_override = 0, int size_mode = MODE_JVP) {
    ++p->gen;                                     // new patch buffers
    const int NL = nl_override > 0 ? std::min(nl_override, 255) : choose_nl(p->N, sizeof(T), budget, size_mode);
    const int EP = 3 * NL;
    HostPatches hp = build_patches(tets_ord, p->n_tets, p->n_nodes, NL, EP, std::max(1, 31 / p->N));
    ps.P = int(hp.eptr.size()) - 1;
    ps.nl_max = hp.nl_max;
    ps.ep_max = hp.ep_max;
    HB_TRY(upload(p, ps.lconn, hp.lconn));
    ps.h_eptr = hp.eptr;
    ps.h_nptr = hp.nptr;
    ps.h_nodes = hp.nodes;
    HB_TRY(upload_slots(p, ps, nullptr));         // no Dirichlet nodes until boundary data are set
    std::vector<int> tets_p(size_t(4 * p->n_tets));
    for (int64_t k = 0; k < p->n_tets; ++k)
        for (int a = 0; a < 4; ++a) tets_p[size_t(4 * k + a)] = tets_ord[size_t(4 * hp.perm[size_t(k)] + a)];
    HB_TRY(upload(p, p->d_tets_ord, tets_p));
    {
        std::vector<int> ptr, list;
        node_slot_lists(tets_p, p->n_nodes, ptr, list);
        HB_TRY(upload(p, ps.det_ptr, ptr));
        HB_TRY(upload(p, ps.det_slot, list));
    }
    HB_TRY(dalloc(p, ps.geom, size_t(p->n_tets) * kGeomStride));
    launch_geom<T>(p->d_xyz.p, p->d_tets_ord.p, int(p->n_tets), p->mu / p->rho, ps.geom.p, p->stream);
    HB_LAUNCHED(p, 1);
    if constexpr (sizeof(T) == 4) {
        launch_pack_conn(ps.lconn.p, ps.geom.p, int(p->n_tets), p->stream);
        HB_LAUNCHED(p, 1);
    }
    HB_CUDA(cudaStreamSynchronize(p->stream));   // host vectors above are about to go out of scope
    return HB_OK;
}

template <typename T>
PatchSetDev<T> &patches(hb_problem *p, int mode = MODE_JVP);
template <>
PatchSetDev<float> &patches<float>(hb_problem *p, int mode) { return mode == MODE_JVE ? p->ps32e : p->ps32; }
template <>
PatchSetDev<double> &patches<double>(hb_problem *p, int) { return p->ps64; }

template <typename T>
const T *Hmat(hb_problem *p);
template <>
const float *Hmat<float>(hb_problem *p) { return p->H32.p; }
template <>
const double *Hmat<double>(hb_problem *p) { return p->H64.p; }

// ---------------------------------------------------------------------------------------------------
// boundary data

std::vector<double> real_series(const double *a, const double *b, int n_h) {
    std::vector<double> c(size_t(2 * n_h + 1), 0.0);
    c[0] = a[0];
    for (int k = 1; k <= n_h; ++k) {
        c[size_t(2 * k - 1)] = a[k];
        c[size_t(2 * k)] = b[k];
    }
    return c;
}

// parabolic unit-flow profile on cap `tag` (definition in hbgls.h); returns per-node vectors
void parabolic_profile(const hb_problem *p, int tag, std::vector<double> &prof) {
    prof.assign(size_t(3 * p->n_nodes), 0.0);
    double A = 0, c[3] = {0, 0, 0}, nrm[3] = {0, 0, 0};
    std::vector<int> nodes;
    for (int64_t f = 0; f < p->n_faces; ++f) {
        if (p->face_tag[size_t(f)] != tag) continue;
        const double S = p->farea[size_t(f)];
        A += S;
        for (int i = 0; i < 3; ++i) {
            double m = 0;
            for (int b = 0; b < 3; ++b) m += p->xyz[size_t(3 * p->faces[size_t(3 * f + b)] + i)] / 3.0;
            c[i] += S * m;
            nrm[i] += S * p->fnormal[size_t(3 * f + i)];
        }
        for (int b = 0; b < 3; ++b) nodes.push_back(p->faces[size_t(3 * f + b)]);
    }
    if (A <= 0) return;
    double nn = std::sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
    for (int i = 0; i < 3; ++i) {
        c[i] /= A;
        nrm[i] /= nn;
    }
    std::sort(nodes.begin(), nodes.end());
    nodes.erase(std::unique(nodes.begin(), nodes.end()), nodes.end());
    std::vector<double> r2(nodes.size());
    double R2 = 0;
    for (size_t k = 0; k < nodes.size(); ++k) {
        double d[3], dn = 0;
        for (int i = 0; i < 3; ++i) {
            d[i] = p->xyz[size_t(3 * nodes[k] + i)] - c[i];
            dn += d[i] * nrm[i];
        }
        double s = 0;
        for (int i = 0; i < 3; ++i) {
            const double e = d[i] - dn * nrm[i];
            s += e * e;
        }
        r2[k] = s;
        R2 = std::max(R2, s);
    }
    const double scale = 2.0 / (M_PI * R2);
    for (size_t k = 0; k < nodes.size(); ++k) {
        const double v = scale * std::max(0.0, 1.0 - r2[k] / R2);
        for (int i = 0; i < 3; ++i) prof[size_t(3 * nodes[k] + i)] = -v * nrm[i];
    }
}

template <typename T>
hb_status dirichlet_lists(hb_problem *p, PatchSetDev<T> &ps, const std::vector<uint8_t> &flag) {
    return upload_slots(p, ps, &flag);
}

hb_status prepare_bc(hb_problem *p) {
    if (!p->bc_dirty) return HB_OK;
    const int N = p->N, M = 2 * p->n_h + 1;
    const int64_t n = p->n_nodes;
    std::vector<int> wave(size_t(n), -2);      // -2 free, -1 wall, >= 0 inflow index
    std::vector<double> prof(size_t(3 * n), 0.0);
    for (size_t k = 0; k < p->inflows.size(); ++k) {
        const Inflow &in = p->inflows[k];
        std::vector<double> pp;
        const std::vector<double> *src = &in.profile;
        if (!in.harm.empty()) {            // general data: its mean (a0) stands for the profile
            pp.assign(size_t(3 * n), 0.0);
            for (int64_t a = 0; a < n; ++a)
                for (int i = 0; i < 3; ++i) pp[size_t(3 * a + i)] = in.harm[size_t((3 * a + i) * M)];
            src = &pp;
        } else if (in.profile.empty()) {
            parabolic_profile(p, in.tag, pp);
            src = &pp;
        }
        for (int64_t f = 0; f < p->n_faces; ++f) {
            if (p->face_tag[size_t(f)] != in.tag) continue;
            for (int b = 0; b < 3; ++b) {
                const int nd = p->faces[size_t(3 * f + b)];   // the cap set last wins
                wave[size_t(nd)] = int(k);
                for (int i = 0; i < 3; ++i) prof[size_t(3 * nd + i)] = (*src)[size_t(3 * nd + i)];
            }
        }
    }
    for (int64_t f = 0; f < p->n_faces; ++f)
        if (p->face_tag[size_t(f)] == 0)
            for (int b = 0; b < 3; ++b) wave[size_t(p->faces[size_t(3 * f + b)])] = -1;
    p->h_prof = prof;
    p->h_wave = wave;
    // harmonics of the Dirichlet data per Dirichlet node [n_dir][3][M]: 0 on walls, profile x waveform
    // series for separable inflows, the given per-point series otherwise
    std::vector<int> dir_nodes, dir_index(size_t(n), -1);
    std::vector<double> dir_harm;
    std::vector<uint8_t> flag(size_t(n), 0);
    for (int64_t a = 0; a < n; ++a) {
        const int w = wave[size_t(a)];
        if (w == -2) continue;
        dir_index[size_t(a)] = int(dir_nodes.size());
        dir_nodes.push_back(int(a));
        for (int i = 0; i < 3; ++i)
            for (int m = 0; m < M; ++m) {
                double c = 0.0;
                if (w >= 0) {
                    const Inflow &in = p->inflows[size_t(w)];
                    c = in.harm.empty() ? prof[size_t(3 * a + i)] * in.coef[size_t(m)]
                                        : in.harm[size_t((3 * a + i) * M + m)];
                }
                dir_harm.push_back(c);
            }
        flag[size_t(a)] = 1;
    }
    // Neumann faces: every cap that is not an inflow (walls are Dirichlet)
    std::vector<int> nf_nodes, nf_out;
    std::vector<double> nf_geo;
    for (int64_t f = 0; f < p->n_faces; ++f) {
        const int tag = p->face_tag[size_t(f)];
        if (tag == 0) continue;
        bool is_in = false;
        for (auto &in : p->inflows) is_in |= (in.tag == tag);
        if (is_in) continue;
        int o = -1;
        for (size_t k = 0; k < p->outlets.size(); ++k)
            if (p->outlets[k].tag == tag) o = int(k);
        for (int b = 0; b < 3; ++b) nf_nodes.push_back(p->faces[size_t(3 * f + b)]);
        nf_out.push_back(o);
        for (int i = 0; i < 3; ++i) nf_geo.push_back(p->fnormal[size_t(3 * f + i)]);
        nf_geo.push_back(p->farea[size_t(f)]);
    }
    p->n_dir = int(dir_nodes.size());
    p->n_nf = int(nf_out.size());
    p->n_out = int(p->outlets.size());
    // waveforms: inflows first, then outlets
    const int n_wave = int(p->inflows.size() + p->outlets.size());
    std::vector<double> coef;
    for (auto &in : p->inflows) coef.insert(coef.end(), in.coef.begin(), in.coef.end());
    for (auto &o : p->outlets) coef.insert(coef.end(), o.coef.begin(), o.coef.end());
    (void)M;
    HB_TRY(upload(p, p->d_coef, coef));
    HB_TRY(dalloc(p, p->d_W, size_t(std::max(1, n_wave * N))));
    launch_sample_waveforms(p->d_coef.p, n_wave, p->n_h, N, p->T, p->d_W.p, p->stream);
    HB_LAUNCHED(p, n_wave > 0 ? 1 : 0);
    HB_TRY(upload(p, p->d_dir_nodes, dir_nodes));
    HB_TRY(upload(p, p->d_dir_prof, dir_harm));
    HB_TRY(upload(p, p->d_flag, flag));
    HB_TRY(dirichlet_lists(p, p->ps32, flag));
    HB_TRY(dirichlet_lists(p, p->ps32e, flag));
    HB_TRY(dirichlet_lists(p, p->ps64, flag));
    HB_TRY(dalloc(p, p->d_g, size_t(std::max(1, p->n_dir * 3 * N))));
    // Dirichlet values at the instances: synthesis of the series at t_n (Eqs. upgh_def, upghharm)
    launch_harmonics(p->d_dir_prof.p, p->d_g.p, int64_t(p->n_dir) * 3, N, p->n_h, 1, p->T, p->stream);
    HB_LAUNCHED(p, p->n_dir > 0 ? 1 : 0);
    HB_TRY(upload(p, p->d_nf_nodes, nf_nodes));
    HB_TRY(upload(p, p->d_nf_out, nf_out));
    {
        std::vector<int> ptr, list;
        node_slot_lists(nf_nodes, n, ptr, list);
        HB_TRY(upload(p, p->det_fptr, ptr));
        HB_TRY(upload(p, p->det_fslot, list));
        node_slot_lists(nf_out, int64_t(p->outlets.size()), ptr, list);
        HB_TRY(upload(p, p->det_optr, ptr));
        HB_TRY(upload(p, p->det_oface, list));
    }
    HB_TRY(upload(p, p->d_nf_geo64, nf_geo));
    std::vector<float> nf_geo32(nf_geo.begin(), nf_geo.end());
    HB_TRY(upload(p, p->d_nf_geo32, nf_geo32));
    std::vector<double> W(size_t(n_wave * N));
    if (n_wave > 0) {
        HB_CUDA(cudaMemcpyAsync(W.data(), p->d_W.p, W.size() * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
        HB_CUDA(cudaStreamSynchronize(p->stream));
    }
    const int n_in = int(p->inflows.size());
    std::vector<double> hbase(size_t(std::max(1, p->n_out * N)), 0.0), R(size_t(std::max(1, p->n_out)), 0.0);
    p->has_res = false;
    p->level.assign(size_t(N), 0.0);
    for (int o = 0; o < p->n_out; ++o) {
        R[size_t(o)] = p->outlets[size_t(o)].R;
        p->has_res |= (R[size_t(o)] != 0.0);
        for (int t = 0; t < N; ++t) {
            hbase[size_t(o * N + t)] = -W[size_t((n_in + o) * N + t)];
            p->level[size_t(t)] += W[size_t((n_in + o) * N + t)] / p->n_out;
        }
    }
    HB_TRY(upload(p, p->d_hbase64, hbase));
    HB_TRY(upload(p, p->d_R64, R));
    std::vector<float> hb32(hbase.begin(), hbase.end()), R32(R.begin(), R.end());
    HB_TRY(upload(p, p->d_hbase32, hb32));
    HB_TRY(upload(p, p->d_R32, R32));
    HB_TRY(dalloc(p, p->d_Q64, size_t(std::max(1, p->n_out * N))));
    HB_TRY(dalloc(p, p->d_Q32, size_t(std::max(1, p->n_out * N))));
    // characteristic inlet velocity of the CFL rule: largest mean inflow speed over the instances
    std::vector<double> g(size_t(p->n_dir) * 3 * N);
    if (!g.empty()) {
        HB_CUDA(cudaMemcpyAsync(g.data(), p->d_g.p, g.size() * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
        HB_CUDA(cudaStreamSynchronize(p->stream));
    }
    p->u_c = 0;
    for (int k = 0; k < n_in; ++k) {
        const Inflow &in = p->inflows[size_t(k)];
        double A = 0;
        std::vector<double> fl(size_t(N), 0.0);
        for (int64_t f = 0; f < p->n_faces; ++f) {
            if (p->face_tag[size_t(f)] != in.tag) continue;
            const double S = p->farea[size_t(f)];
            A += S;
            for (int b = 0; b < 3; ++b) {
                const int nd = p->faces[size_t(3 * f + b)];
                if (wave[size_t(nd)] != k) continue;
                const int d = dir_index[size_t(nd)];
                for (int t = 0; t < N; ++t) {
                    double un = 0;
                    for (int i = 0; i < 3; ++i) un += g[(size_t(d) * 3 + i) * N + t] * p->fnormal[size_t(3 * f + i)];
                    fl[size_t(t)] += S / 3.0 * std::fabs(un);
                }
            }
        }
        for (int t = 0; t < N; ++t)
            if (A > 0) p->u_c = std::max(p->u_c, fl[size_t(t)] / A);
    }
    HB_CUDA(cudaStreamSynchronize(p->stream));
    p->bc_dirty = false;
    ++p->gen;
    return HB_OK;
}

// ---------------------------------------------------------------------------------------------------
// assembled paper tangent: structure (host, once), assembly at a state, application

hb_status asm_structure(hb_problem *p) {
    hb_problem::Assembled &A = p->as;
    if (A.nnz > 0) return HB_OK;
    const int64_t n = p->n_nodes, E = p->n_tets;
    // rows: each node's neighbours over its elements (itself included), sorted
    std::vector<std::vector<int>> nb(static_cast<size_t>(n));
    for (int64_t e = 0; e < E; ++e)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) nb[size_t(p->tets[size_t(4 * e + a)])].push_back(p->tets[size_t(4 * e + b)]);
    std::vector<int> rowptr(static_cast<size_t>(n + 1), 0), col;
    for (int64_t i = 0; i < n; ++i) {
        std::vector<int> &r = nb[size_t(i)];
        std::sort(r.begin(), r.end());
        r.erase(std::unique(r.begin(), r.end()), r.end());
        col.insert(col.end(), r.begin(), r.end());
        rowptr[size_t(i + 1)] = int(col.size());
    }
    if (col.size() >= size_t(1) << 31) return fail(HB_ERR_INVALID_ARG, "too many node pairs for the assembled operator");
    // elements in Morton order; pair slot of each (a, b)
    std::vector<int> tets(static_cast<size_t>(4 * E)), epos(static_cast<size_t>(16 * E));
    for (int64_t k = 0; k < E; ++k) {
        const int32_t *t = p->tets_morton.data() + 4 * k;
        for (int a = 0; a < 4; ++a) {
            tets[size_t(4 * k + a)] = t[a];
            const int r0 = rowptr[size_t(t[a])], r1 = rowptr[size_t(t[a]) + 1];
            for (int b = 0; b < 4; ++b) {
                const int *f = std::lower_bound(col.data() + r0, col.data() + r1, t[b]);
                epos[size_t(16 * k + 4 * a + b)] = int(f - col.data());
            }
        }
    }
    std::vector<int> dpos(static_cast<size_t>(n));
    for (int64_t i = 0; i < n; ++i)
        dpos[size_t(i)] = int(std::lower_bound(col.data() + rowptr[size_t(i)], col.data() + rowptr[size_t(i + 1)], int(i)) -
                              col.data());
    HB_TRY(upload(p, A.dpos, dpos));
    HB_TRY(upload(p, A.rowptr, rowptr));
    HB_TRY(upload(p, A.col, col));
    A.h_rowptr = rowptr;
    A.h_col = col;
    HB_TRY(upload(p, A.tets, tets));
    HB_TRY(upload(p, A.epos, epos));
    {
        std::vector<int> ptr, list;
        node_slot_lists(tets, n, ptr, list);
        HB_TRY(upload(p, A.det_ptr, ptr));
        HB_TRY(upload(p, A.det_slot, list));
    }
    A.nnz = int64_t(col.size());
    return HB_OK;
}

template <typename T>
struct AsmBufs;
template <>
struct AsmBufs<float> {
    static DBuf<float> &geom(hb_problem::Assembled &A) { return A.geom32; }
    static DBuf<float> &coef(hb_problem::Assembled &A) { return A.coef32; }
    static DBuf<float> &mass(hb_problem::Assembled &A) { return A.mass32; }
    static DBuf<float> &W(hb_problem::Assembled &A) { return A.W32; }
    static bool &ready(hb_problem::Assembled &A) { return A.ready32; }
    static bool &mass_done(hb_problem::Assembled &A) { return A.mass32_done; }
};
template <>
struct AsmBufs<double> {
    static DBuf<double> &geom(hb_problem::Assembled &A) { return A.geom64; }
    static DBuf<double> &coef(hb_problem::Assembled &A) { return A.coef64; }
    static DBuf<double> &mass(hb_problem::Assembled &A) { return A.mass64; }
    static DBuf<double> &W(hb_problem::Assembled &A) { return A.W64; }
    static bool &ready(hb_problem::Assembled &A) { return A.ready64; }
    static bool &mass_done(hb_problem::Assembled &A) { return A.mass64_done; }
};

// Assemble the paper tangent's volume blocks at state y (device, precision T) on stream s.
template <typename T>
hb_status assemble_at(hb_problem *p, const T *y, cudaStream_t s) {
    HB_TRY(prepare_bc(p));
    HB_TRY(asm_structure(p));
    hb_problem::Assembled &A = p->as;
    using B = AsmBufs<T>;
    const int N = p->N;
    if (!B::geom(A).p) {
        HB_TRY(dalloc(p, B::geom(A), size_t(p->n_tets) * kGeomStride));
        launch_geom<T>(p->d_xyz.p, A.tets.p, int(p->n_tets), p->mu / p->rho, B::geom(A).p, s);
        HB_LAUNCHED(p, 1);
    }
    HB_TRY(dalloc(p, B::coef(A), size_t(A.nnz) * 8 * size_t(N)));
    HB_TRY(dalloc(p, B::mass(A), size_t(A.nnz)));
    HB_TRY(dalloc(p, B::W(A), size_t(p->n_nodes) * size_t(w_stride(N, int(sizeof(T))))));
    AsmArgs<T> a;
    a.n_tets = p->n_tets;
    a.N = N;
    a.tets = A.tets.p;
    a.geom = B::geom(A).p;
    a.epos = A.epos.p;
    a.flag = p->d_flag.p;
    a.y = y;
    a.coef = B::coef(A).p;
    a.mass = B::mass(A).p;
    a.rho = T(p->rho);
    a.mu = T(p->mu);
    a.omega2 = T(p->omega2 + tau_dt_term(p));
    if (p->scatter == 0) {          // deterministic: rows in list order
        a.n_nodes = p->n_nodes;
        a.rptr = A.det_ptr.p;
        a.rslot = A.det_slot.p;
    }
    if (!B::mass_done(A)) {
        HB_CUDA(cudaMemsetAsync(a.mass, 0, size_t(A.nnz) * sizeof(T), s));
        launch_assemble_mass<T>(a, s);
        HB_LAUNCHED(p, 1);
        B::mass_done(A) = true;
    }
    HB_CUDA(cudaMemsetAsync(a.coef, 0, size_t(A.nnz) * 8 * size_t(N) * sizeof(T), s));
    launch_assemble<T>(a, s);
    HB_LAUNCHED(p, 1);
    B::ready(A) = true;
    return HB_OK;
}

// ---------------------------------------------------------------------------------------------------
// operators

template <typename T>
struct DetBufs;
template <>
struct DetBufs<float> {
    static DBuf<float> &c(hb_problem *p) { return p->det_c32; }
    static DBuf<float> &t(hb_problem *p) { return p->det_t32; }
    static DBuf<float> &f(hb_problem *p) { return p->det_f32; }
};
template <>
struct DetBufs<double> {
    static DBuf<double> &c(hb_problem *p) { return p->det_c64; }
    static DBuf<double> &t(hb_problem *p) { return p->det_t64; }
    static DBuf<double> &f(hb_problem *p) { return p->det_f64; }
};

// Kernel arguments of the element pass over patch set ps and of the boundary-face kernels, from the
// problem's current settings (one place for every caller: operators, the no-allocation product, batches)
template <typename T>
ElemArgs<T> elem_args(hb_problem *p, PatchSetDev<T> &ps, const T *y, const T *v, T *out, double shift,
                      const double *shift_dev) {
    ElemArgs<T> ea;
    ea.pv = ps.view();
    ea.y = y;
    ea.v = v;
    ea.out = out;
    ea.H = Hmat<T>(p);
    ea.flag = p->d_flag.p;
    ea.N = p->N;
    ea.rho = T(p->rho);
    ea.mu = T(p->mu);
    ea.shift = T(shift);
    ea.shift_dev = shift_dev;
    ea.omega2 = T(p->omega2 + tau_dt_term(p));
    ea.ls_mass = p->ls_mass;
    ea.variant = p->jvp_variant;
    ea.err = p->d_err.p;
    ea.rbvms = p->stab;
    return ea;
}

template <typename T>
FaceArgs<T> face_args(hb_problem *p, const T *y, const T *v, T *out) {
    FaceArgs<T> fa;
    fa.n_faces = p->n_nf;
    fa.fnodes = p->d_nf_nodes.p;
    fa.foutlet = p->d_nf_out.p;
    fa.flag = p->d_flag.p;
    fa.y = y;
    fa.v = v;
    fa.out = out;
    fa.N = p->N;
    fa.rho = T(p->rho);
    fa.beta = T(p->beta);
    if constexpr (sizeof(T) == 4) {
        fa.fgeo = p->d_nf_geo32.p;
        fa.hbase = p->d_hbase32.p;
        fa.R = p->d_R32.p;
        fa.Q = p->d_Q32.p;
    } else {
        fa.fgeo = p->d_nf_geo64.p;
        fa.hbase = p->d_hbase64.p;
        fa.R = p->d_R64.p;
        fa.Q = p->d_Q64.p;
    }
    return fa;
}

template <typename T>
hb_status apply_op(hb_problem *p, int mode, const T *y, const T *v, T *out, double shift, cudaStream_t s,
                   const double *shift_dev = nullptr) {
    HB_TRY(prepare_bc(p));
    const int N = p->N;
    const bool det = p->scatter == 0;      // element and face slots, then one fixed-order gather
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto prof_begin = [&]() -> hb_status {
        if (p->prof_on) {
            if (p->prof_used == p->prof_ev.size()) {
                HB_CUDA(cudaEventCreate(&e0));
                HB_CUDA(cudaEventCreate(&e1));
                p->prof_ev.push_back({e0, e1});
            }
            e0 = p->prof_ev[p->prof_used].first;
            e1 = p->prof_ev[p->prof_used].second;
            ++p->prof_used;
            HB_CUDA(cudaEventRecord(e0, s));
        }
        return HB_OK;
    };
    if (mode == MODE_JVA) {
        // assembled paper tangent: W = shift v + rho H v per node, then the row-wise product (every entry
        // of out written); the boundary terms follow as for the element path
        hb_problem::Assembled &A = p->as;
        using B = AsmBufs<T>;
        if (!B::ready(A)) return fail(HB_ERR_STATE, "no assembled operator in this precision (hb_assemble_dev)");
        const int ws = w_stride(N, int(sizeof(T)));
        launch_spectral_w<T>(v, Hmat<T>(p), p->d_flag.p, B::W(A).p, ws, p->n_nodes, N, T(p->rho), T(shift), shift_dev, s,
                             p->spectral_path, p->d_err.p);
        SpmvArgs<T> sa;
        sa.n_nodes = p->n_nodes;
        sa.N = N;
        sa.w_stride = ws;
        sa.rowptr = A.rowptr.p;
        sa.col = A.col.p;
        sa.coef = B::coef(A).p;
        sa.mass = B::mass(A).p;
        sa.v = v;
        sa.W = B::W(A).p;
        sa.out = out;
        sa.flag = p->d_flag.p;
        HB_TRY(prof_begin());
        launch_spmv<T>(sa, s);
        if (p->prof_on) HB_CUDA(cudaEventRecord(e1, s));
        HB_LAUNCHED(p, 2);
    }
    const int fmode = mode == MODE_JVA ? MODE_JVP : mode;     // boundary terms of the paper tangent
    PatchSetDev<T> &ps = patches<T>(p, fmode);
    if (mode != MODE_JVA && !det) HB_CUDA(cudaMemsetAsync(out, 0, size_t(p->n_nodes) * 4 * N * sizeof(T), s));
    ElemArgs<T> ea = elem_args<T>(p, ps, y, v, out, shift, shift_dev);
    if (det && ps.P > 0 && mode != MODE_JVA) {
        DBuf<T> &cb = DetBufs<T>::c(p);
        HB_TRY(dalloc(p, cb, size_t(p->n_tets) * size_t(det_slot_values(mode)) * size_t(N)));
        ea.cbuf = cb.p;
    }
    if (ps.P > 0 && mode != MODE_JVA) {
        if (mode == MODE_JVP) {
            // spectral pass over the nodes (each once): W = shift v + rho H v, gathered by the patches
            using B = AsmBufs<T>;
            DBuf<T> &W = B::W(p->as);
            const int ws = w_stride(N, int(sizeof(T)));
            HB_TRY(dalloc(p, W, size_t(p->n_nodes) * size_t(ws)));
            launch_spectral_w<T>(v, Hmat<T>(p), p->d_flag.p, W.p, ws, p->n_nodes, N, T(p->rho), T(shift), shift_dev, s,
                                 p->spectral_path, p->d_err.p);
            HB_LAUNCHED(p, 1);
            ea.W = W.p;
        }
        HB_TRY(prof_begin());
        launch_elem<T>(mode, ea, ps.P, s);
        HB_LAUNCHED(p, 1);
        if (p->prof_on) HB_CUDA(cudaEventRecord(e1, s));
    }
    if (mode != MODE_DIAG && p->n_nf > 0) {
        FaceArgs<T> fa = face_args<T>(p, y, v, out);
        if (det) {
            DBuf<T> &fb = DetBufs<T>::f(p);
            HB_TRY(dalloc(p, fb, size_t(p->n_nf) * 9 * size_t(N)));
            fa.fbuf = fb.p;
            fa.optr = p->det_optr.p;
            fa.oface = p->det_oface.p;
        } else if (p->has_res) {
            HB_CUDA(cudaMemsetAsync(fa.Q, 0, size_t(p->n_out) * N * sizeof(T), s));
        }
        launch_faces<T>(fmode, fa, p->has_res, p->n_out, s);
        HB_LAUNCHED(p, p->has_res ? 2 : 1);
    }
    if (det) {
        DetGatherArgs<T> g;
        g.n_nodes = p->n_nodes;
        g.N = N;
        g.flag = p->d_flag.p;
        g.v = v;
        g.H = Hmat<T>(p);
        g.out = out;
        g.eptr = g.eslot = g.fptr = g.fslot = nullptr;
        g.cbuf = g.fbuf = g.tbuf = nullptr;
        g.presc = 0;
        const bool faces = mode != MODE_DIAG && p->n_nf > 0;
        if (faces) {
            g.fptr = p->det_fptr.p;
            g.fslot = p->det_fslot.p;
            g.fbuf = DetBufs<T>::f(p).p;
        }
        if (mode == MODE_JVA) {            // faces only, added to the sparse product
            g.F = 3;
            if (faces) {
                launch_det_gather<T>(g, s);
                HB_LAUNCHED(p, 1);
            }
        } else {
            g.F = det_slot_values(mode) / 4;
            g.presc = mode == MODE_DIAG ? 1 : (mode == MODE_RES || mode == MODE_TRES) ? 0 : 2;
            g.eptr = ps.det_ptr.p;
            g.eslot = ps.det_slot.p;
            g.cbuf = DetBufs<T>::c(p).p;
            if (g.F == 7) {
                DBuf<T> &tb = DetBufs<T>::t(p);
                HB_TRY(dalloc(p, tb, size_t(p->n_nodes) * 3 * size_t(N)));
                g.tbuf = tb.p;
            }
            launch_det_gather<T>(g, s);
            HB_LAUNCHED(p, g.F == 7 ? 2 : 1);
        }
    }
    return HB_OK;
}

// Status word of the pipelined element pass, read back by the synchronising entry points: a bounded wait
// inside the kernel that gave up (1: data of a patch, 2: a free stage, 3: copies in flight at exit) is
// reported as HB_ERR_TIMEOUT once, and the word is cleared.
hb_status dev_err_status(hb_problem *p, int err) {
    if (err == 0) return HB_OK;
    cudaMemsetAsync(p->d_err.p, 0, sizeof(int), p->stream);
    return fail(HB_ERR_TIMEOUT, "a bounded wait of the pipelined element pass gave up (code " + std::to_string(err) + ")");
}

hb_status check_precision(int precision) {
    if (precision != 0 && precision != 1) return fail(HB_ERR_INVALID_ARG, "precision must be 0 (FP64) or 1 (FP32)");
    return HB_OK;
}

// host-buffer wrapper: copies in, converts, applies, converts, copies out
hb_status host_op(hb_problem *p, int mode, const double *y, const double *v, double *out, int precision,
                  double shift) {
    if (!p || !y || !out || ((mode == MODE_JVP || mode == MODE_JVE || mode == MODE_TRES || mode == MODE_JVA) && !v))
        return fail(HB_ERR_INVALID_ARG, "null argument");
    HB_TRY(check_precision(precision));
    const size_t nd = size_t(p->n_nodes) * 4 * p->N;
    HB_CUDA(cudaSetDevice(p->device));
    HB_TRY(dalloc(p, p->w64a, nd));
    HB_TRY(dalloc(p, p->w64b, nd));
    HB_CUDA(cudaMemcpyAsync(p->w64a.p, y, nd * sizeof(double), cudaMemcpyHostToDevice, p->stream));
    const bool jv = (mode == MODE_JVP || mode == MODE_JVE || mode == MODE_TRES || mode == MODE_JVA);   // second operand
    if (precision == 0) {
        double *vd = nullptr;
        if (jv) {
            HB_TRY(dalloc(p, p->kres, nd));
            HB_CUDA(cudaMemcpyAsync(p->kres.p, v, nd * sizeof(double), cudaMemcpyHostToDevice, p->stream));
            vd = p->kres.p;
        }
        if (mode == MODE_JVA) HB_TRY(assemble_at<double>(p, p->w64a.p, p->stream));   // at y, then apply
        HB_TRY(apply_op<double>(p, mode, p->w64a.p, vd, p->w64b.p, shift, p->stream));
    } else {
        HB_TRY(dalloc(p, p->w32a, nd));
        HB_TRY(dalloc(p, p->w32b, nd));
        HB_TRY(dalloc(p, p->w32c, nd));
        launch_convert<double, float>(p->w64a.p, p->w32a.p, int64_t(nd), p->stream);
        HB_LAUNCHED(p, 1);
        if (jv) {
            HB_CUDA(cudaMemcpyAsync(p->w64b.p, v, nd * sizeof(double), cudaMemcpyHostToDevice, p->stream));
            launch_convert<double, float>(p->w64b.p, p->w32c.p, int64_t(nd), p->stream);
            HB_LAUNCHED(p, 1);
        }
        if (mode == MODE_JVA) HB_TRY(assemble_at<float>(p, p->w32a.p, p->stream));     // at y, then apply
        HB_TRY(apply_op<float>(p, mode, p->w32a.p, jv ? p->w32c.p : nullptr, p->w32b.p, shift, p->stream));
        launch_convert<float, double>(p->w32b.p, p->w64b.p, int64_t(nd), p->stream);
        HB_LAUNCHED(p, 1);
    }
    HB_CUDA(cudaMemcpyAsync(out, p->w64b.p, nd * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    int err = 0;
    HB_CUDA(cudaMemcpyAsync(&err, p->d_err.p, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    HB_CUDA(cudaStreamSynchronize(p->stream));
    return dev_err_status(p, err);
}

hb_status dev_op(hb_problem *p, int mode, const void *y, const void *v, void *out, int precision, double shift,
                 void *stream) {
    if (!p || !y || !out || ((mode == MODE_JVP || mode == MODE_JVE || mode == MODE_JVA) && !v))
        return fail(HB_ERR_INVALID_ARG, "null argument");
    HB_TRY(check_precision(precision));
    if (out == y || (v && out == v)) return fail(HB_ERR_INVALID_ARG, "output aliases an input");
    HB_CUDA(cudaSetDevice(p->device));
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : p->stream;
    if (precision == 0)
        return apply_op<double>(p, mode, static_cast<const double *>(y), static_cast<const double *>(v),
                                static_cast<double *>(out), shift, s);
    return apply_op<float>(p, mode, static_cast<const float *>(y), static_cast<const float *>(v),
                           static_cast<float *>(out), shift, s);
}

// ---------------------------------------------------------------------------------------------------
// reductions and the Krylov solver

hb_status dev_norm(hb_problem *p, const double *x, int64_t n, double &out) {
    HB_TRY(dalloc(p, p->small, 512));
    launch_dot(x, x, n, p->scratch.p, p->small.p, p->stream);
    HB_LAUNCHED(p, 2);
    double v = 0;
    int err = 0;
    HB_CUDA(cudaMemcpyAsync(&v, p->small.p, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    HB_CUDA(cudaMemcpyAsync(&err, p->d_err.p, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    HB_CUDA(cudaStreamSynchronize(p->stream));
    out = std::sqrt(v);
    return dev_err_status(p, err);
}

hb_status dev_dot(hb_problem *p, const double *x, const double *y, int64_t n, double &out) {
    HB_TRY(dalloc(p, p->small, 512));
    launch_dot(x, y, n, p->scratch.p, p->small.p, p->stream);
    HB_LAUNCHED(p, 2);
    HB_CUDA(cudaMemcpyAsync(&out, p->small.p, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    HB_CUDA(cudaStreamSynchronize(p->stream));
    return HB_OK;
}

// pseudo shift of an operator application (value, or device word if set)
struct OpCtxShift {
    double shift;
    const double *dev;
};

// ---------------------------------------------------------------------------------------------------
// aggregation multigrid (precond = 2): hierarchy, coarse operators, V-cycle

constexpr int kAmgCoarsest = 400;      // stop coarsening below this many nodes
constexpr int kAmgMaxLevels = 8;
constexpr double kAmgOmega = 0.7;      // damping of the node-block Jacobi smoother
constexpr int kAmgPre = 2, kAmgPost = 2, kAmgCoarseSweeps = 8;

// greedy aggregation of a node graph (CSR with the diagonal): roots whose neighbours are all unassigned
// take them; remaining nodes join a neighbouring aggregate of the first pass; isolated leftovers are alone
int aggregate(const std::vector<int> &rowptr, const std::vector<int> &col, int64_t n, std::vector<int> &agg) {
    agg.assign(size_t(n), -1);
    int nc = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (agg[size_t(i)] != -1) continue;
        bool free = true;
        for (int k = rowptr[size_t(i)]; k < rowptr[size_t(i) + 1] && free; ++k) free = agg[size_t(col[size_t(k)])] == -1;
        if (!free) continue;
        for (int k = rowptr[size_t(i)]; k < rowptr[size_t(i) + 1]; ++k) agg[size_t(col[size_t(k)])] = nc;
        ++nc;
    }
    std::vector<int> tent(agg);
    for (int64_t i = 0; i < n; ++i) {
        if (agg[size_t(i)] != -1) continue;
        for (int k = rowptr[size_t(i)]; k < rowptr[size_t(i) + 1]; ++k)
            if (agg[size_t(col[size_t(k)])] != -1) {
                tent[size_t(i)] = agg[size_t(col[size_t(k)])];
                break;
            }
    }
    for (int64_t i = 0; i < n; ++i) {
        if (tent[size_t(i)] == -1) tent[size_t(i)] = nc++;
    }
    agg.swap(tent);
    return nc;
}

hb_status amg_build(hb_problem *p) {
    if (!p->amg.empty()) return HB_OK;
    hb_problem::Assembled &A = p->as;
    std::vector<int> rowptr = A.h_rowptr, col = A.h_col;
    std::vector<uint8_t> flag(static_cast<size_t>(p->n_nodes));
    HB_CUDA(cudaMemcpy(flag.data(), p->d_flag.p, flag.size(), cudaMemcpyDeviceToHost));
    int64_t n = p->n_nodes;
    std::vector<hb_problem::AmgLevel> lv(1);
    lv[0].n = n;
    lv[0].nnz = A.nnz;
    while (n > kAmgCoarsest && int(lv.size()) < kAmgMaxLevels) {
        std::vector<int> agg;
        const int nc = aggregate(rowptr, col, n, agg);
        if (nc >= n * 9 / 10) break;                         // no useful coarsening left
        // coarse pair structure and the fine pairs of each coarse pair
        std::vector<std::vector<int>> crow(static_cast<size_t>(nc));
        for (int64_t i = 0; i < n; ++i)
            for (int k = rowptr[size_t(i)]; k < rowptr[size_t(i) + 1]; ++k)
                crow[size_t(agg[size_t(i)])].push_back(agg[size_t(col[size_t(k)])]);
        std::vector<int> crp(size_t(nc) + 1, 0), ccol;
        for (int I = 0; I < nc; ++I) {
            std::vector<int> &r = crow[size_t(I)];
            std::sort(r.begin(), r.end());
            r.erase(std::unique(r.begin(), r.end()), r.end());
            ccol.insert(ccol.end(), r.begin(), r.end());
            crp[size_t(I) + 1] = int(ccol.size());
        }
        const int64_t cnnz = int64_t(ccol.size());
        const size_t fnnz = size_t(rowptr[size_t(n)]);
        std::vector<int> owner(fnnz);                           // fine pair -> coarse pair
        std::vector<uint8_t> mmask(owner.size());
        for (int64_t i = 0; i < n; ++i)
            for (int k = rowptr[size_t(i)]; k < rowptr[size_t(i) + 1]; ++k) {
                const int I = agg[size_t(i)], J = agg[size_t(col[size_t(k)])];
                owner[size_t(k)] = int(std::lower_bound(ccol.data() + crp[size_t(I)], ccol.data() + crp[size_t(I) + 1], J) -
                                       ccol.data());
                mmask[size_t(k)] = !(flag[size_t(i)] & 1) && !(flag[size_t(col[size_t(k)])] & 1);
            }
        std::vector<int> cptr(size_t(cnnz) + 1, 0), cidx(owner.size());
        for (int o : owner) ++cptr[size_t(o) + 1];
        for (int64_t q = 0; q < cnnz; ++q) cptr[size_t(q) + 1] += cptr[size_t(q)];
        {
            std::vector<int> fill(cptr.begin(), cptr.end() - 1);
            for (size_t k = 0; k < owner.size(); ++k) cidx[size_t(fill[size_t(owner[k])]++)] = int(k);
        }
        std::vector<int> aptr(size_t(nc) + 1, 0), aidx(static_cast<size_t>(n));
        for (int64_t i = 0; i < n; ++i) ++aptr[size_t(agg[size_t(i)]) + 1];
        for (int I = 0; I < nc; ++I) aptr[size_t(I) + 1] += aptr[size_t(I)];
        {
            std::vector<int> fill(aptr.begin(), aptr.end() - 1);
            for (int64_t i = 0; i < n; ++i) aidx[size_t(fill[size_t(agg[size_t(i)])]++)] = int(i);
        }
        std::vector<uint8_t> cflag(static_cast<size_t>(nc), 1);
        for (int64_t i = 0; i < n; ++i)
            if (!(flag[size_t(i)] & 1)) cflag[size_t(agg[size_t(i)])] = 0;
        std::vector<int> cdpos(static_cast<size_t>(nc));
        for (int I = 0; I < nc; ++I)
            cdpos[size_t(I)] = int(std::lower_bound(ccol.data() + crp[size_t(I)], ccol.data() + crp[size_t(I) + 1], I) -
                                   ccol.data());
        hb_problem::AmgLevel &f = lv.back();
        HB_TRY(upload(p, f.agg, agg));
        HB_TRY(upload(p, f.aptr, aptr));
        HB_TRY(upload(p, f.aidx, aidx));
        HB_TRY(upload(p, f.cptr, cptr));
        HB_TRY(upload(p, f.cidx, cidx));
        HB_TRY(upload(p, f.mmask, mmask));
        hb_problem::AmgLevel c;
        c.n = nc;
        c.nnz = cnnz;
        HB_TRY(upload(p, c.rowptr, crp));
        HB_TRY(upload(p, c.col, ccol));
        HB_TRY(upload(p, c.dpos, cdpos));
        HB_TRY(upload(p, c.flag, cflag));
        lv.push_back(std::move(c));
        rowptr.swap(crp);
        col.swap(ccol);
        flag.swap(cflag);
        n = nc;
    }
    p->amg = std::move(lv);
    return HB_OK;
}

template <typename T>
struct AmgBufs;
template <>
struct AmgBufs<float> {
    static DBuf<float> &coef(hb_problem::AmgLevel &l) { return l.coef32; }
    static DBuf<float> &mass(hb_problem::AmgLevel &l) { return l.mass32; }
    static DBuf<float> &x(hb_problem::AmgLevel &l) { return l.x32; }
    static DBuf<float> &b(hb_problem::AmgLevel &l) { return l.b32; }
    static DBuf<float> &r(hb_problem::AmgLevel &l) { return l.r32; }
    static DBuf<float> &ax(hb_problem::AmgLevel &l) { return l.ax32; }
    static DBuf<float> &W(hb_problem::AmgLevel &l) { return l.W32; }
    static bool &mass_done(hb_problem *p) { return p->amg_mass32; }
};
template <>
struct AmgBufs<double> {
    static DBuf<double> &coef(hb_problem::AmgLevel &l) { return l.coef64; }
    static DBuf<double> &mass(hb_problem::AmgLevel &l) { return l.mass64; }
    static DBuf<double> &x(hb_problem::AmgLevel &l) { return l.x64; }
    static DBuf<double> &b(hb_problem::AmgLevel &l) { return l.b64; }
    static DBuf<double> &r(hb_problem::AmgLevel &l) { return l.r64; }
    static DBuf<double> &ax(hb_problem::AmgLevel &l) { return l.ax64; }
    static DBuf<double> &W(hb_problem::AmgLevel &l) { return l.W64; }
    static bool &mass_done(hb_problem *p) { return p->amg_mass64; }
};

// level operator views (level 0 is the assembled tangent itself)
template <typename T>
struct AmgOp {
    int64_t n, nnz;
    const int *rowptr, *col, *dpos;
    const uint8_t *flag;
    const T *coef, *mass;
};
template <typename T>
AmgOp<T> amg_op(hb_problem *p, size_t l) {
    hb_problem::AmgLevel &L = p->amg[l];
    if (l == 0) {
        hb_problem::Assembled &A = p->as;
        return AmgOp<T>{L.n, L.nnz, A.rowptr.p, A.col.p, A.dpos.p, p->d_flag.p, AsmBufs<T>::coef(A).p,
                        AsmBufs<T>::mass(A).p};
    }
    return AmgOp<T>{L.n, L.nnz, L.rowptr.p, L.col.p, L.dpos.p, L.flag.p, AmgBufs<T>::coef(L).p, AmgBufs<T>::mass(L).p};
}

// coarse operators from the last assembly (after assemble_at<T>); allocates every level's work vectors
template <typename T>
hb_status amg_values(hb_problem *p, cudaStream_t s) {
    HB_TRY(amg_build(p));
    const int N = p->N, ws = w_stride(N, int(sizeof(T)));
    const bool mass = !AmgBufs<T>::mass_done(p);
    for (size_t l = 0; l < p->amg.size(); ++l) {
        hb_problem::AmgLevel &L = p->amg[l];
        const size_t nv = size_t(L.n) * 4 * size_t(N);
        HB_TRY(dalloc(p, AmgBufs<T>::x(L), nv));
        HB_TRY(dalloc(p, AmgBufs<T>::b(L), nv));
        HB_TRY(dalloc(p, AmgBufs<T>::r(L), nv));
        HB_TRY(dalloc(p, AmgBufs<T>::ax(L), nv));
        HB_TRY(dalloc(p, AmgBufs<T>::W(L), size_t(L.n) * size_t(ws)));
        if (l > 0) {
            HB_TRY(dalloc(p, AmgBufs<T>::coef(L), size_t(L.nnz) * 8 * size_t(N)));
            HB_TRY(dalloc(p, AmgBufs<T>::mass(L), size_t(L.nnz)));
        }
    }
    for (size_t l = 0; l + 1 < p->amg.size(); ++l) {
        const AmgOp<T> f = amg_op<T>(p, l);
        hb_problem::AmgLevel &F = p->amg[l], &C = p->amg[l + 1];
        launch_amg_coarse<T>(F.cptr.p, F.cidx.p, F.mmask.p, f.coef, f.mass, AmgBufs<T>::coef(C).p,
                             AmgBufs<T>::mass(C).p, C.nnz, N, mass, s);
        HB_LAUNCHED(p, mass ? 2 : 1);
    }
    AmgBufs<T>::mass_done(p) = true;
    return HB_OK;
}

// ax = A_l x on level l (W = shift x + rho H x per node, then the row-wise sparse product)
template <typename T>
void amg_matvec(hb_problem *p, size_t l, const OpCtxShift &sh, const T *x, T *ax, cudaStream_t s) {
    const AmgOp<T> op = amg_op<T>(p, l);
    hb_problem::AmgLevel &L = p->amg[l];
    const int N = p->N, ws = w_stride(N, int(sizeof(T)));
    launch_spectral_w<T>(x, Hmat<T>(p), op.flag, AmgBufs<T>::W(L).p, ws, op.n, N, T(p->rho), T(sh.shift), sh.dev, s,
                         p->spectral_path, p->d_err.p);
    SpmvArgs<T> a;
    a.n_nodes = op.n;
    a.N = N;
    a.w_stride = ws;
    a.rowptr = op.rowptr;
    a.col = op.col;
    a.coef = op.coef;
    a.mass = op.mass;
    a.v = x;
    a.W = AmgBufs<T>::W(L).p;
    a.out = ax;
    a.flag = op.flag;
    launch_spmv<T>(a, s);
    p->launches += 2;
}

// x_l ~= A_l^-1 b_l by one V-cycle from x_l = 0
template <typename T>
void amg_vcycle(hb_problem *p, size_t l, const OpCtxShift &sh, cudaStream_t s) {
    const AmgOp<T> op = amg_op<T>(p, l);
    hb_problem::AmgLevel &L = p->amg[l];
    const int N = p->N;
    T *x = AmgBufs<T>::x(L).p, *b = AmgBufs<T>::b(L).p, *r = AmgBufs<T>::r(L).p, *ax = AmgBufs<T>::ax(L).p;
    const int64_t nv = op.n * 4 * N;
    auto sweep = [&](bool first) {
        if (first) {
            launch_amg_smooth<T>(op.coef, op.mass, op.dpos, op.flag, b, x, op.n, N, kAmgOmega, sh.shift, sh.dev, 0, s);
            p->launches += 1;
            return;
        }
        amg_matvec<T>(p, l, sh, x, ax, s);
        launch_amg_sub<T>(b, ax, r, nv, s);
        launch_amg_smooth<T>(op.coef, op.mass, op.dpos, op.flag, r, x, op.n, N, kAmgOmega, sh.shift, sh.dev, 1, s);
        p->launches += 2;
    };
    const bool coarsest = l + 1 == p->amg.size();
    const int pre = coarsest ? kAmgCoarseSweeps : kAmgPre;
    for (int k = 0; k < pre; ++k) sweep(k == 0);
    if (coarsest) return;
    amg_matvec<T>(p, l, sh, x, ax, s);
    launch_amg_sub<T>(b, ax, r, nv, s);
    hb_problem::AmgLevel &C = p->amg[l + 1];
    launch_amg_restrict<T>(L.aptr.p, L.aidx.p, op.flag, r, AmgBufs<T>::b(C).p, C.n, N, s);
    p->launches += 2;
    amg_vcycle<T>(p, l + 1, sh, s);
    launch_amg_prolong<T>(L.agg.p, op.flag, AmgBufs<T>::x(C).p, x, op.n, N, s);
    p->launches += 1;
    for (int k = 0; k < kAmgPost; ++k) sweep(false);
}

// z = V-cycle(x): x the FP64 Krylov vector, the cycle in the precision of the assembly T, z in Z
template <typename T, typename Z>
hb_status amg_apply(hb_problem *p, const OpCtxShift &sh, const double *x, Z *z, cudaStream_t s) {
    if (p->amg.empty()) return fail(HB_ERR_STATE, "multigrid preconditioner not set up");
    hb_problem::AmgLevel &L0 = p->amg[0];
    const int64_t nv = L0.n * 4 * p->N;
    launch_convert<double, T>(x, AmgBufs<T>::b(L0).p, nv, s);
    HB_LAUNCHED(p, 1);
    amg_vcycle<T>(p, 0, sh, s);
    if constexpr (std::is_same<T, Z>::value) {
        HB_CUDA(cudaMemcpyAsync(z, AmgBufs<T>::x(L0).p, size_t(nv) * sizeof(T), cudaMemcpyDeviceToDevice, s));
    } else {
        launch_convert<T, Z>(AmgBufs<T>::x(L0).p, z, nv, s);
        HB_LAUNCHED(p, 1);
    }
    return HB_OK;
}

struct OpCtx {
    int mode;
    double shift;
    int precision;
    const double *shift_dev = nullptr;   // pseudo shift read from device memory (graph-stable)
    int precond = 0;                     // 0: Jacobi (inverse diagonal in kdiag); 1: node blocks of the
                                         // assembled tangent; 2: aggregation multigrid V-cycle on it
};

// z = M^-1 x for the preconditioner of c (x: FP64 Krylov vector); Z = float writes the mixed path's
// operand, Z = double the FP64 one
template <typename Z>
hb_status apply_precond(hb_problem *p, const OpCtx &c, const double *x, Z *z, cudaStream_t s) {
    const int64_t nd = p->n_nodes * 4 * p->N;
    if (c.precond == 2) {
        const OpCtxShift sh{c.shift, c.shift_dev};
        if (c.precision == 1) return amg_apply<float, Z>(p, sh, x, z, s);
        if constexpr (sizeof(Z) == 8) return amg_apply<double, double>(p, sh, x, z, s);
        return fail(HB_ERR_STATE, "FP32 preconditioner output requested in the FP64 path");
    }
    if (c.precond == 1) {
        const hb_problem::Assembled &A = p->as;
        if (c.precision == 1) {      // coefficients assembled in FP32
            launch_block_jacobi<float, Z>(A.coef32.p, A.mass32.p, A.dpos.p, p->d_flag.p, x, z, p->n_nodes, p->N, c.shift,
                                          c.shift_dev, s);
        } else if constexpr (sizeof(Z) == 8) {
            launch_block_jacobi<double, double>(A.coef64.p, A.mass64.p, A.dpos.p, p->d_flag.p, x, z, p->n_nodes, p->N,
                                                c.shift, c.shift_dev, s);
        } else {
            return fail(HB_ERR_STATE, "FP32 preconditioner output requested in the FP64 path");
        }
    } else {
        launch_precond<Z>(x, p->kdiag.p, z, nd, s);
    }
    HB_LAUNCHED(p, 1);
    return HB_OK;
}

// w(double) = A z, with z given in double (z64) and, for the mixed path, its float copy made here
hb_status apply_A(hb_problem *p, const OpCtx &c, const double *z64, double *w) {
    const int64_t nd = p->n_nodes * 4 * p->N;
    if (c.precision == 0) return apply_op<double>(p, c.mode, p->y.p, z64, w, c.shift, p->stream, c.shift_dev);
    launch_convert<double, float>(z64, p->kz32.p, nd, p->stream);
    HB_LAUNCHED(p, 1);
    HB_TRY(apply_op<float>(p, c.mode, p->ky32.p, p->kz32.p, p->kw32.p, c.shift, p->stream, c.shift_dev));
    launch_convert<float, double>(p->kw32.p, w, nd, p->stream);
    HB_LAUNCHED(p, 1);
    return HB_OK;
}

// Device-side GMRES bookkeeping layout (doubles): pass-1 and pass-2 Gram-Schmidt coefficients, ||w||^2,
// the rotated Hessenberg matrix R [(m+1) x m], Givens cosines and sines, rotated right-hand side g,
// residual estimates, and three scalars.
struct GmLayout {
    size_t h1, h2, nrm2, R, cs, sn, g, resid, invnorm, invbeta, beta2, total;
};

GmLayout gm_layout(int m) {
    GmLayout L;
    size_t o = 0;
    L.h1 = o; o += size_t(m + 2);
    L.h2 = o; o += size_t(m + 2);
    L.nrm2 = o; o += 1;
    L.R = o; o += size_t(m + 1) * size_t(m);
    L.cs = o; o += size_t(m);
    L.sn = o; o += size_t(m);
    L.g = o; o += size_t(m + 1);
    L.resid = o; o += size_t(m);
    L.invnorm = o; o += 1;
    L.invbeta = o; o += 1;
    L.beta2 = o; o += 1;
    L.total = o;
    return L;
}

// Enqueue the m Arnoldi iterations of one restart cycle (V_0 already normalised): right Jacobi
// preconditioning, A z, classical Gram-Schmidt with a second pass when more than half of ||w||^2 was
// removed, then the Hessenberg / Givens update on the device.  No host synchronisation.
hb_status record_cycle(hb_problem *p, const OpCtx &c, int m) {
    const int64_t nd = p->n_nodes * 4 * p->N;
    const GmLayout L = gm_layout(m);
    double *G = p->gm.p;
    double *V = p->kV.p;
    cudaStream_t s = p->stream;
    for (int j = 0; j < m; ++j) {
        double *vj = V + int64_t(j) * nd;
        double *w = V + int64_t(j + 1) * nd;
        if (c.precision == 1) {
            // mixed path: the preconditioned direction goes straight to the FP32 operator
            HB_TRY(apply_precond<float>(p, c, vj, p->kz32.p, s));
            HB_TRY(apply_op<float>(p, c.mode, p->ky32.p, p->kz32.p, p->kw32.p, c.shift, s, c.shift_dev));
            launch_convert<float, double>(p->kw32.p, w, nd, s);
            HB_LAUNCHED(p, 1);
        } else {
            HB_TRY(apply_precond<double>(p, c, vj, p->kz64.p, s));
            HB_TRY(apply_op<double>(p, c.mode, p->y.p, p->kz64.p, w, c.shift, s, c.shift_dev));
        }
        launch_multidot(V, nd, j + 1, w, nd, p->scratch.p, G + L.h1, s);
        launch_multiaxpy_norm(V, nd, j + 1, G + L.h1, w, nd, p->scratch.p, G + L.nrm2, s);
        launch_reorth_gate(G + L.h1 + (j + 1), G + L.nrm2, p->gate.p, s);
        launch_multidot(V, nd, j + 1, w, nd, p->scratch.p, G + L.h2, s, p->gate.p);
        launch_multiaxpy_norm(V, nd, j + 1, G + L.h2, w, nd, p->scratch.p, G + L.nrm2, s, p->gate.p);
        launch_arnoldi_update(j, m, G + L.h1, G + L.h2, G + L.nrm2, G + L.R, G + L.cs, G + L.sn, G + L.g,
                              G + L.resid, G + L.invnorm, s);
        launch_scale_dev(w, G + L.invnorm, w, nd, s);
        HB_LAUNCHED(p, 11);
    }
    return HB_OK;
}

hb_status cycle_graph(hb_problem *p, const OpCtx &c, int m, hb_problem::CycleGraph *&out) {
    hb_problem::CycleGraph &gc = p->cycle[c.mode == MODE_JVE ? 1 : c.mode == MODE_JVA ? 2 : 0];
    out = &gc;
    const double key = c.shift_dev ? -1.0 : c.shift;
    if (gc.exec && gc.m == m && gc.precision == c.precision && gc.shift == key && gc.precond == c.precond &&
        gc.gen == p->gen)
        return HB_OK;
    if (gc.exec) {
        cudaGraphExecDestroy(gc.exec);
        gc.exec = nullptr;
    }
    const int64_t l0 = p->launches;
    HB_CUDA(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeRelaxed));
    hb_status st = record_cycle(p, c, m);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(p->stream, &graph);
    if (st != HB_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return fail(HB_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&gc.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        gc.exec = nullptr;
        return fail(HB_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    gc.m = m;
    gc.precision = c.precision;
    gc.precond = c.precond;
    gc.shift = key;
    gc.gen = p->gen;
    gc.launches = p->launches - l0;
    p->launches = l0;
    return HB_OK;
}

// Right-preconditioned restarted GMRES(m): FP64 Arnoldi vectors and scalars, operator in the
// precision of c.  Each restart cycle is one CUDA-graph launch of m iterations followed by one host
// synchronisation; the host then picks the first iteration that met the tolerance and forms the update.
hb_status gmres(hb_problem *p, const OpCtx &c, const double *b, double *x, double tol, int m, int maxit,
                int &iters, int &jv_calls, double *relres = nullptr) {
    const int64_t nd = p->n_nodes * 4 * p->N;
    cudaStream_t s = p->stream;
    const GmLayout L = gm_layout(m);
    HB_TRY(dalloc(p, p->gm, L.total));
    HB_TRY(dalloc(p, p->gate, 1));
    double *G = p->gm.p;
    double *V = p->kV.p;
    HB_CUDA(cudaMemsetAsync(x, 0, size_t(nd) * sizeof(double), s));
    double bnorm = 0;
    HB_TRY(dev_norm(p, b, nd, bnorm));
    iters = 0;
    if (bnorm == 0) return HB_OK;
    hb_problem::CycleGraph *gc = nullptr;
    HB_TRY(cycle_graph(p, c, m, gc));
    std::vector<double> resid(static_cast<size_t>(m)), g(static_cast<size_t>(m + 1)), R(static_cast<size_t>((m + 1) * m)), yk(static_cast<size_t>(m));
    bool first = true;
    while (true) {
        if (first) {
            HB_CUDA(cudaMemcpyAsync(p->kres.p, b, size_t(nd) * sizeof(double), cudaMemcpyDeviceToDevice, s));
        } else {
            HB_TRY(apply_A(p, c, x, p->ktmp.p));
            ++jv_calls;
            launch_scale_copy(1.0, b, p->kres.p, nd, s);
            launch_axpy(-1.0, p->ktmp.p, p->kres.p, nd, s);
            HB_LAUNCHED(p, 2);
        }
        launch_dot(p->kres.p, p->kres.p, nd, p->scratch.p, G + L.beta2, s);
        launch_cycle_init(G + L.beta2, m, G + L.g, G + L.invbeta, s);
        launch_scale_dev(p->kres.p, G + L.invbeta, V, nd, s);
        HB_LAUNCHED(p, 4);
        HB_CUDA(cudaGraphLaunch(gc->exec, s));
        p->launches += gc->launches;
        jv_calls += m;
        HB_CUDA(cudaMemcpyAsync(resid.data(), G + L.resid, size_t(m) * sizeof(double), cudaMemcpyDeviceToHost, s));
        HB_CUDA(cudaMemcpyAsync(g.data(), G + L.g, size_t(m + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
        HB_CUDA(cudaMemcpyAsync(R.data(), G + L.R, R.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        HB_CUDA(cudaStreamSynchronize(s));
        int k = m;
        for (int j = 0; j < m; ++j) {
            if (!std::isfinite(resid[size_t(j)])) return fail(HB_ERR_NAN, "non-finite value in GMRES");
            if (resid[size_t(j)] <= tol * bnorm) {
                k = j + 1;
                break;
            }
        }
        k = std::max(1, std::min(k, maxit - iters));
        for (int i = k - 1; i >= 0; --i) {
            double acc = g[size_t(i)];
            for (int l = i + 1; l < k; ++l) acc -= R[size_t(i) * m + l] * yk[size_t(l)];
            const double d = R[size_t(i) * m + i];
            yk[size_t(i)] = d != 0 ? acc / d : 0.0;
        }
        HB_CUDA(cudaMemcpyAsync(p->kh.p, yk.data(), size_t(k) * sizeof(double), cudaMemcpyHostToDevice, s));
        launch_combine(V, nd, k, p->kh.p, p->ktmp.p, nd, s);
        HB_TRY(apply_precond<double>(p, c, p->ktmp.p, p->kz64.p, s));
        launch_axpy(1.0, p->kz64.p, x, nd, s);
        HB_LAUNCHED(p, 2);
        HB_CUDA(cudaStreamSynchronize(s));   // yk consumed
        iters += k;
        if (relres) *relres = resid[size_t(k - 1)] / bnorm;
        if (resid[size_t(k - 1)] <= tol * bnorm || iters >= maxit) break;
        first = false;
    }
    return HB_OK;
}

hb_status ensure_krylov(hb_problem *p, int m) {
    const size_t nd = size_t(p->n_nodes) * 4 * p->N;
    if (p->km < m) {
        p->kV.release();
        HB_TRY(dalloc(p, p->kV, nd * size_t(m + 1)));
        p->km = m;
    }
    HB_TRY(dalloc(p, p->kz64, nd));
    HB_TRY(dalloc(p, p->kdx, nd));
    HB_TRY(dalloc(p, p->kdiag, nd));
    HB_TRY(dalloc(p, p->kres, nd));
    HB_TRY(dalloc(p, p->ktmp, nd));
    HB_TRY(dalloc(p, p->kh, size_t(2 * (m + 2) + 8)));   // combination coefficients
    HB_TRY(dalloc(p, p->kz32, nd));
    HB_TRY(dalloc(p, p->kw32, nd));
    HB_TRY(dalloc(p, p->ky32, nd));
    HB_TRY(dalloc(p, p->kdiag32, nd));
    HB_TRY(dalloc(p, p->w64a, nd));
    HB_TRY(dalloc(p, p->w64b, nd));
    // spectral pass output of the paper-tangent operator, allocated here so that no allocation falls
    // inside the captured GMRES cycles
    HB_TRY(dalloc(p, p->as.W32, size_t(p->n_nodes) * size_t(w_stride(p->N, 4))));
    HB_TRY(dalloc(p, p->as.W64, size_t(p->n_nodes) * size_t(w_stride(p->N, 8))));
    return HB_OK;
}

hb_status default_initial(hb_problem *p) {
    const int N = p->N;
    std::vector<double> y(size_t(p->n_nodes) * 4 * N, 0.0);
    for (int64_t a = 0; a < p->n_nodes; ++a)
        for (int t = 0; t < N; ++t) y[size_t((a * 4 + 3) * N + t)] = p->level[size_t(t)];
    HB_TRY(upload(p, p->y, y));
    HB_CUDA(cudaStreamSynchronize(p->stream));
    p->y_set = true;
    return HB_OK;
}

hb_status apply_dirichlet_state(hb_problem *p) {
    launch_apply_dirichlet(p->d_dir_nodes.p, p->n_dir, p->d_g.p, p->y.p, p->N, p->stream);
    HB_LAUNCHED(p, p->n_dir > 0 ? 1 : 0);
    return HB_OK;
}

double h_char(const hb_problem *p) { return std::cbrt(6.0 * std::sqrt(2.0) * p->vol_mean); }

}  // namespace

// ---------------------------------------------------------------------------------------------------
// Jacobian-vector product without any device allocation (hb_jv_dev_noalloc)
//
// The only scratch of the Jv pass is the per-outlet flux Q [n_out][N] of the resistance outlets.  Here
// it lives in this file-scope array, which every GPU that loads the library holds until the process
// exits.  Host code may not use the array's name as a device address (on the host it is a stand-in
// symbol), so its device address is looked up once per device with cudaGetSymbolAddress.

constexpr int kNoAllocScratch = 4096;   // doubles: n_out x N must not exceed this
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratch];
constexpr int kMaxDevices = 64;
static std::atomic<void *> g_noalloc_ptr[kMaxDevices];   // per device; set once, guarded by g_noalloc_mutex
static std::mutex g_noalloc_mutex;

hb_status noalloc_scratch(int device, void **ptr) {
    if (device < 0 || device >= kMaxDevices) return fail(HB_ERR_INVALID_ARG, "device index too large for the no-alloc scratch table");
    void *have = g_noalloc_ptr[device].load(std::memory_order_acquire);
    if (!have) {   // first call on this device, which is current here; host threads serialise the lookup
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        have = g_noalloc_ptr[device].load(std::memory_order_relaxed);
        if (!have) {
            void *q = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&q, g_noalloc_scratch);
            if (e != cudaSuccess || !q) {
                cudaGetLastError();
                return fail(HB_ERR_CUDA, std::string("cudaGetSymbolAddress(no-alloc scratch): ") + cudaGetErrorString(e));
            }
            g_noalloc_ptr[device].store(q, std::memory_order_release);
            have = q;
        }
    }
    *ptr = have;
    return HB_OK;
}

template <typename T>
hb_status apply_jv_noalloc(hb_problem *p, int mode, const T *y, const T *v, T *out, double shift, cudaStream_t s,
                           T *qscratch) {
    PatchSetDev<T> &ps = patches<T>(p, mode);
    HB_CUDA(cudaMemsetAsync(out, 0, size_t(p->n_nodes) * 4 * p->N * sizeof(T), s));
    // no W rows (the in-patch H product) and no device-side shift: the same arguments as every other pass
    const ElemArgs<T> ea = elem_args<T>(p, ps, y, v, out, shift, nullptr);
    if (ps.P > 0) {
        launch_elem<T>(mode, ea, ps.P, s);
        HB_LAUNCHED(p, 1);
    }
    if (p->n_nf > 0) {
        FaceArgs<T> fa = face_args<T>(p, y, v, out);
        fa.Q = qscratch;   // the shared array keeps the last call's values: clear it first
        if (p->has_res) HB_CUDA(cudaMemsetAsync(qscratch, 0, size_t(p->n_out) * p->N * sizeof(T), s));
        launch_faces<T>(mode, fa, p->has_res, p->n_out, s);
        HB_LAUNCHED(p, p->has_res ? 2 : 1);
    }
    return HB_OK;
}

namespace hb {

hb_status set_error(hb_status st, const std::string &msg) { return fail(st, msg); }

uint64_t problem_uid(const hb_problem *p) { return p ? p->uid : 0; }

hb_status learned_inputs(hb_problem *p, LearnedInputs &in) {
    if (!p) return fail(HB_ERR_INVALID_ARG, "null problem");
    HB_CUDA(cudaSetDevice(p->device));
    HB_TRY(prepare_bc(p));
    if (p->inflows.empty()) return fail(HB_ERR_STATE, "the learned warm start needs an inflow");
    in.n_nodes = p->n_nodes;
    in.n_tets = p->n_tets;
    in.n_h = p->n_h;
    in.xyz = p->xyz;
    in.tets = p->tets;
    in.flags.assign(size_t(p->n_nodes), 0);
    for (int64_t a = 0; a < p->n_nodes; ++a) {
        const int w = p->h_wave[size_t(a)];
        if (w == -1) in.flags[size_t(a)] |= 1;
        if (w >= 0) in.flags[size_t(a)] |= 2;
    }
    for (int64_t f = 0; f < p->n_faces; ++f) {
        const int tag = p->face_tag[size_t(f)];
        bool is_in = false;
        for (auto &x : p->inflows) is_in |= (x.tag == tag);
        if (tag != 0 && !is_in)
            for (int b = 0; b < 3; ++b) in.flags[size_t(p->faces[size_t(3 * f + b)])] |= 4;
    }
    in.profile.assign(size_t(3 * p->n_nodes), 0.0);   // the inflow profile on inflow (non-wall) nodes
    for (int64_t a = 0; a < p->n_nodes; ++a)
        if (p->h_wave[size_t(a)] >= 0)
            for (int i = 0; i < 3; ++i) in.profile[size_t(3 * a + i)] = p->h_prof[size_t(3 * a + i)];
    in.wave = p->inflows[0].coef;
    in.u_ref = p->u_c > 0 ? p->u_c : 1.0;
    double pr = 0;
    for (double v : p->level) pr += v / double(p->level.size());
    in.p_ref = pr;
    in.rho = p->rho;
    return HB_OK;
}

hb_status learned_set_initial(hb_problem *p, const double *harmonics_host) {
    return hb_set_initial(p, harmonics_host);
}

// Host checks of a mesh that need no device: finite coordinates, node indices in range, face tags >= 0,
// no tetrahedron of (relative) zero volume.  Inverted orientation is allowed: the geometry uses |det J|.
hb_status validate_mesh(const hb_mesh *m) {
    const int64_t n = m->n_nodes;
    for (int64_t k = 0; k < 3 * n; ++k)
        if (!std::isfinite(m->xyz[k])) return fail(HB_ERR_MESH, "non-finite node coordinate");
    for (int64_t k = 0; k < 4 * m->n_tets; ++k)
        if (m->tets[k] < 0 || m->tets[k] >= n) return fail(HB_ERR_MESH, "tetrahedron node index out of range");
    for (int64_t k = 0; k < 3 * m->n_faces; ++k)
        if (m->faces[k] < 0 || m->faces[k] >= n) return fail(HB_ERR_MESH, "face node index out of range");
    for (int64_t k = 0; k < m->n_faces; ++k)
        if (m->face_tag[k] < 0) return fail(HB_ERR_MESH, "negative face tag");
    double vsum = 0, vmin = 1e300;
    for (int64_t e = 0; e < m->n_tets; ++e) {
        const int32_t *t = m->tets + 4 * e;
        const double *x0 = m->xyz + 3 * t[0], *x1 = m->xyz + 3 * t[1], *x2 = m->xyz + 3 * t[2],
                     *x3 = m->xyz + 3 * t[3];
        double u[3], v[3], w[3];
        for (int i = 0; i < 3; ++i) {
            u[i] = x1[i] - x0[i];
            v[i] = x2[i] - x0[i];
            w[i] = x3[i] - x0[i];
        }
        const double vol = std::fabs(u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0]) +
                                     u[2] * (v[0] * w[1] - v[1] * w[0])) / 6.0;
        vsum += vol;
        vmin = std::min(vmin, vol);
    }
    if (!(vmin > 1e-14 * (vsum / double(m->n_tets)))) return fail(HB_ERR_MESH, "degenerate tetrahedron (zero volume)");
    return HB_OK;
}

}  // namespace hb

// =====================================================================================================
// C ABI

extern "C" {

const char *hb_last_error(void) { return g_err.c_str(); }

hb_status hb_create(const hb_mesh *mesh, double rho, double mu, double period_T, int n_h, int device,
                    void *cuda_stream, hb_problem **out) {
    if (!mesh || !out || !mesh->xyz || !mesh->tets || (mesh->n_faces > 0 && (!mesh->faces || !mesh->face_tag)))
        return fail(HB_ERR_INVALID_ARG, "null mesh array");
    *out = nullptr;
    if (mesh->n_nodes <= 0 || mesh->n_tets <= 0 || mesh->n_faces < 0)
        return fail(HB_ERR_INVALID_ARG, "empty mesh");
    if (mesh->n_nodes >= (int64_t(1) << 21) || mesh->n_tets >= (int64_t(1) << 31) / 4)
        return fail(HB_ERR_INVALID_ARG, "mesh too large (n_nodes must be < 2^21)");
    if (!(rho > 0) || !(mu > 0) || !(period_T > 0)) return fail(HB_ERR_INVALID_ARG, "rho, mu and T must be > 0");
    if (n_h < 0 || 2 * n_h + 1 > kMaxN) return fail(HB_ERR_INVALID_ARG, "n_h must be in [0, 15]");
    HB_TRY(validate_mesh(mesh));
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return fail(HB_ERR_CUDA, "no such CUDA device");
    }
    hb_problem *p = new hb_problem();
    static std::atomic<uint64_t> next_uid{1};
    p->uid = next_uid++;
    auto bail = [&](hb_status st) {
        delete p;
        return st;
    };
    p->device = device;
    if (cudaSetDevice(device) != cudaSuccess) return bail(fail(HB_ERR_CUDA, "cudaSetDevice failed"));
    cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (cuda_stream) {
        p->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(fail(HB_ERR_CUDA, "cudaStreamCreate failed"));
        p->own_stream = true;
    }
    p->n_nodes = mesh->n_nodes;
    p->n_tets = mesh->n_tets;
    p->n_faces = mesh->n_faces;
    p->n_h = n_h;
    p->N = 2 * n_h + 1;
    p->rho = rho;
    p->mu = mu;
    p->T = period_T;
    p->omega = 2.0 * M_PI / period_T;
    p->xyz.assign(mesh->xyz, mesh->xyz + 3 * mesh->n_nodes);
    p->tets.assign(mesh->tets, mesh->tets + 4 * mesh->n_tets);
    if (mesh->n_faces > 0) {
        p->faces.assign(mesh->faces, mesh->faces + 3 * mesh->n_faces);
        p->face_tag.assign(mesh->face_tag, mesh->face_tag + mesh->n_faces);
    }
    for (int32_t v : p->tets)
        if (v < 0 || v >= mesh->n_nodes) return bail(fail(HB_ERR_MESH, "tetrahedron node index out of range"));
    for (int32_t v : p->faces)
        if (v < 0 || v >= mesh->n_nodes) return bail(fail(HB_ERR_MESH, "face node index out of range"));
    for (int32_t t : p->face_tag)
        if (t < 0) return bail(fail(HB_ERR_MESH, "negative face tag"));
    // volumes and Morton keys of the centroids
    const int64_t E = p->n_tets;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t a = 0; a < p->n_nodes; ++a)
        for (int i = 0; i < 3; ++i) {
            lo[i] = std::min(lo[i], p->xyz[size_t(3 * a + i)]);
            hi[i] = std::max(hi[i], p->xyz[size_t(3 * a + i)]);
        }
    std::vector<std::pair<uint64_t, int>> keys(static_cast<size_t>(E));
    double vsum = 0, vmin = 1e300;
    for (int64_t e = 0; e < E; ++e) {
        const int32_t *t = &p->tets[size_t(4 * e)];
        double x[4][3], c[3] = {0, 0, 0};
        for (int a = 0; a < 4; ++a)
            for (int i = 0; i < 3; ++i) {
                x[a][i] = p->xyz[size_t(3 * t[a] + i)];
                c[i] += 0.25 * x[a][i];
            }
        double u[3], v[3], w[3];
        for (int i = 0; i < 3; ++i) {
            u[i] = x[1][i] - x[0][i];
            v[i] = x[2][i] - x[0][i];
            w[i] = x[3][i] - x[0][i];
        }
        const double det = u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0]) +
                           u[2] * (v[0] * w[1] - v[1] * w[0]);
        const double vol = std::fabs(det) / 6.0;
        vsum += vol;
        vmin = std::min(vmin, vol);
        uint64_t code = 0;
        for (int i = 0; i < 3; ++i) {
            const double span = hi[i] - lo[i] > 0 ? hi[i] - lo[i] : 1.0;
            const uint64_t q = uint64_t(std::min(2097151.0, std::max(0.0, (c[i] - lo[i]) / span * 2097151.0)));
            code |= spread3(q) << i;
        }
        keys[size_t(e)] = {code, int(e)};
    }
    p->vol_mean = vsum / double(E);
    p->vol_min = vmin;
    if (!(vmin > 1e-14 * p->vol_mean))
        return bail(fail(HB_ERR_MESH, "degenerate tetrahedron (zero volume)"));
    std::sort(keys.begin(), keys.end());
    std::vector<int32_t> &tets_ord = p->tets_morton;
    tets_ord.assign(size_t(4 * E), 0);
    for (int64_t e = 0; e < E; ++e)
        for (int a = 0; a < 4; ++a) tets_ord[size_t(4 * e + a)] = p->tets[size_t(4 * keys[size_t(e)].second + a)];
    // boundary faces: outward normal away from the owning tetrahedron's opposite vertex, and area
    {
        static const int loc[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
        std::vector<std::pair<uint64_t, int64_t>> tf(static_cast<size_t>(4 * E));
        for (int64_t e = 0; e < E; ++e)
            for (int l = 0; l < 4; ++l) {
                uint64_t s[3];
                for (int b = 0; b < 3; ++b) s[b] = uint64_t(p->tets[size_t(4 * e + loc[l][b])]);
                std::sort(s, s + 3);
                tf[size_t(4 * e + l)] = {(s[0] << 42) | (s[1] << 21) | s[2], 4 * e + l};
            }
        std::sort(tf.begin(), tf.end());
        p->fnormal.assign(size_t(3 * p->n_faces), 0.0);
        p->farea.assign(size_t(p->n_faces), 0.0);
        for (int64_t f = 0; f < p->n_faces; ++f) {
            uint64_t s[3];
            for (int b = 0; b < 3; ++b) s[b] = uint64_t(p->faces[size_t(3 * f + b)]);
            std::sort(s, s + 3);
            const uint64_t key = (s[0] << 42) | (s[1] << 21) | s[2];
            auto it = std::lower_bound(tf.begin(), tf.end(), std::make_pair(key, int64_t(-1)));
            if (it == tf.end() || it->first != key) return bail(fail(HB_ERR_MESH, "boundary face is not a tetrahedron face"));
            const int64_t e = it->second / 4, l = it->second % 4;
            const int opp = p->tets[size_t(4 * e + l)];
            const int32_t *fn = &p->faces[size_t(3 * f)];
            double a[3], b[3], cr[3], away = 0;
            for (int i = 0; i < 3; ++i) {
                a[i] = p->xyz[size_t(3 * fn[1] + i)] - p->xyz[size_t(3 * fn[0] + i)];
                b[i] = p->xyz[size_t(3 * fn[2] + i)] - p->xyz[size_t(3 * fn[0] + i)];
            }
            cr[0] = a[1] * b[2] - a[2] * b[1];
            cr[1] = a[2] * b[0] - a[0] * b[2];
            cr[2] = a[0] * b[1] - a[1] * b[0];
            const double nn = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
            if (!(nn > 0)) return bail(fail(HB_ERR_MESH, "degenerate boundary face"));
            for (int i = 0; i < 3; ++i) {
                const double m = (p->xyz[size_t(3 * fn[0] + i)] + p->xyz[size_t(3 * fn[1] + i)] +
                                  p->xyz[size_t(3 * fn[2] + i)]) / 3.0;
                away += cr[i] * (m - p->xyz[size_t(3 * opp + i)]);
            }
            const double sgn = away >= 0 ? 1.0 : -1.0;
            for (int i = 0; i < 3; ++i) p->fnormal[size_t(3 * f + i)] = sgn * cr[i] / nn;
            p->farea[size_t(f)] = 0.5 * nn;
        }
    }
    hb_status st;
    if ((st = upload(p, p->d_xyz, p->xyz)) != HB_OK) return bail(st);
    if ((st = make_patchset<float>(p, p->ps32, tets_ord, 112 * 1024, 0, MODE_JVP)) != HB_OK) return bail(st);
    if ((st = make_patchset<float>(p, p->ps32e, tets_ord, 112 * 1024, 0, MODE_JVE)) != HB_OK) return bail(st);
    if ((st = make_patchset<double>(p, p->ps64, tets_ord, 200 * 1024, 0, MODE_JVE)) != HB_OK) return bail(st);
    // H = E^-1 Omega E in real closed form: (w/2) (-1)^(j-k) / sin(pi (j-k) / N), zero diagonal
    {
        const int N = p->N;
        std::vector<double> H(size_t(N * N), 0.0);
        for (int j = 0; j < N; ++j)
            for (int k = 0; k < N; ++k)
                if (j != k) {
                    const int d = j - k;
                    H[size_t(j * N + k)] = 0.5 * p->omega * ((d % 2 == 0) ? 1.0 : -1.0) / std::sin(M_PI * double(d) / N);
                }
        if ((st = upload(p, p->H64, H)) != HB_OK) return bail(st);
        if ((st = upload(p, p->H32, std::vector<float>(H.begin(), H.end()))) != HB_OK) return bail(st);
    }
    if ((st = dalloc(p, p->scratch, 300000)) != HB_OK) return bail(st);
    if ((st = dalloc(p, p->small, 512)) != HB_OK) return bail(st);
    if ((st = dalloc(p, p->d_err, 1)) != HB_OK) return bail(st);
    if (cudaMemsetAsync(p->d_err.p, 0, sizeof(int), p->stream) != cudaSuccess)
        return bail(fail(HB_ERR_CUDA, "set-up failed"));
    if ((st = dalloc(p, p->y, size_t(p->n_nodes) * 4 * p->N)) != HB_OK) return bail(st);
    if (cudaStreamSynchronize(p->stream) != cudaSuccess) return bail(fail(HB_ERR_CUDA, "set-up failed"));
    *out = p;
    return HB_OK;
}

hb_status hb_destroy(hb_problem *p) {
    if (!p) return HB_OK;
    if (p->tm) hb_destroy(p->tm);
    cudaSetDevice(p->device);
    if (p->stream) cudaStreamSynchronize(p->stream);
    const bool own = p->own_stream;
    cudaStream_t s = p->stream;
    for (auto &ev : p->prof_ev) {
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
    }
    for (auto &gc : p->cycle)
        if (gc.exec) cudaGraphExecDestroy(gc.exec);
    delete p;
    if (own) cudaStreamDestroy(s);
    return HB_OK;
}

static hb_status check_tag(hb_problem *p, int tag) {
    if (!p) return fail(HB_ERR_INVALID_ARG, "null problem");
    if (tag <= 0) return fail(HB_ERR_INVALID_ARG, "tag must be > 0 (tag 0 is the wall)");
    for (int32_t t : p->face_tag)
        if (t == tag) return HB_OK;
    return fail(HB_ERR_INVALID_ARG, "no boundary face carries tag " + std::to_string(tag));
}

hb_status hb_set_inflow(hb_problem *p, int tag, const double *profile, const double *a, const double *b) {
    HB_TRY(check_tag(p, tag));
    if (!a || !b) return fail(HB_ERR_INVALID_ARG, "null waveform");
    Inflow in;
    in.tag = tag;
    if (profile) in.profile.assign(profile, profile + 3 * p->n_nodes);
    in.coef = real_series(a, b, p->n_h);
    for (auto &o : p->outlets)
        if (o.tag == tag) return fail(HB_ERR_INVALID_ARG, "tag already set as an outlet");
    for (auto &x : p->inflows)
        if (x.tag == tag) {
            x = in;
            p->bc_dirty = true;
            return HB_OK;
        }
    p->inflows.push_back(in);
    p->bc_dirty = true;
    return HB_OK;
}

hb_status hb_set_inflow_harmonics(hb_problem *p, int tag, const double *harmonics) {
    HB_TRY(check_tag(p, tag));
    if (!harmonics) return fail(HB_ERR_INVALID_ARG, "null harmonics");
    for (auto &o : p->outlets)
        if (o.tag == tag) return fail(HB_ERR_INVALID_ARG, "tag already set as an outlet");
    const int M = 2 * p->n_h + 1;
    Inflow in;
    in.tag = tag;
    in.harm.assign(harmonics, harmonics + size_t(p->n_nodes) * 3 * M);
    in.coef.assign(size_t(M), 0.0);
    in.coef[0] = 1.0;
    for (auto &x : p->inflows)
        if (x.tag == tag) {
            x = in;
            p->bc_dirty = true;
            return HB_OK;
        }
    p->inflows.push_back(in);
    p->bc_dirty = true;
    return HB_OK;
}

static hb_status set_outlet(hb_problem *p, int tag, double R, const double *a, const double *b) {
    HB_TRY(check_tag(p, tag));
    if (!a || !b) return fail(HB_ERR_INVALID_ARG, "null waveform");
    if (!(R >= 0) || !std::isfinite(R)) return fail(HB_ERR_INVALID_ARG, "resistance must be finite and >= 0");
    for (auto &in : p->inflows)
        if (in.tag == tag) return fail(HB_ERR_INVALID_ARG, "tag already set as an inflow");
    Outlet o{tag, R, real_series(a, b, p->n_h)};
    for (auto &x : p->outlets)
        if (x.tag == tag) {
            x = o;
            p->bc_dirty = true;
            return HB_OK;
        }
    p->outlets.push_back(o);
    p->bc_dirty = true;
    return HB_OK;
}

hb_status hb_set_outlet_pressure(hb_problem *p, int tag, const double *a, const double *b) {
    return set_outlet(p, tag, 0.0, a, b);
}

hb_status hb_set_outlet_resistance(hb_problem *p, int tag, double R, const double *a, const double *b) {
    return set_outlet(p, tag, R, a, b);
}

hb_status hb_set_backflow(hb_problem *p, double beta) {
    if (!p) return fail(HB_ERR_INVALID_ARG, "null problem");
    if (!(beta >= 0 && beta <= 1)) return fail(HB_ERR_INVALID_ARG, "beta must be in [0, 1]");
    p->beta = beta;
    ++p->gen;                                     // face kernels take beta by value
    return HB_OK;
}

hb_status hb_set_instances(hb_problem *p, const double *y) {
    if (!p) return fail(HB_ERR_INVALID_ARG, "null problem");
    HB_CUDA(cudaSetDevice(p->device));
    HB_TRY(prepare_bc(p));
    if (!y) {
        HB_TRY(default_initial(p));
    } else {
        const size_t nd = size_t(p->n_nodes) * 4 * p->N;
        HB_CUDA(cudaMemcpyAsync(p->y.p, y, nd * sizeof(double), cudaMemcpyHostToDevice, p->stream));
        p->y_set = true;
    }
    HB_TRY(apply_dirichlet_state(p));
    HB_CUDA(cudaStreamSynchronize(p->stream));
    return HB_OK;
}

hb_status hb_set_initial(hb_problem *p, const double *harm) {
    if (!p) return fail(HB_ERR_INVALID_ARG, "null problem");
    if (!harm) return hb_set_instances(p, nullptr);
    HB_CUDA(cudaSetDevice(p->device));
    HB_TRY(prepare_bc(p));
    const int M = 2 * p->n_h + 1;
    const size_t nc = size_t(p->n_nodes) * 4 * M;
    HB_TRY(dalloc(p, p->w64a, std::max(nc, size_t(p->n_nodes) * 4 * p->N)));
    HB_CUDA(cudaMemcpyAsync(p->w64a.p, harm, nc * sizeof(double), cudaMemcpyHostToDevice, p->stream));
    launch_harmonics(p->w64a.p, p->y.p, p->n_nodes * 4, p->N, p->n_h, 1, p->T, p->stream);
    HB_LAUNCHED(p, 1);
    p->y_set = true;
    HB_TRY(apply_dirichlet_state(p));
    HB_CUDA(cudaStreamSynchronize(p->stream));
    return HB_OK;
}

hb_status hb_get_instances(hb_problem *p, double *out) {
    if (!p || !out) return fail(HB_ERR_INVALID_ARG, "null argument");
    if (!p->y_set) return fail(HB_ERR_STATE, "no state yet (set an initial state or solve first)");
    HB_CUDA(cudaSetDevice(p->device));
    const size_t nd = size_t(p->n_nodes) * 4 * p->N;
    HB_CUDA(cudaMemcpyAsync(out, p->y.p, nd * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    HB_CUDA(cudaStreamSynchronize(p->stream));
    return HB_OK;
}

hb_status hb_get_harmonics(hb_problem *p, double *out) {
    if (!p || !out) return fail(HB_ERR_INVALID_ARG, "null argument");
    if (!p->y_set) return fail(HB_ERR_STATE, "no state yet (set an initial state or solve first)");
    HB_CUDA(cudaSetDevice(p->device));
    const int M = 2 * p->n_h + 1;
    const size_t nc = size_t(p->n_nodes) * 4 * M;
    HB_TRY(dalloc(p, p->w64b, std::max(nc, size_t(p->n_nodes) * 4 * p->N)));
    launch_harmonics(p->y.p, p->w64b.p, p->n_nodes * 4, p->N, p->n_h, 0, p->T, p->stream);
    HB_LAUNCHED(p, 1);
    HB_CUDA(cudaMemcpyAsync(out, p->w64b.p, nc * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    HB_CUDA(cudaStreamSynchronize(p->stream));
    return HB_OK;
}

hb_status hb_residual(hb_problem *p, const double *y, double *r, int precision) {
    return host_op(p, MODE_RES, y, nullptr, r, precision, 0.0);
}

static int jv_mode(int kind) { return kind == 0 ? MODE_JVP : kind == 1 ? MODE_JVE : MODE_JVA; }

hb_status hb_jv(hb_problem *p, const double *y, const double *v, double *jv, int kind, int precision, double shift) {
    if (kind < 0 || kind > 2)
        return fail(HB_ERR_INVALID_ARG, "kind must be 0 (paper tangent), 1 (exact) or 2 (assembled paper tangent)");
    return host_op(p, jv_mode(kind), y, v, jv, precision, shift);
}

hb_status hb_jv_f32(hb_problem *p, const float *y, const float *v, float *jv, int kind, double shift) {
    if (!p || !y || !v || !jv) return fail(HB_ERR_INVALID_ARG, "null argument");
    if (kind < 0 || kind > 2)
        return fail(HB_ERR_INVALID_ARG, "kind must be 0 (paper tangent), 1 (exact) or 2 (assembled paper tangent)");
    const int mode = jv_mode(kind);
    const size_t nd = size_t(p->n_nodes) * 4 * p->N;
    HB_CUDA(cudaSetDevice(p->device));
    HB_TRY(dalloc(p, p->w32a, nd));
    HB_TRY(dalloc(p, p->w32b, nd));
    HB_TRY(dalloc(p, p->w32c, nd));
    HB_CUDA(cudaMemcpyAsync(p->w32a.p, y, nd * sizeof(float), cudaMemcpyHostToDevice, p->stream));
    HB_CUDA(cudaMemcpyAsync(p->w32c.p, v, nd * sizeof(float), cudaMemcpyHostToDevice, p->stream));
    if (mode == MODE_JVA) HB_TRY(assemble_at<float>(p, p->w32a.p, p->stream));
    HB_TRY(apply_op<float>(p, mode, p->w32a.p, p->w32c.p, p->w32b.p, shift, p->stream));
    HB_CUDA(cudaMemcpyAsync(jv, p->w32b.p, nd * sizeof(float), cudaMemcpyDeviceToHost, p->stream));
    int err = 0;
    HB_CUDA(cudaMemcpyAsync(&err, p->d_err.p, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    HB_CUDA(cudaStreamSynchronize(p->stream));
    return dev_err_status(p, err);
}

hb_status hb_jacobi_diag(hb_problem *p, const double *y, double *d, int precision, double shift) {
    return host_op(p, MODE_DIAG, y, nullptr, d, precision, shift);
}

hb_status hb_residual_dev(hb_problem *p, const void *y, void *r, int precision, void *stream) {
    return dev_op(p, MODE_RES, y, nullptr, r, precision, 0.0, stream);
}

hb_status hb_jv_dev(hb_problem *p, const void *y, const void *v, void *jv, int kind, int precision, double shift,
                    void *stream) {
    if (kind < 0 || kind > 2)
        return fail(HB_ERR_INVALID_ARG, "kind must be 0 (paper tangent), 1 (exact) or 2 (assembled paper tangent)");
    return dev_op(p, jv_mode(kind), y, v, jv, precision, shift, stream);
}

hb_status hb_assemble_dev(hb_problem *p, const void *y, int precision, void *stream) {
    if (!p || !y) return fail(HB_ERR_INVALID_ARG, "null argument");
    HB_TRY(check_precision(precision));
    HB_CUDA(cudaSetDevice(p->device));
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : p->stream;
    if (precision == 0) return assemble_at<double>(p, static_cast<const double *>(y), s);
    return assemble_at<float>(p, static_cast<const float *>(y), s);
}

hb_status hb_jacobi_diag_dev(hb_problem *p, const void *y, void *d, int precision, double shift, void *stream) {
    return dev_op(p, MODE_DIAG, y, nullptr, d, precision, shift, stream);
}

hb_status hb_default_opts(hb_solve_opts *o) {
    if (!o) return fail(HB_ERR_INVALID_ARG, "null options");
    o->precision = 1;
    o->rtol = 1e-11;
    o->switch_rtol = 1e-3;
    o->gmres_rtol_pseudo = 0.03;
    o->gmres_rtol_newton = 1e-3;
    o->gmres_restart = 30;
    o->max_gmres = 600;
    o->max_steps = 400;
    o->dt_pseudo = 0.0;
    o->cfl = 1.0;
    o->use_learned = 0;
    o->verbose = 0;
    o->ser = 1;
    o->ser_max = 1e4;
    o->r_ref = 0.0;
    o->assembled = 0;
    o->precond = 0;
    o->line_search = 1;
    o->scatter = 1;
    o->backflow_beta = -1.0;
    return HB_OK;
}

static hb_status solve_impl(hb_problem *p, const hb_solve_opts &o, hb_report *rep);

hb_status hb_attach_learned(hb_problem *p, hb_mpnn *net) {
    if (!p) return fail(HB_ERR_INVALID_ARG, "null problem");
    p->learned = net;
    return HB_OK;
}

hb_status hb_solve(hb_problem *p, const hb_solve_opts *opts, hb_report *rep) {
    if (!p) return fail(HB_ERR_INVALID_ARG, "null problem");
    hb_solve_opts o;
    hb_default_opts(&o);
    if (opts) o = *opts;
    HB_TRY(check_precision(o.precision));
    if (o.gmres_restart < 1 || o.gmres_restart > 200) return fail(HB_ERR_INVALID_ARG, "gmres_restart must be in [1, 200]");
    if (o.precond < 0 || o.precond > 2)
        return fail(HB_ERR_INVALID_ARG, "precond must be 0 (Jacobi), 1 (node blocks) or 2 (aggregation multigrid)");
    HB_CUDA(cudaSetDevice(p->device));
    if (o.scatter != p->scatter) HB_TRY(hb_set_scatter(p, o.scatter));
    if (o.backflow_beta >= 0 && o.backflow_beta != p->beta) HB_TRY(hb_set_backflow(p, o.backflow_beta));
    if (o.use_learned < 0 || o.use_learned > 2) return fail(HB_ERR_INVALID_ARG, "use_learned must be 0, 1 or 2");
    p->learned_dir = false;
    if (o.use_learned) {
        if (!p->learned) return fail(HB_ERR_STATE, "use_learned set but no network attached (hb_attach_learned)");
        if (o.use_learned == 2) {
            // keep the prediction as a target direction; the solve starts from the state it had
            HB_TRY(prepare_bc(p));
            if (!p->y_set) HB_TRY(default_initial(p));
            const size_t nd = size_t(p->n_nodes) * 4 * p->N;
            HB_TRY(dalloc(p, p->ylearn, nd));
            HB_TRY(dalloc(p, p->kd, nd));
            HB_CUDA(cudaMemcpyAsync(p->kd.p, p->y.p, nd * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
            HB_TRY(hb_mpnn_warm_start(p->learned, p));
            HB_CUDA(cudaMemcpyAsync(p->ylearn.p, p->y.p, nd * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
            HB_CUDA(cudaMemcpyAsync(p->y.p, p->kd.p, nd * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
            HB_CUDA(cudaStreamSynchronize(p->stream));
            p->learned_dir = true;
        } else {
            HB_TRY(hb_mpnn_warm_start(p->learned, p));
        }
    }
    if (p->own_stream) return solve_impl(p, o, rep);
    // the GMRES cycles are captured as CUDA graphs, which needs a stream of our own: order it after the
    // caller's stream, solve on it, and synchronise before handing the caller's stream back
    cudaStream_t user = p->stream, own = nullptr;
    cudaEvent_t ev = nullptr;
    HB_CUDA(cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking));
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaStreamDestroy(own);
        return fail(HB_ERR_CUDA, "cudaEventCreate failed");
    }
    cudaEventRecord(ev, user);
    cudaStreamWaitEvent(own, ev, 0);
    p->stream = own;
    hb_status st = solve_impl(p, o, rep);
    cudaStreamSynchronize(own);
    p->stream = user;
    cudaEventDestroy(ev);
    cudaStreamDestroy(own);
    return st;
}

static hb_status solve_impl(hb_problem *p, const hb_solve_opts &o, hb_report *rep) {
    const auto t0 = std::chrono::steady_clock::now();
    HB_TRY(prepare_bc(p));
    if (p->inflows.empty()) return fail(HB_ERR_STATE, "no inflow set");
    if (!p->y_set) HB_TRY(default_initial(p));
    HB_TRY(apply_dirichlet_state(p));
    const int64_t nd = p->n_nodes * 4 * p->N;
    HB_TRY(ensure_krylov(p, o.gmres_restart));
    hb_report R;
    std::memset(&R, 0, sizeof(R));
    const double dt = o.dt_pseudo > 0 ? o.dt_pseudo : (p->u_c > 0 ? o.cfl * h_char(p) / p->u_c : INFINITY);
    R.dt_pseudo = dt;
    const double shift0 = std::isfinite(dt) ? kC1 * p->rho / dt : 0.0;
    HB_TRY(dalloc(p, p->shift_dev, 1));
    double *r = p->w64a.p;
    double *b = p->w64b.p;
    HB_TRY(apply_op<double>(p, MODE_RES, p->y.p, nullptr, r, 0.0, p->stream));
    R.residual_calls++;
    double rn = 0;
    HB_TRY(dev_norm(p, r, nd, rn));
    R.res0 = rn;
    const double r0 = o.r_ref > 0 ? o.r_ref : rn;
    bool newton = false;
    hb_status result = HB_ERR_NOT_CONVERGED;
    double dxn = INFINITY;
    double eta = 0.1, rn_prev = rn;   // Eisenstat-Walker forcing term of the Newton phase
    double dtk = dt;                  // current pseudo step (adaptive when o.ser)
    bool ls_fallback = false;         // the last Newton step found no decrease: retake it with the shift
    int pc = o.precond;               // preconditioner in use: multigrid falls back to Jacobi after two
    int pc_misses = 0;                // consecutive linear solves that stall at the cap
    for (int step = 0; step < o.max_steps; ++step) {
        if (!std::isfinite(rn)) {
            result = fail(HB_ERR_NAN, "residual is not finite");
            break;
        }
        if (r0 == 0 || (rn <= o.rtol * r0 && step > 0)) {
            result = HB_OK;
            break;
        }
        if (rn < o.switch_rtol * r0) newton = true;
        // Pseudo shift c1 rho / dt (Sec. 2.3).  Paper mode (o.ser = 0): fixed dt with the paper's tangent,
        // then exact Newton without shift.  Adaptive mode (o.ser = 1): dt grows with the residual drop while
        // GMRES converges within its budget and shrinks when it does not; the exact Jacobian replaces the
        // paper's tangent after the switch, and the shift is dropped once dt exceeds ser_max x the CFL step.
        double shift = 0.0;
        if (!o.ser) shift = newton ? 0.0 : shift0;
        else if (std::isfinite(dtk) && dtk < dt * o.ser_max && !(newton && o.line_search && !ls_fallback))
            shift = kC1 * p->rho / dtk;
        p->shift_host = shift;
        HB_CUDA(cudaMemcpyAsync(p->shift_dev.p, &p->shift_host, sizeof(double), cudaMemcpyHostToDevice, p->stream));
        OpCtx c{newton ? MODE_JVE : MODE_JVP, shift, o.precision, p->shift_dev.p};
        // Jacobi diagonal of P (+ pseudo mass) and the frozen state in the kernels' precision
        if (o.precision == 1) {
            launch_convert_state(p->y.p, p->ky32.p, nd, p->N, p_level(p), p->stream);
            HB_LAUNCHED(p, 1);
            HB_TRY(apply_op<float>(p, MODE_DIAG, p->ky32.p, nullptr, p->kdiag32.p, c.shift, p->stream, c.shift_dev));
            launch_convert<float, double>(p->kdiag32.p, p->kdiag.p, nd, p->stream);
            HB_LAUNCHED(p, 1);
        } else {
            HB_TRY(apply_op<double>(p, MODE_DIAG, p->y.p, nullptr, p->kdiag.p, c.shift, p->stream, c.shift_dev));
        }
        launch_reciprocal(p->kdiag.p, p->kdiag.p, nd, p->stream);   // kdiag holds the inverse diagonal
        HB_LAUNCHED(p, 1);
        if ((o.assembled && c.mode == MODE_JVP) || pc >= 1) {
            // the paper's tangent assembled once for this step: GMRES applies it as a sparse product
            // (assembled, paper-tangent phase) and / or builds the preconditioner from it (node blocks, or
            // the multigrid hierarchy's coarse operators)
            if (o.precision == 1) HB_TRY(assemble_at<float>(p, p->ky32.p, p->stream));
            else HB_TRY(assemble_at<double>(p, p->y.p, p->stream));
            if (pc == 2) {
                if (o.precision == 1) HB_TRY(amg_values<float>(p, p->stream));
                else HB_TRY(amg_values<double>(p, p->stream));
            }
            if (o.assembled && c.mode == MODE_JVP) c.mode = MODE_JVA;
            c.precond = pc;
        }
        launch_scale_copy(-1.0, r, b, nd, p->stream);
        HB_LAUNCHED(p, 1);
        int its = 0, jvc = 0;
        double tol = o.gmres_rtol_pseudo;
        if (newton) {
            if (R.newton_steps > 0) {
                double e = 0.9 * (rn / rn_prev) * (rn / rn_prev);
                const double safe = 0.9 * eta * eta;
                if (safe > 0.1) e = std::max(e, safe);
                eta = e;
            }
            eta = std::min(0.1, std::max(o.gmres_rtol_newton, eta));
            tol = eta;
        }
        const double rn_before = rn;
        rn_prev = rn;
        // learned correction step (use_learned 2): the least-squares multiple alpha of d = y_pred - y
        // against A d is taken first, plain GMRES then works on what is left (alpha = 0 leaves plain
        // GMRES); prescribed entries of y_pred and y agree, so d vanishes there
        double alpha = 0, bscale = 1;
        if (p->learned_dir) {
            launch_scale_copy(1.0, p->ylearn.p, p->kd.p, nd, p->stream);
            launch_axpy(-1.0, p->y.p, p->kd.p, nd, p->stream);
            HB_LAUNCHED(p, 2);
            double dn = 0;
            HB_TRY(dev_norm(p, p->kd.p, nd, dn));
            if (dn > 0) {
                HB_TRY(apply_A(p, c, p->kd.p, p->ktmp.p));
                ++jvc;
                double qb = 0, qq = 0, b0 = 0, b1 = 0;
                HB_TRY(dev_dot(p, p->ktmp.p, b, nd, qb));
                HB_TRY(dev_dot(p, p->ktmp.p, p->ktmp.p, nd, qq));
                HB_TRY(dev_norm(p, b, nd, b0));
                if (qq > 0 && std::isfinite(qb / qq)) {
                    alpha = qb / qq;
                    launch_axpy(-alpha, p->ktmp.p, b, nd, p->stream);
                    HB_LAUNCHED(p, 1);
                    HB_TRY(dev_norm(p, b, nd, b1));
                    bscale = b0 > 0 ? b1 / b0 : 1.0;
                }
            }
        }
        double relres = 0;
        HB_TRY(gmres(p, c, b, p->kdx.p, tol / bscale, o.gmres_restart, o.max_gmres, its, jvc, &relres));
        relres *= bscale;                     // relative to the step's full right-hand side
        if (alpha != 0) {
            launch_axpy(alpha, p->kd.p, p->kdx.p, nd, p->stream);
            HB_LAUNCHED(p, 1);
        }
        R.gmres_iters += its;
        R.jv_calls += jvc;
        if (pc == 2) {   // a stalled multigrid solve: at the cap with less than half the residual removed
            pc_misses = (its >= o.max_gmres && relres > 0.5) ? pc_misses + 1 : 0;
            if (pc_misses >= 2) pc = 0;
        }
        const bool search = newton && o.line_search && shift == 0.0;
        if (search) {
            HB_TRY(dalloc(p, p->yprev, size_t(nd)));
            HB_CUDA(cudaMemcpyAsync(p->yprev.p, p->y.p, size_t(nd) * sizeof(double), cudaMemcpyDeviceToDevice,
                                    p->stream));
        }
        launch_axpy(1.0, p->kdx.p, p->y.p, nd, p->stream);
        HB_LAUNCHED(p, 1);
        HB_TRY(apply_op<double>(p, MODE_RES, p->y.p, nullptr, r, 0.0, p->stream));
        R.residual_calls++;
        double yn = 0;
        HB_TRY(dev_norm(p, r, nd, rn));
        if (search) {
            // backtracking on ||r||: y = y_prev + lambda dx, lambda = 1, 1/2, ..., 1/16
            double lam = 1.0;
            for (int b = 0; b < 4 && !(rn <= (1.0 - 1e-4 * lam) * rn_before); ++b) {
                lam *= 0.5;
                launch_scale_copy(1.0, p->yprev.p, p->y.p, nd, p->stream);
                launch_axpy(lam, p->kdx.p, p->y.p, nd, p->stream);
                HB_LAUNCHED(p, 2);
                HB_TRY(apply_op<double>(p, MODE_RES, p->y.p, nullptr, r, 0.0, p->stream));
                R.residual_calls++;
                HB_TRY(dev_norm(p, r, nd, rn));
            }
            ls_fallback = !(rn < rn_before);
            if (ls_fallback) {            // no decrease: take the step back and retake it with the shift
                launch_scale_copy(1.0, p->yprev.p, p->y.p, nd, p->stream);
                HB_LAUNCHED(p, 1);
                HB_TRY(apply_op<double>(p, MODE_RES, p->y.p, nullptr, r, 0.0, p->stream));
                R.residual_calls++;
                HB_TRY(dev_norm(p, r, nd, rn));
            }
            if (ls_fallback) {
                dtk = std::max(dt, 0.1 * dtk);        // the retaken step gets a noticeable shift
            } else if (lam != 1.0) {
                launch_scale_copy(lam, p->kdx.p, p->kdx.p, nd, p->stream);
                HB_LAUNCHED(p, 1);
            }
        } else {
            ls_fallback = false;
        }
        HB_TRY(dev_norm(p, p->kdx.p, nd, dxn));
        HB_TRY(dev_norm(p, p->y.p, nd, yn));
        R.steps++;
        if (newton) R.newton_steps++;
        if (o.ser) {
            if (relres <= tol * 1.0001) dtk *= std::min(4.0, std::max(1.0, rn_before / std::max(rn, 1e-300)));
            else dtk *= 0.5;
        }
        if (o.verbose)
            std::fprintf(stderr, "hb_solve step %d %s gmres %d |r|/|r0| %.3e |dy|/|y| %.3e\n", step,
                         newton ? "newton" : "pseudo", its, rn / r0, yn > 0 ? dxn / yn : 0.0);
        if (newton && rn <= o.rtol * r0 && dxn <= 10 * o.rtol * yn && shift == 0.0) {
            result = HB_OK;
            break;
        }
    }
    R.res_final = rn;
    R.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    R.status = result;
    if (rep) *rep = R;
    if (result == HB_ERR_NOT_CONVERGED) g_err = "solve reached max_steps";
    return result;
}

hb_status hb_jv_dev_noalloc(hb_problem *p, const void *y, const void *v, void *jv, int kind, int precision,
                            double shift, void *stream) {
    if (!p || !y || !v || !jv) return fail(HB_ERR_INVALID_ARG, "null argument");
    if (kind != 0 && kind != 1) return fail(HB_ERR_INVALID_ARG, "kind must be 0 (paper tangent) or 1 (exact)");
    HB_TRY(check_precision(precision));
    if (jv == y || jv == v) return fail(HB_ERR_INVALID_ARG, "output aliases an input");
    if (p->bc_dirty)
        return fail(HB_ERR_STATE, "boundary data not prepared: after the last hb_set_* call, call hb_get_info "
                                  "(or any other entry point) once before hb_jv_dev_noalloc");
    if (int64_t(p->n_out) * p->N > kNoAllocScratch)
        return fail(HB_ERR_INVALID_ARG, "outlets x instances (" + std::to_string(int64_t(p->n_out) * p->N) +
                                            ") exceeds the no-alloc scratch limit of " +
                                            std::to_string(kNoAllocScratch) + " values");
    HB_CUDA(cudaSetDevice(p->device));
    void *q = nullptr;
    HB_TRY(noalloc_scratch(p->device, &q));
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : p->stream;
    const int mode = kind == 0 ? MODE_JVP : MODE_JVE;
    if (precision == 0)
        return apply_jv_noalloc<double>(p, mode, static_cast<const double *>(y), static_cast<const double *>(v),
                                        static_cast<double *>(jv), shift, s, static_cast<double *>(q));
    return apply_jv_noalloc<float>(p, mode, static_cast<const float *>(y), static_cast<const float *>(v),
                                   static_cast<float *>(jv), shift, s, static_cast<float *>(q));
}

hb_status hb_default_march_opts(hb_march_opts *o) {
    if (!o) return fail(HB_ERR_INVALID_ARG, "null options");
    o->precision = 1;
    o->steps_per_period = 0;
    o->periods = 4;
    o->rho_inf = 0.5;
    o->newton_rtol = 1e-3;
    o->newton_max = 10;
    o->gmres_rtol = 0.03;
    o->gmres_restart = 15;
    o->max_gmres = 300;
    o->tau_acceleration = 1;
    o->verbose = 0;
    return HB_OK;
}

static hb_status march_impl(hb_problem *p, const hb_march_opts &o, hb_march_report *rep);

hb_status hb_march(hb_problem *p, const hb_march_opts *opts, hb_march_report *rep) {
    if (!p) return fail(HB_ERR_INVALID_ARG, "null problem");
    hb_march_opts o;
    hb_default_march_opts(&o);
    if (opts) o = *opts;
    HB_TRY(check_precision(o.precision));
    if (o.steps_per_period <= 0) o.steps_per_period = 100 * p->N;
    if (o.steps_per_period % p->N != 0)
        return fail(HB_ERR_INVALID_ARG, "steps_per_period must be a multiple of N (to sample the instance times)");
    if (o.periods < 1 || o.newton_max < 1 || o.max_gmres < 1 || !(o.rho_inf >= 0 && o.rho_inf <= 1))
        return fail(HB_ERR_INVALID_ARG, "periods, newton_max, max_gmres >= 1 and rho_inf in [0, 1] required");
    if (o.gmres_restart < 1 || o.gmres_restart > 200) return fail(HB_ERR_INVALID_ARG, "gmres_restart must be in [1, 200]");
    HB_CUDA(cudaSetDevice(p->device));
    HB_TRY(prepare_bc(p));
    if (p->inflows.empty()) return fail(HB_ERR_STATE, "no inflow set");
    return march_impl(p, o, rep);
}

hb_status hb_get_march_samples(hb_problem *p, double *out) {
    if (!p || !out) return fail(HB_ERR_INVALID_ARG, "null argument");
    if (!p->march_done) return fail(HB_ERR_STATE, "no march has run (hb_march)");
    HB_CUDA(cudaSetDevice(p->device));
    HB_CUDA(cudaMemcpyAsync(out, p->d_march.p, size_t(p->n_nodes) * 4 * p->N * sizeof(double),
                            cudaMemcpyDeviceToHost, p->tm->stream));
    HB_CUDA(cudaStreamSynchronize(p->tm->stream));
    return HB_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------------
// time-domain march (Sec. 3): the conventional GLS solver with tau_hat (Eq. tauhat), generalized-alpha in
// time, Newton on the paper's tangent with Jacobi-preconditioned GMRES, on a one-instance copy of the
// problem whose boundary values are re-evaluated from the harmonic data at every step

namespace {

// one-instance copy: same mesh, fluid and boundary tags; the series are cut to their means (only the
// Dirichlet node set, the Neumann faces and the resistances matter: values are set per step)
hb_status tm_copy(hb_problem *p) {
    if (p->tm) return HB_OK;
    hb_mesh m;
    m.n_nodes = p->n_nodes;
    m.n_tets = p->n_tets;
    m.n_faces = p->n_faces;
    m.xyz = p->xyz.data();
    m.tets = p->tets.data();
    m.faces = p->faces.data();
    m.face_tag = p->face_tag.data();
    hb_problem *c = nullptr;
    HB_TRY(hb_create(&m, p->rho, p->mu, p->T, 0, p->device, nullptr, &c));
    auto bail = [&](hb_status st) {
        hb_destroy(c);
        return st;
    };
    hb_status st = HB_OK;
    const int M = 2 * p->n_h + 1;
    for (const Inflow &in : p->inflows) {
        if (!in.harm.empty()) {
            std::vector<double> h0(size_t(p->n_nodes) * 3);
            for (size_t r = 0; r < h0.size(); ++r) h0[r] = in.harm[r * size_t(M)];
            st = hb_set_inflow_harmonics(c, in.tag, h0.data());
        } else {
            const double a0 = in.coef[0], b0 = 0.0;
            st = hb_set_inflow(c, in.tag, in.profile.empty() ? nullptr : in.profile.data(), &a0, &b0);
        }
        if (st != HB_OK) return bail(st);
    }
    for (const Outlet &ou : p->outlets) {
        const double a0 = ou.coef[0], b0 = 0.0;
        st = ou.R > 0 ? hb_set_outlet_resistance(c, ou.tag, ou.R, &a0, &b0) : hb_set_outlet_pressure(c, ou.tag, &a0, &b0);
        if (st != HB_OK) return bail(st);
    }
    if ((st = hb_set_backflow(c, p->beta)) != HB_OK) return bail(st);
    if ((st = prepare_bc(c)) != HB_OK) return bail(st);
    if (c->n_dir != p->n_dir || c->n_out != p->n_out) return bail(fail(HB_ERR_STATE, "time-domain copy differs"));
    c->jvp_variant = p->jvp_variant;
    c->ls_mass = 1;
    p->tm = c;
    return HB_OK;
}

// outlet traction levels -P(t) of the copy (h of the resistance outlets adds -R Q in the face kernel)
hb_status tm_outlets_at(hb_problem *p, double t) {
    hb_problem *c = p->tm;
    if (p->n_out == 0) return HB_OK;
    std::vector<double> hb(size_t(p->n_out));
    const double w = p->omega;
    for (int o = 0; o < p->n_out; ++o) {
        const std::vector<double> &cf = p->outlets[size_t(o)].coef;
        double v = cf[0];
        for (int k = 1; k <= p->n_h; ++k) v += cf[size_t(2 * k - 1)] * std::cos(k * w * t) + cf[size_t(2 * k)] * std::sin(k * w * t);
        hb[size_t(o)] = -v;
    }
    std::vector<float> hf(hb.begin(), hb.end());
    HB_CUDA(cudaMemcpyAsync(c->d_hbase64.p, hb.data(), hb.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    HB_CUDA(cudaMemcpyAsync(c->d_hbase32.p, hf.data(), hf.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    HB_CUDA(cudaStreamSynchronize(c->stream));      // the host arrays go out of scope
    return HB_OK;
}

hb_status vel_norm2(hb_problem *p, const double *x, int64_t n, double &out) {
    HB_TRY(dalloc(p, p->small, 512));
    launch_vel_norm2(x, n, p->scratch.p, p->small.p, p->stream);
    HB_LAUNCHED(p, 2);
    HB_CUDA(cudaMemcpyAsync(&out, p->small.p, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    HB_CUDA(cudaStreamSynchronize(p->stream));
    return HB_OK;
}

}  // namespace

static hb_status march_impl(hb_problem *p, const hb_march_opts &o, hb_march_report *rep) {
    const auto t0 = std::chrono::steady_clock::now();
    HB_TRY(tm_copy(p));
    hb_problem *c = p->tm;
    cudaStream_t s = c->stream;
    const int64_t n = c->n_nodes * 4;                // one time level
    HB_TRY(ensure_krylov(c, o.gmres_restart));
    for (DBuf<double> *b : {&p->tm_un, &p->tm_dun, &p->tm_u1, &p->tm_du1, &p->tm_dya, &p->tm_prev})
        HB_TRY(dalloc(c, *b, size_t(n)));
    HB_TRY(dalloc(c, p->d_march, size_t(n) * size_t(p->N)));
    // generalized-alpha for first-order systems (reading R13); c1 = alpha_m / (alpha_f gamma)
    const double ri = o.rho_inf;
    const double am = (3.0 - ri) / (2.0 * (1.0 + ri)), af = 1.0 / (1.0 + ri), gam = 0.5 + am - af;
    const int spp = o.steps_per_period;
    const double dt = p->T / spp, inv_gdt = 1.0 / (gam * dt), cg = (gam - 1.0) / gam;
    const double shift = am / (af * gam) * p->rho / dt;
    const int stride = spp / p->N;
    // initial state: zero interior velocity and acceleration, Dirichlet values at t = 0, pressure at the
    // outlets' mean level
    HB_TRY(default_initial(c));
    launch_series_at(p->d_dir_prof.p, int64_t(3) * p->n_dir, p->n_h, 0.0, c->d_g.p, s);
    launch_apply_dirichlet(c->d_dir_nodes.p, c->n_dir, c->d_g.p, c->y.p, 1, s);
    HB_CUDA(cudaMemcpyAsync(p->tm_un.p, c->y.p, size_t(n) * sizeof(double), cudaMemcpyDeviceToDevice, s));
    HB_CUDA(cudaMemsetAsync(p->tm_dun.p, 0, size_t(n) * sizeof(double), s));
    HB_LAUNCHED(c, 2);
    hb_march_report R;
    std::memset(&R, 0, sizeof(R));
    hb_status result = HB_OK;
    double *r = c->w64a.p, *b = c->w64b.p;
    const int nsteps = spp * o.periods;
    for (int k = 0; k < nsteps && result == HB_OK; ++k) {
        const double frac1 = double((k + 1) % spp) / spp;          // t_{n+1} / T mod 1
        const double t_af = (double(k) + af) * dt;
        launch_series_at(p->d_dir_prof.p, int64_t(3) * p->n_dir, p->n_h, frac1, c->d_g.p, s);
        launch_galpha_predict(p->tm_un.p, p->tm_dun.p, p->tm_u1.p, p->tm_du1.p, n, cg, c->d_dir_nodes.p, c->n_dir,
                              c->d_g.p, inv_gdt, s);
        HB_LAUNCHED(c, c->n_dir > 0 ? 3 : 2);
        HB_TRY(tm_outlets_at(p, t_af));
        double r0 = -1, rn = 0;
        for (int it = 0; it < o.newton_max; ++it) {
            // stage values; the tangent is frozen at c->y = (u, p)_{n+alpha_f}
            launch_galpha_stage(p->tm_un.p, p->tm_u1.p, p->tm_dun.p, p->tm_du1.p, c->y.p, p->tm_dya.p, n, af, am, s);
            HB_LAUNCHED(c, 1);
            c->omega2 = 0;
            if (o.tau_acceleration) {
                double a2 = 0, u2 = 0;
                HB_TRY(vel_norm2(c, p->tm_dya.p, n, a2));
                HB_TRY(vel_norm2(c, c->y.p, n, u2));
                c->omega2 = u2 > 0 ? a2 / u2 : 0.0;              // reading R14
            }
            HB_TRY(apply_op<double>(c, MODE_TRES, c->y.p, p->tm_dya.p, r, 0.0, s));
            HB_TRY(dev_norm(c, r, n, rn));
            if (!std::isfinite(rn)) {
                result = fail(HB_ERR_NAN, "non-finite residual in the time-domain march");
                break;
            }
            if (r0 < 0) r0 = rn;
            if (rn == 0.0 || (it > 0 && rn <= o.newton_rtol * r0)) break;
            // Jacobi diagonal of the tangent (+ c1 rho / dt M), stored inverted
            if (o.precision == 1) {
                launch_convert<double, float>(c->y.p, c->ky32.p, n, s);
                HB_LAUNCHED(c, 1);
                HB_TRY(apply_op<float>(c, MODE_DIAG, c->ky32.p, nullptr, c->kdiag32.p, shift, s));
                launch_convert<float, double>(c->kdiag32.p, c->kdiag.p, n, s);
                HB_LAUNCHED(c, 1);
            } else {
                HB_TRY(apply_op<double>(c, MODE_DIAG, c->y.p, nullptr, c->kdiag.p, shift, s));
            }
            launch_reciprocal(c->kdiag.p, c->kdiag.p, n, s);
            launch_scale_copy(-1.0 / af, r, b, n, s);
            HB_LAUNCHED(c, 2);
            int its = 0, jvc = 0;
            OpCtx ctx{MODE_JVP, shift, o.precision, nullptr};
            HB_TRY(gmres(c, ctx, b, c->kdx.p, o.gmres_rtol, o.gmres_restart, o.max_gmres, its, jvc));
            launch_galpha_correct(p->tm_u1.p, p->tm_du1.p, c->kdx.p, n, inv_gdt, s);
            HB_LAUNCHED(c, 1);
            R.newton_iters++;
            R.gmres_iters += its;
            R.jv_calls += jvc;
        }
        if (r0 > 0) R.max_newton_rel = std::max(R.max_newton_rel, rn / r0);
        p->tm_un.swap(p->tm_u1);
        p->tm_dun.swap(p->tm_du1);
        R.steps++;
        if ((k + 1) % spp == 0 && k + 1 < nsteps)       // state at the end of each period but the last
            HB_CUDA(cudaMemcpyAsync(p->tm_prev.p, p->tm_un.p, size_t(n) * sizeof(double), cudaMemcpyDeviceToDevice, s));
        if (k + 1 > nsteps - spp && (k + 1) % stride == 0) {    // last period: the instance times t_j = j T / N
            const int j = ((k + 1) % spp) / stride;
            launch_put_instance(p->tm_un.p, p->d_march.p, n, j, p->N, s);
            HB_LAUNCHED(c, 1);
        }
        if (o.verbose && ((k + 1) % stride == 0))
            std::fprintf(stderr, "hb_march step %d t/T %.4f |r|/|r0| %.3e\n", k + 1, double(k + 1) / spp,
                         r0 > 0 ? rn / r0 : 0.0);
    }
    if (result == HB_OK && o.periods > 1) {
        // relative change over the last period: ||u(T_end) - u(T_end - T)|| / ||u(T_end)||
        launch_axpy(-1.0, p->tm_un.p, p->tm_prev.p, n, s);
        HB_LAUNCHED(c, 1);
        double dn = 0, un = 0;
        HB_TRY(dev_norm(c, p->tm_prev.p, n, dn));
        HB_TRY(dev_norm(c, p->tm_un.p, n, un));
        R.period_change = un > 0 ? dn / un : 0.0;
    }
    HB_CUDA(cudaStreamSynchronize(s));
    p->launches += c->launches;
    c->launches = 0;
    p->march_done = result == HB_OK;
    R.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    R.status = result;
    if (rep) *rep = R;
    return result;
}

extern "C" {

hb_status hb_time_residual(hb_problem *p, const double *y, const double *ydot, double *r, int precision, double t,
                           double omega2) {
    if (!p || !y || !ydot || !r) return fail(HB_ERR_INVALID_ARG, "null argument");
    HB_TRY(check_precision(precision));
    if (!(omega2 >= 0)) return fail(HB_ERR_INVALID_ARG, "omega2 must be >= 0");
    HB_CUDA(cudaSetDevice(p->device));
    HB_TRY(prepare_bc(p));
    HB_TRY(tm_copy(p));
    HB_TRY(tm_outlets_at(p, t));
    p->tm->omega2 = omega2;
    const hb_status st = host_op(p->tm, MODE_TRES, y, ydot, r, precision, 0.0);
    p->tm->omega2 = 0;
    return st;
}

hb_status hb_time_jv(hb_problem *p, const double *y, const double *v, double *jv, int precision, double omega2,
                     double shift) {
    if (!p || !y || !v || !jv) return fail(HB_ERR_INVALID_ARG, "null argument");
    HB_TRY(check_precision(precision));
    if (!(omega2 >= 0)) return fail(HB_ERR_INVALID_ARG, "omega2 must be >= 0");
    HB_CUDA(cudaSetDevice(p->device));
    HB_TRY(prepare_bc(p));
    HB_TRY(tm_copy(p));
    p->tm->omega2 = omega2;
    const hb_status st = host_op(p->tm, MODE_JVP, y, v, jv, precision, shift);
    p->tm->omega2 = 0;
    return st;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------------
// batches: one captured graph applies the operator of many problems, their element work in one
// persistent launch

struct hb_batch {
    std::vector<hb_problem *> probs;
    int precision = 1, device = 0;
    cudaStream_t stream = nullptr;
    DBuf<ElemArgs<float>> args32;
    DBuf<ElemArgs<double>> args64;
    DBuf<int> bslots, counter;
    int n_items = 0, grid = 0;
    size_t smem = 0;
    cudaGraphExec_t exec = nullptr;
    int mode = -1;
    double shift = 0;
    std::vector<const void *> y, v;
    std::vector<void *> out;
    int64_t launches_per_replay = 0, launches = 0;
    int grouping = 2;                     // launch layout (hb_batch_set_grouping): 2 = members on parallel branches
    std::vector<uint64_t> gens;           // the members' settings generations at the last capture
    static constexpr int kSide = 8;       // side streams of the captured graph's parallel branches
    cudaStream_t side[kSide] = {};
};

namespace {

// grouping 2: every member's whole operator (the single-problem path: clearing, W pass, element pass with
// the member's own kernel arguments, boundary terms) on one of kSide parallel graph branches, members
// q, q + kSide, ... in sequence on branch q mod kSide; the branches run concurrently, so the blocks of one
// member's element launch fill the SMs that another's tail leaves idle.
template <typename T>
hb_status batch_record_branches(hb_batch *b) {
    cudaStream_t s = b->stream;
    const size_t np = b->probs.size();
    std::vector<int64_t> l0(np);
    for (size_t q = 0; q < np; ++q) {
        hb_problem *p = b->probs[q];
        HB_TRY(prepare_bc(p));          // host work and uploads stay outside the capture
        l0[q] = p->launches;
        if (b->mode == MODE_JVP) {     // the W rows, allocated outside the capture
            DBuf<T> &W = AsmBufs<T>::W(p->as);
            HB_TRY(dalloc(p, W, size_t(p->n_nodes) * size_t(w_stride(p->N, int(sizeof(T))))));
        }
    }
    HB_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    hb_status st = HB_OK;
    std::vector<cudaEvent_t> evs;
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) st = fail(HB_ERR_CUDA, "event");
    if (st == HB_OK) {
        evs.push_back(ev);
        cudaEventRecord(ev, s);
        for (int k = 0; k < hb_batch::kSide; ++k) cudaStreamWaitEvent(b->side[k], ev, 0);
    }
    for (size_t q = 0; q < np && st == HB_OK; ++q)
        st = apply_op<T>(b->probs[q], b->mode, static_cast<const T *>(b->y[q]), static_cast<const T *>(b->v[q]),
                         static_cast<T *>(b->out[q]), b->shift, b->side[q % hb_batch::kSide]);
    for (int k = 0; k < hb_batch::kSide && st == HB_OK; ++k) {
        cudaEvent_t j = nullptr;
        if (cudaEventCreateWithFlags(&j, cudaEventDisableTiming) != cudaSuccess) {
            st = fail(HB_ERR_CUDA, "event");
            break;
        }
        evs.push_back(j);
        cudaEventRecord(j, b->side[k]);
        cudaStreamWaitEvent(s, j, 0);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    for (cudaEvent_t x : evs) cudaEventDestroy(x);
    int64_t launched = 0;
    for (size_t q = 0; q < np; ++q) {
        launched += b->probs[q]->launches - l0[q];
        b->probs[q]->launches = l0[q];
    }
    if (st != HB_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return fail(HB_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(e));
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(HB_ERR_CUDA, std::string("batch graph instantiate: ") + cudaGetErrorString(e));
    b->launches_per_replay = launched;
    return HB_OK;
}

template <typename T>
hb_status batch_record(hb_batch *b) {
    if (b->grouping == 2) return batch_record_branches<T>(b);
    cudaStream_t s = b->stream;
    hb_problem *p0 = b->probs[0];
    // problems ordered by instance count: each run of equal N is one persistent launch of the pass
    // specialised for that N
    const size_t np = b->probs.size();
    std::vector<size_t> ord(np);
    for (size_t q = 0; q < np; ++q) ord[q] = q;
    std::stable_sort(ord.begin(), ord.end(), [&](size_t x, size_t y) { return b->probs[x]->N < b->probs[y]->N; });
    std::vector<ElemArgs<T>> args(np);
    size_t smem = 0;
    int slot_cap = 0;
    for (size_t r = 0; r < np; ++r) slot_cap = std::max(slot_cap, slot_ints(patches<T>(b->probs[ord[r]], b->mode).nl_max));
    const int bstride = 4 + slot_cap;               // batch slot: [problem, 0, 0, 0, patch slot]
    for (size_t r = 0; r < np; ++r) {
        const size_t q = ord[r];
        hb_problem *p = b->probs[q];
        PatchSetDev<T> &ps = patches<T>(p, b->mode);
        ElemArgs<T> &ea = args[r];
        ea = elem_args<T>(p, ps, static_cast<const T *>(b->y[q]), static_cast<const T *>(b->v[q]),
                          static_cast<T *>(b->out[q]), b->shift, nullptr);
        if (b->mode == MODE_JVP) {
            // the member's node-level W = shift v + rho H v pass runs inside the graph (parallel branches);
            // the batched element pass gathers its rows as the single-problem pass does
            DBuf<T> &W = AsmBufs<T>::W(p->as);
            HB_TRY(dalloc(p, W, size_t(p->n_nodes) * size_t(w_stride(p->N, int(sizeof(T))))));
            ea.W = W.p;
        }
        smem = std::max(smem, elem_smem_bytes(b->mode, p->N, ps.nl_max, ps.ep_max, sizeof(T), bstride));
    }
    DBuf<ElemArgs<T>> &dargs = [&]() -> DBuf<ElemArgs<T>> & {
        if constexpr (sizeof(T) == 4) return b->args32;
        else return b->args64;
    }();
    HB_TRY(dalloc(p0, dargs, args.size()));
    HB_CUDA(cudaMemcpy(dargs.p, args.data(), args.size() * sizeof(ElemArgs<T>), cudaMemcpyHostToDevice));
    std::vector<int> first(np + 1, 0);
    for (size_t r = 0; r < np; ++r) first[r + 1] = first[r] + args[r].pv.n_patches;
    b->n_items = first.back();
    // batch slot table: each item's header (its problem) and a copy of its patch slot (the slots carry
    // the current Dirichlet bits, so the table is rebuilt with every recording)
    HB_TRY(dalloc(p0, b->bslots, size_t(std::max(1, b->n_items)) * size_t(bstride)));
    {
        std::vector<int> head(size_t(std::max(1, b->n_items)) * 4, 0);
        for (size_t r = 0; r < np; ++r)
            for (int k = first[r]; k < first[r + 1]; ++k) head[size_t(k) * 4] = int(r);
        if (b->n_items > 0)
            HB_CUDA(cudaMemcpy2DAsync(b->bslots.p, size_t(bstride) * 4, head.data(), 16, 16, size_t(b->n_items),
                                      cudaMemcpyHostToDevice, s));
        for (size_t r = 0; r < np; ++r) {
            const PatchView<T> &pv = args[r].pv;
            if (pv.n_patches == 0) continue;
            HB_CUDA(cudaMemcpy2DAsync(b->bslots.p + size_t(first[r]) * bstride + 4, size_t(bstride) * 4, pv.slots,
                                      size_t(pv.slot_stride) * 4, size_t(pv.slot_stride) * 4, size_t(pv.n_patches),
                                      cudaMemcpyDeviceToDevice, s));
        }
        HB_CUDA(cudaStreamSynchronize(s));
    }
    // grouping 0: one persistent launch over every member's patches (N = -1: the kernel dispatches on each
    // member's instance count), so members of different N share the SMs and the launch's tail;
    // grouping 1: one persistent launch per instance count (the kernel specialised for that N), the
    // launches on parallel graph branches so that one's tail overlaps the next one's start
    std::vector<BatchGroup<T>> groups;
    {
        BatchGroup<T> g;
        g.args = dargs.p;
        g.bslots = b->bslots.p;
        g.bslot_stride = bstride;
        g.variant = p0->jvp_variant;
        if (b->grouping == 0) {
            g.N = -1;
            g.item_begin = 0;
            g.item_end = b->n_items;
            if (b->n_items > 0) groups.push_back(g);
        } else {
            for (size_t r = 0; r < np;) {
                size_t r1 = r;
                while (r1 < np && b->probs[ord[r1]]->N == b->probs[ord[r]]->N) ++r1;
                g.N = b->probs[ord[r]]->N;
                g.item_begin = first[r];
                g.item_end = first[r1];
                if (g.item_end > g.item_begin) groups.push_back(g);
                r = r1;
            }
        }
        if (groups.size() > size_t(hb_batch::kSide))
            return fail(HB_ERR_INVALID_ARG, "more distinct instance counts than parallel branches in the batch");
        HB_TRY(dalloc(p0, b->counter, std::max<size_t>(1, groups.size())));
        for (size_t k = 0; k < groups.size(); ++k) groups[k].counter = b->counter.p + k;
    }
    int max_blocks = 1;
    if (smem <= 113 * 1024 && sizeof(T) == 4) max_blocks = 2;
    b->grid = p0->sm_count * max_blocks;
    b->smem = smem;
    const int64_t l0 = p0->launches;
    HB_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    hb_status st = HB_OK;
    std::vector<cudaEvent_t> evs;
    // fork s into the kSide branches (member q on branch q mod kSide), and join them back into s
    auto fork = [&]() {
        cudaEvent_t ev = nullptr;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            st = fail(HB_ERR_CUDA, "event");
            return;
        }
        evs.push_back(ev);
        cudaEventRecord(ev, s);
        for (int k = 0; k < hb_batch::kSide; ++k) cudaStreamWaitEvent(b->side[k], ev, 0);
    };
    auto join = [&]() {
        for (int k = 0; k < hb_batch::kSide && st == HB_OK; ++k) {
            cudaEvent_t ev = nullptr;
            if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
                st = fail(HB_ERR_CUDA, "event");
                return;
            }
            evs.push_back(ev);
            cudaEventRecord(ev, b->side[k]);
            cudaStreamWaitEvent(s, ev, 0);
        }
    };
    if (cudaMemsetAsync(b->counter.p, 0, groups.size() * sizeof(int), s) != cudaSuccess)
        st = fail(HB_ERR_CUDA, "memset in batch capture");
    // branches before the element pass: each member's output cleared, then (paper tangent) its node-level
    // W = shift v + rho H v pass, whose rows the batched element pass gathers
    if (st == HB_OK) fork();
    for (size_t q = 0; q < b->probs.size() && st == HB_OK; ++q) {
        hb_problem *p = b->probs[q];
        cudaStream_t ss = b->side[q % hb_batch::kSide];
        if (cudaMemsetAsync(b->out[q], 0, size_t(p->n_nodes) * 4 * p->N * sizeof(T), ss) != cudaSuccess) {
            st = fail(HB_ERR_CUDA, "memset in batch capture");
            break;
        }
        if (b->mode == MODE_JVP) {
            launch_spectral_w<T>(static_cast<const T *>(b->v[q]), Hmat<T>(p), p->d_flag.p, AsmBufs<T>::W(p->as).p,
                                 w_stride(p->N, int(sizeof(T))), p->n_nodes, p->N, T(p->rho), T(b->shift), nullptr,
                                 ss, p->spectral_path, p->d_err.p);
            p0->launches += 1;
        }
    }
    if (st == HB_OK) join();
    if (groups.size() == 1) {
        const BatchGroup<T> &g = groups[0];
        launch_batch_elem<T>(b->mode, g, smem, std::min(b->grid, g.item_end - g.item_begin), s);
        p0->launches += 1;
    } else if (st == HB_OK && !groups.empty()) {
        fork();
        for (size_t k = 0; k < groups.size(); ++k) {
            const BatchGroup<T> &g = groups[k];
            launch_batch_elem<T>(b->mode, g, smem, std::min(b->grid, g.item_end - g.item_begin), b->side[k]);
            p0->launches += 1;
        }
        join();
    }
    // branches after it: each member's boundary terms
    if (st == HB_OK) fork();
    for (size_t q = 0; q < b->probs.size() && st == HB_OK; ++q) {
        hb_problem *p = b->probs[q];
        cudaStream_t ss = b->side[q % hb_batch::kSide];
        const T *y = static_cast<const T *>(b->y[q]);
        const T *v = static_cast<const T *>(b->v[q]);
        T *out = static_cast<T *>(b->out[q]);
        if (b->mode != MODE_DIAG && p->n_nf > 0) {
            FaceArgs<T> fa = face_args<T>(p, y, v, out);
            if (p->has_res && cudaMemsetAsync(fa.Q, 0, size_t(p->n_out) * p->N * sizeof(T), ss) != cudaSuccess)
                st = fail(HB_ERR_CUDA, "memset in batch capture");
            launch_faces<T>(b->mode, fa, p->has_res, p->n_out, ss);
            p0->launches += p->has_res ? 2 : 1;
        }
    }
    if (st == HB_OK) join();
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
    if (st != HB_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return fail(HB_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(e));
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(HB_ERR_CUDA, std::string("batch graph instantiate: ") + cudaGetErrorString(e));
    b->launches_per_replay = p0->launches - l0;
    p0->launches = l0;
    return HB_OK;
}

}  // namespace

extern "C" {

hb_status hb_batch_create(hb_problem *const *problems, int count, int precision, hb_batch **out) {
    if (!problems || count <= 0 || !out) return fail(HB_ERR_INVALID_ARG, "empty batch");
    HB_TRY(check_precision(precision));
    *out = nullptr;
    const int dev = problems[0]->device;
    for (int q = 0; q < count; ++q) {
        if (!problems[q]) return fail(HB_ERR_INVALID_ARG, "null problem in batch");
        if (problems[q]->device != dev) return fail(HB_ERR_INVALID_ARG, "batch problems must share one device");
    }
    HB_CUDA(cudaSetDevice(dev));
    hb_batch *b = new hb_batch();
    b->probs.assign(problems, problems + count);
    b->precision = precision;
    b->device = dev;
    for (int q = 0; q < count; ++q) {
        hb_status st = prepare_bc(problems[q]);
        if (st != HB_OK) {
            delete b;
            return st;
        }
    }
    hb_problem *p0 = problems[0];
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete b;
        return fail(HB_ERR_CUDA, "cudaStreamCreate failed");
    }
    for (int k = 0; k < hb_batch::kSide; ++k)
        if (cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking) != cudaSuccess) {
            hb_batch_destroy(b);
            return fail(HB_ERR_CUDA, "cudaStreamCreate failed");
        }
    hb_status st = dalloc(p0, b->counter, size_t(count));
    if (st != HB_OK) {
        cudaStreamDestroy(b->stream);
        delete b;
        return st;
    }
    *out = b;
    return HB_OK;
}

hb_status hb_batch_destroy(hb_batch *b) {
    if (!b) return HB_OK;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    cudaStream_t s = b->stream;
    for (int k = 0; k < hb_batch::kSide; ++k)
        if (b->side[k]) cudaStreamDestroy(b->side[k]);
    delete b;
    if (s) cudaStreamDestroy(s);
    return HB_OK;
}

hb_status hb_batch_jv_dev(hb_batch *b, const void *const *y, const void *const *v, void *const *jv, int kind,
                          double shift, void *stream) {
    if (!b || !y || !v || !jv) return fail(HB_ERR_INVALID_ARG, "null argument");
    if (kind != 0 && kind != 1) return fail(HB_ERR_INVALID_ARG, "kind must be 0 (paper tangent) or 1 (exact)");
    HB_CUDA(cudaSetDevice(b->device));
    const size_t n = b->probs.size();
    const int mode = kind == 0 ? MODE_JVP : MODE_JVE;
    for (size_t q = 0; q < n; ++q) HB_TRY(prepare_bc(b->probs[q]));   // boundary data changed since the capture
    bool same = b->exec && b->mode == mode && b->shift == shift && b->y.size() == n && b->gens.size() == n;
    for (size_t q = 0; same && q < n; ++q)
        same = (b->y[q] == y[q] && b->v[q] == v[q] && b->out[q] == jv[q] && b->gens[q] == b->probs[q]->gen);
    for (size_t q = 0; q < n; ++q)
        if (!y[q] || !v[q] || !jv[q] || jv[q] == y[q] || jv[q] == v[q])
            return fail(HB_ERR_INVALID_ARG, "null or aliased operand in batch");
    if (!same) {
        b->mode = mode;
        b->shift = shift;
        b->y.assign(y, y + n);
        b->v.assign(v, v + n);
        b->out.assign(jv, jv + n);
        const hb_status st = b->precision == 0 ? batch_record<double>(b) : batch_record<float>(b);
        if (st != HB_OK) {                        // no graph of other operands may be replayed later
            if (b->exec) cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
            b->mode = -1;
            return st;
        }
        b->gens.resize(n);
        for (size_t q = 0; q < n; ++q) b->gens[q] = b->probs[q]->gen;
    }
    cudaStream_t user = stream ? static_cast<cudaStream_t>(stream) : b->probs[0]->stream;
    cudaEvent_t ev;
    HB_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaEventRecord(ev, user);
    cudaStreamWaitEvent(b->stream, ev, 0);
    cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
    cudaEventRecord(ev, b->stream);
    cudaStreamWaitEvent(user, ev, 0);
    cudaEventDestroy(ev);
    if (e != cudaSuccess) return fail(HB_ERR_CUDA, std::string("batch graph launch: ") + cudaGetErrorString(e));
    b->launches += b->launches_per_replay;
    return HB_OK;
}

int64_t hb_batch_launch_count(const hb_batch *b) { return b ? b->launches : 0; }

hb_status hb_batch_set_grouping(hb_batch *b, int grouping) {
    if (!b) return fail(HB_ERR_INVALID_ARG, "null batch");
    if (grouping < 0 || grouping > 2)
        return fail(HB_ERR_INVALID_ARG, "grouping must be 0 (one launch), 1 (per N) or 2 (per member, concurrent)");
    if (grouping != b->grouping) {
        b->grouping = grouping;
        b->mode = -1;                         // recapture on the next call
    }
    return HB_OK;
}

// Autotuning of the patch node cap: rebuild the patches with each candidate, time `reps` paper-tangent
// Jv applications (CUDA events around the element pass), keep the fastest.
hb_status hb_tune_patches(hb_problem *p, int precision, const int *candidates, int n_cand, int reps, int *best_nl,
                          double *best_ms) {
    if (!p || !candidates || n_cand <= 0 || reps <= 0) return fail(HB_ERR_INVALID_ARG, "bad tuning arguments");
    HB_TRY(check_precision(precision));
    HB_CUDA(cudaSetDevice(p->device));
    HB_TRY(prepare_bc(p));
    const size_t nd = size_t(p->n_nodes) * 4 * p->N;
    double best = INFINITY;
    int bnl = 0;
    const size_t ts = precision == 0 ? sizeof(double) : sizeof(float);
    const size_t budget = precision == 0 ? 200 * 1024 : 112 * 1024;
    HB_TRY(dalloc(p, p->w64a, nd));
    HB_TRY(dalloc(p, p->w64b, nd));
    HB_TRY(dalloc(p, p->w32a, nd));
    HB_TRY(dalloc(p, p->w32b, nd));
    HB_TRY(dalloc(p, p->w32c, nd));
    HB_TRY(dalloc(p, p->kres, nd));
    HB_CUDA(cudaMemsetAsync(p->w64a.p, 0, nd * sizeof(double), p->stream));
    HB_CUDA(cudaMemsetAsync(p->w32a.p, 0, nd * sizeof(float), p->stream));
    HB_CUDA(cudaMemsetAsync(p->w64b.p, 0, nd * sizeof(double), p->stream));
    HB_CUDA(cudaMemsetAsync(p->w32c.p, 0, nd * sizeof(float), p->stream));
    auto rebuild = [&](int nl) -> hb_status {
        if (precision == 0) HB_TRY(make_patchset<double>(p, p->ps64, p->tets_morton, budget, nl));
        else HB_TRY(make_patchset<float>(p, p->ps32, p->tets_morton, budget, nl));
        p->bc_dirty = true;                       // Dirichlet lists follow the new patches
        return prepare_bc(p);
    };
    const int n_var = precision == 0 ? 1 : kJvpVariants;
    int bvar = 0;
    for (int c = 0; c < n_cand; ++c) {
        const int nl = candidates[c];
        bool fits = nl >= 8 && nl <= 255;
        for (int m = 0; m < 4 && fits; ++m) fits = elem_smem_bytes(m, p->N, nl, 3 * nl, ts) <= 227 * 1024;
        if (!fits) continue;
        HB_TRY(rebuild(nl));
        for (int var = 0; var < n_var; ++var) {
            p->jvp_variant = var;
            double ms = 0;
            const bool was = p->prof_on;
            p->prof_on = true;
            double tmp = 0;
            int64_t cnt = 0;
            HB_TRY(hb_profile_read(p, &tmp, &cnt));
            for (int r = 0; r < reps + 1; ++r) {
                if (precision == 0)
                    HB_TRY(apply_op<double>(p, MODE_JVP, p->w64a.p, p->w64b.p, p->kres.p, 0.0, p->stream));
                else HB_TRY(apply_op<float>(p, MODE_JVP, p->w32a.p, p->w32c.p, p->w32b.p, 0.0, p->stream));
                if (r == 0) HB_TRY(hb_profile_read(p, &tmp, &cnt));   // drop the first (cold) launch
            }
            HB_TRY(hb_profile_read(p, &ms, &cnt));
            p->prof_on = was;
            ms /= double(std::max<int64_t>(1, cnt));
            if (ms < best) {
                best = ms;
                bnl = nl;
                bvar = var;
            }
        }
    }
    p->jvp_variant = precision == 0 ? p->jvp_variant : bvar;
    if (bnl == 0) return fail(HB_ERR_INVALID_ARG, "no candidate fits the shared-memory budget");
    HB_TRY(rebuild(bnl));
    if (best_nl) *best_nl = bnl;
    if (best_ms) *best_ms = best;
    return HB_OK;
}

hb_status hb_get_info(hb_problem *p, hb_info *info) {
    if (!p || !info) return fail(HB_ERR_INVALID_ARG, "null argument");
    HB_TRY(prepare_bc(p));
    info->n_nodes = p->n_nodes;
    info->n_tets = p->n_tets;
    info->n_faces = p->n_faces;
    info->n_dirichlet_nodes = p->n_dir;
    info->n_neumann_faces = p->n_nf;
    info->n_h = p->n_h;
    info->N = p->N;
    info->n_patches32 = p->ps32.P;
    info->n_patches64 = p->ps64.P;
    info->patch_nodes_max32 = p->ps32.nl_max;
    info->patch_elems_max32 = p->ps32.ep_max;
    info->device_bytes = p->dev_bytes;
    info->h_char = h_char(p);
    info->u_ref = p->u_c;
    double pr = 0;
    for (double v : p->level) pr += v / double(std::max<size_t>(1, p->level.size()));
    info->p_ref = pr;
    info->assembled_pairs = p->as.nnz;
    return HB_OK;
}

int64_t hb_launch_count(const hb_problem *p) { return p ? p->launches : 0; }

hb_status hb_set_stabilization(hb_problem *p, int variant, double ct_dt) {
    if (!p) return fail(HB_ERR_INVALID_ARG, "null problem");
    if (variant != 0 && variant != 1) return fail(HB_ERR_INVALID_ARG, "variant must be 0 (GLS) or 1 (full RBVMS)");
    if (!(ct_dt >= 0) || !std::isfinite(ct_dt)) return fail(HB_ERR_INVALID_ARG, "ct_dt must be finite and >= 0");
    cudaSetDevice(p->device);
    if (p->stream) cudaStreamSynchronize(p->stream);
    p->stab = variant;
    p->ct_dt = ct_dt;
    ++p->gen;
    // captured GMRES cycles hold the old kernel arguments; assembled coefficients hold the old tau
    for (auto &gc : p->cycle) {
        if (gc.exec) cudaGraphExecDestroy(gc.exec);
        gc = hb_problem::CycleGraph{};
    }
    p->as.ready32 = p->as.ready64 = false;
    return HB_OK;
}

hb_status hb_set_scatter(hb_problem *p, int scatter) {
    if (!p) return fail(HB_ERR_INVALID_ARG, "null problem");
    if (scatter != 0 && scatter != 1) return fail(HB_ERR_INVALID_ARG, "scatter must be 0 (deterministic) or 1 (atomic)");
    if (scatter == p->scatter) return HB_OK;
    cudaSetDevice(p->device);
    if (p->stream) cudaStreamSynchronize(p->stream);
    p->scatter = scatter;
    ++p->gen;
    for (auto &gc : p->cycle) {                   // captured cycles hold the old launches
        if (gc.exec) cudaGraphExecDestroy(gc.exec);
        gc = hb_problem::CycleGraph{};
    }
    // assembled values (and the multigrid levels' mass) were summed in the other order
    p->as.ready32 = p->as.ready64 = false;
    p->as.mass32_done = p->as.mass64_done = false;
    p->amg_mass32 = p->amg_mass64 = false;
    return HB_OK;
}

int hb_get_scatter(const hb_problem *p) { return p ? p->scatter : -1; }

hb_status hb_set_spectral_path(hb_problem *p, int path) {
    if (!p) return fail(HB_ERR_INVALID_ARG, "null problem");
    if (path < 0 || path > 2) return fail(HB_ERR_INVALID_ARG, "path must be 0 (tcgen05), 1 (mma.sync) or 2 (FMA)");
    if (path != p->spectral_path) ++p->gen;
    p->spectral_path = path;
    for (auto &gc : p->cycle) {                   // captured cycles hold the old launch
        if (gc.exec) cudaGraphExecDestroy(gc.exec);
        gc = hb_problem::CycleGraph{};
    }
    return HB_OK;
}

int hb_get_spectral_path(const hb_problem *p) { return p ? p->spectral_path : -1; }

hb_status hb_set_launch_variant(hb_problem *p, int variant) {
    if (!p) return fail(HB_ERR_INVALID_ARG, "null problem");
    if (variant < 0 || variant >= kJvpVariants) return fail(HB_ERR_INVALID_ARG, "unknown launch variant");
    if (variant != p->jvp_variant) ++p->gen;
    p->jvp_variant = variant;
    return HB_OK;
}

int hb_get_launch_variant(const hb_problem *p) { return p ? p->jvp_variant : -1; }

hb_status hb_profile_elem(hb_problem *p, int enable) {
    if (!p) return fail(HB_ERR_INVALID_ARG, "null problem");
    p->prof_on = enable != 0;
    return HB_OK;
}

hb_status hb_profile_read(hb_problem *p, double *ms, int64_t *launches) {
    if (!p || !ms || !launches) return fail(HB_ERR_INVALID_ARG, "null argument");
    HB_CUDA(cudaSetDevice(p->device));
    double total = 0;
    for (size_t i = 0; i < p->prof_used; ++i) {
        HB_CUDA(cudaEventSynchronize(p->prof_ev[i].second));
        float t = 0;
        HB_CUDA(cudaEventElapsedTime(&t, p->prof_ev[i].first, p->prof_ev[i].second));
        total += t;
    }
    *ms = total;
    *launches = int64_t(p->prof_used);
    p->prof_used = 0;
    return HB_OK;
}

}  // extern "C"
