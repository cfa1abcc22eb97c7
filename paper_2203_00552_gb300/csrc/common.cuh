// common.cuh -- context, error plumbing and device math shared by the ddLPB kernels.
//
// Method: Jha, Nottoli, Mikhalev, Quan, Stamm, arXiv:2203.00552 (ddLPB energy and
// forces).  Section / equation names below refer to that paper.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "ddlpb.h"

#define DDLPB_LMAX_MAX 16
#define DDLPB_FMM_PMAX 21               // highest FMM expansion order (J of degree p in shared memory)
#define DDLPB_LT 32                     // row stride of the (l, m) coefficient tables (degrees <= 31)
#define DDLPB_TCHUNK 512                // hits per CTA of the transposed A/B product

// ---------------------------------------------------------------------------
// Tables of the real spherical-harmonic recurrence (Sec. 2.2, Eq. definition_ylm).
// Y_lm = sqrt(2) Q_l^m(z) Re (x+iy)^m, Y_l-m = sqrt(2) Q_l^m(z) Im (x+iy)^m,
// Y_l0 = Q_l^0(z), with Q_l^m = P~_l^m / sin^m(theta) the fully normalised
// associated Legendre function (no Condon-Shortley phase) divided by sin^m.
//   Q_m^m     = qmm[m]
//   Q_{m+1}^m = q1[m] z Q_m^m
//   Q_l^m     = a[l][m] (z Q_{l-1}^m - b[l][m] Q_{l-2}^m)
// kr[l] = 1/((2l+1)(2l-1)) drives the scaled k_l recurrence, si[l] the series of
// the scaled i_l.
template <typename T>
struct YTabT {
    const T* a;     // [DDLPB_LT * DDLPB_LT]
    const T* b;
    const T* qmm;   // [DDLPB_LT]
    const T* q1;    // [DDLPB_LT]
};
using YTab = YTabT<double>;

template <typename T> struct V4T;
template <> struct V4T<double> { using type = double4; };
template <> struct V4T<float> { using type = float4; };

// Tables and scratch of the matrix-free operators in one arithmetic type T
// (double: the FP64 path; float: the inner solves of the mixed-precision form).
// Positions of the float set are taken relative to the centroid of the solute.
template <typename T>
struct OpSet {
    using V4 = typename V4T<T>::type;
    bool ready = false;
    V4* sph = nullptr;      // [M] centre, radius
    V4* leb = nullptr;      // [N] s_n, w_n
    T* Y = nullptr;         // [N][nb]
    T* YT = nullptr;        // [nb][N]
    T* ytab = nullptr;
    YTabT<T> yt{};
    T* Sinv = nullptr;      // [M][lmax+2]
    T* Khinv = nullptr;     // [M][lmax+2]
    T* di = nullptr;        // [M][lmax+1]
    T* cik = nullptr;       // [M][lmax+1]
    T* hit_w = nullptr;     // [H]
    T* thit_w = nullptr;    // [H]
    V4* ext_x = nullptr;    // [E] position, chi
    T* mu = nullptr;        // [M][nb] scratch
    T* extA = nullptr;      // [E] scratch
    T* gridA = nullptr;     // [M*N] scratch
    T* gridB = nullptr;     // [M*N] scratch
    T* acc = nullptr;       // [2*M*nb] scratch of the transposed A/B product
    // stored basis of the forward A/B product (built on its first use)
    bool stored = false, store_tried = false;
    int nbp = 0;            // nb rounded up to a multiple of 32
    T* Bp = nullptr;        // [nb][H]   omega r^l Y; within a sphere, hits ordered by (neighbour, point)
    T* Rp = nullptr;        // [L+1][H]  i-ratio corrections, same order
    int* hps = nullptr;     // [H] point index of the stored hit
    int* hjs = nullptr;     // [H] neighbour sphere of the stored hit
    // Chunk layout of the stored basis (FP32 set): the target-major hit list cut into chunks
    // of one neighbour, each padded to whole groups of 8 hits, coefficient-major [lm][8 G8], so
    // that one load holds one basis function at 8 hits of one neighbour.  Two copies: FP32
    // (the outer products, both directions) and FP16 (the preconditioner's inner solves).
    bool chunk_tried = false, chunk_ready = false;
    long long G8 = 0;         // groups of 8 hits
    long long* tpos = nullptr;  // [H] storage position of each entry of the target-major list
    int* hp8 = nullptr;       // [8 G8] point index, -1 in the padding
    int* gj = nullptr;        // [G8] neighbour sphere of the group
    int* cg0 = nullptr;       // [n_chunks] first group of the chunk
    int* cng = nullptr;       // [n_chunks] groups in the chunk
    float* Bc = nullptr;      // [nb][8 G8]   FP32 copy
    float* Rc = nullptr;      // [L+1][8 G8]
    __half* Bh = nullptr;     // [nb][8 G8]   FP16 copy
    __half* Rh = nullptr;     // [L+1][8 G8]
};

// Tree and interaction lists of the Yukawa FMM (Appendix), built at setup when fmm_order > 0.
// Nodes are numbered level by level (the root is 0; the children of a node are child0 and
// child0 + 1); every leaf holds one sphere.  The M2L list is sorted by target node and cut into
// chunks of at most DDLPB_FMM_CHUNK translations (work items whose partial sums are added per
// target in a fixed order); a second view sorts it by source node for the transposed pass.
#define DDLPB_FMM_CHUNK 16
struct FmmTree {
    bool on = false;
    int p = 0, q = 0;                 // expansion order; degree of the leaf multipoles (min(p, lmax + 1))
    double theta = 0.4;
    int n_nodes = 0, depth = 0;
    std::vector<int> lev;             // host: first node of each level, lev[depth + 1] = n_nodes
    std::vector<int> host_child0;     // host copy of child0 (internal nodes per level)
    int* order = nullptr;             // [M] spheres in Morton order
    int* node_a = nullptr;            // [n_nodes] range of the sorted list
    int* node_b = nullptr;
    int* parent = nullptr;            // [n_nodes], -1 at the root
    int* child0 = nullptr;            // [n_nodes], -1 at a leaf
    int* leaf_sphere = nullptr;       // [n_nodes], -1 at an internal node
    int* leaf_node = nullptr;         // [M]
    double4* node_g = nullptr;        // [n_nodes] centre c, scale radius Rt
    double* node_Rs = nullptr;        // [n_nodes] source radius
    int n_m2l = 0;
    int* m2l_t = nullptr;             // [n_m2l] target node (sorted)
    int* m2l_s = nullptr;             // [n_m2l] source node
    long long* m2l_off = nullptr;     // [n_m2l] coaxial block of the translation
    int n_ck = 0;
    int* ck_b = nullptr;              // [n_ck] chunk [ck_b, ck_e) of the target-sorted list
    int* ck_e = nullptr;
    int* tck_ptr = nullptr;           // [n_nodes + 1] chunks of target node k
    int* m2lT_k = nullptr;            // [n_m2l] the list sorted by source node (indices into the above)
    int n_ckT = 0;
    int* ckT_b = nullptr;             // [n_ckT] chunk of the source-sorted view
    int* ckT_e = nullptr;
    int* sck_ptr = nullptr;           // [n_nodes + 1] chunks of source node k
    long long* m2m_off = nullptr;     // [n_nodes] coaxial block of M2M(node -> parent)
    long long* l2l_off = nullptr;     // [n_nodes] coaxial block of L2L(parent -> node)
    long long* coax_off = nullptr;    // [n_m2l + 2 n_nodes] the three offset arrays above, contiguous
    long long coax_size = 0;
    int n_near = 0;
    int* near_ptr = nullptr;          // [M + 1] near sources of target sphere i (leaf pairs, not admissible)
    int* near_j = nullptr;
    int* nearT_ptr = nullptr;         // [M + 1] near targets of source sphere j
    int* nearT_i = nullptr;
};

// Per-precision data of the FMM: stored coaxial blocks, rotation table, Y_lm table to degree p
// and the expansion buffers (translation vectors are always formed from the FP64 node centres).
template <typename T>
struct FmmOps {
    using V4 = typename V4T<T>::type;
    bool ready = false;
    T* coax = nullptr;        // [coax_size] coaxial translation blocks
    T* JP = nullptr;          // rotation about x by -90 degrees, degree blocks padded to multiples of 4
    long long jpsize = 0;
    int* btab = nullptr;      // integer tables of the batched translations (degree offsets, work items)
    T* Yp = nullptr;          // [N][(p+1)^2] Y_lm(s_n), l <= p
    T* Mx = nullptr;          // [n_nodes][(p+1)^2] multipoles (transposed pass: their adjoints)
    T* Lx = nullptr;          // [n_nodes][(p+1)^2] locals (transposed pass: their adjoints)
    T* part = nullptr;        // [max(n_ck, n_ckT)][(p+1)^2] partial sums of the chunks
    T* leafq = nullptr;       // [M][(q+1)^2] adjoint of the leaf multipoles to degree q
    double* grad = nullptr;   // gradient map of the real basis (fmm_host.h), FP64 set only
    long long* grad_off = nullptr;
};

// Scratch of the force assembly, allocated on the first ddlpb_forces call.
struct ForceScratch {
    bool ready = false;
    double *xir = nullptr, *xie = nullptr, *UA = nullptr, *UB = nullptr, *ch = nullptr, *Ft = nullptr;
    double *G = nullptr, *muC = nullptr, *nu = nullptr, *muc = nullptr;
    double4* fs = nullptr;
    int* extpos = nullptr;
};

// Per-kernel launch timing (CUDA events on the context's stream), enabled by
// ddlpb_options.kernel_timing.
struct KernelTimes {
    std::vector<cudaEvent_t> ev;  // start, end pairs not yet read
    long long launches = 0;
    double ms = 0.0;
};

struct ddlpb_ctx {
    // problem
    int M = 0, lmax = 0, nb = 0, N = 0, degree = 0;
    double eps1 = 1.0, eps2 = 78.54, kappa = 0.0, eta = 0.1;
    ddlpb_options opt{};
    cudaStream_t stream = nullptr;
    int device = 0;
    std::string err;
    bool solved = false, adjoint_done = false;
    bool X_zero = true, Xa_zero = true;   // solution vectors still all zero (skip the first residual matvec)
    ddlpb_info info{};
    std::vector<void*> allocs;

    // geometry / tables (device)
    double4* sph = nullptr;     // [M] x y z r (cavity radius)
    double* q = nullptr;        // [M]
    double4* leb = nullptr;     // [N] s_n, w_n
    double* Y = nullptr;        // [N][nb]   Y_lm(s_n)
    double* YT = nullptr;       // [nb][N]
    double* ytab = nullptr;     // a | b | qmm | q1
    YTab yt{};
    double* Sinv = nullptr;     // [M][lmax+2] 1 / S_l(kappa r_j) (scaled i_l)
    double* Khinv = nullptr;    // [M][lmax+2] 1 / khat_l(kappa r_j) (scaled k_l)
    double* di = nullptr;       // [M][lmax+1] i_l'(r_j)/i_l(r_j)
    double* dk = nullptr;       // [M][lmax+1] k_l'(r_j)/k_l(r_j)
    double* cik = nullptr;      // [M][lmax+1] C_ik^j(l)
    int* nbr_ptr = nullptr;     // [M+1]
    int* nbr_idx = nullptr;
    long long n_pairs = 0;
    double* fval = nullptr;     // [M*N] f^i(x_i^n)
    double* chi = nullptr;      // [M*N] chi_i^eta(x_i^n)
    int* hit_ptr = nullptr;     // [M*N+1]
    int* hit_j = nullptr;       // [H]
    double* hit_w = nullptr;    // [H] omega_ij^eta(x_i^n)
    int* hit_p = nullptr;       // [H] point index i*N+n of the hit
    unsigned short* hit_s = nullptr;  // [H] slot of j in the neighbour list of i
    int* thit_ptr = nullptr;    // [M+1] hits grouped by the sphere j they point at
    int* thit_p = nullptr;      // [H] point index i*N+n
    int* thit_h = nullptr;      // [H] index of the hit in the point-major list
    double* thit_w = nullptr;   // [H]
    long long H = 0;
    int* chunk_j = nullptr;     // transposed hit list cut into chunks of at most DDLPB_TCHUNK hits:
    int* chunk_t0 = nullptr;    // target sphere, first position, count
    int* chunk_cnt = nullptr;
    int n_chunks = 0;
    int* ext_ptr = nullptr;     // [M+1] external points grouped by sphere
    int* ext_p = nullptr;       // [E] point index i*N+n
    double4* ext_x = nullptr;   // [E] position and chi
    int E = 0;
    int* src = nullptr;         // spheres with at least one external point
    int n_src = 0;

    // right-hand side and solutions (device), vectors of length nvec = 2*M*nb
    long long nvec = 0;
    double* g = nullptr;
    double* X = nullptr;
    double* Xa = nullptr;
    double* Qv = nullptr;
    double* psi0 = nullptr;     // [E] psi_0 at external points
    double* dnpsi0 = nullptr;   // [E] d_n psi_0 at external points
    double* mu0 = nullptr;      // [M][nb] C_ik C0 (multipoles of F0)
    double* S0 = nullptr;       // [E] potential of mu0 at external points

    // scratch
    void* solver = nullptr;     // Krylov workspaces (solve.cu)
    std::vector<double*> host_bufs;  // host mirrors of the Krylov scalars
    double* mu = nullptr;       // [M][nb]
    double* gridA = nullptr;    // [M*N]
    double* gridB = nullptr;    // [M*N]
    double* extA = nullptr;     // [E]
    double* extB = nullptr;     // [E]
    double* tmpv = nullptr;     // [nvec]
    double* force_acc = nullptr;
    ForceScratch fscr;
    FmmTree fmm;                // Yukawa FMM (fmm_order > 0)
    FmmOps<double> fmm64;
    FmmOps<float> fmm32;
    OpSet<double> d64;          // aliases the double tables above
    OpSet<float> f32;           // built on first use by the mixed-precision solve
    double centroid[3] = {0, 0, 0};
    std::map<std::string, KernelTimes> ktimes;
    int timer_block = 0;        // open group timers (KernelTimer)
    float* f32_vec = nullptr;   // FP32 Krylov workspace
};

// ---------------------------------------------------------------------------
// Error plumbing
#define DDLPB_CK(ctx, call)                                                        \
    do {                                                                           \
        cudaError_t e__ = (call);                                                  \
        if (e__ != cudaSuccess) {                                                  \
            (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e__);      \
            return DDLPB_ECUDA;                                                    \
        }                                                                          \
    } while (0)

#define DDLPB_LAUNCHED(ctx, name)                                                  \
    do {                                                                           \
        ++(ctx)->info.kernel_launches;                                             \
        cudaError_t e__ = cudaGetLastError();                                      \
        if (e__ != cudaSuccess) {                                                  \
            (ctx)->err = std::string("launch ") + (name) + ": " + cudaGetErrorString(e__); \
            return DDLPB_ECUDA;                                                    \
        }                                                                          \
    } while (0)

#define DDLPB_TRY(x)                                                               \
    do {                                                                           \
        ddlpb_status s__ = (x);                                                    \
        if (s__ != DDLPB_OK) return s__;                                           \
    } while (0)

template <typename T>
static ddlpb_status ctx_alloc(ddlpb_ctx* c, T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    // stream-ordered: no device-wide synchronisation, so contexts on other streams keep running
    cudaError_t e = cudaMallocAsync((void**)p, count * sizeof(T), c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->err = std::string("cudaMallocAsync of ") + std::to_string(count * sizeof(T)) + " bytes: " +
                 cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? DDLPB_ENOMEM : DDLPB_ECUDA;
    }
    c->allocs.push_back((void*)*p);
    return DDLPB_OK;
}

static inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// Event pair around one launch when kernel timing is on.
struct KernelTimer {
    ddlpb_ctx* c;
    cudaEvent_t e1 = nullptr;
    bool group = false;
    // level 1: the hot kernels (kernel_timing >= 1); level 2: every other group of launches
    // (kernel_timing >= 2), for a full breakdown of a step.  A group timer (setup, forces)
    // suppresses the timers nested in it, so that the recorded times add up.
    KernelTimer(ddlpb_ctx* ctx, const char* name, bool fp32, int level = 1, bool grp = false)
        : KernelTimer(ctx, std::string(name) + (fp32 ? "_f32" : "_f64"), level, grp) {}
    KernelTimer(ddlpb_ctx* ctx, const std::string& full_name, int level = 1, bool grp = false) : c(ctx) {
        if (c->opt.kernel_timing < level || c->timer_block > 0) return;
        cudaEvent_t e0;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            e1 = nullptr;
            return;
        }
        KernelTimes& k = c->ktimes[full_name];
        k.ev.push_back(e0);
        k.ev.push_back(e1);
        cudaEventRecord(e0, c->stream);
        if (grp) {
            group = true;
            ++c->timer_block;
        }
    }
    ~KernelTimer() {
        if (e1) cudaEventRecord(e1, c->stream);
        if (group) --c->timer_block;
    }
};

// ---------------------------------------------------------------------------
// Device math.

// Stream all Y_lm(u), u = (x, y, z) a unit vector, calling f(idx, l, Y).
template <typename T, typename F>
__device__ __forceinline__ void ylm_stream(int lmax, T x, T y, T z, const YTabT<T>& yt, F&& f) {
    const T SQ2 = (T)1.4142135623730951;
    T cr = 1, ci = 0;
    for (int m = 0; m <= lmax; ++m) {
        if (m > 0) {
            T nr = cr * x - ci * y;
            ci = cr * y + ci * x;
            cr = nr;
        }
        T q0 = (T)__ldg(yt.qmm + m);
        T sr = SQ2 * cr, si = SQ2 * ci;
        if (m == 0) {
            f(0, 0, q0);
        } else {
            f(m * m + 2 * m, m, q0 * sr);
            f(m * m, m, q0 * si);
        }
        if (m + 1 <= lmax) {
            T q1 = (T)__ldg(yt.q1 + m) * z * q0;
            int l = m + 1;
            if (m == 0) f(l * l + l, l, q1);
            else { f(l * l + l + m, l, q1 * sr); f(l * l + l - m, l, q1 * si); }
            for (l = m + 2; l <= lmax; ++l) {
                T q2 = (T)__ldg(yt.a + l * DDLPB_LT + m) * (z * q1 - (T)__ldg(yt.b + l * DDLPB_LT + m) * q0);
                q0 = q1;
                q1 = q2;
                if (m == 0) f(l * l + l, l, q2);
                else { f(l * l + l + m, l, q2 * sr); f(l * l + l - m, l, q2 * si); }
            }
        }
    }
}

// Stream Y_lm at two unit vectors u0, u1 at once, calling f(idx, l, Y(u0), Y(u1)).
template <typename T, typename F>
__device__ __forceinline__ void ylm_stream2(int lmax, T x0, T y0, T z0, T x1, T y1, T z1, const YTabT<T>& yt,
                                            F&& f) {
    const T SQ2 = (T)1.4142135623730951;
    T cr0 = 1, ci0 = 0, cr1 = 1, ci1 = 0;
    for (int m = 0; m <= lmax; ++m) {
        if (m > 0) {
            T n0 = cr0 * x0 - ci0 * y0;
            ci0 = cr0 * y0 + ci0 * x0;
            cr0 = n0;
            T n1 = cr1 * x1 - ci1 * y1;
            ci1 = cr1 * y1 + ci1 * x1;
            cr1 = n1;
        }
        const T qmm = (T)__ldg(yt.qmm + m);
        T p0 = qmm, p1 = qmm;
        const T sr0 = SQ2 * cr0, si0 = SQ2 * ci0, sr1 = SQ2 * cr1, si1 = SQ2 * ci1;
        if (m == 0) {
            f(0, 0, p0, p1);
        } else {
            f(m * m + 2 * m, m, p0 * sr0, p1 * sr1);
            f(m * m, m, p0 * si0, p1 * si1);
        }
        if (m + 1 <= lmax) {
            const T c1 = (T)__ldg(yt.q1 + m);
            T q0 = c1 * z0 * p0, q1 = c1 * z1 * p1;
            int l = m + 1;
            if (m == 0) f(l * l + l, l, q0, q1);
            else { f(l * l + l + m, l, q0 * sr0, q1 * sr1); f(l * l + l - m, l, q0 * si0, q1 * si1); }
            for (l = m + 2; l <= lmax; ++l) {
                const T a = (T)__ldg(yt.a + l * DDLPB_LT + m), bb = (T)__ldg(yt.b + l * DDLPB_LT + m);
                T r0 = a * (z0 * q0 - bb * p0), r1 = a * (z1 * q1 - bb * p1);
                p0 = q0; q0 = r0;
                p1 = q1; q1 = r1;
                if (m == 0) f(l * l + l, l, r0, r1);
                else { f(l * l + l + m, l, r0 * sr0, r1 * sr1); f(l * l + l - m, l, r0 * si0, r1 * si1); }
            }
        }
    }
}

// Stream Y_lm(u) and the ambient gradient G of F(x,y,z) = Q_l^m(z) C_m(x,y),
// whose tangential projection G - (u.G) u is the surface gradient of Y_lm at u
// (used for Eq. derivative_ylm).  Calls f(idx, l, Y, Gx, Gy, Gz).
template <typename T, typename F>
__device__ __forceinline__ void ylm_grad_stream(int lmax, T x, T y, T z, const YTabT<T>& yt, F&& f) {
    const T SQ2 = (T)1.4142135623730951;
    T cr = 1, ci = 0, pr = 0, pi = 0;  // w^m, w^(m-1), w = x + i y
    for (int m = 0; m <= lmax; ++m) {
        if (m > 0) {
            pr = cr;
            pi = ci;
            T nr = cr * x - ci * y;
            ci = cr * y + ci * x;
            cr = nr;
        }
        T fm = (T)m;
        // d/dx Re w^m = m Re w^(m-1), d/dy Re w^m = -m Im w^(m-1)
        // d/dx Im w^m = m Im w^(m-1), d/dy Im w^m =  m Re w^(m-1)
        T q0 = (T)__ldg(yt.qmm + m), d0 = 0;
        auto emit = [&](int l, T q, T d) {
            if (m == 0) {
                f(l * l + l, l, q, (T)0, (T)0, d);
            } else {
                f(l * l + l + m, l, SQ2 * q * cr, SQ2 * q * fm * pr, -SQ2 * q * fm * pi, SQ2 * d * cr);
                f(l * l + l - m, l, SQ2 * q * ci, SQ2 * q * fm * pi, SQ2 * q * fm * pr, SQ2 * d * ci);
            }
        };
        emit(m, q0, d0);
        if (m + 1 <= lmax) {
            T c1 = (T)__ldg(yt.q1 + m);
            T q1 = c1 * z * q0, d1 = c1 * q0;
            emit(m + 1, q1, d1);
            for (int l = m + 2; l <= lmax; ++l) {
                T a = (T)__ldg(yt.a + l * DDLPB_LT + m), b = (T)__ldg(yt.b + l * DDLPB_LT + m);
                T q2 = a * (z * q1 - b * q0);
                T d2 = a * (q1 + z * d1 - b * d0);
                q0 = q1; q1 = q2;
                d0 = d1; d1 = d2;
                emit(l, q2, d2);
            }
        }
    }
}

// Scaled modified spherical Bessel function of the first kind,
//   S_l(x) = (2l+1)!! i_l(x) / x^l = sum_k (x^2/2)^k (2l+1)!! / (k! (2l+2k+1)!!),
// a series of positive terms (stable for every x >= 0).
template <typename T>
__device__ __forceinline__ T scaled_i_series(int l, T x) {
    T h = (T)0.5 * x * x, t = 1, s = 1;
    const T eps = sizeof(T) == 8 ? (T)1e-17 : (T)3e-8;
    for (int k = 1; k < 400; ++k) {
        t *= h / (T)(k * (2 * l + 2 * k + 1));
        s += t;
        if (t < eps * s) break;
    }
    return s;
}

// Radial factors of the three bases of Sec. 2.2 at distance rho from centre j
// (radius rj), for l = 0..lmax, written to rad[l*stride] (and their rho-
// derivatives to drad[l*stride] when drad != nullptr):
//   kind 0: r_l^j       = (rho/rj)^l                                      (Eq. definition_radial_scaling)
//   kind 1: i_l ratio   = i_l(kappa rho)/i_l(kappa rj)                     (Eq. definition_of_bessel_func_first)
//           = (rho/rj)^l S_l(kappa rho) / S_l(kappa rj)
//   kind 2: k_l ratio   = k_l(kappa rho)/k_l(kappa rj)                     (Eq. definition_of_bessel_func_second)
//           = exp(-kappa(rho - rj)) (rj/rho)^(l+1) khat_l(kappa rho)/khat_l(kappa rj),
//           khat_0 = 1, khat_1 = 1 + x, khat_{l+1} = khat_l + x^2 khat_{l-1} / ((2l+1)(2l-1)).
// inv_tab holds 1/S_l(kappa rj) (kind 1) or 1/khat_l(kappa rj) (kind 2), l = 0..lmax+1.
template <typename T>
__device__ __forceinline__ void radial(int kind, int lmax, T rho, T rj, T kappa, const T* inv_tab,
                                       T* rad, T* drad, int stride) {
    if (kind == 0) {
        T s = rho / rj, v = 1;
        for (int l = 0; l <= lmax; ++l) {
            rad[l * stride] = v;
            if (drad) drad[l * stride] = (T)l * v / rho;
            v *= s;
        }
    } else if (kind == 1) {
        T x = kappa * rho, x2 = x * x;
        // downward recurrence S_{l-1} = S_l + x^2 S_{l+1} / ((2l+1)(2l+3)), from S_{L+2}, S_{L+1}
        int L = lmax;
        T s_hi = scaled_i_series<T>(L + 2, x);
        T s_mid = scaled_i_series<T>(L + 1, x);
        // rad[l] temporarily holds S_l(x)
        T sp1 = s_mid, sp2 = s_hi;
        for (int l = L; l >= 0; --l) {
            T sl = sp1 + x2 * sp2 / (T)((2 * l + 3) * (2 * l + 5));
            if (drad) drad[l * stride] = sp1 / sl;   // S_{l+1}/S_l
            rad[l * stride] = sl;
            sp2 = sp1;
            sp1 = sl;
        }
        T s = rho / rj, v = 1;
        for (int l = 0; l <= L; ++l) {
            T sl = rad[l * stride];
            T r = v * sl * inv_tab[l];
            rad[l * stride] = r;
            if (drad) drad[l * stride] = r * ((T)l / rho + kappa * kappa * rho / (T)(2 * l + 3) * drad[l * stride]);
            v *= s;
        }
    } else {
        T x = kappa * rho, x2 = x * x;
        T e = exp(-kappa * (rho - rj));
        T s = rj / rho, v = e * s;
        T k0 = 1, k1 = 1 + x;
        for (int l = 0; l <= lmax; ++l) {
            T kl = (l == 0) ? k0 : k1;
            T knext = (l == 0) ? k1 : k1 + x2 * k0 / (T)((2 * l + 1) * (2 * l - 1));
            T r = v * kl * inv_tab[l];
            rad[l * stride] = r;
            if (drad) drad[l * stride] = r * ((T)l - (T)(2 * l + 1) * knext / kl) / rho;
            if (l >= 1) { k0 = k1; k1 = knext; }
            v *= s;
        }
    }
}

// Smooth switch chi_eta(t) of Eq. regular_char_function, with the constant of p_eta
// read as 10 eta^2 - 15 eta + 6 (the only reading that makes chi_eta continuous).
__device__ __forceinline__ double chi_eta(double t, double eta) {
    if (t <= 1.0 - eta) return 1.0;
    if (t >= 1.0) return 0.0;
    double a = 1.0 - t;
    double ie = 1.0 / eta;
    double ie5 = ie * ie * ie * ie * ie;
    return ie5 * a * a * a * (6.0 * t * t + (15.0 * eta - 12.0) * t + 10.0 * eta * eta - 15.0 * eta + 6.0);
}

__device__ __forceinline__ double dchi_eta(double t, double eta) {
    if (t <= 1.0 - eta || t >= 1.0) return 0.0;
    double a = 1.0 - t;
    double ie = 1.0 / eta;
    double ie5 = ie * ie * ie * ie * ie;
    double poly = 6.0 * t * t + (15.0 * eta - 12.0) * t + 10.0 * eta * eta - 15.0 * eta + 6.0;
    double dpoly = 12.0 * t + 15.0 * eta - 12.0;
    return ie5 * (-3.0 * a * a * poly + a * a * a * dpoly);
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// Host-side internal entry points (defined across the .cu files).
template <typename T> ddlpb_status opset_prepare(ddlpb_ctx* c, OpSet<T>& S);
template <typename T> ddlpb_status op_apply_L_T(ddlpb_ctx* c, OpSet<T>& S, const T* x, T* y, bool transpose);
template <typename T>
ddlpb_status op_apply_AB_T(ddlpb_ctx* c, OpSet<T>& S, const T* x, T* y, bool transpose, T* gridR, T* gridE);
template <typename T> ddlpb_status op_apply_P_T(ddlpb_ctx* c, OpSet<T>& S, const T* x, T* y, bool transpose);
// The A/B operator of the preconditioner's inner solves: the FP16 stored basis for the FP32
// set when ddlpb_options.precond_fp16 is set, otherwise op_apply_AB_T.
template <typename T> ddlpb_status op_apply_AB_precond(ddlpb_ctx* c, OpSet<T>& S, const T* x, T* y, bool transpose);
ddlpb_status ddlpb_internal_setup(ddlpb_ctx* c, const double* centres, const double* radii,
                                  const double* charges, bool device_ptrs, int surface);
ddlpb_status op_apply_L(ddlpb_ctx* c, const double* x, double* y, bool transpose);
ddlpb_status op_apply_AB(ddlpb_ctx* c, const double* x, double* y, bool transpose, double* gridR,
                         double* gridE);
ddlpb_status op_apply_C(ddlpb_ctx* c, const double* x, double* y, bool transpose, bool accumulate);
ddlpb_status op_synthesis(ddlpb_ctx* c, const double* coef, int rows, double* grid, bool weighted);
ddlpb_status op_yukawa_potential(ddlpb_ctx* c, const double* mu, double* phi_ext);
ddlpb_status op_yukawa_adjoint(ddlpb_ctx* c, const double* c_ext, double* nu);
ddlpb_status op_masked_analysis(ddlpb_ctx* c, const double* val_ext, double scale, const double* cik_scale,
                                double* out, int out_stride, int accumulate);
ddlpb_status op_ext_weights(ddlpb_ctx* c, const double* x, double* cext);
ddlpb_status op_source_multipoles(ddlpb_ctx* c, const double* x, double* mu);
ddlpb_status solve_system(ddlpb_ctx* c, bool transpose, const double* b, double* x, int* iters,
                          double* resid);
ddlpb_status compute_forces(ddlpb_ctx* c, double* f_dev);
void solver_state_free(ddlpb_ctx* c);
ddlpb_status op_apply_fp32(ddlpb_ctx* c, int op, const double* x, double* y);
// Yukawa FMM (fmm.cu): tree and lists at setup; potential of the sphere multipoles mu at the
// external points (far field by the FMM, near pairs directly); its transpose.
ddlpb_status fmm_build(ddlpb_ctx* c, const double* host_centres);
template <typename T> ddlpb_status fmm_potential(ddlpb_ctx* c, OpSet<T>& S, const T* mu, T* phi_ext);
template <typename T> ddlpb_status fmm_adjoint(ddlpb_ctx* c, OpSet<T>& S, const T* c_ext, T* nu);
// Yukawa force terms with the FMM (target side added to Ft, source side to G); needs the
// transposed pass of the same c_t = fs[t].w to have run last.
ddlpb_status fmm_force_terms(ddlpb_ctx* c, const double* mu, const double4* fs, double* Ft, double* G);
