// fmm.cu -- fast multipole method for the Yukawa far field of the coupling C (Appendix of
// arXiv:2203.00552): the potential, at the external grid points, of the degree-lmax sphere
// multipoles mu_j (k-ratio basis k_l(kappa|x - x_j|)/k_l(kappa r_j) Y_lm), and its transpose.
//
// Tree (built on the device at setup): spheres sorted by the Morton key of their centres; a
// binary tree over the sorted list (node [a, b) splits at a + (b - a)/2) down to single-sphere
// leaves.  Node centre c = midpoint of the bounding box of its centres; Rs = max |x_j - c|
// (sources); Rt = max |x_j - c| + r_j (targets on the spheres), also the scale radius of the
// node's expansions; a leaf has c = x_j, Rs = 0, Rt = r_j.  A dual traversal from (root, root)
// emits an M2L for (target A, source B) when Rt_A + Rs_B < theta |c_A - c_B|, a near pair for
// two leaves that fail the test, and otherwise splits A if B is a leaf or (A is not a leaf and
// Rt_A >= Rs_B), else B.
//
// Expansions, order p: multipole sum M_lm k_l(kappa|x-c|)/k_l(kappa Rt) Y_lm, local
// sum L_lm i_l(kappa|x-c|)/i_l(kappa Rt) Y_lm.  A leaf's multipole is mu_j (degree lmax; the
// transposed pass returns it to degree q = lmax + 1 for the force gradients), and a leaf's
// local evaluated on its own sphere is sum L_lm Y_lm(s_n).
//
// Translations (M2M, M2L, L2L, the Appendix's OZ-axis scheme): rotate the expansion so that the
// translation vector is the z axis, translate along z (m is kept), rotate back.  Rotations use
// the cheap rotation about z and a fixed table J (the rotation about x by -90 degrees, degree by
// degree): a rotation about y by b is J Rz(b) J^T.  The coaxial coefficients come from the
// addition theorem of the modified spherical Bessel functions (Gaunt integrals times i_b or k_b
// of kappa t, b = l + a - 2j): for t = c_target - c_source along +z and input degree l, output a,
//   M2L: (-1)^a     sum_j g k_b(kappa t)  i_a(kappa Rt_T) / k_l(kappa Rt_S)
//   M2M: (-1)^(l+a) sum_j g i_b(kappa t)  k_a(kappa Rt_T) / k_l(kappa Rt_S)
//   L2L:            sum_j g i_b(kappa t)  i_a(kappa Rt_T) / i_l(kappa Rt_S)
// They are evaluated once per translation at setup in FP64 and stored in the precision of the
// operator set (HBM holds them easily); the rotations are applied on the fly, a batch of
// translations per CTA, with J in shared memory.
//
// Every pass gathers (a CTA per chunk of a target's M2L list, per group of tree nodes, or per
// leaf sphere; partial sums added in a fixed order), so the operator is deterministic: the
// mixed-precision refinement evaluates it repeatedly and needs the same rounding each time.
#include <cub/cub.cuh>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "fmm_host.h"


// ---------------------------------------------------------------- tree construction

// Morton key of each centre: 21 bits per coordinate, floor(2^21 (x - lo) / side) clamped,
// bits interleaved x, y, z from the most significant.
__global__ void k_fmm_morton(int M, const double4* __restrict__ sph, double lx, double ly, double lz, double side,
                             unsigned long long* __restrict__ key, int* __restrict__ idx) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    const double4 s = sph[j];
    const double lo[3] = {lx, ly, lz};
    const double v[3] = {s.x, s.y, s.z};
    unsigned long long q[3];
    for (int d = 0; d < 3; ++d) {
        double t = floor(__dmul_rn(__ddiv_rn(__dsub_rn(v[d], lo[d]), side), 2097152.0));
        if (t > 2097151.0) t = 2097151.0;
        if (t < 0.0) t = 0.0;
        q[d] = (unsigned long long)t;
    }
    unsigned long long k = 0;
    for (int b = 0; b < 21; ++b)
        for (int d = 0; d < 3; ++d) k |= ((q[d] >> b) & 1ULL) << (3 * b + (2 - d));
    key[j] = k;
    idx[j] = j;
}

// Node geometry (FP64, written without fused multiply-adds so that the admissibility tests
// round as the specification's plain arithmetic does).
__global__ void k_fmm_node_geom(int n_nodes, const int* __restrict__ na, const int* __restrict__ nb,
                                const int* __restrict__ order, const double4* __restrict__ sph,
                                double4* __restrict__ g, double* __restrict__ Rs, int* __restrict__ leaf_sphere,
                                int* __restrict__ leaf_node) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_nodes) return;
    const int a = na[k], b = nb[k];
    if (b - a == 1) {
        const int j = order[a];
        const double4 s = sph[j];
        g[k] = s;
        Rs[k] = 0.0;
        leaf_sphere[k] = j;
        leaf_node[j] = k;
        return;
    }
    leaf_sphere[k] = -1;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int u = a; u < b; ++u) {
        const double4 s = sph[order[u]];
        lo[0] = fmin(lo[0], s.x); hi[0] = fmax(hi[0], s.x);
        lo[1] = fmin(lo[1], s.y); hi[1] = fmax(hi[1], s.y);
        lo[2] = fmin(lo[2], s.z); hi[2] = fmax(hi[2], s.z);
    }
    const double cx = __dmul_rn(0.5, __dadd_rn(lo[0], hi[0]));
    const double cy = __dmul_rn(0.5, __dadd_rn(lo[1], hi[1]));
    const double cz = __dmul_rn(0.5, __dadd_rn(lo[2], hi[2]));
    double rs = 0.0, rt = 0.0;
    for (int u = a; u < b; ++u) {
        const double4 s = sph[order[u]];
        const double dx = __dsub_rn(s.x, cx), dy = __dsub_rn(s.y, cy), dz = __dsub_rn(s.z, cz);
        const double d = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
        rs = fmax(rs, d);
        rt = fmax(rt, __dadd_rn(d, s.w));
    }
    g[k] = make_double4(cx, cy, cz, rt);
    Rs[k] = rs;
}

// One level of the dual traversal: every pair (A, B) of the frontier becomes an M2L, a near
// pair, or two pairs of the next frontier.  Counters beyond a capacity are still counted (the
// host then enlarges the arrays and traverses again); nothing is written past a capacity.
__global__ void k_fmm_traverse(int n_front, const int2* __restrict__ front, const double4* __restrict__ g,
                               const double* __restrict__ Rs, const int* __restrict__ child0, double theta,
                               int2* __restrict__ next, int* __restrict__ n_next, int cap_next,
                               int2* __restrict__ m2l, int* __restrict__ n_m2l, int cap_m2l,
                               int2* __restrict__ near, int* __restrict__ n_near, int cap_near) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_front) return;
    const int A = front[k].x, B = front[k].y;
    const double4 ga = g[A], gb = g[B];
    const double dx = __dsub_rn(ga.x, gb.x), dy = __dsub_rn(ga.y, gb.y), dz = __dsub_rn(ga.z, gb.z);
    const double d = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
    if (__dadd_rn(ga.w, Rs[B]) < __dmul_rn(theta, d)) {
        const int u = atomicAdd(n_m2l, 1);
        if (u < cap_m2l) m2l[u] = make_int2(A, B);
        return;
    }
    const int ca = child0[A], cb = child0[B];
    if (ca < 0 && cb < 0) {
        const int u = atomicAdd(n_near, 1);
        if (u < cap_near) near[u] = make_int2(A, B);
        return;
    }
    const int u = atomicAdd(n_next, 2);
    int2 p0, p1;
    if (cb < 0 || (ca >= 0 && ga.w >= Rs[B])) {
        p0 = make_int2(ca, B);
        p1 = make_int2(ca + 1, B);
    } else {
        p0 = make_int2(A, cb);
        p1 = make_int2(A, cb + 1);
    }
    if (u + 1 < cap_next) {
        next[u] = p0;
        next[u + 1] = p1;
    }
}

// Segment starts of a sorted key array: ptr[k] = first position with key >= k, k = 0..K.
__global__ void k_fmm_seg_starts(int n, int K, const int* __restrict__ keys, int* __restrict__ ptr) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u > n) return;
    const int kp = u == 0 ? -1 : keys[u - 1];
    const int kc = u == n ? K : keys[u];
    for (int k = kp + 1; k <= kc; ++k) ptr[k] = u;
}

__global__ void k_fmm_split_pairs(int n, const int2* __restrict__ pr, int* __restrict__ a, int* __restrict__ b) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n) {
        a[u] = pr[u].x;
        b[u] = pr[u].y;
    }
}

// out[u] = k for the positions u of run k of a CSR (the key of every sorted entry).
__global__ void k_fmm_fill_keys(int K, const int* __restrict__ ptr, int* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    for (int u = ptr[k]; u < ptr[k + 1]; ++u) out[u] = k;
}

__global__ void k_fmm_iota(int n, int* __restrict__ v) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n) v[u] = u;
}

// Near pairs hold node ids; turn them into sphere ids.
__global__ void k_fmm_near_spheres(int n, const int* __restrict__ leaf_sphere, int* __restrict__ a,
                                   int* __restrict__ b) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n) {
        a[u] = leaf_sphere[a[u]];
        b[u] = leaf_sphere[b[u]];
    }
}

// Chunks of each node's run in a sorted list: count, then fill after the scan.
__global__ void k_fmm_chunk_count(int K, const int* __restrict__ ptr, int* __restrict__ cnt) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < K) cnt[k] = (ptr[k + 1] - ptr[k] + DDLPB_FMM_CHUNK - 1) / DDLPB_FMM_CHUNK;
}

__global__ void k_fmm_chunk_fill(int K, const int* __restrict__ ptr, const int* __restrict__ cpos,
                                 int* __restrict__ cb, int* __restrict__ ce) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    int c = cpos[k];
    for (int u = ptr[k]; u < ptr[k + 1]; u += DDLPB_FMM_CHUNK, ++c) {
        cb[c] = u;
        ce[c] = min(u + DDLPB_FMM_CHUNK, ptr[k + 1]);
    }
}

__device__ __forceinline__ long long coax_size_dev(int pin, int pout) {
    long long s = 0;
    for (int m = 0; m <= min(pin, pout); ++m) s += (long long)(pin + 1 - m) * (pout + 1 - m);
    return s;
}

// Sizes of the coaxial blocks: the M2L list, then M2M(k -> parent) and L2L(parent -> k) per node.
__global__ void k_fmm_coax_sizes(int n_m2l, int n_nodes, int p, int q, const int* __restrict__ m2l_s,
                                 const int* __restrict__ child0, const int* __restrict__ parent,
                                 long long* __restrict__ sz) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n_m2l) {
        sz[u] = coax_size_dev(child0[m2l_s[u]] < 0 ? q : p, p);
    } else if (u < n_m2l + n_nodes) {
        const int k = u - n_m2l;
        sz[u] = parent[k] < 0 ? 0 : coax_size_dev(child0[k] < 0 ? q : p, p);
    } else if (u < n_m2l + 2 * n_nodes) {
        const int k = u - n_m2l - n_nodes;
        sz[u] = parent[k] < 0 ? 0 : coax_size_dev(p, p);
    }
}

// Number of M2L translations whose source is a leaf (input degree q instead of p).
__global__ void k_fmm_count_leaf_src(int n, const int* __restrict__ m2l_s, const int* __restrict__ child0,
                                     int* __restrict__ cnt) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n && child0[m2l_s[u]] < 0) atomicAdd(cnt, 1);
}

__global__ void k_fmm_coax_offsets(int n_m2l, int n_nodes, const long long* __restrict__ off,
                                   long long* __restrict__ m2l_off, long long* __restrict__ m2m_off,
                                   long long* __restrict__ l2l_off) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n_m2l) m2l_off[u] = off[u];
    else if (u < n_m2l + n_nodes) m2m_off[u - n_m2l] = off[u];
    else if (u < n_m2l + 2 * n_nodes) l2l_off[u - n_m2l - n_nodes] = off[u];
}

// k_n(x), n = 0..n_max (k_0 = exp(-x)/x; only ratios and products with i enter the blocks).
__device__ void bessel_k_all(int n_max, double x, double* k) {
    const double e = exp(-x);
    k[0] = e / x;
    if (n_max >= 1) k[1] = e * (1.0 + x) / (x * x);
    for (int n = 1; n < n_max; ++n) k[n + 1] = k[n - 1] + (2.0 * n + 1.0) / x * k[n];
}

// i_n(x) = x^n S_n(x) / (2n+1)!!, n = 0..n_max (S_n the positive series, downward recurrence).
__device__ void bessel_i_all(int n_max, double x, double* v) {
    const double x2 = x * x;
    double s1 = scaled_i_series<double>(n_max + 1, x), s0 = scaled_i_series<double>(n_max, x);
    v[n_max] = s0;
    for (int n = n_max - 1; n >= 0; --n) {
        const double sn = s0 + x2 * s1 / (double)((2 * n + 3) * (2 * n + 5));
        s1 = s0;
        s0 = sn;
        v[n] = sn;
    }
    double f = 1.0;
    for (int n = 0; n <= n_max; ++n) {
        v[n] *= f;
        f *= x / (double)(2 * n + 3);
    }
}

// The coaxial block of translation u (one CTA): kind 0 M2L, 1 M2M, 2 L2L.
template <typename T>
__global__ void k_fmm_coax(int n_m2l, int n_nodes, int p, int q, double kappa, const int* __restrict__ m2l_t,
                           const int* __restrict__ m2l_s, const int* __restrict__ child0,
                           const int* __restrict__ parent, const double4* __restrict__ g,
                           const double* __restrict__ gtab, const long long* __restrict__ goff,
                           const long long* __restrict__ off, T* __restrict__ coax) {
    __shared__ double f[2 * DDLPB_FMM_PMAX + 2];
    __shared__ double so[DDLPB_FMM_PMAX + 2], si[DDLPB_FMM_PMAX + 2];
    const int u = blockIdx.x;
    int kind, S, Tn;
    if (u < n_m2l) {
        kind = 0;
        S = m2l_s[u];
        Tn = m2l_t[u];
    } else if (u < n_m2l + n_nodes) {
        kind = 1;
        S = u - n_m2l;
        Tn = parent[S];
    } else {
        kind = 2;
        Tn = u - n_m2l - n_nodes;
        S = parent[Tn];
    }
    if (S < 0 || Tn < 0) return;   // the root has no M2M / L2L
    const int pin = (kind != 2 && child0[S] < 0) ? q : p, pout = p;
    const double4 gs = g[S], gt = g[Tn];
    const double dx = gt.x - gs.x, dy = gt.y - gs.y, dz = gt.z - gs.z;
    const double t = sqrt(dx * dx + dy * dy + dz * dz);
    if (threadIdx.x == 0) {
        double tmp[2 * DDLPB_FMM_PMAX + 2];
        if (kind == 0) bessel_k_all(pin + pout, kappa * t, f);
        else bessel_i_all(pin + pout, kappa * t, f);
        // output scale (a <= pout) and input scale (l <= pin)
        if (kind == 1) bessel_k_all(pout, kappa * gt.w, tmp);
        else bessel_i_all(pout, kappa * gt.w, tmp);
        for (int a = 0; a <= pout; ++a) so[a] = tmp[a];
        if (kind == 2) bessel_i_all(pin, kappa * gs.w, tmp);
        else bessel_k_all(pin, kappa * gs.w, tmp);
        for (int l = 0; l <= pin; ++l) si[l] = 1.0 / tmp[l];
    }
    __syncthreads();
    const long long base = off[u];
    long long bo = 0;
    for (int m = 0; m <= min(pin, pout); ++m) {
        const int nl = pin + 1 - m, na = pout + 1 - m;
        for (int e = threadIdx.x; e < nl * na; e += blockDim.x) {
            const int l = m + e / na, a = m + e % na;
            const double* gg = gtab + goff[((size_t)m * (p + 1) + l) * (p + 1) + a];
            double s = 0.0;
            for (int j = 0; j <= min(l, a); ++j) s += gg[j] * f[l + a - 2 * j];
            double sign = 1.0;
            if (kind == 0 && (a & 1)) sign = -1.0;
            if (kind == 1 && ((l + a) & 1)) sign = -1.0;
            coax[base + bo + e] = (T)(sign * s * so[a] * si[l]);
        }
        bo += (long long)nl * na;
    }
}

// Y_lm(s_n) to degree p at the Lebedev points.
template <typename T>
__global__ void k_fmm_ytab(int N, int p, const double4* __restrict__ leb, YTab yt, T* __restrict__ Yp) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int nbp = (p + 1) * (p + 1);
    const double4 s = leb[n];
    ylm_stream<double>(p, s.x, s.y, s.z, yt, [&](int idx, int, double v) { Yp[(size_t)n * nbp + idx] = (T)v; });
}

__device__ __forceinline__ int deg_of(int idx) { return (int)sqrtf((float)idx + 0.5f); }

// ---------------------------------------------------------------- forward pass

// Leaf multipoles: the sphere multipoles mu_j (degree lmax), zero above.
template <typename T>
__global__ void k_fmm_leaf_mult(int M, int nb, int nbp, const int* __restrict__ leaf_node, const T* __restrict__ mu,
                                T* __restrict__ Mx) {
    const int j = blockIdx.x;
    T* out = Mx + (size_t)leaf_node[j] * nbp;
    for (int k = threadIdx.x; k < nbp; k += blockDim.x) out[k] = k < nb ? mu[(size_t)j * nb + k] : (T)0;
}

// Potential at the external points of target sphere i: the leaf local (sum L_lm Y_lm(s_n)) plus
// the near sources summed directly.  Offsets to the near sources are formed in FP64 and then
// rounded, so the FP32 set keeps full relative accuracy near the sources.
template <typename T, typename V4>
__global__ void k_fmm_leaf_pot(int N, int nb, int L, int p, T kappa, const int* __restrict__ ext_ptr,
                               const int* __restrict__ ext_p, const double4* __restrict__ sph64,
                               const double4* __restrict__ leb64, const int* __restrict__ leaf_node,
                               const T* __restrict__ Lx, const T* __restrict__ Yp, const int* __restrict__ near_ptr,
                               const int* __restrict__ near_j, const T* __restrict__ mu, const T* __restrict__ Khinv,
                               YTabT<T> yt, T* __restrict__ phi) {
    extern __shared__ unsigned char smraw[];
    const int bd = blockDim.x, tid = threadIdx.x;
    const int nbp = (p + 1) * (p + 1);
    T* Li = (T*)smraw;
    T* rad = Li + nbp;
    T* part = rad + (size_t)(L + 1) * bd;
    const int i = blockIdx.x;
    const int t0 = ext_ptr[i], cnt = ext_ptr[i + 1] - t0;
    if (cnt == 0) return;
    for (int k = tid; k < nbp; k += bd) Li[k] = Lx[(size_t)leaf_node[i] * nbp + k];
    const double4 a = sph64[i];
    const int k0 = near_ptr[i], k1 = near_ptr[i + 1];
    // S slices of the near sources per point (thread = point pi of the round, slice sl), partial
    // sums added in slice order
    const int S = max(1, min(bd / cnt, k1 - k0)), P = bd / S;
    const int pi = tid % P, sl = tid / P;
    for (int base = 0; base < cnt; base += P) {
        __syncthreads();
        const int t = t0 + base + pi;
        T v = 0;
        if (sl < S && base + pi < cnt) {
            const double4 sn = leb64[ext_p[t] % N];
            for (int kk = k0 + sl; kk < k1; kk += S) {
                const int j = near_j[kk];
                const double4 b = sph64[j];
                const T dx = (T)(a.x - b.x + a.w * sn.x), dy = (T)(a.y - b.y + a.w * sn.y),
                        dz = (T)(a.z - b.z + a.w * sn.z);
                const T rho = sqrt(dx * dx + dy * dy + dz * dz), inv = (T)1 / rho;
                radial<T>(2, L, rho, (T)b.w, kappa, Khinv + (size_t)j * (L + 2), rad + tid, nullptr, bd);
                const T* m = mu + (size_t)j * nb;
                T w = 0;
                ylm_stream<T>(L, dx * inv, dy * inv, dz * inv, yt,
                              [&](int idx, int l, T yv) { w += __ldg(m + idx) * rad[tid + l * bd] * yv; });
                v += w;
            }
        }
        part[tid] = v;
        __syncthreads();
        if (sl == 0 && base + pi < cnt) {
            const T* Y = Yp + (size_t)(ext_p[t] % N) * nbp;
            T acc = 0;
            for (int k = 0; k < nbp; ++k) acc += Li[k] * __ldg(Y + k);
            for (int q = 0; q < S; ++q) acc += part[q * P + pi];
            phi[t] = acc;
        }
    }
}

// ---------------------------------------------------------------- transposed pass

// Adjoint of the leaf locals: Lambda_i = sum_t c_t Y_lm(s_n) over the external points of i.
template <typename T>
__global__ void k_fmm_leaf_lambda(int N, int p, const int* __restrict__ ext_ptr, const int* __restrict__ ext_p,
                                  const int* __restrict__ leaf_node, const T* __restrict__ Yp,
                                  const T* __restrict__ cext, T* __restrict__ Lx) {
    extern __shared__ unsigned char smraw[];
    const int i = blockIdx.x;
    const int nbp = (p + 1) * (p + 1);
    const int t0 = ext_ptr[i], cnt = ext_ptr[i + 1] - t0;
    T* cv = (T*)smraw;
    int* nn = (int*)(cv + N);
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
        cv[k] = cext[t0 + k];
        nn[k] = ext_p[t0 + k] % N;
    }
    __syncthreads();
    T* out = Lx + (size_t)leaf_node[i] * nbp;
    for (int idx = threadIdx.x; idx < nbp; idx += blockDim.x) {
        T s = 0;
        for (int k = 0; k < cnt; ++k) s += cv[k] * Yp[(size_t)nn[k] * nbp + idx];
        out[idx] = s;
    }
}

// nu_j = (far adjoint of the leaf multipole, l <= lmax) + sum over the near targets t of
// sphere j's near list of c_t k-ratio basis of j at x_t.  Also keeps the far part to degree q.
// Spheres without external points are no sources of the coupling (P chi_j = 0): their rows of
// nu are left untouched (zero), since the forward pass reads every sphere's multipole.
template <typename T, typename V4>
__global__ void k_fmm_leaf_adj(int N, int nb, int L, int p, int q, T kappa, const int* __restrict__ ext_ptr,
                               const int* __restrict__ ext_p, const double4* __restrict__ sph64,
                               const double4* __restrict__ leb64, const int* __restrict__ leaf_node,
                               const T* __restrict__ Mx, const int* __restrict__ nearT_ptr,
                               const int* __restrict__ nearT_i, const T* __restrict__ cext,
                               const T* __restrict__ Khinv, YTabT<T> yt, T* __restrict__ nu, T* __restrict__ leafq) {
    extern __shared__ unsigned char smraw[];
    const int bd = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = bd >> 5;
    const int nbp = (p + 1) * (p + 1), nq = (q + 1) * (q + 1);
    T* acc = (T*)smraw;
    T* kh = acc + nw * nb;
    T* rad = kh + (L + 2);
    const int j = blockIdx.x;
    if (ext_ptr[j + 1] == ext_ptr[j]) return;
    const double4 b = sph64[j];
    for (int k = tid; k < nw * nb; k += bd) acc[k] = 0;
    for (int k = tid; k < L + 2; k += bd) kh[k] = Khinv[(size_t)j * (L + 2) + k];
    __syncthreads();
    // warp w takes the near targets w, w + nw, ... and its lanes their points, 32 at a time
    for (int kk = nearT_ptr[j] + warp; kk < nearT_ptr[j + 1]; kk += nw) {
        const int i = nearT_i[kk];
        const double4 a = sph64[i];
        const int t0 = ext_ptr[i], cnt = ext_ptr[i + 1] - t0;
        for (int base = 0; base < cnt; base += 32) {
            T dx = (T)b.w, dy = 0, dz = 0, c = 0;
            if (base + lane < cnt) {
                const int t = t0 + base + lane;
                const double4 s = leb64[ext_p[t] % N];
                dx = (T)(a.x - b.x + a.w * s.x);
                dy = (T)(a.y - b.y + a.w * s.y);
                dz = (T)(a.z - b.z + a.w * s.z);
                c = cext[t];
            }
            const T rho = sqrt(dx * dx + dy * dy + dz * dz), inv = (T)1 / rho;
            radial<T>(2, L, rho, (T)b.w, kappa, kh, rad + tid, nullptr, bd);
            ylm_stream<T>(L, dx * inv, dy * inv, dz * inv, yt, [&](int idx, int l, T yv) {
                const T v = warp_sum(c * rad[tid + l * bd] * yv);
                if (lane == 0) acc[warp * nb + idx] += v;
            });
        }
    }
    __syncthreads();
    const T* far = Mx + (size_t)leaf_node[j] * nbp;
    for (int idx = tid; idx < nb; idx += bd) {
        T s = far[idx];
        for (int w = 0; w < nw; ++w) s += acc[w * nb + idx];
        nu[(size_t)j * nb + idx] = s;
    }
    if (leafq)
        for (int idx = tid; idx < nq; idx += bd) leafq[(size_t)j * nq + idx] = far[idx];
}

// ---------------------------------------------------------------- batched translations
//
// A CTA translates TB expansions at a time (TB = 16 for the FP32 M2L chunks, 8 otherwise).  In
// shared memory an expansion is kept in a padded layout: degree l occupies n4 = 2l+1 rounded up
// to 4 slots from poff[l] (a multiple of 4), the padding held at zero, so that four consecutive
// coefficients are one vector load.  The rotation about x by -90 degrees (J) sits in shared
// memory with every degree block zero-padded to n4 x n4, row-major.  Only products with J^T are
// formed: J^T = S J S with S = diag(-1 for m < 0), because the reflection y -> -y maps Y_lm to
// S Y_lm and turns the rotation about x by an angle into the rotation by minus that angle; so a
// product with J is S J^T S, and both S are folded into the neighbouring steps.  A product
// J^T [n x n] x [n x TB] per degree is tiled 4 rows x 4 translations per item: per four input
// coefficients, four vector loads of J (rows k..k+3 at the item's four columns, consecutive
// items on consecutive columns) and four of the inputs (one per translation, the same address
// across the items of a degree) feed 64 multiply-adds.  An item's cost grows with its degree, so
// when there are more items than threads each thread takes row groups s and R-1-s of one
// translation group.  The coaxial step reads each translation's stored block once (8 loads in
// flight), one load serving +m and -m.  Used by the M2L chunks and by the tree passes.

#define FMM_TB 8           // translations per batch (tree passes, FP64 M2L)
#define FMM_TB_M2L32 16    // translations per batch of the FP32 M2L chunks
#define FMM_BT 256         // threads of a batched CTA
#define FMM_BT_M2L32 384   // threads of an FP32 M2L CTA (two per SM: 24 warps)
#define FMM_RG_MAX 140     // row groups of 4 up to degree DDLPB_FMM_PMAX (132 at 21)
#define FMM_OM_MAX 256     // (m, o) items of the coaxial step, (p+1)(p+2)/2 (253 at 21)
// integer tables of a batched CTA (built on the host, copied to shared memory)
#define FMM_BTAB_RGOFF 0
#define FMM_BTAB_JPOFF (DDLPB_FMM_PMAX + 4)
#define FMM_BTAB_POFF (2 * (DDLPB_FMM_PMAX + 4))
#define FMM_BTAB_RGL (3 * (DDLPB_FMM_PMAX + 4))
#define FMM_BTAB_RGR0 (FMM_BTAB_RGL + FMM_RG_MAX)
#define FMM_BTAB_OMM (FMM_BTAB_RGR0 + FMM_RG_MAX)
#define FMM_BTAB_OMO (FMM_BTAB_OMM + FMM_OM_MAX)
#define FMM_BTAB_CMP (FMM_BTAB_OMO + FMM_OM_MAX)           // [m] order-m offset in a block p -> p
#define FMM_BTAB_CMQ (FMM_BTAB_CMP + DDLPB_FMM_PMAX + 4)   // [m] order-m offset in a block q -> p
#define FMM_BTAB (FMM_BTAB_CMQ + DDLPB_FMM_PMAX + 4)
// tables read through the cache only (after the shared part of the same array)
#define FMM_GTAB_UNPAD FMM_BTAB                              // [(p+1)^2] padded slot of index l*l+l+m
#define FMM_GTAB_LM (FMM_GTAB_UNPAD + (DDLPB_FMM_PMAX + 1) * (DDLPB_FMM_PMAX + 1))   // (l, m > 0) items
#define FMM_GTAB (FMM_GTAB_LM + DDLPB_FMM_PMAX * (DDLPB_FMM_PMAX + 1) / 2)

// shared-memory head: per translation the block offset (long long), input degree and source
// row (int), then the integer tables; rounded up to 16 bytes
template <int TB>
__host__ __device__ constexpr int batch_head_bytes() {
    return (8 * TB + 4 * (2 * TB + FMM_BTAB) + 15) / 16 * 16;
}

struct BatchHead {
    long long* zoff;   // [TB] coaxial block of translation b
    int* pin;          // [TB] input degree (forward direction) of translation b
    int* row;          // [TB] row of the input vector (node index), -1: no translation
    int* tab;          // the integer tables (FMM_BTAB ints)
    int* rgoff;        // [p+2] row groups of 4 below degree l
    int* jpoff;        // [p+2] offset of the padded J block of degree l (elements)
    int* poff;         // [p+2] offset of degree l in the padded layout
    int* rg_l;         // [R] degree of row group r
    int* rg_r0;        // [R] first row (within its degree) of row group r
    int* om_m;         // [(p+1)(p+2)/2] order m of coaxial item t (m-major, o = m..p)
    int* om_o;         // output degree of coaxial item t
    int* cmp;          // [m] offset of the order-m part of a coaxial block with input degree p
    int* cmq;          // [m] the same with input degree q
};

template <int TB>
__device__ __forceinline__ BatchHead batch_head(unsigned char* sm) {
    BatchHead h;
    h.zoff = (long long*)sm;
    h.pin = (int*)(h.zoff + TB);
    h.row = h.pin + TB;
    h.tab = h.row + TB;
    h.rgoff = h.tab + FMM_BTAB_RGOFF;
    h.jpoff = h.tab + FMM_BTAB_JPOFF;
    h.poff = h.tab + FMM_BTAB_POFF;
    h.rg_l = h.tab + FMM_BTAB_RGL;
    h.rg_r0 = h.tab + FMM_BTAB_RGR0;
    h.om_m = h.tab + FMM_BTAB_OMM;
    h.om_o = h.tab + FMM_BTAB_OMO;
    h.cmp = h.tab + FMM_BTAB_CMP;
    h.cmq = h.tab + FMM_BTAB_CMQ;
    return h;
}

// Host: the integer tables for order p (layout of FMM_BTAB_*), the padded J and the sizes.
static inline int fmm_padded_size(int p) {
    int s = 0;
    for (int l = 0; l <= p; ++l) s += 4 * (l / 2 + 1);
    return s;
}

static void fmm_batch_tables(int p, int q, std::vector<int>& tab) {
    tab.assign(FMM_GTAB, 0);
    int rg = 0, jp = 0, po = 0;
    for (int l = 0; l <= p + 1; ++l) {
        tab[FMM_BTAB_RGOFF + l] = rg;
        tab[FMM_BTAB_JPOFF + l] = jp;
        tab[FMM_BTAB_POFF + l] = po;
        if (l > p) break;
        const int n4 = 4 * (l / 2 + 1);
        for (int r = 0; r < n4 / 4; ++r) {
            tab[FMM_BTAB_RGL + rg + r] = l;
            tab[FMM_BTAB_RGR0 + rg + r] = 4 * r;
        }
        rg += n4 / 4;
        jp += n4 * n4;
        po += n4;
    }
    int t = 0;
    for (int m = 0; m <= p; ++m)
        for (int o = m; o <= p; ++o, ++t) {
            tab[FMM_BTAB_OMM + t] = m;
            tab[FMM_BTAB_OMO + t] = o;
        }
    // order-m offsets of the coaxial blocks: sum_{k < m} (pin + 1 - k)(p + 1 - k)
    for (int m = 0, sp = 0, sq = 0; m <= p + 1; ++m) {
        tab[FMM_BTAB_CMP + m] = sp;
        tab[FMM_BTAB_CMQ + m] = sq;
        sp += (p + 1 - m) * (p + 1 - m);
        if (m <= q) sq += (q + 1 - m) * (p + 1 - m);
    }
    for (int l = 0; l <= p; ++l)
        for (int m = -l; m <= l; ++m) tab[FMM_GTAB_UNPAD + l * l + l + m] = tab[FMM_BTAB_POFF + l] + l + m;
    t = 0;
    for (int l = 1; l <= p; ++l)
        for (int m = 1; m <= l; ++m, ++t) tab[FMM_GTAB_LM + t] = (tab[FMM_BTAB_POFF + l] + l) | (m << 16);
}

// e / d for 0 <= e < 2^20 and d >= 1, given inv = 1.0f / d: the float quotient is within one of
// the exact one and is corrected.
__device__ __forceinline__ int qdiv(int e, int d, float inv) {
    int q = __float2int_rz((float)e * inv);
    if (q * d > e) --q;
    else if ((q + 1) * d <= e) ++q;
    return q;
}

// Four consecutive values (16-byte aligned for float, 32 for double) to registers and back.
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
    const float4 t = *(const float4*)p;
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
    const double2 a = *(const double2*)p, b = *(const double2*)(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, const float (&v)[4]) { *(float4*)p = make_float4(v[0], v[1], v[2], v[3]); }
__device__ __forceinline__ void st4(double* p, const double (&v)[4]) {
    *(double2*)p = make_double2(v[0], v[1]);
    *(double2*)(p + 2) = make_double2(v[2], v[3]);
}

// Rz(s angle_b) on the whole batch, degree <= deg; ang[b][which][cos|sin][32].  flip_in: the
// input holds S v (its m < 0 entries negated); flip_out: write S of the result.
template <typename T, int TB>
__device__ __forceinline__ void brot_z(T* V, int nbpp, int deg, const T* ang, int which, T s, bool flip_in,
                                       bool flip_out, const int* __restrict__ gtab) {
    const int nd = deg * (deg + 1) / 2;   // (l, m) with 1 <= m <= l <= deg, l-major
    const float inv = 1.0f / (float)nd;
    for (int e = threadIdx.x; e < TB * nd; e += blockDim.x) {
        const int b = qdiv(e, nd, inv), t = e - b * nd;
        const int lm = __ldg(gtab + FMM_GTAB_LM + t), m = lm >> 16;
        const T* a = ang + (b * 4 + which * 2) * 32;
        const T c = a[m], sn = s * a[32 + m];
        T* v = V + (size_t)b * nbpp + (lm & 0xffff);
        const T x = v[m], y = flip_in ? -v[-m] : v[-m];
        const T nx = c * x - sn * y, ny = sn * x + c * y;
        v[m] = nx;
        v[-m] = flip_out ? -ny : ny;
    }
    __syncthreads();
}

// Out[b] = J^T In[b], degree by degree up to deg, all TB rows (padded layout).
template <typename T, int TB>
__device__ __forceinline__ void bmul_JT(const T* __restrict__ JP, const T* In, T* Out, int nbpp, int deg,
                                        const BatchHead& h) {
    constexpr int G = TB / 4;                      // translation groups of 4
    const int R = h.rgoff[deg + 1];
    const bool pairs = R * G > (int)blockDim.x;
    const int ns = pairs ? (R + 1) >> 1 : R;
    const float inv = 1.0f / (float)ns;
    for (int e = threadIdx.x; e < ns * G; e += blockDim.x) {
        const int cg = qdiv(e, ns, inv), s = e - cg * ns;
        const size_t b0 = 4 * (size_t)cg * nbpp;
        for (int pass = 0; pass < 2; ++pass) {
            const int r = pass ? R - 1 - s : s;
            if (pass && (!pairs || r == s)) break;
            const int l = h.rg_l[r], r0 = h.rg_r0[r];
            const int n4 = 4 * ((l >> 1) + 1);
            const T* Jc = JP + h.jpoff[l] + r0;
            const T* x = In + b0 + h.poff[l];
            T acc[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = 0;
            for (int k = 0; k < n4; k += 4) {
                T xv[4][4];
#pragma unroll
                for (int j = 0; j < 4; ++j) ld4(x + (size_t)j * nbpp + k, xv[j]);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    T jv[4];
                    ld4(Jc + (size_t)(k + u) * n4, jv);
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] += jv[i] * xv[j][u];
                }
            }
            T* o = Out + b0 + h.poff[l] + r0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const T v[4] = {acc[0][j], acc[1][j], acc[2][j], acc[3][j]};
                st4(o + (size_t)j * nbpp, v);
            }
        }
    }
    __syncthreads();
}

// Coaxial step (forward degrees pin_b -> pout): forward Out = Z_b In (degree pout), transposed
// Out = Z_b^T In (degree pin_b).  flip_in: In holds S of the input.  Rows without a translation
// are skipped (their Out is zero).  The stored block is read from global memory 8 entries at a
// time per thread (independent loads in flight) before the multiply-adds.
template <typename T, int TB>
__device__ __forceinline__ void bcoax(const T* __restrict__ coax, const BatchHead& h, int pout, bool tr, bool flip_in,
                                      const T* In, T* Out, int nbpp) {
    // pout is the expansion order p, and a block's input degree is p or q
    for (int i = threadIdx.x; i < TB * nbpp; i += blockDim.x) Out[i] = 0;
    __syncthreads();
    const int nom = (pout + 1) * (pout + 2) / 2;
    const float inv = 1.0f / (float)nom;
    for (int e = threadIdx.x; e < TB * nom; e += blockDim.x) {
        const int b = qdiv(e, nom, inv), t = e - b * nom;
        if (h.row[b] < 0) continue;
        const int pb = h.pin[b];
        const int m = h.om_m[t], o = h.om_o[t];
        if (m > min(pb, pout) || (tr && o > pb)) continue;
        const int na = pout + 1 - m;
        const T* Z = coax + h.zoff[b] + (pb == pout ? h.cmp[m] : h.cmq[m]);
        const T* x = In + (size_t)b * nbpp;
        T sp = 0, sm = 0;
        // forward: z_k = Z[(k - m) na + (o - m)], coefficient index k over input degrees l;
        // transposed: z_k = Z[(o - m) na + (k - m)], k over output degrees a
        const int kend = tr ? pout : pb;
        const long long zs = tr ? 1 : na;
        const T* zp = tr ? Z + (long long)(o - m) * na : Z + (o - m);
        for (int k0 = m; k0 <= kend; k0 += 8) {
            T z[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) z[u] = (k0 + u <= kend) ? __ldg(zp + (long long)(k0 + u - m) * zs) : (T)0;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int k = k0 + u;
                if (k <= kend) {
                    const T* xk = x + h.poff[k] + k;
                    sp += z[u] * xk[m];
                    sm += z[u] * xk[-m];
                }
            }
        }
        T* y = Out + (size_t)b * nbpp + h.poff[o] + o;
        y[m] = sp;
        if (m > 0) y[-m] = flip_in ? -sm : sm;
    }
    __syncthreads();
}

// Angle tables of translation b from the FP64 node centres (t = target - source).
template <typename T>
__device__ __forceinline__ void batch_angles(T* ang, int b, int lane, int p, const double4& ct, const double4& cs) {
    const T tx = (T)(ct.x - cs.x), ty = (T)(ct.y - cs.y), tz = (T)(ct.z - cs.z);
    const T rxy = sqrt(tx * tx + ty * ty);
    const T alpha = rxy > (T)0 ? atan2(ty, tx) : (T)0;
    const T beta = atan2(rxy, tz);
    if (lane <= p) {
        T s, c;
        T* a = ang + b * 128;
        if constexpr (sizeof(T) == 8) sincos((double)lane * alpha, &s, &c);
        else sincosf((float)lane * alpha, &s, &c);
        a[lane] = c;
        a[32 + lane] = s;
        if constexpr (sizeof(T) == 8) sincos((double)lane * beta, &s, &c);
        else sincosf((float)lane * beta, &s, &c);
        a[64 + lane] = c;
        a[96 + lane] = s;
    }
}

// Translate the batch in place: V holds the inputs (rows b, degree d1), W receives the outputs
// (degree d2).  TR: the transposed translations.  J = S J^T S: the S on the right is applied by
// the rotation before, the one on the left by the step after.
template <typename T, int TB>
__device__ __forceinline__ void batch_translate(const T* JP, const T* coax, const BatchHead& h,
                                                const int* __restrict__ gtab, const T* ang, int p, bool tr, int d1,
                                                int d2, T* V, T* W, int nbpp) {
    brot_z<T, TB>(V, nbpp, d1, ang, 0, (T)-1, false, false, gtab);   // Rz(-alpha)
    bmul_JT<T, TB>(JP, V, W, nbpp, d1, h);                            // J^T
    brot_z<T, TB>(W, nbpp, d1, ang, 1, (T)-1, false, true, gtab);    // S Rz(-beta)
    bmul_JT<T, TB>(JP, W, V, nbpp, d1, h);                            // J^T S (J up to the left S)
    bcoax<T, TB>(coax, h, p, tr, true, V, W, nbpp);                   // left S, then along z
    bmul_JT<T, TB>(JP, W, V, nbpp, d2, h);                            // J^T
    brot_z<T, TB>(V, nbpp, d2, ang, 1, (T)1, false, true, gtab);     // S Rz(beta)
    bmul_JT<T, TB>(JP, V, W, nbpp, d2, h);                            // J^T S
    brot_z<T, TB>(W, nbpp, d2, ang, 0, (T)1, true, false, gtab);     // left S, then Rz(alpha)
}

// Pull the batch's stored coaxial blocks towards L2 while the first rotations run: one warp per
// translation, one prefetch per 128-byte line.
template <typename T, int TB>
__device__ __forceinline__ void batch_prefetch(const T* coax, const BatchHead& h, int p, int q) {
    const int lane = threadIdx.x & 31;
    for (int b = threadIdx.x >> 5; b < TB; b += blockDim.x >> 5) {
        if (h.row[b] < 0) continue;
        const int bytes = (int)sizeof(T) * (h.pin[b] == p ? h.cmp[p + 1] : h.cmq[min(q, p) + 1]);
        const char* base = (const char*)(coax + h.zoff[b]);
        for (int off = lane * 128; off < bytes; off += 32 * 128)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(base + off));
    }
}

// Shared-memory layout of a batched CTA after the head: JP, V, W, acc, angles.
template <typename T>
struct BatchArrays {
    T* JP;
    T* V;
    T* W;
    T* acc;
    T* ang;
};

template <typename T, int TB>
__device__ __forceinline__ BatchArrays<T> batch_arrays(unsigned char* sm, long long jpsize, int nbpp, int nacc) {
    BatchArrays<T> a;
    a.JP = (T*)(sm + batch_head_bytes<TB>());
    a.V = a.JP + jpsize;
    a.W = a.V + (size_t)TB * nbpp;
    a.acc = a.W + (size_t)TB * nbpp;
    a.ang = a.acc + (size_t)nacc * nbpp;
    return a;
}

// Copy J and the integer tables into shared memory and zero V, W and acc (their padding stays
// zero: the J^T products write zeros there and nothing else writes it).
template <typename T, int TB>
__device__ __forceinline__ void batch_setup(const BatchArrays<T>& a, const BatchHead& h, const T* __restrict__ JPg,
                                            long long jpsize, const int* __restrict__ btab, int nbpp, int nacc) {
    for (long long k = threadIdx.x; k < jpsize; k += blockDim.x) a.JP[k] = JPg[k];
    for (int k = threadIdx.x; k < FMM_BTAB; k += blockDim.x) h.tab[k] = btab[k];
    const int nz = (2 * TB + nacc) * nbpp;
    for (int k = threadIdx.x; k < nz; k += blockDim.x) a.V[k] = (T)0;
    __syncthreads();
}

// Load the batch's input rows into the padded layout (zero above their degree and for absent
// translations).
template <typename T, int TB>
__device__ __forceinline__ void batch_load(const BatchHead& h, const int* __restrict__ gtab, const T* __restrict__ X,
                                           T* V, int nbp, int nbpp, int din_tr, bool tr) {
    const float inv = 1.0f / (float)nbp;
    for (int e = threadIdx.x; e < TB * nbp; e += blockDim.x) {
        const int b = qdiv(e, nbp, inv), i = e - b * nbp;
        const int rw = h.row[b];
        const int dl = tr ? din_tr : h.pin[b];
        V[(size_t)b * nbpp + __ldg(gtab + FMM_GTAB_UNPAD + i)] =
            (rw >= 0 && i < (dl + 1) * (dl + 1)) ? X[(size_t)rw * nbp + i] : (T)0;
    }
    __syncthreads();
}

// M2L, one CTA per chunk.  Forward: the chunk's translations share the target; part[ck] = their
// sum (degree p).  Transposed: they share the source; part[ck] = the sum of the transposed
// translations of the targets' local adjoints (degree of the source's multipole).
template <typename T, bool TR, int TB, int BT>
__global__ void __launch_bounds__(BT, BT == FMM_BT_M2L32 ? 2 : 1) k_fmm_m2l_batch(int n_ck, int p, int q, long long jpsize,
                                                          const int* __restrict__ btab,
                                                          const int* __restrict__ ck_b, const int* __restrict__ ck_e,
                                                          const int* __restrict__ perm, const int* __restrict__ m2l_t,
                                                          const int* __restrict__ m2l_s,
                                                          const long long* __restrict__ m2l_off,
                                                          const int* __restrict__ child0,
                                                          const double4* __restrict__ nc, const T* __restrict__ JPg,
                                                          const T* __restrict__ coax, const T* __restrict__ X,
                                                          T* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nbp = (p + 1) * (p + 1);
    const BatchHead h = batch_head<TB>(smraw);
    const int nbpp = btab[FMM_BTAB_POFF + p + 1];
    const BatchArrays<T> a = batch_arrays<T, TB>(smraw, jpsize, nbpp, 1);
    batch_setup<T, TB>(a, h, JPg, jpsize, btab, nbpp, 1);
    const int ck = blockIdx.x;
    const int u0 = ck_b[ck], u1 = ck_e[ck];
    for (int ub = u0; ub < u1; ub += TB) {
        const int nt = min(TB, u1 - ub);
        for (int b = threadIdx.x >> 5; b < TB; b += BT / 32) {
            const int lane = threadIdx.x & 31;
            if (b < nt) {
                const int u = perm ? perm[ub + b] : ub + b;
                const int A = m2l_t[u], B = m2l_s[u];
                batch_angles<T>(a.ang, b, lane, p, nc[A], nc[B]);
                if (lane == 0) {
                    h.zoff[b] = m2l_off[u];
                    h.pin[b] = child0[B] < 0 ? q : p;
                    h.row[b] = TR ? A : B;
                }
            } else if (lane == 0) {
                h.row[b] = -1;
                h.pin[b] = 0;
            }
        }
        __syncthreads();
        int dmax = 0;
        for (int b = 0; b < nt; ++b) dmax = max(dmax, h.pin[b]);
        batch_prefetch<T, TB>(coax, h, p, q);
        batch_load<T, TB>(h, btab, X, a.V, nbp, nbpp, p, TR);
        const int d1 = TR ? p : dmax, d2 = TR ? dmax : p;
        batch_translate<T, TB>(a.JP, coax, h, btab, a.ang, p, TR, d1, d2, a.V, a.W, nbpp);
        const int nd2 = h.poff[d2 + 1];
        for (int i = threadIdx.x; i < nd2; i += blockDim.x) {
            T s = a.acc[i];
            for (int b = 0; b < nt; ++b) s += a.W[(size_t)b * nbpp + i];
            a.acc[i] = s;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < nbp; i += blockDim.x) part[(size_t)ck * nbp + i] = a.acc[__ldg(btab + FMM_GTAB_UNPAD + i)];
}

// Tree passes, FMM_TB translations per CTA, nodes [first, first + count) of one level.
//   KIND 0 (M2M):   M_k = sum over the two children c of M2M(c -> k) M_c          (4 nodes per CTA)
//   KIND 1 (L2L):   L_k = (k's M2L chunks) + L2L(parent -> k) L_parent            (8 nodes per CTA)
//   KIND 2 (L2L^T): Lambda_k = sum over the children c of L2L(k -> c)^T Lambda_c  (4 nodes per CTA)
//   KIND 3 (M2M^T): Psi_k = (k's transposed M2L chunks) + M2M(k -> parent)^T Psi_parent (8 per CTA)
// Leaves are skipped by the kinds 0 and 2 (their rows were written by the leaf kernels).
template <typename T, int KIND>
__global__ void __launch_bounds__(FMM_BT) k_fmm_tree_batch(int first, int count, int p, int q, long long jpsize,
                                                           const int* __restrict__ btab,
                                                           const int* __restrict__ parent,
                                                           const int* __restrict__ child0,
                                                           const int* __restrict__ ck_ptr, const T* __restrict__ part,
                                                           const long long* __restrict__ off,
                                                           const double4* __restrict__ nc, const T* __restrict__ JPg,
                                                           const T* __restrict__ coax, T* __restrict__ X) {
    constexpr int TB = FMM_TB;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nbp = (p + 1) * (p + 1);
    const BatchHead h = batch_head<TB>(smraw);
    const int nbpp = btab[FMM_BTAB_POFF + p + 1];
    const BatchArrays<T> a = batch_arrays<T, TB>(smraw, jpsize, nbpp, 0);
    batch_setup<T, TB>(a, h, JPg, jpsize, btab, nbpp, 0);
    constexpr bool pairs = (KIND == 0 || KIND == 2);
    constexpr int per = pairs ? TB / 2 : TB;     // nodes per CTA
    constexpr bool TR = (KIND >= 2);
    const int k0 = first + blockIdx.x * per;
    {
        const int b = threadIdx.x >> 5, lane = threadIdx.x & 31;   // FMM_BT / 32 == FMM_TB
        const int k = k0 + (pairs ? b / 2 : b);
        int src = -1, tgt = -1;
        long long zo = 0;
        int pn = p;
        if (k < first + count) {
            if (KIND == 0) {            // child -> k
                if (child0[k] >= 0) { src = child0[k] + (b & 1); tgt = k; zo = off[src]; pn = child0[src] < 0 ? q : p; }
            } else if (KIND == 1) {     // parent -> k
                if (parent[k] >= 0) { src = parent[k]; tgt = k; zo = off[k]; }
            } else if (KIND == 2) {     // k -> child (transposed)
                if (child0[k] >= 0) { tgt = child0[k] + (b & 1); src = k; zo = off[tgt]; }
            } else {                    // k -> parent (transposed)
                if (parent[k] >= 0) { src = k; tgt = parent[k]; zo = off[k]; pn = child0[k] < 0 ? q : p; }
            }
        }
        if (src >= 0) batch_angles<T>(a.ang, b, lane, p, nc[tgt], nc[src]);
        if (lane == 0) {
            h.zoff[b] = zo;
            h.pin[b] = pn;
            h.row[b] = src < 0 ? -1 : (TR ? tgt : src);   // the row read: the forward input, or the transposed input
        }
    }
    __syncthreads();
    // forward inputs have degree pin (M2M) or p (L2L); transposed inputs degree p
    batch_prefetch<T, TB>(coax, h, p, q);
    batch_load<T, TB>(h, btab, X, a.V, nbp, nbpp, p, TR);
    int dmax = 0;
    for (int b = 0; b < TB; ++b) dmax = max(dmax, h.pin[b]);
    const int d1 = TR ? p : dmax, d2 = TR ? dmax : p;
    batch_translate<T, TB>(a.JP, coax, h, btab, a.ang, p, TR, d1, d2, a.V, a.W, nbpp);
    // combine and write (each node owned by one thread per coefficient: fixed order)
    for (int e = threadIdx.x; e < per * nbp; e += blockDim.x) {
        const int g = e / nbp, i = e - g * nbp;
        const int k = k0 + g;
        if (k >= first + count) continue;
        const int pi = __ldg(btab + FMM_GTAB_UNPAD + i);
        if (pairs) {
            if (child0[k] < 0) continue;
            X[(size_t)k * nbp + i] = a.W[(size_t)(2 * g) * nbpp + pi] + a.W[(size_t)(2 * g + 1) * nbpp + pi];
        } else {
            T s = 0;
            for (int ck = ck_ptr[k]; ck < ck_ptr[k + 1]; ++ck) s += part[(size_t)ck * nbp + i];
            if (h.row[g] >= 0) s += a.W[(size_t)g * nbpp + pi];
            X[(size_t)k * nbp + i] = s;
        }
    }
}

template <typename T, int TB>
size_t fmm_batch_smem(int p, long long jpsize, int nacc) {
    const int nbpp = fmm_padded_size(p);
    return batch_head_bytes<TB>() + sizeof(T) * ((size_t)jpsize + (2 * (size_t)TB + nacc) * nbpp + TB * 4 * 32);
}

// ---------------------------------------------------------------- host

static ddlpb_status fmm_scan_ll(ddlpb_ctx* c, const long long* in, long long* out, int n) {
    size_t bytes = 0;
    DDLPB_CK(c, cub::DeviceScan::ExclusiveSum(nullptr, bytes, in, out, n, c->stream));
    void* tmp = nullptr;
    DDLPB_TRY(ctx_alloc(c, (char**)&tmp, bytes));
    DDLPB_CK(c, cub::DeviceScan::ExclusiveSum(tmp, bytes, in, out, n, c->stream));
    return DDLPB_OK;
}

static ddlpb_status fmm_scan_int(ddlpb_ctx* c, const int* in, int* out, int n) {
    size_t bytes = 0;
    DDLPB_CK(c, cub::DeviceScan::ExclusiveSum(nullptr, bytes, in, out, n, c->stream));
    void* tmp = nullptr;
    DDLPB_TRY(ctx_alloc(c, (char**)&tmp, bytes));
    DDLPB_CK(c, cub::DeviceScan::ExclusiveSum(tmp, bytes, in, out, n, c->stream));
    return DDLPB_OK;
}

template <typename TK, typename TV>
static ddlpb_status fmm_sort_pairs(ddlpb_ctx* c, const TK* kin, TK* kout, const TV* vin, TV* vout, int n, int bits) {
    if (n <= 0) return DDLPB_OK;
    size_t bytes = 0;
    DDLPB_CK(c, cub::DeviceRadixSort::SortPairs(nullptr, bytes, kin, kout, vin, vout, n, 0, bits, c->stream));
    void* tmp = nullptr;
    DDLPB_TRY(ctx_alloc(c, (char**)&tmp, bytes));
    DDLPB_CK(c, cub::DeviceRadixSort::SortPairs(tmp, bytes, kin, kout, vin, vout, n, 0, bits, c->stream));
    return DDLPB_OK;
}

static int bits_for(int n) {
    int b = 1;
    while ((1LL << b) < (long long)n + 1) ++b;
    return b;
}

// Sorted (key, value) pairs -> CSR over K keys and the values in key order.
static ddlpb_status fmm_csr(ddlpb_ctx* c, const int* keys, const int* vals, int n, int K, int** ptr, int** vout) {
    int *ks = nullptr;
    DDLPB_TRY(ctx_alloc(c, &ks, std::max(n, 1)));
    DDLPB_TRY(ctx_alloc(c, vout, std::max(n, 1)));
    DDLPB_TRY(ctx_alloc(c, ptr, K + 1));
    DDLPB_TRY(fmm_sort_pairs(c, keys, ks, vals, *vout, n, bits_for(K)));
    k_fmm_seg_starts<<<ceil_div(n + 1, 256), 256, 0, c->stream>>>(n, K, ks, *ptr);
    DDLPB_LAUNCHED(c, "fmm_seg_starts");
    return DDLPB_OK;
}

// Chunks of at most DDLPB_FMM_CHUNK entries of each of K runs given by ptr.
static ddlpb_status fmm_chunks(ddlpb_ctx* c, const int* ptr, int K, int* n_ck, int** cb, int** ce, int** ckptr) {
    int* cnt = nullptr;
    DDLPB_TRY(ctx_alloc(c, &cnt, K + 1));
    DDLPB_TRY(ctx_alloc(c, ckptr, K + 1));
    DDLPB_CK(c, cudaMemsetAsync(cnt, 0, sizeof(int) * (K + 1), c->stream));
    k_fmm_chunk_count<<<ceil_div(K, 256), 256, 0, c->stream>>>(K, ptr, cnt);
    DDLPB_LAUNCHED(c, "fmm_chunk_count");
    DDLPB_TRY(fmm_scan_int(c, cnt, *ckptr, K + 1));
    int n = 0;
    DDLPB_CK(c, cudaMemcpyAsync(&n, *ckptr + K, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    DDLPB_CK(c, cudaStreamSynchronize(c->stream));
    *n_ck = n;
    DDLPB_TRY(ctx_alloc(c, cb, std::max(n, 1)));
    DDLPB_TRY(ctx_alloc(c, ce, std::max(n, 1)));
    k_fmm_chunk_fill<<<ceil_div(K, 256), 256, 0, c->stream>>>(K, ptr, *ckptr, *cb, *ce);
    DDLPB_LAUNCHED(c, "fmm_chunk_fill");
    return DDLPB_OK;
}

ddlpb_status fmm_build(ddlpb_ctx* c, const double* hc) {
    FmmTree& F = c->fmm;
    const int M = c->M, p = c->opt.fmm_order;
    cudaStream_t st = c->stream;
    F.on = true;
    F.p = p;
    F.q = std::min(p, c->lmax + 1);
    F.theta = c->opt.fmm_theta;
    // -- topology: ranges of the sorted list, level by level (depends on M only)
    std::vector<int> na(1, 0), nbv(1, M), par(1, -1);
    F.lev.assign(1, 0);
    for (size_t lo = 0; lo < na.size();) {
        const size_t hi = na.size();
        for (size_t k = lo; k < hi; ++k) {
            const int a = na[k], b = nbv[k];
            if (b - a >= 2) {
                const int m = a + (b - a) / 2;
                na.push_back(a); nbv.push_back(m); par.push_back((int)k);
                na.push_back(m); nbv.push_back(b); par.push_back((int)k);
            }
        }
        if (na.size() > hi) F.lev.push_back((int)hi);
        lo = hi;
    }
    const int n_nodes = (int)na.size();
    F.lev.push_back(n_nodes);
    std::vector<int> ch0(n_nodes, -1);
    for (int k = 1; k < n_nodes; ++k)
        if (ch0[par[k]] < 0) ch0[par[k]] = k;
    F.n_nodes = n_nodes;
    F.depth = (int)F.lev.size() - 2;
    F.host_child0 = ch0;
    DDLPB_TRY(ctx_alloc(c, &F.node_a, n_nodes));
    DDLPB_TRY(ctx_alloc(c, &F.node_b, n_nodes));
    DDLPB_TRY(ctx_alloc(c, &F.parent, n_nodes));
    DDLPB_TRY(ctx_alloc(c, &F.child0, n_nodes));
    DDLPB_CK(c, cudaMemcpyAsync(F.node_a, na.data(), sizeof(int) * n_nodes, cudaMemcpyHostToDevice, st));
    DDLPB_CK(c, cudaMemcpyAsync(F.node_b, nbv.data(), sizeof(int) * n_nodes, cudaMemcpyHostToDevice, st));
    DDLPB_CK(c, cudaMemcpyAsync(F.parent, par.data(), sizeof(int) * n_nodes, cudaMemcpyHostToDevice, st));
    DDLPB_CK(c, cudaMemcpyAsync(F.child0, ch0.data(), sizeof(int) * n_nodes, cudaMemcpyHostToDevice, st));
    // -- Morton order of the centres
    double lx = hc[0], ly = hc[1], lz = hc[2], hx = hc[0], hy = hc[1], hz = hc[2];
    for (int k = 1; k < M; ++k) {
        lx = std::min(lx, hc[3 * k]); hx = std::max(hx, hc[3 * k]);
        ly = std::min(ly, hc[3 * k + 1]); hy = std::max(hy, hc[3 * k + 1]);
        lz = std::min(lz, hc[3 * k + 2]); hz = std::max(hz, hc[3 * k + 2]);
    }
    double side = std::max(hx - lx, std::max(hy - ly, hz - lz));
    if (!(side > 0.0)) side = 1.0;
    {
        unsigned long long *kin = nullptr, *kout = nullptr;
        int* vin = nullptr;
        DDLPB_TRY(ctx_alloc(c, &kin, M));
        DDLPB_TRY(ctx_alloc(c, &kout, M));
        DDLPB_TRY(ctx_alloc(c, &vin, M));
        DDLPB_TRY(ctx_alloc(c, &F.order, M));
        k_fmm_morton<<<ceil_div(M, 256), 256, 0, st>>>(M, c->sph, lx, ly, lz, side, kin, vin);
        DDLPB_LAUNCHED(c, "fmm_morton");
        DDLPB_TRY(fmm_sort_pairs(c, kin, kout, vin, F.order, M, 63));
    }
    // -- node geometry
    DDLPB_TRY(ctx_alloc(c, &F.node_g, n_nodes));
    DDLPB_TRY(ctx_alloc(c, &F.node_Rs, n_nodes));
    DDLPB_TRY(ctx_alloc(c, &F.leaf_sphere, n_nodes));
    DDLPB_TRY(ctx_alloc(c, &F.leaf_node, M));
    k_fmm_node_geom<<<ceil_div(n_nodes, 128), 128, 0, st>>>(n_nodes, F.node_a, F.node_b, F.order, c->sph, F.node_g,
                                                             F.node_Rs, F.leaf_sphere, F.leaf_node);
    DDLPB_LAUNCHED(c, "fmm_node_geom");
    // -- dual traversal, level by level (retried with larger arrays if a capacity was exceeded)
    long long cap_front = 64LL * n_nodes + 1024, cap_m2l = 256LL * n_nodes + 1024, cap_near = 64LL * M + 1024;
    int2 *m2l = nullptr, *near = nullptr;
    int n_m2l = 0, n_near = 0;
    for (int attempt = 0;; ++attempt) {
        int2 *fa = nullptr, *fb = nullptr;
        int* cnt = nullptr;
        DDLPB_TRY(ctx_alloc(c, &fa, cap_front));
        DDLPB_TRY(ctx_alloc(c, &fb, cap_front));
        DDLPB_TRY(ctx_alloc(c, &m2l, cap_m2l));
        DDLPB_TRY(ctx_alloc(c, &near, cap_near));
        DDLPB_TRY(ctx_alloc(c, &cnt, 3));
        const int2 root = make_int2(0, 0);
        DDLPB_CK(c, cudaMemcpyAsync(fa, &root, sizeof(int2), cudaMemcpyHostToDevice, st));
        DDLPB_CK(c, cudaMemsetAsync(cnt, 0, 3 * sizeof(int), st));
        int n_front = 1, h[3] = {0, 0, 0};
        bool overflow = false;
        long long max_front = 1;
        for (int level = 0; n_front > 0 && level < 4 * (F.depth + 2); ++level) {
            DDLPB_CK(c, cudaMemsetAsync(cnt, 0, sizeof(int), st));
            k_fmm_traverse<<<ceil_div(n_front, 256), 256, 0, st>>>(n_front, fa, F.node_g, F.node_Rs, F.child0, F.theta,
                                                                   fb, cnt, (int)cap_front, m2l, cnt + 1, (int)cap_m2l,
                                                                   near, cnt + 2, (int)cap_near);
            DDLPB_LAUNCHED(c, "fmm_traverse");
            DDLPB_CK(c, cudaMemcpyAsync(h, cnt, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
            DDLPB_CK(c, cudaStreamSynchronize(st));
            if (h[0] > cap_front || h[1] > cap_m2l || h[2] > cap_near) {
                overflow = true;
                max_front = std::max<long long>(max_front, h[0]);
                break;
            }
            n_front = h[0];
            std::swap(fa, fb);
        }
        if (!overflow && n_front > 0) {
            c->err = "FMM traversal did not terminate";
            return DDLPB_ECUDA;
        }
        if (!overflow) {
            n_m2l = h[1];
            n_near = h[2];
            break;
        }
        if (attempt >= 3) {
            c->err = "FMM interaction lists exceed their capacity";
            return DDLPB_ENOMEM;
        }
        cap_front = std::max(cap_front * 4, max_front + 1024);
        cap_m2l *= 4;
        cap_near *= 4;
    }
    F.n_m2l = n_m2l;
    F.n_near = n_near;
    // -- M2L list sorted by target, chunks; the source-sorted view
    {
        int *t = nullptr, *s = nullptr, *tptr = nullptr, *sorted_s = nullptr;
        DDLPB_TRY(ctx_alloc(c, &t, std::max(n_m2l, 1)));
        DDLPB_TRY(ctx_alloc(c, &s, std::max(n_m2l, 1)));
        if (n_m2l > 0) {
            k_fmm_split_pairs<<<ceil_div(n_m2l, 256), 256, 0, st>>>(n_m2l, m2l, t, s);
            DDLPB_LAUNCHED(c, "fmm_split_pairs");
        }
        DDLPB_TRY(fmm_csr(c, t, s, n_m2l, n_nodes, &tptr, &sorted_s));
        F.m2l_s = sorted_s;
        DDLPB_TRY(ctx_alloc(c, &F.m2l_t, std::max(n_m2l, 1)));
        k_fmm_fill_keys<<<ceil_div(n_nodes, 256), 256, 0, st>>>(n_nodes, tptr, F.m2l_t);
        DDLPB_LAUNCHED(c, "fmm_fill_keys");
        DDLPB_TRY(fmm_chunks(c, tptr, n_nodes, &F.n_ck, &F.ck_b, &F.ck_e, &F.tck_ptr));
        // by source: keys m2l_s (sorted list order), values = position in the sorted list
        int* pos = nullptr;
        int* sptr = nullptr;
        DDLPB_TRY(ctx_alloc(c, &pos, std::max(n_m2l, 1)));
        if (n_m2l > 0) {
            k_fmm_iota<<<ceil_div(n_m2l, 256), 256, 0, st>>>(n_m2l, pos);
            DDLPB_LAUNCHED(c, "fmm_iota");
        }
        DDLPB_TRY(fmm_csr(c, F.m2l_s, pos, n_m2l, n_nodes, &sptr, &F.m2lT_k));
        DDLPB_TRY(fmm_chunks(c, sptr, n_nodes, &F.n_ckT, &F.ckT_b, &F.ckT_e, &F.sck_ptr));
    }
    // -- near pairs (node ids -> sphere ids), CSR by target and by source sphere
    {
        int *a = nullptr, *b = nullptr;
        DDLPB_TRY(ctx_alloc(c, &a, std::max(n_near, 1)));
        DDLPB_TRY(ctx_alloc(c, &b, std::max(n_near, 1)));
        if (n_near > 0) {
            k_fmm_split_pairs<<<ceil_div(n_near, 256), 256, 0, st>>>(n_near, near, a, b);
            DDLPB_LAUNCHED(c, "fmm_split_pairs");
            k_fmm_near_spheres<<<ceil_div(n_near, 256), 256, 0, st>>>(n_near, F.leaf_sphere, a, b);
            DDLPB_LAUNCHED(c, "fmm_near_spheres");
        }
        DDLPB_TRY(fmm_csr(c, a, b, n_near, M, &F.near_ptr, &F.near_j));
        DDLPB_TRY(fmm_csr(c, b, a, n_near, M, &F.nearT_ptr, &F.nearT_i));
    }
    // -- offsets of the coaxial blocks
    {
        const int n_tr = n_m2l + 2 * n_nodes;
        long long *sz = nullptr, *off = nullptr;
        DDLPB_TRY(ctx_alloc(c, &sz, n_tr + 1));
        DDLPB_TRY(ctx_alloc(c, &off, n_tr + 1));
        DDLPB_CK(c, cudaMemsetAsync(sz, 0, sizeof(long long) * (n_tr + 1), st));
        k_fmm_coax_sizes<<<ceil_div(n_tr, 256), 256, 0, st>>>(n_m2l, n_nodes, p, F.q, F.m2l_s, F.child0, F.parent, sz);
        DDLPB_LAUNCHED(c, "fmm_coax_sizes");
        DDLPB_TRY(fmm_scan_ll(c, sz, off, n_tr + 1));
        DDLPB_CK(c, cudaMemcpyAsync(&F.coax_size, off + n_tr, sizeof(long long), cudaMemcpyDeviceToHost, st));
        F.coax_off = off;
        DDLPB_TRY(ctx_alloc(c, &F.m2l_off, std::max(n_m2l, 1)));
        DDLPB_TRY(ctx_alloc(c, &F.m2m_off, n_nodes));
        DDLPB_TRY(ctx_alloc(c, &F.l2l_off, n_nodes));
        k_fmm_coax_offsets<<<ceil_div(n_tr, 256), 256, 0, st>>>(n_m2l, n_nodes, off, F.m2l_off, F.m2m_off, F.l2l_off);
        DDLPB_LAUNCHED(c, "fmm_coax_offsets");
        int* cnt = nullptr;
        DDLPB_TRY(ctx_alloc(c, &cnt, 1));
        DDLPB_CK(c, cudaMemsetAsync(cnt, 0, sizeof(int), st));
        if (n_m2l > 0) {
            k_fmm_count_leaf_src<<<ceil_div(n_m2l, 256), 256, 0, st>>>(n_m2l, F.m2l_s, F.child0, cnt);
            DDLPB_LAUNCHED(c, "fmm_count_leaf_src");
        }
        int n_leaf_src = 0;
        DDLPB_CK(c, cudaMemcpyAsync(&n_leaf_src, cnt, sizeof(int), cudaMemcpyDeviceToHost, st));
        DDLPB_CK(c, cudaStreamSynchronize(st));
        // per translation: two J products at the input degree, two at the output degree, the
        // coaxial products (m and -m), 2 flops per multiply-add
        auto flops = [&](int pin) {
            auto S = [](int d) { double s = 0; for (int l = 0; l <= d; ++l) s += (2.0 * l + 1) * (2.0 * l + 1); return s; };
            double cx = 0;
            for (int m = 0; m <= std::min(pin, p); ++m) cx += (m == 0 ? 1.0 : 2.0) * (pin + 1 - m) * (p + 1 - m);
            return 2.0 * (2.0 * S(pin) + 2.0 * S(p) + cx);
        };
        c->info.fmm_nodes = n_nodes;
        c->info.fmm_m2l = n_m2l;
        c->info.fmm_near_pairs = n_near;
        c->info.fmm_m2l_flops = n_leaf_src * flops(F.q) + (double)(n_m2l - n_leaf_src) * flops(p);
    }
    return DDLPB_OK;
}

// Per-precision data: coaxial blocks (FP64 evaluation, stored as T), J, the Y table to degree p,
// node centres, expansion buffers.
template <typename T>
static ddlpb_status fmm_prepare(ddlpb_ctx* c, FmmOps<T>& O) {
    if (O.ready) return DDLPB_OK;
    FmmTree& F = c->fmm;
    const int p = F.p, nbp = (p + 1) * (p + 1);
    cudaStream_t st = c->stream;
    // constant tables (host): Gaunt coaxial sums and the rotation J
    fmmhost::CoaxIndex gi;
    std::vector<double> g, Jh;
    fmmhost::gaunt_coax_table(p, gi, g);
    fmmhost::rotation_J(p, Jh);
    double* gtab = nullptr;
    long long* goff = nullptr;
    DDLPB_TRY(ctx_alloc(c, &gtab, g.size()));
    DDLPB_TRY(ctx_alloc(c, &goff, gi.off.size()));
    DDLPB_CK(c, cudaMemcpyAsync(gtab, g.data(), sizeof(double) * g.size(), cudaMemcpyHostToDevice, st));
    DDLPB_CK(c, cudaMemcpyAsync(goff, gi.off.data(), sizeof(long long) * gi.off.size(), cudaMemcpyHostToDevice, st));
    // J with every degree block zero-padded to n4 x n4 (n4 = 2l+1 rounded up to 4), row-major
    std::vector<T> Jp;
    for (int l = 0; l <= p; ++l) {
        const int n = 2 * l + 1, n4 = (n + 3) / 4 * 4;
        const double* Jl = Jh.data() + fmmhost::jblock(l);
        for (int r = 0; r < n4; ++r)
            for (int k = 0; k < n4; ++k) Jp.push_back(r < n && k < n ? (T)Jl[(size_t)r * n + k] : (T)0);
    }
    O.jpsize = (long long)Jp.size();
    DDLPB_TRY(ctx_alloc(c, &O.JP, Jp.size()));
    DDLPB_CK(c, cudaMemcpyAsync(O.JP, Jp.data(), sizeof(T) * Jp.size(), cudaMemcpyHostToDevice, st));
    std::vector<int> bt;
    fmm_batch_tables(p, F.q, bt);
    DDLPB_TRY(ctx_alloc(c, &O.btab, bt.size()));
    DDLPB_CK(c, cudaMemcpyAsync(O.btab, bt.data(), sizeof(int) * bt.size(), cudaMemcpyHostToDevice, st));
    DDLPB_TRY(ctx_alloc(c, &O.coax, std::max<long long>(F.coax_size, 1)));
    const int n_tr = F.n_m2l + 2 * F.n_nodes;
    k_fmm_coax<T><<<n_tr, 128, 0, st>>>(F.n_m2l, F.n_nodes, p, F.q, c->kappa, F.m2l_t, F.m2l_s, F.child0, F.parent,
                                        F.node_g, gtab, goff, F.coax_off, O.coax);
    DDLPB_LAUNCHED(c, "fmm_coax");
    DDLPB_TRY(ctx_alloc(c, &O.Yp, (size_t)c->N * nbp));
    k_fmm_ytab<T><<<ceil_div(c->N, 128), 128, 0, st>>>(c->N, p, c->leb, c->yt, O.Yp);
    DDLPB_LAUNCHED(c, "fmm_ytab");
    DDLPB_TRY(ctx_alloc(c, &O.Mx, (size_t)F.n_nodes * nbp));
    DDLPB_TRY(ctx_alloc(c, &O.Lx, (size_t)F.n_nodes * nbp));
    DDLPB_TRY(ctx_alloc(c, &O.part, (size_t)std::max(std::max(F.n_ck, F.n_ckT), 1) * nbp));
    DDLPB_TRY(ctx_alloc(c, &O.leafq, (size_t)c->M * (F.q + 1) * (F.q + 1)));
    O.ready = true;
    return DDLPB_OK;
}

template <typename T> static FmmOps<T>& fmm_ops(ddlpb_ctx* c);
template <> FmmOps<double>& fmm_ops<double>(ddlpb_ctx* c) { return c->fmm64; }
template <> FmmOps<float>& fmm_ops<float>(ddlpb_ctx* c) { return c->fmm32; }

template <typename T, typename K>
static ddlpb_status fmm_smem_attr(ddlpb_ctx* c, K kernel, size_t bytes) {
    if (bytes > 48 * 1024)
        DDLPB_CK(c, cudaFuncSetAttribute((const void*)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return DDLPB_OK;
}

// phi_ext[t] = sum_j mu_j . (k-ratio basis of sphere j)(x_t) at every external point t: far
// field by the FMM, near pairs directly.  Timers (kernel_timing): fmm_m2l (level 1), fmm_tree
// (leaf multipoles, M2M and L2L passes) and fmm_near (leaf evaluation with the near pairs).
template <typename T>
ddlpb_status fmm_potential(ddlpb_ctx* c, OpSet<T>& S, const T* mu, T* phi_ext) {
    using V4 = typename FmmOps<T>::V4;
    FmmTree& F = c->fmm;
    FmmOps<T>& O = fmm_ops<T>(c);
    DDLPB_TRY(fmm_prepare<T>(c, O));
    const int p = F.p, q = F.q, nbp = (p + 1) * (p + 1), M = c->M, L = c->lmax;
    cudaStream_t st = c->stream;
    const bool f32 = sizeof(T) == 4;
    constexpr int TBM = sizeof(T) == 4 ? FMM_TB_M2L32 : FMM_TB, BTM = sizeof(T) == 4 ? FMM_BT_M2L32 : FMM_BT;
    const size_t sm0 = fmm_batch_smem<T, FMM_TB>(p, O.jpsize, 0), sm1 = fmm_batch_smem<T, TBM>(p, O.jpsize, 1);
    {
        KernelTimer kt(c, "fmm_tree", f32, 2);
        k_fmm_leaf_mult<T><<<M, 128, 0, st>>>(M, c->nb, nbp, F.leaf_node, mu, O.Mx);
        DDLPB_LAUNCHED(c, "fmm_leaf_mult");
        DDLPB_TRY((fmm_smem_attr<T>(c, k_fmm_tree_batch<T, 0>, sm0)));
        for (int lv = F.depth - 1; lv >= 0; --lv) {
            const int first = F.lev[lv], count = F.lev[lv + 1] - first;
            k_fmm_tree_batch<T, 0><<<ceil_div(count, FMM_TB / 2), FMM_BT, sm0, st>>>(
                first, count, p, q, O.jpsize, O.btab, F.parent, F.child0, nullptr, nullptr, F.m2m_off, F.node_g, O.JP, O.coax,
                O.Mx);
            DDLPB_LAUNCHED(c, "fmm_m2m");
        }
    }
    if (F.n_ck > 0) {
        KernelTimer kt(c, "fmm_m2l", f32);
        DDLPB_TRY((fmm_smem_attr<T>(c, k_fmm_m2l_batch<T, false, TBM, BTM>, sm1)));
        k_fmm_m2l_batch<T, false, TBM, BTM><<<F.n_ck, BTM, sm1, st>>>(F.n_ck, p, q, O.jpsize, O.btab, F.ck_b, F.ck_e, nullptr, F.m2l_t,
                                                                F.m2l_s, F.m2l_off, F.child0, F.node_g, O.JP, O.coax,
                                                                O.Mx, O.part);
        DDLPB_LAUNCHED(c, "fmm_m2l");
    }
    {
        KernelTimer kt(c, "fmm_tree", f32, 2);
        DDLPB_TRY((fmm_smem_attr<T>(c, k_fmm_tree_batch<T, 1>, sm0)));
        for (int lv = 0; lv <= F.depth; ++lv) {
            const int first = F.lev[lv], count = F.lev[lv + 1] - first;
            k_fmm_tree_batch<T, 1><<<ceil_div(count, FMM_TB), FMM_BT, sm0, st>>>(
                first, count, p, q, O.jpsize, O.btab, F.parent, F.child0, F.tck_ptr, O.part, F.l2l_off, F.node_g, O.JP, O.coax,
                O.Lx);
            DDLPB_LAUNCHED(c, "fmm_l2l");
        }
    }
    if (c->E > 0) {
        KernelTimer kt(c, "fmm_near", f32, 2);
        const size_t sm2 = sizeof(T) * ((size_t)nbp + (size_t)(L + 2) * 128);
        DDLPB_TRY((fmm_smem_attr<T>(c, k_fmm_leaf_pot<T, V4>, sm2)));
        k_fmm_leaf_pot<T, V4><<<M, 128, sm2, st>>>(c->N, c->nb, L, p, (T)c->kappa, c->ext_ptr, c->ext_p, c->sph,
                                                   c->leb, F.leaf_node, O.Lx, O.Yp, F.near_ptr, F.near_j, mu, S.Khinv,
                                                   S.yt, phi_ext);
        DDLPB_LAUNCHED(c, "fmm_leaf_pot");
    }
    return DDLPB_OK;
}

// nu_j = sum_t c_t (k-ratio basis of sphere j)(x_t) over the external points (the transpose of
// fmm_potential); the far part of sphere j's adjoint to degree q is kept in FmmOps::leafq.
// Timers: fmm_m2l_T (level 1), fmm_tree, fmm_near.
template <typename T>
ddlpb_status fmm_adjoint(ddlpb_ctx* c, OpSet<T>& S, const T* c_ext, T* nu) {
    using V4 = typename FmmOps<T>::V4;
    FmmTree& F = c->fmm;
    FmmOps<T>& O = fmm_ops<T>(c);
    DDLPB_TRY(fmm_prepare<T>(c, O));
    const int p = F.p, q = F.q, M = c->M, L = c->lmax, N = c->N;
    cudaStream_t st = c->stream;
    const bool f32 = sizeof(T) == 4;
    constexpr int TBM = sizeof(T) == 4 ? FMM_TB_M2L32 : FMM_TB, BTM = sizeof(T) == 4 ? FMM_BT_M2L32 : FMM_BT;
    const size_t sm0 = fmm_batch_smem<T, FMM_TB>(p, O.jpsize, 0), sm1 = fmm_batch_smem<T, TBM>(p, O.jpsize, 1);
    {
        KernelTimer kt(c, "fmm_tree", f32, 2);
        const size_t smL = (sizeof(T) + sizeof(int)) * (size_t)N;
        k_fmm_leaf_lambda<T><<<M, 128, smL, st>>>(N, p, c->ext_ptr, c->ext_p, F.leaf_node, O.Yp, c_ext, O.Lx);
        DDLPB_LAUNCHED(c, "fmm_leaf_lambda");
        DDLPB_TRY((fmm_smem_attr<T>(c, k_fmm_tree_batch<T, 2>, sm0)));
        for (int lv = F.depth - 1; lv >= 0; --lv) {
            const int first = F.lev[lv], count = F.lev[lv + 1] - first;
            k_fmm_tree_batch<T, 2><<<ceil_div(count, FMM_TB / 2), FMM_BT, sm0, st>>>(
                first, count, p, q, O.jpsize, O.btab, F.parent, F.child0, nullptr, nullptr, F.l2l_off, F.node_g, O.JP, O.coax,
                O.Lx);
            DDLPB_LAUNCHED(c, "fmm_l2l_T");
        }
    }
    if (F.n_ckT > 0) {
        KernelTimer kt(c, "fmm_m2l_T", f32);
        DDLPB_TRY((fmm_smem_attr<T>(c, k_fmm_m2l_batch<T, true, TBM, BTM>, sm1)));
        k_fmm_m2l_batch<T, true, TBM, BTM><<<F.n_ckT, BTM, sm1, st>>>(F.n_ckT, p, q, O.jpsize, O.btab, F.ckT_b, F.ckT_e, F.m2lT_k,
                                                                F.m2l_t, F.m2l_s, F.m2l_off, F.child0, F.node_g, O.JP,
                                                                O.coax, O.Lx, O.part);
        DDLPB_LAUNCHED(c, "fmm_m2l_T");
    }
    {
        KernelTimer kt(c, "fmm_tree", f32, 2);
        DDLPB_TRY((fmm_smem_attr<T>(c, k_fmm_tree_batch<T, 3>, sm0)));
        for (int lv = 0; lv <= F.depth; ++lv) {
            const int first = F.lev[lv], count = F.lev[lv + 1] - first;
            k_fmm_tree_batch<T, 3><<<ceil_div(count, FMM_TB), FMM_BT, sm0, st>>>(
                first, count, p, q, O.jpsize, O.btab, F.parent, F.child0, F.sck_ptr, O.part, F.m2m_off, F.node_g, O.JP, O.coax,
                O.Mx);
            DDLPB_LAUNCHED(c, "fmm_m2m_T");
        }
    }
    {
        KernelTimer kt(c, "fmm_near", f32, 2);
        const int nw = 128 / 32;
        const size_t sm3 = sizeof(T) * ((size_t)nw * c->nb + (L + 2) + (size_t)(L + 1) * 128);
        DDLPB_TRY((fmm_smem_attr<T>(c, k_fmm_leaf_adj<T, V4>, sm3)));
        k_fmm_leaf_adj<T, V4><<<M, 128, sm3, st>>>(N, c->nb, L, p, q, (T)c->kappa, c->ext_ptr, c->ext_p, c->sph,
                                                   c->leb, F.leaf_node, O.Mx, F.nearT_ptr, F.nearT_i, c_ext, S.Khinv,
                                                   S.yt, nu, O.leafq);
        DDLPB_LAUNCHED(c, "fmm_leaf_adj");
    }
    return DDLPB_OK;
}

template ddlpb_status fmm_potential<double>(ddlpb_ctx*, OpSet<double>&, const double*, double*);
template ddlpb_status fmm_potential<float>(ddlpb_ctx*, OpSet<float>&, const float*, float*);
template ddlpb_status fmm_adjoint<double>(ddlpb_ctx*, OpSet<double>&, const double*, double*);
template ddlpb_status fmm_adjoint<float>(ddlpb_ctx*, OpSet<float>&, const float*, float*);

// ---------------------------------------------------------------- force terms (FP64)

// Target side of the Yukawa force terms: Ft[t] += c_t grad phi(x_t) at every external point t of
// sphere i, phi the potential of mu from every sphere j != i: the far field from i's local
// expansion (its gradient on the sphere: dR_l Y s + (grad_S Y)/r_i, R_l = 1 at rho = r_i) and the
// near sources directly.
__global__ void k_fmm_force_targets(int N, int nb, int L, int p, double kappa, const int* __restrict__ ext_ptr,
                                    const int* __restrict__ ext_p, const double4* __restrict__ sph,
                                    const double4* __restrict__ leb, const int* __restrict__ leaf_node,
                                    const double* __restrict__ Lx, const int* __restrict__ near_ptr,
                                    const int* __restrict__ near_j, const double* __restrict__ mu,
                                    const double* __restrict__ Khinv, YTab yt, const double4* __restrict__ fs,
                                    double* __restrict__ Ft) {
    extern __shared__ double fsm[];
    const int bd = blockDim.x, tid = threadIdx.x;
    const int nbp = (p + 1) * (p + 1);
    const int i = blockIdx.x;
    const int t0 = ext_ptr[i], cnt = ext_ptr[i + 1] - t0;
    if (cnt == 0) return;
    double* Li = fsm;
    double* dR = Li + nbp;
    double* rad = dR + (p + 2);
    double* drad = rad + (size_t)(L + 1) * bd;
    const double4 a = sph[i];
    for (int k = tid; k < nbp; k += bd) Li[k] = Lx[(size_t)leaf_node[i] * nbp + k];
    // d/drho of i_l(kappa rho)/i_l(kappa r_i) at rho = r_i
    for (int l = tid; l <= p; l += bd) {
        const double x = kappa * a.w;
        dR[l] = (double)l / a.w + kappa * kappa * a.w / (double)(2 * l + 3) * scaled_i_series<double>(l + 1, x) /
                                      scaled_i_series<double>(l, x);
    }
    __syncthreads();
    const int k0 = near_ptr[i], k1 = near_ptr[i + 1];
    for (int t = t0 + tid; t < t0 + cnt; t += bd) {
        const int n = ext_p[t] % N;
        const double4 s = leb[n];
        double A = 0, Bx = 0, By = 0, Bz = 0;
        ylm_grad_stream<double>(p, s.x, s.y, s.z, yt, [&](int idx, int l, double yv, double gx, double gy, double gz) {
            const double cl = Li[idx];
            A += cl * dR[l] * yv;
            Bx += cl * gx;
            By += cl * gy;
            Bz += cl * gz;
        });
        const double pr = Bx * s.x + By * s.y + Bz * s.z, ir = 1.0 / a.w;
        double gx = A * s.x + (Bx - pr * s.x) * ir, gy = A * s.y + (By - pr * s.y) * ir, gz = A * s.z + (Bz - pr * s.z) * ir;
        for (int kk = k0; kk < k1; ++kk) {
            const int j = near_j[kk];
            if (j == i) continue;
            const double4 b = sph[j];
            const double dx = a.x - b.x + a.w * s.x, dy = a.y - b.y + a.w * s.y, dz = a.z - b.z + a.w * s.z;
            const double rho = sqrt(dx * dx + dy * dy + dz * dz), inv = 1.0 / rho;
            const double ex = dx * inv, ey = dy * inv, ez = dz * inv;
            radial<double>(2, L, rho, b.w, kappa, Khinv + (size_t)j * (L + 2), rad + tid, drad + tid, bd);
            const double* m = mu + (size_t)j * nb;
            double Aa = 0, Cx = 0, Cy = 0, Cz = 0;
            ylm_grad_stream<double>(L, ex, ey, ez, yt, [&](int idx, int l, double yv, double hx, double hy, double hz) {
                const double cc = m[idx];
                Aa += cc * drad[tid + l * bd] * yv;
                const double fr = cc * rad[tid + l * bd] * inv;
                Cx += fr * hx;
                Cy += fr * hy;
                Cz += fr * hz;
            });
            const double pq = Cx * ex + Cy * ey + Cz * ez;
            gx += Aa * ex + Cx - pq * ex;
            gy += Aa * ey + Cy - pq * ey;
            gz += Aa * ez + Cz - pq * ez;
        }
        const double ct = fs[t].w;
        Ft[3 * (size_t)t] += ct * gx;
        Ft[3 * (size_t)t + 1] += ct * gy;
        Ft[3 * (size_t)t + 2] += ct * gz;
    }
}

// Source side: G[j] -= sum_{t not on j} c_t grad (mu_j . B_j)(x_t).  Far part: the adjoint of
// the leaf multipole to degree q (leafq, from the transposed pass with the same c_t) contracted
// with the gradient map of the k-ratio basis (degrees l -> l +- 1); near targets directly.
__global__ void k_fmm_force_sources(int N, int nb, int L, int q, double kappa, const int* __restrict__ ext_ptr,
                                    const int* __restrict__ ext_p, const double4* __restrict__ sph,
                                    const double4* __restrict__ leb, const int* __restrict__ nearT_ptr,
                                    const int* __restrict__ nearT_i, const double* __restrict__ mu,
                                    const double* __restrict__ Khinv, YTab yt, const double4* __restrict__ fs,
                                    const double* __restrict__ leafq, const double* __restrict__ gtab,
                                    const long long* __restrict__ goff, double* __restrict__ G) {
    extern __shared__ double fsm[];
    const int bd = blockDim.x, tid = threadIdx.x;
    const int j = blockIdx.x;
    if (ext_ptr[j + 1] == ext_ptr[j]) return;   // no external points: mu_j = 0
    const int nq = (q + 1) * (q + 1);
    double* m = fsm;
    double* kh = m + nb;
    double* rad = kh + (L + 2);
    double* drad = rad + (size_t)(L + 1) * bd;
    double* red = drad + (size_t)(L + 1) * bd;
    const double4 b = sph[j];
    for (int k = tid; k < nb; k += bd) m[k] = mu[(size_t)j * nb + k];
    for (int k = tid; k < L + 2; k += bd) kh[k] = Khinv[(size_t)j * (L + 2) + k];
    __syncthreads();
    double fx = 0, fy = 0, fz = 0;
    // far part: input (l, m) per thread
    const double x = kappa * b.w;
    const double* Q = leafq + (size_t)j * nq;
    for (int idx = tid; idx < nb; idx += bd) {
        const int l = (int)sqrtf((float)idx + 0.5f), mi = idx - l * l;
        const double cm = m[idx];
        for (int up = 1; up >= 0; --up) {
            const int lp = up ? l + 1 : l - 1;
            if (lp < 0 || lp > q) continue;
            // -kappa k_lp(kappa r_j) / k_l(kappa r_j) with k_l = (2l-1)!! exp(-x) khat_l(x) / x^(l+1)
            const double ratio = up ? -kappa * (2.0 * l + 1.0) * kh[l] / (kh[l + 1] * x)
                                    : -kappa * x * kh[l] / ((2.0 * l - 1.0) * kh[l - 1]);
            const int n = 2 * l + 1, np = 2 * lp + 1;
            const double* T = gtab + goff[(size_t)l * 2 + up];
            const double* qv = Q + lp * lp;
            double sx = 0, sy = 0, sz = 0;
            for (int c = 0; c < np; ++c) {
                sx += T[((size_t)0 * n + mi) * np + c] * qv[c];
                sy += T[((size_t)1 * n + mi) * np + c] * qv[c];
                sz += T[((size_t)2 * n + mi) * np + c] * qv[c];
            }
            fx += cm * ratio * sx;
            fy += cm * ratio * sy;
            fz += cm * ratio * sz;
        }
    }
    // near targets t on spheres i != j of j's near list
    for (int kk = nearT_ptr[j]; kk < nearT_ptr[j + 1]; ++kk) {
        const int i = nearT_i[kk];
        if (i == j) continue;
        const double4 a = sph[i];
        const int t0 = ext_ptr[i], cnt = ext_ptr[i + 1] - t0;
        for (int base = 0; base < cnt; base += bd) {
            const bool ok = base + tid < cnt;
            const int t = t0 + base + tid;
            double dx = b.w, dy = 0, dz = 0, ct = 0;
            if (ok) {
                const double4 s = leb[ext_p[t] % N];
                dx = a.x - b.x + a.w * s.x;
                dy = a.y - b.y + a.w * s.y;
                dz = a.z - b.z + a.w * s.z;
                ct = fs[t].w;
            }
            const double rho = sqrt(dx * dx + dy * dy + dz * dz), inv = 1.0 / rho;
            const double ex = dx * inv, ey = dy * inv, ez = dz * inv;
            radial<double>(2, L, rho, b.w, kappa, kh, rad + tid, drad + tid, bd);
            double Aa = 0, Cx = 0, Cy = 0, Cz = 0;
            ylm_grad_stream<double>(L, ex, ey, ez, yt, [&](int idx, int l, double yv, double hx, double hy, double hz) {
                const double cc = m[idx];
                Aa += cc * drad[tid + l * bd] * yv;
                const double fr = cc * rad[tid + l * bd] * inv;
                Cx += fr * hx;
                Cy += fr * hy;
                Cz += fr * hz;
            });
            const double pq = Cx * ex + Cy * ey + Cz * ez;
            fx += ct * (Aa * ex + Cx - pq * ex);
            fy += ct * (Aa * ey + Cy - pq * ey);
            fz += ct * (Aa * ez + Cz - pq * ez);
        }
    }
    fx = warp_sum(fx);
    fy = warp_sum(fy);
    fz = warp_sum(fz);
    if ((tid & 31) == 0) {
        red[3 * (tid >> 5)] = fx;
        red[3 * (tid >> 5) + 1] = fy;
        red[3 * (tid >> 5) + 2] = fz;
    }
    __syncthreads();
    if (tid < 3) {
        double s = 0;
        for (int w = 0; w < bd / 32; ++w) s += red[3 * w + tid];
        G[3 * (size_t)j + tid] -= s;
    }
}

// The Yukawa force terms with the FMM (FP64): target side into Ft, source side into G.  The
// caller has run the transposed pass with c_t = fs[t].w (FmmOps::leafq holds its far part).
ddlpb_status fmm_force_terms(ddlpb_ctx* c, const double* mu, const double4* fs, double* Ft, double* G) {
    FmmTree& F = c->fmm;
    FmmOps<double>& O = c->fmm64;
    const int p = F.p, q = F.q, nbp = (p + 1) * (p + 1), M = c->M, L = c->lmax;
    cudaStream_t st = c->stream;
    if (!O.grad) {
        fmmhost::GradIndex gi;
        std::vector<double> tab;
        fmmhost::gradient_table(L, gi, tab);
        DDLPB_TRY(ctx_alloc(c, &O.grad, tab.size()));
        DDLPB_TRY(ctx_alloc(c, &O.grad_off, gi.off.size()));
        DDLPB_CK(c, cudaMemcpyAsync(O.grad, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, st));
        DDLPB_CK(c, cudaMemcpyAsync(O.grad_off, gi.off.data(), sizeof(long long) * gi.off.size(), cudaMemcpyHostToDevice,
                                    st));
    }
    // leaf locals of mu (the potential itself goes to scratch)
    DDLPB_TRY(fmm_potential<double>(c, c->d64, mu, c->extA));
    const size_t sm1 = sizeof(double) * ((size_t)nbp + (p + 2) + 2 * (size_t)(L + 1) * 128);
    DDLPB_TRY((fmm_smem_attr<double>(c, k_fmm_force_targets, sm1)));
    k_fmm_force_targets<<<M, 128, sm1, st>>>(c->N, c->nb, L, p, c->kappa, c->ext_ptr, c->ext_p, c->sph, c->leb,
                                              F.leaf_node, O.Lx, F.near_ptr, F.near_j, mu, c->Khinv, c->yt, fs, Ft);
    DDLPB_LAUNCHED(c, "fmm_force_targets");
    const size_t sm2 = sizeof(double) * ((size_t)c->nb + (L + 2) + 2 * (size_t)(L + 1) * 128 + 3 * 4);
    DDLPB_TRY((fmm_smem_attr<double>(c, k_fmm_force_sources, sm2)));
    k_fmm_force_sources<<<M, 128, sm2, st>>>(c->N, c->nb, L, q, c->kappa, c->ext_ptr, c->ext_p, c->sph, c->leb,
                                              F.nearT_ptr, F.nearT_i, mu, c->Khinv, c->yt, fs, O.leafq, O.grad,
                                              O.grad_off, G);
    DDLPB_LAUNCHED(c, "fmm_force_sources");
    return DDLPB_OK;
}

