// Pressure at every cell of an adaptive (multiresolution) grid in FP64, Eq. greenSum with
// each source cell clamped at its own rho_h: the fast multipole method on the tree and the
// interaction lists of pp_atree (dual-tree walk).  Leaves are blocks of 8 x 8 cells; a box of
// level l has side s = 2^-l of the unit domain and centre ((ix + 1/2) s, (iy + 1/2) s).
// Expansions are kept in units of their own box side (multipole M_k = alpha_k / s^k, local
// L_l = b_l s^l, Appendix A.2's series and their standard local shifts, for 2 pi P):
//   P2M   S = sum q, M_k = sum q w^k / k, w = (z - c) / s
//   M2M   parent M_k += S u^k / k + sum_{l<=k} M_l 2^-l u^(k-l) C(k-1, l-1), u = (c_child - c) / s
//   M2L   with tau = (c_src - c_tgt) / s_tgt, rho = s_src / s_tgt, x_k = -M_k (-1)^k (rho/tau)^k:
//         L_0 += S (log|tau| + log s_tgt) + sum_k x_k,
//         L_l += tau^-l (-S / l + sum_k x_k C(l+k-1, k-1))
//   L2L   child L_l += 2^-l sum_{k>=l} L_k C(k, l) v^(k-l), v = (c_child - c) / s
//   L2P   P = Re sum_l L_l w^l / (2 pi); near field over the near-field leaf pairs: between
//         leaves of one level every cell pair sits at an integer offset D (in cells of side h),
//         so q log max(h|D|, rho_h) = q (log h + T[D]) with T[D] = log|D| (T[0] = c0) tabulated
//         once in FP64; leaves of different levels are summed directly.
// One launch per step and level; every sum runs in a fixed order, so results repeat bitwise.
// The first solve on a tree uploads the tree, the lists and the table and allocates the
// expansions; they stay with the tree for later solves.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <new>
#include <vector>

#include "../../include/pp.h"
#include "pp_atree_state.h"

namespace {

constexpr int kMaxOrderA = 30;
constexpr double kInv2PiA = 0.15915494309189533576888376337251;
constexpr double kC0A = 0.78539816339744830962 - 1.5 - 0.34657359027997265471;  // pi/4 - 3/2 - ln2/2

struct AGeo {
    double cx, cy, s;     // centre and side
    int level, ix, iy;    // the box's position in the tree
};

__host__ __device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    return double2{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
__host__ __device__ __forceinline__ double2 zadd(double2 a, double2 b) { return double2{a.x + b.x, a.y + b.y}; }
__host__ __device__ __forceinline__ double2 zscale(double2 a, double f) { return double2{a.x * f, a.y * f}; }
__host__ __device__ __forceinline__ double2 zinv(double2 a) {
    const double d = a.x * a.x + a.y * a.y;
    return double2{a.x / d, -a.y / d};
}

// Cell (cx, cy) of a leaf block, index cy * 8 + cx, in units of the block side about its centre.
__host__ __device__ __forceinline__ double2 cell_w(int c) {
    return double2{((c & 7) + 0.5) / 8.0 - 0.5, ((c >> 3) + 0.5) / 8.0 - 0.5};
}

// Each step is a body over (CTA index, thread index) with no shared memory and no barrier,
// wrapped by a kernel; the threads of a step are independent.

// P2M: one CTA of 32 threads per leaf, thread k forms coefficient k (k = 0 is S).
__host__ __device__ inline void ap2m_body(int i, int k, int nleaf, const int* __restrict__ leafbox,
                                          const double* __restrict__ q, int p, double* __restrict__ S,
                                          double2* __restrict__ M) {
    if (i >= nleaf || k > p) return;
    const int b = leafbox[i];
    const double* qq = q + int64_t(i) * 64;
    if (k == 0) {
        double s = 0.0;
        for (int c = 0; c < 64; ++c) s += qq[c];
        S[b] = s;
        M[int64_t(b) * (p + 1)] = double2{0.0, 0.0};
        return;
    }
    double2 acc{0.0, 0.0};
    for (int c = 0; c < 64; ++c) {
        const double2 w = cell_w(c);
        double2 wk = w;
        for (int j = 1; j < k; ++j) wk = zmul(wk, w);
        acc = zadd(acc, zscale(wk, qq[c]));
    }
    M[int64_t(b) * (p + 1) + k] = zscale(acc, 1.0 / k);
}

__global__ void k_ap2m(int nleaf, const int* __restrict__ leafbox, const double* __restrict__ q, int p,
                       double* __restrict__ S, double2* __restrict__ M) {
    ap2m_body(blockIdx.x, threadIdx.x, nleaf, leafbox, q, p, S, M);
}

// M2M for the internal boxes in [b0, b1): thread k of CTA (b - b0) forms the parent's M_k.
__host__ __device__ inline void am2m_body(int blk, int k, int b0, int b1, const int* __restrict__ first_child,
                                          const AGeo* __restrict__ geo, int p, double* __restrict__ S,
                                          double2* __restrict__ M) {
    const int b = b0 + blk;
    if (b >= b1 || k > p) return;
    const int fc = first_child[b];
    if (fc < 0) return;  // a leaf: its expansion came from P2M
    double2 acc{0.0, 0.0};
    double ssum = 0.0;
    for (int ch = fc; ch < fc + 4; ++ch) {
        const double Sc = S[ch];
        ssum += Sc;
        if (k == 0) continue;
        const double2 u{(geo[ch].cx - geo[b].cx) / geo[b].s, (geo[ch].cy - geo[b].cy) / geo[b].s};
        // S u^k / k
        double2 uk = u;
        for (int j = 1; j < k; ++j) uk = zmul(uk, u);
        acc = zadd(acc, zscale(uk, Sc / k));
        // sum_{l=1..k} M_l 2^-l u^(k-l) C(k-1, l-1), u^(k-l) built downwards from u^0
        double binom = 1.0;  // C(k-1, l-1) at l = 1
        for (int l = 1; l <= k; ++l) {
            double2 ukl{1.0, 0.0};
            for (int j = 0; j < k - l; ++j) ukl = zmul(ukl, u);
            const double2 ml = M[int64_t(ch) * (p + 1) + l];
            acc = zadd(acc, zscale(zmul(ml, ukl), ldexp(binom, -l)));
            binom = binom * double(k - l) / double(l);  // C(k-1, l) from C(k-1, l-1)
        }
    }
    if (k == 0) {
        S[b] = ssum;
        M[int64_t(b) * (p + 1)] = double2{0.0, 0.0};
    } else {
        M[int64_t(b) * (p + 1) + k] = acc;
    }
}

__global__ void k_am2m(int b0, int b1, const int* __restrict__ first_child, const AGeo* __restrict__ geo, int p,
                       double* __restrict__ S, double2* __restrict__ M) {
    am2m_body(blockIdx.x, threadIdx.x, b0, b1, first_child, geo, p, S, M);
}

// M2L: CTA per target box, thread l forms L_l from the box's sources in list order.
__host__ __device__ inline void am2l_body(int a, int l, int nb, const int* __restrict__ ptr,
                                          const int* __restrict__ src, const AGeo* __restrict__ geo, int p,
                                          const double* __restrict__ S, const double2* __restrict__ M,
                                          double2* __restrict__ L) {
    if (a >= nb || l > p) return;
    double2 acc{0.0, 0.0};
    for (int e = ptr[a]; e < ptr[a + 1]; ++e) {
        const int b = src[e];
        const double st = geo[a].s;
        const double2 tau{(geo[b].cx - geo[a].cx) / st, (geo[b].cy - geo[a].cy) / st};
        const double rho = geo[b].s / st;
        const double2 rt = zscale(zinv(tau), rho);  // rho / tau
        const double Sb = S[b];
        // sum_k x_k C(l+k-1, k-1), x_k = -M_k (-1)^k (rho/tau)^k
        double2 sum{0.0, 0.0};
        double2 pw = rt;
        double binom = 1.0;  // C(l+k-1, k-1) at k = 1
        for (int k = 1; k <= p; ++k) {
            const double2 x = zscale(zmul(M[int64_t(b) * (p + 1) + k], pw), (k & 1) ? 1.0 : -1.0);
            sum = zadd(sum, l == 0 ? x : zscale(x, binom));
            pw = zmul(pw, rt);
            binom = binom * double(l + k) / double(k);  // C(l+k, k) from C(l+k-1, k-1)
        }
        if (l == 0) {
            const double lt = 0.5 * log(tau.x * tau.x + tau.y * tau.y) + log(st);
            acc = zadd(acc, zadd(double2{Sb * lt, 0.0}, sum));
        } else {
            double2 tl = zinv(tau);  // tau^-l
            const double2 ti = tl;
            for (int j = 1; j < l; ++j) tl = zmul(tl, ti);
            acc = zadd(acc, zmul(tl, zadd(double2{-Sb / l, 0.0}, sum)));
        }
    }
    L[int64_t(a) * (p + 1) + l] = acc;
}

__global__ void k_am2l(int nb, const int* __restrict__ ptr, const int* __restrict__ src, const AGeo* __restrict__ geo,
                       int p, const double* __restrict__ S, const double2* __restrict__ M, double2* __restrict__ L) {
    am2l_body(blockIdx.x, threadIdx.x, nb, ptr, src, geo, p, S, M, L);
}

// L2L for the boxes in [b0, b1) (one level, parents final): thread l of CTA (b - b0).
__host__ __device__ inline void al2l_body(int blk, int l, int b0, int b1, const int* __restrict__ parent,
                                          const AGeo* __restrict__ geo, int p, double2* __restrict__ L) {
    const int b = b0 + blk;
    if (b >= b1 || l > p) return;
    const int pa = parent[b];
    if (pa < 0) return;
    const double2 v{(geo[b].cx - geo[pa].cx) / geo[pa].s, (geo[b].cy - geo[pa].cy) / geo[pa].s};
    double2 acc{0.0, 0.0};
    double2 vp{1.0, 0.0};  // v^(k-l)
    double binom = 1.0;    // C(k, l) at k = l
    for (int k = l; k <= p; ++k) {
        acc = zadd(acc, zscale(zmul(L[int64_t(pa) * (p + 1) + k], vp), binom));
        vp = zmul(vp, v);
        binom = binom * double(k + 1) / double(k + 1 - l);  // C(k+1, l) from C(k, l)
    }
    L[int64_t(b) * (p + 1) + l] = zadd(L[int64_t(b) * (p + 1) + l], zscale(acc, ldexp(1.0, -l)));
}

__global__ void k_al2l(int b0, int b1, const int* __restrict__ parent, const AGeo* __restrict__ geo, int p,
                       double2* __restrict__ L) {
    al2l_body(blockIdx.x, threadIdx.x, b0, b1, parent, geo, p, L);
}

// Leaves: CTA of 64 threads per leaf, thread = target cell: local expansion, then the near
// field over the leaf's near-field sources in list order (sources clamped at their own rho_h).
// tab: (2R + 1)^2 values T[dy][dx] = log sqrt(dx^2 + dy^2) for |dx|, |dy| <= R (T[0][0] = c0),
// R covering every same-level near-field offset; S: leaf sums of q (from P2M).
__host__ __device__ inline void aleaf_body(int i, int c, int nleaf, const int* __restrict__ leafbox,
                                           const int* __restrict__ ptr, const int* __restrict__ src,
                                           const AGeo* __restrict__ geo, int p, const double2* __restrict__ L,
                                           const double* __restrict__ tab, int R, const double* __restrict__ S,
                                           const double* __restrict__ q, double* __restrict__ p_out) {
    if (i >= nleaf || c >= 64) return;
    const int b = leafbox[i];
    const AGeo g = geo[b];
    const double2 w = cell_w(c);
    // Horner: Re sum_l L_l w^l
    double2 h = L[int64_t(b) * (p + 1) + p];
    for (int l = p - 1; l >= 0; --l) h = zadd(zmul(h, w), L[int64_t(b) * (p + 1) + l]);
    const double xt = g.cx + g.s * w.x, yt = g.cy + g.s * w.y;
    const double logh = log(g.s / 8.0);
    const int W = 2 * R + 1;
    double near = 0.0;
    for (int e = ptr[i]; e < ptr[i + 1]; ++e) {
        const int j = src[e];
        const int bj = leafbox[j];
        const AGeo gs = geo[bj];
        const double* qs = q + int64_t(j) * 64;
        if (gs.level == g.level) {  // offsets (source cell - target cell) in cells, |.| <= R
            const int ox = 8 * (gs.ix - g.ix) - (c & 7) + R, oy = 8 * (gs.iy - g.iy) - (c >> 3) + R;
            double t = 0.0;
            for (int cs = 0; cs < 64; ++cs) t += qs[cs] * tab[(oy + (cs >> 3)) * W + ox + (cs & 7)];
            near += S[bj] * logh + t;
        } else {
            const double rho = gs.s / 8.0 * exp(kC0A);
            for (int cs = 0; cs < 64; ++cs) {
                const double2 ws = cell_w(cs);
                const double dx = xt - (gs.cx + gs.s * ws.x), dy = yt - (gs.cy + gs.s * ws.y);
                const double r = fmax(sqrt(dx * dx + dy * dy), rho);
                near += qs[cs] * log(r);
            }
        }
    }
    p_out[int64_t(i) * 64 + c] = (h.x + near) * kInv2PiA;
}

__global__ void k_aleaf(int nleaf, const int* __restrict__ leafbox, const int* __restrict__ ptr,
                        const int* __restrict__ src, const AGeo* __restrict__ geo, int p,
                        const double2* __restrict__ L, const double* __restrict__ tab, int R,
                        const double* __restrict__ S, const double* __restrict__ q, double* __restrict__ p_out) {
    aleaf_body(blockIdx.x, threadIdx.x, nleaf, leafbox, ptr, src, geo, p, L, tab, R, S, q, p_out);
}

// Surface pressure at off-grid points by the tree-code over the adaptive tree (Sec. 2.3.1's
// targets; Appendix A.2's group acceptance): depth-first from the root, a box is accepted for
// the point when its half-diagonal r is below theta d (d the distance from its centre) and its
// multipole is evaluated there, S log|w| - Re sum_k M_k (s / w)^k with w = z - c (Eq.
// pressTruncated about the box centre); a leaf that is not accepted is summed directly over its
// 64 cells, each clamped at its own rho_h; any other box opens its four children.  One thread
// per point; the stack holds at most 3 boxes per level plus 4.
constexpr int kSurfStack = 3 * 21 + 4;

__host__ __device__ inline void asurf_body(int i, int npts, const double* __restrict__ pts, const AGeo* __restrict__ geo,
                                           const int* __restrict__ fchild, const int* __restrict__ boxleaf, int p,
                                           const double* __restrict__ S, const double2* __restrict__ M,
                                           const double* __restrict__ q, double theta, double* __restrict__ P_out,
                                           bool* overflow_out) {
    if (i >= npts) return;
    const double zx = pts[2 * i], zy = pts[2 * i + 1];
    int stack[kSurfStack];
    int top = 0;
    stack[top++] = 0;
    double acc = 0.0;
    bool overflow = false;
    const double th2 = theta * theta;
    while (top > 0) {
        const int b = stack[--top];
        const AGeo g = geo[b];
        const double dx = zx - g.cx, dy = zy - g.cy;
        const double d2 = dx * dx + dy * dy;
        if (0.5 * g.s * g.s < th2 * d2) {
            // u = s / w; Horner for sum_k M_k u^k
            const double2 u = zscale(double2{dx / d2, -dy / d2}, g.s);
            const double2* Mb = M + int64_t(b) * (p + 1);
            double2 h = Mb[p];
            for (int k = p - 1; k >= 1; --k) h = zadd(zmul(h, u), Mb[k]);
            const double2 ser = zmul(h, u);
            acc += S[b] * 0.5 * log(d2) - ser.x;
        } else if (fchild[b] < 0) {
            const int lf = boxleaf[b];
            const double* qs = q + int64_t(lf) * 64;
            const double rho = g.s / 8.0 * exp(kC0A);
            for (int c = 0; c < 64; ++c) {
                const double2 w = cell_w(c);
                const double ex = zx - (g.cx + g.s * w.x), ey = zy - (g.cy + g.s * w.y);
                acc += qs[c] * log(fmax(sqrt(ex * ex + ey * ey), rho));
            }
        } else if (top + 4 <= kSurfStack) {
            for (int c = 3; c >= 0; --c) stack[top++] = fchild[b] + c;
        } else {
            overflow = true;
        }
    }
    P_out[i] = acc * kInv2PiA;
    *overflow_out = overflow;
}

__global__ void k_asurf(int npts, const double* __restrict__ pts, const AGeo* __restrict__ geo,
                        const int* __restrict__ fchild, const int* __restrict__ boxleaf, int p,
                        const double* __restrict__ S, const double2* __restrict__ M, const double* __restrict__ q,
                        double theta, double* __restrict__ P_out, int* __restrict__ err) {
    bool overflow = false;
    asurf_body(blockIdx.x * blockDim.x + threadIdx.x, npts, pts, geo, fchild, boxleaf, p, S, M, q, theta, P_out,
               &overflow);
    if (overflow) atomicExch(err, 1);
}

template <typename T>
cudaError_t upload(std::vector<void*>& bufs, T** dst, const std::vector<T>& src, cudaStream_t st) {
    const size_t bytes = sizeof(T) * (src.empty() ? 1 : src.size());
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), bytes);
    if (e != cudaSuccess) return e;
    bufs.push_back(*dst);
    if (!src.empty()) e = cudaMemcpyAsync(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, st);
    return e;
}

// Host arrays of one solve: box geometry, leaf -> box, level ranges (boxes are stored level by
// level, parents first), and both interaction lists as CSR by target.
struct AdaptivePrep {
    int nb = 0, nleaf = 0, L = 0, R = 0;
    std::vector<AGeo> geo;
    std::vector<int> fchild, parent, leafbox, boxleaf, lev_start, m2l_ptr, m2l_src, p2p_ptr, p2p_src;
    std::vector<double> tab;  // the same-level near-field table, (2R + 1)^2
};

int prepare_adaptive(pp_atree tree, AdaptivePrep& a) {
    int64_t sz[4];
    if (pp_atree_sizes(tree, sz) != PP_OK) return PP_ERR_ARG;
    const int nb = int(sz[0]), nm = int(sz[1]), np2 = int(sz[2]), L = int(sz[3]);
    try {
        std::vector<int> level(nb), ix(nb), iy(nb), leaf(nb), m2l(2 * size_t(nm)), p2p(2 * size_t(np2));
        a.parent.resize(nb);
        a.fchild.resize(nb);
        pp_atree_boxes(tree, level.data(), ix.data(), iy.data(), a.parent.data(), a.fchild.data(), leaf.data());
        pp_atree_lists(tree, m2l.data(), p2p.data());
        a.nb = nb;
        a.L = L;
        a.nleaf = 0;
        for (int b = 0; b < nb; ++b) a.nleaf += leaf[b] >= 0;
        a.geo.resize(nb);
        a.leafbox.assign(a.nleaf, -1);
        a.boxleaf = leaf;
        a.lev_start.assign(L + 2, nb);
        a.m2l_ptr.assign(nb + 1, 0);
        a.m2l_src.resize(nm);
        a.p2p_ptr.assign(a.nleaf + 1, 0);
        a.p2p_src.resize(np2);
        for (int b = nb - 1; b >= 0; --b) a.lev_start[level[b]] = b;
        for (int b = 0; b < nb; ++b) {
            const double s = std::ldexp(1.0, -level[b]);
            a.geo[b] = AGeo{(ix[b] + 0.5) * s, (iy[b] + 0.5) * s, s, level[b], ix[b], iy[b]};
            if (leaf[b] >= 0) a.leafbox[leaf[b]] = b;
        }
        for (int e = 0; e < nm; ++e) {  // pairs are sorted by target
            ++a.m2l_ptr[m2l[2 * e] + 1];
            a.m2l_src[e] = m2l[2 * e + 1];
        }
        for (int b = 0; b < nb; ++b) a.m2l_ptr[b + 1] += a.m2l_ptr[b];
        for (int e = 0; e < np2; ++e) {
            ++a.p2p_ptr[p2p[2 * e] + 1];
            a.p2p_src[e] = p2p[2 * e + 1];
        }
        for (int i = 0; i < a.nleaf; ++i) a.p2p_ptr[i + 1] += a.p2p_ptr[i];
        // the largest same-level near-field leaf offset, and the table of log|D| over cell offsets
        int dmax = 0;
        for (int e = 0; e < np2; ++e) {
            const AGeo& gt = a.geo[a.leafbox[p2p[2 * e]]];
            const AGeo& gs = a.geo[a.leafbox[p2p[2 * e + 1]]];
            if (gt.level == gs.level) dmax = std::max(dmax, std::max(std::abs(gs.ix - gt.ix), std::abs(gs.iy - gt.iy)));
        }
        a.R = 8 * dmax + 7;
        const int W = 2 * a.R + 1;
        a.tab.resize(size_t(W) * W);
        for (int dy = -a.R; dy <= a.R; ++dy)
            for (int dx = -a.R; dx <= a.R; ++dx)
                a.tab[size_t(dy + a.R) * W + dx + a.R] =
                    (dx == 0 && dy == 0) ? kC0A : 0.5 * std::log(double(dx * dx + dy * dy));
    } catch (const std::bad_alloc&) {
        return PP_ERR_OOM;
    }
    return PP_OK;
}

// What a tree keeps between solves: the prepared arrays on the device and the expansions
// (sized for the largest order solved so far).
struct AdaptiveState {
    AdaptivePrep a;
    std::vector<void*> bufs;
    int *d_leafbox = nullptr, *d_fchild = nullptr, *d_parent = nullptr, *d_mptr = nullptr, *d_msrc = nullptr,
        *d_pptr = nullptr, *d_psrc = nullptr, *d_boxleaf = nullptr, *d_err = nullptr;
    AGeo* d_geo = nullptr;
    double *d_tab = nullptr, *d_S = nullptr;
    double2 *d_M = nullptr, *d_L = nullptr;
    int p_cap = 0;
    int last_p = 0;  // order of the last solve: the multipoles the surface tree-code reads
    // mixed-precision solve (set up on its first call): FP32 expansions with the FP64 monopoles
    // and constant terms, per-pair translation geometry, the shift and P2M tables, the FP32
    // near-field table
    bool mixed_ready = false;
    float2 *d_Mf = nullptr, *d_Lf = nullptr;
    double* d_L0 = nullptr;
    float4* d_mgeo = nullptr;   // per M2L pair: tau (target side units), rho, unused
    double* d_mlog = nullptr;   // per M2L pair: log|tau| + log s_target
    float2 *d_Wf = nullptr, *d_Af = nullptr, *d_Bf = nullptr, *d_Cf = nullptr;
    float* d_tabf = nullptr;
};

void release_state(void* v) {
    AdaptiveState* s = static_cast<AdaptiveState*>(v);
    for (void* b : s->bufs) cudaFree(b);
    cudaFree(s->d_M);
    cudaFree(s->d_L);
    delete s;
}

// Host tables of the mixed-precision solve, order up to kMaxOrderA (stride kTP = 31), built in
// FP64: W[c][k] = w_c^k / k (P2M at the 64 cells), and per child quadrant q with
// u_q = (c_child - c_parent) / s_parent = (+-1/4, +-1/4):
//   B[q][k] = u_q^k / k, A[q][l][k] = 2^-l u_q^(k-l) C(k-1, l-1) (M2M),
//   C[q][k][l] = 2^-l C(k, l) u_q^(k-l) (L2L).
constexpr int kTP = kMaxOrderA + 1;

struct MixedTables {
    std::vector<float2> W, A, B, C;
};

MixedTables mixed_tables() {
    MixedTables t;
    t.W.assign(size_t(64) * kTP, float2{0.f, 0.f});
    t.A.assign(size_t(4) * kTP * kTP, float2{0.f, 0.f});
    t.B.assign(size_t(4) * kTP, float2{0.f, 0.f});
    t.C.assign(size_t(4) * kTP * kTP, float2{0.f, 0.f});
    auto f2 = [](double2 z) { return float2{float(z.x), float(z.y)}; };
    auto zpow = [](double2 z, int k) {
        double2 r{1.0, 0.0};
        for (int j = 0; j < k; ++j) r = zmul(r, z);
        return r;
    };
    auto binom = [](int n, int r) {
        double c = 1.0;
        for (int i = 1; i <= r; ++i) c = c * double(n - r + i) / double(i);
        return c;
    };
    for (int c = 0; c < 64; ++c)
        for (int k = 1; k < kTP; ++k) t.W[size_t(c) * kTP + k] = f2(zscale(zpow(cell_w(c), k), 1.0 / k));
    for (int q = 0; q < 4; ++q) {
        const double2 u{((q & 1) - 0.5) * 0.5, ((q >> 1) - 0.5) * 0.5};
        for (int k = 1; k < kTP; ++k) {
            t.B[size_t(q) * kTP + k] = f2(zscale(zpow(u, k), 1.0 / k));
            for (int l = 1; l <= k; ++l)
                t.A[(size_t(q) * kTP + l) * kTP + k] = f2(zscale(zpow(u, k - l), std::ldexp(binom(k - 1, l - 1), -l)));
        }
        for (int k = 0; k < kTP; ++k)
            for (int l = 0; l <= k; ++l)
                t.C[(size_t(q) * kTP + k) * kTP + l] = f2(zscale(zpow(u, k - l), std::ldexp(binom(k, l), -l)));
    }
    return t;
}

cudaError_t setup_mixed(AdaptiveState* s, cudaStream_t st) {
    const AdaptivePrep& a = s->a;
    std::vector<float4> mg(a.m2l_src.size());
    std::vector<double> ml(a.m2l_src.size());
    for (int t = 0; t < a.nb; ++t)
        for (int e = a.m2l_ptr[t]; e < a.m2l_ptr[t + 1]; ++e) {
            const AGeo& gt = a.geo[t];
            const AGeo& gs = a.geo[a.m2l_src[e]];
            const double tx = (gs.cx - gt.cx) / gt.s, ty = (gs.cy - gt.cy) / gt.s;
            mg[e] = make_float4(float(tx), float(ty), float(gs.s / gt.s), 0.f);
            ml[e] = 0.5 * std::log(tx * tx + ty * ty) + std::log(gt.s);
        }
    std::vector<float> tf(a.tab.size());
    for (size_t i = 0; i < tf.size(); ++i) tf[i] = float(a.tab[i]);
    const MixedTables mt = mixed_tables();
    cudaError_t e;
    if ((e = upload(s->bufs, &s->d_mgeo, mg, st)) || (e = upload(s->bufs, &s->d_mlog, ml, st)) ||
        (e = upload(s->bufs, &s->d_tabf, tf, st)) || (e = upload(s->bufs, &s->d_Wf, mt.W, st)) ||
        (e = upload(s->bufs, &s->d_Af, mt.A, st)) || (e = upload(s->bufs, &s->d_Bf, mt.B, st)) ||
        (e = upload(s->bufs, &s->d_Cf, mt.C, st)))
        return e;
    const size_t ne = size_t(a.nb) * kTP;
    if ((e = cudaMalloc(reinterpret_cast<void**>(&s->d_Mf), sizeof(float2) * ne)) != cudaSuccess) return e;
    s->bufs.push_back(s->d_Mf);
    if ((e = cudaMalloc(reinterpret_cast<void**>(&s->d_Lf), sizeof(float2) * ne)) != cudaSuccess) return e;
    s->bufs.push_back(s->d_Lf);
    if ((e = cudaMalloc(reinterpret_cast<void**>(&s->d_L0), sizeof(double) * a.nb)) != cudaSuccess) return e;
    s->bufs.push_back(s->d_L0);
    return cudaSuccess;
}

cudaError_t setup_state(AdaptiveState* s, cudaStream_t st) {
    const AdaptivePrep& a = s->a;
    cudaError_t e;
    if ((e = upload(s->bufs, &s->d_leafbox, a.leafbox, st)) || (e = upload(s->bufs, &s->d_fchild, a.fchild, st)) ||
        (e = upload(s->bufs, &s->d_parent, a.parent, st)) || (e = upload(s->bufs, &s->d_mptr, a.m2l_ptr, st)) ||
        (e = upload(s->bufs, &s->d_msrc, a.m2l_src, st)) || (e = upload(s->bufs, &s->d_pptr, a.p2p_ptr, st)) ||
        (e = upload(s->bufs, &s->d_psrc, a.p2p_src, st)) || (e = upload(s->bufs, &s->d_geo, a.geo, st)) ||
        (e = upload(s->bufs, &s->d_tab, a.tab, st)) || (e = upload(s->bufs, &s->d_boxleaf, a.boxleaf, st)))
        return e;
    if ((e = cudaMalloc(reinterpret_cast<void**>(&s->d_err), sizeof(int))) != cudaSuccess) return e;
    s->bufs.push_back(s->d_err);
    if ((e = cudaMalloc(reinterpret_cast<void**>(&s->d_S), sizeof(double) * a.nb)) != cudaSuccess) return e;
    s->bufs.push_back(s->d_S);
    return cudaSuccess;
}

// ------------------------------------------------------------------------------------
// Mixed precision: the same steps with FP32 expansions (and FP32 q and output), the box
// monopoles S and the constant terms L_0 in FP64 (they carry the log terms whose sum
// cancels across the domain), the shifts and the leaf P2M from the FP64-built tables, the
// translations' geometry per pair from the host, the near field in FP32 with compensated
// sums.  One warp (32 threads) per box for the expansion steps, thread k forming coefficient
// k; 64 threads per leaf, one per cell, for the evaluation.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 cfmaf(float2 a, float2 b, float2 c) {  // a b + c
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__device__ __forceinline__ int child_quadrant(const AGeo& g) { return (g.ix & 1) + 2 * (g.iy & 1); }

// P2M: S (FP64 of the FP32 warp sum) and M_k = sum_c q_c w_c^k / k from the table.
__global__ void k_ap2m_f(int nleaf, const int* __restrict__ leafbox, const float* __restrict__ q, int p,
                         const float2* __restrict__ W, double* __restrict__ S, float2* __restrict__ M) {
    const int i = blockIdx.x, k = threadIdx.x;
    const float* qq = q + int64_t(i) * 64;
    const int b = leafbox[i];
    float s = qq[k] + qq[k + 32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (k == 0) {
        S[b] = double(s);
        M[int64_t(b) * kTP] = make_float2(0.f, 0.f);
    } else if (k <= p) {
        float2 acc = make_float2(0.f, 0.f);
        for (int c = 0; c < 64; ++c) {
            const float2 w = W[c * kTP + k];
            acc.x = fmaf(qq[c], w.x, acc.x);
            acc.y = fmaf(qq[c], w.y, acc.y);
        }
        M[int64_t(b) * kTP + k] = acc;
    }
}

// M2M for the internal boxes in [b0, b1): M_k = sum_children [S u^k / k + sum_{l<=k} A[q][l][k] M_l].
__global__ void k_am2m_f(int b0, int b1, const int* __restrict__ first_child, const AGeo* __restrict__ geo, int p,
                         const float2* __restrict__ A, const float2* __restrict__ B, double* __restrict__ S,
                         float2* __restrict__ M) {
    const int b = b0 + blockIdx.x, k = threadIdx.x;
    const int fc = first_child[b];
    if (fc < 0 || k > p) return;  // a leaf: its expansion came from P2M
    float2 acc = make_float2(0.f, 0.f);
    double ssum = 0.0;
    for (int ch = fc; ch < fc + 4; ++ch) {
        const double Sc = S[ch];
        ssum += Sc;
        if (k == 0) continue;
        const int q = child_quadrant(geo[ch]);
        const float2 bk = B[q * kTP + k];
        acc.x = fmaf(float(Sc), bk.x, acc.x);
        acc.y = fmaf(float(Sc), bk.y, acc.y);
        const float2* Mc = M + int64_t(ch) * kTP;
        const float2* Aq = A + size_t(q) * kTP * kTP;
        for (int l = 1; l <= k; ++l) acc = cfmaf(Aq[l * kTP + k], Mc[l], acc);
    }
    if (k == 0) {
        S[b] = ssum;
        M[int64_t(b) * kTP] = make_float2(0.f, 0.f);
    } else {
        M[int64_t(b) * kTP + k] = acc;
    }
}

// M2L: one warp per target box.  Per pair (tau, rho from the host, in target-side units):
// thread k forms x_k = -M_k (-1)^k (rho / tau)^k into shared memory; thread l >= 1 adds
// tau^-l (-S / l + sum_k x_k C(l+k-1, k-1)); thread 0 adds S (log|tau| + log s) + Re sum_k x_k
// to the FP64 constant.
__global__ void k_am2l_f(int nb, const int* __restrict__ ptr, const int* __restrict__ src,
                         const float4* __restrict__ mgeo, const double* __restrict__ mlog, int p,
                         const double* __restrict__ S, const float2* __restrict__ M, float2* __restrict__ L,
                         double* __restrict__ L0) {
    __shared__ float2 xs[32];
    const int a = blockIdx.x, t = threadIdx.x;
    float2 acc = make_float2(0.f, 0.f);
    double acc0 = 0.0;
    for (int e = ptr[a]; e < ptr[a + 1]; ++e) {
        const int b = src[e];
        const float4 g = mgeo[e];
        const float d = g.x * g.x + g.y * g.y;
        const float2 ti = make_float2(g.x / d, -g.y / d);  // 1 / tau
        const double Sb = S[b];
        float2 x = make_float2(0.f, 0.f);
        if (t >= 1 && t <= p) {
            const float2 rt = make_float2(g.z * ti.x, g.z * ti.y);  // rho / tau
            float2 pw = rt;
            for (int j = 1; j < t; ++j) pw = cmulf(pw, rt);
            x = cmulf(M[int64_t(b) * kTP + t], pw);
            if (!(t & 1)) x = make_float2(-x.x, -x.y);  // -M_k (-1)^k: the sign flips for even k
        }
        xs[t] = x;
        __syncwarp();
        if (t == 0) {
            float r = 0.f;
            for (int k = 1; k <= p; ++k) r += xs[k].x;
            acc0 += Sb * mlog[e] + double(r);
        } else if (t <= p) {
            float2 sum = make_float2(0.f, 0.f);
            float binom = 1.f;  // C(l+k-1, k-1) at k = 1
            for (int k = 1; k <= p; ++k) {
                sum.x = fmaf(binom, xs[k].x, sum.x);
                sum.y = fmaf(binom, xs[k].y, sum.y);
                binom = binom * float(t + k) / float(k);
            }
            sum.x -= float(Sb) / float(t);
            float2 tl = ti;  // tau^-l
            for (int j = 1; j < t; ++j) tl = cmulf(tl, ti);
            acc = cfmaf(tl, sum, acc);
        }
        __syncwarp();
    }
    if (t == 0) L0[a] = acc0;
    else if (t <= p) L[int64_t(a) * kTP + t] = acc;
}

// L2L for the boxes in [b0, b1) (parents final): L_l += sum_{k>=l} C[q][k][l] L_k(parent), and the
// FP64 constant L_0 += L_0(parent) + Re sum_{k>=1} C[q][k][0] L_k(parent).
__global__ void k_al2l_f(int b0, int b1, const int* __restrict__ parent, const AGeo* __restrict__ geo, int p,
                         const float2* __restrict__ C, float2* __restrict__ L, double* __restrict__ L0) {
    const int b = b0 + blockIdx.x, l = threadIdx.x;
    const int pa = parent[b];
    if (pa < 0 || l > p) return;
    const int q = child_quadrant(geo[b]);
    const float2* Lp = L + int64_t(pa) * kTP;
    const float2* Cq = C + size_t(q) * kTP * kTP;
    float2 acc = make_float2(0.f, 0.f);
    for (int k = (l == 0 ? 1 : l); k <= p; ++k) acc = cfmaf(Cq[k * kTP + l], Lp[k], acc);
    if (l == 0) {
        L0[b] += L0[pa] + double(acc.x);
    } else {
        float2* Lb = L + int64_t(b) * kTP + l;
        *Lb = make_float2(Lb->x + acc.x, Lb->y + acc.y);
    }
}

// Leaves: 64 threads per leaf, one per cell: Re sum_{l>=1} L_l w^l (FP32 Horner) plus the FP64
// constant, and the near field in FP32 with a compensated sum: same-level source leaves from
// the FP32 table of log|D| (their log h part, S log h, in FP64), other levels directly.
__global__ void k_aleaf_f(int nleaf, const int* __restrict__ leafbox, const int* __restrict__ ptr,
                          const int* __restrict__ src, const AGeo* __restrict__ geo, int p,
                          const float2* __restrict__ L, const double* __restrict__ L0, const float* __restrict__ tab,
                          int R, const double* __restrict__ S, const float* __restrict__ q, float* __restrict__ p_out) {
    const int i = blockIdx.x, c = threadIdx.x;
    const int b = leafbox[i];
    const AGeo g = geo[b];
    const float wx = ((c & 7) + 0.5f) * 0.125f - 0.5f, wy = ((c >> 3) + 0.5f) * 0.125f - 0.5f;
    const float2* Lb = L + int64_t(b) * kTP;
    float2 h = Lb[p];
    for (int l = p - 1; l >= 1; --l) h = cfmaf(h, make_float2(wx, wy), Lb[l]);
    const float ser = h.x * wx - h.y * wy;
    const double logh = log(g.s / 8.0);
    const int W = 2 * R + 1;
    float sum = 0.f, comp = 0.f;  // Kahan
    double slog = 0.0;            // sum of S log h over the same-level source leaves
    for (int e = ptr[i]; e < ptr[i + 1]; ++e) {
        const int j = src[e];
        const int bj = leafbox[j];
        const AGeo gs = geo[bj];
        const float* qs = q + int64_t(j) * 64;
        float t = 0.f;
        if (gs.level == g.level) {  // offsets (source cell - target cell) in cells, |.| <= R
            const int ox = 8 * (gs.ix - g.ix) - (c & 7) + R, oy = 8 * (gs.iy - g.iy) - (c >> 3) + R;
            for (int cs = 0; cs < 64; ++cs) t = fmaf(qs[cs], tab[(oy + (cs >> 3)) * W + ox + (cs & 7)], t);
            slog += S[bj];
        } else {
            // source cell centres relative to the target cell, in units of the target's cell side
            const double hc = g.s / 8.0;
            const float ox = float((gs.cx - 0.5 * gs.s - (g.cx + g.s * double(wx))) / hc);
            const float oy = float((gs.cy - 0.5 * gs.s - (g.cy + g.s * double(wy))) / hc);
            const float step = float(gs.s / 8.0 / hc);   // source cell side / target cell side
            const float rho = step * 0.34604881609982794f;  // rho_h of the source cell: exp(pi/4 - 3/2 - ln2/2) h
            const float lhc = float(log(hc));
            for (int cs = 0; cs < 64; ++cs) {
                const float dx = ox + ((cs & 7) + 0.5f) * step, dy = oy + ((cs >> 3) + 0.5f) * step;
                const float r = fmaxf(sqrtf(dx * dx + dy * dy), rho);
                t = fmaf(qs[cs], logf(r) + lhc, t);
            }
        }
        const float y = t - comp;
        const float tt = sum + y;
        comp = (tt - sum) - y;
        sum = tt;
    }
    p_out[int64_t(i) * 64 + c] = float((L0[b] + slog * logh + double(ser) + double(sum)) * kInv2PiA);
}

}  // namespace

extern "C" int pp_atree_solve(pp_atree tree, int order, const double* q, double* p_out, void* stream) {
    if (!tree || !q || !p_out || order < 2 || order > kMaxOrderA) return PP_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    AdaptiveState* s = static_cast<AdaptiveState*>(pp::atree_state(tree));
    if (!s) {
        s = new (std::nothrow) AdaptiveState();
        if (!s) return PP_ERR_OOM;
        const int pst = prepare_adaptive(tree, s->a);
        cudaError_t e = pst == PP_OK ? setup_state(s, st) : cudaSuccess;
        if (pst == PP_OK && e == cudaSuccess) e = cudaStreamSynchronize(st);  // uploads done before reuse
        if (pst != PP_OK || e != cudaSuccess) {
            release_state(s);
            cudaGetLastError();
            return pst != PP_OK ? pst : e == cudaErrorMemoryAllocation ? PP_ERR_OOM : PP_ERR_CUDA;
        }
        pp::atree_set_state(tree, s, release_state);
    }
    const AdaptivePrep& a = s->a;
    const int nb = a.nb, nleaf = a.nleaf, L = a.L, p = order;
    if (p > s->p_cap) {  // expansions for a higher order than before
        cudaStreamSynchronize(st);
        cudaFree(s->d_M);
        cudaFree(s->d_L);
        s->d_M = s->d_L = nullptr;
        s->p_cap = 0;
        cudaError_t e;
        if ((e = cudaMalloc(reinterpret_cast<void**>(&s->d_M), sizeof(double2) * size_t(nb) * (p + 1))) ||
            (e = cudaMalloc(reinterpret_cast<void**>(&s->d_L), sizeof(double2) * size_t(nb) * (p + 1)))) {
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? PP_ERR_OOM : PP_ERR_CUDA;
        }
        s->p_cap = p;
    }
    if (cudaMemsetAsync(s->d_L, 0, sizeof(double2) * size_t(nb) * (p + 1), st) != cudaSuccess) return PP_ERR_CUDA;
    k_ap2m<<<nleaf, 32, 0, st>>>(nleaf, s->d_leafbox, q, p, s->d_S, s->d_M);
    for (int l = L - 1; l >= 0; --l) {  // upward, deepest internal level first
        const int b0 = a.lev_start[l], b1 = a.lev_start[l + 1];
        if (b1 > b0) k_am2m<<<b1 - b0, 32, 0, st>>>(b0, b1, s->d_fchild, s->d_geo, p, s->d_S, s->d_M);
    }
    k_am2l<<<nb, 32, 0, st>>>(nb, s->d_mptr, s->d_msrc, s->d_geo, p, s->d_S, s->d_M, s->d_L);
    for (int l = 1; l <= L; ++l) {  // downward, parents before children
        const int b0 = a.lev_start[l], b1 = a.lev_start[l + 1];
        if (b1 > b0) k_al2l<<<b1 - b0, 32, 0, st>>>(b0, b1, s->d_parent, s->d_geo, p, s->d_L);
    }
    k_aleaf<<<nleaf, 64, 0, st>>>(nleaf, s->d_leafbox, s->d_pptr, s->d_psrc, s->d_geo, p, s->d_L, s->d_tab, a.R,
                                  s->d_S, q, p_out);
    if (cudaGetLastError() != cudaSuccess) return PP_ERR_CUDA;
    s->last_p = p;
    return PP_OK;
}

extern "C" int pp_atree_solve_mixed(pp_atree tree, int order, const float* q, float* p_out, void* stream) {
    if (!tree || !q || !p_out || order < 2 || order > kMaxOrderA) return PP_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    AdaptiveState* s = static_cast<AdaptiveState*>(pp::atree_state(tree));
    if (!s) {
        s = new (std::nothrow) AdaptiveState();
        if (!s) return PP_ERR_OOM;
        const int pst = prepare_adaptive(tree, s->a);
        cudaError_t e = pst == PP_OK ? setup_state(s, st) : cudaSuccess;
        if (pst == PP_OK && e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (pst != PP_OK || e != cudaSuccess) {
            release_state(s);
            cudaGetLastError();
            return pst != PP_OK ? pst : e == cudaErrorMemoryAllocation ? PP_ERR_OOM : PP_ERR_CUDA;
        }
        pp::atree_set_state(tree, s, release_state);
    }
    if (!s->mixed_ready) {
        cudaError_t e = setup_mixed(s, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // uploads done before the host arrays go
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? PP_ERR_OOM : PP_ERR_CUDA;
        }
        s->mixed_ready = true;
    }
    const AdaptivePrep& a = s->a;
    const int nb = a.nb, nleaf = a.nleaf, L = a.L, p = order;
    if (cudaMemsetAsync(s->d_Lf, 0, sizeof(float2) * size_t(nb) * kTP, st) != cudaSuccess) return PP_ERR_CUDA;
    k_ap2m_f<<<nleaf, 32, 0, st>>>(nleaf, s->d_leafbox, q, p, s->d_Wf, s->d_S, s->d_Mf);
    for (int l = L - 1; l >= 0; --l) {  // upward, deepest internal level first
        const int b0 = a.lev_start[l], b1 = a.lev_start[l + 1];
        if (b1 > b0)
            k_am2m_f<<<b1 - b0, 32, 0, st>>>(b0, b1, s->d_fchild, s->d_geo, p, s->d_Af, s->d_Bf, s->d_S, s->d_Mf);
    }
    k_am2l_f<<<nb, 32, 0, st>>>(nb, s->d_mptr, s->d_msrc, s->d_mgeo, s->d_mlog, p, s->d_S, s->d_Mf, s->d_Lf,
                                s->d_L0);
    for (int l = 1; l <= L; ++l) {  // downward, parents before children
        const int b0 = a.lev_start[l], b1 = a.lev_start[l + 1];
        if (b1 > b0) k_al2l_f<<<b1 - b0, 32, 0, st>>>(b0, b1, s->d_parent, s->d_geo, p, s->d_Cf, s->d_Lf, s->d_L0);
    }
    k_aleaf_f<<<nleaf, 64, 0, st>>>(nleaf, s->d_leafbox, s->d_pptr, s->d_psrc, s->d_geo, p, s->d_Lf, s->d_L0,
                                    s->d_tabf, a.R, s->d_S, q, p_out);
    if (cudaGetLastError() != cudaSuccess) return PP_ERR_CUDA;
    s->last_p = 0;  // the FP64 multipoles no longer match S: the surface tree-code needs an FP64 solve
    return PP_OK;
}

extern "C" int pp_atree_surface_pressure(pp_atree tree, const double* q, int npts, const double* points, double theta,
                                         double* P_out, void* stream) {
    if (!tree || !q || !points || !P_out || npts < 1 || npts > (1 << 24) || !(theta >= 0.25 && theta <= 0.95))
        return PP_ERR_ARG;
    AdaptiveState* s = static_cast<AdaptiveState*>(pp::atree_state(tree));
    if (!s || s->last_p < 1) return PP_ERR_STATE;  // the multipoles come from a solve
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(s->d_err, 0, sizeof(int), st) != cudaSuccess) return PP_ERR_CUDA;
    k_asurf<<<(npts + 127) / 128, 128, 0, st>>>(npts, points, s->d_geo, s->d_fchild, s->d_boxleaf, s->last_p, s->d_S,
                                               s->d_M, q, theta, P_out, s->d_err);
    if (cudaGetLastError() != cudaSuccess) return PP_ERR_CUDA;
    int err = 0;
    if (cudaMemcpyAsync(&err, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return PP_ERR_CUDA;
    return err ? PP_ERR_STATE : PP_OK;
}
