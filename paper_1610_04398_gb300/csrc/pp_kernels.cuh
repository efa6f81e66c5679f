// CUDA kernels of the pressure-recovery path, templated on the real type T
// (double for the FP64 path, float for the mixed path).  Included once per
// precision by pp_kernels_f32.cu / pp_kernels_f64.cu.
#pragma once

#include <cmath>

#include "pp_common.h"

namespace pp {

template <typename C>
__device__ __forceinline__ void cfma(C& acc, const C a, const C b) {
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}

template <typename T>
__device__ __forceinline__ typename cplx_of<T>::type cmake(T x, T y) {
    typename cplx_of<T>::type r;
    r.x = x;
    r.y = y;
    return r;
}

template <typename T> __device__ __forceinline__ T log_t(T x);
template <> __device__ __forceinline__ float log_t<float>(float x) { return logf(x); }
template <> __device__ __forceinline__ double log_t<double>(double x) { return log(x); }

constexpr double kInv2Pi = 0.15915494309189533576888376337251;

// Orders with register-resident translation kernels; other orders use the warp kernels.
#define PP_FAST_ORDERS(X) X(13) X(17) X(21) X(25)

}  // namespace pp

#include "pp_fast.cuh"

namespace pp {

// ------------------------------------------------------------------------------------
// (a1) Poisson source, Eq. PoissonFinal, fused with the leaf multipoles, Eq. alphaK.
// One CTA per 32 x 32 cell tile (a 4 x 4 block of leaves); the tile and its one-cell
// halo are staged in shared memory, so every field is read from HBM once.
// ------------------------------------------------------------------------------------
constexpr int kRT = 32;
constexpr int kRW = kRT + 2;

template <typename T>
__device__ __forceinline__ T d_dx(const T* s, int c, int gi, int n, T inv2h) {
    if (gi == 0) return (T(-3) * s[c] + T(4) * s[c + 1] - s[c + 2]) * inv2h;
    if (gi == n - 1) return (T(3) * s[c] - T(4) * s[c - 1] + s[c - 2]) * inv2h;
    return (s[c + 1] - s[c - 1]) * inv2h;
}

template <typename T>
__device__ __forceinline__ T d_dy(const T* s, int c, int gj, int n, T inv2h) {
    if (gj == 0) return (T(-3) * s[c] + T(4) * s[c + kRW] - s[c + 2 * kRW]) * inv2h;
    if (gj == n - 1) return (T(3) * s[c] - T(4) * s[c - kRW] + s[c - 2 * kRW]) * inv2h;
    return (s[c + kRW] - s[c - kRW]) * inv2h;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_rhs_p2m(Tree<T> t, const T* __restrict__ u, const T* __restrict__ v, const T* __restrict__ chi,
          const T* __restrict__ usx, const T* __restrict__ usy, T rho, T lam, T* __restrict__ f_out) {
    typedef typename cplx_of<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* su = reinterpret_cast<T*>(smem_raw);
    T* sv = su + kRW * kRW;
    T* sa = sv + kRW * kRW;
    T* sb = sa + kRW * kRW;

    const int n = t.n;
    const int P1 = t.P1;
    const int tx0 = blockIdx.x * kRT;
    const int ty0 = blockIdx.y * kRT;
    const int tid = threadIdx.x;

    for (int idx = tid; idx < kRW * kRW; idx += blockDim.x) {
        const int hi = idx % kRW, hj = idx / kRW;
        const int gi = tx0 + hi - 1, gj = ty0 + hj - 1;
        T a = T(0), b = T(0), uu = T(0), vv = T(0);
        if (gi >= 0 && gi < n && gj >= 0 && gj < n) {
            const int64_t g = int64_t(gj) * n + gi;
            uu = u[g];
            vv = v[g];
            const T c = chi[g];
            a = c * (usx[g] - uu);
            b = c * (usy[g] - vv);
        }
        su[idx] = uu;
        sv[idx] = vv;
        sa[idx] = a;
        sb[idx] = b;
    }
    __syncthreads();

    const T inv2h = T(0.5) / T(t.h);
    const T hh = T(t.h) * T(t.h);
    for (int c = tid; c < kRT * kRT; c += blockDim.x) {
        const int li = c % kRT, lj = c / kRT;
        const int gi = tx0 + li, gj = ty0 + lj;
        if (gi >= n || gj >= n) continue;
        const int s = (lj + 1) * kRW + (li + 1);
        const T ux = d_dx(su, s, gi, n, inv2h), uy = d_dy(su, s, gj, n, inv2h);
        const T vx = d_dx(sv, s, gi, n, inv2h), vy = d_dy(sv, s, gj, n, inv2h);
        const T pen = d_dx(sa, s, gi, n, inv2h) + d_dy(sb, s, gj, n, inv2h);
        const T f = -rho * (ux * ux + T(2) * uy * vx + vy * vy) + rho * lam * pen;
        if (f_out) f_out[int64_t(gj) * n + gi] = f;
        const T qq = f * hh;
        const int64_t leaf = int64_t(gj >> 3) * t.nL + (gi >> 3);
        const int64_t qi = leaf * 64 + (gj & 7) * 8 + (gi & 7);
        t.q[qi] = qq;
    }
}

// Leaf multipoles, Eq. alphaK about the leaf centre, scaled by the leaf side:
// S = sum q, M_k = sum q omega^k / k with omega = (cell - centre) / 8.  Eight threads per
// leaf (one per cell row) run the powers of their 8 cells; the row partials are summed
// with shuffles inside each group of 8 lanes.
template <typename T>
__global__ void __launch_bounds__(256) k_p2m(Tree<T> t) {
    typedef typename cplx_of<T>::type C;
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t leaf = g >> 3;
    const int row = int(g & 7);
    const int64_t nleaf = int64_t(t.nL) * t.nL;
    const bool act = leaf < nleaf;
    const int P1 = t.P1;
    T pr[8], pi[8], zr[8];
    const T zi = (T(row) - T(3.5)) * T(0.125);
    T s0 = T(0);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        pr[c] = act ? t.q[leaf * 64 + row * 8 + c] : T(0);
        pi[c] = T(0);
        zr[c] = (T(c) - T(3.5)) * T(0.125);
        s0 += pr[c];
    }
    const int64_t off = level_offset(t.Lleaf);
    for (int o = 1; o < 8; o <<= 1) s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    if (act && row == 0) {
        // FP64 monopole of the leaf (sum of the eight FP32/FP64 row sums)
        store_S_leaf(t, off + leaf, s0);
        t.mp[(off + leaf) * P1] = cmake<T>(s0, T(0));
    }
    for (int k = 1; k < P1; ++k) {
        T ar = T(0), ai = T(0);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const T nr = pr[c] * zr[c] - pi[c] * zi;
            const T ni = pr[c] * zi + pi[c] * zr[c];
            pr[c] = nr;
            pi[c] = ni;
            ar += nr;
            ai += ni;
        }
        for (int o = 1; o < 8; o <<= 1) {
            ar += __shfl_xor_sync(0xffffffffu, ar, o);
            ai += __shfl_xor_sync(0xffffffffu, ai, o);
        }
        if (act && row == (k & 7)) {
            const T ik = T(1) / T(k);
            t.mp[(off + leaf) * P1 + k] = cmake<T>(ar * ik, ai * ik);
        }
    }
}

// The same leaf multipoles with the order known at compile time: the power sums stay in
// registers and one butterfly over the 8 row threads combines them.
template <typename T, int P1>
__global__ void __launch_bounds__(256) k_p2m_reg(Tree<T> t) {
    typedef typename cplx_of<T>::type C;
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t leaf = g >> 3;
    const int row = int(g & 7);
    const bool act = leaf < int64_t(t.nL) * t.nL;
    T pr[8], pi[8], zr[8];
    const T zi = (T(row) - T(3.5)) * T(0.125);
    T ar[P1], ai[P1];
    ar[0] = T(0);
    ai[0] = T(0);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        pr[c] = act ? t.q[leaf * 64 + row * 8 + c] : T(0);
        pi[c] = T(0);
        zr[c] = (T(c) - T(3.5)) * T(0.125);
        ar[0] += pr[c];
    }
#pragma unroll
    for (int k = 1; k < P1; ++k) {
        ar[k] = T(0);
        ai[k] = T(0);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const T nr = pr[c] * zr[c] - pi[c] * zi;
            const T ni = pr[c] * zi + pi[c] * zr[c];
            pr[c] = nr;
            pi[c] = ni;
            ar[k] += nr;
            ai[k] += ni;
        }
    }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1)
#pragma unroll
        for (int k = 0; k < P1; ++k) {
            ar[k] += __shfl_xor_sync(0xffffffffu, ar[k], o);
            ai[k] += __shfl_xor_sync(0xffffffffu, ai[k], o);
        }
    if (!act) return;
    const int64_t base = (level_offset(t.Lleaf) + leaf) * P1;
    if (row == 0) store_S_leaf(t, level_offset(t.Lleaf) + leaf, ar[0]);
#pragma unroll
    for (int k = 0; k < P1; ++k)
        if ((k & 7) == row) t.mp[base + k] = k == 0 ? cmake<T>(ar[0], T(0)) : cmake<T>(ar[k] / T(k), ai[k] / T(k));
}

// ------------------------------------------------------------------------------------
// (a3) Upward pass: children -> parent shift, Eqs. expandedShift/expandedBeta (with the
// S term's sign read as +).  One warp per parent box, lanes over coefficients.
// ------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(128) k_m2m(Tree<T> t, int l) {
    typedef typename cplx_of<T>::type C;
    __shared__ C buf[4][4 * kMaxP1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t b = int64_t(blockIdx.x) * 4 + warp;
    const int side = 1 << l;
    if (b >= int64_t(side) * side) return;
    const int P1 = t.P1;
    const int bx = int(b % side), by = int(b / side);
    const int cs = side * 2;
    const int64_t coff = level_offset(l + 1), poff = level_offset(l);
    C* cb = buf[warp];
    for (int idx = lane; idx < 4 * P1; idx += 32) {
        const int q = idx / P1, k = idx % P1;
        const int64_t child = int64_t(2 * by + (q >> 1)) * cs + 2 * bx + (q & 1);
        cb[idx] = t.mp[(coff + child) * P1 + k];
    }
    __syncwarp();
    for (int k = 1 + lane; k < P1; k += 32) {
        C acc = cmake<T>(T(0), T(0));
        for (int q = 0; q < 4; ++q) {
            const C* A = t.Am2m + int64_t(q) * P1 * P1;
            for (int j = 0; j <= k; ++j) cfma(acc, A[j * P1 + k], cb[q * P1 + j]);
        }
        t.mp[(poff + b) * P1 + k] = acc;
    }
    if (lane == 0) {
        double S = 0.0;
        for (int q = 0; q < 4; ++q) {
            const int64_t child = int64_t(2 * by + (q >> 1)) * cs + 2 * bx + (q & 1);
            S += t.S[coff + child];
        }
        store_S(t, poff + b, S);
        t.mp[(poff + b) * P1] = cmake<T>(T(S), T(0));
    }
}

// ------------------------------------------------------------------------------------
// (a4, a5) Downward pass at level l: local = L2L(parent local) + sum over the
// interaction list of M2L(source multipole).  One warp per target box.
// ------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(128) k_m2l(Tree<T> t, int l) {
    typedef typename cplx_of<T>::type C;
    __shared__ C buf[4][kMaxP1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t b = int64_t(blockIdx.x) * 4 + warp;
    const int side = 1 << l;
    if (b >= int64_t(side) * side) return;
    const int P1 = t.P1;
    const int bx = int(b % side), by = int(b / side);
    const int par = (bx & 1) + 2 * (by & 1);
    const int64_t off = level_offset(l);
    C* sb = buf[warp];
    C acc[2];
    acc[0] = cmake<T>(T(0), T(0));
    acc[1] = cmake<T>(T(0), T(0));
    double a0 = 0.0;

    if (l >= 3) {
        const int64_t pb = level_offset(l - 1) + int64_t(by >> 1) * (side >> 1) + (bx >> 1);
        for (int k = lane; k < P1; k += 32) sb[k] = t.loc[pb * P1 + k];
        __syncwarp();
        const C* Cq = t.Cl2l + int64_t(par) * P1 * P1;
        for (int r = 0; r < 2; ++r) {
            const int ll = lane + 32 * r;
            if (ll >= P1) break;
            for (int k = max(ll, 1); k < P1; ++k) cfma(acc[r], Cq[k * P1 + ll], sb[k]);
        }
        if (lane == 0) a0 = t.L0[pb];
        __syncwarp();
    }

    const double lnS = log(double(t.n) * t.h / double(side));
    const int cnt = t.il_count[par];
    const M2LEntry* lst = t.il + int64_t(par) * t.il_stride;
    for (int e = 0; e < cnt; ++e) {
        const M2LEntry en = lst[e];
        int64_t src;
        if (en.pad == 0) {
            const int sx = bx + en.dx, sy = by + en.dy;
            if (sx < 0 || sy < 0 || sx >= side || sy >= side) continue;
            src = off + int64_t(sy) * side + sx;
        } else {
            const int hs = side >> 1;
            const int sx = (bx >> 1) + en.dx, sy = (by >> 1) + en.dy;
            if (sx < 0 || sy < 0 || sx >= hs || sy >= hs) continue;
            src = level_offset(l - 1) + int64_t(sy) * hs + sx;
        }
        __syncwarp();
        for (int k = lane; k < P1; k += 32) sb[k] = t.mp[src * P1 + k];
        __syncwarp();
        const C* B = t.Bm2l + int64_t(en.op) * P1 * P1;
        for (int r = 0; r < 2; ++r) {
            const int ll = lane + 32 * r;
            if (ll >= P1) break;
            const int k0 = (ll == 0) ? 1 : 0;
            for (int k = k0; k < P1; ++k) cfma(acc[r], B[k * P1 + ll], sb[k]);
        }
        if (lane == 0) a0 += t.S[src] * (lnS + t.lnTau[en.op]);
    }
    for (int r = 0; r < 2; ++r) {
        const int ll = lane + 32 * r;
        if (ll >= P1) break;
        if (ll == 0) {
            const double L0 = a0 + double(acc[0].x);
            t.L0[off + b] = L0;
            t.loc[(off + b) * P1] = cmake<T>(T(L0), T(0));
        } else {
            t.loc[(off + b) * P1 + ll] = acc[r];
        }
    }
}

// ------------------------------------------------------------------------------------
// (a5, a6) Leaf evaluation: local expansion at the 64 cells plus the direct near-field
// sum over the theta-near leaves.  On the uniform grid the kernel between two cells
// depends only on their integer offset, so log max(h|Delta|, rho_h) comes from a table.
// One CTA per row of 4 leaves, one thread per target cell.
// ------------------------------------------------------------------------------------
template <typename T, bool COMP>
__global__ void __launch_bounds__(256) k_leaf(Tree<T> t, int has_far, T* __restrict__ p_out) {
    typedef typename cplx_of<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int D = t.Dmax;
    const int SW = 4 + 2 * D, SH = 2 * D + 1;
    const int QS = 65;  // padded leaf stride: the 4 leaves of a warp hit different banks
    const int KW = 2 * t.Rk + 1;
    const int P1 = t.P1;
    C* sV = reinterpret_cast<C*>(smem_raw);
    C* sL = sV + 64 * P1;
    double* sL0 = reinterpret_cast<double*>(sL + 4 * P1);
    T* sK = reinterpret_cast<T*>(sL0 + 4);
    T* sq = sK + KW * KW;

    const int nL = t.nL;
    const int LX0 = blockIdx.x * 4, LY = blockIdx.y;
    const int tid = threadIdx.x;
    for (int idx = tid; idx < SW * SH * 64; idx += blockDim.x) {
        const int slot = idx >> 6, c = idx & 63;
        const int sx = slot % SW, sy = slot / SW;
        const int LXs = LX0 - D + sx, LYs = LY - D + sy;
        T val = T(0);
        if (LXs >= 0 && LXs < nL && LYs >= 0 && LYs < nL)
            val = t.q[(int64_t(LYs) * nL + LXs) * 64 + c];
        sq[slot * QS + c] = val;
    }
    for (int idx = tid; idx < KW * KW; idx += blockDim.x) sK[idx] = t.Ktab[idx];
    if (has_far) {
        for (int idx = tid; idx < 64 * P1; idx += blockDim.x) sV[idx] = t.Vl2p[idx];
        const int64_t off = level_offset(t.Lleaf);
        for (int idx = tid; idx < 4 * P1; idx += blockDim.x) {
            const int li = idx / P1, k = idx % P1;
            const int LX = LX0 + li;
            sL[idx] = (LX < nL) ? t.loc[(off + int64_t(LY) * nL + LX) * P1 + k] : cmake<T>(T(0), T(0));
        }
        if (tid < 4) sL0[tid] = (LX0 + tid < nL) ? t.L0[off + int64_t(LY) * nL + LX0 + tid] : 0.0;
    }
    __syncthreads();

    const int r = tid >> 5, cc = tid & 31;
    const int li = cc >> 3, cx = cc & 7;
    const int LX = LX0 + li;
    if (LX >= nL) return;

    T acc = T(0), comp = T(0);
    for (int e = 0; e < t.n_near; ++e) {
        const int2 o = t.near[e];
        const int sLX = LX + o.x, sLY = LY + o.y;
        if (sLX < 0 || sLY < 0 || sLX >= nL || sLY >= nL) continue;
        const T* ql = sq + ((o.y + D) * SW + (li + o.x + D)) * QS;
        const T* kb = sK + (8 * o.y - r + t.Rk) * KW + (8 * o.x - cx + t.Rk);
        T part = T(0);
#pragma unroll
        for (int sy = 0; sy < 8; ++sy) {
#pragma unroll
            for (int sx = 0; sx < 8; ++sx) part = fma(ql[sy * 8 + sx], kb[sy * KW + sx], part);
        }
        if (COMP) {  // Kahan-compensated sum of the per-leaf partial sums
            const T y = part - comp;
            const T s = acc + y;
            comp = (s - acc) - y;
            acc = s;
        } else {
            acc += part;
        }
    }
    double phi = double(acc) - double(comp);
    if (has_far) {
        const int c = r * 8 + cx;
        T ser = T(0);
        for (int k = 1; k < P1; ++k) {
            const C L = sL[li * P1 + k];
            const C w = sV[c * P1 + k];
            ser = fma(L.x, w.x, fma(-L.y, w.y, ser));
        }
        phi += sL0[li] + double(ser);
    }
    p_out[int64_t(LY * 8 + r) * t.n + LX * 8 + cx] = T(phi * kInv2Pi);
}

// ------------------------------------------------------------------------------------
// (a7) Surface pressure by the tree-code (Sec. A.2, Fig. "multipole"): each point walks
// the quadtree from the root; a box is accepted when r_box < theta d and then
// contributes its multipole (Eq. pressTruncated about its centre); leaves that are never
// accepted are summed directly.  One warp per point, lanes over candidate boxes.
// ------------------------------------------------------------------------------------
constexpr int kCandCap = 256;
constexpr int kLeafCap = 64;

template <typename T, int P1T>
__global__ void __launch_bounds__(128) k_treecode(Tree<T> t, SurfaceArgs a) {
    typedef typename cplx_of<T>::type C;
    __shared__ int cand[4][2][kCandCap];
    __shared__ int leaves[4][kLeafCap];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pt = blockIdx.x * 4 + warp;
    if (pt >= a.npts) return;
    const int P1 = P1T > 0 ? P1T : t.P1;
    const double zx = a.pts[2 * pt], zy = a.pts[2 * pt + 1];
    const double L = double(t.n) * t.h;
    double mono = 0.0;
    float mh = 0.f, ml = 0.f;  // cell-unit points of mixed plans: the monopole sum as a double-float pair
    T ser = T(0);
    int cur = 0, ncand = 1, nleaf = 0;
    bool overflow = false;
    // The root box is never accepted for a point inside the domain (no such point is
    // farther than its half-diagonal from the centre), so such points start from the
    // four boxes of level 1.
    const bool inside = zx >= t.x0 && zx <= t.x0 + L && zy >= t.y0 && zy <= t.y0 + L && t.Lleaf >= 1;
    const int l_start = inside ? 1 : 0;
    // Mixed plans, points inside the domain: offsets in cell units, an exact integer
    // difference plus the point's fraction of a cell (split once in FP64), so no FP64 per
    // box.  The log h parts of every accepted box and near cell add up to log h times the
    // root monopole (they partition the domain) and enter once at the end.
    const bool cellu = sizeof(T) == 4 && inside && t.Sf != nullptr;
    int ix = 0, iy = 0;
    float fx = 0.f, fy = 0.f;
    if (cellu) {
        const double cxd = (zx - t.x0) * t.inv_h, cyd = (zy - t.y0) * t.inv_h;
        ix = int(floor(cxd));
        iy = int(floor(cyd));
        fx = float(cxd - ix);
        fy = float(cyd - iy);
    }
    if (inside) {
        ncand = 4;
        if (lane < 4) cand[warp][0][lane] = lane;
    } else if (lane == 0) {
        cand[warp][0][0] = 0;
    }
    __syncwarp();
    const T th2 = T(a.theta * a.theta);
    for (int l = l_start; l <= t.Lleaf; ++l) {
        const int side = 1 << l;
        const double s = cellu ? 0.0 : L / side;  // box side and half-diagonal (FP64 offsets only)
        const double rb = s * 0.70710678118654752440;
        const int64_t off = level_offset(l);
        int nnext = 0;
        for (int base = 0; base < ncand; base += 32) {
            const int i = base + lane;
            bool open = false;
            int b = 0;
            if (i < ncand) {
                b = cand[warp][cur][i];
                const int bx = b % side, by = b / side;
                T dx, dy, sT, rb2;
                if (cellu) {  // cell units
                    const int sc = 8 << (t.Lleaf - l);
                    dx = T(float(ix - (bx * sc + (sc >> 1))) + fx);
                    dy = T(float(iy - (by * sc + (sc >> 1))) + fy);
                    sT = T(sc);
                    rb2 = T(0.5) * sT * sT;
                } else {
                    // offsets in FP64 (exact enough at any distance), the rest in the plan precision
                    dx = T(zx - (t.x0 + (bx + 0.5) * s));
                    dy = T(zy - (t.y0 + (by + 0.5) * s));
                    sT = T(s);
                    rb2 = T(rb * rb);
                }
                const T d2 = dx * dx + dy * dy;
                if (rb2 < th2 * d2) {
                    // Eq. pressTruncated about the box centre: S log|w| - Re sum_k M_k (s / w)^k
                    const T lg = T(0.5) * log_t<T>(d2);
                    if (cellu) {  // double-float S log|w| on the FP32 pipe (mixed plans)
                        const float2 sp = t.Sf[off + b];
                        df_fma(mh, ml, sp.x, sp.y, float(lg), 0.f);
                    } else {
                        mono += t.S[off + b] * double(lg);
                    }
                    const T sd = sT / d2;
                    const C u = cmake<T>(sd * dx, -sd * dy);
                    const C* M = t.mp + (off + b) * P1;
                    C acc = M[P1 - 1];
#pragma unroll
                    for (int k = P1 - 2; k >= 1; --k) {
                        const C m = M[k];
                        const T nr = fma(acc.x, u.x, fma(-acc.y, u.y, m.x));
                        const T ni = fma(acc.x, u.y, fma(acc.y, u.x, m.y));
                        acc.x = nr;
                        acc.y = ni;
                    }
                    ser -= acc.x * u.x - acc.y * u.y;
                } else {
                    open = true;
                }
            }
    const unsigned mask = __ballot_sync(0xffffffffu, open);
            const int pos = __popc(mask & ((1u << lane) - 1u));
            if (l < t.Lleaf) {
                if (open) {
                    const int at = nnext + 4 * pos;
                    if (at + 4 <= kCandCap) {
                        const int bx = b % side, by = b / side;
                        for (int q = 0; q < 4; ++q)
                            cand[warp][cur ^ 1][at + q] = (2 * by + (q >> 1)) * (2 * side) + 2 * bx + (q & 1);
                    } else {
                        overflow = true;
                    }
                }
                nnext += 4 * __popc(mask);
            } else {
                if (open) {
                    const int at = nleaf + pos;
                    if (at < kLeafCap) leaves[warp][at] = b;
                    else overflow = true;
                }
                nleaf += __popc(mask);
            }
        }
        __syncwarp();
        cur ^= 1;
        ncand = min(nnext, kCandCap);
    }
    nleaf = min(nleaf, kLeafCap);
    const T rh2 = cellu ? T((a.rho_h / t.h) * (a.rho_h / t.h)) : T(a.rho_h * a.rho_h);
    const T hT = cellu ? T(1) : T(t.h);
    double nearsum = 0.0;
    T nearf = T(0);  // cell units: the lane's near-field partial in T, converted once
    for (int e = 0; e < nleaf; ++e) {
        const int b = leaves[warp][e];
        const int LX = b % t.nL, LY = b / t.nL;
        // point relative to the leaf corner (FP64, or exact cell units), cells relative to that in T
        const T ox = cellu ? T(float(ix - 8 * LX) + fx) : T(zx - (t.x0 + 8.0 * LX * t.h));
        const T oy = cellu ? T(float(iy - 8 * LY) + fy) : T(zy - (t.y0 + 8.0 * LY * t.h));
        T part = T(0);
        for (int c = lane; c < 64; c += 32) {
            const T dx = ox - (T(c & 7) + T(0.5)) * hT;
            const T dy = oy - (T(c >> 3) + T(0.5)) * hT;
            const T r2 = dx * dx + dy * dy;
            part += t.q[int64_t(b) * 64 + c] * (T(0.5) * log_t<T>(r2 > rh2 ? r2 : rh2));
        }
        if (cellu)
            nearf += part;
        else
            nearsum += double(part);
    }
    double tot;
    if (cellu) {  // warp-uniform: the lanes' sums as double-float pairs, reduced on the FP32 pipe
        df_add(mh, ml, float(ser), 0.f);
        df_add(mh, ml, float(nearf), 0.f);
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, mh, o), ol = __shfl_xor_sync(0xffffffffu, ml, o);
            df_add(mh, ml, oh, ol);
        }
        tot = df_to(mh, ml) + t.lnh * t.S[0];  // log h times the root monopole, once per point
    } else {
        tot = mono + double(ser) + nearsum;
        for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    const bool ovf = __any_sync(0xffffffffu, overflow);
    if (lane == 0) {
        a.Psurf[pt] = tot * kInv2Pi;
        if (ovf) atomicExch(a.err, 1);
    }
}

// ------------------------------------------------------------------------------------
// (a8) Tractions and their integrals (Sec. 2.3).  One thread per point; a deterministic
// block tree reduction of the four force sums, then one final CTA.
// ------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void cell_grad(const T* u, const T* v, int n, double inv2h, int i, int j,
                                          double g[4]) {
    const int64_t c = int64_t(j) * n + i;
    g[0] = (double(u[c + 1]) - double(u[c - 1])) * inv2h;
    g[1] = (double(u[c + n]) - double(u[c - n])) * inv2h;
    g[2] = (double(v[c + 1]) - double(v[c - 1])) * inv2h;
    g[3] = (double(v[c + n]) - double(v[c - n])) * inv2h;
}

__device__ __forceinline__ int clampi(double x, int lo, int hi) {
    if (!(x == x)) return lo;  // NaN
    if (x < double(lo)) return lo;
    if (x > double(hi)) return hi;
    return int(x);
}

template <typename T>
__global__ void __launch_bounds__(kSurfaceBlock)
k_traction(Tree<T> t, const T* __restrict__ u, const T* __restrict__ v, SurfaceArgs a) {
    __shared__ double red[4][kSurfaceBlock];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double fx = 0.0, fy = 0.0, gx = 0.0, gy = 0.0;
    if (i < a.npts) {
        const int n = t.n;
        const double px = a.pts[2 * i], py = a.pts[2 * i + 1];
        const double nx = a.nrm[2 * i], ny = a.nrm[2 * i + 1];
        double dS;
        if (a.dS) {
            dS = a.dS[i];
        } else {
            const int ip = (i + 1 == a.npts) ? 0 : i + 1;
            const int im = (i == 0) ? a.npts - 1 : i - 1;
            const double l1 = hypot(a.pts[2 * ip] - px, a.pts[2 * ip + 1] - py);
            const double l0 = hypot(px - a.pts[2 * im], py - a.pts[2 * im + 1]);
            dS = 0.5 * (l0 + l1);
        }
        const double yx = px + a.lift * nx, yy = py + a.lift * ny;
        const double inv2h = 0.5 / t.h;
        double g[4];
        if (a.interp == 0) {
            const int ci = clampi(floor((yx - t.x0) / t.h), 1, n - 2);
            const int cj = clampi(floor((yy - t.y0) / t.h), 1, n - 2);
            cell_grad(u, v, n, inv2h, ci, cj, g);
        } else {
            const double fxx = (yx - t.x0) / t.h - 0.5, fyy = (yy - t.y0) / t.h - 0.5;
            const int i0 = clampi(floor(fxx), 1, n - 3), j0 = clampi(floor(fyy), 1, n - 3);
            const double ax = fmin(fmax(fxx - i0, 0.0), 1.0), ay = fmin(fmax(fyy - j0, 0.0), 1.0);
            const double wts[4] = {(1 - ax) * (1 - ay), ax * (1 - ay), (1 - ax) * ay, ax * ay};
            for (int c = 0; c < 4; ++c) g[c] = 0.0;
            for (int q = 0; q < 4; ++q) {
                double gq[4];
                cell_grad(u, v, n, inv2h, i0 + (q & 1), j0 + (q >> 1), gq);
                for (int c = 0; c < 4; ++c) g[c] += wts[q] * gq[c];
            }
        }
        const double dxy = 0.5 * (g[1] + g[2]);
        const double tnx = a.mu2 * (g[0] * nx + dxy * ny);
        const double tny = a.mu2 * (dxy * nx + g[3] * ny);
        const double P = a.Psurf[i];
        const double tpx = -P * nx, tpy = -P * ny;
        if (a.per_point) {
            double* o = a.per_point + int64_t(5) * i;
            o[0] = P;
            o[1] = tpx;
            o[2] = tpy;
            o[3] = tnx;
            o[4] = tny;
        }
        fx = tpx * dS;
        fy = tpy * dS;
        gx = tnx * dS;
        gy = tny * dS;
    }
    red[0][threadIdx.x] = fx;
    red[1][threadIdx.x] = fy;
    red[2][threadIdx.x] = gx;
    red[3][threadIdx.x] = gy;
    __syncthreads();
    for (int s = kSurfaceBlock / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int c = 0; c < 4; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 4) a.partial[int64_t(blockIdx.x) * 4 + threadIdx.x] = red[threadIdx.x][0];
}

template <typename T>
__global__ void __launch_bounds__(256) k_forces_final(int nblocks, SurfaceArgs a) {
    // Fixed-order sums over the per-block partials: the result does not depend on timing.
    __shared__ double red[4][256];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int c = 0; c < 4; ++c) acc[c] += a.partial[int64_t(b) * 4 + c];
    for (int c = 0; c < 4; ++c) red[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int c = 0; c < 4; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double fpx = red[0][0], fpy = red[1][0], fnx = red[2][0], fny = red[3][0];
        const double Fx = fpx + fnx, Fy = fpy + fny;
        a.forces[0] = fpx;
        a.forces[1] = fpy;
        a.forces[2] = fnx;
        a.forces[3] = fny;
        a.forces[4] = Fx * a.uhat_x + Fy * a.uhat_y;
        a.forces[5] = -Fx * a.uhat_y + Fy * a.uhat_x;
    }
}

template <typename T>
__global__ void k_export(Tree<T> t, int kind, int level, double* dst) {
    const int64_t nb = int64_t(1) << (2 * level);
    const int64_t off = level_offset(level);
    const int64_t tot = nb * t.P1;
    for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < tot;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int64_t b = idx / t.P1;
        const int k = int(idx % t.P1);
        double re, im;
        if (kind == 0) {
            const typename cplx_of<T>::type c = t.mp[(off + b) * t.P1 + k];
            re = (k == 0) ? t.S[off + b] : double(c.x);
            im = (k == 0) ? 0.0 : double(c.y);
        } else {
            const typename cplx_of<T>::type c = t.loc[(off + b) * t.P1 + k];
            re = (k == 0) ? t.L0[off + b] : double(c.x);
            im = (k == 0) ? 0.0 : double(c.y);
        }
        dst[2 * idx] = re;
        dst[2 * idx + 1] = im;
    }
}

// ------------------------------------------------------------------------------------
// Launchers
// ------------------------------------------------------------------------------------
template <typename T>
cudaError_t launch_rhs_p2m(const Tree<T>& t, const T* u, const T* v, const T* chi, const T* usx,
                           const T* usy, double rho, double lam, T* f_out, cudaStream_t st, int* launches) {
    typedef typename cplx_of<T>::type C;
    if constexpr (sizeof(T) == 4) {
        // register-blocked source + leaf multipoles: float4 accesses need 16-byte aligned fields
        auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
        const bool aligned = al(u) && al(v) && al(chi) && al(usx) && al(usy) && al(f_out);
        if (aligned) {
            const int64_t warps = int64_t((t.n + 127) / 128) * ((t.nL + kRhsLeafRows - 1) / kRhsLeafRows);
            const unsigned blocks = unsigned((warps + kRhsWarps - 1) / kRhsWarps);
            const Tree<float>& tf = reinterpret_cast<const Tree<float>&>(t);
            const float* fu = reinterpret_cast<const float*>(u);
            const float* fv = reinterpret_cast<const float*>(v);
            const float* fc = reinterpret_cast<const float*>(chi);
            const float* fsx = reinterpret_cast<const float*>(usx);
            const float* fsy = reinterpret_cast<const float*>(usy);
            float* ff = reinterpret_cast<float*>(f_out);
            switch (t.P1) {
#define PP_CASE(P)                                                                                         \
    case P:                                                                                                \
        k_rhs_p2m_fast<P><<<blocks, 32 * kRhsWarps, rhs_smem_bytes(P), st>>>(tf, fu, fv, fc, fsx, fsy, float(rho), \
                                                                            float(lam), ff);                    \
        *launches = 1;                                                                                     \
        return cudaGetLastError();
                PP_FAST_ORDERS(PP_CASE)
#undef PP_CASE
                default: break;
            }
        }
    }
    *launches = 2;
    const size_t smem = sizeof(T) * (4 * kRW * kRW);
    const int tiles = (t.n + kRT - 1) / kRT;
    dim3 grid(tiles, tiles);
    k_rhs_p2m<T><<<grid, 256, smem, st>>>(t, u, v, chi, usx, usy, T(rho), T(lam), f_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t threads = int64_t(t.nL) * t.nL * 8;
    const unsigned blocks = unsigned((threads + 255) / 256);
    switch (t.P1) {
#define PP_CASE(P) \
    case P: k_p2m_reg<T, P><<<blocks, 256, 0, st>>>(t); break;
        PP_FAST_ORDERS(PP_CASE)
#undef PP_CASE
        default: k_p2m<T><<<blocks, 256, 0, st>>>(t); break;
    }
    return cudaGetLastError();
}


// The subtree root level of k_up_tree (subtrees of up to 4 levels) and whether its last CTA
// also does the levels above (at most 64 parents there).
template <typename T>
int up_tree_root(const Tree<T>& t) {
    return t.Lleaf > 4 ? t.Lleaf - 4 : 0;
}

template <typename T, int P1>
cudaError_t upward_fast(const Tree<T>& t, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        if (t.up_counter && t.Lleaf >= 1 && t.Lleaf <= 8) {  // one launch: subtrees and, by the last CTA, the top
            const int lr = up_tree_root(t);
            const Tree<float>& tf = reinterpret_cast<const Tree<float>&>(t);
            if (t.mmax)  // the tensor-core translations scale by the largest coefficient
                k_up_tree<P1, true><<<unsigned(int64_t(1) << (2 * lr)), 256, 0, st>>>(tf, lr, t.up_counter);
            else
                k_up_tree<P1, false><<<unsigned(int64_t(1) << (2 * lr)), 256, 0, st>>>(tf, lr, t.up_counter);
            return cudaGetLastError();
        }
    }
    // fine levels: 4 threads per parent; levels <= 3 in one CTA
    int l = t.Lleaf - 1;
    for (; l > 3; --l) {
        const int64_t threads = (int64_t(1) << (2 * l)) * 4;
        k_m2m_reg<T, P1><<<unsigned((threads + 127) / 128), 128, 0, st>>>(t, l, 4);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (l >= 0) {
        k_m2m_top<T, P1><<<1, 128, 0, st>>>(t, l);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

// Threads per target box (power of two <= 32): about four waves of resident threads, so
// that the last partial wave costs little.
inline int m2l_group(int64_t nb, int64_t resident) {
    int S = 1;
    while (S < 32 && nb * S < resident) S <<= 1;
    return S;
}

template <typename T, int P1>
cudaError_t downward_fast(const Tree<T>& t, int l0, int l1, T* p_out, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        const int lt = chain_top<T>(t, l0, l1, p_out != nullptr);
        if (lt > 0) {  // levels 2..lt in one launch
            LevelLogs lg;
            for (int l = 0; l < 16; ++l) lg.lnS[l] = std::log(double(t.n) * t.h / double(int64_t(1) << l));
            const int64_t threads = (int64_t(1) << (2 * lt)) * 32;
            k_m2l_chain<P1><<<unsigned((threads + 127) / 128), 128, 0, st>>>(
                reinterpret_cast<const Tree<float>&>(t), lt, lg);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            l0 = lt + 1;
        }
    }
    for (int l = l0; l <= l1; ++l) {
        const int64_t nb = int64_t(1) << (2 * l);
        const int S = m2l_group(nb, t.resident_threads);
        const int64_t threads = nb * S;
        const unsigned blocks = unsigned((threads + 127) / 128);
        const double lnS = std::log(double(t.n) * t.h / double(int64_t(1) << l));
        if (p_out && l == t.Lleaf)
            k_m2l_reg<T, P1, true><<<blocks, 128, 0, st>>>(t, l, S, lnS, p_out);
        else
            k_m2l_reg<T, P1, false><<<blocks, 128, 0, st>>>(t, l, S, lnS, nullptr);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// FP64 keeps the register kernels only where they fit without spilling.
template <typename T>
inline bool fast_order_ok(int P1) {
    return sizeof(T) == 4 || P1 <= 21;
}

template <typename T>
int upward_launches(const Tree<T>& t) {
    bool fast = false;
#define PP_CASE(P) fast = fast || t.P1 == P;
    PP_FAST_ORDERS(PP_CASE)
#undef PP_CASE
    if (!fast || !fast_order_ok<T>(t.P1)) return t.Lleaf;
    if (sizeof(T) == 4 && t.up_counter && t.Lleaf >= 1 && t.Lleaf <= 8) return 1;
    // levels Lleaf-1 .. 4 one launch each, levels <= 3 in one
    return (t.Lleaf - 1 > 3 ? t.Lleaf - 4 : 0) + (t.Lleaf >= 1 ? 1 : 0);
}

template <typename T>
cudaError_t launch_upward(const Tree<T>& t, cudaStream_t st) {
    switch (fast_order_ok<T>(t.P1) ? t.P1 : 0) {
#define PP_CASE(P) \
    case P: return upward_fast<T, P>(t, st);
        PP_FAST_ORDERS(PP_CASE)
#undef PP_CASE
        default: break;
    }
    for (int l = t.Lleaf - 1; l >= 0; --l) {
        const int64_t nb = int64_t(1) << (2 * l);
        k_m2m<T><<<unsigned((nb + 3) / 4), 128, 0, st>>>(t, l);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Downward levels l0..l1; with p_out the leaf level also adds the local expansion at
// every cell to the near field already stored in p_out (register kernels only).
template <typename T>
cudaError_t launch_downward_levels(const Tree<T>& t, int l0, int l1, T* p_out, cudaStream_t st) {
    switch (fast_order_ok<T>(t.P1) ? t.P1 : 0) {
#define PP_CASE(P) \
    case P: return downward_fast<T, P>(t, l0, l1, p_out, st);
        PP_FAST_ORDERS(PP_CASE)
#undef PP_CASE
        default: break;
    }
    if (p_out) return cudaErrorInvalidValue;
    for (int l = l0; l <= l1; ++l) {
        const int64_t nb = int64_t(1) << (2 * l);
        k_m2l<T><<<unsigned((nb + 3) / 4), 128, 0, st>>>(t, l);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T>
bool leaf_l2p_ok(const Tree<T>& t, const void* p_out) {
    bool fast = false;
#define PP_CASE(P) fast = fast || t.P1 == P;
    PP_FAST_ORDERS(PP_CASE)
#undef PP_CASE
    return sizeof(T) == 4 && fast && t.Lleaf >= 3 && t.Dmax <= kMaxD &&
           (reinterpret_cast<uintptr_t>(p_out) & 15) == 0;
}

template <typename T>
cudaError_t launch_leaf_l2p(const Tree<T>& t, T* p_out, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        const dim3 grid(unsigned(t.nL / 8), unsigned(t.nL / 8));
        const Tree<float>& tf = reinterpret_cast<const Tree<float>&>(t);
        float* pf = reinterpret_cast<float*>(p_out);
        switch (t.P1) {
#define PP_CASE(P)                                         \
    case P:                                                \
        k_l2p_leaf<P><<<grid, 256, 0, st>>>(tf, pf);       \
        return cudaGetLastError();
            PP_FAST_ORDERS(PP_CASE)
#undef PP_CASE
            default: break;
        }
    }
    return cudaErrorInvalidValue;
}

// Two-launch downward pass of the split solve (k_m2l_far, then k_down_tree after the near
// field): mixed precision, register-kernel orders, leaf level 5..15, an aligned output.
template <typename T>
bool down_tree_ok(const Tree<T>& t, const void* p_out) {
    return leaf_l2p_ok<T>(t, p_out) && t.Lleaf >= 5 && t.Lleaf <= 15 && t.Lleaf - 5 <= kDownAnc &&
           t.locA != nullptr && t.L0A != nullptr;
}

template <typename T>
cudaError_t launch_m2l_far(const Tree<T>& t, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        const Tree<float>& tf = reinterpret_cast<const Tree<float>&>(t);
        int64_t boxes = 0;
        for (int l = 2; l <= t.Lleaf; ++l) boxes += int64_t(1) << (2 * l);
        // S threads per box so that the grid fills at least three quarters of the resident
        // threads of k_m2l_far (resident_threads counts 384 per SM for mixed plans)
        const double lnRoot = std::log(double(t.n) * t.h);
        switch (t.P1) {
#define PP_CASE(P)                                                                      \
    case P: {                                                                           \
        const int64_t slots = t.resident_threads / 384 * 128 * FarOcc<P>::value;        \
        int S = 1;                                                                      \
        while (S < 32 && 4 * boxes * S < 3 * slots) S <<= 1;                            \
        const unsigned blocks = unsigned((boxes * S + 127) / 128);                      \
        k_m2l_far<P><<<blocks, 128, 0, st>>>(tf, t.Lleaf - 3, S, lnRoot);               \
        return cudaGetLastError();                                                      \
    }
            PP_FAST_ORDERS(PP_CASE)
#undef PP_CASE
            default: break;
        }
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_down_tree(const Tree<T>& t, T* p_out, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        const dim3 grid(unsigned(t.nL / 8), unsigned(t.nL / 8));
        const Tree<float>& tf = reinterpret_cast<const Tree<float>&>(t);
        float* pf = reinterpret_cast<float*>(p_out);
        switch (t.P1) {
#define PP_CASE(P)                                                 \
    case P:                                                        \
        k_down_tree<P><<<grid, kDownThreads, t.Dmax >= 2 ? kDownRoom : 0, st>>>(tf, t.Lleaf - 3, pf); \
        return cudaGetLastError();
            PP_FAST_ORDERS(PP_CASE)
#undef PP_CASE
            default: break;
        }
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_downward(const Tree<T>& t, cudaStream_t st) {
    switch (fast_order_ok<T>(t.P1) ? t.P1 : 0) {
#define PP_CASE(P) \
    case P: return downward_fast<T, P>(t, 2, t.Lleaf, (T*)nullptr, st);
        PP_FAST_ORDERS(PP_CASE)
#undef PP_CASE
        default: break;
    }
    for (int l = 2; l <= t.Lleaf; ++l) {
        const int64_t nb = int64_t(1) << (2 * l);
        k_m2l<T><<<unsigned((nb + 3) / 4), 128, 0, st>>>(t, l);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T>
size_t leaf_smem_bytes(const Tree<T>& t) {
    typedef typename cplx_of<T>::type C;
    const int D = t.Dmax;
    const int KW = 2 * t.Rk + 1;
    return sizeof(C) * (64 * t.P1 + 4 * t.P1) + sizeof(double) * 4 + sizeof(T) * KW * KW +
           sizeof(T) * (4 + 2 * D) * (2 * D + 1) * 65;
}

template <int D, bool FAR>
cudaError_t leaf_fast(const Tree<float>& t, float* p_out, cudaStream_t st) {
    const size_t smem = LeafFastGeom<D>::smem_bytes;
    dim3 grid(t.nL / 4, t.nL / 4);
    k_leaf_fast<D, FAR><<<grid, 128, smem, st>>>(t, t.near_mask, p_out);
    return cudaGetLastError();
}

inline bool leaf_fast_ok(const Tree<float>& t) {
    return t.nL >= 4 && (t.nL & 3) == 0 && t.Dmax >= 1 && t.Dmax <= 3;
}

template <bool FAR>
cudaError_t leaf_fast_run(const Tree<float>& t, float* p_out, cudaStream_t st) {
    switch (t.Dmax) {
        case 1: return leaf_fast<1, FAR>(t, p_out, st);
        case 2: return leaf_fast<2, FAR>(t, p_out, st);
        default: return leaf_fast<3, FAR>(t, p_out, st);
    }
}

inline cudaError_t leaf_fast_dispatch(const Tree<float>& t, float* p_out, cudaStream_t st, bool* done) {
    *done = leaf_fast_ok(t);
    return *done ? leaf_fast_run<true>(t, p_out, st) : cudaSuccess;
}

inline cudaError_t leaf_fast_dispatch(const Tree<double>&, double*, cudaStream_t, bool* done) {
    *done = false;  // the FP64 path keeps one thread per target cell
    return cudaSuccess;
}

// The split solve: near field alone on a second stream, far field added by the
// leaf-level multipole-to-local kernel (mixed precision, register kernels).
template <typename T>
bool split_solve_ok(const Tree<T>& t) {
    if (sizeof(T) != 4) return false;
    bool order = false;
#define PP_CASE(P) order = order || t.P1 == P;
    PP_FAST_ORDERS(PP_CASE)
#undef PP_CASE
    return order && t.Lleaf >= 2 && leaf_fast_ok(reinterpret_cast<const Tree<float>&>(t));
}

template <int D>
cudaError_t near16(const Tree<float>& t, float* p_out, cudaStream_t st) {
    dim3 grid(t.nL / 4, t.nL / 8);
    k_near16<D><<<grid, 128, Near16Geom<D>::smem_bytes, st>>>(t, t.near_mask, p_out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_near_only(const Tree<T>& t, T* p_out, cudaStream_t st) {
    if (sizeof(T) != 4) return cudaErrorInvalidValue;
    const Tree<float>& tf = reinterpret_cast<const Tree<float>&>(t);
    float* pf = reinterpret_cast<float*>(p_out);
    if (t.near_tile == 16 && t.nL >= 8 && (t.nL & 7) == 0) {
        switch (t.Dmax) {
            case 1: return near16<1>(tf, pf, st);
            case 2: return near16<2>(tf, pf, st);
            default: return near16<3>(tf, pf, st);
        }
    }
    return leaf_fast_run<false>(tf, pf, st);
}

template <typename T>
cudaError_t launch_leaf_eval(const Tree<T>& t, T* p_out, cudaStream_t st) {
    bool done = false;
    cudaError_t ef = leaf_fast_dispatch(t, p_out, st, &done);
    if (done || ef != cudaSuccess) return ef;
    const bool comp = sizeof(T) == 4;
    const size_t smem = leaf_smem_bytes(t);
    dim3 grid((t.nL + 3) / 4, t.nL);
    const int has_far = t.Lleaf >= 2 ? 1 : 0;
    if (comp)
        k_leaf<T, true><<<grid, 256, smem, st>>>(t, has_far, p_out);
    else
        k_leaf<T, false><<<grid, 256, smem, st>>>(t, has_far, p_out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_surface(const Tree<T>& t, const T* u, const T* v, const SurfaceArgs& a,
                           cudaStream_t st) {
    const unsigned nb4 = unsigned((a.npts + 3) / 4);
    switch (t.P1) {
#define PP_CASE(P) \
    case P: k_treecode<T, P><<<nb4, 128, 0, st>>>(t, a); break;
        PP_FAST_ORDERS(PP_CASE)
#undef PP_CASE
        default: k_treecode<T, 0><<<nb4, 128, 0, st>>>(t, a); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int nb = (a.npts + kSurfaceBlock - 1) / kSurfaceBlock;
    k_traction<T><<<nb, kSurfaceBlock, 0, st>>>(t, u, v, a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_forces_final<T><<<1, 256, 0, st>>>(nb, a);
    return cudaGetLastError();
}

// Opt every kernel with dynamic shared memory into the same generous limit, once per
// device, at plan creation (never inside a launch sequence, so steps can be captured).
template <typename T>
cudaError_t prepare_kernels() {
    const int lim = kDynSmemLimit;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_rhs_p2m<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_leaf<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_leaf<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) != cudaSuccess)
        return e;
    if (sizeof(T) == 4) {
        const void* fns[] = {(const void*)k_leaf_fast<1, true>, (const void*)k_leaf_fast<2, true>,
                             (const void*)k_leaf_fast<3, true>, (const void*)k_leaf_fast<1, false>,
                             (const void*)k_leaf_fast<2, false>, (const void*)k_leaf_fast<3, false>,
                             (const void*)k_near16<1>, (const void*)k_near16<2>, (const void*)k_near16<3>,
                             (const void*)k_rhs_p2m_fast<13>, (const void*)k_rhs_p2m_fast<17>,
                             (const void*)k_rhs_p2m_fast<21>, (const void*)k_rhs_p2m_fast<25>};
        for (const void* f : fns)
            if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) != cudaSuccess)
                return e;
    }
    return cudaSuccess;
}

// Dynamic shared memory a plan's launches need (checked against kDynSmemLimit at creation).
template <typename T>
size_t plan_smem_bytes(const Tree<T>& t) {
    const size_t rhs = sizeof(T) * (4 * kRW * kRW);
    const size_t leaf = leaf_smem_bytes(t);
    return rhs > leaf ? rhs : leaf;
}

template <typename T>
cudaError_t launch_export_expansion(const Tree<T>& t, int kind, int level, double* dst,
                                    cudaStream_t st) {
    const int64_t tot = (int64_t(1) << (2 * level)) * t.P1;
    const int blocks = int((tot + 255) / 256 < 4096 ? (tot + 255) / 256 : 4096);
    k_export<T><<<blocks, 256, 0, st>>>(t, kind, level, dst);
    return cudaGetLastError();
}

}  // namespace pp
