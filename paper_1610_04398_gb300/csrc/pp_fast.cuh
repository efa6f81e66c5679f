// Register-resident translation kernels and the register-blocked near field.
//
// Every translation of the log series factors as diag * R * diag with a REAL matrix R
// that depends neither on the offset nor on the level (scaled coefficients, Sec. A.2):
//   multipole-to-local, offset tau (box units), x_k = tau^-k M_k:
//       L_l += tau^-l sum_k R[l][k] x_k,  R[l][0] = -1/l, R[l][k] = (-1)^(k+1) C(l+k-1, k-1)
//       (plus S log|tau| on L_0, accumulated in FP64);
//   local-to-local to child quadrant q, w_k = zeta^k b_k:  c_l = (2 zeta)^-l sum_{k>=l} C(k, l) w_k;
//   multipole-to-multipole from child quadrant q (Eq. expandedBeta with the S sign read as +),
//       w_j = (2 zeta)^-j M_j:  beta_k = zeta^k [S / k + sum_{j<=k} C(k-1, j-1) w_j].
// R lives in constant memory (compile-time tables), so the inner products are FFMAs with
// constant-bank operands on register-resident vectors; the complex diagonals come from
// small per-offset / per-quadrant tables.
#pragma once

#include "pp_common.h"

#ifndef PP_REAL
#define PP_REAL float
#endif

namespace pp {

constexpr int kFastMaxP1 = 25;

constexpr double cbinom(int n, int k) {
    if (k < 0 || k > n) return 0.0;
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * double(n - k + i) / double(i);
    return r;
}

template <typename T>
struct RealOps {
    T m2l[kFastMaxP1][kFastMaxP1];  // [l][k]
    T l2l[kFastMaxP1][kFastMaxP1];  // [l][k] = C(k, l) for k >= l
    T m2m[kFastMaxP1][kFastMaxP1];  // [k][j] = C(k-1, j-1) for 1 <= j <= k; [k][0] = 1/k
    constexpr RealOps() : m2l(), l2l(), m2m() {
        for (int l = 0; l < kFastMaxP1; ++l)
            for (int k = 0; k < kFastMaxP1; ++k) {
                double r = 0.0;
                if (k == 0) r = (l == 0) ? 0.0 : -1.0 / double(l);
                else r = ((k + 1) % 2 == 0 ? 1.0 : -1.0) * cbinom(l + k - 1, k - 1);
                m2l[l][k] = T(r);
                l2l[l][k] = T(k >= l ? cbinom(k, l) : 0.0);
                double m = 0.0;
                if (l >= 1 && k == 0) m = 1.0 / double(l);
                else if (l >= 1 && k >= 1 && k <= l) m = cbinom(l - 1, k - 1);
                m2m[l][k] = T(m);
            }
    }
};

__constant__ RealOps<PP_REAL> c_ops = RealOps<PP_REAL>();

// ------------------------------------------------------------------------------------
// Multipole-to-local translations into one target box (bx, by) at level l: the entries
// e0, e0 + stride, ... of its interaction list (same-level boxes and parent-level boxes
// that stand for four separated children), added to the FP32 coefficients (Lr, Li) and to
// the FP64 constant-term parts a0 (S log|tau|) and sumS (S, times the log of the box side
// by the caller).
// ------------------------------------------------------------------------------------
template <typename T, int P1>
__device__ __forceinline__ void m2l_list(const Tree<T>& t, int l, int bx, int by, int e0, int stride,
                                         T (&Lr)[P1], T (&Li)[P1], double& a0, double& sumS) {
    typedef typename cplx_of<T>::type C;
    const int side = 1 << l;
    const int64_t off = level_offset(l);
    const int par = (bx & 1) + 2 * (by & 1);
    const int cnt = t.il_count[par];
    const M2LEntry* lst = t.il + int64_t(par) * t.il_stride;
    for (int e = e0; e < cnt; e += stride) {
        const M2LEntry en = lst[e];
        int64_t src;
        if (en.pad == 0) {  // same-level source box
            const int sx = bx + en.dx, sy = by + en.dy;
            if (sx < 0 || sy < 0 || sx >= side || sy >= side) continue;
            src = off + int64_t(sy) * side + sx;
        } else {  // parent-level source box standing for four separated children
            const int hs = side >> 1;
            const int sx = (bx >> 1) + en.dx, sy = (by >> 1) + en.dy;
            if (sx < 0 || sy < 0 || sx >= hs || sy >= hs) continue;
            src = level_offset(l - 1) + int64_t(sy) * hs + sx;
        }
        const C* M = t.mp + src * P1;
        const C* tp = t.Tpow + int64_t(en.op) * P1;
        const C* tl = t.TpowL + int64_t(en.op) * P1;
        const double Sd = t.S[src];
        const T St = T(Sd);
        // y = R x, accumulated column by column: 2 P1 - 1 independent FMA chains
        T yr[P1], yi[P1];
        yr[0] = T(0);
        yi[0] = T(0);
#pragma unroll
        for (int ll = 1; ll < P1; ++ll) {
            yr[ll] = c_ops.m2l[ll][0] * St;
            yi[ll] = T(0);
        }
#pragma unroll
        for (int k = 1; k < P1; ++k) {
            const C m = M[k];
            const C w = tp[k];
            const T xr = m.x * w.x - m.y * w.y;
            const T xi = m.x * w.y + m.y * w.x;
            yr[0] = fma(c_ops.m2l[0][k], xr, yr[0]);
#pragma unroll
            for (int ll = 1; ll < P1; ++ll) {
                yr[ll] = fma(c_ops.m2l[ll][k], xr, yr[ll]);
                yi[ll] = fma(c_ops.m2l[ll][k], xi, yi[ll]);
            }
        }
        Lr[0] += yr[0];
#pragma unroll
        for (int ll = 1; ll < P1; ++ll) {
            const C w = tl[ll];
            Lr[ll] = fma(yr[ll], w.x, fma(-yi[ll], w.y, Lr[ll]));
            Li[ll] = fma(yr[ll], w.y, fma(yi[ll], w.x, Li[ll]));
        }
        a0 = fma(Sd, t.lnTau[en.op], a0);
        sumS += Sd;
    }
}

// The same translations with the constant-term parts accumulated in double-float on the
// FP32 pipe: (ah, al) = sum S log|tau|, (sh, sl) = sum S, from the pairs Sf and lnTauF.
template <int P1>
__device__ __forceinline__ void m2l_list_df(const Tree<float>& t, int l, int bx, int by, int e0, int stride,
                                            float (&Lr)[P1], float (&Li)[P1], float& ah, float& al, float& sh,
                                            float& sl) {
    typedef float2 C;
    typedef float T;
    const int side = 1 << l;
    const int64_t off = level_offset(l);
    const int par = (bx & 1) + 2 * (by & 1);
    const int cnt = t.il_count[par];
    const M2LEntry* lst = t.il + int64_t(par) * t.il_stride;
    for (int e = e0; e < cnt; e += stride) {
        const M2LEntry en = lst[e];
        int64_t src;
        if (en.pad == 0) {  // same-level source box
            const int sx = bx + en.dx, sy = by + en.dy;
            if (sx < 0 || sy < 0 || sx >= side || sy >= side) continue;
            src = off + int64_t(sy) * side + sx;
        } else {  // parent-level source box standing for four separated children
            const int hs = side >> 1;
            const int sx = (bx >> 1) + en.dx, sy = (by >> 1) + en.dy;
            if (sx < 0 || sy < 0 || sx >= hs || sy >= hs) continue;
            src = level_offset(l - 1) + int64_t(sy) * hs + sx;
        }
        const C* M = t.mp + src * P1;
        const C* tp = t.Tpow + int64_t(en.op) * P1;
        const C* tl = t.TpowL + int64_t(en.op) * P1;
        const float2 Sd = t.Sf[src];
        const T St = Sd.x;
        // y = R x, accumulated column by column: 2 P1 - 1 independent FMA chains
        T yr[P1], yi[P1];
        yr[0] = T(0);
        yi[0] = T(0);
#pragma unroll
        for (int ll = 1; ll < P1; ++ll) {
            yr[ll] = c_ops.m2l[ll][0] * St;
            yi[ll] = T(0);
        }
#pragma unroll
        for (int k = 1; k < P1; ++k) {
            const C m = M[k];
            const C w = tp[k];
            const T xr = m.x * w.x - m.y * w.y;
            const T xi = m.x * w.y + m.y * w.x;
            yr[0] = fma(c_ops.m2l[0][k], xr, yr[0]);
#pragma unroll
            for (int ll = 1; ll < P1; ++ll) {
                yr[ll] = fma(c_ops.m2l[ll][k], xr, yr[ll]);
                yi[ll] = fma(c_ops.m2l[ll][k], xi, yi[ll]);
            }
        }
        Lr[0] += yr[0];
#pragma unroll
        for (int ll = 1; ll < P1; ++ll) {
            const C w = tl[ll];
            Lr[ll] = fma(yr[ll], w.x, fma(-yi[ll], w.y, Lr[ll]));
            Li[ll] = fma(yr[ll], w.y, fma(yi[ll], w.x, Li[ll]));
        }
        const float2 lt = t.lnTauF[en.op];
        df_fma(ah, al, Sd.x, Sd.y, lt.x, lt.y);
        df_add(sh, sl, Sd.x, Sd.y);
    }
}

// ------------------------------------------------------------------------------------
// Downward pass at level l (>= 2): S threads per target box split its interaction list
// and combine with shuffles; thread 0 of the group adds the parent's local (L2L).
// ------------------------------------------------------------------------------------
template <typename T, int P1>
struct M2LOcc {  // resident 128-thread blocks per SM the register budget aims for
    static constexpr int value = sizeof(T) == 4 ? (P1 <= 17 ? 4 : 3) : 2;
};

template <typename T, int P1, bool L2P>
__global__ void __launch_bounds__(128, M2LOcc<T, P1>::value) k_m2l_reg(Tree<T> t, int l, int S, double lnS, T* p_out) {
    typedef typename cplx_of<T>::type C;
    const int side = 1 << l;
    const int64_t nb = int64_t(side) * side;
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t b = g / S;
    const int sub = int(g % S);
    const bool act = b < nb;
    const int64_t off = level_offset(l);
    T Lr[P1], Li[P1];
#pragma unroll
    for (int i = 0; i < P1; ++i) {
        Lr[i] = T(0);
        Li[i] = T(0);
    }
    double a0 = 0.0, sumS = 0.0;
    if (act) {
        const int bx = int(b % side), by = int(b / side);
        const int par = (bx & 1) + 2 * (by & 1);
        if (l >= 3 && sub == 0) {
            const int64_t pb = level_offset(l - 1) + int64_t(by >> 1) * (side >> 1) + (bx >> 1);
            const C* Lp = t.loc + pb * P1;
            const C* zq = t.Zq + par * P1;
            const C* ziq = t.Ziq + par * P1;
            T yr[P1], yi[P1];
#pragma unroll
            for (int ll = 0; ll < P1; ++ll) {
                yr[ll] = T(0);
                yi[ll] = T(0);
            }
            T c0 = T(0);
#pragma unroll
            for (int k = 1; k < P1; ++k) {
                const C bk = Lp[k];
                const C z = zq[k];
                const T wr = bk.x * z.x - bk.y * z.y;
                const T wi = bk.x * z.y + bk.y * z.x;
                c0 += wr;
#pragma unroll
                for (int ll = 1; ll <= k; ++ll) {
                    yr[ll] = fma(c_ops.l2l[ll][k], wr, yr[ll]);
                    yi[ll] = fma(c_ops.l2l[ll][k], wi, yi[ll]);
                }
            }
            a0 = t.L0[pb] + double(c0);
#pragma unroll
            for (int ll = 1; ll < P1; ++ll) {
                const C z = ziq[ll];
                Lr[ll] = yr[ll] * z.x - yi[ll] * z.y;
                Li[ll] = yr[ll] * z.y + yi[ll] * z.x;
            }
        }
        m2l_list<T, P1>(t, l, bx, by, sub, S, Lr, Li, a0, sumS);
    }
    for (int o = 1; o < S; o <<= 1) {
#pragma unroll
        for (int i = 0; i < P1; ++i) {
            Lr[i] += __shfl_xor_sync(0xffffffffu, Lr[i], o);
            Li[i] += __shfl_xor_sync(0xffffffffu, Li[i], o);
        }
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        sumS += __shfl_xor_sync(0xffffffffu, sumS, o);
    }
    if (act && sub == 0) {
        const double L0 = a0 + lnS * sumS + double(Lr[0]);
        C* out = t.loc + (off + b) * P1;
        t.L0[off + b] = L0;
        out[0] = cmake<T>(T(L0), T(0));
#pragma unroll
        for (int ll = 1; ll < P1; ++ll) out[ll] = cmake<T>(Lr[ll], Li[ll]);
    }
    double nearS = 0.0;  // leaf level: the near leaves' monopoles (the log h part of the near field)
    if (L2P) {
        if (act) {
            const int bx = int(b % side), by = int(b / side);
            for (int e = sub; e < t.n_near; e += S) {
                const int2 o = t.near[e];
                const int sx = bx + o.x, sy = by + o.y;
                if (sx >= 0 && sy >= 0 && sx < side && sy < side) nearS += t.S[off + int64_t(sy) * side + sx];
            }
        }
        for (int o = 1; o < S; o <<= 1) nearS += __shfl_xor_sync(0xffffffffu, nearS, o);
    }
    if (L2P && act) {
        // leaf level: every thread of the group holds the full local (butterfly sums) and
        // adds the far field at 64 / S of the leaf's cells to the near field already in p_out
        const T inv2pi = T(0.15915494309189533576888376337251);
        const double lnh = t.lnh;
        const T c0 = T((a0 + lnS * sumS + lnh * nearS) * 0.15915494309189533576888376337251) + Lr[0] * inv2pi;
        const int bx = int(b % side), by = int(b / side);
        for (int c = sub; c < 64; c += S) {
            const T wr = (T(c & 7) - T(3.5)) * T(0.125);
            const T wi = (T(c >> 3) - T(3.5)) * T(0.125);
            T sr = Lr[P1 - 1], si = Li[P1 - 1];
#pragma unroll
            for (int ll = P1 - 2; ll >= 1; --ll) {
                const T nr = fma(sr, wr, fma(-si, wi, Lr[ll]));
                const T ni = fma(sr, wi, fma(si, wr, Li[ll]));
                sr = nr;
                si = ni;
            }
            const T ser = sr * wr - si * wi;
            T* dst = p_out + int64_t(by * 8 + (c >> 3)) * t.n + bx * 8 + (c & 7);
            *dst = *dst + fma(ser, inv2pi, c0);
        }
    }
}

// ------------------------------------------------------------------------------------
// (a1) + leaf multipoles, mixed precision: one warp per strip of 128 cells (4 per lane)
// and kRhsLeafRows leaf rows (8 grid rows each), so the two halo rows are read once per 16
// rows.  Rows of the five fields stream through a kRhsRing-slot ring in shared memory per
// warp by asynchronous 16-byte copies (each slot also holds the float4 left and right of
// the strip), kRhsRing - 1 rows in flight.  As a row lands each lane turns it into the
// four values the stencil needs, u, v, a = chi (us_x - u) and b = chi (us_y - v), held in a
// register window of three rows (the slot is free again at once); the row in the middle
// of the window is then differenced (x neighbours by shuffles, the strip's edge columns
// from the halo float4) and its q written.  The leaf multipoles (Eq. alphaK) accumulate
// over a leaf row's 8 rows in registers, from the CTA's shared copy of the table
// omega_c^k / k (two entries per 16-byte read): each lane holds half a leaf row, and the
// two halves of a leaf are combined by one shuffle when the leaf row is done.  The cell
// (7 - x, 7 - y) of a leaf sits at -omega of the cell (x, y), so its powers differ only
// by (-1)^k: rows 0-3 park their q in shared memory, and rows 4-7 add s = q + q' to the
// even powers and d = q - q' to the odd ones (half the table, half the FMAs).
// CTAs of two warps: the 2048 warps of a 2048^2 grid spread over the 152 SMs 13 or 14 to
// an SM (eight-warp CTAs put 16 on some SMs and 8 on the rest).
// ------------------------------------------------------------------------------------
constexpr int kRhsRing = 4;                              // ring slots per warp (rows in flight + 1)
constexpr int kRhsWarps = 2;                             // warps per CTA
constexpr int kRhsLeafRows = 2;                          // leaf rows per warp
constexpr int kRhsSlot = 5 * 34;                         // float4 per slot: 5 fields x (32 lanes + 2 halo)
constexpr size_t kRhsRingBytes = size_t(kRhsWarps) * kRhsRing * kRhsSlot * sizeof(float4);
constexpr size_t kRhsParkBytes = size_t(kRhsWarps) * 4 * 32 * sizeof(float4);  // rows 0-3 of a leaf row
// dynamic shared memory: the P2M table (omega_c^k / k, k = 1..P1-1, for the 32 cells of
// leaf rows 4-7; P1 is odd, so a row of P1 + 1 entries starts 16-byte aligned and the rows
// of the two cells a warp reads at once, 4 apart, sit 16 banks apart), the parked q, then
// the rings
__host__ __device__ constexpr int rhs_wstride(int P1) { return P1 + 1; }
constexpr size_t rhs_smem_bytes(int P1) {
    return size_t(32) * rhs_wstride(P1) * sizeof(float2) + kRhsParkBytes + kRhsRingBytes;
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int P1>
__global__ void __launch_bounds__(32 * kRhsWarps, (P1 <= 17 ? 16 : 8) / kRhsWarps) k_rhs_p2m_fast(Tree<float> t, const float* __restrict__ u,
                                                    const float* __restrict__ v, const float* __restrict__ chi,
                                                    const float* __restrict__ usx, const float* __restrict__ usy,
                                                    float rho, float lam, float* __restrict__ f_out) {
    static_assert(P1 % 2 == 1, "the table is read two entries at a time");
    constexpr int WS = rhs_wstride(P1);
    extern __shared__ __align__(16) float4 rhs_smem[];
    float2* Ws = reinterpret_cast<float2*>(rhs_smem);  // [32 cells of rows 4-7][WS]: entries 0..P1-2 used
    float4* park = rhs_smem + 32 * WS / 2;            // [warp][row 0-3][lane]
    float4* rhs_ring = park + kRhsWarps * 4 * 32;
    const int n = t.n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t wid = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int strips = (n + 127) >> 7;
    const int LY0 = int(wid / strips) * kRhsLeafRows, sxi = int(wid % strips);
    const bool live = LY0 < t.nL;                   // warp-uniform
    const int nly = min(kRhsLeafRows, t.nL - LY0);  // leaf rows of this warp
    const int xs = sxi * 128, x0 = xs + 4 * lane;
    const bool act = x0 < n;
    const bool hasL = xs > 0, hasR = xs + 128 < n;  // the strip's neighbours exist
    const int y0 = 8 * LY0, ylast = y0 + 8 * nly - 1;
    const float inv2h = 0.5f / float(t.h);
    const float hh = float(t.h) * float(t.h);
    // ring[slot][field][34]: entry 0 the float4 left of the strip, 1 + lane the lane's, 33 the
    // float4 right of it; fields u, v, chi, us_x, us_y
    float4* ring = rhs_ring + size_t(warp) * kRhsRing * kRhsSlot;
    const float* fld[5] = {u, v, chi, usx, usy};
    auto slot = [&](int yy) { return ring + ((yy - y0 + 1) % kRhsRing) * kRhsSlot; };
    auto issue = [&](int yy) {  // one commit group per row (empty outside the grid or the band's rows)
        if (yy >= 0 && yy < n && yy <= ylast + 1) {
            const int64_t g = int64_t(yy) * n;
            float4* sl = slot(yy);
#pragma unroll
            for (int f = 0; f < 5; ++f) {
                if (act) cp_async16(sl + f * 34 + 1 + lane, fld[f] + g + x0);
                if (lane == 0 && hasL) cp_async16(sl + f * 34, fld[f] + g + xs - 4);
                if (lane == 31 && hasR) cp_async16(sl + f * 34 + 33, fld[f] + g + xs + 128);
            }
        }
        cp_async_commit();
    };
    // x-derivative of the lane's 4 values e (with left / right neighbours) at cells x0..x0+3
    const bool xedge = x0 == 0 || x0 + 4 >= n;  // lanes holding the first or last column
    auto ddx = [&](const float e[4], float left, float right, float d[4]) {
        if (!xedge) {
            d[0] = (e[1] - left) * inv2h;
            d[1] = (e[2] - e[0]) * inv2h;
            d[2] = (e[3] - e[1]) * inv2h;
            d[3] = (right - e[2]) * inv2h;
            return;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int x = x0 + i;
            const float em = i == 0 ? left : e[i - 1];
            const float ep = i == 3 ? right : e[i + 1];
            if (x == 0)
                d[i] = (-3.f * e[0] + 4.f * e[1] - e[2]) * inv2h;
            else if (x == n - 1)
                d[i] = (3.f * e[3] - 4.f * e[2] + e[1]) * inv2h;
            else
                d[i] = (ep - em) * inv2h;
        }
    };
    // a row's u, v, b read straight from global memory (the one-sided differences of the
    // grid's first and last rows need a third row)
    auto row_uvb = [&](int yy, float uo[4], float vo[4], float bo[4]) {
        const int64_t g = int64_t(yy) * n + x0;
        const float4 u4 = ld4(u + g), v4 = ld4(v + g), c4 = ld4(chi + g), s4 = ld4(usy + g);
        uo[0] = u4.x, uo[1] = u4.y, uo[2] = u4.z, uo[3] = u4.w;
        vo[0] = v4.x, vo[1] = v4.y, vo[2] = v4.z, vo[3] = v4.w;
        bo[0] = c4.x * (s4.x - v4.x), bo[1] = c4.y * (s4.y - v4.y), bo[2] = c4.z * (s4.z - v4.z),
        bo[3] = c4.w * (s4.w - v4.w);
    };

    // register window: rows y - 1 (0), y (1), y + 1 (2); per row the lane's u, v, a, b and the
    // edge column's u, v, a (lane 0: the column left of the strip, lane 31: right of it)
    float U[3][4], V[3][4], A[3][4], B[3][4], HU[3], HV[3], HA[3];
#pragma unroll
    for (int w = 0; w < 3; ++w) {
#pragma unroll
        for (int i = 0; i < 4; ++i) U[w][i] = V[w][i] = A[w][i] = B[w][i] = 0.f;
        HU[w] = HV[w] = HA[w] = 0.f;
    }
    float ar[P1], ai[P1];
#pragma unroll
    for (int k = 0; k < P1; ++k) {
        ar[k] = 0.f;
        ai[k] = 0.f;
    }
    // the first rows go out before the table is staged (its loads then overlap them)
    if (live) {
#pragma unroll
        for (int d = -1; d < kRhsRing - 1; ++d) issue(y0 + d);
    }
#pragma unroll
    for (int j = 0; j < (32 * (P1 - 1)) / (32 * kRhsWarps); ++j) {
        const int i = int(threadIdx.x) + j * 32 * kRhsWarps;
        const int c = i / (P1 - 1), k = i % (P1 - 1);
        Ws[c * WS + k] = t.Wp2m[(32 + c) * P1 + 1 + k];
    }
    static_assert((32 * (P1 - 1)) % (32 * kRhsWarps) == 0, "whole table rows per thread");
    float4* parked = park + warp * 4 * 32;
    __syncthreads();
    if (!live) return;
    // one row: shift the window, convert row yy into slot 2, then difference the row in slot
    // 1 (y = yy - 1) with slots 0 (y - 1) and 2 (y + 1)
    constexpr int OW = 0, MW = 1, NW = 2;
    auto step = [&](int yy) {
        cp_async_wait<kRhsRing - 1>();  // row yy has landed (kRhsRing - 1 later rows may be in flight)
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            U[0][i] = U[1][i], V[0][i] = V[1][i], A[0][i] = A[1][i], B[0][i] = B[1][i];
            U[1][i] = U[2][i], V[1][i] = V[2][i], A[1][i] = A[2][i], B[1][i] = B[2][i];
        }
        HU[0] = HU[1], HV[0] = HV[1], HA[0] = HA[1];
        HU[1] = HU[2], HV[1] = HV[2], HA[1] = HA[2];
        if (yy >= 0 && yy < n) {
            const float4* sl = slot(yy);
            if (act) {
                const float4 u4 = sl[1 + lane], v4 = sl[34 + 1 + lane], c4 = sl[68 + 1 + lane],
                             x4 = sl[102 + 1 + lane], y4 = sl[136 + 1 + lane];
                U[NW][0] = u4.x, U[NW][1] = u4.y, U[NW][2] = u4.z, U[NW][3] = u4.w;
                V[NW][0] = v4.x, V[NW][1] = v4.y, V[NW][2] = v4.z, V[NW][3] = v4.w;
                A[NW][0] = c4.x * (x4.x - u4.x), A[NW][1] = c4.y * (x4.y - u4.y), A[NW][2] = c4.z * (x4.z - u4.z),
                A[NW][3] = c4.w * (x4.w - u4.w);
                B[NW][0] = c4.x * (y4.x - v4.x), B[NW][1] = c4.y * (y4.y - v4.y), B[NW][2] = c4.z * (y4.z - v4.z),
                B[NW][3] = c4.w * (y4.w - v4.w);
            }
            if (lane == 0 && hasL) {
                const float uu = sl[0].w, vv = sl[34].w, cc = sl[68].w, xx = sl[102].w;
                HU[NW] = uu, HV[NW] = vv, HA[NW] = cc * (xx - uu);
            } else if (lane == 31 && hasR) {
                const float uu = sl[33].x, vv = sl[34 + 33].x, cc = sl[68 + 33].x, xx = sl[102 + 33].x;
                HU[NW] = uu, HV[NW] = vv, HA[NW] = cc * (xx - uu);
            }
        }
        __syncwarp();  // every lane has read the slot: it takes row yy + kRhsRing
        issue(yy + kRhsRing);
        const int y = yy - 1;  // the row in the middle of the window
        if (y < y0) return;    // warp-uniform
        // x neighbours of row y: the adjacent lanes' edge values, the strip's edges from the halo
        float uL = __shfl_up_sync(0xffffffffu, U[MW][3], 1), vL = __shfl_up_sync(0xffffffffu, V[MW][3], 1),
              aL = __shfl_up_sync(0xffffffffu, A[MW][3], 1);
        float uR = __shfl_down_sync(0xffffffffu, U[MW][0], 1), vR = __shfl_down_sync(0xffffffffu, V[MW][0], 1),
              aR = __shfl_down_sync(0xffffffffu, A[MW][0], 1);
        if (lane == 0) uL = HU[MW], vL = HV[MW], aL = HA[MW];
        if (lane == 31) uR = HU[MW], vR = HV[MW], aR = HA[MW];
        float ux[4], vx[4], ax[4];
        ddx(U[MW], uL, uR, ux);
        ddx(V[MW], vL, vR, vx);
        ddx(A[MW], aL, aR, ax);
        float uy[4], vy[4], by[4];
        if (y == 0) {  // one-sided: rows 0, 1 (window) and 2 (global)
            float u2[4] = {0, 0, 0, 0}, v2[4] = {0, 0, 0, 0}, b2[4] = {0, 0, 0, 0};
            if (act && n >= 3) row_uvb(2, u2, v2, b2);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                uy[i] = (-3.f * U[MW][i] + 4.f * U[NW][i] - u2[i]) * inv2h;
                vy[i] = (-3.f * V[MW][i] + 4.f * V[NW][i] - v2[i]) * inv2h;
                by[i] = (-3.f * B[MW][i] + 4.f * B[NW][i] - b2[i]) * inv2h;
            }
        } else if (y == n - 1) {  // one-sided: rows n-1, n-2 (window) and n-3 (global)
            float um[4] = {0, 0, 0, 0}, vm[4] = {0, 0, 0, 0}, bm[4] = {0, 0, 0, 0};
            if (act && n >= 3) row_uvb(n - 3, um, vm, bm);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                uy[i] = (3.f * U[MW][i] - 4.f * U[OW][i] + um[i]) * inv2h;
                vy[i] = (3.f * V[MW][i] - 4.f * V[OW][i] + vm[i]) * inv2h;
                by[i] = (3.f * B[MW][i] - 4.f * B[OW][i] + bm[i]) * inv2h;
            }
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                uy[i] = (U[NW][i] - U[OW][i]) * inv2h;
                vy[i] = (V[NW][i] - V[OW][i]) * inv2h;
                by[i] = (B[NW][i] - B[OW][i]) * inv2h;
            }
        }
        float q[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float pen = ax[i] + by[i];
            const float f = -rho * (ux[i] * ux[i] + 2.f * uy[i] * vx[i] + vy[i] * vy[i]) + rho * lam * pen;
            q[i] = f * hh;
            if (f_out && act) f_out[int64_t(y) * n + x0 + i] = f;
        }
        const int r = y - y0;
        const int LY = LY0 + (r >> 3), ry = r & 7;
        if (act) {
            const int cx0 = x0 & 7;
            const int64_t leaf = int64_t(LY) * t.nL + (x0 >> 3);
            *reinterpret_cast<float4*>(t.q + leaf * 64 + ry * 8 + cx0) = make_float4(q[0], q[1], q[2], q[3]);
            if (ry < 4) {
                parked[ry * 32 + lane] = make_float4(q[0], q[1], q[2], q[3]);
            } else {
                // the mirror of cell cx0 + i is cell 7 - cx0 - i of row 7 - ry: the other lane
                // of the leaf, its parked entry 3 - i
                const float4 m = parked[(7 - ry) * 32 + (lane ^ 1)];
                const float qm[4] = {m.w, m.z, m.y, m.x};
                // leaf multipole partials: (q + (-1)^k q') omega^k / k, omega = (cell - leaf
                // centre) / 8, from the table
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float4* w = reinterpret_cast<const float4*>(Ws + ((ry - 4) * 8 + cx0 + i) * WS);
                    const float sp = q[i] + qm[i], dm = q[i] - qm[i];
                    ar[0] += sp;
#pragma unroll
                    for (int k = 1; k < P1; k += 2) {
                        const float4 wk = w[(k - 1) >> 1];  // entries k (odd) and k + 1 (even)
                        ar[k] = fmaf(dm, wk.x, ar[k]);
                        ai[k] = fmaf(dm, wk.y, ai[k]);
                        ar[k + 1] = fmaf(sp, wk.z, ar[k + 1]);
                        ai[k + 1] = fmaf(sp, wk.w, ai[k + 1]);
                    }
                }
            }
        }
        if (ry == 7) {  // the leaf row is done: the two halves of each leaf (lanes 2L, 2L + 1)
#pragma unroll
            for (int k = 0; k < P1; ++k) {
                ar[k] += __shfl_xor_sync(0xffffffffu, ar[k], 1);
                ai[k] += __shfl_xor_sync(0xffffffffu, ai[k], 1);
            }
            if (act && !(lane & 1)) {
                const int64_t box = level_offset(t.Lleaf) + int64_t(LY) * t.nL + (x0 >> 3);
                store_S_leaf(t, box, ar[0]);
                float2* M = t.mp + box * P1;
                M[0] = make_float2(ar[0], 0.f);
#pragma unroll
                for (int k = 1; k < P1; ++k) M[k] = make_float2(ar[k], ai[k]);
            }
#pragma unroll
            for (int k = 0; k < P1; ++k) {
                ar[k] = 0.f;
                ai[k] = 0.f;
            }
        }
    };
#pragma unroll 1
    for (int yy = y0 - 1; yy <= ylast + 1; ++yy) step(yy);
    cp_async_wait<0>();  // no copy outlives the warp
}

// ------------------------------------------------------------------------------------
// Local evaluation at the leaf cells, mixed precision, after the near field: the leaf
// locals (written by the leaf-level translations, which run beside the near field) are
// evaluated at all 64 cells of every leaf and added to the near field already in P.
// One CTA per 8 x 8 leaves (64 x 64 cells), 256 threads; a thread owns 4 cells in each of
// 4 rows (float4 read-modify-writes, the reads issued first).  The constant term of each leaf, Re b_0 (FP64) plus the
// log h part of the near field (log h times the near leaves' monopoles), is formed once.
// ------------------------------------------------------------------------------------
constexpr int kMaxD = 3;  // near radius (in leaves) of the split solve

template <int P1>
__global__ void __launch_bounds__(256) k_l2p_leaf(Tree<float> t, float* __restrict__ p_out) {
    typedef float2 C;
    constexpr int TL = 8;  // leaves per side of the CTA's tile
    __shared__ C Ls[TL * TL][P1];
    __shared__ float c0s[TL * TL];
    __shared__ double nS[(TL + 2 * kMaxD) * (TL + 2 * kMaxD)];
    const int l = t.Lleaf, side = 1 << l;
    const int LX0 = blockIdx.x * TL, LY0 = blockIdx.y * TL;
    const int64_t off = level_offset(l);
    const int tid = threadIdx.x;
    // this thread's 4 rows x 4 cells: quad q of the 16 per 64-cell row, rows r0 + 16 j
    const int q = tid & 15, r0 = tid >> 4;
    float4* dst[4];
    float4 pv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {  // the near field already in P, loaded first
        dst[j] = reinterpret_cast<float4*>(p_out + int64_t(LY0 * 8 + r0 + 16 * j) * t.n + LX0 * 8 + q * 4);
        pv[j] = *dst[j];
    }
    for (int i = tid; i < TL * TL * P1; i += 256) {
        const int lf = i / P1, k = i - lf * P1;
        const int64_t b = int64_t(LY0 + lf / TL) * side + LX0 + lf % TL;
        Ls[lf][k] = t.loc[(off + b) * P1 + k];
    }
    // the monopoles of the (TL + 2D)^2 leaves around the tile, staged once; each leaf then
    // sums its near leaves in near-list order (out-of-grid leaves read zero)
    const int D = t.Dmax, W = TL + 2 * D;
    for (int i = tid; i < W * W; i += 256) {
        const int sx = LX0 - D + i % W, sy = LY0 - D + i / W;
        nS[i] = (sx >= 0 && sy >= 0 && sx < side && sy < side) ? t.S[off + int64_t(sy) * side + sx] : 0.0;
    }
    __syncthreads();
    if (tid < TL * TL) {
        const int lx = tid % TL, ly = tid / TL;
        double nearS = 0.0;
        for (int e = 0; e < t.n_near; ++e) {
            const int2 o = t.near[e];
            nearS += nS[(ly + o.y + D) * W + lx + o.x + D];
        }
        const double L0 = t.L0[off + int64_t(LY0 + ly) * side + LX0 + lx];
        c0s[tid] = float((L0 + t.lnh * nearS) * 0.15915494309189533576888376337251);
    }
    __syncthreads();
    const float inv2pi = 0.15915494309189533576888376337251f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int row = r0 + 16 * j;
        const int lf = (row >> 3) * TL + (q >> 1);
        const C* L = Ls[lf];
        const float wi = (float(row & 7) - 3.5f) * 0.125f;
        float out[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float wr = (float((q & 1) * 4 + c) - 3.5f) * 0.125f;
            float sr = L[P1 - 1].x, si = L[P1 - 1].y;
#pragma unroll
            for (int ll = P1 - 2; ll >= 1; --ll) {
                const float nr = fmaf(sr, wr, fmaf(-si, wi, L[ll].x));
                const float ni = fmaf(sr, wi, fmaf(si, wr, L[ll].y));
                sr = nr;
                si = ni;
            }
            const float ser = sr * wr - si * wi;
            out[c] = fmaf(ser, inv2pi, c0s[lf]);
        }
        float4 p = pv[j];
        p.x += out[0];
        p.y += out[1];
        p.z += out[2];
        p.w += out[3];
        *dst[j] = p;
    }
}

// ------------------------------------------------------------------------------------
// Downward pass, levels 2..lt in one launch (mixed precision): one warp per box of level
// lt walks its ancestors from level 2 down.  At each level the lanes split the box's
// interaction list (entry e to lane e mod 32) and combine by a butterfly, then add the
// local-to-local shift of the level above, which the warp holds in registers.  Every
// ancestor's local is written by each of its descendants' warps, with identical values:
// per level the arithmetic and its order are those of k_m2l_reg with 32 threads per box.
// ------------------------------------------------------------------------------------
struct LevelLogs {
    double lnS[16];  // log of the box side at each level
};

template <int P1>
__global__ void __launch_bounds__(128) k_m2l_chain(Tree<float> t, int lt, LevelLogs lg) {
    typedef float2 C;
    const int lane = threadIdx.x & 31;
    const int64_t wb = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;  // box at level lt
    const int sidet = 1 << lt;
    if (wb >= int64_t(sidet) * sidet) return;  // warp-uniform
    const int bxt = int(wb % sidet), byt = int(wb / sidet);
    float Pr[P1], Pi[P1];  // the parent's local (levels >= 3)
    double P0 = 0.0;       // and its FP64 constant term
#pragma unroll
    for (int i = 0; i < P1; ++i) {
        Pr[i] = 0.f;
        Pi[i] = 0.f;
    }
    for (int l = 2; l <= lt; ++l) {
        const int side = 1 << l;
        const int bx = bxt >> (lt - l), by = byt >> (lt - l);
        const int64_t off = level_offset(l);
        const int64_t b = int64_t(by) * side + bx;
        const int par = (bx & 1) + 2 * (by & 1);
        float Lr[P1], Li[P1];
#pragma unroll
        for (int i = 0; i < P1; ++i) {
            Lr[i] = 0.f;
            Li[i] = 0.f;
        }
        double a0 = 0.0, sumS = 0.0;
        if (l >= 3 && lane == 0) {  // local-to-local from the parent held in registers
            const C* zq = t.Zq + par * P1;
            const C* ziq = t.Ziq + par * P1;
            float yr[P1], yi[P1];
#pragma unroll
            for (int ll = 0; ll < P1; ++ll) {
                yr[ll] = 0.f;
                yi[ll] = 0.f;
            }
            float c0 = 0.f;
#pragma unroll
            for (int k = 1; k < P1; ++k) {
                const C z = zq[k];
                const float wr = Pr[k] * z.x - Pi[k] * z.y;
                const float wi = Pr[k] * z.y + Pi[k] * z.x;
                c0 += wr;
#pragma unroll
                for (int ll = 1; ll <= k; ++ll) {
                    yr[ll] = fmaf(c_ops.l2l[ll][k], wr, yr[ll]);
                    yi[ll] = fmaf(c_ops.l2l[ll][k], wi, yi[ll]);
                }
            }
            a0 = P0 + double(c0);
#pragma unroll
            for (int ll = 1; ll < P1; ++ll) {
                const C z = ziq[ll];
                Lr[ll] = yr[ll] * z.x - yi[ll] * z.y;
                Li[ll] = yr[ll] * z.y + yi[ll] * z.x;
            }
        }
        m2l_list<float, P1>(t, l, bx, by, lane, 32, Lr, Li, a0, sumS);
        for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
            for (int i = 0; i < P1; ++i) {
                Lr[i] += __shfl_xor_sync(0xffffffffu, Lr[i], o);
                Li[i] += __shfl_xor_sync(0xffffffffu, Li[i], o);
            }
            a0 += __shfl_xor_sync(0xffffffffu, a0, o);
            sumS += __shfl_xor_sync(0xffffffffu, sumS, o);
        }
        const double L0 = a0 + lg.lnS[l] * sumS + double(Lr[0]);
        if (lane == 0) {
            C* out = t.loc + (off + b) * P1;
            t.L0[off + b] = L0;
            out[0] = make_float2(float(L0), 0.f);
#pragma unroll
            for (int ll = 1; ll < P1; ++ll) out[ll] = make_float2(Lr[ll], Li[ll]);
        }
        P0 = L0;
#pragma unroll
        for (int ll = 1; ll < P1; ++ll) {
            Pr[ll] = Lr[ll];
            Pi[ll] = Li[ll];
        }
    }
}

// ------------------------------------------------------------------------------------
// Downward pass in two launches (mixed precision, leaf level >= 5).  The multipole-to-local
// part of every box's local expansion depends only on the multipoles, so all levels
// 2..L run as one grid (k_m2l_far); the local-to-local shifts, which chain the levels,
// then run per subtree inside k_down_tree, which ends with the local evaluation at the
// cells.  lr = L - 3 is the level of the subtrees' roots: one CTA per level-lr box owns
// its box and the 84 boxes below it.
// ------------------------------------------------------------------------------------
template <int P1>
struct FarOcc {  // resident 128-thread CTAs per SM of k_m2l_far (register budget without spills)
    static constexpr int value = P1 <= 13 ? 5 : P1 <= 17 ? 4 : 3;
};
constexpr int kDownAnc = 12;     // ancestor levels 2..lr-1 a CTA of k_down_tree can hold (L <= 17)
constexpr int kDownSub = 85;     // boxes of a subtree: 1 + 4 + 16 + 64
// threads of a k_down_tree CTA: 128 lets seven CTAs share an SM, so the 1024 subtrees of a
// 2048^2 grid run in one wave (256-thread CTAs, four an SM, took 1.7)
constexpr int kDownThreads = 128;
// Dynamic shared memory a k_down_tree CTA reserves and does not use, for near radius >= 2:
// with it six CTAs (not seven) fit an SM.  The longer near field of those plans holds back
// the surface path (lower priority), whose tractions and force sums can still be pending
// when the subtrees start; with the room they run beside the subtrees instead of after the
// last one.  At near radius 1 the surface path is done by then, and the seventh CTA wins.
constexpr int kDownRoom = 4096;

// Multipole-to-local part of the local expansion of every box of levels 2..L: S threads per
// box (a power of two), levels finest first in one grid.  The FP64 constant term is
// a0 + log(box side) sum S + Re part (lnRoot: log of the root box side); it and the coefficients go to loc/L0 for levels >= lr and
// to the side buffers locA/L0A for the shared ancestor levels below lr, which k_down_tree
// reads from every CTA while it writes the complete locals to loc/L0.
template <int P1>
__global__ void __launch_bounds__(128, FarOcc<P1>::value) k_m2l_far(Tree<float> t, int lr, int S, double lnRoot) {
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    int64_t b = g / S;
    const int sub = int(g % S);
    int l = t.Lleaf;
    while (l >= 2 && b >= (int64_t(1) << (2 * l))) {
        b -= int64_t(1) << (2 * l);
        --l;
    }
    const bool act = l >= 2;
    float Lr[P1], Li[P1];
#pragma unroll
    for (int i = 0; i < P1; ++i) {
        Lr[i] = 0.f;
        Li[i] = 0.f;
    }
    float ah = 0.f, al = 0.f, sh = 0.f, sl = 0.f;  // double-float sum S log|tau|, sum S
    if (act) {
        const int side = 1 << l;
        m2l_list_df<P1>(t, l, int(b % side), int(b / side), sub, S, Lr, Li, ah, al, sh, sl);
    }
    for (int o = 1; o < S; o <<= 1) {
#pragma unroll
        for (int i = 0; i < P1; ++i) {
            Lr[i] += __shfl_xor_sync(0xffffffffu, Lr[i], o);
            Li[i] += __shfl_xor_sync(0xffffffffu, Li[i], o);
        }
        const float oah = __shfl_xor_sync(0xffffffffu, ah, o), oal = __shfl_xor_sync(0xffffffffu, al, o);
        const float osh = __shfl_xor_sync(0xffffffffu, sh, o), osl = __shfl_xor_sync(0xffffffffu, sl, o);
        df_add(ah, al, oah, oal);
        df_add(sh, sl, osh, osl);
    }
    if (act && sub == 0) {
        const int64_t i = level_offset(l) + b;
        const double lnS = fma(double(-l), 0.69314718055994530941723212145818, lnRoot);  // log(side / 2^l)
        const double L0 = df_to(ah, al) + lnS * df_to(sh, sl) + double(Lr[0]);
        float2* out = (l < lr ? t.locA : t.loc) + i * P1;
        (l < lr ? t.L0A : t.L0)[i] = L0;
        out[0] = make_float2(float(L0), 0.f);
#pragma unroll
        for (int ll = 1; ll < P1; ++ll) out[ll] = make_float2(Lr[ll], Li[ll]);
    }
}

// Local-to-local shift of a parent's complete local (Lp; constant term P0 as a double-float
// pair) to its child in quadrant q, added in place to the child's multipole-to-local part
// (Lc; constant term L0c, a pair): w_k = zeta_q^k b_k, c_l = (2 zeta_q)^-l sum_{k >= l}
// C(k, l) w_k, and the constant b_0 + sum_k Re w_k.  One thread, every loop unrolled
// (constant-bank binomials); zq, ziq: the quadrant's zeta_q^k and (2 zeta_q)^-k.
template <int P1>
__device__ __forceinline__ void l2l_child(const float2* Lp, float2 P0, const float2* zq, const float2* ziq,
                                          float2* Lc, float2* L0c) {
    float yr[P1], yi[P1];
#pragma unroll
    for (int ll = 0; ll < P1; ++ll) {
        yr[ll] = 0.f;
        yi[ll] = 0.f;
    }
    float c0 = 0.f;
#pragma unroll
    for (int k = 1; k < P1; ++k) {
        const float2 bk = Lp[k], z = zq[k];
        const float wr = bk.x * z.x - bk.y * z.y;
        const float wi = bk.x * z.y + bk.y * z.x;
        c0 += wr;
#pragma unroll
        for (int ll = 1; ll <= k; ++ll) {
            yr[ll] = fmaf(c_ops.l2l[ll][k], wr, yr[ll]);
            yi[ll] = fmaf(c_ops.l2l[ll][k], wi, yi[ll]);
        }
    }
    float hi = P0.x, lo = P0.y;
    df_add(hi, lo, c0, 0.f);
    df_add(hi, lo, L0c->x, L0c->y);
    *L0c = make_float2(hi, lo);
    Lc[0] = make_float2(hi + lo, 0.f);
#pragma unroll
    for (int ll = 1; ll < P1; ++ll) {
        const float2 z = ziq[ll], m = Lc[ll];
        Lc[ll] = make_float2(m.x + (yr[ll] * z.x - yi[ll] * z.y), m.y + (yr[ll] * z.y + yi[ll] * z.x));
    }
}

// 8-byte asynchronous copy global -> shared through L1; with valid == false it writes zeros.
__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool valid = true) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src), "r"(valid ? 8 : 0)
                 : "memory");
}

// Local-to-local shifts and local evaluation, one CTA (kDownThreads threads) per box of level
// lr = L - 3, after the near field: the CTA forms the complete locals of its ancestors
// (levels 2..lr-1, from their multipole-to-local parts) and of its 85 subtree boxes,
// writes those it owns (and each ancestor from the one CTA at the ancestor's lower-left
// corner) to loc/L0, and evaluates the 64 leaf locals at the subtree's 64 x 64 cells,
// adding them to the near field in P.  The constant term of each leaf is Re b_0 plus the
// log h part of the near field (log h times the near leaves' monopoles).  Every global
// read (the locals' parts, the leaf monopoles around the subtree, the near field's 64 x 64
// tile) is an asynchronous copy into shared memory issued at the start, so the CTA waits
// for memory once.  Shared slots: ancestors 0 .. na-1 (levels 2 .. lr-1), then the subtree
// by level (1, 4, 16, 64 boxes), row-major within a level: subtree level j's rows are
// runs of 2^j consecutive boxes in the global arrays.
template <int P1>
__global__ void __launch_bounds__(kDownThreads, P1 <= 13 ? 7 : (P1 <= 17 ? 6 : 5)) k_down_tree(Tree<float> t, int lr, float* __restrict__ p_out) {
    typedef float2 C;
    constexpr int TL = 8;  // leaves per side of the subtree
    __shared__ __align__(16) float Pt[TL * 8][TL * 8];  // the near field of the subtree's cells
    __shared__ C Ls[kDownAnc + kDownSub][P1];
    __shared__ double L0s[kDownAnc + kDownSub];  // FP64 constant terms as read and written
    __shared__ float2 L0f[kDownAnc + kDownSub];  // the same as double-float pairs while shifted
    __shared__ float c0s[TL * TL];
    __shared__ double nS[(TL + 2 * kMaxD) * (TL + 2 * kMaxD)];
    __shared__ C Zs[4][P1], Zis[4][P1];
    const int l = t.Lleaf, side = 1 << l;
    const int X = blockIdx.x, Y = blockIdx.y;  // the subtree root at level lr
    const int LX0 = X * TL, LY0 = Y * TL;
    const int tid = threadIdx.x;
    const int na = lr - 2;
    const int nslot = na + kDownSub;
    // the multipole maximum of this solve has been used (the translations ran before)
    if (t.mmax && X == 0 && Y == 0 && tid == 0) *t.mmax = 0u;
    // near-field tile: 64 rows of 16 float4
    for (int i = tid; i < 64 * 16; i += kDownThreads) {
        const int r = i >> 4, c4 = i & 15;
        cp_async16(&Pt[r][c4 * 4], p_out + int64_t(LY0 * 8 + r) * t.n + LX0 * 8 + c4 * 4);
    }
    // multipole-to-local parts: the ancestors (one box a level) ...
    for (int i = tid; i < na * P1; i += kDownThreads) {
        const int s = i / P1, k = i - s * P1, lev = 2 + s;
        const int64_t bi = level_offset(lev) + int64_t(Y >> (lr - lev)) * (1 << lev) + (X >> (lr - lev));
        cp_async8(&Ls[s][k], t.locA + bi * P1 + k);
        if (k == 0) cp_async8(&L0s[s], t.L0A + bi);
    }
    // ... and the subtree, level j as 2^j runs of 2^j P1 coefficients
#pragma unroll
    for (int j = 0; j <= 3; ++j) {
        const int w = 1 << j, lev = lr + j, run = w * P1;
        const int sb = na + (j == 0 ? 0 : j == 1 ? 1 : j == 2 ? 5 : 21);
        const int64_t row0 = level_offset(lev) + int64_t(Y * w) * (1 << lev) + X * w;
        for (int i = tid; i < w * run; i += kDownThreads) {
            const int r = i / run, c = i - r * run;
            cp_async8(&Ls[sb][0] + i, t.loc + (row0 + int64_t(r) * (1 << lev)) * P1 + c);
        }
        for (int i = tid; i < w * w; i += kDownThreads)
            cp_async8(&L0s[sb + i], t.L0 + row0 + int64_t(i >> j) * (1 << lev) + (i & (w - 1)));
    }
    // the monopoles of the (TL + 2D)^2 leaves around the subtree (out-of-grid leaves read zero)
    const int64_t off = level_offset(l);
    const int D = t.Dmax, WD = TL + 2 * D;
    for (int i = tid; i < WD * WD; i += kDownThreads) {
        const int sx = LX0 - D + i % WD, sy = LY0 - D + i / WD;
        const bool in = sx >= 0 && sy >= 0 && sx < side && sy < side;
        cp_async8(&nS[i], t.S + (in ? off + int64_t(sy) * side + sx : 0), in);
    }
    for (int i = tid; i < 4 * P1; i += kDownThreads) {
        cp_async8(&Zs[0][0] + i, t.Zq + i);
        cp_async8(&Zis[0][0] + i, t.Ziq + i);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    for (int i = tid; i < nslot; i += kDownThreads) L0f[i] = df_from(L0s[i]);
    __syncthreads();
    // ancestors 3..lr-1 and the subtree root, each from the slot above (one thread), then
    // the subtree levels 1..3 (one thread per child)
    if (tid == 0) {
        for (int lev = 3; lev <= lr; ++lev) {
            const int ax = X >> (lr - lev), ay = Y >> (lr - lev);
            const int qd = (ax & 1) + 2 * (ay & 1);
            l2l_child<P1>(Ls[lev - 3], L0f[lev - 3], Zs[qd], Zis[qd], Ls[lev - 2], &L0f[lev - 2]);
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int j = 1, cb = na + 1, pb = na; j <= 3; pb = cb, cb += 1 << (2 * j), ++j) {
        if (tid < (1 << (2 * j))) {
            const int sd = 1 << j, cx = tid & (sd - 1), cy = tid >> j;
            const int qd = (cx & 1) + 2 * (cy & 1);
            const int ps = pb + (cy >> 1) * (sd >> 1) + (cx >> 1);
            l2l_child<P1>(Ls[ps], L0f[ps], Zs[qd], Zis[qd], Ls[cb + tid], &L0f[cb + tid]);
        }
        __syncthreads();
    }
    for (int i = tid; i < nslot; i += kDownThreads) L0s[i] = df_to(L0f[i].x, L0f[i].y);
    __syncthreads();
    // write back the complete locals this CTA owns (each ancestor from one CTA)
    for (int i = tid; i < na * P1; i += kDownThreads) {
        const int s = i / P1, k = i - s * P1, lev = 2 + s, sh = lr - lev;
        if (((X | Y) & ((1 << sh) - 1)) != 0) continue;
        const int64_t bi = level_offset(lev) + int64_t(Y >> sh) * (1 << lev) + (X >> sh);
        t.loc[bi * P1 + k] = Ls[s][k];
        if (k == 0) t.L0[bi] = L0s[s];
    }
#pragma unroll
    for (int j = 0; j <= 3; ++j) {
        const int w = 1 << j, lev = lr + j, run = w * P1;
        const int sb = na + (j == 0 ? 0 : j == 1 ? 1 : j == 2 ? 5 : 21);
        const int64_t row0 = level_offset(lev) + int64_t(Y * w) * (1 << lev) + X * w;
        for (int i = tid; i < w * run; i += kDownThreads) {
            const int r = i / run, c = i - r * run;
            t.loc[(row0 + int64_t(r) * (1 << lev)) * P1 + c] = (&Ls[sb][0])[i];
        }
        for (int i = tid; i < w * w; i += kDownThreads) t.L0[row0 + int64_t(i >> j) * (1 << lev) + (i & (w - 1))] = L0s[sb + i];
    }
    const int lb = na + 21;  // the 64 leaf slots, row-major in the subtree
    if (tid < TL * TL) {
        const int lx = tid % TL, ly = tid / TL;
        double nearS = 0.0;
        for (int e = 0; e < t.n_near; ++e) {
            const int2 o = t.near[e];
            nearS += nS[(ly + o.y + D) * WD + lx + o.x + D];
        }
        c0s[tid] = float((L0s[lb + tid] + t.lnh * nearS) * 0.15915494309189533576888376337251);
    }
    __syncthreads();
    // 8 rows x 4 cells per thread: quad q of the 16 per 64-cell row, rows r0 + 8 jr
    const int q = tid & 15, r0 = tid >> 4;
    const float inv2pi = 0.15915494309189533576888376337251f;
    static_assert(kDownThreads == 128, "16 quads x 8 row groups");
#pragma unroll 2
    for (int jr = 0; jr < 8; ++jr) {
        const int row = r0 + 8 * jr;
        const int lf = (row >> 3) * TL + (q >> 1);
        const C* L = Ls[lb + lf];
        const float wi = (float(row & 7) - 3.5f) * 0.125f;
        float out[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float wr = (float((q & 1) * 4 + c) - 3.5f) * 0.125f;
            float sr = L[P1 - 1].x, si = L[P1 - 1].y;
#pragma unroll
            for (int ll = P1 - 2; ll >= 1; --ll) {
                const float nr = fmaf(sr, wr, fmaf(-si, wi, L[ll].x));
                const float ni = fmaf(sr, wi, fmaf(si, wr, L[ll].y));
                sr = nr;
                si = ni;
            }
            const float ser = sr * wr - si * wi;
            out[c] = fmaf(ser, inv2pi, c0s[lf]);
        }
        float4 pq = *reinterpret_cast<const float4*>(&Pt[row][q * 4]);
        pq.x += out[0];
        pq.y += out[1];
        pq.z += out[2];
        pq.w += out[3];
        *reinterpret_cast<float4*>(p_out + int64_t(LY0 * 8 + row) * t.n + LX0 * 8 + q * 4) = pq;
    }
}

// ------------------------------------------------------------------------------------
// Upward pass: G threads per parent box (G = 1, 2 or 4), each shifting 4/G children;
// the partial expansions are combined with shuffles.
// ------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T ld_child(const T* p, bool cg) {
    return cg ? __ldcg(p) : *p;
}

// kCg: read the children through L2 only (they were written by other CTAs of the same launch).
// With kMax, returns the largest |value| among the children's coefficients this thread read
// and (for the thread that writes it) the parent's; else 0.
template <typename T, int P1, bool kCg = false, bool kMax = false>
__device__ __forceinline__ float m2m_parent(const Tree<T>& t, int l, int64_t b, int G, int sub, bool act) {
    typedef typename cplx_of<T>::type C;
    const int side = 1 << l;
    const int64_t coff = level_offset(l + 1), poff = level_offset(l);
    T Br[P1], Bi[P1];
#pragma unroll
    for (int i = 0; i < P1; ++i) {
        Br[i] = T(0);
        Bi[i] = T(0);
    }
    double S = 0.0;
    float mx = 0.f;
    if (act) {
        const int bx = int(b % side), by = int(b / side);
        const int cs = 2 * side;
        for (int q = sub; q < 4; q += G) {
            const int64_t child = coff + int64_t(2 * by + (q >> 1)) * cs + 2 * bx + (q & 1);
            const C* M = t.mp + child * P1;
            const C* zi = t.Ziq + q * P1;
            const C* z = t.Zq + q * P1;
            const double Sd = ld_child(t.S + child, kCg);
            S += Sd;
            const T St = T(Sd);
            if constexpr (kMax) mx = fmaxf(mx, fabsf(float(Sd)));
            T yr[P1], yi[P1];
#pragma unroll
            for (int k = 0; k < P1; ++k) {
                yr[k] = c_ops.m2m[k][0] * St;
                yi[k] = T(0);
            }
#pragma unroll
            for (int j = 1; j < P1; ++j) {
                const C m = ld_child(M + j, kCg);
                if constexpr (kMax) mx = fmaxf(mx, fmaxf(fabsf(float(m.x)), fabsf(float(m.y))));
                const C w = zi[j];
                const T wr = m.x * w.x - m.y * w.y;
                const T wi = m.x * w.y + m.y * w.x;
#pragma unroll
                for (int k = j; k < P1; ++k) {
                    yr[k] = fma(c_ops.m2m[k][j], wr, yr[k]);
                    yi[k] = fma(c_ops.m2m[k][j], wi, yi[k]);
                }
            }
#pragma unroll
            for (int k = 1; k < P1; ++k) {
                const C zk = z[k];
                Br[k] = fma(yr[k], zk.x, fma(-yi[k], zk.y, Br[k]));
                Bi[k] = fma(yr[k], zk.y, fma(yi[k], zk.x, Bi[k]));
            }
        }
    }
    for (int o = 1; o < G; o <<= 1) {
#pragma unroll
        for (int i = 1; i < P1; ++i) {
            Br[i] += __shfl_xor_sync(0xffffffffu, Br[i], o);
            Bi[i] += __shfl_xor_sync(0xffffffffu, Bi[i], o);
        }
        S += __shfl_xor_sync(0xffffffffu, S, o);
    }
    if (act && sub == 0) {
        C* out = t.mp + (poff + b) * P1;
        store_S(t, poff + b, S);
        out[0] = cmake<T>(T(S), T(0));
        if constexpr (kMax) mx = fmaxf(mx, fabsf(float(S)));
#pragma unroll
        for (int k = 1; k < P1; ++k) {
            out[k] = cmake<T>(Br[k], Bi[k]);
            if constexpr (kMax) mx = fmaxf(mx, fmaxf(fabsf(float(Br[k])), fabsf(float(Bi[k]))));
        }
    }
    return mx;
}

// A CTA's largest |coefficient| into the plan-wide maximum (every thread of the CTA calls it).
__device__ __forceinline__ void publish_max(unsigned* dst, float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v > 0.f) atomicMax(dst, __float_as_uint(v));
}

template <typename T, int P1>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 2) k_m2m_reg(Tree<T> t, int l, int G) {
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t nb = int64_t(1) << (2 * l);
    m2m_parent<T, P1>(t, l, g / G, G, int(g % G), g / G < nb);
}

// Levels lmax..0 (lmax <= 3: at most 64 parents) in one CTA of 128 threads, four threads
// per parent, levels separated by block barriers; global writes of one level are read by
// the next.  Small enough (128 threads, <= 128 registers) to share an SM with the
// tensor-core near field, which otherwise holds every SM while the upward pass runs.
template <typename T, int P1>
__global__ void __launch_bounds__(128, 4) k_m2m_top(Tree<T> t, int lmax) {
    for (int l = lmax; l >= 0; --l) {
        const int64_t nb = int64_t(1) << (2 * l);
        for (int64_t base = 0; base < nb * 4; base += 128) {  // trip count uniform over the CTA
            const int64_t g = base + threadIdx.x;
            m2m_parent<T, P1>(t, l, g / 4, 4, int(g % 4), g / 4 < nb);
        }
        __threadfence_block();
        __syncthreads();
    }
}

// Upward pass in one launch (mixed precision): one CTA of 256 threads per box of level lr
// shifts the multipoles of its subtree up from the leaves (up to 4 levels, four threads per
// parent, levels separated by block barriers), and the CTA that finishes last (an arrival
// counter it resets) shifts the levels above lr up to the root, reading the other CTAs'
// results through L2.  In place of one launch per level: the pass is latency-bound.
template <int P1, bool kMax>
__global__ void __launch_bounds__(256, 2) k_up_tree(Tree<float> t, int lr, unsigned* counter) {
    __shared__ bool last;
    const int rx = int(blockIdx.x & ((1u << lr) - 1)), ry = int(blockIdx.x >> lr);
    const int i = threadIdx.x;
    float mx = 0.f;  // largest |coefficient| seen (the tensor-core translations scale by it)
    for (int l = t.Lleaf - 1; l >= lr; --l) {
        const int w = 1 << (l - lr);  // parents per side of the subtree at level l
        const int cnt = 4 * w * w;    // four threads per parent
        if ((i & ~31) < cnt) {        // warps past the last parent skip the level (uniform)
            const int p = i >> 2;
            const int64_t b = int64_t(ry * w + p / w) * (int64_t(1) << l) + rx * w + p % w;
            mx = fmaxf(mx, m2m_parent<float, P1, false, kMax>(t, l, b, 4, i & 3, i < cnt));
        }
        __threadfence_block();
        __syncthreads();
    }
    if (kMax) publish_max(t.mmax, mx);
    if (!counter || lr == 0) return;
    __threadfence();
    if (i == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    mx = 0.f;
    for (int l = lr - 1; l >= 0; --l) {  // at most 64 parents (lr <= 4): one pass of 256 threads
        const int64_t nb = int64_t(1) << (2 * l);
        if ((i & ~31) < 4 * nb) mx = fmaxf(mx, m2m_parent<float, P1, true, kMax>(t, l, i >> 2, 4, i & 3, i < 4 * nb));
        __threadfence_block();
        __syncthreads();
    }
    if (kMax) publish_max(t.mmax, mx);
    if (i == 0) *counter = 0u;
}

// ------------------------------------------------------------------------------------
// Near field + local evaluation, FP32, near offsets within [-D, D]^2 (a bit mask picks
// the theta-near ones).  CTA = 4 x 4 target leaves, 128 threads; a thread owns one target
// column of 8 cells.  For each source column the 16D+15 kernel values it needs along y
// sit in registers; the source column is read as float4 (broadcast to the 8 threads of a
// leaf).  Per source column: (16D+16)/4 + (2D+1)*2 vector loads for (2D+1)*64 FMAs.
// ------------------------------------------------------------------------------------
template <int D>
struct LeafFastGeom {
    static constexpr int NL = 4 + 2 * D;   // source leaves per side
    static constexpr int W = 8 * NL;       // source cells per side
    static constexpr int CS = W + 16;      // smem column stride (floats); room for the 4-float skew
    static constexpr int RK = 8 * D + 7;
    static constexpr int KN = 2 * RK + 1;  // kernel-table rows and entries per row
    static constexpr int KREG = (KN + 3) / 4 * 4;
    static constexpr int KS = ((KREG / 4) % 2 == 1) ? KREG : KREG + 4;  // odd count of 16 B chunks
    static constexpr size_t smem_bytes = sizeof(float) * (size_t(W) * CS + size_t(KN) * KS);
};

template <int D, bool FAR>
__global__ void __launch_bounds__(128) k_leaf_fast(Tree<float> t, unsigned long long nmask, float* __restrict__ p_out) {
    typedef LeafFastGeom<D> G;
    extern __shared__ __align__(16) float smf[];
    float* qs = smf;
    float* ks = smf + G::W * G::CS;
    const int nL = t.nL;
    const int LX0 = blockIdx.x * 4, LY0 = blockIdx.y * 4;
    const int tid = threadIdx.x;
    for (int idx = tid; idx < G::NL * G::NL * 16; idx += blockDim.x) {
        const int leaf = idx >> 4, gr = idx & 15;
        const int sx = leaf % G::NL, sy = leaf / G::NL;
        const int LXs = LX0 - D + sx, LYs = LY0 - D + sy;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (LXs >= 0 && LXs < nL && LYs >= 0 && LYs < nL)
            v = *reinterpret_cast<const float4*>(t.q + (int64_t(LYs) * nL + LXs) * 64 + gr * 4);
        const int y = 8 * sy + (gr >> 1);
        const int x0 = 8 * sx + (gr & 1) * 4;
        const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int x = x0 + i;
            qs[x * G::CS + 4 * ((x >> 3) & 3) + y] = vv[i];
        }
    }
    const float* ktab = FAR ? t.Ktab : t.Krel;  // near-only: log h comes from the monopoles
    for (int idx = tid; idx < G::KN * G::KS; idx += blockDim.x) {
        const int r = idx / G::KS, m = idx % G::KS;
        ks[idx] = (m < G::KN) ? ktab[r * G::KN + m] : 0.f;
    }
    __syncthreads();

    const int tcol = tid & 31, lrow = tid >> 5;
    const int tx = tcol & 7, li = tcol >> 3;
    const int LX = LX0 + li, LY = LY0 + lrow;
    float acc[8], comp[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        acc[j] = 0.f;
        comp[j] = 0.f;
    }
#pragma unroll 1
    for (int dxl = -D; dxl <= D; ++dxl) {
        float part[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) part[j] = 0.f;
#pragma unroll 1
        for (int c = 0; c < 8; ++c) {
            const int dxc = 8 * dxl + c - tx;
            const float4* krow = reinterpret_cast<const float4*>(ks + (dxc + G::RK) * G::KS);
            float kc[G::KREG];
#pragma unroll
            for (int i = 0; i < G::KREG / 4; ++i) {
                const float4 v = krow[i];
                kc[4 * i] = v.x;
                kc[4 * i + 1] = v.y;
                kc[4 * i + 2] = v.z;
                kc[4 * i + 3] = v.w;
            }
            const int xs = 8 * (li + D + dxl) + c;
            const float* qcol = qs + xs * G::CS + 4 * ((xs >> 3) & 3);
#pragma unroll
            for (int dyl = -D; dyl <= D; ++dyl) {
                const int bit = (dyl + D) * (2 * D + 1) + (dxl + D);
                if ((nmask >> bit) & 1ull) {
                    const float4* q4 = reinterpret_cast<const float4*>(qcol + 8 * (lrow + D + dyl));
                    const float4 a = q4[0], bq = q4[1];
                    const float qv[8] = {a.x, a.y, a.z, a.w, bq.x, bq.y, bq.z, bq.w};
#pragma unroll
                    for (int r = 0; r < 8; ++r)
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            part[j] = fmaf(qv[r], kc[8 * (dyl + D) + r - j + 7], part[j]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {  // Kahan-compensated sum of the per-source-column-band partials
            const float y = part[j] - comp[j];
            const float s = acc[j] + y;
            comp[j] = (s - acc[j]) - y;
            acc[j] = s;
        }
    }
    constexpr double inv2pi = 0.15915494309189533576888376337251;
    if (!FAR) {  // near field only: the leaf-level multipole-to-local kernel adds the far field
#pragma unroll
        for (int j = 0; j < 8; ++j)
            p_out[int64_t(LY * 8 + j) * t.n + LX * 8 + tx] = (acc[j] - comp[j]) * float(inv2pi);
        return;
    }
    // local expansion at the 8 targets (Horner in omega = (cell - leaf centre) / 8)
    const int P1 = t.P1;
    const int64_t leaf = level_offset(t.Lleaf) + int64_t(LY) * nL + LX;
    const float2* Lc = t.loc + leaf * P1;
    const float wr = (float(tx) - 3.5f) * 0.125f;
    float sr[8], si[8];
    {
        const float2 top = Lc[P1 - 1];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            sr[j] = top.x;
            si[j] = top.y;
        }
    }
    for (int l = P1 - 2; l >= 1; --l) {
        const float2 Ll = Lc[l];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float wi = (float(j) - 3.5f) * 0.125f;
            const float nr = fmaf(sr[j], wr, fmaf(-si[j], wi, Ll.x));
            const float ni = fmaf(sr[j], wi, fmaf(si[j], wr, Ll.y));
            sr[j] = nr;
            si[j] = ni;
        }
    }
    const double L0 = t.L0[leaf];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float wi = (float(j) - 3.5f) * 0.125f;
        const float ser = sr[j] * wr - si[j] * wi;
        const double phi = L0 + double(ser) + (double(acc[j]) - double(comp[j]));
        p_out[int64_t(LY * 8 + j) * t.n + LX * 8 + tx] = float(phi * inv2pi);
    }
}

// ------------------------------------------------------------------------------------
// Near field only, FP32, 16 targets per thread: a thread owns one target column across
// two vertically adjacent leaves (A above B), so each kernel column in registers serves
// twice as many FMAs.  CTA = 4 x 8 target leaves.  The kernel table in shared memory
// spans |dy| <= 8D + 15 (entries beyond 8D + 7 are never near and hold zeros).
// ------------------------------------------------------------------------------------
template <int D>
struct Near16Geom {
    static constexpr int NLX = 4 + 2 * D;
    static constexpr int NLY = 8 + 2 * D;
    static constexpr int W = 8 * NLX;
    static constexpr int H = 8 * NLY;
    static constexpr int CS = H + 16;
    static constexpr int RKX = 8 * D + 7;
    static constexpr int RKY = 8 * D + 15;
    static constexpr int KR = 2 * RKX + 1;   // rows: dx offsets
    static constexpr int KN = 2 * RKY + 1;   // entries per row: dy offsets
    static constexpr int KREG = (KN + 3) / 4 * 4;
    static constexpr int KS = ((KREG / 4) % 2 == 1) ? KREG : KREG + 4;
    static constexpr size_t smem_bytes = sizeof(float) * (size_t(W) * CS + size_t(KR) * KS);
};

template <int D>
__global__ void __launch_bounds__(128) k_near16(Tree<float> t, unsigned long long nmask, float* __restrict__ p_out) {
    typedef Near16Geom<D> G;
    extern __shared__ __align__(16) float smn[];
    float* qs = smn;
    float* ks = smn + G::W * G::CS;
    const int nL = t.nL;
    const int LX0 = blockIdx.x * 4, LY0 = blockIdx.y * 8;
    const int tid = threadIdx.x;
    for (int idx = tid; idx < G::NLX * G::NLY * 16; idx += blockDim.x) {
        const int leaf = idx >> 4, gr = idx & 15;
        const int sx = leaf % G::NLX, sy = leaf / G::NLX;
        const int LXs = LX0 - D + sx, LYs = LY0 - D + sy;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (LXs >= 0 && LXs < nL && LYs >= 0 && LYs < nL)
            v = *reinterpret_cast<const float4*>(t.q + (int64_t(LYs) * nL + LXs) * 64 + gr * 4);
        const int y = 8 * sy + (gr >> 1);
        const int x0 = 8 * sx + (gr & 1) * 4;
        const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int x = x0 + i;
            qs[x * G::CS + 4 * ((x >> 3) & 3) + y] = vv[i];
        }
    }
    const int KW = 2 * t.Rk + 1;  // host table: |dx|, |dy| <= 8D + 7
    for (int idx = tid; idx < G::KR * G::KS; idx += blockDim.x) {
        const int r = idx / G::KS, m = idx % G::KS;
        const int dy = m - G::RKY;
        float val = 0.f;
        if (m < G::KN && dy >= -t.Rk && dy <= t.Rk) val = t.Krel[r * KW + (dy + t.Rk)];
        ks[idx] = val;
    }
    __syncthreads();

    const int tcol = tid & 31, trow = tid >> 5;
    const int tx = tcol & 7, li = tcol >> 3;
    const int LX = LX0 + li, LYA = LY0 + 2 * trow;
    float acc[16], comp[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        acc[j] = 0.f;
        comp[j] = 0.f;
    }
#pragma unroll 1
    for (int dxl = -D; dxl <= D; ++dxl) {
        float part[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) part[j] = 0.f;
#pragma unroll 1
        for (int c = 0; c < 8; ++c) {
            const int dxc = 8 * dxl + c - tx;
            const float4* krow = reinterpret_cast<const float4*>(ks + (dxc + G::RKX) * G::KS);
            float kc[G::KREG];
#pragma unroll
            for (int i = 0; i < G::KREG / 4; ++i) {
                const float4 v = krow[i];
                kc[4 * i] = v.x;
                kc[4 * i + 1] = v.y;
                kc[4 * i + 2] = v.z;
                kc[4 * i + 3] = v.w;
            }
            const int xs = 8 * (li + D + dxl) + c;
            const float* qcol = qs + xs * G::CS + 4 * ((xs >> 3) & 3);
#pragma unroll
            for (int dyl = -D; dyl <= D + 1; ++dyl) {
                const bool nearA = dyl <= D && ((nmask >> ((dyl + D) * (2 * D + 1) + (dxl + D))) & 1ull);
                const bool nearB = dyl - 1 >= -D && ((nmask >> ((dyl - 1 + D) * (2 * D + 1) + (dxl + D))) & 1ull);
                if (nearA || nearB) {
                    const float4* q4 = reinterpret_cast<const float4*>(qcol + 8 * (2 * trow + D + dyl));
                    const float4 a = q4[0], bq = q4[1];
                    const float qv[8] = {a.x, a.y, a.z, a.w, bq.x, bq.y, bq.z, bq.w};
                    if (nearA) {
#pragma unroll
                        for (int r = 0; r < 8; ++r)
#pragma unroll
                            for (int j = 0; j < 8; ++j)
                                part[j] = fmaf(qv[r], kc[8 * dyl + r - j + G::RKY], part[j]);
                    }
                    if (nearB) {
#pragma unroll
                        for (int r = 0; r < 8; ++r)
#pragma unroll
                            for (int j = 8; j < 16; ++j)
                                part[j] = fmaf(qv[r], kc[8 * dyl + r - j + G::RKY], part[j]);
                    }
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {  // Kahan-compensated sum of the per-source-column-band partials
            const float y = part[j] - comp[j];
            const float s2 = acc[j] + y;
            comp[j] = (s2 - acc[j]) - y;
            acc[j] = s2;
        }
    }
    const float inv2pi = 0.15915494309189533576888376337251f;
#pragma unroll
    for (int j = 0; j < 16; ++j)
        p_out[int64_t(LYA * 8 + j) * t.n + LX * 8 + tx] = (acc[j] - comp[j]) * inv2pi;
}

}  // namespace pp
