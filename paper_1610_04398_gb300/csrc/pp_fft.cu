// Pressure at every grid cell by the zero-padded FFT convolution of Hockney, the Fourier-based
// fast Poisson solver the paper names as an alternative to the tree-code (Appendix A.1).  It
// evaluates the same discrete sum as the multipole solve (Eq. greenSum, self term clamped at
// rho_h), without truncation: on an M x M periodic grid, M = 2n >= 2n - 1, the circular
// convolution of the zero-padded n x n weights q with the wrapped kernel table
//   K[y][x] = (1/2pi) log max(h |(dx, dy)|, rho_h),  dx = x or x - M, dy = y or y - M, |dx|, |dy| < n
// (zero elsewhere) equals the linear one on the first n x n cells, so
//   P = IDFT2( DFT2(q) * DFT2(K) )[0:n, 0:n].
//
// Three launches per solve, every line transform held whole in shared memory:
//   1. rows: two real rows packed as one complex line (a + i b), forward transform, the half
//      spectra of both rows untangled from Z(k) and Z(M - k) and stored, k in [0, M/2];
//   2. columns: each column k_x of the half spectrum (n values, zero padded to M) forward
//      transformed, multiplied by the real transformed kernel, inverse transformed, and its
//      first n values stored back in place;
//   3. rows: the Hermitian half spectra of two rows combined into one complex line, inverse
//      transformed, real and imaginary parts stored as the two pressure rows.
// The forward transforms are decimation in frequency (natural order in, bit-reversed out)
// and the inverse ones decimation in time (bit-reversed in, natural out), so no permutation
// pass is needed: the kernel spectrum is stored permuted to the bit-reversed order, and the
// row kernels read and place the half spectra through the bit reversal.  Each transform is
// a sequence of radix-16 steps (plus one radix-2/4/8 step when log2 M is not a multiple of
// 4): a thread loads the 16 elements of one group into registers, runs four radix-2 passes
// on them and stores them back.  Twiddles come from per-step tables (contiguous in the
// group offset, read through L1); shared-memory lines are padded by one element in 16 and
// one more in 256, which keeps the strided steps and the bit-reversed accesses free of bank
// conflicts.  The first forward step skips the zero
// upper half of its input, the last inverse step forms only the lower half it stores, and
// in the column kernel the last forward step, the product with the kernel spectrum and the
// first inverse step run on the same registers.
//
// The transformed kernel is formed once per plan in FP64 (a plain radix-2 transform of the
// wrapped table, scaled by 1/M^2 for the unnormalised inverse) and stored in the plan's
// precision as a (M/2 + 1) x M table in the bit-reversed order of the column transform,
// followed by the twiddle tables.
#include <cuda_runtime.h>

#include <cstdint>

#include "pp_common.h"

namespace pp {
namespace {

template <typename R> struct Cplx;
template <> struct Cplx<float> { typedef float2 type; };
template <> struct Cplx<double> { typedef double2 type; };

constexpr int kFftThreads = 256;
constexpr int kFftSmemLimit = 227 * 1024;  // dynamic shared memory of one CTA on sm_103a

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return C{a.x, -a.y}; }

// Shared-memory position of line element i: one pad slot after every 16 elements and one more
// after every 256.  Both the strided steps (stride S/R = M/16, M/256, ..., 1) and the
// bit-reversed reads and writes of the row kernels then hit each bank at most once more than
// the 8- or 16-byte accesses of a warp need.
__device__ __forceinline__ int fpad(int i) { return i + (i >> 4) + (i >> 8); }

__device__ __forceinline__ int brev_bits(int k, int m) { return int(__brev(unsigned(k)) >> (32 - m)); }

// exp(-2 pi i e / 16) for e in [0, 8): cos and -sin of multiples of pi/8.
template <typename C>
__device__ __forceinline__ C root16(int e) {
    typedef decltype(C::x) R;
    const R a = R(0.92387953251128675613), b = R(0.38268343236508977173), h = R(0.70710678118654752440);
    switch (e) {
        case 0: return C{R(1), R(0)};
        case 1: return C{a, -b};
        case 2: return C{h, -h};
        case 3: return C{b, -a};
        case 4: return C{R(0), R(-1)};
        case 5: return C{-b, -a};
        case 6: return C{-h, -h};
        default: return C{-a, -b};
    }
}

// d * exp(-+2 pi i e / 16) (conjugate root when INV); e = 0 and e = 4 (-+i) without a product.
template <bool INV, typename C>
__device__ __forceinline__ C mul_root(C d, int e) {
    if (e == 0) return d;
    if (e == 4) return INV ? C{-d.y, d.x} : C{d.y, -d.x};
    const C w = root16<C>(e);
    return cmul(d, INV ? cconj(w) : w);
}

// Schedule of a transform of M = 2^m points: DIF step sd (sd = 0 first) has block size
// S = M / 16^sd and radix 16, except the last step, of radix 2^(m mod 4) when m mod 4 != 0;
// SR = S / radix.  Its twiddle table (per plan, in step order) holds, at off + q SR + o,
// exp(-2 pi i o 2^q / S) for q < log2 radix and o < SR.  The inverse transform runs the
// same steps in the reverse order with conjugate twiddles.
struct FftStep {
    int logr, SR, off;
};
__host__ __device__ __forceinline__ int fft_nsteps(int m) { return (m + 3) >> 2; }
__host__ __device__ __forceinline__ FftStep fft_step_info(int M, int m, int sd) {
    const int ns = fft_nsteps(m), r0 = m & 3;
    FftStep st;
    st.logr = (sd == ns - 1 && r0) ? r0 : 4;
    st.SR = (M >> (4 * sd)) >> st.logr;
    st.off = 0;
    for (int k = 0; k < sd; ++k) st.off += 4 * ((M >> (4 * k)) >> 4);  // earlier steps are radix 16
    return st;
}

// Addressing of a group's elements o + j SR of block b: AD_UNIT (SR = 1: consecutive),
// AD_BIG (SR >= 256: the pads shift by SR/16 + SR/256 per element), AD_GEN (other SR).
enum { AD_UNIT = 0, AD_BIG = 1, AD_GEN = 2 };
// HALF_IN: a forward first step whose upper half (j >= R/2, the zero padding) is not read;
// HALF_OUT: an inverse last step whose upper half (never stored) is not formed or written.
enum { HALF_NONE = 0, HALF_IN = 1, HALF_OUT = 2 };

// One radix-2^LOGR step on group g of a line: the elements o + j SR of block b (g = b SR + o)
// undergo the LOGR radix-2 passes of block sizes S, S/2, ... (forward, decimation in
// frequency) or the same passes in the reverse order with conjugate twiddles (inverse,
// decimation in time).  The pass of block size S/2^q multiplies the difference of the pair
// (j, j + m), m = R/2^(q+1), by exp(-+2 pi i (o + (j mod m) SR) 2^q / S)
// = twq[q SR + o] * exp(-+2 pi i (j mod m) 2^q / R).
template <int LOGR, bool INV, int HALF, int AD, typename C>
__device__ __forceinline__ void fft_group(C* line, const C* __restrict__ twq, int SR, int g) {
    constexpr int RR = 1 << LOGR;
    const int o = AD == AD_UNIT ? 0 : (g & (SR - 1));
    const int base = AD == AD_UNIT ? g * RR : (g - o) * RR + o;
    const int p0 = fpad(base), ps = SR + (SR >> 4) + (SR >> 8);
    auto pos = [&](int j) { return AD == AD_UNIT ? p0 + j : AD == AD_BIG ? p0 + j * ps : fpad(base + j * SR); };
    C v[RR];
#pragma unroll
    for (int j = 0; j < RR; ++j)
        if (HALF != HALF_IN || j < RR / 2) v[j] = line[pos(j)];
    if (!INV) {
#pragma unroll
        for (int q = 0; q < LOGR; ++q) {
            const int mm = RR >> (q + 1);
            const C t = AD == AD_UNIT ? C{1, 0} : __ldg(twq + q * SR + o);
#pragma unroll
            for (int j = 0; j < RR; ++j) {
                if (j & mm) continue;
                const int e = ((j & (mm - 1)) << q) * (16 / RR);
                if (HALF == HALF_IN && q == 0) {  // partner is zero: (a, 0) -> (a, a W)
                    v[j + mm] = AD == AD_UNIT ? mul_root<false>(v[j], e) : cmul(v[j], mul_root<false>(t, e));
                    continue;
                }
                const C a = v[j], c = v[j + mm];
                v[j] = cadd(a, c);
                v[j + mm] = AD == AD_UNIT ? mul_root<false>(csub(a, c), e) : cmul(csub(a, c), mul_root<false>(t, e));
            }
        }
    } else {
#pragma unroll
        for (int q = LOGR - 1; q >= 0; --q) {
            const int mm = RR >> (q + 1);
            const C t = AD == AD_UNIT ? C{1, 0} : cconj(__ldg(twq + q * SR + o));
#pragma unroll
            for (int j = 0; j < RR; ++j) {
                if (j & mm) continue;
                const int e = ((j & (mm - 1)) << q) * (16 / RR);
                const C c = AD == AD_UNIT ? mul_root<true>(v[j + mm], e) : cmul(v[j + mm], mul_root<true>(t, e));
                const C a = v[j];
                v[j] = cadd(a, c);
                if (!(HALF == HALF_OUT && q == 0)) v[j + mm] = csub(a, c);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < RR; ++j)
        if (HALF != HALF_OUT || j < RR / 2) line[pos(j)] = v[j];
}

template <int LOGR, bool INV, int HALF, typename C>
__device__ __forceinline__ void fft_group_ad(C* line, const C* twq, int SR, int g) {
    if (SR == 1) {
        if constexpr (HALF == HALF_NONE) fft_group<LOGR, INV, HALF_NONE, AD_UNIT>(line, twq, SR, g);
    } else if (SR >= 256) {
        fft_group<LOGR, INV, HALF, AD_BIG>(line, twq, SR, g);
    } else {
        fft_group<LOGR, INV, HALF, AD_GEN>(line, twq, SR, g);
    }
}

// Step sd (DIF numbering) on NL lines of M = 2^m points (line stride ls), then a barrier.
template <bool INV, int HALF, int NL, typename C>
__device__ void fft_step(C* lines, int ls, const C* __restrict__ tab, int M, int m, int sd) {
    const FftStep st = fft_step_info(M, m, sd);
    const int gpl = M >> st.logr;  // groups per line
    const C* twq = tab + st.off;
    for (int gi = threadIdx.x; gi < NL * gpl; gi += blockDim.x) {
        C* line = lines + (gi >> (m - st.logr)) * ls;
        const int g = gi & (gpl - 1);
        switch (st.logr) {
            case 4: fft_group_ad<4, INV, HALF>(line, twq, st.SR, g); break;
            case 3: fft_group_ad<3, INV, HALF>(line, twq, st.SR, g); break;
            case 2: fft_group_ad<2, INV, HALF>(line, twq, st.SR, g); break;
            default: fft_group_ad<1, INV, HALF>(line, twq, st.SR, g); break;
        }
    }
    __syncthreads();
}

// Forward transform (all DIF steps) of NL lines; the first step skips the zero upper half
// when there is more than one step (lines hold data only below M/2).
template <int NL, typename C>
__device__ void fft_forward(C* lines, int ls, const C* tab, int M, int m) {
    const int ns = fft_nsteps(m);
    if (ns == 1) {
        fft_step<false, HALF_NONE, NL>(lines, ls, tab, M, m, 0);
        return;
    }
    fft_step<false, HALF_IN, NL>(lines, ls, tab, M, m, 0);
    for (int sd = 1; sd < ns; ++sd) fft_step<false, HALF_NONE, NL>(lines, ls, tab, M, m, sd);
}

// Inverse transform from step sd_first down to step 0; the last step forms only the lower
// half (the only part stored) when there is more than one step.
template <int NL, typename C>
__device__ void fft_inverse(C* lines, int ls, const C* tab, int M, int m, int sd_first) {
    const int ns = fft_nsteps(m);
    for (int sd = sd_first; sd >= 1; --sd) fft_step<true, HALF_NONE, NL>(lines, ls, tab, M, m, sd);
    if (sd_first >= 0) {
        if (ns == 1)
            fft_step<true, HALF_NONE, NL>(lines, ls, tab, M, m, 0);
        else
            fft_step<true, HALF_OUT, NL>(lines, ls, tab, M, m, 0);
    }
}

// Column middle: the last forward step (unit stride), the product with the kernel spectrum
// and the first inverse step on the same group, in registers.
template <int LOGR, typename C, typename R>
__device__ __forceinline__ void fft_middle_group(C* line, const R* __restrict__ kp, int g) {
    constexpr int RR = 1 << LOGR;
    const int base = g * RR, p0 = fpad(base);
    C v[RR];
#pragma unroll
    for (int j = 0; j < RR; ++j) v[j] = line[p0 + j];
#pragma unroll
    for (int q = 0; q < LOGR; ++q) {
        const int mm = RR >> (q + 1);
#pragma unroll
        for (int j = 0; j < RR; ++j) {
            if (j & mm) continue;
            const int e = ((j & (mm - 1)) << q) * (16 / RR);
            const C a = v[j], c = v[j + mm];
            v[j] = cadd(a, c);
            v[j + mm] = mul_root<false>(csub(a, c), e);
        }
    }
    if constexpr (RR == 16 && sizeof(R) == 4) {  // 64-byte aligned: four 16-byte loads
        const float4* k4 = reinterpret_cast<const float4*>(kp + base);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float4 k = __ldg(k4 + u);
            v[4 * u] = C{v[4 * u].x * k.x, v[4 * u].y * k.x};
            v[4 * u + 1] = C{v[4 * u + 1].x * k.y, v[4 * u + 1].y * k.y};
            v[4 * u + 2] = C{v[4 * u + 2].x * k.z, v[4 * u + 2].y * k.z};
            v[4 * u + 3] = C{v[4 * u + 3].x * k.w, v[4 * u + 3].y * k.w};
        }
    } else {
#pragma unroll
        for (int j = 0; j < RR; ++j) {
            const R k = __ldg(kp + base + j);
            v[j] = C{v[j].x * k, v[j].y * k};
        }
    }
#pragma unroll
    for (int q = LOGR - 1; q >= 0; --q) {
        const int mm = RR >> (q + 1);
#pragma unroll
        for (int j = 0; j < RR; ++j) {
            if (j & mm) continue;
            const int e = ((j & (mm - 1)) << q) * (16 / RR);
            const C c = mul_root<true>(v[j + mm], e), a = v[j];
            v[j] = cadd(a, c);
            v[j + mm] = csub(a, c);
        }
    }
#pragma unroll
    for (int j = 0; j < RR; ++j) line[p0 + j] = v[j];
}

template <typename C>
struct CPair {
    C a, b;
};

// for i in [0, total): store(i, load(i)), U loads in flight per thread before their stores.
template <int U, typename Load, typename Store>
__device__ __forceinline__ void batched_copy(int total, Load load, Store store) {
    for (int i0 = threadIdx.x; i0 < total; i0 += blockDim.x * U) {
        decltype(load(0)) r[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * int(blockDim.x);
            if (i < total) r[u] = load(i);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * int(blockDim.x);
            if (i < total) store(i, r[u]);
        }
    }
}

// Launch 1.  CTA b transforms rows 2 NL b .. 2 NL b + 2 NL - 1 of q (leaf-major: cell (x, y)
// at ((y/8) nL + x/8) 64 + (y mod 8) 8 + x mod 8) and writes their half spectra, k in
// [0, M/2], to rows of H (row stride W; columns M/2 + 1 .. W - 1 are set to zero).
template <typename R, int NL>
__global__ void __launch_bounds__(kFftThreads, sizeof(R) == 4 ? 3 : 1)
    k_fft_rows_fwd(const R* __restrict__ q, int n, int nL, int M, int m, int W, int ls,
                   const typename Cplx<R>::type* __restrict__ tab, typename Cplx<R>::type* __restrict__ H) {
    typedef typename Cplx<R>::type C;
    extern __shared__ __align__(16) unsigned char fft_smem[];
    C* lines = reinterpret_cast<C*>(fft_smem);
    const int y0 = blockIdx.x * (2 * NL);
    const int ln = __ffs(n) - 1;
    if (fft_nsteps(m) == 1)  // the single step reads the zero padding x in [n, M)
        for (int i = threadIdx.x; i < NL * n; i += blockDim.x) lines[(i >> ln) * ls + fpad(n + (i & (n - 1)))] = C{0, 0};
    batched_copy<8>(
        NL * n,
        [&](int i) {
            const int x = i & (n - 1), y = y0 + 2 * (i >> ln);  // y even: row y + 1 is in the same leaf
            const int64_t a = (int64_t(y >> 3) * nL + (x >> 3)) * 64 + (y & 7) * 8 + (x & 7);
            return C{q[a], q[a + 8]};
        },
        [&](int i, C v) { lines[(i >> ln) * ls + fpad(i & (n - 1))] = v; });
    __syncthreads();
    fft_forward<NL>(lines, ls, tab, M, m);
    const int half = M >> 1;
    for (int i = threadIdx.x; i < NL * W; i += blockDim.x) {
        const int l = i / W, k = i - l * W;
        const C* x = lines + l * ls;
        C A = {R(0), R(0)}, B = {R(0), R(0)};
        if (k <= half) {
            // a_k = (Z_k + conj Z_{M-k}) / 2, b_k = (Z_k - conj Z_{M-k}) / 2i
            const C zk = x[fpad(brev_bits(k, m))];
            const C zm = x[fpad(brev_bits((M - k) & (M - 1), m))];
            A = C{R(0.5) * (zk.x + zm.x), R(0.5) * (zk.y - zm.y)};
            B = C{R(0.5) * (zk.y + zm.y), R(0.5) * (zm.x - zk.x)};
        }
        C* h0 = H + int64_t(y0 + 2 * l) * W + k;
        h0[0] = A;
        h0[W] = B;
    }
}

// Launch 2.  CTA b takes columns k_x = NL b .. NL b + NL - 1 of H (those <= M/2): forward
// transform along y of the n values zero-padded to M, product with the kernel spectrum
// Kp[k_x][p] (already in the bit-reversed order and scaled by 1/M^2), inverse transform,
// first n values back to H.
template <typename R, int NL>
__global__ void __launch_bounds__(kFftThreads, sizeof(R) == 4 ? 3 : 1)
    k_fft_cols(typename Cplx<R>::type* __restrict__ H, const R* __restrict__ Kp, int n, int M, int m, int W, int ls,
               const typename Cplx<R>::type* __restrict__ tab) {
    typedef typename Cplx<R>::type C;
    extern __shared__ __align__(16) unsigned char fft_smem[];
    C* lines = reinterpret_cast<C*>(fft_smem);
    const int kx0 = blockIdx.x * NL, half = M >> 1;
    const int ns = fft_nsteps(m);
    if (ns == 1)  // the single step reads the zero padding y in [n, M)
        for (int i = threadIdx.x; i < NL * n; i += blockDim.x) lines[(i % NL) * ls + fpad(n + i / NL)] = C{0, 0};
    batched_copy<8>(
        NL * n, [&](int i) { return H[int64_t(i / NL) * W + kx0 + i % NL]; },
        [&](int i, C v) { lines[(i % NL) * ls + fpad(i / NL)] = v; });
    __syncthreads();
    // forward steps but the last (the first one skips the zero half)
    if (ns > 1) {
        fft_step<false, HALF_IN, NL>(lines, ls, tab, M, m, 0);
        for (int sd = 1; sd < ns - 1; ++sd) fft_step<false, HALF_NONE, NL>(lines, ls, tab, M, m, sd);
    }
    // last forward step, product, first inverse step
    {
        const FftStep st = fft_step_info(M, m, ns - 1);
        const int gpl = M >> st.logr;
        for (int gi = threadIdx.x; gi < NL * gpl; gi += blockDim.x) {
            const int l = gi >> (m - st.logr), g = gi & (gpl - 1);
            const int kx = min(kx0 + l, half);  // columns past M/2 are padding: any finite values
            C* line = lines + l * ls;
            const R* kp = Kp + int64_t(kx) * M;
            switch (st.logr) {
                case 4: fft_middle_group<4>(line, kp, g); break;
                case 3: fft_middle_group<3>(line, kp, g); break;
                case 2: fft_middle_group<2>(line, kp, g); break;
                default: fft_middle_group<1>(line, kp, g); break;
            }
        }
        __syncthreads();
    }
    fft_inverse<NL>(lines, ls, tab, M, m, ns - 2);
    if (ns == 1) {
        // nothing left: the middle was the whole transform
    }
    for (int i = threadIdx.x; i < NL * n; i += blockDim.x) {
        const int y = i / NL, l = i - y * NL;
        if (kx0 + l <= half) H[int64_t(y) * W + kx0 + l] = lines[l * ls + fpad(y)];
    }
}

// Launch 3.  CTA b combines the half spectra A, B of rows 2 NL b + 2l and + 2l + 1 into
// Z_k = A_k + i B_k (Z_{M-k} = conj A_k + i conj B_k), inverse transforms and writes the real
// and imaginary parts, x < n, as the two pressure rows (row-major n x n).
template <typename R, int NL>
__global__ void __launch_bounds__(kFftThreads, sizeof(R) == 4 ? 3 : 1)
    k_fft_rows_inv(const typename Cplx<R>::type* __restrict__ H, int n, int M, int m, int W, int ls,
                   const typename Cplx<R>::type* __restrict__ tab, R* __restrict__ p_out) {
    typedef typename Cplx<R>::type C;
    extern __shared__ __align__(16) unsigned char fft_smem[];
    C* lines = reinterpret_cast<C*>(fft_smem);
    const int y0 = blockIdx.x * (2 * NL), half = M >> 1;
    const int nk = half + 1;
    batched_copy<4>(
        NL * nk,
        [&](int i) {
            const int l = i / nk, k = i - l * nk;
            const C* h0 = H + int64_t(y0 + 2 * l) * W + k;
            return CPair<C>{h0[0], h0[W]};
        },
        [&](int i, CPair<C> ab) {
            const int l = i / nk, k = i - l * nk;
            C* x = lines + l * ls;
            const C A = ab.a, B = ab.b;
            x[fpad(brev_bits(k, m))] = C{A.x - B.y, A.y + B.x};
            if (k > 0 && k < half) x[fpad(brev_bits(M - k, m))] = C{A.x + B.y, B.x - A.y};
        });
    __syncthreads();
    fft_inverse<NL>(lines, ls, tab, M, m, fft_nsteps(m) - 1);
    for (int i = threadIdx.x; i < NL * n; i += blockDim.x) {
        const int l = i / n, x = i - l * n;
        const C v = lines[l * ls + fpad(x)];
        p_out[int64_t(y0 + 2 * l) * n + x] = v.x;
        p_out[int64_t(y0 + 2 * l + 1) * n + x] = v.y;
    }
}

// Per-step twiddle tables (layout of fft_step_info), in FP64 then rounded.
template <typename R>
__global__ void k_fft_twiddles(int M, int m, typename Cplx<R>::type* __restrict__ tab) {
    typedef typename Cplx<R>::type C;
    for (int sd = 0; sd < fft_nsteps(m); ++sd) {
        const FftStep st = fft_step_info(M, m, sd);
        const int S = M >> (4 * sd);
        for (int i = threadIdx.x; i < st.logr * st.SR; i += blockDim.x) {
            const int qq = i / st.SR, o = i - qq * st.SR;
            double sn, cs;
            sincospi(2.0 * double(o << qq) / double(S), &sn, &cs);
            tab[st.off + i] = C{R(cs), R(-sn)};
        }
    }
}

// ---------------------------------------------------------------- kernel spectrum (FP64, once)

// One CTA per row of M points, natural order in and out: bit-reversed load, then radix-2
// decimation-in-time passes with twiddles exp(-2 pi i k / 2hs) from sincospi.
__global__ void __launch_bounds__(512) k_spec_rows(double2* __restrict__ data, int M, int m) {
    extern __shared__ __align__(16) unsigned char fft_smem[];
    double2* x = reinterpret_cast<double2*>(fft_smem);
    double2* row = data + int64_t(blockIdx.x) * M;
    for (int j = threadIdx.x; j < M; j += blockDim.x) x[brev_bits(j, m)] = row[j];
    __syncthreads();
    for (int hs = 1; hs < M; hs <<= 1) {
        for (int b = threadIdx.x; b < (M >> 1); b += blockDim.x) {
            const int k = b & (hs - 1), i = ((b - k) << 1) + k, j = i + hs;
            double s, c;
            sincospi(-double(k) / double(hs), &s, &c);
            const double2 a = x[i], w = cmul(x[j], double2{c, s});
            x[i] = cadd(a, w);
            x[j] = csub(a, w);
        }
        __syncthreads();
    }
    for (int j = threadIdx.x; j < M; j += blockDim.x) row[j] = x[j];
}

__global__ void __launch_bounds__(256) k_spec_transpose(const double2* __restrict__ in, double2* __restrict__ out,
                                                        int M) {
    __shared__ double2 tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += 8)
        if (by + r < M && bx + int(threadIdx.x) < M) tile[r][threadIdx.x] = in[int64_t(by + r) * M + bx + threadIdx.x];
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8)
        if (bx + r < M && by + int(threadIdx.x) < M) out[int64_t(bx + r) * M + by + threadIdx.x] = tile[threadIdx.x][r];
}

// The wrapped kernel table K[y][x] as complex values (zero imaginary part).
__global__ void k_spec_table(int n, int M, double h, double rh, double2* __restrict__ out) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= int64_t(M) * M) return;
    const int x = int(i % M), y = int(i / M);
    const int dx = x < n ? x : x - M, dy = y < n ? y : y - M;
    double val = 0.0;
    if (dx > -n && dx < n && dy > -n && dy < n) {
        const double r = h * sqrt(double(dx) * dx + double(dy) * dy);
        val = log(r > rh ? r : rh) * 0.15915494309189533576888376337251;
    }
    out[i] = double2{val, 0.0};
}

// Kp[k_x][p] = Re DFT2(K)[k_y = rev(p)][k_x] / M^2 for k_x in [0, M/2] (the spectrum of the
// real table that is even in x and y is real).
template <typename R>
__global__ void k_spec_store(const double2* __restrict__ spec, int M, int m, double scale, R* __restrict__ Kp) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= int64_t((M >> 1) + 1) * M) return;
    const int kx = int(i >> m), p = int(i & (M - 1));
    Kp[i] = R(spec[int64_t(brev_bits(p, m)) * M + kx].x * scale);
}

int log2i(int M) {
    int l = 0;
    while ((1 << l) < M) ++l;
    return l;
}

// Line stride in shared memory: padded length plus an 8-element stagger, so that the two
// lines a CTA interleaves in its column loads and stores fall in different bank halves.
int line_stride(int M) { return M + M / 16 + M / 256 + 8; }

// Lines per CTA (three CTAs per SM either way in FP32): two up to M = 2048, one above, where
// the finer grain balances the waves better (2n = 4096: 0.116 against 0.122 ms a solve).
template <typename R>
int lines_per_cta(int M) {
    return sizeof(R) == 4 && M <= 2048 ? 2 : 1;
}

template <typename R>
size_t fft_smem(int M) {
    return size_t(lines_per_cta<R>(M)) * size_t(line_stride(M)) * sizeof(typename Cplx<R>::type);
}

int twiddle_entries(int M, int m) {
    int t = 0;
    for (int sd = 0; sd < fft_nsteps(m); ++sd) {
        const FftStep st = fft_step_info(M, m, sd);
        t += st.logr * st.SR;
    }
    return t;
}

// The spectrum buffer: Kp ((M/2 + 1) x M reals), then the twiddle tables at a 256-byte offset.
size_t kp_bytes(int M, size_t rsize) { return ((size_t(M / 2 + 1) * size_t(M) * rsize + 255) / 256) * 256; }

template <typename R, int NL>
cudaError_t set_smem_attrs() {
    const int lim = kFftSmemLimit;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_fft_rows_fwd<R, NL>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) ||
        (e = cudaFuncSetAttribute(k_fft_cols<R, NL>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) ||
        (e = cudaFuncSetAttribute(k_fft_rows_inv<R, NL>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)))
        return e;
    return cudaSuccess;
}

}  // namespace

bool fft_size_ok(int n, bool fp64) {
    if (n < 8 || n > 4096 || (n & (n - 1))) return false;
    const int M = 2 * n;
    return (fp64 ? fft_smem<double>(M) : fft_smem<float>(M)) <= size_t(kFftSmemLimit) &&
           size_t(M) * 16 <= size_t(kFftSmemLimit);  // one FP64 line of the spectrum transform
}

size_t fft_work_bytes(int n, bool fp64) { return size_t(n) * size_t(n + 4) * (fp64 ? 16 : 8); }

size_t fft_spectrum_bytes(int n, bool fp64) {
    const int M = 2 * n;
    return kp_bytes(M, fp64 ? 8 : 4) + size_t(twiddle_entries(M, log2i(M))) * (fp64 ? 16 : 8);
}

int fft_launches_per_solve() { return 3; }

// Forms the spectrum buffer (fft_spectrum_bytes: Kp and the twiddle tables) on stream st;
// allocates two M x M FP64 complex scratch arrays, synchronises st and frees them.
cudaError_t fft_prepare_spectrum(int n, double h, double rh, bool fp64, void* Kp, cudaStream_t st) {
    cudaError_t e;
    if ((e = fp64 ? set_smem_attrs<double, 1>() : set_smem_attrs<float, 1>())) return e;
    if (!fp64 && (e = set_smem_attrs<float, 2>())) return e;
    const int M = 2 * n, m = log2i(M);
    if ((e = cudaFuncSetAttribute(k_spec_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, kFftSmemLimit)))
        return e;
    const size_t bytes = size_t(M) * M * sizeof(double2);
    double2 *a = nullptr, *t = nullptr;
    if ((e = cudaMalloc(&a, bytes)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&t, bytes)) != cudaSuccess) {
        cudaFree(a);
        return e;
    }
    const int64_t tot = int64_t(M) * M;
    k_spec_table<<<unsigned((tot + 255) / 256), 256, 0, st>>>(n, M, h, rh, a);
    const dim3 tg((M + 31) / 32, (M + 31) / 32), tb(32, 8);
    const size_t sm = size_t(M) * sizeof(double2);
    k_spec_rows<<<M, 512, sm, st>>>(a, M, m);  // along x: a[y][k_x]
    k_spec_transpose<<<tg, tb, 0, st>>>(a, t, M);
    k_spec_rows<<<M, 512, sm, st>>>(t, M, m);  // along y: t[k_x][k_y]
    k_spec_transpose<<<tg, tb, 0, st>>>(t, a, M);  // a[k_y][k_x]
    const int64_t nk = int64_t(M / 2 + 1) * M;
    const double scale = 1.0 / (double(M) * double(M));
    unsigned char* base = static_cast<unsigned char*>(Kp);
    if (fp64) {
        k_spec_store<double><<<unsigned((nk + 255) / 256), 256, 0, st>>>(a, M, m, scale, static_cast<double*>(Kp));
        k_fft_twiddles<double><<<1, 256, 0, st>>>(M, m, reinterpret_cast<double2*>(base + kp_bytes(M, 8)));
    } else {
        k_spec_store<float><<<unsigned((nk + 255) / 256), 256, 0, st>>>(a, M, m, scale, static_cast<float*>(Kp));
        k_fft_twiddles<float><<<1, 256, 0, st>>>(M, m, reinterpret_cast<float2*>(base + kp_bytes(M, 4)));
    }
    e = cudaGetLastError();
    const cudaError_t es = cudaStreamSynchronize(st);
    cudaFree(a);
    cudaFree(t);
    return e != cudaSuccess ? e : es;
}

// One solve: q (leaf-major weights f h^2) -> p_out (row-major n x n).  H: fft_work_bytes;
// Kp: the spectrum buffer fft_prepare_spectrum formed.
template <typename R, int NL>
cudaError_t launch_fft_lines(const R* q, int n, int nL, const void* Kp, void* H, R* p_out, cudaStream_t st) {
    typedef typename Cplx<R>::type C;
    const int M = 2 * n, m = log2i(M), W = n + 4, ls = line_stride(M);
    const size_t sm = fft_smem<R>(M);
    const R* K = static_cast<const R*>(Kp);
    const C* tab = reinterpret_cast<const C*>(static_cast<const unsigned char*>(Kp) + kp_bytes(M, sizeof(R)));
    C* Hc = static_cast<C*>(H);
    k_fft_rows_fwd<R, NL><<<n / (2 * NL), kFftThreads, sm, st>>>(q, n, nL, M, m, W, ls, tab, Hc);
    k_fft_cols<R, NL><<<(M / 2 + NL) / NL, kFftThreads, sm, st>>>(Hc, K, n, M, m, W, ls, tab);
    k_fft_rows_inv<R, NL><<<n / (2 * NL), kFftThreads, sm, st>>>(Hc, n, M, m, W, ls, tab, p_out);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_fft_solve(const R* q, int n, int nL, const void* Kp, void* H, R* p_out, cudaStream_t st) {
    if constexpr (sizeof(R) == 4) {
        if (lines_per_cta<R>(2 * n) == 2) return launch_fft_lines<R, 2>(q, n, nL, Kp, H, p_out, st);
    }
    return launch_fft_lines<R, 1>(q, n, nL, Kp, H, p_out, st);
}

template cudaError_t launch_fft_solve<float>(const float*, int, int, const void*, void*, float*, cudaStream_t);
template cudaError_t launch_fft_solve<double>(const double*, int, int, const void*, void*, double*, cudaStream_t);

}  // namespace pp
