// Multipole-to-local translations on the 5th-generation tensor cores (tcgen05, kind::tf32,
// FP32 accumulate), mixed precision: the tensor-core form of k_m2l_far.
//
// The factored operator of App. A.2's translation (scaled coefficients), for one entry e of a
// target box's interaction list with offset tau and source multipole M:
//   x_k = tau^-k M_k (k = 1..p),  y_l = sum_k R[l][k] x_k + R[l][0] S,  L_l += tau^-l y_l,
// R real, the same for every offset and level.  The product y = R x is the bulk of the work
// (2 p^2 of ~3.5 p^2 flops) and is a dense contraction once 128 target boxes are stacked: for
// entry slot e, row m of A holds box m's x (real parts, then imaginary parts: K = 2p), and
//   D = A B,  B[k-1][l] = R[l][k] (l = 0..p, real inputs), B[p+k-1][p+l] = R[l][k] (l = 1..p,
// imaginary inputs), so that row m of D is y_re[0..p], y_im[1..p] (N = 2p + 1, padded to 16).
// The monopole column R[l][0] S and both diagonals stay with the threads: each thread owns
// one target box (one TMEM lane), forms its x, and folds D's row into its local.
//
// Precision: FP32 accuracy from TF32 by splitting both operands, v = v_hi + v_lo with v_hi
// the value with its 13 low mantissa bits cleared (TF32 keeps 10) and v_lo = v - v_hi:
//   A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi,
// nine MMAs of K = 8 per entry slot at p = 12 into a fresh accumulator.  B holds integers
// below 2^21 (binomials), which the split represents exactly.  The constant-term parts
// (sum S log|tau|, sum S) are double-float sums on the FP32 pipe, as in k_m2l_far.
//
// Pipeline per CTA (128 boxes of one level): warps 0-3 form entry e's A rows in shared
// stage e & 1 while the MMAs of entries e - 1 and e - 2 run, then drain e - 2's accumulator
// (TMEM buffer (e - 2) & 3); warp 4's elected thread issues the MMAs.  mbarriers: a_full (the four row
// warps wrote a stage), a_empty (the MMAs that read a stage completed), acc_full (an
// accumulator is ready), acc_empty (the four row warps drained it).  Every wait is bounded;
// a wait that gives up sets the error flag and the CTA winds down.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "pp_common.h"
#include "pp_tcgen05.cuh"

namespace pp {
namespace {

using namespace tc;

constexpr int kAccBufs = 4;  // TMEM accumulators: an entry's is drained two entries after its MMAs

template <int P1>
struct M2lTc {
    static constexpr int p = P1 - 1;
    static constexpr int K = 2 * p;                              // x_re[1..p], x_im[1..p]
    static constexpr int N = ((2 * P1 - 1) + 15) / 16 * 16;     // y_re[0..p], y_im[1..p], padded
    static constexpr uint32_t kLboA = 16u * 128u;                // 16 row groups of 8 rows x 16 B
    static constexpr uint32_t kLboB = uint32_t(N / 8) * 128u;
    static constexpr uint32_t a_bytes = 128u * K * 4u;           // one split of one stage
    static constexpr uint32_t b_bytes = uint32_t(N) * K * 4u;    // one split of B
    static constexpr uint32_t smem = 128 + 4 * a_bytes + 2 * b_bytes;
    static constexpr uint32_t tmem_cols = kAccBufs * N <= 32 ? 32u : kAccBufs * N <= 64 ? 64u : kAccBufs * N <= 128 ? 128u : 256u;
    static_assert(K % 8 == 0, "K steps of 8");
};

constexpr int kM2lThreads = 160;  // 4 row warps + the MMA warp

// byte offset of element (row m, k-element j) in a K-major no-swizzle tile whose 8-row
// core matrices are 128 B: [k chunk of 4][row group][row in group][4 elements]
__host__ __device__ constexpr uint32_t kmaj_off(int m, int j, int groups) {
    return (uint32_t(j >> 2) * uint32_t(groups) + uint32_t(m >> 3)) * 128u + uint32_t(m & 7) * 16u + uint32_t(j & 3) * 4u;
}

__device__ __forceinline__ float tf32_hi(float v) { return __uint_as_float(__float_as_uint(v) & 0xFFFFE000u); }

template <int P1>
__global__ void __launch_bounds__(kM2lThreads, P1 <= 13 ? 3 : 2)
    k_m2l_tc(Tree<float> t, int lr, double lnRoot, int n_ops, const float* __restrict__ bmat, int* __restrict__ err) {
    typedef M2lTc<P1> G;
    constexpr int p = G::p;
    extern __shared__ uint8_t smem_dyn[];
    __shared__ __align__(8) uint64_t b_full, a_full[2], a_empty[2], acc_full[kAccBufs], acc_empty[kAccBufs];
    __shared__ uint32_t tmem_base;
    uint8_t* sbase = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_dyn) + 127) & ~uintptr_t(127));
    // stage s: A_hi at sbase + 2 s a_bytes, A_lo right after it
    auto a_hi = [&](int s) { return sbase + uint32_t(2 * s) * G::a_bytes; };
    auto a_lo = [&](int s) { return sbase + uint32_t(2 * s + 1) * G::a_bytes; };
    uint8_t* b_hi = sbase + 4 * G::a_bytes;
    uint8_t* b_lo = b_hi + G::b_bytes;
    // shared copies of the four interaction lists and of the per-operator tables (the
    // diagonals tau^-k of both sides and log|tau|), read once per CTA instead of per entry
    float2* s_tp = reinterpret_cast<float2*>(b_lo + G::b_bytes);    // [n_ops][P1]
    float2* s_tl = s_tp + size_t(n_ops) * P1;                        // [n_ops][P1]
    float2* s_lt = s_tl + size_t(n_ops) * P1;                        // [n_ops]
    M2LEntry* s_il = reinterpret_cast<M2LEntry*>(s_lt + n_ops);      // [4][il_stride]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // this CTA's level and first box: tiles of 128 boxes, levels finest first
    int l = t.Lleaf;
    int64_t tile = blockIdx.x;
    while (l >= 2) {
        const int64_t nt = ((int64_t(1) << (2 * l)) + 127) / 128;
        if (tile < nt) break;
        tile -= nt;
        --l;
    }
    if (l < 2) return;  // past the last tile (uniform over the CTA)
    const int side = 1 << l;
    const int64_t nb = int64_t(side) * side;
    const int E = t.il_stride;

    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sptr(&tmem_base)),
                     "r"(G::tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        if (lane == 0) {
            mbar_init(&b_full, 1);
            for (int s = 0; s < 2; ++s) {
                mbar_init(&a_full[s], 4);   // one arrival per row warp
                mbar_init(&a_empty[s], 1);  // MMA commit
            }
            for (int s = 0; s < kAccBufs; ++s) {
                mbar_init(&acc_full[s], 1);   // MMA commit
                mbar_init(&acc_empty[s], 4);  // one arrival per row warp
            }
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
    }
    for (int i = threadIdx.x; i < n_ops * P1; i += kM2lThreads) {
        s_tp[i] = t.Tpow[i];
        s_tl[i] = t.TpowL[i];
    }
    for (int i = threadIdx.x; i < n_ops; i += kM2lThreads) s_lt[i] = t.lnTauF[i];
    for (int i = threadIdx.x; i < 4 * E; i += kM2lThreads) s_il[i] = t.il[i];
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 4) {
        if (lane == 0) {
            // B (hi and lo, already in the K-major core-matrix layout) by one bulk copy
            mbar_expect_tx(&b_full, 2 * G::b_bytes);
            bulk_load(b_hi, bmat, 2 * G::b_bytes, &b_full);
            constexpr uint32_t idesc = idesc_tf32(G::N);
            int done = 0;
            bool ok = mbar_wait(&b_full, 0);
            if (!ok) atomicExch(err, 11);
            for (int e = 0; ok && e < E; ++e) {
                const int s = e & 1, ab = e & (kAccBufs - 1);
                if (!mbar_wait(&a_full[s], (e >> 1) & 1) ||
                    (e >= kAccBufs && !mbar_wait(&acc_empty[ab], ((e / kAccBufs) - 1) & 1))) {
                    atomicExch(err, 12);
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + uint32_t(ab) * G::N;
#pragma unroll
                for (int ks = 0; ks < G::K / 8; ++ks) {
                    const uint64_t ah = desc_noswz(sptr(a_hi(s)) + 2 * ks * G::kLboA, G::kLboA, 128);
                    const uint64_t al = desc_noswz(sptr(a_lo(s)) + 2 * ks * G::kLboA, G::kLboA, 128);
                    const uint64_t bh = desc_noswz(sptr(b_hi) + 2 * ks * G::kLboB, G::kLboB, 128);
                    const uint64_t bl = desc_noswz(sptr(b_lo) + 2 * ks * G::kLboB, G::kLboB, 128);
                    umma_tf32(d, ah, bh, idesc, ks != 0);
                    umma_tf32(d, ah, bl, idesc, 1);
                    umma_tf32(d, al, bh, idesc, 1);
                }
                umma_commit(&a_empty[s]);    // the stage may be rewritten once these MMAs are done
                umma_commit(&acc_full[ab]);  // and the accumulator is ready
                done = e + 1;
            }
            // TMEM is freed below only after every MMA issued here has completed
            if (done > 0 && !mbar_wait(&acc_full[(done - 1) & (kAccBufs - 1)], ((done - 1) / kAccBufs) & 1))
                atomicExch(err, 13);
        }
    } else {
        // row warps: thread m owns box tile * 128 + m (TMEM lane m)
        const int m = warp * 32 + lane;
        const int64_t b = tile * 128 + m;
        const bool act = b < nb;
        const int bx = act ? int(b % side) : 0, by = act ? int(b / side) : 0;
        const int par = (bx & 1) + 2 * (by & 1);
        const int cnt = act ? t.il_count[par] : 0;
        const M2LEntry* lst = s_il + par * E;
        const int64_t off = level_offset(l);
        float Lr[P1], Li[P1];
#pragma unroll
        for (int i = 0; i < P1; ++i) {
            Lr[i] = 0.f;
            Li[i] = 0.f;
        }
        float ah = 0.f, al = 0.f, sh = 0.f, sl = 0.f;  // double-float sum S log|tau|, sum S
        const uint32_t lane_base = uint32_t(warp * 32) << 16;
        bool good = true;
        int hist_op[2] = {-1, -1};      // operators of entries e - 2 and e - 1 (-1: none), drained two late
        float hist_S[2] = {0.f, 0.f};   // their source monopoles (hi parts), for the R[l][0] column

        // source box and operator of entry e (src < 0: none)
        auto entry = [&](int e, int& op) -> int64_t {
            op = -1;
            if (e >= cnt) return -1;
            const M2LEntry en = lst[e];
            if (en.pad == 0) {
                const int sx = bx + en.dx, sy = by + en.dy;
                if (sx < 0 || sy < 0 || sx >= side || sy >= side) return -1;
                op = en.op;
                return off + int64_t(sy) * side + sx;
            }
            const int hs = side >> 1;
            const int sx = (bx >> 1) + en.dx, sy = (by >> 1) + en.dy;
            if (sx < 0 || sy < 0 || sx >= hs || sy >= hs) return -1;
            op = en.op;
            return level_offset(l - 1) + int64_t(sy) * hs + sx;
        };
        // the multipole (k = 1..p) and the monopole pair of the next entry, loaded one entry ahead
        float2 mk[p];
        float2 Sd = make_float2(0.f, 0.f);
        auto fetch = [&](int64_t src) {
            if (src >= 0) {
                const float2* M = t.mp + src * P1;
#pragma unroll
                for (int k = 0; k < p; ++k) mk[k] = M[k + 1];
                Sd = t.Sf[src];
            }
        };

        auto drain = [&](int i, int dop, float dS) {  // entry i's accumulator into the local
            const int s = i & (kAccBufs - 1);
            bool got = mbar_wait(&acc_full[s], (i / kAccBufs) & 1);
            got = __all_sync(0xffffffffu, got);
            if (!got) {
                if (lane == 0) atomicExch(err, 14);
                return false;
            }
            tc_fence_after();
            float y[G::N];
#pragma unroll
            for (int c = 0; c < G::N / 16; ++c) tmem_ld16(tmem + lane_base + uint32_t(s) * G::N + 16 * c, y + 16 * c);
            tmem_wait_ld();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sptr(&acc_empty[s])) : "memory");
            if (dop >= 0) {
                const float2* tl = s_tl + dop * P1;
                Lr[0] += y[0];
#pragma unroll
                for (int ll = 1; ll < P1; ++ll) {
                    const float yr = fmaf(-1.f / float(ll), dS, y[ll]);  // R[l][0] = -1/l
                    const float yi = y[p + ll];
                    const float2 w = tl[ll];
                    Lr[ll] = fmaf(yr, w.x, fmaf(-yi, w.y, Lr[ll]));
                    Li[ll] = fmaf(yr, w.y, fmaf(yi, w.x, Li[ll]));
                }
            }
            return true;
        };

        int op_cur;
        fetch(entry(0, op_cur));
        for (int e = 0; e < E && good; ++e) {
            const int s = e & 1;
            bool free_ok = e < 2 || mbar_wait(&a_empty[s], ((e >> 1) - 1) & 1);
            free_ok = __all_sync(0xffffffffu, free_ok);
            if (!free_ok) {
                if (lane == 0) atomicExch(err, 15);
                good = false;
                break;
            }
            // entry e of this box: x (or zeros), written split into stage s
            float xr[p], xi[p];
            const int op = op_cur;
            const float Sh = op >= 0 ? Sd.x : 0.f;
            if (op >= 0) {
                const float2* tp = s_tp + op * P1;
                const float2 lt = s_lt[op];
                df_fma(ah, al, Sd.x, Sd.y, lt.x, lt.y);
                df_add(sh, sl, Sd.x, Sd.y);
#pragma unroll
                for (int k = 1; k < P1; ++k) {
                    const float2 w = tp[k];
                    xr[k - 1] = mk[k - 1].x * w.x - mk[k - 1].y * w.y;
                    xi[k - 1] = mk[k - 1].x * w.y + mk[k - 1].y * w.x;
                }
            } else {
#pragma unroll
                for (int k = 0; k < p; ++k) {
                    xr[k] = 0.f;
                    xi[k] = 0.f;
                }
            }
#pragma unroll
            for (int c = 0; c < G::K / 4; ++c) {
                float v[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int j = 4 * c + i;
                    v[i] = j < p ? xr[j] : xi[j - p];
                }
                const float4 hi = make_float4(tf32_hi(v[0]), tf32_hi(v[1]), tf32_hi(v[2]), tf32_hi(v[3]));
                const float4 lo = make_float4(v[0] - hi.x, v[1] - hi.y, v[2] - hi.z, v[3] - hi.w);
                const uint32_t at = kmaj_off(m, 4 * c, 16);
                *reinterpret_cast<float4*>(a_hi(s) + at) = hi;
                *reinterpret_cast<float4*>(a_lo(s) + at) = lo;
            }
            // the rows are read by the tensor cores (async proxy)
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sptr(&a_full[s])) : "memory");
            // the next entry's loads go out before the drain
            if (e + 1 < E) fetch(entry(e + 1, op_cur));
            if (e >= 2 && !drain(e - 2, hist_op[0], hist_S[0])) {
                good = false;
                break;
            }
            hist_op[0] = hist_op[1];
            hist_S[0] = hist_S[1];
            hist_op[1] = op;
            hist_S[1] = Sh;
        }
        if (good && E >= 2) good = drain(E - 2, hist_op[0], hist_S[0]);
        if (good && E >= 1) good = drain(E - 1, hist_op[1], hist_S[1]);
        if (good && act) {
            const int64_t i = off + b;
            const double lnS = fma(double(-l), 0.69314718055994530941723212145818, lnRoot);  // log(side / 2^l)
            const double L0 = df_to(ah, al) + lnS * df_to(sh, sl) + double(Lr[0]);
            float2* out = (l < lr ? t.locA : t.loc) + i * P1;
            (l < lr ? t.L0A : t.L0)[i] = L0;
            out[0] = make_float2(float(L0), 0.f);
#pragma unroll
            for (int ll = 1; ll < P1; ++ll) out[ll] = make_float2(Lr[ll], Li[ll]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 4)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G::tmem_cols) : "memory");
}

template <int P1>
void fill_bmat(float* out) {
    typedef M2lTc<P1> G;
    constexpr int p = G::p;
    std::vector<float> B(size_t(G::K) * G::N, 0.f);  // [j][n]
    auto R = [](int l, int k) {                      // R[l][k], k >= 1
        double c = 1.0;
        for (int i = 1; i <= k - 1; ++i) c = c * double(l + i) / double(i);  // C(l + k - 1, k - 1)
        return ((k + 1) % 2 == 0 ? 1.0 : -1.0) * c;
    };
    for (int k = 1; k <= p; ++k) {
        for (int ll = 0; ll <= p; ++ll) B[size_t(k - 1) * G::N + ll] = float(R(ll, k));
        for (int ll = 1; ll <= p; ++ll) B[size_t(p + k - 1) * G::N + p + ll] = float(R(ll, k));
    }
    uint8_t* hi = reinterpret_cast<uint8_t*>(out);
    uint8_t* lo = hi + G::b_bytes;
    for (int j = 0; j < G::K; ++j)
        for (int n = 0; n < G::N; ++n) {
            const float v = B[size_t(j) * G::N + n];
            uint32_t u;
            std::memcpy(&u, &v, 4);
            u &= 0xFFFFE000u;
            float h;
            std::memcpy(&h, &u, 4);
            const float l = v - h;
            const uint32_t at = kmaj_off(n, j, G::N / 8);
            std::memcpy(hi + at, &h, 4);
            std::memcpy(lo + at, &l, 4);
        }
}

}  // namespace

bool m2l_tc_ok(int P1) { return P1 == 13 || P1 == 17; }

size_t m2l_tc_bmat_bytes(int P1) {
    switch (P1) {
        case 13: return 2 * M2lTc<13>::b_bytes;
        case 17: return 2 * M2lTc<17>::b_bytes;
        default: return 0;
    }
}

void m2l_tc_fill_bmat(int P1, void* out) {
    if (P1 == 13) fill_bmat<13>(static_cast<float*>(out));
    if (P1 == 17) fill_bmat<17>(static_cast<float*>(out));
}

// dynamic shared memory of one CTA: A stages and B, then the operator tables and the lists
size_t m2l_tc_smem(int P1, int n_ops, int il_stride) {
    const size_t tables = size_t(n_ops) * (2 * P1 + 1) * sizeof(float2) + size_t(4) * il_stride * sizeof(M2LEntry);
    return (P1 == 13 ? M2lTc<13>::smem : M2lTc<17>::smem) + tables;
}

constexpr int kM2lSmemLimit = 200 * 1024;

cudaError_t launch_m2l_tc(const Tree<float>& t, int n_ops, const void* bmat, int* err, cudaStream_t st) {
    int64_t tiles = 0;
    for (int l = 2; l <= t.Lleaf; ++l) tiles += ((int64_t(1) << (2 * l)) + 127) / 128;
    const double lnRoot = std::log(double(t.n) * t.h);
    const float* bm = static_cast<const float*>(bmat);
    const size_t smem = m2l_tc_smem(t.P1, n_ops, t.il_stride);
    if (smem > size_t(kM2lSmemLimit)) return cudaErrorInvalidValue;
    switch (t.P1) {
        case 13: k_m2l_tc<13><<<unsigned(tiles), kM2lThreads, smem, st>>>(t, t.Lleaf - 3, lnRoot, n_ops, bm, err); break;
        case 17: k_m2l_tc<17><<<unsigned(tiles), kM2lThreads, smem, st>>>(t, t.Lleaf - 3, lnRoot, n_ops, bm, err); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t prepare_m2l_tc() {
    cudaError_t e = cudaFuncSetAttribute(k_m2l_tc<13>, cudaFuncAttributeMaxDynamicSharedMemorySize, kM2lSmemLimit);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_m2l_tc<17>, cudaFuncAttributeMaxDynamicSharedMemorySize, kM2lSmemLimit);
    return e;
}

}  // namespace pp
