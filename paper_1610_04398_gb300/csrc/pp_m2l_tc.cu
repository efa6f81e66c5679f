// Multipole-to-local translations on the 5th-generation tensor cores (tcgen05, kind::f16,
// FP32 accumulate), mixed precision, p = 12: the tensor-core form of k_m2l_far.
//
// On the uniform quadtree with scaled coefficients (App. A.2) the translation of one
// interaction-list entry is a fixed complex (p+1) x (p+1) matrix per operator (offset tau
// and side ratio r): b_l = sum_k B[k][l] M_k with M_0 = S, B[0][l] = -1 / (l tau^l) and
// B[k][l] = (-1)^(k+1) C(l+k-1, k-1) r^k tau^-(l+k) (k >= 1); the S log|tau| part of b_0
// stays with the threads (double-float sums, as in k_m2l_far).  In real form, a box's
// coefficients are a row of K = 32 values (Re M_k, Im M_k at 2k, 2k + 1; zero padding) and
// the operator a 32 x 32 matrix W (Re b, Im b in the columns), so that for 128 target boxes
// that share an interaction list (one child position, an 8 x 16 block of its sub-grid) the
// translations of one entry are one dense product D += A_e W_e, A_e the 128 source rows.
//
// The source rows of every entry are windows of one halo held in shared memory: for a
// block of targets of child position (a, b), the same-level sources of child position
// (a', b') form the block shifted by a whole number of boxes on the (a', b') sub-grid, and
// the parent-level sources the block shifted on the parent level.  The halo is five regions
// (four sub-grids, the parent level) of (8 + 2 MG) x (16 + 2 MG) boxes, MG the largest
// shift, and it is the same for the four child positions of a block: a tile is the block
// for all four (4 x 128 targets, one halo).  Layout K-major without swizzle: [K chunk][row]
// [box][8 values], so that an entry's A is the descriptor at the window's first box (8-box
// rows 16 B apart, rows of the window HX boxes apart).
//
// Precision: FP32 accuracy from FP16 operands by splitting both, v = v_hi + v_lo (11 + 11
// bits): A W ~ [A_hi | A_lo] [W_hi ; W_hi] + A_hi W_lo, six MMAs of K = 16 per entry.  FP16
// range: the multipoles are scaled by 2^(14 - e), 2^e above the largest |coefficient| (the
// upward pass keeps that maximum), the operators by one power of two for all of them; the
// epilogue divides both out.  Every product of FP16 values is exact in FP32.
//
// One persistent CTA per SM; tiles are claimed from a global counter, finest level first.
// Warps 0-7 stage the five regions by 8-byte asynchronous copies (two regions in flight;
// seven lanes a box, two coefficients a lane), convert them into the halo (packed FP16
// pairs) and hand it to the MMA warp; warps 0-3 then form the double-float constant terms
// of their rows' four targets and drain the eight accumulators (TMEM, 4 child positions x
// 2 x 32 columns) into the locals.  Warp 8 issues the MMAs, the child positions interleaved;
// warp 9 claims the tiles and streams the operators (4 KB each) through a ring of stages.
// Every wait is bounded and watches a shared abort flag: a wait that gives up sets the error
// flag and the CTA winds down.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>

#include "pp_common.h"
#include "pp_tcgen05.cuh"

namespace pp {
namespace {

using namespace tc;

constexpr int kP1 = 13;                  // coefficients (p = 12): 2 x 13 real values fit K = 32
constexpr int kConvWarps = 8;            // staging / conversion warps
constexpr int kTcThreads = 32 * kConvWarps + 64;  // + the MMA warp and the operator warp
constexpr int kMaxBStages = 8;
constexpr uint32_t kOpBytes = 4096;      // W_hi and W_lo, 32 x 32 FP16 each
constexpr uint32_t kRecBytes = (kP1 + 1) * 8;  // staged box: 13 FP32 coefficients, the double-float S
constexpr int kRecLanes = 7;             // lanes per staged box: two coefficients each (the last: M_12, S)
constexpr int kRecPerStep = 4;           // boxes per warp step (28 lanes)
constexpr uint32_t kEntReserve = 2560;   // shared bytes kept for the entry table (4 x list stride <= 40 x 16)
constexpr int kTcSmemLimit = 226 * 1024;  // dynamic; the static barriers and queue take the rest of 227 KB
constexpr int kQueue = 8;                // claimed tiles the roles may be apart
// Per child position, entries alternate between two accumulators of 32 columns, and the MMA
// warp interleaves the four child positions: eight independent accumulate chains (an MMA of
// N = 32 is short next to the dependency of the next one into the same columns).
constexpr int kAcc = 2;
constexpr uint32_t kTmemCols = 4u * kAcc * 32u;

template <int MG>
struct HcGeom {
    static constexpr int HX = 8 + 2 * MG, HY = 16 + 2 * MG, NREC = HX * HY;
    static constexpr uint32_t PS = uint32_t(NREC) * 16u;  // one K chunk (8 values) of every box
    static constexpr uint32_t RB = 8u * PS;               // region: 4 hi chunks, 4 lo chunks
    static constexpr uint32_t HALO = 5u * RB;
    static constexpr int STEPS = (NREC + kRecPerStep * kConvWarps - 1) / (kRecPerStep * kConvWarps);
    static constexpr uint32_t SLOT = uint32_t(kRecPerStep * STEPS) * kRecBytes;  // a multiple of 16
    static constexpr uint32_t STG = uint32_t(kConvWarps) * 2u * SLOT;
    static constexpr uint32_t SF = 5u * uint32_t(NREC) * 8u;  // the halo boxes' S as double-float pairs
    static constexpr uint32_t base = 128u + HALO + STG + SF;
    // operator stages: as many as fit beside the entry table, at most kMaxBStages
    static constexpr int NB_fit = int((int64_t(kTcSmemLimit) - int64_t(base) - int64_t(kEntReserve)) / kOpBytes);
    static constexpr int NB = NB_fit > kMaxBStages ? kMaxBStages : NB_fit;
    static constexpr uint32_t fixed = base + uint32_t(NB > 0 ? NB : 0) * kOpBytes;
};

// kind::f16 instruction descriptor: D = F32, A = B = F16, both K-major, M = 128, N = 32
constexpr uint32_t kIdesc = (1u << 4) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void umma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void cp_async8z(void* dst, const void* src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(sptr(dst)), "l"(src), "r"(valid ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sptr(b)) : "memory");
}

// Bounded wait that also gives up once another role has raised the abort flag.
__device__ __forceinline__ bool wait_ab(uint64_t* b, uint32_t parity, volatile int* abort_flag) {
    for (uint32_t i = 0; i < kWaitLimit; ++i) {
        if (mbar_try_wait(b, parity)) return true;
        if ((i & 255u) == 255u && *abort_flag) return false;
    }
    return false;
}

// A tile: level l >= 2 and the origin (i0, j0) of an 8 x 16 block of the level's child-
// position sub-grids: the 4 x 128 target boxes that share one halo.
struct Tile {
    int l, i0, j0;
};

__host__ __device__ inline int64_t tiles_of_level(int l) {
    const int s = 1 << (l - 1);
    return int64_t((s + 7) >> 3) * ((s + 15) >> 4);
}

__device__ inline Tile tile_of(int64_t id, int L) {
    Tile T{-1, 0, 0};
    for (int l = L; l >= 2; --l) {
        const int64_t n = tiles_of_level(l);
        if (id < n) {
            const int s = 1 << (l - 1), nbx = (s + 7) >> 3;
            T.l = l;
            T.i0 = int(id % nbx) * 8;
            T.j0 = int(id / nbx) * 16;
            return T;
        }
        id -= n;
    }
    return T;
}

// Box index (level_offset + row-major) behind halo record (hx, hy) of region r; false
// outside the level.  Regions 0-3: level-l boxes of child position r; region 4: the parent level.
template <int MG>
__device__ __forceinline__ bool record_box(const Tile& T, int r, int hx, int hy, int64_t& box) {
    const int sx = T.i0 - MG + hx, sy = T.j0 - MG + hy, s = 1 << (T.l - 1);
    if (sx < 0 || sy < 0 || sx >= s || sy >= s) return false;
    if (r < 4) {
        const int X = 2 * sx + (r & 1), Y = 2 * sy + (r >> 1);
        box = level_offset(T.l) + (int64_t(Y) << T.l) + X;
    } else {
        box = level_offset(T.l - 1) + (int64_t(sy) << (T.l - 1)) + sx;
    }
    return true;
}

// two FP32 values, scaled, as FP16 hi and lo pairs
__device__ __forceinline__ void split2(float x, float y, float s, uint32_t& hi, uint32_t& lo) {
    const float a = x * s, b = y * s;
    const __half2 h = __floats2half2_rn(a, b);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

template <int MG>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_m2l_tc(Tree<float> t, int lr, double lnRoot, const uint8_t* __restrict__ ops, const int4* __restrict__ ents_g,
             int il_stride, int64_t n_tiles, float inv_sb, unsigned* __restrict__ claim, int* __restrict__ err) {
    typedef HcGeom<MG> G;
    constexpr int kBStages = G::NB;
    static_assert(kBStages >= 2, "two operator stages at least");
    extern __shared__ uint8_t smem_dyn[];
    __shared__ __align__(8) uint64_t bfull[kMaxBStages], bempty[kMaxBStages], halo_full, acc_full, acc_empty,
        sums_done, tq_full[kQueue], mma_done;
    __shared__ int tq[kQueue];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    uint8_t* sbase = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_dyn) + 127) & ~uintptr_t(127));
    uint8_t* halo = sbase;
    uint8_t* stg = halo + G::HALO;
    float2* sf_halo = reinterpret_cast<float2*>(stg + G::STG);  // [region][box]
    uint8_t* bring = stg + G::STG + G::SF;
    // [4][il_stride]: region | window << 4, operator, log|tau| as a double-float pair
    int4* ents = reinterpret_cast<int4*>(bring + kBStages * kOpBytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int* ab = &abort_flag;
    int cnt[4], emax = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        cnt[c] = t.il_count[c];
        emax = cnt[c] > emax ? cnt[c] : emax;
    }

    for (int i = threadIdx.x; i < 4 * il_stride; i += blockDim.x) ents[i] = ents_g[i];
    for (uint32_t i = threadIdx.x; i < G::HALO / 16; i += blockDim.x)  // padding chunks stay zero
        reinterpret_cast<uint4*>(halo)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (warp == kConvWarps) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sptr(&tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < kBStages; ++s) {
            mbar_init(&bfull[s], 1);
            mbar_init(&bempty[s], 1);
        }
        mbar_init(&halo_full, kConvWarps);
        mbar_init(&acc_full, 1);
        mbar_init(&acc_empty, 4);
        mbar_init(&sums_done, 4);
        for (int q = 0; q < kQueue; ++q) mbar_init(&tq_full[q], 1);
        mbar_init(&mma_done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the zeroed halo is read by the tensor cores
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    // scale of the multipoles: the largest |coefficient| below 2^15
    const float mx = __uint_as_float(__ldcg(t.mmax));
    int e = (mx > 0.f && mx <= 3.4e38f) ? ilogbf(mx) + 1 : 0;
    e = e > 100 ? 100 : (e < -100 ? -100 : e);
    const float sA = ldexpf(1.f, 14 - e);
    const float unscale = ldexpf(inv_sb, e - 14);  // 1 / (sA sB)

    // the claimed tile of the it-th iteration (-1: no more), published by the operator warp
    auto next_tile = [&](int it, int& id) -> bool {
        if (!wait_ab(&tq_full[it % kQueue], uint32_t(it / kQueue) & 1u, ab)) return false;
        id = tq[it % kQueue];
        return true;
    };

    if (warp == kConvWarps + 1) {
        // ---- operator warp: claims tiles two ahead (the staging warps read the next tile's
        // id before the current tile's operators have all gone out), streams the operators in
        // the MMA order: round r, child positions 0-3
        if (lane == 0) {
            auto publish = [&](int i) -> int {
                const int64_t c = int64_t(atomicAdd(claim, 1u));
                const int v = c < n_tiles ? int(c) : -1;
                tq[i % kQueue] = v;
                arrive(&tq_full[i % kQueue]);
                return v;
            };
            uint32_t gc = 0;  // operators issued
            bool ok = true;
            int cur = publish(0);
            int nxt = cur >= 0 ? publish(1) : -1;
            for (int it = 0; cur >= 0 && ok; ++it) {
                const int nxt2 = nxt >= 0 ? publish(it + 2) : -1;
                for (int r = 0; r < emax && ok; ++r)
                    for (int c = 0; c < 4; ++c) {
                        if (r >= cnt[c]) continue;
                        const uint32_t s = gc % kBStages;
                        if (gc >= uint32_t(kBStages) && !wait_ab(&bempty[s], ((gc / kBStages) - 1u) & 1u, ab)) {
                            ok = false;
                            break;
                        }
                        const int op = ents[c * il_stride + r].y;
                        mbar_expect_tx(&bfull[s], kOpBytes);
                        bulk_load(bring + s * kOpBytes, ops + size_t(op) * kOpBytes, kOpBytes, &bfull[s]);
                        ++gc;
                    }
                cur = nxt;
                nxt = nxt2;
            }
            if (!ok) {
                *ab = 1;
                atomicExch(err, 7);
            }
            // every copy issued above has landed before the CTA may exit
            for (int64_t i = int64_t(gc) - 1; i >= 0 && i >= int64_t(gc) - kBStages; --i)
                if (!mbar_wait(&bfull[i % kBStages], uint32_t(i / kBStages) & 1u)) atomicExch(err, 7);
        }
    } else if (warp == kConvWarps) {
        // ---- MMA warp: per entry, [A_hi | A_lo] [W_hi ; W_hi] (four K steps) + A_hi W_lo (two),
        // into accumulator (child position, round & 1)
        if (lane == 0) {
            uint32_t gc = 0;
            bool ok = true, any = false;
            for (int it = 0; ok; ++it) {
                int id;
                if (!next_tile(it, id)) {
                    ok = false;
                    break;
                }
                if (id < 0) break;
                if (!wait_ab(&halo_full, uint32_t(it) & 1u, ab) ||
                    (it >= 1 && !wait_ab(&acc_empty, uint32_t(it - 1) & 1u, ab))) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                for (int r = 0; r < emax && ok; ++r)
                    for (int c = 0; c < 4; ++c) {
                        if (r >= cnt[c]) continue;
                        const uint32_t s = gc % kBStages;
                        if (!wait_ab(&bfull[s], (gc / kBStages) & 1u, ab)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const int4 en = ents[c * il_stride + r];
                        const uint32_t a0 = sptr(halo) + uint32_t(en.x & 15) * G::RB + uint32_t(en.x >> 4) * 16u;
                        const uint32_t b0 = sptr(bring + s * kOpBytes);
                        const uint32_t d = tmem + uint32_t(c) * (kAcc * 32u) + uint32_t(r % kAcc) * 32u;
                        const uint32_t acc0 = r < kAcc ? 0u : 1u;  // the accumulator's first entry overwrites
#pragma unroll
                        for (uint32_t ks = 0; ks < 4; ++ks)
                            umma_f16(d, desc_noswz(a0 + 2u * ks * G::PS, G::PS, uint32_t(G::HX) * 16u),
                                     desc_noswz(b0 + ((2u * ks) & 3u) * 512u, 512u, 128u), ks == 0u ? acc0 : 1u);
#pragma unroll
                        for (uint32_t ks = 0; ks < 2; ++ks)
                            umma_f16(d, desc_noswz(a0 + 2u * ks * G::PS, G::PS, uint32_t(G::HX) * 16u),
                                     desc_noswz(b0 + 2048u + 2u * ks * 512u, 512u, 128u), 1u);
                        umma_commit(&bempty[s]);  // the stage is free once these MMAs are done
                        any = true;
                        ++gc;
                    }
                if (!ok) break;
                umma_commit(&acc_full);  // the accumulators are ready and the halo free
            }
            if (!ok) {
                *ab = 1;
                atomicExch(err, 8);
            }
            // TMEM is freed below only after every MMA issued here has completed
            if (any) {
                umma_commit(&mma_done);
                if (!mbar_wait(&mma_done, 0)) atomicExch(err, 8);
            }
        }
    } else {
        // ---- staging warps: lanes 0-27 in groups of 7, a group per box and step, a lane per
        // two coefficients (the last lane: M_12 and the double-float S)
        const int rl = lane / kRecLanes, kk = 2 * (lane % kRecLanes);
        const bool slane = lane < kRecLanes * kRecPerStep;
        auto slot_of = [&](int sl) { return stg + (uint32_t(warp) * 2u + uint32_t(sl)) * G::SLOT; };
        // region r of tile T -> staging slot sl: one commit group
        auto issue = [&](const Tile& T, int r, int sl) {
            uint8_t* sb = slot_of(sl);
#pragma unroll 2
            for (int s = 0; s < G::STEPS; ++s) {
                const int q = kRecPerStep * (warp + kConvWarps * s) + rl;
                if (slane && q < G::NREC) {
                    int64_t box = 0;
                    const bool in = record_box<MG>(T, r, q % G::HX, q / G::HX, box);
                    const float2* m = t.mp + box * kP1 + kk;
                    const float2* second = kk + 1 < kP1 ? m + 1 : t.Sf + box;
                    uint8_t* d = sb + (uint32_t(kRecPerStep * s + rl) * (kP1 + 1) + uint32_t(kk)) * 8u;
                    cp_async8z(d, in ? m : t.Sf, in);
                    cp_async8z(d + 8, in ? second : t.Sf, in);
                }
            }
            cp_commit();
        };
        // staging slot sl -> region r of the halo: K index 2k = Re M_k, 2k + 1 = Im M_k, scaled
        // and split; each lane reads what it copied
        auto convert = [&](int r, int sl) {
            const uint8_t* sb = slot_of(sl);
            uint8_t* reg = halo + uint32_t(r) * G::RB + uint32_t(kk >> 2) * G::PS + uint32_t(kk & 3) * 4u;
#pragma unroll 2
            for (int s = 0; s < G::STEPS; ++s) {
                const int q = kRecPerStep * (warp + kConvWarps * s) + rl;
                if (slane && q < G::NREC) {
                    const float4 v = *reinterpret_cast<const float4*>(
                        sb + (uint32_t(kRecPerStep * s + rl) * (kP1 + 1) + uint32_t(kk)) * 8u);
                    uint32_t h0, l0;
                    split2(v.x, v.y, sA, h0, l0);
                    uint8_t* rec = reg + uint32_t(q) * 16u;
                    if (kk + 1 < kP1) {
                        uint32_t h1, l1;
                        split2(v.z, v.w, sA, h1, l1);
                        *reinterpret_cast<uint2*>(rec) = make_uint2(h0, h1);
                        *reinterpret_cast<uint2*>(rec + 4u * G::PS) = make_uint2(l0, l1);
                    } else {
                        *reinterpret_cast<uint32_t*>(rec) = h0;
                        *reinterpret_cast<uint32_t*>(rec + 4u * G::PS) = l0;
                        sf_halo[r * G::NREC + q] = make_float2(v.z, v.w);
                    }
                }
            }
        };
        // double-float constant-term sums of the target in row threadIdx.x (warps 0-3) for
        // child position c: sum S log|tau| and sum S over its list, S from the halo (zero
        // outside the level)
        auto const_sums = [&](int c, float4& cs) {
            float ah = 0.f, al = 0.f, sh = 0.f, sl = 0.f;
            const int m = threadIdx.x;
            const int at = (m >> 3) * G::HX + (m & 7);
            const int4* le = ents + c * il_stride;
#pragma unroll 4
            for (int e2 = 0; e2 < cnt[c]; ++e2) {
                const int4 en = le[e2];
                const float2 Sd = sf_halo[(en.x & 15) * G::NREC + (en.x >> 4) + at];
                df_fma(ah, al, Sd.x, Sd.y, __int_as_float(en.z), __int_as_float(en.w));
                df_add(sh, sl, Sd.x, Sd.y);
            }
            cs = make_float4(ah, al, sh, sl);
        };
        // the accumulators -> the locals of tile T (warps 0-3: TMEM lanes 32 warp.. = rows)
        auto drain = [&](const Tile& T, const float4 (&cs)[4]) {
            tc_fence_after();
            const int m = threadIdx.x, s = 1 << (T.l - 1);
            const int sx = T.i0 + (m & 7), sy = T.j0 + (m >> 3);
            const bool act = sx < s && sy < s;
            const double lnS = fma(double(-T.l), 0.69314718055994530941723212145818, lnRoot);  // log(side / 2^l)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float v[32];
                const uint32_t ta = tmem + (uint32_t(warp * 32) << 16) + uint32_t(c) * (kAcc * 32u);
                tmem_ld16(ta, v);
                tmem_ld16(ta + 16u, v + 16);
                tmem_wait_ld();
                if (cnt[c] > 1) {
                    float w[32];
                    tmem_ld16(ta + 32u, w);
                    tmem_ld16(ta + 48u, w + 16);
                    tmem_wait_ld();
#pragma unroll
                    for (int i = 0; i < 32; ++i) v[i] += w[i];
                }
                if (act) {
                    const int bx = 2 * sx + (c & 1), by = 2 * sy + (c >> 1);
                    const int64_t i = level_offset(T.l) + (int64_t(by) << T.l) + bx;
                    const double L0 = df_to(cs[c].x, cs[c].y) + lnS * df_to(cs[c].z, cs[c].w) + double(v[0] * unscale);
                    float2* out = (T.l < lr ? t.locA : t.loc) + i * kP1;
                    (T.l < lr ? t.L0A : t.L0)[i] = L0;
                    out[0] = make_float2(float(L0), 0.f);
#pragma unroll
                    for (int ll = 1; ll < kP1; ++ll) out[ll] = make_float2(v[ll] * unscale, v[kP1 + ll] * unscale);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) arrive(&acc_empty);
        };

        bool ok = true, got;
        int rc = 0;  // regions staged so far: staging slot rc & 1
        int it = 0, id = -1;
        got = next_tile(0, id);
        ok = __all_sync(0xffffffffu, got);
        Tile T = (ok && id >= 0) ? tile_of(id, t.Lleaf) : Tile{-1, 0, 0};
        if (T.l >= 2) issue(T, 0, 0);
        while (ok && T.l >= 2) {
            // the halo is free once the previous tile's MMAs have completed and warps 0-3 have
            // formed its constant terms from the staged S
            if (it >= 1) {
                got = wait_ab(&acc_full, uint32_t(it - 1) & 1u, ab) && wait_ab(&sums_done, uint32_t(it - 1) & 1u, ab);
                if (!__all_sync(0xffffffffu, got)) {
                    ok = false;
                    break;
                }
            }
            Tile N{-1, 0, 0};
            for (int r = 0; r < 5; ++r) {
                // the next region's copies (after the last region: the next tile's first) go out first
                if (r < 4) {
                    issue(T, r + 1, (rc + 1) & 1);
                } else {
                    int nid = -1;
                    got = next_tile(it + 1, nid);
                    if (!__all_sync(0xffffffffu, got)) ok = false;
                    if (ok && nid >= 0) {
                        N = tile_of(nid, t.Lleaf);
                        issue(N, 0, (rc + 1) & 1);
                    } else {
                        cp_commit();
                    }
                }
                cp_wait<1>();
                convert(r, rc & 1);
                ++rc;
                __syncwarp();
            }
            if (!ok) break;
            // the halo is read by the tensor cores (async proxy)
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) arrive(&halo_full);
            if (warp < 4) {
                // every staging warp's part of the halo S is in place
                got = wait_ab(&halo_full, uint32_t(it) & 1u, ab);
                if (!__all_sync(0xffffffffu, got)) {
                    ok = false;
                    break;
                }
                float4 cs[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) const_sums(c, cs[c]);
                __syncwarp();
                if (lane == 0) arrive(&sums_done);
                got = wait_ab(&acc_full, uint32_t(it) & 1u, ab);
                if (!__all_sync(0xffffffffu, got)) {
                    ok = false;
                    break;
                }
                drain(T, cs);
            }
            T = N;
            ++it;
        }
        cp_wait<0>();  // no copy outlives the CTA
        if (!ok) {
            *ab = 1;
            if (lane == 0) atomicExch(err, 9);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kConvWarps)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    // the last CTA to finish resets the tile counter for the next launch
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(claim + 1, 1u) == gridDim.x - 1) {
            atomicExch(claim, 0u);
            atomicExch(claim + 1, 0u);
        }
    }
}

int fdiv2(int v) { return v >= 0 ? v / 2 : -((1 - v) / 2); }
int mod2(int v) { return v & 1; }  // two's complement: also right for negative v

template <int MG>
size_t smem_of(int il_stride) {
    return HcGeom<MG>::fixed + size_t(4) * il_stride * sizeof(int4);
}

}  // namespace

// The largest shift, in boxes, of an entry's window on its sub-grid (same level) or on the
// parent level: the halo margin.  -1 when it exceeds 2 or a list is empty.
int m2l_tc_margin(const M2LEntry* il, const int* il_count, int il_stride) {
    int mg = 1;
    for (int c = 0; c < 4; ++c) {
        if (il_count[c] < 1) return -1;
        const int a = c & 1, b = c >> 1;
        for (int e = 0; e < il_count[c]; ++e) {
            const M2LEntry& en = il[size_t(c) * il_stride + e];
            const int sx = en.pad == 0 ? fdiv2(a + en.dx) : en.dx;
            const int sy = en.pad == 0 ? fdiv2(b + en.dy) : en.dy;
            mg = std::max(mg, std::max(std::abs(sx), std::abs(sy)));
        }
    }
    return mg <= 2 ? mg : -1;
}

bool m2l_tc_ok(int P1, int margin, int il_stride) {
    if (P1 != kP1 || (margin != 1 && margin != 2)) return false;
    return (margin == 1 ? smem_of<1>(il_stride) : smem_of<2>(il_stride)) <= size_t(kTcSmemLimit);
}

size_t m2l_tc_table_bytes(int n_ops, int il_stride) {
    return size_t(n_ops) * kOpBytes + size_t(4) * il_stride * sizeof(int4);
}

int64_t m2l_tc_tiles(int Lleaf) {
    int64_t n = 0;
    for (int l = 2; l <= Lleaf; ++l) n += tiles_of_level(l);
    return n;
}

// Operators: W[j][n] (j = 2k: Re M_k, 2k + 1: Im M_k; n: Re b_0..b_12, Im b_0..b_12) of
// b_l = sum_k B[k][l] M_k, scaled by one power of two and split in FP16 hi and lo, each in
// the K-major core-matrix layout [K chunk j/8][N group n/8][n % 8][j % 8]; then per child
// position the entries {region, window, operator, 0}.
float m2l_tc_fill_tables(const double* op_geo, int n_ops, const M2LEntry* il, const int* il_count, int il_stride,
                         int margin, void* out) {
    typedef std::complex<double> cd;
    std::vector<double> W(size_t(n_ops) * 32 * 32, 0.0);
    double wmax = 0.0;
    for (int o = 0; o < n_ops; ++o) {
        const cd tau(op_geo[3 * o], op_geo[3 * o + 1]);
        const double r = op_geo[3 * o + 2];
        double* w = W.data() + size_t(o) * 32 * 32;
        for (int k = 0; k < kP1; ++k)
            for (int l = 0; l < kP1; ++l) {
                cd bkl(0.0, 0.0);
                if (k == 0 && l >= 1) {
                    bkl = -1.0 / (double(l) * std::pow(tau, l));
                } else if (k >= 1) {
                    double c = 1.0;  // C(l + k - 1, k - 1)
                    for (int i = 1; i <= k - 1; ++i) c = c * double(l + i) / double(i);
                    bkl = ((k + 1) % 2 == 0 ? 1.0 : -1.0) * c * std::pow(r, k) * std::pow(tau, -(l + k));
                }
                w[size_t(2 * k) * 32 + l] = bkl.real();  // row 2k: Re M_k
                w[size_t(2 * k) * 32 + kP1 + l] = bkl.imag();
                w[size_t(2 * k + 1) * 32 + l] = -bkl.imag();  // row 2k + 1: Im M_k
                w[size_t(2 * k + 1) * 32 + kP1 + l] = bkl.real();
            }
    }
    for (double v : W) wmax = std::max(wmax, std::fabs(v));
    const int eb = wmax > 0.0 ? std::ilogb(wmax) + 1 : 0;
    const double sB = std::ldexp(1.0, 14 - eb);
    uint8_t* base = static_cast<uint8_t*>(out);
    for (int o = 0; o < n_ops; ++o) {
        uint8_t* hi = base + size_t(o) * kOpBytes;
        uint8_t* lo = hi + kOpBytes / 2;
        for (int j = 0; j < 32; ++j)
            for (int n = 0; n < 32; ++n) {
                const double v = W[(size_t(o) * 32 + j) * 32 + n] * sB;
                const __half h = __double2half(v);
                const __half l = __double2half(v - double(__half2float(h)));
                const size_t at = size_t(((j >> 3) * 4 + (n >> 3)) * 128 + (n & 7) * 16 + (j & 7) * 2);
                std::memcpy(hi + at, &h, 2);
                std::memcpy(lo + at, &l, 2);
            }
    }
    const int HX = 8 + 2 * margin;
    int4* ents = reinterpret_cast<int4*>(base + size_t(n_ops) * kOpBytes);
    for (int c = 0; c < 4; ++c) {
        const int a = c & 1, b = c >> 1;
        for (int e = 0; e < il_stride; ++e) {
            int4 v = make_int4(0, 0, 0, 0);
            if (e < il_count[c]) {
                const M2LEntry& en = il[size_t(c) * il_stride + e];
                int region, ox, oy;
                if (en.pad == 0) {
                    region = mod2(a + en.dx) + 2 * mod2(b + en.dy);
                    ox = fdiv2(a + en.dx) + margin;
                    oy = fdiv2(b + en.dy) + margin;
                } else {
                    region = 4;
                    ox = en.dx + margin;
                    oy = en.dy + margin;
                }
                const double lt = std::log(std::hypot(op_geo[3 * en.op], op_geo[3 * en.op + 1]));
                const float lh = float(lt), ll = float(lt - double(lh));
                int zh, zl;
                std::memcpy(&zh, &lh, 4);
                std::memcpy(&zl, &ll, 4);
                v = make_int4(region | ((oy * HX + ox) << 4), en.op, zh, zl);
            }
            ents[size_t(c) * il_stride + e] = v;
        }
    }
    return float(1.0 / sB);
}

cudaError_t launch_m2l_tc(const Tree<float>& t, const void* tables, int n_ops, int il_stride, int margin, float inv_sb,
                          unsigned* claim, int sms, int* err, cudaStream_t st) {
    if (t.P1 != kP1 || !t.mmax || !claim || sms < 1) return cudaErrorInvalidValue;
    const int64_t tiles = m2l_tc_tiles(t.Lleaf);
    const unsigned grid = unsigned(std::min<int64_t>(tiles, sms));
    const uint8_t* ops = static_cast<const uint8_t*>(tables);
    const int4* ents = reinterpret_cast<const int4*>(ops + size_t(n_ops) * kOpBytes);
    const double lnRoot = std::log(double(t.n) * t.h);
    const int lr = t.Lleaf - 3;
    switch (margin) {
        case 1:
            k_m2l_tc<1><<<grid, kTcThreads, smem_of<1>(il_stride), st>>>(t, lr, lnRoot, ops, ents, il_stride, tiles,
                                                                        inv_sb, claim, err);
            break;
        case 2:
            k_m2l_tc<2><<<grid, kTcThreads, smem_of<2>(il_stride), st>>>(t, lr, lnRoot, ops, ents, il_stride, tiles,
                                                                        inv_sb, claim, err);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t prepare_m2l_tc() {
    cudaError_t e = cudaFuncSetAttribute(k_m2l_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemLimit);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_m2l_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemLimit);
    return e;
}

}  // namespace pp
