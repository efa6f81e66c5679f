// Near field on the 5th-generation tensor cores (tcgen05, kind::f16, FP32 accumulate).
//
// On the uniform grid the near-field sum of a target leaf is, for every near offset o,
//   P_leaf[t] += sum_c K_o[t][c] q_{leaf+o}[c],  K_o[t][c] = log max(|8 o + c - t|, rho_h / h),
// a dense 64 x 64 contraction whose matrix K_o is the same for every leaf.  A CTA takes
// 128 leaves (8 x 16) as the M dimension: D[leaf][t] = sum_o A_o . B_o^T with A_o the
// 128 x 64 source weights of the leaves shifted by o and B_o = K_o (64 x 64, precomputed).
//
// Precision.  FP32 accuracy from FP16 operands by splitting both, x = x_hi + x_lo with
// x_hi = fp16(x) and x_lo = fp16(x - x_hi) (11 + 11 significant bits):
//   A.B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi.
// FP16's exponent range is narrow, so each CTA scales its source weights by a power of two
// s that puts the largest |q| of its halo in [2^14, 2^15); the output is divided by s.  A
// power of two changes no significant bit, so the split is the same as for unscaled data
// wherever FP16 has the range.  K_o lies in [log(rho_h / h), log(31 sqrt 2)] = [-1.07, 3.79].
//
// Operand staging.  The CTA loads the halo of its tile once, (8 + 2D) x (16 + 2D) leaves
// (D the near radius) of the FP32 weights q (leaf-major, 64 cells per leaf), with one TMA
// copy; out-of-grid leaves read as zero.  All threads then write it split and scaled, in the
// tensor cores' no-swizzle K-major layout [cell row r][leaf row][leaf column][8 cells of the
// row], so that for every offset o the A operand is a window of the halo: 8-row core
// matrices are 8 consecutive leaves of one row (16 B apart), row groups are one halo row
// apart, K core matrices one cell row apart.  Only K_o streams per offset (16 KB, hi and lo,
// one bulk copy into a ring of stages that reuses the FP32 staging area), stored
// [source row r][hi, lo][target t][8 cells] so that [B_hi; B_lo] is one N = 128 operand:
// A_hi [B_hi; B_lo] and A_lo B_hi are two MMAs per K step of 16 (8 per offset).  Every CTA
// starts the near list at its own offset, so that the CTAs in flight do not all read the
// same K_o lines of L2 at once.  Two CTAs fit on one SM for near radius 1.
//
// The tensor cores' FP32 accumulation loses precision over long MMA chains, so every
// offset gets a fresh accumulator (two TMEM buffers of 128 columns: A_hi B_hi, then the
// correction terms) that the epilogue warps add into FP32 registers while the next offset
// is being multiplied.
//
// Roles: warps 0-3 drain TMEM (warp w owns TMEM lanes 32w..32w+31) and store, warp 4 lane 0
// issues the copies, warp 5 lane 0 issues the MMAs (one elected thread); all six warps
// split and scale the halo.  Every wait is bounded; a wait that gives up sets the error
// flag and the CTA winds down.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "pp_common.h"
#include "pp_tcgen05.cuh"

namespace pp {
namespace {

using namespace tc;

constexpr int kTileLX = 8, kTileLY = 16;          // leaves per CTA tile (M = 128)
constexpr uint32_t kStageBytes = 2 * 64 * 64 * 2;  // K_o hi and lo in FP16, [r][split][t][8]
constexpr uint32_t kMaxStages = 4;
constexpr uint32_t kTmemCols = 256;  // 2 buffers x (64 main + 64 correction columns)
constexpr int kThreads = 192;

__host__ __device__ constexpr uint32_t halo_leaves(int D) { return uint32_t(kTileLX + 2 * D) * uint32_t(kTileLY + 2 * D); }
__host__ __device__ constexpr uint32_t staging_bytes(int D) { return halo_leaves(D) * 256u; }  // FP32, 64 cells
__host__ __device__ constexpr uint32_t half_halo_bytes(int D) { return halo_leaves(D) * 128u; }  // FP16, 64 cells
// Near radius 2 reads the halo straight from global memory (L2: the source kernel has just
// written it) instead of staging it in FP32: two CTAs fit on an SM, and the stage ring has
// bytes of its own, so the first K_o copies start before the halo is split.  Radii 1 and 3
// stage it by one TMA copy, in bytes the stage ring reuses afterwards (radius 1 fits two
// CTAs either way, and its staged halo is the faster of the two there).
__host__ __device__ constexpr bool direct_halo(int D) { return D == 2; }
__host__ __device__ constexpr uint32_t stages_for(int D) { return D <= 2 ? 3u : kMaxStages; }
__host__ __device__ constexpr uint32_t ring_bytes(int D) {
    return direct_halo(D) || stages_for(D) * kStageBytes > staging_bytes(D) ? stages_for(D) * kStageBytes
                                                                            : staging_bytes(D);
}
__host__ __device__ constexpr uint32_t smem_for(int D) { return 128 + 2 * half_halo_bytes(D) + ring_bytes(D); }
static_assert(smem_for(1) * 2 <= 226 * 1024, "near radius 1 must fit two CTAs per SM");
static_assert(smem_for(2) * 2 <= 226 * 1024, "near radius 2 must fit two CTAs per SM");
static_assert(smem_for(3) <= 227 * 1024, "near radius 3 must fit one CTA per SM");

// Instruction descriptors: kind::f16, D = F32, A = B = F16, both K-major, M = 128, N = 128 or 64.
constexpr uint32_t idesc_f16(uint32_t N) { return (1u << 4) | ((N >> 3) << 17) | ((128u >> 4) << 24); }
constexpr uint32_t kIdescN128 = idesc_f16(128), kIdescN64 = idesc_f16(64);

__device__ __forceinline__ void umma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Split 8 scaled FP32 values into FP16 hi and lo parts, packed as two 16-byte rows.
__device__ __forceinline__ void split8(const float* x, float s, uint4& hi, uint4& lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float a = x[2 * i] * s, b = x[2 * i + 1] * s;
        const __half ha = __float2half_rn(a), hb = __float2half_rn(b);
        const __half la = __float2half_rn(a - __half2float(ha)), lb = __float2half_rn(b - __half2float(hb));
        h[i] = uint32_t(__half_as_ushort(ha)) | (uint32_t(__half_as_ushort(hb)) << 16);
        l[i] = uint32_t(__half_as_ushort(la)) | (uint32_t(__half_as_ushort(lb)) << 16);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

template <int D>
__global__ void __launch_bounds__(kThreads, D <= 2 ? 2 : 1)
k_near_tc(const __grid_constant__ CUtensorMap tm_q, const float* __restrict__ q, const __half* __restrict__ kmat,
          const int2* __restrict__ near, int n_near, int n, float* __restrict__ p_out, int* __restrict__ err) {
    constexpr int HX = kTileLX + 2 * D;
    constexpr uint32_t nst = stages_for(D);
    extern __shared__ uint8_t smem_dyn[];
    __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages], acc_full[2], acc_empty[2], halo_full;
    __shared__ uint32_t tmem_base;
    __shared__ float red[kThreads / 32];
    uint8_t* sbase = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_dyn) + 127) & ~uintptr_t(127));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int LX0 = blockIdx.x * kTileLX, LY0 = blockIdx.y * kTileLY;
    uint8_t* halo_hi = sbase;
    uint8_t* halo_lo = sbase + half_halo_bytes(D);
    uint8_t* ring = sbase + 2 * half_halo_bytes(D);  // FP32 staging first, then the K_o stages
    const float* stage_q = reinterpret_cast<const float*>(ring);
    const int rot = int((blockIdx.y * gridDim.x + blockIdx.x) % uint32_t(n_near));  // first offset of this CTA

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sptr(&tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 32) {
        for (uint32_t s = 0; s < nst; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);   // MMA commit: the buffer holds one offset's products
            mbar_init(&acc_empty[b], 4);  // one arrival per epilogue warp: buffer drained
        }
        mbar_init(&halo_full, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    // the halo's float4 i (leaf i / 16 of the halo, row-major over HX columns; 4 cells i % 16):
    // from the staging copy, or (near radius 2) from global memory, zero outside the grid
    const float4* q4 = reinterpret_cast<const float4*>(stage_q);
    const int nL = n / 8;
    auto halo4 = [&](int i) -> float4 {
        if constexpr (direct_halo(D)) {
            const int l = i >> 4, hx = l % HX, hy = l / HX;
            const int LX = LX0 - D + hx, LY = LY0 - D + hy;
            if (LX < 0 || LY < 0 || LX >= nL || LY >= nL) return make_float4(0.f, 0.f, 0.f, 0.f);
            return __ldg(reinterpret_cast<const float4*>(q) + (int64_t(LY) * nL + LX) * 16 + (i & 15));
        } else {
            return q4[i];
        }
    };
    // the first K_o stages go out at once when the ring does not share the staging bytes
    const int npre = direct_halo(D) ? (n_near < int(nst) ? n_near : int(nst)) : 0;
    if (threadIdx.x == 128) {
        for (int i = 0; i < npre; ++i) {
            const int io = (i + rot) % n_near;
            mbar_expect_tx(&full[i], kStageBytes);
            bulk_load(ring + i * kStageBytes, kmat + size_t(io) * (kStageBytes / 2), kStageBytes, &full[i]);
        }
    }
    // 1. the FP32 halo, one copy: box {64 cells, HX leaves, HY leaf rows} at leaf (LX0-D, LY0-D)
    bool ok = true;
    if constexpr (!direct_halo(D)) {
        if (threadIdx.x == 128) {
            mbar_expect_tx(&halo_full, staging_bytes(D));
            tma_load_3d(ring, &tm_q, &halo_full, 0, LX0 - D, LY0 - D);
        }
        ok = mbar_wait(&halo_full, 0);
    }
    ok = __syncthreads_and(ok);
    if (!ok) {
        if (threadIdx.x == 0) atomicExch(err, 5);
    } else {
        // 2. the CTA's scale: largest |q| of the halo into [2^14, 2^15)
        float m = 0.f;
#pragma unroll 4
        for (int i = threadIdx.x; i < int(halo_leaves(D)) * 16; i += kThreads) {
            const float4 v = halo4(i);
            m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
        }
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) red[warp] = m;
        __syncthreads();
        m = red[0];
#pragma unroll
        for (int w = 1; w < kThreads / 32; ++w) m = fmaxf(m, red[w]);
        int e = 0;
        if (m > 0.f && m <= 3.4e38f) e = 14 - ilogbf(m);
        e = e > 126 ? 126 : (e < -126 ? -126 : e);
        const float scale = ldexpf(1.f, e);
        // 3. split and scale: one cell row (8 cells) of one leaf per thread and step; leaf l
        //    = halo row * HX + halo column, row r of the leaf -> [r][l][8 cells]
#pragma unroll 2
        for (int i = threadIdx.x; i < int(halo_leaves(D)) * 8; i += kThreads) {
            const int l = i >> 3, r = i & 7;
            float x[8];
            const float4 a = halo4(l * 16 + r * 2), b = halo4(l * 16 + r * 2 + 1);
            x[0] = a.x, x[1] = a.y, x[2] = a.z, x[3] = a.w, x[4] = b.x, x[5] = b.y, x[6] = b.z, x[7] = b.w;
            uint4 hi, lo;
            split8(x, scale, hi, lo);
            const uint32_t at = (uint32_t(r) * halo_leaves(D) + uint32_t(l)) * 16u;
            *reinterpret_cast<uint4*>(halo_hi + at) = hi;
            *reinterpret_cast<uint4*>(halo_lo + at) = lo;
        }
        // the split halo is read by the tensor cores (async proxy); the staging bytes are
        // overwritten by the copies below (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();

        if (warp == 4) {
            if (lane == 0) {
                // K_o of every offset, from offset rot on, through the ring (the first npre
                // copies went out at the start)
                int issued = npre;
                for (int i = npre; i < n_near; ++i) {
                    const uint32_t s = i % nst;
                    if (i >= int(nst) && !mbar_wait(&empty[s], ((i / nst) - 1) & 1)) {
                        atomicExch(err, 2);
                        break;
                    }
                    const int io = (i + rot) % n_near;
                    mbar_expect_tx(&full[s], kStageBytes);
                    bulk_load(ring + s * kStageBytes, kmat + size_t(io) * (kStageBytes / 2), kStageBytes, &full[s]);
                    issued = i + 1;
                }
                // before the CTA may exit, every copy issued above has landed (bounded waits)
                for (int i = issued - 1; i >= 0 && i >= issued - int(nst); --i)
                    if (!mbar_wait(&full[i % nst], (i / nst) & 1)) atomicExch(err, 5);
            }
        } else if (warp == 5) {
            if (lane == 0) {
                // MMA issuer: the i-th offset of this CTA -> TMEM buffer i & 1 (columns 128 (i & 1)):
                // columns 0-63 A_hi B_hi, 64-127 A_hi B_lo + A_lo B_hi
                constexpr uint32_t rowA = uint32_t(HX) * 16, krA = halo_leaves(D) * 16;
                int done = 0;
                for (int i = 0; i < n_near; ++i) {
                    const uint32_t s = i % nst;
                    const int buf = i & 1;
                    if (!mbar_wait(&full[s], (i / nst) & 1) ||
                        (i >= 2 && !mbar_wait(&acc_empty[buf], ((i >> 1) - 1) & 1))) {
                        atomicExch(err, 3);
                        break;
                    }
                    tc_fence_after();
                    const int2 o = near[(i + rot) % n_near];
                    const uint32_t win = uint32_t(o.y + D) * rowA + uint32_t(o.x + D) * 16;
                    // descriptors of K step 0; K step j is 2 cell rows on (start address field in 16 B units)
                    const uint64_t ahi = desc_noswz(sptr(halo_hi) + win, krA, rowA);
                    const uint64_t alo = desc_noswz(sptr(halo_lo) + win, krA, rowA);
                    const uint64_t bhl = desc_noswz(sptr(ring + s * kStageBytes), 2048, 128);
                    const uint64_t da = uint64_t(2 * krA) >> 4, db = uint64_t(2 * 2048) >> 4;
                    const uint32_t d0 = tmem + uint32_t(buf) * 128;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        umma_f16(d0, ahi + j * da, bhl + j * db, kIdescN128, j != 0);
                        umma_f16(d0 + 64, alo + j * da, bhl + j * db, kIdescN64, 1);
                    }
                    umma_commit(&empty[s]);       // the stage is free once these MMAs are done
                    umma_commit(&acc_full[buf]);  // and the buffer is ready
                    done = i + 1;
                }
                // TMEM is freed below only after every MMA issued here has completed
                if (done > 0 && !mbar_wait(&acc_full[(done - 1) & 1], ((done - 1) >> 1) & 1)) atomicExch(err, 6);
            }
        } else {
            // epilogue warps 0-3: TMEM lane = leaf of the tile, column = target cell
            float acc[64];
#pragma unroll
            for (int c = 0; c < 64; ++c) acc[c] = 0.f;
            bool good = true;
            const uint32_t lane_base = uint32_t(warp * 32) << 16;
            for (int i = 0; i < n_near; ++i) {
                const int buf = i & 1;
                bool got = mbar_wait(&acc_full[buf], (i >> 1) & 1);
                got = __all_sync(0xffffffffu, got);
                if (!got) {
                    if (lane == 0) atomicExch(err, 4);
                    good = false;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float vm[16], vc[16];
                    tmem_ld16(tmem + lane_base + buf * 128 + q * 16, vm);
                    tmem_ld16(tmem + lane_base + buf * 128 + 64 + q * 16, vc);
                    tmem_wait_ld();
#pragma unroll
                    for (int c = 0; c < 16; ++c) acc[q * 16 + c] += vm[c] + vc[c];
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0)
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sptr(&acc_empty[buf])) : "memory");
            }
            if (good) {
                const int mrow = warp * 32 + lane;
                const int LX = LX0 + (mrow & 7), LY = LY0 + (mrow >> 3);
                const float f = 0.15915494309189533577f / scale;  // 1 / (2 pi s)
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    float* dst = p_out + int64_t(LY * 8 + r) * n + LX * 8;
                    reinterpret_cast<float4*>(dst)[0] =
                        make_float4(acc[8 * r] * f, acc[8 * r + 1] * f, acc[8 * r + 2] * f, acc[8 * r + 3] * f);
                    reinterpret_cast<float4*>(dst)[1] =
                        make_float4(acc[8 * r + 4] * f, acc[8 * r + 5] * f, acc[8 * r + 6] * f, acc[8 * r + 7] * f);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace

size_t near_tc_smem_bytes(int D) { return D >= 1 && D <= 3 ? smem_for(D) : 0; }

bool near_tc_ok(int nL, int D) { return nL >= 16 && (nL % kTileLY) == 0 && D >= 1 && D <= 3; }

size_t near_tc_kmat_bytes(int n_near) { return size_t(n_near) * kStageBytes; }

// K_o for every near offset, split in FP16 hi and lo: [offset][source row r][hi, lo][target t]
// [8 source cells of row r], from the FP64 values K_o[t][c] = log max(|8 o + c - t|, rho_h / h).
void near_tc_fill_kmat(const int2* offs, int n_near, double rh_over_h, void* out) {
    __half* k = static_cast<__half*>(out);
    for (int i = 0; i < n_near; ++i)
        for (int t = 0; t < 64; ++t)
            for (int c = 0; c < 64; ++c) {
                const double dx = 8.0 * offs[i].x + (c & 7) - (t & 7), dy = 8.0 * offs[i].y + (c >> 3) - (t >> 3);
                const double r = std::sqrt(dx * dx + dy * dy);
                const double v = std::log(r > rh_over_h ? r : rh_over_h);
                const __half hi = __double2half(v);
                const __half lo = __double2half(v - double(__half2float(hi)));
                const size_t row = size_t(i) * 8 + size_t(c >> 3);  // [offset][r]
                const size_t at = (row * 2 * 64 + size_t(t)) * 8 + size_t(c & 7);
                k[at] = hi;
                k[at + 64 * 8] = lo;
            }
}

cudaError_t launch_near_tc(const NearTcMaps& maps, const float* q, const void* kmat, const int2* near, int n_near, int D,
                           int n, float* p_out, int* err, cudaStream_t st) {
    const int nL = n / 8;
    dim3 grid(nL / kTileLX, nL / kTileLY);
    const CUtensorMap& tq = *reinterpret_cast<const CUtensorMap*>(maps.q);
    const __half* km = static_cast<const __half*>(kmat);
    switch (D) {
        case 1: k_near_tc<1><<<grid, kThreads, smem_for(1), st>>>(tq, q, km, near, n_near, n, p_out, err); break;
        case 2: k_near_tc<2><<<grid, kThreads, smem_for(2), st>>>(tq, q, km, near, n_near, n, p_out, err); break;
        case 3: k_near_tc<3><<<grid, kThreads, smem_for(3), st>>>(tq, q, km, near, n_near, n, p_out, err); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t prepare_near_tc() {
    cudaError_t e = cudaFuncSetAttribute(k_near_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_for(1)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_near_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_for(2)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_near_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_for(3)));
    return e;
}

}  // namespace pp
