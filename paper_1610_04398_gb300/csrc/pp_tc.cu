// Near field on the 5th-generation tensor cores (tcgen05, kind::tf32, FP32 accumulate).
//
// On the uniform grid the near-field sum of a target leaf is, for every near offset o,
//   P_leaf[t] += sum_c K_o[t][c] q_{leaf+o}[c],  K_o[t][c] = log max(h |8 o + c - t|, rho_h),
// a dense 64 x 64 contraction whose matrix K_o is the same for every leaf.  A CTA takes
// 128 leaves (8 x 16) as the M dimension: D[leaf][t] = sum_o A_o . B_o^T with A_o the
// 128 x 64 source weights of the leaves shifted by o and B_o = K_o (64 x 64, precomputed).
// FP32 accuracy from TF32 inputs by splitting both operands, x = x_hi + x_lo with x_hi the
// top 19 bits:  A.B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi.
//
// Operand staging.  The CTA loads the halo of its tile once, (8 + 2D) x (16 + 2D) leaves
// (D the near radius), hi and lo, with one TMA copy each; out-of-grid leaves read as zero.
// It is stored in the tensor cores' no-swizzle K-major layout, [cell quad kc][leaf row]
// [leaf column][4 cells], so that for every offset o the A operand is a window of the halo:
// 8-row core matrices are 8 consecutive leaves of one row (16 B apart), row groups are one
// halo row apart, K core matrices one cell quad apart.  Only K_o streams per offset
// (32 KB, hi and lo, one TMA copy into a ring of stages), stored [kc][hi, lo][t][4 cells]
// so that [B_hi; B_lo] is one N = 128 operand: A_hi [B_hi; B_lo] and A_lo B_hi are two
// MMAs per K step (16 per offset; one thread issues them and the issue rate, not the
// tensor pipe, is what small MMAs run into).  Every CTA starts the near list at its own
// offset, so that the CTAs in flight do not all read the same K_o lines of L2 at once.
//
// The tensor cores' FP32 accumulation loses precision over long MMA chains, so every
// offset gets a fresh accumulator (two TMEM buffers of 128 columns: A_hi B_hi, then the
// correction terms) that the epilogue warps drain into Kahan-compensated FP32 registers
// while the next offset is being multiplied.
//
// Roles: warps 0-3 drain TMEM (warp w owns TMEM lanes 32w..32w+31) and store, warp 4 lane 0
// issues the copies, warp 5 lane 0 issues the MMAs (one elected thread).  Every wait is
// bounded; a wait that gives up sets the error flag and the CTA winds down.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "pp_common.h"

namespace pp {
namespace {

constexpr int kTileLX = 8, kTileLY = 16;          // leaves per CTA tile (M = 128)
constexpr uint32_t kStageBytes = 2 * 64 * 64 * 4;  // K_o hi and lo, [kc][split][t][4]
constexpr uint32_t kMaxStages = 4;
constexpr uint32_t kSmemLimit = 227 * 1024;        // dynamic shared memory of one CTA
constexpr uint32_t kSmemPad = 6 * 1024;            // slack after the last stage
constexpr uint32_t kWaitLimit = 1u << 24;
constexpr uint32_t kTmemCols = 256;  // 2 buffers x (64 main + 64 correction columns)

__host__ __device__ constexpr uint32_t halo_bytes(int D) {
    return uint32_t(kTileLX + 2 * D) * uint32_t(kTileLY + 2 * D) * 256u;  // 64 cells x 4 B per leaf
}
__host__ __device__ constexpr uint32_t stages_for(int D) {
    const uint32_t room = (kSmemLimit - 1024 - kSmemPad - 2 * halo_bytes(D)) / kStageBytes;
    return room < kMaxStages ? room : kMaxStages;
}
__host__ __device__ constexpr uint32_t smem_for(int D) {
    return 1024 + 2 * halo_bytes(D) + stages_for(D) * kStageBytes + kSmemPad;
}
static_assert(stages_for(3) >= 2 && smem_for(3) <= kSmemLimit, "near radius 3 must fit two stages");

__device__ __forceinline__ uint32_t sptr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sptr(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sptr(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(sptr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on a phase of an mbarrier: false if it never completed.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) {
    for (uint32_t i = 0; i < kWaitLimit; ++i)
        if (mbar_try_wait(b, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            sptr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(sptr(bar)), "r"(c0), "r"(c1)
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
        "[%2];" ::"r"(sptr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(sptr(bar)), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

// Shared-memory matrix descriptor, K-major, no swizzle: core matrices of 8 rows x 16 B
// stored contiguously; lbo = byte distance of core matrices adjacent in K, sbo = of 8-row
// groups adjacent in M (or N).
__device__ __forceinline__ uint64_t desc_noswz(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = uint64_t((saddr & 0x3FFFF) >> 4);
    d |= uint64_t((lbo >> 4) & 0x3FFF) << 16;
    d |= uint64_t((sbo >> 4) & 0x3FFF) << 32;
    d |= uint64_t(1) << 46;  // descriptor version; base offset 0, layout type 0 (no swizzle)
    return d;
}

// Instruction descriptors: kind::tf32, D = F32, A = B = TF32, both K-major, M = 128, N = 128 or 64.
constexpr uint32_t idesc_tf32(uint32_t N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((N >> 3) << 17) | ((128u >> 4) << 24);
}
constexpr uint32_t kIdescN128 = idesc_tf32(128), kIdescN64 = idesc_tf32(64);

__device__ __forceinline__ void umma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sptr(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void kahan_add(float& sum, float& comp, float x) {
    const float y = x - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(192, 1)
k_near_tc(const __grid_constant__ CUtensorMap tm_qhi, const __grid_constant__ CUtensorMap tm_qlo,
          const __grid_constant__ CUtensorMap tm_k, const int2* __restrict__ near, int n_near, int D, int n,
          float* __restrict__ p_out, int* __restrict__ err) {
    extern __shared__ uint8_t smem_dyn[];
    __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages], acc_full[2], acc_empty[2], halo_full;
    __shared__ uint32_t tmem_base;
    uint8_t* sbase = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int LX0 = blockIdx.x * kTileLX, LY0 = blockIdx.y * kTileLY;
    const int HX = kTileLX + 2 * D, HY = kTileLY + 2 * D;
    const uint32_t hbytes = halo_bytes(D), nst = stages_for(D);
    uint8_t* halo_hi = sbase;
    uint8_t* halo_lo = sbase + hbytes;
    uint8_t* stage0 = sbase + 2 * hbytes;
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
            mbar_init(&acc_full[b], 1);   // MMA commit: the buffer holds one offset's main product
            mbar_init(&acc_empty[b], 4);  // one arrival per epilogue warp: buffer drained
        }
        mbar_init(&halo_full, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 4) {
        if (lane == 0) {
            // the halo, once: box {4 HX floats, HY leaf rows, 16 cell quads} at leaf (LX0-D, LY0-D)
            mbar_expect_tx(&halo_full, 2 * hbytes);
            tma_load_3d(halo_hi, &tm_qhi, &halo_full, 4 * (LX0 - D), LY0 - D, 0);
            tma_load_3d(halo_lo, &tm_qlo, &halo_full, 4 * (LX0 - D), LY0 - D, 0);
            // K_o of every offset, from offset rot on, through the ring
            int issued = 0;
            for (int i = 0; i < n_near; ++i) {
                const uint32_t s = i % nst;
                if (i >= int(nst) && !mbar_wait(&empty[s], ((i / nst) - 1) & 1)) {
                    atomicExch(err, 2);
                    break;
                }
                const int io = (i + rot) % n_near;
                mbar_expect_tx(&full[s], kStageBytes);
                tma_load_2d(stage0 + s * kStageBytes, &tm_k, &full[s], 0, 32 * io);
                issued = i + 1;
            }
            // before the CTA may exit, every copy issued above has landed (bounded waits)
            if (!mbar_wait(&halo_full, 0)) atomicExch(err, 5);
            for (int i = issued - 1; i >= 0 && i >= issued - int(nst); --i)
                if (!mbar_wait(&full[i % nst], (i / nst) & 1)) atomicExch(err, 5);
        }
    } else if (warp == 5) {
        if (lane == 0) {
            // MMA issuer: the i-th offset of this CTA -> TMEM buffer i & 1 (columns 128 (i & 1)):
            // columns 0-63 A_hi B_hi, 64-127 A_hi B_lo + A_lo B_hi
            const uint32_t kcA = uint32_t(HX * HY) * 16, rowA = uint32_t(HX) * 16;
            int done = 0;
            if (!mbar_wait(&halo_full, 0)) atomicExch(err, 3);
            else
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
                    // descriptors of K step 0; K step j is 2 cell quads on (start address field in 16 B units)
                    const uint64_t ahi = desc_noswz(sptr(halo_hi) + win, kcA, rowA);
                    const uint64_t alo = desc_noswz(sptr(halo_lo) + win, kcA, rowA);
                    const uint64_t bhl = desc_noswz(sptr(stage0 + s * kStageBytes), 2048, 128);
                    const uint64_t da = uint64_t(2 * kcA) >> 4, db = uint64_t(2 * 2048) >> 4;
                    const uint32_t d0 = tmem + uint32_t(buf) * 128;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        umma_tf32(d0, ahi + j * da, bhl + j * db, kIdescN128, j != 0);
                        umma_tf32(d0 + 64, alo + j * da, bhl + j * db, kIdescN64, 1);
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
        float acc[64], comp[64];
#pragma unroll
        for (int c = 0; c < 64; ++c) {
            acc[c] = 0.f;
            comp[c] = 0.f;
        }
        bool ok = true;
        const uint32_t lane_base = uint32_t(warp * 32) << 16;
        for (int i = 0; i < n_near && ok; ++i) {
            const int buf = i & 1;
            bool got = mbar_wait(&acc_full[buf], (i >> 1) & 1);
            got = __all_sync(0xffffffffu, got);
            if (!got) {
                if (lane == 0) atomicExch(err, 4);
                ok = false;
                break;
            }
            tc_fence_after();
#pragma unroll
            for (int hcol = 0; hcol < 2; ++hcol) {
                float vm[32], vc[32];
                tmem_ld32(tmem + lane_base + buf * 128 + hcol * 32, vm);
                tmem_ld32(tmem + lane_base + buf * 128 + 64 + hcol * 32, vc);
#pragma unroll
                for (int c = 0; c < 32; ++c) kahan_add(acc[hcol * 32 + c], comp[hcol * 32 + c], vm[c] + vc[c]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sptr(&acc_empty[buf])) : "memory");
        }
        if (ok) {
            const int m = warp * 32 + lane;
            const int LX = LX0 + (m & 7), LY = LY0 + (m >> 3);
            const float inv2pi = 0.15915494309189533576888376337251f;
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                float* dst = p_out + int64_t(LY * 8 + r) * n + LX * 8;
                float4 a = make_float4((acc[8 * r] - comp[8 * r]) * inv2pi, (acc[8 * r + 1] - comp[8 * r + 1]) * inv2pi,
                                       (acc[8 * r + 2] - comp[8 * r + 2]) * inv2pi,
                                       (acc[8 * r + 3] - comp[8 * r + 3]) * inv2pi);
                float4 b = make_float4((acc[8 * r + 4] - comp[8 * r + 4]) * inv2pi,
                                       (acc[8 * r + 5] - comp[8 * r + 5]) * inv2pi,
                                       (acc[8 * r + 6] - comp[8 * r + 6]) * inv2pi,
                                       (acc[8 * r + 7] - comp[8 * r + 7]) * inv2pi);
                reinterpret_cast<float4*>(dst)[0] = a;
                reinterpret_cast<float4*>(dst)[1] = b;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace

size_t near_tc_smem_bytes(int D) { return smem_for(D); }

bool near_tc_ok(int nL, int D) { return nL >= 16 && (nL % kTileLY) == 0 && D >= 1 && D <= 3; }

cudaError_t launch_near_tc(const NearTcMaps& maps, const int2* near, int n_near, int D, int n, float* p_out,
                           int* err, cudaStream_t st) {
    const int nL = n / 8;
    dim3 grid(nL / kTileLX, nL / kTileLY);
    k_near_tc<<<grid, 192, smem_for(D), st>>>(*reinterpret_cast<const CUtensorMap*>(maps.qhi),
                                              *reinterpret_cast<const CUtensorMap*>(maps.qlo),
                                              *reinterpret_cast<const CUtensorMap*>(maps.k), near, n_near, D,
                                              n, p_out, err);
    return cudaGetLastError();
}

cudaError_t prepare_near_tc() {
    uint32_t most = 0;
    for (int D = 1; D <= 3; ++D) most = smem_for(D) > most ? smem_for(D) : most;
    return cudaFuncSetAttribute(k_near_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(most));
}

}  // namespace pp
