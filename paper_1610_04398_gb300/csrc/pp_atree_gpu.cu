// The adaptive quadtree and its interaction lists built on the GPU (the same tree and the
// same sorted lists as the host build in pp_atree.cu; Appendix A.2 groups the sources of the
// multiresolution grid hierarchically).
//
//  1. Morton keys.  A leaf block (l, ix, iy) covers the Z-order range [key, key + 4^(20 - l))
//     of the finest level 20, key = interleave(ix 2^(20 - l), iy 2^(20 - l)) (x in the lower
//     bit of each pair, so child c = (x & 1) + 2 (y & 1) follows Z-order).
//  2. An LSD radix sort of the keys (8-bit digits: per-block digit histograms, a scan of the
//     histograms in digit-major order, a stable scatter ranked by warp match masks).
//  3. Validation in one pass: the leaves tile the domain exactly iff, in key order, each range
//     starts where the previous one ends, the first at 0 and the last ending at 4^20.
//  4. Boxes level by level.  The boxes of level k in Z-order are the distinct level-k
//     prefixes of the sorted leaves of level >= k; leaf i opens the level-k boxes
//     k in (min(level of leaf i-1, common depth of leaves i-1 and i), level of leaf i].  A
//     device-wide exclusive scan (warp shuffles within a block, block totals scanned) of those
//     flags gives every box its index; the top-down, level-by-level Z-order is the host
//     build's order (children of a box together).  The first child of an internal box is the
//     level-(k+1) box its first leaf opens.
//  5. Lists by a breadth-first dual-tree walk: a frontier of (target, source) box pairs, each
//     either a well-separated pair (multipole-to-local), two leaves that are not (near field),
//     or split into four pairs; warp-aggregated output slots (ballot, popcount, one atomic per
//     warp and kind).  The acceptance test is the host's, in the same exact integer units.
//  6. Both lists radix-sorted by (target, source).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <new>
#include <utility>
#include <vector>

#include "../../include/pp.h"
#include "pp_atree_state.h"

namespace {

constexpr int kDepth = 20;  // finest level of the Morton keys (the host build's limit)
constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;
constexpr int kBins = 256;

__device__ __forceinline__ uint64_t spread_bits(uint32_t v) {  // bit b of v -> bit 2b
    uint64_t x = v & 0xfffffu;
    x = (x | (x << 16)) & 0x0000ffff0000ffffull;
    x = (x | (x << 8)) & 0x00ff00ff00ff00ffull;
    x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    x = (x | (x << 1)) & 0x5555555555555555ull;
    return x;
}

__device__ __forceinline__ uint32_t gather_bits(uint64_t x) {  // bit 2b of x -> bit b
    x &= 0x5555555555555555ull;
    x = (x | (x >> 1)) & 0x3333333333333333ull;
    x = (x | (x >> 2)) & 0x0f0f0f0f0f0f0f0full;
    x = (x | (x >> 4)) & 0x00ff00ff00ff00ffull;
    x = (x | (x >> 8)) & 0x0000ffff0000ffffull;
    x = (x | (x >> 16)) & 0x00000000ffffffffull;
    return uint32_t(x);
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ------------------------------------------------------------------ radix sort (keys, values)
__global__ void __launch_bounds__(kThreads) k_digit_hist(const uint64_t* __restrict__ keys, int n, int shift,
                                                         uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[kBins];
    for (int i = threadIdx.x; i < kBins; i += kThreads) h[i] = 0;
    __syncthreads();
    const int64_t base = int64_t(blockIdx.x) * kTile;
    for (int j = 0; j < kItems; ++j) {
        const int64_t i = base + int64_t(j) * kThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & (kBins - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kBins; d += kThreads) hist[int64_t(d) * gridDim.x + blockIdx.x] = h[d];
}

// Exclusive scan of n counts in place by one CTA of 1024 threads; *total (if given) = the sum.
__global__ void __launch_bounds__(1024) k_scan_small(uint32_t* __restrict__ a, int64_t n, uint32_t* total) {
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b = 0; b < n; b += 1024) {
        const int64_t i = b + threadIdx.x;
        const uint32_t v = i < n ? a[i] : 0u;
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            wsum[lane] = w;  // inclusive over warps
        }
        __syncthreads();
        const uint32_t before = carry + (warp > 0 ? wsum[warp - 1] : 0u) + x - v;
        if (i < n) a[i] = before;
        __syncthreads();
        if (threadIdx.x == 0) carry += wsum[31];
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void __launch_bounds__(kThreads) k_digit_scatter(const uint64_t* __restrict__ kin,
                                                            const uint32_t* __restrict__ vin, uint64_t* __restrict__ kout,
                                                            uint32_t* __restrict__ vout, int n, int shift,
                                                            const uint32_t* __restrict__ hist) {
    __shared__ uint32_t base[kBins];
    __shared__ uint32_t wcount[kThreads / 32][kBins];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < kBins; d += kThreads) base[d] = hist[int64_t(d) * gridDim.x + blockIdx.x];
    for (int r = 0; r < kItems; ++r) {
        const int64_t i = int64_t(blockIdx.x) * kTile + int64_t(r) * kThreads + threadIdx.x;
        const bool valid = i < n;
        const uint64_t key = valid ? kin[i] : 0ull;
        const uint32_t digit = valid ? uint32_t((key >> shift) & (kBins - 1)) : uint32_t(kBins);
        for (int j = threadIdx.x; j < (kThreads / 32) * kBins; j += kThreads) (&wcount[0][0])[j] = 0u;
        __syncthreads();
        const uint32_t peers = __match_any_sync(0xffffffffu, digit);
        const uint32_t rank = __popc(peers & lanemask_lt());
        if (valid && lane == __ffs(peers) - 1) wcount[warp][digit] = __popc(peers);
        __syncthreads();
        uint32_t tot = 0;  // thread d: prefix of digit d over the warps, in place
        if (threadIdx.x < kBins) {
            for (int w = 0; w < kThreads / 32; ++w) {
                const uint32_t c = wcount[w][threadIdx.x];
                wcount[w][threadIdx.x] = tot;
                tot += c;
            }
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = base[digit] + wcount[warp][digit] + rank;
            kout[pos] = key;
            if (vin) vout[pos] = vin[i];
        }
        __syncthreads();
        if (threadIdx.x < kBins) base[threadIdx.x] += tot;
        __syncthreads();
    }
}

// Sorts n keys (and values, if given) on their low `bits` bits; the result is in *keys / *vals
// (the pointers may come back swapped with the temporaries).
cudaError_t radix_sort(uint64_t** keys, uint32_t** vals, uint64_t** ktmp, uint32_t** vtmp, int n, int bits,
                       uint32_t* hist, cudaStream_t st) {
    if (n <= 1) return cudaSuccess;
    const int nb = (n + kTile - 1) / kTile;
    for (int shift = 0; shift < bits; shift += 8) {
        k_digit_hist<<<nb, kThreads, 0, st>>>(*keys, n, shift, hist);
        k_scan_small<<<1, 1024, 0, st>>>(hist, int64_t(kBins) * nb, nullptr);
        k_digit_scatter<<<nb, kThreads, 0, st>>>(*keys, vals ? *vals : nullptr, *ktmp, vals ? *vtmp : nullptr, n,
                                                shift, hist);
        std::swap(*keys, *ktmp);
        if (vals) std::swap(*vals, *vtmp);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ device-wide exclusive scan
__global__ void __launch_bounds__(1024) k_scan_blocks(uint32_t* __restrict__ a, int64_t n,
                                                      uint32_t* __restrict__ sums) {
    __shared__ uint32_t wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i = int64_t(blockIdx.x) * 1024 + threadIdx.x;
    const uint32_t v = i < n ? a[i] : 0u;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    if (i < n) a[i] = (warp > 0 ? wsum[warp - 1] : 0u) + x - v;
    if (threadIdx.x == 0) sums[blockIdx.x] = wsum[31];
}

__global__ void k_scan_add(uint32_t* __restrict__ a, int64_t n, const uint32_t* __restrict__ sums) {
    const int64_t i = int64_t(blockIdx.x) * 1024 + threadIdx.x;
    if (i < n) a[i] += sums[blockIdx.x];
}

// a[0..n) -> exclusive prefix sums; *total = the sum (device).
cudaError_t scan_exclusive(uint32_t* a, int64_t n, uint32_t* sums, uint32_t* total, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t nb = (n + 1023) / 1024;
    k_scan_blocks<<<unsigned(nb), 1024, 0, st>>>(a, n, sums);
    k_scan_small<<<1, 1024, 0, st>>>(sums, nb, total);
    k_scan_add<<<unsigned(nb), 1024, 0, st>>>(a, n, sums);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ the tree
// err bits: 1 = a block out of range, 2 = the blocks do not tile the domain
__global__ void k_leaf_keys(const int* __restrict__ level, const int* __restrict__ ix, const int* __restrict__ iy,
                            int n, uint64_t* __restrict__ key, uint32_t* __restrict__ idx, int* err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int l = level[i], x = ix[i], y = iy[i];
    if (l < 0 || l > kDepth || x < 0 || y < 0 || x >= (1 << l) || y >= (1 << l)) {
        atomicOr(err, 1);
        key[i] = 0;
    } else {
        const int sh = kDepth - l;
        key[i] = spread_bits(uint32_t(x) << sh) | (spread_bits(uint32_t(y) << sh) << 1);
    }
    idx[i] = uint32_t(i);
}

__device__ __forceinline__ uint64_t leaf_area(int l) { return uint64_t(1) << (2 * (kDepth - l)); }

// Z-order contiguity of the sorted ranges (exact tiling); the leaf levels in key order.
__global__ void k_check_tiling(const uint64_t* __restrict__ key, const uint32_t* __restrict__ idx,
                               const int* __restrict__ level, int n, int* __restrict__ lev_sorted, int* err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int l = level[idx[i]];
    lev_sorted[i] = l;
    if (l < 0 || l > kDepth) return;  // reported by k_leaf_keys
    const uint64_t end = key[i] + leaf_area(l);
    if (i == 0 && key[0] != 0) atomicOr(err, 2);
    if (i + 1 < n) {
        if (key[i + 1] != end) atomicOr(err, 2);
    } else if (end != (uint64_t(1) << (2 * kDepth))) {
        atomicOr(err, 2);
    }
}

// The deepest level at which leaves i-1 and i share a box, capped by the level of leaf i-1
// (-1 for i = 0): leaf i opens the level-k boxes for k in (lo_i, level_i].
__global__ void k_open_from(const uint64_t* __restrict__ key, const int* __restrict__ lev, int n,
                            int* __restrict__ lo) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (i == 0) {
        lo[0] = -1;
        return;
    }
    const uint64_t d = key[i] ^ key[i - 1];
    const int common = d == 0 ? kDepth : (63 - __clzll(d)) / 2;  // highest differing digit
    const int depth = d == 0 ? kDepth : kDepth - 1 - common;      // levels 0..depth shared
    lo[i] = min(lev[i - 1], depth);
}

__global__ void k_flags(const int* __restrict__ lo, const int* __restrict__ lev, int n, int k,
                        uint32_t* __restrict__ f) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) f[i] = (lo[i] < k && k <= lev[i]) ? 1u : 0u;
}

// Boxes of level k: index off_k + rank_k(i) for every leaf i that opens one; first child =
// the level-(k+1) box the same leaf opens; parents written from the parent's side.
__global__ void k_fill_level(const uint64_t* __restrict__ key, const uint32_t* __restrict__ idx,
                             const int* __restrict__ lo, const int* __restrict__ lev, int n, int k,
                             const uint32_t* __restrict__ rank_k, const uint32_t* __restrict__ rank_k1,
                             const uint32_t* __restrict__ level_count, int* __restrict__ b_level, int* __restrict__ b_ix,
                             int* __restrict__ b_iy, int* __restrict__ b_parent, int* __restrict__ b_child,
                             int* __restrict__ b_leaf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !(lo[i] < k && k <= lev[i])) return;
    uint32_t off = 0, off1 = 0;
    for (int j = 0; j < k; ++j) off += level_count[j];
    off1 = off + level_count[k];
    const uint32_t b = off + rank_k[i];
    const uint64_t pre = key[i] >> (2 * (kDepth - k));
    b_level[b] = k;
    b_ix[b] = int(gather_bits(pre));
    b_iy[b] = int(gather_bits(pre >> 1));
    if (k == 0) b_parent[b] = -1;
    if (lev[i] == k) {
        b_leaf[b] = int(idx[i]);
        b_child[b] = -1;
    } else {
        b_leaf[b] = -1;
        const uint32_t c0 = off1 + rank_k1[i];
        b_child[b] = int(c0);
        for (int c = 0; c < 4; ++c) b_parent[c0 + c] = int(b);
    }
}

// ------------------------------------------------------------------ the lists
struct BoxArrays {
    const int *level, *ix, *iy, *child, *leaf;
};

// Well separated in units of half the finest box side (the host build's test; the units of
// level kDepth instead of the deepest level scale both sides by the same power of two).
__device__ __forceinline__ bool separated(int la, int xa, int ya, int lb, int xb, int yb, double theta) {
    const int64_t sa = int64_t(1) << (kDepth - la + 1), sb = int64_t(1) << (kDepth - lb + 1);
    const int64_t ax = (2 * int64_t(xa) + 1) * (sa / 2), ay = (2 * int64_t(ya) + 1) * (sa / 2);
    const int64_t bx = (2 * int64_t(xb) + 1) * (sb / 2), by = (2 * int64_t(yb) + 1) * (sb / 2);
    const int64_t dx = ax - bx, dy = ay - by;
    const double d2 = double(dx * dx + dy * dy);
    const double s = double(sa + sb);
    return theta * theta * d2 > 0.5 * s * s;
}

// counters: 0 multipole-to-local pairs, 1 near-field pairs, 2 next frontier
__global__ void __launch_bounds__(kThreads) k_walk(BoxArrays bx, const int2* __restrict__ front, int nf, double theta,
                                                   int2* __restrict__ next, int2* __restrict__ m2l,
                                                   int2* __restrict__ p2p, uint32_t* __restrict__ counters) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    int kind = -1;  // 0 m2l, 1 p2p, 2 split the target, 3 split the source
    int a = 0, b = 0;
    if (i < nf) {
        a = front[i].x;
        b = front[i].y;
        const int la = bx.level[a], lb = bx.level[b];
        if (separated(la, bx.ix[a], bx.iy[a], lb, bx.ix[b], bx.iy[b], theta)) {
            kind = 0;
        } else {
            const bool al = bx.leaf[a] >= 0, bl = bx.leaf[b] >= 0;
            if (al && bl) kind = 1;
            else if (!al && (bl || la <= lb)) kind = 2;
            else kind = 3;
        }
    }
    const uint32_t lt = lanemask_lt();
    const uint32_t m_m2l = __ballot_sync(0xffffffffu, kind == 0);
    const uint32_t m_p2p = __ballot_sync(0xffffffffu, kind == 1);
    const uint32_t m_spl = __ballot_sync(0xffffffffu, kind >= 2);
    uint32_t b0 = 0, b1 = 0, b2 = 0;
    if (lane == 0) {
        if (m_m2l) b0 = atomicAdd(&counters[0], uint32_t(__popc(m_m2l)));
        if (m_p2p) b1 = atomicAdd(&counters[1], uint32_t(__popc(m_p2p)));
        if (m_spl) b2 = atomicAdd(&counters[2], 4u * uint32_t(__popc(m_spl)));
    }
    b0 = __shfl_sync(0xffffffffu, b0, 0);
    b1 = __shfl_sync(0xffffffffu, b1, 0);
    b2 = __shfl_sync(0xffffffffu, b2, 0);
    if (kind == 0) {
        m2l[b0 + __popc(m_m2l & lt)] = make_int2(a, b);
    } else if (kind == 1) {
        p2p[b1 + __popc(m_p2p & lt)] = make_int2(bx.leaf[a], bx.leaf[b]);
    } else if (kind >= 2) {
        const uint32_t o = b2 + 4u * uint32_t(__popc(m_spl & lt));
        for (int c = 0; c < 4; ++c)
            next[o + c] = kind == 2 ? make_int2(bx.child[a] + c, b) : make_int2(a, bx.child[b] + c);
    }
}

__global__ void k_pack_pairs(const int2* __restrict__ p, int n, int bits, uint64_t* __restrict__ key) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) key[i] = (uint64_t(uint32_t(p[i].x)) << bits) | uint64_t(uint32_t(p[i].y));
}

__global__ void k_unpack_pairs(const uint64_t* __restrict__ key, int n, int bits, int* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        out[2 * i] = int(key[i] >> bits);
        out[2 * i + 1] = int(key[i] & ((uint64_t(1) << bits) - 1));
    }
}

// ------------------------------------------------------------------ host orchestration
struct DevBufs {
    std::vector<void*> ptrs;
    ~DevBufs() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <typename T>
    T* get(size_t count) {
        void* p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) return nullptr;
        ptrs.push_back(p);
        return static_cast<T*>(p);
    }
};

int blocks(int64_t n, int t = kThreads) { return int((n + t - 1) / t); }

int sort_pairs(DevBufs& mem, int2* pairs, int n, int bits, uint32_t* hist_cap, int64_t hist_n, int* out_host,
               cudaStream_t st) {
    if (n == 0) return PP_OK;
    uint64_t* k = mem.get<uint64_t>(n);
    uint64_t* kt = mem.get<uint64_t>(n);
    int* o = mem.get<int>(2 * int64_t(n));
    uint32_t* hist = hist_cap;
    if (int64_t(kBins) * ((n + kTile - 1) / kTile) > hist_n) hist = mem.get<uint32_t>(size_t(kBins) * ((n + kTile - 1) / kTile));
    if (!k || !kt || !o || !hist) return PP_ERR_OOM;
    k_pack_pairs<<<blocks(n), kThreads, 0, st>>>(pairs, n, bits, k);
    if (radix_sort(&k, nullptr, &kt, nullptr, n, 2 * bits, hist, st) != cudaSuccess) return PP_ERR_CUDA;
    k_unpack_pairs<<<blocks(n), kThreads, 0, st>>>(k, n, bits, o);
    if (cudaMemcpyAsync(out_host, o, sizeof(int) * 2 * size_t(n), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return PP_ERR_CUDA;
    return PP_OK;
}

int build_device(int nleaf, const int* d_level, const int* d_ix, const int* d_iy, double theta, cudaStream_t st,
                 pp::AtreeHost* out) {
    DevBufs mem;
    const int n = nleaf;
    uint64_t* key = mem.get<uint64_t>(n);
    uint64_t* ktmp = mem.get<uint64_t>(n);
    uint32_t* idx = mem.get<uint32_t>(n);
    uint32_t* itmp = mem.get<uint32_t>(n);
    int* lev = mem.get<int>(n);
    int* lo = mem.get<int>(n);
    int* err = mem.get<int>(1);
    const int64_t hist_n = int64_t(kBins) * ((n + kTile - 1) / kTile);
    uint32_t* hist = mem.get<uint32_t>(size_t(hist_n));
    uint32_t* cnt = mem.get<uint32_t>(2 * (kDepth + 1) + 4);
    uint32_t* ranks[2] = {mem.get<uint32_t>(n), mem.get<uint32_t>(n)};
    uint32_t* sums = mem.get<uint32_t>(size_t((n + 1023) / 1024) + 1);
    if (!key || !ktmp || !idx || !itmp || !lev || !lo || !err || !hist || !cnt || !ranks[0] || !ranks[1] || !sums)
        return PP_ERR_OOM;
    if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess ||
        cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (2 * (kDepth + 1) + 4), st) != cudaSuccess)
        return PP_ERR_CUDA;
    // 1-3: keys, sort, tiling check
    k_leaf_keys<<<blocks(n), kThreads, 0, st>>>(d_level, d_ix, d_iy, n, key, idx, err);
    if (radix_sort(&key, &idx, &ktmp, &itmp, n, 2 * kDepth, hist, st) != cudaSuccess) return PP_ERR_CUDA;
    k_check_tiling<<<blocks(n), kThreads, 0, st>>>(key, idx, d_level, n, lev, err);
    int herr = 0;
    if (cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return PP_ERR_CUDA;
    if (herr) return PP_ERR_ARG;
    if ((n - 1) % 3 != 0) return PP_ERR_ARG;  // a full quadtree has 3 I + 1 leaves
    const int nbox = (4 * n - 1) / 3;
    // 4: boxes level by level (level counts in cnt[0..kDepth])
    int* b_level = mem.get<int>(nbox);
    int* b_ix = mem.get<int>(nbox);
    int* b_iy = mem.get<int>(nbox);
    int* b_parent = mem.get<int>(nbox);
    int* b_child = mem.get<int>(nbox);
    int* b_leaf = mem.get<int>(nbox);
    if (!b_level || !b_ix || !b_iy || !b_parent || !b_child || !b_leaf) return PP_ERR_OOM;
    k_open_from<<<blocks(n), kThreads, 0, st>>>(key, lev, n, lo);
    int Lmax = 0;
    {
        std::vector<int> hl(n);
        if (cudaMemcpyAsync(hl.data(), lev, sizeof(int) * size_t(n), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return PP_ERR_CUDA;
        for (int v : hl) Lmax = std::max(Lmax, v);
    }
    // ranks of level 0 first; at level k the ranks of k + 1 are formed before the fill
    k_flags<<<blocks(n), kThreads, 0, st>>>(lo, lev, n, 0, ranks[0]);
    if (scan_exclusive(ranks[0], n, sums, cnt + 0, st) != cudaSuccess) return PP_ERR_CUDA;
    for (int k = 0; k <= Lmax; ++k) {
        uint32_t* rk = ranks[k & 1];
        uint32_t* rk1 = ranks[(k + 1) & 1];
        if (k < Lmax) {
            k_flags<<<blocks(n), kThreads, 0, st>>>(lo, lev, n, k + 1, rk1);
            if (scan_exclusive(rk1, n, sums, cnt + k + 1, st) != cudaSuccess) return PP_ERR_CUDA;
        }
        k_fill_level<<<blocks(n), kThreads, 0, st>>>(key, idx, lo, lev, n, k, rk, rk1, cnt, b_level, b_ix, b_iy,
                                                     b_parent, b_child, b_leaf);
    }
    if (cudaGetLastError() != cudaSuccess) return PP_ERR_CUDA;
    // 5: the breadth-first dual-tree walk
    BoxArrays ba{b_level, b_ix, b_iy, b_child, b_leaf};
    uint32_t* wc = cnt + 2 * (kDepth + 1);  // three counters
    int64_t cap_front = std::max<int64_t>(4 * int64_t(n), 64), cap_next = cap_front;
    int64_t cap_m = cap_front, cap_p = cap_front;
    int2* front = mem.get<int2>(size_t(cap_front));
    int2* next = mem.get<int2>(size_t(cap_next));
    int2* m2l = mem.get<int2>(size_t(cap_m));
    int2* p2p = mem.get<int2>(size_t(cap_p));
    if (!front || !next || !m2l || !p2p) return PP_ERR_OOM;
    const int2 root = make_int2(0, 0);
    if (cudaMemcpyAsync(front, &root, sizeof(int2), cudaMemcpyHostToDevice, st) != cudaSuccess) return PP_ERR_CUDA;
    int64_t nf = 1, nm = 0, np = 0;
    // a list that must hold `need` pairs keeps its first `used` ones when it grows
    auto grow = [&](int2*& buf, int64_t& cap, int64_t used, int64_t need, bool keep) -> int {
        if (need <= cap) return PP_OK;
        const int64_t nc = std::max(need, 2 * cap);
        int2* nb = mem.get<int2>(size_t(nc));
        if (!nb) return PP_ERR_OOM;
        if (keep && used > 0 &&
            cudaMemcpyAsync(nb, buf, sizeof(int2) * size_t(used), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return PP_ERR_CUDA;
        buf = nb;
        cap = nc;
        return PP_OK;
    };
    int rounds = 0;
    while (nf > 0) {
        // every pair of the frontier adds at most one pair to one list, or four to the next frontier
        int s = grow(m2l, cap_m, nm, nm + nf, true);
        if (s == PP_OK) s = grow(p2p, cap_p, np, np + nf, true);
        if (s == PP_OK) s = grow(next, cap_next, 0, 4 * nf, false);
        if (s != PP_OK) return s;
        if (nm + nf > (int64_t(1) << 31) || np + nf > (int64_t(1) << 31) || 4 * nf > (int64_t(1) << 31) ||
            ++rounds > 4 * (kDepth + 2))
            return PP_ERR_OOM;
        const uint32_t init[3] = {uint32_t(nm), uint32_t(np), 0u};
        if (cudaMemcpyAsync(wc, init, sizeof(init), cudaMemcpyHostToDevice, st) != cudaSuccess) return PP_ERR_CUDA;
        k_walk<<<blocks(nf), kThreads, 0, st>>>(ba, front, int(nf), theta, next, m2l, p2p, wc);
        uint32_t got[3];
        if (cudaMemcpyAsync(got, wc, sizeof(got), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return PP_ERR_CUDA;
        nm = got[0];
        np = got[1];
        nf = got[2];
        std::swap(front, next);
        std::swap(cap_front, cap_next);
    }
    // 6: sort both lists; copy the tree and the lists to the host
    int bb = 1;
    while ((int64_t(1) << bb) < std::max(nbox, n)) ++bb;
    out->max_level = Lmax;
    out->level.resize(nbox);
    out->ix.resize(nbox);
    out->iy.resize(nbox);
    out->parent.resize(nbox);
    out->first_child.resize(nbox);
    out->leaf.resize(nbox);
    out->m2l.resize(2 * size_t(nm));
    out->p2p.resize(2 * size_t(np));
    int s = sort_pairs(mem, m2l, int(nm), bb, hist, hist_n, out->m2l.data(), st);
    if (s == PP_OK) s = sort_pairs(mem, p2p, int(np), bb, hist, hist_n, out->p2p.data(), st);
    if (s != PP_OK) return s;
    const std::pair<int*, std::vector<int>*> cp[6] = {{b_level, &out->level}, {b_ix, &out->ix}, {b_iy, &out->iy},
                                                      {b_parent, &out->parent}, {b_child, &out->first_child},
                                                      {b_leaf, &out->leaf}};
    for (auto& c : cp)
        if (cudaMemcpyAsync(c.second->data(), c.first, sizeof(int) * size_t(nbox), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess)
            return PP_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return PP_ERR_CUDA;
    return PP_OK;
}

}  // namespace

extern "C" int pp_atree_create_device(int nleaf, const int* level, const int* ix, const int* iy, double theta,
                                      void* stream, pp_atree* out) {
    if (!out) return PP_ERR_ARG;
    *out = nullptr;
    if (nleaf < 1 || nleaf > (1 << 26) || !level || !ix || !iy || !(theta >= 0.25 && theta <= 0.95)) return PP_ERR_ARG;
    pp::AtreeHost h;
    int st;
    try {
        st = build_device(nleaf, level, ix, iy, theta, static_cast<cudaStream_t>(stream), &h);
    } catch (const std::bad_alloc&) {
        st = PP_ERR_OOM;
    }
    if (st != PP_OK) {
        cudaGetLastError();
        return st;
    }
    return pp::atree_adopt(h, theta, out);
}
