// Penalisation force, Eq. dragPenal (Sec. 3.1), for FP32 (mixed) and FP64 plans.
#include <cuda_runtime.h>

#include <cstdint>

#include "pp_common.h"

namespace pp {

// ------------------------------------------------------------------------------------
// Penalisation force, Eq. dragPenal (Sec. 3.1): F = sum over cells of lambda chi (u - u_s)
// h^2.  Deterministic: a fixed grid of kPenalBlocks CTAs (two per SM), each thread summing a
// fixed stride of cells (FP32 plans with Kahan compensation, FP64 plans in FP64), block tree
// reductions in FP64; the CTA that finishes last (a counter it resets) sums the block
// partials in block order and forms drag/lift.  No CTA waits on another.
// ------------------------------------------------------------------------------------
constexpr int kPenalBlocks = 304;

// Block partial (rs[.][0] after the block's tree) into partial[]; the last block to arrive
// sums all partials in a fixed order and writes out[0..3] = Fx, Fy, drag, lift.
__device__ __forceinline__ void penal_finish(double (*rs)[256], double* __restrict__ partial,
                                             unsigned* __restrict__ counter, double scale, double uhx,
                                             double uhy, double* __restrict__ out) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = rs[0][0];
        partial[2 * blockIdx.x + 1] = rs[1][0];
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double sx = 0.0, sy = 0.0;
    for (int b = threadIdx.x; b < int(gridDim.x); b += blockDim.x) {
        sx += __ldcg(partial + 2 * b);
        sy += __ldcg(partial + 2 * b + 1);
    }
    rs[0][threadIdx.x] = sx;
    rs[1][threadIdx.x] = sy;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (int(threadIdx.x) < o) {
            rs[0][threadIdx.x] += rs[0][threadIdx.x + o];
            rs[1][threadIdx.x] += rs[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double fx = scale * rs[0][0], fy = scale * rs[1][0];
        out[0] = fx;
        out[1] = fy;
        out[2] = fx * uhx + fy * uhy;
        out[3] = -fx * uhy + fy * uhx;
        *counter = 0u;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_penal_partial(const T* __restrict__ u, const T* __restrict__ v,
                                                       const T* __restrict__ chi, const T* __restrict__ usx,
                                                       const T* __restrict__ usy, int64_t ncell,
                                                       double* __restrict__ partial, unsigned* __restrict__ counter,
                                                       double scale, double uhx, double uhy, double* __restrict__ out) {
    __shared__ double rs[2][256];
    T sx = T(0), sy = T(0), cx = T(0), cy = T(0);  // running sums and their compensations
    for (int64_t i = int64_t(blockIdx.x) * 256 + threadIdx.x; i < ncell; i += int64_t(gridDim.x) * 256) {
        const T c = chi[i];
        const T ax = c * (u[i] - usx[i]), ay = c * (v[i] - usy[i]);
        if (sizeof(T) == 4) {
            const T yx = ax - cx, tx = sx + yx;
            cx = (tx - sx) - yx;
            sx = tx;
            const T yy = ay - cy, ty = sy + yy;
            cy = (ty - sy) - yy;
            sy = ty;
        } else {
            sx += ax;
            sy += ay;
        }
    }
    rs[0][threadIdx.x] = double(sx) - double(cx);
    rs[1][threadIdx.x] = double(sy) - double(cy);
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (int(threadIdx.x) < o) {
            rs[0][threadIdx.x] += rs[0][threadIdx.x + o];
            rs[1][threadIdx.x] += rs[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    penal_finish(rs, partial, counter, scale, uhx, uhy, out);
}

// FP32 fields, 16-byte aligned, ncell a multiple of 4: four cells per load; each thread issues
// the loads of four strides before their compensated sums (the only serial part).
template <typename T>
__global__ void __launch_bounds__(256) k_penal_partial4(const float4* __restrict__ u, const float4* __restrict__ v,
                                                        const float4* __restrict__ chi, const float4* __restrict__ usx,
                                                        const float4* __restrict__ usy, int64_t nvec,
                                                        double* __restrict__ partial, unsigned* __restrict__ counter,
                                                        double scale, double uhx, double uhy,
                                                        double* __restrict__ out) {
    __shared__ double rs[2][256];
    float sx = 0.f, sy = 0.f, cx = 0.f, cy = 0.f;
    auto add = [](float& sum, float& comp, float a) {
        const float y = a - comp, t = sum + y;
        comp = (t - sum) - y;
        sum = t;
    };
    const int64_t stride = int64_t(gridDim.x) * 256;
    constexpr int B = 4;  // strides whose 5 x B loads are issued before any of their sums
    for (int64_t i0 = int64_t(blockIdx.x) * 256 + threadIdx.x; i0 < nvec; i0 += B * stride) {
        float4 c[B], a[B], b[B], sa[B], sb[B];
#pragma unroll
        for (int k = 0; k < B; ++k) {
            const int64_t i = i0 + k * stride;
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            const bool in = i < nvec;
            c[k] = in ? chi[i] : z;
            a[k] = in ? u[i] : z;
            b[k] = in ? v[i] : z;
            sa[k] = in ? usx[i] : z;
            sb[k] = in ? usy[i] : z;
        }
#pragma unroll
        for (int k = 0; k < B; ++k) {
            if (i0 + k * stride >= nvec) break;
            add(sx, cx, c[k].x * (a[k].x - sa[k].x) + c[k].y * (a[k].y - sa[k].y) +
                            (c[k].z * (a[k].z - sa[k].z) + c[k].w * (a[k].w - sa[k].w)));
            add(sy, cy, c[k].x * (b[k].x - sb[k].x) + c[k].y * (b[k].y - sb[k].y) +
                            (c[k].z * (b[k].z - sb[k].z) + c[k].w * (b[k].w - sb[k].w)));
        }
    }
    rs[0][threadIdx.x] = double(sx) - double(cx);
    rs[1][threadIdx.x] = double(sy) - double(cy);
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (int(threadIdx.x) < o) {
            rs[0][threadIdx.x] += rs[0][threadIdx.x + o];
            rs[1][threadIdx.x] += rs[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    penal_finish(rs, partial, counter, scale, uhx, uhy, out);
}

template <typename T>
cudaError_t launch_penal_force(const T* u, const T* v, const T* chi, const T* usx, const T* usy, int64_t ncell,
                               double scale, double uhx, double uhy, double* partial, double* out, cudaStream_t st) {
    auto al = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
    // the arrival counter sits after the partials (zeroed at plan creation, reset by the last CTA)
    unsigned* counter = reinterpret_cast<unsigned*>(partial + 2 * kPenalBlocks);
    if (sizeof(T) == 4 && ncell % 4 == 0 && al(u) && al(v) && al(chi) && al(usx) && al(usy))
        k_penal_partial4<T><<<kPenalBlocks, 256, 0, st>>>(
            reinterpret_cast<const float4*>(u), reinterpret_cast<const float4*>(v), reinterpret_cast<const float4*>(chi),
            reinterpret_cast<const float4*>(usx), reinterpret_cast<const float4*>(usy), ncell / 4, partial, counter,
            scale, uhx, uhy, out);
    else
        k_penal_partial<T><<<kPenalBlocks, 256, 0, st>>>(u, v, chi, usx, usy, ncell, partial, counter, scale, uhx,
                                                         uhy, out);
    return cudaGetLastError();
}


int penal_partial_doubles() { return 2 * kPenalBlocks + 1; }  // partials, then the arrival counter

// ------------------------------------------------------------------------------------
// Mass and centre-of-mass velocity of the body (Eqs. aPenal and aSF, Sec. 3.3): the sums
// sum chi, sum chi u, sum chi v, deterministic in the same way as the penalisation force
// (fixed grid, compensated FP32 or FP64 per thread, FP64 block trees, the last CTA sums
// the block partials in block order).  out = {rho h^2 sum chi, sum chi u / sum chi,
// sum chi v / sum chi}.
// ------------------------------------------------------------------------------------
template <typename T, bool kVec>
__global__ void __launch_bounds__(256) k_body_moments(const T* __restrict__ u, const T* __restrict__ v,
                                                      const T* __restrict__ chi, int64_t ncell,
                                                      double* __restrict__ partial, unsigned* __restrict__ counter,
                                                      double mass_scale, double* __restrict__ out) {
    __shared__ double rs[3][256];
    __shared__ bool last;
    T s[3] = {T(0), T(0), T(0)}, c[3] = {T(0), T(0), T(0)};
    auto add = [&](int k, T a) {
        if (sizeof(T) == 4) {
            const T y = a - c[k], t = s[k] + y;
            c[k] = (t - s[k]) - y;
            s[k] = t;
        } else {
            s[k] += a;
        }
    };
    const int64_t stride = int64_t(gridDim.x) * 256;
    if constexpr (kVec) {  // FP32, 16-byte aligned, ncell a multiple of 4
        const float4* u4 = reinterpret_cast<const float4*>(u);
        const float4* v4 = reinterpret_cast<const float4*>(v);
        const float4* c4 = reinterpret_cast<const float4*>(chi);
        for (int64_t i = int64_t(blockIdx.x) * 256 + threadIdx.x; i < ncell / 4; i += stride) {
            const float4 a = c4[i], b = u4[i], d = v4[i];
            add(0, T((a.x + a.y) + (a.z + a.w)));
            add(1, T((a.x * b.x + a.y * b.y) + (a.z * b.z + a.w * b.w)));
            add(2, T((a.x * d.x + a.y * d.y) + (a.z * d.z + a.w * d.w)));
        }
    } else {
        for (int64_t i = int64_t(blockIdx.x) * 256 + threadIdx.x; i < ncell; i += stride) {
            const T a = chi[i];
            add(0, a);
            add(1, a * u[i]);
            add(2, a * v[i]);
        }
    }
    for (int k = 0; k < 3; ++k) rs[k][threadIdx.x] = double(s[k]) - double(c[k]);
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (int(threadIdx.x) < o)
            for (int k = 0; k < 3; ++k) rs[k][threadIdx.x] += rs[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int k = 0; k < 3; ++k) partial[3 * blockIdx.x + k] = rs[k][0];
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double a[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < int(gridDim.x); b += blockDim.x)
        for (int k = 0; k < 3; ++k) a[k] += __ldcg(partial + 3 * b + k);
    for (int k = 0; k < 3; ++k) rs[k][threadIdx.x] = a[k];
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (int(threadIdx.x) < o)
            for (int k = 0; k < 3; ++k) rs[k][threadIdx.x] += rs[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = mass_scale * rs[0][0];
        out[1] = rs[1][0] / rs[0][0];
        out[2] = rs[2][0] / rs[0][0];
        *counter = 0u;
    }
}

int moments_partial_doubles() { return 3 * kPenalBlocks + 1; }  // partials, then the arrival counter

template <typename T>
cudaError_t launch_body_moments(const T* u, const T* v, const T* chi, int64_t ncell, double mass_scale,
                                double* partial, double* out, cudaStream_t st) {
    auto al = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
    unsigned* counter = reinterpret_cast<unsigned*>(partial + 3 * kPenalBlocks);
    if (sizeof(T) == 4 && ncell % 4 == 0 && al(u) && al(v) && al(chi))
        k_body_moments<T, true><<<kPenalBlocks, 256, 0, st>>>(u, v, chi, ncell, partial, counter, mass_scale, out);
    else
        k_body_moments<T, false><<<kPenalBlocks, 256, 0, st>>>(u, v, chi, ncell, partial, counter, mass_scale, out);
    return cudaGetLastError();
}

template cudaError_t launch_body_moments<float>(const float*, const float*, const float*, int64_t, double, double*,
                                                double*, cudaStream_t);
template cudaError_t launch_body_moments<double>(const double*, const double*, const double*, int64_t, double,
                                                 double*, double*, cudaStream_t);

template cudaError_t launch_penal_force<float>(const float*, const float*, const float*, const float*, const float*,
                                              int64_t, double, double, double, double*, double*, cudaStream_t);
template cudaError_t launch_penal_force<double>(const double*, const double*, const double*, const double*,
                                               const double*, int64_t, double, double, double, double*, double*,
                                               cudaStream_t);

}  // namespace pp
