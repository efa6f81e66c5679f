// Surface tractions and force integrals without any device allocation.
//
// The plan-based pp_surface_traction keeps its per-block partial force sums in
// plan-owned device memory.  Some callers cannot allocate: a flow solver that
// reserves the whole device up front and hands out no further memory, or a
// real-time loop that must not pay cudaMalloc's implicit device synchronisation.
// pp_surface_forces_noalloc runs the same traction and reduction kernels with
// that scratch placed in a fixed file-scope device array instead.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/pp.h"
#include "pp_kernels.cuh"

namespace {

constexpr int kMaxPoints = 1 << 20;                                        // PP_NOALLOC_MAX_POINTS
constexpr int kMaxBlocks = (kMaxPoints + pp::kSurfaceBlock - 1) / pp::kSurfaceBlock;
constexpr int kScratchDoubles = 4 * kMaxBlocks + 8;                        // partial sums + forces
static_assert(kMaxPoints == PP_NOALLOC_MAX_POINTS, "scratch sized for the documented point limit");
static_assert(kScratchDoubles * sizeof(double) == PP_NOALLOC_SCRATCH_BYTES,
              "the header's scratch size must follow the traction kernel's block size");

// Shared by every call on a device and kept until the process exits
// (4 partial sums per 64-point block of the largest request, plus the forces: 512 KB).
static __device__ __align__(256) double g_forces_scratch[kScratchDoubles];

// Device address of the scratch array in the current context.  Host code cannot use the
// symbol itself: on the host it names a stand-in, not device memory.  The lookup is made on
// every call (it allocates nothing): a cached address would go stale if the context were
// destroyed and the module loaded again at another address.
int scratch_address(double** out) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_forces_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return PP_ERR_CUDA;
    }
    *out = static_cast<double*>(p);
    return PP_OK;
}

bool device_pointer(const void* ptr) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <typename T>
int run(pp_grid grid, double h, const void* u, const void* v, int npts, const double* points,
        const double* normals, const double* dS, const double* P_points, double rho, double nu, double lift,
        int interp, double uhx, double uhy, double* per_point, double* forces, cudaStream_t st) {
    double* scratch = nullptr;
    int s = scratch_address(&scratch);
    if (s != PP_OK) return s;
    pp::Tree<T> t = {};
    t.n = grid.n;
    t.h = h;
    t.x0 = grid.x0;
    t.y0 = grid.y0;
    const bool dev_forces = forces && device_pointer(forces);
    pp::SurfaceArgs a = {};
    a.npts = npts;
    a.pts = points;
    a.nrm = normals;
    a.dS = dS;
    a.Psurf = const_cast<double*>(P_points);  // read only by the traction kernel
    a.per_point = per_point;
    a.partial = scratch;                       // every slot read is written first: no clearing needed
    a.forces = dev_forces ? forces : scratch + 4 * kMaxBlocks;
    a.lift = lift < 0 ? 2.0 * h : lift;
    a.mu2 = 2.0 * rho * nu;
    a.uhat_x = uhx;
    a.uhat_y = uhy;
    a.interp = interp;
    const int nb = (npts + pp::kSurfaceBlock - 1) / pp::kSurfaceBlock;
    pp::k_traction<T><<<nb, pp::kSurfaceBlock, 0, st>>>(t, static_cast<const T*>(u), static_cast<const T*>(v), a);
    if (cudaGetLastError() != cudaSuccess) return PP_ERR_CUDA;
    pp::k_forces_final<T><<<1, 256, 0, st>>>(nb, a);
    if (cudaGetLastError() != cudaSuccess) return PP_ERR_CUDA;
    if (forces && !dev_forces) {
        if (cudaMemcpyAsync(forces, a.forces, 6 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return PP_ERR_CUDA;
    }
    return PP_OK;
}

}  // namespace

extern "C" int pp_surface_forces_noalloc(int precision, pp_grid grid, double h, const void* u, const void* v,
                                         int npts, const double* points, const double* normals,
                                         const double* dS, const double* P_points, double rho, double nu,
                                         double lift, int interp, double uinf_x, double uinf_y,
                                         double* per_point, double* forces, void* stream) {
    const int n = grid.n;
    if (n < 8 || n > 16384 || (n & (n - 1)) != 0 || !(h > 0.0) || !std::isfinite(h)) return PP_ERR_ARG;
    if (precision != PP_FP64 && precision != PP_MIXED) return PP_ERR_ARG;
    if (interp != PP_NEAREST && interp != PP_BILINEAR) return PP_ERR_ARG;
    if (!u || !v || !points || !normals || !P_points) return PP_ERR_ARG;
    if (npts < 1 || npts > kMaxPoints) return PP_ERR_ARG;
    const double un = std::hypot(uinf_x, uinf_y);
    if (!(un > 0.0) || !std::isfinite(un) || !std::isfinite(rho) || !std::isfinite(nu) || !std::isfinite(lift))
        return PP_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return precision == PP_FP64
               ? run<double>(grid, h, u, v, npts, points, normals, dS, P_points, rho, nu, lift, interp,
                             uinf_x / un, uinf_y / un, per_point, forces, st)
               : run<float>(grid, h, u, v, npts, points, normals, dS, P_points, rho, nu, lift, interp,
                            uinf_x / un, uinf_y / un, per_point, forces, st);
}
