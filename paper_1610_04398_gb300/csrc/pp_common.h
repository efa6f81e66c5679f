// Shared declarations of the pressure-recovery path: device data layout,
// kernel-launch entry points (one instantiation per precision) and helpers.
//
// Notation (Appendix A of the paper): the potential handled internally is
// Phi = 2 pi P = sum_s q_s log|x - x_s|, q = f h^2.  A box of side s centred at
// z_c carries the multipole of Eq. pressTruncated,
//   Phi(z) = S log|z - z_c| - Re sum_k alpha_k (z - z_c)^-k,
// stored scaled as M[0] = S, M[k] = alpha_k / s^k, and a local (Taylor) expansion
//   Phi(z) = Re sum_l b_l (z - z_c)^l,  stored as L[l] = b_l s^l.
// The FP64 monopole S and the FP64 constant term Re b_0 of every box are kept in
// separate double arrays in both precisions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pp {

// Largest supported expansion order (coefficients 0..kMaxOrder).
constexpr int kMaxOrder = 40;
constexpr int kMaxP1 = kMaxOrder + 1;

// Boxes of all levels 0..l-1 precede level l in the coefficient arrays.
__host__ __device__ inline int64_t level_offset(int l) {
    return ((int64_t(1) << (2 * l)) - 1) / 3;
}

template <typename T> struct cplx_of;
template <> struct cplx_of<float> { typedef float2 type; };
template <> struct cplx_of<double> { typedef double2 type; };

// One interaction-list entry: the index of its translation operator and the source box,
// either the same-level box at offset (dx, dy) (pad == 0) or the parent-level box at
// offset (dx, dy) from the target's parent (pad == 1).
struct M2LEntry {
    int dx, dy, op, pad;
};

// Device-resident data of one plan, shared by all kernels of one precision.
template <typename T>
struct Tree {
    typedef typename cplx_of<T>::type C;
    int n;          // cells per side
    int nL;         // leaves per side (n / 8)
    int Lleaf;      // leaf level, nL = 2^Lleaf
    int P1;         // order + 1 coefficients
    double h, x0, y0;
    double lnh;     // log h, formed on the host (FP64 log is a long software sequence on the GPU)
    double inv_h;   // 1 / h, likewise
    T* q;           // source weights q = f h^2, leaf-major: leaf (LY * nL + LX) * 64 + cy * 8 + cx
    C* mp;          // multipoles, all levels: (level_offset(l) + box) * P1 + k
    double* S;      // FP64 monopole per box (same box indexing)
    C* loc;         // locals, same indexing as mp (levels >= 2 used)
    unsigned* mmax; // mixed plans with tensor-core translations: largest |coefficient| of the
                    // multipoles (FP32 bits), raised by the upward pass, cleared by the downward
    double* L0;     // FP64 constant term Re b_0 per box
    // constant tables (built on the host in FP64, stored in T)
    const C* Wp2m;  // [64][P1]: omega_c^k / k (k >= 1), omega_c = cell offset from leaf centre / 8
    const C* Vl2p;  // [64][P1]: omega_c^l
    const C* Am2m;  // [4][j][k]: child quadrant -> parent, beta_k = sum_j A[q][j][k] M_j
    const C* Cl2l;  // [4][k][l]: parent -> child quadrant, c_l = sum_k C[q][k][l] b_k
    const C* Bm2l;  // [op][k][l]: same-level multipole-to-local operator for one offset
    const C* Tpow;  // [op][k]: (r / tau)^k, source-side diagonal of operator op (factored M2L)
    const C* TpowL; // [op][k]: tau^-k, target-side diagonal of operator op
    const C* Zq;    // [4][k]: zeta_q^k, zeta_q = child centre - parent centre in parent sides
    const C* Ziq;   // [4][k]: (2 zeta_q)^-k
    const double* lnTau;   // [op]: log|tau| for the offset of operator op
    const M2LEntry* il;    // [4][il_stride] interaction lists per child position
    int il_count[4];
    int il_stride;
    const T* Ktab;         // [(2 Rk + 1)^2]: log max(h |Delta|, rho_h) for integer cell offsets
    const T* Krel;         // same offsets, log max(|Delta|, rho_h / h) = Ktab - log h (split solve: the
                           // log h part is added exactly from the near leaves' monopoles)
    int Rk;                // largest |Delta| component in the near field (8 Dmax + 7)
    const int2* near;      // theta-near leaf offsets
    int n_near;
    int Dmax;              // largest |dx|, |dy| in the near list
    unsigned long long near_mask;  // bit (dy + Dmax) * (2 Dmax + 1) + (dx + Dmax) set for near offsets (Dmax <= 3)
    int64_t resident_threads;      // threads the device keeps resident for the translation kernels
    int near_tile;                 // mixed near field: 8 or 16 targets per thread
    unsigned* up_counter;          // arrival counter of the one-launch upward pass (mixed plans), zeroed
    C* locA;                       // mixed plans, leaf level >= 5: multipole-to-local parts of the locals
    double* L0A;                   // of levels 2..L-4 (box indexing of loc/L0), else null
    float2* Sf;                    // mixed plans: S per box as a double-float pair (hi, lo), else null
    const float2* lnTauF;          // mixed plans: log|tau| per operator as a double-float pair, else null
};

// ------------------------------------------------------------------------------------
// Double-float arithmetic: a value hi + lo held in two floats (|lo| <= ulp(hi) / 2), about
// 48 significant bits, on the FP32 pipe.  The FP64 constant-term sums of the translations
// use it: an FP64 instruction costs a warp some 20 cycles of its SM's narrow FP64 pipe
// (about 1/64 of the FP32 rate), whatever its number of active lanes.  Error-free sum
// (Knuth's two-sum) and product (by a fused multiply-add).
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void df_add(float& hi, float& lo, float bh, float bl) {
    const float s = hi + bh;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (bh - bb);
    lo = lo + (err + bl);
    hi = s;
}
// (hi, lo) += (ah + al) (bh + bl), dropping al bl
__device__ __forceinline__ void df_fma(float& hi, float& lo, float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    const float e = fmaf(ah, bh, -p) + (ah * bl + al * bh);
    df_add(hi, lo, p, e);
}
__device__ __forceinline__ float2 df_from(double d) {
    const float h = float(d);
    return make_float2(h, float(d - double(h)));
}
__device__ __forceinline__ double df_to(float hi, float lo) { return double(hi) + double(lo); }

// Monopole of a box: FP64, and in mixed plans also as a double-float pair for the
// translation kernels that keep their constant-term sums on the FP32 pipe.
template <typename T>
__device__ __forceinline__ void store_S(const Tree<T>& t, int64_t i, double S) {
    t.S[i] = S;
    if (sizeof(T) == 4 && t.Sf) {
        const float h = float(S);
        t.Sf[i] = make_float2(h, float(S - double(h)));
    }
}
// Leaf monopoles are FP32 sums: the pair is exact with lo = 0.
template <typename T>
__device__ __forceinline__ void store_S_leaf(const Tree<T>& t, int64_t i, T S) {
    t.S[i] = double(S);
    if (sizeof(T) == 4 && t.Sf) t.Sf[i] = make_float2(float(S), 0.f);
}

// Tensor map (opaque 128-byte CUtensorMap object) of the tensor-core near field: the FP32
// source weights q (leaf-major) viewed as {64 cells, nL leaf columns, nL leaf rows}, with the
// box of one CTA's halo.
struct NearTcMaps {
    alignas(64) unsigned char q[128];
};

// Mixed plans with register-kernel orders run the downward levels 2..lt (lt <= 5, never
// the leaf level when it evaluates into an output) as one chain launch; 0 when that does
// not apply.
template <typename T>
int chain_top(const Tree<T>& t, int l0, int l1, bool leaf_out) {
    const bool fast = t.P1 == 13 || t.P1 == 17 || t.P1 == 21 || t.P1 == 25;
    if (sizeof(T) != 4 || !fast || l0 != 2) return 0;
    int lt = l1 < 5 ? l1 : 5;
    if (leaf_out && lt == t.Lleaf) --lt;
    return lt >= 3 ? lt : 0;
}

// Kernel launches of launch_downward_levels(t, l0, l1, ...).
template <typename T>
int downward_level_launches(const Tree<T>& t, int l0, int l1, bool leaf_out) {
    if (l1 < l0) return 0;
    const int lt = chain_top<T>(t, l0, l1, leaf_out);
    return lt > 0 ? 1 + (l1 - lt) : l1 - l0 + 1;
}

size_t near_tc_smem_bytes(int D);
bool near_tc_ok(int nL, int D);
// Bytes of the split FP16 kernel matrices K_o of n_near offsets, and their host-side values.
size_t near_tc_kmat_bytes(int n_near);
void near_tc_fill_kmat(const int2* offs, int n_near, double rh_over_h, void* out);
cudaError_t launch_near_tc(const NearTcMaps& maps, const float* q, const void* kmat, const int2* near, int n_near, int D, int n,
                           float* p_out, int* err, cudaStream_t st);
cudaError_t prepare_near_tc();
// Multipole-to-local translations on the tensor cores (mixed plans, p = 12): every operator
// as a dense split-FP16 matrix, built on the host from the operators' offsets and side
// ratios (op_geo: [op][tau_x, tau_y, ratio]) together with each child position's list of
// window entries; then one persistent launch over every level (in place of k_m2l_far).
// m2l_tc_margin: the halo margin (in boxes) the lists need, or -1 when they need more
// than the kernel holds.
int m2l_tc_margin(const M2LEntry* il, const int* il_count, int il_stride);
bool m2l_tc_ok(int P1, int margin, int il_stride);
size_t m2l_tc_table_bytes(int n_ops, int il_stride);
// fills the tables (operators, then the entries) and returns 1 / the operators' scale
float m2l_tc_fill_tables(const double* op_geo, int n_ops, const M2LEntry* il, const int* il_count, int il_stride,
                         int margin, void* out);
int64_t m2l_tc_tiles(int Lleaf);
cudaError_t launch_m2l_tc(const Tree<float>& t, const void* tables, int n_ops, int il_stride, int margin, float inv_sb,
                          unsigned* claim, int sms, int* err, cudaStream_t st);
cudaError_t prepare_m2l_tc();

struct SurfaceArgs {
    int npts;
    const double* pts;
    const double* nrm;
    const double* dS;      // may be null: trapezoid weights
    double* Psurf;         // [npts] pressure at the points (FP64)
    double* per_point;     // [npts][5] or null
    double* partial;       // [blocks][4]
    double* forces;        // [6] device
    double lift, mu2, uhat_x, uhat_y, theta, rho_h;
    int interp;
    int* err;              // device error flag (tree-code list overflow)
};

template <typename T>
cudaError_t launch_rhs_p2m(const Tree<T>& t, const T* u, const T* v, const T* chi, const T* usx,
                           const T* usy, double rho, double lam, T* f_out, cudaStream_t st, int* launches);
template <typename T>
cudaError_t launch_upward(const Tree<T>& t, cudaStream_t st);
// Penalisation force sums (Eq. dragPenal): out = {Fx, Fy, drag, lift} with F = scale * sum
// chi (u - u_s); partial holds 2 doubles per reduction block and the blocks' arrival counter
// (penal_partial_doubles(), zeroed once before the first call).
template <typename T>
cudaError_t launch_penal_force(const T* u, const T* v, const T* chi, const T* usx, const T* usy, int64_t ncell,
                               double scale, double uhx, double uhy, double* partial, double* out, cudaStream_t st);
int penal_partial_doubles();
// Mass rho h^2 sum chi and centre-of-mass velocity of the body marked by chi (Eqs. aPenal,
// aSF); partial holds 3 doubles per block and the arrival counter (moments_partial_doubles(),
// zeroed once); out = {M, u_CM_x, u_CM_y}.
template <typename T>
cudaError_t launch_body_moments(const T* u, const T* v, const T* chi, int64_t ncell, double mass_scale,
                                double* partial, double* out, cudaStream_t st);
int moments_partial_doubles();
// Zero-padded FFT (Hockney) solve of the same discrete sum on the whole grid: sizes it supports,
// its per-plan buffers (the half-spectrum work array and the transformed kernel), the
// one-time FP64 formation of the transformed kernel, and one solve q -> p_out.
bool fft_size_ok(int n, bool fp64);
size_t fft_work_bytes(int n, bool fp64);
size_t fft_spectrum_bytes(int n, bool fp64);
int fft_launches_per_solve();
cudaError_t fft_prepare_spectrum(int n, double h, double rh, bool fp64, void* Kp, cudaStream_t st);
template <typename R>
cudaError_t launch_fft_solve(const R* q, int n, int nL, const void* Kp, void* H, R* p_out, cudaStream_t st);
// Kernel launches one launch_upward issues.
template <typename T>
int upward_launches(const Tree<T>& t);
template <typename T>
cudaError_t launch_downward(const Tree<T>& t, cudaStream_t st);
template <typename T>
cudaError_t launch_leaf_eval(const Tree<T>& t, T* p_out, cudaStream_t st);
template <typename T>
cudaError_t launch_downward_levels(const Tree<T>& t, int l0, int l1, T* p_out, cudaStream_t st);
// Local evaluation of the leaf locals, added to p_out (mixed plans whose leaf-level
// translations ran without it); leaf_l2p_ok says whether it applies.
template <typename T>
bool leaf_l2p_ok(const Tree<T>& t, const void* p_out);
template <typename T>
cudaError_t launch_leaf_l2p(const Tree<T>& t, T* p_out, cudaStream_t st);
// Two-launch downward pass of the split solve: every level's multipole-to-local part in one
// launch (beside the near field), then the local-to-local shifts and the evaluation per
// subtree (after it).  down_tree_ok says whether it applies.
template <typename T>
bool down_tree_ok(const Tree<T>& t, const void* p_out);
template <typename T>
cudaError_t launch_m2l_far(const Tree<T>& t, cudaStream_t st);
template <typename T>
cudaError_t launch_down_tree(const Tree<T>& t, T* p_out, cudaStream_t st);
template <typename T>
bool split_solve_ok(const Tree<T>& t);
template <typename T>
cudaError_t launch_near_only(const Tree<T>& t, T* p_out, cudaStream_t st);
template <typename T>
cudaError_t launch_surface(const Tree<T>& t, const T* u, const T* v, const SurfaceArgs& a,
                           cudaStream_t st);
template <typename T>
cudaError_t launch_export_expansion(const Tree<T>& t, int kind, int level, double* dst,
                                    cudaStream_t st);

constexpr int kSurfaceBlock = 64;
// Surface scratch of a plan: a new plan holds it for kInitialSurfaceCap points and grows it
// to surface_cap_after(cap, npts) points when a call brings more; surface_scratch_bytes is
// what `cap` points take (the pressure per point and 4 partial sums per block).
constexpr int kInitialSurfaceCap = 4096;
int64_t surface_scratch_bytes(int cap);
int surface_cap_after(int cap, int npts);
constexpr int kDynSmemLimit = 200 * 1024;  // dynamic shared memory any launch may use

template <typename T>
cudaError_t prepare_kernels();
template <typename T>
size_t plan_smem_bytes(const Tree<T>& t);

}  // namespace pp
