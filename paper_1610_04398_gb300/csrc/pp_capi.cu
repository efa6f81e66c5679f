// C ABI of the pressure-recovery library: plan creation (tables built on the host
// in FP64), argument validation, call-order state and dispatch to the FP64 or the
// mixed-precision kernels.  Every entry point returns a pp_status.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <set>
#include <utility>
#include <vector>

#include "../../include/pp.h"
#include "pp_common.h"

using cd = std::complex<double>;

namespace pp {

int64_t surface_scratch_bytes(int cap) {
    const int64_t nb = (int64_t(cap) + kSurfaceBlock - 1) / kSurfaceBlock;
    return int64_t(sizeof(double)) * cap + int64_t(sizeof(double)) * 4 * nb;
}

int surface_cap_after(int cap, int npts) {
    if (npts <= cap) return cap;
    const int64_t grown = std::max<int64_t>(npts, 2 * int64_t(cap));
    return int(std::min<int64_t>(grown, int64_t(1) << 24));
}

}  // namespace pp

namespace {

constexpr double kC0 = 0.78539816339744830962 - 1.5 - 0.34657359027997265471;  // pi/4 - 3/2 - ln2/2

double binom(int n, int k) {
    if (k < 0 || k > n) return 0.0;
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * double(n - k + i) / double(i);
    return r;
}

// Same-level offsets (dx, dy) that are NOT well separated: theta^2 |d|^2 <= 2,
// i.e. r_A + r_B = sqrt(2) s >= theta |d| s (the tie at equality counts as near).
std::vector<std::pair<int, int>> near_offsets(double theta) {
    std::vector<std::pair<int, int>> out;
    const int R = int(std::ceil(std::sqrt(2.0) / theta)) + 1;
    for (int dy = -R; dy <= R; ++dy)
        for (int dx = -R; dx <= R; ++dx)
            if (theta * theta * double(dx * dx + dy * dy) <= 2.0) out.emplace_back(dx, dy);
    return out;
}

bool is_near(double theta, int dx, int dy) { return theta * theta * double(dx * dx + dy * dy) <= 2.0; }

// Interaction list of a box at child position c: children of the parent's near
// boxes that are themselves well separated from the box.
std::vector<std::pair<int, int>> m2l_offsets(double theta, int c) {
    std::vector<std::pair<int, int>> out;
    const int cx = c & 1, cy = c >> 1;
    for (auto& D : near_offsets(theta))
        for (int cp = 0; cp < 4; ++cp) {
            const int tx = 2 * D.first + (cp & 1) - cx;
            const int ty = 2 * D.second + (cp >> 1) - cy;
            if (!is_near(theta, tx, ty)) out.emplace_back(tx, ty);
        }
    return out;
}

// Interaction list entries of a box at child position c: (dx, dy, kind).  kind 0: a box of
// the same level at offset (dx, dy).  kind 1: the parent-level box at offset (dx, dy) from
// the target's parent, used in place of its four children when all four are well
// separated from the target and the parent itself passes the acceptance test for boxes
// of unequal size, r_target + r_parent < theta d  (in target-box units: (3/2) sqrt(2) <
// theta |2D + 1/2 - c|; equality counts as not separated).
struct Entry {
    int dx, dy, kind;
};

std::vector<Entry> m2l_entries(double theta, int c) {
    std::vector<Entry> out;
    const int cx = c & 1, cy = c >> 1;
    for (auto& D : near_offsets(theta)) {
        int nsep = 0;
        for (int cp = 0; cp < 4; ++cp)
            nsep += !is_near(theta, 2 * D.first + (cp & 1) - cx, 2 * D.second + (cp >> 1) - cy);
        const double ox = 2.0 * D.first + 0.5 - cx, oy = 2.0 * D.second + 0.5 - cy;
        if (nsep == 4 && theta * theta * (ox * ox + oy * oy) > 4.5) {
            out.push_back(Entry{D.first, D.second, 1});
            continue;
        }
        for (int cp = 0; cp < 4; ++cp) {
            const int tx = 2 * D.first + (cp & 1) - cx, ty = 2 * D.second + (cp >> 1) - cy;
            if (!is_near(theta, tx, ty)) out.push_back(Entry{tx, ty, 0});
        }
    }
    return out;
}

template <typename T>
struct Buf {
    T* p = nullptr;
    size_t n = 0;
};

}  // namespace

struct pp_plan_s {
    int n = 0, nL = 0, Lleaf = 0, order = 0, P1 = 0, precision = PP_FP64, interp = PP_NEAREST, near_tile = 16;
    double h = 0, x0 = 0, y0 = 0, theta = 0, rho = 1, lift = 0, uhx = 1, uhy = 0;
    double theta_surf = 0;  // acceptance parameter of the surface tree-code
    cudaStream_t stream = nullptr;
    int device = 0;
    bool dead = false, have_q = false, have_up = false;
    void* near_forked = nullptr;  // output whose near field is already on the side stream
    // device memory
    std::vector<void*> allocs;
    void* q = nullptr;
    void* mp = nullptr;
    void* loc = nullptr;
    double* S = nullptr;
    double* L0 = nullptr;
    void* tabs = nullptr;  // W, V, A, C, B tables of the plan's precision
    double* lnTau = nullptr;
    float2* lnTauF = nullptr;  // mixed plans: log|tau| as double-float pairs
    float2* Sf = nullptr;      // mixed plans: box monopoles as double-float pairs
    pp::M2LEntry* il = nullptr;
    void* Ktab = nullptr;
    void* Krel = nullptr;
    int2* near = nullptr;
    int n_near = 0, Dmax = 0, Rk = 0, il_stride = 0, il_count[4] = {0, 0, 0, 0}, n_ops = 0;
    unsigned long long near_mask = 0;
    size_t off_W = 0, off_V = 0, off_A = 0, off_C = 0, off_B = 0;  // element offsets in tabs
    size_t off_T = 0, off_TL = 0, off_Z = 0, off_ZI = 0;
    // surface scratch
    int surf_cap = 0;
    double* Psurf = nullptr;
    double* partial = nullptr;
    double* forces_dev = nullptr;
    double* penal_buf = nullptr;  // penalisation force: block partials, then 4 results
    double* moments_buf = nullptr;  // body moments: block partials and counter, then 3 results
    unsigned* up_counter = nullptr;  // arrival counter of the one-launch upward pass
    void* locA = nullptr;            // two-launch downward pass: M2L parts of levels 2..L-4
    double* L0A = nullptr;
    // zero-padded FFT solve: half-spectrum work array and transformed kernel (first call)
    void* fft_H = nullptr;
    void* fft_Kp = nullptr;
    int* err = nullptr;
    int64_t resident_threads = 0;
    int prio_hi = 0;
    // tensor-core near field (mixed precision, tile 128)
    bool use_tc = false;
    // tensor-core translations (mixed plans, option m2l_tensor)
    bool use_m2l_tc = false;
    void* m2l_tab = nullptr;       // split FP16 operators, then the window entries per child position
    int m2l_margin = -1;
    float m2l_inv_sb = 1.f;
    int sms = 0;
    std::vector<double> op_geo;            // [op][tau_x, tau_y, side ratio]
    std::vector<pp::M2LEntry> il_host;     // the interaction lists as uploaded
    void* ktc = nullptr;
    pp::NearTcMaps tc_maps;
    int64_t workspace = 0;
    int64_t near_pairs = 0, m2l_pairs = 0;
    int64_t launches = 0;
    int64_t m2l_pairs_leaf = 0;
    // stage timing
    bool timing = false;
    cudaEvent_t ev[2 * 6] = {};
    bool ran[6] = {false, false, false, false, false, false};
    // concurrency inside a step: near field and surface path on side streams
    cudaStream_t aux = nullptr, aux2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_up = nullptr, ev_surf = nullptr;
};

namespace {

void release_sync(pp_plan p) {
    for (cudaEvent_t* e : {&p->ev_fork, &p->ev_join, &p->ev_up, &p->ev_surf})
        if (*e) {
            cudaEventDestroy(*e);
            *e = nullptr;
        }
    for (cudaStream_t* s : {&p->aux, &p->aux2})
        if (*s) {
            cudaStreamDestroy(*s);
            *s = nullptr;
        }
}

int cuda_fail(pp_plan p) {
    if (p) p->dead = true;
    return PP_ERR_CUDA;
}

cudaError_t dalloc(pp_plan p, void** ptr, size_t bytes) {
    *ptr = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e == cudaSuccess) {
        p->allocs.push_back(*ptr);
        p->workspace += int64_t(bytes);
    }
    return e;
}

void free_all(pp_plan p) {
    for (void* a : p->allocs) cudaFree(a);
    p->allocs.clear();
}

template <typename T>
pp::Tree<T> make_tree(const pp_plan p) {
    typedef typename pp::cplx_of<T>::type C;
    pp::Tree<T> t = {};
    t.n = p->n;
    t.nL = p->nL;
    t.Lleaf = p->Lleaf;
    t.P1 = p->P1;
    t.h = p->h;
    t.lnh = std::log(p->h);
    t.inv_h = 1.0 / p->h;
    t.x0 = p->x0;
    t.y0 = p->y0;
    t.q = static_cast<T*>(p->q);
    t.mp = static_cast<C*>(p->mp);
    t.S = p->S;
    t.loc = static_cast<C*>(p->loc);
    t.L0 = p->L0;
    const C* tb = static_cast<const C*>(p->tabs);
    t.Wp2m = tb + p->off_W;
    t.Vl2p = tb + p->off_V;
    t.Am2m = tb + p->off_A;
    t.Cl2l = tb + p->off_C;
    t.Bm2l = tb + p->off_B;
    t.Tpow = tb + p->off_T;
    t.TpowL = tb + p->off_TL;
    t.Zq = tb + p->off_Z;
    t.Ziq = tb + p->off_ZI;
    t.lnTau = p->lnTau;
    t.lnTauF = p->lnTauF;
    t.Sf = p->Sf;
    t.il = p->il;
    for (int c = 0; c < 4; ++c) t.il_count[c] = p->il_count[c];
    t.il_stride = p->il_stride;
    t.Ktab = static_cast<const T*>(p->Ktab);
    t.Krel = static_cast<const T*>(p->Krel);
    t.Rk = p->Rk;
    t.near = p->near;
    t.n_near = p->n_near;
    t.Dmax = p->Dmax;
    t.near_mask = p->near_mask;
    t.resident_threads = p->resident_threads;
    t.near_tile = p->near_tile;
    t.up_counter = p->up_counter;
    t.mmax = p->use_m2l_tc ? p->up_counter + 1 : nullptr;  // [0] upward pass, [1] maximum, [2..3] tile counter
    t.locA = static_cast<C*>(p->locA);
    t.L0A = p->L0A;
    return t;
}

// Build every constant table in FP64 and upload it in the plan's precision.
template <typename T>
int upload_tables(pp_plan p) {
    const int P1 = p->P1;
    std::vector<cd> tab;
    auto omega = [](int c) { return cd((c & 7) - 3.5, (c >> 3) - 3.5) / 8.0; };
    // W: leaf P2M, omega^k / k (entry 0 = 1 for the monopole)
    p->off_W = tab.size();
    for (int c = 0; c < 64; ++c)
        for (int k = 0; k < P1; ++k) tab.push_back(k == 0 ? cd(1, 0) : std::pow(omega(c), k) / double(k));
    // V: leaf L2P, omega^l
    p->off_V = tab.size();
    for (int c = 0; c < 64; ++c)
        for (int l = 0; l < P1; ++l) tab.push_back(std::pow(omega(c), l));
    auto zeta = [](int q) { return cd(2 * (q & 1) - 1, 2 * (q >> 1) - 1) / 4.0; };
    // A: M2M from child quadrant q, [q][j][k]: beta_k = S zeta^k / k + sum_j M_j 2^-j zeta^(k-j) C(k-1, j-1)
    p->off_A = tab.size();
    for (int q = 0; q < 4; ++q)
        for (int j = 0; j < P1; ++j)
            for (int k = 0; k < P1; ++k) {
                cd a(0, 0);
                if (j == 0 && k == 0) a = 1.0;
                else if (j == 0) a = std::pow(zeta(q), k) / double(k);
                else if (j <= k) a = std::pow(0.5, j) * std::pow(zeta(q), k - j) * binom(k - 1, j - 1);
                tab.push_back(a);
            }
    // C: L2L to child quadrant q, [q][k][l]: c_l = sum_{k>=l} b_k C(k, l) zeta^(k-l) 2^-l
    p->off_C = tab.size();
    for (int q = 0; q < 4; ++q)
        for (int k = 0; k < P1; ++k)
            for (int l = 0; l < P1; ++l)
                tab.push_back(k >= l ? binom(k, l) * std::pow(zeta(q), k - l) * std::pow(0.5, l) : cd(0, 0));
    // B: M2L per distinct operator, [op][k][l].  An operator is the source-centre offset
    // tau from the target centre in target-box units (half-integer for parent-level
    // sources) and the source/target side ratio r (1 or 2): with x_k = (r / tau)^k M_k,
    // b_l = tau^-l sum_k R[l][k] x_k.
    struct Op {
        int tx2, ty2, ratio;  // 2 tau (exact integers) and the side ratio
        bool operator==(const Op& o) const { return tx2 == o.tx2 && ty2 == o.ty2 && ratio == o.ratio; }
    };
    std::vector<Op> ops;
    std::vector<std::vector<pp::M2LEntry>> lists(4);
    for (int c = 0; c < 4; ++c) {
        for (auto& en : m2l_entries(p->theta, c)) {
            Op o = en.kind == 0 ? Op{2 * en.dx, 2 * en.dy, 1}
                                : Op{4 * en.dx + 1 - 2 * (c & 1), 4 * en.dy + 1 - 2 * (c >> 1), 2};
            int id = -1;
            for (size_t i = 0; i < ops.size(); ++i)
                if (ops[i] == o) id = int(i);
            if (id < 0) {
                id = int(ops.size());
                ops.push_back(o);
            }
            lists[c].push_back(pp::M2LEntry{en.dx, en.dy, id, en.kind});
        }
    }
    p->off_B = tab.size();
    p->op_geo.clear();
    for (auto& o : ops) {
        p->op_geo.push_back(0.5 * o.tx2);
        p->op_geo.push_back(0.5 * o.ty2);
        p->op_geo.push_back(double(o.ratio));
    }
    std::vector<double> lnt;
    for (auto& o : ops) {
        const cd tau(0.5 * o.tx2, 0.5 * o.ty2);
        const double r = double(o.ratio);
        lnt.push_back(std::log(std::abs(tau)));
        for (int k = 0; k < P1; ++k)
            for (int l = 0; l < P1; ++l) {
                cd b(0, 0);
                if (k == 0 && l >= 1) b = -1.0 / (double(l) * std::pow(tau, l));
                else if (k >= 1)
                    b = ((k + 1) % 2 == 0 ? 1.0 : -1.0) * binom(l + k - 1, k - 1) * std::pow(r, k) *
                        std::pow(tau, -(l + k));
                tab.push_back(b);
            }
    }
    p->n_ops = int(ops.size());
    // factored operators: (r / tau)^k per operator, zeta_q^k and (2 zeta_q)^-k per child quadrant
    p->off_T = tab.size();
    for (auto& o : ops) {
        const cd tau(0.5 * o.tx2, 0.5 * o.ty2);
        for (int k = 0; k < P1; ++k) tab.push_back(std::pow(double(o.ratio) / tau, k));
    }
    p->off_TL = tab.size();
    for (auto& o : ops) {
        const cd tau(0.5 * o.tx2, 0.5 * o.ty2);
        for (int k = 0; k < P1; ++k) tab.push_back(std::pow(tau, -k));
    }
    p->off_Z = tab.size();
    for (int q = 0; q < 4; ++q)
        for (int k = 0; k < P1; ++k) tab.push_back(std::pow(zeta(q), k));
    p->off_ZI = tab.size();
    for (int q = 0; q < 4; ++q)
        for (int k = 0; k < P1; ++k) tab.push_back(std::pow(2.0 * zeta(q), -k));
    // K: near-field kernel log max(h |Delta|, rho_h) over integer cell offsets
    auto nearl = near_offsets(p->theta);
    p->Dmax = 0;
    for (auto& o : nearl) p->Dmax = std::max(p->Dmax, std::max(std::abs(o.first), std::abs(o.second)));
    p->Rk = 8 * p->Dmax + 7;
    p->near_mask = 0;
    if (p->Dmax <= 3)
        for (auto& o : nearl)
            p->near_mask |= 1ull << ((o.second + p->Dmax) * (2 * p->Dmax + 1) + (o.first + p->Dmax));
    const int KW = 2 * p->Rk + 1;
    const double rh = p->h * std::exp(kC0);
    std::vector<T> K(size_t(KW) * KW), Kr(size_t(KW) * KW);
    for (int dy = -p->Rk; dy <= p->Rk; ++dy)
        for (int dx = -p->Rk; dx <= p->Rk; ++dx) {
            const double r = std::sqrt(double(dx * dx + dy * dy));
            K[size_t(dy + p->Rk) * KW + dx + p->Rk] = T(std::log(std::max(p->h * r, rh)));
            Kr[size_t(dy + p->Rk) * KW + dx + p->Rk] = T(std::log(std::max(r, std::exp(kC0))));
        }

    typedef typename pp::cplx_of<T>::type C;
    std::vector<C> tabT(tab.size());
    for (size_t i = 0; i < tab.size(); ++i) {
        tabT[i].x = T(tab[i].real());
        tabT[i].y = T(tab[i].imag());
    }
    int maxl = 0;
    for (int c = 0; c < 4; ++c) maxl = std::max(maxl, int(lists[c].size()));
    p->il_stride = std::max(maxl, 1);
    std::vector<pp::M2LEntry> ilh(size_t(4) * p->il_stride, pp::M2LEntry{0, 0, 0, 0});
    for (int c = 0; c < 4; ++c) {
        p->il_count[c] = int(lists[c].size());
        for (size_t i = 0; i < lists[c].size(); ++i) ilh[size_t(c) * p->il_stride + i] = lists[c][i];
    }
    p->il_host = ilh;
    std::vector<int2> nh;
    for (auto& o : nearl) nh.push_back(make_int2(o.first, o.second));
    p->n_near = int(nh.size());

    cudaError_t e;
    if ((e = dalloc(p, &p->tabs, sizeof(C) * tabT.size())) != cudaSuccess) return PP_ERR_OOM;
    if ((e = dalloc(p, (void**)&p->lnTau, sizeof(double) * std::max<size_t>(lnt.size(), 1))) != cudaSuccess)
        return PP_ERR_OOM;
    std::vector<float2> lntf;
    if (sizeof(T) == 4) {
        for (double d : lnt) {
            const float h = float(d);
            lntf.push_back(make_float2(h, float(d - double(h))));
        }
        if (dalloc(p, (void**)&p->lnTauF, sizeof(float2) * std::max<size_t>(lntf.size(), 1)) != cudaSuccess)
            return PP_ERR_OOM;
        if (!lntf.empty() &&
            cudaMemcpy(p->lnTauF, lntf.data(), sizeof(float2) * lntf.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return PP_ERR_CUDA;
    }
    if ((e = dalloc(p, (void**)&p->il, sizeof(pp::M2LEntry) * ilh.size())) != cudaSuccess) return PP_ERR_OOM;
    if ((e = dalloc(p, &p->Ktab, sizeof(T) * K.size())) != cudaSuccess) return PP_ERR_OOM;
    if ((e = dalloc(p, &p->Krel, sizeof(T) * Kr.size())) != cudaSuccess) return PP_ERR_OOM;
    if ((e = dalloc(p, (void**)&p->near, sizeof(int2) * nh.size())) != cudaSuccess) return PP_ERR_OOM;
    if (cudaMemcpy(p->tabs, tabT.data(), sizeof(C) * tabT.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        (!lnt.empty() &&
         cudaMemcpy(p->lnTau, lnt.data(), sizeof(double) * lnt.size(), cudaMemcpyHostToDevice) != cudaSuccess) ||
        cudaMemcpy(p->il, ilh.data(), sizeof(pp::M2LEntry) * ilh.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->Ktab, K.data(), sizeof(T) * K.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->Krel, Kr.data(), sizeof(T) * Kr.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->near, nh.data(), sizeof(int2) * nh.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return PP_ERR_CUDA;

    // work counts of one full-grid solve
    p->near_pairs = 0;
    for (auto& o : nearl) {
        const int64_t ax = std::max(0, p->nL - std::abs(o.first)), ay = std::max(0, p->nL - std::abs(o.second));
        p->near_pairs += ax * ay * 64 * 64;
    }
    p->m2l_pairs = 0;
    p->m2l_pairs_leaf = 0;
    for (int l = 2; l <= p->Lleaf; ++l) {
        const int m = 1 << l;
        for (int c = 0; c < 4; ++c)
            for (auto& en : lists[c]) {
                int64_t cx = 0, cy = 0;
                if (en.pad == 0) {
                    for (int x = (c & 1); x < m; x += 2) cx += (x + en.dx >= 0 && x + en.dx < m);
                    for (int y = (c >> 1); y < m; y += 2) cy += (y + en.dy >= 0 && y + en.dy < m);
                } else {
                    for (int x = (c & 1); x < m; x += 2) cx += ((x >> 1) + en.dx >= 0 && (x >> 1) + en.dx < m / 2);
                    for (int y = (c >> 1); y < m; y += 2) cy += ((y >> 1) + en.dy >= 0 && (y >> 1) + en.dy < m / 2);
                }
                p->m2l_pairs += cx * cy;
                if (l == p->Lleaf) p->m2l_pairs_leaf += cx * cy;
            }
    }
    return PP_OK;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    if (!fn) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
        else
            cudaGetLastError();
    }
    return fn;
}

// Split kernel matrices and the tensor map of the tensor-core near field.
int setup_near_tc(pp_plan p) {
    const int nL = p->nL;
    const int nn = p->n_near;
    if (dalloc(p, &p->ktc, pp::near_tc_kmat_bytes(nn)) != cudaSuccess) return PP_ERR_OOM;
    // K_o[t][c] = log max(|8 o + c - t|, rho_h / h) (the log h part is added from the near
    // leaves' monopoles), split into FP16 hi and lo parts
    std::vector<int2> nh(nn);
    if (cudaMemcpy(nh.data(), p->near, sizeof(int2) * nn, cudaMemcpyDeviceToHost) != cudaSuccess) return PP_ERR_CUDA;
    std::vector<unsigned char> k(pp::near_tc_kmat_bytes(nn));
    pp::near_tc_fill_kmat(nh.data(), nn, std::exp(kC0), k.data());
    if (cudaMemcpy(p->ktc, k.data(), k.size(), cudaMemcpyHostToDevice) != cudaSuccess) return PP_ERR_CUDA;
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return PP_ERR_CUDA;
    const cuuint32_t estr[3] = {1, 1, 1};
    // q (leaf-major FP32) as {64 cells, nL leaf columns, nL leaf rows}; box: one CTA's halo of
    // 8 + 2D leaf columns and 16 + 2D leaf rows
    const cuuint64_t dims[3] = {64, cuuint64_t(nL), cuuint64_t(nL)};
    const cuuint64_t strides[2] = {64 * 4, cuuint64_t(nL) * 64 * 4};
    const cuuint32_t box[3] = {64, cuuint32_t(8 + 2 * p->Dmax), cuuint32_t(16 + 2 * p->Dmax)};
    if (enc(reinterpret_cast<CUtensorMap*>(p->tc_maps.q), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, p->q, dims, strides,
            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return PP_ERR_CUDA;
    p->use_tc = true;
    return PP_OK;
}

template <typename T>
int alloc_tree(pp_plan p) {
    typedef typename pp::cplx_of<T>::type C;
    const int64_t nbox = pp::level_offset(p->Lleaf + 1);
    if (dalloc(p, &p->q, sizeof(T) * size_t(p->n) * p->n) != cudaSuccess) return PP_ERR_OOM;
    if (dalloc(p, &p->mp, sizeof(C) * size_t(nbox) * p->P1) != cudaSuccess) return PP_ERR_OOM;
    if (dalloc(p, &p->loc, sizeof(C) * size_t(nbox) * p->P1) != cudaSuccess) return PP_ERR_OOM;
    if (dalloc(p, (void**)&p->S, sizeof(double) * size_t(nbox)) != cudaSuccess) return PP_ERR_OOM;
    if (dalloc(p, (void**)&p->L0, sizeof(double) * size_t(nbox)) != cudaSuccess) return PP_ERR_OOM;
    if (dalloc(p, (void**)&p->forces_dev, sizeof(double) * 8) != cudaSuccess) return PP_ERR_OOM;
    if (dalloc(p, (void**)&p->penal_buf, sizeof(double) * (pp::penal_partial_doubles() + 4)) != cudaSuccess)
        return PP_ERR_OOM;
    if (cudaMemset(p->penal_buf, 0, sizeof(double) * (pp::penal_partial_doubles() + 4)) != cudaSuccess)
        return PP_ERR_CUDA;
    if (dalloc(p, (void**)&p->moments_buf, sizeof(double) * (pp::moments_partial_doubles() + 3)) != cudaSuccess)
        return PP_ERR_OOM;
    if (cudaMemset(p->moments_buf, 0, sizeof(double) * (pp::moments_partial_doubles() + 3)) != cudaSuccess)
        return PP_ERR_CUDA;
    if (dalloc(p, (void**)&p->up_counter, sizeof(unsigned) * 4) != cudaSuccess) return PP_ERR_OOM;
    if (cudaMemset(p->up_counter, 0, sizeof(unsigned) * 4) != cudaSuccess) return PP_ERR_CUDA;
    if (dalloc(p, (void**)&p->err, sizeof(int) * 4) != cudaSuccess) return PP_ERR_OOM;
    if (cudaMemset(p->err, 0, sizeof(int) * 4) != cudaSuccess) return PP_ERR_CUDA;
    if (sizeof(T) == 4 && dalloc(p, (void**)&p->Sf, sizeof(float2) * size_t(nbox)) != cudaSuccess)
        return PP_ERR_OOM;
    if (sizeof(T) == 4 && p->Lleaf >= 5) {  // side buffers of the two-launch downward pass
        const int64_t na = pp::level_offset(p->Lleaf - 3);
        if (dalloc(p, &p->locA, sizeof(C) * size_t(na) * p->P1) != cudaSuccess) return PP_ERR_OOM;
        if (dalloc(p, (void**)&p->L0A, sizeof(double) * size_t(na)) != cudaSuccess) return PP_ERR_OOM;
    }
    if (cudaMemset(p->loc, 0, sizeof(C) * size_t(nbox) * p->P1) != cudaSuccess) return PP_ERR_CUDA;
    if (cudaMemset(p->L0, 0, sizeof(double) * size_t(nbox)) != cudaSuccess) return PP_ERR_CUDA;
    return upload_tables<T>(p);
}

// Kernel attributes are process-wide per device: set them once per device and precision.
int prepare_device(int device, int precision) {
    static std::mutex mu;
    static bool done[64][2] = {};
    if (device < 0 || device >= 64) return PP_ERR_CUDA;
    std::lock_guard<std::mutex> lk(mu);
    const int k = precision == PP_FP64 ? 0 : 1;
    if (done[device][k]) return PP_OK;
    cudaError_t e = precision == PP_FP64 ? pp::prepare_kernels<double>() : pp::prepare_kernels<float>();
    if (e == cudaSuccess && precision == PP_MIXED) e = pp::prepare_near_tc();
    if (e == cudaSuccess && precision == PP_MIXED) e = pp::prepare_m2l_tc();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PP_ERR_CUDA;
    }
    done[device][k] = true;
    return PP_OK;
}

// Device bytes pp_plan_create allocates for a plan (the same arrays alloc_tree, upload_tables
// and setup_near_tc make, each rounded up as dalloc rounds an empty request), with its surface
// scratch grown for calls of up to npts points.  The FFT buffers are not included.
int64_t plan_bytes(int n, int order, double theta, int precision, int tile, int npts, int m2l_tensor) {
    auto al = [](int64_t b) { return b == 0 ? int64_t(16) : b; };
    const int64_t sz = precision == PP_FP64 ? 8 : 4;
    const int64_t csz = 2 * sz;
    const int nL = n / 8;
    int Lleaf = 0;
    while ((1 << Lleaf) < nL) ++Lleaf;
    const int64_t P1 = order + 1;
    const int64_t nbox = pp::level_offset(Lleaf + 1);
    int64_t b = 0;
    b += al(sz * int64_t(n) * n);                                  // q
    b += 2 * al(csz * nbox * P1);                                  // multipoles, locals
    b += 2 * al(8 * nbox);                                         // S, L0
    b += al(8 * 8);                                                // forces
    b += al(8 * (int64_t(pp::penal_partial_doubles()) + 4));       // penalisation partials
    b += al(8 * (int64_t(pp::moments_partial_doubles()) + 3));     // body-moment partials
    b += al(4 * 4);                                                // upward arrival counter
    if (precision == PP_MIXED && Lleaf >= 5) {                     // downward side buffers
        const int64_t na = pp::level_offset(Lleaf - 3);
        b += al(csz * na * P1) + al(8 * na);
    }
    b += al(4 * 4);                                                // error flags
    // constant tables: leaf P2M/L2P, M2M/L2L per quadrant, one M2L operator per distinct
    // (offset, side ratio), its two diagonals, the quadrant diagonals
    int64_t n_ops = 0, il_stride = 1;
    {
        struct Op {
            int tx2, ty2, ratio;
        };
        std::vector<Op> ops;
        for (int c = 0; c < 4; ++c) {
            auto ent = m2l_entries(theta, c);
            il_stride = std::max<int64_t>(il_stride, int64_t(ent.size()));
            for (auto& en : ent) {
                Op o = en.kind == 0 ? Op{2 * en.dx, 2 * en.dy, 1}
                                    : Op{4 * en.dx + 1 - 2 * (c & 1), 4 * en.dy + 1 - 2 * (c >> 1), 2};
                bool seen = false;
                for (auto& x : ops) seen = seen || (x.tx2 == o.tx2 && x.ty2 == o.ty2 && x.ratio == o.ratio);
                if (!seen) ops.push_back(o);
            }
        }
        n_ops = int64_t(ops.size());
    }
    const int64_t ntab = 2 * 64 * P1 + 2 * 4 * P1 * P1 + n_ops * P1 * P1 + 2 * n_ops * P1 + 2 * 4 * P1;
    b += al(csz * ntab);
    b += al(8 * std::max<int64_t>(n_ops, 1));                      // log|tau|
    if (precision == PP_MIXED) b += al(8 * std::max<int64_t>(n_ops, 1)) + al(8 * nbox);  // pairs: log|tau|, S
    b += al(int64_t(sizeof(pp::M2LEntry)) * 4 * il_stride);        // interaction lists
    const auto nearl = near_offsets(theta);
    int Dmax = 0;
    for (auto& o : nearl) Dmax = std::max(Dmax, std::max(std::abs(o.first), std::abs(o.second)));
    const int64_t KW = 2 * (8 * Dmax + 7) + 1;
    b += 2 * al(sz * KW * KW);                                     // near-field kernel tables
    b += al(int64_t(sizeof(int2)) * int64_t(nearl.size()));        // near offsets
    if (precision == PP_MIXED && tile == 128 && pp::near_tc_ok(nL, Dmax) && Lleaf >= 2)
        b += al(int64_t(pp::near_tc_kmat_bytes(int(nearl.size()))));  // split K_o
    if (precision == PP_MIXED && m2l_tensor) {  // split FP16 operators and window entries
        std::vector<pp::M2LEntry> ilh(size_t(4) * il_stride, pp::M2LEntry{0, 0, 0, 0});
        int cnt[4];
        for (int c = 0; c < 4; ++c) {
            auto ent = m2l_entries(theta, c);
            cnt[c] = int(ent.size());
            for (size_t i = 0; i < ent.size(); ++i)
                ilh[size_t(c) * il_stride + i] = pp::M2LEntry{ent[i].dx, ent[i].dy, 0, ent[i].kind};
        }
        const int mg = pp::m2l_tc_margin(ilh.data(), cnt, int(il_stride));
        if (pp::m2l_tc_ok(order + 1, mg, int(il_stride)))
            b += al(int64_t(pp::m2l_tc_table_bytes(int(n_ops), int(il_stride))));
    }
    b += pp::surface_scratch_bytes(pp::surface_cap_after(pp::kInitialSurfaceCap, std::max(npts, 0)));
    return b;
}

int ensure_surface(pp_plan p, int npts) {
    if (npts <= p->surf_cap) return PP_OK;
    const int cap = pp::surface_cap_after(p->surf_cap, npts);
    // release the old buffers (stream-ordered work must not still use them)
    if (p->Psurf) {
        if (cudaStreamSynchronize(p->stream) != cudaSuccess) return PP_ERR_CUDA;
        p->workspace -= pp::surface_scratch_bytes(p->surf_cap);
        for (void* ptr : {(void*)p->Psurf, (void*)p->partial}) {
            for (size_t i = 0; i < p->allocs.size(); ++i)
                if (p->allocs[i] == ptr) {
                    cudaFree(ptr);
                    p->allocs.erase(p->allocs.begin() + long(i));
                    break;
                }
        }
    }
    const int nb = (cap + pp::kSurfaceBlock - 1) / pp::kSurfaceBlock;
    if (dalloc(p, (void**)&p->Psurf, sizeof(double) * size_t(cap)) != cudaSuccess) return PP_ERR_OOM;
    if (dalloc(p, (void**)&p->partial, sizeof(double) * 4 * size_t(nb)) != cudaSuccess) return PP_ERR_OOM;
    p->surf_cap = cap;
    return PP_OK;
}

bool is_device_pointer(const void* ptr) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

enum { ST_RHS = 0, ST_UP = 1, ST_DOWN = 2, ST_LEAF = 3, ST_LEAFM2L = 4, ST_SURF = 5, N_STAGES = 6 };

// Inside a stream capture an event record must be an explicit graph node (External),
// otherwise the capture treats it as an internal dependency and it is never timed.
void record(cudaEvent_t e, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else
        cudaEventRecord(e, st);
}

void stage_begin(pp_plan p, int s, cudaStream_t st) {
    if (p->timing) record(p->ev[2 * s], st);
}

void stage_end(pp_plan p, int s, cudaStream_t st) {
    if (p->timing) {
        record(p->ev[2 * s + 1], st);
        p->ran[s] = true;
    }
}

void stage_begin(pp_plan p, int s) { stage_begin(p, s, p->stream); }
void stage_end(pp_plan p, int s) { stage_end(p, s, p->stream); }

template <typename T>
int run_rhs(pp_plan p, const void* u, const void* v, const void* chi, const void* usx, const void* usy,
            double lam, void* f_out) {
    pp::Tree<T> t = make_tree<T>(p);
    p->near_forked = nullptr;  // new source weights: any pending near field is stale
    stage_begin(p, ST_RHS);
    int nk = 0;
    if (pp::launch_rhs_p2m<T>(t, (const T*)u, (const T*)v, (const T*)chi, (const T*)usx, (const T*)usy,
                              p->rho, lam, (T*)f_out, p->stream, &nk) != cudaSuccess)
        return cuda_fail(p);
    stage_end(p, ST_RHS);
    p->launches += nk;
    p->have_q = true;
    p->have_up = false;
    return PP_OK;
}

template <typename T>
int ensure_up(pp_plan p) {
    if (p->have_up) return PP_OK;
    pp::Tree<T> t = make_tree<T>(p);
    stage_begin(p, ST_UP);
    if (pp::launch_upward<T>(t, p->stream) != cudaSuccess) return cuda_fail(p);
    stage_end(p, ST_UP);
    p->launches += pp::upward_launches<T>(t);
    p->have_up = true;
    return PP_OK;
}

// Near field of the split solve on the side stream: it needs only q, so it may start as
// soon as the source weights exist, beside the whole expansion chain.
template <typename T>
int fork_near(pp_plan p, void* p_out) {
    pp::Tree<T> t = make_tree<T>(p);
    if (cudaEventRecord(p->ev_fork, p->stream) != cudaSuccess ||
        cudaStreamWaitEvent(p->aux, p->ev_fork, 0) != cudaSuccess)
        return cuda_fail(p);
    stage_begin(p, ST_LEAF, p->aux);
    // the tensor-core kernel stores 16-byte vectors: an output off that alignment takes the
    // FP32-core kernel
    const bool tc = p->use_tc && (reinterpret_cast<uintptr_t>(p_out) & 15) == 0;
    const cudaError_t en = tc ? pp::launch_near_tc(p->tc_maps, static_cast<const float*>(p->q), p->ktc, p->near,
                                                   p->n_near, p->Dmax, p->n,
                                                          (float*)p_out, p->err + 1, p->aux)
                                     : pp::launch_near_only<T>(t, (T*)p_out, p->aux);
    if (en != cudaSuccess) return cuda_fail(p);
    stage_end(p, ST_LEAF, p->aux);
    if (cudaEventRecord(p->ev_join, p->aux) != cudaSuccess) return cuda_fail(p);
    p->near_forked = p_out;
    return PP_OK;
}

template <typename T>
int run_solve(pp_plan p, void* p_out) {
    pp::Tree<T> t = make_tree<T>(p);
    if (p_out && pp::split_solve_ok<T>(t)) {
        if (p->near_forked != p_out) {
            const int sf = fork_near<T>(p, p_out);
            if (sf != PP_OK) return sf;
        }
        p->near_forked = nullptr;
        int st = ensure_up<T>(p);
        if (st != PP_OK) return st;
        if (pp::down_tree_ok<T>(t, p_out)) {
            // every level's translations in one launch beside the near field; the shifts
            // down the tree and the evaluation, per subtree, after it
            stage_begin(p, ST_DOWN);
            const cudaError_t ef =
                p->use_m2l_tc ? pp::launch_m2l_tc(reinterpret_cast<const pp::Tree<float>&>(t), p->m2l_tab, p->n_ops,
                                                  p->il_stride, p->m2l_margin, p->m2l_inv_sb, p->up_counter + 2,
                                                  p->sms, p->err + 2, p->stream)
                              : pp::launch_m2l_far<T>(t, p->stream);
            if (ef != cudaSuccess) return cuda_fail(p);
            stage_end(p, ST_DOWN);
            if (cudaStreamWaitEvent(p->stream, p->ev_join, 0) != cudaSuccess) return cuda_fail(p);
            stage_begin(p, ST_LEAFM2L);
            if (pp::launch_down_tree<T>(t, (T*)p_out, p->stream) != cudaSuccess) return cuda_fail(p);
            stage_end(p, ST_LEAFM2L);
            p->launches += 3;  // translations, shifts + evaluation, near field
            return PP_OK;
        }
        // With an aligned output the leaf-level translations run before the join too, beside
        // the near field; only the local evaluation waits for it.  Otherwise the leaf level
        // runs after the join with the evaluation fused in.
        const bool sep = pp::leaf_l2p_ok<T>(t, p_out);
        stage_begin(p, ST_DOWN);
        if (pp::launch_downward_levels<T>(t, 2, sep ? t.Lleaf : t.Lleaf - 1, (T*)nullptr, p->stream) !=
            cudaSuccess)
            return cuda_fail(p);
        stage_end(p, ST_DOWN);
        if (cudaStreamWaitEvent(p->stream, p->ev_join, 0) != cudaSuccess) return cuda_fail(p);
        stage_begin(p, ST_LEAFM2L);
        const cudaError_t el = sep ? pp::launch_leaf_l2p<T>(t, (T*)p_out, p->stream)
                                   : pp::launch_downward_levels<T>(t, t.Lleaf, t.Lleaf, (T*)p_out, p->stream);
        if (el != cudaSuccess) return cuda_fail(p);
        stage_end(p, ST_LEAFM2L);
        // translation levels 2..L, the evaluation (or the fused leaf level) and the near field
        p->launches += pp::downward_level_launches<T>(t, 2, sep ? t.Lleaf : t.Lleaf - 1, false) + 1 + 1;
        return PP_OK;
    }
    int st = ensure_up<T>(p);
    if (st != PP_OK) return st;
    stage_begin(p, ST_DOWN);
    if (pp::launch_downward<T>(t, p->stream) != cudaSuccess) return cuda_fail(p);
    stage_end(p, ST_DOWN);
    p->launches += pp::downward_level_launches<T>(t, 2, p->Lleaf, false);
    if (p_out) {
        stage_begin(p, ST_LEAF);
        if (pp::launch_leaf_eval<T>(t, (T*)p_out, p->stream) != cudaSuccess) return cuda_fail(p);
        stage_end(p, ST_LEAF);
        p->launches += 1;
    }
    return PP_OK;
}

// forces_on_device: 1 device memory, 0 host memory, -1 ask the runtime.
template <typename T>
int run_surface(pp_plan p, const void* u, const void* v, int npts, const double* pts, const double* nrm,
                const double* dS, double nu, double* per_point, double* forces, int forces_on_device = -1) {
    int st = ensure_up<T>(p);
    if (st != PP_OK) return st;
    if ((st = ensure_surface(p, npts)) != PP_OK) return st == PP_ERR_CUDA ? cuda_fail(p) : st;
    const bool dev_forces = forces && (forces_on_device >= 0 ? forces_on_device == 1 : is_device_pointer(forces));
    pp::SurfaceArgs a;
    a.npts = npts;
    a.pts = pts;
    a.nrm = nrm;
    a.dS = dS;
    a.Psurf = p->Psurf;
    a.per_point = per_point;
    a.partial = p->partial;
    a.forces = dev_forces ? forces : p->forces_dev;
    a.lift = p->lift < 0 ? 2.0 * p->h : p->lift;
    a.mu2 = 2.0 * p->rho * nu;
    a.uhat_x = p->uhx;
    a.uhat_y = p->uhy;
    a.theta = p->theta_surf;
    a.rho_h = p->h * std::exp(kC0);
    a.interp = p->interp;
    a.err = p->err;
    pp::Tree<T> t = make_tree<T>(p);
    stage_begin(p, ST_SURF);
    if (pp::launch_surface<T>(t, (const T*)u, (const T*)v, a, p->stream) != cudaSuccess) return cuda_fail(p);
    stage_end(p, ST_SURF);
    p->launches += 3;
    if (forces && !dev_forces) {
        int errflag = 0;
        if (cudaMemcpyAsync(forces, p->forces_dev, 6 * sizeof(double), cudaMemcpyDeviceToHost, p->stream) !=
                cudaSuccess ||
            cudaMemcpyAsync(&errflag, p->err, sizeof(int), cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
            cudaStreamSynchronize(p->stream) != cudaSuccess)
            return cuda_fail(p);
        if (errflag) return PP_ERR_STATE;
    }
    return PP_OK;
}

}  // namespace

extern "C" {

void pp_options_default(pp_options* opt) {
    if (!opt) return;
    opt->rho = 1.0;
    opt->precision = PP_FP64;
    opt->lift = -1.0;
    opt->interp = PP_NEAREST;
    opt->uinf_x = 1.0;
    opt->uinf_y = 0.0;
    opt->stream = nullptr;
    opt->tile = 16;
    opt->theta_surface = 0.0;
    opt->m2l_tensor = 0;
}

int pp_plan_create(pp_plan* out, pp_grid grid, double h, int order, double theta, const pp_options* opt) {
    if (!out) return PP_ERR_ARG;
    *out = nullptr;
    pp_options o;
    pp_options_default(&o);
    if (opt) o = *opt;
    int n = grid.n;
    if (n < 8 || n > 16384 || (n & (n - 1)) != 0) return PP_ERR_ARG;
    if (!(h > 0.0) || !std::isfinite(h)) return PP_ERR_ARG;
    if (order < 2 || order > pp::kMaxOrder) return PP_ERR_ARG;
    if (!(theta >= 0.25 && theta <= 0.95)) return PP_ERR_ARG;
    if (!std::isfinite(grid.x0) || !std::isfinite(grid.y0)) return PP_ERR_ARG;
    if (o.precision != PP_FP64 && o.precision != PP_MIXED) return PP_ERR_ARG;
    if (o.interp != PP_NEAREST && o.interp != PP_BILINEAR) return PP_ERR_ARG;
    if (o.tile != 8 && o.tile != 16 && o.tile != 128) return PP_ERR_ARG;
    if (o.theta_surface != 0.0 && !(o.theta_surface >= 0.25 && o.theta_surface <= 0.95)) return PP_ERR_ARG;
    if (o.m2l_tensor != 0 && o.m2l_tensor != 1) return PP_ERR_ARG;
    const double un = std::hypot(o.uinf_x, o.uinf_y);
    if (!(un > 0.0) || !std::isfinite(un) || !std::isfinite(o.rho) || !std::isfinite(o.lift)) return PP_ERR_ARG;

    pp_plan p = new (std::nothrow) pp_plan_s();
    if (!p) return PP_ERR_OOM;
    p->n = n;
    p->nL = n / 8;
    p->Lleaf = 0;
    while ((1 << p->Lleaf) < p->nL) ++p->Lleaf;
    p->order = order;
    p->P1 = order + 1;
    p->precision = o.precision;
    p->interp = o.interp;
    p->near_tile = o.tile;
    p->h = h;
    p->x0 = grid.x0;
    p->y0 = grid.y0;
    p->theta = theta;
    p->theta_surf = o.theta_surface != 0.0 ? o.theta_surface : std::min(theta, 0.6);
    p->rho = o.rho;
    p->lift = o.lift;
    p->uhx = o.uinf_x / un;
    p->uhy = o.uinf_y / un;
    p->stream = static_cast<cudaStream_t>(o.stream);
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete p;
        return PP_ERR_CUDA;
    }
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess || nsm <= 0) {
        delete p;
        return PP_ERR_CUDA;
    }
    p->resident_threads = int64_t(nsm) * (p->precision == PP_FP64 ? 256 : 384);
    // Priorities: the expansion chain (the step's critical path) gets SMs first; the near
    // field (side stream aux) and the surface path (aux2), which finish well inside it, fill
    // whatever is left.
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    p->prio_hi = prio_hi;
    if (cudaStreamCreateWithPriority(&p->aux, cudaStreamNonBlocking, prio_lo) != cudaSuccess ||
        cudaStreamCreateWithPriority(&p->aux2, cudaStreamNonBlocking, prio_lo) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_up, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_surf, cudaEventDisableTiming) != cudaSuccess) {
        release_sync(p);
        delete p;
        return PP_ERR_CUDA;
    }
    int st = prepare_device(p->device, p->precision);
    if (st == PP_OK) st = (p->precision == PP_FP64) ? alloc_tree<double>(p) : alloc_tree<float>(p);
    if (st == PP_OK) {
        const size_t need = p->precision == PP_FP64 ? pp::plan_smem_bytes<double>(make_tree<double>(p))
                                                    : pp::plan_smem_bytes<float>(make_tree<float>(p));
        if (need > size_t(pp::kDynSmemLimit)) st = PP_ERR_ARG;
    }
    if (st == PP_OK && p->precision == PP_MIXED && p->near_tile == 128 && pp::near_tc_ok(p->nL, p->Dmax) && p->Lleaf >= 2)
        st = setup_near_tc(p);
    if (st == PP_OK && p->precision == PP_MIXED && o.m2l_tensor) {
        p->m2l_margin = pp::m2l_tc_margin(p->il_host.data(), p->il_count, p->il_stride);
        if (pp::m2l_tc_ok(p->P1, p->m2l_margin, p->il_stride) &&
            cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device) == cudaSuccess) {
            std::vector<unsigned char> tb(pp::m2l_tc_table_bytes(p->n_ops, p->il_stride));
            p->m2l_inv_sb = pp::m2l_tc_fill_tables(p->op_geo.data(), p->n_ops, p->il_host.data(), p->il_count,
                                                   p->il_stride, p->m2l_margin, tb.data());
            if (dalloc(p, &p->m2l_tab, tb.size()) != cudaSuccess) st = PP_ERR_OOM;
            else if (cudaMemcpy(p->m2l_tab, tb.data(), tb.size(), cudaMemcpyHostToDevice) != cudaSuccess) st = PP_ERR_CUDA;
            else p->use_m2l_tc = true;
        }
    }
    if (st == PP_OK) st = ensure_surface(p, pp::kInitialSurfaceCap);
    if (st != PP_OK) {
        free_all(p);
        release_sync(p);
        delete p;
        cudaGetLastError();
        return st;
    }
    *out = p;
    return PP_OK;
}

int pp_plan_bytes(int n, int order, double theta, const pp_options* opt, int npts, int64_t* bytes) {
    if (!bytes) return PP_ERR_ARG;
    *bytes = 0;
    pp_options o;
    pp_options_default(&o);
    if (opt) o = *opt;
    if (n < 8 || n > 16384 || (n & (n - 1)) != 0) return PP_ERR_ARG;
    if (order < 2 || order > pp::kMaxOrder) return PP_ERR_ARG;
    if (!(theta >= 0.25 && theta <= 0.95)) return PP_ERR_ARG;
    if (o.precision != PP_FP64 && o.precision != PP_MIXED) return PP_ERR_ARG;
    if (o.tile != 8 && o.tile != 16 && o.tile != 128) return PP_ERR_ARG;
    if (npts < 0 || npts > (1 << 24)) return PP_ERR_ARG;
    if (o.m2l_tensor != 0 && o.m2l_tensor != 1) return PP_ERR_ARG;
    *bytes = plan_bytes(n, order, theta, o.precision, o.tile, npts, o.m2l_tensor);
    return PP_OK;
}

int pp_plan_destroy(pp_plan p) {
    if (!p) return PP_OK;
    cudaStreamSynchronize(p->stream);
    if (p->aux) cudaStreamSynchronize(p->aux);
    if (p->aux2) cudaStreamSynchronize(p->aux2);
    free_all(p);
    release_sync(p);
    for (auto& e : p->ev)
        if (e) cudaEventDestroy(e);
    delete p;
    return PP_OK;
}

int pp_plan_set_stream(pp_plan p, void* stream) {
    if (!p) return PP_ERR_ARG;
    if (p->dead) return PP_ERR_STATE;
    p->stream = static_cast<cudaStream_t>(stream);
    return PP_OK;
}

int pp_rhs(pp_plan p, const void* u, const void* v, const void* chi, const void* us_x, const void* us_y,
           double lambda, void* f_out) {
    if (!p || !u || !v || !chi || !us_x || !us_y || !std::isfinite(lambda)) return PP_ERR_ARG;
    if (p->dead) return PP_ERR_STATE;
    return p->precision == PP_FP64 ? run_rhs<double>(p, u, v, chi, us_x, us_y, lambda, f_out)
                                   : run_rhs<float>(p, u, v, chi, us_x, us_y, lambda, f_out);
}

int pp_pressure_solve(pp_plan p, void* p_out) {
    if (!p) return PP_ERR_ARG;
    if (p->dead || !p->have_q) return PP_ERR_STATE;
    return p->precision == PP_FP64 ? run_solve<double>(p, p_out) : run_solve<float>(p, p_out);
}

int pp_surface_traction(pp_plan p, const void* u, const void* v, int npts, const double* points,
                        const double* normals, const double* dS, double nu, double* per_point, double* forces) {
    if (!p || !u || !v || !points || !normals || npts < 1 || npts > (1 << 24) || !std::isfinite(nu))
        return PP_ERR_ARG;
    if (p->dead || !p->have_q) return PP_ERR_STATE;
    return p->precision == PP_FP64
               ? run_surface<double>(p, u, v, npts, points, normals, dS, nu, per_point, forces)
               : run_surface<float>(p, u, v, npts, points, normals, dS, nu, per_point, forces);
}

int pp_penal_force(pp_plan p, const void* u, const void* v, const void* chi, const void* us_x, const void* us_y,
                   double lambda, double* forces) {
    if (!p || !u || !v || !chi || !us_x || !us_y || !forces || !std::isfinite(lambda)) return PP_ERR_ARG;
    if (p->dead) return PP_ERR_STATE;
    const bool dev = is_device_pointer(forces);
    double* out = dev ? forces : p->penal_buf + pp::penal_partial_doubles();
    const int64_t nc = int64_t(p->n) * p->n;
    const double scale = lambda * p->h * p->h;
    const cudaError_t e =
        p->precision == PP_FP64
            ? pp::launch_penal_force<double>((const double*)u, (const double*)v, (const double*)chi,
                                             (const double*)us_x, (const double*)us_y, nc, scale, p->uhx, p->uhy,
                                             p->penal_buf, out, p->stream)
            : pp::launch_penal_force<float>((const float*)u, (const float*)v, (const float*)chi, (const float*)us_x,
                                            (const float*)us_y, nc, scale, p->uhx, p->uhy, p->penal_buf, out,
                                            p->stream);
    if (e != cudaSuccess) return cuda_fail(p);
    p->launches += 1;
    if (!dev && (cudaMemcpyAsync(forces, out, 4 * sizeof(double), cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
                 cudaStreamSynchronize(p->stream) != cudaSuccess))
        return cuda_fail(p);
    return PP_OK;
}

int pp_body_moments(pp_plan p, const void* u, const void* v, const void* chi, double* out) {
    if (!p || !u || !v || !chi || !out) return PP_ERR_ARG;
    if (p->dead) return PP_ERR_STATE;
    const bool dev = is_device_pointer(out);
    double* res = dev ? out : p->moments_buf + pp::moments_partial_doubles();
    const int64_t nc = int64_t(p->n) * p->n;
    const double ms = p->rho * p->h * p->h;
    const cudaError_t e =
        p->precision == PP_FP64
            ? pp::launch_body_moments<double>((const double*)u, (const double*)v, (const double*)chi, nc, ms,
                                              p->moments_buf, res, p->stream)
            : pp::launch_body_moments<float>((const float*)u, (const float*)v, (const float*)chi, nc, ms,
                                             p->moments_buf, res, p->stream);
    if (e != cudaSuccess) return cuda_fail(p);
    p->launches += 1;
    if (!dev && (cudaMemcpyAsync(out, res, 3 * sizeof(double), cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
                 cudaStreamSynchronize(p->stream) != cudaSuccess))
        return cuda_fail(p);
    return PP_OK;
}

int pp_pressure_solve_fft(pp_plan p, void* p_out) {
    if (!p || !p_out) return PP_ERR_ARG;
    const bool fp64 = p->precision == PP_FP64;
    if (!pp::fft_size_ok(p->n, fp64)) return PP_ERR_ARG;
    if (p->dead || !p->have_q) return PP_ERR_STATE;
    if (!p->fft_Kp) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(p->stream, &cs) != cudaSuccess) return cuda_fail(p);
        if (cs != cudaStreamCaptureStatusNone) return PP_ERR_STATE;
        void *H = nullptr, *Kp = nullptr;
        if (dalloc(p, &H, pp::fft_work_bytes(p->n, fp64)) != cudaSuccess ||
            dalloc(p, &Kp, pp::fft_spectrum_bytes(p->n, fp64)) != cudaSuccess) {
            cudaGetLastError();
            return PP_ERR_OOM;
        }
        const cudaError_t e = pp::fft_prepare_spectrum(p->n, p->h, p->h * std::exp(kC0), fp64, Kp, p->stream);
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            return PP_ERR_OOM;
        }
        if (e != cudaSuccess) return cuda_fail(p);
        p->launches += 6;
        p->fft_H = H;
        p->fft_Kp = Kp;
    }
    const cudaError_t e =
        fp64 ? pp::launch_fft_solve<double>(static_cast<const double*>(p->q), p->n, p->nL, p->fft_Kp, p->fft_H,
                                            static_cast<double*>(p_out), p->stream)
             : pp::launch_fft_solve<float>(static_cast<const float*>(p->q), p->n, p->nL, p->fft_Kp, p->fft_H,
                                           static_cast<float*>(p_out), p->stream);
    if (e != cudaSuccess) return cuda_fail(p);
    p->launches += pp::fft_launches_per_solve();
    return PP_OK;
}

int pp_plan_info(pp_plan p, pp_plan_info_t* info) {
    if (!p || !info) return PP_ERR_ARG;
    info->n = p->n;
    info->order = p->order;
    info->levels = p->Lleaf + 1;
    info->precision = p->precision;
    info->h = p->h;
    info->theta = p->theta;
    info->theta_surface = p->theta_surf;
    info->n_near = p->n_near;
    for (int c = 0; c < 4; ++c) info->n_m2l[c] = p->il_count[c];
    info->near_pairs = p->near_pairs;
    info->m2l_pairs = p->m2l_pairs;
    info->workspace_bytes = p->workspace;
    info->launches = p->launches;
    info->m2l_pairs_leaf = p->m2l_pairs_leaf;
    info->near_kernel = 0;
    if (p->precision == PP_MIXED && pp::split_solve_ok<float>(make_tree<float>(p)))
        info->near_kernel = p->use_tc ? 128 : (p->near_tile == 16 && p->nL >= 8 && (p->nL & 7) == 0) ? 16 : 8;
    info->downward = 0;
    if (p->precision == PP_MIXED && info->near_kernel != 0) {
        const void* aligned = reinterpret_cast<const void*>(uintptr_t(256));
        info->downward = pp::down_tree_ok<float>(make_tree<float>(p), aligned) ? (p->use_m2l_tc ? 3 : 2) : 1;
    }
    return PP_OK;
}

int pp_plan_device_status(pp_plan p, int* flags) {
    if (!p || !flags) return PP_ERR_ARG;
    if (cudaStreamSynchronize(p->stream) != cudaSuccess ||
        cudaMemcpy(flags, p->err, 4 * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemset(p->err, 0, 4 * sizeof(int)) != cudaSuccess)
        return cuda_fail(p);
    return (flags[1] || flags[2]) ? PP_ERR_TIMEOUT : PP_OK;
}

int pp_plan_enable_timing(pp_plan p, int on) {
    if (!p) return PP_ERR_ARG;
    if (p->dead) return PP_ERR_STATE;
    if (on && !p->ev[0]) {
        for (auto& e : p->ev)
            if (cudaEventCreate(&e) != cudaSuccess) return cuda_fail(p);
    }
    p->timing = on != 0;
    for (bool& r : p->ran) r = false;
    return PP_OK;
}

int pp_plan_stage_times(pp_plan p, double* ms, int cap) {
    if (!p || (cap > 0 && !ms) || cap < 0) return -PP_ERR_ARG;
    if (p->dead) return -PP_ERR_STATE;
    for (int s = 0; s < N_STAGES && s < cap; ++s) {
        ms[s] = -1.0;
        if (!p->ran[s]) continue;
        // a timing query that fails (events not yet recorded) leaves the plan usable
        float t = 0.f;
        if (cudaEventSynchronize(p->ev[2 * s + 1]) != cudaSuccess ||
            cudaEventElapsedTime(&t, p->ev[2 * s], p->ev[2 * s + 1]) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        ms[s] = double(t);
    }
    return N_STAGES;
}

int pp_get_expansion(pp_plan p, int kind, int level, double* dst) {
    if (!p || !dst || (kind != 0 && kind != 1) || level < 0 || level > p->Lleaf) return PP_ERR_ARG;
    if (kind == 1 && level < 2) return PP_ERR_ARG;
    if (p->dead || !p->have_q) return PP_ERR_STATE;
    if (kind == 0) {
        int st = p->precision == PP_FP64 ? ensure_up<double>(p) : ensure_up<float>(p);
        if (st != PP_OK) return st;
    }
    cudaError_t e = p->precision == PP_FP64
                        ? pp::launch_export_expansion<double>(make_tree<double>(p), kind, level, dst, p->stream)
                        : pp::launch_export_expansion<float>(make_tree<float>(p), kind, level, dst, p->stream);
    return e == cudaSuccess ? PP_OK : cuda_fail(p);
}

int pp_near_offsets(double theta, int* out, int cap) {
    if (!(theta >= 0.25 && theta <= 0.95) || cap < 0 || (cap > 0 && !out)) return -PP_ERR_ARG;
    auto v = near_offsets(theta);
    for (size_t i = 0; i < v.size() && int(i) < cap; ++i) {
        out[2 * i] = v[i].first;
        out[2 * i + 1] = v[i].second;
    }
    return int(v.size());
}

int pp_m2l_entries(double theta, int child, int* out, int cap) {
    if (!(theta >= 0.25 && theta <= 0.95) || child < 0 || child > 3 || cap < 0 || (cap > 0 && !out))
        return -PP_ERR_ARG;
    auto v = m2l_entries(theta, child);
    for (size_t i = 0; i < v.size() && int(i) < cap; ++i) {
        out[3 * i] = v[i].dx;
        out[3 * i + 1] = v[i].dy;
        out[3 * i + 2] = v[i].kind;
    }
    return int(v.size());
}

int pp_m2l_offsets(double theta, int child, int* out, int cap) {
    if (!(theta >= 0.25 && theta <= 0.95) || child < 0 || child > 3 || cap < 0 || (cap > 0 && !out))
        return -PP_ERR_ARG;
    auto v = m2l_offsets(theta, child);
    for (size_t i = 0; i < v.size() && int(i) < cap; ++i) {
        out[2 * i] = v[i].first;
        out[2 * i + 1] = v[i].second;
    }
    return int(v.size());
}

struct pp_graph_s {
    pp_plan plan = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0;
};

int pp_step_graph_create(pp_plan p, const void* u, const void* v, const void* chi, const void* us_x,
                         const void* us_y, double lambda, void* p_out, int npts, const double* points,
                         const double* normals, const double* dS, double nu, double* per_point,
                         double* forces, pp_graph* out) {
    if (!out) return PP_ERR_ARG;
    *out = nullptr;
    if (!p || !u || !v || !chi || !us_x || !us_y || !std::isfinite(lambda) || !std::isfinite(nu)) return PP_ERR_ARG;
    if (npts < 0 || npts > (1 << 24) || (npts > 0 && (!points || !normals))) return PP_ERR_ARG;
    if (npts > 0 && forces && !is_device_pointer(forces)) return PP_ERR_ARG;
    if (p->dead) return PP_ERR_STATE;
    int st = ensure_surface(p, npts > 0 ? npts : 1);
    if (st != PP_OK) return st;
    pp_graph g = new (std::nothrow) pp_graph_s();
    if (!g) return PP_ERR_OOM;
    g->plan = p;
    cudaStream_t cap = nullptr;
    if (cudaStreamCreateWithPriority(&cap, cudaStreamNonBlocking, p->prio_hi) != cudaSuccess) {
        delete g;
        return PP_ERR_CUDA;
    }
    cudaStream_t saved = p->stream;
    const int64_t l0 = p->launches;
    p->stream = cap;
    st = PP_OK;
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = PP_ERR_CUDA;
    if (st == PP_OK) st = pp_rhs(p, u, v, chi, us_x, us_y, lambda, nullptr);
    // the near field forks right after the source weights, ahead of the upward pass
    if (st == PP_OK && p_out && p->precision == PP_MIXED && pp::split_solve_ok<float>(make_tree<float>(p)))
        st = fork_near<float>(p, p_out);
    if (st == PP_OK) st = p->precision == PP_FP64 ? ensure_up<double>(p) : ensure_up<float>(p);
    if (st == PP_OK && npts > 0) {
        // the surface path needs only q and the multipoles: run it beside the solve
        if (cudaEventRecord(p->ev_up, cap) != cudaSuccess || cudaStreamWaitEvent(p->aux2, p->ev_up, 0) != cudaSuccess)
            st = PP_ERR_CUDA;
        p->stream = p->aux2;
        if (st == PP_OK)
            st = p->precision == PP_FP64
                     ? run_surface<double>(p, u, v, npts, points, normals, dS, nu, per_point, forces, 1)
                     : run_surface<float>(p, u, v, npts, points, normals, dS, nu, per_point, forces, 1);
        p->stream = cap;
        if (st == PP_OK && cudaEventRecord(p->ev_surf, p->aux2) != cudaSuccess) st = PP_ERR_CUDA;
    }
    if (st == PP_OK) st = pp_pressure_solve(p, p_out);
    if (st == PP_OK && npts > 0 && cudaStreamWaitEvent(cap, p->ev_surf, 0) != cudaSuccess) st = PP_ERR_CUDA;
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(cap, &graph);
    p->stream = saved;
    p->near_forked = nullptr;
    cudaStreamDestroy(cap);
    g->launches = p->launches - l0;
    p->launches = l0;
    if (st == PP_OK && (ee != cudaSuccess || !graph)) st = PP_ERR_CUDA;
    if (st == PP_OK && cudaGraphInstantiate(&g->exec, graph, cudaGraphInstantiateFlagUseNodePriority) != cudaSuccess)
        st = PP_ERR_CUDA;
    g->graph = graph;
    if (st != PP_OK) {
        cudaGetLastError();
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        p->dead = false;  // capture failures do not touch device state
        return st;
    }
    *out = g;
    return PP_OK;
}

int pp_step_graph_launch(pp_graph g, void* stream) {
    if (!g || !g->exec) return PP_ERR_ARG;
    if (g->plan->dead) return PP_ERR_STATE;
    if (cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)) != cudaSuccess) return cuda_fail(g->plan);
    g->plan->launches += g->launches;
    return PP_OK;
}

int pp_step_graph_destroy(pp_graph g) {
    if (!g) return PP_OK;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return PP_OK;
}

struct pp_batch_s {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<pp_plan> plans;
    int64_t launches = 0;
};

int pp_batch_create(int count, const pp_graph* graphs, pp_batch* out) {
    if (!out) return PP_ERR_ARG;
    *out = nullptr;
    if (count < 1 || !graphs) return PP_ERR_ARG;
    for (int i = 0; i < count; ++i) {
        if (!graphs[i] || !graphs[i]->graph) return PP_ERR_ARG;
        for (int j = 0; j < i; ++j)  // the branches run at once: one solve per plan workspace
            if (graphs[j]->plan == graphs[i]->plan) return PP_ERR_ARG;
    }
    pp_batch b = new (std::nothrow) pp_batch_s();
    if (!b) return PP_ERR_OOM;
    int st = PP_OK;
    if (cudaGraphCreate(&b->graph, 0) != cudaSuccess) st = PP_ERR_CUDA;
    for (int i = 0; st == PP_OK && i < count; ++i) {
        cudaGraphNode_t node;
        // independent branches: the snapshots of a batch have no dependencies on each other
        if (cudaGraphAddChildGraphNode(&node, b->graph, nullptr, 0, graphs[i]->graph) != cudaSuccess)
            st = PP_ERR_CUDA;
        b->plans.push_back(graphs[i]->plan);
        b->launches += graphs[i]->launches;
    }
    if (st == PP_OK && cudaGraphInstantiate(&b->exec, b->graph, cudaGraphInstantiateFlagUseNodePriority) != cudaSuccess)
        st = PP_ERR_CUDA;
    if (st != PP_OK) {
        cudaGetLastError();
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        delete b;
        return st;
    }
    *out = b;
    return PP_OK;
}

int pp_batch_launch(pp_batch b, void* stream) {
    if (!b || !b->exec) return PP_ERR_ARG;
    for (pp_plan p : b->plans)
        if (p->dead) return PP_ERR_STATE;
    if (cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)) != cudaSuccess) {
        for (pp_plan p : b->plans) p->dead = true;
        return PP_ERR_CUDA;
    }
    if (!b->plans.empty()) b->plans[0]->launches += b->launches;
    return PP_OK;
}

int pp_batch_destroy(pp_batch b) {
    if (!b) return PP_OK;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    delete b;
    return PP_OK;
}

const char* pp_error_string(int status) {
    switch (status) {
        case PP_OK: return "ok";
        case PP_ERR_ARG: return "invalid argument";
        case PP_ERR_STATE: return "call order violated or plan unusable";
        case PP_ERR_OOM: return "device allocation failed";
        case PP_ERR_CUDA: return "CUDA error";
        case PP_ERR_TIMEOUT: return "bounded device wait gave up";
        case PP_ERR_BUDGET: return "request exceeds the memory budget";
        default: return "unknown status";
    }
}

}  // extern "C"
