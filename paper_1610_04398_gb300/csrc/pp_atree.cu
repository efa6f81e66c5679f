// Adaptive quadtree over the leaf blocks of a multiresolution grid, and its interaction lists
// (host code).  The paper's grids are adaptive and block-structured (Sec. 3, its citation of
// wavelet-adapted multiresolution grids; Appendix A.2 groups sources hierarchically for the
// tree-code).  Here the caller gives the leaves as blocks (level l, column ix, row iy) of side
// 2^-l of the unit domain; they must tile it exactly.  The tree is every leaf plus all of its
// ancestors; a box's four children are stored together, child c = (x & 1) + 2 (y & 1).
//
// Lists come from one dual-tree walk from (root, root) with the acceptance test of the grid
// solve (boxes A, B well separated iff r_A + r_B < theta d, r the half-diagonal, d the
// distance of the centres; the tie counts as not separated): a separated pair becomes a
// multipole-to-local pair (target box <- source box, possibly of different levels); two leaves
// that are not separated become a near-field pair; otherwise the larger box of the pair is
// split (the target when both are the same size and neither is a leaf).  The walk splits the
// product of the leaf sets into disjoint pieces, so every (target leaf, source leaf) pair is
// covered exactly once, by one near-field pair or by one multipole-to-local pair of their
// ancestors.  The test runs in exact integer units (half the finest box side), so it agrees
// with the uniform grid's offset lists.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <new>
#include <unordered_map>
#include <utility>
#include <vector>

#include "../../include/pp.h"
#include "pp_atree_state.h"

namespace {

constexpr int kMaxLevel = 20;

struct ABox {
    int level, ix, iy, parent, first_child, leaf;
};

}  // namespace

struct pp_atree_s {
    int max_level = 0;
    double theta = 0.0;
    std::vector<ABox> box;
    std::vector<int> m2l;  // pairs (target box, source box), sorted
    std::vector<int> p2p;  // pairs (target leaf, source leaf), sorted
    void* state = nullptr;  // what a solve keeps between calls (device arrays)
    void (*release)(void*) = nullptr;
};

namespace pp {

void* atree_state(pp_atree t) { return t->state; }

void atree_set_state(pp_atree t, void* state, void (*release)(void*)) {
    t->state = state;
    t->release = release;
}

int atree_adopt(const AtreeHost& h, double theta, pp_atree* out) {
    pp_atree t = nullptr;
    try {
        t = new pp_atree_s();
        t->theta = theta;
        t->max_level = h.max_level;
        t->box.resize(h.level.size());
        for (size_t i = 0; i < h.level.size(); ++i)
            t->box[i] = ABox{h.level[i], h.ix[i], h.iy[i], h.parent[i], h.first_child[i], h.leaf[i]};
        t->m2l = h.m2l;
        t->p2p = h.p2p;
    } catch (const std::bad_alloc&) {
        delete t;
        return PP_ERR_OOM;
    }
    *out = t;
    return PP_OK;
}

}  // namespace pp

namespace {

uint64_t akey(int level, int ix, int iy) {
    return (uint64_t(level) << 48) | (uint64_t(uint32_t(ix)) << 24) | uint64_t(uint32_t(iy));
}

// Separation test in units of half the finest box side: centre (2 ix + 1) 2^(L - l), side
// 2^(L - l + 1); separated iff theta^2 d^2 > (s_A + s_B)^2 / 2.
bool separated(const ABox& a, const ABox& b, int L, double theta) {
    const int64_t sa = int64_t(1) << (L - a.level + 1), sb = int64_t(1) << (L - b.level + 1);
    const int64_t ax = (2 * int64_t(a.ix) + 1) * (sa / 2), ay = (2 * int64_t(a.iy) + 1) * (sa / 2);
    const int64_t bx = (2 * int64_t(b.ix) + 1) * (sb / 2), by = (2 * int64_t(b.iy) + 1) * (sb / 2);
    const int64_t dx = ax - bx, dy = ay - by;
    const double d2 = double(dx * dx + dy * dy);
    const double s = double(sa + sb);
    return theta * theta * d2 > 0.5 * s * s;
}

int build(pp_atree t, int nleaf, const int* level, const int* ix, const int* iy) {
    // every leaf and all of its ancestors; a leaf may not also be an ancestor of a leaf
    std::unordered_map<uint64_t, int> kind;  // 1 = leaf (index + 1 stored below), 2 = internal
    std::unordered_map<uint64_t, int> leaf_of;
    kind.reserve(size_t(nleaf) * 2);
    int L = 0;
    for (int i = 0; i < nleaf; ++i) {
        const int l = level[i];
        if (l < 0 || l > kMaxLevel || ix[i] < 0 || iy[i] < 0 || ix[i] >= (1 << l) || iy[i] >= (1 << l))
            return PP_ERR_ARG;
        const uint64_t k = akey(l, ix[i], iy[i]);
        if (kind.count(k)) return PP_ERR_ARG;  // duplicate, or a leaf that covers another leaf
        kind[k] = 1;
        leaf_of[k] = i;
        L = std::max(L, l);
    }
    for (int i = 0; i < nleaf; ++i) {
        int l = level[i], x = ix[i], y = iy[i];
        while (l > 0) {
            --l;
            x >>= 1;
            y >>= 1;
            const uint64_t k = akey(l, x, y);
            auto it = kind.find(k);
            if (it != kind.end()) {
                if (it->second == 1) return PP_ERR_ARG;  // a leaf above another leaf: overlap
                break;                                   // the rest of the chain is already in
            }
            kind[k] = 2;
        }
    }
    // top-down, four children together; every internal box must have all four (no gaps)
    t->box.clear();
    t->box.reserve(kind.size());
    {
        const uint64_t rk = akey(0, 0, 0);
        if (!kind.count(rk)) return PP_ERR_ARG;
        const bool rleaf = kind[rk] == 1;
        t->box.push_back(ABox{0, 0, 0, -1, -1, rleaf ? leaf_of[rk] : -1});
    }
    for (size_t b = 0; b < t->box.size(); ++b) {
        if (t->box[b].leaf >= 0) continue;
        const ABox parent = t->box[b];
        t->box[b].first_child = int(t->box.size());
        for (int c = 0; c < 4; ++c) {
            const int l = parent.level + 1, x = 2 * parent.ix + (c & 1), y = 2 * parent.iy + (c >> 1);
            const uint64_t k = akey(l, x, y);
            auto it = kind.find(k);
            if (it == kind.end()) return PP_ERR_ARG;  // a gap in the tiling
            t->box.push_back(ABox{l, x, y, int(b), -1, it->second == 1 ? leaf_of[k] : -1});
        }
    }
    if (t->box.size() != kind.size()) return PP_ERR_ARG;
    t->max_level = L;
    // the dual-tree walk
    std::vector<std::pair<int, int>> stack{{0, 0}};
    std::vector<std::pair<int, int>> m2l, p2p;
    while (!stack.empty()) {
        const auto [a, b] = stack.back();
        stack.pop_back();
        const ABox& A = t->box[a];
        const ABox& B = t->box[b];
        if (separated(A, B, L, t->theta)) {
            m2l.emplace_back(a, b);
            continue;
        }
        const bool al = A.leaf >= 0, bl = B.leaf >= 0;
        if (al && bl) {
            p2p.emplace_back(A.leaf, B.leaf);
            continue;
        }
        if (!al && (bl || A.level <= B.level)) {
            for (int c = 0; c < 4; ++c) stack.emplace_back(A.first_child + c, b);
        } else {
            for (int c = 0; c < 4; ++c) stack.emplace_back(a, B.first_child + c);
        }
    }
    std::sort(m2l.begin(), m2l.end());
    std::sort(p2p.begin(), p2p.end());
    t->m2l.resize(2 * m2l.size());
    for (size_t i = 0; i < m2l.size(); ++i) {
        t->m2l[2 * i] = m2l[i].first;
        t->m2l[2 * i + 1] = m2l[i].second;
    }
    t->p2p.resize(2 * p2p.size());
    for (size_t i = 0; i < p2p.size(); ++i) {
        t->p2p[2 * i] = p2p[i].first;
        t->p2p[2 * i + 1] = p2p[i].second;
    }
    return PP_OK;
}

}  // namespace

extern "C" {

int pp_atree_create(int nleaf, const int* level, const int* ix, const int* iy, double theta, pp_atree* out) {
    if (!out) return PP_ERR_ARG;
    *out = nullptr;
    if (nleaf < 1 || !level || !ix || !iy || !(theta >= 0.25 && theta <= 0.95)) return PP_ERR_ARG;
    pp_atree t = nullptr;
    try {
        t = new pp_atree_s();
        t->theta = theta;
        const int st = build(t, nleaf, level, ix, iy);
        if (st != PP_OK) {
            delete t;
            return st;
        }
    } catch (const std::bad_alloc&) {
        delete t;
        return PP_ERR_OOM;
    }
    *out = t;
    return PP_OK;
}

int pp_atree_destroy(pp_atree t) {
    if (t && t->state && t->release) t->release(t->state);
    delete t;
    return PP_OK;
}

int pp_atree_sizes(pp_atree t, int64_t* sizes) {
    if (!t || !sizes) return PP_ERR_ARG;
    sizes[0] = int64_t(t->box.size());
    sizes[1] = int64_t(t->m2l.size() / 2);
    sizes[2] = int64_t(t->p2p.size() / 2);
    sizes[3] = t->max_level;
    return PP_OK;
}

int pp_atree_boxes(pp_atree t, int* level, int* ix, int* iy, int* parent, int* first_child, int* leaf) {
    if (!t) return PP_ERR_ARG;
    for (size_t i = 0; i < t->box.size(); ++i) {
        const ABox& b = t->box[i];
        if (level) level[i] = b.level;
        if (ix) ix[i] = b.ix;
        if (iy) iy[i] = b.iy;
        if (parent) parent[i] = b.parent;
        if (first_child) first_child[i] = b.first_child;
        if (leaf) leaf[i] = b.leaf;
    }
    return PP_OK;
}

int pp_atree_lists(pp_atree t, int* m2l, int* p2p) {
    if (!t) return PP_ERR_ARG;
    if (m2l) std::copy(t->m2l.begin(), t->m2l.end(), m2l);
    if (p2p) std::copy(t->p2p.begin(), t->p2p.end(), p2p);
    return PP_OK;
}

}  // extern "C"
