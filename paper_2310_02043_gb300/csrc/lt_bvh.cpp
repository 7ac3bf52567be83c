// lt_bvh.cpp -- host builder of the 8-wide BVH the tracing kernels traverse.
//
// 1. A binary BVH by the surface-area heuristic: for nodes of at most
//    kSahExactMax triangles every split between consecutive centroids along
//    each axis (exact), above that 256 bins along the largest centroid
//    extent; leaves of at most kLeafMax triangles.
// 2. Collapse to 8-wide nodes by the surface-area-optimal distribution of
//    the 8 slots of every wide node over binary subtrees (dynamic program
//    over the binary tree, see build_wide_bvh).
// 3. Nodes are emitted breadth-first, so the top levels form a prefix of the
//    node array, and leaf triangles are laid out contiguously in the order
//    their leaves appear.
// Child boxes are the float bounds of their triangles, padded (see step 3).
#include <algorithm>
#include <array>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <deque>
#include <functional>

#include "lt_internal.h"

// Build knobs: SAH bins of the binary build's large nodes, the largest node
// split by the exact sweep, and the cost of a triangle test relative to a
// wide-node visit in the 8-wide collapse.
#ifndef LT_SAH_BINS
#define LT_SAH_BINS 256
#endif
#ifndef LT_SAH_EXACT_MAX
#define LT_SAH_EXACT_MAX 4096
#endif
#ifndef LT_SAH_TRI_COST
#define LT_SAH_TRI_COST 0.23
#endif

namespace lt {
namespace {

struct Box {
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX};
    float hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    void grow(const float *p) {
        for (int k = 0; k < 3; ++k) { lo[k] = std::min(lo[k], p[k]); hi[k] = std::max(hi[k], p[k]); }
    }
    void grow(const Box &b) {
        for (int k = 0; k < 3; ++k) { lo[k] = std::min(lo[k], b.lo[k]); hi[k] = std::max(hi[k], b.hi[k]); }
    }
    double area() const {
        if (hi[0] < lo[0]) return 0.0;
        double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
        return 2.0 * (dx * dy + dy * dz + dz * dx);
    }
};

struct BNode {
    Box box;
    int32_t left = -1, right = -1;   // inner node children
    int32_t first = 0, count = 0;    // leaf triangle range in `idx`
    bool leaf() const { return left < 0; }
};

struct Binary {
    std::vector<BNode> nodes;
    std::vector<int32_t> idx;
};

void build_binary(const float *xyz, int32_t n_tri, Binary *b) {
    std::vector<Box> tbox(n_tri);
    std::vector<float> cen(3 * (size_t)n_tri);
    for (int32_t i = 0; i < n_tri; ++i) {
        for (int v = 0; v < 3; ++v) tbox[i].grow(xyz + 9 * (size_t)i + 3 * v);
        for (int k = 0; k < 3; ++k) cen[3 * (size_t)i + k] = 0.5f * (tbox[i].lo[k] + tbox[i].hi[k]);
    }
    b->idx.resize(n_tri);
    for (int32_t i = 0; i < n_tri; ++i) b->idx[i] = i;
    b->nodes.clear();
    b->nodes.reserve(2 * (size_t)n_tri);
    b->nodes.emplace_back();
    struct Job { int32_t node, first, count; };
    std::vector<Job> stack;
    stack.push_back({0, 0, n_tri});
    constexpr int kBins = LT_SAH_BINS;
    constexpr int32_t kSahExactMax = LT_SAH_EXACT_MAX;
    std::vector<int32_t> sweep;          // the node's triangles sorted along one axis (exact sweep)
    std::vector<double> right_area;      // area of the boxes right of each split (exact sweep)
    while (!stack.empty()) {
        Job j = stack.back();
        stack.pop_back();
        Box box, cbox;
        for (int32_t i = j.first; i < j.first + j.count; ++i) {
            box.grow(tbox[b->idx[i]]);
            cbox.grow(&cen[3 * (size_t)b->idx[i]]);
        }
        b->nodes[j.node].box = box;
        if (j.count <= kLeafMax) {
            b->nodes[j.node].first = j.first;
            b->nodes[j.node].count = j.count;
            continue;
        }
        int axis = 0;
        float ext[3];
        for (int k = 0; k < 3; ++k) ext[k] = cbox.hi[k] - cbox.lo[k];
        if (ext[1] > ext[axis]) axis = 1;
        if (ext[2] > ext[axis]) axis = 2;
        int32_t mid = j.first + j.count / 2;
        int32_t *beg = b->idx.data() + j.first, *end = beg + j.count;
        bool split_done = false;
        auto by_centroid = [&](int a) {
            return [&cen, a](int32_t x, int32_t y) {
                const float cx = cen[3 * (size_t)x + a], cy = cen[3 * (size_t)y + a];
                return cx < cy || (cx == cy && x < y);
            };
        };
        if (j.count <= kSahExactMax) {
            // every split between consecutive centroids along each axis
            double best = 1e300;
            int best_axis = -1;
            int32_t best_i = -1;
            sweep.assign(beg, end);
            right_area.resize((size_t)j.count);
            for (int a = 0; a < 3; ++a) {
                std::sort(sweep.begin(), sweep.end(), by_centroid(a));
                Box acc;
                for (int32_t i = j.count - 1; i > 0; --i) {
                    acc.grow(tbox[sweep[i]]);
                    right_area[i] = acc.area();
                }
                Box lacc;
                for (int32_t i = 1; i < j.count; ++i) {
                    lacc.grow(tbox[sweep[i - 1]]);
                    const double cost = lacc.area() * i + right_area[i] * (j.count - i);
                    if (cost < best) { best = cost; best_axis = a; best_i = i; }
                }
            }
            if (best_axis >= 0) {
                std::sort(beg, end, by_centroid(best_axis));
                mid = j.first + best_i;
                split_done = true;
            }
        } else if (ext[axis] > 0.0f) {
            Box bin_box[kBins];
            int32_t bin_cnt[kBins] = {0};
            const float inv = (float)kBins / ext[axis];
            auto bin_of = [&](int32_t t) {
                int k = (int)((cen[3 * (size_t)t + axis] - cbox.lo[axis]) * inv);
                return std::min(kBins - 1, std::max(0, k));
            };
            for (int32_t *p = beg; p < end; ++p) {
                int k = bin_of(*p);
                bin_box[k].grow(tbox[*p]);
                bin_cnt[k] += 1;
            }
            double right_area[kBins];
            int32_t right_cnt[kBins];
            Box acc;
            int32_t c = 0;
            for (int k = kBins - 1; k > 0; --k) {
                acc.grow(bin_box[k]);
                c += bin_cnt[k];
                right_area[k] = acc.area();
                right_cnt[k] = c;
            }
            Box lacc;
            int32_t lc = 0;
            double best = 1e300;
            int best_k = -1;
            for (int k = 1; k < kBins; ++k) {
                lacc.grow(bin_box[k - 1]);
                lc += bin_cnt[k - 1];
                if (lc == 0 || right_cnt[k] == 0) continue;
                double cost = lacc.area() * lc + right_area[k] * right_cnt[k];
                if (cost < best) { best = cost; best_k = k; }
            }
            if (best_k > 0) {
                int32_t *m = std::partition(beg, end, [&](int32_t t) { return bin_of(t) < best_k; });
                if (m != beg && m != end) { mid = (int32_t)(m - b->idx.data()); split_done = true; }
            }
        }
        if (!split_done) {
            // all centroids in one bin: split at the median along the axis
            std::nth_element(beg, b->idx.data() + mid, end, by_centroid(axis));
        }
        int32_t l = (int32_t)b->nodes.size();
        b->nodes.emplace_back();
        b->nodes.emplace_back();
        b->nodes[j.node].left = l;
        b->nodes[j.node].right = l + 1;
        stack.push_back({l + 1, mid, j.first + j.count - mid});
        stack.push_back({l, j.first, mid - j.first});
    }
}

// Slot of every child: slot s stands for the direction whose component a is
// + when bit a of s is set. A child goes to the slot that best matches where
// it lies relative to the parent's centre; the assignment minimising the sum
// of -dot(child centre - parent centre, slot direction) is found exactly by
// dynamic programming over subsets of slots (8 slots, at most 8 children).
std::vector<int> assign_slots(const std::vector<Box> &boxes, const Box &parent) {
    const int n = (int)boxes.size();
    double pc[3];
    for (int a = 0; a < 3; ++a) pc[a] = 0.5 * ((double)parent.lo[a] + parent.hi[a]);
    double cost[kWide][kWide];
    for (int j = 0; j < n; ++j) {
        const Box &bx = boxes[j];
        for (int s = 0; s < kWide; ++s) {
            double c = 0.0;
            for (int a = 0; a < 3; ++a) {
                const double v = 0.5 * ((double)bx.lo[a] + bx.hi[a]) - pc[a];
                c -= ((s >> a) & 1 ? 1.0 : -1.0) * v;
            }
            cost[j][s] = c;
        }
    }
    // dp[m] = best cost of giving children 0..popcount(m)-1 the slots in m
    std::vector<double> dp(1 << kWide, 1e300);
    std::vector<int> from(1 << kWide, -1);
    dp[0] = 0.0;
    for (int m = 0; m < (1 << kWide); ++m) {
        const int j = __builtin_popcount(m);
        if (j >= n || dp[m] >= 1e300) continue;
        for (int s = 0; s < kWide; ++s) {
            if (m & (1 << s)) continue;
            const double c = dp[m] + cost[j][s];
            if (c < dp[m | (1 << s)]) { dp[m | (1 << s)] = c; from[m | (1 << s)] = s; }
        }
    }
    int best = -1;
    for (int m = 0; m < (1 << kWide); ++m)
        if (__builtin_popcount(m) == n && (best < 0 || dp[m] < dp[best])) best = m;
    std::vector<int> slot(n);
    for (int m = best, j = n - 1; j >= 0; --j) {
        slot[j] = from[m];
        m &= ~(1 << from[m]);
    }
    return slot;
}

}  // namespace

bool build_wide_bvh(const float *xyz, int32_t n_tri, BvhBuild *out, std::string *err) {
    if (n_tri <= 0 || n_tri >= (1 << 28)) {
        *err = "triangle count must be in [1, 2^28)";
        return false;
    }
    Binary b;
    build_binary(xyz, n_tri, &b);
    out->nodes.clear();
    out->parent.clear();
    out->order.clear();
    out->order.reserve(n_tri);
    out->depth = 0;

    // 1-2. Wide nodes by the surface-area-optimal distribution of slots
    //    (Ylitie, Karras and Laine, "Efficient incoherent ray traversal on
    //    GPUs through compressed wide BVHs", HPG 2017): C(n, i) is the least
    //    cost of the subtree of binary node n occupying at most i slots of
    //    the wide node above it, D(n, j) the least cost of giving j >= 2 slots
    //    to n's two children. A subtree in one slot is a leaf (its triangles)
    //    or a wide node of its own (one node visit plus D(n, 8)). The costs
    //    are the kernel's: a node visit tests 8 boxes, about 4.3 triangle
    //    tests' worth of arithmetic.
    struct Entry { int32_t bnode; int32_t wide; };        // wide >= 0: an inner child
    struct Wide { std::vector<Entry> kids; };
    std::vector<Wide> wide;
    {
        constexpr double kNodeCost = 1.0, kTriCost = LT_SAH_TRI_COST;
        const int32_t NB = (int32_t)b.nodes.size();
        std::vector<std::array<double, kWide + 1>> C(NB), D(NB);
        std::vector<std::array<int8_t, kWide + 1>> split(NB), open(NB);
        for (int32_t n = NB - 1; n >= 0; --n) {          // children come after their parent
            const BNode &bn = b.nodes[n];
            const double area = bn.box.area();
            if (bn.leaf()) {
                for (int i = 1; i <= kWide; ++i) { C[n][i] = area * kTriCost * bn.count; open[n][i] = 0; }
                continue;
            }
            for (int j = 2; j <= kWide; ++j) {
                double best = 1e300;
                int arg = 1;
                for (int k = 1; k < j; ++k) {
                    const double c = C[bn.left][k] + C[bn.right][j - k];
                    if (c < best) { best = c; arg = k; }
                }
                D[n][j] = best;
                split[n][j] = (int8_t)arg;
            }
            C[n][1] = area * kNodeCost + D[n][kWide];
            open[n][1] = 0;
            for (int i = 2; i <= kWide; ++i) {
                if (D[n][i] < C[n][i - 1]) { C[n][i] = D[n][i]; open[n][i] = 1; }
                else { C[n][i] = C[n][i - 1]; open[n][i] = 0; }
            }
        }
        // the entries of a wide node rooted at binary node r: its j slots
        // distributed by the recorded choices
        std::deque<std::pair<int32_t, int32_t>> queue;      // (binary node, wide node)
        std::vector<Entry> entries;
        std::function<void(int32_t, int)> take = [&](int32_t m, int i) {
            while (i > 1 && !open[m][i]) --i;
            if (i <= 1) {
                if (b.nodes[m].leaf()) {
                    entries.push_back({m, -1});
                } else {
                    const int32_t w = (int32_t)wide.size();
                    wide.emplace_back();
                    entries.push_back({m, w});
                    queue.push_back({m, w});
                }
                return;
            }
            const int k = split[m][i];
            take(b.nodes[m].left, k);
            take(b.nodes[m].right, i - k);
        };
        wide.emplace_back();
        queue.push_back({0, 0});
        while (!queue.empty()) {
            const auto [bn, wn] = queue.front();
            queue.pop_front();
            entries.clear();
            if (b.nodes[bn].leaf()) {
                entries.push_back({bn, -1});
            } else {
                const int k = split[bn][kWide];
                take(b.nodes[bn].left, k);
                take(b.nodes[bn].right, kWide - k);
            }
            wide[wn].kids = entries;
        }
    }

    // 3. Emit breadth-first: slots by direction, padded boxes, leaf ranges.
    // Child boxes grow by pad on every side: the traversal computes a plane
    // distance as fma(plane, 1/d, -o/d), whose rounding of o/d moves the
    // plane by up to |o| 2^-24; 2^-19 (|coordinate| + 1) covers ray origins
    // anywhere within eight times the scene's extent from the world origin.
    float amax = 0.0f;
    for (size_t i = 0; i < (size_t)n_tri * 9; ++i) amax = std::max(amax, std::fabs(xyz[i]));
    const float pad = (amax + 1.0f) * 0x1p-19f;

    struct Item { int32_t wide, node, depth; };
    std::deque<Item> queue;
    out->nodes.emplace_back();
    out->parent.push_back(-1);
    queue.push_back({0, 0, 0});
    while (!queue.empty()) {
        const Item it = queue.front();
        queue.pop_front();
        out->depth = std::max(out->depth, it.depth + 1);
        if (it.depth >= kMaxDepth) {
            *err = "BVH deeper than the traversal trail supports";
            return false;
        }
        const std::vector<Entry> &kids = wide[it.wide].kids;
        std::vector<Box> boxes;
        Box all;
        for (const Entry &e : kids) {
            boxes.push_back(b.nodes[e.bnode].box);
            all.grow(boxes.back());
        }
        Node node;
        std::memset(&node, 0, sizeof(node));
        for (int k = 0; k < kWide; ++k) {
            node.lox[k] = node.loy[k] = node.loz[k] = 3.0e38f;
            node.hix[k] = node.hiy[k] = node.hiz[k] = -3.0e38f;
            node.child[k] = kEmptyChild;
        }
        const std::vector<int> slot_of = assign_slots(boxes, all);
        for (int j = 0; j < (int)kids.size(); ++j) {
            const int k = slot_of[j];
            const Box &bx = boxes[j];
            node.lox[k] = bx.lo[0] - pad; node.hix[k] = bx.hi[0] + pad;
            node.loy[k] = bx.lo[1] - pad; node.hiy[k] = bx.hi[1] + pad;
            node.loz[k] = bx.lo[2] - pad; node.hiz[k] = bx.hi[2] + pad;
            const BNode &c = b.nodes[kids[j].bnode];
            if (kids[j].wide < 0) {
                const int32_t first = (int32_t)out->order.size();
                for (int32_t i = c.first; i < c.first + c.count; ++i) out->order.push_back(b.idx[i]);
                node.child[k] = -1 - ((first << 2) | (c.count - 1));
            } else {
                const int32_t wn = (int32_t)out->nodes.size();
                out->nodes.emplace_back();
                out->parent.push_back(it.node);
                node.child[k] = wn;
                node.inner_mask |= 1u << k;
                queue.push_back({kids[j].wide, wn, it.depth + 1});
            }
        }
        out->nodes[it.node] = node;
    }
    if ((int32_t)out->order.size() != n_tri) {
        *err = "BVH builder lost triangles";
        return false;
    }
    return true;
}

// Node compression. Per axis the origin p is a float a little below the
// lowest plane of the node's children and the step 2^e the smallest power of
// two with 254 steps covering the planes; lo planes round down and hi planes
// up. The kernel decodes a plane distance as fma(1 + q 2^-15, S, B) with
// S = 2^(e+15) / d and B = (p - 2^(e+15) - o) / d, each rounded in float,
// which moves a plane by at most about 2^-24 (6 |coordinate| + 400 extent);
// the float node's padding covers the first term (8x over), and a margin of
// 2^-14 of the node's extent on every side covers the second.
bool compress_nodes(const Node *nodes, int32_t n_nodes, CNode *out) {
    for (int32_t i = 0; i < n_nodes; ++i) {
        const Node &nd = nodes[i];
        CNode &cn = out[i];
        std::memset(&cn, 0, sizeof(cn));
        uint32_t meta = (nd.inner_mask & 0xffu) << 24;
        const float *lo[3] = {nd.lox, nd.loy, nd.loz}, *hi[3] = {nd.hix, nd.hiy, nd.hiz};
        for (int a = 0; a < 3; ++a) {
            double mn = INFINITY, mx = -INFINITY;
            for (int k = 0; k < kWide; ++k) {
                if (nd.child[k] == kEmptyChild) continue;
                mn = std::min(mn, (double)lo[a][k]);
                mx = std::max(mx, (double)hi[a][k]);
            }
            if (!(mn <= mx)) mn = mx = 0.0;            // no child (not built): any valid origin
            const double m = (mx - mn) * 0x1p-14;
            float p = (float)(mn - m);
            while ((double)p > mn - m) p = std::nextafter(p, -INFINITY);
            const double ext = mx + m - (double)p;
            int e = -126;
            while (std::ldexp(254.0, e) < ext) ++e;
            // E = 2^(e+15) at most 2^28, so that E / d stays finite for the
            // 1e30 reciprocal of an axis-parallel ray (node extents up to
            // 254 x 2^13, about 2e6)
            const int biased = e + 15 + 127;
            if (biased < 1 || biased > 127 + 28) return false;
            cn.p[a] = p;
            meta |= (uint32_t)biased << (8 * a);
            const double step = std::ldexp(1.0, e);
            for (int k = 0; k < kWide; ++k) {
                int ql = 255, qh = 0;                   // empty slot: an inverted box
                if (nd.child[k] != kEmptyChild) {
                    ql = (int)std::floor(((double)lo[a][k] - m - (double)p) / step);
                    qh = (int)std::ceil(((double)hi[a][k] + m - (double)p) / step);
                    if (ql < 0 || qh > 254 || ql > qh) return false;
                }
                cn.q[a][k] = (uint8_t)ql;
                cn.q[a][8 + k] = (uint8_t)qh;
            }
        }
        cn.meta = meta;
        for (int k = 0; k < kWide; ++k) cn.child[k] = nd.child[k];
    }
    return true;
}

}  // namespace lt
