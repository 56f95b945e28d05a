// Balanced binary cluster tree and geometric block partition (host, float64).
//
// The paper builds the H-matrix on balanced cluster trees with a purely
// geometric admissibility condition, one block structure shared by every
// frequency (Section 4, paragraph after eq. (outerProd), and the first
// implementation remark).  Its concrete rules are not given; this file
// implements one fixed reading exactly (compiled without FMA contraction so
// the result is identical on every host):
//   * cluster box = bounding box of all vertices of the cluster's elements;
//   * a cluster of n > leaf elements splits along the longest box side (lowest
//     axis on ties): elements sorted by (centroid[axis], element index),
//     centroid = ((v0 + v1) + v2) / 3, left child = first floor(n/2);
//     node ids in preorder;
//   * (t, s) admissible iff min(diam2(t), diam2(s)) <= eta^2 dist2(t, s) and
//     dist2 > 0 (squared box diameter / box distance, summed x, y, z);
//   * partition from (root, root): admissible -> far; two leaves -> near;
//     two inner nodes -> (LL, LR, RL, RR); else split the inner one;
//   * optional cap max_block > 0: an admissible pair whose larger cluster has
//     more than max_block elements is split by the same rule as an
//     inadmissible one (children of an admissible pair stay admissible: their
//     boxes shrink and their distance grows), so no far block exceeds the cap
//     unless both clusters are leaves.
#include <algorithm>
#include <climits>
#include <cmath>
#include <numeric>

#include "g3_internal.h"

namespace g3 {
namespace {

struct Builder {
    const std::vector<double>& V;
    const std::vector<int32_t>& T;
    int leaf;
    double eta;
    int max_block = 0;
    std::vector<double> cen;        // [ne][3]
    std::vector<double> tmin, tmax; // [ne][3]
    std::vector<int32_t> perm;
    std::vector<int32_t> nodes;     // begin, end, left, right
    std::vector<double> boxes;      // lo[3], hi[3]
    std::vector<int32_t> blocks;

    Builder(const std::vector<double>& v, const std::vector<int32_t>& t, int lf, double e)
        : V(v), T(t), leaf(lf), eta(e) {}

    void prepare(int ne) {
        cen.resize(3 * (size_t)ne);
        tmin.resize(3 * (size_t)ne);
        tmax.resize(3 * (size_t)ne);
        for (int e = 0; e < ne; ++e) {
            const double* a = &V[3 * (size_t)T[3 * e + 0]];
            const double* b = &V[3 * (size_t)T[3 * e + 1]];
            const double* c = &V[3 * (size_t)T[3 * e + 2]];
            for (int d = 0; d < 3; ++d) {
                double sum = a[d] + b[d];
                sum = sum + c[d];
                cen[3 * e + d] = sum / 3.0;
                tmin[3 * e + d] = std::min(std::min(a[d], b[d]), c[d]);
                tmax[3 * e + d] = std::max(std::max(a[d], b[d]), c[d]);
            }
        }
    }

    // idx: elements of this node (already in the parent's sorted order)
    int node(std::vector<int32_t>& idx, int start) {
        const int nid = (int)(nodes.size() / 4);
        const int n = (int)idx.size();
        nodes.insert(nodes.end(), {start, start + n, -1, -1});
        double lo[3], hi[3];
        for (int d = 0; d < 3; ++d) {
            lo[d] = tmin[3 * (size_t)idx[0] + d];
            hi[d] = tmax[3 * (size_t)idx[0] + d];
        }
        for (int e : idx)
            for (int d = 0; d < 3; ++d) {
                lo[d] = std::min(lo[d], tmin[3 * (size_t)e + d]);
                hi[d] = std::max(hi[d], tmax[3 * (size_t)e + d]);
            }
        boxes.insert(boxes.end(), {lo[0], lo[1], lo[2], hi[0], hi[1], hi[2]});
        if (n > leaf) {
            int axis = 0;
            double ext[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
            for (int d = 1; d < 3; ++d)
                if (ext[d] > ext[axis]) axis = d;
            const double* c = cen.data();
            auto before = [c, axis](int32_t x, int32_t y) {
                double cx = c[3 * (size_t)x + axis], cy = c[3 * (size_t)y + axis];
                if (cx < cy) return true;
                if (cy < cx) return false;
                return x < y;
            };
            // the keys are unique (index tie-break), so a selection of the
            // first h gives the same halves as a full sort; a child that is a
            // leaf keeps the sorted order of its elements
            const int h = n / 2;
            std::nth_element(idx.begin(), idx.begin() + h, idx.end(), before);
            if (h <= leaf) std::sort(idx.begin(), idx.begin() + h, before);
            if (n - h <= leaf) std::sort(idx.begin() + h, idx.end(), before);
            std::vector<int32_t> L(idx.begin(), idx.begin() + h), R(idx.begin() + h, idx.end());
            std::vector<int32_t>().swap(idx);
            int l = node(L, start);
            int r = node(R, start + h);
            nodes[4 * (size_t)nid + 2] = l;
            nodes[4 * (size_t)nid + 3] = r;
        } else {
            perm.insert(perm.end(), idx.begin(), idx.end());
        }
        return nid;
    }

    static double diam2(const double* b) {
        double dx = b[3] - b[0];
        double dy = b[4] - b[1];
        double dz = b[5] - b[2];
        double a = dx * dx;
        double bb = dy * dy;
        double cc = dz * dz;
        return (a + bb) + cc;
    }
    static double dist2(const double* t, const double* s) {
        double acc = 0.0;
        for (int d = 0; d < 3; ++d) {
            double g = std::max(0.0, std::max(s[d] - t[3 + d], t[d] - s[3 + d]));
            double gg = g * g;
            acc = acc + gg;
        }
        return acc;
    }
    bool admissible(int t, int s) const {
        const double* bt = &boxes[6 * (size_t)t];
        const double* bs = &boxes[6 * (size_t)s];
        double d2 = dist2(bt, bs);
        double e2 = eta * eta;
        double rhs = e2 * d2;
        return std::min(diam2(bt), diam2(bs)) <= rhs && d2 > 0.0;
    }
    void part(int t, int s) {
        auto N = [&](int id, int k) { return nodes[4 * (size_t)id + k]; };
        bool tl = N(t, 2) < 0, sl = N(s, 2) < 0;
        if (admissible(t, s)) {
            const int big = std::max(N(t, 1) - N(t, 0), N(s, 1) - N(s, 0));
            if (max_block <= 0 || big <= max_block || (tl && sl)) {
                blocks.insert(blocks.end(), {N(t, 0), N(t, 1), N(s, 0), N(s, 1), 1});
                return;
            }
        } else if (tl && sl) {
            blocks.insert(blocks.end(), {N(t, 0), N(t, 1), N(s, 0), N(s, 1), 0});
            return;
        }
        if (!tl && !sl) {
            part(N(t, 2), N(s, 2));
            part(N(t, 2), N(s, 3));
            part(N(t, 3), N(s, 2));
            part(N(t, 3), N(s, 3));
        } else if (tl) {
            part(t, N(s, 2));
            part(t, N(s, 3));
        } else {
            part(N(t, 2), s);
            part(N(t, 3), s);
        }
    }
};

}  // namespace

g3_status build_tree_host(g3_tree* t) {
    const int ne = t->ne;
    for (int e = 0; e < ne; ++e) {
        for (int k = 0; k < 3; ++k) {
            int v = t->tris[3 * (size_t)e + k];
            if (v < 0 || v >= t->nv) return fail(G3_EINVAL, "tris[%d] references vertex %d outside [0, %d)", e, v, t->nv);
        }
        // degenerate triangle check: zero cross product
        const double* a = &t->verts[3 * (size_t)t->tris[3 * e]];
        const double* b = &t->verts[3 * (size_t)t->tris[3 * e + 1]];
        const double* c = &t->verts[3 * (size_t)t->tris[3 * e + 2]];
        double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        double w[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        double cr[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
        if (!(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2] > 0.0))
            return fail(G3_EINVAL, "triangle %d is degenerate", e);
    }
    Builder B(t->verts, t->tris, t->leaf, t->eta);
    B.max_block = t->max_block;
    B.prepare(ne);
    std::vector<int32_t> all(ne);
    std::iota(all.begin(), all.end(), 0);
    B.perm.reserve(ne);
    B.node(all, 0);
    B.part(0, 0);
    t->perm.swap(B.perm);
    t->nodes.swap(B.nodes);
    t->boxes.swap(B.boxes);
    t->blocks.swap(B.blocks);
    tree_index_blocks(t);
    return G3_OK;
}

// ---------------------------------------------------------------------------
// Row-cluster sharding of a block partition over ranks (host only)
// ---------------------------------------------------------------------------
//
// The blocks of the partition are independent units of assembly and
// compression, and the apply adds each block's product into the rows of its
// row cluster.  Giving every rank whole row clusters therefore splits the
// work with disjoint output rows and no exchange on the data path (the
// densities are read by all ranks).  Units: the clusters at the smallest
// depth d at which some block has its row cluster (every block's row cluster
// lies in exactly one of them), plus the leaves above d; blocks are
// assigned with their unit, units longest first (cost = sum of the costs of
// their blocks) to the least loaded rank (ties: the lower unit begin, the
// lower rank).
g3_status shard_rows_host(const int32_t* nodes, int n_nodes, const int32_t* blocks, int nb, const double* cost,
                          int n_ranks, int32_t* owner, double* load, int* n_units) {
    if (!nodes || !blocks || !owner || n_nodes < 1 || nb < 0 || n_ranks < 1)
        return fail(G3_EINVAL, "g3_shard_rows: bad argument");
    auto N = [&](int id, int k) { return nodes[4 * (size_t)id + k]; };
    // depth of every node (preorder: a child's id is larger than its parent's)
    std::vector<int> depth(n_nodes, -1);
    depth[0] = 0;
    for (int id = 0; id < n_nodes; ++id) {
        if (depth[id] < 0) return fail(G3_EINVAL, "g3_shard_rows: node %d is not reachable from the root", id);
        for (int c = 2; c < 4; ++c) {
            const int ch = N(id, c);
            if (ch < 0) continue;
            if (ch <= id || ch >= n_nodes) return fail(G3_EINVAL, "g3_shard_rows: child %d of node %d", ch, id);
            depth[ch] = depth[id] + 1;
        }
    }
    const int ne = N(0, 1) - N(0, 0);
    // node of each (begin, end) row range: descend from the root
    auto find = [&](int b, int e) -> int {
        int id = 0;
        for (;;) {
            if (N(id, 0) == b && N(id, 1) == e) return id;
            const int l = N(id, 2), r = N(id, 3);
            if (l < 0) return -1;
            if (e <= N(l, 1)) id = l;
            else if (b >= N(r, 0)) id = r;
            else return -1;
        }
    };
    std::vector<int> rnode(nb);
    int dmin = INT32_MAX;
    for (int b = 0; b < nb; ++b) {
        const int id = find(blocks[5 * (size_t)b], blocks[5 * (size_t)b + 1]);
        if (id < 0) return fail(G3_EINVAL, "g3_shard_rows: block %d has no row cluster in the tree", b);
        rnode[b] = id;
        dmin = std::min(dmin, depth[id]);
    }
    if (nb == 0) dmin = 0;
    // units: nodes at depth dmin and leaves above it, by element position
    std::vector<int> unit_of_pos(ne > 0 ? ne : 1, -1);
    std::vector<int> ubegin;
    for (int id = 0; id < n_nodes; ++id) {
        const bool leaf = N(id, 2) < 0;
        if (depth[id] == dmin || (leaf && depth[id] < dmin)) {
            const int u = (int)ubegin.size();
            ubegin.push_back(N(id, 0));
            for (int p = N(id, 0); p < N(id, 1); ++p) unit_of_pos[p - N(0, 0)] = u;
        }
    }
    const int nu = (int)ubegin.size();
    std::vector<double> ucost(nu, 0.0);
    std::vector<int> bunit(nb);
    for (int b = 0; b < nb; ++b) {
        const int32_t* r = &blocks[5 * (size_t)b];
        const int u = unit_of_pos[r[0] - N(0, 0)];
        bunit[b] = u;
        const double c = cost ? cost[b] : (double)(r[1] - r[0]) * (double)(r[3] - r[2]);
        if (!(c >= 0.0) || !std::isfinite(c)) return fail(G3_EINVAL, "g3_shard_rows: cost[%d] = %g", b, c);
        ucost[u] += c;
    }
    std::vector<int> order(nu);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        if (ucost[a] != ucost[b]) return ucost[a] > ucost[b];
        return ubegin[a] < ubegin[b];
    });
    std::vector<double> ld(n_ranks, 0.0);
    std::vector<int> urank(nu, 0);
    for (int u : order) {
        int best = 0;
        for (int k = 1; k < n_ranks; ++k)
            if (ld[k] < ld[best]) best = k;
        urank[u] = best;
        ld[best] += ucost[u];
    }
    for (int b = 0; b < nb; ++b) owner[b] = urank[bunit[b]];
    if (load)
        for (int k = 0; k < n_ranks; ++k) load[k] = ld[k];
    if (n_units) *n_units = nu;
    return G3_OK;
}

// far / near lists of a tree's (possibly filtered) block list
void tree_index_blocks(g3_tree* t) {
    const int nb = (int)(t->blocks.size() / 5);
    t->far_index.clear();
    t->near_index.clear();
    t->max_far_m = t->max_far_n = 0;
    for (int b = 0; b < nb; ++b) {
        const int32_t* r = &t->blocks[5 * (size_t)b];
        if (r[4]) {
            t->far_index.push_back(b);
            t->max_far_m = std::max(t->max_far_m, r[1] - r[0]);
            t->max_far_n = std::max(t->max_far_n, r[3] - r[2]);
        } else {
            t->near_index.push_back(b);
        }
    }
}

}  // namespace g3

extern "C" g3_status g3_shard_rows(const int32_t* nodes, int n_nodes, const int32_t* blocks, int n_blocks,
                                   const double* cost, int n_ranks, int32_t* owner, double* load, int* n_units) {
    return g3::shard_rows_host(nodes, n_nodes, blocks, n_blocks, cost, n_ranks, owner, load, n_units);
}

// the host part of build_cluster_tree_capped alone (no context, no device):
// the permutation and the block list, for host-side use and checks
extern "C" g3_status g3_tree_partition_host(const double* verts, int nv, const int32_t* tris, int ne, int leaf,
                                            double eta, int max_block, int32_t* perm, int32_t* blocks,
                                            int64_t blocks_cap, int64_t* n_blocks) {
    if (!verts || !tris || nv < 3 || ne < 1 || leaf < 1 || max_block < 0 || !(eta > 0) || !std::isfinite(eta))
        return g3::fail(G3_EINVAL, "g3_tree_partition_host: bad argument");
    for (long long i = 0; i < 3LL * nv; ++i)
        if (!std::isfinite(verts[i]))
            return g3::fail(G3_EINVAL, "g3_tree_partition_host: non-finite vertex coordinate at %lld", i);
    g3_tree t;
    t.ne = ne;
    t.nv = nv;
    t.leaf = leaf;
    t.max_block = max_block;
    t.eta = eta;
    t.verts.assign(verts, verts + 3 * (size_t)nv);
    t.tris.assign(tris, tris + 3 * (size_t)ne);
    const g3_status st = g3::build_tree_host(&t);
    if (st != G3_OK) return st;
    const int64_t nb = (int64_t)(t.blocks.size() / 5);
    if (n_blocks) *n_blocks = nb;
    if (perm) std::copy(t.perm.begin(), t.perm.end(), perm);
    if (blocks) {
        if (blocks_cap < nb)
            return g3::fail(G3_EINVAL, "g3_tree_partition_host: %lld blocks do not fit in %lld", (long long)nb,
                            (long long)blocks_cap);
        std::copy(t.blocks.begin(), t.blocks.end(), blocks);
    }
    return G3_OK;
}
