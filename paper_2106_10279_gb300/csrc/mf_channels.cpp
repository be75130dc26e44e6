// Channels of the multichannel phase space, derived on the host from the
// diagram program of a process descriptor (the paper's outlook, Sec. 4: a
// phase space built from the process topology in place of RAMBO, Sec. 2.4),
// and Neyman's allocation of an iteration's points over the channels.
//
// Every AMP op of the program is one diagram; its currents are the
// propagators.  A current whose legs hold exactly one of the incoming legs
// (0 and 1) lies on the t-channel path between them; the others are
// s-channel propagators of a cluster of final legs (a current holding both
// incoming legs carries the final legs outside it).  Diagrams with a
// four-gluon vertex are left out; diagrams with equal channels are merged.
// The table layout, the order of a channel's unit numbers and the weight
// are those of device/mf_channels.cuh.
#include <algorithm>
#include <cmath>
#include <map>
#include <vector>

#include "mf_internal.h"
#include "device/mf_channels.cuh"

namespace mfi {
namespace {

int popcount(int m) {
    int c = 0;
    for (; m; m &= m - 1) ++c;
    return c;
}

int lowest(int m) {
    int i = 0;
    while (!((m >> i) & 1)) ++i;
    return i;
}

bool four_vertex(int routine) {
    return routine >= MF_R_VVVV1_AMP && routine <= MF_R_VVVV3_VEC;
}

struct Node {
    int mask, mass, left, right;
};

struct Chan {
    int k = 0;
    int cmask[MF_CH_MAX_FINAL] = {0};
    int cnode[MF_CH_MAX_FINAL] = {0};
    int tmass[MF_CH_MAX_FINAL] = {0};
    int tside[MF_CH_MAX_FINAL] = {0};   // F_j: final legs on the side of leg 0
    std::vector<Node> nodes;
};

// Binary tree of the s-clusters inside S, appended to nodes in pre-order;
// returns the node index, or -1 if some node has other than two children.
int cluster_tree(int S, const std::map<int, int> &s_mass, std::vector<Node> &nodes) {
    std::vector<int> maximal;
    for (const auto &kv : s_mass) {
        const int X = kv.first;
        if ((X & S) != X || X == S) continue;
        bool inside_other = false;
        for (const auto &kw : s_mass) {
            const int Y = kw.first;
            if (Y != X && Y != S && (Y & S) == Y && (X & Y) == X) inside_other = true;
        }
        if (!inside_other) maximal.push_back(X);
    }
    int covered = 0;
    for (int X : maximal) covered |= X;
    std::vector<int> parts = maximal;
    for (int i = 0; i < 31; ++i)
        if (((S & ~covered) >> i) & 1) parts.push_back(1 << i);
    if (parts.size() != 2) return -1;
    std::sort(parts.begin(), parts.end(), [](int a, int b) { return lowest(a) < lowest(b); });
    const int idx = (int)nodes.size();
    nodes.push_back({S, s_mass.at(S), 0, 0});
    int kid[2];
    for (int side = 0; side < 2; ++side) {
        if (popcount(parts[side]) >= 2) {
            kid[side] = cluster_tree(parts[side], s_mass, nodes);
            if (kid[side] < 0) return -1;
        } else {
            kid[side] = -1 - lowest(parts[side]);
        }
    }
    nodes[idx].left = kid[0];
    nodes[idx].right = kid[1];
    return idx;
}

}  // namespace

mf_status derive_channels(int n_legs, const std::vector<mf_op> &ops, ChannelSet &out) {
    out = ChannelSet();
    const int nout = n_legs - 2;
    if (nout < 2 || nout > MF_CH_MAX_FINAL) return MF_OK;     // no channels
    const int all_fin = (1 << nout) - 1;
    std::vector<int> mask(ops.size(), 0);
    for (size_t i = 0; i < ops.size(); ++i) {
        const mf_op &o = ops[i];
        if (o.kind == MF_OP_EXT) {
            mask[i] = 1 << o.leg;
        } else if (o.kind == MF_OP_CUR) {
            for (int a = 0; a < 4; ++a)
                if (o.in[a] >= 0) mask[i] |= mask[o.in[a]];
        }
    }
    std::map<std::vector<int>, Chan> found;
    for (size_t a = 0; a < ops.size(); ++a) {
        const mf_op &amp = ops[a];
        if (amp.kind != MF_OP_AMP || four_vertex(amp.routine)) continue;
        // the diagram's currents
        std::vector<int> stack, curs;
        for (int q = 0; q < 4; ++q)
            if (amp.in[q] >= 0) stack.push_back(amp.in[q]);
        bool skip = false;
        while (!stack.empty()) {
            const int i = stack.back();
            stack.pop_back();
            if (ops[i].kind != MF_OP_CUR) continue;
            if (four_vertex(ops[i].routine)) skip = true;
            curs.push_back(i);
            for (int q = 0; q < 4; ++q)
                if (ops[i].in[q] >= 0) stack.push_back(ops[i].in[q]);
        }
        if (skip) continue;
        std::map<int, int> s_mass, t_mass;
        for (int i : curs) {
            const int S = mask[i], fin = (S >> 2) & all_fin, m = ops[i].mass_id;
            const bool has_a = S & 1, has_b = (S >> 1) & 1;
            if (!has_a && !has_b) s_mass[fin] = m;
            else if (has_a && has_b) s_mass[all_fin & ~fin] = m;
            else t_mass[has_a ? fin : (all_fin & ~fin)] = m;
        }
        std::vector<int> F;
        for (const auto &kv : t_mass) F.push_back(kv.first);
        std::sort(F.begin(), F.end(), [](int x, int y) { return popcount(x) < popcount(y); });
        Chan ch;
        ch.k = (int)F.size() + 1;
        int prev = 0;
        bool bad = false;
        for (int j = 0; j < ch.k; ++j) {
            const int Fj = j < (int)F.size() ? F[j] : all_fin;
            if ((prev & Fj) != prev || prev == Fj) bad = true;
            ch.cmask[j] = Fj & ~prev;
            if (j < (int)F.size()) {
                ch.tmass[j] = t_mass[Fj];
                ch.tside[j] = Fj;
            }
            prev = Fj;
        }
        if (bad) continue;
        for (int j = 0; j < ch.k && !bad; ++j) {
            if (popcount(ch.cmask[j]) >= 2) {
                if (!s_mass.count(ch.cmask[j])) bad = true;
                else ch.cnode[j] = cluster_tree(ch.cmask[j], s_mass, ch.nodes);
                if (ch.cnode[j] < 0) bad = true;
            } else {
                ch.cnode[j] = -1;
            }
        }
        if (bad) continue;
        std::vector<int> key = {ch.k};
        for (int j = 0; j < ch.k; ++j) key.push_back(ch.cmask[j]);
        for (int j = 0; j + 1 < ch.k; ++j) key.push_back(ch.tmass[j]);
        std::vector<std::pair<int, int>> sl(s_mass.begin(), s_mass.end());
        std::sort(sl.begin(), sl.end());
        key.push_back((int)sl.size());
        for (const auto &pr : sl) {
            key.push_back(pr.first);
            key.push_back(pr.second);
        }
        found.emplace(key, ch);
    }
    // the table: distinct propagators, then the channels in key order
    std::vector<std::vector<int>> edge_of;    // per channel
    std::map<std::vector<int>, int> edge_index;
    std::vector<std::vector<int>> edges;
    for (const auto &kv : found) {
        const Chan &ch = kv.second;
        std::vector<int> mine;
        auto use = [&](int type, int m, int mass) {
            const std::vector<int> e = {type, m, mass};
            auto it = edge_index.find(e);
            if (it == edge_index.end()) {
                it = edge_index.emplace(e, (int)edges.size()).first;
                edges.push_back(e);
            }
            mine.push_back(it->second);
        };
        for (const Node &n : ch.nodes) use(0, n.mask, n.mass);
        for (int j = 0; j + 1 < ch.k; ++j) use(1, ch.tside[j], ch.tmass[j]);
        edge_of.push_back(mine);
        out.keys.push_back(kv.first);
    }
    const int K = (int)found.size(), E = (int)edges.size();
    if (K == 0) return MF_OK;
    if (E > MF_CH_MAX_EDGES) return fail(MF_EUNSUPPORTED, "too many distinct propagators for the channel table");
    out.K = K;
    out.table.assign(MF_CH_HDR + MF_CH_EDGE * E + MF_CH_STRIDE * K, 0);
    int32_t *t = out.table.data();
    t[0] = K;
    t[1] = E;
    t[2] = nout;
    for (int e = 0; e < E; ++e)
        for (int q = 0; q < 3; ++q) t[MF_CH_HDR + MF_CH_EDGE * e + q] = edges[e][q];
    int i = 0;
    for (const auto &kv : found) {
        const Chan &ch = kv.second;
        int32_t *c = t + MF_CH_HDR + MF_CH_EDGE * E + MF_CH_STRIDE * i;
        c[MF_CH_K] = ch.k;
        c[MF_CH_NNODE] = (int)ch.nodes.size();
        c[MF_CH_NEDGE] = (int)edge_of[i].size();
        for (int j = 0; j < MF_CH_MAX_FINAL; ++j) {
            c[MF_CH_CMASK + j] = j < ch.k ? ch.cmask[j] : 0;
            c[MF_CH_CNODE + j] = j < ch.k ? ch.cnode[j] : -1;
            c[MF_CH_TMASS + j] = j + 1 < ch.k ? ch.tmass[j] : -1;
        }
        for (size_t a = 0; a < edge_of[i].size(); ++a) c[MF_CH_EDGES + a] = edge_of[i][a];
        for (size_t nd = 0; nd < ch.nodes.size(); ++nd) {
            int32_t *r = c + MF_CH_NODES + MF_CH_NODE_W * nd;
            r[0] = ch.nodes[nd].mask;
            r[1] = ch.nodes[nd].mass;
            r[2] = ch.nodes[nd].left;
            r[3] = ch.nodes[nd].right;
        }
        ++i;
    }
    return MF_OK;
}

}  // namespace mfi

namespace {

mf_status channels_of_desc(const mf_process_desc *d, mfi::ChannelSet &cs) {
    if (!d || !d->ops || d->n_ops < 1 || d->n_legs < 3 || d->n_legs > MF_MAX_LEGS)
        return mfi::fail(MF_EINVAL, "bad descriptor");
    for (int i = 0; i < d->n_ops; ++i) {
        const mf_op &o = d->ops[i];
        if (o.kind == MF_OP_EXT && (o.leg < 0 || o.leg >= d->n_legs)) return mfi::fail(MF_EINVAL, "bad leg");
        for (int a = 0; a < 4; ++a)
            if (o.in[a] >= i || o.in[a] < -1) return mfi::fail(MF_EINVAL, "op input out of order");
    }
    std::vector<mf_op> ops(d->ops, d->ops + d->n_ops);
    return mfi::derive_channels(d->n_legs, ops, cs);
}

}  // namespace

extern "C" mf_status mf_channels_describe(const mf_process_desc *d, int32_t *n_channels, int32_t *keys,
                                          int32_t key_stride) {
    if (!n_channels) return mfi::fail(MF_EINVAL, "n_channels is NULL");
    mfi::ChannelSet cs;
    mf_status st = channels_of_desc(d, cs);
    if (st != MF_OK) return st;
    *n_channels = cs.K;
    if (!keys) return MF_OK;
    for (int i = 0; i < cs.K; ++i) {
        const std::vector<int> &k = cs.keys[i];
        if ((int)k.size() + 1 > key_stride) return mfi::fail(MF_EINVAL, "key_stride too small");
        keys[i * key_stride] = (int32_t)k.size();
        for (size_t a = 0; a < k.size(); ++a) keys[i * key_stride + 1 + a] = k[a];
    }
    return MF_OK;
}

extern "C" mf_status mf_channels_table(const mf_process_desc *d, int32_t *table, int32_t *len) {
    if (!len) return mfi::fail(MF_EINVAL, "len is NULL");
    mfi::ChannelSet cs;
    mf_status st = channels_of_desc(d, cs);
    if (st != MF_OK) return st;
    const int32_t need = (int32_t)cs.table.size();
    if (table && *len < need) return mfi::fail(MF_EINVAL, "table buffer too small");
    *len = need;
    if (table) std::copy(cs.table.begin(), cs.table.end(), table);
    return MF_OK;
}

extern "C" mf_status mf_channels_allocate(int32_t n_channels, const double *sigma, const int64_t *n_prev, double m0,
                                          int64_t n_total, int64_t n_floor, int64_t *n_out) {
    if (n_channels < 1 || !sigma || !n_out || n_floor < 0) return mfi::fail(MF_EINVAL, "bad arguments");
    if (!(m0 >= 0.0) || !std::isfinite(m0)) return mfi::fail(MF_EINVAL, "bad m0");
    const int64_t free_pts = n_total - (int64_t)n_channels * n_floor;
    if (free_pts < 0) return mfi::fail(MF_EINVAL, "fewer points than the floors need");
    std::vector<double> sg(n_channels);
    for (int i = 0; i < n_channels; ++i) {
        if (!(sigma[i] >= 0.0) || !std::isfinite(sigma[i])) return mfi::fail(MF_EINVAL, "bad sigma");
        if (n_prev && n_prev[i] < 0) return mfi::fail(MF_EINVAL, "bad n_prev");
        sg[i] = sigma[i];
    }
    if (n_prev) {
        // shrink every deviation towards the pooled one (m0 pseudo-points)
        double num = 0.0, den = 0.0;
        for (int i = 0; i < n_channels; ++i) {
            num += (double)n_prev[i] * sigma[i] * sigma[i];
            den += (double)n_prev[i];
        }
        const double pooled = den > 0.0 ? num / den : 0.0;
        for (int i = 0; i < n_channels; ++i) {
            const double n = (double)n_prev[i];
            sg[i] = n + m0 > 0.0 ? std::sqrt((n * sigma[i] * sigma[i] + m0 * pooled) / (n + m0)) : 0.0;
        }
    }
    double S = 0.0;
    for (int i = 0; i < n_channels; ++i) S += sg[i];
    for (int i = 0; i < n_channels; ++i)
        n_out[i] = S > 0.0 ? n_floor + (int64_t)std::floor((double)free_pts * (sg[i] / S))
                           : n_floor + free_pts / n_channels;
    return MF_OK;
}
