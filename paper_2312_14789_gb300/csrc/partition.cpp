// Partitioning a node set for the partitioned step (host side).
//
// The step of a node reads only the post-collision state of its own stencil
// members (the streaming of Sec. 2.2, Eq. (12)), so a node set split into
// contiguous ranges of its Hilbert-ordered positions can be advanced range by
// range if every range first receives copies of the members it references
// but does not own (its halo).  This file builds that plan and the per-range
// host stencils; the device side (state buffers with halo slots, the copies
// after each step) is in context.cu.
#include <algorithm>
#include <string>
#include <type_traits>

#include "mlbm_internal.h"

namespace mlbm {

mlbm_status make_part_plan(const HostStencils& H, int P, const int64_t* bounds, PartPlan& out) {
    if (P < 1 || (int64_t)P > std::max<int64_t>(H.n, 1))
        return set_error(MLBM_E_INVALID, "partition: need 1 <= parts <= nodes");
    out = PartPlan{};
    out.P = P;
    out.bounds.resize((size_t)P + 1);
    if (bounds) {
        for (int q = 0; q <= P; ++q) out.bounds[q] = bounds[q];
        if (out.bounds[0] != 0 || out.bounds[P] != H.n)
            return set_error(MLBM_E_INVALID, "partition: bounds must start at 0 and end at the node count");
        for (int q = 0; q < P; ++q)
            if (out.bounds[q + 1] <= out.bounds[q])
                return set_error(MLBM_E_INVALID, "partition: bounds must increase strictly");
    } else {
        for (int q = 0; q <= P; ++q) out.bounds[q] = H.n * q / P;
    }
    const int K = H.K;
    out.halo.assign(P, {});
    out.halo_off.assign(P, std::vector<int64_t>((size_t)P + 1, 0));
    for (int q = 0; q < P; ++q) {
        const int64_t a = out.bounds[q], e = out.bounds[q + 1];
        std::vector<int64_t>& h = out.halo[q];
        for (int64_t p = a; p < e; ++p)
            for (int j = 0; j < K; ++j) {
                const int64_t m = H.idx[(size_t)p * K + j];
                if (m < a || m >= e) h.push_back(m);
            }
        // ascending positions are also grouped by owner, the ranges being
        // contiguous and in order
        std::sort(h.begin(), h.end());
        h.erase(std::unique(h.begin(), h.end()), h.end());
        for (int o = 0; o <= P; ++o)
            out.halo_off[q][o] = std::lower_bound(h.begin(), h.end(), out.bounds[o]) - h.begin();
    }
    return MLBM_OK;
}

HostStencils slice_partition(const HostStencils& H, const PartPlan& plan, int q) {
    const int K = H.K;
    const int64_t a = plan.bounds[q], e = plan.bounds[q + 1], n = e - a;
    const std::vector<int64_t>& halo = plan.halo[q];
    auto local = [&](int64_t m) -> int32_t {
        if (m >= a && m < e) return (int32_t)(m - a);
        return (int32_t)(n + (std::lower_bound(halo.begin(), halo.end(), m) - halo.begin()));
    };
    HostStencils S;
    S.n = n;
    S.K = K;
    S.s = H.s;
    S.bb_mode = H.bb_mode;
    S.box_area = H.box_area;
    S.interp = H.interp;
    S.order = H.order;
    S.bx0 = H.bx0;
    S.by0 = H.by0;
    S.blx = H.blx;
    S.bly = H.bly;
    S.n_halo = (int64_t)halo.size();
    S.perm.resize(n);
    S.inv.resize(n);
    S.idx.resize((size_t)n * K);
    S.slot_key.resize((size_t)n * K);
    for (int64_t p = 0; p < n; ++p) {
        S.perm[p] = p;
        S.inv[p] = p;
        for (int j = 0; j < K; ++j) {
            const int64_t m = H.idx[(size_t)(a + p) * K + j];
            S.idx[(size_t)p * K + j] = local(m);
            S.slot_key[(size_t)p * K + j] = m;
        }
    }
    auto cut = [&](const auto& v, size_t per) {
        using T = typename std::decay_t<decltype(v)>::value_type;
        if (v.empty()) return std::vector<T>();
        return std::vector<T>(v.begin() + (size_t)a * per, v.begin() + (size_t)e * per);
    };
    S.M = cut(H.M, (size_t)6 * K);
    S.Wr = cut(H.Wr, (size_t)8 * K);
    S.kind = cut(H.kind, 1);
    S.center = cut(H.center, 1);
    S.lag_h = cut(H.lag_h, 1);
    S.lag_slot = cut(H.lag_slot, 9);
    S.link_mask = cut(H.link_mask, 1);
    S.q = cut(H.q, 9);
    S.eqv = cut(H.eqv, 3);
    S.area = cut(H.area, 1);
    S.s_node = cut(H.s_node, 1);
    if (!H.xy.empty()) {
        S.xy.resize((size_t)n * 2);
        for (int64_t p = 0; p < n; ++p) {
            S.xy[(size_t)p * 2] = H.xy[(size_t)H.perm[a + p] * 2];
            S.xy[(size_t)p * 2 + 1] = H.xy[(size_t)H.perm[a + p] * 2 + 1];
        }
    }
    S.info = H.info;
    S.info.n = n;
    S.info.n_wls = S.info.n_lagrange = S.info.n_eq = S.info.n_link_nodes = S.info.n_links = 0;
    for (int64_t p = 0; p < n; ++p) {
        if (S.kind[p] == kKindWls) ++S.info.n_wls;
        else if (S.kind[p] == kKindLagrange) ++S.info.n_lagrange;
        else ++S.info.n_eq;
        if (S.link_mask[p]) {
            ++S.info.n_link_nodes;
            S.info.n_links += __builtin_popcount((unsigned)S.link_mask[p]);
        }
    }
    return S;
}

}  // namespace mlbm

extern "C" mlbm_status mlbm_partition_plan(const mlbm_stencils* st, int n_parts, const int64_t* bounds,
                                           int64_t* first, int64_t* n_owned, int64_t* n_halo,
                                           int64_t* halo_from) {
    mlbm::clear_error();
    if (!st) return mlbm::set_error(MLBM_E_INVALID, "partition_plan: NULL stencils");
    mlbm::PartPlan plan;
    mlbm_status s = mlbm::make_part_plan(st->h, n_parts, bounds, plan);
    if (s != MLBM_OK) return s;
    for (int q = 0; q < n_parts; ++q) {
        if (first) first[q] = plan.bounds[q];
        if (n_owned) n_owned[q] = plan.bounds[q + 1] - plan.bounds[q];
        if (n_halo) n_halo[q] = (int64_t)plan.halo[q].size();
        if (halo_from)
            for (int o = 0; o < n_parts; ++o)
                halo_from[(size_t)q * n_parts + o] = plan.halo_off[q][o + 1] - plan.halo_off[q][o];
    }
    return MLBM_OK;
}

extern "C" mlbm_status mlbm_partition_nodes(const mlbm_stencils* st, int n_parts, const int64_t* bounds, int part,
                                            int64_t* owned_ids, int64_t* halo_ids) {
    mlbm::clear_error();
    if (!st) return mlbm::set_error(MLBM_E_INVALID, "partition_nodes: NULL stencils");
    mlbm::PartPlan plan;
    mlbm_status s = mlbm::make_part_plan(st->h, n_parts, bounds, plan);
    if (s != MLBM_OK) return s;
    if (part < 0 || part >= n_parts) return mlbm::set_error(MLBM_E_INVALID, "partition_nodes: bad part");
    if (owned_ids)
        for (int64_t p = plan.bounds[part]; p < plan.bounds[part + 1]; ++p)
            owned_ids[p - plan.bounds[part]] = st->h.perm[p];
    if (halo_ids)
        for (size_t i = 0; i < plan.halo[part].size(); ++i) halo_ids[i] = st->h.perm[plan.halo[part][i]];
    return MLBM_OK;
}
