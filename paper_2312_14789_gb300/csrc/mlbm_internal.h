// Internal declarations shared by the library's translation units (host
// stencil builder, CUDA step kernels, C-ABI glue).  Not part of the ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mlbm.h"

namespace mlbm {

// D2Q9 velocity set in the paper's order (Eq. (2)); weights (Eq. (8)).
constexpr int kQ = 9;
constexpr int kEx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
constexpr int kEy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
constexpr int kOpp[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

enum Kind : uint8_t { kKindWls = 0, kKindLagrange = 1, kKindEq = 2 };

// Host-side result of mlbm_build_stencils, already in the Hilbert order the
// device uses ("position" p = 0..n-1); perm[p] is the caller's node id.
struct HostStencils {
    int64_t n = 0;
    int K = 0;
    double s = 1.0;
    int bb_mode = 0;
    double box_area = 0.0;
    std::vector<int64_t> perm;     // position -> caller id
    std::vector<int64_t> inv;      // caller id -> position
    std::vector<int32_t> idx;      // [n][K] neighbour positions, search order
    std::vector<double> M;         // [n][6][K] least-squares matrix, units of s
    int interp = 0;                // MLBM_INTERP_*
    std::vector<double> Wr;        // [n][8][K] RBF-FD weights of directions 1..8 (RBF stencils)
    std::vector<uint8_t> kind;     // Kind
    std::vector<uint8_t> center;   // Lagrange block centre direction m
    std::vector<double> lag_h;     // Lagrange block spacing
    std::vector<int8_t> lag_slot;  // [n][9] stencil slot of block point (a, b)
    std::vector<uint16_t> link_mask;
    std::vector<double> q;         // [n][9]
    std::vector<double> eqv;       // [n][3] rho_b, ux_b, uy_b
    std::vector<double> area;      // [n]
    // batches: streaming distance of each node (empty: s for all)
    std::vector<double> s_node;
    // node positions in the caller's order and the box, for re-ordering
    std::vector<double> xy;
    double bx0 = 0, by0 = 0, blx = 1, bly = 1;
    int order = 0;  // MLBM_ORDER_*
    mlbm_stencil_info info{};
    // partitions of a node set (see PartPlan): state slots beyond the n nodes
    // for the halo copies of other partitions' nodes, and the key that orders
    // each node's stencil slots on the device (the unpartitioned positions, so
    // that a partition sums its stencil in the same order; idx when empty)
    int64_t n_halo = 0;
    std::vector<int64_t> slot_key;  // [n][K]
    // a batch's concatenation keeps no M or Wr of its own: the rows of node q
    // of sample i (part_off[i] <= q < part_off[i + 1]) are read from that
    // sample's stencils, part_M[i] (and part_Wr[i]) at q - part_off[i]
    std::vector<const double*> part_M, part_Wr;
    std::vector<int64_t> part_off;
};

// Partition of a node set into contiguous ranges of device positions (Hilbert
// order): partition q owns positions [bounds[q], bounds[q + 1]); its halo is
// every position outside the range that its nodes' stencils reference,
// grouped by owning partition and ascending within a group.
struct PartPlan {
    int P = 0;
    std::vector<int64_t> bounds;                  // [P + 1]
    std::vector<std::vector<int64_t>> halo;       // [P][n_halo_q] positions
    std::vector<std::vector<int64_t>> halo_off;   // [P][P + 1] start of owner o's block in halo[q]
};

mlbm_status make_part_plan(const HostStencils& H, int P, const int64_t* bounds, PartPlan& out);
// host stencils of partition q: its owned nodes in local positions
// 0..n_owned-1 and its halo at n_owned.., perm / inv the identity
HostStencils slice_partition(const HostStencils& H, const PartPlan& plan, int q);

}  // namespace mlbm

struct mlbm_stencils {
    mlbm::HostStencils h;
};

// error reporting shared by all translation units
namespace mlbm {
mlbm_status set_error(mlbm_status st, const std::string& msg);
void clear_error();
}  // namespace mlbm
