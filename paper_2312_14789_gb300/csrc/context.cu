// C-ABI glue: simulation contexts, state I/O, the step loop and observables.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.h"
#include "mlbm_internal.h"

namespace mlbm {

thread_local std::string g_last_error;

mlbm_status set_error(mlbm_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}
void clear_error() { g_last_error.clear(); }

}  // namespace mlbm

using namespace mlbm;

struct mlbm_ctx {
    int device = 0;
    mlbm_params params{};
    int64_t n = 0, n_pad = 0;
    int64_t n_halo = 0;  // state slots after the n nodes (partitions only)
    int K = 0;
    double s = 1.0, box_area = 1.0;
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;
    // stencil data on the device
    int4* idx = nullptr;
    float4* M = nullptr;
    uint8_t* meta = nullptr;
    float* lag_r = nullptr;
    int* link_slot = nullptr;
    dev::LinkRec* links = nullptr;
    float4* eqv = nullptr;
    int* perm = nullptr;
    float* area = nullptr;
    float* area_over_s2 = nullptr;
    uint8_t* mask = nullptr;
    int* link_nodes = nullptr;
    int n_link_nodes = 0;
    // state
    float4* f8[2] = {nullptr, nullptr};
    float* f0[2] = {nullptr, nullptr};
    float4* ruv[2] = {nullptr, nullptr};
    int cur = 0;
    // work
    float *rho = nullptr, *ux = nullptr, *uy = nullptr, *px = nullptr, *py = nullptr;
    double* io = nullptr;
    double* scratch = nullptr;
    int64_t scratch_len = 0;
    double* small = nullptr;
    int64_t steps = 0;
    int64_t steps_in_last_run = 0;  // steps taken by the last run to steady state
    bool timing = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    double last_ms = -1.0;
    int variant = 25;
    std::vector<int> inv_perm;  // caller's node id -> device position
    int* err = nullptr;  // device error word of the bounded waits
    dev::Stencil S{};
    dev::Collide C{};
    std::vector<void*> allocations;
    // batch of independent samples (empty for a single sample)
    std::vector<int64_t> seg_off;  // position offset of each sample, plus the total
    std::vector<mlbm_params> seg_params;
    std::vector<double> seg_box_area;
    std::vector<double> seg_s;  // streaming distance of each sample
    double* seg_out = nullptr;  // device, 6 doubles per sample
    // captured step graphs: chunk of kGraphSteps steps starting from buffer 0 / 1
    bool use_graphs = true;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int graph_variant = -1;
    cudaStream_t graph_stream = nullptr;
    // bounded waits of the bulk-copy ring variants (4..7): budget of one wait,
    // and the test switch that makes the next launch withhold one tile
    unsigned long long wait_ns = 2000000000ULL;
    int withhold_next = 0;
    // device buffer of mlbm_wall_stress_force, grown on demand and kept:
    // positions, normals, lengths and tractions of up to wall_cap wall nodes
    uint8_t* wall_buf = nullptr;
    int64_t wall_cap = 0;
    // per-step time of every variant in the last autotune (-1: not timed)
    std::vector<double> tune_ms;
};

namespace {
constexpr int kGraphSteps = 16;
constexpr int kMaxK = 64;  // widest device stencil (RBF-FD unions per Lagrangian point)
constexpr int kMaxVariant = 29;  // step kernel variants 0..29 (see mlbm_set_kernel_variant)
}

// Cold-cache start for timed steps: reading a zeroed buffer several times the
// size of L2 leaves L2 holding clean lines of that buffer only, so a timed
// step neither hits its own data nor pays for writing back dirty lines left
// by whatever ran before (which a memset flush would leave behind).
__global__ void l2_flush_read(const float4* __restrict__ buf, size_t n, float* sink) {
    float acc = 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float4 v = __ldcg(buf + i);
        acc += (v.x + v.y) + (v.z + v.w);
    }
    if (acc != 0.f) *sink = acc;  // never taken on the zeroed buffer; keeps the loads
}

// Sending side of a halo copy: the states of the listed positions into one
// contiguous block, w float4 per node (out[i*w + c] = in[list[i]*w + c]).
__global__ void gather_states(const float4* __restrict__ in, const int* __restrict__ list, int64_t m, int w,
                              float4* __restrict__ out) {
    const int64_t total = m * w;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t node = i / w;
        const int c = (int)(i - node * w);
        out[i] = in[(size_t)list[node] * w + c];
    }
}

namespace {

#define MLBM_CUDA(call)                                                                                      \
    do {                                                                                                     \
        cudaError_t e_ = (call);                                                                             \
        if (e_ != cudaSuccess)                                                                               \
            return set_error(MLBM_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));               \
    } while (0)

template <class T>
mlbm_status dalloc(mlbm_ctx* c, T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return set_error(e == cudaErrorMemoryAllocation ? MLBM_E_OOM : MLBM_E_CUDA,
                         std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    c->allocations.push_back(q);
    *p = static_cast<T*>(q);
    return MLBM_OK;
}

#define MLBM_TRY(expr)                       \
    do {                                     \
        mlbm_status s_ = (expr);             \
        if (s_ != MLBM_OK) return s_;        \
    } while (0)

mlbm_status upload(mlbm_ctx* c, void* dst, const void* src, size_t bytes) {
    MLBM_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream));
    return MLBM_OK;
}

void set_collide(mlbm_ctx* c) {
    const double tp = c->params.tau;
    const double tm = c->params.tau_minus > 0 ? c->params.tau_minus : tp;
    c->C.omega_p = (float)(1.0 / tp);
    c->C.omega_m = (float)(1.0 / tm);
    c->C.src_p = (float)(1.0 - 0.5 / tp);
    c->C.src_m = (float)(1.0 - 0.5 / tm);
    c->C.ax = (float)c->params.gx;
    c->C.ay = (float)c->params.gy;
}

mlbm_status check_params(const mlbm_params* p) {
    if (p->model != MLBM_MODEL_BGK && p->model != MLBM_MODEL_TAU1) return set_error(MLBM_E_INVALID, "bad model");
    if (!(p->tau > 0.5) || !std::isfinite(p->tau)) return set_error(MLBM_E_INVALID, "tau must be > 1/2");
    if (p->tau_minus > 0 && !(p->tau_minus > 0.5)) return set_error(MLBM_E_INVALID, "tau_minus must be > 1/2");
    if (p->model == MLBM_MODEL_TAU1 && (p->tau != 1.0 || (p->tau_minus > 0 && p->tau_minus != 1.0)))
        return set_error(MLBM_E_INVALID, "the tau = 1 model needs tau = tau_minus = 1");
    if (!std::isfinite(p->gx) || !std::isfinite(p->gy)) return set_error(MLBM_E_INVALID, "non-finite body force");
    return MLBM_OK;
}

mlbm_status sync(mlbm_ctx* c) {
    MLBM_CUDA(cudaStreamSynchronize(c->stream));
    if (c->err) {
        int e = 0;
        MLBM_CUDA(cudaMemcpyAsync(&e, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        MLBM_CUDA(cudaStreamSynchronize(c->stream));
        if (e != 0) {
            // cleared in stream order, before any later launch can set it again
            MLBM_CUDA(cudaMemsetAsync(c->err, 0, sizeof(int), c->stream));
            MLBM_CUDA(cudaStreamSynchronize(c->stream));
            return set_error(MLBM_E_TIMEOUT, "a bounded device wait gave up (code " + std::to_string(e) +
                                                 "); the step result is invalid");
        }
    }
    return MLBM_OK;
}

mlbm_status launch_one_step(mlbm_ctx* c, int variant) {
    const int a = c->cur, b = c->cur ^ 1;
    const int model = c->params.model == MLBM_MODEL_BGK ? 0 : 1;
    if (((variant >= 4 && variant <= 7) || (variant >= 27 && variant <= 29)) && !c->S.Wr) {
        const dev::Wait W{c->wait_ns, c->withhold_next};
        c->withhold_next = 0;
        if (variant <= 7)
            MLBM_CUDA(launch_step_tma(variant, model, c->S, c->f8[a], c->f0[a], c->f8[b], c->f0[b], c->ruv[a],
                                      c->ruv[b], c->C, c->err, W, c->stream));
        else
            MLBM_CUDA(launch_step_ring1(variant, model, c->S, c->f8[a], c->f0[a], c->f8[b], c->f0[b], c->ruv[a],
                                        c->ruv[b], c->C, c->err, W, c->stream));
    }
    else if (model == 0)
        MLBM_CUDA(launch_bgk_step(c->S, c->f8[a], c->f0[a], c->f8[b], c->f0[b], c->C, variant, c->stream));
    else
        MLBM_CUDA(launch_tau1_step(c->S, c->ruv[a], c->ruv[b], c->C, variant, c->stream));
    c->cur = b;
    return MLBM_OK;
}

mlbm_status do_init(mlbm_ctx* c, const mlbm_stencils* st, const mlbm_params* p, const double* rho0, const double* u0) {
    const HostStencils& H = st->h;
    MLBM_CUDA(cudaGetDevice(&c->device));
    MLBM_CUDA(cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking));
    c->stream = c->own_stream;
    c->params = *p;
    c->n = H.n;
    c->K = H.K;
    c->s = H.s;
    c->box_area = H.box_area;
    c->n_pad = (H.n + 127) / 128 * 128;
    const int64_t n = H.n, np = c->n_pad;
    if (H.K < 4 || H.K > kMaxK || H.K % 4 != 0)
        return set_error(MLBM_E_INVALID, "init: stencil width must be a multiple of 4 in [4, 64]");
    // state slots: the nodes, then the halo copies of a partition's neighbours
    c->n_halo = H.n_halo;
    const int64_t nps = (H.n + H.n_halo + 127) / 128 * 128;
    const int K = H.K, Kq = K / 4;
    // ---- host-side device layout
    const bool rbf = H.interp != MLBM_INTERP_WLS;  // per-direction RBF-FD weights
    std::vector<int32_t> hidx((size_t)Kq * np * 4, 0);
    std::vector<float> hM((size_t)6 * Kq * np * 4, 0.f);
    std::vector<float> hW(rbf ? (size_t)8 * Kq * np * 4 : 0, 0.f);
    std::vector<uint8_t> hmeta(np, 0), hmask(np, 0);
    std::vector<float> hlag(np, 0.f), harea(np, 0.f), has2(np, 0.f);
    std::vector<int> hslot(np, -1), hperm(np, 0), hlinknodes;
    std::vector<dev::LinkRec> hlinks;
    std::vector<float4> heqv(np, make_float4(0, 0, 0, 0));
    // link records in node order: their slots first, then every node's rows
    // in parallel (each node writes only its own positions)
    for (int64_t q = 0; q < n; ++q)
        if (H.link_mask[q]) {
            hslot[q] = (int)hlinknodes.size();
            hlinknodes.push_back((int)q);
        }
    hlinks.resize(hlinknodes.size());
    const bool parts = !H.part_off.empty();
#pragma omp parallel for schedule(static, 4096)
    for (int64_t q = 0; q < n; ++q) {
        const uint8_t kind = H.kind[q];
        const uint16_t lm = H.link_mask[q];
        hmeta[q] = (uint8_t)(kind | (lm ? 4 : 0) | (H.center[q] << 4));
        hmask[q] = kind != kKindEq;
        hperm[q] = (int)H.perm[q];
        harea[q] = (float)H.area[q];
        const double sq = H.s_node.empty() ? H.s : H.s_node[q];
        has2[q] = (float)(H.area[q] / (sq * sq));
        if (kind == kKindWls) {
            // stencil slots in increasing node position: lanes of a warp that
            // gather slot j of consecutive (Hilbert-ordered) nodes then touch
            // nearby addresses; the matrix columns follow the same order
            int order[kMaxK];
            for (int j = 0; j < K; ++j) order[j] = j;
            if (H.slot_key.empty())
                std::sort(order, order + K,
                          [&](int a, int b) { return H.idx[(size_t)q * K + a] < H.idx[(size_t)q * K + b]; });
            else
                std::sort(order, order + K, [&](int a, int b) {
                    return H.slot_key[(size_t)q * K + a] < H.slot_key[(size_t)q * K + b];
                });
            // the node's matrix (and RBF-FD weight) rows: its own, or its sample's
            const double* Mq;
            const double* Wq = nullptr;
            if (parts) {
                const size_t i =
                    (size_t)(std::upper_bound(H.part_off.begin(), H.part_off.end(), q) - H.part_off.begin()) - 1;
                const size_t l = (size_t)(q - H.part_off[i]);
                Mq = H.part_M[i] + l * 6 * K;
                if (rbf) Wq = H.part_Wr[i] + l * 8 * K;
            } else {
                Mq = H.M.data() + (size_t)q * 6 * K;
                if (rbf) Wq = H.Wr.data() + (size_t)q * 8 * K;
            }
            for (int jj = 0; jj < K; ++jj) {
                const int j = order[jj];
                hidx[(((size_t)(jj / 4)) * np + q) * 4 + (jj % 4)] = H.idx[(size_t)q * K + j];
                double m[6];
                for (int a = 0; a < 6; ++a) m[a] = Mq[(size_t)a * K + j];
                // D2Q9 departure basis (see device_common.cuh), formed in FP64
                const double t[6] = {m[0] + m[3], m[0] + m[5], m[0] + m[3] + m[4] + m[5], m[0] + m[3] - m[4] + m[5],
                                     m[1], m[2]};
                for (int a = 0; a < 6; ++a)
                    hM[(((size_t)(a * Kq + jj / 4)) * np + q) * 4 + (jj % 4)] = (float)t[a];
                if (rbf)
                    for (int k = 0; k < 8; ++k)
                        hW[(((size_t)(k * Kq + jj / 4)) * np + q) * 4 + (jj % 4)] =
                            (float)Wq[(size_t)k * K + j];
            }
        } else if (kind == kKindLagrange) {
            for (int b = 0; b < 9; ++b) {
                const int j = H.lag_slot[(size_t)q * 9 + b];
                hidx[(((size_t)(b / 4)) * np + q) * 4 + (b % 4)] = H.idx[(size_t)q * K + j];
            }
            hlag[q] = (float)(sq / H.lag_h[q]);
        } else {
            heqv[q] = make_float4((float)(H.eqv[q * 3] - 1.0), (float)H.eqv[q * 3 + 1], (float)H.eqv[q * 3 + 2], 0.f);
        }
        if (lm) {
            dev::LinkRec r{};
            r.mask = lm;
            for (int k = 1; k < 9; ++k) r.t[k - 1] = (float)(1.0 - 2.0 * H.q[(size_t)q * 9 + k]);
            hlinks[(size_t)hslot[q]] = r;
        }
    }
    c->n_link_nodes = (int)hlinknodes.size();
    c->inv_perm.assign((size_t)n, -1);
    for (int64_t q = 0; q < n; ++q) c->inv_perm[(size_t)hperm[q]] = (int)q;
    // ---- neighbourhood staging (variant 22, least-squares BGK): per tile of
    // kStageTile nodes the sorted union of the stencil members of its
    // least-squares nodes without links, and each member's local index
    std::vector<uint16_t> hlidx;
    std::vector<int> hsoff, hsids;
    int stage_max = 0;
    if (p->model == MLBM_MODEL_BGK && !rbf && tma_supported(Kq)) {
        const int64_t T = dev::kStageTile, nt = (n + T - 1) / T;
        std::vector<std::vector<int>> lists((size_t)nt);
        hlidx.assign((size_t)Kq * np * 4, 0);
#pragma omp parallel for schedule(dynamic, 8)
        for (int64_t b = 0; b < nt; ++b) {
            std::vector<int>& L = lists[(size_t)b];
            const int64_t q0 = b * T, q1 = std::min<int64_t>(n, q0 + T);
            for (int64_t q = q0; q < q1; ++q)
                if ((hmeta[q] & 7) == 0)
                    for (int jj = 0; jj < K; ++jj) L.push_back(hidx[(((size_t)(jj / 4)) * np + q) * 4 + (jj % 4)]);
            std::sort(L.begin(), L.end());
            L.erase(std::unique(L.begin(), L.end()), L.end());
            if ((int64_t)L.size() > dev::kStageMax) continue;  // too wide: the whole structure is dropped below
            for (int64_t q = q0; q < q1; ++q)
                if ((hmeta[q] & 7) == 0)
                    for (int jj = 0; jj < K; ++jj) {
                        const size_t at = (((size_t)(jj / 4)) * np + q) * 4 + (jj % 4);
                        hlidx[at] = (uint16_t)(std::lower_bound(L.begin(), L.end(), hidx[at]) - L.begin());
                    }
        }
        hsoff.assign((size_t)nt + 1, 0);
        for (int64_t b = 0; b < nt; ++b) {
            stage_max = std::max(stage_max, (int)lists[(size_t)b].size());
            hsoff[(size_t)b + 1] = hsoff[(size_t)b] + (int)lists[(size_t)b].size();
        }
        if (stage_max <= dev::kStageMax && (int64_t)hsoff.back() < (int64_t)1 << 30) {
            hsids.reserve((size_t)hsoff.back() + 8);
            for (const auto& L : lists) hsids.insert(hsids.end(), L.begin(), L.end());
            hsids.resize((size_t)hsoff.back() + 8, 0);  // the L2 prefetch reads whole 16-byte groups
        } else {
            hlidx.clear();
            hsoff.clear();
            stage_max = 0;
        }
    }
    // ---- device buffers
    MLBM_TRY(dalloc(c, &c->idx, (size_t)Kq * np));
    MLBM_TRY(dalloc(c, &c->M, (size_t)6 * Kq * np));
    float4* dW = nullptr;
    if (rbf) MLBM_TRY(dalloc(c, &dW, (size_t)8 * Kq * np));
    MLBM_TRY(dalloc(c, &c->meta, np));
    MLBM_TRY(dalloc(c, &c->mask, np));
    MLBM_TRY(dalloc(c, &c->lag_r, np));
    MLBM_TRY(dalloc(c, &c->link_slot, np));
    MLBM_TRY(dalloc(c, &c->links, hlinks.size()));
    MLBM_TRY(dalloc(c, &c->link_nodes, hlinknodes.size()));
    MLBM_TRY(dalloc(c, &c->eqv, np));
    MLBM_TRY(dalloc(c, &c->perm, np));
    MLBM_TRY(dalloc(c, &c->area, np));
    MLBM_TRY(dalloc(c, &c->area_over_s2, np));
    for (int b = 0; b < 2; ++b) {
        if (p->model == MLBM_MODEL_BGK) {
            MLBM_TRY(dalloc(c, &c->f8[b], (size_t)2 * nps));
            MLBM_TRY(dalloc(c, &c->f0[b], nps));
        } else {
            MLBM_TRY(dalloc(c, &c->ruv[b], nps));
        }
    }
    MLBM_TRY(dalloc(c, &c->rho, np));
    MLBM_TRY(dalloc(c, &c->ux, np));
    MLBM_TRY(dalloc(c, &c->uy, np));
    MLBM_TRY(dalloc(c, &c->px, np));
    MLBM_TRY(dalloc(c, &c->py, np));
    MLBM_TRY(dalloc(c, &c->io, (size_t)9 * np));
    c->scratch_len = std::max<int64_t>(6 * reduce_blocks(np), 2 * force_blocks(c->n_link_nodes));
    MLBM_TRY(dalloc(c, &c->scratch, c->scratch_len));
    MLBM_TRY(dalloc(c, &c->small, 16));
    if (c->seg_off.empty()) {
        c->seg_off = {0, n};
        c->seg_params = {*p};
        c->seg_box_area = {H.box_area};
    }
    MLBM_TRY(dalloc(c, &c->seg_out, 6 * (c->seg_off.size() - 1)));
    MLBM_TRY(dalloc(c, &c->err, 1));
    MLBM_CUDA(cudaMemsetAsync(c->err, 0, sizeof(int), c->stream));
    if (!tma_supported(Kq)) c->variant = 1;  // variants >= 4 exist for K in {12, 16, 24, 32}
    MLBM_TRY(upload(c, c->idx, hidx.data(), hidx.size() * 4));
    MLBM_TRY(upload(c, c->M, hM.data(), hM.size() * 4));
    if (rbf) MLBM_TRY(upload(c, dW, hW.data(), hW.size() * 4));
    MLBM_TRY(upload(c, c->meta, hmeta.data(), np));
    MLBM_TRY(upload(c, c->mask, hmask.data(), np));
    MLBM_TRY(upload(c, c->lag_r, hlag.data(), np * 4));
    MLBM_TRY(upload(c, c->link_slot, hslot.data(), np * 4));
    if (!hlinks.empty()) MLBM_TRY(upload(c, c->links, hlinks.data(), hlinks.size() * sizeof(dev::LinkRec)));
    if (!hlinknodes.empty()) MLBM_TRY(upload(c, c->link_nodes, hlinknodes.data(), hlinknodes.size() * 4));
    MLBM_TRY(upload(c, c->eqv, heqv.data(), np * sizeof(float4)));
    MLBM_TRY(upload(c, c->perm, hperm.data(), np * 4));
    MLBM_TRY(upload(c, c->area, harea.data(), np * 4));
    MLBM_TRY(upload(c, c->area_over_s2, has2.data(), np * 4));
    MLBM_CUDA(cudaMemsetAsync(c->px, 0, np * 4, c->stream));
    MLBM_CUDA(cudaMemsetAsync(c->py, 0, np * 4, c->stream));
    for (int b = 0; b < 2; ++b) {
        if (c->f8[b]) {
            MLBM_CUDA(cudaMemsetAsync(c->f8[b], 0, (size_t)2 * nps * sizeof(float4), c->stream));
            MLBM_CUDA(cudaMemsetAsync(c->f0[b], 0, nps * 4, c->stream));
        }
        if (c->ruv[b]) MLBM_CUDA(cudaMemsetAsync(c->ruv[b], 0, nps * sizeof(float4), c->stream));
    }
    c->S.n = (int)n;
    c->S.n_pad = (int)np;
    c->S.K = K;
    c->S.Kq = Kq;
    c->S.bb_mode = H.bb_mode;
    c->S.idx = c->idx;
    c->S.M = c->M;
    c->S.meta = c->meta;
    c->S.lag_r = c->lag_r;
    c->S.link_slot = c->link_slot;
    c->S.links = c->links;
    c->S.eqv = c->eqv;
    c->S.link_nodes = c->link_nodes;
    c->S.Wr = dW;
    c->S.n_link_nodes = c->n_link_nodes;
    c->S.lidx = nullptr;
    c->S.stage_off = nullptr;
    c->S.stage_ids = nullptr;
    c->S.stage_max = 0;
    if (!hsoff.empty()) {  // built (a context without least-squares nodes stages nothing)
        ushort4* dl = nullptr;
        int *doff = nullptr, *dids = nullptr;
        MLBM_TRY(dalloc(c, &dl, (size_t)Kq * np));
        MLBM_TRY(dalloc(c, &doff, hsoff.size()));
        MLBM_TRY(dalloc(c, &dids, hsids.size()));
        MLBM_TRY(upload(c, dl, hlidx.data(), hlidx.size() * 2));
        MLBM_TRY(upload(c, doff, hsoff.data(), hsoff.size() * 4));
        MLBM_TRY(upload(c, dids, hsids.data(), hsids.size() * 4));
        if (stage_max > 0) MLBM_CUDA(prepare_staged_step(Kq, stage_max));
        c->S.lidx = dl;
        c->S.stage_off = doff;
        c->S.stage_ids = dids;
        c->S.stage_max = stage_max;
    }
    set_collide(c);
    // ---- initial state
    std::vector<double> ru((size_t)n * 3);
    for (int64_t i = 0; i < n; ++i) {
        ru[i * 3] = rho0 ? rho0[i] : 1.0;
        ru[i * 3 + 1] = u0 ? u0[2 * i] : 0.0;
        ru[i * 3 + 2] = u0 ? u0[2 * i + 1] : 0.0;
    }
    MLBM_TRY(upload(c, c->io, ru.data(), ru.size() * 8));
    if (p->model == MLBM_MODEL_BGK) {
        MLBM_CUDA(launch_set_bgk_equilibrium((int)n, c->perm, c->io, c->f8[0], c->f0[0], c->stream));
    } else {
        MLBM_CUDA(launch_set_tau1((int)n, c->perm, c->io, c->ruv[0], c->stream));
    }
    MLBM_CUDA(cudaEventCreate(&c->ev0));
    MLBM_CUDA(cudaEventCreate(&c->ev1));
    return sync(c);
}

// instantiate the graph of kGraphSteps step launches that starts from buffer
// `parity` (capture only: nothing runs, and the state is left as it was)
mlbm_status ensure_graph(mlbm_ctx* c, int parity) {
    cudaGraphExec_t& ex = c->graph[parity];
    if (ex) return MLBM_OK;
    const int saved = c->cur, saved_withhold = c->withhold_next;
    c->cur = parity;
    c->withhold_next = 0;  // never captured into a graph
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (ee != cudaSuccess) {
        c->cur = saved;
        c->withhold_next = saved_withhold;
        return set_error(MLBM_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(ee));
    }
    mlbm_status cs = MLBM_OK;
    for (int i = 0; i < kGraphSteps && cs == MLBM_OK; ++i) cs = launch_one_step(c, c->variant);
    ee = cudaStreamEndCapture(c->stream, &g);
    c->cur = saved;  // an even number of launches returns to it as well
    c->withhold_next = saved_withhold;
    if (cs != MLBM_OK) {
        if (g) cudaGraphDestroy(g);
        return cs;
    }
    if (ee != cudaSuccess) return set_error(MLBM_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(ee));
    ee = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ee != cudaSuccess) {
        ex = nullptr;
        return set_error(MLBM_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ee));
    }
    return MLBM_OK;
}

// graphs are tied to the variant and stream they were captured with
void refresh_graphs(mlbm_ctx* c);

void drop_graphs(mlbm_ctx* c) {
    for (int i = 0; i < 2; ++i)
        if (c->graph[i]) {
            cudaGraphExecDestroy(c->graph[i]);
            c->graph[i] = nullptr;
        }
    c->graph_variant = -1;
}

void refresh_graphs(mlbm_ctx* c) {
    if (c->graph_variant != c->variant || c->graph_stream != c->stream) {
        drop_graphs(c);
        c->graph_variant = c->variant;
        c->graph_stream = c->stream;
    }
}

void free_ctx(mlbm_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    for (void* p : c->allocations) cudaFree(p);
    if (c->wall_buf) cudaFree(c->wall_buf);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    delete c;
}

mlbm_status fields_to_work(mlbm_ctx* c, double* ru_dev_or_null) {
    const int n = (int)c->n;
    MLBM_CUDA(launch_macroscopics(c->params.model, n, c->perm, c->f8[c->cur], c->f0[c->cur], c->ruv[c->cur],
                                  (float)c->params.gx, (float)c->params.gy, c->S.node_sample, c->S.coll, c->rho,
                                  c->ux, c->uy, ru_dev_or_null, c->stream));
    return MLBM_OK;
}

// Steady-state iteration shared by the single and batched entry points.
//
// Criterion kFieldNorm (the build's own): every `check` steps each sample's
// velocity is compared with its own snapshot of `window` steps earlier (a
// ring of window / check snapshots), delta = |u(t) - u(t - window)|_2 /
// (window |u(t)|_2) over non-equilibrium nodes; a sample is steady at the
// first t >= window with delta < tol.
//
// Criterion kMeanVelocity (Sec. 3.2): every `check` steps the superficial
// mean velocity <u>(t) = sum u_x A / box area of each sample is recorded; at
// t >= window (the paper's Delta n_t) the relative rate
//   Delta u = |<u>(t) - <u>(t - window)| / (|<u>(t - window)| dt window)
// is formed with the sample's physical time step dt, and the sample is
// steady at the first such t with Delta u < tol (the paper's threshold is
// 1e-2 with Delta n_t = 2e4).  A zero earlier mean is never steady.
//
// Both criteria also check, at every snapshot, that each sample's density is
// positive and its fields finite on every fluid node (MLBM_E_DIVERGED
// otherwise).  at[i] receives the step of sample i's steady state, or -1.
// Steps stop once every sample is steady.  In a tau = 1 batch a sample that
// is steady is held at that state while the others go on (its nodes become
// equilibrium-kind nodes whose record is their state, so each step copies
// it: ~33 B per node update instead of ~473), and it ends at its own steady
// step as a single-sample run does; the kind bytes and records are restored
// when the run ends.
enum SteadyMode { kFieldNorm = 0, kMeanVelocity = 1 };

mlbm_status run_steady(mlbm_ctx* c, int mode, double tol, int64_t window, int64_t check, int64_t max_steps,
                       const double* dt, int64_t* at, const char* name) {
    const std::string nm(name);
    if (!(tol > 0) || window < 1 || check < 1 || window % check != 0 || max_steps < 0)
        return set_error(MLBM_E_INVALID, nm + ": bad arguments (window must be a positive multiple of check)");
    const int ns = (int)c->seg_off.size() - 1;
    if (mode == kMeanVelocity && dt)
        for (int i = 0; i < ns; ++i)
            if (!(dt[i] > 0) || !std::isfinite(dt[i]))
                return set_error(MLBM_E_INVALID, nm + ": time steps must be positive and finite");
    const int64_t R = mode == kFieldNorm ? window / check : 1;
    const int64_t n = c->n;
    std::vector<int64_t> done_at(ns, -1);
    c->steps_in_last_run = 0;
    float* ring = nullptr;
    double* means = nullptr;
    if (R > 1) {
        if ((double)R * 2.0 * (double)n * 4.0 > 64e9)
            return set_error(MLBM_E_INVALID, nm + ": snapshot ring over 64 GB (use a larger check interval)");
        MLBM_CUDA(cudaMallocAsync(&ring, (size_t)R * 2 * (size_t)n * sizeof(float), c->stream));
    }
    if (mode == kMeanVelocity) {
        cudaError_t e = cudaMallocAsync(&means, 48 * (size_t)ns, c->stream);
        if (e != cudaSuccess) {
            if (ring) cudaFreeAsync(ring, c->stream);
            cudaStreamSynchronize(c->stream);
            return set_error(MLBM_E_OOM, nm + ": " + cudaGetErrorString(e));
        }
    }
    // converged samples of a tau = 1 batch are held (see above)
    uint8_t* saved_meta = nullptr;
    float4* saved_eqv = nullptr;
    bool frozen_any = false;
    if (c->params.model == MLBM_MODEL_TAU1 && ns > 1 && n > 0) {
        const size_t np = (size_t)c->n_pad;
        if (cudaMallocAsync(&saved_meta, np, c->stream) != cudaSuccess ||
            cudaMallocAsync(&saved_eqv, np * sizeof(float4), c->stream) != cudaSuccess) {
            (void)cudaGetLastError();  // no room: every sample steps to the end
            if (saved_meta) cudaFreeAsync(saved_meta, c->stream);
            saved_meta = nullptr;
            saved_eqv = nullptr;
        } else if (cudaMemcpyAsync(saved_meta, c->meta, np, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess ||
                   cudaMemcpyAsync(saved_eqv, c->eqv, np * sizeof(float4), cudaMemcpyDeviceToDevice,
                                   c->stream) != cudaSuccess) {
            (void)cudaGetLastError();  // nothing frozen yet: step every sample to the end
            cudaFreeAsync(saved_meta, c->stream);
            cudaFreeAsync(saved_eqv, c->stream);
            saved_meta = nullptr;
            saved_eqv = nullptr;
        }
    }
    auto slot_u = [&](int64_t k) { return R > 1 ? ring + (size_t)k * 2 * n : c->px; };
    auto slot_v = [&](int64_t k) { return R > 1 ? ring + ((size_t)k * 2 + 1) * n : c->py; };
    std::vector<double> h(3 * (size_t)ns), hm(6 * (size_t)ns);
    std::vector<std::vector<double>> hist(ns);  // <u> every `check` steps (mean-velocity criterion)
    // physical time step of each sample: the caller's, else the paper's
    // units (side length 1, kinematic viscosity 1): dt = nu_lb (s / L)^2 with
    // L the side of a square of the sample's box area
    std::vector<double> dts(ns, 1.0);
    for (int i = 0; i < ns; ++i) {
        const double si = c->seg_s.empty() ? c->s : c->seg_s[i];
        const double L = std::sqrt(c->seg_box_area[i]);
        dts[i] = dt ? dt[i] : (c->seg_params[i].tau - 0.5) / 3.0 * (si / L) * (si / L);
    }
    auto snapshot = [&](int64_t k) -> mlbm_status {
        MLBM_TRY(fields_to_work(c, nullptr));
        for (int i = 0; i < ns; ++i) {
            const int64_t o = c->seg_off[i], m = c->seg_off[i + 1] - o;
            MLBM_CUDA(launch_change(c->rho + o, c->ux + o, c->uy + o, slot_u(k) + o, slot_v(k) + o, c->mask + o, m,
                                    c->scratch, c->seg_out + 3 * i, c->stream));
            if (means)
                MLBM_CUDA(launch_reduce_fields(c->rho + o, c->ux + o, c->uy + o, c->area + o, c->mask + o, m,
                                               c->scratch, means + 6 * i, c->stream));
        }
        MLBM_CUDA(cudaMemcpyAsync(h.data(), c->seg_out, 24 * (size_t)ns, cudaMemcpyDeviceToHost, c->stream));
        if (means) MLBM_CUDA(cudaMemcpyAsync(hm.data(), means, 48 * (size_t)ns, cudaMemcpyDeviceToHost, c->stream));
        MLBM_TRY(sync(c));
        for (int i = 0; i < ns; ++i) {
            if (h[3 * i + 2] != 0.0 || !std::isfinite(h[3 * i]) || !std::isfinite(h[3 * i + 1]))
                return set_error(MLBM_E_DIVERGED, nm + ": non-positive density or non-finite field in sample " +
                                                      std::to_string(i) + " (" +
                                                      std::to_string((int64_t)h[3 * i + 2]) + " nodes)");
            if (means) hist[i].push_back(hm[6 * i + 2] / c->seg_box_area[i]);
        }
        return MLBM_OK;
    };
    auto body = [&]() -> mlbm_status {
        MLBM_TRY(snapshot(0));
        int64_t t = 0;
        int remaining = ns;
        while (t < max_steps && remaining > 0) {
            const int64_t w = std::min(check, max_steps - t);
            MLBM_TRY(mlbm_step(c, w));
            t += w;
            c->steps_in_last_run = t;
            if (w != check) break;  // a partial chunk at max_steps is not evaluated
            MLBM_TRY(snapshot((t / check) % R));
            if (t < window) continue;
            for (int i = 0; i < ns; ++i) {
                if (done_at[i] >= 0) continue;
                bool steady;
                if (mode == kFieldNorm) {
                    const double delta = h[3 * i + 1] > 0 ? std::sqrt(h[3 * i] / h[3 * i + 1]) / (double)window : 0.0;
                    steady = delta < tol;
                } else {
                    const size_t j = hist[i].size() - 1, lag = (size_t)(window / check);
                    const double now = hist[i][j], then = hist[i][j - lag];
                    steady = then != 0.0 && std::fabs(now - then) / (std::fabs(then) * dts[i] * (double)window) < tol;
                }
                if (steady) {
                    done_at[i] = t;
                    --remaining;
                    if (saved_meta && remaining > 0) {
                        const int64_t o = c->seg_off[i];
                        MLBM_CUDA(launch_freeze_tau1((int)(c->seg_off[i + 1] - o), c->meta + o, c->eqv + o,
                                                     c->ruv[c->cur] + o, c->stream));
                        frozen_any = true;
                    }
                }
            }
        }
        return remaining == 0 ? MLBM_OK : set_error(MLBM_E_NOT_CONVERGED, nm + ": max_steps reached");
    };
    mlbm_status st = body();
    if (frozen_any) {
        const size_t np = (size_t)c->n_pad;
        cudaMemcpyAsync(c->meta, saved_meta, np, cudaMemcpyDeviceToDevice, c->stream);
        cudaMemcpyAsync(c->eqv, saved_eqv, np * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream);
    }
    if (saved_meta) cudaFreeAsync(saved_meta, c->stream);
    if (saved_eqv) cudaFreeAsync(saved_eqv, c->stream);
    if (ring) cudaFreeAsync(ring, c->stream);
    if (means) cudaFreeAsync(means, c->stream);
    if (ring || means || saved_meta) cudaStreamSynchronize(c->stream);
    if (at)
        for (int i = 0; i < ns; ++i) at[i] = done_at[i];
    return st;
}

}  // namespace


extern "C" {

const char* mlbm_last_error(void) { return mlbm::g_last_error.c_str(); }

const char* mlbm_version(void) { return "mlbm-gb300 0.1 (sm_103a)"; }

mlbm_status mlbm_init(mlbm_ctx** out, const mlbm_stencils* st, const mlbm_params* p, const double* rho0,
                      const double* u0) {
    clear_error();
    if (!out || !st || !p) return set_error(MLBM_E_INVALID, "init: NULL argument");
    *out = nullptr;
    MLBM_TRY(check_params(p));
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        (void)cudaGetLastError();
        return set_error(MLBM_E_CUDA, std::string("init: no CUDA device (") + cudaGetErrorString(e) + ")");
    }
    auto* c = new (std::nothrow) mlbm_ctx;
    if (!c) return set_error(MLBM_E_OOM, "init: out of host memory");
    mlbm_status s = do_init(c, st, p, rho0, u0);
    if (s != MLBM_OK) {
        std::string msg = g_last_error;
        free_ctx(c);
        return set_error(s, msg);
    }
    *out = c;
    return MLBM_OK;
}

void mlbm_destroy(mlbm_ctx* ctx) { free_ctx(ctx); }

mlbm_status mlbm_set_stream(mlbm_ctx* c, void* stream) {
    if (!c) return set_error(MLBM_E_INVALID, "set_stream: NULL context");
    MLBM_CUDA(cudaStreamSynchronize(c->stream));
    c->stream = stream ? static_cast<cudaStream_t>(stream) : c->own_stream;
    return MLBM_OK;
}

mlbm_status mlbm_set_populations(mlbm_ctx* c, const double* f) {
    if (!c || !f) return set_error(MLBM_E_INVALID, "set_populations: NULL argument");
    if (c->params.model != MLBM_MODEL_BGK) return set_error(MLBM_E_INVALID, "set_populations: BGK contexts only");
    MLBM_TRY(upload(c, c->io, f, (size_t)c->n * 9 * 8));
    MLBM_CUDA(launch_set_bgk((int)c->n, c->perm, c->io, c->f8[c->cur], c->f0[c->cur], c->stream));
    c->steps = 0;
    return sync(c);
}

mlbm_status mlbm_set_fields(mlbm_ctx* c, const double* ru) {
    if (!c || !ru) return set_error(MLBM_E_INVALID, "set_fields: NULL argument");
    MLBM_TRY(upload(c, c->io, ru, (size_t)c->n * 3 * 8));
    if (c->params.model == MLBM_MODEL_BGK)
        MLBM_CUDA(launch_set_bgk_equilibrium((int)c->n, c->perm, c->io, c->f8[c->cur], c->f0[c->cur], c->stream));
    else
        MLBM_CUDA(launch_set_tau1((int)c->n, c->perm, c->io, c->ruv[c->cur], c->stream));
    c->steps = 0;
    return sync(c);
}

mlbm_status mlbm_get_populations(mlbm_ctx* c, double* f) {
    if (!c || !f) return set_error(MLBM_E_INVALID, "get_populations: NULL argument");
    if (c->params.model != MLBM_MODEL_BGK) return set_error(MLBM_E_INVALID, "get_populations: BGK contexts only");
    MLBM_CUDA(launch_get_bgk((int)c->n, c->perm, c->f8[c->cur], c->f0[c->cur], c->io, c->stream));
    MLBM_CUDA(cudaMemcpyAsync(f, c->io, (size_t)c->n * 9 * 8, cudaMemcpyDeviceToHost, c->stream));
    return sync(c);
}

mlbm_status mlbm_get_fields(mlbm_ctx* c, double* ru) {
    if (!c || !ru) return set_error(MLBM_E_INVALID, "get_fields: NULL argument");
    MLBM_TRY(fields_to_work(c, c->io));
    MLBM_CUDA(cudaMemcpyAsync(ru, c->io, (size_t)c->n * 3 * 8, cudaMemcpyDeviceToHost, c->stream));
    return sync(c);
}

mlbm_status mlbm_step(mlbm_ctx* c, int64_t n_steps) {
    if (!c) return set_error(MLBM_E_INVALID, "step: NULL context");
    if (n_steps < 0) return set_error(MLBM_E_INVALID, "step: negative step count");
    if (n_steps == 0) return MLBM_OK;
    if (c->timing) MLBM_CUDA(cudaEventRecord(c->ev0, c->stream));
    int64_t left = n_steps;
    // a launch that must withhold a tile runs directly, not from a graph
    if (c->use_graphs && n_steps >= kGraphSteps && !c->withhold_next) {
        refresh_graphs(c);
        while (left >= kGraphSteps) {
            MLBM_TRY(ensure_graph(c, c->cur));
            MLBM_CUDA(cudaGraphLaunch(c->graph[c->cur], c->stream));
            left -= kGraphSteps;
        }
    }
    for (int64_t t = 0; t < left; ++t) MLBM_TRY(launch_one_step(c, c->variant));
    c->steps += n_steps;
    if (c->timing) {
        MLBM_CUDA(cudaEventRecord(c->ev1, c->stream));
        MLBM_CUDA(cudaEventSynchronize(c->ev1));
        float ms = 0.f;
        MLBM_CUDA(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
        c->last_ms = ms / (double)n_steps;
    }
    return MLBM_OK;
}

mlbm_status mlbm_prepare_graphs(mlbm_ctx* c) {
    if (!c) return set_error(MLBM_E_INVALID, "prepare_graphs: NULL context");
    if (!c->use_graphs) return MLBM_OK;
    refresh_graphs(c);
    MLBM_TRY(ensure_graph(c, 0));
    MLBM_TRY(ensure_graph(c, 1));
    return MLBM_OK;
}

mlbm_status mlbm_set_wait_limit(mlbm_ctx* c, double seconds) {
    if (!c) return set_error(MLBM_E_INVALID, "set_wait_limit: NULL context");
    if (!(seconds >= 1e-4 && seconds <= 60.0))
        return set_error(MLBM_E_INVALID, "set_wait_limit: the limit must lie in [1e-4, 60] seconds");
    c->wait_ns = (unsigned long long)(seconds * 1e9);
    drop_graphs(c);  // captured launches carry the old limit
    return MLBM_OK;
}

mlbm_status mlbm_test_withhold_copy(mlbm_ctx* c) {
    if (!c) return set_error(MLBM_E_INVALID, "test_withhold_copy: NULL context");
    if (!((c->variant >= 4 && c->variant <= 7) || (c->variant >= 27 && c->variant <= 29)) || c->S.Wr)
        return set_error(MLBM_E_INVALID, "test_withhold_copy: the context's kernel variant has no bulk-copy ring");
    c->withhold_next = 1;
    return MLBM_OK;
}

int64_t mlbm_step_count(const mlbm_ctx* c) { return c ? c->steps : -1; }

mlbm_status mlbm_set_timing(mlbm_ctx* c, int enable) {
    if (!c) return set_error(MLBM_E_INVALID, "set_timing: NULL context");
    c->timing = enable != 0;
    c->last_ms = -1.0;
    return MLBM_OK;
}

double mlbm_last_step_ms(const mlbm_ctx* c) { return c ? c->last_ms : -1.0; }

mlbm_status mlbm_macroscopics(mlbm_ctx* c, double* rho, double* u) {
    if (!c) return set_error(MLBM_E_INVALID, "macroscopics: NULL context");
    MLBM_TRY(fields_to_work(c, c->io));
    std::vector<double> ru((size_t)c->n * 3);
    MLBM_CUDA(cudaMemcpyAsync(ru.data(), c->io, ru.size() * 8, cudaMemcpyDeviceToHost, c->stream));
    MLBM_TRY(sync(c));
    for (int64_t i = 0; i < c->n; ++i) {
        if (rho) rho[i] = ru[i * 3];
        if (u) {
            u[2 * i] = ru[i * 3 + 1];
            u[2 * i + 1] = ru[i * 3 + 2];
        }
    }
    return MLBM_OK;
}

mlbm_status mlbm_wall_stress_force(mlbm_ctx* c, const int64_t* nodes, const double* normals, const double* ds,
                                   int64_t m, double* fx, double* fy) {
    if (!c || (m > 0 && (!nodes || !normals || !ds)) || m < 0)
        return set_error(MLBM_E_INVALID, "wall_stress_force: bad arguments");
    if (c->seg_off.size() > 2) return set_error(MLBM_E_INVALID, "wall_stress_force: single-sample contexts only");
    if (c->S.Wr) return set_error(MLBM_E_INVALID, "wall_stress_force: least-squares stencils only");
    if (m > (int64_t)1 << 30) return set_error(MLBM_E_INVALID, "wall_stress_force: too many wall nodes");
    // caller's node ids -> device positions
    std::vector<int> pos((size_t)m);
    for (int64_t i = 0; i < m; ++i) {
        if (nodes[i] < 0 || nodes[i] >= c->n) return set_error(MLBM_E_INVALID, "wall_stress_force: node id out of range");
        pos[(size_t)i] = c->inv_perm[(size_t)nodes[i]];
    }
    double sx = 0.0, sy = 0.0;
    if (m > 0) {
        const size_t mm = (size_t)m;
        if (m > c->wall_cap) {  // grow (rare: the wall node list is usually fixed)
            if (c->wall_buf) {
                MLBM_CUDA(cudaStreamSynchronize(c->stream));
                cudaFree(c->wall_buf);
                c->wall_buf = nullptr;
                c->wall_cap = 0;
            }
            void* q = nullptr;
            cudaError_t e = cudaMalloc(&q, mm * 48);
            if (e != cudaSuccess) {
                (void)cudaGetLastError();
                return set_error(MLBM_E_OOM, std::string("wall_stress_force: cudaMalloc: ") + cudaGetErrorString(e));
            }
            c->wall_buf = static_cast<uint8_t*>(q);
            c->wall_cap = m;
        }
        // normals | tractions | lengths | positions (16-, 16-, 8-, 4-byte items)
        const size_t cap = (size_t)c->wall_cap;
        double* dn = reinterpret_cast<double*>(c->wall_buf);
        double* dout = reinterpret_cast<double*>(c->wall_buf + cap * 16);
        double* dds = reinterpret_cast<double*>(c->wall_buf + cap * 32);
        int* dpos = reinterpret_cast<int*>(c->wall_buf + cap * 40);
        std::vector<double> out(2 * mm, 0.0);
        cudaError_t e = cudaMemcpyAsync(dpos, pos.data(), mm * 4, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dn, normals, mm * 16, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dds, ds, mm * 8, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) {
            const int model = c->params.model == MLBM_MODEL_BGK ? 0 : 1;
            const double nu = (c->params.tau - 0.5) / 3.0;
            e = launch_wall_traction(c->S, model, c->f8[c->cur], c->f0[c->cur], c->ruv[c->cur], c->C.ax, c->C.ay,
                                     nu, c->s, dpos, dn, dds, (int)m, dout, c->stream);
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(out.data(), dout, mm * 16, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return set_error(MLBM_E_CUDA, std::string("wall_stress_force: ") + cudaGetErrorString(e));
        for (size_t i = 0; i < mm; ++i) {  // fixed order: reproducible
            if (std::isnan(out[2 * i])) return set_error(MLBM_E_INVALID, "wall_stress_force: node " +
                                                                         std::to_string(nodes[i]) +
                                                                         " is not a least-squares node");
            sx += out[2 * i];
            sy += out[2 * i + 1];
        }
    }
    if (fx) *fx = sx;
    if (fy) *fy = sy;
    return MLBM_OK;
}

mlbm_status mlbm_drag_lift(mlbm_ctx* c, double ref_length, double u_ref, double* fx, double* fy, double* cd,
                           double* cl) {
    if (!c) return set_error(MLBM_E_INVALID, "drag_lift: NULL context");
    double h[2] = {0, 0};
    if (c->n_link_nodes > 0) {
        MLBM_CUDA(launch_force(c->S, c->params.model, c->n_link_nodes, c->link_nodes, c->area_over_s2,
                               c->f8[c->cur], c->ruv[c->cur], c->C, c->scratch, c->small, c->stream));
        MLBM_CUDA(cudaMemcpyAsync(h, c->small, 16, cudaMemcpyDeviceToHost, c->stream));
        MLBM_TRY(sync(c));
    }
    if (fx) *fx = h[0];
    if (fy) *fy = h[1];
    const double L = ref_length / c->s;
    const double den = u_ref * u_ref * L;
    if (cd) *cd = den != 0 ? 2.0 * h[0] / den : 0.0;
    if (cl) *cl = den != 0 ? 2.0 * h[1] / den : 0.0;
    return MLBM_OK;
}

mlbm_status mlbm_permeability(mlbm_ctx* c, double* k, double* us, double* ui, double* tort) {
    if (!c) return set_error(MLBM_E_INVALID, "permeability: NULL context");
    MLBM_TRY(fields_to_work(c, nullptr));
    MLBM_CUDA(launch_reduce_fields(c->rho, c->ux, c->uy, c->area, c->mask, c->n, c->scratch, c->small, c->stream));
    double h[6];
    MLBM_CUDA(cudaMemcpyAsync(h, c->small, 48, cudaMemcpyDeviceToHost, c->stream));
    MLBM_TRY(sync(c));
    const double sup = h[2] / c->box_area;
    const double gmag = std::sqrt(c->params.gx * c->params.gx + c->params.gy * c->params.gy);
    const double nu = (c->params.tau - 0.5) / 3.0;
    if (us) *us = sup;
    if (ui) *ui = h[0] != 0 ? h[2] / h[0] : 0.0;
    if (k) *k = gmag > 0 ? nu * sup / gmag : 0.0;
    if (tort) *tort = h[2] != 0 ? h[4] / h[2] : 0.0;
    return MLBM_OK;
}

mlbm_status mlbm_run_to_steady(mlbm_ctx* c, double tol, int64_t window, int64_t max_steps, int64_t* taken) {
    return mlbm_run_to_steady_ex(c, tol, window, window, max_steps, taken);
}

mlbm_status mlbm_run_to_steady_ex(mlbm_ctx* c, double tol, int64_t window, int64_t check, int64_t max_steps,
                                  int64_t* taken) {
    if (!c) return set_error(MLBM_E_INVALID, "run_to_steady: NULL context");
    if (taken) *taken = 0;
    int64_t at = -1;
    mlbm_status st = run_steady(c, kFieldNorm, tol, window, check, max_steps, nullptr, &at, "run_to_steady");
    if (taken) *taken = at >= 0 ? at : c->steps_in_last_run;
    return st;
}

mlbm_status mlbm_run_to_steady_mean(mlbm_ctx* c, double threshold, int64_t dn, int64_t check, double dt,
                                    int64_t max_steps, int64_t* taken) {
    if (!c) return set_error(MLBM_E_INVALID, "run_to_steady_mean: NULL context");
    if (taken) *taken = 0;
    if (c->seg_off.size() != 2) return set_error(MLBM_E_INVALID, "run_to_steady_mean: batched context");
    int64_t at = -1;
    const double* dtp = dt > 0 ? &dt : nullptr;
    if (dt < 0 || !std::isfinite(dt)) return set_error(MLBM_E_INVALID, "run_to_steady_mean: bad time step");
    mlbm_status st = run_steady(c, kMeanVelocity, threshold, dn, check, max_steps, dtp, &at, "run_to_steady_mean");
    if (taken) *taken = at >= 0 ? at : c->steps_in_last_run;
    return st;
}

mlbm_status mlbm_save(mlbm_ctx* c, const char* path) {
    if (!c || !path) return set_error(MLBM_E_INVALID, "save: NULL argument");
    const int per = c->params.model == MLBM_MODEL_BGK ? 9 : 3;
    std::vector<double> buf((size_t)c->n * per);
    MLBM_TRY(per == 9 ? mlbm_get_populations(c, buf.data()) : mlbm_get_fields(c, buf.data()));
    FILE* f = std::fopen(path, "wb");
    if (!f) return set_error(MLBM_E_IO, std::string("save: cannot open ") + path);
    const char magic[8] = {'M', 'L', 'B', 'M', 'S', 'T', '0', '1'};
    int64_t hdr[4] = {c->n, c->K, c->params.model, c->steps};
    bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(hdr, 8, 4, f) == 4 &&
              std::fwrite(&c->params, sizeof(mlbm_params), 1, f) == 1 &&
              std::fwrite(buf.data(), 8, buf.size(), f) == buf.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? MLBM_OK : set_error(MLBM_E_IO, "save: write failed");
}

mlbm_status mlbm_load(mlbm_ctx* c, const char* path) {
    if (!c || !path) return set_error(MLBM_E_INVALID, "load: NULL argument");
    FILE* f = std::fopen(path, "rb");
    if (!f) return set_error(MLBM_E_IO, std::string("load: cannot open ") + path);
    char magic[8];
    int64_t hdr[4];
    mlbm_params p;
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "MLBMST01", 8) == 0 &&
              std::fread(hdr, 8, 4, f) == 4 && std::fread(&p, sizeof(p), 1, f) == 1;
    if (!ok || hdr[0] != c->n || hdr[1] != c->K || hdr[2] != c->params.model) {
        std::fclose(f);
        return set_error(MLBM_E_IO, "load: file does not match this context");
    }
    const int per = c->params.model == MLBM_MODEL_BGK ? 9 : 3;
    std::vector<double> buf((size_t)c->n * per);
    ok = std::fread(buf.data(), 8, buf.size(), f) == buf.size();
    std::fclose(f);
    if (!ok) return set_error(MLBM_E_IO, "load: truncated file");
    c->params = p;
    set_collide(c);
    if (per == 9) {
        MLBM_TRY(upload(c, c->io, buf.data(), buf.size() * 8));
        MLBM_CUDA(launch_set_bgk((int)c->n, c->perm, c->io, c->f8[c->cur], c->f0[c->cur], c->stream));
    } else {
        MLBM_TRY(upload(c, c->io, buf.data(), buf.size() * 8));
        MLBM_CUDA(launch_set_tau1((int)c->n, c->perm, c->io, c->ruv[c->cur], c->stream));
    }
    MLBM_TRY(sync(c));
    c->steps = hdr[3];
    return MLBM_OK;
}

mlbm_status mlbm_set_kernel_variant(mlbm_ctx* c, int variant) {
    if (!c) return set_error(MLBM_E_INVALID, "set_kernel_variant: NULL context");
    if (variant < 0 || variant > kMaxVariant || (variant >= 4 && !tma_supported(c->K / 4)))
        return set_error(MLBM_E_INVALID, "set_kernel_variant: variant not available for this K");
    if (variant == 22 && c->params.model == MLBM_MODEL_BGK && !c->S.Wr && !c->S.lidx)
        return set_error(MLBM_E_INVALID, "set_kernel_variant: no staged neighbourhoods for this context");
    c->variant = variant;
    return MLBM_OK;
}

int mlbm_kernel_variant(const mlbm_ctx* c) { return c ? c->variant : -1; }

int mlbm_autotune_times(const mlbm_ctx* c, double* ms, int n) {
    if (!c) return -1;
    for (int v = 0; v < n && v <= kMaxVariant; ++v)
        ms[v] = v < (int)c->tune_ms.size() ? c->tune_ms[v] : -1.0;
    return kMaxVariant + 1;
}

mlbm_status mlbm_autotune(mlbm_ctx* c, int steps_per_variant, double* best_ms) {
    return mlbm_autotune_ex(c, steps_per_variant, 0, best_ms);
}

mlbm_status mlbm_autotune_ex(mlbm_ctx* c, int steps_per_variant, int flush_l2, double* best_ms) {
    if (!c || steps_per_variant < 1) return set_error(MLBM_E_INVALID, "autotune: bad arguments");
    // optional L2 flush between timed steps: a zeroed 512 MiB device buffer
    // read before every step, so each timed step reads its stencil data from
    // HBM and starts with no dirty lines in L2
    void* flush = nullptr;
    const size_t flush_bytes = size_t(512) << 20;
    if (flush_l2 && cudaMalloc(&flush, flush_bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        return set_error(MLBM_E_OOM, "autotune: no room for the L2 flush buffer");
    }
    if (flush_l2 && cudaMemsetAsync(flush, 0, flush_bytes, c->stream) != cudaSuccess) {
        cudaFree(flush);
        return set_error(MLBM_E_CUDA, "autotune: flush buffer memset failed");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (flush_l2) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
    }
    // keep the state: tuning steps run on a copy and the buffers are restored
    const size_t np = (size_t)c->n_pad;
    std::vector<void*> saved;
    auto save_buf = [&](void* d, size_t bytes) -> mlbm_status {
        void* q = nullptr;
        if (cudaMalloc(&q, bytes) != cudaSuccess) {
            (void)cudaGetLastError();
            return set_error(MLBM_E_OOM, "autotune: no room for a state copy");
        }
        saved.push_back(q);
        MLBM_CUDA(cudaMemcpyAsync(q, d, bytes, cudaMemcpyDeviceToDevice, c->stream));
        return MLBM_OK;
    };
    const int cur0 = c->cur;
    const int64_t steps0 = c->steps;
    mlbm_status st = MLBM_OK;
    if (c->params.model == MLBM_MODEL_BGK) {
        st = save_buf(c->f8[cur0], 2 * np * sizeof(float4));
        if (st == MLBM_OK) st = save_buf(c->f0[cur0], np * sizeof(float));
    } else {
        st = save_buf(c->ruv[cur0], np * sizeof(float4));
    }
    int best = c->variant;
    double best_t = 1e30;
    c->tune_ms.assign(kMaxVariant + 1, -1.0);
    for (int v = 0; v <= kMaxVariant && st == MLBM_OK; ++v) {
        if (v >= 14 && v <= 24 && c->params.model != MLBM_MODEL_BGK) continue;
        if (v >= 4 && !tma_supported(c->K / 4)) continue;
        // one untimed warm-up launch, then the timed ones
        st = launch_one_step(c, v);
        if (st != MLBM_OK) {  // a variant that cannot launch here (resources) is skipped
            (void)cudaGetLastError();
            st = MLBM_OK;
            continue;
        }
        double per = 0.0;
        if (flush_l2) {
            double tot = 0.0;
            for (int i = 0; i < steps_per_variant && st == MLBM_OK; ++i) {
                l2_flush_read<<<152 * 8, 256, 0, c->stream>>>(static_cast<const float4*>(flush),
                                                               flush_bytes / sizeof(float4),
                                                               static_cast<float*>(flush));
                cudaEventRecord(e0, c->stream);
                st = launch_one_step(c, v);
                cudaEventRecord(e1, c->stream);
                if (cudaEventSynchronize(e1) != cudaSuccess) {
                    st = set_error(MLBM_E_CUDA, "autotune: event wait failed");
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                tot += ms;
            }
            if (st != MLBM_OK) break;
            per = tot / steps_per_variant;
        } else {
            if (cudaEventRecord(c->ev0, c->stream) != cudaSuccess) break;
            for (int i = 0; i < steps_per_variant && st == MLBM_OK; ++i) st = launch_one_step(c, v);
            if (st != MLBM_OK) break;
            cudaEventRecord(c->ev1, c->stream);
            if (cudaEventSynchronize(c->ev1) != cudaSuccess) {
                st = set_error(MLBM_E_CUDA, "autotune: event wait failed");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, c->ev0, c->ev1);
            per = ms / steps_per_variant;
        }
        c->tune_ms[v] = per;
        if (per < best_t) {
            best_t = per;
            best = v;
        }
    }
    // restore
    if (st == MLBM_OK) {
        c->cur = cur0;
        if (c->params.model == MLBM_MODEL_BGK) {
            cudaMemcpyAsync(c->f8[cur0], saved[0], 2 * np * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream);
            cudaMemcpyAsync(c->f0[cur0], saved[1], np * sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
        } else {
            cudaMemcpyAsync(c->ruv[cur0], saved[0], np * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream);
        }
        st = sync(c);
    }
    for (void* q : saved) cudaFree(q);
    if (flush) cudaFree(flush);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    c->steps = steps0;
    if (st != MLBM_OK) return st;
    c->variant = best;
    if (best_ms) *best_ms = best_t;
    return MLBM_OK;
}

mlbm_status mlbm_batch_init(mlbm_ctx** out, const mlbm_stencils* const* sts, const mlbm_params* params,
                            int n_samples) {
    clear_error();
    if (!out || !sts || !params || n_samples < 1 || n_samples > 65535)
        return set_error(MLBM_E_INVALID, "batch_init: bad arguments");
    *out = nullptr;
    for (int i = 0; i < n_samples; ++i) {
        if (!sts[i]) return set_error(MLBM_E_INVALID, "batch_init: NULL stencils");
        MLBM_TRY(check_params(&params[i]));
        if (sts[i]->h.K != sts[0]->h.K || sts[i]->h.bb_mode != sts[0]->h.bb_mode ||
            params[i].model != params[0].model || sts[i]->h.interp != sts[0]->h.interp)
            return set_error(MLBM_E_INVALID,
                             "batch_init: samples must share K, bounce-back rule, interpolant and model");
    }
    // concatenate the samples' host stencils; sample i keeps its own Hilbert
    // order inside positions [off_i, off_i + n_i)
    auto* cat = new (std::nothrow) mlbm_stencils;
    if (!cat) return set_error(MLBM_E_OOM, "batch_init: out of host memory");
    HostStencils& C = cat->h;
    const int K = sts[0]->h.K;
    C.K = K;
    C.s = sts[0]->h.s;
    C.bb_mode = sts[0]->h.bb_mode;
    C.interp = sts[0]->h.interp;
    std::vector<int64_t> off(n_samples + 1, 0);
    for (int i = 0; i < n_samples; ++i) off[i + 1] = off[i] + sts[i]->h.n;
    const int64_t n = off[n_samples];
    if (n > (int64_t(1) << 31) - 1) {
        delete cat;
        return set_error(MLBM_E_INVALID, "batch_init: more than 2^31 - 1 nodes in total");
    }
    C.n = n;
    C.box_area = 0;
    C.perm.resize(n); C.inv.resize(n); C.idx.resize((size_t)n * K);
    C.kind.resize(n); C.center.resize(n); C.lag_h.resize(n); C.lag_slot.resize((size_t)n * 9);
    C.link_mask.resize(n); C.q.resize((size_t)n * 9); C.eqv.resize((size_t)n * 3); C.area.resize(n);
    C.s_node.resize(n);
    std::vector<uint16_t> node_sample(n);
    for (int i = 0; i < n_samples; ++i) {
        const HostStencils& H = sts[i]->h;
        const int64_t o = off[i];
        const bool wr = C.interp != MLBM_INTERP_WLS;
        // the matrix and weight rows stay in the sample's stencils
        C.part_M.push_back(H.M.data());
        C.part_Wr.push_back(wr ? H.Wr.data() : nullptr);
        // every node's rows in parallel (each node writes only its own)
#pragma omp parallel for schedule(static, 4096)
        for (int64_t p = 0; p < H.n; ++p) {
            const size_t g = (size_t)(o + p);
            C.perm[g] = o + H.perm[p];
            C.inv[o + H.perm[p]] = o + p;
            for (int j = 0; j < K; ++j) C.idx[g * K + j] = (int32_t)(o + H.idx[(size_t)p * K + j]);
            std::copy_n(H.lag_slot.begin() + (size_t)p * 9, 9, C.lag_slot.begin() + g * 9);
            std::copy_n(H.q.begin() + (size_t)p * 9, 9, C.q.begin() + g * 9);
            std::copy_n(H.eqv.begin() + (size_t)p * 3, 3, C.eqv.begin() + g * 3);
            C.kind[g] = H.kind[p];
            C.center[g] = H.center[p];
            C.lag_h[g] = H.lag_h[p];
            C.link_mask[g] = H.link_mask[p];
            C.area[g] = H.area[p];
            C.s_node[g] = H.s;
            node_sample[g] = (uint16_t)i;
        }
        C.info.n_wls += H.info.n_wls;
        C.info.n_lagrange += H.info.n_lagrange;
        C.info.n_eq += H.info.n_eq;
        C.info.n_link_nodes += H.info.n_link_nodes;
        C.info.n_links += H.info.n_links;
    }
    C.part_off = off;
    C.info.n = n;
    C.info.K = K;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        (void)cudaGetLastError();
        delete cat;
        return set_error(MLBM_E_CUDA, "batch_init: no CUDA device");
    }
    auto* c = new (std::nothrow) mlbm_ctx;
    if (!c) {
        delete cat;
        return set_error(MLBM_E_OOM, "batch_init: out of host memory");
    }
    c->seg_off = off;
    c->seg_params.assign(params, params + n_samples);
    for (int i = 0; i < n_samples; ++i) {
        c->seg_box_area.push_back(sts[i]->h.box_area);
        c->seg_s.push_back(sts[i]->h.s);
    }
    mlbm_status st = do_init(c, cat, &params[0], nullptr, nullptr);
    delete cat;
    if (st == MLBM_OK) {
        // per-sample collision table and per-node sample index
        std::vector<dev::Collide> table(n_samples);
        for (int i = 0; i < n_samples; ++i) {
            mlbm_ctx tmp;
            tmp.params = params[i];
            set_collide(&tmp);
            table[i] = tmp.C;
        }
        uint16_t* d_ns = nullptr;
        dev::Collide* d_coll = nullptr;
        st = dalloc(c, &d_ns, (size_t)c->n_pad);
        if (st == MLBM_OK) st = dalloc(c, &d_coll, (size_t)n_samples);
        if (st == MLBM_OK) st = upload(c, d_ns, node_sample.data(), (size_t)n * 2);
        if (st == MLBM_OK) st = upload(c, d_coll, table.data(), table.size() * sizeof(dev::Collide));
        if (st == MLBM_OK) {
            c->S.node_sample = d_ns;
            c->S.coll = d_coll;
            st = sync(c);
        }
    }
    if (st != MLBM_OK) {
        std::string msg = g_last_error;
        free_ctx(c);
        return set_error(st, msg);
    }
    *out = c;
    return MLBM_OK;
}

int mlbm_batch_size(const mlbm_ctx* c) { return c ? (int)c->seg_off.size() - 1 : -1; }

mlbm_status mlbm_batch_range(const mlbm_ctx* c, int sample, int64_t* first, int64_t* count) {
    if (!c || sample < 0 || sample >= (int)c->seg_off.size() - 1) return set_error(MLBM_E_INVALID, "batch_range: bad sample");
    if (first) *first = c->seg_off[sample];
    if (count) *count = c->seg_off[sample + 1] - c->seg_off[sample];
    return MLBM_OK;
}

mlbm_status mlbm_batch_permeability(mlbm_ctx* c, double* k, double* us, double* ui, double* tort) {
    if (!c) return set_error(MLBM_E_INVALID, "batch_permeability: NULL context");
    const int ns = (int)c->seg_off.size() - 1;
    MLBM_TRY(fields_to_work(c, nullptr));
    for (int i = 0; i < ns; ++i) {
        const int64_t o = c->seg_off[i], m = c->seg_off[i + 1] - o;
        MLBM_CUDA(launch_reduce_fields(c->rho + o, c->ux + o, c->uy + o, c->area + o, c->mask + o, m, c->scratch,
                                       c->seg_out + 6 * i, c->stream));
    }
    std::vector<double> h(6 * (size_t)ns);
    MLBM_CUDA(cudaMemcpyAsync(h.data(), c->seg_out, h.size() * 8, cudaMemcpyDeviceToHost, c->stream));
    MLBM_TRY(sync(c));
    for (int i = 0; i < ns; ++i) {
        const double* v = &h[6 * (size_t)i];
        const mlbm_params& p = c->seg_params[i];
        const double sup = v[2] / c->seg_box_area[i];
        const double gmag = std::sqrt(p.gx * p.gx + p.gy * p.gy);
        const double nu = (p.tau - 0.5) / 3.0;
        if (us) us[i] = sup;
        if (ui) ui[i] = v[0] != 0 ? v[2] / v[0] : 0.0;
        if (k) k[i] = gmag > 0 ? nu * sup / gmag : 0.0;
        if (tort) tort[i] = v[2] != 0 ? v[4] / v[2] : 0.0;
    }
    return MLBM_OK;
}

mlbm_status mlbm_batch_run_to_steady(mlbm_ctx* c, double tol, int64_t window, int64_t max_steps, int64_t* taken) {
    return mlbm_batch_run_to_steady_ex(c, tol, window, window, max_steps, taken);
}

mlbm_status mlbm_batch_run_to_steady_ex(mlbm_ctx* c, double tol, int64_t window, int64_t check, int64_t max_steps,
                                        int64_t* taken) {
    if (!c) return set_error(MLBM_E_INVALID, "batch_run_to_steady: NULL context");
    return run_steady(c, kFieldNorm, tol, window, check, max_steps, nullptr, taken, "batch_run_to_steady");
}

mlbm_status mlbm_batch_run_to_steady_mean(mlbm_ctx* c, double threshold, int64_t dn, int64_t check,
                                          const double* dt, int64_t max_steps, int64_t* taken) {
    if (!c) return set_error(MLBM_E_INVALID, "batch_run_to_steady_mean: NULL context");
    return run_steady(c, kMeanVelocity, threshold, dn, check, max_steps, dt, taken, "batch_run_to_steady_mean");
}

mlbm_status mlbm_batch_drag_lift(mlbm_ctx* c, const double* ref_length, const double* u_ref, double* fx, double* fy,
                                 double* cd, double* cl) {
    if (!c) return set_error(MLBM_E_INVALID, "batch_drag_lift: NULL context");
    const int ns = (int)c->seg_off.size() - 1;
    // link nodes are listed in position order and samples own contiguous
    // position ranges, so each sample's links are a contiguous slice
    std::vector<int> lo(ns + 1, 0);
    {
        std::vector<int> hl(c->n_link_nodes);
        if (c->n_link_nodes)
            MLBM_CUDA(cudaMemcpyAsync(hl.data(), c->link_nodes, hl.size() * 4, cudaMemcpyDeviceToHost, c->stream));
        MLBM_TRY(sync(c));
        for (int i = 0; i <= ns; ++i)
            lo[i] = (int)(std::lower_bound(hl.begin(), hl.end(), (int)c->seg_off[i]) - hl.begin());
    }
    std::vector<double> h(2 * (size_t)ns, 0.0);
    for (int i = 0; i < ns; ++i) {
        const int m = lo[i + 1] - lo[i];
        if (m == 0) continue;
        MLBM_CUDA(launch_force(c->S, c->params.model, m, c->link_nodes + lo[i], c->area_over_s2, c->f8[c->cur],
                               c->ruv[c->cur], c->C, c->scratch, c->seg_out + 2 * i, c->stream));
    }
    std::vector<double> dv(2 * (size_t)ns);
    MLBM_CUDA(cudaMemcpyAsync(dv.data(), c->seg_out, dv.size() * 8, cudaMemcpyDeviceToHost, c->stream));
    MLBM_TRY(sync(c));
    for (int i = 0; i < ns; ++i) {
        const bool any = lo[i + 1] > lo[i];
        const double Fx = any ? dv[2 * i] : 0.0, Fy = any ? dv[2 * i + 1] : 0.0;
        if (fx) fx[i] = Fx;
        if (fy) fy[i] = Fy;
        const double sq = c->seg_s.empty() ? c->s : c->seg_s[i];
        const double L = ref_length ? ref_length[i] / sq : 0.0;
        const double u = u_ref ? u_ref[i] : 0.0;
        const double den = u * u * L;
        if (cd) cd[i] = den != 0 ? 2.0 * Fx / den : 0.0;
        if (cl) cl[i] = den != 0 ? 2.0 * Fy / den : 0.0;
    }
    return MLBM_OK;
}

mlbm_status mlbm_warm_start(mlbm_ctx* c, mlbm_mlp* m, const float* X, const double* scale_u,
                            const double* scale_rho, int* n_cold) {
    if (!c || !m || !X || !scale_u) return set_error(MLBM_E_INVALID, "warm_start: NULL argument");
    const int no = mlbm_mlp_outputs(m);
    if (no != 2 && no != 3) return set_error(MLBM_E_INVALID, "warm_start: the network must have 2 or 3 outputs");
    if (no == 3 && !scale_rho) return set_error(MLBM_E_INVALID, "warm_start: NULL density scale");
    const int ns = (int)c->seg_off.size() - 1;
    for (int i = 0; i < ns; ++i)
        if (!std::isfinite(scale_u[i]) || (no == 3 && !std::isfinite(scale_rho[i])))
            return set_error(MLBM_E_INVALID, "warm_start: non-finite scale");
    if (n_cold) *n_cold = 0;
    const int n = (int)c->n;
    // one temporary buffer: scales (2 ns doubles), density means (ns
    // doubles), flags (ns ints), then the prediction Y[n][no] (16-byte aligned)
    const size_t head = ((size_t)ns * 28 + 15) / 16 * 16;
    void* buf = nullptr;
    MLBM_CUDA(cudaMallocAsync(&buf, head + (size_t)n * no * sizeof(float) + 16, c->stream));
    double* dscale_u = static_cast<double*>(buf);
    double* dscale_r = dscale_u + ns;
    double* dmean = dscale_r + ns;
    int* flag = reinterpret_cast<int*>(dmean + ns);
    float* Y = reinterpret_cast<float*>(static_cast<char*>(buf) + head);
    // releases the temporary buffer (stream-ordered) and passes a status on
    auto release = [&](mlbm_status s) {
        cudaFreeAsync(buf, c->stream);
        return s;
    };
    std::vector<double> hs(2 * (size_t)ns, 0.0);
    for (int i = 0; i < ns; ++i) {
        hs[i] = scale_u[i];
        hs[ns + i] = no == 3 ? scale_rho[i] : 0.0;
    }
    cudaError_t e = cudaMemcpyAsync(dscale_u, hs.data(), 16 * (size_t)ns, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, (size_t)ns * 4, c->stream);
    if (e != cudaSuccess) return release(set_error(MLBM_E_CUDA, std::string("warm_start: ") + cudaGetErrorString(e)));
    mlbm_status st = mlbm_mlp_forward_device(m, X, n, Y, c->stream);
    if (st != MLBM_OK) return release(st);
    e = launch_warm_check(n, c->perm, c->S.node_sample, c->meta, Y, no, dscale_u, dscale_r, 0.3f, 0.1f, flag,
                          c->stream);
    std::vector<double> hmean(ns, 0.0);
    if (e == cudaSuccess && no == 3) {
        // area-weighted mean of the predicted density deviation per sample
        e = launch_warm_drho(n, c->perm, c->S.node_sample, c->meta, Y, no, dscale_r, c->rho, c->stream);
        std::vector<double> sums(6 * (size_t)ns);
        for (int i = 0; i < ns && e == cudaSuccess; ++i) {
            const int64_t o = c->seg_off[i], cnt = c->seg_off[i + 1] - o;
            e = launch_reduce_fields(c->rho + o, c->ux + o, c->uy + o, c->area + o, c->mask + o, cnt, c->scratch,
                                     c->seg_out + 6 * i, c->stream);
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sums.data(), c->seg_out, 48 * (size_t)ns, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        for (int i = 0; i < ns && e == cudaSuccess; ++i) hmean[i] = sums[6 * i] > 0 ? sums[6 * i + 1] / sums[6 * i] : 0.0;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dmean, hmean.data(), 8 * (size_t)ns, cudaMemcpyHostToDevice, c->stream);
    }
    if (e == cudaSuccess)
        e = launch_warm_fill(n, c->perm, c->S.node_sample, c->meta, c->eqv, Y, no, dscale_u, c->rho, dmean, flag, c->io,
                             c->stream);
    if (e == cudaSuccess) {
        if (c->params.model == MLBM_MODEL_BGK)
            e = launch_set_bgk_equilibrium(n, c->perm, c->io, c->f8[c->cur], c->f0[c->cur], c->stream);
        else
            e = launch_set_tau1(n, c->perm, c->io, c->ruv[c->cur], c->stream);
    }
    std::vector<int> hflag(ns, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hflag.data(), flag, (size_t)ns * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return release(set_error(MLBM_E_CUDA, std::string("warm_start: ") + cudaGetErrorString(e)));
    MLBM_TRY(release(MLBM_OK));
    MLBM_TRY(sync(c));
    if (n_cold)
        for (int i = 0; i < ns; ++i) *n_cold += hflag[i] != 0;
    c->steps = 0;
    return MLBM_OK;
}

mlbm_status mlbm_autotune_order(mlbm_stencils* const* sts, const mlbm_params* params, int n_samples,
                                int steps_per_variant, int flush_l2, int* best_order, int* best_variant,
                                double* best_ms) {
    clear_error();
    if (!sts || !params || n_samples < 1 || steps_per_variant < 1)
        return set_error(MLBM_E_INVALID, "autotune_order: bad arguments");
    int bo = -1, bv = -1;
    double bt = 1e300;
    for (int order = MLBM_ORDER_HILBERT; order <= MLBM_ORDER_INPUT; ++order) {
        for (int i = 0; i < n_samples; ++i) MLBM_TRY(mlbm_stencils_set_order(sts[i], order));
        mlbm_ctx* c = nullptr;
        mlbm_status st = n_samples == 1 ? mlbm_init(&c, sts[0], &params[0], nullptr, nullptr)
                                        : mlbm_batch_init(&c, sts, params, n_samples);
        if (st != MLBM_OK) return st;
        double ms = 0.0;
        st = mlbm_autotune_ex(c, steps_per_variant, flush_l2, &ms);
        const int v = c->variant;
        mlbm_destroy(c);
        if (st != MLBM_OK) return st;
        if (ms < bt) {
            bt = ms;
            bo = order;
            bv = v;
        }
    }
    for (int i = 0; i < n_samples; ++i) MLBM_TRY(mlbm_stencils_set_order(sts[i], bo));
    if (best_order) *best_order = bo;
    if (best_variant) *best_variant = bv;
    if (best_ms) *best_ms = bt;
    return MLBM_OK;
}

mlbm_status mlbm_set_graphs(mlbm_ctx* c, int enable) {
    if (!c) return set_error(MLBM_E_INVALID, "set_graphs: NULL context");
    c->use_graphs = enable != 0;
    if (!c->use_graphs) drop_graphs(c);
    return MLBM_OK;
}

int64_t mlbm_reduce_scratch_doubles(int64_t n) { return n < 0 ? -1 : 6 * (int64_t)reduce_blocks(n); }

mlbm_status mlbm_reduce_fields_device(const float* rho, const float* ux, const float* uy, const float* area,
                                      const uint8_t* mask, int64_t n, double* scratch, int64_t scratch_len,
                                      double* out, void* stream) {
    clear_error();
    // the node arrays may be NULL when there are no nodes
    if ((n > 0 && (!rho || !ux || !uy || !area)) || !scratch || !out || n < 0)
        return set_error(MLBM_E_INVALID, "reduce_fields_device: NULL pointer or negative n");
    if (scratch_len < mlbm_reduce_scratch_doubles(n))
        return set_error(MLBM_E_INVALID, "reduce_fields_device: scratch too small");
    MLBM_CUDA(launch_reduce_fields(rho, ux, uy, area, mask, n, scratch, out, static_cast<cudaStream_t>(stream)));
    return MLBM_OK;
}

// ------------------------------------------------------ partitioned step
// P logical partitions of one node set, each a context over a contiguous
// range of the device positions with halo slots after its own nodes.  After
// every step each partition's new states of the nodes that another
// partition references are packed (on the owner) and copied into that
// partition's own halo slots, so every step reads local memory only.  All
// partitions live on the current device and run on one stream, in order.
}  // extern "C"

struct mlbm_part {
    int P = 0;
    int model = 0;
    double box_area = 1.0;
    std::vector<mlbm_ctx*> ctx;
    std::vector<std::vector<int64_t>> caller_ids;  // [P][n_owned]: the caller's node id of each local position
    std::vector<int64_t> first, n_owned, n_halo;
    struct Block {
        int q, o;           // receiver, owner
        int64_t count;      // nodes
        int64_t halo_off;   // first halo slot of the block in q
        int* list;          // device: positions local to o
        float4* buf;        // device: packed states
    };
    std::vector<Block> blocks;
    cudaStream_t stream = nullptr;
    std::vector<void*> allocations;
    int64_t steps = 0;
};

namespace {

void free_part(mlbm_part* P) {
    if (!P) return;
    if (P->stream) cudaStreamSynchronize(P->stream);
    for (mlbm_ctx* c : P->ctx) free_ctx(c);
    for (void* q : P->allocations) cudaFree(q);
    if (P->stream) cudaStreamDestroy(P->stream);
    delete P;
}

int state_width(const mlbm_part* P) { return P->model == MLBM_MODEL_BGK ? 2 : 1; }

float4* state_of(mlbm_ctx* c) { return c->f8[c->cur] ? c->f8[c->cur] : c->ruv[c->cur]; }

// fill every partition's halo slots from the owners' current states
mlbm_status exchange(mlbm_part* P) {
    const int w = state_width(P);
    for (const mlbm_part::Block& b : P->blocks) {
        const int grid = (int)std::min<int64_t>(4 * 152, (b.count * w + 255) / 256);
        gather_states<<<std::max(grid, 1), 256, 0, P->stream>>>(state_of(P->ctx[b.o]), b.list, b.count, w, b.buf);
        MLBM_CUDA(cudaGetLastError());
        float4* dst = state_of(P->ctx[b.q]) + (size_t)(P->n_owned[b.q] + b.halo_off) * w;
        MLBM_CUDA(cudaMemcpyAsync(dst, b.buf, (size_t)b.count * w * sizeof(float4), cudaMemcpyDeviceToDevice,
                                  P->stream));
    }
    return MLBM_OK;
}

}  // namespace

extern "C" {

mlbm_status mlbm_part_init(mlbm_part** out, const mlbm_stencils* st, const mlbm_params* p, int n_parts,
                           const int64_t* bounds) {
    clear_error();
    if (!out || !st || !p) return set_error(MLBM_E_INVALID, "part_init: NULL argument");
    *out = nullptr;
    MLBM_TRY(check_params(p));
    if (st->h.n > (int64_t(1) << 31) - 1) return set_error(MLBM_E_INVALID, "part_init: too many nodes");
    PartPlan plan;
    MLBM_TRY(make_part_plan(st->h, n_parts, bounds, plan));
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        (void)cudaGetLastError();
        return set_error(MLBM_E_CUDA, "part_init: no CUDA device");
    }
    auto* P = new (std::nothrow) mlbm_part;
    if (!P) return set_error(MLBM_E_OOM, "part_init: out of host memory");
    P->P = n_parts;
    P->model = p->model;
    P->box_area = st->h.box_area;
    auto fail = [&](mlbm_status s) {
        std::string msg = g_last_error;
        free_part(P);
        return set_error(s, msg);
    };
    if (cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking) != cudaSuccess)
        return fail(set_error(MLBM_E_CUDA, "part_init: stream"));
    for (int q = 0; q < n_parts; ++q) {
        auto* sub = new (std::nothrow) mlbm_stencils;
        if (!sub) return fail(set_error(MLBM_E_OOM, "part_init: out of host memory"));
        sub->h = slice_partition(st->h, plan, q);
        auto* c = new (std::nothrow) mlbm_ctx;
        if (!c) {
            delete sub;
            return fail(set_error(MLBM_E_OOM, "part_init: out of host memory"));
        }
        P->ctx.push_back(c);
        mlbm_status s = do_init(c, sub, p, nullptr, nullptr);
        delete sub;
        if (s != MLBM_OK) return fail(s);
        c->stream = P->stream;
        c->use_graphs = false;
        const int64_t a = plan.bounds[q], e = plan.bounds[q + 1];
        P->first.push_back(a);
        P->n_owned.push_back(e - a);
        P->n_halo.push_back((int64_t)plan.halo[q].size());
        P->caller_ids.emplace_back(st->h.perm.begin() + a, st->h.perm.begin() + e);
    }
    const int w = p->model == MLBM_MODEL_BGK ? 2 : 1;
    for (int q = 0; q < n_parts; ++q)
        for (int o = 0; o < n_parts; ++o) {
            const int64_t h0 = plan.halo_off[q][o], h1 = plan.halo_off[q][o + 1];
            if (h1 == h0) continue;
            std::vector<int> list((size_t)(h1 - h0));
            for (int64_t i = h0; i < h1; ++i) list[(size_t)(i - h0)] = (int)(plan.halo[q][(size_t)i] - plan.bounds[o]);
            mlbm_part::Block b{q, o, h1 - h0, h0, nullptr, nullptr};
            void* d = nullptr;
            if (cudaMalloc(&d, list.size() * sizeof(int)) != cudaSuccess)
                return fail(set_error(MLBM_E_OOM, "part_init: cudaMalloc"));
            P->allocations.push_back(d);
            b.list = static_cast<int*>(d);
            if (cudaMalloc(&d, (size_t)b.count * w * sizeof(float4)) != cudaSuccess)
                return fail(set_error(MLBM_E_OOM, "part_init: cudaMalloc"));
            P->allocations.push_back(d);
            b.buf = static_cast<float4*>(d);
            if (cudaMemcpyAsync(b.list, list.data(), list.size() * sizeof(int), cudaMemcpyHostToDevice, P->stream) !=
                cudaSuccess)
                return fail(set_error(MLBM_E_CUDA, "part_init: upload"));
            if (cudaStreamSynchronize(P->stream) != cudaSuccess)
                return fail(set_error(MLBM_E_CUDA, "part_init: upload"));
            P->blocks.push_back(b);
        }
    mlbm_status s = exchange(P);
    if (s == MLBM_OK) s = sync(P->ctx[0]);
    if (s != MLBM_OK) return fail(s);
    *out = P;
    return MLBM_OK;
}

void mlbm_part_destroy(mlbm_part* P) { free_part(P); }

mlbm_status mlbm_part_info(const mlbm_part* P, int part, int64_t* first, int64_t* n_owned, int64_t* n_halo,
                           int64_t* halo_bytes_per_step) {
    if (!P || part < 0 || part >= P->P) return set_error(MLBM_E_INVALID, "part_info: bad argument");
    if (first) *first = P->first[part];
    if (n_owned) *n_owned = P->n_owned[part];
    if (n_halo) *n_halo = P->n_halo[part];
    if (halo_bytes_per_step) *halo_bytes_per_step = P->n_halo[part] * state_width(P) * (int64_t)sizeof(float4);
    return MLBM_OK;
}

mlbm_status mlbm_part_set_kernel_variant(mlbm_part* P, int variant) {
    if (!P) return set_error(MLBM_E_INVALID, "part_set_kernel_variant: NULL");
    for (mlbm_ctx* c : P->ctx) MLBM_TRY(mlbm_set_kernel_variant(c, variant));
    return MLBM_OK;
}

mlbm_status mlbm_part_step(mlbm_part* P, int64_t n_steps) {
    if (!P) return set_error(MLBM_E_INVALID, "part_step: NULL");
    if (n_steps < 0) return set_error(MLBM_E_INVALID, "part_step: negative step count");
    for (int64_t t = 0; t < n_steps; ++t) {
        for (mlbm_ctx* c : P->ctx) {
            MLBM_TRY(launch_one_step(c, c->variant));
            ++c->steps;
        }
        MLBM_TRY(exchange(P));
        ++P->steps;
    }
    for (mlbm_ctx* c : P->ctx) MLBM_TRY(sync(c));  // also reports a bounded wait that ran out
    return MLBM_OK;
}

// fields or populations in the caller's order for all nodes; `width` values per node
static mlbm_status part_set(mlbm_part* P, const double* v, int width, bool fields) {
    std::vector<double> loc;
    for (int q = 0; q < P->P; ++q) {
        const std::vector<int64_t>& ids = P->caller_ids[q];
        loc.assign(ids.size() * width, 0.0);
        for (size_t p = 0; p < ids.size(); ++p)
            for (int k = 0; k < width; ++k) loc[p * width + k] = v[(size_t)ids[p] * width + k];
        MLBM_TRY(fields ? mlbm_set_fields(P->ctx[q], loc.data()) : mlbm_set_populations(P->ctx[q], loc.data()));
    }
    MLBM_TRY(exchange(P));
    P->steps = 0;
    return sync(P->ctx[0]);
}

static mlbm_status part_get(mlbm_part* P, double* v, int width, bool fields) {
    std::vector<double> loc;
    for (int q = 0; q < P->P; ++q) {
        const std::vector<int64_t>& ids = P->caller_ids[q];
        loc.assign(ids.size() * width, 0.0);
        MLBM_TRY(fields ? mlbm_get_fields(P->ctx[q], loc.data()) : mlbm_get_populations(P->ctx[q], loc.data()));
        for (size_t p = 0; p < ids.size(); ++p)
            for (int k = 0; k < width; ++k) v[(size_t)ids[p] * width + k] = loc[p * width + k];
    }
    return MLBM_OK;
}

mlbm_status mlbm_part_set_fields(mlbm_part* P, const double* ru) {
    if (!P || !ru) return set_error(MLBM_E_INVALID, "part_set_fields: NULL argument");
    return part_set(P, ru, 3, true);
}

mlbm_status mlbm_part_get_fields(mlbm_part* P, double* ru) {
    if (!P || !ru) return set_error(MLBM_E_INVALID, "part_get_fields: NULL argument");
    return part_get(P, ru, 3, true);
}

mlbm_status mlbm_part_set_populations(mlbm_part* P, const double* f) {
    if (!P || !f) return set_error(MLBM_E_INVALID, "part_set_populations: NULL argument");
    if (P->model != MLBM_MODEL_BGK) return set_error(MLBM_E_INVALID, "part_set_populations: BGK only");
    return part_set(P, f, 9, false);
}

mlbm_status mlbm_part_get_populations(mlbm_part* P, double* f) {
    if (!P || !f) return set_error(MLBM_E_INVALID, "part_get_populations: NULL argument");
    if (P->model != MLBM_MODEL_BGK) return set_error(MLBM_E_INVALID, "part_get_populations: BGK only");
    return part_get(P, f, 9, false);
}

mlbm_status mlbm_part_permeability(mlbm_part* P, double* k, double* us, double* ui, double* tort) {
    if (!P) return set_error(MLBM_E_INVALID, "part_permeability: NULL");
    // each partition's six FP64 sums, then added in partition order (the
    // all-reduce of a run whose partitions live on separate devices)
    double tot[6] = {0, 0, 0, 0, 0, 0};
    for (mlbm_ctx* c : P->ctx) {
        MLBM_TRY(fields_to_work(c, nullptr));
        MLBM_CUDA(launch_reduce_fields(c->rho, c->ux, c->uy, c->area, c->mask, c->n, c->scratch, c->small, c->stream));
        double h[6];
        MLBM_CUDA(cudaMemcpyAsync(h, c->small, 48, cudaMemcpyDeviceToHost, c->stream));
        MLBM_TRY(sync(c));
        for (int i = 0; i < 6; ++i) tot[i] += h[i];
    }
    const mlbm_params& pp = P->ctx[0]->params;
    const double sup = tot[2] / P->box_area;
    const double gmag = std::sqrt(pp.gx * pp.gx + pp.gy * pp.gy);
    const double nu = (pp.tau - 0.5) / 3.0;
    if (us) *us = sup;
    if (ui) *ui = tot[0] != 0 ? tot[2] / tot[0] : 0.0;
    if (k) *k = gmag > 0 ? nu * sup / gmag : 0.0;
    if (tort) *tort = tot[2] != 0 ? tot[4] / tot[2] : 0.0;
    return MLBM_OK;
}

}  // extern "C"
