// Host part of the C ABI declared in include/biolog.h: instance validation,
// the initial plan of Algorithm 1 Steps 1-3 (Sec. 2.5), the fixed-point
// tables the kernels use for exact sums, the device workspace, and the
// CUDA-graph replay of search iterations.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/biolog.h"
#include "biolog_internal.h"

using namespace biolog;

namespace biolog {
cudaStream_t mlp_stream_of(const bl_mlp *m);   // biolog_mlp_host.cpp
}

namespace {

thread_local std::string g_error;

constexpr size_t kAlign = 256;
constexpr int kGraphChunk = 32;              // iterations per captured graph
constexpr size_t kScratchBytes = 8u << 20;   // inspection scratch inside the workspace
constexpr int kSmemDistLimit = 150 * 1024;   // stage distances in shared memory below this blob size

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// A set of positive FP32 values written exactly as integers times a common
// power of two: value = m * 2^exp.
struct FixedPoint {
    int exp = 0;
    std::vector<long long> m;
};

bool to_fixed(const float *v, int n, FixedPoint &fp, int *bits)
{
    int emin = 100000, emax = -100000;
    for (int i = 0; i < n; ++i) {
        int e;
        std::frexp((double)v[i], &e);
        emin = std::min(emin, e);
        emax = std::max(emax, e);
    }
    int lg = 0;
    while ((1 << lg) < n + 1) ++lg;
    *bits = (emax - emin) + 24 + lg;
    if (*bits > 52) return false;
    fp.exp = emin - 24;
    fp.m.resize((size_t)n);
    for (int i = 0; i < n; ++i) fp.m[(size_t)i] = (long long)std::ldexp((double)v[i], -fp.exp);
    return fp.exp >= -126 && fp.exp <= 100;
}

struct HostInst {
    int F = 0, B = 0, T = 0, H = 0, S = 0, N = 0;
    std::vector<float> D;          // FP32 distances (FP64 computed, rounded)
    std::vector<double> D64;       // FP64 distances used by the initial heuristics
    std::vector<float> area, supply, demand, hu_rate, su_cap, su_fill, su_speed;
    float hu_speed = 0.f;
    FixedPoint supq, hurq, sufq, sucq, areaq;
    int dq_exp = 0;                // distances in fixed point: quantum 2^dq_exp
    std::vector<int32_t> Dq;
    std::vector<long long> demq;
    std::vector<int> hu_sorted, su_sorted;
    BlobLayout L{};
    std::vector<unsigned char> blob;
    int plan_len = 0;
    std::vector<int16_t> xinit;
};

int fail(std::string *err, int code, const std::string &msg)
{
    if (err) *err = msg;
    return code;
}

bool finite_pos(const float *v, int n)
{
    for (int i = 0; i < n; ++i)
        if (!(std::isfinite(v[i]) && v[i] > 0.f)) return false;
    return true;
}

// Validate and copy one instance; distances in FP64 from the FP32 coordinates.
int load_instance(const bl_instance &in, HostInst &h, std::string *err)
{
    if (in.n_fields < 1 || in.n_bps < 1 || in.n_tours < 1 || in.n_hu < 1 || in.n_su < 1)
        return fail(err, BL_EINVAL, "sizes must be positive");
    if (in.n_fields > BL_MAX_FIELDS || in.n_bps > BL_MAX_BPS || in.n_tours > BL_MAX_TOURS || in.n_hu > BL_MAX_HU ||
        in.n_su > BL_MAX_SU)
        return fail(err, BL_ETOO_LARGE, "instance exceeds the limits of this build");
    if (in.n_hu < in.n_tours || in.n_su < in.n_tours)
        return fail(err, BL_EINVAL, "need at least one HU and one SU per tour");
    if (!in.area_ha || !in.supply_t || !in.demand_t || !in.hu_rate_ha_h || !in.su_cap_t || !in.su_fill_ha ||
        !in.su_speed_kmh || (!in.xy && !in.dist))
        return fail(err, BL_EINVAL, "missing instance array");
    h.F = in.n_fields; h.B = in.n_bps; h.T = in.n_tours; h.H = in.n_hu; h.S = in.n_su;
    h.N = 1 + h.B + h.F;
    const int N = h.N;
    if (!finite_pos(in.area_ha, h.F) || !finite_pos(in.supply_t, h.F)) return fail(err, BL_EINVAL, "field areas and supplies must be finite and > 0");
    if (!finite_pos(in.demand_t, h.B)) return fail(err, BL_EINVAL, "BP demands must be finite and > 0");
    if (!finite_pos(in.hu_rate_ha_h, h.H) || !(std::isfinite(in.hu_speed_kmh) && in.hu_speed_kmh > 0.f))
        return fail(err, BL_EINVAL, "HU rates and speed must be finite and > 0");
    if (!finite_pos(in.su_cap_t, h.S) || !finite_pos(in.su_fill_ha, h.S) || !finite_pos(in.su_speed_kmh, h.S))
        return fail(err, BL_EINVAL, "SU capacities, fill areas and speeds must be finite and > 0");
    h.D.resize((size_t)N * N);
    h.D64.resize((size_t)N * N);
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            double d;
            if (in.dist) {
                d = (double)in.dist[(size_t)i * N + j];
            } else {
                const double dx = (double)in.xy[2 * i] - (double)in.xy[2 * j];
                const double dy = (double)in.xy[2 * i + 1] - (double)in.xy[2 * j + 1];
                d = std::sqrt(dx * dx + dy * dy);
            }
            if (!std::isfinite(d) || d < 0.0) return fail(err, BL_EINVAL, "distances must be finite and >= 0");
            h.D64[(size_t)i * N + j] = d;
            h.D[(size_t)i * N + j] = (float)d;
        }
    h.area.assign(in.area_ha, in.area_ha + h.F);
    h.supply.assign(in.supply_t, in.supply_t + h.F);
    h.demand.assign(in.demand_t, in.demand_t + h.B);
    h.hu_rate.assign(in.hu_rate_ha_h, in.hu_rate_ha_h + h.H);
    h.su_cap.assign(in.su_cap_t, in.su_cap_t + h.S);
    h.su_fill.assign(in.su_fill_ha, in.su_fill_ha + h.S);
    h.su_speed.assign(in.su_speed_kmh, in.su_speed_kmh + h.S);
    h.hu_speed = in.hu_speed_kmh;
    int bits;
    if (!to_fixed(h.supply.data(), h.F, h.supq, &bits) || !to_fixed(h.hu_rate.data(), h.H, h.hurq, &bits) ||
        !to_fixed(h.su_fill.data(), h.S, h.sufq, &bits) || !to_fixed(h.su_cap.data(), h.S, h.sucq, &bits) ||
        !to_fixed(h.area.data(), h.F, h.areaq, &bits))
        return fail(err, BL_ETOO_LARGE, "value range too wide for exact sums");
    // distances in fixed point: quantum 2^(e-30) with e the exponent of the largest distance, so
    // every rounded distance is < 2^30 and a tour's sum of edges stays far below 2^63
    {
        float dmax = 0.f;
        for (float d : h.D) dmax = std::max(dmax, d);
        int e = 0;
        std::frexp((double)std::max(dmax, 1e-30f), &e);
        h.dq_exp = e - 30;
        h.Dq.resize(h.D.size());
        for (size_t k = 0; k < h.D.size(); ++k) h.Dq[k] = (int32_t)std::nearbyint(std::ldexp((double)h.D[k], -h.dq_exp));
    }
    // Eq. 2 in fixed point: sum m_f >= ceil(d_b / 2^exp)
    long long total = 0;
    for (long long m : h.supq.m) total += m;
    h.demq.resize((size_t)h.B);
    long long dsum = 0;
    for (int b = 0; b < h.B; ++b) {
        const double t = std::ceil(std::ldexp((double)h.demand[(size_t)b], -h.supq.exp));
        if (t > 4.0e18) return fail(err, BL_ETOO_LARGE, "demand too large for the fixed-point supply scale");
        h.demq[(size_t)b] = (long long)t;
        dsum += h.demq[(size_t)b];
    }
    if (dsum > total) return fail(err, BL_EINFEASIBLE_INSTANCE, "total supply is below total demand");
    // units sorted by (rate or fill area, id)
    h.hu_sorted.resize((size_t)h.H);
    for (int i = 0; i < h.H; ++i) h.hu_sorted[(size_t)i] = i;
    std::stable_sort(h.hu_sorted.begin(), h.hu_sorted.end(),
                     [&](int a, int b) { return h.hu_rate[(size_t)a] < h.hu_rate[(size_t)b]; });
    h.su_sorted.resize((size_t)h.S);
    for (int i = 0; i < h.S; ++i) h.su_sorted[(size_t)i] = i;
    std::stable_sort(h.su_sorted.begin(), h.su_sorted.end(),
                     [&](int a, int b) { return h.su_fill[(size_t)a] < h.su_fill[(size_t)b]; });
    return BL_OK;
}

// Algorithm 1, Steps 1-3 (Sec. 2.5). Same readings as everywhere in this
// library: ties go to the lowest id, the BP chain is cut into contiguous
// pieces of floor((g+1)B/T) - floor(gB/T) BPs, field orders start at the HQ.
void initial_plan(HostInst &h)
{
    const int B = h.B, F = h.F, T = h.T, N = h.N;
    auto dist = [&](int i, int j) { return h.D64[(size_t)i * N + j]; };
    std::vector<int> chain;
    std::vector<char> taken((size_t)B, 0);
    int at = 0;
    while ((int)chain.size() < B) {
        int pick = -1;
        for (int b = 0; b < B; ++b)
            if (!taken[(size_t)b] && (pick < 0 || dist(at, 1 + b) < dist(at, 1 + pick))) pick = b;
        taken[(size_t)pick] = 1;
        chain.push_back(pick);
        at = 1 + pick;
    }
    std::vector<int> tour_cnt((size_t)T);
    for (int g = 0; g < T; ++g) tour_cnt[(size_t)g] = (int)((long)(g + 1) * B / T - (long)g * B / T);
    // Step 2: demand-driven field assignment, in exact fixed point
    std::vector<long long> acc((size_t)B, 0);
    std::vector<std::vector<int>> members((size_t)B);
    for (int f = 0; f < F; ++f) {
        bool open = false;
        for (int b = 0; b < B; ++b) open = open || acc[(size_t)b] < h.demq[(size_t)b];
        int pick = -1;
        for (int b = 0; b < B; ++b) {
            if (open && acc[(size_t)b] >= h.demq[(size_t)b]) continue;
            if (pick < 0 || dist(1 + B + f, 1 + b) < dist(1 + B + f, 1 + pick)) pick = b;
        }
        members[(size_t)pick].push_back(f);
        acc[(size_t)pick] += h.supq.m[(size_t)f];
    }
    // Step 3: nearest-neighbour order from the HQ within each BP
    std::vector<std::vector<int>> order((size_t)B);
    for (int b = 0; b < B; ++b) {
        std::vector<int> left = members[(size_t)b];   // ascending field ids
        int cur = 0;
        while (!left.empty()) {
            size_t best = 0;
            for (size_t k = 1; k < left.size(); ++k)
                if (dist(cur, 1 + B + left[k]) < dist(cur, 1 + B + left[best])) best = k;
            order[(size_t)b].push_back(left[best]);
            cur = 1 + B + left[best];
            left.erase(left.begin() + (long)best);
        }
    }
    h.plan_len = (int)align_up((size_t)(2 * B + T + F), 8);
    h.xinit.assign((size_t)h.plan_len, 0);
    for (int k = 0; k < B; ++k) h.xinit[(size_t)k] = (int16_t)chain[(size_t)k];
    for (int g = 0; g < T; ++g) h.xinit[(size_t)(B + g)] = (int16_t)tour_cnt[(size_t)g];
    int k = B + T;
    for (int b = 0; b < B; ++b)
        for (int f : order[(size_t)b]) h.xinit[(size_t)k++] = (int16_t)f;
    for (int b = 0; b < B; ++b) h.xinit[(size_t)(B + T + F + b)] = (int16_t)order[(size_t)b].size();
}

template <class T>
void put(std::vector<unsigned char> &blob, int off, const T *src, size_t n)
{
    std::memcpy(blob.data() + off, src, n * sizeof(T));
}

void build_blob(HostInst &h)
{
    const int F = h.F, B = h.B, T = h.T, H = h.H, S = h.S, N = h.N;
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t at = o; o = align_up(o + bytes, 16); return (int32_t)at; };
    BlobLayout &L = h.L;
    L.off_area = take((size_t)F * 4);
    L.off_areaq = take((size_t)F * 8);
    L.off_supply = take((size_t)F * 4);
    L.off_supq = take((size_t)F * 8);
    L.off_demq = take((size_t)B * 8);
    L.off_hurq = take((size_t)H * 8);
    L.off_sufq = take((size_t)S * 8);
    L.off_sucq = take((size_t)S * 8);
    L.off_suinv = take((size_t)S * 4);
    L.off_sufill = take((size_t)S * 4);
    L.off_rcp = take((size_t)(std::max(F, B) + 1) * 4);
    L.off_sugrp = take((size_t)S * 4);
    L.off_hudeal_m = take((size_t)T * T * 8);
    L.off_hudeal_q = take((size_t)T * T * 8);
    L.off_sudeal_m = take((size_t)T * T * 16);
    L.off_sudeal_q = take((size_t)T * T * 8);
    L.off_sudeal_c = take((size_t)T * T * 8);
    L.off_hu_id = take((size_t)H * 4);
    L.off_su_id = take((size_t)S * 4);
    L.prefix_bytes = (int32_t)o;
    L.off_D = take((size_t)N * N * 4);
    L.total_bytes = (int32_t)o;
    h.blob.assign(o, 0);
    put(h.blob, L.off_area, h.area.data(), (size_t)F);
    put(h.blob, L.off_areaq, h.areaq.m.data(), (size_t)F);
    put(h.blob, L.off_supply, h.supply.data(), (size_t)F);
    put(h.blob, L.off_supq, h.supq.m.data(), (size_t)F);
    put(h.blob, L.off_demq, h.demq.data(), (size_t)B);
    std::vector<long long> hurq((size_t)H), sufq((size_t)S), sucq((size_t)S);
    std::vector<float> inv_spd((size_t)S), fill_sorted((size_t)S);
    std::vector<float> rcp((size_t)(std::max(F, B) + 1), 0.f);
    for (size_t k = 1; k < rcp.size(); ++k) rcp[k] = (float)(1.0 / (double)k);
    std::vector<int32_t> grp((size_t)S), hu_id((size_t)H), su_id((size_t)S);
    for (int k = 0; k < H; ++k) { hurq[(size_t)k] = h.hurq.m[(size_t)h.hu_sorted[(size_t)k]]; hu_id[(size_t)k] = h.hu_sorted[(size_t)k]; }
    for (int k = 0; k < S; ++k) {
        const int s = h.su_sorted[(size_t)k];
        sufq[(size_t)k] = h.sufq.m[(size_t)s];
        sucq[(size_t)k] = h.sucq.m[(size_t)s];
        inv_spd[(size_t)k] = (float)(1.0 / (double)h.su_speed[(size_t)s]);
        fill_sorted[(size_t)k] = h.su_fill[(size_t)s];
        su_id[(size_t)k] = s;
        int g0 = k;
        while (g0 > 0 && h.su_fill[(size_t)h.su_sorted[(size_t)(g0 - 1)]] == h.su_fill[(size_t)s]) --g0;
        grp[(size_t)k] = g0;
    }
    put(h.blob, L.off_hurq, hurq.data(), (size_t)H);
    put(h.blob, L.off_sufq, sufq.data(), (size_t)S);
    put(h.blob, L.off_sucq, sucq.data(), (size_t)S);
    put(h.blob, L.off_suinv, inv_spd.data(), (size_t)S);
    put(h.blob, L.off_sufill, fill_sorted.data(), (size_t)S);
    put(h.blob, L.off_rcp, rcp.data(), rcp.size());
    put(h.blob, L.off_sugrp, grp.data(), (size_t)S);
    put(h.blob, L.off_hu_id, hu_id.data(), (size_t)H);
    put(h.blob, L.off_su_id, su_id.data(), (size_t)S);
    // round-robin dealing of sorted units over na active tours (Sec. 2.5,
    // "the average number ... assigned to each group")
    std::vector<unsigned long long> hm((size_t)T * T, 0), sm((size_t)T * T * 2, 0);
    std::vector<long long> hq((size_t)T * T, 0), sq((size_t)T * T, 0), sc((size_t)T * T, 0);
    for (int na = 1; na <= T; ++na) {
        for (int k = 0; k < H; ++k) {
            const size_t j = (size_t)(na - 1) * T + (size_t)(k % na);
            hm[j] |= 1ull << k;
            hq[j] += hurq[(size_t)k];
        }
        for (int k = 0; k < S; ++k) {
            const size_t j = (size_t)(na - 1) * T + (size_t)(k % na);
            sm[j * 2 + (size_t)(k / 64)] |= 1ull << (k % 64);
            sq[j] += sufq[(size_t)k];
            sc[j] += sucq[(size_t)k];
        }
    }
    put(h.blob, L.off_hudeal_m, hm.data(), hm.size());
    put(h.blob, L.off_hudeal_q, hq.data(), hq.size());
    put(h.blob, L.off_sudeal_m, sm.data(), sm.size());
    put(h.blob, L.off_sudeal_q, sq.data(), sq.size());
    put(h.blob, L.off_sudeal_c, sc.data(), sc.size());
    put(h.blob, L.off_D, h.Dq.data(), (size_t)N * N);
}

struct WsLayout {
    size_t meta, work, slot_key, slot_tmax, slot_base, scratch;
    std::vector<size_t> blob, xold, xbest, state, log_istar, log_cistar, log_use, log_cstar, log_ind;
    size_t total;
};

}  // namespace

struct bl_handle {
    int n_inst = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t capture_stream = nullptr;
    bl_params prm{};
    SearchParams sp{};
    std::vector<HostInst> insts;
    LaunchCfg cfg{};
    WsLayout ws{};
    unsigned char *base = nullptr;
    bool own_ws = false;
    std::vector<InstMeta> meta;
    std::vector<WorkItem> work;
    std::vector<int32_t> slot_base;
    int log_cap = 4096;
    cudaGraphExec_t graph = nullptr;
    InstState staged_state{};
    // learned proposal mode: pool features, predictions, selected list (allocated on first use)
    int32_t learned_pool = 0;
    uint32_t learned_iters = 0;   // salt of the random fallback
    uint16_t *l_feat = nullptr;
    float *l_y = nullptr, *l_thresh = nullptr;
    uint32_t *l_list = nullptr;
    int32_t *l_count = nullptr;
    // pinned staging of bl_set_states (h_states) and bl_get_states (h_states_out), allocated at first use;
    // states_in_done: recorded after bl_set_states' copy out of h_states, so that the next one waits only
    // for that copy and bl_get_states for nothing but its own transfer
    unsigned char *h_states = nullptr, *h_states_out = nullptr;
    size_t states_bytes = 0;
    cudaEvent_t states_in_done = nullptr;
    int dev = -1;                      // the device current at plan_init
    void *noalloc_scratch = nullptr;   // device address of bl_argmin_noalloc's static scratch (first call)
    std::string err;
    bool failed = false;
    template <class T>
    T *at(size_t off) const { return reinterpret_cast<T *>(base + off); }
};

namespace {

int cuda_fail(bl_handle *h, cudaError_t e, const char *what)
{
    if (h) {
        h->err = std::string(what) + ": " + cudaGetErrorString(e);
        h->failed = true;
    } else {
        g_error = std::string(what) + ": " + cudaGetErrorString(e);
    }
    return BL_ECUDA;
}

#define CK(h, call)                                                   \
    do {                                                              \
        cudaError_t _e = (call);                                      \
        if (_e != cudaSuccess) return cuda_fail((h), _e, #call);      \
    } while (0)

WsLayout layout_ws(const std::vector<HostInst> &insts, int n_work, int log_cap)
{
    WsLayout w;
    const size_t n = insts.size();
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t at = o; o = align_up(o + bytes, kAlign); return at; };
    w.meta = take(sizeof(InstMeta) * n);
    w.work = take(sizeof(WorkItem) * (size_t)n_work);
    w.slot_key = take(8 * (size_t)n_work);
    w.slot_tmax = take(4 * (size_t)n_work);
    w.slot_base = take(4 * n);
    w.scratch = take(kScratchBytes);
    for (const HostInst &h : insts) {
        w.blob.push_back(take((size_t)h.L.total_bytes));
        w.xold.push_back(take((size_t)h.plan_len * 2));
        w.xbest.push_back(take((size_t)h.plan_len * 2));
        w.state.push_back(take(sizeof(InstState)));
        w.log_istar.push_back(take(4 * (size_t)log_cap));
        w.log_cistar.push_back(take(4 * (size_t)log_cap));
        w.log_use.push_back(take((size_t)log_cap));
        w.log_cstar.push_back(take(4 * (size_t)log_cap));
        w.log_ind.push_back(take((size_t)log_cap));
    }
    w.total = o;
    return w;
}

int pick_shape(const std::vector<HostInst> &insts)
{
    int maxT = 0, maxS = 0, maxH = 0, maxTotal = 0;
    bool fits32 = true;   // unit sums of every instance fit in 31 bits
    for (const HostInst &h : insts) {
        maxT = std::max(maxT, h.T);
        maxS = std::max(maxS, h.S);
        maxH = std::max(maxH, h.H);
        maxTotal = std::max(maxTotal, h.L.total_bytes);
        long long a = 0, b = 0, cq = 0;
        for (long long v : h.hurq.m) a += v;
        for (long long v : h.sufq.m) b += v;
        for (long long v : h.sucq.m) cq += v;
        fits32 = fits32 && a < (1ll << 31) && b < (1ll << 31) && cq < (1ll << 31);
    }
    if (maxT <= 4 && maxS <= 32 && maxH <= 32 && fits32 && maxTotal <= kSmemDistLimit) return SHAPE_T4_S64_DSMEM;
    if (maxT <= 6 && maxS <= 64 && maxH <= 64) return SHAPE_T6_S64_GMEM;
    if (maxT <= 10) return SHAPE_T10_S128_GMEM;
    return SHAPE_T16_S128_GMEM;
}

// Work items: every instance's candidates cut into tiles; items ordered by
// instance size, largest first, so the grid-stride assignment spreads the
// long items over the blocks first.
void plan_work(bl_handle *h, int sms, int blocks_per_sm)
{
    const int n = h->n_inst;
    // at least one candidate per thread, or per lane group of the cooperative kernel
    const int threads = h->cfg.lanes > 1 ? kCoopThreads / h->cfg.lanes : h->cfg.threads;
    const int grid = sms * blocks_per_sm;
    long long total = (long long)n * h->prm.n_cand;
    int tile = h->prm.tile;
    if (tile <= 0) {
        // about 4 work items per block over the whole batch, at least one candidate per
        // thread; whole warps (not whole blocks), so a single instance fills every block
        long long per = (total + (long long)grid * 4 - 1) / ((long long)grid * 4);
        if (n == 1) per = (total + grid - 1) / grid;   // one balanced item per block
        per = std::max<long long>(per, threads);
        per = (per + 31) / 32 * 32;
        tile = (int)std::min<long long>(per, 1 << 30);
    }
    std::vector<int> order((size_t)n);
    for (int i = 0; i < n; ++i) order[(size_t)i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const HostInst &x = h->insts[(size_t)a], &y = h->insts[(size_t)b];
        return (long long)(x.F + x.B) * x.T > (long long)(y.F + y.B) * y.T;
    });
    h->work.clear();
    h->slot_base.assign((size_t)n, 0);
    std::vector<int> ntiles((size_t)n);
    int acc = 0;
    for (int i = 0; i < n; ++i) {
        ntiles[(size_t)i] = (int)((h->prm.n_cand + (long long)tile - 1) / tile);
        h->slot_base[(size_t)i] = acc;
        acc += ntiles[(size_t)i];
    }
    // interleave: round t of every instance (in size order), so each block's
    // stride visits a mix of instances
    int maxt = 0;
    for (int i = 0; i < n; ++i) maxt = std::max(maxt, ntiles[(size_t)i]);
    for (int t = 0; t < maxt; ++t)
        for (int i : order)
            if (t < ntiles[(size_t)i]) h->work.push_back(WorkItem{i, t});
    h->cfg.grid = std::min<int>(grid, (int)h->work.size());
    for (int i = 0; i < n; ++i) {
        h->meta[(size_t)i].tile = tile;
        h->meta[(size_t)i].n_tiles = ntiles[(size_t)i];
    }
}

// A device-side error flag: 1 = a bounded wait gave up, 2 = a split iteration's reduced key did not
// score as this iteration's candidate. Either way the handle refuses further work.
int state_error(bl_handle *h, uint32_t code, int inst)
{
    h->failed = true;
    if (code == 2) {
        h->err = "bl_search_apply: the key is not the argmin of this iteration's slices (instance " +
                 std::to_string(inst) + ")";
        return BL_ESTATE;
    }
    h->err = "a bounded device wait gave up (instance " + std::to_string(inst) + ")";
    return BL_ETIMEOUT;
}

int sync_and_check(bl_handle *h)
{
    CK(h, cudaStreamSynchronize(h->stream));
    for (int i = 0; i < h->n_inst; ++i) {
        InstState st;
        CK(h, cudaMemcpy(&st, h->at<InstState>(h->ws.state[(size_t)i]), sizeof(st), cudaMemcpyDeviceToHost));
        if (st.error) return state_error(h, st.error, i);
    }
    return BL_OK;
}

int score_base(bl_handle *h, int inst, int use_best, float *cost, float *tmax)
{
    float *d = h->at<float>(h->ws.scratch);
    CK(h, launch_score_dump(h->cfg, h->at<InstMeta>(h->ws.meta), inst, use_best, 0, INFINITY, 0, 1, 1, h->sp, d,
                            d + 1, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, h->stream));
    float out[2];
    CK(h, cudaMemcpyAsync(out, d, sizeof(out), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    *cost = out[0];
    *tmax = out[1];
    return BL_OK;
}

int check_plan(const HostInst &hi, const int16_t *bo, const int16_t *tc, const int16_t *fo, const int16_t *bc)
{
    const int B = hi.B, T = hi.T, F = hi.F;
    int s = 0;
    for (int g = 0; g < T; ++g) { if (tc[g] < 0) return -1; s += tc[g]; }
    if (s != B) return -1;
    s = 0;
    for (int b = 0; b < B; ++b) { if (bc[b] < 0) return -1; s += bc[b]; }
    if (s != F) return -1;
    std::vector<char> seen((size_t)std::max(B, F), 0);
    for (int k = 0; k < B; ++k) { if (bo[k] < 0 || bo[k] >= B || seen[(size_t)bo[k]]) return -1; seen[(size_t)bo[k]] = 1; }
    std::fill(seen.begin(), seen.end(), 0);
    for (int k = 0; k < F; ++k) { if (fo[k] < 0 || fo[k] >= F || seen[(size_t)fo[k]]) return -1; seen[(size_t)fo[k]] = 1; }
    return 0;
}

int init_common(const bl_instance *insts, int32_t n_inst, const bl_params *params, void *stream, bl_handle **out,
                bool size_only, size_t *bytes_out)
{
    if (out) *out = nullptr;
    if (!insts || n_inst < 1 || !params) { g_error = "null argument or no instance"; return BL_EINVAL; }
    if (params->n_cand < 1) { g_error = "n_cand must be >= 1"; return BL_EINVAL; }
    if (!(params->eps >= 0.f && params->eps <= 1.f) || !(params->p_swap >= 0.f && params->p_swap <= 1.f)) {
        g_error = "eps and p_swap must be in [0, 1]";
        return BL_EINVAL;
    }
    if (params->gate < 0 || params->gate > 2) { g_error = "gate must be 0, 1 or 2"; return BL_EINVAL; }
    if (params->k_moves < 0 || params->k_moves > kMaxMoves) {
        g_error = "k_moves must be in [0, " + std::to_string(kMaxMoves) + "]";
        return BL_EINVAL;
    }
    if ((int64_t)params->cand_offset + (int64_t)params->n_cand > (int64_t)INT32_MAX) {
        g_error = "cand_offset + n_cand must not exceed INT32_MAX";
        return BL_EINVAL;
    }
    if (params->k_moves > 1 && params->lanes_per_cand > 1) {
        g_error = "chained moves (k_moves > 1) are scored one thread per candidate: lanes_per_cand must be <= 1";
        return BL_EINVAL;
    }
    bl_handle *h = new bl_handle();
    h->n_inst = n_inst;
    h->prm = *params;
    h->stream = (cudaStream_t)stream;
    h->log_cap = params->log_capacity > 0 ? params->log_capacity : 4096;
    h->sp.eps = params->eps;
    h->sp.p_swap = params->p_swap;
    h->sp.seed_lo = (uint32_t)params->seed;
    h->sp.seed_hi = (uint32_t)(params->seed >> 32);
    h->sp.fix_field_bp = params->fix_field_bp;
    h->sp.fix_resources = params->fix_resources;
    h->sp.gate = params->gate;
    h->sp.k_moves = params->k_moves <= 1 ? 1 : params->k_moves;
    h->sp.cand_offset = params->cand_offset;
    h->sp.defer_update = 0;
    h->insts.resize((size_t)n_inst);
    for (int i = 0; i < n_inst; ++i) {
        std::string err;
        const int rc = load_instance(insts[i], h->insts[(size_t)i], &err);
        if (rc != BL_OK) {
            g_error = "instance " + std::to_string(i) + ": " + err;
            delete h;
            return rc;
        }
        initial_plan(h->insts[(size_t)i]);
        build_blob(h->insts[(size_t)i]);
    }
    int shape = pick_shape(h->insts);
    int maxT = 0;
    for (const HostInst &hi : h->insts) maxT = std::max(maxT, hi.T);
    h->cfg.max_plan_len = h->cfg.max_F = h->cfg.max_B = h->cfg.max_T = 0;
    for (const HostInst &hi : h->insts) {
        h->cfg.max_plan_len = std::max(h->cfg.max_plan_len, hi.plan_len);
        h->cfg.max_F = std::max(h->cfg.max_F, hi.F);
        h->cfg.max_B = std::max(h->cfg.max_B, hi.B);
        h->cfg.max_T = std::max(h->cfg.max_T, hi.T);
    }
    // shared memory of a shape for these instances; shape A, which stages the distances,
    // gives way to a shape that reads them through L2 when it does not fit
    auto smem_of = [&](int sh, int32_t &prefix) {
        prefix = 0;
        for (const HostInst &hi : h->insts)
            prefix = std::max(prefix, dist_in_smem(sh) ? hi.L.total_bytes : hi.L.prefix_bytes);
        return shared_bytes(sh, threads_of(sh), prefix, h->cfg.max_plan_len, h->cfg.max_F, h->cfg.max_B,
                            h->cfg.max_T);
    };
    const size_t smem_limit = 227 * 1024 - 2048;   // leave room for the static shared memory of the kernels
    int32_t prefix = 0;
    size_t smem = smem_of(shape, prefix);
    if (smem > smem_limit && shape == SHAPE_T4_S64_DSMEM) {
        shape = SHAPE_T6_S64_GMEM;   // shape A's limits are within shape B's
        smem = smem_of(shape, prefix);
    }
    h->cfg.shape = shape;
    h->cfg.threads = threads_of(shape);
    h->cfg.max_prefix = prefix;
    h->cfg.smem = smem;
    h->cfg.lanes = params->lanes_per_cand <= 1 ? 1 : params->lanes_per_cand;
    if (h->cfg.lanes > 1 && (!coop_supported(shape, h->cfg.lanes) || h->cfg.lanes < maxT)) {
        g_error = "lanes_per_cand " + std::to_string(h->cfg.lanes) + " is not built for this shape or is below the "
                  "largest tour count " + std::to_string(maxT);
        delete h;
        return BL_EINVAL;
    }
    for (const HostInst &hi : h->insts)
        if (hi.T > max_tours_of(shape) || hi.S > max_su_of(shape) || hi.H > ((shape == SHAPE_T16_S128_GMEM || shape == SHAPE_T10_S128_GMEM) ? 64 : max_su_of(shape))) {
            g_error = "no kernel shape fits";
            delete h;
            return BL_ETOO_LARGE;
        }
    if (h->cfg.smem > smem_limit) {
        g_error = "instance tables do not fit in shared memory";
        delete h;
        return BL_ETOO_LARGE;
    }
    // work decomposition needs the SM count and occupancy; for a size query use a fixed guess
    h->meta.assign((size_t)n_inst, InstMeta{});
    int sms = 152, bps = 1;
    if (!size_only) {
        int dev = 0;
        CK(nullptr, cudaGetDevice(&dev));
        h->dev = dev;
        CK(nullptr, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        cudaError_t e = configure_kernels(shape, h->cfg.smem);
        if (e != cudaSuccess) { delete h; return cuda_fail(nullptr, e, "configure_kernels"); }
        // as many blocks per SM as registers and shared memory allow
        if (h->cfg.lanes > 1) {
            const size_t csm = coop_shared_bytes(h->cfg);
            e = configure_coop(shape, h->cfg.lanes, csm);
            if (e != cudaSuccess) { delete h; return cuda_fail(nullptr, e, "configure_coop"); }
            bps = std::max(1, coop_blocks_per_sm(shape, h->cfg.lanes, csm));
        } else {
            bps = std::max(1, search_blocks_per_sm(shape, h->cfg.smem));
        }
        if (params->blocks_per_sm > 0) bps = params->blocks_per_sm;
    } else {
        bps = std::max(1, params->blocks_per_sm);
    }
    plan_work(h, sms, bps);
    h->ws = layout_ws(h->insts, (int)h->work.size(), h->log_cap);
    if (size_only) {
        *bytes_out = h->ws.total + kAlign;
        delete h;
        return BL_OK;
    }
    if (params->workspace) {
        if ((reinterpret_cast<uintptr_t>(params->workspace) % kAlign) != 0 || params->workspace_bytes < h->ws.total) {
            g_error = "workspace too small or not 256-byte aligned (see bl_workspace_bytes)";
            delete h;
            return BL_EINVAL;
        }
        h->base = (unsigned char *)params->workspace;
        h->own_ws = false;
    } else {
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, h->ws.total);
        if (e != cudaSuccess) { delete h; return cuda_fail(nullptr, e, "cudaMalloc"); }
        h->base = (unsigned char *)p;
        h->own_ws = true;
    }
    // device records
    for (int i = 0; i < n_inst; ++i) {
        const HostInst &hi = h->insts[(size_t)i];
        InstMeta &M = h->meta[(size_t)i];
        M.F = hi.F; M.B = hi.B; M.T = hi.T; M.H = hi.H; M.S = hi.S; M.N = hi.N;
        M.n_cand = params->n_cand;
        M.inst_idx = params->inst_idx + (uint32_t)i;
        M.plan_len = hi.plan_len;
        M.log_cap = h->log_cap;
        M.inv_hu_speed = 1.0f / hi.hu_speed;
        M.rq_scale = std::ldexp(1.0f, hi.hurq.exp);
        M.fq_scale = std::ldexp(1.0f, hi.sufq.exp);
        M.cq_scale = std::ldexp(1.0f, hi.sucq.exp);
        M.cq_scale_d = std::ldexp(1.0, hi.sucq.exp);
        M.dq_inv = std::ldexp(1.0f, -hi.dq_exp);
        M.dq_scale = std::ldexp(1.0f, hi.dq_exp);
        M.aq_scale = std::ldexp(1.0f, hi.areaq.exp);
        {
            double dsum = 0.0, ssum = 0.0, asum = 0.0;
            for (int f = 0; f < hi.F; ++f) {
                for (int b = 0; b < hi.B; ++b) dsum += hi.D64[(size_t)(1 + hi.B + f) * hi.N + 1 + b];
                ssum += hi.supply[(size_t)f];
                asum += hi.area[(size_t)f];
            }
            const double l0 = dsum / ((double)hi.F * hi.B);
            M.inv_l0 = (float)(l0 > 0 ? 1.0 / l0 : 1.0);
            M.inv_mean_supply = (float)(hi.F / ssum);
            M.inv_mean_area = (float)(hi.F / asum);
            M.mean_fields_per_bp = (float)hi.F / (float)hi.B;
        }
        M.L = hi.L;
        M.blob = h->at<unsigned char>(h->ws.blob[(size_t)i]);
        M.xold = h->at<int16_t>(h->ws.xold[(size_t)i]);
        M.xbest = h->at<int16_t>(h->ws.xbest[(size_t)i]);
        M.state = h->at<InstState>(h->ws.state[(size_t)i]);
        M.log_istar = h->at<int32_t>(h->ws.log_istar[(size_t)i]);
        M.log_cistar = h->at<float>(h->ws.log_cistar[(size_t)i]);
        M.log_usebest = h->at<int8_t>(h->ws.log_use[(size_t)i]);
        M.log_cstar = h->at<float>(h->ws.log_cstar[(size_t)i]);
        M.log_ind = h->at<int8_t>(h->ws.log_ind[(size_t)i]);
        CK(h, cudaMemcpyAsync((void *)M.blob, hi.blob.data(), hi.blob.size(), cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaMemcpyAsync(M.xold, hi.xinit.data(), hi.xinit.size() * 2, cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaMemcpyAsync(M.xbest, hi.xinit.data(), hi.xinit.size() * 2, cudaMemcpyHostToDevice, h->stream));
        InstState st{};
        st.cstar = INFINITY;
        st.tmaxstar = INFINITY;
        CK(h, cudaMemcpyAsync(M.state, &st, sizeof(st), cudaMemcpyHostToDevice, h->stream));
    }
    CK(h, cudaMemcpyAsync(h->at<InstMeta>(h->ws.meta), h->meta.data(), sizeof(InstMeta) * h->meta.size(),
                          cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->at<WorkItem>(h->ws.work), h->work.data(), sizeof(WorkItem) * h->work.size(),
                          cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->at<int32_t>(h->ws.slot_base), h->slot_base.data(), 4 * h->slot_base.size(),
                          cudaMemcpyHostToDevice, h->stream));
    // Step 4: C* and Tmax* of the initial plan (scored without the gate)
    const int32_t gate = h->sp.gate;
    h->sp.gate = 0;
    for (int i = 0; i < n_inst; ++i) {
        float c, t;
        const int rc = score_base(h, i, 1, &c, &t);
        if (rc != BL_OK) { h->sp.gate = gate; g_error = h->err; bl_plan_free(h); return rc; }
        InstState st{};
        st.cstar = c;
        st.tmaxstar = std::isfinite(c) ? t : INFINITY;
        CK(h, cudaMemcpyAsync(h->meta[(size_t)i].state, &st, sizeof(st), cudaMemcpyHostToDevice, h->stream));
    }
    h->sp.gate = gate;
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
    *out = h;
    return BL_OK;
}

int build_graph(bl_handle *h)
{
    cudaGraph_t g = nullptr;
    CK(h, cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < kGraphChunk; ++k) {
        cudaError_t e = launch_search_iteration(h->cfg, h->at<InstMeta>(h->ws.meta), h->at<WorkItem>(h->ws.work),
                                                (int32_t)h->work.size(), h->sp, h->at<unsigned long long>(h->ws.slot_key),
                                                h->at<float>(h->ws.slot_tmax), h->at<int32_t>(h->ws.slot_base),
                                                h->capture_stream);
        if (e != cudaSuccess) {
            cudaStreamEndCapture(h->capture_stream, &g);
            if (g) cudaGraphDestroy(g);
            return cuda_fail(h, e, "launch_search_iteration (capture)");
        }
    }
    CK(h, cudaStreamEndCapture(h->capture_stream, &g));
    cudaError_t e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
    return BL_OK;
}

}  // namespace

extern "C" {

const char *bl_global_error(void) { return g_error.c_str(); }

const char *bl_last_error(const bl_handle *h) { return h ? h->err.c_str() : g_error.c_str(); }

int bl_wait_selftest(void *stream, uint64_t limit_ns, uint64_t *elapsed_ns)
{
    if (limit_ns == 0 || limit_ns > 10000000000ull) {
        g_error = "bl_wait_selftest: limit_ns in (0, 10 s]";
        return BL_EINVAL;
    }
    unsigned long long *d = nullptr, hbuf[2] = {0ull, 0ull};
    const cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMalloc((void **)&d, sizeof(hbuf));
    if (e == cudaSuccess) e = launch_wait_selftest(limit_ns, d, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hbuf, d, sizeof(hbuf), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (d) cudaFree(d);
    if (e != cudaSuccess) {
        g_error = std::string("bl_wait_selftest: ") + cudaGetErrorString(e);
        return BL_ECUDA;
    }
    if (elapsed_ns) *elapsed_ns = hbuf[1];
    if (hbuf[0]) {
        g_error = "bl_wait_selftest: the bounded wait gave up, as it should";
        return BL_ETIMEOUT;
    }
    return BL_OK;
}

int bl_workspace_bytes(const bl_instance *insts, int32_t n_inst, const bl_params *params, size_t *bytes)
{
    if (!bytes) { g_error = "null bytes"; return BL_EINVAL; }
    bl_params p = *params;
    // size with the largest work decomposition the device can produce
    if (p.blocks_per_sm <= 0) p.blocks_per_sm = 16;
    return init_common(insts, n_inst, &p, nullptr, nullptr, true, bytes);
}

int bl_plan_init(const bl_instance *inst, const bl_params *params, void *cuda_stream, bl_handle **out)
{
    return init_common(inst, 1, params, cuda_stream, out, false, nullptr);
}

int bl_plan_init_batch(const bl_instance *insts, int32_t n_inst, const bl_params *params, void *cuda_stream,
                       bl_handle **out)
{
    return init_common(insts, n_inst, params, cuda_stream, out, false, nullptr);
}

int bl_search_step(bl_handle *h, int32_t n_iters)
{
    if (!h) return BL_EINVAL;
    if (h->failed) return BL_ESTATE;
    if (n_iters < 0) { h->err = "n_iters must be >= 0"; return BL_EINVAL; }
    if (n_iters >= kGraphChunk && !h->graph) {
        const int rc = build_graph(h);
        if (rc != BL_OK) return rc;
    }
    int left = n_iters;
    while (left >= kGraphChunk) {
        CK(h, cudaGraphLaunch(h->graph, h->stream));
        left -= kGraphChunk;
    }
    for (; left > 0; --left)
        CK(h, launch_search_iteration(h->cfg, h->at<InstMeta>(h->ws.meta), h->at<WorkItem>(h->ws.work),
                                      (int32_t)h->work.size(), h->sp, h->at<unsigned long long>(h->ws.slot_key),
                                      h->at<float>(h->ws.slot_tmax), h->at<int32_t>(h->ws.slot_base), h->stream));
    return BL_OK;
}

int bl_search_step_inspect(bl_handle *h, float *d_out, int32_t stride)
{
    if (!h || !d_out) return BL_EINVAL;
    if (h->failed) return BL_ESTATE;
    int32_t n_max = 0;
    for (const InstMeta &M : h->meta) n_max = std::max(n_max, M.n_cand);
    if (stride < n_max) {
        h->err = "bl_search_step_inspect: stride must be at least the candidates per iteration";
        return BL_EINVAL;
    }
    CK(h, launch_search_iteration(h->cfg, h->at<InstMeta>(h->ws.meta), h->at<WorkItem>(h->ws.work),
                                  (int32_t)h->work.size(), h->sp, h->at<unsigned long long>(h->ws.slot_key),
                                  h->at<float>(h->ws.slot_tmax), h->at<int32_t>(h->ws.slot_base), h->stream, nullptr,
                                  nullptr, 0, reinterpret_cast<float2 *>(d_out), stride));
    return BL_OK;
}

namespace {
// Layout of the packed states: n_inst byte offsets, then per instance x_old, x* and the state record.
size_t states_layout(const bl_handle *h, std::vector<int32_t> &offs)
{
    offs.assign((size_t)h->n_inst, 0);
    size_t o = align_up(4 * (size_t)h->n_inst, 16);
    for (int k = 0; k < h->n_inst; ++k) {
        offs[(size_t)k] = (int32_t)o;
        o = align_up(o + 4 * (size_t)h->insts[(size_t)k].plan_len + sizeof(InstState), 16);
    }
    return o;
}

int states_staging(bl_handle *h, size_t bytes)
{
    if (bytes > kScratchBytes) { h->err = "too many instances for one packed state transfer"; return BL_ETOO_LARGE; }
    if (!h->states_in_done) CK(h, cudaEventCreateWithFlags(&h->states_in_done, cudaEventDisableTiming));
    if (h->states_bytes < bytes) {
        if (h->h_states) {
            CK(h, cudaStreamSynchronize(h->stream));   // a copy out of the old staging may still be queued
            cudaFreeHost(h->h_states);
        }
        h->h_states = h->h_states_out = nullptr;
        h->states_bytes = 0;
        const size_t half = align_up(bytes, 256);
        CK(h, cudaMallocHost((void **)&h->h_states, 2 * half));
        h->h_states_out = h->h_states + half;
        h->states_bytes = bytes;
    }
    return BL_OK;
}
}  // namespace

int bl_get_states(bl_handle *h, bl_state *out)
{
    if (!h || !out) return BL_EINVAL;
    if (h->failed) return BL_ESTATE;
    std::vector<int32_t> offs;
    const size_t bytes = states_layout(h, offs);
    int rc = states_staging(h, bytes);
    if (rc != BL_OK) return rc;
    // its own staging: no earlier copy reads it (every bl_get_states ends synchronised), so the offsets,
    // the pack and the copy back queue behind the stream's work with one synchronisation at the end
    unsigned char *d = h->at<unsigned char>(h->ws.scratch);
    unsigned char *hs = h->h_states_out;
    std::memcpy(hs, offs.data(), 4 * offs.size());
    CK(h, cudaMemcpyAsync(d, hs, 4 * offs.size(), cudaMemcpyHostToDevice, h->stream));
    CK(h, launch_state_pack(h->at<InstMeta>(h->ws.meta), h->n_inst, (const int32_t *)d, d, 0, h->stream));
    CK(h, cudaMemcpyAsync(hs, d, bytes, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    for (int k = 0; k < h->n_inst; ++k) {
        const HostInst &hi = h->insts[(size_t)k];
        const int B = hi.B, T = hi.T, F = hi.F;
        const int16_t *p = (const int16_t *)(hs + offs[(size_t)k]);
        InstState st;
        std::memcpy(&st, p + 2 * hi.plan_len, sizeof(st));
        if (st.error) return state_error(h, st.error, k);
        bl_state &o = out[k];
        struct Part { int16_t *dst; const int16_t *src; int n; } parts[8] = {
            {o.xold_bp_order, p, B}, {o.xold_tour_cnt, p + B, T}, {o.xold_field_order, p + B + T, F},
            {o.xold_bp_cnt, p + B + T + F, B}, {o.xbest_bp_order, p + hi.plan_len, B},
            {o.xbest_tour_cnt, p + hi.plan_len + B, T}, {o.xbest_field_order, p + hi.plan_len + B + T, F},
            {o.xbest_bp_cnt, p + hi.plan_len + B + T + F, B}};
        for (const Part &q : parts)
            if (q.dst) std::memcpy(q.dst, q.src, 2 * (size_t)q.n);
        o.cstar = st.cstar;
        o.tmaxstar = st.tmaxstar;
        o.iter = st.iter;
    }
    return BL_OK;
}

int bl_set_states(bl_handle *h, const bl_state *in)
{
    if (!h || !in) return BL_EINVAL;
    if (h->failed) return BL_ESTATE;
    for (int k = 0; k < h->n_inst; ++k) {
        const bl_state &s = in[k];
        if (!s.xold_bp_order || !s.xold_tour_cnt || !s.xold_field_order || !s.xold_bp_cnt || !s.xbest_bp_order ||
            !s.xbest_tour_cnt || !s.xbest_field_order || !s.xbest_bp_cnt) {
            h->err = "null plan array (instance " + std::to_string(k) + ")";
            return BL_EINVAL;
        }
        const HostInst &hi = h->insts[(size_t)k];
        if (check_plan(hi, s.xold_bp_order, s.xold_tour_cnt, s.xold_field_order, s.xold_bp_cnt) ||
            check_plan(hi, s.xbest_bp_order, s.xbest_tour_cnt, s.xbest_field_order, s.xbest_bp_cnt)) {
            h->err = "invalid plan encoding (instance " + std::to_string(k) + ")";
            return BL_EINVAL;
        }
    }
    std::vector<int32_t> offs;
    const size_t bytes = states_layout(h, offs);
    int rc = states_staging(h, bytes);
    if (rc != BL_OK) return rc;
    // the staging may still feed the previous bl_set_states' copy: wait for that copy only
    CK(h, cudaEventSynchronize(h->states_in_done));
    std::memcpy(h->h_states, offs.data(), 4 * offs.size());
    for (int k = 0; k < h->n_inst; ++k) {
        const HostInst &hi = h->insts[(size_t)k];
        const int B = hi.B, T = hi.T, F = hi.F;
        int16_t *p = (int16_t *)(h->h_states + offs[(size_t)k]);
        std::memset(p, 0, 4 * (size_t)hi.plan_len);
        const bl_state &s = in[k];
        struct Part { int16_t *dst; const int16_t *src; int n; } parts[8] = {
            {p, s.xold_bp_order, B}, {p + B, s.xold_tour_cnt, T}, {p + B + T, s.xold_field_order, F},
            {p + B + T + F, s.xold_bp_cnt, B}, {p + hi.plan_len, s.xbest_bp_order, B},
            {p + hi.plan_len + B, s.xbest_tour_cnt, T}, {p + hi.plan_len + B + T, s.xbest_field_order, F},
            {p + hi.plan_len + B + T + F, s.xbest_bp_cnt, B}};
        for (const Part &q : parts) std::memcpy(q.dst, q.src, 2 * (size_t)q.n);
        InstState st{};
        st.cstar = s.cstar;
        st.tmaxstar = s.tmaxstar;
        st.iter = s.iter;
        std::memcpy(p + 2 * hi.plan_len, &st, sizeof(st));
    }
    unsigned char *d = h->at<unsigned char>(h->ws.scratch);
    CK(h, cudaMemcpyAsync(d, h->h_states, bytes, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaEventRecord(h->states_in_done, h->stream));
    CK(h, launch_state_pack(h->at<InstMeta>(h->ws.meta), h->n_inst, (const int32_t *)d, d, 1, h->stream));
    return BL_OK;
}

int bl_search_score_slice(bl_handle *h, uint64_t *d_key)
{
    if (!h || !d_key) return BL_EINVAL;
    if (h->failed) return BL_ESTATE;
    if (h->n_inst != 1) { h->err = "split iterations search one instance per handle"; return BL_EINVAL; }
    SearchParams sp = h->sp;
    sp.defer_update = 1;
    CK(h, launch_search_iteration(h->cfg, h->at<InstMeta>(h->ws.meta), h->at<WorkItem>(h->ws.work),
                                  (int32_t)h->work.size(), sp, h->at<unsigned long long>(h->ws.slot_key),
                                  h->at<float>(h->ws.slot_tmax), h->at<int32_t>(h->ws.slot_base), h->stream));
    CK(h, cudaMemcpyAsync(d_key, &h->meta[0].state->key, sizeof(uint64_t), cudaMemcpyDeviceToDevice, h->stream));
    return BL_OK;
}

int bl_search_apply(bl_handle *h, const uint64_t *d_key)
{
    if (!h || !d_key) return BL_EINVAL;
    if (h->failed) return BL_ESTATE;
    if (h->n_inst != 1) { h->err = "split iterations search one instance per handle"; return BL_EINVAL; }
    CK(h, launch_apply_key(h->cfg, h->at<InstMeta>(h->ws.meta), h->sp,
                           reinterpret_cast<const unsigned long long *>(d_key), h->stream));
    return BL_OK;
}

int bl_get_state(bl_handle *h, int32_t inst, bl_state *out)
{
    if (!h || !out || inst < 0 || inst >= h->n_inst) return BL_EINVAL;
    if (h->failed) return BL_ESTATE;
    const HostInst &hi = h->insts[(size_t)inst];
    const InstMeta &M = h->meta[(size_t)inst];
    const int B = hi.B, T = hi.T, F = hi.F;
    // straight into the caller's buffers (pinned buffers make these true async DMA copies)
    struct Part { int16_t *dst; const int16_t *src; int n; } parts[8] = {
        {out->xold_bp_order, M.xold, B}, {out->xold_tour_cnt, M.xold + B, T},
        {out->xold_field_order, M.xold + B + T, F}, {out->xold_bp_cnt, M.xold + B + T + F, B},
        {out->xbest_bp_order, M.xbest, B}, {out->xbest_tour_cnt, M.xbest + B, T},
        {out->xbest_field_order, M.xbest + B + T, F}, {out->xbest_bp_cnt, M.xbest + B + T + F, B}};
    for (const Part &q : parts)
        if (q.dst) CK(h, cudaMemcpyAsync(q.dst, q.src, 2 * (size_t)q.n, cudaMemcpyDeviceToHost, h->stream));
    InstState st;
    CK(h, cudaMemcpyAsync(&st, M.state, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (st.error) return state_error(h, st.error, inst);
    out->cstar = st.cstar;
    out->tmaxstar = st.tmaxstar;
    out->iter = st.iter;
    return BL_OK;
}

int bl_set_state(bl_handle *h, int32_t inst, const bl_state *in)
{
    if (!h || !in || inst < 0 || inst >= h->n_inst) return BL_EINVAL;
    if (h->failed) return BL_ESTATE;
    const HostInst &hi = h->insts[(size_t)inst];
    if (!in->xold_bp_order || !in->xold_tour_cnt || !in->xold_field_order || !in->xold_bp_cnt || !in->xbest_bp_order ||
        !in->xbest_tour_cnt || !in->xbest_field_order || !in->xbest_bp_cnt) {
        h->err = "null plan array";
        return BL_EINVAL;
    }
    if (check_plan(hi, in->xold_bp_order, in->xold_tour_cnt, in->xold_field_order, in->xold_bp_cnt) ||
        check_plan(hi, in->xbest_bp_order, in->xbest_tour_cnt, in->xbest_field_order, in->xbest_bp_cnt)) {
        h->err = "invalid plan encoding";
        return BL_EINVAL;
    }
    const int B = hi.B, T = hi.T, F = hi.F;
    const InstMeta &M = h->meta[(size_t)inst];
    struct Part { int16_t *dst; const int16_t *src; int n; } parts[8] = {
        {M.xold, in->xold_bp_order, B}, {M.xold + B, in->xold_tour_cnt, T},
        {M.xold + B + T, in->xold_field_order, F}, {M.xold + B + T + F, in->xold_bp_cnt, B},
        {M.xbest, in->xbest_bp_order, B}, {M.xbest + B, in->xbest_tour_cnt, T},
        {M.xbest + B + T, in->xbest_field_order, F}, {M.xbest + B + T + F, in->xbest_bp_cnt, B}};
    for (const Part &q : parts) CK(h, cudaMemcpyAsync(q.dst, q.src, 2 * (size_t)q.n, cudaMemcpyHostToDevice, h->stream));
    h->staged_state.cstar = in->cstar;
    h->staged_state.tmaxstar = in->tmaxstar;
    h->staged_state.iter = in->iter;
    h->staged_state.done = 0;
    h->staged_state.error = 0;
    CK(h, cudaMemcpyAsync(M.state, &h->staged_state, sizeof(InstState), cudaMemcpyHostToDevice, h->stream));
    // the copies read the caller's buffers: finish them before returning
    CK(h, cudaStreamSynchronize(h->stream));
    return BL_OK;
}

int bl_get_log(bl_handle *h, int32_t inst, uint32_t first, int32_t n, int32_t *istar, float *c_istar, int8_t *use_best,
               float *cstar, int8_t *indicator)
{
    if (!h || inst < 0 || inst >= h->n_inst || n < 0) return BL_EINVAL;
    if (h->failed) return BL_ESTATE;
    int rc = sync_and_check(h);
    if (rc != BL_OK) return rc;
    InstState st;
    const InstMeta &M = h->meta[(size_t)inst];
    CK(h, cudaMemcpy(&st, M.state, sizeof(st), cudaMemcpyDeviceToHost));
    if ((uint64_t)first + (uint64_t)n > st.iter || (uint64_t)first + (uint64_t)h->log_cap < st.iter) {
        h->err = "requested iterations are not in the log";
        return BL_EINVAL;
    }
    std::vector<int32_t> a((size_t)h->log_cap);
    std::vector<float> b((size_t)h->log_cap), d((size_t)h->log_cap);
    std::vector<int8_t> c((size_t)h->log_cap), e((size_t)h->log_cap);
    CK(h, cudaMemcpy(a.data(), M.log_istar, 4 * a.size(), cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(b.data(), M.log_cistar, 4 * b.size(), cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(c.data(), M.log_usebest, c.size(), cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(d.data(), M.log_cstar, 4 * d.size(), cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(e.data(), M.log_ind, e.size(), cudaMemcpyDeviceToHost));
    for (int k = 0; k < n; ++k) {
        const size_t j = (size_t)((first + (uint32_t)k) % (uint32_t)h->log_cap);
        if (istar) istar[k] = a[j];
        if (c_istar) c_istar[k] = b[j];
        if (use_best) use_best[k] = c[j];
        if (cstar) cstar[k] = d[j];
        if (indicator) indicator[k] = e[j];
    }
    return BL_OK;
}

int bl_score_candidates(bl_handle *h, int32_t inst, int32_t use_best, uint32_t iter, float tmax_star, int32_t i0,
                        int32_t n, float *cost, float *tmax, int16_t *moves, int16_t *n_hu, int16_t *n_su,
                        int16_t *hu_tour, int16_t *su_tour)
{
    if (!h || inst < 0 || inst >= h->n_inst || n < 0 || i0 < 0) return BL_EINVAL;
    if (h->failed) return BL_ESTATE;
    const HostInst &hi = h->insts[(size_t)inst];
    const int T = hi.T, H = hi.H, S = hi.S;
    const size_t nh = hu_tour ? (size_t)H : 0, ns = su_tour ? (size_t)S : 0;
    const size_t km = (size_t)h->sp.k_moves;   // move records per candidate
    const size_t per = 4 + 4 + 8 * km + 4 * (size_t)T + 2 * (nh + ns) + 16;
    const int chunk = (int)((kScratchBytes - 1024) / per);
    unsigned char *s = h->at<unsigned char>(h->ws.scratch);
    for (int k0 = 0; k0 < n; k0 += chunk) {
        const int m = std::min(chunk, n - k0);
        float *dc = (float *)s;
        float *dt = dc + m;
        int16_t *dm = (int16_t *)(dt + m);
        int16_t *dh = dm + 4 * km * (size_t)m;
        int16_t *ds = dh + (size_t)m * T;
        int16_t *dhu = hu_tour ? ds + (size_t)m * T : nullptr;
        int16_t *dsu = su_tour ? ds + (size_t)m * T + (size_t)m * nh : nullptr;
        CK(h, launch_score_dump(h->cfg, h->at<InstMeta>(h->ws.meta), inst, use_best, iter, tmax_star, i0 + k0, m, 0,
                                h->sp, dc, dt, dm, dh, ds, nullptr, nullptr, nullptr, dhu, dsu, h->stream));
        if (cost) CK(h, cudaMemcpyAsync(cost + k0, dc, 4 * (size_t)m, cudaMemcpyDeviceToHost, h->stream));
        if (tmax) CK(h, cudaMemcpyAsync(tmax + k0, dt, 4 * (size_t)m, cudaMemcpyDeviceToHost, h->stream));
        if (moves)
            CK(h, cudaMemcpyAsync(moves + 4 * km * (size_t)k0, dm, 8 * km * (size_t)m, cudaMemcpyDeviceToHost,
                                  h->stream));
        if (n_hu) CK(h, cudaMemcpyAsync(n_hu + (size_t)k0 * T, dh, 2 * (size_t)m * T, cudaMemcpyDeviceToHost, h->stream));
        if (n_su) CK(h, cudaMemcpyAsync(n_su + (size_t)k0 * T, ds, 2 * (size_t)m * T, cudaMemcpyDeviceToHost, h->stream));
        if (hu_tour)
            CK(h, cudaMemcpyAsync(hu_tour + (size_t)k0 * H, dhu, 2 * (size_t)m * H, cudaMemcpyDeviceToHost, h->stream));
        if (su_tour)
            CK(h, cudaMemcpyAsync(su_tour + (size_t)k0 * S, dsu, 2 * (size_t)m * S, cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    }
    return BL_OK;
}

int bl_decode_candidates(bl_handle *h, int32_t inst, int32_t use_best, uint32_t iter, const int32_t *idx, int32_t n,
                         int16_t *plans)
{
    if (!h || inst < 0 || inst >= h->n_inst || n < 0 || (n > 0 && (!idx || !plans))) return BL_EINVAL;
    if (h->failed) return BL_ESTATE;
    const HostInst &hi = h->insts[(size_t)inst];
    const size_t row = (size_t)(2 * hi.B + hi.T + hi.F);
    const int chunk = (int)((kScratchBytes - 1024) / (row * 2 + 4));
    unsigned char *s = h->at<unsigned char>(h->ws.scratch);
    for (int k0 = 0; k0 < n; k0 += chunk) {
        const int m = std::min(chunk, n - k0);
        int32_t *di = (int32_t *)s;
        int16_t *dp = (int16_t *)(s + align_up(4 * (size_t)m, 16));
        CK(h, cudaMemcpyAsync(di, idx + k0, 4 * (size_t)m, cudaMemcpyHostToDevice, h->stream));
        CK(h, launch_decode(h->cfg, h->at<InstMeta>(h->ws.meta), inst, use_best, iter, di, m, h->sp, dp, h->stream));
        CK(h, cudaMemcpyAsync(plans + row * (size_t)k0, dp, 2 * row * (size_t)m, cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    }
    return BL_OK;
}

int bl_argmin_noalloc(bl_handle *h, int32_t inst, int32_t use_best, uint32_t iter, float tmax_star, int32_t i0,
                      int32_t n, uint64_t *d_key, float *d_tmax)
{
    // the size limits come first: they do not depend on the handle
    if (n < 1 || n > BL_NOALLOC_MAX_CAND || i0 < 0 || (int64_t)i0 + (int64_t)n > (int64_t)INT32_MAX) {
        const char *msg = "bl_argmin_noalloc: n must be in [1, BL_NOALLOC_MAX_CAND], i0 >= 0 and i0 + n <= INT32_MAX";
        if (h) h->err = msg; else g_error = msg;
        return BL_ETOO_LARGE;
    }
    if (!h || inst < 0 || inst >= h->n_inst || !d_key || !d_tmax) return BL_EINVAL;
    if (h->failed) return BL_ESTATE;
    if (h->sp.k_moves > 1) { h->err = "bl_argmin_noalloc scores one-move candidates only"; return BL_EINVAL; }
    int dev = -1;
    CK(h, cudaGetDevice(&dev));
    if (dev != h->dev) {
        h->err = "bl_argmin_noalloc: the current device is not the handle's device";
        return BL_EINVAL;
    }
    if (!h->noalloc_scratch) CK(h, noalloc_scratch_address(&h->noalloc_scratch));
    CK(h, launch_argmin_noalloc(h->cfg, h->at<InstMeta>(h->ws.meta), inst, use_best, iter, tmax_star, i0, n, h->sp,
                                h->noalloc_scratch, reinterpret_cast<unsigned long long *>(d_key), d_tmax, h->stream));
    return BL_OK;
}

int bl_features(bl_handle *h, int32_t inst, int32_t use_best, uint32_t iter, int32_t i0, int32_t n, uint16_t *d_feat,
                float *d_base_cost)
{
    if (!h || inst < 0 || inst >= h->n_inst || i0 < 0 || n < 1 || !d_feat) return BL_EINVAL;
    if (h->failed) return BL_ESTATE;
    if (h->sp.k_moves > 1) { h->err = "bl_features describes one-move candidates only"; return BL_EINVAL; }
    CK(h, launch_features(h->cfg, h->at<InstMeta>(h->ws.meta), inst, use_best, iter, i0, n, h->sp, d_feat, d_base_cost,
                          h->stream));
    return BL_OK;
}

int bl_search_step_learned(bl_handle *h, bl_mlp *mlp, int32_t n_iters, int32_t pool, int32_t n_keep, float rand_frac)
{
    if (!h || !mlp || n_iters < 0 || pool < 1 || n_keep < 1 || n_keep > pool || !(rand_frac >= 0.f && rand_frac <= 1.f))
        return BL_EINVAL;
    if (h->failed) return BL_ESTATE;
    if (h->sp.k_moves > 1) { h->err = "learned proposals rank one-move candidates only"; return BL_EINVAL; }
    if (h->sp.cand_offset != 0) { h->err = "learned proposals rank the pool from candidate 0"; return BL_EINVAL; }
    if (mlp_stream_of(mlp) != h->stream) {
        h->err = "learned proposals: create the MLP on the search handle's stream";
        return BL_EINVAL;
    }
    if (pool > h->meta[0].n_cand) {
        h->err = "learned proposals: pool must not exceed the handle's n_cand (the work decomposition)";
        return BL_EINVAL;
    }
    const int nb = h->n_inst;
    const size_t rows = (size_t)pool * nb;
    if (h->learned_pool < pool) {
        if (h->l_feat) { cudaFree(h->l_feat); cudaFree(h->l_y); cudaFree(h->l_list); cudaFree(h->l_count); }
        h->l_feat = nullptr; h->l_y = nullptr; h->l_list = nullptr; h->l_count = nullptr; h->learned_pool = 0;
        CK(h, cudaMalloc((void **)&h->l_feat, rows * NFEAT * 2));
        CK(h, cudaMalloc((void **)&h->l_y, rows * 4));
        CK(h, cudaMalloc((void **)&h->l_list, rows * 4));
        CK(h, cudaMalloc((void **)&h->l_count, (size_t)nb * 8));   // counts, then thresholds
        h->l_thresh = reinterpret_cast<float *>(h->l_count + nb);
        h->learned_pool = pool;
    }
    if (rows > (size_t)INT32_MAX) { h->err = "learned proposals: pool x instances exceeds 2^31 rows"; return BL_ETOO_LARGE; }
    for (int it = 0; it < n_iters; ++it) {
        // each instance's base (Eq. 5) and counter are read on the device by every kernel;
        // instance b's pool occupies rows [b * pool, (b + 1) * pool)
        CK(h, launch_features(h->cfg, h->at<InstMeta>(h->ws.meta), 0, -1, 0xffffffffu, 0, pool, h->sp, h->l_feat,
                              nullptr, h->stream, nb));
        int rc = bl_mlp_forward(mlp, h->l_feat, (int32_t)rows, h->l_y);
        if (rc != BL_OK) { h->err = "learned proposals: MLP forward failed"; return rc; }
        CK(h, launch_select(h->l_y, pool, n_keep, rand_frac, 0x9E37u + h->learned_iters++, h->l_list, h->l_count,
                            h->l_thresh, nb, h->stream));
        CK(h, launch_search_iteration(h->cfg, h->at<InstMeta>(h->ws.meta), h->at<WorkItem>(h->ws.work),
                                      (int32_t)h->work.size(), h->sp, h->at<unsigned long long>(h->ws.slot_key),
                                      h->at<float>(h->ws.slot_tmax), h->at<int32_t>(h->ws.slot_base), h->stream,
                                      h->l_list, h->l_count, pool));
    }
    return BL_OK;
}

int bl_best_plan(bl_handle *h, int32_t inst, bl_plan *out)
{
    if (!h || !out || inst < 0 || inst >= h->n_inst) return BL_EINVAL;
    if (h->failed) return BL_ESTATE;
    int rc = sync_and_check(h);
    if (rc != BL_OK) return rc;
    const HostInst &hi = h->insts[(size_t)inst];
    const InstMeta &M = h->meta[(size_t)inst];
    InstState st;
    CK(h, cudaMemcpy(&st, M.state, sizeof(st), cudaMemcpyDeviceToHost));
    std::vector<int16_t> x((size_t)hi.plan_len);
    CK(h, cudaMemcpy(x.data(), M.xbest, x.size() * 2, cudaMemcpyDeviceToHost));
    const int B = hi.B, T = hi.T, F = hi.F;
    if (out->bp_order) std::memcpy(out->bp_order, x.data(), (size_t)B * 2);
    if (out->tour_cnt) std::memcpy(out->tour_cnt, x.data() + B, (size_t)T * 2);
    if (out->field_order) std::memcpy(out->field_order, x.data() + B + T, (size_t)F * 2);
    if (out->bp_cnt) std::memcpy(out->bp_cnt, x.data() + B + T + F, (size_t)B * 2);
    out->cost_km = st.cstar;
    out->tmax_h = st.tmaxstar;
    out->iter = st.iter;
    // re-score x* once for the per-tour report (gate off)
    unsigned char *s = h->at<unsigned char>(h->ws.scratch);
    float *dc = (float *)s;
    float *dtc = dc + 4, *dtw = dtc + T, *dtk = dtw + T;
    int16_t *dnh = (int16_t *)(dtk + T), *dns = dnh + T, *dhu = dns + T, *dsu = dhu + hi.H;
    const int32_t gate = h->sp.gate;
    h->sp.gate = 0;
    cudaError_t e = launch_score_dump(h->cfg, h->at<InstMeta>(h->ws.meta), inst, 1, 0, INFINITY, 0, 1, 1, h->sp, dc,
                                      dc + 1, nullptr, dnh, dns, dtc, dtw, dtk, dhu, dsu, h->stream);
    h->sp.gate = gate;
    if (e != cudaSuccess) return cuda_fail(h, e, "launch_score_dump");
    std::vector<float> tc((size_t)T), tw((size_t)T), tk((size_t)T);
    std::vector<int16_t> nh((size_t)T), ns((size_t)T), hu((size_t)hi.H), su((size_t)hi.S);
    CK(h, cudaMemcpyAsync(tc.data(), dtc, 4 * (size_t)T, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(tw.data(), dtw, 4 * (size_t)T, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(tk.data(), dtk, 4 * (size_t)T, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(nh.data(), dnh, 2 * (size_t)T, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(ns.data(), dns, 2 * (size_t)T, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(hu.data(), dhu, 2 * (size_t)hi.H, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(su.data(), dsu, 2 * (size_t)hi.S, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (out->tour_cost_km) std::memcpy(out->tour_cost_km, tk.data(), 4 * (size_t)T);
    if (out->tour_tcompl_h) std::memcpy(out->tour_tcompl_h, tc.data(), 4 * (size_t)T);
    if (out->tour_twait_h) std::memcpy(out->tour_twait_h, tw.data(), 4 * (size_t)T);
    if (out->tour_n_hu) std::memcpy(out->tour_n_hu, nh.data(), 2 * (size_t)T);
    if (out->tour_n_su) std::memcpy(out->tour_n_su, ns.data(), 2 * (size_t)T);
    if (out->hu_tour) std::memcpy(out->hu_tour, hu.data(), 2 * (size_t)hi.H);
    if (out->su_tour) std::memcpy(out->su_tour, su.data(), 2 * (size_t)hi.S);
    return BL_OK;
}

int bl_get_config(bl_handle *h, int32_t *block_threads, int32_t *grid_blocks, int32_t *tile, int32_t *launches_per_iter,
                  int32_t *lanes_per_cand)
{
    if (!h) return BL_EINVAL;
    if (lanes_per_cand) *lanes_per_cand = h->cfg.lanes;
    if (block_threads) *block_threads = h->cfg.lanes > 1 ? kCoopThreads : h->cfg.threads;
    if (grid_blocks) *grid_blocks = h->cfg.grid;
    if (tile) *tile = h->meta.empty() ? 0 : h->meta[0].tile;
    if (launches_per_iter) *launches_per_iter = 1;
    return BL_OK;
}

int bl_plan_free(bl_handle *h)
{
    if (!h) return BL_EINVAL;
    if (h->stream || h->base) cudaStreamSynchronize(h->stream);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->h_states) cudaFreeHost(h->h_states);
    if (h->states_in_done) cudaEventDestroy(h->states_in_done);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    if (h->own_ws && h->base) cudaFree(h->base);
    if (h->l_feat) cudaFree(h->l_feat);
    if (h->l_y) cudaFree(h->l_y);
    if (h->l_list) cudaFree(h->l_list);
    if (h->l_count) cudaFree(h->l_count);
    delete h;
    return BL_OK;
}

}  // extern "C"
