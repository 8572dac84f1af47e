// Kernels of the candidate search (Plessen, arXiv 1909.10286, Algorithm 1).
//
// One launch = one iteration of Steps 6-16 for every instance of the handle:
//   * each block stages an instance's tables (distances, supplies, fleet
//     tables) into shared memory with one bulk asynchronous copy completed on
//     an mbarrier, loads the base plan chosen by the eps rule (Eq. 5) and
//     traces the base plan's tours once (route aggregates per tour);
//   * every warp draws the Step 8 moves of 32 candidates at a time from
//     Philox4x32-10 with counter (i, iter, inst, 0), checks the Eq. 2 demands
//     exactly in 64-bit fixed point, and appends the feasible ones to its own
//     queue; whenever 32 are queued, each lane scores one of them:
//       - route aggregates of the tours the move touches, traced as in Fig. 1
//         (the other tours reuse the base plan's aggregates: every per-tour
//         value is a deterministic function of that tour's content, so the
//         reuse is bit-identical to re-tracing);
//       - HU assignment and SU assignment by the local minimisation of
//         Sec. 2.5 (Eq. 6, Algorithm 2);
//       - the path-length cost of Sec. 2.2 with the exact Eq. 4 ceiling, the
//         shuttle sum in order-independent fixed point;
//       - the completion-time gate;
//   * a warp-shuffle + block argmin over keys (cost bits << 32 | i) gives one
//     slot per work item; the block that finishes an instance's last work
//     item reduces the slots, replays move i* on the base and updates x_old,
//     x*, C*, Tmax* (Steps 13-16).
// Per-tour state of a candidate lives in registers (up to 4 tours) or in
// shared memory, one column per thread (more tours).
#include <cstdint>
#include <cuda_bf16.h>
#include <type_traits>
#include <cuda_runtime.h>

#include <algorithm>
#include "biolog_internal.h"

namespace biolog {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11), counter-based: no state, any thread
// can draw the numbers of any candidate.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox10(uint32_t c[4], uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
}

__device__ __forceinline__ float unit24f(uint32_t r) { return (float)(r >> 8) * (1.0f / 16777216.0f); }

// ---------------------------------------------------------------------------
// Async-proxy helpers (bulk copy global -> shared completed on an mbarrier)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded wait: gives up after limit_ns of wall time (1 s unless told otherwise)
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns = 1000000000ull)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// Self-test of the bounded wait: one thread waits on a barrier that nothing
// will ever complete (no copy, no arrival is pending on it), with a short
// limit; out[0] = 1 if the wait gave up, out[1] = the nanoseconds it took.
__global__ void wait_selftest_kernel(uint64_t limit_ns, unsigned long long *out)
{
    __shared__ uint64_t bar;
    mbar_init(&bar, 1);
    fence_mbar_init();
    const uint64_t t0 = global_ns();
    const bool done = mbar_wait_bounded(&bar, 0u, limit_ns);
    out[0] = done ? 0ull : 1ull;
    out[1] = global_ns() - t0;
}

// ---------------------------------------------------------------------------
// Shapes
// ---------------------------------------------------------------------------
// MAXT tours; SW 64-bit words per SU set (SW = 0: one 32-bit word, with
// 32-bit fixed-point unit sums); distances in shared memory or read through
// L2; NT threads per block (a compile-time constant: per-tour state offsets
// become immediates); MINB resident blocks per SM the register budget targets.
template <int MAXT_, int SW_, bool DSM_, int NT_, int MINB_>
struct Shape {
    static constexpr int MAXT = MAXT_;
    static constexpr int SW = SW_;
    static constexpr bool DSM = DSM_;
    static constexpr int NT = NT_;
    static constexpr int MINB = MINB_;
    using Mask = typename std::conditional<SW_ == 0, uint32_t, unsigned long long>::type;
    using Sum = typename std::conditional<SW_ == 0, int32_t, long long>::type;
    static constexpr int WORDS = SW_ == 0 ? 1 : SW_;
};

#ifndef BIOLOG_SHAPEA_MINB
#define BIOLOG_SHAPEA_MINB 2
#endif
// Shape B reads the distances through L2: its tour-state columns and survivor
// records for 6 tours then take about 100 KB, and two blocks reside per SM.
using ShapeA = Shape<4, 0, true, 256, BIOLOG_SHAPEA_MINB>;   // <= 4 tours, <= 32 HUs/SUs, 32-bit sums
using ShapeB = Shape<6, 1, false, 128, 2>;                   // <= 6 tours, <= 64 HUs/SUs, distances via L2
using ShapeC = Shape<16, 2, false, 128, 2>;                   // <= 16 tours, <= 128 SUs, distances via L2
using ShapeD = Shape<10, 2, false, 128, 2>;                   // <= 10 tours, <= 128 SUs, distances via L2

constexpr int NF32 = 5;   // per-tour floats: LHU, LSU, A, DB2 (2 Dbar), 1/R
constexpr int WQ = 64;    // per-warp queue of feasible candidates (ring buffer)

template <typename M>
__device__ __forceinline__ int popc_m(M m) { if constexpr (sizeof(M) == 4) return __popc(m); else return __popcll(m); }
template <typename M>
__device__ __forceinline__ int ffs_m(M m) { if constexpr (sizeof(M) == 4) return __ffs((int)m) - 1; else return __ffsll((long long)m) - 1; }
template <typename M>
__device__ __forceinline__ int hibit_m(M m) { if constexpr (sizeof(M) == 4) return 31 - __clz((int)m); else return 63 - __clzll((long long)m); }
template <typename S>
__device__ __forceinline__ float to_f(S v) { if constexpr (sizeof(S) == 4) return __int2float_rn(v); else return __ll2float_rn(v); }

// A per-tour value of the calling thread: a shared-memory column.
template <typename T, int NT>
struct Col {
    T *p;
    __device__ __forceinline__ T get(int g) const { return p[g * NT]; }
    __device__ __forceinline__ void set(int g, T v) { p[g * NT] = v; }
};

// Instance tables and base plan as seen by one block.
struct Ctx {
    int F, B, T, H, S, N;
    const int *Dq;                          // fixed-point distances (dq_scale km units)
    const float *area, *supply;
    const long long *areaq;
    const long long *supq, *demq, *hurq, *sufq, *sucq;
    const float *suinv, *sufill, *rcp;
    const int *sugrp;
    const unsigned long long *hudeal_m, *sudeal_m;
    const long long *hudeal_q, *sudeal_q, *sudeal_c;
    const int *hu_id, *su_id;
    float inv_v, rqs, fqs, cqs, dq_inv, dq_scale, aq_scale;
    double cqs_d;
    // base plan and derived tables (shared memory)
    const int16_t *bp_order, *tour_cnt, *field_order, *bp_cnt;
    const int16_t *tour_start, *bp_start, *field_bp, *field_pos, *bp_tour, *bp_pos;
    const long long *base_supq;
    const int8_t *bad;
    // base plan, per BP: first/last field node, internal HU edges, field-to-BP distances, area
    const int16_t *bfirst, *blast;
    const long long *bint, *bsb, *barea;
    // base plan, per tour: HU route, SU route, area (fixed point) and 2 x mean of per-BP means
    const long long *tLHU, *tLSU, *tA;
    const float *tDB2;
    const int2 *psd;                       // per base field position: {supply (float bits), distance to its BP}
    const float *kf_base;                  // base plan's shuttle ratio N_SU/sum cap per tour
    const long long *sh_base;              // base plan's shuttle sum per tour (fixed point)
    int memo;                              // 1 = reuse the base's shuttle sums where valid
    int nbad;
    __device__ __forceinline__ long long dq(int i, int j) const { return (long long)Dq[i * N + j]; }
};

struct MoveRec {
    int kind, v, a, b;   // 0 field reinsert, 1 BP reinsert, 2 field swap, 3 BP swap, 4 identity
};

// Step 8 with the counter layout (i, iter, inst, 0).
__device__ __forceinline__ MoveRec draw_move(const Ctx &c, const SearchParams &p, uint32_t i, uint32_t iter,
                                             uint32_t inst_idx)
{
    uint32_t r[4] = {i, iter, inst_idx, 0u};
    philox10(r, p.seed_lo, p.seed_hi);
    const int v = (int)__umulhi(r[0], (uint32_t)(c.F + c.B));
    MoveRec m;
    if (unit24f(r[3]) < p.p_swap) {
        if (v < c.F) m = {2, v, (int)__umulhi(r[1], (uint32_t)c.F), 0};
        else m = {3, v - c.F, (int)__umulhi(r[1], (uint32_t)c.B), 0};
        return m;
    }
    if (v < c.F) {
        const int bs = c.field_bp[v];
        const int bd = p.fix_field_bp ? bs : (int)__umulhi(r[1], (uint32_t)c.B);
        const int len = c.bp_cnt[bd] - (bd == bs ? 1 : 0);
        m = {0, v, bd, (int)__umulhi(r[2], (uint32_t)(len + 1))};
    } else {
        const int b = v - c.F;
        const int gs = c.bp_tour[b];
        const int gd = (int)__umulhi(r[1], (uint32_t)c.T);
        const int len = c.tour_cnt[gd] - (gd == gs ? 1 : 0);
        m = {1, b, gd, (int)__umulhi(r[2], (uint32_t)(len + 1))};
    }
    return m;
}

// Candidate plan = base with one move applied, read through index remapping
// (nothing is materialised).
struct View {
    int kind, v, w, sg, sp, dg, dp;

    __device__ __forceinline__ void set(const Ctx &c, const MoveRec &m)
    {
        kind = m.kind; v = m.v; w = m.a; sg = sp = dg = dp = -1;
        if (m.kind == 0) { sg = c.field_bp[m.v]; sp = c.field_pos[m.v]; dg = m.a; dp = m.b; }
        else if (m.kind == 1) { sg = c.bp_tour[m.v]; sp = c.bp_pos[m.v]; dg = m.a; dp = m.b; }
    }
    __device__ __forceinline__ int tour_len(const Ctx &c, int g) const
    {
        int n = c.tour_cnt[g];
        if (kind == 1) n += (g == dg ? 1 : 0) - (g == sg ? 1 : 0);
        return n;
    }
    __device__ __forceinline__ int bp_at(const Ctx &c, int g, int m) const
    {
        if (kind == 1) {
            int j = m;
            if (g == dg) {
                if (m == dp) return v;
                j = m - (m > dp ? 1 : 0);
            }
            if (g == sg) j += (j >= sp ? 1 : 0);
            return c.bp_order[c.tour_start[g] + j];
        }
        int b = c.bp_order[c.tour_start[g] + m];
        if (kind == 3) b = (b == v) ? w : (b == w ? v : b);
        return b;
    }
    __device__ __forceinline__ int bp_len(const Ctx &c, int b) const
    {
        int n = c.bp_cnt[b];
        if (kind == 0) n += (b == dg ? 1 : 0) - (b == sg ? 1 : 0);
        return n;
    }
    __device__ __forceinline__ int field_at(const Ctx &c, int b, int k) const
    {
        if (kind == 0) {
            int j = k;
            if (b == dg) {
                if (k == dp) return v;
                j = k - (k > dp ? 1 : 0);
            }
            if (b == sg) j += (j >= sp ? 1 : 0);
            return c.field_order[c.bp_start[b] + j];
        }
        int f = c.field_order[c.bp_start[b] + k];
        if (kind == 2) f = (f == v) ? w : (f == w ? v : f);
        return f;
    }
    // tour of BP b in the candidate
    __device__ __forceinline__ int tour_of_bp(const Ctx &c, int b) const
    {
        if (kind == 1 && b == v) return dg;
        if (kind == 3) {
            if (b == v) return c.bp_tour[w];
            if (b == w) return c.bp_tour[v];
        }
        return c.bp_tour[b];
    }
    // BP of field f in the candidate
    __device__ __forceinline__ int bp_of_field(const Ctx &c, int f) const
    {
        if (kind == 0 && f == v) return dg;
        if (kind == 2) {
            if (f == v) return c.field_bp[w];
            if (f == w) return c.field_bp[v];
        }
        return c.field_bp[f];
    }
    // tours whose field sequence differs from the base plan (bit mask)
    __device__ __forceinline__ unsigned touched(const Ctx &c) const
    {
        switch (kind) {
        case 0: return (1u << c.bp_tour[sg]) | (1u << c.bp_tour[dg]);
        case 1: return (1u << sg) | (1u << dg);
        case 2: return (1u << c.bp_tour[c.field_bp[v]]) | (1u << c.bp_tour[c.field_bp[w]]);
        case 3: return (1u << c.bp_tour[v]) | (1u << c.bp_tour[w]);
        default: return 0u;
        }
    }
};

// ---------------------------------------------------------------------------
// Candidates of k chained moves (Step 8 repeated; Sec. 2.5 mentions applying
// it a second time): level l turns the plan after l moves (plan l) into plan
// l + 1, and queries descend the levels by index remapping down to the base
// plan -- nothing is materialised. Move j is drawn on plan j from Philox
// counter (i, iter, inst, 0) for j = 0 and (i, iter, inst, j + 1) after
// (word 3 = 1 is the eps rule's counter).
// ---------------------------------------------------------------------------
struct Lvl {
    int kind;   // 0 field reinsert, 1 BP reinsert, 2 field swap, 3 BP swap
    int v, w;   // moved vertex; swap partner
    int s, sp;  // reinserts: source group (BP or tour) and position in plan l
    int d, dp;  // destination group and slot in its list after the removal
};

__device__ __forceinline__ int swap_id(int q, int v, int w) { return q == v ? w : (q == w ? v : q); }

struct ChainView {
    int n;   // levels (moves)
    Lvl L[kMaxMoves];

    // length of tour g / BP b in plan m
    __device__ __forceinline__ int tour_len(const Ctx &c, int g, int m) const
    {
        int len = c.tour_cnt[g];
#pragma unroll
        for (int l = 0; l < kMaxMoves; ++l)
            if (l < m && L[l].kind == 1) len += (g == L[l].d ? 1 : 0) - (g == L[l].s ? 1 : 0);
        return len;
    }
    __device__ __forceinline__ int bp_len(const Ctx &c, int b, int m) const
    {
        int len = c.bp_cnt[b];
#pragma unroll
        for (int l = 0; l < kMaxMoves; ++l)
            if (l < m && L[l].kind == 0) len += (b == L[l].d ? 1 : 0) - (b == L[l].s ? 1 : 0);
        return len;
    }
    // BP at position j of tour g in plan m: undo the levels' insertions and removals down to the
    // base, then redo the swaps of the levels above the one that placed it
    __device__ __forceinline__ int bp_at(const Ctx &c, int g, int j, int m) const
    {
        int res = -1, up = 0;
#pragma unroll
        for (int l = kMaxMoves - 1; l >= 0; --l) {
            if (l >= m || res >= 0 || L[l].kind != 1) continue;
            if (g == L[l].d) {
                if (j == L[l].dp) { res = L[l].v; up = l + 1; continue; }
                j -= (j > L[l].dp ? 1 : 0);
            }
            if (g == L[l].s) j += (j >= L[l].sp ? 1 : 0);
        }
        if (res < 0) res = c.bp_order[c.tour_start[g] + j];
#pragma unroll
        for (int l = 0; l < kMaxMoves; ++l)
            if (l >= up && l < m && L[l].kind == 3) res = swap_id(res, L[l].v, L[l].w);
        return res;
    }
    // field at position k of BP b in plan m
    __device__ __forceinline__ int field_at(const Ctx &c, int b, int k, int m) const
    {
        int res = -1, up = 0;
#pragma unroll
        for (int l = kMaxMoves - 1; l >= 0; --l) {
            if (l >= m || res >= 0 || L[l].kind != 0) continue;
            if (b == L[l].d) {
                if (k == L[l].dp) { res = L[l].v; up = l + 1; continue; }
                k -= (k > L[l].dp ? 1 : 0);
            }
            if (b == L[l].s) k += (k >= L[l].sp ? 1 : 0);
        }
        if (res < 0) res = c.field_order[c.bp_start[b] + k];
#pragma unroll
        for (int l = 0; l < kMaxMoves; ++l)
            if (l >= up && l < m && L[l].kind == 2) res = swap_id(res, L[l].v, L[l].w);
        return res;
    }
    // tour and position of BP b in plan m: follow its slot down through the swaps to the level
    // that inserted it (or the base), then shift the position by the reinserts above
    __device__ __forceinline__ void bp_place(const Ctx &c, int b, int m, int &t, int &p) const
    {
        int q = b, stop = -1;
#pragma unroll
        for (int l = kMaxMoves - 1; l >= 0; --l) {
            if (l >= m || stop >= 0) continue;
            if (L[l].kind == 1 && q == L[l].v) { stop = l; continue; }
            if (L[l].kind == 3) q = swap_id(q, L[l].v, L[l].w);
        }
        if (stop >= 0) { t = L[stop].d; p = L[stop].dp; }
        else { t = c.bp_tour[q]; p = c.bp_pos[q]; }
#pragma unroll
        for (int l = 0; l < kMaxMoves; ++l)
            if (l > stop && l < m && L[l].kind == 1) {
                p -= (t == L[l].s && p > L[l].sp) ? 1 : 0;
                p += (t == L[l].d && p >= L[l].dp) ? 1 : 0;
            }
    }
    // BP and position of field f in plan m
    __device__ __forceinline__ void field_place(const Ctx &c, int f, int m, int &b, int &p) const
    {
        int q = f, stop = -1;
#pragma unroll
        for (int l = kMaxMoves - 1; l >= 0; --l) {
            if (l >= m || stop >= 0) continue;
            if (L[l].kind == 0 && q == L[l].v) { stop = l; continue; }
            if (L[l].kind == 2) q = swap_id(q, L[l].v, L[l].w);
        }
        if (stop >= 0) { b = L[stop].d; p = L[stop].dp; }
        else { b = c.field_bp[q]; p = c.field_pos[q]; }
#pragma unroll
        for (int l = 0; l < kMaxMoves; ++l)
            if (l > stop && l < m && L[l].kind == 0) {
                p -= (b == L[l].s && p > L[l].sp) ? 1 : 0;
                p += (b == L[l].d && p >= L[l].dp) ? 1 : 0;
            }
    }
    __device__ __forceinline__ int tour_of_bp(const Ctx &c, int b) const { int t, p; bp_place(c, b, n, t, p); return t; }
    __device__ __forceinline__ int bp_of_field(const Ctx &c, int f) const { int b, p; field_place(c, f, n, b, p); return b; }
    // tours whose content may differ from the base plan: every tour some level changed, in the
    // BP-to-tour mapping of that level's plan (a superset)
    __device__ __forceinline__ unsigned touched(const Ctx &c) const
    {
        unsigned t = 0u;
#pragma unroll
        for (int l = 0; l < kMaxMoves; ++l) {
            if (l >= n) continue;
            const Lvl &e = L[l];
            int g0, g1, p, b0, b1;
            switch (e.kind) {
            case 0: bp_place(c, e.s, l, g0, p); bp_place(c, e.d, l, g1, p); break;
            case 1: g0 = e.s; g1 = e.d; break;
            case 2:
                field_place(c, e.v, l, b0, p); field_place(c, e.w, l, b1, p);
                bp_place(c, b0, l, g0, p); bp_place(c, b1, l, g1, p);
                break;
            default: bp_place(c, e.v, l, g0, p); bp_place(c, e.w, l, g1, p);
            }
            t |= (1u << g0) | (1u << g1);
        }
        return t;
    }
};

// Step 8 applied k times: move j drawn on plan j with the same rules as draw_move.
__device__ __forceinline__ void draw_chain(const Ctx &c, const SearchParams &p, uint32_t i, uint32_t iter,
                                           uint32_t inst_idx, ChainView &cv)
{
    cv.n = 0;
#pragma unroll
    for (int j = 0; j < kMaxMoves; ++j) {
        if (j >= p.k_moves) continue;
        uint32_t r[4] = {i, iter, inst_idx, j == 0 ? 0u : (uint32_t)j + 1u};
        philox10(r, p.seed_lo, p.seed_hi);
        const int v = (int)__umulhi(r[0], (uint32_t)(c.F + c.B));
        Lvl e = {4, 0, 0, -1, -1, -1, -1};
        if (unit24f(r[3]) < p.p_swap) {
            if (v < c.F) { e.kind = 2; e.v = v; e.w = (int)__umulhi(r[1], (uint32_t)c.F); }
            else { e.kind = 3; e.v = v - c.F; e.w = (int)__umulhi(r[1], (uint32_t)c.B); }
        } else if (v < c.F) {
            int bs, ps;
            cv.field_place(c, v, j, bs, ps);
            const int bd = p.fix_field_bp ? bs : (int)__umulhi(r[1], (uint32_t)c.B);
            const int len = cv.bp_len(c, bd, j) - (bd == bs ? 1 : 0);
            e = {0, v, 0, bs, ps, bd, (int)__umulhi(r[2], (uint32_t)(len + 1))};
        } else {
            const int b = v - c.F;
            int gs, ps;
            cv.bp_place(c, b, j, gs, ps);
            const int gd = (int)__umulhi(r[1], (uint32_t)c.T);
            const int len = cv.tour_len(c, gd, j) - (gd == gs ? 1 : 0);
            e = {1, b, 0, gs, ps, gd, (int)__umulhi(r[2], (uint32_t)(len + 1))};
        }
        cv.L[j] = e;
        cv.n = j + 1;
    }
}

// Route aggregates (Fig. 1, Sec. 2.2), exact in fixed point so that they do
// not depend on summation order: every per-tour value is a function of the
// tour's content only.
//   per BP: first and last field node, the HU edges between its consecutive
//   fields, the sum of field-to-BP distances, the harvested area;
//   per tour: HU route HQ -> fields in order (across its BPs) -> HQ, SU route
//   HQ -> first field of the first BP -> ... -> (previous BP -> first field of
//   the next BP) ... -> last BP -> HQ, area, and 2 x the mean over its BPs of
//   the mean field-to-BP distance (Algorithm 2, Step 1).
struct BpAgg {
    int first, last, nf;
    long long internal, sb, area;
};

struct TourAgg {
    long long LHU, LSU, A;
    float DB2;
};

__device__ __forceinline__ BpAgg walk_bp(const Ctx &c, const View &x, int b)
{
    BpAgg r;
    r.nf = x.bp_len(c, b);
    r.internal = r.sb = r.area = 0;
    r.first = r.last = -1;
    const int bn = 1 + b;
    int prev = -1;
    for (int k = 0; k < r.nf; ++k) {
        const int f = x.field_at(c, b, k);
        const int fn = 1 + c.B + f;
        if (prev >= 0) r.internal += c.dq(prev, fn);
        else r.first = fn;
        r.sb += c.dq(fn, bn);
        r.area += c.areaq[f];
        prev = fn;
    }
    r.last = prev;
    return r;
}

// A field reinsert (Step 8) changes two BP lists by one element each: update
// the base aggregates from the neighbours of the removed and of the inserted
// field instead of re-walking (exact integer arithmetic, so the result equals
// the walk's).
__device__ __forceinline__ BpAgg bp_agg_reinsert(const Ctx &c, const View &x, int b)
{
    BpAgg r;
    r.nf = c.bp_cnt[b];
    r.first = c.bfirst[b];
    r.last = c.blast[b];
    r.internal = c.bint[b];
    r.sb = c.bsb[b];
    r.area = c.barea[b];
    const int st = c.bp_start[b];
    const int vn = 1 + c.B + x.v;
    if (b == x.sg) {   // removal at position sp
        const int ps = x.sp;
        const int pn = ps > 0 ? 1 + c.B + c.field_order[st + ps - 1] : -1;
        const int nn = ps < r.nf - 1 ? 1 + c.B + c.field_order[st + ps + 1] : -1;
        if (pn >= 0 && nn >= 0) r.internal += c.dq(pn, nn) - c.dq(pn, vn) - c.dq(vn, nn);
        else if (pn >= 0) { r.internal -= c.dq(pn, vn); r.last = pn; }
        else if (nn >= 0) { r.internal -= c.dq(vn, nn); r.first = nn; }
        else { r.first = r.last = -1; }
        r.sb -= c.dq(vn, 1 + b);
        r.area -= c.areaq[x.v];
        r.nf -= 1;
    }
    if (b == x.dg) {   // insertion at position dp of the post-removal list
        const int len = r.nf;
        const bool same = (b == x.sg);
        const int dp = x.dp;
        int an = -1, cn = -1;
        if (dp > 0) { const int j = dp - 1; an = 1 + c.B + c.field_order[st + (same && j >= x.sp ? j + 1 : j)]; }
        if (dp < len) { const int j = dp; cn = 1 + c.B + c.field_order[st + (same && j >= x.sp ? j + 1 : j)]; }
        if (an >= 0 && cn >= 0) r.internal += c.dq(an, vn) + c.dq(vn, cn) - c.dq(an, cn);
        else if (an >= 0) r.internal += c.dq(an, vn);
        else if (cn >= 0) r.internal += c.dq(vn, cn);
        if (dp == 0) r.first = vn;
        if (dp == len) r.last = vn;
        r.sb += c.dq(vn, 1 + b);
        r.area += c.areaq[x.v];
        r.nf += 1;
    }
    return r;
}

// BP b in the candidate: updated or re-walked if its field list changed, else the base's
__device__ __forceinline__ BpAgg bp_agg(const Ctx &c, const View &x, int b)
{
    if (x.kind == 0 && (b == x.sg || b == x.dg)) return bp_agg_reinsert(c, x, b);
    if (x.kind == 2 && (b == c.field_bp[x.v] || b == c.field_bp[x.w])) return walk_bp(c, x, b);
    BpAgg r;
    r.nf = c.bp_cnt[b];
    r.first = c.bfirst[b];
    r.last = c.blast[b];
    r.internal = c.bint[b];
    r.sb = c.bsb[b];
    r.area = c.barea[b];
    return r;
}

__device__ __forceinline__ TourAgg tour_agg(const Ctx &c, const View &x, int g, int nb)
{
    TourAgg t;
    t.LHU = t.LSU = t.A = 0;
    int prev_last = 0, anchor = 0, nonempty = 0;
    float dsum = 0.f;
    for (int j = 0; j < nb; ++j) {
        const int b = x.bp_at(c, g, j);
        const BpAgg a = bp_agg(c, x, b);
        if (a.nf == 0) continue;   // BPs without fields are skipped in routing
        t.LHU += c.dq(prev_last, a.first) + a.internal;
        t.LSU += c.dq(anchor, a.first);
        t.A += a.area;
        dsum = __fadd_rn(dsum, __fmul_rn(__fmul_rn(__ll2float_rn(a.sb), c.dq_scale), c.rcp[a.nf]));
        prev_last = a.last;
        anchor = 1 + b;
        ++nonempty;
    }
    t.LHU += c.dq(prev_last, 0);
    t.LSU += c.dq(anchor, 0);
    t.DB2 = nonempty ? __fmul_rn(2.0f, __fmul_rn(dsum, c.rcp[nonempty])) : 0.f;
    return t;
}

// Eq. 2 for the candidate, exactly: only the BPs whose field set changed are
// re-summed; the others keep the base's status.
__device__ __forceinline__ bool demand_ok(const Ctx &c, const MoveRec &m)
{
    if (m.kind == 0 || m.kind == 2) {
        int b1, b2;
        long long d1, d2;
        if (m.kind == 0) {
            b1 = c.field_bp[m.v]; b2 = m.a;
            d1 = -c.supq[m.v]; d2 = c.supq[m.v];
        } else {
            b1 = c.field_bp[m.v]; b2 = c.field_bp[m.a];
            d1 = c.supq[m.a] - c.supq[m.v]; d2 = -d1;
        }
        if (b1 == b2) return c.nbad == 0;
        const int others = c.nbad - c.bad[b1] - c.bad[b2];
        return others == 0 && c.base_supq[b1] + d1 >= c.demq[b1] && c.base_supq[b2] + d2 >= c.demq[b2];
    }
    return c.nbad == 0;
}

// The same aggregates for a candidate of chained moves, walked through the chain's view.
__device__ __forceinline__ BpAgg walk_bp_chain(const Ctx &c, const ChainView &cv, int b)
{
    BpAgg r;
    r.nf = cv.bp_len(c, b, cv.n);
    r.internal = r.sb = r.area = 0;
    r.first = r.last = -1;
    const int bn = 1 + b;
    int prev = -1;
    for (int k = 0; k < r.nf; ++k) {
        const int fn = 1 + c.B + cv.field_at(c, b, k, cv.n);
        if (prev >= 0) r.internal += c.dq(prev, fn);
        else r.first = fn;
        r.sb += c.dq(fn, bn);
        r.area += c.areaq[fn - 1 - c.B];
        prev = fn;
    }
    r.last = prev;
    return r;
}

__device__ __forceinline__ TourAgg tour_agg_chain(const Ctx &c, const ChainView &cv, int g, int nb)
{
    TourAgg t;
    t.LHU = t.LSU = t.A = 0;
    int prev_last = 0, anchor = 0, nonempty = 0;
    float dsum = 0.f;
    for (int j = 0; j < nb; ++j) {
        const int b = cv.bp_at(c, g, j, cv.n);
        const BpAgg a = walk_bp_chain(c, cv, b);
        if (a.nf == 0) continue;   // BPs without fields are skipped in routing
        t.LHU += c.dq(prev_last, a.first) + a.internal;
        t.LSU += c.dq(anchor, a.first);
        t.A += a.area;
        dsum = __fadd_rn(dsum, __fmul_rn(__fmul_rn(__ll2float_rn(a.sb), c.dq_scale), c.rcp[a.nf]));
        prev_last = a.last;
        anchor = 1 + b;
        ++nonempty;
    }
    t.LHU += c.dq(prev_last, 0);
    t.LSU += c.dq(anchor, 0);
    t.DB2 = nonempty ? __fmul_rn(2.0f, __fmul_rn(dsum, c.rcp[nonempty])) : 0.f;
    return t;
}

// Eq. 2 for a candidate of chained moves: the BPs some field move touched are re-summed exactly
// over their fields in the final plan; the others keep the base's status.
__device__ __forceinline__ bool demand_ok_chain(const Ctx &c, const ChainView &cv)
{
    int bl[2 * kMaxMoves];
    int nb = 0;
#pragma unroll
    for (int l = 0; l < kMaxMoves; ++l) {
        if (l >= cv.n) continue;
        const Lvl &e = cv.L[l];
        int b0 = -1, b1 = -1, p;
        if (e.kind == 0) { b0 = e.s; b1 = e.d; }
        else if (e.kind == 2) { cv.field_place(c, e.v, l, b0, p); cv.field_place(c, e.w, l, b1, p); }
        if (b0 >= 0 && b0 != b1) { bl[nb++] = b0; bl[nb++] = b1; }
    }
    int others = c.nbad;
    bool ok = true;
    for (int q = 0; q < nb; ++q) {
        const int b = bl[q];
        bool dup = false;
        for (int r = 0; r < q; ++r) dup |= (bl[r] == b);
        if (dup) continue;
        others -= c.bad[b];
        long long sum = 0;
        const int nf = cv.bp_len(c, b, cv.n);
        for (int k = 0; k < nf; ++k) sum += c.supq[cv.field_at(c, b, k, cv.n)];
        ok &= sum >= c.demq[b];
    }
    return ok && others == 0;
}

// Eq. 4: n = ceil(s * nsu / cap). FP32 fast path; within 2^-21 of an integer the
// smallest k with k * cap >= s * nsu is found exactly in FP64 (a - p is exact
// by Sterbenz since p is within 1e-6 of a; k*cap = p + e exactly by FMA).
__device__ __noinline__ int exact_ceil(float s, int nsu, double cap, float q)
{
    const double a = (double)s * (double)nsu;
    const double k = rint((double)q);
    const double p = k * cap;
    const double e = fma(k, cap, -p);
    const double dlt = a - p;
    return (dlt > e) ? (int)k + 1 : (int)k;
}

// Critical SU of a set (Eq. 6 reading): largest fill area, ties to the lowest
// id = the first member of the highest tie group in sorted order. m1 is the
// second 64-bit word (sets of more than 64 SUs only).
template <class SH>
__device__ __forceinline__ int su_star(const Ctx &c, typename SH::Mask m0, unsigned long long m1)
{
    using M = typename SH::Mask;
    int hb;
    if (SH::SW > 1 && m1) hb = 64 + hibit_m(m1);
    else hb = hibit_m(m0);
    const int grp = c.sugrp[hb];
    if (SH::SW > 1 && grp >= 64) return 64 + ffs_m(m1 & (~0ull << (grp - 64)));
    const M lo = m0 & (M)(~(M)0 << grp);
    if (lo) return ffs_m(lo);
    return 64 + ffs_m(m1);
}

template <class SH>
__device__ __forceinline__ long long cap_sum(const Ctx &c, typename SH::Mask s0, unsigned long long s1)
{
    long long q = 0;
    while (s0) { const int k = ffs_m(s0); s0 &= s0 - 1; q += c.sucq[k]; }
    if (SH::SW > 1)
        while (s1) { const int k = ffs_m(s1); s1 &= s1 - 1; q += c.sucq[64 + k]; }
    return q;
}

struct ScoreOut {
    float cost, tmax;
    unsigned amask;   // active tours (STAGE 1)
};

// What the full score of a candidate that passed the gate needs from the first
// stage (route aggregates and HU assignment), kept per queued candidate so the
// full score does not repeat them: per tour the HU and SU route lengths, 2 x the
// mean of per-BP means, the HU rate sum and the HU set; the active tours and Tmax.
template <class SH>
struct Survivor {
    float lhu[SH::MAXT], lsu[SH::MAXT], db2[SH::MAXT];
    typename SH::Sum rq[SH::MAXT];
    typename SH::Mask hm[SH::MAXT];
    unsigned amask;
    float tmax;
};
// kept for shapes of at most 8 tours (A and B), where the records fit in shared memory next to the rest
template <class SH>
constexpr bool kKeepSurvivors = SH::MAXT <= 8;

// Per-thread per-tour state: one shared-memory column per value. (Completion
// and waiting times live in registers during the local minimisations; the
// per-tour report of the inspection kernel keeps its own copies.)
template <class SH>
struct TourState {
    static constexpr int MAXT = SH::MAXT, NT = SH::NT;
    using M = typename SH::Mask;
    using S = typename SH::Sum;
    Col<float, NT> LHU, LSU, A, DB2, iR;
    Col<int, NT> star;
    Col<S, NT> Rq, Saq;
    Col<M, NT> Hm, S0;
    Col<unsigned long long, NT> S1;
    __device__ __forceinline__ void bind(unsigned char *base, int tid)
    {
        constexpr int C = MAXT * NT;
        float *f = (float *)base + tid;
        LHU.p = f; LSU.p = f + C; A.p = f + 2 * C; DB2.p = f + 3 * C; iR.p = f + 4 * C;
        int *i = (int *)base + (size_t)NF32 * C + tid;
        star.p = i;
        S *q = (S *)((int *)base + (size_t)(NF32 + 1) * C) + tid;
        Rq.p = q; Saq.p = q + C;
        M *m = (M *)((S *)((int *)base + (size_t)(NF32 + 1) * C) + 2 * C) + tid;
        Hm.p = m; S0.p = m + C;
        // the second SU mask word exists only for sets of more than 64 SUs
        S1.p = (unsigned long long *)((M *)((S *)((int *)base + (size_t)(NF32 + 1) * C) + 2 * C) + 2 * C) + tid;
    }
    __host__ __device__ static constexpr size_t bytes()
    {
        constexpr size_t C = (size_t)MAXT * NT;
        return (NF32 + 1) * C * 4 + 2 * C * sizeof(S) + 2 * C * sizeof(M) + (SH::SW > 1 ? C * 8 : 0);
    }
};

// Per-candidate scoring. DUMP: the inspection kernel's full per-tour report;
// IDENT: the base plan's own T_compl, shuttle ratio and shuttle sum per active
// tour (o_tc, o_kf, o_sh), written without local arrays. STAGE 1: only as far
// as the completion-time gate (route aggregates, HU assignment, Tmax): the cost
// is +inf if the gate discards the candidate, else 0 (not a cost); Tmax depends
// on the HU assignment alone, so the gate decision is final at that point.
// STAGE 2: the rest of the score, resumed from a Survivor record of stage 1.
// CHAIN: the candidate is the chained moves of *cv (m is ignored); its route aggregates and
// shuttle sums are walked through the chain's view.
template <class SH, bool DUMP, bool IDENT = false, int STAGE = 0, bool CHAIN = false>
__device__ ScoreOut score_candidate(const Ctx &c, const SearchParams &p, const MoveRec &m, float tmax_star,
                                    unsigned char *tstate, int tid, int16_t *o_nhu, int16_t *o_nsu, float *o_tc,
                                    float *o_tw, float *o_tcost, int16_t *o_hu, int16_t *o_su, float *o_kf = nullptr,
                                    long long *o_sh = nullptr, const Survivor<SH> *rec = nullptr,
                                    const ChainView *cv = nullptr)
{
    constexpr int MAXT = SH::MAXT, SW = SH::SW;
    using M = typename SH::Mask;
    using S = typename SH::Sum;
    TourState<SH> ts;
    ts.bind(tstate, tid);
    unsigned amask = 0;
    int na = 0;
    float tv[MAXT];   // the round's times, in registers for the picks
    float tmax;
    // per-tour report (DUMP only): completion and waiting times, shuttle sums
    [[maybe_unused]] float dTc[MAXT], dTw[MAXT];
    [[maybe_unused]] long long dSh[MAXT];
#define FOR_ACTIVE(g) _Pragma("unroll") for (int g = 0; g < MAXT; ++g) if ((amask >> g) & 1u)
    ScoreOut out;
    View x;
    if constexpr (CHAIN) x.set(c, MoveRec{4, 0, 0, 0});
    else x.set(c, m);

    if constexpr (STAGE == 2) {
        amask = rec->amask;
        na = __popc(amask);
        tmax = rec->tmax;
#pragma unroll
        for (int g = 0; g < MAXT; ++g)
            if ((amask >> g) & 1u) {
                ts.LHU.set(g, rec->lhu[g]); ts.LSU.set(g, rec->lsu[g]); ts.DB2.set(g, rec->db2[g]);
                ts.Rq.set(g, rec->rq[g]); ts.Hm.set(g, rec->hm[g]);
            }
    } else {
    // --- route aggregates (Fig. 1, Sec. 2.2): rebuild the touched tours, reuse the base's
    unsigned touched;
    if constexpr (CHAIN) touched = cv->touched(c);
    else touched = x.touched(c);
    for (int g = 0; g < c.T; ++g) {
        int nb;
        if constexpr (CHAIN) nb = cv->tour_len(c, g, cv->n);
        else nb = x.tour_len(c, g);
        if (nb == 0) continue;
        amask |= 1u << g;
        ++na;
        long long lhu, lsu, ar;
        float db2;
        if ((touched >> g) & 1u) {
            TourAgg t;
            if constexpr (CHAIN) t = tour_agg_chain(c, *cv, g, nb);
            else t = tour_agg(c, x, g, nb);
            lhu = t.LHU; lsu = t.LSU; ar = t.A; db2 = t.DB2;
        } else {
            lhu = c.tLHU[g]; lsu = c.tLSU[g]; ar = c.tA[g]; db2 = c.tDB2[g];
        }
        ts.LHU.set(g, __fmul_rn(__ll2float_rn(lhu), c.dq_scale));
        ts.LSU.set(g, __fmul_rn(__ll2float_rn(lsu), c.dq_scale));
        ts.A.set(g, __fmul_rn(__ll2float_rn(ar), c.aq_scale));
        ts.DB2.set(g, db2);
    }
    const int di = (na - 1) * c.T;
    const int g_first = __ffs(amask) - 1;

    // --- HU assignment (Sec. 2.5): round-robin dealing, then Algorithm 2 on T_compl
    {
        int j = 0;
        FOR_ACTIVE(g) {
            ts.Hm.set(g, (M)c.hudeal_m[di + j]);
            const S rq = (S)c.hudeal_q[di + j];
            ts.Rq.set(g, rq);
            const float R = __fmul_rn(to_f(rq), c.rqs);
            const float t = __fmaf_rn(ts.LHU.get(g), c.inv_v, __fdividef(ts.A.get(g), R));
            tv[g] = t;
            ++j;
        }
    }
    if (!p.fix_resources && na >= 2) {
        for (int round = 0; round < c.H; ++round) {
            int gx = g_first, gx2 = -1, gn = -1;
            float tx = 0.f, tx2 = 0.f, tn = 0.f;
#pragma unroll
            for (int g = 0; g < MAXT; ++g)
                if (((amask >> g) & 1u) && g == g_first) tx = tv[g];
            FOR_ACTIVE(g) if (tv[g] > tx) { tx = tv[g]; gx = g; }
            FOR_ACTIVE(g) if (g != gx && (gx2 < 0 || tv[g] > tx2)) { tx2 = tv[g]; gx2 = g; }
            if (na == 2) { gn = gx2; tn = tx2; }
            else FOR_ACTIVE(g) if (g != gx && g != gx2 && (gn < 0 || tv[g] < tn)) { tn = tv[g]; gn = g; }
            const M mn = ts.Hm.get(gn);
            if (popc_m(mn) <= 1) break;
            const int last = hibit_m(mn);
            const float Lx = ts.LHU.get(gx), Ax = ts.A.get(gx), Ln = ts.LHU.get(gn), An = ts.A.get(gn);
            const S rqx = ts.Rq.get(gx), rqn = ts.Rq.get(gn);
            M mm = mn;
            int k = -1;
            float tmx = 0.f, tmn = 0.f;
            S nqx = 0, nqn = 0;
            while (mm) {
                k = ffs_m(mm);
                mm &= mm - 1;
                nqx = rqx + (S)c.hurq[k];
                nqn = rqn - (S)c.hurq[k];
                tmx = __fmaf_rn(Lx, c.inv_v, __fdividef(Ax, __fmul_rn(to_f(nqx), c.rqs)));
                tmn = __fmaf_rn(Ln, c.inv_v, __fdividef(An, __fmul_rn(to_f(nqn), c.rqs)));
                const float ref = (na == 2) ? tmn : tx2;
                if (tmx < ref || k == last) break;
            }
            float nm = (tmx > tmn) ? tmx : tmn;
            FOR_ACTIVE(g) if (g != gx && g != gn && tv[g] > nm) nm = tv[g];
            if (!(nm < tx)) break;   // the accepted move does not lower the maximum: keep the old state
            const M bit = (M)1 << k;
            ts.Hm.set(gx, ts.Hm.get(gx) | bit);
            ts.Hm.set(gn, mn & ~bit);
            ts.Rq.set(gx, nqx); ts.Rq.set(gn, nqn);
#pragma unroll
            for (int g = 0; g < MAXT; ++g) tv[g] = (g == gx) ? tmx : ((g == gn) ? tmn : tv[g]);
        }
    }
    tmax = tv[0];
    {
        bool first = true;
        FOR_ACTIVE(g) { tmax = first ? tv[g] : fmaxf(tmax, tv[g]); first = false; }
    }
    if constexpr (DUMP) {
#pragma unroll
        for (int g = 0; g < MAXT; ++g) dTc[g] = tv[g];
    }
    if constexpr (IDENT) {
        FOR_ACTIVE(g) o_tc[g] = tv[g];
    }
    if constexpr (STAGE == 1) {
        out.cost = ((p.gate == 1 && tmax > tmax_star) || (p.gate == 2 && tmax >= tmax_star)) ? __int_as_float(0x7f800000)
                                                                                              : 0.f;
        out.tmax = tmax;
        out.amask = amask;
        return out;
    }
    }   // STAGE != 2
    const int di = (na - 1) * c.T;
    const int g_first = __ffs(amask) - 1;

    // --- SU assignment (Algorithm 2, Eq. 6). R(g) is fixed now: one reciprocal per tour.
    {
        int j = 0;
        FOR_ACTIVE(g) {
            const M m0 = (M)c.sudeal_m[(di + j) * 2];
            const unsigned long long m1 = (SW > 1) ? c.sudeal_m[(di + j) * 2 + 1] : 0ull;
            ts.S0.set(g, m0);
            if (SW > 1) ts.S1.set(g, m1);
            const S sq = (S)c.sudeal_q[di + j];
            ts.Saq.set(g, sq);
            const float ir = __fdividef(1.0f, __fmul_rn(to_f(ts.Rq.get(g)), c.rqs));
            // R(g) is not needed any more: its column holds the tour's SU capacity sum from here on
            ts.Rq.set(g, (S)c.sudeal_c[di + j]);
            ts.iR.set(g, ir);
            const int st = su_star<SH>(c, m0, m1);
            ts.star.set(g, st);
            const float fill = __fmul_rn(to_f((S)(sq - (S)c.sufq[st])), c.fqs);
            const float t = __fmaf_rn(-fill, ir, __fmul_rn(ts.DB2.get(g), c.suinv[st]));
            tv[g] = t;
            ++j;
        }
    }
    if (!p.fix_resources && na >= 2) {
        for (int round = 0; round < c.S; ++round) {
            int gx = g_first, gx2 = -1, gn = -1;
            float tx = 0.f, tx2 = 0.f, tn = 0.f;
#pragma unroll
            for (int g = 0; g < MAXT; ++g)
                if (((amask >> g) & 1u) && g == g_first) tx = tv[g];
            FOR_ACTIVE(g) if (tv[g] > tx) { tx = tv[g]; gx = g; }
            FOR_ACTIVE(g) if (g != gx && (gx2 < 0 || tv[g] > tx2)) { tx2 = tv[g]; gx2 = g; }
            if (na == 2) { gn = gx2; tn = tx2; }
            else FOR_ACTIVE(g) if (g != gx && g != gx2 && (gn < 0 || tv[g] < tn)) { tn = tv[g]; gn = g; }
            const M n0 = ts.S0.get(gn);
            const unsigned long long n1 = (SW > 1) ? ts.S1.get(gn) : 0ull;
            if (popc_m(n0) + (SW > 1 ? popc_m(n1) : 0) <= 1) break;
            const int last = (SW > 1 && n1) ? 64 + hibit_m(n1) : hibit_m(n0);
            const int star_x = ts.star.get(gx), grp_x = c.sugrp[star_x];
            const int star_n = ts.star.get(gn);
            const S sqx = ts.Saq.get(gx), sqn = ts.Saq.get(gn);
            const float DBx = ts.DB2.get(gx), DBn = ts.DB2.get(gn), iRx = ts.iR.get(gx), iRn = ts.iR.get(gn);
            M r0 = n0;
            unsigned long long r1 = n1;
            int k = -1, sx = star_x, sn = star_n;
            float tmx = 0.f, tmn = 0.f;
            while (r0 | (SW > 1 ? r1 : 0ull)) {
                if (r0) { k = ffs_m(r0); r0 &= r0 - 1; }
                else { k = 64 + ffs_m(r1); r1 &= r1 - 1; }
                const float ak = c.sufill[k];
                // g_max gains SU k. Unless k becomes its critical SU (a higher tie group, or the
                // same group at a lower position), one more SU fills during the critical round
                // trip: T_wait drops by a_k / R(g_max) (Eq. 6).
                const int gk = c.sugrp[k];
                if (gk > grp_x || (gk == grp_x && k < star_x)) {
                    sx = k;
                    tmx = __fmaf_rn(-__fmul_rn(to_f(sqx), c.fqs), iRx, __fmul_rn(DBx, c.suinv[k]));
                } else {
                    sx = star_x;
                    tmx = __fmaf_rn(-ak, iRx, tx);
                }
                // g_min loses SU k: T_wait rises by a_k / R(g_min), unless k was its critical SU
                if (k != star_n) {
                    sn = star_n;
                    tmn = __fmaf_rn(ak, iRn, tn);
                } else {
                    M b0 = n0;
                    unsigned long long b1 = n1;
                    if (k < 64) b0 &= ~((M)1 << k); else b1 &= ~(1ull << (k - 64));
                    sn = su_star<SH>(c, b0, b1);
                    tmn = __fmaf_rn(-__fmul_rn(to_f((S)(sqn - (S)c.sufq[k] - (S)c.sufq[sn])), c.fqs), iRn,
                                    __fmul_rn(DBn, c.suinv[sn]));
                }
                const float ref = (na == 2) ? tmn : tx2;
                if (tmx < ref || k == last) break;
            }
            float nm = (tmx > tmn) ? tmx : tmn;
            FOR_ACTIVE(g) if (g != gx && g != gn && tv[g] > nm) nm = tv[g];
            if (!(nm < tx)) break;
            if (k < 64) {
                const M bit = (M)1 << k;
                ts.S0.set(gx, ts.S0.get(gx) | bit);
                ts.S0.set(gn, n0 & ~bit);
            } else {
                ts.S1.set(gx, ts.S1.get(gx) | (1ull << (k - 64)));
                ts.S1.set(gn, n1 & ~(1ull << (k - 64)));
            }
            ts.Saq.set(gx, (S)(sqx + (S)c.sufq[k])); ts.Saq.set(gn, (S)(sqn - (S)c.sufq[k]));
            ts.Rq.set(gx, (S)(ts.Rq.get(gx) + (S)c.sucq[k])); ts.Rq.set(gn, (S)(ts.Rq.get(gn) - (S)c.sucq[k]));
            ts.star.set(gx, sx); ts.star.set(gn, sn);
#pragma unroll
            for (int g = 0; g < MAXT; ++g) tv[g] = (g == gx) ? tmx : ((g == gn) ? tmn : tv[g]);
        }
    }

    if constexpr (DUMP) {
#pragma unroll
        for (int g = 0; g < MAXT; ++g) dTw[g] = tv[g];
    }

    // --- path-length cost (Sec. 2.2, Eq. 4). Shuttle sums in fixed point are exact, so the
    // order in which fields are visited does not matter: walk the base's BP lists and
    // route the (at most two) fields that changed BP separately. The plan's shuttle total
    // is one exact integer; the inspection kernel also keeps it per tour.
    float kfv[MAXT];
#pragma unroll
    for (int g = 0; g < MAXT; ++g) {
        kfv[g] = 0.f;
        if ((amask >> g) & 1u) {
            const M s0 = ts.S0.get(g);
            const unsigned long long s1 = (SW > 1) ? ts.S1.get(g) : 0ull;
            const int nsu = popc_m(s0) + (SW > 1 ? popc_m(s1) : 0);
            kfv[g] = __fdividef((float)nsu, __fmul_rn(__ll2float_rn((long long)ts.Rq.get(g)), c.cqs));
            if constexpr (IDENT) o_kf[g] = kfv[g];
        }
    }
    // A tour's shuttle sum is exact and depends only on its fields, their BPs and its
    // ratio N_SU/sum cap: if neither changed against the base plan, reuse the base's.
    unsigned fresh = amask;
    if (c.memo) {
        unsigned moved = 0u;   // tours whose field -> BP content changed (chains: every touched tour)
        if constexpr (CHAIN) moved = cv->touched(c);
        else if (x.kind == 0 && x.sg != x.dg) moved = (1u << c.bp_tour[x.sg]) | (1u << c.bp_tour[x.dg]);
        else if (x.kind == 1 && x.sg != x.dg) moved = (1u << x.sg) | (1u << x.dg);
        else if (x.kind == 2 && c.field_bp[x.v] != c.field_bp[x.w])
            moved = (1u << c.bp_tour[c.field_bp[x.v]]) | (1u << c.bp_tour[c.field_bp[x.w]]);
        else if (x.kind == 3 && c.bp_tour[x.v] != c.bp_tour[x.w]) moved = (1u << c.bp_tour[x.v]) | (1u << c.bp_tour[x.w]);
        fresh = 0u;
#pragma unroll
        for (int g = 0; g < MAXT; ++g)
            if (((amask >> g) & 1u) && (((moved >> g) & 1u) || kfv[g] != c.kf_base[g])) fresh |= 1u << g;
    }
    // rare exact path of Eq. 4, with the tour's exact capacity sum
    auto ceil_n = [&](int g, float sup, float kf) -> int {
        const float q = __fmul_rn(sup, kf);
        const float rq = rintf(q);
        if (fabsf(q - rq) > q * (1.0f / 2097152.0f)) return (int)ceilf(q);
        const M s0 = ts.S0.get(g);
        const unsigned long long s1 = (SW > 1) ? ts.S1.get(g) : 0ull;
        const int nsu = popc_m(s0) + (SW > 1 ? popc_m(s1) : 0);
        return exact_ceil(sup, nsu, (double)ts.Rq.get(g) * c.cqs_d, q);
    };
    long long shq = 0;
    for (int g = 0; g < c.T; ++g) {
        if (!((amask >> g) & 1u)) continue;
        const long long v0 = ((fresh >> g) & 1u) ? 0ll : c.sh_base[g];
        if constexpr (DUMP) dSh[g] = v0;
        if constexpr (IDENT) o_sh[g] = v0;
        shq += v0;
    }
    if (CHAIN && fresh) {
        // chained moves: walk the fresh tours' BPs through the chain's view
        for (int b = 0; b < c.B; ++b) {
            const int g = cv->tour_of_bp(c, b);
            if (!((fresh >> g) & 1u)) continue;
            float kf = kfv[0];
#pragma unroll
            for (int t = 1; t < MAXT; ++t)
                if (g == t) kf = kfv[t];
            long long acc = 0;
            const int nf = cv->bp_len(c, b, cv->n);
            for (int k = 0; k < nf; ++k) {
                const int f = cv->field_at(c, b, k, cv->n);
                const int n = ceil_n(g, c.supply[f], kf);
                acc += (long long)n * c.dq(1 + c.B + f, 1 + b);
            }
            shq += acc;
            if constexpr (DUMP) dSh[g] += acc;
            if constexpr (IDENT) o_sh[g] += acc;
        }
    } else if (fresh) {
        // base positions of the fields that left their BP (added at their new BP below)
        int skip0 = -1, skip1 = -1;
        if (x.kind == 0 && x.sg != x.dg) skip0 = c.bp_start[x.sg] + c.field_pos[x.v];
        if (x.kind == 2 && c.field_bp[x.v] != c.field_bp[x.w]) {
            skip0 = c.bp_start[c.field_bp[x.v]] + c.field_pos[x.v];
            skip1 = c.bp_start[c.field_bp[x.w]] + c.field_pos[x.w];
        }
        for (int b = 0; b < c.B; ++b) {
            const int g = x.tour_of_bp(c, b);
            if (!((fresh >> g) & 1u)) continue;
            float kf = kfv[0];
#pragma unroll
            for (int t = 1; t < MAXT; ++t)
                if (g == t) kf = kfv[t];
            long long acc = 0;
            const int k0 = c.bp_start[b], k1 = k0 + c.bp_cnt[b];
            for (int kk = k0; kk < k1; ++kk) {
                if (kk == skip0 || kk == skip1) continue;
                const int2 sd = c.psd[kk];
                const int n = ceil_n(g, __int_as_float(sd.x), kf);
                acc += (long long)n * (long long)sd.y;
            }
            shq += acc;
            if constexpr (DUMP) dSh[g] += acc;
            if constexpr (IDENT) o_sh[g] += acc;
        }
        int mv_f0 = -1, mv_f1 = -1;
        if (x.kind == 0 && x.sg != x.dg) mv_f0 = x.v;
        if (x.kind == 2 && c.field_bp[x.v] != c.field_bp[x.w]) { mv_f0 = x.v; mv_f1 = x.w; }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int f = q == 0 ? mv_f0 : mv_f1;
            if (f >= 0) {
                const int b = x.bp_of_field(c, f);
                const int g = x.tour_of_bp(c, b);
                float kf = kfv[0];
#pragma unroll
                for (int t = 1; t < MAXT; ++t)
                    if (g == t) kf = kfv[t];
                const int n = ceil_n(g, c.supply[f], kf);
                const long long a = (long long)n * c.dq(1 + c.B + f, 1 + b);
                shq += a;
                if constexpr (DUMP) dSh[g] += a;
                if constexpr (IDENT) o_sh[g] += a;
            }
        }
    }
    float cost = 0.f;
    for (int g = 0; g < c.T; ++g) {
        if (!((amask >> g) & 1u)) continue;
        const M hm = ts.Hm.get(g);
        const M s0 = ts.S0.get(g);
        const unsigned long long s1 = (SW > 1) ? ts.S1.get(g) : 0ull;
        const int nhu = popc_m(hm);
        const int nsu = popc_m(s0) + (SW > 1 ? popc_m(s1) : 0);
        const float route = __fadd_rn(__fmul_rn((float)nhu, ts.LHU.get(g)), __fmul_rn((float)nsu, ts.LSU.get(g)));
        cost = __fadd_rn(cost, route);
        if constexpr (DUMP) {
            const float shuttle = __fmul_rn(__fmul_rn(__ll2float_rn(dSh[g]), c.dq_scale), 2.0f);
            if (o_nhu) o_nhu[g] = (int16_t)nhu;
            if (o_nsu) o_nsu[g] = (int16_t)nsu;
            if (o_tc) o_tc[g] = dTc[g];
            if (o_tw) o_tw[g] = dTw[g];
            if (o_kf) o_kf[g] = kfv[g];
            if (o_sh) o_sh[g] = dSh[g];
            if (o_tcost) o_tcost[g] = __fadd_rn(route, shuttle);
            if (o_hu) {
                M r = hm;
                while (r) { const int k = ffs_m(r); r &= r - 1; o_hu[c.hu_id[k]] = (int16_t)g; }
            }
            if (o_su) {
                M r = s0;
                while (r) { const int k = ffs_m(r); r &= r - 1; o_su[c.su_id[k]] = (int16_t)g; }
                if (SW > 1) {
                    unsigned long long r2 = s1;
                    while (r2) { const int k = ffs_m(r2); r2 &= r2 - 1; o_su[c.su_id[64 + k]] = (int16_t)g; }
                }
            }
        }
    }
    cost = __fadd_rn(cost, __fmul_rn(__fmul_rn(__ll2float_rn(shq), c.dq_scale), 2.0f));
    // --- completion-time gate (Sec. 2.5)
    if ((p.gate == 1 && tmax > tmax_star) || (p.gate == 2 && tmax >= tmax_star)) cost = __int_as_float(0x7f800000);
    out.cost = cost;
    out.tmax = tmax;
    return out;
#undef FOR_ACTIVE
}

// ---------------------------------------------------------------------------
// Shared-memory carving
// ---------------------------------------------------------------------------
__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

struct SmemPlan {
    size_t off_blob, off_plan, off_derived, off_supq, off_bad, off_base_agg, off_tour, off_qidx, off_qmv, off_qidx2,
        off_qmv2, off_surv, total;
};

__host__ __device__ inline SmemPlan carve(size_t tour_bytes, int threads, int max_prefix, int max_plan_len, int max_F,
                                          int max_B, int max_T, size_t surv_bytes = 0)
{
    SmemPlan s;
    size_t o = 0;
    s.off_blob = o; o += align16((size_t)max_prefix);
    s.off_plan = o; o += align16((size_t)max_plan_len * 2);
    s.off_derived = o; o += align16((size_t)(max_T + 3 * max_B + 2 * max_F) * 2);
    s.off_supq = o; o += align16((size_t)max_B * 8);
    s.off_bad = o; o += align16((size_t)max_B);
    s.off_base_agg = o; o += align16((size_t)max_B * 3 * 8 + (size_t)max_T * (3 * 8 + 4 + 4) + (size_t)max_T * 8 +
                                     (size_t)max_F * 8 + (size_t)max_B * 2 * 2);
    s.off_tour = o; o += align16(tour_bytes);
    s.off_qidx = o; o += align16((size_t)(threads / 32) * WQ * 4);
    s.off_qmv = o; o += align16((size_t)(threads / 32) * WQ * 8);
    s.off_qidx2 = o; o += align16((size_t)(threads / 32) * WQ * 4);   // candidates that passed the gate
    s.off_qmv2 = o; o += align16((size_t)(threads / 32) * WQ * 8);
    s.off_surv = o; o += align16((size_t)(threads / 32) * WQ * surv_bytes);   // and their first-stage results
    s.total = o;
    return s;
}

template <class SH>
__host__ __device__ inline SmemPlan carve_shape(int max_prefix, int max_plan_len, int max_F, int max_B, int max_T)
{
    return carve(TourState<SH>::bytes(), SH::NT, max_prefix, max_plan_len, max_F, max_B, max_T,
                 kKeepSurvivors<SH> ? sizeof(Survivor<SH>) : 0);
}

struct BlockShared {
    uint64_t mbar;
    uint32_t phase;
    int32_t staged;
    int32_t nbad;
    int32_t last;
    int32_t use_best;
    uint32_t iter;
    int32_t cursor;   // next undrawn candidate position of the work item (chunks of 32)
    float base_cost;
    float base_tc[16];
    unsigned long long red[32];
    float redt[32];
};

// Stage instance `inst` (tables by bulk copy, base plan, derived tables, base
// per-BP and per-tour aggregates), without the base plan's own scoring.
// Returns false if the bounded wait gave up (error flag set).
template <class SH>
__device__ bool stage_base(const InstMeta &M, BlockShared &bs, unsigned char *smem, const SmemPlan &sp,
                           const SearchParams &p, int use_best_override, uint32_t iter_override, Ctx &c)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    const uint32_t bytes = SH::DSM ? (uint32_t)M.L.total_bytes : (uint32_t)M.L.prefix_bytes;
    __syncthreads();
    if (tid == 0) {
        fence_proxy_async_smem();
        mbar_expect_tx(&bs.mbar, bytes);
        bulk_copy_g2s(smem + sp.off_blob, M.blob, bytes, &bs.mbar);
        uint32_t it = (iter_override == 0xffffffffu) ? M.state->iter : iter_override;
        int ub;
        if (use_best_override >= 0) ub = use_best_override;
        else {
            // Eq. 5: x = x* if u < eps, else x_old; u from counter (0, iter, inst, 1)
            uint32_t r[4] = {0u, it, M.inst_idx, 1u};
            philox10(r, p.seed_lo, p.seed_hi);
            ub = unit24f(r[0]) < p.eps;
        }
        bs.use_best = ub;
        bs.iter = it;
    }
    __syncthreads();
    int16_t *plan = (int16_t *)(smem + sp.off_plan);
    {
        const int16_t *src = bs.use_best ? M.xbest : M.xold;
        const int n4 = M.plan_len / 4;   // plan_len is a multiple of 8
        const uint2 *s2 = (const uint2 *)src;
        uint2 *d2 = (uint2 *)plan;
        for (int k = tid; k < n4; k += nt) d2[k] = s2[k];
    }
    // every thread must take the same branch below: agree on the outcome
    const bool ok = __syncthreads_and(mbar_wait_bounded(&bs.mbar, bs.phase) ? 1 : 0) != 0;
    if (tid == 0) bs.phase ^= 1u;
    if (!ok) {
        if (tid == 0) atomicExch(&M.state->error, 1u);
        return false;
    }
    const unsigned char *blob = smem + sp.off_blob;
    c.F = M.F; c.B = M.B; c.T = M.T; c.H = M.H; c.S = M.S; c.N = M.N;
    c.Dq = SH::DSM ? (const int *)(blob + M.L.off_D) : (const int *)(M.blob + M.L.off_D);
    c.area = (const float *)(blob + M.L.off_area);
    c.areaq = (const long long *)(blob + M.L.off_areaq);
    c.supply = (const float *)(blob + M.L.off_supply);
    c.supq = (const long long *)(blob + M.L.off_supq);
    c.demq = (const long long *)(blob + M.L.off_demq);
    c.hurq = (const long long *)(blob + M.L.off_hurq);
    c.sufq = (const long long *)(blob + M.L.off_sufq);
    c.sucq = (const long long *)(blob + M.L.off_sucq);
    c.suinv = (const float *)(blob + M.L.off_suinv);
    c.sufill = (const float *)(blob + M.L.off_sufill);
    c.rcp = (const float *)(blob + M.L.off_rcp);
    c.sugrp = (const int *)(blob + M.L.off_sugrp);
    c.hudeal_m = (const unsigned long long *)(blob + M.L.off_hudeal_m);
    c.hudeal_q = (const long long *)(blob + M.L.off_hudeal_q);
    c.sudeal_m = (const unsigned long long *)(blob + M.L.off_sudeal_m);
    c.sudeal_q = (const long long *)(blob + M.L.off_sudeal_q);
    c.sudeal_c = (const long long *)(blob + M.L.off_sudeal_c);
    c.hu_id = (const int *)(blob + M.L.off_hu_id);
    c.su_id = (const int *)(blob + M.L.off_su_id);
    c.inv_v = M.inv_hu_speed; c.rqs = M.rq_scale; c.fqs = M.fq_scale; c.cqs = M.cq_scale; c.cqs_d = M.cq_scale_d;
    c.dq_inv = M.dq_inv; c.dq_scale = M.dq_scale; c.aq_scale = M.aq_scale;
    const int B = M.B, T = M.T, F = M.F;
    c.bp_order = plan;
    c.tour_cnt = plan + B;
    c.field_order = plan + B + T;
    c.bp_cnt = plan + B + T + F;
    int16_t *der = (int16_t *)(smem + sp.off_derived);
    int16_t *tour_start = der, *bp_start = der + T, *bp_tour = der + T + B, *bp_pos = der + T + 2 * B;
    int16_t *field_bp = der + T + 3 * B, *field_pos = der + T + 3 * B + F;
    long long *base_supq = (long long *)(smem + sp.off_supq);
    int8_t *bad = (int8_t *)(smem + sp.off_bad);
    unsigned char *bt = smem + sp.off_base_agg;   // base per-BP and per-tour tables
    long long *bint = (long long *)bt, *bsb = bint + B, *barea = bsb + B;
    long long *tLHU = barea + B, *tLSU = tLHU + T, *tA = tLSU + T;
    float *tDB2 = (float *)(tA + T);
    float *kf_base = tDB2 + T;
    long long *sh_base = (long long *)(bt + (size_t)B * 3 * 8 + (size_t)T * (3 * 8 + 4 + 4));
    int2 *psd = (int2 *)(sh_base + T);
    int16_t *bfirst = (int16_t *)(psd + F), *blast = bfirst + B;
    c.tour_start = tour_start; c.bp_start = bp_start; c.bp_tour = bp_tour; c.bp_pos = bp_pos;
    c.field_bp = field_bp; c.field_pos = field_pos; c.base_supq = base_supq; c.bad = bad;
    c.bint = bint; c.bsb = bsb; c.barea = barea; c.tLHU = tLHU; c.tLSU = tLSU; c.tA = tA; c.tDB2 = tDB2;
    c.psd = psd; c.bfirst = bfirst; c.blast = blast; c.kf_base = kf_base; c.sh_base = sh_base; c.memo = 0;
    if (tid == 0) {
        int s = 0;
        for (int g = 0; g < T; ++g) { tour_start[g] = (int16_t)s; s += c.tour_cnt[g]; }
        s = 0;
        for (int b = 0; b < B; ++b) { bp_start[b] = (int16_t)s; s += c.bp_cnt[b]; }
    }
    __syncthreads();
    for (int g = tid; g < T; g += nt)
        for (int m = 0; m < c.tour_cnt[g]; ++m) {
            const int b = c.bp_order[tour_start[g] + m];
            bp_tour[b] = (int16_t)g; bp_pos[b] = (int16_t)m;
        }
    for (int b = tid; b < B; b += nt) {
        long long s = 0;
        for (int k = 0; k < c.bp_cnt[b]; ++k) {
            const int f = c.field_order[bp_start[b] + k];
            field_bp[f] = (int16_t)b; field_pos[f] = (int16_t)k;
            s += c.supq[f];
            psd[bp_start[b] + k] = make_int2(__float_as_int(c.supply[f]), c.Dq[(1 + B + f) * c.N + 1 + b]);
        }
        base_supq[b] = s;
        bad[b] = (int8_t)(s < c.demq[b] ? 1 : 0);
    }
    __syncthreads();
    if (tid == 0) {
        int nb = 0;
        for (int b = 0; b < B; ++b) nb += bad[b];
        bs.nbad = nb;
    }
    // base plan's per-BP aggregates, then per-tour aggregates, with the same code as candidates
    View idv;
    idv.kind = 4; idv.v = idv.w = idv.sg = idv.sp = idv.dg = idv.dp = -1;
    for (int b = tid; b < B; b += nt) {
        const BpAgg a = walk_bp(c, idv, b);
        bfirst[b] = (int16_t)a.first; blast[b] = (int16_t)a.last;
        bint[b] = a.internal; bsb[b] = a.sb; barea[b] = a.area;
    }
    __syncthreads();
    for (int g = tid; g < T; g += nt) {
        const int nb = c.tour_cnt[g];
        TourAgg t;
        t.LHU = t.LSU = t.A = 0; t.DB2 = 0.f;
        if (nb > 0) t = tour_agg(c, idv, g, nb);
        tLHU[g] = t.LHU; tLSU[g] = t.LSU; tA[g] = t.A; tDB2[g] = t.DB2;
    }
    __syncthreads();
    return true;
}

// The base plan's own per-tour T_compl, shuttle ratio and shuttle sum (the
// shuttle memo of the candidates' scoring), scored by the calling thread with
// the candidates' code; c.memo must still be 0.
template <class SH>
__device__ __forceinline__ void score_base(const InstMeta &M, BlockShared &bs, unsigned char *smem, const SmemPlan &sp,
                                        const SearchParams &p, Ctx &c)
{
    const int T = M.T;
    float *kf_base = const_cast<float *>(c.kf_base);
    long long *sh_base = const_cast<long long *>(c.sh_base);
    c.nbad = bs.nbad;
    for (int g = 0; g < T; ++g) { kf_base[g] = 0.f; sh_base[g] = 0; }
    bs.base_cost = __int_as_float(0x7f800000);
    for (int g = 0; g < T && g < 16; ++g) bs.base_tc[g] = 0.f;
    if (bs.nbad == 0) {
        const MoveRec idm = {4, 0, 0, 0};
        bs.base_cost = score_candidate<SH, false, true>(c, p, idm, __int_as_float(0x7f800000), smem + sp.off_tour,
                                                        threadIdx.x, nullptr, nullptr, bs.base_tc, nullptr, nullptr,
                                                        nullptr, nullptr, kf_base, sh_base)
                           .cost;
    }
}

// stage_base, then the base plan scored by thread 0 (score_base).
template <class SH>
__device__ bool stage_instance(const InstMeta &M, BlockShared &bs, unsigned char *smem, const SmemPlan &sp,
                               const SearchParams &p, int use_best_override, uint32_t iter_override, Ctx &c)
{
    if (!stage_base<SH>(M, bs, smem, sp, p, use_best_override, iter_override, c)) return false;
    if (threadIdx.x == 0) score_base<SH>(M, bs, smem, sp, p, c);
    __syncthreads();
    c.nbad = bs.nbad;
    c.memo = 1;
    return true;
}

// Named barrier 1 (barrier 0 is __syncthreads): the producer warp arrives
// without waiting, the consumer warps wait until all `n` threads have arrived.
__device__ __forceinline__ void named_arrive(int n)
{
    asm volatile("bar.arrive 1, %0;" ::"r"(n) : "memory");
}
__device__ __forceinline__ void named_sync(int n)
{
    asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory");
}

// List mode: an instance's kept candidates are dealt to as many of its work
// items as the grid runs side by side (about one per block), a multiple of 32
// each; its remaining work items are empty and only report an empty slot.
__device__ __forceinline__ int list_tile(const InstMeta &M, int list_n, int n_work)
{
    const int n = min(M.n_cand, list_n);
    const long long share = (long long)M.n_tiles * gridDim.x / (n_work > 0 ? n_work : 1);
    const int items = (int)(share < 1 ? 1 : (share < M.n_tiles ? share : M.n_tiles));
    return max(32, ((n + items - 1) / items + 31) & ~31);
}

__device__ __forceinline__ unsigned long long make_key(float cost, uint32_t i)
{
    return ((unsigned long long)__float_as_uint(cost) << 32) | (unsigned long long)i;
}

// Write the candidate plan (base + move) as an encoding.
__device__ void write_plan(const Ctx &c, const MoveRec &m, int16_t *out)
{
    View x;
    x.set(c, m);
    int k = 0;
    for (int g = 0; g < c.T; ++g) {
        const int nb = x.tour_len(c, g);
        for (int j = 0; j < nb; ++j) out[k++] = (int16_t)x.bp_at(c, g, j);
    }
    for (int g = 0; g < c.T; ++g) out[c.B + g] = (int16_t)x.tour_len(c, g);
    k = c.B + c.T;
    for (int b = 0; b < c.B; ++b) {
        const int nf = x.bp_len(c, b);
        for (int j = 0; j < nf; ++j) out[k++] = (int16_t)x.field_at(c, b, j);
    }
    for (int b = 0; b < c.B; ++b) out[c.B + c.T + c.F + b] = (int16_t)x.bp_len(c, b);
}

// Write a candidate of chained moves as an encoding.
__device__ void write_plan_chain(const Ctx &c, const ChainView &cv, int16_t *out)
{
    int k = 0;
    for (int g = 0; g < c.T; ++g) {
        const int nb = cv.tour_len(c, g, cv.n);
        for (int j = 0; j < nb; ++j) out[k++] = (int16_t)cv.bp_at(c, g, j, cv.n);
    }
    for (int g = 0; g < c.T; ++g) out[c.B + g] = (int16_t)cv.tour_len(c, g, cv.n);
    k = c.B + c.T;
    for (int b = 0; b < c.B; ++b) {
        const int nf = cv.bp_len(c, b, cv.n);
        for (int j = 0; j < nf; ++j) out[k++] = (int16_t)cv.field_at(c, b, j, cv.n);
    }
    for (int b = 0; b < c.B; ++b) out[c.B + c.T + c.F + b] = (int16_t)cv.bp_len(c, b, cv.n);
}

// ---------------------------------------------------------------------------
// The search iteration kernel
// ---------------------------------------------------------------------------
// Block argmin of the work item's candidates (warp shuffle, then across
// warps) into its slot; the last work item of the instance to finish takes the
// argmin over the instance's slots and runs Steps 13-16 (replay the move,
// update x_old, x*, C*, Tmax*, the log and the iteration counter).
// Steps 13-16 of one instance with the iteration's argmin key bk (cost bits << 32 | i*) and the
// winner's Tmax bt: replay move(s) i* on the staged base into x_old (x_old <- base if no candidate
// is feasible), update x*, C*, Tmax* if C_{i*} < C*, log the iteration and advance the counter.
// One thread.
template <bool CHAIN>
__device__ void apply_update(const Ctx &c, const SearchParams &prm, const InstMeta &M, int use_best, uint32_t iter,
                             unsigned long long bk, float bt)
{
    const uint32_t istar = (uint32_t)(bk & 0xffffffffu);
    const float cst = __uint_as_float((uint32_t)(bk >> 32));
    InstState *st = M.state;
    int ind = 0;
    if (isfinite(cst)) {
        int kind0;
        if constexpr (CHAIN) {
            ChainView cv;
            draw_chain(c, prm, istar, iter, M.inst_idx, cv);
            write_plan_chain(c, cv, M.xold);
            kind0 = cv.L[0].kind;
        } else {
            const MoveRec m = draw_move(c, prm, istar, iter, M.inst_idx);
            write_plan(c, m, M.xold);
            kind0 = m.kind;
        }
        if (cst < st->cstar) {
            for (int k = 0; k < M.plan_len; ++k) M.xbest[k] = M.xold[k];
            st->cstar = cst;
            st->tmaxstar = bt;
            ind = (kind0 == 0 || kind0 == 2) ? 1 : 2;   // the (first) move's type (Fig. 3)
        }
    } else {
        const int16_t *pl = c.bp_order;
        for (int k = 0; k < M.plan_len; ++k) M.xold[k] = pl[k];
    }
    const int li = (int)(iter % (uint32_t)M.log_cap);
    M.log_istar[li] = (int32_t)istar;
    M.log_cistar[li] = cst;
    M.log_usebest[li] = (int8_t)use_best;
    M.log_cstar[li] = st->cstar;
    M.log_ind[li] = (int8_t)ind;
    st->iter = iter + 1;
    st->done = 0;
}

template <int NT, bool CHAIN = false>
__device__ __forceinline__ void block_argmin_finalize(unsigned long long best, float best_t, BlockShared &bs,
                                                      const InstMeta &M, const WorkItem &wi,
                                                      unsigned long long *__restrict__ slot_key,
                                                      float *__restrict__ slot_tmax,
                                                      const int32_t *__restrict__ slot_base, const Ctx &c,
                                                      const SearchParams &prm, uint32_t iter)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // block argmin: warp shuffle, then across warps
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(0xffffffffu, best, o);
        const float ot = __shfl_xor_sync(0xffffffffu, best_t, o);
        if (ok < best) { best = ok; best_t = ot; }
    }
    if (lane == 0) { bs.red[warp] = best; bs.redt[warp] = best_t; }
    __syncthreads();
    if (tid < 32) {
        const int nw = NT >> 5;
        best = (tid < nw) ? bs.red[tid] : ~0ull;
        best_t = (tid < nw) ? bs.redt[tid] : 0.f;
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ok = __shfl_xor_sync(0xffffffffu, best, o);
            const float ot = __shfl_xor_sync(0xffffffffu, best_t, o);
            if (ok < best) { best = ok; best_t = ot; }
        }
        if (tid == 0) {
            const int slot = slot_base[wi.inst] + wi.tile_idx;
            slot_key[slot] = best;
            slot_tmax[slot] = best_t;
            __threadfence();
            const uint32_t prev = atomicAdd(&M.state->done, 1u);
            bs.last = (prev == (uint32_t)(M.n_tiles - 1)) ? 1 : 0;
        }
    }
    __syncthreads();
    if (bs.last) {
        // Steps 13-16 for this instance: argmin over its work items
        __threadfence();
        if (tid < 32) {
            unsigned long long bk = ~0ull;
            float bt = 0.f;
            const int s0 = slot_base[wi.inst];
            for (int s = tid; s < M.n_tiles; s += 32) {
                const unsigned long long k = __ldcg(&slot_key[s0 + s]);
                const float t = __ldcg(&slot_tmax[s0 + s]);
                if (k < bk) { bk = k; bt = t; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
                const float ot = __shfl_xor_sync(0xffffffffu, bt, o);
                if (ok < bk) { bk = ok; bt = ot; }
            }
            if (tid == 0) {
                if (prm.defer_update) {   // a slice of a split iteration: the key waits for the other slices
                    M.state->key = bk;
                    M.state->done = 0;
                } else {
                    apply_update<CHAIN>(c, prm, M, bs.use_best, iter, bk, bt);
                }
            }
        }
    }
    __syncthreads();
}

template <class SH, bool CHAIN>
__global__ void __launch_bounds__(SH::NT, SH::MINB) search_iteration_kernel(const InstMeta *__restrict__ meta,
                                                                  const WorkItem *__restrict__ work, int32_t n_work,
                                                                  SearchParams prm, SmemPlan sp,
                                                                  unsigned long long *__restrict__ slot_key,
                                                                  float *__restrict__ slot_tmax,
                                                                  const int32_t *__restrict__ slot_base,
                                                                  const uint32_t *__restrict__ cand_list,
                                                                  const int32_t *__restrict__ cand_count,
                                                                  int32_t list_stride, float2 *__restrict__ insp,
                                                                  int32_t insp_stride)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BlockShared bs;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int NT = SH::NT;
    if (tid == 0) {
        mbar_init(&bs.mbar, 1);
        fence_mbar_init();
        bs.phase = 0;
        bs.staged = -1;
    }
    __syncthreads();
    unsigned char *tstate = smem + sp.off_tour;
    int32_t *qidx = (int32_t *)(smem + sp.off_qidx) + warp * WQ;
    int2 *qmv = (int2 *)(smem + sp.off_qmv) + warp * WQ;
    int32_t *qidx2 = (int32_t *)(smem + sp.off_qidx2) + warp * WQ;
    int2 *qmv2 = (int2 *)(smem + sp.off_qmv2) + warp * WQ;
    Survivor<SH> *surv = (Survivor<SH> *)(smem + sp.off_surv) + warp * WQ;   // used where kKeepSurvivors
    Ctx c;
    for (int w = blockIdx.x; w < n_work; w += gridDim.x) {
        const WorkItem wi = work[w];
        const InstMeta &M = meta[wi.inst];
        const bool fresh_inst = bs.staged != wi.inst;
        if (fresh_inst) {
            if (!stage_base<SH>(M, bs, smem, sp, prm, -1, 0xffffffffu, c)) return;
            if (tid == 0) bs.staged = wi.inst;
        }
        const float tmax_star = M.state->tmaxstar;
        const uint32_t iter = bs.iter;
        // list mode (learned proposals): positions index instance wi.inst's list of candidate numbers
        const int list_n = cand_list ? cand_count[wi.inst] : 0;
        const uint32_t *ilist = cand_list ? cand_list + (size_t)wi.inst * list_stride : nullptr;
        // list mode: the kept candidates go to about one work item per block (list_tile),
        // whatever the tile the full pool was planned with
        const int tl = cand_list ? list_tile(M, list_n, n_work) : M.tile;
        // positions [c0, c1) of the instance's candidates (or of its list); empty past the end
        const long long cend = cand_list ? min(M.n_cand, list_n) : M.n_cand;
        const long long c0l = (long long)wi.tile_idx * tl;
        const int c0 = (int)min(c0l, cend);
        const int c1 = (int)min(c0l + tl, cend);
        // inspection (off in the timed path): {C_i, Tmax_i} of candidate i where it is decided
        float2 *const ins = insp ? insp + (size_t)wi.inst * insp_stride : nullptr;
        unsigned long long best = ~0ull;
        float best_t = 0.f;
        // each warp: draw 32 moves at a time and queue the feasible ones (Eq. 2); take 32 queued
        // at a time as far as the completion-time gate and queue those it keeps; score 32 of
        // those at a time in full. The gate discards most feasible candidates: their cost is
        // +inf once Tmax is known, and the SU assignment and shuttle pass run in full warps
        // of the others only.
        // Warps take chunks of 32 positions from a block-wide cursor, so a warp whose candidates
        // ran through the gate quickly draws more and all warps run out of draws together.
        int qhead = 0, qcount = 0;     // warp-uniform ring-buffer state, feasible candidates
        int q2head = 0, q2count = 0;   // candidates the gate kept
        if (tid == 0) bs.cursor = c0 + NT;
        __syncthreads();
        // A freshly staged instance: warp 0 scores the base plan (the shuttle memo) while the
        // other warps draw and take candidates to the gate; they wait for it (named barrier 1)
        // before their first full score, or at the end if they have none.
        bool memo_wait = false;
        if (fresh_inst) {
            if (warp == 0) {
                if (lane == 0) score_base<SH>(M, bs, smem, sp, prm, c);
                __syncwarp();
                __threadfence_block();
                named_arrive(NT);
            } else {
                memo_wait = true;
            }
            c.nbad = bs.nbad;
            c.memo = 1;
        }
        for (int base = c0 + warp * 32;;) {
            // (an empty range, past the end of a list, only reports an empty slot)
            int next = c1;   // this warp's next chunk
            if (base < c1) {
                const int pos = base + lane;
                const int i = (ilist && pos < c1) ? (int)ilist[pos] : (int)prm.cand_offset + pos;
                bool feas = false;
                MoveRec m = {4, 0, 0, 0};
                if (pos < c1) {
                    if constexpr (CHAIN) {   // the queue keeps i only: later stages draw the chain again
                        ChainView cv;
                        draw_chain(c, prm, (uint32_t)i, iter, M.inst_idx, cv);
                        feas = demand_ok_chain(c, cv);
                    } else {
                        m = draw_move(c, prm, (uint32_t)i, iter, M.inst_idx);
                        feas = demand_ok(c, m);
                    }
                    if (!feas) {
                        const unsigned long long k = make_key(__int_as_float(0x7f800000), (uint32_t)i);
                        if (k < best) { best = k; best_t = __int_as_float(0x7f800000); }
                        if (ins) ins[i - (int)prm.cand_offset] = make_float2(__int_as_float(0x7f800000), __int_as_float(0x7f800000));
                    }
                }
                const unsigned ball = __ballot_sync(0xffffffffu, feas);
                if (feas) {
                    const int slot = (qhead + qcount + __popc(ball & ((1u << lane) - 1u))) & (WQ - 1);
                    qidx[slot] = i;
                    qmv[slot] = make_int2((m.kind & 0xffff) | (m.v << 16), (m.a & 0xffff) | (m.b << 16));
                }
                qcount += __popc(ball);
                __syncwarp();
                int nb = 0;
                if (lane == 0) nb = atomicAdd(&bs.cursor, 32);
                next = __shfl_sync(0xffffffffu, nb, 0);
            }
            const bool drained = next >= c1;   // no more draws for this warp
            // up to the gate for a full warp of feasible candidates, or the remainder once drained
            const int take = (qcount >= 32) ? 32 : (drained ? qcount : 0);
            if (take > 0) {
                bool kept = false;
                int i = 0;
                int2 pm = make_int2(0, 0);
                ScoreOut r1 = {0.f, 0.f, 0u};
                if (lane < take) {
                    const int slot = (qhead + lane) & (WQ - 1);
                    i = qidx[slot];
                    pm = qmv[slot];
                    const MoveRec m = {pm.x & 0xffff, pm.x >> 16, pm.y & 0xffff, pm.y >> 16};
                    if constexpr (CHAIN) {
                        ChainView cv;
                        draw_chain(c, prm, (uint32_t)i, iter, M.inst_idx, cv);
                        r1 = score_candidate<SH, false, false, 1, true>(c, prm, m, tmax_star, tstate, tid, nullptr,
                                                                        nullptr, nullptr, nullptr, nullptr, nullptr,
                                                                        nullptr, nullptr, nullptr, nullptr, &cv);
                    } else {
                        r1 = score_candidate<SH, false, false, 1>(c, prm, m, tmax_star, tstate, tid, nullptr, nullptr,
                                                                  nullptr, nullptr, nullptr, nullptr, nullptr);
                    }
                    if (isinf(r1.cost)) {   // discarded by the gate: C = +inf (Sec. 2.5)
                        const unsigned long long k = make_key(r1.cost, (uint32_t)i);
                        if (k < best) { best = k; best_t = r1.tmax; }
                        if (ins) ins[i - (int)prm.cand_offset] = make_float2(r1.cost, r1.tmax);
                    } else {
                        kept = true;
                    }
                }
                const unsigned ball = __ballot_sync(0xffffffffu, kept);
                if (kept) {
                    const int slot = (q2head + q2count + __popc(ball & ((1u << lane) - 1u))) & (WQ - 1);
                    qidx2[slot] = i;
                    qmv2[slot] = pm;
                    if constexpr (kKeepSurvivors<SH>) {
                        // this lane's first-stage results, from its own tour-state columns
                        TourState<SH> ts;
                        ts.bind(tstate, tid);
                        Survivor<SH> &sv = surv[slot];
#pragma unroll
                        for (int g = 0; g < SH::MAXT; ++g)
                            if ((r1.amask >> g) & 1u) {
                                sv.lhu[g] = ts.LHU.get(g); sv.lsu[g] = ts.LSU.get(g); sv.db2[g] = ts.DB2.get(g);
                                sv.rq[g] = ts.Rq.get(g); sv.hm[g] = ts.Hm.get(g);
                            }
                        sv.amask = r1.amask;
                        sv.tmax = r1.tmax;
                    }
                }
                q2count += __popc(ball);
                __syncwarp();
                qhead = (qhead + take) & (WQ - 1);
                qcount -= take;
            }
            // the full score of a warp of candidates the gate kept, or the remainder at the end
            const int take2 = (q2count >= 32) ? 32 : ((drained && qcount == 0) ? q2count : 0);
            if (take2 > 0) {
                if (memo_wait) { named_sync(NT); memo_wait = false; }
                if (lane < take2) {
                    const int slot = (q2head + lane) & (WQ - 1);
                    const int i = qidx2[slot];
                    const int2 pm = qmv2[slot];
                    const MoveRec m = {pm.x & 0xffff, pm.x >> 16, pm.y & 0xffff, pm.y >> 16};
                    ScoreOut r;
                    ChainView cv;
                    if constexpr (CHAIN) draw_chain(c, prm, (uint32_t)i, iter, M.inst_idx, cv);
                    if constexpr (kKeepSurvivors<SH>)
                        r = score_candidate<SH, false, false, 2, CHAIN>(c, prm, m, tmax_star, tstate, tid, nullptr,
                                                                        nullptr, nullptr, nullptr, nullptr, nullptr,
                                                                        nullptr, nullptr, nullptr, &surv[slot], &cv);
                    else
                        r = score_candidate<SH, false, false, 0, CHAIN>(c, prm, m, tmax_star, tstate, tid, nullptr,
                                                                        nullptr, nullptr, nullptr, nullptr, nullptr,
                                                                        nullptr, nullptr, nullptr, nullptr, &cv);
                    const unsigned long long k = make_key(r.cost, (uint32_t)i);
                    if (k < best) { best = k; best_t = r.tmax; }
                    if (ins) ins[i - (int)prm.cand_offset] = make_float2(r.cost, r.tmax);
                }
                __syncwarp();
                q2head = (q2head + take2) & (WQ - 1);
                q2count -= take2;
            }
            if (drained && qcount == 0 && q2count == 0) {
                if (memo_wait) { named_sync(NT); memo_wait = false; }
                break;
            }
            base = next;
        }
        block_argmin_finalize<NT, CHAIN>(best, best_t, bs, M, wi, slot_key, slot_tmax, slot_base, c, prm, iter);
    }
}

// Steps 13-16 of an iteration whose candidates were scored in slices (bl_search_score_slice) and whose
// argmin key -- the minimum over the slices' keys, possibly of other processes -- is read from device
// memory. The winner's Tmax is recomputed by scoring candidate i* again on the same staged base; a key
// that does not score as this iteration's candidate i* sets error 2. One instance, one block.
template <class SH, bool CHAIN>
__global__ void __launch_bounds__(SH::NT) apply_key_kernel(const InstMeta *__restrict__ meta, SearchParams prm,
                                                           SmemPlan sp, const unsigned long long *__restrict__ d_key)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BlockShared bs;
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bs.mbar, 1);
        fence_mbar_init();
        bs.phase = 0;
    }
    __syncthreads();
    const InstMeta &M = meta[0];
    Ctx c;
    if (!stage_instance<SH>(M, bs, smem, sp, prm, -1, 0xffffffffu, c)) return;
    if (tid == 0) {
        const unsigned long long bk = *d_key;
        const float cst = __uint_as_float((uint32_t)(bk >> 32));
        float bt = 0.f;
        if (isfinite(cst)) {
            const uint32_t istar = (uint32_t)(bk & 0xffffffffu);
            MoveRec m = {4, 0, 0, 0};
            ChainView cv;
            bool feas;
            if constexpr (CHAIN) {
                draw_chain(c, prm, istar, bs.iter, M.inst_idx, cv);
                feas = demand_ok_chain(c, cv);
            } else {
                m = draw_move(c, prm, istar, bs.iter, M.inst_idx);
                feas = demand_ok(c, m);
            }
            ScoreOut r = {__int_as_float(0x7f800000), 0.f, 0u};
            if (feas)
                r = score_candidate<SH, false, false, 0, CHAIN>(c, prm, m, M.state->tmaxstar, smem + sp.off_tour, tid,
                                                                nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                                nullptr, nullptr, nullptr, nullptr, &cv);
            if (__float_as_uint(r.cost) != (uint32_t)(bk >> 32)) atomicExch(&M.state->error, 2u);
            bt = r.tmax;
        }
        apply_update<CHAIN>(c, prm, M, bs.use_best, bs.iter, bk, bt);
    }
}

// The search states of all instances to or from one packed buffer (one transfer each way for the
// host): per instance, at byte offset offs[k], x_old and x* (plan_len int16 each) and the state record.
// dir 0: device -> buffer, 1: buffer -> device (the state's work counter and error flag are cleared).
__global__ void state_pack_kernel(const InstMeta *__restrict__ meta, const int32_t *__restrict__ offs,
                                  unsigned char *__restrict__ buf, int32_t dir)
{
    const InstMeta &M = meta[blockIdx.x];
    int16_t *p = (int16_t *)(buf + offs[blockIdx.x]);
    InstState *st = (InstState *)(p + 2 * M.plan_len);
    for (int k = threadIdx.x; k < M.plan_len; k += blockDim.x) {
        if (dir == 0) { p[k] = M.xold[k]; p[M.plan_len + k] = M.xbest[k]; }
        else { M.xold[k] = p[k]; M.xbest[k] = p[M.plan_len + k]; }
    }
    if (threadIdx.x == 0) {
        if (dir == 0) *st = *M.state;
        else {
            InstState s = *st;
            s.done = 0;
            s.error = 0;
            *M.state = s;
        }
    }
}

cudaError_t launch_state_pack(const InstMeta *d_meta, int32_t n_inst, const int32_t *d_offs, unsigned char *d_buf,
                              int32_t dir, cudaStream_t s)
{
    state_pack_kernel<<<n_inst, 128, 0, s>>>(d_meta, d_offs, d_buf, dir);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Cooperative scoring: L lanes per candidate, lane g holds tour g
// ---------------------------------------------------------------------------
// The same arithmetic as score_candidate, value for value, so a cooperative
// search follows the same trajectory bit for bit. A group of L lanes (L >= the
// number of tours, a power of two dividing 32) scores one candidate:
//  - lane g keeps tour g's aggregates, unit sets and times in registers;
//  - every local-minimisation round finds g_max, g_max2 and g_min by shuffle
//    reductions (lowest tour index on ties, as the sequential scan), then tries
//    up to L members of g_min at once: the first accepted in the sequential
//    order (a ballot) is the one the sequential loop stops at;
//  - the shuttle pass runs over the field positions, L at a time; its sums are
//    exact integers, so their order does not matter;
//  - the float cost is summed over the tours in index order, like the
//    sequential sum.
__device__ __forceinline__ int select_bit32(uint32_t w, int n)   // position of the n-th (0-based) set bit
{
    int pos = 0;
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) {
        const uint32_t lo = w & ((1u << sh) - 1u);
        const int cnt = __popc(lo);
        if (n >= cnt) { n -= cnt; w >>= sh; pos += sh; }
        else w = lo;
    }
    return pos;
}
__device__ __forceinline__ int select_bit64(unsigned long long w, int n)
{
    const uint32_t lo = (uint32_t)w;
    const int cl = __popc(lo);
    return n < cl ? select_bit32(lo, n) : 32 + select_bit32((uint32_t)(w >> 32), n - cl);
}
template <typename Mk>
__device__ __forceinline__ int select_m(Mk w, int n)
{
    if constexpr (sizeof(Mk) == 4) return select_bit32((uint32_t)w, n);
    else return select_bit64((unsigned long long)w, n);
}
// clear the lowest `n` set bits of a one- or two-word set (at least n + 1 are set)
template <typename Mk>
__device__ __forceinline__ void drop_lowest(Mk &w0, unsigned long long &w1, int n)
{
    const int c0 = popc_m(w0);
    if (n >= c0) {
        w0 = 0;
        const int p = select_bit64(w1, n - c0 - 1 < 0 ? 0 : n - c0 - 1);
        if (n > c0) w1 &= (p == 63) ? 0ull : (~0ull << (p + 1));
    } else {
        const int p = select_m(w0, n - 1);
        constexpr int BITS = 8 * (int)sizeof(Mk);
        w0 &= (p == BITS - 1) ? (Mk)0 : (Mk)(~(Mk)0 << (p + 1));
    }
}

template <int L>
__device__ __forceinline__ unsigned grp_ballot(unsigned gm, bool pred)
{
    const unsigned b = __ballot_sync(gm, pred);
    const int base = (threadIdx.x & 31) & ~(L - 1);
    return L == 32 ? b : ((b >> base) & ((1u << L) - 1u));
}
// (value, index) reductions over the group; invalid lanes carry +-inf and a large index
template <int L>
__device__ __forceinline__ void grp_argmax(float &x, int &i, unsigned gm)
{
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) {
        const float ox = __shfl_xor_sync(gm, x, o, L);
        const int oi = __shfl_xor_sync(gm, i, o, L);
        if (ox > x || (ox == x && oi < i)) { x = ox; i = oi; }
    }
}
template <int L>
__device__ __forceinline__ void grp_argmin(float &x, int &i, unsigned gm)
{
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) {
        const float ox = __shfl_xor_sync(gm, x, o, L);
        const int oi = __shfl_xor_sync(gm, i, o, L);
        if (ox < x || (ox == x && oi < i)) { x = ox; i = oi; }
    }
}
template <int L>
__device__ __forceinline__ float grp_max(float x, unsigned gm)
{
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) {
        const float ox = __shfl_xor_sync(gm, x, o, L);
        if (ox > x) x = ox;
    }
    return x;
}
template <int L>
__device__ __forceinline__ long long grp_sum(long long v, unsigned gm)
{
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(gm, v, o, L);
    return v;
}
template <int L, typename V>
__device__ __forceinline__ V grp_bcast(V v, int src, unsigned gm) { return __shfl_sync(gm, v, src, L); }

constexpr int kNoTour = 1 << 20;

// g_max, g_max2 and g_min of one local-minimisation round (Algorithm 2)
template <int L>
__device__ __forceinline__ void grp_picks(float t, bool act, int g, int na, unsigned gm, int &gx, float &tx, int &gx2,
                                          float &tx2, int &gn, float &tn)
{
    tx = act ? t : -INFINITY;
    gx = act ? g : kNoTour;
    grp_argmax<L>(tx, gx, gm);
    const bool c2 = act && g != gx;
    tx2 = c2 ? t : -INFINITY;
    gx2 = c2 ? g : kNoTour;
    grp_argmax<L>(tx2, gx2, gm);
    if (na == 2) { gn = gx2; tn = tx2; return; }
    const bool c3 = c2 && g != gx2;
    tn = c3 ? t : INFINITY;
    gn = c3 ? g : kNoTour;
    grp_argmin<L>(tn, gn, gm);
}

template <class SH, int L, bool IDENT>
__device__ ScoreOut score_coop(const Ctx &c, const SearchParams &p, const MoveRec &m, float tmax_star, int lane,
                               unsigned gm, float *o_tc, float *o_kf, long long *o_sh)
{
    constexpr int SW = SH::SW;
    using M = typename SH::Mask;
    using S = typename SH::Sum;
    ScoreOut out;
    View x;
    x.set(c, m);
    const unsigned touched = x.touched(c);
    const int g = lane;   // this lane's tour
    const int nb = g < c.T ? x.tour_len(c, g) : 0;
    const bool act = nb > 0;
    const unsigned amask = grp_ballot<L>(gm, act);
    const int na = __popc(amask);
    const int j = __popc(amask & ((1u << g) - 1u));   // rank among the active tours

    // --- route aggregates (Fig. 1, Sec. 2.2)
    long long lhu = 0, lsu = 0, ar = 0;
    float db2 = 0.f;
    if (act) {
        if ((touched >> g) & 1u) {
            const TourAgg t = tour_agg(c, x, g, nb);
            lhu = t.LHU; lsu = t.LSU; ar = t.A; db2 = t.DB2;
        } else {
            lhu = c.tLHU[g]; lsu = c.tLSU[g]; ar = c.tA[g]; db2 = c.tDB2[g];
        }
    }
    const float LHU = __fmul_rn(__ll2float_rn(lhu), c.dq_scale);
    const float LSU = __fmul_rn(__ll2float_rn(lsu), c.dq_scale);
    const float A = __fmul_rn(__ll2float_rn(ar), c.aq_scale);
    const float DB2 = db2;
    const int di = (na - 1) * c.T;

    // --- HU assignment (Sec. 2.5): round-robin dealing, then Algorithm 2 on T_compl
    M Hm = 0;
    S Rq = 0;
    float tv = 0.f;
    if (act) {
        Hm = (M)c.hudeal_m[di + j];
        Rq = (S)c.hudeal_q[di + j];
        const float R = __fmul_rn(to_f(Rq), c.rqs);
        tv = __fmaf_rn(LHU, c.inv_v, __fdividef(A, R));
    }
    if (!p.fix_resources && na >= 2) {
        for (int round = 0; round < c.H; ++round) {
            int gx, gx2, gn;
            float tx, tx2, tn;
            grp_picks<L>(tv, act, g, na, gm, gx, tx, gx2, tx2, gn, tn);
            const M mn = grp_bcast<L>(Hm, gn, gm);
            if (popc_m(mn) <= 1) break;
            const int last = hibit_m(mn);
            const float Lx = grp_bcast<L>(LHU, gx, gm), Ax = grp_bcast<L>(A, gx, gm);
            const float Ln = grp_bcast<L>(LHU, gn, gm), An = grp_bcast<L>(A, gn, gm);
            const S rqx = grp_bcast<L>(Rq, gx, gm), rqn = grp_bcast<L>(Rq, gn, gm);
            M rem = mn;
            unsigned long long rem1 = 0ull;
            int k;
            float tmx, tmn;
            S nqx, nqn;
            while (true) {
                const int cnt = popc_m(rem);
                bool cond = false;
                int kk = 0;
                float a_tmx = 0.f, a_tmn = 0.f;
                S a_nqx = 0, a_nqn = 0;
                if (lane < cnt) {
                    kk = select_m(rem, lane);
                    a_nqx = rqx + (S)c.hurq[kk];
                    a_nqn = rqn - (S)c.hurq[kk];
                    a_tmx = __fmaf_rn(Lx, c.inv_v, __fdividef(Ax, __fmul_rn(to_f(a_nqx), c.rqs)));
                    a_tmn = __fmaf_rn(Ln, c.inv_v, __fdividef(An, __fmul_rn(to_f(a_nqn), c.rqs)));
                    const float ref = (na == 2) ? a_tmn : tx2;
                    cond = (a_tmx < ref) || (kk == last);
                }
                const unsigned bal = grp_ballot<L>(gm, cond);
                if (bal) {
                    const int w = __ffs(bal) - 1;
                    k = grp_bcast<L>(kk, w, gm);
                    tmx = grp_bcast<L>(a_tmx, w, gm);
                    tmn = grp_bcast<L>(a_tmn, w, gm);
                    nqx = grp_bcast<L>(a_nqx, w, gm);
                    nqn = grp_bcast<L>(a_nqn, w, gm);
                    break;
                }
                drop_lowest(rem, rem1, L);   // none of these L accepted (the last member always is)
            }
            float nm = (tmx > tmn) ? tmx : tmn;
            const float other = grp_max<L>((act && g != gx && g != gn) ? tv : -INFINITY, gm);
            if (other > nm) nm = other;
            if (!(nm < tx)) break;   // the accepted move does not lower the maximum: keep the old state
            const M bit = (M)1 << k;
            if (g == gx) { Hm |= bit; Rq = nqx; tv = tmx; }
            if (g == gn) { Hm &= ~bit; Rq = nqn; tv = tmn; }
        }
    }
    const float tmax = grp_max<L>(act ? tv : -INFINITY, gm);
    if (IDENT && act) o_tc[g] = tv;
    // the gate depends on Tmax alone: a discarded candidate's cost is +inf (Sec. 2.5)
    if (!IDENT && ((p.gate == 1 && tmax > tmax_star) || (p.gate == 2 && tmax >= tmax_star))) {
        out.cost = __int_as_float(0x7f800000);
        out.tmax = tmax;
        return out;
    }

    // --- SU assignment (Algorithm 2, Eq. 6); R(g) is fixed now
    M S0 = 0;
    unsigned long long S1 = 0ull;
    S Saq = 0;
    float iR = 0.f, tw = 0.f;
    int star = 0;
    if (act) {
        S0 = (M)c.sudeal_m[(di + j) * 2];
        if (SW > 1) S1 = c.sudeal_m[(di + j) * 2 + 1];
        Saq = (S)c.sudeal_q[di + j];
        iR = __fdividef(1.0f, __fmul_rn(to_f(Rq), c.rqs));
        star = su_star<SH>(c, S0, S1);
        const float fill = __fmul_rn(to_f((S)(Saq - (S)c.sufq[star])), c.fqs);
        tw = __fmaf_rn(-fill, iR, __fmul_rn(DB2, c.suinv[star]));
    }
    if (!p.fix_resources && na >= 2) {
        for (int round = 0; round < c.S; ++round) {
            int gx, gx2, gn;
            float tx, tx2, tn;
            grp_picks<L>(tw, act, g, na, gm, gx, tx, gx2, tx2, gn, tn);
            const M n0 = grp_bcast<L>(S0, gn, gm);
            const unsigned long long n1 = (SW > 1) ? grp_bcast<L>(S1, gn, gm) : 0ull;
            if (popc_m(n0) + (SW > 1 ? popc_m(n1) : 0) <= 1) break;
            const int last = (SW > 1 && n1) ? 64 + hibit_m(n1) : hibit_m(n0);
            const int star_x = grp_bcast<L>(star, gx, gm), grp_x = c.sugrp[star_x];
            const int star_n = grp_bcast<L>(star, gn, gm);
            const S sqx = grp_bcast<L>(Saq, gx, gm), sqn = grp_bcast<L>(Saq, gn, gm);
            const float DBx = grp_bcast<L>(DB2, gx, gm), DBn = grp_bcast<L>(DB2, gn, gm);
            const float iRx = grp_bcast<L>(iR, gx, gm), iRn = grp_bcast<L>(iR, gn, gm);
            M r0 = n0;
            unsigned long long r1 = n1;
            int k, sx, sn;
            float tmx, tmn;
            while (true) {
                const int c0 = popc_m(r0);
                const int cnt = c0 + (SW > 1 ? popc_m(r1) : 0);
                bool cond = false;
                int kk = 0, a_sx = 0, a_sn = 0;
                float a_tmx = 0.f, a_tmn = 0.f;
                if (lane < cnt) {
                    kk = lane < c0 ? select_m(r0, lane) : 64 + select_bit64(r1, lane - c0);
                    const float ak = c.sufill[kk];
                    const int gk = c.sugrp[kk];
                    if (gk > grp_x || (gk == grp_x && kk < star_x)) {
                        a_sx = kk;
                        a_tmx = __fmaf_rn(-__fmul_rn(to_f(sqx), c.fqs), iRx, __fmul_rn(DBx, c.suinv[kk]));
                    } else {
                        a_sx = star_x;
                        a_tmx = __fmaf_rn(-ak, iRx, tx);
                    }
                    if (kk != star_n) {
                        a_sn = star_n;
                        a_tmn = __fmaf_rn(ak, iRn, tn);
                    } else {
                        M b0 = n0;
                        unsigned long long b1 = n1;
                        if (kk < 64) b0 &= ~((M)1 << kk); else b1 &= ~(1ull << (kk - 64));
                        a_sn = su_star<SH>(c, b0, b1);
                        a_tmn = __fmaf_rn(-__fmul_rn(to_f((S)(sqn - (S)c.sufq[kk] - (S)c.sufq[a_sn])), c.fqs), iRn,
                                          __fmul_rn(DBn, c.suinv[a_sn]));
                    }
                    const float ref = (na == 2) ? a_tmn : tx2;
                    cond = (a_tmx < ref) || (kk == last);
                }
                const unsigned bal = grp_ballot<L>(gm, cond);
                if (bal) {
                    const int w = __ffs(bal) - 1;
                    k = grp_bcast<L>(kk, w, gm);
                    sx = grp_bcast<L>(a_sx, w, gm);
                    sn = grp_bcast<L>(a_sn, w, gm);
                    tmx = grp_bcast<L>(a_tmx, w, gm);
                    tmn = grp_bcast<L>(a_tmn, w, gm);
                    break;
                }
                drop_lowest(r0, r1, L);
            }
            float nm = (tmx > tmn) ? tmx : tmn;
            const float other = grp_max<L>((act && g != gx && g != gn) ? tw : -INFINITY, gm);
            if (other > nm) nm = other;
            if (!(nm < tx)) break;
            if (g == gx) {
                if (k < 64) S0 |= (M)1 << k; else S1 |= 1ull << (k - 64);
                Saq = (S)(sqx + (S)c.sufq[k]);
                star = sx;
                tw = tmx;
            }
            if (g == gn) {
                if (k < 64) S0 &= ~((M)1 << k); else S1 &= ~(1ull << (k - 64));
                Saq = (S)(sqn - (S)c.sufq[k]);
                star = sn;
                tw = tmn;
            }
        }
    }

    // --- path-length cost (Sec. 2.2, Eq. 4): exact shuttle sums in fixed point
    int nsu = 0;
    float kf = 0.f;
    double capd = 0.0;
    if (act) {
        nsu = popc_m(S0) + (SW > 1 ? popc_m(S1) : 0);
        const long long cs = cap_sum<SH>(c, S0, S1);
        kf = __fdividef((float)nsu, __fmul_rn(__ll2float_rn(cs), c.cqs));
        capd = (double)cs * c.cqs_d;
        if (IDENT) o_kf[g] = kf;
    }
    unsigned moved = 0u;   // tours whose field -> BP content changed
    if (x.kind == 0 && x.sg != x.dg) moved = (1u << c.bp_tour[x.sg]) | (1u << c.bp_tour[x.dg]);
    else if (x.kind == 1 && x.sg != x.dg) moved = (1u << x.sg) | (1u << x.dg);
    else if (x.kind == 2 && c.field_bp[x.v] != c.field_bp[x.w])
        moved = (1u << c.bp_tour[c.field_bp[x.v]]) | (1u << c.bp_tour[c.field_bp[x.w]]);
    else if (x.kind == 3 && c.bp_tour[x.v] != c.bp_tour[x.w]) moved = (1u << c.bp_tour[x.v]) | (1u << c.bp_tour[x.w]);
    const bool fr = act && (!c.memo || ((moved >> g) & 1u) || kf != c.kf_base[g]);
    const unsigned fresh = grp_ballot<L>(gm, fr);
    long long acc = (act && !fr) ? c.sh_base[g] : 0ll;
    if (IDENT && act) o_sh[g] = 0;
    if (IDENT) __syncwarp(gm);
    // Eq. 4 for a field of tour t: FP32 fast path, the exact test near an integer
    auto ceil_fast = [&](float sup, float kft, bool &amb) -> int {
        const float q = __fmul_rn(sup, kft);
        const float rq = rintf(q);
        amb = !(fabsf(q - rq) > q * (1.0f / 2097152.0f));
        return (int)ceilf(q);
    };
    if (fresh) {
        for (int k0 = 0; k0 < c.F; k0 += L) {
            const int kk = k0 + lane;
            int t = -1;
            float sup = 0.f;
            int dq = 0;
            if (kk < c.F) {
                const int f = c.field_order[kk];
                const int b = c.field_bp[f];   // base BP of this position
                if (x.bp_of_field(c, f) == b) {   // moved fields are added below
                    const int tb = x.tour_of_bp(c, b);
                    if ((fresh >> tb) & 1u) { const int2 sd = c.psd[kk]; t = tb; sup = __int_as_float(sd.x); dq = sd.y; }
                }
            }
            const int src = t < 0 ? 0 : t;
            const float kft = grp_bcast<L>(kf, src, gm);
            bool amb = false;
            int n = 0;
            if (t >= 0) n = ceil_fast(sup, kft, amb);
            if (grp_ballot<L>(gm, amb)) {   // rare: the tour's exact capacity sum decides
                const int nst = grp_bcast<L>(nsu, src, gm);
                const double cdt = grp_bcast<L>(capd, src, gm);
                if (amb) n = exact_ceil(sup, nst, cdt, __fmul_rn(sup, kft));
            }
            if (t >= 0) {
                const long long a = (long long)n * (long long)dq;
                acc += a;
                if (IDENT) atomicAdd((unsigned long long *)&o_sh[t], (unsigned long long)a);
            }
        }
        int mv_f0 = -1, mv_f1 = -1;
        if (x.kind == 0 && x.sg != x.dg) mv_f0 = x.v;
        if (x.kind == 2 && c.field_bp[x.v] != c.field_bp[x.w]) { mv_f0 = x.v; mv_f1 = x.w; }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int f = q == 0 ? mv_f0 : mv_f1;
            if (f >= 0) {   // uniform over the group
                const int b = x.bp_of_field(c, f);
                const int t = x.tour_of_bp(c, b);
                const float kft = grp_bcast<L>(kf, t, gm);
                const int nst = grp_bcast<L>(nsu, t, gm);
                const double cdt = grp_bcast<L>(capd, t, gm);
                bool amb;
                int n = ceil_fast(c.supply[f], kft, amb);
                if (amb) n = exact_ceil(c.supply[f], nst, cdt, __fmul_rn(c.supply[f], kft));
                if (lane == 0) {
                    const long long a = (long long)n * c.dq(1 + c.B + f, 1 + b);
                    acc += a;
                    if (IDENT) atomicAdd((unsigned long long *)&o_sh[t], (unsigned long long)a);
                }
            }
        }
    }
    const long long shq = grp_sum<L>(acc, gm);
    // cost: tours in index order, as the sequential sum
    const float route = act ? __fadd_rn(__fmul_rn((float)popc_m(Hm), LHU), __fmul_rn((float)nsu, LSU)) : 0.f;
    float cost = 0.f;
    for (int t = 0; t < c.T; ++t) {
        const float r = grp_bcast<L>(route, t, gm);
        if ((amask >> t) & 1u) cost = __fadd_rn(cost, r);
    }
    cost = __fadd_rn(cost, __fmul_rn(__fmul_rn(__ll2float_rn(shq), c.dq_scale), 2.0f));
    // --- completion-time gate (Sec. 2.5)
    if ((p.gate == 1 && tmax > tmax_star) || (p.gate == 2 && tmax >= tmax_star)) cost = __int_as_float(0x7f800000);
    out.cost = cost;
    out.tmax = tmax;
    return out;
}

constexpr int COOP_NT = 256;   // threads per block of the cooperative kernel

// stage_base, then the base plan's own per-tour report scored by the first group
template <class SH, int L>
__device__ bool stage_coop(const InstMeta &M, BlockShared &bs, unsigned char *smem, const SmemPlan &sp,
                           const SearchParams &p, Ctx &c)
{
    if (!stage_base<SH>(M, bs, smem, sp, p, -1, 0xffffffffu, c)) return false;
    const int tid = threadIdx.x;
    if (tid < L) {
        const unsigned gm = L == 32 ? 0xffffffffu : ((1u << L) - 1u);
        float *kf_base = const_cast<float *>(c.kf_base);
        long long *sh_base = const_cast<long long *>(c.sh_base);
        c.nbad = bs.nbad;
        if (tid < M.T) { kf_base[tid] = 0.f; sh_base[tid] = 0; }
        if (tid < 16) bs.base_tc[tid] = 0.f;
        __syncwarp(gm);
        float cost = __int_as_float(0x7f800000);
        if (bs.nbad == 0) {
            const MoveRec idm = {4, 0, 0, 0};
            cost = score_coop<SH, L, true>(c, p, idm, __int_as_float(0x7f800000), tid, gm, bs.base_tc, kf_base,
                                           sh_base)
                       .cost;
        }
        if (tid == 0) bs.base_cost = cost;
    }
    __syncthreads();
    c.nbad = bs.nbad;
    c.memo = 1;
    return true;
}

// One iteration of Algorithm 1 with L lanes per candidate: the work
// decomposition, list mode, argmin slots and Steps 13-16 of the one-thread
// kernel; each group of L lanes draws and scores candidates of the tile in turn.
template <class SH, int L>
__global__ void __launch_bounds__(COOP_NT) search_iteration_coop_kernel(
    const InstMeta *__restrict__ meta, const WorkItem *__restrict__ work, int32_t n_work, SearchParams prm, SmemPlan sp,
    unsigned long long *__restrict__ slot_key, float *__restrict__ slot_tmax, const int32_t *__restrict__ slot_base,
    const uint32_t *__restrict__ cand_list, const int32_t *__restrict__ cand_count, int32_t list_stride,
    float2 *__restrict__ insp, int32_t insp_stride)
{
    static_assert(L >= SH::MAXT && L <= 32 && (32 % L) == 0, "one lane per tour, groups inside a warp");
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BlockShared bs;
    const int tid = threadIdx.x;
    const int gl = tid & (L - 1), grp = tid / L;
    constexpr int NG = COOP_NT / L;
    const unsigned gm = L == 32 ? 0xffffffffu : (((1u << L) - 1u) << ((tid & 31) & ~(L - 1)));
    if (tid == 0) {
        mbar_init(&bs.mbar, 1);
        fence_mbar_init();
        bs.phase = 0;
        bs.staged = -1;
    }
    __syncthreads();
    Ctx c;
    for (int w = blockIdx.x; w < n_work; w += gridDim.x) {
        const WorkItem wi = work[w];
        const InstMeta &M = meta[wi.inst];
        if (bs.staged != wi.inst) {
            if (!stage_coop<SH, L>(M, bs, smem, sp, prm, c)) return;
            if (tid == 0) bs.staged = wi.inst;
            __syncthreads();
        }
        const float tmax_star = M.state->tmaxstar;
        const uint32_t iter = bs.iter;
        const int list_n = cand_list ? cand_count[wi.inst] : 0;
        const uint32_t *ilist = cand_list ? cand_list + (size_t)wi.inst * list_stride : nullptr;
        const int tl = cand_list ? list_tile(M, list_n, n_work) : M.tile;
        // positions [c0, c1) of the instance's candidates (or of its list); empty past the end
        const long long cend = cand_list ? min(M.n_cand, list_n) : M.n_cand;
        const long long c0l = (long long)wi.tile_idx * tl;
        const int c0 = (int)min(c0l, cend);
        const int c1 = (int)min(c0l + tl, cend);
        float2 *const ins = insp ? insp + (size_t)wi.inst * insp_stride : nullptr;
        unsigned long long best = ~0ull;
        float best_t = 0.f;
        for (int pos = c0 + grp; pos < c1; pos += NG) {
            const int i = ilist ? (int)ilist[pos] : (int)prm.cand_offset + pos;
            const MoveRec m = draw_move(c, prm, (uint32_t)i, iter, M.inst_idx);
            unsigned long long k;
            float t = __int_as_float(0x7f800000);
            if (demand_ok(c, m)) {
                const ScoreOut r = score_coop<SH, L, false>(c, prm, m, tmax_star, gl, gm, nullptr, nullptr, nullptr);
                k = make_key(r.cost, (uint32_t)i);
                t = r.tmax;
            } else {
                k = make_key(__int_as_float(0x7f800000), (uint32_t)i);
            }
            if (k < best) { best = k; best_t = t; }
            if (ins && gl == 0) ins[i - (int)prm.cand_offset] = make_float2(__uint_as_float((uint32_t)(k >> 32)), t);
        }
        block_argmin_finalize<COOP_NT>(best, best_t, bs, M, wi, slot_key, slot_tmax, slot_base, c, prm, iter);
    }
}

// ---------------------------------------------------------------------------
// Inspection kernels
// ---------------------------------------------------------------------------
template <class SH, bool CHAIN>
__global__ void __launch_bounds__(SH::NT) score_dump_kernel(const InstMeta *__restrict__ meta, int32_t inst,
                                                            int32_t use_best, uint32_t iter, float tmax_star,
                                                            int32_t i0, int32_t n, int32_t identity, SearchParams prm,
                                                            SmemPlan sp, float *cost, float *tmax, int16_t *moves,
                                                            int16_t *nhu, int16_t *nsu, float *tcompl, float *twait,
                                                            float *tcost, int16_t *hu_tour, int16_t *su_tour)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BlockShared bs;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) {
        mbar_init(&bs.mbar, 1);
        fence_mbar_init();
        bs.phase = 0;
    }
    __syncthreads();
    const InstMeta &M = meta[inst];
    Ctx c;
    if (!stage_instance<SH>(M, bs, smem, sp, prm, use_best, iter, c)) return;
    unsigned char *tstate = smem + sp.off_tour;
    const int T = M.T;
    for (int k = blockIdx.x * nt + tid; k < n; k += gridDim.x * nt) {
        const int i = i0 + k;
        MoveRec m = {4, 0, 0, 0};
        ChainView cv;
        if constexpr (CHAIN) {
            if (identity) cv.n = 0;   // the base plan itself: a chain of no moves
            else draw_chain(c, prm, (uint32_t)i, bs.iter, M.inst_idx, cv);
            // one record per move: {kind, vertex, BP / tour / partner, slot (0 for swaps)}
            if (moves)
                for (int l = 0; l < cv.n; ++l) {
                    const Lvl &e = cv.L[l];
                    int16_t *mv = moves + (size_t)k * 4 * prm.k_moves + 4 * l;
                    mv[0] = (int16_t)e.kind; mv[1] = (int16_t)e.v;
                    mv[2] = (int16_t)(e.kind < 2 ? e.d : e.w); mv[3] = (int16_t)(e.kind < 2 ? e.dp : 0);
                }
        } else {
            if (!identity) m = draw_move(c, prm, (uint32_t)i, bs.iter, M.inst_idx);
            if (moves) {
                moves[k * 4] = (int16_t)m.kind; moves[k * 4 + 1] = (int16_t)m.v;
                moves[k * 4 + 2] = (int16_t)m.a; moves[k * 4 + 3] = (int16_t)m.b;
            }
        }
        int16_t *o_nhu = nhu ? nhu + (size_t)k * T : nullptr;
        int16_t *o_nsu = nsu ? nsu + (size_t)k * T : nullptr;
        float *o_tc = tcompl ? tcompl + (size_t)k * T : nullptr;
        float *o_tw = twait ? twait + (size_t)k * T : nullptr;
        float *o_tk = tcost ? tcost + (size_t)k * T : nullptr;
        int16_t *o_hu = hu_tour ? hu_tour + (size_t)k * M.H : nullptr;
        int16_t *o_su = su_tour ? su_tour + (size_t)k * M.S : nullptr;
        for (int g = 0; g < T; ++g) {
            if (o_nhu) o_nhu[g] = 0;
            if (o_nsu) o_nsu[g] = 0;
            if (o_tc) o_tc[g] = 0.f;
            if (o_tw) o_tw[g] = 0.f;
            if (o_tk) o_tk[g] = 0.f;
        }
        if (o_hu) for (int h = 0; h < M.H; ++h) o_hu[h] = -1;
        if (o_su) for (int s = 0; s < M.S; ++s) o_su[s] = -1;
        ScoreOut r;
        bool feas;
        if constexpr (CHAIN) feas = demand_ok_chain(c, cv);
        else feas = demand_ok(c, m);
        if (feas)
            r = score_candidate<SH, true, false, 0, CHAIN>(c, prm, m, tmax_star, tstate, tid, o_nhu, o_nsu, o_tc, o_tw,
                                                           o_tk, o_hu, o_su, nullptr, nullptr, nullptr, &cv);
        else { r.cost = __int_as_float(0x7f800000); r.tmax = __int_as_float(0x7f800000); }
        if (cost) cost[k] = r.cost;
        if (tmax) tmax[k] = r.tmax;
    }
}

template <class SH, bool CHAIN>
__global__ void __launch_bounds__(SH::NT) decode_kernel(const InstMeta *__restrict__ meta, int32_t inst,
                                                        int32_t use_best, uint32_t iter, const int32_t *idx, int32_t n,
                                                        SearchParams prm, SmemPlan sp, int16_t *plans)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BlockShared bs;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) {
        mbar_init(&bs.mbar, 1);
        fence_mbar_init();
        bs.phase = 0;
    }
    __syncthreads();
    const InstMeta &M = meta[inst];
    Ctx c;
    if (!stage_instance<SH>(M, bs, smem, sp, prm, use_best, iter, c)) return;
    const int rowlen = 2 * M.B + M.T + M.F;
    for (int k = blockIdx.x * nt + tid; k < n; k += gridDim.x * nt) {
        if constexpr (CHAIN) {
            ChainView cv;
            draw_chain(c, prm, (uint32_t)idx[k], bs.iter, M.inst_idx, cv);
            write_plan_chain(c, cv, plans + (size_t)k * rowlen);
        } else {
            const MoveRec m = draw_move(c, prm, (uint32_t)idx[k], bs.iter, M.inst_idx);
            write_plan(c, m, plans + (size_t)k * rowlen);
        }
    }
}

// ---------------------------------------------------------------------------
// Features of candidate moves for the learned ranking (an extension: the
// paper draws moves uniformly). One row of NFEAT BF16 values per candidate,
// normalised per instance (distances by the mean field-to-BP distance, times
// by Tmax*, supplies and areas by their means).
// ---------------------------------------------------------------------------
template <class SH>
__global__ void __launch_bounds__(SH::NT) features_kernel(const InstMeta *__restrict__ meta, int32_t inst,
                                                          int32_t use_best, uint32_t iter, int32_t i0, int32_t n,
                                                          SearchParams prm, SmemPlan sp, __nv_bfloat16 *__restrict__ feat,
                                                          float *__restrict__ base_cost, int32_t batched)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BlockShared bs;
    const int tid = threadIdx.x, nt = blockDim.x;
    // batched: grid row y serves instance y, whose n rows start at row y * n
    if (batched) {
        inst = (int32_t)blockIdx.y;
        feat += (size_t)inst * n * NFEAT;
        if (base_cost) base_cost += inst;
    }
    if (tid == 0) {
        mbar_init(&bs.mbar, 1);
        fence_mbar_init();
        bs.phase = 0;
    }
    __syncthreads();
    const InstMeta &M = meta[inst];
    Ctx c;
    // the base plan's per-tour T_compl (and its cost, only when the caller asks for it: the
    // completion times need the HU assignment alone, the cost the whole score)
    if (!stage_base<SH>(M, bs, smem, sp, prm, use_best, iter, c)) return;
    if (tid == 0) {
        if (base_cost) {
            score_base<SH>(M, bs, smem, sp, prm, c);
        } else {
            c.nbad = bs.nbad;
            for (int g = 0; g < 16; ++g) bs.base_tc[g] = 0.f;
            if (bs.nbad == 0) {
                const MoveRec idm = {4, 0, 0, 0};
                score_candidate<SH, false, true, 1>(c, prm, idm, __int_as_float(0x7f800000), smem + sp.off_tour, tid,
                                                    nullptr, nullptr, bs.base_tc, nullptr, nullptr, nullptr, nullptr);
            }
        }
    }
    __syncthreads();
    c.nbad = bs.nbad;
    if (blockIdx.x == 0 && tid == 0 && base_cost) *base_cost = bs.base_cost;
    const uint32_t it = bs.iter;   // resolved from the state when the caller passed 0xffffffff
    const float tstar = M.state->tmaxstar;
    const float inv_t = (tstar > 0.f && isfinite(tstar)) ? 1.f / tstar : 0.f;
    const float L = c.dq_scale * M.inv_l0;   // fixed-point distance -> normalised distance
    auto dn = [&](int a, int b) -> float { return (float)c.dq(a, b) * L; };
    auto xy_of = [&](int node, float *out) {   // node position relative to the HQ, from distances to two references
        out[0] = dn(0, node);
        out[1] = dn(1, node);   // distance to BP 0 as the second coordinate
    };
    for (int k = blockIdx.x * nt + tid; k < n; k += gridDim.x * nt) {
        const int i = i0 + k;
        const MoveRec m = draw_move(c, prm, (uint32_t)i, it, M.inst_idx);
        float f[NFEAT];
#pragma unroll
        for (int j = 0; j < NFEAT; ++j) f[j] = 0.f;
        f[0] = m.kind == 0; f[1] = m.kind == 1; f[2] = m.kind >= 2;
        View x;
        x.set(c, m);
        int tgs = -1, tgd = -1;   // source and destination tour of a reinsert
        long long aqm = 0;        // area it moves (fixed point)
        if (m.kind == 0) {
            const int v = m.v, vn = 1 + c.B + v, bsrc = x.sg, bdst = x.dg, ps = x.sp, pd = x.dp;
            const int gs = c.bp_tour[bsrc], gd = c.bp_tour[bdst];
            tgs = gs; tgd = gd; aqm = c.areaq[v];
            const int st = c.bp_start[bsrc], cnt = c.bp_cnt[bsrc];
            // neighbours of v in its tour's field sequence (HQ at the ends)
            int p = 0, q = 0;
            if (ps > 0) p = 1 + c.B + c.field_order[st + ps - 1];
            else if (c.bp_pos[bsrc] > 0) p = c.blast[c.bp_order[c.tour_start[gs] + c.bp_pos[bsrc] - 1]];
            if (ps < cnt - 1) q = 1 + c.B + c.field_order[st + ps + 1];
            else if (c.bp_pos[bsrc] < c.tour_cnt[gs] - 1) q = c.bfirst[c.bp_order[c.tour_start[gs] + c.bp_pos[bsrc] + 1]];
            if (p < 0) p = 0;
            if (q < 0) q = 0;
            // neighbours at the insertion slot (destination list after the removal)
            const int dst = c.bp_start[bdst];
            const int len = c.bp_cnt[bdst] - (bdst == bsrc ? 1 : 0);
            const bool same = (bdst == bsrc);
            int a = (c.bp_pos[bdst] > 0) ? c.blast[c.bp_order[c.tour_start[gd] + c.bp_pos[bdst] - 1]] : 0;
            int cc = (c.bp_pos[bdst] < c.tour_cnt[gd] - 1) ? c.bfirst[c.bp_order[c.tour_start[gd] + c.bp_pos[bdst] + 1]] : 0;
            if (pd > 0) { const int j = pd - 1; a = 1 + c.B + c.field_order[dst + (same && j >= ps ? j + 1 : j)]; }
            if (pd < len) { const int j = pd; cc = 1 + c.B + c.field_order[dst + (same && j >= ps ? j + 1 : j)]; }
            if (a < 0) a = 0;
            if (cc < 0) cc = 0;
            f[3] = dn(p, vn); f[4] = dn(vn, q); f[5] = dn(p, q);
            f[6] = dn(a, vn); f[7] = dn(vn, cc); f[8] = dn(a, cc);
            f[9] = f[5] - f[3] - f[4];
            f[10] = f[6] + f[7] - f[8];
            f[11] = dn(vn, 1 + bsrc); f[12] = dn(vn, 1 + bdst); f[13] = f[12] - f[11];
            f[14] = c.supply[v] * M.inv_mean_supply;
            f[15] = c.area[v] * M.inv_mean_area;
            // Eq. 2 slack of both BPs after the move, relative to the demand: numerators exact in
            // fixed point, the ratio in FP32 (FP64 division is slow on this GPU and the features
            // are rounded to BF16)
            const long long mv = same ? 0ll : c.supq[v];
            f[16] = __ll2float_rn(c.base_supq[bsrc] - mv - c.demq[bsrc]) / __ll2float_rn(c.demq[bsrc]);
            f[17] = __ll2float_rn(c.base_supq[bdst] + mv - c.demq[bdst]) / __ll2float_rn(c.demq[bdst]);
            f[18] = same; f[19] = (gs == gd);
            f[20] = gs < 16 ? (tstar - bs.base_tc[gs]) * inv_t : 0.f;
            f[21] = gd < 16 ? (tstar - bs.base_tc[gd]) * inv_t : 0.f;
            f[22] = (float)ps / (float)cnt;
            f[23] = (float)pd / (float)(len + 1);
            xy_of(vn, f + 24); xy_of(1 + bsrc, f + 26); xy_of(1 + bdst, f + 28);
            f[30] = (float)cnt / M.mean_fields_per_bp;
            f[31] = (float)(len + 1) / M.mean_fields_per_bp;
            f[32] = f[9] + f[10];
        } else if (m.kind == 1) {
            const int b = m.v, gs = x.sg, gd = x.dg, qs = x.sp, qd = x.dp;
            tgs = gs; tgd = gd; aqm = c.barea[b];
            const int f1 = c.bfirst[b] >= 0 ? c.bfirst[b] : 0, fl = c.blast[b] >= 0 ? c.blast[b] : 0;
            int p = 0, q = 0;
            if (qs > 0) { const int t = c.blast[c.bp_order[c.tour_start[gs] + qs - 1]]; p = t >= 0 ? t : 0; }
            if (qs < c.tour_cnt[gs] - 1) { const int t = c.bfirst[c.bp_order[c.tour_start[gs] + qs + 1]]; q = t >= 0 ? t : 0; }
            // insertion slot in the destination tour after the removal
            const int lenT = c.tour_cnt[gd] - (gd == gs ? 1 : 0);
            auto bp_after = [&](int j) { return c.bp_order[c.tour_start[gd] + ((gd == gs && j >= qs) ? j + 1 : j)]; };
            int a = 0, cc = 0;
            if (qd > 0) { const int t = c.blast[bp_after(qd - 1)]; a = t >= 0 ? t : 0; }
            if (qd < lenT) { const int t = c.bfirst[bp_after(qd)]; cc = t >= 0 ? t : 0; }
            f[3] = dn(p, f1); f[4] = dn(fl, q); f[5] = dn(p, q);
            f[6] = dn(a, f1); f[7] = dn(fl, cc); f[8] = dn(a, cc);
            f[9] = f[5] - f[3] - f[4];
            f[10] = f[6] + f[7] - f[8];
            f[14] = __ll2float_rn(c.base_supq[b]) / __ll2float_rn(c.demq[b]);
            f[15] = __ll2float_rn(c.barea[b]) * c.aq_scale * M.inv_mean_area / fmaxf(M.mean_fields_per_bp, 1.f);
            f[19] = (gs == gd);
            f[20] = gs < 16 ? (tstar - bs.base_tc[gs]) * inv_t : 0.f;
            f[21] = gd < 16 ? (tstar - bs.base_tc[gd]) * inv_t : 0.f;
            f[22] = (float)qs / (float)c.tour_cnt[gs];
            f[23] = (float)qd / (float)(lenT + 1);
            xy_of(1 + b, f + 26);
            f[30] = (float)c.bp_cnt[b] / M.mean_fields_per_bp;
            f[32] = f[9] + f[10];
        } else {
            const int v = m.v, w = m.a;
            const int vn = (m.kind == 2) ? 1 + c.B + v : 1 + v, wn = (m.kind == 2) ? 1 + c.B + w : 1 + w;
            f[3] = dn(vn, wn);
            xy_of(vn, f + 24); xy_of(wn, f + 26);
        }
        f[33] = demand_ok(c, m);   // Eq. 2, exact
        if (tgs >= 0) {
            // completion-time gate signals: share of each tour's area the move
            // shifts, base completion times scaled by it, criticality, and the
            // HU-route change relative to each tour's route
            float tcmax = 0.f;
            for (int g = 0; g < c.T; ++g) tcmax = fmaxf(tcmax, bs.base_tc[g]);
            const bool other = (tgs != tgd);
            const float fa = __ll2float_rn(aqm);
            const float ad = other && c.tA[tgd] > 0 ? fa / __ll2float_rn(c.tA[tgd]) : 0.f;
            const float as = other && c.tA[tgs] > 0 ? fa / __ll2float_rn(c.tA[tgs]) : 0.f;
            f[34] = fminf(ad, 4.f);
            f[35] = as;
            f[36] = bs.base_tc[tgd] * inv_t * (1.f + f[34]) - 1.f;
            f[37] = bs.base_tc[tgs] * inv_t * (1.f - f[35]) - 1.f;
            f[38] = bs.base_tc[tgs] >= tcmax;
            f[39] = bs.base_tc[tgd] >= tcmax;
            const float rl = 1.f / L;
            f[40] = c.tLHU[tgd] > 0 ? fminf(f[10] * rl / (float)c.tLHU[tgd], 4.f) : 0.f;
            f[41] = c.tLHU[tgs] > 0 ? fmaxf(f[9] * rl / (float)c.tLHU[tgs], -4.f) : 0.f;
            f[42] = tcmax * inv_t - 1.f;
        }
#pragma unroll
        for (int j = 0; j < NFEAT; ++j) f[j] = isfinite(f[j]) ? fminf(fmaxf(f[j], -64.f), 64.f) : 0.f;
        // the row (128 bytes, 16-byte aligned) in eight 16-byte stores
        uint4 *row = reinterpret_cast<uint4 *>(feat + (size_t)k * NFEAT);
#pragma unroll
        for (int j = 0; j < NFEAT; j += 8) {
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const __nv_bfloat162 pr = __floats2bfloat162_rn(f[j + 2 * q], f[j + 2 * q + 1]);
                w[q] = *reinterpret_cast<const uint32_t *>(&pr);
            }
            row[j / 8] = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// Selection of the moves to score exactly: the n_keep best predicted
// (threshold from a sorted sample of 4096 predictions) plus a uniform random
// fraction of the rest as fallback.
__global__ void select_threshold_kernel(const float *__restrict__ y, int32_t P, int32_t n_keep, float *__restrict__ thresh)
{
    // The value at rank r of the 4096-prediction sample, found by radix selection on an
    // order-preserving 32-bit key (8 bits per pass, from the top): the same value a sort of
    // the sample would put at position r.
    constexpr int S = 4096;
    __shared__ unsigned int hist[256];
    __shared__ unsigned int sel_prefix, sel_rank;
    y += (size_t)blockIdx.x * P;   // block b: instance b of a batch
    thresh += blockIdx.x;
    constexpr int PER = S / 1024;   // keys per thread (blockDim.x = 1024)
    unsigned int key[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int j = threadIdx.x + q * 1024;
        const long long idx = (long long)j * P / S;
        float v = y[idx];
        if (!isfinite(v)) v = __int_as_float(0x7f800000);
        const unsigned int b = __float_as_uint(v);
        key[q] = (b & 0x80000000u) ? ~b : (b | 0x80000000u);   // float order -> unsigned order
    }
    if (threadIdx.x == 0) {
        long long r = (long long)n_keep * S / P;
        if (r >= S) r = S - 1;
        if (r < 0) r = 0;
        sel_prefix = 0u;
        sel_rank = (unsigned int)r;
    }
    unsigned int mask = 0u;
    for (int shift = 24; shift >= 0; shift -= 8) {
        if (threadIdx.x < 256) hist[threadIdx.x] = 0u;
        __syncthreads();
        const unsigned int prefix = sel_prefix;
#pragma unroll
        for (int q = 0; q < PER; ++q)
            if ((key[q] & mask) == prefix) atomicAdd(&hist[(key[q] >> shift) & 255u], 1u);
        __syncthreads();
        if (threadIdx.x < 32) {
            // lane l owns digits 8l .. 8l + 7: find the digit whose cumulative count passes the rank
            const int lane = threadIdx.x;
            unsigned int c[8], tot = 0u;
#pragma unroll
            for (int d = 0; d < 8; ++d) { c[d] = hist[8 * lane + d]; tot += c[d]; }
            unsigned int incl = tot;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const unsigned int excl = incl - tot, r = sel_rank;
            if (r >= excl && r < incl) {   // exactly one lane
                unsigned int below = excl;
                int d = 0;
                while (below + c[d] <= r) { below += c[d]; ++d; }
                sel_prefix = prefix | ((unsigned int)(8 * lane + d) << shift);
                sel_rank = r - below;
            }
        }
        mask |= 255u << shift;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const unsigned int k = sel_prefix;
        *thresh = __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
    }
}

__global__ void __launch_bounds__(256) select_compact_kernel(const float *__restrict__ y, int32_t P,
                                                            const float *__restrict__ thresh, float rand_frac,
                                                            uint32_t salt, uint32_t *__restrict__ list,
                                                            int32_t *__restrict__ count)
{
    // grid row b: instance b of a batch (its own predictions, threshold, list and count).
    // Each warp gathers its kept indices in shared memory and appends them with one atomic
    // per 224+ entries (the list's order is free: the argmin over it is order-independent).
    __shared__ uint32_t wbuf[8][256];
    const uint32_t b = blockIdx.y;
    y += (size_t)b * P;
    list += (size_t)b * P;
    thresh += b;
    count += b;
    const float th = *thresh;
    const uint32_t cut = (uint32_t)(rand_frac * 4294967295.0f);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *buf = wbuf[warp];
    int n = 0;   // warp-uniform: entries in buf
    auto flush = [&]() {
        int off = 0;
        if (lane == 0) off = atomicAdd(count, n);
        off = __shfl_sync(0xffffffffu, off, 0);
        for (int k = lane; k < n; k += 32) list[off + k] = buf[k];
        __syncwarp();
        n = 0;
    };
    const int stride = gridDim.x * blockDim.x;
    for (int base = blockIdx.x * blockDim.x + warp * 32; base < P; base += stride) {
        const int i = base + lane;
        bool keep = false;
        if (i < P) {
            keep = y[i] <= th;
            if (!keep) {
                uint32_t r[4] = {(uint32_t)i, salt, 0x5E1EC7u + b, 2u};
                philox10(r, 0x243F6A88u, 0x85A308D3u);
                keep = r[0] < cut;
            }
        }
        const unsigned ball = __ballot_sync(0xffffffffu, keep);
        if (keep) buf[n + __popc(ball & ((1u << lane) - 1u))] = (uint32_t)i;
        n += __popc(ball);
        __syncwarp();
        if (n > 256 - 32) flush();
    }
    if (n > 0) flush();
}

// ---------------------------------------------------------------------------
// Argmin without allocation
// ---------------------------------------------------------------------------
// Scores candidates i0..i0+n-1 of one iteration and reduces them to the
// argmin key, like the search iteration kernel, but its scratch (one partial
// result per block and a completion counter) lives in this file-scope device
// array instead of memory someone allocated. Every call on a device shares
// the array and finds the previous call's contents in it: the counter is
// cleared before each launch, and calls that overlap on the GPU race.
constexpr int kNoAllocMaxBlocks = 1024;   // partial results: 1024 x 16 B, plus the counter
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocMaxBlocks * 16 + 256];

template <class SH>
__global__ void __launch_bounds__(SH::NT) argmin_noalloc_kernel(const InstMeta *__restrict__ meta, int32_t inst,
                                                                int32_t use_best, uint32_t iter, float tmax_star,
                                                                int32_t i0, int32_t n, SearchParams prm, SmemPlan sp,
                                                                unsigned char *scratch,
                                                                unsigned long long *__restrict__ out_key,
                                                                float *__restrict__ out_tmax)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BlockShared bs;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int NT = SH::NT;
    unsigned int *counter = (unsigned int *)scratch;
    unsigned long long *part_key = (unsigned long long *)(scratch + 256);
    float *part_tmax = (float *)(scratch + 256 + kNoAllocMaxBlocks * 8);
    if (tid == 0) {
        mbar_init(&bs.mbar, 1);
        fence_mbar_init();
        bs.phase = 0;
    }
    __syncthreads();
    const InstMeta &M = meta[inst];
    Ctx c;
    // A block whose staging wait gave up (error flag set) scores nothing but still
    // reports an empty partial result, so the last block always writes the outputs:
    // after a timeout *out_key is ~0 (no candidate) and *out_tmax NaN.
    const bool staged = stage_instance<SH>(M, bs, smem, sp, prm, use_best, iter, c);
    unsigned char *tstate = smem + sp.off_tour;
    int32_t *qidx = (int32_t *)(smem + sp.off_qidx) + warp * WQ;
    int2 *qmv = (int2 *)(smem + sp.off_qmv) + warp * WQ;
    unsigned long long best = ~0ull;
    float best_t = staged ? 0.f : __int_as_float(0x7fc00000);
    int qhead = 0, qcount = 0;
    // 64-bit positions: i0 + n may lie within one grid stride of INT32_MAX
    const long long stride = (long long)NT * gridDim.x;
    const long long c1 = staged ? (long long)i0 + n : (long long)i0;
    for (long long base = (long long)i0 + (long long)blockIdx.x * NT + warp * 32; base < c1 || qcount > 0;
         base += stride) {
        if (base < c1) {
            const int i = (int)(base + lane);   // < c1 <= INT32_MAX when i < c1
            bool feas = false;
            MoveRec m = {4, 0, 0, 0};
            if (base + lane < c1) {
                m = draw_move(c, prm, (uint32_t)i, bs.iter, M.inst_idx);
                feas = demand_ok(c, m);
                if (!feas) {
                    const unsigned long long k = make_key(__int_as_float(0x7f800000), (uint32_t)i);
                    if (k < best) { best = k; best_t = __int_as_float(0x7f800000); }
                }
            }
            const unsigned ball = __ballot_sync(0xffffffffu, feas);
            if (feas) {
                const int slot = (qhead + qcount + __popc(ball & ((1u << lane) - 1u))) & (WQ - 1);
                qidx[slot] = i;
                qmv[slot] = make_int2((m.kind & 0xffff) | (m.v << 16), (m.a & 0xffff) | (m.b << 16));
            }
            qcount += __popc(ball);
            __syncwarp();
        }
        const int take = (qcount >= 32) ? 32 : ((base + stride >= c1) ? qcount : 0);
        if (take > 0) {
            if (lane < take) {
                const int slot = (qhead + lane) & (WQ - 1);
                const int i = qidx[slot];
                const int2 pm = qmv[slot];
                const MoveRec m = {pm.x & 0xffff, pm.x >> 16, pm.y & 0xffff, pm.y >> 16};
                const ScoreOut r = score_candidate<SH, false>(c, prm, m, tmax_star, tstate, tid, nullptr, nullptr,
                                                              nullptr, nullptr, nullptr, nullptr, nullptr);
                const unsigned long long k = make_key(r.cost, (uint32_t)i);
                if (k < best) { best = k; best_t = r.tmax; }
            }
            __syncwarp();
            qhead = (qhead + take) & (WQ - 1);
            qcount -= take;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(0xffffffffu, best, o);
        const float ot = __shfl_xor_sync(0xffffffffu, best_t, o);
        if (ok < best) { best = ok; best_t = ot; }
    }
    if (lane == 0) { bs.red[warp] = best; bs.redt[warp] = best_t; }
    __syncthreads();
    if (tid < 32) {
        best = (tid < (NT >> 5)) ? bs.red[tid] : ~0ull;
        best_t = (tid < (NT >> 5)) ? bs.redt[tid] : 0.f;
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ok = __shfl_xor_sync(0xffffffffu, best, o);
            const float ot = __shfl_xor_sync(0xffffffffu, best_t, o);
            if (ok < best) { best = ok; best_t = ot; }
        }
        if (tid == 0) {
            part_key[blockIdx.x] = best;
            part_tmax[blockIdx.x] = best_t;
            __threadfence();
            bs.last = (atomicAdd(counter, 1u) == gridDim.x - 1) ? 1 : 0;
        }
    }
    __syncthreads();
    if (bs.last && tid < 32) {
        __threadfence();
        unsigned long long bk = ~0ull;
        float bt = 0.f;
        for (int b = tid; b < (int)gridDim.x; b += 32) {
            const unsigned long long k = __ldcg(&part_key[b]);
            const float t = __ldcg(&part_tmax[b]);
            if (k < bk) { bk = k; bt = t; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
            const float ot = __shfl_xor_sync(0xffffffffu, bt, o);
            if (ok < bk) { bk = ok; bt = ot; }
        }
        if (tid == 0) {
            *out_key = bk;
            *out_tmax = bt;
            *counter = 0u;
        }
    }
}

// ---------------------------------------------------------------------------
// Host-side launch wrappers
// ---------------------------------------------------------------------------
int max_tours_of(int32_t shape)
{
    return shape == SHAPE_T4_S64_DSMEM ? 4 : shape == SHAPE_T6_S64_GMEM ? 6 : shape == SHAPE_T10_S128_GMEM ? 10 : 16;
}
int threads_of(int32_t shape)
{
    return shape == SHAPE_T4_S64_DSMEM ? ShapeA::NT
           : shape == SHAPE_T6_S64_GMEM ? ShapeB::NT
           : shape == SHAPE_T10_S128_GMEM ? ShapeD::NT : ShapeC::NT;
}
int max_su_of(int32_t shape)
{
    return (shape == SHAPE_T16_S128_GMEM || shape == SHAPE_T10_S128_GMEM) ? 128 : (shape == SHAPE_T4_S64_DSMEM ? 32 : 64);
}
bool dist_in_smem(int32_t shape) { return shape == SHAPE_T4_S64_DSMEM; }

static SmemPlan plan_for(const LaunchCfg &cfg)
{
    switch (cfg.shape) {
    case SHAPE_T4_S64_DSMEM:
        return carve_shape<ShapeA>(cfg.max_prefix, cfg.max_plan_len, cfg.max_F, cfg.max_B, cfg.max_T);
    case SHAPE_T6_S64_GMEM:
        return carve_shape<ShapeB>(cfg.max_prefix, cfg.max_plan_len, cfg.max_F, cfg.max_B, cfg.max_T);
    case SHAPE_T10_S128_GMEM:
        return carve_shape<ShapeD>(cfg.max_prefix, cfg.max_plan_len, cfg.max_F, cfg.max_B, cfg.max_T);
    default:
        return carve_shape<ShapeC>(cfg.max_prefix, cfg.max_plan_len, cfg.max_F, cfg.max_B, cfg.max_T);
    }
}

// the cooperative kernel keeps tour state in registers and needs no queues
static SmemPlan coop_plan_for(const LaunchCfg &cfg)
{
    return carve(0, 0, cfg.max_prefix, cfg.max_plan_len, cfg.max_F, cfg.max_B, cfg.max_T);
}

size_t coop_shared_bytes(const LaunchCfg &cfg) { return coop_plan_for(cfg).total; }

// Calls f with the cooperative kernel instance for (shape, lanes), or returns
// cudaErrorInvalidValue if that pair is not built.
template <class F>
static cudaError_t with_coop_kernel(int32_t shape, int32_t lanes, F &&f)
{
    switch (shape) {
    case SHAPE_T4_S64_DSMEM:
        if (lanes == 4) return f(search_iteration_coop_kernel<ShapeA, 4>);
        if (lanes == 8) return f(search_iteration_coop_kernel<ShapeA, 8>);
        break;
    case SHAPE_T6_S64_GMEM:
        if (lanes == 8) return f(search_iteration_coop_kernel<ShapeB, 8>);
        if (lanes == 16) return f(search_iteration_coop_kernel<ShapeB, 16>);
        break;
    case SHAPE_T10_S128_GMEM:
        if (lanes == 16) return f(search_iteration_coop_kernel<ShapeD, 16>);
        if (lanes == 32) return f(search_iteration_coop_kernel<ShapeD, 32>);
        break;
    default:
        if (lanes == 16) return f(search_iteration_coop_kernel<ShapeC, 16>);
        if (lanes == 32) return f(search_iteration_coop_kernel<ShapeC, 32>);
    }
    return cudaErrorInvalidValue;
}

bool coop_supported(int32_t shape, int32_t lanes)
{
    switch (shape) {
    case SHAPE_T4_S64_DSMEM: return lanes == 4 || lanes == 8;
    case SHAPE_T6_S64_GMEM: return lanes == 8 || lanes == 16;
    default: return lanes == 16 || lanes == 32;
    }
}

cudaError_t configure_coop(int32_t shape, int32_t lanes, size_t smem)
{
    return with_coop_kernel(shape, lanes, [&](auto kern) {
        return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
}

int coop_blocks_per_sm(int32_t shape, int32_t lanes, size_t smem)
{
    int n = 0;
    const cudaError_t e = with_coop_kernel(shape, lanes, [&](auto kern) {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, COOP_NT, smem);
    });
    return e == cudaSuccess ? n : 0;
}

size_t shared_bytes(int32_t shape, int32_t threads, int32_t max_prefix, int32_t max_plan_len, int32_t max_F,
                    int32_t max_B, int32_t max_T)
{
    LaunchCfg cfg{};
    cfg.shape = shape; cfg.threads = threads; cfg.max_prefix = max_prefix; cfg.max_plan_len = max_plan_len;
    cfg.max_F = max_F; cfg.max_B = max_B; cfg.max_T = max_T;
    return plan_for(cfg).total;
}

// f(Shape{}, std::integral_constant<bool, chain>{}) for the shape class `shape`
template <class F>
static cudaError_t with_shape(int32_t shape, bool chain, F &&f)
{
    using T = std::true_type;
    using N = std::false_type;
    switch (shape) {
    case SHAPE_T4_S64_DSMEM: return chain ? f(ShapeA{}, T{}) : f(ShapeA{}, N{});
    case SHAPE_T6_S64_GMEM: return chain ? f(ShapeB{}, T{}) : f(ShapeB{}, N{});
    case SHAPE_T10_S128_GMEM: return chain ? f(ShapeD{}, T{}) : f(ShapeD{}, N{});
    default: return chain ? f(ShapeC{}, T{}) : f(ShapeC{}, N{});
    }
}

template <class SH, bool CHAIN>
static cudaError_t set_attrs_of(size_t smem)
{
    cudaError_t e = cudaFuncSetAttribute(search_iteration_kernel<SH, CHAIN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(score_dump_kernel<SH, CHAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(apply_key_kernel<SH, CHAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(decode_kernel<SH, CHAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <class SH>
static cudaError_t set_attrs(size_t smem)
{
    const cudaError_t e = set_attrs_of<SH, false>(smem);
    if (e != cudaSuccess) return e;
    return set_attrs_of<SH, true>(smem);
}

cudaError_t configure_kernels(int32_t shape, size_t smem)
{
    switch (shape) {
    case SHAPE_T4_S64_DSMEM: return set_attrs<ShapeA>(smem);
    case SHAPE_T6_S64_GMEM: return set_attrs<ShapeB>(smem);
    case SHAPE_T10_S128_GMEM:
        return set_attrs<ShapeD>(smem);
    default: return set_attrs<ShapeC>(smem);
    }
}

// Resident blocks per SM of the search kernel with this much dynamic shared
// memory (registers and shared memory both counted); 0 on error.
int search_blocks_per_sm(int32_t shape, size_t smem)
{
    int n = 0;
    cudaError_t e;
    switch (shape) {
    case SHAPE_T4_S64_DSMEM:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, search_iteration_kernel<ShapeA, false>, ShapeA::NT, smem);
        break;
    case SHAPE_T6_S64_GMEM:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, search_iteration_kernel<ShapeB, false>, ShapeB::NT, smem);
        break;
    case SHAPE_T10_S128_GMEM:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, search_iteration_kernel<ShapeD, false>, ShapeD::NT, smem);
        break;
    default:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, search_iteration_kernel<ShapeC, false>, ShapeC::NT, smem);
    }
    return e == cudaSuccess ? n : 0;
}

cudaError_t launch_search_iteration(const LaunchCfg &cfg, const InstMeta *d_meta, const WorkItem *d_work,
                                    int32_t n_work, SearchParams prm, unsigned long long *slot_key, float *slot_tmax,
                                    const int32_t *slot_base, cudaStream_t s, const uint32_t *cand_list,
                                    const int32_t *cand_count, int32_t list_stride, float2 *insp, int32_t insp_stride)
{
    if (cfg.lanes > 1) {
        const SmemPlan cp = coop_plan_for(cfg);
        const cudaError_t e = with_coop_kernel(cfg.shape, cfg.lanes, [&](auto kern) {
            kern<<<cfg.grid, COOP_NT, cp.total, s>>>(d_meta, d_work, n_work, prm, cp, slot_key, slot_tmax, slot_base,
                                                     cand_list, cand_count, list_stride, insp, insp_stride);
            return cudaSuccess;
        });
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    }
    const SmemPlan sp = plan_for(cfg);
    const cudaError_t e = with_shape(cfg.shape, prm.k_moves > 1, [&](auto sh, auto ch) {
        using SH = decltype(sh);
        search_iteration_kernel<SH, decltype(ch)::value><<<cfg.grid, SH::NT, sp.total, s>>>(
            d_meta, d_work, n_work, prm, sp, slot_key, slot_tmax, slot_base, cand_list, cand_count, list_stride, insp,
            insp_stride);
        return cudaSuccess;
    });
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_apply_key(const LaunchCfg &cfg, const InstMeta *d_meta, SearchParams prm,
                             const unsigned long long *d_key, cudaStream_t s)
{
    const SmemPlan sp = plan_for(cfg);
    const cudaError_t e = with_shape(cfg.shape, prm.k_moves > 1, [&](auto sh, auto ch) {
        using SH = decltype(sh);
        apply_key_kernel<SH, decltype(ch)::value><<<1, SH::NT, sp.total, s>>>(d_meta, prm, sp, d_key);
        return cudaSuccess;
    });
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// Device address of the no-allocation scratch array on the current device (the
// name is only a host-side stand-in: passing it to a kernel would hand the GPU a
// host address). The caller looks it up once per handle, with the handle's
// device current, and keeps it: a handle does not outlive its device's context.
cudaError_t noalloc_scratch_address(void **ptr)
{
    return cudaGetSymbolAddress(ptr, g_noalloc_scratch);
}

cudaError_t launch_argmin_noalloc(const LaunchCfg &cfg, const InstMeta *d_meta, int32_t inst, int32_t use_best,
                                  uint32_t iter, float tmax_star, int32_t i0, int32_t n, SearchParams prm,
                                  void *scratch, unsigned long long *d_key, float *d_tmax, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    // the counter must start at zero; the partial results are written before they are read
    e = cudaMemsetAsync(scratch, 0, 256, s);
    if (e != cudaSuccess) return e;
    const SmemPlan sp = plan_for(cfg);
    const int nt = threads_of(cfg.shape);
    int grid = (n + nt - 1) / nt;
    if (grid > cfg.grid) grid = cfg.grid;
    if (grid > kNoAllocMaxBlocks) grid = kNoAllocMaxBlocks;
    if (grid < 1) grid = 1;
    unsigned char *sc = (unsigned char *)scratch;
#define NA_ARGS d_meta, inst, use_best, iter, tmax_star, i0, n, prm, sp, sc, d_key, d_tmax
    switch (cfg.shape) {
    case SHAPE_T4_S64_DSMEM:
        e = cudaFuncSetAttribute(argmin_noalloc_kernel<ShapeA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sp.total);
        if (e == cudaSuccess) argmin_noalloc_kernel<ShapeA><<<grid, nt, sp.total, s>>>(NA_ARGS);
        break;
    case SHAPE_T6_S64_GMEM:
        e = cudaFuncSetAttribute(argmin_noalloc_kernel<ShapeB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sp.total);
        if (e == cudaSuccess) argmin_noalloc_kernel<ShapeB><<<grid, nt, sp.total, s>>>(NA_ARGS);
        break;
    case SHAPE_T10_S128_GMEM:
        e = cudaFuncSetAttribute(argmin_noalloc_kernel<ShapeD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sp.total);
        if (e == cudaSuccess) argmin_noalloc_kernel<ShapeD><<<grid, nt, sp.total, s>>>(NA_ARGS);
        break;
    default:
        e = cudaFuncSetAttribute(argmin_noalloc_kernel<ShapeC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sp.total);
        if (e == cudaSuccess) argmin_noalloc_kernel<ShapeC><<<grid, nt, sp.total, s>>>(NA_ARGS);
    }
#undef NA_ARGS
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_features(const LaunchCfg &cfg, const InstMeta *d_meta, int32_t inst, int32_t use_best,
                            uint32_t iter, int32_t i0, int32_t n, SearchParams prm, uint16_t *d_feat,
                            float *d_base_cost, cudaStream_t s, int32_t n_batch)
{
    const SmemPlan sp = plan_for(cfg);
    const int nt = threads_of(cfg.shape);
    const int batched = n_batch > 0 ? 1 : 0;
    const int gy = batched ? n_batch : 1;
    int grid = (n + nt - 1) / nt;
    const int cap = std::max(1, cfg.grid / gy);   // about one resident wave over all instances
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    __nv_bfloat16 *f = reinterpret_cast<__nv_bfloat16 *>(d_feat);
    cudaError_t e;
    switch (cfg.shape) {
    case SHAPE_T4_S64_DSMEM:
        e = cudaFuncSetAttribute(features_kernel<ShapeA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sp.total);
        if (e == cudaSuccess)
            features_kernel<ShapeA><<<dim3(grid, gy), nt, sp.total, s>>>(d_meta, inst, use_best, iter, i0, n, prm, sp, f, d_base_cost, batched);
        break;
    case SHAPE_T6_S64_GMEM:
        e = cudaFuncSetAttribute(features_kernel<ShapeB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sp.total);
        if (e == cudaSuccess)
            features_kernel<ShapeB><<<dim3(grid, gy), nt, sp.total, s>>>(d_meta, inst, use_best, iter, i0, n, prm, sp, f, d_base_cost, batched);
        break;
    case SHAPE_T10_S128_GMEM:
        e = cudaFuncSetAttribute(features_kernel<ShapeD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sp.total);
        if (e == cudaSuccess)
            features_kernel<ShapeD><<<dim3(grid, gy), nt, sp.total, s>>>(d_meta, inst, use_best, iter, i0, n, prm, sp, f, d_base_cost, batched);
        break;
    default:
        e = cudaFuncSetAttribute(features_kernel<ShapeC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sp.total);
        if (e == cudaSuccess)
            features_kernel<ShapeC><<<dim3(grid, gy), nt, sp.total, s>>>(d_meta, inst, use_best, iter, i0, n, prm, sp, f, d_base_cost, batched);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_select(const float *d_y, int32_t P, int32_t n_keep, float rand_frac, uint32_t salt,
                          uint32_t *d_list, int32_t *d_count, float *d_thresh, int32_t n_batch, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(d_count, 0, sizeof(int32_t) * (size_t)n_batch, s);
    if (e != cudaSuccess) return e;
    select_threshold_kernel<<<n_batch, 1024, 0, s>>>(d_y, P, n_keep, d_thresh);
    const int gx = std::max(1, std::min(592, (P + 255) / 256));
    select_compact_kernel<<<dim3(gx, n_batch), 256, 0, s>>>(d_y, P, d_thresh, rand_frac, salt, d_list, d_count);
    return cudaGetLastError();
}

cudaError_t launch_score_dump(const LaunchCfg &cfg, const InstMeta *d_meta, int32_t inst, int32_t use_best,
                              uint32_t iter, float tmax_star, int32_t i0, int32_t n, int32_t identity,
                              SearchParams prm, float *d_cost, float *d_tmax, int16_t *d_moves, int16_t *d_nhu,
                              int16_t *d_nsu, float *d_tcompl, float *d_twait, float *d_tcost, int16_t *d_hu_tour,
                              int16_t *d_su_tour, cudaStream_t s)
{
    const SmemPlan sp = plan_for(cfg);
    const int nt = threads_of(cfg.shape);
    int grid = (n + nt - 1) / nt;
    if (grid > cfg.grid) grid = cfg.grid;
    if (grid < 1) grid = 1;
    const cudaError_t e = with_shape(cfg.shape, prm.k_moves > 1, [&](auto sh, auto ch) {
        using SH = decltype(sh);
        score_dump_kernel<SH, decltype(ch)::value><<<grid, nt, sp.total, s>>>(
            d_meta, inst, use_best, iter, tmax_star, i0, n, identity, prm, sp, d_cost, d_tmax, d_moves, d_nhu, d_nsu,
            d_tcompl, d_twait, d_tcost, d_hu_tour, d_su_tour);
        return cudaSuccess;
    });
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_decode(const LaunchCfg &cfg, const InstMeta *d_meta, int32_t inst, int32_t use_best,
                          uint32_t iter, const int32_t *d_idx, int32_t n, SearchParams prm, int16_t *d_plans,
                          cudaStream_t s)
{
    const SmemPlan sp = plan_for(cfg);
    const int nt = threads_of(cfg.shape);
    int grid = (n + nt - 1) / nt;
    if (grid > cfg.grid) grid = cfg.grid;
    if (grid < 1) grid = 1;
    const cudaError_t e = with_shape(cfg.shape, prm.k_moves > 1, [&](auto sh, auto ch) {
        decode_kernel<decltype(sh), decltype(ch)::value><<<grid, nt, sp.total, s>>>(d_meta, inst, use_best, iter,
                                                                                   d_idx, n, prm, sp, d_plans);
        return cudaSuccess;
    });
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace biolog

namespace biolog {
cudaError_t launch_wait_selftest(uint64_t limit_ns, unsigned long long *d_out, cudaStream_t s)
{
    wait_selftest_kernel<<<1, 1, 0, s>>>(limit_ns, d_out);
    return cudaGetLastError();
}
}  // namespace biolog
