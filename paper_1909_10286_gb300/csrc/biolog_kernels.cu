// Kernels of the candidate search (Plessen, arXiv 1909.10286, Algorithm 1).
//
// One launch = one iteration of Steps 6-16 for every instance of the handle:
//   * each block stages an instance's tables (distances, supplies, fleet
//     tables) into shared memory with one bulk asynchronous copy completed on
//     an mbarrier, and loads the base plan chosen by the eps rule (Eq. 5);
//   * for each candidate index i of its work item a thread draws the Step 8
//     move from Philox4x32-10 with counter (i, iter, inst, 0), checks the
//     Eq. 2 demands exactly in 64-bit fixed point and, if they hold, queues it;
//   * queued candidates are scored one per thread: route aggregates traced as
//     in Fig. 1, HU assignment and SU assignment by the local minimisation of
//     Sec. 2.5 (Eq. 6, Algorithm 2), the path-length cost of Sec. 2.2 with the
//     exact Eq. 4 ceiling, and the completion-time gate;
//   * a warp-shuffle + block argmin over keys (cost bits << 32 | i) gives one
//     slot per work item; the block that finishes an instance's last work
//     item reduces the slots, replays move i* on the base and updates x_old,
//     x*, C*, Tmax* (Steps 13-16).
// Per-tour state of a candidate lives in shared memory, one column per thread.
// Every per-tour value is a deterministic function of that tour's content
// (sequential sums in tour order, fixed-point unit sums, explicitly rounded FP
// operations), so identical tours give bit-identical times in every candidate.
#include <cstdint>
#include <cuda_runtime.h>

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

// bounded wait: gives up after ~1 s of wall time
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > 1000000000ull) return false;
    }
}

// ---------------------------------------------------------------------------
// Shapes
// ---------------------------------------------------------------------------
template <int MAXT_, int SW_, bool DSM_, int NT_>
struct Shape {
    static constexpr int MAXT = MAXT_;   // tours
    static constexpr int SW = SW_;       // 64-bit words of an SU set
    static constexpr bool DSM = DSM_;    // distances in shared memory
    static constexpr int NT = NT_;       // threads per block (compile time: per-tour state offsets are immediates)
};

using ShapeA = Shape<4, 1, true, 256>;
using ShapeB = Shape<8, 1, true, 128>;
using ShapeC = Shape<16, 2, false, 128>;

constexpr int NFLT = 7;   // per-tour floats: LHU, LSU, A, DB2 (2 Dbar), Tc, Tw, Rf
constexpr int F_LHU = 0, F_LSU = 1, F_A = 2, F_DB2 = 3, F_TC = 4, F_TW = 5, F_RF = 6;
constexpr int NI64 = 2;   // per-tour int64: HU rate sum, SU fill sum (fixed point)
constexpr int Q_RQ = 0, Q_SAQ = 1;
constexpr int QUEUE_PER_THREAD = 2;

// Instance tables and base plan as seen by one block.
struct Ctx {
    int F, B, T, H, S, N;
    const float *D;
    const float *area, *supply;
    const long long *supq, *demq, *hurq, *sufq, *sucq;
    const float *suspd;
    const int *sugrp;
    const unsigned long long *hudeal_m, *sudeal_m;
    const long long *hudeal_q, *sudeal_q;
    const int *hu_id, *su_id;
    float inv_v, rqs, fqs, cqs;
    double cqs_d;
    // base plan and derived tables (shared memory)
    const int16_t *bp_order, *tour_cnt, *field_order, *bp_cnt;
    const int16_t *tour_start, *bp_start, *field_bp, *field_pos, *bp_tour, *bp_pos;
    const long long *base_supq;
    const int8_t *bad;
    int nbad;
    __device__ __forceinline__ float d(int i, int j) const { return D[i * N + j]; }
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
};

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

// smallest k with k * cap >= s * nsu, exactly, near an integer hint (FP64 on a
// rare path; a - p is exact by Sterbenz since p is within 1e-6 of a)
__device__ __noinline__ int exact_ceil(float s, int nsu, double cap, float q)
{
    const double a = (double)s * (double)nsu;
    const double k = rint((double)q);
    const double p = k * cap;
    const double e = fma(k, cap, -p);
    const double dlt = a - p;
    return (dlt > e) ? (int)k + 1 : (int)k;
}

__device__ __forceinline__ int popc_su(const unsigned long long *w, int SW)
{
    int n = __popcll(w[0]);
    if (SW > 1) n += __popcll(w[1]);
    return n;
}

// Per-candidate scoring. Tour state: tf[(field*MAXT+g)*nt + tid], etc.
struct ScoreOut {
    float cost, tmax;
};

template <class SH, bool DUMP>
__device__ ScoreOut score_candidate(const Ctx &c, const SearchParams &p, const MoveRec &m, float tmax_star,
                                    float *tf, long long *tq, unsigned long long *tm, int nt, int tid,
                                    int16_t *o_nhu, int16_t *o_nsu, float *o_tc, float *o_tw, float *o_tcost,
                                    int16_t *o_hu, int16_t *o_su)
{
    constexpr int MAXT = SH::MAXT, SW = SH::SW, NT = SH::NT;
    (void)nt;
    tf += tid; tq += tid; tm += tid;
#define TF(fld, g) tf[((fld) * MAXT + (g)) * NT]
#define TQ(fld, g) tq[((fld) * MAXT + (g)) * NT]
#define TM(fld, g) tm[((fld) * MAXT + (g)) * NT]
#define FOR_ACTIVE(g) _Pragma("unroll") for (int g = 0; g < MAXT; ++g) if ((amask >> g) & 1u)
    ScoreOut out;
    out.cost = __int_as_float(0x7f800000);
    out.tmax = __int_as_float(0x7f800000);
    View x;
    x.set(c, m);

    // --- route aggregates (Fig. 1, Sec. 2.2)
    unsigned amask = 0;
    int na = 0;
    for (int g = 0; g < c.T; ++g) {
        const int nb = x.tour_len(c, g);
        if (nb == 0) continue;
        amask |= 1u << g;
        ++na;
        int prevF = 0, anchor = 0;
        float LHU = 0.f, LSU = 0.f, A = 0.f, Dsum = 0.f;
        for (int j = 0; j < nb; ++j) {
            const int b = x.bp_at(c, g, j);
            const int nf = x.bp_len(c, b);
            const int bn = 1 + b;
            float Sb = 0.f;
            for (int k = 0; k < nf; ++k) {
                const int f = x.field_at(c, b, k);
                const int fn = 1 + c.B + f;
                LHU = __fadd_rn(LHU, c.d(prevF, fn));
                if (k == 0) LSU = __fadd_rn(LSU, c.d(anchor, fn));
                A = __fadd_rn(A, c.area[f]);
                Sb = __fadd_rn(Sb, c.d(fn, bn));
                prevF = fn;
            }
            Dsum = __fadd_rn(Dsum, __fdiv_rn(Sb, (float)nf));
            anchor = bn;
        }
        LHU = __fadd_rn(LHU, c.d(prevF, 0));
        LSU = __fadd_rn(LSU, c.d(anchor, 0));
        TF(F_LHU, g) = LHU;
        TF(F_LSU, g) = LSU;
        TF(F_A, g) = A;
        TF(F_DB2, g) = __fmul_rn(2.0f, __fdiv_rn(Dsum, (float)nb));
    }

    // --- HU assignment (Sec. 2.5): round-robin dealing, then Algorithm 2 on T_compl
    const int di = (na - 1) * c.T;
    const int g_first = __ffs(amask) - 1;
    {
    int j = 0;
    FOR_ACTIVE(g) {
        TM(0, g) = c.hudeal_m[di + j];
        const long long rq = c.hudeal_q[di + j];
        TQ(Q_RQ, g) = rq;
        const float R = __fmul_rn(__ll2float_rn(rq), c.rqs);
        TF(F_RF, g) = R;
        TF(F_TC, g) = __fmaf_rn(TF(F_LHU, g), c.inv_v, __fdiv_rn(TF(F_A, g), R));
        ++j;
    }
    }
    if (!p.fix_resources && na >= 2) {
        for (int round = 0; round < c.H; ++round) {
            int gx = g_first, gx2 = -1, gn = -1;
            FOR_ACTIVE(g) if (TF(F_TC, g) > TF(F_TC, gx)) gx = g;
            FOR_ACTIVE(g) if (g != gx && (gx2 < 0 || TF(F_TC, g) > TF(F_TC, gx2))) gx2 = g;
            if (na == 2) gn = gx2;
            else
                FOR_ACTIVE(g) if (g != gx && g != gx2 && (gn < 0 || TF(F_TC, g) < TF(F_TC, gn))) gn = g;
            const unsigned long long mn = TM(0, gn);
            if (__popcll(mn) <= 1) break;
            const float old_max = TF(F_TC, gx);
            const int last = 63 - __clzll((long long)mn);
            const float ref2 = TF(F_TC, gx2);
            const float Lx = TF(F_LHU, gx), Ax = TF(F_A, gx), Ln = TF(F_LHU, gn), An = TF(F_A, gn);
            const long long rqx = TQ(Q_RQ, gx), rqn = TQ(Q_RQ, gn);
            unsigned long long mm = mn;
            int k = -1;
            float tmx = 0.f, tmn = 0.f, Rx = 0.f, Rn = 0.f;
            long long nqx = 0, nqn = 0;
            while (mm) {
                k = __ffsll((long long)mm) - 1;
                mm &= mm - 1;
                nqx = rqx + c.hurq[k];
                nqn = rqn - c.hurq[k];
                Rx = __fmul_rn(__ll2float_rn(nqx), c.rqs);
                Rn = __fmul_rn(__ll2float_rn(nqn), c.rqs);
                tmx = __fmaf_rn(Lx, c.inv_v, __fdiv_rn(Ax, Rx));
                tmn = __fmaf_rn(Ln, c.inv_v, __fdiv_rn(An, Rn));
                const float ref = (na == 2) ? tmn : ref2;
                if (tmx < ref || k == last) break;
            }
            float nm = (tmx > tmn) ? tmx : tmn;
            FOR_ACTIVE(g) if (g != gx && g != gn && TF(F_TC, g) > nm) nm = TF(F_TC, g);
            if (!(nm < old_max)) break;   // the accepted move does not lower the maximum: keep the old state
            const unsigned long long bit = 1ull << k;
            TM(0, gx) |= bit;
            TM(0, gn) &= ~bit;
            TQ(Q_RQ, gx) = nqx; TQ(Q_RQ, gn) = nqn;
            TF(F_RF, gx) = Rx; TF(F_RF, gn) = Rn;
            TF(F_TC, gx) = tmx; TF(F_TC, gn) = tmn;
        }
    }
    float tmax = TF(F_TC, g_first);
    FOR_ACTIVE(g) tmax = fmaxf(tmax, TF(F_TC, g));

    // --- SU assignment (Algorithm 2, Eq. 6)
    {
    int j = 0;
    FOR_ACTIVE(g) {
#pragma unroll
        for (int w = 0; w < SW; ++w) TM(1 + w, g) = c.sudeal_m[(di + j) * 2 + w];
        TQ(Q_SAQ, g) = c.sudeal_q[di + j];
        ++j;
    }
    }
    // T_wait of tour g with SU set `ms` and fill sum `saq`
    auto twait = [&](int g, const unsigned long long *ms, long long saq) -> float {
        int hb;
        if (SW > 1 && ms[1]) hb = 64 + 63 - __clzll((long long)ms[1]);
        else hb = 63 - __clzll((long long)ms[0]);
        const int grp = c.sugrp[hb];
        int star;
        if (SW > 1 && grp >= 64) {
            star = 64 + __ffsll((long long)(ms[1] & (~0ull << (grp - 64)))) - 1;
        } else {
            const unsigned long long lo = ms[0] & (~0ull << grp);
            if (lo) star = __ffsll((long long)lo) - 1;
            else star = 64 + __ffsll((long long)ms[1]) - 1;
        }
        const float fill = __fmul_rn(__ll2float_rn(saq - c.sufq[star]), c.fqs);
        return __fsub_rn(__fdiv_rn(TF(F_DB2, g), c.suspd[star]), __fdiv_rn(fill, TF(F_RF, g)));
    };
    FOR_ACTIVE(g) {
        unsigned long long ms[2] = {TM(1, g), SW > 1 ? TM(2, g) : 0ull};
        TF(F_TW, g) = twait(g, ms, TQ(Q_SAQ, g));
    }
    if (!p.fix_resources && na >= 2) {
        for (int round = 0; round < c.S; ++round) {
            int gx = g_first, gx2 = -1, gn = -1;
            FOR_ACTIVE(g) if (TF(F_TW, g) > TF(F_TW, gx)) gx = g;
            FOR_ACTIVE(g) if (g != gx && (gx2 < 0 || TF(F_TW, g) > TF(F_TW, gx2))) gx2 = g;
            if (na == 2) gn = gx2;
            else
                FOR_ACTIVE(g) if (g != gx && g != gx2 && (gn < 0 || TF(F_TW, g) < TF(F_TW, gn))) gn = g;
            unsigned long long mn[2] = {TM(1, gn), SW > 1 ? TM(2, gn) : 0ull};
            if (popc_su(mn, SW) <= 1) break;
            unsigned long long mx[2] = {TM(1, gx), SW > 1 ? TM(2, gx) : 0ull};
            const float old_max = TF(F_TW, gx);
            int last;
            if (SW > 1 && mn[1]) last = 64 + 63 - __clzll((long long)mn[1]);
            else last = 63 - __clzll((long long)mn[0]);
            const float ref2 = TF(F_TW, gx2);
            const long long sqx = TQ(Q_SAQ, gx), sqn = TQ(Q_SAQ, gn);
            unsigned long long rest[2] = {mn[0], mn[1]};
            int k = -1;
            float tmx = 0.f, tmn = 0.f;
            long long nqx = 0, nqn = 0;
            unsigned long long ax[2], an[2];
            while (rest[0] | (SW > 1 ? rest[1] : 0ull)) {
                if (rest[0]) { k = __ffsll((long long)rest[0]) - 1; rest[0] &= rest[0] - 1; }
                else { k = 64 + __ffsll((long long)rest[1]) - 1; rest[1] &= rest[1] - 1; }
                ax[0] = mx[0]; an[0] = mn[0];
                ax[1] = mx[1]; an[1] = mn[1];
                if (k < 64) { ax[0] |= 1ull << k; an[0] &= ~(1ull << k); }
                else { ax[1] |= 1ull << (k - 64); an[1] &= ~(1ull << (k - 64)); }
                nqx = sqx + c.sufq[k];
                nqn = sqn - c.sufq[k];
                tmx = twait(gx, ax, nqx);
                tmn = twait(gn, an, nqn);
                const float ref = (na == 2) ? tmn : ref2;
                if (tmx < ref || k == last) break;
            }
            float nm = (tmx > tmn) ? tmx : tmn;
            FOR_ACTIVE(g) if (g != gx && g != gn && TF(F_TW, g) > nm) nm = TF(F_TW, g);
            if (!(nm < old_max)) break;
            TM(1, gx) = ax[0]; TM(1, gn) = an[0];
            if (SW > 1) { TM(2, gx) = ax[1]; TM(2, gn) = an[1]; }
            TQ(Q_SAQ, gx) = nqx; TQ(Q_SAQ, gn) = nqn;
            TF(F_TW, gx) = tmx; TF(F_TW, gn) = tmn;
        }
    }

    // --- path-length cost (Sec. 2.2, Eq. 4)
    float cost = 0.f;
    for (int g = 0; g < c.T; ++g) {
        if (!((amask >> g) & 1u)) continue;
        const unsigned long long hm = TM(0, g);
        unsigned long long sm[2] = {TM(1, g), SW > 1 ? TM(2, g) : 0ull};
        const int nhu = __popcll(hm);
        const int nsu = popc_su(sm, SW);
        long long capq = 0;
#pragma unroll
        for (int w = 0; w < SW; ++w) {
            unsigned long long r = sm[w];
            while (r) {
                const int k = __ffsll((long long)r) - 1;
                r &= r - 1;
                capq += c.sucq[w * 64 + k];
            }
        }
        const float capf = __fmul_rn(__ll2float_rn(capq), c.cqs);
        const float kf = __fdiv_rn((float)nsu, capf);
        const double capd = (double)capq * c.cqs_d;
        float shuttle = 0.f;
        const int nb = x.tour_len(c, g);
        for (int jj = 0; jj < nb; ++jj) {
            const int b = x.bp_at(c, g, jj);
            const int nf = x.bp_len(c, b);
            for (int k = 0; k < nf; ++k) {
                const int f = x.field_at(c, b, k);
                const float s = c.supply[f];
                const float q = __fmul_rn(s, kf);
                const float rq = rintf(q);
                int n;
                if (fabsf(q - rq) <= q * (1.0f / 2097152.0f)) n = exact_ceil(s, nsu, capd, q);
                else n = (int)ceilf(q);
                shuttle = __fmaf_rn((float)(2 * n), c.d(1 + c.B + f, 1 + b), shuttle);
            }
        }
        const float tc = __fadd_rn(__fadd_rn(__fmul_rn((float)nhu, TF(F_LHU, g)), __fmul_rn((float)nsu, TF(F_LSU, g))),
                                   shuttle);
        cost = __fadd_rn(cost, tc);
        if (DUMP) {
            if (o_nhu) o_nhu[g] = (int16_t)nhu;
            if (o_nsu) o_nsu[g] = (int16_t)nsu;
            if (o_tc) o_tc[g] = TF(F_TC, g);
            if (o_tw) o_tw[g] = TF(F_TW, g);
            if (o_tcost) o_tcost[g] = tc;
            if (o_hu) {
                unsigned long long r = hm;
                while (r) { const int k = __ffsll((long long)r) - 1; r &= r - 1; o_hu[c.hu_id[k]] = (int16_t)g; }
            }
            if (o_su) {
#pragma unroll
                for (int w = 0; w < SW; ++w) {
                    unsigned long long r = sm[w];
                    while (r) { const int k = __ffsll((long long)r) - 1; r &= r - 1; o_su[c.su_id[w * 64 + k]] = (int16_t)g; }
                }
            }
        }
    }
    // --- completion-time gate (Sec. 2.5)
    if ((p.gate == 1 && tmax > tmax_star) || (p.gate == 2 && tmax >= tmax_star)) cost = __int_as_float(0x7f800000);
    out.cost = cost;
    out.tmax = tmax;
    return out;
#undef TF
#undef TQ
#undef TM
#undef FOR_ACTIVE
}

// ---------------------------------------------------------------------------
// Shared-memory carving
// ---------------------------------------------------------------------------
__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

struct SmemPlan {
    size_t off_blob, off_plan, off_derived, off_supq, off_bad, off_tf, off_tq, off_tm, off_qidx, off_qmv, total;
};

__host__ __device__ inline SmemPlan carve(int maxt, int sw, int threads, int max_prefix, int max_plan_len, int max_F,
                                          int max_B, int max_T)
{
    SmemPlan s;
    size_t o = 0;
    s.off_blob = o; o += align16((size_t)max_prefix);
    s.off_plan = o; o += align16((size_t)max_plan_len * 2);
    s.off_derived = o; o += align16((size_t)(max_T + 3 * max_B + 2 * max_F) * 2);
    s.off_supq = o; o += align16((size_t)max_B * 8);
    s.off_bad = o; o += align16((size_t)max_B);
    s.off_tf = o; o += align16((size_t)NFLT * maxt * threads * 4);
    s.off_tq = o; o += align16((size_t)NI64 * maxt * threads * 8);
    s.off_tm = o; o += align16((size_t)(1 + sw) * maxt * threads * 8);
    s.off_qidx = o; o += align16((size_t)QUEUE_PER_THREAD * threads * 4);
    s.off_qmv = o; o += align16((size_t)QUEUE_PER_THREAD * threads * 8);
    s.total = o;
    return s;
}

template <class SH>
__host__ __device__ inline SmemPlan carve_shape(int threads, int max_prefix, int max_plan_len, int max_F, int max_B,
                                                int max_T)
{
    return carve(SH::MAXT, SH::SW, threads, max_prefix, max_plan_len, max_F, max_B, max_T);
}

struct BlockShared {
    uint64_t mbar;
    uint32_t phase;
    int32_t staged;
    int32_t qcount;
    int32_t nbad;
    int32_t last;
    int32_t use_best;
    uint32_t iter;
    unsigned long long red[32];
    float redt[32];
};

// Stage instance `inst` (tables by bulk copy, base plan, derived tables).
// Returns false if the bounded wait gave up (error flag set).
template <class SH>
__device__ bool stage_instance(const InstMeta &M, BlockShared &bs, unsigned char *smem, const SmemPlan &sp,
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
    c.D = SH::DSM ? (const float *)(blob + M.L.off_D) : (const float *)(M.blob + M.L.off_D);
    c.area = (const float *)(blob + M.L.off_area);
    c.supply = (const float *)(blob + M.L.off_supply);
    c.supq = (const long long *)(blob + M.L.off_supq);
    c.demq = (const long long *)(blob + M.L.off_demq);
    c.hurq = (const long long *)(blob + M.L.off_hurq);
    c.sufq = (const long long *)(blob + M.L.off_sufq);
    c.sucq = (const long long *)(blob + M.L.off_sucq);
    c.suspd = (const float *)(blob + M.L.off_suspd);
    c.sugrp = (const int *)(blob + M.L.off_sugrp);
    c.hudeal_m = (const unsigned long long *)(blob + M.L.off_hudeal_m);
    c.hudeal_q = (const long long *)(blob + M.L.off_hudeal_q);
    c.sudeal_m = (const unsigned long long *)(blob + M.L.off_sudeal_m);
    c.sudeal_q = (const long long *)(blob + M.L.off_sudeal_q);
    c.hu_id = (const int *)(blob + M.L.off_hu_id);
    c.su_id = (const int *)(blob + M.L.off_su_id);
    c.inv_v = M.inv_hu_speed; c.rqs = M.rq_scale; c.fqs = M.fq_scale; c.cqs = M.cq_scale; c.cqs_d = M.cq_scale_d;
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
    c.tour_start = tour_start; c.bp_start = bp_start; c.bp_tour = bp_tour; c.bp_pos = bp_pos;
    c.field_bp = field_bp; c.field_pos = field_pos; c.base_supq = base_supq; c.bad = bad;
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
    __syncthreads();
    c.nbad = bs.nbad;
    return true;
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

// ---------------------------------------------------------------------------
// The search iteration kernel
// ---------------------------------------------------------------------------
template <class SH>
__global__ void __launch_bounds__(SH::NT) search_iteration_kernel(const InstMeta *__restrict__ meta,
                                                               const WorkItem *__restrict__ work, int32_t n_work,
                                                               SearchParams prm, SmemPlan sp,
                                                               unsigned long long *__restrict__ slot_key,
                                                               float *__restrict__ slot_tmax,
                                                               const int32_t *__restrict__ slot_base)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BlockShared bs;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) {
        mbar_init(&bs.mbar, 1);
        fence_mbar_init();
        bs.phase = 0;
        bs.staged = -1;
        bs.qcount = 0;
    }
    __syncthreads();
    float *tf = (float *)(smem + sp.off_tf);
    long long *tq = (long long *)(smem + sp.off_tq);
    unsigned long long *tm = (unsigned long long *)(smem + sp.off_tm);
    int32_t *qidx = (int32_t *)(smem + sp.off_qidx);
    int16_t *qmv = (int16_t *)(smem + sp.off_qmv);
    const int QN = QUEUE_PER_THREAD * nt;
    Ctx c;
    for (int w = blockIdx.x; w < n_work; w += gridDim.x) {
        const WorkItem wi = work[w];
        const InstMeta &M = meta[wi.inst];
        if (bs.staged != wi.inst) {
            if (!stage_instance<SH>(M, bs, smem, sp, prm, -1, 0xffffffffu, c)) return;
            if (tid == 0) bs.staged = wi.inst;
        }
        const float tmax_star = M.state->tmaxstar;
        const uint32_t iter = bs.iter;
        const int c0 = wi.tile_idx * M.tile;
        const int c1 = min(c0 + M.tile, M.n_cand);
        unsigned long long best = ~0ull;
        float best_t = 0.f;
        for (int q0 = c0; q0 < c1; q0 += QN) {
            // phase A: draw moves, exact demand check, compact the feasible ones
            for (int qq = 0; qq < QN; qq += nt) {
                const int i = q0 + qq + tid;
                bool feas = false;
                MoveRec m = {4, 0, 0, 0};
                if (i < c1) {
                    m = draw_move(c, prm, (uint32_t)i, iter, M.inst_idx);
                    feas = demand_ok(c, m);
                    if (!feas) {
                        const unsigned long long k = make_key(__int_as_float(0x7f800000), (uint32_t)i);
                        if (k < best) { best = k; best_t = __int_as_float(0x7f800000); }
                    }
                }
                const unsigned ball = __ballot_sync(0xffffffffu, feas);
                int base = 0;
                if ((tid & 31) == 0 && ball) base = atomicAdd(&bs.qcount, __popc(ball));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (feas) {
                    const int pos = base + __popc(ball & ((1u << (tid & 31)) - 1u));
                    qidx[pos] = i;
                    qmv[pos * 4 + 0] = (int16_t)m.kind; qmv[pos * 4 + 1] = (int16_t)m.v;
                    qmv[pos * 4 + 2] = (int16_t)m.a; qmv[pos * 4 + 3] = (int16_t)m.b;
                }
            }
            __syncthreads();
            const int nq = bs.qcount;
            // phase B: score the queued candidates, one per thread
            for (int q = tid; q < nq; q += nt) {
                const int i = qidx[q];
                MoveRec m = {qmv[q * 4], qmv[q * 4 + 1], qmv[q * 4 + 2], qmv[q * 4 + 3]};
                ScoreOut r = score_candidate<SH, false>(c, prm, m, tmax_star, tf, tq, tm, nt, tid, nullptr, nullptr,
                                                        nullptr, nullptr, nullptr, nullptr, nullptr);
                const unsigned long long k = make_key(r.cost, (uint32_t)i);
                if (k < best) { best = k; best_t = r.tmax; }
            }
            __syncthreads();
            if (tid == 0) bs.qcount = 0;
            __syncthreads();
        }
        // block argmin: warp shuffle, then across warps
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ok = __shfl_xor_sync(0xffffffffu, best, o);
            const float ot = __shfl_xor_sync(0xffffffffu, best_t, o);
            if (ok < best) { best = ok; best_t = ot; }
        }
        if ((tid & 31) == 0) { bs.red[tid >> 5] = best; bs.redt[tid >> 5] = best_t; }
        __syncthreads();
        if (tid < 32) {
            const int nw = nt >> 5;
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
                    const uint32_t istar = (uint32_t)(bk & 0xffffffffu);
                    const float cst = __uint_as_float((uint32_t)(bk >> 32));
                    InstState *st = M.state;
                    int ind = 0;
                    if (isfinite(cst)) {
                        const MoveRec m = draw_move(c, prm, istar, iter, M.inst_idx);
                        write_plan(c, m, M.xold);
                        if (cst < st->cstar) {
                            for (int k = 0; k < M.plan_len; ++k) M.xbest[k] = M.xold[k];
                            st->cstar = cst;
                            st->tmaxstar = bt;
                            ind = (m.kind == 0 || m.kind == 2) ? 1 : 2;
                        }
                    } else {
                        const int16_t *pl = c.bp_order;
                        for (int k = 0; k < M.plan_len; ++k) M.xold[k] = pl[k];
                    }
                    const int li = (int)(iter % (uint32_t)M.log_cap);
                    M.log_istar[li] = (int32_t)istar;
                    M.log_cistar[li] = cst;
                    M.log_usebest[li] = (int8_t)bs.use_best;
                    M.log_cstar[li] = st->cstar;
                    M.log_ind[li] = (int8_t)ind;
                    st->iter = iter + 1;
                    st->done = 0;
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Inspection kernels
// ---------------------------------------------------------------------------
template <class SH>
__global__ void __launch_bounds__(SH::NT) score_dump_kernel(const InstMeta *__restrict__ meta, int32_t inst,
                                                         int32_t use_best, uint32_t iter, float tmax_star, int32_t i0,
                                                         int32_t n, int32_t identity, SearchParams prm, SmemPlan sp,
                                                         float *cost, float *tmax, int16_t *moves, int16_t *nhu,
                                                         int16_t *nsu, float *tcompl, float *twait, float *tcost,
                                                         int16_t *hu_tour, int16_t *su_tour)
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
    float *tf = (float *)(smem + sp.off_tf);
    long long *tq = (long long *)(smem + sp.off_tq);
    unsigned long long *tm = (unsigned long long *)(smem + sp.off_tm);
    const int T = M.T;
    for (int k = blockIdx.x * nt + tid; k < n; k += gridDim.x * nt) {
        const int i = i0 + k;
        MoveRec m = identity ? MoveRec{4, 0, 0, 0} : draw_move(c, prm, (uint32_t)i, iter, M.inst_idx);
        if (moves) { moves[k * 4] = (int16_t)m.kind; moves[k * 4 + 1] = (int16_t)m.v; moves[k * 4 + 2] = (int16_t)m.a; moves[k * 4 + 3] = (int16_t)m.b; }
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
        if (demand_ok(c, m))
            r = score_candidate<SH, true>(c, prm, m, tmax_star, tf, tq, tm, nt, tid, o_nhu, o_nsu, o_tc, o_tw, o_tk,
                                          o_hu, o_su);
        else { r.cost = __int_as_float(0x7f800000); r.tmax = __int_as_float(0x7f800000); }
        if (cost) cost[k] = r.cost;
        if (tmax) tmax[k] = r.tmax;
    }
}

template <class SH>
__global__ void __launch_bounds__(SH::NT) decode_kernel(const InstMeta *__restrict__ meta, int32_t inst, int32_t use_best,
                                                     uint32_t iter, const int32_t *idx, int32_t n, SearchParams prm,
                                                     SmemPlan sp, int16_t *plans)
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
        const MoveRec m = draw_move(c, prm, (uint32_t)idx[k], iter, M.inst_idx);
        write_plan(c, m, plans + (size_t)k * rowlen);
    }
}

// ---------------------------------------------------------------------------
// Host-side launch wrappers
// ---------------------------------------------------------------------------
int max_tours_of(int32_t shape) { return shape == SHAPE_T4_S64_DSMEM ? 4 : shape == SHAPE_T8_S64_DSMEM ? 8 : 16; }
int threads_of(int32_t shape)
{
    return shape == SHAPE_T4_S64_DSMEM ? ShapeA::NT : shape == SHAPE_T8_S64_DSMEM ? ShapeB::NT : ShapeC::NT;
}
int max_su_of(int32_t shape) { return shape == SHAPE_T16_S128_GMEM ? 128 : 64; }
bool dist_in_smem(int32_t shape) { return shape != SHAPE_T16_S128_GMEM; }

static SmemPlan plan_for(const LaunchCfg &cfg)
{
    switch (cfg.shape) {
    case SHAPE_T4_S64_DSMEM:
        return carve_shape<ShapeA>(cfg.threads, cfg.max_prefix, cfg.max_plan_len, cfg.max_F, cfg.max_B, cfg.max_T);
    case SHAPE_T8_S64_DSMEM:
        return carve_shape<ShapeB>(cfg.threads, cfg.max_prefix, cfg.max_plan_len, cfg.max_F, cfg.max_B, cfg.max_T);
    default:
        return carve_shape<ShapeC>(cfg.threads, cfg.max_prefix, cfg.max_plan_len, cfg.max_F, cfg.max_B, cfg.max_T);
    }
}

size_t shared_bytes(int32_t shape, int32_t threads, int32_t max_prefix, int32_t max_plan_len, int32_t max_F,
                    int32_t max_B, int32_t max_T)
{
    LaunchCfg cfg{};
    cfg.shape = shape; cfg.threads = threads; cfg.max_prefix = max_prefix; cfg.max_plan_len = max_plan_len;
    cfg.max_F = max_F; cfg.max_B = max_B; cfg.max_T = max_T;
    return plan_for(cfg).total;
}

template <class SH>
static cudaError_t set_attrs(size_t smem)
{
    cudaError_t e = cudaFuncSetAttribute(search_iteration_kernel<SH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(score_dump_kernel<SH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(decode_kernel<SH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t configure_kernels(int32_t shape, size_t smem)
{
    switch (shape) {
    case SHAPE_T4_S64_DSMEM: return set_attrs<ShapeA>(smem);
    case SHAPE_T8_S64_DSMEM: return set_attrs<ShapeB>(smem);
    default: return set_attrs<ShapeC>(smem);
    }
}

cudaError_t launch_search_iteration(const LaunchCfg &cfg, const InstMeta *d_meta, const WorkItem *d_work,
                                          int32_t n_work, SearchParams prm, unsigned long long *slot_key,
                                          float *slot_tmax, const int32_t *slot_base, cudaStream_t s)
{
    const SmemPlan sp = plan_for(cfg);
    switch (cfg.shape) {
    case SHAPE_T4_S64_DSMEM:
        search_iteration_kernel<ShapeA><<<cfg.grid, cfg.threads, sp.total, s>>>(d_meta, d_work, n_work, prm, sp,
                                                                              slot_key, slot_tmax, slot_base);
        break;
    case SHAPE_T8_S64_DSMEM:
        search_iteration_kernel<ShapeB><<<cfg.grid, cfg.threads, sp.total, s>>>(d_meta, d_work, n_work, prm, sp,
                                                                              slot_key, slot_tmax, slot_base);
        break;
    default:
        search_iteration_kernel<ShapeC><<<cfg.grid, cfg.threads, sp.total, s>>>(d_meta, d_work, n_work, prm, sp,
                                                                              slot_key, slot_tmax, slot_base);
    }
    return cudaGetLastError();
}

cudaError_t launch_score_dump(const LaunchCfg &cfg, const InstMeta *d_meta, int32_t inst, int32_t use_best,
                              uint32_t iter, float tmax_star, int32_t i0, int32_t n, int32_t identity,
                              SearchParams prm, float *d_cost, float *d_tmax, int16_t *d_moves, int16_t *d_nhu,
                              int16_t *d_nsu, float *d_tcompl, float *d_twait, float *d_tcost, int16_t *d_hu_tour,
                              int16_t *d_su_tour, cudaStream_t s)
{
    const SmemPlan sp = plan_for(cfg);
    int grid = (n + cfg.threads - 1) / cfg.threads;
    if (grid > cfg.grid) grid = cfg.grid;
    if (grid < 1) grid = 1;
#define DUMP_ARGS d_meta, inst, use_best, iter, tmax_star, i0, n, identity, prm, sp, d_cost, d_tmax, d_moves, d_nhu, \
                  d_nsu, d_tcompl, d_twait, d_tcost, d_hu_tour, d_su_tour
    switch (cfg.shape) {
    case SHAPE_T4_S64_DSMEM: score_dump_kernel<ShapeA><<<grid, cfg.threads, sp.total, s>>>(DUMP_ARGS); break;
    case SHAPE_T8_S64_DSMEM: score_dump_kernel<ShapeB><<<grid, cfg.threads, sp.total, s>>>(DUMP_ARGS); break;
    default: score_dump_kernel<ShapeC><<<grid, cfg.threads, sp.total, s>>>(DUMP_ARGS);
    }
#undef DUMP_ARGS
    return cudaGetLastError();
}

cudaError_t launch_decode(const LaunchCfg &cfg, const InstMeta *d_meta, int32_t inst, int32_t use_best,
                          uint32_t iter, const int32_t *d_idx, int32_t n, SearchParams prm, int16_t *d_plans,
                          cudaStream_t s)
{
    const SmemPlan sp = plan_for(cfg);
    int grid = (n + cfg.threads - 1) / cfg.threads;
    if (grid > cfg.grid) grid = cfg.grid;
    if (grid < 1) grid = 1;
    switch (cfg.shape) {
    case SHAPE_T4_S64_DSMEM:
        decode_kernel<ShapeA><<<grid, cfg.threads, sp.total, s>>>(d_meta, inst, use_best, iter, d_idx, n, prm, sp, d_plans);
        break;
    case SHAPE_T8_S64_DSMEM:
        decode_kernel<ShapeB><<<grid, cfg.threads, sp.total, s>>>(d_meta, inst, use_best, iter, d_idx, n, prm, sp, d_plans);
        break;
    default:
        decode_kernel<ShapeC><<<grid, cfg.threads, sp.total, s>>>(d_meta, inst, use_best, iter, d_idx, n, prm, sp, d_plans);
    }
    return cudaGetLastError();
}

}  // namespace biolog
