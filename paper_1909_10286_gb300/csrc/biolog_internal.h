// Internal layout shared by the host part (biolog_host.cpp) and the kernels
// (biolog_kernels.cu). Not part of the public ABI (include/biolog.h).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace biolog {

// Per-instance table blob in device memory. Every section starts on a
// 16-byte boundary so the staging bulk copy can move it in one piece; the
// distance matrix comes last so a kernel that reads it from global memory can
// stage only the prefix.
struct BlobLayout {
    int32_t off_area;      // f32[F]   field sizes (ha)
    int32_t off_areaq;     // i64[F]   field sizes in fixed point (quantum 2^area exp)
    int32_t off_supply;    // f32[F]   supplies (t)
    int32_t off_supq;      // i64[F]   supplies in fixed point (quantum 2^sup_exp)
    int32_t off_demq;      // i64[B]   smallest fixed-point supply sum meeting d_b
    int32_t off_hurq;      // i64[H]   HU rates, sorted by (rate, id), fixed point
    int32_t off_sufq;      // i64[S]   SU fill areas, sorted by (fill, id), fixed point
    int32_t off_sucq;      // i64[S]   SU capacities in the same sorted order, fixed point
    int32_t off_suinv;     // f32[S]   1 / SU speed, same order
    int32_t off_sufill;    // f32[S]   SU fill areas (ha), same order
    int32_t off_rcp;       // f32[R]   1/k for k = 0..R-1 (entry 0 unused), R = max(F, B) + 1
    int32_t off_sugrp;     // i32[S]   first sorted index with the same fill area
    int32_t off_hudeal_m;  // u64[T*T] HU masks of the round-robin dealing: [na-1][j]
    int32_t off_hudeal_q;  // i64[T*T] their fixed-point rate sums
    int32_t off_sudeal_m;  // u64[T*T*2] SU masks of the dealing (two words)
    int32_t off_sudeal_q;  // i64[T*T] their fixed-point fill sums
    int32_t off_sudeal_c;  // i64[T*T] their fixed-point capacity sums
    int32_t off_hu_id;     // i32[H]   HU id at each sorted position
    int32_t off_su_id;     // i32[S]   SU id at each sorted position
    int32_t off_D;         // i32[N*N] distances in fixed point: round(d * dq_inv), row-major
    int32_t prefix_bytes;  // bytes before off_D (multiple of 16)
    int32_t total_bytes;   // multiple of 16
};

// Per-instance constants and pointers, one record per instance in device memory.
struct InstMeta {
    int32_t F, B, T, H, S, N;
    int32_t n_cand;            // candidates per iteration
    int32_t n_tiles;           // work items of this instance per iteration
    int32_t tile;              // candidates per work item
    uint32_t inst_idx;         // Philox counter word 2
    int32_t plan_len;          // 2B+T+F int16 words (padded to a multiple of 8)
    int32_t log_cap;           // ring-buffer capacity (iterations)
    float inv_hu_speed;        // 1 / HU road speed
    float rq_scale;            // fixed point -> value: multiply by these powers of two
    float fq_scale;
    float cq_scale;
    double cq_scale_d;
    float dq_inv;              // distances -> fixed point: round(d * dq_inv)
    float dq_scale;            // and back: 2^k
    float aq_scale;            // fixed-point areas -> ha
    float inv_l0;              // 1 / mean field-to-BP distance (feature scale)
    float inv_mean_supply;     // 1 / mean field supply
    float inv_mean_area;       // 1 / mean field area
    float mean_fields_per_bp;  // F / B
    BlobLayout L;
    const unsigned char *blob; // device: this instance's table blob
    int16_t *xold;             // device: plan encodings (plan_len int16 each)
    int16_t *xbest;
    struct InstState *state;   // device
    int32_t *log_istar;        // device ring buffers [log_cap]
    float *log_cistar;
    int8_t *log_usebest;
    float *log_cstar;
    int8_t *log_ind;
};

// Mutable per-instance search state in device memory.
struct InstState {
    unsigned long long key;    // running argmin key of the current iteration
    float cstar;               // C*
    float tmaxstar;            // Tmax*
    uint32_t iter;             // iteration counter (Philox counter word 1)
    uint32_t done;             // work items finished in the current iteration
    uint32_t error;            // nonzero: a bounded device wait gave up
    uint32_t pad;
};

struct SearchParams {
    float eps;
    float p_swap;
    uint32_t seed_lo, seed_hi;
    int32_t fix_field_bp;
    int32_t fix_resources;
    int32_t gate;
    int32_t k_moves;           // moves chained per candidate (Step 8 repeated), 1..kMaxMoves
    uint32_t cand_offset;      // candidate numbers of this handle: cand_offset + [0, n_cand)
    int32_t defer_update;      // 1: the iteration only leaves its argmin key in InstState::key
};
constexpr int kMaxMoves = 3;

// One work item: a contiguous candidate range of one instance.
struct WorkItem {
    int32_t inst;
    int32_t tile_idx;
};

// Kernel shape class chosen per handle from the largest instance.
enum ShapeClass : int32_t {
    SHAPE_T4_S64_DSMEM = 0,   // tours <= 4,  HUs and SUs <= 32 (32-bit sets and sums), distances in shared memory
    SHAPE_T6_S64_GMEM = 1,    // tours <= 6,  HUs and SUs <= 64, distances read through L2
    SHAPE_T16_S128_GMEM = 2,  // tours <= 16, SUs <= 128, distances read through L2
    SHAPE_T10_S128_GMEM = 3,  // tours <= 10, SUs <= 128, distances read through L2
};

struct LaunchCfg {
    int32_t shape;
    int32_t lanes;          // lanes per candidate of the search kernel (1: one thread per candidate)
    int32_t threads;        // threads per block
    int32_t grid;           // blocks
    size_t smem;            // dynamic shared memory bytes
    int32_t max_prefix;     // largest staged blob (bytes) over the instances
    int32_t max_plan_len;
    int32_t max_F, max_B, max_T;
};

// Launch wrappers (biolog_kernels.cu).
cudaError_t launch_search_iteration(const LaunchCfg &cfg, const InstMeta *d_meta, const WorkItem *d_work,
                                    int32_t n_work, SearchParams prm, unsigned long long *slot_key,
                                    float *slot_tmax, const int32_t *slot_base, cudaStream_t s,
                                    const uint32_t *cand_list = nullptr, const int32_t *cand_count = nullptr,
                                    int32_t list_stride = 0, float2 *insp = nullptr, int32_t insp_stride = 0);
constexpr int NFEAT = 64;   // features per candidate move
cudaError_t launch_features(const LaunchCfg &cfg, const InstMeta *d_meta, int32_t inst, int32_t use_best,
                            uint32_t iter, int32_t i0, int32_t n, SearchParams prm, uint16_t *d_feat,
                            float *d_base_cost, cudaStream_t s, int32_t n_batch = 0);
cudaError_t launch_select(const float *d_y, int32_t P, int32_t n_keep, float rand_frac, uint32_t salt,
                          uint32_t *d_list, int32_t *d_count, float *d_thresh, int32_t n_batch, cudaStream_t s);
cudaError_t launch_score_dump(const LaunchCfg &cfg, const InstMeta *d_meta, int32_t inst, int32_t use_best,
                              uint32_t iter, float tmax_star, int32_t i0, int32_t n, int32_t identity,
                              SearchParams prm, float *d_cost, float *d_tmax, int16_t *d_moves, int16_t *d_nhu,
                              int16_t *d_nsu, float *d_tcompl, float *d_twait, float *d_tcost, int16_t *d_hu_tour,
                              int16_t *d_su_tour, cudaStream_t s);
cudaError_t launch_decode(const LaunchCfg &cfg, const InstMeta *d_meta, int32_t inst, int32_t use_best,
                          uint32_t iter, const int32_t *d_idx, int32_t n, SearchParams prm, int16_t *d_plans,
                          cudaStream_t s);
cudaError_t launch_apply_key(const LaunchCfg &cfg, const InstMeta *d_meta, SearchParams prm,
                             const unsigned long long *d_key, cudaStream_t s);
cudaError_t launch_state_pack(const InstMeta *d_meta, int32_t n_inst, const int32_t *d_offs, unsigned char *d_buf,
                              int32_t dir, cudaStream_t s);
cudaError_t noalloc_scratch_address(void **ptr);
cudaError_t launch_argmin_noalloc(const LaunchCfg &cfg, const InstMeta *d_meta, int32_t inst, int32_t use_best,
                                  uint32_t iter, float tmax_star, int32_t i0, int32_t n, SearchParams prm,
                                  void *scratch, unsigned long long *d_key, float *d_tmax, cudaStream_t s);
size_t shared_bytes(int32_t shape, int32_t threads, int32_t max_prefix, int32_t max_plan_len, int32_t max_F,
                    int32_t max_B, int32_t max_T);
cudaError_t configure_kernels(int32_t shape, size_t smem);
int search_blocks_per_sm(int32_t shape, size_t smem);
cudaError_t launch_wait_selftest(uint64_t limit_ns, unsigned long long *d_out, cudaStream_t s);
// cooperative search kernel (lanes per candidate > 1)
constexpr int kCoopThreads = 256;
bool coop_supported(int32_t shape, int32_t lanes);
size_t coop_shared_bytes(const LaunchCfg &cfg);
cudaError_t configure_coop(int32_t shape, int32_t lanes, size_t smem);
int coop_blocks_per_sm(int32_t shape, int32_t lanes, size_t smem);
int max_tours_of(int32_t shape);
int threads_of(int32_t shape);
int max_su_of(int32_t shape);
bool dist_in_smem(int32_t shape);

}  // namespace biolog
