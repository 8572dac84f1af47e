// Tensor-core kernels of the learned move ranking: a BF16 GEMM on the 5th
// generation tensor cores (tcgen05.mma, FP32 accumulators in tensor memory),
// plus the small elementwise kernels of the MLP's forward pass, backward pass
// and Adam update. Nothing here is from the paper (the learned proposal is an
// extension of its random Step 8).
//
// GEMM: C[M x N] = A[M x K] * B[N x K]^T (+ bias[N], optional ReLU), A and B
// BF16 row-major with K contiguous, C written as FP32 and/or BF16. One CTA of
// 128 threads per 128-row tile and the whole N (<= 256): the accumulator tile
// is 128 TMEM lanes x N FP32 columns. K is staged in chunks of 64 into shared
// memory in the canonical no-swizzle K-major layout -- each 16-wide K slice a
// slab of 8x8 core matrices, (row group, k block) at offset (2 * rg + kb) * 128
// bytes -- and one elected thread issues one tcgen05.mma per slice, committed
// to an mbarrier that the CTA waits on with a wall-clock bound.
#include <algorithm>
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace biolog {

namespace mlp {

constexpr int BM = 128;        // rows per CTA (TMEM lanes)
constexpr int BK = 64;         // K per staged chunk
constexpr int THREADS = 128;   // 4 warps: warp w owns TMEM lanes 32w..32w+31
constexpr int TMEM_COLS = 256;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t now_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// wait for the MMAs committed to `bar`; gives up after ~1 s
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = now_ns();
    while (!mbar_try(bar, parity))
        if (now_ns() - t0 > 1000000000ull) return false;
    return true;
}

// Shared-memory matrix descriptor (no swizzle, K-major): start address, byte
// offset between core matrices adjacent in K (leading) and in M/N (stride),
// descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(const void *p, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((smem_u32(p) >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major.
__host__ __device__ constexpr uint32_t instr_desc(int m, int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// eight FP32 values rounded to BF16 (round to nearest even), packed into 16 bytes
__device__ __forceinline__ uint4 pack8_bf16(const float *x)
{
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const __nv_bfloat162 p = __floats2bfloat162_rn(x[2 * q], x[2 * q + 1]);
        w[q] = *reinterpret_cast<const uint32_t *>(&p);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// max(x, 0) rounded to BF16 for a pair (lo, hi), packed lo | hi << 16: one cvt with
// ReLU (rounding is monotonic and keeps 0, so it equals rounding max(x, 0); a NaN
// stays NaN, where fmaxf would give 0)
__device__ __forceinline__ uint32_t relu_bf16x2(float lo, float hi)
{
    uint32_t w;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(w) : "f"(hi), "f"(lo));
    return w;
}

// Copy a [rows x 64] BF16 chunk (row stride ld elements, starting at column k0)
// into 4 slabs of 16 K each; rows >= nrows and columns >= K are zero.
__device__ __forceinline__ void stage_chunk(__nv_bfloat16 *dst, const __nv_bfloat16 *src, int rows, int nrows, int ld,
                                            int k0, int K)
{
    // one 16-byte segment = one core-matrix row: 8 consecutive K elements
    const int segs = rows * (BK / 8);
    for (int s = threadIdx.x; s < segs; s += blockDim.x) {
        const int r = s / (BK / 8);
        const int kb = s % (BK / 8);          // k block within the chunk (0..7)
        const int slab = kb >> 1, kin = kb & 1;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        const int k = k0 + kb * 8;
        if (r < nrows && k < K) {
            if (k + 8 <= K && ((ld & 7) == 0)) {
                v = *reinterpret_cast<const uint4 *>(src + (size_t)r * ld + k);
            } else {
                __nv_bfloat16 tmp[8];
                for (int e = 0; e < 8; ++e)
                    tmp[e] = (k + e < K) ? src[(size_t)r * ld + k + e] : __float2bfloat16(0.f);
                v = *reinterpret_cast<uint4 *>(tmp);
            }
        }
        // slab layout: slab s holds rows x 16 elements; core matrix (rg, kin) at (2*rg + kin)*128 bytes
        unsigned char *base = reinterpret_cast<unsigned char *>(dst) + (size_t)slab * rows * 32;
        *reinterpret_cast<uint4 *>(base + (size_t)((r >> 3) * 2 + kin) * 128 + (r & 7) * 16) = v;
    }
}

__global__ void __launch_bounds__(THREADS, 1)
gemm_bf16_tn_kernel(const __nv_bfloat16 *__restrict__ A, const __nv_bfloat16 *__restrict__ B,
                    const float *__restrict__ bias, float *__restrict__ Cf, __nv_bfloat16 *__restrict__ Cb,
                    int M, int N, int K, int relu, unsigned int *__restrict__ err, int ksplit)
{
    // split K (ksplit > 0, a multiple of BK): grid row y takes K elements [y ksplit, (y + 1) ksplit)
    // and writes its partial product to slice y of Cf (no bias, ReLU or BF16 output then)
    const int kbeg = ksplit > 0 ? (int)blockIdx.y * ksplit : 0;
    const int kend = ksplit > 0 ? min(K, kbeg + ksplit) : K;
    if (ksplit > 0) Cf += (size_t)blockIdx.y * M * N;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_base_sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * BM;
    const int Np = (N + 15) & ~15;   // MMA N, a multiple of 16
    __nv_bfloat16 *As = reinterpret_cast<__nv_bfloat16 *>(smem);
    __nv_bfloat16 *Bs = As + BM * BK;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;
    const uint32_t idesc = instr_desc(BM, Np);
    uint32_t phase = 0;
    bool ok = true;
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        stage_chunk(As, A + (size_t)m0 * K, BM, min(BM, M - m0), K, k0, K);
        stage_chunk(Bs, B, Np, N, K, k0, K);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> tensor-core reads
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int s = 0; s < BK / 16; ++s) {
                if (k0 + s * 16 >= K) break;
                const uint64_t ad = smem_desc(reinterpret_cast<unsigned char *>(As) + (size_t)s * BM * 32, 128, 256);
                const uint64_t bd = smem_desc(reinterpret_cast<unsigned char *>(Bs) + (size_t)s * Np * 32, 128, 256);
                const uint32_t acc = (k0 > kbeg || s > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&mbar))
                         : "memory");
        }
        // every thread waits for this chunk's MMAs before the buffers are overwritten
        const bool done = mbar_wait(&mbar, phase);
        phase ^= 1u;
        ok = __syncthreads_and(done ? 1 : 0) != 0;
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (ok) {
        const bool vec_ok = (N % 8) == 0 && ((reinterpret_cast<uintptr_t>(Cb) | reinterpret_cast<uintptr_t>(Cf)) & 15) == 0;
        // epilogue: thread (warp w, lane l) owns row 32w + l of the tile
        const int row = m0 + warp * 32 + lane;
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < Np; c0 += 16) {
            uint32_t v[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
                : "r"(taddr + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < M) {
                float x[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = c0 + j;
                    x[j] = __uint_as_float(v[j]);
                    if (bias && col < N) x[j] += bias[col];
                    if (relu) x[j] = fmaxf(x[j], 0.f);
                }
                // whole 16-column pieces of the row go out as 16-byte stores
                if (vec_ok && c0 + 16 <= N) {
                    if (Cb) {
                        uint4 *d = reinterpret_cast<uint4 *>(Cb + (size_t)row * N + c0);
                        d[0] = pack8_bf16(x);
                        d[1] = pack8_bf16(x + 8);
                    }
                    if (Cf) {
                        float4 *d = reinterpret_cast<float4 *>(Cf + (size_t)row * N + c0);
#pragma unroll
                        for (int q = 0; q < 4; ++q) d[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int col = c0 + j;
                        if (col >= N) break;
                        if (Cf) Cf[(size_t)row * N + col] = x[j];
                        if (Cb) Cb[(size_t)row * N + col] = __float2bfloat16(x[j]);
                    }
                }
            }
        }
    } else {
        if (tid == 0) atomicExch(err, 1u);
        mbar_wait(&mbar, phase ^ 1u);   // give MMAs still in flight a second bounded chance before freeing TMEM
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// ---- fused inference: all three layers and the head per 128-row tile ------
//
// y = w4 . relu(W3 relu(W2 relu(W1 x + b1) + b2) + b3) + b4 for M rows, one
// persistent CTA per SM looping over pairs of 128-row tiles (A and B). The
// accumulator of a tile's layer in flight is 128 TMEM lanes x H FP32 columns;
// the hidden activations never leave shared memory: each layer's epilogue
// (bias, ReLU, BF16 rounding -- the same rounding the layer-by-layer path
// stores) writes them straight into the A-operand layout of the tile's next
// layer. The weights of the three layers are pre-packed (fused_pack_kernel)
// into K chunks of 64 in the B-operand layout, so each chunk is one bulk copy
// into a ring of NBUF shared buffers, loaded ahead while the tensor cores work
// on earlier chunks.
//
// Shared layouts (no swizzle, K-major, 8x8 core matrices of 16-byte rows):
//   activations X (tile of the input) and Hs (hidden): core matrix (row group
//   rg, k block kb) at kb * 2048 + rg * 128 bytes   -> LBO 2048, SBO 128
//   weight chunk: core matrix (n group ng, k block kb) at kb * (H * 16) + ng * 128
//                                                      -> LBO H * 16, SBO 128
// Roles (18 warps). The two tiles run staggered: while the tensor cores work
// on one tile's layer, the other tile's epilogue runs.
//   warps 0-7 / 8-15: the epilogue group of tile A / B. Warp w of a group reads
//     TMEM lanes 32 (w % 4) .. +31 of its tile's accumulator, column half
//     (w / 4) % 2; the group stages its tile's input rows too.
//   warp 16, lane 0: issues the tiles' layers in the order of fused_event, each
//     as soon as the tile's operand is written, chunk by chunk as the weights
//     land, and never waits for the tensor cores.
//   warp 17, lane 0: refills the weight ring in the issuer's order (each tile's
//     layer streams its weights again): waits until a slot's MMAs are done and
//     copies the next chunk into it.
// The issuer and the producer are alone in their warps: lanes of one warp that
// wait on different barriers would take turns.
constexpr int FGROUP = 256;                // threads of one epilogue group
constexpr int FEPI = 2 * FGROUP;           // epilogue threads
constexpr int FTHREADS = FEPI + 64;   // + the issuer warp and the producer warp
constexpr int FKMAX = 64;   // largest K per weight chunk

// Weight chunking: a bulk copy costs about the same time whatever its size up
// to at least 64 KB, so chunks are as wide in K as shared memory allows next to
// two tiles' activations: K1 per chunk for layer 1 and K2 for layers 2 and 3
// (multiples of 16, at most 64; a chunk is H x K BF16, 32 KB at H = 256).
// Chunk order: the layer-1 chunks, then layer 2's, then layer 3's.
struct FusedGeom {
    int k1, k2, nch1, nch2, cpt;
    int xkb, hkb;          // 8-element K blocks of the X and H operand layouts
    int max_chunk_bytes;
};

__host__ __device__ inline FusedGeom fused_geom(int I, int H)
{
    FusedGeom g;
    const int i16 = (I + 15) & ~15;
    g.k1 = i16 < FKMAX ? i16 : FKMAX;
    g.nch1 = (i16 + g.k1 - 1) / g.k1;
    g.k2 = H < FKMAX ? H : FKMAX;
    g.nch2 = (H + g.k2 - 1) / g.k2;
    g.cpt = g.nch1 + 2 * g.nch2;
    g.xkb = g.nch1 * g.k1 / 8;
    g.hkb = g.nch2 * g.k2 / 8;
    g.max_chunk_bytes = H * (g.k1 > g.k2 ? g.k1 : g.k2) * 2;
    return g;
}

// chunk jj of a tile: its layer, index within the layer, K width and byte offset in the packed weights
__host__ __device__ inline void fused_chunk(const FusedGeom &g, int H, int jj, int &layer, int &c, int &kc,
                                            size_t &off)
{
    const size_t b1 = (size_t)H * g.k1 * 2, b2 = (size_t)H * g.k2 * 2;
    if (jj < g.nch1) { layer = 0; c = jj; kc = g.k1; off = c * b1; }
    else if (jj < g.nch1 + g.nch2) { layer = 1; c = jj - g.nch1; kc = g.k2; off = g.nch1 * b1 + c * b2; }
    else { layer = 2; c = jj - g.nch1 - g.nch2; kc = g.k2; off = g.nch1 * b1 + (g.nch2 + c) * b2; }
}

__device__ __forceinline__ void mbar_expect_tx_bytes(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}

// 16 accumulator columns of this warp's 32 TMEM lanes; the load and its wait are one asm statement, so
// the registers cannot be read before they have landed
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t *v)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
}

// Pack W (layer l: [H x K_l] row-major BF16) into the chunked B-operand layout.
// Chunk order: layer 1 chunks, layer 2 chunks, layer 3 chunks; K beyond K_l is zero.
__global__ void fused_pack_kernel(const __nv_bfloat16 *__restrict__ w1, const __nv_bfloat16 *__restrict__ w2,
                                  const __nv_bfloat16 *__restrict__ w3, int I, int H, uint4 *__restrict__ out)
{
    const FusedGeom g = fused_geom(I, H);
    for (int jj = blockIdx.y; jj < g.cpt; jj += gridDim.y) {
        int layer, c, kc;
        size_t off;
        fused_chunk(g, H, jj, layer, c, kc, off);
        const __nv_bfloat16 *w = layer == 0 ? w1 : (layer == 1 ? w2 : w3);
        const int K = layer == 0 ? I : H;
        const int segs = H * (kc / 8);
        uint4 *dst = out + off / 16;
        for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < segs; s += gridDim.x * blockDim.x) {
            const int kb = s / H, n = s % H;   // 16-byte segment = row n of core matrix (n / 8, kb)
            __nv_bfloat16 e[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int k = c * kc + kb * 8 + q;
                e[q] = k < K ? w[(size_t)n * K + k] : __float2bfloat16(0.f);
            }
            // byte offset kb * H * 16 + (n / 8) * 128 + (n % 8) * 16 = (kb * H + n) * 16
            dst[(size_t)kb * H + n] = *reinterpret_cast<const uint4 *>(e);
        }
    }
}

// Two tiles (A and B) in flight: each has one activation buffer that holds its
// input X for layer 1 and then the hidden activations, in the operand layout.
struct FusedSmem {
    int act0, act1, act_bytes, wb, par, nbuf, total;
};

__host__ __device__ inline FusedSmem fused_smem(int I, int H, int nbuf)
{
    FusedSmem f;
    const FusedGeom g = fused_geom(I, H);
    f.act_bytes = (g.xkb > g.hkb ? g.xkb : g.hkb) * 2048;
    f.act0 = 0;
    f.act1 = f.act_bytes;
    f.wb = 2 * f.act_bytes;
    f.par = f.wb + nbuf * g.max_chunk_bytes;
    f.nbuf = nbuf;
    f.total = f.par + (4 * H + 4) * 4;
    return f;
}

// Stage rows [r0, r0 + 128) of X [M x I] into the activation layout (zero rows >= M, k >= I).
__device__ __forceinline__ void fused_stage_x(unsigned char *xs, const __nv_bfloat16 *__restrict__ X, int M, int I,
                                              int nkb, int r0, int t0, int nthr)
{
    const bool vec = (I % 8) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0;
    for (int s = t0; s < 128 * nkb; s += nthr) {
        const int r = s & 127, kb = s >> 7;   // consecutive threads: consecutive rows, conflict-free stores
        const int row = r0 + r, k = kb * 8;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (row < M && k < I) {
            if (vec) v = __ldg(reinterpret_cast<const uint4 *>(X + (size_t)row * I + k));
            else {
                __nv_bfloat16 e[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) e[q] = (k + q < I) ? X[(size_t)row * I + k + q] : __float2bfloat16(0.f);
                v = *reinterpret_cast<const uint4 *>(e);
            }
        }
        *reinterpret_cast<uint4 *>(xs + kb * 2048 + (r >> 3) * 128 + (r & 7) * 16) = v;
    }
}

// Named barrier `id` over the 256 threads of one epilogue group; returns the AND of `v` over them
__device__ __forceinline__ bool group_and(int id, bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(FGROUP)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void group_sync(int id)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(FGROUP) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// The issue order of the tiles' layers (0, 1, 2 = the three hidden layers), shared by the issuer
// and the producer: event e of [0, 6 (P + 1)) is layer `layer` of tile `t`, or none. Per pair q:
// A0(q) B2(q-1) A1(q) B0(q) A2(q) B1(q), and B2 of the last pair at the end. Tile B runs a layer
// and a half behind tile A, so that each head epilogue (the longest) and most hidden-layer
// epilogues overlap the other tile's long layers (K = H) rather than its short first layer.
__device__ __forceinline__ bool fused_event(int e, int P, int &t, int &layer)
{
    const int q = e / 6, r = e % 6;
    t = r & 1;
    if (!t) { layer = r >> 1; return q < P; }
    if (r == 1) { layer = 2; return q >= 1 && q <= P; }
    layer = r == 3 ? 0 : 1;
    return q < P;
}

// 18 warps: a sub-partition holds five of them, which caps a thread at 96 registers
__global__ void __launch_bounds__(FTHREADS, 1)
fused_mlp_forward_kernel(const __nv_bfloat16 *__restrict__ X, int M, int I, int H, const uint4 *__restrict__ wpack,
                         const float *__restrict__ b1, const float *__restrict__ b2, const float *__restrict__ b3,
                         const float *__restrict__ w4, const float *__restrict__ b4, float *__restrict__ y, int nbuf,
                         unsigned int *__restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    // tma_bar[s]: slot s's weights landed; mma_bar[s]: slot s's MMAs done;
    // acc_bar[t]: tile t's layer done; act_bar[t]: tile t's operand for its next layer written (FGROUP arrivals)
    __shared__ uint64_t tma_bar[4], mma_bar[4], acc_bar[2], act_bar[2], drain_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int fail_sh;
    __shared__ unsigned long long loaded_sh;   // chunk copies the producer issued (for the drain)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const FusedGeom G = fused_geom(I, H);
    const int nch1 = G.nch1, nch2 = G.nch2, cpt = G.cpt;
    const FusedSmem L = fused_smem(I, H, nbuf);
    unsigned char *wb = smem + L.wb;
    float *par = reinterpret_cast<float *>(smem + L.par);   // b1 | b2 | b3 | w4 | b4
    for (int i = tid; i < H; i += FTHREADS) {
        par[i] = b1[i]; par[H + i] = b2[i]; par[2 * H + i] = b3[i]; par[3 * H + i] = w4[i];
    }
    if (tid == 0) par[4 * H] = b4[0];
    const uint32_t buf_bytes = (uint32_t)G.max_chunk_bytes;   // ring buffer stride
    const int ntiles = (M + 127) / 128;
    const int npairs = (ntiles + 1) / 2;
    const int my_pairs = blockIdx.x < npairs ? (npairs - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(2 * TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < 4; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tma_bar[b])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mma_bar[b])) : "memory");
        }
        for (int t = 0; t < 2; ++t) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&acc_bar[t])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&act_bar[t])), "r"(FGROUP) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&drain_bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fail_sh = 0;
        loaded_sh = 0ull;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;   // tile A's accumulator at column 0, tile B's at column 256
    auto failed = [&]() { return (volatile int &)fail_sh != 0; };

    // the issuer's state, kept for the drain
    long long consumed = 0;      // chunks whose MMAs were issued
    uint32_t tma_ph = 0;         // bit b: parity of the next wait on tma_bar[b]

    if (warp == FEPI / 32) {
        if (lane == 0) {
            // ---- MMA issuer: the tiles' layers in the order of fused_event ----
            const uint32_t idesc = instr_desc(128, H);
            // descriptors: the start-address field (bits 0-13, address >> 4) is added per operand
            const uint64_t a_tmpl = smem_desc(smem, 2048, 128) & ~0x3FFFull;
            const uint64_t b_tmpl = smem_desc(smem, (uint32_t)H * 16, 128) & ~0x3FFFull;
            const uint32_t a_addr0 = smem_u32(smem + L.act0) >> 4, a_addr1 = smem_u32(smem + L.act1) >> 4;
            const uint32_t w_addr = smem_u32(wb) >> 4;
            uint32_t act_ph = 0;   // bit t: parity of the next wait on act_bar[t]
            int cb = 0;            // ring slot of the next chunk
            bool good = true;
            for (int e = 0; e < 6 * (my_pairs + 1) && good; ++e) {
                int t, layer;
                if (!fused_event(e, my_pairs, t, layer)) continue;
                const int nch = layer == 0 ? nch1 : nch2;
                // tile t's operand (its input, or the previous layer's epilogue) is in place, and that
                // epilogue has read its accumulator
                if (failed() || !mbar_wait(&act_bar[t], (act_ph >> t) & 1u)) { good = false; break; }
                act_ph ^= 1u << t;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a_addr = t ? a_addr1 : a_addr0, acc_t = tmem + (uint32_t)(t * TMEM_COLS);
                // K steps of 16 in the layer and per full chunk (zero padded past K). A's descriptor advances
                // 256 per step (two 2048-byte core-matrix blocks), the chunk's 2 H (two H * 16-byte blocks).
                // The chunk geometry is fixed per layer, so only the wait, the fence and the commit sit
                // between one chunk's MMAs and the next's (an address field stays below 2^14, so + is |).
                const int K = layer == 0 ? I : H, spc = (layer == 0 ? G.k1 : G.k2) / 16, nsteps = (K + 15) / 16;
                uint64_t ad = a_tmpl + (uint64_t)a_addr;
                for (int c = 0, s0 = 0; c < nch; ++c, s0 += spc) {
                    if (!mbar_wait(&tma_bar[cb], (tma_ph >> cb) & 1u)) { good = false; break; }
                    tma_ph ^= 1u << cb;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint64_t bd = b_tmpl + (uint64_t)(w_addr + (uint32_t)cb * (buf_bytes >> 4));
                    const int ns = min(spc, nsteps - s0);
                    if (ns == 4) {
#pragma unroll
                        for (int s = 0; s < 4; ++s)
                            tc_mma(acc_t, ad + 256u * s, bd + (uint64_t)(2 * s * H), idesc, (s0 + s) > 0 ? 1u : 0u);
                    } else {
                        for (int s = 0; s < ns; ++s)
                            tc_mma(acc_t, ad + 256u * s, bd + (uint64_t)(2 * s * H), idesc, (s0 + s) > 0 ? 1u : 0u);
                    }
                    ad += 256u * ns;
                    tc_commit(&mma_bar[cb]);
                    ++consumed;
                    cb = cb + 1 == nbuf ? 0 : cb + 1;
                }
                if (good) tc_commit(&acc_bar[t]);
            }
            if (!good) fail_sh = 1;
        }
        __syncwarp();
    } else if (warp == FEPI / 32 + 1) {
        if (lane == 0) {
            // ---- weight producer: the chunks in the issuer's order (fused_event, then chunk) ----
            const long long total = (long long)my_pairs * 2 * cpt;
            long long loaded = 0;
            uint32_t mma_ph = 0;   // bit b: parity of the next wait on mma_bar[b]
            int lb = 0, e = 0, t = 0, layer = 0, c = 0;
            while (e < 6 * (my_pairs + 1) && !fused_event(e, my_pairs, t, layer)) ++e;
            for (; loaded < total; ++loaded) {
                // slot lb's previous chunk (loaded - nbuf) must be consumed first
                if (loaded >= nbuf) {
                    if (failed() || !mbar_wait(&mma_bar[lb], (mma_ph >> lb) & 1u)) { fail_sh = 1; break; }
                    mma_ph ^= 1u << lb;
                }
                int lay, cc, kc;
                size_t off;
                fused_chunk(G, H, (layer == 0 ? 0 : (layer == 1 ? nch1 : nch1 + nch2)) + c, lay, cc, kc, off);
                const uint32_t bytes = (uint32_t)H * kc * 2;
                mbar_expect_tx_bytes(&tma_bar[lb], bytes);
                bulk_g2s(wb + (size_t)lb * buf_bytes, wpack + off / 16, bytes, &tma_bar[lb]);
                lb = lb + 1 == nbuf ? 0 : lb + 1;
                if (++c == (layer == 0 ? nch1 : nch2)) {
                    c = 0;
                    do ++e;
                    while (e < 6 * (my_pairs + 1) && !fused_event(e, my_pairs, t, layer));
                }
            }
            loaded_sh = (unsigned long long)loaded;
        }
        __syncwarp();
    } else {
        // ---- epilogue group t (warps 8 t .. 8 t + 7): tile t of every pair ----
        const int t = warp >> 3, gw = warp & 7, gtid = tid & (FGROUP - 1), bar_id = 1 + t;
        const int q = gw & 3, half = gw >> 2;   // TMEM lanes 32 q .. 32 q + 31, column half
        const int row_in_tile = 32 * q + lane;
        const int col_lo = half * (H / 2), col_hi = col_lo + H / 2;   // H / 2 is a multiple of 16
        unsigned char *act = smem + (t ? L.act1 : L.act0);
        const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(t * TMEM_COLS);
        // The next pair's input rows are loaded into registers while this tile's last layer runs
        // (16-byte rows, at most XPRE segments per thread); other widths are staged directly.
        constexpr int XPRE = 4;
        const int xsegs = 128 * G.xkb;   // 16-byte segments per tile
        const bool xpre = (I % 8) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0 && xsegs <= XPRE * FGROUP;
        uint4 xr[XPRE];
        auto x_load = [&](int tile) {
#pragma unroll
            for (int k = 0; k < XPRE; ++k) {
                const int s = gtid + k * FGROUP;
                const int row = tile * 128 + (s & 127), kk = (s >> 7) * 8;
                xr[k] = (s < xsegs && row < M && kk < I) ? __ldg(reinterpret_cast<const uint4 *>(X + (size_t)row * I + kk))
                                                        : make_uint4(0u, 0u, 0u, 0u);
            }
        };
        auto x_store = [&]() {
#pragma unroll
            for (int k = 0; k < XPRE; ++k) {
                const int s = gtid + k * FGROUP, r = s & 127;
                if (s < xsegs) *reinterpret_cast<uint4 *>(act + (s >> 7) * 2048 + (r >> 3) * 128 + (r & 7) * 16) = xr[k];
            }
        };
        uint32_t acc_ph = 0;
        bool gok = true;   // uniform over the group (every decision below is voted on)
        for (int p = 0; p < my_pairs && gok; ++p) {
            const int pair = (int)blockIdx.x + p * (int)gridDim.x, tile = 2 * pair + t;
            if (xpre && p > 0) x_store();
            else fused_stage_x(act, X, M, I, G.xkb, tile * 128, gtid, FGROUP);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&act_bar[t]);
            for (int layer = 0; layer < 3; ++layer) {
                if (layer == 2 && xpre && p + 1 < my_pairs) x_load(tile + 2 * (int)gridDim.x);
                const bool got = !failed() && mbar_wait(&acc_bar[t], acc_ph);
                acc_ph ^= 1u;
                gok = group_and(bar_id, got);
                if (!gok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const float *bias = par + layer * H;
                if (layer < 2) {
                    unsigned char *dst0 = act + (row_in_tile >> 3) * 128 + (row_in_tile & 7) * 16;
                    for (int cb = col_lo; cb < col_hi; cb += 16) {   // 16 columns per TMEM load (96 registers)
                        uint32_t v[16];
                        tmem_ld16(taddr + (uint32_t)cb, v);
                        const float4 *b4v = reinterpret_cast<const float4 *>(bias + cb);
                        uint32_t w[8];
#pragma unroll
                        for (int qq = 0; qq < 4; ++qq) {
                            const float4 bb = b4v[qq];
                            w[2 * qq] = relu_bf16x2(__uint_as_float(v[4 * qq]) + bb.x, __uint_as_float(v[4 * qq + 1]) + bb.y);
                            w[2 * qq + 1] =
                                relu_bf16x2(__uint_as_float(v[4 * qq + 2]) + bb.z, __uint_as_float(v[4 * qq + 3]) + bb.w);
                        }
                        unsigned char *dst = dst0 + (size_t)(cb / 8) * 2048;
                        *reinterpret_cast<uint4 *>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
                        *reinterpret_cast<uint4 *>(dst + 2048) = make_uint4(w[4], w[5], w[6], w[7]);
                    }
                    // the next layer's operand is written and this accumulator read: the issuer may go on
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    mbar_arrive(&act_bar[t]);
                } else {
                    float acc = 0.f;
                    for (int cb = col_lo; cb < col_hi; cb += 16) {
                        uint32_t v[16];
                        tmem_ld16(taddr + (uint32_t)cb, v);
#pragma unroll
                        for (int qq = 0; qq < 4; ++qq) {
                            const float4 bb = reinterpret_cast<const float4 *>(bias + cb)[qq];
                            const float4 ww = reinterpret_cast<const float4 *>(par + 3 * H + cb)[qq];
                            const uint32_t h01 =
                                relu_bf16x2(__uint_as_float(v[4 * qq]) + bb.x, __uint_as_float(v[4 * qq + 1]) + bb.y);
                            const uint32_t h23 =
                                relu_bf16x2(__uint_as_float(v[4 * qq + 2]) + bb.z, __uint_as_float(v[4 * qq + 3]) + bb.w);
                            acc = fmaf(__uint_as_float(h01 << 16), ww.x, acc);
                            acc = fmaf(__uint_as_float(h01 & 0xFFFF0000u), ww.y, acc);
                            acc = fmaf(__uint_as_float(h23 << 16), ww.z, acc);
                            acc = fmaf(__uint_as_float(h23 & 0xFFFF0000u), ww.w, acc);
                        }
                    }
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    // the two column halves' dot products meet in this tile's (now free) activation buffer
                    float *ypart = reinterpret_cast<float *>(act);
                    ypart[half * 128 + row_in_tile] = acc;
                    group_sync(bar_id);
                    const int row = tile * 128 + row_in_tile;
                    if (half == 0 && row < M) y[row] = (acc + ypart[128 + row_in_tile]) + par[4 * H];
                    group_sync(bar_id);   // ypart read before the buffer takes the next input
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if ((volatile int &)fail_sh) {
        if (tid == FEPI) {
            atomicExch(err, 1u);
            // give copies and MMAs still in flight a bounded chance to land before TMEM is freed
            for (long long j = consumed; j < (long long)loaded_sh; ++j) {
                const int b = (int)(j % nbuf);
                if (mbar_wait(&tma_bar[b], (tma_ph >> b) & 1u)) tma_ph ^= 1u << b;
            }
            tc_commit(&drain_bar);   // completes once every MMA this thread issued is done
            mbar_wait(&drain_bar, 0u);
        }
        __syncthreads();
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TMEM_COLS) : "memory");
}

// ---- elementwise kernels of the MLP ---------------------------------------
// sum of the split-K partial products, slice by slice in order (deterministic)
__global__ void splitk_reduce_kernel(const float *__restrict__ part, float *__restrict__ out, int n, int splits)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float s = part[i];
        for (int y = 1; y < splits; ++y) s += part[(size_t)y * n + i];
        out[i] = s;
    }
}

__global__ void transpose_bf16_kernel(const __nv_bfloat16 *__restrict__ in, __nv_bfloat16 *__restrict__ out, int R,
                                      int Cn)
{
    __shared__ __nv_bfloat16 t[32][33];
    const int c = blockIdx.x * 32 + threadIdx.x, r0 = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int r = r0 + j;
        t[j][threadIdx.x] = (r < R && c < Cn) ? in[(size_t)r * Cn + c] : __float2bfloat16(0.f);
    }
    __syncthreads();
    const int oc = r0 + threadIdx.x;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int orow = blockIdx.x * 32 + j;
        if (orow < Cn && oc < R) out[(size_t)orow * R + oc] = t[threadIdx.x][j];
    }
}

// output layer y = h . w + b (one warp per row) and the MSE gradient dy = 2 (y - t) / M
__global__ void head_forward_kernel(const __nv_bfloat16 *__restrict__ h, const float *__restrict__ w, const float *b,
                                    float *__restrict__ y, const float *__restrict__ target, float *__restrict__ dy,
                                    float *__restrict__ loss, int M, int H)
{
    const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (row >= M) return;
    float s = 0.f;
    for (int j = lane; j < H; j += 32) s = fmaf(__bfloat162float(h[(size_t)row * H + j]), w[j], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    s += b[0];
    if (lane == 0) {
        y[row] = s;
        if (target) {
            const float e = s - target[row];
            dy[row] = 2.f * e / (float)M;
            atomicAdd(loss, e * e / (float)M);
        }
    }
}

// dh = dy (outer) w, masked by h > 0 (ReLU of the layer below); dw = h^T dy, db = sum dy
__global__ void head_backward_kernel(const __nv_bfloat16 *__restrict__ h, const float *__restrict__ w,
                                     const float *__restrict__ dy, __nv_bfloat16 *__restrict__ dz, float *__restrict__ dw,
                                     float *__restrict__ db, int M, int H)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < H) {
        float acc = 0.f;
        for (int m = 0; m < M; ++m) acc = fmaf(__bfloat162float(h[(size_t)m * H + j]), dy[m], acc);
        dw[j] = acc;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        float s = 0.f;
        for (int m = 0; m < M; ++m) s += dy[m];
        db[0] = s;
    }
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < M * H; idx += gridDim.x * blockDim.x) {
        const int m = idx / H, jj = idx % H;
        const float hv = __bfloat162float(h[idx]);
        dz[idx] = __float2bfloat16(hv > 0.f ? dy[m] * w[jj] : 0.f);
    }
}

// dz = dh * (h > 0), in place on BF16 (ReLU backward), and db[j] = sum_m dz
__global__ void relu_backward_kernel(__nv_bfloat16 *__restrict__ dh, const __nv_bfloat16 *__restrict__ h, int M, int H)
{
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < M * H; idx += gridDim.x * blockDim.x)
        if (!(__bfloat162float(h[idx]) > 0.f)) dh[idx] = __float2bfloat16(0.f);
}

// a block covers 32 columns with 32 row lanes: lane r sums rows r, r + 32, ..., then a
// fixed-order tree over the lanes (deterministic)
__global__ void colsum_kernel(const __nv_bfloat16 *__restrict__ x, float *__restrict__ out, int M, int H)
{
    __shared__ float part[32][33];
    const int j = blockIdx.x * 32 + threadIdx.x, r = threadIdx.y;
    float s = 0.f;
    if (j < H)
        for (int m = r; m < M; m += 32) s += __bfloat162float(x[(size_t)m * H + j]);
    part[r][threadIdx.x] = s;
    __syncthreads();
    for (int w = 16; w > 0; w >>= 1) {
        if (r < w) part[r][threadIdx.x] += part[r + w][threadIdx.x];
        __syncthreads();
    }
    if (r == 0 && j < H) out[j] = part[0][threadIdx.x];
}

// Adam on FP32 master weights; the BF16 copy used by the GEMMs is refreshed
__global__ void adam_kernel(float *__restrict__ w, __nv_bfloat16 *__restrict__ wb, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v, int n, float lr, float b1, float b2, float eps,
                            float c1, float c2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        if (wb) wb[i] = __float2bfloat16(wi);
    }
}

__global__ void f32_to_bf16_kernel(const float *__restrict__ x, __nv_bfloat16 *__restrict__ y, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = __float2bfloat16(x[i]);
}

// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): a counter-based 64-bit mix, here the row draw of a
// training minibatch: row r of step t reads mix(seed + (t * batch + r) * golden) -> uniform below n.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Gather a minibatch of `batch` rows drawn uniformly with replacement from n rows of X [n x in] (BF16)
// and T [n] into xb [batch x in] and tb [batch].
__global__ void sample_rows_kernel(const __nv_bfloat16 *__restrict__ X, const float *__restrict__ T, long long n,
                                   int in, int batch, unsigned long long seed, unsigned long long step,
                                   __nv_bfloat16 *__restrict__ xb, float *__restrict__ tb)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)batch * in;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / in), k = (int)(e % in);
        const unsigned long long z = splitmix64(seed + (step * (unsigned long long)batch + (unsigned long long)r) *
                                                           0x9E3779B97F4A7C15ull);
        const long long row = (long long)__umul64hi(z, (unsigned long long)n);   // floor(z n / 2^64)
        xb[e] = X[row * in + k];
        if (k == 0) tb[r] = T[row];
    }
}

}  // namespace mlp

// at least 80 KB, so no more than two CTAs (2 x 256 TMEM columns) are resident on one SM
// and the tensor-memory allocation never has to wait
size_t mlp_gemm_smem(int N)
{
    const size_t need = (size_t)mlp::BM * mlp::BK * 2 + (size_t)((N + 15) & ~15) * mlp::BK * 2 + 1024;
    return need > 80 * 1024 ? need : 80 * 1024;
}

cudaError_t launch_gemm_bf16(const void *A, const void *B, const float *bias, float *Cf, void *Cb, int M, int N, int K,
                             int relu, unsigned int *err, cudaStream_t s)
{
    const size_t smem = mlp_gemm_smem(N);
    cudaError_t e = cudaFuncSetAttribute(mlp::gemm_bf16_tn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = (M + mlp::BM - 1) / mlp::BM;
    mlp::gemm_bf16_tn_kernel<<<grid, mlp::THREADS, smem, s>>>(
        reinterpret_cast<const __nv_bfloat16 *>(A), reinterpret_cast<const __nv_bfloat16 *>(B), bias, Cf,
        reinterpret_cast<__nv_bfloat16 *>(Cb), M, N, K, relu, err, 0);
    return cudaGetLastError();
}

// Cf [M x N] FP32 = A B^T over a long K, in up to `splits` slices of K (one grid row each,
// partial products in `part`, splits x M x N floats), then summed in slice order.
cudaError_t launch_gemm_bf16_splitk(const void *A, const void *B, float *Cf, float *part, int M, int N, int K,
                                    int splits, unsigned int *err, cudaStream_t s)
{
    const int per = ((K + splits - 1) / splits + mlp::BK - 1) / mlp::BK * mlp::BK;   // K per slice
    const int ns = (K + per - 1) / per;
    const size_t smem = mlp_gemm_smem(N);
    cudaError_t e = cudaFuncSetAttribute(mlp::gemm_bf16_tn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    mlp::gemm_bf16_tn_kernel<<<dim3((M + mlp::BM - 1) / mlp::BM, ns), mlp::THREADS, smem, s>>>(
        reinterpret_cast<const __nv_bfloat16 *>(A), reinterpret_cast<const __nv_bfloat16 *>(B), nullptr, part, nullptr,
        M, N, K, 0, err, per);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    mlp::splitk_reduce_kernel<<<(M * N + 255) / 256, 256, 0, s>>>(part, Cf, M * N, ns);
    return cudaGetLastError();
}

// Whether the fused forward fits: H a multiple of 32 (two column halves of
// whole 16-column TMEM loads), shared memory for the layouts and 2+ buffers.
int fused_mlp_nbuf(int I, int H)
{
    if (H % 32 != 0 || H > 256 || I > 256) return 0;
    for (int nb = 4; nb >= 2; --nb)
        if (mlp::fused_smem(I, H, nb).total <= 227 * 1024 - 2048) return nb;   // room for the static shared memory
    return 0;
}

size_t fused_mlp_pack_bytes(int I, int H)
{
    const mlp::FusedGeom g = mlp::fused_geom(I, H);
    return (size_t)H * 2 * ((size_t)g.nch1 * g.k1 + 2 * (size_t)g.nch2 * g.k2);
}

cudaError_t launch_fused_pack(const void *w1, const void *w2, const void *w3, int I, int H, void *out, cudaStream_t s)
{
    const int cpt = mlp::fused_geom(I, H).cpt;
    mlp::fused_pack_kernel<<<dim3(32, cpt), 256, 0, s>>>(reinterpret_cast<const __nv_bfloat16 *>(w1),
                                                         reinterpret_cast<const __nv_bfloat16 *>(w2),
                                                         reinterpret_cast<const __nv_bfloat16 *>(w3), I, H,
                                                         reinterpret_cast<uint4 *>(out));
    return cudaGetLastError();
}

cudaError_t launch_fused_mlp_forward(const void *x, int M, int I, int H, const void *wpack, const float *b1,
                                     const float *b2, const float *b3, const float *w4, const float *b4, float *y,
                                     unsigned int *err, cudaStream_t s)
{
    const int nbuf = fused_mlp_nbuf(I, H);
    if (nbuf == 0) return cudaErrorInvalidValue;
    // at least 116 KB: one CTA per SM, so its TMEM allocation never waits on another's
    const int smem = std::max(mlp::fused_smem(I, H, nbuf).total, 116 * 1024);
    cudaError_t e = cudaFuncSetAttribute(mlp::fused_mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int npairs = ((M + 127) / 128 + 1) / 2;
    const int grid = std::max(1, std::min(npairs, sms));
    mlp::fused_mlp_forward_kernel<<<grid, mlp::FTHREADS, smem, s>>>(
        reinterpret_cast<const __nv_bfloat16 *>(x), M, I, H, reinterpret_cast<const uint4 *>(wpack), b1, b2, b3, w4,
        b4, y, nbuf, err);
    return cudaGetLastError();
}

cudaError_t launch_transpose_bf16(const void *in, void *out, int R, int Cn, cudaStream_t s)
{
    dim3 grid((Cn + 31) / 32, (R + 31) / 32), block(32, 8);
    mlp::transpose_bf16_kernel<<<grid, block, 0, s>>>(reinterpret_cast<const __nv_bfloat16 *>(in),
                                                      reinterpret_cast<__nv_bfloat16 *>(out), R, Cn);
    return cudaGetLastError();
}

cudaError_t launch_head_forward(const void *h, const float *w, const float *b, float *y, const float *target, float *dy,
                                float *loss, int M, int H, cudaStream_t s)
{
    const int rows_per_block = 8;
    mlp::head_forward_kernel<<<(M + rows_per_block - 1) / rows_per_block, 32 * rows_per_block, 0, s>>>(
        reinterpret_cast<const __nv_bfloat16 *>(h), w, b, y, target, dy, loss, M, H);
    return cudaGetLastError();
}

cudaError_t launch_head_backward(const void *h, const float *w, const float *dy, void *dz, float *dw, float *db, int M,
                                 int H, cudaStream_t s)
{
    // the first (H + 127) / 128 blocks also reduce dW; all of them share the element-wise dz
    const long long elems = (long long)M * H;
    const int grid = (int)std::max<long long>((H + 127) / 128, std::min<long long>((elems + 127) / 128, 1024));
    mlp::head_backward_kernel<<<grid, 128, 0, s>>>(reinterpret_cast<const __nv_bfloat16 *>(h), w, dy,
                                                   reinterpret_cast<__nv_bfloat16 *>(dz), dw, db, M, H);
    return cudaGetLastError();
}

cudaError_t launch_relu_backward(void *dh, const void *h, int M, int H, cudaStream_t s)
{
    mlp::relu_backward_kernel<<<1024, 256, 0, s>>>(reinterpret_cast<__nv_bfloat16 *>(dh),
                                                   reinterpret_cast<const __nv_bfloat16 *>(h), M, H);
    return cudaGetLastError();
}

cudaError_t launch_colsum(const void *x, float *out, int M, int H, cudaStream_t s)
{
    mlp::colsum_kernel<<<(H + 31) / 32, dim3(32, 32), 0, s>>>(reinterpret_cast<const __nv_bfloat16 *>(x), out, M, H);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *w, void *wb, const float *g, float *m, float *v, int n, float lr, float b1, float b2,
                        float eps, int step, cudaStream_t s)
{
    float c1 = 1.f, c2 = 1.f;
    for (int i = 0; i < step; ++i) { c1 *= b1; c2 *= b2; }
    mlp::adam_kernel<<<256, 256, 0, s>>>(w, reinterpret_cast<__nv_bfloat16 *>(wb), g, m, v, n, lr, b1, b2, eps,
                                         1.f - c1, 1.f - c2);
    return cudaGetLastError();
}

cudaError_t launch_sample_rows(const void *X, const float *T, long long n, int in, int batch, unsigned long long seed,
                               unsigned long long step, void *xb, float *tb, cudaStream_t s)
{
    mlp::sample_rows_kernel<<<592, 256, 0, s>>>(reinterpret_cast<const __nv_bfloat16 *>(X), T, n, in, batch, seed,
                                                step, reinterpret_cast<__nv_bfloat16 *>(xb), tb);
    return cudaGetLastError();
}

cudaError_t launch_f32_to_bf16(const float *x, void *y, int n, cudaStream_t s)
{
    mlp::f32_to_bf16_kernel<<<256, 256, 0, s>>>(x, reinterpret_cast<__nv_bfloat16 *>(y), n);
    return cudaGetLastError();
}

}  // namespace biolog
