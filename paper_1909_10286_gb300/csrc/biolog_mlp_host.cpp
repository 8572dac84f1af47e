// Host part of the learned move ranker: an MLP in -> H -> H -> H -> 1 (ReLU)
// whose GEMMs run on the tensor cores (biolog_mlp.cu). Master weights FP32,
// GEMM operands BF16, accumulation FP32, MSE loss, Adam.
#include <cmath>
#include <cstring>
#include <random>
#include <algorithm>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/biolog.h"

namespace biolog {
cudaError_t launch_gemm_bf16(const void *A, const void *B, const float *bias, float *Cf, void *Cb, int M, int N, int K,
                             int relu, unsigned int *err, cudaStream_t s);
cudaError_t launch_transpose_bf16(const void *in, void *out, int R, int Cn, cudaStream_t s);
cudaError_t launch_head_forward(const void *h, const float *w, const float *b, float *y, const float *target, float *dy,
                                float *loss, int M, int H, cudaStream_t s);
cudaError_t launch_gemm_bf16_splitk(const void *A, const void *B, float *Cf, float *part, int M, int N, int K,
                                    int splits, unsigned int *err, cudaStream_t s);
cudaError_t launch_head_backward(const void *h, const float *w, const float *dy, void *dz, float *dw, float *db, int M,
                                 int H, cudaStream_t s);
cudaError_t launch_relu_backward(void *dh, const void *h, int M, int H, cudaStream_t s);
cudaError_t launch_colsum(const void *x, float *out, int M, int H, cudaStream_t s);
cudaError_t launch_adam(float *w, void *wb, const float *g, float *m, float *v, int n, float lr, float b1, float b2,
                        float eps, int step, cudaStream_t s);
cudaError_t launch_f32_to_bf16(const float *x, void *y, int n, cudaStream_t s);
cudaError_t launch_sample_rows(const void *X, const float *T, long long n, int in, int batch, unsigned long long seed,
                               unsigned long long step, void *xb, float *tb, cudaStream_t s);
int fused_mlp_nbuf(int I, int H);
size_t fused_mlp_pack_bytes(int I, int H);
cudaError_t launch_fused_pack(const void *w1, const void *w2, const void *w3, int I, int H, void *out, cudaStream_t s);
cudaError_t launch_fused_mlp_forward(const void *x, int M, int I, int H, const void *wpack, const float *b1,
                                     const float *b2, const float *b3, const float *w4, const float *b4, float *y,
                                     unsigned int *err, cudaStream_t s);
}  // namespace biolog

using namespace biolog;

namespace {
thread_local std::string g_mlp_error;
}

namespace biolog {
cudaStream_t mlp_stream_of(const bl_mlp *m);
}

constexpr int kSplitK = 16;   // most K slices of a weight-gradient product

struct bl_mlp {
    int in = 0, H = 0, max_batch = 0;
    cudaStream_t stream = nullptr;
    int step = 0;
    // parameters: layer l weight [out x in] (FP32 master + BF16), bias; head w4 [H], b4 [1]
    float *w[3] = {}, *b[3] = {}, *w4 = nullptr, *b4 = nullptr;
    uint16_t *wb[3] = {}, *wbt[3] = {};   // BF16 weights and their transposes (for dX)
    float *gw[3] = {}, *gb[3] = {}, *gw4 = nullptr, *gb4 = nullptr;
    float *mw[3] = {}, *vw[3] = {}, *mb[3] = {}, *vb[3] = {}, *mw4 = nullptr, *vw4 = nullptr, *mb4 = nullptr, *vb4 = nullptr;
    // activations (BF16) and scratch
    uint16_t *h[3] = {}, *dz = nullptr, *dzt = nullptr, *ht = nullptr, *dh = nullptr;
    float *y = nullptr, *dy = nullptr, *loss = nullptr, *gtmp = nullptr;
    float *kpart = nullptr;   // split-K partial products of the weight gradients (kSplitK x H x max(H, in))
    unsigned int *err = nullptr;
    // inference: BF16 weights of the three layers packed for the fused kernel (repacked
    // after every change of the weights), or none if the shape does not fit it
    void *wpack = nullptr;
    bool packed = false;
    int fused_nbuf = 0;
    uint16_t *xs = nullptr;   // sampled minibatch (bl_mlp_train_step_sampled), max_batch rows
    float *ts = nullptr;
    std::vector<void *> allocs;
    std::string msg;
    int lin(int l) const { return l == 0 ? in : H; }
};

namespace {

int mlp_fail(bl_mlp *m, cudaError_t e, const char *what)
{
    if (m) m->msg = std::string(what) + ": " + cudaGetErrorString(e);
    else g_mlp_error = std::string(what) + ": " + cudaGetErrorString(e);
    return BL_ECUDA;
}

#define MK(m, call)                                               \
    do {                                                          \
        cudaError_t _e = (call);                                  \
        if (_e != cudaSuccess) return mlp_fail((m), _e, #call);   \
    } while (0)

template <class T>
cudaError_t dalloc(bl_mlp *m, T **p, size_t n)
{
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, n * sizeof(T));
    if (e != cudaSuccess) return e;
    m->allocs.push_back(q);
    *p = reinterpret_cast<T *>(q);
    return cudaMemset(q, 0, n * sizeof(T));
}

int check_err(bl_mlp *m)
{
    unsigned int e = 0;
    MK(m, cudaMemcpyAsync(&e, m->err, 4, cudaMemcpyDeviceToHost, m->stream));
    MK(m, cudaStreamSynchronize(m->stream));
    if (e) {
        m->msg = "a bounded wait in the tensor-core GEMM gave up";
        return BL_ETIMEOUT;
    }
    return BL_OK;
}

int upload_params(bl_mlp *m, const std::vector<std::vector<float>> &W, const std::vector<std::vector<float>> &Bv,
                  const std::vector<float> &w4, float b4)
{
    for (int l = 0; l < 3; ++l) {
        MK(m, cudaMemcpyAsync(m->w[l], W[l].data(), W[l].size() * 4, cudaMemcpyHostToDevice, m->stream));
        MK(m, cudaMemcpyAsync(m->b[l], Bv[l].data(), Bv[l].size() * 4, cudaMemcpyHostToDevice, m->stream));
        MK(m, launch_f32_to_bf16(m->w[l], m->wb[l], (int)W[l].size(), m->stream));
    }
    MK(m, cudaMemcpyAsync(m->w4, w4.data(), w4.size() * 4, cudaMemcpyHostToDevice, m->stream));
    MK(m, cudaMemcpyAsync(m->b4, &b4, 4, cudaMemcpyHostToDevice, m->stream));
    MK(m, cudaStreamSynchronize(m->stream));
    m->packed = false;
    return BL_OK;
}

// inference pass: the fused three-layer kernel where the shape fits it
int infer(bl_mlp *m, const uint16_t *x, int M, float *y_out)
{
    if (m->fused_nbuf == 0) {
        const uint16_t *a = x;
        for (int l = 0; l < 3; ++l) {
            MK(m, launch_gemm_bf16(a, m->wb[l], m->b[l], nullptr, m->h[l], M, m->H, m->lin(l), 1, m->err, m->stream));
            a = m->h[l];
        }
        MK(m, launch_head_forward(m->h[2], m->w4, m->b4, y_out, nullptr, nullptr, nullptr, M, m->H, m->stream));
        return BL_OK;
    }
    if (!m->packed) {
        MK(m, launch_fused_pack(m->wb[0], m->wb[1], m->wb[2], m->in, m->H, m->wpack, m->stream));
        m->packed = true;
    }
    MK(m, launch_fused_mlp_forward(x, M, m->in, m->H, m->wpack, m->b[0], m->b[1], m->b[2], m->w4, m->b4, y_out,
                                   m->err, m->stream));
    return BL_OK;
}

// forward pass; target/dy/loss only when training
int forward(bl_mlp *m, const uint16_t *x, int M, float *y_out, const float *target)
{
    const uint16_t *a = x;
    for (int l = 0; l < 3; ++l) {
        MK(m, launch_gemm_bf16(a, m->wb[l], m->b[l], nullptr, m->h[l], M, m->H, m->lin(l), 1, m->err, m->stream));
        a = m->h[l];
    }
    if (target) MK(m, cudaMemsetAsync(m->loss, 0, 4, m->stream));
    MK(m, launch_head_forward(m->h[2], m->w4, m->b4, y_out, target, m->dy, m->loss, M, m->H, m->stream));
    return BL_OK;
}

// backward pass: gradients of the mean squared error into gw/gb/gw4/gb4
int backward(bl_mlp *m, const uint16_t *x, int M)
{
    const int H = m->H;
    // head: dz3 = dy w4 * (h3 > 0), gw4 = h3^T dy, gb4 = sum dy
    MK(m, launch_head_backward(m->h[2], m->w4, m->dy, m->dz, m->gw4, m->gb4, M, H, m->stream));
    for (int l = 2; l >= 0; --l) {
        const int K = m->lin(l);
        const uint16_t *a = (l == 0) ? x : m->h[l - 1];
        // gw[l] [H x K] = dz^T [H x M] * a [M x K]  ->  A = dz^T, B = a^T [K x M]
        MK(m, launch_transpose_bf16(m->dz, m->dzt, M, H, m->stream));
        MK(m, launch_transpose_bf16(a, m->ht, M, K, m->stream));
        // (K of this product is the batch: split it over kSplitK grid rows, so that more than H / 128 blocks work)
        const int splits = std::min(kSplitK, std::max(1, M / 256));
        if (splits > 1)
            MK(m, launch_gemm_bf16_splitk(m->dzt, m->ht, m->gw[l], m->kpart, H, K, M, splits, m->err, m->stream));
        else
            MK(m, launch_gemm_bf16(m->dzt, m->ht, nullptr, m->gw[l], nullptr, H, K, M, 0, m->err, m->stream));
        MK(m, launch_colsum(m->dz, m->gb[l], M, H, m->stream));
        if (l > 0) {
            // dh [M x K] = dz [M x H] * W [H x K]  ->  A = dz, B = W^T [K x H]
            MK(m, launch_transpose_bf16(m->wb[l], m->wbt[l], H, K, m->stream));
            MK(m, launch_gemm_bf16(m->dz, m->wbt[l], nullptr, nullptr, m->dh, M, K, H, 0, m->err, m->stream));
            MK(m, launch_relu_backward(m->dh, m->h[l - 1], M, K, m->stream));
            MK(m, cudaMemcpyAsync(m->dz, m->dh, (size_t)M * K * 2, cudaMemcpyDeviceToDevice, m->stream));
        }
    }
    return BL_OK;
}

}  // namespace

cudaStream_t biolog::mlp_stream_of(const bl_mlp *m) { return m->stream; }

extern "C" {

const char *bl_mlp_last_error(const bl_mlp *m) { return m ? m->msg.c_str() : g_mlp_error.c_str(); }

int bl_mlp_create(int32_t in_dim, int32_t hidden, int32_t max_batch, uint64_t seed, void *stream, bl_mlp **out)
{
    if (!out) return BL_EINVAL;
    *out = nullptr;
    if (in_dim < 1 || in_dim > 256 || hidden < 16 || hidden > 256 || (hidden % 16) || max_batch < 1) {
        g_mlp_error = "in_dim in [1,256], hidden in [16,256] a multiple of 16, max_batch >= 1";
        return BL_EINVAL;
    }
    bl_mlp *m = new bl_mlp();
    m->in = in_dim; m->H = hidden; m->max_batch = max_batch; m->stream = (cudaStream_t)stream;
    const int H = hidden;
    std::mt19937_64 rng(seed);
    std::vector<std::vector<float>> W(3), Bv(3);
    for (int l = 0; l < 3; ++l) {
        const int K = m->lin(l);
        std::uniform_real_distribution<float> u(-std::sqrt(6.f / K), std::sqrt(6.f / K));   // He-uniform for ReLU
        W[l].resize((size_t)H * K);
        for (float &v : W[l]) v = u(rng);
        Bv[l].assign((size_t)H, 0.f);
    }
    std::vector<float> w4((size_t)H);
    std::uniform_real_distribution<float> u4(-std::sqrt(3.f / H), std::sqrt(3.f / H));
    for (float &v : w4) v = u4(rng);
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < 3 && e == cudaSuccess; ++l) {
        const size_t n = (size_t)H * m->lin(l);
        e = dalloc(m, &m->w[l], n); if (e) break;
        e = dalloc(m, &m->b[l], (size_t)H); if (e) break;
        e = dalloc(m, &m->wb[l], n); if (e) break;
        e = dalloc(m, &m->wbt[l], n); if (e) break;
        e = dalloc(m, &m->gw[l], n); if (e) break;
        e = dalloc(m, &m->gb[l], (size_t)H); if (e) break;
        e = dalloc(m, &m->mw[l], n); if (e) break;
        e = dalloc(m, &m->vw[l], n); if (e) break;
        e = dalloc(m, &m->mb[l], (size_t)H); if (e) break;
        e = dalloc(m, &m->vb[l], (size_t)H); if (e) break;
        e = dalloc(m, &m->h[l], (size_t)max_batch * H);
    }
    const size_t wide = (size_t)max_batch * (size_t)std::max(H, in_dim);
    if (e == cudaSuccess) e = dalloc(m, &m->w4, (size_t)H);
    if (e == cudaSuccess) e = dalloc(m, &m->b4, (size_t)1);
    if (e == cudaSuccess) e = dalloc(m, &m->gw4, (size_t)H);
    if (e == cudaSuccess) e = dalloc(m, &m->gb4, (size_t)1);
    if (e == cudaSuccess) e = dalloc(m, &m->mw4, (size_t)H);
    if (e == cudaSuccess) e = dalloc(m, &m->vw4, (size_t)H);
    if (e == cudaSuccess) e = dalloc(m, &m->mb4, (size_t)1);
    if (e == cudaSuccess) e = dalloc(m, &m->vb4, (size_t)1);
    if (e == cudaSuccess) e = dalloc(m, &m->dz, wide);
    if (e == cudaSuccess) e = dalloc(m, &m->dzt, wide);
    if (e == cudaSuccess) e = dalloc(m, &m->ht, wide);
    if (e == cudaSuccess) e = dalloc(m, &m->dh, wide);
    if (e == cudaSuccess) e = dalloc(m, &m->kpart, (size_t)kSplitK * hidden * std::max(hidden, in_dim));
    if (e == cudaSuccess) e = dalloc(m, &m->y, (size_t)max_batch);
    if (e == cudaSuccess) e = dalloc(m, &m->dy, (size_t)max_batch);
    if (e == cudaSuccess) e = dalloc(m, &m->loss, (size_t)1);
    if (e == cudaSuccess) e = dalloc(m, &m->err, (size_t)1);
    m->fused_nbuf = fused_mlp_nbuf(in_dim, hidden);
    if (e == cudaSuccess && m->fused_nbuf) {
        uint16_t *wp = nullptr;
        e = dalloc(m, &wp, fused_mlp_pack_bytes(in_dim, hidden) / 2);
        m->wpack = wp;
    }
    if (e != cudaSuccess) {
        g_mlp_error = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        bl_mlp_free(m);
        return BL_ECUDA;
    }
    const int rc = upload_params(m, W, Bv, w4, 0.f);
    if (rc != BL_OK) { g_mlp_error = m->msg; bl_mlp_free(m); return rc; }
    *out = m;
    return BL_OK;
}

int bl_mlp_free(bl_mlp *m)
{
    if (!m) return BL_EINVAL;
    if (m->stream) cudaStreamSynchronize(m->stream);
    for (void *p : m->allocs) cudaFree(p);
    delete m;
    return BL_OK;
}

int bl_mlp_forward(bl_mlp *m, const uint16_t *d_x, int32_t M, float *d_y)
{
    if (!m || !d_x || !d_y || M < 1) return BL_EINVAL;
    if (m->fused_nbuf == 0 && M > m->max_batch) return BL_EINVAL;   // the layer-by-layer path uses the batch buffers
    return infer(m, d_x, M, d_y);
}

int bl_mlp_grads(bl_mlp *m, const uint16_t *d_x, const float *d_target, int32_t M, float *h_loss)
{
    if (!m || !d_x || !d_target || M < 1 || M > m->max_batch) return BL_EINVAL;
    int rc = forward(m, d_x, M, m->y, d_target);
    if (rc != BL_OK) return rc;
    rc = backward(m, d_x, M);
    if (rc != BL_OK) return rc;
    if (h_loss) MK(m, cudaMemcpyAsync(h_loss, m->loss, 4, cudaMemcpyDeviceToHost, m->stream));
    return check_err(m);
}

int bl_mlp_train_step(bl_mlp *m, const uint16_t *d_x, const float *d_target, int32_t M, float lr, float *h_loss)
{
    int rc = bl_mlp_grads(m, d_x, d_target, M, h_loss);
    if (rc != BL_OK) return rc;
    m->step += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int l = 0; l < 3; ++l) {
        const int n = m->H * m->lin(l);
        MK(m, launch_adam(m->w[l], m->wb[l], m->gw[l], m->mw[l], m->vw[l], n, lr, b1, b2, eps, m->step, m->stream));
        MK(m, launch_adam(m->b[l], nullptr, m->gb[l], m->mb[l], m->vb[l], m->H, lr, b1, b2, eps, m->step, m->stream));
    }
    MK(m, launch_adam(m->w4, nullptr, m->gw4, m->mw4, m->vw4, m->H, lr, b1, b2, eps, m->step, m->stream));
    MK(m, launch_adam(m->b4, nullptr, m->gb4, m->mb4, m->vb4, 1, lr, b1, b2, eps, m->step, m->stream));
    m->packed = false;
    return BL_OK;
}

int bl_mlp_train_step_sampled(bl_mlp *m, const uint16_t *d_X, const float *d_T, int64_t n_rows, int32_t batch,
                              uint64_t seed, float lr, float *h_loss)
{
    if (!m || !d_X || !d_T || n_rows < 1 || batch < 1 || batch > m->max_batch) return BL_EINVAL;
    if (!m->xs) {
        MK(m, dalloc(m, &m->xs, (size_t)m->max_batch * m->in));
        MK(m, dalloc(m, &m->ts, (size_t)m->max_batch));
    }
    MK(m, launch_sample_rows(d_X, d_T, n_rows, m->in, batch, seed, (unsigned long long)m->step, m->xs, m->ts,
                             m->stream));
    return bl_mlp_train_step(m, m->xs, m->ts, batch, lr, h_loss);
}

// Parameters and gradients in host buffers, layer by layer: w1 [H x in], b1 [H],
// w2 [H x H], b2, w3 [H x H], b3, w4 [H], b4 [1] (any pointer may be NULL).
int bl_mlp_get(bl_mlp *m, int32_t which, float *w1, float *b1, float *w2, float *b2, float *w3, float *b3, float *w4,
               float *b4)
{
    if (!m) return BL_EINVAL;
    float *const *W = which ? m->gw : m->w;
    float *const *Bv = which ? m->gb : m->b;
    float *hw[3] = {w1, w2, w3}, *hb[3] = {b1, b2, b3};
    for (int l = 0; l < 3; ++l) {
        if (hw[l]) MK(m, cudaMemcpyAsync(hw[l], W[l], (size_t)m->H * m->lin(l) * 4, cudaMemcpyDeviceToHost, m->stream));
        if (hb[l]) MK(m, cudaMemcpyAsync(hb[l], Bv[l], (size_t)m->H * 4, cudaMemcpyDeviceToHost, m->stream));
    }
    if (w4) MK(m, cudaMemcpyAsync(w4, which ? m->gw4 : m->w4, (size_t)m->H * 4, cudaMemcpyDeviceToHost, m->stream));
    if (b4) MK(m, cudaMemcpyAsync(b4, which ? m->gb4 : m->b4, 4, cudaMemcpyDeviceToHost, m->stream));
    MK(m, cudaStreamSynchronize(m->stream));
    return BL_OK;
}

int bl_mlp_set(bl_mlp *m, const float *w1, const float *b1, const float *w2, const float *b2, const float *w3,
               const float *b3, const float *w4, const float *b4)
{
    if (!m || !w1 || !b1 || !w2 || !b2 || !w3 || !b3 || !w4 || !b4) return BL_EINVAL;
    std::vector<std::vector<float>> W(3), Bv(3);
    const float *hw[3] = {w1, w2, w3}, *hb[3] = {b1, b2, b3};
    for (int l = 0; l < 3; ++l) {
        W[l].assign(hw[l], hw[l] + (size_t)m->H * m->lin(l));
        Bv[l].assign(hb[l], hb[l] + m->H);
    }
    return upload_params(m, W, Bv, std::vector<float>(w4, w4 + m->H), b4[0]);
}

int bl_gemm_bf16(const uint16_t *d_a, const uint16_t *d_b, const float *d_bias, float *d_cf, uint16_t *d_cb, int32_t M,
                 int32_t N, int32_t K, int32_t relu, uint32_t *d_err, void *stream)
{
    if (!d_a || !d_b || (!d_cf && !d_cb) || !d_err || M < 1 || N < 1 || N > 256 || K < 1) {
        g_mlp_error = "bl_gemm_bf16: bad arguments (1 <= N <= 256)";
        return BL_EINVAL;
    }
    cudaError_t e = launch_gemm_bf16(d_a, d_b, d_bias, d_cf, d_cb, M, N, K, relu, d_err, (cudaStream_t)stream);
    if (e != cudaSuccess) { g_mlp_error = std::string("gemm: ") + cudaGetErrorString(e); return BL_ECUDA; }
    return BL_OK;
}

}  // extern "C"
