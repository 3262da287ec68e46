// Small multilayer perceptron for the learned warm start: inference and
// training kernels.  Layer l maps X_l [B x K_l] to Z_l = X_l W_l^T + b_l
// (W_l stored [N_l x K_l] row-major), hidden layers apply GELU
// (x Phi(x), Phi the normal CDF); the last layer is linear.  Loss: mean
// squared error over all outputs.  Training: backpropagation and Adam.
//
// Precision: matrix products take BF16 operands on the tensor cores
// (mma.sync m16n8k16, FP32 accumulation); weights, biases, pre-activations,
// gradients and Adam moments are FP32; BF16 copies of the weights and of the
// layer inputs feed the products.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/phonon_lbm.h"
#include "lbm_kernels.h"

namespace plbm {
namespace {

constexpr int TK = 32;                     // k depth of a block tile
constexpr int GEMM_THREADS = 128;          // 4 warps

__device__ __forceinline__ unsigned pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4],
                                         const unsigned (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, "
        "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ float gelu(float x) {
    return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad(float x) {
    const float cdf = 0.5f * (1.0f + erff(x * 0.70710678118654752f));
    const float pdf = 0.39894228040143268f * expf(-0.5f * x * x);
    return cdf + x * pdf;
}

enum { EPI_NONE = 0, EPI_GELU = 1, EPI_GELU_BWD = 2 };

// C[m, n] = sum_k A(m, k) B(k, n) (+ bias[n]) with A(m, k) = A[m*am + k*ak],
// B(k, n) = B[k*bk + n*bn] (any strides: every transposition the forward and
// backward passes need).  Outputs (each optional): pre = the FP32 result,
// out = the FP32 result after the epilogue, outb = the same in BF16.
// Epilogues: GELU (forward), GELU backward (the result times GELU'(aux[m, n]),
// aux the pre-activation of the layer below: dZ = dX (.) GELU'(Z)).
// Block tile BM x BN (64 or 32 each), four warps of (BM / 2) x (BN / 2).
template <int BM, int BN>
__global__ void __launch_bounds__(GEMM_THREADS)
gemm_bf16(const __nv_bfloat16 *__restrict__ A, long long am, long long ak,
          const __nv_bfloat16 *__restrict__ B, long long bk, long long bn,
          const float *__restrict__ bias, int M, int N, int K, int epi,
          const float *__restrict__ aux, float *__restrict__ pre, float *__restrict__ out,
          __nv_bfloat16 *__restrict__ outb) {
    __shared__ __align__(16) __nv_bfloat16 As[BM][TK + 8];
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][TK + 8];     // stored [n][k]
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int MI = BM / 32, NJ = BN / 16;     // m16 x n8 tiles per warp
    const int wm = (warp >> 1) * (BM / 2), wn = (warp & 1) * (BN / 2);
    const int g = lane >> 2, tg = lane & 3;
    float acc[MI][NJ][4] = {};
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    // The tiles are filled along the operand's contiguous index with 16-byte
    // loads (8 values) where the rows are 16-byte aligned, element by element
    // otherwise (the first layer's 3 inputs) and at the matrix edges.
    const bool a_k_vec = ak == 1 && am % 8 == 0 && ((uintptr_t)A & 15) == 0;
    const bool a_m_vec = am == 1 && ak % 8 == 0 && ((uintptr_t)A & 15) == 0;
    const bool b_k_vec = bk == 1 && bn % 8 == 0 && ((uintptr_t)B & 15) == 0;
    const bool b_n_vec = bn == 1 && bk % 8 == 0 && ((uintptr_t)B & 15) == 0;
    for (int k0 = 0; k0 < K; k0 += TK) {
        if (a_k_vec) {
            for (int idx = threadIdx.x; idx < BM * TK / 8; idx += GEMM_THREADS) {
                const int r = idx / (TK / 8), c = (idx % (TK / 8)) * 8;
                const int m = m0 + r, k = k0 + c;
                if (m < M && k + 8 <= K) {
                    *reinterpret_cast<uint4 *>(&As[r][c]) =
                        *reinterpret_cast<const uint4 *>(A + (long long)m * am + k);
                } else {
                    for (int j = 0; j < 8; ++j)
                        As[r][c + j] = (m < M && k + j < K) ? A[(long long)m * am + k + j] : zero;
                }
            }
        } else if (a_m_vec) {
            for (int idx = threadIdx.x; idx < BM * TK / 8; idx += GEMM_THREADS) {
                const int c = idx / (BM / 8), r = (idx % (BM / 8)) * 8;
                const int m = m0 + r, k = k0 + c;
                if (k < K && m + 8 <= M) {
                    const uint4 v = *reinterpret_cast<const uint4 *>(A + m + (long long)k * ak);
                    const __nv_bfloat16 *h = reinterpret_cast<const __nv_bfloat16 *>(&v);
                    for (int j = 0; j < 8; ++j) As[r + j][c] = h[j];
                } else {
                    for (int j = 0; j < 8; ++j)
                        As[r + j][c] = (k < K && m + j < M) ? A[m + j + (long long)k * ak] : zero;
                }
            }
        } else {
            for (int idx = threadIdx.x; idx < BM * TK; idx += GEMM_THREADS) {
                const int r = idx / TK, c = idx % TK;
                const int m = m0 + r, k = k0 + c;
                As[r][c] = (m < M && k < K) ? A[(long long)m * am + (long long)k * ak] : zero;
            }
        }
        if (b_k_vec) {
            for (int idx = threadIdx.x; idx < BN * TK / 8; idx += GEMM_THREADS) {
                const int r = idx / (TK / 8), c = (idx % (TK / 8)) * 8;
                const int n = n0 + r, k = k0 + c;
                if (n < N && k + 8 <= K) {
                    *reinterpret_cast<uint4 *>(&Bs[r][c]) =
                        *reinterpret_cast<const uint4 *>(B + k + (long long)n * bn);
                } else {
                    for (int j = 0; j < 8; ++j)
                        Bs[r][c + j] = (n < N && k + j < K) ? B[k + j + (long long)n * bn] : zero;
                }
            }
        } else if (b_n_vec) {
            for (int idx = threadIdx.x; idx < BN * TK / 8; idx += GEMM_THREADS) {
                const int c = idx / (BN / 8), r = (idx % (BN / 8)) * 8;
                const int n = n0 + r, k = k0 + c;
                if (k < K && n + 8 <= N) {
                    const uint4 v = *reinterpret_cast<const uint4 *>(B + (long long)k * bk + n);
                    const __nv_bfloat16 *h = reinterpret_cast<const __nv_bfloat16 *>(&v);
                    for (int j = 0; j < 8; ++j) Bs[r + j][c] = h[j];
                } else {
                    for (int j = 0; j < 8; ++j)
                        Bs[r + j][c] = (k < K && n + j < N) ? B[(long long)k * bk + n + j] : zero;
                }
            }
        } else {
            for (int idx = threadIdx.x; idx < BN * TK; idx += GEMM_THREADS) {
                const int r = idx / TK, c = idx % TK;
                const int n = n0 + r, k = k0 + c;
                Bs[r][c] = (n < N && k < K) ? B[(long long)k * bk + (long long)n * bn] : zero;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; kk += 16) {
            unsigned a[MI][4], b[NJ][2];
#pragma unroll
            for (int i = 0; i < MI; ++i) {
                const int r = wm + 16 * i + g;
                a[i][0] = pack_bf16(As[r][kk + 2 * tg], As[r][kk + 2 * tg + 1]);
                a[i][1] = pack_bf16(As[r + 8][kk + 2 * tg], As[r + 8][kk + 2 * tg + 1]);
                a[i][2] = pack_bf16(As[r][kk + 2 * tg + 8], As[r][kk + 2 * tg + 9]);
                a[i][3] = pack_bf16(As[r + 8][kk + 2 * tg + 8], As[r + 8][kk + 2 * tg + 9]);
            }
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                const int c = wn + 8 * j + g;
                b[j][0] = pack_bf16(Bs[c][kk + 2 * tg], Bs[c][kk + 2 * tg + 1]);
                b[j][1] = pack_bf16(Bs[c][kk + 2 * tg + 8], Bs[c][kk + 2 * tg + 9]);
            }
#pragma unroll
            for (int i = 0; i < MI; ++i)
#pragma unroll
                for (int j = 0; j < NJ; ++j) mma_bf16(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < MI; ++i)
#pragma unroll
        for (int j = 0; j < NJ; ++j)
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int m = m0 + wm + 16 * i + g + (h >= 2 ? 8 : 0);
                const int n = n0 + wn + 8 * j + 2 * tg + (h & 1);
                if (m >= M || n >= N) continue;
                float v = acc[i][j][h] + (bias ? bias[n] : 0.f);
                const long long o = (long long)m * N + n;
                if (pre) pre[o] = v;
                if (epi == EPI_GELU) v = gelu(v);
                if (epi == EPI_GELU_BWD) v = v * gelu_grad(aux[o]);
                if (out) out[o] = v;
                if (outb) outb[o] = __float2bfloat16_rn(v);
            }
}

__global__ void to_bf16(const float *__restrict__ x, __nv_bfloat16 *__restrict__ y, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

// dY = 2 (Y - T) / (B N) (mean squared error), and the loss partial sums.
__global__ void mse_grad(const float *__restrict__ y, const float *__restrict__ t, long long n,
                         float scale, float *__restrict__ dy, __nv_bfloat16 *__restrict__ dyb,
                         double *__restrict__ loss_partials) {
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float d = y[i] - t[i];
        s += (double)(d * d);
        const float gval = 2.0f * d * scale;
        dy[i] = gval;
        dyb[i] = __float2bfloat16_rn(gval);
    }
    double acc[5] = {s, 0.0, 0.0, 0.0, 0.0};
    block_sum5_store(acc, loss_partials + (size_t)blockIdx.x * 5);
}

// db[n] = sum over the batch of dZ[b, n]: a block of 8 warps per 32
// columns, warp w summing rows w, w + 8, ... (lanes on consecutive columns,
// loads independent of the running sums), then the 8 warp sums added in
// warp order: a fixed order, so the result does not vary between runs.
constexpr int BIAS_WARPS = 8;
__global__ void __launch_bounds__(32 * BIAS_WARPS)
bias_grad(const float *__restrict__ dz, int B, int N, float *__restrict__ db) {
    __shared__ float part[BIAS_WARPS][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = blockIdx.x * 32 + lane;
    float s = 0.f;
    if (n < N) {
#pragma unroll 8
        for (int b = warp; b < B; b += BIAS_WARPS) s += dz[(long long)b * N + n];
    }
    part[warp][lane] = s;
    __syncthreads();
    if (warp == 0 && n < N) {
        float t = 0.f;
#pragma unroll
        for (int w = 0; w < BIAS_WARPS; ++w) t += part[w][lane];
        db[n] = t;
    }
}

// One Adam update of parameter i (refreshing its BF16 copy if it is a weight).
__device__ __forceinline__ void adam_update(long long i, float *__restrict__ p,
                                            const float *__restrict__ g, float *__restrict__ m,
                                            float *__restrict__ v, float lr, float b1, float b2,
                                            float eps, float c1, float c2,
                                            const long long *__restrict__ wmap,
                                            __nv_bfloat16 *__restrict__ pb) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float w = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = w;
    if (wmap[i] >= 0) pb[wmap[i]] = __float2bfloat16_rn(w);
}

// Adam on the flat FP32 parameters, refreshing the BF16 copy of every weight.
__global__ void adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                     float *__restrict__ v, long long n, float lr, float b1, float b2, float eps,
                     float c1, float c2, const long long *__restrict__ wmap,
                     __nv_bfloat16 *__restrict__ pb) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        adam_update(i, p, g, m, v, lr, b1, b2, eps, c1, c2, wmap, pb);
}

// Per-step scalars of the device training loop (train_setup writes them).
struct TrainState {
    long long t;          // Adam steps taken so far (all calls)
    long long local;      // steps of this call so far
    long long cur;        // the step being run (this call's numbering)
    float lr, c1, c2;     // learning rate and bias corrections of the step
};

// One thread: the step's learning rate (cosine from lr to lr_final over
// `steps`) and Adam's bias corrections 1 - beta^t, then the counters.
__global__ void train_setup(TrainState *st, long long steps, float lr, float lr_final,
                            float b1, float b2) {
    const long long t = st->t + 1, s = st->local;
    st->cur = s;
    st->lr = (float)((double)lr_final +
                     0.5 * ((double)lr - (double)lr_final) *
                         (1.0 + cos(3.14159265358979323846 * (double)s / (double)steps)));
    st->c1 = 1.f - (float)pow((double)b1, (double)t);     // as lbm_mlp_train_step forms them
    st->c2 = 1.f - (float)pow((double)b2, (double)t);
    st->t = t;
    st->local = s + 1;
}

// SplitMix64 (Steele, Lea and Flood's generator) of a 64-bit counter.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// The step's minibatch: row j is sample (batch >= n ? j : SplitMix64(seed ^
// (step batch + j)) mod n), drawn with replacement; rows of x [n x kx] and
// t [n x kt] are copied to xb and tb.
__global__ void gather_rows(const float *__restrict__ x, const float *__restrict__ t, int n,
                            int kx, int kt, int batch, unsigned long long seed,
                            const TrainState *__restrict__ st, float *__restrict__ xb,
                            float *__restrict__ tb) {
    const int kw = kx > kt ? kx : kt;
    const long long total = (long long)batch * kw;
    const unsigned long long base = (unsigned long long)st->cur * (unsigned long long)batch;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(i / kw), c = (int)(i - (long long)j * kw);
        const long long src = batch >= n ? j
                                         : (long long)(splitmix64(seed ^ (base + (unsigned)j)) %
                                                       (unsigned long long)n);
        if (c < kx) xb[(long long)j * kx + c] = x[src * kx + c];
        if (c < kt) tb[(long long)j * kt + c] = t[src * kt + c];
    }
}

// The step's loss (mean of the squared errors) into the history.
__global__ void record_loss(const double *__restrict__ total, double inv_n,
                            const TrainState *__restrict__ st, float *__restrict__ hist) {
    hist[st->cur] = (float)(*total * inv_n);
}

// Adam with the step's scalars from the device (the training loop).
__global__ void adam_dev(float *__restrict__ p, const float *__restrict__ g,
                         float *__restrict__ m, float *__restrict__ v, long long n, float b1,
                         float b2, float eps, const TrainState *__restrict__ st,
                         const long long *__restrict__ wmap, __nv_bfloat16 *__restrict__ pb) {
    const float lr = st->lr, c1 = st->c1, c2 = st->c2;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        adam_update(i, p, g, m, v, lr, b1, b2, eps, c1, c2, wmap, pb);
}

unsigned grid1(long long n) {
    long long b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

}  // namespace
}  // namespace plbm

using namespace plbm;

struct lbm_mlp {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::vector<int> widths;             // K_0, N_0 = K_1, ..., N_{L-1}
    int layers = 0;
    int max_batch = 0;
    std::vector<long long> w_off, b_off;  // offsets in the flat FP32 parameters
    std::vector<long long> wb_off;        // offsets in the BF16 weight copy
    long long n_params = 0, n_wb = 0;
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *wb = nullptr;          // BF16 weights
    long long *wmap = nullptr;            // flat index -> BF16 index (or -1)
    std::vector<float *> pre;             // pre-activations per layer [B x N_l]
    std::vector<float *> act;             // FP32 outputs per layer
    std::vector<__nv_bfloat16 *> actb;    // BF16 layer inputs: actb[0] = X, actb[l+1] = out of l
    float *g0 = nullptr, *g1 = nullptr;   // gradient ping-pong [B x max width]
    __nv_bfloat16 *gb = nullptr, *gb1 = nullptr;   // BF16 copies of the two
    // device training loop: state, gathered minibatch, capture stream
    TrainState *tstate = nullptr;
    float *xb = nullptr, *tb = nullptr;
    cudaStream_t cap = nullptr;
    double *loss_part = nullptr;
    long long steps = 0;
    std::string err;
};

namespace {

lbm_status mfail(lbm_mlp *m, lbm_status s, const std::string &msg) {
    if (m) m->err = msg;
    else set_global_error(msg.c_str());
    return s;
}

lbm_status mcuda(lbm_mlp *m, cudaError_t e, const char *where) {
    std::string msg = std::string(where) + ": " + cudaGetErrorName(e);
    (void)cudaGetLastError();
    return mfail(m, e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, msg);
}

#define MCK(m, call)                                           \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return mcuda(m, e_, #call);     \
    } while (0)

cudaError_t gemm(cudaStream_t s, const __nv_bfloat16 *A, long long am, long long ak,
                 const __nv_bfloat16 *B, long long bk, long long bn, const float *bias, int M,
                 int N, int K, int epi, const float *aux, float *pre, float *out,
                 __nv_bfloat16 *outb) {
    // 64 x 64 tiles when they give at least two blocks per SM, else 32 x 32
    // (the network's products are small: a few hundred rows and columns)
    const long long big = (long long)((N + 63) / 64) * ((M + 63) / 64);
    if (big >= 2 * 152) {
        dim3 grid((N + 63) / 64, (M + 63) / 64);
        gemm_bf16<64, 64><<<grid, GEMM_THREADS, 0, s>>>(A, am, ak, B, bk, bn, bias, M, N, K,
                                                        epi, aux, pre, out, outb);
    } else {
        dim3 grid((N + 31) / 32, (M + 31) / 32);
        gemm_bf16<32, 32><<<grid, GEMM_THREADS, 0, s>>>(A, am, ak, B, bk, bn, bias, M, N, K,
                                                        epi, aux, pre, out, outb);
    }
    return cudaGetLastError();
}

// Forward pass of `batch` rows of X (FP32 device [batch x K_0]) on stream
// s; the output layer's FP32 result is act[L-1].
cudaError_t forward(lbm_mlp *m, const float *x, int batch, cudaStream_t s) {
    to_bf16<<<grid1((long long)batch * m->widths[0]), 256, 0, s>>>(
        x, m->actb[0], (long long)batch * m->widths[0]);
    cudaError_t e = cudaGetLastError();
    for (int l = 0; l < m->layers && e == cudaSuccess; ++l) {
        const int K = m->widths[l], N = m->widths[l + 1];
        const bool last = l == m->layers - 1;
        e = gemm(s, m->actb[l], K, 1, m->wb + m->wb_off[l], 1, K, m->params + m->b_off[l], batch,
                 N, K, last ? EPI_NONE : EPI_GELU, nullptr, m->pre[l], m->act[l],
                 last ? nullptr : m->actb[l + 1]);
    }
    return e;
}

// Loss partial sums and every parameter's gradient (into m->grads) for
// targets t of the rows forward() last ran, on stream s; no host copy, no
// synchronisation.  The total loss (sum of squares) lands at
// loss_part[5 * 4096].
cudaError_t backward(lbm_mlp *m, const float *t, int batch, cudaStream_t s) {
    const int L = m->layers;
    const long long no = (long long)batch * m->widths[L];
    const unsigned gl = grid1(no);
    mse_grad<<<gl, 256, 0, s>>>(m->act[L - 1], t, no, 1.0f / (float)no, m->g0, m->gb,
                                m->loss_part);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_finalize(m->loss_part, (int)gl, m->loss_part + 5 * 4096, s);
    float *g = m->g0, *gn = m->g1;
    __nv_bfloat16 *gbf = m->gb, *gbn = m->gb1;
    for (int l = L - 1; l >= 0 && e == cudaSuccess; --l) {
        const int K = m->widths[l], N = m->widths[l + 1];
        // dW_l = dZ_l^T X_l   ([N x K], sum over the batch)
        e = gemm(s, gbf, 1, N, m->actb[l], K, 1, nullptr, N, K, batch, EPI_NONE, nullptr,
                 nullptr, m->grads + m->w_off[l], nullptr);
        if (e != cudaSuccess) break;
        bias_grad<<<(N + 31) / 32, 32 * BIAS_WARPS, 0, s>>>(g, batch, N, m->grads + m->b_off[l]);
        e = cudaGetLastError();
        if (l == 0 || e != cudaSuccess) break;
        // dZ_{l-1} = (dZ_l W_l) (.) GELU'(Z_{l-1})   ([B x K], the GELU of
        // layer l - 1 in the product's epilogue)
        e = gemm(s, gbf, N, 1, m->wb + m->wb_off[l], K, 1, nullptr, batch, K, N, EPI_GELU_BWD,
                 m->pre[l - 1], nullptr, gn, gbn);
        std::swap(g, gn);
        std::swap(gbf, gbn);
    }
    return e;
}

}  // namespace

extern "C" {

lbm_status lbm_mlp_create(const int *widths, int n_widths, int max_batch, void *stream,
                          lbm_mlp **out) {
    if (!out) return mfail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!widths || n_widths < 2) return mfail(nullptr, LBM_EINVAL, "need at least 2 widths");
    if (max_batch < 1) return mfail(nullptr, LBM_EINVAL, "max_batch must be >= 1");
    for (int i = 0; i < n_widths; ++i)
        if (widths[i] < 1 || widths[i] > 65536)
            return mfail(nullptr, LBM_EINVAL, "layer widths must be in [1, 65536]");
    lbm_mlp *m = new lbm_mlp();
    cudaGetDevice(&m->device);
    m->stream = (cudaStream_t)stream;
    m->widths.assign(widths, widths + n_widths);
    m->layers = n_widths - 1;
    m->max_batch = max_batch;
    int wmax = 0;
    for (int l = 0; l < m->layers; ++l) {
        const int K = widths[l], N = widths[l + 1];
        m->w_off.push_back(m->n_params);
        m->n_params += (long long)N * K;
        m->b_off.push_back(m->n_params);
        m->n_params += N;
        m->wb_off.push_back(m->n_wb);
        m->n_wb += (long long)N * K;
    }
    for (int i = 0; i < n_widths; ++i) wmax = std::max(wmax, widths[i]);
    cudaError_t e = cudaSuccess;
    auto al = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    al((void **)&m->params, sizeof(float) * m->n_params);
    al((void **)&m->grads, sizeof(float) * m->n_params);
    al((void **)&m->m, sizeof(float) * m->n_params);
    al((void **)&m->v, sizeof(float) * m->n_params);
    al((void **)&m->wb, sizeof(__nv_bfloat16) * m->n_wb);
    al((void **)&m->wmap, sizeof(long long) * m->n_params);
    m->pre.assign(m->layers, nullptr);
    m->act.assign(m->layers, nullptr);
    m->actb.assign(m->layers + 1, nullptr);
    for (int l = 0; l < m->layers; ++l) {
        al((void **)&m->pre[l], sizeof(float) * (size_t)max_batch * widths[l + 1]);
        al((void **)&m->act[l], sizeof(float) * (size_t)max_batch * widths[l + 1]);
    }
    for (int l = 0; l <= m->layers; ++l)
        al((void **)&m->actb[l], sizeof(__nv_bfloat16) * (size_t)max_batch * widths[l]);
    al((void **)&m->g0, sizeof(float) * (size_t)max_batch * wmax);
    al((void **)&m->g1, sizeof(float) * (size_t)max_batch * wmax);
    al((void **)&m->gb, sizeof(__nv_bfloat16) * (size_t)max_batch * wmax);
    al((void **)&m->gb1, sizeof(__nv_bfloat16) * (size_t)max_batch * wmax);
    al((void **)&m->loss_part, sizeof(double) * 5 * 4097);   // partials + total
    if (e == cudaSuccess) {
        std::vector<long long> map(m->n_params, -1);
        for (int l = 0; l < m->layers; ++l) {
            const long long nw = (long long)widths[l] * widths[l + 1];
            for (long long i = 0; i < nw; ++i) map[m->w_off[l] + i] = m->wb_off[l] + i;
        }
        e = cudaMemcpy(m->wmap, map.data(), sizeof(long long) * m->n_params,
                       cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemset(m->params, 0, sizeof(float) * m->n_params);
    if (e == cudaSuccess) e = cudaMemset(m->m, 0, sizeof(float) * m->n_params);
    if (e == cudaSuccess) e = cudaMemset(m->v, 0, sizeof(float) * m->n_params);
    if (e == cudaSuccess) e = cudaMemset(m->wb, 0, sizeof(__nv_bfloat16) * m->n_wb);
    if (e != cudaSuccess) {
        lbm_status s = mcuda(nullptr, e, "lbm_mlp_create");
        lbm_mlp_destroy(m);
        return s;
    }
    *out = m;
    return LBM_OK;
}

void lbm_mlp_destroy(lbm_mlp *m) {
    if (!m) return;
    cudaStreamSynchronize(m->stream);
    cudaFree(m->params);
    cudaFree(m->grads);
    cudaFree(m->m);
    cudaFree(m->v);
    cudaFree(m->wb);
    cudaFree(m->wmap);
    for (auto p : m->pre) cudaFree(p);
    for (auto p : m->act) cudaFree(p);
    for (auto p : m->actb) cudaFree(p);
    cudaFree(m->g0);
    cudaFree(m->g1);
    cudaFree(m->gb);
    cudaFree(m->gb1);
    cudaFree(m->loss_part);
    cudaFree(m->tstate);
    cudaFree(m->xb);
    cudaFree(m->tb);
    if (m->cap) cudaStreamDestroy(m->cap);
    delete m;
}

size_t lbm_mlp_param_count(const lbm_mlp *m) { return m ? (size_t)m->n_params : 0; }

lbm_status lbm_mlp_set_params(lbm_mlp *m, const float *host) {
    if (!m || !host) return mfail(m, LBM_EINVAL, "NULL argument");
    MCK(m, cudaMemcpyAsync(m->params, host, sizeof(float) * m->n_params, cudaMemcpyHostToDevice,
                           m->stream));
    MCK(m, cudaMemsetAsync(m->m, 0, sizeof(float) * m->n_params, m->stream));
    MCK(m, cudaMemsetAsync(m->v, 0, sizeof(float) * m->n_params, m->stream));
    for (int l = 0; l < m->layers; ++l) {
        const long long nw = (long long)m->widths[l] * m->widths[l + 1];
        to_bf16<<<grid1(nw), 256, 0, m->stream>>>(m->params + m->w_off[l], m->wb + m->wb_off[l],
                                                  nw);
        MCK(m, cudaGetLastError());
    }
    m->steps = 0;
    MCK(m, cudaStreamSynchronize(m->stream));
    return LBM_OK;
}

lbm_status lbm_mlp_get_params(lbm_mlp *m, float *host) {
    if (!m || !host) return mfail(m, LBM_EINVAL, "NULL argument");
    MCK(m, cudaMemcpyAsync(host, m->params, sizeof(float) * m->n_params, cudaMemcpyDeviceToHost,
                           m->stream));
    MCK(m, cudaStreamSynchronize(m->stream));
    return LBM_OK;
}

lbm_status lbm_mlp_forward(lbm_mlp *m, const float *x, int batch, float *y) {
    NvtxRange nvtx_("lbm_mlp_forward");
    if (!m || !x || !y) return mfail(m, LBM_EINVAL, "NULL argument");
    if (batch < 1 || batch > m->max_batch) return mfail(m, LBM_EINVAL, "batch out of range");
    MCK(m, forward(m, x, batch, m->stream));
    MCK(m, cudaMemcpyAsync(y, m->act[m->layers - 1],
                           sizeof(float) * (size_t)batch * m->widths[m->layers],
                           cudaMemcpyDeviceToDevice, m->stream));
    return LBM_OK;
}

// Loss and its gradient with respect to every parameter (into m->grads; a
// host copy when grads_host is not NULL).
static lbm_status loss_and_grad(lbm_mlp *m, const float *x, const float *t, int batch,
                                double *loss, float *grads_host) {
    cudaStream_t s = m->stream;
    MCK(m, forward(m, x, batch, s));
    MCK(m, backward(m, t, batch, s));
    const long long no = (long long)batch * m->widths[m->layers];
    double hl = 0.0;
    MCK(m, cudaMemcpyAsync(&hl, m->loss_part + 5 * 4096, sizeof(double), cudaMemcpyDeviceToHost,
                           s));
    if (grads_host)
        MCK(m, cudaMemcpyAsync(grads_host, m->grads, sizeof(float) * m->n_params,
                               cudaMemcpyDeviceToHost, s));
    MCK(m, cudaStreamSynchronize(s));
    if (loss) *loss = hl / (double)no;
    return LBM_OK;
}

lbm_status lbm_mlp_loss_grad(lbm_mlp *m, const float *x, const float *t, int batch,
                             double *loss, float *grads_host) {
    if (!m || !x || !t) return mfail(m, LBM_EINVAL, "NULL argument");
    if (batch < 1 || batch > m->max_batch) return mfail(m, LBM_EINVAL, "batch out of range");
    return loss_and_grad(m, x, t, batch, loss, grads_host);
}

lbm_status lbm_mlp_train_step(lbm_mlp *m, const float *x, const float *t, int batch, float lr,
                              double *loss) {
    NvtxRange nvtx_("lbm_mlp_train_step");
    if (!m || !x || !t) return mfail(m, LBM_EINVAL, "NULL argument");
    if (batch < 1 || batch > m->max_batch) return mfail(m, LBM_EINVAL, "batch out of range");
    if (!(lr > 0.f)) return mfail(m, LBM_EINVAL, "lr must be > 0");
    if (lbm_status s = loss_and_grad(m, x, t, batch, loss, nullptr)) return s;
    m->steps += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - (float)std::pow(b1, (double)m->steps);
    const float c2 = 1.f - (float)std::pow(b2, (double)m->steps);
    adam<<<grid1(m->n_params), 256, 0, m->stream>>>(m->params, m->grads, m->m, m->v, m->n_params,
                                                    lr, b1, b2, 1e-8f, c1, c2, m->wmap, m->wb);
    MCK(m, cudaGetLastError());
    return LBM_OK;
}

lbm_status lbm_mlp_train(lbm_mlp *m, const float *x, const float *t, int n, int batch,
                         long steps, float lr, float lr_final, unsigned long long seed,
                         float *loss_host) {
    NvtxRange nvtx_("lbm_mlp_train");
    if (!m || !x || !t) return mfail(m, LBM_EINVAL, "NULL argument");
    if (n < 1) return mfail(m, LBM_EINVAL, "n must be >= 1");
    if (batch < 1 || batch > m->max_batch) return mfail(m, LBM_EINVAL, "batch out of range");
    if (steps < 0) return mfail(m, LBM_EINVAL, "steps must be >= 0");
    if (!(lr > 0.f) || !(lr_final > 0.f)) return mfail(m, LBM_EINVAL, "learning rates must be > 0");
    if (steps == 0) return LBM_OK;
    const int L = m->layers, kx = m->widths[0], kt = m->widths[L];
    if (!m->tstate) {
        MCK(m, cudaMalloc(&m->tstate, sizeof(TrainState)));
        MCK(m, cudaMalloc(&m->xb, sizeof(float) * (size_t)m->max_batch * kx));
        MCK(m, cudaMalloc(&m->tb, sizeof(float) * (size_t)m->max_batch * kt));
        MCK(m, cudaStreamCreateWithFlags(&m->cap, cudaStreamNonBlocking));
    }
    TrainState st0{m->steps, 0, 0, 0.f, 0.f, 0.f};
    float *hist = nullptr;
    MCK(m, cudaMalloc(&hist, sizeof(float) * (size_t)steps));
    cudaError_t e = cudaMemcpyAsync(m->tstate, &st0, sizeof(st0), cudaMemcpyHostToDevice,
                                    m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    // one Adam step, captured once and replayed: every per-step value (the
    // minibatch, the learning rate, the bias corrections) comes from the
    // device state, so the graph is the same for every step
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    const float b1 = 0.9f, b2 = 0.999f;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(m->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaStream_t s = m->cap;
        cudaError_t le;
        train_setup<<<1, 1, 0, s>>>(m->tstate, (long long)steps, lr, lr_final, b1, b2);
        le = cudaGetLastError();
        if (le == cudaSuccess) {
            gather_rows<<<grid1((long long)batch * (kx > kt ? kx : kt)), 256, 0, s>>>(
                x, t, n, kx, kt, batch, seed, m->tstate, m->xb, m->tb);
            le = cudaGetLastError();
        }
        if (le == cudaSuccess) le = forward(m, m->xb, batch, s);
        if (le == cudaSuccess) le = backward(m, m->tb, batch, s);
        if (le == cudaSuccess) {
            record_loss<<<1, 1, 0, s>>>(m->loss_part + 5 * 4096,
                                        1.0 / ((double)batch * kt), m->tstate, hist);
            le = cudaGetLastError();
        }
        if (le == cudaSuccess) {
            adam_dev<<<grid1(m->n_params), 256, 0, s>>>(m->params, m->grads, m->m, m->v,
                                                        m->n_params, b1, b2, 1e-8f, m->tstate,
                                                        m->wmap, m->wb);
            le = cudaGetLastError();
        }
        e = cudaStreamEndCapture(s, &g);
        if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
    for (long i = 0; i < steps && e == cudaSuccess; ++i) e = cudaGraphLaunch(ge, m->stream);
    if (e == cudaSuccess && loss_host)
        e = cudaMemcpyAsync(loss_host, hist, sizeof(float) * (size_t)steps,
                            cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    cudaFree(hist);
    if (e != cudaSuccess) return mcuda(m, e, "lbm_mlp_train");
    m->steps += steps;
    return LBM_OK;
}

const char *lbm_mlp_last_error(const lbm_mlp *m) { return m ? m->err.c_str() : "mlp is NULL"; }

}  // extern "C"
