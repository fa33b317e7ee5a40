// Learned initial level populations: a 4 -> 128 -> 128 -> 128 -> n_out network (ReLU,
// log-softmax output) mapping four local features of a cell to its log fractional level
// populations, trained on populations the ALI itself converged to.
//
// Kernels:
//   k_features     FP64 features per cell (log n, log T, log |grad v|, log Sobolev tau)
//   k_mlp_tile     one CTA per 64 rows, one warp per 16 rows: the 128-wide layers and the
//                  back-propagated deltas run on the tensor cores (mma.sync m16n8k16, BF16
//                  operands, FP32 accumulation); weight gradients are per-CTA FP32 partial
//                  sums on the CUDA cores, summed over CTAs in a fixed order
//   k_grad_reduce  fixed-order sum of the per-CTA partials
//   k_adam         Adam on FP32 master weights, refreshing the BF16 copies
#include <cuda_bf16.h>
#include <chrono>
#include <cmath>
#include <cstring>
#include <algorithm>
#include <random>
#include <cstdio>
#include <cstring>
#include "common.cuh"

using namespace mg;

namespace {

constexpr int kHid = 128;          // hidden width
constexpr int kIn = 4;           // features
constexpr int kRows = 64;        // rows per CTA
constexpr int kMaxOut = 32;      // padded output width
constexpr float kFracMin = 1e-12f;

struct Layout {
    int n_out, npad;
    // offsets into the flat FP32 parameter vector
    int64_t W1, b1, W2, b2, W3, b3, W4, b4, total;
};

Layout make_layout(int n_out) {
    Layout L{};
    L.n_out = n_out;
    L.npad = n_out <= 16 ? 16 : 32;
    int64_t k = 0;
    L.W1 = k; k += kIn * kHid;
    L.b1 = k; k += kHid;
    L.W2 = k; k += kHid * kHid;
    L.b2 = k; k += kHid;
    L.W3 = k; k += kHid * kHid;
    L.b3 = k; k += kHid;
    L.W4 = k; k += kHid * n_out;
    L.b4 = k; k += n_out;
    L.total = k;
    return L;
}

// BF16 weight copies: forward operands stored [out][in] (WT), backward operands stored
// [in][out] (W), W4 padded to npad outputs with zeros.
struct BfWeights {
    __nv_bfloat16 *W2T, *W3T, *W4T;   // [128][128], [128][128], [npad][128]
    __nv_bfloat16 *W2, *W3, *W4;      // [128][128], [128][128], [128][npad]
};

__device__ __forceinline__ uint32_t ld_u32(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// acc[16 x 8 NT] = A[16 x 16 KT] (bf16, row-major in shared memory, stride lda) times B,
// where B is supplied transposed: BT[n][k] (bf16, row stride ldb). Fragment layouts of
// mma.m16n8k16: lane = 4 g + c holds rows g and g+8, columns 2c, 2c+1 (+8).
template <int KT, int NT>
__device__ __forceinline__ void warp_gemm(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *BT, int ldb,
                                          float (&acc)[NT][4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
#pragma unroll
    for (int nt = 0; nt < NT; nt++) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
    for (int kt = 0; kt < KT; kt++) {
        const uint32_t a0 = ld_u32(A + g * lda + 16 * kt + 2 * c);
        const uint32_t a1 = ld_u32(A + (g + 8) * lda + 16 * kt + 2 * c);
        const uint32_t a2 = ld_u32(A + g * lda + 16 * kt + 8 + 2 * c);
        const uint32_t a3 = ld_u32(A + (g + 8) * lda + 16 * kt + 8 + 2 * c);
#pragma unroll
        for (int nt = 0; nt < NT; nt++) {
            const __nv_bfloat16 *bp = BT + (8 * nt + g) * ldb + 16 * kt + 2 * c;
            mma_bf16(acc[nt], a0, a1, a2, a3, ld_u32(bp), ld_u32(bp + 8));
        }
    }
}

struct TileArgs {
    int64_t rows;
    const float *X;            // [rows][4] raw features
    const int32_t *index;      // optional row permutation
    const float *Y;            // [rows][n_out] target fractions (training) or nullptr
    const float *theta;        // FP32 master (W1, biases)
    BfWeights w;
    Layout L;
    float mean[kIn], istd[kIn];
    float inv_count;           // 1 / number of (row, level) targets >= 1e-12 in the batch
    float *logp;               // [rows][n_out] output (forward) or nullptr
    float *partial;            // [gridDim][L.total + 1] gradient partials and loss (training)
};

// Shared memory per CTA: activations h1, h2, h3 and two delta buffers (bf16), inputs.
struct TileSmem {
    __nv_bfloat16 h1[kRows][kHid], h2[kRows][kHid], h3[kRows][kHid];
    __nv_bfloat16 da[kRows][kHid], db[kRows][kHid];
    __nv_bfloat16 dz[kRows][kMaxOut];
    float x[kRows][kIn];
    float loss[4];
};

// Stores an accumulator block (16 rows of warp w) plus bias into bf16 rows with ReLU.
template <int NT>
__device__ __forceinline__ void store_relu(float (&acc)[NT][4], const float *bias, __nv_bfloat16 (*dst)[kHid], int r0) {
    const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
#pragma unroll
    for (int nt = 0; nt < NT; nt++) {
        const int col = 8 * nt + 2 * c;
        dst[r0 + g][col] = __float2bfloat16(fmaxf(acc[nt][0] + bias[col], 0.f));
        dst[r0 + g][col + 1] = __float2bfloat16(fmaxf(acc[nt][1] + bias[col + 1], 0.f));
        dst[r0 + g + 8][col] = __float2bfloat16(fmaxf(acc[nt][2] + bias[col], 0.f));
        dst[r0 + g + 8][col + 1] = __float2bfloat16(fmaxf(acc[nt][3] + bias[col + 1], 0.f));
    }
}

// Delta through a ReLU layer: dst = acc masked by (h > 0).
template <int NT>
__device__ __forceinline__ void store_masked(float (&acc)[NT][4], __nv_bfloat16 (*h)[kHid], __nv_bfloat16 (*dst)[kHid],
                                             int r0) {
    const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
    const __nv_bfloat16 z = __float2bfloat16(0.f);
#pragma unroll
    for (int nt = 0; nt < NT; nt++) {
        const int col = 8 * nt + 2 * c;
        dst[r0 + g][col] = __bfloat162float(h[r0 + g][col]) > 0.f ? __float2bfloat16(acc[nt][0]) : z;
        dst[r0 + g][col + 1] = __bfloat162float(h[r0 + g][col + 1]) > 0.f ? __float2bfloat16(acc[nt][1]) : z;
        dst[r0 + g + 8][col] = __bfloat162float(h[r0 + g + 8][col]) > 0.f ? __float2bfloat16(acc[nt][2]) : z;
        dst[r0 + g + 8][col + 1] = __bfloat162float(h[r0 + g + 8][col + 1]) > 0.f ? __float2bfloat16(acc[nt][3]) : z;
    }
}

// dW[i][j] += sum_rows a[r][i] d[r][j] for this CTA (CUDA cores, fixed order over rows).
__device__ void weight_grad(const __nv_bfloat16 (*a)[kHid], const __nv_bfloat16 (*d)[kHid], int nrows, int ni, int nj,
                            float *out, const float *bias_out) {
    for (int t = threadIdx.x; t < ni * nj; t += blockDim.x) {
        const int i = t / nj, j = t - (t / nj) * nj;
        float s = 0.f;
        for (int r = 0; r < nrows; r++) s += __bfloat162float(a[r][i]) * __bfloat162float(d[r][j]);
        out[t] = s;
    }
    (void)bias_out;
}

__global__ void __launch_bounds__(128) k_mlp_tile(TileArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileSmem &S = *reinterpret_cast<TileSmem *>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
    const int r0 = warp * 16;
    const int64_t row0 = (int64_t)blockIdx.x * kRows;
    const int n_out = a.L.n_out, npad = a.L.npad;
    const float *th = a.theta;
    // inputs (normalised); rows beyond the end are zero and carry no loss
    for (int t = threadIdx.x; t < kRows * kIn; t += blockDim.x) {
        const int r = t / kIn, i = t - r * kIn;
        const int64_t gr = row0 + r;
        float v = 0.f;
        if (gr < a.rows) {
            const int64_t src = a.index ? a.index[gr] : gr;
            v = (a.X[src * kIn + i] - a.mean[i]) * a.istd[i];
        }
        S.x[r][i] = v;
    }
    __syncthreads();
    // layer 1 (K = 4) on the CUDA cores
    for (int t = threadIdx.x; t < kRows * kHid; t += blockDim.x) {
        const int r = t / kHid, j = t - r * kHid;
        float s = th[a.L.b1 + j];
#pragma unroll
        for (int i = 0; i < kIn; i++) s += S.x[r][i] * th[a.L.W1 + i * kHid + j];
        S.h1[r][j] = __float2bfloat16(fmaxf(s, 0.f));
    }
    __syncthreads();
    {   // layers 2 and 3 on the tensor cores, each warp its own 16 rows
        float acc[16][4];
        warp_gemm<8, 16>(&S.h1[r0][0], kHid, a.w.W2T, kHid, acc);
        store_relu<16>(acc, th + a.L.b2, S.h2, r0);
        __syncwarp();
        warp_gemm<8, 16>(&S.h2[r0][0], kHid, a.w.W3T, kHid, acc);
        store_relu<16>(acc, th + a.L.b3, S.h3, r0);
        __syncwarp();
    }
    // output layer and log-softmax; lanes 4g..4g+3 hold rows r0+g and r0+g+8
    float z[4][4];
    float lp[4][4];
    {
        float acc[4][4];
        if (npad == 16) {
            float a2[2][4];
            warp_gemm<8, 2>(&S.h3[r0][0], kHid, a.w.W4T, kHid, a2);
            for (int nt = 0; nt < 4; nt++)
                for (int k = 0; k < 4; k++) acc[nt][k] = nt < 2 ? a2[nt][k] : 0.f;
        } else {
            warp_gemm<8, 4>(&S.h3[r0][0], kHid, a.w.W4T, kHid, acc);
        }
        float mx[2] = {-INFINITY, -INFINITY};
        for (int nt = 0; nt < 4; nt++)
            for (int k = 0; k < 4; k++) {
                const int col = 8 * nt + 2 * c + (k & 1);
                z[nt][k] = col < n_out ? acc[nt][k] + th[a.L.b4 + col] : -INFINITY;
                mx[k >> 1] = fmaxf(mx[k >> 1], z[nt][k]);
            }
        for (int s = 0; s < 2; s++) {
            mx[s] = fmaxf(mx[s], __shfl_xor_sync(0xffffffffu, mx[s], 1));
            mx[s] = fmaxf(mx[s], __shfl_xor_sync(0xffffffffu, mx[s], 2));
        }
        float se[2] = {0.f, 0.f};
        for (int nt = 0; nt < 4; nt++)
            for (int k = 0; k < 4; k++) se[k >> 1] += (z[nt][k] == -INFINITY) ? 0.f : expf(z[nt][k] - mx[k >> 1]);
        for (int s = 0; s < 2; s++) {
            se[s] += __shfl_xor_sync(0xffffffffu, se[s], 1);
            se[s] += __shfl_xor_sync(0xffffffffu, se[s], 2);
        }
        for (int nt = 0; nt < 4; nt++)
            for (int k = 0; k < 4; k++) lp[nt][k] = z[nt][k] - mx[k >> 1] - logf(se[k >> 1]);
    }
    if (a.logp) {
        for (int nt = 0; nt < 4; nt++)
            for (int k = 0; k < 4; k++) {
                const int col = 8 * nt + 2 * c + (k & 1);
                const int64_t gr = row0 + r0 + g + 8 * (k >> 1);
                if (col < n_out && gr < a.rows) a.logp[gr * n_out + col] = lp[nt][k];
            }
    }
    if (!a.partial) return;
    // ---- training: dL/dlogp, through log-softmax, then back through the layers
    float lsum = 0.f;
    {
        float gsum[2] = {0.f, 0.f};
        float gv[4][4];
        for (int nt = 0; nt < 4; nt++)
            for (int k = 0; k < 4; k++) {
                const int col = 8 * nt + 2 * c + (k & 1);
                const int64_t gr = row0 + r0 + g + 8 * (k >> 1);
                float gg = 0.f;
                if (col < n_out && gr < a.rows) {
                    const int64_t src = a.index ? a.index[gr] : gr;
                    const float y = a.Y[src * n_out + col];
                    if (y >= kFracMin) {
                        const float d = lp[nt][k] - logf(y);
                        lsum += d * d;
                        gg = 2.f * d * a.inv_count;
                    }
                }
                gv[nt][k] = gg;
                gsum[k >> 1] += gg;
            }
        for (int s = 0; s < 2; s++) {
            gsum[s] += __shfl_xor_sync(0xffffffffu, gsum[s], 1);
            gsum[s] += __shfl_xor_sync(0xffffffffu, gsum[s], 2);
        }
        for (int nt = 0; nt < 4; nt++)
            for (int k = 0; k < 4; k++) {
                const int col = 8 * nt + 2 * c + (k & 1);
                const float dzv = col < n_out ? gv[nt][k] - expf(lp[nt][k]) * gsum[k >> 1] : 0.f;
                if (col < npad) S.dz[r0 + g + 8 * (k >> 1)][col] = __float2bfloat16(dzv);
            }
    }
    for (int d = 16; d; d >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, d);
    if (lane == 0) S.loss[warp] = lsum;
    __syncwarp();
    {   // dh3 = (dz W4^T) masked by h3 > 0; B^T is W4 stored [128][npad]
        float acc[16][4];
        if (npad == 16) warp_gemm<1, 16>(&S.dz[r0][0], kMaxOut, a.w.W4, npad, acc);
        else warp_gemm<2, 16>(&S.dz[r0][0], kMaxOut, a.w.W4, npad, acc);
        store_masked<16>(acc, S.h3, S.da, r0);
        __syncwarp();
        warp_gemm<8, 16>(&S.da[r0][0], kHid, a.w.W3, kHid, acc);     // dh2 = dh3 W3^T, masked
        store_masked<16>(acc, S.h2, S.db, r0);
        __syncwarp();
    }
    __syncthreads();
    float *P = a.partial + (size_t)blockIdx.x * (a.L.total + 1);
    // weight gradients of layers 4 and 3 (need dz, h3, dh3 = da, h2)
    {
        for (int t = threadIdx.x; t < kHid * n_out; t += blockDim.x) {
            const int i = t / n_out, j = t - i * n_out;
            float s = 0.f;
            for (int r = 0; r < kRows; r++) s += __bfloat162float(S.h3[r][i]) * __bfloat162float(S.dz[r][j]);
            P[a.L.W4 + t] = s;
        }
        for (int j = threadIdx.x; j < n_out; j += blockDim.x) {
            float s = 0.f;
            for (int r = 0; r < kRows; r++) s += __bfloat162float(S.dz[r][j]);
            P[a.L.b4 + j] = s;
        }
        weight_grad(S.h2, S.da, kRows, kHid, kHid, P + a.L.W3, nullptr);
        for (int j = threadIdx.x; j < kHid; j += blockDim.x) {
            float s = 0.f;
            for (int r = 0; r < kRows; r++) s += __bfloat162float(S.da[r][j]);
            P[a.L.b3 + j] = s;
        }
    }
    __syncthreads();
    {   // dh1 = dh2 W2^T, masked by h1 > 0 (into da, which is free now)
        float acc[16][4];
        warp_gemm<8, 16>(&S.db[r0][0], kHid, a.w.W2, kHid, acc);
        store_masked<16>(acc, S.h1, S.da, r0);
    }
    __syncthreads();
    weight_grad(S.h1, S.db, kRows, kHid, kHid, P + a.L.W2, nullptr);
    for (int j = threadIdx.x; j < kHid; j += blockDim.x) {
        float s = 0.f, s1 = 0.f;
        for (int r = 0; r < kRows; r++) {
            s += __bfloat162float(S.db[r][j]);
            s1 += __bfloat162float(S.da[r][j]);
        }
        P[a.L.b2 + j] = s;
        P[a.L.b1 + j] = s1;
    }
    for (int t = threadIdx.x; t < kIn * kHid; t += blockDim.x) {
        const int i = t / kHid, j = t - i * kHid;
        float s = 0.f;
        for (int r = 0; r < kRows; r++) s += S.x[r][i] * __bfloat162float(S.da[r][j]);
        P[a.L.W1 + t] = s;
    }
    if (threadIdx.x == 0) P[a.L.total] = S.loss[0] + S.loss[1] + S.loss[2] + S.loss[3];
}

__global__ void k_grad_reduce(const float *partial, int nblk, int64_t stride, float *grad, double *loss) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= stride) return;
    double s = 0.0;
    for (int b = 0; b < nblk; b++) s += (double)partial[(size_t)b * stride + t];
    if (t == stride - 1) *loss = s;
    else grad[t] = (float)s;
}

__global__ void k_refresh_bf16(const float *theta, Layout L, BfWeights w) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < kHid * kHid) {
        const int i = t / kHid, j = t - (t / kHid) * kHid;   // W[i][j], i = in, j = out
        w.W2[t] = __float2bfloat16(theta[L.W2 + t]);
        w.W3[t] = __float2bfloat16(theta[L.W3 + t]);
        w.W2T[j * kHid + i] = __float2bfloat16(theta[L.W2 + t]);
        w.W3T[j * kHid + i] = __float2bfloat16(theta[L.W3 + t]);
    }
    if (t < kHid * L.npad) {
        const int i = t / L.npad, j = t - (t / L.npad) * L.npad;
        const float v = j < L.n_out ? theta[L.W4 + i * L.n_out + j] : 0.f;
        w.W4[i * L.npad + j] = __float2bfloat16(v);
        w.W4T[j * kHid + i] = __float2bfloat16(v);
    }
}

__global__ void k_adam(float *theta, float *m, float *v, const float *grad, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float g = grad[t];
    const float mt = b1 * m[t] + (1.f - b1) * g;
    const float vt = b2 * v[t] + (1.f - b2) * g * g;
    m[t] = mt;
    v[t] = vt;
    theta[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
}

// Features per cell (FP64): log10 n_coll, log10 T, log10 |grad v| (least-squares velocity
// gradient over the neighbours, regularised by 1e-6 tr/3), log10 of the Sobolev optical
// depth of line 0 at LTE populations with velocity scale max(|grad v|, b / l), l the mean
// neighbour distance.
__global__ void k_features(int64_t n, const double *pos, const double *vel, const int64_t *off, const int32_t *idx,
                           const double *T, const double *ncoll, const double *nspec, const double *b, int nlev,
                           const double *E, const double *g, LineConst l0, float *out) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    double M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, B[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    double ell = 0.0;
    const int64_t e0 = off[c], e1 = off[c + 1];
    for (int64_t e = e0; e < e1; e++) {
        const int64_t m = idx[e];
        double dx[3], dv[3];
        for (int k = 0; k < 3; k++) {
            dx[k] = pos[3 * m + k] - pos[3 * c + k];
            dv[k] = vel[3 * m + k] - vel[3 * c + k];
        }
        ell += sqrt(dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2]);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                M[i][j] += dx[i] * dx[j];
                B[i][j] += dv[i] * dx[j];
            }
    }
    double gv = 0.0;
    if (e1 > e0) {
        ell /= (double)(e1 - e0);
        const double reg = 1e-6 * (M[0][0] + M[1][1] + M[2][2]) / 3.0;
        for (int i = 0; i < 3; i++) M[i][i] += reg;
        // inverse of the symmetric 3x3 matrix by cofactors
        const double c00 = M[1][1] * M[2][2] - M[1][2] * M[2][1], c01 = M[1][2] * M[2][0] - M[1][0] * M[2][2],
                     c02 = M[1][0] * M[2][1] - M[1][1] * M[2][0];
        const double det = M[0][0] * c00 + M[0][1] * c01 + M[0][2] * c02;
        double Mi[3][3];
        Mi[0][0] = c00 / det; Mi[1][0] = c01 / det; Mi[2][0] = c02 / det;
        Mi[0][1] = (M[0][2] * M[2][1] - M[0][1] * M[2][2]) / det;
        Mi[1][1] = (M[0][0] * M[2][2] - M[0][2] * M[2][0]) / det;
        Mi[2][1] = (M[0][1] * M[2][0] - M[0][0] * M[2][1]) / det;
        Mi[0][2] = (M[0][1] * M[1][2] - M[0][2] * M[1][1]) / det;
        Mi[1][2] = (M[0][2] * M[1][0] - M[0][0] * M[1][2]) / det;
        Mi[2][2] = (M[0][0] * M[1][1] - M[0][1] * M[1][0]) / det;
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                const double G = B[i][0] * Mi[0][j] + B[i][1] * Mi[1][j] + B[i][2] * Mi[2][j];
                gv += G * G;
            }
        gv = sqrt(gv);
    } else {
        ell = 1.0;
    }
    const double ikT = 1.0 / (kKB * T[c]);
    double Z = 0.0;
    for (int i = 0; i < nlev; i++) Z += g[i] * exp(-E[i] * ikT);
    const double nl = nspec[c] * g[l0.lo] * exp(-E[l0.lo] * ikT) / Z;
    const double nu_ = nspec[c] * g[l0.up] * exp(-E[l0.up] * ikT) / Z;
    const double chi_int = l0.pre * (nl * l0.Blu - nu_ * l0.Bul);
    const double vs = fmax(gv, b[c] / ell);
    const double tau = chi_int * kC / (l0.nu * vs);
    out[4 * c + 0] = (float)log10(ncoll[c]);
    out[4 * c + 1] = (float)log10(T[c]);
    out[4 * c + 2] = (float)log10(fmax(gv, 1e-30));
    out[4 * c + 3] = (float)log10(fmax(tau, 1e-30));
}

// Populations n_i = n_species exp(log p_i); a row with a non-finite output keeps LTE.
__global__ void k_pops_from_logp(int64_t n, int nlev, const float *logp, const double *nspec, double *pops,
                                 unsigned long long *bad) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    bool ok = true;
    for (int i = 0; i < nlev; i++) ok = ok && isfinite(logp[c * nlev + i]);
    if (!ok) { atomicAdd(bad, 1ull); return; }
    double s = 0.0;
    for (int i = 0; i < nlev; i++) s += exp((double)logp[c * nlev + i]);
    for (int i = 0; i < nlev; i++) pops[c * nlev + i] = nspec[c] * exp((double)logp[c * nlev + i]) / s;
}

}  // namespace

struct mg_mlp {
    int device = 0;
    cudaStream_t stream = nullptr;
    Layout L{};
    float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    BfWeights w{};
    __nv_bfloat16 *wbuf = nullptr;
    float mean[kIn] = {0, 0, 0, 0}, istd[kIn] = {1, 1, 1, 1};
    int64_t step = 0;
    std::string err;
};

static int mfail(mg_mlp *p, int code, const std::string &msg) {
    if (p) p->err = msg;
    return code;
}

#define M_CUDA(call)                                                                            \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return mfail(p, MG_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

static void refresh(mg_mlp *p) {
    k_refresh_bf16<<<(kHid * kHid + 255) / 256, 256, 0, p->stream>>>(p->theta, p->L, p->w);
}

extern "C" int mg_mlp_create(mg_mlp **out, int32_t n_out, uint64_t seed, int32_t device) {
    if (!out || n_out < 2 || n_out > kMaxOut) return MG_ERR_ARG;
    mg_mlp *p = new mg_mlp();
    p->device = device;
    p->L = make_layout(n_out);
    if (cudaSetDevice(device) != cudaSuccess || cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete p;
        return MG_ERR_CUDA;
    }
    const int64_t T = p->L.total;
    const size_t nbf = 4 * (size_t)kHid * kHid + 2 * (size_t)kHid * kMaxOut;
    if (cudaMalloc(&p->theta, 4 * T) || cudaMalloc(&p->m, 4 * T) || cudaMalloc(&p->v, 4 * T) ||
        cudaMalloc(&p->grad, 4 * T) || cudaMalloc(&p->wbuf, 2 * nbf)) {
        mg_mlp_destroy(p);
        return MG_ERR_OOM;
    }
    p->w.W2T = p->wbuf;
    p->w.W3T = p->w.W2T + kHid * kHid;
    p->w.W2 = p->w.W3T + kHid * kHid;
    p->w.W3 = p->w.W2 + kHid * kHid;
    p->w.W4T = p->w.W3 + kHid * kHid;
    p->w.W4 = p->w.W4T + kHid * kMaxOut;
    // He-uniform initial weights from a seeded generator, zero biases
    std::mt19937_64 rng(seed);
    std::vector<float> th(T, 0.f);
    auto fill = [&](int64_t o, int fan_in, int64_t cnt) {
        std::uniform_real_distribution<double> U(-std::sqrt(6.0 / fan_in), std::sqrt(6.0 / fan_in));
        for (int64_t k = 0; k < cnt; k++) th[o + k] = (float)U(rng);
    };
    fill(p->L.W1, kIn, kIn * kHid);
    fill(p->L.W2, kHid, kHid * kHid);
    fill(p->L.W3, kHid, kHid * kHid);
    fill(p->L.W4, kHid, kHid * n_out);
    cudaMemcpyAsync(p->theta, th.data(), 4 * T, cudaMemcpyHostToDevice, p->stream);
    cudaMemsetAsync(p->m, 0, 4 * T, p->stream);
    cudaMemsetAsync(p->v, 0, 4 * T, p->stream);
    refresh(p);
    if (cudaStreamSynchronize(p->stream) != cudaSuccess) { mg_mlp_destroy(p); return MG_ERR_CUDA; }
    *out = p;
    return MG_OK;
}

extern "C" int mg_mlp_destroy(mg_mlp *p) {
    if (!p) return MG_OK;
    cudaSetDevice(p->device);
    if (p->stream) cudaStreamSynchronize(p->stream);
    cudaFree(p->theta); cudaFree(p->m); cudaFree(p->v); cudaFree(p->grad); cudaFree(p->wbuf);
    if (p->stream) cudaStreamDestroy(p->stream);
    delete p;
    return MG_OK;
}

extern "C" const char *mg_mlp_last_error(const mg_mlp *p) { return p ? p->err.c_str() : "null network"; }

extern "C" int mg_mlp_param_count(const mg_mlp *p, int64_t *count) {
    if (!p || !count) return MG_ERR_ARG;
    *count = p->L.total;
    return MG_OK;
}

extern "C" int mg_mlp_set_params(mg_mlp *p, const float *theta, int64_t count) {
    if (!p || !theta || count != p->L.total) return MG_ERR_ARG;
    cudaSetDevice(p->device);
    M_CUDA(cudaMemcpyAsync(p->theta, theta, 4 * count, cudaMemcpyHostToDevice, p->stream));
    M_CUDA(cudaMemsetAsync(p->m, 0, 4 * count, p->stream));
    M_CUDA(cudaMemsetAsync(p->v, 0, 4 * count, p->stream));
    p->step = 0;
    refresh(p);
    M_CUDA(cudaStreamSynchronize(p->stream));
    return MG_OK;
}

extern "C" int mg_mlp_get_params(const mg_mlp *cp, float *theta, int64_t count) {
    mg_mlp *p = const_cast<mg_mlp *>(cp);
    if (!p || !theta || count != p->L.total) return MG_ERR_ARG;
    cudaSetDevice(p->device);
    M_CUDA(cudaMemcpyAsync(theta, p->theta, 4 * count, cudaMemcpyDeviceToHost, p->stream));
    M_CUDA(cudaStreamSynchronize(p->stream));
    return MG_OK;
}

extern "C" int mg_mlp_set_normalisation(mg_mlp *p, const float *mean, const float *stdv) {
    if (!p || !mean || !stdv) return MG_ERR_ARG;
    for (int i = 0; i < kIn; i++) {
        if (!(stdv[i] > 0)) return mfail(p, MG_ERR_ARG, "normalisation: std must be > 0");
        p->mean[i] = mean[i];
        p->istd[i] = 1.f / stdv[i];
    }
    return MG_OK;
}

static TileArgs tile_args(mg_mlp *p, int64_t rows, const float *X, const int32_t *index, const float *Y, float *logp,
                          float *partial, float inv_count) {
    TileArgs a{};
    a.rows = rows; a.X = X; a.index = index; a.Y = Y; a.theta = p->theta; a.w = p->w; a.L = p->L;
    for (int i = 0; i < kIn; i++) { a.mean[i] = p->mean[i]; a.istd[i] = p->istd[i]; }
    a.inv_count = inv_count; a.logp = logp; a.partial = partial;
    return a;
}

static int launch_tile(mg_mlp *p, const TileArgs &a) {
    const int64_t blocks = (a.rows + kRows - 1) / kRows;
    const size_t sm = sizeof(TileSmem);
    cudaFuncSetAttribute(k_mlp_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_mlp_tile<<<(unsigned)blocks, 128, sm, p->stream>>>(a);
    M_CUDA(cudaGetLastError());
    return MG_OK;
}

// Device-pointer forward pass: X [rows][4] raw features -> logp [rows][n_out].
int mg_mlp_forward_dev(mg_mlp *p, int64_t rows, const float *d_X, float *d_logp, cudaStream_t s) {
    cudaStream_t keep = p->stream;
    p->stream = s;
    int rc = launch_tile(p, tile_args(p, rows, d_X, nullptr, nullptr, d_logp, nullptr, 0.f));
    p->stream = keep;
    return rc;
}

extern "C" int mg_mlp_forward(mg_mlp *p, int64_t rows, const float *X, float *logp) {
    if (!p || rows < 1 || !X || !logp) return MG_ERR_ARG;
    cudaSetDevice(p->device);
    float *dX = nullptr, *dL = nullptr;
    M_CUDA(cudaMalloc(&dX, 16 * rows));
    M_CUDA(cudaMalloc(&dL, 4 * rows * p->L.n_out));
    M_CUDA(cudaMemcpyAsync(dX, X, 16 * rows, cudaMemcpyHostToDevice, p->stream));
    int rc = launch_tile(p, tile_args(p, rows, dX, nullptr, nullptr, dL, nullptr, 0.f));
    if (!rc) {
        M_CUDA(cudaMemcpyAsync(logp, dL, 4 * rows * p->L.n_out, cudaMemcpyDeviceToHost, p->stream));
        M_CUDA(cudaStreamSynchronize(p->stream));
    }
    cudaFree(dX);
    cudaFree(dL);
    return rc;
}

// One gradient evaluation over device rows (index optional); leaves grad in p->grad.
static int grad_dev(mg_mlp *p, int64_t rows, const float *dX, const int32_t *didx, const float *dY, float inv_count,
                    float *dpart, double *dloss) {
    const int64_t blocks = (rows + kRows - 1) / kRows;
    int rc = launch_tile(p, tile_args(p, rows, dX, didx, dY, nullptr, dpart, inv_count));
    if (rc) return rc;
    const int64_t stride = p->L.total + 1;
    k_grad_reduce<<<(unsigned)((stride + 255) / 256), 256, 0, p->stream>>>(dpart, (int)blocks, stride, p->grad, dloss);
    M_CUDA(cudaGetLastError());
    return MG_OK;
}

static float count_inv(const float *Y, int64_t rows, int n_out, const std::vector<int32_t> *idx, int64_t start) {
    int64_t cnt = 0;
    for (int64_t r = 0; r < rows; r++) {
        const int64_t src = idx ? (*idx)[start + r] : start + r;
        for (int j = 0; j < n_out; j++) cnt += Y[src * n_out + j] >= kFracMin;
    }
    return cnt ? 1.f / (float)cnt : 0.f;
}

extern "C" int mg_mlp_loss_grad(mg_mlp *p, int64_t rows, const float *X, const float *Y, double *loss, float *grad) {
    if (!p || rows < 1 || !X || !Y) return MG_ERR_ARG;
    cudaSetDevice(p->device);
    const int n_out = p->L.n_out;
    const int64_t blocks = (rows + kRows - 1) / kRows, stride = p->L.total + 1;
    float *dX = nullptr, *dY = nullptr, *dP = nullptr;
    double *dl = nullptr;
    M_CUDA(cudaMalloc(&dX, 16 * rows));
    M_CUDA(cudaMalloc(&dY, 4 * rows * n_out));
    M_CUDA(cudaMalloc(&dP, 4 * blocks * stride));
    M_CUDA(cudaMalloc(&dl, 8));
    M_CUDA(cudaMemcpyAsync(dX, X, 16 * rows, cudaMemcpyHostToDevice, p->stream));
    M_CUDA(cudaMemcpyAsync(dY, Y, 4 * rows * n_out, cudaMemcpyHostToDevice, p->stream));
    const float ic = count_inv(Y, rows, n_out, nullptr, 0);
    int rc = grad_dev(p, rows, dX, nullptr, dY, ic, dP, dl);
    double lsum = 0.0;
    if (!rc) {
        if (grad) M_CUDA(cudaMemcpyAsync(grad, p->grad, 4 * p->L.total, cudaMemcpyDeviceToHost, p->stream));
        M_CUDA(cudaMemcpyAsync(&lsum, dl, 8, cudaMemcpyDeviceToHost, p->stream));
        M_CUDA(cudaStreamSynchronize(p->stream));
        if (loss) *loss = lsum * ic;
    }
    cudaFree(dX); cudaFree(dY); cudaFree(dP); cudaFree(dl);
    return rc;
}

extern "C" int mg_mlp_train(mg_mlp *p, int64_t rows, const float *X, const float *Y, const mg_train_opts *o,
                            mg_train_report *rep) {
    if (!p || rows < 1 || !X || !Y || !o || o->epochs < 1 || o->batch < kRows || !(o->lr > 0)) return MG_ERR_ARG;
    cudaSetDevice(p->device);
    auto t0 = std::chrono::steady_clock::now();
    const int n_out = p->L.n_out;
    const int64_t B = o->batch, stride = p->L.total + 1, blocks = (B + kRows - 1) / kRows;
    float *dX = nullptr, *dY = nullptr, *dP = nullptr;
    int32_t *dI = nullptr;
    double *dl = nullptr;
    M_CUDA(cudaMalloc(&dX, 16 * rows));
    M_CUDA(cudaMalloc(&dY, 4 * rows * n_out));
    M_CUDA(cudaMalloc(&dI, 4 * rows));
    M_CUDA(cudaMalloc(&dP, 4 * blocks * stride));
    M_CUDA(cudaMalloc(&dl, 8));
    M_CUDA(cudaMemcpyAsync(dX, X, 16 * rows, cudaMemcpyHostToDevice, p->stream));
    M_CUDA(cudaMemcpyAsync(dY, Y, 4 * rows * n_out, cudaMemcpyHostToDevice, p->stream));
    std::vector<int32_t> idx(rows);
    std::mt19937_64 rng(o->seed);
    mg_train_report r{};
    r.first_loss = -1;
    int rc = MG_OK;
    for (int ep = 0; ep < o->epochs && !rc; ep++) {
        for (int64_t i = 0; i < rows; i++) idx[i] = (int32_t)i;
        std::shuffle(idx.begin(), idx.end(), rng);
        M_CUDA(cudaMemcpyAsync(dI, idx.data(), 4 * rows, cudaMemcpyHostToDevice, p->stream));
        double ep_loss = 0.0;
        int64_t nb = 0;
        for (int64_t s = 0; s + B <= rows || (s == 0 && rows < B); s += B) {
            const int64_t nr = std::min<int64_t>(B, rows - s);
            const float ic = count_inv(Y, nr, n_out, &idx, s);
            if ((rc = grad_dev(p, nr, dX, dI + s, dY, ic, dP, dl))) break;
            p->step++;
            const float c1 = 1.f - std::pow(0.9f, (float)p->step), c2 = 1.f - std::pow(0.999f, (float)p->step);
            k_adam<<<(unsigned)((p->L.total + 255) / 256), 256, 0, p->stream>>>(p->theta, p->m, p->v, p->grad,
                                                                                 p->L.total, o->lr, 0.9f, 0.999f,
                                                                                 1e-8f, c1, c2);
            refresh(p);
            double lsum = 0.0;
            cudaMemcpyAsync(&lsum, dl, 8, cudaMemcpyDeviceToHost, p->stream);
            cudaStreamSynchronize(p->stream);
            ep_loss += lsum * ic;
            nb++;
            r.steps++;
        }
        if (nb) {
            if (r.first_loss < 0) r.first_loss = ep_loss / nb;
            r.last_loss = ep_loss / nb;
        }
    }
    cudaFree(dX); cudaFree(dY); cudaFree(dI); cudaFree(dP); cudaFree(dl);
    r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (rep) *rep = r;
    return rc;
}

// ---------------------------------------------------------------- context side
extern "C" int mg_features(mg_ctx *ctx, float *out) {
    if (!ctx || !out) return MG_ERR_ARG;
    if (!ctx->have_mesh || !ctx->have_model || !ctx->have_species)
        return mg_fail(ctx, MG_ERR_STATE, "mg_features: needs mesh, model and species");
    cudaSetDevice(ctx->device);
    float *d = nullptr;
    int rc;
    if ((rc = mg_alloc(ctx, &d, 4 * ctx->n))) return rc;
    k_features<<<(unsigned)((ctx->n + 127) / 128), 128, 0, ctx->stream>>>(
        ctx->n, ctx->d_pos, ctx->d_vel, ctx->d_nbr_off, ctx->d_nbr_idx, ctx->d_T, ctx->d_ncoll, ctx->d_nspec, ctx->d_b,
        ctx->n_lev, ctx->d_E, ctx->d_g, ctx->h_lines[0], d);
    cudaError_t e = cudaMemcpyAsync(out, d, 16 * ctx->n, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(d);
    if (e != cudaSuccess) return mg_cuda_check(ctx, e, "mg_features");
    return MG_OK;
}

extern "C" int mg_init_populations_mlp(mg_ctx *ctx, mg_mlp *p) {
    if (!ctx || !p) return MG_ERR_ARG;
    if (!ctx->have_mesh || !ctx->have_model || !ctx->have_species)
        return mg_fail(ctx, MG_ERR_STATE, "mg_init_populations_mlp: needs mesh, model and species");
    if (p->L.n_out != ctx->n_lev) return mg_fail(ctx, MG_ERR_ARG, "mg_init_populations_mlp: network outputs != levels");
    cudaSetDevice(ctx->device);
    int rc;
    if ((rc = mg_init_populations(ctx, MG_INIT_LTE))) return rc;   // fallback for rows the network cannot give
    float *dF = nullptr, *dL = nullptr;
    if ((rc = mg_alloc(ctx, &dF, 4 * ctx->n))) return rc;
    if ((rc = mg_alloc(ctx, &dL, ctx->n * ctx->n_lev))) {
        cudaFree(dF);
        return rc;
    }
    k_features<<<(unsigned)((ctx->n + 127) / 128), 128, 0, ctx->stream>>>(
        ctx->n, ctx->d_pos, ctx->d_vel, ctx->d_nbr_off, ctx->d_nbr_idx, ctx->d_T, ctx->d_ncoll, ctx->d_nspec, ctx->d_b,
        ctx->n_lev, ctx->d_E, ctx->d_g, ctx->h_lines[0], dF);
    rc = mg_mlp_forward_dev(p, ctx->n, dF, dL, ctx->stream);
    if (!rc) {
        cudaMemsetAsync(ctx->d_scal + 5, 0, 8, ctx->stream);
        k_pops_from_logp<<<(unsigned)((ctx->n + 127) / 128), 128, 0, ctx->stream>>>(ctx->n, ctx->n_lev, dL,
                                                                                   ctx->d_nspec, ctx->d_pops,
                                                                                   ctx->d_scal + 5);
        unsigned long long bad = 0;
        cudaMemcpyAsync(&bad, ctx->d_scal + 5, 8, cudaMemcpyDeviceToHost, ctx->stream);
        cudaStreamSynchronize(ctx->stream);
        ctx->last_fallback = (int64_t)bad;
    }
    cudaFree(dF);
    cudaFree(dL);
    mg_band_restart(ctx);
    ctx->have_pops = true;
    ctx->have_rad = false;
    return rc;
}

extern "C" int mg_attach_mlp(mg_ctx *ctx, mg_mlp *p) {
    if (!ctx) return MG_ERR_ARG;
    if (p && ctx->have_species && p->L.n_out != ctx->n_lev)
        return mg_fail(ctx, MG_ERR_ARG, "mg_attach_mlp: network outputs != levels");
    ctx->mlp = p;
    return MG_OK;
}

// ------------------------------------------------------------------ file format
static const char kMagic[8] = {'M', 'G', 'M', 'L', 'P', '0', '0', '1'};

extern "C" int mg_mlp_save(const mg_mlp *cp, const char *path) {
    mg_mlp *p = const_cast<mg_mlp *>(cp);
    if (!p || !path) return MG_ERR_ARG;
    std::vector<float> th(p->L.total);
    int rc = mg_mlp_get_params(p, th.data(), p->L.total);
    if (rc) return rc;
    FILE *f = std::fopen(path, "wb");
    if (!f) return mfail(p, MG_ERR_ARG, std::string("mg_mlp_save: cannot open ") + path);
    const int32_t hdr[2] = {p->L.n_out, 0};
    const int64_t np = p->L.total;
    float mean[kIn], sd[kIn];
    for (int i = 0; i < kIn; i++) { mean[i] = p->mean[i]; sd[i] = 1.f / p->istd[i]; }
    bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(hdr, 4, 2, f) == 2 && std::fwrite(&np, 8, 1, f) == 1 &&
              std::fwrite(mean, 4, kIn, f) == (size_t)kIn && std::fwrite(sd, 4, kIn, f) == (size_t)kIn &&
              std::fwrite(th.data(), 4, th.size(), f) == th.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? MG_OK : mfail(p, MG_ERR_ARG, std::string("mg_mlp_save: short write to ") + path);
}

extern "C" int mg_mlp_load(mg_mlp **out, const char *path, int32_t device) {
    if (!out || !path) return MG_ERR_ARG;
    *out = nullptr;
    FILE *f = std::fopen(path, "rb");
    if (!f) return MG_ERR_ARG;
    char magic[8];
    int32_t hdr[2];
    int64_t np = 0;
    float mean[kIn], sd[kIn];
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
              std::fread(hdr, 4, 2, f) == 2 && std::fread(&np, 8, 1, f) == 1 &&
              std::fread(mean, 4, kIn, f) == (size_t)kIn && std::fread(sd, 4, kIn, f) == (size_t)kIn &&
              hdr[0] >= 2 && hdr[0] <= kMaxOut && np == make_layout(hdr[0]).total;
    std::vector<float> th(ok ? (size_t)np : 0);
    ok = ok && std::fread(th.data(), 4, th.size(), f) == th.size();
    std::fclose(f);
    if (!ok) return MG_ERR_ARG;
    mg_mlp *p = nullptr;
    int rc = mg_mlp_create(&p, hdr[0], 0, device);
    if (rc) return rc;
    if ((rc = mg_mlp_set_params(p, th.data(), np)) || (rc = mg_mlp_set_normalisation(p, mean, sd))) {
        mg_mlp_destroy(p);
        return rc;
    }
    *out = p;
    return MG_OK;
}
