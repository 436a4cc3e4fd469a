// Learned proposer: BF16 training and inference kernels of the surrogate MLP.
//
// The paper has no learned component.  The network predicts log cycles from
// the size, the hardware and a learned 64-d embedding of the kernel's fitted
// coefficients (layout in klr.h), in one of two output forms: per row (one
// output for a (kernel, N, block shape) row whose features include the
// shape) or per query (one output per block shape for a (kernel, N) row, the
// shape features zero; loss masked to the meaningful shapes).  Dense layers run on the tensor cores through mma.sync m16n8k16
// (BF16 operands, FP32 accumulation) in one tiled GEMM kernel whose operands
// may each be stored transposed, so the forward pass, the input gradients and
// the weight gradients all use it; bias, GELU and the GELU derivative are fused
// into its epilogue.  The width-1 output layer, the loss, bias gradients and
// AdamW are small elementwise or reduction kernels.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "klr_common.cuh"

namespace klr {

namespace {

constexpr int FEAT = 16, EMB = 64, IN = 80, H = 256;
constexpr int64_t kMaxRows = 262144;

struct Offsets {
    int64_t E, W1, b1, W2, b2, W3, b3, W4, b4, total;
};

// n_out: 0 for the per-row output, else the per-query output count
Offsets offsets(int n_coef, int n_out) {
    const int k = n_out > 0 ? n_out : 1;
    Offsets o;
    o.E = 0;
    o.W1 = o.E + (int64_t)EMB * n_coef;
    o.b1 = o.W1 + (int64_t)H * IN;
    o.W2 = o.b1 + H;
    o.b2 = o.W2 + (int64_t)H * H;
    o.W3 = o.b2 + H;
    o.b3 = o.W3 + (int64_t)H * H;
    o.W4 = o.b3 + H;
    o.b4 = o.W4 + (int64_t)k * H;
    o.total = o.b4 + k;
    return o;
}

// outputs per row and the padded row length of their BF16 copy
int out_cols(int n_out) { return n_out > 0 ? n_out : 1; }
int out_ld(int n_out) { return (out_cols(n_out) + 7) & ~7; }

__device__ __forceinline__ float gelu(float z) {
    const float c = 0.7978845608028654f;   // sqrt(2 / pi)
    return 0.5f * z * (1.0f + tanhf(c * (z + 0.044715f * z * z * z)));
}
__device__ __forceinline__ float gelu_grad(float z) {
    const float c = 0.7978845608028654f;
    const float t = tanhf(c * (z + 0.044715f * z * z * z));
    return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * c * (1.0f + 3.0f * 0.044715f * z * z);
}

// ---------------------------------------------------------------------------
// GEMM: C[m][n] = sum_k A(m, k) B(n, k) (+ bias[n]).
// A(m, k) = TA ? A[k * lda + m] : A[m * lda + k]; B(n, k) likewise with TB.
// The contiguous dimension of each stored operand must be a multiple of 8 with
// a leading dimension that is a multiple of 8 and a 16-byte aligned base.
// ---------------------------------------------------------------------------
enum { EPI_F32 = 0, EPI_GELU = 1, EPI_BF16 = 2, EPI_DGELU = 3 };

struct GemmArgs {
    int M, N, K;
    const __nv_bfloat16* A;
    int64_t lda;
    const __nv_bfloat16* B;
    int64_t ldb;
    const float* bias;          // [N] or NULL
    float* C32;                 // EPI_F32 output; EPI_GELU pre-activation (or NULL)
    int64_t ldc32;
    __nv_bfloat16* Cb;          // EPI_GELU activation, EPI_BF16, EPI_DGELU output
    int64_t ldcb;
    const float* Z;             // EPI_DGELU: pre-activation to differentiate
    int64_t ldz;
    int kchunk;                 // K per grid z-slice (split-K, EPI_F32 only)
    float* part;                // split-K slices [z][M][N], summed in z order; NULL: no split
};

constexpr int BM = 128, BN = 64, BK = 32, PADK = 40;

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Load a ROWS x BK tile of operand X(r, k) into S[r][k] (k contiguous).
template <bool T, int ROWS>
__device__ __forceinline__ void load_tile(__nv_bfloat16 (*S)[PADK], const __nv_bfloat16* X,
                                          int64_t ld, int r0, int R, int k0, int K) {
    const uint4 zero = make_uint4(0, 0, 0, 0);
    if (!T) {
        // stored R x K: 8 consecutive k per chunk
        for (int c = threadIdx.x; c < ROWS * BK / 8; c += blockDim.x) {
            const int r = c / (BK / 8), kc = (c % (BK / 8)) * 8;
            const int gr = r0 + r, gk = k0 + kc;
            uint4 v = zero;
            if (gr < R && gk < K) v = *reinterpret_cast<const uint4*>(X + (int64_t)gr * ld + gk);
            *reinterpret_cast<uint4*>(&S[r][kc]) = v;
        }
    } else {
        // stored K x R: 8 consecutive r per chunk, scattered into S
        for (int c = threadIdx.x; c < ROWS * BK / 8; c += blockDim.x) {
            const int kr = c / (ROWS / 8), rc = (c % (ROWS / 8)) * 8;
            const int gk = k0 + kr, gr = r0 + rc;
            uint4 v = zero;
            if (gk < K && gr < R) v = *reinterpret_cast<const uint4*>(X + (int64_t)gk * ld + gr);
            const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
            for (int i = 0; i < 8; ++i) S[rc + i][kr] = e[i];
        }
    }
}

template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(128) gemm_bf16_kernel(const __grid_constant__ GemmArgs g) {
    __shared__ __align__(16) __nv_bfloat16 As[BM][PADK];
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][PADK];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gid = lane >> 2, tig = lane & 3;
    const int wm = (warp >> 1) * 64, wn = (warp & 1) * 32;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    float acc[4][4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
    const int kb = blockIdx.z * g.kchunk;
    const int ke = min(g.K, kb + g.kchunk);
    for (int k0 = kb; k0 < ke; k0 += BK) {
        load_tile<TA, BM>(As, g.A, g.lda, m0, g.M, k0, ke);
        load_tile<TB, BN>(Bs, g.B, g.ldb, n0, g.N, k0, ke);
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[4][4], bf[4][2];
#pragma unroll
            for (int mt = 0; mt < 4; ++mt) {
                const int r = wm + mt * 16 + gid;
                af[mt][0] = *reinterpret_cast<const uint32_t*>(&As[r][kk + 2 * tig]);
                af[mt][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + 2 * tig]);
                af[mt][2] = *reinterpret_cast<const uint32_t*>(&As[r][kk + 8 + 2 * tig]);
                af[mt][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + 8 + 2 * tig]);
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int c = wn + nt * 8 + gid;
                bf[nt][0] = *reinterpret_cast<const uint32_t*>(&Bs[c][kk + 2 * tig]);
                bf[nt][1] = *reinterpret_cast<const uint32_t*>(&Bs[c][kk + 8 + 2 * tig]);
            }
#pragma unroll
            for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], af[mt], bf[nt]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int row = m0 + wm + mt * 16 + gid + h * 8;
                    const int col = n0 + wn + nt * 8 + 2 * tig + j;
                    if (row >= g.M || col >= g.N) continue;
                    float v = acc[mt][nt][h * 2 + j];
                    if (g.bias && blockIdx.z == 0) v += g.bias[col];
                    if (EPI == EPI_F32) {
                        if (gridDim.z > 1)
                            g.part[((int64_t)blockIdx.z * g.M + row) * g.N + col] = v;
                        else
                            g.C32[(int64_t)row * g.ldc32 + col] = v;
                    } else if (EPI == EPI_GELU) {
                        if (g.C32) g.C32[(int64_t)row * g.ldc32 + col] = v;
                        g.Cb[(int64_t)row * g.ldcb + col] = __float2bfloat16(gelu(v));
                    } else if (EPI == EPI_BF16) {
                        g.Cb[(int64_t)row * g.ldcb + col] = __float2bfloat16(v);
                    } else {
                        const float z = g.Z[(int64_t)row * g.ldz + col];
                        g.Cb[(int64_t)row * g.ldcb + col] = __float2bfloat16(v * gelu_grad(z));
                    }
                }
}

// Deterministic reductions.  Every sum over rows (split-K slices, bias
// gradients, the loss) is formed as fixed partial slices and then added in
// slice order, so a training step is bitwise reproducible: no atomics.
constexpr int kSplitSlots = 304;                  // split-K: slices x output tiles
constexpr int kRedBlocks = 152;                   // row-sum partial slices
constexpr int64_t kPartFloats = (int64_t)kSplitSlots * BM * BN;

// out[(i / width) * ldo + i % width] = sum over z in order of part[z * count + i]
__global__ void reduce_slices_kernel(const float* __restrict__ part, int nz, int64_t count,
                                     int width, float* __restrict__ out, int64_t ldo) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int z = 0; z < nz; ++z) acc += part[z * count + i];
        out[(i / width) * ldo + i % width] = acc;
    }
}

// Launch; with EPI_F32, a slice buffer and few output tiles the K range is
// split over grid z and the slices are summed afterwards in z order.
template <bool TA, bool TB, int EPI>
klr_status gemm(const GemmArgs& g_in, cudaStream_t s) {
    if (g_in.M <= 0 || g_in.N <= 0 || g_in.K <= 0) return KLR_OK;
    GemmArgs g = g_in;
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, 1);
    int splits = 1;
    if (EPI == EPI_F32 && g.part) {
        const int tiles = grid.x * grid.y;
        splits = std::max(1, std::min(kSplitSlots / tiles, (g.K + 4 * BK - 1) / (4 * BK)));
    }
    g.kchunk = ((g.K + splits - 1) / splits + BK - 1) / BK * BK;
    grid.z = (g.K + g.kchunk - 1) / g.kchunk;
    gemm_bf16_kernel<TA, TB, EPI><<<grid, 128, 0, s>>>(g);
    KLR_CHECK_CUDA(cudaGetLastError());
    if (grid.z > 1) {
        const int64_t count = (int64_t)g.M * g.N;
        reduce_slices_kernel<<<(int)std::min<int64_t>((count + 255) / 256, 4 * 152), 256, 0, s>>>(
            g.part, (int)grid.z, count, g.N, g.C32, g.ldc32);
        KLR_CHECK_CUDA(cudaGetLastError());
    }
    return KLR_OK;
}

// ---------------------------------------------------------------------------
// Small kernels
// ---------------------------------------------------------------------------
__global__ void cast_bf16_kernel(const float* __restrict__ x, __nv_bfloat16* __restrict__ y,
                                 int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16(x[i]);
}

struct RowArgs {
    int64_t n;
    const int32_t* kernel;
    const int64_t* N;
    const int32_t* cfg_idx;
    const int32_t* cfg;
    const float* coef;
    int n_coef;
    float hw[7];
    __nv_bfloat16* X0;          // n x 80 (features written here)
    __nv_bfloat16* CR;          // n x n_coef gathered coefficients, or NULL
};

// feature block of X0 and the gathered coefficient rows (cfg_idx NULL:
// per-query rows, shape features 0)
__global__ void gather_rows_kernel(const __grid_constant__ RowArgs a) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < a.n;
         r += (int64_t)gridDim.x * blockDim.x) {
        float f[FEAT];
        f[0] = log2f((float)a.N[r]) * (1.0f / 23.0f);
        f[1] = f[2] = f[3] = 0.f;
        if (a.cfg_idx) {
            const int c = a.cfg_idx[r];
            f[1] = log2f((float)a.cfg[3 * c]) * 0.1f;
            f[2] = log2f((float)a.cfg[3 * c + 1]) * 0.1f;
            f[3] = log2f((float)a.cfg[3 * c + 2]) * 0.1f;
        }
        for (int i = 0; i < 7; ++i) f[4 + i] = a.hw[i];
        for (int i = 11; i < FEAT; ++i) f[i] = 0.f;
        for (int i = 0; i < FEAT; ++i) a.X0[r * IN + i] = __float2bfloat16(f[i]);
    }
    if (a.CR) {
        const int64_t total = a.n * a.n_coef;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
             i += (int64_t)gridDim.x * blockDim.x) {
            const int64_t r = i / a.n_coef;
            const int j = (int)(i - r * a.n_coef);
            a.CR[i] = __float2bfloat16(a.coef[(int64_t)a.kernel[r] * a.n_coef + j]);
        }
    }
}

// copy each row's kernel embedding (from a per-kernel table) into X0
__global__ void embed_rows_kernel(const int32_t* __restrict__ kernel, int64_t n,
                                  const __nv_bfloat16* __restrict__ table,
                                  __nv_bfloat16* __restrict__ X0) {
    const int64_t total = n * EMB;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / EMB;
        const int j = (int)(i - r * EMB);
        X0[r * IN + FEAT + j] = table[(int64_t)kernel[r] * EMB + j];
    }
}

// pred[r] = a3[r] . w4 + b4, one warp per row
__global__ void last_forward_kernel(const __nv_bfloat16* __restrict__ A3,
                                    const __nv_bfloat16* __restrict__ w4, const float* b4,
                                    int64_t n, float* __restrict__ pred) {
    const int lane = threadIdx.x & 31;
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < n;
         r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        float s = 0.f;
        for (int h = lane; h < H; h += 32)
            s += __bfloat162float(A3[r * H + h]) * __bfloat162float(w4[h]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) pred[r] = s + b4[0];
    }
}

// Sum over the block in a fixed order (warp trees, then warp sums in order);
// the result is valid in thread 0.
__device__ float block_sum(float v) {
    __shared__ float wsum[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
    __syncthreads();
    float r = 0.f;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += wsum[i];
    __syncthreads();
    return r;
}

// dpred = 2 (pred - target) / n; part[block] = this block's share of
// sum (pred - target)^2 / n (the loss is the in-order sum of the slices)
__global__ void loss_kernel(const float* __restrict__ pred, const float* __restrict__ target,
                            int64_t n, float* __restrict__ dpred, float* __restrict__ part) {
    float acc = 0.f;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const float d = pred[r] - target[r];
        dpred[r] = 2.0f * d / (float)n;
        acc += d * d / (float)n;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// dZ3[r][h] = dpred[r] w4[h] gelu'(Z3[r][h])
__global__ void last_backward_kernel(const float* __restrict__ dpred,
                                     const __nv_bfloat16* __restrict__ w4,
                                     const float* __restrict__ Z3, int64_t n,
                                     __nv_bfloat16* __restrict__ dZ3) {
    const int64_t total = n * H;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / H;
        const int h = (int)(i - r * H);
        dZ3[i] = __float2bfloat16(dpred[r] * __bfloat162float(w4[h]) * gelu_grad(Z3[i]));
    }
}

__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f32(float v) { return v; }

// part[block][h] = sum_r w[r] X[r][h] (w NULL: 1) over block's contiguous
// chunk of ceil(n / gridDim.x) rows
template <typename T>
__global__ void colsum_kernel(const T* __restrict__ X, const float* __restrict__ w, int64_t n,
                              int width, float* __restrict__ part) {
    const int64_t rows_per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = blockIdx.x * rows_per;
    const int64_t r1 = r0 + rows_per < n ? r0 + rows_per : n;
    for (int h = threadIdx.x; h < width; h += blockDim.x) {
        float s = 0.f;
        for (int64_t r = r0; r < r1; ++r) s += (w ? w[r] : 1.0f) * to_f32(X[r * width + h]);
        part[(int64_t)blockIdx.x * width + h] = s;
    }
}

// per-query head: part[block] = this block's count of finite targets
__global__ void count_finite_kernel(const float* __restrict__ target, int64_t total,
                                    float* __restrict__ part) {
    float acc = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x)
        acc += isfinite(target[i]) ? 1.0f : 0.0f;
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// per-query head: with V = *count finite targets, dpred = 2 (pred - t) / V
// where t is finite (else 0), part[block] = the block's share of the loss
__global__ void masked_loss_kernel(const float* __restrict__ pred, const float* __restrict__ target,
                                   int64_t total, const float* __restrict__ count,
                                   float* __restrict__ dpred, float* __restrict__ part) {
    const float inv = 1.0f / fmaxf(*count, 1.0f);
    float acc = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float t = target[i];
        const float d = isfinite(t) ? pred[i] - t : 0.f;
        dpred[i] = 2.0f * d * inv;
        acc += d * d * inv;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// BF16 copy of an n x cols FP32 matrix with rows padded to ld (pads zero)
__global__ void pad_bf16_kernel(const float* __restrict__ x, int64_t n, int cols, int ld,
                                __nv_bfloat16* __restrict__ y) {
    const int64_t total = n * ld;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / ld;
        const int c = (int)(i - r * ld);
        y[i] = __float2bfloat16(c < cols ? x[r * cols + c] : 0.f);
    }
}

// part[block] = this block's grid-stride share of sum_r x[r]
__global__ void sum_kernel(const float* __restrict__ x, int64_t n, float* __restrict__ part) {
    float acc = 0.f;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x)
        acc += x[r];
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

int red_blocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, kRedBlocks)); }

// out[0..width) = sum over rows of w[r] X[r][:] (deterministic)
template <typename T>
void colsum(const T* X, const float* w, int64_t n, int width, float* part, float* out,
            cudaStream_t s) {
    const int nb = red_blocks(n);
    colsum_kernel<T><<<nb, 256, 0, s>>>(X, w, n, width, part);
    reduce_slices_kernel<<<1, 256, 0, s>>>(part, nb, width, width, out, 0);
}

// out[0] = sum over rows of x[r] (deterministic)
void rowsum(const float* x, int64_t n, float* part, float* out, cudaStream_t s) {
    const int nb = red_blocks(n);
    sum_kernel<<<nb, 256, 0, s>>>(x, n, part);
    reduce_slices_kernel<<<1, 32, 0, s>>>(part, nb, 1, 1, out, 0);
}

__global__ void adamw_kernel(float* __restrict__ p, const float* __restrict__ g,
                             float* __restrict__ m, float* __restrict__ v, int64_t n, float lr,
                             float wd, float c1, float c2) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float mh = mi / c1, vh = vi / c2;
        p[i] -= lr * (mh / (sqrtf(vh) + eps) + wd * p[i]);
    }
}

// ---------------------------------------------------------------------------
// Workspace of one batch
// ---------------------------------------------------------------------------
struct MlpWs {
    __nv_bfloat16 *pb, *X0, *CR, *A1, *A2, *A3, *dZa, *dZb, *dE, *emb_table, *dpb;
    float *Z1, *Z2, *Z3, *pred, *dpred, *grads, *loss, *part, *count;
};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t mlp_ws_bytes(int64_t n, int n_coef, int n_out, int64_t n_kernels_table, bool train) {
    const Offsets o = offsets(n_coef, n_out);
    const size_t oc = (size_t)out_cols(n_out);
    size_t b = 0;
    b += align256(2 * (size_t)o.total);                       // pb
    b += align256(2 * (size_t)n * IN);                        // X0
    b += align256(2 * (size_t)n * H) * 3;                     // A1..A3
    b += align256(4 * (size_t)n * oc) * 2;                    // pred, dpred
    b += align256(2 * (size_t)n_kernels_table * EMB);         // emb table
    if (train) {
        b += align256(2 * (size_t)n * n_coef);                // CR
        b += align256(4 * (size_t)n * H) * 3;                 // Z1..Z3
        b += align256(2 * (size_t)n * H) * 2;                 // dZa, dZb
        b += align256(2 * (size_t)n * EMB);                   // dE (embedding grads)
        b += align256(4 * (size_t)o.total);                   // grads
        b += 256;                                              // loss
        b += align256(4 * (size_t)kPartFloats);               // reduction slices
        b += 256;                                              // count
        b += align256(2 * (size_t)n * out_ld(n_out));         // dpb
    }
    return b;
}

MlpWs carve(void* base, int64_t n, int n_coef, int n_out, int64_t n_kernels_table, bool train) {
    const Offsets o = offsets(n_coef, n_out);
    const size_t oc = (size_t)out_cols(n_out);
    char* p = reinterpret_cast<char*>(base);
    auto take = [&](size_t bytes) { char* q = p; p += align256(bytes); return q; };
    MlpWs w{};
    w.pb = reinterpret_cast<__nv_bfloat16*>(take(2 * (size_t)o.total));
    w.X0 = reinterpret_cast<__nv_bfloat16*>(take(2 * (size_t)n * IN));
    w.A1 = reinterpret_cast<__nv_bfloat16*>(take(2 * (size_t)n * H));
    w.A2 = reinterpret_cast<__nv_bfloat16*>(take(2 * (size_t)n * H));
    w.A3 = reinterpret_cast<__nv_bfloat16*>(take(2 * (size_t)n * H));
    w.pred = reinterpret_cast<float*>(take(4 * (size_t)n * oc));
    w.dpred = reinterpret_cast<float*>(take(4 * (size_t)n * oc));
    w.emb_table = reinterpret_cast<__nv_bfloat16*>(take(2 * (size_t)n_kernels_table * EMB));
    if (train) {
        w.CR = reinterpret_cast<__nv_bfloat16*>(take(2 * (size_t)n * n_coef));
        w.Z1 = reinterpret_cast<float*>(take(4 * (size_t)n * H));
        w.Z2 = reinterpret_cast<float*>(take(4 * (size_t)n * H));
        w.Z3 = reinterpret_cast<float*>(take(4 * (size_t)n * H));
        w.dZa = reinterpret_cast<__nv_bfloat16*>(take(2 * (size_t)n * H));
        w.dZb = reinterpret_cast<__nv_bfloat16*>(take(2 * (size_t)n * H));
        w.dE = reinterpret_cast<__nv_bfloat16*>(take(2 * (size_t)n * EMB));
        w.grads = reinterpret_cast<float*>(take(4 * (size_t)o.total));
        w.loss = reinterpret_cast<float*>(take(256));
        w.part = reinterpret_cast<float*>(take(4 * (size_t)kPartFloats));
        w.count = reinterpret_cast<float*>(take(256));
        w.dpb = reinterpret_cast<__nv_bfloat16*>(take(2 * (size_t)n * out_ld(n_out)));
    }
    return w;
}

int blocks_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

// Forward of the three hidden layers and the output for rows whose X0 is set
// (pred: n values per row, or n x n_out for the per-query head).
klr_status forward_hidden(const MlpWs& w, const float* params, const Offsets& o, int n_out,
                          int64_t n, bool keep_z, cudaStream_t s) {
    klr_status st;
    GemmArgs g{};
    g.M = (int)n;
    g.N = H;
    g.K = IN;
    g.A = w.X0;
    g.lda = IN;
    g.B = w.pb + o.W1;
    g.ldb = IN;
    g.bias = params + o.b1;
    g.C32 = keep_z ? w.Z1 : nullptr;
    g.ldc32 = H;
    g.Cb = w.A1;
    g.ldcb = H;
    if ((st = gemm<false, false, EPI_GELU>(g, s)) != KLR_OK) return st;
    g.K = H;
    g.A = w.A1;
    g.lda = H;
    g.B = w.pb + o.W2;
    g.ldb = H;
    g.bias = params + o.b2;
    g.C32 = keep_z ? w.Z2 : nullptr;
    g.Cb = w.A2;
    if ((st = gemm<false, false, EPI_GELU>(g, s)) != KLR_OK) return st;
    g.A = w.A2;
    g.B = w.pb + o.W3;
    g.bias = params + o.b3;
    g.C32 = keep_z ? w.Z3 : nullptr;
    g.Cb = w.A3;
    if ((st = gemm<false, false, EPI_GELU>(g, s)) != KLR_OK) return st;
    if (n_out > 0) {
        // pred = A3 W4^T + b4 on the tensor cores
        GemmArgs go{};
        go.M = (int)n;
        go.N = n_out;
        go.K = H;
        go.A = w.A3;
        go.lda = H;
        go.B = w.pb + o.W4;
        go.ldb = H;
        go.bias = params + o.b4;
        go.C32 = w.pred;
        go.ldc32 = n_out;
        return gemm<false, false, EPI_F32>(go, s);
    }
    last_forward_kernel<<<blocks_for(n * 32, 256), 256, 0, s>>>(w.A3, w.pb + o.W4, params + o.b4,
                                                                n, w.pred);
    KLR_CHECK_CUDA(cudaGetLastError());
    return KLR_OK;
}

klr_status check_net(const klr_mlp* net) {
    KLR_REQUIRE(net && net->params, "NULL network or parameters");
    KLR_REQUIRE(net->n_coef > 0 && net->n_coef % 8 == 0 && net->n_coef <= 4096,
                "n_coef %d must be a positive multiple of 8", net->n_coef);
    KLR_REQUIRE(net->n_out >= 0 && net->n_out <= 256, "n_out %d not in 0..256", net->n_out);
    return KLR_OK;
}

klr_status check_rows(const klr_mlp_rows* rows, bool need_target, bool per_query) {
    KLR_REQUIRE(rows, "NULL rows");
    KLR_REQUIRE(rows->n >= 0 && rows->n <= kMaxRows, "rows n %lld not in 0..%lld",
                (long long)rows->n, (long long)kMaxRows);
    if (rows->n > 0)
        KLR_REQUIRE(rows->kernel && rows->N && (per_query || rows->cfg_idx) &&
                        (!need_target || rows->target),
                    "NULL row array");
    return KLR_OK;
}

}  // namespace

}  // namespace klr

using namespace klr;

extern "C" {

int64_t klr_mlp_param_count(int32_t n_coef, int32_t n_out) {
    if (n_coef <= 0 || n_out < 0 || n_out > 256) return 0;
    return offsets(n_coef, n_out).total;
}

klr_status klr_mlp_train_step(klr_ctx* ctx, klr_mlp* net, const float* coef, const int32_t* cfg,
                              int n_cfg, const klr_mlp_rows* rows, float lr, float weight_decay,
                              int apply_update, float* loss_out, float* grads_out,
                              void* stream_) {
    KLR_REQUIRE(ctx, "klr_mlp_train_step: NULL context");
    klr_status st = check_net(net);
    if (st != KLR_OK) return st;
    const int no = net->n_out;
    if ((st = check_rows(rows, true, no > 0)) != KLR_OK) return st;
    KLR_REQUIRE(net->adam_m && net->adam_v, "klr_mlp_train_step: NULL optimiser state");
    KLR_REQUIRE(coef && cfg && n_cfg > 0, "klr_mlp_train_step: NULL coef or cfg");
    KLR_REQUIRE(std::isfinite(lr) && lr >= 0 && std::isfinite(weight_decay) && weight_decay >= 0,
                "klr_mlp_train_step: bad lr or weight decay");
    Context* c = reinterpret_cast<Context*>(ctx);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    const int64_t n = rows->n;
    if (n == 0) return KLR_OK;
    KLR_CHECK_CUDA(cudaSetDevice(c->device));
    const int nc = net->n_coef;
    const Offsets o = offsets(nc, no);
    if ((st = ensure_workspace(c, mlp_ws_bytes(n, nc, no, 0, true), s)) != KLR_OK) return st;
    const MlpWs w = carve(c->ws, n, nc, no, 0, true);
    KLR_CHECK_CUDA(cudaMemsetAsync(w.grads, 0, 4 * (size_t)o.total, s));
    KLR_CHECK_CUDA(cudaMemsetAsync(w.loss, 0, sizeof(float), s));
    cast_bf16_kernel<<<blocks_for(o.total, 256), 256, 0, s>>>(net->params, w.pb, o.total);
    RowArgs ra{};
    ra.n = n;
    ra.kernel = rows->kernel;
    ra.N = rows->N;
    ra.cfg_idx = no > 0 ? nullptr : rows->cfg_idx;
    ra.cfg = cfg;
    ra.coef = coef;
    ra.n_coef = nc;
    for (int i = 0; i < 7; ++i) ra.hw[i] = net->hw_feat[i];
    ra.X0 = w.X0;
    ra.CR = w.CR;
    gather_rows_kernel<<<blocks_for(n * nc, 256), 256, 0, s>>>(ra);
    KLR_CHECK_CUDA(cudaGetLastError());
    // embedding: X0[:, 16:80] = CR E^T
    GemmArgs g{};
    g.M = (int)n;
    g.N = EMB;
    g.K = nc;
    g.A = w.CR;
    g.lda = nc;
    g.B = w.pb + o.E;
    g.ldb = nc;
    g.Cb = w.X0 + FEAT;
    g.ldcb = IN;
    if ((st = gemm<false, false, EPI_BF16>(g, s)) != KLR_OK) return st;
    if ((st = forward_hidden(w, net->params, o, no, n, true, s)) != KLR_OK) return st;
    if (no > 0) {
        // per-query head: masked loss over the finite targets
        const int64_t total = n * no;
        const int nb = red_blocks(total);
        count_finite_kernel<<<nb, 256, 0, s>>>(rows->target, total, w.part);
        reduce_slices_kernel<<<1, 32, 0, s>>>(w.part, nb, 1, 1, w.count, 0);
        masked_loss_kernel<<<nb, 256, 0, s>>>(w.pred, rows->target, total, w.count, w.dpred,
                                              w.part);
        reduce_slices_kernel<<<1, 32, 0, s>>>(w.part, nb, 1, 1, w.loss, 0);
        const int ld = out_ld(no);
        pad_bf16_kernel<<<blocks_for(n * ld, 256), 256, 0, s>>>(w.dpred, n, no, ld, w.dpb);
        KLR_CHECK_CUDA(cudaGetLastError());
        // output layer: dW4 = dpred^T A3, db4, dZ3 = (dpred W4) * gelu'(Z3)
        GemmArgs g4{};
        g4.M = no;
        g4.N = H;
        g4.K = (int)n;
        g4.A = w.dpb;
        g4.lda = ld;
        g4.B = w.A3;
        g4.ldb = H;
        g4.C32 = w.grads + o.W4;
        g4.ldc32 = H;
        g4.part = w.part;
        if ((st = gemm<true, true, EPI_F32>(g4, s)) != KLR_OK) return st;
        colsum<float>(w.dpred, nullptr, n, no, w.part, w.grads + o.b4, s);
        GemmArgs gz{};
        gz.M = (int)n;
        gz.N = H;
        gz.K = no;
        gz.A = w.dpb;
        gz.lda = ld;
        gz.B = w.pb + o.W4;
        gz.ldb = H;
        gz.Cb = w.dZa;
        gz.ldcb = H;
        gz.Z = w.Z3;
        gz.ldz = H;
        if ((st = gemm<false, true, EPI_DGELU>(gz, s)) != KLR_OK) return st;
    } else {
        const int nb = red_blocks(n);
        loss_kernel<<<nb, 256, 0, s>>>(w.pred, rows->target, n, w.dpred, w.part);
        reduce_slices_kernel<<<1, 32, 0, s>>>(w.part, nb, 1, 1, w.loss, 0);
        // output layer
        colsum(w.A3, w.dpred, n, H, w.part, w.grads + o.W4, s);
        rowsum(w.dpred, n, w.part, w.grads + o.b4, s);
        last_backward_kernel<<<blocks_for(n * H, 256), 256, 0, s>>>(w.dpred, w.pb + o.W4, w.Z3, n,
                                                                   w.dZa);
        KLR_CHECK_CUDA(cudaGetLastError());
    }
    // layer 3: dW3 = dZ3^T A2, db3, dZ2 = (dZ3 W3) * gelu'(Z2)
    GemmArgs gw{};
    gw.M = H;
    gw.N = H;
    gw.K = (int)n;
    gw.A = w.dZa;
    gw.lda = H;
    gw.B = w.A2;
    gw.ldb = H;
    gw.C32 = w.grads + o.W3;
    gw.ldc32 = H;
    gw.part = w.part;
    if ((st = gemm<true, true, EPI_F32>(gw, s)) != KLR_OK) return st;
    colsum(w.dZa, nullptr, n, H, w.part, w.grads + o.b3, s);
    GemmArgs gx{};
    gx.M = (int)n;
    gx.N = H;
    gx.K = H;
    gx.A = w.dZa;
    gx.lda = H;
    gx.B = w.pb + o.W3;
    gx.ldb = H;
    gx.Cb = w.dZb;
    gx.ldcb = H;
    gx.Z = w.Z2;
    gx.ldz = H;
    if ((st = gemm<false, true, EPI_DGELU>(gx, s)) != KLR_OK) return st;
    // layer 2
    gw.A = w.dZb;
    gw.B = w.A1;
    gw.C32 = w.grads + o.W2;
    if ((st = gemm<true, true, EPI_F32>(gw, s)) != KLR_OK) return st;
    colsum(w.dZb, nullptr, n, H, w.part, w.grads + o.b2, s);
    gx.A = w.dZb;
    gx.B = w.pb + o.W2;
    gx.Cb = w.dZa;
    gx.Z = w.Z1;
    if ((st = gemm<false, true, EPI_DGELU>(gx, s)) != KLR_OK) return st;
    // layer 1: dW1 = dZ1^T X0, db1, dEmb = dZ1 W1[:, 16:80]
    gw.N = IN;
    gw.A = w.dZa;
    gw.B = w.X0;
    gw.ldb = IN;
    gw.C32 = w.grads + o.W1;
    gw.ldc32 = IN;
    if ((st = gemm<true, true, EPI_F32>(gw, s)) != KLR_OK) return st;
    colsum(w.dZa, nullptr, n, H, w.part, w.grads + o.b1, s);
    GemmArgs ge{};
    ge.M = (int)n;
    ge.N = EMB;
    ge.K = H;
    ge.A = w.dZa;
    ge.lda = H;
    ge.B = w.pb + o.W1 + FEAT;
    ge.ldb = IN;
    ge.Cb = w.dE;
    ge.ldcb = EMB;
    if ((st = gemm<false, true, EPI_BF16>(ge, s)) != KLR_OK) return st;
    // dE = dEmb^T CR
    GemmArgs gE{};
    gE.M = EMB;
    gE.N = nc;
    gE.K = (int)n;
    gE.A = w.dE;
    gE.lda = EMB;
    gE.B = w.CR;
    gE.ldb = nc;
    gE.C32 = w.grads + o.E;
    gE.ldc32 = nc;
    gE.part = w.part;
    if ((st = gemm<true, true, EPI_F32>(gE, s)) != KLR_OK) return st;
    if (grads_out)
        KLR_CHECK_CUDA(cudaMemcpyAsync(grads_out, w.grads, 4 * (size_t)o.total,
                                       cudaMemcpyDeviceToDevice, s));
    if (loss_out)
        KLR_CHECK_CUDA(cudaMemcpyAsync(loss_out, w.loss, sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (apply_update) {
        net->step += 1;
        const float c1 = 1.0f - powf(0.9f, (float)net->step);
        const float c2 = 1.0f - powf(0.999f, (float)net->step);
        adamw_kernel<<<blocks_for(o.total, 256), 256, 0, s>>>(net->params, w.grads, net->adam_m,
                                                              net->adam_v, o.total, lr,
                                                              weight_decay, c1, c2);
        KLR_CHECK_CUDA(cudaGetLastError());
    }
    return KLR_OK;
}

klr_status klr_mlp_predict(klr_ctx* ctx, const klr_mlp* net, const float* coef, const int32_t* cfg,
                           int n_cfg, const klr_mlp_rows* rows, float* pred_out, void* stream_) {
    KLR_REQUIRE(ctx, "klr_mlp_predict: NULL context");
    klr_status st = check_net(net);
    if (st != KLR_OK) return st;
    const int no = net->n_out;
    if ((st = check_rows(rows, false, no > 0)) != KLR_OK) return st;
    KLR_REQUIRE(coef && cfg && n_cfg > 0 && (rows->n == 0 || pred_out),
                "klr_mlp_predict: NULL coef, cfg or output");
    Context* c = reinterpret_cast<Context*>(ctx);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    const int64_t n = rows->n;
    if (n == 0) return KLR_OK;
    KLR_CHECK_CUDA(cudaSetDevice(c->device));
    const int nc = net->n_coef;
    const Offsets o = offsets(nc, no);
    // rows carry their own coefficient gather and embedding GEMM
    const size_t extra = align256(2 * (size_t)n * nc);
    const size_t base = mlp_ws_bytes(n, nc, no, 0, false);
    if ((st = ensure_workspace(c, base + extra, s)) != KLR_OK) return st;
    MlpWs w = carve(c->ws, n, nc, no, 0, false);
    w.CR = reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<char*>(c->ws) + base);
    cast_bf16_kernel<<<blocks_for(o.total, 256), 256, 0, s>>>(net->params, w.pb, o.total);
    RowArgs ra{};
    ra.n = n;
    ra.kernel = rows->kernel;
    ra.N = rows->N;
    ra.cfg_idx = no > 0 ? nullptr : rows->cfg_idx;
    ra.cfg = cfg;
    ra.coef = coef;
    ra.n_coef = nc;
    for (int i = 0; i < 7; ++i) ra.hw[i] = net->hw_feat[i];
    ra.X0 = w.X0;
    ra.CR = w.CR;
    gather_rows_kernel<<<blocks_for(n * nc, 256), 256, 0, s>>>(ra);
    GemmArgs g{};
    g.M = (int)n;
    g.N = EMB;
    g.K = nc;
    g.A = w.CR;
    g.lda = nc;
    g.B = w.pb + o.E;
    g.ldb = nc;
    g.Cb = w.X0 + FEAT;
    g.ldcb = IN;
    if ((st = gemm<false, false, EPI_BF16>(g, s)) != KLR_OK) return st;
    if ((st = forward_hidden(w, net->params, o, no, n, false, s)) != KLR_OK) return st;
    KLR_CHECK_CUDA(cudaMemcpyAsync(pred_out, w.pred, 4 * (size_t)n * out_cols(no),
                                   cudaMemcpyDeviceToDevice, s));
    return KLR_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Training targets from a cycles table: per-query centred log2 cycles.
// ---------------------------------------------------------------------------
namespace klr {
namespace {

// one warp per query row: out = log2(cycles) - mean over the row's finite
// positive entries of log2(cycles); NaN where the entry is not finite or not
// positive (a shape that is not meaningful)
__global__ void query_targets_kernel(const float* __restrict__ cyc, int64_t n_rows, int n_cfg,
                                     float* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < n_rows;
         r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const float* row = cyc + r * n_cfg;
        float sum = 0.f, cnt = 0.f;
        for (int c = lane; c < n_cfg; c += 32) {
            const float v = row[c];
            if (isfinite(v) && v > 0.f) {
                sum += log2f(v);
                cnt += 1.f;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sum += __shfl_xor_sync(0xffffffffu, sum, o);
            cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        }
        const float mean = cnt > 0.f ? sum / cnt : 0.f;
        for (int c = lane; c < n_cfg; c += 32) {
            const float v = row[c];
            out[r * n_cfg + c] = (isfinite(v) && v > 0.f) ? log2f(v) - mean : __int_as_float(0x7fc00000);
        }
    }
}

}  // namespace
}  // namespace klr

extern "C" klr_status klr_mlp_query_targets(const float* cycles, int64_t n_rows, int32_t n_cfg,
                                            float* out, void* stream_) {
    KLR_REQUIRE(n_rows >= 0 && n_cfg >= 1, "klr_mlp_query_targets: bad sizes");
    if (n_rows == 0) return KLR_OK;
    KLR_REQUIRE(cycles && out, "klr_mlp_query_targets: NULL array");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    klr::query_targets_kernel<<<klr::blocks_for(n_rows * 32, 256), 256, 0, s>>>(cycles, n_rows,
                                                                               n_cfg, out);
    KLR_CHECK_CUDA(cudaGetLastError());
    return KLR_OK;
}

// ---------------------------------------------------------------------------
// Proposal: every shape of every query through the network, top-k of the
// meaningful shapes by predicted value.
// ---------------------------------------------------------------------------
namespace klr {
namespace {

struct ProposeArgs {
    int64_t q0, nq;                 // query range of this chunk
    const int64_t* q_off;
    const int64_t* q_N;
    int32_t n_kernels;
    int n_cfg;
    const int32_t* cfg;
    const int32_t* regs;
    const int32_t* smem;
    long long Bm, Wm, Rm, Zm, Tmax;
    int dims;
    int32_t* row_kernel;            // chunk rows: nq x n_cfg
    int64_t* row_N;
    int32_t* row_cfg;
    int64_t* row_query;
    const float* pred;
    int k;
    int32_t* cand;
    float hw[7];
    __nv_bfloat16* X0;
};

// kernel of a query by binary search in the CSR offsets
__device__ int32_t kernel_of(const int64_t* off, int32_t nk, int64_t q) {
    int32_t lo = 0, hi = nk;   // off[lo] <= q < off[hi]
    while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (off[mid] <= q) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void propose_rows_kernel(const __grid_constant__ ProposeArgs a) {
    const int64_t total = a.nq * a.n_cfg;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < total;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t qi = r / a.n_cfg;
        const int c = (int)(r - qi * a.n_cfg);
        const int64_t q = a.q0 + qi;
        const int32_t k = kernel_of(a.q_off, a.n_kernels, q);
        const int64_t N = a.q_N[q];
        a.row_kernel[r] = k;
        float f[FEAT];
        f[0] = log2f((float)N) * (1.0f / 23.0f);
        f[1] = log2f((float)a.cfg[3 * c]) * 0.1f;
        f[2] = log2f((float)a.cfg[3 * c + 1]) * 0.1f;
        f[3] = log2f((float)a.cfg[3 * c + 2]) * 0.1f;
        for (int i = 0; i < 7; ++i) f[4 + i] = a.hw[i];
        for (int i = 11; i < FEAT; ++i) f[i] = 0.f;
        for (int i = 0; i < FEAT; ++i) a.X0[r * IN + i] = __float2bfloat16(f[i]);
    }
}

// per-query head: one row per query (shape features 0)
__global__ void propose_query_rows_kernel(const __grid_constant__ ProposeArgs a) {
    for (int64_t qi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; qi < a.nq;
         qi += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = a.q0 + qi;
        a.row_kernel[qi] = kernel_of(a.q_off, a.n_kernels, q);
        float f[FEAT];
        f[0] = log2f((float)a.q_N[q]) * (1.0f / 23.0f);
        f[1] = f[2] = f[3] = 0.f;
        for (int i = 0; i < 7; ++i) f[4 + i] = a.hw[i];
        for (int i = 11; i < FEAT; ++i) f[i] = 0.f;
        for (int i = 0; i < FEAT; ++i) a.X0[qi * IN + i] = __float2bfloat16(f[i]);
    }
}

// one thread per query: the k smallest predictions among meaningful shapes
// (predictions laid out [query][shape] in both output forms)
__global__ void topk_kernel(const __grid_constant__ ProposeArgs a) {
    for (int64_t qi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; qi < a.nq;
         qi += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = a.q0 + qi;
        const int32_t kk = kernel_of(a.q_off, a.n_kernels, q);
        const long long N = a.q_N[q];
        float bv[16];
        int bi[16];
        for (int j = 0; j < a.k; ++j) { bv[j] = INFINITY; bi[j] = -1; }
        for (int c = 0; c < a.n_cfg; ++c) {
            const long long b0 = a.cfg[3 * c], b1 = a.cfg[3 * c + 1], b2 = a.cfg[3 * c + 2];
            const long long T = b0 * b1 * b2;
            const int B = occupancy_blocks(T, a.regs[kk], a.smem[kk], a.Bm, a.Wm, a.Rm, a.Zm, a.Tmax);
            const bool ok = B > 0 && b0 <= N && (a.dims < 2 || b1 <= N) && (a.dims < 3 || b2 <= N);
            if (!ok) continue;
            float v = a.pred[qi * a.n_cfg + c];
            if (!(v < bv[a.k - 1])) continue;
            int vi = c;
            for (int j = 0; j < a.k; ++j) {
                if (v < bv[j]) {
                    const float tv = bv[j]; const int ti = bi[j];
                    bv[j] = v; bi[j] = vi;
                    v = tv; vi = ti;
                }
            }
        }
        for (int j = 0; j < a.k; ++j) a.cand[q * a.k + j] = bi[j];
    }
}

}  // namespace
}  // namespace klr

extern "C" klr_status klr_propose(klr_ctx* ctx, const klr_mlp* net, const float* coef,
                                  const int32_t* regs, const int32_t* smem, int32_t n_kernels,
                                  const klr_hw* hw, const int32_t* cfg, int n_cfg,
                                  const klr_queries* q, int k, int32_t* cand_out, void* stream_) {
    KLR_REQUIRE(ctx && hw && q, "klr_propose: NULL context, hw or queries");
    klr_status st = check_net(net);
    if (st != KLR_OK) return st;
    KLR_REQUIRE(k >= 1 && k <= 16, "klr_propose: k %d not in 1..16", k);
    KLR_REQUIRE(n_cfg >= 1 && n_cfg <= 256, "klr_propose: n_cfg %d not in 1..256", n_cfg);
    KLR_REQUIRE(n_kernels >= 1 && q->n_queries >= 0, "klr_propose: bad sizes");
    if (q->n_queries == 0) return KLR_OK;
    KLR_REQUIRE(coef && regs && smem && cfg && q->q_offsets && q->q_N && cand_out,
                "klr_propose: NULL device array");
    Context* c = reinterpret_cast<Context*>(ctx);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    KLR_CHECK_CUDA(cudaSetDevice(c->device));
    const int nc = net->n_coef;
    const int no = net->n_out;
    KLR_REQUIRE(no == 0 || no == n_cfg, "klr_propose: the network has %d outputs for %d shapes",
                no, n_cfg);
    const Offsets o = offsets(nc, no);
    // per row: one network row per (query, shape); per query: one per query
    const int64_t qchunk = no > 0 ? kMaxRows : std::max<int64_t>(1, kMaxRows / n_cfg);
    const int64_t rows = no > 0 ? qchunk : qchunk * n_cfg;
    // workspace: network buffers for `rows` rows + per-kernel embeddings + row tables
    const size_t base = mlp_ws_bytes(rows, nc, no, n_kernels, false);
    const size_t extra = align256(2 * (size_t)n_kernels * nc) + align256(4 * (size_t)rows) * 2 +
                         align256(8 * (size_t)rows) * 2;
    if ((st = ensure_workspace(c, base + extra, s)) != KLR_OK) return st;
    MlpWs w = carve(c->ws, rows, nc, no, n_kernels, false);
    char* p = reinterpret_cast<char*>(c->ws) + base;
    __nv_bfloat16* coef_b = reinterpret_cast<__nv_bfloat16*>(p);
    p += align256(2 * (size_t)n_kernels * nc);
    int32_t* row_kernel = reinterpret_cast<int32_t*>(p);
    p += align256(4 * (size_t)rows);
    int32_t* row_cfg = reinterpret_cast<int32_t*>(p);
    p += align256(4 * (size_t)rows);
    int64_t* row_N = reinterpret_cast<int64_t*>(p);
    p += align256(8 * (size_t)rows);
    int64_t* row_query = reinterpret_cast<int64_t*>(p);
    cast_bf16_kernel<<<blocks_for(o.total, 256), 256, 0, s>>>(net->params, w.pb, o.total);
    cast_bf16_kernel<<<blocks_for((int64_t)n_kernels * nc, 256), 256, 0, s>>>(
        coef, coef_b, (int64_t)n_kernels * nc);
    // per-kernel embedding table: coef E^T
    GemmArgs g{};
    g.M = n_kernels;
    g.N = EMB;
    g.K = nc;
    g.A = coef_b;
    g.lda = nc;
    g.B = w.pb + o.E;
    g.ldb = nc;
    g.Cb = w.emb_table;
    g.ldcb = EMB;
    if ((st = gemm<false, false, EPI_BF16>(g, s)) != KLR_OK) return st;
    for (int64_t q0 = 0; q0 < q->n_queries; q0 += qchunk) {
        const int64_t nq = std::min(qchunk, q->n_queries - q0);
        ProposeArgs a{};
        a.q0 = q0;
        a.nq = nq;
        a.q_off = q->q_offsets;
        a.q_N = q->q_N;
        a.n_kernels = n_kernels;
        a.n_cfg = n_cfg;
        a.cfg = cfg;
        a.regs = regs;
        a.smem = smem;
        a.Bm = hw->max_blocks_per_sm;
        a.Wm = hw->max_warps_per_sm;
        a.Rm = hw->regs_per_sm;
        a.Zm = hw->smem_per_sm;
        a.Tmax = hw->max_threads_per_block;
        a.dims = 3;
        a.row_kernel = row_kernel;
        a.row_N = row_N;
        a.row_cfg = row_cfg;
        a.row_query = row_query;
        a.pred = w.pred;
        a.k = k;
        a.cand = cand_out;
        for (int i = 0; i < 7; ++i) a.hw[i] = net->hw_feat[i];
        a.X0 = w.X0;
        const int64_t nr = no > 0 ? nq : nq * n_cfg;
        if (no > 0)
            propose_query_rows_kernel<<<blocks_for(nr, 256), 256, 0, s>>>(a);
        else
            propose_rows_kernel<<<blocks_for(nr, 256), 256, 0, s>>>(a);
        embed_rows_kernel<<<blocks_for(nr * EMB, 256), 256, 0, s>>>(row_kernel, nr, w.emb_table, w.X0);
        KLR_CHECK_CUDA(cudaGetLastError());
        if ((st = forward_hidden(w, net->params, o, no, nr, false, s)) != KLR_OK) return st;
        topk_kernel<<<blocks_for(nq, 128), 128, 0, s>>>(a);
        KLR_CHECK_CUDA(cudaGetLastError());
    }
    return KLR_OK;
}
