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
#include "klr_umma.cuh"

namespace klr {

namespace {

constexpr int FEAT = 16, EMB = 64, IN = 80, H = 256;
// per-kernel table row: the 64 embedding values, then (proposal, per-query
// form) eight 32-bit occupancy words, bit c of word w for shape 32 w + c
constexpr int kEmbLd = EMB + 16;
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

// tanh by the hardware approximation (relative error about 2^-11, below the
// BF16 rounding of the activations it feeds)
__device__ __forceinline__ float tanh_hw(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// gelu(z) = z/2 (1 + tanh(u)), u = sqrt(2/pi) (z + 0.044715 z^3) written as
// z (c + c3 z^2); the same operations, in the same order, as gelu2_bf16
constexpr float kGeluC = 0.7978845608028654f;      // sqrt(2 / pi)
constexpr float kGeluC3 = 0.035677408136300125f;   // sqrt(2 / pi) x 0.044715
__device__ __forceinline__ float gelu(float z) {
    const float u = z * fmaf(z * z, kGeluC3, kGeluC);
    const float h = 0.5f * z;
    return fmaf(h, tanh_hw(u), h);
}

// two GELUs of (a + bias_a, b + bias_b) on packed FP32 pairs, rounded to a
// BF16 pair (first value in the low half)
__device__ __forceinline__ uint32_t gelu2_bf16(float a, float b, float bias_a, float bias_b) {
    uint32_t out;
    asm("{\n"
        ".reg .b64 z, t, k, w;\n"
        ".reg .f32 u0, u1, t0, t1;\n"
        "mov.b64 z, {%1, %2};\n"
        "mov.b64 t, {%3, %4};\n"
        "add.rn.f32x2 z, z, t;\n"               // z
        "mul.rn.f32x2 w, z, z;\n"               // z^2
        "mov.b64 k, {%5, %5};\n"
        "mov.b64 t, {%6, %6};\n"
        "fma.rn.f32x2 w, w, k, t;\n"            // c + c3 z^2
        "mul.rn.f32x2 w, z, w;\n"               // u
        "mov.b64 {u0, u1}, w;\n"
        "tanh.approx.f32 t0, u0;\n"
        "tanh.approx.f32 t1, u1;\n"
        "mov.b64 k, {%7, %7};\n"
        "mul.rn.f32x2 z, z, k;\n"               // h = z / 2
        "mov.b64 t, {t0, t1};\n"
        "fma.rn.f32x2 z, z, t, z;\n"            // h tanh(u) + h
        "mov.b64 {u0, u1}, z;\n"
        "cvt.rn.bf16x2.f32 %0, u1, u0;\n"
        "}\n"
        : "=r"(out)
        : "f"(a), "f"(b), "f"(bias_a), "f"(bias_b), "f"(kGeluC3), "f"(kGeluC), "f"(0.5f));
    return out;
}
__device__ __forceinline__ float gelu_grad(float z) {
    const float c = 0.7978845608028654f;
    const float t = tanh_hw(c * (z + 0.044715f * z * z * z));
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
        X0[r * IN + FEAT + j] = table[(int64_t)kernel[r] * kEmbLd + j];
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
    b += align256(2 * (size_t)n_kernels_table * kEmbLd);      // emb table
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
    w.emb_table = reinterpret_cast<__nv_bfloat16*>(take(2 * (size_t)n_kernels_table * kEmbLd));
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

// ---------------------------------------------------------------------------
// Inference on the 5th-generation tensor cores: the whole network for a tile
// of 128 rows in one CTA.  Per layer, the weights (pre-packed once per call
// in the shared-memory image below) arrive by one bulk asynchronous copy
// completing on an mbarrier; one thread issues the tcgen05.mma chain (BF16
// operands from shared memory, FP32 accumulator of 128 lanes x N columns in
// tensor memory); the epilogue reads the accumulator back with tcgen05.ld,
// adds the bias, applies GELU and writes BF16 activations into the operand
// buffer of the next layer, so activations never leave the SM.  The next
// layer's weights are copied while the epilogue runs.
//
// Operand image (K-major, 128-byte swizzle): a matrix of R rows and K
// columns is stored as K/64 blocks of R x 128 bytes; row r of a block holds
// its 64 elements as eight 16-byte chunks, chunk c at position c ^ (r mod 8);
// rows come in groups of 8 (1024 bytes).  Matrix descriptors: start address,
// stride 1024 bytes between 8-row groups, 128-byte swizzle; each K step of 16
// elements advances the start address by 32 bytes within a block.
// ---------------------------------------------------------------------------
constexpr int kTileRows = 128;
constexpr int kKPad1 = 128;                 // layer-1 K (80) padded to whole blocks


// packed weight images: W1 (256 x 128, K 80 + zero pad), W2, W3 (256 x 256),
// W4 (np x 256, rows past the outputs zero)
struct Packed {
    int64_t w1, w2, w3, w4, total;          // byte offsets
};
Packed packed_layout(int np) {
    Packed p;
    p.w1 = 0;
    p.w2 = p.w1 + (int64_t)H * kKPad1 * 2;
    p.w3 = p.w2 + (int64_t)H * H * 2;
    p.w4 = p.w3 + (int64_t)H * H * 2;
    p.total = p.w4 + (int64_t)np * H * 2;
    return p;
}

// one thread per 16-byte chunk of the packed images
__global__ void pack_weights_kernel(const __nv_bfloat16* __restrict__ pb, Offsets o, int n_outs,
                                    int np, Packed pk, unsigned char* __restrict__ img) {
    const int64_t c1 = (int64_t)H * kKPad1 / 8, c2 = (int64_t)H * H / 8, c4 = (int64_t)np * H / 8;
    const int64_t total = c1 + 2 * c2 + c4;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t j = i;
        const __nv_bfloat16* src;
        int K, rows, rows_valid;
        int64_t dst;
        if (j < c1) {
            src = pb + o.W1; K = IN; rows = H; rows_valid = H; dst = pk.w1;
        } else if ((j -= c1) < c2) {
            src = pb + o.W2; K = H; rows = H; rows_valid = H; dst = pk.w2;
        } else if ((j -= c2) < c2) {
            src = pb + o.W3; K = H; rows = H; rows_valid = H; dst = pk.w3;
        } else {
            j -= c2;
            src = pb + o.W4; K = H; rows = np; rows_valid = n_outs; dst = pk.w4;
        }
        const int kpad = (K == IN) ? kKPad1 : K;
        const int r = (int)(j / (kpad / 8)), k = (int)(j % (kpad / 8)) * 8;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (r < rows_valid && k < K) v = *reinterpret_cast<const uint4*>(src + (int64_t)r * K + k);
        *reinterpret_cast<uint4*>(img + dst + swz_off(r, k, rows)) = v;
    }
}

// thread 0: bulk-copy `bytes` (multiple of 16) of a packed image into shared
// memory, completing on mbar
__device__ __forceinline__ void tma_load(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* mbar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(smem_addr(mbar)), "r"(bytes) : "memory");
    constexpr uint32_t kChunk = 32768;
    for (uint32_t o = 0; o < bytes; o += kChunk) {
        const uint32_t n = bytes - o < kChunk ? bytes - o : kChunk;
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
                     "[%0], [%1], %2, [%3];"
                     :: "r"(smem_addr(static_cast<unsigned char*>(dst) + o)),
                        "l"(static_cast<const unsigned char*>(src) + o), "r"(n),
                        "r"(smem_addr(mbar))
                     : "memory");
    }
}

struct FusedArgs {
    const __nv_bfloat16* X0;     // n x IN, row-major
    const unsigned char* img;    // packed weight images
    Packed pk;
    const float* params;         // FP32 parameters (biases)
    Offsets o;
    int64_t n;
    int n_out;                   // outputs written per row (1 for the per-row form)
    int np;                      // output columns computed (multiple of 16, >= n_out)
    float* pred;                 // n x n_out
    int* err;                    // set when a wait gave up
    // proposal mode (per-query form): rows are queries q0.. of the CSR list;
    // the input tile is built here and the layer-4 epilogue keeps the k
    // least predictions among the meaningful shapes instead of writing pred
    int propose;
    int64_t q0;
    const int32_t* q_kernel;          // kernel of every query
    const int64_t* q_off;
    const int64_t* q_N;
    int32_t n_kernels;
    const __nv_bfloat16* emb_table;   // n_kernels x kEmbLd: embedding, then occupancy words
    float hw[7];
    const int32_t* cfg;
    int k;                            // 1..16
    int32_t* cand;                    // n_queries x k
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

// ---------------------------------------------------------------------------
// Fused forward pass on the tensor cores, pipelined across layers.
//
// One CTA per SM, persistent over tiles of 128 rows; 16 epilogue warps, one
// warp whose lane 0 issues the products and one whose lane 0 streams the
// weights.  Tensor memory holds two 128 x 256 FP32 accumulators, so
// a layer's products go to one while the previous layer's are read from the
// other.  The epilogue of a layer hands the next layer's operand over one
// 64-column K-block at a time (mbarrier act[g]: the 16 epilogue warps,
// one arrival per warp once all its lanes have written and fenced their
// part), and the issuing thread starts that K-block's products as soon as it
// is complete, so the products of layer L + 1 overlap the epilogue of layer L.
// Weights stream through four 32 KB slots, one K-block of one layer each
// (mbarrier full[g]); the producer refills a slot with its next K-block as
// soon as the products that read it have completed (free[g], by
// tcgen05.commit), a whole layer ahead of its use.  In the last layer's epilogue one warp per lane
// quadrant keeps each row's top-k over all columns (or writes the outputs)
// while the other twelve build the next tile's input rows, whose first
// products start at once (they use the other accumulator).
//
// Every wait is bounded and gives up when another thread has given up; the
// issuer then drains the tensor pipe, the producer its outstanding copies, and
// the CTA marks its rows (NaN outputs, -1 candidates) and sets the error flag.
// ---------------------------------------------------------------------------
constexpr int kEpiWarps = 16;
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kFusedThreads = kEpiThreads + 64;     // + the MMA issuer and the weight producer
constexpr uint32_t kKBlockBytes = kTileRows * 128;        // one K-block of the activations
constexpr uint32_t kSlotBytes = H * 128;                  // one K-block of a layer's weights
// Dynamic shared memory, from a 1 KB boundary: activations (128 x 256 BF16),
// four weight slots, and in proposal mode each row's occupancy words and size
// for two tiles (by tile parity); every offset is a multiple of 1 KB.
constexpr uint32_t kRowOccBytes = 2 * kTileRows * 8 * 4;
constexpr uint32_t kRowNBytes = 2 * kTileRows * 8;
constexpr size_t kFusedSmem = 1024 + (size_t)kTileRows * H * 2 + 4 * (size_t)kSlotBytes +
                              kRowOccBytes + kRowNBytes;


// bounded wait that also gives up once `abort` is set
__device__ __forceinline__ bool mbar_wait_ab(uint64_t* mbar, uint32_t parity,
                                             volatile int* abort) {
    for (int it = 0; it < (1 << 22); ++it) {
        if (mbar_try(mbar, parity)) return true;
        if ((it & 15) == 15 && *abort) return false;
    }
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_addr(mbar)) : "memory");
}

// the wait of every lane of a warp; true only when it ended for all of
// them, so that the warp stays converged on the way out
__device__ __forceinline__ bool warp_wait(uint64_t* mbar, uint32_t parity, volatile int* abort) {
    const bool ok = mbar_wait_ab(mbar, parity, abort);
    return __all_sync(0xffffffffu, ok);
}

// every lane's shared-memory writes made visible to the tensor core (async
// proxy) and ordered before one arrival for the warp
__device__ __forceinline__ void warp_arrive_async(uint64_t* mbar, int lane) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncwarp();
    if (lane == 0) mbar_arrive(mbar);
}


template <int KMAX>
__global__ void __launch_bounds__(kFusedThreads, 1)
fused_forward_kernel(const __grid_constant__ FusedArgs a) {
    extern __shared__ unsigned char fsm_raw[];
    unsigned char* As = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(fsm_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char* Bs = As + kTileRows * H * 2;
    // proposal mode: row_occ[buf][row][w] and row_N[buf][row]
    auto row_occ = reinterpret_cast<uint32_t (*)[kTileRows][8]>(Bs + 4 * kSlotBytes);
    auto row_N = reinterpret_cast<long long (*)[kTileRows]>(Bs + 4 * kSlotBytes + kRowOccBytes);
    __shared__ uint64_t mb_full[4], mb_free[4], mb_act[4], mb_mma, mb_rows, mb_final;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ float bias_s[4 * H];                  // b1, b2, b3, b4 (np <= 256)
    __shared__ int32_t cfg_max[H];                   // proposal mode: largest block dimension
    volatile int* abort_v = &abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t n_tiles = (a.n + kTileRows - 1) / kTileRows;
    if ((int64_t)blockIdx.x >= n_tiles) return;
    if (tid == 0) {
        for (int g = 0; g < 4; ++g) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&mb_full[g])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&mb_free[g])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;"
                         :: "r"(smem_addr(&mb_act[g])), "r"(kEpiWarps));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&mb_mma)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;"
                     :: "r"(smem_addr(&mb_rows)), "r"(kEpiWarps - 4));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&mb_final)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    if (warp == kEpiWarps) {
        // both accumulators: 512 columns
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_addr(&tmem_base)), "r"((uint32_t)(2 * H)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    for (int i = tid; i < 4 * H; i += kFusedThreads) {
        const int l = i / H, c = i - l * H;
        const int64_t off = l == 0 ? a.o.b1 : l == 1 ? a.o.b2 : l == 2 ? a.o.b3 : a.o.b4;
        bias_s[i] = (l < 3 || c < a.n_out) ? a.params[off + c] : 0.f;
    }
    if (a.propose)
        for (int c = tid; c < a.n_out; c += kFusedThreads)
            cfg_max[c] = max(a.cfg[3 * c], max(a.cfg[3 * c + 1], a.cfg[3 * c + 2]));
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t sA = smem_addr(As), sB = smem_addr(Bs);

    if (warp == kEpiWarps) {
        // ------------------------------------------------------- MMA issuer
        if (lane == 0) {
            uint32_t ph_full = 0, ph_act = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
                for (int L = 0; L < 4 && ok; ++L) {
                    const int nkb = L == 0 ? 2 : 4;
                    const uint32_t idesc = umma_idesc_bf16(kTileRows, L == 3 ? a.np : H);
                    const uint32_t acc = tmem + (uint32_t)((L & 1) * H);
                    for (int g = 0; g < nkb; ++g) {
                        if (!mbar_wait_ab(&mb_full[g], (ph_full >> g) & 1u, abort_v) ||
                            !mbar_wait_ab(&mb_act[g], (ph_act >> g) & 1u, abort_v)) {
                            ok = false;
                            break;
                        }
                        ph_full ^= 1u << g;
                        ph_act ^= 1u << g;
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const int steps = (L == 0 && g == 1) ? (IN - 64) / 16 : 4;
                        for (int s = 0; s < steps; ++s)
                            umma_bf16(acc, umma_desc(sA + g * kKBlockBytes + s * 32),
                                      umma_desc(sB + g * kSlotBytes + s * 32), idesc, (g | s) != 0);
                        umma_commit(&mb_free[g]);       // slot g and K-block g read
                    }
                    if (ok) umma_commit(&mb_mma);
                }
            }
            if (!ok) *abort_v = 1;
            // drain: every product issued has completed
            umma_commit(&mb_final);
            mbar_wait(&mb_final, 0);
        }
        __syncwarp();
    } else if (warp == kEpiWarps + 1) {
        // -------------------------------------------------- weight producer
        // K-block g of each layer's weights into slot g, in the order the
        // products use them; a slot is refilled once the products that read
        // its previous K-block have completed (a layer ahead of its use)
        if (lane == 0) {
            uint32_t ph_free = 0, used = 0, n_issued[4] = {0u, 0u, 0u, 0u};
            bool ok = true;
            for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
                for (int L = 0; L < 4 && ok; ++L) {
                    const int nkb = L == 0 ? 2 : 4;
                    const uint32_t bytes = (uint32_t)(L == 3 ? a.np : H) * 128u;
                    const int64_t base = L == 0 ? a.pk.w1 : L == 1 ? a.pk.w2 : L == 2 ? a.pk.w3 : a.pk.w4;
                    for (int g = 0; g < nkb; ++g) {
                        if ((used >> g) & 1u) {
                            if (!mbar_wait_ab(&mb_free[g], (ph_free >> g) & 1u, abort_v)) {
                                ok = false;
                                break;
                            }
                            ph_free ^= 1u << g;
                        }
                        used |= 1u << g;
                        tma_load(Bs + g * kSlotBytes, a.img + base + (int64_t)g * bytes, bytes,
                                 &mb_full[g]);
                        ++n_issued[g];
                    }
                }
            }
            if (!ok) *abort_v = 1;
            // drain: every copy issued has landed
            for (int g = 0; g < 4; ++g)
                if (n_issued[g]) mbar_wait(&mb_full[g], (n_issued[g] - 1) & 1u);
        }
        __syncwarp();
    } else {
        // ----------------------------------------------------------- epilogue
        const int qd = warp & 3, cg = warp >> 2;       // lane quadrant, column group
        const int row = 32 * qd + lane;                // row of the tile (TMEM lane)
        const uint32_t lane_base = (uint32_t)(32 * qd) << 16;
        // Column group 0 keeps the last layer's outputs (one thread per row,
        // every column); groups 1-3 build the next tile's input meanwhile,
        // three threads per row: input chunks (8 columns) 0-3, 4-6 and 7-9.
        const int bj = cg - 1;
        const int ch_lo = bj == 0 ? 0 : bj == 1 ? 4 : 7, ch_hi = bj == 0 ? 4 : bj == 1 ? 7 : 10;
        // input row `row` of tile tt (columns 0-79: K-blocks 0 and 1), and in
        // proposal mode the row's size and occupancy words (rows buffer `rb`)
        auto build_input = [&](int64_t tt, int rb) {
            const int64_t gr = tt * kTileRows + row;
            const bool in = gr < a.n;
            if (a.propose) {
                // rows are queries: features (log2 N / 23, shape features 0,
                // the hardware vector) and the kernel's embedding
                const int64_t q = a.q0 + (in ? gr : 0);
                const long long N = in ? a.q_N[q] : 1;
                const int32_t kk = in ? a.q_kernel[q] : 0;
                const __nv_bfloat16* erow = a.emb_table + (int64_t)kk * kEmbLd;
                for (int ch = ch_lo; ch < ch_hi; ++ch) {
                    unsigned char* dst = As + swz_off(row, ch * 8, kTileRows);
                    if (ch < 2) {
                        float f[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) f[i] = 0.f;
                        if (in) {
                            if (ch == 0) {
                                f[0] = log2f((float)N) * (1.0f / 23.0f);
                                for (int i = 0; i < 4; ++i) f[4 + i] = a.hw[i];
                            } else {
                                for (int i = 0; i < 3; ++i) f[i] = a.hw[4 + i];
                            }
                        }
                        uint32_t w[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const __nv_bfloat162 h2 = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
                            w[i] = *reinterpret_cast<const uint32_t*>(&h2);
                        }
                        *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
                    } else {
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                                     :: "r"(smem_addr(dst)), "l"(erow + (ch - 2) * 8),
                                        "r"(in ? 16u : 0u)
                                     : "memory");
                    }
                }
                if (bj == 0) row_N[rb][row] = N;
                if (bj == 2) {
                    // the occupancy words stored after the embedding
                    for (int h = 0; h < 2; ++h)
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                                     :: "r"(smem_addr(&row_occ[rb][row][4 * h])),
                                        "l"(erow + EMB + 8 * h)
                                     : "memory");
                }
            } else {
                for (int ch = ch_lo; ch < ch_hi; ++ch) {
                    const void* src = a.X0 + (in ? gr : 0) * IN + ch * 8;
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                                 :: "r"(smem_addr(As + swz_off(row, ch * 8, kTileRows))), "l"(src),
                                    "r"(in ? 16u : 0u)
                                 : "memory");
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        // builders: copies done, both input K-blocks (and the rows) announced
        auto input_ready = [&]() {
            asm volatile("cp.async.wait_all;" ::: "memory");
            warp_arrive_async(&mb_act[0], lane);
            if (lane == 0) {
                mbar_arrive(&mb_act[1]);
                if (a.propose) mbar_arrive(&mb_rows);
            }
        };
        // group 0: no writes of its own; its arrival only counts
        auto input_count = [&]() {
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&mb_act[0]);
                mbar_arrive(&mb_act[1]);
            }
        };
        uint32_t ph_mma = 0, ph_rows = 0;
        bool ok = true;
        if (cg > 0) {
            build_input(blockIdx.x, 0);
            input_ready();
        } else {
            input_count();
        }
        int it = 0;
        for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, ++it) {
            const int64_t r0 = t * kTileRows;
            const bool more = t + gridDim.x < n_tiles;
            const int rb = it & 1;
            // group 0, proposal mode: this tile's rows are staged (waited
            // here, before the next tile's builders can reuse the phase)
            if (cg == 0 && a.propose) {
                if (!warp_wait(&mb_rows, ph_rows, abort_v)) { ok = false; break; }
                ph_rows ^= 1;
            }
            // hidden layers: bias + GELU, BF16 operand of the next layer
            for (int L = 0; L < 3; ++L) {
                if (!warp_wait(&mb_mma, ph_mma, abort_v)) { ok = false; break; }
                ph_mma ^= 1;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t tb = tmem + lane_base + (uint32_t)(L & 1) * H + (uint32_t)(cg * 16);
                const float* bias = bias_s + L * H;
                float v[32];                           // K-blocks two at a time
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    if ((g & 1) == 0) tmem_ld16x2(tb + 64 * g, tb + 64 * (g + 1), v);
                    const int c0 = g * 64 + cg * 16;
                    uint32_t packed[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        packed[j] = gelu2_bf16(v[16 * (g & 1) + 2 * j], v[16 * (g & 1) + 2 * j + 1],
                                               bias[c0 + 2 * j], bias[c0 + 2 * j + 1]);
                    *reinterpret_cast<uint4*>(As + swz_off(row, c0, kTileRows)) =
                        make_uint4(packed[0], packed[1], packed[2], packed[3]);
                    *reinterpret_cast<uint4*>(As + swz_off(row, c0 + 8, kTileRows)) =
                        make_uint4(packed[4], packed[5], packed[6], packed[7]);
                    warp_arrive_async(&mb_act[g], lane);
                }
            }
            if (!ok) break;
            // output layer
            if (!warp_wait(&mb_mma, ph_mma, abort_v)) { ok = false; break; }
            ph_mma ^= 1;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (cg > 0) {
                // K-blocks 0-1 are free: the next tile's input
                if (more) {
                    build_input(t + gridDim.x, rb ^ 1);
                    input_ready();
                }
                continue;
            }
            // group 0: the next tile's first products may start (they use
            // the other accumulator)
            if (more) input_count();
            const int64_t gr = r0 + row;
            const float* bias = bias_s + 3 * H;
            const uint32_t tb = tmem + lane_base + (uint32_t)H;
            if (a.propose) {
                // the k least predictions among the meaningful shapes of the
                // row's query, ties to the lower shape index
                const long long qN = row_N[rb][row];
                float bv[KMAX];
                int bi[KMAX];
#pragma unroll
                for (int j = 0; j < KMAX; ++j) { bv[j] = INFINITY; bi[j] = -1; }
                for (int c0 = 0; c0 < a.np; c0 += 32) {
                    float v[32];
                    tmem_ld16x2(tb + c0, tb + c0 + 16, v);
                    const uint32_t ob = row_occ[rb][row][c0 >> 5];
                    // branch-free: a shape that is not meaningful enters as
                    // +inf and never displaces an entry (nor does a NaN)
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int c = c0 + j;
                        if (c >= a.n_out) break;          // the same for every lane
                        const bool use = cfg_max[c] <= qN && ((ob >> j) & 1u);
                        float x = use ? v[j] + bias[c] : INFINITY;
                        int xi = c;
#pragma unroll
                        for (int m = 0; m < KMAX; ++m) {
                            const bool sw = x < bv[m];
                            const float tv = bv[m];
                            const int ti = bi[m];
                            bv[m] = sw ? x : tv;
                            bi[m] = sw ? xi : ti;
                            x = sw ? tv : x;
                            xi = sw ? ti : xi;
                        }
                    }
                }
                if (gr < a.n) {
                    const int64_t q = a.q0 + gr;
#pragma unroll
                    for (int m = 0; m < KMAX; ++m)
                        if (m < a.k) a.cand[q * a.k + m] = bi[m];
                }
            } else {
                for (int c0 = 0; c0 < a.np; c0 += 32) {
                    float v[32];
                    tmem_ld16x2(tb + c0, tb + c0 + 16, v);
                    if (gr < a.n) {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (c0 + j < a.n_out) a.pred[gr * a.n_out + c0 + j] = v[j] + bias[c0 + j];
                    }
                }
            }
        }
        if (!ok) *abort_v = 1;
        asm volatile("cp.async.wait_all;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (abort_flag) {
        // a wait gave up: every prediction of this CTA's tiles NaN (proposal
        // mode: no candidates)
        if (tid == 0) atomicExch(a.err, 1);
        for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
            const int64_t e = min((t + 1) * kTileRows, a.n);
            if (a.propose) {
                for (int64_t i = t * kTileRows * a.k + tid; i < e * a.k; i += kFusedThreads)
                    a.cand[a.q0 * a.k + i] = -1;
            } else {
                for (int64_t i = t * kTileRows * a.n_out + tid; i < e * a.n_out; i += kFusedThreads)
                    a.pred[i] = __int_as_float(0x7fc00000);
            }
        }
    }
    if (warp == kEpiWarps) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :: "r"(tmem), "r"((uint32_t)(2 * H)));
    }
}

// Packed weight images for the fused kernel, from the BF16 parameter copy;
// fills the image fields of `a` (outputs, padded output columns).
klr_status pack_weights(const MlpWs& w, const float* params, const Offsets& o, int n_out,
                        unsigned char* img, int* err, FusedArgs& a, cudaStream_t s) {
    const int outs = out_cols(n_out);
    const int np = (outs + 15) & ~15;
    const Packed pk = packed_layout(np);
    pack_weights_kernel<<<blocks_for(pk.total / 16, 256), 256, 0, s>>>(w.pb, o, outs, np, pk, img);
    KLR_CHECK_CUDA(cudaGetLastError());
    a.img = img;
    a.pk = pk;
    a.params = params;
    a.o = o;
    a.n_out = outs;
    a.np = np;
    a.err = err;
    return KLR_OK;
}

klr_status launch_fused(const Context* c, const FusedArgs& a, cudaStream_t s) {
    if (a.n == 0) return KLR_OK;
    const int64_t tiles = (a.n + kTileRows - 1) / kTileRows;
    const int grid = (int)std::min<int64_t>(tiles, c->n_sm);
    auto go = [&](auto kern) -> klr_status {
        KLR_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)kFusedSmem));
        kern<<<grid, kFusedThreads, kFusedSmem, s>>>(a);
        KLR_CHECK_CUDA(cudaGetLastError());
        return KLR_OK;
    };
    // top-k lists of 8 or 16 entries (proposal mode)
    return a.k > 8 ? go(fused_forward_kernel<16>) : go(fused_forward_kernel<8>);
}

// Forward pass of rows whose X0 is set, on the tensor cores (one CTA per SM
// over tiles of 128 rows); pred as in forward_hidden.
klr_status fused_forward(const Context* c, const MlpWs& w, const float* params, const Offsets& o,
                         int n_out, int64_t n, unsigned char* img, int* err, cudaStream_t s) {
    if (n == 0) return KLR_OK;
    FusedArgs a{};
    klr_status st = pack_weights(w, params, o, n_out, img, err, a, s);
    if (st != KLR_OK) return st;
    a.X0 = w.X0;
    a.n = n;
    a.pred = w.pred;
    return launch_fused(c, a, s);
}

// scratch of the fused forward: packed weights (at most 448 KB) and a flag
constexpr size_t kFusedScratch = 512 * 1024;

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
    if ((st = ensure_workspace(c, base + extra + kFusedScratch, s)) != KLR_OK) return st;
    MlpWs w = carve(c->ws, n, nc, no, 0, false);
    w.CR = reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<char*>(c->ws) + base);
    unsigned char* img = reinterpret_cast<unsigned char*>(c->ws) + base + extra;
    int* err = reinterpret_cast<int*>(img + kFusedScratch - 256);
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
    if ((st = fused_forward(c, w, net->params, o, no, n, img, err, s)) != KLR_OK) return st;
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
    uint8_t* occ;                   // [n_kernels x n_cfg]: 1 where B_active > 0
};

// the kernel of every query, from the CSR offsets (one thread per kernel)
__global__ void query_kernel_map_kernel(const int64_t* __restrict__ q_off, int32_t n_kernels,
                                        int32_t* __restrict__ q_kernel) {
    for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n_kernels;
         k += gridDim.x * blockDim.x)
        for (int64_t q = q_off[k]; q < q_off[k + 1]; ++q) q_kernel[q] = k;
}

// occupancy of every (kernel, shape), once per proposal call
__global__ void occupancy_table_kernel(const __grid_constant__ ProposeArgs a) {
    const int64_t total = (int64_t)a.n_kernels * a.n_cfg;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t kk = (int32_t)(i / a.n_cfg);
        const int c = (int)(i - (int64_t)kk * a.n_cfg);
        const long long T = (long long)a.cfg[3 * c] * a.cfg[3 * c + 1] * a.cfg[3 * c + 2];
        a.occ[i] = occupancy_blocks(T, a.regs[kk], a.smem[kk], a.Bm, a.Wm, a.Rm, a.Zm, a.Tmax) > 0;
    }
}

// the same facts as bits, stored after each kernel's embedding in the
// table row: word w holds shapes 32 w .. 32 w + 31 (zero past the shapes)
__global__ void occupancy_bits_kernel(const __grid_constant__ ProposeArgs a,
                                      __nv_bfloat16* table) {
    const int64_t total = (int64_t)a.n_kernels * 8;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t kk = (int32_t)(i >> 3);
        const int w = (int)(i & 7);
        uint32_t b = 0;
        for (int j = 0; j < 32; ++j) {
            const int c = 32 * w + j;
            if (c >= a.n_cfg) break;
            const long long T = (long long)a.cfg[3 * c] * a.cfg[3 * c + 1] * a.cfg[3 * c + 2];
            if (occupancy_blocks(T, a.regs[kk], a.smem[kk], a.Bm, a.Wm, a.Rm, a.Zm, a.Tmax) > 0)
                b |= 1u << j;
        }
        reinterpret_cast<uint32_t*>(table + (int64_t)kk * kEmbLd + EMB)[w] = b;
    }
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
        const uint8_t* occ = a.occ + (int64_t)kk * a.n_cfg;
        for (int c = 0; c < a.n_cfg; ++c) {
            const long long b0 = a.cfg[3 * c], b1 = a.cfg[3 * c + 1], b2 = a.cfg[3 * c + 2];
            const bool ok = occ[c] && b0 <= N && (a.dims < 2 || b1 <= N) && (a.dims < 3 || b2 <= N);
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
    // per row: one network row per (query, shape), in chunks; per query: the
    // fused kernel builds its rows itself and needs no row buffers
    const int64_t qchunk = no > 0 ? kMaxRows : std::max<int64_t>(1, kMaxRows / n_cfg);
    const int64_t rows = no > 0 ? 0 : qchunk * n_cfg;
    // occupancy per (kernel, shape): bytes here for the per-row form; the
    // per-query form keeps bits in the embedding table's rows
    const size_t occ_bytes = (size_t)n_cfg;
    // workspace: network buffers for `rows` rows + per-kernel embeddings + row tables
    const size_t base = mlp_ws_bytes(rows, nc, no, n_kernels, false);
    const size_t extra = align256(2 * (size_t)n_kernels * nc) + align256(4 * (size_t)rows) * 2 +
                         align256(8 * (size_t)rows) * 2 + align256((size_t)n_kernels * occ_bytes) +
                         kFusedScratch + (no > 0 ? align256(4 * (size_t)q->n_queries) : 0);
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
    p += align256(8 * (size_t)rows);
    uint8_t* occ = reinterpret_cast<uint8_t*>(p);
    p += align256((size_t)n_kernels * occ_bytes);
    unsigned char* img = reinterpret_cast<unsigned char*>(p);
    int* err = reinterpret_cast<int*>(img + kFusedScratch - 256);
    p += kFusedScratch;
    int32_t* q_kernel = reinterpret_cast<int32_t*>(p);
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
    g.ldcb = kEmbLd;
    if ((st = gemm<false, false, EPI_BF16>(g, s)) != KLR_OK) return st;
    {
        ProposeArgs ta{};
        ta.n_kernels = n_kernels;
        ta.n_cfg = n_cfg;
        ta.cfg = cfg;
        ta.regs = regs;
        ta.smem = smem;
        ta.Bm = hw->max_blocks_per_sm;
        ta.Wm = hw->max_warps_per_sm;
        ta.Rm = hw->regs_per_sm;
        ta.Zm = hw->smem_per_sm;
        ta.Tmax = hw->max_threads_per_block;
        ta.occ = occ;
        if (no > 0)
            occupancy_bits_kernel<<<blocks_for((int64_t)n_kernels * 8, 256), 256, 0, s>>>(
                ta, w.emb_table);
        else
            occupancy_table_kernel<<<blocks_for((int64_t)n_kernels * n_cfg, 256), 256, 0, s>>>(ta);
        KLR_CHECK_CUDA(cudaGetLastError());
    }
    if (no > 0) {
        // per-query form: features, network and top-k in one tensor-core kernel
        FusedArgs fa{};
        if ((st = pack_weights(w, net->params, o, no, img, err, fa, s)) != KLR_OK) return st;
        fa.propose = 1;
        query_kernel_map_kernel<<<blocks_for(n_kernels, 128), 128, 0, s>>>(q->q_offsets, n_kernels,
                                                                          q_kernel);
        KLR_CHECK_CUDA(cudaGetLastError());
        fa.q_kernel = q_kernel;
        fa.q_off = q->q_offsets;
        fa.q_N = q->q_N;
        fa.n_kernels = n_kernels;
        fa.emb_table = w.emb_table;
        for (int i = 0; i < 7; ++i) fa.hw[i] = net->hw_feat[i];
        fa.cfg = cfg;
        fa.k = k;
        fa.cand = cand_out;
        fa.q0 = 0;
        fa.n = q->n_queries;
        return launch_fused(c, fa, s);
    }
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
        a.occ = occ;
        const int64_t nr = no > 0 ? nq : nq * n_cfg;
        if (no > 0)
            propose_query_rows_kernel<<<blocks_for(nr, 256), 256, 0, s>>>(a);
        else
            propose_rows_kernel<<<blocks_for(nr, 256), 256, 0, s>>>(a);
        embed_rows_kernel<<<blocks_for(nr * EMB, 256), 256, 0, s>>>(row_kernel, nr, w.emb_table, w.X0);
        KLR_CHECK_CUDA(cudaGetLastError());
        if ((st = fused_forward(c, w, net->params, o, no, nr, img, err, s)) != KLR_OK) return st;
        topk_kernel<<<blocks_for(nq, 128), 128, 0, s>>>(a);
        KLR_CHECK_CUDA(cudaGetLastError());
    }
    return KLR_OK;
}
