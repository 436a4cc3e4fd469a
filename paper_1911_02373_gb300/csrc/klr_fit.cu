// F1-F4: batched rational fits (Section V-E; Section IV, step 2).
//
// Three kernels.
//
// moments_kernel (F1 + F2), one warp per fit: the fit's samples are streamed
// once from HBM (coalesced, 32 samples per step, staged as powers of the
// scaled coordinates in shared memory) while the warp accumulates the moment
// sums
//     M_k[mu] = sum_s y_s^k x_s^mu,  k = 0, 1, 2,  deg(mu) <= 2d,
// which determine every entry of the Gram matrix G = A^T A of
// A = [Phi | -y Phi]:  G_pp[i][j] = M_0[mu_i + mu_j],
// G_pq[i][j] = -M_1[mu_i + mu_j], G_qq[i][j] = M_2[mu_i + mu_j].
// The moments are about half the multiply-adds of a direct Gram at degree 2
// and a third at degree 3.  Lanes split the work as (sample group x moment
// group) so each lane keeps only a few accumulators in registers.  The
// moments go to the context's scratch memory.
//
// solve_lane_kernel (F3), one lane per fit: FP64 power-of-two column
// equilibration from the Gram diagonal, then shifted Cholesky factorisation
// and inverse iteration for the smallest eigenpair of the equilibrated Gram
// matrix (the smallest right singular vector of A D).  GB300 issues FP64 at
// 1/64 of the FP32 rate, so every lane works on its own fit and no FP64
// instruction is spent on a uniform value; each lane's factor lives in
// shared memory, interleaved across lanes.  A noisy fit re-factors at the
// largest shift of a ladder below the Rayleigh quotient that keeps the matrix
// positive definite, for a few rounds; deflated inverse iteration estimates
// the next eigenvalue for the rank test.
//
// solve_warp_kernel (F3 + F4), one warp per fit: the same solve done
// cooperatively by a warp, followed by optional refinement passes that
// recompute A^T A v from the samples in FP64 and take a preconditioned
// inverse-iteration step (Knyazev-Neymeyr PINVIT) with the Cholesky factor as
// preconditioner.  Used when refinement is asked for or the problem is too
// large for a lane's share of shared memory.
#include <algorithm>
#include <cfloat>
#include <type_traits>

#include <cuda_bf16.h>

#include "klr_common.cuh"
#include "klr_umma.cuh"

namespace klr {

namespace {

constexpr int kRefineMaxU = 40;         // unknowns supported by refinement passes
constexpr int kLaneMaxU = 30;           // unknowns supported by the lane-per-fit solver
constexpr int kLanczosSteps = 7;        // Lanczos steps of the group solver's first phase

enum { ACC_FP64 = 0, ACC_DF32 = 1, ACC_FP32 = 2 };

struct FitParams {
    int n_fits, n_vars, degree, m, u, n_mom;
    int box;       // per-variable degree bounds (degree: the largest bound)
    int n_scale_log2, b_scale_log2;
    const int64_t* offsets;
    const void* x;
    int64_t x_stride;
    const void* y;
    void* coef;
    int coef_f64;
    int32_t* status;
    double* diag;
    int refine;
    int ld;        // leading dimension of the Gram matrix in shared memory
    int warp_smem; // bytes of shared memory per warp
    double* mom;   // scratch: n_fits x 3 x n_mom moment sums (FP64, or
                   // double-word float2 pairs when mom_dw), or n_fits x u x u
                   // Gram matrices when gram_direct
    int mom_dw;
    int gram_direct;
    double gram_eps;  // unit roundoff of the Gram entries (sets shifts and thresholds)
    double f_jit, f_null, f_rank;   // shift, noise and rank levels as multiples of
                                    // gram_eps * trace
    int32_t* flags;// scratch: n_fits, bit 0 non-finite sample, bit 1 inexact DF32,
                   // bit 2 left to the per-sample moments kernel by the binned one
    int fallback_only;  // moments_fast_kernel: only the fits with flag bit 2
    int x_fmt;     // coordinates: kXFloat (TS), kXExp8 (uint8 base-2 logarithms,
                   // KLR_EXP8) or kXExp16 (one packed uint16 per sample, KLR_EXP16)
    int fit_warps; // solve_warp_kernel: warps per fit (> 1: one fit per block, the
                   // others join the refinement passes)
    int mom_warps; // moments_fast_kernel with FP64 sums: warps per fit (> 1: one fit
                   // per block, the warps over its samples)
    uint8_t exps[kMaxMoments][kMaxVars];
    uint8_t pair[kMaxBasis][kMaxBasis];
};

// sample coordinate formats
constexpr int kXFloat = 0;   // TS, n_vars rows
constexpr int kXExp8 = 1;    // KLR_EXP8: uint8 e per coordinate, n_vars rows
constexpr int kXExp16 = 2;   // KLR_EXP16: one uint16 per sample, log2 N in bits
                             // 0-5, log2 b0 in 6-10, log2 b1 in 11-15

// coordinate of a KLR_EXP8 (or KLR_EXP16) sample: 2^e exactly, +inf above 127
__device__ __forceinline__ float exp8_value(uint8_t e) {
    return e <= 127 ? __int_as_float((int)(e + 127u) << 23) : __int_as_float(0x7f800000);
}

// exponent field v (0: N, 1: b0, 2: b1) of a KLR_EXP16 code
__device__ __forceinline__ unsigned exp16_field(unsigned code, int v) {
    return v == 0 ? (code & 63u) : v == 1 ? ((code >> 6) & 31u) : (code >> 11);
}

// Coordinate v of sample s in two steps, so that a prefetched load is not
// waited for until its value is used: load_coord gives the raw element (a
// KLR_EXP8 byte or a KLR_EXP16 exponent field carried in the bits of a
// float), coord_value the coordinate.
template <typename TS, int XF>
__device__ __forceinline__ TS load_coord(const FitParams& P, int v, int64_t s) {
    if constexpr (XF == kXExp8) {
        static_assert(sizeof(TS) == 4, "KLR_EXP8 samples come with FP32 values");
        return __uint_as_float((unsigned)reinterpret_cast<const uint8_t*>(P.x)[(int64_t)v * P.x_stride + s]);
    } else if constexpr (XF == kXExp16) {
        static_assert(sizeof(TS) == 4, "KLR_EXP16 samples come with FP32 values");
        return __uint_as_float(exp16_field(reinterpret_cast<const uint16_t*>(P.x)[s], v));
    } else {
        return reinterpret_cast<const TS*>(P.x)[(int64_t)v * P.x_stride + s];
    }
}
template <typename TS, int XF>
__device__ __forceinline__ TS coord_value(TS raw) {
    if constexpr (XF != kXFloat) return exp8_value((uint8_t)__float_as_uint(raw));
    else return raw;
}

__device__ __forceinline__ bool is_pow2_positive(float v) {
    unsigned b = __float_as_uint(v);
    return (b & 0x007FFFFFu) == 0u && (b >> 23) != 0u && (b >> 31) == 0u;
}
__device__ __forceinline__ bool is_pow2_positive(double v) {
    unsigned long long b = __double_as_longlong(v);
    return (b & 0x000FFFFFFFFFFFFFull) == 0ull && (b >> 52) != 0ull && (b >> 63) == 0ull;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Cholesky of (Ghat - shift I), Ghat = L L^T, kept as the unit lower factor
// Lt = L diag(L)^-1 in the strict lower triangle of G (leading dim ld) and
// rinv = 1 / diag(L); the strict upper triangle keeps Ghat, gdiag its
// diagonal.  Warp-cooperative.  GB300 issues FP64 at 1/64 of the FP32 rate,
// so the count of FP64 warp instructions on the chain decides the time: one
// reciprocal square root per column, the column scaled by it, and the
// trailing update spread over the lanes pair by pair (about n^2 / 64
// instructions for an n x n trailing block, not n).
__device__ __noinline__ bool warp_cholesky(double* G, const double* gdiag, double* rinv, int u, int ld,
                              double shift) {
    const int lane = lane_id();
    for (int idx = lane; idx < u * u; idx += 32) {
        int i = idx / u, j = idx % u;
        if (i > j) G[i * ld + j] = G[j * ld + i];
        else if (i == j) G[i * ld + i] = gdiag[i] - shift;
    }
    __syncwarp();
    for (int k = 0; k < u; ++k) {
        const double akk = G[k * ld + k];
        if (!(akk > 0.0)) return false;   // uniform across the warp
        const double r = rsqrt(akk);
        for (int i = k + 1 + lane; i < u; i += 32) G[i * ld + k] *= r;
        __syncwarp();
        if (lane == 0) {
            G[k * ld + k] = akk * r;
            rinv[k] = r;
        }
        // trailing update G[i][j] -= L[i][k] L[j][k], k < j <= i: pair p of
        // the n x n lower triangle is row rr, column p - rr (rr + 1) / 2
        const int n = u - k - 1;
        for (int p = lane; p < n * (n + 1) / 2; p += 32) {
            int rr = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
            while ((rr + 1) * (rr + 2) / 2 <= p) ++rr;
            while (rr * (rr + 1) / 2 > p) --rr;
            const int i = k + 1 + rr, j = k + 1 + (p - rr * (rr + 1) / 2);
            G[i * ld + j] -= G[i * ld + k] * G[j * ld + k];
        }
        __syncwarp();
    }
    // L -> Lt: column k divided by L[k][k]
    for (int idx = lane; idx < u * u; idx += 32) {
        const int i = idx / u, j = idx % u;
        if (i > j) G[i * ld + j] *= rinv[j];
    }
    __syncwarp();
    return true;
}

// Solve Lt diag(rinv)^-2 Lt^T w = b in place (w holds b on entry), with the
// vector in registers, row i in lane i % 32: a step is one shuffle of the
// pivot and one fused multiply-add.
template <int R>
__device__ void warp_chol_solve_r(const double* G, const double* rinv, int u, int ld, double* w) {
    const unsigned full = 0xffffffffu;
    const int lane = lane_id();
    double x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = lane + 32 * r;
        x[r] = i < u ? w[i] : 0.0;
    }
#pragma unroll 4
    for (int k = 0; k < u; ++k) {
        const int kr = k >> 5;
        double src = x[0];
#pragma unroll
        for (int r = 1; r < R; ++r) if (kr == r) src = x[r];
        const double xk = __shfl_sync(full, src, k & 31);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = lane + 32 * r;
            if (i > k && i < u) x[r] = fma(-G[i * ld + k], xk, x[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = lane + 32 * r;
        if (i < u) {
            const double ri = rinv[i];
            x[r] *= ri * ri;
        }
    }
#pragma unroll 4
    for (int k = u - 1; k >= 0; --k) {
        const int kr = k >> 5;
        double src = x[0];
#pragma unroll
        for (int r = 1; r < R; ++r) if (kr == r) src = x[r];
        const double xk = __shfl_sync(full, src, k & 31);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = lane + 32 * r;
            if (i < k) x[r] = fma(-G[k * ld + i], xk, x[r]);
        }
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = lane + 32 * r;
        if (i < u) w[i] = x[r];
    }
    __syncwarp();
}

__device__ __noinline__ void warp_chol_solve(const double* G, const double* rinv, int u, int ld, double* w) {
    static_assert(2 * kMaxBasis <= 96, "three rows per lane at most");
    if (u <= 32) warp_chol_solve_r<1>(G, rinv, u, ld, w);
    else if (u <= 64) warp_chol_solve_r<2>(G, rinv, u, ld, w);
    else warp_chol_solve_r<3>(G, rinv, u, ld, w);
}

// y = Ghat v (Ghat in the strict upper triangle + gdiag).
__device__ __noinline__ void warp_gram_matvec(const double* G, const double* gdiag, int u, int ld,
                                 const double* v, double* y) {
    const int lane = lane_id();
    for (int i = lane; i < u; i += 32) {
        double acc = gdiag[i] * v[i];
        for (int j = 0; j < u; ++j)
            if (j != i) acc += G[min(i, j) * ld + max(i, j)] * v[j];
        y[i] = acc;
    }
    __syncwarp();
}

__device__ double warp_dot(const double* a, const double* b, int u) {
    double s = 0.0;
    for (int i = lane_id(); i < u; i += 32) s += a[i] * b[i];
    return warp_sum(s);
}

__device__ void warp_scale(double* a, int u, double s) {
    for (int i = lane_id(); i < u; i += 32) a[i] *= s;
    __syncwarp();
}

// w <- w - (w.v) v, then normalise.  Returns the norm before normalising.
__device__ __noinline__ double warp_orth_normalise(double* w, const double* v, int u, bool orth) {
    if (orth) {
        double c = warp_dot(w, v, u);
        for (int i = lane_id(); i < u; i += 32) w[i] -= c * v[i];
        __syncwarp();
    }
    const double n2 = warp_dot(w, w, u);
    double n = 0.0;
    if (n2 > 0.0) {
        const double rn = rsqrt(n2);
        n = n2 * rn;
        warp_scale(w, u, rn);
    }
    __syncwarp();
    return n;
}

__device__ void warp_copy(double* dst, const double* src, int u) {
    for (int i = lane_id(); i < u; i += 32) dst[i] = src[i];
    __syncwarp();
}

// Compile-time list of the monomials of total degree <= D in NV variables,
// graded, then decreasing exponent tuple (the same order as make_basis).
template <int NV, int D>
struct MonoTable {
    __host__ __device__ static constexpr int count() {
        int c = 1;
        for (int i = 1; i <= D; ++i) c = c * (NV + i) / i;
        return c;
    }
    int e[count()][4];
    __host__ __device__ constexpr MonoTable() : e{} {
        int idx = 0;
        for (int d = 0; d <= D; ++d)
            for (int a = d; a >= 0; --a)
                for (int b = (NV > 1 ? d - a : 0); b >= 0; --b)
                    for (int c = (NV > 2 ? d - a - b : 0); c >= 0; --c) {
                        const int r = d - a - b - c;
                        if (NV == 3 && r != 0) continue;
                        if (NV == 4 || r == 0) {
                            e[idx][0] = a;
                            e[idx][1] = b;
                            e[idx][2] = c;
                            e[idx][3] = NV == 4 ? r : 0;
                            ++idx;
                        }
                    }
    }
};

// moments_kernel specialised on the basis: the staging lane computes all
// n_mom monomials of its sample once (compile-time exponents, registers
// only), and each accumulating lane reads its monomial with one load.
//
// FB (the fallback launch after the binned kernel; W = 1): a small grid whose
// warps step over the fits and take only those with flag bit 2.
template <typename TS, int ACC, int NV, int D2, int MG, int MAXT, int XF = kXFloat,
          bool FB = false>
__global__ void __launch_bounds__(128, 4)
moments_fast_kernel(const __grid_constant__ FitParams P) {
    constexpr MonoTable<NV, D2> tab{};
    constexpr int NM = MonoTable<NV, D2>::count();
    constexpr int REC = NM + 3 + ((NM + 3) % 2 == 0 ? 1 : 0);   // odd stride
    constexpr int SG = 32 / MG;
    static_assert(MG * MAXT >= NM, "too few lanes for the moments");
    using TC = typename std::conditional<ACC == ACC_FP64, double, float>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int flag_w[8];
    const int lane = lane_id();
    const int wib = threadIdx.x >> 5;
    // W > 1 (FP64 sums only): one fit per block, warp hw takes every W-th tile
    const int W = ACC == ACC_FP64 ? P.mom_warps : 1;
    const int hw = W > 1 ? wib : 0;
    // one fit per warp (W = 1) or per block (W > 1); with FB, every fit left by
    // the binned kernel (flag bit 2) from this warp's index on in steps of the
    // grid, the lanes testing 32 of those fits per load
    static_assert(!FB || ACC != ACC_FP64, "the fallback launch has one warp per fit");
    const int64_t fstep = (int64_t)gridDim.x * (blockDim.x >> 5);
    auto next_left = [&](int64_t g) -> int {
        for (; g < P.n_fits; g += 32 * fstep) {
            const int64_t cand = g + lane * fstep;
            const unsigned hit =
                __ballot_sync(0xffffffffu, cand < P.n_fits && (P.flags[cand] & 4) != 0);
            if (hit) return (int)(g + (__ffs(hit) - 1) * fstep);
        }
        return P.n_fits;
    };
    int f = W > 1 ? (int)blockIdx.x : blockIdx.x * (blockDim.x >> 5) + wib;
    if constexpr (FB) f = next_left(f);
    if (f >= P.n_fits) return;
    do {
        TC* stage = reinterpret_cast<TC*>(smem_raw + (size_t)wib * P.warp_smem);
        const int64_t s0 = P.offsets[f] + 32 * hw, s1 = P.offsets[f + 1];
        const TS* Y = reinterpret_cast<const TS*>(P.y);
        const TC sN = (TC)ldexpf(1.0f, -P.n_scale_log2), sB = (TC)ldexpf(1.0f, -P.b_scale_log2);
        const int mg = lane % MG, sg = lane / MG;
        TC a0[MAXT], a1[MAXT], a2[MAXT];
        float c0[MAXT], c1[MAXT], c2[MAXT];
    #pragma unroll
        for (int i = 0; i < MAXT; ++i) {
            a0[i] = a1[i] = a2[i] = TC(0);
            c0[i] = c1[i] = c2[i] = 0.f;
        }
        bool bad = false, inexact = false;
        TS cx[NV], cy = TS(0), nx[NV], ny = TS(0);
    #pragma unroll
        for (int v = 0; v < NV; ++v) cx[v] = nx[v] = TS(1);
        if (s0 + lane < s1) {
    #pragma unroll
            for (int v = 0; v < NV; ++v) cx[v] = load_coord<TS, XF>(P, v, s0 + lane);
            cy = Y[s0 + lane];
        }
        for (int64_t base = s0; base < s1; base += 32 * W) {
            const int64_t s = base + lane;
            const int64_t sn = s + 32 * W;
            if (sn < s1) {
    #pragma unroll
                for (int v = 0; v < NV; ++v) nx[v] = load_coord<TS, XF>(P, v, sn);
                ny = Y[sn];
            }
            if (s < s1) {
                TC pw[NV][D2 + 1];
    #pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const TS raw = coord_value<TS, XF>(cx[v]);
                    bad |= !isfinite(raw);
                    if constexpr (ACC == ACC_DF32) inexact |= !is_pow2_positive(raw);
                    const TC xv = (TC)raw * (v == 0 ? sN : sB);
                    pw[v][0] = TC(1);
    #pragma unroll
                    for (int k = 1; k <= D2; ++k) pw[v][k] = pw[v][k - 1] * xv;
                }
                TC* r = stage + lane * REC;
    #pragma unroll
                for (int t = 0; t < NM; ++t) {
                    TC x = pw[0][tab.e[t][0]] * pw[1][tab.e[t][1]];
                    if constexpr (NV > 2) x *= pw[2][tab.e[t][2]];
                    if constexpr (NV > 3) x *= pw[3][tab.e[t][3]];
                    r[t] = x;
                }
                bad |= !isfinite(cy);
                const TC yv = (TC)cy;
                const TC y2h = yv * yv;
                TC y2l = TC(0);
                if constexpr (ACC != ACC_FP64) y2l = fmaf(yv, yv, -y2h);
                r[NM + 0] = yv;
                r[NM + 1] = y2h;
                r[NM + 2] = y2l;
            }
    #pragma unroll
            for (int v = 0; v < NV; ++v) cx[v] = nx[v];
            cy = ny;
            __syncwarp();
            const int nvalid = (int)min((int64_t)32, s1 - base);
            for (int ts = sg; ts < nvalid; ts += SG) {
                const TC* r = stage + ts * REC;
                const TC yv = r[NM + 0], y2h = r[NM + 1], y2l = r[NM + 2];
    #pragma unroll
                for (int i = 0; i < MAXT; ++i) {
                    const int mu = mg + MG * i;
                    if (mu < NM) {
                        const TC xm = r[mu];
                        if constexpr (ACC == ACC_FP64) {
                            a0[i] += xm;
                            a1[i] = fma(yv, xm, a1[i]);
                            a2[i] = fma(y2h, xm, a2[i]);
                        } else if constexpr (ACC == ACC_DF32) {
                            df_add(a0[i], c0[i], xm);
                            df_add(a1[i], c1[i], __fmul_rn(yv, xm));
                            df_add(a2[i], c2[i], __fmul_rn(y2h, xm));
                            c2[i] = fmaf(y2l, xm, c2[i]);
                        } else {
                            a0[i] += xm;
                            a1[i] = fmaf(yv, xm, a1[i]);
                            a2[i] = fmaf(y2h, xm, a2[i]);
                        }
                    }
                }
            }
            __syncwarp();
        }
    #pragma unroll
        for (int i = 0; i < MAXT; ++i) {
    #pragma unroll
            for (int o = MG; o < 32; o <<= 1) {
                if constexpr (ACC == ACC_DF32) {
                    float h, e;
                    float oh0 = __shfl_xor_sync(0xffffffffu, a0[i], o);
                    float ol0 = __shfl_xor_sync(0xffffffffu, c0[i], o);
                    two_sum(a0[i], oh0, h, e);
                    a0[i] = h; c0[i] = c0[i] + ol0 + e;
                    float oh1 = __shfl_xor_sync(0xffffffffu, a1[i], o);
                    float ol1 = __shfl_xor_sync(0xffffffffu, c1[i], o);
                    two_sum(a1[i], oh1, h, e);
                    a1[i] = h; c1[i] = c1[i] + ol1 + e;
                    float oh2 = __shfl_xor_sync(0xffffffffu, a2[i], o);
                    float ol2 = __shfl_xor_sync(0xffffffffu, c2[i], o);
                    two_sum(a2[i], oh2, h, e);
                    a2[i] = h; c2[i] = c2[i] + ol2 + e;
                } else {
                    a0[i] += __shfl_xor_sync(0xffffffffu, a0[i], o);
                    a1[i] += __shfl_xor_sync(0xffffffffu, a1[i], o);
                    a2[i] += __shfl_xor_sync(0xffffffffu, a2[i], o);
                }
            }
        }
        bad = __any_sync(0xffffffffu, bad);
        inexact = __any_sync(0xffffffffu, inexact);
        if constexpr (ACC == ACC_FP64) {
            if (W > 1) {
                // the warps' sums, added by warp 0 in warp order
                double* part = reinterpret_cast<double*>(smem_raw + (size_t)W * P.warp_smem);
                if (sg == 0) {
    #pragma unroll
                    for (int i = 0; i < MAXT; ++i) {
                        const int mu = mg + MG * i;
                        if (mu < NM) {
                            part[hw * 3 * NM + mu] = a0[i];
                            part[hw * 3 * NM + NM + mu] = a1[i];
                            part[hw * 3 * NM + 2 * NM + mu] = a2[i];
                        }
                    }
                }
                if (lane == 0) flag_w[hw] = (bad ? 1 : 0) | (inexact ? 2 : 0);
                __syncthreads();
                if (hw != 0) return;
                double* mom = P.mom + (int64_t)f * 3 * NM;
                for (int idx = lane; idx < 3 * NM; idx += 32) {
                    double acc = part[idx];
                    for (int g = 1; g < W; ++g) acc += part[g * 3 * NM + idx];
                    mom[idx] = acc;
                }
                if (lane == 0) {
                    int fl = 0;
                    for (int g = 0; g < W; ++g) fl |= flag_w[g];
                    P.flags[f] = fl;
                }
                return;
            }
        }
        if (sg == 0) {
            double* mom = P.mom + (int64_t)f * 3 * NM;
    #pragma unroll
            for (int i = 0; i < MAXT; ++i) {
                const int mu = mg + MG * i;
                if (mu < NM) {
                    if constexpr (ACC == ACC_FP64) {
                        mom[mu] = a0[i];
                        mom[NM + mu] = a1[i];
                        mom[2 * NM + mu] = a2[i];
                    } else {
                        float2* m2 = reinterpret_cast<float2*>(mom);
                        const dw q0 = dw_2sum(a0[i], c0[i]), q1 = dw_2sum(a1[i], c1[i]),
                                 q2 = dw_2sum(a2[i], c2[i]);
                        m2[mu] = make_float2(q0.h, q0.l);
                        m2[NM + mu] = make_float2(q1.h, q1.l);
                        m2[2 * NM + mu] = make_float2(q2.h, q2.l);
                    }
                }
            }
        }
        if (lane == 0) P.flags[f] = (bad ? 1 : 0) | (inexact ? 2 : 0);
        if constexpr (!FB) break;
        f = next_left((int64_t)f + fstep);
    } while (f < P.n_fits);
}

// ---------------------------------------------------------------------------
// Moments through per-cell sums (degree 2 in (N, b0, b1), double-FP32, FP32
// samples whose coordinates are powers of two).
//
// With x_N = N 2^-ns = 2^-t and b = (2^e0, 2^e1), the monomial x^mu of a
// sample, mu = (a, i, j), is the power of two 2^(-a t + i (e0 - bs) + j (e1 - bs)).
// Samples that share a cell (t, e0, e1) therefore contribute
//     M_k[mu] = sum_cells 2^(-a t + i (e0 - bs) + j (e1 - bs)) S_k[cell],
//     S_k[cell] = sum_{s in cell} y_s^k   (k = 0, 1, 2).
// A warp owns one fit at a time (a persistent grid strides over the fits).
// It streams the samples once, adding (1, y, y^2) into its cell's
// double-FP32 sums in shared memory (2 double-word additions per sample
// instead of 105 moment updates), then folds: over t for each block shape,
//     F_k[shape][a] = sum_t 2^-at S_k[t][shape],
// then over the shapes for each moment.  Every scaling is by a power of two
// (exact), so the roundings are those of double-word sums, as in the direct
// accumulation.  Cells: 16 octaves of N, t = ns - log2 N in 0..15, times the
// 51 block shapes of 32..1024 threads.  A fit with any sample outside that
// set (another N or shape, a coordinate that is not a power of two, a
// non-finite value) or with more than 65,535 samples (the cell counts are 16
// bits) is marked with flag bit 2 and left to moments_fast_kernel, which then
// runs over the marked fits only.
// ---------------------------------------------------------------------------
constexpr int kBinT = 16;                 // octaves of N per fit
constexpr int kBinS = 51;                 // block shapes (b0, b1), 5 <= log2 b0 b1 <= 10
constexpr int kBinC = kBinT * kBinS;      // cells
constexpr int kBinU = 4;                  // 32-sample tiles per load batch
constexpr size_t kBinWarpSmem = (size_t)kBinC * (sizeof(float4) + sizeof(uint16_t));
constexpr int64_t kBinMaxSamples = 65535;   // per fit: a cell count fits in 16 bits

__constant__ MonoTable<3, 4> c_mono34{};

// index of shape (2^e0, 2^e1) among the 51 cell shapes, ordered by thread
// count 2^(e0 + e1), then by decreasing b0; for 5 <= e0 + e1 <= 10, e0, e1 >= 0
__device__ __forceinline__ int bin_shape_index(int e0, int e1) {
    const int T = e0 + e1;
    return T * (T + 1) / 2 - 15 + (T - e0);
}

__device__ __forceinline__ float pow2f(int e) {   // 2^e for -126 <= e <= 127
    return __int_as_float((127 + e) << 23);
}

// (h, l) += v * p for a power of two p (exact product), TwoSum on the high part
__device__ __forceinline__ void dw_acc_scaled(float& h, float& l, float vh, float vl, float p) {
    float s, e;
    two_sum(h, __fmul_rn(vh, p), s, e);
    h = s;
    l = __fadd_rn(l, __fadd_rn(e, __fmul_rn(vl, p)));
}

// dw_acc_scaled on packed pairs
__device__ __forceinline__ void dw_acc_scaled2(f2p& h, f2p& l, f2p vh, f2p vl, f2p p) {
    f2p s, e;
    two_sum2(h, f2p_mul(vh, p), s, e);
    h = s;
    l = f2p_add(l, f2p_add(e, f2p_mul(vl, p)));
}

template <int XF>
__global__ void __launch_bounds__(32)
moments_binned_kernel(const __grid_constant__ FitParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = lane_id();
    const unsigned full = 0xffffffffu;
    const unsigned lt = (1u << lane) - 1u;
    // per warp: float4 (sum y hi, lo, sum y^2 hi, lo) and the 16-bit count per
    // cell; after the first fold the float4 region holds F as float2 [3][5][51]
    float4* cv = reinterpret_cast<float4*>(smem_raw);
    uint16_t* cn = reinterpret_cast<uint16_t*>(cv + kBinC);
    unsigned* cnw = reinterpret_cast<unsigned*>(cn);   // the counts of cells 2w, 2w + 1
    float2* Fs = reinterpret_cast<float2*>(cv);
    const float* Y = reinterpret_cast<const float*>(P.y);
    const int ns = P.n_scale_log2, bs = P.b_scale_log2;
    for (int f = blockIdx.x; f < P.n_fits; f += gridDim.x) {
        const int64_t s0 = P.offsets[f], s1 = P.offsets[f + 1];
        for (int c = lane; c < kBinC; c += 32) cv[c] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int w = lane; w < kBinC / 2; w += 32) cnw[w] = 0u;
        __syncwarp();
        bool fallback = s1 - s0 > kBinMaxSamples;
        // ---- stream: two batches of kBinU tiles in flight ----------------------
        // (32-bit sample indices within the fit: at most kBinMaxSamples)
        const int ns_f = fallback ? 0 : (int)(s1 - s0);
        const float* Yf = Y + s0;
        const unsigned char* xb[3];
        constexpr int64_t xes = XF == kXFloat ? 4 : XF == kXExp8 ? 1 : 2;   // bytes per element
#pragma unroll
        for (int v = 0; v < 3; ++v)
            xb[v] = reinterpret_cast<const unsigned char*>(P.x) +
                    ((XF == kXExp16 ? 0 : (int64_t)v * P.x_stride) + s0) * xes;
        float nb[kBinU][4] = {};
        auto load = [&](int base, float (&b)[kBinU][4]) {
#pragma unroll
            for (int u = 0; u < kBinU; ++u) {
                const int si = base + u * 32 + lane;
                if (si < ns_f) {
                    if constexpr (XF == kXExp16) {
                        b[u][0] = __uint_as_float(
                            (unsigned)reinterpret_cast<const uint16_t*>(xb[0])[si]);
                    } else {
#pragma unroll
                        for (int v = 0; v < 3; ++v) {
                            if constexpr (XF == kXExp8) b[u][v] = __uint_as_float((unsigned)xb[v][si]);
                            else b[u][v] = reinterpret_cast<const float*>(xb[v])[si];
                        }
                    }
                    b[u][3] = Yf[si];
                }
            }
        };
        load(0, nb);
        for (int base = 0; base < ns_f && !fallback; base += 32 * kBinU) {
            float cb[kBinU][4];
#pragma unroll
            for (int u = 0; u < kBinU; ++u) {
                if constexpr (XF == kXExp16) {
                    const unsigned code = __float_as_uint(nb[u][0]);
#pragma unroll
                    for (int v = 0; v < 3; ++v) cb[u][v] = exp8_value((uint8_t)exp16_field(code, v));
                } else {
#pragma unroll
                    for (int v = 0; v < 3; ++v) cb[u][v] = coord_value<float, XF>(nb[u][v]);
                }
                cb[u][3] = nb[u][3];
            }
            if (base + 32 * kBinU < ns_f) load(base + 32 * kBinU, nb);
#pragma unroll
            for (int u = 0; u < kBinU; ++u) {
                if (base + u * 32 >= ns_f) break;   // (uniform)
                const bool live = base + u * 32 + lane < ns_f;
                int cell = -1 - lane;   // distinct for idle lanes
                bool ok = true;
                if (live) {
                    const unsigned un = __float_as_uint(cb[u][0]);
                    const unsigned u0 = __float_as_uint(cb[u][1]);
                    const unsigned u1 = __float_as_uint(cb[u][2]);
                    // positive powers of two: sign and mantissa bits clear (zero
                    // and infinity fail the range tests below)
                    const bool p2 = ((un | u0 | u1) & 0x807FFFFFu) == 0u;
                    const int t = ns - ((int)(un >> 23) - 127);
                    const int e0 = (int)(u0 >> 23) - 127, e1 = (int)(u1 >> 23) - 127;
                    const int T = e0 + e1;
                    ok = p2 && t >= 0 && t < kBinT && e0 >= 0 && e1 >= 0 && T >= 5 && T <= 10 &&
                         isfinite(cb[u][3]);
                    if (ok) cell = t * kBinS + bin_shape_index(e0, e1);
                }
                if (__any_sync(full, !ok)) {
                    fallback = true;
                    break;
                }
                // the count by a shared-memory atomic (16-bit halves: at most
                // kBinMaxSamples per cell); lanes with the same cell add their
                // values one after the other
                if (live) atomicAdd(&cnw[cell >> 1], 1u << ((cell & 1) << 4));
                const unsigned peers = __match_any_sync(full, cell);
                const unsigned rank = __popc(peers & lt);
                const unsigned rounds = __reduce_max_sync(full, rank) + 1u;
                const float y = cb[u][3];
                const float y2h = __fmul_rn(y, y);
                const float y2l = fmaf(y, y, -y2h);
                for (unsigned r = 0; r < rounds; ++r) {
                    if (live && rank == r) {
                        float4 v = cv[cell];
                        float hs, e;
                        two_sum(v.x, y, hs, e);
                        v.x = hs;
                        v.y = __fadd_rn(v.y, e);
                        two_sum(v.z, y2h, hs, e);
                        v.z = hs;
                        v.w = __fadd_rn(v.w, __fadd_rn(e, y2l));
                        cv[cell] = v;
                    }
                    __syncwarp();
                }
            }
            if (fallback) break;
        }
        if (fallback) {
            if (lane == 0) P.flags[f] = 4;
            __syncwarp();
            continue;
        }
        __syncwarp();
        // ---- fold over the octaves of N: items (k, shape) -------------------------
        // the powers a = (0, 1) and (2, 3) as packed pairs, a = 4 alone
        constexpr int R1 = (3 * kBinS + 31) / 32;
        f2p ph[R1][2], pl[R1][2];
        float fh4[R1], fl4[R1];
#pragma unroll
        for (int r = 0; r < R1; ++r) {
            const int it = r * 32 + lane;
            const int k = it / kBinS, sh = it - k * kBinS;
            ph[r][0] = ph[r][1] = pl[r][0] = pl[r][1] = 0ull;
            fh4[r] = fl4[r] = 0.f;
            if (it < 3 * kBinS) {
#pragma unroll 2
                for (int t = 0; t < kBinT; ++t) {
                    const int c = t * kBinS + sh;
                    float vh, vl;
                    if (k == 0) {
                        vh = (float)cn[c];
                        vl = 0.f;
                    } else {
                        const float4 v = cv[c];
                        vh = k == 1 ? v.x : v.z;
                        vl = k == 1 ? v.y : v.w;
                    }
                    const float pt = pow2f(-t), pt2 = pow2f(-2 * t);
                    const f2p vh2 = f2p_make(vh, vh), vl2 = f2p_make(vl, vl);
                    const f2p p01 = f2p_make(1.f, pt), p23 = f2p_mul(p01, f2p_make(pt2, pt2));
                    dw_acc_scaled2(ph[r][0], pl[r][0], vh2, vl2, p01);
                    dw_acc_scaled2(ph[r][1], pl[r][1], vh2, vl2, p23);
                    dw_acc_scaled(fh4[r], fl4[r], vh, vl, pow2f(-4 * t));
                }
            }
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < R1; ++r) {
            const int it = r * 32 + lane;
            const int k = it / kBinS, sh = it - k * kBinS;
            if (it < 3 * kBinS) {
                float2* Fk = Fs + (k * 5) * kBinS + sh;
#pragma unroll
                for (int g = 0; g < 2; ++g) {
                    const float2 h = f2p_get(ph[r][g]), l = f2p_get(pl[r][g]);
                    Fk[(2 * g) * kBinS] = make_float2(h.x, l.x);
                    Fk[(2 * g + 1) * kBinS] = make_float2(h.y, l.y);
                }
                Fk[4 * kBinS] = make_float2(fh4[r], fl4[r]);
            }
        }
        __syncwarp();
        // ---- fold over the block shapes, one exponent at a time ------------------
        // Shape (2^e0, 2^e1) scales moment (a, i, j) by 2^(i e0' + j e1'), e' =
        // e - bs.  First H[k][a, j][e0] = sum over e1 of F[k][a][shape] 2^(j e1')
        // (items as packed pairs), then moment (k; a, i, j) = sum over e0 of
        // H[k][a, j][e0] 2^(i e0'): 3 x 15 x 51 + 105 x 11 scaled additions
        // instead of 105 x 51.  (a, j) with j <= 4 - a is numbered
        // 5a - a(a - 1)/2 + j.
        constexpr int kAJ = 15, kE0 = 11, kHA = 3 * kAJ * kE0, kHP = (kHA + 1) / 2;
        float2* Hs = Fs + 3 * 5 * kBinS;              // [3][15][11] after F
#pragma unroll 1
        for (int pi = lane; pi < kHP; pi += 32) {
            int idx[2], n1[2], Tv[2];
            const float2* Fp[2];
            float p0[2], qf[2];
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                const int it = g == 0 ? pi : (pi + kHP < kHA ? pi + kHP : pi);
                const int e0 = it % kE0, r = it / kE0;
                const int k = r / kAJ;
                int aj = r - k * kAJ, a = 0;
                while (aj >= 5 - a) { aj -= 5 - a; ++a; }
                const int j = aj;
                const int e1 = e0 < 5 ? 5 - e0 : 0;   // the first shape with this e0
                n1[g] = 10 - e0 - e1 + 1;
                Tv[g] = e0 + e1;
                idx[g] = bin_shape_index(e0, e1);
                Fp[g] = Fs + (k * 5 + a) * kBinS;
                p0[g] = pow2f(j * (e1 - bs));
                qf[g] = pow2f(j);
            }
            f2p h = 0ull, l = 0ull;
            f2p p = f2p_make(p0[0], p0[1]);
            const f2p q2 = f2p_make(qf[0], qf[1]);
#pragma unroll
            for (int mstep = 0; mstep < 6; ++mstep) {
                float2 v[2];
#pragma unroll
                for (int g = 0; g < 2; ++g) {
                    v[g] = mstep < n1[g] ? Fp[g][idx[g]] : make_float2(0.f, 0.f);
                    idx[g] += Tv[g] + 2;   // index of (e0, e1 + 1): T (T + 1) / 2 grows by T + 1
                    Tv[g] += 1;
                }
                dw_acc_scaled2(h, l, f2p_make(v[0].x, v[1].x), f2p_make(v[0].y, v[1].y), p);
                p = f2p_mul(p, q2);
            }
            const float2 hh = f2p_get(h), ll = f2p_get(l);
            const dw r0 = dw_2sum(hh.x, ll.x);
            Hs[pi] = make_float2(r0.h, r0.l);
            if (pi + kHP < kHA) {
                const dw r1 = dw_2sum(hh.y, ll.y);
                Hs[pi + kHP] = make_float2(r1.h, r1.l);
            }
        }
        __syncwarp();
        float2* mom = reinterpret_cast<float2*>(P.mom) + (int64_t)f * 3 * 35;
#pragma unroll 1
        for (int it = lane; it < 53; it += 32) {
            const int i2 = it + 53;                 // item 105 does not exist
            const bool two = i2 < 3 * 35;
            const int items[2] = {it, two ? i2 : it};
            const float2* Hp[2];
            float p0[2], qf[2];
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                const int kk = items[g] / 35, mu = items[g] - kk * 35;
                const int a = c_mono34.e[mu][0], i = c_mono34.e[mu][1], j = c_mono34.e[mu][2];
                Hp[g] = Hs + (kk * kAJ + 5 * a - a * (a - 1) / 2 + j) * kE0;
                p0[g] = pow2f(-i * bs);
                qf[g] = pow2f(i);
            }
            f2p h = 0ull, l = 0ull;
            f2p p = f2p_make(p0[0], p0[1]);
            const f2p q2 = f2p_make(qf[0], qf[1]);
#pragma unroll
            for (int e0 = 0; e0 < kE0; ++e0) {
                const float2 v0 = Hp[0][e0], v1 = Hp[1][e0];
                dw_acc_scaled2(h, l, f2p_make(v0.x, v1.x), f2p_make(v0.y, v1.y), p);
                p = f2p_mul(p, q2);
            }
            const float2 hh = f2p_get(h), ll = f2p_get(l);
            const dw q0 = dw_2sum(hh.x, ll.x);
            mom[it] = make_float2(q0.h, q0.l);
            if (two) {
                const dw q1 = dw_2sum(hh.y, ll.y);
                mom[i2] = make_float2(q1.h, q1.l);
            }
        }
        if (lane == 0) P.flags[f] = 0;
        __syncwarp();
    }
}

template <typename TS, int ACC, int MG, int MAXT>
__global__ void __launch_bounds__(128, 4)
moments_kernel(const __grid_constant__ FitParams P) {
    constexpr int SG = 32 / MG;
    using TC = typename std::conditional<ACC == ACC_FP64, double, float>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = lane_id();
    const int wib = threadIdx.x >> 5;
    const int f = blockIdx.x * (blockDim.x >> 5) + wib;
    if (f >= P.n_fits) return;
    unsigned char* wsm = smem_raw + (size_t)wib * P.warp_smem;

    const int nv = P.n_vars, d = P.degree, n_mom = P.n_mom;
    const int PW = 2 * d + 1;              // powers 0..2d per variable
    const int REC = nv * PW + 3;           // powers + (y, y^2 hi, y^2 lo)
    TC* stage = reinterpret_cast<TC*>(wsm);
    double* mom = P.mom + (int64_t)f * 3 * n_mom;

    const int64_t s0 = P.offsets[f], s1 = P.offsets[f + 1];
    const TS* X = reinterpret_cast<const TS*>(P.x);
    const TS* Y = reinterpret_cast<const TS*>(P.y);
    const double n_scale = ldexp(1.0, -P.n_scale_log2);
    const double b_scale = ldexp(1.0, -P.b_scale_log2);

    // ---- F1 + F2: stream samples, accumulate moments ------------------------
    const int mg = lane % MG, sg = lane / MG;
    // offsets into a staged record of the powers that make up each of this
    // lane's moments, one byte per variable
    unsigned off[MAXT];
    int my_n = 0;
#pragma unroll
    for (int i = 0; i < MAXT; ++i) {
        int mu = mg + MG * i;
        if (mu < n_mom) my_n = i + 1;
        unsigned o = 0;
#pragma unroll
        for (int vv = 0; vv < kMaxVars; ++vv)
            o |= (unsigned)((mu < n_mom && vv < nv) ? vv * PW + P.exps[mu][vv] : 0) << (8 * vv);
        off[i] = o;
    }
    TC a0[MAXT], a1[MAXT], a2[MAXT];
    float c0[MAXT], c1[MAXT], c2[MAXT];
#pragma unroll
    for (int i = 0; i < MAXT; ++i) {
        a0[i] = a1[i] = a2[i] = TC(0);
        c0[i] = c1[i] = c2[i] = 0.f;
    }
    bool bad = false, inexact = false;
    // software pipeline: the next step's 32 samples are loaded into registers
    // while the current step's are accumulated
    const TC sN = (TC)n_scale, sB = (TC)b_scale;   // powers of two: exact scaling
    TS cx[kMaxVars], cy = TS(0), nx[kMaxVars], ny = TS(0);
#pragma unroll
    for (int vv = 0; vv < kMaxVars; ++vv) cx[vv] = nx[vv] = TS(1);
    if (s0 + lane < s1) {
#pragma unroll
        for (int vv = 0; vv < kMaxVars; ++vv)
            if (vv < nv) cx[vv] = X[(int64_t)vv * P.x_stride + s0 + lane];
        cy = Y[s0 + lane];
    }
    for (int64_t base = s0; base < s1; base += 32) {
        const int64_t s = base + lane;
        const int64_t sn = s + 32;
        if (sn < s1) {
#pragma unroll
            for (int vv = 0; vv < kMaxVars; ++vv)
                if (vv < nv) nx[vv] = X[(int64_t)vv * P.x_stride + sn];
            ny = Y[sn];
        }
        if (s < s1) {
            TC* r = stage + lane * REC;
#pragma unroll
            for (int vv = 0; vv < kMaxVars; ++vv) {
                if (vv < nv) {
                    const TS raw = cx[vv];
                    bad |= !isfinite(raw);
                    if constexpr (ACC == ACC_DF32) inexact |= !is_pow2_positive(raw);
                    const TC xv = (TC)raw * (vv == 0 ? sN : sB);
                    TC p = TC(1);
                    for (int k = 0; k < PW; ++k) {
                        r[vv * PW + k] = p;
                        p *= xv;
                    }
                }
            }
            bad |= !isfinite(cy);
            const TC yv = (TC)cy;
            const TC y2h = yv * yv;
            TC y2l = TC(0);
            if constexpr (ACC != ACC_FP64) y2l = fmaf(yv, yv, -y2h);
            r[nv * PW + 0] = yv;
            r[nv * PW + 1] = y2h;
            r[nv * PW + 2] = y2l;
        }
#pragma unroll
        for (int vv = 0; vv < kMaxVars; ++vv) cx[vv] = nx[vv];
        cy = ny;
        __syncwarp();
        const int nvalid = (int)min((int64_t)32, s1 - base);
        for (int ts = sg; ts < nvalid; ts += SG) {
            const TC* r = stage + ts * REC;
            const TC yv = r[nv * PW + 0], y2h = r[nv * PW + 1], y2l = r[nv * PW + 2];
#pragma unroll
            for (int i = 0; i < MAXT; ++i) {
                if (i < my_n) {
                    TC xm = r[off[i] & 0xFF] * r[(off[i] >> 8) & 0xFF];
                    if (nv > 2) xm *= r[(off[i] >> 16) & 0xFF];
                    if (nv > 3) xm *= r[off[i] >> 24];
                    if constexpr (ACC == ACC_FP64) {
                        a0[i] += xm;
                        a1[i] = fma(yv, xm, a1[i]);
                        a2[i] = fma(y2h, xm, a2[i]);
                    } else if constexpr (ACC == ACC_DF32) {
                        // products of a value and a power of two are exact
                        df_add(a0[i], c0[i], xm);
                        df_add(a1[i], c1[i], yv * xm);
                        df_add(a2[i], c2[i], y2h * xm);
                        c2[i] = fmaf(y2l, xm, c2[i]);
                    } else {
                        a0[i] += xm;
                        a1[i] = fmaf(yv, xm, a1[i]);
                        a2[i] = fmaf(y2h, xm, a2[i]);
                    }
                }
            }
        }
        __syncwarp();
    }
    // reduce across sample groups (lanes mg, mg + 16)
#pragma unroll
    for (int i = 0; i < MAXT; ++i) {
#pragma unroll
        for (int o = MG; o < 32; o <<= 1) {
            if constexpr (ACC == ACC_DF32) {
                float h, e;
                float oh0 = __shfl_xor_sync(0xffffffffu, a0[i], o);
                float ol0 = __shfl_xor_sync(0xffffffffu, c0[i], o);
                two_sum(a0[i], oh0, h, e);
                a0[i] = h; c0[i] = c0[i] + ol0 + e;
                float oh1 = __shfl_xor_sync(0xffffffffu, a1[i], o);
                float ol1 = __shfl_xor_sync(0xffffffffu, c1[i], o);
                two_sum(a1[i], oh1, h, e);
                a1[i] = h; c1[i] = c1[i] + ol1 + e;
                float oh2 = __shfl_xor_sync(0xffffffffu, a2[i], o);
                float ol2 = __shfl_xor_sync(0xffffffffu, c2[i], o);
                two_sum(a2[i], oh2, h, e);
                a2[i] = h; c2[i] = c2[i] + ol2 + e;
            } else {
                a0[i] += __shfl_xor_sync(0xffffffffu, a0[i], o);
                a1[i] += __shfl_xor_sync(0xffffffffu, a1[i], o);
                a2[i] += __shfl_xor_sync(0xffffffffu, a2[i], o);
            }
        }
    }
    bad = __any_sync(0xffffffffu, bad);
    inexact = __any_sync(0xffffffffu, inexact);
    if (sg == 0) {
#pragma unroll
        for (int i = 0; i < MAXT; ++i) {
            if (i < my_n) {
                int mu = mg + MG * i;
                if constexpr (ACC == ACC_FP64) {
                    mom[mu] = a0[i];
                    mom[n_mom + mu] = a1[i];
                    mom[2 * n_mom + mu] = a2[i];
                } else {
                    // normalised double-word pairs (c is 0 in FP32 mode)
                    float2* m2 = reinterpret_cast<float2*>(mom);
                    const dw s0 = dw_2sum(a0[i], c0[i]), s1 = dw_2sum(a1[i], c1[i]),
                             s2 = dw_2sum(a2[i], c2[i]);
                    m2[mu] = make_float2(s0.h, s0.l);
                    m2[n_mom + mu] = make_float2(s1.h, s1.l);
                    m2[2 * n_mom + mu] = make_float2(s2.h, s2.l);
                }
            }
        }
    }
    if (lane == 0) P.flags[f] = (bad ? 1 : 0) | (inexact ? 2 : 0);
}

// Sums of K values over the 32 lanes (K = 32 or 64): halve the values at
// each of the five exchange distances, each lane keeping the half its lane
// bit selects, so that K - K/32 additions replace 5 K of one warp_sum per
// value.  On return a[i], i < K/32, holds the sum of value (K/32) lane + i.
template <int K>
__device__ __forceinline__ void warp_reduce_scatter(double (&a)[K]) {
    const int lane = lane_id();
#pragma unroll
    for (int lvl = 0; lvl < 5; ++lvl) {
        const int o = 16 >> lvl, half = K >> (lvl + 1);
        const bool hi = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const double keep = hi ? a[i + half] : a[i];
            const double send = hi ? a[i] : a[i + half];
            a[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
}

template <typename TS>
__global__ void __launch_bounds__(128)
solve_warp_kernel(const __grid_constant__ FitParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = lane_id();
    const int wib = threadIdx.x >> 5;
    const int H = P.fit_warps;                  // warps per fit
    const int h = H > 1 ? wib : 0;              // this warp's rank within its fit
    const int f = H > 1 ? (int)blockIdx.x : blockIdx.x * (blockDim.x >> 5) + wib;
    if (f >= P.n_fits) return;
    const int nv = P.n_vars, m = P.m, u = P.u, n_mom = P.n_mom, ld = P.ld;
    double* mom = reinterpret_cast<double*>(smem_raw + (size_t)(H > 1 ? 0 : wib) * P.warp_smem);
    double* part = reinterpret_cast<double*>(smem_raw + P.warp_smem);   // H x 64 (H > 1)
    __shared__ int ok_s;
    double* G = mom + 3 * n_mom;
    double* gdiag = G + u * ld;
    double* D = gdiag + u;
    double* v = D + u;
    double* w = v + u;
    double* t = w + u;
    double* rinv = t + u;
    const int64_t s0 = P.offsets[f], s1 = P.offsets[f + 1];
    const TS* X = reinterpret_cast<const TS*>(P.x);
    const TS* Y = reinterpret_cast<const TS*>(P.y);
    const double n_scale = ldexp(1.0, -P.n_scale_log2);
    const double b_scale = ldexp(1.0, -P.b_scale_log2);
    for (int i = lane; i < 3 * n_mom && !P.gram_direct && h == 0; i += 32) {
        if (P.mom_dw) {
            const float2 g = reinterpret_cast<const float2*>(P.mom)[(int64_t)f * 3 * n_mom + i];
            mom[i] = (double)g.x + (double)g.y;
        } else {
            mom[i] = P.mom[(int64_t)f * 3 * n_mom + i];
        }
    }
    const int32_t fl = P.flags[f];
    const bool bad = fl & 1, inexact = fl & 2;
    __syncwarp();

    const int64_t S = s1 - s0;
    int32_t status = 0;
    if (S == 0) status = KLR_FIT_EMPTY;
    else if (bad) status = KLR_FIT_NONFINITE;
    if (status) {
        if (h != 0) return;
        for (int j = lane; j < u; j += 32) {
            if (P.coef_f64) reinterpret_cast<double*>(P.coef)[(int64_t)f * u + j] = 0.0;
            else reinterpret_cast<float*>(P.coef)[(int64_t)f * u + j] = 0.f;
        }
        if (lane == 0) {
            P.status[f] = status;
            if (P.diag) for (int k = 0; k < 4; ++k) P.diag[(int64_t)f * 4 + k] = 0.0;
        }
        return;
    }
    if (inexact) status |= KLR_FIT_INEXACT;

    bool ok = false;
    double trace = 0.0, theta = 0.0, theta2 = 0.0;
    if (h == 0) {
        // ---- assemble the Gram matrix (upper triangle + diagonal) ---------------
        for (int idx = lane; idx < u * u; idx += 32) {
            int i = idx / u, j = idx % u;
            if (j < i) continue;
            double val;
            if (P.gram_direct) {
                val = P.mom[((int64_t)f * u + i) * u + j];
            } else {
                int bi = i >= m, bj = j >= m;
                val = mom[(bi + bj) * n_mom + P.pair[i - bi * m][j - bj * m]];
                if (bi != bj) val = -val;
            }
            if (i == j) gdiag[i] = val;
            else G[i * ld + j] = val;
        }
        __syncwarp();
        // power-of-two equilibration: D_j = 2^-floor(e_j / 2), e_j = frexp exponent of G_jj
        for (int j = lane; j < u; j += 32) {
            double g = gdiag[j];
            double dj = 1.0;
            if (g > 0.0) {
                int e;
                frexp(g, &e);
                dj = ldexp(1.0, -(e >> 1));
            }
            D[j] = dj;
        }
        __syncwarp();
        for (int idx = lane; idx < u * u; idx += 32) {
            int i = idx / u, j = idx % u;
            if (j < i) continue;
            if (i == j) gdiag[i] *= D[i] * D[i];
            else G[i * ld + j] *= D[i] * D[j];
        }
        __syncwarp();
        trace = 0.0;
        for (int i = lane; i < u; i += 32) trace += gdiag[i];
        trace = warp_sum(trace);

        // ---- F3: smallest eigenpair by shifted inverse iteration ----------------
        const double eps = P.gram_eps;
        const double jitter = P.f_jit * eps * trace;
        double shift = -jitter;                       // factor Ghat + jitter I
        ok = warp_cholesky(G, gdiag, rinv, u, ld, shift);
        if (!ok) {
            shift = -1024.0 * jitter;
            ok = warp_cholesky(G, gdiag, rinv, u, ld, shift);
        }
        if (!ok) {
            status |= KLR_FIT_SOLVE_FAILED;
        }
        for (int i = lane; i < u; i += 32) v[i] = 1.0 + 0.0625 * (double)((i * 7) % 11);
        __syncwarp();
        warp_orth_normalise(v, v, u, false);
        if (ok) {
            // iterate until v stops moving (a large shift, as for the low-precision
            // Gram matrices, converges slowly): change below 1e-11, or a stall
            // (rate above 1/2) below 1e-8, at most 32 steps
            double prev = 1.0;
            for (int it = 0; it < 32; ++it) {
                warp_copy(w, v, u);
                warp_chol_solve(G, rinv, u, ld, v);
                warp_orth_normalise(v, v, u, false);
                double dv2 = 0.0;
                for (int i = lane; i < u; i += 32) dv2 += (v[i] - w[i]) * (v[i] - w[i]);
                dv2 = warp_sum(dv2);
                if (it >= 2 && (dv2 <= 1e-22 || (dv2 <= 1e-16 && dv2 >= 0.25 * prev))) break;
                prev = dv2;
            }
            warp_gram_matvec(G, gdiag, u, ld, v, t);
            theta = warp_dot(v, t, u);
            if (theta > P.f_null * eps * trace) {
                // A noisy fit: the smallest eigenvalue is well above round-off.  Each
                // round factors Ghat - sigma I for the largest sigma of a ladder
                // below the Rayleigh quotient that keeps the matrix positive
                // definite (so sigma < lambda_min), then iterates; the quotient
                // moves down toward lambda_min and the next round's shift closer.
                const double ladder[8] = {1.0 - 1.0 / 64, 1.0 - 1.0 / 32, 1.0 - 1.0 / 16,
                                          1.0 - 1.0 / 8, 1.0 - 1.0 / 4, 0.5, 0.25, 0.0};
                for (int round = 0; round < 3 && ok; ++round) {
                    bool ok2 = false;
                    for (int k = 0; k < 8 && !ok2; ++k) {
                        shift = k < 7 ? theta * ladder[k] : -jitter;
                        ok2 = warp_cholesky(G, gdiag, rinv, u, ld, shift);
                    }
                    if (!ok2) {
                        status |= KLR_FIT_SOLVE_FAILED;
                        ok = false;
                        break;
                    }
                    for (int it = 0; it < 4; ++it) {
                        warp_chol_solve(G, rinv, u, ld, v);
                        warp_orth_normalise(v, v, u, false);
                    }
                    warp_gram_matvec(G, gdiag, u, ld, v, t);
                    theta = warp_dot(v, t, u);
                }
            }
        }
        // next-smallest eigenvalue: deflated inverse iteration (rank test)
        if (ok) {
            for (int i = lane; i < u; i += 32) w[i] = 1.0 + 0.03125 * (double)((i * 5) % 13) - 0.5 * (i & 1);
            __syncwarp();
            warp_orth_normalise(w, v, u, true);
            for (int it = 0; it < 3; ++it) {
                warp_chol_solve(G, rinv, u, ld, w);
                warp_orth_normalise(w, v, u, true);
            }
            warp_gram_matvec(G, gdiag, u, ld, w, t);
            theta2 = warp_dot(w, t, u);
            if (theta2 <= P.f_rank * eps * trace) status |= KLR_FIT_RANK_DEFICIENT;
        }
    }

    // ---- F4: FP64 refinement passes over the samples --------------------------
    // With H > 1 warps per fit the other warps join here: warp h takes every
    // H-th group of 32 samples, and warp 0 adds the warps' sums in warp order.
    if (H > 1) {
        if (threadIdx.x == 0) ok_s = ok;
        __syncthreads();
        ok = ok_s;
    }
    int passes = 0;
    if (ok && P.refine > 0 && u <= kRefineMaxU) {
        for (int pass = 0; pass < P.refine; ++pass) {
            constexpr int HM = kRefineMaxU / 2;
            // with w = D v (D: powers of two, so every scaling below is exact):
            // r = (A D v)_s = sum_j p_j w_j - (y_s p_j) w_{m+j}, summed term by term,
            // t_j = D_j sum_s r p_j and t_{m+j} = -D_{m+j} sum_s r (y_s p_j)
            if (h == 0) for (int i = lane; i < u; i += 32) w[i] = D[i] * v[i];
            if (H > 1) __syncthreads();
            else __syncwarp();
            double gp[HM], gq[HM];
#pragma unroll
            for (int j = 0; j < HM; ++j) gp[j] = gq[j] = 0.0;
            for (int64_t s = s0 + 32 * h + lane; s < s1; s += 32 * H) {
                double xs[kMaxVars];
                for (int vv = 0; vv < nv; ++vv)
                    xs[vv] = (double)X[(int64_t)vv * P.x_stride + s] * (vv == 0 ? n_scale : b_scale);
                const double ys = (double)Y[s];
                double pm[HM], qm[HM];
                double r = 0.0;
#pragma unroll
                for (int j = 0; j < HM; ++j) {
                    pm[j] = qm[j] = 0.0;
                    if (j < m) {
                        double p = 1.0;
                        for (int vv = 0; vv < nv; ++vv)
                            for (int e = 0; e < P.exps[j][vv]; ++e) p *= xs[vv];
                        pm[j] = p;
                        qm[j] = ys * p;
                        r = fma(p, w[j], r);
                        r = fma(-qm[j], w[m + j], r);
                    }
                }
#pragma unroll
                for (int j = 0; j < HM; ++j) {
                    if (j < m) {
                        gp[j] = fma(r, pm[j], gp[j]);
                        gq[j] = fma(r, qm[j], gq[j]);
                    }
                }
            }
            // sums over the lanes: value j of gp at slot j, of gq at slot OFF + j;
            // this lane ends with slots NL lane + i, i < NL
            double red[2];
            int NL, OFF;
            if (m <= 16) {
                double a32[32];
#pragma unroll
                for (int j = 0; j < 16; ++j) { a32[j] = gp[j]; a32[16 + j] = gq[j]; }
                warp_reduce_scatter<32>(a32);
                red[0] = a32[0];
                red[1] = 0.0;
                NL = 1;
                OFF = 16;
            } else {
                double a64[64];
#pragma unroll
                for (int j = 0; j < HM; ++j) { a64[j] = gp[j]; a64[HM + j] = gq[j]; }
#pragma unroll
                for (int j = 2 * HM; j < 64; ++j) a64[j] = 0.0;
                warp_reduce_scatter<64>(a64);
                red[0] = a64[0];
                red[1] = a64[1];
                NL = 2;
                OFF = HM;
            }
            if (H > 1) {
                for (int i = 0; i < NL; ++i) part[h * 64 + NL * lane + i] = red[i];
                __syncthreads();
                if (h == 0)
                    for (int i = 0; i < NL; ++i) {
                        double acc = part[NL * lane + i];
                        for (int g = 1; g < H; ++g) acc += part[g * 64 + NL * lane + i];
                        red[i] = acc;
                    }
            }
            if (h == 0) {
                // t = (A D)^T (A D) v
                for (int i = 0; i < NL; ++i) {
                    const int slot = NL * lane + i;
                    if (slot < OFF) {
                        if (slot < m) t[slot] = D[slot] * red[i];
                    } else if (slot - OFF < m) {
                        t[m + slot - OFF] = -D[m + slot - OFF] * red[i];
                    }
                }
                __syncwarp();
                theta = warp_dot(v, t, u);
                // residual r = A^T A v - theta v; correction w = (Ghat - shift)^-1 r,
                // orthogonal to v
                for (int i = lane; i < u; i += 32) w[i] = t[i] - theta * v[i];
                __syncwarp();
                warp_chol_solve(G, rinv, u, ld, w);
                double c = warp_dot(w, v, u);
                for (int i = lane; i < u; i += 32) v[i] -= w[i] - c * v[i];
                __syncwarp();
                warp_orth_normalise(v, v, u, false);
            }
            ++passes;
        }
    }
    if (h != 0) return;

    // ---- coefficients: c = D v, unit norm, sign rule --------------------------
    for (int i = lane; i < u; i += 32) w[i] = D[i] * v[i];
    __syncwarp();
    double nrm = sqrt(warp_dot(w, w, u));
    double sgn = 1.0;
    {
        double q0 = w[m] / nrm;
        if (fabs(q0) >= 1e-12) {
            sgn = q0 > 0.0 ? 1.0 : -1.0;
        } else {
            // largest-magnitude denominator coefficient (first on ties) positive
            double best = -1.0;
            int bi = m;
            for (int j = m; j < u; ++j)
                if (fabs(w[j]) > best) { best = fabs(w[j]); bi = j; }
            sgn = w[bi] > 0.0 ? 1.0 : -1.0;
        }
    }
    const double scale = ok ? sgn / nrm : 0.0;
    for (int j = lane; j < u; j += 32) {
        double cj = w[j] * scale;
        if (P.coef_f64) reinterpret_cast<double*>(P.coef)[(int64_t)f * u + j] = cj;
        else reinterpret_cast<float*>(P.coef)[(int64_t)f * u + j] = (float)cj;
    }
    if (lane == 0) {
        P.status[f] = status;
        if (P.diag) {
            double* dg = P.diag + (int64_t)f * 4;
            dg[0] = trace > 0 ? theta / trace : 0.0;
            dg[1] = trace > 0 ? theta2 / trace : 0.0;
            dg[2] = sqrt(fmax(theta, 0.0) / (double)S) / nrm;
            dg[3] = (double)passes;
        }
    }
}



// One lane per fit.  Shared memory holds, per lane and interleaved across the
// 32 lanes of the block (element e of lane l at [e * 32 + l]): the packed
// lower Cholesky factor, the reciprocal diagonal, D, v and w.
__global__ void __launch_bounds__(32)
solve_lane_kernel(const __grid_constant__ FitParams P) {
    extern __shared__ __align__(16) double lsm[];
    const int lane = threadIdx.x;
    const int f = blockIdx.x * 32 + lane;
    if (f >= P.n_fits) return;
    const int m = P.m, u = P.u, n_mom = P.n_mom;
    const int nL = u * (u + 1) / 2;
    double* Lf = lsm;                 // packed: (i, j), j <= i at i (i + 1) / 2 + j
    double* rinv = Lf + nL * 32;
    double* Dv = rinv + u * 32;
    double* vv = Dv + u * 32;
    double* wv = vv + u * 32;
#define LF(i, j) Lf[((i) * ((i) + 1) / 2 + (j)) * 32 + lane]
#define RI(i) rinv[(i) * 32 + lane]
#define DD(i) Dv[(i) * 32 + lane]
#define VV(i) vv[(i) * 32 + lane]
#define WV(i) wv[(i) * 32 + lane]
    const double* M = P.mom + (int64_t)f * 3 * n_mom;
    const int64_t S = P.offsets[f + 1] - P.offsets[f];
    const int32_t fl = P.flags[f];
    int32_t status = 0;
    if (S == 0) status = KLR_FIT_EMPTY;
    else if (fl & 1) status = KLR_FIT_NONFINITE;
    if (status) {
        for (int j = 0; j < u; ++j) {
            if (P.coef_f64) reinterpret_cast<double*>(P.coef)[(int64_t)f * u + j] = 0.0;
            else reinterpret_cast<float*>(P.coef)[(int64_t)f * u + j] = 0.f;
        }
        P.status[f] = status;
        if (P.diag) for (int k = 0; k < 4; ++k) P.diag[(int64_t)f * 4 + k] = 0.0;
        return;
    }
    if (fl & 2) status |= KLR_FIT_INEXACT;
    // equilibration from the Gram diagonal (families 0 and 2 have sign +)
    double trace = 0.0;
    for (int j = 0; j < u; ++j) {
        const int bj = j >= m, jj = j - bj * m;
        const double g = __ldg(M + 2 * bj * n_mom + P.pair[jj][jj]);
        double dj = 1.0;
        if (g > 0.0) {
            int e;
            frexp(g, &e);
            dj = ldexp(1.0, -(e >> 1));
        }
        DD(j) = dj;
        trace += g * dj * dj;
    }
    // entry (i, j) of the equilibrated Gram matrix, assembled from the moments
    auto gh = [&](int i, int j) -> double {
        const int bi = i >= m, bj = j >= m;
        double val = __ldg(M + (bi + bj) * n_mom + P.pair[i - bi * m][j - bj * m]);
        if (bi != bj) val = -val;
        return val * DD(i) * DD(j);
    };
    // Cholesky of (Ghat - shift I); false if a pivot is not positive
    // (two partial sums in the inner products keep two FP64 chains in flight)
    auto cholesky = [&](double shift) -> bool {
        for (int j = 0; j < u; ++j) {
            double s0 = gh(j, j) - shift, s1 = 0.0;
            int k = 0;
            for (; k + 1 < j; k += 2) {
                s0 -= LF(j, k) * LF(j, k);
                s1 -= LF(j, k + 1) * LF(j, k + 1);
            }
            if (k < j) s0 -= LF(j, k) * LF(j, k);
            const double sjj = s0 + s1;
            if (!(sjj > 0.0)) return false;
            const double r = 1.0 / sqrt(sjj);
            RI(j) = r;
            for (int i = j + 1; i < u; ++i) {
                double t0 = gh(i, j), t1 = 0.0;
                int kk = 0;
                for (; kk + 1 < j; kk += 2) {
                    t0 -= LF(i, kk) * LF(j, kk);
                    t1 -= LF(i, kk + 1) * LF(j, kk + 1);
                }
                if (kk < j) t0 -= LF(i, kk) * LF(j, kk);
                LF(i, j) = (t0 + t1) * r;
            }
        }
        return true;
    };
    // w <- (L L^T)^-1 w
    auto solve = [&]() {
        for (int i = 0; i < u; ++i) {
            double t0 = WV(i), t1 = 0.0;
            int k = 0;
            for (; k + 1 < i; k += 2) {
                t0 -= LF(i, k) * WV(k);
                t1 -= LF(i, k + 1) * WV(k + 1);
            }
            if (k < i) t0 -= LF(i, k) * WV(k);
            WV(i) = (t0 + t1) * RI(i);
        }
        for (int i = u - 1; i >= 0; --i) {
            double t0 = WV(i), t1 = 0.0;
            int k = i + 1;
            for (; k + 1 < u; k += 2) {
                t0 -= LF(k, i) * WV(k);
                t1 -= LF(k + 1, i) * WV(k + 1);
            }
            if (k < u) t0 -= LF(k, i) * WV(k);
            WV(i) = (t0 + t1) * RI(i);
        }
    };
    // one inverse-iteration step v <- normalise((Ghat - shift)^-1 v); returns
    // the Rayleigh quotient of the new v, shift + (v.w) / (w.w), and in dv2
    // the squared change of v (no sign flips: the shifted matrix is positive
    // definite, so v.w > 0)
    auto step = [&](double shift, double& dv2) -> double {
        for (int i = 0; i < u; ++i) WV(i) = VV(i);
        solve();
        double vw = 0.0, ww = 0.0;
        for (int i = 0; i < u; ++i) {
            vw += VV(i) * WV(i);
            ww += WV(i) * WV(i);
        }
        const double inv = 1.0 / sqrt(ww);
        dv2 = 0.0;
        for (int i = 0; i < u; ++i) {
            const double nv_ = WV(i) * inv;
            const double dd = nv_ - VV(i);
            dv2 += dd * dd;
            VV(i) = nv_;
        }
        return shift + vw / ww;
    };

    const double eps = P.gram_eps;
    const double jitter = P.f_jit * eps * trace;
    const double null_level = P.f_null * eps * trace;
    const double rank_level = P.f_rank * eps * trace;
    double shift = -jitter;
    bool ok = cholesky(shift);
    if (!ok) {
        shift = -1024.0 * jitter;
        ok = cholesky(shift);
    }
    double theta = 0.0, theta2 = 0.0;
    if (ok) {
        double nn = 0.0;
        for (int i = 0; i < u; ++i) {
            const double x = 1.0 + 0.0625 * (double)((i * 7) % 11);
            VV(i) = x;
            nn += x * x;
        }
        nn = 1.0 / sqrt(nn);
        for (int i = 0; i < u; ++i) VV(i) *= nn;
        // stop when v moved by less than 1e-11, or stalls (rate above 1/2) at
        // the rounding floor below 1e-8
        auto converged = [](double dv2, double prev) {
            return dv2 <= 1e-22 || (dv2 <= 1e-16 && dv2 >= 0.25 * prev);
        };
        double dv2 = 1.0, prev = 1.0;
        for (int it = 0; it < 6; ++it) {
            theta = step(shift, dv2);
            if (converged(dv2, prev)) break;
            prev = dv2;
        }
        if (theta > null_level) {
            // A noisy fit: re-factor at the largest rung of a ladder below the
            // Rayleigh quotient that keeps the matrix positive definite (so
            // shift < lambda_min), iterate, and repeat with the better quotient.
            const double ladder[7] = {1.0 - 1.0 / 64, 1.0 - 1.0 / 32, 1.0 - 1.0 / 16,
                                      1.0 - 1.0 / 8, 1.0 - 1.0 / 4, 0.5, 0.25};
            bool done = false;
            for (int round = 0; round < 3 && !done; ++round) {
                bool ok2 = false;
                for (int k = 0; k < 8 && !ok2; ++k) {
                    shift = k < 7 ? theta * ladder[k] : -jitter;
                    ok2 = cholesky(shift);
                }
                if (!ok2) {
                    status |= KLR_FIT_SOLVE_FAILED;
                    ok = false;
                    break;
                }
                prev = 1.0;
                for (int it = 0; it < 8; ++it) {
                    theta = step(shift, dv2);
                    if (converged(dv2, prev)) { done = true; break; }
                    prev = dv2;
                }
            }
        }
    } else {
        status |= KLR_FIT_SOLVE_FAILED;
    }
    if (ok) {
        // next eigenvalue: inverse iteration on the complement of v.  The
        // diagonal slots of the packed factor are free (the factor keeps its
        // reciprocal diagonal in rinv) and hold the previous iterate.
        auto project_normalise = [&]() {
            double c = 0.0;
            for (int i = 0; i < u; ++i) c += WV(i) * VV(i);
            double nn = 0.0;
            for (int i = 0; i < u; ++i) {
                WV(i) -= c * VV(i);
                nn += WV(i) * WV(i);
            }
            nn = 1.0 / sqrt(nn);
            for (int i = 0; i < u; ++i) WV(i) *= nn;
        };
        for (int i = 0; i < u; ++i) WV(i) = 1.0 + 0.03125 * (double)((i * 5) % 13) - 0.5 * (i & 1);
        project_normalise();
        for (int it = 0; it < 3; ++it) {
            for (int i = 0; i < u; ++i) LF(i, i) = WV(i);
            solve();
            double zw = 0.0, zz = 0.0;
            for (int i = 0; i < u; ++i) {
                zw += WV(i) * LF(i, i);
                zz += WV(i) * WV(i);
            }
            theta2 = shift + zw / zz;
            project_normalise();
        }
        if (theta2 <= rank_level) status |= KLR_FIT_RANK_DEFICIENT;
    }
    // c = D v, unit norm, sign rule
    double nrm = 0.0;
    for (int i = 0; i < u; ++i) {
        const double ci = DD(i) * VV(i);
        WV(i) = ci;
        nrm += ci * ci;
    }
    nrm = sqrt(nrm);
    double sgn = 1.0;
    const double q0 = WV(m) / nrm;
    if (fabs(q0) >= 1e-12) {
        sgn = q0 > 0.0 ? 1.0 : -1.0;
    } else {
        double best = -1.0;
        int bi = m;
        for (int j = m; j < u; ++j)
            if (fabs(WV(j)) > best) { best = fabs(WV(j)); bi = j; }
        sgn = WV(bi) > 0.0 ? 1.0 : -1.0;
    }
    const double scale = ok ? sgn / nrm : 0.0;
    for (int j = 0; j < u; ++j) {
        const double cj = WV(j) * scale;
        if (P.coef_f64) reinterpret_cast<double*>(P.coef)[(int64_t)f * u + j] = cj;
        else reinterpret_cast<float*>(P.coef)[(int64_t)f * u + j] = (float)cj;
    }
    P.status[f] = status;
    if (P.diag) {
        double* dg = P.diag + (int64_t)f * 4;
        dg[0] = trace > 0 ? theta / trace : 0.0;
        dg[1] = trace > 0 ? theta2 / trace : 0.0;
        dg[2] = sqrt(fmax(theta, 0.0) / (double)S) / nrm;
        dg[3] = 0.0;
    }
#undef LF
#undef RI
#undef DD
#undef VV
#undef WV
}

// The lane-per-fit solver in double-word FP32 arithmetic (on the FP32 pipes).
// Moments arrive as normalised double-word pairs; the factor, D, v and w live
// in shared memory interleaved across the 32 lanes, 8 bytes per entry.
__global__ void __launch_bounds__(32)
solve_lane_dw_kernel(const __grid_constant__ FitParams P) {
    extern __shared__ __align__(16) float2 lsm2[];
    const int lane = threadIdx.x;
    const int f = blockIdx.x * 32 + lane;
    if (f >= P.n_fits) return;
    const int m = P.m, u = P.u, n_mom = P.n_mom;
    const int nL = u * (u + 1) / 2;
    float2* Lf = lsm2;
    float2* rinv = Lf + nL * 32;
    float2* Dv = rinv + u * 32;
    float2* vv = Dv + u * 32;
    float2* wv = vv + u * 32;
    auto ld2 = [](const float2 v) -> dw { return dw{v.x, v.y}; };
    auto st2 = [](dw x) -> float2 { return make_float2(x.h, x.l); };
#define LF(i, j) Lf[((i) * ((i) + 1) / 2 + (j)) * 32 + lane]
#define RI(i) rinv[(i) * 32 + lane]
#define DD(i) Dv[(i) * 32 + lane].x
#define VV(i) vv[(i) * 32 + lane]
#define WV(i) wv[(i) * 32 + lane]
    const float2* M = reinterpret_cast<const float2*>(P.mom) + (int64_t)f * 3 * n_mom;
    const int64_t S = P.offsets[f + 1] - P.offsets[f];
    const int32_t fl = P.flags[f];
    int32_t status = 0;
    if (S == 0) status = KLR_FIT_EMPTY;
    else if (fl & 1) status = KLR_FIT_NONFINITE;
    if (status) {
        for (int j = 0; j < u; ++j) {
            if (P.coef_f64) reinterpret_cast<double*>(P.coef)[(int64_t)f * u + j] = 0.0;
            else reinterpret_cast<float*>(P.coef)[(int64_t)f * u + j] = 0.f;
        }
        P.status[f] = status;
        if (P.diag) for (int k = 0; k < 4; ++k) P.diag[(int64_t)f * 4 + k] = 0.0;
        return;
    }
    if (fl & 2) status |= KLR_FIT_INEXACT;
    // equilibration: 2^-floor(e/2), e the frexp exponent of the (exact)
    // double-word diagonal entry
    dw trace{0.f, 0.f};
    for (int j = 0; j < u; ++j) {
        const int bj = j >= m, jj = j - bj * m;
        const float2 g2 = M[2 * bj * n_mom + P.pair[jj][jj]];
        float dj = 1.0f;
        if (g2.x > 0.f) {
            int e;
            const float mant = frexpf(g2.x, &e);
            if (mant == 0.5f && g2.y < 0.f) e -= 1;   // h rounded up to a power of two
            dj = ldexpf(1.0f, -(e >> 1));
        }
        Dv[j * 32 + lane] = make_float2(dj, 0.f);
        trace = dw_add(trace, dw{g2.x * dj * dj, g2.y * dj * dj});
    }
    auto gh = [&](int i, int j) -> dw {
        const int bi = i >= m, bj = j >= m;
        const float2 g = M[(bi + bj) * n_mom + P.pair[i - bi * m][j - bj * m]];
        const float sc = ((bi != bj) ? -1.f : 1.f) * DD(i) * DD(j);   // exact
        return dw{g.x * sc, g.y * sc};
    };
    auto cholesky = [&](dw shift) -> bool {
        for (int j = 0; j < u; ++j) {
            dw_acc a0, a1;
            a0.init(dw_sub(gh(j, j), shift));
            a1.init(dw{0.f, 0.f});
            int k = 0;
            for (; k + 1 < j; k += 2) {
                const dw x0 = ld2(LF(j, k)), x1 = ld2(LF(j, k + 1));
                a0.sub_prod(x0, x0);
                a1.sub_prod(x1, x1);
            }
            if (k < j) {
                const dw x0 = ld2(LF(j, k));
                a0.sub_prod(x0, x0);
            }
            const dw sjj = dw_add(a0.value(), a1.value());
            if (!(sjj.h > 0.f)) return false;
            const dw r = dw_div(dw{1.f, 0.f}, dw_sqrt(sjj));
            RI(j) = st2(r);
            for (int i = j + 1; i < u; ++i) {
                dw_acc t0, t1;
                t0.init(gh(i, j));
                t1.init(dw{0.f, 0.f});
                int kk = 0;
                for (; kk + 1 < j; kk += 2) {
                    t0.sub_prod(ld2(LF(i, kk)), ld2(LF(j, kk)));
                    t1.sub_prod(ld2(LF(i, kk + 1)), ld2(LF(j, kk + 1)));
                }
                if (kk < j) t0.sub_prod(ld2(LF(i, kk)), ld2(LF(j, kk)));
                LF(i, j) = st2(dw_mul(dw_add(t0.value(), t1.value()), r));
            }
        }
        return true;
    };
    auto solve = [&]() {
        for (int i = 0; i < u; ++i) {
            dw_acc t0, t1;
            t0.init(ld2(WV(i)));
            t1.init(dw{0.f, 0.f});
            int k = 0;
            for (; k + 1 < i; k += 2) {
                t0.sub_prod(ld2(LF(i, k)), ld2(WV(k)));
                t1.sub_prod(ld2(LF(i, k + 1)), ld2(WV(k + 1)));
            }
            if (k < i) t0.sub_prod(ld2(LF(i, k)), ld2(WV(k)));
            WV(i) = st2(dw_mul(dw_add(t0.value(), t1.value()), ld2(RI(i))));
        }
        for (int i = u - 1; i >= 0; --i) {
            dw_acc t0, t1;
            t0.init(ld2(WV(i)));
            t1.init(dw{0.f, 0.f});
            int k = i + 1;
            for (; k + 1 < u; k += 2) {
                t0.sub_prod(ld2(LF(k, i)), ld2(WV(k)));
                t1.sub_prod(ld2(LF(k + 1, i)), ld2(WV(k + 1)));
            }
            if (k < u) t0.sub_prod(ld2(LF(k, i)), ld2(WV(k)));
            WV(i) = st2(dw_mul(dw_add(t0.value(), t1.value()), ld2(RI(i))));
        }
    };
    // inverse-iteration step; returns the Rayleigh quotient shift + (v.w)/(w.w)
    // and the squared change of v (double-word norms, FP32 change)
    auto step = [&](dw shift, float& dv2) -> dw {
        for (int i = 0; i < u; ++i) WV(i) = VV(i);
        solve();
        dw_acc vw, ww;
        vw.init(dw{0.f, 0.f});
        ww.init(dw{0.f, 0.f});
        for (int i = 0; i < u; ++i) {
            const dw wi = ld2(WV(i));
            vw.add_prod(ld2(VV(i)), wi);
            ww.add_prod(wi, wi);
        }
        const dw wwv = ww.value();
        const dw inv = dw_div(dw{1.f, 0.f}, dw_sqrt(wwv));
        dv2 = 0.f;
        for (int i = 0; i < u; ++i) {
            const dw nvi = dw_mul(ld2(WV(i)), inv);
            const dw d = dw_sub(nvi, ld2(VV(i)));
            dv2 += d.h * d.h;
            VV(i) = st2(nvi);
        }
        return dw_add(shift, dw_div(vw.value(), wwv));
    };
    // stop when v moved by less than 1e-10, or stalls (rate above 1/2) below 1e-7
    auto converged = [](float dv2, float prev) {
        return dv2 <= 1e-20f || (dv2 <= 1e-14f && dv2 >= 0.25f * prev);
    };

    const float eps = (float)P.gram_eps;
    const dw jitter = dw_mul_f(trace, (float)P.f_jit * eps);
    const dw null_level = dw_mul_f(trace, (float)P.f_null * eps);
    const dw rank_level = dw_mul_f(trace, (float)P.f_rank * eps);
    dw shift = dw_neg(jitter);
    bool ok = cholesky(shift);
    if (!ok) {
        shift = dw_mul_f(shift, 1024.f);
        ok = cholesky(shift);
    }
    dw theta{0.f, 0.f}, theta2{0.f, 0.f};
    if (ok) {
        dw_acc nn;
        nn.init(dw{0.f, 0.f});
        for (int i = 0; i < u; ++i) {
            const float x = 1.0f + 0.0625f * (float)((i * 7) % 11);
            VV(i) = make_float2(x, 0.f);
            nn.add_prod(dw{x, 0.f}, dw{x, 0.f});
        }
        const dw inv = dw_div(dw{1.f, 0.f}, dw_sqrt(nn.value()));
        for (int i = 0; i < u; ++i) VV(i) = st2(dw_mul(ld2(VV(i)), inv));
        float dv2 = 1.f, prev = 1.f;
        for (int it = 0; it < 6; ++it) {
            theta = step(shift, dv2);
            if (converged(dv2, prev)) break;
            prev = dv2;
        }
        if (dw_gt(theta, null_level)) {
            const float ladder[7] = {1.0f - 1.0f / 64, 1.0f - 1.0f / 32, 1.0f - 1.0f / 16,
                                     1.0f - 1.0f / 8, 1.0f - 1.0f / 4, 0.5f, 0.25f};
            bool done = false;
            for (int round = 0; round < 3 && !done; ++round) {
                bool ok2 = false;
                for (int k = 0; k < 8 && !ok2; ++k) {
                    shift = k < 7 ? dw_mul_f(theta, ladder[k]) : dw_neg(jitter);
                    ok2 = cholesky(shift);
                }
                if (!ok2) {
                    status |= KLR_FIT_SOLVE_FAILED;
                    ok = false;
                    break;
                }
                prev = 1.f;
                for (int it = 0; it < 8; ++it) {
                    theta = step(shift, dv2);
                    if (converged(dv2, prev)) { done = true; break; }
                    prev = dv2;
                }
            }
        }
    } else {
        status |= KLR_FIT_SOLVE_FAILED;
    }
    if (ok) {
        // next eigenvalue: inverse iteration on the complement of v; the
        // diagonal slots of the packed factor are free and hold the iterate
        auto project_normalise = [&]() {
            dw_acc c;
            c.init(dw{0.f, 0.f});
            for (int i = 0; i < u; ++i) c.add_prod(ld2(WV(i)), ld2(VV(i)));
            const dw cv = c.value();
            dw_acc nn;
            nn.init(dw{0.f, 0.f});
            for (int i = 0; i < u; ++i) {
                const dw wi = dw_sub(ld2(WV(i)), dw_mul(cv, ld2(VV(i))));
                WV(i) = st2(wi);
                nn.add_prod(wi, wi);
            }
            const dw inv = dw_div(dw{1.f, 0.f}, dw_sqrt(nn.value()));
            for (int i = 0; i < u; ++i) WV(i) = st2(dw_mul(ld2(WV(i)), inv));
        };
        for (int i = 0; i < u; ++i)
            WV(i) = make_float2(1.0f + 0.03125f * (float)((i * 5) % 13) - 0.5f * (float)(i & 1), 0.f);
        project_normalise();
        for (int it = 0; it < 3; ++it) {
            for (int i = 0; i < u; ++i) LF(i, i) = WV(i);
            solve();
            dw_acc zw, zz;
            zw.init(dw{0.f, 0.f});
            zz.init(dw{0.f, 0.f});
            for (int i = 0; i < u; ++i) {
                const dw wi = ld2(WV(i));
                zw.add_prod(wi, ld2(LF(i, i)));
                zz.add_prod(wi, wi);
            }
            theta2 = dw_add(shift, dw_div(zw.value(), zz.value()));
            project_normalise();
        }
        if (!dw_gt(theta2, rank_level)) status |= KLR_FIT_RANK_DEFICIENT;
    }
    // c = D v, unit norm, sign rule
    dw_acc nrm2;
    nrm2.init(dw{0.f, 0.f});
    for (int i = 0; i < u; ++i) {
        const dw ci = dw_mul_f(ld2(VV(i)), DD(i));
        WV(i) = st2(ci);
        nrm2.add_prod(ci, ci);
    }
    const dw nrm = dw_sqrt(nrm2.value());
    const double nrm_d = dw_to_double(nrm);
    float sgn = 1.f;
    const float q0 = WV(m).x / nrm.h;
    if (fabsf(q0) >= 1e-12f) {
        sgn = q0 > 0.f ? 1.f : -1.f;
    } else {
        float best = -1.f;
        int bi = m;
        for (int j = m; j < u; ++j)
            if (fabsf(WV(j).x) > best) { best = fabsf(WV(j).x); bi = j; }
        sgn = WV(bi).x > 0.f ? 1.f : -1.f;
    }
    const dw scale = ok ? dw_div(dw{sgn, 0.f}, nrm) : dw{0.f, 0.f};
    for (int j = 0; j < u; ++j) {
        const dw cj = dw_mul(ld2(WV(j)), scale);
        if (P.coef_f64) reinterpret_cast<double*>(P.coef)[(int64_t)f * u + j] = dw_to_double(cj);
        else reinterpret_cast<float*>(P.coef)[(int64_t)f * u + j] = cj.h + cj.l;
    }
    P.status[f] = status;
    if (P.diag) {
        double* dg = P.diag + (int64_t)f * 4;
        const double tr = dw_to_double(trace), th = dw_to_double(theta);
        dg[0] = tr > 0 ? th / tr : 0.0;
        dg[1] = tr > 0 ? dw_to_double(theta2) / tr : 0.0;
        dg[2] = sqrt(fmax(th, 0.0) / (double)S) / nrm_d;
        dg[3] = 0.0;
    }
#undef LF
#undef RI
#undef DD
#undef VV
#undef WV
}

// Group-solver steps, out of line so that the kernel holds one copy of each
// (its schedule calls them from several places).  Q lanes serve one fit; lane
// q = lane % Q owns rows i = q (mod Q) of the packed lower factor Lf (row i
// starts at i (i + 1) / 2; the diagonal slots are not used by these steps).
#define GLF(i, j) Lf[(i) * ((i) + 1) / 2 + (j)]

// Cholesky factor of (D G D - shift I), G from the moment sums M (pair table
// `pair`, m monomials, n_mom moments per power of y), into Lf (strictly lower
// part) and rinv (1 / diagonal).  Writes only when `write`; returns the
// group's success (false also when not writing).
template <int Q>
__device__ __noinline__ bool group_cholesky(float2* Lf, float2* rinv, const float2* M,
                                            const uint8_t (*pair)[kMaxBasis], const float* Dv,
                                            int m, int u, int n_mom, dw shift, bool write) {
    const unsigned full = 0xffffffffu;
    const int q = (threadIdx.x & 31) % Q;
    auto ld2 = [](const float2 v) -> dw { return dw{v.x, v.y}; };
    auto st2 = [](dw x) -> float2 { return make_float2(x.h, x.l); };
    auto gh = [&](int i, int j) -> dw {
        const int bi = i >= m, bj = j >= m;
        const float2 gg = M[(bi + bj) * n_mom + pair[i - bi * m][j - bj * m]];
        const float sc = ((bi != bj) ? -1.f : 1.f) * Dv[i] * Dv[j];
        return dw{gg.x * sc, gg.y * sc};
    };
    bool good = write;
    for (int j = 0; j < u; ++j) {
        dw_acc a;
        a.init(dw{0.f, 0.f});
        for (int k = q; k < j; k += Q) {
            const dw x = ld2(GLF(j, k));
            a.add_prod(x, x);
        }
        dw sum = a.value();
#pragma unroll
        for (int o = 1; o < Q; o <<= 1) {
            const dw y{__shfl_xor_sync(full, sum.h, o), __shfl_xor_sync(full, sum.l, o)};
            sum = dw_add(sum, y);
        }
        const dw sjj = dw_sub(dw_sub(gh(j, j), shift), sum);
        good = good && (sjj.h > 0.f);
        const dw r = good ? dw_rsqrt(sjj) : dw{1.f, 0.f};
        if (good && q == 0) rinv[j] = st2(r);
        for (int i = j + 1 + ((q - (j + 1) % Q) + Q) % Q; i < u; i += Q) {
            dw_acc t0, t1;
            t0.init(gh(i, j));
            t1.init(dw{0.f, 0.f});
            int k = 0;
            for (; k + 1 < j; k += 2) {
                t0.sub_prod(ld2(GLF(i, k)), ld2(GLF(j, k)));
                t1.sub_prod(ld2(GLF(i, k + 1)), ld2(GLF(j, k + 1)));
            }
            if (k < j) t0.sub_prod(ld2(GLF(i, k)), ld2(GLF(j, k)));
            if (good) GLF(i, j) = st2(dw_mul(dw_add(t0.value(), t1.value()), r));
        }
        __syncwarp();
    }
    return good;
}

// w <- (L L^T)^-1 w, column-oriented.  Lane q keeps the rows i = q + r Q
// it owns as unnormalised Dot2 accumulators in registers (r < MAXR, a
// compile-time count, so the updates of different rows are independent
// instructions); the finished component of column j is broadcast from its
// owner by shuffles.  Only L is read from shared memory.
template <int Q, int MAXR>
__device__ __noinline__ void group_tri_solve(float2* wv, const float2* Lf, const float2* rinv,
                                             int u, bool write) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, q = lane % Q;
    auto ld2 = [](const float2 v) -> dw { return dw{v.x, v.y}; };
    auto st2 = [](dw x) -> float2 { return make_float2(x.h, x.l); };
    const int gbase = lane & ~(Q - 1);
    dw_acc a[MAXR];
    dw x[MAXR];
#pragma unroll
    for (int r = 0; r < MAXR; ++r) {
        const int i = q + r * Q;
        a[r].init(i < u ? ld2(wv[i]) : dw{0.f, 0.f});
        x[r] = dw{0.f, 0.f};
    }
    // forward: L y = w
#pragma unroll
    for (int r = 0; r < MAXR; ++r) {
#pragma unroll 1
        for (int jj = 0; jj < Q; ++jj) {
            const int j = r * Q + jj;
            if (j >= u) break;
            const dw aj = a[r].value();
            dw yj{__shfl_sync(full, aj.h, gbase | jj), __shfl_sync(full, aj.l, gbase | jj)};
            yj = dw_mul(yj, ld2(rinv[j]));
            if (q == jj) x[r] = yj;
#pragma unroll
            for (int r2 = r; r2 < MAXR; ++r2) {
                const int i = q + r2 * Q;
                if (i > j && i < u) a[r2].sub_prod(ld2(GLF(i, j)), yj);
            }
        }
    }
    // backward: L^T x = y
#pragma unroll
    for (int r = 0; r < MAXR; ++r) a[r].init(x[r]);
#pragma unroll
    for (int r = MAXR - 1; r >= 0; --r) {
#pragma unroll 1
        for (int jj = Q - 1; jj >= 0; --jj) {
            const int j = r * Q + jj;
            if (j >= u) continue;
            const dw bj = a[r].value();
            dw xj{__shfl_sync(full, bj.h, gbase | jj), __shfl_sync(full, bj.l, gbase | jj)};
            xj = dw_mul(xj, ld2(rinv[j]));
            if (q == jj) x[r] = xj;
#pragma unroll
            for (int r2 = 0; r2 <= r; ++r2) {
                const int i = q + r2 * Q;
                if (i < j) a[r2].sub_prod(ld2(GLF(j, i)), xj);
            }
        }
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < MAXR; ++r) {
        const int i = q + r * Q;
        if (write && i < u) wv[i] = st2(x[r]);
    }
    __syncwarp();
}

#undef GLF

// Largest eigenpair of the K x K symmetric tridiagonal matrix (a on the
// diagonal, b beside it), in FP32.  Newton's method on the characteristic
// polynomial from Gershgorin's upper bound: for a polynomial with real roots
// it decreases monotonically to the largest root.  The pivots r_i of
// T - x I (all negative above the largest eigenvalue) give p'/p =
// sum_i r_i'/r_i.  The eigenvector comes from two steps of inverse iteration
// with x I - T (positive definite for x just above the root), solved by the
// Thomas recurrence without pivoting, when VEC.  s is normalised to unit
// length.
template <int K, bool VEC>
__device__ float tridiag_top_eigen(const float (&a)[K], const float (&b)[K], float (&s)[K]) {
    float x = -FLT_MAX;
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const float r = (i > 0 ? fabsf(b[i - 1]) : 0.f) + (i + 1 < K ? fabsf(b[i]) : 0.f);
        x = fmaxf(x, a[i] + r);
    }
    x = x + 1e-6f * fabsf(x) + FLT_MIN;
#pragma unroll 1
    for (int it = 0; it < 40; ++it) {
        float r = a[0] - x, dr = -1.f, sum = dr / r;
#pragma unroll
        for (int i = 1; i < K; ++i) {
            const float bb = b[i - 1] * b[i - 1];
            const float rn = (a[i] - x) - bb / r;
            dr = -1.f + bb * dr / (r * r);
            r = rn;
            sum += dr / r;
        }
        // p / p' = 1 / sum; the step is negative above the root
        const float dx = 1.f / sum;
        const float xn = x - dx;
        if (!(xn < x) || !(xn == xn)) break;
        x = xn;
        if (fabsf(dx) <= 1e-7f * fabsf(x)) break;
    }
    if (!VEC) return x;
    const float xs = x + 2e-6f * fabsf(x) + FLT_MIN;   // above the root: x I - T is definite
#pragma unroll
    for (int i = 0; i < K; ++i) s[i] = 1.f;
#pragma unroll 1
    for (int it = 0; it < 2; ++it) {
        // (xs I - T) z = s by the Thomas recurrence
        float c[K], d[K];
        float den = xs - a[0];
        c[0] = -b[0] / den;
        d[0] = s[0] / den;
#pragma unroll
        for (int i = 1; i < K; ++i) {
            den = (xs - a[i]) + b[i - 1] * c[i - 1];
            c[i] = i + 1 < K ? -b[i] / den : 0.f;
            d[i] = (s[i] + b[i - 1] * d[i - 1]) / den;
        }
        s[K - 1] = d[K - 1];
#pragma unroll
        for (int i = K - 2; i >= 0; --i) s[i] = d[i] - c[i] * s[i + 1];
        float nn = 0.f;
#pragma unroll
        for (int i = 0; i < K; ++i) nn += s[i] * s[i];
        const float inv = rsqrtf(nn);
#pragma unroll
        for (int i = 0; i < K; ++i) s[i] *= inv;
    }
    return x;
}

// The double-word solver with Q lanes per fit (32 / Q fits per warp).  Each
// fit's factor lives in shared memory (packed lower triangle, 8-byte pairs);
// row i of the factor is computed by lane i % Q of the fit's group, so a fit's
// dependency chains are Q times shorter than with one lane per fit and four
// times as many fits fit in an SM's shared memory per warp.  The triangular
// solves are column-oriented (each lane updates the rows it owns, at most
// MAXR, held in registers), so they need no reductions.  Control flow is
// uniform across the warp: every group runs the same schedule and a group
// that has finished (or failed) keeps running it with its writes switched off.
template <int Q, int MAXR>
__global__ void __launch_bounds__(32)
solve_group_dw_kernel(const __grid_constant__ FitParams P) {
    constexpr int GPW = 32 / Q;
    extern __shared__ __align__(16) float2 gsm[];
    const int lane = threadIdx.x;
    const int q = lane % Q, g = lane / Q;
    const int f_raw = blockIdx.x * GPW + g;
    const bool live = f_raw < P.n_fits;
    const int f = live ? f_raw : P.n_fits - 1;   // clamp reads for the spare groups
    const int m = P.m, u = P.u, n_mom = P.n_mom;
    const int nL = u * (u + 1) / 2;
    const int stride = P.ld;                      // float2 per fit (padded)
    float2* base = gsm + g * stride;
    float2* Lf = base;
    float2* rinv = Lf + nL;
    float2* vv = rinv + u;
    float2* wv = vv + u;
    float* Dv = reinterpret_cast<float*>(wv + u);   // the powers of two D, u floats
    auto ld2 = [](const float2 v) -> dw { return dw{v.x, v.y}; };
    auto st2 = [](dw x) -> float2 { return make_float2(x.h, x.l); };
    const unsigned full = 0xffffffffu;
    // sum over the Q lanes of a group of a double-word value
    auto gsum = [&](dw x) -> dw {
#pragma unroll
        for (int o = 1; o < Q; o <<= 1) {
            dw y{__shfl_xor_sync(full, x.h, o), __shfl_xor_sync(full, x.l, o)};
            x = dw_add(x, y);
        }
        return x;
    };
#define LF(i, j) Lf[(i) * ((i) + 1) / 2 + (j)]
    const float2* M = reinterpret_cast<const float2*>(P.mom) + (int64_t)f * 3 * n_mom;
    const int64_t S = P.offsets[f + 1] - P.offsets[f];
    const int32_t fl = P.flags[f];
    int32_t status = 0;
    if (S == 0) status = KLR_FIT_EMPTY;
    else if (fl & 1) status = KLR_FIT_NONFINITE;
    bool ok = (status == 0);
    if (fl & 2) status |= KLR_FIT_INEXACT;
    // equilibration (every lane of the group computes all of D; lane 0 stores)
    dw trace{0.f, 0.f};
    for (int j = 0; j < u; ++j) {
        const int bj = j >= m, jj = j - bj * m;
        const float2 g2 = M[2 * bj * n_mom + P.pair[jj][jj]];
        float dj = 1.0f;
        if (g2.x > 0.f) {
            int e;
            const float mant = frexpf(g2.x, &e);
            if (mant == 0.5f && g2.y < 0.f) e -= 1;
            dj = ldexpf(1.0f, -(e >> 1));
        }
        if (q == 0) Dv[j] = dj;
        trace = dw_add(trace, dw{g2.x * dj * dj, g2.y * dj * dj});
    }
    __syncwarp();
    auto gh = [&](int i, int j) -> dw {
        const int bi = i >= m, bj = j >= m;
        const float2 gg = M[(bi + bj) * n_mom + P.pair[i - bi * m][j - bj * m]];
        const float sc = ((bi != bj) ? -1.f : 1.f) * Dv[i] * Dv[j];
        return dw{gg.x * sc, gg.y * sc};
    };
    // Cholesky of (Ghat - shift I) for groups with `write`; returns the
    // group's success (false also for groups not writing)
    auto cholesky = [&](dw shift, bool write) -> bool {
        return group_cholesky<Q>(Lf, rinv, M, P.pair, Dv, m, u, n_mom, shift, write);
    };
    // w <- (L L^T)^-1 w for groups with `write`
    auto solve = [&](bool write) { group_tri_solve<Q, MAXR>(wv, Lf, rinv, u, write); };
    auto gdot = [&](const float2* a, const float2* b) -> dw {
        dw_acc s;
        s.init(dw{0.f, 0.f});
        for (int i = q; i < u; i += Q) s.add_prod(ld2(a[i]), ld2(b[i]));
        return gsum(s.value());
    };
    // inverse-iteration step for groups with `write`
    auto step = [&](dw shift, bool write, float& dv2) -> dw {
        for (int i = q; i < u; i += Q) wv[i] = vv[i];
        __syncwarp();
        solve(write);
        const dw vw = gdot(vv, wv), ww = gdot(wv, wv);
        const dw inv = dw_rsqrt(ww);
        float part = 0.f;
        for (int i = q; i < u; i += Q) {
            const dw nvi = dw_mul(ld2(wv[i]), inv);
            const dw dd = dw_sub(nvi, ld2(vv[i]));
            part += dd.h * dd.h;
            if (write) vv[i] = st2(nvi);
        }
#pragma unroll
        for (int o = 1; o < Q; o <<= 1) part += __shfl_xor_sync(full, part, o);
        dv2 = part;
        __syncwarp();
        return dw_add(shift, dw_div(vw, ww));
    };
    auto converged = [](float dv2, float prev) {
        return dv2 <= 1e-20f || (dv2 <= 1e-14f && dv2 >= 0.25f * prev);
    };

    const float eps = (float)P.gram_eps;
    const dw jitter = dw_mul_f(trace, (float)P.f_jit * eps);
    const dw null_level = dw_mul_f(trace, (float)P.f_null * eps);
    const dw rank_level = dw_mul_f(trace, (float)P.f_rank * eps);
    dw shift = dw_neg(jitter);
    bool fact = cholesky(shift, ok);
    if (ok && !fact) {
        shift = dw_mul_f(shift, 1024.f);
    }
    {
        const bool retry = ok && !fact;
        if (__any_sync(full, retry)) {
            const bool f2 = cholesky(shift, retry);
            if (retry) fact = f2;
        }
    }
    if (ok && !fact) {
        ok = false;
        status |= KLR_FIT_SOLVE_FAILED;
    }
    dw theta{0.f, 0.f}, theta2{0.f, 0.f};
    // the start vector (a fixed pattern), normalised
    auto start_vector = [&]() {
        for (int i = q; i < u; i += Q)
            vv[i] = make_float2(1.0f + 0.0625f * (float)((i * 7) % 11), 0.f);
        __syncwarp();
        const dw nn = gdot(vv, vv);
        const dw inv = dw_div(dw{1.f, 0.f}, dw_sqrt(nn));
        for (int i = q; i < u; i += Q) vv[i] = st2(dw_mul(ld2(vv[i]), inv));
        __syncwarp();
    };
    start_vector();
    float2 bas[kLanczosSteps][MAXR];   // the Lanczos vectors q_j, this lane's rows
    float sv[kLanczosSteps];           // the top eigenvector of their projection
    // Phase 1: Lanczos on T = (Ghat - shift I)^-1 from the start vector, by
    // its three-term recurrence (every group runs the same kLanczosSteps
    // solves): alpha_j = q_j . T q_j, r = T q_j - alpha_j q_j - beta_{j-1}
    // q_{j-1}, beta_j = |r|, q_{j+1} = r / beta_j.  The largest eigenvalue mu
    // of the tridiagonal projection gives the Ritz value theta = shift + 1/mu
    // >= lambda_1, which places the next shift.  Its accuracy grows like that
    // of a Chebyshev-accelerated inverse iteration (about 0.12 per solve at
    // lambda_1/lambda_2 = 0.4); over seven steps the basis keeps its
    // orthogonality in double-word arithmetic (a Ritz vector converges to
    // about 1e-6, far from the square root of the rounding where Lanczos
    // loses it), so no reorthogonalisation is needed; this lane's rows of the
    // basis stay in registers for the Ritz vector.  (Seven steps measured
    // fastest on the bench batch: six 1.48 ms, eight 1.51, five 1.91.)
    {
        float2* pv = wv + u + (u + 1) / 2;   // the previous Lanczos vector (after D)
        float la[kLanczosSteps], lb[kLanczosSteps];
        dw bprev{0.f, 0.f};
#pragma unroll 1
        for (int j = 0; j < kLanczosSteps; ++j) {
            // keep q_j's rows of this lane for the Ritz vector
            {
                float2 cur[MAXR];
#pragma unroll
                for (int r = 0; r < MAXR; ++r) {
                    const int i = q + r * Q;
                    cur[r] = i < u ? vv[i] : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int jj = 0; jj < kLanczosSteps; ++jj)
#pragma unroll
                    for (int r = 0; r < MAXR; ++r)
                        if (jj == j) bas[jj][r] = cur[r];
            }
            for (int i = q; i < u; i += Q) wv[i] = vv[i];
            __syncwarp();
            solve(ok);
            const dw aj = gdot(vv, wv);
            for (int i = q; i < u; i += Q) {
                dw r = dw_sub(ld2(wv[i]), dw_mul(aj, ld2(vv[i])));
                if (j > 0) r = dw_sub(r, dw_mul(bprev, ld2(pv[i])));
                if (ok) wv[i] = st2(r);
            }
            __syncwarp();
            const dw bb = gdot(wv, wv);
            const dw inv = dw_rsqrt(bb.h > 0.f ? bb : dw{FLT_MIN, 0.f});
            const dw bj = dw_mul(bb, inv);
            la[j] = aj.h + aj.l;
            lb[j] = bj.h + bj.l;
            if (j + 1 < kLanczosSteps) {
                for (int i = q; i < u; i += Q) {
                    if (ok) {
                        pv[i] = vv[i];
                        vv[i] = st2(dw_mul(ld2(wv[i]), inv));
                    }
                }
                __syncwarp();
            }
            bprev = bj;
        }
        const float mu = tridiag_top_eigen<kLanczosSteps, true>(la, lb, sv);
        if (ok) theta = dw_add(shift, dw_div(dw{1.f, 0.f}, dw{mu > 0.f ? mu : FLT_MIN, 0.f}));
    }
    // the iterations below start from the Ritz vector sum_j s_j q_j (the
    // start vector where it is not usable)
    {
#pragma unroll
        for (int r = 0; r < MAXR; ++r) {
            const int i = q + r * Q;
            dw y{0.f, 0.f};
#pragma unroll
            for (int jj = 0; jj < kLanczosSteps; ++jj)
                y = dw_add(y, dw_mul_f(ld2(bas[jj][r]), sv[jj]));
            if (i < u) vv[i] = st2(y);
        }
        __syncwarp();
        const dw nn = gdot(vv, vv);
        if (!(nn.h > 0.f && isfinite(nn.h)))
            for (int i = q; i < u; i += Q)
                vv[i] = make_float2(1.0f + 0.0625f * (float)((i * 7) % 11), 0.f);
        __syncwarp();
        const dw inv = dw_rsqrt(gdot(vv, vv));
        for (int i = q; i < u; i += Q) vv[i] = st2(dw_mul(ld2(vv[i]), inv));
        __syncwarp();
    }
    bool active = ok;
    float dv2 = 1.f, prev = 1.f;
    // noisy fits: rounds of re-factoring on a ladder of shifts below theta
    // (the Ritz value is accurate to far better than its first rung)
    bool noisy = ok && dw_gt(theta, null_level);
    // fits whose lambda_1 is at the rounding level: inverse iteration at the
    // first shift (the next eigenvalue is far above, a step gains about
    // lambda_2 / jitter)
    {
        bool act = active && !noisy;
        for (int it = 0; it < 4 && __any_sync(full, act); ++it) {
            const dw th = step(shift, act, dv2);
            if (act) {
                theta = th;
                if (converged(dv2, prev)) act = false;
                prev = dv2;
            }
        }
    }
    bool done = !noisy;
    const float ladder[8] = {1.0f - 1.0f / 4096, 1.0f - 1.0f / 64, 1.0f - 1.0f / 16,
                             1.0f - 1.0f / 8, 1.0f - 1.0f / 4, 0.5f, 0.25f, 0.0625f};
    for (int round = 0; round < 3 && __any_sync(full, !done); ++round) {
        bool need = !done;      // this group still needs a factor in this pass
        bool have = false;
        int rung = 9;
        for (int k = 0; k < 9 && __any_sync(full, need && !have); ++k) {
            const bool try_ = need && !have;
            const dw sh = k < 8 ? dw_mul_f(theta, ladder[k]) : dw_neg(jitter);
            const bool good = cholesky(sh, try_);
            if (try_ && good) {
                have = true;
                shift = sh;
                rung = k;
            }
        }
        if (need && !have) {
            status |= KLR_FIT_SOLVE_FAILED;
            ok = false;
            done = true;
        }
        bool act = need && have;
        prev = 1.f;
        for (int it = 0; it < 8 && __any_sync(full, act); ++it) {
            const dw th = step(shift, act, dv2);
            if (act) {
                theta = th;
                // on the first two rungs a step leaves at most about 1/64 of
                // the error (1/4096 on the first): a change below 1e-8 leaves
                // an error below 2e-10
                if ((rung <= 1 && dv2 <= 1e-16f) || converged(dv2, prev)) {
                    act = false;
                    done = true;
                }
                prev = dv2;
            }
        }
    }
    // next eigenvalue on the complement of v (rank test); w holds the iterate,
    // the diagonal slots of the packed factor hold the previous one
    {
        auto project_normalise = [&](bool write) {
            const dw c = gdot(wv, vv);
            dw_acc nn;
            nn.init(dw{0.f, 0.f});
            for (int i = q; i < u; i += Q) {
                const dw wi = dw_sub(ld2(wv[i]), dw_mul(c, ld2(vv[i])));
                if (write) wv[i] = st2(wi);
                nn.add_prod(wi, wi);
            }
            __syncwarp();
            const dw inv = dw_div(dw{1.f, 0.f}, dw_sqrt(gsum(nn.value())));
            for (int i = q; i < u; i += Q)
                if (write) wv[i] = st2(dw_mul(ld2(wv[i]), inv));
            __syncwarp();
        };
        // A noisy fit whose iteration converged to an eigenvalue above twice
        // the rank level needs no test: the next eigenvalue is at least as
        // large.  It reports that eigenvalue as the estimate.
        const bool need = ok && !(noisy && done && dw_gt(theta, dw_mul_f(rank_level, 2.f)));
        if (ok && !need) theta2 = theta;
        if (__any_sync(full, need)) {
            for (int i = q; i < u; i += Q)
                wv[i] = make_float2(1.0f + 0.03125f * (float)((i * 5) % 13) - 0.5f * (float)(i & 1),
                                    0.f);
            __syncwarp();
            project_normalise(need);
            for (int it = 0; it < 3; ++it) {
                for (int i = q; i < u; i += Q)
                    if (need) LF(i, i) = wv[i];
                __syncwarp();
                solve(need);
                dw_acc zw, zz;
                zw.init(dw{0.f, 0.f});
                zz.init(dw{0.f, 0.f});
                for (int i = q; i < u; i += Q) {
                    const dw wi = ld2(wv[i]);
                    zw.add_prod(wi, ld2(LF(i, i)));
                    zz.add_prod(wi, wi);
                }
                const dw zwv = gsum(zw.value()), zzv = gsum(zz.value());
                if (need) theta2 = dw_add(shift, dw_div(zwv, zzv));
                project_normalise(need);
            }
            if (need && !dw_gt(theta2, rank_level)) status |= KLR_FIT_RANK_DEFICIENT;
        }
    }
    // c = D v, unit norm, sign rule; lane q writes coefficients i = q mod Q
    for (int i = q; i < u; i += Q) wv[i] = st2(dw_mul_f(ld2(vv[i]), Dv[i]));
    __syncwarp();
    const dw nrm = dw_sqrt(gdot(wv, wv));
    float sgn = 1.f;
    {
        const float q0 = wv[m].x / nrm.h;
        if (fabsf(q0) >= 1e-12f) {
            sgn = q0 > 0.f ? 1.f : -1.f;
        } else {
            float best = -1.f;
            int bi = m;
            for (int j = m; j < u; ++j)
                if (fabsf(wv[j].x) > best) { best = fabsf(wv[j].x); bi = j; }
            sgn = wv[bi].x > 0.f ? 1.f : -1.f;
        }
    }
    if (live) {
        const dw scale = ok ? dw_div(dw{sgn, 0.f}, nrm) : dw{0.f, 0.f};
        for (int j = q; j < u; j += Q) {
            const dw cj = ok ? dw_mul(ld2(wv[j]), scale) : dw{0.f, 0.f};
            if (P.coef_f64) reinterpret_cast<double*>(P.coef)[(int64_t)f * u + j] = dw_to_double(cj);
            else reinterpret_cast<float*>(P.coef)[(int64_t)f * u + j] = cj.h + cj.l;
        }
        if (q == 0) {
            P.status[f] = status;
            if (P.diag) {
                double* dg = P.diag + (int64_t)f * 4;
                const double tr = dw_to_double(trace), th = dw_to_double(theta);
                dg[0] = (ok && tr > 0) ? th / tr : 0.0;
                dg[1] = (ok && tr > 0) ? dw_to_double(theta2) / tr : 0.0;
                dg[2] = ok ? sqrt(fmax(th, 0.0) / (double)S) / dw_to_double(nrm) : 0.0;
                dg[3] = 0.0;
            }
        }
    }
#undef LF
}

// TF32 operand: FP32 rounded to nearest (ties away) to TF32
__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
    return r;
}


// ---------------------------------------------------------------------------
// Tensor-core Gram matrix on tcgen05 (KLR_FIT_BF16 and KLR_FIT_TF32): G =
// A^T A per fit as one product chain D = X X^T, X the fit's design matrix
// transposed (u rows = unknowns, padded to M = 128; K = the samples).  Both
// operands are the same shared-memory tile: 64 samples of X in the 128-byte
// swizzled K-major layout (BF16, or TF32 in two 32-sample blocks), built by
// the CTA's 128 threads (thread t: sample t mod 64, the numerator rows Phi
// for t < 64, the denominator rows -y Phi otherwise); one thread issues the
// M = 128, N = round16(u) products of the tile (four of K = 16 in BF16, eight
// of K = 8 in TF32) into an FP32 accumulator in tensor memory (row i in lane
// i) and commits them to the tile's mbarrier, so the threads build the next
// tile in the other buffer meanwhile.  At the end of a fit the four warps
// read their 32 lanes back (tcgen05.ld) and write G as FP64 for the solver.
// Rows of X past u need no zeros (they only reach rows and columns of D that
// are not read); samples past the fit's end are zero columns.  Every wait is
// bounded; a CTA whose wait gave up marks its fits as non-finite (status)
// and waits again, bounded, for its products in flight before freeing its
// tensor memory.
// ---------------------------------------------------------------------------
constexpr int kGramThreads = 128;
constexpr int kGramK = 64;                               // samples per tile
template <bool TF32>
__host__ __device__ constexpr uint32_t gram_tile_bytes() { return 128u * 64u * (TF32 ? 4u : 2u); }   // 128 rows x 64 samples

// NV, D > 0: the total-degree basis of D in NV variables, its monomials from
// compile-time exponents; D = 0: any basis, from the exponent table
template <typename TS, int NV, int D, bool TF32>
__global__ void __launch_bounds__(kGramThreads)
gram_umma_kernel(const __grid_constant__ FitParams P, int n_cols, int tmem_cols) {
    constexpr uint32_t kGramTileBytes = gram_tile_bytes<TF32>();
    extern __shared__ unsigned char gsm_raw[];
    unsigned char* tiles = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t mb[2];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&mb[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&mb[1])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_addr(&tmem_base)), "r"((uint32_t)tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t s_tiles = smem_addr(tiles);
    const uint32_t idesc = TF32 ? umma_idesc_tf32(128, n_cols) : umma_idesc_bf16(128, n_cols);
    const int nv = P.n_vars, m = P.m, u = P.u;
    const TS* X = reinterpret_cast<const TS*>(P.x);
    const TS* Y = reinterpret_cast<const TS*>(P.y);
    const float sN = ldexpf(1.0f, -P.n_scale_log2), sB = ldexpf(1.0f, -P.b_scale_log2);
    const int k = tid & (kGramK - 1);            // this thread's sample within a tile
    const int half = tid >> 6;                   // 0: rows Phi, 1: rows -y Phi
    // one element of the design matrix into the tile, in the operand type
    auto put = [&](unsigned char* tile, int r, float v) {
        if constexpr (TF32) *reinterpret_cast<uint32_t*>(tile + swz_off4(r, k, 128)) = to_tf32(v);
        else *reinterpret_cast<__nv_bfloat16*>(tile + swz_off(r, k, 128)) = __float2bfloat16_rn(v);
    };
    uint32_t phase[2] = {0u, 0u};
    bool pending[2] = {false, false};
    // wait for buffer b's products (bounded; a wait that gives up stops the
    // CTA's products, and its buffer stays pending for the final wait)
    auto drain = [&](int b) {
        if (!pending[b] || abort_flag) return;
        if (mbar_wait(&mb[b], phase[b])) {
            phase[b] ^= 1u;
            pending[b] = false;
        } else {
            abort_flag = 1;
        }
    };
    for (int f = blockIdx.x; f < P.n_fits; f += gridDim.x) {
        const int64_t s0 = P.offsets[f], s1 = P.offsets[f + 1];
        const int64_t n_tiles = (s1 - s0 + kGramK - 1) / kGramK;
        bool bad = false;
        // this thread's sample of the next tile is loaded while the current
        // one is built, so that its loads are in flight meanwhile
        TS cx[kMaxVars] = {}, cy = TS(0);
        auto fetch = [&](int64_t c, TS (&xv)[kMaxVars], TS& yv) {
            const int64_t s = s0 + c * kGramK + k;
            if (s < s1) {
#pragma unroll
                for (int v = 0; v < kMaxVars; ++v)
                    if (v < nv) xv[v] = X[(int64_t)v * P.x_stride + s];
                yv = Y[s];
            }
        };
        if (n_tiles > 0) fetch(0, cx, cy);
        for (int64_t c = 0; c < n_tiles; ++c) {
            const int b = (int)(c & 1);
            TS nx[kMaxVars] = {}, ny = TS(0);
            if (c + 1 < n_tiles) fetch(c + 1, nx, ny);
            drain(b);                            // the products that read this buffer are done
            unsigned char* tile = tiles + b * kGramTileBytes;
            const bool live = s0 + c * kGramK + k < s1;
            float xs[kMaxVars] = {0.f, 0.f, 0.f, 0.f};
            float sc = 0.f;                      // 0 past the fit's end: zero columns
            if (live) {
#pragma unroll
                for (int v = 0; v < kMaxVars; ++v) {
                    if (v < nv) {
                        bad |= !isfinite(cx[v]);
                        xs[v] = (float)cx[v] * (v == 0 ? sN : sB);
                    }
                }
                bad |= !isfinite(cy);
                sc = half ? -(float)cy : 1.0f;
            }
#pragma unroll
            for (int v = 0; v < kMaxVars; ++v) cx[v] = nx[v];
            cy = ny;
            if constexpr (D > 0) {
                constexpr MonoTable<NV, D> tab{};
                constexpr int NM = MonoTable<NV, D>::count();
                float pw[NV][D + 1];
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    pw[v][0] = 1.f;
#pragma unroll
                    for (int e = 1; e <= D; ++e) pw[v][e] = pw[v][e - 1] * xs[v];
                }
#pragma unroll
                for (int t = 0; t < NM; ++t) {
                    float ph = pw[0][tab.e[t][0]] * pw[1][tab.e[t][1]];
                    if constexpr (NV > 2) ph *= pw[2][tab.e[t][2]];
                    if constexpr (NV > 3) ph *= pw[3][tab.e[t][3]];
                    put(tile, half * NM + t, sc * ph);
                }
            } else {
                for (int t = 0; t < m; ++t) {
                    float ph = 1.f;
                    for (int v = 0; v < nv; ++v)
                        for (int e = 0; e < P.exps[t][v]; ++e) ph *= xs[v];
                    put(tile, half * m + t, sc * ph);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            if (tid == 0 && !abort_flag) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if constexpr (TF32) {
#pragma unroll
                    for (int kk = 0; kk < kGramK / 8; ++kk) {   // 32-byte steps, two blocks
                        const uint64_t d = umma_desc(s_tiles + b * kGramTileBytes +
                                                     (kk >> 2) * 128 * 128 + (kk & 3) * 32);
                        umma_tf32(tmem, d, d, idesc, (c > 0 || kk > 0) ? 1u : 0u);
                    }
                } else {
#pragma unroll
                    for (int kk = 0; kk < kGramK / 16; ++kk) {
                        const uint64_t d = umma_desc(s_tiles + b * kGramTileBytes + kk * 32);
                        umma_bf16(tmem, d, d, idesc, (c > 0 || kk > 0) ? 1u : 0u);
                    }
                }
                umma_commit(&mb[b]);
            }
            if (!abort_flag) pending[b] = true;
        }
        drain(0);
        drain(1);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // the accumulator of rows 32 warp .. 32 warp + 31, read 32 columns at a time
        double* G = P.mom + (int64_t)f * u * u;
        const int i = 32 * warp + lane;
        for (int c0 = 0; c0 < n_cols; c0 += 32) {
            float v[32];
            const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
            tmem_ld16x2(ta, ta + 16, v);
            if (i < u && n_tiles > 0 && !abort_flag)
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (c0 + j < u) G[(int64_t)i * u + c0 + j] = (double)v[j];
        }
        const int any_bad = __syncthreads_or(bad ? 1 : 0);
        if (tid == 0) P.flags[f] = (any_bad || abort_flag) ? 1 : 0;
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    // the last products of a CTA that gave up a wait: wait again (bounded)
    if (abort_flag) {
        if (pending[0]) mbar_wait(&mb[0], phase[0]);
        if (pending[1]) mbar_wait(&mb[1], phase[1]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :: "r"(tmem), "r"((uint32_t)tmem_cols));
    }
}

template <typename TS, bool TF32>
klr_status launch_gram_umma(const FitParams& P, int n_sm, size_t smem_optin, cudaStream_t stream) {
    const size_t kGramSmemMin = 1024 + 2 * (size_t)gram_tile_bytes<TF32>();
    const int n_cols = (P.u + 15) / 16 * 16;             // N: a multiple of 16 for M = 128
    const int read_cols = (n_cols + 31) / 32 * 32;
    const int tmem_cols = read_cols <= 32 ? 32 : read_cols <= 64 ? 64 : read_cols <= 128 ? 128 : 256;
    if (P.u > 128 || n_cols > 256) {
        set_error("klr_fit: %d unknowns exceed the tensor-core Gram's 128 rows", P.u);
        return KLR_ENOTSUP;
    }
    // CTAs per SM: as many as tensor memory holds (512 columns), at most 6;
    // the shared memory asked for keeps more from sharing an SM
    const int per_sm = std::min(6, 512 / tmem_cols);
    const size_t smem = std::max(kGramSmemMin, std::min((size_t)smem_optin, (size_t)(228 * 1024) / per_sm - 1024));
    auto kern = P.box ? gram_umma_kernel<TS, 0, 0, TF32>
              : P.n_vars == 3 ? (P.degree == 1 ? gram_umma_kernel<TS, 3, 1, TF32>
                                 : P.degree == 2 ? gram_umma_kernel<TS, 3, 2, TF32>
                                                 : gram_umma_kernel<TS, 3, 3, TF32>)
                              : (P.degree == 1 ? gram_umma_kernel<TS, 4, 1, TF32>
                                 : P.degree == 2 ? gram_umma_kernel<TS, 4, 2, TF32>
                                                 : gram_umma_kernel<TS, 4, 3, TF32>);
    KLR_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
    const int grid = (int)std::min<int64_t>(P.n_fits, (int64_t)per_sm * n_sm);
    kern<<<grid, kGramThreads, smem, stream>>>(P, n_cols, tmem_cols);
    KLR_CHECK_CUDA(cudaGetLastError());
    return KLR_OK;
}

// wpb: warps (fits) per block, 1, 2 or 4 (an autotuned choice)
template <typename TS, int ACC>
klr_status launch_moments(const FitParams& P, int n_mom, int rec, int wpb, cudaStream_t stream) {
    // lanes per sample (moment groups) so that a lane holds at most MAXT moments
    const size_t tc = ACC == ACC_FP64 ? 8 : 4;
    FitParams Q = P;
    Q.warp_smem = (int)((32 * rec * tc + 15) & ~(size_t)15);
    const int blocks = (P.n_fits + wpb - 1) / wpb;
    // specialised kernels for the common bases (degree 2 in 3 or 4 variables,
    // degree 3 in 3 variables)
    auto fast = [&](auto kern, int nm) -> klr_status {
        FitParams R = P;
        const int rec_ = nm + 3 + ((nm + 3) % 2 == 0 ? 1 : 0);
        R.warp_smem = (int)((32 * rec_ * tc + 15) & ~(size_t)15);
        int nb = blocks, nw = wpb;
        size_t smem = (size_t)R.warp_smem * wpb;
        if (ACC == ACC_FP64 && P.mom_warps > 1) {
            nb = P.n_fits;
            nw = P.mom_warps;
            smem = (size_t)R.warp_smem * nw + sizeof(double) * 3 * nm * nw;
        } else {
            R.mom_warps = 1;
        }
        KLR_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem));
        kern<<<nb, nw * 32, smem, stream>>>(R);
        KLR_CHECK_CUDA(cudaGetLastError());
        return KLR_OK;
    };
    if (!P.box && P.n_vars == 3 && P.degree == 2)
        return fast(moments_fast_kernel<TS, ACC, 3, 4, 4, 9>, 35);
    if (!P.box && P.n_vars == 4 && P.degree == 2)
        return fast(moments_fast_kernel<TS, ACC, 4, 4, 8, 9>, 70);
    if (!P.box && P.n_vars == 3 && P.degree == 3)
        return fast(moments_fast_kernel<TS, ACC, 3, 6, 8, 11>, 84);
    const size_t smem = (size_t)Q.warp_smem * wpb;
    auto generic = [&](auto kern) -> klr_status {
        KLR_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem));
        kern<<<blocks, wpb * 32, smem, stream>>>(Q);
        return KLR_OK;
    };
    klr_status st;
    if (n_mom <= 4 * 9) st = generic(moments_kernel<TS, ACC, 4, 9>);
    else if (n_mom <= 8 * 11) st = generic(moments_kernel<TS, ACC, 8, 11>);
    else st = generic(moments_kernel<TS, ACC, 16, 14>);
    if (st != KLR_OK) return st;
    KLR_CHECK_CUDA(cudaGetLastError());
    return KLR_OK;
}

// moments_fast_kernel for the degree-2 basis in (N, b0, b1), DF32, FP32,
// KLR_EXP8 or KLR_EXP16 samples (the binned path's per-sample kernel).  The
// fallback launch (P.fallback_only) takes one resident wave of blocks whose
// warps step over the fits, so that a batch the binned kernel covered whole
// costs a scan of the flags (one load per 32 fits a warp) instead of a block
// per wpb fits.
template <int XF>
klr_status launch_moments_fast_xf(const FitParams& P, int n_sm, int wpb, cudaStream_t stream) {
    auto kern = P.fallback_only ? moments_fast_kernel<float, ACC_DF32, 3, 4, 4, 9, XF, true>
                                : moments_fast_kernel<float, ACC_DF32, 3, 4, 4, 9, XF, false>;
    FitParams R = P;
    const int rec_ = 35 + 3 + ((35 + 3) % 2 == 0 ? 1 : 0);
    R.warp_smem = (int)((32 * rec_ * 4 + 15) & ~(size_t)15);
    KLR_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        R.warp_smem * wpb));
    int64_t grid = (P.n_fits + wpb - 1) / wpb;
    if (P.fallback_only) {
        int per_sm = 0;
        KLR_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, kern, wpb * 32, (size_t)R.warp_smem * wpb));
        grid = std::min<int64_t>(grid, (int64_t)std::max(1, per_sm) * std::max(1, n_sm));
    }
    kern<<<(int)grid, wpb * 32, (size_t)R.warp_smem * wpb, stream>>>(R);
    KLR_CHECK_CUDA(cudaGetLastError());
    return KLR_OK;
}

// DF32 degree-2 fits in (N, b0, b1): the binned moments kernel on a
// persistent grid (one warp per fit at a time), then the per-sample kernel
// over the fits it left (flag bit 2).
template <int XF>
klr_status launch_moments_binned_t(const FitParams& P, int n_sm, int wpb, cudaStream_t stream) {
    const size_t smem = kBinWarpSmem;
    auto kern = moments_binned_kernel<XF>;
    KLR_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
    int per_sm = 0;
    KLR_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32, smem));
    const int64_t slots = (int64_t)std::max(1, per_sm) * std::max(1, n_sm);
    const int grid = (int)std::min<int64_t>(P.n_fits, slots);
    kern<<<grid, 32, smem, stream>>>(P);
    KLR_CHECK_CUDA(cudaGetLastError());
    // the per-sample kernel over the fits left (flag bit 2)
    FitParams Q = P;
    Q.fallback_only = 1;
    return launch_moments_fast_xf<XF>(Q, n_sm, wpb, stream);
}

klr_status launch_moments_binned(const FitParams& P, int n_sm, int rec, int wpb,
                                 cudaStream_t stream) {
    (void)rec;
    return P.x_fmt == kXExp8    ? launch_moments_binned_t<kXExp8>(P, n_sm, wpb, stream)
         : P.x_fmt == kXExp16 ? launch_moments_binned_t<kXExp16>(P, n_sm, wpb, stream)
                              : launch_moments_binned_t<kXFloat>(P, n_sm, wpb, stream);
}

template <typename TS>
klr_status launch_solve_warp(const FitParams& P, size_t smem_optin, int n_sm, cudaStream_t stream) {
    size_t per_warp = sizeof(double) * (3 * (size_t)P.n_mom + (size_t)P.u * P.ld + 6 * (size_t)P.u);
    per_warp = (per_warp + 15) & ~(size_t)15;
    FitParams Q = P;
    Q.warp_smem = (int)per_warp;
    Q.fit_warps = 1;
    int wpb = 4;
    while (wpb > 1 && per_warp * wpb > 96 * 1024) wpb >>= 1;
    size_t smem = per_warp * wpb;
    int blocks = (P.n_fits + wpb - 1) / wpb;
    if (P.n_fits <= (int64_t)n_sm) {
        // a few fits (a latency): a block per fit, and with refinement passes
        // one warp per scheduler for the passes over the samples
        Q.fit_warps = P.refine > 0 ? 4 : 1;
        wpb = Q.fit_warps;
        smem = per_warp + (Q.fit_warps > 1 ? sizeof(double) * 64 * Q.fit_warps : 0);
        blocks = P.n_fits;
    }
    if (smem > smem_optin) {
        set_error("klr_fit: %zu bytes of shared memory per fit exceed the device limit", per_warp);
        return KLR_ENOTSUP;
    }
    KLR_CHECK_CUDA(cudaFuncSetAttribute(solve_warp_kernel<TS>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    solve_warp_kernel<TS><<<blocks, wpb * 32, smem, stream>>>(Q);
    KLR_CHECK_CUDA(cudaGetLastError());
    return KLR_OK;
}

klr_status launch_solve_lane_dw(const FitParams& P, cudaStream_t stream) {
    const size_t smem = sizeof(float2) * 32 * ((size_t)P.u * (P.u + 1) / 2 + 4 * (size_t)P.u);
    KLR_CHECK_CUDA(cudaFuncSetAttribute(solve_lane_dw_kernel,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    solve_lane_dw_kernel<<<(P.n_fits + 31) / 32, 32, smem, stream>>>(P);
    KLR_CHECK_CUDA(cudaGetLastError());
    return KLR_OK;
}

template <int Q, int MAXR>
klr_status launch_solve_group_dw_q(const FitParams& P, cudaStream_t stream) {
    constexpr int GPW = 32 / Q;
    if (P.u > Q * MAXR) {
        set_error("group solver: %d unknowns exceed %d rows per lane", P.u, MAXR);
        return KLR_ENOTSUP;
    }
    FitParams Q_ = P;
    // L, 1/L_jj, v, w, D (floats) and the previous Lanczos vector
    int stride = P.u * (P.u + 1) / 2 + 4 * P.u + (P.u + 1) / 2;
    // stride = Q mod 2Q float2: the eight groups of a half-warp then meet
    // fewest shared-memory bank conflicts in the solves and the factor (the
    // lanes of a group read rows i, i + 1, ... of one column)
    while (stride % (2 * Q) != Q) ++stride;
    Q_.ld = stride;
    const size_t smem = sizeof(float2) * (size_t)stride * GPW;
    KLR_CHECK_CUDA(cudaFuncSetAttribute(solve_group_dw_kernel<Q, MAXR>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    solve_group_dw_kernel<Q, MAXR><<<(P.n_fits + GPW - 1) / GPW, 32, smem, stream>>>(Q_);
    KLR_CHECK_CUDA(cudaGetLastError());
    return KLR_OK;
}

// q_lanes: lanes per fit, 2, 4 or 8 (an autotuned choice)
// (rows per lane: enough for 20 unknowns, the degree-2 basis in (N, b0, b1),
// else for the solver's limit of 30)
klr_status launch_solve_group_dw(const FitParams& P, int q_lanes, cudaStream_t stream) {
    const bool small = P.u <= 20;
    if (q_lanes == 2)
        return small ? launch_solve_group_dw_q<2, 10>(P, stream)
                     : launch_solve_group_dw_q<2, 15>(P, stream);
    if (q_lanes == 8)
        return small ? launch_solve_group_dw_q<8, 3>(P, stream)
                     : launch_solve_group_dw_q<8, 4>(P, stream);
    return small ? launch_solve_group_dw_q<4, 5>(P, stream) : launch_solve_group_dw_q<4, 8>(P, stream);
}

klr_status launch_solve_lane(const FitParams& P, cudaStream_t stream) {
    const size_t smem = sizeof(double) * 32 * ((size_t)P.u * (P.u + 1) / 2 + 4 * (size_t)P.u);
    KLR_CHECK_CUDA(cudaFuncSetAttribute(solve_lane_kernel,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    solve_lane_kernel<<<(P.n_fits + 31) / 32, 32, smem, stream>>>(P);
    KLR_CHECK_CUDA(cudaGetLastError());
    return KLR_OK;
}


// Held-out error of fitted rational functions: one warp per fit, lanes over
// its samples, in FP64: sqrt(mean(((p/q)(x_s) - y_s) / y_s)^2).
template <typename TS>
__global__ void __launch_bounds__(128)
heldout_kernel(const __grid_constant__ FitParams P, double* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int f = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (f >= P.n_fits) return;
    const int m = P.m, nv = P.n_vars;
    const int64_t s0 = P.offsets[f], s1 = P.offsets[f + 1];
    const TS* X = reinterpret_cast<const TS*>(P.x);
    const TS* Y = reinterpret_cast<const TS*>(P.y);
    const double sN = ldexp(1.0, -P.n_scale_log2), sB = ldexp(1.0, -P.b_scale_log2);
    double acc = 0.0;
    for (int64_t s = s0 + lane; s < s1; s += 32) {
        double pw[kMaxVars][4];
        for (int v = 0; v < nv; ++v) {
            const double xv = (double)X[(int64_t)v * P.x_stride + s] * (v == 0 ? sN : sB);
            pw[v][0] = 1.0;
            for (int e = 1; e < 4; ++e) pw[v][e] = pw[v][e - 1] * xv;
        }
        double p = 0.0, q = 0.0;
        for (int t = 0; t < m; ++t) {
            double phi = 1.0;
            for (int v = 0; v < nv; ++v) phi *= pw[v][P.exps[t][v]];
            const double a = P.coef_f64 ? reinterpret_cast<const double*>(P.coef)[(int64_t)f * P.u + t]
                                        : (double)reinterpret_cast<const float*>(P.coef)[(int64_t)f * P.u + t];
            const double b = P.coef_f64 ? reinterpret_cast<const double*>(P.coef)[(int64_t)f * P.u + m + t]
                                        : (double)reinterpret_cast<const float*>(P.coef)[(int64_t)f * P.u + m + t];
            p += a * phi;
            q += b * phi;
        }
        const double y = (double)Y[s];
        const double r = (p / q - y) / y;
        acc += r * r;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[f] = s1 > s0 ? sqrt(acc / (double)(s1 - s0)) : 0.0;
}

// The basis choice of klr_choose_basis, one thread per fit, in FP64: the
// least finite error, the threshold (least (1 + tol)) + floor with each
// operation rounded on its own, then the eligible column with the fewest
// monomials (the lower column on ties).
struct ChooseBasisParams {
    int32_t sizes[KLR_CHOOSE_BASIS_MAX_CAND];
    int n_cand;
    double tol1, floor;
};

__global__ void __launch_bounds__(256)
choose_basis_kernel(const double* __restrict__ err, int64_t n_fits,
                    const __grid_constant__ ChooseBasisParams P, int32_t* __restrict__ out) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n_fits) return;
    const double* e = err + f * P.n_cand;
    double lo = INFINITY;
    for (int j = 0; j < P.n_cand; ++j)
        if (isfinite(e[j]) && e[j] < lo) lo = e[j];
    int pick = -1;
    if (lo < INFINITY) {
        const double lim = __dadd_rn(__dmul_rn(lo, P.tol1), P.floor);
        for (int j = 0; j < P.n_cand; ++j)
            if (isfinite(e[j]) && e[j] <= lim && (pick < 0 || P.sizes[j] < P.sizes[pick]))
                pick = j;
    }
    out[f] = pick;
}

}  // namespace

size_t fit_workspace_bytes(int64_t n_fits, int n_mom) {
    return 256 + (size_t)n_fits * (3 * (size_t)n_mom * sizeof(double) + sizeof(int32_t));
}

constexpr int32_t kFitDefaultChoice = 0x21;   // 4 warps per block, 4 lanes per fit

// Problem class of a fit batch for the autotuner: basis, precision, sample
// type, refinement on/off, and log2 buckets of the fit count and of the mean
// samples per fit (x_stride is the sample count of the SoA layout).
uint64_t fit_tune_key(const klr_fit_batch* b) {
    const int64_t per_fit = b->n_fits > 0 ? b->x_stride / b->n_fits : 0;
    return tune_key(TUNE_FIT, {b->n_vars, b->degree, b->precision, b->sample_dtype,
                               b->refine_iters > 0, log2_bucket(b->n_fits),
                               log2_bucket(per_fit), b->var_degree[0], b->var_degree[1],
                               b->var_degree[2], b->var_degree[3]});
}

}  // namespace klr

using namespace klr;

namespace {

enum { STAGE_GRAM = 1, STAGE_SOLVE = 2 };

// The fit in two stages: F1-F2 (moment sums, or the tensor-core Gram matrix,
// into the context's scratch) and F3-F4 (the null-vector solve and any
// refinement, from that scratch).
klr_status fit_impl(klr_ctx* ctx, const klr_fit_batch* b, void* coef_out, int32_t coef_dtype,
                    int32_t* fit_status, double* fit_diag, void* stream_, int stages) {
    KLR_REQUIRE(ctx && b, "klr_fit: NULL context or batch");
    Context* c = reinterpret_cast<Context*>(ctx);
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    KLR_REQUIRE(b->n_fits >= 0, "klr_fit: n_fits < 0");
    KLR_REQUIRE(b->n_vars == 3 || b->n_vars == 4, "klr_fit: n_vars %d not 3 or 4", b->n_vars);
    const bool box = b->var_degree[0] > 0;
    KLR_REQUIRE(box || (b->degree >= 1 && b->degree <= 3), "klr_fit: degree %d not in 1..3",
                b->degree);
    KLR_REQUIRE(b->sample_dtype == KLR_F32 || b->sample_dtype == KLR_F64 ||
                b->sample_dtype == KLR_EXP8 || b->sample_dtype == KLR_EXP16,
                "klr_fit: bad sample_dtype");
    KLR_REQUIRE(!(stages & STAGE_SOLVE) || coef_dtype == KLR_F32 || coef_dtype == KLR_F64,
                "klr_fit: bad coef_dtype");
    KLR_REQUIRE(b->precision >= KLR_FIT_FP64 && b->precision <= KLR_FIT_BF16,
                "klr_fit: bad precision %d", b->precision);
    KLR_REQUIRE(b->refine_iters >= 0 && b->refine_iters <= 8, "klr_fit: refine_iters not in 0..8");
    KLR_REQUIRE(b->n_scale_log2 >= -64 && b->n_scale_log2 <= 64 &&
                b->b_scale_log2 >= -64 && b->b_scale_log2 <= 64, "klr_fit: scale out of range");
    if (b->n_fits == 0) return KLR_OK;
    KLR_REQUIRE(b->offsets && b->x && b->y, "klr_fit: NULL device array");
    KLR_REQUIRE(!(stages & STAGE_SOLVE) || (coef_out && fit_status),
                "klr_fit: NULL coef_out or fit_status");
    KLR_REQUIRE(b->x_stride >= 0, "klr_fit: x_stride < 0");
    if (b->precision == KLR_FIT_DF32)
        KLR_REQUIRE(b->sample_dtype == KLR_F32 || b->sample_dtype == KLR_EXP8 ||
                    b->sample_dtype == KLR_EXP16,
                    "klr_fit: DF32 needs KLR_F32, KLR_EXP8 or KLR_EXP16 samples");
    if ((b->sample_dtype == KLR_EXP8 || b->sample_dtype == KLR_EXP16) &&
        !(b->precision == KLR_FIT_DF32 && b->n_vars == 3 && !box && b->degree == 2 &&
          b->refine_iters == 0)) {
        set_error("klr_fit: KLR_EXP8 and KLR_EXP16 samples need KLR_FIT_DF32, the degree-2 "
                  "basis in (N, b0, b1) and no refinement");
        return KLR_ENOTSUP;
    }
    Basis basis;
    KLR_REQUIRE(make_basis(b->n_vars, b->degree, b->var_degree, &basis),
                "klr_fit: no basis (per-variable bounds must be 0..3, at most %d monomials)",
                kMaxBasis);
    const int m = basis.m, u = 2 * m;
    if (b->refine_iters > 0 && u > kRefineMaxU) {
        set_error("klr_fit: refinement supports at most %d unknowns (have %d)", kRefineMaxU, u);
        return KLR_ENOTSUP;
    }
    KLR_CHECK_CUDA(cudaSetDevice(c->device));
    // launch shapes: moments warps per block (bits 4-7: 1, 2, 4) and lanes
    // per fit of the group solver (bits 0-3: 2, 4, 8)
    // (a batch of at most one fit per SM: one moments warp per block, so the
    // fits spread over the SMs)
    const int32_t choice = tune_choice(c, fit_tune_key(b),
                                       b->n_fits <= (int64_t)c->n_sm ? (kFitDefaultChoice & ~0xF0)
                                                                     : kFitDefaultChoice);
    const int wpb = 1 << std::min(2, (choice >> 4) & 15);
    const int q_lanes = 2 << std::min(2, choice & 15);

    FitParams P{};
    P.n_fits = b->n_fits;
    P.n_vars = b->n_vars;
    // the moments kernel tabulates powers up to twice the largest bound
    P.box = box ? 1 : 0;
    P.degree = b->degree;
    if (box) {
        P.degree = 0;
        for (int v = 0; v < b->n_vars; ++v) P.degree = std::max(P.degree, (int)b->var_degree[v]);
    }
    P.m = m;
    P.u = u;
    P.n_mom = basis.n_mom;
    P.n_scale_log2 = b->n_scale_log2;
    P.b_scale_log2 = b->b_scale_log2;
    P.offsets = b->offsets;
    P.x = b->x;
    P.x_stride = b->x_stride;
    P.y = b->y;
    P.coef = coef_out;
    P.coef_f64 = coef_dtype == KLR_F64;
    P.status = fit_status;
    P.diag = fit_diag;
    P.refine = b->refine_iters;
    P.fallback_only = 0;
    P.x_fmt = b->sample_dtype == KLR_EXP8 ? kXExp8 : b->sample_dtype == KLR_EXP16 ? kXExp16 : kXFloat;
    // a few FP64 fits (a latency): each fit's samples over one warp per scheduler
    P.mom_warps = b->precision == KLR_FIT_FP64 && b->n_fits <= (int64_t)c->n_sm ? 4 : 1;
    P.ld = (u % 2) ? u : u + 1;
    memcpy(P.exps, basis.exps, sizeof(P.exps));
    memcpy(P.pair, basis.pair, sizeof(P.pair));

    // unit roundoff of the Gram entries in each mode (the accumulated error of
    // the low-precision modes is a few of these, hence the factor 16)
    // FP64/DF32: the error of an entry is tiny next to the spectrum, the levels
    // carry a factor u; FP32/TF32/BF16: the levels sit at a few roundoffs of
    // the trace, below the second eigenvalue of the fits they can resolve.
    switch (b->precision) {
        case KLR_FIT_FP64: P.gram_eps = ldexp(1.0, -53); break;
        case KLR_FIT_DF32: P.gram_eps = ldexp(1.0, -44); break;
        case KLR_FIT_FP32: P.gram_eps = ldexp(1.0, -24); break;
        case KLR_FIT_TF32: P.gram_eps = ldexp(1.0, -11); break;
        default: P.gram_eps = ldexp(1.0, -8); break;
    }
    if (b->precision == KLR_FIT_FP64 || b->precision == KLR_FIT_DF32) {
        P.f_jit = 4.0 * u;
        P.f_null = 64.0 * u;
        P.f_rank = 8.0 * u;
    } else {
        P.f_jit = 2.0;
        P.f_null = 8.0;
        P.f_rank = 1.0;
    }
    const bool tc = b->precision == KLR_FIT_TF32 || b->precision == KLR_FIT_BF16;
    if (tc) {
        // tensor-core Gram matrix, then the FP64 warp solver (+ refinement)
        const size_t bytes = 256 + (size_t)b->n_fits * ((size_t)u * u * sizeof(double) + 4);
        klr_status st = ensure_workspace(c, bytes, stream);
        if (st != KLR_OK) return st;
        P.mom = reinterpret_cast<double*>(reinterpret_cast<char*>(c->ws) + 256);
        P.flags = reinterpret_cast<int32_t*>(P.mom + (size_t)b->n_fits * u * u);
        P.mom_dw = 0;
        P.gram_direct = 1;
        const bool s64 = b->sample_dtype == KLR_F64;
        const bool bf = b->precision == KLR_FIT_BF16;
        if (stages & STAGE_GRAM) {
            st = s64 ? (bf ? launch_gram_umma<double, false>(P, c->n_sm, c->smem_optin, stream)
                           : launch_gram_umma<double, true>(P, c->n_sm, c->smem_optin, stream))
                     : (bf ? launch_gram_umma<float, false>(P, c->n_sm, c->smem_optin, stream)
                           : launch_gram_umma<float, true>(P, c->n_sm, c->smem_optin, stream));
            if (st != KLR_OK) return st;
        }
        if (!(stages & STAGE_SOLVE)) return KLR_OK;
        return s64 ? launch_solve_warp<double>(P, c->smem_optin, c->n_sm, stream)
                   : launch_solve_warp<float>(P, c->smem_optin, c->n_sm, stream);
    }
    P.gram_direct = 0;
    klr_status st = ensure_workspace(c, fit_workspace_bytes(b->n_fits, basis.n_mom), stream);
    if (st != KLR_OK) return st;
    P.mom = reinterpret_cast<double*>(reinterpret_cast<char*>(c->ws) + 256);
    P.flags = reinterpret_cast<int32_t*>(P.mom + (size_t)b->n_fits * 3 * basis.n_mom);
    P.mom_dw = b->precision != KLR_FIT_FP64;
    const int rec = b->n_vars * (2 * P.degree + 1) + 3;
    const bool s64 = b->sample_dtype == KLR_F64;
    if (stages & STAGE_GRAM) switch (b->precision) {
        case KLR_FIT_FP64:
            st = s64 ? launch_moments<double, ACC_FP64>(P, basis.n_mom, rec, wpb, stream)
                     : launch_moments<float, ACC_FP64>(P, basis.n_mom, rec, wpb, stream);
            break;
        case KLR_FIT_DF32:
            // binned moments where they apply (degree 2 in (N, b0, b1); the
            // block-size scale keeps every monomial's power of two normal)
            if (!box && b->n_vars == 3 && b->degree == 2 && b->b_scale_log2 >= 5 &&
                b->b_scale_log2 <= 15)
                st = launch_moments_binned(P, c->n_sm, rec, wpb, stream);
            else if (P.x_fmt == kXExp8)   // (the exponent formats come only with this basis)
                st = launch_moments_fast_xf<kXExp8>(P, c->n_sm, wpb, stream);
            else if (P.x_fmt == kXExp16)
                st = launch_moments_fast_xf<kXExp16>(P, c->n_sm, wpb, stream);
            else
                st = launch_moments<float, ACC_DF32>(P, basis.n_mom, rec, wpb, stream);
            break;
        case KLR_FIT_FP32:
            st = s64 ? launch_moments<double, ACC_FP32>(P, basis.n_mom, rec, wpb, stream)
                     : launch_moments<float, ACC_FP32>(P, basis.n_mom, rec, wpb, stream);
            break;
        default:
            set_error("klr_fit: unsupported precision");
            return KLR_ENOTSUP;
    }
    if (b->precision != KLR_FIT_FP64 && b->precision != KLR_FIT_DF32 &&
        b->precision != KLR_FIT_FP32) {
        set_error("klr_fit: unsupported precision");
        return KLR_ENOTSUP;
    }
    if (st != KLR_OK) return st;
    if (!(stages & STAGE_SOLVE)) return KLR_OK;
    if (b->refine_iters == 0 && u <= kLaneMaxU)
        return P.mom_dw ? launch_solve_group_dw(P, q_lanes, stream) : launch_solve_lane(P, stream);
    return s64 ? launch_solve_warp<double>(P, c->smem_optin, c->n_sm, stream)
               : launch_solve_warp<float>(P, c->smem_optin, c->n_sm, stream);
}

}  // namespace

extern "C" klr_status klr_fit(klr_ctx* ctx, const klr_fit_batch* b, void* coef_out,
                              int32_t coef_dtype, int32_t* fit_status, double* fit_diag,
                              void* stream) {
    return fit_impl(ctx, b, coef_out, coef_dtype, fit_status, fit_diag, stream,
                    STAGE_GRAM | STAGE_SOLVE);
}

extern "C" klr_status klr_fit_gram(klr_ctx* ctx, const klr_fit_batch* b, void* stream) {
    return fit_impl(ctx, b, nullptr, KLR_F32, nullptr, nullptr, stream, STAGE_GRAM);
}

extern "C" klr_status klr_fit_solve(klr_ctx* ctx, const klr_fit_batch* b, void* coef_out,
                                    int32_t coef_dtype, int32_t* fit_status, double* fit_diag,
                                    void* stream) {
    return fit_impl(ctx, b, coef_out, coef_dtype, fit_status, fit_diag, stream, STAGE_SOLVE);
}

extern "C" klr_status klr_autotune_fit(klr_ctx* ctx, const klr_fit_batch* b, void* coef_out,
                                       int32_t coef_dtype, int32_t* fit_status, double* fit_diag,
                                       int32_t* choice_out, float* ms_out, void* stream_) {
    KLR_REQUIRE(ctx && b, "klr_autotune_fit: NULL context or batch");
    Context* c = reinterpret_cast<Context*>(ctx);
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    auto run = [&]() -> klr_status {
        return klr_fit(ctx, b, coef_out, coef_dtype, fit_status, fit_diag, stream_);
    };
    if (b->n_fits == 0) return run();
    const uint64_t key = fit_tune_key(b);
    Basis basis;
    KLR_REQUIRE(make_basis(b->n_vars, b->degree, b->var_degree, &basis), "klr_autotune_fit: no basis");
    const int u = 2 * basis.m;
    const bool tc = b->precision == KLR_FIT_TF32 || b->precision == KLR_FIT_BF16;
    const bool group = !tc && b->precision != KLR_FIT_FP64 && b->refine_iters == 0 &&
                       u <= kLaneMaxU;
    if (tc) {   // one launch shape: time it so the outputs and timing are reported alike
        const int32_t only = kFitDefaultChoice;
        return tune_candidates(c, key, stream, &only, 1, 3, run, choice_out, ms_out);
    }
    // the two stages are independent: moments block shape first, then the
    // solver's lanes per fit with the chosen moments shape
    const int32_t s0 = kFitDefaultChoice & 15;
    const int32_t cm[3] = {0x00 | s0, 0x10 | s0, 0x20 | s0};
    int32_t best = kFitDefaultChoice;
    klr_status st = tune_candidates(c, key, stream, cm, 3, 3, run, &best, ms_out);
    if (st != KLR_OK || !group) {
        if (st == KLR_OK && choice_out) *choice_out = best;
        return st;
    }
    const int32_t cs[3] = {(best & 0xF0) | 0, (best & 0xF0) | 1, (best & 0xF0) | 2};
    return tune_candidates(c, key, stream, cs, 3, 3, run, choice_out, ms_out);
}

extern "C" klr_status klr_fit_heldout(klr_ctx* ctx, const klr_fit_batch* b, const void* coef,
                                      int32_t coef_dtype, double* err_out, void* stream_) {
    KLR_REQUIRE(ctx && b, "klr_fit_heldout: NULL context or batch");
    Context* c = reinterpret_cast<Context*>(ctx);
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    KLR_REQUIRE(b->n_fits >= 0, "klr_fit_heldout: n_fits < 0");
    KLR_REQUIRE(b->n_vars == 3 || b->n_vars == 4, "klr_fit_heldout: n_vars %d not 3 or 4", b->n_vars);
    KLR_REQUIRE(b->sample_dtype == KLR_F32 || b->sample_dtype == KLR_F64,
                "klr_fit_heldout: bad sample_dtype");
    KLR_REQUIRE(coef_dtype == KLR_F32 || coef_dtype == KLR_F64, "klr_fit_heldout: bad coef_dtype");
    const bool box = b->var_degree[0] > 0;
    KLR_REQUIRE(box || (b->degree >= 1 && b->degree <= 3), "klr_fit_heldout: degree %d not in 1..3",
                b->degree);
    if (b->n_fits == 0) return KLR_OK;
    KLR_REQUIRE(b->offsets && b->x && b->y && coef && err_out, "klr_fit_heldout: NULL array");
    Basis basis;
    KLR_REQUIRE(make_basis(b->n_vars, b->degree, b->var_degree, &basis), "klr_fit_heldout: no basis");
    KLR_CHECK_CUDA(cudaSetDevice(c->device));
    FitParams P{};
    P.n_fits = b->n_fits;
    P.n_vars = b->n_vars;
    P.m = basis.m;
    P.u = 2 * basis.m;
    P.n_scale_log2 = b->n_scale_log2;
    P.b_scale_log2 = b->b_scale_log2;
    P.offsets = b->offsets;
    P.x = b->x;
    P.x_stride = b->x_stride;
    P.y = b->y;
    P.coef = const_cast<void*>(coef);
    P.coef_f64 = coef_dtype == KLR_F64;
    memcpy(P.exps, basis.exps, sizeof(P.exps));
    const int grid = (int)(((int64_t)b->n_fits * 32 + 127) / 128);
    if (b->sample_dtype == KLR_F64) heldout_kernel<double><<<grid, 128, 0, stream>>>(P, err_out);
    else heldout_kernel<float><<<grid, 128, 0, stream>>>(P, err_out);
    KLR_CHECK_CUDA(cudaGetLastError());
    return KLR_OK;
}


extern "C" klr_status klr_choose_basis(klr_ctx* ctx, const double* errors, const int32_t* sizes,
                                       int64_t n_fits, int32_t n_cand, double tol, double floor,
                                       int32_t* choice_out, void* stream_) {
    KLR_REQUIRE(ctx, "klr_choose_basis: NULL context");
    Context* c = reinterpret_cast<Context*>(ctx);
    KLR_REQUIRE(n_fits >= 0, "klr_choose_basis: n_fits < 0");
    KLR_REQUIRE(n_cand >= 1 && n_cand <= KLR_CHOOSE_BASIS_MAX_CAND,
                "klr_choose_basis: n_cand %d not in 1..%d", n_cand, KLR_CHOOSE_BASIS_MAX_CAND);
    KLR_REQUIRE(std::isfinite(tol) && tol >= 0 && std::isfinite(floor) && floor >= 0,
                "klr_choose_basis: tol and floor must be finite and >= 0");
    KLR_REQUIRE(sizes, "klr_choose_basis: NULL sizes");
    ChooseBasisParams P{};
    for (int j = 0; j < n_cand; ++j) {
        KLR_REQUIRE(sizes[j] > 0, "klr_choose_basis: sizes[%d] = %d not > 0", j, sizes[j]);
        P.sizes[j] = sizes[j];
    }
    P.n_cand = n_cand;
    P.tol1 = 1.0 + tol;
    P.floor = floor;
    if (n_fits == 0) return KLR_OK;
    KLR_REQUIRE(errors && choice_out, "klr_choose_basis: NULL device array");
    KLR_CHECK_CUDA(cudaSetDevice(c->device));
    const int grid = (int)((n_fits + 255) / 256);
    choose_basis_kernel<<<grid, 256, 0, reinterpret_cast<cudaStream_t>(stream_)>>>(
        errors, n_fits, P, choice_out);
    KLR_CHECK_CUDA(cudaGetLastError());
    return KLR_OK;
}
