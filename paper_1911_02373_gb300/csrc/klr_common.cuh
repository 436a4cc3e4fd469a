// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <functional>
#include <string>
#include <utility>
#include <vector>

#include "klr.h"

namespace klr {

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
void set_error(const char* fmt, ...);

#define KLR_CHECK_CUDA(call)                                                       \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            ::klr::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                             __FILE__, __LINE__);                                  \
            return KLR_ECUDA;                                                      \
        }                                                                          \
    } while (0)

#define KLR_REQUIRE(cond, ...)                                                     \
    do {                                                                           \
        if (!(cond)) {                                                             \
            ::klr::set_error(__VA_ARGS__);                                         \
            return KLR_EINVAL;                                                     \
        }                                                                          \
    } while (0)

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
struct Context {
    int device = 0;
    int n_sm = 0;
    size_t smem_optin = 0;
    void* ws = nullptr;        // scratch memory owned by the context
    size_t ws_bytes = 0;
    // launch shapes chosen by the autotuner, per problem class (key)
    std::vector<std::pair<uint64_t, int32_t>> tuned;
    int32_t forced = -1;       // >= 0 while the autotuner times a candidate
};

// ---------------------------------------------------------------------------
// Autotuning of launch shapes.  A problem class is a key built from the
// parameters that decide which shape is fastest (operation, basis, precision,
// size buckets); a choice is an operation-specific shape code.
// ---------------------------------------------------------------------------
enum { TUNE_FIT = 1, TUNE_EVAL = 2 };

uint64_t tune_key(int op, std::initializer_list<int64_t> parts);
// the forced candidate, else the tuned choice for `key`, else `dflt`
int32_t tune_choice(const Context* c, uint64_t key, int32_t dflt);
void tune_store(Context* c, uint64_t key, int32_t choice);
// floor(log2(max(v, 1))): size buckets of the keys
int log2_bucket(int64_t v);
// Time run() once per candidate (each forced in turn): one untimed launch,
// then `reps` launches between CUDA events on `stream`.  Stores the fastest
// under `key`, then runs it once more so the outputs are its own.  Refuses
// (KLR_EINVAL) while `stream` is capturing a graph.
klr_status tune_candidates(Context* c, uint64_t key, cudaStream_t stream, const int32_t* cand,
                           int n_cand, int reps, const std::function<klr_status()>& run,
                           int32_t* choice_out, float* ms_out);

// Make sure the context scratch holds `bytes`; allocates only when the stream
// is not capturing.  Returns KLR_ENOMEM during capture if too small.
klr_status ensure_workspace(Context* ctx, size_t bytes, cudaStream_t stream);

// ---------------------------------------------------------------------------
// Monomial bases (graded lexicographic, total degree <= d)
// ---------------------------------------------------------------------------
constexpr int kMaxVars = 4;
constexpr int kMaxBasis = 35;     // C(4 + 3, 3)
constexpr int kMaxMoments = 210;  // C(4 + 6, 6): monomials of degree <= 2d

struct Basis {
    int n_vars;
    int degree;   // total degree bound, or the largest total degree of a box basis
    int box;      // 1: per-variable degree bounds
    int d_n;      // largest exponent of N in the basis
    int m;        // basis size
    int n_mom;    // monomials that are products of two basis monomials (the basis first)
    uint8_t exps[kMaxMoments][kMaxVars];   // exponents: the basis, then the other moments
    uint8_t pair[kMaxBasis][kMaxBasis];    // index of exps[i] + exps[j]
};

// Fill `b` for (n_vars, degree), or, when var_degree is not NULL and
// var_degree[0] > 0, for the per-variable bounds var_degree[0..n_vars) (the
// box basis of Section V-E); false if out of range.  Within each part,
// monomials are ordered by total degree, then by decreasing exponent tuple.
bool make_basis(int n_vars, int degree, const int32_t* var_degree, Basis* b);
int n_monomials(int n_vars, int degree);

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Occupancy rational program of Fig. 1: B_active by the four tests in order
// (blocks, warps, registers, shared memory per SM); T > T_max fails to launch.
__device__ __forceinline__ int occupancy_blocks(long long T, long long R, long long Z,
                                                long long Bm, long long Wm, long long Rm,
                                                long long Zm, long long Tmax) {
    if (T > Tmax || T <= 0) return 0;
    if (T * Bm <= 32 * Wm && R * T * Bm <= Rm && Z * Bm <= Zm) return (int)Bm;
    if (32 * Wm <= T * Bm && 32 * Wm * R <= Rm && 32 * Wm * Z <= Zm * T) return (int)((32 * Wm) / T);
    if (R > 0 && Rm <= R * T * Bm && Rm <= R * 32 * Wm && Rm * Z <= R * T * Zm)
        return (int)(Rm / (R * T));
    if (Z > 0 && Zm <= Bm * Z && Zm * T <= 32 * Wm * Z && Zm * R * T <= Z * Rm)
        return (int)(Zm / Z);
    return 0;
}

// Error-free sum (Knuth's TwoSum): a + b = s + e exactly.  The _rn
// intrinsics keep the compiler from contracting a product into these sums,
// which would break the error-free property.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

// Two FP32 values in one 64-bit register (the first in the low half), for
// the packed FP32x2 instructions of this architecture: one instruction
// computes both halves, each rounded as its scalar form is (round to nearest,
// no contraction).
typedef unsigned long long f2p;
__device__ __forceinline__ f2p f2p_make(float lo, float hi) {
    f2p r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float2 f2p_get(f2p v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ f2p f2p_add(f2p a, f2p b) {
    f2p d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2p f2p_sub(f2p a, f2p b) {
    f2p d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2p f2p_mul(f2p a, f2p b) {
    f2p d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// TwoSum (Knuth) of both halves at once: a + b = s + e exactly, per half
__device__ __forceinline__ void two_sum2(f2p a, f2p b, f2p& s, f2p& e) {
    s = f2p_add(a, b);
    const f2p bp = f2p_sub(s, a);
    e = f2p_add(f2p_sub(a, f2p_sub(s, bp)), f2p_sub(b, bp));
}

// Double-FP32 accumulator (hi, lo) += t with an error-free TwoSum.
__device__ __forceinline__ void df_add(float& hi, float& lo, float t) {
    float s, e;
    two_sum(hi, t, s, e);
    hi = s;
    lo += e;
}

// ---------------------------------------------------------------------------
// Double-word (two FP32) arithmetic: the error-free transformations of
// Knuth (TwoSum), Dekker (Fast2Sum) and FMA-based TwoProduct, and the
// double-word algorithms of Joldes, Muller and Popescu (ACM TOMS 2017):
// AccurateDWPlusDW, DWTimesDW, DWTimesFP.  A value is h + l with
// |l| <= ulp(h) / 2; about 2^-44 relative accuracy per operation.
// ---------------------------------------------------------------------------
struct dw {
    float h, l;
};

__device__ __forceinline__ dw dw_fast2sum(float a, float b) {  // needs |a| >= |b|
    float s = __fadd_rn(a, b);
    float t = __fsub_rn(b, __fsub_rn(s, a));
    return {s, t};
}
__device__ __forceinline__ dw dw_2sum(float a, float b) {
    float s, e;
    two_sum(a, b, s, e);
    return {s, e};
}
__device__ __forceinline__ dw dw_add(dw x, dw y) {
    dw s = dw_2sum(x.h, y.h);
    dw t = dw_2sum(x.l, y.l);
    float c = __fadd_rn(s.l, t.h);
    dw v = dw_fast2sum(s.h, c);
    float w = __fadd_rn(t.l, v.l);
    return dw_fast2sum(v.h, w);
}
__device__ __forceinline__ dw dw_neg(dw x) { return {-x.h, -x.l}; }
__device__ __forceinline__ dw dw_sub(dw x, dw y) { return dw_add(x, dw_neg(y)); }
__device__ __forceinline__ dw dw_mul(dw x, dw y) {
    float ch = __fmul_rn(x.h, y.h);
    float cl1 = fmaf(x.h, y.h, -ch);
    float tl0 = __fmul_rn(x.l, y.l);
    float tl1 = fmaf(x.h, y.l, tl0);
    float cl2 = fmaf(x.l, y.h, tl1);
    return dw_fast2sum(ch, __fadd_rn(cl1, cl2));
}
__device__ __forceinline__ dw dw_mul_f(dw x, float y) {
    float ch = __fmul_rn(x.h, y);
    float cl1 = fmaf(x.h, y, -ch);
    float cl3 = fmaf(x.l, y, cl1);
    return dw_fast2sum(ch, cl3);
}
// x / y: an FP32 quotient, then one correction from the exact residual
__device__ __forceinline__ dw dw_div(dw x, dw y) {
    float q1 = __fdividef(x.h, y.h);
    dw r = dw_sub(x, dw_mul_f(y, q1));
    float q2 = __fdividef(r.h, y.h);
    r = dw_sub(r, dw_mul_f(y, q2));
    float q3 = __fdividef(r.h, y.h);
    dw q = dw_fast2sum(q1, q2);
    return dw_add(q, dw{q3, 0.f});
}
// sqrt(x), x > 0: FP32 root, then one Newton correction from the exact square
__device__ __forceinline__ dw dw_sqrt(dw x) {
    float s = sqrtf(x.h);
    float p = __fmul_rn(s, s);
    float pe = fmaf(s, s, -p);
    float r = __fadd_rn(__fsub_rn(__fsub_rn(x.h, p), pe), x.l);
    return dw_fast2sum(s, __fdividef(r, 2.0f * s));
}
__device__ __forceinline__ dw dw_from_double(double v) {
    float h = (float)v;
    return {h, (float)(v - (double)h)};
}
__device__ __forceinline__ double dw_to_double(dw x) { return (double)x.h + (double)x.l; }
// 1/sqrt(x) for x > 0: the FP32 estimate r0, then one correction from the
// residual e = 1 - x r0^2, formed from exact products: 1/sqrt(x) =
// r0 (1 - e)^(-1/2) = r0 (1 + e/2 + 3e^2/8 + O(e^3)) (binomial series; |e| is
// about 2^-22, so the truncation is far below the double-word rounding)
__device__ __forceinline__ dw dw_rsqrt(dw x) {
    const float r0 = rsqrtf(x.h);
    const dw t = dw_mul_f(x, r0);
    const dw w = dw_mul_f(t, r0);
    const float e = __fsub_rn(__fsub_rn(1.f, w.h), w.l);
    const float c = __fmul_rn(e, fmaf(0.375f, e, 0.5f));
    return dw_fast2sum(r0, __fmul_rn(r0, c));
}
// x > y, x and y normalised
__device__ __forceinline__ bool dw_gt(dw x, dw y) { return x.h > y.h || (x.h == y.h && x.l > y.l); }

// Compensated dot-product accumulator (Ogita, Rump and Oishi's Dot2 on the
// high parts, plus the cross terms of the low parts): s + c tracks
// target - sum a_k b_k.
struct dw_acc {
    float s, c;
    __device__ __forceinline__ void init(dw t) { s = t.h; c = t.l; }
    __device__ __forceinline__ void sub_prod(dw a, dw b) {
        float ph = __fmul_rn(a.h, b.h);
        float pe = fmaf(a.h, b.h, -ph);
        float pl = fmaf(a.h, b.l, __fmul_rn(a.l, b.h));
        float ns, e;
        two_sum(s, -ph, ns, e);
        s = ns;
        c += e - pe - pl;
    }
    __device__ __forceinline__ void add_prod(dw a, dw b) {
        float ph = __fmul_rn(a.h, b.h);
        float pe = fmaf(a.h, b.h, -ph);
        float pl = fmaf(a.h, b.l, __fmul_rn(a.l, b.h));
        float ns, e;
        two_sum(s, ph, ns, e);
        s = ns;
        c += e + pe + pl;
    }
    __device__ __forceinline__ dw value() const { return dw_2sum(s, c); }
};

}  // namespace klr
