// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

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
};

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
    int degree;
    int m;        // basis size, degree <= d
    int n_mom;    // monomials of degree <= 2d (the basis is its prefix)
    uint8_t exps[kMaxMoments][kMaxVars];   // exponents, graded lex
    uint8_t pair[kMaxBasis][kMaxBasis];    // index of exps[i] + exps[j]
};

// Fill `b` for (n_vars, degree); false if out of range.
bool make_basis(int n_vars, int degree, Basis* b);
int n_monomials(int n_vars, int degree);

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Error-free sum (Knuth's TwoSum): a + b = s + e exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

// Double-FP32 accumulator (hi, lo) += t with an error-free TwoSum.
__device__ __forceinline__ void df_add(float& hi, float& lo, float t) {
    float s, e;
    two_sum(hi, t, s, e);
    hi = s;
    lo += e;
}

}  // namespace klr
