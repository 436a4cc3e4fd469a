// E2-E5: evaluation of the rational program over every configuration and the
// constrained argmin (Section IV, steps 4-5; Fig. 1 / Eq. 1; Example 2).
//
// Layout: a persistent grid walks the kernels of the program.  For its current
// kernel a block
//   1. stages the kernel's 8 x 2m coefficients in shared memory;
//   2. specialises every metric to every configuration: with the block shape
//      fixed, p(N, b) and q(N, b) become univariate polynomials in the scaled N
//      (d + 1 coefficients each), folded once per (kernel, configuration);
//   3. computes the occupancy cascade of Fig. 1 and Eq. 1 per configuration in
//      integer arithmetic (B_active, W_active);
// then each thread takes one query (data size N) and sweeps all
// configurations: Horner evaluation of the 16 univariate polynomials, the
// metric map L = lo + s |p/q|, the integer wave counts, MWP-CWP, and a running
// top-4 of (cycles, index).  FP32 argmin queries whose runner-up lies within
// the FP32 error window of the best are appended to a compact list and
// re-decided by a second kernel in FP64 from the unspecialised program.
#include <cfloat>
#include <cmath>
#include <mutex>
#include <type_traits>

#include "klr_common.cuh"

namespace klr {

namespace {

constexpr int kMaxCfg = 256;
constexpr int kTopK = 4;
// FP32 relative error window for the argmin decision (see the tie kernel).
constexpr double kTieWindow = 5e-5;

struct TieRecord {
    int64_t q;
    int32_t kernel;
    int32_t n;                  // candidates, -1: every configuration, -2: every one of
                                // the query's proposed candidates (candidate mode)
    int32_t cand[kTopK];
};

struct EvalParams {
    int n_kernels, n_vars, dims, degree, m, u, n_scale_log2, b_scale_log2;
    int coef_f64;
    const void* coef;
    const int32_t* regs;
    const int32_t* smem;
    double lo[8], sc[8];
    int n_sm, W_max, R_max, Z_max, B_max, T_max;
    double mem_ld, bw, freq, dep_c, dep_u;
    int n_cfg;
    const int32_t* cfg;
    const int64_t* q_off;
    const int64_t* q_N;
    int64_t n_q;
    int table;                  // 1: write cycles table, 0: argmin
    void* cycles;               // table output
    int32_t* best;
    void* best_cycles;
    float* margin;
    int32_t* q_status;
    int32_t* launch;
    int* tie_count;
    TieRecord* ties;
    int64_t tie_cap;
    const int32_t* cand;        // candidate mode: n_q x kc shape indices, or NULL
    int kc;
    const uint8_t* done;        // history mode: 1 for queries answered already, or NULL
    int slots;                  // warp re-rank: shapes specialised per kernel
    uint8_t exps[kMaxBasis][kMaxVars];
};

// Fig. 1 with the program's hardware limits.
__device__ __forceinline__ int active_blocks(long long T, long long R, long long Z,
                                             const EvalParams& P) {
    return occupancy_blocks(T, R, Z, P.B_max, P.W_max, P.R_max, P.Z_max, P.T_max);
}

// Products and sums of the per-shape specialisation, rounded one by one
// (never fused), so that every kernel that specialises gets the same bits.
template <typename T> __device__ __forceinline__ T mul_rn(T a, T b);
template <> __device__ __forceinline__ float mul_rn<float>(float a, float b) { return __fmul_rn(a, b); }
template <> __device__ __forceinline__ double mul_rn<double>(double a, double b) { return __dmul_rn(a, b); }
template <typename T> __device__ __forceinline__ T add_rn(T a, T b);
template <> __device__ __forceinline__ float add_rn<float>(float a, float b) { return __fadd_rn(a, b); }
template <> __device__ __forceinline__ double add_rn<double>(double a, double b) { return __dadd_rn(a, b); }

// a / b: the fast approximate quotient in FP32 (2 ulp), IEEE in FP64
template <typename T> __device__ __forceinline__ T qdiv(T a, T b) { return a / b; }
template <> __device__ __forceinline__ float qdiv<float>(float a, float b) { return __fdividef(a, b); }

// MWP-CWP (Example 2; Hong and Kim's model) in precision T.
template <typename T>
__device__ __forceinline__ T mwpcwp(const T L[8], T Nw, T Bact, T active_sms, T rep,
                                    const EvalParams& P) {
    const T comp = L[0], coal = L[1], uncoal = L[2], synch = L[3];
    const T coal_mw = L[4], uncoal_mw = L[5], load_bytes = L[6], issue = L[7];
    const T mem_ld = (T)P.mem_ld, dep_c = (T)P.dep_c, dep_u = (T)P.dep_u;
    const T one = T(1);
    const T mem_l_uncoal = mem_ld + (uncoal_mw - one) * dep_u;
    const T mem_l_coal = mem_ld + (coal_mw - one) * dep_c;
    const T mem_insts = coal + uncoal;
    const T inv_mi = qdiv<T>(T(1), mem_insts);
    const T w_u = uncoal * inv_mi;
    const T w_c = coal * inv_mi;
    const T mem_l = mem_l_uncoal * w_u + mem_l_coal * w_c;
    const T departure = dep_u * uncoal_mw * w_u + dep_c * coal_mw * w_c;
    const T mwp_nobw = qdiv<T>(mem_l, departure);
    const T bw_per_warp = qdiv<T>((T)P.freq * load_bytes, mem_l);
    const T mwp_peakbw = qdiv<T>((T)P.bw, bw_per_warp * active_sms);
    const T mwp = fmin(fmin(mwp_nobw, mwp_peakbw), Nw);
    const T comp_cycles = issue * (comp + coal + uncoal);
    const T mem_cycles = mem_l_uncoal * uncoal + mem_l_coal * coal;
    const T cwp_full = qdiv<T>(mem_cycles + comp_cycles, comp_cycles);
    const T cwp = fmin(cwp_full, Nw);
    const T per_mem = comp_cycles * inv_mi * (mwp - one);
    T e;
    if (mwp == Nw && cwp == Nw) e = (mem_cycles + comp_cycles + per_mem) * rep;
    else if (cwp >= mwp || comp_cycles > mem_cycles) e = (qdiv<T>(mem_cycles * Nw, mwp) + per_mem) * rep;
    else e = (mem_l + comp_cycles * Nw) * rep;
    return e + departure * (mwp - one) * synch * Bact * rep;
}

__device__ __forceinline__ long long ceil_div(long long a, long long b) { return (a + b - 1) / b; }

// Full (unspecialised) evaluation of one (kernel, N, configuration) in
// precision T: the same algorithm as the oracle.  FP64 re-decides FP32
// near-ties.
template <typename T>
__device__ T eval_full(const EvalParams& P, int k, long long N, int c, bool& usable) {
    const int m = P.m, u = P.u, nv = P.n_vars;
    const long long b0 = P.cfg[3 * c], b1 = P.cfg[3 * c + 1], b2 = P.cfg[3 * c + 2];
    const long long Tt = b0 * b1 * b2;
    const int B = active_blocks(Tt, P.regs[k], P.smem[k], P);
    const int W = (int)min((long long)B * Tt / 32, (long long)P.W_max);
    usable = B > 0 && Tt <= P.T_max && b0 <= N && (P.dims < 2 || b1 <= N) && (P.dims < 3 || b2 <= N);
    if (!usable) return (T)INFINITY;
    T xs[kMaxVars];
    xs[0] = (T)ldexp((double)N, -P.n_scale_log2);
    xs[1] = (T)ldexp((double)b0, -P.b_scale_log2);
    xs[2] = (T)ldexp((double)b1, -P.b_scale_log2);
    xs[3] = (T)ldexp((double)b2, -P.b_scale_log2);
    T L[8];
    for (int i = 0; i < 8; ++i) {
        T p = 0, q = 0;
        for (int t = 0; t < m; ++t) {
            T ph = 1;
            for (int v = 0; v < nv; ++v)
                for (int e = 0; e < P.exps[t][v]; ++e) ph *= xs[v];
            T a, b;
            if (P.coef_f64) {
                const double* cf = reinterpret_cast<const double*>(P.coef) + ((int64_t)k * 8 + i) * u;
                a = (T)cf[t]; b = (T)cf[m + t];
            } else {
                const float* cf = reinterpret_cast<const float*>(P.coef) + ((int64_t)k * 8 + i) * u;
                a = (T)cf[t]; b = (T)cf[m + t];
            }
            p += a * ph;
            q += b * ph;
        }
        const T g = p / q;
        if (q == T(0) || !isfinite(g)) { usable = false; return (T)INFINITY; }
        L[i] = (T)P.lo[i] + (T)P.sc[i] * fabs(g);
    }
    const long long nb = ceil_div(N, Tt);
    const long long asm_ = min((long long)P.n_sm, nb);
    const long long rep = ceil_div(nb, max((long long)B * asm_, 1LL));
    return mwpcwp<T>(L, (T)W, (T)B, (T)asm_, (T)rep, P);
}

// Section IV step 4's meaningful configurations: some block is active, the
// shape fits the thread limit and no block side exceeds N.
__device__ __noinline__ bool e_meaningful(const EvalParams& P, int k, long long N, int c) {
    const long long b0 = P.cfg[3 * c], b1 = P.cfg[3 * c + 1], b2 = P.cfg[3 * c + 2];
    const long long Tt = b0 * b1 * b2;
    return active_blocks(Tt, P.regs[k], P.smem[k], P) > 0 && Tt <= P.T_max && b0 <= N &&
           (P.dims < 2 || b1 <= N) && (P.dims < 3 || b2 <= N);
}

__device__ double eval_full_f64(const EvalParams& P, int k, long long N, int c, bool& usable) {
    return eval_full<double>(P, k, N, c, usable);
}

__device__ void write_launch(const EvalParams& P, int64_t q, long long N, int c) {
    if (!P.launch) return;
    int32_t* o = P.launch + 6 * q;
    if (c < 0) {
        for (int i = 0; i < 6; ++i) o[i] = 0;
        return;
    }
    const int b0 = P.cfg[3 * c], b1 = P.cfg[3 * c + 1], b2 = P.cfg[3 * c + 2];
    o[0] = (int32_t)ceil_div(N, b0);
    o[1] = P.dims >= 2 ? (int32_t)ceil_div(N, b1) : 1;
    o[2] = P.dims >= 3 ? (int32_t)ceil_div(N, b2) : 1;
    o[3] = b0;
    o[4] = b1;
    o[5] = b2;
}

// floor(n / d) for n < 2^24 from an FP32 reciprocal, corrected to exact
__device__ __forceinline__ unsigned udiv_small(unsigned n, unsigned d, float rd) {
    unsigned q = (unsigned)((float)n * rd);
    int r = (int)(n - q * d);
    while (r < 0) { --q; r += (int)d; }
    while (r >= (int)d) { ++q; r -= (int)d; }
    return q;
}

// The rare in-place FP64 re-decision when the tie list is full (kept out of
// line so the sweep's register allocation does not carry it).
__device__ __noinline__ void decide_f64_inplace(const EvalParams& P, int k, int64_t q,
                                                long long N, int st) {
    double bv = INFINITY, sv = INFINITY;
    int bj = -1;
    for (int c = 0; c < P.n_cfg; ++c) {
        bool us;
        double v = eval_full_f64(P, k, N, c, us);
        if (v < bv) { sv = bv; bv = v; bj = c; }
        else if (v < sv) sv = v;
    }
    P.best[q] = bj;
    reinterpret_cast<float*>(P.best_cycles)[q] = (float)bv;
    if (P.margin) P.margin[q] = isfinite(sv) ? (float)((sv - bv) / bv) : INFINITY;
    if (P.q_status) P.q_status[q] = st;
    write_launch(P, q, N, bj);
}

// Candidate mode, the rare case of a full tie list: the FP64 decision among
// the query's own candidates, in place (out of line, as above).
__device__ __noinline__ void decide_cand_f64_inplace(const EvalParams& P, int k, int64_t q,
                                                     long long N, int st) {
    double bv = INFINITY;
    int bj = -1;
    for (int j = 0; j < P.kc; ++j) {
        const int c = P.cand[q * P.kc + j];
        if (c < 0 || c >= P.n_cfg) continue;
        bool us;
        const double v = eval_full_f64(P, k, N, c, us);
        if (v < bv || (v == bv && bj >= 0 && c < bj)) { bv = v; bj = c; }
    }
    P.best[q] = bj;
    reinterpret_cast<float*>(P.best_cycles)[q] = (float)bv;
    if (P.q_status) P.q_status[q] = st | (bj < 0 ? KLR_Q_NONE_FEASIBLE : 0);
}

// Candidate mode, after the FP32 decision of one query (by lane j == 0 of
// its group): a near-tie (another candidate within the FP32 error window of
// the best) goes to the FP64 re-decision among the tied candidates (`tied`
// of them, listed in tc; more than kTopK: among all of the query's
// candidates), as in the full sweep.
__device__ __noinline__ void cand_write(const EvalParams& P, int k, int64_t q, long long N,
                                        float e, int ci, int st, int tied, int tc0, int tc1,
                                        int tc2, int tc3) {
    static_assert(kTopK == 4, "four tied candidates per record");
    const int tc[kTopK] = {tc0, tc1, tc2, tc3};
    const bool none = !(e < INFINITY);
    if (!none && tied >= 2) {
        st |= KLR_Q_TIE_RESOLVED;
        const int slot = atomicAdd(P.tie_count, 1);
        if (slot < P.tie_cap) {
            TieRecord r;
            r.q = q;
            r.kernel = k;
            r.n = tied <= kTopK ? tied : -2;
#pragma unroll
            for (int m = 0; m < kTopK; ++m) r.cand[m] = tc[m];
            P.ties[slot] = r;
        } else {
            decide_cand_f64_inplace(P, k, q, N, st);   // scratch full
            return;
        }
    }
    P.best[q] = none ? -1 : ci;
    reinterpret_cast<float*>(P.best_cycles)[q] = e;
    if (P.q_status) P.q_status[q] = st | (none ? KLR_Q_NONE_FEASIBLE : 0);
}

// Candidate mode, kc lanes per query (kc a power of two <= 32): from each
// lane's own (cycles, shape), the query's least (ties to the lower shape),
// the status bits, and the near-tied shapes; lane j == 0 writes the result.
// Every lane of the warp calls it.
__device__ __forceinline__ void cand_group_finish(const EvalParams& P, int k, int64_t q,
                                                  long long N, bool valid, int j, int kc,
                                                  float e, int c, int st) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const float e_own = e;
    const int c_own = e < INFINITY ? c : -1;
    int ci = e < INFINITY ? c : 0x7fffffff;
    for (int o = 1; o < kc; o <<= 1) {
        const float oe = __shfl_xor_sync(full, e, o);
        const int oc = __shfl_xor_sync(full, ci, o);
        st |= __shfl_xor_sync(full, st, o);
        if (oe < e || (oe == e && oc < ci)) { e = oe; ci = oc; }
    }
    // other shapes within the window of the least (a repeat of the chosen
    // shape is no tie)
    const bool near = c_own >= 0 && c_own != ci && (double)e_own <= (double)e * (1.0 + kTieWindow);
    const unsigned bal = __ballot_sync(full, near);
    if (bal == 0u) {
        // no near-tie in the warp (the common case)
        if (valid && j == 0) {
            const bool none = !(e < INFINITY);
            P.best[q] = none ? -1 : ci;
            reinterpret_cast<float*>(P.best_cycles)[q] = e;
            if (P.q_status) P.q_status[q] = st | (none ? KLR_Q_NONE_FEASIBLE : 0);
        }
        return;
    }
    const unsigned gmask = kc >= 32 ? full : (((1u << kc) - 1u) << (lane & ~(kc - 1)));
    unsigned rest = bal & gmask;
    const int others = __popc(rest);
    int tc[kTopK];
    tc[0] = ci;
#pragma unroll
    for (int m = 1; m < kTopK; ++m) {
        const int src = rest ? __ffs(rest) - 1 : lane;
        tc[m] = __shfl_sync(full, c_own, src);
        rest = rest ? (rest & (rest - 1)) : 0u;
    }
    if (valid && j == 0)
        cand_write(P, k, q, N, e, ci, st, others > 0 ? others + 1 : 1, tc[0], tc[1], tc[2], tc[3]);
}

// Per-configuration integer facts staged in shared memory.
struct CfgInfo {
    int T, B, W, b0, b1, b2;
    int t_shift;      // log2 T when T is a power of two, else -1
    unsigned wave;    // B_active * #SMs: blocks per full wave
};

// Cycles of configuration c for one query (N, its scaled xN) from the
// specialised per-kernel tables (configuration c's 8 x NC coefficients at
// spec + c * sstride); +inf when c is not meaningful or its metrics are
// invalid (then KLR_Q_BAD_METRIC is added to st).
template <typename T, int D>
__device__ __forceinline__ T eval_cfg(const EvalParams& P, const CfgInfo* __restrict__ cinfo,
                                      const float* __restrict__ wave_rcp,
                                      const T* __restrict__ spec, const T* lo, const T* sc,
                                      unsigned n_sm, long long N, bool small, T xN, int c,
                                      int& st, int sstride = 8 * 2 * (D + 1)) {
    constexpr int NC = 2 * (D + 1);
    const CfgInfo ci = cinfo[c];
    const int B = ci.B;
    const bool meaningful = B > 0 && ci.b0 <= N && ci.b1 <= N && ci.b2 <= N;
    T e = (T)INFINITY;
    if (meaningful) {
        T a[8 * NC];
        const T* sp = spec + (size_t)c * sstride;
        if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int t = 0; t < 2 * NC; ++t) {
                const float4 f4 = reinterpret_cast<const float4*>(sp)[t];
                a[4 * t] = f4.x; a[4 * t + 1] = f4.y; a[4 * t + 2] = f4.z; a[4 * t + 3] = f4.w;
            }
        } else {
#pragma unroll
            for (int t = 0; t < 4 * NC; ++t) {
                const double2 d2 = reinterpret_cast<const double2*>(sp)[t];
                a[2 * t] = d2.x; a[2 * t + 1] = d2.y;
            }
        }
        T L[8];
        bool valid = true;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const T* ai = a + i * NC;
            T p = ai[D], qq = ai[2 * D + 1];
#pragma unroll
            for (int j = D - 1; j >= 0; --j) {
                p = p * xN + ai[j];
                qq = qq * xN + ai[D + 1 + j];
            }
            const T g = qdiv<T>(p, qq);
            valid = valid && (qq != T(0)) && isfinite(g);
            L[i] = lo[i] + sc[i] * fabs(g);
        }
        if (valid) {
            long long nb, asm_, rep;
            if (small) {
                const unsigned n32 = (unsigned)N, t32 = (unsigned)ci.T;
                const unsigned nb32 = ci.t_shift >= 0 ? (n32 + t32 - 1) >> ci.t_shift
                                                      : (n32 + t32 - 1) / t32;
                nb = nb32;
                if (nb32 <= n_sm) {
                    asm_ = nb32;
                    rep = 1;   // ceil(nb / (B nb)) with B >= 1
                } else {
                    asm_ = n_sm;
                    rep = udiv_small(nb32 + ci.wave - 1, ci.wave, wave_rcp[c]);
                }
            } else {
                nb = ceil_div(N, (long long)ci.T);
                asm_ = min((long long)n_sm, nb);
                rep = ceil_div(nb, (long long)B * asm_);
            }
            e = mwpcwp<T>(L, (T)ci.W, (T)B, (T)asm_, (T)rep, P);
            if (!isfinite(e)) { e = (T)INFINITY; st |= KLR_Q_BAD_METRIC; }
        } else {
            st |= KLR_Q_BAD_METRIC;
        }
    }
    return e;
}

// Per-kernel tables of the sweep, by the threads of one block: the kernel's
// coefficients, the per-shape integer facts (occupancy, warps, wave size)
// and the specialised polynomials in N of every shape (of the proposed ones
// in candidate mode).  Ends with the block synchronised.
template <typename T, int D, bool kMonoTable = (sizeof(T) == 4)>
__device__ __forceinline__ void eval_setup(const EvalParams& P, int k, T* coef_s, T* spec,
                                           const T* bmon, CfgInfo* cinfo, float* wave_rcp,
                                           unsigned* cmask, unsigned n_sm) {
    constexpr int NC = 2 * (D + 1);
    const int m = P.m, u = P.u, n_cfg = P.n_cfg;
    const int64_t qa = P.q_off[k], qb = P.q_off[k + 1];
    __syncthreads();   // previous kernel's tables no longer in use
    for (int i = threadIdx.x; i < 8 * u; i += blockDim.x) {
        if (P.coef_f64) coef_s[i] = (T)reinterpret_cast<const double*>(P.coef)[(int64_t)k * 8 * u + i];
        else coef_s[i] = (T)reinterpret_cast<const float*>(P.coef)[(int64_t)k * 8 * u + i];
    }
    // candidate mode: the shapes proposed for any of this kernel's queries
    if (P.cand) {
        for (int i = threadIdx.x; i < 8; i += blockDim.x) cmask[i] = 0u;
        __syncthreads();
        for (int64_t i = qa * P.kc + threadIdx.x; i < qb * P.kc; i += blockDim.x) {
            const int c = P.cand[i];
            if (c >= 0 && c < n_cfg) atomicOr(&cmask[c >> 5], 1u << (c & 31));
        }
    }
    const int R = P.regs[k], Z = P.smem[k];
    for (int c = threadIdx.x; c < n_cfg; c += blockDim.x) {
        const long long b0 = P.cfg[3 * c], b1 = P.cfg[3 * c + 1], b2 = P.cfg[3 * c + 2];
        const long long Tt = b0 * b1 * b2;
        int B = active_blocks(Tt, R, Z, P);
        if (Tt > P.T_max) B = 0;
        const int W = (int)min((long long)B * Tt / 32, (long long)P.W_max);
        CfgInfo ci;
        ci.T = (int)Tt;
        ci.B = B;
        ci.W = W;
        ci.b0 = (int)b0;
        ci.b1 = P.dims >= 2 ? (int)b1 : 1;
        ci.b2 = P.dims >= 3 ? (int)b2 : 1;
        ci.t_shift = (Tt > 0 && (Tt & (Tt - 1)) == 0) ? __ffsll(Tt) - 1 : -1;
        ci.wave = (unsigned)max(B, 1) * n_sm;
        cinfo[c] = ci;
        wave_rcp[c] = 1.0f / (float)ci.wave;
    }
    __syncthreads();
    // fold the block shape into univariate polynomials in the scaled N
    for (int idx = threadIdx.x; idx < n_cfg * 8; idx += blockDim.x) {
        const int c = idx >> 3, i = idx & 7;
        if (P.cand && !((cmask[c >> 5] >> (c & 31)) & 1u)) continue;
        T xb[3];
        xb[0] = (T)ldexp((double)P.cfg[3 * c], -P.b_scale_log2);
        xb[1] = (T)ldexp((double)P.cfg[3 * c + 1], -P.b_scale_log2);
        xb[2] = (T)ldexp((double)P.cfg[3 * c + 2], -P.b_scale_log2);
        // coefficient of N^j: its terms in increasing index order
        T acc[2][D + 1];
#pragma unroll
        for (int s2 = 0; s2 < 2; ++s2)
#pragma unroll
            for (int j = 0; j <= D; ++j) acc[s2][j] = T(0);
        for (int t = 0; t < m; ++t) {
            T bm = T(1);
            if (kMonoTable) {
                bm = bmon[c * m + t];
            } else {
                for (int v = 1; v < P.n_vars; ++v)
                    for (int e = 0; e < P.exps[t][v]; ++e) bm *= xb[v - 1];
            }
            const int j = P.exps[t][0];
            const T pa = mul_rn(coef_s[i * u + t], bm), qa = mul_rn(coef_s[i * u + m + t], bm);
#pragma unroll
            for (int jj = 0; jj <= D; ++jj)
                if (jj == j) { acc[0][jj] = add_rn(acc[0][jj], pa); acc[1][jj] = add_rn(acc[1][jj], qa); }
        }
        T* sp = spec + (size_t)idx * NC;
#pragma unroll
        for (int j = 0; j <= D; ++j) {
            sp[j] = acc[0][j];
            sp[D + 1 + j] = acc[1][j];
        }
    }
    __syncthreads();
}

template <typename T, int D>
__global__ void __launch_bounds__(256)
eval_kernel(const __grid_constant__ EvalParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned cmask[8];             // candidate mode: shapes in use (n_cfg <= 256)
    constexpr int NC = 2 * (D + 1);           // coefficients per (config, metric)
    const int m = P.m, u = P.u, n_cfg = P.n_cfg;
    constexpr bool kMonoTable = sizeof(T) == 4;   // FP32: block-shape monomials in a table
    T* coef_s = reinterpret_cast<T*>(smem_raw);                 // 8 x u
    T* spec = coef_s + 8 * u;                                   // n_cfg x 8 x NC
    T* bmon = spec + (size_t)n_cfg * 8 * NC;                    // n_cfg x m (FP32 only)
    CfgInfo* cinfo = reinterpret_cast<CfgInfo*>(bmon + (kMonoTable ? (size_t)n_cfg * m : 0));
    float* wave_rcp = reinterpret_cast<float*>(cinfo + n_cfg);
    const T n_scale = (T)ldexp(1.0, -P.n_scale_log2);
    T lo[8], sc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) { lo[i] = (T)P.lo[i]; sc[i] = (T)P.sc[i]; }
    const unsigned n_sm = (unsigned)P.n_sm;
    // the block-shape part of every monomial, once per block (the same
    // products, in the same order, as the per-entry loop below)
    if (kMonoTable) {
        for (int idx = threadIdx.x; idx < n_cfg * m; idx += blockDim.x) {
            const int c = idx / m, t = idx - c * m;
            T xb[3];
            xb[0] = (T)ldexp((double)P.cfg[3 * c], -P.b_scale_log2);
            xb[1] = (T)ldexp((double)P.cfg[3 * c + 1], -P.b_scale_log2);
            xb[2] = (T)ldexp((double)P.cfg[3 * c + 2], -P.b_scale_log2);
            T bm = T(1);
            for (int v = 1; v < P.n_vars; ++v)
                for (int e = 0; e < P.exps[t][v]; ++e) bm *= xb[v - 1];
            bmon[idx] = bm;
        }
    }

    for (int k = blockIdx.x; k < P.n_kernels; k += gridDim.x) {
        const int64_t qa = P.q_off[k], qb = P.q_off[k + 1];
        if (qa == qb) continue;
        if (P.done) {
            // history mode: nothing to do for a kernel whose queries all hit
            int open = 0;
            for (int64_t q = qa + threadIdx.x; q < qb; q += blockDim.x) open |= !P.done[q];
            if (!__syncthreads_or(open)) continue;
        }
        eval_setup<T, D>(P, k, coef_s, spec, bmon, cinfo, wave_rcp, cmask, n_sm);

        if (P.cand && P.kc <= 32 && (P.kc & (P.kc - 1)) == 0) {
            // candidate mode: one (query, candidate) pair per lane, kc lanes
            // per query, reduced by shuffles to the least (cycles, index)
            const int kc = P.kc;
            const int64_t npairs = (qb - qa) * kc;
            const int64_t span = (npairs + 31) & ~(int64_t)31;   // whole warps
            for (int64_t pi = threadIdx.x; pi < span; pi += blockDim.x) {
                const bool valid = pi < npairs;
                const int64_t q = qa + (valid ? pi / kc : 0);
                const int j = (int)(pi & (kc - 1));
                const int c = valid ? P.cand[q * kc + j] : -1;
                int st = 0;
                T e = (T)INFINITY;
                if (c >= 0 && c < n_cfg) {
                    const long long N = P.q_N[q];
                    e = eval_cfg<T, D>(P, cinfo, wave_rcp, spec, lo, sc, n_sm, N, N < (1LL << 24),
                                       (T)N * n_scale, c, st);
                }
                cand_group_finish(P, k, q, P.q_N[q], valid, j, kc, (float)e, c, st);
            }
            continue;
        }
        if (P.cand) {
            // candidate mode, one thread per query (kc not a power of two or
            // above 32): a sorted top-k by (value, shape) over the candidates,
            // which come in any order, a repeated shape entered once
            for (int64_t q = qa + threadIdx.x; q < qb; q += blockDim.x) {
                const long long N = P.q_N[q];
                const bool small = N < (1LL << 24);
                const T xN = (T)N * n_scale;
                T topv[kTopK];
                int topi[kTopK];
#pragma unroll
                for (int j = 0; j < kTopK; ++j) { topv[j] = (T)INFINITY; topi[j] = -1; }
                int st = 0;
#pragma unroll 1
                for (int it = 0; it < P.kc; ++it) {
                    const int c = P.cand[q * P.kc + it];
                    if (c < 0 || c >= n_cfg) continue;
                    T e = eval_cfg<T, D>(P, cinfo, wave_rcp, spec, lo, sc, n_sm, N, small, xN, c, st);
                    if (!(e < (T)INFINITY)) continue;
                    bool seen = false;
#pragma unroll
                    for (int j = 0; j < kTopK; ++j) seen = seen || topi[j] == c;
                    if (seen) continue;
                    T ve = e;
                    int vi = c;
#pragma unroll
                    for (int j = 0; j < kTopK; ++j) {
                        if (topi[j] < 0 || ve < topv[j] || (ve == topv[j] && vi < topi[j])) {
                            T tv = topv[j]; int ti = topi[j];
                            topv[j] = ve; topi[j] = vi;
                            ve = tv; vi = ti;
                            if (vi < 0) break;
                        }
                    }
                }
                // near-ties of the best go to the FP64 re-decision (all of the
                // query's candidates when every kept entry is tied)
                int tied = 0, tc[kTopK];
#pragma unroll
                for (int j = 0; j < kTopK; ++j) {
                    tc[j] = topi[j];
                    if (topi[j] >= 0 && (double)topv[j] <= (double)topv[0] * (1.0 + kTieWindow)) ++tied;
                }
                if (tied == kTopK) tied = kTopK + 1;
                cand_write(P, k, q, N, (float)topv[0], topi[0], st, tied, tc[0], tc[1], tc[2], tc[3]);
            }
            continue;
        }
        for (int64_t q = qa + threadIdx.x; q < qb; q += blockDim.x) {
            if (P.done && P.done[q]) continue;
            const long long N = P.q_N[q];
            const bool small = N < (1LL << 24);   // 32-bit wave counts exact
            const T xN = (T)N * n_scale;
            T topv[kTopK];
            int topi[kTopK];
#pragma unroll
            for (int j = 0; j < kTopK; ++j) { topv[j] = (T)INFINITY; topi[j] = -1; }
            int st = 0;
#pragma unroll 1
            for (int c = 0; c < n_cfg; ++c) {
                T e = eval_cfg<T, D>(P, cinfo, wave_rcp, spec, lo, sc, n_sm, N, small, xN, c, st);
                if (P.table) {
                    reinterpret_cast<T*>(P.cycles)[q * n_cfg + c] = e;
                } else if (e < topv[kTopK - 1]) {
                    // insert into the sorted top-k; ties keep the lower index first
                    T ve = e;
                    int vi = c;
#pragma unroll
                    for (int j = 0; j < kTopK; ++j) {
                        if (ve < topv[j]) {
                            T tv = topv[j]; int ti = topi[j];
                            topv[j] = ve; topi[j] = vi;
                            ve = tv; vi = ti;
                        }
                    }
                }
            }
            if (P.table) continue;
            const int bi = topi[0];
            if (bi < 0) st |= KLR_Q_NONE_FEASIBLE;
            float mg = 0.f;
            if (bi >= 0) mg = isfinite((float)topv[1]) ? (float)((topv[1] - topv[0]) / topv[0]) : INFINITY;
            if (std::is_same<T, float>::value && bi >= 0 && isfinite(topv[1]) &&
                (double)topv[1] <= (double)topv[0] * (1.0 + kTieWindow)) {
                // near-tie in FP32: hand the candidates to the FP64 re-decision
                st |= KLR_Q_TIE_RESOLVED;
                const int slot = atomicAdd(P.tie_count, 1);
                if (slot < P.tie_cap) {
                    TieRecord r;
                    r.q = q;
                    r.kernel = k;
                    int n = 0;
                    for (int j = 0; j < kTopK; ++j)
                        if (topi[j] >= 0 && (double)topv[j] <= (double)topv[0] * (1.0 + kTieWindow))
                            r.cand[n++] = topi[j];
                    r.n = (n == kTopK) ? -1 : n;   // all top-k tied: re-sweep everything
                    P.ties[slot] = r;
                } else {
                    decide_f64_inplace(P, k, q, N, st);   // scratch full
                    continue;
                }
            }
            P.best[q] = bi;
            reinterpret_cast<T*>(P.best_cycles)[q] = topv[0];
            if (P.margin) P.margin[q] = mg;
            if (P.q_status) P.q_status[q] = st;
            write_launch(P, q, N, bi);
        }
    }
}

// ---------------------------------------------------------------------------
// Latency mode of the FP64 argmin (a few queries, e.g. one kernel's sizes at
// launch time): one block per query, so that the queries spread over the SMs
// instead of sharing one block per kernel.  The block builds its query's
// kernel tables as the per-kernel sweep does (eval_setup, with the
// block-shape monomials first put in a table: the same products in the same
// order), each thread evaluates its shapes with the sweep's eval_cfg, and
// shuffles then shared memory reduce the query to its least (cycles, shape),
// lowest shape on ties, and the runner-up: the outputs are bitwise those of
// the per-kernel sweep.  FP64 issues at 1/64 of the FP32 rate on GB300, so
// the block's 8 warps are there to occupy every scheduler's FP64 unit.
// ---------------------------------------------------------------------------
constexpr int64_t kLatencyMaxQueries = 1024;
constexpr int kLatencyThreads = 256;

size_t latency_smem_bytes(const EvalParams& P) {
    const int NC = 2 * (P.degree + 1);
    size_t b = sizeof(double) * (8 * (size_t)P.u + (size_t)P.n_cfg * 8 * NC + (size_t)P.n_cfg * P.m);
    b = (b + 15) & ~(size_t)15;
    return b + (sizeof(CfgInfo) + sizeof(float)) * (size_t)P.n_cfg;
}

template <int D>
__global__ void __launch_bounds__(kLatencyThreads)
eval_query_block_kernel(const __grid_constant__ EvalParams P) {
    using T = double;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned cmask[8];
    __shared__ T red_v[kLatencyThreads / 32], red_r[kLatencyThreads / 32];
    __shared__ int red_j[kLatencyThreads / 32], red_s[kLatencyThreads / 32];
    constexpr int NC = 2 * (D + 1);
    const int n_cfg = P.n_cfg, m = P.m;
    T* coef_s = reinterpret_cast<T*>(smem_raw);                 // 8 x u
    T* spec = coef_s + 8 * P.u;                                 // n_cfg x 8 x NC
    T* bmon = spec + (size_t)n_cfg * 8 * NC;                    // n_cfg x m
    CfgInfo* cinfo = reinterpret_cast<CfgInfo*>(bmon + (size_t)n_cfg * m);
    float* wave_rcp = reinterpret_cast<float*>(cinfo + n_cfg);
    const int64_t q = blockIdx.x;
    if (q >= P.n_q) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned full = 0xffffffffu;
    // the query's kernel: the last k with q_off[k] <= q
    int kl = 0, kh = P.n_kernels - 1;
    while (kl < kh) {
        const int mid = (kl + kh + 1) >> 1;
        if (P.q_off[mid] <= q) kl = mid;
        else kh = mid - 1;
    }
    const int k = kl;
    const unsigned n_sm = (unsigned)P.n_sm;
    for (int idx = threadIdx.x; idx < n_cfg * m; idx += blockDim.x) {
        const int c = idx / m, t = idx - c * m;
        T xb[3];
        xb[0] = (T)ldexp((double)P.cfg[3 * c], -P.b_scale_log2);
        xb[1] = (T)ldexp((double)P.cfg[3 * c + 1], -P.b_scale_log2);
        xb[2] = (T)ldexp((double)P.cfg[3 * c + 2], -P.b_scale_log2);
        T bm = T(1);
        for (int v = 1; v < P.n_vars; ++v)
            for (int e = 0; e < P.exps[t][v]; ++e) bm *= xb[v - 1];
        bmon[idx] = bm;
    }
    eval_setup<T, D, true>(P, k, coef_s, spec, bmon, cinfo, wave_rcp, cmask, n_sm);
    T lo[8], sc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) { lo[i] = (T)P.lo[i]; sc[i] = (T)P.sc[i]; }
    const long long N = P.q_N[q];
    const bool small = N < (1LL << 24);
    const T xN = (T)N * (T)ldexp(1.0, -P.n_scale_log2);
    int st = 0;
    T bv = (T)INFINITY, sv = (T)INFINITY;
    int bj = 0x7fffffff;
    for (int c = threadIdx.x; c < n_cfg; c += blockDim.x) {
        const T e = eval_cfg<T, D>(P, cinfo, wave_rcp, spec, lo, sc, n_sm, N, small, xN, c, st);
        if (e < bv) { sv = bv; bv = e; bj = c; }
        else if (e < sv) sv = e;
    }
    // least (value, index) of the warp, then its runner-up value
    T gv = bv;
    int gj = bj;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(full, gv, o);
        const int oj = __shfl_xor_sync(full, gj, o);
        if (ov < gv || (ov == gv && oj < gj)) { gv = ov; gj = oj; }
    }
    T rv = (bj == gj) ? sv : fmin(bv, sv);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rv = fmin(rv, __shfl_xor_sync(full, rv, o));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) st |= __shfl_xor_sync(full, st, o);
    if (lane == 0) { red_v[wid] = gv; red_j[wid] = gj; red_r[wid] = rv; red_s[wid] = st; }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        int w0 = 0;
        for (int w = 1; w < nw; ++w)
            if (red_v[w] < red_v[w0] || (red_v[w] == red_v[w0] && red_j[w] < red_j[w0])) w0 = w;
        gv = red_v[w0];
        gj = red_j[w0];
        rv = red_r[w0];
        st = 0;
        for (int w = 0; w < nw; ++w) {
            st |= red_s[w];
            if (w != w0) rv = fmin(rv, red_v[w]);   // another warp's least: at most its runner-up
        }
        const int best = gv < (T)INFINITY ? gj : -1;
        if (best < 0) st |= KLR_Q_NONE_FEASIBLE;
        float mg = 0.f;
        if (best >= 0) mg = isfinite((float)rv) ? (float)((rv - gv) / gv) : INFINITY;
        P.best[q] = best;
        reinterpret_cast<T*>(P.best_cycles)[q] = gv;
        if (P.margin) P.margin[q] = mg;
        if (P.q_status) P.q_status[q] = st;
        write_launch(P, q, N, best);
    }
}

// ---------------------------------------------------------------------------
// Candidate re-rank with one warp per kernel: the kernel's coefficients, the
// union of the shapes proposed for its queries (at most P.slots specialised
// per kernel; others are evaluated unspecialised) and their specialised
// polynomials live in the warp's own shared memory, so warps never wait on
// one another; lanes then take (query, candidate) pairs, kc lanes per query.
// ---------------------------------------------------------------------------
constexpr int kRerankWarps = 4;

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

// bytes of one warp's region
// specialised coefficients of one slot, padded by 16 bytes: lanes that read
// different slots at once then fall in different banks
__host__ __device__ inline int rerank_slot_stride(int nc) { return 8 * nc + 4; }
__host__ __device__ inline size_t rerank_warp_bytes(int u, int n_cfg, int nc, int slots) {
    const size_t ns = (size_t)slots;
    return align16(4 * (size_t)8 * u) + align16(4 * ns * rerank_slot_stride(nc)) +
           align16(sizeof(CfgInfo) * ns) +
           align16(4 * ns) + align16(4 * ns) + align16(2 * (size_t)n_cfg) + 32;
}

template <int D>
__global__ void __launch_bounds__(32 * kRerankWarps)
rerank_kernel(const __grid_constant__ EvalParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int NC = 2 * (D + 1);
    const int m = P.m, u = P.u, n_cfg = P.n_cfg, kc = P.kc, n_slot = P.slots;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned full = 0xffffffffu;
    float* bmon = reinterpret_cast<float*>(smem_raw);                 // n_cfg x m
    unsigned char* wb = smem_raw + align16(4 * (size_t)n_cfg * m) +
                        (size_t)w * rerank_warp_bytes(u, n_cfg, NC, n_slot);
    float* coef_s = reinterpret_cast<float*>(wb);
    wb += align16(4 * (size_t)8 * u);
    float* spec = reinterpret_cast<float*>(wb);
    constexpr int SS = 8 * NC + 4;                                     // rerank_slot_stride
    wb += align16(4 * (size_t)n_slot * SS);
    CfgInfo* cinfo = reinterpret_cast<CfgInfo*>(wb);
    wb += align16(sizeof(CfgInfo) * (size_t)n_slot);
    float* wrcp = reinterpret_cast<float*>(wb);
    wb += align16(4 * (size_t)n_slot);
    int* slot_cfg = reinterpret_cast<int*>(wb);
    wb += align16(4 * (size_t)n_slot);
    int16_t* slot_of = reinterpret_cast<int16_t*>(wb);
    wb += align16(2 * (size_t)n_cfg);
    unsigned* mask = reinterpret_cast<unsigned*>(wb);                 // 8 words
    const float n_scale = (float)ldexp(1.0, -P.n_scale_log2);
    float lo[8], sc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) { lo[i] = (float)P.lo[i]; sc[i] = (float)P.sc[i]; }
    const unsigned n_sm = (unsigned)P.n_sm;
    for (int idx = threadIdx.x; idx < n_cfg * m; idx += blockDim.x) {
        const int c = idx / m, t = idx - c * m;
        float xb[3];
        xb[0] = (float)ldexp((double)P.cfg[3 * c], -P.b_scale_log2);
        xb[1] = (float)ldexp((double)P.cfg[3 * c + 1], -P.b_scale_log2);
        xb[2] = (float)ldexp((double)P.cfg[3 * c + 2], -P.b_scale_log2);
        float bm = 1.f;
        for (int v = 1; v < P.n_vars; ++v)
            for (int e = 0; e < P.exps[t][v]; ++e) bm *= xb[v - 1];
        bmon[idx] = bm;
    }
    __syncthreads();
    for (int64_t k = (int64_t)blockIdx.x * kRerankWarps + w; k < P.n_kernels;
         k += (int64_t)gridDim.x * kRerankWarps) {
        const int64_t qa = P.q_off[k], qb = P.q_off[k + 1];
        if (qa == qb) continue;
        for (int i = lane; i < 8 * u; i += 32) {
            coef_s[i] = P.coef_f64 ? (float)reinterpret_cast<const double*>(P.coef)[k * 8 * u + i]
                                   : reinterpret_cast<const float*>(P.coef)[k * 8 * u + i];
        }
        if (lane < 8) mask[lane] = 0u;
        __syncwarp();
        for (int64_t i = qa * kc + lane; i < qb * kc; i += 32) {
            const int c = P.cand[i];
            if (c >= 0 && c < n_cfg) atomicOr(&mask[c >> 5], 1u << (c & 31));
        }
        __syncwarp();
        // slots for the proposed shapes, in shape order
        int n_slots = 0;
        for (int c0 = 0; c0 < n_cfg; c0 += 32) {
            const int c = c0 + lane;
            const bool bit = c < n_cfg && ((mask[c >> 5] >> (c & 31)) & 1u);
            const unsigned bal = __ballot_sync(full, bit);
            const int pos = n_slots + __popc(bal & ((1u << lane) - 1u));
            if (c < n_cfg) slot_of[c] = (int16_t)((bit && pos < n_slot) ? pos : -1);
            if (bit && pos < n_slot) slot_cfg[pos] = c;
            n_slots += __popc(bal);
        }
        const int n_used = min(n_slots, n_slot);
        __syncwarp();
        const int R = P.regs[k], Z = P.smem[k];
        for (int s = lane; s < n_used; s += 32) {
            const int c = slot_cfg[s];
            const long long b0 = P.cfg[3 * c], b1 = P.cfg[3 * c + 1], b2 = P.cfg[3 * c + 2];
            const long long Tt = b0 * b1 * b2;
            int B = active_blocks(Tt, R, Z, P);
            if (Tt > P.T_max) B = 0;
            CfgInfo ci;
            ci.T = (int)Tt;
            ci.B = B;
            ci.W = (int)min((long long)B * Tt / 32, (long long)P.W_max);
            ci.b0 = (int)b0;
            ci.b1 = P.dims >= 2 ? (int)b1 : 1;
            ci.b2 = P.dims >= 3 ? (int)b2 : 1;
            ci.t_shift = (Tt > 0 && (Tt & (Tt - 1)) == 0) ? __ffsll(Tt) - 1 : -1;
            ci.wave = (unsigned)max(B, 1) * n_sm;
            cinfo[s] = ci;
            wrcp[s] = 1.0f / (float)ci.wave;
        }
        // two (shape, metric) items per lane at a time: the same products
        // and sums, in the same order, as the sweep's specialisation
        for (int idx = lane; idx < n_used * 8; idx += 64) {
            const int idx2 = idx + 32 < n_used * 8 ? idx + 32 : idx;   // a repeat is harmless
            const int c1 = slot_cfg[idx >> 3], i1 = idx & 7;
            const int c2 = slot_cfg[idx2 >> 3], i2 = idx2 & 7;
            float acc1[2][D + 1], acc2[2][D + 1];
#pragma unroll
            for (int s2 = 0; s2 < 2; ++s2)
#pragma unroll
                for (int j = 0; j <= D; ++j) { acc1[s2][j] = 0.f; acc2[s2][j] = 0.f; }
            for (int t = 0; t < m; ++t) {
                const float bm1 = bmon[c1 * m + t], bm2 = bmon[c2 * m + t];
                const int j = P.exps[t][0];
                const float pa1 = mul_rn(coef_s[i1 * u + t], bm1), qa1 = mul_rn(coef_s[i1 * u + m + t], bm1);
                const float pa2 = mul_rn(coef_s[i2 * u + t], bm2), qa2 = mul_rn(coef_s[i2 * u + m + t], bm2);
#pragma unroll
                for (int jj = 0; jj <= D; ++jj)
                    if (jj == j) {
                        acc1[0][jj] = add_rn(acc1[0][jj], pa1);
                        acc1[1][jj] = add_rn(acc1[1][jj], qa1);
                        acc2[0][jj] = add_rn(acc2[0][jj], pa2);
                        acc2[1][jj] = add_rn(acc2[1][jj], qa2);
                    }
            }
            float* sp1 = spec + (size_t)(idx >> 3) * SS + (idx & 7) * NC;
            float* sp2 = spec + (size_t)(idx2 >> 3) * SS + (idx2 & 7) * NC;
#pragma unroll
            for (int j = 0; j <= D; ++j) {
                sp1[j] = acc1[0][j];
                sp1[D + 1 + j] = acc1[1][j];
                sp2[j] = acc2[0][j];
                sp2[D + 1 + j] = acc2[1][j];
            }
        }
        __syncwarp();
        const int64_t npairs = (qb - qa) * kc;
        const int64_t span = (npairs + 31) & ~(int64_t)31;
        // cycles of pair pi (query pi / kc, its candidate pi mod kc)
        auto pair_eval = [&](int64_t pi, float& e, int& st, int& c, int64_t& q, bool& valid,
                             long long& N) {
            valid = pi < npairs;
            q = qa + (valid ? pi / kc : 0);
            c = valid ? P.cand[q * kc + (int)(pi & (kc - 1))] : -1;
            st = 0;
            e = INFINITY;
            N = P.q_N[q];
            if (c >= 0 && c < n_cfg) {
                const int s = slot_of[c];
                if (s >= 0) {
                    e = eval_cfg<float, D>(P, cinfo, wrcp, spec, lo, sc, n_sm, N, N < (1LL << 24),
                                           (float)N * n_scale, s, st, SS);
                } else {
                    // beyond the specialised slots: the unspecialised form
                    bool us;
                    e = eval_full<float>(P, (int)k, N, c, us);
                    if (!us) {
                        // meaningful but with an invalid metric: flagged
                        if (e_meaningful(P, (int)k, N, c)) st |= KLR_Q_BAD_METRIC;
                        e = INFINITY;
                    } else if (!isfinite(e)) {
                        e = INFINITY;
                        st |= KLR_Q_BAD_METRIC;
                    }
                }
            }
        };
        // every lane runs the same number of iterations
        for (int64_t pi = lane; pi < span; pi += 32) {
            float e1;
            int s1, c1;
            int64_t q1;
            bool v1;
            long long N1;
            pair_eval(pi, e1, s1, c1, q1, v1, N1);
            cand_group_finish(P, (int)k, q1, N1, v1, (int)(pi & (kc - 1)), kc, e1, c1, s1);
        }
        __syncwarp();
    }
}


// Re-decide FP32 near-ties: FP64 evaluation of the tied candidates (or of
// every configuration) with the unspecialised program, lowest index on ties.
// One group of G lanes per tie record, lanes over its configurations: one
// pass takes the records that list their tied configurations (G = kTopK, or
// the candidate count rounded up to a power of two in candidate mode), the
// other those that re-sweep every configuration (G = 32), so that the scarce
// FP64 issue slots run with every lane busy.  The least (value, index) and
// the runner-up value (the least over every other configuration) by shuffles
// within the group.
constexpr int kTieWarps = 4;
__global__ void __launch_bounds__(32 * kTieWarps)
tie_kernel(const __grid_constant__ EvalParams P, int G, int full_sweeps) {
    const int64_t n = min((int64_t)*P.tie_count, P.tie_cap);
    const int lane = threadIdx.x & 31, gl = lane & (G - 1);
    const unsigned full = 0xffffffffu;
    const int per_warp = 32 / G;
    const int64_t groups = ((int64_t)gridDim.x * kTieWarps) * per_warp;
    const int64_t first = ((int64_t)blockIdx.x * kTieWarps + (threadIdx.x >> 5)) * per_warp + lane / G;
    // every lane of a warp runs the same number of iterations
    const int64_t rounds = (n + groups - 1) / groups;
    for (int64_t it = 0; it < rounds; ++it) {
        const int64_t r = first + it * groups;
        TieRecord rec;
        rec.n = 0;
        if (r < n) rec = P.ties[r];
        const bool live = r < n && ((rec.n == -1) == (full_sweeps != 0));
        const long long N = live ? P.q_N[rec.q] : 1;
        const int cnt = !live ? 0 : rec.n == -2 ? P.kc : rec.n < 0 ? P.n_cfg : rec.n;
        double bv = INFINITY, sv = INFINITY;     // this lane's least and runner-up
        int bj = 0x7fffffff;
        for (int j = gl; j < cnt; j += G) {
            const int c = rec.n == -2 ? P.cand[rec.q * P.kc + j] : rec.n < 0 ? j : rec.cand[j];
            if (c < 0 || c >= P.n_cfg) continue;
            bool us;
            const double v = eval_full_f64(P, rec.kernel, N, c, us);
            if (v < bv || (v == bv && c < bj)) { sv = bv; bv = v; bj = c; }
            else if (v < sv) sv = v;
        }
        // the least (value, index) over the group
        double gv = bv;
        int gj = bj;
        for (int o = G >> 1; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(full, gv, o);
            const int oj = __shfl_xor_sync(full, gj, o);
            if (ov < gv || (ov == gv && oj < gj)) { gv = ov; gj = oj; }
        }
        // runner-up: every lane's least except the chosen one, and its own
        // runner-up
        double rv = (bj == gj) ? sv : fmin(bv, sv);
        for (int o = G >> 1; o > 0; o >>= 1) rv = fmin(rv, __shfl_xor_sync(full, rv, o));
        if (live && gl == 0) {
            const int best = (gv < INFINITY) ? gj : -1;
            P.best[rec.q] = best;
            reinterpret_cast<float*>(P.best_cycles)[rec.q] = (float)gv;
            if (P.margin) P.margin[rec.q] = isfinite(rv) ? (float)((rv - gv) / gv) : INFINITY;
            write_launch(P, rec.q, N, best);
        }
    }
}

// lanes per listed tie record: kTopK for the sweep; in candidate mode the
// candidates per query rounded up to a power of two (at least kTopK)
inline int tie_group(const EvalParams& P) {
    if (!P.cand) return kTopK;
    int g = kTopK;
    while (g < P.kc && g < 32) g <<= 1;
    return g;
}

// the FP64 re-decision of the tie records (grids sized by the tie capacity;
// the groups past the recorded count do nothing): listed records, then (the
// sweep only) the full re-sweeps
klr_status launch_ties(const Context* c, const EvalParams& P, cudaStream_t stream) {
    for (int pass = 0; pass < (P.cand ? 1 : 2); ++pass) {
        const int G = pass == 0 ? tie_group(P) : 32;
        const int64_t per_block = (int64_t)kTieWarps * (32 / G);
        const int grid = (int)std::min<int64_t>((P.tie_cap + per_block - 1) / per_block,
                                                (int64_t)c->n_sm * 8);
        tie_kernel<<<grid, 32 * kTieWarps, 0, stream>>>(P, G, pass);
        KLR_CHECK_CUDA(cudaGetLastError());
    }
    return KLR_OK;
}

int64_t tie_capacity(int64_t n_q) {
    return std::max<int64_t>(65536, std::min<int64_t>(n_q, 1 << 22) / 4);
}

// Scratch of klr_argmin_noalloc: a tie counter (first 256 bytes) and
// KLR_ARGMIN_NOALLOC_TIE_RECORDS tie records.  Every GPU that loads the
// library holds it until the process exits.
constexpr size_t kNoallocHeader = 256;
constexpr size_t kNoallocBytes = kNoallocHeader + sizeof(TieRecord) * KLR_ARGMIN_NOALLOC_TIE_RECORDS;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// Device address of g_noalloc_scratch, looked up once per device (the host
// symbol is only a stand-in and must never be passed to a kernel).
constexpr int kMaxDevices = 256;
static std::mutex g_noalloc_mutex;
static void* g_noalloc_addr[kMaxDevices] = {};

klr_status noalloc_scratch(int device, void** out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (device < 0 || device >= kMaxDevices) {
        set_error("klr_argmin_noalloc: device %d out of range", device);
        return KLR_EINVAL;
    }
    if (!g_noalloc_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            set_error("klr_argmin_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return KLR_ECUDA;
        }
        g_noalloc_addr[device] = p;
    }
    *out = g_noalloc_addr[device];
    return KLR_OK;
}

klr_status prepare(Context* c, const klr_program* prog, const klr_hw* hw, const int32_t* cfg,
                   int n_cfg, const klr_queries* q, int out_dtype, EvalParams& P) {
    KLR_REQUIRE(prog && hw && q, "klr_eval/argmin: NULL program, hw or queries");
    KLR_REQUIRE(prog->n_kernels >= 0, "n_kernels < 0");
    KLR_REQUIRE(prog->n_vars == 3 || prog->n_vars == 4, "n_vars %d not 3 or 4", prog->n_vars);
    const bool box = prog->var_degree[0] > 0;
    KLR_REQUIRE(box || (prog->degree >= 1 && prog->degree <= 3), "degree %d not in 1..3",
                prog->degree);
    KLR_REQUIRE(prog->coef_dtype == KLR_F32 || prog->coef_dtype == KLR_F64, "bad coef_dtype");
    KLR_REQUIRE(out_dtype == KLR_F32 || out_dtype == KLR_F64, "bad out_dtype");
    KLR_REQUIRE(n_cfg >= 1 && n_cfg <= kMaxCfg, "n_cfg %d not in 1..%d", n_cfg, kMaxCfg);
    KLR_REQUIRE(q->n_queries >= 0, "n_queries < 0");
    KLR_REQUIRE(hw->n_sm > 0 && hw->max_warps_per_sm > 0 && hw->regs_per_sm > 0 &&
                hw->smem_per_sm >= 0 && hw->max_blocks_per_sm > 0 && hw->max_threads_per_block > 0,
                "bad hardware limits");
    KLR_REQUIRE(hw->mem_latency > 0 && hw->mem_bandwidth > 0 && hw->clock_hz > 0 &&
                hw->departure_delay_coal > 0 && hw->departure_delay_uncoal > 0,
                "bad hardware timing parameters");
    for (int i = 0; i < 8; ++i)
        KLR_REQUIRE(std::isfinite(prog->metric_lo[i]) && std::isfinite(prog->metric_scale[i]),
                    "non-finite metric map");
    if (prog->n_kernels > 0 && q->n_queries > 0)
        KLR_REQUIRE(prog->coef && prog->regs && prog->smem && cfg && q->q_offsets && q->q_N,
                    "NULL device array");
    Basis basis;
    KLR_REQUIRE(make_basis(prog->n_vars, prog->degree, prog->var_degree, &basis), "no basis");
    memset(&P, 0, sizeof(P));
    P.n_kernels = prog->n_kernels;
    P.n_vars = prog->n_vars;
    P.dims = prog->n_vars - 1;
    // the specialised polynomials in N have the basis's largest power of N
    P.degree = box ? basis.d_n : prog->degree;
    P.m = basis.m;
    P.u = 2 * basis.m;
    P.n_scale_log2 = prog->n_scale_log2;
    P.b_scale_log2 = prog->b_scale_log2;
    P.coef_f64 = prog->coef_dtype == KLR_F64;
    P.coef = prog->coef;
    P.regs = prog->regs;
    P.smem = prog->smem;
    for (int i = 0; i < 8; ++i) { P.lo[i] = prog->metric_lo[i]; P.sc[i] = prog->metric_scale[i]; }
    P.n_sm = hw->n_sm;
    P.W_max = hw->max_warps_per_sm;
    P.R_max = hw->regs_per_sm;
    P.Z_max = hw->smem_per_sm;
    P.B_max = hw->max_blocks_per_sm;
    P.T_max = hw->max_threads_per_block;
    P.mem_ld = hw->mem_latency;
    P.bw = hw->mem_bandwidth;
    P.freq = hw->clock_hz;
    P.dep_c = hw->departure_delay_coal;
    P.dep_u = hw->departure_delay_uncoal;
    P.n_cfg = n_cfg;
    P.cfg = cfg;
    P.q_off = q->q_offsets;
    P.q_N = q->q_N;
    P.n_q = q->n_queries;
    for (int t = 0; t < basis.m; ++t)
        for (int v = 0; v < kMaxVars; ++v) P.exps[t][v] = basis.exps[t][v];
    (void)c;
    return KLR_OK;
}

size_t eval_smem_bytes(const EvalParams& P, size_t tsz) {
    const int NC = 2 * (P.degree + 1);
    size_t b = tsz * (8 * (size_t)P.u + (size_t)P.n_cfg * 8 * NC +
                      (tsz == 4 ? (size_t)P.n_cfg * P.m : 0));
    b = (b + 15) & ~(size_t)15;
    return b + (sizeof(CfgInfo) + sizeof(float)) * (size_t)P.n_cfg;
}

template <typename T, int D>
klr_status launch_eval_t(Context* c, EvalParams& P, size_t smem, int threads, cudaStream_t stream) {
    auto k = eval_kernel<T, D>;
    int per_sm = 0;
    KLR_CHECK_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    KLR_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem));
    const int grid = (int)std::min<int64_t>(P.n_kernels, (int64_t)c->n_sm * std::max(per_sm, 1));
    k<<<grid, threads, smem, stream>>>(P);
    KLR_CHECK_CUDA(cudaGetLastError());
    return KLR_OK;
}

// Problem class of an evaluation for the autotuner: basis, precision, mode,
// |F| and log2 buckets of the queries per kernel and of the kernel count.
uint64_t eval_tune_key(const EvalParams& P, bool f64) {
    const int64_t per_kernel = P.n_kernels ? (P.n_q + P.n_kernels - 1) / P.n_kernels : 1;
    const int mode = P.table ? 1 : (P.cand ? 2 : 0);
    return tune_key(TUNE_EVAL, {P.n_vars, P.degree, f64, mode, P.n_cfg,
                                log2_bucket(per_kernel), log2_bucket(P.n_kernels)});
}

klr_status launch_eval(Context* c, EvalParams& P, bool f64, cudaStream_t stream) {
    const size_t smem = eval_smem_bytes(P, f64 ? 8 : 4);
    if (smem > c->smem_optin) {
        set_error("evaluator needs %zu bytes of shared memory", smem);
        return KLR_ENOTSUP;
    }
    // threads per block: the autotuned choice (32 << choice), else enough for
    // the queries (candidate mode: query-candidate pairs) of a typical kernel,
    // in whole warps
    int64_t per_kernel = P.n_kernels ? (P.n_q + P.n_kernels - 1) / P.n_kernels : 1;
    if (P.cand) per_kernel *= P.kc;
    int threads = 32;
    const int cap = P.cand ? 128 : 256;   // candidate mode: more blocks per SM
    while (threads < cap && threads < per_kernel) threads <<= 1;
    const int32_t choice = tune_choice(c, eval_tune_key(P, f64), -1);
    if (choice >= 0) threads = 32 << std::min(3, (int)choice);
    switch (P.degree * 2 + (f64 ? 1 : 0)) {
        case 2: return launch_eval_t<float, 1>(c, P, smem, threads, stream);
        case 3: return launch_eval_t<double, 1>(c, P, smem, threads, stream);
        case 4: return launch_eval_t<float, 2>(c, P, smem, threads, stream);
        case 5: return launch_eval_t<double, 2>(c, P, smem, threads, stream);
        case 6: return launch_eval_t<float, 3>(c, P, smem, threads, stream);
        default: return launch_eval_t<double, 3>(c, P, smem, threads, stream);
    }
}


// Section IV, step 5's refinement from a cycles table: one warp per kernel
// (the kernel's warps per SM for every shape staged once), one lane per query.
constexpr int kRefineWarps = 4;
__global__ void __launch_bounds__(32 * kRefineWarps)
refine_kernel(const __grid_constant__ EvalParams P, const float* __restrict__ table, double eps) {
    __shared__ int warps_s[kRefineWarps][kMaxCfg];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int* W = warps_s[wib];
    for (int64_t k = (int64_t)blockIdx.x * kRefineWarps + wib; k < P.n_kernels;
         k += (int64_t)gridDim.x * kRefineWarps) {
        const int R = P.regs[k], Z = P.smem[k];
        for (int c = lane; c < P.n_cfg; c += 32) {
            const long long T = (long long)P.cfg[3 * c] * P.cfg[3 * c + 1] * P.cfg[3 * c + 2];
            int B = active_blocks(T, R, Z, P);
            if (T > P.T_max) B = 0;
            W[c] = (int)min((long long)B * T / 32, (long long)P.W_max);
        }
        __syncwarp();
        for (int64_t q = P.q_off[k] + lane; q < P.q_off[k + 1]; q += 32) {
            const float* row = table + q * P.n_cfg;
            float lo = INFINITY;
            int first = -1;
            for (int c = 0; c < P.n_cfg; ++c)
                if (row[c] < lo) { lo = row[c]; first = c; }
            int best = first, st = 0;
            if (first < 0) {
                st = KLR_Q_NONE_FEASIBLE;
            } else {
                const double thr = (double)lo * (1.0 + eps);
                for (int c = 0; c < P.n_cfg; ++c) {
                    const float v = row[c];
                    if (!((double)v <= thr) || c == best) continue;
                    if (W[c] > W[best] || (W[c] == W[best] && v < row[best])) best = c;
                }
                if (best != first) st = KLR_Q_REFINED;
            }
            P.best[q] = best;
            reinterpret_cast<float*>(P.best_cycles)[q] = best >= 0 ? row[best] : INFINITY;
            if (P.q_status) P.q_status[q] = st;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Runtime history (Section III-B: the tool keeps a history of its decisions
// so that later launches of the same kernel at the same size get the result
// at once): an open-addressing hash table on the device from (kernel, N) to
// the argmin outputs.
// ---------------------------------------------------------------------------
constexpr uint64_t kEmptyKey = ~0ull;
constexpr int kMaxProbe = 64;

struct History {
    int device;
    int64_t cap;                 // slots, a power of two
    unsigned long long* keys;    // kernel << 40 | N, or kEmptyKey
    int4* vals;                  // best, cycles bits, margin bits, status
};

// splitmix64 finaliser (Steele, Lea and Flood)
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

// key of a query, or kEmptyKey when it cannot be stored (N >= 2^40)
__device__ __forceinline__ uint64_t history_key(int32_t k, long long N) {
    if (N < 0 || N >= (1LL << 40) || k < 0 || k >= (1 << 23)) return kEmptyKey;
    return ((uint64_t)k << 40) | (uint64_t)N;
}

// look every query up (one warp per kernel over its queries); hits write
// their outputs and are marked done
__global__ void history_lookup_kernel(const __grid_constant__ EvalParams P, History h,
                                      uint8_t* __restrict__ done) {
    const int lane = threadIdx.x & 31;
    for (int64_t wk = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; wk < P.n_kernels;
         wk += ((int64_t)gridDim.x * blockDim.x) >> 5)
    for (int64_t q = P.q_off[wk] + lane; q < P.q_off[wk + 1]; q += 32) {
        const long long N = P.q_N[q];
        const uint64_t key = history_key((int32_t)wk, N);
        uint8_t hit = 0;
        if (key != kEmptyKey) {
            uint64_t i = mix64(key) & (uint64_t)(h.cap - 1);
            for (int p = 0; p < kMaxProbe; ++p, i = (i + 1) & (uint64_t)(h.cap - 1)) {
                const uint64_t kk = h.keys[i];
                if (kk == kEmptyKey) break;
                if (kk == key) {
                    const int4 v = h.vals[i];
                    P.best[q] = v.x;
                    reinterpret_cast<float*>(P.best_cycles)[q] = __int_as_float(v.y);
                    if (P.margin) P.margin[q] = __int_as_float(v.z);
                    if (P.q_status) P.q_status[q] = v.w | KLR_Q_HISTORY;
                    write_launch(P, q, N, v.x);
                    hit = 1;
                    break;
                }
            }
        }
        done[q] = hit;
    }
}

// record the evaluated queries (one warp per kernel; a full probe window
// leaves a query out)
__global__ void history_insert_kernel(const __grid_constant__ EvalParams P, History h,
                                      const uint8_t* __restrict__ done) {
    const int lane = threadIdx.x & 31;
    for (int64_t wk = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; wk < P.n_kernels;
         wk += ((int64_t)gridDim.x * blockDim.x) >> 5)
    for (int64_t q = P.q_off[wk] + lane; q < P.q_off[wk + 1]; q += 32) {
        if (done[q]) continue;
        const uint64_t key = history_key((int32_t)wk, P.q_N[q]);
        if (key == kEmptyKey) continue;
        const int32_t b = P.best[q];
        int4 v;
        v.x = b;
        v.y = __float_as_int(reinterpret_cast<const float*>(P.best_cycles)[q]);
        v.z = __float_as_int(P.margin ? P.margin[q] : 0.f);
        v.w = P.q_status ? P.q_status[q] : (b < 0 ? KLR_Q_NONE_FEASIBLE : 0);
        uint64_t i = mix64(key) & (uint64_t)(h.cap - 1);
        for (int p = 0; p < kMaxProbe; ++p, i = (i + 1) & (uint64_t)(h.cap - 1)) {
            const unsigned long long prev = atomicCAS(h.keys + i, kEmptyKey, key);
            if (prev == kEmptyKey) { h.vals[i] = v; break; }
            if (prev == key) break;      // recorded by another query with the same key
        }
    }
}

// the FP32 decision of every query among its candidates
klr_status launch_candidates(Context* c, EvalParams& P, cudaStream_t stream) {
    const int k = P.kc;
    if (k <= 32 && (k & (k - 1)) == 0) {
        // one warp per kernel
        // as many shapes specialised per kernel as keep three blocks per SM
        // (every shape when they fit), at least 48 (or every shape)
        const int NC = 2 * (P.degree + 1);
        auto smem_for = [&](int sl) {
            return align16(4 * (size_t)P.n_cfg * P.m) +
                   kRerankWarps * rerank_warp_bytes(P.u, P.n_cfg, NC, sl);
        };
        int slots = std::min(P.n_cfg, 48);
        for (int sl = std::min(P.n_cfg, 256); sl > slots; sl -= 4)
            if (3 * (smem_for(sl) + 1024) <= (size_t)c->smem_optin + 1024) { slots = sl; break; }
        P.slots = slots;
        const size_t smem = smem_for(slots);
        if (smem <= c->smem_optin) {
            auto go = [&](auto kern) -> klr_status {
                int per_sm = 0;
                KLR_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    (int)smem));
                KLR_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern,
                                                                             32 * kRerankWarps, smem));
                const int grid = (int)std::min<int64_t>(
                    ((int64_t)P.n_kernels + kRerankWarps - 1) / kRerankWarps,
                    (int64_t)c->n_sm * std::max(per_sm, 1));
                kern<<<grid, 32 * kRerankWarps, smem, stream>>>(P);
                KLR_CHECK_CUDA(cudaGetLastError());
                return KLR_OK;
            };
            if (P.degree == 1) return go(rerank_kernel<1>);
            if (P.degree == 2) return go(rerank_kernel<2>);
            return go(rerank_kernel<3>);
        }
    }
    return launch_eval(c, P, false, stream);
}

}  // namespace

size_t fit_workspace_bytes(int64_t n_fits, int n_mom);

// A context's scratch serves one call at a time: the larger of the fit's
// moment sums (sized here for fits of total degree <= 2 in up to four
// variables) and the argmin's tie records.
size_t workspace_bytes(int64_t max_fits, int64_t max_queries) {
    // tie records, then the history mode's per-query mask
    const size_t ties = 256 + sizeof(TieRecord) * (size_t)tie_capacity(max_queries) +
                        (((size_t)max_queries + 255) & ~(size_t)255);
    return std::max(ties, fit_workspace_bytes(max_fits, n_monomials(4, 4)));
}

}  // namespace klr

using namespace klr;

extern "C" {

size_t klr_workspace_bytes(int64_t max_fits, int64_t max_queries) {
    return workspace_bytes(max_fits, max_queries);
}

klr_status klr_eval(klr_ctx* ctx, const klr_program* prog, const klr_hw* hw, const int32_t* cfg,
                    int n_cfg, const klr_queries* q, void* cycles_out, int32_t out_dtype,
                    void* stream_) {
    KLR_REQUIRE(ctx, "klr_eval: NULL context");
    Context* c = reinterpret_cast<Context*>(ctx);
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    EvalParams P;
    klr_status st = prepare(c, prog, hw, cfg, n_cfg, q, out_dtype, P);
    if (st != KLR_OK) return st;
    if (P.n_q == 0 || P.n_kernels == 0) return KLR_OK;
    KLR_REQUIRE(cycles_out, "klr_eval: NULL cycles_out");
    KLR_CHECK_CUDA(cudaSetDevice(c->device));
    P.table = 1;
    P.cycles = cycles_out;
    return launch_eval(c, P, out_dtype == KLR_F64, stream);
}

klr_status klr_argmin(klr_ctx* ctx, const klr_program* prog, const klr_hw* hw,
                      const int32_t* cfg, int n_cfg, const klr_queries* q, int32_t* best_idx,
                      void* best_cycles, int32_t out_dtype, float* margin, int32_t* q_status,
                      int32_t* launch_out, void* stream_) {
    KLR_REQUIRE(ctx, "klr_argmin: NULL context");
    Context* c = reinterpret_cast<Context*>(ctx);
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    EvalParams P;
    klr_status st = prepare(c, prog, hw, cfg, n_cfg, q, out_dtype, P);
    if (st != KLR_OK) return st;
    if (P.n_q == 0 || P.n_kernels == 0) return KLR_OK;
    KLR_REQUIRE(best_idx && best_cycles, "klr_argmin: NULL best_idx or best_cycles");
    KLR_CHECK_CUDA(cudaSetDevice(c->device));
    P.table = 0;
    P.best = best_idx;
    P.best_cycles = best_cycles;
    P.margin = margin;
    P.q_status = q_status;
    P.launch = launch_out;
    const bool f64 = out_dtype == KLR_F64;
    if (!f64) {
        st = ensure_workspace(c, workspace_bytes(0, P.n_q), stream);
        if (st != KLR_OK) return st;
        P.tie_count = reinterpret_cast<int*>(c->ws);
        P.ties = reinterpret_cast<TieRecord*>(reinterpret_cast<char*>(c->ws) + 256);
        P.tie_cap = tie_capacity(P.n_q);
        KLR_CHECK_CUDA(cudaMemsetAsync(P.tie_count, 0, sizeof(int), stream));
    }
    if (f64 && P.n_q <= kLatencyMaxQueries && latency_smem_bytes(P) <= c->smem_optin) {
        // a few FP64 queries: one block each, spread over the SMs (its tables
        // add the block-shape monomials; without room for them, the sweep)
        const size_t smem = latency_smem_bytes(P);
        auto kern = P.degree == 1 ? eval_query_block_kernel<1>
                  : P.degree == 2 ? eval_query_block_kernel<2> : eval_query_block_kernel<3>;
        KLR_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem));
        kern<<<(unsigned)P.n_q, kLatencyThreads, smem, stream>>>(P);
        KLR_CHECK_CUDA(cudaGetLastError());
        return KLR_OK;
    }
    st = launch_eval(c, P, f64, stream);
    if (st != KLR_OK || f64) return st;
    return launch_ties(c, P, stream);
}

klr_status klr_argmin_candidates(klr_ctx* ctx, const klr_program* prog, const klr_hw* hw,
                                 const int32_t* cfg, int n_cfg, const klr_queries* q,
                                 const int32_t* cand, int k, int32_t* best_idx,
                                 float* best_cycles, int32_t* q_status, void* stream_) {
    KLR_REQUIRE(ctx, "klr_argmin_candidates: NULL context");
    Context* c = reinterpret_cast<Context*>(ctx);
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    EvalParams P;
    klr_status st = prepare(c, prog, hw, cfg, n_cfg, q, KLR_F32, P);
    if (st != KLR_OK) return st;
    KLR_REQUIRE(k >= 1 && k <= 256, "klr_argmin_candidates: k %d not in 1..256", k);
    if (P.n_q == 0 || P.n_kernels == 0) return KLR_OK;
    KLR_REQUIRE(cand && best_idx && best_cycles, "klr_argmin_candidates: NULL array");
    KLR_CHECK_CUDA(cudaSetDevice(c->device));
    // the specialised evaluator in candidate mode: per kernel, only the
    // proposed shapes are specialised and evaluated
    P.table = 0;
    P.best = best_idx;
    P.best_cycles = best_cycles;
    P.q_status = q_status;
    P.cand = cand;
    P.kc = k;
    // near-ties among the candidates are re-decided in FP64, as in the sweep
    st = ensure_workspace(c, workspace_bytes(0, P.n_q), stream);
    if (st != KLR_OK) return st;
    P.tie_count = reinterpret_cast<int*>(c->ws);
    P.ties = reinterpret_cast<TieRecord*>(reinterpret_cast<char*>(c->ws) + 256);
    P.tie_cap = tie_capacity(P.n_q);
    KLR_CHECK_CUDA(cudaMemsetAsync(P.tie_count, 0, sizeof(int), stream));
    st = launch_candidates(c, P, stream);
    if (st != KLR_OK) return st;
    return launch_ties(c, P, stream);
}


klr_status klr_argmin_noalloc(const klr_program* prog, const klr_hw* hw, const int32_t* cfg,
                              int n_cfg, const klr_queries* q, int32_t* best_idx,
                              float* best_cycles, float* margin, int32_t* q_status,
                              int32_t* launch_out, void* stream_) {
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    // a context on the stack: device facts only, no scratch
    Context c;
    KLR_CHECK_CUDA(cudaGetDevice(&c.device));
    int v = 0;
    KLR_CHECK_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, c.device));
    c.n_sm = v;
    KLR_CHECK_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, c.device));
    c.smem_optin = (size_t)v;
    EvalParams P;
    klr_status st = prepare(&c, prog, hw, cfg, n_cfg, q, KLR_F32, P);
    if (st != KLR_OK) return st;
    KLR_REQUIRE(P.n_q <= KLR_ARGMIN_NOALLOC_MAX_QUERIES,
                "klr_argmin_noalloc: %lld queries exceed the maximum of %d",
                (long long)P.n_q, KLR_ARGMIN_NOALLOC_MAX_QUERIES);
    if (P.n_q == 0 || P.n_kernels == 0) return KLR_OK;
    KLR_REQUIRE(best_idx && best_cycles, "klr_argmin_noalloc: NULL best_idx or best_cycles");
    void* scratch = nullptr;
    st = noalloc_scratch(c.device, &scratch);
    if (st != KLR_OK) return st;
    P.table = 0;
    P.best = best_idx;
    P.best_cycles = best_cycles;
    P.margin = margin;
    P.q_status = q_status;
    P.launch = launch_out;
    P.tie_count = reinterpret_cast<int*>(scratch);
    P.ties = reinterpret_cast<TieRecord*>(reinterpret_cast<char*>(scratch) + kNoallocHeader);
    P.tie_cap = KLR_ARGMIN_NOALLOC_TIE_RECORDS;
    // the array keeps the previous call's contents: the tie counter starts at zero
    KLR_CHECK_CUDA(cudaMemsetAsync(P.tie_count, 0, sizeof(int), stream));
    st = launch_eval(&c, P, false, stream);
    if (st != KLR_OK) return st;
    {
        const klr_status ts = launch_ties(&c, P, stream);
        if (ts != KLR_OK) return ts;
    }
    KLR_CHECK_CUDA(cudaGetLastError());
    return KLR_OK;
}

klr_status klr_autotune_argmin(klr_ctx* ctx, const klr_program* prog, const klr_hw* hw,
                               const int32_t* cfg, int n_cfg, const klr_queries* q,
                               int32_t* best_idx, void* best_cycles, int32_t out_dtype,
                               float* margin, int32_t* q_status, int32_t* launch_out,
                               int32_t* choice_out, float* ms_out, void* stream_) {
    KLR_REQUIRE(ctx, "klr_autotune_argmin: NULL context");
    Context* c = reinterpret_cast<Context*>(ctx);
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    auto run = [&]() -> klr_status {
        return klr_argmin(ctx, prog, hw, cfg, n_cfg, q, best_idx, best_cycles, out_dtype, margin,
                          q_status, launch_out, stream_);
    };
    EvalParams P;
    klr_status st = prepare(c, prog, hw, cfg, n_cfg, q, out_dtype, P);
    if (st != KLR_OK) return st;
    if (P.n_q == 0 || P.n_kernels == 0) return run();
    P.table = 0;
    const int32_t cand[4] = {0, 1, 2, 3};           // 32, 64, 128, 256 threads per block
    return tune_candidates(c, eval_tune_key(P, out_dtype == KLR_F64), stream, cand, 4, 3, run,
                           choice_out, ms_out);
}

klr_status klr_history_create(klr_ctx* ctx, int32_t capacity_log2, klr_history** out) {
    KLR_REQUIRE(ctx && out, "klr_history_create: NULL context or output");
    KLR_REQUIRE(capacity_log2 >= 10 && capacity_log2 <= 30,
                "klr_history_create: capacity_log2 %d not in 10..30", capacity_log2);
    Context* c = reinterpret_cast<Context*>(ctx);
    KLR_CHECK_CUDA(cudaSetDevice(c->device));
    History* h = new History();
    h->device = c->device;
    h->cap = (int64_t)1 << capacity_log2;
    if (cudaMalloc(&h->keys, sizeof(unsigned long long) * h->cap) != cudaSuccess ||
        cudaMalloc(&h->vals, sizeof(int4) * h->cap) != cudaSuccess) {
        cudaGetLastError();
        if (h->keys) cudaFree(h->keys);
        delete h;
        set_error("klr_history_create: cudaMalloc of %lld slots failed", (long long)(1LL << capacity_log2));
        return KLR_ENOMEM;
    }
    KLR_CHECK_CUDA(cudaMemset(h->keys, 0xFF, sizeof(unsigned long long) * h->cap));
    KLR_CHECK_CUDA(cudaDeviceSynchronize());
    *out = reinterpret_cast<klr_history*>(h);
    return KLR_OK;
}

klr_status klr_history_destroy(klr_history* hist) {
    if (!hist) return KLR_OK;
    History* h = reinterpret_cast<History*>(hist);
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    cudaFree(h->keys);
    cudaFree(h->vals);
    delete h;
    return KLR_OK;
}

klr_status klr_history_clear(klr_history* hist, void* stream_) {
    KLR_REQUIRE(hist, "klr_history_clear: NULL history");
    History* h = reinterpret_cast<History*>(hist);
    KLR_CHECK_CUDA(cudaSetDevice(h->device));
    KLR_CHECK_CUDA(cudaMemsetAsync(h->keys, 0xFF, sizeof(unsigned long long) * h->cap,
                                   reinterpret_cast<cudaStream_t>(stream_)));
    return KLR_OK;
}

klr_status klr_argmin_history(klr_ctx* ctx, klr_history* hist, const klr_program* prog,
                              const klr_hw* hw, const int32_t* cfg, int n_cfg,
                              const klr_queries* q, int32_t* best_idx, float* best_cycles,
                              float* margin, int32_t* q_status, int32_t* launch_out,
                              void* stream_) {
    KLR_REQUIRE(ctx && hist, "klr_argmin_history: NULL context or history");
    Context* c = reinterpret_cast<Context*>(ctx);
    History* h = reinterpret_cast<History*>(hist);
    KLR_REQUIRE(h->device == c->device, "klr_argmin_history: history of another device");
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    EvalParams P;
    klr_status st = prepare(c, prog, hw, cfg, n_cfg, q, KLR_F32, P);
    if (st != KLR_OK) return st;
    if (P.n_q == 0 || P.n_kernels == 0) return KLR_OK;
    KLR_REQUIRE(best_idx && best_cycles, "klr_argmin_history: NULL best_idx or best_cycles");
    KLR_CHECK_CUDA(cudaSetDevice(c->device));
    P.table = 0;
    P.best = best_idx;
    P.best_cycles = best_cycles;
    P.margin = margin;
    P.q_status = q_status;
    P.launch = launch_out;
    st = ensure_workspace(c, workspace_bytes(0, P.n_q), stream);
    if (st != KLR_OK) return st;
    P.tie_count = reinterpret_cast<int*>(c->ws);
    P.ties = reinterpret_cast<TieRecord*>(reinterpret_cast<char*>(c->ws) + 256);
    P.tie_cap = tie_capacity(P.n_q);
    uint8_t* done = reinterpret_cast<uint8_t*>(c->ws) + 256 + sizeof(TieRecord) * (size_t)P.tie_cap;
    KLR_CHECK_CUDA(cudaMemsetAsync(P.tie_count, 0, sizeof(int), stream));
    // one warp per kernel
    const int grid = (int)std::min<int64_t>(((int64_t)P.n_kernels * 32 + 255) / 256,
                                            (int64_t)c->n_sm * 16);
    history_lookup_kernel<<<grid, 256, 0, stream>>>(P, *h, done);
    KLR_CHECK_CUDA(cudaGetLastError());
    P.done = done;
    if ((st = launch_eval(c, P, false, stream)) != KLR_OK) return st;
    {
        const klr_status ts = launch_ties(c, P, stream);
        if (ts != KLR_OK) return ts;
    }
    KLR_CHECK_CUDA(cudaGetLastError());
    history_insert_kernel<<<grid, 256, 0, stream>>>(P, *h, done);
    KLR_CHECK_CUDA(cudaGetLastError());
    return KLR_OK;
}

klr_status klr_argmin_refined(klr_ctx* ctx, const klr_program* prog, const klr_hw* hw,
                              const int32_t* cfg, int n_cfg, const klr_queries* q,
                              const float* cycles_table, double eps, int32_t* best_idx,
                              float* best_cycles, int32_t* q_status, void* stream_) {
    KLR_REQUIRE(ctx, "klr_argmin_refined: NULL context");
    KLR_REQUIRE(std::isfinite(eps) && eps >= 0.0, "klr_argmin_refined: eps must be >= 0");
    Context* c = reinterpret_cast<Context*>(ctx);
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    EvalParams P;
    klr_status st = prepare(c, prog, hw, cfg, n_cfg, q, KLR_F32, P);
    if (st != KLR_OK) return st;
    if (P.n_q == 0 || P.n_kernels == 0) return KLR_OK;
    KLR_REQUIRE(cycles_table && best_idx && best_cycles, "klr_argmin_refined: NULL array");
    KLR_CHECK_CUDA(cudaSetDevice(c->device));
    P.best = best_idx;
    P.best_cycles = best_cycles;
    P.q_status = q_status;
    const int grid = (int)std::min<int64_t>((P.n_kernels + kRefineWarps - 1) / kRefineWarps,
                                            (int64_t)c->n_sm * 16);
    refine_kernel<<<grid, 32 * kRefineWarps, 0, stream>>>(P, cycles_table, eps);
    KLR_CHECK_CUDA(cudaGetLastError());
    return KLR_OK;
}

}  // extern "C"
